// gmg_residual64_noalloc: the FP64 true-residual reduction of the fine level,
// for callers that cannot allocate device memory.
//
// Why it exists: gmg_residual64 needs a handle, and gmg_setup allocates the
// handle's buffers with cudaMalloc.  Some callers cannot do that -- code that
// runs inside a framework which owns every device allocation through its own
// pool, a plugin that must not grow the process's device footprint behind its
// host's back, or a check that must still work when the device is out of free
// memory.  This entry point takes the moduli, the node mask and the vectors
// from the caller and keeps its only scratch (the element stiffness and the
// per-block partial sums) in the file-scope device array below.
//
// The array lives in every GPU that loads this library until the process
// exits.  All calls share it: two calls whose kernels overlap on the GPU (for
// example on two streams) race on it.  Each call rewrites every word it reads,
// so nothing has to be cleared between calls.
#include <cmath>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace gmg {
namespace {

constexpr int kNoallocMaxBlocks = 65536;                 // partial sums: 512 KiB
constexpr int kNoallocWords = 576 + 2 + kNoallocMaxBlocks;  // K_e, two results, partials

static __device__ __align__(256) double g_noalloc_scratch[kNoallocWords];

// Same tile geometry as the fine-level kernels.
constexpr int TX = 32, TY = 4, TZ = 2;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
constexpr int EX = TX + 1, EY = TY + 1, EZ = TZ + 1;
constexpr int NT = TX * TY * TZ;

__device__ __forceinline__ bool fixed_bit(uint8_t m, int c) { return (m >> c) & 1; }

__device__ __forceinline__ double sum_block(double v, int tid) {
    __shared__ double part[NT / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) part[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < NT / 32; ++w) s += part[w];
    return s;
}

// K_e of the unit hex8 element (2x2x2 Gauss rule, tensor form of the isotropic
// energy) into scratch[0..576).
__global__ void k_na_ke(double nu, double* Ke) {
    const int I = threadIdx.x;
    if (I >= 576) return;
    const int row = I / 24, col = I % 24;
    const int a = row / 3, c = row % 3, b = col / 3, d = col % 3;
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = 1.0 / (2.0 * (1.0 + nu));
    const double h = 0.5 / sqrt(3.0), pts[2] = {0.5 - h, 0.5 + h};
    double s = 0.0;
    for (int q = 0; q < 8; ++q) {
        const double x = pts[q & 1], y = pts[(q >> 1) & 1], z = pts[q >> 2];
        double ga[3], gb[3];
        {
            const double fx = ldx(a) ? x : 1 - x, fy = ldy(a) ? y : 1 - y, fz = ldz(a) ? z : 1 - z;
            ga[0] = (ldx(a) ? 1 : -1) * fy * fz; ga[1] = fx * (ldy(a) ? 1 : -1) * fz; ga[2] = fx * fy * (ldz(a) ? 1 : -1);
        }
        {
            const double fx = ldx(b) ? x : 1 - x, fy = ldy(b) ? y : 1 - y, fz = ldz(b) ? z : 1 - z;
            gb[0] = (ldx(b) ? 1 : -1) * fy * fz; gb[1] = fx * (ldy(b) ? 1 : -1) * fz; gb[2] = fx * fy * (ldz(b) ? 1 : -1);
        }
        double v = lam * ga[c] * gb[d] + mu * ga[d] * gb[c];
        if (c == d) v += mu * (ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2]);
        s += 0.125 * v;
    }
    Ke[I] = s;
}

// r = f - K u on the fine level (FP64), one partial ||r_free||^2 per block.
__global__ void __launch_bounds__(NT) k_na_resid64(int nx, int ny, int nz, const double* E, const uint8_t* mask,
                                                   const double* f, const double* uvec, double* r64,
                                                   const double* Ke, double* partial) {
    __shared__ double su[HZ][HY][HX * 3];
    __shared__ double sE[EZ][EY][EX];
    __shared__ double sK[576];
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int tid = tx + TX * (ty + TY * tz);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const int NX = nx + 1, NY = ny + 1, NZ = nz + 1;
    for (int q = tid; q < 576; q += NT) sK[q] = Ke[q];
    for (int idx = tid; idx < HZ * HY * HX * 3; idx += NT) {
        const int c3 = idx % (HX * 3), row = idx / (HX * 3);
        const int yy = row % HY, zz = row / HY;
        const int gx = x0 - 1 + c3 / 3, comp = c3 % 3, gy = y0 - 1 + yy, gz = z0 - 1 + zz;
        double v = 0.0;
        if (gx >= 0 && gx < NX && gy >= 0 && gy < NY && gz >= 0 && gz < NZ) {
            const long long node = gx + (long long)NX * (gy + (long long)NY * gz);
            if (!fixed_bit(mask[node], comp)) v = uvec[3 * node + comp];
        }
        su[zz][yy][c3] = v;
    }
    for (int idx = tid; idx < EZ * EY * EX; idx += NT) {
        const int ex = idx % EX, ey = (idx / EX) % EY, ez = idx / (EX * EY);
        const int gx = x0 - 1 + ex, gy = y0 - 1 + ey, gz = z0 - 1 + ez;
        sE[ez][ey][ex] = (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
                             ? E[gx + (long long)nx * (gy + (long long)ny * gz)] : 0.0;
    }
    __syncthreads();
    const int i = x0 + tx, j = y0 + ty, k = z0 + tz;
    double rr = 0.0;
    if (i < NX && j < NY && k < NZ) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int ea = 0; ea < 8; ++ea) {
            const double Ee = sE[tz + 1 - ldz(ea)][ty + 1 - ldy(ea)][tx + 1 - ldx(ea)];
            for (int eb = 0; eb < 8; ++eb) {
                const int ox = ldx(eb) - ldx(ea) + 1, oy = ldy(eb) - ldy(ea) + 1, oz = ldz(eb) - ldz(ea) + 1;
                for (int d = 0; d < 3; ++d) {
                    const double ud = Ee * su[tz + oz][ty + oy][(tx + ox) * 3 + d];
                    for (int c = 0; c < 3; ++c) acc[c] = fma(sK[(3 * ea + c) * 24 + 3 * eb + d], ud, acc[c]);
                }
            }
        }
        const long long node = i + (long long)NX * (j + (long long)NY * k);
        const uint8_t m = mask[node];
        for (int c = 0; c < 3; ++c) {
            const double v = fixed_bit(m, c) ? 0.0 : f[3 * node + c] - acc[c];
            if (r64) r64[3 * node + c] = v;
            rr += v * v;
        }
    }
    const double s = sum_block(rr, tid);
    if (tid == 0) partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
}

// One partial ||f_free||^2 per block over a fixed grid of blocks.
__global__ void __launch_bounds__(256) k_na_ff(const double* f, const uint8_t* mask, long long nn, double* partial) {
    double s = 0.0;
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < 3 * nn; q += (long long)gridDim.x * 256)
        if (!fixed_bit(mask[q / 3], (int)(q % 3))) s += f[q] * f[q];
    __shared__ double part[8];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += part[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(256) k_na_sum(const double* partial, int n, double* out) {
    __shared__ double part[256];
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += 256) s += partial[q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mu;
double* g_na_ptr[64] = {};

int scratch_for_current_device(double** out, std::string* err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { *err = cudaGetErrorString(e); return GMG_ERR_NO_DEVICE; }
    if (dev < 0 || dev >= 64) { *err = "device ordinal above 63"; return GMG_ERR_NO_DEVICE; }
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e); return GMG_ERR_CUDA; }
        g_na_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_na_ptr[dev];
    return GMG_OK;
}

}  // namespace
}  // namespace gmg

extern "C" int gmg_residual64_noalloc(const gmg_grid* g, const double* E_dev, const uint8_t* mask_dev, double nu,
                                      const double* f_dev, const double* u_dev, double* r_dev, double* rel_out,
                                      void* stream) {
    using namespace gmg;
    if (!g || !E_dev || !mask_dev || !f_dev || !u_dev || !rel_out) {
        set_error_text("gmg_residual64_noalloc: null argument");
        return GMG_ERR_ARG;
    }
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(nu > -1.0 && nu < 0.5)) {
        set_error_text("gmg_residual64_noalloc: element counts must be >= 1 and nu in (-1, 0.5)");
        return GMG_ERR_ARG;
    }
    // Sizes in 64-bit before anything is launched: the node count must keep
    // every DOF index below 2^31 (the limit gmg_setup applies too), and the
    // block grid must fit the static array of partial sums.
    const long long NX = (long long)g->nx + 1, NY = (long long)g->ny + 1, NZ = (long long)g->nz + 1;
    const long long nn = NX * NY * NZ;
    if (nn > (1LL << 31) / 3) {
        set_error_text("gmg_residual64_noalloc: grid too large (" + std::to_string(nn) +
                       " nodes; 3 x nodes must stay below 2^31)");
        return GMG_ERR_ARG;
    }
    const long long gx = (NX + TX - 1) / TX, gy = (NY + TY - 1) / TY, gz = (NZ + TZ - 1) / TZ;
    if (gx < 1 || gy < 1 || gz < 1 || gx * gy * gz > kNoallocMaxBlocks || gy > 65535 || gz > 65535) {
        set_error_text("gmg_residual64_noalloc: the grid needs " + std::to_string(gx * gy * gz) +
                       " partial sums; the static scratch holds at most " + std::to_string(kNoallocMaxBlocks) +
                       " (nodes per block 32x4x2)");
        return GMG_ERR_ARG;
    }
    double* scratch = nullptr;
    std::string err;
    const int rc = scratch_for_current_device(&scratch, &err);
    if (rc != GMG_OK) {
        set_error_text("gmg_residual64_noalloc: " + err);
        return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* Ke = scratch;
    double* res = scratch + 576;
    double* partial = scratch + 578;
    note_launch(5);
    k_na_ke<<<1, 576, 0, s>>>(nu, Ke);
    k_na_resid64<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(TX, TY, TZ), 0, s>>>(
        g->nx, g->ny, g->nz, E_dev, mask_dev, f_dev, u_dev, r_dev, Ke, partial);
    k_na_sum<<<1, 256, 0, s>>>(partial, (int)(gx * gy * gz), res);
    k_na_ff<<<592, 256, 0, s>>>(f_dev, mask_dev, nn, partial);
    k_na_sum<<<1, 256, 0, s>>>(partial, 592, res + 1);
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) {
        set_error_text(std::string("gmg_residual64_noalloc: launch failed: ") + cudaGetErrorString(le));
        return GMG_ERR_CUDA;
    }
    double host[2] = {0.0, 0.0};
    cudaError_t ce = cudaMemcpyAsync(host, res, sizeof host, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        // Faults of the kernels above, and a call made inside a stream capture,
        // surface here.
        set_error_text(std::string("gmg_residual64_noalloc: ") + cudaGetErrorString(ce));
        return GMG_ERR_CUDA;
    }
    // A load with no nonzero free entry has no relative scale: the result is 0
    // when the residual is zero too (u = 0 solves K u = 0) and +inf otherwise.
    if (host[1] == 0.0) {
        *rel_out = host[0] == 0.0 ? 0.0 : HUGE_VAL;
        return GMG_OK;
    }
    *rel_out = sqrt(host[0]) / sqrt(host[1]);
    return GMG_OK;
}
