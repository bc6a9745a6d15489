/*
 * gmg_warmnet.h -- C ABI of the learned warm start for the GMG-PCG solver of
 * gmg.h: a small 3-D convolutional encoder-decoder that maps a cantilever
 * problem (density field, load, clamp) to an initial displacement guess u0,
 * trained on the GPU by this library's own forward and backward kernels.
 *
 * The paper solves every state equation from u0 = 0 (Sec. "Outer Krylov
 * Solver and Convergence Statement": PCG stops on ||f - K u|| / ||f|| < tol
 * from whatever x0 it is given); the network is this library's addition and the
 * cold-start solve stays both the fallback and the measure of its error.
 *
 * Network (4 resolution levels on the vertex grids of the multigrid levels,
 * 16/32/64/64 channels, 3x3x3 kernels, zero padding, leaky ReLU slope 0.1):
 *
 *   layer  cin cout stride                     layer  cin cout stride
 *   0 e0a   12   16   1                        6 d3    64   64   2
 *   1 e0b   16   16   1  -> s0                 7 e3    64   64   1
 *   2 d1    16   32   2                        8 u2   128   64   1  in [up(e3), s2]
 *   3 e1    32   32   1  -> s1                 9 u1    96   32   1  in [up(u2), s1]
 *   4 d2    32   64   2                       10 u0    48   16   1  in [up(u1), s0]
 *   5 e2    64   64   1  -> s2                11 out   16    3   1  (no activation)
 *
 * up = vertex-centred trilinear interpolation; [a, b] = channel concatenation.
 * A stride-2 layer maps the vertex grid of n elements to that of n/2 (output
 * node o reads input nodes 2o-1..2o+1), so nx, ny, nz must be multiples of 8.
 *
 * Conventions:
 *   - fields are channels-last: value (node n, channel c) at [n*C + c], node
 *     n = i + (nx+1)*(j + (ny+1)*k); a batch of B fields of one grid is stored
 *     back to back.  The 3-channel output of one problem is therefore the
 *     solver's DOF vector (3n + c);
 *   - input features (12 channels, gmg_net_features): nodal density (mean over
 *     the adjacent elements), load f / max|f| (3), 1 on nodes with a fixed DOF,
 *     normalised coordinates i/nx, j/ny, k/nz, the resultant load direction
 *     sum(f) / |sum(f)| as a constant field (3; 0 when the resultant vanishes)
 *     and a constant 1 -- the constant fields carry the load direction to nodes
 *     beyond the network's receptive field;
 *   - parameters: one flat FP32 vector, per layer the weights W[cout][27][cin]
 *     (tap t = dx + 3 dy + 9 dz, offset d - 1 per axis) then the cout biases,
 *     layers in the order of the table (gmg_net_num_params() values);
 *   - arithmetic: the convolutions use the weights rounded to bfloat16 (round
 *     to nearest even) with FP32 activations, biases and accumulation; the
 *     gradient is rescaled to global L2 norm <= clip (clip > 0; a non-finite
 *     norm skips the update), then Adam (beta1 0.9, beta2 0.999, eps 1e-8,
 *     bias-corrected) updates FP32 master weights and re-rounds them;
 *   - *_dev pointers are CUDA device memory owned by the caller; the network
 *     owns its parameters, optimiser state and per-shape workspaces;
 *   - status codes are those of gmg.h; gmg_last_error() describes errors;
 *   - work runs on the stream given to gmg_net_create (gmg_warm_start uses the
 *     solver handle's stream) and is asynchronous unless stated.
 */
#ifndef GMG_B300_WARMNET_H
#define GMG_B300_WARMNET_H

#include <stdint.h>

#include "gmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmg_net gmg_net;

#define GMG_NET_IN 12
#define GMG_NET_OUT 3
#define GMG_NET_LAYERS 12

/* Arithmetic of the stride-1 convolutions (gmg_net_set_arith). */
#define GMG_NET_FP32 0   /* FP32 CUDA-core direct convolution (default) */
#define GMG_NET_TF32 1   /* tcgen05 tensor cores, kind::tf32: activations read as TF32, weights exact */

/* Number of FP32 values in the flat parameter vector (767,267). */
long long gmg_net_num_params(void);

/* shape = {cin, cout, stride, has_activation} of layer 0..GMG_NET_LAYERS-1. */
int gmg_net_layer_shape(int layer, int shape[4]);

/* Creates a network with parameters params_dev (device FP32, gmg_net_num_params()
 * values, copied) and zeroed Adam state.  stream: cudaStream_t or NULL. */
int gmg_net_create(gmg_net** net, const float* params_dev, void* stream);

/* Replaces the parameters (device FP32) and resets the Adam state and step count. */
int gmg_net_set_params(gmg_net* net, const float* params_dev);

/* Copies the FP32 master parameters / the (unclipped) gradient of the last
 * gmg_net_train_step into params_dev / grads_dev. */
int gmg_net_get_params(gmg_net* net, float* params_dev);
int gmg_net_get_grads(gmg_net* net, float* grads_dev);

/* Selects the arithmetic of the forward stride-1 convolutions (inference and
 * the forward pass of training; the stride-2 layers and every backward pass
 * stay on the FP32 path).  GMG_NET_TF32 runs them as implicit GEMMs on the
 * tensor cores (tcgen05.mma kind::tf32, FP32 accumulation in TMEM, operands
 * staged by TMA): the activations lose their 13 low mantissa bits inside the
 * product, so outputs differ from GMG_NET_FP32 by ~1e-3 relative.
 * Synchronises the network's stream; captured training graphs are rebuilt
 * on the next step. */
int gmg_net_set_arith(gmg_net* net, int arith);

/* Synchronous check of the sticky error word of the tensor-core kernels
 * (a bounded wait for operands that gave up): GMG_OK or GMG_ERR_CUDA. */
int gmg_net_status(gmg_net* net);

/* g_dev[B][n_nodes][3] = network(x_dev[B][n_nodes][12]) on the grid nx x ny x nz
 * (multiples of 8, each >= 8).  Errors: GMG_ERR_ARG, GMG_ERR_NOMEM, GMG_ERR_CUDA. */
int gmg_net_forward(gmg_net* net, int nx, int ny, int nz, int batch, const float* x_dev, float* g_dev);

/* One training step on a batch of `batch` problems of one grid: the inputs
 * x_dev[b] ([n_nodes][12]) and targets t_dev[b] ([n_nodes][3]) are host arrays
 * of device pointers.  Loss:
 *   ops == NULL: mean over the DOFs of nodes without a fixed DOF (feature
 *     channel 4 < 0.5) of (g - t)^2, summed over the batch before the division;
 *   ops != NULL: ops[b] is a solver handle of problem b (same grid and
 *     Poisson's ratio for the whole batch); the batch mean of the relative
 *     energy-norm error left after the best rescaling of the output,
 *     L_b = min_a ||t_b - a g_b||^2_K / ||t_b||^2_K
 *         = 1 - (t.K g)^2 / ((g.K g)(t.K t))  (g, t on the free DOFs),
 *     K = K_b applied by the handle's matrix-free fine operator (FP32) -- the
 *     quantity gmg_warm_start's rescaling leaves.
 * The gradient goes through every layer (straight through the bf16 rounding
 * of the weights), is clipped to L2 norm clip (clip <= 0: no clipping), then
 * one Adam update with step size lr.  loss_dev (device float, may be NULL)
 * receives the batch loss.  The kernels of a step are captured once per
 * (grid, batch, loss) in a CUDA graph and replayed; the operators' moduli and
 * masks are copied into the step's workspace, so the handles may differ from
 * call to call. */
int gmg_net_train_step(gmg_net* net, int nx, int ny, int nz, int batch, const float* const* x_dev,
                       const float* const* t_dev, gmg_handle* const* ops, float lr, float clip, float* loss_dev);

/* Input features of one problem: rho_dev element densities (device float
 * [nz][ny][nx]), f_dev load (device double[3*n_nodes]), fixed_dev per-DOF flags
 * (device uint8[3*n_nodes], 1 = fixed) -> x_dev (device float[n_nodes][12]).
 * stream: cudaStream_t or NULL. */
int gmg_net_features(int nx, int ny, int nz, const float* rho_dev, const double* f_dev,
                     const uint8_t* fixed_dev, float* x_dev, void* stream);

/* Training target of one problem: t = u / RMS(u) over all 3*n_nodes entries
 * (u device double, t device float; u = 0 gives t = 0). */
int gmg_net_target(int nx, int ny, int nz, const double* u_dev, float* t_dev, void* stream);

/* Warm start for gmg_solve on handle h (same grid, nx, ny, nz multiples of 8):
 * features from rho_dev, f_dev and the handle's Dirichlet mask, one forward
 * pass, fixed DOFs zeroed, then the energy-optimal rescaling
 * u0 = alpha g, alpha = f.g / g.K g (the minimiser of ||u - alpha g||_K over
 * all real alpha, with K applied by gmg_apply, so never farther from u in
 * the energy norm than u0 = 0); g.K g <= 0 or a non-finite product keeps
 * u0 = 0 (the cold start).  u0_dev: device double[3*n_nodes].  alpha_out
 * (host, may be NULL) receives alpha (0 = cold start kept) and makes the call
 * synchronous. */
int gmg_warm_start(gmg_handle* h, gmg_net* net, const float* rho_dev, const double* f_dev, double* u0_dev,
                   double* alpha_out);

/* Frees the network and its workspaces.  NULL is accepted. */
void gmg_net_destroy(gmg_net* net);

#ifdef __cplusplus
}
#endif

#endif /* GMG_B300_WARMNET_H */
