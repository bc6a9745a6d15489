"""Oracle: the learned warm start's 3-D convolutional encoder-decoder (TEST
INFRASTRUCTURE ONLY; FP64).

The paper solves every state equation from a zero initial guess and has no
network; this module states, in plain FP64 numpy, the small U-Net that the CUDA
library trains and runs to produce an initial displacement u0 for PCG
(Sec. "Outer Krylov Solver and Convergence Statement": PCG accepts any x0 and
stops on ||f - K x|| / ||f||).  Every definition below is this project's own
reading, and each one is pinned in ``tests/test_oracle_warmnet.py`` against a
library routine (scipy.ndimage.correlate for the convolution, torch's bfloat16
cast for the rounding), an exact identity (adjoints, stride-2 = subsampled
stride-1, trilinear reproduction, Adam under a constant gradient), or finite
differences of the loss.

Grid and layout.  Level l of the network lives on the vertex grid of
(nx/2^l, ny/2^l, nz/2^l) elements (nx, ny, nz multiples of 8), i.e. the same
nodes as the multigrid levels; a field is an array [Z][Y][X][C] (x fastest,
channels last), so a 3-channel output reshaped to (-1,) is the solver's DOF
vector 3*n + c.

Architecture (4 resolution levels, 16/32/64/64 channels, 3x3x3 kernels):

    e0a  conv s1  12 -> 16  lrelu   level 0          x0   -> a0
    e0b  conv s1  16 -> 16  lrelu   level 0          a0   -> s0
    d1   conv s2  16 -> 32  lrelu   level 0 -> 1     s0   -> b1
    e1   conv s1  32 -> 32  lrelu   level 1          b1   -> s1
    d2   conv s2  32 -> 64  lrelu   level 1 -> 2     s1   -> b2
    e2   conv s1  64 -> 64  lrelu   level 2          b2   -> s2
    d3   conv s2  64 -> 64  lrelu   level 2 -> 3     s2   -> b3
    e3   conv s1  64 -> 64  lrelu   level 3          b3   -> c3
    u2   conv s1 128 -> 64  lrelu   level 2   [up(c3), s2] -> y2
    u1   conv s1  96 -> 32  lrelu   level 1   [up(y2), s1] -> y1
    u0   conv s1  48 -> 16  lrelu   level 0   [up(y1), s0] -> y0
    out  conv s1  16 ->  3  linear  level 0          y0   -> g

* conv (stride s, zero padding): out[o] = b + sum_t W[:, t, :] x[s*o + d_t - 1],
  taps t = dx + 3 dy + 9 dz, d_t = (dx, dy, dz) in {0,1,2}^3; a stride-2 conv
  maps the vertex grid of n elements to that of n/2 (output node o reads input
  nodes 2o-1 .. 2o+1);
* up = vertex-centred trilinear interpolation (even fine node 2i copies coarse
  node i, odd node 2i+1 averages i and i+1, per axis);
* lrelu(z) = z for z > 0, 0.1 z otherwise; its derivative is taken from the
  stored output (1 where y > 0, else 0.1);
* [a, b] = channel concatenation, upsampled part first.

Inputs (12 channels per node): nodal density (mean of the adjacent elements'
rho), the load f / max|f| (3), an indicator of nodes with a fixed DOF, the
normalised coordinates i/nx, j/ny, k/nz, the direction of the resultant load
sum(f) / |sum(f)| as a constant field (3; zero when the resultant vanishes) and
a constant 1.  The constant fields carry the load direction to nodes beyond the
network's receptive field (about 40 nodes), which the local load channels
cannot reach on the larger grids.  Target: the PCG solution divided by
its RMS over all 3N entries.  Two losses: (mse) the mean squared error over the
DOFs of nodes without a fixed DOF; (energy) the relative error in the energy
norm of the sample's own stiffness after the best rescaling of the output,
L_b = min_a ||t_b - a g_b||_K^2 / ||t_b||_K^2 = 1 - (t.K g)^2 / ((g.K g)(t.K t))
(g, t restricted to the free DOFs), averaged over the batch -- exactly the
quantity the warm start's rescaling leaves, measured in the norm in which PCG
measures the error of its initial guess (roughness of the output costs little
in L2 and much in energy).  Optimiser: the gradient is rescaled to global L2 norm at most
``clip`` (when clip > 0), then Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias
corrected) updates FP32 master weights; the network computes with the weights
rounded to bfloat16 (round to nearest even) and FP32 biases.  Warm start: the
masked output g is rescaled by the energy-optimal factor
alpha = f.g / g.K g (minimiser of ||u - alpha g||_K over all real alpha, so
never worse than u0 = 0); g.K g <= 0 or a non-finite value keeps u0 = 0.
"""

from __future__ import annotations

import numpy as np

SLOPE = 0.1
BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8
N_IN, N_OUT = 12, 3

# (name, cin, cout, stride, activation) in parameter order.
LAYERS = [
    ("e0a", 12, 16, 1, True),
    ("e0b", 16, 16, 1, True),
    ("d1", 16, 32, 2, True),
    ("e1", 32, 32, 1, True),
    ("d2", 32, 64, 2, True),
    ("e2", 64, 64, 1, True),
    ("d3", 64, 64, 2, True),
    ("e3", 64, 64, 1, True),
    ("u2", 128, 64, 1, True),
    ("u1", 96, 32, 1, True),
    ("u0", 48, 16, 1, True),
    ("out", 16, 3, 1, False),
]


def layer_shapes():
    """[(cout, 27, cin), ...] in parameter order."""
    return [(co, 27, ci) for _, ci, co, _, _ in LAYERS]


def n_params() -> int:
    return sum(co * 27 * ci + co for _, ci, co, _, _ in LAYERS)


def unpack(theta: np.ndarray) -> dict:
    """Flat parameter vector -> {name: (W [cout][27][cin], b [cout])}; per layer
    the weights come first, then the biases."""
    out, k = {}, 0
    for name, ci, co, _, _ in LAYERS:
        W = theta[k:k + co * 27 * ci].reshape(co, 27, ci)
        k += co * 27 * ci
        b = theta[k:k + co]
        k += co
        out[name] = (W, b)
    assert k == theta.size
    return out


def pack(params: dict) -> np.ndarray:
    return np.concatenate([np.concatenate([params[n][0].reshape(-1), params[n][1]]) for n, *_ in LAYERS])


# ---------------------------------------------------------------- primitives

def bf16_round(x: np.ndarray) -> np.ndarray:
    """Rounds to the nearest bfloat16 (ties to even), returned as float64.
    The value is first rounded to float32, then its low 16 bits are rounded
    away on the bit pattern."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def out_dims(dims, stride: int):
    """Vertex-grid node counts after a conv of the given stride."""
    return tuple(d if stride == 1 else (d - 1) // 2 + 1 for d in dims)


def conv3d(x: np.ndarray, W: np.ndarray, b: np.ndarray, stride: int) -> np.ndarray:
    """x [Z][Y][X][cin] -> out [Zo][Yo][Xo][cout]; zero padding of one node."""
    Z, Y, X, _ = x.shape
    Zo, Yo, Xo = out_dims((Z, Y, X), stride)
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.broadcast_to(b, (Zo, Yo, Xo, b.size)).copy()
    s = stride
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                t = dx + 3 * dy + 9 * dz
                win = xp[dz:dz + s * (Zo - 1) + 1:s, dy:dy + s * (Yo - 1) + 1:s, dx:dx + s * (Xo - 1) + 1:s, :]
                out += win @ W[:, t, :].T
    return out


def conv3d_backward(x: np.ndarray, W: np.ndarray, gout: np.ndarray, stride: int):
    """Adjoint of ``conv3d`` in (x, W, b): returns (gx, gW, gb)."""
    Z, Y, X, _ = x.shape
    Zo, Yo, Xo, _ = gout.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    s = stride
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                t = dx + 3 * dy + 9 * dz
                sl = (slice(dz, dz + s * (Zo - 1) + 1, s), slice(dy, dy + s * (Yo - 1) + 1, s),
                      slice(dx, dx + s * (Xo - 1) + 1, s))
                win = xp[sl]
                gW[:, t, :] = gout.reshape(-1, gout.shape[3]).T @ win.reshape(-1, win.shape[3])
                gxp[sl] += gout @ W[:, t, :]
    gb = gout.reshape(-1, gout.shape[3]).sum(axis=0)
    return gxp[1:-1, 1:-1, 1:-1, :], gW, gb


def interp_1d(nc: int) -> np.ndarray:
    """Dense (2 nc - 1) x nc vertex-centred linear interpolation matrix."""
    P = np.zeros((2 * nc - 1, nc))
    for i in range(nc):
        P[2 * i, i] = 1.0
    for i in range(nc - 1):
        P[2 * i + 1, i] = 0.5
        P[2 * i + 1, i + 1] = 0.5
    return P


def upsample(x: np.ndarray) -> np.ndarray:
    """[Zc][Yc][Xc][C] -> [2Zc-1][2Yc-1][2Xc-1][C], trilinear per axis."""
    Zc, Yc, Xc, _ = x.shape
    y = np.einsum("zk,kyxc->zyxc", interp_1d(Zc), x)
    y = np.einsum("yk,zkxc->zyxc", interp_1d(Yc), y)
    return np.einsum("xk,zykc->zyxc", interp_1d(Xc), y)


def upsample_adjoint(g: np.ndarray) -> np.ndarray:
    Zf, Yf, Xf, _ = g.shape
    y = np.einsum("zk,zyxc->kyxc", interp_1d((Zf + 1) // 2), g)
    y = np.einsum("yk,zyxc->zkxc", interp_1d((Yf + 1) // 2), y)
    return np.einsum("xk,zyxc->zykc", interp_1d((Xf + 1) // 2), y)


def lrelu(z: np.ndarray) -> np.ndarray:
    return np.where(z > 0, z, SLOPE * z)


def lrelu_grad_from_output(y: np.ndarray) -> np.ndarray:
    return np.where(y > 0, 1.0, SLOPE)


# ---------------------------------------------------------------- network

def forward(theta: np.ndarray, x0: np.ndarray, round_weights: bool = True):
    """x0 [Z][Y][X][8] -> (g [Z][Y][X][3], cache).  With ``round_weights`` the
    weights are rounded to bfloat16 first (the CUDA path's arithmetic);
    biases stay as given."""
    P = unpack(np.asarray(theta, dtype=np.float64))
    if round_weights:
        P = {k: (bf16_round(W), b) for k, (W, b) in P.items()}

    def layer(name, x):
        W, b = P[name]
        _, ci, co, s, act = next(L for L in LAYERS if L[0] == name)
        assert x.shape[3] == ci
        z = conv3d(x, W, b, s)
        return lrelu(z) if act else z

    c = {"x0": x0}
    c["a0"] = layer("e0a", x0)
    c["s0"] = layer("e0b", c["a0"])
    c["b1"] = layer("d1", c["s0"])
    c["s1"] = layer("e1", c["b1"])
    c["b2"] = layer("d2", c["s1"])
    c["s2"] = layer("e2", c["b2"])
    c["b3"] = layer("d3", c["s2"])
    c["c3"] = layer("e3", c["b3"])
    c["cat2"] = np.concatenate([upsample(c["c3"]), c["s2"]], axis=3)
    c["y2"] = layer("u2", c["cat2"])
    c["cat1"] = np.concatenate([upsample(c["y2"]), c["s1"]], axis=3)
    c["y1"] = layer("u1", c["cat1"])
    c["cat0"] = np.concatenate([upsample(c["y1"]), c["s0"]], axis=3)
    c["y0"] = layer("u0", c["cat0"])
    c["g"] = layer("out", c["y0"])
    c["P"] = P
    return c["g"], c


def backward(cache: dict, gg: np.ndarray):
    """Gradient of a scalar loss with respect to the flat parameter vector,
    given dLoss/dg; the derivative is taken through the bf16-rounded weights
    (straight-through: dL/dW_master = dL/dW_rounded).  Returns (dtheta, dx0)."""
    c, P = cache, cache["P"]
    grads = {}

    def back(name, x_in, gout):
        W, _ = P[name]
        s = next(L for L in LAYERS if L[0] == name)[3]
        gx, gW, gb = conv3d_backward(x_in, W, gout, s)
        grads[name] = (gW, gb)
        return gx

    g_y0 = back("out", c["y0"], gg) * lrelu_grad_from_output(c["y0"])
    g_cat0 = back("u0", c["cat0"], g_y0)
    n1 = c["y1"].shape[3]
    g_y1 = upsample_adjoint(g_cat0[..., :n1]) * lrelu_grad_from_output(c["y1"])
    g_s0 = g_cat0[..., n1:]
    g_cat1 = back("u1", c["cat1"], g_y1)
    n2 = c["y2"].shape[3]
    g_y2 = upsample_adjoint(g_cat1[..., :n2]) * lrelu_grad_from_output(c["y2"])
    g_s1 = g_cat1[..., n2:]
    g_cat2 = back("u2", c["cat2"], g_y2)
    n3 = c["c3"].shape[3]
    g_c3 = upsample_adjoint(g_cat2[..., :n3]) * lrelu_grad_from_output(c["c3"])
    g_s2 = g_cat2[..., n3:]
    g_b3 = back("e3", c["b3"], g_c3) * lrelu_grad_from_output(c["b3"])
    g_s2 = (g_s2 + back("d3", c["s2"], g_b3)) * lrelu_grad_from_output(c["s2"])
    g_b2 = back("e2", c["b2"], g_s2) * lrelu_grad_from_output(c["b2"])
    g_s1 = (g_s1 + back("d2", c["s1"], g_b2)) * lrelu_grad_from_output(c["s1"])
    g_b1 = back("e1", c["b1"], g_s1) * lrelu_grad_from_output(c["b1"])
    g_s0 = (g_s0 + back("d1", c["s0"], g_b1)) * lrelu_grad_from_output(c["s0"])
    g_a0 = back("e0b", c["a0"], g_s0) * lrelu_grad_from_output(c["a0"])
    g_x0 = back("e0a", c["x0"], g_a0)
    return pack(grads), g_x0


def loss_mask(x0: np.ndarray) -> np.ndarray:
    """[Z][Y][X][1] weight: 1 on nodes whose fixed indicator (channel 4) is 0."""
    return (x0[..., 4:5] < 0.5).astype(np.float64)


def mse_loss(g: np.ndarray, target: np.ndarray, mask: np.ndarray):
    """Mean squared error over the DOFs of unmasked nodes (the count sums over
    the batch when the arrays carry one); returns (loss, dLoss/dg)."""
    cnt = 3.0 * mask.sum()
    d = (g - target) * mask
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def adam_step(w, m, v, grad, t: int, lr: float):
    """One bias-corrected Adam update (t counts from 1); returns (w, m, v)."""
    m = BETA1 * m + (1.0 - BETA1) * grad
    v = BETA2 * v + (1.0 - BETA2) * grad * grad
    mh = m / (1.0 - BETA1 ** t)
    vh = v / (1.0 - BETA2 ** t)
    return w - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def energy_loss(g: np.ndarray, t: np.ndarray, fixed: np.ndarray, apply_K):
    """Scale-free energy loss of one sample, (L, dL/dg): with g and t
    restricted to the free DOFs (DOF vectors), a = t.K g, b = g.K g,
    c = t.K t, L = 1 - a^2 / (b c) and dL/dg = (2a / (b c)) ((a/b) K g - K t);
    L = 1 with a zero gradient when b or c is not positive."""
    free = ~np.asarray(fixed).astype(bool)
    gm = np.where(free, np.asarray(g, dtype=np.float64).reshape(-1), 0.0)
    tm = np.where(free, np.asarray(t, dtype=np.float64).reshape(-1), 0.0)
    Kg = np.where(free, apply_K(gm), 0.0)
    Kt = np.where(free, apply_K(tm), 0.0)
    a, b, c = float(tm @ Kg), float(gm @ Kg), float(tm @ Kt)
    if not (b > 0 and c > 0):
        return 1.0, np.zeros_like(gm)
    return 1.0 - a * a / (b * c), (2.0 * a / (b * c)) * ((a / b) * Kg - Kt)


def clip_gradient(grad, clip: float):
    """grad scaled to L2 norm at most clip (clip <= 0: unchanged); a
    non-finite norm gives a zero gradient."""
    if clip <= 0:
        return grad
    nrm = float(np.sqrt(np.sum(grad * grad)))
    if not np.isfinite(nrm):
        return np.zeros_like(grad)
    return grad * min(1.0, clip / nrm) if nrm > 0 else grad


def train_step(theta, m, v, t: int, lr: float, batch, clip: float = 0.0, ops=None):
    """Loss, gradient and Adam update on a batch [(x0, target), ...] of one
    grid size.  ops = None: the mean squared error over all unmasked DOFs of
    the batch; else ops[b] = (fixed, apply_K) of sample b and the batch mean
    of the scale-free energy loss.  The returned gradient is the unclipped one."""
    grad = np.zeros_like(theta)
    if ops is None:
        cnt = sum(3.0 * loss_mask(x).sum() for x, _ in batch)
        total = 0.0
        for x, tgt in batch:
            g, cache = forward(theta, x)
            d = (g - tgt) * loss_mask(x)
            total += float((d * d).sum())
            gt, _ = backward(cache, 2.0 * d / cnt)
            grad += gt
        loss = total / cnt
    else:
        loss = 0.0
        for (x, tgt), (fixed, apply_K) in zip(batch, ops):
            g, cache = forward(theta, x)
            L, dg = energy_loss(g, tgt, fixed, apply_K)
            loss += L / len(batch)
            gt, _ = backward(cache, (dg / len(batch)).reshape(g.shape))
            grad += gt
    theta, m, v = adam_step(theta, m, v, clip_gradient(grad, clip), t, lr)
    return loss, grad, theta, m, v


# ---------------------------------------------------------------- features

def node_features(nx: int, ny: int, nz: int, rho: np.ndarray, f: np.ndarray, fixed: np.ndarray) -> np.ndarray:
    """[nz+1][ny+1][nx+1][12] network input for one cantilever problem."""
    rho = np.asarray(rho, dtype=np.float64).reshape(nz, ny, nx)
    acc = np.zeros((nz + 1, ny + 1, nx + 1))
    cnt = np.zeros_like(acc)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                acc[dz:dz + nz, dy:dy + ny, dx:dx + nx] += rho
                cnt[dz:dz + nz, dy:dy + ny, dx:dx + nx] += 1.0
    x = np.zeros((nz + 1, ny + 1, nx + 1, N_IN))
    x[..., 0] = acc / cnt
    F = np.asarray(f, dtype=np.float64).reshape(nz + 1, ny + 1, nx + 1, 3)
    fmax = np.abs(F).max()
    if fmax > 0:
        x[..., 1:4] = F / fmax
    x[..., 4] = np.asarray(fixed).reshape(nz + 1, ny + 1, nx + 1, 3).any(axis=3)
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    x[..., 5] = i / nx
    x[..., 6] = j / ny
    x[..., 7] = k / nz
    res = F.reshape(-1, 3).sum(axis=0)
    rn = np.linalg.norm(res)
    if rn > 0:
        x[..., 8:11] = res / rn
    x[..., 11] = 1.0
    return x


def normalised_target(u: np.ndarray) -> np.ndarray:
    """u / RMS(u) over all entries (0 stays 0)."""
    u = np.asarray(u, dtype=np.float64)
    rms = np.sqrt(np.mean(u * u))
    return u / rms if rms > 0 else u.copy()


def warm_start(apply_K, f: np.ndarray, g: np.ndarray, fixed: np.ndarray):
    """Energy-optimal rescaling of the network output g (DOF vector).
    Returns (u0, alpha); alpha = 0 means the cold start was kept."""
    g = np.where(np.asarray(fixed).astype(bool), 0.0, np.asarray(g, dtype=np.float64))
    fg = float(f @ g)
    gKg = float(g @ apply_K(g))
    if not (gKg > 0 and np.isfinite(fg) and np.isfinite(gKg)):
        return np.zeros_like(g), 0.0
    alpha = fg / gKg
    return alpha * g, alpha
