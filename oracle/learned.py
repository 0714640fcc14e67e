"""Learned unrolled proximal-gradient solver (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper has no learned component; this is the learned form of the task,
defined here step by step so that the device kernels can be checked against it.

Stages s = 0 .. S-1, starting from x_0 (zero, or the per-frequency Tikhonov
solution of the measurement, ``solvers.tikhonov``, passed in), with the
normalised operator A_n = C K / s (unit norm) and m_n = m / s:
    g_s     = A_n^T (A_n x_s - m_n)                 (gradient of 1/2 ||A_n x - m_n||^2)
    z_s     = x_s - eta_s g_s                       (gradient step, eta_s learnable)
    x_{s+1} = z_s + mu0 f(z_s / mu0)                (residual proximal step)
At inference the stages may be followed by data-consistency steps
x <- x - T(A_n x - m_n), T the per-frequency Tikhonov solve (``dc_solve``),
which is scale-free, so T for A_n is T for A.
f is a 3-D CNN shared by all stages: conv(1->16) + b, ReLU, conv(16->16) + b,
ReLU, conv(16->16) + b, ReLU, conv(16->1) + b, all 3 x 3 x 3 with zero 'same'
padding on the N x N x Z volume; mu0 = 0.01 / mm fixes the scale of its input.
Loss: mean over voxels of ((x_S - mu_true) / mu0)^2.

Parameters (flat, float): w1 [16][1][27], b1 [16], w2 [16][16][27], b2 [16],
w3 [16][16][27], b3 [16], w4 [1][16][27], b4 [1], eta [S]; the tap index is
(dz+1)*9 + (dy+1)*3 + (dx+1) for offsets dz, dy, dx in {-1, 0, 1}.
"""

import numpy as np

MU0 = 0.01
CH = 16
LAYERS = [(1, CH), (CH, CH), (CH, CH), (CH, 1)]


def param_count(stages):
    return sum(co * ci * 27 + co for ci, co in LAYERS) + stages


def unpack(theta, stages):
    """Flat parameters -> ([(w [co][ci][27], b [co])...], eta [S])."""
    out, off = [], 0
    for ci, co in LAYERS:
        w = np.asarray(theta[off:off + co * ci * 27], dtype=np.float64).reshape(co, ci, 27)
        off += co * ci * 27
        b = np.asarray(theta[off:off + co], dtype=np.float64)
        off += co
        out.append((w, b))
    eta = np.asarray(theta[off:off + stages], dtype=np.float64)
    return out, eta


def pack(layers, eta):
    parts = []
    for w, b in layers:
        parts += [np.ravel(w), np.ravel(b)]
    parts.append(np.ravel(eta))
    return np.concatenate(parts)


def _taps():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def conv3d(x, w, b):
    """y[co] = b[co] + sum_ci sum_tap w[co][ci][tap] x[ci](v + offset(tap)), zero padding.

    x [ci][Z][Y][X], w [co][ci][27], b [co] -> y [co][Z][Y][X].
    """
    _, z, yy, xx = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    y = np.zeros((w.shape[0], z, yy, xx)) + b[:, None, None, None]
    for t, (dz, dy, dx) in enumerate(_taps()):
        sl = xp[:, 1 + dz:1 + dz + z, 1 + dy:1 + dy + yy, 1 + dx:1 + dx + xx]
        y += np.einsum("oc,czyx->ozyx", w[:, :, t], sl)
    return y


def conv3d_backward(x, w, gy):
    """Gradients of conv3d w.r.t. its input, weights and bias for output gradient gy."""
    _, z, yy, xx = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(_taps()):
        sl = (slice(None), slice(1 + dz, 1 + dz + z), slice(1 + dy, 1 + dy + yy), slice(1 + dx, 1 + dx + xx))
        gw[:, :, t] = np.einsum("ozyx,czyx->oc", gy, xp[sl])
        gxp[sl] += np.einsum("oc,ozyx->czyx", w[:, :, t], gy)
    gx = gxp[:, 1:-1, 1:-1, 1:-1]
    gb = gy.sum(axis=(1, 2, 3))
    return gx, gw, gb


def bf16(a):
    """Round to BF16 (8 significant bits, round to nearest, ties to even), returned as float64.

    Values are first rounded to FP32, as a device that accumulates in FP32 and
    stores BF16 does.  Used only to emulate the storage points of the BF16
    device kernels (``rnd`` below).
    """
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def cnn_forward(u, layers, rnd=None):
    """f(u) for u [Z][Y][X]; returns (out [Z][Y][X], cache).

    With ``rnd`` (e.g. ``bf16``) the network input and every layer output are
    rounded as they are stored; the cache keeps the rounded values, so the
    ReLU masks of the backward pass see them too.
    """
    r = rnd or (lambda v: v)
    a = r(u)[None]
    cache = []
    for li, (w, b) in enumerate(layers):
        y = r(conv3d(a, w, b))
        cache.append((a, y))
        a = np.maximum(y, 0.0) if li < len(layers) - 1 else y
    return a[0], cache


def cnn_backward(cache, layers, gout, rnd=None):
    """Backprop of f: returns (g_u [Z][Y][X], [(gw, gb) per layer]).

    With ``rnd`` the incoming gradient and every layer's input gradient are
    rounded as they are stored.
    """
    r = rnd or (lambda v: v)
    g = r(gout)[None]
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        a = cache[li][0]
        ga, gw, gb = conv3d_backward(a, layers[li][0], g)
        grads[li] = (gw, gb)
        # the input of layer li > 0 is ReLU(y_{li-1}): mask to get the gradient of y_{li-1}
        g = r(ga * (cache[li - 1][1] > 0)) if li > 0 else r(ga)
    return g[0], grads


def unrolled(theta, stages, op_fwd, op_adj, m_n, with_cache=False, rnd=None, x0=None, dc_steps=0, dc_solve=None):
    """The S-stage solver from x0 (default 0), then ``dc_steps`` data-consistency steps
    x <- x - dc_solve(A_n x - m_n): returns the result (and the per-stage cache if asked)."""
    layers, eta = unpack(theta, stages)
    x = np.zeros_like(op_adj(m_n)) if x0 is None else np.array(x0, dtype=np.float64)
    cache = []
    for s in range(stages):
        g = op_adj(op_fwd(x) - m_n)
        z = x - eta[s] * g
        f, cc = cnn_forward(z / MU0, layers, rnd)
        cache.append((g, z, cc))
        x = z + MU0 * f
    for _ in range(dc_steps):
        x = x - dc_solve(op_fwd(x) - m_n)
    return (x, cache) if with_cache else x


def loss_and_grad(theta, stages, op_fwd, op_adj, m_n, mu_true, rnd=None, x0=None):
    """Loss mean(((x_S - mu)/mu0)^2) and its gradient w.r.t. the flat parameters.

    ``rnd`` rounds the CNN's stored activations and gradients (see
    cnn_forward / cnn_backward); the gradient is then that of the network
    with the roundings held fixed.
    """
    layers, eta = unpack(theta, stages)
    x, cache = unrolled(theta, stages, op_fwd, op_adj, m_n, with_cache=True, rnd=rnd, x0=x0)
    r = (x - mu_true) / MU0
    loss = float(np.mean(r * r))
    gx = 2.0 * r / (MU0 * r.size)
    g_layers = [(np.zeros_like(w), np.zeros_like(b)) for w, b in layers]
    g_eta = np.zeros_like(eta)
    for s in range(stages - 1, -1, -1):
        g, z, cc = cache[s]
        # x_{s+1} = z + mu0 f(z / mu0)
        gu, gl = cnn_backward(cc, layers, MU0 * gx, rnd)
        for li in range(len(layers)):
            g_layers[li] = (g_layers[li][0] + gl[li][0], g_layers[li][1] + gl[li][1])
        gz = gx + gu / MU0
        # z = x - eta g(x),  g = A^T (A x - m)
        g_eta[s] = -float(np.sum(gz * g))
        gx = gz - eta[s] * op_adj(op_fwd(gz))
    return loss, pack(g_layers, g_eta)
