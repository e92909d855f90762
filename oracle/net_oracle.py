"""FP64 oracle of the learned smoother (test infrastructure only).

The learned smoother is not in the paper; it is a small convolutional network
N that maps the residual r of a multigrid level to a correction, used as
u <- u + N(h^2 r) = u + h^2 N(r) after a red-black sweep on the finest levels
(N is positively homogeneous; the loss below then takes the operator in units
of h^2, c = e^{-2i gamma} and q = (kh)^2 (1 + chi)).  Complex values are two
real channels (re, im).

    h1 = relu(conv(x0, w1)),  h2 = relu(conv(h1, w2)),  y = conv(h2, w3)
    x0 = (Re r, Im r),  w1: 16x2x3x3, w2: 16x16x3x3, w3: 2x16x3x3, no biases

conv is a 3x3 cross-correlation with zero padding:
    out[o, i, j] = sum_c sum_{a,b in 0..2} w[o, c, a, b] x[c, i + a - 1, j + b - 1].

The 3D network (3x3x3 cross-correlations, 7-point operator) follows the same
definitions with a third spatial index; see the functions ending in 3.

Training loss for one patch (the residual after the learned step, relative):
    L = sum_mask |r - A y|^2 / sum_mask |r|^2,
    A y = c (4 y - sum_nbr y) - q y  (the level's rotated-grid operator,
          eq. csg with the Sec. 5.2 stencil, zero outside the patch),
over an interior mask that leaves out a margin of width `margin`.
A is complex symmetric, so the adjoint used in the gradient is conj(A(conj .)).
"""
from __future__ import annotations

import numpy as np

SHAPES = ((16, 2), (16, 16), (2, 16))
N_PARAMS = sum(o * i * 9 for o, i in SHAPES)


def split(theta: np.ndarray):
    """Flat parameter vector -> [w1, w2, w3] with shapes (out, in, 3, 3)."""
    out, p = [], 0
    for o, i in SHAPES:
        n = o * i * 9
        out.append(theta[p:p + n].reshape(o, i, 3, 3))
        p += n
    return out


def init_params(seed: int) -> np.ndarray:
    """He-style normal initialisation, the last layer scaled down."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l, (o, i) in enumerate(SHAPES):
        std = np.sqrt(2.0 / (9 * i)) * (0.1 if l == 2 else 1.0)
        parts.append(rng.standard_normal(o * i * 9) * std)
    return np.concatenate(parts)


def conv3x3(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    cin, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    out = np.zeros((w.shape[0], H, W))
    for a in range(3):
        for b in range(3):
            out += np.einsum("oc,chw->ohw", w[:, :, a, b], xp[:, a:a + H, b:b + W])
    return out


def conv3x3_input_grad(dout: np.ndarray, w: np.ndarray) -> np.ndarray:
    """d/dx of sum(dout * conv(x, w))."""
    cout, H, W = dout.shape
    dp = np.pad(dout, ((0, 0), (1, 1), (1, 1)))
    dx = np.zeros((w.shape[1], H, W))
    for a in range(3):
        for b in range(3):
            # x[c, i + a - 1, j + b - 1] feeds out[o, i, j]
            dx += np.einsum("oc,ohw->chw", w[:, :, a, b], dp[:, 2 - a:2 - a + H, 2 - b:2 - b + W])
    return dx


def conv3x3_weight_grad(dout: np.ndarray, x: np.ndarray) -> np.ndarray:
    cin, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    dw = np.zeros((dout.shape[0], cin, 3, 3))
    for a in range(3):
        for b in range(3):
            dw[:, :, a, b] = np.einsum("ohw,chw->oc", dout, xp[:, a:a + H, b:b + W])
    return dw


def forward(theta: np.ndarray, r: np.ndarray):
    """r: complex (H, W) -> complex correction y and the activations."""
    w1, w2, w3 = split(theta)
    x0 = np.stack([r.real, r.imag])
    z1 = conv3x3(x0, w1)
    h1 = np.maximum(z1, 0.0)
    z2 = conv3x3(h1, w2)
    h2 = np.maximum(z2, 0.0)
    y = conv3x3(h2, w3)
    return y[0] + 1j * y[1], (x0, z1, h1, z2, h2)


def apply_A_patch(c: complex, q: np.ndarray, y: np.ndarray) -> np.ndarray:
    yp = np.pad(y, 1)
    nb = yp[:-2, 1:-1] + yp[2:, 1:-1] + yp[1:-1, :-2] + yp[1:-1, 2:]
    return c * (4 * y - nb) - q * y


def mask_of(shape, margin):
    m = np.zeros(shape, bool)
    m[margin:shape[0] - margin, margin:shape[1] - margin] = True
    return m


def loss_and_grad(theta: np.ndarray, r: np.ndarray, q: np.ndarray, c: complex, margin: int = 4):
    """Loss of one patch and its gradient with respect to theta (manual backprop)."""
    w1, w2, w3 = split(theta)
    y, (x0, z1, h1, z2, h2) = forward(theta, r)
    msk = mask_of(r.shape, margin)
    S = np.sum(np.abs(r[msk]) ** 2)
    E = (r - apply_A_patch(c, q, y)) * msk
    L = np.sum(np.abs(E) ** 2) / S
    G = 2.0 * E / S                                   # dL/dE as complex (re, im)
    gy = -np.conj(apply_A_patch(c, q, np.conj(G)))    # dL/dy = -A^H G
    dy = np.stack([gy.real, gy.imag])
    g3 = conv3x3_weight_grad(dy, h2)
    dh2 = conv3x3_input_grad(dy, w3) * (z2 > 0)
    g2 = conv3x3_weight_grad(dh2, h1)
    dh1 = conv3x3_input_grad(dh2, w2) * (z1 > 0)
    g1 = conv3x3_weight_grad(dh1, x0)
    return L, np.concatenate([g1.ravel(), g2.ravel(), g3.ravel()])


# ---- the 3D network: the same three layers with 3x3x3 cross-correlations,
#   out[o, z, i, j] = sum_c sum_{a,b,e in 0..2} w[o, c, a, b, e] x[c, z + a - 1, i + b - 1, j + e - 1],
# zero padding, weights (out, in, a, b, e); the loss with the 7-point operator
#   A y = c (6 y - sum_nbr y) - q y   (eq. csg with the Sec. 5.2 stencil in 3D).

N_PARAMS_3D = sum(o * i * 27 for o, i in SHAPES)
_TAPS3 = [(a, b, e) for a in range(3) for b in range(3) for e in range(3)]


def split3(theta: np.ndarray):
    """Flat parameter vector -> [w1, w2, w3] with shapes (out, in, 3, 3, 3)."""
    out, p = [], 0
    for o, i in SHAPES:
        n = o * i * 27
        out.append(theta[p:p + n].reshape(o, i, 3, 3, 3))
        p += n
    return out


def init_params3(seed: int) -> np.ndarray:
    """He-style normal initialisation (fan-in 27 per input channel), the last
    layer scaled down."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l, (o, i) in enumerate(SHAPES):
        std = np.sqrt(2.0 / (27 * i)) * (0.1 if l == 2 else 1.0)
        parts.append(rng.standard_normal(o * i * 27) * std)
    return np.concatenate(parts)


def conv3x3x3(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    cin, Z, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((w.shape[0], Z, H, W))
    for a, b, e in _TAPS3:
        out += np.einsum("oc,czhw->ozhw", w[:, :, a, b, e], xp[:, a:a + Z, b:b + H, e:e + W])
    return out


def conv3x3x3_input_grad(dout: np.ndarray, w: np.ndarray) -> np.ndarray:
    """d/dx of sum(dout * conv3x3x3(x, w))."""
    cout, Z, H, W = dout.shape
    dp = np.pad(dout, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dx = np.zeros((w.shape[1], Z, H, W))
    for a, b, e in _TAPS3:
        dx += np.einsum("oc,ozhw->czhw", w[:, :, a, b, e], dp[:, 2 - a:2 - a + Z, 2 - b:2 - b + H, 2 - e:2 - e + W])
    return dx


def conv3x3x3_weight_grad(dout: np.ndarray, x: np.ndarray) -> np.ndarray:
    cin, Z, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    dw = np.zeros((dout.shape[0], cin, 3, 3, 3))
    for a, b, e in _TAPS3:
        dw[:, :, a, b, e] = np.einsum("ozhw,czhw->oc", dout, xp[:, a:a + Z, b:b + H, e:e + W])
    return dw


def forward3(theta: np.ndarray, r: np.ndarray):
    """r: complex (Z, H, W) -> complex correction y and the activations."""
    w1, w2, w3 = split3(theta)
    x0 = np.stack([r.real, r.imag])
    z1 = conv3x3x3(x0, w1)
    h1 = np.maximum(z1, 0.0)
    z2 = conv3x3x3(h1, w2)
    h2 = np.maximum(z2, 0.0)
    y = conv3x3x3(h2, w3)
    return y[0] + 1j * y[1], (x0, z1, h1, z2, h2)


def apply_A_patch3(c: complex, q: np.ndarray, y: np.ndarray) -> np.ndarray:
    yp = np.pad(y, 1)
    nb = (yp[:-2, 1:-1, 1:-1] + yp[2:, 1:-1, 1:-1] + yp[1:-1, :-2, 1:-1] + yp[1:-1, 2:, 1:-1] +
          yp[1:-1, 1:-1, :-2] + yp[1:-1, 1:-1, 2:])
    return c * (6 * y - nb) - q * y


def mask_of3(shape, margin):
    m = np.zeros(shape, bool)
    m[margin:shape[0] - margin, margin:shape[1] - margin, margin:shape[2] - margin] = True
    return m


def loss_and_grad3(theta: np.ndarray, r: np.ndarray, q: np.ndarray, c: complex, margin: int = 4):
    """loss_and_grad for a 3D patch (Z, H, W)."""
    w1, w2, w3 = split3(theta)
    y, (x0, z1, h1, z2, h2) = forward3(theta, r)
    msk = mask_of3(r.shape, margin)
    S = np.sum(np.abs(r[msk]) ** 2)
    E = (r - apply_A_patch3(c, q, y)) * msk
    L = np.sum(np.abs(E) ** 2) / S
    G = 2.0 * E / S
    gy = -np.conj(apply_A_patch3(c, q, np.conj(G)))
    dy = np.stack([gy.real, gy.imag])
    g3 = conv3x3x3_weight_grad(dy, h2)
    dh2 = conv3x3x3_input_grad(dy, w3) * (z2 > 0)
    g2 = conv3x3x3_weight_grad(dh2, h1)
    dh1 = conv3x3x3_input_grad(dh2, w2) * (z1 > 0)
    g1 = conv3x3x3_weight_grad(dh1, x0)
    return L, np.concatenate([g1.ravel(), g2.ravel(), g3.ravel()])


def batch_loss_and_grad(theta, rs, qs, cs, margin=4):
    """Mean over patches of loss_and_grad."""
    L, g = 0.0, np.zeros_like(theta)
    for r, q, c in zip(rs, qs, cs):
        l, gg = loss_and_grad(theta, r, q, c, margin)
        L += l
        g += gg
    return L / len(rs), g / len(rs)
