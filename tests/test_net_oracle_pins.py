"""Pins of the learned-smoother oracle: library cross-correlation, positive
homogeneity of a bias-free ReLU network, finite-difference gradients of the
loss, and the loss of the zero network.  CPU only."""
import numpy as np
import pytest
import scipy.signal as ss

import oracle.net_oracle as N
import workloads as W


def _patch(H=12, seed=0):
    r = W.rand_complex((H, H), seed)
    q = W.rand_complex((H, H), seed + 1, scale=0.3) + 2.0
    c = complex(np.exp(-1j * np.pi / 3) * 4.0)
    return r, q, c


def test_conv_matches_scipy_correlate():
    x = W.rand_real((3, 9, 11), 5)
    w = W.rand_real((4, 3, 3, 3), 6)
    out = N.conv3x3(x, w)
    for o in range(4):
        ref = sum(ss.correlate2d(x[c], w[o, c], mode="same", boundary="fill") for c in range(3))
        assert np.abs(out[o] - ref).max() < 1e-12


def test_conv_gradients_are_adjoints():
    x = W.rand_real((3, 7, 8), 7)
    w = W.rand_real((4, 3, 3, 3), 8)
    d = W.rand_real((4, 7, 8), 9)
    lhs = np.sum(d * N.conv3x3(x, w))
    assert abs(np.sum(N.conv3x3_input_grad(d, w) * x) - lhs) < 1e-10 * abs(lhs)
    assert abs(np.sum(N.conv3x3_weight_grad(d, x) * w) - lhs) < 1e-10 * abs(lhs)


def test_network_is_positively_homogeneous():
    theta = N.init_params(3)
    r, _, _ = _patch()
    y1, _ = N.forward(theta, r)
    y2, _ = N.forward(theta, 7.5 * r)
    assert np.abs(y2 - 7.5 * y1).max() < 1e-12 * np.abs(y2).max()


def test_zero_network_leaves_the_residual():
    theta = np.zeros(N.N_PARAMS)
    r, q, c = _patch()
    L, g = N.loss_and_grad(theta, r, q, c)
    assert abs(L - 1.0) < 1e-15


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_central_differences(seed):
    theta = N.init_params(10 + seed)
    r, q, c = _patch(10, seed)
    L, g = N.loss_and_grad(theta, r, q, c, margin=2)
    rng = np.random.default_rng(seed)
    idx = np.concatenate([rng.choice(288, 6, False), 288 + rng.choice(2304, 6, False),
                          2592 + rng.choice(288, 6, False)])
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (N.loss_and_grad(tp, r, q, c, 2)[0] - N.loss_and_grad(tm, r, q, c, 2)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def _patch_operator_agrees_with_level_operator(apply_patch):
    """The loss's patch operator, given the level's coefficients in units of
    h^2, must equal h^2 times the multigrid oracle's operator (eq. csg with the
    Sec. 5.2 stencil, built by the other oracle module) applied to a field that
    vanishes outside the patch, on every point of the patch."""
    import oracle.csff_oracle as O
    p = O.Problem(2, 33, -6.0, 6.0, np.pi / 6, 3.0, [O.Gaussian(-0.8 + 0.1j, 2.0, (0.5, -0.4, 0.0))])
    lv = O.make_level(p, p.n)
    y = W.rand_complex((9, 11), 17)
    Y = np.zeros((lv.m, lv.m), complex)
    i0, j0 = 7, 12
    Y[i0:i0 + 9, j0:j0 + 11] = y
    ref = lv.h ** 2 * O.apply_A(lv, Y)[i0:i0 + 9, j0:j0 + 11]
    got = apply_patch(lv.h ** 2 * lv.c, lv.h ** 2 * lv.q[i0:i0 + 9, j0:j0 + 11], y)
    return np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_loss_operator_is_the_level_operator_in_units_of_h2():
    assert _patch_operator_agrees_with_level_operator(N.apply_A_patch)


def test_planted_mistakes_in_the_loss_operator_fail_its_pin():
    def sign_on_c(c, q, y):
        return N.apply_A_patch(-c, q, y)                     # c (nb - 4 y) - q y

    def missing_q(c, q, y):
        return N.apply_A_patch(c, 0 * q, y)

    def conj_c(c, q, y):
        return N.apply_A_patch(np.conj(c), q, y)

    def diagonal_2(c, q, y):
        return N.apply_A_patch(c, q, y) - 2 * c * y           # 2 y in place of 4 y

    for bad in (sign_on_c, missing_q, conj_c, diagonal_2):
        assert not _patch_operator_agrees_with_level_operator(bad), bad.__name__
