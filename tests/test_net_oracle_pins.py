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


# ---- 3D network


def _patch3(S=(7, 8, 6), seed=0):
    r = W.rand_complex(S, seed)
    q = W.rand_complex(S, seed + 1, scale=0.3) + 2.0
    c = complex(np.exp(-1j * np.pi / 3) * 4.0)
    return r, q, c


def test_conv3d_matches_scipy_correlate():
    x = W.rand_real((2, 6, 7, 5), 15)
    w = W.rand_real((3, 2, 3, 3, 3), 16)
    out = N.conv3x3x3(x, w)
    for o in range(3):
        ref = sum(ss.correlate(x[c], w[o, c], mode="same") for c in range(2))
        assert np.abs(out[o] - ref).max() < 1e-12


def test_conv3d_with_one_plane_of_taps_is_the_2d_conv_per_slice():
    """Weights only on the middle plane a = 1 act slice by slice as the pinned
    2D cross-correlation."""
    x = W.rand_real((3, 4, 9, 8), 17)
    w2 = W.rand_real((4, 3, 3, 3), 18)
    w3 = np.zeros((4, 3, 3, 3, 3))
    w3[:, :, 1] = w2
    out = N.conv3x3x3(x, w3)
    for z in range(4):
        assert np.abs(out[:, z] - N.conv3x3(x[:, z], w2)).max() < 1e-12


def test_conv3d_gradients_are_adjoints():
    x = W.rand_real((3, 5, 6, 4), 19)
    w = W.rand_real((4, 3, 3, 3, 3), 20)
    d = W.rand_real((4, 5, 6, 4), 21)
    lhs = np.sum(d * N.conv3x3x3(x, w))
    assert abs(np.sum(N.conv3x3x3_input_grad(d, w) * x) - lhs) < 1e-10 * abs(lhs)
    assert abs(np.sum(N.conv3x3x3_weight_grad(d, x) * w) - lhs) < 1e-10 * abs(lhs)


def test_zero_3d_network_leaves_the_residual():
    r, q, c = _patch3()
    L, g = N.loss_and_grad3(np.zeros(N.N_PARAMS_3D), r, q, c, margin=1)
    assert abs(L - 1.0) < 1e-15 and np.all(g == 0)


def test_3d_gradient_matches_central_differences():
    theta = N.init_params3(4)
    r, q, c = _patch3((7, 7, 7), 3)
    L, g = N.loss_and_grad3(theta, r, q, c, margin=1)
    rng = np.random.default_rng(5)
    n1, n2 = 16 * 2 * 27, 16 * 16 * 27
    idx = np.concatenate([rng.choice(n1, 5, False), n1 + rng.choice(n2, 5, False),
                          n1 + n2 + rng.choice(2 * 16 * 27, 5, False)])
    eps = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (N.loss_and_grad3(tp, r, q, c, 1)[0] - N.loss_and_grad3(tm, r, q, c, 1)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def _patch3_operator_agrees_with_level_operator(apply_patch):
    """As the 2D pin: the 3D loss operator in units of h^2 against h^2 times the
    multigrid oracle's 7-point operator on a field that vanishes outside the
    patch."""
    import oracle.csff_oracle as O
    p = O.Problem(3, 17, -4.0, 4.0, np.pi / 6, 2.5, [O.Gaussian(-0.7 + 0.2j, 1.5, (0.3, -0.2, 0.1))])
    lv = O.make_level(p, p.n)
    y = W.rand_complex((5, 6, 7), 23)
    Y = np.zeros((lv.m,) * 3, complex)
    z0, i0, j0 = 3, 4, 5
    Y[z0:z0 + 5, i0:i0 + 6, j0:j0 + 7] = y
    ref = lv.h ** 2 * O.apply_A(lv, Y)[z0:z0 + 5, i0:i0 + 6, j0:j0 + 7]
    got = apply_patch(lv.h ** 2 * lv.c, lv.h ** 2 * lv.q[z0:z0 + 5, i0:i0 + 6, j0:j0 + 7], y)
    return np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_3d_loss_operator_is_the_level_operator_in_units_of_h2():
    assert _patch3_operator_agrees_with_level_operator(N.apply_A_patch3)


def test_planted_mistakes_in_the_3d_loss_operator_fail_its_pin():
    def sign_on_c(c, q, y):
        return N.apply_A_patch3(-c, q, y)

    def missing_q(c, q, y):
        return N.apply_A_patch3(c, 0 * q, y)

    def diagonal_4(c, q, y):
        return N.apply_A_patch3(c, q, y) - 2 * c * y           # the 2D diagonal

    for bad in (sign_on_c, missing_q, diagonal_4):
        assert not _patch3_operator_agrees_with_level_operator(bad), bad.__name__
