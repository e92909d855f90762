"""The 3D learned smoother (3x3x3 network) on the GPU against the FP64 network
oracle: forward, loss and gradients, training on the method's own 3D
residuals, and the learned step inside 3D mixed-precision solves.  BF16
storage with FP32 accumulation bounds the agreement as in 2D."""
import math

import numpy as np
import pytest

import oracle.net_oracle as NO
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def csff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4461_gb300 as m
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(torch.complex64)


def _bf16(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _patches(B=2, S=(9, 10, 11), seed=0):
    r = W.rand_complex((B,) + S, seed)
    q = W.rand_complex((B,) + S, seed + 1, scale=0.3) + 3.0
    c = np.array([complex(np.exp(-1j * math.pi / 3) * (6.0 + b)) for b in range(B)])
    return r, q, c


def test_forward3_matches_oracle(csff):
    theta = NO.init_params3(5)
    net = csff.Net(theta, dim=3)
    r, _, _ = _patches()
    y = torch.empty(r.shape, dtype=torch.complex64, device="cuda")
    net.forward(_dev(r), y)
    tb = _bf16(theta)
    for b in range(r.shape[0]):
        rb = _bf16(r[b].real) + 1j * _bf16(r[b].imag)
        ref, _ = NO.forward3(tb, rb)
        got = y[b].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 2e-2 * np.linalg.norm(ref)
        assert np.abs(got - ref).max() <= 5e-2 * np.abs(ref).max()
    net.close()


def test_loss3_and_gradient_match_oracle(csff):
    theta = NO.init_params3(6)
    net = csff.Net(theta, dim=3)
    r, q, c = _patches(2, (8, 8, 8), 3)
    L, g = net.loss_grad(_dev(r), _dev(q), c, margin=2)
    tb = _bf16(theta)
    Lo, go = 0.0, np.zeros_like(theta)
    for b in range(r.shape[0]):
        rb = _bf16(r[b].real) + 1j * _bf16(r[b].imag)
        l, gg = NO.loss_and_grad3(tb, rb, q[b], c[b], margin=2)
        Lo += l / r.shape[0]
        go += gg / r.shape[0]
    assert abs(L - Lo) <= 2e-2 * abs(Lo)
    assert np.linalg.norm(g - go) <= 5e-2 * np.linalg.norm(go)
    n1, n2 = 16 * 2 * 27, 16 * 16 * 27
    for sl in (slice(0, n1), slice(n1, n1 + n2), slice(n1 + n2, None)):
        assert np.linalg.norm(g[sl] - go[sl]) <= 8e-2 * np.linalg.norm(go[sl])
    net.close()


def test_dimension_mismatch_is_refused(csff):
    """A 3D network is refused by the 2D calls and by 2D plans (and the other
    way round)."""
    net3 = csff.Net(NO.init_params3(1), dim=3)
    net2 = csff.Net(NO.init_params(1))
    r = torch.zeros((1, 8, 8), dtype=torch.complex64, device="cuda")
    assert csff._lib.csff_net_forward(net3._h, 1, 8, 8, csff._ptr(r), csff._ptr(r), None) == csff.ERR_INVALID_ARG
    assert csff._lib.csff_net_forward3(net2._h, 1, 1, 8, 8, csff._ptr(r), csff._ptr(r), None) == \
        csff.ERR_INVALID_ARG
    c = W.small_2d(n=33)
    plan = csff.Plan(c["problem"], dict(c["opts"], smoother="rbgs", precision="mixed"))
    with pytest.raises(csff.CsffError):
        plan.set_learned(net3)
    plan.close()
    c3 = _problems3([0], n=17)[0][0]
    plan3 = csff.Plan(c3, dict(OPTS3, precision="mixed"))
    with pytest.raises(csff.CsffError):
        plan3.set_learned(net2)
    plan3.close()
    net3.close()
    net2.close()


def _problems3(seeds, n=33):
    """3D problems on [-6, 6]^3 with k h in 0.8-1.2 on the finest level."""
    out = []
    for s in seeds:
        rng = np.random.Generator(np.random.PCG64(3000 + s))
        h = 12.0 / (n - 1)
        k = float(rng.uniform(0.8, 1.2)) / h
        amp = float(rng.uniform(-1.5, -0.5))
        w = float(rng.uniform(1.5, 3.0))
        th, ph = float(rng.uniform(0, math.pi)), float(rng.uniform(0, 2 * math.pi))
        eta = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        out.append((W.problem(3, n, 6.0, math.pi / 6, k, [W.gauss(amp, w)]), eta))
    return out


OPTS3 = {"smoother": "rbgs", "omega": 1.0, "nu1": 1, "nu2": 1, "coarsest_n": 5, "rel_tol": 1e-8,
         "max_cycles": 300, "inner_cycles": 3}


@pytest.fixture(scope="module")
def trained3(csff):
    from paper_1211_4461_gb300 import learned as LR
    data = LR.collect_patches(_problems3(range(6)), OPTS3, n_cycles=4, patch=12, per_field=6, seed=1)
    net = csff.Net(LR.init_weights(7, dim=3), dim=3)
    hist = LR.train(net, data, steps=300, batch=8, lr=2e-3, margin=2, seed=2)
    return net, hist


def test_training_on_3d_solver_residuals_reduces_the_loss(trained3):
    net, hist = trained3
    assert np.all(np.isfinite(hist))
    assert np.mean(hist[-20:]) < 0.8 * np.mean(hist[:5])


def test_learned_smoother_in_3d_solves(csff, trained3):
    """Held-out 3D problems: the learned variant reaches 1e-8 (re-checked with
    the oracle's FP64 operator), the network is used, and the cycle count is
    recorded against plain red-black sweeps (at worst a few more through the
    fallback)."""
    import oracle.csff_oracle as O
    net, _ = trained3
    for prob, eta in _problems3([100, 101]):
        plan = csff.Plan(prob, dict(OPTS3, precision="mixed", refine_fp64=1))
        u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
        _, base = plan.solve(np.atleast_2d(eta), u)
        plan.set_learned(net, levels=1)
        u2 = torch.zeros_like(u)
        st, lrn = plan.solve(np.atleast_2d(eta), u2)
        assert st == csff.OK and lrn[0]["rel_res"] <= 1e-8 and lrn[0]["flags"] & 1
        assert lrn[0]["cycles"] <= base[0]["cycles"] + 3
        p = O.problem_from_dict(prob)
        b = O.rhs(p, eta)
        ug = u2.cpu().numpy().reshape((p.m,) * 3)
        assert O.norm2(O.residual(O.make_level(p, p.n), ug, b)) <= 1.01e-8 * O.norm2(b)
        plan.close()
