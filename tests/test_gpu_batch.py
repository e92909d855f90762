"""Batched persistent solve (csff_batch_*) against the single-problem path and
the CPU oracle; the bounded grid barrier's failure path.  GPU only."""
import numpy as np
import pytest

import oracle.csff_oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def csff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4461_gb300 as m
    return m


def _cases(n=8, sizes=(65, 129, 257)):
    cs = W.batch_2d(n, seed=4461, sizes=sizes)
    for c in cs:
        c["opts"].update(precision="mixed", inner_cycles=3, refine_fp64=1)
    return cs


@pytest.fixture(scope="module")
def batch(csff):
    cs = _cases()
    b = csff.Batch([c["problem"] for c in cs], cs[0]["opts"])
    eta = np.vstack([c["eta"] for c in cs])
    yield b, cs, eta
    b.close()


def test_batch_solutions_meet_tolerance_and_match_single_solves(csff, batch):
    b, cs, eta = batch
    st, infos = b.solve(eta)
    assert st == csff.OK
    for i, c in enumerate(cs):
        p = O.problem_from_dict(c["problem"])
        rhs = O.rhs(p, c["eta"][0])
        u = b.solution(i).cpu().numpy().reshape((p.m, p.m))
        lv = O.make_level(p, p.n)
        # the oracle's residual of the batched solution (property at any size)
        assert O.norm2(O.residual(lv, u, rhs)) <= 1.01e-8 * O.norm2(rhs)
        assert infos[i]["status"] == csff.OK and infos[i]["rel_res"] <= 1e-8
        # the single-problem mixed path runs the same iteration
        plan = csff.Plan(c["problem"], c["opts"])
        us = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
        _, inf1 = plan.solve(c["eta"], us)
        assert inf1[0]["cycles"] == infos[i]["cycles"]
        assert np.allclose(inf1[0]["history"], infos[i]["history"], rtol=1e-5, atol=1e-14)
        assert np.linalg.norm(us.cpu().numpy() - u.ravel()) <= 1e-7 * np.linalg.norm(u)
        plan.close()


def test_batch_far_field_matches_oracle_on_same_solution(csff, batch):
    b, cs, eta = batch
    b.solve(eta)
    al = [c["alphas"][::9] for c in cs]
    F = [torch.zeros(len(a), dtype=torch.complex128, device="cuda") for a in al]
    E = [torch.zeros(len(a), dtype=torch.int32, device="cuda") for a in al]
    b.far_field(eta, al, F, E)
    for i, c in enumerate(cs):
        p = O.problem_from_dict(c["problem"])
        u = b.solution(i).cpu().numpy().reshape((p.m, p.m))
        m, e2, tn = O.far_field(p, u, c["eta"][0], al[i], return_terms_norm=True)
        Fg = F[i].cpu().numpy() * 2.0 ** (E[i].cpu().numpy().astype(np.float64) - e2)
        assert np.abs(Fg - m).max() <= 1e-12 * tn.max()


def test_batch_with_all_four_sizes_and_repeat(csff):
    """Uneven sizes up to 513^2 (every level count from 6 to 9), solved twice
    in a row through the replayed graph."""
    cs = _cases(6, sizes=(65, 129, 257, 513))
    b = csff.Batch([c["problem"] for c in cs], cs[0]["opts"])
    eta = np.vstack([c["eta"] for c in cs])
    st1, i1 = b.solve(eta)
    st2, i2 = b.solve(eta)
    assert st1 == st2 == csff.OK
    assert [x["cycles"] for x in i1] == [x["cycles"] for x in i2]
    assert all(x["rel_res"] <= 1e-8 for x in i2)
    b.close()


def test_batch_autotune_keeps_results(csff, batch):
    b, cs, eta = batch
    _, ref = b.solve(eta)
    tc, per = b.autotune(eta)
    assert tc in (8, 16) and per >= 1
    st, infos = b.solve(eta)
    assert st == csff.OK
    assert [x["cycles"] for x in infos] == [x["cycles"] for x in ref]


def test_bounded_barrier_reports_timeout_and_context_survives(csff):
    """A barrier that waits for a CTA that does not exist gives up after the
    spin limit: the solve returns TIMEOUT (no trap, no hang) and the next
    normal solve on the same context succeeds."""
    cs = _cases(3, sizes=(65, 129))
    b = csff.Batch([c["problem"] for c in cs], cs[0]["opts"])
    eta = np.vstack([c["eta"] for c in cs])
    b.debug_barrier(1, spin_limit=1 << 14)
    st, infos = b.solve(eta, ok=(csff.ERR_TIMEOUT,))
    assert st == csff.ERR_TIMEOUT and all(x["status"] == csff.ERR_TIMEOUT for x in infos)
    b.debug_barrier(0)
    st, infos = b.solve(eta)
    assert st == csff.OK and all(x["rel_res"] <= 1e-8 for x in infos)
    b.close()


def test_batch_adaptive_schedule_matches_single_plans(csff):
    """With adaptive_inner each instance sizes its refinement steps from the
    previous step's reduction factor inside the persistent kernel: the same
    cycle counts and histories as the single-plan FP64-refinement solves with
    the same schedule, no more cycles than the fixed schedule, and every
    solution meets 1e-8 under the oracle's operator."""
    cs = _cases(6, sizes=(65, 129, 257))
    for c in cs:
        c["opts"].update(inner_cycles=6, adaptive_inner=1)
    eta = np.vstack([c["eta"] for c in cs])
    b = csff.Batch([c["problem"] for c in cs], cs[0]["opts"])
    st, infos = b.solve(eta)
    assert st == csff.OK
    bf = csff.Batch([c["problem"] for c in cs], dict(cs[0]["opts"], adaptive_inner=0))
    _, fixed = bf.solve(eta)
    assert sum(x["cycles"] for x in infos) <= sum(x["cycles"] for x in fixed)
    for i, c in enumerate(cs):
        p = O.problem_from_dict(c["problem"])
        rhs = O.rhs(p, c["eta"][0])
        u = b.solution(i).cpu().numpy().reshape((p.m, p.m))
        assert O.norm2(O.residual(O.make_level(p, p.n), u, rhs)) <= 1.01e-8 * O.norm2(rhs)
        plan = csff.Plan(c["problem"], c["opts"])
        us = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
        _, inf1 = plan.solve(c["eta"], us)
        assert inf1[0]["cycles"] == infos[i]["cycles"]
        assert np.allclose(inf1[0]["history"], infos[i]["history"], rtol=1e-5, atol=1e-14)
        plan.close()
    b.close()
    bf.close()
