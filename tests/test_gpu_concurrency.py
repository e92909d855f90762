"""Plans driven from several host threads at once, one stream each (the bench
solves its four maps this way): every solution, residual history and far-field
map must equal the one-after-the-other results bit for bit (plans share no
state; graph capture is per thread)."""
import threading

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def csff():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1211_4461_gb300 as m
    return m


def test_concurrent_plans_match_sequential(csff):
    cases = [W.mixed_2d(k, n=257) for k in (5.0, 10.0, 20.0, 40.0)]
    for c in cases:
        c["opts"].update(precision="mixed", inner_cycles=6, coarsest_n=9)
    streams = [torch.cuda.Stream() for _ in cases]
    plans = [csff.Plan(c["problem"], c["opts"], stream=s) for c, s in zip(cases, streams)]
    us = [torch.zeros(p.N, dtype=torch.complex128, device="cuda") for p in plans]
    Fs = [torch.zeros(len(c["alphas"]), dtype=torch.complex128, device="cuda") for c in cases]
    Es = [torch.zeros(len(c["alphas"]), dtype=torch.int32, device="cuda") for c in cases]
    infos = [None] * len(cases)

    def work(i):
        with torch.cuda.stream(streams[i]):
            _, infos[i] = plans[i].solve(cases[i]["eta"], us[i])
            plans[i].far_field(cases[i]["eta"], us[i], cases[i]["alphas"], Fs[i], Es[i])
            streams[i].synchronize()

    def snapshot():
        return [(u.cpu().numpy().copy(), F.cpu().numpy().copy(), E.cpu().numpy().copy(), inf[0]["history"])
                for u, F, E, inf in zip(us, Fs, Es, infos)]

    for i in range(len(cases)):
        work(i)
    ref = snapshot()
    for rep in range(2):
        for u in us:
            u.zero_()
        th = [threading.Thread(target=work, args=(i,)) for i in range(len(cases))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        got = snapshot()
        for (u0, f0, e0, h0), (u1, f1, e1, h1) in zip(ref, got):
            assert np.array_equal(u0, u1) and np.array_equal(f0, f1) and np.array_equal(e0, e1)
            assert h0 == h1
    for p in plans:
        p.close()
