"""Training of the learned smoother on residuals produced by the method's own
solves.  Every computation runs in the library's CUDA kernels (per-step
multigrid calls for the data, csff_net_* for forward, backward and Adam);
this module only draws patches and loops over steps.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Net, Plan


def init_weights(seed: int, dim: int = 2) -> np.ndarray:
    """He-normal weights (last layer scaled by 0.1), layout (out, in, taps):
    3^dim taps per input channel."""
    taps = 3 ** dim
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for l, (o, i) in enumerate(((16, 2), (16, 16), (2, 16))):
        std = np.sqrt(2.0 / (taps * i)) * (0.1 if l == 2 else 1.0)
        parts.append(rng.standard_normal(o * i * taps) * std)
    return np.concatenate(parts).astype(np.float32)


def collect_patches(problems, opts, n_cycles=5, patch=64, per_field=4, seed=0, core_margin=0, min_core=0.0):
    """Residual patches as the learned step sees them: in FP32 from u = 0 on
    A u = b (b the scaled right-hand side), after each red-black sweep that
    starts a V-cycle.  Returns (r, q, c): complex64 CUDA tensors (B, P, P)
    (3D problems: (B, P, P, P)) of residuals normalised to unit RMS, the
    matching windows of h^2 q = (kh)^2(1+chi), and the per-patch constants
    h^2 c = e^{-2i gamma}: the
    operator in the units in which the plan applies the network,
    u <- u + N(h^2 r).  With min_core > 0 a window is kept only if at least
    that fraction of its residual energy lies inside its core (the window
    less core_margin on every side, the part the loss weighs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rs, qs, cs = [], [], []
    for prob, eta in problems:
        plan = Plan(prob, dict(opts, precision="mixed"))
        m = plan.m
        b64 = torch.empty(plan.N, dtype=torch.complex128, device="cuda")
        plan.rhs(np.atleast_2d(eta), b64)
        b = (b64 / b64.abs().max()).to(torch.complex64)
        u = torch.zeros(plan.N, dtype=torch.complex64, device="cuda")
        r = torch.empty_like(u)
        q, c = plan.coefficients(0)
        h2 = plan.describe()["h"][0] ** 2
        q, c = q * h2, c * h2
        d = int(prob["dim"])
        for _ in range(n_cycles):
            plan.smooth(0, u, b, 1)
            plan.residual(0, u, b, r)
            R = r.view((m,) * d)
            Q = q.view((m,) * d)
            for _ in range(per_field):
                o = rng.integers(0, m - patch + 1, size=d)
                win = tuple(slice(int(a), int(a) + patch) for a in o)
                rp = R[win]
                e2 = rp.abs().square()
                s = e2.mean().sqrt()
                if not torch.isfinite(s) or s.item() == 0.0:
                    continue
                if min_core > 0.0:
                    core = tuple(slice(core_margin, patch - core_margin) for _ in range(d))
                    if e2[core].sum().item() < min_core * e2.sum().item():
                        continue
                rs.append(rp / s)
                qs.append(Q[win])
                cs.append(c)
            plan.vcycle(u, b)
        plan.close()
    return (torch.stack(rs).contiguous(), torch.stack(qs).contiguous(), np.array(cs))


def train(net: Net, data, steps=300, batch=32, lr=1e-3, margin=4, seed=0, log_every=0):
    """Adam on random mini-batches of the patches; returns the loss history."""
    r, q, c = data
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = []
    for s in range(steps):
        idx = rng.choice(r.shape[0], size=min(batch, r.shape[0]), replace=False)
        it = torch.as_tensor(idx, device=r.device)
        loss = net.train_step(r[it].contiguous(), q[it].contiguous(), c[idx], lr, margin)
        hist.append(loss)
        if log_every and s % log_every == 0:
            print(f"step {s} loss {loss:.4f}")
    return hist
