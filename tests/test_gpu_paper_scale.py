"""The paper's system size on the tensor-core path: d = 2, N = 2 x 10^6 at unit density, chi = 0.10
(M = 400000, 8 x 10^11 pairs per sum), in the launch configuration of a plain evaluation.

The oracle cannot sum every pair at this size, so (Eqs. ntilde, energy and force of arXiv:2304.09139):
  - n~ on 48 sampled wavevectors against the binary128 oracle, each a full sum over the 2 x 10^6 particles,
    within |dC|, |dS| <= 1e-28 N;
  - Phi against the sum of |n~|^2 over the library's own (C, S) (the reduction), and S_max against their
    largest |n~|^2 / N;
  - F against the integer-pipe implementation (checked against the oracle at the smaller sizes) within the
    normwise bound, and sum_j F_j = 0.
"""
import math
import os

import numpy as np
import pytest

from paper_2304_09139_b300 import ssh, synth

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 8
TOL = 1e-28


def ddv(x):
    return x[..., 0] + x[..., 1]


def ddiff(a, b):
    return (a[..., 0] - b[..., 0]) + (a[..., 1] - b[..., 1])


@pytest.fixture(scope="module")
def built():
    from paper_2304_09139_b300 import _build
    _build.build()
    ssh.load()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return True


def test_paper_scale_d2_sampled(built, oracle_mod):
    cfg = synth.PAPER_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    res = {}
    for impl in (ssh.FX_TENSOR, ssh.FX_INTEGER):
        ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, fx_impl=impl)
        assert ctx.fx_impl == impl
        n = ctx.kset()
        assert ctx.M == 400_000
        ctx.set_positions_frac(s)
        r = ctx.energy_grad(ssh.FX)
        C, S = ctx.ntilde()
        res[impl] = (r, C, S)
        ctx.close()
    N = cfg.N
    rng = np.random.default_rng(2_000_000)
    pick = np.sort(np.concatenate([[0, len(n) - 1], rng.choice(np.arange(1, len(n) - 1), 46, replace=False)]))
    Cr, Sr = oracle_mod.ntilde(s, None, n[pick], nthreads=NTHREADS)
    for impl, (r, C, S) in res.items():
        assert np.all(np.abs(ddiff(C[pick], Cr)) <= TOL * N), (impl, np.abs(ddiff(C[pick], Cr)).max())
        assert np.all(np.abs(ddiff(S[pick], Sr)) <= TOL * N), (impl, np.abs(ddiff(S[pick], Sr)).max())
    (rt, Ct, St), (ri, Ci, Si) = res[ssh.FX_TENSOR], res[ssh.FX_INTEGER]
    assert np.all(np.abs(ddiff(Ct, Ci)) <= 2 * TOL * N) and np.all(np.abs(ddiff(St, Si)) <= 2 * TOL * N)
    # the reduction: Phi = sum |n~|^2 and S_max = max |n~|^2 / N over the returned (C, S)
    a2 = ddv(Ct) ** 2 + ddv(St) ** 2
    phi, smax = float(rt["phi"].sum()), float(rt["smax"].sum())
    assert abs(phi - math.fsum(a2)) <= 1e-12 * phi
    assert abs(smax - a2.max() / N) <= 1e-12 * smax
    # the force of the two implementations, and sum_j F_j = 0
    Cabs = np.abs(ddv(Ci)) + np.abs(ddv(Si)) + math.sqrt(N)
    scale = TOL * 4 * math.pi / cfg.L * (np.abs(n).astype(np.float64) * Cabs[:, None]).sum(0)
    Ft = np.stack([rt["F_hi"], rt["F_lo"]], -1)
    Fi = np.stack([ri["F_hi"], ri["F_lo"]], -1)
    assert np.all(np.abs(ddiff(Ft, Fi)) <= 2 * scale[None, :]), (np.abs(ddiff(Ft, Fi)) / scale[None, :]).max()
    for F in (Ft, Fi):
        tot = np.array([math.fsum(np.concatenate([F[:, a, 0], F[:, a, 1]])) for a in range(cfg.d)])
        assert np.all(np.abs(tot) <= N * scale * 4), (tot, scale)
