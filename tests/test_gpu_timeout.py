"""Failure detection of the tensor-core GEMM: a bounded wait that runs out is reported, never trapped.

Every wait of k_tc_gemm on its pipeline has a limit (ssh_set_wait_limit).  These tests set it to one clock
cycle, far below any real wait, so that waits give up.  The kernel then skips its remaining work, lets its copies
and MMAs in flight land and returns, and the host must report SSH_ETIMEOUT: for one evaluation, for a whole
minimisation and for a batch.  A failed step is undone, and once the limit is restored the context gives the
same bits as before the failure.  Nothing here faults or hangs the GPU: the kernel returns in every case.
"""
import numpy as np
import pytest

from paper_2304_09139_b300 import ssh, synth

pytestmark = pytest.mark.gpu
ETIMEOUT = 6


@pytest.fixture(scope="module")
def built():
    from paper_2304_09139_b300 import _build
    _build.build()
    import torch
    assert torch.cuda.is_available()
    yield True
    ssh.set_wait_limit(0)


def _ctx(cfg):
    ctx = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, fx_impl=ssh.FX_TENSOR)
    ctx.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
    return ctx


def test_evaluation_reports_a_wait_that_ran_out(built):
    cfg = synth.Config(d=2, N=2000, L=2000 ** 0.5, chi=0.45, seed=31)
    ctx = _ctx(cfg)
    r0 = ctx.energy_grad(ssh.FX)
    try:
        ssh.set_wait_limit(1)
        with pytest.raises(ssh.SshError) as e:
            ctx.energy_grad(ssh.FX)
        assert e.value.status == ETIMEOUT
    finally:
        ssh.set_wait_limit(0)
    # the failure was reported once; the context is usable and gives the same bits again
    r1 = ctx.energy_grad(ssh.FX)
    for key in ("phi", "smax", "F_hi", "F_lo"):
        assert np.array_equal(r0[key], r1[key]), key


@pytest.mark.parametrize("method", [ssh.MIN_FIRE, ssh.MIN_LBFGS], ids=["fire", "lbfgs"])
def test_minimiser_stops_on_a_wait_that_ran_out(built, method):
    cfg = synth.SMALL_D2
    ctx = _ctx(cfg)
    s0 = ctx.positions_frac()
    try:
        ssh.set_wait_limit(1)
        r = ctx.minimize(stages=[ssh.FX], method=method, max_steps=200)
    finally:
        ssh.set_wait_limit(0)
    assert r["status"] == ETIMEOUT, r
    s1 = ctx.positions_frac()   # the failing evaluation came first: nothing moved
    assert np.array_equal(s0[0], s1[0]) and np.array_equal(s0[1], s1[1])
    r = ctx.minimize(stages=[ssh.FX], method=method, max_steps=20000)
    assert r["status"] == 0 and r["smax"][0] <= 1e-36, r


def test_batch_member_reports_a_wait_that_ran_out(built):
    b = ssh.Batch(fx_impl=ssh.FX_TENSOR)
    for seed in (41, 42):
        cfg = synth.Config(d=2, N=300, L=300 ** 0.5, chi=0.30, seed=seed)
        b.add(cfg.d, cfg.N, cfg.L, synth.positions(cfg.seed, cfg.N, cfg.d), chi=cfg.chi)
    try:
        ssh.set_wait_limit(1)
        st, res = b.minimize(stages=[ssh.FX], max_steps=100)
    finally:
        ssh.set_wait_limit(0)
    assert st == ETIMEOUT
    assert all(r["status"] == ETIMEOUT for r in res), res


def test_gemm_counters_instance_gives_the_same_bits():
    """The counting instance of the tensor-core GEMM (ssh_gemm_counters) computes the same integers as the
    production instance, so Phi, S_max, n~ and F agree bit for bit, with the counters on and after they are off;
    its records are consistent (every CTA that ran wrote items and K-steps, the MMA thread's waits fit inside its
    cycles and those inside the CTA's)."""
    from paper_2304_09139_b300 import _build, ssh, synth
    _build.build()
    cfg = synth.MEDIUM_D2
    with ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi) as ctx:
        ctx.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
        a = ctx.energy_grad(ssh.FX)
        Ca, Sa = ctx.ntilde()
        ssh.gemm_counters(True)
        try:
            b = ctx.energy_grad(ssh.FX)
            Cb, Sb = ctx.ntilde()
            rec = ssh.gemm_counters_read()
        finally:
            ssh.gemm_counters(False)
        c = ctx.energy_grad(ssh.FX)
    for x in (b, c):
        assert np.array_equal(a["phi"], x["phi"]) and np.array_equal(a["smax"], x["smax"])
        assert np.array_equal(a["F_hi"], x["F_hi"]) and np.array_equal(a["F_lo"], x["F_lo"])
    assert np.array_equal(Ca, Cb) and np.array_equal(Sa, Sb)
    f = {n: i for i, n in enumerate(ssh.GEMM_COUNTER_FIELDS)}
    for kind in (0, 1):
        r = rec[kind][rec[kind][:, f["cycles"]] > 0].astype(np.int64)
        assert len(r) > 0
        assert np.all(r[:, f["ksteps"]] > 0) and np.all(r[:, f["items"]] > 0)
        waits = r[:, f["mma_wait_operands"]] + r[:, f["mma_wait_accumulator"]] + r[:, f["mma_wait_item"]]
        assert np.all(waits <= r[:, f["mma_thread_cycles"]]) and np.all(r[:, f["mma_thread_cycles"]] <= r[:, f["cycles"]])
        assert np.all(r[:, f["t1_ns"]] >= r[:, f["t0_ns"]])
