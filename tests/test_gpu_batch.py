"""Batched evaluation and minimisation of many configurations, and the continuous-batching server.

Every configuration keeps its own launch shape and is skipped by every kernel once its run ends, so its
arithmetic does not depend on what else is in the batch: results must be bit-identical alone and in the mix
(n~, Phi, F of one evaluation; steps, S_max and final positions of a whole quench).  Quenches are judged by
S_max <= 1e-36, confirmed by the binary128 oracle on some members.
"""
import math
import os
import time

import numpy as np
import pytest

from conftest import launches_per_role
from paper_2304_09139_b300 import ssh, synth

pytestmark = pytest.mark.gpu
NTHREADS = os.cpu_count() or 8


@pytest.fixture(scope="module")
def built():
    from paper_2304_09139_b300 import _build
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return True


def small_mix(count, seed, n_lo=64, n_hi=400, dims=(2, 3)):
    return synth.mixed_batch(seed, count, n_lo=n_lo, n_hi=n_hi, dims=dims)


@pytest.mark.parametrize("impl", [ssh.FX_AUTO, ssh.FX_INTEGER], ids=["auto", "int"])
def test_batched_evaluation_equals_single(built, impl):
    cfgs = small_mix(7, 41) + [synth.Config(d=1, N=300, L=300.0, chi=0.3, seed=9),
                              synth.Config(d=2, N=2000, L=2000 ** 0.5, chi=0.45, seed=10)]
    b = ssh.Batch(fx_impl=impl)
    for c in cfgs:
        b.add(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi)
    n, pairs = b.size()
    assert n == len(cfgs) and pairs > 0
    for prec in (ssh.FP64, ssh.DD, ssh.FX):
        b.eval(prec)
        for i, c in enumerate(cfgs):
            rb = b.member(i).results()
            Cb, Sb = b.member(i).ntilde()
            with ssh.Context(c.d, c.N, c.L, chi=c.chi, fx_impl=impl) as ctx:
                ctx.set_positions_frac(synth.positions(c.seed, c.N, c.d))
                ra = ctx.energy_grad(prec)
                Ca, Sa = ctx.ntilde()
            assert np.array_equal(ra["phi"], rb["phi"]) and np.array_equal(ra["smax"], rb["smax"]), (prec, i)
            assert np.array_equal(ra["F_hi"], rb["F_hi"]) and np.array_equal(ra["F_lo"], rb["F_lo"]), (prec, i)
            assert np.array_equal(Ca, Cb) and np.array_equal(Sa, Sb), (prec, i)
    b.close()


def test_tensor_members_equal_single(built):
    """A batch of d = 1..4 members on the tensor cores: every member bit-identical to a lone context, in an
    evaluation and a quench."""
    cfgs = small_mix(6, 46, dims=(1, 2, 3)) + [synth.Config(d=2, N=2000, L=2000 ** 0.5, chi=0.45, seed=11),
                                              synth.Config(d=4, N=120, L=120 ** 0.25, chi=0.3, seed=12)]
    b = ssh.Batch(fx_impl=ssh.FX_TENSOR)
    for c in cfgs:
        b.add(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi)
    b.eval(ssh.FX)
    for i, c in enumerate(cfgs):
        impl = ssh.FX_TENSOR
        assert b.member(i).fx_impl == impl
        rb = b.member(i).results()
        with ssh.Context(c.d, c.N, c.L, chi=c.chi, fx_impl=impl) as ctx:
            ctx.set_positions_frac(synth.positions(c.seed, c.N, c.d))
            ra = ctx.energy_grad(ssh.FX)
        assert np.array_equal(ra["phi"], rb["phi"]) and np.array_equal(ra["F_hi"], rb["F_hi"]), i
        assert np.array_equal(ra["F_lo"], rb["F_lo"]), i
    st, res = b.minimize(max_steps=40000, chunk_steps=16)
    assert st == 0, res
    for i, c in enumerate(cfgs):
        assert res[i]["status"] == 0 and res[i]["smax"][0] <= 1e-36, (i, res[i])
    b.close()


def test_batched_quench_equals_single_and_converges(built, oracle_mod):
    cfgs = small_mix(10, 43)
    b = ssh.Batch()
    for c in cfgs:
        b.add(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi)
    st, res = b.minimize(max_steps=40000, chunk_steps=16)
    assert st == 0, res
    for i, c in enumerate(cfgs):
        assert res[i]["status"] == 0 and res[i]["smax"][0] <= 1e-36, (i, res[i])
        hb, lb = b.member(i).positions_frac()
        with ssh.Context(c.d, c.N, c.L, chi=c.chi) as ctx:
            ctx.set_positions_frac(synth.positions(c.seed, c.N, c.d))
            ra = ctx.minimize(max_steps=40000)
            ha, la = ctx.positions_frac()
        assert ra["steps"] == res[i]["steps"] and ra["smax"] == res[i]["smax"], (i, ra, res[i])
        assert np.array_equal(ha, hb) and np.array_equal(la, lb), i
        if i < 3:
            r = oracle_mod.phi_grad(hb, lb, b.member(i).kset(), c.L, want_force=False, nthreads=NTHREADS)
            assert r["smax"][0] + r["smax"][1] <= 1.01e-36
    b.close()


def test_batch_stepper_runs_exact_steps(built):
    cfgs = small_mix(5, 44)
    b = ssh.Batch()
    for c in cfgs:
        b.add(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi)
    b.begin(stages=[ssh.FX], smax_target=1e-300)
    b.steps(10)
    b.prof_enable(True)
    b.steps(3)
    pr = b.prof_read()
    b.prof_enable(False)
    assert pr["fire"][1] == 6
    for role in ("density", "force"):   # one launch per step of each implementation present
        counts = launches_per_role(pr, role)
        assert counts and all(n == 3 for n in counts), (role, pr)
    b.close()


def test_server_continuous_batching(built):
    """Requests arrive while others run; each is admitted, converges, and ends bit-identical to a lone quench."""
    cfgs = small_mix(12, 45, dims=(1, 2, 3))
    sv = ssh.Server(max_slots=5, chunk_steps=16)
    tickets = []
    for i, c in enumerate(cfgs):
        tickets.append(sv.submit(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi, want_positions=True))
        time.sleep(0.01 if i % 3 else 0.05)
    deadline = time.time() + 300
    done = {}
    overlap = False
    while len(done) < len(tickets) and time.time() < deadline:
        s = sv.stats()
        overlap = overlap or s["running"] >= 2
        assert s["running"] <= 5
        for t in tickets:
            if t not in done:
                r = sv.poll(t)
                if r is not None:
                    done[t] = r
        time.sleep(0.01)
    assert len(done) == len(tickets)
    assert overlap   # several requests were on the GPU at once
    lat = []
    for t, c in zip(tickets, cfgs):
        r = done[t]
        assert r["status"] == 0 and r["smax"][0] <= 1e-36, r
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        lat.append(r["t_done"] - r["t_submit"])
        hs, ls = sv.positions(t)
        with ssh.Context(c.d, c.N, c.L, chi=c.chi) as ctx:
            ctx.set_positions_frac(synth.positions(c.seed, c.N, c.d))
            ra = ctx.minimize()
            ha, la = ctx.positions_frac()
        assert ra["steps"] == r["steps"], (ra, r)
        assert np.array_equal(ha, hs) and np.array_equal(la, ls)
        sv.release(t)
    assert np.percentile(lat, 99) >= np.percentile(lat, 50) > 0
    with pytest.raises(ssh.SshError):
        sv.poll(tickets[0])       # released
    sv.close()


def test_server_admission_by_memory_budget_and_cancel(built):
    c = synth.Config(d=2, N=400, L=20.0, chi=0.4, seed=3)
    s = synth.positions(c.seed, c.N, c.d)
    sv = ssh.Server(max_slots=64, hbm_budget_bytes=6 << 20, chunk_steps=8)   # room for only a few at a time
    ts = [sv.submit(c.d, c.N, c.L, s, chi=c.chi) for _ in range(8)]
    extra = sv.submit(c.d, c.N, c.L, s, chi=c.chi)
    try:
        sv.cancel(extra)
        cancelled = True
    except ssh.SshError:
        cancelled = False   # already admitted: allowed
    peak = 0
    deadline = time.time() + 240
    while time.time() < deadline:
        st = sv.stats()
        peak = max(peak, st["running"])
        assert st["hbm_used_bytes"] <= 6 << 20 or st["running"] == 1
        if all(sv.poll(t) is not None for t in ts):
            break
        time.sleep(0.01)
    assert all(sv.poll(t)["status"] == 0 for t in ts)
    assert 1 <= peak < 8
    if cancelled:
        with pytest.raises(ssh.SshError):
            sv.poll(extra)
    with pytest.raises(ssh.SshError):     # larger than the whole budget
        big = synth.Config(d=2, N=20000, L=20000 ** 0.5, chi=0.45, seed=4)
        sv.submit(big.d, big.N, big.L, synth.positions(4, big.N, 2), chi=big.chi)
    sv.close()


def test_batched_lbfgs_equals_single(built):
    """A batch quenched with L-BFGS: each member's quench is bit-identical to a lone run (fixed-order reductions
    everywhere, so a member's arithmetic does not depend on the batch)."""
    cfgs = small_mix(6, 47, dims=(1, 2, 3))
    b = ssh.Batch()
    for c in cfgs:
        b.add(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi)
    st, res = b.minimize(max_steps=40000, chunk_steps=16, method=ssh.MIN_LBFGS)
    assert st == 0, res
    for i, c in enumerate(cfgs):
        assert res[i]["status"] == 0 and res[i]["smax"][0] <= 1e-36, (i, res[i])
        hb, lb = b.member(i).positions_frac()
        with ssh.Context(c.d, c.N, c.L, chi=c.chi) as ctx:
            ctx.set_positions_frac(synth.positions(c.seed, c.N, c.d))
            ra = ctx.minimize(method=ssh.MIN_LBFGS, max_steps=40000)
            ha, la = ctx.positions_frac()
        assert ra["steps"] == res[i]["steps"] and ra["smax"] == res[i]["smax"], (i, ra, res[i])
        assert np.array_equal(ha, hb) and np.array_equal(la, lb), i
    b.close()


def test_autotune_keeps_results_and_remembers(built):
    """The batch autotuner times every candidate decomposition of the tensor-core GEMMs, keeps one, and the
    batch's evaluations stay bit-identical (only the order of exact integer sums changes); a second call on the
    same member shapes reuses the remembered choice."""
    cfgs = small_mix(12, 47, dims=(1, 2, 3)) + [synth.Config(d=2, N=3000, L=3000 ** 0.5, chi=0.45, seed=13)]
    b = ssh.Batch()
    for c in cfgs:
        b.add(c.d, c.N, c.L, synth.positions(c.seed, c.N, c.d), chi=c.chi)
    b.eval(ssh.FX)
    before = [(b.member(i).results(), b.member(i).ntilde()) for i in range(len(cfgs))]
    t = b.autotune(ssh.FX, reps=3)
    assert t["candidates"] == 8 and t["dens_pieces_pct"] in (50, 100, 200, 400) and t["force_bundles"] in (0, 1)
    assert 0 < t["ms_tuned"] <= t["ms_default"]
    b.eval(ssh.FX)
    for i in range(len(cfgs)):
        ra, (Ca, Sa) = before[i]
        rb = b.member(i).results()
        Cb, Sb = b.member(i).ntilde()
        for k in ("phi", "smax", "F_hi", "F_lo"):
            assert np.array_equal(ra[k], rb[k]), (i, k)
        assert np.array_equal(Ca, Cb) and np.array_equal(Sa, Sb), i
    t2 = b.autotune(ssh.FX, reps=2)
    assert t2["candidates"] == 0 and (t2["dens_pieces_pct"], t2["force_bundles"]) == (t["dens_pieces_pct"], t["force_bundles"])
    # batched steps run with the tuned decomposition and still converge
    st, r = b.minimize(stages=[ssh.FX], max_seconds=120)
    assert all(x["status"] == 0 for x in r), r
    b.close()
