"""Particle shards of one configuration (ssh_opts.shard_first / shard_count, ssh_shard_*) on one GPU, against one
unsharded context of the same configuration.

Two or three shard contexts are driven by ShardGroup, their exchanges summed in this process (the sum a NCCL
all-reduce would do across GPUs).  The shards run one after another on one stream, so no kernel of one shard waits
for another's.  Because the density partials are exact integers and each FIRE dot-product chunk belongs to one
shard, the results must agree bit for bit: Phi, S_max and every n~(k) on every shard, each shard's forces, and after
20 FIRE steps the same step count, rejections, Phi, S_max, dt and positions.
"""
import numpy as np
import pytest

from paper_2304_09139_b300 import ssh, synth
from paper_2304_09139_b300.shard import ShardGroup, shard_ranges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2304_09139_b300 import _build
    _build.build()
    import torch
    assert torch.cuda.is_available()
    return torch


def _group(torch, cfg, ranges, s, stream, tc_chunk=0):
    shards = [ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, shard=r, tc_chunk=tc_chunk) for r in ranges]
    for c in shards:
        c.set_stream(stream.cuda_stream)
        c.set_positions_frac(s)

    def alloc(n, kind):
        return torch.zeros(n, dtype=torch.int64 if kind == "i64" else torch.float64, device="cuda:0")
    return shards, ShardGroup(shards, alloc=alloc)


CASES = [  # configuration, shards, particles per chunk of the tensor-core path (0: one chunk)
    (synth.MEDIUM_D2, 2, 0),
    (synth.Config(d=3, N=6000, L=6000 ** (1 / 3), chi=0.30, seed=61), 2, 1024),
    (synth.Config(d=1, N=4500, L=4500.0, chi=0.30, seed=62), 2, 0),
    (synth.Config(d=2, N=7000, L=7000 ** 0.5, chi=0.40, seed=63), 3, 0),
]


@pytest.mark.parametrize("cfg,G,chunk", CASES, ids=["d2_N10000", "d3_N6000_chunked", "d1_N4500", "d2_N7000_3shards"])
def test_sharded_evaluation_is_bit_identical(env, cfg, G, chunk):
    torch = env
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    ref = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, tc_chunk=chunk)
    assert ref.fx_impl == ssh.FX_TENSOR
    ref.set_positions_frac(s)
    r0 = ref.energy_grad(ssh.FX)
    C0, S0 = ref.ntilde()
    ref.close()
    ranges = shard_ranges(cfg.N, G)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        shards, g = _group(torch, cfg, ranges, s, stream, chunk)
        g.eval(True)
    for (f, c), sh in zip(ranges, shards):
        r = sh.results(True)
        C, S = sh.ntilde()
        assert np.array_equal(r["phi"], r0["phi"]) and np.array_equal(r["smax"], r0["smax"])
        assert np.array_equal(C, C0) and np.array_equal(S, S0)
        assert np.array_equal(r["F_hi"][f:f + c], r0["F_hi"][f:f + c])
        assert np.array_equal(r["F_lo"][f:f + c], r0["F_lo"][f:f + c])
        assert not np.any(r["F_hi"][:f]) and not np.any(r["F_hi"][f + c:])   # other shards' particles: no force here
        sh.close()


def _fire_params(ctx):
    p = ctx.min_defaults()
    p.n_stages = 1
    p.stage_prec[0] = ssh.FX
    p.smax_target = 1e-300
    p.max_steps = 1 << 40
    p.stall_window[0] = 1 << 40
    return p


@pytest.mark.parametrize("cfg,G", [(synth.MEDIUM_D2, 2), (synth.Config(d=3, N=6000, L=6000 ** (1 / 3), chi=0.30,
                                                                      seed=61), 3)], ids=["d2_N10000", "d3_N6000"])
def test_sharded_fire_steps_are_bit_identical(env, cfg, G):
    torch = env
    steps = 20
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    ref = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    ref.set_positions_frac(s)
    ref.fire_begin(_fire_params(ref))
    ref.fire_steps(ssh.FX, steps)
    st0 = ref.fire_state()
    pos0 = ref.positions_frac()
    ref.close()
    assert st0["steps"] == steps and st0["running"]
    ranges = shard_ranges(cfg.N, G)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        shards, g = _group(torch, cfg, ranges, s, stream)
        g.fire_begin(_fire_params(shards[0]))
        g.steps(steps)
        st = g.state()
    for k in ("steps", "rejected", "smax", "phi", "dt", "running"):
        assert st[k] == st0[k], (k, st[k], st0[k])
    for (f, c), sh in zip(ranges, shards):
        hi, lo = sh.positions_frac()
        assert np.array_equal(hi[f:f + c], pos0[0][f:f + c]) and np.array_equal(lo[f:f + c], pos0[1][f:f + c])
        sh.close()


def test_shard_context_rules(env):
    cfg = synth.MEDIUM_D2
    with pytest.raises(ssh.SshError):      # boundaries must lie on multiples of 2048
        ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, shard=(1000, 3000))
    with pytest.raises(ssh.SshError):      # the integer pipes do not shard
        ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, shard=(0, 4096), fx_impl=ssh.FX_INTEGER)
    sh = ssh.Context(cfg.d, cfg.N, cfg.L, chi=cfg.chi, shard=(0, 4096))
    sh.set_positions_frac(synth.positions(cfg.seed, cfg.N, cfg.d))
    for call in (lambda: sh.energy_grad(ssh.FX), lambda: sh.minimize(check=True), lambda: sh.eval(ssh.FX)):
        with pytest.raises(ssh.SshError) as e:
            call()
        assert e.value.status == 1
    with pytest.raises(ssh.SshError):      # no FIRE run begun
        sh.shard_step_dots(1)
    sh.close()
