"""The allocation-free collective density, ssh_ntilde_noalloc.

Callers that cannot allocate device memory use this entry point: a program that gives a GPU's memory to
another framework's pool or arena at start-up (its own cudaMalloc would fail or fragment that pool), or a
real-time loop that must not allocate after start-up (cudaMalloc and cudaFree can synchronise the device).
It takes caller-owned device inputs and outputs and keeps its own working memory in one fixed 8 MiB device
array instead of calling cudaMalloc.  These tests call it through the C ABI and compare its n~(k) with the one
from the regular entry points (ssh_create + ssh_eval(SSH_FX) + ssh_get_ntilde) on calls made back to back,
with the same tolerance as the other parity tests (1e-28 N per component), and check that the device's free
memory does not move across its calls.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [  # d, N, L, chi, seed -- different sizes so a later call cannot reuse an earlier call's scratch
    (2, 2000, 2000 ** 0.5, 0.45, 21),
    (3, 300, 300 ** (1 / 3), 0.40, 22),
    (2, 2000, 2000 ** 0.5, 0.45, 21),
]


def _reference(ssh, synth, d, N, L, chi, seed):
    s = synth.positions(seed, N, d)
    with ssh.Context(d, N, L, chi=chi) as ctx:
        ctx.set_positions_frac(s)
        ctx.eval(ssh.FX, want_force=False)
        C, S = ctx.ntilde()
        n = ctx.kset()
    return s, n, C, S


def test_noalloc_matches_regular_entry_point_on_consecutive_calls():
    import torch

    from paper_2304_09139_b300 import _build, ssh, synth
    _build.build()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    first = None
    for i, (d, N, L, chi, seed) in enumerate(CASES):
        s, n, C_ref, S_ref = _reference(ssh, synth, d, N, L, chi, seed)
        M = len(n)
        s_d = torch.tensor(s, dtype=torch.float64, device=dev).contiguous()
        n_d = torch.tensor(n, dtype=torch.int32, device=dev).contiguous()
        out = [torch.full((M,), float("nan"), dtype=torch.float64, device=dev) for _ in range(4)]
        stream = torch.cuda.current_stream(dev)
        ssh.ntilde_noalloc(d, N, M, s_d.data_ptr(), None, n_d.data_ptr(), *[o.data_ptr() for o in out],
                           stream.cuda_stream)
        torch.cuda.synchronize(dev)
        Ch, Cl, Sh, Sl = (o.cpu().numpy() for o in out)
        dC = (Ch - C_ref[:, 0]) + (Cl - C_ref[:, 1])
        dS = (Sh - S_ref[:, 0]) + (Sl - S_ref[:, 1])
        assert np.all(np.isfinite(dC)) and np.all(np.isfinite(dS)), i
        assert np.abs(dC).max() <= 1e-28 * N, (i, np.abs(dC).max())
        assert np.abs(dS).max() <= 1e-28 * N, (i, np.abs(dS).max())
        if i == 0:
            first = (Ch, Cl, Sh, Sl)
        if i == 2:   # the same input again after a different call: bit-identical
            assert all(np.array_equal(a, b) for a, b in zip(first, (Ch, Cl, Sh, Sl)))
        # allocation-free: with inputs and outputs in place, repeated calls leave the free device memory as it was
        free0 = torch.cuda.mem_get_info(dev)[0]
        for _ in range(2):
            ssh.ntilde_noalloc(d, N, M, s_d.data_ptr(), None, n_d.data_ptr(), *[o.data_ptr() for o in out],
                               stream.cuda_stream)
        torch.cuda.synchronize(dev)
        assert torch.cuda.mem_get_info(dev)[0] == free0, i


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    from paper_2304_09139_b300 import _build, ssh
    _build.build()
    with pytest.raises(ssh.SshError) as e:
        # 2e5 wavevectors x 40 bytes alone exceed the 8 MiB array; rejected before any device work
        ssh.ntilde_noalloc(2, 100, 220_000, 1, None, 1, 1, 1, 1, 1, None)
    assert e.value.status == 1
    assert "8 MiB" in str(e.value)
