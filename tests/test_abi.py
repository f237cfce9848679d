"""Host-side checks of the C ABI (no GPU): the library loads, exports every entry point that
include/ssh.h declares, rejects bad arguments, and builds the same wavevector set as the oracle,
bit for bit (Definitions: k = 2 pi n / L, inversion symmetry, chi = M / (d (N - 1)))."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_2304_09139_b300 import _build, ssh, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ssh.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ssh_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n   # ctypes resolves the symbol or raises AttributeError
    assert ssh.version().startswith("ssh ")


@pytest.mark.parametrize("d,N,L,chi,K", [
    (2, 100, 1.0, 0.30, 0.0), (2, 10_000, 100.0, 0.45, 0.0), (3, 32_768, 32.0, 0.40, 0.0),
    (1, 500, 500.0, 0.2, 0.0), (1, 64, 64.0, 0.49, 0.0), (4, 300, 300 ** 0.25, 0.3, 0.0),
    (2, 10, 1.0, 0.0, 2 * math.pi * math.sqrt(50)), (3, 10, 2.0, 0.0, 2 * math.pi * 3.0 / 2.0),
    (2, 7, 3.0, 0.11, 0.0)])
def test_kset_bit_exact_against_oracle(lib, oracle_mod, d, N, L, chi, K):
    a = ssh.kset_build(d, N, L, chi=chi, K=K)
    b = oracle_mod.kset(d, N, L, chi=chi, K=K)
    assert a.dtype == b.dtype and a.shape == b.shape
    assert np.array_equal(a, b)


def test_kset_bit_exact_on_batched_and_serving_mixes(lib, oracle_mod):
    cfgs = synth.mixed_batch(4, 256)[:40] + synth.serving_requests(5, 60)[0][:40]
    for c in cfgs:
        assert np.array_equal(ssh.kset_build(c.d, c.N, c.L, chi=c.chi), oracle_mod.kset(c.d, c.N, c.L, chi=c.chi)), c


@pytest.mark.parametrize("args", [(0, 10, 1.0, 0.3, 0.0), (5, 10, 1.0, 0.3, 0.0), (2, 0, 1.0, 0.3, 0.0),
                                  (2, 10, -1.0, 0.3, 0.0), (2, 10, 1.0, 0.3, 2.0), (2, 10, 1.0, 0.0, 0.0),
                                  (2, 10, float("nan"), 0.3, 0.0)])
def test_kset_rejects_bad_arguments(lib, args):
    with pytest.raises(ssh.SshError) as e:
        ssh.kset_build(*args[:3], chi=args[3], K=args[4])
    assert e.value.status == 1
    assert lib.ssh_last_error()


def test_kset_buffer_too_small_reports_m(lib):
    M = ctypes.c_int64(0)
    buf = (ctypes.c_int32 * 4)()
    st = lib.ssh_kset_build(2, 100, 1.0, 0.3, 0.0, 2, buf, ctypes.byref(M))
    assert st == 1 and M.value == 59


@pytest.mark.parametrize("d,N,L,w,chi,K", [
    (2, 500, 500 ** 0.5, (1, 3), 0.3, 0.0), (2, 2000, 2000 ** 0.5, (4, 1), 0.45, 0.0),
    (3, 400, 400 ** (1 / 3), (1, 2, 5), 0.3, 0.0), (1, 300, 300.0, (3,), 0.4, 0.0),
    (4, 200, 200 ** 0.25, (1, 1, 2, 3), 0.2, 0.0), (2, 10, 1.0, (1, 1), 0.0, 2 * math.pi * math.sqrt(30.5)),
    (3, 10, 2.0, (2, 1, 3), 0.0, 2 * math.pi * math.sqrt(40.5) / 2.0)])
def test_region_bit_exact_against_bruteforce(lib, oracle_mod, d, N, L, w, chi, K):
    """Anisotropic exclusion regions sum_a w_a n_a^2 <= R^2 (the paper's other region shapes): the library's set
    equals the oracle's brute-force enumeration, order included; all weights 1 gives the ball's set."""
    a = ssh.kset_region(d, N, L, w, chi=chi, K=K)
    b = oracle_mod.kset_region(d, N, L, w, chi=chi, K=K)
    assert a.shape == b.shape and np.array_equal(a, b)
    if chi > 0:
        assert np.array_equal(ssh.kset_region(d, N, L, (1,) * d, chi=chi), oracle_mod.kset(d, N, L, chi=chi))


def test_create_kset_rejects_bad_lists(lib):
    good = np.array([[1, 0], [0, 1], [1, 1]], dtype=np.int32)
    for bad in (np.array([[1, 0], [-1, 0]]), np.array([[1, 0], [1, 0]]), np.array([[0, 0]]),
                np.array([[0, -2]]), np.array([[40000, 1]])):
        n = np.ascontiguousarray(bad, dtype=np.int32)
        h = ctypes.c_void_p()
        st = lib.ssh_create_kset(2, 10, 1.0, n.shape[0], n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None,
                                 ctypes.byref(h))
        assert st == 1 and not h.value, bad
    assert good.shape == (3, 2)
    with pytest.raises(ssh.SshError):
        ssh.kset_region(2, 10, 1.0, (0, 1), chi=0.3)
