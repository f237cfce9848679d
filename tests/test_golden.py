"""Stored oracle values (tests/golden/, written by tests/golden/make_golden.py from the oracle alone).

CPU: the oracle still reproduces the stored values bit for bit (guards the oracle against drift; the oracle's
own pins are in test_oracle.py).  GPU: the CUDA path in all three arithmetics against the stored values, with
the normwise bounds of the parity tests.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2304_09139_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_d2_N100.json")


def load():
    with open(GOLDEN) as f:
        return json.load(f)


def test_oracle_reproduces_golden(oracle_mod):
    g = load()
    w = g["workload"]
    s = synth.positions(w["seed"], w["N"], w["d"])
    n = oracle_mod.kset(w["d"], w["N"], w["L"], chi=w["chi"])
    assert len(n) == g["M"] == round(w["chi"] * w["d"] * (w["N"] - 1))
    assert n.tolist() == g["kset"]
    r = oracle_mod.phi_grad(s, None, n, w["L"], want_cs=True, nthreads=2)
    assert [float(x) for x in r["phi"]] == g["phi"]
    assert [float(x) for x in r["smax"]] == g["smax"]
    assert np.asarray(r["C"][:16]).tolist() == g["C"] and np.asarray(r["S"][:16]).tolist() == g["S"]
    assert np.asarray(r["F"][:8]).tolist() == g["F"]


@pytest.mark.gpu
def test_cuda_path_against_golden():
    from paper_2304_09139_b300 import _build, ssh
    _build.build()
    g = load()
    w = g["workload"]
    N, d, L = w["N"], w["d"], w["L"]
    s = synth.positions(w["seed"], N, d)
    with ssh.Context(d, N, L, chi=w["chi"]) as ctx:
        assert ctx.kset().tolist() == g["kset"]
        ctx.set_positions_frac(s)
        C_ref, S_ref = np.array(g["C"]), np.array(g["S"])
        F_ref = np.array(g["F"])
        n = np.array(g["kset"])
        for prec, tol in ((ssh.FP64, 1e-13), (ssh.DD, 1e-28), (ssh.FX, 1e-28)):
            r = ctx.energy_grad(prec)
            C, S = ctx.ntilde()
            dphi = (r["phi"][0] - g["phi"][0]) + (r["phi"][1] - g["phi"][1])
            assert abs(dphi) <= 4 * tol * max(g["phi"][0], g["M"] * N)
            sm = g["smax"][0]
            dsm = (r["smax"][0] - g["smax"][0]) + (r["smax"][1] - g["smax"][1])
            assert abs(dsm) <= 4 * tol * (2 * math.sqrt(N * sm) + 1)
            for got, ref in ((C[:16], C_ref), (S[:16], S_ref)):
                assert np.all(np.abs((got[:, 0] - ref[:, 0]) + (got[:, 1] - ref[:, 1])) <= tol * N)
            F = np.stack([r["F_hi"][:8], r["F_lo"][:8]], -1)
            # the normwise force scale needs every C, S: bound it by |C|, |S| <= N
            scale = tol * 4 * math.pi / L * np.abs(n).sum(0) * (2 * N + math.sqrt(N))
            assert np.all(np.abs((F[..., 0] - F_ref[..., 0]) + (F[..., 1] - F_ref[..., 1])) <= scale[None, :])
