"""Host-side check of the dd phase reduction and sincos (csrc/dd.cuh is compiled for host and device).

The phase of k at fractional position s is frac(n.s) turns; the dd kernels reduce m (sh + sl) exactly
(TwoProd, then removal of the integer part by TwoSum) and evaluate e^{2 pi i t} from two 256-entry tables
and a Taylor series.  Compared with mpmath at 50 digits over random multipliers of both signs, positions
with full-mantissa bits and non-zero low words, and edge cases at 0, 1 and just below integers.
"""
import os
import random
import subprocess
import tempfile

import mpmath
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def harness():
    subprocess.run([os.sys.executable, os.path.join(ROOT, "paper_2304_09139_b300", "csrc", "gen_tables.py"),
                    os.path.join(ROOT, "paper_2304_09139_b300", "csrc", "gen", "tables.h")], check=True)
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "dd_host_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(HERE, "dd_host_check.cpp")], check=True)
    return exe


def test_dd_phase_and_sincos_against_mpmath(harness):
    mpmath.mp.dps = 50
    rnd = random.Random(7)
    cases = []
    for _ in range(4000):
        m = rnd.choice([-96, -64, -33, -32, -7, -1, 0, 1, 2, 3, 31, 32, 64, 95])
        sh = rnd.random() ** rnd.choice([1, 3, 9])
        sl = rnd.choice([0.0, (rnd.random() - 0.5) * 2.0 ** -53 * sh])
        cases.append((m, float(sh), float(sl)))
    cases += [(1, 0.0, -1e-20), (1, 1.0, -1e-20), (-32, 0.01, 0.0), (3, 1 / 3, -1e-17), (-1, 0.3, 0.0),
              (7, 0.5, 0.0), (-5, 0.2, -2e-17), (64, 2.0 ** -60, 0.0)]
    inp = "\n".join(f"{m} {sh.hex()} {sl.hex()}" for m, sh, sl in cases)
    out = subprocess.run([harness], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    worst = 0.0
    for (m, sh, sl), line in zip(cases, out):
        a = [float.fromhex(x) for x in line.split()]
        t = mpmath.mpf(m) * (mpmath.mpf(sh) + mpmath.mpf(sl))
        c, s = mpmath.cos(2 * mpmath.pi * t), mpmath.sin(2 * mpmath.pi * t)
        err = max(abs(mpmath.mpf(a[0]) + a[1] - c), abs(mpmath.mpf(a[2]) + a[3] - s))
        bound = 2.0 ** -104 * 2 * 3.1416 * (abs(m) + 4)   # dd rounding of the phase, plus the tables
        assert err <= bound, (m, sh, sl, float(err))
        worst = max(worst, float(err))
    assert worst < 2e-30
