"""Write the stored expected values under tests/golden/ from the binary128 oracle alone.

Run from the repository root: ``python tests/golden/make_golden.py``.  It imports only ``oracle`` and the
seeded input generator (which holds none of the method's arithmetic); nothing here comes from the CUDA path.

c1_d2_N100.json: the d=2, N=100, L=1, chi=0.30 workload (seed 1): its k-set (Definitions: the M smallest
half-space vectors, M = round(chi d (N-1))), Phi and S_max (Eqs. energy, structurefactor, smax), the first 16
collective densities (Eq. ntilde) and the forces on the first 8 particles (Eq. force), each value as the
(hi, lo) pair of doubles of the binary128 result.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2304_09139_b300 import synth  # noqa: E402


def c1():
    cfg = synth.SMALL_D2
    s = synth.positions(cfg.seed, cfg.N, cfg.d)
    n = oracle.kset(cfg.d, cfg.N, cfg.L, chi=cfg.chi)
    r = oracle.phi_grad(s, None, n, cfg.L, want_cs=True, nthreads=1)
    return {
        "source": "oracle (binary128), tests/golden/make_golden.py",
        "workload": {"d": cfg.d, "N": cfg.N, "L": cfg.L, "chi": cfg.chi, "seed": cfg.seed},
        "M": int(len(n)),
        "kset": n.tolist(),
        "phi": [float(x) for x in r["phi"]],
        "smax": [float(x) for x in r["smax"]],
        "C": np.asarray(r["C"][:16]).tolist(),
        "S": np.asarray(r["S"][:16]).tolist(),
        "F": np.asarray(r["F"][:8]).tolist(),
    }


def main():
    d = c1()
    with open(os.path.join(HERE, "c1_d2_N100.json"), "w") as f:     # one key per line
        f.write("{\n" + ",\n".join(f" {json.dumps(k)}: {json.dumps(v)}" for k, v in d.items()) + "\n}\n")


if __name__ == "__main__":
    main()
