"""Host-side post-processing (no GPU): the library's g_2 normalisation (ssh_g2, host arithmetic over the bins)
against the oracle's binary128 one, on counts of known structure."""
import numpy as np

import oracle
from paper_2304_09139_b300 import ssh, synth


def test_g2_matches_the_oracle():
    """ssh_g2 and the oracle's g_2 agree to double rounding in d = 1..4, on exact pair counts of uniform points
    and on arbitrary counts (empty bins included)."""
    oracle.build()
    for d in (1, 2, 3, 4):
        N = 1500
        L = N ** (1 / d)
        if d <= 3:
            counts = oracle.pair_histogram(synth.positions(40 + d, N, d), L, 300, 0.4 * L, 12)
        else:
            counts = np.array([0, 3, 17, 250, 1, 0, 999, 12345, 7, 2, 0, 5], dtype=np.uint64)
        r, g = ssh.g2(counts, d, N, L, 300, 0.4 * L)
        r_o, g_o = oracle.g2(counts, d, N, L, 300, 0.4 * L)
        assert np.allclose(r, r_o, rtol=1e-15, atol=0)
        assert np.allclose(g, g_o, rtol=1e-13, atol=0), (d, g, g_o)


def test_g2_rejects_bad_arguments():
    for args in ((0, 10, 1.0, 1, 0.4), (2, 1, 1.0, 1, 0.4), (2, 10, 1.0, 11, 0.4), (2, 10, 1.0, 1, 0.0)):
        try:
            ssh.g2(np.zeros(4, dtype=np.uint64), *args)
        except ssh.SshError as e:
            assert e.status == 1
        else:
            raise AssertionError(args)
