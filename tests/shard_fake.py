"""A CPU stand-in for a particle-shard context (a test double, not part of the library): the shard_* methods of
ssh.Context with the same exchange contract, so that ShardGroup and its Comm can run on gloo ranks without a GPU.

It keeps the properties the real shards rely on:
  * the density partial is exact integers (each phasor rounded to 2^-40 and summed in int64), so the element-wise
    sum over shards equals one context's sum over every particle in any order;
  * the dot products F.v, F.F, v.v are partial sums per chunk of 2048 particles of one axis, exactly 0 for chunks
    outside the shard (their force and velocity stay 0), so their sum over shards is exact;
  * every shard holds all N positions but moves and forces only its own.
The arithmetic is plain binary64 FIRE (Bitzek et al. 2006) with the energy guard: it exercises the exchanges and
the call order, not the library's precision.
"""
import math

import numpy as np
import torch

SCALE = 2.0 ** 40
CHUNK = 2048


class FakeShard:
    def __init__(self, s, n, L, first, count):
        self.s = np.array(s, dtype=np.float64).copy()
        self.N, self.d = self.s.shape
        self.n = np.asarray(n, dtype=np.int64)
        self.M = len(self.n)
        self.L = float(L)
        self.loc = slice(first, first + count)
        self.F = np.zeros_like(self.s)
        self.v = np.zeros_like(self.s)
        self.nq1 = math.ceil(self.N / CHUNK)
        self.phi = self.smax = None
        self.st = None

    def shard_words(self):
        return 2 * self.M, 3 * self.d * self.nq1

    def _density(self, out):
        th = 2 * math.pi * (self.s[self.loc] @ self.n.T)
        out[:self.M] = torch.from_numpy(np.rint(np.cos(th) * SCALE).astype(np.int64).sum(0))
        out[self.M:] = torch.from_numpy(np.rint(np.sin(th) * SCALE).astype(np.int64).sum(0))

    def shard_density(self, out):
        self._density(out)

    def shard_finish(self, tot, want_force=True):
        t = tot.numpy()
        C, S = t[:self.M] / SCALE, t[self.M:] / SCALE
        a2 = C * C + S * S
        self.phi, self.smax = float(a2.sum()), float(a2.max() / self.N)
        if want_force:
            th = 2 * math.pi * (self.s[self.loc] @ self.n.T)
            self.F[:] = 0.0
            self.F[self.loc] = 4 * math.pi / self.L * ((C * np.sin(th) - S * np.cos(th)) @ self.n)

    def shard_fire_begin(self, params=None, dt0=0.01, **kw):
        self.st = {"dt": dt0, "dt_max": 10 * dt0, "alpha": 0.1, "n_pos": 0, "steps": 0, "rejected": 0,
                   "phi": self.phi, "smax": self.smax, "cv": 0.0, "cf": 0.0, "zero_v": True}
        self.v[:] = 0.0

    def shard_step_dots(self, out):
        part = np.zeros((3, self.d * self.nq1))
        for a in range(self.d):
            for jb in range(self.nq1):
                j0, j1 = jb * CHUNK, min(self.N, (jb + 1) * CHUNK)
                f, w = self.F[j0:j1, a], self.v[j0:j1, a]
                part[:, a * self.nq1 + jb] = (np.dot(f, w), np.dot(f, f), np.dot(w, w))
        out[:] = torch.from_numpy(part.reshape(-1))

    def shard_step_move(self, tot, out):
        st = self.st
        P, f2, v2 = (math.fsum(x) for x in tot.numpy().reshape(3, -1))
        if P > 0:
            st["zero_v"], st["cv"] = False, 1.0 - st["alpha"]
            st["cf"] = st["alpha"] * math.sqrt(v2) / math.sqrt(f2) if f2 > 0 else 0.0
            if st["n_pos"] > 5:
                st["dt"] = min(st["dt"] * 1.1, st["dt_max"])
                st["alpha"] *= 0.99
            st["n_pos"] += 1
        else:
            st.update(zero_v=True, cv=0.0, cf=0.0, dt=st["dt"] * 0.5, alpha=0.1, n_pos=0)
        self._saved = (self.s.copy(), self.F.copy())
        v = np.zeros_like(self.v) if st["zero_v"] else st["cv"] * self.v + st["cf"] * self.F
        self.v = v + st["dt"] * self.F
        self.s[self.loc] = np.mod(self.s[self.loc] + st["dt"] * self.v[self.loc] / self.L, 1.0)
        self._density(out)

    def shard_step_finish(self, tot):
        st = self.st
        self.shard_finish(tot, True)
        st["steps"] += 1
        if self.phi > st["phi"]:
            st["rejected"] += 1
            self.s, self.F = self._saved
            self.v[:] = 0.0
            st.update(dt=st["dt"] * 0.5, alpha=0.1, n_pos=0)
        else:
            st["phi"], st["smax"] = self.phi, self.smax

    def fire_state(self):
        st = self.st
        return {"steps": st["steps"], "rejected": st["rejected"], "smax": [st["smax"], 0.0], "phi": [st["phi"], 0.0],
                "dt": st["dt"], "running": True}
