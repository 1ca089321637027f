"""Sample maintenance under edge updates, sequential reference semantics.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Algorithm 2 (BSM) and Algorithm 3 (ISM) of Sec. 4, one edge update at
a time, with the readings listed in the design notes:

* R(u, v) is the effective resistance in the graph that contains (u, v),
  exact here (dense FP64 solve) unless given;
* ceil(R |S|) trees are chosen uniformly without replacement (Floyd's method on
  the Philox select stream);
* BSM insert replaces each chosen tree by a uniform tree of G' conditioned on
  containing (u, v), re-rooted at r; BSM delete replaces every tree containing
  (u, v) by a fresh tree of G'.  Replacement trees take new sample ids in
  increasing pool index order and keep the weight slot of the tree they replace;
* ISM insert applies link-cut with weight w' = w d(tau)/d(tau'); the chosen group
  is rescaled to total R W and the rest to (1 - R) W, W the total weight before
  the update (Algorithm 3 normalisation); ISM delete applies cut-link with
  w' = w d(tau_old)/d(tau_new) (Theorem 7's orientation) and rescales the
  updated group to its former total w_org;
* f of untouched trees is left as computed on the old graph (STALE, the BSM
  theorem's proof) unless `refresh` recomputes every f on G';
* deleting an edge of tau0 rebuilds tau0 as the BFS tree of G' from the same
  root and recomputes every f;
* K_hat = sum w f / (2m sum w) with the current m.
"""
from __future__ import annotations

import math

import numpy as np

from . import core as O
from . import exact as X

__all__ = ["DynamicOracle", "BSM", "ISM"]

BSM, ISM = 0, 1


def _csr(n, edges):
    from paper_2511_16356_gb300.synth import csr_from_edges

    e = np.array(sorted(edges), dtype=np.int64).reshape(-1, 2)
    return csr_from_edges(n, e[:, 0], e[:, 1])


class DynamicOracle:
    def __init__(self, g, seed: int, n_trees: int, r: int | None = None):
        self.n = g.n
        self.edges = {(int(a), int(b)) for a, b in g.edges()}
        self.g = g
        self.t0 = O.tau0(g, r)
        self.r = self.t0.r
        self.seed = seed
        self.seq = 0
        self.next_sid = 0
        self.parents, self.f, self.w, self.sid, self.steps = [], [], [], [], []
        for _ in range(n_trees):
            p, st = O.wilson(g, self.r, seed, self.next_sid)
            self._append(p, st)

    # ------------------------------------------------------------------
    def _append(self, p, st):
        self.parents.append(p)
        self.f.append(self.f_of(p))
        self.w.append(1.0)
        self.sid.append(self.next_sid)
        self.steps.append(st)
        self.next_sid += 1

    def f_of(self, parent) -> int:
        t = O.traverse(self.g, self.r, parent)
        return O.f_alg1(self.g, self.t0, parent, t.vol)

    def refresh(self):
        self.f = [self.f_of(p) for p in self.parents]

    def estimate(self) -> float:
        twom = 2 * len(self.edges)
        num = math.fsum(w * (f / twom) for w, f in zip(self.w, self.f))
        return num / math.fsum(self.w)

    def contains(self, k: int, u: int, v: int) -> bool:
        p = self.parents[k]
        return p[u] == v or p[v] == u

    # ------------------------------------------------------------------
    def insert(self, u: int, v: int, mode: int, R: float | None = None, refresh: bool = False):
        key = (min(u, v), max(u, v))
        if key in self.edges:
            raise ValueError("edge exists")
        self.edges.add(key)
        self.g = _csr(self.n, self.edges)
        if R is None:
            R = X.resistance(self.g, u, v)
        N = len(self.parents)
        k = min(N, int(math.ceil(R * N)))
        sel = sorted(int(x) for x in O.select(self.seed, self.seq, N, k))
        W = math.fsum(self.w)
        if mode == BSM:
            for idx in sel:
                p, st = O.cond_wilson(self.g, u, v, self.r, self.seed, self.next_sid)
                self.parents[idx] = p
                self.sid[idx] = self.next_sid
                self.steps[idx] = st
                self.next_sid += 1
                self.f[idx] = self.f_of(p)
        else:
            for idx in sel:
                p, d_old, d_new = O.link_cut(self.g, self.parents[idx], self.r, u, v, self.seed,
                                             self.seq, idx)
                self.parents[idx] = p
                self.w[idx] = self.w[idx] * d_old / d_new
                self.f[idx] = self.f_of(p)
            selset = set(sel)
            A = math.fsum(self.w[i] for i in sel)
            B = math.fsum(self.w[i] for i in range(N) if i not in selset)
            for i in range(N):
                if i in selset:
                    self.w[i] = self.w[i] / A * (R * W)
                elif B > 0:
                    self.w[i] = self.w[i] / B * ((1.0 - R) * W)
        if refresh:
            self.refresh()
        self.seq += 1
        return sel

    def delete(self, u: int, v: int, mode: int, refresh: bool = False):
        key = (min(u, v), max(u, v))
        if key not in self.edges:
            raise ValueError("edge missing")
        edges2 = set(self.edges)
        edges2.remove(key)
        g2 = _csr(self.n, edges2)
        from paper_2511_16356_gb300.synth import is_connected

        if g2.n != self.n or np.any(g2.deg == 0) or not is_connected(g2):
            raise ValueError("bridge")
        hit = [k for k in range(len(self.parents)) if self.contains(k, u, v)]
        tau0_hit = self.t0.p0[u] == v or self.t0.p0[v] == u
        self.edges = edges2
        self.g = g2
        if tau0_hit:
            self.t0 = O.tau0(self.g, self.r)
        if mode == BSM:
            for idx in hit:
                p, st = O.wilson(self.g, self.r, self.seed, self.next_sid)
                self.parents[idx] = p
                self.sid[idx] = self.next_sid
                self.steps[idx] = st
                self.next_sid += 1
                self.f[idx] = self.f_of(p)
        else:
            w_org = math.fsum(self.w[i] for i in hit)
            for idx in hit:
                p, d_old, d_new = O.cut_link(self.g, self.parents[idx], self.r, u, v, self.seed,
                                             self.seq, idx)
                self.parents[idx] = p
                self.w[idx] = self.w[idx] * d_old / d_new
                self.f[idx] = self.f_of(p)
            A = math.fsum(self.w[i] for i in hit)
            for i in hit:
                self.w[i] = self.w[i] / A * w_org
        if refresh or tau0_hit:
            self.refresh()
        self.seq += 1
        return hit
