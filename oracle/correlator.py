"""The correlator by definition and in canonical form (test infrastructure; see oracle/__init__).

arXiv 2201.04269 Eq. 1 with the index set I = {(a, a') : W != 0}, for an operator whose
weight factorises over sink and source,

    W(a, a') = sum_{j,j'} P_jj' s_j(a) conj(r_j'(a')),

where j, j' run over the free spin index of the operator and P is the spin projector.
Reading (the paper never writes the source operator): r_j = s_j on the same slot
pattern.  With the determinant form of the contraction,

    C_x = (-1)^{n(n-1)/2} sum_{(a,a') in I} W(a,a') det U_x[a_u, a'_u] det D_x[a_d, a'_d],
    C(t) = sum_{x in time slice t} C_x       (local sink, zero momentum).
"""
from __future__ import annotations

import math

import numpy as np

from . import native
from .canonical import canonical_side, pairs
from .wick import pairings, wick_sign


def sides(op):
    """Per free index j: (idx int8 [n, n_u + n_d], w complex [n]) of the sink; the source
    uses the same lists (its weights enter conjugated)."""
    snk = [op.arrays(j) for j in range(op.n_free)]
    return snk, snk


def site_pairings(op, U, D) -> complex:
    """Eq. 1 at one site with every contraction done by explicit Wick pairing (tiny cases)."""
    total = 0j
    props = {0: U, 1: D}
    for j, k, p in pairs(op.proj):
        for (a_u, a_d), wa in op.terms[j].items():
            q = [(0, i) for i in a_u] + [(1, i) for i in a_d]
            for (b_u, b_d), wb in op.terms[k].items():
                qb = [(0, i) for i in b_u] + [(1, i) for i in b_d]
                total += p * wa * np.conj(wb) * pairings(q, qb, props)
    return total * op.norm * op.norm


def site_direct(op, U, D, n_threads=1):
    """Eq. 1 per site over the index set with LU determinants (plain C)."""
    snk, src = sides(op)
    return native.direct(op.n_u, op.n_d, snk, src, op.proj, U, D, n_threads)


class CanonicalPlan:
    """Canonical merged term list of an operator's correlator (Sec. 3).

    Row sets R_f and column sets C_f of each flavour are the distinct ascending slot
    sets of the merged sink and source; every (R, C) pair is a minor; a term is
    (minor_u, minor_d, W) with W folding the Wick sign, the projector and the weights;
    duplicate (minor_u, minor_d) terms are merged and exact zeros dropped."""

    def __init__(self, op):
        self.op = op
        can = [canonical_side(t) for t in op.terms]
        used = sorted({j for j, k, _ in pairs(op.proj)} | {k for _, k, _ in pairs(op.proj)})
        self.rows_u = sorted({k[0] for j in used for k in can[j]})
        self.rows_d = sorted({k[1] for j in used for k in can[j]})
        self.cols_u, self.cols_d = self.rows_u, self.rows_d   # source pattern = sink pattern
        iu = {r: i for i, r in enumerate(self.rows_u)}
        idd = {r: i for i, r in enumerate(self.rows_d)}
        n_cu, n_cd = len(self.cols_u), len(self.cols_d)
        ws = wick_sign(op.n_u + op.n_d) * op.norm * op.norm
        mu_l, md_l, w_l = [], [], []
        for j, k, p in pairs(op.proj):
            sj = [(iu[a[0]], idd[a[1]], w) for a, w in can[j].items()]
            rk = [(iu[b[0]], idd[b[1]], w) for b, w in can[k].items()]
            if not sj or not rk:
                continue
            a_u, a_d, a_w = (np.array(v) for v in zip(*sj))
            b_u, b_d, b_w = (np.array(v) for v in zip(*rk))
            mu_l.append((a_u[:, None] * n_cu + b_u[None, :]).ravel())
            md_l.append((a_d[:, None] * n_cd + b_d[None, :]).ravel())
            w_l.append((ws * p * a_w[:, None] * np.conj(b_w)[None, :]).ravel())
        if mu_l:
            mu, md, w = np.concatenate(mu_l), np.concatenate(md_l), np.concatenate(w_l)
            key = mu.astype(np.int64) * (len(self.rows_d) * n_cd) + md
            uk, inv = np.unique(key, return_inverse=True)
            wr = np.bincount(inv, weights=w.real, minlength=len(uk))
            wi = np.bincount(inv, weights=w.imag, minlength=len(uk))
            W = wr + 1j * wi
            keep = W != 0
            self.mu = (uk[keep] // (len(self.rows_d) * n_cd)).astype(np.int32)
            self.md = (uk[keep] % (len(self.rows_d) * n_cd)).astype(np.int32)
            self.W = W[keep]
        else:
            self.mu = np.zeros(0, np.int32)
            self.md = np.zeros(0, np.int32)
            self.W = np.zeros(0, np.complex128)

    def minor_defs(self, flavour):
        rows, cols = (self.rows_u, self.cols_u) if flavour == 0 else (self.rows_d, self.cols_d)
        k = self.op.n_u if flavour == 0 else self.op.n_d
        r = np.array([rr for rr in rows for _ in cols], dtype=np.int8).reshape(-1, k)
        c = np.array([cc for _ in rows for cc in cols], dtype=np.int8).reshape(-1, k)
        return r, c

    @property
    def n_terms(self):
        return len(self.W)

    def site_values(self, U, D, n_threads=1):
        U = np.asarray(U).reshape(-1, 12, 12)
        if self.n_terms == 0:
            return np.zeros(U.shape[0], np.complex128)
        return native.canonical(self.op.n_u, self.op.n_d, self.minor_defs(0), self.minor_defs(1),
                                self.mu, self.md, self.W, U, D, n_threads)


def correlator(site_fn, U, D):
    """C(t) = sum over sites of a per-site function; U, D: [T, V3, 12, 12]."""
    T, V3 = U.shape[:2]
    vals = site_fn(U.reshape(-1, 12, 12), D.reshape(-1, 12, 12)).reshape(T, V3)
    return np.array([complex(math.fsum(v.real), math.fsum(v.imag)) for v in vals])


def correlator_momentum(site_fn, U, D, L, p):
    """C(t, p) = sum_x e^{-i 2 pi p.x / L} C_x(t): the sink projected to momentum p (the
    phase of the momentum projection in Sec. 2); site x of a slice sits at
    (x mod L, (x / L) mod L, x / L^2).  p = (0, 0, 0) is ``correlator``."""
    T, V3 = U.shape[:2]
    assert V3 == L ** 3
    vals = site_fn(U.reshape(-1, 12, 12), D.reshape(-1, 12, 12)).reshape(T, V3)
    x = np.arange(V3)
    k = (p[0] * (x % L) + p[1] * ((x // L) % L) + p[2] * (x // (L * L))) % L
    phase = np.exp(-2j * np.pi * k / L)
    return np.array([np.sum(v * phase) for v in vals])

