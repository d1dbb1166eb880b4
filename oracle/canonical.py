"""Canonical ordering and multiplicity merging (test infrastructure; see oracle/__init__).

arXiv 2201.04269 Sec. 3 orders the factors of each expanded term canonically and merges
identical terms into one term whose coefficient carries the multiplicity.  At the quark
level used here the factors are determinants: reordering the rows of det U[a_u, a'_u]
into ascending order multiplies it by the sign of the sorting permutation, and a
repeated row index makes it vanish (these zero tuples are the Index-List pruning of
Sec. 1).  So every sink tuple a becomes (sign, R_u, R_d) with R_u, R_d ascending index
sets, and the correlator at one site is

    C_x = w_n sum_{j,j'} P_jj' sum_{(R_u,R_d)} s_j(R_u,R_d) sum_{(C_u,C_d)} conj(r_j'(C_u,C_d))
          det U[R_u, C_u] det D[R_d, C_d]

with merged weights s_j, r_j' and w_n = (-1)^{n(n-1)/2}.
"""
from __future__ import annotations

import numpy as np

from .wick import wick_sign


def sort_with_sign(t):
    """(sign, ascending tuple) of a slot tuple, or (0, None) if an index repeats."""
    t = list(t)
    if len(set(t)) < len(t):
        return 0, None
    s = 1
    for i in range(len(t)):            # bubble sort, one sign flip per swap
        for k in range(len(t) - 1 - i):
            if t[k] > t[k + 1]:
                t[k], t[k + 1] = t[k + 1], t[k]
                s = -s
    return s, tuple(t)


def canonical_side(terms: dict) -> dict:
    """Merge a {(a_u, a_d): w} slot-ordered term dict into {(R_u, R_d): w}."""
    out = {}
    for (a_u, a_d), w in terms.items():
        su, ru = sort_with_sign(a_u)
        sd, rd = sort_with_sign(a_d)
        if su == 0 or sd == 0:
            continue
        out[(ru, rd)] = out.get((ru, rd), 0) + su * sd * w
    return {k: v for k, v in out.items() if v != 0}


def pairs(proj):
    """(j, j', P_jj') for the nonzero projector entries."""
    return [(j, k, proj[j, k]) for j in range(proj.shape[0]) for k in range(proj.shape[1]) if proj[j, k] != 0]


def canonical_terms(op):
    """Canonical index set of an operator's correlator: list of (R_u, R_d, C_u, C_d, W).

    W folds the Wick sign, the projector and the merged sink and (conjugated) source
    weights; terms whose merged weight is exactly zero are dropped."""
    snk = [canonical_side(t) for t in op.terms]
    ws = wick_sign(op.n_u + op.n_d) * op.norm * op.norm
    acc = {}
    for j, k, p in pairs(op.proj):
        for (ru, rd), a in snk[j].items():
            for (cu, cd), b in snk[k].items():
                key = (ru, rd, cu, cd)
                acc[key] = acc.get(key, 0) + ws * p * a * np.conj(b)
    return [(k[0], k[1], k[2], k[3], v) for k, v in sorted(acc.items()) if v != 0]
