"""Quark-level Wick contractions and determinants (test infrastructure; see oracle/__init__).

arXiv 2201.04269 Sec. 1: the contraction <q(a_1)...q(a_n) qbar(a'_1)...qbar(a'_n)> of
quark-only operators is a sum over the n_u! n_d! ways of pairing each quark with an
antiquark of the same flavour; the determinant formulation (cited in Sec. 1) rewrites
it as the determinant of the matrix of propagators S(a_i; a'_j), evaluated by LU
factorisation.

Functions here:
* ``pairings``   the Wick sum taken literally: every flavour-preserving pairing, with
                 the sign of the Grassmann reordering that brings each pair together
                 (no determinant anywhere);
* ``det_leibniz`` determinant as the signed sum over permutations;
* ``det_lu``     determinant by LU with partial pivoting (pivot = largest |re|+|im|,
                 first index on ties, each row swap flips the sign, an exactly zero
                 pivot gives 0);
* ``contraction`` the signed determinant form used everywhere else:
                 (-1)^{n(n-1)/2} det U[a_u, a'_u] det D[a_d, a'_d] for flavour-grouped
                 slots (the reordering signs are part of the operator weights).
"""
from __future__ import annotations

import itertools

import numpy as np


def perm_sign(p) -> int:
    p = list(p)
    inv = sum(1 for i in range(len(p)) for k in range(i + 1, len(p)) if p[i] > p[k])
    return -1 if inv % 2 else 1


def pairings(q, qbar, props) -> complex:
    """<q_1 ... q_n qbar_1 ... qbar_n> by explicit Grassmann pairing.

    ``q`` and ``qbar`` are lists of (flavour, index) with index = 3*spin + colour;
    ``props[f]`` is the 12x12 propagator of flavour f (row = quark, column = antiquark).
    Each flavour-preserving permutation pi pairs q_i with qbar_{pi(i)}; its sign is that
    of the rearrangement of the 2n Grassmann fields into (q_1 qbar_pi1)(q_2 qbar_pi2)...
    """
    n = len(q)
    assert len(qbar) == n
    flavours = sorted({f for f, _ in q} | {f for f, _ in qbar})
    qi = {f: [i for i in range(n) if q[i][0] == f] for f in flavours}
    bi = {f: [k for k in range(n) if qbar[k][0] == f] for f in flavours}
    if any(len(qi[f]) != len(bi[f]) for f in flavours):
        return 0j
    total = 0j
    for choice in itertools.product(*[itertools.permutations(bi[f]) for f in flavours]):
        pi = [0] * n
        for f, perm in zip(flavours, choice):
            for i, k in zip(qi[f], perm):
                pi[i] = k
        # positions of the fields in the original product: q_i at i, qbar_k at n + k
        seq = []
        for i in range(n):
            seq += [i, n + pi[i]]
        val = 1.0 + 0j
        for i in range(n):
            val *= props[q[i][0]][q[i][1], qbar[pi[i]][1]]
        total += perm_sign(seq) * val
    return total


def det_leibniz(m: np.ndarray) -> complex:
    n = m.shape[0]
    if n == 0:
        return 1.0 + 0j
    total = 0j
    for p in itertools.permutations(range(n)):
        val = 1.0 + 0j
        for i in range(n):
            val *= m[i, p[i]]
        total += perm_sign(p) * val
    return total


def det_lu(m: np.ndarray) -> complex:
    """Determinant by Gaussian elimination with partial pivoting, in complex128."""
    a = np.array(m, dtype=np.complex128, copy=True)
    n = a.shape[0]
    det = 1.0 + 0j
    for k in range(n):
        mag = np.abs(a[k:, k].real) + np.abs(a[k:, k].imag)
        p = k + int(np.argmax(mag))  # first maximum wins
        if mag[p - k] == 0.0:
            return 0j
        if p != k:
            a[[k, p]] = a[[p, k]]
            det = -det
        det *= a[k, k]
        if k + 1 < n:
            f = a[k + 1:, k] / a[k, k]
            a[k + 1:, k + 1:] -= np.outer(f, a[k, k + 1:])
    return det


def wick_sign(n: int) -> int:
    """(-1)^{n(n-1)/2}: reverses the antiquark order so that the pairing is nested."""
    return -1 if (n * (n - 1) // 2) % 2 else 1


def contraction(a_u, a_d, b_u, b_d, U, D, det=det_lu) -> complex:
    """<q...q qbar...qbar> for flavour-grouped slots via determinants."""
    n = len(a_u) + len(a_d)
    du = det(U[np.ix_(list(a_u), list(b_u))]) if a_u else 1.0
    dd = det(D[np.ix_(list(a_d), list(b_d))]) if a_d else 1.0
    return wick_sign(n) * du * dd
