"""Grassmann expansion of the paper's baryon and multi-baryon operators (test infrastructure).

Follows arXiv 2201.04269 Sec. 1: single-baryon operators

    p^a = eps_abc (u_a^T G d_b) u_c^alpha,   n^a = eps_abc (d_a^T G u_b) d_c^alpha,

with G = C gamma_5 (relativistic) or C gamma_5 P_+- (non-relativistic), and the
multi-baryon operators of Eq. 2 (D_I, D_II, 3He_I, 3He_II) built by tying two
baryons with C gamma_5, X^T (C gamma_5) Y = sum_{ab} X^a (C gamma_5)_{ab} Y^b.

An operator is expanded into ordered products of quark fields q^{f,c}_s; each product
is then written in flavour-grouped slot order (all up fields first, then all down
fields, each keeping its relative order), multiplying the coefficient by the sign of
that Grassmann reordering.  Spin-colour index of a slot: i = 3 * spin + colour.

Readings (the paper is silent): the free spin index of the proton and of 3He is
projected with P_+ = (1 + gamma_4)/2 and traced (j = j' in {0, 1}); the source
operator uses the complex-conjugated sink weights on the same slot pattern; the
stand-in operator 3He_II-s keeps printed terms 1, 2 and 5 of 3He_II with their signs
and normalisation 2/sqrt(6) (the printed 3He_II and D_II vanish identically because
baryons are Grassmann-odd and C gamma_5 is antisymmetric).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

from . import dirac

U, D = 0, 1  # flavour labels


def eps3():
    """Nonzero entries of the Levi-Civita symbol eps_abc, eps_012 = +1."""
    out = []
    for p in itertools.permutations(range(3)):
        inv = sum(1 for i in range(3) for k in range(i + 1, 3) if p[i] > p[k])
        out.append((p, -1 if inv % 2 else 1))
    return out


def nonzeros(m):
    return [(a, b, m[a, b]) for a in range(4) for b in range(4) if m[a, b] != 0]


def baryon(flavours, gamma):
    """Terms of a baryon eps_abc (q1_a^T G q2_b) q3_c^alpha for each free spin alpha.

    Returns a list over alpha of lists of (coefficient, fields); a field is
    (flavour, colour, spin)."""
    f1, f2, f3 = flavours
    out = []
    for alpha in range(4):
        terms = []
        for (a, b, c), s in eps3():
            for beta, gam, g in nonzeros(gamma):
                fields = ((f1, a, beta), (f2, b, gam), (f3, c, alpha))
                terms.append((s * g, fields))
        out.append(terms)
    return out


def proton(gamma=dirac.CG5):
    return baryon((U, D, U), gamma)


def neutron(gamma=dirac.CG5):
    return baryon((D, U, D), gamma)


def tie(x, y, gamma=dirac.CG5):
    """X^T G Y = sum_ab X^a G_ab Y^b for baryons X, Y given per free spin."""
    terms = []
    for a, b, g in nonzeros(gamma):
        for cx, fx in x[a]:
            for cy, fy in y[b]:
                terms.append((g * cx * cy, fx + fy))
    return terms


def times(terms, z):
    """(two-baryon terms) x (third baryon Z^j), per free spin j of Z."""
    return [[(c * cz, f + fz) for c, f in terms for cz, fz in z[j]] for j in range(4)]


def scale(terms, s):
    return [(s * c, f) for c, f in terms]


def grouped(fields):
    """Flavour-grouped slot form of an ordered field product.

    Returns (sign, a_u, a_d): sign of the Grassmann reordering that moves the up fields
    ahead of the down fields (stable), and the spin-colour indices of each group."""
    order = [k for k, f in enumerate(fields) if f[0] == U] + [k for k, f in enumerate(fields) if f[0] == D]
    inv = sum(1 for i in range(len(order)) for k in range(i + 1, len(order)) if order[i] > order[k])
    a_u = tuple(3 * fields[k][2] + fields[k][1] for k in order if fields[k][0] == U)
    a_d = tuple(3 * fields[k][2] + fields[k][1] for k in order if fields[k][0] == D)
    return (-1 if inv % 2 else 1), a_u, a_d


@dataclass
class Operator:
    """Sink operator in flavour-grouped slot form, one term dict per free spin index.

    ``terms[j]`` maps (a_u, a_d) to the merged weight before normalisation (a Gaussian
    integer, so merging is exact); ``norm`` is the operator's normalisation; ``proj`` is
    the spin projector P_jj' applied between sink index j and source index j'."""
    name: str
    n_u: int
    n_d: int
    terms: list
    proj: np.ndarray
    norm: float = 1.0
    raw_counts: list = field(default_factory=list)

    @property
    def n_free(self):
        return len(self.terms)

    def arrays(self, j):
        """(idx int8 [n, n_u + n_d], w complex128 [n]) for free index j, in sorted key order."""
        keys = sorted(self.terms[j])
        idx = np.array([ku + kd for ku, kd in keys], dtype=np.int8).reshape(len(keys), self.n_u + self.n_d)
        w = np.array([self.terms[j][k] for k in keys], dtype=np.complex128) * self.norm
        return idx, w


def _collect(per_j):
    terms, raw = [], []
    for tl in per_j:
        d = {}
        for c, f in tl:
            s, a_u, a_d = grouped(f)
            d[(a_u, a_d)] = d.get((a_u, a_d), 0) + s * c
        terms.append({k: complex(v) for k, v in d.items() if v != 0})
        raw.append(len(tl))
    return terms, raw


PROJ_PLUS_TRACE = np.diag([1.0, 1.0, 0.0, 0.0]).astype(np.complex128)


def build(name: str) -> Operator:
    """Expand a named operator of Eq. 2 (or a single baryon)."""
    cg5 = dirac.CG5
    if name == "proton":
        per_j, n_u, n_d, proj, norm = proton(), 2, 1, PROJ_PLUS_TRACE, 1.0
    elif name == "neutron":
        per_j, n_u, n_d, proj, norm = neutron(), 1, 2, PROJ_PLUS_TRACE, 1.0
    elif name == "dinucleon_I":
        per_j, n_u, n_d, proj, norm = [tie(neutron(), proton())], 3, 3, np.ones((1, 1), complex), 1.0
    elif name == "dinucleon_II":
        t = tie(neutron(), proton()) + scale(tie(proton(), neutron()), -1)
        per_j, n_u, n_d, proj, norm = [t], 3, 3, np.ones((1, 1), complex), 1.0 / np.sqrt(2.0)
    elif name in ("he3_I", "he3_II", "he3_II_s"):
        pm, pp = proton(dirac.CG5_PMINUS), proton(dirac.CG5_PPLUS)
        npl = neutron(dirac.CG5_PPLUS)
        t1 = times(tie(pm, npl, cg5), pp)                 # + p_-^T Cg5 n_+ p_+^j
        if name == "he3_I":
            per_j, norm = t1, 1.0
        else:
            t2 = times(scale(tie(pp, npl, cg5), -1), pm)  # - p_+^T Cg5 n_+ p_-^j
            t5 = times(tie(pp, pm, cg5), npl)             # + p_+^T Cg5 p_- n_+^j
            if name == "he3_II":
                t3 = times(tie(npl, pp, cg5), pm)         # + n_+^T Cg5 p_+ p_-^j
                t4 = times(scale(tie(npl, pm, cg5), -1), pp)  # - n_+^T Cg5 p_- p_+^j
                t6 = times(scale(tie(pm, pp, cg5), -1), npl)  # - p_-^T Cg5 p_+ n_+^j
                parts, norm = (t1, t2, t3, t4, t5, t6), 1.0 / np.sqrt(6.0)
            else:
                parts, norm = (t1, t2, t5), 2.0 / np.sqrt(6.0)
            per_j = [sum((p[j] for p in parts), []) for j in range(4)]
        n_u, n_d, proj = 5, 4, PROJ_PLUS_TRACE
    else:
        raise ValueError(f"unknown operator {name!r}")
    terms, raw = _collect(per_j)
    return Operator(name, n_u, n_d, terms, proj, norm, raw)


NAMES = ("proton", "neutron", "dinucleon_I", "dinucleon_II", "he3_I", "he3_II", "he3_II_s")
