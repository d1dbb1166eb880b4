"""Hadron blocks and the block-level correlator (test infrastructure; see oracle/__init__).

arXiv 2201.04269 Sec. 2 (hadron blocks) and Sec. 3 (the general and the expanded block
form of a multi-baryon correlator).

Block (Sec. 2, the proton block equation), for a baryon B = eps_abc (q1_a^T G q2_b) q3_c
with q1 = q3, at sink site x and source point x':

    f^B(x; s1, s2, s3)_alpha = < B_alpha(x) qbar1(s1) qbar2(s2) qbar3(s3) >
        = eps_abc G_beta,gamma [ Q1[(a beta), s3] Q1[(c alpha), s1]
                                 - Q1[(a beta), s1] Q1[(c alpha), s3] ] Q2[(b gamma), s2]

where Q1, Q2 are the 12x12 propagators of flavours q1 and q2 at x, row (colour a,
spin beta) = 3 beta + a, and s1, s2, s3 are source spin-colour indices.  A momentum
projected block sums e^{-i p.x} f^B(x) over the sink sites of a time slice.

Block types (the baryons of the paper's operators): P = (u, d, u) and N = (d, u, d),
each with G = C gamma_5, C gamma_5 P_+ or C gamma_5 P_-.  A factor is a block entry
(type h, eta) with eta = ((s1 * 12 + s2) * 12 + s3) * 4 + alpha; its id is
h * 6912 + eta.

Block form of the correlator (Sec. 3, general form and expanded form).  The sink
operator is a sum of products of A baryons whose free spins are tied by a tensor
T(alpha_1..alpha_A; j); the source operator is the one used by the quark-level oracle
(conjugated sink weights in flavour-grouped slot order, reading of the paper's silence
on the source).  Wick's theorem distributes the source fields over the A sink baryons:
an assignment sigma gives each block the source fields of its flavours (one fixed order
per set; the block itself sums the orders), with the sign of the permutation that
brings the source fields into block order times (-1)^{A(A-1)/2} from interleaving the
odd sink and source groups.  The number of assignments is N_w of the general form
(9 for dinucleon I).  Expanding every index gives strings of factors with fixed eta;
factors are ordered canonically (ascending id, i.e. lexicographic on (h, eta)) and
identical strings merged with their multiplicities (Sec. 3).

    C_local(t) = sum_x sum_k w_k prod_i f^{h_ik}(x; eta_ik)          (local sink)
    C_proj(t)  = sum_k w_k prod_i F^{h_ik}(eta_ik),  F = sum_x e^{-i p.x} f(x)

C_local is the quark-level correlator of the other oracle modules (pinned in tests);
C_proj projects every baryon of the sink separately (the paper's block setting).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

from . import dirac
from .canonical import canonical_side
from .operators import U, D, build, eps3, nonzeros

N_ETA = 12 * 12 * 12 * 4

# (name, flavours of (q1, q2, q3), G)
BLOCK_TYPES = (
    ("P", (U, D, U), dirac.CG5),
    ("N", (D, U, D), dirac.CG5),
    ("P+", (U, D, U), dirac.CG5_PPLUS),
    ("P-", (U, D, U), dirac.CG5_PMINUS),
    ("N+", (D, U, D), dirac.CG5_PPLUS),
    ("N-", (D, U, D), dirac.CG5_PMINUS),
)
TYPE_INDEX = {name: h for h, (name, _, _) in enumerate(BLOCK_TYPES)}


def block_site(U_x, D_x, h):
    """f^h(x; s1, s2, s3)_alpha for one or more sites, straight from the block equation.

    U_x, D_x: [..., 12, 12]; returns [..., 12, 12, 12, 4] indexed (s1, s2, s3, alpha)."""
    _, (f1, f2, _), gamma = BLOCK_TYPES[h]
    props = (np.asarray(U_x), np.asarray(D_x))
    Q1, Q2 = props[f1], props[f2]
    out = np.zeros(Q1.shape[:-2] + (12, 12, 12, 4), np.complex128)
    for alpha in range(4):
        for (a, b, c), e in eps3():
            for beta, gam, g in nonzeros(gamma):
                r1, r2, r3 = 3 * beta + a, 3 * gam + b, 3 * alpha + c
                q2 = Q2[..., r2, :][..., None, :, None]
                # Q1[(a beta), s3] Q1[(c alpha), s1]
                t1 = Q1[..., r3, :][..., :, None, None] * Q1[..., r1, :][..., None, None, :]
                # Q1[(a beta), s1] Q1[(c alpha), s3]
                t2 = Q1[..., r1, :][..., :, None, None] * Q1[..., r3, :][..., None, None, :]
                out[..., alpha] += (e * g) * (t1 - t2) * q2
    return out


@dataclass
class Product:
    """One product of baryons in a sink operator: coef * sum_alpha T(alpha; j) prod_i B_i^{alpha_i}."""
    coef: complex
    types: tuple          # block type index per baryon, in operator order
    tie: list             # per free index j: {alpha tuple: weight}


def _tie2(gamma):
    return {(a, b): g for a, b, g in nonzeros(gamma)}


def structure(name):
    """Baryon-level form of an operator of Eq. 2: (products, norm); the same products
    the quark-level expansion in ``operators.build`` multiplies out."""
    cg5 = dirac.CG5
    t = TYPE_INDEX
    if name == "proton":
        return [Product(1, (t["P"],), [{(j,): 1} for j in range(4)])], 1.0
    if name == "neutron":
        return [Product(1, (t["N"],), [{(j,): 1} for j in range(4)])], 1.0
    if name in ("dinucleon_I", "dinucleon_II"):
        prods = [Product(1, (t["N"], t["P"]), [_tie2(cg5)])]
        if name == "dinucleon_I":
            return prods, 1.0
        prods.append(Product(-1, (t["P"], t["N"]), [_tie2(cg5)]))
        return prods, 1.0 / math.sqrt(2.0)
    if name in ("he3_I", "he3_II", "he3_II_s"):
        def three(coef, x, y, z):
            tie = [{(a, b, j): g for (a, b), g in _tie2(cg5).items()} for j in range(4)]
            return Product(coef, (t[x], t[y], t[z]), tie)
        p1 = three(1, "P-", "N+", "P+")       # + p_-^T Cg5 n_+ p_+^j
        if name == "he3_I":
            return [p1], 1.0
        p2 = three(-1, "P+", "N+", "P-")      # - p_+^T Cg5 n_+ p_-^j
        p5 = three(1, "P+", "P-", "N+")       # + p_+^T Cg5 p_- n_+^j
        if name == "he3_II_s":
            return [p1, p2, p5], 2.0 / math.sqrt(6.0)
        p3 = three(1, "N+", "P+", "P-")
        p4 = three(-1, "N+", "P-", "P+")
        p6 = three(-1, "P-", "P+", "N+")
        return [p1, p2, p3, p4, p5, p6], 1.0 / math.sqrt(6.0)
    raise ValueError(f"unknown operator {name!r}")


def _pattern(h):
    return BLOCK_TYPES[h][1]


def assignments(types, n_u, n_d):
    """Every way to hand the source fields (u slots 0..n_u-1, then d slots) to the sink
    blocks: list of (per-block global source positions in block order, sign)."""
    out = []
    A = len(types)

    def rec(i, free_u, free_d, acc):
        if i == A:
            if free_u or free_d:
                return
            seq = [p for blk in acc for p in blk]
            inv = sum(1 for x in range(len(seq)) for y in range(x + 1, len(seq)) if seq[x] > seq[y])
            sign = (-1) ** inv * (-1) ** (A * (A - 1) // 2)
            out.append((tuple(acc), sign))
            return
        pat = _pattern(types[i])
        need_u = sum(1 for f in pat if f == U)
        need_d = 3 - need_u
        for cu in itertools.combinations(free_u, need_u):
            for cd in itertools.combinations(free_d, need_d):
                iu, idd = iter(cu), iter(cd)
                blk = tuple(next(iu) if f == U else n_u + next(idd) for f in pat)
                rec(i + 1, [p for p in free_u if p not in cu], [p for p in free_d if p not in cd], acc + [blk])

    rec(0, list(range(n_u)), list(range(n_d)), [])
    return out


class BlockPlan:
    """Merged expanded block form of an operator's correlator.

    ``ids`` [K, A] factor ids in canonical (ascending) order, ``W`` [K] merged weights
    (projector, Wick signs, both normalisations folded in), ``multiplicity`` [K] number of
    expanded terms merged into each, ``n_w`` the number of source assignments per product.

    ``source="slots"`` expands the source operator tuple by tuple, as written;
    ``source="canonical"`` first merges source tuples that differ by a permutation of
    same-flavour slots into ascending sets with the permutation sign (the canonical
    form of Sec. 3 applied to the source operator; the value is unchanged because the
    contraction is antisymmetric in same-flavour source fields), which leaves far fewer
    expanded terms."""

    def __init__(self, name, source="slots"):
        op = build(name)
        prods, norm = structure(name)
        self.name, self.op = name, op
        self.A = len(prods[0].types)
        self.n_w = [len(assignments(p.types, op.n_u, op.n_d)) for p in prods]
        keys, wts = [], []
        for j in range(op.n_free):
            for jp in range(op.n_free):
                pj = op.proj[j, jp]
                if pj == 0:
                    continue
                terms = op.terms[jp] if source == "slots" else canonical_side(op.terms[jp])
                src = sorted(terms)
                if not src:
                    continue
                a_src = np.array([ku + kd for ku, kd in src], dtype=np.int64)       # [n_src, n_u + n_d]
                w_src = np.conj(np.array([terms[k] for k in src], dtype=np.complex128))
                for prod in prods:
                    sig = assignments(prod.types, op.n_u, op.n_d)
                    for alphas, tw in prod.tie[j].items():
                        for blocks, sign in sig:
                            ids = np.empty((len(src), self.A), np.int64)
                            for i, (h, blk, al) in enumerate(zip(prod.types, blocks, alphas)):
                                s1, s2, s3 = (a_src[:, p] for p in blk)
                                ids[:, i] = h * N_ETA + ((s1 * 12 + s2) * 12 + s3) * 4 + al
                            keys.append(np.sort(ids, axis=1))
                            wts.append(complex(pj * prod.coef * tw * sign) * w_src)
        ids = np.concatenate(keys) if keys else np.zeros((0, self.A), np.int64)
        w = np.concatenate(wts) if wts else np.zeros(0, np.complex128)
        self.n_expanded = len(w)
        base = 6 * N_ETA
        key = np.zeros(len(w), np.int64)
        for i in range(self.A):
            key = key * base + ids[:, i]
        uk, inv, cnt = np.unique(key, return_inverse=True, return_counts=True)
        wr = np.bincount(inv, weights=w.real, minlength=len(uk))
        wi = np.bincount(inv, weights=w.imag, minlength=len(uk))
        W = (wr + 1j * wi) * (norm * op.norm)
        keep = W != 0
        uk, W, cnt = uk[keep], W[keep], cnt[keep]
        out = np.empty((len(uk), self.A), np.int64)
        for i in reversed(range(self.A)):
            out[:, i] = uk % base
            uk = uk // base
        self.ids, self.W, self.multiplicity = out, W, cnt
        self.types = sorted({int(i) // N_ETA for i in np.unique(out)}) if len(out) else []

    @property
    def n_terms(self):
        return len(self.W)

    def factors(self, U_x, D_x):
        """All block values of the plan's types at the given sites: [..., 6 * N_ETA]."""
        U_x, D_x = np.asarray(U_x), np.asarray(D_x)
        out = np.zeros(U_x.shape[:-2] + (6 * N_ETA,), np.complex128)
        for h in self.types:
            out[..., h * N_ETA:(h + 1) * N_ETA] = block_site(U_x, D_x, h).reshape(U_x.shape[:-2] + (N_ETA,))
        return out

    def evaluate(self, F):
        """sum_k W_k prod_i F[ids_ki] for factor values F [..., 6 * N_ETA]."""
        F = np.asarray(F)
        prod = np.ones(F.shape[:-1] + (self.n_terms,), np.complex128)
        for i in range(self.A):
            prod = prod * F[..., self.ids[:, i]]
        return prod @ self.W

    def site_values(self, U_x, D_x, chunk=16):
        """Local-sink block-form correlator at each site: [S]."""
        U_x = np.asarray(U_x).reshape(-1, 12, 12)
        D_x = np.asarray(D_x).reshape(-1, 12, 12)
        return np.concatenate([self.evaluate(self.factors(U_x[k:k + chunk], D_x[k:k + chunk]))
                               for k in range(0, len(U_x), chunk)])


def site_coords(L):
    """Lattice coordinates (x, y, z) of sink sites in the field order (x fastest)."""
    idx = np.arange(L ** 3)
    return np.stack([idx % L, (idx // L) % L, idx // (L * L)], axis=1)


def projected_blocks(plan, U, D, L, p=(0, 0, 0)):
    """F(t) = sum_x e^{-i p.x} f(x) per time slice for the plan's block types, with
    p in units of 2 pi / L.  U, D: [T, L^3, 12, 12]; returns [T, 6 * N_ETA]."""
    U, D = np.asarray(U), np.asarray(D)
    T, V3 = U.shape[:2]
    phase = np.exp(-2j * np.pi * (site_coords(L) @ np.asarray(p, float)) / L)
    out = np.zeros((T, 6 * N_ETA), np.complex128)
    for t in range(T):
        for k in range(0, V3, 16):
            f = plan.factors(U[t, k:k + 16], D[t, k:k + 16])
            out[t] += phase[k:k + 16] @ f
    return out


def correlator_projected(plan, U, D, L, p=(0, 0, 0)):
    """C_proj(t) with every baryon of the sink projected to momentum p."""
    return plan.evaluate(projected_blocks(plan, U, D, L, p))
