"""Pins of the hadron-block oracle (oracle/blocks.py) against the paper and independent
statements of the same quantities (arXiv 2201.04269 Secs. 2-4)."""
import itertools
import math

import numpy as np
import pytest

import mbc_inputs as mi
from oracle import blocks as bl
from oracle import correlator as cor
from oracle import factor_tree as ft
from oracle import operators as ops
from oracle.wick import pairings


def rand_sites(seed, n):
    sites = np.arange(n)
    return mi.site_matrices(seed, 0, 0, 1, sites), mi.site_matrices(seed, 0, 1, 1, sites)


def test_block_equals_explicit_pairings():
    """Sec. 2 block equation vs the Wick sum taken literally, on random source indices."""
    Us, Ds = rand_sites(11, 1)
    rng = np.random.default_rng(0)
    for h, (name, flav, gamma) in enumerate(bl.BLOCK_TYPES):
        f = bl.block_site(Us[0], Ds[0], h)
        baryon = ops.baryon(flav, gamma)
        for _ in range(6):
            s = [int(v) for v in rng.integers(0, 12, 3)]
            alpha = int(rng.integers(0, 4))
            want = 0j
            for coef, fields in baryon[alpha]:
                q = [(fl, 3 * sp + col) for fl, col, sp in fields]
                qb = [(flav[0], s[0]), (flav[1], s[1]), (flav[2], s[2])]
                want += coef * pairings(q, qb, {0: Us[0], 1: Ds[0]})
            assert abs(f[s[0], s[1], s[2], alpha] - want) <= 1e-13 * (1 + abs(want)), (name, s, alpha)


def test_block_antisymmetric_in_same_flavour_sources():
    Us, Ds = rand_sites(12, 2)
    for h in range(6):
        f = bl.block_site(Us, Ds, h)
        np.testing.assert_allclose(f, -np.swapaxes(f, 1, 3), atol=1e-13)
        i = np.arange(12)
        assert np.max(np.abs(f[:, i, :, i, :])) <= 1e-13


def test_assignment_counts_match_paper():
    """N_w of the general form: 9 for dinucleon I (Sec. 3), and for 3He the multinomial
    5!/(2!2!1!) x 4!/(1!1!2!) = 360 ways to hand 5 u and 4 d source quarks to (P, P, N)."""
    prods, _ = bl.structure("dinucleon_I")
    assert [len(bl.assignments(p.types, 3, 3)) for p in prods] == [9]
    for name in ("he3_I", "he3_II", "he3_II_s"):
        prods, _ = bl.structure(name)
        for p in prods:
            assert len(bl.assignments(p.types, 5, 4)) == 360
    multinom = math.factorial(5) // (2 * 2 * 1) * math.factorial(4) // (1 * 1 * 2)
    assert multinom == 360
    prods, _ = bl.structure("proton")
    assert len(bl.assignments(prods[0].types, 2, 1)) == 1


def test_assignment_signs_are_permutation_parities():
    """Every assignment is a distinct partition; its sign is the parity of the source
    reordering times (-1)^{A(A-1)/2}."""
    types = (bl.TYPE_INDEX["N"], bl.TYPE_INDEX["P"])
    seen = set()
    for blocks, sign in bl.assignments(types, 3, 3):
        seq = [p for b in blocks for p in b]
        assert sorted(seq) == list(range(6))
        key = tuple(frozenset(b) for b in blocks)
        assert key not in seen
        seen.add(key)
        inv = sum(1 for i, j in itertools.combinations(range(6), 2) if seq[i] > seq[j])
        assert sign == (-1) ** inv * (-1)


def test_printed_dinucleon_term_is_present():
    """Sec. 3 prints the k = 1 expanded term of dinucleon I,
    f^P(x', 1,1,2,2,3,1)_1 f^N(x', 1,1,2,2,3,2)_2 (1-based colour/spin values); it must
    be a term of the expansion (index s = 3 spin + colour, zero-based)."""
    plan = bl.BlockPlan("dinucleon_I")

    def fid(h, a, beta, b, gam, c, alpha_src, alpha):
        s1, s2, s3 = 3 * (beta - 1) + (a - 1), 3 * (gam - 1) + (b - 1), 3 * (alpha_src - 1) + (c - 1)
        return bl.TYPE_INDEX[h] * bl.N_ETA + ((s1 * 12 + s2) * 12 + s3) * 4 + (alpha - 1)

    key = sorted([fid("P", 1, 1, 2, 2, 3, 1, 1), fid("N", 1, 1, 2, 2, 3, 2, 2)])
    hit = np.all(plan.ids == np.array(key), axis=1)
    assert hit.sum() == 1 and plan.W[hit][0] != 0


@pytest.mark.parametrize("name", ["proton", "neutron", "dinucleon_I", "he3_I"])
def test_local_block_form_equals_determinant_form(name):
    """Sum over blocks at one site = the quark-level determinant correlator."""
    Us, Ds = rand_sites(13, 2)
    want = cor.CanonicalPlan(ops.build(name)).site_values(Us, Ds)
    for source in ("slots", "canonical"):
        got = bl.BlockPlan(name, source).site_values(Us, Ds)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)


def test_vanishing_operator_has_no_block_terms():
    assert bl.BlockPlan("dinucleon_II").n_terms == 0


def test_canonical_source_merges_permutations():
    a, b = bl.BlockPlan("dinucleon_I", "slots"), bl.BlockPlan("dinucleon_I", "canonical")
    assert b.n_expanded < a.n_expanded
    assert a.n_w == b.n_w == [9]


def two_site_brute_force(name, Ux, Dx, Uy, Dy):
    """<B_1(x) B_2(y) Obar(0)> for a two-baryon operator with the baryons at different
    sink sites: quark-level expansion with each field tagged by its baryon, every
    contraction a signed product of determinants whose rows come from that baryon's site."""
    op = ops.build(name)
    cg5 = ops.dirac.CG5
    sink = ops.tie(ops.neutron(), ops.proton(), cg5)      # fields: 3 of N, then 3 of P
    props = {(0, 0): Ux, (1, 0): Dx, (0, 1): Uy, (1, 1): Dy}
    total = 0j
    src = op.terms[0]
    src_keys = sorted(src)
    src_u = np.array([k[0] for k in src_keys])
    src_d = np.array([k[1] for k in src_keys])
    src_w = np.conj(np.array([src[k] for k in src_keys]))
    wsign = (-1) ** (6 * 5 // 2)
    for coef, fields in sink:
        sgn, a_u, a_d = ops.grouped(fields)
        order = [k for k, f in enumerate(fields) if f[0] == 0] + [k for k, f in enumerate(fields) if f[0] == 1]
        site = [k // 3 for k in order]
        n_u = len(a_u)
        Mu = np.stack([props[(0, site[i])][a_u[i]] for i in range(n_u)])            # [3, 12]
        Md = np.stack([props[(1, site[n_u + i])][a_d[i]] for i in range(len(a_d))])
        du = np.linalg.det(Mu[:, src_u].transpose(1, 0, 2))
        dd = np.linalg.det(Md[:, src_d].transpose(1, 0, 2))
        total += coef * sgn * wsign * np.sum(src_w * du * dd)
    return total * op.norm * op.norm


def test_projected_two_site_term_matches_brute_force():
    """The block expansion with blocks taken at two different sink sites equals the
    quark-level contraction with each baryon's rows taken at its own site."""
    Us, Ds = rand_sites(14, 2)
    plan = bl.BlockPlan("dinucleon_I", "canonical")
    Fx, Fy = plan.factors(Us[0], Ds[0]), plan.factors(Us[1], Ds[1])
    # sink order is (N, P): type N at site x, type P at site y
    hN = bl.TYPE_INDEX["N"]
    first_is_N = plan.ids[:, 0] // bl.N_ETA == hN
    vals = np.where(first_is_N, Fx[plan.ids[:, 0]] * Fy[plan.ids[:, 1]], Fy[plan.ids[:, 0]] * Fx[plan.ids[:, 1]])
    got = vals @ plan.W
    want = two_site_brute_force("dinucleon_I", Us[0], Ds[0], Us[1], Ds[1])
    assert abs(got - want) <= 1e-12 * abs(want)


def test_projected_single_site_lattice_equals_local():
    U, D = mi.workload_fields("proton_4x8", L=1, T=2)
    for name in ("proton", "dinucleon_I"):
        plan = bl.BlockPlan(name, "canonical")
        got = bl.correlator_projected(plan, U, D, 1)
        want = cor.correlator(plan.site_values, U, D)
        np.testing.assert_allclose(got, want, rtol=1e-12)


def test_projected_blocks_translation_phase():
    """Shifting the sink fields by a lattice vector a multiplies F(p) by e^{-i p.a}
    (p in units of 2 pi / L); with p = 0 the projection is the plain site sum."""
    L = 2
    U, D = mi.workload_fields("proton_4x8", L=L, T=1)
    plan = bl.BlockPlan("proton")
    p = (1, 0, 1)
    F = bl.projected_blocks(plan, U, D, L, p)
    xyz = bl.site_coords(L)
    a = np.array([1, 1, 0])
    shifted = ((xyz + a) % L) @ np.array([1, L, L * L])
    Us, Ds = U.copy(), D.copy()
    Us[:, shifted], Ds[:, shifted] = U, D          # field at x moves to x + a
    Fs = bl.projected_blocks(plan, Us, Ds, L, p)
    np.testing.assert_allclose(Fs, F * np.exp(-2j * np.pi * np.dot(p, a) / L), atol=1e-12)
    F0 = bl.projected_blocks(plan, U, D, L)
    np.testing.assert_allclose(F0, plan.factors(U[0], D[0]).sum(axis=0)[None], atol=1e-12)


def test_factor_tree_over_blocks_reproduces_sum():
    """Sec. 4 factor tree built over the merged block terms evaluates to the same sum."""
    plan = bl.BlockPlan("dinucleon_I", "canonical")
    Us, Ds = rand_sites(15, 1)
    F = plan.factors(Us[0], Ds[0])
    terms = [(w, tuple(int(i) for i in ids)) for w, ids in zip(plan.W, plan.ids)]
    f, c, co = ft.build(terms)
    got = ft.evaluate(f, c, co, lambda k: F[k])
    assert abs(got - plan.evaluate(F)) <= 1e-12 * abs(got)
    assert len(co) == plan.n_terms
