"""Pins of the oracle's Dirac algebra, determinants and Wick signs (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle import dirac, wick
from oracle import operators as ops


def test_dirac_algebra():
    I4 = np.eye(4)
    for mu, g in enumerate(dirac.GAMMA):
        assert np.allclose(g @ g, I4)
        assert np.allclose(g, g.conj().T)
        # charge conjugation: C gamma_mu C^-1 = -gamma_mu^T
        assert np.allclose(dirac.C @ g @ np.linalg.inv(dirac.C), -g.T)
        for nu, h in enumerate(dirac.GAMMA):
            if nu != mu:
                assert np.allclose(g @ h + h @ g, 0)
        assert np.allclose(dirac.G5 @ g + g @ dirac.G5, 0)
    # C gamma_5 is antisymmetric: the fact that makes D_II and 3He_II vanish
    assert np.allclose(dirac.CG5, -dirac.CG5.T)
    assert np.allclose(dirac.P_PLUS @ dirac.P_PLUS, dirac.P_PLUS)
    assert np.allclose(dirac.P_PLUS + dirac.P_MINUS, I4)
    assert np.allclose(dirac.P_PLUS @ dirac.P_MINUS, 0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_det_lu_matches_leibniz(n):
    rng = np.random.default_rng(n)
    for _ in range(3):
        m = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        ref = wick.det_leibniz(m)
        assert abs(wick.det_lu(m) - ref) <= 1e-12 * max(1.0, abs(ref)) * 10
        assert abs(np.linalg.det(m) - ref) <= 1e-12 * max(1.0, abs(ref)) * 10


def test_native_det_matches_leibniz(oracle_lib):
    rng = np.random.default_rng(7)
    for n in range(1, 7):
        m = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        ref = wick.det_leibniz(m)
        assert abs(oracle_lib.det(m) - ref) <= 1e-11 * max(1.0, abs(ref))


def test_det_exact_zero_and_pivoting(oracle_lib):
    rng = np.random.default_rng(3)
    m = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    m[3] = m[1]                       # repeated row: a zero-det index tuple
    assert wick.det_lu(m) == 0 or abs(wick.det_lu(m)) < 1e-14
    z = np.zeros((3, 3), complex)
    assert wick.det_lu(z) == 0 and oracle_lib.det(z) == 0
    # a zero leading entry needs a row swap: det [[0,1],[1,0]] = -1
    p = np.array([[0, 1], [1, 0]], complex)
    assert wick.det_lu(p) == -1 and oracle_lib.det(p) == -1


def _grouped_contraction(fields_q, fields_qb, U, D):
    """Contraction via the flavour-grouped determinant form with the reordering signs."""
    def group(fs):
        order = [k for k, f in enumerate(fs) if f[0] == 0] + [k for k, f in enumerate(fs) if f[0] == 1]
        return wick.perm_sign(order), [fs[k][1] for k in order if fs[k][0] == 0], \
            [fs[k][1] for k in order if fs[k][0] == 1]
    s1, au, ad = group(fields_q)
    s2, bu, bd = group(fields_qb)
    if len(au) != len(bu):
        return 0
    return s1 * s2 * wick.contraction(au, ad, bu, bd, U, D, det=wick.det_leibniz)


def test_pairing_sum_equals_signed_determinants():
    """The Wick sum taken literally (Grassmann pairings) against the determinant form:
    pins (-1)^{n(n-1)/2} and the flavour-grouping signs."""
    rng = np.random.default_rng(11)
    U = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    D = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    for n_u, n_d in [(1, 0), (2, 0), (1, 1), (2, 1), (3, 1), (2, 2), (3, 3), (4, 2)]:
        for _ in range(3):
            fl = [0] * n_u + [1] * n_d
            q = [(f, int(rng.integers(12))) for f in rng.permutation(fl)]
            qb = [(f, int(rng.integers(12))) for f in rng.permutation(fl)]
            a = wick.pairings(q, qb, {0: U, 1: D})
            b = _grouped_contraction(q, qb, U, D)
            assert abs(a - b) <= 1e-11 * max(1.0, abs(a))


def test_proton_block_closed_form():
    """Sec. 2, Eq. 3: <u^a_b d^b_g u^c_al ubar^a'_b' dbar^b'_g' ubar^c'_al'> equals
    [S^u_(a b)(c' al') S^u_(c al)(a' b') - S^u_(a b)(a' b') S^u_(c al)(c' al')] S^d_(b g)(b' g')."""
    rng = np.random.default_rng(5)
    U = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    D = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    ix = lambda colour, spin: 3 * spin + colour
    for _ in range(20):
        a, b, c, a2, b2, c2 = rng.integers(3, size=6)
        be, ga, al, be2, ga2, al2 = rng.integers(4, size=6)
        q = [(0, ix(a, be)), (1, ix(b, ga)), (0, ix(c, al))]
        qb = [(0, ix(a2, be2)), (1, ix(b2, ga2)), (0, ix(c2, al2))]
        lhs = wick.pairings(q, qb, {0: U, 1: D})
        rhs = (U[ix(a, be), ix(c2, al2)] * U[ix(c, al), ix(a2, be2)]
               - U[ix(a, be), ix(a2, be2)] * U[ix(c, al), ix(c2, al2)]) * D[ix(b, ga), ix(b2, ga2)]
        assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


def test_operator_term_counts():
    """Closed-form expansion sizes: eps has 6 nonzeros, C g5 has 4, C g5 P_+- has 2."""
    p = ops.build("proton")
    assert p.raw_counts == [6 * 4] * 4
    d1 = ops.build("dinucleon_I")
    assert d1.raw_counts == [4 * 24 * 24]
    h = ops.build("he3_I")
    assert h.raw_counts == [4 * 12 * 12 * 12] * 4
    h2 = ops.build("he3_II")
    assert h2.raw_counts == [6 * 6912] * 4
    assert (p.n_u, p.n_d, d1.n_u, d1.n_d, h.n_u, h.n_d) == (2, 1, 3, 3, 5, 4)
    for name in ops.NAMES:
        op = ops.build(name)
        for t in op.terms:
            for w in t.values():       # merged weights stay Gaussian integers (exact merging)
                assert w.real == int(w.real) and w.imag == int(w.imag)


def test_grouping_sign():
    # u d u -> (u u)(d): one transposition
    s, au, ad = ops.grouped(((0, 0, 1), (1, 1, 2), (0, 2, 3)))
    assert s == -1 and au == (3 * 1 + 0, 3 * 3 + 2) and ad == (3 * 2 + 1,)
    # d u d u: order (1, 3, 0, 2) has 3 inversions
    s, au, ad = ops.grouped(((1, 0, 0), (0, 0, 0), (1, 1, 0), (0, 1, 0)))
    assert s == -1
