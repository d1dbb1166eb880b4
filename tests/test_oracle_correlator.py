"""Pins of the oracle's correlator: brute force, closed forms and invariants (CPU only)."""
import numpy as np
import pytest

import mbc_inputs as mi
from oracle import canonical as can
from oracle import correlator as cor
from oracle import operators as ops
from oracle.wick import wick_sign


def sub_operator(op, n_per_j, seed=0):
    """A random subset of an operator's sink terms (same slots, same weights)."""
    rng = np.random.default_rng(seed)
    terms = []
    for t in op.terms:
        keys = sorted(t)
        pick = rng.choice(len(keys), size=min(n_per_j, len(keys)), replace=False) if keys else []
        terms.append({keys[i]: t[keys[i]] for i in pick})
    return ops.Operator(op.name + "_sub", op.n_u, op.n_d, terms, op.proj, op.norm)


def rand_props(seed, n=1, scale=1.0):
    rng = np.random.default_rng(seed)
    U = (rng.standard_normal((n, 12, 12)) + 1j * rng.standard_normal((n, 12, 12))) * scale
    D = (rng.standard_normal((n, 12, 12)) + 1j * rng.standard_normal((n, 12, 12))) * scale
    return U, D


def close(a, b, rtol=1e-12):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= rtol * np.maximum(np.abs(b), 1e-300) + 1e-300)


def test_proton_three_ways(oracle_lib):
    op = ops.build("proton")
    U, D = rand_props(1)
    a = cor.site_pairings(op, U[0], D[0])
    b = cor.site_direct(op, U, D)[0]
    c = cor.CanonicalPlan(op).site_values(U, D)[0]
    assert close(b, a) and close(c, a)


@pytest.mark.parametrize("name,n", [("dinucleon_I", 40), ("he3_I", 5), ("he3_II_s", 4)])
def test_subsets_pairings_vs_direct_vs_canonical(oracle_lib, name, n):
    """Brute-force Wick pairings (n_u! n_d! per term) against the determinant sums."""
    op = sub_operator(ops.build(name), n, seed=3)
    U, D = rand_props(2)
    a = cor.site_pairings(op, U[0], D[0])
    b = cor.site_direct(op, U, D)[0]
    c = cor.CanonicalPlan(op).site_values(U, D)[0]
    assert close(b, a, 1e-11) and close(c, a, 1e-11)


def test_dinucleon_direct_vs_canonical(oracle_lib):
    op = ops.build("dinucleon_I")
    U, D = rand_props(4, n=2)
    a = cor.site_direct(op, U, D, n_threads=2)
    b = cor.CanonicalPlan(op).site_values(U, D)
    assert close(b, a, 1e-12)


def canonical_inner(op, lam_u=None, lam_d=None):
    """Closed form for identity (lam = 1) or diagonal propagators: det diag(lam)[R, C] =
    delta_RC prod_{r in R} lam_r for ascending R, C."""
    snk = [can.canonical_side(t) for t in op.terms]
    tot = 0j
    for j, k, p in can.pairs(op.proj):
        for key, a in snk[j].items():
            b = snk[k].get(key)
            if b is None:
                continue
            f = 1.0
            if lam_u is not None:
                f = np.prod([lam_u[r] for r in key[0]]) * np.prod([lam_d[r] for r in key[1]])
            tot += p * a * np.conj(b) * f
    return wick_sign(op.n_u + op.n_d) * op.norm ** 2 * tot


@pytest.mark.parametrize("name", ["proton", "dinucleon_I", "he3_I"])
def test_identity_and_diagonal_closed_forms(oracle_lib, name):
    op = ops.build(name)
    if name == "he3_I":
        op = sub_operator(op, 400, seed=9)
    I = np.eye(12)[None].astype(complex)
    got = cor.site_direct(op, I, I)[0]
    assert close(got, canonical_inner(op), 1e-12)
    rng = np.random.default_rng(8)
    lu = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    ld = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    got = cor.site_direct(op, np.diag(lu)[None], np.diag(ld)[None])[0]
    assert close(got, canonical_inner(op, lu, ld), 1e-12)


def test_scaling_and_phase(oracle_lib):
    op = sub_operator(ops.build("he3_I"), 30, seed=1)
    plan = cor.CanonicalPlan(op)
    U, D = rand_props(6)
    c0 = plan.site_values(U, D)[0]
    s = 0.37
    assert close(plan.site_values(s * U, s * D)[0], s ** 9 * c0, 1e-12)
    phi = 0.7
    assert close(plan.site_values(np.exp(1j * phi) * U, D)[0], np.exp(5j * phi) * c0, 1e-12)


def colour_rotate(S, g, h):
    """S -> g S h^dagger acting on the colour part of i = 3*spin + colour."""
    G = np.kron(np.eye(4), g)
    H = np.kron(np.eye(4), h)
    return G @ S @ H.conj().T


@pytest.mark.parametrize("name", ["proton", "dinucleon_I", "he3_I", "he3_II_s"])
def test_colour_invariance(oracle_lib, name):
    """Every operator is a product of eps colour singlets, so C is unchanged by a
    sink-site SU(3) rotation g and a source rotation h (the same for both flavours)."""
    op = ops.build(name)
    plan = cor.CanonicalPlan(op)
    U, D = rand_props(10, n=2)
    rng = np.random.default_rng(12)
    g = mi.su3_random(rng, 2)
    h = mi.su3_random(rng, 1)[0]
    Ur = np.stack([colour_rotate(U[x], g[x], h) for x in range(2)])
    Dr = np.stack([colour_rotate(D[x], g[x], h) for x in range(2)])
    assert close(plan.site_values(Ur, Dr), plan.site_values(U, D), 1e-10)


def test_antisymmetry_under_slot_exchange(oracle_lib):
    """Swapping two up slots of every sink tuple (source unchanged) flips C."""
    op = sub_operator(ops.build("he3_I"), 25, seed=4)
    snk, src = cor.sides(op)
    sw = []
    for idx, w in snk:
        idx2 = idx.copy()
        idx2[:, [0, 2]] = idx2[:, [2, 0]]
        sw.append((idx2, w))
    from oracle import native
    U, D = rand_props(13)
    a = native.direct(op.n_u, op.n_d, snk, src, op.proj, U, D)[0]
    b = native.direct(op.n_u, op.n_d, sw, src, op.proj, U, D)[0]
    assert close(b, -a, 1e-12)


@pytest.mark.parametrize("name", ["dinucleon_II", "he3_II"])
def test_printed_spin_isospin_operators_vanish(oracle_lib, name):
    """D_II and 3He_II of Eq. 2 are identically zero: their canonical term sets are empty
    and their direct sum is rounding residue only (measured against sum |terms|)."""
    op = ops.build(name)
    assert cor.CanonicalPlan(op).n_terms == 0
    assert all(len(can.canonical_side(t)) == 0 for t in op.terms)
    if name == "dinucleon_II":
        U, D = rand_props(14)
        v = cor.site_direct(op, U, D)[0]
        ref = cor.site_direct(ops.build("dinucleon_I"), U, D)[0]
        assert abs(v) < 1e-10 * abs(ref)


def test_synthetic_inputs_regenerate_per_site():
    full = mi.propagator_field(1, 0, 0, T=2, V3=8)
    one = mi.site_matrices(1, 0, 0, 1, [5])
    assert np.array_equal(full[1, 5], one[0])
    assert not np.allclose(mi.site_matrices(1, 0, 1, 1, [5]), one)   # flavours differ
    # exp(-kappa t) envelope and unit variance per component pair
    g = mi.site_matrices(2, 0, 0, 0, np.arange(2000)).ravel()
    assert abs(np.mean(np.abs(g) ** 2) - 1.0) < 0.02
    assert np.allclose(mi.site_matrices(2, 0, 0, 4, [3], kappa=0.5) * np.exp(2.0), mi.site_matrices(2, 0, 0, 4, [3], kappa=0.0))
    b = mi.site_matrices(2, 0, 0, 3, [0, 1], kappa=0.3, noise=1e-3)
    assert np.abs(b[0] - b[1]).max() < 1e-2 * np.abs(b[0]).max()


def test_momentum_projection_pins(oracle_lib):
    """Sink momentum (Sec. 2 projection phase): p = 0 is the plain site sum; the sum over
    all L^3 momenta is L^3 times the value at site 0 (discrete Fourier inversion);
    translating the fields by a multiplies C(p) by e^{-i 2 pi p.a / L}."""
    L = 2
    U, D = mi.workload_fields("proton_4x8", L=L, T=2)
    plan = cor.CanonicalPlan(ops.build("proton"))
    c0 = cor.correlator(plan.site_values, U, D)
    assert close(cor.correlator_momentum(plan.site_values, U, D, L, (0, 0, 0)), c0)
    total = sum(cor.correlator_momentum(plan.site_values, U, D, L, (a, b, c))
                for a in range(L) for b in range(L) for c in range(L))
    site0 = plan.site_values(U[:, 0], D[:, 0])
    assert close(total, L ** 3 * site0)
    p, a = (1, 0, 1), np.array([1, 1, 0])
    x = np.arange(L ** 3)
    xyz = np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)
    moved = ((xyz + a) % L) @ np.array([1, L, L * L])
    Us, Ds = U.copy(), D.copy()
    Us[:, moved], Ds[:, moved] = U, D
    cp = cor.correlator_momentum(plan.site_values, U, D, L, p)
    cs = cor.correlator_momentum(plan.site_values, Us, Ds, L, p)
    assert close(cs, cp * np.exp(-2j * np.pi * np.dot(p, a) / L))
