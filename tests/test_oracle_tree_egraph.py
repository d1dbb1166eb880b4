"""Pins of the oracle's factor trees and tensor e-graphs against the paper's worked
examples (Figs. 4-5 and the rewrite of Sec. 5) and against plain sums (CPU only)."""
import json
import os

import numpy as np
import pytest

from oracle import correlator as cor
from oracle import egraph as eg
from oracle import factor_tree as ft
from oracle import native
from oracle import operators as ops

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_factor_tree_fig5_arrays():
    g = load("factor_tree_fig5.json")
    terms = [(c, tuple(k)) for c, k in g["terms"]]
    factors, children, coefficients = ft.build(terms)
    assert factors == g["factors"]
    assert children == g["children"]
    assert coefficients == g["coefficients"]


def test_factor_tree_evaluates_expression():
    g = load("factor_tree_fig5.json")
    terms = [(c, tuple(k)) for c, k in g["terms"]]
    rng = np.random.default_rng(0)
    T1, T2 = rng.standard_normal((2, 4, 4, 4))
    val = lambda key: (T1 if key[1] == "1" else T2)[tuple(int(ch) for ch in key.split("_")[1])]
    ref = 5 * T1[1, 2, 2] * T2[2, 3, 2] + T1[1, 2, 3] * T2[2, 3, 2] - T1[1, 2, 3] * T2[3, 2, 3]
    f, c, co = ft.build(terms)
    assert abs(ft.evaluate(f, c, co, val) - ref) < 1e-13
    # the same arrays through the C walker
    ids = {k: i for i, k in enumerate(sorted(set(f[1:])))}
    vals = np.array([val(k) for k in sorted(ids)], dtype=complex)
    got = native.tree([-1] + [ids[k] for k in f[1:]], c, co, vals[None])[0]
    assert abs(got - ref) < 1e-13


def test_factor_tree_merges_and_round_trips():
    rng = np.random.default_rng(1)
    terms = [(int(rng.integers(-3, 4)) or 1, (f"A{rng.integers(3)}", f"B{rng.integers(3)}", f"C{rng.integers(2)}"))
             for _ in range(40)]
    f, c, co = ft.build(terms)
    merged = {}
    for coef, k in terms:
        merged[k] = merged.get(k, 0) + coef
    assert sorted(ft.expand(f, c, co)) == sorted((v, k) for k, v in merged.items())
    assert len(co) == len(merged)          # one leaf per distinct factor string


def test_correlator_factor_tree_matches_canonical(oracle_lib):
    """C_x through the linearised factor tree of the canonical terms (level 1 = up
    minor, level 2 = down minor) equals the canonical sum."""
    op = ops.build("dinucleon_I")
    plan = cor.CanonicalPlan(op)
    n_cu = len(plan.cols_u)
    terms = [(complex(w), (("u", int(mu)), ("d", int(md)))) for mu, md, w in zip(plan.mu, plan.md, plan.W)]
    f, c, co = ft.build(terms)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((2, 12, 12)) + 1j * rng.standard_normal((2, 12, 12))
    D = rng.standard_normal((2, 12, 12)) + 1j * rng.standard_normal((2, 12, 12))
    vu = native.minors(op.n_u, *plan.minor_defs(0), U)
    vd = native.minors(op.n_d, *plan.minor_defs(1), D)
    n_u_minors = vu.shape[1]
    ids = [-1] + [k[1] if k[0] == "u" else n_u_minors + k[1] for k in f[1:]]
    got = native.tree(ids, c, np.array(co), np.concatenate([vu, vd], axis=1))
    ref = plan.site_values(U, D)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    assert len(co) == plan.n_terms and n_cu == 208


def test_egraph_worked_example_canonical_forms():
    g = load("egraph_sec5_example.json")
    to = lambda lst: [(n, tuple(i)) for n, i in lst]
    k1, s1, o1 = eg.canonical(to(g["E1"]), {"eps"})
    k2, s2, o2 = eg.canonical(to(g["E2"]), {"eps"})
    assert k1 == k2                                  # one e-class: B
    assert s1 * s2 == g["relative_sign"]             # relative minus sign
    assert sorted(o1) == ["k", "l"] and o2 == o1[::-1]  # same slots, exchanged: B_kl vs B_lk


def test_egraph_worked_example_extraction():
    g = load("egraph_sec5_example.json")
    E = [(n, tuple(i)) for n, i in g["E"]]
    e = eg.TensorEGraph()
    root, sign, _ = e.add_expr(E)
    e.saturate(root)
    best, cost = e.extract()
    nd = best[root]
    assert nd[0] == "prod" and e.find(nd[1]) == e.find(nd[3])   # E = (+-) B . B
    rng = np.random.default_rng(2)
    T = rng.standard_normal((3, 3, 3))
    tens = {"eps": eg.levi_civita(), "T": T}
    val = sign * e.evaluate(root, tens, best)
    B = np.einsum("ijk,ijl->kl", tens["eps"], T)
    assert abs(val - (-np.einsum("kl,lk->", B, B))) < 1e-12
    assert abs(val - np.einsum("ijk,lmn,ijl,nmk->", tens["eps"], tens["eps"], T, T)) < 1e-12
    assert cost[e.find(root)] < eg.flops(E)


def test_egraph_random_expression():
    E = [("eps", ("i", "j", "k")), ("T", ("i", "j", "l")), ("T", ("k", "m", "n")), ("S", ("l", "m")),
         ("S", ("n", "p")), ("eps", ("p", "q", "r")), ("S", ("q", "r"))]
    e = eg.TensorEGraph()
    root, sign, _ = e.add_expr(E)
    e.saturate(root)
    best, _ = e.extract()
    rng = np.random.default_rng(4)
    tens = {"eps": eg.levi_civita(), "T": rng.standard_normal((3, 3, 3)), "S": rng.standard_normal((3, 3))}
    ref = eg.einsum_expr(E, tens, [])
    assert abs(sign * e.evaluate(root, tens, best) - ref) < 1e-10 * max(1, abs(ref))


@pytest.mark.parametrize("name", ["proton", "dinucleon_I"])
def test_minor_egraph_plan_matches_lu(oracle_lib, name):
    """Laplace sub-minor plan extracted from the determinant e-graph reproduces every
    minor the canonical form needs."""
    op = ops.build(name)
    plan = cor.CanonicalPlan(op)
    rng = np.random.default_rng(5)
    M = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    for flav, k in ((0, op.n_u), (1, op.n_d)):
        rows, cols = plan.minor_defs(flav)
        roots = [(tuple(int(v) for v in r), tuple(int(v) for v in c)) for r, c in zip(rows, cols)]
        g = eg.MinorEGraph()
        g.saturate(roots)
        p = g.extract(roots)
        got = np.array(g.evaluate(p, M, roots))
        ref = native.minors(k, rows, cols, M[None])[0]
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)
        n_sub = sum(1 for key in p if len(key[0]) == k - 1) if k > 1 else 0
        assert k == 1 or n_sub < len(roots) * k      # sub-minors are shared
