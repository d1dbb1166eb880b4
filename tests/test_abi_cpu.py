"""CPU-only checks of libmbc: the library loads, exports every entry point declared in
include/mbc.h, and its host planner (operator library, canonical form, factor tree,
minor e-graph, plan files, argument checks) agrees with the oracle.  No GPU needed:
plans are built in a host-only context (device -1)."""
import os
import re

import numpy as np
import pytest

from oracle import canonical as ocan
from oracle import correlator as ocor
from oracle import operators as oops
from oracle.wick import wick_sign

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2201_04269_gb300 import build
    build.build()
    from paper_2201_04269_gb300 import abi as a
    a.load()
    return a


@pytest.fixture(scope="module")
def hctx(abi):
    ctx = abi.mbc_create(-1)
    yield ctx
    abi.mbc_destroy(ctx)


def header_functions():
    src = open(os.path.join(ROOT, "include", "mbc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mbc_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(abi):
    lib = abi.load()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert {s[0] for s in abi.SIGNATURES} == set(names)
    assert abi.mbc_version().startswith("mbc")


@pytest.mark.parametrize("name", oops.NAMES)
def test_operator_library_matches_oracle(abi, name):
    t = abi.mbc_operator_terms(name)
    op = oops.build(name)
    assert (t["n_u"], t["n_d"], t["n_free"]) == (op.n_u, op.n_d, op.n_free)
    for j in range(op.n_free):
        idx, w = op.arrays(j)
        a, b = t["offsets"][j], t["offsets"][j + 1]
        assert np.array_equal(t["idx"][a:b], idx)
        assert np.array_equal(t["w"][a:b], w / op.norm)          # unnormalised Gaussian integers
    assert np.array_equal(t["proj"], op.proj)
    assert t["scale"] == pytest.approx(wick_sign(op.n_u + op.n_d) * op.norm ** 2, rel=1e-15)


def plan_of(abi, ctx, name, algo="tree", prec="fp64"):
    t = abi.mbc_operator_terms(name)
    return abi.mbc_plan_create(ctx, t["n_u"], t["n_d"], t["idx"], t["w"], t["offsets"], t["idx"], t["w"],
                               t["offsets"], t["proj"], t["scale"], algo, prec), t


@pytest.mark.parametrize("name", ["proton", "neutron", "dinucleon_I", "dinucleon_II", "he3_I", "he3_II_s"])
def test_plan_counts_match_oracle(abi, hctx, name):
    plan, t = plan_of(abi, hctx, name)
    info = abi.mbc_plan_get_info(plan)
    op = oops.build(name)
    cp = ocor.CanonicalPlan(op)
    nnz = [len(x) for x in op.terms]
    assert info["index_size"] == sum(nnz[j] * nnz[k] for j, k, _ in ocan.pairs(op.proj))
    assert info["canonical_terms"] == cp.n_terms
    assert (info["rows_u"], info["rows_d"]) == (len(cp.rows_u), len(cp.rows_d))
    assert info["tree_nodes"] == (1 + len(set(cp.mu)) + cp.n_terms if cp.n_terms else 1)
    abi.mbc_plan_destroy(plan)


@pytest.mark.parametrize("name", ["proton", "dinucleon_I"])
def test_factor_tree_matches_oracle_terms(abi, hctx, name):
    """Expanding the product's linearised tree gives exactly the oracle's canonical
    terms (minor row/column sets and weights, scale folded)."""
    plan, t = plan_of(abi, hctx, name)
    f, ch, co = abi.mbc_plan_get_tree(plan)
    info = abi.mbc_plan_get_info(plan)
    op = oops.build(name)
    n_umin = info["minors_u"]
    got = {}
    k, leaf = 1, 0
    assert f[0] == -1 and ch[0] > 0
    while k < len(f):
        mu = abi.mbc_plan_get_minor(plan, 0, int(f[k]), op.n_u)
        n = ch[k]
        k += 1
        for _ in range(n):
            md = abi.mbc_plan_get_minor(plan, 1, int(f[k]) - n_umin, op.n_d)
            got[(mu, md)] = co[leaf] * t["scale"]
            k += 1
            leaf += 1
    ref = {}
    for ru, rd, cu, cd, w in ocan.canonical_terms(op):
        ref[((ru, cu), (rd, cd))] = w
    assert got.keys() == ref.keys()
    for key in ref:
        assert abs(got[key] - ref[key]) <= 1e-14 * abs(ref[key])
    # children in lexicographic order of the factors (Sec. 4, Fig. 5 ordering)
    l1 = [abi.mbc_plan_get_minor(plan, 0, int(f[i]), op.n_u) for i in np.nonzero(ch)[0][1:]]
    assert l1 == sorted(l1)
    abi.mbc_plan_destroy(plan)


def test_explicit_terms_plan(abi, hctx):
    """mbc_plan_from_terms canonicalises an explicit index set: (a, a') and its slot
    permutations merge with the permutation signs, zero-det tuples drop."""
    sink = np.array([[0, 1, 2], [1, 0, 2], [0, 0, 2]], np.int8)
    source = np.array([[3, 4, 5], [3, 4, 5], [3, 4, 5]], np.int8)
    W = np.array([1.0, 1.0, 5.0], complex)
    plan = abi.mbc_plan_from_terms(hctx, 2, 1, sink, source, W, 1.0, "tree", "fp64")
    info = abi.mbc_plan_get_info(plan)
    assert info["index_size"] == 3
    assert info["canonical_terms"] == 0      # (0,1) and (1,0) cancel, (0,0) vanishes
    abi.mbc_plan_destroy(plan)
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_from_terms(hctx, 2, 1, sink, source, W, 1.0, "egraph", "fp64")
    assert e.value.status == 2


def test_argument_errors(abi, hctx):
    t = abi.mbc_operator_terms("proton")
    bad = t["idx"].copy()
    bad[0, 0] = 12
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_create(hctx, 2, 1, bad, t["w"], t["offsets"], t["idx"], t["w"], t["offsets"], t["proj"], -1.0,
                            "direct", "fp64")
    assert e.value.status == 2 and "0..11" in abi.mbc_last_error(hctx)
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_create(hctx, 7, 1, t["idx"], t["w"], t["offsets"], t["idx"], t["w"], t["offsets"], t["proj"],
                            -1.0, "direct", "fp64")
    assert e.value.status == 2
    off = t["offsets"].copy()
    off[2] = off[1] - 1
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_create(hctx, 2, 1, t["idx"], t["w"], off, t["idx"], t["w"], t["offsets"], t["proj"], -1.0,
                            "direct", "fp64")
    assert e.value.status == 1
    w = t["w"].copy()
    w[0] = np.nan
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_create(hctx, 2, 1, t["idx"], w, t["offsets"], t["idx"], t["w"], t["offsets"], t["proj"], -1.0,
                            "direct", "fp64")
    assert e.value.status == 6
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_create(hctx, 2, 1, t["idx"], t["w"], t["offsets"], t["idx"], t["w"], t["offsets"], t["proj"],
                            -1.0, "direct", "quad")
    plan, _ = plan_of(abi, hctx, "proton", "egraph")
    with pytest.raises(abi.MbcError) as e:     # a host-only context cannot evaluate
        abi.mbc_correlator(plan, 1, 1, 1, 1, 1, 1, ctx=hctx)
    assert e.value.status == 2
    abi.mbc_plan_destroy(plan)


def test_plan_file_round_trip(abi, hctx, tmp_path):
    plan, t = plan_of(abi, hctx, "dinucleon_I", "egraph", "mixed")
    p = str(tmp_path / "d1.mbcplan")
    abi.mbc_plan_save(plan, p, hctx)
    plan2 = abi.mbc_plan_load(hctx, p)
    assert abi.mbc_plan_get_info(plan2) == abi.mbc_plan_get_info(plan)
    a = abi.mbc_plan_get_tree(plan)
    b = abi.mbc_plan_get_tree(plan2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    with open(p, "r+b") as f:
        f.truncate(100)
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_load(hctx, p)
    assert e.value.status == 7
    with pytest.raises(abi.MbcError):
        abi.mbc_plan_load(hctx, str(tmp_path / "missing"))
    abi.mbc_plan_destroy(plan)
    abi.mbc_plan_destroy(plan2)


@pytest.mark.parametrize("n_u,n_d,seed", [(1, 1, 0), (2, 1, 1), (3, 2, 2), (4, 4, 3), (6, 0, 4), (2, 5, 5), (6, 6, 6)])
def test_planner_on_random_factored_problems(abi, hctx, n_u, n_d, seed):
    """Random factored problems (repeated indices, Gaussian-integer weights, a projector with
    zeros): the planner's linearised tree expands to exactly the oracle's canonical terms
    (row and column sets, merged weights, Wick sign), and every algorithm's plan passes the
    structural checks."""
    rng = np.random.default_rng(seed)
    n_free, per_j = 2, 12
    terms = []
    for j in range(n_free):
        d = {}
        for _ in range(per_j):
            a_u = tuple(int(v) for v in rng.integers(0, 12, n_u))
            a_d = tuple(int(v) for v in rng.integers(0, 12, n_d))
            w = complex(int(rng.integers(-3, 4)), int(rng.integers(-2, 3)))
            if w != 0:
                d[(a_u, a_d)] = d.get((a_u, a_d), 0) + w
        terms.append({k: v for k, v in d.items() if v != 0})
    proj = np.array([[1.0, 0.5j], [0.0, -2.0]], dtype=np.complex128)
    op = oops.Operator("random", n_u, n_d, terms, proj, 1.0)
    idx, w, off = [], [], [0]
    for j in range(n_free):
        a, b = op.arrays(j)
        idx.append(a.reshape(-1, n_u + n_d))
        w.append(b)
        off.append(off[-1] + len(b))
    idx, w, off = np.concatenate(idx), np.concatenate(w), np.array(off)
    scale = wick_sign(n_u + n_d)
    for algo in ("direct", "tree", "egraph"):
        plan = abi.mbc_plan_create(hctx, n_u, n_d, idx, w, off, idx, w, off, proj, scale, algo, "fp64")
        abi.mbc_plan_destroy(plan)
    plan = abi.mbc_plan_create(hctx, n_u, n_d, idx, w, off, idx, w, off, proj, scale, "tree", "fp64")
    f, ch, co = abi.mbc_plan_get_tree(plan)
    n_umin = abi.mbc_plan_get_info(plan)["minors_u"]
    got = {}
    k, leaf = 1, 0
    while k < len(f):
        mu = abi.mbc_plan_get_minor(plan, 0, int(f[k]), n_u)
        n = ch[k]
        k += 1
        for _ in range(n):
            md = abi.mbc_plan_get_minor(plan, 1, int(f[k]) - n_umin, n_d)
            got[(mu, md)] = co[leaf] * scale
            k += 1
            leaf += 1
    ref = {((ru, cu), (rd, cd)): wv for ru, rd, cu, cd, wv in ocan.canonical_terms(op)}
    assert got.keys() == ref.keys()
    for key in ref:
        assert abs(got[key] - ref[key]) <= 1e-12 * max(1.0, abs(ref[key]))
    abi.mbc_plan_destroy(plan)


def test_damaged_plan_files_are_rejected_on_the_host(abi, hctx, tmp_path):
    """A plan file whose index arrays were damaged must fail to load (every index a kernel
    uses is checked on the host), or load as a plan that passes the same checks."""
    plan, _ = plan_of(abi, hctx, "proton", "egraph", "fp64")
    p = str(tmp_path / "p.mbcplan")
    abi.mbc_plan_save(plan, p, hctx)
    abi.mbc_plan_destroy(plan)
    raw = open(p, "rb").read()
    rng = np.random.default_rng(5)
    detected = 0
    for k in range(60):
        buf = bytearray(raw)
        pos = int(rng.integers(8, len(buf)))
        buf[pos] ^= 0xFF
        q = str(tmp_path / f"bad{k}.mbcplan")
        open(q, "wb").write(bytes(buf))
        try:
            ok = abi.mbc_plan_load(hctx, q)
            abi.mbc_plan_get_info(ok)
            abi.mbc_plan_destroy(ok)
        except abi.MbcError as e:
            assert e.status in (1, 2, 3, 7)
            detected += "damaged plan file" in abi.mbc_last_error(hctx)
    assert detected > 0


@pytest.mark.parametrize("name", ["dinucleon_I", "he3_I", "he3_II_s"])
def test_minor_egraph_size_and_flops(abi, hctx, name):
    """The extracted Laplace plan costs less than one LU per minor, and the saturated
    e-graph holds every (row subset, column subset) class of each level."""
    plan, _ = plan_of(abi, hctx, name, "egraph")
    info = abi.mbc_plan_get_info(plan)
    assert info["egraph_classes"] > info["minors_u"]
    assert 0 < info["flops_per_site"] < info["direct_flops_per_site"]
    tree_plan, _ = plan_of(abi, hctx, name, "tree")
    assert info["flops_per_site"] < abi.mbc_plan_get_info(tree_plan)["flops_per_site"]
    abi.mbc_plan_destroy(plan)
    abi.mbc_plan_destroy(tree_plan)


def test_fp32_plan_settings_on_the_host(abi, hctx):
    """MBC_PREC_FP32 plans on a host-only context: FP32 is accepted only for the e-graph
    algorithm; guard settings round-trip (NaN rejected); kernel shapes are validated
    (threads a multiple of 128 up to 768, one or two blocks per site, leaf batch 1..3)."""
    plan, _ = plan_of(abi, hctx, "he3_II_s", "egraph", "fp32")
    assert abi.mbc_plan_get_guard(plan) == (2.0, 1e-6)
    abi.mbc_plan_set_guard(plan, 3.5, 2e-6, hctx)
    assert abi.mbc_plan_get_guard(plan) == (3.5, 2e-6)
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_plan_set_guard(plan, float("nan"), 1e-6, hctx)
    assert e.value.status == 1
    assert abi.mbc_plan_get_guard(plan) == (3.5, 2e-6)
    for bad in ((100, 1, 3), (896, 1, 3), (640, 3, 3), (640, 1, 4), (640, 0, 1)):
        with pytest.raises(abi.MbcError):
            abi.mbc_set_schedule(plan, *bad, ctx=hctx)
    abi.mbc_set_schedule(plan, 512, 2, 2, ctx=hctx)
    assert abi.mbc_get_schedule(plan) == dict(threads=512, blocks_per_sm=2, sites_per_unit=2)
    for algo in ("direct", "tree"):
        with pytest.raises(abi.MbcError) as e:
            plan_of(abi, hctx, "proton", algo, "fp32")
        assert e.value.status == 2                          # MBC_UNSUPPORTED
    abi.mbc_plan_destroy(plan)
