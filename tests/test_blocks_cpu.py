"""CPU-only checks of the block planner of libmbc (host-only context): the expanded and
merged block form of each library operator agrees with the oracle's construction
(arXiv 2201.04269 Sec. 3), term by term, and the argument checks of the block entry
points reject bad input without touching a device."""
import numpy as np
import pytest

from oracle import blocks as obl


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


@pytest.mark.parametrize("name", ["proton", "neutron", "dinucleon_I", "dinucleon_II", "he3_I"])
def test_block_plan_matches_oracle(abi, hctx, name):
    ref = obl.BlockPlan(name, "canonical")
    plan = abi.mbc_block_plan_create(hctx, name)
    info = abi.mbc_block_plan_get_info(plan)
    assert info["n_w"] == ref.n_w
    assert info["n_baryons"] == ref.A
    assert info["expanded_terms"] == ref.n_expanded
    assert info["merged_terms"] == ref.n_terms
    ids, w = abi.mbc_block_plan_get_terms(plan)
    assert np.array_equal(ids, ref.ids)
    np.testing.assert_allclose(w, ref.W, rtol=1e-15, atol=0)
    assert np.array_equal(abi.mbc_block_plan_get_multiplicities(plan), ref.multiplicity)
    # factors and factor-tree levels from the merged terms
    assert info["factors"] == len(np.unique(ref.ids)) if ref.n_terms else info["factors"] == 0
    for a in range(ref.A):
        n = len(np.unique(ref.ids[:, :a + 1], axis=0)) if ref.n_terms else 0
        assert info["level_nodes"][a] == n
    abi.mbc_block_plan_destroy(plan)


def test_block_counts_of_the_paper(abi, hctx):
    """N_w = 9 for dinucleon I (Sec. 3) and 360 per product for 3He."""
    p = abi.mbc_block_plan_create(hctx, "dinucleon_I")
    assert abi.mbc_block_plan_get_info(p)["n_w"] == [9]
    abi.mbc_block_plan_destroy(p)
    p = abi.mbc_block_plan_create(hctx, "he3_II_s")
    info = abi.mbc_block_plan_get_info(p)
    assert info["n_w"] == [360, 360, 360] and info["n_baryons"] == 3 and info["merged_terms"] > 0
    abi.mbc_block_plan_destroy(p)


def test_block_argument_errors(abi, hctx):
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_block_plan_create(hctx, "no_such_operator")
    assert e.value.status == 1
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_block_plan_create(hctx, "proton", "no_such_precision")
    assert e.value.status == 1
    abi.mbc_block_plan_destroy(abi.mbc_block_plan_create(hctx, "proton", "mixed"))
    # a host-only context cannot evaluate (checked before any pointer is used)
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_hadron_blocks(hctx, "P", 1, 1, 1, 1)
    assert e.value.status == 2
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_hadron_blocks_projected(hctx, "N", 1, 1, 1, 1, 2, 1)
    assert e.value.status == 2
    p = abi.mbc_block_plan_create(hctx, "proton")
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_block_correlator(p, 1, 1, 1, 1, 2, 1, ctx=hctx)
    assert e.value.status == 2
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_block_correlator(p, 1, 1, -1, 1, 2, 1, ctx=hctx)
    assert e.value.status == 1
    abi.mbc_block_plan_destroy(p)


@pytest.mark.parametrize("name", ["dinucleon_I", "he3_I"])
def test_shared_leaf_sums_match_oracle(abi, hctx, name):
    """The planner's hash-consing of the factor tree's level-(A-2) vertices by their leaf
    sums (Sec. 5's congruence on the block terms) counts the same distinct sums, and the
    same leaf terms among them, as a plain grouping of the oracle's merged terms."""
    ref = obl.BlockPlan(name, "canonical")
    A = ref.A
    prefix = ref.ids[:, :A - 1]
    starts = np.flatnonzero(np.r_[True, np.any(prefix[1:] != prefix[:-1], axis=1)])
    ends = np.r_[starts[1:], len(ref.W)]
    sums = {tuple(zip(ref.ids[a:b, A - 1].tolist(), ref.W[a:b].tolist())) for a, b in zip(starts, ends)}
    plan = abi.mbc_block_plan_create(hctx, name)
    info = abi.mbc_block_plan_get_info(plan)
    assert info["level_nodes"][A - 2] == len(starts)
    assert info["shared_sums"] == len(sums)
    assert info["shared_sum_terms"] == sum(len(s) for s in sums)
    abi.mbc_block_plan_destroy(plan)
