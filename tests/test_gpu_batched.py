"""Batched evaluation in the FP32 arithmetic (MBC_PREC_FP32) through mbc_batch: a small
batch of every operator against separate calls and the oracle, and the batched workload
at its stated size -- 64 propagator sets (16 configurations x 4 source times), the five
operators, sets 0-31 on 16^3 x 32 and 32-63 on 24^3 x 48 (about 117 GB of fields,
generated on the GPU by the seeded recipe) -- in one persistent launch, with sampled sites
of every item checked against the oracle (needs a GB300; marked gpu)."""
import numpy as np
import pytest

import mbc_inputs as mi
from oracle import correlator as ocor
from oracle import native as onat
from oracle import operators as oops

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OPS = ("proton", "dinucleon_I", "dinucleon_II", "he3_I", "he3_II")
SITE_TOL = 1e-5           # per-site, the mixed-arithmetic tolerance
C_TOL = 1e-6              # C(t) of the FP32 path against the double-float path


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04269_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


_oracles = {}


def oracle_sites(name, U, D):
    if name not in _oracles:
        _oracles[name] = ocor.CanonicalPlan(oops.build(name))
    return _oracles[name].site_values(U.reshape(-1, 12, 12), D.reshape(-1, 12, 12), n_threads=onat.max_threads())


def relerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.maximum(np.abs(b), 1e-300)))


def test_fp32_batch_matches_separate_calls_and_oracle(ctx):
    from paper_2201_04269_gb300 import abi
    plans = {op: ctx.plan_operator(op, "egraph", "fp32") for op in OPS}
    # kernel shapes that differ between items: the launch takes the largest walker count
    # and cluster size, items of fewer leave warps or blocks idle
    abi.mbc_set_schedule(plans["proton"].handle, 256, 1, 1)
    abi.mbc_set_schedule(plans["dinucleon_I"].handle, 512, 2, 2)
    items, meta, keep = [], [], []
    for (L, T) in ((3, 2), (4, 3)):
        fs = [mi.workload_fields("batched_64", set_index=s, L=L, T=T) for s in range(2)]
        U = np.stack([f[0] for f in fs])
        D = np.stack([f[1] for f in fs])
        Ud, Dd = torch.from_numpy(U).cuda(), torch.from_numpy(D).cuda()
        keep += [Ud, Dd]
        for op in OPS:
            C = torch.zeros(2, T, dtype=torch.complex128, device="cuda")
            S = torch.zeros(2, T, L ** 3, dtype=torch.complex128, device="cuda")
            keep += [C, S]
            items.append(dict(plan=plans[op].handle, U=Ud, D=Dd, C=C, site_out=S, n_sets=2, T=T, V3=L ** 3))
            meta.append((op, U, D, Ud, Dd))
    abi.mbc_batch_reserve(ctx.handle, items)
    ctx.batch(items)
    torch.cuda.synchronize()
    for it, (op, U, D, Ud, Dd) in zip(items, meta):
        got_C, got_S = it["C"].cpu().numpy(), it["site_out"].cpu().numpy()
        if op in ("dinucleon_II", "he3_II"):
            assert np.all(got_C == 0)
            continue
        ref = oracle_sites(op, U, D).reshape(got_S.shape)
        assert relerr(got_S, ref) <= SITE_TOL, op
        # the same plan called alone (per-site values requested, as in the batch)
        C1 = torch.zeros_like(it["C"])
        S1 = torch.zeros_like(it["site_out"])
        plans[op].correlator(Ud, Dd, C1, S1)
        torch.cuda.synchronize()
        assert relerr(C1.cpu().numpy(), got_C) <= 1e-12, op
    # the batch in a CUDA graph gives the same C
    ref_C = [it["C"].cpu().numpy().copy() for it in items]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        ctx.batch(items, stream=torch.cuda.current_stream())
    for it in items:
        it["C"].zero_()
    g.replay()
    torch.cuda.synchronize()
    for it, r in zip(items, ref_C):
        assert np.array_equal(it["C"].cpu().numpy(), r)
    for p in plans.values():
        p.destroy()


def test_fp32_batch_recompute_interleaved_plans(ctx):
    """Site guard below every estimate: every unit of every item goes to the double-float
    recompute, whose list interleaves the items' plans in the order the FP32 blocks flagged
    them (a block meets plan after plan, and returns to each), so the staged tables of one
    plan must never be taken for another's.  The result matches the double-float batch of
    the same items and the oracle; a guard changed after mbc_batch_reserve takes effect."""
    from paper_2201_04269_gb300 import abi
    ops = ("proton", "dinucleon_I", "he3_I", "dinucleon_II")
    p32 = {op: ctx.plan_operator(op, "egraph", "fp32") for op in ops}
    pdf = {op: ctx.plan_operator(op, "egraph", "mixed") for op in ops}
    L, T, n = 3, 2, 6
    fs = [mi.workload_fields("batched_64", set_index=s, L=L, T=T) for s in range(n)]
    keep, it32, itdf, meta = [], [], [], []
    for s, (U, D) in enumerate(fs):
        Ud, Dd = torch.from_numpy(U[None]).cuda(), torch.from_numpy(D[None]).cuda()
        keep += [Ud, Dd]
        for op in ops:
            for its, plans in ((it32, p32), (itdf, pdf)):
                C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
                S = torch.zeros(1, T, L ** 3, dtype=torch.complex128, device="cuda")
                keep += [C, S]
                its.append(dict(plan=plans[op].handle, U=Ud, D=Dd, C=C, site_out=S, n_sets=1, T=T, V3=L ** 3))
            meta.append((op, U, D))
    abi.mbc_batch_reserve(ctx.handle, it32)
    for p in p32.values():
        p.set_guard(site_threshold=-1.0)          # after the reserve: the batch must see it
    ctx.batch(it32)
    torch.cuda.synchronize()
    n_units = sum(T * L ** 3 for op, *_ in meta if op != "dinucleon_II")
    assert ctx.fp32_recomputed == n_units
    ctx.batch(itdf)
    torch.cuda.synchronize()
    for a, b, (op, U, D) in zip(it32, itdf, meta):
        ga, gb = a["site_out"].cpu().numpy(), b["site_out"].cpu().numpy()
        if op == "dinucleon_II":
            assert np.all(a["C"].cpu().numpy() == 0)
            continue
        assert relerr(ga, gb) <= 1e-12, op
        assert relerr(a["C"].cpu().numpy(), b["C"].cpu().numpy()) <= 1e-12, op
        assert relerr(ga, oracle_sites(op, U, D).reshape(ga.shape)) <= SITE_TOL, op
    for p in list(p32.values()) + list(pdf.values()):
        p.destroy()


def test_batch_mixing_all_three_arithmetics(ctx):
    """FP64, double-float and FP32 items in one mbc_batch (one launch per precision, the
    FP32 launch with its guards and recompute): each item's C equals its own call."""
    from paper_2201_04269_gb300 import abi
    L, T = 4, 3
    U, D = mi.workload_fields("batched_64", set_index=5, L=L, T=T)
    Ud, Dd = torch.from_numpy(U[None]).cuda(), torch.from_numpy(D[None]).cuda()
    plans, items, keep = [], [], []
    for op in ("dinucleon_I", "he3_I"):
        for prec in ("fp64", "mixed", "fp32"):
            pl = ctx.plan_operator(op, "egraph", prec)
            C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
            keep.append(C)
            plans.append(pl)
            items.append(dict(plan=pl.handle, U=Ud, D=Dd, C=C, site_out=None, n_sets=1, T=T, V3=L ** 3))
    ctx.batch(items)
    torch.cuda.synchronize()
    for it, pl in zip(items, plans):
        C1 = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
        pl.correlator(Ud, Dd, C1)
        torch.cuda.synchronize()
        assert relerr(it["C"].cpu().numpy(), C1.cpu().numpy()) <= 1e-12
    for pl in plans:
        pl.destroy()


def test_fp32_batch_with_complex_weight_item(ctx):
    """An item with complex weights (and a projector) in an FP32 batch switches the launch to
    the complex-weight records for every item: the real-weight He-3 I item and the complex
    item still equal their separate calls, and the complex item matches the oracle's
    index-set sum."""
    from paper_2201_04269_gb300 import abi, Plan
    from oracle import native as onat_
    n_u, n_d = 3, 2
    rng = np.random.default_rng(33)

    def side(n):
        idx = np.zeros((n, n_u + n_d), np.int8)
        for t in range(n):
            idx[t, :n_u] = rng.choice(12, n_u, replace=False)
            idx[t, n_u:] = rng.choice(12, n_d, replace=False)
        return idx, rng.standard_normal(n) + 1j * rng.standard_normal(n)
    si, sw = side(20)
    ri, rw = side(16)
    soff, roff = np.array([0, 9, 20]), np.array([0, 7, 16])
    P = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    pc = Plan(ctx, abi.mbc_plan_create(ctx.handle, n_u, n_d, si, sw, soff, ri, rw, roff, P, 1.0, "egraph", "fp32"))
    pr = ctx.plan_operator("he3_I", "egraph", "fp32")
    L, T = 3, 2
    U, D = mi.workload_fields("batched_64", set_index=9, L=L, T=T)
    Ud, Dd = torch.from_numpy(U[None]).cuda(), torch.from_numpy(D[None]).cuda()
    items, keep = [], []
    for pl in (pr, pc):
        C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
        S = torch.zeros(1, T, L ** 3, dtype=torch.complex128, device="cuda")
        keep += [C, S]
        items.append(dict(plan=pl.handle, U=Ud, D=Dd, C=C, site_out=S, n_sets=1, T=T, V3=L ** 3))
    ctx.batch(items)
    torch.cuda.synchronize()
    for it, pl in zip(items, (pr, pc)):
        C1 = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
        S1 = torch.zeros(1, T, L ** 3, dtype=torch.complex128, device="cuda")
        pl.correlator(Ud, Dd, C1, S1)
        torch.cuda.synchronize()
        assert relerr(it["C"].cpu().numpy(), C1.cpu().numpy()) <= 1e-9
        assert relerr(it["site_out"].cpu().numpy(), S1.cpu().numpy()) <= 1e-9
    snk = [(si[soff[j]:soff[j + 1]], sw[soff[j]:soff[j + 1]]) for j in range(2)]
    src = [(ri[roff[j]:roff[j + 1]], rw[roff[j]:roff[j + 1]]) for j in range(2)]
    n = n_u + n_d
    ref = (-1) ** (n * (n - 1) // 2) * onat_.direct(n_u, n_d, snk, src, P, U.reshape(-1, 12, 12), D.reshape(-1, 12, 12))
    assert relerr(items[1]["site_out"].cpu().numpy().ravel(), ref) <= SITE_TOL
    ref_he3 = oracle_sites("he3_I", U, D)
    assert relerr(items[0]["site_out"].cpu().numpy().ravel(), ref_he3) <= SITE_TOL
    pr.destroy()
    pc.destroy()


def test_batched_workload_64_sets_full_size(ctx):
    """The batched workload at its stated size in one persistent FP32 launch (plus its
    guard, recompute and site-sum launches): three sampled sites of every item against
    the oracle at the mixed tolerance, and the vanishing operators exactly zero."""
    from paper_2201_04269_gb300 import abi
    w = mi.WORKLOADS["batched_64"]
    free = torch.cuda.mem_get_info()[0]
    need = 32 * 2 * (16 ** 3 * 32 + 24 ** 3 * 48) * 2304 * 1.06 + 3 * 5 * 32 * (16 ** 3 * 32 + 24 ** 3 * 48) * 48
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    plans = {op: ctx.plan_operator(op, "egraph", "fp32") for op in OPS}
    st = torch.cuda.current_stream().cuda_stream
    items, keep, meta = [], [], []
    for s in range(w["sets"]):
        L, T = (16, 32) if s < 32 else (24, 48)
        V3 = L ** 3
        U = torch.empty(1, T, V3, 12, 12, dtype=torch.complex128, device="cuda")
        D = torch.empty_like(U)
        mi.fill_device(U.data_ptr(), w["seed"] + s, s, 0, V3, list(range(T)), w["kappa"], None, st)
        mi.fill_device(D.data_ptr(), w["seed"] + s, s, 1, V3, list(range(T)), w["kappa"], None, st)
        keep += [U, D]
        for op in OPS:
            C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
            S = torch.zeros(1, T, V3, dtype=torch.complex128, device="cuda") if op not in ("dinucleon_II", "he3_II") else None
            keep += [C, S]
            items.append(dict(plan=plans[op].handle, U=U, D=D, C=C, site_out=S, n_sets=1, T=T, V3=V3))
            meta.append((op, s, L, T))
    abi.mbc_batch_reserve(ctx.handle, items)
    n0 = ctx.launches
    ctx.batch(items)
    torch.cuda.synchronize()
    launches = ctx.launches - n0
    # one FP32 launch over every unit, its slice guard, the double-float recompute, and one
    # site-sum launch or two (with per-site values) per non-vanishing item
    assert launches <= 3 + 2 * sum(1 for op, *_ in meta if op not in ("dinucleon_II", "he3_II"))
    rng = np.random.default_rng(64)
    worst = 0.0
    for it, (op, s, L, T) in zip(items, meta):
        got_C = it["C"].cpu().numpy()
        if op in ("dinucleon_II", "he3_II"):
            assert np.all(got_C == 0)
            continue
        ts = rng.integers(0, T, size=3)
        xs = rng.integers(0, L ** 3, size=3)
        Uh = np.stack([mi.site_matrices(w["seed"] + s, s, 0, int(t), [int(x)], w["kappa"])[0] for t, x in zip(ts, xs)])
        Dh = np.stack([mi.site_matrices(w["seed"] + s, s, 1, int(t), [int(x)], w["kappa"])[0] for t, x in zip(ts, xs)])
        ref = oracle_sites(op, Uh, Dh)
        S = it["site_out"]
        got = np.array([S[0, int(t), int(x)].item() for t, x in zip(ts, xs)])
        e = relerr(got, ref)
        worst = max(worst, e)
        assert e <= SITE_TOL, (op, s, e)
    print(f"batched 64 sets: {len(items)} items, {launches} launches, worst sampled-site error {worst:.2e}")
    for p in plans.values():
        p.destroy()
