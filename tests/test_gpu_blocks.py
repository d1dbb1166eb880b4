"""GPU parity of the hadron-block path (arXiv 2201.04269 Secs. 2-4) through the C ABI
against the oracle (oracle/blocks.py): per-site blocks, momentum-projected blocks, and
the block form of the correlator; FP64 tolerance 1e-12."""
import numpy as np
import pytest

import mbc_inputs as mi
from oracle import blocks as obl
from oracle import correlator as ocor
from oracle import operators as oops

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04269_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def fields(wl, **kw):
    U, D = mi.workload_fields(wl, **kw)
    return U, D


def rel(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


@pytest.mark.parametrize("h", range(6))
def test_site_blocks_match_oracle(ctx, h):
    U, D = fields("dinucleon_16x32", L=2, T=2)          # 16 sites
    Us, Ds = U.reshape(-1, 12, 12), D.reshape(-1, 12, 12)
    f = torch.zeros(len(Us), obl.N_ETA, dtype=torch.complex128, device="cuda")
    ctx.hadron_blocks(h, dev(Us), dev(Ds), f)
    torch.cuda.synchronize()
    want = obl.block_site(Us, Ds, h).reshape(len(Us), obl.N_ETA)
    assert rel(f.cpu().numpy(), want) <= TOL


@pytest.mark.parametrize("p", [None, (1, 0, 1), (0, -1, 2)])
def test_projected_blocks_match_oracle(ctx, p):
    L = 3
    U, D = fields("proton_4x8", L=L, T=2)
    plan = obl.BlockPlan("neutron")
    want = obl.projected_blocks(plan, U, D, L, p or (0, 0, 0))[:, obl.N_ETA:2 * obl.N_ETA]
    F = torch.zeros(1, 2, obl.N_ETA, dtype=torch.complex128, device="cuda")
    ctx.hadron_blocks_projected("N", dev(U[None]), dev(D[None]), F, L, p)
    torch.cuda.synchronize()
    assert rel(F.cpu().numpy()[0], want) <= TOL


@pytest.mark.parametrize("name,wl,L,T,p", [("proton", "proton_4x8", 4, 3, (1, 2, 0)),
                                           ("dinucleon_I", "dinucleon_16x32", 4, 2, None),
                                           ("dinucleon_I", "dinucleon_16x32", 3, 2, (0, 1, 1)),
                                           ("he3_I", "he3_24x48", 2, 2, None)])
def test_block_correlator_matches_oracle(ctx, name, wl, L, T, p):
    U, D = fields(wl, L=L, T=T)
    ref = obl.BlockPlan(name, "canonical")
    want = obl.correlator_projected(ref, U, D, L, p or (0, 0, 0))
    plan = ctx.block_plan(name)
    C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None]), dev(D[None]), C, L, p)
    torch.cuda.synchronize()
    got = C.cpu().numpy()[0]
    assert np.max(np.abs(got - want) / np.abs(want)) <= TOL
    plan.destroy()


@pytest.mark.parametrize("name,wl,L,T,p", [("proton", "proton_4x8", 4, 3, (1, 2, 0)),
                                           ("dinucleon_I", "dinucleon_16x32", 3, 2, (0, 1, 1)),
                                           ("he3_I", "he3_24x48", 2, 2, None)])
def test_mixed_block_correlator_matches_oracle(ctx, name, wl, L, T, p):
    """Double-float projected blocks: within the mixed tolerance 1e-5 and, by design
    (about 2^-46 per operation), within 1e-9."""
    U, D = fields(wl, L=L, T=T)
    ref = obl.BlockPlan(name, "canonical")
    want = obl.correlator_projected(ref, U, D, L, p or (0, 0, 0))
    plan = ctx.block_plan(name, "mixed")
    C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None]), dev(D[None]), C, L, p)
    torch.cuda.synchronize()
    got = C.cpu().numpy()[0]
    assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-9
    plan.destroy()


def test_mixed_block_correlator_wide_exponent_range(ctx):
    """Sites of one slice whose propagators differ by 2^40 in scale (and slices at
    exp(-0.5 t) down to t = 47): the per-site power-of-two scaling keeps the double-float
    projection accurate."""
    L, T = 3, 2
    U, D = fields("he3_24x48", L=L, t_list=[0, 47])
    s = np.ones(L ** 3)
    s[::5] = 2.0 ** 20
    s[1::7] = 2.0 ** -20
    U = U * s[None, :, None, None]
    D = D * s[None, :, None, None]
    ref = obl.BlockPlan("he3_I", "canonical")
    want = obl.correlator_projected(ref, U, D, L)
    plan = ctx.block_plan("he3_I", "mixed")
    C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None]), dev(D[None]), C, L)
    torch.cuda.synchronize()
    got = C.cpu().numpy()[0]
    assert np.max(np.abs(got - want) / np.abs(want)) <= 1e-9
    plan.destroy()


def test_he3_II_s_block_correlator_ragged_lattice(ctx):
    """3He_II-s on 5^3 x 2: several tiles per slice with a ragged last tile."""
    L, T = 5, 2
    U, D = fields("he3_24x48", L=L, t_list=[0, 7])
    ref = obl.BlockPlan("he3_II_s", "canonical")
    want = obl.correlator_projected(ref, U, D, L)
    plan = ctx.block_plan("he3_II_s")
    C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None]), dev(D[None]), C, L)
    torch.cuda.synchronize()
    got = C.cpu().numpy()[0]
    assert np.max(np.abs(got - want) / np.abs(want)) <= TOL
    plan.destroy()


@pytest.mark.parametrize("name", ["proton", "dinucleon_I", "he3_I"])
def test_single_site_lattice_equals_local_correlator(ctx, name):
    """With L = 1 the projected block form is the local-sink correlator of the
    determinant path (two independent GPU paths and the oracle agree)."""
    U, D = fields("he3_24x48", L=1, T=4)
    want = ocor.correlator(ocor.CanonicalPlan(oops.build(name)).site_values, U, D)
    bp = ctx.block_plan(name)
    Cb = torch.zeros(1, 4, dtype=torch.complex128, device="cuda")
    bp.correlator(dev(U[None]), dev(D[None]), Cb, 1)
    qp = ctx.plan_operator(name, "egraph", "fp64")
    Cq = torch.zeros(1, 4, dtype=torch.complex128, device="cuda")
    qp.correlator(dev(U[None]), dev(D[None]), Cq)
    torch.cuda.synchronize()
    for got in (Cb.cpu().numpy()[0], Cq.cpu().numpy()[0]):
        assert np.max(np.abs(got - want) / np.abs(want)) <= TOL
    bp.destroy()
    qp.destroy()


def test_empty_and_vanishing(ctx):
    plan = ctx.block_plan("dinucleon_II")                # no block terms at all
    assert plan.info["merged_terms"] == 0
    U, D = fields("dinucleon_16x32", L=2, T=2)
    C = torch.full((1, 2), complex(3.0, 1.0), dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None]), dev(D[None]), C, 2)
    torch.cuda.synchronize()
    assert np.all(C.cpu().numpy() == 0)
    plan.destroy()
    plan = ctx.block_plan("proton")
    C = torch.zeros(0, 2, dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None][:0]), dev(D[None][:0]), C, 2)
    plan.destroy()


def test_colour_invariance_full_size(ctx):
    """At the benchmark size (3He_II-s, 24^3, two slices), S_x -> g_x S_x h^dagger with
    random SU(3) g_x per site and h at the source leaves C unchanged: a property of the
    exact correlator at any size."""
    L = 24
    t_list = [0, 24]
    U, D = fields("he3_24x48", t_list=t_list)
    rng = np.random.default_rng(91)
    g = mi.su3_random(rng, U.shape[0] * U.shape[1]).reshape(U.shape[0], U.shape[1], 3, 3)
    h = mi.su3_random(rng, 1)[0]
    # index i = 3 spin + colour: colour acts as kron(1_spin, g)
    G = np.einsum("ab,tsxy->tsaxby", np.eye(4), g).reshape(U.shape[0], U.shape[1], 12, 12)
    H = np.kron(np.eye(4), h)

    def rotate(S):
        return np.einsum("tsij,tsjk,lk->tsil", G, S, H.conj())

    plan = ctx.block_plan("he3_II_s")
    C0 = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
    C1 = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None]), dev(D[None]), C0, L)
    plan.correlator(dev(rotate(U)[None]), dev(rotate(D)[None]), C1, L)
    torch.cuda.synchronize()
    a, b = C0.cpu().numpy()[0], C1.cpu().numpy()[0]
    assert np.all(np.abs(a) > 0)
    assert np.max(np.abs(a - b) / np.abs(a)) <= 1e-10
    plan.destroy()


def test_block_correlator_deterministic(ctx):
    U, D = fields("dinucleon_16x32", L=6, T=2)
    plan = ctx.block_plan("dinucleon_I")
    outs = []
    for _ in range(2):
        C = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
        plan.correlator(dev(U[None]), dev(D[None]), C, 6)
        torch.cuda.synchronize()
        outs.append(C.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    plan.destroy()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_translation_full_size(ctx, prec):
    """3He_II-s on the full 24^3 lattice (two slices): translating the sink fields by a
    lattice vector a leaves the zero-momentum block correlator unchanged and multiplies
    the one at momentum p by e^{-i 2 pi A p.a / L} (every one of the A baryons picks up
    the phase of its own projection) -- a property of the exact result at any size."""
    L = 24
    U, D = fields("he3_24x48", t_list=[5, 40])
    x = np.arange(L ** 3)
    xyz = np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)
    a = np.array([3, 0, 7])
    moved = ((xyz + a) % L) @ np.array([1, L, L * L])
    Us, Ds = np.empty_like(U), np.empty_like(D)
    Us[:, moved], Ds[:, moved] = U, D
    plan = ctx.block_plan("he3_II_s", prec)
    p = (1, 2, 0)
    out = {}
    for key, (uu, dd, mom) in {"0": (U, D, None), "0s": (Us, Ds, None), "p": (U, D, p), "ps": (Us, Ds, p)}.items():
        C = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
        plan.correlator(dev(uu[None]), dev(dd[None]), C, L, mom)
        torch.cuda.synchronize()
        out[key] = C.cpu().numpy()[0]
    tol = 1e-10 if prec == "fp64" else 1e-9
    assert np.max(np.abs(out["0s"] - out["0"]) / np.abs(out["0"])) <= tol
    phase = np.exp(-2j * np.pi * 3 * np.dot(p, a) / L)
    assert np.max(np.abs(out["ps"] - out["p"] * phase) / np.abs(out["p"])) <= tol
    plan.destroy()


@pytest.mark.parametrize("name,wl,L,T", [("proton", "proton_4x8", 3, 2), ("dinucleon_I", "dinucleon_16x32", 3, 2),
                                         ("he3_I", "he3_24x48", 2, 2), ("he3_II_s", "he3_24x48", 2, 1)])
def test_local_block_form_matches_determinant_oracle(ctx, name, wl, L, T):
    """The block form of the local-sink correlator (blocks of each site, block factor tree
    per site) against the quark-level oracle, per site and summed, and against the
    e-graph plan on the GPU."""
    U, D = fields(wl, L=L, T=T)
    cp = ocor.CanonicalPlan(oops.build(name))
    want_sites = cp.site_values(U.reshape(-1, 12, 12), D.reshape(-1, 12, 12))
    want = ocor.correlator(cp.site_values, U, D)
    plan = ctx.block_plan(name)
    C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
    S = torch.zeros(1, T, L ** 3, dtype=torch.complex128, device="cuda")
    plan.correlator_local(dev(U[None]), dev(D[None]), C, S)
    qp = ctx.plan_operator(name, "egraph", "fp64")
    Cq = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
    qp.correlator(dev(U[None]), dev(D[None]), Cq)
    torch.cuda.synchronize()
    got, sites = C.cpu().numpy()[0], S.cpu().numpy().ravel()
    assert np.max(np.abs(sites - want_sites) / np.abs(want_sites)) <= TOL
    assert np.max(np.abs(got - want) / np.abs(want)) <= TOL
    assert np.max(np.abs(Cq.cpu().numpy()[0] - got) / np.abs(got)) <= TOL
    plan.destroy()
    qp.destroy()


def test_local_block_form_vanishing_and_empty(ctx):
    U, D = fields("dinucleon_16x32", L=2, T=2)
    plan = ctx.block_plan("dinucleon_II")
    C = torch.full((1, 2), complex(1.0, 2.0), dtype=torch.complex128, device="cuda")
    plan.correlator_local(dev(U[None]), dev(D[None]), C)
    torch.cuda.synchronize()
    assert np.all(C.cpu().numpy() == 0)
    plan.destroy()
    plan = ctx.block_plan("proton")
    C = torch.zeros(0, 2, dtype=torch.complex128, device="cuda")
    plan.correlator_local(dev(U[None][:0]), dev(D[None][:0]), C)
    plan.destroy()
