"""GPU parity of the sink-momentum projection (the e^{-i p.x} phase of arXiv 2201.04269
Sec. 2 applied to the quark-level site sum) through mbc_correlator_momentum, against
the oracle's correlator_momentum; 1e-12 in FP64, 1e-5 in mixed, 1e-6 for C(t) in FP32 with
its guards (the slice guard judges the phased C(t))."""
import numpy as np
import pytest

import mbc_inputs as mi
from oracle import correlator as ocor
from oracle import operators as oops

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5, "fp32": 1e-6}


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


@pytest.mark.parametrize("name,wl,L,T,algo,prec,p", [
    ("proton", "proton_4x8", 4, 8, "direct", "fp64", (0, 1, 2)),
    ("proton", "proton_4x8", 4, 8, "tree", "mixed", (1, 0, 0)),
    ("dinucleon_I", "dinucleon_16x32", 4, 2, "egraph", "fp64", (1, 0, 0)),
    ("dinucleon_I", "dinucleon_16x32", 3, 2, "egraph", "mixed", (2, 1, -1)),
    ("he3_II_s", "he3_24x48", 2, 2, "egraph", "fp64", (1, 1, 1)),
    ("dinucleon_I", "dinucleon_16x32", 4, 2, "egraph", "fp32", (0, 1, 0)),
    ("he3_I", "he3_24x48", 3, 2, "egraph", "fp32", (1, 0, 2)),
])
def test_momentum_matches_oracle(ctx, name, wl, L, T, algo, prec, p):
    U, D = mi.workload_fields(wl, L=L, T=T)
    want = ocor.correlator_momentum(ocor.CanonicalPlan(oops.build(name)).site_values, U, D, L, p)
    plan = ctx.plan_operator(name, algo, prec)
    C = torch.zeros(1, T, dtype=torch.complex128, device="cuda")
    plan.correlator_momentum(dev(U[None]), dev(D[None]), C, L, p)
    torch.cuda.synchronize()
    got = C.cpu().numpy()[0]
    assert np.max(np.abs(got - want) / np.abs(want)) <= TOL[prec]
    plan.destroy()


def test_zero_momentum_is_the_plain_sum(ctx):
    U, D = mi.workload_fields("dinucleon_16x32", L=4, T=2)
    plan = ctx.plan_operator("dinucleon_I", "egraph", "fp64")
    C0 = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
    C1 = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
    S0 = torch.zeros(1, 2, 64, dtype=torch.complex128, device="cuda")
    S1 = torch.zeros(1, 2, 64, dtype=torch.complex128, device="cuda")
    plan.correlator(dev(U[None]), dev(D[None]), C0, site_out=S0)
    plan.correlator_momentum(dev(U[None]), dev(D[None]), C1, 4, None, site_out=S1)
    torch.cuda.synchronize()
    assert np.array_equal(C0.cpu().numpy(), C1.cpu().numpy())
    # site values carry no phase, whatever the momentum
    S2 = torch.zeros(1, 2, 64, dtype=torch.complex128, device="cuda")
    C2 = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
    plan.correlator_momentum(dev(U[None]), dev(D[None]), C2, 4, (1, 2, 3), site_out=S2)
    torch.cuda.synchronize()
    assert np.array_equal(S0.cpu().numpy(), S2.cpu().numpy())
    plan.destroy()


def test_translation_phase_at_benchmark_lattice(ctx):
    """3He_II-s, 24^3 lattice, two slices, mixed e-graph plan: translating the sink fields
    by a multiplies C(p) by e^{-i 2 pi p.a / L} and leaves C(0) unchanged (exact property,
    any size)."""
    L = 24
    U, D = mi.workload_fields("he3_24x48", t_list=[3, 33])
    x = np.arange(L ** 3)
    xyz = np.stack([x % L, (x // L) % L, x // (L * L)], axis=1)
    a = np.array([5, 11, 2])
    moved = ((xyz + a) % L) @ np.array([1, L, L * L])
    Us, Ds = np.empty_like(U), np.empty_like(D)
    Us[:, moved], Ds[:, moved] = U, D
    plan = ctx.plan_operator("he3_II_s", "egraph", "mixed")
    p = (2, 0, 1)
    res = []
    for uu, dd in ((U, D), (Us, Ds)):
        C0 = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
        Cp = torch.zeros(1, 2, dtype=torch.complex128, device="cuda")
        plan.correlator_momentum(dev(uu[None]), dev(dd[None]), C0, L, None)
        plan.correlator_momentum(dev(uu[None]), dev(dd[None]), Cp, L, p)
        torch.cuda.synchronize()
        res.append((C0.cpu().numpy()[0], Cp.cpu().numpy()[0]))
    (c0, cp), (c0s, cps) = res
    # the site sum of C(0) is reordered by the translation: equal within the summation's rounding
    assert np.max(np.abs(c0s - c0) / np.abs(c0)) <= 1e-9
    phase = np.exp(-2j * np.pi * np.dot(p, a) / L)
    assert np.max(np.abs(cps - cp * phase) / np.abs(cp)) <= 1e-9
    plan.destroy()
