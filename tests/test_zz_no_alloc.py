"""mbc_correlator_noalloc: the correlator evaluated without any device allocation, for
callers that may not allocate device memory when they evaluate (services with a fixed
device-memory carve-out, plug-ins inside a host that owns every allocation, real-time
loops that cannot take an allocation's latency).  Checked through the C ABI against
mbc_correlator on the same plan and fields, on two calls in a row (the fixed scratch
array keeps the previous call's contents): the two entry points run the same kernel in
the same order, so the results must be bit-identical.  Both cases take the path where
the fixed array holds fewer K slots than the device has resident blocks (the grid
shrinks).  Collected last on purpose; runs alone or after the other tests."""
import numpy as np
import pytest

import mbc_inputs as mi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04269_gb300 import Context, build
    build.build()
    c = Context(0)
    yield c
    c.close()


def fields(wl, **kw):
    U, D = mi.workload_fields(wl, **kw)
    return torch.from_numpy(U[None]).cuda(), torch.from_numpy(D[None]).cuda()


@pytest.mark.parametrize("name,wl,kw", [("dinucleon_I", "dinucleon_16x32", dict(L=4, T=4)),
                                        ("he3_II_s", "he3_24x48", dict(L=6, t_list=[3, 30]))])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_pooled_entry_point(ctx, name, wl, kw, prec):
    from paper_2201_04269_gb300 import abi
    U, D = fields(wl, **kw)
    n_sets, T, V3 = U.shape[:3]
    plan = ctx.plan_operator(name, "egraph", prec)
    # one K slot per block: the 64 MiB array holds fewer slots than 152 SMs x resident blocks
    kslot = plan.info["cols_d"] * plan.info["rows_d"] * 16
    assert (64 << 20) // kslot < 152 * abi.mbc_get_schedule(plan.handle)["blocks_per_sm"]
    C_ref = torch.zeros(n_sets, T, dtype=torch.complex128, device="cuda")
    plan.correlator(U, D, C_ref)
    torch.cuda.synchronize()
    ref = C_ref.cpu().numpy()
    for _ in range(2):
        C = torch.full((n_sets, T), complex(7.0, -3.0), dtype=torch.complex128, device="cuda")
        abi.mbc_correlator_noalloc(plan.handle, U, D, n_sets, T, V3, C, ctx=ctx.handle)
        torch.cuda.synchronize()
        assert np.array_equal(C.cpu().numpy(), ref)
    plan.destroy()


def test_noalloc_rejects_oversized_requests(ctx):
    from paper_2201_04269_gb300 import abi
    # small real device buffers: the size check must reject the call before any use
    U = torch.zeros(144 * 2, dtype=torch.float64, device="cuda")
    D = torch.zeros(144 * 2, dtype=torch.float64, device="cuda")
    C = torch.full((1, 1), complex(5.0, 5.0), dtype=torch.complex128, device="cuda")
    plan = ctx.plan_operator("dinucleon_I", "egraph", "mixed")
    # 2^22 sites need 128 MiB of per-site partial sums: more than the fixed array holds
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_correlator_noalloc(plan.handle, U, D, 1, 1, 1 << 22, C, ctx=ctx.handle)
    assert e.value.status == 2
    assert "fixed array holds" in abi.mbc_last_error(ctx.handle)
    torch.cuda.synchronize()
    assert C.cpu().numpy()[0, 0] == complex(5.0, 5.0)            # output untouched
    tree = ctx.plan_operator("dinucleon_I", "tree", "mixed")
    with pytest.raises(abi.MbcError):
        abi.mbc_correlator_noalloc(tree.handle, U, D, 1, 1, 1, C, ctx=ctx.handle)
    # a vanishing operator (empty canonical term set) gives C = 0 at any size, without a kernel
    zero = ctx.plan_operator("dinucleon_II", "egraph", "mixed")
    abi.mbc_correlator_noalloc(zero.handle, U, D, 1, 1, 1 << 22, C, ctx=ctx.handle)
    torch.cuda.synchronize()
    assert C.cpu().numpy()[0, 0] == 0
    plan.destroy()
    tree.destroy()
    zero.destroy()


def test_noalloc_fp32_plan_uses_double_float(ctx):
    """An MBC_PREC_FP32 plan through the allocation-free entry point is evaluated in
    double-float: C(t) agrees with the pooled FP32 call to the FP32 target (1e-6) and with
    the double-float plan to 1e-12."""
    from paper_2201_04269_gb300 import abi
    U, D = fields("he3_24x48", L=6, t_list=[3, 30])
    n_sets, T, V3 = U.shape[:3]
    p32 = ctx.plan_operator("he3_I", "egraph", "fp32")
    pdf = ctx.plan_operator("he3_I", "egraph", "mixed")
    C32 = torch.zeros(n_sets, T, dtype=torch.complex128, device="cuda")
    Cdf = torch.zeros_like(C32)
    p32.correlator(U, D, C32)
    pdf.correlator(U, D, Cdf)
    C = torch.zeros_like(C32)
    abi.mbc_correlator_noalloc(p32.handle, U, D, n_sets, T, V3, C, ctx=ctx.handle)
    torch.cuda.synchronize()
    got, ref32, refdf = C.cpu().numpy(), C32.cpu().numpy(), Cdf.cpu().numpy()
    assert np.max(np.abs(got - ref32) / np.abs(ref32)) <= 1e-6
    assert np.max(np.abs(got - refdf) / np.abs(refdf)) <= 1e-12
    p32.destroy()
    pdf.destroy()
