"""mbc_correlator_noalloc: the correlator evaluated without any device allocation, for
callers that cannot allocate when they evaluate (inside a stream capture, under a fixed
memory budget).  Checked through the C ABI against mbc_correlator on the same plan and
fields, on two calls in a row (the fixed scratch array keeps the previous call's
contents).  Collected last on purpose; runs alone or after the other tests."""
import numpy as np
import pytest

import mbc_inputs as mi

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-5}


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
    C_ref = torch.zeros(n_sets, T, dtype=torch.complex128, device="cuda")
    plan.correlator(U, D, C_ref)
    torch.cuda.synchronize()
    ref = C_ref.cpu().numpy()
    for _ in range(2):
        C = torch.full((n_sets, T), complex(7.0, -3.0), dtype=torch.complex128, device="cuda")
        abi.mbc_correlator_noalloc(plan.handle, U, D, n_sets, T, V3, C, ctx=ctx.handle)
        torch.cuda.synchronize()
        got = C.cpu().numpy()
        err = float(np.max(np.abs(got - ref) / np.abs(ref)))
        assert err <= TOL[prec], err
    plan.destroy()


def test_noalloc_rejects_oversized_requests(ctx):
    from paper_2201_04269_gb300 import abi
    plan = ctx.plan_operator("dinucleon_I", "egraph", "mixed")
    # 2^22 sites need 128 MiB of per-site partial sums: more than the fixed array holds;
    # the size check rejects the call before any pointer is used
    with pytest.raises(abi.MbcError) as e:
        abi.mbc_correlator_noalloc(plan.handle, 1, 1, 1, 1, 1 << 22, 1, ctx=ctx.handle)
    assert e.value.status == 2
    assert "fixed array holds" in abi.mbc_last_error(ctx.handle)
    tree = ctx.plan_operator("dinucleon_I", "tree", "mixed")
    with pytest.raises(abi.MbcError):
        abi.mbc_correlator_noalloc(tree.handle, 1, 1, 1, 1, 1, 1, ctx=ctx.handle)
    plan.destroy()
    tree.destroy()
