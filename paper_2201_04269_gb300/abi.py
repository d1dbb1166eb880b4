"""ctypes binding of libmbc (include/mbc.h): the same entry points, argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only converts Python
and torch arguments into the C types of the ABI and raises ``MbcError`` on a non-zero
status.  Device buffers are passed as raw pointers (``tensor.data_ptr()``) and streams
as raw handles (``torch.cuda.current_stream().cuda_stream``).  Importing the module does
not need a GPU; loading the library does need ``libmbc.so`` (built by ``build.py``) and
fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmbc.so")

c_i8p = ctypes.POINTER(ctypes.c_int8)
c_i32p = ctypes.POINTER(ctypes.c_int32)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_dp = ctypes.POINTER(ctypes.c_double)
c_vp = ctypes.c_void_p

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "OOM", 4: "CUDA", 5: "TIMEOUT", 6: "NUMERIC", 7: "IO"}
ALGO = {"direct": 0, "tree": 1, "egraph": 2}
PREC = {"fp64": 0, "mixed": 1, "fp32": 2}
OPERATOR = {"proton": 0, "neutron": 1, "dinucleon_I": 2, "dinucleon_II": 3, "he3_I": 4, "he3_II": 5, "he3_II_s": 6}
BLOCK_TYPE = {"P": 0, "N": 1, "P+": 2, "P-": 3, "N+": 4, "N-": 5}
BLOCK_ENTRIES = 6912


class MbcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"mbc status {STATUS.get(status, status)}: {msg}")
        self.status = status


class mbc_problem(ctypes.Structure):
    _fields_ = [("n_u", ctypes.c_int), ("n_d", ctypes.c_int), ("n_free", ctypes.c_int),
                ("snk_idx", c_i8p), ("snk_w", c_dp), ("snk_off", c_i64p),
                ("src_idx", c_i8p), ("src_w", c_dp), ("src_off", c_i64p),
                ("proj", c_dp), ("scale", ctypes.c_double * 2)]


class mbc_plan_info(ctypes.Structure):
    _fields_ = [("n_u", ctypes.c_int), ("n_d", ctypes.c_int), ("algo", ctypes.c_int), ("prec", ctypes.c_int),
                ("index_size", ctypes.c_int64), ("canonical_terms", ctypes.c_int64),
                ("rows_u", ctypes.c_int64), ("rows_d", ctypes.c_int64), ("cols_u", ctypes.c_int64),
                ("cols_d", ctypes.c_int64), ("minors_u", ctypes.c_int64), ("minors_d", ctypes.c_int64),
                ("tree_nodes", ctypes.c_int64), ("egraph_classes", ctypes.c_int64), ("egraph_nodes", ctypes.c_int64),
                ("flops_per_site", ctypes.c_double), ("direct_flops_per_site", ctypes.c_double),
                ("scratch_bytes_per_site", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class mbc_schedule(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("sites_per_unit", ctypes.c_int)]


class mbc_work(ctypes.Structure):
    _fields_ = [("plan", c_vp), ("U", c_vp), ("D", c_vp), ("n_sets", ctypes.c_int), ("T", ctypes.c_int),
                ("V3", ctypes.c_int64), ("C", c_vp), ("site_out", c_vp)]


class mbc_block_plan_info(ctypes.Structure):
    _fields_ = [("n_baryons", ctypes.c_int), ("n_products", ctypes.c_int), ("n_w", ctypes.c_int * 8),
                ("expanded_terms", ctypes.c_int64), ("merged_terms", ctypes.c_int64), ("factors", ctypes.c_int64),
                ("level_nodes", ctypes.c_int64 * 4), ("block_flops_per_site", ctypes.c_double),
                ("tree_flops_per_slice", ctypes.c_double), ("shared_sums", ctypes.c_int64),
                ("shared_sum_terms", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["n_w"] = list(self.n_w)[:self.n_products]
        d["level_nodes"] = list(self.level_nodes)[:self.n_baryons]
        return d


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("mbc_create", ctypes.c_int, [ctypes.POINTER(c_vp), ctypes.c_int]),
    ("mbc_destroy", None, [c_vp]),
    ("mbc_last_error", ctypes.c_char_p, [c_vp]),
    ("mbc_version", ctypes.c_char_p, []),
    ("mbc_operator_terms", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), c_i64p, c_i8p, c_dp, c_i64p, c_dp, c_dp]),
    ("mbc_plan_create", ctypes.c_int, [c_vp, ctypes.POINTER(mbc_problem), ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_vp)]),
    ("mbc_plan_from_terms", ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, c_i8p, c_i8p, c_dp, c_dp,
                                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_vp)]),
    ("mbc_plan_destroy", None, [c_vp]),
    ("mbc_plan_get_info", ctypes.c_int, [c_vp, ctypes.POINTER(mbc_plan_info)]),
    ("mbc_plan_get_tree", ctypes.c_int, [c_vp, c_i64p, c_i64p, c_i32p, c_i32p, c_dp]),
    ("mbc_plan_get_minor", ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int64, c_i8p, c_i8p]),
    ("mbc_plan_save", ctypes.c_int, [c_vp, ctypes.c_char_p]),
    ("mbc_plan_load", ctypes.c_int, [c_vp, ctypes.c_char_p, ctypes.POINTER(c_vp)]),
    ("mbc_correlator", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, c_vp, c_vp, c_vp]),
    ("mbc_correlator_momentum", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_i32p,
                                               c_vp, c_vp, c_vp]),
    ("mbc_correlator_host", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, c_vp, c_vp]),
    ("mbc_batch_reserve", ctypes.c_int, [c_vp, ctypes.POINTER(mbc_work), ctypes.c_int]),
    ("mbc_batch", ctypes.c_int, [c_vp, ctypes.POINTER(mbc_work), ctypes.c_int, c_vp]),
    ("mbc_autotune", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int64, c_vp, ctypes.POINTER(mbc_schedule)]),
    ("mbc_set_schedule", ctypes.c_int, [c_vp, ctypes.POINTER(mbc_schedule)]),
    ("mbc_get_schedule", ctypes.c_int, [c_vp, ctypes.POINTER(mbc_schedule)]),
    ("mbc_launch_count", ctypes.c_int64, [c_vp]),
    ("mbc_plan_set_guard", ctypes.c_int, [c_vp, ctypes.c_double, ctypes.c_double]),
    ("mbc_plan_get_guard", ctypes.c_int, [c_vp, c_dp, c_dp]),
    ("mbc_fp32_recomputed", ctypes.c_int, [c_vp, c_i64p]),
    ("mbc_tensor_egraph", ctypes.c_int, [c_vp, ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int64, ctypes.c_int,
                                         ctypes.c_char_p, ctypes.c_int64, c_i64p, c_i64p, c_i64p]),
    ("mbc_correlator_noalloc", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, c_vp, c_vp]),
    ("mbc_hadron_blocks", ctypes.c_int, [c_vp, ctypes.c_int, c_vp, c_vp, ctypes.c_int64, c_vp, c_vp]),
    ("mbc_hadron_blocks_projected", ctypes.c_int, [c_vp, ctypes.c_int, c_vp, c_vp, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_int, c_i32p, c_vp, c_vp]),
    ("mbc_block_plan_create", ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(c_vp)]),
    ("mbc_block_plan_destroy", None, [c_vp]),
    ("mbc_block_plan_get_info", ctypes.c_int, [c_vp, ctypes.POINTER(mbc_block_plan_info)]),
    ("mbc_block_plan_get_terms", ctypes.c_int, [c_vp, c_i32p, c_dp]),
    ("mbc_block_plan_get_multiplicities", ctypes.c_int, [c_vp, c_i32p]),
    ("mbc_block_correlator_local", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                                  c_vp, c_vp, c_vp]),
    ("mbc_block_correlator", ctypes.c_int, [c_vp, c_vp, c_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_i32p,
                                            c_vp, c_vp]),
]

_LIB = None


def load(path: str = LIB_PATH):
    """Load libmbc.so and attach the signatures (raises if the library is missing)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(path):
            raise FileNotFoundError(f"{path} not found: run paper_2201_04269_gb300.build.build() first "
                                    "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def _enum(table, v):
    """Enum value of a name (unknown names become -1, which the library rejects)."""
    return table.get(v, -1) if isinstance(v, str) else int(v)


def _ptr(a, ctype):
    return a.ctypes.data_as(ctype) if a is not None and a.size else None


def check(status, ctx=None):
    if status != 0:
        msg = load().mbc_last_error(ctx).decode() if ctx else ""
        raise MbcError(status, msg)


def dptr(x):
    """Raw device (or host) address of a tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def sptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------- entry points
def mbc_version():
    return load().mbc_version().decode()


def mbc_create(device=0):
    ctx = c_vp()
    st = load().mbc_create(ctypes.byref(ctx), device)
    if st != 0:
        raise MbcError(st, f"mbc_create(device={device})")
    return ctx.value


def mbc_destroy(ctx):
    load().mbc_destroy(ctx)


def mbc_last_error(ctx):
    return load().mbc_last_error(ctx).decode()


def mbc_launch_count(ctx):
    return int(load().mbc_launch_count(ctx))


def mbc_operator_terms(op):
    """Expanded sink terms of a named operator: dict with n_u, n_d, n_free, idx, w,
    offsets, proj, scale (host numpy arrays)."""
    op = OPERATOR[op] if isinstance(op, str) else op
    lib = load()
    nu, nd, nf = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    nt = ctypes.c_int64()
    check(lib.mbc_operator_terms(op, ctypes.byref(nu), ctypes.byref(nd), ctypes.byref(nf), ctypes.byref(nt),
                                 None, None, None, None, None))
    nq = nu.value + nd.value
    idx = np.zeros((nt.value, nq), np.int8)
    w = np.zeros(nt.value, np.complex128)
    off = np.zeros(nf.value + 1, np.int64)
    proj = np.zeros((nf.value, nf.value), np.complex128)
    scale = ctypes.c_double()
    check(lib.mbc_operator_terms(op, ctypes.byref(nu), ctypes.byref(nd), ctypes.byref(nf), ctypes.byref(nt),
                                 _ptr(idx, c_i8p), w.ctypes.data_as(c_dp), off.ctypes.data_as(c_i64p),
                                 proj.ctypes.data_as(c_dp), ctypes.byref(scale)))
    return dict(n_u=nu.value, n_d=nd.value, n_free=nf.value, idx=idx, w=w, offsets=off, proj=proj, scale=scale.value)


def mbc_plan_create(ctx, n_u, n_d, snk_idx, snk_w, snk_off, src_idx, src_w, src_off, proj, scale, algo, prec):
    keep = []

    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    si, sw, so = arr(snk_idx, np.int8), arr(snk_w, np.complex128), arr(snk_off, np.int64)
    ri, rw, ro = arr(src_idx, np.int8), arr(src_w, np.complex128), arr(src_off, np.int64)
    pj = arr(proj, np.complex128)
    pr = mbc_problem()
    pr.n_u, pr.n_d, pr.n_free = n_u, n_d, len(so) - 1
    pr.snk_idx, pr.snk_w, pr.snk_off = _ptr(si, c_i8p), _ptr(sw.view(np.float64), c_dp), so.ctypes.data_as(c_i64p)
    pr.src_idx, pr.src_w, pr.src_off = _ptr(ri, c_i8p), _ptr(rw.view(np.float64), c_dp), ro.ctypes.data_as(c_i64p)
    pr.proj = pj.view(np.float64).ctypes.data_as(c_dp)
    sc = complex(scale)
    pr.scale[0], pr.scale[1] = sc.real, sc.imag
    plan = c_vp()
    check(load().mbc_plan_create(ctx, ctypes.byref(pr), _enum(ALGO, algo), _enum(PREC, prec),
                                 ctypes.byref(plan)), ctx)
    return plan.value


def mbc_plan_from_terms(ctx, n_u, n_d, sink, source, W, scale, algo, prec):
    sink = np.ascontiguousarray(sink, np.int8)
    source = np.ascontiguousarray(source, np.int8)
    W = np.ascontiguousarray(W, np.complex128)
    sc = np.array([complex(scale).real, complex(scale).imag])
    plan = c_vp()
    check(load().mbc_plan_from_terms(ctx, n_u, n_d, len(W), _ptr(sink, c_i8p), _ptr(source, c_i8p),
                                     _ptr(W.view(np.float64), c_dp), sc.ctypes.data_as(c_dp),
                                     _enum(ALGO, algo), _enum(PREC, prec), ctypes.byref(plan)), ctx)
    return plan.value


def mbc_plan_destroy(plan):
    load().mbc_plan_destroy(plan)


def mbc_plan_get_info(plan):
    info = mbc_plan_info()
    check(load().mbc_plan_get_info(plan, ctypes.byref(info)))
    return info.as_dict()


def mbc_plan_get_tree(plan):
    n_nodes, n_leaves = ctypes.c_int64(), ctypes.c_int64()
    lib = load()
    check(lib.mbc_plan_get_tree(plan, ctypes.byref(n_nodes), ctypes.byref(n_leaves), None, None, None))
    f = np.zeros(n_nodes.value, np.int32)
    c = np.zeros(n_nodes.value, np.int32)
    co = np.zeros(n_leaves.value, np.complex128)
    check(lib.mbc_plan_get_tree(plan, ctypes.byref(n_nodes), ctypes.byref(n_leaves), f.ctypes.data_as(c_i32p),
                                c.ctypes.data_as(c_i32p), co.view(np.float64).ctypes.data_as(c_dp)))
    return f, c, co


def mbc_plan_get_minor(plan, flavour, m, n):
    r = np.zeros(12, np.int8)
    c = np.zeros(12, np.int8)
    check(load().mbc_plan_get_minor(plan, flavour, m, r.ctypes.data_as(c_i8p), c.ctypes.data_as(c_i8p)))
    return tuple(int(v) for v in r[:n]), tuple(int(v) for v in c[:n])


def mbc_plan_save(plan, path, ctx=None):
    check(load().mbc_plan_save(plan, path.encode()), ctx)


def mbc_plan_load(ctx, path):
    plan = c_vp()
    check(load().mbc_plan_load(ctx, path.encode(), ctypes.byref(plan)), ctx)
    return plan.value


def mbc_correlator(plan, U, D, n_sets, T, V3, C, site_out=None, stream=None, ctx=None):
    check(load().mbc_correlator(plan, dptr(U), dptr(D), n_sets, T, V3, dptr(C), dptr(site_out), sptr(stream)), ctx)


def mbc_correlator_momentum(plan, U, D, n_sets, T, L, p, C, site_out=None, stream=None, ctx=None):
    """mbc_correlator with the sink momentum phase e^{-i 2 pi p.x / L} in the site sum."""
    check(load().mbc_correlator_momentum(plan, dptr(U), dptr(D), n_sets, T, L, _mom(p), dptr(C), dptr(site_out),
                                         sptr(stream)), ctx)


def mbc_correlator_noalloc(plan, U, D, n_sets, T, V3, C, stream=None, ctx=None):
    """mbc_correlator without device allocation (fixed scratch array in the library)."""
    check(load().mbc_correlator_noalloc(plan, dptr(U), dptr(D), n_sets, T, V3, dptr(C), sptr(stream)), ctx)


def mbc_correlator_host(plan, U_host, D_host, n_sets, T, V3, C_host, stream=None, ctx=None):
    check(load().mbc_correlator_host(plan, dptr(U_host), dptr(D_host), n_sets, T, V3, dptr(C_host), sptr(stream)), ctx)


def _works(items):
    arr = (mbc_work * len(items))()
    for i, it in enumerate(items):
        arr[i].plan = it["plan"]
        arr[i].U, arr[i].D, arr[i].C = dptr(it["U"]), dptr(it["D"]), dptr(it["C"])
        arr[i].n_sets, arr[i].T, arr[i].V3 = it["n_sets"], it["T"], it["V3"]
        arr[i].site_out = dptr(it.get("site_out"))
    return arr


def mbc_batch_reserve(ctx, items):
    check(load().mbc_batch_reserve(ctx, _works(items), len(items)), ctx)


def mbc_batch(ctx, items, stream=None):
    check(load().mbc_batch(ctx, _works(items), len(items), sptr(stream)), ctx)


def mbc_autotune(plan, U, D, n_sites, stream=None, ctx=None):
    s = mbc_schedule()
    check(load().mbc_autotune(plan, dptr(U), dptr(D), n_sites, sptr(stream), ctypes.byref(s)), ctx)
    return dict(threads=s.threads, blocks_per_sm=s.blocks_per_sm, sites_per_unit=s.sites_per_unit)


def mbc_set_schedule(plan, threads, blocks_per_sm, sites_per_unit=1, ctx=None):
    s = mbc_schedule(threads, blocks_per_sm, sites_per_unit)
    check(load().mbc_set_schedule(plan, ctypes.byref(s)), ctx)


def mbc_get_schedule(plan):
    s = mbc_schedule()
    check(load().mbc_get_schedule(plan, ctypes.byref(s)))
    return dict(threads=s.threads, blocks_per_sm=s.blocks_per_sm, sites_per_unit=s.sites_per_unit)


def mbc_plan_set_guard(plan, site_threshold, slice_tolerance, ctx=None):
    check(load().mbc_plan_set_guard(plan, float(site_threshold), float(slice_tolerance)), ctx)


def mbc_plan_get_guard(plan):
    a, b = ctypes.c_double(), ctypes.c_double()
    check(load().mbc_plan_get_guard(plan, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def mbc_fp32_recomputed(ctx):
    n = ctypes.c_int64()
    check(load().mbc_fp32_recomputed(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def mbc_tensor_egraph(ctx, expression, antisymmetric="eps", node_limit=100000, dim=3):
    """Extracted plan (text lines) and (classes, e-nodes) of a tensor expression's e-graph."""
    need, nc, nn = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lib = load()
    e, a = expression.encode(), (antisymmetric or "").encode()
    check(lib.mbc_tensor_egraph(ctx, e, a, node_limit, dim, None, 0, ctypes.byref(need), ctypes.byref(nc),
                                ctypes.byref(nn)), ctx)
    buf = ctypes.create_string_buffer(need.value)
    check(lib.mbc_tensor_egraph(ctx, e, a, node_limit, dim, buf, need.value, ctypes.byref(need), ctypes.byref(nc),
                                ctypes.byref(nn)), ctx)
    return buf.value.decode().splitlines(), (nc.value, nn.value)


# ------------------------------------------------------------------- hadron blocks
def _mom(p):
    if p is None:
        return None
    a = (ctypes.c_int32 * 3)(*[int(v) for v in p])
    return ctypes.cast(a, c_i32p)


def mbc_hadron_blocks(ctx, block_type, U, D, n_sites, f, stream=None):
    check(load().mbc_hadron_blocks(ctx, _enum(BLOCK_TYPE, block_type), dptr(U), dptr(D), n_sites, dptr(f),
                                   sptr(stream)), ctx)


def mbc_hadron_blocks_projected(ctx, block_type, U, D, n_sets, T, L, F, p=None, stream=None):
    check(load().mbc_hadron_blocks_projected(ctx, _enum(BLOCK_TYPE, block_type), dptr(U), dptr(D), n_sets, T, L,
                                             _mom(p), dptr(F), sptr(stream)), ctx)


def mbc_block_plan_create(ctx, op, prec="fp64"):
    plan = c_vp()
    check(load().mbc_block_plan_create(ctx, _enum(OPERATOR, op), _enum(PREC, prec), ctypes.byref(plan)), ctx)
    return plan.value


def mbc_block_plan_destroy(plan):
    load().mbc_block_plan_destroy(plan)


def mbc_block_plan_get_info(plan):
    info = mbc_block_plan_info()
    check(load().mbc_block_plan_get_info(plan, ctypes.byref(info)))
    return info.as_dict()


def mbc_block_plan_get_terms(plan):
    """Merged block terms: (ids int32 [K, A], w complex128 [K])."""
    info = mbc_block_plan_get_info(plan)
    K, A = info["merged_terms"], info["n_baryons"]
    ids = np.zeros((K, A), np.int32)
    w = np.zeros(K, np.complex128)
    if K:
        check(load().mbc_block_plan_get_terms(plan, ids.ctypes.data_as(c_i32p), w.view(np.float64).ctypes.data_as(c_dp)))
    return ids, w


def mbc_block_plan_get_multiplicities(plan):
    """Multiplicity of every merged block term: int32 [K]."""
    K = mbc_block_plan_get_info(plan)["merged_terms"]
    m = np.zeros(K, np.int32)
    if K:
        check(load().mbc_block_plan_get_multiplicities(plan, m.ctypes.data_as(c_i32p)))
    return m


def mbc_block_correlator(plan, U, D, n_sets, T, L, C, p=None, stream=None, ctx=None):
    check(load().mbc_block_correlator(plan, dptr(U), dptr(D), n_sets, T, L, _mom(p), dptr(C), sptr(stream)), ctx)


def mbc_block_correlator_local(plan, U, D, n_sets, T, V3, C, site_out=None, stream=None, ctx=None):
    """The block form of the local-sink correlator (same quantity as mbc_correlator)."""
    check(load().mbc_block_correlator_local(plan, dptr(U), dptr(D), n_sets, T, V3, dptr(C), dptr(site_out),
                                            sptr(stream)), ctx)
