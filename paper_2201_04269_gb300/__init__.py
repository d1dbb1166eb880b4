"""GB300-native multi-baryon correlators (arXiv 2201.04269): libmbc and its Python binding.

The product is the C-ABI library ``libmbc.so`` (include/mbc.h) built from ``csrc/`` for
sm_103a; ``abi`` binds its entry points one to one, and ``Context``/``Plan`` below are a
small convenience layer over them (argument marshalling only; every step of the
correlator runs in the library).  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

from . import abi
from .abi import ALGO, OPERATOR, PREC, MbcError


class Context:
    """Owns an mbc context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.handle = abi.mbc_create(device)
        self.device = device

    def close(self):
        if self.handle:
            abi.mbc_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def launches(self):
        return abi.mbc_launch_count(self.handle)

    @property
    def fp32_recomputed(self):
        """Sites the last MBC_PREC_FP32 evaluation recomputed in double-float (synchronises)."""
        return abi.mbc_fp32_recomputed(self.handle)

    def plan(self, problem: dict, algo="egraph", prec="fp64"):
        """Plan a factored problem (dict with n_u, n_d, idx, w, offsets, proj, scale and
        optionally src_idx/src_w/src_offsets; the source defaults to the sink)."""
        h = abi.mbc_plan_create(self.handle, problem["n_u"], problem["n_d"], problem["idx"], problem["w"],
                                problem["offsets"], problem.get("src_idx", problem["idx"]),
                                problem.get("src_w", problem["w"]), problem.get("src_offsets", problem["offsets"]),
                                problem["proj"], problem["scale"], algo, prec)
        return Plan(self, h)

    def plan_operator(self, name: str, algo="egraph", prec="fp64"):
        return self.plan(abi.mbc_operator_terms(name), algo, prec)

    def plan_terms(self, n_u, n_d, sink, source, W, scale=1.0, algo="direct", prec="fp64"):
        return Plan(self, abi.mbc_plan_from_terms(self.handle, n_u, n_d, sink, source, W, scale, algo, prec))

    def load_plan(self, path):
        return Plan(self, abi.mbc_plan_load(self.handle, path))

    def batch(self, items, stream=None):
        abi.mbc_batch(self.handle, items, stream)

    def block_plan(self, name: str, prec="fp64"):
        """Block form of a library operator (hadron blocks, Secs. 2-4)."""
        return BlockPlan(self, abi.mbc_block_plan_create(self.handle, name, prec))

    def hadron_blocks(self, block_type, U, D, f, stream=None):
        """Per-site blocks: U, D cuda complex128 [..., 12, 12]; f [..., 6912]."""
        n_sites = U.numel() // 144
        abi.mbc_hadron_blocks(self.handle, block_type, U, D, n_sites, f, stream)

    def hadron_blocks_projected(self, block_type, U, D, F, L, p=None, stream=None):
        """Projected blocks: U, D [n_sets, T, L^3, 12, 12]; F [n_sets, T, 6912]."""
        n_sets, T = U.shape[:2]
        abi.mbc_hadron_blocks_projected(self.handle, block_type, U, D, n_sets, T, L, F, p, stream)


class Plan:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    def destroy(self):
        if self.handle:
            abi.mbc_plan_destroy(self.handle)
            self.handle = None

    @property
    def info(self):
        return abi.mbc_plan_get_info(self.handle)

    def correlator(self, U, D, C, site_out=None, stream=None):
        """U, D: cuda complex128 tensors [n_sets, T, V3, 12, 12]; C: cuda complex128 [n_sets, T]."""
        n_sets, T, V3 = U.shape[:3]
        abi.mbc_correlator(self.handle, U, D, n_sets, T, V3, C, site_out, stream, self.ctx.handle)

    def correlator_momentum(self, U, D, C, L, p, site_out=None, stream=None):
        """Sink momentum p (units of 2 pi / L): U, D [n_sets, T, L^3, 12, 12]; C [n_sets, T]."""
        n_sets, T = U.shape[:2]
        abi.mbc_correlator_momentum(self.handle, U, D, n_sets, T, L, p, C, site_out, stream, self.ctx.handle)

    def correlator_host(self, U, D, C, stream=None):
        n_sets, T, V3 = U.shape[:3]
        abi.mbc_correlator_host(self.handle, U, D, n_sets, T, V3, C, stream, self.ctx.handle)

    def set_guard(self, site_threshold=None, slice_tolerance=None):
        """Guards of an MBC_PREC_FP32 plan: the per-site error-estimate threshold and the
        relative error tolerance of C(t); sites they flag are recomputed in double-float
        arithmetic (None keeps the current value)."""
        cur = self.guard
        abi.mbc_plan_set_guard(self.handle, cur[0] if site_threshold is None else site_threshold,
                               cur[1] if slice_tolerance is None else slice_tolerance, self.ctx.handle)

    @property
    def guard(self):
        """(site threshold, slice tolerance)"""
        return abi.mbc_plan_get_guard(self.handle)

    def autotune(self, U, D, n_sites, stream=None):
        return abi.mbc_autotune(self.handle, U, D, n_sites, stream, self.ctx.handle)

    def save(self, path):
        abi.mbc_plan_save(self.handle, path, self.ctx.handle)

    def tree(self):
        return abi.mbc_plan_get_tree(self.handle)


class BlockPlan:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle

    def destroy(self):
        if self.handle:
            abi.mbc_block_plan_destroy(self.handle)
            self.handle = None

    @property
    def info(self):
        return abi.mbc_block_plan_get_info(self.handle)

    def terms(self):
        return abi.mbc_block_plan_get_terms(self.handle)

    def correlator(self, U, D, C, L, p=None, stream=None):
        """Every sink baryon projected to momentum p: U, D [n_sets, T, L^3, 12, 12]; C [n_sets, T]."""
        n_sets, T = U.shape[:2]
        abi.mbc_block_correlator(self.handle, U, D, n_sets, T, L, C, p, stream, self.ctx.handle)

    def correlator_local(self, U, D, C, site_out=None, stream=None):
        """Local sink (the quantity of Plan.correlator): U, D [n_sets, T, V3, 12, 12]; C [n_sets, T]."""
        n_sets, T, V3 = U.shape[:3]
        abi.mbc_block_correlator_local(self.handle, U, D, n_sets, T, V3, C, site_out, stream, self.ctx.handle)


__all__ = ["abi", "Context", "Plan", "BlockPlan", "MbcError", "ALGO", "PREC", "OPERATOR"]
