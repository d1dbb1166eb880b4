// blocks_api.cu - C ABI of the hadron-block path (see include/mbc.h): per-site and
// momentum-projected blocks (arXiv 2201.04269 Sec. 2), block plans and the block form of
// the correlator (Secs. 3-4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "mbc.h"
#include "blocks.cuh"
#include "blocks.hpp"
#include "ctx.hpp"

using namespace mbc;

struct mbc_block_plan {
    mbc_ctx* ctx = nullptr;
    BlockHostPlan hp;
    void* dev = nullptr;
    BlockDev bd{};
    BlockTreeDev td{};
};

namespace {

void fill_types(BlockDev& b, const std::vector<int>& types) {
    b.n_types = (int)types.size();
    for (size_t i = 0; i < types.size(); ++i) {
        GammaNz g;
        block_gamma(types[i], g);
        BlockTypeDev& t = b.t[i];
        t.q1 = block_q1(types[i]);
        t.n = g.n;
        for (int k = 0; k < g.n && k < 4; ++k) {
            t.be[k] = g.be[k];
            t.ga[k] = g.ga[k];
            t.g_re[k] = g.g[k].real();
            t.g_im[k] = g.g[k].imag();
        }
    }
}

mbc_status check_fields(mbc_ctx* c, const void* U, const void* D, int64_t n_sites) {
    if (!c) return MBC_INVALID_ARG;
    if (c->device < 0) return fail(c, MBC_UNSUPPORTED, "host-only context (device -1) cannot evaluate");
    if (n_sites < 0) return fail(c, MBC_INVALID_ARG, "negative size");
    if (n_sites > 0 && (!U || !D)) return fail(c, MBC_INVALID_ARG, "null propagator field");
    return MBC_OK;
}

// projected blocks of b into F (n_slices x b.n_f complex double; NULL = the context's
// buffer), with the tile partials in the context's pool
mbc_status project(mbc_ctx* c, const BlockDev& b, int prec, const void* U, const void* D, int64_t n_slices, int64_t V3,
                   int L, const int* p, void* F, cudaStream_t s) {
    const int64_t nscr = block_project_scratch(b.n_f, b.n_types, n_slices, V3, c->sms);
    mbc_status st = ensure(c, c->blk_part, sizeof(cd) * (size_t)std::max<int64_t>(nscr, 1), s);
    if (st != MBC_OK) return st;
    if (!F) {
        st = ensure(c, c->blk_F, sizeof(cd) * (size_t)std::max<int64_t>(n_slices * b.n_f, 1), s);
        if (st != MBC_OK) return st;
        F = c->blk_F.p;
    }
    cudaError_t e = launch_blocks_projected(b, prec, (const double*)U, (const double*)D, n_slices, V3, L, p, (cd*)c->blk_part.p,
                                            (cd*)F, c->sms, s, &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "projected block launch");
    return MBC_OK;
}

mbc_status check_lattice(mbc_ctx* c, int n_sets, int T, int L) {
    if (n_sets < 0 || T < 0 || L < 0) return fail(c, MBC_INVALID_ARG, "negative size");
    if (L > 1290) return fail(c, MBC_UNSUPPORTED, "L^3 sites per slice beyond the supported range");
    return MBC_OK;
}

}  // namespace

namespace mbc {
void destroy_block_plans(mbc_ctx* c) {
    for (mbc_block_plan* p : c->block_plans) {
        if (p->dev) cudaFree(p->dev);
        delete p;
    }
    c->block_plans.clear();
}
}  // namespace mbc

extern "C" {

mbc_status mbc_hadron_blocks(mbc_ctx* c, int type, const void* U, const void* D, int64_t n_sites, void* f,
                             mbc_stream stream) {
    Range range_("mbc_hadron_blocks");
    mbc_status st = check_fields(c, U, D, n_sites);
    if (st != MBC_OK) return st;
    if (type < 0 || type >= kBlockTypes) return fail(c, MBC_INVALID_ARG, "unknown block type");
    if (n_sites > 0 && !f) return fail(c, MBC_INVALID_ARG, "null output");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    BlockDev b{};
    b.n_f = kEta;
    b.entry = nullptr;
    fill_types(b, std::vector<int>{type});
    e = launch_blocks_site(b, (const double*)U, (const double*)D, n_sites, (cd*)f, c->sms, (cudaStream_t)stream,
                           &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "block launch");
    c->err.clear();
    return MBC_OK;
}

mbc_status mbc_hadron_blocks_projected(mbc_ctx* c, int type, const void* U, const void* D, int n_sets, int T, int L,
                                       const int* p, void* F, mbc_stream stream) {
    Range range_("mbc_hadron_blocks_projected");
    if (!c) return MBC_INVALID_ARG;
    mbc_status st = check_lattice(c, n_sets, T, L);
    if (st != MBC_OK) return st;
    const int64_t V3 = (int64_t)L * L * L, n_slices = (int64_t)n_sets * T;
    st = check_fields(c, U, D, n_slices * V3);
    if (st != MBC_OK) return st;
    if (type < 0 || type >= kBlockTypes) return fail(c, MBC_INVALID_ARG, "unknown block type");
    if (n_slices > 0 && !F) return fail(c, MBC_INVALID_ARG, "null output");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    BlockDev b{};
    b.n_f = kEta;
    b.entry = nullptr;
    fill_types(b, std::vector<int>{type});
    cudaStream_t s = (cudaStream_t)stream;
    if (n_slices > 0) {
        st = project(c, b, MBC_PREC_FP64, U, D, n_slices, V3, L, p, F, s);
        if (st != MBC_OK) return st;
    }
    c->err.clear();
    return MBC_OK;
}

mbc_status mbc_block_plan_create(mbc_ctx* c, int op, int prec, mbc_block_plan** out) {
    Range range_("mbc_block_plan_create");
    if (!c || !out) return MBC_INVALID_ARG;
    *out = nullptr;
    if (op < 0 || op > MBC_OP_HE3_II_S) return fail(c, MBC_INVALID_ARG, "unknown operator");
    if (prec != MBC_PREC_FP64 && prec != MBC_PREC_MIXED) return fail(c, MBC_INVALID_ARG, "unknown precision");
    mbc_block_plan* P = new (std::nothrow) mbc_block_plan();
    if (!P) return fail(c, MBC_OOM, "host allocation failed");
    P->ctx = c;
    P->hp.op = op;
    P->hp.prec = prec;
    std::string err;
    try {
        err = plan_blocks(P->hp);
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(c, MBC_OOM, "host allocation failed while planning");
    }
    if (!err.empty()) { delete P; return fail(c, MBC_INVALID_ARG, err); }
    BlockHostPlan& h = P->hp;
    std::vector<float2> lw(h.w.size());
    for (size_t i = 0; i < h.w.size(); ++i) {
        lw[i] = make_float2((float)h.w[i].real(), (float)h.w[i].imag());
        if ((double)lw[i].x != h.w[i].real() || (double)lw[i].y != h.w[i].imag()) {
            delete P;
            return fail(c, MBC_UNSUPPORTED, "merged block weight not exact in float");
        }
    }
    if (c->device >= 0 && !h.w.empty()) {
        cudaError_t e = cudaSetDevice(c->device);
        if (e != cudaSuccess) { delete P; return cuda_fail(c, e, "cudaSetDevice"); }
        // packed entries
        std::vector<uint32_t> entry(h.factor.size());
        for (size_t f = 0; f < h.factor.size(); ++f) {
            const int g = h.factor[f], type = g / kEta, eta = g % kEta;
            const int slot = (int)(std::lower_bound(h.types.begin(), h.types.end(), type) - h.types.begin());
            const int s1 = eta / 576, s2 = (eta / 48) % 12, s3 = (eta / 4) % 12, al = eta % 4;
            entry[f] = (uint32_t)((slot << 16) | (s1 << 12) | (s2 << 8) | (s3 << 4) | al);
        }
        // chunks of units with about equal leaf counts: two per SM for one slice
        const int64_t n_units = (int64_t)h.unit_leaf.size() - 1;
        const int64_t K = (int64_t)h.w.size();
        const int64_t n_chunks = std::max<int64_t>(1, std::min<int64_t>(2LL * std::max(c->sms, 1), (n_units + 63) / 64));
        std::vector<int64_t> chunk_unit(1, 0);
        for (int64_t k = 1; k < n_chunks; ++k) {
            const int64_t target = K * k / n_chunks;
            int64_t u = std::upper_bound(h.unit_leaf.begin(), h.unit_leaf.end(), (int32_t)target) - h.unit_leaf.begin() - 1;
            u = std::max(u, chunk_unit.back());
            chunk_unit.push_back(u);
        }
        chunk_unit.push_back(n_units);
        // one device allocation: entries | unit_pre | unit_leaf | leaf_f | leaf_w | chunk_unit
        size_t off = 0;
        auto place = [&](size_t bytes) { size_t o = off; off = (off + bytes + 255) / 256 * 256; return o; };
        const size_t o_e = place(entry.size() * 4), o_pre = place(h.unit_pre.size() * 2),
                     o_ul = place(h.unit_leaf.size() * 4), o_lf = place(h.leaf_f.size() * 2),
                     o_lw = place(lw.size() * 8), o_lwd = place(h.w.size() * 16), o_cu = place(chunk_unit.size() * 8);
        std::vector<unsigned char> blob(std::max<size_t>(off, 256));
        std::memcpy(blob.data() + o_e, entry.data(), entry.size() * 4);
        if (!h.unit_pre.empty()) std::memcpy(blob.data() + o_pre, h.unit_pre.data(), h.unit_pre.size() * 2);
        std::memcpy(blob.data() + o_ul, h.unit_leaf.data(), h.unit_leaf.size() * 4);
        std::memcpy(blob.data() + o_lf, h.leaf_f.data(), h.leaf_f.size() * 2);
        std::memcpy(blob.data() + o_lw, lw.data(), lw.size() * 8);
        for (size_t i = 0; i < h.w.size(); ++i) {
            const double wd[2] = {h.w[i].real(), h.w[i].imag()};
            std::memcpy(blob.data() + o_lwd + 16 * i, wd, 16);
        }
        std::memcpy(blob.data() + o_cu, chunk_unit.data(), chunk_unit.size() * 8);
        e = cudaMalloc(&P->dev, blob.size());
        if (e != cudaSuccess) { delete P; return fail(c, MBC_OOM, std::string("cudaMalloc of block plan: ") + cudaGetErrorString(e)); }
        e = cudaMemcpy(P->dev, blob.data(), blob.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(P->dev); delete P; return cuda_fail(c, e, "cudaMemcpy of block plan"); }
        unsigned char* base = static_cast<unsigned char*>(P->dev);
        P->bd.n_f = (int)entry.size();
        P->bd.entry = reinterpret_cast<const uint32_t*>(base + o_e);
        fill_types(P->bd, h.types);
        P->td.A = h.A;
        P->td.n_f = (int)entry.size();
        P->td.n_units = n_units;
        P->td.unit_pre = reinterpret_cast<const uint16_t*>(base + o_pre);
        P->td.unit_leaf = reinterpret_cast<const int32_t*>(base + o_ul);
        P->td.leaf_f = reinterpret_cast<const uint16_t*>(base + o_lf);
        P->td.leaf_w = reinterpret_cast<const float2*>(base + o_lw);
        P->td.leaf_wd = reinterpret_cast<const double2*>(base + o_lwd);
        P->td.n_chunks = (int)n_chunks;
        P->td.chunk_unit = reinterpret_cast<const int64_t*>(base + o_cu);
    }
    c->block_plans.push_back(P);
    *out = P;
    c->err.clear();
    return MBC_OK;
}

void mbc_block_plan_destroy(mbc_block_plan* P) {
    if (!P) return;
    mbc_ctx* c = P->ctx;
    auto it = std::find(c->block_plans.begin(), c->block_plans.end(), P);
    if (it != c->block_plans.end()) c->block_plans.erase(it);
    if (P->dev) {
        cudaSetDevice(c->device);
        cudaDeviceSynchronize();
        cudaFree(P->dev);
    }
    delete P;
}

mbc_status mbc_block_plan_get_info(const mbc_block_plan* P, mbc_block_plan_info* info) {
    if (!P || !info) return MBC_INVALID_ARG;
    const BlockHostPlan& h = P->hp;
    std::memset(info, 0, sizeof(*info));
    info->n_baryons = h.A;
    info->n_products = (int)h.n_w.size();
    for (size_t i = 0; i < h.n_w.size() && i < 8; ++i) info->n_w[i] = h.n_w[i];
    info->expanded_terms = h.expanded;
    info->merged_terms = (int64_t)h.w.size();
    info->factors = (int64_t)h.factor.size();
    for (int a = 0; a < 4; ++a) info->level_nodes[a] = h.level_nodes[a];
    info->block_flops_per_site = h.block_flops_per_site;
    info->tree_flops_per_slice = h.tree_flops_per_slice;
    info->shared_sums = h.shared_sums;
    info->shared_sum_terms = h.shared_sum_terms;
    return MBC_OK;
}

mbc_status mbc_block_plan_get_terms(const mbc_block_plan* P, int32_t* ids, double* w) {
    if (!P || !ids || !w) return MBC_INVALID_ARG;
    const BlockHostPlan& h = P->hp;
    std::copy(h.ids.begin(), h.ids.end(), ids);
    for (size_t i = 0; i < h.w.size(); ++i) {
        w[2 * i] = h.w[i].real() * h.scale;
        w[2 * i + 1] = h.w[i].imag() * h.scale;
    }
    return MBC_OK;
}

mbc_status mbc_block_correlator_local(mbc_block_plan* P, const void* U, const void* D, int n_sets, int T, int64_t V3,
                                      void* C, void* site_out, mbc_stream stream) {
    Range range_("mbc_block_correlator_local");
    if (!P) return MBC_INVALID_ARG;
    mbc_ctx* c = P->ctx;
    if (n_sets < 0 || T < 0 || V3 < 0) return fail(c, MBC_INVALID_ARG, "negative size");
    const int64_t n_sites = (int64_t)n_sets * T * V3, n_slices = (int64_t)n_sets * T;
    mbc_status st = check_fields(c, U, D, n_sites);
    if (st != MBC_OK) return st;
    if (n_slices > 0 && !C) return fail(c, MBC_INVALID_ARG, "null output");
    if (n_sites > ((int64_t)1 << 32)) return fail(c, MBC_UNSUPPORTED, "more than 2^32 sites in one call");
    if (P->hp.prec != MBC_PREC_FP64) return fail(c, MBC_UNSUPPORTED, "the local block form evaluates in MBC_PREC_FP64 plans");
    if (!P->hp.w.empty() && block_kernel_smem(P->bd.n_f, P->bd.n_types, true) > 200 * 1024)
        return fail(c, MBC_UNSUPPORTED, "the plan's block entries do not fit shared memory for the local block form");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (n_slices == 0) { c->err.clear(); return MBC_OK; }
    if (P->hp.w.empty() || n_sites == 0) {
        e = cudaMemsetAsync(C, 0, sizeof(double2) * (size_t)n_slices, s);
        if (e == cudaSuccess && site_out && n_sites) e = cudaMemsetAsync(site_out, 0, sizeof(double2) * (size_t)n_sites, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
        c->err.clear();
        return MBC_OK;
    }
    st = ensure(c, c->partials, sizeof(d4) * (size_t)n_sites, s);
    if (st == MBC_OK && site_out) st = ensure(c, c->site_tmp, sizeof(d4) * (size_t)n_sites, s);
    if (st != MBC_OK) return st;
    e = launch_block_local(P->bd, P->td, (const double*)U, (const double*)D, n_sites, (d4*)c->partials.p, c->sms, s,
                           &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "local block kernel launch");
    Geometry g{n_sets, T, V3};
    Partials pt{(d4*)c->partials.p, 1};
    e = launch_reduce(pt, g, cd_make(P->hp.scale, 0.0), (double2*)C, (double2*)site_out, (d4*)c->site_tmp.p, s,
                      &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduction launch");
    c->err.clear();
    return MBC_OK;
}

mbc_status mbc_block_plan_get_multiplicities(const mbc_block_plan* P, int32_t* multiplicity) {
    if (!P || !multiplicity) return MBC_INVALID_ARG;
    std::copy(P->hp.multiplicity.begin(), P->hp.multiplicity.end(), multiplicity);
    return MBC_OK;
}

mbc_status mbc_block_correlator(mbc_block_plan* P, const void* U, const void* D, int n_sets, int T, int L,
                                const int* p, void* C, mbc_stream stream) {
    Range range_("mbc_block_correlator");
    if (!P) return MBC_INVALID_ARG;
    mbc_ctx* c = P->ctx;
    mbc_status st = check_lattice(c, n_sets, T, L);
    if (st != MBC_OK) return st;
    const int64_t V3 = (int64_t)L * L * L, n_slices = (int64_t)n_sets * T;
    st = check_fields(c, U, D, n_slices * V3);
    if (st != MBC_OK) return st;
    if (n_slices > 0 && !C) return fail(c, MBC_INVALID_ARG, "null output");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (n_slices == 0) { c->err.clear(); return MBC_OK; }
    if (P->hp.w.empty() || V3 == 0) {
        e = cudaMemsetAsync(C, 0, sizeof(double2) * (size_t)n_slices, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
        c->err.clear();
        return MBC_OK;
    }
    st = project(c, P->bd, P->hp.prec, U, D, n_slices, V3, L, p, nullptr, s);
    if (st != MBC_OK) return st;
    st = ensure(c, c->blk_tree, sizeof(d4) * (size_t)(n_slices * P->td.n_chunks), s);
    if (st != MBC_OK) return st;
    e = launch_block_tree(P->td, P->hp.prec, (const cd*)c->blk_F.p, n_slices, (d4*)c->blk_tree.p, s, &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "block tree launch");
    Geometry g{n_sets, T, (int64_t)P->td.n_chunks};
    Partials pt{(d4*)c->blk_tree.p, 1};
    e = launch_reduce(pt, g, cd_make(P->hp.scale, 0.0), (double2*)C, nullptr, nullptr, s, &c->launches);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduction launch");
    c->err.clear();
    return MBC_OK;
}

}  // extern "C"
