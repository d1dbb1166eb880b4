// api.cu - the C ABI of libmbc (see include/mbc.h): contexts, plans, device upload,
// evaluation, batching, autotuning and plan files.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mbc.h"
#include "device.cuh"
#include "plan.hpp"
#include "walk.hpp"
#include "tegraph.hpp"
#include "checks.cuh"
#include "noalloc.hpp"
#include "ctx.hpp"

using namespace mbc;

namespace {
// Default guards of MBC_PREC_FP32 plans (see include/mbc.h): the per-site error-estimate
// threshold and the relative error tolerance of C(t).
constexpr double kDefaultGuard = 2.0;
constexpr double kDefaultSliceTol = 1e-6;
}

namespace mbc {
// Shape of an MBC_PREC_FP32 plan's kernel: walkers per block (128 threads each), A leaves
// per leaf batch, blocks per site (a cluster sharing the site's B table); 0 = automatic.
struct F32Shape {
    int walkers = 0, leaf_batch = 0, cluster = 0;
};
}  // namespace mbc

struct mbc_plan {
    mbc_ctx* ctx = nullptr;
    HostPlan hp;
    void* dev = nullptr;          // one device allocation holding every plan array
    size_t dev_bytes = 0;
    DirectDev dd{};
    TreeDev td{};
    EgraphDev ed{};
    Eg32Dev e32{};                // FP32 e-graph view (MBC_PREC_FP32 plans)
    void* dev32 = nullptr;        // its arrays (walk programs, packed words, G and pair records)
    mbc::F32Shape f32_shape;      // forced walkers / leaf batch / blocks per site (0: automatic)
    mbc_schedule sched{256, 2, 1};
    mbc_schedule sched_df{384, 1, 1};   // the double-float recompute of flagged sites (MBC_PREC_FP32)
    double guard = kDefaultGuard;        // per-site error-estimate threshold (MBC_PREC_FP32)
    double slice_tol = kDefaultSliceTol; // relative error tolerance of C(t) (MBC_PREC_FP32)
    std::string signature;
};

namespace mbc {

mbc_status fail(mbc_ctx* c, mbc_status s, const std::string& m) {
    if (c) c->err = m;
    return s;
}

mbc_status cuda_fail(mbc_ctx* c, cudaError_t e, const char* what) {
    return fail(c, MBC_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Bounds-checking build: synchronise and turn a recorded device check into an error
// (normal build: nothing).
mbc_status post_checks(mbc_ctx* c, const char* what) {
#ifdef MBC_DEVICE_CHECKS
    CheckRecord r1, r2;
    cudaError_t e = egraph32_checks(&r1);
    if (e == cudaSuccess) e = egraph_checks(&r2);
    if (e != cudaSuccess) return cuda_fail(c, e, what);
    for (const CheckRecord* r : {&r1, &r2})
        if (r->count > 0) {
            char buf[256];
            snprintf(buf, sizeof buf, "%s: device check %d failed %d time(s): value %lld, bound %lld", what, r->code,
                     r->count, r->value, r->bound);
            return fail(c, MBC_CUDA, buf);
        }
#else
    (void)c;
    (void)what;
#endif
    return MBC_OK;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// Grow a pool buffer (never during a stream capture).
mbc_status ensure(mbc_ctx* c, Buf& b, size_t bytes, cudaStream_t s) {
    if (b.n >= bytes) return MBC_OK;
    if (capturing(s))
        return fail(c, MBC_OOM, "device pool too small while a stream capture is active: run the call once "
                                "outside the capture (or mbc_batch_reserve) first");
    if (b.p) {
        cudaStreamSynchronize(s);
        cudaFree(b.p);
        b.p = nullptr;
        b.n = 0;
    }
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) return fail(c, MBC_OOM, std::string("cudaMalloc of pool buffer failed: ") + cudaGetErrorString(e));
    b.n = want;
    return MBC_OK;
}

}  // namespace mbc

namespace {

// ---------------------------------------------------------------- device upload
struct Blob {
    std::vector<unsigned char> host;
    std::vector<std::pair<size_t, void**>> fixups;
    template <class T> size_t add(const T* p, size_t n) {
        size_t off = (host.size() + 255) / 256 * 256;
        host.resize(off + n * sizeof(T));
        if (n) std::memcpy(host.data() + off, p, n * sizeof(T));
        return off;
    }
    template <class T> size_t add(const std::vector<T>& v) { return add(v.data(), v.size()); }
};

template <class T> const T* at(void* base, size_t off) { return reinterpret_cast<const T*>(static_cast<unsigned char*>(base) + off); }

// 16-byte device values of a precision: complex double, or complex double-float
// (each part split into hi = float(x), lo = float(x - hi))
struct Val16 { unsigned char b[16]; };
std::vector<Val16> to_val(const std::vector<cplx>& v, int prec) {
    std::vector<Val16> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        if (prec == 0) {
            double x[2] = {v[i].real(), v[i].imag()};
            std::memcpy(o[i].b, x, 16);
        } else {
            float x[4];
            const double re = v[i].real(), im = v[i].imag();
            x[0] = (float)re; x[1] = (float)(re - (double)x[0]);
            x[2] = (float)im; x[3] = (float)(im - (double)x[2]);
            std::memcpy(o[i].b, x, 16);
        }
    }
    return o;
}

std::vector<cd> to_cd(const std::vector<cplx>& v) {
    std::vector<cd> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = cd_make(v[i].real(), v[i].imag());
    return o;
}

void minor_dev_offsets(const MinorPlan& m, int upto, int* size, int* off) {
    int acc = 0;
    for (int k = 0; k < 7; ++k) {
        size[k] = (k == 0) ? 1 : (k <= m.n ? (int)m.level_rows[k].size() : 0);
        off[k] = acc;
        if (k <= upto) acc += size[k];
    }
}

// ---------------------------------------------------------------- FP32 e-graph arrays
struct F32Offsets {
    bool used = false;
    size_t steps[2], step_off[2], leaves[2], pk, sell_off, sell_w, sell, sellc, sell1, term_off, term2, term4, jmask, b_pos;
};

// Walker count and leaf batch size that fit the kernel's shared memory: as many walkers
// (up to 6, i.e. 768 threads: the kernel's register budget) and then as large a batch
// (up to 3: larger batches measured slower) as fit.
int f32_smem(int W, int LB, int pk_words, int stack_vals, int leaf_size) {
    return 2 * kBlk * 8 + pk_words * 4 + W * (stack_vals + LB * leaf_size) * 8;
}

std::string add_f32(const HostPlan& h, const F32Shape& shape, Eg32Dev& v, Blob& b, F32Offsets& o) {
    const EgraphPlan& e = h.eg;
    if (e.n_j < 1 || e.n_j > 4) return "MBC_PREC_FP32 supports at most 4 free indices in use";
    const MinorPlan* mp[2] = {&e.A, &e.B};
    WalkDev* wd[2] = {&v.A, &v.B};
    int stack[2] = {0, 0};
    int pk_words = 0;
    for (int f = 0; f < 2; ++f) {
        const MinorPlan& m = *mp[f];
        WalkDev& x = *wd[f];
        x = WalkDev();
        x.n = m.n;
        x.size[0] = 1;
        for (int k = 1; k < 7; ++k) x.size[k] = k <= m.n ? (int)m.level_rows[k].size() : 0;
        int acc = 0;
        for (int k = 0; k < 7; ++k) {
            x.off[k] = acc;
            if (k < m.n) acc += x.size[k];
        }
        stack[f] = std::max(1, acc);
        for (int k = 1; k <= m.n; ++k) {
            x.pk_off[k] = pk_words;
            pk_words += x.size[k] * k;
        }
    }
    pk_words = (pk_words + 3) / 4 * 4;
    const int nA = e.A.n;
    const int leaf_size = v.A.size[nA];
    const int stack_vals = std::max(stack[0], stack[1]);
    // (the leaf stage keeps G of every leaf of a batch in registers: one leaf per batch
    // when more than two free indices are in use)
    const int max_lb = std::min(e.n_j <= 2 ? 3 : 1, kMaxLeafBatch);
    int W = 0, LB = 0;
    if (shape.walkers) {
        if (shape.walkers < 1 || shape.walkers > 6 || shape.leaf_batch < 1 || shape.leaf_batch > max_lb ||
            shape.cluster < 0 || shape.cluster > 2)
            return "MBC_PREC_FP32 shape out of range (walkers 1..6, leaf batch 1..3 (1 with more than two free "
                   "indices), blocks per site 1..2)";
        if (f32_smem(shape.walkers, shape.leaf_batch, pk_words, stack_vals, leaf_size) > 220 * 1024)
            return "MBC_PREC_FP32 shape needs more shared memory than a block has";
        W = shape.walkers;
        LB = shape.leaf_batch;
    }
    for (int w : {6, 4, 2, 1}) {
        if (W) break;
        for (int lb = max_lb; lb >= 1 && !W; --lb)
            if (f32_smem(w, lb, pk_words, stack_vals, leaf_size) <= 220 * 1024) { W = w; LB = lb; }
    }
    if (!W) return "MBC_PREC_FP32: the plan's tables do not fit shared memory";
    const int nrb = e.B.n ? (int)e.B.level_rows[e.B.n].size() : 1;
    const int ncb = e.B.n ? (int)e.B.cols.size() : 1;
    const int nj = e.n_j;
    // walker programs, leaves balanced by cost
    std::vector<int64_t> nnz_j(nj, 0);
    for (int rb = 0; rb < nrb; ++rb)
        for (int j = 0; j < nj; ++j) nnz_j[j] += e.g_off[rb * nj + j + 1] - e.g_off[rb * nj + j];
    std::vector<double> costA(e.A.cols.size(), 0.0), costB(e.B.n ? e.B.cols.size() : 1, 1.0);
    for (size_t l = 0; l < costA.size(); ++l) {
        const int np = e.pair_off[l + 1] - e.pair_off[l];
        double c = 4.0 * nA * leaf_size + (double)nrb * (16.0 + 10.0 * np);
        for (int j = 0; j < nj; ++j) {
            bool used = false;
            for (int q = e.pair_off[l]; q < e.pair_off[l + 1]; ++q) used = used || e.pair_coef[(size_t)q * nj + j] != 0.0;
            if (used) c += 2.0 * nnz_j[j];
        }
        costA[l] = c;
    }
    // blocks per site: one unless the shape asks for two (a thread-block cluster sharing
    // one B table, which halves the tables in flight in L2 but adds two cluster barriers
    // and an exchange per site: measured 5 % slower on 3He_II-s at 24^3 x 48, where one
    // table per SM, 152 x 0.94 MB, slightly exceeds the L2)
    const int cs = shape.cluster ? shape.cluster : 1;
    Walks wk[2];
    std::string err = build_walks(e.A, cs * W, LB, costA, wk[0]);
    if (err.empty()) err = build_walks(e.B, cs * W, kMaxLeafBatch, costB, wk[1]);
    if (!err.empty()) return err;
    for (int f = 0; f < 2; ++f) {
        o.steps[f] = b.add(wk[f].steps);
        o.step_off[f] = b.add(wk[f].step_off);
        o.leaves[f] = b.add(wk[f].leaves);
    }
    // packed Laplace words (transposed per level), A levels then B levels
    std::vector<uint32_t> pk(pk_words, 0u);
    for (int f = 0; f < 2; ++f) {
        const MinorPlan& m = *mp[f];
        for (int k = 1; k <= m.n; ++k) {
            const size_t n = m.level_rows[k].size();
            for (size_t q = 0; q < n; ++q)
                for (int i = 0; i < k; ++i)
                    pk[wd[f]->pk_off[k] + i * n + q] =
                        (uint32_t)m.child[k][q * k + i] | ((uint32_t)m.row[k][q * k + i] << 16);
        }
    }
    o.pk = b.add(pk);
    // B row sets ordered by their G entry counts (descending, free index 0 first, then 1, ...,
    // then by index), so that a slice's 32 row sets have similar widths for every free
    // index (3He_II-s: 1.44x the entries in padded slots instead of 1.61x): the leaf stage's
    // row b is B leaf-level row set order[b], and the B table is written in that order
    std::vector<int32_t> order(nrb), b_pos(nrb);
    {
        auto cnt = [&](int rb, int j) { return e.B.n ? e.g_off[rb * nj + j + 1] - e.g_off[rb * nj + j] : 0; };
        for (int rb = 0; rb < nrb; ++rb) order[rb] = rb;
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            for (int j = 0; j < nj; ++j)
                if (cnt(x, j) != cnt(y, j)) return cnt(x, j) > cnt(y, j);
            return false;
        });
        for (int b = 0; b < nrb; ++b) b_pos[order[b]] = b;
    }
    o.b_pos = b.add(b_pos);
    // G entries in sliced-ELL form (FP32 weights); 4-byte entries (index | bf16 weight)
    // when every weight is real with at most 8 significant bits
    bool real = true, small = true;
    for (auto& x : e.g_w) {
        real = real && x.imag() == 0.0;
        const float f = (float)x.real();
        uint32_t bits;
        std::memcpy(&bits, &f, 4);
        small = small && x.imag() == 0.0 && (double)f == x.real() && (bits & 0xFFFFu) == 0;
    }
    for (auto& x : e.pair_coef) real = real && x.imag() == 0.0;
    for (int32_t a : e.g_a) small = small && a < 65536;
    small = small && real;
    std::vector<int32_t> soff, sw;
    std::vector<int2> sr;
    std::vector<int4> sc;
    std::vector<uint32_t> s1;
    const int n_slices = (nrb + 31) / 32;
    size_t rec = 0;
    for (int sl = 0; sl < n_slices; ++sl)
        for (int j = 0; j < nj; ++j) {
            int width = 0;
            for (int l = 0; l < 32 && sl * 32 + l < nrb; ++l) {
                const int it = order[sl * 32 + l] * nj + j;
                width = std::max(width, e.g_off[it + 1] - e.g_off[it]);
            }
            soff.push_back((int32_t)rec);
            sw.push_back(width);
            // the complex form always (a batched launch with complex-weight items uses it
            // for every item), the real forms when the weights allow
            if (small) s1.resize(rec + (size_t)width * 32, 0u);
            if (real) sr.resize(rec + (size_t)width * 32, int2{0, 0});
            sc.resize(rec + (size_t)width * 32, int4{0, 0, 0, 0});
            for (int l = 0; l < 32 && sl * 32 + l < nrb; ++l) {
                const int it = order[sl * 32 + l] * nj + j;
                for (int k = 0; k < e.g_off[it + 1] - e.g_off[it]; ++k) {
                    const int a = e.g_a[e.g_off[it] + k];
                    const float wr = (float)e.g_w[e.g_off[it] + k].real(), wi = (float)e.g_w[e.g_off[it] + k].imag();
                    int br, bi;
                    std::memcpy(&br, &wr, 4);
                    std::memcpy(&bi, &wi, 4);
                    if (small) s1[rec + (size_t)k * 32 + l] = (uint32_t)a | ((uint32_t)br & 0xFFFF0000u);
                    if (real) sr[rec + (size_t)k * 32 + l] = int2{a, br};
                    sc[rec + (size_t)k * 32 + l] = int4{a, br, bi, 0};
                }
            }
            rec += (size_t)width * 32;
        }
    o.sell_off = b.add(soff);
    o.sell_w = b.add(sw);
    o.sell = b.add(sr);
    o.sellc = b.add(sc);
    o.sell1 = b.add(s1);
    // pair terms: one per pair and free index with a nonzero coefficient
    std::vector<int32_t> toff(1, 0);
    std::vector<int2> t2;
    std::vector<int4> t4;
    for (size_t l = 0; l + 1 < e.pair_off.size(); ++l) {
        for (int q = e.pair_off[l]; q < e.pair_off[l + 1]; ++q)
            for (int j = 0; j < nj; ++j) {
                const cplx cf = e.pair_coef[(size_t)q * nj + j];
                if (cf == 0.0) continue;
                const float cr = (float)cf.real(), ci = (float)cf.imag();
                int br, bi;
                std::memcpy(&br, &cr, 4);
                std::memcpy(&bi, &ci, 4);
                const int x = (e.pair_b[q] * nrb) * 4 + j;      // B-table offset of column C_b, free index
                if (real) t2.push_back(int2{x, br});
                t4.push_back(int4{x, br, bi, 0});
            }
        toff.push_back((int32_t)t4.size());
    }
    o.term_off = b.add(toff);
    o.term2 = b.add(t2);
    o.term4 = b.add(t4);
    v.g_small = small ? 1 : 0;
    std::vector<uint8_t> jm(e.A.cols.size(), 0);
    for (size_t l = 0; l < jm.size(); ++l)
        for (int q = e.pair_off[l]; q < e.pair_off[l + 1]; ++q)
            for (int j = 0; j < nj; ++j)
                if (e.pair_coef[(size_t)q * nj + j] != 0.0) jm[l] |= (uint8_t)(1u << j);
    o.jmask = b.add(jm);
    v.flav_a = e.flav_a;
    v.n_j = nj;
    v.real_w = real ? 1 : 0;
    v.walkers = W;
    v.cs = cs;
    v.lb = LB;
    v.n_rows_b = nrb;
    v.n_cols_b = ncb;
    v.stack_vals = stack_vals;
    v.leafbuf_vals = LB * leaf_size;
    v.pk_words = pk_words;
    v.smem_bytes = f32_smem(W, LB, pk_words, stack_vals, leaf_size);
    v.n_cols_a = (int)e.A.cols.size();
    v.n_terms = (int64_t)t4.size();
    v.n_sell = (int64_t)sc.size();
    for (int f = 0; f < 2; ++f) {
        wd[f]->n_steps = (int)wk[f].steps.size();
        wd[f]->n_leaves = (int)wk[f].leaves.size();
    }
    o.used = true;
    return "";
}

void bind_f32(Eg32Dev& v, void* dev, const F32Offsets& o, float guard) {
    WalkDev* wd[2] = {&v.A, &v.B};
    for (int f = 0; f < 2; ++f) {
        wd[f]->steps = at<WalkStep>(dev, o.steps[f]);
        wd[f]->step_off = at<int32_t>(dev, o.step_off[f]);
        wd[f]->leaves = at<WalkLeaf>(dev, o.leaves[f]);
    }
    v.pk = at<uint32_t>(dev, o.pk);
    v.sell_off = at<int32_t>(dev, o.sell_off);
    v.sell_w = at<int32_t>(dev, o.sell_w);
    v.sell = at<int2>(dev, o.sell);
    v.sellc = at<int4>(dev, o.sellc);
    v.sell1 = at<uint32_t>(dev, o.sell1);
    v.term_off = at<int32_t>(dev, o.term_off);
    v.term2 = at<int2>(dev, o.term2);
    v.term4 = at<int4>(dev, o.term4);
    v.leaf_jmask = at<uint8_t>(dev, o.jmask);
    v.b_pos = at<int32_t>(dev, o.b_pos);
    v.guard = guard;
}

// The FP32 view of an MBC_PREC_FP32 e-graph plan in its own device allocation (rebuilt
// alone when the plan's shape changes).  On failure P->dev32 and P->e32 are unchanged.
mbc_status upload_f32(mbc_plan* P) {
    const HostPlan& h = P->hp;
    if (!(h.prec == MBC_PREC_FP32 && h.algo == MBC_ALGO_EGRAPH && !h.terms.empty())) return MBC_OK;
    Blob b;
    F32Offsets f32;
    Eg32Dev v{};
    std::string msg = add_f32(h, P->f32_shape, v, b, f32);
    if (!msg.empty()) return fail(P->ctx, MBC_UNSUPPORTED, msg);
    void* dev = nullptr;
    cudaError_t err = cudaMalloc(&dev, std::max<size_t>(b.host.size(), 256));
    if (err != cudaSuccess) return fail(P->ctx, MBC_OOM, std::string("cudaMalloc of FP32 plan arrays failed: ") + cudaGetErrorString(err));
    err = cudaMemcpy(dev, b.host.data(), b.host.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) { cudaFree(dev); return cuda_fail(P->ctx, err, "cudaMemcpy of FP32 plan arrays"); }
    bind_f32(v, dev, f32, P->guard > 3.0e38 ? INFINITY : (float)std::max(P->guard, -1.0));
    if (P->dev32) {
        cudaDeviceSynchronize();        // work queued with the previous arrays
        cudaFree(P->dev32);
    }
    P->dev32 = dev;
    P->e32 = v;
    return MBC_OK;
}

// The schedule of an MBC_PREC_FP32 plan describes its kernel's shape: threads = 128 x
// walkers, blocks_per_sm = blocks per site (cluster size), sites_per_unit = leaf batch.
mbc_schedule f32_schedule(const Eg32Dev& v) { return mbc_schedule{128 * std::max(1, v.walkers), std::max(1, v.cs), std::max(1, v.lb)}; }

// Validate and apply a schedule.  For an MBC_PREC_FP32 plan a new shape rebuilds the
// plan's FP32 arrays (their device addresses change, so a batch reservation of the
// context is dropped and re-made by the next mbc_batch); on failure nothing changes.
mbc_status apply_schedule(mbc_plan* P, const mbc_schedule& s) {
    if (P->hp.prec == MBC_PREC_FP32 && P->hp.algo == MBC_ALGO_EGRAPH) {
        if (s.threads < 128 || s.threads > 768 || s.threads % 128 || s.blocks_per_sm < 1 || s.blocks_per_sm > 2 ||
            s.sites_per_unit < 1 || s.sites_per_unit > 3)
            return fail(P->ctx, MBC_INVALID_ARG, "MBC_PREC_FP32 schedule out of range (threads 128..768 in steps "
                                                 "of 128, blocks per site 1..2, leaf batch 1..3)");
        const mbc_schedule cur = P->sched;
        if (cur.threads == s.threads && cur.blocks_per_sm == s.blocks_per_sm && cur.sites_per_unit == s.sites_per_unit)
            return MBC_OK;
        if (P->hp.terms.empty() || !P->dev32) { P->sched = s; return MBC_OK; }
        const F32Shape old = P->f32_shape;
        P->f32_shape = F32Shape{s.threads / 128, s.sites_per_unit, s.blocks_per_sm};
        const mbc_status st = upload_f32(P);
        if (st != MBC_OK) { P->f32_shape = old; return st; }
        P->sched = f32_schedule(P->e32);
        P->ctx->batch_reserved.clear();
        return MBC_OK;
    }
    const int max_threads = P->hp.algo == MBC_ALGO_EGRAPH ? 384 : 256;
    if (s.threads < 32 || s.threads > max_threads || s.threads % 32 || s.blocks_per_sm < 1 || s.blocks_per_sm > 32 ||
        s.sites_per_unit < 1)
        return fail(P->ctx, MBC_INVALID_ARG, "schedule out of range (threads 32..256, or ..384 for the e-graph kernels, "
                                             "a multiple of 32)");
    P->sched = s;
    return MBC_OK;
}

mbc_status upload(mbc_plan* P) {
    HostPlan& h = P->hp;
    Blob b;
    // direct
    std::vector<int64_t> blk_start(1, 0), blk_nr, blk_ns;
    const int pr = h.prec;
    std::vector<Val16> blk_p = to_val(h.direct.blk_p, pr);
    for (size_t i = 0; i < h.direct.blk_s0.size(); ++i) {
        int64_t ns = h.direct.blk_s1[i] - h.direct.blk_s0[i], nr = h.direct.blk_r1[i] - h.direct.blk_r0[i];
        blk_start.push_back(blk_start.back() + ns * nr);
        blk_nr.push_back(nr);
        blk_ns.push_back(ns);
    }
    blk_start.push_back(INT64_MAX);   // sentinel: the block scan never runs past the end
    size_t o_bs = b.add(blk_start), o_s0 = b.add(h.direct.blk_s0), o_r0 = b.add(h.direct.blk_r0), o_nr = b.add(blk_nr), o_ns = b.add(blk_ns);
    size_t o_bp = b.add(blk_p);
    size_t o_si = b.add(h.snk_idx), o_sw = b.add(to_val(h.snk_w, pr)), o_ri = b.add(h.src_idx), o_rw = b.add(to_val(h.src_w, pr));
    size_t o_es = b.add(h.ex_snk), o_er = b.add(h.ex_src), o_ew = b.add(to_val(h.ex_w, pr));
    // tree
    std::vector<int8_t> mr[2], mc[2];
    int nf[2] = {h.n_u, h.n_d};
    for (int f = 0; f < 2; ++f)
        for (size_t m = 0; m < h.tree.minor_rows[f].size(); ++m) {
            int8_t r[12], c[12];
            mask_list(h.tree.minor_rows[f][m], r);
            mask_list(h.tree.minor_cols[f][m], c);
            for (int i = 0; i < nf[f]; ++i) { mr[f].push_back(r[i]); mc[f].push_back(c[i]); }
        }
    size_t o_mr0 = b.add(mr[0]), o_mc0 = b.add(mc[0]), o_mr1 = b.add(mr[1]), o_mc1 = b.add(mc[1]);
    size_t o_tf = b.add(h.tree.factors), o_tc = b.add(h.tree.children), o_tco = b.add(to_val(h.tree.coefficients, pr));
    size_t o_cn = b.add(h.tree.chunk_node), o_cl = b.add(h.tree.chunk_leaf), o_cc = b.add(h.tree.chunk_count);
    // e-graph
    EgraphPlan& e = h.eg;
    struct MinorOffs { size_t child[7], row[7], pack[7], lev, col, sign, leaf; } mo[2];
    const MinorPlan* mps[2] = {&e.A, &e.B};
    for (int w = 0; w < 2; ++w) {
        const MinorPlan& m = *mps[w];
        for (int k = 0; k < 7; ++k) {
            mo[w].child[k] = b.add(m.child[k]);
            mo[w].row[k] = b.add(m.row[k]);
            // transposed: word i of entry e at [i * n + e]
            std::vector<uint32_t> pk(m.child[k].size());
            const size_t n = k ? pk.size() / k : 0;
            for (size_t e = 0; e < n; ++e)
                for (int i = 0; i < k; ++i)
                    pk[i * n + e] = (uint32_t)m.child[k][e * k + i] | ((uint32_t)m.row[k][e * k + i] << 16);
            mo[w].pack[k] = b.add(pk);
        }
        std::vector<uint8_t> lev, col;
        std::vector<int8_t> sg;
        std::vector<int32_t> leaf;
        for (auto& nd : m.nodes) { lev.push_back(nd.level); col.push_back(nd.col); sg.push_back(nd.sign); leaf.push_back(nd.leaf); }
        mo[w].lev = b.add(lev); mo[w].col = b.add(col); mo[w].sign = b.add(sg); mo[w].leaf = b.add(leaf);
    }
    size_t o_goff = b.add(e.g_off), o_ga = b.add(e.g_a), o_gw = b.add(to_val(e.g_w, pr));
    size_t o_poff = b.add(e.pair_off), o_pb = b.add(e.pair_b), o_pf = b.add(e.pair_first), o_pc = b.add(to_val(e.pair_coef, pr));
    // compact form: real weights that a float holds exactly
    bool compact = true;
    for (auto& x : e.g_w) compact = compact && x.imag() == 0.0 && (double)(float)x.real() == x.real();
    for (auto& x : e.pair_coef) compact = compact && x.imag() == 0.0 && (double)(float)x.real() == x.real();
    std::vector<float> gwf, pcf;
    std::vector<double> gwd, pcd;
    if (compact) {
        for (auto& x : e.g_w) { gwf.push_back((float)x.real()); gwd.push_back(x.real()); }
        for (auto& x : e.pair_coef) { pcf.push_back((float)x.real()); pcd.push_back(x.real()); }
    }
    size_t o_gp = pr == 0 ? b.add(gwd) : b.add(gwf), o_pcf = pr == 0 ? b.add(pcd) : b.add(pcf);
    // sliced-ELL copy of the G entries (slices of 32 B row sets; weights exact in float)
    std::vector<int2> sell;
    std::vector<int32_t> sell_off, sell_w;
    {
        const int nrb = e.B.n ? (int)e.B.level_rows[e.B.n].size() : 1, nj = e.n_j;
        const int n_slices = (nrb + 31) / 32;
        if (compact && nj > 0 && (int)e.g_off.size() == nrb * nj + 1)
            for (int sl = 0; sl < n_slices; ++sl)
                for (int j = 0; j < nj; ++j) {
                    int width = 0;
                    for (int l = 0; l < 32 && sl * 32 + l < nrb; ++l) {
                        const int it = (sl * 32 + l) * nj + j;
                        width = std::max(width, e.g_off[it + 1] - e.g_off[it]);
                    }
                    sell_off.push_back((int32_t)sell.size());
                    sell_w.push_back(width);
                    const size_t base = sell.size();
                    sell.resize(base + (size_t)width * 32, int2{0, 0});
                    for (int l = 0; l < 32 && sl * 32 + l < nrb; ++l) {
                        const int it = (sl * 32 + l) * nj + j;
                        for (int k = 0; k < e.g_off[it + 1] - e.g_off[it]; ++k) {
                            const float wf = (float)e.g_w[e.g_off[it] + k].real();
                            int bits;
                            std::memcpy(&bits, &wf, 4);
                            sell[base + (size_t)k * 32 + l] = int2{e.g_a[e.g_off[it] + k], bits};
                        }
                    }
                }
    }
    size_t o_sell = b.add(sell), o_soff = b.add(sell_off), o_sellw = b.add(sell_w);
    std::vector<int4> prec_;
    if (compact && e.n_j >= 1 && e.n_j <= 2)
        for (size_t q = 0; q < e.pair_b.size(); ++q) {
            int4 r{e.pair_b[q] | (e.pair_first[q] ? (int)0x80000000u : 0), 0, 0, 0};
            const float c0 = (float)e.pair_coef[q * e.n_j].real();
            const float c1 = (float)e.pair_coef[q * e.n_j + e.n_j - 1].real();
            std::memcpy(&r.y, &c0, 4);
            std::memcpy(&r.z, &c1, 4);
            prec_.push_back(r);
        }
    size_t o_prec = b.add(prec_);
    std::vector<uint8_t> jmask(e.pair_off.empty() ? 0 : e.pair_off.size() - 1, 0);
    for (size_t l = 0; l + 1 < e.pair_off.size(); ++l)
        for (int32_t q = e.pair_off[l]; q < e.pair_off[l + 1]; ++q)
            for (int j = 0; j < e.n_j && j < 8; ++j)
                if (e.pair_coef[(size_t)q * e.n_j + j] != 0.0) jmask[l] |= (uint8_t)(1u << j);
    size_t o_jm = b.add(jmask);

    void* dev = nullptr;
    cudaError_t err = cudaMalloc(&dev, std::max<size_t>(b.host.size(), 256));
    if (err != cudaSuccess) return fail(P->ctx, MBC_OOM, std::string("cudaMalloc of plan arrays failed: ") + cudaGetErrorString(err));
    if (!b.host.empty()) {
        err = cudaMemcpy(dev, b.host.data(), b.host.size(), cudaMemcpyHostToDevice);
        if (err != cudaSuccess) { cudaFree(dev); return cuda_fail(P->ctx, err, "cudaMemcpy of plan arrays"); }
    }
    P->dev = dev;
    P->dev_bytes = b.host.size();

    DirectDev& dd = P->dd;
    dd.n_u = h.n_u; dd.n_d = h.n_d; dd.explicit_terms = h.explicit_terms;
    dd.n_blocks = (int)h.direct.blk_s0.size();
    dd.blk_start = at<int64_t>(dev, o_bs); dd.blk_s0 = at<int64_t>(dev, o_s0); dd.blk_r0 = at<int64_t>(dev, o_r0);
    dd.blk_nr = at<int64_t>(dev, o_nr); dd.blk_ns = at<int64_t>(dev, o_ns); dd.blk_p = at<Val16>(dev, o_bp);
    dd.snk_idx = at<int8_t>(dev, o_si); dd.snk_w = at<Val16>(dev, o_sw); dd.src_idx = at<int8_t>(dev, o_ri); dd.src_w = at<Val16>(dev, o_rw);
    dd.ex_snk = at<int8_t>(dev, o_es); dd.ex_src = at<int8_t>(dev, o_er); dd.ex_w = at<Val16>(dev, o_ew);
    dd.index_size = h.direct.index_size;

    TreeDev& td = P->td;
    td.n_u = h.n_u; td.n_d = h.n_d;
    td.n_minors[0] = (int64_t)h.tree.minor_rows[0].size(); td.n_minors[1] = (int64_t)h.tree.minor_rows[1].size();
    td.minor_rows[0] = at<int8_t>(dev, o_mr0); td.minor_cols[0] = at<int8_t>(dev, o_mc0);
    td.minor_rows[1] = at<int8_t>(dev, o_mr1); td.minor_cols[1] = at<int8_t>(dev, o_mc1);
    td.n_nodes = (int64_t)h.tree.factors.size();
    td.factors = at<int32_t>(dev, o_tf); td.children = at<int32_t>(dev, o_tc); td.coefficients = at<Val16>(dev, o_tco);
    td.n_chunks = (int)h.tree.chunk_node.size();
    td.chunk_node = at<int64_t>(dev, o_cn); td.chunk_leaf = at<int64_t>(dev, o_cl); td.chunk_count = at<int32_t>(dev, o_cc);

    EgraphDev& ed = P->ed;
    ed.flav_a = e.flav_a; ed.n_j = e.n_j;
    MinorDev* md[2] = {&ed.A, &ed.B};
    for (int w = 0; w < 2; ++w) {
        const MinorPlan& m = *mps[w];
        MinorDev& x = *md[w];
        x.n = m.n;
        minor_dev_offsets(m, m.n, x.size, x.off);
        for (int k = 0; k < 7; ++k) {
            x.child[k] = at<uint16_t>(dev, mo[w].child[k]);
            x.row[k] = at<uint8_t>(dev, mo[w].row[k]);
            x.pack[k] = at<uint32_t>(dev, mo[w].pack[k]);
        }
        x.n_nodes = (int)m.nodes.size();
        x.node_level = at<uint8_t>(dev, mo[w].lev); x.node_col = at<uint8_t>(dev, mo[w].col);
        x.node_sign = at<int8_t>(dev, mo[w].sign); x.node_leaf = at<int32_t>(dev, mo[w].leaf);
    }
    ed.compact = compact ? 1 : 0;
    ed.g_ws = at<unsigned char>(dev, o_gp);
    ed.pair_cs = at<unsigned char>(dev, o_pcf);
    ed.real_w = 1;
    for (auto& x : e.g_w) if (x.imag() != 0.0) ed.real_w = 0;
    for (auto& x : e.pair_coef) if (x.imag() != 0.0) ed.real_w = 0;
    ed.n_rows_b = e.B.n ? (int)e.B.level_rows[e.B.n].size() : 1;
    ed.n_cols_b = e.B.n ? (int)e.B.cols.size() : 1;
    ed.g_off = at<int32_t>(dev, o_goff); ed.g_a = at<int32_t>(dev, o_ga); ed.g_w = at<Val16>(dev, o_gw);
    ed.pair_off = at<int32_t>(dev, o_poff); ed.pair_b = at<int32_t>(dev, o_pb); ed.pair_first = at<uint8_t>(dev, o_pf);
    ed.pair_coef = at<Val16>(dev, o_pc);
    ed.sell = at<int2>(dev, o_sell); ed.sell_off = at<int32_t>(dev, o_soff); ed.sell_w = at<int32_t>(dev, o_sellw);
    ed.pair_rec = at<int4>(dev, o_prec);
    ed.leaf_jmask = at<uint8_t>(dev, o_jm);
    // levels 0..n-1 plus two buffers for the leaf level; G only for the general leaf path
    ed.stack_a = ed.A.off[ed.A.n] + 2 * ed.A.size[ed.A.n];
    ed.stack_b = ed.B.off[ed.B.n] + 2 * ed.B.size[ed.B.n];
    const bool fused = compact && ed.n_j <= 2;
    const int base = 2 * kBlk + ed.stack_a + ed.stack_b + (fused ? 0 : ed.n_j * ed.n_rows_b);
    // the packed tables of the two leaf levels (uint32 words, in 16-byte units) go to shared
    // memory too when that costs no resident block at 384 threads (the double-float kernel
    // is issue-bound and needs the warps), and always for FP64 (bound by the FP64 pipe,
    // it gains more from the shorter table reads than it loses in occupancy)
    const int pk16 = (ed.A.size[ed.A.n] * ed.A.n + ed.B.size[ed.B.n] * ed.B.n + 3) / 4;
    auto resident = [](int values) { return std::min(225 * 1024 / (values * 16 + 3 * 1024), 2048 / 384); };
    ed.stage_pk = (base + pk16) * 16 <= 200 * 1024 &&
                  (h.prec == MBC_PREC_FP64 || resident(base + pk16) >= resident(base));
    ed.smem_values = base + (ed.stage_pk ? pk16 : 0);
    return upload_f32(P);
}

std::string signature(const HostPlan& h) {
    // identifies the plan's kernel workload for the autotune cache
    char buf[256];
    snprintf(buf, sizeof buf, "%d/%d/%d/%d/%lld/%lld/%zu/%zu", h.n_u, h.n_d, h.algo, h.prec, (long long)h.direct.index_size,
             (long long)h.terms.size(), h.eg.A.nodes.size(), h.eg.pair_b.size());
    return buf;
}

mbc_status finish_plan(mbc_ctx* ctx, mbc_plan* P, mbc_plan** out) {
    HostPlan& h = P->hp;
    {
        const std::string bad = validate_plan(h);
        if (!bad.empty()) { delete P; return fail(ctx, MBC_INVALID_ARG, bad); }
    }
    if (h.algo == MBC_ALGO_EGRAPH) {
        if (h.explicit_terms) { delete P; return fail(ctx, MBC_UNSUPPORTED, "MBC_ALGO_EGRAPH needs a factored problem (mbc_plan_create)"); }
        if (h.eg.n_j > 64) { delete P; return fail(ctx, MBC_UNSUPPORTED, "e-graph kernels support at most 64 free indices in use"); }
    }
    if (h.algo == MBC_ALGO_TREE) {
        for (size_t i = 1; i < h.tree.factors.size();) {   // the walk expects level 1 -> leaves
            int32_t nch = h.tree.children[i];
            for (int32_t k = 1; k <= nch; ++k)
                if (h.tree.children[i + k] != 0) { delete P; return fail(ctx, MBC_UNSUPPORTED, "factor tree deeper than two levels"); }
            i += 1 + nch;
        }
    }
    if (ctx->device < 0) {                   // host-only context: keep the host plan only
        P->signature = signature(h);
        ctx->plans.push_back(P);
        *out = P;
        ctx->err.clear();
        return MBC_OK;
    }
    mbc_status st;
    try {
        st = upload(P);
    } catch (const std::bad_alloc&) {
        st = fail(ctx, MBC_OOM, "host allocation while uploading the plan");
    }
    if (st != MBC_OK) {
        if (P->dev) cudaFree(P->dev);
        delete P;
        return st;
    }
    if (h.algo == MBC_ALGO_EGRAPH && P->ed.smem_values * 16 > 200 * 1024) {
        cudaFree(P->dev);
        if (P->dev32) cudaFree(P->dev32);
        delete P;
        return fail(ctx, MBC_UNSUPPORTED, "e-graph plan needs more shared memory than a block has");
    }
    P->signature = signature(h);
    if (h.algo == MBC_ALGO_EGRAPH) {
        // 384 threads (12 warps) per block, or the B row-set count rounded up to whole warps
        // when that lies in 257..384 (one row set per thread in the leaf stage, no idle
        // warp), as many blocks per SM as shared memory and the 2048-thread limit allow
        const int rows_w = (P->ed.n_rows_b + 31) / 32 * 32;
        P->sched.threads = (rows_w > 256 && rows_w <= 384) ? rows_w : 384;
        const int by_smem = (int)(225 * 1024 / (P->ed.smem_values * 16 + 3 * 1024));
        P->sched.blocks_per_sm = std::max(1, std::min(by_smem, 2048 / P->sched.threads));
        P->sched_df = P->sched;
        if (h.prec == MBC_PREC_FP32) P->sched = f32_schedule(P->e32);
    }
    // a schedule tuned earlier for the same plan signature (kept only if it applies)
    auto it = ctx->tune_cache.find(P->signature);
    if (it != ctx->tune_cache.end() && apply_schedule(P, it->second) != MBC_OK) ctx->err.clear();
    ctx->plans.push_back(P);
    *out = P;
    ctx->err.clear();
    return MBC_OK;
}

int64_t direct_chunk(const mbc_plan* P) { return std::max<int64_t>(1, (int64_t)P->sched.sites_per_unit * 65536); }

mbc_status run(mbc_plan* P, const void* U, const void* D, int n_sets, int T, int64_t V3, void* C, void* site_out,
               cudaStream_t s, Momentum mom = Momentum()) {
    mbc_ctx* c = P->ctx;
    if (c->device < 0) return fail(c, MBC_UNSUPPORTED, "host-only context (device -1) cannot evaluate");
    HostPlan& h = P->hp;
    Geometry g{n_sets, T, V3};
    const int64_t n_sites = g.n_sites();
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    const cd scale = cd_make(h.scale.real(), h.scale.imag());
    // plans with an empty canonical term set have C = 0 identically (tree, e-graph)
    const bool empty = (h.algo != MBC_ALGO_DIRECT && h.terms.empty()) || (h.algo == MBC_ALGO_DIRECT && h.direct.index_size == 0);
    if (empty || n_sites == 0) {
        if (n_sets * T > 0) {
            e = cudaMemsetAsync(C, 0, sizeof(double2) * (size_t)n_sets * T, s);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
        }
        if (site_out && n_sites) {
            e = cudaMemsetAsync(site_out, 0, sizeof(double2) * (size_t)n_sites, s);
            if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
        }
        return MBC_OK;
    }
    int n_chunks = 1;
    int64_t chunk = 0;
    if (h.algo == MBC_ALGO_DIRECT) {
        chunk = direct_chunk(P);
        n_chunks = (int)((h.direct.index_size + chunk - 1) / chunk);
    } else if (h.algo == MBC_ALGO_TREE) {
        n_chunks = P->td.n_chunks;
    }
    mbc_status st = ensure(c, c->partials, sizeof(d4) * (size_t)n_sites * n_chunks, s);
    if (st == MBC_OK) st = ensure(c, c->site_tmp, sizeof(d4) * (size_t)n_sites, s);
    if (st == MBC_OK) st = ensure(c, c->counter, 256, s);
    if (st != MBC_OK) return st;
    Partials parts{(d4*)c->partials.p, n_chunks};
    const double* u = (const double*)U;
    const double* d = (const double*)D;
    if (h.algo == MBC_ALGO_DIRECT) {
        e = launch_direct(P->dd, h.prec, u, d, g, chunk, parts, P->sched.threads, s, &c->launches);
    } else if (h.algo == MBC_ALGO_TREE) {
        const int64_t per_site = (int64_t)(P->td.n_minors[0] + P->td.n_minors[1]) * 16;
        int64_t wave = std::max<int64_t>(32, (int64_t)(2048LL << 20) / std::max<int64_t>(per_site, 1)) / 32 * 32;
        wave = std::min<int64_t>(wave, (n_sites + 31) / 32 * 32);
        st = ensure(c, c->scratch, (size_t)per_site * wave, s);
        if (st == MBC_OK) st = ensure(c, c->exps, sizeof(int) * 2 * (size_t)wave, s);
        if (st != MBC_OK) return st;
        e = launch_tree(P->td, h.prec, u, d, g, c->scratch.p, wave, (int*)c->exps.p, parts, P->sched.threads, s, &c->launches);
    } else if (h.prec == MBC_PREC_FP32) {
        // FP32 pass (one block per SM, a B table per block), then the double-float
        // kernel over the sites whose error estimate exceeded the guard
        const int grid32 = c->sms;
        const int grid_df = (int)std::min<int64_t>(n_sites, (int64_t)c->sms * P->sched_df.blocks_per_sm);
        st = ensure(c, c->bslot, sizeof(float2) * (size_t)P->e32.n_cols_b * P->e32.n_rows_b * (grid32 / P->e32.cs), s);
        if (st == MBC_OK) st = ensure(c, c->flags, sizeof(unsigned int) * (size_t)n_sites, s);
        if (st == MBC_OK) st = ensure(c, c->gscale, sizeof(double) * (size_t)n_sites, s);
        if (st == MBC_OK) st = ensure(c, c->scratch, egraph_kslot_bytes(P->ed) * (size_t)grid_df, s);
        if (st != MBC_OK) return st;
        unsigned int* cnt = (unsigned int*)c->counter.p;
        e = cudaMemsetAsync(cnt + 1, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess)
            // the per-site guard protects per-site values and applies only when they are
            // returned; the slice guard protects C(t)
            e = launch_egraph32(P->e32, u, d, g, parts.part, grid32, c->bslot.p, cnt + 1, (unsigned int*)c->flags.p,
                                site_out ? P->e32.guard : INFINITY, P->slice_tol, (double*)c->gscale.p, mom, s,
                                &c->launches);
        if (e == cudaSuccess)
            e = launch_egraph_list(P->ed, u, d, parts, P->sched_df.threads, grid_df, cnt + 2, c->scratch.p,
                                   (const unsigned int*)c->flags.p, cnt + 1, n_sites, s, &c->launches);
    } else {
        const int grid = (int)std::min<int64_t>(n_sites, (int64_t)c->sms * P->sched.blocks_per_sm);
        st = ensure(c, c->scratch, egraph_kslot_bytes(P->ed) * (size_t)grid, s);
        if (st != MBC_OK) return st;
        e = launch_egraph(P->ed, h.prec, u, d, g, parts, P->sched.threads, grid, (unsigned int*)c->counter.p,
                          c->scratch.p, s, &c->launches);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    st = post_checks(c, "kernel");
    if (st != MBC_OK) return st;
    e = launch_reduce(parts, g, scale, (double2*)C, (double2*)site_out, (d4*)c->site_tmp.p, s, &c->launches, mom);
    if (e != cudaSuccess) return cuda_fail(c, e, "reduction launch");
    return MBC_OK;
}

bool bad_ptr(const void* p) { return p == nullptr; }

}  // namespace

namespace mbc {
// Read-only view of a plan for the allocation-free entry point (noalloc.cu).
bool noalloc_view(mbc_plan* P, NoallocView* v) {
    if (!P || !P->ctx) return false;
    v->device = P->ctx->device;
    v->algo = P->hp.algo;
    v->prec = P->hp.prec;
    // an MBC_PREC_FP32 plan is evaluated by the double-float kernel, with that kernel's
    // schedule (its own schedule is the FP32 kernel's shape)
    const mbc_schedule& sc = P->hp.prec == MBC_PREC_FP32 ? P->sched_df : P->sched;
    v->threads = sc.threads;
    v->blocks_per_sm = sc.blocks_per_sm;
    v->sms = P->ctx->sms;
    v->scale = cd_make(P->hp.scale.real(), P->hp.scale.imag());
    v->ed = P->ed;
    v->empty = P->hp.terms.empty();
    v->err = &P->ctx->err;
    v->launches = &P->ctx->launches;
    return true;
}
}  // namespace mbc

// ====================================================================== C ABI
extern "C" {

const char* mbc_version(void) { return "mbc 1.0"; }

mbc_status mbc_create(mbc_ctx** ctx, int device) {
    if (!ctx) return MBC_INVALID_ARG;
    *ctx = nullptr;
    if (device == -1) {                      // host-only: planning and plan files, no evaluation
        mbc_ctx* c = new (std::nothrow) mbc_ctx();
        if (!c) return MBC_OOM;
        c->device = -1;
        *ctx = c;
        return MBC_OK;
    }
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) return MBC_CUDA;
    if (device < 0 || device >= n) return MBC_INVALID_ARG;
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return MBC_CUDA;
    mbc_ctx* c = new (std::nothrow) mbc_ctx();
    if (!c) return MBC_OOM;
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    *ctx = c;
    return MBC_OK;
}

void mbc_destroy(mbc_ctx* c) {
    if (!c) return;
    if (c->device < 0) {
        for (mbc_plan* p : c->plans) delete p;
        destroy_block_plans(c);
        delete c;
        return;
    }
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (mbc_plan* p : c->plans) {
        if (p->dev) cudaFree(p->dev);
        if (p->dev32) cudaFree(p->dev32);
        delete p;
    }
    destroy_block_plans(c);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->h2d_start) cudaEventDestroy(c->h2d_start);
    for (cudaEvent_t ev : c->h2d_done) if (ev) cudaEventDestroy(ev);
    Buf* bufs[] = {&c->partials, &c->site_tmp, &c->scratch, &c->exps, &c->counter, &c->hU, &c->hD, &c->hC,
                   &c->batch_items, &c->batch_parts, &c->batch_k, &c->blk_part, &c->blk_F, &c->blk_tree,
                   &c->bslot, &c->flags, &c->gscale, &c->batch32_items, &c->batch32_scale};
    for (Buf* b : bufs) if (b->p) cudaFree(b->p);
    delete c;
}

const char* mbc_last_error(const mbc_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t mbc_launch_count(const mbc_ctx* c) { return c ? c->launches : 0; }

mbc_status mbc_operator_terms(int op, int* n_u, int* n_d, int* n_free, int64_t* n_terms, int8_t* idx, double* w,
                              int64_t* offsets, double* proj, double* scale) {
    if (!n_u || !n_d || !n_free || !n_terms) return MBC_INVALID_ARG;
    int nu, nd, nf;
    std::vector<int8_t> vi;
    std::vector<cplx> vw, vp;
    std::vector<int64_t> vo;
    double sc;
    std::string err = operator_terms(op, nu, nd, nf, vi, vw, vo, vp, sc);
    if (!err.empty()) return MBC_INVALID_ARG;
    *n_u = nu; *n_d = nd; *n_free = nf; *n_terms = (int64_t)vw.size();
    if (!idx) return MBC_OK;
    if (!w || !offsets || !proj) return MBC_INVALID_ARG;
    std::memcpy(idx, vi.data(), vi.size());
    for (size_t i = 0; i < vw.size(); ++i) { w[2 * i] = vw[i].real(); w[2 * i + 1] = vw[i].imag(); }
    std::memcpy(offsets, vo.data(), vo.size() * sizeof(int64_t));
    for (size_t i = 0; i < vp.size(); ++i) { proj[2 * i] = vp[i].real(); proj[2 * i + 1] = vp[i].imag(); }
    if (scale) *scale = sc;
    return MBC_OK;
}

mbc_status mbc_plan_create(mbc_ctx* ctx, const mbc_problem* pr, int algo, int prec, mbc_plan** out) {
    Range range_("mbc_plan_create");
    if (!ctx) return MBC_INVALID_ARG;
    if (!pr || !out) return fail(ctx, MBC_INVALID_ARG, "null problem or output pointer");
    if (algo < 0 || algo > 2 || prec < 0 || prec > 2) return fail(ctx, MBC_INVALID_ARG, "bad algorithm or precision");
    if (prec == MBC_PREC_FP32 && algo != MBC_ALGO_EGRAPH)
        return fail(ctx, MBC_UNSUPPORTED, "MBC_PREC_FP32 is available for MBC_ALGO_EGRAPH plans");
    if (pr->n_u < 0 || pr->n_d < 0 || pr->n_u > 6 || pr->n_d > 6 || pr->n_u + pr->n_d == 0)
        return fail(ctx, MBC_UNSUPPORTED, "n_u, n_d must be in 0..6 (not both 0)");
    if (pr->n_free < 1 || pr->n_free > 64) return fail(ctx, MBC_INVALID_ARG, "n_free must be in 1..64");
    if (bad_ptr(pr->snk_off) || bad_ptr(pr->src_off) || bad_ptr(pr->proj)) return fail(ctx, MBC_INVALID_ARG, "null offsets or projector");
    const int nf = pr->n_free, nq = pr->n_u + pr->n_d;
    if (pr->snk_off[0] != 0 || pr->src_off[0] != 0) return fail(ctx, MBC_INVALID_ARG, "offsets must start at 0");
    for (int j = 0; j < nf; ++j)
        if (pr->snk_off[j + 1] < pr->snk_off[j] || pr->src_off[j + 1] < pr->src_off[j])
            return fail(ctx, MBC_INVALID_ARG, "offsets must be non-decreasing");
    const int64_t ns = pr->snk_off[nf], nr = pr->src_off[nf];
    if ((ns && (bad_ptr(pr->snk_idx) || bad_ptr(pr->snk_w))) || (nr && (bad_ptr(pr->src_idx) || bad_ptr(pr->src_w))))
        return fail(ctx, MBC_INVALID_ARG, "null term arrays");
    mbc_plan* P = new (std::nothrow) mbc_plan();
    if (!P) return fail(ctx, MBC_OOM, "host allocation");
    P->ctx = ctx;
    HostPlan& h = P->hp;
    h.n_u = pr->n_u; h.n_d = pr->n_d; h.n_free = nf; h.algo = algo; h.prec = prec;
    h.scale = cplx(pr->scale[0], pr->scale[1]);
    try {
        h.snk_idx.assign(pr->snk_idx, pr->snk_idx + ns * nq);
        h.src_idx.assign(pr->src_idx, pr->src_idx + nr * nq);
        h.snk_w.resize(ns); h.src_w.resize(nr);
        for (int64_t i = 0; i < ns; ++i) h.snk_w[i] = cplx(pr->snk_w[2 * i], pr->snk_w[2 * i + 1]);
        for (int64_t i = 0; i < nr; ++i) h.src_w[i] = cplx(pr->src_w[2 * i], pr->src_w[2 * i + 1]);
        h.snk_off.assign(pr->snk_off, pr->snk_off + nf + 1);
        h.src_off.assign(pr->src_off, pr->src_off + nf + 1);
        h.proj.resize((size_t)nf * nf);
        for (size_t i = 0; i < h.proj.size(); ++i) h.proj[i] = cplx(pr->proj[2 * i], pr->proj[2 * i + 1]);
        for (auto& x : h.snk_w) if (!std::isfinite(x.real()) || !std::isfinite(x.imag())) { delete P; return fail(ctx, MBC_NUMERIC, "non-finite sink weight"); }
        for (auto& x : h.src_w) if (!std::isfinite(x.real()) || !std::isfinite(x.imag())) { delete P; return fail(ctx, MBC_NUMERIC, "non-finite source weight"); }
        std::string err = plan_factored(h);
        if (!err.empty()) { delete P; return fail(ctx, MBC_UNSUPPORTED, err); }
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(ctx, MBC_OOM, "host allocation during planning");
    }
    return finish_plan(ctx, P, out);
}

mbc_status mbc_plan_from_terms(mbc_ctx* ctx, int n_u, int n_d, int64_t n_terms, const int8_t* sink, const int8_t* source,
                               const double* W, const double* scale, int algo, int prec, mbc_plan** out) {
    Range range_("mbc_plan_from_terms");
    if (!ctx) return MBC_INVALID_ARG;
    if (!out || n_terms < 0 || (n_terms && (!sink || !source || !W))) return fail(ctx, MBC_INVALID_ARG, "bad term arrays");
    if (algo < 0 || algo > 2 || prec < 0 || prec > 2) return fail(ctx, MBC_INVALID_ARG, "bad algorithm or precision");
    if (prec == MBC_PREC_FP32) return fail(ctx, MBC_UNSUPPORTED, "MBC_PREC_FP32 is available for MBC_ALGO_EGRAPH plans");
    if (algo == MBC_ALGO_EGRAPH) return fail(ctx, MBC_UNSUPPORTED, "MBC_ALGO_EGRAPH needs a factored problem (mbc_plan_create)");
    if (n_u < 0 || n_d < 0 || n_u > 6 || n_d > 6 || n_u + n_d == 0) return fail(ctx, MBC_UNSUPPORTED, "n_u, n_d must be in 0..6");
    mbc_plan* P = new (std::nothrow) mbc_plan();
    if (!P) return fail(ctx, MBC_OOM, "host allocation");
    P->ctx = ctx;
    HostPlan& h = P->hp;
    h.n_u = n_u; h.n_d = n_d; h.n_free = 1; h.algo = algo; h.prec = prec;
    h.scale = scale ? cplx(scale[0], scale[1]) : cplx(1.0, 0.0);
    const int nq = n_u + n_d;
    try {
        h.ex_snk.assign(sink, sink + n_terms * nq);
        h.ex_src.assign(source, source + n_terms * nq);
        h.ex_w.resize(n_terms);
        for (int64_t i = 0; i < n_terms; ++i) h.ex_w[i] = cplx(W[2 * i], W[2 * i + 1]);
        std::string err = plan_explicit(h);
        if (!err.empty()) { delete P; return fail(ctx, MBC_UNSUPPORTED, err); }
    } catch (const std::bad_alloc&) {
        delete P;
        return fail(ctx, MBC_OOM, "host allocation during planning");
    }
    return finish_plan(ctx, P, out);
}

void mbc_plan_destroy(mbc_plan* P) {
    if (!P) return;
    mbc_ctx* c = P->ctx;
    if (c) {
        if (c->device >= 0) {
            cudaSetDevice(c->device);
            cudaDeviceSynchronize();
        }
        c->plans.erase(std::remove(c->plans.begin(), c->plans.end(), P), c->plans.end());
    }
    if (P->dev) cudaFree(P->dev);
    if (P->dev32) cudaFree(P->dev32);
    delete P;
}

mbc_status mbc_plan_get_info(const mbc_plan* P, mbc_plan_info* info) {
    if (!P || !info) return MBC_INVALID_ARG;
    const HostPlan& h = P->hp;
    std::memset(info, 0, sizeof *info);
    info->n_u = h.n_u; info->n_d = h.n_d; info->algo = h.algo; info->prec = h.prec;
    info->index_size = h.direct.index_size;
    info->canonical_terms = (int64_t)h.terms.size();
    info->rows_u = (int64_t)h.rows[0].size(); info->rows_d = (int64_t)h.rows[1].size();
    info->cols_u = (int64_t)h.cols[0].size(); info->cols_d = (int64_t)h.cols[1].size();
    info->minors_u = (int64_t)h.tree.minor_rows[0].size(); info->minors_d = (int64_t)h.tree.minor_rows[1].size();
    info->tree_nodes = (int64_t)h.tree.factors.size();
    info->egraph_classes = h.eg.A.classes + h.eg.B.classes;
    info->egraph_nodes = h.eg.A.enodes + h.eg.B.enodes;
    info->flops_per_site = h.algo == MBC_ALGO_DIRECT ? h.flops_direct : (h.algo == MBC_ALGO_TREE ? h.flops_tree : h.flops_egraph);
    info->direct_flops_per_site = h.flops_direct;
    info->scratch_bytes_per_site = h.algo == MBC_ALGO_TREE ? (int64_t)(h.tree.minor_rows[0].size() + h.tree.minor_rows[1].size()) * 16 : 32;
    return MBC_OK;
}

mbc_status mbc_plan_get_tree(const mbc_plan* P, int64_t* n_nodes, int64_t* n_leaves, int32_t* factors, int32_t* children,
                             double* coefficients) {
    if (!P || !n_nodes || !n_leaves) return MBC_INVALID_ARG;
    const TreePlan& t = P->hp.tree;
    *n_nodes = (int64_t)t.factors.size();
    *n_leaves = (int64_t)t.coefficients.size();
    if (factors) std::memcpy(factors, t.factors.data(), t.factors.size() * sizeof(int32_t));
    if (children) std::memcpy(children, t.children.data(), t.children.size() * sizeof(int32_t));
    if (coefficients)
        for (size_t i = 0; i < t.coefficients.size(); ++i) { coefficients[2 * i] = t.coefficients[i].real(); coefficients[2 * i + 1] = t.coefficients[i].imag(); }
    return MBC_OK;
}

mbc_status mbc_plan_get_minor(const mbc_plan* P, int flavour, int64_t m, int8_t* rows, int8_t* cols) {
    if (!P || flavour < 0 || flavour > 1 || !rows || !cols) return MBC_INVALID_ARG;
    const TreePlan& t = P->hp.tree;
    if (m < 0 || m >= (int64_t)t.minor_rows[flavour].size()) return MBC_INVALID_ARG;
    mask_list(t.minor_rows[flavour][m], rows);
    mask_list(t.minor_cols[flavour][m], cols);
    return MBC_OK;
}

mbc_status mbc_plan_save(const mbc_plan* P, const char* path) {
    if (!P || !path) return MBC_INVALID_ARG;
    std::string err = plan_write(P->hp, path);
    if (!err.empty()) return fail(P->ctx, MBC_IO, err);
    return MBC_OK;
}

mbc_status mbc_plan_load(mbc_ctx* ctx, const char* path, mbc_plan** out) {
    Range range_("mbc_plan_load");
    if (!ctx) return MBC_INVALID_ARG;
    if (!path || !out) return fail(ctx, MBC_INVALID_ARG, "null path or output");
    mbc_plan* P = new (std::nothrow) mbc_plan();
    if (!P) return fail(ctx, MBC_OOM, "host allocation");
    P->ctx = ctx;
    std::string err;
    try { err = plan_read(P->hp, path); } catch (const std::bad_alloc&) { err = "host allocation while reading"; }
    if (!err.empty()) { delete P; return fail(ctx, MBC_IO, err); }
    return finish_plan(ctx, P, out);
}

mbc_status mbc_correlator(mbc_plan* P, const void* U, const void* D, int n_sets, int T, int64_t V3, void* C, void* site_out,
                          mbc_stream stream) {
    Range range_("mbc_correlator");
    if (!P) return MBC_INVALID_ARG;
    mbc_ctx* c = P->ctx;
    if (n_sets < 0 || T < 0 || V3 < 0) return fail(c, MBC_INVALID_ARG, "negative size");
    if (!C && (int64_t)n_sets * T > 0) return fail(c, MBC_INVALID_ARG, "null output");
    if ((!U || !D) && (int64_t)n_sets * T * V3 > 0) return fail(c, MBC_INVALID_ARG, "null propagator field");
    if ((int64_t)n_sets * T * V3 > ((int64_t)1 << 32)) return fail(c, MBC_UNSUPPORTED, "more than 2^32 sites in one call");
    mbc_status st = run(P, U, D, n_sets, T, V3, C, site_out, (cudaStream_t)stream);
    if (st == MBC_OK) c->err.clear();
    return st;
}

mbc_status mbc_correlator_momentum(mbc_plan* P, const void* U, const void* D, int n_sets, int T, int L, const int* p,
                                   void* C, void* site_out, mbc_stream stream) {
    Range range_("mbc_correlator_momentum");
    if (!P) return MBC_INVALID_ARG;
    mbc_ctx* c = P->ctx;
    if (n_sets < 0 || T < 0 || L < 0) return fail(c, MBC_INVALID_ARG, "negative size");
    if (L > 1290) return fail(c, MBC_UNSUPPORTED, "L^3 sites per slice beyond the supported range");
    const int64_t V3 = (int64_t)L * L * L;
    if (!C && (int64_t)n_sets * T > 0) return fail(c, MBC_INVALID_ARG, "null output");
    if ((!U || !D) && (int64_t)n_sets * T * V3 > 0) return fail(c, MBC_INVALID_ARG, "null propagator field");
    if ((int64_t)n_sets * T * V3 > ((int64_t)1 << 32)) return fail(c, MBC_UNSUPPORTED, "more than 2^32 sites in one call");
    Momentum mom;
    mom.L = std::max(L, 1);
    if (p) { mom.px = p[0]; mom.py = p[1]; mom.pz = p[2]; }
    mbc_status st = run(P, U, D, n_sets, T, V3, C, site_out, (cudaStream_t)stream, mom);
    if (st == MBC_OK) c->err.clear();
    return st;
}

mbc_status mbc_correlator_host(mbc_plan* P, const void* U_host, const void* D_host, int n_sets, int T, int64_t V3,
                               void* C_host, mbc_stream stream) {
    Range range_("mbc_correlator_host");
    if (!P) return MBC_INVALID_ARG;
    mbc_ctx* c = P->ctx;
    if (n_sets < 0 || T < 0 || V3 < 0) return fail(c, MBC_INVALID_ARG, "negative size");
    const int64_t n_sites = (int64_t)n_sets * T * V3;
    if (!C_host || (n_sites && (!U_host || !D_host))) return fail(c, MBC_INVALID_ARG, "null host buffer");
    cudaStream_t s = (cudaStream_t)stream;
    if (c->device < 0) return fail(c, MBC_UNSUPPORTED, "host-only context (device -1) cannot evaluate");
    cudaSetDevice(c->device);
    const size_t fb = sizeof(double) * 288 * (size_t)n_sites, cb = sizeof(double2) * (size_t)n_sets * T;
    mbc_status st = ensure(c, c->hU, fb, s);
    if (st == MBC_OK) st = ensure(c, c->hD, fb, s);
    if (st == MBC_OK) st = ensure(c, c->hC, cb, s);
    if (st != MBC_OK) return st;
    cudaError_t e = cudaSuccess;
    // the time slices in up to kHostChunks chunks: the copy of chunk k + 1 (on the copy
    // stream) overlaps the evaluation of chunk k (on the caller's stream); a chunk is
    // evaluated as its own slices, so the results equal one evaluation of all of them
    const int64_t n_slices = (int64_t)n_sets * T;
    int chunks = (int)std::min<int64_t>(mbc_ctx::kHostChunks, n_slices);
    if (n_sites < (int64_t)c->sms * 64) chunks = 1;             // too small to gain from overlap
    if (fb && chunks > 1) {
        if (!c->copy_stream) {          // created once, all or nothing
            cudaStream_t cs = nullptr;
            cudaEvent_t ev[mbc_ctx::kHostChunks + 1] = {};
            e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            for (int k = 0; k <= mbc_ctx::kHostChunks && e == cudaSuccess; ++k)
                e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
            if (e != cudaSuccess) {
                for (cudaEvent_t x : ev) if (x) cudaEventDestroy(x);
                if (cs) cudaStreamDestroy(cs);
                return cuda_fail(c, e, "copy stream");
            }
            c->copy_stream = cs;
            c->h2d_start = ev[mbc_ctx::kHostChunks];
            for (int k = 0; k < mbc_ctx::kHostChunks; ++k) c->h2d_done[k] = ev[k];
        }
        // the copies wait for the caller's earlier work on s
        e = cudaEventRecord(c->h2d_start, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, c->h2d_start, 0);
        const size_t per_slice = sizeof(double) * 288 * (size_t)V3;
        for (int k = 0; k < chunks && e == cudaSuccess; ++k) {
            const int64_t a = n_slices * k / chunks, b = n_slices * (k + 1) / chunks;
            const size_t off = per_slice * (size_t)a, len = per_slice * (size_t)(b - a);
            e = cudaMemcpyAsync((char*)c->hU.p + off, (const char*)U_host + off, len, cudaMemcpyHostToDevice,
                                c->copy_stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync((char*)c->hD.p + off, (const char*)D_host + off, len, cudaMemcpyHostToDevice,
                                    c->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(c->h2d_done[k], c->copy_stream);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "host to device copy");
        for (int k = 0; k < chunks; ++k) {
            const int64_t a = n_slices * k / chunks, b = n_slices * (k + 1) / chunks;
            const size_t off = per_slice * (size_t)a;
            e = cudaStreamWaitEvent(s, c->h2d_done[k], 0);
            if (e != cudaSuccess) return cuda_fail(c, e, "stream wait");
            st = run(P, (const char*)c->hU.p + off, (const char*)c->hD.p + off, 1, (int)(b - a), V3,
                     (double2*)c->hC.p + a, nullptr, s);
            if (st != MBC_OK) {
                cudaStreamSynchronize(c->copy_stream);
                return st;
            }
        }
    } else {
        if (fb) {
            e = cudaMemcpyAsync(c->hU.p, U_host, fb, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c->hD.p, D_host, fb, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(c, e, "host to device copy");
        }
        st = run(P, c->hU.p, c->hD.p, n_sets, T, V3, c->hC.p, nullptr, s);
        if (st != MBC_OK) return st;
    }
    if (cb) {
        e = cudaMemcpyAsync(C_host, c->hC.p, cb, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "device to host copy");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
    c->err.clear();
    return MBC_OK;
}

namespace {
bool same_items(const std::vector<mbc_work>& a, const mbc_work* b, int n) {
    if ((int)a.size() != n) return false;
    for (int i = 0; i < n; ++i)
        if (std::memcmp(&a[i], &b[i], sizeof(mbc_work)) != 0) return false;
    return true;
}

// The FP32 item table holds each plan's guard settings as they were at mbc_batch_reserve;
// true when mbc_plan_set_guard changed one since.
bool guards_changed(const mbc_ctx* c, const mbc_work* items) {
    for (size_t k = 0; k < c->batch32_host.size(); ++k) {
        const mbc_work& w = items[c->batch32_src[k]];
        const float g = w.site_out ? w.plan->e32.guard : INFINITY;
        const BatchItem32& b = c->batch32_host[k];
        if (!(b.site_guard == g) || !(b.slice_tol == w.plan->slice_tol)) return true;
    }
    return false;
}

mbc_status check_items(mbc_ctx* c, const mbc_work* items, int n_items) {
    if (n_items < 0 || (n_items && !items)) return fail(c, MBC_INVALID_ARG, "bad items");
    if (c->device < 0) return fail(c, MBC_UNSUPPORTED, "host-only context (device -1) cannot evaluate");
    for (int i = 0; i < n_items; ++i) {
        const mbc_work& w = items[i];
        if (!w.plan || w.plan->ctx != c) return fail(c, MBC_INVALID_ARG, "item plan of another context");
        if (w.plan->hp.algo != MBC_ALGO_EGRAPH) return fail(c, MBC_UNSUPPORTED, "batched items must use MBC_ALGO_EGRAPH");
        if (w.n_sets < 0 || w.T < 0 || w.V3 < 0) return fail(c, MBC_INVALID_ARG, "negative item size");
        const int64_t ns = (int64_t)w.n_sets * w.T * w.V3;
        if ((ns && (!w.U || !w.D)) || ((int64_t)w.n_sets * w.T && !w.C)) return fail(c, MBC_INVALID_ARG, "null item buffer");
    }
    return MBC_OK;
}
}  // namespace

mbc_status mbc_batch_reserve(mbc_ctx* c, const mbc_work* items, int n_items) {
    Range range_("mbc_batch_reserve");
    if (!c) return MBC_INVALID_ARG;
    mbc_status st = check_items(c, items, n_items);
    if (st != MBC_OK) return st;
    cudaSetDevice(c->device);
    // partial sums of every item, one K slot size for all, item tables per precision
    int64_t total = 0, kslot = 1;
    size_t smem[2] = {0, 0};
    std::vector<int64_t> part_off(n_items);
    for (int i = 0; i < n_items; ++i) {
        part_off[i] = total;
        total += (int64_t)items[i].n_sets * items[i].T * items[i].V3;
        kslot = std::max<int64_t>(kslot, (int64_t)items[i].plan->ed.n_cols_b * items[i].plan->ed.n_rows_b);
        const int pr = items[i].plan->hp.prec == MBC_PREC_FP64 ? 0 : 1;
        smem[pr] = std::max(smem[pr], egraph_smem_bytes(items[i].plan->ed, pr));
    }
    int64_t tmp_sites = 0;               // items returning per-site values share site_tmp
    for (int i = 0; i < n_items; ++i)
        if (items[i].site_out) tmp_sites = std::max<int64_t>(tmp_sites, (int64_t)items[i].n_sets * items[i].T * items[i].V3);
    if (tmp_sites) {
        st = ensure(c, c->site_tmp, sizeof(d4) * (size_t)tmp_sites, nullptr);
        if (st != MBC_OK) return st;
    }
    const size_t max_smem = std::max(smem[0], smem[1]);
    const int by_smem = (int)(225 * 1024 / (max_smem + 3 * 1024));
    const int bps = std::max(1, std::min(by_smem, 2048 / 384));
    const int grid = std::max(1, c->sms * bps);
    st = ensure(c, c->batch_parts, sizeof(d4) * (size_t)std::max<int64_t>(total, 1), nullptr);
    if (st == MBC_OK) st = ensure(c, c->batch_k, (size_t)kslot * 16 * grid, nullptr);
    if (st == MBC_OK) st = ensure(c, c->counter, 256, nullptr);
    if (st == MBC_OK) st = ensure(c, c->batch_items, sizeof(BatchItem) * (size_t)std::max(n_items, 1) * 2, nullptr);
    if (st != MBC_OK) return st;
    for (int pr = 0; pr < 2; ++pr) {
        c->batch_host[pr].clear();
        int64_t units = 0;
        for (int i = 0; i < n_items; ++i) {
            const int ip = items[i].plan->hp.prec == MBC_PREC_FP64 ? 0 : 1;
            if (ip != pr || items[i].plan->hp.prec == MBC_PREC_FP32 || items[i].plan->hp.terms.empty()) continue;
            BatchItem b;
            b.d = items[i].plan->ed;
            b.U = (const double*)items[i].U;
            b.D = (const double*)items[i].D;
            b.part = (d4*)c->batch_parts.p + part_off[i];
            b.unit_begin = units;
            b.n_sites = (int64_t)items[i].n_sets * items[i].T * items[i].V3;
            units += b.n_sites;
            c->batch_host[pr].push_back(b);
        }
        c->batch_units[pr] = units;
        c->batch_smem[pr] = smem[pr];
        if (!c->batch_host[pr].empty()) {
            cudaError_t e = cudaMemcpy((BatchItem*)c->batch_items.p + (size_t)pr * std::max(n_items, 1),
                                       c->batch_host[pr].data(), sizeof(BatchItem) * c->batch_host[pr].size(),
                                       cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(c, e, "item table upload");
        }
    }
    // FP32 items: one cluster launch over their (item, site) units with their FP32 views,
    // and their double-float views (same unit numbering) for the recompute
    c->batch32_host.clear();
    c->batch32_src.clear();
    c->batch32_df_host.clear();
    c->batch32_units = 0;
    c->batch32_slices = 0;
    int64_t units32 = 0, slices32 = 0, bvals = 1;
    int cs32 = 0, w32 = 0, smem32 = 0, nj32 = 1;
    bool real32 = true;
    for (int i = 0; i < n_items; ++i) {
        const mbc_plan* P = items[i].plan;
        if (P->hp.prec != MBC_PREC_FP32 || P->hp.terms.empty()) continue;
        const Eg32Dev& d = P->e32;
        // items of smaller clusters leave blocks idle, items of fewer walkers leave warps idle
        w32 = std::max(w32, d.walkers);
        cs32 = std::max(cs32, d.cs);
        smem32 = std::max(smem32, d.smem_bytes);
        nj32 = std::max(nj32, d.n_j);
        real32 = real32 && d.real_w;
        bvals = std::max<int64_t>(bvals, (int64_t)d.n_cols_b * d.n_rows_b);
        const int64_t ns = (int64_t)items[i].n_sets * items[i].T * items[i].V3;
        BatchItem32 b;
        b.d = d;
        b.U = (const double*)items[i].U;
        b.D = (const double*)items[i].D;
        b.part = (d4*)c->batch_parts.p + part_off[i];
        b.scale = nullptr;                           // set below, once the buffer is sized
        b.g = Geometry{items[i].n_sets, items[i].T, items[i].V3};
        b.unit_begin = units32;
        b.slice_begin = slices32;
        // the per-site guard protects per-site values, when the item returns them
        b.site_guard = items[i].site_out ? (float)P->e32.guard : INFINITY;
        b.slice_tol = P->slice_tol;
        c->batch32_host.push_back(b);
        c->batch32_src.push_back(i);
        BatchItem bd;
        bd.d = P->ed;
        bd.U = b.U;
        bd.D = b.D;
        bd.part = b.part;
        bd.unit_begin = units32;
        bd.n_sites = ns;
        c->batch32_df_host.push_back(bd);
        units32 += ns;
        slices32 += (int64_t)items[i].n_sets * items[i].T;
    }
    if (!c->batch32_host.empty()) {
        const int clusters = c->sms / cs32;
        st = ensure(c, c->bslot, sizeof(float2) * (size_t)bvals * clusters, nullptr);
        if (st == MBC_OK) st = ensure(c, c->flags, sizeof(unsigned int) * (size_t)units32, nullptr);
        if (st == MBC_OK) st = ensure(c, c->batch32_scale, sizeof(double) * (size_t)units32, nullptr);
        if (st == MBC_OK) st = ensure(c, c->batch32_items, (sizeof(BatchItem32) + sizeof(BatchItem)) *
                                                               c->batch32_host.size(), nullptr);
        if (st != MBC_OK) return st;
        for (auto& b : c->batch32_host) b.scale = (double*)c->batch32_scale.p + b.unit_begin;
        const size_t n32 = c->batch32_host.size();
        cudaError_t e = cudaMemcpy(c->batch32_items.p, c->batch32_host.data(), sizeof(BatchItem32) * n32,
                                   cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy((unsigned char*)c->batch32_items.p + sizeof(BatchItem32) * n32, c->batch32_df_host.data(),
                           sizeof(BatchItem) * n32, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "FP32 item table upload");
        c->batch32_units = units32;
        c->batch32_slices = slices32;
        c->batch32_cs = cs32;
        c->batch32_walkers = w32;
        c->batch32_smem = smem32;
        c->batch32_nj = nj32;
        c->batch32_real = real32;
        c->batch32_bvals = bvals;
        size_t smem_df = 0;
        int threads_df = 32;
        for (int i = 0; i < n_items; ++i)
            if (items[i].plan->hp.prec == MBC_PREC_FP32 && !items[i].plan->hp.terms.empty()) {
                smem_df = std::max(smem_df, egraph_smem_bytes(items[i].plan->ed, 1));
                threads_df = std::max(threads_df, items[i].plan->sched_df.threads);
            }
        c->batch32_df_smem = smem_df;
        c->batch32_df_threads = std::min(threads_df, 384);
    }
    // block size: the largest e-graph schedule among the items (a multiple of 32, <= 384)
    int threads = 32;
    for (int i = 0; i < n_items; ++i)
        if (items[i].plan->hp.prec != MBC_PREC_FP32) threads = std::max(threads, items[i].plan->sched.threads);
    c->batch_threads = std::min(threads, 384);
    c->batch_kslot = kslot;
    c->batch_grid = grid;
    c->batch_reserved.assign(items, items + n_items);
    c->err.clear();
    return MBC_OK;
}

mbc_status mbc_batch(mbc_ctx* c, const mbc_work* items, int n_items, mbc_stream stream) {
    Range range_("mbc_batch");
    if (!c) return MBC_INVALID_ARG;
    mbc_status st = check_items(c, items, n_items);
    if (st != MBC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (!same_items(c->batch_reserved, items, n_items) || guards_changed(c, items)) {
        if (capturing(s))
            return fail(c, MBC_OOM, "mbc_batch inside a stream capture needs mbc_batch_reserve with the same items "
                                    "(and guard settings) first");
        st = mbc_batch_reserve(c, items, n_items);
        if (st != MBC_OK) return st;
    }
    cudaSetDevice(c->device);
    const int n_slots = std::max(n_items, 1);
    // one persistent launch per precision over every (item, site) unit
    for (int pr = 0; pr < 2; ++pr) {
        if (c->batch_host[pr].empty()) continue;
        cudaError_t e = launch_egraph_batch((const BatchItem*)c->batch_items.p + (size_t)pr * n_slots,
                                            (int)c->batch_host[pr].size(), c->batch_units[pr], pr, c->batch_threads,
                                            c->batch_grid,
                                            c->batch_smem[pr], (unsigned int*)c->counter.p, c->batch_k.p,
                                            c->batch_kslot, s, &c->launches);
        if (e != cudaSuccess) return cuda_fail(c, e, "batched kernel launch");
    }
    // FP32 items: the FP32 launch and its slice guard, then the double-float recompute of
    // the units the guard listed
    if (!c->batch32_host.empty()) {
        unsigned int* cnt = (unsigned int*)c->counter.p;
        const size_t n32 = c->batch32_host.size();
        const BatchItem32* t32 = (const BatchItem32*)c->batch32_items.p;
        const BatchItem* tdf = (const BatchItem*)((const unsigned char*)c->batch32_items.p + sizeof(BatchItem32) * n32);
        cudaError_t e = cudaMemsetAsync(cnt + 1, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess)
            e = launch_egraph32_batch(t32, (int)n32, c->batch32_units, c->batch32_slices, c->batch32_real,
                                      c->batch32_nj, c->batch32_cs, c->batch32_walkers, c->batch32_smem, c->sms,
                                      c->bslot.p, c->batch32_bvals, cnt + 1, (unsigned int*)c->flags.p, s,
                                      &c->launches);
        if (e == cudaSuccess)
            e = launch_egraph_batch_list(tdf, (int)n32, c->batch32_units, c->batch32_df_threads, c->batch_grid,
                                         c->batch32_df_smem,
                                         cnt + 2, c->batch_k.p, c->batch_kslot, (const unsigned int*)c->flags.p,
                                         cnt + 1, s, &c->launches);
        if (e != cudaSuccess) return cuda_fail(c, e, "batched FP32 launch");
        st = post_checks(c, "batched FP32 launch");
        if (st != MBC_OK) return st;
    }
    // site sums per item
    int64_t off = 0;
    for (int i = 0; i < n_items; ++i) {
        const mbc_work& w = items[i];
        Geometry g{w.n_sets, w.T, w.V3};
        const HostPlan& h = w.plan->hp;
        const cd scale = cd_make(h.scale.real(), h.scale.imag());
        if (h.terms.empty() || g.n_sites() == 0) {
            if ((int64_t)w.n_sets * w.T) {
                cudaError_t e = cudaMemsetAsync(w.C, 0, sizeof(double2) * (size_t)w.n_sets * w.T, s);
                if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemsetAsync");
            }
        } else {
            Partials pt{(d4*)c->batch_parts.p + off, 1};
            // (mbc_batch_reserve sized site_tmp for the items that return per-site values)
            cudaError_t e = launch_reduce(pt, g, scale, (double2*)w.C, (double2*)w.site_out,
                                          w.site_out ? (d4*)c->site_tmp.p : nullptr, s, &c->launches);
            if (e != cudaSuccess) return cuda_fail(c, e, "reduction launch");
        }
        off += g.n_sites();
    }
    c->err.clear();
    return MBC_OK;
}

mbc_status mbc_plan_set_guard(mbc_plan* P, double site_threshold, double slice_tolerance) {
    if (!P) return MBC_INVALID_ARG;
    if (std::isnan(site_threshold) || std::isnan(slice_tolerance))
        return fail(P->ctx, MBC_INVALID_ARG, "guard threshold or tolerance is NaN");
    P->guard = site_threshold;
    P->slice_tol = slice_tolerance;
    P->e32.guard = site_threshold > 3.0e38 ? INFINITY : (float)std::max(site_threshold, -1.0);
    return MBC_OK;
}

mbc_status mbc_plan_get_guard(const mbc_plan* P, double* site_threshold, double* slice_tolerance) {
    if (!P || !site_threshold || !slice_tolerance) return MBC_INVALID_ARG;
    *site_threshold = P->guard;
    *slice_tolerance = P->slice_tol;
    return MBC_OK;
}

mbc_status mbc_fp32_recomputed(mbc_ctx* c, int64_t* n_sites) {
    if (!c || !n_sites) return MBC_INVALID_ARG;
    *n_sites = 0;
    if (c->device < 0 || !c->counter.p) return MBC_OK;
    cudaSetDevice(c->device);
    unsigned int v = 0;
    cudaError_t e = cudaMemcpy(&v, (unsigned int*)c->counter.p + 1, sizeof v, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the recompute count");
    *n_sites = v;
    return MBC_OK;
}

mbc_status mbc_tensor_egraph(mbc_ctx* c, const char* expression, const char* antisymmetric, int64_t node_limit, int dim,
                             char* plan, int64_t plan_len, int64_t* plan_needed, int64_t* n_classes, int64_t* n_enodes) {
    Range range_("mbc_tensor_egraph");
    if (!c) return MBC_INVALID_ARG;
    if (!expression || !plan_needed || !n_classes || !n_enodes || dim < 1 || plan_len < 0)
        return fail(c, MBC_INVALID_ARG, "null argument, dim < 1 or negative buffer length");
    std::string text;
    mbc_status st = MBC_OK;
    try {
        int64_t nc = 0, nn = 0;
        std::string err = tensor_egraph(expression, antisymmetric ? antisymmetric : "", node_limit, dim, text, nc, nn);
        if (!err.empty()) return fail(c, MBC_INVALID_ARG, err);
        *n_classes = nc;
        *n_enodes = nn;
    } catch (const std::bad_alloc&) {
        return fail(c, MBC_OOM, "host allocation in the tensor e-graph");
    }
    *plan_needed = (int64_t)text.size() + 1;
    if (plan) {
        if (plan_len < (int64_t)text.size() + 1) return fail(c, MBC_INVALID_ARG, "plan buffer too small");
        std::memcpy(plan, text.c_str(), text.size() + 1);
    }
    c->err.clear();
    return st;
}

mbc_status mbc_set_schedule(mbc_plan* P, const mbc_schedule* s) {
    if (!P || !s) return MBC_INVALID_ARG;
    return apply_schedule(P, *s);
}

mbc_status mbc_get_schedule(const mbc_plan* P, mbc_schedule* s) {
    if (!P || !s) return MBC_INVALID_ARG;
    *s = P->sched;
    return MBC_OK;
}

mbc_status mbc_autotune(mbc_plan* P, const void* U, const void* D, int64_t n_sites, mbc_stream stream, mbc_schedule* best) {
    Range range_("mbc_autotune");
    if (!P) return MBC_INVALID_ARG;
    mbc_ctx* c = P->ctx;
    if (!U || !D || n_sites <= 0) return fail(c, MBC_INVALID_ARG, "autotune needs fields and a positive site count");
    if (c->device < 0) return fail(c, MBC_UNSUPPORTED, "host-only context (device -1) cannot evaluate");
    cudaStream_t s = (cudaStream_t)stream;
    const mbc_schedule orig = P->sched;
    const bool fp32 = P->hp.prec == MBC_PREC_FP32 && P->hp.algo == MBC_ALGO_EGRAPH;
    auto same = [](const mbc_schedule& a, const mbc_schedule& b) {
        return a.threads == b.threads && a.blocks_per_sm == b.blocks_per_sm && a.sites_per_unit == b.sites_per_unit;
    };
    // candidates: the plan's current (default) schedule first, then the grid of block
    // sizes x blocks per SM (x sites per unit for the direct sweep); for an FP32 plan the
    // grid of kernel shapes, walkers x blocks per site x leaf batch
    std::vector<mbc_schedule> cands{orig};
    if (fp32) {
        for (int w : {3, 4, 5, 6})
            for (int cs : {1, 2})
                for (int lb : {1, 2, 3}) {
                    const mbc_schedule cand{128 * w, cs, lb};
                    if (!same(cand, orig)) cands.push_back(cand);
                }
    } else {
        const int smem = P->ed.smem_values * 16 + 1024;
        for (int th : {128, 256, 320, 352, 384})
            for (int bps : {1, 2, 3, 4, 6, 8}) {
                if (th > 256 && P->hp.algo != MBC_ALGO_EGRAPH) continue;
                if (th * bps > 2048) continue;
                if (P->hp.algo == MBC_ALGO_EGRAPH && bps * smem > 220 * 1024) continue;
                if (P->hp.algo != MBC_ALGO_EGRAPH && bps != 2) continue;
                for (int spu : {1, 4}) {
                    if (P->hp.algo != MBC_ALGO_DIRECT && spu != 1) continue;
                    const mbc_schedule cand{th, bps, spu};
                    if (!same(cand, orig)) cands.push_back(cand);
                }
            }
    }
    Buf C;
    cudaError_t e = cudaMalloc(&C.p, sizeof(double2) * (size_t)n_sites);
    if (e != cudaSuccess) return fail(c, MBC_OOM, "autotune output");
    cudaEvent_t a = nullptr, b = nullptr;
    auto done = [&](mbc_status st) {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        cudaFree(C.p);
        return st;
    };
    // leave the plan with `keep` (its original schedule when tuning fails)
    auto restore = [&](const mbc_schedule& keep) {
        const std::string msg = c->err;
        apply_schedule(P, keep);          // (on failure the plan keeps a shape it ran with)
        c->err = msg;
    };
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        restore(orig);
        return done(fail(c, MBC_CUDA, "autotune events"));
    }
    float best_ms = -1.f;
    mbc_schedule keep = orig;
    for (auto& cand : cands) {
        // a candidate that does not apply (shape too large for shared memory) or cannot
        // run is skipped
        if (apply_schedule(P, cand) != MBC_OK) continue;
        mbc_status st = run(P, U, D, 1, 1, n_sites, C.p, nullptr, s);      // warm-up (and pool growth)
        if (st != MBC_OK) {
            if (st == MBC_CUDA) { restore(orig); return done(st); }   // the context may be unusable
            continue;
        }
        cudaEventRecord(a, s);
        for (int r = 0; r < 3 && st == MBC_OK; ++r) st = run(P, U, D, 1, 1, n_sites, C.p, nullptr, s);
        cudaEventRecord(b, s);
        e = cudaEventSynchronize(b);
        if (e != cudaSuccess) { restore(orig); return done(cuda_fail(c, e, "autotune timing")); }
        if (st != MBC_OK) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (best_ms < 0 || ms < best_ms) { best_ms = ms; keep = cand; }
    }
    c->err.clear();
    restore(keep);
    keep = P->sched;
    c->tune_cache[P->signature] = keep;
    if (best) *best = keep;
    return done(MBC_OK);
}

}  // extern "C"
