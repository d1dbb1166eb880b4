// blocks_planner.cpp - host planner of the block form of a correlator.
//
// arXiv 2201.04269 Sec. 3: a multi-baryon correlator in terms of hadron blocks is a sum
// over N_w ways of handing the source fields to the sink baryons, each term a product of
// A blocks with fixed source indices (the expanded form); factors are put in canonical
// (lexicographic) order and identical factor strings merged with their multiplicity.
// Sec. 4: the merged terms form a factor tree.
//
// Steps:
//   1. sink operator as baryon products with spin ties (operator_products), source
//      operator as the conjugated flavour-grouped slot weights (operator_terms), put in
//      canonical form: ascending slot sets per flavour with the sorting sign; repeated
//      indices dropped (their contraction vanishes);
//   2. assignments: every split of the source u slots and d slots over the baryons by
//      their flavour content, the slots of each baryon in the block's order
//      (q1, q2, q3) with ascending positions for the two q1 slots, sign = parity of the
//      source reordering times (-1)^{A(A-1)/2} (interleaving A odd sink groups with their
//      odd source groups);
//   3. expansion: for every (j, j') with P_jj' != 0, product, spin tuple of the tie,
//      assignment and canonical source set, the A block entries (type, s1, s2, s3,
//      alpha); ids sorted ascending inside the term; terms merged by sorting their
//      packed keys;
//   4. compact factor numbering and the factor tree's device walk (units = vertices of
//      level A-2 with their leaves).
#include <algorithm>
#include <cmath>
#include <functional>
#include <map>

#include "blocks.hpp"

#include <cstring>

namespace mbc {

namespace {

struct Assignment {
    int8_t pos[4][3];     // per baryon: source slot positions (u slots 0..n_u-1, d slots n_u..)
    int sign;
};

void assignments(const BaryonProduct& p, int n_u, int n_d, std::vector<Assignment>& out) {
    out.clear();
    Assignment cur{};
    std::vector<int> free_u, free_d;
    for (int i = 0; i < n_u; ++i) free_u.push_back(i);
    for (int i = 0; i < n_d; ++i) free_d.push_back(i);
    std::function<void(int, std::vector<int>&, std::vector<int>&)> rec = [&](int i, std::vector<int>& fu,
                                                                            std::vector<int>& fd) {
        if (i == p.A) {
            if (!fu.empty() || !fd.empty()) return;
            int seq[12], n = 0;
            for (int b = 0; b < p.A; ++b)
                for (int k = 0; k < 3; ++k) seq[n++] = cur.pos[b][k];
            int inv = 0;
            for (int x = 0; x < n; ++x)
                for (int y = x + 1; y < n; ++y) inv += seq[x] > seq[y];
            const int inter = (p.A * (p.A - 1) / 2) & 1;
            cur.sign = ((inv + inter) & 1) ? -1 : 1;
            out.push_back(cur);
            return;
        }
        // block order (q1, q2, q3): two slots of flavour q1, one of q2
        const int q1 = block_q1(p.types[i]);
        std::vector<int>& f1 = q1 == 0 ? fu : fd;
        std::vector<int>& f2 = q1 == 0 ? fd : fu;
        const int off1 = q1 == 0 ? 0 : n_u, off2 = q1 == 0 ? n_u : 0;
        for (size_t a = 0; a < f1.size(); ++a)
            for (size_t c = a + 1; c < f1.size(); ++c)
                for (size_t b = 0; b < f2.size(); ++b) {
                    cur.pos[i][0] = (int8_t)(off1 + f1[a]);
                    cur.pos[i][1] = (int8_t)(off2 + f2[b]);
                    cur.pos[i][2] = (int8_t)(off1 + f1[c]);
                    std::vector<int> r1, r2;
                    for (size_t k = 0; k < f1.size(); ++k) if (k != a && k != c) r1.push_back(f1[k]);
                    for (size_t k = 0; k < f2.size(); ++k) if (k != b) r2.push_back(f2[k]);
                    if (q1 == 0) rec(i + 1, r1, r2);
                    else rec(i + 1, r2, r1);
                }
    };
    rec(0, free_u, free_d);
}

// ascending order of k slot indices with the permutation sign; 0 if an index repeats
int sort_sign(int8_t* v, int k) {
    int s = 1;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j + 1 < k - i; ++j)
            if (v[j] > v[j + 1]) { std::swap(v[j], v[j + 1]); s = -s; }
    for (int i = 0; i + 1 < k; ++i)
        if (v[i] == v[i + 1]) return 0;
    return s;
}

struct KeyW {
    uint64_t key;
    double re, im;
};

}  // namespace

std::string plan_blocks(BlockHostPlan& bp) {
    BaryonForm bf;
    std::string err = operator_products(bp.op, bf);
    if (!err.empty()) return err;
    int n_u = 0, n_d = 0, n_free = 0;
    std::vector<int8_t> idx;
    std::vector<cplx> w, proj;
    std::vector<int64_t> off;
    double wick_scale = 1.0;
    err = operator_terms(bp.op, n_u, n_d, n_free, idx, w, off, proj, wick_scale);
    if (!err.empty()) return err;
    const int nq = n_u + n_d;
    bp.n_u = n_u;
    bp.n_d = n_d;
    bp.A = bf.products[0].A;
    bp.scale = bf.norm * bf.norm;

    // 1. canonical source sets per free index j'
    std::vector<std::vector<std::pair<std::vector<int8_t>, cplx>>> src(n_free);
    for (int j = 0; j < n_free; ++j) {
        std::map<std::vector<int8_t>, cplx> m;
        for (int64_t t = off[j]; t < off[j + 1]; ++t) {
            std::vector<int8_t> v(idx.begin() + t * nq, idx.begin() + (t + 1) * nq);
            const int su = sort_sign(v.data(), n_u), sd = sort_sign(v.data() + n_u, n_d);
            if (!su || !sd) continue;
            m[v] += (double)(su * sd) * w[t];
        }
        for (auto& kv : m)
            if (kv.second != 0.0) src[j].push_back({kv.first, std::conj(kv.second)});
    }

    // 2-3. assignments and expansion
    std::vector<std::vector<Assignment>> asg(bf.products.size());
    bp.n_w.clear();
    for (size_t q = 0; q < bf.products.size(); ++q) {
        assignments(bf.products[q], n_u, n_d, asg[q]);
        bp.n_w.push_back((int)asg[q].size());
    }
    std::vector<KeyW> terms;
    const int A = bp.A;
    for (int j = 0; j < n_free; ++j)
        for (int jp = 0; jp < n_free; ++jp) {
            const cplx pj = proj[(size_t)j * n_free + jp];
            if (pj == 0.0) continue;
            for (size_t q = 0; q < bf.products.size(); ++q) {
                const BaryonProduct& pr = bf.products[q];
                for (auto& tie : pr.tie[j])
                    for (auto& as : asg[q]) {
                        const cplx c0 = pj * pr.coef * tie.second * (double)as.sign;
                        for (auto& s : src[jp]) {
                            int32_t id[4];
                            for (int i = 0; i < A; ++i) {
                                const int s1 = s.first[as.pos[i][0]], s2 = s.first[as.pos[i][1]],
                                          s3 = s.first[as.pos[i][2]];
                                id[i] = pr.types[i] * kEta + ((s1 * 12 + s2) * 12 + s3) * 4 + tie.first[i];
                            }
                            std::sort(id, id + A);
                            uint64_t key = 0;
                            for (int i = 0; i < A; ++i) key = (key << 16) | (uint64_t)id[i];
                            const cplx v = c0 * s.second;
                            terms.push_back({key, v.real(), v.imag()});
                        }
                    }
            }
        }
    bp.expanded = (int64_t)terms.size();
    std::sort(terms.begin(), terms.end(), [](const KeyW& a, const KeyW& b) { return a.key < b.key; });
    bp.ids.clear();
    bp.w.clear();
    bp.multiplicity.clear();
    for (size_t i = 0; i < terms.size();) {
        size_t k = i;
        double re = 0, im = 0;
        for (; k < terms.size() && terms[k].key == terms[i].key; ++k) { re += terms[k].re; im += terms[k].im; }
        if (re != 0.0 || im != 0.0) {
            uint64_t key = terms[i].key;
            int32_t id[4];
            for (int a = A - 1; a >= 0; --a) { id[a] = (int32_t)(key & 0xffff); key >>= 16; }
            bp.ids.insert(bp.ids.end(), id, id + A);
            bp.w.push_back(cplx(re, im));
            bp.multiplicity.push_back((int32_t)(k - i));
        }
        i = k;
    }
    terms.clear();
    terms.shrink_to_fit();
    const int64_t K = (int64_t)bp.w.size();

    // 4. compact factors, types, tree walk
    bp.factor.assign(bp.ids.begin(), bp.ids.end());
    std::sort(bp.factor.begin(), bp.factor.end());
    bp.factor.erase(std::unique(bp.factor.begin(), bp.factor.end()), bp.factor.end());
    bp.types.clear();
    for (int32_t g : bp.factor)
        if (bp.types.empty() || bp.types.back() != g / kEta) bp.types.push_back(g / kEta);
    auto compact = [&](int32_t g) {
        return (uint16_t)(std::lower_bound(bp.factor.begin(), bp.factor.end(), g) - bp.factor.begin());
    };
    bp.leaf_f.resize(K);
    for (int64_t t = 0; t < K; ++t) bp.leaf_f[t] = compact(bp.ids[t * A + A - 1]);
    bp.unit_pre.clear();
    bp.unit_leaf.assign(1, 0);
    for (int a = 0; a < 4; ++a) bp.level_nodes[a] = 0;
    for (int64_t t = 0; t < K; ++t) {
        // first level at which term t differs from term t - 1
        int d = 0;
        if (t > 0)
            while (d < A && bp.ids[t * A + d] == bp.ids[(t - 1) * A + d]) ++d;
        for (int a = d; a < A; ++a) ++bp.level_nodes[a];
        if (A >= 2 && t > 0 && d < A - 1) bp.unit_leaf.push_back((int32_t)t);
        if (A >= 2 && (t == 0 || d < A - 1))
            for (int a = 0; a < A - 1; ++a) bp.unit_pre.push_back(compact(bp.ids[t * A + a]));
        if (A == 1 && t > 0 && t % 8 == 0) bp.unit_leaf.push_back((int32_t)t);
    }
    if (K > 0) bp.unit_leaf.push_back((int32_t)K);
    else bp.unit_leaf.assign(1, 0);

    // flops: diquarks (432 entries x 2 eps terms x nnz(G) complex multiply-adds per type)
    // and 6 complex multiply-adds per used entry, per sink site; tree: one per leaf plus
    // A-1 products per unit, per time slice
    double fl = 0;
    for (int t : bp.types) {
        GammaNz g;
        block_gamma(t, g);
        fl += 432.0 * 2 * g.n * 8;
    }
    bp.block_flops_per_site = fl + (double)bp.factor.size() * 6 * 8;
    const int64_t n_units = (int64_t)bp.unit_leaf.size() - 1;
    bp.tree_flops_per_slice = 8.0 * ((double)K + (double)n_units * (A - 1));
    // hash-consed leaf sums: a 64-bit hash per unit (FNV-1a over its leaves' factors and
    // weight bits), units sorted by hash, equal hashes compared leaf by leaf
    bp.shared_sums = bp.shared_sum_terms = 0;
    if (A >= 2 && n_units > 0) {
        auto leaf_eq = [&](int64_t x, int64_t y) {
            return bp.leaf_f[x] == bp.leaf_f[y] && bp.w[x] == bp.w[y];
        };
        std::vector<std::pair<uint64_t, int64_t>> hu((size_t)n_units);
        for (int64_t u = 0; u < n_units; ++u) {
            uint64_t h = 1469598103934665603ull;
            auto mix = [&](uint64_t v) {
                for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xFFu; h *= 1099511628211ull; }
            };
            for (int32_t l = bp.unit_leaf[u]; l < bp.unit_leaf[u + 1]; ++l) {
                uint64_t re, im;
                const double wr = bp.w[l].real(), wi = bp.w[l].imag();
                std::memcpy(&re, &wr, 8);
                std::memcpy(&im, &wi, 8);
                mix(bp.leaf_f[l]);
                mix(re);
                mix(im);
            }
            hu[(size_t)u] = {h, u};
        }
        std::sort(hu.begin(), hu.end());
        std::vector<int64_t> reps;                   // distinct units among one hash value
        for (size_t i = 0; i < hu.size(); ++i) {
            if (i == 0 || hu[i].first != hu[i - 1].first) reps.clear();
            const int64_t u = hu[i].second;
            const int32_t a0 = bp.unit_leaf[u], n = bp.unit_leaf[u + 1] - a0;
            bool found = false;
            for (int64_t r : reps) {
                const int32_t b0 = bp.unit_leaf[r];
                if (bp.unit_leaf[r + 1] - b0 != n) continue;
                bool same = true;
                for (int32_t k = 0; k < n && same; ++k) same = leaf_eq(a0 + k, b0 + k);
                if (same) { found = true; break; }
            }
            if (!found) {
                reps.push_back(u);
                ++bp.shared_sums;
                bp.shared_sum_terms += n;
            }
        }
    }
    return "";
}

}  // namespace mbc
