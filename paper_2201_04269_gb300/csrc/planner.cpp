// planner.cpp - host planner of libmbc.
//
// Steps (once per operator pair; the paper amortises this cost over configurations,
// arXiv 2201.04269 Sec. 4):
//   1. operator library: Grassmann expansion of the baryon operators of Sec. 1 and the
//      multi-baryon operators of Eq. 2 into flavour-grouped slot tuples;
//   2. canonical form (Sec. 3): ascending slot sets per flavour with the sorting sign,
//      repeated indices dropped (their determinant vanishes: the Index-List pruning of
//      Sec. 1), identical terms merged with their multiplicity;
//   3. linearised factor tree (Sec. 4, Fig. 5) over the canonical terms, level 1 = up
//      minor, level 2 = down minor, children in lexicographic order;
//   4. minor e-graph (Sec. 5): e-classes are minors det M[R, C]; the rewrite is the
//      Laplace split of the eps-contraction along one column, det M[R, C] =
//      sum_r (-1)^{p+q} M[r, c] det M[R\r, C\c]; extraction keeps, per class, the split
//      with the most excess parents from distinct classes weighted by flops.  Because
//      the needed classes always form a product (row sets) x (column sets), the row
//      factor of the objective is common to every split of a class, so the e-graph is
//      held over column sets (each class standing for all its row sets) and the choice
//      of column c depends on C only.  The extracted plan is a tree over column
//      subsets: every node's table of minors follows from its parent's table.
//   5. staged contraction for the e-graph kernels: G_j = s_j . A-minors per A column,
//      then coefficient-weighted dot products with B-minor columns.
#include "plan.hpp"
#include "blocks.hpp"

#include <algorithm>
#include <array>
#include <tuple>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <unordered_map>
#include <unordered_set>

namespace mbc {

// ------------------------------------------------------------------------ masks
int mask_size(Mask m) { return __builtin_popcount((unsigned)m); }
void mask_list(Mask m, int8_t* out) {
    int k = 0;
    for (int i = 0; i < 12; ++i)
        if (m & (1u << i)) out[k++] = (int8_t)i;
}
bool mask_lex_less(Mask a, Mask b) {
    int8_t x[12], y[12];
    int na = mask_size(a), nb = mask_size(b);
    mask_list(a, x);
    mask_list(b, y);
    for (int i = 0; i < na && i < nb; ++i)
        if (x[i] != y[i]) return x[i] < y[i];
    return na < nb;
}
static void sort_lex(std::vector<Mask>& v) { std::sort(v.begin(), v.end(), mask_lex_less); }

// sort k slot indices ascending; sign of the permutation, 0 if an index repeats
static int sort_slots(const int8_t* in, int k, Mask* mask) {
    int8_t t[12];
    std::memcpy(t, in, k);
    int sign = 1;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j + 1 < k - i; ++j)
            if (t[j] > t[j + 1]) { std::swap(t[j], t[j + 1]); sign = -sign; }
    Mask m = 0;
    for (int i = 0; i < k; ++i) {
        if (i && t[i] == t[i - 1]) return 0;
        m |= (Mask)(1u << t[i]);
    }
    *mask = m;
    return sign;
}

double flops_lu(int n) {
    if (n <= 1) return 0.0;
    return 8.0 * (n - 1) * n * (2 * n - 1) / 6.0 + 6.0 * (n * (n - 1) / 2.0 + n - 1) + 8.0 * (n - 1);
}

// ------------------------------------------------------------------------ operator library
namespace {
struct Field { int8_t f, c, s; };
struct OpTerm { cplx w; std::vector<Field> fields; };
typedef std::vector<OpTerm> Terms;
typedef std::vector<Terms> PerSpin;            // indexed by the free spin index
typedef std::array<std::array<cplx, 4>, 4> Mat4;

Mat4 mat_mul(const Mat4& a, const Mat4& b) {
    Mat4 r{};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
            r[i][j] = s;
        }
    return r;
}

struct Dirac {
    Mat4 g[4], g5, C, cg5, cg5p, cg5m;
    Dirac() {
        const cplx I(0, 1);
        // gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = diag(1, 1, -1, -1)
        cplx sig[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
        for (int k = 0; k < 3; ++k) {
            g[k] = Mat4{};
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    g[k][a][2 + b] = -I * sig[k][a][b];
                    g[k][2 + a][b] = I * sig[k][a][b];
                }
        }
        g[3] = Mat4{};
        g[3][0][0] = g[3][1][1] = 1.0;
        g[3][2][2] = g[3][3][3] = -1.0;
        g5 = mat_mul(mat_mul(g[0], g[1]), mat_mul(g[2], g[3]));
        C = mat_mul(g[3], g[1]);
        cg5 = mat_mul(C, g5);
        Mat4 pp{}, pm{};
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                cplx id = (a == b) ? 1.0 : 0.0;
                pp[a][b] = 0.5 * (id + g[3][a][b]);
                pm[a][b] = 0.5 * (id - g[3][a][b]);
            }
        cg5p = mat_mul(cg5, pp);
        cg5m = mat_mul(cg5, pm);
    }
};

// eps_abc (q1_a^T G q2_b) q3_c^alpha for each free spin alpha
PerSpin baryon(int8_t f1, int8_t f2, int8_t f3, const Mat4& G) {
    static const int perm[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
    static const int sgn[6] = {1, 1, 1, -1, -1, -1};
    PerSpin out(4);
    for (int al = 0; al < 4; ++al)
        for (int p = 0; p < 6; ++p)
            for (int be = 0; be < 4; ++be)
                for (int ga = 0; ga < 4; ++ga) {
                    if (G[be][ga] == 0.0) continue;
                    OpTerm t;
                    t.w = (double)sgn[p] * G[be][ga];
                    t.fields = {{f1, (int8_t)perm[p][0], (int8_t)be}, {f2, (int8_t)perm[p][1], (int8_t)ga},
                                {f3, (int8_t)perm[p][2], (int8_t)al}};
                    out[al].push_back(t);
                }
    return out;
}
// X^T G Y = sum_ab X^a G_ab Y^b
Terms tie_baryons(const PerSpin& x, const PerSpin& y, const Mat4& G, double s = 1.0) {
    Terms out;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            if (G[a][b] == 0.0) continue;
            for (auto& tx : x[a])
                for (auto& ty : y[b]) {
                    OpTerm t;
                    t.w = s * G[a][b] * tx.w * ty.w;
                    t.fields = tx.fields;
                    t.fields.insert(t.fields.end(), ty.fields.begin(), ty.fields.end());
                    out.push_back(std::move(t));
                }
        }
    return out;
}
PerSpin times(const Terms& t2, const PerSpin& z) {
    PerSpin out(4);
    for (int j = 0; j < 4; ++j)
        for (auto& a : t2)
            for (auto& b : z[j]) {
                OpTerm t;
                t.w = a.w * b.w;
                t.fields = a.fields;
                t.fields.insert(t.fields.end(), b.fields.begin(), b.fields.end());
                out[j].push_back(std::move(t));
            }
    return out;
}
}  // namespace

std::string operator_terms(int op, int& n_u, int& n_d, int& n_free, std::vector<int8_t>& idx,
                           std::vector<cplx>& w, std::vector<int64_t>& off, std::vector<cplx>& proj, double& scale) {
    static const Dirac dirac;
    const int8_t U = 0, D = 1;
    PerSpin per;
    double norm2 = 1.0;
    bool traced = true;
    switch (op) {
        case 0: per = baryon(U, D, U, dirac.cg5); n_u = 2; n_d = 1; break;
        case 1: per = baryon(D, U, D, dirac.cg5); n_u = 1; n_d = 2; break;
        case 2: case 3: {
            PerSpin n = baryon(D, U, D, dirac.cg5), p = baryon(U, D, U, dirac.cg5);
            Terms t = tie_baryons(n, p, dirac.cg5);
            if (op == 3) {
                Terms t2 = tie_baryons(p, n, dirac.cg5, -1.0);
                t.insert(t.end(), t2.begin(), t2.end());
                norm2 = 0.5;
            }
            per = PerSpin{t};
            n_u = 3; n_d = 3; traced = false;
            break;
        }
        case 4: case 5: case 6: {
            PerSpin pm = baryon(U, D, U, dirac.cg5m), pp = baryon(U, D, U, dirac.cg5p);
            PerSpin np = baryon(D, U, D, dirac.cg5p);
            std::vector<PerSpin> parts;
            parts.push_back(times(tie_baryons(pm, np, dirac.cg5), pp));              // + p_-^T Cg5 n_+ p_+^j
            if (op != 4) {
                parts.push_back(times(tie_baryons(pp, np, dirac.cg5, -1.0), pm));    // - p_+^T Cg5 n_+ p_-^j
                if (op == 5) {
                    parts.push_back(times(tie_baryons(np, pp, dirac.cg5), pm));      // + n_+^T Cg5 p_+ p_-^j
                    parts.push_back(times(tie_baryons(np, pm, dirac.cg5, -1.0), pp)); // - n_+^T Cg5 p_- p_+^j
                }
                parts.push_back(times(tie_baryons(pp, pm, dirac.cg5), np));          // + p_+^T Cg5 p_- n_+^j
                if (op == 5) parts.push_back(times(tie_baryons(pm, pp, dirac.cg5, -1.0), np));  // - p_-^T Cg5 p_+ n_+^j
                norm2 = (op == 5) ? 1.0 / 6.0 : 4.0 / 6.0;
            }
            per = PerSpin(4);
            for (auto& pt : parts)
                for (int j = 0; j < 4; ++j) per[j].insert(per[j].end(), pt[j].begin(), pt[j].end());
            n_u = 5; n_d = 4;
            break;
        }
        default: return "unknown operator id";
    }
    n_free = (int)per.size();
    const int nq = n_u + n_d;
    idx.clear(); w.clear(); off.assign(1, 0);
    for (int j = 0; j < n_free; ++j) {
        std::map<std::vector<int8_t>, cplx> merged;
        for (auto& t : per[j]) {
            // flavour-grouped slot order (stable), sign of the Grassmann reordering
            std::vector<int> order;
            for (int k = 0; k < (int)t.fields.size(); ++k) if (t.fields[k].f == U) order.push_back(k);
            for (int k = 0; k < (int)t.fields.size(); ++k) if (t.fields[k].f == D) order.push_back(k);
            int inv = 0;
            for (size_t a = 0; a < order.size(); ++a)
                for (size_t b = a + 1; b < order.size(); ++b) inv += order[a] > order[b];
            std::vector<int8_t> key;
            for (int k : order) key.push_back((int8_t)(3 * t.fields[k].s + t.fields[k].c));
            merged[key] += (inv & 1) ? -t.w : t.w;
        }
        for (auto& kv : merged) {
            if (kv.second == 0.0) continue;
            idx.insert(idx.end(), kv.first.begin(), kv.first.end());
            w.push_back(kv.second);
        }
        off.push_back((int64_t)w.size());
    }
    (void)nq;
    proj.assign((size_t)n_free * n_free, 0.0);
    if (traced) { proj[0] = 1.0; proj[n_free + 1] = 1.0; }   // P_+ traced: j = j' in {0, 1}
    else proj[0] = 1.0;
    int nq2 = n_u + n_d;
    double wick = ((nq2 * (nq2 - 1) / 2) % 2) ? -1.0 : 1.0;
    scale = wick * norm2;
    return "";
}

// ------------------------------------------------------------------------ baryon-level form
// The same operators as operator_terms, kept as products of baryons (for hadron blocks).
void block_gamma(int type, GammaNz& out) {
    static const Dirac dirac;
    const Mat4& G = (type <= 1) ? dirac.cg5 : (type == 2 || type == 4) ? dirac.cg5p : dirac.cg5m;
    out.n = 0;
    for (int be = 0; be < 4; ++be)
        for (int ga = 0; ga < 4; ++ga)
            if (G[be][ga] != 0.0) {
                out.be[out.n] = be;
                out.ga[out.n] = ga;
                out.g[out.n] = G[be][ga];
                ++out.n;
            }
}

std::string operator_products(int op, BaryonForm& out) {
    static const Dirac dirac;
    enum { P = 0, N = 1, PP = 2, PM = 3, NP = 4 };
    // X^T (C gamma_5) Y: tie of the first two baryons' spins
    std::vector<std::pair<std::array<int8_t, 4>, cplx>> tie2;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            if (dirac.cg5[a][b] != 0.0) tie2.push_back({{(int8_t)a, (int8_t)b, 0, 0}, dirac.cg5[a][b]});
    auto single = [&](int type) {
        BaryonProduct p;
        p.A = 1;
        p.types[0] = type;
        p.tie.resize(4);
        for (int j = 0; j < 4; ++j) p.tie[j].push_back({{(int8_t)j, 0, 0, 0}, 1.0});
        return p;
    };
    auto two = [&](double coef, int x, int y) {
        BaryonProduct p;
        p.coef = coef;
        p.A = 2;
        p.types[0] = x; p.types[1] = y;
        p.tie.assign(1, tie2);
        return p;
    };
    auto three = [&](double coef, int x, int y, int z) {     // X^T Cg5 Y Z^j
        BaryonProduct p;
        p.coef = coef;
        p.A = 3;
        p.types[0] = x; p.types[1] = y; p.types[2] = z;
        p.tie.resize(4);
        for (int j = 0; j < 4; ++j)
            for (auto& t : tie2) p.tie[j].push_back({{t.first[0], t.first[1], (int8_t)j, 0}, t.second});
        return p;
    };
    out.products.clear();
    out.norm = 1.0;
    switch (op) {
        case 0: out.products.push_back(single(P)); break;
        case 1: out.products.push_back(single(N)); break;
        case 2: out.products.push_back(two(1.0, N, P)); break;
        case 3:
            out.products.push_back(two(1.0, N, P));
            out.products.push_back(two(-1.0, P, N));
            out.norm = 1.0 / std::sqrt(2.0);
            break;
        case 4: out.products.push_back(three(1.0, PM, NP, PP)); break;              // + p_-^T Cg5 n_+ p_+^j
        case 5: case 6:
            out.products.push_back(three(1.0, PM, NP, PP));                         // + p_-^T Cg5 n_+ p_+^j
            out.products.push_back(three(-1.0, PP, NP, PM));                        // - p_+^T Cg5 n_+ p_-^j
            if (op == 5) {
                out.products.push_back(three(1.0, NP, PP, PM));                     // + n_+^T Cg5 p_+ p_-^j
                out.products.push_back(three(-1.0, NP, PM, PP));                    // - n_+^T Cg5 p_- p_+^j
            }
            out.products.push_back(three(1.0, PP, PM, NP));                         // + p_+^T Cg5 p_- n_+^j
            if (op == 5) out.products.push_back(three(-1.0, PM, PP, NP));           // - p_-^T Cg5 p_+ n_+^j
            out.norm = (op == 5) ? 1.0 / std::sqrt(6.0) : 2.0 / std::sqrt(6.0);
            break;
        default: return "unknown operator id";
    }
    return "";
}

// ------------------------------------------------------------------------ canonical form
namespace {
struct Acc { long double re = 0, im = 0; };

// canonicalise one side: per free index, {(mask_u, mask_d) -> merged weight}
std::vector<std::map<uint32_t, Acc>> canon_side(const HostPlan& p, const std::vector<int8_t>& idx,
                                               const std::vector<cplx>& w, const std::vector<int64_t>& off) {
    const int nq = p.n_u + p.n_d;
    std::vector<std::map<uint32_t, Acc>> out(p.n_free);
    for (int j = 0; j < p.n_free; ++j)
        for (int64_t t = off[j]; t < off[j + 1]; ++t) {
            Mask mu = 0, md = 0;
            int su = p.n_u ? sort_slots(&idx[t * nq], p.n_u, &mu) : 1;
            int sd = p.n_d ? sort_slots(&idx[t * nq + p.n_u], p.n_d, &md) : 1;
            if (!su || !sd) continue;                 // repeated index: the minor vanishes
            Acc& a = out[j][(uint32_t)mu | ((uint32_t)md << 12)];
            a.re += (long double)(su * sd) * w[t].real();
            a.im += (long double)(su * sd) * w[t].imag();
        }
    return out;
}

int64_t index_of(const std::vector<Mask>& v, Mask m) {
    auto it = std::lower_bound(v.begin(), v.end(), m, mask_lex_less);
    return (it != v.end() && *it == m) ? (int64_t)(it - v.begin()) : -1;
}
}  // namespace

static void build_tree(HostPlan& p) {
    // p.terms: (u minor id, d minor id, W), minor ids ordered lexicographically
    std::sort(p.terms.begin(), p.terms.end(), [](const CanonTerm& x, const CanonTerm& y) {
        return x.a != y.a ? x.a < y.a : x.b < y.b;
    });
    TreePlan& t = p.tree;
    const int32_t n_umin = (int32_t)t.minor_rows[0].size();
    t.factors.assign(1, -1);
    t.children.assign(1, 0);
    t.coefficients.clear();
    t.chunk_node.clear(); t.chunk_leaf.clear(); t.chunk_count.clear();
    int64_t nl1 = 0;
    const int64_t target = 2048;                 // leaves per chunk of the device walk
    int64_t chunk_leaves = target;
    for (size_t i = 0; i < p.terms.size();) {
        size_t j = i;
        while (j < p.terms.size() && p.terms[j].a == p.terms[i].a) ++j;
        if (chunk_leaves >= target) {
            t.chunk_node.push_back((int64_t)t.factors.size());
            t.chunk_leaf.push_back((int64_t)t.coefficients.size());
            t.chunk_count.push_back(0);
            chunk_leaves = 0;
        }
        t.chunk_count.back() += 1;
        t.factors.push_back(p.terms[i].a);
        t.children.push_back((int32_t)(j - i));
        for (size_t k = i; k < j; ++k) {
            t.factors.push_back(n_umin + p.terms[k].b);
            t.children.push_back(0);
            t.coefficients.push_back(p.terms[k].w);
        }
        chunk_leaves += (int64_t)(j - i);
        ++nl1;
        i = j;
    }
    t.children[0] = (int32_t)nl1;
    t.n_level1 = nl1;
}

// ------------------------------------------------------------------------ minor e-graph
static void build_minor_plan(MinorPlan& mp, int n, const std::vector<Mask>& rows, const std::vector<Mask>& cols) {
    mp = MinorPlan();
    mp.n = n;
    mp.cols = cols;
    if (n == 0) return;
    // row families F_k: closure of the needed rows under removing one row
    mp.level_rows[n] = rows;
    for (int k = n; k >= 2; --k) {
        std::unordered_set<Mask> s;
        for (Mask r : mp.level_rows[k])
            for (int i = 0; i < 12; ++i) if (r & (1u << i)) s.insert((Mask)(r & ~(1u << i)));
        mp.level_rows[k - 1].assign(s.begin(), s.end());
        sort_lex(mp.level_rows[k - 1]);
    }
    mp.level_rows[0] = {0};
    for (int k = 1; k <= n; ++k) {
        const auto& F = mp.level_rows[k];
        mp.child[k].resize(F.size() * k);
        mp.row[k].resize(F.size() * k);
        for (size_t e = 0; e < F.size(); ++e) {
            int8_t rl[12];
            mask_list(F[e], rl);
            for (int i = 0; i < k; ++i) {
                Mask c = (Mask)(F[e] & ~(1u << rl[i]));
                int64_t ci = (k == 1) ? 0 : index_of(mp.level_rows[k - 1], c);
                mp.child[k][e * k + i] = (uint16_t)ci;
                mp.row[k][e * k + i] = (uint8_t)rl[i];
            }
        }
    }
    // saturated e-graph size: classes (R, C) for R in F_k and C in every k-subset reachable
    // from the needed column sets by removing columns; k e-nodes (column splits) per class
    std::vector<Mask> all = cols;
    for (int k = n; k >= 1; --k) {
        mp.classes += (int64_t)mp.level_rows[k].size() * (int64_t)all.size();
        mp.enodes += (k >= 2 ? k : 1) * (int64_t)mp.level_rows[k].size() * (int64_t)all.size();
        std::unordered_set<Mask> s;
        for (Mask c : all)
            for (int i = 0; i < 12; ++i) if (c & (1u << i)) s.insert((Mask)(c & ~(1u << i)));
        all.assign(s.begin(), s.end());
    }
    // extraction, top-down: each needed column set keeps the split whose child column set
    // has the most distinct parents among the needed sets of its level (ties: the largest
    // column, which gives the lexicographic prefix trie)
    std::vector<std::vector<Mask>> P(n + 1);
    std::vector<std::unordered_map<Mask, Mask>> parent_of(n + 1);   // level-k set -> chosen child
    P[n] = cols;
    for (int k = n; k >= 1; --k) {
        std::unordered_map<Mask, int> cnt;
        for (Mask c : P[k])
            for (int i = 0; i < 12; ++i) if (c & (1u << i)) cnt[(Mask)(c & ~(1u << i))] += 1;
        std::unordered_set<Mask> next;
        for (Mask c : P[k]) {
            int best_i = -1, best = -1;
            for (int i = 0; i < 12; ++i) {
                if (!(c & (1u << i))) continue;
                int v = cnt[(Mask)(c & ~(1u << i))];
                if (v >= best) { best = v; best_i = i; }       // ">=": the largest column wins ties
            }
            Mask ch = (Mask)(c & ~(1u << best_i));
            parent_of[k][c] = ch;
            next.insert(ch);
        }
        P[k - 1].assign(next.begin(), next.end());
        sort_lex(P[k - 1]);
    }
    // column tree in depth-first order
    std::vector<std::unordered_map<Mask, std::vector<Mask>>> kids(n + 1);
    for (int k = 1; k <= n; ++k)
        for (Mask c : P[k]) kids[k - 1][parent_of[k][c]].push_back(c);
    for (int k = 0; k < n; ++k)
        for (auto& kv : kids[k]) sort_lex(kv.second);
    std::function<void(Mask, int, int32_t)> visit = [&](Mask c, int k, int32_t parent) {
        auto it = kids[k].find(c);
        if (it == kids[k].end()) return;
        for (Mask ch : it->second) {
            Mask added = (Mask)(ch & ~c);
            int col = __builtin_ctz((unsigned)added);
            int q = __builtin_popcount((unsigned)(ch & (added - 1)));   // position of col in ch
            MinorPlan::Node nd;
            nd.level = (uint8_t)(k + 1);
            nd.col = (uint8_t)col;
            nd.sign = (q & 1) ? -1 : 1;
            nd.leaf = (k + 1 == n) ? (int32_t)index_of(mp.cols, ch) : -1;
            nd.parent = parent;
            nd.cols = ch;
            int32_t me = (int32_t)mp.nodes.size();
            mp.nodes.push_back(nd);
            mp.dp_cfma += (double)mp.level_rows[k + 1].size() * (k + 1);
            visit(ch, k + 1, me);
        }
    };
    visit(0, 0, -1);
}

// ------------------------------------------------------------------------ e-graph contraction
static double egraph_cost(const HostPlan& p, int fa, const MinorPlan& A, const MinorPlan& B,
                          const std::vector<int>& used_j, const std::vector<int>& used_jp, double weight_factor = 1.0) {
    // complex multiply-adds per site of the staged evaluation:
    //   A column tree, G_j per A leaf, K(:, C_b) += sum_j coef_j G_j per pair,
    //   B column tree, <K(:, C_b), det B[:, C_b]> per B leaf
    double cf = A.dp_cfma + B.dp_cfma;
    int64_t nnz_s = 0;
    for (int j : used_j) nnz_s += (int64_t)p.snk_can[j].size();
    // real weights multiply a complex value with two real multiply-adds (factor 1/2)
    cf += weight_factor * (double)A.cols.size() * (double)nnz_s;
    std::unordered_set<uint64_t> s;
    for (int jp : used_jp)
        for (auto& t : p.src_can[jp]) {
            int64_t a = fa == 0 ? t.a : t.b, b = fa == 0 ? t.b : t.a;
            s.insert(((uint64_t)a << 32) | (uint64_t)b);
        }
    const double nb = (double)(B.n ? B.level_rows[B.n].size() : 1);
    const double ncb = (double)(B.n ? B.cols.size() : 1);
    cf += weight_factor * (double)s.size() * nb * (double)used_j.size();
    cf += ncb * nb;
    return cf;
}

static void build_egraph(HostPlan& p, const std::vector<int>& used_j, const std::vector<int>& used_jp) {
    EgraphPlan best;
    double best_cost = -1;
    const int n_j = (int)used_j.size();
    for (int fa = 0; fa < 2; ++fa) {
        int na = fa == 0 ? p.n_u : p.n_d, nb = fa == 0 ? p.n_d : p.n_u;
        if (na == 0) continue;
        EgraphPlan e;
        e.flav_a = fa;
        e.n_j = n_j;
        build_minor_plan(e.A, na, p.rows[fa], p.cols[fa]);
        // B row sets ordered by their number of G entries (most first), so that the
        // threads of a warp, which own consecutive row sets, do similar work
        std::vector<Mask> rows_b = p.rows[1 - fa];
        if (nb) {
            std::vector<int64_t> cnt(rows_b.size(), 0);
            for (int j : used_j)
                for (auto& t : p.snk_can[j]) cnt[fa == 0 ? t.b : t.a] += 1;
            std::vector<int32_t> order(rows_b.size());
            for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
            std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cnt[x] > cnt[y]; });
            for (size_t i = 0; i < order.size(); ++i) rows_b[i] = p.rows[1 - fa][order[i]];
        }
        build_minor_plan(e.B, nb, rows_b, p.cols[1 - fa]);
        double cost = egraph_cost(p, fa, e.A, e.B, used_j, used_jp);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = std::move(e); }
    }
    EgraphPlan& e = best;
    const int fa = e.flav_a;
    const int nB = e.B.n;
    // G entries grouped by (B row set, j): (A row set, w); B row sets are numbered by
    // their position in the B plan's leaf level (which the K rows and B tables follow)
    const size_t n_rb = nB ? p.rows[1 - fa].size() : 1;
    std::vector<int32_t> bpos(n_rb, 0);
    if (nB)
        for (size_t i = 0; i < n_rb; ++i) bpos[index_of(p.rows[1 - fa], e.B.level_rows[nB][i])] = (int32_t)i;
    std::vector<std::vector<std::pair<int32_t, cplx>>> byb(n_rb * (size_t)n_j);
    for (int jj = 0; jj < n_j; ++jj)
        for (auto& t : p.snk_can[used_j[jj]]) {
            int32_t a = fa == 0 ? t.a : t.b, b = fa == 0 ? t.b : t.a;
            byb[(size_t)(nB ? bpos[b] : 0) * n_j + jj].emplace_back(a, t.w);
        }
    e.g_off.assign(1, 0);
    for (auto& v : byb) {
        for (auto& x : v) { e.g_a.push_back(x.first); e.g_w.push_back(x.second); }
        e.g_off.push_back((int32_t)e.g_a.size());
    }
    // pairs per A column: coef_j = sum_j' P_jj' conj(r_j'(C_a, C_b))
    const size_t n_ca = p.cols[fa].size();
    std::vector<std::map<int32_t, std::vector<cplx>>> pairs(n_ca);
    for (int jp : used_jp)
        for (auto& t : p.src_can[jp]) {
            int32_t a = fa == 0 ? t.a : t.b, b = fa == 0 ? t.b : t.a;
            auto& coef = pairs[a][nB ? b : 0];
            coef.resize(n_j, 0.0);
            for (int jj = 0; jj < n_j; ++jj) coef[jj] += p.proj[(size_t)used_j[jj] * p.n_free + jp] * std::conj(t.w);
        }
    e.pair_off.assign(1, 0);
    std::vector<char> seen(nB ? p.cols[1 - fa].size() : 1, 0);
    // leaves are visited in column-tree order: first touches follow that order
    std::vector<int32_t> leaf_order;
    for (auto& nd : e.A.nodes) if (nd.leaf >= 0) leaf_order.push_back(nd.leaf);
    std::vector<int32_t> first_of_leaf(n_ca, 0);
    std::vector<std::vector<uint8_t>> first(n_ca);
    for (int32_t leaf : leaf_order) {
        for (auto& kv : pairs[leaf]) {
            first[leaf].push_back(seen[kv.first] ? 0 : 1);
            seen[kv.first] = 1;
        }
    }
    for (size_t ca = 0; ca < n_ca; ++ca) {
        size_t i = 0;
        for (auto& kv : pairs[ca]) {
            e.pair_b.push_back(kv.first);
            e.pair_first.push_back(first[ca].empty() ? 0 : first[ca][i]);
            for (int jj = 0; jj < n_j; ++jj) e.pair_coef.push_back(kv.second[jj]);
            ++i;
        }
        e.pair_off.push_back((int32_t)e.pair_b.size());
    }
    bool real = true;
    for (auto& x : e.g_w) real = real && x.imag() == 0.0;
    for (auto& x : e.pair_coef) real = real && x.imag() == 0.0;
    // algorithmic flops of the built plan: the Laplace tables of both trees, the G entries of
    // the free indices each A leaf's pairs use, one multiply-add per nonzero pair
    // coefficient and B row set, and the final dot products (real weights: half a complex
    // multiply-add each)
    {
        const double wf = real ? 0.5 : 1.0;
        const int64_t nrb = e.B.n ? (int64_t)e.B.level_rows[e.B.n].size() : 1;
        const int64_t ncb = e.B.n ? (int64_t)e.B.cols.size() : 1;
        std::vector<int64_t> nnz_j(n_j, 0);
        for (int64_t b = 0; b < nrb; ++b)
            for (int jj = 0; jj < n_j; ++jj) nnz_j[jj] += e.g_off[b * n_j + jj + 1] - e.g_off[b * n_j + jj];
        double cf = e.A.dp_cfma + e.B.dp_cfma + (double)ncb * (double)nrb;
        for (size_t l = 0; l + 1 < e.pair_off.size(); ++l) {
            uint32_t used = 0;
            for (int32_t q = e.pair_off[l]; q < e.pair_off[l + 1]; ++q)
                for (int jj = 0; jj < n_j; ++jj)
                    if (e.pair_coef[(size_t)q * n_j + jj] != 0.0) {
                        used |= 1u << (jj & 31);
                        cf += wf * (double)nrb;
                    }
            for (int jj = 0; jj < n_j; ++jj)
                if (n_j > 32 || ((used >> jj) & 1)) cf += wf * (double)nnz_j[jj];
        }
        e.flops_per_site = 8.0 * cf;
    }
    p.eg = std::move(e);
    p.flops_egraph = p.eg.flops_per_site;
}

// ------------------------------------------------------------------------ planning
static std::string validate_idx(const std::vector<int8_t>& v) {
    for (int8_t x : v) if (x < 0 || x > 11) return "slot index outside 0..11";
    return "";
}

std::string plan_factored(HostPlan& p) {
    if (p.n_u < 0 || p.n_u > 6 || p.n_d < 0 || p.n_d > 6 || p.n_u + p.n_d == 0) return "n_u, n_d must be in 0..6";
    if (p.n_free < 1) return "n_free must be >= 1";
    std::string err = validate_idx(p.snk_idx);
    if (err.empty()) err = validate_idx(p.src_idx);
    if (!err.empty()) return err;
    p.explicit_terms = false;
    // used free indices
    std::vector<int> used_j, used_jp;
    for (int j = 0; j < p.n_free; ++j) {
        bool a = false, b = false;
        for (int k = 0; k < p.n_free; ++k) {
            a = a || p.proj[(size_t)j * p.n_free + k] != 0.0;
            b = b || p.proj[(size_t)k * p.n_free + j] != 0.0;
        }
        if (a) used_j.push_back(j);
        if (b) used_jp.push_back(j);
    }
    // direct sweep blocks
    p.direct = DirectPlan();
    for (int j : used_j)
        for (int k : used_jp) {
            cplx pj = p.proj[(size_t)j * p.n_free + k];
            if (pj == 0.0) continue;
            int64_t ns = p.snk_off[j + 1] - p.snk_off[j], nr = p.src_off[k + 1] - p.src_off[k];
            if (!ns || !nr) continue;
            p.direct.blk_s0.push_back(p.snk_off[j]); p.direct.blk_s1.push_back(p.snk_off[j + 1]);
            p.direct.blk_r0.push_back(p.src_off[k]); p.direct.blk_r1.push_back(p.src_off[k + 1]);
            p.direct.blk_p.push_back(pj);
            p.direct.index_size += ns * nr;
        }
    // canonical sides
    auto cs = canon_side(p, p.snk_idx, p.snk_w, p.snk_off);
    auto cr = canon_side(p, p.src_idx, p.src_w, p.src_off);
    std::unordered_set<Mask> ru, rd, cu, cd;
    for (int j : used_j) for (auto& kv : cs[j]) if (kv.second.re != 0 || kv.second.im != 0) { ru.insert(kv.first & 0xFFF); rd.insert(kv.first >> 12); }
    for (int j : used_jp) for (auto& kv : cr[j]) if (kv.second.re != 0 || kv.second.im != 0) { cu.insert(kv.first & 0xFFF); cd.insert(kv.first >> 12); }
    p.rows[0].assign(ru.begin(), ru.end()); p.rows[1].assign(rd.begin(), rd.end());
    p.cols[0].assign(cu.begin(), cu.end()); p.cols[1].assign(cd.begin(), cd.end());
    for (int f = 0; f < 2; ++f) { sort_lex(p.rows[f]); sort_lex(p.cols[f]); }
    auto side_list = [&](std::vector<std::map<uint32_t, Acc>>& m, const std::vector<Mask>* sets) {
        std::vector<std::vector<CanonTerm>> out(p.n_free);
        for (int j = 0; j < p.n_free; ++j)
            for (auto& kv : m[j]) {
                if (kv.second.re == 0 && kv.second.im == 0) continue;
                int64_t a = index_of(sets[0], (Mask)(kv.first & 0xFFF)), b = index_of(sets[1], (Mask)(kv.first >> 12));
                if (a < 0 || b < 0) continue;            // belongs to an unused free index only
                out[j].push_back({(int32_t)a, (int32_t)b, cplx((double)kv.second.re, (double)kv.second.im)});
            }
        return out;
    };
    p.snk_can = side_list(cs, p.rows);
    p.src_can = side_list(cr, p.cols);
    // merged canonical terms: minor (R_u, C_u) x minor (R_d, C_d)
    const int64_t ncu = (int64_t)p.cols[0].size(), ncd = (int64_t)p.cols[1].size();
    std::vector<std::pair<uint64_t, cplx>> raw;
    for (int j : used_j)
        for (int k : used_jp) {
            cplx pj = p.proj[(size_t)j * p.n_free + k];
            if (pj == 0.0) continue;
            for (auto& s : p.snk_can[j])
                for (auto& r : p.src_can[k]) {
                    uint64_t mu = (uint64_t)s.a * ncu + r.a, md = (uint64_t)s.b * ncd + r.b;
                    raw.emplace_back((mu << 32) | md, pj * s.w * std::conj(r.w));
                }
        }
    std::sort(raw.begin(), raw.end(), [](const std::pair<uint64_t, cplx>& x, const std::pair<uint64_t, cplx>& y) { return x.first < y.first; });
    std::vector<std::pair<uint64_t, cplx>> merged;
    for (size_t i = 0; i < raw.size();) {
        size_t j = i;
        long double re = 0, im = 0;
        while (j < raw.size() && raw[j].first == raw[i].first) { re += raw[j].second.real(); im += raw[j].second.imag(); ++j; }
        if (re != 0 || im != 0) merged.emplace_back(raw[i].first, cplx((double)re, (double)im));
        i = j;
    }
    raw.clear(); raw.shrink_to_fit();
    // compact minor ids (order of (row idx, col idx) = lexicographic minor order)
    std::vector<uint64_t> umin, dmin;
    for (auto& m : merged) { umin.push_back(m.first >> 32); dmin.push_back(m.first & 0xFFFFFFFFu); }
    std::sort(umin.begin(), umin.end()); umin.erase(std::unique(umin.begin(), umin.end()), umin.end());
    std::sort(dmin.begin(), dmin.end()); dmin.erase(std::unique(dmin.begin(), dmin.end()), dmin.end());
    TreePlan& t = p.tree;
    t = TreePlan();
    for (uint64_t m : umin) { t.minor_rows[0].push_back(p.rows[0][m / ncu]); t.minor_cols[0].push_back(p.cols[0][m % ncu]); }
    for (uint64_t m : dmin) { t.minor_rows[1].push_back(p.rows[1][m / ncd]); t.minor_cols[1].push_back(p.cols[1][m % ncd]); }
    p.terms.clear();
    p.terms.reserve(merged.size());
    for (auto& m : merged) {
        int32_t a = (int32_t)(std::lower_bound(umin.begin(), umin.end(), m.first >> 32) - umin.begin());
        int32_t b = (int32_t)(std::lower_bound(dmin.begin(), dmin.end(), m.first & 0xFFFFFFFFu) - dmin.begin());
        p.terms.push_back({a, b, m.second});
    }
    build_tree(p);
    // flops per site
    p.flops_direct = (double)p.direct.index_size * (flops_lu(p.n_u) + flops_lu(p.n_d) + 14.0);
    p.flops_tree = (double)t.minor_rows[0].size() * flops_lu(p.n_u) + (double)t.minor_rows[1].size() * flops_lu(p.n_d) +
                   8.0 * (double)t.coefficients.size() + 8.0 * (double)t.n_level1;
    if (!p.rows[0].empty() || !p.rows[1].empty()) build_egraph(p, used_j, used_jp);
    else { p.eg = EgraphPlan(); p.flops_egraph = 0; }
    return "";
}

std::string plan_explicit(HostPlan& p) {
    if (p.n_u < 0 || p.n_u > 6 || p.n_d < 0 || p.n_d > 6 || p.n_u + p.n_d == 0) return "n_u, n_d must be in 0..6";
    std::string err = validate_idx(p.ex_snk);
    if (err.empty()) err = validate_idx(p.ex_src);
    if (!err.empty()) return err;
    p.explicit_terms = true;
    const int nq = p.n_u + p.n_d;
    const int64_t n = (int64_t)p.ex_w.size();
    p.direct = DirectPlan();
    p.direct.index_size = n;
    // canonicalise every term: (R_u, C_u, R_d, C_d) with the four sorting signs
    std::map<uint64_t, Acc> m;
    for (int64_t t = 0; t < n; ++t) {
        Mask a[4] = {0, 0, 0, 0};
        int s = 1;
        s *= p.n_u ? sort_slots(&p.ex_snk[t * nq], p.n_u, &a[0]) : 1;
        s *= p.n_u ? sort_slots(&p.ex_src[t * nq], p.n_u, &a[1]) : 1;
        s *= p.n_d ? sort_slots(&p.ex_snk[t * nq + p.n_u], p.n_d, &a[2]) : 1;
        s *= p.n_d ? sort_slots(&p.ex_src[t * nq + p.n_u], p.n_d, &a[3]) : 1;
        if (!s) continue;
        uint64_t key = (uint64_t)a[0] | ((uint64_t)a[1] << 12) | ((uint64_t)a[2] << 24) | ((uint64_t)a[3] << 36);
        Acc& x = m[key];
        x.re += (long double)s * p.ex_w[t].real();
        x.im += (long double)s * p.ex_w[t].imag();
    }
    std::unordered_set<Mask> sets[4];
    for (auto& kv : m)
        if (kv.second.re != 0 || kv.second.im != 0)
            for (int i = 0; i < 4; ++i) sets[i].insert((Mask)((kv.first >> (12 * i)) & 0xFFF));
    p.rows[0].assign(sets[0].begin(), sets[0].end()); p.cols[0].assign(sets[1].begin(), sets[1].end());
    p.rows[1].assign(sets[2].begin(), sets[2].end()); p.cols[1].assign(sets[3].begin(), sets[3].end());
    for (int f = 0; f < 2; ++f) { sort_lex(p.rows[f]); sort_lex(p.cols[f]); }
    const int64_t ncu = (int64_t)p.cols[0].size(), ncd = (int64_t)p.cols[1].size();
    std::vector<std::pair<uint64_t, cplx>> merged;
    for (auto& kv : m) {
        if (kv.second.re == 0 && kv.second.im == 0) continue;
        uint64_t mu = (uint64_t)index_of(p.rows[0], (Mask)(kv.first & 0xFFF)) * ncu + index_of(p.cols[0], (Mask)((kv.first >> 12) & 0xFFF));
        uint64_t md = (uint64_t)index_of(p.rows[1], (Mask)((kv.first >> 24) & 0xFFF)) * ncd + index_of(p.cols[1], (Mask)((kv.first >> 36) & 0xFFF));
        merged.emplace_back((mu << 32) | md, cplx((double)kv.second.re, (double)kv.second.im));
    }
    std::sort(merged.begin(), merged.end(), [](const std::pair<uint64_t, cplx>& x, const std::pair<uint64_t, cplx>& y) { return x.first < y.first; });
    std::vector<uint64_t> umin, dmin;
    for (auto& e : merged) { umin.push_back(e.first >> 32); dmin.push_back(e.first & 0xFFFFFFFFu); }
    std::sort(umin.begin(), umin.end()); umin.erase(std::unique(umin.begin(), umin.end()), umin.end());
    std::sort(dmin.begin(), dmin.end()); dmin.erase(std::unique(dmin.begin(), dmin.end()), dmin.end());
    TreePlan& t = p.tree;
    t = TreePlan();
    for (uint64_t x : umin) { t.minor_rows[0].push_back(p.rows[0][x / ncu]); t.minor_cols[0].push_back(p.cols[0][x % ncu]); }
    for (uint64_t x : dmin) { t.minor_rows[1].push_back(p.rows[1][x / ncd]); t.minor_cols[1].push_back(p.cols[1][x % ncd]); }
    p.terms.clear();
    for (auto& e : merged) {
        int32_t a = (int32_t)(std::lower_bound(umin.begin(), umin.end(), e.first >> 32) - umin.begin());
        int32_t b = (int32_t)(std::lower_bound(dmin.begin(), dmin.end(), e.first & 0xFFFFFFFFu) - dmin.begin());
        p.terms.push_back({a, b, e.second});
    }
    build_tree(p);
    p.flops_direct = (double)n * (flops_lu(p.n_u) + flops_lu(p.n_d) + 6.0);
    p.flops_tree = (double)t.minor_rows[0].size() * flops_lu(p.n_u) + (double)t.minor_rows[1].size() * flops_lu(p.n_d) +
                   8.0 * (double)t.coefficients.size() + 8.0 * (double)t.n_level1;
    p.eg = EgraphPlan();
    p.flops_egraph = 0;
    return "";
}

// ------------------------------------------------------------------------ validation
// Structural checks of everything the kernels index with: every table index, offset and
// count a device array holds lies inside the array it refers to.  Run before a plan is
// uploaded and after a plan file is read, so that a damaged or hand-made plan is rejected
// on the host instead of reaching a kernel.
namespace {
bool monotone(const std::vector<int32_t>& v, int64_t last) {
    if (v.empty() || v[0] != 0) return false;
    for (size_t i = 1; i < v.size(); ++i) if (v[i] < v[i - 1]) return false;
    return v.back() == last;
}
std::string check_minor_plan(const MinorPlan& m, const char* which) {
    const std::string w(which);
    if (m.n < 0 || m.n > 6) return w + ": minor size outside 0..6";
    if (m.n == 0) return "";
    for (int k = 1; k <= m.n; ++k) {
        const size_t n = m.level_rows[k].size();
        if (n == 0 || n > 65535) return w + ": level table size out of range";
        if (m.child[k].size() != n * k || m.row[k].size() != n * k) return w + ": level table arrays inconsistent";
        const size_t parent = k == 1 ? 1 : m.level_rows[k - 1].size();
        for (size_t i = 0; i < n * k; ++i)
            if (m.child[k][i] >= parent || m.row[k][i] >= 12) return w + ": level table entry out of range";
    }
    for (auto& nd : m.nodes)
        if (nd.level < 1 || nd.level > m.n || nd.col >= 12 || (nd.sign != 1 && nd.sign != -1) || nd.leaf < -1 ||
            nd.leaf >= (int32_t)m.cols.size())
            return w + ": column-tree node out of range";
    return "";
}
}  // namespace

std::string validate_plan(const HostPlan& p) {
    if (p.n_u < 0 || p.n_u > 6 || p.n_d < 0 || p.n_d > 6 || p.n_u + p.n_d == 0) return "plan: n_u, n_d out of range";
    if (p.algo < 0 || p.algo > 2 || p.prec < 0 || p.prec > 2 || (p.prec == 2 && p.algo != 2)) return "plan: algorithm or precision out of range";
    const int nq = p.n_u + p.n_d;
    for (int8_t v : p.snk_idx) if (v < 0 || v > 11) return "plan: sink index outside 0..11";
    for (int8_t v : p.src_idx) if (v < 0 || v > 11) return "plan: source index outside 0..11";
    for (int8_t v : p.ex_snk) if (v < 0 || v > 11) return "plan: sink index outside 0..11";
    for (int8_t v : p.ex_src) if (v < 0 || v > 11) return "plan: source index outside 0..11";
    if (p.ex_snk.size() != p.ex_w.size() * nq || p.ex_src.size() != p.ex_w.size() * nq) return "plan: explicit terms inconsistent";
    if (!p.explicit_terms) {
        if ((int)p.snk_off.size() != p.n_free + 1 || (int)p.src_off.size() != p.n_free + 1) return "plan: offsets size";
        for (int j = 0; j < p.n_free; ++j)
            if (p.snk_off[j] > p.snk_off[j + 1] || p.src_off[j] > p.src_off[j + 1]) return "plan: offsets decrease";
        if (p.snk_off[0] != 0 || p.src_off[0] != 0 || (size_t)p.snk_off.back() * nq != p.snk_idx.size() ||
            (size_t)p.src_off.back() * nq != p.src_idx.size() || (size_t)p.snk_off.back() != p.snk_w.size() ||
            (size_t)p.src_off.back() != p.src_w.size())
            return "plan: term arrays inconsistent with offsets";
        if (p.proj.size() != (size_t)p.n_free * p.n_free) return "plan: projector size";
    }
    // direct sweep blocks: sink and source ranges inside the term lists
    const DirectPlan& d = p.direct;
    const size_t nb = d.blk_s0.size();
    if (d.blk_s1.size() != nb || d.blk_r0.size() != nb || d.blk_r1.size() != nb || d.blk_p.size() != nb)
        return "plan: direct blocks inconsistent";
    for (size_t i = 0; i < nb; ++i)
        if (d.blk_s0[i] < 0 || d.blk_s0[i] > d.blk_s1[i] || (size_t)d.blk_s1[i] > p.snk_w.size() || d.blk_r0[i] < 0 ||
            d.blk_r0[i] > d.blk_r1[i] || (size_t)d.blk_r1[i] > p.src_w.size())
            return "plan: direct block range out of range";
    // factor tree: two levels, factor ids inside the minor tables, chunks inside the arrays
    const TreePlan& t = p.tree;
    if (t.children.size() != t.factors.size()) return "plan: tree arrays inconsistent";
    const int64_t n_um = (int64_t)t.minor_rows[0].size(), n_dm = (int64_t)t.minor_rows[1].size();
    if (t.minor_cols[0].size() != (size_t)n_um || t.minor_cols[1].size() != (size_t)n_dm) return "plan: tree minors inconsistent";
    int64_t leaves = 0;
    for (size_t i = 1; i < t.factors.size(); ++i) {
        const int64_t f = t.factors[i];
        if (t.children[i] < 0 || f < 0 || f >= n_um + n_dm) return "plan: tree factor out of range";
        if (t.children[i] == 0) ++leaves;
    }
    if (leaves != (int64_t)t.coefficients.size()) return "plan: tree leaves and coefficients differ";
    if (t.chunk_leaf.size() != t.chunk_node.size() || t.chunk_count.size() != t.chunk_node.size())
        return "plan: tree chunks inconsistent";
    for (size_t c = 0; c < t.chunk_node.size(); ++c)
        if (t.chunk_node[c] < 1 || t.chunk_node[c] > (int64_t)t.factors.size() || t.chunk_leaf[c] < 0 ||
            t.chunk_leaf[c] > (int64_t)t.coefficients.size() || t.chunk_count[c] < 0)
            return "plan: tree chunk out of range";
    // e-graph plan
    const EgraphPlan& e = p.eg;
    if (p.algo == 2 && !p.terms.empty()) {
        std::string err = check_minor_plan(e.A, "e-graph A");
        if (err.empty()) err = check_minor_plan(e.B, "e-graph B");
        if (!err.empty()) return err;
        if (e.A.n == 0 || e.n_j < 1 || e.n_j > 64) return "plan: e-graph shape out of range";
        const int64_t nrb = e.B.n ? (int64_t)e.B.level_rows[e.B.n].size() : 1;
        const int64_t ncb = e.B.n ? (int64_t)e.B.cols.size() : 1;
        const int64_t nra = (int64_t)e.A.level_rows[e.A.n].size();
        if ((int64_t)e.g_off.size() != nrb * e.n_j + 1 || !monotone(e.g_off, (int64_t)e.g_a.size()) ||
            e.g_w.size() != e.g_a.size())
            return "plan: e-graph G entries inconsistent";
        for (int32_t a : e.g_a) if (a < 0 || a >= nra) return "plan: e-graph G entry out of range";
        if ((int64_t)e.pair_off.size() != (int64_t)e.A.cols.size() + 1 || !monotone(e.pair_off, (int64_t)e.pair_b.size()) ||
            e.pair_first.size() != e.pair_b.size() || e.pair_coef.size() != e.pair_b.size() * (size_t)e.n_j)
            return "plan: e-graph pairs inconsistent";
        for (int32_t b : e.pair_b) if (b < 0 || b >= ncb) return "plan: e-graph pair column out of range";
        for (uint8_t f : e.pair_first) if (f > 1) return "plan: e-graph first-update flag out of range";
    }
    return "";
}

// ------------------------------------------------------------------------ serialisation
namespace {
const char kMagic[8] = {'M', 'B', 'C', 'P', 'L', 'A', 'N', '2'};
struct W {
    FILE* f;
    bool ok = true;
    void raw(const void* p, size_t n) { if (ok && n && fwrite(p, 1, n, f) != n) ok = false; }
    template <class T> void pod(const T& v) { raw(&v, sizeof(T)); }
    template <class T> void vec(const std::vector<T>& v) { uint64_t n = v.size(); pod(n); raw(v.data(), n * sizeof(T)); }
};
struct R {
    FILE* f;
    bool ok = true;
    void raw(void* p, size_t n) { if (ok && n && fread(p, 1, n, f) != n) ok = false; }
    template <class T> void pod(T& v) { raw(&v, sizeof(T)); }
    template <class T> void vec(std::vector<T>& v) {
        uint64_t n = 0; pod(n);
        if (!ok || n > (uint64_t)1 << 34) { ok = false; return; }
        v.resize(n); raw(v.data(), n * sizeof(T));
    }
};
template <class S> void minor_io(S& s, MinorPlan& m) {
    s.pod(m.n);
    for (int k = 0; k < 7; ++k) { s.vec(m.level_rows[k]); s.vec(m.child[k]); s.vec(m.row[k]); }
    s.vec(m.nodes); s.vec(m.cols); s.pod(m.classes); s.pod(m.enodes); s.pod(m.dp_cfma);
}
template <class S> void plan_io(S& s, HostPlan& p) {
    s.pod(p.n_u); s.pod(p.n_d); s.pod(p.n_free); s.pod(p.algo); s.pod(p.prec); s.pod(p.scale); s.pod(p.explicit_terms);
    s.vec(p.snk_idx); s.vec(p.src_idx); s.vec(p.snk_w); s.vec(p.src_w); s.vec(p.snk_off); s.vec(p.src_off); s.vec(p.proj);
    s.vec(p.ex_snk); s.vec(p.ex_src); s.vec(p.ex_w);
    for (int f = 0; f < 2; ++f) { s.vec(p.rows[f]); s.vec(p.cols[f]); }
    uint64_t nj = p.snk_can.size(); s.pod(nj); p.snk_can.resize(nj); for (auto& v : p.snk_can) s.vec(v);
    nj = p.src_can.size(); s.pod(nj); p.src_can.resize(nj); for (auto& v : p.src_can) s.vec(v);
    s.vec(p.terms);
    TreePlan& t = p.tree;
    for (int f = 0; f < 2; ++f) { s.vec(t.minor_rows[f]); s.vec(t.minor_cols[f]); }
    s.vec(t.factors); s.vec(t.children); s.vec(t.coefficients); s.pod(t.n_level1);
    s.vec(t.chunk_node); s.vec(t.chunk_leaf); s.vec(t.chunk_count);
    EgraphPlan& e = p.eg;
    s.pod(e.flav_a); s.pod(e.n_j); minor_io(s, e.A); minor_io(s, e.B);
    s.vec(e.g_off); s.vec(e.g_a); s.vec(e.g_w);
    s.vec(e.pair_off); s.vec(e.pair_b); s.vec(e.pair_first); s.vec(e.pair_coef); s.pod(e.flops_per_site);
    DirectPlan& d = p.direct;
    s.vec(d.blk_s0); s.vec(d.blk_s1); s.vec(d.blk_r0); s.vec(d.blk_r1); s.vec(d.blk_p); s.pod(d.index_size);
    s.pod(p.flops_direct); s.pod(p.flops_tree); s.pod(p.flops_egraph);
}
}  // namespace

std::string plan_write(const HostPlan& p, const std::string& path) {
    FILE* f = fopen(path.c_str(), "wb");
    if (!f) return "cannot open " + path + " for writing";
    W w{f};
    w.raw(kMagic, 8);
    plan_io(w, const_cast<HostPlan&>(p));
    bool ok = w.ok;
    if (fclose(f) != 0) ok = false;
    return ok ? "" : "write error on " + path;
}

std::string plan_read(HostPlan& p, const std::string& path) {
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) return "cannot open " + path;
    R r{f};
    char magic[8] = {0};
    r.raw(magic, 8);
    if (!r.ok || std::memcmp(magic, kMagic, 8) != 0) { fclose(f); return "not an mbc plan file (or another version): " + path; }
    plan_io(r, p);
    bool ok = r.ok;
    fclose(f);
    if (!ok) return "truncated plan file: " + path;
    const std::string bad = validate_plan(p);
    return bad.empty() ? "" : "damaged plan file (" + bad + "): " + path;
}

}  // namespace mbc
