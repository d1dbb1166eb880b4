// plan.hpp - host-side plan of libmbc (internal).
//
// A plan holds the problem (factored or explicit weights), its canonical form
// (arXiv 2201.04269 Sec. 3), the linearised factor tree (Sec. 4) and the minor plan
// extracted from the determinant e-graph (Sec. 5), plus device copies of what the
// chosen algorithm reads.
#pragma once
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace mbc {

typedef std::complex<double> cplx;

// Ascending index set of one flavour, as a 12-bit mask.
typedef uint16_t Mask;
int mask_size(Mask m);
void mask_list(Mask m, int8_t* out);   // ascending indices
bool mask_lex_less(Mask a, Mask b);     // lexicographic order of the ascending tuples

struct CanonTerm { int32_t a, b; cplx w; };   // row/col-set index of flavour u, d; weight

// Minor plan of one flavour for the e-graph kernels: row families F_k (k = 1..n), the
// column tree chosen by extraction, and per-level transition tables.
struct MinorPlan {
    int n = 0;                                  // minor size of this flavour
    std::vector<Mask> level_rows[7];            // F_k, k = 1..n (level_rows[n] = needed rows)
    // per entry e of F_k (k >= 2): child index into F_{k-1} of F_k[e] minus its i-th row, and that row
    std::vector<uint16_t> child[7];             // [e * k + i]
    std::vector<uint8_t> row[7];                // [e * k + i]
    // column tree in depth-first order: node level (1..n), added column, sign (-1)^q of
    // that column's position q in the node's column set, and the index of the node's
    // column set among the needed columns (level n) or -1
    struct Node { uint8_t level; uint8_t col; int8_t sign; int32_t leaf; int32_t parent; Mask cols; };
    std::vector<Node> nodes;
    std::vector<Mask> cols;                     // needed column sets (level n), in plan order
    int64_t classes = 0, enodes = 0;            // saturated e-graph size
    double dp_cfma = 0;                         // complex FMAs of one full pass over the tree
};

struct EgraphPlan {
    int flav_a = 0;                             // flavour streamed first (0 = u)
    int n_j = 0;                                // sink free indices in use
    MinorPlan A, B;
    // G_j(b) = sum over entries (a, w) of w * A(a); entries grouped by (b, j)
    std::vector<int32_t> g_off;                 // [|rows_B| * n_j + 1]
    std::vector<int32_t> g_a;
    std::vector<cplx> g_w;
    // per A leaf (needed A column): pairs (B column, coef_j for each j); a pair is the
    // first update of its B column in traversal order when pair_first is 1
    std::vector<int32_t> pair_off;              // [|cols_A| + 1]
    std::vector<int32_t> pair_b;
    std::vector<uint8_t> pair_first;
    std::vector<cplx> pair_coef;                // [pair * n_j + j]
    double flops_per_site = 0;
};

struct TreePlan {
    std::vector<Mask> minor_rows[2], minor_cols[2];   // minors per flavour
    std::vector<int32_t> factors, children;           // linearised tree (Sec. 4)
    std::vector<cplx> coefficients;
    int64_t n_level1 = 0;
    // chunks of consecutive level-1 subtrees: first node, first leaf, number of subtrees
    std::vector<int64_t> chunk_node, chunk_leaf;
    std::vector<int32_t> chunk_count;
};

struct DirectPlan {
    // factored: blocks (sink range) x (source range) with coefficient P
    std::vector<int64_t> blk_s0, blk_s1, blk_r0, blk_r1;
    std::vector<cplx> blk_p;
    int64_t index_size = 0;
};

struct HostPlan {
    int n_u = 0, n_d = 0, n_free = 0;
    int algo = 0, prec = 0;
    cplx scale = 1.0;
    bool explicit_terms = false;
    // the problem as given (factored form)
    std::vector<int8_t> snk_idx, src_idx;
    std::vector<cplx> snk_w, src_w;
    std::vector<int64_t> snk_off, src_off;
    std::vector<cplx> proj;
    // explicit form: (sink tuple, source tuple, W)
    std::vector<int8_t> ex_snk, ex_src;
    std::vector<cplx> ex_w;
    // canonical form
    std::vector<Mask> rows[2], cols[2];          // distinct ascending sets, lexicographic order
    std::vector<std::vector<CanonTerm>> snk_can, src_can;   // per free index (factored)
    std::vector<CanonTerm> terms;                // merged canonical terms: a = u minor id, b = d minor id
    TreePlan tree;
    EgraphPlan eg;
    DirectPlan direct;
    double flops_direct = 0, flops_tree = 0, flops_egraph = 0;
};

// planner entry points (planner.cpp); return "" on success or an error message
std::string plan_factored(HostPlan& p);
std::string plan_explicit(HostPlan& p);
std::string operator_terms(int op, int& n_u, int& n_d, int& n_free, std::vector<int8_t>& idx,
                           std::vector<cplx>& w, std::vector<int64_t>& off, std::vector<cplx>& proj, double& scale);
double flops_lu(int n);

// structural checks of a plan's device arrays ("" when every index is in range)
std::string validate_plan(const HostPlan& p);

// serialisation (planner.cpp)
std::string plan_write(const HostPlan& p, const std::string& path);
std::string plan_read(HostPlan& p, const std::string& path);

}  // namespace mbc
