// blocks.hpp - hadron blocks and block plans, host side (internal).
//
// arXiv 2201.04269 Sec. 2 (hadron blocks), Sec. 3 (general and expanded block form of a
// multi-baryon correlator, canonical factor order, multiplicities) and Sec. 4 (factor
// trees over the expanded terms).
#pragma once
#include <array>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "plan.hpp"

namespace mbc {

constexpr int kEta = 6912;          // entries of one block: (s1, s2, s3, alpha)
constexpr int kBlockTypes = 6;      // P, N, P+, P-, N+, N- (mbc_block_type)

// Flavour of q1 (= q3) of a block type: 0 = up (P types), 1 = down (N types); q2 is the other.
inline int block_q1(int type) { return (type == 1 || type == 4 || type == 5) ? 1 : 0; }

// Nonzero entries of the block type's G (C gamma_5, C gamma_5 P_+ or C gamma_5 P_-).
struct GammaNz {
    int n = 0;
    int be[16], ga[16];
    cplx g[16];
};
void block_gamma(int type, GammaNz& out);                  // planner.cpp

// One product of baryons of a sink operator: coef * sum_alpha T_j(alpha) prod_i B_i^{alpha_i}.
struct BaryonProduct {
    double coef = 1.0;
    int A = 0;
    int types[4] = {0, 0, 0, 0};
    std::vector<std::vector<std::pair<std::array<int8_t, 4>, cplx>>> tie;   // [j] -> (alpha tuple, weight)
};
struct BaryonForm {
    double norm = 1.0;                                     // normalisation of the sink operator
    std::vector<BaryonProduct> products;
};
std::string operator_products(int op, BaryonForm& out);   // planner.cpp

struct BlockHostPlan {
    int op = 0, prec = 0, A = 0, n_u = 0, n_d = 0;
    std::vector<int> n_w;                  // source assignments per product
    int64_t expanded = 0;                  // terms before merging
    double scale = 1.0;                    // sink norm x source norm
    std::vector<int32_t> ids;              // merged terms [K][A], global ids (type * kEta + eta), ascending
    std::vector<cplx> w;                   // [K] merged weights (integer valued, scale not applied)
    std::vector<int32_t> multiplicity;     // [K] expanded terms merged into each (Sec. 3)
    std::vector<int32_t> factor;           // distinct global ids, ascending: compact index = position
    std::vector<int> types;                // block types used, ascending
    // device walk of the factor tree: a unit is a level A-2 vertex (A >= 2; its path
    // prefix multiplies the sum over its leaves) or a group of leaves (A == 1)
    std::vector<uint16_t> unit_pre;        // [n_units][A - 1] compact factors of the path
    std::vector<int32_t> unit_leaf;        // [n_units + 1] first leaf of each unit
    std::vector<uint16_t> leaf_f;          // [K] compact factor of each leaf
    int64_t level_nodes[4] = {0, 0, 0, 0};
    // hash-consing of the units' leaf sums (Sec. 5's congruence step on the block terms):
    // distinct sums sum_leaves w F[leaf] among the units (equal factor and weight lists),
    // and the leaf terms of those distinct sums (A >= 2; 0 otherwise)
    int64_t shared_sums = 0, shared_sum_terms = 0;
    double block_flops_per_site = 0, tree_flops_per_slice = 0;
};
std::string plan_blocks(BlockHostPlan& bp);                // blocks_planner.cpp

}  // namespace mbc
