// walk.hpp - walker programs of the FP32 e-graph kernel (internal; plain structs shared
// by the host planner and the device code).
//
// The extracted minor plan of one flavour is a column tree (arXiv 2201.04269 Sec. 5):
// a node at level k adds one column to its parent's column set, and its table
// det M[R, C] over every needed row set R of level k follows from the parent's table by
// one Laplace step.  The FP32 kernel splits the leaves of that tree (the needed column
// sets, in depth-first order) into W contiguous ranges, one per walker (a group of 128
// threads of a block), and gives every walker the depth-first sequence of the internal
// nodes its leaves need.  A walker computes the leaf tables in batches: the children of
// one level-(n-1) node share its table, so up to LB of them are formed together.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace mbc {

// Largest leaf batch of a walker program (the kernel keeps a batch's leaves in registers).
constexpr int kMaxLeafBatch = 4;

// One step of a walker program.  level >= 1: compute the level-`level` table of the
// node that adds column `col` (sign (-1)^q of its position q in the node's column set)
// from the walker's level-(level-1) table.  nleaf > 0: afterwards, form the leaf tables
// of leaves[leaf0 .. leaf0 + nleaf) from the level-(n-1) table.  level == 0: no Laplace
// step, only the leaf batch (a further batch of the same parent, or the children of the
// root when n == 1).
struct WalkStep {
    uint8_t level;
    uint8_t col;
    int8_t sign;
    uint8_t nleaf;
    int32_t leaf0;
};

// A leaf of a walker program: the added column, its sign and the index of the leaf's
// column set among the plan's needed column sets.
struct WalkLeaf {
    uint8_t col;
    int8_t sign;
    uint16_t pad;
    int32_t leaf;
};

struct Walks {
    std::vector<WalkStep> steps;       // all walkers, walker w at [step_off[w], step_off[w + 1])
    std::vector<int32_t> step_off;     // [W + 1]
    std::vector<WalkLeaf> leaves;
    double dup_cfma = 0;               // Laplace multiply-adds of internal nodes computed by more than one walker
};

struct MinorPlan;
// Split the leaves of the column tree m into W contiguous depth-first ranges of about
// equal cost (leaf_cost indexed by the leaf's column-set index) and write every walker's
// program; leaf batches hold at most LB leaves.  Returns "" or a description of an
// inconsistent tree.
std::string build_walks(const MinorPlan& m, int W, int LB, const std::vector<double>& leaf_cost, Walks& out);

}  // namespace mbc
