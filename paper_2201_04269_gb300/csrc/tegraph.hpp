// tegraph.hpp - tensor e-graph of arXiv 2201.04269 Sec. 5 (host planner, internal).
#pragma once
#include <cstdint>
#include <string>

namespace mbc {
// Saturate and extract the tensor e-graph of a product of tensors written as text,
// "name(i,j,k) name(l,m) ..." (a label used twice is summed), with the tensors named in
// antisym_names (space separated) antisymmetric in their slots; dim is the index range
// used by the flop counts.  plan receives the extracted plan: "root <id> sign <s>" (E = s x
// the root class's canonical form), then one line per class reached from the root:
//   class <id> <canonical form> cost <flops> : leaf
//   class <id> <canonical form> cost <flops> : prod <id1> [labels] <id2> [labels] sign <+-1>
// Returns "" or an error message.
std::string tensor_egraph(const std::string& text, const std::string& antisym_names, int64_t node_limit, int dim,
                          std::string& plan, int64_t& n_classes, int64_t& n_nodes);
}  // namespace mbc
