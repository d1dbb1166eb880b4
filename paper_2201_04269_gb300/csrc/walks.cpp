// walks.cpp - walker programs of the FP32 e-graph kernel (see walk.hpp).
#include "walk.hpp"
#include "plan.hpp"

#include <algorithm>

namespace mbc {

std::string build_walks(const MinorPlan& m, int W, int LB, const std::vector<double>& leaf_cost, Walks& out) {
    out = Walks();
    out.step_off.assign(1, 0);
    if (W < 1 || LB < 1 || LB > kMaxLeafBatch) return "walks: bad walker count or batch size";
    const int n = m.n;
    if (n == 0) {                                   // no minors: every walker is empty
        out.step_off.assign(W + 1, 0);
        return "";
    }
    const int nn = (int)m.nodes.size();
    // the node list must be a depth-first order whose parents are the most recent node
    // one level up (the kernel keeps one table per level)
    {
        std::vector<int> last(8, -1);
        for (int i = 0; i < nn; ++i) {
            const auto& nd = m.nodes[i];
            if (nd.level < 1 || nd.level > n) return "walks: node level out of range";
            const int want = nd.level == 1 ? -1 : last[nd.level - 1];
            if (nd.parent != want) return "walks: column tree is not in depth-first order";
            if ((nd.level == n) != (nd.leaf >= 0)) return "walks: leaf flags inconsistent";
            if (nd.leaf >= (int32_t)leaf_cost.size()) return "walks: leaf index out of range";
            last[nd.level] = i;
            for (int k = nd.level + 1; k < 8; ++k) last[k] = -1;
        }
    }
    std::vector<int> leaf_nodes;
    for (int i = 0; i < nn; ++i)
        if (m.nodes[i].level == n) leaf_nodes.push_back(i);
    const int nl = (int)leaf_nodes.size();
    // contiguous ranges of about equal cost
    double total = 0;
    for (int i : leaf_nodes) total += leaf_cost[m.nodes[i].leaf];
    std::vector<int> cut(W + 1, nl);
    cut[0] = 0;
    {
        double acc = 0;
        int w = 1;
        for (int q = 0; q < nl && w < W; ++q) {
            acc += leaf_cost[m.nodes[leaf_nodes[q]].leaf];
            while (w < W && acc >= total * w / W) cut[w++] = q + 1;
        }
        for (; w < W; ++w) cut[w] = nl;
    }
    std::vector<int> times_computed(nn, 0);
    for (int w = 0; w < W; ++w) {
        std::vector<char> need(nn, 0), in_range(nn, 0);
        for (int q = cut[w]; q < cut[w + 1]; ++q) {
            int i = leaf_nodes[q];
            in_range[i] = 1;
            for (int p = m.nodes[i].parent; p >= 0; p = m.nodes[p].parent) need[p] = 1;
        }
        auto emit_batches = [&](std::vector<int>& kids, bool attach_first) {
            for (size_t s = 0; s < kids.size(); s += (size_t)LB) {
                const int cnt = (int)std::min<size_t>((size_t)LB, kids.size() - s);
                if (!(attach_first && s == 0)) {
                    WalkStep st{0, 0, 1, 0, 0};
                    out.steps.push_back(st);
                }
                WalkStep& st = out.steps.back();
                st.nleaf = (uint8_t)cnt;
                st.leaf0 = (int32_t)out.leaves.size();
                for (int c = 0; c < cnt; ++c) {
                    const auto& nd = m.nodes[kids[s + c]];
                    out.leaves.push_back(WalkLeaf{nd.col, nd.sign, 0, nd.leaf});
                }
            }
        };
        if (n == 1) {
            std::vector<int> kids;
            for (int q = cut[w]; q < cut[w + 1]; ++q) kids.push_back(leaf_nodes[q]);
            emit_batches(kids, false);
        } else {
            for (int i = 0; i < nn; ++i) {
                const auto& nd = m.nodes[i];
                if (nd.level == n || !need[i]) continue;
                out.steps.push_back(WalkStep{nd.level, nd.col, nd.sign, 0, 0});
                times_computed[i] += 1;
                if (nd.level == n - 1) {
                    std::vector<int> kids;
                    for (int j = i + 1; j < nn && m.nodes[j].level == n; ++j)
                        if (in_range[j]) kids.push_back(j);
                    emit_batches(kids, true);
                }
            }
        }
        out.step_off.push_back((int32_t)out.steps.size());
    }
    for (int i = 0; i < nn; ++i)
        if (times_computed[i] > 1)
            out.dup_cfma += (double)(times_computed[i] - 1) * (double)m.level_rows[m.nodes[i].level].size() *
                            m.nodes[i].level;
    return "";
}

}  // namespace mbc
