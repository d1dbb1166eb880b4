// Host check of the FP32 kernel's walker programs (csrc/walks.cpp) on the operator
// library's e-graph plans: each walker's steps, replayed on column sets, must produce
// exactly the A (or B) leaf column sets of the plan with the plan's Laplace signs; every
// leaf appears once over all walkers; batches hold at most LB leaves; the walkers' leaf
// costs are balanced.  Built and run by tests/test_walks_cpu.py; prints "OK <summary>"
// or the first failure.
#include "walk.hpp"
#include "plan.hpp"

#include <cstdio>
#include <string>
#include <vector>

using namespace mbc;

static int popcount_below(Mask m, int c) {
    int k = 0;
    for (int i = 0; i < c; ++i) k += (m >> i) & 1u;
    return k;
}

static std::string check(const MinorPlan& m, int W, int LB) {
    if (m.n == 0) return "";
    std::vector<double> cost(m.cols.size());
    for (size_t l = 0; l < cost.size(); ++l) cost[l] = 1.0 + (double)(l % 7);
    Walks wk;
    std::string err = build_walks(m, W, LB, cost, wk);
    if (!err.empty()) return "build_walks: " + err;
    if ((int)wk.step_off.size() != W + 1) return "step_off size";
    std::vector<int> seen(m.cols.size(), 0);
    std::vector<double> wcost(W, 0.0);
    double maxleaf = 0;
    for (double c : cost) maxleaf = std::max(maxleaf, c);
    for (int w = 0; w < W; ++w) {
        Mask cols[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int depth = 0;                 // deepest level with a valid table
        for (int s = wk.step_off[w]; s < wk.step_off[w + 1]; ++s) {
            const WalkStep& st = wk.steps[s];
            if (st.level > 0) {
                if (st.level > depth + 1) return "step skips a level";
                const Mask parent = st.level == 1 ? 0 : cols[st.level - 1];
                if (parent & (1u << st.col)) return "step adds a column already present";
                const Mask c = parent | (1u << st.col);
                const int want = (popcount_below(c, st.col) & 1) ? -1 : 1;
                if (st.sign != want) return "node sign";
                cols[st.level] = c;
                depth = st.level;
                if (st.nleaf > 0 && st.level != m.n - 1) return "leaves attached below level n-1";
            } else if (st.nleaf == 0) {
                return "empty step";
            }
            if (st.nleaf > LB) return "batch larger than LB";
            if (st.nleaf > 0 && m.n > 1 && depth < m.n - 1) return "leaves without a parent table";
            const Mask parent = m.n == 1 ? 0 : cols[m.n - 1];
            for (int q = 0; q < st.nleaf; ++q) {
                const WalkLeaf& lf = wk.leaves[st.leaf0 + q];
                if (lf.leaf < 0 || lf.leaf >= (int)m.cols.size()) return "leaf index";
                if (parent & (1u << lf.col)) return "leaf adds a column already present";
                const Mask c = parent | (1u << lf.col);
                if (c != m.cols[lf.leaf]) return "leaf column set differs from the plan's";
                const int want = (popcount_below(c, lf.col) & 1) ? -1 : 1;
                if (lf.sign != want) return "leaf sign";
                seen[lf.leaf] += 1;
                wcost[w] += cost[lf.leaf];
            }
        }
    }
    for (size_t l = 0; l < seen.size(); ++l)
        if (seen[l] != 1) return "leaf " + std::to_string(l) + " produced " + std::to_string(seen[l]) + " times";
    double total = 0, mx = 0;
    for (double c : wcost) { total += c; mx = std::max(mx, c); }
    if (mx > total / W + maxleaf + 1e-9) return "walkers unbalanced";
    return "";
}

int main() {
    const int ops[] = {0, 2, 4, 6};         // proton, dinucleon I, He-3 I, He-3 II-s
    int checked = 0;
    for (int op : ops) {
        HostPlan p;
        double scale;
        std::vector<int8_t> idx;
        std::vector<cplx> w, proj;
        std::vector<int64_t> off;
        std::string e = operator_terms(op, p.n_u, p.n_d, p.n_free, idx, w, off, proj, scale);
        if (!e.empty()) { printf("FAIL operator %d: %s\n", op, e.c_str()); return 1; }
        p.snk_idx = idx; p.snk_w = w; p.snk_off = off; p.src_idx = idx; p.src_w = w; p.src_off = off; p.proj = proj;
        p.algo = 2;
        p.prec = 2;
        e = plan_factored(p);
        if (!e.empty()) { printf("FAIL plan %d: %s\n", op, e.c_str()); return 1; }
        for (const MinorPlan* m : {&p.eg.A, &p.eg.B})
            for (int W : {1, 3, 6, 12})
                for (int LB : {1, 2, 3, kMaxLeafBatch}) {
                    const std::string r = check(*m, W, LB);
                    if (!r.empty()) {
                        printf("FAIL op %d W %d LB %d: %s\n", op, W, LB, r.c_str());
                        return 1;
                    }
                    ++checked;
                }
    }
    printf("OK %d walker sets\n", checked);
    return 0;
}
