// tegraph.cpp - tensor e-graph of arXiv 2201.04269 Sec. 5 for tensor-network expressions
// (host planner; the C-ABI entry point is mbc_tensor_egraph in include/mbc.h).
//
// An expression E is a product of tensors with index labels; a label used twice is
// summed (contracted), a label used once is open.  The e-graph is the triple of Sec. 5:
//   U  a union-find over e-class ids,
//   M  the map from a class id to its e-nodes,
//   H  the hash-cons from an e-node to its class id.
// The e-nodes of a class are the expression itself (a leaf: contract it directly) and
// its splits E -> sigma -> E1 E2 into two sub-products, each held as the e-class of its
// canonical form; sigma is the relative sign of the two canonicalisations (a signed
// permutation of the slots of antisymmetric tensors).  A split is admitted when
//   (1) each part contracts at least one index internally, and
//   (2) at least one part holds a tensor all of whose indices are contracted in E,
// the two restrictions of Sec. 5.  Saturation stops at an e-node limit.  Extraction keeps
// in every class the e-node whose children have the most excess parents from distinct
// classes, weighted by the children's flops (the objective of Sec. 5), ties broken by
// the smaller cost.
//
// Canonical form: every order of the factors and every reordering of the slots of the
// antisymmetric tensors (with the sign of that reordering) is tried; contracted labels are
// renamed s0, s1, ... and open labels o0, o1, ... in order of first appearance; the
// smallest string wins.  Brute force, fine for the few-tensor expressions of Sec. 5.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <sstream>
#include <string>
#include <vector>

#include "tegraph.hpp"

namespace mbc {
namespace {

struct Factor {
    std::string name;
    std::vector<std::string> idx;
};
typedef std::vector<Factor> Expr;

std::map<std::string, int> counts(const Expr& e) {
    std::map<std::string, int> c;
    for (auto& f : e)
        for (auto& i : f.idx) c[i] += 1;
    return c;
}

int parity(const std::vector<int>& p) {
    int s = 1;
    std::vector<int> q = p;
    for (size_t i = 0; i < q.size(); ++i)
        while (q[i] != (int)i) {
            std::swap(q[i], q[q[i]]);
            s = -s;
        }
    return s;
}

struct Canon {
    std::string key;
    int sign = 1;
    std::vector<std::string> open;    // original open labels in canonical slot order
    Expr expr;                        // the canonical expression (renamed labels)
};

Canon canonical(const Expr& e, const std::set<std::string>& antisym) {
    const auto cnt = counts(e);
    Canon best;
    bool have = false;
    std::vector<int> order(e.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    // slot permutations per factor
    std::vector<std::vector<std::vector<int>>> perms(e.size());
    for (size_t f = 0; f < e.size(); ++f) {
        std::vector<int> p(e[f].idx.size());
        for (size_t i = 0; i < p.size(); ++i) p[i] = (int)i;
        if (antisym.count(e[f].name)) {
            do perms[f].push_back(p);
            while (std::next_permutation(p.begin(), p.end()));
        } else {
            perms[f].push_back(p);
        }
    }
    do {
        std::vector<size_t> pick(e.size(), 0);
        for (;;) {
            std::map<std::string, std::string> ren;
            int ns = 0, no = 0, sign = 1;
            std::vector<std::string> open;
            Expr ce;
            std::string key;
            for (int f : order) {
                const auto& p = perms[f][pick[f]];
                sign *= parity(p);
                Factor cf;
                cf.name = e[f].name;
                key += e[f].name + "(";
                for (size_t s = 0; s < p.size(); ++s) {
                    const std::string& lab = e[f].idx[p[s]];
                    auto it = ren.find(lab);
                    if (it == ren.end()) {
                        const bool summed = cnt.at(lab) == 2;
                        const std::string nl = summed ? "s" + std::to_string(ns++) : "o" + std::to_string(no++);
                        if (!summed) open.push_back(lab);
                        it = ren.emplace(lab, nl).first;
                    }
                    cf.idx.push_back(it->second);
                    key += it->second + (s + 1 < p.size() ? "," : "");
                }
                key += ")";
                ce.push_back(cf);
            }
            if (!have || key < best.key) {
                best.key = key;
                best.sign = sign;
                best.open = open;
                best.expr = ce;
                have = true;
            }
            size_t f = 0;                      // next slot-permutation combination
            for (; f < e.size(); ++f) {
                if (++pick[f] < perms[f].size()) break;
                pick[f] = 0;
            }
            if (f == e.size()) break;
        }
    } while (std::next_permutation(order.begin(), order.end()));
    return best;
}

// multiplies of a direct contraction: dim^(labels) x (factors - 1)
double flops_of(const Expr& e, int dim) {
    std::set<std::string> labs;
    for (auto& f : e)
        for (auto& i : f.idx) labs.insert(i);
    double v = 1;
    for (size_t k = 0; k < labs.size(); ++k) v *= dim;
    return v * std::max<size_t>(e.size() - 1, 1);
}

struct ENode {
    bool leaf = true;
    int c1 = -1, c2 = -1;
    std::vector<std::string> o1, o2;   // labels (in the class's canonical expression) of the children's open slots
    int sign = 1;
};

struct EGraph {
    std::vector<int> parent;                       // U
    std::vector<std::vector<ENode>> nodes;         // M
    std::map<std::string, int> hashcons;           // H (keyed by canonical form)
    std::vector<Expr> expr;                        // canonical expression of each class
    std::set<std::string> antisym;
    int64_t n_nodes = 0, limit = 100000;

    int find(int a) {
        while (parent[a] != a) {
            parent[a] = parent[parent[a]];
            a = parent[a];
        }
        return a;
    }

    int add(const Expr& e, int& sign, std::vector<std::string>& open) {
        Canon c = canonical(e, antisym);
        sign = c.sign;
        open = c.open;
        auto it = hashcons.find(c.key);
        if (it != hashcons.end()) return find(it->second);
        const int id = (int)parent.size();
        parent.push_back(id);
        nodes.push_back({ENode()});
        expr.push_back(c.expr);
        hashcons.emplace(c.key, id);
        ++n_nodes;
        return id;
    }

    void saturate(int root) {
        std::vector<int> todo{root};
        std::set<int> done;
        while (!todo.empty() && n_nodes < limit) {
            const int cid = find(todo.back());
            todo.pop_back();
            if (!done.insert(cid).second) continue;
            const Expr e = expr[cid];
            const auto cnt = counts(e);
            const size_t n = e.size();
            for (uint32_t mask = 1; mask + 1 < (1u << n) && n_nodes < limit; ++mask) {
                if (!(mask & 1u)) continue;           // each unordered split once
                Expr e1, e2;
                for (size_t f = 0; f < n; ++f) (mask >> f & 1u ? e1 : e2).push_back(e[f]);
                auto internal = [](const Expr& p) {
                    for (auto& kv : counts(p))
                        if (kv.second == 2) return true;
                    return false;
                };
                if (!internal(e1) || !internal(e2)) continue;                       // restriction 1
                auto full = [&](const Expr& p) {
                    for (auto& f : p) {
                        bool all = true;
                        for (auto& i : f.idx) all = all && cnt.at(i) == 2;
                        if (all) return true;
                    }
                    return false;
                };
                if (!full(e1) && !full(e2)) continue;                               // restriction 2
                ENode nd;
                nd.leaf = false;
                int s1, s2;
                nd.c1 = add(e1, s1, nd.o1);
                nd.c2 = add(e2, s2, nd.o2);
                nd.sign = s1 * s2;
                nodes[cid].push_back(nd);
                ++n_nodes;
                todo.push_back(nd.c1);
                todo.push_back(nd.c2);
            }
        }
    }
};

}  // namespace

std::string tensor_egraph(const std::string& text, const std::string& antisym_names, int64_t node_limit, int dim,
                          std::string& plan, int64_t& n_classes, int64_t& n_nodes) {
    // parse "name(i,j,k) name(l,m) ..."
    Expr e;
    {
        std::string t = text;
        size_t p = 0;
        while (p < t.size()) {
            while (p < t.size() && (t[p] == ' ' || t[p] == '*')) ++p;
            if (p >= t.size()) break;
            const size_t lp = t.find('(', p), rp = t.find(')', p);
            if (lp == std::string::npos || rp == std::string::npos || rp < lp) return "tensor expression: expected name(i,j,...)";
            Factor f;
            f.name = t.substr(p, lp - p);
            std::stringstream ss(t.substr(lp + 1, rp - lp - 1));
            std::string lab;
            while (std::getline(ss, lab, ',')) {
                lab.erase(std::remove(lab.begin(), lab.end(), ' '), lab.end());
                if (lab.empty()) return "tensor expression: empty index label";
                f.idx.push_back(lab);
            }
            if (f.name.empty() || f.idx.empty()) return "tensor expression: empty tensor";
            e.push_back(f);
            p = rp + 1;
        }
    }
    if (e.empty() || e.size() > 8) return "tensor expression: 1 to 8 tensors";
    for (auto& kv : counts(e))
        if (kv.second > 2) return "tensor expression: a label appears more than twice";
    EGraph g;
    g.limit = std::max<int64_t>(node_limit, 1);
    {
        std::stringstream ss(antisym_names);
        std::string nm;
        while (ss >> nm) g.antisym.insert(nm);
    }
    int sign;
    std::vector<std::string> open;
    const int root = g.add(e, sign, open);
    g.saturate(root);
    // extraction (Sec. 5 objective)
    std::map<int, std::set<int>> par;
    for (size_t c = 0; c < g.nodes.size(); ++c)
        for (auto& nd : g.nodes[c])
            if (!nd.leaf) {
                par[g.find(nd.c1)].insert((int)c);
                par[g.find(nd.c2)].insert((int)c);
            }
    std::map<int, int> best;
    std::map<int, double> cost;
    std::function<double(int)> solve = [&](int cid) -> double {
        cid = g.find(cid);
        auto it = cost.find(cid);
        if (it != cost.end()) return it->second;
        cost[cid] = 1e300;                        // guards against cycles
        double bobj = -1, bcost = 1e300;
        int bi = 0;
        for (size_t k = 0; k < g.nodes[cid].size(); ++k) {
            const ENode& nd = g.nodes[cid][k];
            double obj = 0, c;
            if (nd.leaf) {
                c = flops_of(g.expr[cid], dim);
            } else {
                std::set<int> kids{g.find(nd.c1), g.find(nd.c2)};
                for (int kk : kids) obj += ((double)par[kk].size() - 1) * flops_of(g.expr[kk], dim);
                std::set<std::string> labs(nd.o1.begin(), nd.o1.end());
                labs.insert(nd.o2.begin(), nd.o2.end());
                c = 1;
                for (size_t q = 0; q < labs.size(); ++q) c *= dim;
                for (int kk : kids) c += solve(kk);
            }
            if (obj > bobj || (obj == bobj && c < bcost)) { bobj = obj; bcost = c; bi = (int)k; }
        }
        best[cid] = bi;
        cost[cid] = bcost;
        return bcost;
    };
    solve(root);
    // the extracted plan, root first: one line per class reached from the root
    auto show = [&](int cid) {
        std::string s;
        for (auto& f : g.expr[cid]) {
            s += f.name + "(";
            for (size_t i = 0; i < f.idx.size(); ++i) s += f.idx[i] + (i + 1 < f.idx.size() ? "," : "");
            s += ")";
        }
        return s;
    };
    std::ostringstream os;
    // E = sign x (value of the root class's canonical form)
    os << "root " << g.find(root) << " sign " << sign << "\n";
    std::vector<int> stack{root};
    std::set<int> seen;
    while (!stack.empty()) {
        const int cid = g.find(stack.back());
        stack.pop_back();
        if (!seen.insert(cid).second) continue;
        const ENode& nd = g.nodes[cid][best.count(cid) ? best[cid] : 0];
        os << "class " << cid << " " << show(cid) << " cost " << cost[cid] << " : ";
        if (nd.leaf) {
            os << "leaf\n";
        } else {
            os << "prod " << g.find(nd.c1) << " [";
            for (size_t i = 0; i < nd.o1.size(); ++i) os << nd.o1[i] << (i + 1 < nd.o1.size() ? "," : "");
            os << "] " << g.find(nd.c2) << " [";
            for (size_t i = 0; i < nd.o2.size(); ++i) os << nd.o2[i] << (i + 1 < nd.o2.size() ? "," : "");
            os << "] sign " << nd.sign << "\n";
            stack.push_back(nd.c2);
            stack.push_back(nd.c1);
        }
    }
    plan = os.str();
    n_classes = (int64_t)g.nodes.size();
    n_nodes = g.n_nodes;
    return "";
}

}  // namespace mbc
