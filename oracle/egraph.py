"""Tensor e-graphs (test infrastructure; see oracle/__init__).

arXiv 2201.04269 Sec. 5.  An e-graph is (U, M, H): a union-find over e-class ids, a map
from class ids to classes (sets of e-nodes) and a hash-cons from e-nodes to class ids.
Here an e-node of a tensor expression E (a product of tensors with summed repeated
indices) is either E itself ("leaf") or a split E -> sigma -> E1 E2 into two
sub-expressions whose canonical forms are children e-classes.  Splits obey the two
restrictions of Sec. 5, in this reading (the text admits several):

  1. each part contracts at least one index internally (an index appearing twice in
     the part), and
  2. at least one part holds a tensor all of whose indices are contracted in E.

Canonicalisation (cited work of Li et al.; own brute-force restatement): over every
order of the factors and every reordering of the slots of antisymmetric tensors (with
its sign), rename contracted indices s0, s1, ... and open indices f0, f1, ... in order
of first appearance; the lexicographically smallest string is the canonical form, its
sign the product of the slot-reordering signs, and the open indices keep the order of
their first appearance (the slot order of the canonical tensor).

Extraction (Sec. 5): in every class choose the e-node with the largest objective =
sum over its child classes of (distinct parent classes - 1) x flops of the child; ties
are broken by the smaller total flop count.  Flops count one multiply per term of a
naive contraction.

Also here: the determinant e-graph used for the Laplace minor plan.  A minor
det M[R, C] is the same kind of expression, eps_{c...} M_{r1 c1} ... M_{rk ck}; the
split "expand along row r" gives E1 = M_{r c} (one entry, summed c) and E2 = the
sub-minor det M[R\\r, C\\c], whose canonical form is the ascending (R, C) pair.
"""
from __future__ import annotations

import itertools
from collections import defaultdict

import numpy as np

from .wick import perm_sign


# ----------------------------------------------------------------------------------------
# tensor expressions
# ----------------------------------------------------------------------------------------
def index_counts(factors):
    cnt = defaultdict(int)
    for _, idx in factors:
        for i in idx:
            cnt[i] += 1
    return cnt


def open_indices(factors):
    """Open (free) indices in order of first appearance."""
    cnt = index_counts(factors)
    seen, out = set(), []
    for _, idx in factors:
        for i in idx:
            if cnt[i] == 1 and i not in seen:
                out.append(i)
                seen.add(i)
    return out


def canonical(factors, antisym):
    """(key, sign, open_order): canonical string, its sign, and the original open index
    labels in canonical slot order."""
    best = None
    cnt = index_counts(factors)
    for order in itertools.permutations(range(len(factors))):
        choices = []
        for f in order:
            name, idx = factors[f]
            if name in antisym:
                choices.append([(tuple(idx[p] for p in perm), perm_sign(perm))
                                for perm in itertools.permutations(range(len(idx)))])
            else:
                choices.append([(tuple(idx), 1)])
        for combo in itertools.product(*choices):
            ren, ns, nf, opens = {}, 0, 0, []
            sign = 1
            key = []
            for f, (idx, s) in zip(order, combo):
                sign *= s
                lab = []
                for i in idx:
                    if i not in ren:
                        if cnt[i] == 2:
                            ren[i] = f"s{ns}"
                            ns += 1
                        else:
                            ren[i] = f"f{nf}"
                            nf += 1
                            opens.append(i)
                    lab.append(ren[i])
                key.append((factors[f][0], tuple(lab)))
            key = tuple(key)
            if best is None or key < best[0]:
                best = (key, sign, opens)
    return best


def flops(factors):
    """Multiplies of a naive contraction: (#index assignments) x (#factors - 1), dims 3."""
    labels = {i for _, idx in factors for i in idx}
    return (3 ** len(labels)) * max(len(factors) - 1, 1)


def contracted_in(part):
    cnt = index_counts(part)
    return {i for i, c in cnt.items() if c == 2}


class TensorEGraph:
    """(U, M, H) over canonical tensor expressions."""

    def __init__(self, antisym=("eps",), node_limit=10000):
        self.parent = []           # U: union-find over class ids
        self.classes = {}          # M: class id -> list of e-nodes
        self.hashcons = {}         # H: e-node key -> class id
        self.expr = {}             # class id -> representative factors
        self.antisym = set(antisym)
        self.node_limit = node_limit
        self.n_nodes = 0

    def find(self, a):
        while self.parent[a] != a:
            self.parent[a] = self.parent[self.parent[a]]
            a = self.parent[a]
        return a

    def add_expr(self, factors):
        """Class of a tensor expression (canonicalised) and the (sign, open order)."""
        key, sign, opens = canonical(factors, self.antisym)
        leaf = ("leaf", key)
        if leaf in self.hashcons:
            return self.find(self.hashcons[leaf]), sign, opens
        cid = len(self.parent)
        self.parent.append(cid)
        self.classes[cid] = [leaf]
        self.hashcons[leaf] = cid
        self.n_nodes += 1
        # representative expression with canonical labels
        self.expr[cid] = [(name, lab) for name, lab in key]
        return cid, sign, opens

    def splits(self, factors):
        n = len(factors)
        outer = contracted_in(factors) | {i for _, idx in factors for i in idx if index_counts(factors)[i] == 2}
        for r in range(1, n):
            for part in itertools.combinations(range(n), r):
                if 0 not in part:          # each unordered split once
                    continue
                e1 = [factors[i] for i in part]
                e2 = [factors[i] for i in range(n) if i not in part]
                if not contracted_in(e1) or not contracted_in(e2):
                    continue                                        # restriction 1
                full = lambda p: any(all(i in outer for i in idx) for _, idx in p)
                if not (full(e1) or full(e2)):
                    continue                                        # restriction 2
                yield e1, e2

    def saturate(self, root):
        """Apply the split rewrite to every class until saturation or the e-node limit.

        A split e-node is ("prod", c1, labels1, c2, labels2, sign): the child classes,
        the labels (in this class's representative) of their canonical open slots, and
        the relative sign of the two canonicalisations."""
        todo = [root]
        done = set()
        while todo and self.n_nodes < self.node_limit:
            cid = self.find(todo.pop())
            if cid in done:
                continue
            done.add(cid)
            for e1, e2 in self.splits(self.expr[cid]):
                c1, s1, o1 = self.add_expr(e1)
                c2, s2, o2 = self.add_expr(e2)
                self.classes[cid].append(("prod", c1, tuple(o1), c2, tuple(o2), s1 * s2))
                self.n_nodes += 1
                todo += [c1, c2]
                if self.n_nodes >= self.node_limit:
                    break
        return root

    def parents(self):
        par = defaultdict(set)
        for cid, nodes in self.classes.items():
            for nd in nodes:
                if nd[0] == "prod":
                    par[self.find(nd[1])].add(cid)
                    par[self.find(nd[3])].add(cid)
        return par

    def extract(self):
        """Best e-node per class: max objective, then min cost (shared children once)."""
        par = self.parents()
        best, cost = {}, {}

        def solve(cid):
            cid = self.find(cid)
            if cid in best:
                return cost[cid]
            cands = []
            for nd in self.classes[cid]:
                if nd[0] == "leaf":
                    cands.append((0, flops(self.expr[cid]), nd))
                else:
                    kids = {self.find(nd[1]), self.find(nd[3])}
                    obj = sum((len(par[k]) - 1) * flops(self.expr[k]) for k in kids)
                    own = 3 ** len(set(nd[2]) | set(nd[4]))
                    cands.append((obj, own + sum(solve(k) for k in kids), nd))
            obj, c, nd = max(cands, key=lambda t: (t[0], -t[1]))
            best[cid], cost[cid] = nd, c
            return c

        for cid in list(self.classes):
            solve(cid)
        return best, cost

    def evaluate(self, cid, tensors, best):
        """Value of class cid as an ndarray over its canonical open slots."""
        cid = self.find(cid)
        nd = best[cid]
        fac = self.expr[cid]
        if nd[0] == "leaf":
            return einsum_expr(fac, tensors, open_indices(fac))
        _, c1, p1, c2, p2, sign = nd
        v1 = self.evaluate(c1, tensors, best)
        v2 = self.evaluate(c2, tensors, best)
        labs = sorted(set(p1) | set(p2), key=str)
        sym = {l: chr(ord("a") + k) for k, l in enumerate(labs)}
        spec = "".join(sym[l] for l in p1) + "," + "".join(sym[l] for l in p2) + "->" + \
            "".join(sym[l] for l in open_indices(fac))
        return sign * np.einsum(spec, v1, v2)


def einsum_expr(factors, tensors, out_labels):
    labs = sorted({i for _, idx in factors for i in idx}, key=str)
    sym = {l: chr(ord("a") + k) for k, l in enumerate(labs)}
    spec = ",".join("".join(sym[i] for i in idx) for _, idx in factors) + "->" + "".join(sym[i] for i in out_labels)
    return np.einsum(spec, *[tensors[name] for name, _ in factors])


def levi_civita(n=3):
    e = np.zeros((n,) * n)
    for p in itertools.permutations(range(n)):
        e[p] = perm_sign(p)
    return e


# ----------------------------------------------------------------------------------------
# determinant e-graph (Laplace sub-minor sharing)
# ----------------------------------------------------------------------------------------
class MinorEGraph:
    """E-classes are minors (R, C) (ascending index tuples, equal length); e-nodes of a
    k x k class (k >= 2) are the Laplace expansions along each row r in R and each
    column c in C; a 1 x 1 class is a leaf (a matrix entry).  Hash-cons key = (R, C)."""

    def __init__(self, node_limit=10**7):
        self.nodes = {}          # (R, C) -> list of ("row", r) / ("col", c)
        self.node_limit = node_limit
        self.n_nodes = 0

    @staticmethod
    def children(R, C, node):
        kind, v = node
        if kind == "row":
            p = R.index(v)
            return [((R[:p] + R[p + 1:], C[:q] + C[q + 1:]), (-1) ** (p + q), (v, C[q])) for q in range(len(C))]
        q = C.index(v)
        return [((R[:p] + R[p + 1:], C[:q] + C[q + 1:]), (-1) ** (p + q), (R[p], v)) for p in range(len(R))]

    def saturate(self, roots):
        todo = list(roots)
        while todo and self.n_nodes < self.node_limit:
            R, C = todo.pop()
            if (R, C) in self.nodes:
                continue
            if len(R) == 1:
                self.nodes[(R, C)] = [("leaf", None)]
                continue
            nds = [("row", r) for r in R] + [("col", c) for c in C]
            self.nodes[(R, C)] = nds
            self.n_nodes += len(nds)
            for nd in nds:
                for ch, _, _ in self.children(R, C, nd):
                    if ch not in self.nodes:
                        todo.append(ch)

    def extract(self, roots):
        """Top-down, level by level: every needed k x k class takes the expansion whose
        children have the most excess distinct parents (weighted by child flops)."""
        plan = {}
        need = set(roots)
        while need:
            k = len(next(iter(need))[0])
            if k == 1:
                for key in need:
                    plan[key] = ("leaf", None)
                break
            par = defaultdict(set)
            for key in need:
                for nd in self.nodes[key]:
                    for ch, _, _ in self.children(key[0], key[1], nd):
                        par[ch].add(key)
            fl = 8 * (k - 1)   # complex multiply-adds of a (k-1) x (k-1) child, per term
            nxt = set()
            for key in sorted(need):
                cands = []
                for nd in self.nodes[key]:
                    kids = [ch for ch, _, _ in self.children(key[0], key[1], nd)]
                    cands.append((sum(len(par[c]) - 1 for c in kids) * fl, nd))
                obj, nd = max(cands, key=lambda t: t[0])
                plan[key] = nd
                nxt.update(ch for ch, _, _ in self.children(key[0], key[1], nd))
            need = nxt
        return plan

    def evaluate(self, plan, M, roots):
        memo = {}

        def val(key):
            if key in memo:
                return memo[key]
            R, C = key
            nd = plan[key]
            if nd[0] == "leaf":
                v = M[R[0], C[0]]
            else:
                v = 0j
                for ch, s, (r, c) in self.children(R, C, nd):
                    v += s * M[r, c] * val(ch)
            memo[key] = v
            return v

        return [val(k) for k in roots]
