"""The library's tensor e-graph (mbc_tensor_egraph, Sec. 5) against the oracle's, through
the C ABI on a host-only context: the worked rewrite of Sec. 5 (E = eps_ijk eps_lmn T_ijl
T_nmk = -B_kl B_lk, tests/golden/egraph_sec5_example.json) and random tensor networks.
Compared: e-graph size after saturation, the extracted root e-node (leaf or split, its
children as e-classes, the overall sign) and the extracted cost."""
import itertools
import json
import os
import random

import pytest

from oracle import egraph as oe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hctx():
    from paper_2201_04269_gb300 import abi, build
    build.build()
    ctx = abi.mbc_create(-1)
    yield ctx
    abi.mbc_destroy(ctx)


def text(factors):
    return " ".join(f"{n}({','.join(idx)})" for n, idx in factors)


def parse(plan):
    root = plan[0].split()
    assert root[0] == "root"
    classes = {}
    for line in plan[1:]:
        head, _, tail = line.partition(" : ")
        parts = head.split()
        cid, form, cost = int(parts[1]), parts[2], float(parts[4])
        t = tail.split()
        node = ("leaf",) if t[0] == "leaf" else ("prod", int(t[1]), t[2], int(t[3]), t[4], int(t[6]))
        classes[cid] = (form, cost, node)
    return int(root[1]), int(root[3]), classes


def oracle_run(factors, antisym=("eps",)):
    g = oe.TensorEGraph(antisym=antisym)
    r, sign, _ = g.add_expr(factors)
    g.saturate(r)
    best, cost = g.extract()
    return g, r, sign, best, cost


def test_sec5_worked_rewrite(hctx):
    from paper_2201_04269_gb300 import abi
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "egraph_sec5_example.json")))
    E = [(n, tuple(i)) for n, i in gold["E"]]
    plan, (nc, nn) = abi.mbc_tensor_egraph(hctx, text(E), "eps", 100000, 3)
    root, sign, classes = parse(plan)
    g, r, osign, best, ocost = oracle_run(E)
    assert (nc, nn) == (len(g.classes), g.n_nodes)
    form, cost, node = classes[root]
    assert node[0] == "prod" and node[1] == node[3]          # E = (sign) B . B, one class B
    assert sign * node[5] == gold["relative_sign"] == osign * best[r][5]
    assert cost == ocost[r]
    # B is eps_ijk T_ijl: two tensors, both contracted labels internal, two open slots
    bform = classes[node[1]][0]
    assert bform.count("(") == 2 and bform.count("o0") == 1 and bform.count("o1") == 1


def random_network(rng, n_tensors):
    """A random product of tensors (names eps, T, S, with eps of rank 3), every label used
    once or twice, at least one label summed."""
    while True:
        factors, labels = [], []
        for k in range(n_tensors):
            name = rng.choice(["eps", "T", "S"])
            rank = 3 if name == "eps" else rng.choice([2, 3])
            factors.append([name, []])
            labels += [k] * rank
        pool = [f"i{j}" for j in range(12)]
        slots = [(k, s) for k, f in enumerate(factors) for s in range(3 if f[0] == "eps" else 0)]
        # assign labels: pair up slots at random (summed), leftovers open
        ranks = [3 if f[0] == "eps" else rng.choice([2, 3]) for f in factors]
        slots = [(k, s) for k in range(n_tensors) for s in range(ranks[k])]
        rng.shuffle(slots)
        idx = {}
        q = 0
        while q < len(slots):
            lab = pool.pop()
            if q + 1 < len(slots) and rng.random() < 0.75:
                idx[slots[q]] = lab
                idx[slots[q + 1]] = lab
                q += 2
            else:
                idx[slots[q]] = lab
                q += 1
            if not pool:
                pool = [f"j{q}_{m}" for m in range(12)]
        out = [(factors[k][0], tuple(idx[(k, s)] for s in range(ranks[k]))) for k in range(n_tensors)]
        # no tensor may carry the same label twice (a trace of one tensor)
        if any(len(set(i)) < len(i) for _, i in out):
            continue
        if any(c == 2 for c in oe.index_counts(out).values()):
            return out


@pytest.mark.parametrize("seed", range(12))
def test_random_networks_match_oracle(hctx, seed):
    from paper_2201_04269_gb300 import abi
    rng = random.Random(seed)
    E = random_network(rng, rng.choice([2, 3, 4]))
    plan, (nc, nn) = abi.mbc_tensor_egraph(hctx, text(E), "eps", 100000, 3)
    root, sign, classes = parse(plan)
    g, r, osign, best, ocost = oracle_run(E)
    assert (nc, nn) == (len(g.classes), g.n_nodes), E
    form, cost, node = classes[root]
    onode = best[r]
    assert cost == ocost[r], E
    assert node[0] == onode[0], E
    if node[0] == "prod":
        assert sign * node[5] == osign * onode[5], E
        assert (node[1] == node[3]) == (g.find(onode[1]) == g.find(onode[3])), E
    else:
        assert sign == osign, E


def test_rejects_malformed_expressions(hctx):
    from paper_2201_04269_gb300 import abi
    for bad in ("", "T(i,j", "T(i,i,i) S(i)", "T()"):
        with pytest.raises(abi.MbcError):
            abi.mbc_tensor_egraph(hctx, bad, "eps", 1000, 3)


@pytest.mark.parametrize("seed", range(6))
def test_enode_limit_matches_oracle(hctx, seed):
    """Saturation stopped by the e-node limit (Sec. 5) leaves the same e-graph size as the
    oracle's with the same limit, and the extracted cost is the oracle's."""
    from paper_2201_04269_gb300 import abi
    rng = random.Random(100 + seed)
    E = random_network(rng, rng.choice([3, 4]))
    for lim in (2, 4, 7, 12, 30):
        g = oe.TensorEGraph(antisym=("eps",), node_limit=lim)
        r, _, _ = g.add_expr(E)
        g.saturate(r)
        best, cost = g.extract()
        plan, (nc, nn) = abi.mbc_tensor_egraph(hctx, text(E), "eps", lim, 3)
        assert (nc, nn) == (len(g.classes), g.n_nodes), (lim, E)
        root, _, classes = parse(plan)
        assert classes[root][1] == cost[r], (lim, E)
