"""Factor trees (test infrastructure; see oracle/__init__).

arXiv 2201.04269 Sec. 4: a factor tree represents a sum of products of factors; every
root-to-leaf path, times the coefficient stored at its leaf, is one term.  Terms whose
factor strings are identical share their whole path (their coefficients add: the
multiplicity merge of Sec. 3) and terms with a common prefix share that prefix.  The
linearised form (Fig. 5) is three arrays in depth-first order: the factors of every
vertex (the root first, as a placeholder), the number of children of every vertex,
and the leaf coefficients.

Reading: children are visited in ascending lexicographic order of their factor keys,
which reproduces the arrays printed for the worked example of Figs. 4 and 5.
"""
from __future__ import annotations

ROOT = "o"


def build(terms):
    """Linearised factor tree of a list of (coefficient, factor_key_tuple).

    Returns (factors, children, coefficients); factors[0] is ROOT."""
    trie = {}
    for coef, keys in terms:
        node = trie
        for k in keys[:-1]:
            node = node.setdefault(k, {})
        last = keys[-1]
        node[last] = node.get(last, 0) + coef       # identical strings merge (multiplicity)
    factors, children, coefficients = [ROOT], [len(trie)], []

    def visit(node):
        for k in sorted(node):
            sub = node[k]
            factors.append(k)
            if isinstance(sub, dict):
                children.append(len(sub))
                visit(sub)
            else:
                children.append(0)
                coefficients.append(sub)

    visit(trie)
    return factors, children, coefficients


def evaluate(factors, children, coefficients, value):
    """Sum over root-to-leaf paths of (product of value(factor)) x leaf coefficient,
    walking the linearised arrays depth first with a stack of open vertices."""
    prod = [1.0]
    remaining = [children[0]]
    leaf = 0
    total = 0
    for k in range(1, len(factors)):
        while remaining[-1] == 0:
            prod.pop()
            remaining.pop()
        remaining[-1] -= 1
        p = prod[-1] * value(factors[k])
        if children[k] == 0:
            total += coefficients[leaf] * p
            leaf += 1
        else:
            prod.append(p)
            remaining.append(children[k])
    return total


def expand(factors, children, coefficients):
    """Back to the list of (coefficient, factor_key_tuple) terms (inverse of build)."""
    out = []
    path = []
    remaining = [children[0]]
    leaf = 0
    for k in range(1, len(factors)):
        while remaining[-1] == 0:
            path.pop()
            remaining.pop()
        remaining[-1] -= 1
        if children[k] == 0:
            out.append((coefficients[leaf], tuple(path + [factors[k]])))
            leaf += 1
        else:
            path.append(factors[k])
            remaining.append(children[k])
    return out
