"""ctypes loader for the oracle's plain-C sums (test infrastructure; see oracle/__init__).

``build()`` compiles ``csrc/oracle.c`` with gcc (OpenMP when available) into
``oracle/liboracle.so``; ``lib()`` loads it, building on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_LIB = None


def build(force: bool = False) -> str:
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build())
        _LIB.oracle_max_threads.restype = ctypes.c_int
    return _LIB


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def det(m) -> complex:
    m = _c128(m)
    out = np.zeros(2)
    lib().oracle_det(ctypes.c_int(m.shape[0]), _p(m), _p(out))
    return complex(out[0], out[1])


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def direct(n_u, n_d, snk, src, proj, U, D, n_threads=1):
    """Per-site Eq. 1 over the factored index set.  snk/src: list over free index j of
    (idx int8 [n, n_u+n_d], w complex [n]).  U, D: [n_sites, 12, 12].  Returns [n_sites]."""
    U, D = _c128(U).reshape(-1, 12, 12), _c128(D).reshape(-1, 12, 12)
    n_sites = U.shape[0]
    nq = n_u + n_d

    def pack(side):
        idx = np.ascontiguousarray(np.concatenate([s[0] for s in side]).reshape(-1, nq), dtype=np.int8)
        w = _c128(np.concatenate([s[1] for s in side]))
        off = np.zeros(len(side) + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(s[1]) for s in side])
        return idx, w, off

    si, sw, so = pack(snk)
    ri, rw, ro = pack(src)
    P = _c128(proj)
    out = np.zeros(2 * n_sites)
    lib().oracle_direct(ctypes.c_int(n_u), ctypes.c_int(n_d), ctypes.c_int(len(snk)),
                        _p(si), _p(sw), _p(so), _p(ri), _p(rw), _p(ro), _p(P), _p(U), _p(D),
                        ctypes.c_int64(n_sites), _p(out), ctypes.c_int(n_threads))
    return out.view(np.complex128)


def canonical(n_u, n_d, minors_u, minors_d, mu, md, W, U, D, n_threads=1):
    """Per-site canonical sum.  minors_f = (rows int8 [m, n_f], cols int8 [m, n_f])."""
    U, D = _c128(U).reshape(-1, 12, 12), _c128(D).reshape(-1, 12, 12)
    n_sites = U.shape[0]
    ru, cu = (np.ascontiguousarray(a, dtype=np.int8) for a in minors_u)
    rd, cd = (np.ascontiguousarray(a, dtype=np.int8) for a in minors_d)
    mu = np.ascontiguousarray(mu, dtype=np.int32)
    md = np.ascontiguousarray(md, dtype=np.int32)
    W = _c128(W)
    out = np.zeros(2 * n_sites)
    lib().oracle_canonical(ctypes.c_int(n_u), ctypes.c_int(n_d),
                           ctypes.c_int64(ru.shape[0]), _p(ru), _p(cu),
                           ctypes.c_int64(rd.shape[0]), _p(rd), _p(cd),
                           ctypes.c_int64(len(W)), _p(mu), _p(md), _p(W),
                           _p(U), _p(D), ctypes.c_int64(n_sites), _p(out), ctypes.c_int(n_threads))
    return out.view(np.complex128)


def minors(n, rows, cols, M, n_threads=1):
    M = _c128(M).reshape(-1, 12, 12)
    rows = np.ascontiguousarray(rows, dtype=np.int8)
    cols = np.ascontiguousarray(cols, dtype=np.int8)
    out = np.zeros((M.shape[0], rows.shape[0]), dtype=np.complex128)
    lib().oracle_minors(ctypes.c_int(n), ctypes.c_int64(rows.shape[0]), _p(rows), _p(cols), _p(M),
                        ctypes.c_int64(M.shape[0]), _p(out), ctypes.c_int(n_threads))
    return out


def tree(factors, children, coefficients, values, n_threads=1):
    """Linearised factor tree value for each row of ``values`` ([n_sites, n_factor_values])."""
    f = np.ascontiguousarray(factors, dtype=np.int32)
    ch = np.ascontiguousarray(children, dtype=np.int32)
    co = _c128(coefficients)
    v = _c128(values)
    v = v.reshape(-1, v.shape[-1])
    out = np.zeros(2 * v.shape[0])
    lib().oracle_tree(ctypes.c_int64(len(f)), _p(f), _p(ch), _p(co), ctypes.c_int64(v.shape[1]), _p(v),
                      ctypes.c_int64(v.shape[0]), _p(out), ctypes.c_int(n_threads))
    return out.view(np.complex128)
