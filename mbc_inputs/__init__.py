"""Seeded synthetic quark-propagator fields shared by the CUDA path's tests and the oracle.

This module holds only the input recipe (random numbers and their layout), none of the
correlator arithmetic, so that both sides of a parity test can regenerate exactly the same
inputs without depending on each other.

Recipe
------
A propagator field for flavour ``f`` on an ``L^3 x T`` lattice is a complex array
``S[set][t][site][i][j]`` of 12x12 spin-colour matrices (row ``i`` = sink, column ``j`` =
source, ``i = 3*spin + colour``).  Every entry is

    S = exp(-kappa * t) * G            (plain fields)
    S = exp(-kappa * t) * (B_t + eps * G)   (``noise=eps``: a base matrix shared by all
                                              sites of a time slice plus relative noise)

with ``G`` complex standard normal, CN(0, 1): real and imaginary parts independent
N(0, 1/2).  ``G`` is drawn from a counter-based generator so that any single site can be
regenerated on its own:

* ``stream = mix(mix(mix(seed) ^ set) ^ (flavour << 32 | t))`` with ``mix`` the SplitMix64
  output function (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
  OOPSLA 2014), ``flavour`` 0 for up and 1 for down;
* the entry with flat index ``n = site * 144 + 12 * i + j`` takes outputs ``2n + 1`` and
  ``2n + 2`` of the SplitMix64 sequence started at ``stream``, i.e.
  ``z_k = mix(stream + k * 0x9e3779b97f4a7c15)``;
* the two outputs become uniforms ``u1 = ((z1 >> 11) + 1) * 2^-53`` in (0, 1] and
  ``u2 = (z2 >> 11) * 2^-53`` in [0, 1), and the Box-Muller transform gives
  ``G = sqrt(-ln u1) * (cos(2 pi u2) + i sin(2 pi u2))``;
* the shared base ``B_t`` uses ``site = -1`` mapped to ``2^40`` in the counter.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SITE = 1 << 40
N_SC = 12  # spin x colour


def _mix(z):
    """SplitMix64 output function on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, set_index: int, flavour: int, t: int) -> np.uint64:
    """Per-(seed, set, flavour, t) starting point of the SplitMix64 sequence."""
    with np.errstate(over="ignore"):
        h = _mix(np.uint64(seed) + GOLDEN)
        h = _mix(h ^ np.uint64(set_index))
        h = _mix(h ^ np.uint64((flavour << 32) | t))
    return np.uint64(h)


def gaussian_entries(stream: np.uint64, counters: np.ndarray) -> np.ndarray:
    """CN(0,1) values for the given flat entry counters of one stream."""
    n = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        k1 = np.uint64(2) * n + np.uint64(1)
        z1 = _mix(stream + k1 * GOLDEN)
        z2 = _mix(stream + (k1 + np.uint64(1)) * GOLDEN)
    u1 = ((z1 >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0**-53
    u2 = (z2 >> np.uint64(11)).astype(np.float64) * 2.0**-53
    r = np.sqrt(-np.log(u1))
    th = 2.0 * np.pi * u2
    return r * np.cos(th) + 1j * r * np.sin(th)


def site_matrices(seed: int, set_index: int, flavour: int, t: int, sites, kappa: float = 0.5,
                  noise: float | None = None) -> np.ndarray:
    """12x12 propagator matrices of the listed sites of one time slice, shape [n, 12, 12]."""
    sites = np.asarray(sites, dtype=np.int64).reshape(-1)
    st = stream_key(seed, set_index, flavour, t)
    e = np.arange(N_SC * N_SC, dtype=np.uint64)
    cnt = sites.astype(np.uint64)[:, None] * np.uint64(N_SC * N_SC) + e[None, :]
    g = gaussian_entries(st, cnt).reshape(-1, N_SC, N_SC)
    if noise is not None:
        base_cnt = np.uint64(BASE_SITE) * np.uint64(N_SC * N_SC) + e
        b = gaussian_entries(st, base_cnt).reshape(N_SC, N_SC)
        g = b[None] + noise * g
    return np.exp(-kappa * t) * g


def propagator_field(seed: int, set_index: int, flavour: int, T: int, V3: int, kappa: float = 0.5,
                     noise: float | None = None, t_list=None) -> np.ndarray:
    """Whole field of one set and flavour, shape [T, V3, 12, 12] complex128 (or the listed t)."""
    ts = list(range(T) if t_list is None else t_list)
    out = np.empty((len(ts), V3, N_SC, N_SC), dtype=np.complex128)
    sites = np.arange(V3, dtype=np.int64)

    def fill(k):
        out[k] = site_matrices(seed, set_index, flavour, ts[k], sites, kappa, noise)

    # numpy releases the GIL inside its array loops, so time slices fill in parallel
    workers = max(1, min(len(ts), os.cpu_count() or 1, 32))
    if workers > 1 and V3 * len(ts) > 4096:
        with ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(fill, range(len(ts))))
    else:
        for k in range(len(ts)):
            fill(k)
    return out


def su3_random(rng: np.random.Generator, n: int) -> np.ndarray:
    """n Haar-ish random SU(3) matrices (QR of a complex Gaussian, phase-fixed, det 1)."""
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[:, None, None]
    return q


# Synthetic stand-ins for the paper's workloads (lattice L^3 x T, one propagator set per
# source time or configuration); the paper's gauge ensembles are not available.
WORKLOADS = {
    "proton_4x8": dict(ops=("proton",), L=4, T=8, seed=1, kappa=0.5, noise=None, sets=1),
    "dinucleon_16x32": dict(ops=("dinucleon_I", "dinucleon_II"), L=16, T=32, seed=2, kappa=0.5, noise=None, sets=1),
    "he3_24x48": dict(ops=("he3_I", "he3_II", "he3_II_s"), L=24, T=48, seed=3, kappa=0.5, noise=None, sets=1),
    "batched_64": dict(ops=("proton", "dinucleon_I", "dinucleon_II", "he3_I", "he3_II"), L=(16, 24), T=(32, 48),
                       seed=100, kappa=0.5, noise=None, sets=64),
    "he3_32x64_8src": dict(ops=("he3_II", "he3_II_s"), L=32, T=64, seed=5, kappa=0.3, noise=1e-3, sets=8),
}


def workload_fields(name: str, set_index: int = 0, t_list=None, L=None, T=None):
    """(U, D) numpy fields [T', V3, 12, 12] of one set of a named workload."""
    w = WORKLOADS[name]
    L = L or (w["L"] if isinstance(w["L"], int) else w["L"][0])
    T = T or (w["T"] if isinstance(w["T"], int) else w["T"][0])
    V3 = L ** 3
    seed = w["seed"] + (set_index if name == "batched_64" else 0)
    U = propagator_field(seed, set_index, 0, T, V3, w["kappa"], w["noise"], t_list)
    D = propagator_field(seed, set_index, 1, T, V3, w["kappa"], w["noise"], t_list)
    return U, D


# ------------------------------------------------------------------ the same recipe on the GPU
# gen.cu implements the recipe above as a CUDA kernel for fields too large to generate on
# the host; libmbcgen.so is built next to it by build_gpu() (nvcc, sm_103a).
_GEN_DIR = os.path.dirname(os.path.abspath(__file__))
_GEN_SO = os.path.join(_GEN_DIR, "libmbcgen.so")
_GEN = None


def build_gpu(force: bool = False) -> str:
    """Compile gen.cu into libmbcgen.so (skipped when the library is newer than the source)."""
    import shutil
    import subprocess
    src = os.path.join(_GEN_DIR, "gen.cu")
    if not force and os.path.exists(_GEN_SO) and os.path.getmtime(_GEN_SO) >= os.path.getmtime(src):
        return _GEN_SO
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = shutil.which("nvcc") or "nvcc"
    tmp = _GEN_SO + ".tmp"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared", "-Xcompiler", "-fPIC", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stderr}")
    os.replace(tmp, _GEN_SO)
    return _GEN_SO


def _gen():
    global _GEN
    if _GEN is None:
        import ctypes
        lib = ctypes.CDLL(build_gpu())
        lib.mbcgen_fill.restype = ctypes.c_int
        lib.mbcgen_fill.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_void_p]
        _GEN = lib
    return _GEN


def fill_device(out_ptr: int, seed: int, set_index: int, flavour: int, V3: int, t_list, kappa: float = 0.5,
                noise: float | None = None, stream: int = 0) -> None:
    """Write the field of one (seed, set, flavour) for the listed time slices into device
    memory at out_ptr: complex double [len(t_list)][V3][12][12] (same recipe as
    propagator_field; the transcendental functions are the GPU's)."""
    import ctypes
    ts = (ctypes.c_int * len(t_list))(*[int(t) for t in t_list])
    rc = _gen().mbcgen_fill(ctypes.c_void_p(out_ptr), ctypes.c_uint64(seed), ctypes.c_uint64(set_index), flavour,
                            ts, len(t_list), V3, kappa, -1.0 if noise is None else float(noise),
                            ctypes.c_void_p(stream))
    if rc != 0:
        raise RuntimeError(f"mbcgen_fill failed with CUDA error {rc}")
