"""CPU oracle for causal-set interval abundances and the Benincasa-Dowker action.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference legs may import this package; the
library in ``paper_1805_04463_gb300`` never does.  The arithmetic lives in
``oracle.c`` (plain C, OpenMP, binary128 for the action); this module only
compiles it with gcc and marshals numpy arrays through ctypes.

Source: W. J. Cunningham, arXiv:1805.04463 -- Section "Action Algorithms"
(Algorithms "Naive" and "Optimized Interval Abundance Measurement"), Section
"The Benincasa-Dowker Action" (local and smeared actions), Appendix "Causal
Set Sprinklings" (1+1 and 3+1 Minkowski diamonds).

Pins (tests/test_oracle_*.py): published SplitMix64 outputs, brute force at
small N, a bitset-free dominance count and link count for 2D orders, chain
and antichain closed forms, the eps = 1 reduction of the smeared action and
exact rational arithmetic for the smeared sums, and statistical checks of
the generator (E[R] = N(N-1)/4, 4D acceptance pi/24).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KIND_2D_ORDER, KIND_2D_DIAMOND, KIND_4D_DIAMOND, KIND_3D_DIAMOND, KIND_2D_DS_SLAB = 0, 1, 2, 3, 4
KIND_2D_SQUARE, KIND_2D_CYLINDER = 5, 6
DS_CELLS = 83443  # coarse eta cells of 2 pi / 2^20 rad: eta_0 = 0.5 rad
DS_SUB = 4096     # fine units (2 pi / 2^32 rad) per coarse cell
GRID = 1 << 20


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        i64, u64, i32, u32, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                  ctypes.c_uint32, ctypes.c_void_p)
        lib.oracle_splitmix64_next.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_splitmix64_next.restype = u64
        lib.oracle_draw.argtypes = [u64, u32, u64, u32]
        lib.oracle_draw.restype = u64
        lib.oracle_ds_threshold.argtypes = [i64]
        lib.oracle_ds_threshold.restype = u64
        lib.oracle_sprinkle.argtypes = [i32, i64, u64, vp]
        lib.oracle_precedes.argtypes = [i32, i64, vp, i64, i64]
        lib.oracle_row_words.argtypes = [i64]
        lib.oracle_row_words.restype = i64
        lib.oracle_causal_matrix.argtypes = [i32, i64, vp, vp, i64]
        lib.oracle_interval_size.argtypes = [i64, vp, i64, i64, i64]
        lib.oracle_interval_size.restype = i64
        lib.oracle_interval_abundance_rows.argtypes = [i64, vp, i64, i64, i64, i64, vp, i64, i32]
        lib.oracle_interval_abundance.argtypes = [i64, vp, i64, vp, i64, i32]
        lib.oracle_interval_abundance_naive.argtypes = [i32, i64, vp, vp, i64]
        lib.oracle_interval_abundance_dominance2d.argtypes = [i64, vp, i64, i64, i64, vp, i64]
        lib.oracle_links_2d.argtypes = [i64, vp]
        lib.oracle_links_2d.restype = i64
        lib.oracle_degrees.argtypes = [i64, vp, i64, vp, vp]
        lib.oracle_sparse_relations.argtypes = [i64, vp, i64, i32, vp, vp, i64]
        lib.oracle_longest_chain.argtypes = [i64, vp, i64, i64, i64]
        lib.oracle_longest_chain.restype = i64
        lib.oracle_greedy_antichain.argtypes = [i64, vp, i64, i64, vp]
        lib.oracle_greedy_antichain.restype = i64
        lib.oracle_layer_sums.argtypes = [i64, vp, i64, vp, i32, vp]
        lib.oracle_dalembertian.argtypes = [i32, i64, vp, vp, i32, ctypes.c_double, vp]
        lib.oracle_action.argtypes = [i32, i64, vp, i64, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")
    return rc


def dim(kind: int) -> int:
    return {KIND_4D_DIAMOND: 4, KIND_3D_DIAMOND: 3}.get(kind, 2)


def splitmix64_outputs(state: int, count: int) -> list[int]:
    st = ctypes.c_uint64(state)
    lib = _load()
    return [int(lib.oracle_splitmix64_next(ctypes.byref(st))) for _ in range(count)]


def draw(seed: int, stream: int, elem: int, slot: int) -> int:
    return int(_load().oracle_draw(seed, stream, elem, slot))


def ds_threshold(g: int) -> int:
    """Cumulative sec^2 mass (scaled to 2^53) of the de Sitter slab up to the end of eta cell g."""
    return int(_load().oracle_ds_threshold(g))


def sprinkle(kind: int, n: int, seed: int) -> np.ndarray:
    """Time-sorted int32 coordinates, shape (dim, n) (structure of arrays)."""
    c = np.zeros((dim(kind), max(n, 0)), dtype=np.int32)
    _check(_load().oracle_sprinkle(kind, n, seed, _ptr(c)), "sprinkle")
    return c


def row_words(n: int) -> int:
    return int(_load().oracle_row_words(n))


def precedes(kind: int, coords: np.ndarray, a: int, b: int) -> bool:
    c = np.ascontiguousarray(coords, dtype=np.int32)
    return bool(_load().oracle_precedes(kind, c.shape[1], _ptr(c), a, b))


def causal_matrix(kind: int, coords: np.ndarray) -> np.ndarray:
    """Symmetrised causal matrix as uint64 row bitsets, shape (n, row_words)."""
    c = np.ascontiguousarray(coords, dtype=np.int32)
    n = c.shape[1]
    w = row_words(n)
    bits = np.zeros((n, w), dtype=np.uint64)
    _check(_load().oracle_causal_matrix(kind, n, _ptr(c), _ptr(bits), w), "causal_matrix")
    return bits


def hist_len(n: int) -> int:
    return max(n - 1, 1)


def interval_size(bits: np.ndarray, i: int, j: int) -> int:
    n, w = bits.shape
    return int(_load().oracle_interval_size(n, _ptr(bits), w, i, j))


def interval_abundance(bits: np.ndarray, threads: int = 0, rows=None) -> np.ndarray:
    """N_k for k = 0..n-2 from the bitset.  rows = (begin, end, step) samples rows i."""
    n, w = bits.shape
    hist = np.zeros(hist_len(n), dtype=np.int64)
    b, e, s = rows if rows is not None else (0, n, 1)
    _check(_load().oracle_interval_abundance_rows(n, _ptr(bits), w, b, e, s, _ptr(hist), hist.size,
                                                  threads), "interval_abundance")
    return hist


def interval_abundance_threads(bits: np.ndarray, threads: int = 0, rows=None):
    """As interval_abundance, also returning the number of threads used."""
    n, w = bits.shape
    hist = np.zeros(hist_len(n), dtype=np.int64)
    b, e, s = rows if rows is not None else (0, n, 1)
    t = _check(_load().oracle_interval_abundance_rows(n, _ptr(bits), w, b, e, s, _ptr(hist),
                                                      hist.size, threads), "interval_abundance")
    return hist, t


def interval_abundance_naive(kind: int, coords: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(coords, dtype=np.int32)
    n = c.shape[1]
    hist = np.zeros(hist_len(n), dtype=np.int64)
    _check(_load().oracle_interval_abundance_naive(kind, n, _ptr(c), _ptr(hist), hist.size), "naive")
    return hist


def interval_abundance_dominance2d(v: np.ndarray, rows=None) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.int32)
    n = v.size
    hist = np.zeros(hist_len(n), dtype=np.int64)
    b, e, s = rows if rows is not None else (0, n, 1)
    _check(_load().oracle_interval_abundance_dominance2d(n, _ptr(v), b, e, s, _ptr(hist), hist.size),
           "dominance2d")
    return hist


def links_2d(v: np.ndarray) -> int:
    v = np.ascontiguousarray(v, dtype=np.int32)
    return int(_load().oracle_links_2d(v.size, _ptr(v)))


def action(dim_: int, n: int, hist: np.ndarray, eps: float = 0.0):
    """(S, bracket): local action for eps <= 0 or eps == 1, smeared otherwise."""
    h = np.ascontiguousarray(hist, dtype=np.int64)
    out = ctypes.c_double(0.0)
    br = ctypes.c_int64(0)
    _check(_load().oracle_action(dim_, n, _ptr(h) if h.size else None, h.size, float(eps),
                                 ctypes.byref(out), ctypes.byref(br)), "action")
    return out.value, br.value


def degrees(bits: np.ndarray):
    """(kin, kout) int32: past and future relation counts of every element."""
    n, w = bits.shape
    kin = np.zeros(n, dtype=np.int32)
    kout = np.zeros(n, dtype=np.int32)
    _check(_load().oracle_degrees(n, _ptr(bits), w, _ptr(kin), _ptr(kout)), "degrees")
    return kin, kout


def sparse_relations(bits: np.ndarray, direction: int):
    """(offsets int64[n+1], cols int32): past (0) or future (1) relation lists."""
    n, w = bits.shape
    offsets = np.zeros(n + 1, dtype=np.int64)
    lib = _load()
    _check(lib.oracle_sparse_relations(n, _ptr(bits), w, direction, _ptr(offsets), None, 0), "sparse_relations")
    cols = np.zeros(max(int(offsets[n]), 1), dtype=np.int32)
    _check(lib.oracle_sparse_relations(n, _ptr(bits), w, direction, _ptr(offsets), _ptr(cols), cols.size),
           "sparse_relations")
    return offsets, cols[:int(offsets[n])]


def longest_chain(bits: np.ndarray, i: int = -1, j: int = -1) -> int:
    """Longest chain from i to j in relations (-1 if i does not precede j);
    i = j = -1: the height of the whole set in elements."""
    n, w = bits.shape
    return int(_load().oracle_longest_chain(n, _ptr(bits), w, i, j))


def greedy_antichain(bits: np.ndarray, seed: int):
    """(size, member bitset uint64[row_words]) of the greedy maximal antichain from `seed`."""
    n, w = bits.shape
    out = np.zeros(w, dtype=np.uint64)
    size = int(_load().oracle_greedy_antichain(n, _ptr(bits), w, seed, _ptr(out)))
    return size, out


def layer_sums(bits: np.ndarray, kmax: int, phi=None) -> np.ndarray:
    """S[m, j] = sum of phi(i) over i preceding j with |A_ij| = m, m = 0..kmax."""
    n, w = bits.shape
    out = np.zeros((kmax + 1, n), dtype=np.float64)
    ph = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    _check(_load().oracle_layer_sums(n, _ptr(bits), w, None if ph is None else _ptr(ph), kmax, _ptr(out)),
           "layer_sums")
    return out


def dalembertian(dim_: int, layers: np.ndarray, ell: float = 1.0, phi=None) -> np.ndarray:
    """B phi(j) (Eqs. b2d_local, b4d_local) from the layer sums."""
    L = np.ascontiguousarray(layers, dtype=np.float64)
    n = L.shape[1]
    out = np.zeros(n, dtype=np.float64)
    ph = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    _check(_load().oracle_dalembertian(dim_, n, None if ph is None else _ptr(ph), _ptr(L), L.shape[0] - 1,
                                       float(ell), _ptr(out)), "dalembertian")
    return out
