"""CPU oracle of the colour-coding dynamic programme (arXiv 1908.11248, Sections 2-4).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline leg of the
benchmark are its only users.  The GPU library never imports, links or runs it, and it shares no
code with the GPU library.  The arithmetic lives in ``oracle.cpp`` (plain C++ with std::map);
this module compiles it with g++ and marshals arguments through ctypes.

Every public function names the passage it restates:
  * ``philox4x32_10`` / ``colors``: Philox4x32-10 (Salmon et al., SC'11) and the random
    colouring of Section 2.1.
  * ``nice_td``: the nice tree decomposition (Section 1.2 definitions, Section 3).
  * ``run_dp``: the node rules of Section 3.1 with counts, and the root test.
  * ``Run.enumerate``: result reconstruction R(x, M), Section 4.
  * ``backtrack``: an independent plain backtracking counter (second oracle).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None

LEAF, INTRODUCE, FORGET, JOIN = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.cpp into a shared library (g++ -O2); returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, u64 = ctypes.c_int32, ctypes.c_uint64
    lib.or_philox4x32_10.argtypes = [P, P, P]
    lib.or_philox4x32_10.restype = None
    lib.or_color.argtypes = [i32, i32, i32, u64, P]
    lib.or_color.restype = None
    lib.or_nice_td.argtypes = [i32, i32, P, i32, P, P, P, i32, P, P, P, P, P, P]
    lib.or_nice_td.restype = i32
    lib.or_dp_run.argtypes = [i32, P, P, i32, i32, P, i32, P, P, P, P, i32, i32, i32, P, i32]
    lib.or_dp_run.restype = P
    lib.or_dp_free.argtypes = [P]
    lib.or_dp_free.restype = None
    lib.or_dp_num_nodes.argtypes = [P]
    lib.or_dp_num_nodes.restype = i32
    lib.or_dp_results.argtypes = [P, P, P, P]
    lib.or_dp_results.restype = None
    lib.or_dp_table.argtypes = [P, i32, i32, P, P, P]
    lib.or_dp_table.restype = None
    lib.or_enumerate.argtypes = [P, u64, P, P]
    lib.or_enumerate.restype = u64
    lib.or_backtrack.argtypes = [i32, P, P, i32, i32, P, P, i32, u64, P, P]
    lib.or_backtrack.restype = u64
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _td_arrays(td):
    bags, parent = td
    bag_ptr = np.zeros(len(bags) + 1, dtype=np.int32)
    bag_ptr[1:] = np.cumsum([len(b) for b in bags])
    bag_vtx = _i32([u for b in bags for u in b]) if bag_ptr[-1] else np.zeros(1, np.int32)
    return len(bags), bag_ptr, bag_vtx, _i32(parent)


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11): four 32-bit outputs."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def colors(n: int, trials: int, k: int, seed: int) -> np.ndarray:
    """Random colouring of Section 2.1: uint8[trials, n], colour of v in trial t from the first
    Philox word of counter (v, t, 0, 0) and key (seed lo, seed hi), scaled as (x * k) >> 32."""
    lib = _load()
    out = np.zeros((trials, n), dtype=np.uint8)
    lib.or_color(n, trials, k, seed, _ptr(out))
    return out


def nice_td(nF, edges, td):
    """Nice tree decomposition (Section 1.2) of F from a tree decomposition; a list of nodes
    (type, child0, child1, vertex, bag) in post-order, root last.  None if td is invalid."""
    lib = _load()
    e = _i32(edges).reshape(-1)
    nb, bp, bv, par = _td_arrays(td)
    cap = 4 * nF * max(1, nb) + 8
    ty, c0, c1, vx = (np.zeros(cap, np.int32) for _ in range(4))
    optr = np.zeros(cap + 1, np.int32)
    ovtx = np.zeros(cap * max(1, nF), np.int32)
    r = lib.or_nice_td(nF, len(e) // 2, _ptr(e) if len(e) else None, nb, _ptr(bp), _ptr(bv),
                       _ptr(par), cap, _ptr(ty), _ptr(c0), _ptr(c1), _ptr(vx), _ptr(optr),
                       _ptr(ovtx))
    if r < 0:
        return None
    return [(int(ty[i]), int(c0[i]), int(c1[i]), int(vx[i]),
             [int(u) for u in ovtx[optr[i]:optr[i + 1]]]) for i in range(r)]


class Run:
    """Result of the dynamic programme (Section 3.1) over every trial of a colouring."""

    def __init__(self, handle, nF, trials):
        self._h = handle
        self.nF = nF
        self.trials = trials
        lib = _load()
        self.num_nodes = lib.or_dp_num_nodes(handle)
        self.exists = np.zeros(trials, np.uint8)
        self.count = np.zeros(trials, np.uint64)
        self.node_sizes = np.zeros((trials, self.num_nodes), np.uint64)
        lib.or_dp_results(handle, _ptr(self.exists), _ptr(self.count), _ptr(self.node_sizes))

    def __del__(self):
        if getattr(self, "_h", None):
            _load().or_dp_free(self._h)
            self._h = None

    def table(self, t: int, x: int, bag_size: int):
        """Table D_x of trial t in key order: (phi int32[N, b], C uint32[N], count uint64[N])."""
        N = int(self.node_sizes[t, x])
        phi = np.zeros((N, max(1, bag_size)), np.int32)
        mask = np.zeros(N, np.uint32)
        cnt = np.zeros(N, np.uint64)
        _load().or_dp_table(self._h, t, x, _ptr(phi), _ptr(mask), _ptr(cnt))
        return phi[:, :bag_size], mask, cnt

    def enumerate(self, limit: int):
        """Reconstruction from the root (Section 4): (sorted distinct embeddings int32[m, n_F]
        truncated to limit, distinct total, sum of per-trial list lengths)."""
        out = np.zeros((max(1, limit), self.nF), np.int32)
        per = ctypes.c_uint64(0)
        tot = _load().or_enumerate(self._h, limit, _ptr(out), ctypes.byref(per))
        return out[:min(limit, tot)], int(tot), int(per.value)


def run_dp(graph, pattern, colours, k: int, degree_filter: bool = True, allow=None,
           distance_prune: bool = False) -> Run:
    """Bottom-up dynamic programme of Section 3.1 for every row of ``colours`` (uint8[T, n]).
    ``allow`` (uint32[n], optional): bit y of allow[x] lets pattern vertex y map to host vertex x
    (Section 3.2, masking unprofitable mappings).  ``distance_prune``: an introduced vertex with
    no bag neighbour whose nearest same-component bag vertex w is at F-distance 2 takes only the
    host vertices within distance 2 of phi(w) (Section 3.2, mapping expansion)."""
    lib = _load()
    row_ptr, col = graph
    nF, edges, td = pattern
    rp, cl = _i32(row_ptr), _i32(col)
    if len(cl) == 0:
        cl = np.zeros(1, np.int32)
    e = _i32(edges).reshape(-1)
    nb, bp, bv, par = _td_arrays(td)
    colours = np.ascontiguousarray(np.asarray(colours, dtype=np.uint8))
    if colours.ndim == 1:
        colours = colours[None, :]
    T = colours.shape[0]
    am = None if allow is None else np.ascontiguousarray(np.asarray(allow, dtype=np.uint32))
    h = lib.or_dp_run(len(rp) - 1, _ptr(rp), _ptr(cl), nF, len(e) // 2,
                      _ptr(e) if len(e) else None, nb, _ptr(bp), _ptr(bv), _ptr(par),
                      _ptr(colours), T, k, int(bool(degree_filter)),
                      _ptr(am) if am is not None else None, int(bool(distance_prune)))
    if not h:
        raise ValueError("oracle: invalid input")
    return Run(h, nF, T)


def backtrack(graph, pattern, colours_row, limit: int = 0, degree_filter: bool = False):
    """Independent second oracle: (count, sorted first `limit` embeddings) of colourful
    embeddings under one colouring by plain backtracking."""
    lib = _load()
    row_ptr, col = graph
    nF, edges, _ = pattern
    rp, cl = _i32(row_ptr), _i32(col)
    if len(cl) == 0:
        cl = np.zeros(1, np.int32)
    e = _i32(edges).reshape(-1)
    z = np.ascontiguousarray(np.asarray(colours_row, dtype=np.uint8))
    out = np.zeros((max(1, limit), nF), np.int32)
    nout = ctypes.c_uint64(0)
    c = lib.or_backtrack(len(rp) - 1, _ptr(rp), _ptr(cl), nF, len(e) // 2,
                         _ptr(e) if len(e) else None, _ptr(z), int(bool(degree_filter)), limit,
                         _ptr(out), ctypes.byref(nout))
    return int(c), out[:nout.value]
