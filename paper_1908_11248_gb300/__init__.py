"""Python binding of the colour-coding C ABI (include/cc.h): argument marshalling only.

Every function below has the name of the C entry point it calls and does no work of its own
beyond converting arguments (numpy arrays for host buffers) and raising ``CCError`` on a nonzero
return code.  The dynamic programme, colouring and reconstruction all run in the CUDA library
``_build/libcc.so``; there is no CPU fallback: importing works without a GPU, but every call
that needs the library raises if it has not been built.

``Context`` is a convenience holder: it takes the device arena from PyTorch (a uint8 tensor) and
the stream from ``torch.cuda.current_stream()``, which is all PyTorch is used for.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LIB_PATH = _build.LIB
LEAF, INTRODUCE, FORGET, JOIN = 0, 1, 2, 3

CC_OK, CC_EINVAL, CC_ENOMEM, CC_ECAPACITY, CC_ETIMEOUT, CC_ECUDA, CC_ENOTFOUND, CC_EKEYWIDTH = \
    0, -1, -2, -3, -4, -5, -6, -7
CC_EBUSY = -8
CC_ECANCELED = -9

EXPORTS = [
    "cc_strerror", "cc_create", "cc_destroy", "cc_load_graph", "cc_load_pattern",
    "cc_pattern_info", "cc_pattern_nodes", "cc_color", "cc_set_colors", "cc_get_colors",
    "cc_release_colors", "cc_default_opts", "cc_run_dp", "cc_run_batch", "cc_decide", "cc_count",
    "cc_table_stats", "cc_table_dump", "cc_enumerate", "cc_release", "cc_serve_start",
    "cc_serve_submit", "cc_serve_poll", "cc_serve_cancel", "cc_serve_stop", "cc_run_timings",
    "cc_context_stats",
    "cc_nice_decomposition", "cc_check_graph", "cc_count_noalloc", "cc_run_mode",
    "cc_serve_stats", "cc_autotune", "cc_solve_trials", "cc_solve",
    "cc_load_pattern_masked", "cc_enumerate_sets", "cc_probe_bounded_wait",
]
RUN_MODES = ["exact", "planned", "graph", "streamed", "sliced"]
KERNEL_KINDS = ["color", "leaf", "intro_count", "intro_write", "intro_fused", "forget",
                "join_build", "join_count", "join_write", "root", "sort", "reduce", "merge",
                "intro_chain"]


class CCError(RuntimeError):
    def __init__(self, what, code):
        super().__init__(f"{what}: {cc_strerror(code)} ({code})")
        self.code = code


class cc_td(ctypes.Structure):
    _fields_ = [("num_bags", ctypes.c_int32), ("h_bag_ptr", ctypes.c_void_p),
                ("h_bag_vtx", ctypes.c_void_p), ("h_parent", ctypes.c_void_p)]


class cc_run_opts(ctypes.Structure):
    _fields_ = [("degree_filter", ctypes.c_int32), ("retain", ctypes.c_int32),
                ("fuse", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("load_factor", ctypes.c_float), ("block", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("group", ctypes.c_int32),
                ("sort_sweep", ctypes.c_int32), ("distance_prune", ctypes.c_int32),
                ("max_slices", ctypes.c_int32), ("part_bits", ctypes.c_int32),
                ("chain", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                            ctypes.c_size_t)
    sig = {
        "cc_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "cc_create": ([P, ctypes.c_int, P, P, sz], ctypes.c_int),
        "cc_destroy": ([P], ctypes.c_int),
        "cc_load_graph": ([P, i32, P, P], ctypes.c_int),
        "cc_load_pattern": ([P, i32, i32, P, P, P], ctypes.c_int),
        "cc_pattern_info": ([P, i32, P, P], ctypes.c_int),
        "cc_pattern_nodes": ([P, i32, P, P, P, P, P, P], ctypes.c_int),
        "cc_color": ([P, u64, i32, i32, P], ctypes.c_int),
        "cc_set_colors": ([P, P, i32, i32, P], ctypes.c_int),
        "cc_get_colors": ([P, i32, P], ctypes.c_int),
        "cc_release_colors": ([P, i32], ctypes.c_int),
        "cc_default_opts": ([P], None),
        "cc_run_dp": ([P, i32, i32, P, P], ctypes.c_int),
        "cc_run_batch": ([P, i32, P, P, P, P], ctypes.c_int),
        "cc_decide": ([P, i32, P], ctypes.c_int),
        "cc_count": ([P, i32, P], ctypes.c_int),
        "cc_table_stats": ([P, i32, P, P], ctypes.c_int),
        "cc_table_dump": ([P, i32, i32, u64, P, P, P, P, P], ctypes.c_int),
        "cc_enumerate": ([P, i32, u64, P, P, P], ctypes.c_int),
        "cc_enumerate_sets": ([P, i32, u64, P, P, P], ctypes.c_int),
        "cc_probe_bounded_wait": ([P, ctypes.c_uint32], ctypes.c_int),
        "cc_release": ([P, i32], ctypes.c_int),
        "cc_serve_start": ([P, sz, i32], ctypes.c_int),
        "cc_serve_submit": ([P, i32, u64, i32, i32, u64, P], ctypes.c_int),
        "cc_serve_poll": ([P, i64, P, P, P, P, P, P, P], ctypes.c_int),
        "cc_serve_stop": ([P], ctypes.c_int),
        "cc_serve_cancel": ([P, P], ctypes.c_int),
        "cc_run_timings": ([P, i32, i32, P, P, P, P, P], ctypes.c_int),
        "cc_context_stats": ([P, P, P, P], ctypes.c_int),
        "cc_nice_decomposition": ([i32, i32, P, P, i32, P, P, P, P, P, P, P, P], ctypes.c_int),
        "cc_check_graph": ([i32, P, P], ctypes.c_int),
        "cc_run_mode": ([P, i32, P], ctypes.c_int),
        "cc_serve_stats": ([P, P, P, P, P, P, P, P], ctypes.c_int),
        "cc_autotune": ([P, i32, i32, P, i32, i32, P, P, P, P], ctypes.c_int),
        "cc_solve_trials": ([i32, ctypes.c_double], i32),
        "cc_load_pattern_masked": ([P, i32, i32, P, P, P, P], ctypes.c_int),
        "cc_solve": ([P, i32, u64, i32, ctypes.c_double, i32, i32, u64, P, P, P, P, P],
                     ctypes.c_int),
        "cc_count_noalloc": ([ctypes.c_int, P, i32, P, P, i32, i32, P, P, u64, i32, i32, P, P],
                             ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _check(rc, what):
    if rc != 0:
        raise CCError(what, rc)


def cc_strerror(code: int) -> str:
    return lib().cc_strerror(code).decode()


def cc_create(device: int = 0, stream: int = 0, d_arena: int = 0, arena_bytes: int = 1 << 30):
    h = ctypes.c_void_p()
    _check(lib().cc_create(ctypes.byref(h), device, stream or None, d_arena or None,
                           arena_bytes), "cc_create")
    return h


def cc_destroy(ctx):
    _check(lib().cc_destroy(ctx), "cc_destroy")


def cc_load_graph(ctx, row_ptr, col):
    rp, cl = _i32(row_ptr), _i32(col)
    _check(lib().cc_load_graph(ctx, len(rp) - 1, _p(rp), _p(cl) if len(cl) else None),
           "cc_load_graph")


def _td_struct(td):
    """(cc_td by reference or None, arrays to keep alive)."""
    if td is None:
        return None, []
    bags, parent = td
    bp = np.zeros(len(bags) + 1, np.int32)
    bp[1:] = np.cumsum([len(b) for b in bags])
    bv = _i32([u for b in bags for u in b]) if bp[-1] else np.zeros(1, np.int32)
    par = _i32(parent)
    st = cc_td(len(bags), _p(bp), _p(bv), _p(par))
    return ctypes.byref(st), [bp, bv, par, st]


def cc_load_pattern(ctx, nF: int, edges, td=None) -> int:
    e = _i32(edges).reshape(-1)
    pid = ctypes.c_int32(0)
    tdp, keep = _td_struct(td)
    _check(lib().cc_load_pattern(ctx, nF, len(e) // 2, _p(e) if len(e) else None, tdp,
                                 ctypes.byref(pid)), "cc_load_pattern")
    del keep
    return pid.value


def cc_load_pattern_masked(ctx, nF: int, edges, td, allow) -> int:
    """A pattern with allowed mappings: bit u of allow[v] (uint32[n]) lets F-vertex u map to v."""
    e = _i32(edges).reshape(-1)
    a = np.ascontiguousarray(np.asarray(allow, dtype=np.uint32))
    pid = ctypes.c_int32(0)
    tdp, keep = _td_struct(td)
    _check(lib().cc_load_pattern_masked(ctx, nF, len(e) // 2, _p(e) if len(e) else None, tdp,
                                        _p(a), ctypes.byref(pid)), "cc_load_pattern_masked")
    del keep
    return pid.value


def cc_nice_decomposition(nF: int, edges, td=None):
    """Host-only: (nodes in the layout of cc_pattern_nodes, width)."""
    e = _i32(edges).reshape(-1)
    tdp, keep = _td_struct(td)
    cap = 8 * nF * (len(td[0]) if td is not None else nF) + 16
    ty, c0, c1, vx = (np.zeros(cap, np.int32) for _ in range(4))
    bp = np.zeros(cap + 1, np.int32)
    bv = np.zeros(cap * nF + 1, np.int32)
    nn, w = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().cc_nice_decomposition(nF, len(e) // 2, _p(e) if len(e) else None, tdp, cap,
                                       _p(ty), _p(c0), _p(c1), _p(vx), _p(bp), _p(bv),
                                       ctypes.byref(nn), ctypes.byref(w)),
           "cc_nice_decomposition")
    del keep
    N = nn.value
    return [(int(ty[i]), int(c0[i]), int(c1[i]), int(vx[i]),
             [int(u) for u in bv[bp[i]:bp[i + 1]]]) for i in range(N)], w.value


def cc_check_graph(row_ptr, col) -> int:
    """Host-only CSR validation; returns the C return code."""
    rp, cl = _i32(row_ptr), _i32(col)
    return lib().cc_check_graph(len(rp) - 1, _p(rp), _p(cl) if len(cl) else None)


def cc_pattern_info(ctx, pid: int):
    nn, w = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(lib().cc_pattern_info(ctx, pid, ctypes.byref(nn), ctypes.byref(w)), "cc_pattern_info")
    return nn.value, w.value


def cc_pattern_nodes(ctx, pid: int, nF: int):
    N, _ = cc_pattern_info(ctx, pid)
    ty, c0, c1, vx = (np.zeros(N, np.int32) for _ in range(4))
    bp = np.zeros(N + 1, np.int32)
    bv = np.zeros(max(1, N * nF), np.int32)
    _check(lib().cc_pattern_nodes(ctx, pid, _p(ty), _p(c0), _p(c1), _p(vx), _p(bp), _p(bv)),
           "cc_pattern_nodes")
    return [(int(ty[i]), int(c0[i]), int(c1[i]), int(vx[i]),
             [int(u) for u in bv[bp[i]:bp[i + 1]]]) for i in range(N)]


def cc_color(ctx, seed: int, trials: int, k: int) -> int:
    cid = ctypes.c_int32(0)
    _check(lib().cc_color(ctx, seed, trials, k, ctypes.byref(cid)), "cc_color")
    return cid.value


def cc_set_colors(ctx, colors, k: int) -> int:
    z = np.ascontiguousarray(np.asarray(colors, dtype=np.uint8))
    if z.ndim == 1:
        z = z[None, :]
    cid = ctypes.c_int32(0)
    _check(lib().cc_set_colors(ctx, _p(z), z.shape[0], k, ctypes.byref(cid)), "cc_set_colors")
    return cid.value


def cc_get_colors(ctx, cid: int, trials: int, n: int):
    out = np.zeros((trials, n), np.uint8)
    _check(lib().cc_get_colors(ctx, cid, _p(out)), "cc_get_colors")
    return out


def cc_release_colors(ctx, cid: int):
    _check(lib().cc_release_colors(ctx, cid), "cc_release_colors")


def cc_default_opts(**kw) -> cc_run_opts:
    o = cc_run_opts()
    lib().cc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def cc_run_dp(ctx, pid: int, cid: int, opts: cc_run_opts | None = None) -> int:
    rid = ctypes.c_int32(0)
    _check(lib().cc_run_dp(ctx, pid, cid, ctypes.byref(opts) if opts is not None else None,
                           ctypes.byref(rid)), "cc_run_dp")
    return rid.value


def cc_run_batch(ctx, pids, cids, opts: cc_run_opts | None = None):
    p, c = _i32(pids), _i32(cids)
    out = np.zeros(len(p), np.int32)
    _check(lib().cc_run_batch(ctx, len(p), _p(p), _p(c),
                              ctypes.byref(opts) if opts is not None else None, _p(out)),
           "cc_run_batch")
    return [int(x) for x in out]


def cc_decide(ctx, run: int, trials: int):
    out = np.zeros(trials, np.uint8)
    _check(lib().cc_decide(ctx, run, _p(out)), "cc_decide")
    return out


def cc_count(ctx, run: int, trials: int):
    out = np.zeros(trials, np.uint64)
    _check(lib().cc_count(ctx, run, _p(out)), "cc_count")
    return out


def cc_table_stats(ctx, run: int, num_nodes: int):
    out = np.zeros(num_nodes, np.uint64)
    tot = ctypes.c_uint64(0)
    _check(lib().cc_table_stats(ctx, run, _p(out), ctypes.byref(tot)), "cc_table_stats")
    return out, int(tot.value)


def cc_table_dump(ctx, run: int, node: int, capacity: int, bag_size: int):
    cap = max(1, capacity)
    trial = np.zeros(cap, np.int32)
    phi = np.zeros((cap, max(1, bag_size)), np.int32)
    mask = np.zeros(cap, np.uint32)
    cnt = np.zeros(cap, np.uint64)
    n = ctypes.c_uint64(0)
    _check(lib().cc_table_dump(ctx, run, node, cap, _p(trial), _p(phi), _p(mask), _p(cnt),
                               ctypes.byref(n)), "cc_table_dump")
    m = n.value
    return trial[:m], phi[:m, :bag_size], mask[:m], cnt[:m]


def cc_enumerate(ctx, run: int, limit: int, nF: int):
    out = np.zeros((max(1, limit), nF), np.int32)
    n_out, n_tot = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().cc_enumerate(ctx, run, limit, _p(out), ctypes.byref(n_out), ctypes.byref(n_tot)),
           "cc_enumerate")
    return out[:n_out.value], int(n_tot.value)


def cc_enumerate_sets(ctx, run: int, limit: int, nF: int):
    out = np.zeros((max(1, limit), nF), np.int32)
    n_out, n_tot = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().cc_enumerate_sets(ctx, run, limit, _p(out), ctypes.byref(n_out),
                                   ctypes.byref(n_tot)), "cc_enumerate_sets")
    return out[:n_out.value], int(n_tot.value)


def cc_release(ctx, run: int):
    _check(lib().cc_release(ctx, run), "cc_release")


def cc_run_timings(ctx, run: int, capacity: int = 4096):
    node, kind = np.zeros(capacity, np.int32), np.zeros(capacity, np.int32)
    ms, cand = np.zeros(capacity, np.float32), np.zeros(capacity, np.uint64)
    n = ctypes.c_int32(0)
    _check(lib().cc_run_timings(ctx, run, capacity, _p(node), _p(kind), _p(ms), _p(cand),
                                ctypes.byref(n)), "cc_run_timings")
    m = n.value
    return node[:m], kind[:m], ms[:m], cand[:m]


def cc_autotune(ctx, pid: int, cid: int, base: cc_run_opts | None = None,
                max_schedules: int = 8, repeats: int = 2):
    """(best options, best pattern id, best ms, configurations tried)."""
    best, bp = cc_run_opts(), ctypes.c_int32(0)
    ms, n = ctypes.c_float(0), ctypes.c_int32(0)
    _check(lib().cc_autotune(ctx, pid, cid, ctypes.byref(base) if base is not None else None,
                             max_schedules, repeats, ctypes.byref(best), ctypes.byref(bp),
                             ctypes.byref(ms), ctypes.byref(n)), "cc_autotune")
    return best, bp.value, ms.value, n.value


def cc_solve_trials(nF: int, epsilon: float) -> int:
    return int(lib().cc_solve_trials(nF, epsilon))


def cc_solve(ctx, pid: int, seed: int, k: int, epsilon: float, batch: int, max_trials: int,
             limit: int, nF: int):
    """(found, trials run, embeddings int32[m, nF], estimate)."""
    out = np.zeros((max(1, limit), nF), np.int32)
    n_out, found = ctypes.c_uint64(0), ctypes.c_uint8(0)
    tr, est = ctypes.c_int32(0), ctypes.c_double(0)
    _check(lib().cc_solve(ctx, pid, seed, k, epsilon, batch, max_trials, limit,
                          _p(out) if limit else None, ctypes.byref(n_out), ctypes.byref(found),
                          ctypes.byref(tr), ctypes.byref(est)), "cc_solve")
    return bool(found.value), tr.value, out[:n_out.value], est.value


def cc_run_mode(ctx, run: int) -> str:
    m = ctypes.c_int32(0)
    _check(lib().cc_run_mode(ctx, run, ctypes.byref(m)), "cc_run_mode")
    return RUN_MODES[m.value]


def cc_probe_bounded_wait(ctx, polls: int) -> int:
    """Return code of a bounded device wait made to run out (CC_ETIMEOUT = -4 expected)."""
    return int(lib().cc_probe_bounded_wait(ctx, polls))


def cc_context_stats(ctx):
    a, b, c = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().cc_context_stats(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "cc_context_stats")
    return int(a.value), int(b.value), int(c.value)


def cc_count_noalloc(device: int, stream: int, row_ptr, col, nF: int, edges, td, seed: int,
                     trials: int, k: int):
    """Counts and exists flags computed in the library's fixed device array, allocating no device
    memory (see include/cc.h)."""
    rp, cl = _i32(row_ptr), _i32(col)
    e = _i32(edges).reshape(-1)
    tdp, keep = _td_struct(td)
    counts = np.zeros(trials, np.uint64)
    exists = np.zeros(trials, np.uint8)
    _check(lib().cc_count_noalloc(device, stream or None, len(rp) - 1, _p(rp),
                                  _p(cl) if len(cl) else None, nF, len(e) // 2,
                                  _p(e) if len(e) else None, tdp, seed, trials, k, _p(counts),
                                  _p(exists)), "cc_count_noalloc")
    del keep
    return counts, exists


def cc_serve_start(ctx, mem_budget: int = 0, max_inflight: int = 8):
    _check(lib().cc_serve_start(ctx, mem_budget, max_inflight), "cc_serve_start")


def cc_serve_submit(ctx, pid: int, seed: int, trials: int, k: int, limit: int = 0) -> int:
    t = ctypes.c_int64(0)
    _check(lib().cc_serve_submit(ctx, pid, seed, trials, k, limit, ctypes.byref(t)),
           "cc_serve_submit")
    return t.value


def cc_serve_poll(ctx, ticket: int, trials: int, limit: int = 0, nF: int = 0):
    """(done, status, counts, exists, latency ns, rows int32[n_rows, nF])."""
    done, status, lat = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    counts = np.zeros(trials, np.uint64)
    exists = np.zeros(trials, np.uint8)
    rows = np.zeros((max(1, limit), max(1, nF)), np.int32)
    nrows = ctypes.c_uint64(0)
    _check(lib().cc_serve_poll(ctx, ticket, ctypes.byref(done), ctypes.byref(status), _p(counts),
                               _p(exists), _p(rows) if limit else None, ctypes.byref(nrows),
                               ctypes.byref(lat)), "cc_serve_poll")
    return (bool(done.value), status.value, counts, exists, lat.value,
            rows[:nrows.value, :nF] if limit else rows[:0, :0])


def cc_serve_stats(ctx) -> dict:
    v = [ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_int32(0), ctypes.c_uint64(0),
         ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)]
    _check(lib().cc_serve_stats(ctx, *[ctypes.byref(x) for x in v]), "cc_serve_stats")
    names = ["submitted", "completed", "inflight_max", "reserved_max", "exact_runs", "reruns",
             "sliced"]
    return {k: int(x.value) for k, x in zip(names, v)}


def cc_serve_cancel(ctx) -> int:
    """Drops the queued queries that have not started (status CC_ECANCELED); their number."""
    n = ctypes.c_uint64(0)
    _check(lib().cc_serve_cancel(ctx, ctypes.byref(n)), "cc_serve_cancel")
    return n.value


def cc_serve_stop(ctx):
    _check(lib().cc_serve_stop(ctx), "cc_serve_stop")


class Context:
    """A context whose arena is a PyTorch uint8 tensor and whose stream is torch's current one."""

    def __init__(self, arena_bytes: int = 1 << 30, device: int = 0):
        import torch
        self.device = device
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=f"cuda:{device}")
        self.stream = torch.cuda.current_stream(device)
        self.h = cc_create(device, self.stream.cuda_stream, self.arena.data_ptr(), arena_bytes)

    def close(self):
        if getattr(self, "h", None) is not None:
            cc_destroy(self.h)
            self.h = None
        self.arena = None  # the device memory goes back to PyTorch's allocator

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
