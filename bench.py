"""Benchmark of the colour-coding dynamic programme (arXiv 1908.11248) on one GB300.

Default workload (the largest single-GPU configuration): Erdos-Renyi host graph n=100000,
average degree 10 (seed 1, int32 CSR); pattern the 3x3 grid (9 vertices, treewidth 3); k=9
colours from Philox4x32-10 seed 7; 32 colouring trials in one batched run with options picked by
the library's autotuner; enumeration of the first 10^5 embeddings.  One step = colour all trials,
run every node of the nice decomposition for all trials at once (tables kept for the
reconstruction), test the root, read the per-trial uint64 counts back and enumerate.

Metric: DP entries/s, entries = sum over nodes and trials of |D_x| (distinct table entries; the
same number on the CPU oracle for the same decomposition and flags).

Extra keys of the same JSON line: the Barabasi-Albert n=20000, 2x4 grid, 64-trial workload; the
latency (p50/p99) of one query on Erdos-Renyi n=200 with the 5-cycle; the same 64 trials run
plain (one trial per call), batched (all trials in one call) and as a batch of single-trial
requests replayed from a captured CUDA graph; the serving workload (2000 Poisson queries on a
resident Barabasi-Albert n=200000 graph) against the plain per-query path under the same
arrivals.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (test infrastructure, never the product path) on a
bounded sample of the same workload.  With N > 1 (torchrun) every rank runs an independent
replica with its own colouring seed; rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "DP entries/s"
UNIT = "entries/s"
MAIN = "er100k_grid3x3"
ENUM_LIMIT = 100000


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash():
    """Hash of the library's sources: a DRAM-traffic ratio measured on one build is reported only
    while the sources are unchanged."""
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_1908_11248_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def traffic_ratios(workload, out_dir=None):
    """Measured DRAM bytes per algorithmic byte of each node rule's kernels for `workload`, from
    the committed capture summary of this build (profiles/dram_<workload>.txt: lines
    `ratio <group> <dram bytes> <algorithmic bytes>` and `sources <hash>`); {} if there is none
    or the sources changed since it was taken."""
    path = os.path.join(out_dir or os.path.join(ROOT, "profiles"), f"dram_{workload}.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return {}
    src, out = None, {}
    for ln in lines:
        f = ln.split()
        if len(f) == 2 and f[0] == "sources":
            src = f[1]
        if len(f) == 4 and f[0] == "ratio":
            out[f[1]] = float(f[2]) / float(f[3])
    return out if src == source_hash() else {}


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


T_START = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - T_START:7.1f} s] {msg}", file=sys.stderr, flush=True)


def slot_bytes(b, k):
    """Algorithmic bytes of one table entry: b vertex ids, the colour set and the count."""
    return 4 * b + (2 if k <= 16 else 4) + 8


def algorithmic_bytes(kind, node, nodes, sizes, cand, n, T, k):
    """Bytes a launch must move by the method's definition (not by this implementation): an
    introduce reads its child's entries, one adjacency word and one colour byte per candidate
    examined, and writes its own entries; a forget reads its child's entries and writes its own
    (merging them by sort + reduce, or by hashing, is implementation); a join reads both
    children and writes its entries."""
    ty, c0, c1, u, bag = nodes[node]
    S = lambda x: slot_bytes(len(nodes[x][4]), k)  # noqa: E731
    if kind == "color":
        return T * n
    if kind == "leaf":
        return n * T * (1 + S(node))
    if kind == "intro_chain":  # two introduces in one pass: the lower one's child in, the
        y = nodes[c0][1]         # upper one's entries out (the lower table is never stored)
        return int(sizes[y]) * S(y) + int(cand) * 5 + int(sizes[node]) * S(node)
    if kind in ("intro_count", "intro_write", "intro_fused"):
        b = int(sizes[c0]) * S(c0) + int(cand) * 5
        if kind != "intro_count":  # the introduce's own table, written once
            b += int(sizes[node]) * S(node)
        return b
    if kind in ("forget", "sort", "reduce", "merge"):
        if ty != 2:
            return 0
        # the sort's share of the forget is its whole read of the child's entries; the
        # reduce writes the merged entries
        if kind == "sort":
            return int(sizes[c0]) * S(c0)
        if kind == "reduce":
            return int(sizes[node]) * S(node)
        return int(sizes[c0]) * S(c0) + int(sizes[node]) * S(node)
    if kind.startswith("join"):
        b = (int(sizes[c0]) + int(sizes[c1])) * S(node)
        if kind == "join_write":
            b += int(sizes[node]) * S(node)
        return b
    if kind == "root":
        return int(sizes[node]) * S(node)
    return 0


# kernel kinds grouped by the node rule they implement (Section 3.1)
GROUPS = {"color": "colour", "leaf": "leaf", "intro_count": "introduce",
          "intro_write": "introduce", "intro_chain": "introduce",
          "intro_fused": "introduce+forget", "forget": "forget",
          "sort": "forget", "reduce": "forget", "merge": "forget", "join_build": "join",
          "join_count": "join", "join_write": "join", "root": "root"}


# device kernels (by function name) grouped by the node rule they implement, for the DRAM-traffic
# summary of an ncu capture; kernels of no node rule (graph set-up, enumeration) are "other"
KERNEL_GROUPS = {
    "color_kernel": "colour", "leaf_kernel": "leaf",
    "intro_kernel": "introduce", "intro_warp_kernel": "introduce",
    "intro_group_warp_kernel": "introduce", "nb_colour_hist_kernel": "introduce",
    "sort_hist_kernel": "forget", "row_scan_kernel": "forget", "digit_base_kernel": "forget",
    "sort_scatter_kernel": "forget", "sweep_hist_kernel": "forget",
    "sweep_bases_kernel": "forget", "sweep_pass_kernel": "forget",
    "sweep_pass_wide_kernel": "forget", "sweep_pass_tma_kernel": "forget",
    "reduce_count_kernel": "forget", "blk_scan_kernel": "forget",
    "reduce_write_kernel": "forget", "forget_kernel": "forget", "part_hist_kernel": "forget",
    "part_cursor_kernel": "forget", "part_split_kernel": "forget",
    "part_local_kernel": "forget",
    "join_build_kernel": "join", "join_probe_kernel": "join", "root_kernel": "root",
}


def kernel_base(name):
    """Function name of a kernel as ncu lists it (demangled, with namespaces, template and
    argument lists): the first word ending in _kernel, else the whole name."""
    m = re.search(r"(\w+_kernel)\b", name)
    return m.group(1) if m else name.strip()


def kernel_group(name, fused):
    """Node-rule group of a device kernel named `name` in an ncu listing (demangled names carry
    templates and arguments); introduce kernels count as "introduce+forget" in a fused run."""
    g = KERNEL_GROUPS.get(kernel_base(name), "other")
    if fused and g == "introduce":
        return "introduce+forget"
    return g


def ncu_kernels(csv_path):
    """Per launch of an ncu CSV listing (--csv --log-file): kernel name, DRAM bytes read and
    written and device time in ms (the metrics the listing has; the others 0)."""
    import csv

    rows = list(csv.reader(open(csv_path)))
    head = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    cols = rows[head]
    ci = {c: cols.index(c) for c in ("ID", "Kernel Name", "Metric Name", "Metric Unit",
                                     "Metric Value")}
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1e3, "MB": 1e6,
             "GB": 1e9, "nsecond": 1e-6, "usecond": 1e-3, "msecond": 1.0, "ns": 1e-6,
             "us": 1e-3, "ms": 1.0}
    per = {}
    for r in rows[head + 1:]:
        if len(r) < len(cols):
            continue
        kid, kname, metric = r[ci["ID"]], r[ci["Kernel Name"]], r[ci["Metric Name"]]
        v = float(r[ci["Metric Value"]].replace(",", "")) * scale.get(r[ci["Metric Unit"]], 1)
        d = per.setdefault(kid, {"name": kname, "read": 0.0, "write": 0.0, "ms": 0.0})
        if metric == "dram__bytes_read.sum":
            d["read"] = v
        elif metric == "dram__bytes_write.sum":
            d["write"] = v
        elif metric == "gpu__time_duration.sum":
            d["ms"] = v
    return list(per.values())


def kernel_table(launches, fused=False):
    """Launches summed per kernel function and per node-rule group."""
    by_kernel, by_group = {}, {}
    for d in launches:
        k = by_kernel.setdefault(kernel_base(d["name"]),
                                 {"launches": 0, "read": 0.0, "write": 0.0, "ms": 0.0})
        k["launches"] += 1
        for f in ("read", "write", "ms"):
            k[f] += d[f]
        g = by_group.setdefault(kernel_group(d["name"], fused),
                                {"launches": 0, "dram": 0.0, "ms": 0.0})
        g["launches"] += 1
        g["dram"] += d["read"] + d["write"]
        g["ms"] += d["ms"]
    return by_kernel, by_group


def traffic_summary(csv_path, alg_path, cmd, out_dir=None):
    """profiles/dram_<workload>.txt from an ncu capture of one `--capture` step: DRAM bytes
    (dram__bytes_read.sum + dram__bytes_write.sum) and device time of every kernel of the step,
    summed per node rule, beside the algorithmic bytes the same step's node rules moved (written
    by --capture); the bench scales each group's ratio to its own launches."""
    alg = json.load(open(alg_path))
    fused = "introduce+forget" in alg["groups"]
    by_kernel, by_group = kernel_table(ncu_kernels(csv_path), fused)
    total_ms = sum(g["ms"] for g in by_group.values()) or 1.0
    out = [f"# DRAM traffic per node rule: {alg['workload']}, {alg['trials']} trials, one planned "
           "step (profiled launches)",
           f"# capture: {cmd}",
           f"sources {alg['sources']}",
           f"opts {json.dumps(alg['opts'], sort_keys=True)}",
           "# ratio <group> <DRAM bytes of the step> <algorithmic bytes of the step>"]
    for g, v in sorted(by_group.items(), key=lambda x: -x[1]["ms"]):
        if g in alg["groups"] and alg["groups"][g]["bytes"] > 0:
            out.append(f"ratio {g} {v['dram']:.0f} {alg['groups'][g]['bytes']:.0f}")
    out.append("# group  share-of-kernel-time  DRAM-GB  algorithmic-GB  ms (cold-cache, "
               "serialised under ncu)")
    for g, v in sorted(by_group.items(), key=lambda x: -x[1]["ms"]):
        ab = alg["groups"].get(g, {}).get("bytes", 0) / 1e9
        out.append(f"#   {g:18s} {v['ms'] / total_ms:6.3f} {v['dram'] / 1e9:9.3f} {ab:9.3f} "
                   f"{v['ms']:9.3f}")
    out.append("# kernel  launches  DRAM read GB  DRAM write GB  ms")
    for k, v in sorted(by_kernel.items(), key=lambda x: -x[1]["ms"]):
        out.append(f"#   {k:26s} {v['launches']:5d} {v['read'] / 1e9:9.3f} "
                   f"{v['write'] / 1e9:9.3f} {v['ms']:9.3f}")
    path = os.path.join(out_dir or os.path.join(ROOT, "profiles"), f"dram_{alg['workload']}.txt")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    return path


def launch_summary(csv_path, workload, cmd, out_dir=None, skip_steps=0):
    """profiles/launches_<workload>.txt from an ncu launch list (gpu__time_duration.sum of every
    launch of a bench command): per kernel and per node rule the launches, total device time and
    share, from the (skip_steps + 1)-th colouring launch on (a step starts by colouring: the
    warm-up steps, whose first run of a key is exact, are left out).  Under ncu launches are
    serialised and run cold: the shares compare with the bench's event-timed shares, the
    absolute times do not."""
    launches = ncu_kernels(csv_path)
    colour_at = [i for i, d in enumerate(launches) if kernel_base(d["name"]) == "color_kernel"]
    if skip_steps and len(colour_at) > skip_steps:
        launches = launches[colour_at[skip_steps]:]
    by_kernel, by_group = kernel_table(launches)
    total = sum(v["ms"] for v in by_kernel.values()) or 1.0
    out = [f"# ncu launch list: {workload}", f"# command: {cmd}",
           f"# launches from colouring launch {skip_steps + 1} on (warm-up steps left out): "
           f"{sum(v['launches'] for v in by_kernel.values())} launches, {total:.3f} ms of "
           "device time (serialised, cold caches)",
           "# group  launches  ms  share"]
    for g, v in sorted(by_group.items(), key=lambda x: -x[1]["ms"]):
        out.append(f"{g:18s} {v['launches']:6d} {v['ms']:10.3f} {v['ms'] / total:6.3f}")
    out.append("# kernel  launches  ms  share")
    for k, v in sorted(by_kernel.items(), key=lambda x: -x[1]["ms"]):
        out.append(f"{k:26s} {v['launches']:6d} {v['ms']:10.3f} {v['ms'] / total:6.3f}")
    path = os.path.join(out_dir or os.path.join(ROOT, "profiles"), f"launches_{workload}.txt")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
    return path


def describe(name):
    w = synth.WORKLOADS[name]
    g = w["graph"]
    gd = {"er": lambda s: f"ER n={s[1]} p={s[2]:.6g} seed {s[3]}",
          "ba": lambda s: f"BA n={s[1]} m={s[2]} seed {s[3]}",
          "pl": lambda s: f"power-law n={s[1]} mean degree {s[2]} exponent {s[3]} seed {s[4]}"}
    return {"workload": name, "graph": gd[g[0]](g), "pattern": " ".join(map(str, w["pattern"])),
            "k": w["k"], "trials": w["trials"]}


# ------------------------------------------------------------------------------------------------
# CPU oracle (test infrastructure): bounded samples timed on the host cores
# ------------------------------------------------------------------------------------------------

def _noop(x):
    return x


_JOB = {}


def _init_worker(g, pat, k, allow):
    _JOB.update(g=g, pat=pat, k=k, allow=allow)


def _oracle_one(row):
    """One oracle trial in a spawned worker: (table entries, count) of that colouring."""
    import oracle

    r = oracle.run_dp(_JOB["g"], _JOB["pat"], row[None, :], _JOB["k"], allow=_JOB["allow"])
    return int(r.node_sizes.sum()), int(r.count[0])


def host_cores(mem_per_trial_gb):
    """Worker processes for the oracle: every host core, capped so that the workers' tables fit
    the host memory available now; (workers, cores, cap reason or None)."""
    cores = os.cpu_count() or 1
    avail = None
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                avail = int(ln.split()[1]) * 1024 / 1e9
    except OSError:
        pass
    workers, why = cores, None
    if avail is not None and mem_per_trial_gb > 0:
        fit = max(1, int(0.7 * avail / mem_per_trial_gb))
        if fit < workers:
            workers, why = fit, (f"capped at {fit} workers: {avail:.0f} GB host memory available, "
                                 f"~{mem_per_trial_gb:g} GB per trial")
    return workers, cores, why


def oracle_trials(g, pat, k, rows, allow, workers):
    """The oracle, as it stands, on the colourings `rows` (one trial per task), on `workers`
    spawned processes (spawned: the parent has touched the GPU), the graph and pattern sent once
    per worker.  Returns the per-trial (entries, count) and the wall time of the parallel run
    (workers started and warmed first)."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(workers, initializer=_init_worker,
                                      initargs=(g, pat, k, allow)) as pool:
        pool.map_async(_noop, range(workers)).get(timeout=300)
        t0 = time.perf_counter()
        res = pool.map_async(_oracle_one, list(rows), chunksize=1).get(timeout=1800)
        return res, time.perf_counter() - t0


def slice_allow(n, u, modulus, residue=0):
    """Allowed-mapping masks (Section 3.2, masking unprofitable mappings) that restrict pattern
    vertex u to the host vertices v = residue (mod modulus) and leave every other pattern vertex
    free: the embeddings split by the image of u, so a slice's tables and counts are a bounded
    part of the whole run's."""
    allow = np.full(n, 0xFFFFFFFF, np.uint32)
    off = np.arange(n) % modulus != residue
    allow[off] &= np.uint32(~np.uint32(1 << u) & 0xFFFFFFFF)
    return allow


# sample of each workload the oracle is timed on: (colourings, pattern vertex sliced, modulus,
# GB of host memory per trial)
ORACLE_SAMPLE = {"er100k_grid3x3": (16, 0, 16, 6.0), "ba20k_grid2x4": (16, 0, 1, 2.0),
                 "er200_c5": (1, 0, 1, 0.1)}


def run_reference(args, rank):
    """--impl reference: the CPU oracle, as it stands, on a bounded sample of the workload each
    step (the same colourings and slice as the GPU leg's cpu_baseline), on the host cores."""
    import oracle

    if rank != 0:
        return
    name = args.workload
    w = synth.WORKLOADS[name]
    g = synth.make_graph(w["graph"])
    pat = synth.make_pattern(w["pattern"])
    n, k = len(g[0]) - 1, w["k"]
    ntr, u, mod, gb = ORACLE_SAMPLE[name]
    workers, cores, why = host_cores(gb)
    workers = min(workers, ntr)
    allow = slice_allow(n, u, mod) if mod > 1 else None
    z = oracle.colors(n, w["trials"], k, w["seed"])
    oracle.build()
    times, entries = [], 0
    for s in range(args.warmup + args.steps):
        rows = [z[(s * workers + i) % w["trials"]] for i in range(workers)]
        res, dt = oracle_trials(g, pat, k, rows, allow, workers)
        if s >= args.warmup:
            times.append(dt)
            entries += sum(e for e, _ in res)
    tot = sum(times)
    value = entries / tot
    sample = (f"{workers} of the {w['trials']} trials per step, one per process on {workers} of "
              f"{cores} host cores" + (f", pattern vertex {u} sliced to 1/{mod} of the host "
                                       "vertices" if mod > 1 else "") + ", std::map oracle"
              + (f"; {why}" if why else ""))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": dict(describe(name), trials_per_step=workers, l2="n/a (host)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": sample, "host_cores": cores},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
# GPU legs
# ------------------------------------------------------------------------------------------------

def rank_seed(seed, rank):
    """Colouring seed of a replica: every rank colours its own independent trials."""
    return seed + 1000003 * rank


def over_ranks(dist, torch, total_ms, entries, device):
    """Whole-job figures of the replicas: the slowest rank's time (max) and all ranks' entries
    (sum); dist None is one process."""
    if not dist:
        return float(total_ms), float(entries)
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([entries], device=device, dtype=torch.float64)
    dist.all_reduce(e)
    return float(t.item()), float(e.item())


def pct(xs, q):
    """q-th percentile (nearest rank) of a nonempty list."""
    xs = sorted(xs)
    return xs[min(len(xs) - 1, max(0, int(np.ceil(q / 100.0 * len(xs))) - 1))]


def roofline(kern, steps, workload):
    """Roofline of the dominant node rule (largest share of device time): its algorithmic bytes
    over its event-timed duration against the measured HBM copy bandwidth; traffic = the
    measured DRAM-bytes ratio of that group (committed capture of this build) times its
    algorithmic bytes per launch, or null."""
    grp = {}
    for kn, v in kern.items():
        g2 = grp.setdefault(GROUPS.get(kn, kn), {"launches": 0, "ms": 0.0, "bytes": 0})
        for f in ("launches", "ms", "bytes"):
            g2[f] += v[f]
    dom = max(grp, key=lambda x: grp[x]["ms"])
    d = grp[dom]
    achieved = d["bytes"] / (d["ms"] / 1000.0) / 1e9
    peak, peak_kind = peaks()
    ratios = traffic_ratios(workload)
    total_kms = sum(x["ms"] for x in kern.values())
    bpl = d["bytes"] / d["launches"]
    return {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
            "peak_source": peak_kind, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ratios[dom] * bpl if dom in ratios else None,
            "bytes_per_launch": bpl, "ms_per_launch": d["ms"] / d["launches"],
            "groups": {g: {"ms_per_step": v["ms"] / steps, "share": v["ms"] / total_kms,
                           "launches_per_step": v["launches"] / steps,
                           "gbs": v["bytes"] / (v["ms"] / 1000.0) / 1e9 if v["ms"] else None,
                           "frac": (v["bytes"] / (v["ms"] / 1000.0) / 1e9 / peak
                                    if v["ms"] else None),
                           "traffic_per_launch": (ratios[g] * v["bytes"] / v["launches"]
                                                  if g in ratios else None)}
                       for g, v in sorted(grp.items(), key=lambda x: -x[1]["ms"])},
            "kernels": {kn: {"launches": v["launches"] // steps, "ms_per_step": v["ms"] / steps,
                             "share": v["ms"] / total_kms}
                        for kn, v in sorted(kern.items(), key=lambda x: -x[1]["ms"])}}


def dp_leg(cc, torch, name, args, rank, dist, tune=True, enum_limit=0, sampler=None,
           capture=None):
    """The DP of workload `name` on one context: (optionally) autotune, W untimed warm-up steps,
    K timed steps (colour, DP with profiled launches, counts back, enumerate), then the same
    steps end to end through the C ABI with the graph copied from pinned host memory."""
    w = synth.WORKLOADS[name]
    g = synth.make_graph(w["graph"])
    nF, edges, td = synth.make_pattern(w["pattern"])
    n = len(g[0]) - 1
    T, k = (args.trials or w["trials"]) if name == args.workload else w["trials"], w["k"]
    seed = rank_seed(w["seed"], rank)
    ctx = cc.Context(arena_bytes=args.arena_gb << 30, device=torch.cuda.current_device())
    h = ctx.h
    cc.cc_load_graph(h, *g)
    pid = cc.cc_load_pattern(h, nF, edges, td)
    out = {"config": describe(name)}
    out["config"]["trials"] = T
    tuned = cc.cc_default_opts(**(json.loads(args.opts) if args.opts else {}))
    if tune and not args.opts:
        cid = cc.cc_color(h, seed, T, k)
        t0 = time.perf_counter()
        pid0 = pid
        log(f"{name}: autotuning")
        tuned, pid, best_ms, tried = cc.cc_autotune(h, pid, cid, None, 6, 2)
        log(f"{name}: autotuned ({tried} configurations, best {best_ms:.1f} ms)")
        out["autotune"] = {"configs_tried": tried, "best_ms": best_ms,
                           "seconds": time.perf_counter() - t0,
                           "schedule": "re-rooted" if pid != pid0 else "as given"}
        cc.cc_release_colors(h, cid)
    out["config"]["opts"] = {f: getattr(tuned, f) for f, _ in tuned._fields_}
    nodes = cc.cc_pattern_nodes(h, pid, nF)
    opts = cc.cc_run_opts.from_buffer_copy(tuned)
    opts.profile = 1
    opts.retain = 1 if enum_limit else 0
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step(o):
        cid = cc.cc_color(h, seed, T, k)
        run = cc.cc_run_dp(h, pid, cid, o)
        counts = cc.cc_count(h, run, T)
        rows = cc.cc_enumerate(h, run, enum_limit, nF)[0] if enum_limit else None
        return cid, run, counts, rows

    for _ in range(max(args.warmup, 1 if capture else 0)):  # a capture's step is planned
        cid, run, counts, rows = step(opts)
        cc.cc_release(h, run)
        cc.cc_release_colors(h, cid)
    torch.cuda.synchronize()
    if capture:  # one planned step inside the profiler range, for an ncu capture
        torch.cuda.profiler.start()
        cid, run, counts, rows = step(opts)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        sizes, total = cc.cc_table_stats(h, run, len(nodes))
        node, kind, ms, cand = cc.cc_run_timings(h, run)
        groups = {}
        for i in range(len(node)):
            kn = cc.KERNEL_KINDS[int(kind[i])]
            g2 = groups.setdefault(GROUPS.get(kn, kn), {"launches": 0, "bytes": 0})
            g2["launches"] += 1
            g2["bytes"] += algorithmic_bytes(kn, int(node[i]), nodes, sizes, cand[i], n, T, k)
        with open(capture, "w") as f:
            json.dump({"workload": name, "trials": T, "sources": source_hash(),
                       "opts": out["config"]["opts"], "entries": int(total),
                       "groups": groups}, f)
        ctx.close()
        return None
    if dist:
        dist.barrier()
    if sampler:
        sampler.start()
    log(f"{name}: warm-up done, timing {args.steps} steps")
    launches0 = cc.cc_context_stats(h)[0]
    step_ms, entries, kern, modes = [], 0, {}, set()
    for _ in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (256 MB > 129 MB L2)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        cid, run, counts, rows = step(opts)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        sizes, total = cc.cc_table_stats(h, run, len(nodes))
        entries += total
        modes.add(cc.cc_run_mode(h, run))
        node, kind, ms, cand = cc.cc_run_timings(h, run)
        for i in range(len(node)):
            kn = cc.KERNEL_KINDS[int(kind[i])]
            d = kern.setdefault(kn, {"launches": 0, "ms": 0.0, "bytes": 0})
            d["launches"] += 1
            d["ms"] += float(ms[i])
            d["bytes"] += algorithmic_bytes(kn, int(node[i]), nodes, sizes, cand[i], n, T, k)
        cc.cc_release(h, run)
        cc.cc_release_colors(h, cid)
    torch.cuda.synchronize()
    launches = cc.cc_context_stats(h)[0] - launches0
    clocks = sampler.stop() if sampler else None
    total_ms, entries_all = over_ranks(dist, torch, sum(step_ms), entries, "cuda")
    out.update({
        "value": entries_all / (total_ms / 1000.0), "ms_per_step": total_ms / args.steps,
        "entries_per_step": int(entries / args.steps), "gpu_launches": launches,
        "run_modes": sorted(modes), "roofline": roofline(kern, args.steps, name),
        "counts": [int(c) for c in counts], "clocks": clocks,
        "max_table_entries": int(max(sizes)),
    })
    if enum_limit:
        out["enumerated_rows"] = int(len(rows))

    log(f"{name}: timed steps done ({sum(step_ms) / args.steps:.1f} ms per step)")
    # end to end through the C ABI: graph from pinned host memory, counts (and rows) back
    if rank == 0:
        rp_h = torch.from_numpy(np.asarray(g[0], np.int32)).pin_memory().numpy()
        col_h = torch.from_numpy(np.asarray(g[1], np.int32)).pin_memory().numpy()
        e_opts = cc.cc_run_opts.from_buffer_copy(tuned)
        e_opts.retain = 1 if enum_limit else 0
        e2e_t, e2e_ent, d2h = [], 0, 0
        for _ in range(max(2, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cc.cc_load_graph(h, rp_h, col_h)
            cid, run, c2, rows2 = step(e_opts)
            e2e_t.append(time.perf_counter() - t0)
            assert np.array_equal(c2, counts), "end-to-end counts differ from the timed steps"
            d2h = T * 8 + (int(rows2.nbytes) if rows2 is not None else 0)
            e2e_ent += cc.cc_table_stats(h, run, len(nodes))[1]
            cc.cc_release(h, run)
            cc.cc_release_colors(h, cid)
        out["e2e"] = {"value": e2e_ent / sum(e2e_t), "unit": UNIT,
                      "h2d_bytes_per_step": int(rp_h.nbytes + col_h.nbytes),
                      "d2h_bytes_per_step": int(d2h)}
    out["_ctx"] = (ctx, pid, tuned, g, (nF, edges, td), seed, T, k)
    return out


def cpu_baseline(cc, name, leg, gpu_counts):
    """The oracle, as it stands, on a bounded sample of the workload: trials 0..C-1 (C = the
    host-core count, capped by host memory), one per spawned process, and trial 0 alone on one
    core; for config-3-sized graphs one pattern vertex is restricted to a slice of the host
    vertices (allowed-mapping masks), and the GPU runs the same sliced pattern so that every
    sampled count is checked against it."""
    import oracle

    ctx, pid, tuned, g, pat, seed, T, k = leg["_ctx"]
    h = ctx.h
    n = len(g[0]) - 1
    ntr, u, mod, gb = ORACLE_SAMPLE[name]
    workers, cores, why = host_cores(gb)
    workers = min(workers, ntr, T)
    allow = slice_allow(n, u, mod) if mod > 1 else None
    if allow is not None:  # the GPU's counts for the same sliced pattern
        spid = cc.cc_load_pattern_masked(h, pat[0], pat[1], pat[2], allow)
        cid = cc.cc_color(h, seed, T, k)
        run = cc.cc_run_dp(h, spid, cid, cc.cc_default_opts())
        want = cc.cc_count(h, run, T)
        cc.cc_release(h, run)
        cc.cc_release_colors(h, cid)
    else:
        want = gpu_counts
    z = oracle.colors(n, workers, k, seed)
    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.run_dp(g, pat, z[:1], k, allow=allow)
    dt = time.perf_counter() - t0
    assert int(ref.count[0]) == int(want[0]), "oracle and GPU disagree on trial 0"
    slice_txt = (f", pattern vertex {u} sliced to the host vertices = 0 mod {mod}"
                 if mod > 1 else "")
    single = {"value": float(ref.node_sizes.sum()) / dt, "unit": UNIT, "cores": 1,
              "kind": "oracle",
              "sample": f"trial 0 of the {T}{slice_txt}, single-threaded std::map oracle, "
                        f"{dt:.1f} s"}
    if workers < 2:
        return dict(single, host_cores=cores)
    res, wall = oracle_trials(g, pat, k, [z[t] for t in range(workers)], allow, workers)
    assert all(int(c) == int(want[t]) for t, (_, c) in enumerate(res)), "oracle and GPU disagree"
    return {"value": sum(e for e, _ in res) / wall, "unit": UNIT, "cores": workers,
            "kind": "oracle", "host_cores": cores,
            "sample": f"trials 0..{workers - 1} of the {T}{slice_txt}, one per process on "
                      f"{workers} of {cores} host cores, std::map oracle, {wall:.1f} s"
                      + (f"; {why}" if why else ""),
            "counts_checked": workers, "single_core": single}


def latency_leg(cc, torch, reps=50):
    """One query of the 1-trial workload (Erdos-Renyi n=200, 5-cycle, k=5): colour, DP with its
    tables kept, counts back and every embedding reconstructed, sorted and copied back; p50/p99
    of the host wall time over `reps` queries after a planning run."""
    w = synth.WORKLOADS["er200_c5"]
    g = synth.make_graph(w["graph"])
    nF, edges, td = synth.make_pattern(w["pattern"])
    with cc.Context(arena_bytes=1 << 30) as ctx:
        h = ctx.h
        cc.cc_load_graph(h, *g)
        pid = cc.cc_load_pattern(h, nF, edges, td)
        opts = cc.cc_default_opts(retain=1)
        lat, rows = [], None
        for i in range(reps + 3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cid = cc.cc_color(h, w["seed"], 1, w["k"])
            run = cc.cc_run_dp(h, pid, cid, opts)
            counts = cc.cc_count(h, run, 1)
            rows, tot = cc.cc_enumerate(h, run, 1 << 20, nF)
            dt = (time.perf_counter() - t0) * 1e3
            cc.cc_release(h, run)
            cc.cc_release_colors(h, cid)
            if i >= 3:
                lat.append(dt)
    return {"workload": "er200_c5", "query": "colour 1 trial, DP (tables kept), count, "
            "enumerate all embeddings sorted", "reps": reps, "p50_ms": pct(lat, 50),
            "p99_ms": pct(lat, 99), "count": int(counts[0]), "rows": int(len(rows))}


def batching_leg(cc, torch, name="ba20k_grid2x4"):
    """The same colourings three ways: plain (one trial per cc_run_dp call, no graph), batched
    (all trials in the key of one cc_run_dp call, planned launches) and graph-batched (the
    single-trial requests as parallel branches of one captured CUDA graph, cc_run_batch with
    use_graph); entries/s of each over the whole set, counts compared bit for bit."""
    w = synth.WORKLOADS[name]
    g = synth.make_graph(w["graph"])
    nF, edges, td = synth.make_pattern(w["pattern"])
    T, k = w["trials"], w["k"]
    res = {"workload": name, "trials": T}
    with cc.Context(arena_bytes=96 << 30) as ctx:
        h = ctx.h
        cc.cc_load_graph(h, *g)
        pid = cc.cc_load_pattern(h, nF, edges, td)
        N = len(cc.cc_pattern_nodes(h, pid, nF))
        cid_all = cc.cc_color(h, w["seed"], T, k)
        z = cc.cc_get_colors(h, cid_all, T, len(g[0]) - 1)
        singles = [cc.cc_set_colors(h, z[t], k) for t in range(T)]
        plain_o = cc.cc_default_opts()
        graph_o = cc.cc_default_opts(use_graph=1)

        def timed(fn, reps=3):
            fn()  # plans every key (and captures the graph)
            best = None
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                out = fn()
                dt = time.perf_counter() - t0
                if best is None or dt < best[0]:
                    best = (dt, out)
            return best

        def plain():
            c, e = [], 0
            for cid in singles:
                r = cc.cc_run_dp(h, pid, cid, plain_o)
                c.append(int(cc.cc_count(h, r, 1)[0]))
                e += cc.cc_table_stats(h, r, N)[1]
                cc.cc_release(h, r)
            return c, e

        def batched():
            r = cc.cc_run_dp(h, pid, cid_all, plain_o)
            c = [int(x) for x in cc.cc_count(h, r, T)]
            e = cc.cc_table_stats(h, r, N)[1]
            cc.cc_release(h, r)
            return c, e

        def graphed():
            rs = cc.cc_run_batch(h, [pid] * T, singles, graph_o)
            c, e = [], 0
            for r in rs:
                c.append(int(cc.cc_count(h, r, 1)[0]))
                e += cc.cc_table_stats(h, r, N)[1]
                mode = cc.cc_run_mode(h, r)
                cc.cc_release(h, r)
            return c, e, mode

        for label, fn in (("plain", plain), ("batched", batched), ("graph_batched", graphed)):
            dt, out = timed(fn)
            res[label] = {"entries_per_s": out[1] / dt, "seconds": dt, "entries": out[1]}
            res[label]["_counts"] = out[0]
            if label == "graph_batched":
                res[label]["run_mode"] = out[2]
        # idle time of a graph replay: one all-trials request replayed from its captured graph
        # (CUDA events around the replay) against the summed device time of the same kernels
        # (a profiled run: events around every launch)
        stream = torch.cuda.current_stream()
        prof = cc.cc_run_dp(h, pid, cid_all, cc.cc_default_opts(profile=1))
        ksum = float(cc.cc_run_timings(h, prof)[2].sum())
        cc.cc_release(h, prof)
        go = cc.cc_default_opts(use_graph=1)
        reps, gms, mode = 5, [], None
        for i in range(reps + 2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            r = cc.cc_run_dp(h, pid, cid_all, go)
            e1.record(stream)
            e1.synchronize()
            mode = cc.cc_run_mode(h, r)
            cc.cc_release(h, r)
            if i >= 2:
                gms.append(e0.elapsed_time(e1))
        res["graph_replay"] = {"run_mode": mode, "replay_ms": min(gms), "kernel_ms": ksum,
                               "idle_fraction": max(0.0, 1.0 - ksum / min(gms))}
    ref = res["plain"].pop("_counts")
    res["identical"] = all(res[x].pop("_counts") == ref for x in ("batched", "graph_batched"))
    res["note"] = ("entries/s = table entries of all trials / host wall time of the calls (counts "
                   "and sizes read back); plain: one cc_run_dp per trial; batched: one cc_run_dp "
                   "over all trials; graph_batched: cc_run_batch of the single-trial requests "
                   "replayed from a captured CUDA graph; best of 3 after a planning pass")
    return res


def tree_hom_counts(row_ptr, col, t):
    """Injective homomorphism counts into G[V_t], the subgraph of G induced by the vertices of
    degree >= t (every map into it passes a degree filter of at most t), of the forests on at
    most four vertices, keyed by (vertices, edges, sorted vertex degrees); exact except the
    4-vertex path, a lower bound (its maps with a = d are at most min(d_b, d_c) - 1 per middle
    edge)."""
    rp = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    n = len(rp) - 1
    deg = np.diff(rp)
    src = np.repeat(np.arange(n), deg)
    keep = deg >= t
    m = keep[src] & keep[col]
    s2, c2 = src[m], col[m]
    d = np.bincount(s2, minlength=n).astype(np.float64)
    nv = float(keep.sum())
    m2 = float(len(s2))  # ordered edges = 2m'
    p3 = float((d * (d - 1)).sum())
    return {
        (1, 0, (0,)): nv,
        (2, 0, (0, 0)): nv * (nv - 1),
        (2, 1, (1, 1)): m2,
        (3, 1, (0, 1, 1)): m2 * (nv - 2),
        (3, 2, (1, 1, 2)): p3,
        (4, 2, (0, 1, 1, 2)): p3 * (nv - 3),
        (4, 2, (1, 1, 1, 1)): m2 * m2 - 4.0 * float((d * d).sum()) + 2.0 * m2,
        (4, 3, (1, 1, 1, 3)): float((d * (d - 1) * (d - 2)).sum()),
        (4, 3, (1, 1, 2, 2)): float(((d[s2] - 1) * (d[c2] - 1)).sum()
                                    - np.maximum(np.minimum(d[s2], d[c2]) - 1, 0).sum()),
    }


def pl_bound_leg(cc, hbm_bytes):
    """The batched power-law configuration (n = 10^6, 64 random partial 3-trees of 10-12
    vertices, k = n_F, 16 trials each) against one GPU's memory, on the host: for every pattern,
    the library's nice decomposition; a node whose subtree holds only a leaf and introduces has
    V*_x = V_x, so its table holds one entry per trial and colourful injective map of F[V_x]
    (Section 2.1, table semantics): in expectation T * inj(F[V_x], G) * k!/((k-b)! k^b).  For
    the forest-shaped F[V_x] the count is taken in G[V_t] (t the largest F-degree in the bag, so
    the degree filter of Section 3.2 keeps every such map), a lower bound on the table; times the
    entry size 4b + 2 + 8 bytes it is compared with the GPU's memory.  Patterns whose pure nodes
    all contain a cycle get no bound here."""
    w = synth.WORKLOADS["pl1m_ktree3"]
    g = synth.make_graph(w["graph"])
    T = w["trials"]
    counts = {}
    out, proven = [], 0
    for i, (nF, edges, td) in enumerate(synth.ktree_batch(w)):
        nodes, width = cc.cc_nice_decomposition(nF, edges, td)
        adj = [set() for _ in range(nF)]
        for a, b in np.asarray(edges).reshape(-1, 2).tolist():
            adj[a].add(b)
            adj[b].add(a)
        pure, best = [False] * len(nodes), None
        for x, (ty, c0, _, _, bag) in enumerate(nodes):
            pure[x] = ty == 0 or (ty == 1 and pure[c0])
            if not pure[x]:
                continue
            b = len(bag)
            e = sum(1 for a in bag for c in bag if a < c and c in adj[a])
            shape = (b, e, tuple(sorted(sum(1 for c in bag if c in adj[a]) for a in bag)))
            t = max(len(adj[u]) for u in bag)
            if t not in counts:
                counts[t] = tree_hom_counts(g[0], g[1], t)
            if shape not in counts[t]:
                continue
            falling = float(np.prod([nF - j for j in range(b)])) / float(nF) ** b
            ent = T * counts[t][shape] * falling
            byt = ent * slot_bytes(b, nF)
            if best is None or byt > best["bytes"]:
                best = {"pattern": i, "n_F": nF, "width": width, "node": x, "bag": b,
                        "edges": e, "degree_threshold": t, "entries": ent, "bytes": byt}
        if best is None:
            out.append({"pattern": i, "n_F": nF, "bound": None})
            continue
        best["exceeds_gpu_memory"] = bool(best["bytes"] > hbm_bytes)
        proven += best["exceeds_gpu_memory"]
        out.append(best)
    return {"workload": "pl1m_ktree3", "trials": T, "gpu_memory_bytes": hbm_bytes,
            "patterns": len(out), "with_forest_bound": sum(1 for o in out if "bytes" in o),
            "proven_too_large": int(proven), "per_pattern": out,
            "note": "expected entries of one table (a node whose subtree is a leaf and "
                    "introduces) counted in the subgraph of vertices of degree >= the bag's "
                    "largest F-degree: a lower bound on the DP's memory for the library's "
                    "decomposition of each pattern"}


def hash_leg(cc, torch):
    """The hashed node rules, event-timed: `ba20k_grid2x4` (64 trials) with every introduce
    adding its projected entries into its forget's open-addressing hash table (fuse 1: one
    compare-and-swap to claim a key, one atomic add of the count, per entry), and pattern A of
    Fig. 1 (three joins: hash join on the shared bag map) on the same graph with 16 trials, k =
    n_F.  Reports each group's time and entries per second: for the hashed forget, entries
    inserted (= atomic updates) per second."""
    w = synth.WORKLOADS["ba20k_grid2x4"]
    g = synth.make_graph(w["graph"])
    out = {"graph": "BA n=20000 m=4 seed 1"}
    with cc.Context(arena_bytes=64 << 30) as ctx:
        h = ctx.h
        cc.cc_load_graph(h, *g)
        for label, pat, T, k, opts in (
                ("forget_hashed", synth.make_pattern(w["pattern"]), w["trials"], w["k"],
                 dict(fuse=1)),
                ("join", synth.make_pattern(("A",)), 16, 9, {})):
            pid = cc.cc_load_pattern(h, *pat)
            N, _ = cc.cc_pattern_info(h, pid)
            cid = cc.cc_color(h, w["seed"], T, k)
            kinds = {}
            for rep in range(3):  # exact, then planned runs
                run = cc.cc_run_dp(h, pid, cid, cc.cc_default_opts(profile=1, **opts))
                sizes = cc.cc_table_stats(h, run, N)[0]
                if rep == 2:
                    node, kind, ms, _ = cc.cc_run_timings(h, run)
                    for i in range(len(node)):
                        kn = cc.KERNEL_KINDS[int(kind[i])]
                        x = int(node[i])
                        d = kinds.setdefault(kn, {"launches": 0, "ms": 0.0, "entries": 0})
                        d["launches"] += 1
                        d["ms"] += float(ms[i])
                        # entries a launch handles: an introduce's own entries (each inserted
                        # into the forget's hash table when fused); a join's output entries
                        d["entries"] += int(sizes[x])
                    mode = cc.cc_run_mode(h, run)
                cc.cc_release(h, run)
            cc.cc_release_colors(h, cid)
            for d in kinds.values():
                d["entries_per_s"] = d["entries"] / (d["ms"] / 1e3) if d["ms"] else None
            out[label] = {"pattern": "grid 2 4" if label == "forget_hashed" else "A (Fig. 1)",
                          "trials": T, "k": k, "run_mode": mode, "kinds": kinds,
                          "entries_per_step": int(sizes.sum())}
    out["note"] = ("event-timed planned runs; intro_fused = introduce whose entries are inserted "
                   "into the forget's hash table (entries_per_s = hash inserts per second, one "
                   "claim and one atomic count update each); join_* = hash join build and "
                   "probe/write (entries_per_s = join output entries per second)")
    return out


def er_phase_point(cc, h, pat, k, seed, trials):
    """One point of the Erdos-Renyi study on the loaded target: load the pattern (minimum-width
    decomposition), colour `trials` times, run the DP over all colourings at once and decide.
    Returns (status, width, any colourful copy, per-trial counts or None, table entries)."""
    nF, edges, td = pat
    pid = cc.cc_load_pattern(h, nF, edges, td)
    width = cc.cc_pattern_info(h, pid)[1]
    cid = cc.cc_color(h, seed, trials, k)
    try:  # a point whose tables do not fit is reported, not split into slices
        run = cc.cc_run_dp(h, pid, cid, cc.cc_default_opts(max_slices=1))
    except cc.CCError as ex:
        cc.cc_release_colors(h, cid)
        return ex.code, width, None, None, 0
    counts = cc.cc_count(h, run, trials)
    found = bool(cc.cc_decide(h, run, trials).any())
    N = cc.cc_pattern_info(h, pid)[0]
    ent = cc.cc_table_stats(h, run, N)[1]
    cc.cc_release(h, run)
    cc.cc_release_colors(h, cid)
    return 0, width, found, counts, ent


def er_phase_leg(cc, torch, step=None, arena_gb=8):
    """The Erdos-Renyi phase-transition study (Section 5.4): for every p, q on the grid of the
    study, target G(150, p) against pattern G(10, q), ten colourings (iterations) with k = 10;
    per point the time of the ten iterations, whether a copy was found, the pattern's
    decomposition width and the status (0, or CC_ENOMEM / CC_EKEYWIDTH where the tables do not
    fit the arena or the width exceeds what the kernels take: the paper's time-outs)."""
    spec = dict(synth.ER_PHASE)
    if step:
        spec["step"] = step
    probs = synth.er_phase_probs(spec["step"])
    P = len(probs)
    ms = np.zeros((P, P))
    found = np.zeros((P, P), np.int8)
    width = np.zeros((P, P), np.int8)
    status = np.zeros((P, P), np.int8)
    entries = 0
    t_all = time.perf_counter()
    with cc.Context(arena_bytes=arena_gb << 30) as ctx:
        h = ctx.h
        for ip in range(P):
            for iq in range(P):
                p, q, g, pat, seed = synth.er_phase_instance(ip, iq, spec)
                if iq == 0:
                    cc.cc_load_graph(h, *g)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, w, f, _, ent = er_phase_point(cc, h, pat, spec["n_pattern"], seed,
                                                 spec["iterations"])
                ms[ip, iq] = (time.perf_counter() - t0) * 1e3
                status[ip, iq], width[ip, iq], found[ip, iq] = st, w, 1 if f else 0
                entries += ent
            log(f"er_phase: row p={probs[ip]:.2f} done ({ms[ip].sum() / 1e3:.1f} s, "
                f"max point {ms[ip].max() / 1e3:.2f} s)")
    ok = status == 0
    return {
        "workload": "er_phase", "target": f"G({spec['n_target']}, p)",
        "pattern": f"G({spec['n_pattern']}, q)", "iterations": spec["iterations"],
        "probs": probs, "points": P * P, "seconds": time.perf_counter() - t_all,
        "completed": int(ok.sum()), "enomem": int((status == -2).sum()),
        "width_limit": int((status == -7).sum()), "found": int(found.sum()),
        "entries": int(entries),
        # rows p, columns q
        "ms": np.round(ms, 2).tolist(), "found_grid": found.tolist(),
        "status_grid": status.tolist(),
        "width_vs_q": [float(np.mean(width[:, j])) for j in range(P)],
        "note": "per point: load the pattern (minimum-width decomposition), colour ten times, one "
                "DP over the ten colourings, decide; ms = host wall time of those calls",
    }


def serve_leg(cc, torch, count, arena_gb, budget_gb, slots, window_s):
    """Serving workload: the first `count` queries of the seeded Poisson stream over the resident
    BA n=200000 m=5 graph.  Every (pattern, trials, k) of the stream is first run once, unsplit
    (untimed): keys that fit the budget are planned ("light"); keys whose single trial does not
    fit ("heavy": they run in slices, seconds to minutes each on this graph) are counted and
    left out of the timed legs.  The light queries are then submitted at their arrival times to
    the library's server for `window_s` seconds (queries not started by then are cancelled), and
    run through the plain path (cc_color, cc_run_dp, cc_count, one query at a time, no server)
    under the same arrivals for the same time; queries both legs completed are compared bit for
    bit."""
    w = synth.WORKLOADS["serve_ba200k"]
    g = synth.make_graph(w["graph"])
    stream = synth.serve_stream(w, count)
    torch.cuda.empty_cache()
    ctx = cc.Context(arena_bytes=arena_gb << 30)
    h = ctx.h
    cc.cc_load_graph(h, *g)
    pids = {}
    for q in stream:
        if q["pattern"] not in pids:
            pids[q["pattern"]] = cc.cc_load_pattern(h, *synth.make_pattern(q["pattern"]))
    # classify (and plan) every key with one unsplit run of a colouring the stream does not use
    light, t_cls = set(), time.perf_counter()
    keys = {}
    for q in stream:
        keys.setdefault((q["pattern"], q["trials"], q["k"]), q)
    for key, q in keys.items():
        cid = cc.cc_color(h, q["seed"] ^ 0x5A5A, q["trials"], q["k"])
        try:
            run = cc.cc_run_dp(h, pids[q["pattern"]], cid, cc.cc_default_opts(max_slices=1))
            cc.cc_count(h, run, q["trials"])
            cc.cc_release(h, run)
            light.add(key)
        except cc.CCError as ex:
            if ex.code != cc.CC_ENOMEM:
                raise
        cc.cc_release_colors(h, cid)
    t_cls = time.perf_counter() - t_cls
    lq = [q for q in stream if (q["pattern"], q["trials"], q["k"]) in light]
    n_heavy = len(stream) - len(lq)
    log(f"serving: {len(light)} of {len(keys)} keys fit unsplit ({t_cls:.1f} s); "
        f"{len(lq)} light queries, {n_heavy} heavy; served leg")

    def poll(t, trials):
        return cc.cc_serve_poll(h, t, trials)

    cc.cc_serve_start(h, budget_gb << 30, slots)
    t0 = time.perf_counter()
    tickets, res = [], {}
    for q in lq:
        dt = t0 + q["t"] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(cc.cc_serve_submit(h, pids[q["pattern"]], q["seed"], q["trials"], q["k"]))
    while len(res) < len(tickets) and time.perf_counter() - t0 < window_s:
        for i, t in enumerate(tickets):
            if i not in res:
                done, status, counts, _, lat, _ = poll(t, lq[i]["trials"])
                if done:
                    res[i] = (status, counts, lat, time.perf_counter() - t0)
        time.sleep(0.0005)
    cancelled = cc.cc_serve_cancel(h)
    while len(res) < len(tickets):  # the running queries finish
        for i, t in enumerate(tickets):
            if i not in res:
                done, status, counts, _, lat, _ = poll(t, lq[i]["trials"])
                if done:
                    res[i] = (status, counts, lat, time.perf_counter() - t0)
        time.sleep(0.0005)
    stats = cc.cc_serve_stats(h)
    cc.cc_serve_stop(h)
    ok = [i for i in range(len(lq)) if res[i][0] == 0]
    lat_ms = [res[i][2] / 1e6 for i in ok]
    span = max([res[i][3] for i in ok] + [1e-9])
    log(f"serving: served {len(ok)} in {span:.1f} s; plain leg")
    # plain path under the same arrivals, measured: query i starts at max(arrival, previous end)
    plain_lat, plain_ms, same, plain_done = [], [], True, 0
    t0 = time.perf_counter()
    for i, q in enumerate(lq):
        dt = t0 + q["t"] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        if time.perf_counter() - t0 >= window_s:
            break
        t1 = time.perf_counter()
        cid = cc.cc_color(h, q["seed"], q["trials"], q["k"])
        run = cc.cc_run_dp(h, pids[q["pattern"]], cid, cc.cc_default_opts())
        counts = cc.cc_count(h, run, q["trials"])
        t2 = time.perf_counter()
        plain_ms.append((t2 - t1) * 1e3)
        plain_lat.append((t2 - (t0 + q["t"])) * 1e3)
        plain_done += 1
        if i in res and res[i][0] == 0:
            same = same and bool(np.array_equal(counts, res[i][1]))
        cc.cc_release(h, run)
        cc.cc_release_colors(h, cid)
    plain_span = time.perf_counter() - t0
    ctx.close()
    del ctx
    torch.cuda.empty_cache()
    return {
        "workload": "serve_ba200k", "graph": "BA n=200000 m=5 seed 1",
        "queries": len(stream), "offered_rate_qps": w["rate"],
        "arrivals_s": stream[-1]["t"], "slots": slots, "budget_gb": budget_gb,
        "keys": len(keys), "light_keys": len(light), "light_queries": len(lq),
        "heavy_queries": n_heavy, "classify_s": t_cls, "window_s": window_s,
        "served": {"completed": len(ok), "cancelled": int(cancelled),
                   "failed": len(lq) - len(ok) - sum(1 for i in res if res[i][0] == -9),
                   "qps": len(ok) / span, "p50_ms": pct(lat_ms, 50) if lat_ms else None,
                   "p99_ms": pct(lat_ms, 99) if lat_ms else None, "span_s": span},
        "plain": {"completed": plain_done, "qps": plain_done / plain_span,
                  "p50_ms": pct(plain_lat, 50) if plain_lat else None,
                  "p99_ms": pct(plain_lat, 99) if plain_lat else None,
                  "service_p50_ms": pct(plain_ms, 50) if plain_ms else None,
                  "service_p99_ms": pct(plain_ms, 99) if plain_ms else None,
                  "span_s": plain_span},
        "identical": same, "server": stats,
        "note": "light queries (keys whose single trial fits the budget unsplit, planned by one "
                "untimed run each) submitted at their arrival times; each leg runs for the "
                "window (the server's unstarted queries are then cancelled, the plain loop "
                "starts no more); latency from arrival to completion, queueing included (the "
                "offered rate is far above either path's capacity); heavy queries (their "
                "tables need splitting into slices) are counted, not timed here",
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=MAIN, choices=sorted(ORACLE_SAMPLE),
                    help="workload of the bench line")
    ap.add_argument("--legs", default="ba20k,latency,batching,hash,serve,er_phase,pl_bound",
                    help="extra keys to measure (comma list of ba20k, latency, batching, hash, "
                         "serve, er_phase, pl_bound; 'none' for none)")
    ap.add_argument("--er-phase-step", type=float, default=0.0,
                    help="grid step of the Erdos-Renyi study (default: the paper's 0.03)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="default options instead of autotuning")
    ap.add_argument("--trials", type=int, default=0,
                    help="colouring trials per step (default: the workload's); smaller values "
                         "only for small profiling captures")
    ap.add_argument("--arena-gb", type=int, default=200,
                    help="device arena of the DP context (small values for profiling captures)")
    ap.add_argument("--serve-queries", type=int, default=2000,
                    help="queries of the serving stream to run (the full stream has 2000)")
    ap.add_argument("--serve-window", type=float, default=45.0,
                    help="seconds each serving leg (served, plain) runs")
    ap.add_argument("--opts", default="",
                    help="run options as a JSON object of cc_run_opts fields (default options "
                         "otherwise); given options are used as they are, without autotuning")
    ap.add_argument("--capture", default="", metavar="JSON",
                    help="for an ncu capture: warm-up steps, then one step inside the profiler "
                         "range (ncu --profile-from-start off); writes the step's algorithmic "
                         "bytes per node rule to JSON and prints nothing else")
    ap.add_argument("--traffic-summary", nargs=2, metavar=("CSV", "JSON"),
                    help="write profiles/dram_<workload>.txt from the ncu CSV of a --capture "
                         "run (dram__bytes_read.sum, dram__bytes_write.sum, "
                         "gpu__time_duration.sum) and its JSON; runs nothing on the GPU")
    ap.add_argument("--capture-cmd", default="", help="the capture's command line, recorded in "
                    "the summary")
    ap.add_argument("--launch-summary", default="", metavar="CSV",
                    help="write profiles/launches_<workload>.txt from the ncu launch list "
                         "(gpu__time_duration.sum) of a bench command; runs nothing on the GPU")
    args = ap.parse_args()
    if args.launch_summary:
        print(launch_summary(args.launch_summary, args.workload, args.capture_cmd,
                             skip_steps=args.warmup))
        return
    if args.traffic_summary:
        print(traffic_summary(*args.traffic_summary, args.capture_cmd))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_1908_11248_gb300 as cc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    legs = set() if args.legs == "none" else set(args.legs.split(","))
    enum_limit = ENUM_LIMIT if args.workload == MAIN else 0
    if args.capture:
        dp_leg(cc, torch, args.workload, args, rank, None, tune=False,
               enum_limit=ENUM_LIMIT if args.workload == MAIN else 0, capture=args.capture)
        return
    sampler = ClockSampler(torch.cuda.current_device())
    main_leg = dp_leg(cc, torch, args.workload, args, rank, dist, tune=not args.no_tune,
                      enum_limit=enum_limit, sampler=sampler)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("cpu baseline (oracle)")
        cpu = cpu_baseline(cc, args.workload, main_leg, main_leg["counts"])
    main_leg.pop("_ctx")[0].close()
    torch.cuda.empty_cache()
    line = None
    if rank == 0:
        cfg = dict(main_leg["config"], entries_per_step=main_leg["entries_per_step"],
                   parallelism=f"replicas x{world}",
                   l2="flushed between timed steps (256 MB write); tables exceed L2")
        if enum_limit:
            cfg["enumerate_limit"] = enum_limit
            cfg["enumerated_rows"] = main_leg["enumerated_rows"]
        cfg["max_table_entries"] = main_leg["max_table_entries"]
        cfg["run_modes"] = main_leg["run_modes"]
        line = {
            "metric": METRIC, "value": main_leg["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": main_leg["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": cfg, "roofline": main_leg["roofline"],
            "cpu_baseline": cpu, "e2e": main_leg.get("e2e"),
            "gpu_launches": main_leg["gpu_launches"], "clocks": main_leg["clocks"],
            "autotune": main_leg.get("autotune"),
        }
    if rank == 0 and world == 1:
        if "ba20k" in legs and args.workload != "ba20k_grid2x4":
            a2 = argparse.Namespace(**vars(args))
            a2.arena_gb = min(args.arena_gb, 96)
            log("leg: ba20k_grid2x4")
            leg = dp_leg(cc, torch, "ba20k_grid2x4", a2, rank, None, tune=False,
                         sampler=ClockSampler(torch.cuda.current_device()))
            leg.pop("_ctx")[0].close()
            leg.pop("counts")
            torch.cuda.empty_cache()
            line["ba20k_grid2x4"] = leg
        if "latency" in legs:
            log("leg: latency")
            line["er200_c5_latency"] = latency_leg(cc, torch)
        if "batching" in legs:
            log("leg: batching")
            line["batched_vs_plain"] = batching_leg(cc, torch)
            torch.cuda.empty_cache()
        if "hash" in legs:
            log("leg: hash")
            try:
                line["hashed_rules"] = hash_leg(cc, torch)
            except Exception as ex:  # noqa: BLE001
                line["hashed_rules"] = {"error": repr(ex)}
            torch.cuda.empty_cache()
        if "pl_bound" in legs:
            log("leg: pl_bound")
            try:  # host-only arithmetic; a failure here must not cost the bench line
                line["pl1m_ktree3_bound"] = pl_bound_leg(
                    cc, torch.cuda.get_device_properties(torch.cuda.current_device()).total_memory)
            except Exception as ex:  # noqa: BLE001
                line["pl1m_ktree3_bound"] = {"error": repr(ex)}
        if "er_phase" in legs:
            log("leg: er_phase")
            line["er_phase"] = er_phase_leg(cc, torch, args.er_phase_step or None)
            torch.cuda.empty_cache()
        if "serve" in legs and args.serve_queries > 0:
            log("leg: serving")
            line["serving"] = serve_leg(cc, torch, args.serve_queries, 200, 160, 8,
                                        args.serve_window)
    log("done")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
