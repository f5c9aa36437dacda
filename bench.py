"""Benchmark: kernel columns per second of phi(L) E_W on one GB300 (or N replicas).

Workload (default): random geometric graph, n = 1,000,000 nodes in the unit square,
radius for mean degree 10, unweighted standard Laplacian (int32 CSR, FP32 values);
M = 64 seeded nodes; diffusion kernel e^{-tL} with t in {0.5, 2.0}; all five block
Krylov methods (cbl, gbl, sbl, cheb, cheb2) with m = 30 products each.  One step = those
10 solves (640 kernel columns).  The graph and the output buffers are resident in HBM
before timing; each solve takes its scratch from the stream-ordered pool inside the
timed region.  Between steps a 256 MiB buffer is written to flush the 129 MB L2 (the
per-solve working set, 2-8 GB, is also far above L2).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload
(the 10 solves with the first 4 of the 64 nodes), on the host cores.

Under torchrun each rank is an independent replica (its own node seed); no collective
is used on the data path ("replicas only", weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METHODS = ["cbl", "gbl", "sbl", "cheb", "cheb2"]
METRIC = "kernel columns/sec at 1e-6 rel err vs FP64 oracle"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kb", choices=["kb", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--M", type=int, default=64)
    ap.add_argument("--m", type=int, default=30)
    ap.add_argument("--ts", default="0.5,2.0")
    ap.add_argument("--graph", default="rgg", choices=["rgg", "ba"],
                    help="random geometric graph (mean degree 10) or Barabasi-Albert (5 edges per node)")
    ap.add_argument("--weighted", action="store_true", help="BA edge weights uniform in [0.5, 1.5]")
    ap.add_argument("--phi", default="exp", choices=["exp", "spline"],
                    help="diffusion kernel e^{-tL} (times --ts) or spline (eps I + L)^{-s}")
    ap.add_argument("--eps", type=float, default=0.01)
    ap.add_argument("--s", type=float, default=2.0)
    ap.add_argument("--reorth", type=int, default=0, help="cbl reorthogonalisation: 0, 1 full, 2 local")
    ap.add_argument("--methods", default=",".join(METHODS))
    ap.add_argument("--graph-seed", type=int, default=1)
    ap.add_argument("--node-seed", type=int, default=2)
    ap.add_argument("--basis", default="f32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="steps of the plain FP64 GPU mode timed for comparison (0 = skip)")
    ap.add_argument("--ref-sample-cols", type=int, default=4)
    ap.add_argument("--no-frontier", action="store_true",
                    help="touch all n rows at every step (disables the exact frontier restriction)")
    ap.add_argument("--streams", type=int, default=5,
                    help="CUDA streams the independent solves of a step are spread over")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-latency sample (kb_server_*)")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-max-n", type=int, default=200_000,
                    help="largest of the 8 serving graphs (the others are log-spaced from 1e4)")
    ap.add_argument("--serve-streams", type=int, default=4)
    ap.add_argument("--serve-warmup", type=int, default=0,
                    help="requests in the serving warm-up pass (0: all of them)")
    ap.add_argument("--tensor-cores", action="store_true",
                    help="use the tcgen05 row-block kernels (KB_TENSOR_CORES=1) in the cbl solves")
    ap.add_argument("--schedule", default="lpt", choices=["lpt", "rr"],
                    help="assignment of the independent solves of a step to the streams: "
                         "longest first onto the least loaded stream, or round robin")
    ap.add_argument("--no-priority", action="store_true",
                    help="all solve streams at the same priority (default: the streams holding "
                         "the costliest solves, which form the step's critical path, get the "
                         "highest stream priority)")
    return ap.parse_args()


def kernel_times(a):
    """The diffusion times of the step's solves (one placeholder for the spline kernel)."""
    return [float(x) for x in a.ts.split(",")] if a.phi == "exp" else [0.0]


def phi_kwargs(a, t):
    return dict(t=t) if a.phi == "exp" else dict(eps=a.eps, s=a.s)


def bench_graph(a):
    import synth
    if a.graph == "ba":
        return synth.barabasi_albert_graph(a.n, 5, seed=a.graph_seed, weighted=a.weighted)
    return synth.random_geometric_graph(a.n, 10, seed=a.graph_seed)


def workload_config(a):
    kern = f"exp t={a.ts}" if a.phi == "exp" else f"spline eps={a.eps:g} s={a.s:g}"
    gname = ("rgg n=%d mean_degree=10" % a.n) if a.graph == "rgg" else \
            ("ba n=%d edges_per_node=5%s" % (a.n, " weighted" if a.weighted else ""))
    return {"workload": f"{gname} M={a.M} m={a.m} {kern} methods={a.methods}"
                        + (f" reorth={a.reorth}" if a.reorth else ""),
            "graph": ("random geometric graph, unit square, cell-sorted node order" if a.graph == "rgg"
                      else "Barabasi-Albert, 5 edges per new node"),
            "n": a.n, "mean_degree": 10, "M": a.M, "m": a.m,
            "phi": a.phi, "t": kernel_times(a) if a.phi == "exp" else None,
            "eps": a.eps if a.phi == "spline" else None, "s": a.s if a.phi == "spline" else None,
            "reorth": a.reorth, "methods": a.methods.split(","),
            "graph_seed": a.graph_seed, "node_seed": a.node_seed, "basis": a.basis,
            "l2": "256 MiB flush write between steps; per-solve working set > L2",
            "streams": a.streams, "schedule": a.schedule,
            "stream_priority": "uniform" if a.no_priority else "critical path first",
            "rowblock": "tcgen05 bf16x6" if a.tensor_cores else "simt fp32",
            "frontier": not a.no_frontier}


# relative cost of one solve per method (single-stream solve times at n = 1e6, M = 64,
# m = 30), used only to spread the independent solves of a step over the streams
SOLVE_COST = {"cbl": 3.3, "gbl": 1.0, "sbl": 1.0, "cheb": 0.65, "cheb2": 0.74}


def assign_streams(solves, nstreams, policy):
    """Stream index per solve, and the launch order.  'lpt': solves sorted by decreasing
    cost, each onto the stream with the least cost so far; 'rr': solve i onto stream
    i mod nstreams in the given order."""
    if policy == "rr" or nstreams <= 1:
        return [i % nstreams for i in range(len(solves))], list(range(len(solves)))
    order = sorted(range(len(solves)), key=lambda i: -SOLVE_COST.get(solves[i][0], 1.0))
    load = [0.0] * nstreams
    where = [0] * len(solves)
    for i in order:
        j = min(range(nstreams), key=lambda q: (load[q], q))
        where[i] = j
        load[j] += SOLVE_COST.get(solves[i][0], 1.0)
    return where, order


def critical_streams(solves, where):
    """Streams holding a solve of the largest cost of the step: its critical path, given the
    highest stream priority so that the cheaper solves fill the SMs around it."""
    top = max(SOLVE_COST.get(m_, 1.0) for m_, _ in solves)
    return {where[i] for i, (m_, _) in enumerate(solves) if SOLVE_COST.get(m_, 1.0) == top}


# ----------------------------------------------------------------------------- small config
def small_config(kb, torch):
    """CPU-baseline leg for the 32 x 32 grid (n = 1024), 16 nodes, e^{-L}, cbl m = 20: the
    dense FP64 eigendecomposition on the host beside the GPU kernel columns/s (one stream,
    50 solves), and the relative error of the GPU result against the dense evaluation."""
    import synth
    from oracle import dense
    g = synth.grid_graph((32, 32))
    nodes = synth.sample_nodes(g.n, 16, seed=1)
    with kb.Graph.from_csr(g) as G:
        Y = kb.kernel_columns(G, "cbl", "exp", nodes, 20, t=1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(50):
            Y = kb.kernel_columns(G, "cbl", "exp", nodes, 20, t=1.0)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 50
        y = Y.cpu().numpy().astype(np.float64)
    t0 = time.perf_counter()
    Lh = dense.laplacian_dense(g.n, g.rowptr, g.col, g.val)
    ex = dense.kernel_columns(Lh, nodes, dense.phi_function("exp", t=1.0))
    cpu_s = time.perf_counter() - t0
    return {"workload": "grid 32x32, M=16, exp t=1, cbl m=20", "gpu_ms_per_solve": round(ms, 3),
            "gpu_kernel_columns_per_s": round(16 / (ms / 1e3), 1),
            "cpu_dense_eig_kernel_columns_per_s": round(16 / cpu_s, 1),
            "rel_err_vs_dense_eig": float(np.linalg.norm(y - ex) / np.linalg.norm(ex))}


# ----------------------------------------------------------------------------- serving
M_MAX = 100   # serving: largest number of cbl steps (the stopping rule ends most requests earlier)


def serving_sample(a, kb, torch):
    """Latency of kernel-column requests through the serving front end (kb_server_*).

    8 graphs with n_k = 1e4 * (max_n / 1e4)^(k/7), random geometric for even k and
    Barabasi-Albert (5 edges per node) for odd k.  Requests: method cbl, m = 30, M uniform
    in 1..128, half e^{-tL} with t ~ U[0.1, 5], half (eps I + L)^{-s} with eps log-uniform
    in [1e-3, 1e-1] and s in {1, 2}, graph uniform.  First the saturated throughput is
    measured (all requests submitted at once), then the same requests arrive as a Poisson
    process at 0.8 of that rate; latency = submit to end of the solve.  One reference
    request (the middle graph, M = 64, t = 1) is also timed alone on an idle server.
    """
    import synth
    rng = np.random.default_rng(77)
    K = 8
    ns = [int(round(1e4 * (a.serve_max_n / 1e4) ** (k / 7))) for k in range(K)]
    hg = [synth.random_geometric_graph(n, 10, seed=100 + k) if k % 2 == 0
          else synth.barabasi_albert_graph(n, 5, seed=100 + k) for k, n in enumerate(ns)]
    Gs = [kb.Graph.from_csr(g) for g in hg]
    R = a.serve_requests
    reqs = []
    for i in range(R):
        k = int(rng.integers(0, K))
        M = int(rng.integers(1, 129))
        # local reorthogonalisation keeps the FP32 basis usable on the hub-heavy graphs
        # cbl with the stopping rule tol = 1e-6, at most 100 steps
        if rng.random() < 0.5:
            p = kb.make_params(t=float(rng.uniform(0.1, 5.0)), reorth=2, tol=1e-6)
            phi = "exp"
        else:
            p = kb.make_params(eps=float(10 ** rng.uniform(-3, -1)), s=float(rng.integers(1, 3)),
                               reorth=2, tol=1e-6)
            phi = "spline"
        nodes = synth.sample_nodes(ns[k], M, seed=1000 + i)
        reqs.append((k, phi, p, nodes))
    # latency per request class (graph family x kernel), from the Poisson run
    cls = [("rgg" if k % 2 == 0 else "ba") + "-" + phi for (k, phi, _, _) in reqs]
    # output slots for the requests in flight: at most 16 GB of them (with the 2e6-node graphs
    # of the full serving stream that is 15 slots), the rest of the memory for the solves
    window = int(max(8, min(64, 16e9 // (max(ns) * 128 * 4))))
    slots = [torch.empty(max(ns) * 128, dtype=torch.float32, device="cuda") for _ in range(window)]

    failed = [0]
    retried = [0]
    steps = []

    def finish(sv, tk, lat, idx=None, bycls=None):
        # a request whose block Lanczos process meets a rank-deficient block (a node set
        # spanning a small connected component) is rerun by the server as sbl (counted);
        # a request that still fails is counted, not timed
        try:
            info, ms = sv.poll(tk, wait_ms=-1)
            lat.append(ms)
            if bycls is not None:
                bycls.setdefault(cls[idx], []).append(ms)
            steps.append(info["steps_done"])
            if info["breakdown_step"] >= 0:
                retried[0] += 1
        except kb.KbError:
            failed[0] += 1

    bycls = {}

    def run(arrival_times, record=None, count=None):
        lat = []
        with kb.Server(streams=a.serve_streams, queue_capacity=R + 1, fallback_sbl=True) as sv:
            outstanding = []   # (ticket, slot, request index)
            free = list(range(window))
            t0 = time.perf_counter()
            for i, (k, phi, p, nodes) in enumerate(reqs[:count]):
                if arrival_times is not None:
                    dt = t0 + arrival_times[i] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                while not free:
                    tk, sl, ii = outstanding.pop(0)
                    finish(sv, tk, lat, ii, record)
                    free.append(sl)
                sl = free.pop()
                Y = slots[sl][: ns[k] * nodes.size].view(ns[k], nodes.size)
                outstanding.append((sv.submit(Gs[k], "cbl", phi, p, nodes, M_MAX, Y), sl, i))
            for tk, sl, ii in outstanding:
                finish(sv, tk, lat, ii, record)
            wall = time.perf_counter() - t0
        return lat, wall

    # warm-up (pool growth, lazy module loads); a prefix of the stream when --serve-warmup > 0
    run(None, count=a.serve_warmup if a.serve_warmup > 0 else None)
    failed[0] = 0
    retried[0] = 0
    steps.clear()
    _, wall = run(None)
    failed_sat = failed[0]
    failed[0] = 0
    retried[0] = 0
    steps.clear()
    sat = R / wall
    rate = 0.8 * sat
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=R))
    lat, _ = run(arrivals, bycls)
    kmid = K // 2
    ref_nodes = synth.sample_nodes(ns[kmid], 64, seed=5)
    Yref = torch.empty((ns[kmid], 64), dtype=torch.float32, device="cuda")
    alone = []
    with kb.Server(streams=a.serve_streams, queue_capacity=4) as sv:
        for _ in range(5):
            tk = sv.submit(Gs[kmid], "cbl", "exp", kb.make_params(t=1.0, tol=1e-6), ref_nodes, M_MAX, Yref)
            alone.append(sv.poll(tk, wait_ms=-1)[1])
    for G in Gs:
        G.destroy()
    q = np.percentile(np.array(lat), [50, 99])
    return {"requests": R, "warmup_requests": a.serve_warmup if a.serve_warmup > 0 else R,
            "graph_n": ns, "streams": a.serve_streams,
            "method": "cbl reorth=2, stopping rule tol=1e-6", "m_max": M_MAX,
            "steps_done_mean": round(float(np.mean(steps)), 1) if steps else None,
            "mix": "M~U{1..128}; exp t~U[0.1,5] | spline eps~logU[1e-3,1e-1], s in {1,2}",
            "saturated_rps": round(sat, 2), "rate_rps": round(rate, 2),
            "p50_ms": round(float(q[0]), 3), "p99_ms": round(float(q[1]), 3),
            "mean_ms": round(float(np.mean(lat)), 3),
            "failed_breakdown": failed[0], "failed_breakdown_saturated_run": failed_sat,
            "retried_as_sbl": retried[0],
            "reference_alone_ms": round(float(np.median(alone)), 3),
            "p50_p99_ms_by_class": {c: [round(float(np.percentile(v, 50)), 1), round(float(np.percentile(v, 99)), 1), len(v)]
                                    for c, v in sorted(bycls.items())},
            "columns_per_s_saturated": round(sum(int(r[3].size) for r in reqs) / wall, 1),
            "reference": f"n={ns[kmid]} M=64 exp t=1 cbl tol=1e-6 on an idle server"}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        pass

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic():
    """DRAM traffic per algorithmic byte (kernel class -> (ratio, capture summary file))
    from the committed ncu summaries, if any."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    out = {}
    if os.path.exists(p):
        for line in open(p):
            line = line.strip()
            if line and not line.startswith("#"):
                parts = line.split()
                if len(parts) >= 3:
                    try:
                        out[parts[0]] = (float(parts[1]), parts[2])
                    except ValueError:
                        pass
    return out


# ----------------------------------------------------------------------------- reference arm
def run_reference(a, rank, world):
    if rank != 0:
        return
    import synth
    from oracle import krylov
    ts = kernel_times(a)
    methods = a.methods.split(",")
    g = bench_graph(a)
    nodes = synth.sample_nodes(a.n, a.M, seed=a.node_seed)[: a.ref_sample_cols]
    L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)

    def step():
        for mth in methods:
            for t in ts:
                krylov.apply(mth, L, nodes, a.m, a.phi, reorth=bool(a.reorth == 1), **phi_kwargs(a, t))

    for _ in range(a.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step()
    dt = (time.perf_counter() - t0) / a.steps
    cols = len(methods) * len(ts) * len(nodes)
    val = cols / dt
    sample = (f"{len(methods)}x{len(ts)} solves with the first {len(nodes)} of the {a.M} nodes "
              f"(m={a.m}) on the full graph, numpy/scipy FP64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "kernel_columns/s",
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(a),
        "cpu_baseline": {"value": val, "unit": "kernel_columns/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "kernel_columns/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def cpu_baseline(a, budget_s=25.0):
    """The oracle as it stands on a bounded sample: the step's solves with the first
    ref_sample_cols columns.  Also returns the oracle's columns of the methods whose
    columns are independent (sbl, cheb, cheb2), which equal the GPU's first columns."""
    import synth
    from oracle import krylov
    ts = kernel_times(a)
    methods = a.methods.split(",")
    g = bench_graph(a)
    nodes = synth.sample_nodes(a.n, a.M, seed=a.node_seed)[: a.ref_sample_cols]
    L = krylov.laplacian(g.n, g.rowptr, g.col, g.val)
    t0 = time.perf_counter()
    cols = 0
    ref_cols = {}
    for mth in methods:
        for t in ts:
            Y = krylov.apply(mth, L, nodes, a.m, a.phi, reorth=bool(a.reorth == 1), **phi_kwargs(a, t)).Y
            cols += len(nodes)
            if mth in ("sbl", "cheb", "cheb2"):
                ref_cols[(mth, t)] = Y
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return ({"value": cols / dt, "unit": "kernel_columns/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"{cols // len(nodes)} solves (methods {methods}, t {ts}) with the first "
                       f"{len(nodes)} of {a.M} nodes, m={a.m}, full graph, {dt:.1f} s"}, ref_cols)


def accuracy_vs_oracle(ref_cols, first_cols, solves):
    """Relative Frobenius error of the timed solves' first columns against the oracle's
    columns for the methods with independent columns (the metric's 1e-6 gate)."""
    out = {}
    for (mth, t), Y in zip(solves, first_cols):
        ref = ref_cols.get((mth, t))
        if ref is None:
            continue
        y = Y.numpy().astype(np.float64)
        out[f"{mth} t={t:g}"] = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    return out


# ----------------------------------------------------------------------------- replicas
def replica_node_seed(node_seed: int, rank: int) -> int:
    """Each rank is an independent replica of the workload with its own node set."""
    return node_seed + rank


def job_time_ms(ms_local: float, world: int, device) -> float:
    """Time of the whole job: the slowest rank (max over ranks; no data-path collective)."""
    if world == 1:
        return ms_local
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(tt.item())


def job_value(cols_per_step: int, world: int, ms: float) -> float:
    """Whole-job throughput: the columns all ranks produced per second of job time."""
    return world * cols_per_step / (ms / 1e3)


# ----------------------------------------------------------------------------- GPU arm
def main():
    a = parse()
    if a.tensor_cores:
        os.environ["KB_TENSOR_CORES"] = "1"   # read by the library at each row-block launch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return

    import torch
    import torch.distributed as dist
    import synth
    from paper_2301_06384_gb300 import kb

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.cuda.current_device()
    ts = kernel_times(a)
    methods = a.methods.split(",")
    g = bench_graph(a)
    nodes = synth.sample_nodes(a.n, a.M, seed=replica_node_seed(a.node_seed, rank))
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    tg0 = time.perf_counter()
    G = kb.Graph.from_csr(g, stream=stream)   # host validation + upload + Gershgorin bound
    graph_create_ms = (time.perf_counter() - tg0) * 1e3
    solves = [(mth, t) for mth in methods for t in ts]
    Ys = [torch.empty((a.n, a.M), dtype=torch.float32, device="cuda") for _ in solves]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    params = {t: kb.make_params(basis=a.basis, no_frontier=int(a.no_frontier), reorth=a.reorth,
                                **phi_kwargs(a, t)) for t in ts}

    nstreams = max(1, a.streams)
    where, order = assign_streams(solves, nstreams, a.schedule)
    hot = critical_streams(solves, where)
    if nstreams == 1:
        streams = [stream]
    else:
        streams = [torch.cuda.Stream(priority=(-5 if (j in hot and not a.no_priority) else 0))
                   for j in range(nstreams)]

    def step(pr=params):
        # independent solves spread over the streams; every stream joins the main one
        ev = torch.cuda.Event()
        ev.record(stream)
        for s2 in streams:
            if s2 is not stream:
                s2.wait_event(ev)
        for i in order:
            mth, t = solves[i]
            kb.kb_krylov_apply(G, mth, a.phi, pr[t], nodes, a.M, a.m, Ys[i], stream=streams[where[i]])
        for s2 in streams:
            if s2 is not stream:
                e2 = torch.cuda.Event()
                e2.record(s2)
                stream.wait_event(e2)

    for _ in range(a.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = kb.kb_launch_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev).__enter__()
    kb.kb_profile_enable(True)
    e0.record(stream)
    for _ in range(a.steps):
        flush.zero_()
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    kb.kb_profile_enable(False)
    clocks = sampler.stop()
    launches = (kb.kb_launch_counter() - l0) // max(a.steps, 1)
    stats = kb.kb_profile_read()
    ms = job_time_ms(e0.elapsed_time(e1) / a.steps, world, "cuda")
    cols_per_step = len(solves) * a.M
    value = job_value(cols_per_step, world, ms)

    # Kernel-class profile of the timed region (five streams): the classes' launch
    # durations overlap there (a class's summed time can exceed the step), so the roofline
    # line below takes its launch durations from a one-stream pass of the same solves.
    peak, peak_kind = measured_peaks()
    traffic = ncu_traffic()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    shares = {k: round(v["total_ms"] / a.steps / ms, 4) for k, v in stats.items() if v["launches"]}

    # time of each solve alone (one stream, after the timed region; not part of value), with
    # the kernel-class profile of that pass: launch durations free of other streams' kernels
    solve_ms = {}
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(solves) + 1)]
    flush.zero_()
    kb.kb_profile_enable(True)
    evs[0].record(stream)
    for i, ((mth, t), Y) in enumerate(zip(solves, Ys)):
        kb.kb_krylov_apply(G, mth, a.phi, params[t], nodes, a.M, a.m, Y, stream=stream)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    kb.kb_profile_enable(False)
    stats1 = kb.kb_profile_read()
    for i, (mth, t) in enumerate(solves):
        solve_ms[f"{mth} t={t:g}" if a.phi == "exp" else f"{mth} {a.phi}"] = round(evs[i].elapsed_time(evs[i + 1]), 3)
    ms1 = evs[0].elapsed_time(evs[-1])
    # the FP32 results' first columns, kept for the accuracy check against the oracle (the
    # FP64 comparator below reuses the output buffers)
    first_cols = [Y[:, : a.ref_sample_cols].cpu() for Y in Ys]
    shares_one_stream = {k: round(v["total_ms"] / ms1, 4) for k, v in stats1.items() if v["launches"]}

    def roof(st, name, total_ms, timing):
        """HBM roofline of one kernel class: algorithmic bytes per launch / mean launch time
        against the measured copy bandwidth; traffic = DRAM bytes per launch scaled from
        the ncu capture named in profiles/traffic.txt (ratio x this run's algorithmic
        bytes), null when no capture covers the class."""
        s = st.get(name)
        if not s or s["total_ms"] <= 0:
            return None
        nl = max(s["launches"], 1)
        gbs = s["alg_bytes"] / (s["total_ms"] / 1e3) / 1e9
        ratio = traffic.get(name)
        out = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
               "frac": round(gbs / peak, 4),
               "traffic": round(ratio[0] * s["alg_bytes"] / nl) if ratio else None,
               "traffic_source": (f"scaled: DRAM/algorithmic ratio {ratio[0]} of the capture "
                                  f"profiles/{ratio[1]} x this run's algorithmic bytes per launch")
                                 if ratio else None,
               "kernel": name, "launches": s["launches"],
               "alg_bytes_per_launch": round(s["alg_bytes"] / nl),
               "avg_launch_ms": round(s["total_ms"] / nl, 5),
               "share_of_step": round(s["total_ms"] / total_ms, 4),
               "timing": timing, "peak_kind": f"{peak_kind} hbm_gbs",
               "frac_of_nominal_7900_gbs": round(gbs / 7900.0, 4)}
        if s["alg_flops"] > 0 and name == "rowblock":
            # the SIMT tall-skinny products also meet the FP32 FMA issue limit: unit counts
            # (SMs queried from the device x 128 FP32 lanes x 2 flops) x the sampled clock
            sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
            alu_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
            tfs = s["alg_flops"] / (s["total_ms"] / 1e3) / 1e12
            out["alu_view"] = {"achieved_tflops": round(tfs, 2), "peak_tflops": round(alu_peak, 1),
                               "frac": round(tfs / alu_peak, 4),
                               "peak_kind": f"FP32 FMA peak: {sms} SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz"}
        return out

    one = "one-stream pass of the step's solves after the timed region (launches alone on the GPU)"
    five = ("timed region, five streams: launch durations overlap other streams' kernels, so "
            "share_of_step can exceed 1 and achieved is a lower bound")
    # dominant class among those that move HBM bytes (the FP64 single-CTA classes have none)
    hbm_classes = {k: v for k, v in stats1.items() if v["alg_bytes"] > 0}
    dom1 = max(hbm_classes.items(), key=lambda kv: kv[1]["total_ms"])[0] if hbm_classes else None
    roofline = roof(stats1, dom1, ms1, one) if dom1 else None
    spmm_one_stream = roof(stats1, "spmm", ms1, one)
    rowblock_one_stream = roof(stats1, "rowblock", ms1, one)
    spmm_five_stream = roof(stats, "spmm", ms * a.steps, five)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed
    # region; one host thread per stream, each running its share of the solves
    e2e = None
    if not a.no_e2e:
        from concurrent.futures import ThreadPoolExecutor
        Yh = [torch.empty((a.n, a.M), dtype=torch.float32).pin_memory() for _ in solves]
        pool = ThreadPoolExecutor(max_workers=len(streams))

        def run_share(j):
            for i in (q for q in order if where[q] == j):
                mth, t = solves[i]
                kb.kb_krylov_apply_host(G, mth, a.phi, params[t], nodes, a.M, a.m, Yh[i],
                                        stream=streams[j])

        def step_host():
            list(pool.map(run_share, range(len(streams))))
        step_host()
        torch.cuda.synchronize()
        ksteps = max(1, min(a.steps, 2))
        t0 = time.perf_counter()
        for _ in range(ksteps):
            step_host()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / ksteps
        e2e = {"value": job_value(cols_per_step, world, job_time_ms(dt * 1e3, world, "cuda")),
               "unit": "kernel_columns/s",
               "h2d_bytes_per_step": len(solves) * a.M * 4,
               "d2h_bytes_per_step": len(solves) * a.n * a.M * 4}

    # plain FP64 GPU mode (the comparator of the mixed-precision form), same solves
    fp64 = None
    if a.fp64_steps > 0 and a.basis == "f32":
        p64 = {t: kb.make_params(basis="f64", no_frontier=int(a.no_frontier), reorth=a.reorth,
                                 **phi_kwargs(a, t)) for t in ts}
        try:
            step(p64)
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(a.fp64_steps):
                flush.zero_()
                step(p64)
            f1.record(stream)
            torch.cuda.synchronize()
            fms = f0.elapsed_time(f1) / a.fp64_steps
            fp64 = {"value": cols_per_step / (fms / 1e3), "unit": "kernel_columns/s",
                    "ms_per_step": fms, "speedup_of_fp32_path": round(fms / ms, 3)}
        except kb.KbError as exc:
            fp64 = {"unavailable": str(exc)}

    serving = None
    if not a.no_serving and world == 1:
        try:
            serving = serving_sample(a, kb, torch)
        except kb.KbError as exc:
            serving = {"unavailable": str(exc)}

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 2), "unit": "kernel_columns/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if a.basis == "f32" else a.basis, "data": "synthetic",
            "config": workload_config(a),
            "clocks": clocks, "gpu_launches": int(launches),
            "roofline": roofline,
            "spmm_roofline": spmm_one_stream,
            "spmm_roofline_five_stream": spmm_five_stream,
            "kernel_shares": shares,
            "e2e": e2e, "fp64_plain": fp64, "solve_ms_one_stream": solve_ms,
            "rowblock_roofline": rowblock_one_stream, "kernel_shares_one_stream": shares_one_stream,
            "serving": serving, "graph_create_ms": round(graph_create_ms, 1),
        }
        acc_fail = False
        if world == 1 and not a.no_cpu_baseline:
            out["cpu_baseline"], ref_cols = cpu_baseline(a)
            errs = accuracy_vs_oracle(ref_cols, first_cols, solves)
            out["rel_err_vs_oracle"] = {
                "max": max(errs.values()) if errs else None, "per_solve": errs, "gate": 1e-6,
                "what": (f"first {a.ref_sample_cols} columns of the timed sbl / cheb / cheb2 solves "
                         "(independent columns) against the FP64 oracle's columns")}
            acc_fail = bool(errs) and max(errs.values()) > 1e-6
            # the small grid case with its dense-eigendecomposition baseline
            out["cpu_baseline_small_config"] = small_config(kb, torch)
        print(json.dumps(out))
        if acc_fail:
            sys.stdout.flush()
            sys.exit("accuracy gate failed: relative error above 1e-6 against the FP64 oracle")
    G.destroy()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
