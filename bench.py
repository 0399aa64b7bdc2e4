"""Benchmark of the InfraredGP FFP hot path on GB300 (one JSON line on rank 0).

A step is one pass of the whole hot path over one synthetic graph: CSR
construction from the device-resident edge list, Eq. 1 degree factors, the
Theta draw, L Eq. 4 layers and the sigmoid output (Alg. 1 up to its clustering step). The
metric is edge*dim*layer/s = nnz * d * L per step / step time, nnz counting
the directed CSR entries (twice the undirected edges).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

The default run (the 2M-node workload, one GPU) also measures the other configurations and adds
them as keys of the same JSON line: c2_f32 and c2_bf16 (the 200K-node graph, each with its own
roofline), batched (512 uneven graphs in one batch against the same graphs one at a time in
fp32), served (the Poisson stream of snapshot requests: p50/p99 per snapshot and per graph,
throughput against serial fp32), streaming_vs_static (Alg. 2 step by step against Alg. 1
re-run at every step, with the device clusterer) and clustered (the device clusterer on the FFP
output of a 1M-node benchmark-shaped graph). --no-extras skips them.

Multi-GPU (torchrun): every rank runs an independent replica of the workload
(the FFP of one graph does not shard); value = units of all ranks / max time.
"""
import argparse
import ctypes
import hashlib
import json
import math
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

from paper_2508_19737_gb300 import synth  # noqa: E402

METRIC = "FFP edge*dim*layer/s"
UNIT = "edge*dim*layer/s"
L2_BYTES = 129 * 1024 * 1024
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_layer_dcsbm-2m.json")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="dcsbm-2m", choices=sorted(synth.WORKLOADS) + sorted(synth.BATCH_WORKLOADS)
                   + sorted(synth.SERVE_WORKLOADS) + sorted(synth.STREAM_WORKLOADS)
                   + sorted(synth.CLUSTER_WORKLOADS))
    p.add_argument("--slots", type=int, default=16, help="concurrent requests of the served stream")
    p.add_argument("--batch-rows", type=int, default=0,
                   help="served graphs with fewer nodes share batched FFPs (0: every slot embeds its own)")
    p.add_argument("--d", type=int, default=None, help="override the workload's embedding width")
    p.add_argument("--storage", default=None, choices=[None, "f32", "bf16"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="headline workload only (by default the 2M-node run also measures the 200K-node graph in "
                        "both storages, the 512-graph batch and the served stream)")
    p.add_argument("--e2e-steps", type=int, default=None)
    p.add_argument("--chunk-cols", type=int, default=0, help="columns per layer pass (0: automatic)")
    p.add_argument("--gather", default="auto", choices=["auto", "lsu", "bulk", "tma4"])
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(x, world, device="cuda"):
    """The largest x over all ranks (every rank gets it); x itself when world == 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank_step, steps, world, ms):
    """Whole-job throughput of `world` independent replicas: every rank processes the same units
    per step, and the job takes the slowest rank's time (ms, max over ranks)."""
    return units_per_rank_step * steps * world / (ms / 1e3)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def layer_bytes(N, nnz, d, sb):
    """Algorithmic bytes of one Eq. 4 layer launch: col + row_ptr + dinv read once,
    T^(l-1) read once, T^(l) written once."""
    return 4 * nnz + 4 * (N + 1) + 4 * N + 2 * N * d * sb


def code_hash(text):
    """sha256 prefix of C/CUDA source with its comments and blank space removed: edits of comments
    alone keep the hash, any change to the code changes it."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = "\n".join(" ".join(line.split()) for line in text.splitlines() if line.strip())
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def kernel_source_hash():
    with open(os.path.join(ROOT, "paper_2508_19737_gb300", "csrc", "ffp.cu")) as f:
        return code_hash(f.read())


def recorded_traffic(workload, storage):
    """Per-launch DRAM bytes of k_layer from the committed ncu summary, if it was taken
    on the current kernel code (comments aside); else None."""
    try:
        with open(PROFILE_SUMMARY) as f:
            j = json.load(f)
        e = j["entries"][f"{workload}/{storage}"]
        if e.get("ffp_cu_code_sha256_16") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
class COracle:
    """The FP64 oracle's C version (oracle/ffp_ref.c, as it stands) on all host cores: whole FFPs
    (Eq. 1 factors, L' layers, output) of the workload graph. The oracle's CSR is built once and
    the input drawn once, untimed."""

    def __init__(self, g, wl):
        import oracle
        from oracle import cffp
        self.cffp = cffp
        self.rp, self.col = oracle.build_csr(g.src, g.dst, g.N)
        self.N, self.d, self.tau = g.N, wl["d"], wl["tau"]
        self.nnz = int(self.rp[-1])
        self.X = synth.gaussian_input(0, g.N, self.d)
        self.cores = cffp.threads()

    def run(self, L):
        t0 = time.perf_counter()
        self.cffp.ffp(self.rp, self.col, self.X, self.tau, L)
        dt = time.perf_counter() - t0
        return float(self.nnz) * self.d * L / dt, dt

    def describe(self, L, dt):
        return (f"the whole FFP (Eq. 1 factors, {L} Eq. 4 layers, output) of the {self.N}-node graph "
                f"({self.nnz} CSR entries, d={self.d}) by the FP64 oracle in C on {self.cores} host threads "
                f"(OpenMP), {dt:.2f} s per FFP; the oracle's CSR built beforehand, untimed")


def run_reference(args):
    """The reference arm: the FP64 oracle (its C version, all host cores) on the same workload.
    A step is one FFP of L' <= L layers, L' chosen so that the whole run ends within a few
    minutes; the rate counts the layers run."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload not in synth.WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the single-graph workloads"}))
        return 0
    wl = synth.WORKLOADS[args.workload]
    g = synth.workload_graph(args.workload)
    ref = COracle(g, wl)
    _, t1 = ref.run(1)
    budget = max(0.5, min(30.0, 150.0 / max(1, args.steps + args.warmup)))
    Ls = int(max(1, min(wl["L"], budget // max(t1, 1e-3))))
    rates, dts = [], []
    for k in range(args.warmup + args.steps):
        r, dt = ref.run(Ls)
        if k >= args.warmup:
            rates.append(r)
            dts.append(dt)
    value = statistics.mean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(dts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, **wl["graph"], "d": wl["d"], "tau": wl["tau"], "L": wl["L"],
                   "layers_per_step": Ls},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ref.cores, "kind": "oracle",
                         "sample": ref.describe(Ls, statistics.mean(dts))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- batches
def _batch_graph(args):
    return synth.workload_batch_graph(*args)


def draw_in_pool(fn, items):
    """fn over items in a pool of spawned processes (spawned, so safe next to a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, items, chunksize=4))


def batch_measure(api, torch, name, storage, d, steps, warmup, local):
    """Many graphs embedded together (igp_batch_embed, CUDA-graph replay) against the same
    graphs embedded one after another in fp32 (igp_embed per graph). A step is one FFP of
    every graph; the graphs are built and packed once, before timing. Returns the JSON dict."""
    wl = synth.BATCH_WORKLOADS[name]
    sb = 2 if storage == "bf16" else 4
    tau, L = wl["tau"], wl["L"]
    G0 = wl["batch"]["G"]
    gs = draw_in_pool(_batch_graph, [(name, k) for k in range(G0)])
    graphs = [api.graph_build(torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(), g.N) for g in gs]
    batch = api.Batch(graphs)
    G, N, nnz, offs = batch.info()
    seeds = list(range(G))
    out = torch.empty((N, d), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    opts = api.embed_opts(storage=storage)
    for _ in range(max(warmup, 3)):
        batch.embed(tau, L, d, seeds, out=out, opts=opts, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    n0 = api.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        batch.embed(tau, L, d, seeds, out=out, opts=opts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = api.launch_count() - n0
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    units = float(nnz) * d * L
    value = units * steps / (ms / 1e3)
    # per-launch layer time (plain launches with events)
    prof = api.Profile()
    popts = api.embed_opts(storage=storage, profile=prof)
    batch.embed(tau, L, d, seeds, out=out, opts=popts, stream=stream)
    torch.cuda.synchronize()
    ph = prof.read()
    prof.close()
    # device time per layer: the layer phase of one profiled embedding over its L layers (one launch
    # per layer, or one persistent launch for all of them, whichever plan the schedule tuner chose)
    layer_s = ph["layer"][0] / max(L, 1) / 1e3
    layer_launches = int(ph["layer"][1])
    lb = layer_bytes(N, nnz, d, sb)
    peak, peak_src = peaks()
    # the same graphs one at a time, fp32
    seq_out = [torch.empty((g.N, d), dtype=torch.float32, device="cuda") for g in gs]
    sopts = api.embed_opts(storage="f32")
    for k, g in enumerate(graphs):
        api.embed(g, tau, L, d, seeds[k], out=seq_out[k], opts=sopts, stream=stream)
    torch.cuda.synchronize()
    reps = 2
    e0.record(stream)
    for _ in range(reps):
        for k, g in enumerate(graphs):
            api.embed(g, tau, L, d, seeds[k], out=seq_out[k], opts=sopts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / reps
    seq_value = units / (seq_ms / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": storage, "data": "synthetic",
        "config": {"workload": name, **wl["batch"], "N_total": N, "nnz_total": int(nnz), "d": d,
                   "tau": tau, "L": L, "storage": storage, "accumulate": "f32",
                   "step": "igp_batch_embed of all graphs (CUDA-graph replay); graphs built and packed once",
                   "l2": "inputs larger than L2" if N * d * sb > L2_BYTES else "working set may fit L2"},
        "roofline": {"bound": "hbm", "achieved": lb / layer_s / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": lb / layer_s / 1e9 / peak, "traffic": None, "kernel": "k_layer_batch",
                     "avg_layer_ms": layer_s * 1e3, "algorithmic_bytes_per_layer": lb,
                     "layer_launches_per_embedding": layer_launches,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else
                     "fallback 6800 GB/s"},
        "sequential_fp32": {"value": seq_value, "unit": UNIT, "ms_per_pass": seq_ms,
                            "what": "igp_embed of each graph in turn, fp32 storage, same d, tau, L, seeds"},
        "speedup_vs_sequential_fp32": value / seq_value,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    batch.free()
    for g in graphs:
        g.free()
    return line


def run_batch(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    wl = synth.BATCH_WORKLOADS[args.workload]
    line = batch_measure(api, torch, args.workload, args.storage or wl["storage"], args.d or wl["d"], args.steps,
                         args.warmup, local)
    print(json.dumps(line), flush=True)
    return 0


def _serve_graph(args):
    return synth.serve_graph(*args)


def serve_measure(api, torch, name, storage, d, slots, batch_rows, warmup, local):
    """The served stream: snapshot requests (an edge increment of one graph, then the FFP of
    the whole graph so far) arriving as a Poisson process, handled by igp_server (concurrent
    slots, admission by free device memory, resident graphs). Reported: latency p50/p99 per
    snapshot and per graph under the stream's arrival rate; the server's throughput with every
    request queued at once; and the same requests handled one at a time by direct library
    calls in fp32 storage (and in the served storage). Edges come from host memory and every
    result is copied to host memory inside the timed regions. Returns the JSON dict."""
    wl = synth.SERVE_WORKLOADS[name]
    params = wl["stream"]
    tau, L = wl["tau"], wl["L"]
    G, T = params["G"], params["T"]
    incs = draw_in_pool(_serve_graph, [(params, k) for k in range(G)])
    times, order = synth.serve_schedule(params)
    R = len(order)
    nfinal = [inc[-1][2] for inc in incs]
    outs = [torch.empty((n, d), dtype=torch.float32, pin_memory=True) for n in nfinal]
    # directed CSR entries after each increment (for the edge*dim*layer count): from a fresh
    # build of each graph's cumulative edges on the device, untimed
    nnz_after = {}
    for k in range(G):
        gr = None
        for t, (s_, d_, n_) in enumerate(incs[k]):
            if gr is None:
                gr = api.graph_build(s_, d_, n_)
            else:
                gr.append(s_, d_, n_)
            nnz_after[(k, t)] = gr.nnz
        gr.free()
    units = sum(nnz_after[o] for o in order) * d * L

    def submit(sv, k, t, st, seed):
        s_, d_, n_ = incs[k][t]
        return sv.submit(s_, d_, n_, tau, L, d, seed, kind="embed" if t == 0 else "append", graph_id=k,
                         keep=(t == 0), out=outs[k], storage=st)

    # warm-up: a few requests of the smallest graph
    kmin = int(np.argmin(nfinal))
    sv = api.Server(slots=slots, batch_rows=batch_rows)
    for _ in range(max(warmup, 3)):
        sv.wait(submit(sv, kmin, 0, storage, 0))
    sv.close()

    # (1) open loop at the stream's arrival rate
    clocks = ClockSampler(local)
    clocks.start()
    n0 = api.launch_count()
    sv = api.Server(slots=slots, batch_rows=batch_rows)
    tickets = [None] * R
    t0 = time.perf_counter()
    for r, (k, t) in enumerate(order):
        wait = t0 + times[r] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        tickets[r] = submit(sv, k, t, storage, 1000 * k + t)
    lat = [sv.wait(tk)[1] for tk in tickets]
    t_open = time.perf_counter() - t0
    launches_open = api.launch_count() - n0
    first = {}
    last = {}
    for r, (k, t) in enumerate(order):
        first.setdefault(k, times[r])
        last[k] = times[r] + lat[r]
    per_graph = [last[k] - first[k] for k in range(G)]
    st_open = sv.stats()
    sv.close()

    # (2) saturation: every request queued at once, same order
    sv = api.Server(slots=slots, batch_rows=batch_rows)
    t0 = time.perf_counter()
    tickets = [submit(sv, k, t, storage, 1000 * k + t) for k, t in order]
    for tk in tickets:
        sv.wait(tk)
    t_sat = time.perf_counter() - t0
    st_sat = sv.stats()
    sv.close()
    clk = clocks.stop()

    # (3) one request at a time, direct calls (build / append, then embed to host)
    def serial(st):
        gr = {}
        t0 = time.perf_counter()
        for k, t in order:
            s_, d_, n_ = incs[k][t]
            if t == 0:
                gr[k] = api.graph_build(s_, d_, n_)
            else:
                gr[k].append(s_, d_, n_)
            api.embed(gr[k], tau, L, d, 1000 * k + t, out=outs[k][:n_], storage=st)
            if t == T - 1:
                gr.pop(k).free()
        return time.perf_counter() - t0

    t_ser32 = serial("f32")
    t_ser = serial(storage)
    pct = lambda v, q: float(np.percentile(np.asarray(v), q))  # noqa: E731
    return {
        "metric": "served snapshot requests/s", "value": R / t_sat, "unit": "requests/s", "n_gpus": 1,
        "steps": R, "warmup": max(warmup, 3), "ms_per_step": t_sat / R * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": storage, "data": "synthetic",
        "config": {"workload": name, **params, "d": d, "tau": tau, "L": L, "storage": storage,
                   "slots": slots, "batch_rows": batch_rows, "requests": R, "N_total_final": int(sum(nfinal)),
                   "step": "one snapshot request: increment merge (or CSR build) + FFP + result to host",
                   "l2": "per-request working sets up to the largest graph; not flushed between requests"},
        "edge_dim_layer_per_s": units / t_sat,
        "open_loop": {"rate_offered": params["rate"], "wall_s": t_open, "rate_achieved": R / t_open,
                      "snapshot_latency_p50_s": pct(lat, 50), "snapshot_latency_p99_s": pct(lat, 99),
                      "graph_latency_p50_s": pct(per_graph, 50), "graph_latency_p99_s": pct(per_graph, 99),
                      "server_p50_s": st_open["latency_p50_s"], "server_p99_s": st_open["latency_p99_s"],
                      "shared_batches": st_open["batches"], "requests_in_shared_batches": st_open["batched"]},
        "serial_fp32": {"value": R / t_ser32, "unit": "requests/s", "wall_s": t_ser32},
        f"serial_{storage}": {"value": R / t_ser, "unit": "requests/s", "wall_s": t_ser},
        "speedup_vs_serial_fp32": t_ser32 / t_sat,
        "saturation": {"shared_batches": st_sat["batches"], "requests_in_shared_batches": st_sat["batched"]},
        "gpu_launches": int(launches_open),
        "clocks": clk,
    }


def run_serve(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    wl = synth.SERVE_WORKLOADS[args.workload]
    line = serve_measure(api, torch, args.workload, args.storage or wl["storage"], args.d or wl["d"], args.slots,
                         args.batch_rows, args.warmup, local)
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- streaming (Alg. 2)
def stream_measure(api, torch, name, local):
    """Alg. 2 against Alg. 1 re-run from scratch at every step (the comparison of Figs. 2-3): a
    graph shaped like the paper's benchmark graphs arrives as 10 snowball increments. Streaming:
    each step merges the increment into the resident CSR, runs the FFP over all nodes so far,
    extracts the new nodes' rows, fits the device clusterer on them and assigns every node so
    far (the clustering of a step overlaps the next step's FFP). Static: each step builds the
    cumulative graph, runs the FFP over all nodes, fits a fresh clusterer on every row and
    assigns them. Per step: seconds of each and the NMI / pairwise F1 of its partition against
    the planted blocks of the nodes so far. Returns the JSON dict."""
    from paper_2508_19737_gb300 import metrics, stream
    wl = synth.STREAM_WORKLOADS[name]
    g = synth.challenge_like(wl["N"], seed=wl["seed"])
    incs, order = synth.split_increments(g, wl["T"], "snowball", seed=wl["seed"], return_order=True)
    blocks = g.blocks[order]
    tau, L, d, storage = wl["tau"], wl["L"], wl["d"], wl["storage"]
    T_cl, B_cl = wl["threshold"], wl["batch"]

    def make():
        return api.Clusterer(d, T_cl, batch=B_cl)

    def quality(lab, n):
        return metrics.nmi(blocks[:n], lab), metrics.pairwise_scores(blocks[:n], lab)[2]
    # warm-up (kernels loaded, pools grown)
    with stream.StreamingPartitioner(make(), tau=tau, L=L, d=d, seed=0, storage=storage) as sp:
        sp.step(*incs[0])
        sp.labels(0)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    with stream.StreamingPartitioner(make(), tau=tau, L=L, d=d, seed=0, storage=storage) as sp:
        for s_, d_, n_ in incs:
            sp.step(s_, d_, n_)
        labs = [sp.labels(t) for t in range(len(incs))]
        t_stream = time.perf_counter() - t0
        timings = [sp.timings[t] for t in range(len(incs))]
    st_rows = []
    for t, (s_, d_, n_) in enumerate(incs):
        st_rows.append({"N_t": n_, "ffp_s": timings[t]["ffp_s"], "cluster_s": timings[t]["cluster_s"],
                        **dict(zip(("nmi", "f1"), quality(labs[t], n_)))})
    # static re-runs on the cumulative graph of every step
    static_rows = []
    t_static = 0.0
    for t in range(len(incs)):
        src = np.concatenate([incs[k][0] for k in range(t + 1)])
        dst = np.concatenate([incs[k][1] for k in range(t + 1)])
        n_ = incs[t][2]
        cl = make()
        t1 = time.perf_counter()
        lab, ffp_s, cl_s = stream.static_partition(src, dst, n_, cl, tau=tau, L=L, d=d, seed=t, storage=storage)
        t_static += time.perf_counter() - t1
        cl.free()
        static_rows.append({"N_t": n_, "ffp_s": ffp_s, "cluster_s": cl_s, **dict(zip(("nmi", "f1"), quality(lab, n_)))})
    clk = clocks.stop()
    return {
        "what": "Alg. 2 (merge, FFP, new rows, device clusterer fit + assign, clustering overlapped with the next "
                "FFP) against Alg. 1 from scratch at every step, on the same increments",
        "config": {"workload": name, **{k: v for k, v in wl.items()}, "blocks": int(blocks.max()) + 1,
                   "clusterer": "device BIRCH leaf level (igp_clusterer)"},
        "streaming_total_s": t_stream, "static_total_s": t_static, "speedup": t_static / t_stream,
        "streaming_steps": st_rows, "static_steps": static_rows, "clocks": clk,
    }


def run_stream(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    print(json.dumps(stream_measure(api, torch, args.workload, local)), flush=True)
    return 0


# ----------------------------------------------------------------------------- clustering
def cluster_measure(api, torch, name, local, reps=5):
    """The device clusterer (BIRCH's leaf level) on the FFP output of a benchmark-shaped graph: the
    embedding stays on the device, each fit starts from an empty clusterer; reported: the fit's
    time (CUDA events), the number of entries and the partition's NMI / pairwise F1 against the
    planted blocks. Returns the JSON dict."""
    from paper_2508_19737_gb300 import metrics
    wl = synth.CLUSTER_WORKLOADS[name]
    g = synth.challenge_like(wl["N"], seed=wl["seed"])
    gr = api.graph_build(g.src, g.dst, g.N)
    E = torch.empty((g.N, wl["d"]), dtype=torch.float32, device="cuda")
    api.embed(gr, wl["tau"], wl["L"], wl["d"], 0, out=E, storage=wl["storage"])
    gr.free()
    lab = torch.empty(g.N, dtype=torch.int32, device="cuda")
    warm = api.Clusterer(wl["d"], wl["threshold"], batch=wl["batch"])
    warm.fit(E[:wl["batch"]], labels=lab[:wl["batch"]])
    warm.free()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    n0 = api.launch_count()
    for _ in range(reps):
        cl = api.Clusterer(wl["d"], wl["threshold"], batch=wl["batch"])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        cl.fit(E, labels=lab)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        K = cl.info()[0]
        cl.free()
    launches = (api.launch_count() - n0) // reps
    clk = clocks.stop()
    l = lab.cpu().numpy()
    p, r, f1 = metrics.pairwise_scores(g.blocks, l)
    ms = statistics.median(times)
    return {"metric": "clustered points/s", "value": g.N / (ms / 1e3), "unit": "points/s", "ms_per_fit": ms,
            "config": {"workload": name, **wl, "blocks": int(g.blocks.max()) + 1},
            "entries": int(K), "nmi": metrics.nmi(g.blocks, l), "f1": f1, "precision": p, "recall": r,
            "gpu_launches_per_fit": int(launches), "clocks": clk,
            "what": "igp_clusterer_fit of every row of the FFP output (device memory), fresh clusterer"}


def run_cluster(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    print(json.dumps(cluster_measure(api, torch, args.workload, local)), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def single_measure(api, torch, name, storage, steps, warmup, local, world=1, chunk_cols=0, gather="auto",
                   g=None, barrier=lambda: None):
    """Whole steps (CSR build from the device-resident edge list + Eq. 1 factors + Theta + L
    layers + output) of one single-graph workload, timed with CUDA events on the launching
    stream after warm-up; per-phase device times from the library's profile; clocks sampled
    during the timed region. Returns (dict, context for the end-to-end run)."""
    wl = synth.WORKLOADS[name]
    sb = 2 if storage == "bf16" else 4
    d, tau, L = wl["d"], wl["tau"], wl["L"]
    if g is None:
        g = synth.workload_graph(name)
    N, M = g.N, g.M
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    out = torch.empty((N, d), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    opts = api.embed_opts(storage=storage, chunk_cols=chunk_cols, gather=gather)
    probe = api.graph_build(src, dst, N)
    _, nnz, maxdeg = probe.info()
    probe.free()

    def step(prof=None):
        gr = api.graph_build(src, dst, N, stream=stream, profile=prof)
        opts.profile = prof.handle if prof is not None else None
        api.embed(gr, tau, L, d, 0, out=out, opts=opts, stream=stream)
        gr.free()

    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    prof = api.Profile()
    n0 = api.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step(prof)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = api.launch_count() - n0
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    phases = prof.read()
    prof.close()
    opts.profile = None
    units_step = float(nnz) * d * L
    layer_ms, layer_n = phases["layer"]
    avg_layer_s = layer_ms / max(layer_n, 1) / 1e3
    lb = layer_bytes(N, nnz, d, sb)
    peak, peak_src = peaks()
    achieved = lb / avg_layer_s / 1e9
    ffp_ms = sum(phases[k][0] for k in ("dinv", "theta", "layer", "output")) / steps
    res = {
        "value": replica_rate(units_step, steps, world, ms), "unit": UNIT, "ms_per_step": ms / steps,
        "units_per_step": units_step, "dtype": storage,
        "config": {"workload": name, **wl["graph"], "M_drawn": M, "nnz": int(nnz), "max_deg": int(maxdeg),
                   "d": d, "tau": tau, "L": L, "storage": storage, "accumulate": "f32",
                   "chunk_cols": chunk_cols or "auto", "gather": gather,
                   "l2": "inputs larger than L2 (edge list %d MB, T %d MB each > 129 MB)" % (
                       8 * M >> 20, N * d * sb >> 20) if N * d * sb > L2_BYTES else
                   "working set may fit L2 (inputs not flushed between steps)"},
        "phase_ms_per_step": {k: v[0] / steps for k, v in phases.items()},
        "ffp_only": {"value": units_step / (ffp_ms / 1e3), "unit": UNIT,
                     "what": "dinv + theta + L layers + output, CSR build excluded"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": recorded_traffic(name, storage), "kernel": "k_layer",
                     "algorithmic_bytes_per_launch": lb, "avg_launch_ms": avg_layer_s * 1e3,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else
                     "fallback 6800 GB/s"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    return res, dict(g=g, opts=opts, stream=stream, N=N, M=M, d=d, tau=tau, L=L, units_step=units_step, wl=wl)


def e2e_measure(api, torch, ctx, steps, world, barrier=lambda: None):
    """The same step through the public API with pinned host edges in and pinned host
    embeddings out (host<->device copies inside the timed region). Consecutive steps alternate
    between two CUDA streams, two device edge buffers and two output buffers, as a caller serving
    a stream of graphs would run them: step k+1's edges are uploaded (one copy per array) before
    step k is embedded, so that the upload is not queued behind step k's output copy; the CSR is
    built from the uploaded arrays (igp_graph_build), the embedding is written to pinned host
    memory asynchronously (opts.host_async: formed in device memory, copied by a copy engine),
    and step k-1's graph is synchronised and freed once step k is enqueued. Every step copies its
    own edges in and its own embeddings out."""
    g, opts, N, d, M = ctx["g"], ctx["opts"], ctx["N"], ctx["d"], ctx["M"]
    src_h = torch.from_numpy(g.src).pin_memory()
    dst_h = torch.from_numpy(g.dst).pin_memory()
    outs = [torch.empty((N, d), dtype=torch.float32).pin_memory() for _ in range(2)]
    edges = [(torch.empty(M, dtype=torch.int32, device="cuda"), torch.empty(M, dtype=torch.int32, device="cuda"))
             for _ in range(2)]
    # created streams: the legacy default stream would order every step after the previous one
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    aopts = type(opts)()
    ctypes.memmove(ctypes.byref(aopts), ctypes.byref(opts), ctypes.sizeof(opts))
    aopts.host_async = 1  # the call returns once the step is enqueued; sync() waits for its output

    def upload(k):
        with torch.cuda.stream(streams[k % 2]):
            edges[k % 2][0].copy_(src_h, non_blocking=True)
            edges[k % 2][1].copy_(dst_h, non_blocking=True)

    def run(n):
        prev = None
        upload(0)
        for k in range(n):
            if k + 1 < n:
                upload(k + 1)
            s = streams[k % 2]
            gr = api.graph_build(edges[k % 2][0], edges[k % 2][1], N, stream=s)
            api.embed(gr, ctx["tau"], ctx["L"], d, 0, out=outs[k % 2], opts=aopts, stream=s)
            if prev is not None:
                prev.sync()  # step k-1's embeddings are in host memory (and no wait ran out)
                prev.free()
            prev = gr
        prev.sync()
        prev.free()

    run(2)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    return {"value": replica_rate(ctx["units_step"], steps, world, e2e_s * 1e3), "unit": UNIT,
            "h2d_bytes_per_step": 2 * 4 * M, "d2h_bytes_per_step": N * d * 4, "steps": steps,
            "streams": 2,
            "pipeline": "per step: pinned host edges copied to a device buffer on the step's stream "
                        "(issued before the previous step's embedding), igp_graph_build on them, "
                        "igp_embed into pinned host memory with opts.host_async, igp_graph_sync of the "
                        "previous step; two streams alternate"}


def extras(api, torch, args, local):
    """The other configurations, measured in the same run as the headline: the 200K-node graph
    in both storages, the 512-graph batch and the served stream (keys of the headline line)."""
    out = {}
    for storage in ("f32", "bf16"):
        r, _ = single_measure(api, torch, "dcsbm-200k", storage, 20, 3, local)
        out[f"c2_{storage}"] = r
    wl = synth.BATCH_WORKLOADS["dcsbm-batch512"]
    out["batched"] = batch_measure(api, torch, "dcsbm-batch512", wl["storage"], wl["d"], 5, 3, local)
    wl = synth.SERVE_WORKLOADS["dcsbm-serve"]
    out["served"] = serve_measure(api, torch, "dcsbm-serve", wl["storage"], wl["d"], args.slots, args.batch_rows,
                                  3, local)
    out["streaming_vs_static"] = stream_measure(api, torch, "challenge-stream-100k", local)
    out["clustered"] = cluster_measure(api, torch, "challenge-cluster-1m", local)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in synth.STREAM_WORKLOADS:
        return 0 if dist_env()[0] != 0 else run_stream(args)
    if args.workload in synth.CLUSTER_WORKLOADS:
        return 0 if dist_env()[0] != 0 else run_cluster(args)
    if args.workload in synth.BATCH_WORKLOADS or args.workload in synth.SERVE_WORKLOADS:
        if dist_env()[0] != 0:  # one process runs these modes; other ranks have nothing to do
            return 0
        return run_batch(args) if args.workload in synth.BATCH_WORKLOADS else run_serve(args)
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = synth.WORKLOADS[args.workload]
    storage = args.storage or wl["storage"]
    res, ctx = single_measure(api, torch, args.workload, storage, args.steps, args.warmup, local, world,
                              args.chunk_cols, args.gather, barrier=barrier)
    e2e = e2e_measure(api, torch, ctx, args.e2e_steps or max(3, min(args.steps, 20)), world, barrier)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        ref = COracle(ctx["g"], wl)
        rate, dt = ref.run(wl["L"])
        cpu = {"value": rate, "unit": UNIT, "cores": ref.cores, "kind": "oracle", "sample": ref.describe(wl["L"], dt)}
    line = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": storage, "data": "synthetic",
        "config": {**res["config"], "parallelism": f"replicas{world}"},
        "phase_ms_per_step": res["phase_ms_per_step"],
        "ffp_only": res["ffp_only"],
        "roofline": res["roofline"],
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": res["gpu_launches"],
        "clocks": res["clocks"],
    }
    if world == 1 and not args.no_extras and args.workload == "dcsbm-2m" and args.storage is None:
        line.update(extras(api, torch, args, local))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
