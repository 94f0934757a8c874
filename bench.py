#!/usr/bin/env python3
"""Throughput of BVH traversal with subspace culling on one GB300.

Metric: Mrays/s, closest hit, culled traversal (the method: Alg. 4 with the
ray-mask / object-mask test of Sec. 3.1.2) against plain traversal of the
same BVH on the same GPU, identical hits asserted, with node and triangle
tests per ray.

One step = one pass of the path over one batch of rays, the rays already in
device memory: the primary wave (1920x1080 pinhole rays), then the diffuse
bounce wave(s) spawned from its hits, all in one cooperative launch replayed
from a CUDA graph, with block size, stack depth, refill batch and wave size
picked by the library's autotuner beforehand.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores instead (a bounded sample of rays per step).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, scene kind, scene args, ray kind, grid_res, compress)
    "hair1m": ("1,048,576 thin hair triangles (32,768 strands x 16 segments x 2) + "
               "2-triangle ground quad at y=-1.2, seed 2; 1920x1080 pinhole primary rays "
               "+ one cosine-weighted diffuse bounce wave; R=6 (216-bit) uncompressed masks, L=3",
               dict(strands=32768, ground=True, seed=2), (1920, 1080), 6, 0),
    "hair1m_comp": ("as hair1m with LUT-compressed masks (256 entries, 8-bit index)",
                    dict(strands=32768, ground=True, seed=2), (1920, 1080), 6, 1),
    "hair12m": ("12,100,000 thin hair triangles (378,125 strands x 16 x 2), seed 4; 1920x1080 "
                "pinhole primary rays + two diffuse bounce waves; R=6 LUT-compressed masks, L=3",
                dict(strands=378125, ground=False, seed=4), (1920, 1080), 6, 1),
    "hair12m_unc": ("as hair12m with uncompressed R=6 masks (216 bits per child in the node "
                    "record)", dict(strands=378125, ground=False, seed=4), (1920, 1080), 6, 0),
    "hair65k": ("65,536 hair triangles (2,048 strands), seed 1; 256x256 pinhole rays; R=6 "
                "uncompressed", dict(strands=2048, ground=False, seed=1), (256, 256), 6, 0),
    "soup4m": ("triangle soup stress: 4,194,304 triangles in the unit cube (50% slivers of "
               "aspect 1:1000, 50% axis-aligned slabs, edges log-uniform 1e-4..1e-1), seed 3; "
               "8,388,608 random rays (origins uniform in the cube, directions uniform on the "
               "sphere), closest hit (any hit reported beside); R=6 uncompressed masks, L=3",
               dict(soup=1 << 22, seed=3), (1 << 23, 0), 6, 0),
}


WORKLOAD_BOUNCES = {"hair1m": 1, "hair1m_comp": 1, "hair12m": 2, "hair12m_unc": 2, "hair65k": 1,
                    "soup4m": 0}


# DRAM traffic per launch of the timed kernel (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture, summarised in profiles/), valid
# only while the kernel source is the one that was measured: keyed by the
# workload and the kernel option set the autotuner chose (0; the
# shared-memory stack ring 128; 9 blocks per SM with the hit in shared
# memory 5120, and with the ring as well 5248), and checked against the
# SHA-256 of the traversal kernel header.
_TRAFFIC_SRC = "9bd81071782f1e9abad85e5c18b4b890c5d92ac0d691dd23f101de14390d4ced"
_P12, _P1 = "profiles/waves_kernel_hair12m.md", "profiles/waves_kernel_hair1m.md"
MEASURED_TRAFFIC = {
    # (workload, variant): (bytes per launch, kernel source sha256, profile summary)
    ("hair12m", 0): (1.870604e+09 + 3.807340e+08, _TRAFFIC_SRC, _P12),
    ("hair12m", 128): (1.472805e+09 + 2.905644e+08, _TRAFFIC_SRC, _P12),
    ("hair12m", 5120): (2.369406e+09 + 4.878799e+08, _TRAFFIC_SRC, _P12),
    ("hair12m", 5248): (1.751152e+09 + 3.291162e+08, _TRAFFIC_SRC, _P12),
    ("hair1m", 0): (1.721418e+09 + 2.544407e+08, _TRAFFIC_SRC, _P1),
    ("hair1m", 5120): (2.065885e+09 + 3.354545e+08, _TRAFFIC_SRC, _P1),
}


def traffic_bound(workload: str, variant: int, per_launch_bytes: float, default_config: bool):
    """(traffic, its profile, on chip?, why) for the culled kernel of a run.

    DRAM traffic far below the algorithmic bytes means the fetched bytes come
    from L2 (the working set of one frame stays there), so the L2 read
    bandwidth is the roofline; HBM otherwise.  Traffic is known only for the
    default configuration, and only for the option sets captured on the
    current kernel source.  Without a capture of the chosen option set the
    bound follows the captured option sets of the same source, if every one
    of them is on chip; the traffic then stays None."""
    limit = 0.25 * per_launch_bytes
    if not default_config:
        return None, None, False, ("not the default configuration: bound taken as HBM; the "
                                   "fraction against L2 is given beside it")
    traffic, src = measured_traffic(workload, variant)
    if traffic is not None:
        if traffic < limit:
            return traffic, src, True, (f"DRAM traffic {traffic / 1e9:.2f} GB per launch is "
                                        f"{100 * traffic / per_launch_bytes:.1f}% of the "
                                        f"algorithmic bytes")
        return traffic, src, False, "DRAM traffic is a large part of the algorithmic bytes"
    sibling = [t for t in (measured_traffic(w, v)[0] for (w, v) in MEASURED_TRAFFIC
                           if w == workload) if t is not None]
    if sibling and max(sibling) < limit:
        return None, None, True, (
            f"no DRAM capture of option set {variant}; the {len(sibling)} captured option "
            f"sets of this kernel source move {min(sibling) / 1e9:.2f}-"
            f"{max(sibling) / 1e9:.2f} GB per launch, at most "
            f"{100 * max(sibling) / per_launch_bytes:.1f}% of the algorithmic bytes")
    return None, None, False, ("no DRAM capture of this kernel source: bound taken as HBM; "
                               "the fraction against L2 is given beside it")


def measured_traffic(workload: str, variant: int = 0):
    import hashlib
    entry = MEASURED_TRAFFIC.get((workload, variant))
    if entry is None:
        return None, None
    src = os.path.join(ROOT, "paper_2305_08343_gb300", "csrc", "cuda", "trace_kernel.cuh")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    return (entry[0], entry[2]) if sha == entry[1] else (None, None)


def mean_wide_children(bvh) -> float:
    """Mean children of a 4-wide node: the nodes are the binary nodes at
    even depth, each with 2 + (its inner children) children."""
    e = bvh.export()
    child, count = e["child"], e["count"]
    nn = len(child)
    if nn == 0:
        return 2.0
    depth = np.full(nn, -1, np.int64)
    depth[0] = 0
    level = np.array([0])
    d = 0
    while level.size:
        inner = count[level] == 0
        nxt = child[level][inner]
        depth[nxt] = d + 1
        level, d = nxt, d + 1
    even = depth % 2 == 0
    kids = 2 + (count[even] == 0).sum(1)
    return float(kids.mean())


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest value of x over all ranks (x itself without a process
    group): the timed region of a multi-GPU run is the slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mrays(rays_per_rank_step: int, steps: int, world: int, max_total_ms: float) -> float:
    """Whole-job throughput: every rank traces its own copy of the workload
    (replicas, weak scaling), so the job traces world x the rays of one rank
    in the slowest rank's time."""
    return rays_per_rank_step * steps * world / (max_total_ms * 1e-3) / 1e6


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def measure_l2_peak(dev):
    """Best L2 read bandwidth (GB/s) of the library's probe kernel over
    buffers that stay in the 129 MB L2 (16-64 MB), each launch reading
    about 4 GB; CUDA events on the launching stream, warmed first."""
    import torch
    from paper_2305_08343_gb300 import subcull as sc
    sink = torch.zeros(sc.sc_l2_probe_blocks(), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    best, best_mb = 0.0, 0
    for mb in (16, 32, 48, 64):
        buf = torch.ones((mb << 20) // 4, dtype=torch.int32, device=dev)
        reps = max(1, (4 << 30) // (mb << 20))
        sc.sc_l2_read(buf, 1, sink)  # bring the buffer into L2
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sc.sc_l2_read(buf, reps, sink)
            e1.record(stream)
            e1.synchronize()
            gbs = (mb << 20) * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
            if gbs > best:
                best, best_mb = gbs, mb
        del buf
    return best, best_mb


def oracle_waves_per_s(ob, tris, rays, bounces, cull, threads, budget_s, seed, skip_bits=None,
                       stride=1, leaf_min=0, width=2):
    """Times the oracle on the GPU arm's work, bounded: an evenly spaced
    sample of the primary rays and the bounce waves their hits spawn (the
    oracle's own bounce generator, keyed by path id like the GPU's), sized
    to roughly budget_s seconds.  Threads split each wave statically; the
    time covers tracing and bounce generation.  Returns (rays/s, rays traced,
    primary sample, seconds, per-wave sizes)."""
    import oracle
    n = rays.shape[0]
    m = min(n, 512)
    t0 = time.perf_counter()
    ob.trace(rays[:m], 0, cull, skip_bits=skip_bits, stride=stride, leaf_min=leaf_min,
             width=width)
    per_ray = (time.perf_counter() - t0) / m
    sample = int(min(n, max(threads * 64,
                            budget_s * threads / max(per_ray * (1 + 0.9 * bounces), 1e-9))))
    idx = np.linspace(0, n - 1, sample).astype(np.int64)
    cur, path = np.ascontiguousarray(rays[idx]), idx
    total, sizes = 0, []
    t0 = time.perf_counter()
    for w in range(bounces + 1):
        k = cur.shape[0]
        out = dict(t=np.zeros(k, np.float32), id=np.zeros(k, np.int32),
                   uv=np.zeros((k, 2), np.float32), counts=np.zeros((k, 2), np.uint32),
                   mask_tests=np.zeros(k, np.uint32))
        bounds = np.linspace(0, k, threads + 1).astype(np.int64)
        ts = [threading.Thread(target=ob.trace, args=(cur, 0, cull, int(bounds[i]),
                                                       int(bounds[i + 1]), out, skip_bits,
                                                       stride, leaf_min, width))
              for i in range(threads)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        total += k
        sizes.append(k)
        if w < bounces:
            cur, path = oracle.bounce_wave(cur, out["t"], out["id"], tris, seed, w + 1, path)
            cur = np.ascontiguousarray(cur, dtype=np.float32)
    dt = time.perf_counter() - t0
    return total / dt, total, sample, dt, sizes


def make_inputs(name):
    from paper_2305_08343_gb300 import scenegen as sg
    desc, sargs, (W, H), R, comp = WORKLOADS[name]
    if "soup" in sargs:
        tris = sg.soup(sargs["soup"], seed=sargs["seed"])
        rays = sg.random_rays(W, seed=sargs["seed"])
    else:
        tris = sg.hair(sargs["strands"], 16, sargs["ground"], seed=sargs["seed"])
        rays = sg.pinhole(W, H)
    return desc, tris, rays, R, comp


# ------------------------------------------------------------- reference --

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    desc, tris, rays, R, comp = make_inputs(args.workload)
    bounces = args.bounces if args.bounces >= 0 else WORKLOAD_BOUNCES.get(args.workload, 1)
    threads = cpu_count()
    t0 = time.perf_counter()
    ob = oracle.OracleBVH(tris).build_masks(R, 3)
    cull = 1
    if comp:
        ob.compress(256, 8)
        cull = 2
    build_s = time.perf_counter() - t0
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_waves_per_s(ob, tris, rays, bounces, cull, threads, budget / 4, SEED)
    traced, secs, samples, sizes = [], [], [], None
    for _ in range(args.steps):
        _, tot, samp, dt, sizes = oracle_waves_per_s(ob, tris, rays, bounces, cull, threads,
                                                     budget, SEED)
        traced.append(tot)
        secs.append(dt)
        samples.append(samp)
    mrays = float(np.sum(traced) / np.sum(secs) / 1e6)
    sample_desc = (f"{int(np.mean(samples))} primary rays per step (evenly spaced over the "
                   f"{rays.shape[0]}) and the {bounces} bounce wave(s) their hits spawn "
                   f"(last step's wave sizes {sizes}), culled closest hit; the oracle's own "
                   f"threaded build ({build_s:.0f} s, untimed)")
    line = {
        "impl": "reference", "metric": METRIC, "value": mrays, "unit": "Mrays/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(secs) * 1e3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "bounces": bounces},
        "cpu_baseline": {"value": mrays, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                         "sample": sample_desc},
        "e2e": {"value": mrays, "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


METRIC = "Mrays/s closest-hit, culled vs plain, 1 GB300, identical hits; node+tri tests/ray"
SEED = 2305  # bounce-ray seed of every arm

# Kernel options (sc_trace_opts.variant) of the timed culled and plain wave
# kernels; neither changes a hit or a count.
DEFAULT_VARIANT = 0
DEFAULT_PLAIN_VARIANT = 0


# ------------------------------------------------------------------ gb300 --

def _sorted_waves(bufs, sizes):
    """Per wave: (path ids, hit records as int32 [m,4], counts [m,2]) sorted by
    path id (queue order differs between runs)."""
    import torch
    out = []
    for w, m in enumerate(sizes):
        m = int(m)
        path = bufs.path[w][:m]
        order = torch.argsort(path, stable=True)
        out.append((path[order], bufs.hits[w][:m].view(torch.int32)[order],
                    bufs.counts[w][:m][order] if bufs.counts[w] is not None else None))
    return out


# FLOPs of one network evaluation: 2 (6*64 + 64*64 + 64*256)
NET_FLOPS_PER_RAY = 2 * (6 * 64 + 64 * 64 + 64 * 256)


def seeding_upper_bound(lp, d_masked, rays, bounces, dev):
    """What seeding can gain at best, per wave: node + triangle tests per ray
    of the culled traversal, and of the seeded traversal given every ray's
    true class (the frontier subtree of its closest hit; misses unseeded),
    over one batch of rays and the bounce waves its hits spawn."""
    import torch
    from paper_2305_08343_gb300 import subcull as sc
    n = rays.shape[0]
    bufs = sc.WaveBuffers(n, bounces, with_counts=True, device=dev, with_rays=True)
    _, sizes = sc.trace_waves(d_masked, rays, bounces, SEED, 1, bufs)
    out = {}
    for w in range(bounces + 1):
        m = int(sizes[w])
        if m == 0:
            continue
        r = bufs.rays[w][:m].contiguous()
        hid = bufs.hits[w][:m, 1].contiguous().view(torch.int32)
        lab = torch.where(hid >= 0, lp.class_of_tri[hid.clamp(min=0).long()].int(),
                          torch.full_like(hid, -1))
        cnt = torch.empty((m, 2), dtype=torch.int32, device=dev)
        hits = lp.trace(d_masked, r, lab, counts=cnt)
        torch.cuda.synchronize()
        same = bool(torch.equal(hits.view(torch.int32),
                                bufs.hits[w][:m].contiguous().view(torch.int32)))
        culled = bufs.counts[w][:m].double().sum(1).mean().item()
        seeded = cnt.double().sum(1).mean().item()
        out[f"wave{w}"] = {"rays": m, "culled_node_plus_tri": culled,
                           "true_label_node_plus_tri": seeded,
                           "change": seeded / culled - 1.0, "identical_hits": same}
    return out


def run_learned(args, bvh, d_masked, dev, flush, W, H, bounces):
    """Learned proposal against culled traversal on held-out rays: first the
    true-label upper bound per wave (what any seeding could gain); then
    training on the GPU (pairs from the plain traversal of jittered primary
    rays, or random rays for the soup, and their bounce waves), then [network
    top-1 + seeded traversal] and [culled traversal] timed on 2^22 held-out
    rays (other seeds), identical hits asserted."""
    import torch

    from paper_2305_08343_gb300 import learned
    from paper_2305_08343_gb300 import scenegen as sg
    from paper_2305_08343_gb300 import subcull as sc

    def batch_of_rays(seed):
        # camera workloads: jittered primary rays; the soup: random rays
        if H > 0:
            return learned.primary_rays(W, H, seed, device=dev)
        return torch.from_numpy(sg.random_rays(W, seed=seed)).to(dev)

    t0 = time.perf_counter()
    lp = learned.LearnedProposal(bvh, depth=8, seed=0, device=dev)
    bounds = seeding_upper_bound(lp, d_masked, batch_of_rays(4242), bounces, dev)
    target = args.learned_pairs
    pairs_r, pairs_l, total, s = [], [], 0, 1
    while total < target and s <= 64:
        rays = batch_of_rays(1000 + s)
        r, l = lp.collect(d_masked, [rays], bounces=bounces, seed=77 + s)
        pairs_r.append(r.clone())
        pairs_l.append(l.clone())
        total += r.shape[0]
        s += 1
    tr_r = torch.cat(pairs_r)[:target]
    tr_l = torch.cat(pairs_l)[:target]
    del pairs_r, pairs_l
    collect_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = lp.fit(tr_r, tr_l, steps=args.learned_steps, batch=4096, lr=3e-3, seed=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    n_held = 1 << 22
    per = W * max(H, 1)
    held = torch.cat([batch_of_rays(5 + k)
                      for k in range((n_held + per - 1) // per)])[:n_held].contiguous()
    n = held.shape[0]
    cls = torch.empty(n, dtype=torch.int32, device=dev)
    hits_s = torch.empty((n, 4), dtype=torch.float32, device=dev)
    hits_p = torch.empty((n, 4), dtype=torch.float32, device=dev)
    cnt_s = torch.empty((n, 2), dtype=torch.int32, device=dev)
    cnt_p = torch.empty((n, 2), dtype=torch.int32, device=dev)
    work = torch.empty(sc.sc_trace_workspace_bytes(), dtype=torch.uint8, device=dev)
    out = {"training_pairs": int(tr_r.shape[0]), "train_steps": args.learned_steps,
           "batch": 4096, "final_loss": loss, "collect_s": collect_s, "train_s": train_s,
           "held_out_rays": n, "frontier": lp.n_frontier,
           "true_label_upper_bound": bounds}
    stream = torch.cuda.current_stream()
    for min_prob in (0.0, 0.8):
        key = "top1" if min_prob == 0.0 else f"top1_p{min_prob}"
        lp.predict(held, cls, min_prob=min_prob)
        lp.trace(d_masked, held, cls, hits_s, cnt_s, 1, work)
        sc.sc_trace(d_masked, held, hits_p, cnt_p, 0, 1, work)
        torch.cuda.synchronize()
        same = bool(torch.equal(hits_s.view(torch.int32), hits_p.view(torch.int32)))
        ts = cnt_s.double().mean(0).tolist()
        tp = cnt_p.double().mean(0).tolist()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ms_l, ms_p, ms_net = [], [], []
        for _ in range(args.warmup):
            lp.predict(held, cls, min_prob=min_prob)
            lp.trace(d_masked, held, cls, hits_s, None, 1, work)
            sc.sc_trace(d_masked, held, hits_p, None, 0, 1, work)
        for _ in range(args.steps):
            flush.zero_()
            ev[0].record(stream)
            lp.predict(held, cls, min_prob=min_prob)
            ev[1].record(stream)
            lp.trace(d_masked, held, cls, hits_s, None, 1, work)
            ev[2].record(stream)
            flush.zero_()
            ev[3].record(stream)
            sc.sc_trace(d_masked, held, hits_p, None, 0, 1, work)
            e4 = torch.cuda.Event(enable_timing=True)
            e4.record(stream)
            torch.cuda.synchronize()
            ms_net.append(ev[0].elapsed_time(ev[1]))
            ms_l.append(ev[0].elapsed_time(ev[2]))
            ms_p.append(ev[3].elapsed_time(e4))
        sc.sc_status_poll(work)
        peaks = load_peaks() or {}
        bf16 = peaks.get("bf16_tflops", 1900.0)
        net_tflops = n * NET_FLOPS_PER_RAY / (np.mean(ms_net) * 1e-3) / 1e12
        out[key] = {
            "network_roofline": {"bound": "tensor", "achieved": net_tflops, "peak": bf16,
                                 "unit": "TFLOP/s", "frac": net_tflops / bf16,
                                 "peak_source": "measured" if "bf16_tflops" in peaks
                                 else "fallback", "flops_per_ray": NET_FLOPS_PER_RAY,
                                 "kernel": "infer_tc_kernel (tcgen05)"},
            "identical_hits": same,
            "seeded_fraction": float((cls >= 0).double().mean().item()),
            "learned_mrays_s": n / (np.mean(ms_l) * 1e-3) / 1e6,
            "network_ms": float(np.mean(ms_net)),
            "plain_culled_mrays_s": n / (np.mean(ms_p) * 1e-3) / 1e6,
            "tests_per_ray": {"learned": {"node": ts[0], "tri": ts[1]},
                              "plain_culled": {"node": tp[0], "tri": tp[1]}}}
    return out


def run_gpu(args):
    import torch

    from paper_2305_08343_gb300 import subcull as sc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py: no CUDA device (the product has no CPU fallback)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    desc, tris, rays_np, R, comp = make_inputs(args.workload)
    if args.R:
        R = args.R
    bounces = args.bounces if args.bounces >= 0 else WORKLOAD_BOUNCES.get(args.workload, 1)
    t0 = time.perf_counter()
    gpu_build = 0 if args.host_build else 1
    bvh = sc.sc_bvh_build(tris, R, comp, skip_bits=args.skip_bits, L=args.L,
                          test_stride=args.stride, leaf_min_tris=args.leaf_min,
                          max_leaf=args.max_leaf, gpu_masks=gpu_build, gpu_bvh=gpu_build)
    build_s = time.perf_counter() - t0
    info = bvh.info()
    wide = args.width == 4
    d_masked = sc.DeviceBVH(bvh, sc.SC_LAYOUT_MASKED4 if wide else args.layout)
    d_plain = sc.DeviceBVH(bvh, sc.SC_LAYOUT_PLAIN4 if wide else sc.SC_LAYOUT_PLAIN)
    n = rays_np.shape[0]
    rays = torch.from_numpy(rays_np).to(dev)
    opts = sc._opts(lut_mode=args.lut, refill=args.refill,
                    variant=max(args.variant, 0) if args.variant >= 0 else DEFAULT_VARIANT)
    opts_plain = sc._opts(refill=args.refill,  # the plain kernel looks nothing up
                          variant=args.plain_variant if args.plain_variant >= 0
                          else DEFAULT_PLAIN_VARIANT)
    seed = SEED
    if args.primary_only:
        # a few single-batch traces (culled, then plain) and nothing else:
        # the command used for ncu captures of trace_kernel
        hits = torch.empty((n, 4), dtype=torch.float32, device=dev)
        work = torch.empty(sc.sc_trace_workspace_bytes(), dtype=torch.uint8, device=dev)
        for dbvh, cull in ((d_masked, 1), (d_plain, 0)):
            for _ in range(max(1, args.steps)):
                sc.sc_trace(dbvh, rays, hits, None, 0, cull, work, opts if cull else opts_plain)
        sc.sc_status_poll(work)
        torch.cuda.synchronize()
        print(json.dumps({"primary_only": True, "workload": args.workload, "rays": n}))
        return 0
    if args.waves_once:
        # one culled and one plain wave pipeline launch (default launch
        # options) and nothing else: the command used for ncu captures of
        # waves_kernel
        for dbvh, cull in ((d_masked, 1), (d_plain, 0)):
            b = sc.WaveBuffers(n, bounces, with_counts=False, device=dev)
            sc.sc_trace_waves(dbvh, rays, bounces, seed, cull, b.outs(), b.ws,
                              opts if cull else opts_plain)
            sizes = sc.sc_waves_poll(b.ws, bounces)
            del b
        print(json.dumps({"waves_once": True, "workload": args.workload, "rays": n,
                          "wave_sizes": [int(x) for x in sizes]}))
        return 0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    # reference passes with counts (untimed): wave sizes, identical hits, tests per ray
    ref_c = sc.WaveBuffers(n, bounces, with_counts=True, device=dev)
    ref_p = sc.WaveBuffers(n, bounces, with_counts=True, device=dev)
    _, sizes = sc.trace_waves(d_masked, rays, bounces, seed, 1, ref_c, opts)
    _, sizes_p = sc.trace_waves(d_plain, rays, bounces, seed, 0, ref_p, opts_plain)
    wc, wpl = _sorted_waves(ref_c, sizes), _sorted_waves(ref_p, sizes_p)
    same = bool(np.array_equal(sizes, sizes_p)) and all(
        torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(wc, wpl))
    le = all(bool((a[2] <= b[2]).all().item()) for a, b in zip(wc, wpl))
    cat_c = torch.cat([x[2] for x in wc]).double()
    cat_p = torch.cat([x[2] for x in wpl]).double()
    cnt_c, cnt_p = cat_c.mean(0).tolist(), cat_p.mean(0).tolist()

    def pct(cat):
        # p50 / p99 of node, tri and node + tri tests per ray
        q = torch.tensor([0.5, 0.99], dtype=torch.float64, device=cat.device)
        both = torch.cat([cat, cat.sum(1, keepdim=True)], 1)
        sample = both[torch.linspace(0, both.shape[0] - 1, min(both.shape[0], 1 << 22),
                                     device=cat.device).long()]
        v = torch.quantile(sample, q, dim=0).cpu().numpy()
        return {"p50": {"node": v[0, 0], "tri": v[0, 1], "node_plus_tri": v[0, 2]},
                "p99": {"node": v[1, 0], "tri": v[1, 1], "node_plus_tri": v[1, 2]}}

    pct_c, pct_p = pct(cat_c), pct(cat_p)
    rays_per_step = int(np.sum(sizes))
    hit_ref_c = [x[1].clone() for x in wc]
    del ref_c, ref_p, wc, wpl, cat_c, cat_p

    bufs_c = sc.WaveBuffers(n, bounces, with_counts=False, device=dev)
    bufs_p = sc.WaveBuffers(n, bounces, with_counts=False, device=dev)

    # autotuner: block size, stack depth, refill batch and wave chunk, per variant
    tuned = {}
    opts_c, opts_p = opts, opts_plain
    if not args.no_autotune:
        t0 = time.perf_counter()
        opts_c, rows_c = sc.sc_autotune_waves(d_masked, rays, bounces, seed, 1, bufs_c, opts, 3,
                                              flush)
        opts_p, rows_p = sc.sc_autotune_waves(d_plain, rays, bounces, seed, 0, bufs_p, opts_plain, 3,
                                              flush)
        pick = lambda o: {"block": o.block, "stack": o.stack, "refill": o.refill,
                          "wave_chunk": int(o.wave_chunk), "variant": o.variant}
        tuned = {"culled": pick(opts_c), "plain": pick(opts_p), "candidates": len(rows_c),
                 "seconds": time.perf_counter() - t0}

    def capture(dbvh, cull, bufs):
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream())
        o = opts_c if cull else opts_p
        with torch.cuda.stream(side):
            for _ in range(2):
                sc.sc_trace_waves(dbvh, rays, bounces, seed, cull, bufs.outs(), bufs.ws, o)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sc.sc_trace_waves(dbvh, rays, bounces, seed, cull, bufs.outs(), bufs.ws, o)
        return g

    graphs = None
    try:
        graphs = (capture(d_masked, 1, bufs_c), capture(d_plain, 0, bufs_p))
    except Exception as e:  # report, then time eager launches
        graphs = None
        graph_error = str(e)

    def step(i_graph, dbvh, cull, bufs):
        if graphs is not None:
            graphs[i_graph].replay()
        else:
            sc.sc_trace_waves(dbvh, rays, bounces, seed, cull, bufs.outs(), bufs.ws,
                              opts_c if cull else opts_p)

    def timed(i_graph, dbvh, cull, bufs):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for _ in range(args.warmup):
            flush.zero_()
            step(i_graph, dbvh, cull, bufs)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        # an NVTX range around the timed steps, so that a profiler can be
        # limited to them (ncu --nvtx --nvtx-include "timed_culled/")
        torch.cuda.nvtx.range_push("timed_culled" if cull else "timed_plain")
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(i_graph, dbvh, cull, bufs)
            ev[i][1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return [a.elapsed_time(b) for a, b in ev]

    with ClockSampler(local) as clk:
        ms_cull = timed(0, d_masked, 1, bufs_c)
        ms_plain = timed(1, d_plain, 0, bufs_p)
    sc.sc_waves_poll(bufs_c.ws, bounces)
    sc.sc_waves_poll(bufs_p.ws, bounces)
    tot_cull = max_over_ranks(float(np.sum(ms_cull)), dist, dev)
    value = whole_job_mrays(rays_per_step, args.steps, world, tot_cull)
    plain_value = rays_per_step * args.steps / (float(np.sum(ms_plain)) * 1e-3) / 1e6

    # primary wave alone (single-batch sc_trace), for context
    hits1 = torch.empty((n, 4), dtype=torch.float32, device=dev)
    work = torch.empty(sc.sc_trace_workspace_bytes(), dtype=torch.uint8, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    prim = {}
    for name, dbvh, cull in (("culled", d_masked, 1), ("plain", d_plain, 0),
                             ("plain_kernel_on_masked_image", d_masked, 0)):
        o1 = opts if cull else (opts_plain if dbvh is d_plain else sc._opts(lut_mode=args.lut))
        for _ in range(2):
            sc.sc_trace(dbvh, rays, hits1, None, 0, cull, work, o1)
        flush.zero_()
        ev[0].record(stream)
        for _ in range(3):
            sc.sc_trace(dbvh, rays, hits1, None, 0, cull, work, o1)
        ev[1].record(stream)
        torch.cuda.synchronize()
        prim[name] = 3 * n / (ev[0].elapsed_time(ev[1]) * 1e-3) / 1e6
    anyhit = {}
    if bounces == 0:
        for name, dbvh, cull in (("culled", d_masked, 1), ("plain", d_plain, 0)):
            o1 = opts if cull else opts_plain
            sc.sc_trace(dbvh, rays, hits1, None, 1, cull, work, o1)
            flush.zero_()
            ev[2].record(stream)
            for _ in range(3):
                sc.sc_trace(dbvh, rays, hits1, None, 1, cull, work, o1)
            ev[3].record(stream)
            torch.cuda.synchronize()
            anyhit[name] = 3 * n / (ev[2].elapsed_time(ev[3]) * 1e-3) / 1e6

    # end to end through the C-ABI with host buffers: every step is one
    # sc_trace_waves_host call, which copies the step's rays from pinned host
    # memory, runs the wave pipeline, reads the wave sizes and copies every
    # wave's hits back to pinned host memory, then synchronizes.
    h_rays = torch.from_numpy(rays_np).pin_memory()
    h_outs = [(torch.empty((n, 4), dtype=torch.float32).pin_memory(), None, None, None)
              for _ in range(bounces + 1)]
    d_rays_e = torch.empty((n, 8), dtype=torch.float32, device=dev)
    s_e2e = torch.cuda.Stream(device=dev)

    def e2e_run(k_steps):
        szs = None
        for _ in range(k_steps):
            szs = sc.sc_trace_waves_host(d_masked, h_rays, bounces, seed, 1, h_outs, d_rays_e,
                                         bufs_c.outs(), bufs_c.ws, opts_c, stream=s_e2e)
        return szs

    e2e_run(max(2, args.warmup))
    t0 = time.perf_counter()
    szs = e2e_run(args.steps)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": rays_per_step * args.steps / e2e_s / 1e6, "unit": "Mrays/s",
           "h2d_bytes_per_step": n * 32, "d2h_bytes_per_step": int(np.sum(szs)) * 16,
           "call": "sc_trace_waves_host (host rays in, every wave's hits out, synchronous)"}
    ok_e2e = [int(x) for x in szs] == [int(x) for x in sizes]
    e2e["identical_wave_sizes"] = ok_e2e

    # roofline of the wave kernel.  Algorithmic bytes per ray (the method's
    # own fetches, from the exact per-ray counters): 32 (ray) + 16 (hit) +
    # node visits x B_node + triangle tests x 48, plus 32 per spawned bounce
    # ray.  B_node is the method's record: a 64-byte child pair, plus the two
    # R^3-bit masks when uncompressed (80 / 128 / 192 bytes at R = 4 / 6 / 8);
    # the image's own records (stored scales, 4-wide layouts) are reported
    # beside it as record_bytes_per_ray.
    mstride = {4: 8, 6: 32, 8: 64}[R]
    b_node = 64 + (0 if comp else 2 * mstride)
    if wide:
        # a 4-wide node is made from every binary node at even depth and
        # holds 2 + its inner children: node tests / mean children = visits
        rec_bytes = 176 if comp else 192 + 4 * mstride
        visits = cnt_c[0] / mean_wide_children(bvh)
        b_node_w = 2 * b_node
    else:
        rec_bytes = (96 if args.layout in (1, 5) else 64) + (0 if comp else 2 * mstride)
        rec_bytes = (rec_bytes + 31) // 32 * 32  # records are whole 32-byte sectors
        visits = cnt_c[0] / 2.0
        b_node_w = b_node
    spawned = float(np.sum(sizes[1:])) / rays_per_step
    b_ray = 32 + 16 + visits * b_node_w + cnt_c[1] * 48 + spawned * 32
    b_ray_rec = 32 + 16 + 4 + visits * rec_bytes + cnt_c[1] * 48 + spawned * (32 + 4)
    per_launch_bytes = b_ray * rays_per_step
    avg_ms = float(np.mean(ms_cull))
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
    peaks = load_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    default_config = not (args.layout != 1 or args.R or args.lut or args.skip_bits
                          or args.stride != 1 or args.leaf_min or args.L != 3
                          or args.max_leaf != 4 or wide
                          or bounces != WORKLOAD_BOUNCES.get(args.workload, 1)
                          or opts.variant != DEFAULT_VARIANT)
    traffic, traffic_src, on_chip, bound_basis = traffic_bound(
        args.workload, opts_c.variant, per_launch_bytes, default_config)
    l2_peak, l2_mb = measure_l2_peak(dev)
    bound_l2 = on_chip and bool(l2_peak)
    peak = l2_peak if bound_l2 else hbm_peak
    roofline = {"bound": "l2" if bound_l2 else "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_source": traffic_src, "bound_basis": bound_basis,
                "peak_source": ("measured (sc_l2_read probe, this run)" if bound_l2 else
                                ("measured" if peaks else "fallback")),
                "bytes_per_ray": b_ray, "b_node": b_node, "node_visits_per_ray": visits,
                "record_bytes_per_ray": b_ray_rec, "record_bytes": rec_bytes,
                "kernel": "waves_kernel (culled)",
                "hbm_peak": hbm_peak, "frac_hbm": achieved / hbm_peak,
                "l2_peak": l2_peak, "frac_l2": achieved / l2_peak if l2_peak else None,
                "l2_peak_source": f"sc_l2_read probe, best over 16-64 MB resident buffers "
                                  f"({l2_mb} MB), measured in this run"}

    def measure_alt(comp_a, **build_kw):
        """Culled waves on another mask build of the same tree (the GPU tree
        builder is deterministic): counted pass, autotune, then the bench's
        warm-up and timed steps with the L2 flushed before each."""
        bvh_a = sc.sc_bvh_build(tris, R, comp_a, max_leaf=args.max_leaf, gpu_masks=gpu_build,
                                gpu_bvh=gpu_build, **build_kw)
        d_a = sc.DeviceBVH(bvh_a, args.layout)
        o_a = sc._opts(refill=args.refill)
        ref_a = sc.WaveBuffers(n, bounces, with_counts=True, device=dev)
        _, sizes_a = sc.trace_waves(d_a, rays, bounces, seed, 1, ref_a, o_a)
        wa = _sorted_waves(ref_a, sizes_a)
        same_a = bool(np.array_equal(sizes_a, sizes))
        cnt_a = torch.cat([x[2] for x in wa]).double().mean(0).tolist()
        del ref_a
        bufs_a = sc.WaveBuffers(n, bounces, with_counts=False, device=dev)
        opts_a, _ = sc.sc_autotune_waves(d_a, rays, bounces, seed, 1, bufs_a, o_a, 3, flush)
        ms_a = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sc.sc_trace_waves(d_a, rays, bounces, seed, 1, bufs_a.outs(), bufs_a.ws, opts_a)
            e1.record(stream)
            e1.synchronize()
            if i >= args.warmup:
                ms_a.append(e0.elapsed_time(e1))
        sc.sc_waves_poll(bufs_a.ws, bounces)
        same_a = same_a and all(torch.equal(x[1], h) for x, h in zip(wa, hit_ref_c))
        v_a = rays_per_step * len(ms_a) / (float(np.sum(ms_a)) * 1e-3) / 1e6
        out = {"mrays_s": v_a, "speedup_vs_plain": v_a / plain_value, "identical_hits": same_a,
               "tests_per_ray": {"node": cnt_a[0], "tri": cnt_a[1],
                                 "node_plus_tri": cnt_a[0] + cnt_a[1]},
               "autotuned": {"block": opts_a.block, "stack": opts_a.stack,
                             "refill": opts_a.refill, "variant": opts_a.variant},
               "build_ms": {"bvh": bvh_a.info().ms_bvh, "masks": bvh_a.info().ms_masks,
                            "compress": bvh_a.info().ms_compress}}
        del d_a, bvh_a, bufs_a, wa
        torch.cuda.empty_cache()
        return out

    # Test selection (an option beside the paper's method, which tests
    # every child): children whose decoded mask has at least skip_bits bits
    # set are kept untested.  Same hits; counts between the fully tested
    # culled traversal's and plain's (the oracle applies the same rule).
    tuned_policy = None
    uncompressed_alt = None
    if not args.no_policy and not wide and args.skip_bits == 0:
        kbits = max(1, (R ** 3 * 5) // 9)  # 120 of 216 bits at R = 6
        tuned_policy = measure_alt(comp, skip_bits=kbits, L=args.L)
        tuned_policy = {"skip_bits": kbits, **tuned_policy,
                        "note": "children whose decoded mask has >= skip_bits of R^3 bits set "
                                "are kept untested (not the paper's policy)"}
        if comp and R == 6:
            # the same scene with uncompressed masks, deeper mask approximation
            # (L = 8) and masks of >= 160 of 216 bits untested: the best
            # culled configuration measured on this tree
            uncompressed_alt = {"compressed": False, "L": 8, "skip_bits": 160,
                                **measure_alt(0, skip_bits=160, L=8),
                                "note": "uncompressed 216-bit masks in the node record "
                                        "(160-byte records), L = 8; masks with >= 160 bits "
                                        "set kept untested"}

    learned_out = None
    if not args.no_learned:
        W, H = WORKLOADS[args.workload][2]
        d_learn = sc.DeviceBVH(bvh, args.layout) if wide else d_masked  # binary frontier
        learned_out = run_learned(args, bvh, d_learn, dev, flush, W, H, bounces)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ob = oracle.OracleBVH(tris).build_masks(R, args.L)
        cull_mode = 1
        if comp:
            ob.compress(256, 8)
            cull_mode = 2
        ob_s = time.perf_counter() - t0
        thr = cpu_count()
        v, tot, sample, dt, wsz = oracle_waves_per_s(ob, tris, rays_np, bounces, cull_mode, thr,
                                                     15.0, SEED, args.skip_bits or R ** 3,
                                                     args.stride, args.leaf_min, args.width)
        vp, tot_p, sample_p, dt_p, _ = oracle_waves_per_s(ob, tris, rays_np, bounces, 0, thr,
                                                          6.0, SEED)
        cpu = {"value": v / 1e6, "unit": "Mrays/s", "cores": thr, "kind": "oracle",
               "sample": f"{sample} primary rays evenly spaced over the {n} and the bounce "
                         f"waves they spawn ({wsz} rays), culled closest hit, {dt:.1f} s on "
                         f"{thr} threads (the oracle's own BVH, masks and LUT, built in "
                         f"{ob_s:.0f} s untimed)",
               "plain_value": vp / 1e6,
               "plain_sample": f"{tot_p} rays ({sample_p} primary + bounces), plain closest "
                               f"hit, {dt_p:.1f} s"}
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms_cull)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "primary_rays": n,
                   "bounces": bounces, "rays_per_step": rays_per_step,
                   "wave_sizes": [int(x) for x in sizes], "grid_res": R,
                   "compressed": bool(comp), "L": args.L, "lut_mode": args.lut,
                   "layout": args.layout, "refill": args.refill,
                   "skip_bits": args.skip_bits or R ** 3, "test_stride": args.stride,
                   "leaf_min_tris": args.leaf_min, "max_leaf": args.max_leaf,
                   "node_width": args.width,
                   "gpu_masks": bool(gpu_build), "gpu_bvh": bool(gpu_build),
                   "variant": opts.variant, "plain_variant": opts_plain.variant,
                   "cuda_graph": graphs is not None,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "plain_mrays_s": plain_value, "speedup_vs_plain": value / world / plain_value,
        "primary_only_mrays_s": prim, "any_hit_mrays_s": anyhit or None,
        "autotuned": tuned or None,
        "identical_hits": same, "culled_counts_le_plain": le,
        "tests_per_ray": {"culled": {"node": cnt_c[0], "tri": cnt_c[1],
                                     "node_plus_tri": cnt_c[0] + cnt_c[1],
                                     **{k: {a: float(b) for a, b in v.items()}
                                        for k, v in pct_c.items()}},
                          "plain": {"node": cnt_p[0], "tri": cnt_p[1],
                                    "node_plus_tri": cnt_p[0] + cnt_p[1],
                                    **{k: {a: float(b) for a, b in v.items()}
                                       for k, v in pct_p.items()}}},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "learned_proposal": learned_out, "culled_dense_masks_untested": tuned_policy,
        "culled_uncompressed_l8": uncompressed_alt,
        "gpu_launches": args.steps,
        "build_s": build_s, "bvh": {"nodes": info.num_nodes, "max_depth": info.max_depth,
                                    "ms_bvh": info.ms_bvh, "ms_masks": info.ms_masks,
                                    "ms_compress": info.ms_compress},
    }
    if graphs is None:
        line["config"]["cuda_graph_error"] = graph_error
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="hair12m", choices=sorted(WORKLOADS))
    ap.add_argument("--lut", type=int, default=0,
                    help="0 auto, 1 global table, 2 shared, 3 bit table, 4 the R_ray = 2R table, "
                         "5 factored tables through L1 (R = 6 uncompressed)")
    ap.add_argument("--layout", type=int, default=1,
                    help="1 masked (Alg. 1 scales stored per child), 2 compact (scales "
                         "divided), 5 masked plus the R_ray = 2R table")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--refill", type=int, default=0, help="idle lanes before a warp refills")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--bounces", type=int, default=-1, help="bounce waves (-1: workload's)")
    ap.add_argument("--R", type=int, default=0, help="mask resolution (0: workload's)")
    ap.add_argument("--L", type=int, default=3, help="mask approximation depth (Sec. 3.2.1)")
    ap.add_argument("--stride", type=int, default=1,
                    help="test inner children only at depths that are multiples of this")
    ap.add_argument("--primary-only", action="store_true",
                    help="only a few single-batch traces (for ncu captures)")
    ap.add_argument("--waves-once", action="store_true",
                    help="one culled and one plain wave-pipeline launch (for ncu captures)")
    ap.add_argument("--max-leaf", type=int, default=4, help="triangles per BVH leaf (1..8)")
    ap.add_argument("--width", type=int, default=2, choices=[2, 4],
                    help="children per node record: 2 (binary) or 4 (4-wide layouts)")
    ap.add_argument("--host-build", action="store_true",
                    help="build the tree and the masks on the host cores instead of the GPU "
                         "(the same tree and bits)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="kernel options of the culled traversal (SC_VARIANT_* bits; "
                         "-1: the library's default)")
    ap.add_argument("--plain-variant", type=int, default=-1,
                    help="kernel options of the plain traversal (-1: the library's default)")
    ap.add_argument("--leaf-min", type=int, default=0,
                    help="keep leaf children with fewer triangles untested (0: test all)")
    ap.add_argument("--skip-bits", type=int, default=0,
                    help="keep children with >= this many mask bits untested (0: R^3)")
    ap.add_argument("--no-policy", action="store_true",
                    help="skip the culled run with dense masks kept untested")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned proposal (trained on the GPU, then timed against "
                         "culled traversal on held-out rays)")
    ap.add_argument("--learned-pairs", type=int, default=1 << 24)
    ap.add_argument("--learned-steps", type=int, default=4000)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
