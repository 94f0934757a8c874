#!/usr/bin/env python3
"""Throughput of BVH traversal with subspace culling on one GB300.

Metric: Mrays/s, closest hit, culled traversal (the method: Alg. 4 with the
ray-mask / object-mask test of Sec. 3.1.2) against plain traversal of the
same BVH on the same GPU, identical hits asserted, with node and triangle
tests per ray.

One step = one pass of the path over one batch of rays, the rays already in
device memory: the primary wave (1920x1080 pinhole rays), then the diffuse
bounce wave spawned from its hits, each traced with culling.

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
                "pinhole primary rays + one diffuse bounce wave; R=6 LUT-compressed masks, L=3",
                dict(strands=378125, ground=False, seed=4), (1920, 1080), 6, 1),
    "hair65k": ("65,536 hair triangles (2,048 strands), seed 1; 256x256 pinhole rays; R=6 "
                "uncompressed", dict(strands=2048, ground=False, seed=1), (256, 256), 6, 0),
}


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


def oracle_rays_per_s(ob, tris, rays, cull, threads, budget_s):
    """Times the oracle's traversal (threads split the rays statically) on a
    sample of rays sized to roughly budget_s seconds of CPU time."""
    import oracle  # noqa: F401  (the oracle package; CPU baseline only)
    n = rays.shape[0]
    # calibrate on a small sample
    m = min(n, 512)
    t0 = time.perf_counter()
    ob.trace(rays[:m], 0, cull)
    per_ray = (time.perf_counter() - t0) / m
    sample = int(min(n, max(threads * 256, budget_s * threads / max(per_ray, 1e-9))))
    idx = np.linspace(0, n - 1, sample).astype(np.int64)
    sub = np.ascontiguousarray(rays[idx])
    out = dict(t=np.zeros(sample, np.float32), id=np.zeros(sample, np.int32),
               uv=np.zeros((sample, 2), np.float32), counts=np.zeros((sample, 2), np.uint32),
               mask_tests=np.zeros(sample, np.uint32))
    bounds = np.linspace(0, sample, threads + 1).astype(np.int64)
    ts = [threading.Thread(target=ob.trace, args=(sub, 0, cull, int(bounds[i]),
                                                   int(bounds[i + 1]), out))
          for i in range(threads)]
    t0 = time.perf_counter()
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    dt = time.perf_counter() - t0
    return sample / dt, sample, dt, out


def make_inputs(name):
    from paper_2305_08343_gb300 import scenegen as sg
    desc, sargs, (W, H), R, comp = WORKLOADS[name]
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
    threads = cpu_count()
    ob = oracle.OracleBVH(tris).build_masks(R, 3)
    cull = 1
    if comp:
        ob.compress(256, 8)
        cull = 2
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rays_per_s(ob, tris, rays, cull, threads, budget / 4)
    vals, samples, secs = [], [], []
    for _ in range(args.steps):
        v, s, dt, _ = oracle_rays_per_s(ob, tris, rays, cull, threads, budget)
        vals.append(v)
        samples.append(s)
        secs.append(dt)
    mrays = float(np.sum(samples) / np.sum(secs) / 1e6)
    line = {
        "impl": "reference", "metric": METRIC, "value": mrays, "unit": "Mrays/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(secs) * 1e3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc},
        "cpu_baseline": {"value": mrays, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                         "sample": f"{int(np.mean(samples))} primary rays per step (evenly "
                                   f"spaced over the {rays.shape[0]}), culled closest hit"},
        "e2e": {"value": mrays, "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


METRIC = "Mrays/s closest-hit, culled vs plain, 1 GB300, identical hits; node+tri tests/ray"


# ------------------------------------------------------------------ gb300 --

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
    t0 = time.perf_counter()
    bvh = sc.sc_bvh_build(tris, R, comp)
    build_s = time.perf_counter() - t0
    info = bvh.info()
    d_masked = sc.DeviceBVH(bvh, args.layout)
    d_plain = sc.DeviceBVH(bvh, sc.SC_LAYOUT_PLAIN)
    n = rays_np.shape[0]
    rays = torch.from_numpy(rays_np).to(dev)
    hits = torch.empty((n, 4), dtype=torch.float32, device=dev)
    hits_plain = torch.empty((n, 4), dtype=torch.float32, device=dev)
    counts = torch.empty((n, 2), dtype=torch.int32, device=dev)
    counts_plain = torch.empty((n, 2), dtype=torch.int32, device=dev)
    work = torch.empty(sc.sc_trace_workspace_bytes(), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()
    opts = sc._opts(lut_mode=args.lut, refill=args.refill)

    # reference pass with counts (untimed): identical hits and tests per ray
    sc.sc_trace(d_masked, rays, hits, counts, 0, 1, work, opts)
    sc.sc_trace(d_plain, rays, hits_plain, counts_plain, 0, 0, work, opts)
    sc.sc_status_poll(work)
    # compare the 16-byte records bitwise (a miss stores id -1, a NaN pattern as float)
    same = bool(torch.equal(hits.view(torch.int32), hits_plain.view(torch.int32)))
    cnt_c = counts.double().mean(0).tolist()
    cnt_p = counts_plain.double().mean(0).tolist()
    le = bool((counts <= counts_plain).all().item())

    def timed(dbvh, cull, out_hits):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for _ in range(args.warmup):
            flush.zero_()
            sc.sc_trace(dbvh, rays, out_hits, None, 0, cull, work, opts)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            sc.sc_trace(dbvh, rays, out_hits, None, 0, cull, work, opts)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms

    with ClockSampler(local) as clk:
        ms_cull = timed(d_masked, 1, hits)
        ms_plain = timed(d_plain, 0, hits_plain)
    sc.sc_status_poll(work)
    tot_cull = float(np.sum(ms_cull))
    if dist:
        t = torch.tensor([tot_cull], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_cull = float(t.item())
    rays_total = n * args.steps * world
    value = rays_total / (tot_cull * 1e-3) / 1e6
    plain_value = n * args.steps / (float(np.sum(ms_plain)) * 1e-3) / 1e6

    # end to end through the C-ABI with host buffers (H2D rays, D2H hits)
    h_rays = torch.from_numpy(rays_np).pin_memory()
    h_hits = torch.empty((n, 4), dtype=torch.float32).pin_memory()
    d_rays_buf = torch.empty((n, 8), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        sc.sc_trace_host(d_masked, h_rays, h_hits, None, 0, 1, d_rays_buf, hits, None, work, opts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sc.sc_trace_host(d_masked, h_rays, h_hits, None, 0, 1, d_rays_buf, hits, None, work, opts)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": n * args.steps / e2e_s / 1e6, "unit": "Mrays/s",
           "h2d_bytes_per_step": n * 32, "d2h_bytes_per_step": n * 16}

    # roofline of the traversal kernel: algorithmic bytes per ray
    node_bytes = ((96 if args.layout == 1 else 64) +
                  (0 if comp else 2 * {4: 8, 6: 32, 8: 64}[R]))
    b_ray = 32 + 16 + (cnt_c[0] / 2.0) * node_bytes + cnt_c[1] * 48
    per_launch_bytes = b_ray * n
    avg_ms = float(np.mean(ms_cull))
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
    peaks = load_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "measured" if peaks else "fallback",
                "bytes_per_ray": b_ray}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        ob = oracle.OracleBVH(tris).build_masks(R, 3)
        cull_mode = 1
        if comp:
            ob.compress(256, 8)
            cull_mode = 2
        thr = cpu_count()
        v, sample, dt, ref = oracle_rays_per_s(ob, tris, rays_np, cull_mode, thr, 15.0)
        cpu = {"value": v / 1e6, "unit": "Mrays/s", "cores": thr, "kind": "oracle",
               "sample": f"{sample} primary rays evenly spaced over the {n}, culled closest hit, "
                         f"{dt:.1f} s"}
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ms_cull)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "rays_per_step": n,
                   "grid_res": R, "compressed": bool(comp), "L": 3, "lut_mode": args.lut,
                   "layout": args.layout, "refill": args.refill,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "plain_mrays_s": plain_value, "speedup_vs_plain": value / world / plain_value,
        "identical_hits": same, "culled_counts_le_plain": le,
        "tests_per_ray": {"culled": {"node": cnt_c[0], "tri": cnt_c[1],
                                     "node_plus_tri": cnt_c[0] + cnt_c[1]},
                          "plain": {"node": cnt_p[0], "tri": cnt_p[1],
                                    "node_plus_tri": cnt_p[0] + cnt_p[1]}},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": 2 * args.steps,
        "build_s": build_s, "bvh": {"nodes": info.num_nodes, "max_depth": info.max_depth,
                                    "ms_bvh": info.ms_bvh, "ms_masks": info.ms_masks,
                                    "ms_compress": info.ms_compress},
    }
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
    ap.add_argument("--workload", default="hair1m", choices=sorted(WORKLOADS))
    ap.add_argument("--lut", type=int, default=0, help="0 auto, 1 global table, 2 shared")
    ap.add_argument("--layout", type=int, default=1, help="1 masked (scales stored), 2 compact")
    ap.add_argument("--refill", type=int, default=0, help="idle lanes before a warp refills")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
