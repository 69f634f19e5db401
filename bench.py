"""Benchmark: ODC Mcells/s at 256^3 on the envelope-MLP occupancy workload.

Workload (one step = one whole ODC extraction, every stage): 256^3 cells on
[-1, 1]^3, occ(x) = sigmoid(20 (0.5 - |x| + 0.15 f(x))) with f a random
Kaiming-initialised 64-frequency (sigma 4) Fourier-feature MLP, 4 x 256 ReLU,
iso 0.5, 15 bisection steps, 2D search (4 + 11, 0.8) and (3 + 12, sqrt(2)/2).
Synthetic seeded weights (the paper's trained networks are not available).

``value`` times the device work of each step with CUDA events on the stream
the library runs on, with the source already resident in HBM and L2 flushed
(a 512 MiB write) between steps, outside the timed events.  ``e2e`` times the
public C-ABI call with host source buffers (the weights prepared and uploaded
every step) and the mesh copied back to pinned host buffers.
Under torchrun every rank extracts its own shape (replicas; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

RES = 256
STEPS_1D = 15
FP32_FMA_PER_SM_CLK = 128          # FP32 lanes per SM on GB300
N_SM = 152


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = []
        mx = 0.0
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, n in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(value: float, dist=None, device="cpu") -> float:
    """Max of ``value`` over all ranks (identity without a process group)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(cells: float, world: int, steps: int, t_ms: float) -> float:
    """Whole-job Mcells/s: every rank processed ``steps`` grids of ``cells`` cells in ``t_ms``."""
    return cells * world * steps / (t_ms * 1e-3) / 1e6


def workload(seed: int = 0):
    from paper_2409_13418_gb300 import inputs as I
    return I.envelope_mlp(seed), I.cube_grid(RES)


def cpu_model() -> str:
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def _shell_directions(k: int):
    """k unit directions spread over the sphere (a Fibonacci lattice)."""
    import math
    out = []
    for i in range(k):
        zc = 1.0 - 2.0 * (i + 0.5) / k
        r = math.sqrt(max(0.0, 1.0 - zc * zc))
        phi = i * math.pi * (3.0 - math.sqrt(5.0))
        out.append((r * math.cos(phi), r * math.sin(phi), zc))
    return out


def cpu_sample(mlp, n_cells: int = 40, where: int = -1, n_where: int = 16):
    """Oracle on an n^3-cell block of the same 256^3 grid crossing the surface
    shell: at x ~ 0.31..0.62 on the x axis (where < 0), else centred on the
    shell (radius 0.47) in direction ``where`` of ``n_where``."""
    from oracle import odc as oracle
    from paper_2409_13418_gb300 import inputs as I
    h = 2.0 / RES
    if where < 0:
        i0 = (RES // 2 + 40, RES // 2 - n_cells // 2, RES // 2 - n_cells // 2)   # x in [0.31, 0.31 + n h]
    else:
        d = _shell_directions(n_where)[where]
        i0 = tuple(int(round((0.47 * d[a] + 1.0) / h)) - n_cells // 2 for a in range(3))
    lo = tuple(-1.0 + i0[a] * h for a in range(3))
    hi = tuple(lo[a] + n_cells * h for a in range(3))
    g = I.Grid(lo, hi, (n_cells, n_cells, n_cells))
    t = time.perf_counter()
    r = oracle.extract(mlp, g, steps_1d=STEPS_1D)
    dt = time.perf_counter() - t
    return n_cells ** 3, dt, r.stats


def _oracle_block(job):
    """Process-pool worker: one oracle block (single-threaded numpy)."""
    n_cells, where, n_where = job
    mlp, _ = workload(0)
    return cpu_sample(mlp, n_cells, where, n_where)[:2]


def oracle_all_cores(n_cells: int, n_blocks: int, workers: int):
    """The oracle as it stands on every host core: n_blocks blocks of n_cells^3
    on the surface shell, one per process of a spawned pool (numpy's BLAS
    single-threaded in each).  Returns (cells, wall seconds, processes)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    keep = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            list(ex.map(_oracle_block, [(8, i, workers) for i in range(workers)]))   # interpreters up, imports done
            t = time.perf_counter()
            res = list(ex.map(_oracle_block, [(n_cells, i % n_blocks, n_blocks) for i in range(n_blocks)]))
            wall = time.perf_counter() - t
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return sum(c for c, _ in res), wall, workers


def run_reference(args, rank, world):
    """The oracle as it stands on every host core, on a bounded sample per
    step: one n^3-cell block of the 256^3 grid on the surface shell per core."""
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_all_cores(args.cpu_cells, cores, cores)
    tot_cells, tot_t = 0, 0.0
    for _ in range(args.steps):
        c, dt, _ = oracle_all_cores(args.cpu_cells, cores, cores)
        tot_cells += c
        tot_t += dt
    v = tot_cells / tot_t / 1e6
    line = {"metric": "ODC Mcells/s at 256^3", "value": v, "unit": "Mcells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"envelope MLP 256^3 (k={STEPS_1D}), sampled as {cores} blocks of "
                                   f"{args.cpu_cells}^3 cells of the same grid on the surface shell per step"},
            "cpu_baseline": {"value": v, "unit": "Mcells/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                             "sample": f"{cores} blocks of {args.cpu_cells}^3 cells of the 256^3 grid on the surface "
                                       f"shell per step, one per process (numpy single-threaded in each)"},
            "e2e": {"value": v, "unit": "Mcells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def voxel_bench(odc, I, res: int = 512, vox: int = 513):
    """Dense voxel-grid source: a smooth blob volume of vox^3 float32 samples
    (larger than L2) meshed on a res^3 grid (k = 15).  Reports the extraction
    rate and the grid-label kernel's volume bytes per second (every sample is
    read at least once when the grid is as fine as the volume)."""
    src = I.voxel_blobs(7, dims=(vox, vox, vox))
    g = I.cube_grid(res)
    with odc.Context(0) as ctx:
        ctx.upload(src)
        ms, grid_ms = [], []
        for _ in range(4):
            m = ctx.extract(None, g, steps_1d=15)
            ms.append(m.stats["stage_ms"][7])
            grid_ms.append(m.stats["stage_ms"][0])
        st = m.stats
    t, tg = min(ms[1:]), min(grid_ms[1:])
    vbytes = 4.0 * vox ** 3
    return {"workload": f"smooth blob volume {vox}^3 float32 ({vbytes / 1e6:.0f} MB), {res}^3 cells, k=15",
            "mcells_per_s": res ** 3 / (t * 1e-3) / 1e6, "device_ms": round(t, 3),
            "grid_label_ms": round(tg, 3), "grid_label_volume_gbs": vbytes / (tg * 1e-3) / 1e9,
            "edges": st["n_edges"], "face_segs": st["n_face_segs"], "tris": m.n_tris}


def resolution_scaling(odc, I, resolutions=(128, 256, 512, 1024)):
    """Extraction rate of the envelope MLP (BF16 tiered, k = 15) against grid
    resolution, one GPU, whole grid in one piece (the shape of Tab. A3's
    128/256/512^3 rows; 1024^3 holds ~31 GB of device memory)."""
    mlp = I.envelope_mlp(0)
    rows = {}
    with odc.Context(0) as ctx:
        ctx.upload(mlp, precision=odc.PREC_BF16)
        for r in resolutions:
            g = I.cube_grid(r)
            ctx.extract(None, g, steps_1d=15)          # arenas sized for r
            m = ctx.extract(None, g, steps_1d=15)
            t = m.stats["stage_ms"][7]
            rows[f"{r}^3"] = {"device_ms": round(t, 1), "mcells_per_s": r ** 3 / (t * 1e-3) / 1e6,
                              "edges": m.stats["n_edges"], "tris": m.n_tris,
                              "device_gb_held": round(ctx.device_bytes() / 1e9, 2)}
    return rows


def slab_scaling(odc, I, r: int = 1024, n_slabs: int = 8):
    """The same 1024^3 envelope-MLP extraction in z-slabs, one after the
    other on one context (odc_extract_slabbed): the merged mesh equals the
    whole-grid one byte for byte, and the device memory held is one slab's
    arenas plus the merged mesh.  Wall time around the call (slab
    orchestration and placement included)."""
    import time
    import torch
    mlp = I.envelope_mlp(0)
    g = I.cube_grid(r)
    with odc.Context(0) as ctx:
        ctx.upload(mlp, precision=odc.PREC_BF16)
        ctx.extract_slabbed(None, g, n_slabs, halo=2, steps_1d=15)   # arenas sized for one slab
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = ctx.extract_slabbed(None, g, n_slabs, halo=2, steps_1d=15)
        wall = time.perf_counter() - t0
        held = ctx.device_bytes()
    return {f"{r}^3 in {n_slabs} slabs (halo 2)": {"wall_ms": round(wall * 1e3, 1),
                                                  "mcells_per_s": r ** 3 / wall / 1e6,
                                                  "device_ms_summed": round(m.stats["stage_ms"][7], 1),
                                                  "tris": m.n_tris, "device_gb_held": round(held / 1e9, 2)}}


def batch_bench(odc, I, n_shapes: int = 64, slots: int = 8, seed: int = 9):
    """The batched workload: n_shapes shapes with resolutions log-uniform in
    64^3..256^3, even ones seeded 64-primitive CSG trees (k = 12), odd ones
    latent-conditioned envelope MLPs of one network (128-d latent, BF16,
    k = 15).  Two ways, each after one warm-up pass over the same shapes:
    all shapes at once through odc_extract_many, one context per shape, the
    MLP shapes' search-stage network evaluations merged into shared launches
    (one batch group); and the request loop with ``slots`` slots, each shape
    on its own launches.  The rate is the total cells over the wall time."""
    import numpy as np
    rng = np.random.default_rng(seed)
    res = np.round(np.exp(rng.uniform(np.log(64), np.log(256), n_shapes))).astype(int)
    net = I.envelope_mlp(12, latent_dim=128)
    jobs = []
    for i, r in enumerate(res):
        if i % 2 == 0:
            jobs.append((I.random_csg(1000 + i, n_prims=64), I.cube_grid(int(r)), dict(steps_1d=12)))
        else:
            jobs.append((I.with_latent(net, 2000 + i), I.cube_grid(int(r)), dict(steps_1d=15, precision=odc.PREC_BF16)))
    cells = float(np.sum(res.astype(np.float64) ** 3))
    out = {"workload": f"{n_shapes} shapes, res log-uniform 64^3..256^3 (total {cells / 1e6:.0f} M cells), half "
                       "64-primitive CSG trees (k=12), half latent-conditioned envelope MLPs of one network "
                       "(BF16 tiers, k=15)"}
    ctxs = [odc.Context(0) for _ in jobs]
    try:
        with odc.Batch(0) as b:
            for _ in range(2):
                b0 = b.stats()
                t0 = time.perf_counter()
                odc.extract_many(b, ctxs, jobs)
                span = time.perf_counter() - t0
            st = b.stats()
            rounds, calls = st["rounds"] - b0["rounds"], st["calls"] - b0["calls"]
            for c in ctxs:
                c.join_batch(None)
    finally:
        for c in ctxs:
            c.close()
    out["shared_launches"] = {"contexts": n_shapes, "seconds": round(span, 3), "mcells_per_s": cells / span / 1e6,
                              "shapes_per_s": n_shapes / span, "merged_rounds": rounds,
                              "member_calls": calls, "mean_shapes_per_launch": calls / max(rounds, 1)}
    with odc.Server(0, slots=slots, host_copy=False) as srv:
        for _ in range(2):
            t0 = srv.clock()
            ids = [srv.submit(src, g, **kw) for src, g, kw in jobs]
            res_ = [srv.poll(i) for i in ids]
            for i in ids:
                srv.release(i)
            span = max(o["t_end"] for o in res_) - t0
    assert all(o["status"] == 0 for o in res_)
    out["request_loop"] = {"slots": slots, "seconds": round(span, 3), "mcells_per_s": cells / span / 1e6,
                           "shapes_per_s": n_shapes / span}
    return out


def ablation_table(odc, I, res: int = 128, seed: int = 1):
    """The shape of the paper's ablations (Sec. 6.3, Tab. 3; Tab. A8) on a
    seeded 64-primitive CSG tree at res^3 (k = 12): marching cubes through
    linearly placed and through bisected 1D points, Manifold Dual Contouring,
    + 1D search, + 2D search, + IC split (= ODC).  Per variant: device ms of the
    extraction (CUDA events inside the library), #V, #T, the mean first-order
    surface distance at 2M area-uniform samples (in cells), self-intersecting
    triangle pairs and manifoldness."""
    src = I.random_csg(seed, n_prims=64)
    g = I.cube_grid(res)
    h = 2.0 / res
    rows = {}
    variants = (("MC", dict(linear_1d=True, mc=True)),
                ("MC + 1D search", dict(mc=True)),
                ("MDC", dict(linear_1d=True, gradient_normals=True, ic_split=False)),
                ("+1D search", dict(gradient_normals=True, ic_split=False)),
                ("+2D search", dict(ic_split=False)),
                ("+IC (ODC)", dict()))
    with odc.Context(0) as ctx:
        for name, kw in variants:
            ms = []
            for _ in range(4):
                m = ctx.extract(src, g, steps_1d=12, **kw)
                ms.append(m.stats["stage_ms"][7])
            q = m.quality(n_samples=2_000_000, seed=1)
            rows[name] = {"ms": round(min(ms[1:]), 3), "verts": m.n_verts, "tris": m.n_tris,
                          "dist_mean_cells": q["dist_mean"] / h, "si_pairs": q["n_si_pairs"],
                          "manifold": bool(q["manifold"])}
    return {"workload": f"seeded 64-primitive CSG tree (seed {seed}), {res}^3 cells, k=12", "rows": rows}


def serve_arm(odc, I, net, trace, slots, precision, budget, share=False):
    """Replays an arrival trace through the request loop: a submitter thread
    submits each request at its arrival time, the caller collects them.
    Returns latencies (s), per-request cells and the makespan."""
    srv = odc.Server(0, slots=slots, mem_budget=budget, host_copy=False, share_network=share)
    try:
        # warm-up: every slot grows its arenas for the largest resolution once
        top = max(r for _, r, _ in trace)
        ids = [srv.submit(I.with_latent(net, 10 ** 6 + k), I.cube_grid(top), steps_1d=STEPS_1D,
                          precision=precision) for k in range(slots)]
        for i in ids:
            assert srv.poll(i)["status"] == 0
            srv.release(i)
        ids = [None] * len(trace)
        t0 = time.perf_counter()

        def submitter():
            for k, (t, res, seed) in enumerate(trace):
                d = t0 + t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                ids[k] = srv.submit(I.with_latent(net, seed), I.cube_grid(res), steps_1d=STEPS_1D,
                                    precision=precision)

        th = threading.Thread(target=submitter)
        th.start()
        lat, cells, t_first, t_last, bad = [], [], None, None, 0
        for k in range(len(trace)):
            while ids[k] is None:
                time.sleep(0.0005)
            r = srv.poll(ids[k])
            bad += r["status"] != 0
            lat.append(r["t_end"] - r["t_submit"])
            cells.append(trace[k][1] ** 3)
            t_first = r["t_submit"] if t_first is None else min(t_first, r["t_submit"])
            t_last = r["t_end"] if t_last is None else max(t_last, r["t_end"])
            srv.release(ids[k])
        th.join()
    finally:
        srv.close()
    return lat, cells, t_last - t_first, bad


def serve_bench(odc, I, seconds: float, slots: int, low_rate: float = 2.0, low_seconds: float = 20.0):
    """Serving workload: Poisson arrivals at 40 req/s for ``seconds`` (the
    configured rate, far above any arm's capacity, so its latencies measure
    queue growth) and at a sub-capacity ``low_rate`` for ``low_seconds``;
    cube resolutions {64, 128, 256, 512} with weights 0.4/0.3/0.2/0.1, each
    request a latent-conditioned envelope MLP (one network, a 128-d latent
    per shape), 150 GB admission budget.  Four arms on the same traces: our
    loop (``slots`` slots, FP8 pass + tiers, the slots' search-stage network
    evaluations merged into shared launches), the same without the sharing,
    the same precision one request at a time (1 slot: what the slots and
    overlap add), and plain one-request-at-a-time GPU ODC (1 slot, FP32 plain
    network)."""
    import numpy as np
    net = I.envelope_mlp(11, latent_dim=128)
    budget = 150 * 10 ** 9
    traces = {"rate_40": I.serving_trace(5, 40.0, seconds), f"rate_{low_rate:g}": I.serving_trace(6, low_rate, low_seconds)}
    out = {"workload": f"Poisson 40 req/s for {seconds:g} s ({len(traces['rate_40'])} requests) and {low_rate:g} req/s "
                       f"for {low_seconds:g} s ({len(traces[f'rate_{low_rate:g}'])} requests), cube res "
                       "{64,128,256,512} w 0.4/0.3/0.2/0.1, latent-conditioned envelope MLP (128-d latent), "
                       f"k={STEPS_1D}, 150 GB budget; latency = completion - submission (server clock)"}
    arms = (("ours", slots, odc.PREC_FP8, "fp8 pass + bf16/fp16/split/fp32 tiers", True),
            ("ours_unshared", slots, odc.PREC_FP8, "fp8 pass + bf16/fp16/split/fp32 tiers", False),
            ("fifo_same_precision", 1, odc.PREC_FP8, "fp8 pass + bf16/fp16/split/fp32 tiers", False),
            ("plain_fifo_fp32", 1, odc.PREC_FP32, "fp32 plain", False))
    for tname, trace in traces.items():
        out[tname] = {}
        for name, sl, prec, pname, share in arms:
            lat, cells, span, bad = serve_arm(odc, I, net, trace, sl, prec, budget, share)
            lat = np.asarray(lat)
            out[tname][name] = {"slots": sl, "precision": pname, "shared_network_launches": share,
                                "requests": len(lat), "failed": int(bad),
                                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                                "mean_s": float(lat.mean()), "makespan_s": span,
                                "throughput_req_s": len(lat) / span,
                                "throughput_mcells_s": float(np.sum(cells)) / span / 1e6}
    return out


def csg_run(args):
    """The CSG pipeline alone (a seeded 64-primitive tree, k = 12) at
    --csg-res^3: warm-up and timed extractions with the stage times, for
    profiling the non-network kernels (every stage but the MLP network)."""
    import torch
    from paper_2409_13418_gb300 import build, inputs as I, odc
    build.build()
    src, g = I.random_csg(1, n_prims=64), I.cube_grid(args.csg_res)
    with odc.Context(0) as ctx:
        ctx.upload(src)
        for _ in range(args.warmup):
            ctx.extract(None, g, steps_1d=12)
        ms, stages = [], None
        for _ in range(args.steps):
            m = ctx.extract(None, g, steps_1d=12)
            ms.append(m.stats["stage_ms"][7])
            stages = m.stats["stage_ms"]
        torch.cuda.synchronize()
    t = min(ms)
    print(json.dumps({"workload": f"seeded 64-primitive CSG tree, {args.csg_res}^3 cells, k=12",
                      "device_ms": t, "mcells_per_s": args.csg_res ** 3 / (t * 1e-3) / 1e6,
                      "stage_ms": [round(x, 4) for x in stages], "edges": m.stats["n_edges"],
                      "face_segs": m.stats["n_face_segs"], "cells": m.stats["n_cells"], "tris": m.n_tris}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="bf16")
    ap.add_argument("--band", type=float, default=0.03,
                    help="|occ - 0.5| band re-evaluated in FP32 (covers the measured BF16 logit error)")
    ap.add_argument("--cpu-cells", type=int, default=None,
                    help="oracle sample block edge (default 40 for cpu_baseline, 32 per reference step)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=1.0,
                    help="length of the serving arrival trace (0: skip the serving comparison)")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--no-ablation", action="store_true", help="skip the ablation table (Sec. 6.3 variants)")
    ap.add_argument("--csg-res", type=int, default=0,
                    help="profile run: only the CSG pipeline at this resolution (prints its own JSON line)")
    ap.add_argument("--fp32-points", type=int, default=0,
                    help="profile run: only the FP32 network over this many seeded points (list mode, 3 launches)")
    ap.add_argument("--net-points", type=int, default=0,
                    help="profile run: only one network tier (--net-tier) over this many seeded points, 3 launches")
    ap.add_argument("--net-tier", choices=["fp32", "bf16", "f16", "split", "fp8"], default="fp8")
    ap.add_argument("--slab-res", type=int, default=0,
                    help="only the envelope MLP at this resolution in --slab-count z-slabs (prints its own JSON line)")
    ap.add_argument("--slab-count", type=int, default=8)
    ap.add_argument("--mlp-res", type=int, default=0,
                    help="profile run: only whole envelope-MLP extractions at this resolution (resident BF16 "
                         "source, --warmup untimed, --steps timed; prints its own JSON line)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        args.cpu_cells = args.cpu_cells or 32
        run_reference(args, rank, world)
        return
    args.cpu_cells = args.cpu_cells or 40
    if args.csg_res:
        csg_run(args)
        return
    if args.fp32_points:
        import numpy as np
        from paper_2409_13418_gb300 import build, inputs as I, odc
        build.build()
        odc.load()
        pts = np.random.default_rng(1).uniform(-1, 1, (args.fp32_points, 3)).astype(np.float32)
        with odc.Context(0) as ctx:
            mlp = I.envelope_mlp(0)
            for _ in range(3):
                ctx.eval_points(mlp, pts, precision=odc.PREC_FP32)
        print(json.dumps({"workload": f"FP32 network over {args.fp32_points} seeded points (list mode)",
                          "launches": 3}), flush=True)
        return
    if args.net_points:
        import numpy as np
        from paper_2409_13418_gb300 import build, inputs as I, odc
        build.build()
        odc.load()
        prec = {"fp32": odc.PREC_FP32, "bf16": odc.PREC_BF16, "f16": odc.PREC_F16, "split": odc.PREC_SPLIT,
                "fp8": odc.PREC_FP8_RAW}[args.net_tier]
        pts = np.random.default_rng(1).uniform(-1, 1, (args.net_points, 3)).astype(np.float32)
        with odc.Context(0) as ctx:
            mlp = I.envelope_mlp(0)
            for _ in range(3):   # bf16 without a band: the raw BF16 pass alone
                ctx.eval_points(mlp, pts, precision=prec, band=0.0)
        print(json.dumps({"workload": f"{args.net_tier} network tier over {args.net_points} seeded points "
                                      f"(list mode)", "launches": 3}), flush=True)
        return
    if args.mlp_res:
        import torch
        from paper_2409_13418_gb300 import build, inputs as I, odc
        build.build()
        odc.load()
        g = I.cube_grid(args.mlp_res)
        with odc.Context(0) as ctx:
            ctx.upload(I.envelope_mlp(0), precision=odc.PREC_BF16)
            for _ in range(args.warmup):
                ctx.extract(None, g, steps_1d=15)
            torch.cuda.synchronize()
            l0, t0 = odc.launch_total(), time.perf_counter()
            for _ in range(args.steps):
                ctx.extract(None, g, steps_1d=15)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / max(args.steps, 1)
            launches = (odc.launch_total() - l0) / max(args.steps, 1)
        print(json.dumps({"workload": f"envelope MLP occupancy, {args.mlp_res}^3 cells, k=15, bf16 band 0.03, "
                                      f"resident source", "ms_per_extraction": dt * 1e3,
                          "launches_per_extraction": launches, "steps": args.steps, "warmup": args.warmup}),
              flush=True)
        return
    if args.slab_res:
        from paper_2409_13418_gb300 import build, inputs as I, odc
        build.build()
        odc.load()
        print(json.dumps({"workload": f"envelope MLP occupancy, {args.slab_res}^3 cells, k=15, bf16 band 0.03, "
                                      f"z-slabs on one GPU",
                          "rows": slab_scaling(odc, I, args.slab_res, args.slab_count)}), flush=True)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2409_13418_gb300 import build, odc
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    assert args.warmup >= 3 or os.environ.get("ODC_BENCH_ALLOW_SHORT"), "at least 3 warm-up steps"

    prec = odc.PREC_BF16 if args.precision == "bf16" else odc.PREC_FP32
    mlp, grid = workload(rank)
    ctx = odc.Context(local)
    ctx.upload(mlp, precision=prec, band=args.band)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def step():
        return ctx.extract(None, grid, steps_1d=STEPS_1D, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = odc.launch_total()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    mlp_ms, mlp_flops, mlp_launches, stats = 0.0, 0.0, 0, None
    tc_ms, tc_flops, tc_launches = 0.0, 0.0, 0
    sp_ms, sp_flops, sp_launches, n_split = 0.0, 0.0, 0, 0
    h16_ms, h16_flops, h16_launches = 0.0, 0.0, 0
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        m = step()
        ev[i][1].record(stream)
        stats = m.stats
        mlp_ms += stats["mlp_ms"]
        mlp_flops += stats["mlp_flops"]
        mlp_launches += stats["mlp_launches"]
        tc_ms += stats["tc_ms"]
        tc_flops += stats["tc_flops"]
        tc_launches += stats["tc_launches"]
        sp_ms += stats["split_ms"]
        sp_flops += stats["split_flops"]
        sp_launches += stats["split_launches"]
        h16_ms += stats["h16_ms"]
        h16_flops += stats["h16_flops"]
        h16_launches += stats["h16_launches"]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = odc.launch_total() - l0
    clocks = sampler.stop()
    t_steps = sum(a.elapsed_time(b) for a, b in ev)          # ms, device time of K steps
    t_max = reduce_max(t_steps, dist, "cuda")
    cells = float(RES ** 3)
    value = throughput(cells, world, args.steps, t_max)

    # e2e: host source buffers in, mesh copied back to pinned host buffers
    # (sized from the timed steps' mesh, allocated before the clock starts)
    vbytes = tbytes = 0
    h2d = sum(a.nbytes for a in [mlp.B] + mlp.weights + mlp.biases)
    last = m
    pin_v = torch.empty(max(1, last.n_verts * 3 + 3 * 1024), dtype=torch.float32, pin_memory=True)
    pin_t = torch.empty(max(1, last.n_tris * 3 + 3 * 1024), dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        m = ctx.extract(mlp, grid, steps_1d=STEPS_1D, stream=stream.cuda_stream, precision=prec, band=args.band,
                        reupload=True)
        if m.n_verts * 3 > pin_v.numel() or m.n_tris * 3 > pin_t.numel():   # never for a fixed workload
            pin_v = torch.empty(m.n_verts * 3, dtype=torch.float32, pin_memory=True)
            pin_t = torch.empty(m.n_tris * 3, dtype=torch.int32, pin_memory=True)
        m.copy_to(pin_v.data_ptr(), pin_t.data_ptr(), on_device=False)
        vbytes, tbytes = m.n_verts * 12, m.n_tris * 12
    torch.cuda.synchronize()
    t_e2e = reduce_max((time.perf_counter() - t0) * 1e3, dist, "cuda")
    e2e = throughput(cells, world, args.steps, t_e2e)
    # The FP8 first pass on the same workload (outside the headline's timed
    # region): device time per step, the queries it evaluated and those it
    # decided (outside its band), against the BF16-first tiers above.
    fp8 = None
    if prec == odc.PREC_BF16 and rank == 0:
        vb, tb = m.to_host()
        ctx.upload(mlp, precision=odc.PREC_FP8, band=args.band)
        for _ in range(2):
            ctx.extract(None, grid, steps_1d=STEPS_1D, stream=stream.cuda_stream)
        f_ms, f_stats = [], None
        for _ in range(max(3, min(args.steps, 5))):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mf = ctx.extract(None, grid, steps_1d=STEPS_1D, stream=stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            f_ms.append(e0.elapsed_time(e1))
            f_stats = mf.stats
        fq = f_stats["fp8_flops"] / 459264.0
        bq = f_stats["tc_flops"] / 459264.0
        fp8 = {"ms_per_step": statistics.median(f_ms), "bf16_first_ms_per_step": t_max / args.steps,
               "gain": 1.0 - statistics.median(f_ms) / (t_max / args.steps),
               "fp8_queries": int(round(fq)), "bf16_pass_queries": int(round(bq)),
               "fp8_ms": f_stats["fp8_ms"], "fp8_tflops": f_stats["fp8_flops"] / max(f_stats["fp8_ms"], 1e-9) / 1e9,
               "mesh_equals_bf16_first": None}
        vf, tf = mf.to_host()
        fp8["mesh_equals_bf16_first"] = bool(vf.tobytes() == vb.tobytes() and np.array_equal(tf, tb))
        ctx.upload(mlp, precision=prec, band=args.band)
    # Sec. 6.1 quality measures of the last mesh (outside every timed region)
    tq = time.perf_counter()
    quality = m.quality(n_samples=2_000_000, seed=1)
    mc = ctx.extract(mlp, grid, steps_1d=STEPS_1D, stream=stream.cuda_stream, precision=prec, band=args.band,
                     mc=True)
    qmc = mc.quality(n_samples=2_000_000, seed=1)
    mc_quality = {"occ_dev_mean": qmc["occ_dev_mean"], "manifold": bool(qmc["manifold"]), "si_pairs": qmc["n_si_pairs"],
                  "verts": mc.n_verts, "tris": mc.n_tris, "device_ms": round(mc.stats["stage_ms"][7], 3)}
    quality = {"occ_dev_mean": quality["occ_dev_mean"], "occ_dev_max": quality["occ_dev_max"],
               "samples": quality["n_samples"], "manifold": bool(quality["manifold"]), "euler": quality["euler"],
               "si_pairs": quality["n_si_pairs"], "si_tris": quality["n_si_tris"], "tris": quality["n_tris"],
               "seconds": round(time.perf_counter() - tq, 3),
               "mc_1d_same_grid": mc_quality}

    if rank == 0:
        peaks, peak_src = _peaks()
        fp32_peak = N_SM * FP32_FMA_PER_SM_CLK * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        tc_peak = float(peaks["bf16_tflops_sustained"])
        rows = []
        if mlp_launches:
            a = mlp_flops / (mlp_ms * 1e-3) / 1e12
            # DRAM bytes of one launch: ncu on launches of 256 K and 1 M points
            # (dram__bytes_read + write): 1.01 MB (the weights) + 12.1 B per query
            q_per_launch = mlp_flops / mlp_launches / 459264.0
            rows.append({"bound": "alu", "kernel": "k_mlp_fp32 (FP32 SIMT network; the plain path and the band "
                                                   "re-evaluation)", "achieved": a, "peak": fp32_peak,
                         "unit": "TFLOP/s", "frac": a / fp32_peak,
                         "traffic": 1.01e6 + 12.1 * q_per_launch,
                         "traffic_source": "bytes per launch at this run's mean queries per launch, from ncu "
                                           "dram__bytes_read.sum + dram__bytes_write.sum of launches of 256K and "
                                           "1M points: 1.01 MB + 12.1 B per query",
                         "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock (unit counts)",
                         "ms_per_step": mlp_ms / args.steps, "flops_per_launch": mlp_flops / mlp_launches})
        if tc_launches:
            a = tc_flops / (tc_ms * 1e-3) / 1e12
            rows.append({"bound": "tensor", "kernel": "k_mlp_tc (tcgen05 BF16 network)", "achieved": a,
                         "peak": tc_peak, "unit": "TFLOP/s", "frac": a / tc_peak, "traffic": None,
                         "peak_source": f"bf16_tflops_sustained, {peak_src}",
                         "ms_per_step": tc_ms / args.steps, "flops_per_launch": tc_flops / tc_launches})
        if sp_launches:
            a = sp_flops / (sp_ms * 1e-3) / 1e12
            rows.append({"bound": "tensor", "kernel": "k_mlp_tc3 (split-FP16 band re-evaluation, 3 FP16 products "
                                                      "per layer; tensor-pipe FLOPs)", "achieved": a,
                         "peak": tc_peak, "unit": "TFLOP/s", "frac": a / tc_peak, "traffic": None,
                         "peak_source": f"bf16_tflops_sustained, {peak_src}",
                         "ms_per_step": sp_ms / args.steps, "flops_per_launch": sp_flops / sp_launches})
        if h16_launches:
            a = h16_flops / (h16_ms * 1e-3) / 1e12
            rows.append({"bound": "tensor", "kernel": "k_mlp_tc<FP16> (single-product FP16 band tier)", "achieved": a,
                         "peak": tc_peak, "unit": "TFLOP/s", "frac": a / tc_peak, "traffic": None,
                         "peak_source": f"bf16_tflops_sustained (FP16 has the same dense rate), {peak_src}",
                         "ms_per_step": h16_ms / args.steps, "flops_per_launch": h16_flops / h16_launches})
        rows.sort(key=lambda r: -r["ms_per_step"])
        roof = dict(rows[0])
        if len(rows) > 1:
            roof["other_kernels"] = rows[1:]
        # The MLP occupancy stage as a whole, on the tensor pipe: every query
        # the method makes counted once (459,264 FLOP each), over the summed
        # event time of all network launches of a step (every tier), and over
        # the whole step.  A query re-evaluated by a later tier adds time but
        # no algorithmic FLOPs.
        net_ms = (mlp_ms + tc_ms + sp_ms + h16_ms) / args.steps
        alg = float(stats["n_queries"]) * 459264.0
        a_net = alg / (net_ms * 1e-3) / 1e12 if net_ms > 0 else 0.0
        a_step = alg / (t_max / args.steps * 1e-3) / 1e12
        roof["stage"] = {"bound": "tensor", "what": "MLP occupancy stage: queries x 459,264 FLOP per step over "
                                                    "the summed event time of every network launch (all tiers)",
                         "queries_per_step": int(stats["n_queries"]), "network_ms_per_step": net_ms,
                         "achieved": a_net, "peak": tc_peak, "unit": "TFLOP/s", "frac": a_net / tc_peak,
                         "achieved_over_whole_step": a_step, "frac_over_whole_step": a_step / tc_peak,
                         "peak_source": f"bf16_tflops_sustained, {peak_src}"}
        line = {"metric": "ODC Mcells/s at 256^3", "value": value, "unit": "Mcells/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if prec == odc.PREC_FP32 else "bf16+f16+f32",
                "data": "synthetic (seeded random-init MLP weights)",
                "config": {"workload": f"envelope MLP occupancy, {RES}^3 cells, k={STEPS_1D}, "
                                       f"{args.precision}" + (f" band {args.band}" if prec == odc.PREC_BF16 else ""),
                           "parallelism": f"replicas x{world}", "l2": "flushed (512 MiB write) between steps",
                           "edges": stats["n_edges"], "face_segs": stats["n_face_segs"],
                           "queries": stats["n_queries"],
                           "bf16_pass_queries": int(round(stats["tc_flops"] / 459264.0)),
                           "requeries_fp16": stats["n_h16"],
                           "requeries_split_fp16": stats["n_split"],
                           "requeries_fp32": stats["n_requeries"],
                           "fp32_tile_autotuned": stats["fp32_tile"],
                           "split_margin": stats.get("split_zmargin"),
                           "split_acc_comp": stats.get("split_acc_comp"),
                           "stage_ms": [round(x, 3) for x in stats["stage_ms"]]},
                "e2e": {"value": e2e, "unit": "Mcells/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(vbytes + tbytes)},
                "quality": quality,
                "gpu_launches": int(launches),
                "roofline": roof,
                "clocks": clocks}
        if fp8 is not None:
            line["fp8_first_pass"] = fp8
        if world == 1 and not args.no_ablation:
            from paper_2409_13418_gb300 import inputs as I
            line["ablation"] = ablation_table(odc, I)
            line["voxel"] = voxel_bench(odc, I)
            line["batched"] = batch_bench(odc, I)
            line["resolution_scaling"] = resolution_scaling(odc, I)
            line["resolution_scaling"].update(slab_scaling(odc, I))
        if world == 1 and args.serve_seconds > 0:
            ctx.close()
            from paper_2409_13418_gb300 import inputs as I
            line["serving"] = serve_bench(odc, I, args.serve_seconds, args.serve_slots)
        if world == 1 and not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            ca, dta, _ = oracle_all_cores(args.cpu_cells, cores, cores)
            c1, dt1, _ = cpu_sample(mlp, args.cpu_cells)
            line["cpu_baseline"] = {"value": ca / dta / 1e6, "unit": "Mcells/s", "cores": cores,
                                    "cpu": cpu_model(), "kind": "oracle",
                                    "sample": f"{cores} blocks of {args.cpu_cells}^3 cells of the same 256^3 grid on "
                                              f"the surface shell, one per process (FP64 numpy oracle, BLAS "
                                              f"single-threaded in each), {dta:.1f} s wall",
                                    "single_process": {"value": c1 / dt1 / 1e6, "cores": cores,
                                                       "sample": f"one {args.cpu_cells}^3 block, one Python "
                                                                 f"process (numpy's threaded BLAS for the network "
                                                                 f"products), {dt1:.1f} s"}}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
