#!/usr/bin/env python3
"""Benchmark: BFAST Monitor pixels/s on the full synthetic scene.

Workload (the default): 8,388,608 pixels (4096 x 2048) x 414 irregular dates,
history = first 228 dates, 3 harmonics + intercept + trend (K = 8), f = 23,
h = 0.25 n, lambda for alpha = 0.05; float32 storage with NaN for ~60 %
Markov cloud gaps; 10 % of pixels with a level shift.  One step = one
bfm_monitor call over the whole scene (every step of the per-pixel path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--forms f32hybrid,f32stream,...] [--pixels M] [--no-e2e]
                  [--no-cpu-baseline] [--no-c4c5]

The first of --forms (default: the hybrid form on float32) is the headline
line; the others are timed beside it under "forms".

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank processes
its own full scene (weak scaling, no collective on the data path); value is
all ranks' pixels / the slowest rank's time.

``--impl reference``: the FP64 oracle (plain C, all host cores) on a bounded
sample of the same scene per step -- a deliberately slow baseline, not the
target.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BFAST-monitor pixels/s at 8.4M px x 414 dates; p50/p99 tile latency"
# DRAM bytes per pixel per launch from the ncu captures summarised in
# profiles/ (None once the kernel changes after the capture).
TRAFFIC_PER_PX = {"f32": (1.7866e9 / 1048576,), "f32simt": (1.784346e9 / 1048576,), "f32stream": (None,),
                  "i16": (None,), "f32hybrid": (1.836045e9 / 1048576,), "i16hybrid": (None,),
                  "i16stream": (None,), "f32complete": (None,)}
SAMPLE_PX = 4096  # pixels of each timed form checked against the oracle (outside the timed region)

WORKLOAD = "c2: full scene 8,388,608 px x 414 dates, n_hist=228, K=8, f=23, h=0.25, plain float32"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest_rank(x: float, device) -> float:
    """The largest value of x over the ranks (a job's time is its slowest
    rank's); x itself when there is one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, steps: int, world_size: int, total_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world_size * units_per_rank * steps / (total_ms / 1e3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(Y_host, dates, k, f, n_hist, h_frac, lam, budget_s: float):
    """Time the oracle on a bounded sample: successive blocks of pixel
    columns of the same scene until about budget_s seconds of work."""
    import oracle
    m_all = Y_host.shape[1]
    blk = min(1 << 16, m_all)
    n, dt, c0 = 0, 0.0, 0
    while dt < budget_s and n < m_all:
        cols = np.ascontiguousarray(Y_host[:, c0:c0 + blk].numpy())
        t0 = time.perf_counter()
        oracle.monitor(dates, cols, k=k, f=f, n_hist=n_hist, h_frac=h_frac, lam=lam)
        dt += time.perf_counter() - t0
        n += cols.shape[1]
        c0 += blk
    return n / dt, n, dt


def cpu_oracle_one_core(Y_host, dates, n_hist, h_frac, lam):
    """The oracle on one host core (OMP_NUM_THREADS=1 in a child process) on
    the first 16,384 pixels of the scene."""
    cols = np.ascontiguousarray(Y_host[:, :16384].numpy())
    with tempfile.TemporaryDirectory() as td:
        np.save(os.path.join(td, "y.npy"), cols)
        np.save(os.path.join(td, "d.npy"), np.asarray(dates))
        code = ("import sys, time, numpy as np; sys.path.insert(0, %r); import oracle; "
                "y = np.load(%r); d = np.load(%r); t0 = time.perf_counter(); "
                "oracle.monitor(d, y, k=3, f=23.0, n_hist=%d, h_frac=%r, lam=%r); "
                "print(y.shape[1] / (time.perf_counter() - t0))"
                % (ROOT, os.path.join(td, "y.npy"), os.path.join(td, "d.npy"), n_hist, h_frac, lam))
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    try:
        v = float(r.stdout.strip().splitlines()[-1])
    except (ValueError, IndexError):
        return {"value": None, "error": r.stderr[-300:]}
    return {"value": v, "unit": "pixels/s", "cores": 1, "sample": "first 16384 pixels of the same scene"}


def cpu_oracle_c1():
    """The oracle on the c1 scene (4096 pixels x 228 dates): on all host cores,
    and on one core (OMP_NUM_THREADS=1 in a child process)."""
    import oracle
    import synth
    w1 = synth.workload("c1")
    t0 = time.perf_counter()
    oracle.monitor(w1["dates"], w1["Y"], k=3, f=23.0, n_hist=w1["n_hist"], h_frac=w1["h_frac"], lam=w1["lam"])
    dt = time.perf_counter() - t0
    code = ("import sys, time; sys.path.insert(0, %r); import oracle, synth; w = synth.workload('c1'); "
            "t0 = time.perf_counter(); oracle.monitor(w['dates'], w['Y'], k=3, f=23.0, n_hist=w['n_hist'], "
            "h_frac=w['h_frac'], lam=w['lam']); print(w['m'] / (time.perf_counter() - t0))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       env=dict(os.environ, OMP_NUM_THREADS="1"), timeout=600)
    try:
        one = float(r.stdout.strip().splitlines()[-1])
    except (ValueError, IndexError):
        one = None
    return {"value": w1["m"] / dt, "unit": "pixels/s", "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
            "one_core": one, "workload": "c1: 4096 pixels x 228 dates, n_hist 100, K 8, 30 % i.i.d. missing"}


def oracle_on(Y, dates, n_hist, h_frac, lam):
    import oracle
    return oracle.monitor(dates, np.ascontiguousarray(Y), k=3, f=23.0, n_hist=n_hist, h_frac=h_frac, lam=lam)


def form_errors(gpu: dict, ref: dict, dates) -> dict:
    """Each output's error against the FP64 oracle on the sample: beta in the
    column-scaled norm (max_i |dbeta_i| ||X_i||inf / max_i |beta_i| ||X_i||inf),
    sigma-hat relative, mean MOSUM |d| / max(1, |ref|), status mismatches, and
    break mismatches on pixels whose boundary margin is >= 1e-5 (untied) and
    below it (margin-tied, counted)."""
    import oracle
    st_g, st_r = gpu["status"], ref["status"]
    same = st_g == st_r
    tie = ref["margin"] < 1e-5
    bmis = (gpu["break_idx"] != ref["break_idx"]) & same
    X = oracle.design(dates, 3, 23.0)
    colmax = np.abs(X).max(axis=0)[:, None]
    fitted = same & np.isin(st_r, [0, 3, 4])
    be = 0.0
    if fitted.any():
        num = np.max(np.abs(gpu["beta"].astype(np.float64)[:, fitted] - ref["beta"][:, fitted]) * colmax, axis=0)
        den = np.max(np.abs(ref["beta"][:, fitted]) * colmax, axis=0)
        be = float((num / np.maximum(den, 1e-300)).max())
    so = same & np.isin(st_r, [0, 4])
    se = float((np.abs(gpu["sigma"].astype(np.float64)[so] - ref["sigma"][so]) / ref["sigma"][so]).max()) if so.any() else 0.0
    mo = same & (st_r == 0)
    me = float((np.abs(gpu["mean_mosum"].astype(np.float64)[mo] - ref["mean_mosum"][mo])
                / np.maximum(1.0, np.abs(ref["mean_mosum"][mo]))).max()) if mo.any() else 0.0
    return {"pixels": int(st_r.size), "beta_col_scaled_max": be, "sigma_rel_max": se, "mean_mosum_max": me,
            "status_mismatch": int((~same).sum()), "break_mismatch_untied": int((bmis & ~tie).sum()),
            "break_mismatch_tied": int((bmis & tie).sum()), "margin_tied": int(tie.sum()),
            "breaks": int((ref["break_idx"] >= 0).sum())}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import synth
    import torch
    w = synth.workload_torch("c2", device="cpu", m=1 << 18)
    Y = w["Y"].numpy()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    # size each step so the whole run takes about two minutes
    t0 = time.perf_counter()
    oracle.monitor(w["dates"], Y[:, :512], k=3, f=23.0, n_hist=228, h_frac=0.25, lam=w["lam"])
    rate = 512 / (time.perf_counter() - t0)
    per_step = int(max(256, min(Y.shape[1], rate * 100.0 / max(1, args.steps + args.warmup))))
    times = []
    for s in range(args.warmup + args.steps):
        c0 = (s * per_step) % (Y.shape[1] - per_step + 1)
        sub = Y[:, c0:c0 + per_step]
        t0 = time.perf_counter()
        oracle.monitor(w["dates"], sub, k=3, f=23.0, n_hist=228, h_frac=0.25, lam=w["lam"])
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = per_step * len(times) / tot
    sample = f"{per_step} pixel columns of the c2 scene per step (all 414 dates), oracle in FP64"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pixels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_px_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": "pixels/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "pixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_tiles_and_serving(bfm, synth, torch, dev, stream):
    """c4: 64 uneven int16 tiles (pixel counts rounded up to multiples of 8),
    each through bfm_monitor (the form AUTO picks) with its own CUDA-event
    latency, and all of them as one batched persistent launch (CUDA graph,
    autotuned).  c5: the same tiles served from device memory at Poisson
    arrival rates 10..500 /s; latency from submission to completion as the
    server records it."""
    tiles = []
    for t in synth.tiles_c4(seed=4, count=64, scale=1.0, px_multiple=8):
        d, Y, _ = synth.scene_torch(seed=t["seed"], m=t["m"], N=t["N"], n_hist=t["n_hist"], f=23.0, k_gen=t["k"],
                                    intercept=0.5, slope=0.0, coef_umax=0.3, noise_sd=0.04, miss="markov",
                                    p_a=t["p_a"], p_b=t["p_b"], break_frac=0.15, step=(-0.5, -0.1), dtype="i16",
                                    device=dev)
        design = bfm.Design(d, t["k"], 23.0)
        tiles.append(dict(t, Y=Y, design=design, lam=synth.lambda_for_horizon(t["N"] / t["n_hist"]),
                          out=bfm.empty_outputs(2 + 2 * t["k"], t["m"], dev)))
    total_px = sum(t["m"] for t in tiles)
    torch.cuda.synchronize()

    def call(t):
        o = t["out"]
        bfm.bfm_monitor_ex(t["design"], t["Y"], bfm.BFM_I16, None, t["m"], t["n_hist"], 0.25, t["lam"],
                           o["break_idx"], o["mean_mosum"], o["sigma"], o["beta"], o["status"], 0, stream)

    for t in tiles:  # warm-up
        call(t)
    torch.cuda.synchronize()
    lat, tot = [], 0.0
    for rep in range(3):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(tiles) + 1)]
        evs[0].record(stream)
        for i, t in enumerate(tiles):
            call(t)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(tiles))]
        lat += per
        tot += sum(per)
    lat.sort()
    c4 = {"workload": "c4: 64 int16 tiles, pixels log-U[1e4, 2e6] rounded up to multiples of 8, N ~ U{120..600}, "
                      "k ~ U{1..3}, history U(0.4, 0.7), Markov clouds 20-70 %",
          "pixels": total_px,
          "per_tile_calls": {"value": 3 * total_px / (tot / 1e3), "unit": "pixels/s",
                             "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1,
                                            int(math.ceil(0.99 * len(lat))) - 1)], "unit": "one tile"}}}
    names = {bfm.BFM_ALGO_HYBRID: "hybrid", bfm.BFM_ALGO_MMA: "tensor_core", bfm.BFM_ALGO_SIMT: "cuda_core"}

    def batched(forms):
        b = bfm.Batch(forms=forms)
        bouts = []
        for t in tiles:
            bouts.append(b.add(t["design"], t["Y"], n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]))
        by_form = {}
        for i, t in enumerate(tiles):
            f = names[b.form(i)]
            by_form[f] = by_form.get(f, 0) + t["m"]
        b.autotune(stream)
        b.run(stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            b.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / 5
        b.close()
        del bouts
        return {"value": total_px / (bms / 1e3), "unit": "pixels/s", "ms_per_batch": bms, "pixels_by_form": by_form}

    c4["batched_launch"] = dict(batched(bfm.BFM_ALGO_AUTO),
                                form="one CUDA-graph replay: persistent hybrid kernels per (k, storage, layout) "
                                     "group, persistent tensor-core kernels per (k, storage, CTAs per SM) group for "
                                     "the tiles whose ring does not fit the hybrid form, the CUDA-core kernel for "
                                     "the rest")
    c4["batched_launch_tensor_core_forms"] = dict(batched(bfm.BFM_ALGO_MMA),
                                                  form="the same batch limited to the tensor-core and CUDA-core forms")

    c5 = {"workload": "c5: the c4 tiles from device memory, Poisson arrivals", "rates": {}}
    rng = np.random.default_rng(5)
    for rate in (10, 20, 50, 100, 200, 500):
        n_req = min(1000, max(50, 2 * rate))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        srv = bfm.Server(hbm_budget=150 << 30, slots=4)
        tickets = []
        t0 = time.perf_counter()
        for i, a in enumerate(arrivals):
            while time.perf_counter() - t0 < a:
                pass
            t = tiles[i % len(tiles)]
            tickets.append(srv.submit(t["design"], t["Y"], n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]))
        srv.wait_all(120.0)
        st = srv.stats()
        for tk in tickets:
            srv.release(tk)
        srv.close()
        c5["rates"][str(rate)] = {"requests": n_req, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                                  "completed": st["completed"], "pixels_per_s": st["pixels"] / (st["span_ms"] / 1e3)}

    # the same server with Y in pinned host memory: each request's copy to the device runs on its
    # slot's stream and overlaps other requests' kernels (tiles up to about 4 GB of int16 in all)
    host_tiles, hbytes = [], 0
    for t in tiles:
        nb = t["Y"].numel() * 2
        if hbytes + nb > 4 << 30:
            continue
        hbytes += nb
        yh = torch.empty(t["Y"].shape, dtype=torch.int16, pin_memory=True)
        yh.copy_(t["Y"])
        host_tiles.append(dict(t, Yh=yh))
    torch.cuda.synchronize()
    c5["host_y"] = {"tiles": len(host_tiles), "pixels_per_pass": sum(t["m"] for t in host_tiles),
                    "host_bytes": hbytes, "rates": {}}
    for rate in (50, 200, "burst"):
        n_req = 200 if rate == "burst" else min(1000, max(50, 2 * rate))
        arrivals = np.zeros(n_req) if rate == "burst" else np.cumsum(rng.exponential(1.0 / rate, n_req))
        srv = bfm.Server(hbm_budget=150 << 30, slots=4)
        tickets = []
        t0 = time.perf_counter()
        for i, a in enumerate(arrivals):
            while time.perf_counter() - t0 < a:
                pass
            t = host_tiles[i % len(host_tiles)]
            tickets.append(srv.submit(t["design"], t["Yh"], n_hist=t["n_hist"], h_frac=0.25, lam=t["lam"]))
        srv.wait_all(120.0)
        st = srv.stats()
        for tk in tickets:
            srv.release(tk)
        srv.close()
        c5["host_y"]["rates"][str(rate)] = {"requests": n_req, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                                            "completed": st["completed"],
                                            "pixels_per_s": st["pixels"] / (st["span_ms"] / 1e3)}
    del host_tiles
    for t in tiles:
        t["design"].close()
    return c4, c5


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_1807_01751_gb300 as bfm
    import synth
    bfm.load()

    name = "c2"
    w = synth.workload_torch(name, device=dev, dtype="f32", m=args.pixels)
    m, N, n_hist, K = w["m"], w["N"], w["n_hist"], 8
    Y = w["Y"]
    design = bfm.Design(w["dates"], 3, 23.0)
    out = bfm.empty_outputs(K, m, dev)
    stream = torch.cuda.current_stream(dev)
    hbm, peak_kind = _peaks()

    def time_form(form):
        """Device-resident timing of one form: W warm-up calls, then K calls
        bracketed by CUDA events on the launching stream."""
        if form in ("f32", "f32simt", "f32stream", "f32hybrid"):
            Yf, dt = Y, bfm.BFM_F32
            algo = {"f32": bfm.BFM_ALGO_MMA, "f32simt": bfm.BFM_ALGO_SIMT, "f32stream": bfm.BFM_ALGO_STREAM,
                    "f32hybrid": bfm.BFM_ALGO_HYBRID}[form]
        elif form == "f32complete":
            # the same scene recipe without clouds: the shared pseudo-inverse form
            Yf = synth.workload_torch("c2_complete", device=dev, dtype="f32", m=args.pixels)["Y"]
            dt, algo = bfm.BFM_F32, bfm.BFM_ALGO_COMPLETE
        else:
            Yf = torch.where(torch.isnan(Y), torch.full_like(Y, -32768.0),
                             torch.clamp(torch.round(Y * 1e4), -32767, 32767)).to(torch.int16)
            dt = bfm.BFM_I16
            algo = {"i16stream": bfm.BFM_ALGO_STREAM, "i16hybrid": bfm.BFM_ALGO_HYBRID}.get(form, bfm.BFM_ALGO_MMA)

        def step():
            bfm.bfm_monitor_ex(design, Yf, dt, None, m, n_hist, w["h_frac"], w["lam"], out["break_idx"],
                               out["mean_mosum"], out["sigma"], out["beta"], out["status"], algo, stream)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if bfm.bfm_device_errors(stream) != 0:
            raise RuntimeError("device error word set during warm-up")
        clocks = Clocks(local)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        time.sleep(0.2)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        evs[0].record(stream)
        for i in range(args.steps):
            step()
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        clk = clocks.stop()
        per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
        total_ms = slowest_rank(evs[0].elapsed_time(evs[-1]), dev)
        # outputs and input columns of the seeded sample, for the error statement (after timing)
        samples[form] = dict(out={k: (v[:, sidx] if v.dim() == 2 else v[sidx]).cpu().numpy() for k, v in out.items()},
                             Y=Yf[:, sidx].cpu().numpy(), scene="complete" if form == "f32complete" else
                             ("i16" if form.startswith("i16") else "f32"))
        elt = 2 if form.startswith("i16") else 4
        alg_bytes = N * m * elt + m * (4 + 4 + 4 + 4 * K + 1)
        achieved = alg_bytes / (statistics.mean(per) / 1e3) / 1e9
        srt = sorted(per)
        del Yf
        return {"value": job_rate(m, args.steps, ws, total_ms), "ms_per_step": total_ms / args.steps,
                "latency_ms": {"p50": srt[len(srt) // 2],
                               "p99": srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)],
                               "unit": "one full-scene call"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "traffic": TRAFFIC_PER_PX.get(form, (None,))[0] and
                             TRAFFIC_PER_PX[form][0] * m, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                             "algorithmic_bytes_per_launch": alg_bytes},
                "clocks": clk, "dtype": "i16" if form.startswith("i16") else "f32",
                "algo": {"f32simt": "simt", "f32stream": "stream (CUDA cores, TMA stages)",
                         "i16stream": "stream (CUDA cores, TMA stages)",
                         "f32hybrid": "hybrid (tcgen05 contractions, CUDA-core scans, TMA stages)",
                         "i16hybrid": "hybrid (tcgen05 contractions, CUDA-core scans, TMA stages)",
                         "f32complete": "complete-series (shared pseudo-inverse)"}.get(form, "tcgen05")}

    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    samples = {}
    sidx = torch.from_numpy(np.unique(np.concatenate([
        np.arange(64), np.arange(m - 64, m),
        np.random.default_rng(0).choice(m, SAMPLE_PX - 128, replace=False)]))).to(dev)
    res = {f: time_form(f) for f in forms}
    form = forms[0]
    main = res[form]
    value, ms_step = main["value"], main["ms_per_step"]
    elt = 2 if form.startswith("i16") else 4

    # ---- end to end through the host-buffer entry point (pinned host Y and outputs): float32,
    # and the same scene stored as int16 (half the bytes over the host link)
    e2e = e2e_i16 = link = None
    if not args.no_e2e:
        Yh = torch.empty(Y.shape, dtype=Y.dtype, pin_memory=True)
        Yh.copy_(Y)
        Yh16 = torch.empty(Y.shape, dtype=torch.int16, pin_memory=True)
        Yh16.copy_(torch.where(torch.isnan(Y), torch.full_like(Y, -32768.0),
                               torch.clamp(torch.round(Y * 1e4), -32767, 32767)).to(torch.int16))
        oh = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
        chunk = 1 << 20
        wsb = max(bfm.bfm_monitor_host_workspace(design, bfm.BFM_F32, chunk, False),
                  bfm.bfm_monitor_host_workspace(design, bfm.BFM_I16, chunk, False))
        del Y
        torch.cuda.empty_cache()
        wbuf = torch.empty(wsb, dtype=torch.uint8, device=dev)
        # the host link itself: one pinned 1 GiB host-to-device copy
        lb = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
        lh = Yh.view(torch.uint8).reshape(-1)[:1 << 30]
        lb.copy_(lh, non_blocking=True)
        torch.cuda.synchronize()
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(stream)
        for _ in range(3):
            lb.copy_(lh, non_blocking=True)
        l1.record(stream)
        torch.cuda.synchronize()
        link = {"h2d_gbs": 3 * (1 << 30) / (l0.elapsed_time(l1) / 1e3) / 1e9,
                "how": "pinned host 1 GiB -> device, torch copy, 3 copies timed with CUDA events"}

        def slice_rates(src):
            # every 1 GiB slice of a pinned host buffer once: where its pages sit decides its rate
            flat = src.view(torch.uint8).reshape(-1)
            rates = []
            for o in range(0, flat.numel(), 1 << 30):
                n = min(1 << 30, flat.numel() - o)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lb[:n].copy_(flat[o:o + n], non_blocking=True)
                b.record(stream)
                torch.cuda.synchronize()
                rates.append(n / (a.elapsed_time(b) / 1e3) / 1e9)
            return {"min_gbs": min(rates), "median_gbs": sorted(rates)[len(rates) // 2], "max_gbs": max(rates),
                    "slices": len(rates)}

        link["y_f32_buffer"] = slice_rates(Yh)
        link["y_i16_buffer"] = slice_rates(Yh16)
        del lb

        def host_leg(Yhost, e_dt, e_elt):
            def hstep():
                bfm.bfm_monitor_host(design, Yhost, e_dt, None, m, n_hist, w["h_frac"], w["lam"], oh["break_idx"],
                                     oh["mean_mosum"], oh["sigma"], oh["beta"], oh["status"], wbuf, wsb, chunk, stream)

            hstep()
            torch.cuda.synchronize()
            e_steps = max(2, min(args.steps, 10))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(e_steps):
                hstep()
            e1.record(stream)
            torch.cuda.synchronize()
            e_ms = slowest_rank(e0.elapsed_time(e1) / e_steps, dev)
            return {"value": job_rate(m, 1, ws, e_ms), "unit": "pixels/s", "h2d_bytes_per_step": N * m * e_elt,
                    "d2h_bytes_per_step": m * (4 + 4 + 4 + 4 * K + 1), "ms_per_step": e_ms,
                    "api": "bfm_monitor_host (pinned host Y and outputs, 1 Mi-pixel chunks, form AUTO picks)",
                    "dtype": "f32" if e_elt == 4 else "i16"}

        e2e = host_leg(Yh, bfm.BFM_F32, 4)
        e2e_i16 = host_leg(Yh16, bfm.BFM_I16, 2)
        del Yh16
        Ysrc = Yh
    else:
        Ysrc = Y[:, :1 << 20].cpu()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, n, dt = cpu_oracle_rate(Ysrc, w["dates"], 3, 23.0, n_hist, w["h_frac"], w["lam"], budget_s=15.0)
        cpu = {"value": rate, "unit": "pixels/s", "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
               "kind": "oracle", "sample": f"first {n} pixels of the same scene, all {N} dates, FP64 oracle ({dt:.1f} s)"}
        cpu["one_core"] = cpu_oracle_one_core(Ysrc, w["dates"], n_hist, w["h_frac"], w["lam"])
        cpu["c1"] = cpu_oracle_c1()
        # the same oracle on the seeded sample of every timed form: each output's error against FP64
        ref_cache = {}
        for f, smp in samples.items():
            if smp["scene"] not in ref_cache:
                ref_cache[smp["scene"]] = oracle_on(smp["Y"], w["dates"], n_hist, w["h_frac"], w["lam"])
            res[f]["errors_vs_oracle"] = form_errors(smp["out"], ref_cache[smp["scene"]], w["dates"])

    # critical value of Eq. 4 by simulation (c2's alpha, h and N/n): 1e5 paths, 1000 steps per unit
    lam_sim = None
    if rank == 0:
        t0 = time.perf_counter()
        lam_v = bfm.bfm_lambda(0.05, 0.25, N / n_hist, G=1000, reps=100000, seed=12345, stream=stream)
        lam_ms = (time.perf_counter() - t0) * 1e3
        lam_sim = {"alpha": 0.05, "h": 0.25, "T": N / n_hist, "grid_per_unit": 1000, "paths": 100000,
                   "lambda": lam_v, "ms": lam_ms, "paths_per_s": 1e5 / (lam_ms / 1e3),
                   "note": "bfm_lambda, one FP64 path per thread, host quantile; wall time of the call"}

    # the per-pixel solve of Eq. 6 (two per pixel) in FP64 and in FP32, for every pixel of the scene
    solve = None
    if rank == 0:
        solve = {"systems": m, "K": K, "fp64_ms": bfm.bfm_solve_rate(K, m, True, stream),
                 "fp32_ms": bfm.bfm_solve_rate(K, m, False, stream),
                 "note": "bfm_solve_rate: Cholesky + two triangular solves, twice per system, CUDA events"}

    c4 = c5 = None
    if not args.no_c4c5:
        out = wbuf = Y = None  # the c2 scene's device buffers
        w["Y"] = None
        torch.cuda.empty_cache()
        c4, c5 = run_tiles_and_serving(bfm, synth, torch, dev, stream)

    line = {
        "metric": METRIC, "value": value, "unit": "pixels/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": main["dtype"], "data": "synthetic",
        "config": {"workload": (WORKLOAD if form != "i16" else WORKLOAD.replace("plain float32", "int16 storage"))
                   if args.pixels is None else f"c2 recipe with {m} pixels (profiling case)",
                   "pixels": m, "dates": N, "n_hist": n_hist, "K": K, "form": form, "algo": main["algo"],
                   "l2": "inputs larger than L2 (Y is %.1f GB per step)" % (N * m * elt / 1e9),
                   "parallelism": f"{ws} independent scene(s), one per GPU"},
        "latency_ms": main["latency_ms"], "roofline": main["roofline"],
        "cpu_baseline": cpu, "e2e": e2e, "e2e_int16": e2e_i16, "host_link": link, "clocks": main["clocks"],
        "gpu_launches": args.steps,
        "forms": {f: {k: v for k, v in r.items() if k != "clocks"} for f, r in res.items()},
        "c4": c4, "c5": c5, "lambda_simulation": lam_sim, "solve_fp64_vs_fp32": solve,
        "errors_vs_oracle": main.get("errors_vs_oracle"),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="f32hybrid,f32stream,f32,f32simt,i16hybrid,i16stream,i16,f32complete",
                    help="comma list; the first is the headline (f32hybrid = float storage, tensor-core "
                         "contractions with one CUDA-core thread per pixel for the scans (the form AUTO takes), "
                         "f32stream = float storage, the streaming CUDA-core form, f32 = float "
                         "storage on tensor cores, i16hybrid / i16stream = int16 storage in those forms, "
                         "f32simt = float storage on CUDA cores, i16 = int16 storage on tensor cores, "
                         "f32complete = the same scene without clouds in the shared pseudo-inverse form)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c4c5", action="store_true", help="skip the uneven-tile batch and serving legs")
    ap.add_argument("--pixels", type=int, default=None,
                    help="fewer pixels of the same recipe (profiling captures only; not a bench line)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
