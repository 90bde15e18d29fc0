#!/usr/bin/env python
"""Benchmark: multiple scattering with per-bounce stochastic LoD masks.

Workload (the largest single-GPU configuration): a 6-octave synthetic field of
1,000,000 Gabor primitives in the unit cube (the octave generator of
synth.octave_field, seed 0), a 1024x1024 pinhole camera, 64 samples per pixel,
up to 8 bounces, one directional light, isotropic phase, albedo 0.8, a new
mask per path segment: Uniform + control-variate bands with importance-sampled
orientation cones for camera, bounce and NEE rays.  FP32 records; the same
frame with FP16 records beside it.

One step renders 8 of the 64 samples of every pixel (samples 8j .. 8j+7 of
step j mod 8, through gf_render_opts.first_sample), so eight steps accumulate
the 64-spp frame.  The line reports Mrays/s (traced path segments: camera,
bounce and NEE rays), Gabor evaluations/s, render p50/p99 (per 8-spp step and
per 64-spp frame), the roofline of the render kernel against measured SFU and
FMA peaks, an end-to-end figure through the C ABI with host buffers, the
image RMSE against the FP64 oracle on sampled pixels beside the oracle's own
Monte Carlo noise, the oracle timed on the host cores, and the SM clocks
sampled during the timed region.  The single-scattering configuration (100k
primitives, 512x512, 16 spp, 4 band cutoffs) is reported as an extra key.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

import synth  # noqa: E402

N_PRIMS = 1_000_000
OCTAVES = 6
RES = 1024
SPP = 64          # samples per pixel of the frame
STEP_SPP = 8      # samples per pixel of one step
BOUNCES = 8
SEED = 3
METRIC = "Mrays/s and Gabor evals/s at fixed RMSE vs FP64 oracle; render p50/p99 ms"
WORKLOAD = ("multiple scattering, 1M-primitive 6-octave Gabor field, 1024x1024, 64 spp "
            "(8 per step), <= 8 bounces, per-bounce Uniform+CV bands and importance-sampled "
            "cones (camera, bounce and NEE rays)")
# single scattering, 100k primitives, 512x512, 16 spp, 4 band cutoffs (extra key)
C2_PRIMS, C2_OCTAVES, C2_RES, C2_SPP, C2_CUTOFFS, C2_SEED = 100_000, 4, 512, 16, (3, 2, 1, 0), 1
# DRAM bytes (read + write) per traced ray of k_render_scatter on this workload's field and
# masks, from ncu on a 256x256, 8-spp launch (profiles/k_render_scatter_full_cfg3_256x256_8spp.md:
# 2.371 GB for 3,516,025 rays), scaled to a launch by its traced rays; set to None whenever
# the kernel changes until it is captured again
TRAFFIC_BYTES_PER_RAY = 674.0
# warp instructions issued per traced ray by k_render_scatter on this workload (the same
# capture: 11.807 G for 3,516,025 rays); with the launch's rays per second, the median SM
# clock sampled during the timed steps and 4 schedulers per SM issuing one instruction a
# cycle, this gives the share of issue slots the kernel fills
INST_PER_RAY = 3358.0


def config(extra=None):
    c = {"workload": WORKLOAD, "primitives": N_PRIMS, "octaves": OCTAVES, "image": [RES, RES],
         "spp": SPP, "spp_per_step": STEP_SPP, "max_bounces": BOUNCES,
         "lod": "unif_cv bands + is cones, primary and NEE",
         "integrator": "delta tracking + ratio-tracked NEE, isotropic phase, albedo 0.8",
         "storage": "fp32 records", "l2": "flushed between timed steps (256 MiB write)",
         "parallelism": "replicas"}
    if extra:
        c.update(extra)
    return c


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(prefix="gf_clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--id=%d" % gpu_index, "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_setup():
    import oracle
    p = synth.octave_field(N_PRIMS, OCTAVES, seed=0)
    f = oracle.Field(p, omega_frame="local")
    c = synth.DEFAULT_CAMERA
    cam = oracle.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], RES, RES)
    ro = oracle.render_opts("scatter", SPP, BOUNCES, 0.8, synth.LIGHT_DIR, 1.0)
    lod = oracle.Lod(2, 7, 1)  # Uniform + CV bands, importance-sampled cones
    return oracle, f, cam, ro, lod


def oracle_pixels(seconds, crop=(4, 2), threads=0):
    """The FP64 oracle on crops of the benchmark frame (all 64 samples of each
    pixel, every sample kept) for about `seconds`: its rays/s on the host cores,
    and the per-sample values for the RMSE against the GPU frame."""
    oracle, f, cam, ro, lod = _oracle_setup()
    rng = np.random.default_rng(0)
    oracle.rays_traced(reset=True)
    t0 = time.perf_counter()
    crops = []
    while True:
        x, y = (int(v) for v in rng.integers(RES // 4, 3 * RES // 4 - 4, 2))
        smp = f.render(cam, ro, SEED, lod=lod, lod_nee=lod, crop=(x, y, crop[0], crop[1]),
                       samples=True, threads=threads)
        crops.append((x, y, smp))
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    rays = oracle.rays_traced(reset=True)
    return {"rays_per_s": rays / dt, "rays": rays, "seconds": dt, "crops": crops,
            "threads": threads or os.cpu_count()}


def oracle_sample(seconds):
    """cpu_baseline: the oracle on all host cores for ~`seconds`, plus a short
    single-thread run of one crop."""
    r = oracle_pixels(seconds)
    r1 = oracle_pixels(0.0, crop=(1, 1), threads=1)
    px = sum(c[2].shape[0] * c[2].shape[1] for c in r["crops"])
    return {"value": r["rays_per_s"] / 1e6, "unit": "Mrays/s", "cores": r["threads"],
            "kind": "oracle",
            "sample": "%d crops of 4x2 px of the benchmark frame at 64 spp, <= 8 bounces "
                      "(%d px, %d rays, %.1f s)" % (len(r["crops"]), px, r["rays"], r["seconds"]),
            "single_thread": {"value": r1["rays_per_s"] / 1e6, "unit": "Mrays/s",
                              "sample": "one pixel at 64 spp, %d rays, %.1f s"
                                        % (r1["rays"], r1["seconds"])}}, r["crops"]


def rmse_vs_oracle(frame, crops):
    """Image RMSE of the GPU frame against the oracle on the crops' pixels, beside
    the oracle's own Monte Carlo noise (standard error of each pixel's mean over
    its 64 samples) under the shared Philox streams."""
    d, sig = [], []
    for x, y, smp in crops:
        h, w, n = smp.shape
        d.append((frame[y:y + h, x:x + w] - smp.mean(-1)).ravel())
        sig.append((smp.std(-1, ddof=1) / math.sqrt(n)).ravel())
    d, sig = np.concatenate(d), np.concatenate(sig)
    rmse = float(np.sqrt(np.mean(d ** 2)))
    noise = float(np.sqrt(np.mean(sig ** 2)))
    return {"pixels": int(d.size), "rmse": rmse, "oracle_mc_noise": noise,
            "ratio": rmse / noise if noise > 0 else None,
            "criterion": "rmse <= 0.01 x oracle MC noise (shared streams)"}


SERVER_ASSETS = ((50_000, 4), (200_000, 4), (1_000_000, 6), (2_000_000, 6))


def server_leg(api, ctx, n_requests, load=0.7):
    """Render server on a Poisson stream of mixed requests over 4 resident assets.

    First, per asset, one request (512x512, 16 spp, all bands) through
    gf_render and through the server alone: Mrays/s of each.  Then the first
    n_requests of the seeded request stream (resolution uniform over
    128^2..1024^2, spp over {1,4,16,64}, LoD over the 4 band cutoffs, random
    cameras on a sphere) are submitted all at once to measure the saturated
    request rate, then replayed at load x that rate as Poisson arrivals;
    latency = submit -> image in the caller's (pinned host) buffer.
    """
    import torch
    fields = [api.Field(ctx, synth.octave_field(n, o, seed=10 + k))
              for k, (n, o) in enumerate(SERVER_ASSETS)]
    stream = synth.request_stream(n_requests, 1.0, seed=0, lods=(0, 1, 2, 3))
    srv = api.Server(ctx, fields, mem_budget=512 << 20, max_inflight=32, max_queue=100000)
    c = synth.DEFAULT_CAMERA

    def request_args(r):
        eye = r["eye"]
        d = np.subtract(c["look_at"], eye)
        up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.99 * np.linalg.norm(d) else (0.0, 0.0, 1.0)
        cam = api.camera(eye, c["look_at"], up, c["vfov_deg"], r["res"], r["res"])
        ro = api.render_opts("scatter", r["spp"], 1, 0.8, synth.LIGHT_DIR, 1.0)
        top = SERVER_ASSETS[r["asset"]][1] - 1
        lo = api.lod("cutoff", top - r["lod"])
        return cam, ro, lo

    def submit(r):
        cam, ro, lo = request_args(r)
        t, _ = srv.submit(r["asset"], cam, ro, lo, lo, r["seed"])
        return t

    try:
        # one request per asset, alone: through gf_render and through the server
        per_asset = {}
        for k, (n, _) in enumerate(SERVER_ASSETS):
            r = {"eye": (0.5, 0.5, -1.0), "res": 512, "spp": 16, "asset": k, "lod": 0, "seed": 7}
            cam, ro, lo = request_args(r)
            f = fields[k]
            f.set_lod(lo, lo)
            out = torch.empty(512, 512, device="cuda")
            f.render(cam, ro, seed=7, out=out)
            torch.cuda.synchronize()
            f.stats(reset=True)
            t0 = time.perf_counter()
            f.render(cam, ro, seed=7, out=out)
            torch.cuda.synchronize()
            t_render = time.perf_counter() - t0
            rays = f.stats(reset=True)["rays"]
            s0 = srv.stats()
            t0 = time.perf_counter()
            srv.wait(submit(r))
            t_server = time.perf_counter() - t0
            s1 = srv.stats()
            per_asset[str(n)] = {"gf_render_mrays_per_s": rays / t_render / 1e6,
                                 "server_alone_mrays_per_s":
                                     (s1["work"]["rays"] - s0["work"]["rays"]) / t_server / 1e6,
                                 "gf_render_ms": 1e3 * t_render, "server_ms": 1e3 * t_server}
        # the first 16 requests of the stream through gf_render one after another,
        # and through the server queued at once
        same = stream[:16]
        rays_r, t_r = 0, 0.0
        for r in same:
            cam, ro, lo = request_args(r)
            f = fields[r["asset"]]
            f.set_lod(lo, lo)
            out = torch.empty(r["res"], r["res"], device="cuda")
            torch.cuda.synchronize()
            f.stats(reset=True)
            t0 = time.perf_counter()
            f.render(cam, ro, seed=r["seed"], out=out)
            torch.cuda.synchronize()
            t_r += time.perf_counter() - t0
            rays_r += f.stats(reset=True)["rays"]
        s0 = srv.stats()
        t0 = time.perf_counter()
        for t in [submit(r) for r in same]:
            srv.wait(t)
        t_s = time.perf_counter() - t0
        s1 = srv.stats()
        same_requests = {"requests": len(same), "gf_render_mrays_per_s": rays_r / t_r / 1e6,
                         "server_mrays_per_s": (s1["work"]["rays"] - s0["work"]["rays"]) / t_s / 1e6,
                         "gf_render_s": t_r, "server_s": t_s}
        # saturated throughput: the whole sample queued at once
        s0 = srv.stats()
        t0 = time.perf_counter()
        tk = [submit(r) for r in stream]
        for t in tk:
            srv.wait(t)
        sat_s = time.perf_counter() - t0
        s1 = srv.stats()
        rate = load * n_requests / sat_s
        # Poisson arrivals at `load` of the saturated rate
        t0 = time.perf_counter()
        tk = []
        for r in stream:
            due = t0 + r["t_arrive"] / rate
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                time.sleep(min(0.002, due - now))
            tk.append(submit(r))
        res = [srv.wait(t) for t in tk]
        span_s = time.perf_counter() - t0
        s2 = srv.stats()
    finally:
        srv.close()
        for f in fields:
            f.free()
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in res])
    wait = np.array([r["t_admit_ms"] - r["t_submit_ms"] for r in res])
    samples = sum(r["res"] ** 2 * r["spp"] for r in stream)
    rays = s2["work"]["rays"] - s1["work"]["rays"]
    return {
        "requests": n_requests, "sample": "first %d requests of the seeded 2000-request stream"
                                          % n_requests,
        "assets": [n for n, _ in SERVER_ASSETS], "failed": int(s2["failed"]),
        "per_asset_512x512_16spp": per_asset,
        "same_requests_gf_render_vs_server": same_requests,
        "saturated_requests_per_s": n_requests / sat_s,
        "saturated_mrays_per_s": (s1["work"]["rays"] - s0["work"]["rays"]) / sat_s / 1e6,
        "poisson_rate_per_s": rate, "load": load,
        "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
        "queue_wait_ms_p50": float(np.percentile(wait, 50)),
        "queue_wait_ms_p99": float(np.percentile(wait, 99)),
        "mrays_per_s": rays / span_s / 1e6, "msamples_per_s": samples / span_s / 1e6,
        "launches": int(s2["launches"] - s1["launches"]),
        "gpu_busy_frac": (s2["busy_ms"] - s1["busy_ms"]) / (span_s * 1e3),
        "max_inflight_seen": int(s2["max_inflight_seen"]),
    }


# ---------------------------------------------------------------------------
# Other workloads of the method, one JSON line each (bench.py --workload NAME);
# the default line is the single-scattering workload above.
# ---------------------------------------------------------------------------
def _timed(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def workload_line(name, value, unit, ms, args, extra, higher=True):
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": higher,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_workload(args):
    """Transmittance, multiple scattering with stochastic masks, and the adjoints."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_05081_gb300 import _abi, api
    ctx = api.Context(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    c = synth.DEFAULT_CAMERA
    if args.workload == "transmittance":
        # 256 absorption-only kernels, 64x64 orthographic rays: deterministic optical
        # depth and 1-spp ratio tracking, all bands
        p = synth.absorption_field(256, seed=0)
        f = api.Field(ctx, p)
        o, d, tr = (torch.from_numpy(a).to(dev) for a in synth.orthographic_rays(64))
        n = o.shape[0]
        T = torch.empty(n, device=dev)
        tau = torch.empty(n, device=dev)
        out, batch = {}, {}
        modes = {"det": _abi.GF_TR_DETERMINISTIC, "closed": _abi.GF_TR_CLOSED_FORM,
                 "rt": _abi.GF_TR_RATIO_TRACKING}
        for mode, m in modes.items():
            call = lambda: _abi.gf_transmittance(f.h, o, d, tr, n, m, 1, 0, T, tau, stream)  # noqa: E731
            # one call between two events (latency, host enqueue included) ...
            out[mode] = statistics.median(_timed(call, args.steps * 50, args.warmup, stream))
            # ... and 100 calls enqueued back to back (throughput)
            def hundred():
                for _ in range(100):
                    call()
            batch[mode] = statistics.median(_timed(hundred, args.steps, 1, stream)) / 100
        f.sync()
        # throughput: 1M random rays through the 100k-kernel 4-octave field,
        # Gauss-Legendre quadrature against the closed form
        q = synth.octave_field(100_000, 4, seed=0)
        g = api.Field(ctx, q)
        nb = 1 << 20
        ob, db, trb = (torch.from_numpy(a).to(dev) for a in synth.random_rays(nb, seed=3))
        Tb = torch.empty(nb, device=dev)
        taub = {k: torch.empty(nb, device=dev) for k in ("det", "closed")}
        big = {}
        for mode in ("det", "closed"):
            m = modes[mode]
            call = lambda: _abi.gf_transmittance(g.h, ob, db, trb, nb, m, 1, 0, Tb,  # noqa: E731
                                                 taub[mode], stream)
            big[mode] = statistics.median(_timed(call, args.steps * 2, args.warmup, stream))
        g.sync()
        dtau = (taub["det"] - taub["closed"]).abs().max().item()
        scale = max(1.0, taub["det"].abs().max().item())
        workload_line("absorption transmittance, 256 kernels, 64x64 orthographic rays",
                      n / (batch["det"] * 1e-3) / 1e6, "Mrays/s", batch["det"], args,
                      {"us_per_call_latency": {k: v * 1e3 for k, v in out.items()},
                       "us_per_call_back_to_back": {k: v * 1e3 for k, v in batch.items()},
                       "ratio_tracking_mrays_per_s": n / (batch["rt"] * 1e-3) / 1e6,
                       "closed_form_mrays_per_s": n / (batch["closed"] * 1e-3) / 1e6,
                       "octave_100k_1m_rays_mrays_per_s": {k: nb / (v * 1e-3) / 1e6
                                                           for k, v in big.items()},
                       "octave_100k_max_dtau_det_vs_closed_rel": dtau / scale,
                       "gpu_launches": 1})
    elif args.workload == "multiscatter":
        # 1M kernels in 6 octaves, up to 8 bounces, per-bounce Uniform+CV band and
        # importance-sampled cone masks, FP32 and FP16 records
        res = args.res or 1024
        spp = args.spp or 64
        p = synth.octave_field(1_000_000, 6, seed=0)
        cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], res, res)
        ro = api.render_opts("scatter", spp, 8, 0.8, synth.LIGHT_DIR, 1.0)
        out = torch.empty(res, res, device=dev)
        lo = api.lod("unif_cv", 7, "is")
        res_ms, rays = {}, {}
        for prec in ("fp32", "fp16"):
            f = api.Field(ctx, p, precision=prec)
            f.set_lod(lo, lo)
            f.stats(reset=True)
            ms = _timed(lambda: f.render(cam, ro, seed=3, out=out), args.steps, 1, stream)
            f.sync()
            st = f.stats(reset=True)
            rays[prec] = st["rays"] / (1 + args.steps)
            res_ms[prec] = statistics.mean(ms)
            f.free()
        workload_line("multiple scattering, 1M-kernel 6-octave field, %dx%d, %d spp, <= 8 bounces, "
                      "per-bounce stochastic LoD masks" % (res, res, spp),
                      rays["fp32"] / (res_ms["fp32"] * 1e-3) / 1e6, "Mrays/s", res_ms["fp32"], args,
                      {"ms_per_render": res_ms,
                       "mrays_per_s": {k: rays[k] / (res_ms[k] * 1e-3) / 1e6 for k in rays},
                       "gpu_launches": 2})
    elif args.workload == "clamping":
        # adaptive clamping (Sec. 4.4) on the single-scattering benchmark field and
        # camera, all bands, at several thresholds; camera-Nyquist LoD selection
        # (Supp. A) on 128x128 thumbnails of the same field.  Image differences are
        # set beside the Monte Carlo noise: the RMSE between two renders of the
        # unmodified field that differ only in the seed.
        res = args.res or 512
        spp = args.spp or 16
        p = synth.octave_field(100_000, 4, seed=0)
        ro = api.render_opts("scatter", spp, 1, 0.8, synth.LIGHT_DIR, 1.0)

        def measure(f, cam, seed=2):
            out = torch.empty(cam.height, cam.width, device=dev)
            f.stats(reset=True)
            ms = _timed(lambda: f.render(cam, ro, seed=seed, out=out), args.steps, args.warmup, stream)
            f.sync()
            st = f.stats(reset=True)
            rays = st["rays"] / (args.steps + args.warmup)
            return out.clone(), {"ms_per_render": statistics.mean(ms),
                                 "mrays_per_s": rays / (statistics.mean(ms) * 1e-3) / 1e6,
                                 "chords_per_ray": st["chords"] / max(1, st["rays"]),
                                 "nodes_per_ray": st["nodes"] / max(1, st["rays"])}

        def rmse(a, b):
            return (a - b).pow(2).mean().sqrt().item()

        cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], res, res)
        rows, ref = {}, None
        for eps in (0.0, 1e-3, 3e-3, 1e-2):
            f = api.Field(ctx, p, clamp_eps=eps)
            img, row = measure(f, cam)
            if ref is None:
                ref = img
                other, _ = measure(f, cam, seed=3)
                noise = rmse(img, other)
            row["image_rmse_vs_unclamped"] = rmse(img, ref)
            rows[str(eps)] = row
            f.free()
        thumb = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], 128, 128)
        f = api.Field(ctx, p)
        full, row_full = measure(f, thumb)
        other, _ = measure(f, thumb, seed=3)
        f.set_lod_camera(thumb)
        sel, row_sel = measure(f, thumb)
        f.free()
        row_sel["image_rmse_vs_unfiltered"] = rmse(sel, full)
        workload_line("adaptive clamping, 100k-primitive 4-octave field, %dx%d, %d spp, all bands"
                      % (res, res, spp), rows["0.01"]["mrays_per_s"], "Mrays/s",
                      rows["0.01"]["ms_per_render"], args,
                      {"by_clamp_eps": rows, "image_rms": ref.pow(2).mean().sqrt().item(),
                       "seed_to_seed_rmse": noise,
                       "camera_lod_128x128": {"unfiltered": row_full, "nyquist": row_sel,
                                              "seed_to_seed_rmse": rmse(full, other)},
                       "gpu_launches": 2})
    elif args.workload == "free_flight":
        # free flight by delta tracking against inversion of the optical-depth CDF
        # (bisection on the closed-form tau, closed-form NEE transmittance): the
        # benchmark field's Gaussian band (a non-negative density), single
        # scattering, at equal samples per pixel; the noise of each is the RMSE
        # between two renders that differ only in the seed
        res = args.res or 256
        spp = args.spp or 4
        p = synth.octave_field(100_000, 4, seed=0)
        cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], res, res)
        f = api.Field(ctx, p)
        f.set_lod(api.lod("cutoff", 0))
        # reference: delta tracking (unbiased) at 16x the samples, another seed
        ref = torch.empty(res, res, device=dev)
        f.render(cam, api.render_opts("scatter", 16 * spp, 1, 0.8, synth.LIGHT_DIR, 1.0), seed=7,
                 out=ref)
        f.sync()
        rows, imgs = {}, {}
        for mode in ("delta", "cdf", "segment"):
            ro = api.render_opts("scatter", spp, 1, 0.8, synth.LIGHT_DIR, 1.0, free_flight=mode)
            a = torch.empty(res, res, device=dev)
            b = torch.empty(res, res, device=dev)
            f.stats(reset=True)
            ms = _timed(lambda: f.render(cam, ro, seed=2, out=a), args.steps, args.warmup, stream)
            f.sync()
            st = f.stats(reset=True)
            f.render(cam, ro, seed=3, out=b)
            f.sync()
            imgs[mode] = a.clone()
            noise = (a - b).pow(2).mean().sqrt().item() / math.sqrt(2.0)
            t = statistics.mean(ms)
            rmse = (a - ref).pow(2).mean().sqrt().item()
            rows[mode] = {"ms_per_render": t,
                          "mrays_per_s": st["rays"] / (args.steps + args.warmup) / (t * 1e-3) / 1e6,
                          "nodes_per_ray": st["nodes"] / max(1, st["rays"]),
                          "pixel_noise_rms": noise, "time_x_variance": t * noise * noise,
                          "rmse_vs_reference": rmse, "time_x_mse": t * rmse * rmse}
        f.free()
        rows["image_mean"] = {k: v.mean().item() for k, v in imgs.items()}
        rows["reference"] = {"free_flight": "delta", "spp": 16 * spp, "mean": ref.mean().item()}
        workload_line("free flight, Gaussian band of the 100k-primitive 4-octave field, %dx%d, %d spp"
                      % (res, res, spp), rows["cdf"]["mrays_per_s"], "Mrays/s",
                      rows["cdf"]["ms_per_render"], args, {"by_free_flight": rows, "gpu_launches": 1})
    elif args.workload == "beta":
        # the power-law band choice with the Gaussian band as control variate (App. B,
        # POW_CV) against all bands and Uniform + CV: time and image RMSE against an
        # all-bands reference at 16x the samples, single scattering, 100k-primitive field;
        # time x MSE is the cost of a given RMSE for these unbiased estimators
        res = args.res or 256
        spp = args.spp or 16
        p = synth.octave_field(100_000, 4, seed=0)
        cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], res, res)
        f = api.Field(ctx, p)
        ro = api.render_opts("scatter", spp, 1, 0.8, synth.LIGHT_DIR, 1.0)
        ref = torch.empty(res, res, device=dev)
        f.set_lod(api.lod())
        f.render(cam, api.render_opts("scatter", 16 * spp, 1, 0.8, synth.LIGHT_DIR, 1.0), seed=7,
                 out=ref)
        f.sync()
        rows = {}
        cases = [("all", api.lod()), ("unif_cv", api.lod("unif_cv", 7))] + \
            [("pow_cv beta=%g" % b, api.lod("pow_cv", 7, "all", b)) for b in (0.0, 0.25, 0.5, 0.75)]
        for name, lo in cases:
            f.set_lod(lo, lo)
            out = torch.empty(res, res, device=dev)
            ms = _timed(lambda: f.render(cam, ro, seed=2, out=out), args.steps, args.warmup, stream)
            f.sync()
            t = statistics.mean(ms)
            rmse = (out - ref).pow(2).mean().sqrt().item()
            rows[name] = {"ms_per_render": t, "rmse_vs_reference": rmse, "time_x_mse": t * rmse * rmse}
        f.free()
        best = min((v["time_x_mse"], k) for k, v in rows.items())[1]
        workload_line("power-law band choice with control variate, beta sweep, 100k-primitive "
                      "4-octave field, %dx%d, %d spp, single scattering" % (res, res, spp),
                      rows[best]["ms_per_render"], "ms per render (most efficient strategy)",
                      rows[best]["ms_per_render"], args,
                      {"by_strategy": rows, "most_efficient": best,
                       "reference": "all bands, %d spp, another seed" % (16 * spp),
                       "gpu_launches": 2}, higher=False)
    elif args.workload == "precision":
        # FP32 against FP16/BF16 records as the field outgrows the 129 MB L2: 6-octave
        # fields of 1M, 2M and 4M kernels, single scattering, 512x512, 4 spp, all bands;
        # the image difference between storages beside the seed-to-seed noise
        res = args.res or 512
        spp = args.spp or 4
        cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], res, res)
        ro = api.render_opts("scatter", spp, 1, 0.8, synth.LIGHT_DIR, 1.0)
        rows = {}
        for n in (1_000_000, 2_000_000, 4_000_000):
            p = synth.octave_field(n, 6, seed=0)
            row, ref = {}, None
            for prec in ("fp32", "fp16", "bf16"):
                f = api.Field(ctx, p, precision=prec)
                out = torch.empty(res, res, device=dev)
                ms = _timed(lambda: f.render(cam, ro, seed=2, out=out), args.steps, args.warmup, stream)
                f.sync()
                img = out.clone()
                entry = {"ms_per_render": statistics.mean(ms)}
                if ref is None:
                    ref = img
                    f.render(cam, ro, seed=3, out=out)
                    f.sync()
                    row["seed_to_seed_rmse"] = (img - out).pow(2).mean().sqrt().item()
                else:
                    entry["image_rmse_vs_fp32"] = (img - ref).pow(2).mean().sqrt().item()
                row[prec] = entry
                f.free()
                torch.cuda.empty_cache()
            row["record_mb"] = {"fp32": 64 * n / 2 ** 20, "reduced": 32 * n / 2 ** 20}
            rows[str(n)] = row
        big = rows[str(4_000_000)]
        workload_line("record precision vs field size, 6-octave fields of 1M/2M/4M kernels, %dx%d, "
                      "%d spp, all bands" % (res, res, spp), big["fp32"]["ms_per_render"] /
                      big["fp16"]["ms_per_render"], "x (FP16 speed-up at 4M)",
                      big["fp16"]["ms_per_render"], args, {"by_kernels": rows, "gpu_launches": 2})
    elif args.workload == "adjoint":
        # 200k kernels, 256x256 at 8 spp: forward render plus hand-written adjoint of an
        # L2 loss against a target rendered from perturbed parameters (--res/--spp: profiling)
        res, spp = args.res or 256, args.spp or 8
        p = synth.octave_field(200_000, 4, seed=0)
        rng = np.random.default_rng(1)
        tgt = dict(p)
        for k in ("mu", "log_scale", "weight"):
            tgt[k] = (p[k] * (1 + 0.01 * rng.standard_normal(p[k].shape))).astype(np.float32)
        cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], res, res)
        out = {}
        for name, integ, nb in (("tomo", "tomo", 1), ("scatter", "scatter", 1),
                                ("scatter_3_bounces", "scatter", 3)):
            ro = api.render_opts(integ, spp, nb, 0.8, synth.LIGHT_DIR, 1.0)
            ft = api.Field(ctx, tgt)
            target = ft.render(cam, ro, seed=11)
            ft.free()
            f = api.Field(ctx, p)
            grad = torch.empty(15 * f.n, device=dev)

            def step():
                img = f.render(cam, ro, seed=12)
                g = 2.0 * (img - target)
                f.render_backward(cam, ro, 13, g, grad=grad)
            ms = _timed(step, args.steps, args.warmup, stream)
            f.sync()
            out[name] = statistics.mean(ms)
            f.free()
        workload_line("differentiable rendering, 200k kernels, %dx%d, %d spp, forward + adjoint"
                      % (res, res, spp),
                      res * res * spp / (out["scatter"] * 1e-3) / 1e6, "Msamples/s", out["scatter"],
                      args, {"ms_per_forward_backward": out, "gpu_launches": 3})
    ctx.close()


def run_reference(args, rank, world):
    """The FP64 oracle as the comparison program: each step renders one 4x2-pixel
    crop of the benchmark frame at its full 64 spp and <= 8 bounces on the host
    cores; Mrays/s over the timed steps."""
    if rank != 0:
        return
    import oracle
    oracle_, f, cam, ro, lod = _oracle_setup()
    rng = np.random.default_rng(1)

    def step():
        x, y = (int(v) for v in rng.integers(RES // 4, 3 * RES // 4 - 4, 2))
        f.render(cam, ro, SEED, lod=lod, lod_nee=lod, crop=(x, y, 4, 2))

    for _ in range(args.warmup):
        step()
    oracle.rays_traced(reset=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    rays = oracle.rays_traced(reset=True)
    value = rays / dt / 1e6
    cb = {"value": value, "unit": "Mrays/s", "cores": os.cpu_count(), "kind": "oracle",
          "sample": "%d crops of 4x2 px of the benchmark frame at 64 spp, <= 8 bounces, %d rays, "
                    "%.1f s" % (args.steps, rays, dt)}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mrays/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * dt / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"engine": "FP64 CPU oracle (OpenMP)", "storage": "fp64"}),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def combine_ranks(total_ms, rays, evals, world, device):
    """Whole-job figures of N replicas: the slowest rank's timed milliseconds
    and the work summed over ranks (one all-reduce each; no data-path
    collective exists, every rank renders its own copy of the workload)."""
    if world <= 1:
        return float(total_ms), float(rays), float(evals)
    import torch
    import torch.distributed as dist
    tmax = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    sums = torch.tensor([float(rays), float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(sums, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(sums[0]), float(sums[1])


def config2_leg(api, ctx, dev, stream, steps=2):
    """Single scattering, 100k primitives, 512x512, 16 spp, the 4 band cutoffs:
    Mrays/s and per-render times (the second configuration of the method)."""
    import torch
    p = synth.octave_field(C2_PRIMS, C2_OCTAVES, seed=0)
    f = api.Field(ctx, p)
    c = synth.DEFAULT_CAMERA
    cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], C2_RES, C2_RES)
    ro = api.render_opts("scatter", C2_SPP, 1, 0.8, synth.LIGHT_DIR, 1.0)
    out = torch.empty(C2_RES, C2_RES, device=dev)
    lods = [api.lod("cutoff", k) for k in C2_CUTOFFS]
    for lo in lods:
        f.set_lod(lo)
        f.render(cam, ro, seed=C2_SEED, out=out, stream=stream)
    torch.cuda.synchronize()
    f.stats(reset=True)
    ms = {k: [] for k in C2_CUTOFFS}
    for _ in range(steps):
        for k, lo in zip(C2_CUTOFFS, lods):
            f.set_lod(lo)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f.render(cam, ro, seed=C2_SEED, out=out, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms[k].append(a.elapsed_time(b))
    f.sync()
    st = f.stats(reset=True)
    f.free()
    tot = sum(sum(v) for v in ms.values())
    return {"workload": "single scattering, 100k-primitive 4-octave field, 512x512, 16 spp, "
                        "4 LoD band cutoffs (all, <=1/2, <=1/4, <=1/8)",
            "mrays_per_s": st["rays"] / (tot * 1e-3) / 1e6,
            "gabor_evals_per_s": st["evals"] / (tot * 1e-3),
            "render_ms_by_cutoff": {str(k): statistics.mean(v) for k, v in ms.items()},
            "ms_per_step_of_4_renders": tot / steps}


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2602_05081_gb300 import _abi, api

    ctx = api.Context(local)
    sfu_peak, fma_peak = _abi.gf_measure_peaks(local)
    p = synth.octave_field(N_PRIMS, OCTAVES, seed=0)
    field = api.Field(ctx, p)
    lod = api.lod("unif_cv", 7, "is")
    field.set_lod(lod, lod)
    c = synth.DEFAULT_CAMERA
    cam = api.camera(c["eye"], c["look_at"], c["up"], c["vfov_deg"], RES, RES)
    out = torch.empty(RES, RES, dtype=torch.float32, device=dev)
    frame_sum = torch.zeros(RES, RES, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    nslice = SPP // STEP_SPP
    opts = [api.render_opts("scatter", STEP_SPP, BOUNCES, 0.8, synth.LIGHT_DIR, 1.0,
                            first_sample=STEP_SPP * j) for j in range(nslice)]

    for j in range(args.warmup):
        _abi.gf_render(field.h, cam, opts[j % nslice], SEED, out, stream)
    field.sync(stream)
    field.stats(reset=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    step_ms = []
    frames_done = 0
    for j in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _abi.gf_render(field.h, cam, opts[j % nslice], SEED, out, stream)
        b.record(stream)
        torch.cuda.synchronize()
        step_ms.append(a.elapsed_time(b))
        frame_sum += out.double()
        if j % nslice == nslice - 1:
            frames_done += 1
            if frames_done == 1:
                frame = (frame_sum / nslice).float().cpu().numpy()
            frame_sum.zero_()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    field.sync(stream)
    st = field.stats(reset=True)
    total_ms_max, rays_all, evals_all = combine_ranks(sum(step_ms), st["rays"], st["evals"],
                                                      world, dev)
    if frames_done == 0:  # fewer steps than one frame: finish the frame untimed
        for j in range(args.steps, nslice):
            _abi.gf_render(field.h, cam, opts[j], SEED, out, stream)
            frame_sum += out.double()
        frame = (frame_sum / nslice).float().cpu().numpy()
        field.stats(reset=True)
    # end to end through the C ABI with a host (pinned) output buffer
    host = torch.empty(RES, RES, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    field.stats(reset=True)
    t0 = time.perf_counter()
    for j in range(args.steps):
        _abi.gf_render(field.h, cam, opts[j % nslice], SEED, host, stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    st_e2e = field.stats(reset=True)
    # the whole 64-spp frame with 32-byte FP16 records (FP32 math) and with FP32 records
    frame_ms = {}
    for prec in ("fp32", "fp16"):
        fr = field if prec == "fp32" else api.Field(ctx, p, precision=prec)
        fr.set_lod(lod, lod)
        _abi.gf_render(fr.h, cam, opts[0], SEED, out, stream)
        flush.fill_(1.0)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for j in range(nslice):
            _abi.gf_render(fr.h, cam, opts[j], SEED, out, stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        fr.sync(stream)
        frame_ms[prec] = ev0.elapsed_time(ev1)
        if prec != "fp32":
            fr.free()
    if rank != 0:
        return
    import ctypes
    launches = args.steps  # one k_render_scatter (+ one k_fix_to_image) per step
    evals_per_launch = st["evals"] / launches
    achieved = evals_per_launch / (statistics.mean(step_ms) * 1e-3)
    peaks, peak_kind = measured_peaks()
    value = rays_all / (total_ms_max * 1e-3) / 1e6
    rays_per_launch = st["rays"] / launches
    traffic = TRAFFIC_BYTES_PER_RAY * rays_per_launch if TRAFFIC_BYTES_PER_RAY else None
    nominal = torch.cuda.get_device_properties(dev).multi_processor_count * 8 * \
        peaks.get("sm_max_mhz", 2070.0) * 1e6
    line = {
        "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config(),
        "gabor_evals_per_s": evals_all / (total_ms_max * 1e-3),
        "render_ms_p50": float(np.percentile(step_ms, 50)),
        "render_ms_p99": float(np.percentile(step_ms, 99)),
        "render_ms_per_64spp_frame": frame_ms,
        "rays_per_step": st["rays"] / args.steps,
        "evals_per_step": st["evals"] / args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": sfu_peak / 1e9,
                     "unit": "Geval/s", "frac": achieved / sfu_peak, "traffic": traffic,
                     "kernel": "k_render_scatter (delta + ratio tracking, stochastic masks)",
                     "peak_basis": "measured: (ex2.approx, cos.approx) pairs per second on every "
                                   "SM (gf_measure_peaks), one pair per Gabor evaluation; nominal "
                                   "16 MUFU/clk/SM would give %.0f Geval/s" % (nominal / 1e9),
                     "fma_peak_per_s": fma_peak},
        "e2e": {"value": st_e2e["rays"] / e2e_s / 1e6, "unit": "Mrays/s",
                "h2d_bytes_per_step": ctypes.sizeof(_abi.gf_camera) + ctypes.sizeof(_abi.gf_render_opts),
                "d2h_bytes_per_step": RES * RES * 4},
        "gpu_launches": 2 * args.steps,  # k_render_scatter + k_fix_to_image per step
        "storage_ms_per_frame": frame_ms,
        "clocks": clk,
    }
    if INST_PER_RAY and clk.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        issued = INST_PER_RAY * rays_per_launch / (statistics.mean(step_ms) * 1e-3)
        slots = 4.0 * sms * clk["sm_mhz"] * 1e6
        line["issue_utilisation"] = {
            "warp_inst_per_s": issued, "issue_slots_per_s": slots, "frac": issued / slots,
            "basis": "ncu warp instructions per traced ray of the 256x256 capture x traced "
                     "rays per second / (4 schedulers x SMs x median SM clock)"}
    line["counters_per_ray"] = {k: st[k] / max(1, st["rays"])
                                for k in ("chords", "evals", "nodes", "points", "windows", "steps", "leaves")}
    if any(st["cycles"]):
        tot = max(1, sum(st["cycles"]))
        line["phase_cycles_share"] = dict(zip(("traversal_steps", "leaf_rounds", "chord_walks",
                                               "point_evaluation", "decisions"),
                                              (c_ / tot for c_ in st["cycles"])))
    if world == 1 and args.config2:
        line["config2"] = config2_leg(api, ctx, dev, stream)
    if world == 1 and args.server_requests > 0:
        line["server"] = server_leg(api, ctx, args.server_requests)
    if world == 1 and args.cpu_seconds > 0:
        cb, crops = oracle_sample(args.cpu_seconds)
        line["cpu_baseline"] = cb
        line["rmse_vs_oracle"] = rmse_vs_oracle(frame, crops)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--server-requests", type=int, default=100,
                    help="requests of the render-server leg (0: skip)")
    ap.add_argument("--config2", type=int, default=1,
                    help="add the single-scattering configuration as an extra key (0: skip)")
    ap.add_argument("--workload", choices=["scatter", "transmittance", "multiscatter", "adjoint",
                                           "clamping", "free_flight", "precision", "beta"],
                    default="scatter", help="workload of the JSON line (default: the multiple-"
                    "scattering benchmark)")
    ap.add_argument("--res", type=int, default=None, help="profiling only: image size")
    ap.add_argument("--spp", type=int, default=None, help="profiling only: samples per pixel")
    args = ap.parse_args()
    if args.workload == "scatter":
        globals()["RES"] = args.res or RES
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload != "scatter":
        if rank == 0:
            run_workload(args)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
