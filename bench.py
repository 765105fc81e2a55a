"""Benchmark of the smeared-PSF hot path on GB300.

Workload (default): the MeerKAT-shaped single cutout -- 64 antennas (32 within
1 km, 32 within 8 km; 2016 baselines), 4 h of 1 s samples averaged 8:1, 16
channels of 0.836 MHz from 856 MHz (58 060 800 averaged visibilities), one
128 x 128 cutout at 1.5 arcsec around (l0, m0) = (0.03, 0.03).  One step
evaluates the exact smeared PSF and both approximations (psf_exact and
psf_approx_uv_img, which computes Methods 1 and 2 in one pass) on the tensor cores.

Metric: px.vis terms per second, one term = one (output pixel, averaged
visibility) pair (4 real flops of the complex contraction).  `value` is the
whole-job rate with the plan resident in HBM; `e2e` measures the same steps
through the public API from host buffers (plan upload, compute, read-back).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank evaluates its own cutout (positions shard with no
collective; weak scaling).  --impl reference times the FP64 CPU oracle (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import obsgen  # noqa: E402

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# DRAM bytes (read + write) per contraction launch from the ncu capture summarised in
# profiles/k_psf_tc_meerkat64_1h_128px.md, per visibility (traffic is proportional to
# K; the mean of the step's two launches: exact, fused uv + img), valid only for the
# kernel source it was taken on.
PROFILED_TRAFFIC = {"kernel_sha256_prefix": "86620fd584ed55e3",
                    "bytes_per_vis": ((232.290816e6 + 3.294976e6) + (348.522496e6 + 0.410368e6)) / 2 / 14515200,
                    "profile": "profiles/k_psf_tc_meerkat64_1h_128px.md"}


def profiled_traffic(nvis):
    import hashlib
    src = os.path.join(ROOT, "paper_2009_07010_gb300", "csrc", "k_tc.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != PROFILED_TRAFFIC["kernel_sha256_prefix"] or PROFILED_TRAFFIC["bytes_per_vis"] is None:
        return None
    return PROFILED_TRAFFIC["bytes_per_vis"] * nvis
WORKLOAD = "meerkat64_4h_16ch_128px_single_cutout"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            flat = {}

            def walk(x):
                if isinstance(x, dict):
                    for k, v in x.items():
                        if isinstance(v, (int, float)):
                            flat.setdefault(k, float(v))
                        else:
                            walk(v)
            walk(d)
            if "bf16_tflops" in flat:
                return flat, "measured"
        except Exception:
            pass
    return dict(FALLBACK_PEAKS), "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpus):
        self.gpus = set(gpus)
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if r[0].isdigit() and int(r[0]) in self.gpus]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def terms_per_step(K, batch, nmethods=3):
    return nmethods * K * batch.total_pixels()


def step_config(args, K, N):
    """The benchmark step's workload, the same object on both arms."""
    return {"workload": WORKLOAD if args.workload == "c2" else WORKLOAD + "_1h", "nvis": K, "npix": N,
            "positions_per_gpu": 1, "methods": ["exact", "uv", "img"], "precision": args.prec,
            "accumulate": "f32", "l2": "inputs exceed L2 (per-visibility tables 0.9 GB)",
            "seed_array": obsgen.ARRAY_SEED}


def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, on bounded samples of the same workload."""
    if rank != 0:
        return 0
    import oracle
    obs = obsgen.config2_obs() if args.workload == "c2" else obsgen.config2_obs(hours=1.0)
    batch = obsgen.config2_batch()
    K = obs.nvis()
    N = int(batch.npix[0])
    rng = np.random.default_rng(5)
    npx = 8
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))

    def step():
        sel = np.sort(rng.choice(N * N, npx, replace=False))
        for mid in (oracle.EXACT, oracle.UV, oracle.IMG):
            oracle.psf(obs, mid, batch, pix_sel=sel)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    terms = 3 * npx * K
    val = terms / dt
    line = {"metric": "smeared-PSF px.vis terms/sec (exact + uv + img)", "value": val, "unit": "terms/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": step_config(args, K, N),
            "cpu_baseline": {"value": val, "unit": "terms/s", "cores": cores, "kind": "oracle",
                             "host": f"{platform.machine()}, {os.cpu_count()} logical CPUs",
                             "sample": f"{npx} random pixels per method of the 128x128 cutout, all {K} visibilities"},
            "e2e": {"value": val, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def parity_check(psf):
    """Peak-normalised max error against the FP64 oracle on workload 1 (16 antennas,
    172 800 visibilities, 64 x 64 at (0.02, 0.02)) for every precision and method."""
    import oracle
    obs = obsgen.config1_obs()
    bg = obsgen.config1_batch()
    batch = psf.Batch.from_obsgen(bg)
    res = {}
    refs = {m: oracle.psf(obs, mid, bg) for m, mid in (("exact", 0), ("uv", 1), ("img", 2))}
    with psf.Plan(obs, prec="fp32") as plan:
        for prec in ("fp32", "tc_fp16", "tc_bf16", "tc_fp16x3", "tc_bf16x3"):
            plan.set_opts(prec=prec)
            for m in ("exact", "uv", "img"):
                got = plan.forward(m, batch).cpu().numpy().astype(np.float64)
                res[f"{prec}/{m}"] = float(np.max(np.abs(got - refs[m])) / np.max(np.abs(refs[m])))
            # the fused call of the benchmark step (both approximations in one pass)
            guv, gimg = plan.approx_uv_img(batch)
            for m, got in (("uv", guv), ("img", gimg)):
                got = got.cpu().numpy().astype(np.float64)
                res[f"{prec}/{m}_fused"] = float(np.max(np.abs(got - refs[m])) / np.max(np.abs(refs[m])))
        # Method 2 in the gridded form of Eq. 45 against the oracle's gridded form
        gref = oracle.psf_img_grid(obs, bg.lm, int(bg.npix[0]), bg.cell_rad).ravel()
        for prec in ("fp32", "tc_fp16"):
            plan.set_opts(prec=prec)
            got = plan.approx_img_grid(batch).cpu().numpy().astype(np.float64)
            res[f"{prec}/img_grid"] = float(np.max(np.abs(got - gref)) / np.max(np.abs(gref)))
    return {"workload": "16ant_1km_1h_4ch_64px", "metric": "max |P - P_oracle| / max |P_oracle|", "err_max": res,
            "tolerance": {"fp32": 1e-6, "tc_fp16": 1e-4, "tc_bf16": 1e-3, "tc_fp16x3": 2e-5, "tc_bf16x3": 2e-5,
                          "fp32/img_grid": 1e-5, "tc_fp16/img_grid": 3e-4}}


def measure_ladder(psf, plan, obs, batch_g, batch, outs, step, stream):
    """Precision ladder on the benchmark workload: per precision mode the rate of the same
    step (exact + uv + img) and the peak-normalised max error of the exact cutout against
    the FP64 oracle on sampled pixels (the centre and seven others), plus the error on
    workload 1 (full 64 x 64 cutouts, all methods) from `parity`.  The split modes execute
    three MMA passes per algorithmic product (executed tensor flops = 3 x algorithmic)."""
    import torch
    import oracle
    K = obs.nvis()
    N = int(batch_g.npix[0])
    c = N // 2
    sel = np.array([c * N + c, 0, N - 1, N * N - 1, c * N + c + 1, (c + 3) * N + c - 2, 31 * N + 100, 100 * N + 3])
    ref = oracle.psf(obs, oracle.EXACT, batch_g, pix_sel=sel)[sel]
    terms = terms_per_step(K, batch_g)
    res = {}
    prev = plan.prec
    for prec in ("fp32", "tc_fp16", "tc_bf16", "tc_fp16x3", "tc_bf16x3"):
        plan.set_opts(prec=prec)
        step(plan)
        torch.cuda.synchronize()
        nrep = 2 if prec == "fp32" else 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nrep):
            step(plan)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nrep
        got = outs[0].cpu().numpy().astype(np.float64)[sel]
        split = prec.endswith("x3")
        res[prec] = {"terms_per_s": terms / (ms * 1e-3), "ms_per_step": ms,
                     "err_max_exact_sampled": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
                     "mma_passes": 3 if split else (0 if prec == "fp32" else 1),
                     "executed_tensor_flops_per_term": 12.0 if split else (0.0 if prec == "fp32" else 4.0)}
    plan.set_opts(prec=prev)
    if plan.sync_status() != 0:
        raise RuntimeError("device-side wait timed out in the precision ladder")
    return {"workload": WORKLOAD, "step": "exact + uv + img", "pixels_sampled": len(sel), "modes": res}


def cpu_baseline_sample(obs, batch):
    import oracle
    K = obs.nvis()
    N = int(batch.npix[0])
    npx = 96
    sel = np.sort(np.random.default_rng(3).choice(N * N, npx, replace=False))
    t0 = time.perf_counter()
    oracle.psf(obs, oracle.EXACT, batch, pix_sel=sel)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": npx * K / dt, "unit": "terms/s", "cores": cores, "kind": "oracle",
            "host": f"{platform.machine()}, {os.cpu_count()} logical CPUs",
            "sample": f"exact method, {npx} random pixels of the 128x128 cutout over all {K} visibilities "
                      f"({dt:.1f} s incl. the oracle's binning and decorrelation pass)"}


def measure_batched(psf, prec, steps=2, which="c4", profile_range=False):
    """Batched form on the differentiation workload (c4: 256 positions, 64 x 64
    cutouts) or the batched-positions workload (c3: 4096 positions within 2 degrees,
    sizes drawn from 32..256); both on the baseline-dependent-averaging observation
    (13 710 280 visibilities): forward (exact + uv + img) and, for c4, the adjoint of
    the exact method."""
    import torch
    obs = obsgen.config3_obs()
    bg = obsgen.config4_batch() if which == "c4" else obsgen.config3_batch()
    batch = psf.Batch.from_obsgen(bg)
    K = obs.nvis()
    terms = 3 * K * bg.total_pixels()
    peaks, src = load_peaks()
    plan = psf.Plan(obs, prec=prec)
    out = torch.empty(batch.total(), dtype=torch.float32, device="cuda")
    # per method: whole-call time and the contraction kernel's own time (CUDA events
    # recorded by the library on the launching stream); algorithmic flops per term:
    # 4 for the complex weights of the exact method, 2 for the real weights of the
    # approximations (one multiply-add per pixel-visibility term)
    per, total_ms = {}, 0.0
    for m, fpt in (("exact", 4.0), ("uv", 2.0), ("img", 2.0)):
        plan.forward(m, batch, out=out)
        torch.cuda.synchronize()
        plan.profile_read()
        plan.profile_enable(True)
        if profile_range:   # the timed calls only, for ncu --profile-from-start off
            torch.cuda.profiler.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.forward(m, batch, out=out)
        e1.record()
        torch.cuda.synchronize()
        if profile_range:
            torch.cuda.profiler.stop()
        ms_m = e0.elapsed_time(e1) / steps
        kms, nkc, _ = plan.profile_read()
        plan.profile_enable(False)
        tf = fpt * K * bg.total_pixels() * steps / (kms * 1e-3) / 1e12
        per[m] = {"ms": ms_m, "terms_per_s": K * bg.total_pixels() / (ms_m * 1e-3),
                  "kernel_ms": kms / steps, "kernel_launches_per_call": nkc / steps,
                  "algorithmic_flops_per_term": fpt, "kernel_tflops": tf,
                  "kernel_frac_of_peak": tf / peaks["bf16_tflops"],
                  "kernel_frac_of_sustained_peak": tf / peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])}
        total_ms += ms_m
    ms = total_ms
    adj = None
    if which == "c4":   # adjoint of the exact method: tensor cores (the plan's precision) and FP32
        R = torch.randn(batch.total(), device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
        adj = {}
        for ap in (prec, "fp32"):
            plan.set_opts(prec=ap)
            plan.adjoint("exact", batch, R)
            torch.cuda.synchronize()
            plan.profile_read()
            plan.profile_enable(True)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            plan.adjoint("exact", batch, R)
            a1.record()
            torch.cuda.synchronize()
            kms, nkc, _ = plan.profile_read()
            plan.profile_enable(False)
            ams = a0.elapsed_time(a1)
            tc = ap in ("tc_fp16", "tc_bf16")
            adj[ap] = {"ms": ams, "terms_per_s": K * bg.total_pixels() / (ams * 1e-3),
                       "form": "tensor-core H (k_adj_tc) + FP32 decorrelation gradients (k_adj_fold)" if tc
                       else "FP32 CUDA cores (k_adjoint)"}
            if tc:   # 4 algorithmic flops per (position, pixel, visibility) of H
                adj[ap]["tc_kernel_ms"] = kms
                adj[ap]["tc_kernel_tflops"] = 4.0 * K * bg.total_pixels() / (kms * 1e-3) / 1e12
                adj[ap]["tc_kernel_frac_of_peak"] = adj[ap]["tc_kernel_tflops"] / peaks["bf16_tflops"]
        plan.set_opts(prec=prec)
        adj["speedup_tc_over_fp32"] = adj["fp32"]["ms"] / adj[prec]["ms"] if prec in adj and prec != "fp32" else None
    per_size = None
    if which == "c3":   # the exact method per cutout size (each size group alone)
        per_size = {}
        for N in sorted(set(int(x) for x in bg.npix)):
            sel = np.nonzero(bg.npix == N)[0]
            bN = psf.Batch(bg.lm[sel], N, bg.cell_rad)
            oN = torch.empty(bN.total(), dtype=torch.float32, device="cuda")
            plan.forward("exact", bN, out=oN)
            torch.cuda.synchronize()
            plan.profile_read()
            plan.profile_enable(True)
            plan.forward("exact", bN, out=oN)
            torch.cuda.synchronize()
            kms, nkc, _ = plan.profile_read()
            plan.profile_enable(False)
            tf = 4.0 * K * len(sel) * N * N / (kms * 1e-3) / 1e12
            per_size[f"{N}px"] = {"positions": int(len(sel)), "kernel_ms": kms, "kernel_tflops": tf,
                                  "kernel_frac_of_peak": tf / peaks["bf16_tflops"],
                                  "kernel_frac_of_sustained_peak":
                                      tf / peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])}
    st = plan.sync_status()
    plan.close()
    if st != 0:
        raise RuntimeError("device-side wait timed out in the batched measurement")
    name = "meerkat64_2h_8ch_bda_256pos_64px" if which == "c4" else "meerkat64_2h_8ch_bda_4096pos_32to256px"
    return {"workload": name, "nvis": K, "positions": bg.npos, "npix": sorted(set(int(x) for x in bg.npix)),
            "value": terms / (ms * 1e-3), "unit": "terms/s", "ms_per_step": ms, "methods": ["exact", "uv", "img"],
            "kernel": "k_psf_kr (tcgen05 batched contraction, persistent, work queue)", "per_method": per,
            "peak_source": src, "adjoint_exact": adj, "exact_per_cutout_size": per_size}


# Executed warp-instructions per position of k_img_grid (ncu smsp__inst_executed.sum of one
# launch / positions; profiles/k_img_grid_radial16384.md), for the kernel source below.
PROFILED_GRID = {"kernel_sha256_prefix": "f623518e68ad870c", "inst_per_position": {128: 214640640 / 4096, 64: 44775424 / 4096}}


def grid_inst_per_position(N):
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2009_07010_gb300", "csrc", "k_grid.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != PROFILED_GRID["kernel_sha256_prefix"]:
        return None
    return PROFILED_GRID["inst_per_position"].get(N)


def measure_img_grid(psf, plan, obs, clocks, npos=16384):
    """Method 2 in the gridded form of Eq. 45 on the benchmark observation: npos positions
    of the radial grid out to 3 degrees, cutouts of 128 and 64 pixels at 1.5".  The
    position-independent table (effective PSF, its DFT, per-cell means) is built by the
    first call and kept; the timed calls evaluate Algorithm 1 on the uv cells and one
    inverse FFT per position.  Also: per-position cost against the visibility-level
    Method 2 and the gridding error (max |grid - img| / max |img|) at sampled radii."""
    import torch
    peaks, src = load_peaks()
    lm = obsgen.config5_batch().lm[:npos]
    cell = obsgen.config2_batch().cell_rad
    sm_mhz = (clocks or {}).get("sm_mhz") or 1900.0
    res = {}
    for N in (128, 64):
        b = psf.Batch(lm, N, cell)
        out = torch.empty(b.total(), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.approx_img_grid(b, out=out)
        torch.cuda.synchronize()
        build_ms = (time.perf_counter() - t0) * 1e3
        plan.approx_img_grid(b, out=out)
        torch.cuda.synchronize()
        plan.profile_read()
        plan.profile_enable(True)
        nrep = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(nrep):
            plan.approx_img_grid(b, out=out)
        e1.record()
        torch.cuda.synchronize()
        kms, nkc, _ = plan.profile_read()
        plan.profile_enable(False)
        call_ms = e0.elapsed_time(e1) / nrep
        kms /= nrep
        gbs = 4.0 * N * N * npos / (kms * 1e-3) / 1e9
        ipp = grid_inst_per_position(N)
        roof = {"bound": "alu", "unit": "warp-instructions/s",
                "peak": 152 * 4 * sm_mhz * 1e6, "peak_source": "152 SMs x 4 issue slots x median SM clock",
                "inst_per_position": ipp,
                "achieved": None if ipp is None else ipp * npos / (kms * 1e-3),
                "hbm_output_gbs": gbs, "hbm_output_frac": gbs / peaks["hbm_gbs"], "hbm_peak_source": src}
        roof["frac"] = None if roof["achieved"] is None else roof["achieved"] / roof["peak"]
        res[f"{N}px"] = {"positions": npos, "table_build_ms": build_ms, "call_ms": call_ms, "kernel_ms": kms,
                         "positions_per_s": npos / (call_ms * 1e-3), "kernel_positions_per_s": npos / (kms * 1e-3),
                         "roofline": roof}
    # visibility-level Method 2 at sampled radii: cost per position and the gridding error
    sel = np.array([127, 127 * 4 + 42, 128 * 64 + 127 - 64, 128 * 127 + 5])
    sel = sel[sel < npos]
    N = 128
    bs = psf.Batch(lm[sel], N, cell)
    grid = plan.approx_img_grid(bs).cpu().numpy().astype(np.float64).reshape(len(sel), N, N)
    img_out = torch.empty(bs.total(), dtype=torch.float32, device="cuda")
    plan.approx_img(bs, out=img_out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.approx_img(bs, out=img_out)
    e1.record()
    torch.cuda.synchronize()
    img_ms = e0.elapsed_time(e1) / len(sel)
    img = img_out.cpu().numpy().astype(np.float64).reshape(len(sel), N, N)
    r_deg = np.degrees(np.arcsin(np.hypot(lm[sel, 0], lm[sel, 1])))
    gap = {f"{r:.3f}deg": float(np.max(np.abs(grid[k] - img[k])) / np.max(np.abs(img[k])))
           for k, r in enumerate(r_deg)}
    per_pos_grid = 1e3 / res["128px"]["kernel_positions_per_s"]
    return {"workload": "meerkat64_4h_16ch_radial16384pos_1p5arcsec", "nvis": obs.nvis(),
            "kernel": "k_img_grid (Algorithm 1 on uv cells + inverse FFT per position, FP32)",
            "sizes": res, "img_visibility_level_ms_per_128px_position": img_ms,
            "cost_ratio_img_over_grid_128px": img_ms / per_pos_grid,
            "gridding_error_vs_img_128px": gap}


def measure_clean(psf, plan, nl=2048, nsrc=200, npix=128, gain=0.1, iters=None):
    """Hogbom CLEAN with position-dependent PSFs (Algorithm 2) on the benchmark
    observation: an nl x nl image at 1.5" centred on (0.03, 0.03) holding nsrc seeded
    point sources (fluxes 1 / U^1.5 capped at 100, positions uniform), each shaped like the
    device's gridded PSF at its pixel (a synthetic dirty image, truncated to the 128 x 128
    window).  Per PSF method: iterations run and the mean time per iteration (argmax,
    PSF at the peak, subtraction); the gridded PSF keeps every step on the device."""
    import torch
    rng = np.random.default_rng(obsgen.SEED_BASE + 7)
    cell, centre, N = obsgen.config2_batch().cell_rad, (0.03, 0.03), npix
    xs = rng.integers(N // 2, nl - N // 2, nsrc)
    ys = rng.integers(N // 2, nl - N // 2, nsrc)
    fl = np.minimum(rng.uniform(0.0, 1.0, nsrc) ** -1.5, 100.0)
    lm = np.stack([centre[0] + (xs - nl // 2) * cell, centre[1] + (ys - nl // 2) * cell], axis=1)
    P = plan.approx_img_grid(psf.Batch(lm, N, cell)).view(nsrc, N, N)
    P = P / P[:, N // 2, N // 2].view(nsrc, 1, 1)
    dirty = torch.zeros((nl, nl), dtype=torch.float32, device="cuda")
    for k in range(nsrc):
        dirty[ys[k] - N // 2:ys[k] + N // 2, xs[k] - N // 2:xs[k] + N // 2] += float(fl[k]) * P[k]
    iters = iters or {"img_grid": 2000, "img": 8, "uv": 8, "exact": 4}
    out = {}
    for method, n in iters.items():
        r = dirty.clone()
        plan.clean(r.clone(), cell, N, method=method, gain=gain, max_iter=2, centre=centre)   # tables, warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, cp, _ = plan.clean(r, cell, N, method=method, gain=gain, threshold=0.0, max_iter=n, centre=centre)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[method] = {"iterations": int(len(cp)), "ms_per_iteration": dt * 1e3 / max(1, len(cp)),
                       "iterations_per_s": len(cp) / dt}
    if plan.sync_status() != 0:
        raise RuntimeError("device-side error in the CLEAN measurement")
    ref = out["exact"]["ms_per_iteration"]
    return {"workload": f"meerkat64_4h_16ch_clean_{nl}px_{nsrc}src_psf{N}", "image": [nl, nl],
            "psf_npix": N, "gain": gain, "sources": nsrc, "per_method": out,
            "speedup_over_exact_per_iteration": {m: ref / v["ms_per_iteration"] for m, v in out.items()}}


def measure_facets(psf, plan, nl=2048, nsrc=200, npix=128, gain=0.1, iters=3000):
    """Position-dependent PSFs against one PSF per facet (the faceting approach of
    Sect. 3.3, Eqs. 57-58) on the benchmark observation.  CLEAN: an nl x nl image at 1.5"
    centred 2 deg from the phase centre, nsrc seeded sources shaped like the gridded PSF at
    their pixels; cleaned with the PSF at each peak and with the one PSF at the image
    centre; residual max / rms over the brightest source after `iters` iterations, and time
    per iteration.  PSF cost: 16 facet-centre exact PSFs of 256^2 pixels against nsrc
    per-source exact PSFs of 128^2 and nsrc per-source gridded PSFs."""
    import torch
    rng = np.random.default_rng(obsgen.SEED_BASE + 8)
    cell, N = obsgen.config2_batch().cell_rad, npix
    centre = (float(np.sin(np.radians(2.0))), 0.0)
    xs = rng.integers(N // 2, nl - N // 2, nsrc)
    ys = rng.integers(N // 2, nl - N // 2, nsrc)
    fl = np.minimum(rng.uniform(0.0, 1.0, nsrc) ** -1.5, 100.0)
    lm = np.stack([centre[0] + (xs - nl // 2) * cell, centre[1] + (ys - nl // 2) * cell], axis=1)
    P = plan.approx_img_grid(psf.Batch(lm, N, cell)).view(nsrc, N, N)
    P = P / P[:, N // 2, N // 2].view(nsrc, 1, 1)
    dirty = torch.zeros((nl, nl), dtype=torch.float32, device="cuda")
    for k in range(nsrc):
        dirty[ys[k] - N // 2:ys[k] + N // 2, xs[k] - N // 2:xs[k] + N // 2] += float(fl[k]) * P[k]
    out = {}
    for name, facet in (("position_dependent", False), ("facet_psf", True)):
        r = dirty.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, cp, _ = plan.clean(r, cell, N, method="img_grid", gain=gain, threshold=0.0, max_iter=iters,
                                 centre=centre, facet_psf=facet)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"iterations": int(len(cp)), "ms_per_iteration": dt * 1e3 / max(1, len(cp)),
                     "residual_max_over_brightest": float(r.abs().max()) / float(fl.max()),
                     "residual_rms_over_brightest": float(r.pow(2).mean().sqrt()) / float(fl.max())}
    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3
    fl_lm = []
    for a in range(4):
        for b in range(4):
            fl_lm.append((centre[0] + (a - 1.5) * nl / 4 * cell, centre[1] + (b - 1.5) * nl / 4 * cell))
    fb = psf.Batch(np.array(fl_lm), 256, cell)
    sb = psf.Batch(lm, N, cell)
    cost = {"facet_exact_16x256px_ms": timed(lambda: plan.exact(fb)),
            "per_source_exact_ms": timed(lambda: plan.exact(sb)),
            "per_source_img_grid_ms": timed(lambda: plan.approx_img_grid(sb))}
    if plan.sync_status() != 0:
        raise RuntimeError("device-side error in the facet measurement")
    return {"workload": f"meerkat64_4h_16ch_facet_{nl}px_at_2deg_{nsrc}src", "clean_gridded_psf": out,
            "psf_cost": cost}


def measure_fwhm(psf, prec):
    """PSF size against distance from the phase centre as in the paper's FWHM figure: the
    64-antenna array at 1.4 GHz, 2 h of 1 s samples, 6 MHz of 50 kHz channels averaged
    10 s x 1 MHz (CF 10x20) or 20 s x 2 MHz (CF 20x40); exact smeared PSFs (64 x 64 at 1")
    at 0 to 4.5 deg, eight position angles each; FWHM along the radial and tangential
    directions (psf_fwhm), mean over the angles, in arcsec."""
    bg = obsgen.fig3_batch()
    batch = psf.Batch.from_obsgen(bg)
    r = np.degrees(np.arcsin(np.hypot(bg.lm[:, 0], bg.lm[:, 1])))
    radii = sorted(set(np.round(r, 6)))
    out = {}
    for cf in ("10x20", "20x40"):
        obs = obsgen.fig3_obs(cf)
        with psf.Plan(obs, prec=prec) as plan:
            w = plan.fwhm(batch, plan.exact(batch)).cpu().numpy() / (np.pi / 180 / 3600)
            if plan.sync_status() != 0:
                raise RuntimeError("device-side error in the FWHM measurement")
        out[f"CF_{cf}"] = {"nvis": obs.nvis(),
                           "radial_arcsec": {f"{d:.1f}deg": float(np.nanmean(w[np.abs(r - d) < 1e-6, 0])) for d in radii},
                           "tangential_arcsec": {f"{d:.1f}deg": float(np.nanmean(w[np.abs(r - d) < 1e-6, 1])) for d in radii}}
    return {"workload": "meerkat64_2h_1p4GHz_6MHz_fwhm", "method": "exact", "npix": 64, "cell_arcsec": 1.0,
            "positions": bg.npos, **out}


def measure_c5(psf, prec, nrad=128, nang=128, ref="fp16"):
    """Approximations against the exact smeared PSF on the approximation workload (64-antenna
    8 km array, 4 h of 1 s samples averaged 8:1, 256 channels of 3.34375 MHz averaged 4:1 ->
    232 243 200 visibilities; 64 x 64 cutouts at 1.5" on the radial grid of nrad radii to 3
    deg x nang position angles, 16 384 positions).  Every map is computed on the GPU in one
    batched call per method: the exact PSF (FP16 operands, FP32 accumulation; the map
    reference unless ref="bf16x3", which evaluates the exact PSF of every position in the
    split mode BF16X3 as the reference, about 14 minutes), Method 1 (uv), Method 2 (img),
    Method 2 in the gridded form of Eq. 45
    (img_grid; its position-independent table is built by a first call outside the timing)
    and the effective PSF (the phase-centre cutout, scaled to each position's peak).  Per
    radius: the largest over the angles of the peak-normalised max and RMS error, and the
    max in dB (10 log10 |P - P_ref| of the normalised PSFs).  The reference's own error is
    measured at 256 positions (every radius, 2 angles) against the exact PSF in the split
    mode BF16X3 (per-cutout form, about 3e-6); the approximations are also compared with
    that finer reference there.  tests/test_c5_gpu.py ties these paths to the FP64 oracle.
    Cost ratios t_exact / t_approx from the same engine."""
    import torch
    obs = obsgen.config5_obs()
    bg = obsgen.config5_batch(nrad=nrad, nang=nang)
    batch = psf.Batch.from_obsgen(bg)
    K = obs.nvis()
    N = int(bg.npix[0])
    t0 = time.perf_counter()
    plan = psf.Plan(obs, prec=prec)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    outs, ms, kms, nlaunch = {}, {}, {}, {}
    warm = psf.Batch(bg.lm[:256], N, bg.cell_rad)
    for m in ("exact", "uv", "img", "img_grid"):
        out = torch.empty(batch.total(), dtype=torch.float32, device="cuda")
        plan.forward(m, warm, out=out)                   # tuning, tables and warm-up
        torch.cuda.synchronize()
        plan.profile_read()
        plan.profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.forward(m, batch, out=out)
        e1.record()
        torch.cuda.synchronize()
        kms[m], nlaunch[m], _ = plan.profile_read()
        plan.profile_enable(False)
        ms[m] = e0.elapsed_time(e1)
        outs[m] = out.view(nrad, nang, N * N)
    eff = plan.exact(psf.Batch(np.zeros((1, 2)), N, bg.cell_rad)).view(1, 1, N * N)
    ref_ms = None
    if ref == "bf16x3":
        # the map reference: the exact PSF of every position in the split mode BF16X3
        # (per-cutout form, ~3e-6 of the peak), in chunks of 1024 positions
        plan.set_opts(prec="tc_bf16x3")
        ex = torch.empty(nrad * nang, N * N, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for c0 in range(0, nrad * nang, 1024):
            lmc = bg.lm[c0:c0 + 1024]
            plan.exact(psf.Batch(lmc, N, bg.cell_rad), out=ex[c0:c0 + len(lmc)].view(-1))
        e1.record()
        torch.cuda.synchronize()
        ref_ms = e0.elapsed_time(e1)
        plan.set_opts(prec=prec)
        ex = ex.view(nrad, nang, N * N)
    else:
        ex = outs["exact"]
    peak = ex.abs().amax(dim=2)                                          # [nrad, nang]
    outs["effective"] = eff / eff.abs().max() * peak.unsqueeze(-1)
    radius = 3.0 * (np.arange(nrad) + 1) / nrad
    picks = sorted(set([0, 1, 3, 7, 11] + list(range(15, nrad, 16)) + [nrad - 1]))
    key = [f"{radius[i]:.4f}deg" for i in range(nrad)]
    res = {}
    for m in ("uv", "img", "img_grid", "effective") + (("exact",) if ref == "bf16x3" else ()):
        d = outs[m] - ex
        emax = (d.abs().amax(dim=2) / peak).amax(dim=1).cpu().numpy()                 # worst angle per radius
        erms = ((d * d).mean(dim=2).sqrt() / peak).amax(dim=1).cpu().numpy()
        res[m] = {"err_max": {key[i]: float(emax[i]) for i in picks},
                  "err_rms": {key[i]: float(erms[i]) for i in picks},
                  "err_max_dB": {key[i]: round(float(10 * np.log10(max(emax[i], 1e-30))), 2) for i in picks},
                  "worst": float(emax.max()), "worst_dB": round(float(10 * np.log10(emax.max())), 2)}
        del d
    # finer reference: the exact PSF in BF16X3 at every radius, angles 0 and pi
    ai = np.repeat(np.arange(nrad), 2)
    bi = np.tile(np.array([0, nang // 2]), nrad)
    lm_f = bg.lm[ai * nang + bi]
    plan.set_opts(prec="tc_bf16x3")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fine = plan.exact(psf.Batch(lm_f, N, bg.cell_rad)).view(len(lm_f), N * N)
    e1.record()
    torch.cuda.synchronize()
    fine_ms = e0.elapsed_time(e1)
    plan.set_opts(prec=prec)
    pk = fine.abs().amax(dim=1)
    fine_res = {}
    for m in ("exact", "uv", "img", "img_grid"):
        e = ((outs[m][ai, bi] - fine).abs().amax(dim=1) / pk).view(nrad, 2).amax(dim=1).cpu().numpy()
        fine_res[m] = {key[i]: float(e[i]) for i in picks}
        fine_res[m]["worst"] = float(e.max())
    st = plan.sync_status()
    plan.close()
    if st != 0:
        raise RuntimeError("device-side wait timed out in the approximation workload")
    terms = K * bg.total_pixels()
    peaks, _ = load_peaks()
    # algorithmic flops per term: 4 with the complex weights of the exact method, 2 with real weights
    tfl = {m: (4.0 if m == "exact" else 2.0) * terms / (kms[m] * 1e-3) / 1e12 for m in ("exact", "uv", "img")}
    uvm, imm = res["uv"]["err_max"], res["img"]["err_max"]
    return {"workload": "meerkat64_8km_4h_256ch_avg4_radial16384_64px", "nvis": K, "positions": bg.npos,
            "grid": f"{nrad} radii 3 deg (a+1)/{nrad} x {nang} position angles, 64 px at 1.5 arcsec",
            "precision": prec, "plan_build_s": plan_s,
            "ms": ms, "terms_per_s": {m: terms / (ms[m] * 1e-3) for m in ("exact", "uv", "img")},
            "contraction": {m: {"kernel": "k_psf_kr", "ms": kms[m], "launches": int(nlaunch[m]),
                                "tflops": tfl[m], "frac_of_peak": tfl[m] / peaks["bf16_tflops"],
                                "frac_of_sustained_peak": tfl[m] / peaks.get("bf16_tflops_sustained",
                                                                              peaks["bf16_tflops"])}
                            for m in ("exact", "uv", "img")},
            "cost_ratio_exact_over": {m: ms["exact"] / ms[m] for m in ("uv", "img", "img_grid")},
            "map_reference": ("exact PSF in BF16X3 for every position (per-cutout form), %.1f s" % (ref_ms / 1e3)
                              if ref == "bf16x3" else "exact PSF in the batched %s form" % prec),
            "err_vs_exact": {"uv_plane": res["uv"], "image_plane": res["img"], "image_plane_gridded": res["img_grid"],
                             "effective_psf_scaled_to_peak": res["effective"],
                             **({"exact_batched_" + prec: res["exact"]} if ref == "bf16x3" else {})},
            "finer_reference": {"what": "exact PSF in BF16X3 (per-cutout form), every radius x 2 angles",
                                "positions": int(len(lm_f)), "ms": fine_ms,
                                "err_max_vs_bf16x3_exact": fine_res},
            "uv_not_worse_than_img_at_picked_radii": bool(all(uvm[k] <= imm[k] for k in uvm))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tc_fp16", choices=["tc_fp16", "tc_bf16", "fp32"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-grid", action="store_true")
    ap.add_argument("--no-clean", action="store_true")
    ap.add_argument("--no-fwhm", action="store_true")
    ap.add_argument("--no-facets", action="store_true")
    ap.add_argument("--no-ladder", action="store_true")
    ap.add_argument("--no-c5", action="store_true")
    ap.add_argument("--profile-range", action="store_true",
                    help="c3 / c4: bracket the timed calls with cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    ap.add_argument("--c5-ref", default="fp16", choices=["fp16", "bf16x3"],
                    help="map reference of the approximation workload: the batched exact PSF in the plan's "
                         "precision (default) or the BF16X3 exact PSF of all 16 384 positions (about 15 min)")
    ap.add_argument("--grid-positions", type=int, default=16384,
                    help="positions of the gridded-form measurement (radial grid out to 3 deg)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c2_1h", "c3", "c4", "c5", "grid", "clean", "facets"],
                    help="c2: the 4 h MeerKAT-shaped cutout; c2_1h: the same array and cutout over 1 h "
                         "(a quarter of the visibilities, for profiler captures); c4: only the batched "
                         "256 x 64^2 measurement (profiler captures of the batched kernel); grid: only "
                         "the gridded Method 2 measurement on the benchmark observation; clean: only the "
                         "CLEAN (Algorithm 2) measurement")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload in ("c3", "c4"):
        import torch
        import paper_2009_07010_gb300 as psf
        psf.build_library()
        torch.cuda.set_device(local)
        print(json.dumps(measure_batched(psf, args.prec, steps=args.steps, which=args.workload,
                                         profile_range=args.profile_range)), flush=True)
        return 0
    if args.workload == "clean":
        import torch
        import paper_2009_07010_gb300 as psf
        psf.build_library()
        torch.cuda.set_device(local)
        with psf.Plan(obsgen.config2_obs(), prec=args.prec) as plan:
            res = measure_clean(psf, plan)
        print(json.dumps(res), flush=True)
        return 0
    if args.workload == "facets":
        import torch
        import paper_2009_07010_gb300 as psf
        psf.build_library()
        torch.cuda.set_device(local)
        with psf.Plan(obsgen.config2_obs(), prec=args.prec) as plan:
            res = measure_facets(psf, plan)
        print(json.dumps(res), flush=True)
        return 0
    if args.workload == "grid":
        import torch
        import paper_2009_07010_gb300 as psf
        psf.build_library()
        torch.cuda.set_device(local)
        obs = obsgen.config2_obs()
        with psf.Plan(obs, prec=args.prec) as plan:
            res = measure_img_grid(psf, plan, obs, None, npos=args.grid_positions)
            if plan.sync_status() != 0:
                raise RuntimeError("device-side error in the gridded-form measurement")
        print(json.dumps(res), flush=True)
        return 0
    if args.workload == "c5":
        import torch
        import paper_2009_07010_gb300 as psf
        psf.build_library()
        torch.cuda.set_device(local)
        print(json.dumps(measure_c5(psf, args.prec, ref=args.c5_ref)), flush=True)
        return 0

    import torch
    import paper_2009_07010_gb300 as psf
    psf.build_library()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    obs = obsgen.config2_obs() if args.workload == "c2" else obsgen.config2_obs(hours=1.0)
    batch_g = obsgen.config2_batch()
    batch = psf.Batch.from_obsgen(batch_g)
    K = obs.nvis()
    terms = terms_per_step(K, batch_g)
    stream = torch.cuda.current_stream()

    plan = psf.Plan(obs, prec=args.prec)
    outs = [torch.empty(batch.total(), dtype=torch.float32, device="cuda") for _ in range(3)]

    def step(p):
        p.exact(batch, out=outs[0])
        p.approx_uv_img(batch, out_uv=outs[1], out_img=outs[2])

    for _ in range(args.warmup):
        step(plan)
    torch.cuda.synchronize()
    if plan.sync_status() != 0:
        raise RuntimeError("device-side wait timed out during warm-up")
    plan.profile_read()
    plan.profile_enable(True)

    sampler = ClockSampler(range(world) if world > 1 else [local]) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(plan)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1) / args.steps
    kms, nkc, nk = plan.profile_read()
    plan.profile_enable(False)
    if plan.sync_status() != 0:
        raise RuntimeError("device-side wait timed out in the timed region")
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * terms / (ms * 1e-3)

    # FP32 CUDA-core form of the same step (comparator)
    fp32 = None
    if not args.no_fp32 and args.prec != "fp32":
        plan.set_opts(prec="fp32")
        step(plan)
        torch.cuda.synchronize()
        plan.profile_read()
        plan.profile_enable(True)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        nrep = 2
        for _ in range(nrep):
            step(plan)
        f1.record(stream)
        torch.cuda.synchronize()
        fkms, _, _ = plan.profile_read()
        plan.profile_enable(False)
        fms = f0.elapsed_time(f1) / nrep
        fkms /= nrep
        # roofline of k_psf_fp32: 4 flops (two FMAs) per term against the measured FP32
        # FMA rate (the better of scalar and packed-pair FMAs)
        peak_s, peak_p = psf.fma_rate(False), psf.fma_rate(True)
        fach = 4.0 * terms / (fkms * 1e-3)
        fp32 = {"value": terms / (fms * 1e-3), "unit": "terms/s", "ms_per_step": fms,
                "speedup_tc_over_fp32": fms / ms,
                "roofline": {"bound": "alu", "kernel": "k_psf_fp32", "kernel_ms_per_step": fkms,
                             "achieved": fach, "unit": "FLOP/s", "peak": max(peak_s, peak_p),
                             "peak_source": "measured FP32 FMA rate (psf_selftest_fma_rate)",
                             "fma_rate_scalar": peak_s, "fma_rate_packed_pairs": peak_p,
                             "frac": fach / max(peak_s, peak_p), "flops_per_term": 4}}
        plan.set_opts(prec=args.prec)

    # end to end through the public API from host buffers
    e2e = None
    if not args.no_e2e:
        nrep = max(1, min(3, args.steps))
        h2d = (obs.uvw_m.nbytes + obs.time_s.nbytes + obs.freq_hz.nbytes + obs.chan_width_hz.nbytes
               + obs.tavg.nbytes + batch.lm.nbytes + batch.npix.nbytes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t_plan = 0.0
        for _ in range(nrep):
            tp = time.perf_counter()
            with psf.Plan(obs, prec=args.prec) as p2:
                torch.cuda.synchronize()
                t_plan += time.perf_counter() - tp
                step(p2)
                host = [o.cpu() for o in outs]
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / nrep
        t_plan /= nrep
        if dist:
            t = torch.tensor([dt], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dt = float(t.item())
        e2e = {"value": world * terms / dt, "unit": "terms/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(sum(h.numel() * 4 for h in host)), "ms_per_step": dt * 1e3,
               "plan_build_ms": t_plan * 1e3, "compute_and_readback_ms": (dt - t_plan) * 1e3}

    ladder = None if args.no_ladder or rank != 0 else measure_ladder(psf, plan, obs, batch_g, batch, outs, step,
                                                                     stream)
    img_grid = None if args.no_grid or rank != 0 else measure_img_grid(psf, plan, obs, clocks,
                                                                       npos=args.grid_positions)
    clean = None if args.no_clean or rank != 0 else measure_clean(psf, plan)
    fwhm = None if args.no_fwhm or rank != 0 else measure_fwhm(psf, args.prec)
    facets = None if args.no_facets or rank != 0 else measure_facets(psf, plan)
    # side measurements on rank 0 only; the approximation workload (minutes) with one GPU only
    batched = None if args.no_batched or rank != 0 else measure_batched(psf, args.prec)
    batched_c3 = None if args.no_batched or rank != 0 else measure_batched(psf, args.prec, steps=1, which="c3")
    c5 = None if args.no_c5 or rank != 0 or world > 1 else measure_c5(psf, args.prec)
    parity = None if (args.no_cpu_baseline or rank != 0) else parity_check(psf)

    if rank == 0:
        peaks, src = load_peaks()
        peak = peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"])
        launches = max(nkc, 1)
        avg_ms = kms / launches
        # algorithmic flops of all contraction launches in the timed region: three
        # methods per step, 4 flops per px.vis term (the exact launch does one method,
        # the fused launch two)
        flops_total = 3 * 4.0 * K * batch.total() * args.steps
        flops_launch = flops_total / launches
        achieved = flops_total / (kms * 1e-3) / 1e12
        traffic = profiled_traffic(K)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                "traffic_source": PROFILED_TRAFFIC["profile"] if traffic else None, "peak_source": src,
                "kernel": "k_psf_tc (tcgen05 contraction: exact launch + fused uv/img launch per step)",
                "avg_launch_ms": avg_ms, "launches_per_step": launches / args.steps,
                "algorithmic_flops_per_launch": flops_launch}
        cpu = None if args.no_cpu_baseline else cpu_baseline_sample(obs, batch_g)
        line = {"metric": "smeared-PSF px.vis terms/sec (exact + uv + img)", "value": value, "unit": "terms/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"tc_fp16": "f16", "tc_bf16": "bf16", "fp32": "f32", "tc_fp16x3": "f16x3",
                          "tc_bf16x3": "bf16x3"}[args.prec], "data": "synthetic",
                "config": step_config(args, K, int(batch_g.npix[0])),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp32_plain": fp32, "precision_ladder": ladder,
                "batched": batched, "batched_c3": batched_c3, "c5": c5, "img_grid": img_grid, "clean": clean, "fwhm": fwhm, "facets": facets,
                "parity": parity,
                "gpu_launches": int(nk), "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
