#!/usr/bin/env python3
"""Aerial-image throughput on 2048^2 clips (K=24, 3 focus planes) plus resist.

Workload (the headline configuration): 64 clips of 2048 x 2048 at 8 nm,
193 nm / NA 1.35 immersion (n = 1.44), quadrupole source (poles at sigma 0.8,
radius 0.1) sampled on a 41 x 41 grid (52 points), K = 24 SOCS kernels per
focus plane at defocus -50/0/+50 nm, Manhattan masks of seeded random
rectangles (sides 40-120 nm) at 35 % density, Gaussian resist sigma 10 nm,
threshold 0.3.  Inputs are synthetic (the paper's layouts are not available).

One step = mask spectrum + band multiply + inverse transforms with fused
lam |E|^2 accumulation (every clip, every focus plane, every kernel) + resist
blur and threshold, over the whole batch, inputs resident in HBM.  `value`
is Mpx/s = clips * N^2 / step time (a clip's pixel counts once and includes
all K kernels and all focus planes) for the fastest path whose error bound
is 1e-5 (the FP32 FFT path on the coarse grid).  The same line carries the
plain FP32 FFT path and the split fp16 tensor-core path, timed the same way.
`e2e` is the headline path through the host-buffer C-ABI call: masks copied in
from pinned memory, printed resist bytes copied back.

Other workloads (one JSON line each): --workload ilt (16 clips of 1024^2,
annular, K=16, 5 focus planes, one ILT gradient step per step) and
--workload serve (Poisson stream of mixed requests through litho_serve).

Multi-GPU: clips are independent, so each rank images its own batch (weak
scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

N, PIXEL, K = 2048, 8.0, 24
FOCUS = [-50.0, 0.0, 50.0]
SIGMA_NM, THRESH = 10.0, 0.3
OPTICS = dict(wavelength_nm=193.0, na=1.35, n_medium=1.44, kind="quadrupole", src_grid=41, pole_sigma=0.8,
              pole_radius=0.1)
WORKLOAD = "socs-aerial+resist 2048x2048@8nm quadrupole41 K=24 focus(-50,0,50)"
METRIC = "aerial-image Mpx/s (2048² clips, K=24) vs plain FFT path at ≤1e-5 err; p99 ms"
HEADLINE = "fft32/coarse"
COMPARE = ["fft32", "fp16x3/coarse"]   # the plain FFT path, the split tensor-core path
ERROR_BOUND = {"fft32": 1e-5, "fft32/coarse": 1e-5, "fp16x3": 1e-5, "fp16x3/coarse": 1e-5, "bf16x3": 1e-5,
               "bf16x3/coarse": 1e-5, "fp16": 2e-3, "fp16/coarse": 2e-3, "bf16": 4e-3}

FP32_LANES_PER_SM = 128


def sm_count() -> int:
    """Streaming multiprocessors of the device in use (152 on a GB300)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        pass
    return 152


def sm_max_mhz() -> float:
    p, _ = _peaks()
    return float(p.get("sm_max_mhz") or 2070.0)


def alu_peak_tflops() -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 flops (FMA) x maximum SM clock."""
    return sm_count() * FP32_LANES_PER_SM * 2 * sm_max_mhz() * 1e6 / 1e12


def alu_peak_source() -> str:
    return f"derived: {sm_count()} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x {sm_max_mhz():.0f} MHz"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
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
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def clip_seeds(rank: int, clips: int, base: int = 1234):
    """Seeds of the clips rank `rank` images: disjoint blocks per rank."""
    return [base + rank * clips + i for i in range(clips)]


def whole_job_rate(units_per_rank: float, world: int, rank_seconds: list[float]) -> float:
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / max(rank_seconds)


# ---- algorithmic work models (per step) ------------------------------------------------------------

def fft_group(clips: int, n_focus: int, k: int, ne: int, crop: int) -> int:
    """Clips per FP32 stage launch: the library's rule (stage-1 fields of a group within
    2 GiB, at most 64 clips, groups of equal size)."""
    per_clip = n_focus * k * ne * crop * 8
    cap = max(1, min(64, (2 << 30) // per_clip))
    groups = -(-clips // cap)
    return -(-clips // groups)


def stage_models(prec: str, clips: int, n: int, crop: int, n_focus: int, k_eff: int, nc: int, peaks,
                 resist_taps: int = 11, k_alloc: int = K) -> dict:
    """stage -> (flops per step, algorithmic DRAM bytes per step).

    Bytes count what the stage must move at least: its inputs read once and its
    outputs written once (intermediates of the library's own making that a stage
    writes and reads back, such as the row spectra of a 2D transform, are not
    counted); the kernels Phi count once per launch, since a launch's clips share
    them.  Flops count 5 m log2 m per m-point complex transform and 6 per complex
    multiply-add of the band multiply."""
    coarse = prec.endswith("/coarse") and nc > 0
    ne = nc if coarse else n
    fk = n_focus * k_eff
    fft = lambda m: 5.0 * m * math.log2(m)  # noqa: E731  (radix-2 operation count of an m-point transform)
    base = prec.split("/")[0]
    split = base in ("fp16x3", "bf16x3")
    planes = clips * n_focus
    group = fft_group(clips, n_focus, k_alloc, ne, crop) if base == "fft32" else min(clips, 4)
    launches = -(-clips // group)
    phi_bytes = n_focus * k_alloc * crop * crop * 8.0
    t1_bytes = clips * fk * ne * crop * 8.0
    m = {
        "mask_spectrum": (clips * (n / 2 * fft(n) + crop * fft(n)), clips * (n * n * 4.0 + crop * crop * 8.0)),
        "stage1_fft": (clips * fk * (crop * fft(ne) + 6.0 * crop * crop),
                       launches * phi_bytes + clips * crop * crop * 8.0 + t1_bytes),
        "stage2_fft": (clips * fk * ne * (fft(ne) + 4.0 * ne), t1_bytes + planes * ne * ne * 4.0),
        "stage1_gemm_operands": (clips * fk * (crop * fft(ne) + 6.0 * crop * crop),
                                 launches * phi_bytes + clips * crop * crop * 8.0 +
                                 clips * fk * ne * crop * (12.0 if split else 4.0)),
        # executed tensor-core flops: 2 M N K per real product; the split modes take Gauss's three
        # real products per complex multiply-add (6 M N K), each as three 16-bit products; the plain
        # modes take four (8 M N K)
        "stage2_gemm": (clips * fk * ne * ne * crop * (6.0 * 3 if split else 8.0),
                        clips * fk * ne * crop * (12.0 if split else 4.0) + planes * ne * ne * 4.0),
        "resist": (planes * n * n * 4.0 * resist_taps, planes * n * n * 9.0),
    }
    if coarse:
        c2 = 2 * crop
        # on a 1024-point grid the warp-per-row stage 2 also takes each image row forward and writes
        # its band spectrum (planes x ne x c2 complex) in place of the coarse image
        rows_in_stage2 = base == "fft32" and ne == 1024 and crop <= 512
        row_fft = planes * ne / 2 * fft(ne)  # two real rows per complex transform
        up_in = planes * ne * c2 * 8.0 if rows_in_stage2 else planes * ne * ne * 4.0
        up = planes * (c2 * fft(ne) + c2 * fft(n) + n * fft(n)) + (0.0 if rows_in_stage2 else row_fft)
        if rows_in_stage2:
            f2, b2 = m["stage2_fft"]
            m["stage2_fft"] = (f2 + planes * ne * fft(ne), b2 - planes * ne * ne * 4.0 + up_in)
        m["upsample"] = (up, up_in + planes * n * n * 4.0)
        m["upsample_resist"] = (up + planes * c2 * c2 * 6.0, up_in + planes * n * n * 9.0)
    return m


def ilt_models(clips: int, n: int, ne: int, crop: int, n_focus: int, k: int, coarse: bool, group: int,
               resist_taps: int = 11) -> dict:
    """stage -> (flops per step, algorithmic DRAM bytes per step) of litho_ilt_grad, counted as in
    stage_models (5 m log2 m per m-point transform): the forward pass (mask spectrum, stage 1 and 2
    per kernel, interpolation with the blur channel or the direct blur, resist gradient) and the
    backward pass (low-pass of the blurred dL/dI or the direct blur, adjoint rows: inverse and
    forward transform per kernel and row, adjoint columns, the band-to-full gradient).  Bytes:
    theta, target and the kernels Phi (once per clip group) in, the gradient out."""
    fft = lambda m: 5.0 * m * math.log2(m)  # noqa: E731
    c2 = 2 * crop
    fwd_plane = k * (crop * fft(ne) + 6.0 * crop * crop + ne * (fft(ne) + 4.0 * ne)) + n * n * 10.0
    bwd_plane = k * (ne * (2 * fft(ne) + 8.0 * ne) + crop * fft(ne) + 6.0 * crop * crop)
    if coarse:
        fwd_plane += ne / 2 * fft(ne) + c2 * fft(ne) + c2 * fft(n) + n * fft(n) + 6.0 * c2 * c2
        bwd_plane += n / 2 * fft(n) + c2 * fft(n) + c2 * fft(ne) + ne * fft(ne)
    else:
        fwd_plane += n * n * 4.0 * resist_taps
        bwd_plane += n * n * 4.0 * resist_taps
    fwd = clips * (n / 2 * fft(n) + crop * fft(n) + n_focus * fwd_plane)
    bwd = clips * (crop * fft(n) + n * fft(n) + n_focus * bwd_plane)
    groups = -(-clips // group)
    phi_bytes = groups * n_focus * k * crop * crop * 8.0
    return {"ilt_forward": (fwd, clips * n * n * 8.0 + phi_bytes), "ilt_backward": (bwd, clips * n * n * 4.0)}


def ai_models(clips: int, n: int, ne: int, crop: int, k: int, coarse: bool, round_taps: int) -> dict:
    """stage -> (flops per step, algorithmic DRAM bytes per step) of the AI-input step
    (litho_ai_inputs + litho_print_images), counted as in stage_models: ilt_forward = the image
    channel (mask spectrum, stage 1 and 2 per kernel, interpolation), ilt_backward = the adjoint of
    ones (its closed form N^2 sum_k lam_k |Phi_k|^2 mhat, then the band-to-full gradient), ilt_reduce = the two
    channel normalisations (read, then read and write), resist = the print images (blur of the
    targets, two thresholds, the L1 count).  Bytes: targets in, the three channels out."""
    fft = lambda m: 5.0 * m * math.log2(m)  # noqa: E731
    c2 = 2 * crop
    fwd = clips * (n / 2 * fft(n) + crop * fft(n) +
                   k * (crop * fft(ne) + 6.0 * crop * crop + ne * (fft(ne) + 4.0 * ne)))
    if coarse:
        # the coarse image's row transforms: one per row inside the 1024-point stage 2, else two
        # real rows per transform
        rows = ne * fft(ne) if (ne == 1024 and crop <= 512) else ne / 2 * fft(ne)
        fwd += clips * (rows + c2 * fft(ne) + c2 * fft(n) + n * fft(n))
    bwd = clips * (k * 4.0 * crop * crop + 4.0 * crop * crop + crop * fft(n) + n * fft(n))
    px = clips * n * n
    return {"ilt_forward": (fwd, px * 4.0 + px * 8.0), "ilt_backward": (bwd, px * 4.0),
            "ilt_reduce": (px * 2 * 3.0, px * 2 * 12.0),
            "resist": (px * 4.0 * round_taps, px * (4.0 + 4.0 + 4.0 + 1.0 + 1.0))}


# Sources whose kernels each stage runs: a DRAM-traffic figure taken with ncu
# holds only while they are unchanged.
STAGE_SOURCES = {
    "stage1_fft": ["stage1.cuh", "fft.cu", "fft_common.cuh"],
    "stage2_fft": ["fft.cu", "fft_common.cuh", "stage2_w32.cu"],
    "upsample_resist": ["stage1.cuh", "fft.cu", "fft_common.cuh", "interp.cu"],
}


def sources_digest(stage: str):
    import hashlib
    files = STAGE_SOURCES.get(stage)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2602_15036_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(stage: str, prec: str, clips: int, launches_per_step: float):
    """DRAM bytes per launch of `stage` from the committed ncu summary
    (profiles/dram_traffic.json), if it was taken on the same sources with the
    same clips per launch; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            entries = json.load(f)
    except Exception:
        return None, None
    per_launch = clips / launches_per_step if launches_per_step else None
    for e in entries:
        if (e.get("stage") == stage and e.get("precision") == prec and e.get("sources") == sources_digest(stage)
                and per_launch and abs(e.get("clips_per_launch", -1) - per_launch) < 1e-9):
            return e["bytes_per_launch"], e.get("summary")
    return None, None


def rooflines(prof: dict, steps: int, models: dict, peaks) -> dict:
    """Per stage: the binding resource (the larger of flops / ALU peak and bytes / HBM
    peak) with achieved = work per step / measured time per step, plus the other one."""
    out = {}
    hbm = peaks["hbm_gbs"]
    for stage, (ms, launches) in prof.items():
        if stage not in models:
            continue
        flops, nbytes = models[stage]
        sec = ms / steps * 1e-3
        tensor = stage == "stage2_gemm"
        fpeak = peaks["bf16_tflops_sustained"] if tensor else alu_peak_tflops()
        alu = {"bound": "tensor" if tensor else "alu", "achieved": flops / sec / 1e12, "peak": fpeak,
               "unit": "TFLOP/s"}
        mem = {"bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": hbm, "unit": "GB/s"}
        for d in (alu, mem):
            d["frac"] = d["achieved"] / d["peak"]
        t_alu, t_mem = flops / (fpeak * 1e12), nbytes / (hbm * 1e9)
        main, other = (mem, alu) if t_mem >= t_alu else (alu, mem)
        lps = launches / steps
        out[stage] = dict(main, other=other, algorithmic_work_per_step={"flops": flops, "bytes": nbytes},
                          algorithmic_bytes_per_launch=nbytes / lps if lps else None,
                          ms_per_step=ms / steps, launches_per_step=lps)
    return out


# ---- the oracle as the CPU baseline / reference arm --------------------------------------------------

def _oracle_sample(seed: int, focus_planes):
    """Oracle (FP64 numpy, one thread) on one clip for the given focus planes:
    SOCS image from oracle-built kernels, resist blur and threshold.  Returns
    seconds spent in the imaging + resist (kernel build excluded: it is set-up)."""
    from oracle import imaging as OI
    from oracle import optics as OO
    from oracle import resist as ORR
    oo = OO.Optics(193.0, 1.35, 1.44, OO.QUADRUPOLE, 41, pole_sigma=0.8, pole_radius=0.1)
    kern = [OO.socs_kernels(oo, N, PIXEL, z, K)[:2] for z in focus_planes]
    m = synth.manhattan_mask(N, seed=seed).astype(np.float64)
    t0 = time.perf_counter()
    for lam, phi in kern:
        img = OI.socs_image(m, lam, phi)
        ib = ORR.blur(img, SIGMA_NM, PIXEL)
        ORR.printed(ib, THRESH)
    return time.perf_counter() - t0


def host_facts() -> dict:
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


_SHARED = {}


def _oracle_worker_init(names, shapes):
    """Maps the parent's shared arrays (mask, lambdas, kernels, output slots) in a worker."""
    from multiprocessing import shared_memory
    for key, name in names.items():
        shm = shared_memory.SharedMemory(name=name)
        dt = np.float64 if key in ("m", "lam", "out") else np.complex128
        _SHARED[key] = (shm, np.ndarray(shapes[key], dtype=dt, buffer=shm.buf))


def _oracle_partial(task):
    """One worker's share of the oracle's SOCS sum: the oracle's own socs_image over kernels
    k0..k1 of focus plane f, written to output slot `slot`."""
    from oracle import imaging as OI
    f, k0, k1, slot = task
    m, lam, phi, out = (_SHARED[k][1] for k in ("m", "lam", "phi", "out"))
    out[slot] = OI.socs_image(m, lam[f, k0:k1], phi[f, k0:k1])
    return slot


def _oracle_all_cores(seed: int, focus_planes, workers: int):
    """The same oracle work as _oracle_sample on all host cores: the SOCS sums of every focus
    plane split over spawned processes by kernels (inputs and partial images in shared
    memory, one numpy thread each), then the resist on each plane.  Returns seconds of
    imaging + resist (the set-up of kernels and workers is not timed, as in _oracle_sample)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    from oracle import optics as OO
    from oracle import resist as ORR
    oo = OO.Optics(193.0, 1.35, 1.44, OO.QUADRUPOLE, 41, pole_sigma=0.8, pole_radius=0.1)
    kern = [OO.socs_kernels(oo, N, PIXEL, z, K)[:2] for z in focus_planes]
    F = len(focus_planes)
    per = max(1, -(-K * F // workers))
    tasks = []
    for f in range(F):
        for k0 in range(0, K, per):
            tasks.append((f, k0, min(K, k0 + per), len(tasks)))
    arrays = {"m": synth.manhattan_mask(N, seed=seed).astype(np.float64),
              "lam": np.stack([k[0] for k in kern]), "phi": np.stack([k[1] for k in kern]),
              "out": np.zeros((len(tasks), N, N))}
    shms, names, shapes = [], {}, {}
    try:
        for key, arr in arrays.items():
            shm = shared_memory.SharedMemory(create=True, size=arr.nbytes)
            shms.append(shm)
            np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)[...] = arr
            names[key], shapes[key] = shm.name, arr.shape
        out = np.ndarray(shapes["out"], dtype=np.float64, buffer=shms[-1].buf)
        env_before = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in env_before:
            os.environ[v] = "1"
        try:
            with mp.get_context("spawn").Pool(workers, initializer=_oracle_worker_init,
                                              initargs=(names, shapes)) as pool:
                pool.map(_oracle_partial, tasks[:workers])          # workers started and warm
                t0 = time.perf_counter()
                pool.map(_oracle_partial, tasks)
                for f in range(F):
                    img = sum(out[t[3]] for t in tasks if t[0] == f)
                    ORR.printed(ORR.blur(img, SIGMA_NM, PIXEL), THRESH)
                return time.perf_counter() - t0
        finally:
            for v, old in env_before.items():
                if old is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = old
    finally:
        for shm in shms:
            shm.close()
            shm.unlink()


def cpu_baseline():
    host = host_facts()
    t = _oracle_sample(1234, FOCUS)
    out = {"value": N * N / t / 1e6, "unit": "Mpx/s", "cores": 1, "kind": "oracle",
           "sample": f"1 of 64 clips (seed 1234), all 3 focus planes x 24 kernels + resist; {t:.1f} s",
           "host": host}
    workers = max(1, int(host["nproc"] or 1))
    try:
        ta = _oracle_all_cores(1234, FOCUS, workers)
        out["all_cores"] = {"value": N * N / ta / 1e6, "unit": "Mpx/s", "cores": workers, "kind": "oracle",
                            "sample": f"the same clip, the 72 (focus, kernel) SOCS terms split over {workers} "
                                      f"spawned processes, then the resist; {ta:.2f} s"}
    except Exception as e:  # a baseline, not a target: report why it is missing
        out["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return out


def run_reference(args):
    """The oracle timed as the reference arm on the same workload (bounded samples)."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    times = []
    for s in range(args.warmup + args.steps):
        t = _oracle_sample(1234 + s, [FOCUS[s % 3]])
        if s >= args.warmup:
            times.append(t)
    per_clip = 3.0 * statistics.mean(times)     # one focus plane per step; a clip has three
    val = N * N / per_clip / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpx/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "clips_per_step": "1 clip x 1 focus plane (bounded sample)"},
            "cpu_baseline": {"value": val, "unit": "Mpx/s", "cores": 1, "kind": "oracle",
                             "sample": "per step: one clip, one of its 3 focus planes, 24 kernels + resist; "
                                       "Mpx/s per whole clip = plane time x 3"},
            "e2e": {"value": val, "unit": "Mpx/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- our implementation --------------------------------------------------------------------------------

class Ctx:
    def __init__(self, args):
        import torch
        self.torch = torch
        self.world, self.rank, self.local = _dist()
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=self.dev)

    def barrier(self):
        if self.world > 1:
            self.torch.distributed.barrier()

    def max_over_ranks(self, x: float) -> float:
        if self.world == 1:
            return x
        t = self.torch.tensor([x], device=self.dev)
        self.torch.distributed.all_reduce(t, op=self.torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            self.torch.distributed.destroy_process_group()


def time_steps(ctx, step, steps, warmup, stream, sample_clocks=False):
    """W untimed steps, then K steps bracketed by CUDA events on `stream`;
    returns (per-step ms list, clock summary)."""
    torch = ctx.torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    ctx.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(ctx.local) if sample_clocks else None
    if clk:
        clk.__enter__()
    for a, b in ev:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__()
    ctx.barrier()
    return [a.elapsed_time(b) for a, b in ev], (clk.summary() if clk else None)


def tensor_summary(results, plain, peaks, models_fn, clips, crop, n_focus, k_eff, kern):
    """The split tensor-core path against both FP32 FFT paths, and its tensor-pipe use over the whole
    step (executed MMA flops of the step / step time / the measured sustained bf16/fp16 peak)."""
    tp = "fp16x3/coarse"
    r = results.get(tp)
    if r is None:
        return None
    coarse = results.get("fft32/coarse")
    flops = models_fn(tp, clips, N, crop, n_focus, k_eff, kern.grid(tp), peaks)["stage2_gemm"][0]
    step_s = r["total_ms"] / len(r["step_ms"]) * 1e-3
    return {"precision": tp, "value": r["value"], "ms_per_step": step_s * 1e3,
            "vs_plain_fft_full_grid": r["value"] / plain["value"] if plain else None,
            "vs_fft32_coarse": r["value"] / coarse["value"] if coarse else None,
            "step_tensor_frac": flops / step_s / (peaks["bf16_tflops_sustained"] * 1e12),
            "note": "executed MMA flops (Gauss 3M, split x3) over the whole step time, against the measured "
                    "sustained dense bf16/fp16 peak"}


def run_aerial(args, ctx):
    import paper_2602_15036_gb300 as P
    from paper_2602_15036_gb300 import litho as L
    torch = ctx.torch
    clips = args.clips
    kern = P.litho_make_kernels(P.make_optics(**OPTICS), N, PIXEL, FOCUS, K)
    info = kern.info()
    k_eff = min(K, min(info["rank"]))
    c = kern.crop
    masks_np = np.stack([synth.manhattan_mask(N, seed=s) for s in clip_seeds(ctx.rank, clips)])
    masks = torch.from_numpy(masks_np).to(ctx.dev)
    F = len(FOCUS)
    img = torch.empty((clips, F, N, N), dtype=torch.float32, device=ctx.dev)
    iblur = torch.empty_like(img)
    printed = torch.empty((clips, F, N, N), dtype=torch.uint8, device=ctx.dev)
    paths = [args.precision] + [p for p in COMPARE if p != args.precision and not args.no_compare]
    ws = torch.empty(max(P.litho_aerial_workspace_size(kern, clips, p) for p in paths), dtype=torch.uint8,
                     device=ctx.dev)
    stream = torch.cuda.current_stream()
    peaks, peak_src = _peaks()
    results = {}
    for i, prec in enumerate(paths):
        def step():
            P.litho_aerial_resist(kern, masks, precision=prec, sigma_nm=SIGMA_NM, threshold=THRESH, out=img,
                                  iblur=iblur, printed=printed, workspace=ws, stream=stream)

        L.litho_profile_enable(True)
        L.litho_profile_reset()
        # warm-up steps are profiled too; reset again right before the timed ones
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        L.litho_profile_reset()
        step_ms, clk = time_steps(ctx, step, args.steps, 0, stream, sample_clocks=(i == 0))
        prof = L.litho_profile_read()
        L.litho_profile_enable(False)
        total_ms = ctx.max_over_ranks(sum(step_ms))
        value = whole_job_rate(clips * N * N * args.steps / 1e6, ctx.world, [total_ms * 1e-3])
        models = stage_models(prec, clips, N, c, F, k_eff, kern.grid(prec), peaks)
        roofs = rooflines(prof, args.steps, models, peaks)
        results[prec] = dict(value=value, step_ms=step_ms, total_ms=total_ms, clocks=clk, prof=prof, roofs=roofs,
                             launches=sum(v[1] for v in prof.values()))

    head = results[args.precision]
    # latency distribution of the headline step: >= 100 timed repetitions, one event pair each
    lat_reps = max(100, args.steps)

    def head_step():
        P.litho_aerial_resist(kern, masks, precision=args.precision, sigma_nm=SIGMA_NM, threshold=THRESH, out=img,
                              iblur=iblur, printed=printed, workspace=ws, stream=stream)

    lat_ms, lat_clk = time_steps(ctx, head_step, lat_reps, 0, stream, sample_clocks=True)
    # end to end through the host-buffer C-ABI call: pinned masks in, printed bytes out
    mask_host = torch.from_numpy(masks_np).pin_memory()
    printed_host = torch.empty((clips, F, N, N), dtype=torch.uint8).pin_memory()
    del ws
    ws_host = torch.empty(P.litho_aerial_host_workspace_size(kern, clips, args.precision), dtype=torch.uint8,
                          device=ctx.dev)

    def e2e_step():
        P.litho_aerial_host(kern, mask_host, ws_host, printed_host=printed_host, precision=args.precision,
                            sigma_nm=SIGMA_NM, threshold=THRESH, stream=stream)

    # warm-up: at least 3 steps and half a second, so that the copies run in the GPU's busy state (the
    # first copies after the GPU has idled, here while the host buffers were pinned, run several times slower)
    t_w, n_w = time.perf_counter(), 0
    while n_w < max(3, args.warmup) or time.perf_counter() - t_w < 0.5:
        e2e_step()
        n_w += 1
    ctx.barrier()
    e2e_steps = max(3, min(args.steps, 10))
    e2e_ms, e2e_trace = [], []
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        e2e_step()                       # synchronous: returns after the printed bytes are on the host
        e2e_ms.append(1e3 * (time.perf_counter() - t1))
        tr = dict((tag, ms) for tag, ms in L.litho_host_trace_read())
        # device time per chunk, ms since the call's first work: input copied, kernels done, outputs copied
        dev = []
        for ci in range(64):
            if 100 + 8 * ci not in tr:
                break
            dev.append(tuple(round(tr[100 + 8 * ci + i], 3) for i in range(3)))
        e2e_trace.append((tr.get(-1, 0.0), tr.get(-2, 0.0) - tr.get(-1, 0.0), dev))
    e2e_s = ctx.max_over_ranks(time.perf_counter() - t0)
    ctx.barrier()
    e2e_val = whole_job_rate(clips * N * N * e2e_steps / 1e6, ctx.world, [e2e_s])

    dominant = max(head["roofs"].items(), key=lambda kv: kv[1]["ms_per_step"])
    roof = dict(dominant[1])
    roof["kernel"] = dominant[0]
    roof["traffic"], roof["traffic_source"] = measured_traffic(dominant[0], args.precision, clips,
                                                               roof["launches_per_step"])
    roof["peak_source"] = (f"{peak_src} HBM copy bandwidth" if roof["bound"] == "hbm" else alu_peak_source())
    plain = results.get("fft32")
    line = {"metric": METRIC, "value": head["value"], "unit": "Mpx/s", "n_gpus": ctx.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "clips_per_gpu": clips, "precision": args.precision,
                       "error_bound_abs": ERROR_BOUND.get(args.precision),
                       "parallelism": f"replicas x{ctx.world} (clips sharded, no collective)",
                       "l2": "inputs larger than L2 (1.07 GB masks, 3.2 GB images per step); no flush"},
            "p50_ms": statistics.median(lat_ms), "p99_ms": float(np.percentile(lat_ms, 99)),
            "latency_reps": lat_reps, "latency_clocks": lat_clk,
            "vs_plain_fft": (head["value"] / plain["value"]) if plain else None,
            "tensor_path": tensor_summary(results, plain, peaks, stage_models, clips, c, F, k_eff, kern),
            "paths": {p: {"value": r["value"], "ms_per_step": r["total_ms"] / args.steps,
                          "error_bound_abs": ERROR_BOUND.get(p),
                          "stages_ms_per_step": {k: v[0] / args.steps for k, v in r["prof"].items()},
                          "roofline": r["roofs"]} for p, r in results.items()},
            "gpu_launches": head["launches"],
            "gpu_launches_per_step": head["launches"] / args.steps,
            "e2e": {"value": e2e_val, "unit": "Mpx/s", "h2d_bytes_per_step": int(mask_host.numel() * 4),
                    "d2h_bytes_per_step": int(printed_host.numel()), "steps": e2e_steps, "warmup_steps": n_w,
                    "step_ms": [round(x, 3) for x in e2e_ms],
                    "host_trace": {"enqueue_ms": [round(a, 3) for a, _, _ in e2e_trace],
                                   "wait_ms": [round(b, 3) for _, b, _ in e2e_trace],
                                   "chunk_device_ms": [c for _, _, c in e2e_trace],
                                   "note": "per call: host time to enqueue every chunk's copies and launches, "
                                           "then the wait for the device; per chunk the device times (ms since "
                                           "the call's first work) at which its input copy, its kernels and its "
                                           "output copies ended (litho_host_trace_read)"}},
            "roofline": roof, "peaks_source": peak_src, "clocks": head["clocks"]}
    if ctx.rank == 0 and ctx.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    return line


def run_ilt(args, ctx):
    """16 clips of 1024^2, annular 21x21, K=16, 5 focus planes; one step = litho_ilt_grad on all clips
    plus the gradient-descent update theta -= 0.5 g / max|g| (torch, outside the library).  --precision
    fft32/coarse (default) evaluates fields and adjoint on the 512-point coarse grid, fft32 on 1024."""
    import paper_2602_15036_gb300 as P
    from paper_2602_15036_gb300 import litho as L
    torch = ctx.torch
    prec = args.precision if args.precision in ("fft32", "fft32/coarse") else "fft32/coarse"
    n, pixel, k, focus, clips = 1024, 8.0, 16, [-60.0, -30.0, 0.0, 30.0, 60.0], 16
    optics = dict(wavelength_nm=193.0, na=1.35, n_medium=1.44, kind="annular", src_grid=21, sigma_in=0.6,
                  sigma_out=0.9)
    kern = P.litho_make_kernels(P.make_optics(**optics), n, pixel, focus, k)
    data = [synth.ilt_clip(n, pixel, seed=s) for s in clip_seeds(ctx.rank, clips, base=4000)]
    theta = torch.from_numpy(np.stack([d[0] for d in data])).to(ctx.dev)
    target = torch.from_numpy(np.stack([d[1] for d in data])).to(ctx.dev)
    grad = torch.empty_like(theta)
    ws = torch.empty(P.litho_ilt_workspace_size(kern, clips)[0], dtype=torch.uint8, device=ctx.dev)
    stream = torch.cuda.current_stream()
    losses = []

    def step():
        _, loss = P.litho_ilt_grad(kern, theta, target, grad=grad, workspace=ws, want_loss=True, precision=prec,
                                   stream=stream)
        losses.append(float(loss.sum()))
        theta.sub_(0.5 * grad / grad.abs().amax(dim=(1, 2), keepdim=True).clamp_min(1e-30))

    L.litho_profile_enable(True)
    L.litho_profile_reset()
    step_ms, clk = time_steps(ctx, step, args.steps, args.warmup, stream, sample_clocks=True)
    prof = L.litho_profile_read()
    L.litho_profile_enable(False)
    total = ctx.max_over_ranks(sum(step_ms))
    peaks, peak_src = _peaks()
    ne = kern.grid(prec) if prec.endswith("/coarse") else n
    per_clip = len(focus) * k * n * kern.crop * 8.0  # the library's clip groups: stage-1 fields within 2 GiB
    cap = max(1, min(clips, int((2 << 30) // per_clip)))
    group = -(-clips // -(-clips // cap))
    roofs = rooflines(prof, args.steps + args.warmup,
                      ilt_models(clips, n, ne or n, kern.crop, len(focus), k, bool(ne) and ne < n, group), peaks)
    dominant = max(roofs.items(), key=lambda kv: kv[1]["ms_per_step"])
    roof = dict(dominant[1], kernel=dominant[0], traffic=None,
                peak_source=f"derived ALU peak; {peak_src} HBM copy bandwidth")
    line = {"metric": "ILT gradient Mpx/s (1024² clips, K=16, 5 focus)", "workload": "ilt",
            "value": whole_job_rate(clips * n * n * args.steps / 1e6, ctx.world, [total * 1e-3]), "unit": "Mpx/s",
            "n_gpus": ctx.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ilt 16x1024^2@8nm annular21 K=16 focus(-60..60 step 30)", "clips_per_gpu": clips,
                       "precision": prec, "grid": kern.grid(prec) if prec.endswith("/coarse") else n},
            "loss_first_last": [losses[0], losses[-1]],
            "loss_curve": {"steps": len(losses), "every": 1, "sum_over_clips": [float(f"{v:.6g}") for v in losses]},
            "stages_ms_per_step": {kk: v[0] / (args.steps + args.warmup) for kk, v in prof.items()},
            "roofline": roof, "stage_rooflines": {kk: {x: v[x] for x in ("bound", "frac")} for kk, v in roofs.items()},
            "gpu_launches": sum(v[1] for v in prof.values()), "clocks": clk}
    return line


def run_contour(args, ctx):
    """Contours and edge placement on the headline's resist images: 64 clips of 2048^2 x 3 focus
    planes (made once, untimed, by litho_aerial_resist); one step = marching squares on every plane
    + Eq. (6) EPE at the edge sites of every clip's target (its mask) on its 3 planes + Eqs. (7)-(8)."""
    import paper_2602_15036_gb300 as P
    from paper_2602_15036_gb300 import litho as L
    torch = ctx.torch
    clips = args.clips
    kern = P.litho_make_kernels(P.make_optics(**OPTICS), N, PIXEL, FOCUS, K)
    F = len(FOCUS)
    masks_np = np.stack([synth.manhattan_mask(N, seed=s) for s in clip_seeds(ctx.rank, clips)])
    stream = torch.cuda.current_stream()
    _, iblur, _ = P.litho_aerial_resist(kern, torch.from_numpy(masks_np).to(ctx.dev), precision=HEADLINE,
                                        sigma_nm=SIGMA_NM, threshold=THRESH, stream=stream)
    pts_np = [synth.edge_sites(m).astype(np.float32) for m in masks_np]
    n_pts = sum(len(p) for p in pts_np)
    pts = torch.from_numpy(np.concatenate(pts_np)).to(ctx.dev)          # all clips' edge sites
    pt_start = torch.from_numpy(np.concatenate([[0], np.cumsum([len(p) for p in pts_np])]).astype(np.int64)).to(
        ctx.dev)
    planes = clips * F
    ws = torch.empty(L.contours_workspace_size(planes, N), dtype=torch.uint8, device=ctx.dev)
    starts = torch.empty(planes + 1, dtype=torch.int64, device=ctx.dev)
    _, _, st0 = P.litho_contours(iblur, THRESH, capacity=0, with_cells=False, stream=stream)
    capacity = int(st0[-1]) + 1024
    seg = torch.empty((capacity, 4), dtype=torch.float32, device=ctx.dev)
    cell = torch.empty(capacity, dtype=torch.int32, device=ctx.dev)
    epe = torch.empty((F, n_pts), dtype=torch.float32, device=ctx.dev)
    avg = torch.empty(n_pts, dtype=torch.float32, device=ctx.dev)
    eff = torch.empty(n_pts, dtype=torch.float32, device=ctx.dev)

    def step():
        L.contours_into(iblur, planes, N, THRESH, seg, cell, capacity, starts, ws, stream)
        P.litho_epe_batch(iblur, pts, pt_start, PIXEL, THRESH, out=epe, stream=stream)
        L.epe_through_focus_into(epe, 1, 2, 0, -1.0, 1.0, avg, eff, stream)

    L.litho_profile_enable(True)
    L.litho_profile_reset()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    L.litho_profile_reset()
    step_ms, clk = time_steps(ctx, step, args.steps, 0, stream, sample_clocks=True)
    prof = L.litho_profile_read()
    L.litho_profile_enable(False)
    total = ctx.max_over_ranks(sum(step_ms))
    n_seg = int(starts[-1].item())
    sec = lambda name: prof.get(name, (0.0, 0))[0] / args.steps * 1e-3  # noqa: E731
    c_bytes = planes * N * N * 4.0 + n_seg * 20.0        # read every plane once, write each segment + cell
    e_bytes = n_pts * (8.0 + F * 4.0 + 8.0)              # points in, EPE per plane and avg/eff out
    peaks, peak_src = _peaks()
    roof = {"bound": "hbm", "achieved": c_bytes / sec("contours") / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "kernel": "contours", "algorithmic_bytes_per_step": c_bytes, "ms_per_step": sec("contours") * 1e3,
            "traffic": None, "peak_source": f"{peak_src} HBM copy bandwidth"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    line = {"metric": "contour + EPE Mpx/s (2048² resist images, 3 focus planes)", "workload": "contour",
            "value": whole_job_rate(clips * N * N * args.steps / 1e6, ctx.world, [total * 1e-3]), "unit": "Mpx/s",
            "n_gpus": ctx.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"contours+epe {clips}x2048^2 x3 focus, {n_pts} edge sites", "clips_per_gpu": clips},
            "segments_per_step": n_seg, "edge_sites": n_pts,
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "epe_roofline": {"bound": "hbm", "achieved": e_bytes / sec("epe") / 1e9 if sec("epe") else None,
                             "unit": "GB/s"},
            "gpu_launches": sum(v[1] for v in prof.values()), "roofline": roof, "clocks": clk}
    return line


def run_raster(args, ctx):
    """Area-coverage rasterisation of the headline's masks as shapes off the pixel grid: the
    Manhattan generator's rectangles of 64 clips of 2048^2, shifted by (0.3, 0.6) px so that
    every edge is a grey level; one step = litho_rasterize of all clips."""
    import paper_2602_15036_gb300 as P  # noqa: F401
    from paper_2602_15036_gb300 import litho as L
    torch = ctx.torch
    clips = args.clips
    rl = []
    for s_ in clip_seeds(ctx.rank, clips):
        r, _ = synth.manhattan_rects(N, seed=s_)
        x0, y0 = r[:, 0] + 0.3, r[:, 1] + 0.6
        rl.append(np.stack([x0, y0, x0 + r[:, 2], y0 + r[:, 3]], axis=1).astype(np.float32))
    counts = [len(r) for r in rl]
    start = torch.from_numpy(np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)).to(ctx.dev)
    rects = torch.from_numpy(np.concatenate(rl)).to(ctx.dev)
    max_rects, max_side = max(counts), 16
    ws = torch.empty(L.rasterize_workspace_size(clips, N, max_rects, max_side), dtype=torch.uint8, device=ctx.dev)
    mask = torch.empty((clips, N, N), dtype=torch.float32, device=ctx.dev)
    stream = torch.cuda.current_stream()

    def step():
        L.rasterize_into(rects, start, clips, max_rects, max_side, N, mask, ws, stream)

    L.litho_profile_enable(True)
    L.litho_profile_reset()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    L.litho_profile_reset()
    step_ms, clk = time_steps(ctx, step, args.steps, 0, stream, sample_clocks=True)
    prof = L.litho_profile_read()
    L.litho_profile_enable(False)
    total = ctx.max_over_ranks(sum(step_ms))
    grey = float(((mask > 0) & (mask < 1)).float().mean().item())
    nbytes = clips * N * N * 4.0 + sum(counts) * 16.0
    peaks, peak_src = _peaks()
    sec = total / args.steps * 1e-3
    roof = {"bound": "hbm", "achieved": nbytes / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "kernel": "raster", "algorithmic_bytes_per_step": nbytes, "traffic": None,
            "peak_source": f"{peak_src} HBM copy bandwidth"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    line = {"metric": "area-coverage rasterisation Mpx/s (2048² clips)", "workload": "raster",
            "value": whole_job_rate(clips * N * N * args.steps / 1e6, ctx.world, [total * 1e-3]), "unit": "Mpx/s",
            "n_gpus": ctx.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"raster {clips}x2048^2, {sum(counts)} rectangles", "clips_per_gpu": clips},
            "grey_pixel_fraction": grey, "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "gpu_launches": sum(v[1] for v in prof.values()), "roofline": roof, "clocks": clk}
    return line


def run_ai(args, ctx):
    """AI initialiser inputs for 16 clips of 2048^2 (the headline optics, nominal focus, K = 24):
    one step = the Eq. (9) channels (target, aerial image, intensity gradient, normalised over
    the batch) + Eqs. (15)-(17) print images and loss against the aerial image."""
    import paper_2602_15036_gb300 as P
    from paper_2602_15036_gb300 import litho as L
    torch = ctx.torch
    clips = min(args.clips, 16)
    kern = P.litho_make_kernels(P.make_optics(**OPTICS), N, PIXEL, [0.0], K)
    targets = torch.from_numpy(np.stack([synth.manhattan_mask(N, seed=s) for s in clip_seeds(ctx.rank, clips)])).to(
        ctx.dev)
    stream = torch.cuda.current_stream()
    prec = args.precision if args.precision in ("fft32", "fft32/coarse") else "fft32/coarse"
    ws = torch.empty(L.litho_ai_inputs_workspace_size(kern, clips), dtype=torch.uint8, device=ctx.dev)
    xbuf = torch.empty((clips, 3, N, N), dtype=torch.float32, device=ctx.dev)
    out = {}

    def step():
        x = P.litho_ai_inputs(kern, targets, focus=0, precision=prec, out=xbuf, workspace=ws, stream=stream)
        out["x"] = x
        out["p"] = P.litho_print_images(targets, x[:, 1].contiguous(), PIXEL, 20.0, 0.5, 0.3, stream=stream)

    L.litho_profile_enable(True)
    L.litho_profile_reset()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    L.litho_profile_reset()
    step_ms, clk = time_steps(ctx, step, args.steps, 0, stream, sample_clocks=True)
    prof = L.litho_profile_read()
    L.litho_profile_enable(False)
    total = ctx.max_over_ranks(sum(step_ms))
    peaks, peak_src = _peaks()
    ne = kern.grid(prec) if prec.endswith("/coarse") else N
    round_taps = 2 * math.ceil(4 * 20.0 / PIXEL) + 1
    roofs = rooflines(prof, args.steps, ai_models(clips, N, ne or N, kern.crop, K, bool(ne) and ne < N, round_taps),
                      peaks)
    dominant = max(roofs.items(), key=lambda kv: kv[1]["ms_per_step"])
    roof = dict(dominant[1], kernel=dominant[0], traffic=None,
                peak_source=f"derived ALU peak; {peak_src} HBM copy bandwidth")
    line = {"metric": "AI-input channels + print images Mpx/s (2048² targets, K=24)", "workload": "ai",
            "value": whole_job_rate(clips * N * N * args.steps / 1e6, ctx.world, [total * 1e-3]), "unit": "Mpx/s",
            "n_gpus": ctx.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
            "higher_is_better": True, "scaling": "weak", "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ai inputs {clips}x2048^2 quadrupole41 K=24 nominal focus", "clips_per_gpu": clips,
                       "precision": prec},
            "litho_loss_first_clips": [int(v) for v in out["p"][2][:4].cpu().tolist()],
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "roofline": roof, "stage_rooflines": {kk: {x: v[x] for x in ("bound", "frac")} for kk, v in roofs.items()},
            "gpu_launches": sum(v[1] for v in prof.values()), "clocks": clk}
    return line


def run_serve(args, ctx):
    """Poisson stream of mixed requests through litho_serve (sizes 256..2048, DUV and EUV optics,
    K in {8,16,24}, half images and half ILT steps) at 80 % of the measured saturated rate."""
    from paper_2602_15036_gb300 import litho as L
    duv = dict(wavelength_nm=193.0, na=1.35, n_medium=1.44, kind="annular", src_grid=21, sigma_in=0.6,
               sigma_out=0.9)
    euv = dict(wavelength_nm=13.5, na=0.33, n_medium=1.0, kind="annular", src_grid=21, sigma_in=0.6, sigma_out=0.9)
    st = synth.Stream(77)
    total = args.requests
    sizes = [256, 512, 1024, 2048]
    import torch
    keep = []

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
        keep.append(t)
        return t.numpy()

    # page-locked request buffers: the server DMAs them directly (no staging copy)
    pool = {n: [(pinned(synth.random_rect_mask(n, seed=10 * n + i, count=n // 4)),) +
                tuple(pinned(a) for a in synth.ilt_clip(n, 8.0, seed=20 * n + i)) for i in range(2)]
            for n in sizes}
    reqs = []
    for i in range(total):
        n = sizes[int(st.integers(0, 3, 1)[0])]
        is_euv = bool(st.integers(0, 1, 1)[0])
        k = [8, 16, 24][int(st.integers(0, 2, 1)[0])]
        kind = "image" if st.integers(0, 1, 1)[0] == 0 else "ilt"
        reqs.append((kind, euv if is_euv else duv, n, 1.0 if is_euv else 8.0, k, pool[n][i % 2]))
    srv = L.Server(64 << 30, max_slots=8, max_queue=total + 16)
    outs = {}

    out_bufs = {}

    def submit(r, idx=None):
        kind, opt, n, pixel, k, (mask, theta, tgt) = r
        key = (idx, n) if idx is not None else ("warm", n)
        if key not in out_bufs:
            out_bufs[key] = pinned(np.empty((n, n), dtype=np.float32))
        out = out_bufs[key]
        inp = mask if kind == "image" else theta
        t, _ = srv.submit(kind, L.make_optics(**opt), n, pixel, 0.0, k, inp, out,
                          target_host=tgt if kind == "ilt" else None, precision="fft32/coarse")
        outs[t] = out
        return t

    statuses, first_err = {}, []

    def drain(tickets):
        for t in tickets:
            st_ = srv.poll(t, 1000)
            while st_ == L.ETIMEOUT:
                st_ = srv.poll(t, 1000)
            name = L.STATUS_NAMES[st_]
            statuses[name] = statuses.get(name, 0) + 1
            if st_ != L.OK and not first_err:
                first_err.append(L.litho_last_error())

    # warm the kernel-set cache: one request per (optics, n, k) key, untimed
    keys = {}
    for r in reqs:
        keys.setdefault((r[1]["wavelength_nm"], r[2], r[4]), r)
    drain([submit(r) for r in keys.values()])
    # saturated throughput: the whole stream submitted at once (it batches by key)
    burst = reqs
    for i, r in enumerate(reqs):      # one output buffer per request, allocated before any timing
        out_bufs.setdefault((i, r[2]), pinned(np.empty((r[2], r[2]), dtype=np.float32)))
    srv.stats_reset()
    t0 = time.perf_counter()
    drain([submit(r, i) for i, r in enumerate(burst)])
    sat_s = time.perf_counter() - t0
    sat_rps = len(burst) / sat_s
    sat_px = sum(r[2] * r[2] for r in burst)
    s_sat = srv.stats()
    srv.close()
    px = sum(r[2] * r[2] for r in reqs)
    sweep = {}
    for load in (0.5, 0.8, 0.9):
        srv = L.Server(64 << 30, max_slots=8, max_queue=total + 16)
        drain([submit(r) for r in keys.values()])
        srv.stats_reset()          # latencies of the timed stream only (not the kernel-set warm-up)
        rate = load * sat_rps
        arrivals = np.cumsum(-np.log(1.0 - synth.Stream(78).uniform(total)) / rate)
        tickets = []
        t0 = time.perf_counter()
        for i, (r, ta) in enumerate(zip(reqs, arrivals)):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            tickets.append(submit(r, i))
        drain(tickets)
        wall = time.perf_counter() - t0
        s = srv.stats()
        srv.close()
        sweep[load] = {"arrival_rate_rps": rate, "p50_ms": s["p50_ms"], "p99_ms": s["p99_ms"],
                       "mpx_per_s": px / wall / 1e6, "batches": s["batches"],
                       "mean_batch": s["completed"] / max(1, s["batches"]), "max_batch": s["max_batch"]}
    line = {"metric": "serving p50/p99 latency and Mpx/s (Poisson, mixed sizes/optics/K, image+ILT)",
            "workload": "serve", "value": sweep[0.8]["mpx_per_s"], "unit": "Mpx/s", "n_gpus": ctx.world,
            "requests": total, "arrival_rate_rps": sweep[0.8]["arrival_rate_rps"], "saturated_rps": sat_rps,
            "saturated": {"requests": len(burst), "mpx_per_s": sat_px / sat_s / 1e6, "seconds": sat_s,
                          "batches": s_sat["batches"], "mean_batch": s_sat["completed"] / max(1, s_sat["batches"]),
                          "max_batch": s_sat["max_batch"]},
            "p50_ms": sweep[0.8]["p50_ms"], "p99_ms": sweep[0.8]["p99_ms"], "load_sweep": sweep,
            "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "config": {"precision": "fft32/coarse (images and ILT steps)", "slots": 8},
            "stats": {k: s[k] for k in ("submitted", "completed", "rejected", "cancelled", "hbm_high_water",
                                         "kernel_sets_cached")},
            "status_counts": statuses, "first_error": first_err[0] if first_err else None}
    return line


def run_all_workloads(args, ctx) -> dict:
    """The other workloads of the library, each timed as its own bench mode would time it, for
    the default run's JSON line: ILT (100 gradient steps of 16 x 1024^2, K = 16, 5 planes, with
    the loss curve), AI inputs, contours + EPE, the rasteriser, and serving (4096 Poisson
    requests at 0.5, 0.8 and 0.9 of the saturated rate)."""
    import copy
    out = {}
    plans = [("ilt", run_ilt, dict(steps=100, warmup=3, precision="fft32/coarse")),
             ("ai", run_ai, dict(steps=max(10, args.steps), warmup=3, precision="fft32/coarse", clips=16)),
             ("contour", run_contour, dict(steps=max(10, args.steps), warmup=3, clips=64)),
             ("raster", run_raster, dict(steps=max(10, args.steps), warmup=3, clips=64)),
             ("serve", run_serve, dict(requests=4096))]
    for name, fn, over in plans:
        a = copy.copy(args)
        for k, v in over.items():
            setattr(a, k, v)
        try:
            out[name] = fn(a, ctx)
        except Exception as e:   # report the failure in the line instead of losing the headline
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        ctx.torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["aerial", "ilt", "serve", "contour", "raster", "ai"], default="aerial")
    ap.add_argument("--precision", default=HEADLINE,
                    choices=sorted(ERROR_BOUND) + ["bf16/coarse"])
    ap.add_argument("--clips", type=int, default=64)
    ap.add_argument("--requests", type=int, default=4096)
    ap.add_argument("--no-compare", action="store_true", help="time only --precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="aerial workload only: skip the other workloads of the default line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    ctx = Ctx(args)
    fn = {"ilt": run_ilt, "serve": run_serve, "contour": run_contour, "raster": run_raster, "ai": run_ai,
          "aerial": run_aerial}[args.workload]
    line = fn(args, ctx)
    if args.workload == "aerial" and ctx.world == 1 and not args.headline_only:
        line["workloads"] = run_all_workloads(args, ctx)
    if ctx.rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
