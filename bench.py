"""Benchmark: rotational-OMP coding throughput (patches/s) on GB300.

Workload: 1,000,000 synthetic patches of 11x11 in the steerable basis
(J = 6 rings, harmonics |k| <= 8, n = 102 real coefficients), M = 64 atoms,
R = 64 angles, K = 5 greedy steps, 3 planted atoms per patch plus noise
sigma = 0.1 (seeded, synthetic: the paper's images are not used).  One step =
one rsc_encode of all patches (one kernel launch) with the inputs resident in
HBM; the 432 MB input is larger than the 129 MB L2, so no flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32]
       [--impl reference]
Under torchrun each rank codes its own 1M patches (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1806_04374_gb300 import synth  # noqa: E402

WORKLOAD = "omp_1m"
METRIC = "rotational-OMP patches/s vs plain FP32 path, oracle-matched; p50/p99 latency"
FP32_LANES_PER_SM = 128


def algorithmic_flops_per_patch(wl) -> dict:
    """Per patch per greedy step: (a) per-harmonic contraction 2J(1+4kmax)M
    flops, (b) angle transform 2.5 R log2(R) flops per atom (radix-2
    convention; the direct form is M R (4kmax+1)); times K steps."""
    import math
    fa = 2 * wl.J * (1 + 4 * wl.kmax) * wl.M
    fb = int(2.5 * wl.R * math.log2(wl.R) * wl.M)
    fb_direct = wl.M * wl.R * (4 * wl.kmax + 1)
    return {"a": fa, "b": fb, "b_direct": fb_direct, "per_patch": wl.K * (fa + fb)}


def mma_flops_per_patch(wl) -> int:
    """Dense flops the tensor-core path executes per patch.  Plain layout:
    K steps x 2 x (depth rounded up to 16) x (M R steered atoms).  Paired
    layout (even R, even harmonics in <= 64 slots, odd ones in <= 48): the
    even and odd halves, each rounded up to 16, against M R / 2 atom pairs."""
    ne = wl.J + 2 * wl.J * (wl.kmax // 2)
    no = 2 * wl.J * ((wl.kmax + 1) // 2)
    up = lambda v: ((v + 15) // 16) * 16  # noqa: E731
    if wl.R % 2 == 0 and wl.kmax >= 1 and ne <= 64 and no <= 48:
        return wl.K * 2 * (up(ne) + up(no)) * wl.M * (wl.R // 2)
    n = wl.J * (2 * wl.kmax + 1)
    return wl.K * 2 * up(n) * wl.M * wl.R


def kernel_launch_count(slots, K: int, precision: str) -> int:
    """Kernels launched, from the library's per-phase event slots: a scoring
    slot and a hand-off slot are one kernel each; on the FP16 path each group
    has one refine-phase slot around the init kernel and K around the
    refine's two passes (two kernels each)."""
    score, handoff, refine = (int(v) for v in slots)
    if precision != "f16":
        return score + handoff + refine
    inits = refine // (K + 1)
    return score + handoff + inits + 2 * (refine - inits)


def algorithmic_bytes_per_patch(wl) -> int:
    n_floats = (wl.kmax + 1) * wl.J * 2
    return 4 * n_floats + wl.K * (4 + 4 + 4 + 8) + 4


def recovery(d_learned, d_true, R: int, threshold: float = 0.99, refine: int = 16) -> float:
    """Evaluation of a learned dictionary (host, numpy): the fraction of true
    atoms t with max over learned atoms m and angles theta (an R*refine grid)
    of |<S_theta d_m, t>| >= threshold."""
    dl = np.asarray(d_learned, np.float64)
    dt = np.asarray(d_true, np.float64)
    H = dl.shape[1]
    zl = dl[..., 0] + 1j * dl[..., 1]
    zt = dt[..., 0] + 1j * dt[..., 1]
    zl[:, 0] = zl[:, 0].real
    zt[:, 0] = zt[:, 0].real
    w = np.ones(H)
    w[1:] = 2.0
    G = np.einsum("mkj,tkj->mtk", np.conj(zl), zt)
    th = 2 * np.pi * np.arange(R * refine) / (R * refine)
    ph = np.exp(1j * np.outer(th, np.arange(H)))
    s = np.einsum("ak,mtk->mta", ph * w, G).real
    return float(np.mean(np.abs(s).max(axis=(0, 2)) >= threshold))


def rank_inputs(rank: int, P: int):
    """Rank r codes its own patches: chunks [r*n, (r+1)*n) of the seeded
    generator, with the shared dictionary."""
    wl = synth.WORKLOADS[WORKLOAD]
    d = synth.make_dictionary(wl.M, wl.J, wl.kmax, wl.seed)
    nchunks = (P + synth.CHUNK - 1) // synth.CHUNK
    ids = list(range(rank * nchunks, (rank + 1) * nchunks))
    x, _ = synth.make_patches(d, P + rank * nchunks * synth.CHUNK, wl.n_terms, wl.sigma,
                              wl.seed + 1, chunk_ids=ids)
    return d, x[:P], wl


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms by a
    reader thread; only the samples taken between start() and stop() (the
    timed region) are summarised."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        import threading
        self.lines = []
        self.t0 = self.t1 = None
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # wait (up to 5 s) for the first sample so that the region is covered
        deadline = time.monotonic() + 5.0
        while not self.lines and time.monotonic() < deadline and self.proc.poll() is None:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line))

    def start(self):
        self.t0 = time.monotonic()

    def stop(self) -> dict | None:
        self.t1 = time.monotonic()
        if self.proc is None:
            return None
        time.sleep(0.15)  # the sample that closes the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        inside = [ln for (t, ln) in self.lines if self.t0 <= t <= self.t1 + 0.15]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in inside:
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm),
                "window_s": round(self.t1 - self.t0, 3)}


SCORE_SOURCES = ("romp_score.cu", "tc_ptx.cuh", "tc_common.cuh", "rsc_internal.h")
REFINE_SOURCES = ("romp_refine.cu", "tc_common.cuh", "rsc_internal.h")
# bytes a patch must move in one init or refine launch of the FP16 path: read
# its coefficients x (kmax+1) x J x 2 floats, write its fp16 residual row of
# L slots (the per-patch state in between is this design's, not the method's)


def source_digest(names=SCORE_SOURCES) -> str:
    """sha1 over the code of the CUDA sources a kernel is compiled from, with
    comments, trailing blanks and empty lines removed (a comment edit does not
    change the kernel, so it does not void a capture)."""
    import hashlib
    import re
    h = hashlib.sha1()
    for nm in names:
        with open(os.path.join(ROOT, "paper_1806_04374_gb300", "csrc", nm), encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        lines = (re.sub(r"//.*", "", ln).rstrip() for ln in text.splitlines())
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()


def recorded_traffic(P: float, profile: str = "romp_score_kernel_omp_1m.md",
                     names=SCORE_SOURCES):
    """DRAM bytes per launch of a kernel for a launch over P patches, from its
    committed ncu summary (dram__bytes_read.sum + dram__bytes_write.sum of one
    capture, per patch, scaled to P: the kernel's traffic is linear in the
    patches it reads and writes), or None when the kernel's sources changed
    since the capture."""
    path = os.path.join(ROOT, "profiles", profile)
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        for key in ("dram_bytes_per_patch:", "source_sha1:"):
            if line.strip().startswith(key):
                vals[key] = line.split(":", 1)[1].strip().strip("`")
    if vals.get("source_sha1:") != source_digest(names):
        return None
    try:
        return float(vals["dram_bytes_per_patch:"]) * P
    except (KeyError, ValueError):
        return None


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


PARITY_LO, PARITY_N = 256, 2048  # patches of the timed outputs checked against the oracle
COEF_TOL = {"f16": 1e-3, "fp32": 1e-5}


def oracle_parity(x, d, wl, gpu: dict, free: dict, coef_tol: float, margin: float = 1e-6) -> dict:
    """The parity rule of the tests, counted instead of asserted, on outputs
    of the timed run: (1) at every step whose exact top-two margin in the free
    oracle run exceeds `margin` (relative), the GPU pick equals the oracle's;
    (2) along the GPU's own picks (forced-path oracle run) every pick scores
    within `margin` of its step's best, the weights are within `coef_tol`
    (relative 2-norm per patch) of the FP64 least-squares weights and the
    residual norm^2 within 1e-5 ||x||^2."""
    import oracle
    K = wl.K
    ga, gr = gpu["atom"].reshape(-1, K), gpu["angle_idx"].reshape(-1, K)
    gc, gn = gpu["coef"].reshape(-1, K), gpu["resid_norm2"].reshape(-1)
    forced = oracle.romp(x, d, wl.R, K, forced_atom=ga, forced_angle=gr)
    x64 = x.astype(np.float64)
    xn2 = 2 * np.einsum("phjc,phjc->p", x64, x64) - np.einsum("pjc,pjc->p", x64[:, 0], x64[:, 0])
    sel_mis = pick_mis = coef_mis = rn_mis = pinned = unpinned = 0
    max_coef = max_rn = 0.0
    for p in range(x.shape[0]):
        for t in range(K):
            if free["atom"][p, t] < 0:
                pinned += 1
                sel_mis += int(ga[p, t] >= 0)
                continue
            if free["margin"][p, t] <= margin:
                unpinned += 1
                break
            pinned += 1
            sel_mis += int(ga[p, t] != free["atom"][p, t] or gr[p, t] != free["angle"][p, t])
        for t in range(K):
            if ga[p, t] < 0:
                stop = oracle.STOP_REL * np.sqrt(max(xn2[p], 0.0))
                pick_mis += int(forced["best_score"][p, t] > stop * 1.01 + 1e-300)
                break
            bs, ps = forced["best_score"][p, t], forced["pick_score"][p, t]
            pick_mis += int(ps < bs * (1.0 - margin) - 1e-300)
        ref = forced["coef"][p]
        nref = np.linalg.norm(ref)
        err = np.linalg.norm(gc[p] - ref)
        coef_mis += int(not (err <= coef_tol * max(nref, 1e-300) or err == 0.0))
        if nref > 0:
            max_coef = max(max_coef, float(err / nref))
        rerr = abs(float(gn[p]) - forced["rn2"][p]) / max(xn2[p], 1e-30)
        rn_mis += int(rerr > 1e-5)
        max_rn = max(max_rn, rerr)
    return {"patches": int(x.shape[0]), "pinned_steps": pinned, "unpinned_patches": unpinned,
            "selection_mismatches": sel_mis, "pick_margin_violations": pick_mis,
            "coef_tol": coef_tol, "coef_violations": coef_mis, "rn2_violations": rn_mis,
            "mismatches": sel_mis + pick_mis + coef_mis + rn_mis,
            "max_rel_coef_err": max_coef, "max_rel_rn2_err_of_xnorm2": max_rn}


def cpu_baseline(d, x, wl, budget_s: float = 10.0, parity_outputs: dict | None = None) -> dict:
    """The FP64 oracle as it stands, on all host cores, on a bounded sample.
    With `parity_outputs` ({path: GPU outputs of patches PARITY_LO ..
    PARITY_LO + PARITY_N of a timed run}), the oracle's results on those
    patches (the first part of the timed sample) also state the error of
    those outputs against the oracle (`oracle_parity`)."""
    import oracle
    cores = oracle.max_threads()
    n0 = PARITY_LO
    t = time.perf_counter()
    oracle.romp(x[:n0], d, wl.R, wl.K)
    dt0 = time.perf_counter() - t
    n1 = int(min(max(n0, n0 / max(dt0, 1e-6) * budget_s), 65536, x.shape[0] - n0))
    t = time.perf_counter()
    free = oracle.romp(x[n0:n0 + n1], d, wl.R, wl.K)
    dt1 = time.perf_counter() - t
    res = {"value": n1 / dt1, "unit": "patches/s", "cores": cores, "kind": "oracle",
           "sample": f"{n1} patches of the {WORKLOAD} workload (patches {n0}..{n0 + n1 - 1}), "
                     f"{dt1:.1f} s, FP64 C oracle, OpenMP over patches"}
    if parity_outputs:
        ns = min(PARITY_N, n1)
        fr = {k: v[:ns] for k, v in free.items()}
        res["parity"] = {path: oracle_parity(x[n0:n0 + ns], d, wl,
                                             {k: v[:ns] for k, v in out.items()}, fr,
                                             COEF_TOL[path])
                         for path, out in parity_outputs.items()}
    return res


def run_reference(args) -> None:
    """Reference arm: the FP64 oracle on the host cores, bounded sample/step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    wl = synth.WORKLOADS[WORKLOAD]
    d = synth.make_dictionary(wl.M, wl.J, wl.kmax, wl.seed)
    per_step = 2048
    x, _ = synth.make_patches(d, per_step * (args.steps + args.warmup), wl.n_terms, wl.sigma,
                              wl.seed + 1)
    for w in range(args.warmup):
        oracle.romp(x[w * per_step:(w + 1) * per_step], d, wl.R, wl.K)
    times = []
    for s in range(args.steps):
        lo = (args.warmup + s) * per_step
        t = time.perf_counter()
        oracle.romp(x[lo:lo + per_step], d, wl.R, wl.K)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = per_step * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "patches/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: P=1000000 n=102 (J=6, kmax=8) M=64 R=64 K=5",
                   "sample_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "patches/s", "cores": oracle.max_threads(),
                         "kind": "oracle",
                         "sample": f"{per_step} patches per step of the {WORKLOAD} workload"},
        "e2e": {"value": value, "unit": "patches/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def measure_fused(rsc, torch, dic, xd, K, stream, out, split_value, reps: int = 5) -> dict:
    """The same workload through rsc_encode_noalloc, whose FP16 path is one
    persistent kernel for all K steps (scoring, re-scoring, least squares and
    residual per 128-patch tile) plus the FP32 hand-off launch, timed with
    CUDA events on the launching stream beside the split path's value."""
    P = int(xd.shape[0])
    sh = int(stream.cuda_stream)
    args = (dic.handle, xd.data_ptr(), P, K, out["atom"].data_ptr(), out["angle_idx"].data_ptr(),
            out["angle"].data_ptr(), out["coef"].data_ptr(), out["resid_norm2"].data_ptr(), sh)
    for _ in range(2):
        assert rsc.rsc_encode_noalloc(*args) == rsc.RSC_OK
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        rsc.rsc_encode_noalloc(*args)
    ev[1].record(stream)
    stream.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    return {"value": P / (ms / 1e3), "unit": "patches/s", "ms_per_step": ms,
            "split_over_fused": split_value / (P / (ms / 1e3)),
            "note": "one persistent launch for all K steps (rsc_encode_noalloc) against the "
                    "headline's split path (a scoring and a refine launch per step, two streams)"}


def measure_projection(rsc, torch, dev, stream, reps: int = 5) -> dict:
    """rsc_project over one 2048 x 2048 image (4.15 M windows of 11 x 11,
    n = 102): windows/s from CUDA events on the launching stream; the
    contraction (2 x 97 x 108 algorithmic flops per window) runs on the
    tensor cores as three fp16 products, and the 432-byte output per window
    is the HBM side."""
    N, J, kmax = 11, 6, 8
    basis = rsc.Basis(N, J, kmax)
    rng = np.random.default_rng(20180614)
    img = torch.from_numpy(rng.standard_normal((2048, 2048)).astype(np.float32)).to(dev)
    with torch.cuda.stream(stream):
        out = rsc.project(basis, img, stream=stream)  # warm-up (and output size)
        del out
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(reps):
            out = rsc.project(basis, img, stream=stream)
            del out
        ev[1].record(stream)
        stream.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    P = (2048 - N + 1) ** 2
    nout = (kmax + 1) * J * 2
    flops = 2.0 * basis.npix * nout * P
    basis.close()
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    # algorithmic bytes per launch: the image read once, one packed
    # coefficient vector written per window
    algo = 2048 * 2048 * 4 + P * nout * 4
    return {"windows": P, "ms_per_call": ms, "windows_per_s": P / (ms / 1e3),
            "achieved_tflops": flops / (ms / 1e3) / 1e12,
            "path": "tcgen05, operands split into fp16 hi + lo (3 products)",
            "write_gbs": P * nout * 4 / (ms / 1e3) / 1e9,
            "roofline": {"kernel": "project_tc_kernel", "bound": "hbm",
                         "achieved": algo / (ms / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                         "frac": algo / (ms / 1e3) / 1e9 / hbm, "bytes_per_launch": algo,
                         "peak_note": "measured copy bandwidth"},
            "config": "one 2048x2048 image, N=11 (97 px), J=6, kmax=8, stride 1"}


def measure_roundtrip(rsc, torch, dev, stream, dic, codes, reps: int = 5) -> dict:
    """The way back on the benchmark's own codes (10^6 patches, M = 64,
    R = 64, K = 5): rsc_reconstruct (sum_i a_i S_i d_i, FP64 accumulation)
    and rsc_synthesize (Phi x_hat on the 11 x 11 basis, 97 pixels), patches/s
    of each from CUDA events on the launching stream."""
    N, J, kmax = 11, 6, 8
    basis = rsc.Basis(N, J, kmax)
    P = int(codes["atom"].shape[0])
    with torch.cuda.stream(stream):
        rec = rsc.reconstruct(dic, codes, stream=stream)
        pix = rsc.synthesize(basis, rec, stream=stream)
        del pix
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        for _ in range(reps):
            rec = rsc.reconstruct(dic, codes, stream=stream)
        ev[1].record(stream)
        for _ in range(reps):
            pix = rsc.synthesize(basis, rec, stream=stream)
            del pix
        ev[2].record(stream)
        stream.synchronize()
    ms_rec = ev[0].elapsed_time(ev[1]) / reps
    ms_syn = ev[1].elapsed_time(ev[2]) / reps
    npix = basis.npix
    basis.close()
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    K = int(codes["atom"].shape[1])
    nco = 9 * 6 * 2 * 4  # one patch's half-spectrum coefficients (float32)
    # algorithmic bytes: reconstruct reads the codes (atom, angle, FP64 weight)
    # and writes the coefficients; synthesize reads those and writes the pixels
    b_rec = P * (K * (4 + 4 + 8) + nco)
    b_syn = P * (nco + npix * 4)
    return {"patches": P, "reconstruct_ms": ms_rec, "reconstruct_patches_per_s": P / (ms_rec / 1e3),
            "synthesize_ms": ms_syn, "synthesize_patches_per_s": P / (ms_syn / 1e3),
            "roofline": {
                "reconstruct": {"bound": "hbm", "achieved": b_rec / (ms_rec / 1e3) / 1e9,
                                "peak": hbm, "unit": "GB/s",
                                "frac": b_rec / (ms_rec / 1e3) / 1e9 / hbm},
                "synthesize": {"bound": "hbm", "achieved": b_syn / (ms_syn / 1e3) / 1e9,
                               "peak": hbm, "unit": "GB/s",
                               "frac": b_syn / (ms_syn / 1e3) / 1e9 / hbm},
                "peak_note": "measured copy bandwidth; algorithmic bytes (codes or coefficients "
                             "in, coefficients or pixels out)"},
            "config": "omp_1m codes (M=64, R=64, K=5); synthesis on the 11x11 basis (97 px, n=102)"}


def measure_classify(rsc, torch, dev) -> dict:
    """rsc_classify_images, the coding stage of the paper's texture
    classifier: 8 line-texture images of 256 x 256 (484 k windows of 11 x 11)
    coded with each of C = 4 dictionaries (M = 64, R = 64, K = 5, FP16 path),
    labelled by least coding error and counted per image.  Host clock around
    the blocking call after a warm-up call."""
    N, J, kmax, M, R, K, C = 11, 6, 8, 64, 64, 5, 4
    imgs = [torch.from_numpy(synth.make_line_image(256, 256, 0.01, 20180630 + i)).to(dev)
            for i in range(8)]
    basis = rsc.Basis(N, J, kmax)
    dics = [rsc.Dictionary(torch.from_numpy(synth.make_dictionary(M, J, kmax, 20180640 + c)).to(dev), R)
            for c in range(C)]
    labels, hist = rsc.classify_images(dics, basis, imgs[:1], K, "f16")
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    labels, hist = rsc.classify_images(dics, basis, imgs, K, "f16")
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    P = int(labels.shape[0])
    for dd in dics:
        dd.close()
    basis.close()
    return {"windows": P, "dictionaries": C, "s": dt, "windows_per_s": P / dt,
            "patch_codings_per_s": P * C / dt,
            "config": "8 images 256x256, N=11, J=6, kmax=8; C=4 dictionaries M=64, R=64, K=5; f16"}


def measure_images_c2(rsc, torch, dev) -> dict:
    """rsc_encode_images at the image workload's coder sizes: 21 x 21 patches
    (349 px), J = 10, kmax = 12 (n = 250: tensor-core rows of 256 slots),
    M = 256, R = 128, K = 8, on 4 seeded N(0,1) images of sides 96, 160, 224,
    288 (line textures, synth.make_line_image, 0.01 lines per pixel), FP16
    path and FP32 path.  Host clock around the blocking call (projection +
    coding), after one warm-up call each; hand-offs of the FP16 path counted."""
    N, J, kmax, M, R, K = 21, 10, 12, 256, 128, 8
    imgs = [torch.from_numpy(synth.make_line_image(s_, s_, 0.01, 20180617 + s_)).to(dev)
            for s_ in (96, 160, 224, 288)]
    basis = rsc.Basis(N, J, kmax)
    dic = rsc.Dictionary(torch.from_numpy(synth.make_dictionary(M, J, kmax, 20180618)).to(dev), R)
    res = {"config": "N=21 (349 px), J=10, kmax=12 (n=250), M=256, R=128, K=8; "
                     "4 images, sides 96/160/224/288, projection included"}
    for prec in ("f16", "fp32"):
        rsc.encode_images(dic, basis, imgs[:1], K, prec)
        torch.cuda.synchronize(dev)
        rsc.rsc_dict_fallback_count(dic.handle)
        t0 = time.perf_counter()
        out = rsc.encode_images(dic, basis, imgs, K, prec)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        P = int(out["atom"].shape[0])
        res["patches"] = P
        res[prec] = {"s": dt, "patches_per_s": P / dt,
                     "handoffs": rsc.rsc_dict_fallback_count(dic.handle)}
    dic.close()
    basis.close()
    return res


def measure_rksvd(rsc, torch, dev, iters: int = 20) -> dict:
    """Rotational K-SVD on 200,000 patches drawn from 64 planted atoms
    (3 terms, noise 0.05): learn M = 128 atoms, R = 64, K = 5, from the first
    128 patches normalised; reports seconds per iteration, the MSE trajectory
    and the fraction of planted atoms recovered (|<S_theta d_m, t>| >= 0.99)."""
    from paper_1806_04374_gb300 import rksvd
    R, K, M, P = 64, 5, 128, 200_000
    d_true = synth.make_dictionary(64, 6, 8, 20180615)
    x, _ = synth.make_patches(d_true, P, 3, 0.05, 20180616)
    d0 = x[:M].astype(np.float64)
    d0[:, 0, :, 1] = 0.0
    d0 /= np.sqrt(synth.coef_norm2(d0))[:, None, None, None]
    xd = torch.from_numpy(x).to(dev)
    # warm-up on a slice (loads the library's and torch's kernels once)
    rksvd.learn(xd[:8192], torch.from_numpy(d0.astype(np.float32)).to(dev), R, K, iters=1,
                precision="f16")
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    d, _, hist = rksvd.learn(xd, torch.from_numpy(d0.astype(np.float32)).to(dev), R, K,
                             iters=iters, precision="f16")
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    mse = [h["mse"] for h in hist]
    # one coding pass and one update with the learned dictionary, timed apart
    import paper_1806_04374_gb300 as rsc_
    dic = rsc_.Dictionary(d, R)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    codes = rsc_.encode(dic, xd, K, "f16")
    ev[1].record()
    rsc_.ksvd_update(dic, xd, codes)
    ev[2].record()
    torch.cuda.synchronize(dev)
    dic.close()
    return {"patches": P, "atoms_learned": M, "atoms_planted": 64, "R": R, "K": K,
            "iterations": iters, "s_per_iteration": dt / (iters + 1),
            "encode_ms": ev[0].elapsed_time(ev[1]), "ksvd_update_ms": ev[1].elapsed_time(ev[2]),
            "mse_first": mse[0], "mse_last": mse[-1],
            "recovery_0.99": recovery(d.cpu().numpy(), d_true, R),
            "timing": "host clock around the whole loop (encode + update + sync per iteration)"}


def measure_c2_full(rsc, torch, dev, n_images: int = 512, precision: str = "f16") -> dict:
    """The 21 x 21-patch image workload at full size: 512 images of side
    U{64..512} (square line textures, synth.make_line_image, 0.01 lines per
    pixel, standing in for the rendered texture images), every
    stride-1 window (about 4.5 x 10^7 patches) projected (N = 21, J = 10,
    kmax = 12, n = 250) and coded (M = 256, R = 128, K = 8) in one
    rsc_encode_images call.  Host clock around the blocking call, after a
    warm-up call on two images."""
    N, J, kmax, M, R, K = 21, 10, 12, 256, 128, 8
    rng = np.random.default_rng(20180621)
    sides = rng.integers(64, 513, size=512)[:n_images]
    imgs = [torch.from_numpy(synth.make_line_image(int(s_), int(s_), 0.01, 20180621 + i)).to(dev)
            for i, s_ in enumerate(sides)]
    basis = rsc.Basis(N, J, kmax)
    dic = rsc.Dictionary(torch.from_numpy(synth.make_dictionary(M, J, kmax, 20180622)).to(dev), R)
    out = rsc.encode_images(dic, basis, imgs[:2], K, precision)
    del out
    torch.cuda.synchronize(dev)
    rsc.rsc_dict_fallback_count(dic.handle)
    t0 = time.perf_counter()
    out = rsc.encode_images(dic, basis, imgs, K, precision)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    P = int(out["atom"].shape[0])
    steps = float((out["atom"] >= 0).sum().item()) / P
    res = {"value": P / dt, "unit": "patches/s", "s": dt, "patches": P, "images": len(sides),
           "mean_steps_taken": steps, "handoffs": rsc.rsc_dict_fallback_count(dic.handle),
           "precision": precision,
           "config": f"{len(sides)} images, side U{{64..512}}, N=21 (349 px), J=10, "
                     "kmax=12 (n=250), M=256, R=128, K=8; projection + coding in one "
                     "rsc_encode_images call, host clock"}
    del out, imgs
    dic.close()
    basis.close()
    torch.cuda.empty_cache()
    return res


def run_c2(args) -> None:
    """``bench.py --c2``: the full-size image workload alone, as one JSON line."""
    import torch
    import paper_1806_04374_gb300 as rsc
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rsc.load_library()
    r = measure_c2_full(rsc, torch, dev, args.c2_images, args.precision)
    print(json.dumps({
        "metric": "image workload patches/s (projection + coding, one call)", "value": r["value"],
        "unit": "patches/s", "n_gpus": 1, "dtype": "f16" if args.precision == "f16" else "f32",
        "data": "synthetic", "s": r["s"], "patches": r["patches"],
        "mean_steps_taken": r["mean_steps_taken"], "handoffs": r["handoffs"],
        "config": {"workload": r["config"]}}))


SERVE_DIMS = dict(N=11, J=6, kmax=8, M=128, R=64, K=5)


def serving_pool(n: int, seed: int = 20180620):
    """Request images of the serving workload: n square line textures
    (synth.make_line_image) of side U{128..1024}."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(128, 1025, size=n)
    return [synth.make_line_image(int(s_), int(s_), 0.01, seed + i) for i, s_ in enumerate(sides)]


def offered(srv, pool, arrivals, which):
    """Submits pool[which[i]] at arrivals[i] seconds after the start (host
    clock) and waits for every request; returns the requests."""
    t0 = time.perf_counter()
    reqs = []
    for a_, q in zip(arrivals, which):
        dt = t0 + a_ - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        reqs.append(srv.submit(pool[q]))
    for r in reqs:
        r.wait()
    return reqs


def measure_serving(rsc, torch, dev, rates, seconds: float, n_pool: int,
                    mem_budget: int = 16 << 30, slots: int = 3) -> dict:
    """The serving workload through serve.Server: requests are images of side
    U{128..1024} coded at 11 x 11 (J = 6, kmax = 8) with a resident dictionary
    of M = 128 atoms, R = 64, K = 5, FP16 path, codes copied to the host.
    Runs: every pool image at t = 0 (capacity), then Poisson arrivals at each
    rate for `seconds`.  Latency = completion - submission (host clock)."""
    from paper_1806_04374_gb300 import serve
    dm = SERVE_DIMS
    basis = rsc.Basis(dm["N"], dm["J"], dm["kmax"])
    dic = rsc.Dictionary(torch.from_numpy(
        synth.make_dictionary(dm["M"], dm["J"], dm["kmax"], 20180619)).to(dev), dm["R"])
    pool = serving_pool(n_pool)
    windows = [(im.shape[0] - dm["N"] + 1) * (im.shape[1] - dm["N"] + 1) for im in pool]
    rng = np.random.default_rng(20180623)
    runs = []
    with serve.Server(dic, basis, dm["K"], "f16", mem_budget=mem_budget, slots=slots) as srv:
        for r in [srv.submit(pool[0]), srv.submit(pool[1])]:  # warm-up
            r.result()
        rsc.rsc_dict_fallback_count(dic.handle)
        cap = serve.latency_summary(offered(srv, pool, np.zeros(n_pool), np.arange(n_pool)))
        cap["arrivals"] = f"all {n_pool} pool images at t = 0 (capacity)"
        runs.append(cap)
        for rate in rates:
            n = max(8, int(rate * seconds))
            arr = np.cumsum(rng.exponential(1.0 / rate, size=n))
            reqs = offered(srv, pool, arr, rng.integers(0, n_pool, size=n))
            run = serve.latency_summary(reqs)
            run["arrivals"] = f"Poisson {rate:g} req/s for {seconds:g} s"
            run["offered_windows_per_s"] = rate * float(np.mean(windows))
            runs.append(run)
        handoffs = rsc.rsc_dict_fallback_count(dic.handle)
        peak = srv.peak_reserved
    dic.close()
    basis.close()
    return {"metric": "request latency p50/p99 and sustained patches/s (continuous batching)",
            "config": {"workload": "images side U{128..1024} (line textures), 11x11 windows "
                                   "(97 px), J=6, kmax=8, M=128, R=64, K=5, f16; codes copied "
                                   "to the host",
                       "server": f"serve.Server: {slots} slots (streams), device-memory budget "
                                 f"{mem_budget >> 30} GiB, batches up to 2^20 windows",
                       "pool_images": n_pool},
            "capacity_windows_per_s": runs[0]["windows_per_s"],
            "nominal_offered_200_req_per_s": 200 * float(np.mean(windows)),
            "peak_reserved_bytes": peak, "handoffs": handoffs, "runs": runs}


def run_serving(args) -> None:
    """`--serve`: the serving measurement alone, longer runs."""
    import torch
    import paper_1806_04374_gb300 as rsc
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rsc.load_library()
    res = measure_serving(rsc, torch, dev, args.rates, args.serve_seconds, args.serve_pool)
    res.update({"unit": "ms / patches/s", "n_gpus": 1, "dtype": "f16", "data": "synthetic"})
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="f16", choices=["fp32", "f16"])
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip timing the plain FP32 path beside the headline path")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--patches", type=int, default=None, help="override P (testing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the projection and rotational K-SVD measurements")
    ap.add_argument("--serve", action="store_true",
                    help="run the request-serving loop instead of the throughput bench")
    ap.add_argument("--rates", type=float, nargs="*", default=[200.0, 50.0])
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-pool", type=int, default=64)
    ap.add_argument("--c2", action="store_true",
                    help="code the full 21x21-patch image workload once instead")
    ap.add_argument("--c2-images", type=int, default=512,
                    help="with --c2: code only the first N of its 512 images (profiling)")
    args = ap.parse_args()
    if args.c2:
        run_c2(args)
        return
    if args.serve:
        run_serving(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    assert args.warmup >= 3 or args.patches is not None, "at least 3 warm-up steps"

    import torch
    import paper_1806_04374_gb300 as rsc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    wl = synth.WORKLOADS[WORKLOAD]
    P = wl.P if args.patches is None else args.patches
    d, x, wl = rank_inputs(rank, P)
    rsc.load_library()
    stream = torch.cuda.Stream(device=dev)
    dic = rsc.Dictionary(torch.from_numpy(d).to(dev), wl.R, stream=stream)
    xd = torch.from_numpy(x).to(dev)
    K = wl.K
    out = {
        "atom": torch.empty((P, K), dtype=torch.int32, device=dev),
        "angle_idx": torch.empty((P, K), dtype=torch.int32, device=dev),
        "angle": torch.empty((P, K), dtype=torch.float32, device=dev),
        "coef": torch.empty((P, K), dtype=torch.float64, device=dev),
        "resid_norm2": torch.empty((P,), dtype=torch.float32, device=dev),
    }
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed(precision: str, sample_clocks: bool, timing_mode: int = 1, steps: int = 0):
        """W warm-up steps, then K timed steps between barriers; returns the
        step times, the max-over-ranks total, clocks, hand-offs and the
        per-kernel event times recorded by the library (timing_mode 2: the
        FP16 path's two halves run one after the other)."""
        steps = steps or args.steps
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                rsc.encode(dic, xd, K, precision, stream=stream, out=out)
            stream.synchronize()
            if rsc.rsc_dict_check(dic.handle, int(stream.cuda_stream)) != 0:
                raise RuntimeError("device-side error during warm-up")
            rsc.rsc_dict_fallback_count(dic.handle)
            rsc.rsc_dict_set_timing(dic.handle, timing_mode)
            rsc.rsc_dict_timing(dic.handle)
            barrier()
            torch.cuda.synchronize(dev)
            clocks = ClockSampler(dev.index if dev.index is not None else 0) if sample_clocks else None
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
            if clocks:
                clocks.start()
            evs[0].record(stream)
            for s in range(steps):
                rsc.encode(dic, xd, K, precision, stream=stream, out=out)
                evs[s + 1].record(stream)
            stream.synchronize()
            torch.cuda.synchronize(dev)
            barrier()
            clk = clocks.stop() if clocks else None
        step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        total_ms = evs[0].elapsed_time(evs[-1])
        if rsc.rsc_dict_check(dic.handle, int(stream.cuda_stream)) != 0:
            raise RuntimeError("device-side error during the timed steps")
        kms, kn = rsc.rsc_dict_timing(dic.handle)
        rsc.rsc_dict_set_timing(dic.handle, False)
        handoffs = rsc.rsc_dict_fallback_count(dic.handle)
        if world > 1:
            tt = torch.tensor([total_ms], device=dev)
            torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
            total_ms = float(tt.item())
        return {"step_ms": step_ms, "total_ms": total_ms, "clocks": clk, "handoffs": handoffs,
                "kernel_ms": kms, "kernel_launches": kn}

    def sample_outputs() -> dict:
        """Outputs of patches PARITY_LO .. + PARITY_N of the last timed step."""
        lo, hi = PARITY_LO, min(PARITY_LO + PARITY_N, P)
        return {k: out[k][lo:hi].cpu().numpy() for k in ("atom", "angle_idx", "coef", "resid_norm2")}

    main_run = timed(args.precision, True)
    parity_outputs = {args.precision: sample_outputs()}
    tuning = rsc.rsc_dict_tuning(dic.handle, K)
    # the same steps with the two halves serialised: each kernel timed alone
    iso_run = timed(args.precision, False, timing_mode=2, steps=min(args.steps, 10))
    cmp_run = prune_run = None
    if args.precision != "fp32" and not args.no_fp32_compare:
        cmp_run = timed("fp32", False)
        parity_outputs["fp32"] = sample_outputs()
        # the FP32 path with the exact |G| bound pruning: the same codes
        prune_run = timed("fp32_prune", False, steps=min(args.steps, 5))
        pruned = sample_outputs()
        prune_run["same_codes"] = all(np.array_equal(pruned[k], parity_outputs["fp32"][k])
                                      for k in pruned)
    step_ms, total_ms, clk = main_run["step_ms"], main_run["total_ms"], main_run["clocks"]
    ms_per_step = total_ms / args.steps
    value = world * P * args.steps / (total_ms / 1e3)

    # end-to-end through the public host-buffer entry point (copies timed)
    xh = torch.from_numpy(x).pin_memory()
    oh = {
        "atom": torch.empty((P, K), dtype=torch.int32).pin_memory(),
        "angle_idx": torch.empty((P, K), dtype=torch.int32).pin_memory(),
        "angle": torch.empty((P, K), dtype=torch.float32).pin_memory(),
        "coef": torch.empty((P, K), dtype=torch.float64).pin_memory(),
        "resid_norm2": torch.empty((P,), dtype=torch.float32).pin_memory(),
    }
    for _ in range(2):
        rsc.encode_host(dic, xh, K, args.precision, out=oh)
    # every call blocks until its outputs are in the host buffers: host clock
    # per call; the value is the median call (p90 beside it)
    e2e_steps = max(10, min(args.steps, 20))
    e2e_s = []
    barrier()
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        rsc.encode_host(dic, xh, K, args.precision, out=oh)
        e2e_s.append(time.perf_counter() - t0)
    t_e2e = float(np.median(e2e_s))
    t_e2e90 = float(np.percentile(e2e_s, 90))
    if world > 1:
        tt = torch.tensor([t_e2e, t_e2e90], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_e2e, t_e2e90 = float(tt[0].item()), float(tt[1].item())
    h2d = int(xh.numel() * 4)
    d2h = int(sum(v.numel() * v.element_size() for v in oh.values()))

    if rank == 0:
        fl = algorithmic_flops_per_patch(wl)
        # dominant kernel: the scoring kernel of the path (phase 0 events); the
        # FP32 kernel runs all K steps in one launch, the tensor-core scoring
        # kernel one step per launch
        n_launch = max(main_run["kernel_launches"][0], 1)
        launch_s = main_run["kernel_ms"][0] / n_launch / 1e3
        flops_per_launch = fl["per_patch"] * P * args.steps / n_launch
        achieved = flops_per_launch / launch_s / 1e12
        sm_max = (clk or {}).get("sm_max_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        peaks = measured_peaks()
        if args.precision == "f16":
            kname, bound = "romp_score_kernel", "tensor"
            # dense fp16 and bf16 have the same nominal rate (ratio 1)
            peak = peaks.get("bf16_tflops") or 1900.0
            peak_note = ("dense fp16 = measured dense bf16 (burst) x nominal ratio 1"
                         if peaks.get("bf16_tflops") else "dense fp16, fallback 1.9 PFLOP/s")
        else:
            kname, bound = "romp_f32_kernel", "alu"
            peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
            peak_note = f"FP32 FMA: {nsm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_max:.0f} MHz"
        line = {
            "metric": METRIC,
            "value": value,
            "unit": "patches/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f16",
            "data": "synthetic",
            "config": {
                "workload": f"{WORKLOAD}: P={P} patches/GPU, n=102 (J=6, kmax=8), M=64, R=64, "
                            f"K=5, 3 planted atoms + noise 0.1",
                "path": (f"{args.precision} scoring ("
                         + ("tcgen05 tensor cores" if args.precision == "f16" else "CUDA cores")
                         + ") + double-float re-scoring + FP64 Cholesky"),
                "l2": "inputs (432 MB) larger than L2, no flush",
                "parallelism": f"dp{world} (patches sharded, no collective)",
                "tuning": dict(tuning, source={0: "default", 1: "autotuned table",
                                               2: "override"}[tuning["source"]]),
            },
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99)),
                           "unit": "one step (all patches of one GPU)"},
            "roofline": {
                "kernel": kname,
                "bound": bound,
                "achieved": achieved,
                "peak": peak,
                "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": (recorded_traffic(P * args.steps * wl.K / n_launch)
                            if args.precision == "f16" else None),
                "flops_per_patch": fl["per_patch"],
                "flops_convention": "(a) 2J(1+4kmax)M + (b) 2.5 R log2 R M per patch-step, x K",
                "kernel_ms": launch_s * 1e3,
                "flops_per_launch": flops_per_launch,
                "peak_note": peak_note,
                "limiter": ("measured: the MMA issue rate that two TMEM accumulator buffers "
                            "allow (100-134 cycles per MMA against 64 streamed) balanced with "
                            "the epilogue over all M R / 2 pair values; tensor pipe 25% busy"
                            if args.precision == "f16" else
                            "measured: issue-bound on the FP32 and ALU pipes"),
            },
            "hbm": {"algorithmic_bytes_per_patch": algorithmic_bytes_per_patch(wl),
                    "achieved_gbs": algorithmic_bytes_per_patch(wl) * P / launch_s / 1e9,
                    "peak_gbs": measured_peaks().get("hbm_gbs")},
            "e2e": {"value": world * P / t_e2e, "unit": "patches/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "calls": e2e_steps, "ms_per_call_median": 1e3 * t_e2e,
                    "ms_per_call_p90": 1e3 * t_e2e90,
                    "value_at_p90": world * P / t_e2e90,
                    "timing": "host clock around each blocking rsc_encode_host call (pinned "
                              "host buffers, H2D of x and D2H of every output inside); median "
                              "call"},
            "gpu_launches": kernel_launch_count(main_run["kernel_launches"], wl.K,
                                                args.precision),
            "handoffs": main_run["handoffs"],
            "kernel_ms_per_step": {"scoring": main_run["kernel_ms"][0] / args.steps,
                                   "fp32_handoff": main_run["kernel_ms"][1] / args.steps,
                                   "refine": main_run["kernel_ms"][2] / args.steps},
            "clocks": clk,
        }
        n_iso = max(iso_run["kernel_launches"][0], 1)
        iso_steps = min(args.steps, 10)
        iso_launch_s = iso_run["kernel_ms"][0] / n_iso / 1e3
        iso_flops = fl["per_patch"] * P * iso_steps / n_iso
        line["roofline_isolated"] = {
            "kernel": kname, "bound": bound, "achieved": iso_flops / iso_launch_s / 1e12,
            "peak": peak, "unit": "TFLOP/s",
            "frac": iso_flops / iso_launch_s / 1e12 / peak,
            "kernel_ms": iso_launch_s * 1e3, "flops_per_launch": iso_flops,
            "ms_per_step": iso_run["total_ms"] / iso_steps,
            "note": "same kernel, its launches timed with the two halves of the patches run one "
                    "after the other on one stream (the headline run overlaps them)"}
        if args.precision == "f16":
            # the other half of the path: init + refine launches (one step each),
            # timed alone in the serialised run (one group: P patches a launch)
            n_ref = max(iso_run["kernel_launches"][2], 1)
            ref_s = iso_run["kernel_ms"][2] / n_ref / 1e3
            row_len = 112 if 2 * wl.J * wl.kmax + wl.J <= 112 else 256
            ref_algo = (wl.kmax + 1) * wl.J * 2 * 4 + row_len * 2
            hbm = peaks.get("hbm_gbs") or 6800.0
            line["roofline_refine"] = {
                "kernel": "romp_refine_kernel (with romp_init_kernel)", "bound": "hbm",
                "achieved": ref_algo * P / ref_s / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": ref_algo * P / ref_s / 1e9 / hbm,
                "traffic": recorded_traffic(P, "romp_refine_kernel_omp_1m.md", REFINE_SOURCES),
                "bytes_per_launch": ref_algo * P, "bytes_per_patch": ref_algo,
                "kernel_ms": ref_s * 1e3,
                "peak_note": ("measured copy bandwidth" if peaks.get("hbm_gbs")
                              else "fallback 6.8 TB/s"),
                "note": "algorithmic bytes of a launch: read x, write the fp16 residual row; "
                        "latency-bound (one thread per patch), far below the HBM bound"}
            mf = mma_flops_per_patch(wl)
            mtf = mf * P * args.steps / n_launch / launch_s / 1e12
            line["mma_executed"] = {"flops_per_patch": mf, "tflops": mtf,
                                    "frac_of_peak": mtf / peak}
        if args.precision == "f16" and P <= (1 << 20) and world == 1:
            line["single_launch_fused"] = measure_fused(rsc, torch, dic, xd, K, stream, out,
                                                        value)
        if cmp_run is not None:
            v32 = world * P * args.steps / (cmp_run["total_ms"] / 1e3)
            # the FP32 kernel codes all K steps in one launch with the direct
            # angle transform: its own flops, (a) + M R (4 kmax + 1) per step
            alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
            f32_flops = wl.K * (fl["a"] + fl["b_direct"]) * P
            f32_s = cmp_run["total_ms"] / args.steps / 1e3
            line["fp32_path"] = {"value": v32, "unit": "patches/s",
                                 "ms_per_step": cmp_run["total_ms"] / args.steps,
                                 "speedup_of_headline": value / v32,
                                 "roofline": {
                                     "kernel": "romp_f32_kernel", "bound": "alu",
                                     "achieved": f32_flops / f32_s / 1e12, "peak": alu_peak,
                                     "unit": "TFLOP/s", "frac": f32_flops / f32_s / 1e12 / alu_peak,
                                     "flops_per_patch": wl.K * (fl["a"] + fl["b_direct"]),
                                     "flops_convention": "(a) 2J(1+4kmax)M + direct (b) M R (4kmax+1) "
                                                         "per patch-step, x K; one launch per step",
                                     "peak_note": f"FP32 FMA: {nsm} SMs x {FP32_LANES_PER_SM} lanes x "
                                                  f"2 x {sm_max:.0f} MHz"}}
        if prune_run is not None:
            nst = min(args.steps, 5)
            vp = world * P * nst / (prune_run["total_ms"] / 1e3)
            line["fp32_prune_path"] = {
                "value": vp, "unit": "patches/s", "ms_per_step": prune_run["total_ms"] / nst,
                "over_fp32_path": vp / v32,
                "same_codes_as_fp32_path": prune_run["same_codes"],
                "note": "RSC_FP32_PRUNE: the angle transform only for atoms whose exact bound "
                        "|G_0| + 2 sum_k |G_k| reaches the window of the running best; codes "
                        "compared on the sampled patches of the last timed step"}
        if not args.no_extras and world == 1:
            line["projection"] = measure_projection(rsc, torch, dev, stream)
            line["rksvd"] = measure_rksvd(rsc, torch, dev)
            line["images_c2_sizes"] = measure_images_c2(rsc, torch, dev)
            line["images_c2"] = measure_c2_full(rsc, torch, dev)
            line["roundtrip"] = measure_roundtrip(rsc, torch, dev, stream, dic, out)
            line["classify"] = measure_classify(rsc, torch, dev)
            line["serving"] = measure_serving(rsc, torch, dev, rates=[200.0, 50.0], seconds=3.0,
                                              n_pool=24)
            line["latency_ms"]["requests"] = {
                k: {"p50": r["p50_ms"], "p99": r["p99_ms"], "arrivals": r["arrivals"]}
                for k, r in zip(("capacity", "poisson_200", "poisson_50"),
                                line["serving"]["runs"])}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(d, x, wl, parity_outputs=parity_outputs)
            # the timed outputs against the oracle, on the same sample
            line["parity"] = dict(line["cpu_baseline"].pop("parity"),
                                  rule="selections equal where the oracle's top-two margin "
                                       "> 1e-6 relative; every pick within 1e-6 of its "
                                       "step's best on the forced path; weights within "
                                       "1e-3 (f16) / 1e-5 (fp32) relative",
                                  sample=f"patches {PARITY_LO}..{PARITY_LO + PARITY_N - 1} "
                                         "of the last timed step of each path")
        print(json.dumps(line))
    dic.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
