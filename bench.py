#!/usr/bin/env python
"""Benchmark: forward + adjoint evaluations per second of the coded-aperture
coherent-scatter operators on the paper-scale workload.

Workload (one "step" = one penalised EM-type iteration, i.e. one forward
model, one adjoint and the elementwise update, through caxsi_recon_step; the
likelihood, a monitoring value the update does not use, is not requested):
object 256 (y, across the fan) x 128 (x, along the beam) voxels x 128 q bins
(0.1-3.5 nm^-1), detector 256 x 64 pixels, 64 energy bins (20-100 keV),
tungsten-like spectrum, Bernoulli(0.5) mask with a 2-pixel feature, 10 seeded
phantoms (up to 8 ellipses with Bragg-peak profiles), Poisson counts with a
peak log-uniform in [1e2, 1e4].  Steps cycle through the phantoms, whose
states (10 x 16.8 MB) exceed the 129 MB L2 together with the operator tables.

Multi-GPU: the phantoms are independent problems; ranks take disjoint
phantoms and run without any data-path collective (weak scaling).

Reconstruction experiment (the "recon" key, rank 0): the wall time of the
plain FP32 iterations to a fixed NMSE, and the time of each alternative to
reach the same NMSE: bf16 / fp16 table paths, a 2048-sample u table (FP32 and
bf16), ordered subsets (8, 64 and 128 subsets, with the FP32 table operators and
with the direct ones, whose subset operators cost ~1/P of a full one), and the
learned warm start (a U-Net
trained here for --unet-steps objects, its training time reported apart).  The
"precision" key gives the throughput and the error (against the exact FP32
path) of the 16-bit contractions and of u tables of 1024-4096 samples.  The
"batch" key times the batched operators on 32 objects of uneven size against
one call per object: objects of uneven extent in x, z and q (one plan each, one
persistent launch per stage, direct FP32 path), and depth slabs of the
paper-scale object (table path).  The "symmetric_mask" key times the direct
operators for a mirror-symmetric mask with the mask factor computed online
against the same operators reading per-pair mask bits.  The "paper_table1" key
times one forward and one adjoint on the paper's own timing geometry (2048 x 1536
detector, 28 x 28 voxels), its MATLAB times beside them as context.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

METRIC = "fwd+adj evals/s"
UNIT = "evals/s"
N_PHANTOMS = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 500 steps of ~1.8 ms: the clock sampler (every 100 ms) sees the timed region ~9 times
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--path", default="table_fp32",
                    choices=["direct", "table_fp32", "table_bf16", "table_fp16"])
    ap.add_argument("--workload", choices=["paper", "tiny", "small"], default="paper")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-recon", action="store_true")
    ap.add_argument("--unet-steps", type=int, default=1000,
                    help="training steps (4 objects each) of the learned warm start in the recon experiments "
                         "(0: skip)")
    return ap.parse_args()


def geometry(name):
    if name == "paper":
        return synth.paper_geometry()
    if name == "small":
        # the paper-scale detector, q grid and spectrum with 16 voxels along the beam
        # (for profiler captures: same per-pair work, 1/8 of the pairs)
        return synth.paper_geometry().with_(X=16, dx=4.375)
    return synth.tiny_geometry()


def workload_desc(g, name):
    return (f"{name} fan-beam coded-aperture scatter: "
            f"object {g.J}(y) x {g.X}(x) voxels x {g.Q} q bins ({g.q_min}-{g.q_max} nm^-1), "
            f"detector {g.N}x{g.M} pixels, {g.K} energy bins ({g.E_min:g}-{g.E_max:g} keV); "
            f"penalised EM step (A, ratio, A^T, update) over {N_PHANTOMS} seeded phantoms")


def mask_seed(name):
    return synth.TINY_MASK_SEED if name == "tiny" else synth.PAPER_MASK_SEED


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [s for (t, s) in self.samples if t0 <= t <= t1] or [s for _, s in self.samples]
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_query_id(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


# ---------------------------------------------------------------------------
# roofline bookkeeping
# ---------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def operator_alg_bytes(g):
    """Algorithmic HBM bytes of one application of A (or of A^T): the object f (4 R Q B), the detector image (4 M N B) and the
    per-offset geometry table streamed once (one 16-byte entry per scatter vector
    (i, d, m), X M (N + rho_y (J - 1)) entries).  The design's own records and
    knot rows are not counted: they are this implementation's choice of what to
    precompute (the paper's online/offline trade-off), not the operator's need."""
    nd = g.N + g.rho_y * (g.J - 1)
    return 4.0 * g.X * g.J * g.Q + 4.0 * g.M * g.N + 16.0 * g.X * g.M * nd


def operator_alg_flops(g, open_pairs):
    """The per-energy flop count of one application of A (or A^T) done by direct
    summation (Algorithm 1 / 3): per open (voxel, pixel) pair, K energy terms of
    8 flop plus 30 flop of scatter geometry."""
    return open_pairs * (8.0 * g.K + 30.0)


def kernel_work(name, g, info, path, nsm):
    """Work of one launch of the named kernel on this design's basis: (unit,
    amount, bound)  (the operator's own algorithmic bytes are operator_alg_bytes).

    The amounts are the bytes or flops this design streams or issues: 12-byte
    records, one knot-table row per voxel, partial images; 2 R B Q flop per
    product pass of a contraction.  They are not the operator's algorithmic
    bytes (operator_alg_bytes), which are far fewer: the records and knot rows
    are precomputed state this design chose to stream."""
    open_pairs = info["n_open_pairs"]
    B = info["n_breakpoints"]
    Bp = (B + 1 + 7) // 8 * 8
    n_rec = info["n_records"]
    R, npix = g.X * g.J, g.M * g.N
    chunks = min(2 * nsm, R)
    if name in ("fwd_direct", "adj_direct"):
        # per open (voxel, pixel) pair: K energy terms of 8 flop (tau FMA, floor,
        # fraction, lerp FMA, accumulate FMA) plus 30 flop of scatter geometry
        return "TFLOP/s", open_pairs * (8.0 * g.K + 30.0), "alu"
    sym_chunks = min(nsm, g.X * (g.J // 2))   # one block per SM over the voxel pairs
    if name == "sym_pairs_fwd":
        # one 21-byte record per voxel pair and quadrant pixel (8 pairs), two W rows per
        # voxel pair (FP32; bf16 on the bf16 path), one partial image per block
        recs = (g.X * (g.J // 2)) * ((g.M // 2) * (g.N // 2))
        wb = 2.0 if path == "table_bf16" else 4.0
        return "GB/s", 21.0 * recs + wb * R * Bp + 4.0 * sym_chunks * npix, "hbm"
    if name == "sym_pairs_adj":
        # records of a 4-byte key and two weights (FP32; bf16 on the bf16 path), up to
        # 4 pairs each, one V row per voxel, the input image once per block
        vb = {"table_fp32": 4.0, "table_bf16": 2.0, "table_fp16": 2.0}[path]
        rb = 8.0 if path == "table_bf16" else 12.0
        return "GB/s", rb * info["n_sym_records"] + vb * R * B + 4.0 * sym_chunks * npix, "hbm"
    if name == "rec_pairs_fwd":
        # 12-byte records, one W row per voxel, one partial image per block
        return "GB/s", 12.0 * n_rec + 4.0 * R * Bp + 4.0 * chunks * npix, "hbm"
    if name == "rec_pairs_adj":
        vb = {"table_fp32": 4.0, "table_bf16": 2.0, "table_fp16": 2.0}[path]
        return "GB/s", 12.0 * n_rec + vb * R * B + 4.0 * chunks * npix, "hbm"
    if name.startswith("tc_gemm_fwd"):
        # the forward contraction is bound by writing the FP32 knot table
        ab = 8.0 if name.endswith("3xtf32") else 2.0
        return "GB/s", 4.0 * R * B + ab * R * g.Q, "hbm"
    if name.startswith("tc_gemm_adj"):
        passes = 3 if name.endswith("3xtf32") else 1
        return "TFLOP/s", passes * 2.0 * R * B * g.Q, "tensor"
    return None, None, None


def roofline_line(dom, avg_s, design, g, info, path, kernels, steps, peaks, peak_kind, nsm):
    """The bench line's roofline object.  `frac` is on the operator's algorithmic
    basis: for the table paths the operator's algorithmic HBM bytes (operator_alg_bytes)
    over the dominant kernel's average launch time; for the direct path its FP32
    flops over the FP32 SIMT peak (the two coincide with `design` there).  The
    design's own basis is kept under `design`.  Per step (one A and one A^T) the
    DRAM traffic of the step's kernels that have a current ncu figure is set
    against the two operators' algorithmic bytes."""
    hbm = float(peaks["hbm_gbs"])
    if design["bound"] == "alu":
        line = {"bound": "alu", "kernel": dom, "achieved": design["achieved"], "peak": design["peak"],
                "unit": "TFLOP/s", "frac": design["frac"], "traffic": traffic_for(dom, path),
                "peak_source": design["peak_source"],
                "alg_work_per_launch": design["work_per_launch"],
                "basis": "operator: K energy terms x 8 flop + 30 flop per open pair"}
    else:
        alg = operator_alg_bytes(g)
        achieved = alg / avg_s / 1e9
        line = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic_for(dom, path),
                "peak_source": f"HBM copy bandwidth, {peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "alg_bytes": alg, "alg_frac": achieved / hbm,
                "basis": "operator: f + detector image + per-offset geometry table of one application "
                         "of A or A^T, over the dominant kernel's time"}
    line["design"] = design
    # per step: DRAM traffic of the step's kernels (ncu, current sources only) against 2 operators
    step_traffic, covered = 0.0, []
    for k, st in kernels.items():
        t = traffic_for(k, path)
        if t is not None:
            step_traffic += t * st["launches"] / max(steps, 1)
            covered.append(k)
    if covered:
        alg_step = 2.0 * operator_alg_bytes(g)
        line["step"] = {"traffic_bytes": step_traffic, "alg_bytes": alg_step,
                        "traffic_over_alg": step_traffic / alg_step, "kernels_with_traffic": sorted(covered)}
    # the per-energy flops of A + A^T by direct summation over the step's kernel time: above the FP32
    # SIMT peak when the path does not do the per-energy work (the table paths)
    step_s = sum(st["total_ms"] for st in kernels.values()) / 1e3 / max(steps, 1)
    if step_s > 0 and info.get("n_open_pairs"):
        fp32 = nsm * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        eq = 2.0 * operator_alg_flops(g, info["n_open_pairs"]) / step_s / 1e12
        line["alu_equivalent"] = {"tflops": eq, "fp32_simt_peak": fp32, "frac": eq / fp32,
                                  "note": "per-energy flops of one A + one A^T by direct summation over the "
                                          "step's kernel time; not work this path performs"}
    return line


def traffic_for(name, path):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        ent = d.get(name)
        if not ent:
            return None
        src = os.path.join(ROOT, "paper_1603_06400_gb300", "csrc", ent["source"])
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return ent["dram_bytes_per_launch"] if sha == ent["source_sha"] else None
    except Exception:
        return None


# ---------------------------------------------------------------------------
# CPU oracle timings (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_eval_seconds(g, phi, mask, f, w, n_pix, n_vox, seed, nthreads=0):
    import oracle
    rng = np.random.default_rng(seed)
    pix = rng.choice(g.M * g.N, size=min(n_pix, g.M * g.N), replace=False)
    vox = rng.choice(g.X * g.J, size=min(n_vox, g.X * g.J), replace=False)
    t0 = time.perf_counter()
    oracle.forward_pixels(g, phi, mask, f, pix, nthreads=nthreads)
    t1 = time.perf_counter()
    oracle.adjoint_voxels(g, phi, mask, w, vox, nthreads=nthreads)
    t2 = time.perf_counter()
    per_eval = (t1 - t0) * (g.M * g.N / len(pix)) + (t2 - t1) * (g.X * g.J / len(vox))
    return per_eval, (t2 - t0), len(pix), len(vox)


def cpu_inputs(g):
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, mask_seed("tiny" if g.M == 16 else "paper"))
    f = synth.phantom(g, 0)
    w = synth.uniform_random((g.M, g.N), 1)
    return phi, mask, f, w


def cpu_baseline(g, target_s=15.0, single_s=5.0):
    import oracle
    phi, mask, f, w = cpu_inputs(g)
    cores = oracle.max_threads()   # read first: a thread count given to the oracle persists

    def sampled(target, nthreads, seed):
        # size the sample from a short probe so that it takes ~target seconds
        _, took, _, _ = oracle_eval_seconds(g, phi, mask, f, w, 32, 32, 99, nthreads)
        scale = max(1.0, target / max(took, 1e-3))
        n_pix = int(min(g.M * g.N, 32 * scale))
        n_vox = int(min(g.X * g.J, 32 * scale))
        return oracle_eval_seconds(g, phi, mask, f, w, n_pix, n_vox, seed, nthreads)

    per1, took1, npx1, nvx1 = sampled(single_s, 1, 8)
    per_eval, took, npx, nvx = sampled(target_s, cores, 7)
    return {"value": 1.0 / per_eval, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"FP64 direct-summation oracle on {npx} sampled pixels (forward) and "
                      f"{nvx} sampled voxels (adjoint) of one phantom, {took:.1f} s wall, "
                      f"scaled to one full forward + adjoint",
            "single_thread": {"value": 1.0 / per1, "unit": UNIT, "cores": 1,
                              "sample": f"{npx1} pixels and {nvx1} voxels, {took1:.1f} s wall, scaled"}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    g = geometry(args.workload)
    phi, mask, f, w = cpu_inputs(g)
    # per step a bounded sample of one forward + adjoint: ~1 s of CPU work, less when
    # there are many steps, so that the whole run takes about two minutes at most
    per_step = min(1.0, 120.0 / max(1, args.warmup + args.steps))
    probe, took, _, _ = oracle_eval_seconds(g, phi, mask, f, w, 16, 16, 1)
    scale = max(1.0, per_step / max(took, 1e-3))
    n = int(min(g.M * g.N, 16 * scale))
    times = []
    for s in range(args.warmup + args.steps):
        per_eval, _, npx, nvx = oracle_eval_seconds(g, phi, mask, f, w, n, n, 1000 + s)
        if s >= args.warmup:
            times.append(per_eval)
    mean = float(np.mean(times))
    value = 1.0 / mean
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(g, args.workload), "path": "oracle",
                   "l2": "host CPU"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: FP64 oracle forward on {npx} sampled pixels and "
                                   f"adjoint on {nvx} sampled voxels, scaled to one full "
                                   f"forward + adjoint"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (independent phantoms per rank, no data-path collective)
# ---------------------------------------------------------------------------

def rank_phantoms(rank, world, n=N_PHANTOMS):
    """Phantoms owned by a rank: disjoint across ranks and covering all n when
    world <= n; with more ranks than phantoms the extra ranks repeat phantoms."""
    mine = [p for p in range(n) if p % world == rank]
    return mine or [rank % n]


def max_over_ranks(value, dist, device=None):
    """Maximum of a per-rank scalar (the timing rule: the slowest rank counts)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# reconstruction: time to the plain FP32 method's final NMSE
# ---------------------------------------------------------------------------

def recon_experiment(caxsi, plan, g, dev, phantom, iters=100, max_iters=300, warm=None,
                     make_plan=None):
    """Penalised EM (Huber on the spatial neighbours) on one phantom: the plain
    FP32 table path for `iters` iterations gives the target NMSE; each
    reduced-precision path (16-bit contractions; a 2048-sample u table, in FP32
    and bf16, on a plan from make_plan(2048)), and the ordered-subset algorithm
    with 8 and 64 subsets (FP32 table path, penalty beta / P per step), is run
    until it reaches that NMSE.  Device time of the iterations only (CUDA
    events); NMSE = |f - f_true|^2 / |f_true|^2."""
    import torch
    f_true = torch.tensor(synth.phantom(g, phantom), dtype=torch.float32, device=dev)
    P = caxsi.PATHS
    mean = plan.forward(f_true, path=P["table_fp32"])
    peak = synth.log_uniform_peak(phantom)
    y = torch.tensor(synth.poisson_counts((mean * (peak / mean.max())).cpu().numpy().astype(np.float64),
                                          100 + phantom), dtype=torch.float32, device=dev)
    scale = peak / float(mean.max())     # counts per unit of A f_true
    f_ref = f_true * scale               # the object in count units
    b1 = plan.adjoint(torch.ones((g.M, g.N), device=dev), path=P["table_fp32"])
    f_init = float(y.sum() / b1.sum())
    beta = 1e-3 * float(y.sum()) / (g.X * g.J * g.Q)
    delta = 0.01 * f_init
    nref = float(torch.sum(f_ref.double() ** 2))

    def run(path, target=None, n=iters, on=None):
        on = on or plan
        f = torch.full((g.X, g.J, g.Q), f_init, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        total, hist = 0.0, []
        for it in range(n):
            e0.record()
            on.recon_step(y, f, beta=beta, delta=delta, path=P[path])
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1) / 1e3
            nmse = float(torch.sum((f.double() - f_ref.double()) ** 2)) / nref
            hist.append(nmse)
            if target is not None and nmse <= target:
                return {"iterations": it + 1, "seconds": total, "nmse": nmse, "reached": True}
        out = {"iterations": n, "seconds": total, "nmse": hist[-1]}
        if target is not None:
            out["reached"] = False
        return out

    plain = run("table_fp32")
    res = {"phantom": phantom, "peak_counts": peak, "beta": beta, "delta": delta,
           "plain_fp32": plain, "target_nmse": plain["nmse"]}
    for path in ("table_bf16", "table_fp16"):
        r = run(path, target=plain["nmse"], n=max_iters)
        r["speedup_vs_plain"] = plain["seconds"] / r["seconds"] if r["reached"] else None
        res[path] = r
    if make_plan is not None:
        # the sampled table is another operator: its sensitivity b1 and first
        # iteration are computed once before the timed iterations
        sp = make_plan(2048)
        for path in ("table_fp32", "table_bf16"):
            sp.recon_step(y, torch.full((g.X, g.J, g.Q), f_init, device=dev), beta=beta, delta=delta,
                          path=P[path])
            r = run(path, target=plain["nmse"], n=max_iters, on=sp)
            r["speedup_vs_plain"] = plain["seconds"] / r["seconds"] if r["reached"] else None
            res["utable_2048_" + path.split("_")[1]] = r
        sp.close()
    # ordered subsets (Algorithm 5): passes over the P subsets until the plain
    # target NMSE; the subset sensitivities b1_p are precomputed outside the
    # timing, as b1 is for the plain iterations.  On the direct path a subset
    # operator evaluates only its pixels' pairs (cost ~ 1/P of a full one); on
    # the FP32 table path it still pays the whole-object q contractions.
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rho_z, sigma_y, max_passes in ((8, 2, 30), (8, 16, 12), (16, 16, 12)):
        plan.set_subsets(caxsi.os_partition(g.M, g.N, g.rho_y, rho_z, sigma_y))
        n_sub = plan.n_subsets
        for path, tag in (("table_fp32", ""), ("direct", "_direct")):
            plan.os_pass(y, torch.full((g.X, g.J, g.Q), f_init, device=dev), beta=beta, delta=delta,
                         path=P[path])
            f = torch.full((g.X, g.J, g.Q), f_init, device=dev)
            total, r = 0.0, None
            for k in range(max_passes):
                e0.record()
                plan.os_pass(y, f, beta=beta, delta=delta, path=P[path])
                e1.record()
                torch.cuda.synchronize()
                total += e0.elapsed_time(e1) / 1e3
                nmse = float(torch.sum((f.double() - f_ref.double()) ** 2)) / nref
                r = {"subsets": n_sub, "rho_z": rho_z, "sigma_y": sigma_y, "path": path, "passes": k + 1,
                     "sub_iterations": (k + 1) * n_sub, "seconds": total, "nmse": nmse,
                     "reached": nmse <= plain["nmse"]}
                if r["reached"]:
                    break
            r["speedup_vs_plain"] = plain["seconds"] / r["seconds"] if r["reached"] else None
            res[f"os_em_{n_sub}{tag}"] = r
    res["learned"] = learned_experiment(plan, g, y, f_ref, plain, warm) if warm is not None else None
    return res


def recon_seeds(caxsi, plan, g, dev, warm, seeds=range(N_PHANTOMS), iters=100, max_iters=300):
    """Penalised EM on each benchmark phantom (seeds 0-9, peaks log-uniform in
    [1e2, 1e4]): `iters` plain FP32 iterations give the target NMSE; then the
    time each alternative needs to reach it: the learned warm start (first
    iterate + network + EM-type iterations), bf16 contractions, and ordered
    subsets (128 subsets, FP32 table path).  Device time of the iterations only;
    per-seed entries and the median and worst speedups."""
    import torch
    from paper_1603_06400_gb300 import warmstart  # noqa: F401
    P = caxsi.PATHS
    b1 = plan.adjoint(torch.ones((g.M, g.N), device=dev), path=P["table_fp32"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the partition, its grouped records and the subset sensitivities are set up once,
    # outside the timing (as b1 is for the plain iterations)
    plan.set_subsets(caxsi.os_partition(g.M, g.N, g.rho_y, 16, 16))
    plan.os_pass(torch.zeros((g.M, g.N), device=dev), torch.ones((g.X, g.J, g.Q), device=dev),
                 path=P["table_fp32"])
    per = []
    for p in seeds:
        f_true = torch.tensor(synth.phantom(g, p), dtype=torch.float32, device=dev)
        mean = plan.forward(f_true, path=P["table_fp32"])
        peak = synth.log_uniform_peak(p)
        y = torch.tensor(synth.poisson_counts((mean * (peak / mean.max())).cpu().numpy().astype(np.float64),
                                              100 + p), dtype=torch.float32, device=dev)
        f_ref = f_true * (peak / float(mean.max()))
        f_init = float(y.sum() / b1.sum())
        beta = 1e-3 * float(y.sum()) / (g.X * g.J * g.Q)
        delta = 0.01 * f_init
        nref = float(torch.sum(f_ref.double() ** 2))
        nmse = lambda f: float(torch.sum((f.double() - f_ref.double()) ** 2)) / nref

        def timed(fn):
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 1e3

        def until(f, step, target, cap):
            total, n = 0.0, 0
            cur = nmse(f)
            while (target is None or cur > target) and n < cap:
                total += timed(lambda: step(f))
                n += 1
                cur = nmse(f)
            return {"iterations": n, "seconds": total, "nmse": cur,
                    "reached": target is None or cur <= target}
        f_plain = torch.full((g.X, g.J, g.Q), f_init, device=dev)
        step_plain = lambda x: plan.recon_step(y, x, beta=beta, delta=delta, path=P["table_fp32"])
        plain = until(f_plain, step_plain, None, iters)
        target = plain["nmse"]
        ent = {"phantom": p, "peak_counts": peak, "plain_fp32": plain}
        f = torch.full((g.X, g.J, g.Q), f_init, device=dev)
        ent["table_bf16"] = until(f, lambda x: plan.recon_step(y, x, beta=beta, delta=delta,
                                                               path=P["table_bf16"]), target, max_iters)
        f = torch.full((g.X, g.J, g.Q), f_init, device=dev)
        r = until(f, lambda x: plan.os_pass(y, x, beta=beta, delta=delta, path=P["table_fp32"]), target, 12)
        r["passes"] = r.pop("iterations")
        r["subsets"] = plan.n_subsets
        ent["os_em_128"] = r
        if warm is not None:
            net, maker, _ = warm
            box = {}

            def start():
                f1, *_ = maker.make(0, y=y, f_ref=f_ref)
                sc = float(f1.mean())
                box["f"] = net.predict(f1, sc, 1e-3 * sc)
            t0 = timed(start)
            f0_nmse = nmse(box["f"])
            r = until(box["f"], step_plain, target, max_iters)
            r["seconds"] += t0
            r["first_iterate_and_inference_seconds"] = t0
            r["f0_nmse"] = f0_nmse
            ent["learned"] = r
            # a stronger comparison: the plain iterations (continued past the target)
            # needed to reach the network's starting image f^0
            extra = until(f_plain, step_plain, f0_nmse, 300)
            ent["plain_to_learned_f0"] = {"iterations": iters + extra["iterations"],
                                          "seconds": plain["seconds"] + extra["seconds"],
                                          "reached": extra["reached"], "nmse": extra["nmse"]}
        for k in ("table_bf16", "os_em_128", "learned"):
            if k in ent:
                ent[k]["speedup_vs_plain"] = plain["seconds"] / ent[k]["seconds"] if ent[k]["reached"] else None
        per.append(ent)
    summary = {}
    for k in ("table_bf16", "os_em_128", "learned"):
        sp = [e[k]["speedup_vs_plain"] for e in per if k in e]
        if sp:
            ok = [v for v in sp if v is not None]
            summary[k] = {"reached": f"{len(ok)}/{len(sp)}",
                          "median_speedup": float(np.median(ok)) if ok else None,
                          "worst_speedup": float(min(ok)) if len(ok) == len(sp) else None,
                          "median_time_fraction_of_plain": float(np.median([1.0 / v for v in ok])) if ok else None}
    p2 = [e["plain_to_learned_f0"] for e in per if "plain_to_learned_f0" in e]
    if p2:
        summary["plain_iterations_to_learned_f0"] = {
            "reached": f"{sum(1 for e in p2 if e['reached'])}/{len(p2)}",
            "median_iterations": float(np.median([e["iterations"] for e in p2])),
            "note": "plain FP32 iterations from the flat start needed to reach the NMSE of the network's f^0 "
                    "(capped at the plain run plus 300)"}
    summary["plain_fp32_final_nmse"] = {"median": float(np.median([e["plain_fp32"]["nmse"] for e in per])),
                                        "worst": float(max(e["plain_fp32"]["nmse"] for e in per))}
    return {"iterations": iters, "per_phantom": per, "summary": summary}


def train_warm_start(plan, g, steps, batch=4):
    """Train the warm-start U-Net (hand-written kernels, bf16 tensor-core
    convolutions) on steps x batch objects of the input recipe (seeds 100000+,
    disjoint from the benchmark phantoms 0-9), counts drawn on the device; the
    loss curve is the mean over 8 held-out objects (seeds 150000+).  Returns
    (net, maker, record); the training time is reported apart (done once)."""
    import torch
    from paper_1603_06400_gb300 import warmstart
    maker = warmstart.PairMaker(plan, g)
    net = warmstart.UNet(channels=g.Q, base=32, seed=0)
    torch.cuda.synchronize()
    t0 = time.time()
    losses = warmstart.train(net, maker, steps, lr=1e-3, batch=batch, log=max(1, steps // 10),
                             heldout_seeds=range(150000, 150008))
    torch.cuda.synchronize()
    rec = {"train_steps": steps, "objects_per_step": batch, "train_objects": steps * batch,
           "train_seconds": time.time() - t0, "heldout_objects": 8,
           "loss_curve": [{"step": k, "train_batch": a, "heldout_mean": b} for k, a, b in losses]}
    return net, maker, rec


def learned_experiment(plan, g, y, f_ref, plain, warm):
    """The learned warm start on one phantom, timed: the first EM-type iterate
    from the flat start, the network's f^0, and EM-type iterations from f^0 until
    the plain FP32 target NMSE; then the step scalings learned through 10
    unrolled iterations."""
    import torch
    from paper_1603_06400_gb300 import warmstart
    P = caxsi_paths()
    net, maker, rec = warm
    train_s = rec["train_seconds"]
    nref = float(torch.sum(f_ref.double() ** 2))
    nmse = lambda f: float(torch.sum((f.double() - f_ref.double()) ** 2)) / nref
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    f1, _, _, beta, delta, f_init = maker.make(0, y=y, f_ref=f_ref)
    s = float(f1.mean())
    f = net.predict(f1, s, 1e-3 * s)
    e1.record()
    torch.cuda.synchronize()
    start_s = e0.elapsed_time(e1) / 1e3
    total, n_em = start_s, 0
    cur = nmse(f)
    f0_nmse = cur
    while cur > plain["nmse"] and n_em < 300:
        e0.record()
        plan.recon_step(y, f, beta=beta, delta=delta, path=P["table_fp32"])
        e1.record()
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1) / 1e3
        n_em += 1
        cur = nmse(f)
    reached = cur <= plain["nmse"]
    # the network's second output: per-iteration step scalings of the iterations
    # that follow, learned through 10 unrolled iterations; compared with plain
    # iterations over the same 10 steps from the same f^0
    torch.cuda.synchronize()
    t0 = time.time()
    relax = warmstart.train_step_scalings(net, maker, T=10, samples=40)
    torch.cuda.synchronize()
    relax_s = time.time() - t0
    f0 = net.predict(f1, s, 1e-3 * s)
    ones = torch.ones(10, device="cuda")
    after_plain = nmse(warmstart.relaxed_iterations(maker, y, f0, ones, beta, delta, 1e-3 * s))
    after_learned = nmse(warmstart.relaxed_iterations(maker, y, f0, relax, beta, delta, 1e-3 * s))
    scalings = {"values": [round(float(v), 4) for v in relax], "train_objects": 40, "train_seconds": relax_s,
                "nmse_after_10_plain_from_f0": after_plain, "nmse_after_10_scaled_from_f0": after_learned}
    return {"step_scalings": scalings, "network": "U-Net, 4 levels, base width 32, 3x3 convs (bf16 tensor-core GEMMs, FP32 accumulation)",
            "training": rec, "train_seconds": train_s,
            "first_iterate_and_inference_seconds": start_s, "f0_nmse": f0_nmse, "em_iterations": n_em,
            "seconds": total, "nmse": cur, "reached": reached,
            "speedup_vs_plain": plain["seconds"] / total if reached else None}


def batch_experiment(plan, g, n_objects=32, reps=5):
    """Batched operators (caxsi_forward_batch / caxsi_adjoint_batch) over
    n_objects objects of uneven size: seeded depth slabs [v0, v1) of the voxel
    index, extents uniform in [R/8, R].  Timed (CUDA events, after warm-up): one
    batched forward + adjoint of all objects, against the same objects one call
    each (full-size operators on the object's f with zeros outside its slab)."""
    import torch
    from paper_1603_06400_gb300 import caxsi
    R = g.X * g.J
    rng = np.random.default_rng(2024)
    ranges = []
    for _ in range(n_objects):
        n = int(rng.integers(R // 8, R + 1))
        v0 = int(rng.integers(0, R - n + 1))
        ranges.append((v0, v0 + n))
    ranges = np.array(ranges, np.int32)
    f = torch.rand((n_objects, g.X, g.J, g.Q), device="cuda")
    w = torch.rand((n_objects, g.M, g.N), device="cuda") + 0.5
    fm = torch.zeros_like(f)
    for b, (v0, v1) in enumerate(ranges):
        fm[b].view(R, g.Q)[v0:v1] = f[b].view(R, g.Q)[v0:v1]
    P = caxsi.PATHS["table_fp32"]

    def batched():
        plan.forward_batch(f, ranges=ranges)
        plan.adjoint_batch(w, ranges=ranges)

    def single():
        for b in range(n_objects):
            plan.forward(fm[b], path=P)
            plan.adjoint(w[b], path=P)
    out = {"objects": n_objects, "voxel_rows": int(sum(v1 - v0 for v0, v1 in ranges)),
           "extents": "uniform in [R/8, R], R = %d voxels" % R}
    for name, fn in (("batched", batched), ("single_calls", single)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        out[name] = {"seconds": sec, "objects_per_s": n_objects / sec}
    out["speedup"] = out["single_calls"]["seconds"] / out["batched"]["seconds"]
    return out


def uneven_batch_experiment(dev, n_objects=32, reps=3):
    """Objects of uneven size (x across the fan 64-256, z along the beam 32-128,
    q bins 64-128; seeded, synth.uneven_sizes) on the paper-scale detector,
    spectrum and mask, one plan each, as one caxsi_multi set: one forward + one
    adjoint of all objects (one persistent launch each, direct FP32 path), timed
    with CUDA events after a warm-up, against the same objects one
    caxsi_forward / caxsi_adjoint call each (the same arithmetic; results equal
    bit for bit)."""
    import torch
    from paper_1603_06400_gb300 import caxsi
    base = synth.paper_geometry()
    phi = synth.tungsten_spectrum(base)
    mask = synth.random_mask(base, synth.PAPER_MASK_SEED)
    sizes = synth.uneven_sizes(n_objects, 2024)
    geos = [synth.uneven_object_geometry(X, J, Q) for X, J, Q in sizes]
    plans = [caxsi.Plan(g, phi, mask) for g in geos]
    multi = caxsi.Multi(plans)
    fs = [synth.phantom_torch(g, 300 + k, dev) for k, g in enumerate(geos)]
    gen = torch.Generator(device=dev).manual_seed(5)
    ws = [torch.rand((g.M, g.N), device=dev, generator=gen) + 0.5 for g in geos]
    f, w = multi.pack_f(fs), multi.pack_g(ws)
    gm = torch.empty(multi.g_len, device=dev)
    fm = torch.empty(multi.f_len, device=dev)
    D = caxsi.PATH_DIRECT

    def batched():
        multi.forward(f, out=gm)
        multi.adjoint(w, out=fm)

    def single():
        for b, pl in enumerate(plans):
            pl.forward(fs[b], path=D)
            pl.adjoint(ws[b], path=D)
    out = {"objects": n_objects, "path": "direct",
           "sizes": "X in [32, 128], J in [64, 256], Q in [64, 128] (seed 2024); detector 256 x 64, 64 energies",
           "voxels": int(sum(g.X * g.J for g in geos)), "f_floats": multi.f_len,
           "launches_per_stage": 1}
    for name, fn in (("batched", batched), ("single_calls", single)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        out[name] = {"seconds": sec, "objects_per_s": n_objects / sec}
    out["speedup"] = out["single_calls"]["seconds"] / out["batched"]["seconds"]
    same = all(torch.equal(multi.unpack_g(gm)[b], plans[b].forward(fs[b], path=D)) and
               torch.equal(multi.unpack_f(fm)[b], plans[b].adjoint(ws[b], path=D)) for b in range(n_objects))
    out["bit_identical_to_single_calls"] = bool(same)
    multi.close()
    for pl in plans:
        pl.close()
    return out


def paper_table1_experiment(dev, reps=3):
    """The paper's own timing geometry (Sec. VII, Table I: 2048 x 1536 detector
    pixels of 0.19 mm, 28 x 28 voxels, translation step 16, 79 q bins; 64 energy
    bins and the synthetic spectrum and mask stand in for the paper's 125 kVp
    source and its mask): one forward and one adjoint, timed separately with CUDA
    events after a warm-up, on the direct FP32 path and on the FP32 table path
    (on-the-fly knot interpolation: the detector is too large for 16-bit pair
    records).  The paper's MATLAB times are printed beside them as context; they
    are another machine's and another implementation's (with its own 6.2 %
    forward approximation error), not a target."""
    import torch
    from paper_1603_06400_gb300 import caxsi
    g = synth.paper_table1_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, 1004)
    plan = caxsi.Plan(g, phi, mask)
    f = torch.tensor(synth.phantom(g, 0), dtype=torch.float32, device=dev)
    w = torch.rand((g.M, g.N), device=dev, generator=torch.Generator(device=dev).manual_seed(7)) + 0.5
    out = {"geometry": "detector 2048 x 1536 pixels (0.19 mm), object 28 x 28 voxels (2.5 x 3.04 mm), "
                       "79 q bins 0.1-4 nm^-1, 64 energy bins 15-125 keV",
           "pairs": g.X * g.J * g.M * g.N, "open_pairs": plan.info()["n_open_pairs"],
           "paper_matlab_seconds": {"forward_all_optimisations": 61.04, "backward_all_optimisations": 287.40,
                                    "forward_no_optimisation": 10516.88, "backward_no_optimisation": 10512.32}}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps
    for path in ("direct", "table_fp32"):
        P = caxsi.PATHS[path]
        out[path] = {"forward_seconds": timed(lambda: plan.forward(f, path=P)),
                     "adjoint_seconds": timed(lambda: plan.adjoint(w, path=P))}
    plan.close()
    return out


def symmetric_mask_experiment(dev, reps=3):
    """The joint system design of Sec. III-A / III-C: with a secondary mask that is
    mirror-symmetric about the central ray (synth.symmetric_mask), the direct FP32
    operators share geometry and mask factor among the four mirror pairs and
    compute the mask factor online (CAXSI_OPT_ONLINE_MASK) instead of reading the
    precomputed per-pair bits.  Paper-scale workload, phantom 0; one forward + one
    adjoint timed with CUDA events (after a warm-up), with and without the option,
    and the relative L2 difference between the two (same operator)."""
    import torch
    from paper_1603_06400_gb300 import caxsi
    g = synth.paper_geometry()
    phi = synth.tungsten_spectrum(g)
    mask = synth.symmetric_mask(g, 1003)
    plan = caxsi.Plan(g, phi, mask)
    f = torch.tensor(synth.phantom(g, 0), dtype=torch.float32, device=dev)
    w = torch.rand((g.M, g.N), device=dev, generator=torch.Generator(device=dev).manual_seed(7)) + 0.5
    D = caxsi.PATH_DIRECT
    out = {"mask": "mirror-symmetric Bernoulli(0.5) cells (seed 1003)", "path": "direct"}
    res = {}
    for on in (False, True):
        plan.set_online_mask(on)
        gg, ff = plan.forward(f, path=D), plan.adjoint(w, path=D)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.forward(f, path=D)
            plan.adjoint(w, path=D)
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        key = "online_symmetric" if on else "per_pair_bits"
        out[key] = {"evals_per_s": 1.0 / sec, "seconds": sec}
        res[key] = (gg.double(), ff.double())
    out["speedup"] = out["per_pair_bits"]["seconds"] / out["online_symmetric"]["seconds"]
    a, b = res["per_pair_bits"], res["online_symmetric"]
    out["fwd_rel_l2_vs_bits"] = float(torch.linalg.norm(b[0] - a[0]) / torch.linalg.norm(a[0]))
    out["adj_rel_l2_vs_bits"] = float(torch.linalg.norm(b[1] - a[1]) / torch.linalg.norm(a[1]))
    plan.close()
    return out


def precision_experiment(caxsi, plan, g, dev, make_plan, reps=20):
    """Throughput and error of the reduced-cost operators at full size: 16-bit
    contractions (bf16, fp16) on the exact knots, and u tables of 1024, 2048 and
    4096 uniform samples (FP32 and bf16 contractions).  One evaluation = one
    forward + one adjoint (CUDA events over `reps` after 3 warm-ups, inputs
    resident); errors are relative L2 against the exact FP32 table path, which
    is itself within 1e-6 of the FP64 oracle."""
    import torch
    P = caxsi.PATHS
    f = torch.tensor(synth.phantom(g, 0), dtype=torch.float32, device=dev)
    w = torch.rand((g.M, g.N), device=dev, generator=torch.Generator(device=dev).manual_seed(7)) + 0.5

    def measure(pl, path):
        for _ in range(3):
            pl.forward(f, path=P[path])
            pl.adjoint(w, path=P[path])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            pl.forward(f, path=P[path])
            pl.adjoint(w, path=P[path])
        e1.record()
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        return sec, pl.forward(f, path=P[path]).double(), pl.adjoint(w, path=P[path]).double()

    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    t_ref, g_ref, f_ref = measure(plan, "table_fp32")
    out = {"table_fp32": {"evals_per_s": 1.0 / t_ref, "u_samples": "exact knots"}}
    for path in ("table_bf16", "table_fp16"):
        t, gg, ff = measure(plan, path)
        out[path] = {"evals_per_s": 1.0 / t, "speedup": t_ref / t, "u_samples": "exact knots",
                     "fwd_rel_l2": rel(gg, g_ref), "adj_rel_l2": rel(ff, f_ref)}
    for n in (1024, 2048, 4096):
        sp = make_plan(n)
        for path in ("table_fp32", "table_bf16"):
            t, gg, ff = measure(sp, path)
            out[f"utable_{n}_{path.split('_')[1]}"] = {
                "evals_per_s": 1.0 / t, "speedup": t_ref / t, "u_samples": n,
                "fwd_rel_l2": rel(gg, g_ref), "adj_rel_l2": rel(ff, f_ref)}
        sp.close()
    out["reference"] = "exact FP32 table path (forward and adjoint of phantom 0 and a random image)"
    return out


def caxsi_paths():
    from paper_1603_06400_gb300 import caxsi
    return caxsi.PATHS


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1603_06400_gb300 import build as B
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()
    from paper_1603_06400_gb300 import caxsi

    g = geometry(args.workload)
    phi = synth.tungsten_spectrum(g)
    mask = synth.random_mask(g, mask_seed(args.workload))
    path = caxsi.PATHS[args.path]
    plan = caxsi.Plan(g, phi, mask)
    info = plan.info()

    mine = rank_phantoms(rank, world)
    states = []
    ones = torch.ones((g.M, g.N), device=dev)
    b1 = plan.adjoint(ones, path=path)
    for p in mine:
        f_true = torch.tensor(synth.phantom(g, p), dtype=torch.float32, device=dev)
        mean = plan.forward(f_true, path=path)
        peak = synth.log_uniform_peak(p)
        y = torch.tensor(synth.poisson_counts((mean * (peak / mean.max())).cpu().numpy().astype(
            np.float64), 100 + p), dtype=torch.float32, device=dev)
        f0 = torch.full((g.X, g.J, g.Q), float(y.sum() / b1.sum()), device=dev)
        beta = 1e-3 * float(y.sum()) / (g.X * g.J * g.Q)
        delta = 0.01 * float(f0.max())
        states.append((y, f0, beta, delta))
    torch.cuda.synchronize()

    def step(t):
        y, f, beta, delta = states[t % len(states)]
        plan.recon_step(y, f, beta=beta, delta=delta, path=path)

    for t in range(args.warmup):
        step(t)
    torch.cuda.synchronize()
    info = plan.info()   # after warm-up: the table paths build their tables on first use

    sampler = ClockSampler(gpu_query_id(torch, local))
    time.sleep(0.6)  # let the sampler start
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    plan.profile(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    e0.record(stream)
    for t in range(args.steps):
        step(args.warmup + t)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall1 = time.time()
    ms = e0.elapsed_time(e1)
    kstats = plan.profile_read()
    plan.profile(False)
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)

    ms_max = max_over_ranks(ms, dist, dev)
    total_evals = args.steps * world
    value = total_evals / (ms_max / 1e3)

    # e2e through the host-buffer C calls (pinned host memory), per step one
    # forward + one adjoint with their copies
    e2e = None
    if not args.no_e2e:
        fh = torch.tensor(synth.phantom(g, mine[0]), dtype=torch.float32).pin_memory().numpy()
        wh = torch.rand((g.M, g.N), dtype=torch.float32).pin_memory().numpy()
        gh = torch.empty((g.M, g.N), dtype=torch.float32).pin_memory().numpy()
        fo = torch.empty((g.X, g.J, g.Q), dtype=torch.float32).pin_memory().numpy()
        n_e2e = max(3, min(args.steps, 50))
        for _ in range(3):
            plan.forward_host(fh, out=gh, path=path)
            plan.adjoint_host(wh, out=fo, path=path)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            plan.forward_host(fh, out=gh, path=path)
            plan.adjoint_host(wh, out=fo, path=path)
        el = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": n_e2e * world / el, "unit": UNIT,
               "h2d_bytes_per_step": int((g.f_len + g.g_len) * 4),
               "d2h_bytes_per_step": int((g.g_len + g.f_len) * 4),
               "api": "caxsi_forward_host + caxsi_adjoint_host (pinned host buffers)"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks, peak_kind = measured_peaks()
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    kernels = {k: {"launches": n, "avg_ms": tot / max(n, 1), "total_ms": tot}
               for k, (n, tot) in kstats.items()}
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"]) if kernels else None
    roofline = None
    if dom:
        unit, work, bound = kernel_work(dom, g, info, args.path, nsm)
        if work is not None:
            avg_s = kernels[dom]["avg_ms"] / 1e3
            if bound == "alu":
                # FP32 FMA pipes: 128 lanes per SM x 2 flop at the maximum SM clock
                peak = nsm * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
                peak_note = (f"FP32 SIMT: {nsm} SMs x 128 lanes x 2 flop x "
                             f"{peaks.get('sm_max_mhz', 2070.0):g} MHz ({peak_kind} clock)")
                achieved = work / avg_s / 1e12
            elif bound == "hbm":
                peak = float(peaks["hbm_gbs"])
                peak_note = f"HBM copy bandwidth, {peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                achieved = work / avg_s / 1e9
            else:
                bf16 = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
                tf32 = args.path == "table_fp32"
                peak = bf16 / 2.0 if tf32 else bf16
                peak_note = (f"dense {'TF32 = bf16 / 2 (nominal ratio)' if tf32 else 'bf16/fp16'} from "
                             f"the {peak_kind} sustained bf16 GEMM rate")
                achieved = work / avg_s / 1e12
            design = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                      "frac": achieved / peak, "peak_source": peak_note, "work_per_launch": work,
                      "basis": "the bytes / flops this design streams or issues per launch "
                               "(records, knot-table rows, partial images; contraction passes)"}
            roofline = roofline_line(dom, avg_s, design, g, info, args.path, kernels, args.steps, peaks,
                                     peak_kind, nsm)
    launches = sum(n for n, _ in kstats.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": workload_desc(g, args.workload), "path": args.path,
                   "l2": f"inputs larger than L2: {len(states)} phantom states of "
                         f"{g.f_len * 4 / 1e6:.1f} MB cycled per step plus "
                         f"{info['table_bytes'] / 1e6:.0f} MB of plan tables",
                   "phantoms_per_rank": len(states)},
        "plan": {"n_open_pairs": info["n_open_pairs"], "n_records": info["n_records"],
                 "n_sym_records": info["n_sym_records"],
                 "n_breakpoints": info["n_breakpoints"], "table_bytes": info["table_bytes"]},
        "roofline": roofline,
        "cpu_baseline": None,
        "e2e": e2e,
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                   "reasons": clocks["reasons"], "samples": clocks["samples"]},
        "gpu_launches": launches,
        "kernels": kernels,
    }
    def make_plan(n):
        sp = caxsi.Plan(g, phi, mask)
        sp.set_u_samples(n)
        return sp

    if world == 1 and args.workload != "small" and not args.no_recon:
        line["precision"] = precision_experiment(caxsi, plan, g, dev, make_plan)
        warm = train_warm_start(plan, g, args.unet_steps) if args.unet_steps > 0 else None
        line["recon"] = recon_experiment(caxsi, plan, g, dev, phantom=0, warm=warm, make_plan=make_plan)
        line["recon_seeds"] = recon_seeds(caxsi, plan, g, dev, warm)
    if world == 1 and args.workload == "paper" and not args.no_recon:
        line["symmetric_mask"] = symmetric_mask_experiment(dev)
        line["paper_table1"] = paper_table1_experiment(dev)
        line["batch"] = {"uneven_objects": uneven_batch_experiment(dev),
                         "depth_slabs": batch_experiment(plan, g)}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g)
    print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
