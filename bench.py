#!/usr/bin/env python
"""Benchmark of the trace-estimation hot path on B300.

Headline workload (the largest single-GPU configuration: the two-level
multigrid MLMC one): Wilson-Dirac operator on a 24^3 x 48 lattice
(antiperiodic in t), kappa = 0.13, synthetic SU(3) links (Gram-Schmidt
projection of I + 0.5 G, seed 1004) standing in for the paper's RQCD ensemble;
4^4 aggregates, N_v = 24 test vectors from 3 inverse iterations on Rademacher
starts, coarse operator P^dag D P as a 9-point stencil of 48 x 48 blocks
(2592 coarse sites) applied on the tensor cores (BF16 operands, FP32
accumulate).  One step = one two-level MLMC estimate (Eq. 12, L = 2) of
tr[g5 D^{-1}(t,t)] with 64 level-1 and 512 level-2 samples: RHS generation on
the device, the 64-RHS fine solve and its coarse correction P D_c^{-1} P^dag,
512 coarse solves, per-timeslice FP64 contractions, means and variances; all
solves to a true relative residual of 1e-10 by FP32 (or BF16) inner BiCGStab
inside FP64 defect correction.  The multigrid setup (test vectors, P, D_c) is
a one-off per gauge field, outside the timed steps (reported as setup_s; the
end-to-end steps include it).

`value` = algorithmic Dslash bytes moved by all fine and coarse stencil
launches of the step / step time (GB/s, the metric's unit); `roofline` gives
the dominant stencil kernel against the measured HBM copy bandwidth (and
against the 8 TB/s spec figure).  `trace_time` compares, at the same noise and
so the same statistical error, this mixed-precision batched path with the
plain FP64 single-RHS path on the same GPU (the metric's second half).

python bench.py [--gpus N --steps K --warmup W --prec fp32|bf16 --impl wd|reference]
Under torchrun each rank draws its own samples (seed offset by rank): no
collective on the data path; one barrier and a max/sum over ranks of the
timing only.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (24, 24, 24, 48)
KAPPA = 0.13
SPREAD = 0.5
GAUGE_SEED = 1004
NOISE_SEED = 2004
N1, N2 = 64, 512
NV, AGG, TV_ITERS, TV_SEED = 24, (4, 4, 4, 4), 3, 4
TOL = 1e-10
BC = (1, 1, 1, -1)
SPEC_HBM_GBS = 8000.0
METRIC = "Dslash GB/s (% HBM peak); trace time at fixed error, mixed+batched vs FP64"
WORKLOAD = ("24^3x48 two-level MGMLMC: kappa 0.13, 4^4 aggregates, N_v = 24 (3 inverse iterations), "
            "48x48 coarse blocks on tensor cores; tr[g5 D^-1(t,t)] with 64 level-1 + 512 level-2 samples per step, "
            "solves to 1e-10")


def env_rank():
    return int(os.environ.get('RANK', 0)), int(os.environ.get('WORLD_SIZE', 1)), int(os.environ.get('LOCAL_RANK', 0))


def rank_seed(rank):
    """Noise seed of one replica: every rank draws its own samples."""
    return NOISE_SEED + 7919 * rank


def combine_ranks(dist, ms, nbytes, device):
    """Whole-job numbers over replicas: the slowest rank's time (max) and the
    algorithmic bytes of all ranks (sum), so value = all ranks' bytes / the
    job's time.  dist None: one process."""
    if dist is None:
        return ms, nbytes
    import torch
    t = torch.tensor([ms, nbytes], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, 'MEASURED_PEAKS.json')))
    except Exception:
        return None


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# FP32 fine stencil in this step, averaged over the 52 launches of one profiled
# step (ncu, one pass, full size; command and numbers in
# profiles/hop_kernel_f2_fp32_24x24x24x48_step.md).  It holds for the stencil
# sources it was taken with: their hash is checked, and the field is null once
# they change.
HOP32_TRAFFIC = {"sources": ("paper_2607_05157_b300/csrc/wd_dslash.cu", "paper_2607_05157_b300/csrc/wd_common.cuh",
                             "paper_2607_05157_b300/csrc/wd_internal.h"),
                 "sha256_16": "46273a314bdcfe4b", "bytes_per_launch": 6558.1e6,
                 "algorithmic_bytes_per_launch": 4901.3e6}


def hop32_traffic():
    import hashlib
    h = hashlib.sha256()
    try:
        for f in HOP32_TRAFFIC["sources"]:
            with open(os.path.join(ROOT, f), 'rb') as fh:
                h.update(fh.read())
    except OSError:
        return None
    return HOP32_TRAFFIC["bytes_per_launch"] if h.hexdigest()[:16] == HOP32_TRAFFIC["sha256_16"] else None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""
    Q = ('clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(['nvidia-smi', '-i', str(self.idx), '--query-gpu=' + self.Q,
                                       '--format=csv,noheader,nounits', '-lms', '200'],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ''
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                self.out = ''

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for line in (self.out or '').splitlines():
            f = [x.strip() for x in line.split(',')]
            if len(f) < 6:
                continue
            try:
                sm.append(float(f[0])); mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[2:6]):
                if v.lower().startswith('active'):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU oracle baseline ---------------------------------------------------

def _oracle_apply_worker(args):
    """One worker of the CPU baseline: `napply` applications of the oracle's
    FP64 D (the operator inside every solve of the workload) to a Gaussian
    spinor on the headline lattice.  Returns (seconds, applications)."""
    napply, seed, dims = args
    import numpy as np
    sys.path.insert(0, ROOT)
    import synth
    from oracle import wilson
    U = synth.gauge_field(dims, SPREAD, GAUGE_SEED)
    v = synth.spinors(dims, 1, seed)[0]
    t0 = time.perf_counter()
    for _ in range(napply):
        v = wilson.apply(U, v, KAPPA, BC)
        v /= np.linalg.norm(v)
    return time.perf_counter() - t0, napply


def oracle_baseline(napply=2, dims=DIMS, workers=None):
    """The FP64 CPU oracle on a bounded sample of the headline workload:
    `napply` applications of D per worker process, one worker per host core
    (spawned, so they start clean of any GPU state).  Returns (GB/s of the
    same algorithmic stencil bytes as the GPU model, cores, seconds)."""
    import multiprocessing as mpr
    # one process per host core, at most 16 (each holds its own ~1.5 GB of links and spinors)
    cores = workers or min(len(os.sched_getaffinity(0)), 16)
    ctx = mpr.get_context('spawn')
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_apply_worker, [(napply, 500 + i, dims) for i in range(cores)])
    wall = time.perf_counter() - t0
    busy = max(r[0] for r in res)
    n = sum(r[1] for r in res)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    # FP64, one RHS: input + output (+ addend) spinors and 8 links per site, per application of D
    bytes_per_apply = V * (3 * 192 + 8 * 144)
    return n * bytes_per_apply / busy / 1e9, cores, busy, wall


def run_reference(args):
    """The reference arm: the oracle itself (there is no installable reference
    implementation; the paper ships none), timed on the host cores on the
    headline workload's operator, a bounded sample per step."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    vals, t_all, cores = [], 0.0, 1
    for _ in range(args.steps):
        gbs, cores, busy, wall = oracle_baseline(1)
        vals.append(gbs)
        t_all += busy
    value = statistics.median(vals)
    sample = f"1 application of the FP64 D per host core ({cores} processes) on the 24^3x48 lattice per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle: applications of D)"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- algorithmic bytes of the stencil launches of a profiled region ----------

def dslash_bytes(api, wd, c, ncd, Vc):
    """Fine (FP32/BF16 and FP64 / double-float) stencil bytes and coarse
    stencil bytes, and event times of the launches profiled on context c since
    wd_profile(c, 1).  The coarse launches of the solves multiply BF16 pairs:
    blocks 9 * ncd^2 * 8 B per site and launch, input 8 B and FP32 output 8 B
    per complex entry and RHS."""
    n32, ms32, b32 = api.wd_profile_get(c.h, wd.WD_K_HOP)
    n64, ms64, b64 = api.wd_profile_get(c.h, wd.WD_K_HOP64)
    nco, msco, flco = api.wd_profile_get(c.h, wd.WD_K_COARSE)
    rhs_sites = flco / (8.0 * ncd * ncd * 9.0) if ncd else 0.0      # sum over launches of Vc * nrhs
    bco = nco * Vc * 9 * ncd * ncd * 8.0 + rhs_sites * ncd * (8.0 + 8.0)
    return {"hop32": (n32, ms32, b32), "hop64": (n64, ms64, b64), "coarse": (nco, msco, bco, flco)}


# ---- secondary measurements (other rows and configurations) ------------------

def coarse_measure(wd, api, torch, synth, rhs_list=(64, 512), dims=(24, 24, 24, 48)):
    """The tcgen05 coarse 9-point block stencil on the 24^3x48 two-level
    workload (4^4 aggregates, 24 test vectors -> 48x48 blocks, 2592 coarse
    sites), CUDA-event times of the kernel, algorithmic TFLOP/s (8 ncd^2 per
    block, 9 blocks per site and RHS) and GB/s of the compact algorithmic
    bytes: blocks and input at 4 B (BF16) or 8 B (BF16 pairs, the operator of
    the coarse solves) per complex entry, FP32 output 8 B."""
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1004), 0.13, BC)
    api.wd_mg_setup(ctx.h, None, 24, (4, 4, 4, 4), tv_iters=0, seed=3)
    Vc, ncd = (dims[0] // 4) * (dims[1] // 4) * (dims[2] // 4) * (dims[3] // 4), 48
    out = []
    for mode, prec, eb in (("bf16_pairs", 1, 8.0), ("bf16", 2, 4.0)):
        for nrhs in rhs_list:
            x = torch.randn((nrhs, Vc, ncd), dtype=torch.complex128, device='cuda')
            y = torch.empty_like(x)
            for _ in range(2):
                api.wd_coarse_apply(ctx.h, x, y, prec)
            torch.cuda.synchronize()
            api.wd_profile(ctx.h, True)
            for _ in range(5):
                api.wd_coarse_apply(ctx.h, x, y, prec)
            n, ms, fl = api.wd_profile_get(ctx.h, wd.WD_K_COARSE)
            api.wd_profile(ctx.h, False)
            per = ms / n
            alg = Vc * (9 * ncd * ncd * eb + nrhs * ncd * (eb + 8.0))
            out.append({"operands": mode, "nrhs": nrhs, "ms_per_launch": per,
                        "TFLOP_s": fl / n / (per * 1e-3) / 1e12, "GB_s_algorithmic": alg / (per * 1e-3) / 1e9})
    ctx.close()
    peaks = measured_peaks()
    return {"workload": "x".join(map(str, dims)) + ", 4^4 aggregates, nv=24 (48x48 blocks), tcgen05 BF16 or BF16-pair operands, FP32 accumulate",
            "bf16_peak_TFLOP_s": peaks['bf16_tflops'] if peaks else 1800.0, "points": out}


def gradient_measure(wd, api, torch, synth):
    """The gradient: d/dkappa and the link force of the probing (d=2, full dilution)
    estimate of tr[g5 D^-1] on 8^3x16 (192 solves + force), wall time."""
    dims = (8, 8, 8, 16)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1005), 0.125, BC)
    shape = (4, 16, 8, 8, 8, 3, 3)
    api.trace_gradient(ctx.h, wd.WD_PROBE, 12, 1, 16, d=2, seed=1, op=1, tol=TOL, link_shape=shape)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.trace_gradient(ctx.h, wd.WD_PROBE, 12, 1, 16, d=2, seed=2, op=1, tol=TOL, link_shape=shape)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.close()
    return {"workload": "8^3x16 probing d=2 x 12 dilution (192 RHS), gamma5, dkappa + link force",
            "ms": 1e3 * dt}


def probing_measure(wd, api, torch, synth):
    """The probing workload, 16^3x32 kappa 0.13: distance-2 (16 colours) and
    distance-4 (64 colours) torus-colouring probing x 12 spin-colour dilution
    for tr[g5 D^-1(t,t)] summed over t, against Hutchinson at equal solve count
    (Eq. 14 vs Eq. 3): wall time, solves, the variance of the total of one
    estimate of that cost, and the plain FP64 single-RHS path on a subset of
    the same d = 2 vectors (time per solve, extrapolated to the same solves)."""
    import numpy as np
    dims = (16, 16, 16, 32)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1003), 0.13, BC)

    def svar(S):
        tot = S.sum(1)
        return float(np.sum(np.abs(tot - tot.mean()) ** 2) / (len(tot) - 1))
    out = {"workload": "16^3x32 kappa 0.13, tr[g5 D^-1(t,t)] summed over t; probing d = 2 (16 colours) and "
                       "d = 4 (64 colours) x 12 dilution, 4 noise samples each; Hutchinson with 768 Rademacher "
                       "vectors; solves to 1e-10, FP32 inner, autotuned batches"}
    # warm-up at the measured shapes (tuning, workspaces, graphs)
    for d in (2, 4):
        api.trace_estimate(ctx.h, wd.WD_PROBE, 12, 4, 32, d=d, seed=1, op=1, tol=TOL)
    api.trace_estimate(ctx.h, wd.WD_HUTCH, 1, 768, 32, seed=1, op=1, tol=TOL)
    for d, N in ((2, 4), (4, 4)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = api.trace_estimate(ctx.h, wd.WD_PROBE, 12, N, 32, d=d, seed=2, op=1, tol=TOL, with_samples=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[f"probe_d{d}"] = {"ms": 1e3 * dt, "solves": r["n_solves"], "ms_per_solve": 1e3 * dt / r["n_solves"],
                              "var_per_sample": svar(r["samples"]), "solves_per_sample": r["n_solves"] // N}
        if d == 2:
            rd2 = r
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = api.trace_estimate(ctx.h, wd.WD_HUTCH, 1, 768, 32, seed=2, op=1, tol=TOL, with_samples=True)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    vh = svar(h["samples"])
    out["hutchinson"] = {"ms": 1e3 * dt, "solves": h["n_solves"], "ms_per_solve": 1e3 * dt / h["n_solves"],
                         "var_per_sample": vh}
    for d in (2, 4):
        q = out[f"probe_d{d}"]
        q["var_hutchinson_over_probing_at_equal_solves"] = (vh / q["solves_per_sample"]) / q["var_per_sample"]
    # the plain FP64 single-RHS path on one d = 2 sample (192 solves), per solve
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = api.trace_estimate(ctx.h, wd.WD_PROBE, 12, 1, 32, d=2, seed=2, op=1, prec=wd.WD_FP64, batch=1, tol=TOL,
                           with_samples=True)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    q = out["probe_d2"]
    ms64_per_solve = 1e3 * t64 / f["n_solves"]
    q["fp64_single_rhs_ms_per_solve"] = ms64_per_solve
    q["trace_time_speedup_vs_fp64"] = ms64_per_solve / q["ms_per_solve"]
    # the same vectors through both paths: sample 0's total differs by far less than its spread
    q["fp64_vs_mixed_sample0_diff_over_sd"] = abs(f["samples"][0].sum() - rd2["samples"][0].sum()) / \
        max(q["var_per_sample"], 1e-300) ** 0.5
    ctx.close()
    return out


def mlmc_probe_measure(wd, api, torch, synth):
    """Two-level MLMC with probing on both levels (level 1: probing
    d = 2 x 12 dilution; level 2: colouring of the coarse torus d = 1 x the 48
    coarse dofs of a site; GPU-built 4^4 aggregates with 24 test vectors)
    against plain probing on the same noise samples, 8^3x16: wall time, solves
    and per-sample variances of the total over timeslices."""
    import numpy as np
    dims, N = (8, 8, 8, 16), 4
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1006), 0.125, BC)
    api.wd_mg_setup(ctx.h, None, 24, (4, 4, 4, 4), tv_iters=3, seed=3)

    def svar(S):
        tot = S.sum(1)
        return float(np.sum(np.abs(tot - tot.mean()) ** 2) / (len(tot) - 1))
    api.trace_estimate_mlmc_probe(ctx.h, 12, 2, 2, 48, 1, 2, 16, seed=1, op=1, tol=TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = api.trace_estimate_mlmc_probe(ctx.h, 12, 2, N, 48, 1, N, 16, seed=2, op=1, tol=TOL)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    p = api.trace_estimate(ctx.h, wd.WD_PROBE, 12, N, 16, d=2, seed=2, op=1, tol=TOL, with_samples=True)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ctx.close()
    return {"workload": f"8^3x16, tr[g5 D^-1(t,t)] summed over t, {N} noise samples; level 1: probing d=2 x 12 "
                        "(192 fine + 192 coarse solves per sample); level 2: coarse colouring d=1 x 48 coarse dofs "
                        "(96 coarse solves per sample); plain probing d=2 x 12 (192 fine solves per sample)",
            "mlmc_ms": 1e3 * (t1 - t0), "mlmc_solves": m["n_solves"],
            "mlmc_level1_var_per_sample": svar(m["samples1"]), "mlmc_level2_var_per_sample": svar(m["samples2"]),
            "probe_ms": 1e3 * (t2 - t1), "probe_solves": p["n_solves"],
            "probe_var_per_sample": svar(p["samples"])}


def mlmc3_measure(wd, api, torch, synth):
    """Three-level MLMC on 16^3x32 (kappa 0.13; aggregates 4^4 then
    2^4, i.e. 4^3x8 and 2^3x4, 24 test vectors per level built on the GPU):
    wall time, solves and per-sample variances of each level's total, beside
    the two-level estimator on the same fine noise."""
    import numpy as np
    dims = (16, 16, 16, 32)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1008), 0.13, BC)
    t0 = time.perf_counter()
    api.wd_mg_setup(ctx.h, None, 24, (4, 4, 4, 4), tv_iters=3, seed=5)
    api.wd_mg3_setup(ctx.h, None, 24, (2, 2, 2, 2), tv_iters=3, seed=6)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0

    def svar(S):
        tot = S.sum(1)
        return float(np.sum(np.abs(tot - tot.mean()) ** 2) / (len(tot) - 1))
    api.trace_estimate_mlmc3(ctx.h, 2, 2, 2, 32, seed=1, op=1, tol=TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = api.trace_estimate_mlmc3(ctx.h, 4, 16, 64, 32, seed=2, op=1, tol=TOL)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    r2 = api.trace_estimate(ctx.h, wd.WD_MLMC2, 1, 4, 32, n2=16, seed=2, op=1, tol=TOL, with_samples=True)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ctx.close()
    return {"workload": "16^3x32 kappa 0.13, tr[g5 D^-1(t,t)]; 3 levels: 4 fine + 16 level-2 + 64 level-3 samples; "
                        "2 levels: 4 fine + 16 coarse samples (same fine noise)",
            "setup_s": t_setup, "mlmc3_ms": 1e3 * (t1 - t0), "mlmc3_solves": r["n_solves"],
            "mlmc3_var_per_sample": [svar(r["samples1"]), svar(r["samples2"]), svar(r["samples3"])],
            "mlmc2_ms": 1e3 * (t2 - t1), "mlmc2_solves": r2["n_solves"],
            "mlmc2_level1_var_per_sample": svar(r2["samples"])}


def connected_measure(wd, api, torch, synth):
    """The connected pseudoscalar G(t) with the two-level decomposition on
    8^3x16 (N1 = 4 level-1 samples, N2 = 32 coarse samples): wall time, solves,
    and the variance of the fine term G_11 against the plain estimator on the
    same noise (the variance reduction of Sec. 4)."""
    dims = (8, 8, 8, 16)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1007), 0.125, BC)
    api.wd_mg_setup(ctx.h, None, 24, (4, 4, 4, 4), tv_iters=3, seed=4)
    api.wd_connected_mlmc(ctx.h, 4, 32, 16, seed=1, tol=TOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = api.wd_connected_mlmc(ctx.h, 4, 32, 16, seed=2, tol=TOL)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    ctx.close()
    v11, vplain = r["var"][0], r["var"][5]
    return {"workload": "8^3x16 connected G(t), time-diluted noise, level 1: 4 samples x 16 timeslices (64 fine + "
                        "64 coarse solves), (2,2): 32 samples x 16 coarse solves",
            "ms": 1e3 * dt, "n_solves": r["n_solves"],
            "var_plain_over_var_G11": {str(t): float(vplain[t] / v11[t]) for t in (1, 4, 8)}}


def batched_measure(wd, torch, synth):
    """Batched solves over uneven lattices (the batched part of the two-level configuration):
    8^3x16 (64 RHS) + 12^3x24 (32) + 16^3x32 (16) solved together (persistent
    multi-lattice stencil, CUDA graph) vs one after another."""
    specs = [((8, 8, 8, 16), 0.125, 64), ((12, 12, 12, 24), 0.13, 32), ((16, 16, 16, 32), 0.13, 16)]
    ctxs, bs = [], []
    for i, (d, k, n) in enumerate(specs):
        ctxs.append(wd.Context(d, synth.gauge_field(d, SPREAD, 1100 + i), k, BC))
        bs.append(torch.from_numpy(synth.spinors(d, n, 1200 + i)).cuda())
    B = wd.Batch(ctxs)
    res = {}
    for g in (True, False):
        B.solve(bs, use_graph=g)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            B.solve(bs, use_graph=g)
        torch.cuda.synchronize()
        res["batched_graph_ms" if g else "batched_nograph_ms"] = (time.perf_counter() - t0) / 3 * 1e3
    for c, b in zip(ctxs, bs):
        c.solve(b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(3):
        for c, b in zip(ctxs, bs):
            c.solve(b)
    torch.cuda.synchronize()
    res["sequential_ms"] = (time.perf_counter() - t0) / 3 * 1e3
    B.close()
    for c in ctxs:
        c.close()
    res["workload"] = "8^3x16 (64 RHS) + 12^3x24 (32) + 16^3x32 (16), mixed FP32/FP64 to 1e-10"
    return res


def small_trace_measure(wd, api, torch, synth, steps=10):
    """The 8^3x16 workload: 256 time-diluted RHS (16 samples x 16 timeslices)
    for tr[g5 D^-1(t,t)] and the 12-column point-source correlator C(t) per
    step, one after the other on one context; and the plain FP64 single-RHS
    path on the same trace noise."""
    dims, kappa = (8, 8, 8, 16), 0.125
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1002), kappa, BC)

    def step(i, p=wd.WD_MIXED_FP32, batch=256):
        r = api.trace_estimate(ctx.h, wd.WD_HUTCH, 1 | wd.WD_DIL_TIME, 16, 16, seed=2002 + i, op=1, prec=p,
                               batch=batch, tol=TOL)
        if p != wd.WD_FP64:
            api.wd_point_correlator(ctx.h, (0, 0, 0, 0), 16, prec=p, tol=TOL)
        return r
    for i in range(3):
        step(i)
    torch.cuda.synchronize()
    api.wd_profile(ctx.h, True)
    t0 = time.perf_counter()
    for i in range(steps):
        mix = step(1000 + i)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / steps * 1e3
    n32, ms32, b32 = api.wd_profile_get(ctx.h, wd.WD_K_HOP)
    api.wd_profile(ctx.h, False)
    t0 = time.perf_counter()
    ref = step(1000 + steps - 1, p=wd.WD_FP64, batch=1)
    torch.cuda.synchronize()
    t64 = time.perf_counter() - t0
    ctx.close()
    eps = (mix['var_total'] / 16) ** 0.5
    return {"workload": "8^3x16 kappa 0.125, 256 time-diluted RHS for tr[g5 D^-1(t,t)] + 12 point sources for C(t) "
                        "per step (profiled plain launches, one context)",
            "ms_per_step": ms, "fp32_stencil_GB_s": b32 / (ms32 * 1e-3) / 1e9 if ms32 else None,
            "fp64_single_rhs_trace_ms": 1e3 * t64, "speedup_trace_vs_fp64": 1e3 * t64 / ms,
            "estimate_diff_over_eps": abs(mix['total'] - ref['total']) / eps}


def apply_measure(wd, api, torch, synth, dims, nrhs, steps, warmup):
    """The fine stencil alone: D = 1 - kappa H applied to nrhs Gaussian spinors with
    FP32 storage (two hops per application, each with its same-parity
    addend), CUDA-event times per hop launch and GB/s of the algorithmic
    bytes (96 B in + 96 B out + 96 B addend per site and RHS, 8 links of 72 B
    per site)."""
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1003), 0.13, BC)
    x = torch.randn(ctx.field_shape(nrhs), dtype=torch.complex64, device='cuda')
    y = torch.empty_like(x)
    for _ in range(warmup):
        api.wd_apply(ctx.h, x, y, prec=wd.WD_MIXED_FP32)
    torch.cuda.synchronize()
    api.wd_profile(ctx.h, True)
    for _ in range(steps):
        api.wd_apply(ctx.h, x, y, prec=wd.WD_MIXED_FP32)
    n, ms, b = api.wd_profile_get(ctx.h, wd.WD_K_HOP)
    api.wd_profile(ctx.h, False)
    ctx.close()
    peaks = measured_peaks()
    gbs = b / (ms * 1e-3) / 1e9 if ms else None
    return {"lattice": "x".join(map(str, dims)), "nrhs": nrhs, "hop_launches": n, "us_per_hop": 1e3 * ms / max(n, 1),
            "MB_per_hop": b / max(n, 1) / 1e6, "GB_s": gbs,
            "frac_of_measured_copy": gbs / peaks['hbm_gbs'] if (peaks and gbs) else None}


def step_measure(wd, api, torch, synth, dims, steps, warmup):
    """The headline step (two-level MGMLMC, 64 level-1 + 512 level-2 samples,
    solves to 1e-10, FP32 inner) on another lattice, the other parameters the
    headline's: a small case of the same kernels for profiling.  Returns the
    setup time and the CUDA-event time per step."""
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, GAUGE_SEED), KAPPA, BC)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.wd_mg_setup(ctx.h, None, NV, AGG, tv_iters=TV_ITERS, seed=TV_SEED)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    def step(i):
        return api.trace_estimate(ctx.h, wd.WD_MLMC2, 1, N1, dims[3], n2=N2, seed=rank_seed(0) + i, op=1,
                                  prec=wd.WD_MIXED_FP32, tol=TOL)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize()
    l0 = api.wd_launch_count(ctx.h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for i in range(steps):
        res = step(1000 + i)
    ev1.record()
    torch.cuda.synchronize()
    launches = api.wd_launch_count(ctx.h) - l0
    ctx.close()
    return {"lattice": "x".join(map(str, dims)), "samples": {"level1": N1, "level2": N2}, "setup_s": setup_s,
            "ms_per_step": ev0.elapsed_time(ev1) / max(steps, 1), "launches_per_step": launches / max(steps, 1),
            "n_solves": res["n_solves"] if steps else None}


# ---- the headline ------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=10)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--prec', choices=['fp32', 'bf16'], default='fp32')
    ap.add_argument('--impl', choices=['wd', 'reference'], default='wd')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--no-fp64-compare', action='store_true')
    ap.add_argument('--no-e2e', action='store_true', help='skip the end-to-end steps (profiling runs)')
    ap.add_argument('--no-secondary', action='store_true', help='skip the other rows and configurations')
    ap.add_argument('--coarse-only', action='store_true', help='only the tensor-core coarse stencil measurement')
    ap.add_argument('--coarse-lattice', default='24,24,24,48', help='fine lattice of --coarse-only (X,Y,Z,T)')
    ap.add_argument('--coarse-rhs', default='64,128,256,512', help='RHS counts of --coarse-only')
    ap.add_argument('--apply-only', action='store_true',
                    help='only the fine stencil: D applied (FP32 storage) to --apply-rhs spinors on --apply-lattice')
    ap.add_argument('--apply-lattice', default='24,24,24,48', help='lattice of --apply-only (X,Y,Z,T)')
    ap.add_argument('--apply-rhs', type=int, default=64, help='RHS of --apply-only')
    ap.add_argument('--step-only', action='store_true',
                    help='only the headline step (setup, then --warmup and --steps steps) on --step-lattice')
    ap.add_argument('--step-lattice', default='16,16,16,32', help='lattice of --step-only (X,Y,Z,T)')
    args = ap.parse_args()
    if args.impl == 'reference':
        return run_reference(args)

    rank, world, local = env_rank()
    cpu = None
    if rank == 0 and world == 1 and not (args.no_cpu_baseline or args.coarse_only or args.apply_only or args.step_only):
        # the oracle baseline runs in spawned processes before any GPU work
        gbs, cores, busy, wall = oracle_baseline(1)
        cpu = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"1 application of the FP64 D per process, {cores} processes (one per host core), on "
                         f"the 24^3x48 lattice ({busy:.1f} s busy): the operator inside every solve of the step"}

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
    import synth
    import paper_2607_05157_b300 as wd
    from paper_2607_05157_b300 import api

    if args.coarse_only:
        if rank == 0:
            cd = tuple(int(v) for v in args.coarse_lattice.split(','))
            cr = tuple(int(v) for v in args.coarse_rhs.split(','))
            print(json.dumps({"coarse_tc": coarse_measure(wd, api, torch, synth, cr, cd)}), flush=True)
        return
    if args.apply_only:
        if rank == 0:
            ad = tuple(int(v) for v in args.apply_lattice.split(','))
            print(json.dumps({"fine_stencil": apply_measure(wd, api, torch, synth, ad, args.apply_rhs,
                                                            args.steps, args.warmup)}), flush=True)
        return
    if args.step_only:
        if rank == 0:
            sd = tuple(int(v) for v in args.step_lattice.split(','))
            print(json.dumps({"mlmc2_step": step_measure(wd, api, torch, synth, sd, args.steps, args.warmup)}),
                  flush=True)
        return

    prec = wd.WD_MIXED_FP32 if args.prec == 'fp32' else wd.WD_MIXED_BF16
    T = DIMS[3]
    Vc = int(np.prod([L // a for L, a in zip(DIMS, AGG)]))
    ncd = 2 * NV
    gauge = synth.gauge_field(DIMS, SPREAD, GAUGE_SEED)
    ctx = wd.Context(DIMS, gauge, KAPPA, BC)
    seed0 = rank_seed(rank)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.wd_mg_setup(ctx.h, None, NV, AGG, tv_iters=TV_ITERS, seed=TV_SEED)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    def step(i, p=prec, n1=N1, n2=N2, batch=0, samples=False):
        return api.trace_estimate(ctx.h, wd.WD_MLMC2, 1, n1, T, n2=n2, seed=seed0 + i, op=1, prec=p, batch=batch,
                                  tol=TOL, with_samples=samples)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # timed region: the steps as a user runs them (no per-launch events, so the
    # BiCGStab loops run as captured graphs)
    l0 = api.wd_launch_count(ctx.h)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        results = [step(1000 + i, samples=(i == 0)) for i in range(args.steps)]
        ev1.record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = api.wd_launch_count(ctx.h) - l0

    # profiled repetition of the same steps (same seeds, so the same work):
    # CUDA events around every stencil launch on the library's stream give the
    # per-kernel durations and algorithmic bytes behind `value` and `roofline`
    api.wd_profile(ctx.h, True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for i in range(args.steps):
        step(1000 + i)
    p1.record()
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    prof = dslash_bytes(api, wd, ctx, ncd, Vc)
    api.wd_profile(ctx.h, False)
    step_bytes = prof["hop32"][2] + prof["hop64"][2] + prof["coarse"][2]
    ms, all_bytes = combine_ranks(dist, ms, step_bytes, 'cuda')
    value = all_bytes / (ms * 1e-3) / 1e9

    peaks = measured_peaks()
    peak = peaks['hbm_gbs'] if peaks else 6400.0
    kern = {}
    for name, label in (("hop32", f"hop_kernel ({args.prec} storage, fine stencil)"),
                        ("hop64", "hop_kernel_dd (double-float FP64 steps, fine stencil)"),
                        ("coarse", "coarse 9-point stencil: k_coarse_tc (tcgen05, inner solves) and "
                                   "k_coarse_apply32t (FP32 CUDA cores, recursive residual updates)")):
        n, t_ms, b = prof[name][0], prof[name][1], prof[name][2]
        kern[name] = {"kernel": label, "launches_per_step": n / max(args.steps, 1),
                      "GB_s": b / (t_ms * 1e-3) / 1e9 if t_ms else None,
                      "MB_per_launch": b / n / 1e6 if n else None,
                      "share_of_step": t_ms / ms_prof if ms_prof else None}
    kern["coarse"]["TFLOP_s"] = prof["coarse"][3] / (prof["coarse"][1] * 1e-3) / 1e12 if prof["coarse"][1] else None
    dom = max(kern, key=lambda k: kern[k]["share_of_step"] or 0.0)
    achieved = kern[dom]["GB_s"]
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "frac_of_spec_8000": achieved / SPEC_HBM_GBS if achieved else None,
            "traffic": hop32_traffic() if dom == "hop32" and args.prec == 'fp32' else None,
            "kernel": kern[dom]["kernel"], "peak_source": "measured" if peaks else "fallback",
            "region": "profiled repetition of the timed steps (same seeds; plain launches bracketed by CUDA events)",
            "kernels": kern}

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+bf16+f64" if args.prec == 'fp32' else "bf16+f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "x".join(map(str, DIMS)), "kappa": KAPPA,
                       "samples_per_step": {"level1": N1, "level2": N2}, "solves_per_step": results[-1]["n_solves"],
                       "inner_precision": args.prec, "setup_s": setup_s,
                       "l2": "inputs larger than L2 (each 64-RHS fine stencil launch streams ~4 GB)",
                       "parallelism": f"replicas x{world} (independent samples)"},
            "roofline": roof, "clocks": clk.summary(), "gpu_launches": launches,
            "estimate_total": [results[0]["total"].real, results[0]["total"].imag],
            "std_error": results[0]["var_total"] ** 0.5}

    if not args.no_e2e:
        # end to end through the public API, per gauge configuration: the links
        # uploaded from pinned host memory and ingested, the multigrid setup,
        # the estimate, the result read back
        pinned = torch.from_numpy(gauge.view(np.float64)).pin_memory()
        import ctypes
        api.wd_profile(ctx.h, True)
        api.wd_mg_setup(ctx.h, None, NV, AGG, tv_iters=TV_ITERS, seed=TV_SEED)
        torch.cuda.synchronize()
        sp = dslash_bytes(api, wd, ctx, ncd, Vc)
        api.wd_profile(ctx.h, False)
        setup_bytes = sp["hop32"][2] + sp["hop64"][2] + sp["coarse"][2]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(args.steps):
            wd.lib.wd_update_gauge(ctx.h, ctypes.c_void_p(pinned.data_ptr()), ctypes.c_double(KAPPA))
            api.wd_mg_setup(ctx.h, None, NV, AGG, tv_iters=TV_ITERS, seed=TV_SEED)
            step(1000 + i)
        e1.record()
        torch.cuda.synchronize()
        e_ms = e0.elapsed_time(e1)
        e_ms, e_bytes = combine_ranks(dist, e_ms, step_bytes + setup_bytes * args.steps, 'cuda')
        line["e2e"] = {"value": e_bytes / (e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": gauge.nbytes,
                       "d2h_bytes_per_step": 8 * (2 * (T + 1) + (T + 1)), "ms_per_step": e_ms / args.steps,
                       "includes": "link upload and ingest, multigrid setup (its stencil bytes counted), estimate, "
                                   "result read-back"}

    if rank == 0 and not args.no_fp64_compare:
        # trace time at fixed error: the same noise (so the same estimate and
        # error) through the plain FP64 single-RHS path, on the first 1/8 of the
        # samples of each level (8 + 64), time scaled by the sample count (8x)
        mix = results[0]
        sub1, sub2 = N1 // 8, N2 // 8
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ref = step(1000, p=wd.WD_FP64, n1=sub1, n2=sub2, batch=1, samples=True)
        torch.cuda.synchronize()
        t_sub = time.perf_counter() - t0
        ref_l2 = api.wd_mlmc_level2_samples(ctx.h, sub2, T)
        mix_sub = step(1000, n1=sub1, n2=sub2, samples=True)
        mix_l2 = api.wd_mlmc_level2_samples(ctx.h, sub2, T)
        eps = mix['var_total'] ** 0.5
        dmax = max(np.abs(ref['samples'].sum(1) - mix_sub['samples'].sum(1)).max(),
                   np.abs(ref_l2.sum(1) - mix_l2.sum(1)).max())
        t_fp64 = t_sub * (N1 // sub1)
        line["trace_time"] = {"mixed_batched_ms": ms / args.steps, "fp64_single_rhs_ms": 1e3 * t_fp64,
                              "speedup": 1e3 * t_fp64 / (ms / args.steps),
                              "fp64_measured_on": f"{sub1} level-1 + {sub2} level-2 samples ({t_sub:.2f} s), scaled "
                                                  f"x{N1 // sub1} to the step's {N1} + {N2}",
                              "max_sample_diff_over_eps": dmax / eps, "std_error_eps": eps}
    if rank == 0 and not args.no_secondary:
        # the same 64 fine noise samples through plain Hutchinson (Eq. 3) on the
        # same context: the cost of the two-level split against the estimator
        # it refines (one warm-up, then the mean of three)
        api.trace_estimate(ctx.h, wd.WD_HUTCH, 1, N1, T, seed=seed0 + 1000, op=1, prec=prec, tol=TOL)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record()
        for _ in range(3):
            hut = api.trace_estimate(ctx.h, wd.WD_HUTCH, 1, N1, T, seed=seed0 + 1000, op=1, prec=prec, tol=TOL)
        h1.record()
        torch.cuda.synchronize()
        ms_h = h0.elapsed_time(h1) / 3
        line["mlmc2_vs_hutchinson"] = {
            "workload": f"{WORKLOAD.split(':')[0]}; Hutchinson with the {N1} level-1 noise samples, same solver",
            "hutchinson_ms": ms_h, "mlmc2_ms": ms / args.steps, "mlmc2_over_hutchinson": (ms / args.steps) / ms_h,
            # variances of the two estimates of the total (trace_estimate reports the
            # per-sample variance for Hutchinson, the estimate's for MLMC2)
            "hutchinson_var_of_estimate": hut["var_total"] / N1, "mlmc2_var_of_estimate": results[0]["var_total"],
            "cost_x_variance_mlmc2_over_hutchinson":
                (ms / args.steps) * results[0]["var_total"] / (ms_h * hut["var_total"] / N1)}
        sec = {}
        for name, fn in (("trace_8x8x8x16", lambda: small_trace_measure(wd, api, torch, synth)),
                         ("probing_16x16x16x32", lambda: probing_measure(wd, api, torch, synth)),
                         ("coarse_tc", lambda: coarse_measure(wd, api, torch, synth)),
                         ("batched", lambda: batched_measure(wd, torch, synth)),
                         ("gradient", lambda: gradient_measure(wd, api, torch, synth)),
                         ("mlmc_probe", lambda: mlmc_probe_measure(wd, api, torch, synth)),
                         ("connected", lambda: connected_measure(wd, api, torch, synth)),
                         ("mlmc3", lambda: mlmc3_measure(wd, api, torch, synth))):
            try:
                sec[name] = fn()
            except Exception as e:          # a secondary row must not lose the headline line
                sec[name] = {"error": str(e)}
        line["secondary"] = sec
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
