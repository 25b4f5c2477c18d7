#!/usr/bin/env python
"""Benchmark of the trace-estimation hot path on B300.

Workload (the 8^3 x 16 configuration): Wilson-Dirac operator on an 8^3 x 16
lattice (antiperiodic in t), kappa = 0.125, synthetic SU(3) links
(Gram-Schmidt projection of I + 0.5 G, seed 1002) standing in for the paper's
RQCD ensemble; per step and per GPU 256 right-hand sides = 16 Rademacher
samples x 16 timeslices (time dilution), estimating the disconnected loop
O(t) = tr[g5 D^{-1}(t,t)] (Eq. 21), plus the pseudoscalar correlator
C(t) = sum_x |D^{-1}(x,t;0,0)|^2 from 12 point sources, each solve to a true
FP64 relative residual of 1e-10 by FP32 (or BF16) BiCGStab inside FP64 defect
correction.

A step = one trace_estimate call plus one wd_point_correlator call, issued from two host threads on two
contexts with their own CUDA streams so that the two independent solves overlap on the GPU (--serial: one
after the other on one context): RHS generation on the device, even-odd
source, 256-RHS batched mixed-precision solve (stencil, BLAS-1, FP64 residual),
odd-site reconstruction, FP64 per-timeslice contraction, mean and sample
variance.  `value` = algorithmic stencil bytes moved by all stencil launches
of the step / step time (GB/s), so it is the whole job's rate in the metric's
unit; `roofline` gives the dominant kernel (the FP32/BF16 stencil) against the
measured HBM copy bandwidth.  `trace_time` compares, at the same noise and so
the same statistical error, the mixed batched path with the plain FP64
single-RHS path on the same GPU (the second half of the metric).

python bench.py [--gpus N --steps K --warmup W --prec fp32|bf16 --impl wd|reference]
Under torchrun each rank draws its own samples (seed offset by rank): no
collective on the data path; one barrier and a max/sum over ranks of the
timing only.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = (8, 8, 8, 16)
KAPPA = 0.125
SPREAD = 0.5
GAUGE_SEED = 1002
NOISE_SEED = 2002
SAMPLES = 16
TOL = 1e-10
BC = (1, 1, 1, -1)
METRIC = "Dslash GB/s (% HBM peak); trace time at fixed error, mixed+batched vs FP64"
WORKLOAD = ("8^3x16 Wilson-Dirac, kappa 0.125, 256 time-diluted Rademacher RHS for tr[g5 D^-1(t,t)] + "
            "12 point sources for C(t), solves to 1e-10")


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


def hop_traffic(prec, alg_bytes_per_launch):
    """DRAM bytes per stencil launch: the committed ncu summary's DRAM bytes per
    algorithmic byte (taken on 256-RHS launches of the same workload) times this
    run's algorithmic bytes per launch, if the summary was taken on the current
    stencil source (else None)."""
    try:
        rec = json.load(open(os.path.join(ROOT, 'profiles', 'hop_traffic.json')))
        csrc = os.path.join(ROOT, 'paper_2607_05157_b300', 'csrc')
        src = b''.join(open(os.path.join(csrc, f), 'rb').read() for f in ('wd_dslash.cu', 'wd_spin.cuh'))
        if rec.get('source_sha256') != hashlib.sha256(src).hexdigest():
            return None
        r = rec.get(prec, {}).get('dram_bytes_per_algorithmic_byte')
        return r * alg_bytes_per_launch if r is not None else None
    except Exception:
        return None


def oracle_baseline(n_timeslices=3):
    """The FP64 CPU oracle on a bounded sample of the same workload: the
    time-diluted solves of sample 0 for the first n timeslices (plain
    BiCGStab on D, contraction).  Returns (GB/s of algorithmic stencil bytes,
    seconds, applies)."""
    import contextlib
    import numpy as np
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:          # numpy's einsum/roll used here are single-threaded anyway
        threadpool_limits = lambda limits: contextlib.nullcontext()
    import synth
    from oracle import estimators, noise, solver, wilson
    U = synth.gauge_field(DIMS, SPREAD, GAUGE_SEED)
    V = int(np.prod(DIMS))
    shape = (DIMS[3], DIMS[2], DIMS[1], DIMS[0], 4, 3)
    napply = [0]

    def A(v):
        napply[0] += 1
        return wilson.apply(U, v.reshape(shape), KAPPA, BC)
    eta = noise.rademacher(NOISE_SEED, 0, 12 * V)
    ts = wilson.timeslice_of_dof(DIMS)
    with threadpool_limits(limits=1):
        t0 = time.perf_counter()
        for t in range(n_timeslices):
            v = np.where(ts == t, eta, 0).astype(complex)
            x, it, res = solver.bicgstab(A, v, tol=TOL)
            estimators.contract(v, x.reshape(-1), DIMS, True)
        dt = time.perf_counter() - t0
    # same byte model as the GPU stencil: FP64, one RHS, in + out + addend spinors
    # and 8 links per output site, two half-lattice hops per application of D
    bytes_per_apply = V * (3 * 192 + 8 * 144)
    return napply[0] * bytes_per_apply / dt / 1e9, dt, napply[0]


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        pass   # the oracle has no warm-up state; skip untimed steps
    t_all = 0.0
    for _ in range(args.steps):
        gbs, dt, n = oracle_baseline(1)
        vals.append(gbs)
        t_all += dt
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (oracle: one time-diluted solve per step)"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "one time-diluted RHS of sample 0 per step (1/256 of the GPU step)"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def coarse_measure(wd, api, torch, synth, rhs_list=(64, 512), dims=(24, 24, 24, 48)):
    """Row a8: tcgen05 coarse 9-point block stencil on the 24^3x48 two-level
    workload (4^4 aggregates, 24 test vectors -> 48x48 blocks, 2592 coarse
    sites), CUDA-event times of the kernel, algorithmic TFLOP/s (8 ncd^2 per
    block, 9 blocks per site and RHS) and block-stream GB/s."""
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1004), 0.13, BC)
    api.wd_mg_setup(ctx.h, None, 24, (4, 4, 4, 4), tv_iters=0, seed=3)
    Vc, ncd = (dims[0] // 4) * (dims[1] // 4) * (dims[2] // 4) * (dims[3] // 4), 48
    out = []
    for nrhs in rhs_list:
        x = torch.randn((nrhs, Vc, ncd), dtype=torch.complex128, device='cuda')
        y = torch.empty_like(x)
        for _ in range(2):
            api.wd_coarse_apply(ctx.h, x, y, 1)
        torch.cuda.synchronize()
        api.wd_profile(ctx.h, True)
        for _ in range(5):
            api.wd_coarse_apply(ctx.h, x, y, 1)
        n, ms, fl = api.wd_profile_get(ctx.h, wd.WD_K_COARSE)
        api.wd_profile(ctx.h, False)
        per = ms / n
        wbytes = Vc * 96 * 864 * 2
        out.append({"nrhs": nrhs, "ms_per_launch": per, "TFLOP_s": fl / n / (per * 1e-3) / 1e12,
                    "block_stream_GB_s": wbytes / (per * 1e-3) / 1e9})
    ctx.close()
    peaks = measured_peaks()
    return {"workload": "x".join(map(str, dims)) + ", 4^4 aggregates, nv=24 (48x48 blocks), BF16 tcgen05, FP32 accumulate",
            "bf16_peak_TFLOP_s": peaks['bf16_tflops'] if peaks else 1800.0, "points": out}


def gradient_measure(wd, api, torch, synth):
    """Row a10: d/dkappa and the link force of the probing (d=2, full dilution)
    estimate of tr[g5 D^-1] on 8^3x16 (192 solves + force), wall time."""
    dims = (8, 8, 8, 16)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1005), KAPPA, BC)
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
    distance-4 (64 colours) torus-colouring probing x 12 spin-colour
    dilution for tr[g5 D^-1(t,t)] summed over t, against Hutchinson at equal
    solve count (Eq. 14 vs Eq. 3): wall time, solves, and the variance of the
    total of one estimate of that cost (the per-sample variance divided by
    the samples one such estimate takes)."""
    import numpy as np
    dims = (16, 16, 16, 32)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1003), 0.13, BC)

    def svar(S):
        tot = S.sum(1)
        return float(np.sum(np.abs(tot - tot.mean()) ** 2) / (len(tot) - 1))
    out = {"workload": "16^3x32 kappa 0.13, tr[g5 D^-1(t,t)] summed over t; probing d = 2 (16 colours) and "
                       "d = 4 (64 colours) x 12 dilution, 4 noise samples each; Hutchinson with 768 Rademacher "
                       "vectors; solves to 1e-10, FP32 inner"}
    api.trace_estimate(ctx.h, wd.WD_PROBE, 12, 1, 32, d=2, seed=1, op=1, tol=TOL)    # tuning, workspaces
    for d, N in ((2, 4), (4, 4)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = api.trace_estimate(ctx.h, wd.WD_PROBE, 12, N, 32, d=d, seed=2, op=1, tol=TOL, with_samples=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[f"probe_d{d}"] = {"ms": 1e3 * dt, "solves": r["n_solves"], "ms_per_solve": 1e3 * dt / r["n_solves"],
                              "var_per_sample": svar(r["samples"]), "solves_per_sample": r["n_solves"] // N}
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
        # variance of one estimate costing q["solves_per_sample"] solves, both methods
        q["var_hutchinson_over_probing_at_equal_solves"] = (vh / q["solves_per_sample"]) / q["var_per_sample"]
    ctx.close()
    return out


def mlmc2_large_measure(wd, api, torch, synth):
    """The two-level workload, 24^3x48 kappa 0.13: GPU setup (24 test vectors
    from 3 inverse iterations, 4^4 aggregates, Galerkin D_c), then the
    two-level MLMC estimate of tr[g5 D^-1(t,t)] with 64 level-1 and 512 level-2
    samples (Eq. 12, L = 2), against plain Hutchinson on the same 64 fine
    noise samples: wall times, solves, per-sample variances of the total."""
    import numpy as np
    dims = (24, 24, 24, 48)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1004), 0.13, BC)

    def svar(S):
        tot = S.sum(1)
        return float(np.sum(np.abs(tot - tot.mean()) ** 2) / (len(tot) - 1))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.wd_mg_setup(ctx.h, None, 24, (4, 4, 4, 4), tv_iters=3, seed=4)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    m = api.trace_estimate(ctx.h, wd.WD_MLMC2, 1, 64, 48, n2=512, seed=2004, op=1, tol=TOL, with_samples=True)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    h = api.trace_estimate(ctx.h, wd.WD_HUTCH, 1, 64, 48, seed=2004, op=1, tol=TOL, with_samples=True)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    ctx.close()
    return {"workload": "24^3x48 kappa 0.13, 4^4 aggregates, N_v = 24 (3 inverse iterations); tr[g5 D^-1(t,t)]; "
                        "MLMC2 with 64 level-1 + 512 level-2 samples; Hutchinson with the same 64 fine samples",
            "setup_s": t1 - t0, "mlmc2_s": t2 - t1, "mlmc2_solves": m["n_solves"],
            "mlmc2_level1_var_per_sample": svar(m["samples"]), "mlmc2_var_total": m["var_total"],
            "hutchinson_s": t3 - t2, "hutchinson_solves": h["n_solves"],
            "hutchinson_var_per_sample": svar(h["samples"]), "hutchinson_var_total": h["var_total"]}


def mlmc_probe_measure(wd, api, torch, synth):
    """Row f2: two-level MLMC with probing on both levels (level 1: probing
    d = 2 x 12 dilution; level 2: colouring of the coarse torus d = 1 x the 48
    coarse dofs of a site; GPU-built 4^4 aggregates with 24 test vectors)
    against plain probing on the same noise samples, 8^3x16: wall time, solves
    and per-sample variances of the total over timeslices."""
    import numpy as np
    dims, N = (8, 8, 8, 16), 4
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1006), KAPPA, BC)
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
    """Row f3: three-level MLMC on 16^3x32 (kappa 0.13; aggregates 4^4 then
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
    """Row f4: connected pseudoscalar G(t) with the two-level decomposition on
    8^3x16 (N1 = 4 level-1 samples, N2 = 32 coarse samples): wall time, solves,
    and the variance of the fine term G_11 against the plain estimator on the
    same noise (the variance reduction of Sec. 4)."""
    dims = (8, 8, 8, 16)
    ctx = wd.Context(dims, synth.gauge_field(dims, SPREAD, 1007), KAPPA, BC)
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
    """Row a11: 8^3x16 (64 RHS) + 12^3x24 (32) + 16^3x32 (16) solved together
    (persistent multi-lattice stencil, CUDA graph) vs one after another."""
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=20)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--prec', choices=['fp32', 'bf16'], default='fp32')
    ap.add_argument('--impl', choices=['wd', 'reference'], default='wd')
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--serial', action='store_true',
                    help='run the correlator after the trace solve on one context (no second stream)')
    ap.add_argument('--no-fp64-compare', action='store_true')
    ap.add_argument('--no-secondary', action='store_true', help='skip the coarse / gradient / batched measurements')
    ap.add_argument('--coarse-only', action='store_true', help='only the tensor-core coarse stencil measurement')
    ap.add_argument('--coarse-lattice', default='24,24,24,48', help='fine lattice of --coarse-only (X,Y,Z,T)')
    ap.add_argument('--coarse-rhs', default='64,128,256,512', help='RHS counts of --coarse-only')
    args = ap.parse_args()
    if args.impl == 'reference':
        return run_reference(args)

    import numpy as np
    import torch
    rank, world, local = env_rank()
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

    prec = wd.WD_MIXED_FP32 if args.prec == 'fp32' else wd.WD_MIXED_BF16
    T = DIMS[3]
    gauge = synth.gauge_field(DIMS, SPREAD, GAUGE_SEED)
    # The two independent parts of a step run on two contexts with their own
    # streams, from two host threads, so that the 12-RHS correlator solve (small,
    # latency-bound launches) fills the gaps of the 256-RHS trace solve; with
    # --serial both run one after the other on one context.
    if args.serial:
        ctx = ctx_c = wd.Context(DIMS, gauge, KAPPA, BC)
        pool = None
    else:
        from concurrent.futures import ThreadPoolExecutor
        s_tr, s_c = torch.cuda.Stream(), torch.cuda.Stream()
        ctx = wd.Context(DIMS, gauge, KAPPA, BC, stream=s_tr)
        ctx_c = wd.Context(DIMS, gauge, KAPPA, BC, stream=s_c)
        pool = ThreadPoolExecutor(1)
    ctxs = [ctx] if ctx_c is ctx else [ctx, ctx_c]
    seed0 = rank_seed(rank)

    def trace_only(i, p=prec, batch=SAMPLES * T):
        return api.trace_estimate(ctx.h, wd.WD_HUTCH, 1 | wd.WD_DIL_TIME, SAMPLES, T, seed=seed0 + i, op=1,
                                  prec=p, batch=batch, tol=TOL)

    def correlator(p=prec):
        return api.wd_point_correlator(ctx_c.h, (0, 0, 0, 0), T, prec=p, tol=TOL)

    def step(i, p=prec, batch=SAMPLES * T, concurrent=True):
        # the whole workload: 256 time-diluted RHS for O(t) and 12 point sources for C(t)
        if pool is not None and concurrent:
            fc = pool.submit(correlator, p)
            r = trace_only(i, p, batch)
            r['C'] = fc.result()
        else:
            r = trace_only(i, p, batch)
            r['C'] = correlator(p)
        return r

    # warm-up one part after the other: the autotuner times its launch-shape
    # candidates on the first call of each shape, and the other stream's work
    # would distort those timings
    for i in range(args.warmup):
        step(i, concurrent=False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # timed region: the steps as a user runs them (no per-launch events, so the
    # BiCGStab loops run as captured graphs)
    l0 = sum(api.wd_launch_count(c.h) for c in ctxs)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        results = [step(1000 + i) for i in range(args.steps)]
        ev1.record()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = sum(api.wd_launch_count(c.h) for c in ctxs) - l0

    # profiled repetition of the same steps (same seeds, so the same work):
    # CUDA events around every stencil launch on the library's stream give the
    # per-kernel durations and algorithmic bytes of the roofline.  Events
    # cannot sit inside a captured graph, so these steps run plain launches.
    # The two parts run one after the other here, so that no kernel's
    # duration includes another stream's work.
    for c in ctxs:
        api.wd_profile(c.h, True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for i in range(args.steps):
        step(1000 + i, concurrent=False)
    p1.record()
    torch.cuda.synchronize()
    ms_prof = p0.elapsed_time(p1)
    n_hop = ms_hop = by_hop = n_h64 = ms_h64 = by_h64 = 0
    for c in ctxs:
        n, t, b = api.wd_profile_get(c.h, wd.WD_K_HOP)
        n_hop, ms_hop, by_hop = n_hop + n, ms_hop + t, by_hop + b
        n, t, b = api.wd_profile_get(c.h, wd.WD_K_HOP64)
        n_h64, ms_h64, by_h64 = n_h64 + n, ms_h64 + t, by_h64 + b
        api.wd_profile(c.h, False)
    ms, step_bytes = combine_ranks(dist, ms, by_hop + by_h64, 'cuda')
    value = step_bytes / (ms * 1e-3) / 1e9

    # end to end through the public API: host (pinned) links uploaded and
    # re-ingested every step, estimates read back to the host (same seeds as
    # the timed steps, so the same algorithmic bytes)
    pinned = torch.from_numpy(gauge.view(np.float64)).pin_memory()
    gptr = pinned.data_ptr()
    import ctypes
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(args.steps):
        for c in ctxs:
            wd.lib.wd_update_gauge(c.h, ctypes.c_void_p(gptr), ctypes.c_double(KAPPA))
        step(1000 + i)
    e1.record()
    torch.cuda.synchronize()
    e_ms = e0.elapsed_time(e1)
    e_ms, e_bytes = combine_ranks(dist, e_ms, by_hop + by_h64, 'cuda')
    h2d = gauge.nbytes * len(ctxs)
    d2h = 8 * (2 * (T + 1) + (T + 1))

    peaks = measured_peaks()
    peak = peaks['hbm_gbs'] if peaks else 6400.0
    achieved = (by_hop / n_hop) / (ms_hop / n_hop * 1e-3) / 1e9 if n_hop else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": hop_traffic(args.prec, by_hop / max(n_hop, 1)),
            "kernel": f"hop_kernel ({args.prec} storage, {n_hop // max(args.steps, 1)} launches/step, "
                      f"{by_hop / max(n_hop, 1) / 1e6:.1f} MB algorithmic per launch)",
            "peak_source": "measured" if peaks else "fallback",
            "region": "profiled repetition of the timed steps (same seeds; plain launches bracketed by CUDA events)",
            "share_of_step": ms_hop / ms_prof if ms_prof else None,
            "fp64_stencil": {"arithmetic": "fp64" if os.environ.get('WD_DD') == '0' else
                             "double-float (FP32 pairs, FP64 fields)",
                             "launches_per_step": n_h64 // max(args.steps, 1),
                             "GB_s": (by_h64 / (ms_h64 * 1e-3) / 1e9) if ms_h64 else None,
                             "share_of_step": ms_h64 / ms_prof if ms_prof else None}}

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if args.prec == 'fp32' else "bf16+f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "x".join(map(str, DIMS)), "kappa": KAPPA,
                       "rhs_per_step_per_gpu": SAMPLES * T + 12, "inner_precision": args.prec,
                       "l2": "inputs larger than L2 (each stencil launch streams >100 MB)",
                       "parallelism": f"replicas x{world} (independent samples)"},
            "roofline": roof, "clocks": clk.summary(),
            "e2e": {"value": e_bytes / (e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e_ms / args.steps},
            "gpu_launches": launches,
            "solves_per_step": results[-1]["n_solves"] + 12}

    if rank == 0 and not args.no_fp64_compare:
        # trace time at fixed error: same noise (so the same estimate and error)
        # through the plain FP64 single-RHS path
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ref = trace_only(1000, p=wd.WD_FP64, batch=1)
        torch.cuda.synchronize()
        t_fp64 = time.perf_counter() - t0
        mix = results[0]
        eps = (mix['var_total'] / SAMPLES) ** 0.5
        line["trace_time"] = {"mixed_batched_ms": ms / args.steps, "fp64_single_rhs_ms": 1e3 * t_fp64,
                              "speedup": 1e3 * t_fp64 / (ms / args.steps),
                              "estimate_diff_over_eps": abs(mix['total'] - ref['total']) / eps,
                              "std_error_eps": eps}
    if rank == 0 and not args.no_secondary:
        # secondary measurements of the other rows, outside the timed region
        line["secondary"] = {"coarse_tc": coarse_measure(wd, api, torch, synth),
                             "gradient": gradient_measure(wd, api, torch, synth),
                             "batched": batched_measure(wd, torch, synth),
                             "probing": probing_measure(wd, api, torch, synth),
                             "mlmc2_24": mlmc2_large_measure(wd, api, torch, synth),
                             "mlmc_probe": mlmc_probe_measure(wd, api, torch, synth),
                             "connected": connected_measure(wd, api, torch, synth),
                             "mlmc3": mlmc3_measure(wd, api, torch, synth)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        gbs, dt, n = oracle_baseline(3)
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                                "sample": f"3 of the 256 time-diluted solves of one step ({dt:.1f} s, {n} applies of D)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    if pool is not None:
        pool.shutdown()
    if dist:
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
