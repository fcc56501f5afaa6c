#!/usr/bin/env python
"""Benchmark of the alpha-Mobius red-black domain-wall solve on GB300.

Workload (named in the JSON line): 16^3x32 lattice, Ls = 16, Mobius b = 1.5,
c = 0.5, M5 = -1.8, m = 0.01, alpha = 1.0 (--alpha), synthetic SU(3) links
U = exp(i 0.5 H) (seed 0) and a Gaussian 4D source (seed 1).  One step is one
complete propagator solve through the C ABI (dwf_cgne_solve): right-hand side
D_1(1) P b, Schur source, CG on the normal equations of D_bb with FP32 inner
applies and FP64 reliable updates to FP64 true residual 1e-10, reconstruction
of the red half and extraction of z_1.

value: D_bb-apply bytes per second over the whole timed solve, i.e.
(D_bb + D_bb^+ applies) x algorithmic bytes per apply / wall time of the steps,
with the two-pass byte model 120 w_s + 16 r w_g / Ls per 5D half-site
(w_s, w_g bytes per real of spinor and gauge, r = 18 reals per link).
roofline: the D_bb apply of the CG (hop pass A on B p, which the p update forms,
+ pass B) timed with CUDA events on the solver's stream inside the timed region,
against the measured HBM copy peak.  alu: the same applies as GFLOP/s with the
minimum flop count per site, against the FP32 FFMA throughput measured in the
same run (libdwf_probe).  accuracy (outside the timed region): the 5D residual of
the workload's solution at 24 sampled sites by the single-site oracle, and the
4^4 propagator error against the oracle's own solve.
cpu_baseline / --impl reference: the FP64 numpy oracle's D_bb apply on a
bounded sample (8^3x16 sub-lattice, same parameters), with the FP64 byte model;
also on all host cores (one process per core) and the oracle's 4^4 CGNE time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LATTICE = (16, 16, 16, 32)
LS = 16
M5, MASS, B, C, EPS = -1.8, 0.01, 1.5, 0.5, 0.5
SAMPLE_LATTICE = (8, 8, 8, 16)
METRIC = "D_bb apply GB/s inside CGNE to true residual 1e-10 (16^3x32, Ls=16)"
GAUGE_REALS = 18


def bytes_per_site(ws, wg, Ls, r=GAUGE_REALS):
    """Two-pass algorithmic bytes of one D_bb apply per 5D half-site."""
    return 120 * ws + 16 * r * wg / Ls


# Minimum floating-point work of one D_bb apply per 5D half-site: two Wilson hops
# (1320 each, the conventional count: projection, SU(3) multiply, reconstruction
# over 8 directions) plus the 5th-dimension factors B, K = B I^-1 and I^-1 by
# their cyclic-bidiagonal recurrences and the final axpy.
FLOP_PER_SITE = 3120


def probe_fma_peaks(kinds=(1, 0), iters=None):
    """Measured FMA throughput (TFLOP/s) on the current GPU: 1 FP32 FFMA, 0 FP64
    DFMA, 2 paired FP32 FFMA2, 3 FP16 HFMA2 (libdwf_probe.so, independent chains)."""
    import ctypes
    path = os.path.join(ROOT, "paper_1501_04950_gb300", "libdwf_probe.so")
    lib = ctypes.CDLL(path)
    lib.dwf_probe_fma.restype = ctypes.c_int
    lib.dwf_probe_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    names = {0: "fp64_dfma", 1: "fp32_ffma", 2: "fp32_ffma2", 3: "fp16_hfma2"}
    default_iters = {0: 20000, 1: 200000, 2: 100000, 3: 200000}
    out = {}
    for k in kinds:
        tf, ms = ctypes.c_double(), ctypes.c_double()
        rc = lib.dwf_probe_fma(k, (iters or default_iters)[k], ctypes.byref(tf), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError("FMA probe %d failed (CUDA error %d)" % (k, rc))
        out[names[k]] = round(tf.value, 3)
    return out


def sampled_accuracy(U, src, sol5d, prop, nsites=24, seed=5):
    """5D residual |rhs - D_alpha psi| at sampled 4D sites of a returned solution
    (single-site oracle) over the RMS |rhs| of those sites, and the largest
    deviation of the returned z_1 from P_- psi_1 + P_+ psi_Ls there."""
    import oracle as O
    from oracle.lattice import P_MINUS, P_PLUS
    from oracle.pointwise import PointwiseDalpha
    sysm = O.DWFSystem(LATTICE, LS, M5, MASS, 1.0, np.full(LS, B), np.full(LS, C), U)
    pw = PointwiseDalpha(sysm)
    cache = {}

    def psi_at(c):
        if c not in cache:
            x, y, z, t = c
            cache[c] = sol5d[:, t, z, y, x].cpu().numpy()
        return cache[c]

    rng = np.random.default_rng(seed)
    res, ref, zdev = [], [], 0.0
    for _ in range(nsites):
        site = tuple(int(rng.integers(0, n)) for n in LATTICE)
        x, y, z, t = site
        rhs = pw.rhs_at(src, site)
        res.append(np.linalg.norm(pw.apply_at(psi_at, site) - rhs))
        ref.append(np.linalg.norm(rhs))
        ps = psi_at(site)
        z1 = P_MINUS @ ps[0] + P_PLUS @ ps[LS - 1]
        zdev = max(zdev, float(np.abs(prop[t, z, y, x].cpu().numpy() - z1).max() / np.abs(z1).max()))
    return {"sites": nsites, "resid5d_over_rms_rhs": float(max(res) / np.sqrt(np.mean(np.square(ref)))),
            "z1_extraction_rel_dev": zdev}


def config1_propagator_error():
    """4^4, Ls = 8 Shamir, M5 = -1.8, m = 0.01, eps = 0.3, even-wall Gaussian source:
    the mixed FP32/FP64 GPU solve to 1e-10 against the oracle's FP64 solve to 1e-12,
    max |z_1 - z_1^oracle| / max |z_1^oracle|, and the oracle's CGNE time."""
    import torch
    import oracle as O
    from paper_1501_04950_gb300 import dwf
    from synthetic import gauge_field, gaussian_source4d
    L, Ls = (4, 4, 4, 4), 8
    U = gauge_field(L, 0.3, seed=0)
    src = gaussian_source4d(L, seed=1, even_only=True)
    sysm = O.DWFSystem(L, Ls, M5, 0.01, 1.0, np.ones(Ls), np.zeros(Ls), U)
    t0 = time.perf_counter()
    ref = O.solve_propagator(sysm, src, tol=1e-12)
    t_oracle = time.perf_counter() - t0
    op = dwf.DWF(L, Ls, M5, 0.01, 1.0, np.ones(Ls), np.zeros(Ls))
    op.load_gauge(torch.from_numpy(U).cuda())
    s = torch.from_numpy(src).cuda()
    prop = torch.empty_like(s)
    st = op.cgne_solve(s, prop)[0]
    op.close()
    err = float(np.abs(prop.cpu().numpy() - ref["z1"]).max() / np.abs(ref["z1"]).max())
    return {"workload": "4^4 Ls=8 Shamir m=0.01 eps=0.3, even-wall source", "z1_rel_error": err,
            "true_resid": st["true_resid"], "oracle_iterations": ref["iterations"],
            "oracle_cgne_seconds": t_oracle}


def workload_name(alpha):
    return ("16^3x32 Ls=16 Mobius b=1.5 c=0.5 M5=-1.8 m=0.01 alpha=%g eps=0.5, "
            "Gaussian source; mixed FP32/FP64 CGNE to 1e-10" % alpha)


def replica_throughput(moved, seconds, world, device=None):
    """Whole-job GB/s of N independent replicas (one per rank, no data-path
    collective): the bytes all ranks moved divided by the slowest rank's time
    (sum and max over ranks).  world = 1: moved / seconds."""
    if world > 1:
        import torch
        import torch.distributed as dist
        m = torch.tensor([float(moved)], dtype=torch.float64, device=device)
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(m, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        moved, seconds = float(m.item()), float(t.item())
    return moved / seconds / 1e9


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for name in ["dwf_hop2.cuh", "dwf_fields.cuh", "dwf_internal.cuh"]:
        with open(os.path.join(ROOT, "paper_1501_04950_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic():
    """dram bytes per D_bb apply from the committed ncu summary, if it is current."""
    path = os.path.join(ROOT, "profiles", "dbb_apply_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("kernel_hash") != kernel_hash():
        return None
    return t.get("dram_bytes_per_apply_full_size")


class ClockSampler:
    def __init__(self, index=0):
        self.proc = None
        self.index = index
        self.path = os.path.join(tempfile.gettempdir(), "dwf_bench_clocks_%d.csv" % os.getpid())

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            return parse_clock_samples(f)


def parse_clock_samples(lines):
    """Median SM clock, maximum clock and the throttle reasons seen Active, from
    nvidia-smi --query-gpu=index,clocks.sm,clocks.max.sm,power.draw,
    clocks_event_reasons.{active,hw_slowdown,hw_thermal_slowdown,sw_thermal_slowdown,
    sw_power_cap} rows (csv, noheader, nounits); None without a valid row."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[5:9]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def oracle_apply_sample(reps):
    """Time the FP64 oracle's D_bb apply on the sample lattice; returns (GB/s, seconds list)."""
    import oracle as O
    from synthetic import gauge_field, gaussian_half5d
    U = gauge_field(SAMPLE_LATTICE, EPS, seed=0)
    sysm = O.DWFSystem(SAMPLE_LATTICE, LS, M5, MASS, 1.0, np.full(LS, B), np.full(LS, C), U)
    psi = gaussian_half5d(SAMPLE_LATTICE, LS, seed=2)
    sysm.local_inverse()
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        sysm.dbb(psi)
        times.append(time.perf_counter() - t0)
    n5 = np.prod(SAMPLE_LATTICE) // 2 * LS
    gbs = n5 * bytes_per_site(8, 8, LS) / statistics.median(times) / 1e9
    return gbs, times


def _oracle_worker(reps):
    os.environ["OMP_NUM_THREADS"] = "1"
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    if reps == 0:  # start-up: imports only
        import oracle  # noqa: F401
        import synthetic  # noqa: F401
        return 0.0
    gbs, times = oracle_apply_sample(reps)
    return sum(times)


def oracle_apply_all_cores(reps=2):
    """The oracle's FP64 D_bb apply on the sample lattice in one single-threaded
    process per host core (spawned), all at once: aggregate GB/s and cores."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    n5 = np.prod(SAMPLE_LATTICE) // 2 * LS
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [0] * cores)  # start-up and imports, not timed
        t0 = time.perf_counter()
        pool.map(_oracle_worker, [reps] * cores)
        dt = time.perf_counter() - t0
    return cores * reps * n5 * bytes_per_site(8, 8, LS) / dt / 1e9, cores, dt


def run_reference(args, rank):
    if rank != 0:
        return
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    import oracle as O
    from synthetic import gauge_field, gaussian_half5d
    U = gauge_field(SAMPLE_LATTICE, EPS, seed=0)
    sysm = O.DWFSystem(SAMPLE_LATTICE, LS, M5, MASS, args.alpha, np.full(LS, B), np.full(LS, C), U)
    psi = gaussian_half5d(SAMPLE_LATTICE, LS, seed=2)
    for _ in range(args.warmup):
        sysm.dbb(psi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sysm.dbb(psi)
    dt = time.perf_counter() - t0
    n5 = np.prod(SAMPLE_LATTICE) // 2 * LS
    value = args.steps * n5 * bytes_per_site(8, 8, LS) / dt / 1e9
    sample = "one FP64 D_bb apply per step on an 8^3x16, Ls=16 sub-lattice of the workload"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.alpha), "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_apply_only(args):
    """Time D_bb and D_bb^+ applies alone (inner precision and FP64) with CUDA events."""
    import torch
    from paper_1501_04950_gb300 import dwf
    from synthetic import gauge_field, gaussian_half5d
    lat = tuple(int(v) for v in args.lattice.split(",")) if args.lattice else LATTICE
    dev = torch.device("cuda", 0)
    U = torch.from_numpy(gauge_field(lat, EPS, seed=0)).to(dev)
    op = dwf.DWF(lat, LS, M5, MASS, args.alpha, np.full(LS, B), np.full(LS, C))
    op.load_gauge(U)
    psi = torch.from_numpy(gaussian_half5d(lat, LS, seed=2)).to(dev)
    n5 = op.Vh * LS
    res = {"lattice": list(lat), "Ls": LS}
    for name, prec, ws, wg in [("fp32", dwf.FP32, 4, 4), ("fp16", dwf.FP16, 2, 2),
                               ("bf16", dwf.BF16, 2, 2), ("fp64", dwf.FP64, 8, 8)]:
        x = op.new_field(prec)
        y = op.new_field(prec)
        op.pack_half(x, psi, prec)
        for fn, key in [(op.apply_Dbb, "dbb"), (op.apply_Dbb_dag, "dbb_dag")]:
            reps = args.apply_only if prec != dwf.FP64 else max(1, args.apply_only // 10)
            for _ in range(3):
                fn(y, x, prec)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn(y, x, prec)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            gbs = n5 * bytes_per_site(ws, wg, LS) / (ms / 1e3) / 1e9
            res["%s_%s_us" % (key, name)] = round(ms * 1e3, 2)
            res["%s_%s_gbs" % (key, name)] = round(gbs, 1)
    print(json.dumps(res), flush=True)


def run_batched(args):
    """Batched propagator solves: 12 point sources x alpha in {1, 1.5} in one call per lattice.

    Reports, per lattice, solves per second and the per-solve latency (time from the
    start of its batch to its convergence) p50 / p99, for the FP32-inner solver
    (autotuned right-hand-side block) and the plain FP64 GPU CG.
    """
    import torch
    from paper_1501_04950_gb300 import dwf
    from synthetic import gauge_field, point_source4d
    dev = torch.device("cuda", 0)
    out = []
    lats = [tuple(int(v) for v in lat.split("x")) for lat in args.batched.split(",")]
    # launch shapes tuned by the first solve of a lattice are reused by later handles
    own_cache = "DWF_AUTOTUNE_CACHE" not in os.environ
    if own_cache:
        os.environ["DWF_AUTOTUNE_CACHE"] = os.path.join(
            tempfile.gettempdir(), "dwf_bench_tune_%d.txt" % os.getpid())
    for lat, L in zip(args.batched.split(","), lats):
        U = torch.from_numpy(gauge_field(L, EPS, seed=0)).to(dev)
        srcs = [point_source4d(L, sp, c) for sp in range(4) for c in range(3)]
        src = torch.from_numpy(np.stack(srcs + srcs)).to(dev)
        alphas = [1.0] * 12 + [1.5] * 12
        prop = torch.empty_like(src)
        row = {"lattice": lat, "Ls": LS, "nrhs": 24}
        for name, opts in [("mixed_fp32", {}), ("mixed_fp16", {"precision_inner": dwf.FP16})]:
            op = dwf.DWF(L, LS, M5, MASS, 1.0, np.full(LS, B), np.full(LS, C), **opts)
            op.load_gauge(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = op.cgne_solve(src, prop, nrhs=24, alphas=alphas, allow_not_converged=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            lat_s = sorted(x["seconds"] for x in st)
            row[name] = {
                "seconds": dt, "solves_per_s": 24 / dt,
                "latency_p50_s": float(np.percentile(lat_s, 50)),
                "latency_p99_s": float(np.percentile(lat_s, 99)),
                "iterations_alpha1": int(np.mean([x["iterations"] for x in st[:12]])),
                "iterations_alpha1.5": int(np.mean([x["iterations"] for x in st[12:]])),
                "max_true_resid": max(x["true_resid"] for x in st),
            }
            op.close()
        out.append(row)
        print(json.dumps(row), flush=True)
    if len(lats) > 1:
        out.append(run_multi_lattice(lats, dev, 24))
    # several small single-source problems, none of which fills the GPU alone
    small = [(8, 8, 8, 8), (8, 8, 8, 16), (8, 8, 16, 16), (12, 12, 12, 12)]
    out.append(run_multi_lattice(small, dev, 1))
    if own_cache:
        path = os.environ.pop("DWF_AUTOTUNE_CACHE")
        if os.path.exists(path):
            os.remove(path)
    return out


def run_multi_lattice(lats, dev, nrhs):
    """Point-source solves on several lattices (FP32 inner; nrhs sources each: the 12
    spin-colour sources at alpha 1 and, for 24, again at alpha 1.5) solved one lattice
    after another, then all in one dwf_cgne_solve_multi call (one host thread and stream
    per lattice), on the same tuned handles."""
    import torch
    from paper_1501_04950_gb300 import dwf
    from synthetic import gauge_field, point_source4d
    ops, jobs = [], []
    alphas = ([1.0] * 12 + [1.5] * 12)[:nrhs]
    for L in lats:
        U = torch.from_numpy(gauge_field(L, EPS, seed=0)).to(dev)
        srcs = [point_source4d(L, sp, c) for sp in range(4) for c in range(3)]
        src = torch.from_numpy(np.stack((srcs + srcs)[:nrhs])).to(dev)
        op = dwf.DWF(L, LS, M5, MASS, 1.0, np.full(LS, B), np.full(LS, C))
        op.load_gauge(U)
        ops.append(op)
        jobs.append((op, src, torch.empty_like(src), nrhs, alphas))
    if nrhs == 1:  # first-use costs (launch-shape tuning, workspace) outside the timing
        for op, src, prop, n, al in jobs:
            op.cgne_solve(src, prop, nrhs=n, alphas=al, allow_not_converged=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for op, src, prop, n, al in jobs:
        op.cgne_solve(src, prop, nrhs=n, alphas=al, allow_not_converged=True)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    st = dwf.cgne_solve_multi(jobs, allow_not_converged=True)
    torch.cuda.synchronize()
    t_multi = time.perf_counter() - t0
    nsolve = nrhs * len(lats)
    row = {"multi_lattice_one_call": {
        "lattices": ["x".join(str(v) for v in L) for L in lats], "Ls": LS, "nrhs_each": nrhs,
        "sequential_seconds": t_seq, "one_call_seconds": t_multi,
        "solves_per_s_sequential": nsolve / t_seq, "solves_per_s_one_call": nsolve / t_multi,
        "max_true_resid": max(x["true_resid"] for s in st for x in s)}}
    for op in ops:
        op.close()
    print(json.dumps(row), flush=True)
    return row


def run_zolotarev(args):
    """Zolotarev alpha-Mobius solve, 24^3x48, Ls = 12 (b_i + c_i = 1/omega_i from the
    minimax sign approximation on [0.05, 6], concave order), m = 0.005, alpha = 1.25,
    Gaussian b_1: time to FP64 true residual 1e-10 per inner precision and solver."""
    import torch
    from paper_1501_04950_gb300 import dwf
    from synthetic import gauge_field, gaussian_source4d, zolotarev_mobius
    dev = torch.device("cuda", 0)
    L, Ls, m, alpha = (24, 24, 24, 48), 12, 0.005, 1.25
    b, c, _, _ = zolotarev_mobius(Ls, 0.05, 6.0)
    U = torch.from_numpy(gauge_field(L, EPS, seed=0)).to(dev)
    src = torch.from_numpy(gaussian_source4d(L, seed=1)).to(dev)
    prop = torch.empty_like(src)
    row = {"workload": "24^3x48 Ls=12 Zolotarev [0.05,6] concave, M5=-1.8 m=0.005 alpha=1.25 "
                       "eps=0.5, Gaussian b_1; CGNE to FP64 true residual 1e-10"}
    variants = [("fp32_reliable", dict(precision_inner=dwf.FP32)),
                ("fp16_reliable", dict(precision_inner=dwf.FP16)),
                ("fp16_defect", dict(precision_inner=dwf.FP16, solver=dwf.SOLVER_DEFECT)),
                ("bf16_defect", dict(precision_inner=dwf.BF16, solver=dwf.SOLVER_DEFECT)),
                ("fp64", dict(solver=dwf.SOLVER_FP64))]
    warm = dwf.DWF(L, Ls, M5, m, alpha, b, c, maxiter=64)
    warm.load_gauge(U)
    warm.cgne_solve(src, prop, allow_not_converged=True)  # first-use costs, not timed
    warm.close()
    for name, opts in variants:
        op = dwf.DWF(L, Ls, M5, m, alpha, b, c, maxiter=100000, **opts)
        op.load_gauge(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = op.cgne_solve(src, prop, allow_not_converged=True)[0]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        row[name] = {"solve_ms": dt * 1e3, "iterations": st["iterations"],
                     "restarts": st["restarts"], "true_resid": st["true_resid"],
                     "true_resid_5d": st["true_resid_5d"]}
        op.close()
    print(json.dumps(row), flush=True)
    return row


def sign_error(a, xmin=0.05, xmax=6.0, n=20001):
    """max |1 - R(x)| on [xmin, xmax] of the rational sign approximation
    R = [prod(1 + a_i x) - prod(1 - a_i x)] / [prod(1 + a_i x) + prod(1 - a_i x)]
    (the polar form of App. A) for coefficients a_i = b_i + c_i."""
    x = np.geomspace(xmin, xmax, n)
    ax = np.outer(x, np.asarray(a, dtype=np.float64))
    lp = np.log(np.abs(1.0 + ax)).sum(axis=1)
    lm = np.log(np.abs(1.0 - ax)).sum(axis=1)
    r = np.exp(lm - lp) * np.prod(np.sign(1.0 - ax), axis=1)
    return float(np.max(np.abs(1.0 - (1.0 - r) / (1.0 + r))))


def run_zolo_projection(args, lattice=(16, 16, 16, 32), ls_zolo=8, ls_mobius=32, mass=0.06,
                        alphas=(0.3, 0.4, 0.5, 0.6, 0.8, 1.0), tol=1e-8):
    """Sec. 3 projects that Zolotarev coefficients in concave order together with
    alpha make the solve "2 to 3 times faster".  Measured here: time and
    iterations to the FP64 true residual `tol` (FP32 inner CG) of one point source
    for (1) Zolotarev, concave, best alpha of a scan; (2) the same at alpha = 1;
    (3) Mobius b = 1.5, c = 0.5 at alpha = 1 with Ls chosen for at least the same
    sign-function accuracy on [0.05, 6]."""
    import torch
    from paper_1501_04950_gb300 import dwf
    from synthetic import gauge_field, point_source4d, zolotarev_mobius
    dev = torch.device("cuda", 0)
    U = torch.from_numpy(gauge_field(lattice, EPS, seed=0)).to(dev)
    src1 = torch.from_numpy(point_source4d(lattice, 0, 0)).to(dev)
    bz, cz, _, _ = zolotarev_mobius(ls_zolo, 0.05, 6.0)
    bm, cm = np.full(ls_mobius, B), np.full(ls_mobius, C)
    out = {"workload": "%s Zolotarev Ls=%d (concave) vs Mobius b=1.5 c=0.5 Ls=%d, M5=-1.8 m=%g "
                       "eps=0.5, point source, FP32 inner CG to FP64 true residual %g"
                       % ("x".join(map(str, lattice)), ls_zolo, ls_mobius, mass, tol),
           "sign_error_zolotarev": sign_error(bz + cz), "sign_error_mobius": sign_error(bm + cm)}
    # alpha scan of the Zolotarev operator (one batched call, iteration counts exact to 2)
    op = dwf.DWF(lattice, ls_zolo, M5, mass, 1.0, bz, cz, rel_tol=tol, check_every=2)
    op.load_gauge(U)
    srcn = src1.unsqueeze(0).repeat(len(alphas), *([1] * src1.dim())).contiguous()
    prop = torch.empty_like(srcn)
    st = op.cgne_solve(srcn, prop, nrhs=len(alphas), alphas=list(alphas))
    op.close()
    its = [x["iterations"] for x in st]
    best = alphas[int(np.argmin(its))]
    out["zolotarev_alpha_scan"] = {"alphas": list(alphas), "iterations": its}

    def timed(Ls, b, c, alpha, reps=2):
        o = dwf.DWF(lattice, Ls, M5, mass, alpha, b, c, rel_tol=tol)
        o.load_gauge(U)
        p = torch.empty_like(src1)
        o.cgne_solve(src1, p)  # first-use costs, not timed
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            s = o.cgne_solve(src1, p)[0]
        torch.cuda.synchronize()
        o.close()
        return {"Ls": Ls, "alpha": alpha, "iterations": s["iterations"],
                "seconds": (time.perf_counter() - t0) / reps, "true_resid": s["true_resid"],
                "iterations_x_Ls": s["iterations"] * Ls}

    out["zolotarev_best_alpha"] = timed(ls_zolo, bz, cz, best)
    out["zolotarev_alpha1"] = timed(ls_zolo, bz, cz, 1.0)
    out["mobius_alpha1"] = timed(ls_mobius, bm, cm, 1.0)
    m, z = out["mobius_alpha1"], out["zolotarev_best_alpha"]
    out["factor_time"] = m["seconds"] / z["seconds"]
    out["factor_iterations_x_Ls"] = m["iterations_x_Ls"] / z["iterations_x_Ls"]
    out["factor_alpha_only"] = out["zolotarev_alpha1"]["seconds"] / z["seconds"]
    print(json.dumps(out), flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--alpha", type=float, default=1.0)
    ap.add_argument("--inner", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the alpha sweep")
    ap.add_argument("--no-fp16", action="store_true",
                    help="skip the FP16-inner solve of the workload after the timed region")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the sampled-site accuracy checks after the timed region")
    ap.add_argument("--apply-only", type=int, default=0,
                    help="run this many D_bb and D_bb^+ applies of the workload and report their "
                         "CUDA-event times (the case the ncu captures use)")
    ap.add_argument("--lattice", default=None, help="override Lx,Ly,Lz,Lt (apply-only mode)")
    ap.add_argument("--batched", default=None,
                    help="batched mode: comma-separated lattices such as 8x8x8x8,16x16x16x32; "
                         "12 spin-colour point sources x alpha in {1, 1.5} per lattice")
    ap.add_argument("--zolotarev", action="store_true",
                    help="Zolotarev 24^3x48, Ls=12, m=0.005 solve per inner precision")
    ap.add_argument("--zolo-projection", action="store_true",
                    help="Sec. 3 projection: Zolotarev + alpha against Mobius at matched "
                         "sign-function accuracy (time and iterations to 1e-8)")
    ap.add_argument("--peaks", action="store_true",
                    help="measured FMA throughput of the GPU (FP64, FP32, paired FP32, FP16)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.apply_only:
        run_apply_only(args)
        return
    if args.batched:
        run_batched(args)
        return
    if args.zolotarev:
        run_zolotarev(args)
        return
    if args.zolo_projection:
        lat = tuple(int(v) for v in args.lattice.split(",")) if args.lattice else (16, 16, 16, 32)
        run_zolo_projection(args, lattice=lat)
        return
    if args.peaks:
        print(json.dumps({"fma_tflops": probe_fma_peaks(kinds=(0, 1, 2, 3))}), flush=True)
        return

    import torch
    import torch.distributed as dist
    from paper_1501_04950_gb300 import dwf
    from synthetic import gauge_field, gaussian_source4d

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    inner = {"fp32": dwf.FP32, "fp16": dwf.FP16, "bf16": dwf.BF16}[args.inner]
    ws_bytes = {dwf.FP32: 4, dwf.FP16: 2, dwf.BF16: 2}[inner]
    wg_bytes = 4 if inner == dwf.FP32 else 2

    U = torch.from_numpy(gauge_field(LATTICE, EPS, seed=0)).to(dev)
    src_h = torch.from_numpy(gaussian_source4d(LATTICE, seed=1 + rank)).pin_memory()
    src = src_h.to(dev)
    prop = torch.empty_like(src)
    prop_h = torch.empty_like(src_h).pin_memory()
    op = dwf.DWF(LATTICE, LS, M5, MASS, args.alpha, np.full(LS, B), np.full(LS, C),
                 precision_inner=inner, profile=1)
    op.load_gauge(U)
    torch.cuda.synchronize()
    n5 = op.Vh * LS
    b_inner = n5 * bytes_per_site(ws_bytes, wg_bytes, LS)
    b_fp64 = n5 * bytes_per_site(8, 8, LS)

    def barrier():
        if world > 1:
            dist.barrier()

    def maxtime(t):
        if world > 1:
            x = torch.tensor([t], dtype=torch.float64, device=dev)
            dist.all_reduce(x, op=dist.ReduceOp.MAX)
            return float(x.item())
        return t

    for _ in range(args.warmup):
        op.cgne_solve(src, prop)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats += op.cgne_solve(src, prop)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    dt_local = e0.elapsed_time(e1) / 1e3
    dt = maxtime(dt_local)
    applies = sum(s["applies"] + s["applies_dag"] for s in stats)
    applies64 = sum(s["applies_fp64"] for s in stats)
    moved = applies * b_inner + applies64 * b_fp64
    value = replica_throughput(moved, dt_local, world, dev)
    apply_ms = sum(s["apply_ms"] for s in stats)
    n_timed = sum(s["applies_timed"] for s in stats)
    achieved = n_timed * b_inner / (apply_ms / 1e3) / 1e9 if apply_ms > 0 else None
    peak, peak_kind = peaks()
    launches = sum(s["kernel_launches"] for s in stats)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_stats = []
    for _ in range(args.steps):
        e2e_stats += op.cgne_solve(src_h, prop_h)
    torch.cuda.synchronize()
    dt_e2e_local = time.perf_counter() - t0
    moved_e2e = sum((s["applies"] + s["applies_dag"]) * b_inner + s["applies_fp64"] * b_fp64
                    for s in e2e_stats)
    value_e2e = replica_throughput(moved_e2e, dt_e2e_local, world, dev)
    io_bytes = src_h.numel() * 16

    fp64 = None
    if not args.no_fp64_baseline:
        op64 = dwf.DWF(LATTICE, LS, M5, MASS, args.alpha, np.full(LS, B), np.full(LS, C),
                       solver=dwf.SOLVER_FP64)
        op64.load_gauge(U)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s64 = op64.cgne_solve(src, prop)[0]
        torch.cuda.synchronize()
        fp64 = {"solve_ms": (time.perf_counter() - t0) * 1e3, "iterations": s64["iterations"],
                "true_resid": s64["true_resid"]}
        op64.close()

    # the same workload with FP16 inner fields (FP64 and FP32-tier residual
    # replacements), outside the timed region: one warm-up solve, then two timed
    inner16 = None
    if rank == 0 and inner == dwf.FP32 and not args.no_fp16:
        op16 = dwf.DWF(LATTICE, LS, M5, MASS, args.alpha, np.full(LS, B), np.full(LS, C),
                       precision_inner=dwf.FP16)
        op16.load_gauge(U)
        prop16 = torch.empty_like(src)
        op16.cgne_solve(src, prop16)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s16 = [op16.cgne_solve(src, prop16)[0] for _ in range(2)][-1]
        f1.record(stream)
        torch.cuda.synchronize()
        inner16 = {"time_to_1e-10_ms": f0.elapsed_time(f1) / 2, "iterations": s16["iterations"],
                   "fp64_replacements": s16["restarts"], "fp32_replacements": s16["applies_fp32"],
                   "true_resid": s16["true_resid"],
                   "z1_rel_diff_vs_fp32": float((prop16 - prop).abs().max() / prop.abs().max())}
        op16.close()

    # accuracy of the timed workload's solution (outside the timed region): one
    # more solve with the full 5D solution, checked at sampled sites
    accuracy = None
    if rank == 0 and not args.no_accuracy:
        sol5d = torch.empty((LS,) + tuple(src.shape), dtype=torch.complex128, device=dev)
        op.cgne_solve(src, prop, sol5d)
        torch.cuda.synchronize()
        accuracy = sampled_accuracy(U.cpu().numpy(), src.cpu().numpy(), sol5d, prop)
        del sol5d
        accuracy["config1"] = config1_propagator_error()
    alu = None
    if rank == 0:
        pk = probe_fma_peaks(kinds=(1, 0))
        gflops = n_timed * n5 * FLOP_PER_SITE / (apply_ms / 1e3) / 1e9 if apply_ms > 0 else None
        alu = {"flop_per_site": FLOP_PER_SITE, "gflops": gflops, "peak_tflops": pk["fp32_ffma"],
               "frac": gflops / (pk["fp32_ffma"] * 1e3) if gflops else None,
               "peak_kind": "measured FP32 FFMA (libdwf_probe, this run)",
               "fp64_dfma_tflops": pk["fp64_dfma"]}

    sweep = None
    if not args.no_sweep:
        # config-2 alpha sweep: one batched call per solver, the same source for every alpha
        alphas = [0.5, 0.75, 1.0, 1.25, 1.5, 2.0]
        src6 = src.unsqueeze(0).repeat(len(alphas), *([1] * src.dim())).contiguous()
        prop6 = torch.empty_like(src6)
        sweep = {"alphas": alphas}
        for name, opts in [("mixed_fp32", {}), ("fp64", {"solver": dwf.SOLVER_FP64})]:
            ops = dwf.DWF(LATTICE, LS, M5, MASS, 1.0, np.full(LS, B), np.full(LS, C),
                          rhs_block=len(alphas), **opts)
            ops.load_gauge(U)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st6 = ops.cgne_solve(src6, prop6, nrhs=len(alphas), alphas=alphas)
            torch.cuda.synchronize()
            sweep[name] = {"batch_seconds": time.perf_counter() - t0,
                           "iterations": [x["iterations"] for x in st6],
                           "seconds_to_converge": [round(x["seconds"], 4) for x in st6],
                           "true_resid": [x["true_resid"] for x in st6]}
            ops.close()
        it1 = sweep["mixed_fp32"]["iterations"][2]
        sweep["relative_iterations"] = [round(x / it1, 4) for x in sweep["mixed_fp32"]["iterations"]]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        gbs, times = oracle_apply_sample(3)
        all_gbs, cores, dt_all = oracle_apply_all_cores(reps=2)
        cpu = {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": "median of 3 FP64 D_bb applies on an 8^3x16, Ls=16 sub-lattice "
                         "(%.1f s each)" % statistics.median(times),
               "all_cores": {"value": all_gbs, "unit": "GB/s", "cores": cores,
                             "sample": "2 applies of the same sub-lattice in each of %d "
                                       "single-threaded processes at once (%.1f s)"
                                       % (cores, dt_all)},
               "config1_cgne_seconds": accuracy["config1"]["oracle_cgne_seconds"] if accuracy else None,
               "config1_cgne_note": "oracle FP64 CGNR to 1e-12 on 4^4, Ls=8 (1 core)"}

    if rank == 0:
        solve_ms = dt / args.steps * 1e3
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": solve_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if inner == dwf.FP32 else args.inner, "data": "synthetic",
            "config": {"workload": workload_name(args.alpha), "lattice": list(LATTICE), "Ls": LS,
                       "inner": args.inner, "rel_tol": 1e-10, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "working set (gauge + ~8 half-fields, >1 GB) exceeds the 129 MB L2"},
            "solve": {"time_to_1e-10_ms": solve_ms, "iterations": stats[0]["iterations"],
                      "reliable_updates": stats[0]["restarts"], "true_resid": stats[0]["true_resid"],
                      "true_resid_5d": stats[0]["true_resid_5d"],
                      "fp64_plain": fp64,
                      "speedup_vs_fp64": (fp64["solve_ms"] / solve_ms) if fp64 else None,
                      "fp16_inner": inner16},
            "accuracy": accuracy,
            "alu": alu,
            "roofline": {"kernel": "D_bb apply inside the CG (pass A on B p, pass B; FP32); "
                                   "CUDA events around the applies of the first iteration "
                                   "after each convergence poll",
                         "timed_applies": n_timed,
                         "bound": "hbm",
                         "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                         "peak_kind": peak_kind, "traffic": measured_traffic(),
                         "bytes_per_apply": b_inner},
            "alpha_sweep": sweep,
            "cpu_baseline": cpu,
            "e2e": {"value": value_e2e, "unit": "GB/s",
                    "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
