#!/usr/bin/env python3
"""Benchmark of the REXI linear step (arXiv 1805.06557, Eq. rexi) on GB300.

Workload: T255 spectral states (geopotential, vorticity, divergence; n^-1.5 Gaussian
coefficients, seeded), N = 512 Cauchy-contour poles (p0 = 14, Xc = 1.4 X), dt = 3600 s,
a batch of 16 independent states per rank per step.  One step = one rexi_step call on the
batch (pre-pass, light/heavy mixed-precision solves with the fused pole sums, finalize).

Headline `value`: state-steps/s of the batched mixed-precision plan (all ranks).  Also
reported: the plain FP64 plan one state at a time and batched, the mixed plan one state at
a time, p50/p99 step latency, the mixed-vs-FP64 error, the dominant kernel's roofline, the
end-to-end rate through rexi_step_host with host buffers, and the CPU oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import datetime
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "REXI steps/s at T255, batched/mixed vs plain FP64 at ≤1e-8 rel err; p50/p99"
T_DEF, N_DEF, DT_DEF, B_DEF = 255, 512, 3600.0, 16
SAMPLE_M = list(range(0, 256))         # cpu_baseline sample: every zonal order of SAMPLE_STATES states
SAMPLE_STATES = 3

# Algorithmic flops (FMA = 2) per chain element and pole of the solve kernels, and the pipe
# they run on.  Light (FP32 Thomas, FP32 pole sums) and FP64 paths: forward elimination 22,
# back substitution 8, right-hand side and diagonal 7, weighted pole sums 12.  Heavy (FP32
# solve + one refinement step): FP32 factor and solve 38, residual r - A x in double-float
# arithmetic 228 (zeta rows 165, delta rows 291), correction solve 20, double-float pole sums 90.
# Algorithmic work of the method per chain element of one pole (one (pole, m, n, chain); FMA = 2):
# forward elimination 22, back substitution 8, right-hand side and diagonal 7, weighted pole sums
# 12 -- the same count for every solve kernel (about 100 flops per pole-mode), and the pipe the
# kernel runs it on.  The roofline fraction is taken on this count.
KERNEL_FLOPS = {"k_rexi_light": (49.0, "fp32"), "k_rexi_heavy": (49.0, "fp32"),
                "k_rexi_fp64": (49.0, "fp64")}
# Flops the heavy kernel executes per chain element to reach FP64-level accuracy from FP32
# arithmetic: FP32 factor and solve 38, residual 168 (double-float row, then compensated dot
# products: zeta rows 118, delta rows 219), correction solve 20, double-float pole sums 90
# (reported beside the algorithmic fraction, not instead of it)
EXECUTED_FLOPS = {"k_rexi_light": 49.0, "k_rexi_heavy": 316.0, "k_rexi_fp64": 49.0}
# DRAM bytes (read + write) of one launch from an ncu capture: (bytes, batch of that launch,
# summary file).  Only for kernels unchanged since the capture.
TRAFFIC = {"k_rexi_heavy": (2.271e9, 16, "profiles/rexi_solve_T255_B16.md")}


def shard_seeds(rank, batch):
    """Seeds of the states rank `rank` owns: ranks hold disjoint, independent states
    (the units of the job are sharded, no data-path collective)."""
    return [1000 + rank * batch + i for i in range(batch)]


def job_rate(local_ms, batch, world, steps, dist=None, device="cpu"):
    """Whole-job state-steps/s from each rank's timed-region length: the slowest rank's
    time (max over ranks) bounds the job.  Returns (value, max_ms)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return batch * world * steps / (max_ms * 1e-3), max_ms


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=B_DEF)
    ap.add_argument("--T", type=int, default=T_DEF)
    ap.add_argument("--N", type=int, default=N_DEF)
    ap.add_argument("--dt", type=float, default=DT_DEF)
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the ragged-ensemble figure")
    ap.add_argument("--no-sh", action="store_true",
                    help="skip the SH-transform and nonlinear SWE-step figures")
    ap.add_argument("--dt-sweep", action="store_true",
                    help="error vs time-step size of the nonlinear schemes instead (T127, 12 h)")
    ap.add_argument("--serving", type=int, default=0,
                    help="run the request-stream workload with this many requests instead")
    ap.add_argument("--sh-only", nargs="?", const="fp64,tf32,bf16,tf32x3,df", default=None,
                    help="run only the SH-transform figures, for these Legendre precisions "
                         "(comma list; default all)")
    ap.add_argument("--sh-T", type=int, default=511,
                    help="truncation of --sh-only (Gauss grid 3(T+1)/2 x 3(T+1))")
    return ap.parse_args()


def contour(X):
    """Contour of the benchmark and parity tests: p0 <= Xc, Xc = 1.6 X for X < 20 else
    p0 = 14, Xc = 1.4 X (chosen by a search minimising max(e_s, amplification * eps))."""
    if X < 20:
        return min(6.0, 1.6 * X), 1.6 * X
    return 14.0, 1.4 * X


def workload_config(args, world):
    return {"workload": "REXI linear step, T%d, %d Cauchy poles, dt=%g s, batch %d states/GPU, "
                        "n^-1.5 Gaussian spectral states" % (args.T, args.N, args.dt, args.batch),
            "T": args.T, "N_poles": args.N, "dt_s": args.dt, "batch_per_gpu": args.batch,
            "global_batch": args.batch * world, "precision": "mixed (FP32 solves, FP64 pole sums)",
            "l2": "flushed (256 MB write) between timed steps",
            "parallelism": "independent states sharded over GPUs, no collective"}


# ---------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling (every 50 ms) of SM clocks and throttle reasons during the timed
    region: start() returns once the sampler has written its first line, so that the region
    begins with the sampler running; region_start() / stop() bracket the region, and the
    summary uses the samples whose timestamps fall inside it (all samples if none do, as the
    region can be shorter than the sampling interval)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0
            while time.time() < deadline and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t0 = time.time()

    def region_start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = None
            try:
                rows.append((ts, float(f[2]), float(f[3]), {nm for nm, v in zip(names, f[6:10])
                                                             if v.lower().startswith("active")}))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        inside = [r for r in rows if r[0] is not None and self.t0 - 0.025 <= r[0] <= self.t1 + 0.025]
        use = inside or rows
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in use),
                "reasons": sorted(set().union(*(r[3] for r in use))), "samples": len(use),
                "samples_in_region": len(inside), "region_s": round(self.t1 - self.t0, 4)}


# ---------------------------------------------------------------------------------------
def thomas_rexi_step(U0, T, dt, omega, radius, phibar, z, w, chunk=64, threads=None):
    """Vectorised FP64 CPU REXI step, the fair CPU baseline (not the oracle): for every pole
    z_p and zonal order m, Phi is eliminated from (z_p - dt L_m) u = b (Phi_n = (b_Phi,n -
    dt Phibar delta_n) / z_p) and the zeta/delta coupling splits into two tridiagonal chains by
    the parity of n - m, solved by Thomas elimination without pivoting.  Arrays are [row j of
    the chain (n = m + j)][pole][m], so one elimination step is one contiguous numpy operation
    over `chunk` poles and all zonal orders; pole chunks run in `threads` threads (numpy
    releases the interpreter lock inside its array operations); U1 = sum_p w_p u_p.
    U0: [3, nlm] complex128 (Phi', zeta, delta), m-major."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    M = T + 1
    jj, mm = np.meshgrid(np.arange(M), np.arange(M), indexing="ij")  # [j, m], n = m + j
    n = (mm + jj).astype(float)
    valid = (mm + jj) <= T
    off = mm * (2 * T + 3 - mm) // 2
    idx = np.where(valid, off + jj, 0)
    b = [np.where(valid, U0[f][idx], 0.0) for f in range(3)]
    nz = valid & (n > 0)
    nn = np.where(nz, n, 1.0)
    eps = lambda k: np.sqrt(np.clip((k * k - mm * mm) / (4.0 * k * k - 1.0), 0.0, None))
    om = np.where(nz, 2.0 * omega * mm / (nn * (nn + 1.0)), 0.0)
    q = np.where(nz, n * (n + 1.0) / (radius * radius), 0.0)
    # couplings of row n to n - 1 and n + 1 (times dt); dropped at n - 1 = 0 and beyond T
    cm = np.where(nz & (jj > 0) & (n - 1 > 0), dt * 2.0 * omega * (nn + 1.0) / nn * eps(nn), 0.0)
    cp = np.where(valid & (mm + jj + 1 <= T), dt * 2.0 * omega * n / (n + 1.0) * eps(n + 1.0), 0.0)
    zs = np.asarray(z, dtype=np.complex128)
    ws = np.asarray(w, dtype=np.complex128)

    def solve(p0):
        Z = zs[p0:p0 + chunk][None, :, None]  # [1, P, 1]
        W = ws[p0:p0 + chunk]
        dZ = np.where(nz[:, None, :], Z - 1j * dt * om[:, None, :], Z)
        dD = np.where(nz[:, None, :], dZ + dt * dt * phibar * q[:, None, :] / Z, Z)
        rD = np.where(nz[:, None, :], b[2][:, None, :] + dt * q[:, None, :] * b[0][:, None, :] / Z,
                      b[2][:, None, :])
        zeta = np.empty(dZ.shape, dtype=np.complex128)
        delta = np.empty(dZ.shape, dtype=np.complex128)
        for c in (0, 1):  # chain c: zeta rows where j % 2 == c, delta rows elsewhere
            cpr = np.empty(dZ.shape, dtype=np.complex128)
            y = np.empty(dZ.shape, dtype=np.complex128)
            cprev = np.zeros(dZ.shape[1:], dtype=np.complex128)
            yprev = np.zeros(dZ.shape[1:], dtype=np.complex128)
            for j in range(M):
                isZ = (j % 2) == c
                sg = 1.0 if isZ else -1.0
                d = np.where(valid[j], dZ[j] if isZ else dD[j], 1.0)
                r = np.where(valid[j], b[1][j] if isZ else rD[j], 0.0)
                lo, up = sg * cm[j], sg * cp[j]
                piv = d - lo * cprev
                cprev = up / piv
                yprev = (r - lo * yprev) / piv
                cpr[j] = cprev
                y[j] = yprev
            xn = np.zeros(dZ.shape[1:], dtype=np.complex128)
            for j in range(M - 1, -1, -1):
                xn = y[j] - cpr[j] * xn
                if (j % 2) == c:
                    zeta[j] = xn
                else:
                    delta[j] = xn
        phi = np.where(nz[:, None, :], (b[0][:, None, :] - dt * phibar * delta) / Z, b[0][:, None, :] / Z)
        return [np.einsum("p,jpm->jm", W, v) for v in (phi, zeta, delta)]

    starts = list(range(0, len(zs), chunk))
    nthr = threads or min(len(starts), os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=nthr) as ex:
        parts = list(ex.map(solve, starts))
    U1 = np.zeros((3, (T + 1) * (T + 2) // 2), dtype=np.complex128)
    for f in range(3):
        acc = parts[0][f].copy()
        for pr in parts[1:]:  # pole chunks summed in their fixed order
            acc += pr[f]
        U1[f][idx[valid]] = acc[valid]
    return U1


def cpu_thomas_rate(T, N, dt, states):
    """The vectorised numpy Thomas baseline over whole steps of the given states: (steps/s,
    seconds)."""
    from paper_1805_06557_gb300 import rexi
    from paper_1805_06557_gb300 import synthetic as syn
    X = rexi.spectrum_bound(T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = contour(X)
    z, w = rexi.coeffs(N, p0, Xc)
    t0 = time.perf_counter()
    for U in states:
        thomas_rexi_step(U, T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w)
    sec = time.perf_counter() - t0
    return len(states) / sec, sec


def cpu_oracle_rate(T, N, dt, m_list, states):
    """Oracle (pivoted banded LU per pole and zonal order, FP64 sum) on the zonal orders
    m_list of each state; returns (state-steps/s extrapolated to the full step, seconds)."""
    from oracle import coeffs as oc
    from oracle import rexi as orx
    from paper_1805_06557_gb300 import synthetic as syn
    X = orx.spectrum_bound(T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = contour(X)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    work = sum(T + 1 - m for m in m_list)
    full = (T + 1) * (T + 2) // 2
    t0 = time.perf_counter()
    for U in states:
        orx.rexi_step(U, T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w, m_list=m_list)
    sec = time.perf_counter() - t0
    per_state = sec / len(states) * full / work
    return 1.0 / per_state, sec


def _oracle_orders(args):
    """Worker of the reference arm: the oracle's step restricted to some zonal orders."""
    from oracle import rexi as orx
    U, T, dt, omega, radius, phibar, z, w, ms = args
    return orx.rexi_step(U, T, dt, omega, radius, phibar, z, w, m_list=ms)


def _balanced_orders(T, parts):
    """Zonal orders 0..T dealt into `parts` lists of about equal work (T + 1 - m per order),
    largest first to the least loaded list."""
    load = [0] * parts
    out = [[] for _ in range(parts)]
    for m in range(T + 1):
        k = load.index(min(load))
        out[k].append(m)
        load[k] += T + 1 - m
    return [sorted(o) for o in out if o]


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on full steps of one state (every pole
    and zonal order), the zonal orders spread over worker processes on the host cores (each
    runs the oracle's own step on its orders; the step is their sum).  Rank 0 only."""
    if rank != 0:
        return
    import multiprocessing as mp
    import numpy as np
    from oracle import coeffs as oc
    from oracle import rexi as orx
    from paper_1805_06557_gb300 import synthetic as syn
    T, N, dt = args.T, args.N, args.dt
    U = syn.gaussian_state(T, 1000)
    X = orx.spectrum_bound(T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = contour(X)
    z, w = oc.rexi_coefficients(N, p0, Xc)
    cores = max(1, min(os.cpu_count() or 1, T + 1))
    chunks = _balanced_orders(T, cores)
    jobs = [(U, T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, z, w, ms) for ms in chunks]
    times = []
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            U1 = sum(pool.map(_oracle_orders, jobs))
            sec = time.perf_counter() - t0
            if i >= args.warmup:
                times.append(sec)
    assert np.all(np.isfinite(U1))
    per = statistics.mean(times)
    value = 1.0 / per
    cfg = workload_config(args, 1)
    cfg["precision"] = "FP64 (oracle)"
    sample = ("full steps: every pole and all %d zonal orders of one T%d state per step, the orders "
              "spread over %d worker processes" % (T + 1, T, len(chunks)))
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "impl": "reference",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": len(chunks), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
def ensemble(torch, rexi, syn, steps):
    """Ragged ensemble: 64 states of truncation T ~ U{63..255} (seed 3), 512 poles each,
    dt = 3600 s, one ragged launch per step replayed from a captured CUDA graph after the
    tile-density autotuner; mixed precision, error per field against the FP64 ragged plan."""
    import numpy as np
    Ts = syn.ensemble_truncations(64, seed=3)
    dt, N = 3600.0, 512
    inst = []
    for T in Ts:
        X = rexi.spectrum_bound(T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
        p0, Xc = contour(X)
        inst.append((T, N, dt, p0, Xc))
    elems = sum((T + 1) * (T + 2) // 2 for T in Ts)
    stream = torch.cuda.Stream()
    out = {}
    res = {}
    for prec in ("mixed", "fp64"):
        r = rexi.RaggedPlan(max(Ts), len(Ts), 64 * 512, elems, syn.OMEGA, syn.RADIUS, syn.PHIBAR,
                            precision=prec, stream=stream)
        off = r.set(inst)
        U0 = np.zeros(off[-1], complex)
        for i, T in enumerate(Ts):
            U0[off[i]: off[i + 1]] = syn.gaussian_state(T, 100 + i).reshape(-1)
        u0 = torch.from_numpy(U0).cuda()
        u1 = torch.empty_like(u0)
        torch.cuda.synchronize()
        q, _ = r.tune(u0, u1, reps=2)
        r.capture(u0, u1)
        r.step(u0, u1)
        r.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            r.step(u0, u1)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[prec] = {"steps_per_s": len(Ts) * 1e3 / ms, "ms_per_launch": ms, "tuned_tiles_per_warp": q}
        res[prec] = (u1.cpu().numpy(), off)
        r.close()
    a, off = res["mixed"]
    b, _ = res["fp64"]
    worst = [0.0, 0.0, 0.0]
    for i, T in enumerate(Ts):
        x = a[off[i]: off[i + 1]].reshape(3, -1)
        y = b[off[i]: off[i + 1]].reshape(3, -1)
        w = np.where(np.arange(x.shape[1]) <= T, 1.0, 2.0)
        for f in range(3):
            e = np.sqrt(np.sum(w * np.abs(x[f] - y[f]) ** 2) / np.sum(w * np.abs(y[f]) ** 2))
            worst[f] = max(worst[f], float(e))
    return {"workload": "64 states, T~U{63..255} (seed 3), 512 poles, dt=3600 s, one ragged "
                        "captured-graph launch per step", "mixed": out["mixed"], "fp64": out["fp64"],
            "max_rel_err_mixed_vs_fp64": worst}


def _rel_fields(a, b, T):
    """Per-field relative L2 (m > 0 weighted by 2) of spectral states [3][nlm]."""
    import numpy as np
    nlm = (T + 1) * (T + 2) // 2
    wts = np.where(np.arange(nlm) <= T, 1.0, 2.0)
    out = []
    for f in range(3):
        den = np.sqrt(np.sum(wts * np.abs(b[f]) ** 2))
        out.append(float(np.sqrt(np.sum(wts * np.abs(a[f] - b[f]) ** 2)) / den) if den > 0 else 0.0)
    return out


def sh_transforms(torch, rexi, fp64_peak, fp32_peak, T=511, nlat=768, nlon=1536, nf=2, reps=5,
                  precs=("fp64", "tf32", "bf16", "tf32x3", "df")):
    """Synthesis and analysis of nf scalar fields and of one vector field (psi/chi -> U, V;
    A, B -> div, curl), and the nonlinear term's one-pass combinations (2 scalar fields + 1
    vector pair synthesised, 2 vector pairs + 1 scalar field analysed), at T511 on the
    768 x 1536 Gauss grid in every Legendre precision.
    Per-stage device times from the plan's event profile; the roofline of the Legendre
    contraction is HBM-bound on its table (algorithmic bytes: the table entries the polar-
    truncated sums need, of the nlat/2 x nlm table, read once per transform -- P for scalar
    transforms, P and H for vector transforms -- in the stored element type, plus the
    spectral and Fourier operands), of the FFT on its grid and Fourier arrays.  The FP64 and
    double-float contractions are ALU-bound: 4 flops per needed entry and real array."""
    import numpy as np
    from paper_1805_06557_gb300 import synthetic as syn
    hbm = _hbm_peak()
    nlm = (T + 1) * (T + 2) // 2
    rng = np.random.default_rng(4)
    n = np.concatenate([np.arange(m, T + 1) for m in range(T + 1)]).astype(float)
    amp = np.maximum(n, 1.0) ** -1.5
    c = (rng.standard_normal((nf, nlm)) + 1j * rng.standard_normal((nf, nlm))) * amp
    c[:, :T + 1] = c[:, :T + 1].real
    spec = torch.from_numpy(c).cuda()
    grid = torch.empty(nf, nlat, nlon, dtype=torch.float64, device="cuda")
    back = torch.empty_like(spec)
    U = torch.empty(1, nlat, nlon, dtype=torch.float64, device="cuda")
    V = torch.empty_like(U)
    dv = torch.empty(2, nlm, dtype=torch.complex128, device="cuda")
    cu = torch.empty_like(dv)
    out = {"workload": "T%d, %d x %d Gauss grid, %d scalar fields + 1 vector field, n^-1.5 "
                       "spectra (seed 4)" % (T, nlat, nlon, nf), "hbm_peak_gbs": hbm}
    ref = {}
    for prec in precs:
        p = rexi.ShPlan(T, nlat, nlon, syn.RADIUS, prec, max_fields=3)
        eb = {"fp64": 8, "tf32": 4, "bf16": 2, "tf32x3": 8, "df": 8}[prec]   # split TF32, df: hi and lo words
        use = p.table_use()
        res = {"table_entries": use}
        for kind in ("synthesis", "analysis", "synthesis_uv", "analysis_divcurl", "synthesis_mixed",
                     "analysis_mixed"):
            def call():
                if kind == "synthesis":
                    p.synthesis(spec, grid, nf)
                elif kind == "analysis":
                    p.analysis(grid, back, nf)
                elif kind == "synthesis_uv":
                    p.synthesis_uv(spec[:1], spec[1:2], U, V, 1)
                elif kind == "analysis_divcurl":
                    p.analysis_divcurl(grid[:1], grid[1:2], dv, cu, 1)
                elif kind == "synthesis_mixed":   # the nonlinear term's: 2 scalar + 1 vector
                    p.synthesis_mixed(spec, grid, 2, spec[:1], spec[1:2], U, V, 1)
                else:                             # 2 vector pairs + 1 scalar
                    p.analysis_mixed(grid, grid, dv, cu, 2, grid[:1], back[:1], 1)
            for _ in range(2):
                call()
            p.set_profiling(True)
            p.profile(reset=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                call()
            e1.record()
            torch.cuda.synchronize()
            prof = p.profile(reset=True)
            p.set_profiling(False)
            total = e0.elapsed_time(e1) / reps
            vec = kind in ("synthesis_uv", "analysis_divcurl")
            mixed = kind.endswith("_mixed")
            # tables the method reads: P, or P and H for vector fields -- except the FP64 and
            # double-float plans, whose vector transforms use P alone (synthesis: the scalar
            # syntheses of the velocity components' spectra; analysis: P-sums, whose
            # neighbouring degrees give the H-sums)
            p_only = prec in ("fp64", "df")
            ntab = 2 if (vec or mixed) and not p_only else 1
            need = use["needed_synth" if kind.startswith("synthesis") else "needed_anal"]
            # spectral arrays = Fourier arrays = grids: scalar fields + 2 per vector pair
            narr = 2 if vec else (4 if kind == "synthesis_mixed" else 5 if mixed else nf)
            leg_ms = sum(prof[k][0] for k in ("legendre_fp64", "legendre_df", "tc_gemm", "tc_epilogue")) / reps
            gemm_ms = prof[{"fp64": "legendre_fp64", "df": "legendre_df"}.get(prec, "tc_gemm")][0] / reps
            tab_bytes = ntab * need * eb
            leg_bytes = tab_bytes + narr * (nlm + (T + 1) * nlat) * 16
            fft_ms = prof["fft"][0] / reps
            fft_bytes = narr * (nlat * nlon * 8 + nlat * (T + 1) * 16)
            # FMA = 2; complex coefficient x real table; vector arrays meet P and H (P alone in the
            # FP64 and double-float plans), scalar ones P
            nvec_arr = 2 if kind == "synthesis_mixed" else 4 if kind == "analysis_mixed" else (narr if vec else 0)
            if p_only:
                nvec_arr = 0
            leg_flops = 4.0 * need * (2 * nvec_arr + (narr - nvec_arr))
            if prec == "fp64":   # FP64 CUDA-core contraction: bound by the FP64 pipe on this GPU
                leg_roof = {"bound": "alu", "pipe": "fp64", "kernel": "k_leg_*", "algorithmic_flops": leg_flops,
                            "achieved": leg_flops / (gemm_ms * 1e9), "unit": "TFLOP/s", "peak": fp64_peak,
                            "frac": leg_flops / (gemm_ms * 1e9) / fp64_peak,
                            "achieved_gbs": leg_bytes / (gemm_ms * 1e6)}
            elif prec == "df":   # double-float on the FP32 pipe: 12 FP32 operations per real
                # multiply-add of a compensated dot product (TwoProduct 2, TwoSum 6, low words 4),
                # so 6 per algorithmic flop; the split of the inputs is inside the timed stage
                xops = 6.0 * leg_flops
                leg_roof = {"bound": "alu", "pipe": "fp32", "kernel": "k_df_*", "algorithmic_flops": leg_flops,
                            "achieved": leg_flops / (gemm_ms * 1e9), "unit": "TFLOP/s",
                            "executed_fp32_ops": xops, "executed_tops": xops / (gemm_ms * 1e9), "peak": fp32_peak,
                            "frac": xops / (gemm_ms * 1e9) / fp32_peak,
                            "speed_vs_fp64_peak": leg_flops / (gemm_ms * 1e9) / fp64_peak,
                            "achieved_gbs": leg_bytes / (gemm_ms * 1e6), "hbm_frac": leg_bytes / (gemm_ms * 1e6) / hbm}
            else:                # tensor-core contraction of 16 columns: bound by the table bytes
                leg_roof = {"bound": "hbm", "kernel": "k_tc_gemm", "algorithmic_bytes": leg_bytes,
                            "achieved_gbs": leg_bytes / (gemm_ms * 1e6), "peak": hbm, "unit": "GB/s",
                            "frac": leg_bytes / (gemm_ms * 1e6) / hbm, "tflops": leg_flops / (gemm_ms * 1e9)}
            # FFT: the conventional 5 n log2 n flops per complex length-n sequence (two real rows
            # per sequence).  In FP64 the pipe binds on this GPU (about 2 FP64 FMAs per clock and
            # SM); in FP32 the grid and Fourier bytes do.
            fft_flops = 5.0 * nlon * math.log2(nlon) * narr * nlat / 2
            gbs = fft_bytes / (fft_ms * 1e6) if fft_ms > 0 else None
            if prec == "fp64":   # the FP64 FFT: bound by the FP64 pipe
                fft_roof = {"bound": "alu", "pipe": "fp64", "algorithmic_flops": fft_flops,
                            "achieved": fft_flops / (fft_ms * 1e9) if fft_ms > 0 else None, "unit": "TFLOP/s",
                            "peak": fp64_peak,
                            "frac": fft_flops / (fft_ms * 1e9) / fp64_peak if fft_ms > 0 else None,
                            "algorithmic_bytes": fft_bytes, "achieved_gbs": gbs,
                            "hbm_frac": gbs / hbm if gbs else None}
            else:                # FP32 or double-float arithmetic on the FP32 pipe, FP64 data
                fft_roof = {"bound": "hbm", "algorithmic_bytes": fft_bytes, "achieved_gbs": gbs, "unit": "GB/s",
                            "peak": hbm, "frac": gbs / hbm if gbs else None, "algorithmic_flops": fft_flops}
                if prec == "df" and fft_ms > 0:
                    fft_roof["speed_vs_fp64_peak"] = fft_flops / (fft_ms * 1e9) / fp64_peak
            r = {"ms": total, "stage_ms": {k: v[0] / reps for k, v in prof.items() if v[1]},
                 "legendre_ms": leg_ms, "legendre_roofline": leg_roof,
                 "fft_roofline": fft_roof}
            res[kind] = r
        p.check()
        g, b = grid.cpu().numpy(), back.cpu().numpy()
        if prec == "fp64":
            ref = {"grid": g, "back": b}
            res["rel_err_synthesis_vs_fp64"] = 0.0
        elif ref:
            res["rel_err_synthesis_vs_fp64"] = float(np.linalg.norm(g - ref["grid"]) / np.linalg.norm(ref["grid"]))
            res["rel_err_analysis_vs_fp64"] = float(np.linalg.norm(b - ref["back"]) / np.linalg.norm(ref["back"]))
        out[prec] = res
        p.close()
    return out


def lg_rexi(torch, rexi, fp64_peak, T=511, N=2048, dt=7200.0, batch=32, reps=20):
    """The gravity-only REXI step (the lg_rexi_* methods: L_g alone, a per-degree 2 x 2 pole sum
    applied in one pass) on a batch of T511 states, 2048 poles, dt = 7200 s: device time per
    launch over `reps` launches with CUDA events (input and output 2 x 201 MB, larger than
    L2), against the HBM roof (algorithmic bytes: 3 fields read and written, 96 B per
    coefficient) and the FP64 pipe (14 flops per coefficient triple with real sums)."""
    import numpy as np
    from paper_1805_06557_gb300 import synthetic as syn
    X = dt * np.sqrt(syn.PHIBAR * T * (T + 1.0)) / syn.RADIUS
    p0, Xc = contour(X)
    nlm = (T + 1) * (T + 2) // 2
    base = np.stack([syn.gaussian_state(T, 500 + i) for i in range(4)])
    u0 = torch.from_numpy(np.ascontiguousarray(np.tile(base, (batch // 4, 1, 1)))).cuda()
    u1 = torch.empty_like(u0)
    p = rexi.LgPlan(T, N, dt, syn.RADIUS, syn.PHIBAR, p0=p0, Xc=Xc, max_batch=batch)
    for _ in range(3):
        p.step(u0, u1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        p.step(u0, u1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    _, real = p.operator()
    p.close()
    hbm = _hbm_peak()
    nbytes = 2 * 3 * 16 * nlm * batch
    flops = (14 if real else 28) * nlm * batch
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"workload": "gravity-only REXI step, T%d, %d poles, dt=%g s, batch %d states" % (T, N, dt, batch),
            "ms_per_launch": ms, "states_per_s": batch / (ms * 1e-3), "real_sums": real,
            "roofline": {"bound": "hbm", "kernel": "k_lg_apply", "algorithmic_bytes": nbytes,
                         "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "fp64_tflops": flops / (ms * 1e-3) / 1e12,
                         "fp64_frac": flops / (ms * 1e-3) / 1e12 / fp64_peak if fp64_peak else None}}


def _max_wind(torch, rexi, U0, T, nlat, nlon):
    """Largest wind speed |V| [m/s] of a spectral state on its Gauss grid (FP64 vector synthesis
    of psi = lap^-1 zeta, chi = lap^-1 delta through the library)."""
    import numpy as np
    from paper_1805_06557_gb300 import synthetic as syn
    a = syn.RADIUS
    sh = rexi.ShPlan(T, nlat, nlon, a, "fp64", max_fields=1)
    nn = np.concatenate([np.arange(m, T + 1) for m in range(T + 1)]).astype(float)
    ilap = np.where(nn > 0, -a * a / np.maximum(nn * (nn + 1), 1.0), 0.0)
    psi = torch.from_numpy((U0[1] * ilap)[None].copy()).cuda()
    chi = torch.from_numpy((U0[2] * ilap)[None].copy()).cuda()
    Ug = torch.empty(1, nlat, nlon, dtype=torch.float64, device="cuda")
    Vg = torch.empty_like(Ug)
    sh.synthesis_uv(psi, chi, Ug, Vg, 1)
    mu, _ = sh.grid()
    cos = torch.from_numpy(np.sqrt((1.0 - mu) * (1.0 + mu))).cuda()[None, :, None]
    umax = float(torch.sqrt((Ug / cos) ** 2 + (Vg / cos) ** 2).max())
    sh.close()
    return umax


def swe_steps(torch, rexi, configs):
    """Nonlinear SWE steps (Strang ver1: N by RK2 midpoint for dt/2, REXI L for dt, N for
    dt/2; variants may name another scheme) on balanced n^-3 states: steps/s (timed without
    profiling), per-stage device times (a second, profiled run of the same steps), whether the
    state stayed finite, and each variant's per-field error against the all-FP64 plan after one
    step and after all timed steps from the same state.

    A configuration may carry a time-step treatment (a dict): "contour": "select" (the
    library's contour search, rexi_contour_select, instead of the fixed rule), "courant": c
    (sub-steps of the explicit part from swe_substeps with the state's largest wind), and
    "efold_s": t (del^4 hyper-diffusion whose truncation degree e-folds in t seconds)."""
    import numpy as np
    from paper_1805_06557_gb300 import synthetic as syn
    out = []
    for cfg_in in configs:
        (T, nlat, nlon, N, dt, nsteps, variants) = cfg_in[:7]
        treat = cfg_in[7] if len(cfg_in) > 7 else {}
        X = rexi.spectrum_bound(T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
        p0, Xc = rexi.contour_select(X, N) if treat.get("contour") == "select" else contour(X)
        U0 = syn.balanced_state(T, 2 if T == 127 else 4)
        nsub, visc = 1, 0.0
        if "courant" in treat:
            umax = _max_wind(torch, rexi, U0, T, nlat, nlon)
            nsub = rexi.swe_substeps(T, 0.5 * dt, umax, syn.RADIUS, treat["courant"])
        if "efold_s" in treat:
            visc = 1.0 / (treat["efold_s"] * (T * (T + 1.0) / syn.RADIUS ** 2) ** 2)
        cfg = {"workload": "nonlinear SWE, T%d on %d x %d Gauss grid, %d poles, dt=%g s, %d timed steps, "
                           "balanced n^-3 state (20 m/s rms)" % (T, nlat, nlon, N, dt, nsteps),
               "contour": {"p0": p0, "Xc": Xc, "X": X}, "nsub": nsub, "visc_del4": visc,
               "variants": {}}
        if "courant" in treat:
            cfg["max_wind_ms"] = umax
            cfg["courant"] = treat["courant"]
        if "efold_s" in treat:
            cfg["efold_truncation_s"] = treat["efold_s"]
        ref1 = refn = None
        for var in variants:
            rprec, sprec = var[0], var[1]
            scheme = var[2] if len(var) > 2 else "ver1"
            p = rexi.SwePlan(T, nlat, nlon, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, N, p0, Xc,
                             rexi_precision=rprec, sh_precision=sprec, scheme=scheme, nsub=nsub,
                             visc=visc, visc_order=2)
            u = torch.from_numpy(U0).cuda().contiguous()
            w1 = u.clone()
            p.step(w1, 1)                                  # one step: error figure and warm-up
            one = w1.cpu().numpy()
            u2 = u.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p.step(u2, nsteps)  # timed without the per-kernel event profile
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            last = u2.cpu().numpy()
            # stage times from a separate profiled run of the same steps from the same state
            u3 = u.clone()
            p.set_profiling(True)
            p.profile(reset=True)
            p.step(u3, nsteps)
            prof = p.profile(reset=True)
            p.set_profiling(False)
            key = "%srexi_%s+sh_%s" % ("" if scheme == "ver1" else scheme + ":", rprec, sprec)
            v = {"steps_per_s": nsteps / (ms * 1e-3), "ms_per_step": ms / nsteps,
                 "stage_ms_per_step": {k: val[0] / nsteps for k, val in prof.items()},
                 "finite_after_one_step": bool(np.all(np.isfinite(one))),
                 "finite_after_timed_steps": bool(np.all(np.isfinite(last)))}
            if scheme != "ver1":
                pass   # another scheme: no error against the ver1 FP64 reference
            elif ref1 is None:
                ref1, refn = one, last
            else:
                if v["finite_after_one_step"] and np.all(np.isfinite(ref1)):
                    v["rel_err_vs_fp64_one_step"] = _rel_fields(one, ref1, T)
                if v["finite_after_timed_steps"] and np.all(np.isfinite(refn)):
                    v["rel_err_vs_fp64_after_timed_steps"] = _rel_fields(last, refn, T)
            cfg["variants"][key] = v
            p.close()
        out.append(cfg)
    return out


DT_SWEEP = [15.0, 30.0, 60.0, 120.0, 180.0, 360.0, 480.0, 600.0]   # the paper's REXI time steps


def dt_sweep(args):
    """Error vs time-step size of the nonlinear schemes (Strang ver1 / ver0 with REXI, ETD2RK,
    Crank-Nicolson Strang, and the lg ver1 / lg ETD2RK / lg irk ver0 schemes with Coriolis in
    the explicit part) on the balanced n^-3 T127 state (192 x 384 Gauss grid, 512 poles),
    over 12 h, against Strang ver1 with dt = 5 s: L-infinity of the surface-height error on the
    grid (Phi' / g, the paper's metric) and the per-field relative L2."""
    import numpy as np
    import torch
    from paper_1805_06557_gb300 import rexi
    from paper_1805_06557_gb300 import synthetic as syn
    T, nlat, nlon, N, t_end = 127, 192, 384, 512, 43200.0
    U0 = syn.balanced_state(T, 2)

    def run(scheme, dt, prec="fp64"):
        sub = 0.5 * dt if scheme == "ver0" else dt
        p0, Xc = contour(rexi.spectrum_bound(T, sub, syn.OMEGA, syn.RADIUS, syn.PHIBAR))
        p = rexi.SwePlan(T, nlat, nlon, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR, N, p0, Xc,
                         rexi_precision=prec, scheme=scheme)
        u = torch.from_numpy(U0).cuda().contiguous()
        n = int(round(t_end / dt))
        t0 = time.perf_counter()
        p.step(u, n)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        p.close()
        return u, sec

    ref, _ = run("ver1", 5.0)
    sh = rexi.ShPlan(T, nlat, nlon, syn.RADIUS, "fp64", max_fields=1)
    grid = torch.empty(1, nlat, nlon, dtype=torch.float64, device="cuda")
    out = {"workload": "nonlinear SWE, T127 on 192 x 384, 512 poles, balanced n^-3 state (20 m/s rms), "
                       "12 h; reference: Strang ver1 (FP64) with dt = 5 s", "schemes": {}}
    r = ref.cpu().numpy()
    for scheme in ("ver1", "ver0", "etdrk", "irk", "lg_ver1", "lg_etdrk", "lg_irk_ver0"):
        res = {}
        for dt in DT_SWEEP:
            u, sec = run(scheme, dt)
            d = (u - ref)[0:1].contiguous()
            sh.synthesis(d, grid, 1)
            torch.cuda.synchronize()
            linf = float(grid.abs().max().item()) / syn.GRAVITY
            a = u.cpu().numpy()
            res["%g" % dt] = {"linf_h_m": linf if np.isfinite(linf) else None,
                              "rel_l2": _rel_fields(a, r, T) if np.all(np.isfinite(a)) else None,
                              "wall_s": sec}
        out["schemes"][scheme] = res
    sh.close()
    print(json.dumps(out), flush=True)


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


def serving_run(args):
    import torch
    from paper_1805_06557_gb300 import serving
    from paper_1805_06557_gb300 import rexi, synthetic as syn
    n = args.serving
    # the service's contour table for its pole counts and the largest spectrum width it serves
    # (T511 at dt = 14400 s): planning work before any request, reported, not timed with them
    xmax = rexi.spectrum_bound(511, 14400.0, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    table_s = serving.prepare_contours((256, 512, 1024, 2048), xmax)
    # calibration: capacity of the batched engine with everything queued at once
    cal = serving.make_requests(min(n, 200), seed=5, rate=1e9)
    eng = serving.ServingEngine(Tmax=511, max_slots=64, hbm_bytes=8 << 30, max_poles=64 * 2048)
    cstats = eng.run(cal)
    eng.close()
    rate = 0.8 * cstats["steps_per_s"]
    reqs = serving.make_requests(n, seed=5, rate=rate)
    eng = serving.ServingEngine(Tmax=511, max_slots=64, hbm_bytes=8 << 30, max_poles=64 * 2048)
    st = eng.run(reqs)
    eng.close()
    base = serving.one_at_a_time(serving.make_requests(n, seed=5, rate=rate), precision="fp64")
    line = {"metric": "served REXI steps/s and latency, Poisson stream (T 63-511, dt 600-14400 s, "
                      "N 256-2048)", "unit": "steps/s", "requests": n, "rate_per_s": rate,
            "contour_table_s": table_s, "calibration": cstats, "batched_mixed": st,
            "one_at_a_time_fp64": base}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.serving:
        serving_run(args)
        return
    if args.dt_sweep:
        dt_sweep(args)
        return
    if args.sh_only:
        import torch
        from paper_1805_06557_gb300 import rexi
        fp64_tf, fp32_tf = rexi.alu_peaks()
        Ts = args.sh_T
        nlat = 3 * (Ts + 1) // 2
        out = sh_transforms(torch, rexi, fp64_tf, fp32_tf, T=Ts, nlat=nlat, nlon=2 * nlat,
                            precs=tuple(args.sh_only.split(",")))
        print(json.dumps({"metric": "SH transforms at T%d (Legendre and FFT stages)" % Ts, "sh_transforms": out}),
              flush=True)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1805_06557_gb300 import rexi
    from paper_1805_06557_gb300 import synthetic as syn

    T, N, dt, B = args.T, args.N, args.dt, args.batch
    X = rexi.spectrum_bound(T, dt, syn.OMEGA, syn.RADIUS, syn.PHIBAR)
    p0, Xc = contour(X)
    nlm = rexi.nlm(T)
    host = np.stack([syn.gaussian_state(T, sd) for sd in shard_seeds(rank, B)])
    u0 = torch.from_numpy(host).cuda()
    u1 = torch.empty_like(u0)
    ref64 = torch.empty_like(u0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    fp64_tf, fp32_tf = rexi.alu_peaks()
    kw = dict(omega=syn.OMEGA, radius=syn.RADIUS, phibar=syn.PHIBAR, p0=p0, Xc=Xc)
    mixed = rexi.Plan(T, N, dt, precision="mixed", max_batch=B, **kw)
    fp64 = rexi.Plan(T, N, dt, precision="fp64", max_batch=B, **kw)            # every pole
    # FP64 on the mixed plan's solved poles: pruning at the mixed plan's pruned gain leaves out
    # the same poles (both prune the smallest gains first)
    pg = mixed.info()["pruned_gain"]
    fp64p = rexi.Plan(T, N, dt, precision="fp64", max_batch=B, prune_tau=pg if pg > 0 else -1.0, **kw)

    def timed(plan, a, b, nb, steps, warmup):
        for _ in range(warmup):
            plan.step(a, b, nb)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for e0, e1 in evs:
            flush.zero_()
            e0.record()
            plan.step(a, b, nb)
            e1.record()
        torch.cuda.synchronize()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- headline: batched mixed plan ------------------------------------------------
    for _ in range(args.warmup):
        mixed.step(u0, u1, B)
    mixed.set_profiling(True)
    mixed.profile(reset=True)
    barrier()
    clk = Clocks(local)
    clk.start()
    clk.region_start()
    ms = timed(mixed, u0, u1, B, args.steps, 0)
    clocks = clk.stop()
    prof = mixed.profile(reset=True)
    mixed.set_profiling(False)
    value, total_ms = job_rate(sum(ms), B, world, args.steps, dist, "cuda")
    barrier()

    # ---- secondary measurements (rank-local) -------------------------------------------
    ks = max(3, min(args.steps, 10))
    fp64.step(u0, ref64, B)
    torch.cuda.synchronize()
    err = []
    a, r = u1.cpu().numpy(), ref64.cpu().numpy()
    wts = np.where(np.arange(nlm) <= T, 1.0, 2.0)
    for f in range(3):
        num = np.sqrt(np.sum(wts * np.abs(a[:, f] - r[:, f]) ** 2))
        den = np.sqrt(np.sum(wts * np.abs(r[:, f]) ** 2))
        err.append(float(num / den))
    fp64_b1 = timed(fp64, u0[:1].contiguous(), u1[:1].contiguous(), 1, ks, 2)
    fp64_bb = timed(fp64, u0, u1, B, ks, 1)
    mix_b1 = timed(mixed, u0[:1].contiguous(), u1[:1].contiguous(), 1, ks, 2)
    # FP64 with the same pole pruning as the mixed plan: separates the pruning from the
    # mixed-precision gain
    p64 = torch.empty_like(u0)
    fp64p.step(u0, p64, B)
    torch.cuda.synchronize()
    ap = p64.cpu().numpy()
    err_p64 = [float(np.sqrt(np.sum(wts * np.abs(ap[:, f] - r[:, f]) ** 2)) /
                     np.sqrt(np.sum(wts * np.abs(r[:, f]) ** 2))) for f in range(3)]
    fp64p_b1 = timed(fp64p, u0[:1].contiguous(), u1[:1].contiguous(), 1, ks, 2)
    fp64p_bb = timed(fp64p, u0, u1, B, ks, 1)

    # ---- rooflines of the solve kernels (event times of the timed region) -----------------
    info = mixed.info()
    n_light = N - info["n_pruned"] - info["n_heavy"]
    elems = 2 * nlm * B  # chain elements per pole per launch (two parity chains per m)
    kernels = {}
    for kname, (kms, kn) in prof.items():
        if kn == 0 or kname not in KERNEL_FLOPS:
            continue
        fl, pipe = KERNEL_FLOPS[kname]
        npoles = n_light if kname == "k_rexi_light" else info["n_heavy"]
        flops = fl * elems * npoles
        avg_s = kms / kn * 1e-3
        peak = fp32_tf if pipe == "fp32" else fp64_tf
        xfl = EXECUTED_FLOPS[kname] * elems * npoles
        # the mixed path's two-pipe roofline (the method's solve on the FP32 pipe, its FP64-accurate
        # weighted pole sums, 12 of the 49 flops, on the FP64 pipe), for kernels whose sums must be
        # FP64-accurate; the light kernel's FP32 sums need no FP64
        if kname == "k_rexi_heavy":
            t_min = elems * npoles * ((fl - 12.0) / (fp32_tf * 1e12) + 12.0 / (fp64_tf * 1e12))
            two_pipe = t_min / avg_s
        else:
            two_pipe = None
        kernels[kname] = {"bound": "alu", "pipe": pipe, "flops_per_chain_element": fl, "poles": npoles,
                          "frac_two_pipe": two_pipe,
                          "ms": kms / kn, "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                          "frac": flops / avg_s / 1e12 / peak,
                          "frac_of_fp64_peak": flops / avg_s / 1e12 / fp64_tf,
                          "executed_flops_per_chain_element": EXECUTED_FLOPS[kname],
                          "executed_tflops": xfl / avg_s / 1e12, "executed_frac": xfl / avg_s / 1e12 / peak}
    # the dominant kernel is the one with the most algorithmic work (the heavy kernel: 90 % of the
    # launch list).  Where the heavy tiles leave resident warps idle (one-state steps) the light
    # kernel runs beside them on a side stream, and its event interval then spans its wait for
    # SM room, so event times alone do not rank the kernels; batched steps run it after them
    dom = max(kernels, key=lambda k: kernels[k]["executed_tflops"] * kernels[k]["ms"])
    tr = TRAFFIC.get(dom)
    roof = dict(kernels[dom], kernel=dom,
                traffic=(tr[0] * B / tr[1]) if tr else None,
                traffic_source=tr[2] if tr else None,
                peak_source="measured %s FMA probe (rexi_alu_peaks) in this run" % kernels[dom]["pipe"],
                kernel_ms={k: (v[0] / v[1] if v[1] else None) for k, v in prof.items()},
                kernels=kernels)

    # ---- end to end through the C ABI with host buffers ---------------------------------
    # rexi_step_host_async: every step copies its inputs from pinned host memory and its result
    # back (copy engines), the copies of neighbouring steps overlapping each step's kernels; the
    # wall clock spans all K steps, from the first call to the final sync.  rexi_step_host (one
    # synchronous call per step, its kernels reading and writing the host memory in place) is
    # timed beside it.
    hin = torch.from_numpy(host).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    for _ in range(2):
        mixed.step_host_async_ptr(hin.data_ptr(), hout.data_ptr(), B)
    mixed.sync()
    ke = args.steps
    t0 = time.perf_counter()
    for _ in range(ke):
        mixed.step_host_async_ptr(hin.data_ptr(), hout.data_ptr(), B)
    mixed.sync()
    e2e_s = (time.perf_counter() - t0) / ke
    e2e_same = bool(np.array_equal(hout.numpy(), a))  # a: the headline's mixed step of this input
    for _ in range(2):
        mixed.step_host_ptr(hin.data_ptr(), hout.data_ptr(), B)
    t0 = time.perf_counter()
    for _ in range(ke):
        mixed.step_host_ptr(hin.data_ptr(), hout.data_ptr(), B)
    e2e_sync_s = (time.perf_counter() - t0) / ke
    bytes_step = B * 3 * nlm * 16
    e2e = {"value": B * world / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": bytes_step,
           "d2h_bytes_per_step": bytes_step, "steps": ke,
           "api": "rexi_step_host_async (pinned host buffers; each step's input and result copied "
                  "by the copy engines, overlapping the neighbouring steps' kernels)",
           "result_equals_device_step": e2e_same,
           "l2": "not flushed between the pipelined steps: each step's input arrives through the copy "
                 "engines, and its working set (partial sums, solve scratch, tables) exceeds L2",
           "synchronous_call": {"value": B * world / e2e_sync_s, "unit": "steps/s",
                                "api": "rexi_step_host (one call per step, kernels on the host "
                                       "memory in place)"}}

    ens = None if args.no_ensemble else ensemble(torch, rexi, syn, max(3, min(args.steps, 10)))
    sh = swe = lg = None
    if not args.no_sh:
        sh = sh_transforms(torch, rexi, fp64_tf, fp32_tf)
        swe = swe_steps(torch, rexi, [
            (127, 192, 384, 512, 1800.0, 48, [("fp64", "fp64"), ("mixed", "fp64"), ("mixed", "df"), ("mixed", "tf32x3"),
                                              ("mixed", "tf32"), ("fp64", "fp64", "etdrk"),
                                              ("mixed", "fp64", "etdrk"), ("fp64", "fp64", "irk"),
                                              ("fp64", "fp64", "lg_ver1"), ("fp64", "fp64", "lg_etdrk"),
                                              ("fp64", "fp64", "lg_irk_ver0"), ("fp64", "tf32x3", "lg_ver1")]),
            # T511, dt = 7200 s: the library's contour search (the fixed rule leaves a scalar error
            # of 2e5 at X = 182), the explicit part sub-stepped at Courant 0.5 under the state's
            # largest wind, del^4 diffusion with the truncation degree e-folding in 900 s
            (511, 768, 1536, 2048, 7200.0, 12, [("fp64", "fp64"), ("mixed", "fp64"), ("mixed", "df"), ("mixed", "tf32x3"),
                                                 ("mixed", "tf32"), ("mixed", "bf16"),
                                                 ("fp64", "tf32x3", "lg_ver1")],
             {"contour": "select", "courant": 0.5, "efold_s": 900.0})])
        lg = lg_rexi(torch, rexi, fp64_tf)

    cpu = cpu_fair = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import multiprocessing as mp  # noqa: F401  (the oracle runs in this process)
        rate, sec = cpu_oracle_rate(T, N, dt, SAMPLE_M, [host[i] for i in range(min(SAMPLE_STATES, B))])
        cpu = {"value": rate, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "seconds": sec,
               "sample": "pivoted banded LU oracle, all %d zonal orders of %d states (full steps)"
                         % (len(SAMPLE_M), min(SAMPLE_STATES, B))}
        nthr = os.cpu_count() or 1
        rate_t, sec_t = cpu_thomas_rate(T, N, dt, [host[0]])
        cpu_fair = {"value": rate_t, "unit": "steps/s", "cores": nthr, "seconds": sec_t,
                    "kind": "vectorised numpy FP64 Thomas (two parity chains per pole and zonal order)",
                    "sample": "one full step of one state, pole chunks of 64 on %d threads" % nthr}

    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": workload_config(args, world),
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "rel_err_vs_fp64_gpu": err,
        "fp64_plain_steps_per_s": 1e3 / statistics.mean(fp64_b1),
        "fp64_batched_steps_per_s": B * 1e3 / statistics.mean(fp64_bb),
        "mixed_single_steps_per_s": 1e3 / statistics.mean(mix_b1),
        "speedup_vs_fp64_plain": value / world / (1e3 / statistics.mean(fp64_b1)),
        # the same pole pruning applied to FP64: what mixed precision alone buys
        "speedup_vs_fp64_pruned_batched": value / world / (B * 1e3 / statistics.mean(fp64p_bb)),
        "fp64_pruned": {"single_steps_per_s": 1e3 / statistics.mean(fp64p_b1),
                        "batched_steps_per_s": B * 1e3 / statistics.mean(fp64p_bb),
                        "n_pruned": fp64p.info()["n_pruned"], "rel_err_vs_fp64_plain": err_p64},
        "plan": {k: info[k] for k in ("n_heavy", "n_pruned", "pruned_gain", "n_groups", "q_slots", "grid_light",
                                      "grid_heavy")},
        "alu_peaks_tflops": {"fp64": fp64_tf, "fp32": fp32_tf},
        "ensemble": ens, "sh_transforms": sh, "swe_step": swe, "lg_rexi": lg,
        "roofline": roof, "e2e": e2e, "cpu_baseline": cpu, "cpu_thomas": cpu_fair, "clocks": clocks,
        "gpu_launches": 4 * args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    mixed.close()
    fp64.close()
    fp64p.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
