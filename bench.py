#!/usr/bin/env python
"""Benchmark: slope frames/s to relative residual 1e-4, ELT-scale LTAO, plain FP32 CG.

Workload: 39 m pupil, 28 % obstruction, 74 x 74 subapertures, 6 laser guide
stars at 90 km on a 60"-diameter ring, target on axis, 9 layers (0-20 km),
r0 = 0.129 m, L0 = 25 m, noise 3 % of slope rms; 64 seeded synthetic frames per
GPU per step.  One step = one call of tomo_solve on the 64 frames: CG with the
FFT-based Sigma_ss MVM until every frame's FP64 true relative residual is
<= 1e-4 (FP64 restarts included), then the Sigma_phi_s projection.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded sample of the same workload instead (no GPU).
"""
import argparse
import hashlib
import json
import math
import re
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "slope frames/s to rel. residual 1e-4 (ELT LTAO), learned+mixed vs plain CG"
UNIT = "frames/s"
WORKLOAD = ("elt_ltao: 39 m, 28% obstruction, 6 LGS at 90 km (60\" ring), 74x74 subapertures, 9 layers 0-20 km, "
            "r0 0.129 m, L0 25 m, noise 3%; plain FP32 CG (FP64 scalars, FP64 true residual) to 1e-4, then projection")
FRAMES = 64
TOL = 1e-4
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="time only the headline plain-CG solve (no PCG, MINRES, closed-loop or learned variants)")
    ap.add_argument("--fft-P", type=int, default=-1,
                    help="FFT side of the Sigma_ss product (-1: autotuned; profiling runs pin it, since the "
                         "autotuner's timings are distorted under a profiler)")
    ap.add_argument("--host-loop", action="store_true",
                    help="for profiling: convergence checks on the host instead of the single graph launch with "
                         "conditional nodes (the same kernels)")
    ap.add_argument("--profile-block", action="store_true",
                    help="for profiling: solve the frames W + K times with block PCG and nothing else, print a "
                         "short JSON line (not a bench result)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm_gbs=float(p["hbm_gbs"]), sm_max_mhz=float(p.get("sm_max_mhz", 2070.0)), src="measured")
    except (OSError, KeyError, ValueError):
        return dict(hbm_gbs=6800.0, sm_max_mhz=2070.0, src="fallback")


# --------------------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- algorithmic work model
def fft_flops(L):
    """Complex FFT of length L: 5 L log2 L flops (the paper's a = 5 cost model, Sec. 2.E and 4.B)."""
    return 5.0 * L * math.log2(L)


def paper_opcounts(n, n_gs, n_layer, n_new, a=5.0):
    """Operation counts per frame of the paper's 1-D 2RBT products (Sec. 2.E, with an
    N-point FFT costing a N log2 N operations and a sparse MVM its non-zeros) and of
    the full MVMs they replace:
      Sigma_ss zeta:         4 N_gs {(2n-1)^2 [2a log2(2n-1) + N_gs] + n^2}, full 4 N_gs^2 n^4;
      Sigma_phi_s zeta, NGS: 2 N_gs [4n^2 (2a log2 2n + 1) + n^2] + 8 n^2 log2 2n + (n+1)^2,
                             full 2 N_gs (n+1)^2 n^2 (the backward-FFT term as printed, without a);
      Sigma_phi_s zeta, LGS: 2 (n'+n-1)^2 [(2 N_gs + N_layer) a log2(n'+n-1) + N_gs N_layer]
                             + 2 N_gs n^2 + 4 N_layer (n+1)^2, same full MVM."""
    L = 2 * n - 1
    ss = 4 * n_gs * (L * L * (2 * a * math.log2(L) + n_gs) + n * n)
    ps_ngs = (2 * n_gs * (4 * n * n * (2 * a * math.log2(2 * n) + 1) + n * n) + 8 * n * n * math.log2(2 * n)
              + (n + 1) ** 2)
    Lp = n_new + n - 1
    ps_lgs = (2 * Lp * Lp * ((2 * n_gs + n_layer) * a * math.log2(Lp) + n_gs * n_layer) + 2 * n_gs * n * n
              + 4 * n_layer * (n + 1) ** 2)
    ps_full = 2 * n_gs * (n + 1) ** 2 * n * n
    return {"sigma_ss": ss, "sigma_ss_full": 4 * n_gs ** 2 * n ** 4, "sigma_phi_s_ngs": ps_ngs,
            "sigma_phi_s_lgs": ps_lgs, "sigma_phi_s_full": ps_full}


def whole_product(model, frames, step_ms, iters_mean, hbm_gbs, alu_tflops):
    """The three passes of one product taken as a unit: algorithmic bytes and flops per
    frame-iteration (the spectra once per launch of ``frames``), their intensity against
    the FP32 ridge, the HBM-bound and FP32-bound times, and the solve's measured time per
    frame-iteration (every kernel of the step included) as a fraction of the HBM bound
    and of the larger of the two bounds."""
    byts = sum(m["bytes"] for m in model.values()) + sum(m["per_launch_bytes"] for m in model.values()) / frames
    flops = sum(m["flops"] for m in model.values())
    bound_s = byts / (hbm_gbs * 1e9)
    alu_s = flops / (alu_tflops * 1e12)
    meas_s = step_ms / 1000.0 / (frames * iters_mean)
    return {"bytes_per_frame_iter": byts, "flops_per_frame_iter": flops, "flop_per_byte": flops / byts,
            "ridge_flop_per_byte": alu_tflops * 1e12 / (hbm_gbs * 1e9), "hbm_bound_us": bound_s * 1e6,
            "alu_bound_us": alu_s * 1e6, "solve_us_per_frame_iter": meas_s * 1e6,
            "frac_of_hbm_bound": bound_s / meas_s, "frac_of_roofline": max(bound_s, alu_s) / meas_s}


def kernel_model(layout):
    """Algorithmic flops and bytes per frame-iteration for each MVM pass: complex FFTs at 5 L log2 L
    flops, 8 flops per complex multiply-add of the block product, and the vectors, half spectra and
    spectra each pass must move."""
    n, P, NP, N = layout.n, layout.P, 2 * layout.n_gs, layout.N
    nh = P // 2 + 1
    rows_fft = NP * math.ceil(n / 2) * fft_flops(P)           # two real rows per complex FFT
    inter = NP * nh * n * 8                                    # one pass of the column-major half spectrum
    spectra = nh * P * (NP * (NP + 1) // 2) * 8               # Hermitian K(f): the 78 upper blocks, once per launch
    return {
        # CG mode: reads x, r, p, Ap and writes x, r, p (the fused update), writes the half spectrum
        "rows_fwd": dict(flops=rows_fft, bytes=7 * N * 4 + inter, per_launch_bytes=0),
        "cols_mul": dict(flops=2 * NP * nh * fft_flops(P) + nh * P * NP * NP * 8, bytes=2 * inter,
                         per_launch_bytes=spectra),
        # reads the half spectrum, p and r (for r^T Ap), writes Ap
        "rows_inv": dict(flops=rows_fft, bytes=3 * N * 4 + inter, per_launch_bytes=0),
    }


def kernel_source_hash():
    """Hash of the code (comments and blank space removed) of the files that
    define the iteration kernels: traffic counters stay valid across comment
    edits and become stale with any change of the code itself."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "fft.cuh", "fft_group.cuh"):
        with open(os.path.join(ROOT, "paper_1806_07938_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per frame-iteration of ``kernel`` from the committed ncu summary,
    or None if the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("kernel_source_hash") != kernel_source_hash():
        return None
    e = t.get("kernels", {}).get(kernel)
    return None if e is None else e.get("dram_bytes_per_frame_iter")


# --------------------------------------------------------------------------- CPU oracle sample
def _rows_job(args):
    cfg, rows = args
    from oracle import covariance as cov
    return cov.css_rows(cfg, rows)


def _block_job(args):
    cfg, rows, cols = args
    from oracle import covariance as cov
    return cov.css_block(cfg, rows, cols)


def oracle_pool(cores):
    """A process pool for the oracle (spawned: the parent may hold a CUDA context)."""
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp
    return ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn"))


def oracle_matrix(pool, cfg, cores):
    """The oracle's dense FP64 A = Sigma_ss + Sigma_eta_eta, its rows assembled in parallel."""
    import numpy as np
    from oracle import covariance as cov
    N = cov.slope_points(cfg)[0].shape[0]
    chunks = [c for c in np.array_split(np.arange(N), 4 * cores) if len(c)]
    A = np.concatenate(list(pool.map(_rows_job, [(cfg, c) for c in chunks])))
    A[np.arange(N), np.arange(N)] += cov.noise_variance(cfg)
    return A


def oracle_measured(pool, cores, name, frames, seed, cg_frames=16):
    """The oracle timed end to end on a configuration it finishes in seconds:
    assembly of the dense A, its Cholesky factorisation, the two triangular
    solves per frame (the direct path), and dense FP64 CG to 1e-4 per frame."""
    import numpy as np
    import scipy.linalg as sla
    from oracle import solve as osolve
    from paper_1806_07938_gb300 import workloads as W
    from oracle import geometry as geo
    cfg = W.config(name)
    full, sigma = W.slope_frames(cfg, frames, seed=seed)
    cfg["noise_sigma"] = [float(x) for x in sigma]
    mask = geo.subaperture_mask(cfg["n"], cfg["obstruction"])
    s = full[..., mask].reshape(frames, -1)
    t0 = time.perf_counter()
    A = oracle_matrix(pool, cfg, cores)
    t_asm = time.perf_counter() - t0
    t0 = time.perf_counter()
    c = sla.cho_factor(A, lower=True, check_finite=False)
    t_chol = time.perf_counter() - t0
    t0 = time.perf_counter()
    sla.cho_solve(c, s.T, check_finite=False)
    t_tri = time.perf_counter() - t0
    nc = min(cg_frames, frames)
    t0 = time.perf_counter()
    its = [osolve.cg(A, s[f], tol=TOL, maxit=100000)[1] for f in range(nc)]
    t_cg = (time.perf_counter() - t0) / nc
    return {"workload": name, "N": int(A.shape[0]), "frames": frames,
            "assembly_s": t_asm, "cholesky_s": t_chol, "triangular_s_per_frame": t_tri / frames,
            "cg_s_per_frame": t_cg, "cg_iters_mean": float(np.mean(its)),
            "direct_frames_per_s": frames / (t_asm + t_chol + t_tri),
            "direct_frames_per_s_factor_reused": frames / t_tri,
            "cg_frames_per_s": 1.0 / t_cg}


class OracleTimer:
    """Times the oracle on the host cores.

    ELT (the bench's workload, too large for a dense FP64 solve in minutes):
    a bounded sample of the same path, each piece timed on the oracle's own
    matrix and scaled to the full size: the assembly of R rows of A (x N/R),
    the Cholesky factorisation of a principal n_s x n_s block of A (x (N/n_s)^3),
    the triangular solves of `frames` right-hand sides with that factor
    (x (N/n_s)^2) and a block of dense CG products (one block product x
    (N/n_s)^2 x the CG iterations the GPU needs at 1e-4).  A step's value is
    the faster of the direct and CG paths.  setup() assembles the principal
    block once; step() times the pieces; measured() times the oracle end to
    end on the 8 m system and the mid-size laser-star system."""

    ITERS_GPU = 1982

    def __init__(self, cfg, frames, rows_per_core):
        import numpy as np
        from oracle import covariance as cov
        self.cfg, self.frames = cfg, frames
        self.cores = os.cpu_count() or 1
        self.N = cov.slope_points(cfg)[0].shape[0]
        self.R = rows_per_core * self.cores
        self.rows = np.linspace(0, self.N - 1, self.R).astype(np.int64)
        self.ns = min(4096, self.N)
        self.pool = oracle_pool(self.cores)

    def setup(self):
        import numpy as np
        from oracle import covariance as cov
        idx = np.sort(np.random.default_rng(0).choice(self.N, self.ns, replace=False))
        parts = np.array_split(idx, 2 * self.cores)
        self.Ab = np.concatenate(list(self.pool.map(_block_job, [(self.cfg, p, idx) for p in parts])))
        self.Ab[np.arange(self.ns), np.arange(self.ns)] += cov.noise_variance(self.cfg)[idx]
        self.b = np.random.default_rng(1).standard_normal((self.ns, self.frames))

    def step(self):
        import scipy.linalg as sla
        N, ns, R, frames = self.N, self.ns, self.R, self.frames
        t0 = time.perf_counter()
        list(self.pool.map(_rows_job, [(self.cfg, self.rows[i::self.cores]) for i in range(self.cores)]))
        t_rows = time.perf_counter() - t0
        t0 = time.perf_counter()
        c = sla.cho_factor(self.Ab, lower=True, check_finite=False)
        t_chol = time.perf_counter() - t0
        t0 = time.perf_counter()
        sla.cho_solve(c, self.b, check_finite=False)
        t_tri = time.perf_counter() - t0
        t0 = time.perf_counter()
        for _ in range(3):
            self.Ab @ self.b
        t_mv = (time.perf_counter() - t0) / 3
        T_asm = t_rows * N / R
        T_chol = t_chol * (N / ns) ** 3
        T_tri = t_tri * (N / ns) ** 2
        T_cg = t_mv * (N / ns) ** 2 * self.ITERS_GPU
        direct = frames / (T_asm + T_chol + T_tri)
        cgv = frames / (T_asm + T_cg)
        return dict(value=max(direct, cgv), unit=UNIT, cores=self.cores, kind="oracle",
                    sample=(f"ELT: oracle dense FP64 path on {frames} frames from timed pieces of the oracle's own A: "
                            f"assembly of {R} of {N} rows ({t_rows:.2f} s -> {T_asm:.0f} s by N/{R}), Cholesky of a "
                            f"principal {ns}^2 block ({t_chol:.2f} s -> {T_chol:.0f} s by (N/{ns})^3), triangular "
                            f"solves of {frames} right-hand sides ({t_tri:.3f} s -> {T_tri:.1f} s by (N/{ns})^2), "
                            f"dense CG (block product {t_mv:.3f} s -> {T_cg:.0f} s at {self.ITERS_GPU} iterations); "
                            f"value = the faster path"),
                    model={"assembly_s": T_asm, "cholesky_s": T_chol, "triangular_s": T_tri, "cg_s": T_cg,
                           "direct_frames_per_s": direct, "cg_frames_per_s": cgv},
                    step_wall_s=t_rows + t_chol + t_tri + 3 * t_mv)

    def measured(self):
        return [oracle_measured(self.pool, self.cores, "ngs8m", self.frames, seed=500),
                oracle_measured(self.pool, self.cores, "lgs_mid", self.frames, seed=501)]

    def close(self):
        self.pool.shutdown()


def oracle_sample(cfg, frames=FRAMES):
    """One ELT sample of the oracle plus its end-to-end timings on the two small systems."""
    t0 = time.perf_counter()
    ot = OracleTimer(cfg, frames, rows_per_core=6)
    try:
        ot.setup()
        out = ot.step()
        out["measured"] = ot.measured()
    finally:
        ot.close()
    out["sample"] += "; 'measured' times the oracle end to end on two smaller systems"
    out["wall_s"] = time.perf_counter() - t0
    return out


# --------------------------------------------------------------------------- arms
def dist_setup(use_cuda):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return world, rank, local, dist if world > 1 else None


def max_over_ranks(value, dist, device):
    """The largest `value` over the ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, frames_per_rank, steps, max_ms):
    """frames/s of the whole job: every rank's frames over the slowest rank's time."""
    return world * frames_per_rank * steps / (max_ms / 1000.0)


def workload(frames, seed):
    from paper_1806_07938_gb300 import workloads as W
    cfg = W.config("elt_ltao")
    full, sigma = W.slope_frames_parallel(cfg, frames, seed=seed)
    cfg["noise_sigma"] = [float(s) for s in sigma]
    return cfg, full


def train_warm_start(tomo, torch, h, cfg, layout, sub, seed, n_train=256, steps=200, B=32):
    """Offline: seeded training frames, their PCG solutions, Adam on the warm-start network."""
    import numpy as np
    from paper_1806_07938_gb300 import workloads as W
    full, sigma = W.slope_frames_parallel(cfg, n_train, seed=seed)
    # the reconstructor's noise model is the bench frames'; the training frames only need the same statistics
    s = torch.tensor(tomo.valid_slopes(full, sub), dtype=torch.float32, device="cuda").contiguous()
    z = torch.zeros_like(s)
    opts = tomo.solve_opts(tol=1e-5, max_iter=30000, max_refine=3, precond=True)
    for b0 in range(0, n_train, 64):
        nb = min(64, n_train - b0)
        tomo.tomo_solve(h, s[b0:b0 + nb].contiguous(), nb, opts, z[b0:b0 + nb])
    NP = 2 * layout.n_gs
    tomo.tomo_ws_init(h, hidden=32, max_batch=64, in_scale=float(1.0 / s.std().item()),
                      out_scale=float(z.std().item()))
    tomo.tomo_ws_set_params(h, W.warm_start_init(NP, 32, seed=seed))
    rng = np.random.default_rng(seed)
    losses = []
    for step in range(steps):
        idx = torch.tensor(rng.choice(n_train, B, replace=False), device="cuda")
        losses.append(tomo.tomo_ws_train_step(h, s[idx].contiguous(), z[idx].contiguous(), B,
                                              2e-3 if step < 0.7 * steps else 5e-4))
    return float(np.mean(losses[:5])), float(np.mean(losses[-20:]))


def run_learned_flexible(tomo, torch, W, args, stream, flush, cfg, s, F, P, rank, world, n_train=256, hidden=16,
                         steps=300, B=32):
    """The learned preconditioner in flexible PCG (plain PCG with M as its
    fallback) on the bench frames.  The network (input [r, M r], output a
    correction of M r) is trained offline on (r_k, zeta* - x_k) pairs of
    truncated PCG solves (k = 0, 8, 30, 80 iterations) of other seeded frames,
    each pair scaled to |r_k| = 1."""
    import numpy as np
    h = tomo.tomo_create(cfg, stream=stream, max_batch=F, precond=True, fft_P=P)
    try:
        layout, sub, _ = tomo.tomo_layout(h)
        full, _ = W.slope_frames_parallel(cfg, n_train, seed=2500 + rank)
        st = torch.tensor(tomo.valid_slopes(full, sub), dtype=torch.float32, device="cuda").contiguous()
        t0 = time.perf_counter()
        rp, ep = [], []
        for b0 in range(0, n_train, F):
            nb = min(F, n_train - b0)
            sb = st[b0:b0 + nb].contiguous()
            zs = torch.zeros_like(sb)
            tomo.tomo_solve(h, sb, nb, tomo.solve_opts(tol=1e-6, max_iter=30000, max_refine=3, precond=True), zs)
            for k in (0, 8, 30, 80):
                x = torch.zeros_like(sb)
                if k:
                    tomo.tomo_solve(h, sb, nb, tomo.solve_opts(tol=1e-12, max_iter=k, max_refine=0, check_every=1,
                                                               precond=True), x)
                Ax = torch.empty_like(sb)
                tomo.tomo_apply_css(h, x, Ax, nb)
                r = sb - Ax
                nr = r.norm(dim=1, keepdim=True)
                rp.append(r / nr)
                ep.append((zs - x) / nr)
        rp, ep = torch.cat(rp).contiguous(), torch.cat(ep).contiguous()
        NP = 2 * layout.n_gs
        tomo.tomo_ws_init(h, hidden=hidden, max_batch=F, in_scale=float(1.0 / rp.std()), out_scale=float(ep.std()),
                          precond_input=True, pre_gain=1.0)
        init = W.warm_start_init(NP, hidden, seed=2500 + rank, cin=2 * NP, last_gain=0.0)
        tomo.tomo_ws_set_params(h, init)
        rng = np.random.default_rng(2500 + rank)
        losses = []
        for step in range(steps):
            idx = torch.tensor(rng.choice(rp.shape[0], B, replace=False), device="cuda")
            losses.append(tomo.tomo_ws_train_step(h, rp[idx].contiguous(), ep[idx].contiguous(), B,
                                                  1e-3 if step < 0.75 * steps else 3e-4))
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        z = torch.zeros_like(s)
        out = {}
        for name, pc in (("pcg", True), ("learned", "learned")):
            opts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=16, precond=pc)
            tomo.tomo_solve(h, s, F, opts, z)
            evs, info = [], None
            for _ in range(max(1, min(args.steps, 2))):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                info = tomo.tomo_solve(h, s, F, opts, z)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
            out[name] = {"value": world * F / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms,
                         "iters_mean": float(info["iters"].mean()),
                         "fallbacks": int((info["status"] == tomo.FRAME_FALLBACK_PLAIN_CG).sum()),
                         "all_converged": bool(np.isin(info["status"], [0, tomo.FRAME_FALLBACK_PLAIN_CG]).all()
                                               and (info["relres"] <= TOL).all())}
        res = out["learned"]
        res["pcg_same_handle"] = out["pcg"]
        res["iteration_gain_vs_pcg"] = 1.0 - res["iters_mean"] / out["pcg"]["iters_mean"]
        res["frames_per_s_gain_vs_pcg"] = res["value"] / out["pcg"]["value"] - 1.0
        res["training"] = {"pairs": int(rp.shape[0]), "frames": n_train, "steps": steps, "batch": B,
                           "hidden": hidden, "loss_first": float(np.mean(losses[:5])),
                           "loss_last": float(np.mean(losses[-20:])), "wall_s": train_s,
                           "network": f"3x3 CNN [r, M r] {2 * NP}-{hidden}-{hidden}-{hidden}-{NP}, FP32"}
        return res
    finally:
        tomo.tomo_destroy(h)


def run_moao(tomo, torch, W, args, stream, flush, F, rank, world):
    """MOAO variant: the elt_moao system (32 targets), F frames in four groups
    generated at r0 = 0.10, 0.133, 0.167, 0.20 m and solved in one batch with
    those per-frame r0 values (tomo_solve_r0), PCG to 1e-4, then the projection
    to all 32 targets."""
    import numpy as np
    cfg = W.config("elt_moao")
    r0s = [0.10, 0.133, 0.167, 0.20]
    per = F // len(r0s)
    parts, sigmas = [], []
    for i, r0 in enumerate(r0s):
        full, sigma = W.slope_frames_parallel(dict(cfg, r0=r0), per, seed=4000 + 10 * rank + i)
        parts.append(full)
        sigmas.append(sigma)
    # the reconstructor's noise model: 3 % of the slope rms at the configuration's
    # r0, scaled per frame to the noise its group was drawn with
    _, sig = W.slope_frames(cfg, 1, seed=4000 + 10 * rank)
    cfg["noise_sigma"] = [float(x) for x in sig]
    nu = np.repeat([float(np.mean((sg / sig) ** 2)) for sg in sigmas], per)
    t0 = time.perf_counter()
    h = tomo.tomo_create(cfg, stream=stream, max_batch=F, precond=True)
    create_s = time.perf_counter() - t0
    try:
        layout, sub, _ = tomo.tomo_layout(h)
        B = per * len(r0s)
        s = torch.tensor(tomo.valid_slopes(np.concatenate(parts), sub), dtype=torch.float32,
                         device="cuda").contiguous()
        r0v = np.repeat(np.array(r0s), per)
        z = torch.zeros_like(s)
        phi = torch.empty((B, layout.n_targets, layout.n_vphi), dtype=torch.float32, device="cuda")
        opts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=16, precond=True)
        for _ in range(args.warmup):
            tomo.tomo_solve_r0(h, s, B, r0v, opts, z, phi, noise_scale=nu)
        evs, info = [], None
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = tomo.tomo_solve_r0(h, s, B, r0v, opts, z, phi, noise_scale=nu)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        # block PCG on the same frames: with the noise variance following the
        # seeing (nu_f = c_f) the operators are multiples of one another
        c = (r0v / cfg["r0"]) ** (-5.0 / 3.0)
        bopts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, precond=True, method="block")
        for _ in range(args.warmup):
            tomo.tomo_solve_r0(h, s, B, r0v, bopts, z, phi, noise_scale=c)
        bevs, binfo = [], None
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            binfo = tomo.tomo_solve_r0(h, s, B, r0v, bopts, z, phi, noise_scale=c)
            e1.record(stream)
            bevs.append((e0, e1))
        torch.cuda.synchronize()
        bms = sum(a.elapsed_time(b) for a, b in bevs)
        block = {"value": world * B * args.steps / (bms / 1000.0), "ms_per_step": bms / args.steps,
                 "iters": int(binfo["iters"][0]),
                 "all_converged": bool((binfo["status"] == 0).all() and (binfo["relres"] <= TOL).all()),
                 "noise_model": "nu_f = c_f (noise variance proportional to the turbulence's)"}
        # the projection alone (32 targets) on the solved zeta
        pe0 = torch.cuda.Event(enable_timing=True)
        pe1 = torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        tomo.tomo_apply_cos(h, z, phi, B)
        pe1.record(stream)
        torch.cuda.synchronize()
        return {"value": world * B * args.steps / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / args.steps,
                "frames": B, "targets": layout.n_targets, "r0": r0s, "noise_scale": sorted(set(nu.tolist())),
                "iters_mean": float(info["iters"].mean()),
                "iters_by_r0": [float(info["iters"][i * per:(i + 1) * per].mean()) for i in range(len(r0s))],
                "all_converged": bool((info["status"] == 0).all() and (info["relres"] <= TOL).all()),
                "projection_ms": pe0.elapsed_time(pe1), "create_s": create_s, "block_pcg": block,
                "workload": "elt_moao: the LGS part of config 4 (no NGS), 32 targets within 7', per-frame r0"}
    finally:
        tomo.tomo_destroy(h)


def run_mixed(tomo, torch, W, args, stream, flush, h, cfg, sub, layout, rank, world, frames):
    """Mixed precision (FP64 outer refinement: FP64 zeta and FP64 true
    residuals around FP32 inner CG) on `frames` other seeded frames of the same
    system, timed beside plain FP32 CG on the same frames; each frame's error
    against an FP64 reference (CG entirely in FP64 to 1e-8, whose own error is
    below 1e-8 |s| / sigma^2)."""
    import numpy as np
    full, _ = W.slope_frames_parallel(cfg, frames, seed=5000 + rank)
    s = torch.tensor(tomo.valid_slopes(full, sub), dtype=torch.float32, device="cuda").contiguous()
    z = torch.zeros_like(s)
    steps = max(1, min(args.steps, 2))
    out = {}
    for name, prec in (("mixed", "mixed"), ("fp32", "fp32")):
        opts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=32, precision=prec)
        tomo.tomo_solve(h, s, frames, opts, z)
        evs, info = [], None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = tomo.tomo_solve(h, s, frames, opts, z)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        out[name] = {"value": world * frames / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms,
                     "iters_mean": float(info["iters"].mean()), "refinements_max": int(info["refinements"].max()),
                     "relres_max": float(info["relres"].max()),
                     "all_converged": bool((info["status"] == 0).all() and (info["relres"] <= TOL).all()),
                     "zeta": z.double().cpu().numpy()}
    # FP64 reference
    s64 = s.double()
    z64 = torch.zeros_like(s64)
    t0 = time.perf_counter()
    ref = tomo.tomo_solve_f64(h, s64, frames, tomo.solve_opts(tol=1e-8, max_iter=60000, max_refine=3,
                                                              precision="fp64"), z64)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    zr = z64.cpu().numpy()
    snorm = np.linalg.norm(s64.cpu().numpy(), axis=1)
    sig2 = min(cfg["noise_sigma"]) ** 2
    res = {"frames": frames, "steps": steps,
           "fp64_reference": {"tol": 1e-8, "iters_mean": float(ref["iters"].mean()),
                              "relres_max": float(ref["relres"].max()), "wall_s": t_ref}}
    for name, o in out.items():
        zz = o.pop("zeta")
        err = np.linalg.norm(zz - zr, axis=1) / np.linalg.norm(zr, axis=1)
        o["err_vs_fp64_max"] = float(err.max())
        o["err_vs_fp64_median"] = float(np.median(err))
        o["err_vs_fp64_per_frame"] = [float("%.3g" % e) for e in err]
        res[name] = o
    res["note"] = ("BASELINE config 3 on 256 frames: 'mixed' = FP64 zeta and FP64 true residuals (FP64 2RBT "
                   "product) around FP32 CG; 'fp32' = the headline solver on the same frames; errors are "
                   "relative L2 against FP64 CG to 1e-8 on the same frames (rigorous bound of that reference: "
                   "1e-8 |s| / sigma^2)")
    res["reference_bound_max"] = float((1e-8 * snorm / sig2 / np.linalg.norm(zr, axis=1)).max())
    return res


def gpu_small(tomo, torch, W, name, frames, seed, stream, flush, steps):
    """The library on a small configuration (the oracle is timed on the same frames): plain CG to 1e-4."""
    import numpy as np
    cfg = W.config(name)
    full, sigma = W.slope_frames(cfg, frames, seed=seed)
    cfg["noise_sigma"] = [float(x) for x in sigma]
    h = tomo.tomo_create(cfg, stream=stream, max_batch=frames)
    try:
        _, sub, _ = tomo.tomo_layout(h)
        s = torch.tensor(tomo.valid_slopes(full, sub), dtype=torch.float32, device="cuda").contiguous()
        z = torch.zeros_like(s)
        opts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=16)
        tomo.tomo_solve(h, s, frames, opts, z)
        evs, info = [], None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = tomo.tomo_solve(h, s, frames, opts, z)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        return {"workload": name, "gpu_frames_per_s": frames / (ms / 1000.0), "gpu_iters_mean": float(info["iters"].mean()),
                "gpu_all_converged": bool((info["status"] == 0).all())}
    finally:
        tomo.tomo_destroy(h)


def run_reference(args):
    world, rank, _, dist = dist_setup(False)
    if rank != 0:
        return
    from paper_1806_07938_gb300 import workloads as W
    cfg = W.config("elt_ltao")
    cfg["noise_sigma"] = [0.17] * len(cfg["gs"])
    # one step = the timed pieces of the oracle's ELT path (one row per host
    # core, the Cholesky and triangular solves of a principal block, dense CG
    # products), scaled to the full workload; the block is assembled once
    ot = OracleTimer(cfg, args.frames, rows_per_core=1)
    vals = []
    try:
        ot.setup()
        for i in range(args.warmup + args.steps):
            r = ot.step()
            if i >= args.warmup:
                vals.append(r)
    finally:
        ot.close()
    value = statistics.median(v["value"] for v in vals)
    step_ms = 1000.0 * statistics.mean(v["step_wall_s"] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "ms_per_step_note": ("wall time of one timed oracle sample; value is the full workload's frames/s "
                                 "scaled from it (see cpu_baseline.sample)"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames": args.frames},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1806_07938_gb300 import tomo
    from paper_1806_07938_gb300 import workloads as W

    world, rank, local, dist = dist_setup(True)
    torch.cuda.set_device(local)
    tomo.lib()
    cfg, full = workload(args.frames, seed=1000 + rank)
    stream = torch.cuda.Stream()
    F = args.frames
    with torch.cuda.stream(stream):
        # fft_P = -1: the library times the candidate FFT sides and keeps the fastest
        h = tomo.tomo_create(cfg, stream=stream, max_batch=F, precond=True, fft_P=args.fft_P)
        layout, sub, ph = tomo.tomo_layout(h)
        tune_P, tune_ms = tomo.tomo_autotune_result(h)
        s = torch.tensor(tomo.valid_slopes(full, sub), dtype=torch.float32, device="cuda").contiguous()
        z = torch.zeros_like(s)
        phi = torch.empty((F, layout.n_targets, layout.n_vphi), dtype=torch.float32, device="cuda")
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        if args.profile_block:
            bopts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, precond=True, method="block")
            for _ in range(args.warmup + args.steps):
                binfo = tomo.tomo_solve(h, s, F, bopts, z, phi)
            torch.cuda.synchronize()
            print(json.dumps({"profile": "block_pcg", "iters": int(binfo["iters"][0]),
                              "relres_max": float(binfo["relres"].max())}), flush=True)
            tomo.tomo_destroy(h)
            return
        opts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=32, host_loop=args.host_loop)
        for _ in range(args.warmup):
            tomo.tomo_solve(h, s, F, opts, z, phi)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        launches0 = tomo.tomo_launch_count(h)
        clocks = Clocks(local)
        clocks.start()
        evs = []
        t_wall = time.perf_counter()
        infos = []
        for _ in range(args.steps):
            flush.zero_()                                   # L2 flush between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(tomo.tomo_solve(h, s, F, opts, z, phi))
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        if dist:
            dist.barrier()
        clk = clocks.stop()
        launches = tomo.tomo_launch_count(h) - launches0
        step_ms = [a.elapsed_time(b) for a, b in evs]
        def variant(vopts, **extra):
            """The same frames with other solver options: W warm-up + K timed steps."""
            for _ in range(args.warmup):
                tomo.tomo_solve(h, s, F, vopts, z, phi)
            vevs, vinfos = [], []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                vinfos.append(tomo.tomo_solve(h, s, F, vopts, z, phi))
                e1.record(stream)
                vevs.append((e0, e1))
            torch.cuda.synchronize()
            vms = sum(a.elapsed_time(b) for a, b in vevs)
            vi = vinfos[-1]
            out = {"value": world * F * args.steps / (vms / 1000.0), "unit": UNIT, "ms_per_step": vms / args.steps,
                   "iters_mean": float(vi["iters"].mean()), "iters_max": int(vi["iters"].max()),
                   "relres_max": float(vi["relres"].max()),
                   "all_converged": bool((vi["status"] == 0).all() and (vi["relres"] <= TOL).all())}
            out.update(extra)
            return out

        # the same frames with the block-circulant preconditioner, and with MINRES (reported beside the headline)
        pcg = minres = warm_prev = learned = single = direct = moao = block = learned_block = mixed = None
        learned_flex = None
        small = []
        if not args.no_variants:
            mixed = run_mixed(tomo, torch, W, args, stream, flush, h, cfg, sub, layout, rank, world, 4 * F)
            pcg = variant(tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=16, precond=True),
                          preconditioner=f"block-circulant: per-frequency (K_+(f) + 3 sigma^2)^{{-1}} on the "
                                         f"{layout.P} x {layout.P} torus")
            block = variant(tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, precond=True, method="block"),
                            method="block PCG over the 64 frames (one Krylov space for the batch), block-circulant "
                                   "preconditioner; iters = block iterations")
            minres = variant(tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=32, method="minres"),
                             method="MINRES in conjugate-residual form, unpreconditioned (as the paper ran it)")
            # single-frame latency: one frame per solve (the row passes then run
            # one block per group of 16 row pairs), PCG
            one_opts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=16, precond=True)
            for _ in range(args.warmup):
                tomo.tomo_solve(h, s[:1], 1, one_opts, z[:1], phi[:1])
            oevs, oinfo = [], None
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                oinfo = tomo.tomo_solve(h, s[:1], 1, one_opts, z[:1], phi[:1])
                e1.record(stream)
                oevs.append((e0, e1))
            torch.cuda.synchronize()
            oms = [a.elapsed_time(b) for a, b in oevs]
            single = {"ms_per_frame": statistics.median(oms), "iters": int(oinfo["iters"][0]),
                      "relres": float(oinfo["relres"][0]),
                      "note": "latency of one frame solved alone (PCG, tol 1e-4, projection included)"}
            # the explicit reconstructor (the paper's "direct MVM" comparison):
            # built from n_vphi PCG solves, then applied to the frames as a GEMM
            R = torch.empty((layout.n_vphi, layout.N), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rinfo, wfe = tomo.tomo_reconstructor(h, 0, tomo.solve_opts(tol=1e-5, max_iter=30000, max_refine=3,
                                                                       precond=True, method="block"), R, wfe=True)
            torch.cuda.synchronize()
            build_s = time.perf_counter() - t0
            phiR = torch.empty((F, layout.n_vphi), dtype=torch.float32, device="cuda")
            for _ in range(args.warmup):
                tomo.tomo_apply_reconstructor(h, R, s, F, phiR)
            revs = []
            for _ in range(args.steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tomo.tomo_apply_reconstructor(h, R, s, F, phiR)
                e1.record(stream)
                revs.append((e0, e1))
            torch.cuda.synchronize()
            rms_ = [a.elapsed_time(b) for a, b in revs]
            r_ms = statistics.median(rms_)
            flops_R = 2.0 * F * layout.n_vphi * layout.N
            bytes_R = 4.0 * layout.n_vphi * layout.N
            direct = {"value": world * F / (r_ms / 1000.0), "unit": UNIT, "ms_per_step": r_ms,
                      "build_s": build_s, "build_rows": layout.n_vphi,
                      "build_iters_mean": float(rinfo["iters"].mean()),
                      "build_all_converged": bool((rinfo["status"] == 0).all()),
                      "analytic_wfe_nm": float(wfe[0] * 500.0 / (2 * math.pi)),
                      "R_bytes": bytes_R, "gemm_tflops": flops_R / (r_ms / 1000.0) / 1e12,
                      "gemm_gbs": bytes_R / (r_ms / 1000.0) / 1e9,
                      "note": "R = Sigma_phi_s A^{-1} (target 0) from block-PCG solves at 1e-5 (64 rows at a time), "
                              "applied by the FP32 GEMM; "
                              "value excludes the build; analytic_wfe_nm: Eq. analytical1, piston-removed rms "
                              "over the phase points, the reconstructor's model taken as truth"}
            del R, phiR
            torch.cuda.empty_cache()
            # batched MOAO, laser-star part: 32 target directions within 7', four
            # seeings in one batch (per-frame r0), PCG, projection to every target
            moao = run_moao(tomo, torch, W, args, stream, flush, F, rank, world)
            # closed-loop operation (Sec. 5): frozen-flow sequences at 1 kHz, each step
            # warm-started from the previous step's solution, PCG
            seq, _ = W.slope_sequence_parallel(cfg, F, args.warmup + args.steps + 1, seed=3000 + rank, dt=1e-3)
            seq_s = [torch.tensor(tomo.valid_slopes(seq[t], sub), dtype=torch.float32, device="cuda").contiguous()
                     for t in range(seq.shape[0])]
            wopts = tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=16, precond=True, warm_start=1)
            zs = torch.zeros_like(s)
            cold = tomo.tomo_solve(h, seq_s[0], F, tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3,
                                                                   check_every=16, precond=True), zs, phi)
            for t in range(1, args.warmup + 1):
                tomo.tomo_solve(h, seq_s[t], F, wopts, zs, phi)
            wevs, winfos = [], []
            for t in range(args.warmup + 1, args.warmup + args.steps + 1):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                winfos.append(tomo.tomo_solve(h, seq_s[t], F, wopts, zs, phi))
                e1.record(stream)
                wevs.append((e0, e1))
            torch.cuda.synchronize()
            wms = sum(a.elapsed_time(b) for a, b in wevs)
            wi = winfos[-1]
            warm_prev = {"value": world * F * args.steps / (wms / 1000.0), "unit": UNIT, "ms_per_step": wms / args.steps,
                         "iters_mean": float(np.mean([w["iters"].mean() for w in winfos])),
                         "cold_iters_mean": float(cold["iters"].mean()),
                         "relres_max": float(max(w["relres"].max() for w in winfos)),
                         "all_converged": bool(all((w["status"] == 0).all() and (w["relres"] <= TOL).all()
                                                   for w in winfos)),
                         "workload": ("the same system on frozen-flow sequences (synthetic 9-layer wind, 8-25 m/s, "
                                      "1 ms steps), each step's PCG started from the previous step's zeta")}
            # the learned warm start (trained offline on other seeded frames) in front of the same PCG
            if not args.no_learned:
                l0, l1 = train_warm_start(tomo, torch, h, cfg, layout, sub, seed=2000 + rank)
                learned = variant(tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, check_every=16, precond=True,
                                                  warm_start=2),
                                  training={"frames": 256, "steps": 200, "loss_first": l0, "loss_last": l1,
                                            "network": "3x3 CNN 12-32-32-32-12, FP32, warm start of the PCG"})
                learned_block = variant(tomo.solve_opts(tol=TOL, max_iter=30000, max_refine=3, precond=True,
                                                        warm_start=2, method="block"),
                                        note="the same network as warm start of block PCG")
                learned_flex = run_learned_flexible(tomo, torch, W, args, stream, flush, cfg, s, F, layout.P, rank,
                                                    world)
        if world == 1 and not args.no_cpu_baseline:
            # the library on the small systems the oracle is timed on end to end (same seeds)
            small = [gpu_small(tomo, torch, W, "ngs8m", F, 500, stream, flush, max(1, min(args.steps, 3))),
                     gpu_small(tomo, torch, W, "lgs_mid", F, 501, stream, flush, max(1, min(args.steps, 3)))]
        total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
        value = whole_job_rate(world, F, args.steps, total_ms)
        info = infos[-1]
        iters = info["iters"]
        ok = bool((info["status"] == 0).all() and (info["relres"] <= TOL).all())

        # one extra, separately reported step with per-kernel CUDA-event timing
        tomo.tomo_set_kernel_timing(h, 1)
        tomo.tomo_solve(h, s, F, opts, z, phi)
        torch.cuda.synchronize()
        kms, kn, frame_iters = tomo.tomo_get_kernel_timing(h)
        tomo.tomo_set_kernel_timing(h, 0)
        model = kernel_model(layout)
        # the paper's operation counts for this system beside this design's own model
        cfg_layers = len(cfg["layers"])
        opcount = {k: float(v) for k, v in paper_opcounts(layout.n, layout.n_gs, cfg_layers, layout.n_new).items()}
        opcount["this_design_sigma_ss"] = float(sum(model[k]["flops"] for k in ("rows_fwd", "cols_mul", "rows_inv")))
        opcount["note"] = ("paper: 1-D 2RBT formulation, a = 5 (Sec. 2.E); this design: 2-D real FFTs on a "
                           f"{layout.P}^2 torus, Hermitian block product, same FFT cost model")
        pk = peaks()
        alu_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * pk["sm_max_mhz"] * 1e6 / 1e12   # TFLOP/s
        balance = alu_peak * 1e12 / (pk["hbm_gbs"] * 1e9)
        dom = max(("rows_fwd", "cols_mul", "rows_inv"), key=lambda k: kms[k])
        m = model[dom]
        secs = kms[dom] / 1000.0
        flops = m["flops"] * frame_iters
        byts = m["bytes"] * frame_iters + m["per_launch_bytes"] * kn[dom]
        if flops / byts > balance:
            roof = {"bound": "alu", "achieved": flops / secs / 1e12, "peak": alu_peak, "unit": "TFLOP/s"}
        else:
            roof = {"bound": "hbm", "achieved": byts / secs / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        tr = ncu_traffic(dom)
        roof["traffic"] = None if tr is None else tr * frame_iters / max(1, kn[dom])
        roof["kernel"] = dom
        roof["peak_source"] = ("FP32 FMA: %d SMs x %d lanes x 2 x %.0f MHz" % (SM_COUNT, FP32_LANES_PER_SM, pk["sm_max_mhz"])
                               if roof["bound"] == "alu" else f"HBM copy, {pk['src']}")
        roof["avg_launch_us"] = 1000.0 * kms[dom] / max(1, kn[dom])
        roof["kernel_ms"] = {k: round(v, 3) for k, v in kms.items()}
        # every pass of the product against both bounds (algorithmic bytes and
        # flops of kernel_model over the same CUDA-event time); "bound" is the
        # one the pass's arithmetic intensity puts it under
        per = {}
        for k in ("rows_fwd", "cols_mul", "rows_inv"):
            mk, sk = model[k], kms[k] / 1000.0
            fk = mk["flops"] * frame_iters
            bk = mk["bytes"] * frame_iters + mk["per_launch_bytes"] * kn[k]
            per[k] = {"avg_launch_us": round(1e6 * sk / max(1, kn[k]), 2),
                      "hbm_gbs": round(bk / sk / 1e9, 1), "hbm_frac": round(bk / sk / 1e9 / pk["hbm_gbs"], 4),
                      "alu_tflops": round(fk / sk / 1e12, 2), "alu_frac": round(fk / sk / 1e12 / alu_peak, 4),
                      "bound": "alu" if fk / bk > balance else "hbm"}
        roof["per_kernel"] = per
        roof["whole_product"] = whole_product(model, F, total_ms / args.steps, float(iters.mean()), pk["hbm_gbs"],
                                              alu_peak)

        # end to end through the public host-buffer API, inputs in pinned memory
        s_h = torch.empty((F, layout.N), dtype=torch.float32, pin_memory=True)
        s_h.copy_(s.cpu())
        z_h = torch.empty((F, layout.N), dtype=torch.float32, pin_memory=True)
        p_h = torch.empty((F, layout.n_targets, layout.n_vphi), dtype=torch.float32, pin_memory=True)
        sn, zn, pn = s_h.numpy(), z_h.numpy(), p_h.numpy()
        tomo.tomo_solve_host(h, sn, F, opts, zn, pn)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tomo.tomo_solve_host(h, sn, F, opts, zn, pn)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * F * args.steps / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": F * layout.N * 4,
               "d2h_bytes_per_step": F * layout.N * 4 + F * layout.n_targets * layout.n_vphi * 4}
        tomo.tomo_destroy(h)

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_gpu": F, "N": layout.N, "P": layout.P,
                       "Pcos": layout.Pcos, "n_new": layout.n_new,
                       "fft_P_autotune": {str(int(p)): round(float(t), 4) for p, t in zip(tune_P, tune_ms)},
                       "opcount_per_product": opcount,
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "solver": "CG, FP32 vectors/FFTs/spectra, FP64 dots and alpha/beta, FP64 true residual"},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "pcg": pcg, "block_pcg": block, "minres": minres, "learned_pcg": learned,
            "learned_block_pcg": learned_block, "learned_flexible_pcg": learned_flex,
            "pcg_warm_previous": warm_prev,
            "single_frame_pcg": single, "direct_mvm": direct, "moao_32_targets": moao, "mixed_precision": mixed,
            "solve": {"iters_mean": float(iters.mean()), "iters_max": int(iters.max()),
                      "relres_max": float(info["relres"].max()), "all_converged": ok,
                      "refinements_max": int(info["refinements"].max()),
                      "step_ms": [round(x, 3) for x in step_ms], "wall_s": t_wall}}
    if world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(cfg, frames=F)
        for m, g in zip(cb["measured"], small):
            m.update(g)
        line["cpu_baseline"] = cb
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
