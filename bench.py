"""Benchmark: induced-charge solves/s of Brownian-dynamics steps on the 64-sphere lattice.

One step = one induced-charge solve (mixed precision: FP32 mesh, FP64 Krylov,
FP64-operator residual <= 1e-6), the bead forces, body forces, torques and
energy, and one Brownian-dynamics step of 64 polarizable spheres (642 beads
each) on a 4^3 simple cubic lattice at volume fraction 0.1 with 100,000
monovalent ions (141,088 beads) in a uniform field, on a 256^3 mesh; positions
advance from step to step and each solve starts from the previous step's
charges.  Inputs are resident in HBM when the timed region starts; the L2 is
flushed (a 256 MB write) before every timed step, outside the step's CUDA-event
pair.

Also reported on the same JSON line: PME evaluations/s of the same system
against the HBM roofline, every single-kernel mesh stage against it, the FP64
GPU path with the same algorithm and the plain FP64 GPU path (zero guess, no
preconditioner), the end-to-end rate through the C ABI with host buffers, the
charged-sphere workload (642-bead sphere + 2,050 ions, 128^3) as a second line
of numbers, the oracle on the host cores (extrapolated from a bounded sample),
SM clocks sampled during the timed region and the number of the library's
kernel launches.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload lattice|charged-sphere|polarizability|trajectory]
For N > 1 launch with torchrun: the lattice, charged-sphere and trajectory workloads run one
independent replica per rank (weak scaling); the polarizability batch is split across
the ranks (strong scaling).
--workload charged-sphere times the 2,692-bead charged sphere alone;
--workload polarizability times the batched solve of 64 independent
configurations (three fields each) on the autotuned mesh; --workload
trajectory times BD steps of eight spheres in 20,000 ions with the zero, the
previous-step and the learned initial guess.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "induced-charge solves/s and PME evals/s (HBM roofline %) vs plain FP64 GPU"
LATTICE = ("lattice: 64 polarizable spheres (642 beads each, 41,088 beads) on a 4^3 simple cubic lattice at phi=0.1 "
           "(L=13.89) + 100,000 monovalent ions = 141,088 beads, l_B=0.7, bead radius 0.05, E0=x, mesh 256^3, "
           "tol 1e-6 (xi=7.76, P=9); step = mixed-precision induced-charge solve to FP64 residual 1e-6 from the "
           "previous step's charges + forces/torques/energy + one BD step (dt=1e-3, kT=1), positions advancing")
SPHERE = ("charged sphere: 642-bead icosphere (Q=-50) + 2,050 monovalent ions, L=30, l_B=0.7, bead radius 0.05, "
          "mesh 128^3, tol 1e-6 (xi=1.79, P=9); step = mixed-precision induced-charge solve to FP64 residual "
          "1e-6 from the uniform guess + forces/torques/energy + one BD step (dt=1e-3)")
HBM_FALLBACK_GBS = 6800.0
DT = 1e-3
# Operator applications of a textbook restarted GMRES(50) from the zero guess on the
# lattice's saddle system, the oracle's solver: the Krylov iterations of the plain FP64
# GPU path (zero guess, no preconditioner) at residual 1e-6 plus the initial and final
# residual, as measured on GB300 (see the line's fp64_plain.iters).
ORACLE_MATVECS_LATTICE = 40


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback"


# the kernel behind each single-kernel stage of the library's profiler
STAGE_KERNEL = {"spread": "spread_pairs_kernel<float> / spread_tiles_kernel<float>",
                "gather": "gather_pairs_kernel<float> / gather_tiles_kernel<float>",
                "scale": "scale_kernel<float>", "near_apply": "near_apply_kernel", "near_apply32": "near_apply32_kernel",
                "spread64": "spread_pairs_kernel<double> / spread_tiles_kernel<double>",
                "gather64": "gather_pairs_kernel<double> / gather_tiles_kernel<double>",
                "scale64": "dfz_scale_kernel"}


def measured_traffic(workload, stage):
    """DRAM bytes (read + write) per launch of the stage's kernel on this workload,
    as recorded from an ncu capture in profiles/traffic.json; None if absent."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        return d[workload][stage]["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError, TypeError):
        return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.path is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = []
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), p[5], p[6], p[7], p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([r[0] for r in rows])
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(r[1] for r in rows)),
                "samples": len(rows), "reasons": reasons}


# ---------------------------------------------------------------------------
# the workloads of one BD step per solve
# ---------------------------------------------------------------------------

def make_system(workload: str, rank: int):
    from workloads import configs as C
    if workload == "lattice":
        return C.config3(seed=1002 + 7919 * rank)
    return C.config2(seed=1001 + 7919 * rank)


GUESS = {"lattice": "previous", "charged-sphere": "uniform"}


class Step:
    """Device-resident state of one replica and its one-call step (ibpme_bd_advance).

    guess: "previous" -- the previous step's charges (zero at the first step);
    "uniform" -- the system's own initial charges every step; "zero"."""

    def __init__(self, ib, torch, s, precision, guess, precond=None, ctx=None):
        self.ib, self.torch, self.s = ib, torch, s
        dev = "cuda"
        f64 = torch.float64
        self.n, self.nb = s.n, s.n_bodies
        self.stream = torch.cuda.current_stream()
        self.own_ctx = ctx is None
        self.ctx = ctx if ctx is not None else ib.pme_setup(
            ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=s.a, eps_f=s.eps, precision=precision,
                           max_rhs=1), self.stream)
        self.precision, self.guess = precision, guess
        self.precond = ib.IBPME_PRECOND_BODY if precond is None else precond
        t = lambda a, dt=f64: torch.as_tensor(np.ascontiguousarray(a)).to(dt).to(dev)
        self.x = t(s.x)
        self.x_next = torch.empty_like(self.x)
        self.X = t(s.X)
        self.X_next = torch.empty_like(self.X)
        self.off = t(s.body_offsets, torch.int32)
        self.Q = t(s.Q)
        self.E0 = t(s.E0[:1])
        q0 = s.q_guess if s.q_guess is not None else np.zeros(s.n)
        self.q0 = t(q0.reshape(1, -1))
        self.q = torch.zeros_like(self.q0)
        self.psi = torch.zeros((1, self.nb), dtype=f64, device=dev)
        self.f = torch.zeros((self.n, 3), dtype=f64, device=dev)
        self.F = torch.zeros((self.nb, 3), dtype=f64, device=dev)
        self.L = torch.zeros((self.nb, 3), dtype=f64, device=dev)
        self.U = torch.zeros(1, dtype=f64, device=dev)
        self.step_no = 0
        self.last_stats = None

    def run(self):
        ib = self.ib
        bodies = ib.Bodies(self.off, self.X, self.Q)
        if self.guess == "uniform":
            self.q.copy_(self.q0)
            g = ib.IBPME_GUESS_USER
        elif self.guess == "zero":
            self.q.zero_()
            g = ib.IBPME_GUESS_ZERO
        else:
            g = ib.IBPME_GUESS_USER if self.step_no > 0 else ib.IBPME_GUESS_ZERO
        opts = ib.make_opts(rtol=1e-6, guess=g, precision=self.precision, precond=self.precond)
        # solve + forces/torques/energy + BD step: one library call
        status, st = ib.ibpme_bd_advance(self.ctx, self.n, self.x, bodies, self.E0[0], opts, self.q[0], DT,
                                         1.0, 1.0, 1234, self.step_no, self.F, self.L, self.x_next, self.X_next,
                                         psi_out=self.psi[0], f_bead=self.f, U=self.U)
        if status != ib.IBPME_OK:
            raise RuntimeError(f"solve did not converge: residual {st.rel_residual:.3e}")
        self.x, self.x_next = self.x_next, self.x
        self.X, self.X_next = self.X_next, self.X
        self.step_no += 1
        self.last_stats = st
        return st

    def close(self):
        if self.own_ctx:
            self.ib.pme_destroy(self.ctx)


class HostStep:
    """The same step through the C ABI with host (numpy) buffers: the library
    stages every input to the device and every output back."""

    def __init__(self, ib, s, ctx, guess):
        self.ib, self.s, self.ctx, self.guess = ib, s, ctx, guess
        self.x = np.ascontiguousarray(s.x)
        self.X = np.ascontiguousarray(s.X)
        self.off = np.ascontiguousarray(s.body_offsets, dtype=np.int32)
        self.Q = np.ascontiguousarray(s.Q)
        self.E0 = np.ascontiguousarray(s.E0[:1])
        q0 = s.q_guess if s.q_guess is not None else np.zeros(s.n)
        self.q0 = np.ascontiguousarray(q0.reshape(1, -1))
        n, nb = s.n, s.n_bodies
        self.q = np.zeros((1, n))
        self.psi = np.zeros((1, nb))
        self.f = np.zeros((n, 3))
        self.F = np.zeros((nb, 3))
        self.L = np.zeros((nb, 3))
        self.U = np.zeros(1)
        self.x_next = np.zeros_like(self.x)
        self.X_next = np.zeros_like(self.X)
        self.step_no = 0
        body = self.off.nbytes + self.X.nbytes + self.Q.nbytes
        # bytes copied per step, counted from the arrays the one call stages
        self.h2d = self.x.nbytes + body + 24 + self.q.nbytes                  # q_io read as the guess
        self.d2h = (self.q.nbytes + self.psi.nbytes + self.f.nbytes + self.F.nbytes + self.L.nbytes
                    + self.U.nbytes + self.x_next.nbytes + self.X_next.nbytes)

    def run(self):
        ib = self.ib
        bodies = ib.Bodies(self.off, self.X, self.Q)
        if self.guess == "uniform":
            self.q[:] = self.q0
        g = ib.IBPME_GUESS_USER if (self.guess == "uniform" or self.step_no > 0) else ib.IBPME_GUESS_ZERO
        opts = ib.make_opts(rtol=1e-6, guess=g, precision=ib.IBPME_MIXED)
        status, st = ib.ibpme_bd_advance(self.ctx, self.s.n, self.x, bodies, self.E0[0], opts, self.q[0], DT,
                                         1.0, 1.0, 1234, self.step_no, self.F, self.L, self.x_next, self.X_next,
                                         psi_out=self.psi[0], f_bead=self.f, U=self.U)
        if status != ib.IBPME_OK:
            raise RuntimeError("host-buffer solve did not converge")
        self.x, self.x_next = self.x_next, self.x
        self.X, self.X_next = self.X_next, self.X
        self.step_no += 1


# ---------------------------------------------------------------------------
# roofline work models
# ---------------------------------------------------------------------------

# FP32 operations of the double-float primitives (dfloat.cuh, dffft.cu): two_sum 6,
# fast_two_sum 3, df_add 11, df_mul 7, complex multiply 4 df_mul + 2 df_add = 50, complex
# add 22; an r-point DFT of radix-2 butterflies takes r log2(r) complex additions: radix-2
# 2 x 22 = 44, radix-4 8 x 22 = 176 (its -i is free), radix-8 24 x 22 plus two multiplies by
# w8 (2 x 11 + 2 x 7 = 36 each; w8^2 = -i is free) = 600.  The radix-3 DFT takes five
# complex additions (110), two df_add and two exact halvings (22 + 4) and two df_mul by
# sqrt(3)/2 (14) = 150.
DF_CMUL, DF_DFT = 50, {2: 44, 3: 150, 4: 176, 8: 600}


def df_mesh_size(n):
    """Whether the library's double-float transform takes an axis of n points:
    n = 2^k or 3 2^k with a power-of-two part of at least 8, 16 <= n <= 1024."""
    m = n // 3 if n % 3 == 0 else n
    return 16 <= n <= 1024 and m & (m - 1) == 0 and (m == n or m >= 8)


def df_transform_ops(n):
    """FP32 operations per point of one length-n double-float Stockham transform:
    a radix-3 pass when 3 divides n, radix-8 passes, then one radix-4 or radix-2
    pass; the twiddles of a pass with sub-transform length Ns are trivial for the
    1/Ns of its butterflies with k = 0 and are not counted."""
    passes = [3] if n % 3 == 0 else []
    l = int(round(np.log2(n // 3 if n % 3 == 0 else n)))
    while l >= 3:
        passes.append(8)
        l -= 3
    if l:
        passes.append(2 ** l)
    ops, ns = 0.0, 1
    for r in passes:
        ops += ((1.0 - 1.0 / ns) * (r - 1) * DF_CMUL + DF_DFT[r]) / r
        ns *= r
    return ops


def stage_work(stage, s, npairs, df_mesh):
    """(bound, algorithmic work per launch, unit) of a stage's kernel.  Every mesh stage
    is scored by its algorithmic HBM bytes; the double-float z pass also has an FP32
    operation count (alu_work)."""
    b = stage_bytes(stage, s, npairs, df_mesh)
    return ("hbm", b, "GB/s") if b is not None else (None, None, None)


def alu_work(s):
    """FP32 operations of one double-float z pass: forward z transform, Green's-function
    scaling (2 df_mul), inverse z transform, over the half spectrum (N_z N_y (N_x/2+1)
    points; the padded columns are not counted)."""
    pts = s.mesh[2] * s.mesh[1] * (s.mesh[0] // 2 + 1)
    return pts * (2 * df_transform_ops(s.mesh[2]) + 14)


def alu_peak():
    """FP32 operations per second: 152 SMs x 128 FP32 lanes x the maximum SM clock."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except (OSError, KeyError, ValueError):
        mhz = 2070.0
    return 152 * 128 * mhz * 1e6 / 1e9, f"derived: 152 SMs x 128 FP32 lanes x {mhz:.0f} MHz"


def stage_bytes(stage, s, npairs, df_mesh=False):
    """Algorithmic bytes per launch (one field): the grid written (spread) or read
    (gather) once plus positions (24 B) and a charge or potential (8 B) per bead; the
    scaling reads and writes the half spectrum and reads the Green's table; the
    double-float z pass the same with 16-byte double-float complex points and an
    8-byte double-float Green's table."""
    G = int(np.prod(s.mesh))
    Gc = s.mesh[2] * s.mesh[1] * (s.mesh[0] // 2 + 1)
    n = s.n
    w = 8 if stage.endswith("64") else 4
    base = stage[:-2] if stage.endswith("64") else stage
    if base == "spread":
        return G * w + n * (24 + 8)           # grid written once; positions and charges read
    if base == "gather":
        return G * w + n * (24 + 8)           # grid read once; positions read, potentials written
    if base == "scale":
        if stage == "scale64" and df_mesh:
            return Gc * (2 * 16 + 8)          # float4 half spectrum read + written, float2 Green's table
        return Gc * (2 * 2 * w + w)           # half spectrum read and written, Green's table read
    if base in ("fft_forward", "fft_inverse"):
        return 2 * G * w
    if base == "near_apply":
        return npairs * (4 + 8) + n * (8 + 8 + 8 + 8)   # col + value per pair; q, psi, row offsets
    if base == "near_apply32":
        # (col, FP32 value) word per pair; q read and packed (16 B), row offsets, order, psi
        return npairs * 8 + n * (8 + 16 + 8 + 4 + 8)
    return None


def pme_bytes(s, w=4, R=1):
    """Algorithmic bytes of one PME evaluation: 6 G w R + N (32 + 8 R)."""
    return 6 * int(np.prod(s.mesh)) * w * R + s.n * (32 + 8 * R)


def pair_count(ib, ctx, s, x):
    """Real-space pairs within r_cut of the current configuration (a property of
    the workload, counted on the host with a periodic k-d tree; it sizes the SpMV's
    algorithmic bytes)."""
    from scipy.spatial import cKDTree
    rc = ib.ibpme_get_params(ctx).r_cut
    box = np.asarray(s.box, dtype=np.float64)
    xw = x - box * np.floor(x / box)
    xw = np.where(xw >= box, xw - box, xw)
    return 2 * len(cKDTree(xw, boxsize=box).query_pairs(rc))


def timed_steps(torch, step, k, flush, stream):
    """k steps, each bracketed by CUDA events on the library's stream, the L2 flushed
    before each (outside its events); returns the per-step milliseconds."""
    e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for i in range(k):
        flush.zero_()
        e[i][0].record(stream)
        step.run()
        e[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in e]


def bench_ours(args, ib, torch, rank, world, local):
    dev_index = local
    torch.cuda.set_device(dev_index)
    wl = args.workload
    s = make_system(wl, rank)
    guess = GUESS[wl]
    st = Step(ib, torch, s, ib.IBPME_MIXED, guess)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # warm-up, with every stage timed once to find the dominant kernel
    ib.ibpme_profile((1 << len(ib.STAGES)) - 1)
    for _ in range(args.warmup):
        st.run()
    prof = ib.ibpme_profile_read()
    # candidates: stages of the calling stream that are one own kernel each with a work model
    # (cuFFT is a library; the table build, the Krylov group and the body reductions are
    # composite; the near-field stages run on the second stream, where their events also
    # time the wait for the mesh pass they overlap)
    df_mesh = all(df_mesh_size(int(m)) for m in s.mesh)   # FP64 mesh in double-float transforms
    cand = ("spread", "gather", "scale", "spread64", "gather64", "scale64")
    own = {k: v for k, v in prof.items() if k in cand and v[1] > 0}
    dominant = max(own, key=lambda k: own[k][0]) if own else "spread"
    dom_idx = ib.STAGES.index(dominant)
    warm_profile = {k: {"ms": round(v[0], 4), "launches": v[1]} for k, v in prof.items() if v[1]}

    # timed region: every candidate stage carries events (the events add no work to the step)
    mask = 0
    for k in own:
        mask |= 1 << ib.STAGES.index(k)
    ib.ibpme_profile(mask | (1 << dom_idx))
    launches0 = ib.ibpme_kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters = []
    with ClockSampler(dev_index) as clk:
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(st.stream)
            stats = st.run()
            ev[i][1].record(st.stream)
            iters.append((stats.iters, stats.outer, stats.matvecs_fp64, stats.rel_residual, stats.init_rel_residual))
        barrier()
        wall = time.perf_counter() - t0
    launches = ib.ibpme_kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(np.sum(step_ms))
    timed_prof = ib.ibpme_profile_read()
    ib.ibpme_profile(0)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    npairs = pair_count(ib, st.ctx, s, st.x.cpu().numpy())
    peak, peak_kind = peaks()

    def roof(stage, prof_entry):
        bound, work, unit = stage_work(stage, s, npairs, df_mesh)
        launches_k = prof_entry[1]
        avg = prof_entry[0] / launches_k if launches_k else float("nan")
        ach = work / (avg / 1e3) / 1e9 if work and launches_k else None
        out = {"kernel": STAGE_KERNEL.get(stage, stage), "stage": stage, "bound": bound, "achieved": ach,
               "peak": peak, "unit": unit, "frac": (ach / peak) if ach else None, "peak_source": peak_kind,
               "alg_bytes_per_launch": work, "avg_launch_ms": avg, "launches": launches_k,
               "traffic": measured_traffic(wl, stage)}
        if stage == "scale64" and df_mesh:
            ops = alu_work(s)
            apk, apk_kind = alu_peak()
            a_ach = ops / (avg / 1e3) / 1e9 if launches_k else None
            out["alu_model"] = {"bound": "alu", "alg_ops_per_launch": ops, "achieved": a_ach, "peak": apk,
                                "unit": "Gop/s", "frac": (a_ach / apk) if a_ach else None, "peak_source": apk_kind}
        return out

    # PME evaluations alone on the same system (potential of the current charges)
    pme = pme_rate(ib, torch, st, flush, max(10, args.steps))

    # FP64 GPU paths: the same step with every mesh step in FP64 (same guess and
    # preconditioner), and the plain FP64 path (zero guess, no preconditioner)
    fp64 = {}
    if not args.skip_fp64:
        for name, g, pc in (("fp64_same_algorithm", guess, ib.IBPME_PRECOND_BODY),
                            ("fp64_plain", "zero", ib.IBPME_PRECOND_NONE)):
            st64 = Step(ib, torch, s, ib.IBPME_FP64, g, precond=pc)
            st64.run()
            st64.run()
            torch.cuda.synchronize()
            k64 = 3 if wl == "lattice" else max(3, args.steps // 5)
            ms = timed_steps(torch, st64, k64, flush, st64.stream)
            s64 = st64.last_stats
            fp64[name] = {"solves_per_s": k64 / (sum(ms) / 1e3), "ms_per_step": sum(ms) / k64, "steps": k64,
                          "iters": s64.iters, "fp64_matvecs": s64.matvecs_fp64, "rel_residual": s64.rel_residual,
                          "guess": g, "preconditioner": "body blocks" if pc == ib.IBPME_PRECOND_BODY else "none"}
            st64.close()

    # end to end through the C ABI with host buffers
    hs = HostStep(ib, s, st.ctx, guess)
    hs.run()
    torch.cuda.synchronize()
    k_e2e = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        hs.run()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    stage_roofs = {k: roof(k, timed_prof[k]) for k in own if timed_prof[k][1]}
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 mesh / f64 near-field+krylov",
        "data": "synthetic",
        "config": {"workload": LATTICE if wl == "lattice" else SPHERE, "n_beads": s.n, "n_bodies": s.n_bodies,
                   "mesh": list(s.mesh), "initial_guess": {"previous": "the previous step's charges",
                                                           "uniform": "the uniform charge -50/642"}[guess],
                   "l2": "L2 flushed (256 MB write) before every timed step, outside its events",
                   "parallelism": f"replicas x{world} (independent systems, no collective)"},
        "roofline": stage_roofs.get(dominant),
        "stage_rooflines": {k: {"ms_per_launch": v["avg_launch_ms"], "GB/s": v["achieved"], "frac": v["frac"],
                                "launches": v["launches"]} for k, v in stage_roofs.items()},
        "pme_evals_per_s": pme["evals_per_s"],
        "pme_roofline": pme["roofline"],
        "fp64_gpu": fp64 or None,
        "speedup_vs_fp64_plain": (value / world / fp64["fp64_plain"]["solves_per_s"]) if fp64 else None,
        "speedup_vs_fp64_same_algorithm": (value / world / fp64["fp64_same_algorithm"]["solves_per_s"])
        if fp64 else None,
        "solve": {"iters_mean": float(np.mean([i[0] for i in iters])),
                  "outer_mean": float(np.mean([i[1] for i in iters])),
                  "fp64_matvecs_mean": float(np.mean([i[2] for i in iters])),
                  "rel_residual_max": float(np.max([i[3] for i in iters])),
                  "init_rel_residual_mean": float(np.mean([i[4] for i in iters]))},
        "e2e": {"value": world * k_e2e / e2e_s if world == 1 else k_e2e / e2e_s, "unit": "solves/s",
                "h2d_bytes_per_step": hs.h2d, "d2h_bytes_per_step": hs.d2h},
        "gpu_launches": int(launches),
        "wall_s": wall,
        "warmup_stage_ms": warm_profile,
        "clocks": clk.summary(),
    }
    st.close()
    if wl == "lattice" and not args.skip_second:
        out["charged_sphere"] = second_workload(ib, torch, rank, flush, max(10, args.steps))
        out["unequal_radii"] = radii_workload(ib, torch, s, flush, max(10, args.steps), value / world)
        out["rpy_mobility"] = rpy_at_scale(ib, torch, s, flush, max(10, args.steps))
    elif wl != "lattice" and not args.skip_scale:
        out["pme_at_scale"] = pme_at_scale(ib, torch, flush, 10)
    return out, s


def second_workload(ib, torch, rank, flush, k):
    """The charged-sphere workload (2,692 beads, 128^3) timed the same way."""
    s = make_system("charged-sphere", rank)
    st = Step(ib, torch, s, ib.IBPME_MIXED, GUESS["charged-sphere"])
    for _ in range(5):
        st.run()
    torch.cuda.synchronize()
    ms = timed_steps(torch, st, k, flush, st.stream)
    pme = pme_rate(ib, torch, st, flush, k)
    out = {"workload": SPHERE, "solves_per_s": k / (sum(ms) / 1e3), "ms_per_step": sum(ms) / k, "steps": k,
           "iters": st.last_stats.iters, "pme_evals_per_s": pme["evals_per_s"], "pme_roofline": pme["roofline"]}
    st.close()
    return out


RADII_WORKLOAD = ("the lattice step with the 100,000 ions at bead radius 0.1 and the surface beads at 0.05 "
                  "(two radius classes: class mesh channels, two-radius pair kernel)")


def radii_workload(ib, torch, s, flush, k, one_radius_value):
    """The lattice step (same system, guess and precision) with beads of two radii:
    the ions at twice the surface beads' radius."""
    ion = np.diff(s.body_offsets)[np.repeat(np.arange(s.n_bodies), np.diff(s.body_offsets))] == 1
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, eps_f=s.eps, precision=ib.IBPME_MIXED,
                                      max_rhs=1, class_radius=(s.a, 2.0 * s.a)), torch.cuda.current_stream())
    try:
        ib.ibpme_set_radius_classes(ctx, s.n, ion.astype(np.int32))
        st = Step(ib, torch, s, ib.IBPME_MIXED, GUESS["lattice"], ctx=ctx)
        for _ in range(4):
            st.run()
        ib.ibpme_profile((1 << len(ib.STAGES)) - 1)   # stage times of one warm step, outside the timed steps
        st.run()
        torch.cuda.synchronize()
        prof = ib.ibpme_profile_read()
        ib.ibpme_profile(0)
        ms = timed_steps(torch, st, k, flush, st.stream)
        rate = k / (sum(ms) / 1e3)
        out = {"workload": RADII_WORKLOAD, "solves_per_s": rate, "ms_per_step": sum(ms) / k, "steps": k,
               "iters": st.last_stats.iters, "r_cut": ib.ibpme_get_params(ctx).r_cut,
               "vs_one_radius": rate / one_radius_value,
               "warm_stage_ms": {kk: {"ms": round(v[0], 4), "launches": v[1]} for kk, v in prof.items() if v[1]}}
        st.close()
    finally:
        ib.pme_destroy(ctx)
    return out


RPY_WORKLOAD = ("RPY mobility product U = M F (periodic Rotne-Prager-Yamakawa, Hasimoto split on the "
                "spectral-Ewald mesh) at the lattice's 141,088 bead positions, bead radius 0.05, 256^3 FP32 mesh, "
                "FP64 real space, tol 1e-6, random forces")


def rpy_at_scale(ib, torch, s, flush, k):
    """The RPY mobility product at the lattice positions (FP32 mesh of three force channels,
    FP64 real space); positions unchanged between products, L2 flushed before each."""
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=s.a, eps_f=s.eps,
                                      precision=ib.IBPME_MIXED, max_rhs=3), torch.cuda.current_stream())
    try:
        stream = torch.cuda.current_stream()
        x = torch.as_tensor(np.ascontiguousarray(s.x), device="cuda")
        F = torch.as_tensor(np.random.default_rng(7).normal(size=(s.n, 3)), device="cuda")
        U = torch.zeros_like(F)
        for _ in range(3):
            ib.ibpme_rpy_mobility(ctx, s.n, x, F, 1.0, U)
        ib.ibpme_profile((1 << len(ib.STAGES)) - 1)   # stage times of one warm product
        ib.ibpme_rpy_mobility(ctx, s.n, x, F, 1.0, U)
        torch.cuda.synchronize()
        prof = ib.ibpme_profile_read()
        ib.ibpme_profile(0)
        tot = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(k):
            flush.zero_()
            e0.record(stream)
            ib.ibpme_rpy_mobility(ctx, s.n, x, F, 1.0, U)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
    finally:
        ib.pme_destroy(ctx)
    return {"workload": RPY_WORKLOAD, "products_per_s": k / (tot / 1e3), "ms_per_product": tot / k, "steps": k,
            "warm_stage_ms": {kk: {"ms": round(v[0], 4), "launches": v[1]} for kk, v in prof.items() if v[1]}}


def bench_rpy(args, ib, torch, rank, world, local):
    """--workload rpy: the RPY mobility product at the lattice positions, K products timed
    with CUDA events (L2 flushed before each), the dominant own kernel against the HBM peak,
    and the same product through host buffers end to end."""
    from workloads import configs as C
    torch.cuda.set_device(local)
    s = C.config3(seed=1002 + 7919 * rank)
    stream = torch.cuda.current_stream()
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=s.a, eps_f=s.eps,
                                      precision=ib.IBPME_MIXED, max_rhs=3), stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    x = torch.as_tensor(np.ascontiguousarray(s.x), device="cuda")
    Fh = np.random.default_rng(7 + rank).normal(size=(s.n, 3))
    F = torch.as_tensor(Fh, device="cuda")
    U = torch.zeros_like(F)
    for _ in range(args.warmup):
        ib.ibpme_rpy_mobility(ctx, s.n, x, F, 1.0, U)
    cand = ("spread", "gather", "rpy_near")
    mask = 0
    for k in cand:
        mask |= 1 << ib.STAGES.index(k)
    ib.ibpme_profile(mask)
    launches0 = ib.ibpme_kernel_launches()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            ib.ibpme_rpy_mobility(ctx, s.n, x, F, 1.0, U)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = ib.ibpme_kernel_launches() - launches0
    prof = ib.ibpme_profile_read()
    ib.ibpme_profile(0)
    total_ms = float(sum(a.elapsed_time(b) for a, b in ev))
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    npairs = pair_count(ib, ctx, s, s.x)
    # algorithmic bytes per launch: the spread writes three FP32 grids and reads positions and forces;
    # the gather reads three grids and writes three velocities; the real space reads positions, forces,
    # row offsets and columns once and writes the velocities
    G = int(np.prod(s.mesh))
    alg = {"spread": 3 * G * 4 + s.n * 48, "gather": 3 * G * 4 + s.n * 48,
           "rpy_near": s.n * (24 + 24 + 24 + 8 + 4) + 4 * npairs}
    own = {k: v for k, v in prof.items() if k in cand and v[1] > 0}
    dom = max(own, key=lambda k: own[k][0])
    t_dom = own[dom][0] / own[dom][1] / 1e3
    peak, kind = peaks()
    # end to end: host positions and forces in, host velocities out
    xh = np.ascontiguousarray(s.x)
    Uh = np.zeros((s.n, 3))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ib.ibpme_rpy_mobility(ctx, s.n, xh, Fh, 1.0, Uh)
    e2e_s = time.perf_counter() - t0
    # the rigid-body mobility problem on the lattice's bodies (64 spheres, 100,000 single beads),
    # random forces and torques, rtol 1e-6: one solve after a warm one
    off = np.ascontiguousarray(s.body_offsets, dtype=np.int32)
    bodies = ib.Bodies(torch.as_tensor(off, device="cuda"), torch.as_tensor(np.ascontiguousarray(s.X), device="cuda"),
                       torch.zeros(s.n_bodies, dtype=torch.float64, device="cuda"))
    FLr = torch.as_tensor(np.random.default_rng(11).normal(size=(s.n_bodies, 6)), device="cuda")
    Wr = torch.zeros((s.n_bodies, 6), dtype=torch.float64, device="cuda")
    rig = []
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status, st = ib.ibpme_rigid_mobility(ctx, s.n, x, bodies, FLr, 1.0, ib.make_opts(rtol=1e-6, max_iter=600), Wr)
        torch.cuda.synchronize()
        rig.append((time.perf_counter() - t0, st.iters, st.outer, st.rel_residual, status))
    ib.pme_destroy(ctx)
    value = world * args.steps / (total_ms / 1e3)
    return {
        "rigid_solve": {"what": "rigid-body mobility problem (constraint forces and body motions) of the lattice's "
                                "64 spheres and 100,000 single beads, random (F, L), GMRES(50) to rtol 1e-6, wall "
                                "clock of the second of two solves",
                        "ms": rig[1][0] * 1e3, "iters": rig[1][1], "outer": rig[1][2], "rel_residual": rig[1][3],
                        "status": rig[1][4], "unknowns": 3 * s.n + 6 * s.n_bodies},
        "metric": "RPY mobility products/s", "value": value, "unit": "products/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 mesh / f64 real space",
        "data": "synthetic",
        "config": {"workload": RPY_WORKLOAD, "n_beads": s.n, "mesh": list(s.mesh), "pairs": int(npairs),
                   "l2": "flushed (256 MB write) before each product"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": alg[dom] / t_dom / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg[dom] / t_dom / 1e9 / peak, "alg_bytes_per_launch": alg[dom],
                     "ms_per_launch": t_dom * 1e3, "peak_source": kind, "traffic": None},
        "stage_ms_per_product": {k: round(v[0] / args.steps, 4) for k, v in own.items()},
        "e2e": {"value": world * args.steps / e2e_s, "unit": "products/s", "h2d_bytes_per_step": 2 * 24 * s.n,
                "d2h_bytes_per_step": 24 * s.n},
        "gpu_launches": int(launches), "clocks": clk.summary(),
        "cpu_baseline": None,
        "cpu_baseline_note": ("not timed: the oracle's explicit k-sum over 141,088 sources and its radial "
                              "quadrature per pair take far beyond a bounded sample"),
    }


def pme_rate(ib, torch, st, flush, k):
    """PME evaluations (pme_field, potential of one field, FP32 mesh) of the step's
    system at its current positions and charges; L2 flushed before each one."""
    s = st.s
    psi = torch.zeros((1, s.n), dtype=torch.float64, device="cuda")
    ib.pme_field(st.ctx, s.n, st.x, st.q, 1, psi, None)
    torch.cuda.synchronize()
    tot = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(k):
        flush.zero_()
        e0.record(st.stream)
        ib.pme_field(st.ctx, s.n, st.x, st.q, 1, psi, None)
        e1.record(st.stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    t = tot / k / 1e3
    alg = pme_bytes(s)
    peak, kind = peaks()
    return {"evals_per_s": 1.0 / t, "roofline": {"bound": "hbm", "achieved": alg / t / 1e9, "peak": peak,
                                                  "unit": "GB/s", "frac": alg / t / 1e9 / peak,
                                                  "alg_bytes_per_eval": alg, "ms_per_eval": t * 1e3,
                                                  "peak_source": kind}}


def pme_at_scale(ib, torch, flush, k):
    """The PME evaluation of the lattice (141,088 beads, 256^3 FP32 mesh, one field)
    with random neutral charges; positions unchanged between evaluations."""
    from workloads import configs as C
    s = C.config3()
    ctx = ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=s.a, eps_f=s.eps,
                                      precision=ib.IBPME_MIXED, max_rhs=1), torch.cuda.current_stream())
    try:
        rng = np.random.default_rng(1002)
        qh = rng.choice([-1.0, 1.0], size=s.n)
        qh -= qh.mean()

        class _St:
            pass
        st = _St()
        st.s, st.ctx, st.stream = s, ctx, torch.cuda.current_stream()
        st.x = torch.as_tensor(np.ascontiguousarray(s.x), device="cuda")
        st.q = torch.as_tensor(qh.reshape(1, -1), device="cuda")
        out = pme_rate(ib, torch, st, flush, k)
    finally:
        ib.pme_destroy(ctx)
    out["workload"] = "the lattice (141,088 beads, 256^3 FP32 mesh, tol 1e-6), one field, random charges"
    return out


# ---------------------------------------------------------------------------
# batched polarizability workload (--workload polarizability)
# ---------------------------------------------------------------------------

POL_WORKLOAD = ("polarizability batch: 64 independent configurations of 1-8 rods/cubes/ellipsoids with 500-5,000 "
                "beads each (565,030 beads), L=40, one bead radius 0.45 x the batch's smallest bead spacing, "
                "E0 = x, y, z; step = one batched mixed-precision solve of all 192 systems to FP64 residual 1e-6, "
                "every configuration translated by a new random vector each step (cells, pair tables and stencils "
                "rebuilt inside the step)")


def bench_polarizability(args, ib, torch, rank, world, local):
    """One step = the whole batch solved bucket by bucket (configurations the
    body-block preconditioner covers apart from the others), each bucket one
    induced_charge_solve_batch on the mesh the autotuner picks for it; also the
    first configurations solved one call each."""
    import tempfile as _tf

    from paper_2401_04865_gb300 import batch as B
    from workloads import configs as C
    torch.cuda.set_device(local)
    batch = C.config4_batch(n_configs=args.configs, seed=1003, common_radius=True)
    # one batch for the whole job: each rank solves its longest-processing-time share
    plan = B.shard_lpt([B.cost_model(s.n) for s in batch], world)
    mine = plan[rank]
    systems = [batch[i] for i in mine]
    a, eps, tol = systems[0].a, systems[0].eps, 1e-6
    tuner = B.Autotuner(cache_path=os.path.join(_tf.mkdtemp(), "tune.json"), candidates=(96, 128, 160))
    plan_buckets = []
    for idx in B.buckets([s.n for s in systems], ratio=args.bucket_ratio, max_channels=192, nrhs=3,
                         classes=[B.preconditioned(s) for s in systems]):
        bucket = B.Bucket(ib, [systems[i] for i in idx], np.eye(3))
        mesh, report = tuner.tune(ib, bucket, tol, a, eps, ib.IBPME_MIXED)
        ctx = B.context_for(ib, systems[0].box, mesh, tol, a, eps, ib.IBPME_MIXED, 3)
        plan_buckets.append({"idx": idx, "bucket": bucket, "ctx": ctx, "mesh": mesh, "report": report})
    opts = ib.make_opts(rtol=1e-6)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    # every step solves the batch at new positions (each configuration shifted
    # rigidly), so the cells, pair tables and stencils are built inside the step
    rng = np.random.default_rng(2024 + rank)
    positions = [[p["bucket"].shifted_positions(rng) for p in plan_buckets] for _ in range(args.warmup + args.steps)]

    def step(k):
        for p, (x, X) in zip(plan_buckets, positions[k]):
            p["bucket"].load_positions(x, X)
        flush.zero_()

    def solve_all():
        out = []
        for p in plan_buckets:
            status, st = p["bucket"].solve(p["ctx"], opts)
            if status != ib.IBPME_OK:
                raise RuntimeError("batched solve did not converge")
            out.append(st)
        return out

    for k in range(args.warmup):
        step(k)
        solve_all()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    launches0 = ib.ibpme_kernel_launches()
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            step(args.warmup + i)          # new positions and the L2 flush, outside the events
            torch.cuda.nvtx.range_push("pol_timed")   # lets ncu capture exactly the timed batches
            ev[i][0].record(stream)
            stats.append(solve_all())
            ev[i][1].record(stream)
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    launches = ib.ibpme_kernel_launches() - launches0
    total_ms = float(np.sum([e0.elapsed_time(e1) for e0, e1 in ev]))
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = len(batch) * args.steps / (total_ms / 1e3)
    # the last step's tensors of every configuration, gathered on rank 0 in batch order
    # (host objects, after the timed region)
    mine_tensors = {}
    for p in plan_buckets:
        S = p["bucket"].S.cpu().numpy()
        for k, i in enumerate(p["idx"]):
            lo, hi = p["bucket"].cfg[k], p["bucket"].cfg[k + 1]
            mine_tensors[mine[i]] = np.transpose(S[:, lo:hi, :], (1, 2, 0))
    gathered = [mine_tensors]
    if world > 1:
        gathered = [None] * world if rank == 0 else None
        torch.distributed.gather_object(mine_tensors, gathered, dst=0)
    n_gathered = sum(len(g) for g in gathered) if rank == 0 else None
    # the same configurations one call each (context of their bucket), each at
    # new positions, timed the same way
    where = {i: p for p in plan_buckets for i in p["idx"]}
    t_seq = 0.0
    for i in range(len(systems)):
        one = B.Bucket(ib, [systems[i]], np.eye(3))
        one.solve(where[i]["ctx"], opts)
        x, X = one.shifted_positions(rng)
        one.load_positions(x, X)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status, _ = one.solve(where[i]["ctx"], opts)
        e1.record(stream)
        torch.cuda.synchronize()
        if status != ib.IBPME_OK:
            raise RuntimeError("single-configuration solve did not converge")
        t_seq += e0.elapsed_time(e1) / 1e3
    for p in plan_buckets:
        ib.pme_destroy(p["ctx"])
    n_beads = int(sum(s.n for s in systems))
    return {
        "metric": "polarizability configurations/s (batched induced-charge solves, 3 fields each)",
        "value": value, "unit": "configurations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32 mesh / f64 krylov", "data": "synthetic",
        "config": {"workload": POL_WORKLOAD if args.configs == 64 else
                   f"{args.configs}-configuration prefix of: {POL_WORKLOAD}", "n_configs": args.configs,
                   "n_beads": int(sum(s.n for s in batch)),
                   "l2": "inputs larger than L2; 256 MB flush before every step, outside its events",
                   "parallelism": f"one batch over {world} rank(s): longest-processing-time shares, tensors "
                                  f"gathered on rank 0 over the host (no device collective)",
                   "bucket_ratio": args.bucket_ratio},
        "buckets": [{"configs": len(p["idx"]), "beads": p["bucket"].n, "mesh": p["mesh"],
                     "preconditioned": bool(B.preconditioned(systems[p["idx"][0]])),
                     "iters": stats[-1][k][0].iters, "autotune": p["report"]} for k, p in enumerate(plan_buckets)],
        "gathered_configurations": n_gathered,
        "rank_share": {"configurations": len(systems), "beads": n_beads},
        "one_call_per_configuration": {"value": len(systems) / t_seq, "unit": "configurations/s",
                                       "sample": len(systems),
                                       "note": "every configuration of the batch solved one call each, at new "
                                               "positions, on its bucket's mesh"},
        "solve": {"worst_rel_residual": max(e.rel_residual for st in stats[-1] for e in st)},
        "gpu_launches": int(launches), "clocks": clk.summary(), "cpu_baseline": None,
    }


# ---------------------------------------------------------------------------
# Brownian-dynamics trajectory with three initial guesses (--workload trajectory)
# ---------------------------------------------------------------------------

TRAJ_WORKLOAD = ("trajectory: 8 polarizable spheres (642 beads each) + 20,000 monovalent ions, L=30, l_B=0.7, "
                 "bead radius 0.05, E0=z, mesh 192^3, tol 1e-6; step = mixed-precision solve to FP64 residual "
                 "1e-6 + forces/torques + one BD step (dt=1e-3, kT=1); initial guess: zero, the previous "
                 "step's charges, the learned warm start (trained first on method-generated solves of 2-8 "
                 "spheres and rods with 0-20,000 ions in random fields of magnitude 0.1-2), or the previous "
                 "step's charges plus the learned change; value = the learned warm start")
TRAJ_TRAIN_SOLVES = 1000


def bench_trajectory(args, ib, torch, rank, world, local):
    from paper_2401_04865_gb300 import warmstart as W
    from workloads import configs as C
    torch.cuda.set_device(local)
    s = C.config5_trajectory(seed=1004 + 7919 * rank)
    dev, f64 = "cuda", torch.float64
    t = lambda a, dt=f64: torch.as_tensor(np.ascontiguousarray(a)).to(dt).to(dev)
    stream = torch.cuda.current_stream()

    def make_ctx(prec):
        return ib.pme_setup(ib.make_params(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=s.a, eps_f=s.eps,
                                           precision=prec, max_rhs=1), stream)

    ctx = make_ctx(ib.IBPME_MIXED)
    n, nb = s.n, s.n_bodies
    off, Q, E0 = t(s.body_offsets, torch.int32), t(s.Q), t(s.E0[:1])
    x, X = t(s.x), t(s.X)
    xn, Xn = torch.empty_like(x), torch.empty_like(X)
    q = torch.zeros((1, n), dtype=f64, device=dev)
    fb = torch.zeros((n, 3), dtype=f64, device=dev)
    F = torch.zeros((nb, 3), dtype=f64, device=dev)
    L = torch.zeros((nb, 3), dtype=f64, device=dev)

    # training set: independent configurations of the trajectory's physics, solved from zero
    t0 = time.perf_counter()
    feat, targ, _ = W.collect(ib, ctx, (C.warm_start_training(50_000 + 10_007 * rank + k)
                                        for k in range(TRAJ_TRAIN_SOLVES)))
    t1 = time.perf_counter()
    mlp, loss = W.train(ib, feat, targ, seed=5, epochs=24)
    t2 = time.perf_counter()
    training = {"solves": TRAJ_TRAIN_SOLVES, "rows": int(feat.shape[0]), "final_loss": loss,
                "collect_s": t1 - t0, "train_s": t2 - t1, "epochs": 24}
    del feat, targ

    def run(c, guess, steps, warmup, precond=ib.IBPME_PRECOND_BODY, m=None):
        """steps BD steps from the trajectory's start (after warmup untimed ones):
        (ms per step, mean iterations, mean initial residual, worst final residual)."""
        xa, Xa, xb, Xb = x.clone(), X.clone(), xn, Xn
        q.zero_()
        its, init, worst = [], [], 0.0
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(warmup + steps):
            if guess == ib.IBPME_GUESS_ZERO:
                q.zero_()
            opts = ib.make_opts(rtol=1e-6, guess=guess, mlp=m, precond=precond)
            if i >= warmup:
                ev[i - warmup][0].record(stream)
            status, st = ib.ibpme_bd_advance(c, n, xa, ib.Bodies(off, Xa, Q), E0[0], opts, q[0], 1e-3, 1.0, 1.0,
                                             4321, i, F, L, xb, Xb, f_bead=fb)
            if i >= warmup:
                ev[i - warmup][1].record(stream)
                its.append(st.iters)
                init.append(st.init_rel_residual)
                worst = max(worst, st.rel_residual)
            if status != ib.IBPME_OK:
                raise RuntimeError("trajectory solve did not converge")
            xa, xb, Xa, Xb = xb, xa, Xb, Xa
        torch.cuda.synchronize()
        ms = float(np.sum([a.elapsed_time(b) for a, b in ev])) / steps
        return {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "iters_mean": float(np.mean(its)),
                "init_rel_residual_mean": float(np.mean(init)), "worst_rel_residual": worst, "steps": steps}

    modes = {}
    for name, guess in (("zero", ib.IBPME_GUESS_ZERO), ("previous", ib.IBPME_GUESS_USER),
                        ("learned", ib.IBPME_GUESS_LEARNED), ("learned_step", ib.IBPME_GUESS_LEARNED_STEP)):
        modes[name] = run(ctx, guess, args.steps, args.warmup, m=mlp)
    ib.ibpme_mlp_destroy(mlp)
    ib.pme_destroy(ctx)
    # FP64 comparators on the same trajectory: the same algorithm in FP64 (body-block
    # preconditioner, zero guess) and the plain FP64 solve (zero guess, no preconditioner)
    ctx64 = make_ctx(ib.IBPME_FP64)
    k64 = max(3, min(args.steps, 50))
    fp64_same = run(ctx64, ib.IBPME_GUESS_ZERO, k64, 1)
    kplain = max(3, min(args.steps, 10))
    fp64_plain = run(ctx64, ib.IBPME_GUESS_ZERO, kplain, 1, precond=ib.IBPME_PRECOND_NONE)
    ib.pme_destroy(ctx64)
    best = modes["learned"]
    return {
        "metric": "BD steps/s (induced-charge solve + forces + BD step)", "value": world * best["steps_per_s"],
        "unit": "steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": best["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 mesh / f64 krylov", "data": "synthetic",
        "config": {"workload": TRAJ_WORKLOAD, "n_beads": n, "mesh": list(s.mesh),
                   "l2": "inputs resident; positions advance every step",
                   "parallelism": f"replicas x{world} (independent trajectories, no collective)"},
        "guess_modes": modes, "fp64_same_algorithm": fp64_same, "fp64_plain": fp64_plain,
        "speedup_vs_fp64_plain": best["steps_per_s"] / fp64_plain["steps_per_s"],
        "speedup_vs_fp64_same_algorithm": best["steps_per_s"] / fp64_same["steps_per_s"],
        "learned_vs_zero": best["steps_per_s"] / modes["zero"]["steps_per_s"],
        "learned_step_vs_zero": modes["learned_step"]["steps_per_s"] / modes["zero"]["steps_per_s"],
        "previous_vs_zero": modes["previous"]["steps_per_s"] / modes["zero"]["steps_per_s"],
        "speedup_definition": ("steps/s of the learned-guess mixed-precision trajectory over steps/s of the same "
                               "trajectory solved in FP64 from the zero guess, without preconditioner (plain) or "
                               "with the body-block preconditioner (same algorithm); every solve to FP64 residual "
                               "1e-6"),
        "training": training, "cpu_baseline": None,
    }


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_step(o, s, x, X):
    """One step of the charged-sphere workload with the FP64 oracle: dense saddle
    solve, Ewald forces and torques, energy, hard-sphere forces and the BD step."""
    q, psi = o.solve_dense(x, s.body_offsets, X, s.Q, s.E0[0], s.box, s.a, s.eps)
    S = o.dipoles(x, X, s.body_offsets, q, s.box)
    o.energy(X, s.Q, psi, S, s.E0[0])
    f = o.bead_forces(x, q, s.E0[0], s.box, s.a, s.eps)
    o.body_force_torque(x, X, s.body_offsets, f, s.box)
    f = f + o.hard_sphere_forces(x, s.body_offsets, s.box, s.a, 1.0, DT)
    return o.bd_step(x, X, s.body_offsets, f, s.box, s.a, DT, seed=1234, step=0)


def oracle_eval_seconds(o, s, q, m, seed):
    """Seconds of one oracle evaluation (explicit Ewald sums, every source) at m
    seeded random targets."""
    t = np.random.default_rng(seed).choice(s.n, size=m, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    o.potential(s.x, q, s.box, s.a, s.eps, targets=t, xi=0.5)
    return time.perf_counter() - t0


def lattice_oracle_rate(samples, n, matvecs):
    """Solves/s of the oracle on the lattice from timed evaluations at few targets:
    the evaluation time is fixed (structure factors of all sources) plus linear in the
    targets, fitted on the samples and extrapolated to all n targets; one solve takes
    matvecs such evaluations plus one for the forces (a lower bound on its time: the
    field costs more than the potential, the BD step is left out)."""
    m = np.array([a for a, _ in samples], dtype=np.float64)
    t = np.array([b for _, b in samples], dtype=np.float64)
    b, a = np.polyfit(m, t, 1) if len(set(m.tolist())) > 1 else (t.mean() / m.mean(), 0.0)
    b = max(b, 0.0)
    t_full = max(a, 0.0) + b * n
    return 1.0 / ((matvecs + 1) * t_full), t_full


def cpu_baseline(workload, matvecs=None, min_seconds=10.0, max_steps=4):
    import oracle as o
    if workload == "lattice":
        s = make_system("lattice", 0)
        q = np.random.default_rng(3).normal(size=s.n)
        mv = matvecs if matvecs is not None else ORACLE_MATVECS_LATTICE
        t0 = time.perf_counter()
        samples = [(m, oracle_eval_seconds(o, s, q, m, 10 + i)) for i, m in enumerate((8, 192))]
        dt = time.perf_counter() - t0
        v, t_full = lattice_oracle_rate(samples, s.n, mv)
        return {"value": v, "unit": "solves/s", "cores": o.num_threads(), "kind": "oracle",
                "sample": f"oracle evaluations (explicit Ewald sums over all 141,088 sources) at 8 and 192 random "
                          f"targets in {dt:.1f} s, fitted as fixed + per-target time and extrapolated to one full "
                          f"evaluation ({t_full:.0f} s); one solve = {mv} + 1 evaluations (extrapolated)"}
    s = make_system("charged-sphere", 0)
    x, X = s.x, s.X
    t0 = time.perf_counter()
    k = 0
    while k < max_steps and (k == 0 or time.perf_counter() - t0 < min_seconds):
        x, X = oracle_step(o, s, x, X)
        k += 1
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "solves/s", "cores": o.num_threads(), "kind": "oracle",
            "sample": f"{k} full step(s) of the same workload (dense LU saddle solve, explicit-k Ewald forces, "
                      f"hard spheres, BD step) in {dt:.1f} s"}


def bench_reference(args):
    import oracle as o
    wl = args.workload if args.workload in ("lattice", "charged-sphere") else "lattice"
    s = make_system(wl, 0)
    if wl == "lattice":
        # each step: one oracle evaluation at a bounded number of targets (alternately 8
        # and 192), every source included; the rate is extrapolated from them
        q = np.random.default_rng(3).normal(size=s.n)
        for i in range(args.warmup):
            oracle_eval_seconds(o, s, q, 8, 100 + i)
        samples = []
        t0 = time.perf_counter()
        for i in range(args.steps):
            m = 8 if i % 2 == 0 else 192
            samples.append((m, oracle_eval_seconds(o, s, q, m, 200 + i)))
        dt = time.perf_counter() - t0
        v, t_full = lattice_oracle_rate(samples, s.n, ORACLE_MATVECS_LATTICE)
        sample = (f"{args.steps} timed oracle evaluations at 8 or 192 random targets (all 141,088 sources) after "
                  f"{args.warmup} warm-up ones, fitted as fixed + per-target time, extrapolated to one full "
                  f"evaluation ({t_full:.0f} s); one solve = {ORACLE_MATVECS_LATTICE} + 1 evaluations")
        ms = 1e3 / v
    else:
        x, X = s.x, s.X
        for _ in range(args.warmup):
            x, X = oracle_step(o, s, x, X)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            x, X = oracle_step(o, s, x, X)
        dt = time.perf_counter() - t0
        v = args.steps / dt
        ms = dt / args.steps * 1e3
        sample = f"{args.steps} timed full steps after {args.warmup} warm-up steps"
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": LATTICE if wl == "lattice" else SPHERE},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": o.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--skip-fp64", action="store_true", help="do not time the FP64 paths")
    ap.add_argument("--skip-cpu", action="store_true", help="do not time the oracle on the host")
    ap.add_argument("--skip-scale", action="store_true",
                    help="charged-sphere workload: do not time the PME evaluation on the lattice")
    ap.add_argument("--skip-second", action="store_true",
                    help="lattice workload: do not time the charged-sphere workload beside it")
    ap.add_argument("--workload", default="lattice",
                    choices=["lattice", "charged-sphere", "polarizability", "trajectory", "rpy"],
                    help="the headline lattice step, the charged-sphere step, the batched polarizability "
                         "solve, or a BD trajectory comparing initial guesses")
    ap.add_argument("--bucket-ratio", type=float, default=1.6,
                    help="polarizability: largest / smallest bead count within one batched call")
    ap.add_argument("--configs", type=int, default=64,
                    help="configurations in the polarizability batch (64 = the full workload)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local = dist_env()
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(bench_reference(args)), flush=True)
        return
    import torch

    import paper_2401_04865_gb300 as ib
    ib.load()
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload in ("polarizability", "trajectory", "rpy"):
        fn = {"polarizability": bench_polarizability, "trajectory": bench_trajectory, "rpy": bench_rpy}[args.workload]
        out = fn(args, ib, torch, rank, world, local)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    out, s = bench_ours(args, ib, torch, rank, world, local)
    if rank == 0:
        mv = None
        if out.get("fp64_gpu") and "fp64_plain" in out["fp64_gpu"]:
            mv = out["fp64_gpu"]["fp64_plain"]["iters"] + 2
        out["cpu_baseline"] = None if args.skip_cpu else cpu_baseline(args.workload, mv)
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
