#!/usr/bin/env python
"""Implicit-step benchmark: one BDF2 time step of the compressible Navier-Stokes
equations with the matrix-free modal DG discretisation, solved by Newton with
p-multigrid preconditioned FGMRES, on the Taylor-Green vortex workload
(16^3 hexes, p = 4, pMG 4-2-1-0, FGMRES(30) tol 1e-5).

A step = preconditioner update at W^n (lagged for the step) + `--newton`
Newton iterations, each: BDF2 right-hand side, FGMRES solve, state update.
Every step starts from the same (W^n, W^{n-1}) so every step does the same
work.  Metric: implicit-step DOFs/s = DOFs x steps / time.

Prints one JSON line (rank 0).  `--impl reference` times the plain CPU oracle
(test infrastructure) on a bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1812_04789_gb300 import workloads as wl  # noqa: E402

BJ_KERNEL_VERSION = "colmajor-v1"   # bump when the block-Jacobi apply kernel changes
COOP_KERNEL_VERSION = "coop-fp32-3bar"   # bump when the persistent smoother kernel changes
METRIC = "Implicit-step DOFs/s (mixed vs FP64, 1 GB300); JVP % HBM roofline; p99 latency"
UNIT = "DOFs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="tgv16_p4")
    ap.add_argument("--newton", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-esdirk", action="store_true")
    ap.add_argument("--no-bilu", action="store_true")
    ap.add_argument("--no-triangles", action="store_true")
    ap.add_argument("--no-qspace", action="store_true")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-large-dt", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--c3-fp64", type=int, default=1, help="FP64 steps of the 32^3 p=6 case (0: skip)")
    # profiling mode: one library operation a few times (ncu launch lists and captures)
    ap.add_argument("--profile-op", default=None,
                    choices=["jvp64", "residual64", "bj", "apply", "refresh", "fgmres", "step"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--n", type=int, nargs="*", default=None, help="override the mesh size (--profile-op)")
    ap.add_argument("--bf16", action="store_true", help="BF16 block storage (--profile-op)")
    return ap.parse_args()


def bench_opts(cfg):
    nl = len(cfg["p_levels"])
    return dict(p_levels=cfg["p_levels"], nu_pre=10, nu_post=10, nu_coarse=30,
                cycle=0 if nl > 1 else 2)


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- GPU arm
class Stepper:
    """One BDF2 implicit step on the device through the library's C ABI."""

    def __init__(self, B, torch, cfg, precision, stream, W0, Wm1, coarse=0, order=0, storage=0):
        self.B, self.torch = B, torch
        self.cfg = cfg
        self.stream = stream
        desc, phys = wl.mesh_desc(cfg), wl.physics(cfg)
        self.mesh = B.Mesh.from_workload(desc, phys, stream=stream)
        self.dt = wl.time_step(cfg)
        self.sigma = 1.5 / self.dt
        o = bench_opts(cfg)
        self.opts = B.pmg_opts(o["p_levels"], nu_pre=o["nu_pre"], nu_post=o["nu_post"],
                               nu_coarse=o["nu_coarse"], cycle=o["cycle"], precision=precision,
                               coarse=coarse, order=order, storage=storage)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.W0 = torch.from_numpy(W0).to(dev)
        self.Wm1 = torch.from_numpy(Wm1).to(dev)
        self.Wn = torch.empty_like(self.W0)
        self.Wnm1 = torch.empty_like(self.W0)
        self.Wk = torch.empty_like(self.W0)
        self.b = torch.empty_like(self.W0)
        self.dW = torch.empty_like(self.W0)
        self.pmg = B.PMG(self.mesh, self.W0, self.sigma, self.opts, stream=stream)
        self.iters = []
        self.ndofs = self.mesh.ndofs

    def step(self, newton):
        s = self.stream
        self.Wn.copy_(self.W0)
        self.Wnm1.copy_(self.Wm1)
        self.pmg.refresh(self.Wn, self.sigma, stream=s)
        self.Wk.copy_(self.Wn)
        its = 0
        for _ in range(newton):
            self.mesh.bdf2_rhs(self.Wk, self.Wn, self.Wnm1, self.dt, self.b, stream=s)
            st = self.pmg.fgmres(self.Wk, self.b, self.dW, rtol=1e-5, max_restarts=4, stream=s)
            its += st["iters"]
            self.mesh.axpy(1.0, self.dW, self.Wk, stream=s)
        self.iters.append(its / newton)
        return self.Wk


# ---------------------------------------------------------------- ranks
def dist_on():
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def dist_barrier():
    """Barrier across the ranks of a torchrun launch (no-op for one process)."""
    if dist_on():
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, device):
    """The largest of every rank's value (each rank's timed seconds)."""
    if not dist_on():
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, steps, seconds):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank * steps / seconds


def timed_steps(torch, stepper, steps, warmup, newton, stream, flush):
    for _ in range(warmup):
        stepper.step(newton)
    torch.cuda.synchronize()
    dist_barrier()                          # every rank starts the timed steps together
    times = []
    stepper.iters.clear()
    for _ in range(steps):
        flush.zero_()                       # evict L2 between timed steps (129 MB L2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stepper.step(newton)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    dist_barrier()
    return times


def esdirk3_steps(torch, B, stepper, steps, newton, stream, flush):
    """The paper's own time scheme on the same case: ESDIRK3 steps (three
    implicit stages, `newton` Newton iterations each, preconditioner refreshed
    once per step) through dg_esdirk3_step, on the headline handle's mesh and
    preconditioner.  Device time per step and DOFs/s."""
    dt = stepper.dt
    Wout = torch.empty_like(stepper.W0)
    work = torch.empty(6 * stepper.W0.numel(), dtype=torch.float64, device=stepper.W0.device)
    its = []
    stepper.pmg.esdirk3_step(stepper.W0, dt, Wout, newton=newton, max_restarts=4, work=work, stream=stream)
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = stepper.pmg.esdirk3_step(stepper.W0, dt, Wout, newton=newton, max_restarts=4, work=work,
                                      stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        its.append(st["iters"] / (3.0 * newton))
    ms = statistics.mean(times)
    return {"ms_per_step": ms, "value": stepper.ndofs / (ms * 1e-3), "unit": UNIT,
            "fgmres_iters_per_solve": statistics.mean(its), "steps": steps,
            "scheme": "ESDIRK3 (4 stages, 3 implicit), %d Newton per stage, mixed-precision pMG lagged "
                      "over the step" % newton}


def coarse_bilu_steps(torch, B, cfg, stream, W0, Wm1, newton, flush):
    """The coarsest smoother preconditioned by element block ILU(0) (Table
    MGSettings) instead of block Jacobi, mixed precision, on the headline case:
    one BDF2 step per element order after one warm-up step (device time,
    FGMRES iterations per solve, substitution levels), and one pMG application."""
    out = {}
    r = torch.from_numpy(wl.random_vector(W0.shape, 41)).cuda()
    z = torch.empty_like(r)
    for name, coarse, order in (("bj", B.COARSE_BJ, 0), ("natural", B.COARSE_BILU, B.ORDER_NATURAL),
                                ("colour", B.COARSE_BILU, B.ORDER_COLOUR), ("mdf", B.COARSE_BILU, B.ORDER_MDF)):
        st = Stepper(B, torch, cfg, B.PREC_MIXED, stream, W0, Wm1, coarse=coarse, order=order)
        times = timed_steps(torch, st, 1, 1, newton, stream, flush)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.pmg.apply(r, z, stream=stream)
        e1.record(stream)
        e1.synchronize()
        out[name] = {"ms_per_step": times[0], "fgmres_iters_per_solve": statistics.mean(st.iters),
                     "pmg_apply_ms": e0.elapsed_time(e1),
                     "levels": st.pmg.bilu_order(stream=stream)[1] if coarse == B.COARSE_BILU else None}
        st.pmg.close()
        st.mesh.close()
    return out


def triangle_steps(torch, B, stream, newton, flush, steps=2):
    """The vortex on a periodic triangulation (32 x 32 jittered quads cut into
    2048 triangles, full-order P_4, the paper's triangular grids of Sec. 7.2):
    BDF2 steps through the triangle mesh handle, mixed-precision pMG 4-2-1-0,
    after one warm-up step.  Device time per step, DOFs/s, FGMRES iterations."""
    cfg = wl.tri_config((32, 32), 4, p_levels=(4, 2, 1, 0), dt_conv=0.05)
    try:
        mesh = B.Mesh.from_tri_workload(wl.tri_mesh(cfg), wl.tri_physics(cfg), cfg["p"], stream=stream)
        dt = wl.time_step(cfg)
        sigma = 1.5 / dt
        W0 = torch.from_numpy(wl.tri_initial_state(cfg)).cuda()
        Wm1 = torch.from_numpy(wl.tri_initial_state(cfg, t=-dt)).cuda()
        pmg = B.PMG(mesh, W0, sigma, B.pmg_opts(cfg["p_levels"], nu_pre=10, nu_post=10, nu_coarse=30,
                                                 precision=B.PREC_MIXED), stream=stream)
        Wk, b, dW = torch.empty_like(W0), torch.empty_like(W0), torch.empty_like(W0)
        times, its = [], []
        for k in range(steps + 1):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pmg.refresh(W0, sigma, stream=stream)
            Wk.copy_(W0)
            n_it = 0
            for _ in range(newton):
                mesh.bdf2_rhs(Wk, W0, Wm1, dt, b, stream=stream)
                st = pmg.fgmres(Wk, b, dW, rtol=1e-5, max_restarts=4, stream=stream)
                n_it += st["iters"]
                mesh.axpy(1.0, dW, Wk, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if k > 0:
                times.append(e0.elapsed_time(e1))
                its.append(n_it / newton)
        ms = statistics.mean(times)
        out = {"ms_per_step": ms, "value": mesh.ndofs / (ms * 1e-3), "unit": UNIT, "dofs": mesh.ndofs,
               "fgmres_iters_per_solve": statistics.mean(its), "steps": steps,
               "workload": "vortex on 2048 jittered periodic triangles, P_4 (Dubiner), BDF2 dt 0.05 t_c, "
                           "mixed pMG 4-2-1-0 nu 10/10/30, %d Newton/step" % newton}
        pmg.close()
        mesh.close()
        return out
    except Exception as exc:                 # reported in the JSON line, the headline stands
        return {"error": "%s: %s" % (type(exc).__name__, exc)}


def q_space_jvp(torch, B, stream, n=10):
    """The exact JVP on the tensor-product space Q_4 (TGV 16^3 hexes, 125 modes
    per variable): the volume term runs by sum factorisation.  Mean device time
    of n back-to-back FP64 and FP32 JVPs after three untimed ones, with the
    P_4 JVP of the same mesh beside it (35 modes, direct contractions)."""
    out = {}
    try:
        for space in ("Q", "P"):
            cfg = wl.make_config("tgv", 3, (16, 16, 16), 4, M=0.1, Re=1600.0, space=space)
            mesh = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg), stream=stream)
            W = torch.from_numpy(wl.perturbed_state(cfg)).cuda()
            v = torch.from_numpy(wl.random_vector(W.shape)).cuda()
            Kv = torch.empty_like(W)
            rec = {"dofs": mesh.ndofs}
            for name, mode in (("fp64_ms", B.JVP_EXACT), ("fp32_ms", B.JVP_EXACT_FP32)):
                for _ in range(3):
                    mesh.jvp(W, v, Kv, 100.0, mode=mode, stream=stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(n):
                    mesh.jvp(W, v, Kv, 100.0, mode=mode, stream=stream)
                e1.record(stream)
                e1.synchronize()
                rec[name] = e0.elapsed_time(e1) / n
            out[space] = rec
            mesh.close()
        return out
    except Exception as exc:                 # reported in the JSON line, the headline stands
        return {"error": "%s: %s" % (type(exc).__name__, exc)}


def variant_steps(torch, B, cfg, stream, newton, flush, runs, W0=None, Wm1=None, ref_final=None):
    """One workload in several preconditioner variants: for each (name,
    precision, storage, warm-up, timed steps) in `runs`, BDF2 steps from the same
    (W^n, W^{n-1}) on a fresh handle; device time per step, DOFs/s, FGMRES
    iterations per solve, and W^{n+1} against the FP64 variant when present
    (relative L2 of W^{n+1} and of the step dW).  A failing variant is reported
    as such and the others stand."""
    if W0 is None:
        W0 = wl.initial_state(cfg)
        Wm1 = wl.initial_state(cfg, t=-wl.time_step(cfg)) if cfg["case"] == "vortex" else W0
    out, finals = {}, {}
    for name, prec, storage, warm, steps in runs:
        st = None
        try:
            st = Stepper(B, torch, cfg, prec, stream, W0, Wm1, storage=storage)
            times = timed_steps(torch, st, steps, warm, newton, stream, flush)
            ms = statistics.mean(times)
            out[name] = {"ms_per_step": ms, "value": st.ndofs / (ms * 1e-3), "unit": UNIT,
                         "fgmres_iters_per_solve": statistics.mean(st.iters), "steps": steps,
                         "warmup": warm}
            finals[name] = st.Wk.cpu().numpy()
        except Exception as exc:
            out[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}
        finally:
            if st is not None:
                st.pmg.close()
                st.mesh.close()
            torch.cuda.empty_cache()
    ref = finals.get("fp64", ref_final)
    if ref is not None:
        for name, W in finals.items():
            if name != "fp64":
                out[name]["vs_fp64_rel_l2"] = float(np.linalg.norm(W - ref) / np.linalg.norm(ref))
                out[name]["vs_fp64_dW_rel_l2"] = float(np.linalg.norm(W - ref) / max(np.linalg.norm(ref - W0), 1e-300))
    out["dofs"] = int(W0.size)
    out["workload"] = "TGV %dx%dx%d hex, p=%d, Re=%g, M=%g, BDF2 dt=%g t_c, pMG %s FMG nu=10/10/30, " \
                      "FGMRES(30) rtol 1e-5, %d Newton/step" % (*cfg["n"], cfg["p"], cfg["Re"], cfg["M"],
                                                                cfg["dt_conv"], "-".join(map(str, cfg["p_levels"])),
                                                                newton)
    return out


def kernel_roofline(torch, B, stepper, stream, peaks):
    """Average duration of the fine-level block-Jacobi apply (the HBM-bound
    kernel that streams every inverse diagonal block once) and of the FP64 JVP
    (FP64-ALU bound), each timed alone with CUDA events on the library's stream."""
    mesh = stepper.mesh
    E, nb = mesh.E, mesh.m * mesh.nm
    out = {}
    r = torch.randn_like(stepper.W0)
    z = torch.empty_like(r)
    n = 20
    # block-Jacobi apply through a BJ-only handle of the same precision as the headline
    o = B.pmg_opts((stepper.cfg["p"],), cycle=B.CYCLE_BJ, precision=stepper.opts.precision)
    bj = B.PMG(mesh, stepper.W0, stepper.sigma, o, stream=stream)
    for _ in range(3):
        bj.apply(r, z, stream=stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        bj.apply(r, z, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n
    es = 4 if stepper.opts.precision == B.PREC_MIXED else 8
    # algorithmic bytes: inverse blocks + r in + z out (+ the precision conversions of r, z)
    blk = E * nb * nb * es
    vec = E * nb * (es * 2 + (8 + es) * 2 if es == 4 else es * 2)
    out["bj_apply"] = dict(ms=ms, bytes=blk + vec, gbs=(blk + vec) / (ms * 1e-3) / 1e9)
    bj.close()
    # FP64 exact JVP (face + volume kernels)
    Kv = torch.empty_like(r)
    for _ in range(3):
        mesh.jvp(stepper.W0, r, Kv, stepper.sigma, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n):
        mesh.jvp(stepper.W0, r, Kv, stepper.sigma, stream=stream)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / n
    jb = E * nb * 8 * 3                      # read W and v, write Kv (FP64)
    out["jvp_fp64"] = dict(ms=ms, bytes=jb, gbs=jb / (ms * 1e-3) / 1e9,
                           hbm_frac=jb / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"])
    # tensor-core block probe of the fine diagonal blocks: exporting the
    # un-inverted level-0 blocks reruns exactly that kernel (no neighbour
    # blocks are requested and no direction has a single element)
    if stepper.opts.precision == B.PREC_MIXED and min(stepper.cfg["n"]) > 1:
        D = torch.empty((E, nb, nb), dtype=torch.float32, device=r.device)
        stepper.pmg.export_blocks(0, B.BLOCKS_DIAG, D, stream=stream)
        ts = []
        for _ in range(3):
            e0.record(stream)
            stepper.pmg.export_blocks(0, B.BLOCKS_DIAG, D, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.median(ts)
        d, nm = len(stepper.cfg["n"]), mesh.nm
        nq1 = stepper.cfg["p"] + 2
        # the dense contraction D[(w,v,i'), i] += Z[(w,v,i'), K] Trial[i, K], one pass,
        # K = (volume points + own-face points) x (1 + d)
        K = (nq1 ** d + 2 * d * nq1 ** (d - 1)) * (1 + d)
        flops = 2.0 * E * (mesh.m * mesh.m * nm) * nm * K
        tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25     # nominal dense TF32 / BF16 ratio
        out["probe_tc"] = dict(ms=ms, flops=flops, tflops=flops / (ms * 1e-3) / 1e12, peak_tflops=tf32_peak,
                               frac=flops / (ms * 1e-3) / 1e12 / tf32_peak,
                               peak_source="measured bf16 burst x nominal TF32/BF16 ratio 1.1/2.25")
        del D
    return out


# Peaks for the ALU-bound kernels, from the unit counts and the maximum SM
# clock (the measured peaks cover HBM and the BF16 tensor pipe only):
# FP32: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz; FP64: GB300's
# nominal 1.25 TFLOP/s (152 SMs x 2 DFMA lanes x 2 flop x 2.07 GHz = 1.26).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def kernel_rooflines(torch, B, mixed, fp64, stream, peaks, ref_cfg):
    """Rooflines of the kernels that own the implicit step, each timed alone
    with dg_pmg_kernel_time (CUDA events on the library's stream, 10 launches
    after the handle's own set-up).  Work per launch:
      * ALU-bound JVP kernels: the floating-point operations the kernel executes
        per element, counted by ncu (FADD/FMUL 1, FFMA 2, paired ops twice;
        profiles/kernel_work.json, from one capture of each kernel) times E;
        traffic: DRAM bytes per element of the same capture times E;
      * HBM-bound kernels: the algorithmic bytes (blocks streamed once per
        product, vectors read or written once).
    Returns a list, the kernels ordered by the share of the step that the
    launch list of a step gives them (profiles/)."""
    work = {}
    wf = os.path.join(ROOT, "profiles", "kernel_work.json")
    if os.path.exists(wf):
        work = json.load(open(wf))
    E, nb = mixed.mesh.E, mixed.mesh.m * mixed.mesh.nm
    out = []

    def alu(name, handle, kt, key, peak, dtype):
        ms = handle.pmg.kernel_time(kt, 0, 10, stream=stream)
        rec = work.get(key, {})
        same = rec.get("config") == ref_cfg
        fl = rec.get("flops_per_element")
        tr = rec.get("dram_bytes_per_element")
        ach = fl * E / (ms * 1e-3) / 1e12 if (fl and same) else None
        out.append({"kernel": name, "bound": "alu", "dtype": dtype, "achieved": ach, "peak": peak,
                    "unit": "TFLOP/s", "frac": ach / peak if ach else None,
                    "traffic": int(tr * E) if (tr and same) else None, "ms": ms,
                    "flops": fl * E if (fl and same) else None,
                    "peak_source": "nominal: unit counts x 2.07 GHz max SM clock",
                    "work_source": "executed FP ops per element (ncu, profiles/kernel_work.json)"})

    alu("face_kernel<3,float,1> (smoother JVP, faces; FP32 with cached traces)", mixed, B.KT_FACE_JVP,
        "face_jvp_fp32", FP32_PEAK_TFLOPS, "f32")
    alu("volume_kernel_st<3,1,3> (smoother JVP, volume; FP32, tables in shared memory)", mixed, B.KT_VOLUME_JVP,
        "volume_jvp_fp32", FP32_PEAK_TFLOPS, "f32")
    if fp64 is not None:
        alu("face_sf_kernel<double,1> (outer JVP, faces by sum factorisation; FP64)", fp64, B.KT_FACE_JVP, "face_jvp_fp64",
            FP64_PEAK_TFLOPS, "f64")
        alu("volume_q_kernel<3,double,1> (outer JVP, volume by sum factorisation; FP64)", fp64, B.KT_VOLUME_JVP, "volume_jvp_fp64",
            FP64_PEAK_TFLOPS, "f64")
    # block-Jacobi apply of the fine level (FP32 inverses, column-major, padded rows)
    ld = (nb + 3) // 4 * 4
    ms = mixed.pmg.kernel_time(B.KT_BLOCK_JACOBI, 0, 20, stream=stream)
    by = E * (nb * ld * 4 + 2 * nb * 4)
    out.append({"kernel": "bj_colmajor_kernel<float> (fine block-Jacobi apply)", "bound": "hbm", "dtype": "f32",
                "achieved": by / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": by / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": None, "ms": ms,
                "algorithmic_bytes": by})
    # persistent smoother of level 1 (p = 2): its HBM traffic is the inherited
    # blocks (diagonal + 2d neighbours) of every product and the inverse
    # diagonal blocks of every block-Jacobi apply; the Krylov basis stays on chip
    nl = len(mixed.cfg["p_levels"])
    if nl > 1:
        p1 = mixed.cfg["p_levels"][1]
        nb1 = mixed.mesh.m * wl.n_modes(p1, len(mixed.cfg["n"]))
        ld1 = (nb1 + 3) // 4 * 4
        nu = 10 if nl > 2 else 30
        ms = mixed.pmg.kernel_time(B.KT_SMOOTH, 1, 5, stream=stream)
        nf = 2 * len(mixed.cfg["n"])
        by = E * nb1 * ld1 * 4 * ((nu + 1) * (1 + nf) + nu) + E * nb1 * 4 * (4 + 2 * nu)
        # DRAM bytes of one such call from a committed ncu capture of the same
        # configuration and kernel version (profiles/roofline_traffic.json)
        traffic = None
        tf = os.path.join(ROOT, "profiles", "roofline_traffic.json")
        if os.path.exists(tf):
            rec = json.load(open(tf)).get("coop_level1_mixed", {})
            if rec.get("config") == ref_cfg and rec.get("kernel_version") == COOP_KERNEL_VERSION:
                traffic = rec.get("dram_bytes_per_launch")
        out.append({"kernel": "coop_smooth_kernel<float,6> (one smoother call, level 1, %d iterations)" % nu,
                    "bound": "hbm", "dtype": "f32", "achieved": by / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": by / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": traffic,
                    "ms": ms, "algorithmic_bytes": by})
    return out


def dominant_roofline(roofs):
    """The roofline entry of the kernel with the largest share of a mixed step:
    the share each kernel has in the committed launch list of one step
    (profiles/step_shares.json, from ncu gpu__time_duration of every launch)."""
    shares = {}
    sf = os.path.join(ROOT, "profiles", "step_shares.json")
    if os.path.exists(sf):
        shares = json.load(open(sf)).get("shares", {})
    best, best_share = None, -1.0
    for r in roofs:
        key = r["kernel"].split(" ")[0]
        sh = shares.get(key, 0.0)
        r["share_of_step"] = sh
        if sh > best_share:
            best, best_share = r, sh
    return dict(best) if best else None


def batched_sample(B, count=64, workers=8, budget=120 << 30):
    """The batched workload: `count` independent TGV cases from the seed
    (n 8..24, p 1..5, M and Re drawn, each one implicit BDF2 step in mixed
    precision, pMG down to p = 0), all submitted at once to the serving runtime
    (`workers` concurrent slots, each with its own stream).  Reports the wall
    time from first submission to last result and the aggregate DOFs/s."""
    cases = wl.batch_cases(count)
    inputs = []
    for cfg in cases:
        W0 = wl.initial_state(cfg)
        pl = cfg["p_levels"]
        opts = B.pmg_opts(pl, nu_pre=10, nu_post=10, nu_coarse=30,
                          cycle=B.CYCLE_FMG if len(pl) > 1 else B.CYCLE_BJ, precision=B.PREC_MIXED)
        inputs.append((cfg, opts, W0, np.zeros_like(W0)))
    dofs = sum(int(W0.size) for _, _, W0, _ in inputs)
    srv = B.Server(budget, workers)
    try:
        t0 = time.perf_counter()
        for i, (cfg, opts, W0, out) in enumerate(inputs):
            srv.submit(i, wl.mesh_desc(cfg), wl.physics(cfg), opts, W0, W0, wl.time_step(cfg), out)
        got = []
        while len(got) < count:
            got += srv.poll(1, timeout_ms=600000)
        sec = time.perf_counter() - t0
    finally:
        srv.close()
    ok = sum(1 for r in got if r["status"] == 0)
    lat = sorted(r["latency_ms"] for r in got)
    return {"cases": count, "ok": ok, "workers": workers, "dofs": dofs, "seconds": sec,
            "value": dofs / sec, "unit": UNIT, "p50_ms": lat[len(lat) // 2],
            "sample": "64 seeded TGV cases (n 8..24, p 1..5), one mixed-precision BDF2 step each, "
                      "submitted at once; wall time includes per-case mesh and preconditioner setup"}


def serving_sample(B, count=32, max_dofs=1000000, workers=4, budget=80 << 30, loads=(0.25, 0.5, 1.0, 2.0, 4.0),
                   seed=1812):
    """Serving workload (the request mix of wl.serving_requests: 2-D vortex
    32^2-256^2 / 3-D TGV 8^3-32^3, p 1..6, FP64 or mixed, one implicit step
    each), redrawn above max_dofs so that the sweep ends in minutes: the
    largest cases of the mix (up to 13.8 M DOFs; one FP64 step of TGV 32^3
    p = 6 takes about 84 s) would hold the GPU for the whole run.  Pass 0 runs
    one list at full concurrency (service rate, resident slots); then, for
    every load factor, a fresh list of `count` requests arrives as a Poisson
    stream at load x the service rate.  Reports p50/p99 latency (submit to
    completion) and DOFs/s per load."""
    def inputs_for(s):
        out = []
        for cfg in wl.serving_requests(count, seed=s, max_dofs=max_dofs):
            W0 = wl.initial_state(cfg)
            dt = wl.time_step(cfg)
            Wm1 = wl.initial_state(cfg, t=-dt) if cfg["case"] == "vortex" else W0.copy()
            pl = cfg["p_levels"]
            opts = B.pmg_opts(pl, nu_pre=10, nu_post=10, nu_coarse=30,
                              cycle=B.CYCLE_FMG if len(pl) > 1 else B.CYCLE_BJ,
                              precision=B.PREC_MIXED if cfg["mixed"] else B.PREC_FP64)
            out.append((cfg, opts, W0, Wm1, dt, np.zeros_like(W0)))
        return out

    srv = B.Server(budget, workers)
    sweep = []
    try:
        first = inputs_for(seed)
        t0 = time.perf_counter()
        for i, (cfg, opts, W0, Wm1, dt, out) in enumerate(first):
            srv.submit(i, wl.mesh_desc(cfg), wl.physics(cfg), opts, W0, Wm1, dt, out)
        got = []
        while len(got) < count:
            got += srv.poll(1, timeout_ms=600000)
        rate = count / (time.perf_counter() - t0)
        rid = 1000
        for k, load in enumerate(loads):
            reqs = inputs_for(seed + 1 + k)
            rng = np.random.default_rng(seed + 100 + k)
            gaps = rng.exponential(1.0 / (load * rate), count)
            t0 = time.perf_counter()
            due = t0
            res = []
            for i, (cfg, opts, W0, Wm1, dt, out) in enumerate(reqs):
                due += gaps[i]
                while time.perf_counter() < due:
                    res += srv.poll(0, timeout_ms=1)
                srv.submit(rid, wl.mesh_desc(cfg), wl.physics(cfg), opts, W0, Wm1, dt, out)
                rid += 1
            while len(res) < count:
                res += srv.poll(1, timeout_ms=600000)
            span = time.perf_counter() - t0
            lat = sorted(r["latency_ms"] for r in res)
            sweep.append({"load": load, "requests": count, "ok": int(sum(r["status"] == 0 for r in res)),
                          "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                          "value": sum(c["dofs"] for c, *_ in reqs) / span, "unit": UNIT,
                          "fgmres_iters_mean": float(np.mean([r["fgmres_iters"] for r in res]))})
        st = srv.stats()
    finally:
        srv.close()
    one = next(x for x in sweep if x["load"] == 1.0)
    return {"requests": count, "ok": one["ok"], "workers": workers, "load": 1.0,
            "p50_ms": one["p50_ms"], "p99_ms": one["p99_ms"], "value": one["value"], "unit": UNIT,
            "service_rate_req_s": rate, "resident_slots": st["resident_slots"], "budget_bytes": budget,
            "sweep": sweep,
            "sample": "serving mix (2-D vortex 32^2-256^2 / 3-D TGV 8^3-32^3, p 1..6, FP64|mixed), draws above "
                      "%d DOFs redrawn (time bound: the largest FP64 requests take minutes); Poisson arrivals at "
                      "%s x the measured service rate, %d requests per load" % (max_dofs, list(loads), count)}


def cpu_baseline_sample(cfg, newton, time_budget=40.0):
    """The oracle, as it stands, on a bounded sample of the workload: the same
    TGV case on a 3^3 sub-mesh (same p, physics, dt, pMG levels, tolerances),
    one implicit step; DOFs/s of that sample."""
    from oracle.dg import residual, jvp as ojvp, Mesh as OMesh
    from oracle.physics import Physics
    from oracle import solvers
    sub = dict(cfg)
    d = cfg["dim"]
    sub["n"] = (3, 3, 3) if d == 3 else (3, 3, 1)
    # the sub-mesh keeps the element size (hence dt/h) of the full mesh; the
    # physics constants (mu, dt) are those of the full workload
    sub["hi"] = tuple(cfg["lo"][k] + 3 * (cfg["hi"][k] - cfg["lo"][k]) / cfg["n"][k] if k < d else cfg["hi"][k]
                      for k in range(3))
    desc, phys = wl.mesh_desc(sub), wl.physics(cfg)
    om = OMesh(desc["dim"], desc["n"], desc["lo"], desc["hi"], desc["p"], desc["nq1d"])
    ph = Physics(gamma=phys["gamma"], Pr=phys["Pr"], mu=phys["mu"], Rgas=phys["Rgas"], eta=phys["eta"],
                 roe_delta=phys["roe_delta"])
    W0 = wl.initial_state(sub)
    dt = wl.time_step(cfg)
    sigma = 1.5 / dt
    o = bench_opts(cfg)
    t0 = time.perf_counter()
    mg = solvers.pmg_setup(om, ph, W0, sigma, o["p_levels"], o["nu_pre"], o["nu_post"], o["nu_coarse"])
    Wk = W0.copy()
    its = 0
    for _ in range(newton):
        f = solvers.bdf2_rhs(om, residual(om, ph, Wk), Wk, W0, W0, dt)
        x, st = solvers.fgmres(lambda z: ojvp(om, ph, Wk, z, sigma), mg, -f, rtol=1e-5, max_restarts=4)
        its += st["iters"]
        Wk = Wk + x
        if time.perf_counter() - t0 > time_budget:
            break
    sec = time.perf_counter() - t0
    return dict(value=om.E * om.nb / sec, unit=UNIT, cores=os.cpu_count(), kind="oracle",
                sample="TGV p=%d on a 3^3 sub-mesh (%d DOFs, same element size, physics, dt, pMG levels), one "
                       "implicit step (%d Newton, %d FGMRES its), %.1f s; numpy BLAS threads default to all cores"
                       % (cfg["p"], om.E * om.nb, newton, its, sec), seconds=sec)


def run_gb300(args):
    import torch
    from paper_1812_04789_gb300 import binding as B
    from paper_1812_04789_gb300 import build as BLD
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        BLD.build()
    if world > 1:
        torch.distributed.barrier()
    B.load()
    cfg = wl.CONFIGS[args.config]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                                                          "fallback": True}
    stream = torch.cuda.Stream()
    W0 = wl.initial_state(cfg)
    Wm1 = wl.initial_state(cfg, t=-wl.time_step(cfg)) if cfg["case"] == "vortex" else W0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    results = {}
    steppers = {}
    with torch.cuda.stream(stream):
        clocks = Clocks(local)
        for name, prec, steps in (("mixed", B.PREC_MIXED, args.steps), ("fp64", B.PREC_FP64, args.fp64_steps)):
            if steps <= 0:
                continue
            st = Stepper(B, torch, cfg, prec, stream, W0, Wm1)
            steppers[name] = st
            if name == "mixed":
                clocks.start()
                l0 = B.launch_count()
            times = timed_steps(torch, st, steps, args.warmup if name == "mixed" else 1, args.newton, stream, flush)
            if name == "mixed":
                launches = B.launch_count() - l0
                clk = clocks.stop()
            tot = max_over_ranks(sum(times) / 1e3, "cuda")
            results[name] = dict(ms_per_step=1e3 * tot / steps, value=whole_job_rate(world, st.ndofs, steps, tot),
                                 fgmres_iters_per_solve=statistics.mean(st.iters), ndofs=st.ndofs,
                                 Wfinal=st.Wk.cpu().numpy() if name in ("mixed", "fp64") else None)
            if name == "mixed":
                head = st
        # mixed vs FP64 step error (same step, same inputs)
        err = err_dw = None
        if "fp64" in results and "mixed" in results:
            a, b = results["mixed"]["Wfinal"], results["fp64"]["Wfinal"]
            err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
            err_dw = float(np.linalg.norm(a - b) / max(np.linalg.norm(b - W0), 1e-300))
        roof = kernel_roofline(torch, B, head, stream, peaks)
        roofs = kernel_rooflines(torch, B, head, steppers.get("fp64"), stream, peaks, args.config)
        if "fp64" in steppers:
            steppers["fp64"].pmg.close()
            del steppers["fp64"]
            torch.cuda.empty_cache()
        # BF16 block storage on the headline case (same steps as the headline)
        bf16 = None
        if not args.no_bf16:
            bf16 = variant_steps(torch, B, cfg, stream, args.newton, flush,
                                 [("mixed_bf16", B.PREC_MIXED, B.STORE_BF16, 2, max(1, min(args.steps, 5)))],
                                 W0=W0, Wm1=Wm1, ref_final=results.get("fp64", {}).get("Wfinal"))["mixed_bf16"]
        # the headline case at a large time step (dt = 1 t_c, the paper's vortex runs at dt = 1):
        # the preconditioner has to work here, mixed vs FP64 iterations and states
        large = None
        if not args.no_large_dt:
            cl = dict(cfg)
            cl["dt_conv"] = 1.0
            large = variant_steps(torch, B, cl, stream, args.newton, flush,
                                  [("fp64", B.PREC_FP64, 0, 0, 1), ("mixed", B.PREC_MIXED, 0, 1, 2),
                                   ("mixed_bf16", B.PREC_MIXED, B.STORE_BF16, 1, 2)])
        # the stiff large case the mixed precision is meant for: TGV 32^3, p = 6, M = 0.05
        c3 = None
        if not args.no_c3:
            runs = [("mixed", B.PREC_MIXED, 0, 1, 1), ("mixed_bf16", B.PREC_MIXED, B.STORE_BF16, 1, 1)]
            if args.c3_fp64 > 0:
                runs.insert(0, ("fp64", B.PREC_FP64, 0, 0, args.c3_fp64))
            c3 = variant_steps(torch, B, wl.CONFIGS["tgv32_p6"], stream, args.newton, flush, runs)
            c3["note"] = "FP64 timed without a warm-up step (one step takes about a minute); mixed after one"
        esd = None if args.no_esdirk else esdirk3_steps(torch, B, head, max(1, min(args.steps, 3)), args.newton,
                                                        stream, flush)
        bilu = None if args.no_bilu else coarse_bilu_steps(torch, B, cfg, stream, W0, Wm1, args.newton, flush)
        tris = None if args.no_triangles else triangle_steps(torch, B, stream, args.newton, flush)
        qsp = None if args.no_qspace else q_space_jvp(torch, B, stream)
        # end to end through the public API with pinned host buffers
        e2e = None
        if not args.no_e2e:
            hW0 = torch.from_numpy(W0).pin_memory()
            hWm1 = torch.from_numpy(Wm1).pin_memory()
            hout = torch.empty_like(hW0).pin_memory()
            n = max(1, min(args.steps, 3))
            head.step(args.newton)          # untimed: puts the handle back on the BDF2 shift after ESDIRK3
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(n):
                head.W0.copy_(hW0, non_blocking=True)
                head.Wm1.copy_(hWm1, non_blocking=True)
                out = head.step(args.newton)
                hout.copy_(out, non_blocking=True)
                stream.synchronize()
            sec = time.perf_counter() - t0
            e2e = {"value": world * head.ndofs * n / sec, "unit": UNIT,
                   "h2d_bytes_per_step": int(hW0.numel() * 8 * 2), "d2h_bytes_per_step": int(hout.numel() * 8)}
    mixed = results["mixed"]
    bj = roof["bj_apply"]
    traffic = None
    tf = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if os.path.exists(tf):
        rec = json.load(open(tf)).get("bj_apply_mixed", {})
        if rec.get("config") == args.config and rec.get("kernel_version") == BJ_KERNEL_VERSION:
            traffic = rec.get("dram_bytes_per_launch")
    es = 4
    line = {
        "metric": METRIC, "value": mixed["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mixed["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32 (FP64 outer FGMRES/JVP, FP32 pMG)",
        "data": "synthetic (closed-form Taylor-Green initial state, L2-projected)",
        "config": {"workload": "%s: TGV %dx%dx%d hex, p=%d, Re=%g, M=%g, BDF2 dt=%g t_c, pMG %s FMG "
                               "nu=10/10/30, FGMRES(30) rtol 1e-5, %d Newton/step"
                               % (args.config, *cfg["n"], cfg["p"], cfg["Re"], cfg["M"], cfg["dt_conv"],
                                  "-".join(map(str, cfg["p_levels"])), args.newton),
                   "dofs": mixed["ndofs"], "l2": "256 MB buffer written between timed steps",
                   "parallelism": "replicas (one independent case per GPU)"},
        "fp64": {"value": results.get("fp64", {}).get("value"),
                 "ms_per_step": results.get("fp64", {}).get("ms_per_step"),
                 "fgmres_iters_per_solve": results.get("fp64", {}).get("fgmres_iters_per_solve")},
        "fgmres_iters_per_solve": mixed["fgmres_iters_per_solve"],
        "mixed_vs_fp64_rel_l2": err, "mixed_vs_fp64_dW_rel_l2": err_dw,
        "roofline": dominant_roofline(roofs),
        "rooflines": roofs,
        "bj_apply_with_conversions": {"bound": "hbm",
                     "kernel": "bj_colmajor_kernel<float> (fine block-Jacobi apply; timed with the FP64<->FP32 "
                               "conversions of its input and output, whose bytes are counted)",
                     "achieved": bj["gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": bj["gbs"] / peaks["hbm_gbs"], "traffic": traffic,
                     "peak_source": "of fallback" if peaks.get("fallback") else "of measured (MEASURED_PEAKS.json hbm_gbs)",
                     "ms": bj["ms"], "algorithmic_bytes": bj["bytes"]},
        "jvp_fp64": roof["jvp_fp64"],
        "probe_tc": roof.get("probe_tc"),
        "mixed_bf16": bf16,
        "large_dt": large,
        "tgv32_p6": c3,
        "esdirk3": esd,
        "coarse_bilu": bilu,
        "triangles": tris,
        "q_space_jvp": qsp,
        "clocks": clk, "gpu_launches": launches, "e2e": e2e,
    }
    if not args.no_batched:
        line["batched"] = batched_sample(B)
    if not args.no_serving:
        line["serving"] = serving_sample(B)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = {k: v for k, v in cpu_baseline_sample(cfg, args.newton).items() if k != "seconds"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile_op(args):
    """Run one library operation --reps times after --warmup untimed ones, for
    profiling (ncu launch lists and kernel captures) and quick CUDA-event
    timings: jvp64 (FP64 exact JVP), residual64, bj (block-Jacobi apply), apply
    (one pMG application), refresh (preconditioner update), fgmres (one linear
    solve), step (one BDF2 step with --newton Newton iterations).  Prints the
    event milliseconds per repetition and the library's launches per repetition."""
    import torch
    from paper_1812_04789_gb300 import binding as B
    from paper_1812_04789_gb300 import build as BLD
    BLD.build()
    B.load()
    cfg = dict(wl.CONFIGS[args.config])
    if args.n:
        cfg["n"] = tuple(args.n) + (1,) * (3 - len(args.n))
    prec = B.PREC_MIXED if args.precision == "mixed" else B.PREC_FP64
    storage = B.STORE_BF16 if args.bf16 else B.STORE_NATIVE
    st = torch.cuda.Stream()
    op = args.profile_op
    with torch.cuda.stream(st):
        m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg), stream=st)
        W = torch.from_numpy(wl.initial_state(cfg)).cuda()
        dt = wl.time_step(cfg)
        sigma = 1.5 / dt
        v = torch.randn_like(W)
        out = torch.empty_like(W)
        pl = cfg["p_levels"]
        o = B.pmg_opts(pl, 10, 10, 30, cycle=B.CYCLE_FMG if len(pl) > 1 else B.CYCLE_BJ, precision=prec,
                       storage=storage)
        pmg = B.PMG(m, W, sigma, o, stream=st) if op in ("apply", "refresh", "fgmres", "step") else None
        bj = None
        if op == "bj":
            bj = B.PMG(m, W, sigma, B.pmg_opts((cfg["p"],), cycle=B.CYCLE_BJ, precision=prec, storage=storage),
                       stream=st)
        b = torch.empty_like(W)
        m.bdf2_rhs(W, W, W, dt, b, stream=st)
        Wk = torch.empty_like(W)

        def run():
            if op == "jvp64":
                m.jvp(W, v, out, sigma, stream=st)
            elif op == "residual64":
                m.residual(W, out, stream=st)
            elif op == "bj":
                bj.apply(v, out, stream=st)
            elif op == "apply":
                pmg.apply(v, out, stream=st)
            elif op == "refresh":
                pmg.refresh(W, sigma, stream=st)
            elif op == "fgmres":
                pmg.fgmres(W, b, out, stream=st)
            else:
                pmg.refresh(W, sigma, stream=st)
                Wk.copy_(W)
                for _ in range(args.newton):
                    m.bdf2_rhs(Wk, W, W, dt, b, stream=st)
                    pmg.fgmres(Wk, b, out, stream=st)
                    m.axpy(1.0, out, Wk, stream=st)
        for _ in range(args.warmup):
            run()
        torch.cuda.synchronize()
        l0 = B.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(args.reps):
            run()
        e1.record(st)
        e1.synchronize()
        print(json.dumps({"op": op, "precision": args.precision, "config": args.config, "n": cfg["n"],
                          "bf16": args.bf16, "ms_per_rep": e0.elapsed_time(e1) / args.reps,
                          "launches_per_rep": (B.launch_count() - l0) / args.reps}))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = wl.CONFIGS[args.config]
    times = []
    samples = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline_sample(cfg, args.newton)
        if i >= args.warmup:
            times.append(r["seconds"])
            samples.append(r)
    dofs = samples[0]["value"] * samples[0]["seconds"]
    value = dofs * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (closed-form Taylor-Green initial state, L2-projected)",
            "config": {"workload": "%s sampled on a 3^3 sub-mesh (CPU oracle)" % args.config},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": samples[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.profile_op:
        run_profile_op(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
