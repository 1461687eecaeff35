"""Run one library operation a few times on a workload, for profiling
(ncu launch lists and kernel captures) and quick CUDA-event timings.

  python -m paper_1812_04789_gb300.profile_ops --op apply --precision mixed --reps 2

Operations: jvp64 (FP64 exact JVP), residual64, bj (block-Jacobi apply),
apply (one pMG application), refresh (preconditioner setup), fgmres (one
linear solve), step (one BDF2 implicit step with 2 Newton iterations).
Prints CUDA-event milliseconds per repetition and the kernel launch count.
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="tgv16_p4")
    ap.add_argument("--op", default="apply")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--n", type=int, nargs="*", default=None, help="override the mesh size")
    ap.add_argument("--bf16", action="store_true", help="BF16 block storage (mixed precision)")
    ap.add_argument("--dt", type=float, default=None, help="override the time step (convective units)")
    a = ap.parse_args()
    import torch
    from paper_1812_04789_gb300 import binding as B
    from paper_1812_04789_gb300 import build
    from paper_1812_04789_gb300 import workloads as wl
    build.build()
    B.load()
    cfg = dict(wl.CONFIGS[a.config])
    if a.n:
        cfg["n"] = tuple(a.n) + (1,) * (3 - len(a.n))
    if a.dt:
        cfg["dt_conv"] = a.dt
    prec = B.PREC_MIXED if a.precision == "mixed" else B.PREC_FP64
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg), stream=st)
        W = torch.from_numpy(wl.initial_state(cfg)).cuda()
        dt = wl.time_step(cfg)
        sigma = 1.5 / dt
        v = torch.randn_like(W)
        out = torch.empty_like(W)
        pl = cfg["p_levels"]
        o = B.pmg_opts(pl, 10, 10, 30, cycle=B.CYCLE_FMG if len(pl) > 1 else B.CYCLE_BJ, precision=prec,
                       storage=B.STORE_BF16 if a.bf16 else B.STORE_NATIVE)
        pmg = B.PMG(m, W, sigma, o, stream=st) if a.op in ("apply", "refresh", "fgmres", "step") else None
        bj = None
        if a.op == "bj":
            bj = B.PMG(m, W, sigma, B.pmg_opts((cfg["p"],), cycle=B.CYCLE_BJ, precision=prec,
                                               storage=B.STORE_BF16 if a.bf16 else B.STORE_NATIVE), stream=st)
        b = torch.empty_like(W)
        m.bdf2_rhs(W, W, W, dt, b, stream=st)
        Wk = torch.empty_like(W)

        def op():
            if a.op == "jvp64":
                m.jvp(W, v, out, sigma, stream=st)
            elif a.op == "residual64":
                m.residual(W, out, stream=st)
            elif a.op == "bj":
                bj.apply(v, out, stream=st)
            elif a.op == "apply":
                pmg.apply(v, out, stream=st)
            elif a.op == "refresh":
                pmg.refresh(W, sigma, stream=st)
            elif a.op == "fgmres":
                pmg.fgmres(W, b, out, stream=st)
            elif a.op == "step":
                pmg.refresh(W, sigma, stream=st)
                Wk.copy_(W)
                for _ in range(2):
                    m.bdf2_rhs(Wk, W, W, dt, b, stream=st)
                    pmg.fgmres(Wk, b, out, stream=st)
                    m.axpy(1.0, out, Wk, stream=st)
            else:
                raise SystemExit("unknown op " + a.op)
        for _ in range(a.warmup):
            op()
        torch.cuda.synchronize()
        l0 = B.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(a.reps):
            op()
        e1.record(st)
        e1.synchronize()
        its = None
        if a.op in ("fgmres", "step"):
            its = pmg.fgmres(W, b, out, stream=st)["iters"]
        print(json.dumps({"op": a.op, "precision": a.precision, "config": a.config, "n": cfg["n"], "bf16": a.bf16,
                          "iters": its,
                          "ms_per_rep": e0.elapsed_time(e1) / a.reps,
                          "launches_per_rep": (B.launch_count() - l0) / a.reps}))


if __name__ == "__main__":
    main()
