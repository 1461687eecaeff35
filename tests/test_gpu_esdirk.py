"""ESDIRK3 step through the C ABI (dg_esdirk3_step) against the oracle's
(Sec. 4): three implicit stages, two Newton iterations each, FGMRES with the
preconditioner refreshed once at W^n and lagged over the step.

Bars (the BDF2 step's): FP64 W^{n+1} within 1e-10 relative L2 of the oracle and
FGMRES iterations within one per solve; mixed precision within 1e-6 relative
L2 of the FP64 oracle with at most 10 % + 1 more iterations per solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blocks as oblocks
from oracle import solvers as osolvers
from oracle import timestep as ots
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics

pytestmark = pytest.mark.gpu

CASES = {
    "vortex2d_p2_5x7_bj": (wl.make_config("vortex", 2, (5, 7), 2, M=0.5, Re=1000.0), (2,)),
    "tgv3d_p2_3x2x4_fmg": (wl.make_config("tgv", 3, (3, 2, 4), 2, M=0.3, Re=100.0), (2, 1, 0)),
}
NU, NUC, NEWTON = 4, 8, 2


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def _oracle(cfg, pl):
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.initial_state(cfg)
    dt = wl.time_step(cfg)
    sigma = 1.0 / (ots.GAMMA * dt)
    if len(pl) == 1:
        P = oblocks.BlockJacobi(oblocks.diag_blocks(om, oph, W, sigma), om.m, om.nm)
    else:
        P = osolvers.pmg_setup(om, oph, W, sigma, pl, nu_pre=NU, nu_post=NU, nu_coarse=NUC)
    W1, its = ots.esdirk3_dg_step(om, oph, W, dt, P, newton=NEWTON, rtol=1e-5, max_restarts=3)
    return W, dt, sigma, W1, its


def _gpu(cfg, pl, W, dt, sigma, precision):
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    Wn = torch.from_numpy(W).cuda()
    cyc = B.CYCLE_BJ if len(pl) == 1 else B.CYCLE_FMG
    pmg = B.PMG(m, Wn, sigma, B.pmg_opts(pl, nu_pre=NU, nu_post=NU, nu_coarse=NUC, cycle=cyc, precision=precision))
    Wout = torch.empty_like(Wn)
    st = pmg.esdirk3_step(Wn, dt, Wout, newton=NEWTON, max_restarts=3)
    assert m.status_sync() == B.DG_OK
    return Wout.cpu().numpy(), st


@pytest.mark.parametrize("name", list(CASES))
def test_esdirk3_step_fp64_matches_oracle(name):
    cfg, pl = CASES[name]
    W, dt, sigma, W1_ref, its = _oracle(cfg, pl)
    W1, st = _gpu(cfg, pl, W, dt, sigma, B.PREC_FP64)
    nsolves = 3 * NEWTON
    assert abs(st["iters"] - sum(its)) <= nsolves, (st, its)
    rel = np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref)
    print("%s: FP64 ESDIRK3 step rel L2 %.3e, iterations %d vs oracle %d" % (name, rel, st["iters"], sum(its)))
    assert rel <= 1e-10
    assert np.linalg.norm(W1 - W) / np.linalg.norm(W) > 1e-6     # the step moved the state


def test_esdirk3_step_mixed_precision_vs_fp64_oracle():
    cfg, pl = CASES["tgv3d_p2_3x2x4_fmg"]
    W, dt, sigma, W1_ref, its = _oracle(cfg, pl)
    W1, st = _gpu(cfg, pl, W, dt, sigma, B.PREC_MIXED)
    rel = np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref)
    print("mixed ESDIRK3 step rel L2 %.3e, iterations %d vs oracle %d" % (rel, st["iters"], sum(its)))
    assert rel <= 1e-6
    assert st["iters"] <= int(1.1 * sum(its)) + 3 * NEWTON
