"""The tensor-product space Q_p (the paper's quadrilateral basis, Sec. 3) through
the C ABI against the FP64 oracle with the same space: residual and exact JVP
(bar 1e-12 in the relative max-norm, as for P_p), a p-multigrid application
(1e-10) and the BDF2 FGMRES step in FP64 (iterations +-1, 1e-10) and in mixed
precision (1e-6, at most 10 % + 1 more iterations)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import solvers as osolvers
from oracle.dg import residual as o_residual, jvp as o_jvp
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics, relmax

pytestmark = pytest.mark.gpu

CASES = {
    "tgv3d_q2_3x2x2": wl.make_config("tgv", 3, (3, 2, 2), 2, M=0.3, Re=100.0, space="Q"),
    "vortex2d_q3_4x3": wl.make_config("vortex", 2, (4, 3), 3, M=0.5, Re=1000.0, space="Q"),
    "tgv3d_q1_1x2x3": wl.make_config("tgv", 3, (1, 2, 3), 1, M=0.3, Re=100.0, space="Q"),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_mesh(cfg):
    return B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))


@pytest.mark.parametrize("name", list(CASES))
def test_tensor_space_residual_and_jvp(name):
    cfg = CASES[name]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    m = gpu_mesh(cfg)
    assert m.nm == (cfg["p"] + 1) ** cfg["dim"]
    R = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    Kv = torch.empty_like(R)
    m.residual(dev(W), R)
    m.jvp(dev(W), dev(v), Kv, 3.7)
    assert m.status_sync() == B.DG_OK
    assert relmax(R.cpu().numpy(), o_residual(om, oph, W)) <= 1e-12
    assert relmax(Kv.cpu().numpy(), o_jvp(om, oph, W, v, 3.7)) <= 1e-12


def test_tensor_space_pmg_apply_and_steps():
    cfg = CASES["tgv3d_q2_3x2x2"]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.initial_state(cfg)
    dt = wl.time_step(cfg)
    sigma = 1.5 / dt
    pl, nu, nuc = (2, 1, 0), 4, 8
    mg = osolvers.pmg_setup(om, oph, W, sigma, pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc)
    r = wl.random_vector(W.shape, 21)
    m = gpu_mesh(cfg)
    pmg = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc))
    z = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    pmg.apply(dev(r), z)
    assert relmax(z.cpu().numpy(), mg.mg_full(r)) <= 1e-10
    # one Newton solve of the BDF2 step (W^{n-1} = W^n)
    b = -o_residual(om, oph, W)
    x_ref, st_ref = osolvers.fgmres(lambda q: o_jvp(om, oph, W, q, sigma), mg, b, restart=30, rtol=1e-5,
                                    max_restarts=3)
    W1_ref = W + x_ref
    for prec, bar in ((B.PREC_FP64, 1e-10), (B.PREC_MIXED, 1e-6)):
        p2 = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc, precision=prec))
        dW = torch.empty(W.shape, dtype=torch.float64, device="cuda")
        st = p2.fgmres(dev(W), dev(b), dW, rtol=1e-5, max_restarts=3)
        W1 = W + dW.cpu().numpy()
        rel = np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref)
        print("Q2 step precision %d: rel L2 %.3e, iterations %d vs %d" % (prec, rel, st["iters"], st_ref["iters"]))
        assert rel <= bar
        if prec == B.PREC_FP64:
            assert abs(st["iters"] - st_ref["iters"]) <= 1
        else:
            assert st["iters"] <= int(1.1 * st_ref["iters"]) + 1
