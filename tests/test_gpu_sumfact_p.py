"""The volume term of the total-degree space P_p by sum factorisation: P_p is
the subset a0 + a1 + a2 <= p of the tensor Legendre products of Q_p, so the
sum-factorised Q_p kernel runs on the P_p coefficients with the other tensor
coefficients zero and writes back the P_p modes only.  It serves the FP64
residual and JVP of 3-D P_p meshes, and FP32 ones whose tables do not fit
the shared-memory kernel (p = 6).  Against the direct kernels
(DG_NO_SUMFACT_P=1): equal to rounding (bar 1e-13 relative max-norm, FP64);
against the oracle: the parity bars (1e-12 FP64, 2e-5 FP32)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dg import jvp as o_jvp, residual as o_residual
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics, relmax

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def _eval(cfg, W, v, sigma, mode):
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    Wd, vd = torch.from_numpy(W).cuda(), torch.from_numpy(v).cuda()
    R, K = torch.empty_like(Wd), torch.empty_like(Wd)
    m.residual(Wd, R)
    m.jvp(Wd, vd, K, sigma, mode=mode)
    assert m.status_sync() == B.DG_OK
    return R.cpu().numpy(), K.cpu().numpy()


@pytest.mark.parametrize("n,p", [((3, 4, 2), 2), ((4, 3, 3), 4), ((2, 2, 3), 6)])
def test_sumfact_p_equals_direct_and_oracle(n, p, monkeypatch):
    cfg = wl.make_config("tgv", 3, n, p, M=0.2, Re=200.0)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape, 8)
    sigma = 3.0
    monkeypatch.delenv("DG_NO_SUMFACT_P", raising=False)
    R1, K1 = _eval(cfg, W, v, sigma, B.JVP_EXACT)
    monkeypatch.setenv("DG_NO_SUMFACT_P", "1")
    R0, K0 = _eval(cfg, W, v, sigma, B.JVP_EXACT)
    assert relmax(R1, R0) <= 1e-13 and relmax(K1, K0) <= 1e-13
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    assert relmax(R1, o_residual(om, oph, W)) <= 1e-12
    assert relmax(K1, o_jvp(om, oph, W, v, sigma)) <= 1e-12


def test_sumfact_p6_fp32_jvp_vs_oracle(monkeypatch):
    """p = 6: the FP32 JVP takes the sum-factorised kernel (the shared-memory
    kernel's tables, 688 KB, do not fit); bar 2e-5 as for the FP32 mode."""
    monkeypatch.delenv("DG_NO_SUMFACT_P", raising=False)
    cfg = wl.make_config("tgv", 3, (2, 3, 2), 6, M=0.05, Re=1600.0)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape, 9)
    _, K = _eval(cfg, W, v, 2.0, B.JVP_EXACT_FP32)
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    err = relmax(K, o_jvp(om, oph, W, v, 2.0))
    print("p=6 FP32 JVP (sum factorised volume): %.3e" % err)
    assert err <= 2e-5


@pytest.mark.parametrize("space", ["P", "Q"])
@pytest.mark.parametrize("n,p", [((3, 4, 2), 1), ((1, 3, 2), 3), ((4, 3, 3), 4), ((2, 2, 3), 6)])
def test_sumfact_faces_equal_direct_kernel(n, p, space, monkeypatch):
    """The face term by sum factorisation (3-D; FP64 by default, FP32 here too
    through DG_SUMFACT_FACE_MIN_MODES=1) against the direct face kernel
    (DG_NO_SUMFACT_FACE=1): residual and JVP in
    FP64 to 1e-13, the FP32 JVP mode to 2e-5 (both relative max-norm), and the
    FP64 result against the oracle to 1e-12; a direction with one element
    makes an element its own face neighbour."""
    if space == "Q" and p > 4:
        pytest.skip("Q_6 tables: not a workload size")
    cfg = wl.make_config("tgv", 3, n, p, M=0.2, Re=200.0, space=space)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape, 10)
    sigma = 2.5
    out = {}
    monkeypatch.setenv("DG_SUMFACT_FACE_MIN_MODES", "1")
    for flag in ("0", "1"):
        monkeypatch.setenv("DG_NO_SUMFACT_FACE", flag)
        R, K = _eval(cfg, W, v, sigma, B.JVP_EXACT)
        _, K32 = _eval(cfg, W, v, sigma, B.JVP_EXACT_FP32)
        out[flag] = (R, K, K32)
    assert relmax(out["0"][0], out["1"][0]) <= 1e-13
    assert relmax(out["0"][1], out["1"][1]) <= 1e-13
    assert relmax(out["0"][2], out["1"][2]) <= 2e-5
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    assert relmax(out["0"][1], o_jvp(om, oph, W, v, sigma)) <= 1e-12
