"""Triangle meshes through the C ABI (dg_mesh_create_tri): residual and exact
JVP against the oracle's triangular DG (Sec. 3: full-order P_p on triangles).

Bars: FP64 residual and JVP 1e-12 in the relative max-norm (the quadrature
sums of the oracle in another order), FP32 JVP mode 2e-5; free stream to
rounding; discrete conservation; invalid meshes rejected."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import tri as otri
from oracle.physics import Physics
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import relmax

pytestmark = pytest.mark.gpu

CASES = {
    "tri_4x3_p2": wl.tri_config((4, 3), 2),
    "tri_5x4_p4": wl.tri_config((5, 4), 4),
    "tri_2x2_p0": wl.tri_config((2, 2), 0),
    "tri_3x5_p6_viscous": wl.tri_config((3, 5), 6, Re=50.0),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def both(cfg):
    msh = wl.tri_mesh(cfg)
    P = wl.tri_physics(cfg)
    om = otri.TriMesh(msh["X"], msh["tri"], msh["shift"], msh["lo"], msh["hi"], cfg["p"])
    oph = Physics(gamma=P["gamma"], Pr=P["Pr"], mu=P["mu"], Rgas=P["Rgas"], eta=P["eta"], roe_delta=P["roe_delta"])
    gm = B.Mesh.from_tri_workload(msh, P, cfg["p"])
    return om, oph, gm


@pytest.mark.parametrize("name", list(CASES))
def test_residual_parity(name):
    cfg = CASES[name]
    om, oph, gm = both(cfg)
    W = wl.tri_perturbed_state(cfg, amp=0.05)
    assert gm.shape == W.shape
    R = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    gm.residual(dev(W), R)
    assert gm.status_sync() == B.DG_OK
    ref = otri.residual(om, oph, W)
    err = relmax(R.cpu().numpy(), ref)
    print("%s: residual rel max err %.3e" % (name, err))
    assert err <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_jvp_parity(name):
    cfg = CASES[name]
    om, oph, gm = both(cfg)
    W = wl.tri_perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape, 9)
    sigma = 2.5
    Kv = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    gm.jvp(dev(W), dev(v), Kv, sigma)
    ref = otri.jvp(om, oph, W, v, sigma)
    err = relmax(Kv.cpu().numpy(), ref)
    print("%s: JVP rel max err %.3e" % (name, err))
    assert err <= 1e-12
    Kf = torch.empty_like(Kv)
    gm.jvp(dev(W), dev(v), Kf, sigma, mode=B.JVP_EXACT_FP32)
    assert gm.status_sync() == B.DG_OK
    assert relmax(Kf.cpu().numpy(), ref) <= 2e-5


def test_free_stream_and_conservation():
    cfg = CASES["tri_5x4_p4"]
    om, oph, gm = both(cfg)
    W = np.zeros(wl.tri_state_shape(cfg))
    c0 = math.sqrt(2.0)
    W[:, 0, 0], W[:, 1, 0], W[:, 2, 0] = c0, 0.3 * c0, -0.2 * c0
    W[:, 3, 0] = (1.0 / 0.4 + 0.5 * 0.13) * c0
    R = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    gm.residual(dev(W), R)
    assert R.abs().max().item() <= 1e-13 * np.abs(W).max()
    W = wl.tri_perturbed_state(cfg, amp=0.05)
    gm.residual(dev(W), R)
    Rn = R.cpu().numpy()
    assert np.abs(Rn[:, :, 0].sum(axis=0)).max() <= 1e-13 * np.abs(Rn).max()


def test_invalid_triangulations_and_unsupported_calls():
    cfg = CASES["tri_4x3_p2"]
    msh = wl.tri_mesh(cfg)
    P = wl.tri_physics(cfg)
    cw = dict(msh)
    cw["tri"] = msh["tri"][:, ::-1].copy()          # clockwise
    cw["shift"] = msh["shift"][:, ::-1].copy()
    with pytest.raises(B.DGError):
        B.Mesh.from_tri_workload(cw, P, 2)
    open_ = dict(msh)
    open_["tri"] = msh["tri"][:-1].copy()           # a triangle missing: unmatched edges
    open_["shift"] = msh["shift"][:-1].copy()
    with pytest.raises(B.DGError):
        B.Mesh.from_tri_workload(open_, P, 2)
    gm = B.Mesh.from_tri_workload(msh, P, 2)
    W = dev(wl.tri_initial_state(cfg))
    with pytest.raises(B.DGError):
        B.PMG(gm, W, 1.0, B.pmg_opts((2,), cycle=B.CYCLE_BJ))
    b = torch.empty_like(W)
    with pytest.raises(B.DGError):
        gm.bdf2_rhs(W, W, W, 0.1, b)
