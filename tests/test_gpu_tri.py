"""Triangle meshes through the C ABI (dg_mesh_create_tri): residual, exact
JVP, blocks, p-multigrid and a BDF2 Newton update against the oracle's
triangular DG (Sec. 3: full-order P_p on triangles).

Bars: FP64 residual, JVP and blocks 1e-12 in the relative max-norm (the
quadrature sums of the oracle in another order), FP32 JVP mode 2e-5; pMG
apply 1e-10; FGMRES (FP64) iterations +-1 and 1e-10, mixed 10 % + 1 and
1e-6; free stream to rounding; discrete conservation; invalid meshes and
unsupported calls rejected."""
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
    with pytest.raises(B.DGError):                 # block ILU(0): structured meshes only
        B.PMG(gm, W, 1.0, B.pmg_opts((2, 1), coarse=B.COARSE_BILU))
    Kv = torch.empty_like(W)
    with pytest.raises(B.DGError):                 # the FD JVP: structured meshes only
        gm.jvp(W, W, Kv, 1.0, mode=B.JVP_FD, R_W=Kv.clone())


def _levels_case():
    cfg = wl.tri_config((4, 3), 2, p_levels=(2, 1, 0))
    om, oph, gm = both(cfg)
    W = wl.tri_perturbed_state(cfg, amp=0.05)
    sigma = 1.5 / wl.time_step(cfg)
    return cfg, om, oph, gm, W, sigma


def test_blocks_parity():
    """Coloured JVP probing: diagonal blocks (level 0) and neighbour blocks
    (level 1) against the oracle's complex-step probing."""
    cfg, om, oph, gm, W, sigma = _levels_case()
    pmg = B.PMG(gm, dev(W), sigma, B.pmg_opts((2, 1, 0), nu_pre=3, nu_post=3, nu_coarse=5))
    nb, nbc = 4 * om.nm, 4 * otri.n_modes_tri(1)
    D = torch.empty((om.E, nb, nb), dtype=torch.float64, device="cuda")
    pmg.export_blocks(0, B.BLOCKS_DIAG, D)
    Dref = otri.diag_blocks(om, oph, W, sigma)
    assert relmax(D.cpu().numpy(), Dref) <= 1e-12
    O = torch.empty((om.E, 3, nbc, nbc), dtype=torch.float64, device="cuda")
    pmg.export_blocks(1, B.BLOCKS_NEIGHBOUR, O)
    Oref = otri.offdiag_blocks(om, oph, W, 1)
    assert relmax(O.cpu().numpy(), Oref) <= 1e-12


@pytest.mark.parametrize("cycle", [B.CYCLE_FMG, B.CYCLE_V, B.CYCLE_BJ])
def test_pmg_apply_parity(cycle):
    cfg, om, oph, gm, W, sigma = _levels_case()
    pl, nu, nuc = (2, 1, 0), 3, 5
    mg = otri.pmg_setup(om, oph, W, sigma, pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc)
    r = wl.random_vector(W.shape, 21)
    ref = mg.mg_full(r) if cycle == B.CYCLE_FMG else (mg.mg_v(0, r, np.zeros_like(r)) if cycle == B.CYCLE_V
                                                      else mg.P[0](r))
    pmg = B.PMG(gm, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc, cycle=cycle))
    z = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    pmg.apply(dev(r), z)
    assert gm.status_sync() == B.DG_OK
    err = relmax(z.cpu().numpy(), ref)
    print("triangles, cycle %d: pMG apply rel max err %.3e" % (cycle, err))
    assert err <= 1e-10


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_bdf2_fgmres_step(precision):
    """One BDF2 Newton update (W^{n-1} = W^n) with FGMRES(pMG) on triangles:
    the right-hand side with the per-triangle mass, iterations and the state
    against the oracle (FP64: +-1 and 1e-10; mixed: 10 % + 1 and 1e-6)."""
    cfg, om, oph, gm, W, sigma = _levels_case()
    from oracle.solvers import fgmres
    dt = wl.time_step(cfg)
    bref = -otri.residual(om, oph, W)
    b = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    gm.bdf2_rhs(dev(W), dev(W), dev(W), dt, b)
    assert relmax(b.cpu().numpy(), bref) <= 1e-12
    Wk = W + 0.01 * wl.random_vector(W.shape, 3) * np.abs(W).max()
    bref = -(otri.mass_apply(om, 3.0 * Wk - 4.0 * W + W) / (2.0 * dt) + otri.residual(om, oph, Wk))
    gm.bdf2_rhs(dev(Wk), dev(W), dev(W), dt, b)
    assert relmax(b.cpu().numpy(), bref) <= 1e-12
    pl, nu, nuc = (2, 1, 0), 4, 8
    mg = otri.pmg_setup(om, oph, W, sigma, pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc)
    rhs = -otri.residual(om, oph, W)
    x_ref, st_ref = fgmres(lambda z: otri.jvp(om, oph, W, z, sigma), mg, rhs, restart=30, rtol=1e-5, max_restarts=3)
    pmg = B.PMG(gm, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc, precision=precision))
    dW = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    st = pmg.fgmres(dev(W), dev(rhs), dW, rtol=1e-5, max_restarts=3)
    x = dW.cpu().numpy()
    rel = np.linalg.norm(x - x_ref) / np.linalg.norm(W + x_ref)
    print("triangles, precision %d: FGMRES %d iterations vs oracle %d, rel %.3e" % (precision, st["iters"],
                                                                                     st_ref["iters"], rel))
    if precision == B.PREC_FP64:
        assert abs(st["iters"] - st_ref["iters"]) <= 1 and rel <= 1e-10
    else:
        assert st["iters"] <= int(1.1 * st_ref["iters"]) + 1 and rel <= 1e-6
    res = rhs - otri.jvp(om, oph, W, x, sigma)
    assert np.linalg.norm(res) <= 1.0001e-5 * np.linalg.norm(rhs)


def test_esdirk3_step_on_triangles():
    """dg_esdirk3_step on a triangle handle (per-triangle mass in the stage
    right-hand sides) against the oracle's ESDIRK3 step: FP64, W^{n+1} within
    1e-10 relative L2, FGMRES iterations within one per solve."""
    from oracle import timestep as ots
    cfg, om, oph, gm, W, _ = _levels_case()
    dt = wl.time_step(cfg)
    sigma = 1.0 / (ots.GAMMA * dt)
    pl, nu, nuc, newton = (2, 1, 0), 4, 8, 2
    P = otri.pmg_setup(om, oph, W, sigma, pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc)
    W1_ref, its = ots.esdirk3_dg_step(om, oph, W, dt, P, newton=newton, rtol=1e-5, max_restarts=3)
    pmg = B.PMG(gm, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc))
    Wout = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    st = pmg.esdirk3_step(dev(W), dt, Wout, newton=newton, max_restarts=3)
    assert gm.status_sync() == B.DG_OK
    W1 = Wout.cpu().numpy()
    rel = np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref)
    print("triangles: ESDIRK3 step rel L2 %.3e, iterations %d vs oracle %d" % (rel, st["iters"], sum(its)))
    assert abs(st["iters"] - sum(its)) <= 3 * newton
    assert rel <= 1e-10
    assert np.linalg.norm(W1 - W) / np.linalg.norm(W) > 1e-8     # the step moved the state
