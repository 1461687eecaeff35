"""Block ILU(0) on the coarsest p-multigrid level (Sec. 6.3, Table
MGSettings) through the C ABI, against the oracle's textbook ILU(0).

Bars: the pMG application (FP64) 1e-10 in the relative max-norm, as for block
Jacobi (the library's pivot-block form and the oracle's IKJ form are the same
factors, rounded in another order); the MDF element order equal to the
oracle's (an integer result, taken from blocks that agree to ~1e-13 on a state
with well separated weights); FGMRES step (FP64) iterations +-1 and the state
within 1e-10; mixed precision within 1e-6 of the FP64 oracle's state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bilu as obilu
from oracle import solvers as osolvers
from oracle.dg import residual as o_residual, jvp as o_jvp
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics, relmax

pytestmark = pytest.mark.gpu

CASES = {
    "tgv3d_p2_4x2x4": (wl.make_config("tgv", 3, (4, 2, 4), 2, M=0.3, Re=100.0), (2, 1, 0)),
    "tgv3d_p2_4x2x4_c1": (wl.make_config("tgv", 3, (4, 2, 4), 2, M=0.3, Re=100.0), (2, 1)),
    "vortex2d_p2_5x4": (wl.make_config("vortex", 2, (5, 4), 2, M=0.5, Re=1000.0), (2, 1)),
}
KINDS = {"mdf": B.ORDER_MDF, "natural": B.ORDER_NATURAL, "colour": B.ORDER_COLOUR}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def _state(cfg):
    return wl.perturbed_state(cfg, amp=5e-2)


def _oracle(cfg, W, sigma, pl, nu, nuc, kind):
    return osolvers.pmg_setup(oracle_mesh(cfg), oracle_physics(cfg), W, sigma, pl, nu_pre=nu, nu_post=nu,
                              nu_coarse=nuc, coarse="bilu", order=kind)


def _gpu(cfg, W, sigma, pl, nu, nuc, kind, precision=B.PREC_FP64):
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    pmg = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc, precision=precision,
                                              coarse=B.COARSE_BILU, order=KINDS[kind]))
    return m, pmg


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("kind", list(KINDS))
def test_pmg_apply_with_bilu_matches_oracle(name, kind):
    cfg, pl = CASES[name]
    W = _state(cfg)
    sigma = 1.5 / wl.time_step(cfg)
    nu, nuc = 3, 5
    mg = _oracle(cfg, W, sigma, pl, nu, nuc, kind)
    r = wl.random_vector(W.shape, 31)
    ref = mg.mg_full(r)
    m, pmg = _gpu(cfg, W, sigma, pl, nu, nuc, kind)
    order, nl = pmg.bilu_order()
    P = mg.P[-1]
    assert order.tolist() == list(P.order)
    assert nl == obilu.levels(P.nbrs, P.order).max() + 1
    z = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    pmg.apply(dev(r), z)
    assert m.status_sync() == B.DG_OK
    err = relmax(z.cpu().numpy(), ref)
    print("%s %s: %d levels, pMG apply rel max err %.3e" % (name, kind, nl, err))
    assert err <= 1e-10


def test_refresh_reorders_and_refactors():
    """dg_pmg_refresh at a new state: the MDF order and factors follow the new
    blocks (the captured application graph reads them through pointers)."""
    cfg, pl = CASES["vortex2d_p2_5x4"]
    W0 = _state(cfg)
    W1 = wl.perturbed_state(cfg, seed=77, amp=8e-2)
    sigma = 1.5 / wl.time_step(cfg)
    m, pmg = _gpu(cfg, W0, sigma, pl, 3, 5, "mdf")
    pmg.refresh(dev(W1), 2.0 * sigma)
    mg = _oracle(cfg, W1, 2.0 * sigma, pl, 3, 5, "mdf")
    order, _ = pmg.bilu_order()
    assert order.tolist() == list(mg.P[-1].order)
    r = wl.random_vector(W1.shape, 32)
    z = torch.empty(W1.shape, dtype=torch.float64, device="cuda")
    pmg.apply(dev(r), z)
    assert m.status_sync() == B.DG_OK
    assert relmax(z.cpu().numpy(), mg.mg_full(r)) <= 1e-10


def _bdf2(cfg):
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = _state(cfg)
    sigma = 1.5 / wl.time_step(cfg)
    return om, oph, W, sigma, -o_residual(om, oph, W)


@pytest.mark.parametrize("kind", ["mdf", "natural"])
def test_fgmres_step_with_bilu_fp64(kind):
    cfg, pl = CASES["tgv3d_p2_4x2x4"]
    om, oph, W, sigma, b = _bdf2(cfg)
    nu, nuc = 4, 8
    P = _oracle(cfg, W, sigma, pl, nu, nuc, kind)
    x_ref, st_ref = osolvers.fgmres(lambda z: o_jvp(om, oph, W, z, sigma), P, b, restart=30, rtol=1e-5,
                                    max_restarts=3)
    m, pmg = _gpu(cfg, W, sigma, pl, nu, nuc, kind)
    dW = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    st = pmg.fgmres(dev(W), dev(b), dW, rtol=1e-5, max_restarts=3)
    print("%s: FGMRES iterations %d vs oracle %d" % (kind, st["iters"], st_ref["iters"]))
    assert abs(st["iters"] - st_ref["iters"]) <= 1
    x = dW.cpu().numpy()
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(W + x_ref) <= 1e-10
    res = b - o_jvp(om, oph, W, x, sigma)
    assert np.linalg.norm(res) <= 1.0001e-5 * np.linalg.norm(b)


def test_fgmres_step_with_bilu_mixed_precision():
    cfg, pl = CASES["tgv3d_p2_4x2x4_c1"]
    om, oph, W, sigma, b = _bdf2(cfg)
    nu, nuc = 4, 8
    P = _oracle(cfg, W, sigma, pl, nu, nuc, "natural")
    x_ref, st_ref = osolvers.fgmres(lambda z: o_jvp(om, oph, W, z, sigma), P, b, restart=30, rtol=1e-5)
    m, pmg = _gpu(cfg, W, sigma, pl, nu, nuc, "natural", precision=B.PREC_MIXED)
    dW = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    st = pmg.fgmres(dev(W), dev(b), dW, rtol=1e-5)
    x = dW.cpu().numpy()
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(W + x_ref) <= 1e-6
    assert st["iters"] <= int(1.1 * st_ref["iters"]) + 1
    res = b - o_jvp(om, oph, W, x, sigma)
    assert np.linalg.norm(res) <= 1.0001e-5 * np.linalg.norm(b)


def test_bilu_option_checks():
    W = None
    cfg3 = wl.make_config("tgv", 3, (3, 2, 4), 2, M=0.3, Re=100.0)        # a direction of 3 elements
    W = wl.initial_state(cfg3)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg3), wl.physics(cfg3))
    for opts in (B.pmg_opts((2, 1), coarse=B.COARSE_BILU),
                 B.pmg_opts((2,), cycle=B.CYCLE_BJ, coarse=B.COARSE_BILU)):
        with pytest.raises(B.DGError):
            B.PMG(m, dev(W), 10.0, opts)
    cfg, pl = CASES["tgv3d_p2_4x2x4"]
    W = wl.initial_state(cfg)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    for opts in (B.pmg_opts((2,), coarse=B.COARSE_BILU), B.pmg_opts(pl, coarse=B.COARSE_BILU, order=5),
                 B.pmg_opts(pl, coarse=3)):
        with pytest.raises(B.DGError):
            B.PMG(m, dev(W), 10.0, opts)
    pmg = B.PMG(m, dev(W), 10.0, B.pmg_opts(pl))
    with pytest.raises(B.DGError):
        pmg.bilu_order()                          # block Jacobi handle: no ILU
