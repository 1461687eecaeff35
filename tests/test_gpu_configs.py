"""The workload configurations at full size, through the C ABI.

* vortex 16^2 p=2, block Jacobi only, FP64: the whole BDF2 Newton step against
  the oracle's (iterations +-1, updated state within 1e-10 relative L2);
* TGV 16^3 p=4 and TGV 32^3 p=6: residual and exact JVP on sampled elements
  against the oracle evaluated one element at a time (1e-12 relative max-norm,
  normalised by the full GPU output), then one mixed-precision FGMRES(pMG) solve
  at full size whose true residual, measured with the FP64 JVP, meets the
  tolerance;
* the seeded batch of independent TGV cases (n 8..24, p 1..5): a subset through
  the serving runtime, every case's Newton step reduces its BDF2 residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blocks as oblocks
from oracle import solvers as osolvers
from oracle.dg import jvp as o_jvp, residual as o_residual
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available()
    B.load()


def _gpu(cfg):
    return B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))


def test_vortex16_p2_bj_fp64_step_matches_oracle():
    cfg = wl.CONFIGS["vortex2d_16_p2"]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W0 = wl.initial_state(cfg)
    dt = wl.time_step(cfg)
    Wm1 = wl.initial_state(cfg, t=-dt)
    sigma = 1.5 / dt
    # oracle: 2 Newton iterations, block Jacobi lagged at W^n
    P = oblocks.BlockJacobi(oblocks.diag_blocks(om, oph, W0, sigma), om.m, om.nm)
    Wk = W0.copy()
    its_ref = []
    for _ in range(2):
        f = osolvers.bdf2_rhs(om, o_residual(om, oph, Wk), Wk, W0, Wm1, dt)
        x, st = osolvers.fgmres(lambda z: o_jvp(om, oph, Wk, z, sigma), P, -f, rtol=1e-5, max_restarts=4)
        its_ref.append(st["iters"])
        Wk = Wk + x
    # GPU: same step through the C ABI
    m = _gpu(cfg)
    Wn, Wnm1 = torch.from_numpy(W0).cuda(), torch.from_numpy(Wm1).cuda()
    pmg = B.PMG(m, Wn, sigma, B.pmg_opts((2,), cycle=B.CYCLE_BJ))
    Wg = Wn.clone()
    b, dW = torch.empty_like(Wn), torch.empty_like(Wn)
    its = []
    for _ in range(2):
        m.bdf2_rhs(Wg, Wn, Wnm1, dt, b)
        its.append(pmg.fgmres(Wg, b, dW, rtol=1e-5, max_restarts=4)["iters"])
        m.axpy(1.0, dW, Wg)
    Wg = Wg.cpu().numpy()
    assert all(abs(a - b) <= 1 for a, b in zip(its, its_ref)), (its, its_ref)
    assert np.linalg.norm(Wg - Wk) / np.linalg.norm(Wk) <= 1e-10
    assert np.linalg.norm(Wg - W0) / np.linalg.norm(W0) > 1e-5


def _sampled_parity(cfg, sample):
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.02)
    v = wl.random_vector(W.shape)
    sigma = 1.5 / wl.time_step(cfg)
    m = _gpu(cfg)
    Wd, vd = torch.from_numpy(W).cuda(), torch.from_numpy(v).cuda()
    R, Kv = torch.empty_like(Wd), torch.empty_like(Wd)
    m.residual(Wd, R)
    m.jvp(Wd, vd, Kv, sigma)
    assert m.status_sync() == B.DG_OK
    Rg, Kg = R.cpu().numpy(), Kv.cpu().numpy()
    Rref = o_residual(om, oph, W, elems=sample)
    Kref = o_jvp(om, oph, W, v, sigma, elems=sample)
    assert np.abs(Rg[sample] - Rref).max() <= 1e-12 * np.abs(Rg).max()
    assert np.abs(Kg[sample] - Kref).max() <= 1e-12 * np.abs(Kg).max()
    return m, W


def _mixed_solve_true_residual(cfg, m, W):
    dt = wl.time_step(cfg)
    sigma = 1.5 / dt
    Wd = torch.from_numpy(W).cuda()
    pmg = B.PMG(m, Wd, sigma, B.pmg_opts(cfg["p_levels"], 10, 10, 30, precision=B.PREC_MIXED))
    b = torch.empty_like(Wd)
    m.bdf2_rhs(Wd, Wd, Wd, dt, b)
    dW = torch.empty_like(Wd)
    st = pmg.fgmres(Wd, b, dW, rtol=1e-5, max_restarts=4)
    Kx = torch.empty_like(Wd)
    m.jvp(Wd, dW, Kx, sigma)
    rel = float(torch.linalg.norm(b - Kx) / torch.linalg.norm(b))
    assert rel <= 1.01e-5, (rel, st)
    return st


def test_tgv16_p4_full_size_sampled_parity_and_mixed_solve():
    cfg = wl.CONFIGS["tgv16_p4"]
    rng = np.random.default_rng(5)
    sample = np.unique(np.concatenate([[0, 4095, 15, 255, 256], rng.integers(0, 4096, 11)]))
    m, W = _sampled_parity(cfg, sample)
    _mixed_solve_true_residual(cfg, m, W)


def test_tgv32_p6_full_size_sampled_parity_and_mixed_solve():
    cfg = wl.CONFIGS["tgv32_p6"]
    rng = np.random.default_rng(6)
    E = wl.n_elements(cfg)
    sample = np.unique(np.concatenate([[0, E - 1, 31, 1023, 1024], rng.integers(0, E, 5)]))
    m, W = _sampled_parity(cfg, sample)
    _mixed_solve_true_residual(cfg, m, W)


def test_batched_tgv_cases_through_the_server():
    cases = wl.batch_cases(64)[:8]
    srv = B.Server(budget_bytes=60 << 30, workers=4)
    outs = []
    for i, cfg in enumerate(cases):
        W0 = wl.initial_state(cfg)
        pl = cfg["p_levels"]
        opts = B.pmg_opts(pl, 10, 10, 30, cycle=B.CYCLE_FMG if len(pl) > 1 else B.CYCLE_BJ,
                          precision=B.PREC_MIXED)
        out = np.zeros_like(W0)
        outs.append((cfg, W0, out))
        srv.submit(i, wl.mesh_desc(cfg), wl.physics(cfg), opts, W0, W0, wl.time_step(cfg), out)
    res = []
    while len(res) < len(cases):
        res += srv.poll(1, timeout_ms=600000)
    srv.close()
    assert all(r["status"] == 0 for r in res), res
    for cfg, W0, W1 in outs:
        m = _gpu(cfg)
        dt = wl.time_step(cfg)
        Wn = torch.from_numpy(W0).cuda()
        f0, f1 = torch.empty_like(Wn), torch.empty_like(Wn)
        m.bdf2_rhs(Wn, Wn, Wn, dt, f0)
        m.bdf2_rhs(torch.from_numpy(W1).cuda(), Wn, Wn, dt, f1)
        # two Newton iterations with FGMRES at 1e-5 shrink the BDF2 residual
        assert float(torch.linalg.norm(f1)) <= 1e-4 * float(torch.linalg.norm(f0)), cfg
