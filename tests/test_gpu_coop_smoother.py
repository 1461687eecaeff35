"""The persistent coarse-level smoother (one cooperative launch per SMOOTH
call of Algorithm 2 on the inherited FP32 or BF16 levels) against the
launch-per-operation smoother it replaces, and its bounded grid barrier.

* Same preconditioner: an MG_full application (Algorithm 1) with the
  persistent smoothers equals the launch-per-operation one to FP32 rounding
  carried through the smoothing iterations (the inner products are summed in
  another order): bar 1e-4 relative max-norm, as for the primal-trace cache.
  A mesh of 8^3 elements at p = 4 gives every CTA several elements.
* The FGMRES solve preconditioned by it meets the FP64 oracle as the other
  mixed-precision solves do (test_gpu_parity.py runs with the persistent
  smoother on by default); here the iteration counts of both smoothers agree.
* Failure detection without a fault: a test hook makes every grid barrier
  wait for one CTA that does not exist; the wait runs out after its bound,
  the kernel returns, the status word reads DG_ERR_TIMEOUT, later launches of
  the application return at once, and the context stays usable (a fresh
  handle then gives the normal result)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def _setup(n, p, levels, storage, monkeypatch, coop, nu=10, nuc=30):
    if coop:
        monkeypatch.delenv("DG_PMG_NO_COOP", raising=False)
    else:
        monkeypatch.setenv("DG_PMG_NO_COOP", "1")
    cfg = wl.make_config("tgv", 3, n, p, M=0.1, Re=1600.0)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    W = torch.from_numpy(wl.perturbed_state(cfg, amp=0.05)).cuda()
    sigma = 1.5 / wl.time_step(cfg)
    pmg = B.PMG(m, W, sigma, B.pmg_opts(levels, nu, nu, nuc, precision=B.PREC_MIXED, storage=storage))
    return cfg, m, W, sigma, pmg


@pytest.mark.parametrize("storage", [B.STORE_NATIVE, B.STORE_BF16])
@pytest.mark.parametrize("n,p,levels", [((8, 8, 8), 4, (4, 2, 1, 0)), ((4, 3, 5), 2, (2, 1, 0))])
def test_persistent_smoother_matches_launch_per_operation(n, p, levels, storage, monkeypatch):
    out, launches = [], []
    for coop in (False, True):
        cfg, m, W, sigma, pmg = _setup(n, p, levels, storage, monkeypatch, coop)
        r = torch.from_numpy(wl.random_vector(W.shape, 5)).cuda()
        z = torch.empty_like(r)
        l0 = B.launch_count()
        pmg.apply(r, z)
        torch.cuda.synchronize()
        launches.append(B.launch_count() - l0)
        assert m.status_sync() == B.DG_OK
        out.append(z.cpu().numpy())
        pmg.close()
        m.close()
    err = float(np.abs(out[0] - out[1]).max() / np.abs(out[0]).max())
    print("%s p=%d storage=%d: persistent vs per-operation %.3e; launches %d -> %d"
          % (n, p, storage, err, launches[0], launches[1]))
    assert err <= 1e-4
    assert launches[1] < launches[0] / 3


def test_persistent_smoother_fgmres_iterations(monkeypatch):
    its = []
    for coop in (False, True):
        cfg, m, W, sigma, pmg = _setup((8, 8, 8), 4, (4, 2, 1, 0), B.STORE_NATIVE, monkeypatch, coop)
        b = torch.empty_like(W)
        m.bdf2_rhs(W, W, W, wl.time_step(cfg), b)
        dW = torch.empty_like(W)
        st = pmg.fgmres(W, b, dW, rtol=1e-8, max_restarts=2)
        its.append(st["iters"])
        pmg.close()
        m.close()
    print("FGMRES iterations to 1e-8: per-operation %d, persistent %d" % tuple(its))
    assert abs(its[0] - its[1]) <= 1


def test_grid_barrier_wait_runs_out_and_reports_timeout(monkeypatch):
    monkeypatch.setenv("DG_TEST_COOP_BARRIER_EXTRA", "1")
    cfg, m, W, sigma, pmg = _setup((4, 3, 5), 2, (2, 1, 0), B.STORE_NATIVE, monkeypatch, True, nu=3, nuc=5)
    r = torch.from_numpy(wl.random_vector(W.shape, 6)).cuda()
    z = torch.empty_like(r)
    t0 = time.perf_counter()
    pmg.apply(r, z)
    code = m.status_sync()
    sec = time.perf_counter() - t0
    print("barrier that is never met: %s after %.2f s" % (B.STATUS_NAMES[code], sec))
    assert code == B.DG_ERR_TIMEOUT
    assert sec < 30.0                       # one bounded wait (2 s), the later launches return at once
    pmg.close()
    # the context is still usable: a handle without the hook gives the normal result
    monkeypatch.delenv("DG_TEST_COOP_BARRIER_EXTRA")
    pmg2 = B.PMG(m, W, sigma, B.pmg_opts((2, 1, 0), 3, 3, 5, precision=B.PREC_MIXED))
    pmg2.apply(r, z)
    assert m.status_sync() == B.DG_OK
    assert torch.isfinite(z).all()
    R = torch.empty_like(W)
    m.residual(W, R)
    assert m.status_sync() == B.DG_OK
