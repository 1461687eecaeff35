"""dg_fgmres_step with the convergence test on the device (exact JVP): one
restart cycle is one graph launch, each iteration behind a conditional node
that the previous iteration's check opens, and the host waits once per cycle.
It runs the same kernels in the same order as the host-driven loop
(DG_FGMRES_HOST=1), so the two give the same iteration counts and the same
bits; restarts, the iteration limit and a converged start are covered, in
FP64 and mixed precision."""
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


def _problem(precision, levels=(2, 1, 0), n=(4, 3, 5), p=2):
    cfg = wl.make_config("tgv", 3, n, p, M=0.1, Re=1600.0, dt_conv=0.05)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    W = torch.from_numpy(wl.perturbed_state(cfg, amp=0.05)).cuda()
    sigma = 1.5 / wl.time_step(cfg)
    pmg = B.PMG(m, W, sigma, B.pmg_opts(levels, 3, 3, 6, precision=precision))
    b = torch.from_numpy(wl.random_vector(tuple(W.shape), 4)).cuda()
    return m, pmg, W, b


def _solve(pmg, W, b, host, monkeypatch, **kw):
    if host:
        monkeypatch.setenv("DG_FGMRES_HOST", "1")
    else:
        monkeypatch.delenv("DG_FGMRES_HOST", raising=False)
    dW = torch.empty_like(W)
    st = pmg.fgmres(W, b, dW, raise_on_error=False, **kw)
    return st, dW


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
@pytest.mark.parametrize("kw", [dict(rtol=1e-8), dict(rtol=1e-9, restart=3, max_restarts=8),
                                dict(rtol=1e-12, restart=2, max_restarts=0)])
def test_device_loop_equals_host_loop(precision, kw, monkeypatch):
    m, pmg, W, b = _problem(precision)
    sd, xd = _solve(pmg, W, b, False, monkeypatch, **kw)
    sh, xh = _solve(pmg, W, b, True, monkeypatch, **kw)
    print("device loop: %d iterations %s, host loop: %d %s" % (sd["iters"], B.STATUS_NAMES[sd["status"]],
                                                               sh["iters"], B.STATUS_NAMES[sh["status"]]))
    assert sd["status"] == sh["status"]
    assert sd["iters"] == sh["iters"]
    assert torch.equal(xd, xh)
    assert sd["res_final"] == sh["res_final"]
    if kw.get("max_restarts", 0) == 0 and kw["rtol"] == 1e-12:
        assert sd["status"] == B.DG_ERR_NOT_CONVERGED and sd["iters"] == 2
    else:
        assert sd["status"] == B.DG_OK
        assert sd["res_final"] <= kw["rtol"] * sd["res0"] * 1.0001


def test_zero_right_hand_side_takes_no_iteration(monkeypatch):
    m, pmg, W, b = _problem(B.PREC_MIXED)
    st, dW = _solve(pmg, W, torch.zeros_like(b), False, monkeypatch, rtol=1e-5)
    assert st["status"] == B.DG_OK and st["iters"] == 0
    assert torch.count_nonzero(dW) == 0


def test_new_shift_and_state_between_solves(monkeypatch):
    """The cycle graph works on staging copies of W and b (the caller's
    pointers change between solves) and is rebuilt when the shift changes."""
    m, pmg, W, b = _problem(B.PREC_FP64)
    W2 = W * 1.001
    for sigma_scale in (1.0, 2.0):
        pmg.refresh(W2, pmg.sigma * sigma_scale)
        sd, xd = _solve(pmg, W2, b, False, monkeypatch, rtol=1e-8)
        sh, xh = _solve(pmg, W2, b, True, monkeypatch, rtol=1e-8)
        assert sd["iters"] == sh["iters"] and torch.equal(xd, xh)
