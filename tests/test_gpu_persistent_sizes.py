"""FP32 preconditioner kernels at mesh sizes where every persistent CTA loops
over several elements, against the FP64 oracle on sampled elements.

The tensor-core block probe launches min(E, SMs x occupancy) CTAs (one per SM
on a GB300, 152), the shared-memory FP32 volume kernel one CTA per SM with
three element slots, so meshes of 35 elements or fewer never give a CTA a
second element.  Here TGV 8^3 at p = 4 (E = 512: 3-4 elements per
tensor-core CTA, so its mbarrier phases and TMEM accumulators are reused
across elements, and 512 > 3 x 152 volume slots) and TGV 16^3 at p = 4
(E = 4096: about 27 elements per CTA) are compared element by element on
samples that include the first and last element of consecutive CTAs'
ranges.  Bars (reasoned in tests/test_gpu_probe_tc.py and test_jvp_fp32_mode):
tensor-core diagonal blocks 1e-4, FP32 neighbour blocks 1e-5, FP32 JVP and
inherited operator 2e-5, each relative to the oracle's max-norm over the
sample.  The FP32 JVP is the level-0 operator of a mixed handle
(dg_pmg_operator), with the primal traces cached at setup and without."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blocks as oblocks
from oracle import dg as odg
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics

pytestmark = pytest.mark.gpu

SIGMA = 2.5
CASES = {
    "tgv8_p4": ((8, 8, 8), [0, 1, 2, 3, 150, 151, 152, 153, 303, 304, 455, 456, 457, 510, 511]),
    "tgv16_p4": ((16, 16, 16), [0, 151, 152, 2047, 3000, 4095]),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def _case(name):
    n, elems = CASES[name]
    cfg = wl.make_config("tgv", 3, n, 4, M=0.1, Re=1600.0)
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    return cfg, om, oph, W, m, np.asarray(elems)


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name", list(CASES))
def test_tensor_core_diag_blocks_across_elements(name, monkeypatch):
    monkeypatch.delenv("DG_PROBE_SIMT", raising=False)
    cfg, om, oph, W, m, elems = _case(name)
    D = oblocks.diag_blocks(om, oph, W, SIGMA, elems=elems)
    pmg = B.PMG(m, torch.from_numpy(W).cuda(), SIGMA,
                B.pmg_opts((4,), cycle=B.CYCLE_BJ, precision=B.PREC_MIXED))
    Dg = torch.empty((om.E, om.nb, om.nb), dtype=torch.float32, device="cuda")
    pmg.export_blocks(0, B.BLOCKS_DIAG, Dg)
    assert m.status_sync() == B.DG_OK
    err = _rel(Dg[torch.from_numpy(elems).cuda()].cpu().numpy().astype(np.float64), D)
    print("%s tensor-core diagonal blocks: %.3e" % (name, err))
    assert err <= 1e-4


@pytest.mark.parametrize("name", list(CASES))
def test_fp32_neighbour_blocks_across_elements(name, monkeypatch):
    monkeypatch.delenv("DG_PROBE_SIMT", raising=False)
    cfg, om, oph, W, m, elems = _case(name)
    pc = 2
    nbc = om.m * wl.n_modes(pc, 3)
    O = oblocks.offdiag_blocks(om, oph, W, pc, elems=elems).reshape(len(elems), 6, nbc, nbc)
    pmg = B.PMG(m, torch.from_numpy(W).cuda(), SIGMA,
                B.pmg_opts((4, pc), nu_pre=2, nu_post=2, nu_coarse=4, precision=B.PREC_MIXED))
    Og = torch.empty((om.E, 6, nbc, nbc), dtype=torch.float32, device="cuda")
    pmg.export_blocks(1, B.BLOCKS_NEIGHBOUR, Og)
    assert m.status_sync() == B.DG_OK
    err = _rel(Og[torch.from_numpy(elems).cuda()].cpu().numpy().astype(np.float64), O)
    print("%s FP32 neighbour blocks: %.3e" % (name, err))
    assert err <= 1e-5


@pytest.mark.parametrize("cached", [True, False])
@pytest.mark.parametrize("name", list(CASES))
def test_fp32_smoother_operators_across_elements(name, cached, monkeypatch):
    """Level 0: the FP32 JVP the fine smoother runs (persistent volume kernel,
    face kernel, primal-trace cache on or off).  Level 1: the inherited
    block-sparse operator, against truncate(JVP(zero-pad(x))) (Sec. 6.1)."""
    if cached:
        monkeypatch.delenv("DG_PMG_NO_PRIMAL_CACHE", raising=False)
    else:
        monkeypatch.setenv("DG_PMG_NO_PRIMAL_CACHE", "1")
    cfg, om, oph, W, m, elems = _case(name)
    pmg = B.PMG(m, torch.from_numpy(W).cuda(), SIGMA,
                B.pmg_opts((4, 2, 1), nu_pre=2, nu_post=2, nu_coarse=4, precision=B.PREC_MIXED))
    v = wl.random_vector(W.shape, 21)
    y = torch.empty_like(torch.from_numpy(v)).cuda()
    pmg.operator(0, torch.from_numpy(v).cuda(), y)
    ref = odg.jvp(om, oph, W, v, SIGMA, elems=elems)
    err0 = _rel(y.cpu().numpy()[elems], ref)
    nmc = wl.n_modes(2, 3)
    xc = wl.random_vector((om.E, om.m, nmc), 22)
    yc = torch.empty((om.E, om.m, nmc), dtype=torch.float64, device="cuda")
    pmg.operator(1, torch.from_numpy(xc).cuda(), yc)
    refc = oblocks.restrict(odg.jvp(om, oph, W, oblocks.prolong(xc, om.nm), SIGMA, elems=elems), nmc)
    err1 = _rel(yc.cpu().numpy()[elems], refc)
    assert m.status_sync() == B.DG_OK
    print("%s cached=%s: FP32 JVP %.3e, inherited operator %.3e" % (name, cached, err0, err1))
    assert err0 <= 2e-5
    assert err1 <= 2e-5
