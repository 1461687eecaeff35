"""Batched element-block inverses (block Jacobi, Sec. 6.3) on every kernel path:
register tiles (n_b <= 176 in FP32, <= 128 in FP64), the block in shared
memory, and in place in global memory by panels of 16 columns (rank-16
updates; n_b = 175 in FP64, 280 and 420 in both precisions).  The exported inverse times the
exported (un-inverted) block of the same handle must be the identity.

Bars: FP64 1e-10 in max-norm (Gauss-Jordan with partial pivoting loses about
kappa * n_b * 2^-53; these blocks have kappa < 1e3); FP32 2e-3 (the same with
2^-24)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# (name, config, precision): the comment gives n_b and the path taken
CASES = [
    ("tgv3d_p1_fp64", wl.make_config("tgv", 3, (2, 2, 3), 1, M=0.3, Re=100.0), B.PREC_FP64),     # 20, registers
    ("tgv3d_p3_fp64", wl.make_config("tgv", 3, (2, 2, 2), 3, M=0.3, Re=100.0), B.PREC_FP64),     # 100, registers
    ("tgv3d_p4_fp64", wl.make_config("tgv", 3, (2, 2, 2), 4, M=0.1, Re=1600.0), B.PREC_FP64),    # 175, panels
    ("tgv3d_p4_mixed", wl.make_config("tgv", 3, (2, 2, 2), 4, M=0.1, Re=1600.0), B.PREC_MIXED),  # 175, registers
    ("vortex2d_p8_mixed", wl.make_config("vortex", 2, (3, 2), 8, M=0.5, Re=1000.0), B.PREC_MIXED),  # 180, shared
    ("tgv3d_p5_mixed", wl.make_config("tgv", 3, (2, 1, 2), 5, M=0.1, Re=400.0), B.PREC_MIXED),   # 280, panels
    ("tgv3d_p6_mixed", wl.make_config("tgv", 3, (2, 2, 1), 6, M=0.05, Re=1600.0), B.PREC_MIXED),  # 420, panels
    ("tgv3d_p6_fp64", wl.make_config("tgv", 3, (1, 2, 2), 6, M=0.05, Re=1600.0), B.PREC_FP64),    # 420, panels
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


@pytest.mark.parametrize("name,cfg,prec", CASES, ids=[c[0] for c in CASES])
def test_inverse_times_block_is_identity(name, cfg, prec):
    W = wl.perturbed_state(cfg, amp=0.05)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    pmg = B.PMG(m, torch.from_numpy(W).cuda(), 2.5,
                B.pmg_opts((cfg["p"],), cycle=B.CYCLE_BJ, precision=prec))
    E = W.shape[0]
    nb = W.shape[1] * W.shape[2]
    dt = torch.float64 if prec == B.PREC_FP64 else torch.float32
    D = torch.empty((E, nb, nb), dtype=dt, device="cuda")
    Dinv = torch.empty_like(D)
    pmg.export_blocks(0, B.BLOCKS_DIAG, D)
    pmg.export_blocks(0, B.BLOCKS_DIAG_INV, Dinv)
    assert m.status_sync() == B.DG_OK
    prod = torch.bmm(Dinv.double(), D.double()).cpu().numpy()
    err = np.abs(prod - np.eye(nb)[None]).max()
    print("%s: n_b %d, max |Dinv D - I| = %.3e" % (name, nb, err))
    assert err <= (1e-10 if prec == B.PREC_FP64 else 2e-3)
