"""FP32 element Jacobian blocks of the mixed-precision preconditioner, built on
the tensor cores (tcgen05, three TF32 passes), against the FP64 oracle, and
the SIMT FP32 kernel beside them.  Plus the standalone tcgen05 GEMM
check of the operand layout and descriptors.

Bars, as max |D_gpu - D_oracle| / max |D_oracle| over the sampled elements:
* SIMT FP32: 2e-6.  W, the tables and every pointwise derivative are rounded
  to FP32 (unit roundoff 2^-24 = 6e-8) and each entry sums ~10^3 terms whose
  magnitudes exceed the entry's (the volume and face parts nearly cancel);
  measured 2e-7 .. 6e-7 at p = 1 .. 6.
* tensor cores: 1e-4.  In the split a = a_hi + a_lo (a_hi = TF32(a)) the low
  part keeps 13 significant bits, of which the TF32 operand holds 11, so each
  product of hi*hi + hi*lo + lo*hi carries up to 3 * 2^-22 = 7e-7 relative
  error (the standalone GEMM check measures 3e-7 against the sum of |terms|);
  with the same cancellation this gives 2e-6 .. 4e-5 at p = 1 .. 6.  One TF32
  pass (2^-11 operand rounding) or a wrong operand layout would miss it by
  orders of magnitude."""
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blocks as oblocks
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))

# (config, sampled elements or None for all): 2D and 3D, p = 1..6, a direction
# with one element (its faces add neighbour-seeded terms to the diagonal), the
# full 512-column accumulator (p = 4) and seed-variable groups (p = 5, 6)
CASES = {
    "tgv3d_p2_3x2x4": (wl.make_config("tgv", 3, (3, 2, 4), 2, M=0.3, Re=100.0), None),
    "tgv3d_p1_1x2x5": (wl.make_config("tgv", 3, (1, 2, 5), 1, M=0.3, Re=100.0), None),
    "vortex2d_p2_5x7": (wl.make_config("vortex", 2, (5, 7), 2, M=0.5, Re=1000.0), None),
    "vortex2d_p5_3x4": (wl.make_config("vortex", 2, (3, 4), 5, M=0.5, Re=1000.0), None),
    "tgv3d_p4_3x3x3": (wl.make_config("tgv", 3, (3, 3, 3), 4, M=0.1, Re=1600.0), [0, 13, 26]),
    "tgv3d_p5_2x3x2": (wl.make_config("tgv", 3, (2, 3, 2), 5, M=0.1, Re=400.0), [0, 11]),
    "tgv3d_p6_2x2x2": (wl.make_config("tgv", 3, (2, 2, 2), 6, M=0.05, Re=1600.0), [0, 7]),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def test_umma_tf32_gemm(tmp_path):
    exe = str(tmp_path / "umma_tf32")
    cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "-I", build.CSRC,
           os.path.join(HERE, "csrc", "umma_tf32.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr


@pytest.mark.parametrize("kernel", ["tc", "simt"])
@pytest.mark.parametrize("name", list(CASES))
def test_mixed_diag_blocks_vs_oracle(name, kernel, monkeypatch):
    if kernel == "simt":
        monkeypatch.setenv("DG_PROBE_SIMT", "1")
    else:
        monkeypatch.delenv("DG_PROBE_SIMT", raising=False)
    cfg, sample = CASES[name]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    sigma = 2.5
    elems = np.arange(om.E) if sample is None else np.asarray(sample)
    D = oblocks.diag_blocks(om, oph, W, sigma, elems=elems)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    pmg = B.PMG(m, torch.from_numpy(W).cuda(), sigma,
                B.pmg_opts((cfg["p"],), cycle=B.CYCLE_BJ, precision=B.PREC_MIXED))
    Dg = torch.empty((om.E, om.nb, om.nb), dtype=torch.float32, device="cuda")
    pmg.export_blocks(0, B.BLOCKS_DIAG, Dg)
    assert m.status_sync() == B.DG_OK
    Dg = Dg.cpu().numpy().astype(np.float64)[elems]
    err = np.abs(Dg - D).max() / np.abs(D).max()
    print("%s %s: max |D_gpu - D| / max |D| = %.3e" % (name, kernel, err))
    assert err <= (1e-4 if kernel == "tc" else 2e-6)


# neighbour blocks at the first coarse order: (config, sampled elements, coarse p)
NBR_CASES = {
    "tgv3d_p2_3x2x4": (CASES["tgv3d_p2_3x2x4"][0], None, 1),
    "vortex2d_p2_5x7": (CASES["vortex2d_p2_5x7"][0], None, 1),
    "tgv3d_p4_3x3x3": (CASES["tgv3d_p4_3x3x3"][0], [0, 13, 26], 2),
    "tgv3d_p5_2x3x2": (CASES["tgv3d_p5_2x3x2"][0], [0, 11], 3),
}


@pytest.mark.parametrize("kernel", ["tc", "simt"])
@pytest.mark.parametrize("name", list(NBR_CASES))
def test_mixed_neighbour_blocks_vs_oracle(name, kernel, monkeypatch):
    """FP32 neighbour blocks dR_e/dW_nbr on the first coarse order (the
    inherited block-sparse operator's off-diagonal part).  With the tensor-core
    probe they come from the neighbour-seeded kernel, else from the SIMT probe.
    Bar 1e-5 relative to max |O|: the same FP32 rounding as the SIMT diagonal
    blocks, on sums of n_qf (1 + d) K-terms per entry."""
    if kernel == "simt":
        monkeypatch.setenv("DG_PROBE_SIMT", "1")
    else:
        monkeypatch.delenv("DG_PROBE_SIMT", raising=False)
    cfg, sample, pc = NBR_CASES[name]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    elems = np.arange(om.E) if sample is None else np.asarray(sample)
    O = oblocks.offdiag_blocks(om, oph, W, pc, elems=elems)
    nbc = om.m * wl.n_modes(pc, om.d)
    O = O.reshape(len(elems), 2 * om.d, nbc, nbc)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    pmg = B.PMG(m, torch.from_numpy(W).cuda(), 2.5,
                B.pmg_opts((cfg["p"], pc), nu_pre=2, nu_post=2, nu_coarse=4, precision=B.PREC_MIXED))
    Og = torch.empty((om.E, 2 * om.d, nbc, nbc), dtype=torch.float32, device="cuda")
    pmg.export_blocks(1, B.BLOCKS_NEIGHBOUR, Og)
    assert m.status_sync() == B.DG_OK
    Og = Og.cpu().numpy().astype(np.float64)[elems]
    err = np.abs(Og - O).max() / np.abs(O).max()
    print("%s %s: max |O_gpu - O| / max |O| = %.3e" % (name, kernel, err))
    assert err <= 1e-5
