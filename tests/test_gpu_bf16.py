"""BF16 block storage of the mixed-precision smoothers (DG_STORE_BF16).

* The BF16 blocks are the FP32 blocks rounded to nearest-even: checked bit
  for bit against a rounding written here in integer arithmetic, for the
  inverse diagonal blocks of every level and the inherited neighbour blocks.
* The BF16 block-Jacobi apply and block-sparse operator multiply those
  values in FP32: the block-Jacobi apply is compared with the same product in
  FP64 from the exported BF16 values (bar 1e-5 relative, FP32 accumulation of
  nb terms); the operator of level 1 against the oracle's Galerkin operator
  truncate(JVP(zero-pad(x))) (Sec. 6.1) within the rounding bound
  2^-8 sum_j |A_ij| |x_j| plus 2e-5 max |y| for the FP32 rest.
* A mixed-precision BDF2 FGMRES solve with BF16 blocks meets the FP64
  oracle's solution within 1e-6 relative L2 with at most 10 % + 1 more
  iterations (the workload's mixed-precision bar)."""
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
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def bf16_round(a):
    """FP32 -> BF16 (as FP32 values) by round to nearest, ties to even."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (r.astype(np.uint32) << 16).view(np.float32)


CFG = wl.make_config("tgv", 3, (4, 3, 4), 4, M=0.1, Re=1600.0)
LEVELS = (4, 2, 1, 0)


def _handles(cfg, W, sigma, levels=LEVELS, nu=4, nuc=8):
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    h32 = B.PMG(m, dev(W), sigma, B.pmg_opts(levels, nu, nu, nuc, precision=B.PREC_MIXED))
    h16 = B.PMG(m, dev(W), sigma, B.pmg_opts(levels, nu, nu, nuc, precision=B.PREC_MIXED,
                                             storage=B.STORE_BF16))
    return m, h32, h16


def test_bf16_blocks_are_rounded_fp32_blocks():
    W = wl.perturbed_state(CFG, amp=0.05)
    m, h32, h16 = _handles(CFG, W, 2.5)
    E, d = m.E, 3
    for l, p in enumerate(LEVELS):
        nb = 5 * wl.n_modes(p, d)
        kinds = [B.BLOCKS_DIAG_INV] + ([B.BLOCKS_NEIGHBOUR] if l >= 1 else [])
        for which in kinds:
            n = E * (2 * d if which == B.BLOCKS_NEIGHBOUR else 1)
            a = torch.empty((n, nb, nb), dtype=torch.float32, device="cuda")
            b = torch.empty_like(a)
            h32.export_blocks(l, which, a)
            h16.export_blocks(l, which, b)
            a, b = a.cpu().numpy(), b.cpu().numpy()
            assert np.array_equal(bf16_round(a), b), (l, which)
            assert np.abs(a - b).max() > 0.0          # BF16 really is coarser than FP32
    assert m.status_sync() == B.DG_OK


def test_bf16_block_jacobi_apply():
    W = wl.perturbed_state(CFG, amp=0.05)
    m = B.Mesh.from_workload(wl.mesh_desc(CFG), wl.physics(CFG))
    h = B.PMG(m, dev(W), 2.5, B.pmg_opts((4,), cycle=B.CYCLE_BJ, precision=B.PREC_MIXED,
                                          storage=B.STORE_BF16))
    nb = 175
    Ainv = torch.empty((m.E, nb, nb), dtype=torch.float32, device="cuda")
    h.export_blocks(0, B.BLOCKS_DIAG_INV, Ainv)
    r = wl.random_vector(W.shape, 31)
    z = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    h.apply(dev(r), z)
    r32 = r.astype(np.float32).astype(np.float64).reshape(m.E, nb)
    ref = np.einsum("eij,ej->ei", Ainv.cpu().numpy().astype(np.float64), r32).reshape(W.shape)
    err = np.abs(z.cpu().numpy() - ref).max() / np.abs(ref).max()
    print("BF16 block-Jacobi apply vs FP64 product of the BF16 blocks: %.3e" % err)
    assert err <= 1e-5


def test_bf16_inherited_operator_vs_oracle():
    cfg = CFG
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    sigma = 2.5
    m, h32, h16 = _handles(cfg, W, sigma)
    nmc = wl.n_modes(2, 3)
    nbc = 5 * nmc
    x = wl.random_vector((om.E, om.m, nmc), 32)
    y = torch.empty(x.shape, dtype=torch.float64, device="cuda")
    h16.operator(1, dev(x), y)
    ref = oblocks.restrict(o_jvp(om, oph, W, oblocks.prolong(x, om.nm), sigma), nmc)
    # rounding bound from the oracle's own blocks of the Galerkin operator
    D = oblocks.truncate_block(oblocks.diag_blocks(om, oph, W, sigma), om.m, om.nm, nmc)
    O = oblocks.offdiag_blocks(om, oph, W, 2)
    ax = np.abs(x).reshape(om.E, nbc)
    bound = np.einsum("eab,eb->ea", np.abs(D), ax)
    for k in range(3):
        for s in range(2):
            bound += np.einsum("eab,eb->ea", np.abs(O[:, k, s]), ax[om.nbr[:, k, s]])
    diff = np.abs(y.cpu().numpy() - ref).reshape(om.E, nbc)
    tol = 2.0 ** -8 * bound + 2e-5 * np.abs(ref).max()
    print("BF16 operator: max |diff| / bound = %.3f" % float((diff / tol).max()))
    assert np.all(diff <= tol)
    # and it is not the FP32 operator: BF16 rounding is visible
    y32 = torch.empty_like(y)
    h32.operator(1, dev(x), y32)
    assert not torch.equal(y, y32)


def test_bf16_mixed_fgmres_step_vs_fp64_oracle():
    cfg = wl.make_config("tgv", 3, (3, 3, 3), 4, M=0.1, Re=1600.0)
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.initial_state(cfg)
    sigma = 1.5 / wl.time_step(cfg)
    b = -o_residual(om, oph, W)
    pl, nu, nuc = (4, 2, 1, 0), 10, 30
    P = osolvers.pmg_setup(om, oph, W, sigma, pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc)
    x_ref, st_ref = osolvers.fgmres(lambda z: o_jvp(om, oph, W, z, sigma), P, b, restart=30, rtol=1e-5)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    pmg = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc,
                                              precision=B.PREC_MIXED, storage=B.STORE_BF16))
    dW = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    st = pmg.fgmres(dev(W), dev(b), dW, rtol=1e-5)
    x = dW.cpu().numpy()
    W1, W1_ref = W + x, W + x_ref
    rel = np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref)
    print("BF16 mixed step: iterations %d (oracle %d), W^{n+1} rel L2 %.3e" % (st["iters"], st_ref["iters"], rel))
    assert rel <= 1e-6
    assert st["iters"] <= int(1.1 * st_ref["iters"]) + 1
    res = b - o_jvp(om, oph, W, x, sigma)
    assert np.linalg.norm(res) <= 1.0001e-5 * np.linalg.norm(b)


def test_bf16_rejected_outside_mixed_precision():
    m = B.Mesh.from_workload(wl.mesh_desc(CFG), wl.physics(CFG))
    W = dev(wl.initial_state(CFG))
    with pytest.raises(B.DGError):
        B.PMG(m, W, 2.5, B.pmg_opts(LEVELS, 2, 2, 4, precision=B.PREC_FP64, storage=B.STORE_BF16))
    with pytest.raises(B.DGError):
        B.PMG(m, W, 2.5, B.pmg_opts(LEVELS, 2, 2, 4, precision=B.PREC_MIXED, storage=7))
