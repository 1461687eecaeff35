"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Bars: residual and exact JVP 1e-12 in the relative max-norm (FP64 evaluation
of the same quadrature sums in another order; the workload's bar); block-Jacobi inverses 1e-10 (Dinv_gpu D_oracle = I);
neighbour blocks 1e-12; pMG apply (FP64) 1e-10; FGMRES step (FP64) same
iteration count +-1 and the updated state within 1e-10 relative L2; mixed
precision within 1e-6 relative L2 of the FP64 oracle's updated state with at
most 10 % more iterations (+1)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blocks as oblocks
from oracle import solvers as osolvers
from oracle.dg import residual as o_residual, jvp as o_jvp, jvp_fd as o_jvp_fd
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics, relmax, uniform_state

pytestmark = pytest.mark.gpu

CASES = {
    "tgv3d_p2_3x2x4": wl.make_config("tgv", 3, (3, 2, 4), 2, M=0.3, Re=100.0),
    "tgv3d_p4_3x3x3": wl.make_config("tgv", 3, (3, 3, 3), 4, M=0.1, Re=1600.0),
    "tgv3d_p1_1x2x5": wl.make_config("tgv", 3, (1, 2, 5), 1, M=0.3, Re=100.0),
    "tgv3d_p0_2x2x3": wl.make_config("tgv", 3, (2, 2, 3), 0, M=0.3, Re=100.0),
    "vortex2d_p2_5x7": wl.make_config("vortex", 2, (5, 7), 2, M=0.5, Re=1000.0),
    "vortex2d_p5_3x4": wl.make_config("vortex", 2, (3, 4), 5, M=0.5, Re=1000.0),
    "vortex2d_p3_1x1": wl.make_config("vortex", 2, (1, 1), 3, M=0.5, Re=1000.0),
    "tgv3d_p6_2x2x2": wl.make_config("tgv", 3, (2, 2, 2), 6, M=0.05, Re=1600.0),
}


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_mesh(cfg):
    return B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1812_04789_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.load()


@pytest.mark.parametrize("name", list(CASES))
def test_residual_parity(name):
    cfg = CASES[name]
    W = wl.perturbed_state(cfg, amp=0.05)
    ref = o_residual(oracle_mesh(cfg), oracle_physics(cfg), W)
    m = gpu_mesh(cfg)
    Wd = dev(W)
    R = torch.empty_like(Wd)
    m.residual(Wd, R)
    assert m.status_sync() == B.DG_OK
    assert relmax(R.cpu().numpy(), ref) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_jvp_exact_parity(name):
    cfg = CASES[name]
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    sigma = 3.7
    ref = o_jvp(oracle_mesh(cfg), oracle_physics(cfg), W, v, sigma)
    m = gpu_mesh(cfg)
    Kv = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    m.jvp(dev(W), dev(v), Kv, sigma)
    assert relmax(Kv.cpu().numpy(), ref) <= 1e-12


def test_residual_source_and_free_stream():
    cfg = CASES["tgv3d_p2_3x2x4"]
    m = gpu_mesh(cfg)
    W = uniform_state(cfg)
    R = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    m.residual(dev(W), R)
    assert R.abs().max().item() <= 1e-13 * np.abs(W).max()
    S = wl.random_vector(W.shape, 9)
    m.residual(dev(W), R, S=dev(S))
    assert relmax(R.cpu().numpy(), -S) <= 1e-13


@pytest.mark.parametrize("name", ["tgv3d_p4_3x3x3", "tgv3d_p2_3x2x4", "vortex2d_p5_3x4", "tgv3d_p1_1x2x5",
                                  "tgv3d_p6_2x2x2"])
def test_jvp_fp32_mode(name):
    """The FP32 exact JVP (the fine-level smoother operator of the mixed
    preconditioner) against the FP64 oracle.  Bar 2e-5 in the relative
    max-norm: W and v rounded to FP32 (2^-24) and sums of ~10^3 terms per
    output whose volume and face parts largely cancel."""
    cfg = CASES[name]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    sigma = 1.5 / wl.time_step(cfg)
    ref = o_jvp(om, oph, W, v, sigma)
    m = gpu_mesh(cfg)
    out = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    m.jvp(dev(W), dev(v), out, sigma, mode=B.JVP_EXACT_FP32)
    assert m.status_sync() == B.DG_OK
    err = relmax(out.cpu().numpy(), ref)
    print("%s: FP32 JVP rel max err %.3e" % (name, err))
    assert err <= 2e-5


@pytest.mark.parametrize("mode,variant", [(B.JVP_FD, "printed"), (B.JVP_FD_SCALED, "scaled")])
def test_jvp_fd_modes(mode, variant):
    cfg = CASES["vortex2d_p2_5x7"]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    RW = o_residual(om, oph, W)
    ref_fd = o_jvp_fd(om, oph, W, RW, v, 2.0, variant=variant)
    exact = o_jvp(om, oph, W, v, 2.0)
    m = gpu_mesh(cfg)
    Wd = dev(W)
    RWd = torch.empty_like(Wd)
    m.residual(Wd, RWd)
    Kv = torch.empty_like(Wd)
    m.jvp(Wd, dev(v), Kv, 2.0, mode=mode, R_W=RWd)
    got = Kv.cpu().numpy()
    # both sides take the same finite difference; rounding in R is amplified by 1/h
    assert relmax(got, ref_fd) <= (1e-3 if variant == "printed" else 1e-6)
    assert relmax(got, exact) <= (1e-3 if variant == "printed" else 1e-5)


def test_nonphysical_state_is_flagged():
    cfg = CASES["tgv3d_p2_3x2x4"]
    m = gpu_mesh(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    W[3, 0, 0] = -abs(W[3, 0, 0])          # negative density in one element
    R = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    m.residual(dev(W), R)
    assert m.status_sync() == 4            # DG_ERR_NONPHYSICAL
    assert m.status_sync() == B.DG_OK      # cleared


def test_invalid_arguments():
    cfg = CASES["vortex2d_p2_5x7"]
    m = gpu_mesh(cfg)
    W = dev(wl.perturbed_state(cfg))
    with pytest.raises(B.DGError):
        m.residual(W, W)                    # aliasing
    with pytest.raises(B.DGError):
        B.PMG(m, W, 1.0, B.pmg_opts((3, 1)))   # p_level[0] != mesh p


@pytest.mark.parametrize("name", ["tgv3d_p2_3x2x4", "vortex2d_p2_5x7", "tgv3d_p1_1x2x5"])
def test_blocks_parity(name):
    cfg = CASES[name]
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    sigma = 2.5
    pl = (cfg["p"], 1) if cfg["p"] > 1 else (cfg["p"], 0)
    D = oblocks.diag_blocks(om, oph, W, sigma)
    O = oblocks.offdiag_blocks(om, oph, W, pl[1])
    m = gpu_mesh(cfg)
    pmg = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=2, nu_post=2, nu_coarse=4))
    nb = om.nb
    Dinv = torch.empty((om.E, nb, nb), dtype=torch.float64, device="cuda")
    pmg.export_blocks(0, B.BLOCKS_DIAG_INV, Dinv)
    prod = np.einsum("eab,ebc->eac", Dinv.cpu().numpy(), D)
    assert np.abs(prod - np.eye(nb)[None]).max() <= 1e-10
    nbc = om.m * wl.n_modes(pl[1], om.d)
    Og = torch.empty((om.E, 2 * om.d, nbc, nbc), dtype=torch.float64, device="cuda")
    pmg.export_blocks(1, B.BLOCKS_NEIGHBOUR, Og)
    Oo = O.reshape(om.E, 2 * om.d, nbc, nbc)
    assert relmax(Og.cpu().numpy(), Oo) <= 1e-12


def _oracle_pmg(cfg, W, sigma, pl, nu, nuc):
    return osolvers.pmg_setup(oracle_mesh(cfg), oracle_physics(cfg), W, sigma, pl, nu_pre=nu, nu_post=nu,
                              nu_coarse=nuc)


@pytest.mark.parametrize("cycle", [B.CYCLE_FMG, B.CYCLE_V, B.CYCLE_BJ])
def test_pmg_apply_parity(cycle):
    cfg = CASES["tgv3d_p2_3x2x4"]
    W = wl.initial_state(cfg)
    sigma = 1.5 / wl.time_step(cfg)
    pl, nu, nuc = (2, 1, 0), 3, 5
    r = wl.random_vector(W.shape, 21)
    mg = _oracle_pmg(cfg, W, sigma, pl, nu, nuc)
    if cycle == B.CYCLE_FMG:
        ref = mg.mg_full(r)
    elif cycle == B.CYCLE_V:
        ref = mg.mg_v(0, r, np.zeros_like(r))
    else:
        ref = mg.P[0](r)
    m = gpu_mesh(cfg)
    pmg = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc, cycle=cycle))
    z = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    pmg.apply(dev(r), z)
    assert relmax(z.cpu().numpy(), ref) <= 1e-10


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_refresh_at_a_new_shift_matches_a_fresh_setup(precision):
    """dg_pmg_refresh with another sigma (an ESDIRK stage after a BDF2 setup):
    the captured application takes the new shift, bitwise as a fresh setup."""
    cfg = CASES["tgv3d_p2_3x2x4"]
    W0, W1 = wl.initial_state(cfg), wl.perturbed_state(cfg)
    s0 = 1.5 / wl.time_step(cfg)
    opts = B.pmg_opts((2, 1, 0), nu_pre=3, nu_post=3, nu_coarse=5, precision=precision)
    m = gpu_mesh(cfg)
    a = B.PMG(m, dev(W0), s0, opts)
    a.refresh(dev(W1), 2.5 * s0)
    b = B.PMG(m, dev(W1), 2.5 * s0, opts)
    r = dev(wl.random_vector(W0.shape, 23))
    za, zb = torch.empty_like(r), torch.empty_like(r)
    a.apply(r, za)
    b.apply(r, zb)
    assert m.status_sync() == B.DG_OK
    assert torch.equal(za, zb)
    if precision == B.PREC_FP64:
        ref = _oracle_pmg(cfg, W1, 2.5 * s0, (2, 1, 0), 3, 5).mg_full(wl.random_vector(W0.shape, 23))
        assert relmax(za.cpu().numpy(), ref) <= 1e-10


def _bdf2_problem(cfg):
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.initial_state(cfg)
    dt = wl.time_step(cfg)
    sigma = 1.5 / dt
    b = -o_residual(om, oph, W)           # W^{n-1} = W^n: f(W^n) = R(W^n)
    return om, oph, W, sigma, b


@pytest.mark.parametrize("name,pl", [("tgv3d_p2_3x2x4", (2, 1, 0)), ("vortex2d_p2_5x7", (2,))])
def test_fgmres_step_fp64_parity(name, pl):
    cfg = CASES[name]
    om, oph, W, sigma, b = _bdf2_problem(cfg)
    nu, nuc = 4, 8
    if len(pl) == 1:
        P = oblocks.BlockJacobi(oblocks.diag_blocks(om, oph, W, sigma), om.m, om.nm)
        cycle = B.CYCLE_BJ
    else:
        P = _oracle_pmg(cfg, W, sigma, pl, nu, nuc)
        cycle = B.CYCLE_FMG
    x_ref, st_ref = osolvers.fgmres(lambda z: o_jvp(om, oph, W, z, sigma), P, b, restart=30, rtol=1e-5,
                                    max_restarts=3)
    m = gpu_mesh(cfg)
    pmg = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc, cycle=cycle))
    dW = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    st = pmg.fgmres(dev(W), dev(b), dW, rtol=1e-5, max_restarts=3)
    assert abs(st["iters"] - st_ref["iters"]) <= 1
    x = dW.cpu().numpy()
    W1, W1_ref = W + x, W + x_ref
    assert np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref) <= 1e-10
    # the GPU result meets the tolerance on the oracle's own operator
    res = b - o_jvp(om, oph, W, x, sigma)
    assert np.linalg.norm(res) <= 1.0001e-5 * np.linalg.norm(b)


def test_fgmres_mixed_precision_vs_fp64_oracle():
    cfg = CASES["tgv3d_p4_3x3x3"]
    om, oph, W, sigma, b = _bdf2_problem(cfg)
    pl, nu, nuc = (4, 2, 1, 0), 10, 30
    P = _oracle_pmg(cfg, W, sigma, pl, nu, nuc)
    x_ref, st_ref = osolvers.fgmres(lambda z: o_jvp(om, oph, W, z, sigma), P, b, restart=30, rtol=1e-5)
    m = gpu_mesh(cfg)
    pmg = B.PMG(m, dev(W), sigma, B.pmg_opts(pl, nu_pre=nu, nu_post=nu, nu_coarse=nuc,
                                              precision=B.PREC_MIXED))
    dW = torch.empty(W.shape, dtype=torch.float64, device="cuda")
    st = pmg.fgmres(dev(W), dev(b), dW, rtol=1e-5)
    x = dW.cpu().numpy()
    W1, W1_ref = W + x, W + x_ref
    assert np.linalg.norm(W1 - W1_ref) / np.linalg.norm(W1_ref) <= 1e-6
    assert st["iters"] <= int(1.1 * st_ref["iters"]) + 1
    res = b - o_jvp(om, oph, W, x, sigma)
    assert np.linalg.norm(res) <= 1.0001e-5 * np.linalg.norm(b)


def test_mixed_apply_with_and_without_primal_cache(monkeypatch):
    """The mixed preconditioner's fine JVPs read the primal traces of W from a
    cache built at refresh; without it they interpolate W themselves.  The two
    pMG applications agree to FP32 rounding carried through ~60 smoother
    iterations: bar 1e-4 in the relative max-norm."""
    cfg = CASES["tgv3d_p4_3x3x3"]
    W = wl.initial_state(cfg)
    sigma = 1.5 / wl.time_step(cfg)
    r = dev(wl.random_vector(W.shape, 3))
    m = gpu_mesh(cfg)
    out = []
    for flag in ("0", "1"):
        monkeypatch.setenv("DG_PMG_NO_PRIMAL_CACHE", flag)
        pmg = B.PMG(m, dev(W), sigma, B.pmg_opts((4, 2, 1, 0), 10, 10, 30, precision=B.PREC_MIXED))
        z = torch.empty_like(r)
        pmg.apply(r, z)
        out.append(z.cpu().numpy())
        pmg.close()
    assert m.status_sync() == B.DG_OK
    err = relmax(out[0], out[1])
    print("cached vs interpolated primal: rel max %.3e" % err)
    assert err <= 1e-4


def test_repeat_calls_bitwise_identical():
    """Fixed-order reductions: two evaluations give the same bits (a race or an
    order-dependent sum would show here)."""
    cfg = CASES["tgv3d_p4_3x3x3"]
    m = gpu_mesh(cfg)
    W = dev(wl.perturbed_state(cfg, amp=0.05))
    v = dev(wl.random_vector(W.shape))
    a = torch.empty_like(W)
    b = torch.empty_like(W)
    m.jvp(W, v, a, 1.0)
    m.jvp(W, v, b, 1.0)
    assert torch.equal(a, b)
