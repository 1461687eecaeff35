"""Pins of the oracle's triangular DG (Sec. 3: full-order P_p on triangles):
Jacobi polynomials against scipy, orthonormality and hierarchy of the Dubiner
basis, exactness of the collapsed rule against the simplex integral formula,
reference derivatives against differences and the divergence theorem, mesh
connectivity and edge geometry, free stream, conservation, steady-vortex and
manufactured-solution (dual consistency) rates on jittered meshes, linear
stability, the complex-step JVP, and blocks rebuilding the JVP."""
import math

import numpy as np
import pytest

from oracle import tri
from oracle.blocks import BlockJacobi
from oracle.physics import Physics, flux_c, flux_v
from oracle.solvers import fgmres
from paper_1812_04789_gb300 import workloads as wl
from tests.test_oracle_dg import _mms_field


def tri_mesh(cfg, nq1d=None):
    m = wl.tri_mesh(cfg)
    return tri.TriMesh(m["X"], m["tri"], m["shift"], m["lo"], m["hi"], cfg["p"], nq1d)


def tri_phys(cfg, **kw):
    P = wl.tri_physics(cfg, **kw)
    return Physics(gamma=P["gamma"], Pr=P["Pr"], mu=P["mu"], Rgas=P["Rgas"], eta=P["eta"],
                   roe_delta=P["roe_delta"])


def uniform(cfg, rho=1.0, vel=(0.3, -0.2), p=1.0, g=1.4):
    W = np.zeros(wl.tri_state_shape(cfg))
    c0 = math.sqrt(2.0)                     # psi_0 = 1/sqrt(2) on the reference triangle (area 2)
    W[:, 0, 0] = rho * c0
    W[:, 1, 0] = rho * vel[0] * c0
    W[:, 2, 0] = rho * vel[1] * c0
    W[:, 3, 0] = (p / (g - 1.0) + 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2)) * c0
    return W


def test_jacobi_matches_scipy():
    from scipy.special import eval_jacobi
    x = np.linspace(-0.97, 0.99, 23)
    for alpha in (0, 1, 3, 7):
        P = tri.jacobi(7, alpha, x)
        for n in range(8):
            assert np.abs(P[n] - eval_jacobi(n, alpha, 0, x)).max() < 1e-12 * max(1.0, np.abs(P[n]).max())


@pytest.mark.parametrize("p", [1, 3, 6])
def test_dubiner_orthonormal_and_hierarchical(p):
    phi, dphi, wq, xi = tri.volume_tables(p, p + 2)
    G = (phi * wq[:, None]).T @ phi
    assert np.abs(G - np.eye(tri.n_modes_tri(p))).max() < 1e-12
    r, s = xi[:, 0], xi[:, 1]
    for q in range(p + 1):
        n = tri.n_modes_tri(q)
        # monomials of degree <= q lie in the span of the first n_m(q) modes ...
        for a in range(q + 1):
            for b in range(q + 1 - a):
                f = r ** a * s ** b
                c = (f * wq) @ phi[:, :n]
                assert np.abs(phi[:, :n] @ c - f).max() < 1e-11
        # ... and one of degree q + 1 does not
        if q < p:
            f = r ** (q + 1)
            c = (f * wq) @ phi[:, :n]
            assert np.abs(phi[:, :n] @ c - f).max() > 1e-3


def test_collapsed_rule_is_exact_to_degree_2n_minus_2():
    for nq in (2, 4, 6):
        r, s, w = tri.tri_rule(nq)
        assert abs(w.sum() - 2.0) < 1e-14
        for a in range(2 * nq - 1):
            for b in range(2 * nq - 1 - a):
                exact = 2.0 ** (a + b + 2) * math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
                got = np.sum(w * (1.0 + r) ** a * (1.0 + s) ** b)
                assert abs(got - exact) < 1e-13 * max(1.0, exact), (nq, a, b)


def test_reference_derivatives_and_divergence_theorem():
    p = 4
    phi, dphi, wq, xi = tri.volume_tables(p, p + 2)
    h = 1e-6
    r, s = xi[:, 0], xi[:, 1]
    fd_r = (tri.dubiner(p, r + h, s) - tri.dubiner(p, r - h, s)).T / (2 * h)
    fd_s = (tri.dubiner(p, r, s + h) - tri.dubiner(p, r, s - h)).T / (2 * h)
    assert np.abs(dphi[0] - fd_r).max() < 1e-7 and np.abs(dphi[1] - fd_s).max() < 1e-7
    # int_T d psi / d xi_k = sum over edges int_e psi n_k ds (reference normals)
    lhs = [(dphi[k] * wq[:, None]).sum(axis=0) for k in range(2)]
    rhs = [np.zeros(tri.n_modes_tri(p)) for _ in range(2)]
    for f, (a, b) in enumerate(tri.REF_EDGES):
        ph_e, _, we, _ = tri.edge_tables(p, p + 2, f)
        dv = tri.REF_VERTS[b] - tri.REF_VERTS[a]
        L = float(np.hypot(*dv))
        n = np.array([dv[1], -dv[0]]) / L
        for k in range(2):
            rhs[k] += n[k] * (L / 2.0) * (ph_e * we[:, None]).sum(axis=0)
    for k in range(2):
        assert np.abs(lhs[k] - rhs[k]).max() < 1e-12


@pytest.mark.parametrize("n", [(4, 3), (2, 2), (5, 6)])
def test_mesh_connectivity_and_edge_geometry(n):
    cfg = wl.tri_config(n, 2)
    M = tri_mesh(cfg)
    assert M.E == 2 * n[0] * n[1]
    assert abs(M.detJ.sum() * 2.0 - np.prod(M.Lbox)) < 1e-11 * np.prod(M.Lbox)
    E = np.arange(M.E)
    for f in range(3):
        nb, fn = M.nbr[:, f], M.nbr_f[:, f]
        assert np.all(M.nbr[nb, fn] == E) and np.all(M.nbr_f[nb, fn] == f)
        assert np.abs(M.elen[nb, fn] - M.elen[:, f]).max() < 1e-12
        assert np.abs(M.normal[nb, fn] + M.normal[:, f]).max() < 1e-12
        # the edge points seen from both sides coincide up to a lattice period
        _, _, _, pts = M.edge[f]
        XP = M.vol_points(pts)
        for e in range(M.E):
            _, _, _, ptn = M.edge[fn[e]]
            XM = M.vol_points(ptn[::-1])[nb[e]]
            d = (XP[e] - XM) / M.Lbox
            assert np.abs(d - np.round(d)).max() < 1e-12


def test_free_stream_and_conservation():
    cfg = wl.tri_config((5, 4), 3)
    M, ph = tri_mesh(cfg), tri_phys(cfg)
    W = uniform(cfg)
    assert np.abs(tri.residual(M, ph, W)).max() < 1e-13 * np.abs(W).max()
    W = wl.tri_perturbed_state(cfg, amp=0.05)
    R = tri.residual(M, ph, W)
    assert np.abs(R[:, :, 0].sum(axis=0)).max() < 1e-13 * np.abs(R).max()


def test_steady_vortex_consistency_rate():
    """The vortex without a uniform stream is an exact steady Euler solution; on
    jittered triangles the residual of its projection vanishes at order >= p."""
    g, beta, Rv = 1.4, 0.2, 0.5

    def field(X):
        dx, dy = X[..., 0] - 5.0, X[..., 1] - 5.0
        r2 = (dx * dx + dy * dy) / Rv ** 2
        U = 0.5 * math.sqrt(g)
        u = -U * beta * dy / Rv * np.exp(-r2 / 2)
        v = U * beta * dx / Rv * np.exp(-r2 / 2)
        T = 1.0 - U * U * beta * beta / (2 * g / (g - 1)) * np.exp(-r2)
        rho = T ** (1 / (g - 1))
        return [rho, rho * u, rho * v, rho * T / (g - 1) + 0.5 * rho * (u * u + v * v)]
    p, errs = 2, []
    for n in (8, 16, 32):
        cfg = wl.tri_config((n, n), p)
        M = tri_mesh(cfg)
        ph = Physics(gamma=g, mu=0.0, roe_delta=0.1, eta=4.0)
        R = tri.residual(M, ph, tri.l2_project(M, field)) / M.detJ[:, None, None]
        errs.append(math.sqrt(np.sum(M.detJ[:, None, None] * R * R)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] >= p - 0.3, (errs, rates)


@pytest.mark.parametrize("p", [2, 3])
def test_viscous_manufactured_rates(p):
    """Strong defect order p - 1 and weak defect order 2p (dual consistency of
    the BR2 discretisation, eq. dg_ns / visc_flux) on jittered triangles."""
    g = 1.4
    ph = Physics(gamma=g, Pr=0.72, mu=0.05, roe_delta=0.1, eta=4.0)
    strong, weak = [], []
    for n in (4, 8, 16):
        cfg = wl.tri_config((n, n), p, lo=(0.0, 0.0), hi=(2 * math.pi, 2 * math.pi))
        M = tri_mesh(cfg)

        def source(X):
            out = [0.0] * 4
            for k in range(2):
                Xc = X.astype(np.complex128)
                Xc[..., k] += 1e-30j
                u, du = _mms_field(Xc, 2, g)
                F, Fv = flux_c(u, ph), flux_v(u, du, ph)
                for v in range(4):
                    out[v] = out[v] + np.imag(F[v][k] + Fv[v][k]) / 1e-30
            return out
        W = tri.l2_project(M, lambda X: _mms_field(X, 2, g)[0])
        S = tri.l2_project(M, source)
        psi = tri.l2_project(M, lambda X: [np.sin(X[..., 0] + 0.3) * np.cos(X[..., 1])] * 4)
        D = tri.residual(M, ph, W) / M.detJ[:, None, None] - S
        strong.append(math.sqrt(np.sum(M.detJ[:, None, None] * D * D)))
        weak.append(abs(np.sum(M.detJ[:, None, None] * D * psi)))
    rs = math.log2(strong[1] / strong[2])
    rw = math.log2(weak[1] / weak[2])
    assert rs >= p - 1 - 0.3, (strong, rs)
    assert rw >= 2 * p - 0.6, (weak, rw)


def test_linear_stability_at_rest():
    cfg = wl.tri_config((2, 2), 1, hi=(1.0, 1.0))
    M = tri_mesh(cfg)
    ph = Physics(gamma=1.4, Pr=0.72, mu=0.05, roe_delta=0.1, eta=4.0)
    W = uniform(cfg, vel=(0.0, 0.0))
    N = W.size
    J = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        J[:, j] = tri.jvp(M, ph, W, e.reshape(W.shape), 0.0).reshape(-1)
    Minv = np.repeat(1.0 / M.detJ, 4 * M.nm)
    lam = np.linalg.eigvals(Minv[:, None] * J)
    assert lam.real.min() >= -1e-9 * np.abs(lam).max(), lam.real.min()


def test_jvp_complex_step_vs_fd():
    cfg = wl.tri_config((3, 4), 2)
    M, ph = tri_mesh(cfg), tri_phys(cfg)
    W = wl.tri_perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    Kv = tri.jvp(M, ph, W, v, 3.0)
    e = 1e-6
    fd = 3.0 * M.detJ[:, None, None] * v + (tri.residual(M, ph, W + e * v) - tri.residual(M, ph, W - e * v)) / (2 * e)
    assert np.abs(Kv - fd).max() < 1e-8 * np.abs(fd).max()


def test_blocks_rebuild_the_jvp_and_pmg_converges():
    cfg = wl.tri_config((3, 4), 2)
    M, ph = tri_mesh(cfg), tri_phys(cfg)
    W = wl.tri_perturbed_state(cfg, amp=0.05)
    sigma = 5.0
    D = tri.diag_blocks(M, ph, W, sigma)
    O = tri.offdiag_blocks(M, ph, W, cfg["p"])
    v = wl.random_vector(W.shape)
    Kv = tri.jvp(M, ph, W, v, sigma)
    assert np.abs(tri.bsr_apply(M, D, O, v) - Kv).max() < 1e-12 * np.abs(Kv).max()
    # block Jacobi, then p-multigrid, as FGMRES preconditioners of K
    K = lambda x: tri.jvp(M, ph, W, x, sigma)
    b = wl.random_vector(W.shape, 5)
    _, st_bj = fgmres(K, BlockJacobi(D, 4, M.nm), b, restart=30, rtol=1e-8, max_restarts=3)
    mg = tri.pmg_setup(M, ph, W, sigma, (2, 1, 0), nu_pre=3, nu_post=3, nu_coarse=8)
    x, st_mg = fgmres(K, mg, b, restart=30, rtol=1e-8, max_restarts=3)
    assert st_bj["converged"] and st_mg["converged"]
    assert st_mg["iters"] < st_bj["iters"]
    assert np.linalg.norm(b - K(x)) <= 1.0001e-8 * np.linalg.norm(b)


def test_esdirk3_step_on_triangles():
    """The ESDIRK3 step (Sec. 4) with the per-triangle mass: a uniform state
    stays put, and on the vortex successive halvings of the step change the
    state by amounts that shrink ~8x (third order)."""
    from oracle import timestep as ts
    cfg = wl.tri_config((3, 3), 1, Re=1.0e4)
    M, ph = tri_mesh(cfg), tri_phys(cfg)
    W = uniform(cfg)
    dt = wl.time_step(cfg)
    P = BlockJacobi(tri.diag_blocks(M, ph, W, 1.0 / (ts.GAMMA * dt)), 4, M.nm)
    W1, _ = ts.esdirk3_dg_step(M, ph, W, dt, P, newton=1)
    assert np.abs(W1 - W).max() <= 1e-12 * np.abs(W).max()
    W0 = wl.tri_initial_state(cfg)

    def run(h, n):
        Wc = W0.copy()
        Pc = BlockJacobi(tri.diag_blocks(M, ph, Wc, 1.0 / (ts.GAMMA * h)), 4, M.nm)   # lagged: any P converges
        for _ in range(n):
            Wc, _ = ts.esdirk3_dg_step(M, ph, Wc, h, Pc, newton=3, rtol=1e-12, max_restarts=8)
        return Wc
    T = 0.4
    w1, w2, w4 = run(T, 1), run(T / 2, 2), run(T / 4, 4)
    d1, d2 = np.abs(w1 - w2).max(), np.abs(w2 - w4).max()
    assert d1 / d2 > 5.0, (d1, d2)
