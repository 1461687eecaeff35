"""Pins of the oracle's DG residual and JVP (Sec. 3.1, Sec. 5.1) against
invariants, closed-form solutions, brute-force projections and finite
differences."""
import math

import numpy as np
import pytest

from oracle import basis
from oracle.dg import Mesh, residual, residual_parts, jvp, jvp_fd, lift_face, l2_project
from oracle.physics import Physics, flux_c, flux_v
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics, uniform_state, relmax

CASES = [
    wl.make_config("tgv", 3, (3, 2, 1), 2, M=0.3, Re=50.0),
    wl.make_config("tgv", 3, (2, 3, 3), 1, M=0.3, Re=50.0),
    wl.make_config("vortex", 2, (4, 3), 3, M=0.5, Re=100.0),
    wl.make_config("vortex", 2, (1, 2), 2, M=0.5, Re=100.0),
]


@pytest.mark.parametrize("cfg", CASES)
def test_free_stream_preservation(cfg):
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = uniform_state(cfg)
    R = residual(mesh, ph, W)
    assert np.abs(R).max() <= 1e-13 * np.abs(W).max()


@pytest.mark.parametrize("cfg", CASES)
def test_discrete_conservation(cfg):
    """sum_e R_e,v,mode0 = 0: each face flux enters its two elements with
    opposite signs (evaluated independently from both sides)."""
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    R = residual(mesh, ph, W)
    tot = R[:, :, 0].sum(axis=0)
    assert np.abs(tot).max() <= 1e-13 * np.abs(R).max() * mesh.E


def test_shift_equivariance():
    cfg = wl.make_config("tgv", 3, (3, 4, 2), 2, M=0.3, Re=50.0)
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    R = residual(mesh, ph, W)
    shift = mesh.nbr[:, 1, 1]                       # +y neighbour
    Rs = residual(mesh, ph, W[shift])
    np.testing.assert_allclose(Rs, R[shift], atol=1e-13 * np.abs(R).max())


def test_lifting_brute_force():
    """BR2 lifting against an explicit mass-matrix solve with a richer rule."""
    cfg = wl.make_config("tgv", 3, (2, 2, 2), 3, hi=(1.0, 2.0, 0.5))
    mesh = oracle_mesh(cfg)
    p, d = mesh.p, mesh.d
    nq = p + 4
    phi, _, wq, _ = basis.volume_tables(p, d, nq)
    Mbf = mesh.detJ * (phi.T @ (wq[:, None] * phi))
    rng = np.random.default_rng(11)
    for k in range(d):
        for s in (-1, 1):
            pf, _, wf = mesh.face[(k, s)]
            X = rng.standard_normal((2, len(wf)))
            rhs = 0.5 * mesh.faceJ[k] * ((X * wf) @ pf)         # 1/2 int_F phi_i X
            c = np.linalg.solve(Mbf, rhs.T).T
            brute = c @ pf.T
            np.testing.assert_allclose(lift_face(mesh, k, pf, wf, X), brute, atol=1e-13)


def test_steady_vortex_consistency_rate():
    """The isentropic vortex without the uniform stream is an exact steady Euler
    solution (Sec. 7.1 closed form: radial balance dp/dr = rho u_theta^2 / r);
    the DG residual of its projection vanishes as h -> 0 at order >= p."""
    g = 1.4
    beta, Rv = 0.2, 0.5

    def field(X):
        dx, dy = X[..., 0] - 5.0, X[..., 1] - 5.0
        r2 = (dx * dx + dy * dy) / Rv**2
        U = 0.5 * math.sqrt(g)
        u = -U * beta * dy / Rv * np.exp(-r2 / 2)
        v = U * beta * dx / Rv * np.exp(-r2 / 2)
        T = 1.0 - U * U * beta * beta / (2 * g / (g - 1)) * np.exp(-r2)
        rho = T ** (1 / (g - 1))
        return [rho, rho * u, rho * v, rho * T / (g - 1) + 0.5 * rho * (u * u + v * v)]
    errs = []
    p = 2
    for n in (8, 16, 32):
        cfg = wl.make_config("vortex", 2, (n, n), p)
        mesh = oracle_mesh(cfg)
        ph = Physics(gamma=g, mu=0.0, roe_delta=0.1)
        W = l2_project(mesh, field)
        R = residual(mesh, ph, W) / mesh.detJ
        errs.append(math.sqrt(mesh.detJ * np.sum(R * R)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] >= p - 0.3, (errs, rates)


def _mms_field(X, d, g=1.4, cplx=False):
    """Smooth periodic state on [0, 2 pi]^d and its gradient (closed form)."""
    x = [X[..., k] for k in range(d)]
    s = [np.sin(x[k]) for k in range(d)]
    c = [np.cos(x[k]) for k in range(d)]
    rho = 1.0 + 0.2 * s[0] * c[1]
    drho = [0.2 * c[0] * c[1], -0.2 * s[0] * s[1]] + [0 * x[0]] * (d - 2)
    vel = [0.3 * c[1], 0.2 * s[0]] + [0.1 * s[0] * c[1]] * (d - 2)
    dvel = [[0 * x[0], -0.3 * s[1]] + [0 * x[0]] * (d - 2),
            [0.2 * c[0], 0 * x[0]] + [0 * x[0]] * (d - 2)]
    if d == 3:
        dvel.append([0.1 * c[0] * c[1], -0.1 * s[0] * s[1], 0 * x[0]])
    p = 1.0 + 0.1 * c[0] * s[1]
    dp = [-0.1 * s[0] * s[1], 0.1 * c[0] * c[1]] + [0 * x[0]] * (d - 2)
    q2 = sum(v * v for v in vel)
    E = p / (g - 1) + 0.5 * rho * q2
    u = [rho] + [rho * v for v in vel] + [E]
    du = [drho]
    for j in range(d):
        du.append([drho[k] * vel[j] + rho * dvel[j][k] for k in range(d)])
    du.append([dp[k] / (g - 1) + 0.5 * drho[k] * q2 +
               rho * sum(vel[j] * dvel[j][k] for j in range(d)) for k in range(d)])
    return u, du


@pytest.mark.parametrize("p", [2, 3])
def test_viscous_consistency_rates(p):
    """Manufactured-solution defect of the viscous residual.  The source is the
    exact flux divergence div(F_c + F_v)(u*), by complex-step differentiation in
    x of the closed form (its gradient is analytic).  For R(Pi u*) - M Pi S:
    * strong (L2 of M^-1 R) defect: order p - 1 (a second-order operator);
    * weak defect against a smooth test function: order 2p, which holds only
      for a dual-consistent discretisation (the dual term of eq. dg_ns with the
      BR2 flux of eq. visc_flux); a wrong dual-term sign drops it to order p."""
    g = 1.4
    d = 2
    ph = Physics(gamma=g, Pr=0.72, mu=0.05, roe_delta=0.1)
    strong, weak = [], []
    for n in (4, 8, 16):
        cfg = wl.make_config("tgv", d, (n,) * d, p)
        mesh = oracle_mesh(cfg)

        def source(X):
            out = [0.0] * (d + 2)
            h = 1e-30
            for k in range(d):
                Xc = X.astype(np.complex128)
                Xc[..., k] += 1j * h
                u, du = _mms_field(Xc, d, g)
                F = flux_c(u, ph)
                Fv = flux_v(u, du, ph)
                for v in range(d + 2):
                    out[v] = out[v] + np.imag(F[v][k] + Fv[v][k]) / h
            return out
        W = l2_project(mesh, lambda X: _mms_field(X, d, g)[0])
        S = l2_project(mesh, source)
        psi = l2_project(mesh, lambda X: [np.sin(X[..., 0] + 0.3) * np.cos(X[..., 1])] * (d + 2))
        D = residual(mesh, ph, W) / mesh.detJ - S
        strong.append(math.sqrt(mesh.detJ * np.sum(D * D)))
        weak.append(abs(mesh.detJ * np.sum(D * psi)))
    rs = math.log2(strong[1] / strong[2])
    rw = math.log2(weak[1] / weak[2])
    assert rs >= p - 1 - 0.2, (strong, rs)
    assert rw >= 2 * p - 0.5, (weak, rw)


def test_linear_stability_at_rest():
    """Linearised about a state at rest, Roe upwinding plus BR2 with
    eta > n_faces give a semi-discrete operator M dW/dt = -J W with no growing
    mode: Re eig(M^-1 J) >= 0 (eq. visc_flux penalty requirement, Sec. 3.1)."""
    cfg = wl.make_config("tgv", 2, (3, 3), 1, hi=(1.0, 1.0, 1.0))
    mesh = oracle_mesh(cfg)
    ph = Physics(gamma=1.4, Pr=0.72, mu=0.05, roe_delta=0.1)
    W = uniform_state(cfg, vel=(0.0, 0.0, 0.0))
    N = W.size
    J = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        J[:, j] = jvp(mesh, ph, W, e.reshape(W.shape), 0.0).reshape(-1)
    lam = np.linalg.eigvals(J / mesh.detJ)
    assert lam.real.min() >= -1e-9 * np.abs(lam).max(), lam.real.min()


@pytest.mark.parametrize("cfg", CASES[:3])
def test_jvp_complex_step_vs_fd(cfg):
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    sigma = 3.0
    Kv = jvp(mesh, ph, W, v, sigma)
    e = 1e-6
    fd = sigma * mesh.detJ * v + (residual(mesh, ph, W + e * v) - residual(mesh, ph, W - e * v)) / (2 * e)
    assert relmax(Kv, fd) < 1e-8


def test_jvp_free_stream_uniform_direction():
    """R(W + eps v) = 0 for uniform W and a uniform (mode-0) v, so K v = sigma M v."""
    cfg = CASES[0]
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = uniform_state(cfg)
    v = np.zeros_like(W)
    v[:, :, 0] = np.array([0.1, -0.2, 0.3, 0.05, 0.4])[None, :]
    Kv = jvp(mesh, ph, W, v, 2.5)
    np.testing.assert_allclose(Kv, 2.5 * mesh.detJ * v, atol=1e-13)


def test_jvp_linearity():
    cfg = CASES[2]
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape, 1)
    w = wl.random_vector(W.shape, 2)
    a = -1.7
    lhs = jvp(mesh, ph, W, a * v + w, 1.0)
    rhs = a * jvp(mesh, ph, W, v, 1.0) + jvp(mesh, ph, W, w, 1.0)
    assert relmax(lhs, rhs) < 1e-13


@pytest.mark.parametrize("variant,tol", [("printed", 1e-3), ("scaled", 1e-5)])
def test_jvp_fd_mode(variant, tol):
    cfg = CASES[2]
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    RW = residual(mesh, ph, W)
    ex = jvp(mesh, ph, W, v, 1.0)
    fd = jvp_fd(mesh, ph, W, RW, v, 1.0, variant=variant)
    assert relmax(fd, ex) < tol


def test_element_subset_matches_full():
    cfg = CASES[1]
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    R = residual(mesh, ph, W)
    sub = np.array([4, 0, 7])
    np.testing.assert_allclose(residual(mesh, ph, W, elems=sub), R[sub], atol=0)


Q_CASES = [
    wl.make_config("tgv", 3, (3, 2, 2), 2, M=0.3, Re=50.0, space="Q"),
    wl.make_config("vortex", 2, (4, 3), 3, M=0.5, Re=100.0, space="Q"),
]


@pytest.mark.parametrize("cfg", Q_CASES)
def test_tensor_basis_free_stream_and_conservation(cfg):
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    assert mesh.nm == (cfg["p"] + 1) ** cfg["dim"]
    W = uniform_state(cfg)
    assert np.abs(residual(mesh, ph, W)).max() <= 1e-13 * np.abs(W).max()
    W = wl.perturbed_state(cfg, amp=0.05)
    R = residual(mesh, ph, W)
    assert np.abs(R[:, :, 0].sum(axis=0)).max() <= 1e-13 * np.abs(R).max() * mesh.E


def test_tensor_basis_contains_total_degree_solution():
    """P_p is a subspace of Q_p: for the inviscid residual (mu = 0: no BR2
    lifting, whose projection space differs between the two bases, eq. re) a
    state with only total-degree-<= p modes has the same residual on those
    modes in either basis."""
    cfg_p = wl.make_config("vortex", 2, (3, 3), 2, M=0.5, Re=100.0)
    cfg_q = dict(cfg_p, space="Q")
    mp, mq = oracle_mesh(cfg_p), oracle_mesh(cfg_q)
    ph = Physics(gamma=1.4, mu=0.0, roe_delta=0.1)
    Wp = wl.perturbed_state(cfg_p, amp=0.05)
    mdp, mdq = basis.modes(2, 2), basis.modes(2, 2, "Q")
    idx = [mdq.index(a) for a in mdp]
    Wq = np.zeros((mp.E, mp.m, mq.nm))
    Wq[:, :, idx] = Wp
    Rp, Rq = residual(mp, ph, Wp), residual(mq, ph, Wq)
    assert relmax(Rq[:, :, idx], Rp) <= 1e-12


def test_tensor_basis_steady_vortex_rate_and_jvp():
    g = 1.4
    beta, Rv = 0.2, 0.5

    def field(X):
        dx, dy = X[..., 0] - 5.0, X[..., 1] - 5.0
        r2 = (dx * dx + dy * dy) / Rv**2
        U = 0.5 * math.sqrt(g)
        u = -U * beta * dy / Rv * np.exp(-r2 / 2)
        v = U * beta * dx / Rv * np.exp(-r2 / 2)
        T = 1.0 - U * U * beta * beta / (2 * g / (g - 1)) * np.exp(-r2)
        rho = T ** (1 / (g - 1))
        return [rho, rho * u, rho * v, rho * T / (g - 1) + 0.5 * rho * (u * u + v * v)]
    errs = []
    p = 2
    for n in (8, 16, 32):
        cfg = wl.make_config("vortex", 2, (n, n), p, space="Q")
        mesh = oracle_mesh(cfg)
        ph = Physics(gamma=g, mu=0.0, roe_delta=0.1)
        W = l2_project(mesh, field)
        R = residual(mesh, ph, W) / mesh.detJ
        errs.append(math.sqrt(mesh.detJ * np.sum(R * R)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] >= p - 0.3, (errs, rates)
    cfg = Q_CASES[1]
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.perturbed_state(cfg, amp=0.05)
    v = wl.random_vector(W.shape)
    h = 1e-6
    fd = (residual(mesh, ph, W + h * v) - residual(mesh, ph, W - h * v)) / (2 * h)
    assert relmax(jvp(mesh, ph, W, v, 0.0), fd) <= 1e-7
