"""Convergence pins of the oracle's time step and of its discrete solution.

* BDF2 (the workloads' time scheme; the Newton form of eq. NEWTON with the
  BDF2 shift 3/(2 dt)): ``oracle.solvers.bdf2_rhs`` driven by Newton reaches
  observed second order on scalar ODEs with a non-unit mass, and on the DG
  vortex against a fourth-order Runge-Kutta reference of the same
  semi-discrete system M dW/dt + R(W) = 0.
* Spatial accuracy (Sec. 7.1, the vortex convergence study): the DG solution
  of the inviscid vortex advected by the uniform stream, integrated in time
  with RK4 at a step far below the spatial error, converges to the translated
  closed form (L2-projected) at rate >= p + 1/2 in the L2 norm.
The RK4 integrator and the error norms are written here; only the residual and
the BDF2 right-hand side come from the oracle."""
import types

import numpy as np

from oracle import blocks, solvers
from oracle.dg import jvp, residual
from oracle.physics import Physics
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics


def _rates(errs):
    e = np.asarray(errs)
    return np.log2(e[:-1] / e[1:])


def _bdf2_scalar(R, dR, y0, ym1, dt, n, mass, newton):
    """n BDF2 steps of mass y' + R(y) = 0 with Newton on
    f = bdf2_rhs(...), K = 3/(2 dt) mass + dR/dy."""
    mesh = types.SimpleNamespace(detJ=mass)
    yn, ynm1 = np.array([y0]), np.array([ym1])
    for _ in range(n):
        yk = yn.copy()
        for _ in range(newton):
            f = solvers.bdf2_rhs(mesh, R(yk), yk, yn, ynm1, dt)
            yk = yk - f / (1.5 / dt * mass + dR(yk))
        ynm1, yn = yn, yk
    return yn[0]


def test_bdf2_second_order_on_linear_ode_with_mass():
    """c y' = c lam y (R = -c lam y, c = 2.5): error at t = 1 falls as dt^2."""
    lam, c = -1.3, 2.5
    errs = []
    for n in (10, 20, 40, 80):
        dt = 1.0 / n
        y = _bdf2_scalar(lambda y: -c * lam * y, lambda y: -c * lam, 1.0, np.exp(-lam * dt),
                         dt, n, c, newton=1)
        errs.append(abs(y - np.exp(lam)))
    r = _rates(errs)
    assert np.all(r > 1.9) and np.all(r < 2.1), (errs, r)


def test_bdf2_second_order_on_nonlinear_ode_with_mass():
    """c y' = -c y^2, y(0) = 1, y = 1/(1 + t): second order at t = 1."""
    c = 0.4
    errs = []
    for n in (8, 16, 32, 64):
        dt = 1.0 / n
        y = _bdf2_scalar(lambda y: c * y * y, lambda y: 2.0 * c * y, 1.0, 1.0 / (1.0 - dt),
                         dt, n, c, newton=8)
        errs.append(abs(y - 0.5))
    r = _rates(errs)
    assert np.all(r > 1.9) and np.all(r < 2.2), (errs, r)


def _rk4(mesh, ph, W, T, nsteps):
    """Classical RK4 on dW/dt = -M^{-1} R(W) with M = |J| I."""
    dt = T / nsteps
    f = lambda X: -residual(mesh, ph, X) / mesh.detJ
    for _ in range(nsteps):
        k1 = f(W)
        k2 = f(W + 0.5 * dt * k1)
        k3 = f(W + 0.5 * dt * k2)
        k4 = f(W + dt * k3)
        W = W + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return W


def _l2(mesh, X):
    """L2 norm of a modal field (orthonormal basis: |J| times the coefficient sum)."""
    return float(np.sqrt(mesh.detJ * np.sum(X * X)))


def test_bdf2_dg_vortex_second_order_in_time():
    """BDF2 on the viscous DG vortex (4 x 4 quads, p = 2, Re = 1000): W^{n-1}
    and the reference come from RK4 of the same semi-discrete system; each
    step takes three Newton iterations with FGMRES(BJ) solved to 1e-10, so the
    error at t = 0.4 is the time discretisation error alone, O(dt^2)."""
    cfg = wl.make_config("vortex", 2, (4, 4), 2, M=0.5, Re=1000.0)
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W0 = wl.project(cfg, lambda X: wl.vortex_field(X, cfg, beta=0.2, Rv=1.5))
    T = 0.4
    Wref = _rk4(mesh, ph, W0, T, 80)
    errs = []
    for n in (4, 8, 16):
        dt = T / n
        sigma = 1.5 / dt
        P = blocks.BlockJacobi(blocks.diag_blocks(mesh, ph, W0, sigma), mesh.m, mesh.nm)
        Wn, Wnm1 = W0, _rk4(mesh, ph, W0, -dt, 8)
        for _ in range(n):
            Wk = Wn.copy()
            for _ in range(3):
                f = solvers.bdf2_rhs(mesh, residual(mesh, ph, Wk), Wk, Wn, Wnm1, dt)
                x, st = solvers.fgmres(lambda z: jvp(mesh, ph, Wk, z, sigma), P, -f, rtol=1e-10,
                                       restart=40, max_restarts=3)
                assert st["converged"]
                Wk = Wk + x
            Wnm1, Wn = Wn, Wk
        errs.append(_l2(mesh, Wn - Wref))
    r = _rates(errs)
    assert np.all(r > 1.85) and np.all(r < 2.3), (errs, r)
    assert errs[-1] < 1e-4 * _l2(mesh, Wref)


def _vortex_solution_error(n, p, T=0.5):
    cfg = wl.make_config("vortex", 2, (n, n), p, M=0.5, Re=1e300)
    mesh, ph = oracle_mesh(cfg), Physics(mu=0.0)
    field = lambda t: (lambda X: wl.vortex_field(X, cfg, t=t, beta=0.2, Rv=1.0))
    W0 = wl.project(cfg, field(0.0))
    h = 10.0 / n
    nsteps = int(np.ceil(T / (0.2 * h / 1.8 / (2 * p + 1))))      # RK4 error << spatial
    WT = _rk4(mesh, ph, W0, T, nsteps)
    return _l2(mesh, WT - wl.project(cfg, field(T)))


def test_vortex_solution_converges_at_order_p_plus_one():
    """Inviscid vortex (beta = 0.2, R = 1 on [0, 10]^2, M = 0.5) advected for
    t = 0.5: L2 error against the translated closed form at rate >= p + 1/2
    (measured 1.76 for p = 1 on 16^2 -> 32^2, 2.97 for p = 2 on 8^2 -> 16^2)."""
    for p, ns in ((1, (16, 32)), (2, (8, 16))):
        errs = [_vortex_solution_error(n, p) for n in ns]
        r = _rates(errs)
        assert np.all(r >= p + 0.5), (p, errs, r)
