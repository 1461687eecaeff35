"""Pins of the oracle's ESDIRK3 step (Sec. 4): the tableau against the order
conditions and L-stability, the stage arithmetic against exact solutions of
scalar ODEs (observed third order), and the DG step's free-stream preservation."""
import numpy as np

from oracle import timestep as ts
from oracle import blocks as oblocks
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics, uniform_state


def test_tableau_order_conditions_and_structure():
    A, b, c = ts.A, ts.B, ts.C
    assert np.allclose(A[0], 0.0)                                   # explicit first stage
    assert np.allclose(np.diag(A)[1:], ts.GAMMA)                     # singly diagonal
    assert np.allclose(np.triu(A, 1), 0.0)
    assert abs(b.sum() - 1.0) < 1e-12                                # order 1
    assert abs(b @ c - 0.5) < 1e-12                                  # order 2
    assert abs(b @ c ** 2 - 1.0 / 3.0) < 1e-12                       # order 3
    assert abs(b @ (A @ c) - 1.0 / 6.0) < 1e-12
    # not fourth order (the scheme is third order)
    assert abs(b @ c ** 3 - 0.25) > 1e-6 or abs(b @ (A @ (A @ c)) - 1.0 / 24.0) > 1e-6


def test_gamma_is_the_l_stable_root_and_stability_decays():
    g = ts.GAMMA
    # third-order L-stable SDIRK-type diagonal: g^3 - 3 g^2 + 3/2 g - 1/6 = 0
    assert abs(g ** 3 - 3 * g ** 2 + 1.5 * g - 1.0 / 6.0) < 1e-12
    # stability function R(z) = 1 + z b^T (I - z A)^-1 1 tends to 0 as z -> -inf
    for z in (-1e4, -1e6, -1e8):
        Rz = 1.0 + z * ts.B @ np.linalg.solve(np.eye(4) - z * ts.A, np.ones(4))
        assert abs(Rz) < 10.0 / abs(z) ** 0.5
    # and matches exp(z) to O(z^4) near 0
    z = 1e-2
    Rz = 1.0 + z * ts.B @ np.linalg.solve(np.eye(4) - z * ts.A, np.ones(4))
    assert abs(Rz - np.exp(z)) < 1e-8


def _order(errors):
    return np.log2(errors[:-1] / errors[1:])


def test_third_order_on_linear_scalar_ode():
    lam = -1.0 + 2.0j
    errs = []
    for n in (10, 20, 40, 80):
        dt = 1.0 / n
        y = np.array([1.0 + 0.0j])
        for _ in range(n):
            y = ts.esdirk3_step(lambda w: -lam * w, lambda w, s, f: -f / (s - lam), y, dt, 1.0, newton=1)
        errs.append(abs(y[0] - np.exp(lam)))
    assert np.all(_order(np.array(errs)) > 2.85), errs


def test_third_order_on_nonlinear_scalar_ode():
    # y' = -y^2, y(0) = 1: y = 1/(1+t); R(y) = y^2, dR/dy = 2y
    errs = []
    for n in (8, 16, 32, 64):
        dt = 1.0 / n
        y = np.array([1.0])
        for _ in range(n):
            y = ts.esdirk3_step(lambda w: w * w, lambda w, s, f: -f / (s + 2.0 * w), y, dt, 1.0, newton=6)
        errs.append(abs(y[0] - 0.5))
    assert np.all(_order(np.array(errs)) > 2.85), errs


def test_dg_step_preserves_free_stream():
    cfg = wl.make_config("vortex", 2, (3, 2), 1, M=0.5, Re=1000.0)
    om, oph = oracle_mesh(cfg), oracle_physics(cfg)
    W = uniform_state(cfg)
    dt = wl.time_step(cfg)
    P = oblocks.BlockJacobi(oblocks.diag_blocks(om, oph, W, 1.0 / (ts.GAMMA * dt)), om.m, om.nm)
    W1, its = ts.esdirk3_dg_step(om, oph, W, dt, P, newton=1)
    assert np.abs(W1 - W).max() <= 1e-12 * np.abs(W).max()
