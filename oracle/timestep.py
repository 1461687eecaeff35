"""ESDIRK3 time step with Newton-Krylov stages (Sec. 4, eq. NEWTON; Sec. 7.4
for lagging the preconditioner over the whole step).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Scheme: the four-stage, third-order, explicit-first-stage, singly diagonally
implicit, stiffly accurate Runge-Kutta method the paper uses (Bijl et al.
2002): Kennedy & Carpenter's ESDIRK3(2)4L[2]SA, coefficients as published
(rational forms).  For M dW/dt + R(W) = 0, stage i solves
  M (W^i - W^n) / (a_ii dt) + sum_{j<i} (a_ij / a_ii) R(W^j) + R(W^i) = 0
by Newton iterations with K = M / (a_ii dt) + dR/dW (eq. NEWTON); stage 1 is
W^1 = W^n, and the step returns the last stage (stiffly accurate, b = last row
of A; the printed update line of the scheme is read this way).
"""
import numpy as np

GAMMA = 1767732205903.0 / 4055673282236.0
A = np.array([
    [0.0, 0.0, 0.0, 0.0],
    [GAMMA, GAMMA, 0.0, 0.0],
    [2746238789719.0 / 10658868560708.0, -640167445237.0 / 6845629431997.0, GAMMA, 0.0],
    [1471266399579.0 / 7840856788654.0, -4482444167858.0 / 7529755066697.0,
     11266239266428.0 / 11593286722821.0, GAMMA],
])
B = A[3].copy()
C = A.sum(axis=1)


def esdirk3_step(R, solve, Wn, dt, mass, newton=2):
    """One ESDIRK3 step of mass dW/dt + R(W) = 0.

    R(W): residual; solve(Wk, sigma, f) returns dW with K(Wk) dW = -f,
    K = sigma mass + dR/dW(Wk), sigma = 1 / (a_ii dt) (the same for every
    implicit stage); mass: |J| of M = |J| I, a scalar or an array broadcast
    against W (one |J| per element), or 1 for an ODE.
    Each implicit stage starts from the previous stage's value and takes
    `newton` Newton iterations (eq. NEWTON); R of stages 1..3 is kept for the
    sums of the later stages."""
    sigma = 1.0 / (A[1, 1] * dt)
    Rs = [R(Wn)]
    Wk = np.array(Wn, copy=True)
    for i in range(1, 4):
        racc = sum(A[i, j] / A[i, i] * Rs[j] for j in range(i))
        for _ in range(newton):
            f = sigma * mass * (Wk - Wn) + racc + R(Wk)
            Wk = Wk + solve(Wk, sigma, f)
        if i < 3:
            Rs.append(R(Wk))
    return Wk


def esdirk3_dg_step(mesh, ph, Wn, dt, P, newton=2, rtol=1e-5, max_restarts=4):
    """ESDIRK3 step of the DG system with FGMRES (exact JVP) preconditioned by
    P, assembled once at W^n with sigma = 1/(a_ii dt) and reused for every stage
    and Newton iteration (Sec. 7.4, "MFL").  Returns (W^{n+1}, FGMRES iteration
    counts per solve).  A triangle mesh (``oracle.tri.TriMesh``) takes its own
    residual, JVP and per-triangle mass |J_e|."""
    from . import dg, tri
    from .solvers import fgmres
    if isinstance(mesh, tri.TriMesh):
        residual, jvp, mass = tri.residual, tri.jvp, mesh.detJ[:, None, None]
    else:
        residual, jvp, mass = dg.residual, dg.jvp, mesh.detJ
    its = []

    def solve(Wk, sigma, f):
        x, st = fgmres(lambda z: jvp(mesh, ph, Wk, z, sigma), P, -f, rtol=rtol, max_restarts=max_restarts)
        its.append(st["iters"])
        return x

    W1 = esdirk3_step(lambda W: residual(mesh, ph, W), solve, Wn, dt, mass, newton)
    return W1, its
