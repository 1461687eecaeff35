"""Compressible Navier-Stokes fluxes (Sec. 2, eq. NS; Sec. 3.1, eqs. PDE, dg_ns).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Every function works on real or complex numpy arrays (the oracle's exact JVP is
a complex step), so branches compare real parts and |x| is the analytic
continuation cabs(x) = x if Re x >= 0 else -x.

Layout: a state is u[v] for v = 0..m-1 (rho, rho*v_1..rho*v_d, rho*e0), each an
array of any shape; a gradient or flux tensor is g[v][k], k = 0..d-1.

Closure (Sec. 2): p = (gamma-1) rho e, e0 = e + |v|^2/2, h0 = e0 + p/rho,
tau = 2 mu (S - (div v)/3 I), q = -(mu/Pr) grad h, h = c_p T, p = rho R T,
c_p = gamma R/(gamma-1) (as in the vortex test case, Sec. 7.1).  mu is constant.
"""
import numpy as np


class Physics:
    """gamma, Pr, mu, Rgas, eta (BR2 penalty, eq. visc_flux) and the Roe
    entropy-fix fraction roe_delta (0 = plain Roe)."""

    def __init__(self, gamma=1.4, Pr=0.72, mu=0.0, Rgas=1.0, eta=None, roe_delta=0.1):
        self.gamma, self.Pr, self.mu, self.Rgas = gamma, Pr, mu, Rgas
        self.eta = eta
        self.roe_delta = roe_delta

    def eta_for(self, d):
        """BR2 penalty: must exceed the number of element faces (Sec. 3.1);
        default n_faces + 1."""
        return float(2 * d + 1) if self.eta is None else float(self.eta)


def cabs(x):
    """|x| continued analytically for the complex step (Re x >= 0 -> x)."""
    return np.where(np.real(x) >= 0, x, -x)


def primitives(u, ph):
    """rho, velocity list, specific total energy e0, pressure p, temperature T,
    total enthalpy h0 (Sec. 2 closure)."""
    m = len(u)
    d = m - 2
    rho = u[0]
    vel = [u[1 + j] / rho for j in range(d)]
    e0 = u[m - 1] / rho
    q2 = sum(v * v for v in vel)
    p = (ph.gamma - 1.0) * (u[m - 1] - 0.5 * rho * q2)
    T = p / (rho * ph.Rgas)
    h0 = e0 + p / rho
    return rho, vel, e0, p, T, h0


def flux_c(u, ph):
    """Inviscid flux F_c[v][k] = (rho v_k, rho v_j v_k + p delta_jk, rho v_k h0)
    (eq. NS left-hand sides)."""
    m = len(u)
    d = m - 2
    rho, vel, e0, p, T, h0 = primitives(u, ph)
    F = [[None] * d for _ in range(m)]
    for k in range(d):
        F[0][k] = u[1 + k]
        for j in range(d):
            F[1 + j][k] = u[1 + j] * vel[k] + (p if j == k else 0.0 * p)
        F[m - 1][k] = rho * vel[k] * h0
    return F


def flux_v(u, g, ph):
    """Viscous flux F_v[v][k] with the sign of eq. PDE (u_t + div F_c + div F_v = 0):
    F_v = -(0, tau, v.tau - q).  g[v][k] is the gradient of the conservative
    variables (or any tensor of that shape: F_v is linear in it).

    Primitive gradients from conservative ones:
      grad v_j = (g[1+j] - v_j g[0]) / rho,  grad e0 = (g[m-1] - e0 g[0]) / rho,
      grad T = (gamma-1)/R (grad e0 - sum_j v_j grad v_j).
    """
    m = len(u)
    d = m - 2
    rho, vel, e0, p, T, h0 = primitives(u, ph)
    gv = [[(g[1 + j][k] - vel[j] * g[0][k]) / rho for k in range(d)] for j in range(d)]
    ge = [(g[m - 1][k] - e0 * g[0][k]) / rho for k in range(d)]
    gT = [(ph.gamma - 1.0) / ph.Rgas * (ge[k] - sum(vel[j] * gv[j][k] for j in range(d)))
          for k in range(d)]
    div = sum(gv[j][j] for j in range(d))
    mu = ph.mu
    tau = [[mu * (gv[j][k] + gv[k][j]) - ((2.0 / 3.0) * mu * div if j == k else 0.0)
            for k in range(d)] for j in range(d)]
    kappa = mu * ph.gamma * ph.Rgas / ((ph.gamma - 1.0) * ph.Pr)      # mu c_p / Pr
    qh = [-kappa * gT[k] for k in range(d)]                            # heat flux q
    F = [[None] * d for _ in range(m)]
    for k in range(d):
        F[0][k] = 0.0 * rho
        for j in range(d):
            F[1 + j][k] = -tau[j][k]
        F[m - 1][k] = -(sum(vel[j] * tau[j][k] for j in range(d)) - qh[k])
    return F


def visc_K(u, g, ph):
    """(K . g) with F_v(u, grad u) = -K grad u (Sec. 3.1): K(u) applied to a
    gradient-shaped tensor g, i.e. -F_v(u, g)."""
    F = flux_v(u, g, ph)
    return [[-F[v][k] for k in range(len(F[0]))] for v in range(len(F))]


def entropy_fix(lam, delta):
    """|lam| with Harten's smoothing (lam^2 + delta^2)/(2 delta) for |lam| < delta
    (a reading: the paper names plain Roe; delta = 0 gives plain |lam|)."""
    a = cabs(lam)
    if np.all(np.real(delta) == 0):
        return a
    dsafe = np.where(np.real(delta) > 0, delta, 1.0)
    return np.where(np.real(a) < np.real(delta), (lam * lam + delta * delta) / (2.0 * dsafe), a)


def roe_dissipation(uL, uR, n, ph, absfn=None):
    """|A_Roe(uL, uR; n)| (uR - uL) by the Roe-average wave decomposition.

    Roe averages: sqrt(rho)-weighted velocity and total enthalpy, rho_hat =
    sqrt(rhoL rhoR), c^2 = (gamma-1)(h0_hat - |v_hat|^2/2).  Waves with speeds
    v_n - c, v_n (d-fold: entropy + shear), v_n + c.  absfn maps a speed to its
    modulus (default: entropy_fix with delta = roe_delta * c); passing the
    identity gives A_Roe (uR - uL), which must equal F_c(uR).n - F_c(uL).n.
    """
    m = len(uL)
    d = m - 2
    rL, vL, eL, pL, TL, hL = primitives(uL, ph)
    rR, vR, eR, pR, TR, hR = primitives(uR, ph)
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    rho = sL * sR
    vel = [(sL * vL[j] + sR * vR[j]) / (sL + sR) for j in range(d)]
    h0 = (sL * hL + sR * hR) / (sL + sR)
    q2 = sum(v * v for v in vel)
    c2 = (ph.gamma - 1.0) * (h0 - 0.5 * q2)
    c = np.sqrt(c2)
    vn = sum(vel[j] * n[j] for j in range(d))
    dr = rR - rL
    dp = pR - pL
    dv = [vR[j] - vL[j] for j in range(d)]
    dvn = sum(dv[j] * n[j] for j in range(d))
    a1 = (dp - rho * c * dvn) / (2.0 * c2)
    a3 = (dp + rho * c * dvn) / (2.0 * c2)
    a2 = dr - dp / c2
    if absfn is None:
        delta = ph.roe_delta * c
        absfn = lambda lam: entropy_fix(lam, delta)
    l1, l2, l3 = absfn(vn - c), absfn(vn), absfn(vn + c)
    out = [None] * m
    # acoustic waves
    out[0] = l1 * a1 + l3 * a3
    for j in range(d):
        out[1 + j] = l1 * a1 * (vel[j] - c * n[j]) + l3 * a3 * (vel[j] + c * n[j])
    out[m - 1] = l1 * a1 * (h0 - c * vn) + l3 * a3 * (h0 + c * vn)
    # entropy + shear waves
    out[0] = out[0] + l2 * a2
    for j in range(d):
        out[1 + j] = out[1 + j] + l2 * (a2 * vel[j] + rho * (dv[j] - dvn * n[j]))
    vdv = sum(vel[j] * dv[j] for j in range(d))
    out[m - 1] = out[m - 1] + l2 * (a2 * 0.5 * q2 + rho * (vdv - vn * dvn))
    return out


def roe_flux(uL, uR, n, ph, absfn=None):
    """Roe numerical flux (Sec. 3.1): 1/2 (F_c(uL) + F_c(uR)).n - 1/2 |A|(uR - uL)."""
    d = len(uL) - 2
    FL = flux_c(uL, ph)
    FR = flux_c(uR, ph)
    D = roe_dissipation(uL, uR, n, ph, absfn)
    return [0.5 * sum((FL[v][k] + FR[v][k]) * n[k] for k in range(d)) - 0.5 * D[v]
            for v in range(len(uL))]
