"""Pins of the oracle's NS fluxes and Roe solver (Sec. 2, Sec. 3.1) against
hand-computed states, the Roe-matrix property and symmetries."""
import numpy as np
import pytest

from oracle.physics import (Physics, flux_c, flux_v, visc_K, roe_flux, roe_dissipation,
                            entropy_fix, primitives)

PH = Physics(gamma=1.4, Pr=0.72, mu=0.01, Rgas=1.0, roe_delta=0.1)


def cons(rho, vel, p, g=1.4):
    vel = np.asarray(vel, dtype=float)
    return [np.array(rho)] + [np.array(rho * v) for v in vel] + \
        [np.array(p / (g - 1) + 0.5 * rho * vel @ vel)]


def rand_state(rng, d):
    return cons(rng.uniform(0.5, 2.0), rng.uniform(-0.8, 0.8, d), rng.uniform(0.5, 2.0))


def test_primitives_and_inviscid_flux_hand_values():
    u = cons(1.2, [0.5, -0.25], 0.9)
    rho, vel, e0, p, T, h0 = primitives(u, PH)
    assert float(p) == pytest.approx(0.9)
    assert float(T) == pytest.approx(0.9 / 1.2)
    assert float(h0) == pytest.approx((0.9 / 0.4 + 0.5 * 1.2 * 0.3125 + 0.9) / 1.2)
    F = flux_c(u, PH)
    assert float(F[0][0]) == pytest.approx(1.2 * 0.5)
    assert float(F[1][0]) == pytest.approx(1.2 * 0.25 + 0.9)
    assert float(F[2][0]) == pytest.approx(1.2 * 0.5 * -0.25)
    assert float(F[2][1]) == pytest.approx(1.2 * 0.0625 + 0.9)
    assert float(F[3][1]) == pytest.approx(1.2 * -0.25 * float(h0))


@pytest.mark.parametrize("d", [2, 3])
def test_roe_consistency_and_property(d):
    rng = np.random.default_rng(d)
    for _ in range(20):
        uL, uR = rand_state(rng, d), rand_state(rng, d)
        n = rng.standard_normal(d)
        n /= np.linalg.norm(n)
        # consistency: Fhat(u, u, n) = F_c(u).n
        F = flux_c(uL, PH)
        fn = [sum(F[v][k] * n[k] for k in range(d)) for v in range(d + 2)]
        np.testing.assert_allclose(roe_flux(uL, uL, n, PH), fn, atol=1e-13)
        # Roe property: A(uL, uR)(uR - uL) = F(uR).n - F(uL).n (signed speeds)
        FR = flux_c(uR, PH)
        dF = [sum((FR[v][k] - F[v][k]) * n[k] for k in range(d)) for v in range(d + 2)]
        A = roe_dissipation(uL, uR, n, PH, absfn=lambda lam: lam)
        np.testing.assert_allclose(A, dF, atol=1e-12)
        # conservation: Fhat(uL, uR, n) = -Fhat(uR, uL, -n)
        np.testing.assert_allclose(roe_flux(uL, uR, n, PH),
                                   [-x for x in roe_flux(uR, uL, -n, PH)], atol=1e-13)


def test_roe_supersonic_upwinding():
    """All speeds positive and above the entropy-fix band: Roe = F(uL).n."""
    uL = cons(1.0, [3.0, 0.1, 0.0], 1.0)
    uR = cons(1.1, [2.9, 0.0, 0.1], 1.05)
    n = np.array([1.0, 0.0, 0.0])
    F = flux_c(uL, PH)
    np.testing.assert_allclose(roe_flux(uL, uR, n, PH), [F[v][0] for v in range(5)], atol=1e-12)
    F = flux_c(uR, PH)
    np.testing.assert_allclose(roe_flux(uL, uR, -n, PH), [-F[v][0] for v in range(5)],
                               atol=1e-12)


def test_roe_rotation_invariance():
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    uL, uR = rand_state(rng, 3), rand_state(rng, 3)
    n = np.array([0.0, 0.0, 1.0])

    def rot(u):
        mom = Q @ np.array([u[1], u[2], u[3]], dtype=float)
        return [u[0], mom[0], mom[1], mom[2], u[4]]
    f = roe_flux(uL, uR, n, PH)
    g = roe_flux(rot(uL), rot(uR), Q @ n, PH)
    np.testing.assert_allclose(g, rot(f), atol=1e-13)


def test_entropy_fix_continuity():
    delta = 0.3
    lam = np.array([delta - 1e-12, delta + 1e-12, -delta + 1e-12, -delta - 1e-12])
    v = entropy_fix(lam, delta)
    assert abs(v[0] - v[1]) < 1e-11 and abs(v[2] - v[3]) < 1e-11
    assert entropy_fix(np.array([0.0]), delta)[0] == pytest.approx(delta / 2)
    assert entropy_fix(np.array([-2.0]), 0.0)[0] == 2.0


def _grad_from_prim(u, dvel, dT, drho, ph):
    """Conservative gradient from primitive gradients (rho, v, T)."""
    rho, vel, e0, p, T, h0 = primitives(u, ph)
    d = len(vel)
    cv = ph.Rgas / (ph.gamma - 1)
    g = [[None] * d for _ in range(d + 2)]
    for k in range(d):
        g[0][k] = drho[k]
        for j in range(d):
            g[1 + j][k] = drho[k] * vel[j] + rho * dvel[j][k]
        de0 = cv * dT[k] + sum(vel[j] * dvel[j][k] for j in range(d))
        g[d + 1][k] = drho[k] * e0 + rho * de0
    return g


def test_viscous_shear_dilatation_heat():
    ph = Physics(gamma=1.4, Pr=0.72, mu=0.05, Rgas=1.0)
    u = cons(1.3, [0.4, 0.0, 0.0], 1.1)
    z = [0.0, 0.0, 0.0]
    a = 0.7
    # simple shear du/dy = a
    g = _grad_from_prim(u, [[0, a, 0], z, z], z, z, ph)
    F = flux_v(u, g, ph)
    assert float(F[1][1]) == pytest.approx(-ph.mu * a)
    assert float(F[2][0]) == pytest.approx(-ph.mu * a)
    assert float(F[1][0]) == pytest.approx(0.0, abs=1e-15)
    assert float(F[4][1]) == pytest.approx(-0.4 * ph.mu * a)
    assert all(float(F[0][k]) == 0.0 for k in range(3))
    # isotropic dilatation: zero deviatoric stress (Stokes hypothesis)
    g = _grad_from_prim(u, [[a, 0, 0], [0, a, 0], [0, 0, a]], z, z, ph)
    F = flux_v(u, g, ph)
    for j in range(3):
        for k in range(3):
            assert abs(float(F[1 + j][k])) < 1e-15
    # pure heat conduction at rest: F_v energy = q = -mu c_p/Pr dT/dx
    ur = cons(1.3, [0.0, 0.0, 0.0], 1.1)
    g = _grad_from_prim(ur, [z, z, z], [0.2, 0, 0], [0.1, 0, 0], ph)
    F = flux_v(ur, g, ph)
    cp = ph.gamma * ph.Rgas / (ph.gamma - 1)
    assert float(F[4][0]) == pytest.approx(-ph.mu * cp / ph.Pr * 0.2)
    assert float(F[1][0]) == pytest.approx(0.0, abs=1e-15)


def test_viscous_frame_indifference_and_linearity():
    ph = Physics(gamma=1.4, Pr=0.72, mu=0.03, Rgas=1.0)
    rng = np.random.default_rng(3)
    u = rand_state(rng, 3)
    g = [[rng.standard_normal() for _ in range(3)] for _ in range(5)]
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    F = np.array(flux_v(u, g, ph), dtype=float)
    G = np.array(g)
    # rotate: momentum rows by Q, gradient directions by Q
    uq = [u[0]] + list(Q @ np.array(u[1:4], dtype=float)) + [u[4]]
    Gq = G @ Q.T
    Gq[1:4] = Q @ Gq[1:4]
    Fq = np.array(flux_v(uq, [list(r) for r in Gq], ph), dtype=float)
    Fr = F @ Q.T
    Fr[1:4] = Q @ Fr[1:4]
    np.testing.assert_allclose(Fq, Fr, atol=1e-14)
    # linearity in g; K = -F_v
    g2 = [[rng.standard_normal() for _ in range(3)] for _ in range(5)]
    a = 0.37
    lhs = np.array(flux_v(u, [[a * g[v][k] + g2[v][k] for k in range(3)] for v in range(5)],
                          ph), dtype=float)
    rhs = a * F + np.array(flux_v(u, g2, ph), dtype=float)
    np.testing.assert_allclose(lhs, rhs, atol=1e-14)
    np.testing.assert_allclose(np.array(visc_K(u, g, ph), dtype=float), -F, atol=0)


def test_complex_step_through_fluxes():
    """Complex-step derivative of the Roe + viscous fluxes equals central FD."""
    rng = np.random.default_rng(5)
    uL, uR = rand_state(rng, 2), rand_state(rng, 2)
    du = rng.standard_normal(4)
    n = np.array([0.6, 0.8])
    h = 1e-30
    c = roe_flux([uL[v] + 1j * h * du[v] for v in range(4)], uR, n, PH)
    cs = np.array([np.imag(x) / h for x in c])
    e = 1e-6
    fp = roe_flux([uL[v] + e * du[v] for v in range(4)], uR, n, PH)
    fm = roe_flux([uL[v] - e * du[v] for v in range(4)], uR, n, PH)
    fd = (np.array(fp, dtype=float) - np.array(fm, dtype=float)) / (2 * e)
    np.testing.assert_allclose(cs, fd, rtol=1e-7, atol=1e-8)
