"""Pins of the oracle's basis and quadrature (Sec. 3, eq. BSpace) against
closed forms and numpy's own Legendre routines."""
import math

import numpy as np
import pytest

from oracle import basis


def test_legendre_closed_forms():
    x = np.linspace(-1, 1, 17)
    L, dL = basis.legendre_orthonormal(3, x)
    s = lambda n: math.sqrt((2 * n + 1) / 2.0)
    np.testing.assert_allclose(L[0], s(0) * np.ones_like(x), atol=1e-15)
    np.testing.assert_allclose(L[2], s(2) * (3 * x**2 - 1) / 2, atol=1e-14)
    np.testing.assert_allclose(L[3], s(3) * (5 * x**3 - 3 * x) / 2, atol=1e-14)
    np.testing.assert_allclose(dL[2], s(2) * 3 * x, atol=1e-14)
    np.testing.assert_allclose(dL[3], s(3) * (15 * x**2 - 3) / 2, atol=1e-13)


@pytest.mark.parametrize("nmax", [0, 1, 4, 7])
def test_legendre_vs_numpy(nmax):
    x = np.random.default_rng(0).uniform(-1, 1, 31)
    L, dL = basis.legendre_orthonormal(nmax, x)
    for n in range(nmax + 1):
        c = np.zeros(n + 1)
        c[n] = math.sqrt((2 * n + 1) / 2.0)
        np.testing.assert_allclose(L[n], np.polynomial.legendre.legval(x, c), atol=1e-13)
        np.testing.assert_allclose(dL[n], np.polynomial.legendre.legval(
            x, np.polynomial.legendre.legder(c)), atol=1e-12)
    # endpoint values: Lt_n(+-1) = (+-1)^n sqrt((2n+1)/2)
    Le, _ = basis.legendre_orthonormal(nmax, np.array([-1.0, 1.0]))
    for n in range(nmax + 1):
        assert Le[n, 1] == pytest.approx(math.sqrt((2 * n + 1) / 2.0), abs=1e-14)
        assert Le[n, 0] == pytest.approx((-1) ** n * math.sqrt((2 * n + 1) / 2.0), abs=1e-14)


def test_gauss_exactness():
    for n in range(1, 9):
        x, w = basis.gauss_legendre(n)
        for k in range(2 * n):
            exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
            assert np.dot(w, x**k) == pytest.approx(exact, abs=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_modes_count_and_hierarchy(d):
    for p in range(7):
        md = basis.modes(p, d)
        assert len(md) == basis.n_modes(p, d) == math.comb(p + d, d)
        assert len(set(md)) == len(md)
        for pp in range(p + 1):
            head = md[: basis.n_modes(pp, d)]
            assert all(sum(a) <= pp for a in head)
    assert basis.n_modes(4, 3) == 35 and basis.n_modes(6, 3) == 84
    assert basis.n_modes(2, 2) == 6


@pytest.mark.parametrize("d,p", [(2, 2), (2, 4), (3, 2), (3, 4)])
def test_volume_orthonormal_and_exact(d, p):
    phi, dphi, wq, xi = basis.volume_tables(p, d, p + 2)
    np.testing.assert_allclose(phi.T @ (wq[:, None] * phi), np.eye(phi.shape[1]), atol=1e-13)
    assert wq.sum() == pytest.approx(2.0**d)
    # the tables' reference gradients against central differences of the
    # product basis evaluated pointwise
    h = 1e-6
    md = basis.modes(p, d)

    def ev(y):
        L, _ = basis.legendre_orthonormal(p, y)
        return np.array([np.prod([L[a[kk], kk] for kk in range(d)]) for a in md])

    for q in [0, len(wq) // 2, len(wq) - 1]:
        np.testing.assert_allclose(phi[q], ev(xi[q]), atol=1e-14)
        for k in range(d):
            yp, ym = xi[q].copy(), xi[q].copy()
            yp[k] += h
            ym[k] -= h
            np.testing.assert_allclose(dphi[k, q], (ev(yp) - ev(ym)) / (2 * h), atol=1e-7)


@pytest.mark.parametrize("d,p", [(2, 3), (3, 2)])
def test_divergence_theorem_tables(d, p):
    """int_K d phi_i/dxi_k = int_{dK} phi_i n_k ties volume and face tables."""
    phi, dphi, wq, _ = basis.volume_tables(p, d, p + 2)
    for k in range(d):
        lhs = wq @ dphi[k]
        rhs = 0
        for s in (-1, 1):
            pf, _, wf = basis.face_tables(p, d, p + 2, k, s)
            rhs = rhs + s * (wf @ pf)
        np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_face_trace_matches_volume_function():
    d, p = 3, 3
    md = basis.modes(p, d)
    x, _ = basis.gauss_legendre(p + 2)
    for k in range(d):
        for s in (-1, 1):
            pf, dpf, _ = basis.face_tables(p, d, p + 2, k, s)
            tang = [kk for kk in range(d) if kk != k]
            for q in [0, 3, len(pf) - 1]:
                a = (q % (p + 2), q // (p + 2))
                pt = np.zeros(d)
                pt[k] = s
                pt[tang[0]], pt[tang[1]] = x[a[0]], x[a[1]]
                L, dL = basis.legendre_orthonormal(p, pt)
                val = np.array([np.prod([L[al[kk], kk] for kk in range(d)]) for al in md])
                np.testing.assert_allclose(pf[q], val, atol=1e-14)
                for kk in range(d):
                    der = np.array([np.prod([(dL if k3 == kk else L)[al[k3], k3]
                                             for k3 in range(d)]) for al in md])
                    np.testing.assert_allclose(dpf[kk, q], der, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_modes_count_and_hierarchy(d):
    """Q_p (the paper's quadrilateral basis, Sec. 3): (p+1)^d modes, every 1-D
    degree <= p, and the leading (p'+1)^d modes span Q_p' (inheritance)."""
    for p in range(6):
        md = basis.modes(p, d, "Q")
        assert len(md) == basis.n_modes(p, d, "Q") == (p + 1) ** d
        assert len(set(md)) == len(md) and all(max(a) <= p for a in md)
        for pp in range(p + 1):
            head = md[: basis.n_modes(pp, d, "Q")]
            assert sorted(head) == sorted(a for a in md if max(a) <= pp)


@pytest.mark.parametrize("d,p", [(2, 3), (3, 2)])
def test_tensor_volume_orthonormal_and_divergence(d, p):
    phi, dphi, wq, xi = basis.volume_tables(p, d, p + 2, "Q")
    np.testing.assert_allclose(phi.T @ (wq[:, None] * phi), np.eye(phi.shape[1]), atol=1e-13)
    # int_K d(phi_i phi_j)/dxi_k = boundary terms on the faces xi_k = +-1
    for k in range(d):
        vol = (dphi[k].T * wq) @ phi + ((phi.T * wq) @ dphi[k])
        bnd = np.zeros_like(vol)
        for side in (-1, 1):
            pf, _, wf = basis.face_tables(p, d, p + 2, k, side, "Q")
            bnd += side * (pf.T * wf) @ pf
        np.testing.assert_allclose(vol, bnd, atol=1e-12)
