"""Orthonormal modal basis and Gauss-Legendre quadrature (Sec. 3, eq. BSpace).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's broken space holds polynomials of degree <= k on each element
(eq. BSpace).  On quads/hexes the default is the total-degree space P_p:
products of orthonormal 1-D Legendre polynomials
    phi_a(xi) = prod_k Lt_{a_k}(xi_k),   sum_k a_k <= p,
on the reference cube [-1, 1]^d, where Lt_n = sqrt((2n+1)/2) P_n.  Modes are
ordered by total degree, then lexicographically with the first index
descending, so the first n_m(p') modes span P_{p'} for every p' <= p (this is
what makes p-multigrid restriction a truncation, Sec. 6.1).

Quadrature (the paper is silent): tensor Gauss-Legendre with nq1d points per
direction on the volume and on every face.
"""
import itertools
import math

import numpy as np


def gauss_legendre(n):
    """Nodes and weights of the n-point Gauss-Legendre rule on [-1, 1]
    (library routine; exact for polynomials of degree <= 2n-1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def legendre_orthonormal(nmax, x):
    """Values and first derivatives of Lt_0..Lt_nmax at points x.

    Three-term (Bonnet) recurrence (n+1) P_{n+1} = (2n+1) x P_n - n P_{n-1}
    and P'_{n+1} = P'_{n-1} + (2n+1) P_n, then scaled by sqrt((2n+1)/2) so that
    int_{-1}^{1} Lt_a Lt_b = delta_ab.  Returns arrays (nmax+1, len(x)).
    """
    x = np.asarray(x, dtype=np.float64)
    P = np.zeros((nmax + 1,) + x.shape)
    dP = np.zeros((nmax + 1,) + x.shape)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = x
        dP[1] = 1.0
    for n in range(1, nmax):
        P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1)
        dP[n + 1] = dP[n - 1] + (2 * n + 1) * P[n]
    scale = np.sqrt((2.0 * np.arange(nmax + 1) + 1.0) / 2.0)
    shape = (nmax + 1,) + (1,) * x.ndim
    return P * scale.reshape(shape), dP * scale.reshape(shape)


def modes(p, d, basis="P"):
    """Multi-indices of the total-degree-p space P_p (basis "P") or of the
    tensor-product space Q_p (basis "Q", the paper's quadrilateral basis,
    Sec. 3) in d dimensions, ordered by degree (total degree for P, largest
    one-dimensional degree for Q), then lexicographically with the first index
    descending.  Either way the leading modes span the lower-order space of the
    same kind, which p-multigrid inheritance relies on (Sec. 6.1)."""
    out = []
    for s in range(p + 1):
        if basis == "Q":
            level = [a for a in itertools.product(range(s + 1), repeat=d) if max(a) == s]
        else:
            level = [a for a in itertools.product(range(s + 1), repeat=d) if sum(a) == s]
        level.sort(reverse=True)
        out.extend(level)
    return out


def n_modes(p, d, basis="P"):
    """dim P_p = C(p+d, d) (the paper's prod_i (k+i)/i) or dim Q_p = (p+1)^d."""
    return (p + 1) ** d if basis == "Q" else math.comb(p + d, d)


def volume_tables(p, d, nq1d, basis="P"):
    """Basis and reference gradients at the tensor GL volume points.

    Returns (phi[q, i], dphi[k, q, i], wq[q], xi[q, k]); point index q runs with
    the first coordinate fastest.
    """
    x, w = gauss_legendre(nq1d)
    L, dL = legendre_orthonormal(p, x)
    md = modes(p, d, basis)
    pts = list(itertools.product(range(nq1d), repeat=d))
    pts = [tuple(reversed(t)) for t in pts]          # first coordinate fastest
    nq = len(pts)
    phi = np.ones((nq, len(md)))
    dphi = np.ones((d, nq, len(md)))
    wq = np.ones(nq)
    xi = np.zeros((nq, d))
    for q, a in enumerate(pts):
        for k in range(d):
            wq[q] *= w[a[k]]
            xi[q, k] = x[a[k]]
        for i, al in enumerate(md):
            for k in range(d):
                phi[q, i] *= L[al[k], a[k]]
                for kk in range(d):
                    dphi[kk, q, i] *= (dL if kk == k else L)[al[k], a[k]]
    return phi, dphi, wq, xi


def face_tables(p, d, nq1d, k, side, basis="P"):
    """Basis traces and reference gradients on the local face xi_k = side (+-1).

    Face points are the tensor GL points of the other d-1 coordinates (in
    increasing coordinate order, the first fastest), so the two elements
    sharing a face list the same physical points in the same order.
    Returns (phif[q, i], dphif[kk, q, i], wf[q]).
    """
    x, w = gauss_legendre(nq1d)
    L, dL = legendre_orthonormal(p, x)
    Le, dLe = legendre_orthonormal(p, np.array([float(side)]))
    md = modes(p, d, basis)
    tang = [kk for kk in range(d) if kk != k]
    pts = list(itertools.product(range(nq1d), repeat=d - 1))
    pts = [tuple(reversed(t)) for t in pts]
    nqf = len(pts)
    phif = np.ones((nqf, len(md)))
    dphif = np.ones((d, nqf, len(md)))
    wf = np.ones(nqf)
    for q, a in enumerate(pts):
        for t, kk in enumerate(tang):
            wf[q] *= w[a[t]]
        for i, al in enumerate(md):
            for kk in range(d):
                if kk == k:
                    val, der = Le[al[kk], 0], dLe[al[kk], 0]
                else:
                    t = tang.index(kk)
                    val, der = L[al[kk], a[t]], dL[al[kk], a[t]]
                phif[q, i] *= val
                for k3 in range(d):
                    dphif[k3, q, i] *= der if k3 == kk else val
    return phif, dphif, wf
