"""Modal DG residual of the compressible NS equations and its Jacobian-vector
product (Sec. 3.1, eqs. dg_ns, visc_flux, re; Sec. 5.1, eqs. ODEDG, DG-mf).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Mesh: periodic structured boxes (quads for d = 2, hexes for d = 3) on
[lo, hi]^d with n_k elements per direction; element e = i_0 + n_0 (i_1 + n_1 i_2).
Affine map x = x_c + (h/2) xi, so |J| = prod h_k/2, face area factor
|J_F|_k = prod_{k' != k} h_k'/2 and grad = (2/h_k) d/dxi_k.

State layout W[e, v, i] (element, conservative variable, mode), FP64.

Residual (R defined by M dW/dt + R(W) = 0, Sec. 3.1), for test function phi_i
on element K and every variable v:

  R_K,v,i = - int_K grad phi_i . F_v-row(u, grad u)                  (volume)
            + sum_faces int_F phi_i  Fhat_v                           (flux)
            - sum_faces int_F grad phi_i . [K(u+) ((u+ - uhat) (x) n+)]_v  (dual)

  Fhat = Roe(u+, u-, n+) + {F_v(u, grad u)}.n+ + eta {delta_F}.n+   (eq. visc_flux)
  uhat = (u+ + u-)/2,  {a} = (a+ + a-)/2,
  delta_F+ in [V_h]^{d x m}: int_K tau : delta_F+ = 1/2 int_F tau : K(u+)((u+ - u-) (x) n+)
  delta_F- the same on the neighbour with K(u-) and n- (eq. re),

where (K . g) = -F_v(u, g) is the viscous flux operator applied to a
gradient-shaped tensor g (F_v = -K grad u, Sec. 3.1).  Every element evaluates
its own faces (each interior face is evaluated once from each side), so
discrete conservation is a property the tests check, not a construction.
"""
import numpy as np

from . import basis
from .physics import flux_c, flux_v, visc_K, roe_flux


class Mesh:
    """Periodic structured mesh with the modal basis tables (Sec. 3)."""

    def __init__(self, dim, n, lo, hi, p, nq1d=None, space="P"):
        self.d = d = int(dim)
        self.n = tuple(int(x) for x in n[:d])
        self.lo = tuple(float(x) for x in lo[:d])
        self.hi = tuple(float(x) for x in hi[:d])
        self.p = int(p)
        self.nq1d = int(nq1d) if nq1d else self.p + 2
        self.m = d + 2
        self.space = basis_kind = str(space)      # "P": total degree p, "Q": tensor degree p
        self.nm = basis.n_modes(self.p, d, basis_kind)
        self.nb = self.m * self.nm
        self.E = int(np.prod(self.n))
        self.h = [(self.hi[k] - self.lo[k]) / self.n[k] for k in range(d)]
        self.detJ = float(np.prod([hk / 2.0 for hk in self.h]))
        self.faceJ = [float(np.prod([self.h[kk] / 2.0 for kk in range(d) if kk != k]))
                      for k in range(d)]
        self.metric = [2.0 / hk for hk in self.h]
        self.phi, self.dphi, self.wq, self.xi = basis.volume_tables(self.p, d, self.nq1d, basis_kind)
        self.face = {}
        for k in range(d):
            for s in (-1, 1):
                self.face[(k, s)] = basis.face_tables(self.p, d, self.nq1d, k, s, basis_kind)
        # element multi-indices and periodic face neighbours nbr[e, k, side]
        idx = np.stack(np.unravel_index(np.arange(self.E), tuple(reversed(self.n))), axis=1)
        self.ijk = idx[:, ::-1].copy()                    # (E, d), first index fastest
        self.nbr = np.zeros((self.E, d, 2), dtype=np.int64)
        for k in range(d):
            for side, s in enumerate((-1, 1)):
                j = self.ijk.copy()
                j[:, k] = (j[:, k] + s) % self.n[k]
                self.nbr[:, k, side] = self.elem_index(j)

    def elem_index(self, ijk):
        e = np.zeros(len(ijk), dtype=np.int64)
        for k in reversed(range(self.d)):
            e = e * self.n[k] + ijk[:, k]
        return e

    def centers(self):
        return np.stack([self.lo[k] + (self.ijk[:, k] + 0.5) * self.h[k]
                         for k in range(self.d)], axis=1)

    def vol_points(self):
        """Physical volume quadrature points (E, nq, d)."""
        c = self.centers()
        return c[:, None, :] + self.xi[None, :, :] * (np.array(self.h) / 2.0)[None, None, :]


def _trace(Wt, tab):
    """u[v] (nT, nq) from modal W (nT, m, nm) and a basis table (nq, nm)."""
    U = Wt @ tab.T
    return [U[:, v, :] for v in range(Wt.shape[1])]


def _grad(Wt, dtab, metric):
    """g[v][k] (nT, nq): physical gradient from reference-derivative tables."""
    G = [(Wt @ dtab[k].T) * metric[k] for k in range(len(metric))]
    return [[G[k][:, v, :] for k in range(len(metric))] for v in range(Wt.shape[1])]


def lift_face(mesh, k, tab, wf, X):
    """BR2 lifting (eq. re) of one component: delta in V_h with
    int_K tau delta = 1/2 int_F tau X for all tau in V_h, evaluated at the face
    points.  With M = |J| I: delta_i = |J_F| / (2 |J|) sum_q wf_q phi_i(q) X_q.
    tab = the element's basis traces on that face (nqf, nm); X (nT, nqf)."""
    cl = mesh.faceJ[k] / (2.0 * mesh.detJ)
    return cl * (((X * wf) @ tab) @ tab.T)


def residual_parts(mesh, ph, W, elems=None):
    """Volume and per-face parts of R for the target elements.

    Returns (Rvol[nT, m, nm], Rface[nT, d, 2, m, nm]) with R = Rvol + sum of
    Rface over (k, side); side 0 is the face xi_k = -1, side 1 is xi_k = +1.
    W may be complex (complex-step differentiation).
    """
    d, m, nm = mesh.d, mesh.m, mesh.nm
    T = np.arange(mesh.E) if elems is None else np.asarray(elems, dtype=np.int64)
    Wt = W[T]
    nT = len(T)
    eta = ph.eta_for(d)
    cplx = np.iscomplexobj(W)
    dt = np.complex128 if cplx else np.float64

    # volume term: - int_K grad phi_i . F(u, grad u)
    u = _trace(Wt, mesh.phi)
    g = _grad(Wt, mesh.dphi, mesh.metric)
    Fc = flux_c(u, ph)
    Fv = flux_v(u, g, ph)
    Rvol = np.zeros((nT, m, nm), dtype=dt)
    for v in range(m):
        for k in range(d):
            Rvol[:, v, :] -= mesh.detJ * mesh.metric[k] * (
                ((Fc[v][k] + Fv[v][k]) * mesh.wq) @ mesh.dphi[k])

    # face terms, element by element (each side evaluates its own faces)
    Rface = np.zeros((nT, d, 2, m, nm), dtype=dt)
    for k in range(d):
        for side, s in enumerate((-1, 1)):
            nb = mesh.nbr[T, k, side]
            phP, dphP, wf = mesh.face[(k, s)]         # own face xi_k = s
            phM, dphM, _ = mesh.face[(k, -s)]         # neighbour's face xi_k = -s
            nrm = [float(s) if kk == k else 0.0 for kk in range(d)]
            uP = _trace(Wt, phP)
            gP = _grad(Wt, dphP, mesh.metric)
            uM = _trace(W[nb], phM)
            gM = _grad(W[nb], dphM, mesh.metric)
            jump = [[(uP[v] - uM[v]) * nrm[kk] for kk in range(d)] for v in range(m)]
            GP = visc_K(uP, jump, ph)                 # K(u+) ((u+ - u-) (x) n+)
            GM = visc_K(uM, jump, ph)                 # K(u-) ((u- - u+) (x) n-)
            lift = lambda X, tab: lift_face(mesh, k, tab, wf, X)
            FvP = flux_v(uP, gP, ph)
            FvM = flux_v(uM, gM, ph)
            Fr = roe_flux(uP, uM, nrm, ph)
            fhat = []
            for v in range(m):
                acc = Fr[v]
                for kk in range(d):
                    if nrm[kk] == 0.0:
                        continue
                    dP = lift(GP[v][kk], phP)
                    dM = lift(GM[v][kk], phM)
                    acc = acc + (0.5 * (FvP[v][kk] + FvM[v][kk]) + eta * 0.5 * (dP + dM)) * nrm[kk]
                fhat.append(acc)
            uhat = [0.5 * (uP[v] + uM[v]) for v in range(m)]
            dual = visc_K(uP, [[(uP[v] - uhat[v]) * nrm[kk] for kk in range(d)]
                               for v in range(m)], ph)
            for v in range(m):
                acc = (fhat[v] * wf) @ phP
                for kk in range(d):
                    acc = acc - mesh.metric[kk] * ((dual[v][kk] * wf) @ dphP[kk])
                Rface[:, k, side, v, :] = mesh.faceJ[k] * acc
    return Rvol, Rface


def residual(mesh, ph, W, elems=None):
    """R(W) (Sec. 3.1, M dW/dt + R(W) = 0), shape (nT, m, nm)."""
    Rvol, Rface = residual_parts(mesh, ph, W, elems)
    return Rvol + Rface.sum(axis=(1, 2))


def mass_apply(mesh, v):
    """M v with M = |J| I (orthonormal basis, affine element)."""
    return mesh.detJ * v


def jvp(mesh, ph, W, v, sigma, h=1e-30, elems=None):
    """Exact K v = sigma M v + dR/dW(W) v (Sec. 5.1, eq. ODEDG), with the
    directional derivative taken by the complex step Im R(W + i h v)/h
    (Squire & Trapp 1998): no subtractive cancellation, so it equals the exact
    derivative up to rounding.  sigma is 1/(a_ii dt) (ESDIRK) or 3/(2 dt) (BDF2).
    elems (optional): return only those elements' rows."""
    scale = max(1.0, float(np.max(np.abs(v)))) if v.size else 1.0
    hh = h / scale
    Rc = residual(mesh, ph, W.astype(np.complex128) + 1j * hh * v, elems=elems)
    vt = v if elems is None else v[np.asarray(elems, dtype=np.int64)]
    return sigma * mass_apply(mesh, vt) + Rc.imag / hh


def jvp_fd(mesh, ph, W, RW, v, sigma, eps=1e-7, variant="printed"):
    """Matrix-free finite-difference K v of eq. DG-mf:
    sigma M v + (R(W + h v) - R(W))/h.

    variant "printed": h = eps sqrt(1 + ||v||)/||W|| as printed in Sec. 5.1;
    variant "scaled": h = eps sqrt(1 + ||W||)/||v|| (the usual Jacobian-free
    Newton-Krylov choice).  Norms are Euclidean over all DOFs."""
    nv = float(np.linalg.norm(v))
    nw = float(np.linalg.norm(W))
    if nv == 0.0:
        return np.zeros_like(v)
    if variant == "printed":
        hh = eps * np.sqrt(1.0 + nv) / nw
    else:
        hh = eps * np.sqrt(1.0 + nw) / nv
    return sigma * mass_apply(mesh, v) + (residual(mesh, ph, W + hh * v) - RW) / hh


def l2_project(mesh, f, nq_extra=3):
    """Modal coefficients of the L2 projection of a pointwise field f(x) ->
    list of m arrays, with a (p + 1 + nq_extra)-point tensor GL rule.  Used by
    the oracle's own convergence tests (the orthonormal basis makes the
    projection coefficient extraction: W_i = |J|^-1 int_K f phi_i)."""
    nq1d = mesh.p + 1 + nq_extra
    phi, _, wq, xi = basis.volume_tables(mesh.p, mesh.d, nq1d, mesh.space)
    c = mesh.centers()
    X = c[:, None, :] + xi[None, :, :] * (np.array(mesh.h) / 2.0)[None, None, :]
    vals = f(X)
    W = np.zeros((mesh.E, mesh.m, mesh.nm))
    for v in range(mesh.m):
        W[:, v, :] = (vals[v] * wq) @ phi
    return W
