"""Modal DG on periodic triangular meshes with general face connectivity and
the full-order space P_p on every triangle (Sec. 3: polynomials of total
degree <= k on triangular grids, n_v = (k+1)(k+2)/2 per equation; Sec. 7.2:
a quadrilateral grid split into triangles).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Reference triangle T = {(r, s): r >= -1, s >= -1, r + s <= 0}, vertices
(-1,-1), (1,-1), (-1,1) (area 2), local edges e0 = v0->v1, e1 = v1->v2,
e2 = v2->v0 (counter-clockwise).

Basis: the orthonormal Dubiner (Koornwinder) polynomials
    psi_ij(r, s) = sqrt(2) Ph_i^(0,0)(a) Ph_j^(2i+1,0)(b) (1 - b)^i,
    a = 2 (1 + r)/(1 - s) - 1,  b = s,
where Ph_n^(alpha,0) is the Jacobi polynomial scaled to unit norm with weight
(1-x)^alpha on [-1, 1]; int_T psi_ij psi_kl = delta.  Modes are ordered by
total degree i + j, then i descending, so the first n_m(q) modes span P_q (the
p-multigrid restriction is a truncation, Sec. 6.1).  Reference derivatives are
taken by the complex step (the basis is analytic inside T).

Quadrature: the collapsed (Duffy) tensor Gauss-Legendre rule on T with
nq1d^2 points, weight w_a w_b (1 - b)/2 (exact to degree 2 nq1d - 2), and
nq1d-point Gauss-Legendre rules on the edges.

Mesh: vertices X (wrapped into the periodic box), triangles as three vertex
ids counter-clockwise plus an integer lattice shift per corner (the corner's
coordinates are X[id] + shift * (hi - lo)).  Affine maps x = x0 + J (xi + 1)
with one J per triangle; the edge connectivity is found by matching the
vertex pairs of edges (with their relative lattice shift), each interior edge
seen from both triangles in opposite directions.  The residual is that of
``oracle.dg`` (volume term, Roe flux, BR2 with penalty eta = n_faces + 1 = 4
unless given, dual-consistency term) with per-triangle metrics and normals.
"""
import math

import numpy as np

from .basis import gauss_legendre
from .physics import flux_c, flux_v, visc_K, roe_flux

REF_VERTS = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])
REF_EDGES = ((0, 1), (1, 2), (2, 0))


def n_modes_tri(p):
    return (p + 1) * (p + 2) // 2


def modes_tri(p):
    return [(i, q - i) for q in range(p + 1) for i in range(q, -1, -1)]


def jacobi(n, alpha, x):
    """P_0 .. P_n of the Jacobi family (alpha, 0) at x (real or complex), by
    the three-term recurrence (beta = 0):
    2 (k+1)(k+alpha+1) c P_{k+1} = (c+1)[(c+2) c x + alpha^2] P_k
                                   - 2 (k+alpha) k (c+2) P_{k-1},  c = 2k + alpha."""
    x = np.asarray(x)
    P = [np.ones_like(x)]
    if n >= 1:
        P.append(((alpha + 2.0) * x + alpha) / 2.0)
    for k in range(1, n):
        c = 2 * k + alpha
        P.append(((c + 1) * ((c + 2) * c * x + alpha * alpha) * P[k] - 2.0 * (k + alpha) * k * (c + 2) * P[k - 1])
                 / (2.0 * (k + 1) * (k + alpha + 1) * c))
    return P


def jacobi_norm2(n, alpha):
    """int_{-1}^{1} (1-x)^alpha P_n^(alpha,0)(x)^2 dx = 2^(alpha+1)/(2n+alpha+1)."""
    return 2.0 ** (alpha + 1) / (2 * n + alpha + 1)


def dubiner(p, r, s):
    """psi (n_m, *shape) at reference points (r, s)."""
    r = np.asarray(r)
    s = np.asarray(s)
    a = 2.0 * (1.0 + r) / (1.0 - s) - 1.0
    b = s
    La = jacobi(p, 0, a)
    out = []
    for i, j in modes_tri(p):
        Pa = La[i] / math.sqrt(jacobi_norm2(i, 0))
        Pb = jacobi(j, 2 * i + 1, b)[j] / math.sqrt(jacobi_norm2(j, 2 * i + 1))
        out.append(math.sqrt(2.0) * Pa * Pb * (1.0 - b) ** i)
    return np.array(out)


def dubiner_grad(p, r, s, h=1e-30):
    """(d psi/dr, d psi/ds), each (n_m, *shape), by the complex step."""
    r = np.asarray(r, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    return (dubiner(p, r + 1j * h, s + 0j).imag / h, dubiner(p, r + 0j, s + 1j * h).imag / h)


def tri_rule(nq1d):
    """Collapsed Gauss-Legendre rule on T: points (r, s) and weights, point
    q = ia + nq1d * ib."""
    x, w = gauss_legendre(nq1d)
    a = np.tile(x, nq1d)
    b = np.repeat(x, nq1d)
    wq = np.tile(w, nq1d) * np.repeat(w, nq1d) * (1.0 - b) / 2.0
    r = (1.0 + a) * (1.0 - b) / 2.0 - 1.0
    return r, b.copy(), wq


def volume_tables(p, nq1d):
    r, s, wq = tri_rule(nq1d)
    phi = dubiner(p, r, s).T                              # (nq, nm)
    dr, ds = dubiner_grad(p, r, s)
    return phi, np.stack([dr.T, ds.T]), wq, np.stack([r, s], axis=1)


def edge_tables(p, nq1d, f):
    """Traces on reference edge f at its nq1d Gauss points, in the edge's own
    direction: (phi (nqf, nm), dphi (2, nqf, nm), weights (nqf,), points)."""
    t, w = gauss_legendre(nq1d)
    va, vb = REF_VERTS[REF_EDGES[f][0]], REF_VERTS[REF_EDGES[f][1]]
    pts = va[None, :] * ((1.0 - t) / 2.0)[:, None] + vb[None, :] * ((1.0 + t) / 2.0)[:, None]
    phi = dubiner(p, pts[:, 0], pts[:, 1]).T
    dr, ds = dubiner_grad(p, pts[:, 0], pts[:, 1])
    return phi, np.stack([dr.T, ds.T]), w, pts


class TriMesh:
    """Periodic triangulation with per-triangle affine geometry and the basis
    tables (Sec. 3)."""

    def __init__(self, X, tri, shift, lo, hi, p, nq1d=None):
        self.d, self.m = 2, 4
        self.p = int(p)
        self.nq1d = int(nq1d) if nq1d else self.p + 2
        self.space = "tri"
        self.nm = n_modes_tri(self.p)
        self.nb = self.m * self.nm
        self.lo = np.asarray(lo, dtype=np.float64)[:2]
        self.hi = np.asarray(hi, dtype=np.float64)[:2]
        self.Lbox = self.hi - self.lo
        self.X = np.asarray(X, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        self.shift = np.asarray(shift, dtype=np.int64)
        self.E = len(self.tri)
        self.V = self.X[self.tri] + self.shift * self.Lbox[None, None, :]       # (E, 3, 2) corners
        J = np.zeros((self.E, 2, 2))
        J[:, :, 0] = (self.V[:, 1] - self.V[:, 0]) / 2.0
        J[:, :, 1] = (self.V[:, 2] - self.V[:, 0]) / 2.0
        self.J = J
        self.detJ = np.linalg.det(J)
        if np.any(self.detJ <= 0.0):
            raise ValueError("triangles must be counter-clockwise and non-degenerate")
        self.Jinv = np.linalg.inv(J)                     # Jinv[e, l, k] = d xi_l / d x_k
        self.phi, self.dphi, self.wq, self.xi = volume_tables(self.p, self.nq1d)
        self.edge = [edge_tables(self.p, self.nq1d, f) for f in range(3)]
        # edge geometry: length and outward normal (right of the CCW direction)
        self.elen = np.zeros((self.E, 3))
        self.normal = np.zeros((self.E, 3, 2))
        for f, (a, b) in enumerate(REF_EDGES):
            dv = self.V[:, b] - self.V[:, a]
            L = np.hypot(dv[:, 0], dv[:, 1])
            self.elen[:, f] = L
            self.normal[:, f, 0] = dv[:, 1] / L
            self.normal[:, f, 1] = -dv[:, 0] / L
        # connectivity by matching (vertex pair, relative lattice shift)
        seen = {}
        for e in range(self.E):
            for f, (a, b) in enumerate(REF_EDGES):
                ga, gb = int(self.tri[e, a]), int(self.tri[e, b])
                dl = tuple(int(v) for v in (self.shift[e, b] - self.shift[e, a]))
                key = min((ga, gb, dl), (gb, ga, tuple(-v for v in dl)))
                seen.setdefault(key, []).append((e, f))
        self.nbr = np.full((self.E, 3), -1, dtype=np.int64)
        self.nbr_f = np.full((self.E, 3), -1, dtype=np.int64)
        for key, lst in seen.items():
            if len(lst) != 2:
                raise ValueError("edge %r is shared by %d triangles" % (key, len(lst)))
            (e0, f0), (e1, f1) = lst
            self.nbr[e0, f0], self.nbr_f[e0, f0] = e1, f1
            self.nbr[e1, f1], self.nbr_f[e1, f1] = e0, f0

    def vol_points(self, xi=None):
        """Physical points (E, nq, 2) of reference points xi (default: the rule's)."""
        xi = self.xi if xi is None else xi
        return self.V[:, None, 0, :] + np.einsum("ekl,ql->eqk", self.J, xi + 1.0)


def _phys_grad(Jinv, dref):
    """Physical derivatives of traces: dref[l] (nT, m, nq) -> g[k] = sum_l Jinv[:, l, k] dref[l]."""
    return [sum(Jinv[:, l, k][:, None, None] * dref[l] for l in range(2)) for k in range(2)]


def residual_parts(mesh, ph, W, elems=None):
    """Volume and per-edge parts of R (Sec. 3.1, the terms of ``oracle.dg``):
    (Rvol[nT, m, nm], Rface[nT, 3, m, nm]), R = Rvol + Rface.sum(axis=1)."""
    m, nm = mesh.m, mesh.nm
    T = np.arange(mesh.E) if elems is None else np.asarray(elems, dtype=np.int64)
    Wt = W[T]
    nT = len(T)
    eta = 4.0 if ph.eta is None else float(ph.eta)
    dt = np.complex128 if np.iscomplexobj(W) else np.float64
    JiT, dJT = mesh.Jinv[T], mesh.detJ[T]

    # volume: - int_K grad phi_i . F
    U = Wt @ mesh.phi.T                                    # (nT, m, nq)
    G = _phys_grad(JiT, [Wt @ mesh.dphi[l].T for l in range(2)])
    u = [U[:, v, :] for v in range(m)]
    g = [[G[k][:, v, :] for k in range(2)] for v in range(m)]
    Fc, Fv = flux_c(u, ph), flux_v(u, g, ph)
    dphix = [sum(JiT[:, l, k][:, None, None] * mesh.dphi[l][None] for l in range(2)) for k in range(2)]
    Rvol = np.zeros((nT, m, nm), dtype=dt)
    for v in range(m):
        for k in range(2):
            Rvol[:, v, :] -= dJT[:, None] * np.einsum("eq,eqi->ei", (Fc[v][k] + Fv[v][k]) * mesh.wq, dphix[k])

    Rface = np.zeros((nT, 3, m, nm), dtype=dt)
    phR = np.stack([mesh.edge[h][0][::-1] for h in range(3)])          # neighbour traces, reversed points
    dphR = np.stack([mesh.edge[h][1][:, ::-1] for h in range(3)])
    for f in range(3):
        nb, fn = mesh.nbr[T, f], mesh.nbr_f[T, f]
        phP, dphP, wf, _ = mesh.edge[f]
        phM, dphM = phR[fn], dphR[fn]                                  # (nT, nqf, nm), (nT, 2, nqf, nm)
        nrm = [mesh.normal[T, f, k][:, None] for k in range(2)]
        JF = mesh.elen[T, f] / 2.0
        WM = W[nb]
        UP = Wt @ phP.T
        GP = _phys_grad(JiT, [Wt @ dphP[l].T for l in range(2)])
        UM = np.einsum("evi,eqi->evq", WM, phM)
        GM = _phys_grad(mesh.Jinv[nb], [np.einsum("evi,eqi->evq", WM, dphM[:, l]) for l in range(2)])
        uP = [UP[:, v, :] for v in range(m)]
        uM = [UM[:, v, :] for v in range(m)]
        gP = [[GP[k][:, v, :] for k in range(2)] for v in range(m)]
        gM = [[GM[k][:, v, :] for k in range(2)] for v in range(m)]
        jump = [[(uP[v] - uM[v]) * nrm[k] for k in range(2)] for v in range(m)]
        KP = visc_K(uP, jump, ph)                     # K(u+) ((u+ - u-) (x) n+)
        KM = visc_K(uM, jump, ph)                     # K(u-) ((u- - u+) (x) n-)
        clP = (JF / (2.0 * dJT))[:, None]
        clM = (JF / (2.0 * mesh.detJ[nb]))[:, None]
        liftP = lambda X: clP * (((X * wf) @ phP) @ phP.T)
        liftM = lambda X: clM * np.einsum("ei,eqi->eq", np.einsum("eq,eqi->ei", X * wf, phM), phM)
        FvP, FvM = flux_v(uP, gP, ph), flux_v(uM, gM, ph)
        Fr = roe_flux(uP, uM, nrm, ph)
        uhat = [0.5 * (uP[v] + uM[v]) for v in range(m)]
        dual = visc_K(uP, [[(uP[v] - uhat[v]) * nrm[k] for k in range(2)] for v in range(m)], ph)
        dphPx = [sum(JiT[:, l, k][:, None, None] * dphP[l][None] for l in range(2)) for k in range(2)]
        for v in range(m):
            fhat = Fr[v]
            for k in range(2):
                fhat = fhat + (0.5 * (FvP[v][k] + FvM[v][k]) + eta * 0.5 * (liftP(KP[v][k]) + liftM(KM[v][k]))) * nrm[k]
            acc = (fhat * wf) @ phP
            for k in range(2):
                acc = acc - np.einsum("eq,eqi->ei", dual[v][k] * wf, dphPx[k])
            Rface[:, f, v, :] = JF[:, None] * acc
    return Rvol, Rface


def residual(mesh, ph, W, elems=None):
    Rvol, Rface = residual_parts(mesh, ph, W, elems)
    return Rvol + Rface.sum(axis=1)


def mass_apply(mesh, v, elems=None):
    """M v, M_e = |J_e| I (orthonormal basis, affine triangle)."""
    dJ = mesh.detJ if elems is None else mesh.detJ[np.asarray(elems, dtype=np.int64)]
    return dJ[:, None, None] * v


def jvp(mesh, ph, W, v, sigma, h=1e-30, elems=None):
    """K v = sigma M v + dR/dW v by the complex step (as ``oracle.dg.jvp``)."""
    scale = max(1.0, float(np.max(np.abs(v)))) if v.size else 1.0
    hh = h / scale
    Rc = residual(mesh, ph, W.astype(np.complex128) + 1j * hh * v, elems=elems)
    vt = v if elems is None else v[np.asarray(elems, dtype=np.int64)]
    return sigma * mass_apply(mesh, vt, elems) + Rc.imag / hh


def l2_project(mesh, f, nq_extra=3):
    """W_i = |J|^-1 int_K f psi_i of fields f(X) -> list of m arrays (X: (E, nq, 2))."""
    nq1d = mesh.p + 1 + nq_extra
    r, s, wq = tri_rule(nq1d)
    psi = dubiner(mesh.p, r, s).T
    vals = f(mesh.vol_points(np.stack([r, s], axis=1)))
    W = np.zeros((mesh.E, mesh.m, mesh.nm))
    for v in range(mesh.m):
        W[:, v, :] = (vals[v] * wq) @ psi
    return W


# ---------------------------------------------------------------- blocks / pMG
def colours(mesh):
    """Greedy colouring of the triangle graph in index order (no two face
    neighbours share a colour)."""
    col = np.zeros(mesh.E, dtype=np.int64)
    for e in range(mesh.E):
        used = {int(col[j]) for j in mesh.nbr[e] if j < e}
        c = 0
        while c in used:
            c += 1
        col[e] = c
    return col


def diag_blocks(mesh, ph, W, sigma, h=1e-30):
    """D_e = dR_e/dW_e + sigma |J_e| I (Sec. 5.1) by complex-step probing one
    colour class at a time, shape (E, nb, nb)."""
    col = colours(mesh)
    nm, nb = mesh.nm, mesh.nb
    D = np.zeros((mesh.E, nb, nb))
    for c in range(int(col.max()) + 1):
        tgt = np.nonzero(col == c)[0]
        for j in range(nb):
            Wc = W.astype(np.complex128)
            Wc[tgt, j // nm, j % nm] += 1j * h
            D[tgt, :, j] = (residual(mesh, ph, Wc, elems=tgt).imag / h).reshape(len(tgt), nb)
    D += sigma * mesh.detJ[:, None, None] * np.eye(nb)[None]
    return D


def offdiag_blocks(mesh, ph, W, p_coarse, h=1e-30):
    """O[e, f] = d R_e(edge f part) / d W_nbr(e, f) on the modes of degree <=
    p_coarse, shape (E, 3, nbc, nbc); an edge joining a triangle to itself
    stays zero (its coupling is in D)."""
    col = colours(mesh)
    nm = mesh.nm
    nmc = n_modes_tri(p_coarse)
    nbc = mesh.m * nmc
    O = np.zeros((mesh.E, 3, nbc, nbc))
    T = np.arange(mesh.E)
    for c in range(int(col.max()) + 1):
        src = np.nonzero(col == c)[0]
        hit = np.zeros(mesh.E, dtype=bool)
        for f in range(3):
            hit |= (col[mesh.nbr[:, f]] == c) & (mesh.nbr[:, f] != T)
        tgt = np.nonzero(hit)[0]
        if len(tgt) == 0:
            continue
        for jc in range(nbc):
            v, i = jc // nmc, jc % nmc
            Wc = W.astype(np.complex128)
            Wc[src, v, i] += 1j * h
            _, Rf = residual_parts(mesh, ph, Wc, elems=tgt)
            for f in range(3):
                nbf = mesh.nbr[tgt, f]
                ok = (col[nbf] == c) & (nbf != tgt)
                vals = (Rf[:, f, :, :nmc].imag / h).reshape(len(tgt), nbc)
                O[tgt[ok], f, :, jc] = vals[ok]
    return O


def bsr_apply(mesh, D, O, x):
    """(K_l x)_e = D_e x_e + sum_f O_e,f x_nbr(e, f) (Sec. 6.1)."""
    E, m, nmc = x.shape
    xf = x.reshape(E, m * nmc)
    y = np.einsum("eab,eb->ea", D, xf)
    for f in range(3):
        y += np.einsum("eab,eb->ea", O[:, f], xf[mesh.nbr[:, f]])
    return y.reshape(E, m, nmc)


def pmg_setup(mesh, ph, W, sigma, p_levels, nu_pre=10, nu_post=10, nu_coarse=30):
    """The p-multigrid of ``oracle.solvers.pmg_setup`` on a triangulation:
    matrix-free JVP on level 0, inherited (truncated) blocks below, block
    Jacobi smoothers."""
    from .blocks import truncate_block, BlockJacobi
    from .solvers import PMG
    m = mesh.m
    nm = [n_modes_tri(p) for p in p_levels]
    D0 = diag_blocks(mesh, ph, W, sigma)
    A = [lambda x: jvp(mesh, ph, W, x, sigma)]
    P = [BlockJacobi(D0, m, nm[0])]
    if len(p_levels) > 1:
        O1 = offdiag_blocks(mesh, ph, W, p_levels[1])
        for l in range(1, len(p_levels)):
            Dl = truncate_block(D0, m, nm[0], nm[l])
            Ol = truncate_block(O1, m, nm[1], nm[l])
            A.append(lambda x, Dl=Dl, Ol=Ol: bsr_apply(mesh, Dl, Ol, x))
            P.append(BlockJacobi(Dl, m, nm[l]))
    return PMG(A, P, nm, nu_pre, nu_post, nu_coarse)
