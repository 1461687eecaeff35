"""Krylov solvers and p-multigrid (Sec. 5.1, Sec. 6, Algorithms 1-2) and the
BDF2 Newton step that calls them.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* FGMRES (flexible GMRES, Saad 1993; Sec. 6): right preconditioned, so the
  Arnoldi residual estimate is the unpreconditioned residual ||b - K x|| and the
  stopping test is ||b - K x|| <= rtol ||b|| (Sec. 7.4).  The preconditioner
  may change every iteration (Z is stored).  Orthogonalisation: classical
  Gram-Schmidt applied twice (CGS2; the paper does not say which).  Givens
  rotations reduce the Hessenberg matrix to triangular form.
* SMOOTH / SOLVE: GMRES right-preconditioned by block Jacobi, a fixed number of
  iterations from the given initial guess, no restart (Sec. 6, Table MGSettings).
* MG_V (Algorithm 2) and MG_full (Algorithm 1), with b_l = I_0^l b_0 on every
  level and a zero initial guess for the recursive coarse correction.
"""
import numpy as np

from .blocks import restrict, prolong


def _dot(a, b):
    return float(np.dot(a.reshape(-1), b.reshape(-1)))


def _norm(a):
    return float(np.sqrt(_dot(a, a)))


def _givens(a, b):
    """c, s with [c s; -s c] [a; b] = [r; 0]."""
    r = float(np.hypot(a, b))
    if r == 0.0:
        return 1.0, 0.0
    return a / r, b / r


class _Arnoldi:
    """Shared Arnoldi/Givens bookkeeping for GMRES and FGMRES."""

    def __init__(self, r0, nmax):
        self.beta = _norm(r0)
        self.V = [r0 / self.beta] if self.beta > 0 else []
        self.Z = []
        self.H = np.zeros((nmax + 1, nmax))
        self.cs = np.zeros(nmax)
        self.sn = np.zeros(nmax)
        self.g = np.zeros(nmax + 1)
        self.g[0] = self.beta
        self.k = 0              # columns completed
        self.breakdown = False

    def step(self, z, w):
        """Append z (preconditioned direction) and w = K z; CGS2; Givens."""
        j = self.k
        self.Z.append(z)
        h1 = np.array([_dot(Vi, w) for Vi in self.V])
        w = w - sum(h1[i] * self.V[i] for i in range(len(self.V)))
        h2 = np.array([_dot(Vi, w) for Vi in self.V])
        w = w - sum(h2[i] * self.V[i] for i in range(len(self.V)))
        h = h1 + h2
        hn = _norm(w)
        self.H[:j + 1, j] = h
        self.H[j + 1, j] = hn
        for i in range(j):
            a, b = self.H[i, j], self.H[i + 1, j]
            self.H[i, j] = self.cs[i] * a + self.sn[i] * b
            self.H[i + 1, j] = -self.sn[i] * a + self.cs[i] * b
        c, s = _givens(self.H[j, j], self.H[j + 1, j])
        self.cs[j], self.sn[j] = c, s
        self.H[j, j] = c * self.H[j, j] + s * self.H[j + 1, j]
        self.H[j + 1, j] = 0.0
        self.g[j + 1] = -s * self.g[j]
        self.g[j] = c * self.g[j]
        self.k = j + 1
        if hn == 0.0:
            self.breakdown = True
        else:
            self.V.append(w / hn)
        return abs(self.g[j + 1])

    def update(self, x):
        """x + Z y with H[:k,:k] y = g[:k] (back substitution)."""
        k = self.k
        y = np.zeros(k)
        for i in reversed(range(k)):
            y[i] = (self.g[i] - self.H[i, i + 1:k] @ y[i + 1:k]) / self.H[i, i]
        out = x.copy()
        for i in range(k):
            out = out + y[i] * self.Z[i]
        return out


def gmres_fixed(A, P, b, x0, nu):
    """SMOOTH / SOLVE of Algorithm 2: nu iterations of right-preconditioned
    GMRES (preconditioner P) on A x = b from x0, no restart."""
    r0 = b - A(x0)
    arn = _Arnoldi(r0, nu)
    if arn.beta == 0.0:
        return x0.copy()
    for _ in range(nu):
        z = P(arn.V[arn.k])
        arn.step(z, A(z))
        if arn.breakdown:
            break
    return arn.update(x0)


class PMG:
    """p-multigrid levels l = 0 (fine) .. L (coarsest) with operators A[l],
    block-Jacobi preconditioners P[l] and mode counts nm[l] (Sec. 6)."""

    def __init__(self, A, P, nm, nu_pre=10, nu_post=10, nu_coarse=30):
        self.A, self.P, self.nm = A, P, nm
        self.L = len(A) - 1
        self.nu_pre = nu_pre if np.ndim(nu_pre) else [nu_pre] * (self.L + 1)
        self.nu_post = nu_post if np.ndim(nu_post) else [nu_post] * (self.L + 1)
        self.nu_coarse = nu_coarse

    def mg_v(self, l, b, x):
        """Algorithm 2, MG_V(l, b_l, x_l)."""
        if l == self.L:
            return gmres_fixed(self.A[l], self.P[l], b, x, self.nu_coarse)
        xb = gmres_fixed(self.A[l], self.P[l], b, x, self.nu_pre[l])
        r = b - self.A[l](xb)
        r1 = restrict(r, self.nm[l + 1])
        e1 = self.mg_v(l + 1, r1, np.zeros_like(r1))
        xh = xb + prolong(e1, self.nm[l])
        return gmres_fixed(self.A[l], self.P[l], b, xh, self.nu_post[l])

    def mg_full(self, b0):
        """Algorithm 1, MG_full: b_l = I_0^l b_0; SOLVE on level L; then for
        l = L-1..0 prolong the coarser result and run MG_V(l, b_l, x~_l)."""
        x = None
        for l in range(self.L, -1, -1):
            bl = restrict(b0, self.nm[l])
            if l == self.L:
                x = gmres_fixed(self.A[l], self.P[l], bl, np.zeros_like(bl), self.nu_coarse)
            else:
                x = self.mg_v(l, bl, prolong(x, self.nm[l]))
        return x

    __call__ = mg_full


def fgmres(K, Pinv, b, restart=30, max_restarts=0, rtol=1e-5, atol=0.0):
    """FGMRES(restart) for K x = b from x0 = 0 (Saad 1993; Sec. 6).

    Returns (x, stats) with stats = dict(iters, res0, res_final, rho, converged,
    history) where rho = (res_final/res0)^(1/iters) (Sec. 7.3)."""
    x = np.zeros_like(b)
    bnorm = _norm(b)
    tol = max(rtol * bnorm, atol)
    iters = 0
    hist = [bnorm]
    res = bnorm
    converged = res <= tol
    for cycle in range(max_restarts + 1):
        if converged:
            break
        r = b - K(x) if cycle > 0 else b.copy()
        arn = _Arnoldi(r, restart)
        if arn.beta <= tol:
            converged = True
            break
        for _ in range(restart):
            z = Pinv(arn.V[arn.k])
            res = arn.step(z, K(z))
            iters += 1
            hist.append(res)
            if res <= tol or arn.breakdown:
                break
        x = arn.update(x)
        converged = res <= tol or arn.breakdown
    rho = (res / bnorm) ** (1.0 / iters) if iters and bnorm > 0 else 0.0
    return x, dict(iters=iters, res0=bnorm, res_final=res, rho=rho,
                   converged=bool(converged), history=hist)


def bdf2_rhs(mesh, RW, Wk, Wn, Wnm1, dt):
    """BDF2 nonlinear residual f(W_k) = M (3 W_k - 4 W^n + W^{n-1})/(2 dt) + R(W_k);
    its Jacobian is K = 3/(2 dt) M + dR/dW, the form of eq. ODEDG with the
    shift 3/(2 dt) in place of 1/(a_ii dt)."""
    return mesh.detJ * (3.0 * Wk - 4.0 * Wn + Wnm1) / (2.0 * dt) + RW


def pmg_setup(mesh, ph, W, sigma, p_levels, nu_pre=10, nu_post=10, nu_coarse=30, coarse="bj", order="mdf"):
    """Assemble the p-multigrid preconditioner once (lagged, Sec. 7.4):
    fine diagonal blocks, neighbour blocks at the first coarse order (Sec. 6.3:
    off-diagonal blocks are only needed at coarse order), inheritance by
    truncation for every coarser level, PLU of every diagonal block.
    Level 0 applies the matrix-free exact K; levels >= 1 the inherited blocks.
    coarse="bilu": the coarsest level's smoother is preconditioned by block
    ILU(0) in the given order (Table MGSettings) instead of block Jacobi."""
    from .basis import n_modes
    from .blocks import diag_blocks, offdiag_blocks, truncate_block, BlockJacobi, bsr_apply
    from .dg import jvp
    d, m = mesh.d, mesh.m
    nm = [n_modes(p, d, mesh.space) for p in p_levels]
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
        if coarse == "bilu":
            from .bilu import BILU
            P[-1] = BILU(mesh, Dl, Ol, m, nm[-1], order)
    elif coarse != "bj":
        raise ValueError("block ILU needs a coarse level with neighbour blocks")
    return PMG(A, P, nm, nu_pre, nu_post, nu_coarse)
