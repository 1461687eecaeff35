"""Jacobian blocks, subspace inheritance and element block-Jacobi (Sec. 5.1,
Sec. 6.1, Sec. 6.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Iteration matrix K = sigma M + dR/dW (eq. ODEDG) in block form:
  D_e      = dR_e/dW_e + sigma |J| I              (diagonal block, total derivative:
                                                   a direction with one element makes
                                                   the element its own neighbour)
  O_e,k,s  = dR_e/dW_nbr(e,k,s) through face (k, s)  (zero when nbr = e)
so that (K x)_e = D_e x_e + sum_{k,s} O_e,k,s x_nbr(e,k,s).

Blocks are taken by complex-step differentiation of the residual: every
element of one colour class is perturbed at once in the same local direction;
the colouring makes face neighbours differ in colour, so each R_e (or each face
part of R_e) sees exactly one perturbed element.

Inheritance (Sec. 6.1): with an orthonormal hierarchical basis on affine
elements, M_{l+1} = |J| I and M_{l+1,l} = [I 0], so the coarse block is the
leading n_m(p_{l+1}) x n_m(p_{l+1}) sub-block of every variable pair, for the
diagonal and the off-diagonal blocks alike; restriction keeps the leading
modes and prolongation (its transpose) pads zeros.
"""
import numpy as np

from .dg import residual_parts
from .basis import n_modes


def _colour_1d(i, n):
    if n == 1:
        return np.zeros_like(i)
    if n % 2 == 0:
        return i % 2
    return np.where(i == n - 1, 2, i % 2)


def colours(mesh):
    """A proper colouring of the periodic face-neighbour graph with <= 3
    colours: sum_k c_k(i_k) mod 3 with neighbouring c_k differing mod 3."""
    c = np.zeros(mesh.E, dtype=np.int64)
    for k in range(mesh.d):
        c = c + _colour_1d(mesh.ijk[:, k], mesh.n[k])
    return c % 3


def diag_blocks(mesh, ph, W, sigma, elems=None, h=1e-30):
    """D_e = dR_e/dW_e + sigma |J| I for the requested elements, (nT, nb, nb),
    rows and columns in the [v][i] layout of W[e]."""
    T = np.arange(mesh.E) if elems is None else np.asarray(elems, dtype=np.int64)
    col = colours(mesh)
    nb, nm = mesh.nb, mesh.nm
    D = np.zeros((len(T), nb, nb))
    pos = {int(e): r for r, e in enumerate(T)}
    for c in np.unique(col[T]):
        tgt = T[col[T] == c]
        rows = np.array([pos[int(e)] for e in tgt])
        for j in range(nb):
            Wc = W.astype(np.complex128)
            Wc[tgt, j // nm, j % nm] += 1j * h
            Rv, Rf = residual_parts(mesh, ph, Wc, elems=tgt)
            R = Rv + Rf.sum(axis=(1, 2))
            D[rows, :, j] = (R.imag / h).reshape(len(tgt), nb)
    D += sigma * mesh.detJ * np.eye(nb)[None]
    return D


def offdiag_blocks(mesh, ph, W, p_coarse, elems=None, h=1e-30):
    """O_e,k,s restricted to the modes of degree <= p_coarse (rows and columns),
    shape (nT, d, 2, nbc, nbc) with nbc = m n_m(p_coarse)."""
    T = np.arange(mesh.E) if elems is None else np.asarray(elems, dtype=np.int64)
    col = colours(mesh)
    d, m, nm = mesh.d, mesh.m, mesh.nm
    nmc = n_modes(p_coarse, d, mesh.space)
    nbc = m * nmc
    O = np.zeros((len(T), d, 2, nbc, nbc))
    for c in range(3):
        src = np.nonzero(col == c)[0]
        if len(src) == 0:
            continue
        hit = np.zeros(len(T), dtype=bool)
        for k in range(d):
            for side in range(2):
                nb = mesh.nbr[T, k, side]
                hit |= (col[nb] == c) & (nb != T)
        if not hit.any():
            continue
        rows = np.nonzero(hit)[0]
        tgt = T[rows]
        for jc in range(nbc):
            v, i = jc // nmc, jc % nmc
            Wc = W.astype(np.complex128)
            Wc[src, v, i] += 1j * h
            _, Rf = residual_parts(mesh, ph, Wc, elems=tgt)
            for k in range(d):
                for side in range(2):
                    nb = mesh.nbr[tgt, k, side]
                    ok = (col[nb] == c) & (nb != tgt)
                    vals = (Rf[:, k, side, :, :nmc].imag / h).reshape(len(tgt), nbc)
                    O[rows[ok], k, side, :, jc] = vals[ok]
    return O


def truncate_block(B, m, nm_from, nm_to):
    """Leading sub-block per variable pair: [..., m nm_from, m nm_from] ->
    [..., m nm_to, m nm_to] (inheritance with M_{l+1,l} = [I 0], Sec. 6.1)."""
    lead = B.shape[:-2]
    X = B.reshape(lead + (m, nm_from, m, nm_from))
    return X[..., :, :nm_to, :, :nm_to].reshape(lead + (m * nm_to, m * nm_to))


def restrict(x, nm_to):
    """I_l^{l+1}: L2 projection onto the coarser space = keep leading modes."""
    return x[:, :, :nm_to].copy()


def prolong(x, nm_to):
    """I_{l+1}^l = (I_l^{l+1})^T: pad the finer modes with zeros."""
    out = np.zeros(x.shape[:2] + (nm_to,), dtype=x.dtype)
    out[:, :, :x.shape[2]] = x
    return out


def plu(A):
    """PLU factorisation with partial pivoting (Sec. 6.3: BJ factorises each
    diagonal block by PLU).  Pivot: largest |entry| in the column, lowest row
    index on ties.  Returns (LU, perm) with A[perm] = L U, L unit lower."""
    LU = np.array(A, dtype=np.float64, copy=True)
    n = LU.shape[0]
    perm = np.arange(n)
    for k in range(n):
        r = k + int(np.argmax(np.abs(LU[k:, k])))        # argmax takes the first max
        if r != k:
            LU[[k, r]] = LU[[r, k]]
            perm[[k, r]] = perm[[r, k]]
        piv = LU[k, k]
        if piv == 0.0:
            raise ZeroDivisionError("singular block")
        LU[k + 1:, k] /= piv
        LU[k + 1:, k + 1:] -= np.outer(LU[k + 1:, k], LU[k, k + 1:])
    return LU, perm


def plu_solve(LU, perm, b):
    """Solve A x = b from plu(A): forward then backward substitution."""
    n = LU.shape[0]
    y = np.array(b, dtype=np.float64)[perm]
    for i in range(n):
        y[i] -= LU[i, :i] @ y[:i]
    for i in reversed(range(n)):
        y[i] = (y[i] - LU[i, i + 1:] @ y[i + 1:]) / LU[i, i]
    return y


class BlockJacobi:
    """Element-wise block Jacobi (Sec. 6.3): factor every diagonal block by PLU
    and apply z_e = D_e^{-1} r_e."""

    def __init__(self, D, m, nm):
        self.m, self.nm = m, nm
        self.fac = [plu(Di) for Di in D]

    def __call__(self, r):
        E = r.shape[0]
        z = np.zeros_like(r)
        for e in range(E):
            LU, perm = self.fac[e]
            z[e] = plu_solve(LU, perm, r[e].reshape(-1)).reshape(self.m, self.nm)
        return z


def bsr_apply(mesh, D, O, x):
    """Inherited coarse operator (K_l x)_e = D_e x_e + sum O_e,k,s x_nbr (Sec. 6.1)."""
    E, m, nmc = x.shape
    xf = x.reshape(E, m * nmc)
    y = np.einsum("eab,eb->ea", D, xf)
    for k in range(mesh.d):
        for side in range(2):
            y += np.einsum("eab,eb->ea", O[:, k, side], xf[mesh.nbr[:, k, side]])
    return y.reshape(E, m, nmc)
