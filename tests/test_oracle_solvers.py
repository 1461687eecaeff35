"""Pins of the oracle's Jacobian blocks, inheritance, PLU, GMRES/FGMRES and
p-multigrid (Sec. 5.1, Sec. 6, Algorithms 1-2) against dense linear algebra,
the JVP, minimal-residual optimality and special cases."""
import numpy as np
import pytest

from oracle import blocks, solvers
from oracle.dg import jvp, residual
from paper_1812_04789_gb300 import workloads as wl
from tests.helpers import oracle_mesh, oracle_physics, relmax


def _setup(cfg, amp=0.05):
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    return mesh, ph, wl.perturbed_state(cfg, amp=amp)


def _dense_K(mesh, ph, W, sigma):
    N = W.size
    K = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        K[:, j] = jvp(mesh, ph, W, e.reshape(W.shape), sigma).reshape(-1)
    return K


@pytest.mark.parametrize("n", [(1, 2, 3), (3, 3, 1), (2, 1, 2)])
def test_blocks_reassemble_jvp(n):
    """D_e and O_e,k,s (all modes) rebuild K exactly: (K x)_e = D_e x_e +
    sum O x_nbr, including directions with one or two elements."""
    cfg = wl.make_config("tgv", 3, n, 1, M=0.3, Re=50.0)
    mesh, ph, W = _setup(cfg)
    sigma = 2.0
    D = blocks.diag_blocks(mesh, ph, W, sigma)
    O = blocks.offdiag_blocks(mesh, ph, W, mesh.p)
    x = wl.random_vector(W.shape, 3)
    assert relmax(blocks.bsr_apply(mesh, D, O, x), jvp(mesh, ph, W, x, sigma)) < 1e-12


def test_diag_block_columns_are_local_jvp():
    cfg = wl.make_config("vortex", 2, (3, 4), 2, M=0.5, Re=100.0)
    mesh, ph, W = _setup(cfg)
    sigma = 1.5
    e0 = 5
    D = blocks.diag_blocks(mesh, ph, W, sigma, elems=[e0])
    for j in [0, 7, mesh.nb - 1]:
        v = np.zeros_like(W)
        v[e0, j // mesh.nm, j % mesh.nm] = 1.0
        col = jvp(mesh, ph, W, v, sigma)[e0].reshape(-1)
        np.testing.assert_allclose(D[0, :, j], col, atol=1e-12 * np.abs(col).max())


def test_galerkin_inheritance_identity():
    """K_1 x = I_0^1 K_0 I_1^0 x with the coarse blocks obtained by truncation
    (Sec. 6.1): truncate(JVP(zero-pad(x)))."""
    cfg = wl.make_config("tgv", 3, (3, 2, 3), 2, M=0.3, Re=50.0)
    mesh, ph, W = _setup(cfg)
    sigma = 1.0
    pc = 1
    nmc = wl.n_modes(pc, 3)
    D0 = blocks.diag_blocks(mesh, ph, W, sigma)
    O1 = blocks.offdiag_blocks(mesh, ph, W, pc)
    D1 = blocks.truncate_block(D0, mesh.m, mesh.nm, nmc)
    x = wl.random_vector((mesh.E, mesh.m, nmc), 4)
    lhs = blocks.bsr_apply(mesh, D1, O1, x)
    rhs = blocks.restrict(jvp(mesh, ph, W, blocks.prolong(x, mesh.nm), sigma), nmc)
    assert relmax(lhs, rhs) < 1e-12
    # truncating the level-1 neighbour blocks again gives level 2 directly
    O0 = blocks.offdiag_blocks(mesh, ph, W, 0)
    np.testing.assert_allclose(blocks.truncate_block(O1, mesh.m, nmc, 1), O0, atol=1e-12)


def test_plu_against_dense():
    rng = np.random.default_rng(9)
    for n in (1, 5, 24):
        A = rng.standard_normal((n, n))
        LU, perm = blocks.plu(A)
        L = np.tril(LU, -1) + np.eye(n)
        U = np.triu(LU)
        np.testing.assert_allclose(L @ U, A[perm], atol=1e-13 * n)
        assert np.all(np.abs(np.tril(LU, -1)) <= 1.0 + 1e-15)       # partial pivoting
        b = rng.standard_normal(n)
        np.testing.assert_allclose(blocks.plu_solve(LU, perm, b), np.linalg.solve(A, b),
                                   rtol=1e-11, atol=1e-12)
    # tie: equal |entries| pick the lowest row
    A = np.array([[1.0, 2.0], [-1.0, 3.0]])
    _, perm = blocks.plu(A)
    assert list(perm) == [0, 1]


def test_block_jacobi_exact_on_single_element():
    """One element (periodic in every direction): D_e is all of K, so BJ is
    exact and FGMRES(BJ) converges in one iteration (Sec. 6.3)."""
    cfg = wl.make_config("tgv", 3, (1, 1, 1), 2, M=0.3, Re=50.0)
    mesh, ph, W = _setup(cfg)
    sigma = 1.0
    D = blocks.diag_blocks(mesh, ph, W, sigma)
    BJ = blocks.BlockJacobi(D, mesh.m, mesh.nm)
    b = wl.random_vector(W.shape, 5)
    x, st = solvers.fgmres(lambda z: jvp(mesh, ph, W, z, sigma), BJ, b, rtol=1e-10)
    assert st["iters"] == 1
    assert relmax(jvp(mesh, ph, W, x, sigma), b) < 1e-10


def test_gmres_minimal_residual():
    """k unpreconditioned GMRES steps give the minimiser of ||b - A x|| over the
    Krylov space K_k(A, b) (computed by dense least squares)."""
    rng = np.random.default_rng(1)
    n = 12
    A = np.eye(n) * 3 + rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    for k in (1, 3, 6):
        x = solvers.gmres_fixed(lambda v: A @ v, lambda v: v, b, np.zeros(n), k)
        Kb = np.stack([np.linalg.matrix_power(A, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(Kb)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        np.testing.assert_allclose(x, Q @ y, rtol=1e-9, atol=1e-11)


def test_cgs2_orthonormal_basis():
    rng = np.random.default_rng(2)
    n = 40
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n))
    arn = solvers._Arnoldi(rng.standard_normal(n), 25)
    for _ in range(25):
        z = arn.V[arn.k]
        arn.step(z, A @ z)
    V = np.stack(arn.V, axis=1)
    np.testing.assert_allclose(V.T @ V, np.eye(V.shape[1]), atol=1e-13)


def test_fgmres_vs_dense_solve_with_bj():
    cfg = wl.make_config("vortex", 2, (3, 3), 2, M=0.5, Re=100.0)
    mesh, ph, W = _setup(cfg)
    sigma = 3.0 / (2 * 0.5)
    K = _dense_K(mesh, ph, W, sigma)
    b = wl.random_vector(W.shape, 6)
    BJ = blocks.BlockJacobi(blocks.diag_blocks(mesh, ph, W, sigma), mesh.m, mesh.nm)
    x, st = solvers.fgmres(lambda z: (K @ z.reshape(-1)).reshape(W.shape), BJ, b,
                           rtol=1e-9, restart=60)
    xd = np.linalg.solve(K, b.reshape(-1)).reshape(W.shape)
    assert st["converged"]
    assert np.linalg.norm(b - (K @ x.reshape(-1)).reshape(W.shape)) <= 1e-9 * np.linalg.norm(b) * 1.01
    assert relmax(x, xd) < 1e-6
    # with the exact inverse as preconditioner: one iteration
    Kinv = np.linalg.inv(K)
    x1, st1 = solvers.fgmres(lambda z: (K @ z.reshape(-1)).reshape(W.shape),
                             lambda r: (Kinv @ r.reshape(-1)).reshape(W.shape), b, rtol=1e-9)
    assert st1["iters"] == 1


def test_fgmres_restart_reaches_tolerance():
    rng = np.random.default_rng(4)
    n = 50
    A = np.diag(np.linspace(1, 30, n)) + 0.5 * rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    x, st = solvers.fgmres(lambda v: A @ v, lambda v: v, b, restart=5, max_restarts=200,
                           rtol=1e-8)
    assert st["converged"]
    assert np.linalg.norm(b - A @ x) <= 1.01e-8 * np.linalg.norm(b)


def test_pmg_two_levels_same_space_is_coarse_solve():
    """With a 'coarse' level equal to the fine space, MG_full starts from a
    converged coarse SOLVE, so its output solves K x = b (Algorithm 1)."""
    cfg = wl.make_config("vortex", 2, (3, 2), 1, M=0.5, Re=100.0)
    mesh, ph, W = _setup(cfg)
    sigma = 2.0
    mg = solvers.pmg_setup(mesh, ph, W, sigma, (1, 1), nu_pre=2, nu_post=2, nu_coarse=W.size)
    b = wl.random_vector(W.shape, 7)
    x = mg(b)
    assert relmax(jvp(mesh, ph, W, x, sigma), b) < 1e-8


def test_pmg_preconditioned_fgmres_step():
    """Full path on a small TGV: pMG 2-1-0 preconditioned FGMRES reaches the
    tolerance in fewer iterations than BJ alone; the result solves K x = b."""
    cfg = wl.make_config("tgv", 3, (3, 3, 2), 2, M=0.1, Re=1600.0, dt_conv=0.01)
    mesh, ph = oracle_mesh(cfg), oracle_physics(cfg)
    W = wl.initial_state(cfg)
    dt = wl.time_step(cfg)
    sigma = 1.5 / dt
    b = -residual(mesh, ph, W)
    K = lambda z: jvp(mesh, ph, W, z, sigma)
    mg = solvers.pmg_setup(mesh, ph, W, sigma, (2, 1, 0))
    x, st = solvers.fgmres(K, mg, b, rtol=1e-5)
    BJ = mg.P[0]
    x2, st2 = solvers.fgmres(K, BJ, b, rtol=1e-5, restart=30, max_restarts=5)
    assert st["converged"] and st2["converged"]
    assert st["iters"] <= st2["iters"]
    assert np.linalg.norm(b - K(x)) <= 1.0001e-5 * np.linalg.norm(b)
    assert relmax(x, x2) < 1e-3


# ------------------------------------------------------------------ Algorithm 2 written densely
def _truncation(E, m, nm_f, nm_c):
    """Dense restriction I_l^{l+1} of the [e][v][i] layout: row (e, v, i) of the
    coarse vector takes entry (e, v, i) of the fine one, i < nm_c (Sec. 6.1:
    M_{l+1,l} = [I 0] for an orthonormal hierarchical basis)."""
    R = np.zeros((E * m * nm_c, E * m * nm_f))
    for e in range(E):
        for v in range(m):
            for i in range(nm_c):
                R[(e * m + v) * nm_c + i, (e * m + v) * nm_f + i] = 1.0
    return R


def _block_jacobi_dense(A, nb):
    """Inverse of the element-diagonal part of A (blocks of size nb)."""
    P = np.zeros_like(A)
    for s in range(0, A.shape[0], nb):
        P[s:s + nb, s:s + nb] = np.linalg.inv(A[s:s + nb, s:s + nb])
    return P


def _gmres1(A, P, b, x):
    """One right-preconditioned GMRES iteration from x in closed form:
    x + alpha P r with alpha minimising ||r - alpha A P r||."""
    r = b - A @ x
    z = P @ r
    w = A @ z
    return x + (w @ r) / (w @ w) * z


def _dense_vcycle(A, P, R, l, b, x):
    """Algorithm 2 with one smoothing iteration before and after the coarse
    correction and an exact solve on the coarsest level; A[l] = R_l K R_l^T is
    the Galerkin coarse matrix, R[l] the restriction from level l to l + 1."""
    L = len(A) - 1
    if l == L:
        return np.linalg.solve(A[l], b)
    xb = _gmres1(A[l], P[l], b, x)
    r = b - A[l] @ xb
    e = _dense_vcycle(A, P, R, l + 1, R[l] @ r, np.zeros(R[l].shape[0]))
    xh = xb + R[l].T @ e
    return _gmres1(A[l], P[l], b, xh)


def _levels(mesh, K, p_levels):
    nms = [wl.n_modes(p, mesh.d) for p in p_levels]
    R = [_truncation(mesh.E, mesh.m, nms[l], nms[l + 1]) for l in range(len(nms) - 1)]
    A = [K]
    for Rl in R:
        A.append(Rl @ A[-1] @ Rl.T)
    P = [_block_jacobi_dense(A[l], mesh.m * nms[l]) for l in range(len(A))]
    return nms, R, A, P


def test_vcycle_two_levels_no_smoothing_is_coarse_correction():
    """MG_V(0, b, 0) with no smoothing and an exact coarsest solve is the
    coarse-grid correction alone: x = I^T A_1^{-1} I b with A_1 = I K I^T
    (Algorithm 2); MG_full then adds a second correction of the residual left
    by the first (Algorithm 1).  A dropped or sign-flipped correction fails."""
    cfg = wl.make_config("vortex", 2, (3, 2), 1, M=0.5, Re=100.0)
    mesh, ph, W = _setup(cfg)
    sigma = 2.0
    K = _dense_K(mesh, ph, W, sigma)
    nms, R, A, P = _levels(mesh, K, (1, 0))
    nc = A[1].shape[0]
    mg = solvers.pmg_setup(mesh, ph, W, sigma, (1, 0), nu_pre=0, nu_post=0, nu_coarse=nc)
    b = wl.random_vector(W.shape, 11)
    bf = b.reshape(-1)
    x = mg.mg_v(0, b, np.zeros_like(b)).reshape(-1)
    xd = R[0].T @ np.linalg.solve(A[1], R[0] @ bf)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    # MG_full: x1 = I^T A_1^-1 I b, then one more correction of b - K x1
    xf = mg.mg_full(b).reshape(-1)
    x1 = R[0].T @ np.linalg.solve(A[1], R[0] @ bf)
    xf_d = x1 + R[0].T @ np.linalg.solve(A[1], R[0] @ (bf - K @ x1))
    assert np.linalg.norm(xf - xf_d) <= 1e-9 * np.linalg.norm(xf_d)


def test_vcycle_three_levels_against_dense_algorithm():
    """Three levels p = 2, 1, 0 with one GMRES(BJ) smoothing step before and
    after each coarse correction and an exact coarsest solve: the oracle's
    MG_V and MG_full equal Algorithms 1-2 written with dense Galerkin matrices
    R K R^T (independent of the inherited BSR blocks), dense block-Jacobi
    inverses and GMRES(1) in closed form."""
    cfg = wl.make_config("vortex", 2, (3, 2), 2, M=0.5, Re=100.0)
    mesh, ph, W = _setup(cfg)
    sigma = 3.0
    K = _dense_K(mesh, ph, W, sigma)
    nms, R, A, P = _levels(mesh, K, (2, 1, 0))
    mg = solvers.pmg_setup(mesh, ph, W, sigma, (2, 1, 0), nu_pre=1, nu_post=1,
                           nu_coarse=A[2].shape[0])
    b = wl.random_vector(W.shape, 12)
    x0 = 0.1 * wl.random_vector(W.shape, 13)
    bf = b.reshape(-1)
    xv = mg.mg_v(0, b, x0).reshape(-1)
    xv_d = _dense_vcycle(A, P, R, 0, bf, x0.reshape(-1))
    assert np.linalg.norm(xv - xv_d) <= 1e-9 * np.linalg.norm(xv_d)
    # Algorithm 1: b_l = I_0^l b; coarsest solve; prolong and V-cycle upwards
    bl = [bf, R[0] @ bf, R[1] @ (R[0] @ bf)]
    x = np.linalg.solve(A[2], bl[2])
    for l in (1, 0):
        x = _dense_vcycle(A, P, R, l, bl[l], R[l].T @ x)
    xf = mg.mg_full(b).reshape(-1)
    assert np.linalg.norm(xf - x) <= 1e-9 * np.linalg.norm(x)
    # the coarse correction matters here: without it the result moves by O(1)
    xb = _gmres1(A[0], P[0], bf, x0.reshape(-1))
    assert np.linalg.norm(_gmres1(A[0], P[0], bf, xb) - xv_d) > 1e-3 * np.linalg.norm(xv_d)
