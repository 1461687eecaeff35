"""Pins of the oracle's block ILU(0) and its orderings (Sec. 6.3, Table
MGSettings): the defining property of ILU(0) (L U equals A on the pattern),
exactness where nothing is dropped, the MDF greedy on hand-worked graphs, and
the wavefront counts of the natural and colour orders on periodic grids."""
import numpy as np
import pytest

from oracle import bilu
from oracle import blocks as oblocks
from oracle.dg import Mesh
from oracle.physics import Physics


def grid_nbrs(n):
    """Face neighbour sets of a periodic grid, first index fastest."""
    d = len(n)
    E = int(np.prod(n))
    out = []
    for e in range(E):
        c, r = [], e
        for k in range(d):
            c.append(r % n[k])
            r //= n[k]
        s = set()
        for k in range(d):
            for dl in (-1, 1):
                cc = list(c)
                cc[k] = (cc[k] + dl) % n[k]
                f = 0
                for kk in reversed(range(d)):
                    f = f * n[kk] + cc[kk]
                if f != e:
                    s.add(f)
        out.append(s)
    return out


def random_blocks(nbrs, nb, rng, diag=6.0):
    A = {}
    for i, s in enumerate(nbrs):
        A[(i, i)] = rng.standard_normal((nb, nb)) + diag * np.eye(nb)
        for j in s:
            A[(i, j)] = rng.standard_normal((nb, nb))
    return A


def dense(blocks, E, nb, order, keys=None):
    pos = {e: p for p, e in enumerate(order)}
    M = np.zeros((E * nb, E * nb))
    for (i, j), B in blocks.items():
        if keys is None or (i, j) in keys:
            pi, pj = pos[i], pos[j]
            M[pi * nb:(pi + 1) * nb, pj * nb:(pj + 1) * nb] = B
    return M


def lu_dense(F, E, nb, order):
    pos = {e: p for p, e in enumerate(order)}
    L = np.eye(E * nb)
    U = np.zeros((E * nb, E * nb))
    for (i, j), B in F.items():
        pi, pj = pos[i], pos[j]
        tgt = L if pj < pi else U
        tgt[pi * nb:(pi + 1) * nb, pj * nb:(pj + 1) * nb] = B
    return L, U


@pytest.mark.parametrize("n,kind", [((4, 3), "natural"), ((4, 4), "colour"), ((3, 5), "natural"),
                                    ((2, 2, 3), "natural")])
def test_ilu0_matches_A_on_the_pattern(n, kind):
    """ILU(0) is defined by (L U)_ij = A_ij on the sparsity pattern with L unit
    lower and U upper triangular in the chosen order (Saad, Sec. 10.3)."""
    rng = np.random.default_rng(3)
    nbrs = grid_nbrs(n)
    E, nb = len(nbrs), 3
    A = random_blocks(nbrs, nb, rng)
    order = bilu.order_natural(E) if kind == "natural" else bilu.order_colour(nbrs)
    F = bilu.ilu0(A, nbrs, order)
    L, U = lu_dense(F, E, nb, order)
    Ad = dense(A, E, nb, order)
    mask = dense({k: np.ones((nb, nb)) for k in A}, E, nb, order) > 0
    LU = L @ U
    assert np.abs((LU - Ad)[mask]).max() < 1e-12 * np.abs(Ad).max()
    # something was dropped (the test is not vacuous): L U differs off the pattern
    assert np.abs(LU[~mask]).max() > 1e-3


def test_ilu0_is_exact_lu_on_a_complete_graph():
    rng = np.random.default_rng(4)
    E, nb = 5, 4
    nbrs = [set(range(E)) - {i} for i in range(E)]
    A = random_blocks(nbrs, nb, rng)
    order = [3, 0, 4, 1, 2]
    F = bilu.ilu0(A, nbrs, order)
    L, U = lu_dense(F, E, nb, order)
    Ad = dense(A, E, nb, order)
    assert np.abs(L @ U - Ad).max() < 1e-12 * np.abs(Ad).max()


def _coarse_ops(n, p, pc, seed=5):
    mesh = Mesh(2, n, (0.0, 0.0), (1.0, 1.3), p, p + 2)
    ph = Physics(gamma=1.4, Pr=0.72, mu=1e-3, Rgas=1.0, eta=None, roe_delta=0.1)
    rng = np.random.default_rng(seed)
    W = np.zeros((mesh.E, mesh.m, mesh.nm))
    W[:, 0, 0], W[:, 1, 0], W[:, 2, 0], W[:, 3, 0] = 2.0, 0.4, -0.2, 5.0
    W[:, :, 1:] = 0.05 * rng.standard_normal((mesh.E, mesh.m, mesh.nm - 1))
    from oracle.basis import n_modes
    nmc = n_modes(pc, 2)
    D = oblocks.truncate_block(oblocks.diag_blocks(mesh, ph, W, 3.0), mesh.m, mesh.nm, nmc)
    O = oblocks.offdiag_blocks(mesh, ph, W, pc)
    return mesh, D, O, nmc


def test_bilu_is_exact_on_a_two_element_mesh():
    """Two elements (joined through two faces): nothing can be dropped, so the
    preconditioner is the inverse of the coarse operator."""
    mesh, D, O, nmc = _coarse_ops((2, 1), 2, 1)
    P = bilu.BILU(mesh, D, O, mesh.m, nmc, "mdf")
    nb = mesh.m * nmc
    K = np.zeros((mesh.E * nb, mesh.E * nb))
    for c in range(mesh.E * nb):
        x = np.zeros((mesh.E, mesh.m, nmc))
        x.reshape(-1)[c] = 1.0
        K[:, c] = oblocks.bsr_apply(mesh, D, O, x).reshape(-1)
    r = np.random.default_rng(6).standard_normal((mesh.E, mesh.m, nmc))
    z = P(r)
    assert np.abs(z.reshape(-1) - np.linalg.solve(K, r.reshape(-1))).max() < 1e-12 * np.abs(z).max()


def test_no_fill_inside_the_pattern_without_triangles():
    """On a face graph without triangles (no periodic direction of 3 elements)
    the upper factor keeps A's off-diagonal blocks unchanged; with three
    elements in a direction it does not."""
    rng = np.random.default_rng(7)
    for n, free in (((4, 2), True), ((5, 4), True), ((3, 4), False)):
        nbrs = grid_nbrs(n)
        A = random_blocks(nbrs, 2, rng)
        order = bilu.order_natural(len(nbrs))
        F = bilu.ilu0(A, nbrs, order)
        same = all(np.array_equal(F[(i, j)], A[(i, j)]) for i in range(len(nbrs)) for j in nbrs[i] if j > i)
        assert same == free, n


def test_mdf_star_and_path_by_hand():
    # star: centre 0, leaves 1..3 not joined.  Leaves drop nothing (weight 0),
    # the centre drops the fill between its free leaves: sqrt(6) -> 1 goes first,
    # the centre now weighs sqrt(2) -> 2, the centre has one free leaf (0) and
    # ties with leaf 3 -> lowest index: 0, then 3
    nbrs = [{1, 2, 3}, {0}, {0}, {0}]
    c = {(i, j): 1.0 for i in range(4) for j in nbrs[i]}
    assert bilu.order_mdf(nbrs, c) == [1, 2, 0, 3]
    # path 0-1-2: ends weigh 0, the middle drops the (0,2) fill; after 0 goes,
    # 1 has one neighbour left and weighs 0 -> index order
    nbrs = [{1}, {0, 2}, {1}]
    c = {(0, 1): 2.0, (1, 0): 0.5, (1, 2): 3.0, (2, 1): 1.0}
    assert bilu.order_mdf(nbrs, c) == [0, 1, 2]


def test_mdf_weighted_four_cycle_by_hand():
    # 4-cycle 0-1-2-3-0 without chords: w_i = sqrt((c_ji c_ik)^2 + (c_ki c_ij)^2)
    nbrs = [{1, 3}, {0, 2}, {1, 3}, {2, 0}]
    c = {(0, 1): 1.0, (0, 3): 1.0, (1, 0): 1.0, (1, 2): 1.0,
         (2, 1): 0.1, (2, 3): 0.2, (3, 2): 1.0, (3, 0): 1.0}
    # w0 = sqrt((c10 c03)^2 + (c30 c01)^2) = sqrt(2); w1 = sqrt((c01 c12)^2 + (c21 c10)^2) = sqrt(1.01)
    # w2 = sqrt((c12 c23)^2 + (c32 c21)^2) = sqrt(0.05); w3 = sqrt((c23 c30)^2 + (c03 c32)^2) = sqrt(1.04)
    # -> 2 first; then 1 and 3 have one free neighbour (weight 0): 1, then 0 (one
    # neighbour left: 3), then 3
    assert bilu.order_mdf(nbrs, c) == [2, 1, 0, 3]


@pytest.mark.parametrize("n", [(4, 6), (5, 7), (2, 4), (4, 4, 4), (6, 2, 5), (16, 16, 16)])
def test_natural_order_wavefronts(n):
    """Natural order on a periodic grid: the level of (i, j[, k]) is i + j (+ k),
    so there are sum(n) - d + 1 levels; every level respects the lower neighbours."""
    nbrs = grid_nbrs(n)
    lev = bilu.levels(nbrs, bilu.order_natural(len(nbrs)))
    assert lev.max() + 1 == sum(n) - len(n) + 1
    for i in range(len(nbrs)):
        assert all(lev[k] < lev[i] for k in nbrs[i] if k < i)


@pytest.mark.parametrize("n,ncol", [((4, 6), 2), ((8, 8, 4), 2), ((5, 4), None), ((5, 4, 7), None)])
def test_colour_order_is_a_proper_colouring(n, ncol):
    """Even periodic grids are two-coloured (a checkerboard: two levels); odd
    ones need more, at most 2d + 1 for a greedy colouring of a graph of degree 2d."""
    nbrs = grid_nbrs(n)
    order = bilu.order_colour(nbrs)
    lev = bilu.levels(nbrs, order)
    if ncol is not None:
        assert lev.max() + 1 == ncol
    else:
        assert 3 <= lev.max() + 1 <= 2 * len(n) + 1
    assert all(lev[i] != lev[j] for i in range(len(nbrs)) for j in nbrs[i])
    assert sorted(order) == list(range(len(nbrs)))


def test_mdf_order_is_a_permutation_with_valid_levels():
    mesh, D, O, nmc = _coarse_ops((4, 5), 1, 0)
    P = bilu.BILU(mesh, D, O, mesh.m, nmc, "mdf")
    assert sorted(P.order) == list(range(mesh.E))
    lev = bilu.levels(P.nbrs, P.order)
    for i in range(mesh.E):
        assert all(lev[k] < lev[i] for k in P.nbrs[i] if P.pos[k] < P.pos[i])


@pytest.mark.parametrize("kind", ["mdf", "natural", "colour"])
def test_bilu_beats_block_jacobi_as_coarse_smoother(kind):
    """GMRES on the coarse operator: block ILU(0) keeps the neighbour couplings
    that block Jacobi drops, so the same number of iterations leaves a smaller
    residual (a property of this seeded case, the reason the coarsest level
    uses BILU in Table MGSettings)."""
    from oracle.solvers import gmres_fixed
    mesh, D, O, nmc = _coarse_ops((4, 5), 2, 1)
    K = lambda x: oblocks.bsr_apply(mesh, D, O, x)
    b = np.random.default_rng(8).standard_normal((mesh.E, mesh.m, nmc))
    res = {}
    for name, P in (("bj", oblocks.BlockJacobi(D, mesh.m, nmc)), (kind, bilu.BILU(mesh, D, O, mesh.m, nmc, kind))):
        x = gmres_fixed(K, P, b, np.zeros_like(b), 4)
        res[name] = np.linalg.norm(b - K(x)) / np.linalg.norm(b)
    assert res[kind] < res["bj"], res


def test_mdf_reduced_weights_closed_form():
    """c_ij = ||A_ii^{-1} A_ij||_F: with A_ii = a I and A_ij = b_ij I on nb x nb
    blocks, c_ij = |b_ij| / a * sqrt(nb)."""
    nb = 5
    nbrs = [{1, 2}, {0}, {0}]
    A = {(0, 0): 2.0 * np.eye(nb), (1, 1): 4.0 * np.eye(nb), (2, 2): 0.5 * np.eye(nb),
         (0, 1): 3.0 * np.eye(nb), (0, 2): -1.0 * np.eye(nb), (1, 0): 2.0 * np.eye(nb), (2, 0): 0.25 * np.eye(nb)}
    c = bilu.mdf_weights_c(A, nbrs)
    for (i, j), b in (((0, 1), 3.0), ((0, 2), -1.0), ((1, 0), 2.0), ((2, 0), 0.25)):
        a = A[(i, i)][0, 0]
        assert abs(c[(i, j)] - abs(b) / a * np.sqrt(nb)) < 1e-14
