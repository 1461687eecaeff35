"""Element block ILU(0) of the coarsest p-multigrid level and its orderings
(Sec. 6.3, Table MGSettings: GMRES preconditioned by BILU on the coarsest
level).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The matrix is the inherited coarse operator of Sec. 6.1: one block A_ii per
element (the diagonal block, which already holds any coupling of an element
with itself through a periodic direction of one element) and one block A_ij
per pair of face neighbours (the sum of the face blocks when two faces join the
same pair).  Its block sparsity pattern is the element face graph.

* ILU(0): block incomplete LU with zero fill, the textbook IKJ form taken in the
  chosen element order: rows in order; for each lower neighbour k of row i (in
  order) L_ik = A_ik U_kk^{-1} and A_ij -= L_ik U_kj for every j of the
  pattern of both rows; entries outside the pattern are dropped.  Apply:
  forward substitution with the unit lower factor, backward with the upper.
* Orderings.  MDF (minimum discarded fill, the reordering the paper uses for
  ILU(0)): with c_ij = ||A_ii^{-1} A_ij||_F, the weight of a not yet ordered
  element i is the Frobenius norm of the fill its elimination would drop,
  w_i = sqrt(sum (c_ji c_ik)^2) over ordered pairs (j, k) of distinct not yet
  ordered neighbours of i that are not neighbours of each other; the element
  of least weight comes next (lowest index on ties) and its neighbours'
  weights are recomputed.  Natural: element index order.  Colour: greedy
  colouring in index order (each element takes the least colour no lower
  indexed neighbour has), elements sorted by (colour, index).
* Level schedule of an order: an element's level is one more than the
  highest level of its neighbours that come before it (0 if none), so that the
  substitutions can treat one level at a time.
"""
import heapq

import numpy as np


def neighbour_sets(mesh):
    """Face neighbours of every element, without the element itself."""
    return [set(int(j) for j in mesh.nbr[e].reshape(-1) if j != e) for e in range(mesh.E)]


def coarse_matrix(mesh, D, O):
    """Block dictionary {(i, j): block} of the inherited operator
    (K x)_e = D_e x_e + sum_{k,s} O_e,k,s x_nbr(e,k,s) (Sec. 6.1): self couplings
    go to the diagonal, the blocks of two faces joining the same pair add."""
    A = {}
    for e in range(mesh.E):
        A[(e, e)] = np.array(D[e], dtype=np.float64, copy=True)
        for k in range(mesh.d):
            for side in range(2):
                j = int(mesh.nbr[e, k, side])
                A[(e, j)] = A.get((e, j), 0.0) + O[e, k, side]
    return A


def order_natural(E):
    return list(range(E))


def order_colour(nbrs):
    E = len(nbrs)
    col = [0] * E
    for i in range(E):
        used = {col[j] for j in nbrs[i] if j < i}
        c = 0
        while c in used:
            c += 1
        col[i] = c
    return sorted(range(E), key=lambda i: (col[i], i))


def mdf_weights_c(A, nbrs):
    """c_ij = ||A_ii^{-1} A_ij||_F for every neighbour pair."""
    c = {}
    for i, nb in enumerate(nbrs):
        for j in nb:
            c[(i, j)] = float(np.linalg.norm(np.linalg.solve(A[(i, i)], A[(i, j)])))
    return c


def order_mdf(nbrs, c):
    """Minimum discarded fill ordering from the reduced weights c[(i, j)]."""
    E = len(nbrs)
    done = [False] * E

    def weight(i):
        rest = sorted(j for j in nbrs[i] if not done[j])
        s = 0.0
        for j in rest:
            for k in rest:
                if j != k and k not in nbrs[j]:
                    s += (c[(j, i)] * c[(i, k)]) ** 2
        return float(np.sqrt(s))

    w = [weight(i) for i in range(E)]
    heap = [(w[i], i) for i in range(E)]
    heapq.heapify(heap)
    order = []
    while heap:
        wi, i = heapq.heappop(heap)
        if done[i] or wi != w[i]:
            continue                      # stale entry
        done[i] = True
        order.append(i)
        for j in nbrs[i]:
            if not done[j]:
                w[j] = weight(j)
                heapq.heappush(heap, (w[j], j))
    return order


def levels(nbrs, order):
    """Level of every element in the given order (see the module docstring)."""
    pos = np.empty(len(order), dtype=np.int64)
    pos[np.asarray(order)] = np.arange(len(order))
    lev = np.zeros(len(order), dtype=np.int64)
    for i in order:
        lo = [lev[k] + 1 for k in nbrs[i] if pos[k] < pos[i]]
        lev[i] = max(lo) if lo else 0
    return lev


def ilu0(A, nbrs, order):
    """Block ILU(0) in the given order.  Returns the factor dictionary F with
    F[(i, k)] = L_ik for k before i and F[(i, j)] = U_ij for j = i or after."""
    pos = {e: p for p, e in enumerate(order)}
    F = {key: np.array(v, dtype=np.float64, copy=True) for key, v in A.items()}
    for i in order:
        row = sorted(nbrs[i] | {i}, key=lambda j: pos[j])
        for k in row:
            if pos[k] >= pos[i]:
                break
            # L_ik = A_ik U_kk^{-1}
            F[(i, k)] = np.linalg.solve(F[(k, k)].T, F[(i, k)].T).T
            for j in row:
                if pos[j] > pos[k] and (k, j) in F:
                    F[(i, j)] = F[(i, j)] - F[(i, k)] @ F[(k, j)]
    return F


class BILU:
    """z = (L U)^{-1} r for the coarse operator (D, O) of ``mesh`` (Sec. 6.3);
    ``kind`` is "mdf", "natural" or "colour"."""

    def __init__(self, mesh, D, O, m, nm, kind="mdf"):
        self.m, self.nm = m, nm
        self.nbrs = neighbour_sets(mesh)
        A = coarse_matrix(mesh, D, O)
        if kind == "mdf":
            self.order = order_mdf(self.nbrs, mdf_weights_c(A, self.nbrs))
        elif kind == "natural":
            self.order = order_natural(mesh.E)
        elif kind == "colour":
            self.order = order_colour(self.nbrs)
        else:
            raise ValueError(kind)
        self.pos = {e: p for p, e in enumerate(self.order)}
        self.F = ilu0(A, self.nbrs, self.order)

    def __call__(self, r):
        E = r.shape[0]
        rf = r.reshape(E, -1)
        y = np.zeros_like(rf)
        for i in self.order:                      # L y = r, L unit lower
            acc = rf[i].copy()
            for k in self.nbrs[i]:
                if self.pos[k] < self.pos[i]:
                    acc -= self.F[(i, k)] @ y[k]
            y[i] = acc
        z = np.zeros_like(rf)
        for i in reversed(self.order):            # U z = y
            acc = y[i].copy()
            for j in self.nbrs[i]:
                if self.pos[j] > self.pos[i]:
                    acc -= self.F[(i, j)] @ z[j]
            z[i] = np.linalg.solve(self.F[(i, i)], acc)
        return z.reshape(r.shape)
