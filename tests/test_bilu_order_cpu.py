"""The library's host-side block ILU(0) ordering (dg_bilu_order, Sec. 6.3)
against the oracle's: MDF, natural and colour orders and their level schedules,
integer results compared exactly.  Pure host code: no GPU is used."""
import numpy as np
import pytest

from oracle import bilu as obilu
from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    B.load()


def face_nbr(n):
    """[E][2d] face neighbours of a periodic grid (s = 2k + side, side 0 = -1)."""
    d = len(n)
    E = int(np.prod(n))
    out = np.zeros((E, 2 * d), dtype=np.int32)
    for e in range(E):
        c, r = [], e
        for k in range(d):
            c.append(r % n[k])
            r //= n[k]
        for k in range(d):
            for side, dl in enumerate((-1, 1)):
                cc = list(c)
                cc[k] = (cc[k] + dl) % n[k]
                f = 0
                for kk in reversed(range(d)):
                    f = f * n[kk] + cc[kk]
                out[e, 2 * k + side] = f
    return out


def sets(nbr):
    return [set(int(j) for j in row if j != e) for e, row in enumerate(nbr)]


def pair_weights(nbr, rng):
    """Random c_ij per distinct neighbour pair, laid out per face (first face of a pair)."""
    E, nf = nbr.shape
    cpair = {}
    cf = np.full((E, nf), -1.0)
    for e in range(E):
        for s in range(nf):
            j = int(nbr[e, s])
            if j == e or (e, j) in cpair:
                continue
            cpair[(e, j)] = 0.5 + rng.random()
            cf[e, s] = cpair[(e, j)]
    return cf, cpair


@pytest.mark.parametrize("n", [(4, 6), (5, 2), (2, 1), (4, 4, 2), (6, 5, 4)])
def test_natural_and_colour_match_the_oracle(n):
    nbr = face_nbr(n)
    ns = sets(nbr)
    for kind, ref in ((B.ORDER_NATURAL, obilu.order_natural(len(ns))), (B.ORDER_COLOUR, obilu.order_colour(ns))):
        order, level, nl = B.bilu_order(nbr, kind)
        assert order.tolist() == list(ref)
        lev = obilu.levels(ns, ref)
        assert level.tolist() == lev.tolist() and nl == lev.max() + 1


@pytest.mark.parametrize("n,seed", [((4, 6), 0), ((5, 4), 1), ((4, 4, 4), 2), ((2, 6), 3), ((8, 6, 2), 4)])
def test_mdf_matches_the_oracle(n, seed):
    nbr = face_nbr(n)
    ns = sets(nbr)
    cf, cpair = pair_weights(nbr, np.random.default_rng(seed))
    ref = obilu.order_mdf(ns, cpair)
    order, level, nl = B.bilu_order(nbr, B.ORDER_MDF, cf)
    assert order.tolist() == ref
    lev = obilu.levels(ns, ref)
    assert level.tolist() == lev.tolist() and nl == lev.max() + 1


def test_mdf_hand_graphs():
    # star and weighted 4-cycle of the oracle pins, given as face lists (-> self for unused faces)
    star = np.array([[1, 2, 3], [0, 1, 1], [0, 2, 2], [0, 3, 3]], dtype=np.int32)
    cf = np.array([[1.0, 1.0, 1.0], [1.0, -1, -1], [1.0, -1, -1], [1.0, -1, -1]])
    assert B.bilu_order(star, B.ORDER_MDF, cf)[0].tolist() == [1, 2, 0, 3]
    cyc = np.array([[1, 3], [0, 2], [1, 3], [2, 0]], dtype=np.int32)
    cf = np.array([[1.0, 1.0], [1.0, 1.0], [0.1, 0.2], [1.0, 1.0]])
    assert B.bilu_order(cyc, B.ORDER_MDF, cf)[0].tolist() == [2, 1, 0, 3]


def test_rejects_bad_input():
    nbr = face_nbr((4, 4))
    with pytest.raises(B.DGError):
        B.bilu_order(nbr, B.ORDER_MDF)          # MDF needs the weights
    bad = nbr.copy()
    bad[3, 1] = 99
    with pytest.raises(B.DGError):
        B.bilu_order(bad, B.ORDER_NATURAL)
    with pytest.raises(B.DGError):
        B.bilu_order(nbr, 7)
