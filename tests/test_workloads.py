"""Checks of the seeded input generator against the paper's printed settings
(tests/golden/paper_settings.json) and exact projections."""
import json
import math
import os

import numpy as np
import pytest

from paper_1812_04789_gb300 import workloads as wl

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_settings.json")))


def test_vortex_is_the_papers_rescaled():
    """Sec. 7.1 vortex on [0, 0.1]^2 with R = 0.005, beta = 1/50; the workload
    scales lengths by 100, which leaves velocity and temperature fields unchanged."""
    g = GOLD["vortex"]
    scale = 10.0 / g["domain"][1]
    assert wl.CONFIGS["vortex2d_16_p2"]["hi"][0] == pytest.approx(g["domain"][1] * scale)
    cfg = dict(wl.CONFIGS["vortex2d_16_p2"])
    cfg["M"] = g["M_inf"]
    X = np.random.default_rng(0).uniform(0, 10, (50, 2))
    rho, ru, rv, E = wl.vortex_field(X, cfg, beta=g["beta"], Rv=g["R"] * scale)
    # the paper's formula evaluated directly on the unscaled domain
    gam = 1.4
    Uinf = g["M_inf"] * math.sqrt(gam)
    x, y = X[:, 0] / scale, X[:, 1] / scale
    r2 = ((x - 0.05) ** 2 + (y - 0.05) ** 2) / g["R"] ** 2
    u = Uinf * (1 - g["beta"] * (y - 0.05) / g["R"] * np.exp(-r2 / 2))
    v = Uinf * g["beta"] * (x - 0.05) / g["R"] * np.exp(-r2 / 2)
    T = 1 - Uinf**2 * g["beta"] ** 2 / (2 * gam / (gam - 1)) * np.exp(-r2)
    np.testing.assert_allclose(ru / rho, u, rtol=1e-13)
    np.testing.assert_allclose(rv / rho, v, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(rho, T ** (1 / (gam - 1)), rtol=1e-13)


def test_pmg_defaults_follow_table():
    lv = GOLD["mg_settings"]["levels"]
    assert [x[4] for x in lv] == [10, 10, 30]
    assert wl.CONFIGS["tgv16_p4"]["p_levels"][0] == 4


def test_projection_exact_for_polynomials():
    cfg = wl.make_config("tgv", 3, (2, 3, 2), 3)
    W = wl.project(cfg, lambda X: [1.0 + X[..., 0] * X[..., 1] ** 2] * 5)
    # mean of the field over each element = W[:, v, 0] * 2^{-3/2}
    W2 = wl.project(cfg, lambda X: [1.0 + X[..., 0] * X[..., 1] ** 2] * 5, nq_extra=6)
    np.testing.assert_allclose(W, W2, atol=1e-12)


def test_tgv_state_positive_and_shaped():
    cfg = wl.make_config("tgv", 3, (4, 4, 4), 2, M=0.1)
    W = wl.initial_state(cfg)
    assert W.shape == (64, 5, 10)
    assert np.all(W[:, 0, 0] > 0)
    # zero mean momentum (odd symmetry)
    assert abs(W[:, 1, 0].sum()) < 1e-12 and abs(W[:, 2, 0].sum()) < 1e-12


def test_batch_cases_seeded():
    a = wl.batch_cases(8)
    b = wl.batch_cases(8)
    assert a == b and len(a) == 8
    assert all(1 <= c["p"] <= 5 and 8 <= c["n"][0] <= 24 for c in a)


def test_tri_mesh_seeded_ccw_and_covering():
    cfg = wl.tri_config((5, 4), 2)
    a, b = wl.tri_mesh(cfg), wl.tri_mesh(cfg)
    for k in ("X", "tri", "shift"):
        assert np.array_equal(a[k], b[k])                       # same seed, same mesh
    other = wl.tri_mesh(dict(cfg, seed=7))
    assert not np.array_equal(other["X"], a["X"])
    L = a["hi"] - a["lo"]
    V = a["X"][a["tri"]] + a["shift"] * L[None, None, :]
    area = 0.5 * ((V[:, 1, 0] - V[:, 0, 0]) * (V[:, 2, 1] - V[:, 0, 1])
                  - (V[:, 2, 0] - V[:, 0, 0]) * (V[:, 1, 1] - V[:, 0, 1]))
    assert np.all(area > 0.0)                                    # counter-clockwise
    assert abs(area.sum() - L[0] * L[1]) < 1e-9 * L[0] * L[1]    # the triangles tile the box
    assert a["tri"].shape == (2 * 5 * 4, 3) and wl.tri_state_shape(cfg) == (40, 4, 6)


def test_tri_projection_exact_for_polynomials():
    """The Dubiner projection reproduces a field of degree <= p at any point."""
    from scipy.special import eval_jacobi
    cfg = wl.tri_config((3, 2), 3)
    f = lambda X: [1.0 + 0.1 * X[..., 0] ** 2 * X[..., 1] - 0.02 * X[..., 1] ** 3 + 0.0 * X[..., 0]] * 4
    W = wl.tri_project(cfg, f)
    msh = wl.tri_mesh(cfg)
    L = msh["hi"] - msh["lo"]
    V = msh["X"][msh["tri"]] + msh["shift"] * L[None, None, :]
    r, s = 0.1 - 0.7, -0.35                                      # one reference point inside T
    a, b = 2.0 * (1.0 + r) / (1.0 - s) - 1.0, s
    psi = np.array([math.sqrt(2.0) * eval_jacobi(i, 0, 0, a) / math.sqrt(2.0 / (2 * i + 1))
                    * eval_jacobi(j, 2 * i + 1, 0, b) / math.sqrt(2.0 ** (2 * i + 2) / (2 * j + 2 * i + 2))
                    * (1.0 - b) ** i for i, j in wl.tri_modes(3)])
    X = V[:, 0] + (r + 1.0) / 2.0 * (V[:, 1] - V[:, 0]) + (s + 1.0) / 2.0 * (V[:, 2] - V[:, 0])
    exact = f(X[:, None, :])[0][:, 0]
    assert np.abs(W[:, 0, :] @ psi - exact).max() < 1e-12
