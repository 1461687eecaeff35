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
