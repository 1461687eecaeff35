"""Seeded synthetic inputs: mesh descriptors, physics parameters and modal
initial states of the paper's workloads.

This module holds no residual, Jacobian or solver arithmetic.  It knows the
state layout (W[e, v, i]: element, conservative variable, mode, with modes of
the total-degree space ordered by degree and then lexicographically with the
first index descending) and computes modal coefficients of closed-form
initial fields by L2 projection with numpy's own Legendre and Gauss-Legendre
routines.  Both the CUDA library's tests/bench and the CPU oracle's tests take
their inputs from here; nothing here calls either.

Workloads
  * isentropic vortex advected by a uniform stream (Sec. 7.1 of the paper,
    rescaled from [0, 0.1]^2 to [0, 10]^2: R = 0.5, beta = 1/50, centre (5, 5));
  * Taylor-Green vortex on [0, 2 pi]^3 (standard literature definition; the
    paper has 2-D cases only).
Nondimensionalisation: rho_inf = p_inf = T_inf = R_gas = 1, c_inf = sqrt(gamma);
vortex: U_inf = M sqrt(gamma), mu = U_inf L / Re with L = 10 (domain size);
TGV: V0 = M sqrt(gamma), mu = V0 / Re (L = 1).  Time steps are given in
convective units t_c = L / U_ref and converted to physical time.
"""
import itertools
import math

import numpy as np

SEED = 1812_04789


def mode_list(p, d, space="P"):
    """Mode multi-indices: total degree <= p ("P") or every 1-D degree <= p ("Q"),
    ordered by degree (total, resp. largest 1-D), then first index descending."""
    out = []
    for s in range(p + 1):
        if space == "Q":
            lv = [a for a in itertools.product(range(s + 1), repeat=d) if max(a) == s]
        else:
            lv = [a for a in itertools.product(range(s + 1), repeat=d) if sum(a) == s]
        lv.sort(reverse=True)
        out.extend(lv)
    return out


def n_modes(p, d, space="P"):
    return (p + 1) ** d if space == "Q" else math.comb(p + d, d)


CONFIGS = {
    # 2-D vortex, 16^2 quads, p = 2, BDF2 dt = 0.05 t_c, FGMRES(30) 1e-5, BJ only
    "vortex2d_16_p2": dict(case="vortex", dim=2, n=(16, 16, 1), lo=(0.0, 0.0, 0.0),
                           hi=(10.0, 10.0, 1.0), p=2, M=0.5, Re=1000.0, dt_conv=0.05,
                           p_levels=(2,)),
    # 3-D TGV, 16^3 hexes, p = 4, pMG 4-2-1-0, BDF2 dt = 0.01 t_c
    "tgv16_p4": dict(case="tgv", dim=3, n=(16, 16, 16), lo=(0.0,) * 3,
                     hi=(2 * math.pi,) * 3, p=4, M=0.1, Re=1600.0, dt_conv=0.01,
                     p_levels=(4, 2, 1, 0)),
    # 3-D TGV, 32^3 hexes, p = 6, low Mach stiff case, pMG 6-2-1-0
    "tgv32_p6": dict(case="tgv", dim=3, n=(32, 32, 32), lo=(0.0,) * 3,
                     hi=(2 * math.pi,) * 3, p=6, M=0.05, Re=1600.0, dt_conv=0.01,
                     p_levels=(6, 2, 1, 0)),
}


def make_config(case, dim, n, p, M=0.1, Re=1600.0, dt_conv=0.01, p_levels=None, lo=None,
                hi=None, space="P"):
    """A workload dict of the same shape as CONFIGS entries (smaller meshes for
    tests)."""
    n = tuple(n) + (1,) * (3 - len(n))
    if case == "vortex":
        lo = lo or (0.0, 0.0, 0.0)
        hi = hi or (10.0, 10.0, 1.0)
    else:
        lo = lo or (0.0,) * 3
        hi = hi or (2 * math.pi,) * 3
    return dict(case=case, dim=dim, n=n, lo=lo, hi=hi, p=p, M=M, Re=Re, dt_conv=dt_conv,
                p_levels=tuple(p_levels) if p_levels else (p,), space=space)


def n_elements(cfg):
    return int(np.prod(cfg["n"][: cfg["dim"]]))


def state_shape(cfg, p=None):
    d = cfg["dim"]
    return (n_elements(cfg), d + 2, n_modes(cfg["p"] if p is None else p, d, cfg.get("space", "P")))


def ref_speed_length(cfg, gamma=1.4):
    u = cfg["M"] * math.sqrt(gamma)
    L = (cfg["hi"][0] - cfg["lo"][0]) if cfg["case"] == "vortex" else 1.0
    return u, L


def physics(cfg, gamma=1.4, Pr=0.72, roe_delta=0.1, eta=None):
    u, L = ref_speed_length(cfg, gamma)
    mu = u * L / cfg["Re"]
    d = cfg["dim"]
    return dict(gamma=gamma, Pr=Pr, mu=mu, Rgas=1.0,
                eta=float(2 * d + 1) if eta is None else float(eta), roe_delta=roe_delta)


def time_step(cfg, gamma=1.4):
    u, L = ref_speed_length(cfg, gamma)
    return cfg["dt_conv"] * L / u


def mesh_desc(cfg, nq1d=None):
    return dict(dim=cfg["dim"], n=tuple(cfg["n"]), lo=tuple(cfg["lo"]), hi=tuple(cfg["hi"]),
                p=cfg["p"], nq1d=(cfg["p"] + 2) if nq1d is None else nq1d,
                space=cfg.get("space", "P"))


# ---------------------------------------------------------------- closed forms
def vortex_field(X, cfg, t=0.0, gamma=1.4, beta=1.0 / 50.0, Rv=0.5):
    """Conservative state of the isentropic vortex (Sec. 7.1) at points X[..., 2],
    translated by U_inf t along x (periodic, nearest image)."""
    Uinf, L = ref_speed_length(cfg, gamma)
    Lx = cfg["hi"][0] - cfg["lo"][0]
    Ly = cfg["hi"][1] - cfg["lo"][1]
    xc = cfg["lo"][0] + 0.5 * Lx + Uinf * t
    yc = cfg["lo"][1] + 0.5 * Ly
    dx = np.mod(X[..., 0] - xc + 0.5 * Lx, Lx) - 0.5 * Lx
    dy = np.mod(X[..., 1] - yc + 0.5 * Ly, Ly) - 0.5 * Ly
    r2 = (dx * dx + dy * dy) / (Rv * Rv)
    cp = gamma / (gamma - 1.0)
    u = Uinf * (1.0 - beta * (dy / Rv) * np.exp(-r2 / 2.0))
    v = Uinf * beta * (dx / Rv) * np.exp(-r2 / 2.0)
    T = 1.0 - (Uinf * Uinf * beta * beta / (2.0 * cp)) * np.exp(-r2)
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    return [rho, rho * u, rho * v, E]


def tgv_field(X, cfg, gamma=1.4, phase=(0.0, 0.0, 0.0), amp=1.0):
    """Conservative Taylor-Green state at X[..., 3] (T = T0 = 1, rho = p/(R T0))."""
    V0 = amp * cfg["M"] * math.sqrt(gamma)
    x = X[..., 0] + phase[0]
    y = X[..., 1] + phase[1]
    z = X[..., 2] + phase[2]
    u = V0 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -V0 * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = 1.0 + V0 * V0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = p
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return [rho, rho * u, rho * v, rho * w, E]


def project(cfg, field, nq_extra=3):
    """Modal coefficients W[e, v, i] of the L2 projection of field(X) onto the
    orthonormal total-degree Legendre basis, tensor GL rule with p+1+nq_extra
    points per direction (numpy routines)."""
    d, p = cfg["dim"], cfg["p"]
    n = cfg["n"][:d]
    lo = np.array(cfg["lo"][:d])
    h = (np.array(cfg["hi"][:d]) - lo) / np.array(n)
    nq = p + 1 + nq_extra
    x1, w1 = np.polynomial.legendre.leggauss(nq)
    V1 = np.polynomial.legendre.legvander(x1, p) * np.sqrt((2 * np.arange(p + 1) + 1) / 2.0)
    md = mode_list(p, d, cfg.get("space", "P"))
    grids = np.meshgrid(*([np.arange(nq)] * d), indexing="ij")
    aidx = [g.reshape(-1) for g in grids]               # quadrature multi-index
    wq = np.ones(len(aidx[0]))
    for k in range(d):
        wq = wq * w1[aidx[k]]
    phi = np.ones((len(wq), len(md)))
    for i, al in enumerate(md):
        for k in range(d):
            phi[:, i] *= V1[aidx[k], al[k]]
    E = int(np.prod(n))
    e = np.arange(E)
    ijk = []
    rem = e.copy()
    for k in range(d):
        ijk.append(rem % n[k])
        rem = rem // n[k]
    X = np.zeros((E, len(wq), d))
    for k in range(d):
        X[:, :, k] = lo[k] + (ijk[k][:, None] + 0.5) * h[k] + x1[aidx[k]][None, :] * h[k] / 2.0
    vals = field(X)
    W = np.zeros((E, d + 2, len(md)))
    for v in range(d + 2):
        W[:, v, :] = (vals[v] * wq) @ phi
    return W


def initial_state(cfg, t=0.0, gamma=1.4):
    """W of the workload's closed-form field at time t (vortex) or t = 0 (TGV)."""
    if cfg["case"] == "vortex":
        return project(cfg, lambda X: vortex_field(X, cfg, t=t, gamma=gamma))
    return project(cfg, lambda X: tgv_field(X, cfg, gamma=gamma,
                                            phase=cfg.get("phase", (0.0, 0.0, 0.0)),
                                            amp=cfg.get("amp", 1.0)))


def perturbed_state(cfg, seed=SEED, amp=1e-2):
    """initial_state plus seeded noise on every mode (all modes of all variables
    carry information, so parity tests exercise the whole basis).  The noise on
    mode i of degree s has standard deviation amp * |W0| / (1 + s)^2."""
    W = initial_state(cfg)
    rng = np.random.default_rng(seed)
    deg = np.array([sum(a) for a in mode_list(cfg["p"], cfg["dim"], cfg.get("space", "P"))], dtype=float)
    scale = np.abs(W[:, :, :1]).mean(axis=0, keepdims=True)
    return W + amp * scale * rng.standard_normal(W.shape) / (1.0 + deg) ** 2


def random_vector(shape, seed=SEED + 1):
    """Seeded standard-normal vector (Krylov directions, right-hand sides)."""
    return np.random.default_rng(seed).standard_normal(shape)


def batch_cases(count=64, seed=SEED):
    """Independent TGV cases drawn from the seed: n ~ U{8..24}, p ~ U{1..5},
    M ~ log-U[0.05, 0.5], Re ~ log-U[400, 3200], random phase and +-5 % amplitude."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nn = int(rng.integers(8, 25))
        p = int(rng.integers(1, 6))
        M = float(np.exp(rng.uniform(np.log(0.05), np.log(0.5))))
        Re = float(np.exp(rng.uniform(np.log(400.0), np.log(3200.0))))
        cfg = make_config("tgv", 3, (nn, nn, nn), p, M=M, Re=Re,
                          p_levels=tuple(sorted({p, min(p, 2), min(p, 1), 0}, reverse=True)))
        cfg["phase"] = tuple(float(x) for x in rng.uniform(0, 2 * math.pi, 3))
        cfg["amp"] = float(rng.uniform(0.95, 1.05))
        out.append(cfg)
    return out


def serving_requests(count=32, seed=1812, max_dofs=None):
    """Request mix of the serving workload: 2-D vortex quads 32^2-256^2 and 3-D
    TGV hexes 8^3-32^3 with equal probability, p ~ U{1..6}, FP64 or mixed with
    probability 1/2, each one implicit BDF2 step.  max_dofs (optional) bounds
    the sample: a draw whose DOFs exceed it is redrawn (a bounded sample of the
    same distribution, for runs that must finish in minutes)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        if rng.uniform() < 0.5:
            n = int(rng.integers(32, 257))
            p = int(rng.integers(1, 7))
            cfg = make_config("vortex", 2, (n, n), p, M=0.5, Re=1000.0, dt_conv=0.05)
        else:
            n = int(rng.integers(8, 33))
            p = int(rng.integers(1, 7))
            cfg = make_config("tgv", 3, (n, n, n), p, M=0.1, Re=1600.0, dt_conv=0.01)
        levels = [p]
        for q in (2, 1, 0):
            if q < levels[-1]:
                levels.append(q)
        cfg["p_levels"] = tuple(levels)
        cfg["mixed"] = bool(rng.uniform() < 0.5)
        dofs = n_elements(cfg) * (cfg["dim"] + 2) * n_modes(p, cfg["dim"])
        if max_dofs is not None and dofs > max_dofs:
            continue
        cfg["dofs"] = dofs
        out.append(cfg)
    return out
