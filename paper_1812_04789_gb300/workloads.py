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
    paper has 2-D cases only);
  * the vortex on a periodic triangulation (a seeded, jittered quad lattice cut
    into triangles, the paper's triangular grids of Sec. 7.2 with the full-order
    basis): vertex lists and lattice shifts only, the connectivity is left to
    the consumer; modal states in the orthonormal Dubiner basis, projected
    with scipy's Jacobi polynomials.
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


# ---------------------------------------------------------------- triangles
def tri_config(n, p, M=0.5, Re=1000.0, dt_conv=0.05, p_levels=None, lo=(0.0, 0.0), hi=(10.0, 10.0),
               jitter=0.15, seed=SEED):
    """The isentropic-vortex workload on a periodic triangulation (the paper's
    quadrilateral grid split into triangles, full-order P_p basis, Sec. 7.2):
    n = (n0, n1) quads, each cut into two triangles."""
    return dict(case="vortex", dim=2, mesh="tri", n=(int(n[0]), int(n[1]), 1), lo=(lo[0], lo[1], 0.0),
                hi=(hi[0], hi[1], 1.0), p=p, M=M, Re=Re, dt_conv=dt_conv,
                p_levels=tuple(p_levels) if p_levels else (p,), jitter=jitter, seed=seed, space="tri")


def tri_mesh(cfg):
    """Seeded periodic triangulation of [lo, hi]^2: an n0 x n1 vertex lattice
    displaced by a periodic jitter (uniform in +-jitter of the spacing per
    coordinate), every lattice quad split into two counter-clockwise triangles
    along a seeded diagonal.  Returns dict(X (nv, 2) vertex coordinates, vertex
    id = i + n0 j; tri (E, 3) vertex ids; shift (E, 3, 2) lattice shifts: corner
    k of triangle e sits at X[tri[e, k]] + shift[e, k] * (hi - lo)).  Triangles
    2q and 2q + 1 come from quad q = i + n0 j."""
    n0, n1 = cfg["n"][0], cfg["n"][1]
    lo = np.array(cfg["lo"][:2], dtype=np.float64)
    hi = np.array(cfg["hi"][:2], dtype=np.float64)
    h = (hi - lo) / np.array([n0, n1])
    rng = np.random.default_rng(cfg.get("seed", SEED))
    jit = cfg.get("jitter", 0.15) * h[None, None, :] * rng.uniform(-1.0, 1.0, size=(n1, n0, 2))
    flips = rng.integers(0, 2, size=(n1, n0))
    ii, jj = np.meshgrid(np.arange(n0), np.arange(n1))
    X = np.stack([lo[0] + ii * h[0], lo[1] + jj * h[1]], axis=-1) + jit          # (n1, n0, 2)
    X = X.reshape(-1, 2)

    def corner(i, j):
        return (i % n0) + n0 * (j % n1), (i // n0, j // n1)

    tri, shift = [], []
    for j in range(n1):
        for i in range(n0):
            A, B, C, D = corner(i, j), corner(i + 1, j), corner(i + 1, j + 1), corner(i, j + 1)
            pair = ((A, B, C), (A, C, D)) if flips[j, i] == 0 else ((A, B, D), (B, C, D))
            for t in pair:
                tri.append([c[0] for c in t])
                shift.append([c[1] for c in t])
    return dict(X=X, tri=np.array(tri, dtype=np.int64), shift=np.array(shift, dtype=np.int64), lo=lo, hi=hi)


def tri_modes(p):
    """(i, j) of the Dubiner modes: total degree i + j, then i descending."""
    return [(i, q - i) for q in range(p + 1) for i in range(q, -1, -1)]


def tri_state_shape(cfg):
    return (2 * cfg["n"][0] * cfg["n"][1], 4, (cfg["p"] + 1) * (cfg["p"] + 2) // 2)


def tri_physics(cfg, **kw):
    """physics() with the BR2 penalty n_faces + 1 = 4 of a triangle."""
    kw.setdefault("eta", 4.0)
    return physics(cfg, **kw)


def tri_project(cfg, field, nq_extra=3):
    """Modal coefficients of the L2 projection of field(X) onto the
    orthonormal Dubiner basis of every triangle (scipy's Jacobi polynomials,
    collapsed Gauss-Legendre rule with p + 1 + nq_extra points per direction)."""
    from scipy.special import eval_jacobi
    p = cfg["p"]
    msh = tri_mesh(cfg)
    L = msh["hi"] - msh["lo"]
    V = msh["X"][msh["tri"]] + msh["shift"] * L[None, None, :]               # (E, 3, 2)
    nq = p + 1 + nq_extra
    x, w = np.polynomial.legendre.leggauss(nq)
    a, b = np.tile(x, nq), np.repeat(x, nq)
    wq = np.tile(w, nq) * np.repeat(w, nq) * (1.0 - b) / 2.0
    r, s = (1.0 + a) * (1.0 - b) / 2.0 - 1.0, b
    psi = np.zeros((len(wq), len(tri_modes(p))))
    for t, (i, j) in enumerate(tri_modes(p)):
        na = 2.0 / (2 * i + 1)
        nb_ = 2.0 ** (2 * i + 2) / (2 * j + 2 * i + 2)
        psi[:, t] = (math.sqrt(2.0) * eval_jacobi(i, 0, 0, a) / math.sqrt(na)
                     * eval_jacobi(j, 2 * i + 1, 0, b) / math.sqrt(nb_) * (1.0 - b) ** i)
    lam1, lam2 = (r + 1.0) / 2.0, (s + 1.0) / 2.0
    Xq = V[:, None, 0, :] + lam1[None, :, None] * (V[:, None, 1, :] - V[:, None, 0, :]) \
        + lam2[None, :, None] * (V[:, None, 2, :] - V[:, None, 0, :])
    vals = field(Xq)
    W = np.zeros((len(V), 4, psi.shape[1]))
    for v in range(4):
        W[:, v, :] = (vals[v] * wq) @ psi
    return W


def tri_initial_state(cfg, t=0.0, gamma=1.4):
    return tri_project(cfg, lambda X: vortex_field(X, cfg, t=t, gamma=gamma))


def tri_perturbed_state(cfg, seed=SEED, amp=1e-2):
    """tri_initial_state plus seeded noise, standard deviation amp |W0| / (1 + degree)^2."""
    W = tri_initial_state(cfg)
    rng = np.random.default_rng(seed)
    deg = np.array([i + j for i, j in tri_modes(cfg["p"])], dtype=float)
    scale = np.abs(W[:, :, :1]).mean(axis=0, keepdims=True)
    return W + amp * scale * rng.standard_normal(W.shape) / (1.0 + deg) ** 2
