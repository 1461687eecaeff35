"""Shared test helpers: build oracle meshes/physics from a workload dict."""
import numpy as np

from oracle.dg import Mesh
from oracle.physics import Physics
from paper_1812_04789_gb300 import workloads as wl


def oracle_mesh(cfg, nq1d=None):
    d = wl.mesh_desc(cfg, nq1d)
    return Mesh(d["dim"], d["n"], d["lo"], d["hi"], d["p"], d["nq1d"], space=d.get("space", "P"))


def oracle_physics(cfg, **kw):
    P = wl.physics(cfg, **kw)
    return Physics(gamma=P["gamma"], Pr=P["Pr"], mu=P["mu"], Rgas=P["Rgas"], eta=P["eta"],
                   roe_delta=P["roe_delta"])


def uniform_state(cfg, rho=1.0, vel=(0.3, -0.2, 0.1), p=1.0, gamma=1.4):
    d = cfg["dim"]
    shape = wl.state_shape(cfg)
    W = np.zeros(shape)
    c0 = 1.0 / np.sqrt(2.0) ** d          # phi_0 = 2^{-d/2} on [-1, 1]^d
    v = np.array(vel[:d])
    W[:, 0, 0] = rho / c0
    W[:, 1:1 + d, 0] = rho * v / c0
    W[:, d + 1, 0] = (p / (gamma - 1.0) + 0.5 * rho * v @ v) / c0
    return W


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
