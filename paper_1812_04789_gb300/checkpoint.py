"""Checkpoint / resume of an implicit time loop.

One .npz file holds what the next step needs: the states W^n and W^{n-1}
(BDF2; W^{n-1} may be omitted for one-step schemes such as ESDIRK3), the step
counter and time, and the mesh descriptor, physics and p-multigrid options as
JSON.  The preconditioner is not stored: it is lagged, assembled once per step
at W^n (Sec. 7.4), so a resumed run rebuilds it with dg_pmg_setup at the
restored W^n and takes the same step as an uninterrupted run.  Files are
written to a temporary name and renamed, so a crash mid-write leaves the
previous checkpoint intact.
"""
import json
import os

import numpy as np

from . import binding as B

FORMAT = 1


def opts_to_dict(o):
    """dg_pmg_opts (binding.PmgOpts) -> plain dict of ints / int lists."""
    out = {}
    for name, ctype in B.PmgOpts._fields_:
        v = getattr(o, name)
        out[name] = list(v) if hasattr(ctype, "_length_") else int(v)
    return out


def opts_from_dict(d):
    o = B.PmgOpts()
    for name, ctype in B.PmgOpts._fields_:
        if name not in d:
            continue                        # fields added later keep their zero default
        if hasattr(ctype, "_length_"):
            arr = getattr(o, name)
            for i, x in enumerate(d[name][: ctype._length_]):
                arr[i] = int(x)
        else:
            setattr(o, name, int(d[name]))
    return o


def _host(x):
    if x is None:
        return None
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=np.float64)


def save(path, Wn, step, t, mesh, physics, pmg_opts, Wnm1=None, extra=None):
    """Write a checkpoint.  Wn / Wnm1: numpy arrays or torch tensors (any
    device); mesh, physics: the dicts of ``workloads`` (mesh_desc/tri_mesh,
    physics); pmg_opts: binding.PmgOpts; extra: JSON-serialisable dict."""
    meta = {"format": FORMAT, "step": int(step), "t": float(t), "pmg_opts": opts_to_dict(pmg_opts),
            "physics": dict(physics), "extra": extra or {}}
    arrays = {"Wn": _host(Wn)}
    if Wnm1 is not None:
        arrays["Wnm1"] = _host(Wnm1)
    mesh_json = {}
    for k, v in dict(mesh).items():
        if isinstance(v, np.ndarray):
            arrays["mesh_" + k] = v               # triangulations: vertex and triangle arrays
        else:
            mesh_json[k] = list(v) if isinstance(v, tuple) else v
    meta["mesh"] = mesh_json
    arrays["meta"] = np.frombuffer(json.dumps(meta).encode("utf-8"), dtype=np.uint8)
    tmp = str(path) + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, **arrays)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def load(path):
    """Read a checkpoint: dict(Wn, Wnm1 (or None), step, t, mesh, physics,
    pmg_opts (binding.PmgOpts), extra).  Raises ValueError on an unknown format."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(bytes(z["meta"]).decode("utf-8"))
        if meta.get("format") != FORMAT:
            raise ValueError("unknown checkpoint format %r" % meta.get("format"))
        mesh = dict(meta["mesh"])
        for k in z.files:
            if k.startswith("mesh_"):
                mesh[k[5:]] = z[k].copy()
        return {"Wn": z["Wn"].copy(), "Wnm1": z["Wnm1"].copy() if "Wnm1" in z.files else None,
                "step": meta["step"], "t": meta["t"], "mesh": mesh, "physics": meta["physics"],
                "pmg_opts": opts_from_dict(meta["pmg_opts"]), "extra": meta.get("extra", {})}
