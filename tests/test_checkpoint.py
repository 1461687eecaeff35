"""Checkpoint / resume files (host only): bitwise round trip of the states,
step counter, mesh (structured descriptor and triangulation arrays), physics
and p-multigrid options; atomic replacement; unknown formats rejected."""
import json

import numpy as np
import pytest

from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import checkpoint as ck
from paper_1812_04789_gb300 import workloads as wl


def test_round_trip_structured(tmp_path):
    cfg = wl.make_config("tgv", 3, (3, 2, 4), 2)
    Wn = wl.perturbed_state(cfg)
    Wnm1 = wl.initial_state(cfg)
    opts = B.pmg_opts((2, 1, 0), nu_pre=(3, 4, 5), nu_post=7, nu_coarse=9, precision=B.PREC_MIXED,
                      coarse=B.COARSE_BILU, order=B.ORDER_COLOUR)
    path = tmp_path / "step.npz"
    ck.save(path, Wn, 17, 0.85, wl.mesh_desc(cfg), wl.physics(cfg), opts, Wnm1=Wnm1, extra={"dt": 0.05})
    r = ck.load(path)
    assert np.array_equal(r["Wn"], Wn) and np.array_equal(r["Wnm1"], Wnm1)
    assert r["step"] == 17 and r["t"] == 0.85 and r["extra"] == {"dt": 0.05}
    assert r["mesh"]["n"] == list(cfg["n"]) and r["physics"] == wl.physics(cfg)
    assert ck.opts_to_dict(r["pmg_opts"]) == ck.opts_to_dict(opts)
    assert list(r["pmg_opts"].nu_pre)[:3] == [3, 4, 5] and r["pmg_opts"].coarse_order == B.ORDER_COLOUR
    assert not (tmp_path / "step.npz.tmp").exists()


def test_round_trip_triangles_without_previous_state(tmp_path):
    cfg = wl.tri_config((4, 3), 2)
    msh = wl.tri_mesh(cfg)
    Wn = wl.tri_perturbed_state(cfg)
    path = tmp_path / "tri.npz"
    ck.save(path, Wn, 3, 0.1, msh, wl.tri_physics(cfg), B.pmg_opts((2,), cycle=B.CYCLE_BJ))
    r = ck.load(path)
    assert r["Wnm1"] is None and np.array_equal(r["Wn"], Wn)
    for k in ("X", "tri", "shift", "lo", "hi"):
        assert np.array_equal(r["mesh"][k], msh[k])


def test_overwrite_is_atomic_and_old_fields_default(tmp_path):
    cfg = wl.make_config("vortex", 2, (4, 4), 1)
    path = tmp_path / "c.npz"
    ck.save(path, wl.initial_state(cfg), 1, 0.0, wl.mesh_desc(cfg), wl.physics(cfg), B.pmg_opts((1,)))
    ck.save(path, wl.perturbed_state(cfg), 2, 0.1, wl.mesh_desc(cfg), wl.physics(cfg), B.pmg_opts((1,)))
    assert ck.load(path)["step"] == 2
    d = ck.opts_to_dict(B.pmg_opts((1,)))
    del d["coarse_order"]                                # a file written before the field existed
    assert ck.opts_from_dict(d).coarse_order == 0


def test_unknown_format_rejected(tmp_path):
    path = tmp_path / "bad.npz"
    meta = np.frombuffer(json.dumps({"format": 99}).encode(), dtype=np.uint8)
    np.savez(path, Wn=np.zeros(3), meta=meta)
    with pytest.raises(ValueError):
        ck.load(path)
