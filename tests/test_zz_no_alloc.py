"""The allocation-free residual entry point (dg_residual_noalloc).

Callers that must not trigger any device allocation when they evaluate a
residual (an application that reserved all device memory at start-up, or a
time-critical loop kept out of the CUDA allocator) call dg_residual_noalloc,
which keeps its face scratch in a fixed device array inside the library.  This
test calls it through the C ABI twice in a row and checks each result against
dg_residual (same kernels, so within the residual tolerance of the parity
tests, 1e-12 relative max-norm; on 3-D meshes and on the tensor-product
space Q_p, which a case here uses, dg_residual sums the volume term by
factorisation and this entry point takes the direct contractions: equal to
rounding); that repeated calls
leave the device's free memory unchanged and launch only the face and volume
kernels; and that an oversized mesh is refused.  The file is collected last
so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1812_04789_gb300 import binding as B
from paper_1812_04789_gb300 import build
from paper_1812_04789_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _relmax(a, b):
    return float((a - b).abs().max().item() / max(b.abs().max().item(), 1e-300))


@pytest.mark.parametrize("cfg", [wl.make_config("tgv", 3, (5, 4, 3), 3, M=0.2, Re=400.0),
                                 wl.make_config("vortex", 2, (9, 7), 2, M=0.5, Re=1000.0),
                                 wl.make_config("tgv", 3, (3, 4, 3), 3, M=0.2, Re=400.0, space="Q")])
def test_noalloc_matches_residual_twice(cfg):
    build.build()
    assert torch.cuda.is_available()
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    for seed in (1, 2):                    # two calls in a row, different states
        W = torch.from_numpy(wl.perturbed_state(cfg, seed=seed, amp=0.05)).cuda()
        S = torch.from_numpy(wl.random_vector(tuple(W.shape), seed=seed + 10)).cuda()
        ref = torch.empty_like(W)
        got = torch.empty_like(W)
        m.residual(W, ref, S=S)
        m.residual_noalloc(W, got, S=S)
        torch.cuda.synchronize()
        assert _relmax(got, ref) <= 1e-12
        assert torch.isfinite(got).all()


def test_noalloc_calls_allocate_nothing():
    """After one call, further calls leave the driver's free-memory count as
    it was, and each launches exactly the face and the volume kernel."""
    build.build()
    cfg = wl.make_config("tgv", 3, (6, 5, 4), 3, M=0.2, Re=400.0)
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    W = torch.from_numpy(wl.perturbed_state(cfg, amp=0.05)).cuda()
    R = torch.empty_like(W)
    m.residual_noalloc(W, R)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    l0 = B.launch_count()
    for _ in range(5):
        m.residual_noalloc(W, R)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert B.launch_count() - l0 == 5 * 2


def test_noalloc_rejects_meshes_beyond_the_cap():
    build.build()
    cfg = wl.make_config("tgv", 3, (16, 16, 16), 4)      # 16^3 * 3 * 2 * 175 doubles > 2^20
    m = B.Mesh.from_workload(wl.mesh_desc(cfg), wl.physics(cfg))
    W = torch.from_numpy(wl.initial_state(cfg)).cuda()
    R = torch.empty_like(W)
    with pytest.raises(B.DGError) as e:
        m.residual_noalloc(W, R)
    assert e.value.code == 1
