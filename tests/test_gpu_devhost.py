"""Device vs host compilation of the pointwise physics (values and dual
tangents) must agree to rounding."""
import os
import subprocess

import pytest

from paper_1812_04789_gb300 import build

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_device_matches_host_physics(tmp_path):
    exe = str(tmp_path / "devhost")
    cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "-I", build.CSRC,
           os.path.join(HERE, "csrc", "devhost_physics.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
