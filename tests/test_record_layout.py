"""The recordings' index maps (rec_base, rec32_at, rec32_step, rec32_steps4
in csrc/internal.h), compiled for the host and run on the CPU: every
coefficient index of every (direction, plane, voxel or voxel pair, step)
lies inside the block the context allocates and no two coincide; the FP32
replay's four-step loads start on 16-byte boundaries."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_record_index_maps_are_injective_and_in_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "record_layout")
    src = os.path.join(HERE, "native", "record_layout.cu")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-o", exe, src], check=True,
                   capture_output=True, timeout=300)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    rows = [list(map(int, line.split())) for line in out.strip().splitlines()]
    assert len(rows) == 7
    for nx, ny, nz, ndir, ok64, ok32 in rows:
        assert ok64 == 1, (nx, ny, nz, ndir)
        assert ok32 == 1, (nx, ny, nz, ndir)
