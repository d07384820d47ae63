"""Host logic of bench.py: the CPML cell option and the byte model of the step
(36 B per node in FP32 and 16 B per slab node and axis, Sec. 3.2's memory
variables kept only in their slabs). CPU only."""
import argparse

import pytest

import bench


def test_cells_option_takes_one_or_six_counts():
    assert bench.cells_arg("20") == (20,) * 6
    assert bench.cells_arg("0") == (0,) * 6
    assert bench.cells_arg("20,20,0,0,5,7") == (20, 20, 0, 0, 5, 7)
    for bad in ("1,2", "1,2,3,4,5,6,7", "-1"):
        with pytest.raises(argparse.ArgumentTypeError):
            bench.cells_arg(bad)


def test_byte_model_per_axis():
    shape = (64, 48, 80)   # (z, y, x)
    nz, ny, nx = shape
    n = nx * ny * nz
    assert bench.algorithmic_bytes(shape, (0,) * 6, 4) == 36 * n
    # x slabs only: lo + hi columns of every (z, y) row
    assert bench.algorithmic_bytes(shape, (3, 5, 0, 0, 0, 0), 4) == 36 * n + 16 * 8 * ny * nz
    assert bench.algorithmic_bytes(shape, (0, 0, 2, 4, 0, 0), 4) == 36 * n + 16 * 6 * nx * nz
    assert bench.algorithmic_bytes(shape, (0, 0, 0, 0, 1, 6), 4) == 36 * n + 16 * 7 * nx * ny
    # 16-bit storage: 20 B per node, 8 B per slab node and axis
    assert bench.algorithmic_bytes(shape, (4,) * 6, 2) == 20 * n + 8 * (8 * ny * nz + 8 * nx * nz + 8 * nx * ny)


def test_traffic_entry_is_used_only_for_the_profiled_source(tmp_path, monkeypatch):
    # the ncu traffic figure is reported only while the kernel source and its
    # launch code hash to the value stored with it, scaled by the grid's nodes
    import json
    import os
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench.step_kernel_source_hash()
    entry = {"kernel_sha": h, "shape": [256, 256, 256], "dram_bytes_per_launch": 1000}
    (prof / "step_kernel_traffic.json").write_text(json.dumps({"f32": entry, "f16": dict(entry, kernel_sha="0" * 16)}))
    root = bench.ROOT
    csrc = tmp_path / "paper_2606_06910_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("fdtd_step.cu", "fdtd_internal.cuh", "fdtd_api.cu"):
        (csrc / f).write_bytes(open(os.path.join(root, "paper_2606_06910_gb300", "csrc", f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.step_kernel_traffic("f32", (512, 512, 512)) == 8000
    assert bench.step_kernel_traffic("f16", (512, 512, 512)) is None
    assert bench.step_kernel_traffic("bf16", (512, 512, 512)) is None
    (csrc / "fdtd_api.cu").write_bytes((csrc / "fdtd_api.cu").read_bytes() + b"\n// changed\n")
    assert bench.step_kernel_traffic("f32", (512, 512, 512)) is None
