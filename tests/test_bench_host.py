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
