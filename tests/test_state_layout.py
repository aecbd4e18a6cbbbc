"""The blocked state's slab layout (host arithmetic, no GPU): slab s holds rows
0 .. 32 s + 31 of columns [32 s, 32 s + 32), 32 entries per row, slabs one after another.
Every (row, column) pair a kernel can touch (rows below 32 (c // 32 + 1)) gets its own
index inside the per-sample stride, and the stride is about half of Nc^2."""
import numpy as np
import pytest


def slab_offset(s):
    return 512 * s * (s + 1)


def state_stride(Nc):
    return slab_offset((Nc + 31) // 32)


def sidx(j, c):
    return slab_offset(c >> 5) + j * 32 + (c & 31)


@pytest.mark.parametrize("Nc", [1, 31, 32, 33, 75, 256, 1000])
def test_indices_are_distinct_and_inside_the_stride(Nc):
    idx = [sidx(j, c) for c in range(Nc) for j in range(32 * (c // 32 + 1))]
    assert len(set(idx)) == len(idx)
    assert min(idx) >= 0 and max(idx) < state_stride(Nc)


def test_stride_is_about_half_the_square():
    for Nc in (1024, 2048):
        assert abs(state_stride(Nc) / Nc**2 - 0.5) < 0.02
    # a slab's rows are contiguous runs of 32 entries (one panel row per 32-lane access)
    assert sidx(5, 70) - sidx(4, 70) == 32 and sidx(4, 71) - sidx(4, 70) == 1
