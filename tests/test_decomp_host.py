"""Host-side geometry of the domain decomposition (paper Sec. 3.3): owned
boxes partition the grid, every part's ghost layers are covered exactly once
by the links to their owners, and the CPML stays on the grid's outer faces.
CPU only."""
import itertools

import numpy as np
import pytest

from paper_2606_06910_gb300.decomp import plan, split


def test_split_is_a_partition():
    for n, p in ((10, 3), (96, 4), (7, 7)):
        r = split(n, p)
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1


@pytest.mark.parametrize("shape,parts,s", [((96, 84, 52), (1, 2, 2), 1), ((96, 84, 52), (1, 2, 2), 4),
                                           ((96, 84, 52), (1, 1, 4), 2), ((96, 84, 52), (2, 2, 1), 2),
                                           ((96, 84, 52), (2, 2, 2), 1), ((50, 40, 90), (3, 1, 2), 1)])
def test_ghosts_covered_exactly_once_by_their_owners(shape, parts, s):
    cells = (5, 7, 6, 4, 8, 5)
    geo, links = plan(shape, parts, s, cells)
    owner = np.full(shape, -1)
    for i, g in enumerate(geo):
        (z0, z1), (y0, y1), (x0, x1) = g["own"]
        assert np.all(owner[z0:z1, y0:y1, x0:x1] == -1)
        owner[z0:z1, y0:y1, x0:x1] = i
    assert np.all(owner >= 0)
    g8 = 8 * s
    for i, g in enumerate(geo):
        loc = g["loc"]
        lshape = tuple(hi - lo for lo, hi in loc)
        cover = np.zeros(lshape, int)
        for (a, b, box, shift) in links:
            if a != i:
                continue
            cover[box[0]:box[1], box[2]:box[3], box[4]:box[5]] += 1
            # the source box lies in part b's owned box
            for ax in range(3):
                glo = box[2 * ax] + loc[ax][0]
                ghi = box[2 * ax + 1] + loc[ax][0]
                assert geo[b]["own"][ax][0] <= glo and ghi <= geo[b]["own"][ax][1]
                assert box[2 * ax] + shift[ax] == glo - geo[b]["loc"][ax][0]
        own = np.zeros(lshape, bool)
        sl = tuple(slice(o[0] - l[0], o[1] - l[0]) for o, l in zip(g["own"], loc))
        own[sl] = True
        assert np.all(cover[own] == 0) and np.all(cover[~own] == 1)
        # ghost depth 8 s towards neighbours, none beyond the grid
        for ax, p in zip(range(3), (parts[2], parts[1], parts[0])):
            o, l, n = g["own"][ax], loc[ax], shape[ax]
            assert l[0] == (max(0, o[0] - g8) if p > 1 else 0) and l[1] == (min(n, o[1] + g8) if p > 1 else n)
        # the layer on grid faces only
        for axis, ax in ((0, 2), (1, 1), (2, 0)):
            assert g["cells"][2 * axis] == (cells[2 * axis] if loc[ax][0] == 0 else 0)
            assert g["cells"][2 * axis + 1] == (cells[2 * axis + 1] if loc[ax][1] == shape[ax] else 0)


def test_too_thin_parts_are_refused():
    with pytest.raises(ValueError):
        plan((96, 84, 52), (2, 2, 1), 4, (5, 7, 6, 4, 8, 5))
