"""Box range mappers and transfer inference of the library (paper §3) against the
oracle's, which its pins tie to enumerated cells; runs without a GPU."""
import itertools

import pytest

import oracle
import paper_2505_06022_gb300 as sy
from paper_2505_06022_gb300 import inputs

KINDS = [(sy.SY_RM_ONE_TO_ONE, (0, 0, 0), 0, ((0, 0, 0), (0, 0, 0))),
         (sy.SY_RM_NEIGHBOURHOOD, (1, 0, 2), 0, ((0, 0, 0), (0, 0, 0))),
         (sy.SY_RM_NEIGHBOURHOOD, (4, 4, 4), 0, ((0, 0, 0), (0, 0, 0))),
         (sy.SY_RM_SLICE, (0, 0, 0), 1, ((0, 0, 0), (0, 0, 0))),
         (sy.SY_RM_ALL, (0, 0, 0), 0, ((0, 0, 0), (0, 0, 0))),
         (sy.SY_RM_FIXED, (0, 0, 0), 0, ((-3, 2, 1), (5, 40, 7)))]


def random_boxes(seed, extent, n):
    z = inputs.splitmix64(seed, 6 * n)
    out = []
    for i in range(n):
        lo, hi = [], []
        for d in range(3):
            a = int(z[6 * i + 2 * d] % (extent[d] + 1))
            b = int(z[6 * i + 2 * d + 1] % (extent[d] + 1))
            lo.append(min(a, b))
            hi.append(max(a, b))
        out.append((tuple(lo), tuple(hi)))
    return out


@pytest.mark.parametrize("kind,radius,dim,fixed", KINDS)
def test_rm_box_matches_oracle(kind, radius, dim, fixed):
    extent = (9, 17, 33)
    rm = sy.range_mapper(kind, radius, dim, fixed)
    for chunk in random_boxes(7 + kind, extent, 200):
        assert sy.sy_rm_box(rm, chunk, extent) == oracle.rm_box(kind, chunk, extent, radius, dim, fixed)


def grid_chunks(extent, splits):
    """Chunks tiling the extent: an even split of each dimension into splits[d] parts."""
    parts = [oracle.split_rows(extent[d], splits[d]) for d in range(3)]
    return [((a0, a1, a2), (b0, b1, b2)) for (a0, b0), (a1, b1), (a2, b2) in itertools.product(*parts)]


@pytest.mark.parametrize("kind,radius,dim,fixed", KINDS)
@pytest.mark.parametrize("splits", [(4, 1, 1), (1, 3, 1), (2, 2, 2), (5, 1, 3)])
def test_rm_box_transfers_match_oracle(kind, radius, dim, fixed, splits):
    extent = (10, 12, 9)
    chunks = grid_chunks(extent, splits)
    rm = sy.range_mapper(kind, radius, dim, fixed)
    assert sy.sy_rm_box_transfers(rm, chunks, extent) == oracle.rm_box_transfers(kind, chunks, extent, radius, dim,
                                                                                 fixed)


def test_plane_chunks_match_row_transfers():
    # chunks of planes with a neighbourhood along dimension 0 are the row chunks of the 2D split
    nz, h = 37, 3
    rows = [(0, 1), (1, 3), (3, 30), (30, 37)]
    boxes = [((a, 0, 0), (b, 5, 6)) for a, b in rows]
    got = sy.sy_rm_box_transfers(sy.range_mapper(sy.SY_RM_NEIGHBOURHOOD, (h, 0, 0)), boxes, (nz, 5, 6))
    want = sy.sy_rm_transfers(nz, rows, h)
    assert sorted((s, d, b[0][0], b[1][0]) for s, d, b in got) == sorted(want)


@pytest.mark.parametrize("chunks,err", [
    ([((0, 0, 0), (5, 4, 4)), ((4, 0, 0), (8, 4, 4))], "SY_ERR_BAD_CHUNKS"),   # overlap
    ([((0, 0, 0), (5, 4, 4)), ((6, 0, 0), (8, 4, 4))], "SY_ERR_BAD_CHUNKS"),   # gap
    ([((0, 0, 0), (8, 4, 4)), ((8, 0, 0), (8, 4, 4))], "SY_ERR_BAD_CHUNKS"),   # empty chunk
    ([((0, 0, 0), (9, 4, 4))], "SY_ERR_BAD_CHUNKS"),                           # outside
])
def test_rm_box_transfers_reject_bad_chunk_lists(chunks, err):
    with pytest.raises(sy.SyError) as e:
        sy.sy_rm_box_transfers(sy.range_mapper(sy.SY_RM_ONE_TO_ONE), chunks, (8, 4, 4))
    assert e.value.name == err


def test_rm_box_rejects_bad_mappers():
    for rm in [sy.range_mapper(9), sy.range_mapper(sy.SY_RM_SLICE, dim=3),
               sy.range_mapper(sy.SY_RM_NEIGHBOURHOOD, (0, -1, 0))]:
        with pytest.raises(sy.SyError) as e:
            sy.sy_rm_box(rm, ((0, 0, 0), (1, 1, 1)), (2, 2, 2))
        assert e.value.name == "SY_ERR_INVALID_ARGUMENT"
