"""The allocation-free tile sort (pic_tile_sort_noalloc) against the tile sort that runs inside
a context (pic_load_particles of the FP32 form, which uses the same cell-major order) and
against the oracle's stable order.

Callers that cannot allocate device memory when they sort -- their device memory belongs to
another allocator, or they cannot take the device-wide synchronisation of cudaMalloc -- use
the allocation-free entry point; it must give the same order.  The order is stable (tile, cell
in tile, input index), so the permutation itself, the cell at every sorted position and the
tile offsets are unique and compared bit for bit, twice in a row (the second call reuses the
scratch array the first one left behind).  This file is collected last.
"""
import numpy as np
import pytest

import oracle
import plasma

torch = pytest.importorskip("torch")


def _pic():
    from paper_1909_09613_gb300 import _build
    _build.build()
    oracle.build()
    import paper_1909_09613_gb300 as pic
    return pic


@pytest.mark.gpu
def test_noalloc_tile_sort_matches_context_sort_twice():
    pic = _pic()
    wl = plasma.pair_plasma((96, 40), (1.0, 1.0), 0.3, 3, 1, 4.0, 0.1, 64, omega_p=0.2, seed=77)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=pic.PIC_FP32_MIXED,
                  capacity=caps, tile=(16, 8, 1))
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x, s.u)
    assert run.slot_major == 0  # a dense FP32 run is kept in the cell-major order
    _, _, cells_sorted = run.particles(0)
    ts_ctx = run.tile_offsets(0)
    rng = np.random.default_rng(5)
    shuffled = cells_sorted[rng.permutation(cells_sorted.size)]
    cells_dev = torch.from_numpy(shuffled.astype(np.int32)).cuda()
    perm_orc, ts_orc = oracle.tile_sort(wl.grid, run.tile, shuffled, oracle.CELL_MAJOR)
    assert np.array_equal(ts_orc, ts_ctx)
    for _ in range(2):
        perm, ts = pic.pic_tile_sort_noalloc(wl.grid, run.tile, cells_dev)
        torch.cuda.synchronize()
        perm = perm.cpu().numpy()
        assert np.array_equal(perm, perm_orc)
        assert np.array_equal(shuffled[perm], cells_sorted)
        assert np.array_equal(ts.cpu().numpy(), ts_ctx)
    run.close()


@pytest.mark.gpu
@pytest.mark.parametrize("grid,tile", [((100, 37, 1), (16, 8, 1)), ((13, 11, 9), (4, 4, 4))],
                         ids=["2d_ragged", "3d_ragged"])
def test_noalloc_tile_sort_ragged_tiles_and_cells_outside(grid, tile):
    """Grids that are not a multiple of the tile (partial edge tiles) and some cells outside the
    grid (-1 and >= nx ny nz): the in-grid particles follow the oracle's stable order, the tile
    offsets match a plain count, and the positions past the last tile hold -1."""
    pic = _pic()
    ncell = grid[0] * grid[1] * grid[2]
    rng = np.random.default_rng(11)
    n = 20000
    cells = rng.integers(0, ncell, n)
    bad = rng.choice(n, 37, replace=False)
    cells[bad[:20]] = -1
    cells[bad[20:]] = ncell + rng.integers(0, 1000, 17)
    inside = (cells >= 0) & (cells < ncell)
    cells_dev = torch.from_numpy(cells.astype(np.int32)).cuda()
    idx_in = np.nonzero(inside)[0]
    perm_orc, ts_orc = oracle.tile_sort(grid, tile, cells[idx_in], oracle.CELL_MAJOR)
    # tile offsets from a plain count of the in-grid cells
    i, j, k = cells[idx_in] % grid[0], (cells[idx_in] // grid[0]) % grid[1], cells[idx_in] // (grid[0] * grid[1])
    nt = [(grid[a] + tile[a] - 1) // tile[a] for a in range(3)]
    t = ((k // tile[2]) * nt[1] + j // tile[1]) * nt[0] + i // tile[0]
    ts_count = np.concatenate([[0], np.cumsum(np.bincount(t, minlength=nt[0] * nt[1] * nt[2]))])
    assert np.array_equal(ts_orc, ts_count)
    for _ in range(2):
        perm, ts = pic.pic_tile_sort_noalloc(grid, tile, cells_dev)
        torch.cuda.synchronize()
        perm, ts = perm.cpu().numpy(), ts.cpu().numpy()
        m = int(inside.sum())
        assert ts[-1] == m
        assert np.array_equal(ts, ts_count)
        assert np.array_equal(perm[:m], idx_in[perm_orc])
        assert np.all(perm[m:] == -1)


@pytest.mark.gpu
def test_noalloc_tile_sort_rejects_oversize():
    pic = _pic()
    cells = torch.zeros((1 << 20) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(pic.PicError) as e:
        pic.pic_tile_sort_noalloc((64, 64, 1), (32, 8, 1), cells)
    assert e.value.status == pic.PIC_EINVAL
