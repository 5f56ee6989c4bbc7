"""The allocation-free tile sort (pic_tile_sort_noalloc) against the tile sort that runs inside
a context (pic_load_particles of the FP32 form, which uses the same cell-major order).

Callers that cannot allocate device memory when they sort -- their device memory belongs to
another allocator, or they cannot take the device-wide synchronisation of cudaMalloc -- use
the allocation-free entry point; it must give the same order.  The cell at every sorted
position and the tile offsets are unique and compared bit for bit, twice in a row (the second
call reuses the scratch array the first one left behind).  This file is collected last.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_noalloc_tile_sort_matches_context_sort_twice():
    from paper_1909_09613_gb300 import _build
    _build.build()
    import paper_1909_09613_gb300 as pic

    wl = workloads.pair_plasma((96, 40), (1.0, 1.0), 0.3, 3, 1, 4.0, 0.1, 64, omega_p=0.2, seed=77)
    caps = [int(s.x.shape[1]) for s in wl.species]
    run = pic.Run(wl.grid, wl.dx, wl.dt, wl.l, wl.scheme, precision=pic.PIC_FP32_MIXED,
                  capacity=caps, tile=(16, 8, 1))
    for i, s in enumerate(wl.species):
        run.load(i, s.q, s.m, s.w, s.x.numpy(), s.u.numpy())
    assert run.slot_major == 0  # a dense FP32 run is kept in the cell-major order
    _, _, cells_sorted = run.particles(0)
    ts_ctx = run.tile_offsets(0)
    rng = np.random.default_rng(5)
    shuffled = cells_sorted[rng.permutation(cells_sorted.size)]
    cells_dev = torch.from_numpy(shuffled.astype(np.int32)).cuda()
    for _ in range(2):
        perm, ts = pic.pic_tile_sort_noalloc(wl.grid, run.tile, cells_dev)
        torch.cuda.synchronize()
        perm = perm.cpu().numpy()
        assert np.array_equal(np.sort(perm), np.arange(shuffled.size))
        assert np.array_equal(shuffled[perm], cells_sorted)
        assert np.array_equal(ts.cpu().numpy(), ts_ctx)
    run.close()


@pytest.mark.gpu
def test_noalloc_tile_sort_rejects_oversize():
    from paper_1909_09613_gb300 import _build
    _build.build()
    import paper_1909_09613_gb300 as pic
    cells = torch.zeros((1 << 20) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(pic.PicError) as e:
        pic.pic_tile_sort_noalloc((64, 64, 1), (32, 8, 1), cells)
    assert e.value.status == pic.PIC_EINVAL
