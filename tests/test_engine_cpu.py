"""Host logic of the serving loop that needs no device: which batch lane a request joins, and
the hold policy of short-requests-first (the other lanes wait while short requests run, but
never longer than the hold limit at a stretch)."""
import paper_1909_09613_gb300 as pic
from paper_1909_09613_gb300 import engine


def _req(grid, ppc, l=3, precision=pic.PIC_FP32_MIXED):
    return engine.Request(rid=0, grid=grid, dt=0.3, l=l, gamma=20.0, u_th=0.01, ppc=ppc, steps=10,
                          precision=precision)


def test_lane_of_splits_batchable_requests_by_size():
    srv = engine.Server(small_particles=1 << 20)
    small = _req((256, 128, 1), 16)      # 524,288 particles
    large = _req((512, 256, 1), 16)      # 2,097,152 particles
    assert small.batchable and large.batchable
    assert srv.lane_of(small) == 0
    assert srv.lane_of(large) == 1
    # requests the batched kernel does not take step on their own streams
    assert not _req((64, 32, 1), 8, l=4).batchable
    assert not _req((64, 32, 16), 8, l=2).batchable
    assert not _req((64, 32, 1), 8, precision=pic.PIC_FP64).batchable


def test_hold_policy_holds_while_urgent_and_releases_after_the_limit():
    h = engine.HoldPolicy(0.5)
    assert h.hold(False, 0.0) is False
    assert h.hold(True, 1.0) is True          # short requests arrive: hold
    assert h.hold(True, 1.4) is True
    assert h.hold(True, 1.6) is False         # held longer than 0.5 s: one round released
    assert h.releases == 1
    assert h.hold(True, 1.7) is True          # and the hold starts over
    assert h.hold(True, 2.0) is True
    assert h.hold(False, 2.1) is False        # no short requests: nothing held
    assert h.hold(True, 2.2) is True          # a new hold counts from its own start
    assert h.hold(True, 2.65) is True
    assert h.releases == 1


def test_capacity_reserves_split_work_items_and_cta_cap(monkeypatch):
    class FakeRun:
        ncell = 64 * 32
        ntiles = 4
        ctx = None

    # _capacity reads the stage sizes through pic_smem_info, which needs a context; check the
    # table sizing alone with a stand-in for that query
    monkeypatch.setattr(pic, "pic_smem_info", lambda ctx: (0, 50000, 100000))
    cap = engine.Server._capacity([FakeRun(), FakeRun()], ctas_per_sm=1)
    assert cap.runs >= 8
    assert cap.tiles >= 8 * 2 * 4              # a small set may split each tile into 8 items
    assert cap.ctas_per_sm == 1
    assert cap.stage_bytes == 100000
