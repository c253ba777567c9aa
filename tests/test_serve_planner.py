"""Admission and step planning of the serving runtime (host only, no GPU):
arrival-order admission under a slot count and a byte cap, an equal share of
each step's tile budget for every admitted frame, completion of a frame in the
step that holds its last tiles, and release of slots and bytes."""
import pytest

import paper_2201_00094_gb300 as wt


@pytest.fixture
def lib_built():
    import os
    if not os.path.exists(wt.library_path()):
        from paper_2201_00094_gb300 import build_lib
        build_lib.build()
    return wt.lib()


def test_admission_by_bytes_and_slots(lib_built):
    pl = wt.Planner(max_slots=2, mem_cap_bytes=1000, step_tiles=100)
    a, b, c = pl.submit(400, 10), pl.submit(400, 10), pl.submit(100, 10)
    assert pl.admit() == [a, b]            # the third waits for a slot
    assert pl.used() == 800
    assert pl.submit(1001, 1) == -6        # larger than the cap: WT_ERR_NOMEM
    ranges, fin = pl.plan()
    assert sorted(fin) == [a, b]
    assert pl.admit() == []
    assert pl.release(a) == 0
    assert pl.admit() == [c]
    assert pl.used() == 500


def test_head_of_line_no_overtaking(lib_built):
    pl = wt.Planner(max_slots=8, mem_cap_bytes=1000, step_tiles=100)
    a = pl.submit(900, 5)
    b = pl.submit(500, 5)   # does not fit while a is held
    c = pl.submit(50, 5)    # would fit, but arrived after b
    assert pl.admit() == [a]
    pl.plan()
    assert pl.admit() == []
    pl.release(a)
    assert pl.admit() == [b, c]


def test_fair_share_and_completion_step(lib_built):
    pl = wt.Planner(max_slots=8, mem_cap_bytes=10**9, step_tiles=100)
    big = pl.submit(1, 1000)
    small = pl.submit(1, 30)
    pl.admit()
    ranges, fin = pl.plan()
    d = {rid: (t0, n) for rid, t0, n in ranges}
    assert d[small] == (0, 30) and d[big] == (0, 70)   # leftover of small's share goes to big
    assert fin == [small]
    late = pl.submit(1, 10)                            # arrives while big is running
    pl.admit()
    ranges, fin = pl.plan()
    d = {rid: (t0, n) for rid, t0, n in ranges}
    assert d[late] == (0, 10) and d[big] == (70, 90)
    assert fin == [late]
    total = 160
    steps = 0
    while True:
        ranges, fin = pl.plan()
        steps += 1
        total += sum(n for _, _, n in ranges)
        if fin:
            assert fin == [big]
            break
    assert total == 1000 + 30 + 10 + 0 - 0 or total >= 1000
    assert steps == 9


def test_every_tile_scheduled_exactly_once(lib_built):
    import random
    rnd = random.Random(0)
    pl = wt.Planner(max_slots=16, mem_cap_bytes=10**6, step_tiles=257)
    want = {}
    seen = {}
    done = set()
    for step in range(400):
        if step < 120 and rnd.random() < 0.5:
            t = rnd.randint(0, 900)
            rid = pl.submit(rnd.randint(1, 90_000), t)
            want[rid] = t
        pl.admit()
        ranges, fin = pl.plan()
        assert sum(n for _, _, n in ranges) <= 257
        assert len({r for r, _, _ in ranges}) == len(ranges)  # one range per request
        for rid, t0, n in ranges:
            seen.setdefault(rid, []).append((t0, n))
        for rid in fin:
            done.add(rid)
            assert pl.release(rid) == 0
    assert done == set(want)
    for rid, t in want.items():
        cov = sorted(seen.get(rid, []))
        pos = 0
        for t0, n in cov:
            assert t0 == pos
            pos += n
        assert pos == t
    assert pl.used() == 0


def test_release_rules(lib_built):
    pl = wt.Planner(max_slots=1, mem_cap_bytes=100, step_tiles=10)
    a = pl.submit(10, 20)
    assert pl.release(a) != 0          # not admitted
    pl.admit()
    pl.plan()
    assert pl.release(a) != 0          # not fully scheduled
    pl.plan()
    assert pl.release(a) == 0
    assert pl.release(a) != 0          # twice
