"""Host logic of the force server without a GPU: where the kept |a| of
evicted systems go in the pinned ring (placement, wrap-around, forgetting
the oldest entries)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def ring_cls():
    import __graft_entry__ as g

    g.build()
    from paper_1909_04667_gb300.serve import _RingIndex

    return _RingIndex


def test_ring_places_wraps_and_forgets_the_oldest(ring_cls):
    r = ring_cls(100)
    assert r.place("a", 40) == 0 and r.place("b", 40) == 40 and r.place("c", 15) == 80
    # 30 does not fit at 95: wrap to 0, which overwrites a (the oldest); b and c stay
    assert r.place("d", 30) == 0
    assert list(r.entries) == ["b", "c", "d"]
    # 30 more at 30 overlaps b (40..80) only
    assert r.place("e", 30) == 30
    assert list(r.entries) == ["c", "d", "e"]
    assert r.take("d") == (0, 30, None) and r.take("d") is None
    assert r.place("f", 101) is None and "f" not in r.entries
    # a key saved again replaces its earlier entry
    assert r.place("c", 10) == 60 and list(r.entries) == ["e", "c"]


def test_ring_entries_never_overlap(ring_cls):
    rng = np.random.default_rng(5)
    r = ring_cls(1000)
    live = {}
    for k in range(3000):
        key = int(rng.integers(0, 60))
        if rng.random() < 0.3:
            got = r.take(key)
            assert (got is None) == (key not in live)
            live.pop(key, None)
            continue
        n = int(rng.integers(1, 400))
        off = r.place(key, n)
        assert off is not None and 0 <= off and off + n <= 1000
        live[key] = (off, n)
        # the server's view equals the ring's, and no two kept entries overlap
        live = {q: live[q] for q in r.entries}
        assert {q: v[:2] for q, v in r.entries.items()} == live
        spans = sorted(live.values())
        assert all(a[0] + a[1] <= b[0] for a, b in zip(spans, spans[1:]))
        assert key in r.entries  # the newest entry is always kept
