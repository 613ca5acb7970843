"""Admission logic of the serving loop (host only): arrival order, class caps, memory budget."""
import dataclasses

import pytest

from paper_2511_12235_gb300.sched import admit_order, aged_level  # noqa: E402


@dataclasses.dataclass
class R:
    id: int
    arrival: float
    lv: int
    need: int


def _admit(pending, now=10.0, slots=8, running=None, caps=None, used=0, budget=100):
    caps = caps or {0: 8, 1: 2, 2: 1}
    running = running or {0: 0, 1: 0, 2: 0}
    return admit_order(pending, now, slots, running, caps, used, budget, lambda r: r.lv, lambda r: r.need)


def test_arrival_order_and_slots():
    p = [R(i, float(i), 0, 1) for i in range(5)]
    assert _admit(p, slots=3) == [0, 1, 2]
    assert _admit(p, now=1.5) == [0, 1]          # not yet arrived


def test_full_class_is_passed_over():
    p = [R(0, 0.0, 2, 10), R(1, 1.0, 2, 10), R(2, 2.0, 0, 10)]
    # class 2 allows one request at a time: the second waits, the cheap one behind it goes
    assert _admit(p) == [0, 2]
    assert _admit(p, running={0: 0, 1: 0, 2: 1}) == [2]


def test_memory_blocks_later_requests():
    p = [R(0, 0.0, 0, 60), R(1, 1.0, 0, 50), R(2, 2.0, 0, 10)]
    # the second does not fit next to the first: nothing after it overtakes it
    assert _admit(p) == [0]
    with pytest.raises(ValueError):
        _admit([R(0, 0.0, 0, 101)])


def test_aging_promotes_by_one_level():
    assert aged_level(3, 10.0, None) == 3            # no estimate yet
    assert aged_level(3, 10.0, 20.0) == 3            # waited less than its service time
    assert aged_level(3, 30.0, 20.0) == 2            # waited longer: one level higher
    assert aged_level(0, 30.0, 20.0) == 0            # already at the top


def test_geometry_key():
    from paper_2511_12235_gb300.sched import geometry_key, geometry_seed
    import numpy as np
    import synth
    g1 = synth.geometry(64, 64, 1, n_views=90, s=200.0, sdd=400.0, nu=96)
    g2 = synth.geometry(64, 64, 1, n_views=90, s=200.0, sdd=400.0, nu=96)
    g3 = synth.geometry(64, 64, 1, n_views=90, s=200.0, sdd=400.0, nu=96, angles=synth.uniform_angles(90) + 1e-9)
    g4 = synth.geometry(64, 64, 1, n_views=90, s=200.0, sdd=401.0, nu=96)
    assert geometry_key(g1) == geometry_key(g2) and geometry_seed(g1) == geometry_seed(g2)
    assert len({geometry_key(g) for g in (g1, g3, g4)}) == 3
    assert 0 <= geometry_seed(g1) < 2 ** 63
