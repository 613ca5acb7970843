"""Admission policy of the serving loop: pure host logic, no CUDA."""
from __future__ import annotations


def admit_order(pending, now, slots, running, caps, used, budget, level_of, need_of):
    """Which waiting requests to admit now (indices into `pending`, which is sorted by
    arrival).  Requests are taken in arrival order while a slot is free; a request whose
    class (level_of) already runs caps[class] requests is passed over, a request whose memory
    (need_of) does not fit the budget stops the scan.  Pure host logic."""
    out = []
    running = dict(running)
    i = 0
    while i < len(pending) and pending[i].arrival <= now and slots > 0:
        req = pending[i]
        need = need_of(req)
        if need > budget:
            raise ValueError("request %d needs %d bytes, more than the budget" % (req.id, need))
        lv = level_of(req)
        if running[lv] >= caps[lv]:
            i += 1
            continue
        if used + need > budget:
            break
        out.append(i)
        running[lv] += 1
        used += need
        slots -= 1
        i += 1
    return out


def aged_level(class_index: int, waited_s: float, est_service_s):
    """Priority index (0 = highest) of a request's stream: its cost class, one level higher
    once it has waited longer than its estimated service time (None: no estimate yet)."""
    if est_service_s is not None and waited_s > est_service_s and class_index > 0:
        return class_index - 1
    return class_index
