"""Admission policy and geometry keys of the serving loop: pure host logic, no CUDA."""
from __future__ import annotations

import hashlib
import struct


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


def geometry_key(geom: dict) -> str:
    """A key that is equal for equal geometries (sizes, distances, detector, angle list):
    the spectral norm of W, and the seed of the power iteration that estimates it, are
    functions of this key only."""
    h = hashlib.sha256()
    ints = [int(geom.get(k, 1)) for k in ("nx", "ny", "nz", "n_views", "nu", "nv")]
    flts = [float(geom.get(k, 0.0)) for k in ("a", "b", "c", "s", "sdd", "du", "dv", "u_off", "v_off")]
    h.update(struct.pack("<6q", *ints))
    h.update(struct.pack("<9d", *flts))
    for ang in geom["angles"]:
        h.update(struct.pack("<d", float(ang)))
    return h.hexdigest()


def geometry_seed(geom: dict) -> int:
    """Seed of the power-iteration start vector for this geometry (63 bits of its key)."""
    return int(geometry_key(geom)[:15], 16)
