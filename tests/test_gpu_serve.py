"""The serving loop: every result is the same alone and in the mix (bit-identical for 2D;
within 1e-5 for 3D, whose kernels are instantiated per batch width and may contract
multiply-adds differently); requests of one geometry share a slot batch and join it while
it runs; admission respects the memory budget."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(n=6):
    reqs = []
    for i in range(n):
        if i % 2 == 0:
            N = 48 + 16 * i
            g = synth.geometry(N, N, 1, n_views=60 + 10 * i, s=1.953 * N, sdd=2.930 * N, nu=int(1.5 * N))
            x = synth.ellipse_phantom(N, 100 + i)
        else:
            N = 24 + 4 * i
            nd = int(1.5 * N) + int(1.5 * N) % 2
            g = synth.geometry(N, N, N, n_views=30 + 6 * i, s=1.953 * N, sdd=2.930 * N, nu=nd, nv=nd)
            g["dim"] = 3
            x = synth.ellipsoid_phantom(N, 100 + i)
        reqs.append((g, x))
    return reqs


def test_alone_equals_mixed_and_budget():
    from paper_2511_12235_gb300 import Projector
    from paper_2511_12235_gb300.serve import ReconServer, Request, footprint_bytes, solve_alone
    items = _requests()
    reqs = []
    for i, (g, x) in enumerate(items):
        P = Projector(g)
        sino = P.forward(torch.from_numpy(x).float().cuda()).cpu().numpy()
        P.close()
        reqs.append(Request(id=i, geom=g, sino=sino, arrival=0.0, iters=8, power_iters=10, seed=i))
    alone = [solve_alone(r) for r in reqs]
    # all in flight together, with graphs
    srv = ReconServer(max_active=6, use_graphs=True)
    done = srv.serve([Request(**{**r.__dict__, "result": None}) for r in reqs], realtime=False)
    for r, a in zip(sorted(done, key=lambda r: r.id), alone):
        if r.geom["dim"] == 2:      # gather kernels only: bit-identical
            assert np.array_equal(r.result, a), r.id
        else:                       # the 3D forward adds with atomics: equal to rounding
            assert np.linalg.norm(r.result - a) <= 1e-5 * np.linalg.norm(a), r.id
        assert r.t_done >= r.t_admit >= 0
    # a budget that fits only the largest request at a time still serves everything
    biggest = max(footprint_bytes(r.geom) for r in reqs)
    srv2 = ReconServer(budget_bytes=biggest, max_active=6, use_graphs=False)
    done2 = srv2.serve([Request(**{**r.__dict__, "result": None}) for r in reqs], realtime=False)
    for r, a in zip(sorted(done2, key=lambda r: r.id), alone):
        assert np.linalg.norm(r.result - a) <= 1e-5 * np.linalg.norm(a), r.id
    # no two requests overlapped in time under that budget when each needs more than half
    spans = sorted((r.t_admit, r.t_done) for r in done2 if 2 * footprint_bytes(r.geom) > biggest)
    for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
        assert b0 >= a1 - 1e-3


def test_priority_follows_cost():
    """Cheaper requests get streams of higher (numerically lower) priority."""
    from paper_2511_12235_gb300.serve import ReconServer, Request, cost_estimate
    srv = ReconServer(max_active=2, use_graphs=False)
    small = synth.geometry(256, 256, 1, n_views=360, s=500.0, sdd=750.0, nu=384)
    big = synth.geometry(256, 256, 256, n_views=360, s=500.0, sdd=750.0, nu=384, nv=384)
    big["dim"] = 3
    rs = Request(id=0, geom=small, sino=np.zeros(1, np.float32))
    rb = Request(id=1, geom=big, sino=np.zeros(1, np.float32))
    assert cost_estimate(small, 20, 20) < cost_estimate(big, 20, 20)
    assert srv.level_of(rs) <= srv.level_of(rb)
    if len(srv.levels) > 1:
        assert srv.level_of(rs) < srv.level_of(rb)


def test_norm_cached_per_geometry():
    """Two requests of one geometry: the second reuses the first's spectral-norm estimate
    (seeded by the geometry), and both results equal the same requests solved alone."""
    from paper_2511_12235_gb300 import Projector
    from paper_2511_12235_gb300.serve import ReconServer, Request, solve_alone
    g = synth.geometry(64, 64, 1, n_views=80, s=125.0, sdd=187.0, nu=96)
    P = Projector(g)
    reqs = []
    for i in range(2):
        x = synth.ellipse_phantom(64, 200 + i)
        sino = P.forward(torch.from_numpy(x).float().cuda()).cpu().numpy()
        reqs.append(Request(id=i, geom=g, sino=sino, arrival=0.0, iters=6, power_iters=8))
    P.close()
    alone = [solve_alone(r) for r in reqs]
    srv = ReconServer(max_active=2, use_graphs=True)
    done = srv.serve(reqs, realtime=False)
    assert srv.joined == 1 and srv.max_occupancy == 2      # one batch, one power iteration
    for r, a in zip(sorted(done, key=lambda r: r.id), alone):
        assert np.array_equal(r.result, a), r.id


def test_failing_requests_do_not_stop_the_others():
    """A refused geometry, projections of the wrong size and a request larger than the whole
    budget come back with `error` set; the valid request is served as alone."""
    from paper_2511_12235_gb300 import Projector
    from paper_2511_12235_gb300.serve import ReconServer, Request, footprint_bytes, solve_alone
    good = synth.geometry(48, 48, 1, n_views=60, s=94.0, sdd=141.0, nu=72)
    P = Projector(good)
    sino = P.forward(torch.from_numpy(synth.ellipse_phantom(48, 5)).float().cuda()).cpu().numpy()
    P.close()
    inside = synth.geometry(48, 48, 1, n_views=60, s=20.0, sdd=141.0, nu=72)   # source inside the grid
    big = synth.geometry(48, 48, 1, n_views=60, s=94.0, sdd=141.0, nu=72)
    reqs = [Request(id=0, geom=good, sino=sino, iters=5, power_iters=6),
            Request(id=1, geom=inside, sino=sino, iters=5, power_iters=6),
            Request(id=2, geom=good, sino=sino[:, :-1].copy(), iters=5, power_iters=6),
            Request(id=3, geom=big, sino=sino, iters=5, power_iters=6)]
    srv = ReconServer(budget_bytes=2 * footprint_bytes(good), max_active=4, use_graphs=True)
    # request 3 claims a footprint above the budget
    reqs[3].geom = dict(big, nz=10 ** 6)
    done = {r.id: r for r in srv.serve(reqs, realtime=False)}
    assert done[0].error is None and np.array_equal(done[0].result, solve_alone(reqs[0]))
    for i in (1, 2, 3):
        assert done[i].error and done[i].result is None, (i, done[i].error)
    assert srv.slots == srv.max_active and all(v == 0 for v in srv.running.values())


def test_graph_reused_per_shape_bucket():
    """A second request of the same geometry (after the first finished) reuses the first's
    slot batch and its captured graphs; results equal the requests solved alone."""
    from paper_2511_12235_gb300 import Projector
    from paper_2511_12235_gb300.serve import ReconServer, Request, solve_alone
    ga = synth.geometry(48, 48, 1, n_views=64, s=94.0, sdd=141.0, nu=72)
    gb = synth.geometry(40, 40, 1, n_views=50, s=79.0, sdd=118.0, nu=60)
    reqs = []
    for i, g in enumerate((ga, gb, ga)):
        P = Projector(g)
        x = synth.ellipse_phantom(g["nx"], 300 + i)
        reqs.append(Request(id=i, geom=g, sino=P.forward(torch.from_numpy(x).float().cuda()).cpu().numpy(),
                            arrival=0.0, iters=7, power_iters=8))
        P.close()
    alone = [solve_alone(r) for r in reqs]
    # one batch at a time and one slot per batch: request 2 takes over request 0's batch (its
    # freed slot while the batch drains, or the batch itself once idle)
    srv = ReconServer(max_active=1, use_graphs=True, max_slots=(1, 1))
    done = srv.serve(reqs, realtime=False)
    assert srv.joined + srv.batch_hits == 1
    for r, a in zip(sorted(done, key=lambda r: r.id), alone):
        assert np.array_equal(r.result, a), r.id
    srv.close()
    assert not srv.idle


def test_requests_join_a_running_batch_at_different_iterations():
    """Six requests of one geometry arriving one after another: they share one slot batch,
    joining it while earlier ones are mid-way (each keeps its own momentum sequence), and
    every result is bit-identical to the request solved alone; a 3D bucket likewise within
    1e-5."""
    from paper_2511_12235_gb300 import Projector
    from paper_2511_12235_gb300.serve import ReconServer, Request, solve_alone
    g2 = synth.geometry(64, 64, 1, n_views=96, s=125.0, sdd=187.0, nu=96)
    g3 = synth.geometry(24, 24, 24, n_views=40, s=47.0, sdd=70.0, nu=36, nv=36)
    g3["dim"] = 3
    reqs = []
    for i in range(6):
        g = g2 if i < 4 else g3
        P = Projector(g)
        x = synth.ellipse_phantom(64, 400 + i) if i < 4 else synth.ellipsoid_phantom(24, 400 + i)
        sino = P.forward(torch.from_numpy(x).float().cuda()).cpu().numpy()
        P.close()
        reqs.append(Request(id=i, geom=g, sino=sino, arrival=0.004 * i, iters=40, power_iters=8))
    alone = [solve_alone(r) for r in reqs]
    srv = ReconServer(max_active=4, use_graphs=True, max_slots=(4, 2), inflight=1)
    done = srv.serve(reqs, realtime=True)
    assert srv.joined >= 1
    for r, a in zip(sorted(done, key=lambda r: r.id), alone):
        assert r.error is None
        if r.geom["dim"] == 2:
            assert np.array_equal(r.result, a), r.id
        else:
            assert np.linalg.norm(r.result - a) <= 1e-5 * np.linalg.norm(a), r.id
    srv.close()
