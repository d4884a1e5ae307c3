"""Served form: continuous batching of concurrently submitted requests.

Each request's costs must be the same served (mixed into launches with other
requests of other scenes and sizes) as scored alone by perch_score_hypotheses.
"""
import threading

import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2008_00326_gb300 import build, perch
    build.build()
    perch.load()
    return perch


def _workload(ctx):
    out = []
    for sc in (scenes.tabletop_small(),
               scenes.tabletop_3obj(W=320, H=240, grid_half=4, n_yaw=8, tri_scale=0.25),
               scenes.sixdof_5obj(n_hyp=300, W=320, H=240, tri_scale=0.1)):
        sid = ctx.set_observation(sc)
        mids = [ctx.load_mesh(m) for m in sc.meshes]
        for req in sc.requests:
            out.append((sid, mids[req.mesh_index], req.label, req.roi, req.poses))
    return out


def test_served_equals_alone_under_concurrent_submission(P):
    with P.Context(0) as ctx:
        reqs = _workload(ctx)
        alone = [ctx.score(*r) for r in reqs]
        with P.Server(ctx, slots=2, max_batch_hypotheses=4096, max_wait_us=200) as srv:
            results = {}
            lock = threading.Lock()

            def client(ids):
                for k in ids:
                    t, _ = srv.submit(*reqs[k])
                    c = srv.wait(t)
                    with lock:
                        results[k] = c

            order = list(range(len(reqs))) * 3
            threads = [threading.Thread(target=client, args=(order[i::4],)) for i in range(4)]
            for th in threads:
                th.start()
            for th in threads:
                th.join()
            assert len(results) == len(reqs)
            for k, c in results.items():
                assert np.array_equal(c, alone[k]), k


def test_served_queue_drains_on_stop_and_reports_times(P):
    with P.Context(0) as ctx:
        reqs = _workload(ctx)
        alone = [ctx.score(*r) for r in reqs]
        srv = P.Server(ctx, slots=3, max_batch_hypotheses=8192)
        tickets = [srv.submit(*r) for r in reqs]
        assert srv.poll(10 ** 9) == -4                       # unknown ticket
        srv.stop()                                           # finishes the queue first
        # after stop the handle is gone; the costs arrays were filled
        for (t, costs), a in zip(tickets, alone):
            assert np.array_equal(costs, a)


def test_served_admission(P):
    with P.Context(0) as ctx:
        reqs = _workload(ctx)
        with P.Server(ctx, slots=1, max_batch_hypotheses=500) as srv:
            big = [r for r in reqs if len(r[4]) > 500][0]
            with pytest.raises(P.PerchError) as e:
                srv.submit(*big)
            assert e.value.status == -3
            small = [r for r in reqs if len(r[4]) <= 500][0]
            t, _ = srv.submit(*small)
            srv.wait(t)
            s0, s1 = srv.times(t)
            assert s1 >= s0
    # the slots' staging is charged to the context's HBM budget
    with P.Context(0, hbm_budget_bytes=1 << 20) as tiny:
        with pytest.raises(P.PerchError) as e:
            P.Server(tiny, slots=2, max_batch_hypotheses=1 << 16)
        assert e.value.status == -3
