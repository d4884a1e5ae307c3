"""Lifetime and concurrency rules of the C ABI: what a release, a served
request, a batch graph and an asynchronous call may overlap.

Everything here is decided on the host: a release that could free memory a
kernel still reads is refused (PERCH_E_BUSY) before anything is freed, so
none of these tests runs a kernel on freed memory.  A stream is held back
with torch's device sleep so that "still running" is certain, not a race.
"""
import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

pytestmark = pytest.mark.gpu

BUSY, NOTFOUND = -7, -4


@pytest.fixture(scope="module")
def P():
    from paper_2008_00326_gb300 import build, perch
    build.build()
    perch.load()
    return perch


def _small(ctx):
    sc = scenes.tabletop_small()
    sid = ctx.set_observation(sc)
    mid = ctx.load_mesh(sc.meshes[0])
    return sc, sid, mid


def test_release_refused_while_a_served_request_needs_it(P):
    with P.Context(0) as ctx:
        sc, sid, mid = _small(ctx)
        req = sc.requests[0]
        alone = ctx.score(sid, mid, req.label, req.roi, req.poses)
        # the scheduler holds a lone small request up to 2 s waiting for more
        with P.Server(ctx, slots=1, max_batch_hypotheses=1 << 16, max_wait_us=2_000_000) as srv:
            t, costs = srv.submit(sid, mid, req.label, req.roi, req.poses)
            assert P.load().perch_release_scene(ctx.ctx, sid) == BUSY
            assert P.load().perch_release_mesh(ctx.ctx, mid) == BUSY
            assert "in use" in ctx.last_error()
            # other threads may still load data while the server runs ...
            extra = ctx.load_mesh(sc.meshes[0])
            # ... but the other calls are refused until it stops
            with pytest.raises(P.PerchError) as e:
                ctx.score(sid, mid, req.label, req.roi, req.poses[:4])
            assert e.value.status == BUSY
            srv.wait(t)
            assert srv.held() == 1
            srv.release(t)
            assert srv.held() == 0
            assert srv.poll(t) == NOTFOUND
            # the request is done: nothing reads the objects any more
            P.perch_release_mesh(ctx.ctx, extra)
            P.perch_release_scene(ctx.ctx, sid)
            P.perch_release_mesh(ctx.ctx, mid)
        assert np.array_equal(costs, alone)


def test_unreleased_tickets_are_counted_and_freed_on_release(P):
    with P.Context(0) as ctx:
        sc, sid, mid = _small(ctx)
        req = sc.requests[0]
        with P.Server(ctx, slots=2, max_batch_hypotheses=4096) as srv:
            ts = [srv.submit(sid, mid, req.label, req.roi, req.poses[k::7])[0] for k in range(7)]
            for t in ts:
                srv.wait(t)
            assert srv.held() == 7
            for t in ts:
                srv.release(t)
            assert srv.held() == 0


def test_release_refused_while_an_async_call_is_pending(P):
    import torch
    with P.Context(0) as ctx:
        sc, sid, mid = _small(ctx)
        req = sc.requests[0]
        s = torch.cuda.Stream()
        d_poses = torch.from_numpy(req.poses).cuda()
        d_costs = torch.empty((len(req.poses), 2), dtype=torch.int32, device="cuda")
        want = ctx.score(sid, mid, req.label, req.roi, req.poses)
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            torch.cuda._sleep(2_000_000_000)               # holds the stream about a second
            P.perch_score_hypotheses(ctx.ctx, sid, mid, req.label, req.roi, d_poses, d_costs, s)
        assert P.load().perch_release_scene(ctx.ctx, sid) == BUSY
        assert P.load().perch_release_mesh(ctx.ctx, mid) == BUSY
        P.perch_sync(ctx.ctx, s)                           # the stream passed the call: no kernel errors
        P.perch_release_scene(ctx.ctx, sid)
        P.perch_release_mesh(ctx.ctx, mid)
        assert np.array_equal(d_costs.cpu().numpy(), want)


def test_batch_graph_holds_its_scenes_until_destroyed(P):
    import torch
    with P.Context(0) as ctx:
        sc, sid, mid = _small(ctx)
        req = sc.requests[0]
        n = len(req.poses)
        items = P.work_items([(sid, mid, req.label, req.roi, 0, n)])
        d_poses = torch.from_numpy(req.poses).cuda()
        d_costs = torch.zeros((n, 2), dtype=torch.int32, device="cuda")
        g = P.perch_batch_graph_create(ctx.ctx, items, d_poses, d_costs)
        s = torch.cuda.Stream()
        P.perch_batch_graph_launch(ctx.ctx, g, s)
        s.synchronize()
        assert P.load().perch_release_scene(ctx.ctx, sid) == BUSY
        P.perch_batch_graph_destroy(g)
        want = ctx.score(sid, mid, req.label, req.roi, req.poses)
        assert np.array_equal(d_costs.cpu().numpy(), want)
        P.perch_release_scene(ctx.ctx, sid)


def test_async_argmins_on_two_streams_are_ordered(P):
    """The context's argmins share one scratch buffer: launched on two streams
    back to back, each must still return its own costs' argmin."""
    import torch
    rng = np.random.default_rng(4)
    with P.Context(0) as ctx:
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        runs = []
        for k in range(12):
            n = int(rng.integers(1000, 300_000))
            costs = rng.integers(0, 50, size=(n, 2)).astype(np.int32)
            runs.append((costs, torch.from_numpy(costs).cuda(),
                         torch.full((1,), -1, dtype=torch.int64, device="cuda"),
                         torch.full((1,), -1, dtype=torch.int32, device="cuda")))
        torch.cuda.synchronize()
        for k, (_, dc, bi, bc) in enumerate(runs):
            s = streams[k % 2]
            with torch.cuda.stream(s):
                P.perch_best(ctx.ctx, dc, None, s, bi, bc)
        torch.cuda.synchronize()
        for costs, _, bi, bc in runs:
            assert (int(bi.item()), int(bc.item())) == ctx.best(costs)


def test_sync_reports_kernel_errors_of_async_calls(P):
    """A GICP source cloud over max_source_points is found by the kernel; an
    asynchronous call cannot return it, perch_sync does (and clears it)."""
    import torch
    with P.Context(0) as ctx:
        sc, sid, mid = _small(ctx)
        req = sc.requests[0]
        poses = req.poses[req.gt_index][None].repeat(4, 0)
        d_in = torch.from_numpy(poses).cuda()
        d_out = torch.empty_like(d_in)
        s = torch.cuda.Stream()
        gp = P.perch_default_gicp_params(max_source_points=8)
        P.perch_refine_hypotheses(ctx.ctx, sid, mid, req.label, req.roi, d_in, gp, poses_out=d_out, stream=s)
        with pytest.raises(P.PerchError) as e:
            P.perch_sync(ctx.ctx, s)
        assert e.value.status == -1 and "max_source_points" in str(e.value)
        P.perch_sync(ctx.ctx, s)                          # cleared
