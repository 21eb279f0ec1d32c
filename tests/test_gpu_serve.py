"""Continuous-batching server (clod_server_*): every request's image equals the
same view rendered alone, whatever batch it lands in (requests include
primitive budgets and windows of a frame); graphs on and off agree;
batches that overflow the slot's pair buffer are re-run and still correct;
requests arriving while batches are in flight are admitted."""
import time

import numpy as np
import pytest
import torch

from paper_2510_09997_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2510_09997_gb300 import clod as C
    from paper_2510_09997_gb300 import serve
    C.require_cuda()
    sc = S.tiny_scene(n=20000, seed=50, sh_degree=1)
    ds = C.DeviceScene.from_scene(sc)
    rng = np.random.default_rng(5)
    sizes = [(64, 64), (128, 96), (256, 256), (200, 120), (97, 161), (320, 180)]
    views = []
    for k in range(24):
        w, h = sizes[k % len(sizes)]
        d = rng.uniform(2.2, 6.0)
        dirv = rng.normal(size=3)
        dirv /= np.linalg.norm(dirv)
        s = float(np.float32(np.exp(rng.uniform(0, np.log(8)))))
        v = S.look_at(d * dirv, (0, 0, 0), w, h, s_v=s, bg=(0.1, 0.2, 0.3))
        if k % 5 == 4:      # primitive budget
            v = v.replace(budget=1500 + 300 * k)
        if k % 7 == 3:      # a window of the frame
            v = v.replace(width=w - 16, height=h - 32, region_x=16, region_y=16, full_width=w, full_height=h)
        views.append(v)
    solo = []
    for v in views:
        fr = C.render(ds, [v], want_keys=False)
        solo.append(fr.view_image(0).clone())
    torch.cuda.synchronize()
    return C, serve, ds, views, solo


def run(serve, ds, views, **kw):
    srv = serve.Server(ds, max_width=320, max_height=256, **kw)
    outs = [torch.full((3, v.height, v.width), -7.0, device="cuda") for v in views]
    tickets = [srv.submit(v, o) for v, o in zip(views, outs)]
    stats = [srv.wait(t, 30.0) for t in tickets]
    torch.cuda.synchronize()
    srv.close()
    return outs, stats


@pytest.mark.parametrize("graphs", [True, False])
def test_batched_equals_solo(env, graphs):
    C, serve, ds, views, solo = env
    outs, stats = run(serve, ds, views, max_views_per_batch=6, n_slots=2, use_graphs=graphs)
    for o, s in zip(outs, solo):
        assert torch.equal(o, s)
    assert max(st.batch_size for st in stats) > 1
    assert all(st.status == 0 and st.done_us >= st.launch_us >= st.submit_us for st in stats)


def test_overflowing_batches_are_rerun(env):
    C, serve, ds, views, solo = env
    outs, stats = run(serve, ds, views, max_views_per_batch=4, n_slots=2, pair_capacity=3000)
    for o, s in zip(outs, solo):
        assert torch.equal(o, s)


def test_arrivals_while_busy_and_wait_timeout(env):
    C, serve, ds, views, solo = env
    srv = serve.Server(ds, max_views_per_batch=4, n_slots=2, max_width=320, max_height=256)
    outs = [torch.zeros((3, v.height, v.width), device="cuda") for v in views]
    tickets = []
    for k, (v, o) in enumerate(zip(views, outs)):
        tickets.append(srv.submit(v, o))
        if k % 5 == 4:
            time.sleep(0.002)
    for t in tickets:
        srv.wait(t, 30.0)
    torch.cuda.synchronize()
    for o, s in zip(outs, solo):
        assert torch.equal(o, s)
    # argument errors are reported, the server keeps serving
    with pytest.raises(C.ClodError) as e:
        srv.submit(views[0].replace(width=4000, height=64, cx=2000.0), outs[0])
    assert e.value.status == 1
    with pytest.raises(C.ClodError) as e:
        srv.wait(123456789, 0.01)
    assert e.value.status == 1
    t = srv.submit(views[2], outs[2])
    st = srv.wait(t, 30.0)
    assert st.status == 0
    srv.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_partial_batches_reuse_one_slot(env, graphs):
    """Groups of 1, 3, 5, 2 and 4 requests, each waited for before the next is
    submitted, on one slot of 6 views: every batch is smaller than the slot's
    layout and reuses workspace a previous batch wrote, and every image still
    equals the solo render."""
    C, serve, ds, views, solo = env
    srv = serve.Server(ds, max_width=320, max_height=256, max_views_per_batch=6, n_slots=1, use_graphs=graphs)
    k = 0
    for g in (1, 3, 5, 2, 4):
        idx = list(range(k, k + g))
        k += g
        outs = [torch.full((3, views[i].height, views[i].width), -7.0, device="cuda") for i in idx]
        tickets = [srv.submit(views[i], o) for i, o in zip(idx, outs)]
        stats = [srv.wait(t, 30.0) for t in tickets]
        torch.cuda.synchronize()
        assert all(st.status == 0 for st in stats)
        for i, o in zip(idx, outs):
            assert torch.equal(o, solo[i]), i
    srv.close()


def test_fast_exp_server_equals_solo(env):
    """A server with fast_exp blends every batch with CLOD_FAST_EXP's
    exponential: each request equals the same view rendered alone with the
    flag, bit for bit, in whatever batch it lands."""
    C, serve, ds, views, _ = env
    fviews = [v.replace(flags=v.flags | S.FLAG_FAST_EXP) for v in views]
    solo = []
    for v in fviews:
        fr = C.render(ds, [v], want_keys=False)
        solo.append(fr.view_image(0).clone())
    torch.cuda.synchronize()
    outs, stats = run(serve, ds, views, max_views_per_batch=6, n_slots=2, use_graphs=True, fast_exp=True)
    assert max(st.batch_size for st in stats) > 1
    for k, (o, want) in enumerate(zip(outs, solo)):
        assert torch.equal(o, want), k
