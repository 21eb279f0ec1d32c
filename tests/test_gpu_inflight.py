"""Several frames in flight: one Renderer (workspace, pair list, image) and one
stream per frame in flight, frames issued round-robin with no
synchronisation between them.  Every frame's image, transmittance and
contributor count equal, bit for bit, the same view rendered alone (the
frames share only the read-only scene; each workspace carries its own work
queues and counters)."""
import numpy as np
import pytest
import torch

from paper_2510_09997_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_fl", [2, 3])
def test_frames_in_flight_equal_alone(n_fl):
    from paper_2510_09997_gb300 import clod as C
    C.require_cuda()
    sc = S.tiny_scene(n=20000, seed=61, sh_degree=2)
    ds = C.DeviceScene.from_scene(sc)
    rng = np.random.default_rng(7)
    views = []
    for k in range(9):
        d = rng.uniform(2.2, 6.0)
        dirv = rng.normal(size=3)
        dirv /= np.linalg.norm(dirv)
        s = float(np.float32(np.exp(rng.uniform(0, np.log(16)))))
        views.append(S.look_at(d * dirv, (0, 0, 0), 250, 130, s_v=s, bg=(0.1, 0.2, 0.3)))
    alone = []
    kmax = 0
    for v in views:
        fr = C.render(ds, [v], want_keys=False)
        alone.append((fr.view_image(0).clone(), fr.view_T(0).clone(), fr.view_ncontrib(0).clone()))
        kmax = max(kmax, int(fr.n_pairs))
    torch.cuda.synchronize()
    cap = kmax + 1024
    Rs = [C.Renderer(ds, [views[0]], pair_capacity=cap) for _ in range(n_fl)]
    streams = [torch.cuda.Stream() for _ in range(n_fl)]
    for s_ in streams:
        s_.wait_stream(torch.cuda.current_stream())
    out = []
    for k, v in enumerate(views):
        i = k % n_fl
        Rs[i].set_views([v])
        Rs[i].run(streams[i])
        with torch.cuda.stream(streams[i]):
            out.append((Rs[i].image.clone(), Rs[i].T.clone(), Rs[i].nc.clone()))
    torch.cuda.synchronize()
    for r in Rs:
        r.check()
    for k, ((img, T, nc), (ai, aT, an)) in enumerate(zip(out, alone)):
        assert torch.equal(img.view(3, 130, 250), ai), k
        assert torch.equal(T.view(130, 250), aT), k
        assert torch.equal(nc.view(130, 250), an), k
