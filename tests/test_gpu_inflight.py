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


class _Shot:
    """One rendered view (image, transmittance, contributor counts) with the
    accessors of a Frame, for the shared comparison helper."""

    def __init__(self, v, img, T, nc):
        self.views = [v]
        self._img, self._T, self._nc = img, T, nc

    def view_image(self, k):
        return self._img.view(3, self.views[0].height, self.views[0].width)

    def view_T(self, k):
        return self._T.view(self.views[0].height, self.views[0].width)

    def view_ncontrib(self, k):
        return self._nc.view(self.views[0].height, self.views[0].width)


def test_object_scene_full_size_eight_in_flight():
    """The benchmark's launch configuration at its full size: the 1M-Gaussian
    object scene (SH degree 3) at 1920x1080, eight renderers with a fixed
    pair capacity and eight streams, frames of the sweep issued round-robin
    with no synchronisation; the sixteen frames range from 33 M pairs to none
    (everything culled at s_v = 8 and 16 on the far cameras).  Every frame
    equals the same view rendered alone bit for bit; two of them (camera 0 at
    s_v = 1, camera 20 at s_v = 4) match the oracle on sampled tiles (the
    longest lists and random ones) bit for bit, within 2e-4 of FP64 and
    within 2e-4 of an outcome of the FP64 decisions."""
    from gpu_helpers import assert_image_matches
    from oracle import oracle as O
    from paper_2510_09997_gb300 import clod as C
    C.require_cuda()
    sc = S.object_scene()
    ds = C.DeviceScene.from_scene(sc)
    cams = S.orbit_cameras(64, 1920, 1080)
    scales = (1.0, 2.0, 4.0, 8.0, 16.0)
    views = [cams[(7 * k) % 64].replace(s_v=scales[k % 5]) for k in range(16)]
    alone, kmax = [], 0
    for v in views:
        fr = C.render(ds, [v], want_keys=False)
        alone.append((fr.view_image(0).clone(), fr.view_T(0).clone(), fr.view_ncontrib(0).clone()))
        kmax = max(kmax, int(fr.n_pairs))
        del fr
    torch.cuda.synchronize()
    n_fl = 8
    Rs = [C.Renderer(ds, [views[0]], pair_capacity=int(kmax * 1.02) + 1024) for _ in range(n_fl)]
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
        assert torch.equal(img.view(3, 1080, 1920), ai), k
        assert torch.equal(T.view(1080, 1920), aT), k
        assert torch.equal(nc.view(1080, 1920), an), k
    for k in (0, 12):
        v = views[k]
        s1 = O.stage1(sc, v)
        kk, _ = O.emit_pairs(v, s1)
        lens = np.bincount((kk >> np.uint64(32)).astype(np.int64), minlength=v.tiles)
        rng = np.random.default_rng(100 + k)
        tiles = list(np.argsort(lens)[-4:]) + list(rng.choice(v.tiles, 8, replace=False))
        ref = O.frame(sc, [v], with64=True, tiles=[tiles], pairs=False, dec64=True)
        img, T, nc = out[k]
        assert_image_matches(_Shot(v, img, T, nc), 0, ref["img"][0], tiles)
