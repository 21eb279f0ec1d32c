"""Helpers shared by the GPU parity tests: read libclod's outputs back and
compare them with the oracle's."""
import numpy as np
import torch

from oracle import oracle as O

from branches import match_fp64_branches


def u32(a):
    return np.ascontiguousarray(a).view(np.uint32)


def frame_stage1(fr, n):
    """Device Stage I arrays of a clod.Frame as numpy, per view."""
    V = len(fr.views)
    rec0 = fr.ws_array("rec0", torch.float32, 4 * V * n).view(V, n, 4).cpu().numpy()
    rec1 = fr.ws_array("rec1", torch.float32, 4 * V * n).view(V, n, 4).cpu().numpy()
    rec2 = fr.ws_array("rec2", torch.float32, 4 * V * n).view(V, n, 4)[:, :, 0].cpu().numpy()
    depth = fr.ws_array("depth", torch.float32, V * n).view(V, n).cpu().numpy()
    rect = fr.ws_array("rect", torch.int32, 2 * V * n).view(V, n, 2).cpu().numpy().view(np.uint32)
    key = fr.ws_array("dmax_key", torch.int64, V).cpu().numpy().view(np.uint64)
    out = []
    for v in range(V):
        r = rect[v]
        rr = np.stack([r[:, 0] & 0xFFFF, r[:, 0] >> 16, r[:, 1] & 0xFFFF, r[:, 1] >> 16], 1).astype(np.int32)
        k = int(key[v])
        out.append(dict(
            rec0=rec0[v], rec1=rec1[v], rec2=rec2[v], depth=depth[v], rect=rr,
            dmax_bits=np.uint32(k >> 32), argmax=(0xFFFFFFFF - (k & 0xFFFFFFFF)) if k else -1,
            mask=fr.mask[v].cpu().numpy(), alpha=fr.alpha_eff[v].cpu().numpy(),
            counts=fr.counts[v].cpu().numpy()))
    return out


def assert_stage1_equal(g, s1):
    """Bit-exact comparison of one view's Stage I (GPU dict vs oracle dict)."""
    assert int(g["dmax_bits"]) == int(u32(s1["dmax"])[0])
    assert int(g["argmax"]) == int(s1["argmax"][0])
    assert np.array_equal(g["mask"], s1["mask"])
    assert np.array_equal(u32(g["alpha"]), u32(s1["alpha_eff"]))
    surv = s1["survive"].astype(bool)
    assert np.array_equal(g["rect"], s1["rect"]), np.nonzero((g["rect"] != s1["rect"]).any(1))[0][:10]
    R = s1["rec"][surv]
    pairs = [(g["rec0"][surv, 0], R[:, 0]), (g["rec0"][surv, 1], R[:, 1]), (g["rec0"][surv, 2], R[:, 4]),
             (g["rec0"][surv, 3], R[:, 5]), (g["rec1"][surv, 0], R[:, 6]), (g["rec1"][surv, 1], R[:, 2]),
             (g["rec1"][surv, 2], R[:, 8]), (g["rec1"][surv, 3], R[:, 9]), (g["rec2"][surv], R[:, 10]),
             (g["depth"][surv], R[:, 3])]
    names = ["u", "v", "-A/2", "-B", "-C/2", "alpha''", "r", "g", "b", "depth"]
    for name, (a, b) in zip(names, pairs):
        bad = np.nonzero(u32(a) != u32(b))[0]
        assert bad.size == 0, (name, bad[:5], a[bad[:5]], b[bad[:5]])
    assert int(g["counts"][0]) == int(s1["mask"].sum())
    assert int(g["counts"][1]) == int(surv.sum())


def assert_image_matches(fr, v, ref, tiles=None, tol64=2e-4):
    """GPU image of view v equals the oracle's FP32 evaluation bit for bit and
    lies within tol64 of the FP64 image (on the listed tiles, or all).  With
    the oracle's FP64-decision outcomes in ``ref["dec64"]``, every pixel also
    lies within tol64 of one of them, with that outcome's contributor count;
    the flagged pixel counts are printed."""
    img = fr.view_image(v).cpu().numpy()
    T = fr.view_T(v).cpu().numpy()
    nc = fr.view_ncontrib(v).cpu().numpy().view(np.uint32)
    w = fr.views[v]
    if tiles is not None:
        tx = (w.width + 15) // 16
        sel = np.zeros((w.height, w.width), bool)
        for t in tiles:
            x0, y0 = (t % tx) * 16, (t // tx) * 16
            sel[y0:y0 + 16, x0:x0 + 16] = True
    else:
        sel = np.ones((w.height, w.width), bool)
    assert np.array_equal(nc[sel], ref["ncontrib"][sel])
    assert np.array_equal(u32(T[sel]), u32(ref["T32"][sel]))
    for c in range(3):
        assert np.array_equal(u32(img[c][sel]), u32(ref["img32"][c][sel])), c
    if ref.get("dec64") is not None:
        m = match_fp64_branches(img, T, nc, ref["dec64"], sel, tol64)
        print("FP64 decisions, view %d: %s" % (v, m))
        assert m["bad"] == 0 and m["nc_differs"] == 0, m
    if ref.get("img64") is not None:
        err = np.abs(img.astype(np.float64) - ref["img64"])[:, sel].max()
        assert err <= tol64, err
        return err
    return 0.0


def run_and_compare(C, scene, views, tiles=None, with64=True):
    """Render ``views`` through the C ABI and compare Stage I, the sorted pairs,
    the ranges and the images with the oracle."""
    ds = C.DeviceScene.from_scene(scene)
    fr = C.render(ds, views)
    torch.cuda.synchronize()
    ref = O.frame(scene, views, with64=with64, tiles=tiles, dec64=with64)
    g = frame_stage1(fr, scene.n)
    for v in range(len(views)):
        assert_stage1_equal(g[v], ref["s1"][v])
    assert fr.n_pairs == len(ref["keys"])
    assert np.array_equal(fr.keys.cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(fr.vals.cpu().numpy().view(np.uint32), ref["vals"])
    assert np.array_equal(fr.ranges.cpu().numpy().view(np.uint32), ref["ranges"])
    errs = []
    for v in range(len(views)):
        errs.append(assert_image_matches(fr, v, ref["img"][v], None if tiles is None else tiles[v]))
    return fr, ref, errs


GRAD_NAMES = ("means", "scales", "quats", "opacity", "sh", "decay")


def gpu_grads(A, sc, views, gimgs, galphas=None):
    """Gradients of sum_v <image_v, gimgs[v]> (+ <alpha''_v, galphas[v]>)
    through the autograd binding (clod_render_fwd / clod_render_bwd), as
    FP64 numpy arrays per parameter group."""
    ps = [torch.tensor(np.asarray(getattr(sc, k), np.float32), device="cuda", requires_grad=True)
          for k in GRAD_NAMES]
    imgs, alpha, mask, counts = A.render(*ps, views)
    loss = sum((im * torch.tensor(g, device="cuda", dtype=torch.float32)).sum() for im, g in zip(imgs, gimgs))
    if galphas is not None:
        loss = loss + (alpha * torch.tensor(np.stack(galphas), device="cuda", dtype=torch.float32)).sum()
    loss.backward()
    out = {k: p.grad.detach().cpu().numpy().astype(np.float64) for k, p in zip(GRAD_NAMES, ps)}
    del ps, imgs, alpha, mask, counts, loss
    return out


def rel_errors(g, r):
    """Per group ||g - r||_2 / ||r||_2 (||g||_2 where r is zero)."""
    out = {}
    for k in GRAD_NAMES:
        den = np.linalg.norm(r[k])
        out[k] = np.linalg.norm(g[k] - r[k]) / den if den > 0 else np.linalg.norm(g[k])
    return out


def tile_list_lengths(s1, view):
    """Length of every tile's list (row-major) from the oracle's tile
    rectangles: a 2D difference array over the survivors' rectangles."""
    tx, ty = O.tiles_of(view)
    lens = np.zeros((ty + 1, tx + 1), np.int64)
    r = s1["rect"][s1["survive"].astype(bool)]
    np.add.at(lens, (r[:, 1], r[:, 0]), 1)
    np.add.at(lens, (r[:, 1], r[:, 2]), -1)
    np.add.at(lens, (r[:, 3], r[:, 0]), -1)
    np.add.at(lens, (r[:, 3], r[:, 2]), 1)
    return lens.cumsum(0).cumsum(1)[:ty, :tx].reshape(-1)


def run_and_compare_fast(C, scene, views, tiles=None):
    """As run_and_compare, with every view blended under CLOD_FAST_EXP: the
    integer stages (Stage I, sorted pairs, ranges) bit for bit; the image,
    which no longer follows the FP32 decision sequence bit for bit, within
    2e-4 of the oracle's FP64 image and, pixel by pixel, within 2e-4 of an
    outcome of the FP64 decisions.  Returns the per-view match summaries."""
    from paper_2510_09997_gb300 import synth as S
    fviews = [v.replace(flags=v.flags | S.FLAG_FAST_EXP) for v in views]
    ds = C.DeviceScene.from_scene(scene)
    fr = C.render(ds, fviews)
    torch.cuda.synchronize()
    ref = O.frame(scene, views, with64=True, tiles=tiles, dec64=True)
    g = frame_stage1(fr, scene.n)
    for v in range(len(views)):
        assert_stage1_equal(g[v], ref["s1"][v])
    assert np.array_equal(fr.vals.cpu().numpy().view(np.uint32), ref["vals"])
    assert np.array_equal(fr.ranges.cpu().numpy().view(np.uint32), ref["ranges"])
    out = []
    for v, w in enumerate(views):
        img = fr.view_image(v).cpu().numpy()
        T = fr.view_T(v).cpu().numpy()
        nc = fr.view_ncontrib(v).cpu().numpy().view(np.uint32)
        sel = np.ones((w.height, w.width), bool) if tiles is None else _tile_sel(w, tiles[v])
        r = ref["img"][v]
        err = np.abs(img.astype(np.float64) - r["img64"])[:, sel].max()
        m = match_fp64_branches(img, T, nc, r["dec64"], sel, 2e-4)
        m["err_fp64_image"] = float(err)
        m["differs_from_fp32_spec"] = int((np.abs(img - r["img32"]).max(axis=0)[sel] > 0).sum())
        print("CLOD_FAST_EXP, view %d: %s" % (v, m))
        assert m["bad"] == 0, m
        assert err <= 2e-4, err
        out.append(m)
    return out


def _tile_sel(w, tiles):
    tx = (w.width + 15) // 16
    sel = np.zeros((w.height, w.width), bool)
    for t in tiles:
        sel[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16] = True
    return sel
