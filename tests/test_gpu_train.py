"""The virtual-distance training step (Sec. 3.3) on the GPU: loss scalars
(Eq. 3-5) against the oracle's mask counts and FP64 image, the
straight-through gradient delivered to alpha'', the overwriting backward
against the accumulating one, the fused Adam step against torch's Adam in
FP64, the rendering-loss kernel against the FP64 SSIM oracle,
and short runs that lower the loss."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import losses as OL
from oracle import oracle as O
from paper_2510_09997_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    from paper_2510_09997_gb300 import clod, train
    clod.require_cuda()
    return train


def setup(T, s_max=8.0, dssim=0.0):
    sc = S.tiny_scene(n=4000, seed=40, sh_degree=1)
    views = [S.tiny_view(1.0).replace(width=96, height=96, cx=48.0, cy=48.0),
             S.look_at((2.2, 1.0, 1.2), (0, 0, 0), 80, 64)]
    targets = [S.target_image(v.height, v.width, seed=k) for k, v in enumerate(views)]
    model = T.GaussianModel(sc)
    step = T.TrainStep(model, s_max=s_max, lam_reg=1.0, dssim_weight=dssim)
    return sc, views, targets, model, step


def test_loss_scalars_match_oracle(T):
    """Before any update the rasterizer reads the scene's own values, so the
    oracle runs on the synthetic scene itself."""
    sc, views, targets, model, step = setup(T)
    scales = [1.0, 3.0]
    tg = [torch.tensor(t, device="cuda") for t in targets]
    total, info = step.loss(views, tg, scales)
    info = T.per_view_info(info)
    expect = 0.0
    for k, (v, s) in enumerate(zip(views, scales)):
        vv = v.replace(s_v=s)
        s1 = O.stage1(sc, vv)
        img = O.render(sc, vv, s1, O.stage1_f64(sc, vv, s1))["img64"]
        eta_a = OL.eta_actual(int(s1["mask"].sum()), sc.n)
        l1 = float(np.abs(img - targets[k]).mean())
        assert info[k]["eta_actual"] == pytest.approx(eta_a, abs=0)
        assert info[k]["l_render"] == pytest.approx(l1, rel=1e-5, abs=1e-7)
        assert info[k]["l_reg"] == pytest.approx(OL.l_reg(s, eta_a), rel=1e-6, abs=1e-12)
        assert info[k]["w_s"] == pytest.approx(OL.w_s(s, step.s_max), rel=1e-6)    # f32 weights (clod_step_weights)
        expect += OL.l_total(s, step.s_max, l1, eta_a, 1.0) / len(views)
    assert float(total) == pytest.approx(expect, rel=2e-5)
    assert info[1]["l_reg"] > 0          # s_v = 3 at 4000 Gaussians is above target


def test_straight_through_gradient_on_alpha(T):
    sc, views, targets, model, step = setup(T)
    scales = [1.0, 3.0]
    tg = [torch.tensor(t, device="cuda") for t in targets]
    _, info = step.loss(views, tg, scales)
    g = step.dalpha[:2].cpu().numpy()
    per = T.per_view_info(info)
    for k, s in enumerate(scales):
        want = OL.w_s(s, step.s_max) * OL.dlreg_dalpha_ste(s, per[k]["eta_actual"], model.n) / len(views)
        assert g[k] == pytest.approx(want, rel=1e-5, abs=1e-12)


def test_per_view_alpha_gradient_equals_broadcast_array(T):
    """clod_render_bwd with one dL/dalpha'' per view gives the gradients of the
    same constant passed for every (view, Gaussian)."""
    from paper_2510_09997_gb300 import clod as C
    sc, views, targets, model, step = setup(T)
    ds = C.DeviceScene.from_scene(sc)
    fr = C.render(ds, views, want_keys=False)
    L = C.lib()
    dimg = torch.randn_like(fr.image)
    per_view = torch.tensor([0.3, -1.7], device="cuda")
    arr = per_view[:, None].expand(2, sc.n).contiguous()
    nb = ctypes.c_size_t()
    C.check("ws", L.clod_backward_workspace_size(sc.n, 2, ctypes.byref(nb)))
    out = []
    for a_arr, a_view in ((arr, None), (None, per_view)):
        bws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        grads = [torch.zeros_like(t) for t in (ds.means, ds.scales, ds.quats, ds.opacity, ds.sh, ds.decay)]
        C.check("bwd", L.clod_render_bwd(ctypes.byref(ds.c), C._ptr(fr.ws), C._ptr(fr.vals), C._ptr(fr.ranges),
                                         C._ptr(fr.T_final), C._ptr(fr.n_contrib), C._ptr(dimg),
                                         C._ptr(a_arr) if a_arr is not None else None,
                                         C._ptr(a_view) if a_view is not None else None, C._ptr(bws), bws.numel(),
                                         *[C._ptr(g) for g in grads], None))
        out.append([g.cpu().numpy().astype(np.float64) for g in grads])
    for a, b in zip(*out):
        assert np.linalg.norm(a - b) <= 1e-6 * max(np.linalg.norm(b), 1e-30)


def test_overwriting_backward_equals_accumulating_into_zeros(T):
    """clod_render_bwd_set writes every element of the six gradient arrays
    (buffers filled with NaN beforehand), and its values equal
    clod_render_bwd's added into zeroed buffers (up to the order of the
    backward blend's atomic additions, which varies from run to run); a
    second call overwrites instead of adding.  The scene has Gaussians culled
    in both views: their scale, rotation and SH gradients come out as zeros."""
    from paper_2510_09997_gb300 import clod as C
    sc, views, targets, model, step = setup(T)
    ds = C.DeviceScene.from_scene(sc)
    fr = C.render(ds, views, want_keys=False)
    torch.cuda.synchronize()
    assert int((fr.mask.sum(0) == 0).sum()) > 0        # some Gaussians survive in no view
    L = C.lib()
    dimg = torch.randn(fr.image.shape, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    dav = torch.tensor([0.4, -0.9], device="cuda")
    nb = ctypes.c_size_t()
    C.check("ws", L.clod_backward_workspace_size(sc.n, 2, ctypes.byref(nb)))
    bws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")

    def run(fn, grads):
        C.check("bwd", fn(ctypes.byref(ds.c), C._ptr(fr.ws), C._ptr(fr.vals), C._ptr(fr.ranges),
                          C._ptr(fr.T_final), C._ptr(fr.n_contrib), C._ptr(dimg), None, C._ptr(dav),
                          C._ptr(bws), bws.numel(), *[C._ptr(g) for g in grads], None))
        torch.cuda.synchronize()

    acc = [torch.zeros_like(t) for t in (ds.means, ds.scales, ds.quats, ds.opacity, ds.sh, ds.decay)]
    run(L.clod_render_bwd, acc)
    put = [torch.full_like(t, float("nan")) for t in acc]
    culled = (fr.mask.sum(0) == 0).cpu().numpy()
    for _ in range(2):
        run(L.clod_render_bwd_set, put)
        for k, (a, b) in enumerate(zip(acc, put)):
            an, bn = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
            assert not np.isnan(bn).any(), k
            assert np.linalg.norm(an - bn) <= 1e-6 * max(np.linalg.norm(an), 1e-30), k
        for k in (1, 2, 4):      # scales, quats, SH of the Gaussians culled in every view
            assert not put[k].cpu().numpy().reshape(sc.n, -1)[culled].any(), k


def test_fused_adam_matches_torch_adam(T):
    """Three steps of clod_adam_step against torch.optim.Adam in FP64 on the raw
    parameters, with the activation chain rule (log-scale: g s, logit: g a (1-a))
    applied to the same activated-space gradients."""
    from paper_2510_09997_gb300 import abi, clod as C
    sc = S.tiny_scene(n=3001, seed=44, sh_degree=2)
    model = T.GaussianModel(sc)
    rng = np.random.default_rng(9)
    g_act = [rng.normal(size=t.shape).astype(np.float32) for t in model.activated()]
    lr = [1e-3, 2e-3, 3e-3, 4e-2, 5e-3, 1e-2]
    ref = [torch.tensor(t.cpu().numpy().astype(np.float64), requires_grad=True) for t in model.raw()]
    opt = torch.optim.Adam([{"params": [p], "lr": l} for p, l in zip(ref, lr)], betas=(0.9, 0.999), eps=1e-15)
    ne = ctypes.c_int64()
    C.check("size", C.lib().clod_adam_state_size(model.n, model.sh_degree, ctypes.byref(ne)))
    assert ne.value >= sum(t.numel() for t in model.raw())
    m = torch.zeros(ne.value, device="cuda")
    v = torch.zeros_like(m)
    grads = [torch.zeros_like(t) for t in model.activated()]
    P = ctypes.c_void_p * 6
    for t in range(1, 4):
        # reference: chain rule at the current raw values, in FP64
        with torch.no_grad():
            s = torch.exp(ref[1])
            a = torch.sigmoid(ref[3])
        gr = [torch.tensor(g, dtype=torch.float64) for g in g_act]
        gr[1] = gr[1] * s
        gr[3] = gr[3] * a * (1 - a)
        for p, g in zip(ref, gr):
            p.grad = g
        opt.step()
        for gdev, g in zip(grads, g_act):
            gdev.copy_(torch.tensor(g))
        cfg = abi.clod_adam_cfg()
        for k in range(6):
            cfg.lr[k] = lr[k]
        cfg.beta1, cfg.beta2, cfg.eps, cfg.step = 0.9, 0.999, 1e-15, t
        cfg.keep_grads = 1 if t == 2 else 0          # step 2 leaves the gradients as they were
        C.check("adam", C.lib().clod_adam_step(ctypes.byref(cfg), model.n, model.sh_degree,
                                               P(*[C._ptr(p) for p in model.raw()]), P(*[C._ptr(g) for g in grads]),
                                               C._ptr(model.scales), C._ptr(model.opacity), C._ptr(m), C._ptr(v),
                                               None))
        torch.cuda.synchronize()
        if t == 2:
            assert all(np.array_equal(gdev.cpu().numpy(), g) for gdev, g in zip(grads, g_act))
        else:
            assert all(float(g.abs().max()) == 0.0 for g in grads)
    for k, (p, r) in enumerate(zip(model.raw(), ref)):
        d = p.cpu().numpy().astype(np.float64) - r.detach().numpy()
        step_scale = 3 * lr[k]
        assert np.abs(d).max() <= 1e-4 * step_scale + 1e-6 * np.abs(r.detach().numpy()).max(), k
    np.testing.assert_allclose(model.scales.cpu().numpy(), np.exp(ref[1].detach().numpy()), rtol=2e-6)
    np.testing.assert_allclose(model.opacity.cpu().numpy(), 1 / (1 + np.exp(-ref[3].detach().numpy())), rtol=2e-6,
                               atol=1e-7)


def test_short_run_lowers_loss(T):
    sc, views, targets, model, step = setup(T, s_max=1.0)
    tg = [torch.tensor(t, device="cuda") for t in targets]
    first = None
    for it in range(30):
        total, info = step.step(views, tg, [1.0, 1.0])
        total = float(total)
        first = total if first is None else first
    assert total < 0.8 * first


def test_render_loss_kernel_matches_oracle(T):
    """L_render = 0.8 L1 + 0.2 D-SSIM (value and gradient) against the FP64
    oracle, on a ragged image size (tiles and halo borders); the L1-only path
    (w = 0) and the gradient scale too."""
    from oracle import ssim as SS
    from paper_2510_09997_gb300 import autograd as A, clod as C
    rng = np.random.default_rng(70)
    x = rng.uniform(size=(3, 37, 53)).astype(np.float32)
    y = rng.uniform(size=(3, 37, 53)).astype(np.float32)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    loss = A.RenderLoss.apply(xt, torch.tensor(y, device="cuda"), 0.2)
    loss.backward()
    v, g = SS.render_loss_grad(x.astype(np.float64), y.astype(np.float64), 0.2)
    assert abs(float(loss.detach()) - v) < 1e-5 * abs(v)
    gg = xt.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g) / np.linalg.norm(g) < 1e-4
    # w = 0 and a gradient scale of 0.37
    lo = torch.zeros(1, device="cuda")
    gd = torch.empty(3 * 37 * 53, device="cuda")
    xd, yd = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    C.check("l1", C.lib().clod_render_loss(C._ptr(xd), C._ptr(yd), 3, 37, 53, 0.0, 0.37, None, 0, C._ptr(lo),
                                           C._ptr(gd), None))
    v0, g0 = SS.render_loss_grad(x.astype(np.float64), y.astype(np.float64), 0.0)
    assert abs(float(lo) - v0) < 1e-5 * v0
    np.testing.assert_allclose(gd.cpu().numpy().reshape(3, 37, 53), 0.37 * g0, rtol=1e-5, atol=1e-12)


def test_training_step_with_dssim(T):
    sc, views, targets, model, step = setup(T, dssim=0.2)
    tg = [torch.tensor(t, device="cuda") for t in targets]
    first = None
    for it in range(20):
        total, info = step.step(views, tg, [1.0, 1.0])
        total = float(total)
        first = total if first is None else first
    assert total < first


def test_lreg_descent_follows_oracle_counts(T):
    """Gradient descent on L_reg alone (Sec. 3.3, Eq. 3-4) driven by the
    library (mask counts from clod_preprocess, the straight-through scalar
    from clod_lreg_grad, the chain rule to opacity and sigma_d in
    clod_render_bwd) follows the same steps taken with the oracle's counts
    and FP64 gradients: equal counts before the first update, counts within
    a few Gaussians afterwards (updates computed in FP32 and FP64 may put a
    Gaussian that sits on the threshold on either side), and the count falls
    to the target s_v^-1.5 from above."""
    import dataclasses

    from oracle import grad64 as G
    from paper_2510_09997_gb300 import clod as C
    s_v, lr, w, h = 4.0, 1e3, 64, 64
    sc0 = S.tiny_scene(n=3000, seed=5, sh_degree=0)
    v = S.look_at((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), w, h, up=(0.0, 1.0, 0.0), s_v=s_v)
    L = C.lib()
    nb = ctypes.c_size_t()
    C.check("ws", L.clod_backward_workspace_size(sc0.n, 1, ctypes.byref(nb)))
    s_arr = (ctypes.c_float * 1)(s_v)
    w_arr = (ctypes.c_float * 1)(1.0)

    def update(sc, g_op, g_dec):
        a = sc.opacity.astype(np.float64)
        logit = np.log(a / (1.0 - a)) - lr * g_op * a * (1.0 - a)
        return dataclasses.replace(sc, opacity=(1.0 / (1.0 + np.exp(-logit))).astype(np.float32),
                                   decay=(sc.decay.astype(np.float64) - lr * g_dec).astype(np.float32))

    sg = so = sc0
    counts_g, counts_o = [], []
    for it in range(8):
        ds = C.DeviceScene.from_scene(sg)
        fr = C.render(ds, [v], want_keys=False)
        dav = torch.zeros(1, dtype=torch.float32, device="cuda")
        C.check("lreg", L.clod_lreg_grad(C._ptr(fr.counts), sg.n, 1, s_arr, w_arr, ctypes.c_float(1.0), None,
                                         C._ptr(dav), None, None, None))
        bws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        grads = [torch.zeros_like(t) for t in (ds.means, ds.scales, ds.quats, ds.opacity, ds.sh, ds.decay)]
        C.check("bwd", L.clod_render_bwd(ctypes.byref(ds.c), C._ptr(fr.ws), C._ptr(fr.vals), C._ptr(fr.ranges),
                                         C._ptr(fr.T_final), C._ptr(fr.n_contrib), C._ptr(torch.zeros_like(fr.image)),
                                         None, C._ptr(dav), C._ptr(bws), bws.numel(), *[C._ptr(g) for g in grads],
                                         None))
        torch.cuda.synchronize()
        counts_g.append(int(fr.counts[0, 0]))
        sg = update(sg, grads[3].cpu().numpy().astype(np.float64), grads[5].cpu().numpy().astype(np.float64))
        # the same step on the oracle
        cnt = int(O.stage1(so, v)["mask"].sum())
        counts_o.append(cnt)
        g = OL.dlreg_dalpha_ste(s_v, OL.eta_actual(cnt, so.n), so.n)
        if it == 0:
            assert float(dav[0]) == pytest.approx(g, rel=1e-6)
        gr = G.reference_gradients(so, [v], [np.zeros((3, h, w))], [np.full(so.n, g)])
        so = update(so, gr["opacity"], gr["decay"])
    assert counts_g[0] == counts_o[0]
    assert max(abs(a - b) for a, b in zip(counts_g, counts_o)) <= 3
    target = OL.eta_target(s_v) * sc0.n
    assert counts_g[0] > 3 * target and all(b <= a for a, b in zip(counts_g, counts_g[1:]))
    assert counts_g[-1] <= target + 0.01 * sc0.n
