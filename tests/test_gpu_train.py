"""The virtual-distance training step (Sec. 3.3) on the GPU against the
oracle: loss scalars (Eq. 3-5) from the oracle's mask counts and FP64 image,
the straight-through gradient delivered to alpha'', and a short run that
lowers the loss."""
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


def setup(T, s_max=8.0):
    sc = S.tiny_scene(n=4000, seed=40, sh_degree=1)
    views = [S.tiny_view(1.0).replace(width=96, height=96, cx=48.0, cy=48.0),
             S.look_at((2.2, 1.0, 1.2), (0, 0, 0), 80, 64)]
    targets = [S.target_image(v.height, v.width, seed=k) for k, v in enumerate(views)]
    model = T.GaussianModel(sc)
    step = T.TrainStep(model, s_max=s_max, lam_reg=1.0, dssim_weight=0.0)
    return sc, views, targets, model, step


def test_loss_scalars_match_oracle(T):
    sc, views, targets, model, step = setup(T)
    scales = [1.0, 3.0]
    tg = [torch.tensor(t, device="cuda") for t in targets]
    total, info = step.loss(views, tg, scales)
    # the model's activated parameters, as the rasterizer saw them
    act = [t.detach().cpu().numpy() for t in model.activated()]
    scene = S.Scene(*act)
    expect = 0.0
    for k, (v, s) in enumerate(zip(views, scales)):
        vv = v.replace(s_v=s)
        s1 = O.stage1(scene, vv)
        img = O.render(scene, vv, s1, O.stage1_f64(scene, vv, s1))["img64"]
        eta_a = OL.eta_actual(int(s1["mask"].sum()), scene.n)
        l1 = float(np.abs(img - targets[k]).mean())
        assert info[k]["eta_actual"] == pytest.approx(eta_a, abs=0)
        assert info[k]["l1"] == pytest.approx(l1, rel=1e-5, abs=1e-7)
        assert info[k]["l_reg"] == pytest.approx(OL.l_reg(s, eta_a), rel=1e-6, abs=1e-12)
        assert info[k]["w_s"] == pytest.approx(OL.w_s(s, step.s_max), rel=1e-12)
        expect += OL.l_total(s, step.s_max, l1, eta_a, 1.0) / len(views)
    assert float(total) == pytest.approx(expect, rel=2e-5)
    assert info[1]["l_reg"] > 0          # s_v = 3 at 4000 Gaussians is above target


def test_straight_through_gradient_on_alpha(T):
    sc, views, targets, model, step = setup(T)
    scales = [1.0, 3.0]
    tg = [torch.tensor(t, device="cuda") for t in targets]
    total, info = step.loss(views, tg, scales)
    alpha = step.last["alpha"]
    g = torch.autograd.grad(total, alpha)[0].cpu().numpy()
    for k, s in enumerate(scales):
        want = OL.w_s(s, step.s_max) * OL.dlreg_dalpha_ste(s, info[k]["eta_actual"], model.n) / len(views)
        assert np.allclose(g[k], want, rtol=1e-5, atol=1e-12)


def test_short_run_lowers_loss(T):
    sc, views, targets, model, step = setup(T, s_max=1.0)
    tg = [torch.tensor(t, device="cuda") for t in targets]
    first = None
    for it in range(30):
        total, info = step.step(views, tg, [1.0, 1.0])
        first = total if first is None else first
    assert total < 0.8 * first


def test_render_loss_kernel_matches_oracle(T):
    """L_render = 0.8 L1 + 0.2 D-SSIM (value and gradient) against the FP64
    oracle, on a ragged image size (tiles and halo borders)."""
    from oracle import ssim as SS
    from paper_2510_09997_gb300 import autograd as A
    rng = np.random.default_rng(70)
    x = rng.uniform(size=(3, 37, 53)).astype(np.float32)
    y = rng.uniform(size=(3, 37, 53)).astype(np.float32)
    xt = torch.tensor(x, device="cuda", requires_grad=True)
    loss = A.RenderLoss.apply(xt, torch.tensor(y, device="cuda"), 0.2)
    loss.backward()
    v, g = SS.render_loss_grad(x.astype(np.float64), y.astype(np.float64), 0.2)
    assert abs(float(loss) - v) < 1e-5 * abs(v)
    gg = xt.grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g) / np.linalg.norm(g) < 1e-4


def test_training_step_with_dssim(T):
    sc, views, targets, model, step = setup(T)
    step.dssim = 0.2
    tg = [torch.tensor(t, device="cuda") for t in targets]
    first = None
    for it in range(20):
        total, info = step.step(views, tg, [1.0, 1.0])
        first = total if first is None else first
    assert total < first
