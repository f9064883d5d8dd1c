"""CUDA adjoint of the merge vs the FP64 oracle adjoint (itself pinned by central finite
differences), through the C-ABI; 1e-3 relative."""
import numpy as np
import pytest
import torch

import burstgen
import oracle
import paper_1905_03277_gb300 as hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hm.build()
    return torch.device("cuda:0")


def case(seed, h, w, n, scale, robust=True):
    b = burstgen.make_burst(dict(n=n, h=h, w=w, gain=1.0, read=3.0, motion="global", scale=(1, 1)), seed=seed)
    raw = b["raw"].numpy()
    _, mf, _, _ = oracle.align(raw)
    mv = mf.astype(np.float32)
    mv[min(2, n - 1), 1, 2] += np.float32(0.9)
    p = hm.MergeParams(k_detail=0.3, k_denoise=3.0, d_th=0.004, d_tr=0.05, k_stretch=3.0, k_shrink=1.8, t=0.12,
                       s1=12.0, s2=1.1 if robust else 2.0, m_th=3.0, noise_a=0.02, noise_b=0.5)
    ho, wo = hm.out_size(h, w, scale)
    g = np.random.default_rng(seed).normal(size=(3, ho, wo))
    return raw, mv, p, g


def oparams(p):
    return oracle.MergeParams(**{k: getattr(p, k) for k in oracle.MergeParams.__dataclass_fields__})


def assert_adjoint_close(gp, gm, ogp, ogm, ref):
    """Each of the 8 parameter gradients within 1e-3 relative of the oracle's, on its own
    (exactly 0 where the oracle's is exactly 0: no texel depends on that parameter);
    each motion-gradient element within 1e-3 relative of the oracle's, with an absolute
    floor of 1e-5 of the field's largest element for elements that are near zero (the
    FP32 rounding of the sums that produce them)."""
    gp = gp.cpu().numpy().astype(np.float64)
    gm = gm.cpu().numpy().astype(np.float64)
    assert np.isfinite(gp).all() and np.isfinite(gm).all()
    for k, name in enumerate(hm.PARAM_NAMES):
        if ogp[k] == 0.0:
            assert gp[k] == 0.0, (name, gp[k])
            continue
        assert gp[k] == pytest.approx(ogp[k], rel=1e-3), (name, gp[k], ogp[k])
    floor = 1e-5 * np.abs(ogm).max()
    bad = np.abs(gm - ogm) > 1e-3 * np.abs(ogm) + floor
    assert not bad.any(), (int(bad.sum()), np.abs(gm - ogm)[bad].max(), np.abs(ogm)[bad].min())
    assert np.all(gm[ref] == 0)


@pytest.mark.parametrize("scale,ref", [((1, 1), 0), ((3, 2), 1), ((2, 1), 0)])
def test_adjoint_matches_oracle(dev, scale, ref):
    raw, mv, p, g = case(51, 64, 96, 4, scale)
    burst = torch.from_numpy(raw).to(dev)
    motion = torch.from_numpy(mv).to(dev)
    rgb, den = hm.merge(burst, motion, p, scale, ref, with_den=True)
    gp, gm = hm.merge_backward(burst, motion, p, rgb, den, torch.from_numpy(g).float().to(dev), scale, ref)
    ogp, ogm = oracle.merge_backward(raw, mv, oparams(p), g, scale=scale, ref=ref)
    assert_adjoint_close(gp, gm, ogp, ogm, ref)


def test_adjoint_on_the_fitting_workload(dev):
    # a 256 x 256 crop (even offsets keep the RGGB phase) of an 8-frame 1024 x 1024
    # fitting burst, 1.5x output, the fit's starting parameters and noise model, the
    # oracle's alignment of the crop, and the gradient of an L2 loss against the
    # burst's ground truth.  (Here the robustness saturates at 1 wherever s2 applies,
    # so dL/ds2 is exactly 0 on both sides.)
    b = burstgen.make_burst("fit", seed=burstgen.SEED_BASE + 3, device=dev, with_gt=True)
    y0, x0 = 384, 512
    raw = b["raw"][:, y0:y0 + 256, x0:x0 + 256].contiguous().cpu().numpy()
    gt = b["gt"].cpu().numpy()[:, y0 * 3 // 2:(y0 + 256) * 3 // 2, x0 * 3 // 2:(x0 + 256) * 3 // 2]
    _, mf, _, _ = oracle.align(raw)
    mv = mf.astype(np.float32)
    p = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
    scale = (3, 2)
    burst = torch.from_numpy(raw).to(dev)
    motion = torch.from_numpy(mv).to(dev)
    rgb, den = hm.merge(burst, motion, p, scale, 0, with_den=True)
    orgb = oracle.merge(raw, mv, oparams(p), scale=scale)
    g = 2.0 * (orgb - gt) / orgb.size          # dL/drgb of the mean squared error
    gp, gm = hm.merge_backward(burst, motion, p, rgb, den, torch.from_numpy(g).float().to(dev), scale, 0)
    ogp, ogm = oracle.merge_backward(raw, mv, oparams(p), g, scale=scale)
    assert_adjoint_close(gp, gm, ogp, ogm, 0)


def test_autograd_function_and_descent(dev):
    raw, mv, p, _ = case(52, 64, 64, 4, (1, 1))
    burst = torch.from_numpy(raw).to(dev)
    motion = torch.from_numpy(mv).to(dev).requires_grad_(True)
    theta = torch.tensor([getattr(p, k) for k in hm.PARAM_NAMES], dtype=torch.float32, requires_grad=True)
    target = hm.merge(burst, motion.detach(), p).detach() * 0.98
    rgb = hm.MergeFn.apply(theta, motion, burst, p, (1, 1), 0)
    loss = ((rgb - target) ** 2).mean()
    loss.backward()
    assert theta.grad is not None and motion.grad is not None
    assert torch.isfinite(theta.grad).all() and torch.isfinite(motion.grad).all()
    # a small step against the gradient lowers the loss
    with torch.no_grad():
        theta2 = theta - 1e-4 * theta.grad / theta.grad.abs().max()
        rgb2 = hm.MergeFn.apply(theta2, motion.detach(), burst, p, (1, 1), 0)
        assert ((rgb2 - target) ** 2).mean() < loss


def test_fit_lowers_loss_against_ground_truth(dev):
    from paper_1905_03277_gb300.fit import fit
    bursts, gts = [], []
    for k in range(2):
        b = burstgen.make_burst(dict(n=4, h=128, w=128, gain=1.0, read=3.0, motion="global", scale=(3, 2)),
                                seed=60 + k, device=dev, with_gt=True)
        bursts.append(b["raw"])
        gts.append(b["gt"])
    base = hm.MergeParams(noise_a=1.0, noise_b=9.0)
    params, hist, motions = fit(bursts, gts, base, steps=15, scale=(3, 2))
    assert hist[-1] < hist[0]
    assert all(getattr(params, k) > 0 for k in hm.PARAM_NAMES)


@pytest.mark.parametrize("scale", [(1, 1), (3, 2), (2, 1)])
def test_prepared_adjoint_equals_full_adjoint(dev, scale):
    # hmfsr_merge_backward_prepared on the forward's workspace gives the same bits as the
    # adjoint that prepares the planes itself
    raw, mv, p, g = case(31, 64, 96, 4, scale)
    b = torch.from_numpy(raw).to(dev)
    m = torch.from_numpy(mv).to(dev)
    gr = torch.from_numpy(g.astype(np.float32)).to(dev)
    ws = hm.backward_workspace(tuple(b.shape), p.tile, scale, dev)
    rgb, den = hm.merge(b, m, p, scale, with_den=True, workspace=ws)
    assert torch.equal(rgb, hm.merge(b, m, p, scale))
    gp1, gm1 = hm.merge_backward(b, m, p, rgb, den, gr, scale, workspace=ws, prepared=True)
    gp0, gm0 = hm.merge_backward(b, m, p, rgb, den, gr, scale)
    torch.cuda.synchronize()
    assert torch.equal(gp1, gp0) and torch.equal(gm1, gm0)
    with pytest.raises(ValueError):
        hm.merge_backward(b, m, p, rgb, den, gr, scale, prepared=True)
