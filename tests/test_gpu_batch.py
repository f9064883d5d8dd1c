"""Ragged batches through one persistent, graph-captured launch (hmfsr_batch_*): every
burst's integer vectors bit-exact and its merge within the merge bar against the FP64
oracle; outputs bit-identical to aligning and merging each burst on its own; the bounded
dependency waits report HMFSR_ERR_TIMEOUT (without faulting) when a dependency never
completes."""
import numpy as np
import pytest
import torch

import burstgen
import oracle
import paper_1905_03277_gb300 as hm
from _parity import assert_merge_close, assert_motion_matches_oracle, oparams

pytestmark = pytest.mark.gpu

CASES = [  # (n, h, w, scale, ref)
    (4, 136, 200, (1, 1), 0),
    (6, 96, 128, (3, 2), 2),
    (3, 256, 192, (2, 1), 1),
    (8, 64, 64, (1, 1), 0),
    (5, 200, 264, (3, 2), 4),
    (2, 48, 80, (2, 1), 0),
]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hm.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def batch(dev):
    bursts, params = [], []
    for k, (n, h, w, sc, ref) in enumerate(CASES):
        b = burstgen.make_burst(dict(n=n, h=h, w=w, gain=1.0 + k, read=2.0 + k, motion="global", scale=sc),
                                seed=70 + k, device=dev)
        bursts.append(b["raw"])
        params.append(hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2))
    plain_rgb, plain_mv = [], []
    for raw, p, (n, h, w, sc, ref) in zip(bursts, params, CASES):
        mv = hm.align(raw, ref, hm.AlignParams())
        plain_mv.append(mv)
        plain_rgb.append(hm.merge(raw, mv, p, sc, ref))
    torch.cuda.synchronize()
    return bursts, params, plain_rgb, plain_mv


def make_plan(bursts, params):
    return hm.BatchPlan([tuple(b.shape) for b in bursts], params, [c[3] for c in CASES], [c[4] for c in CASES])


def test_batch_bit_identical_to_plain(dev, batch):
    bursts, params, plain_rgb, plain_mv = batch
    plan = make_plan(bursts, params)
    rgbs = plan.outputs(dev)
    mvs = [torch.full_like(m, float("nan")) for m in plain_mv]
    for _ in range(2):  # graph built on the first run, replayed on the second
        for r in rgbs:
            r.fill_(float("nan"))
        plan.run(bursts, rgbs, mvs, wait=True)
        for k in range(len(CASES)):
            assert torch.equal(mvs[k], plain_mv[k]), f"motion of burst {k}"
            assert torch.equal(rgbs[k], plain_rgb[k]), f"rgb of burst {k}"


def test_batch_matches_the_oracle(dev, batch):
    # each burst of the ragged batch (6 shapes, 3 scales, refs 0-4) against the oracle
    # directly: its alignment from the same frames, and its merge given the batch's own
    # float32 motion
    bursts, params, _, _ = batch
    plan = make_plan(bursts, params)
    rgbs = plan.outputs(dev)
    mvs = [torch.empty((n,) + hm.n_tiles(h, w, 16) + (2,), dtype=torch.float32, device=dev)
           for (n, h, w, _, _) in CASES]
    plan.run(bursts, rgbs, mvs, wait=True)
    for k, (n, h, w, sc, ref) in enumerate(CASES):
        raw_np = bursts[k].cpu().numpy()
        g_int = plan.vectors(k).cpu().numpy()
        g_mv = mvs[k].cpu().numpy()
        assert_motion_matches_oracle(g_int, g_mv, raw_np, ref)
        want = oracle.merge(raw_np, g_mv, oparams(params[k]), scale=sc, ref=ref)
        assert_merge_close(rgbs[k].cpu().numpy(), want, f"burst {k}: {n}x{h}x{w}, scale {sc}, ref {ref}")


def test_batch_stage_profile(dev, batch):
    # the persistent kernel's per-stage counters: every stage that has work records items
    # and cycles, and profiling leaves the results unchanged
    bursts, params, plain_rgb, _ = batch
    plan = make_plan(bursts, params)
    plan.set_mode(0)
    plan.set_profile(True)
    rgbs = plan.outputs(dev)
    plan.run(bursts, rgbs, wait=True)
    prof = plan.stage_profile()
    for name in ("luminance", "preparation", "matching 0", "lucas-kanade", "robustness", "accumulation"):
        wait, run, items = prof[name]
        assert items > 0 and run > 0, (name, prof[name])
    for k in range(len(CASES)):
        assert torch.equal(rgbs[k], plain_rgb[k])


def test_batch_timeout_is_reported_and_recovers(dev, batch):
    bursts, params, plain_rgb, _ = batch
    plan = make_plan(bursts, params)
    rgbs = plan.outputs(dev)
    plan.configure(inject_stall=True, spin_limit=2000)   # a dependency nothing satisfies
    with pytest.raises(RuntimeError, match="timed out"):
        plan.run(bursts, rgbs, wait=True)
    plan.configure(inject_stall=False)
    plan.run(bursts, rgbs, wait=True)
    for k in range(len(CASES)):
        assert torch.equal(rgbs[k], plain_rgb[k])


def test_batch_autotune_keeps_results(dev, batch):
    bursts, params, plain_rgb, _ = batch
    plan = make_plan(bursts, params)
    rgbs = plan.outputs(dev)
    best, log = plan.tune(bursts, rgbs)
    assert best > 0 and all(v > 0 for v in log.values())
    plan.run(bursts, rgbs, wait=True)
    for k in range(len(CASES)):
        assert torch.equal(rgbs[k], plain_rgb[k])
    # the graph mode (per-burst kernels on parallel branches) gives the same bits
    for streams in (1, 3):
        plan.set_mode(streams)
        for r in rgbs:
            r.fill_(float("nan"))
        plan.run(bursts, rgbs, wait=True)
        for k in range(len(CASES)):
            assert torch.equal(rgbs[k], plain_rgb[k])
