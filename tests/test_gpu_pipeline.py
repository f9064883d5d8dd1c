"""The pipelined public call (copies of one burst overlapped with the compute of another)
gives, burst by burst, exactly what the plain align + merge call gives."""
import pytest
import torch

import burstgen
import paper_1905_03277_gb300 as hm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hm.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("scale,depth", [((1, 1), 2), ((3, 2), 3)])
def test_pipeline_matches_plain_calls(dev, scale, depth):
    bursts = [burstgen.make_burst("tiny", seed=burstgen.SEED_BASE + 40 + i)["raw"].pin_memory() for i in range(5)]
    p = hm.MergeParams(noise_a=0.5, noise_b=4.0)
    ho, wo = hm.out_size(bursts[0].shape[1], bursts[0].shape[2], scale)
    outs = [torch.full((3, ho, wo), -1.0, pin_memory=True) for _ in bursts]
    pipe = hm.AlignMergePipeline(tuple(bursts[0].shape), p, scale, device=dev, depth=depth)
    for b, o in zip(bursts, outs):
        pipe.submit(b, o)
    pipe.synchronize()
    for b, o in zip(bursts, outs):
        want = hm.align_merge(b, p, scale)
        torch.cuda.synchronize()
        assert torch.equal(o, want)


def test_pipeline_rejects_wrong_shape(dev):
    pipe = hm.AlignMergePipeline((4, 64, 96), device=dev)
    with pytest.raises(ValueError):
        pipe.submit(torch.zeros((4, 64, 98), dtype=torch.uint16), torch.empty((3, 64, 98)))
