"""The bounded-memory merge (hmfsr_merge_chunked: frames prepared and accumulated a chunk
at a time, the running sums kept per output pixel between chunks) gives exactly what the
resident merge gives, for every chunk size, scale and base frame, with and without the
log2-denominator output."""
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


@pytest.fixture(scope="module")
def tiny(dev):
    b = burstgen.make_burst("tiny", seed=burstgen.SEED_BASE + 80, device=dev)
    return b, hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)


@pytest.mark.parametrize("scale", [(1, 1), (3, 2), (2, 1)])
@pytest.mark.parametrize("ref", [0, 3, 7])
def test_chunked_equals_resident(dev, tiny, scale, ref):
    b, p = tiny
    raw = b["raw"]
    mv = hm.align(raw, ref)
    want, wden = hm.merge(raw, mv, p, scale, ref, with_den=True)
    for k in (1, 2, 3, 7, 8):
        got, gden = hm.merge_chunked(raw, mv, p, scale, ref, chunk_frames=k, with_den=True)
        assert torch.equal(got, want), (k, scale, ref)
        assert torch.equal(gden, wden), (k, scale, ref)


def test_chunked_ragged_and_single_frame(dev):
    b = burstgen.make_burst(dict(n=5, h=136, w=200, gain=2.0, read=4.0, motion="global", scale=(1, 1)),
                            seed=burstgen.SEED_BASE + 81, device=dev)
    raw = b["raw"]
    p = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2)
    for ref, scale in ((2, (1, 1)), (4, (2, 1)), (0, (3, 2))):
        mv = hm.align(raw, ref)
        want = hm.merge(raw, mv, p, scale, ref)
        for k in (1, 3, 4):
            assert torch.equal(hm.merge_chunked(raw, mv, p, scale, ref, chunk_frames=k), want), (ref, scale, k)
    one = raw[:1].contiguous()
    mv1 = torch.zeros((1,) + tuple(hm.n_tiles(136, 200, 16)) + (2,), dtype=torch.float32, device=dev)
    assert torch.equal(hm.merge_chunked(one, mv1, p, (2, 1), 0, chunk_frames=2), hm.merge(one, mv1, p, (2, 1)))


def test_chunked_in_a_graph(dev, tiny):
    b, p = tiny
    raw = b["raw"]
    mv = hm.align(raw, 0)
    want = hm.merge(raw, mv, p, (1, 1))
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        hm.merge_chunked(raw, mv, p, (1, 1), 0, chunk_frames=3, stream=s)  # workspace outside capture
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        out = hm.merge_chunked(raw, mv, p, (1, 1), 0, chunk_frames=3, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, want)
