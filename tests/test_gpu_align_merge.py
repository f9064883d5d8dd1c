"""The one-call path (hmfsr_align_merge: the merge's motion-free preparation beside the
alignment, on two streams joined by events) gives exactly what hmfsr_align followed by
hmfsr_merge gives, on tiny, ragged and 2x inputs, with any base frame, inside a
captured CUDA graph, and when calls alternate between streams."""
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


def sequential(raw, p, ap, scale, ref):
    motion = hm.align(raw, ref, ap)
    return hm.merge(raw, motion, p, scale, ref), motion


CASES = [
    ("tiny", (1, 1), 0, hm.AlignParams()),
    ("tiny", (3, 2), 3, hm.AlignParams()),
    ("tiny", (2, 1), 7, hm.AlignParams(n_levels=2, lk_iters=1)),
    (dict(n=5, h=136, w=200, gain=2.0, read=4.0, motion="global", scale=(1, 1)), (1, 1), 2, hm.AlignParams()),
    (dict(n=3, h=100, w=148, gain=1.0, read=2.0, motion="global", scale=(1, 1)), (2, 1), 0,
     hm.AlignParams(tile=32, radius=(2, 3, 4, 4))),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_one_call_matches_align_then_merge(dev, case):
    spec, scale, ref, ap = CASES[case]
    b = burstgen.make_burst(spec, seed=burstgen.SEED_BASE + 60 + case, device=dev)
    raw = b["raw"]
    p = hm.MergeParams(noise_a=b["gain"], noise_b=b["read"] ** 2, tile=ap.tile)
    want, want_m = sequential(raw, p, ap, scale, ref)
    got, got_m = hm.align_merge(raw, p, scale, ref, ap, with_motion=True)
    torch.cuda.synchronize()
    assert torch.equal(got_m, want_m)
    assert torch.equal(got, want)


def test_one_call_in_a_graph_and_across_streams(dev):
    b1 = burstgen.make_burst("tiny", seed=burstgen.SEED_BASE + 70, device=dev)
    b2 = burstgen.make_burst("tiny", seed=burstgen.SEED_BASE + 71, device=dev)
    p = hm.MergeParams(noise_a=b1["gain"], noise_b=b1["read"] ** 2)
    ap = hm.AlignParams()
    want1, _ = sequential(b1["raw"], p, ap, (3, 2), 0)
    want2, _ = sequential(b2["raw"], p, ap, (3, 2), 0)
    torch.cuda.synchronize()
    # alternating streams: the calls share the thread's side stream, each joins its own
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    outs = []
    for k in range(4):
        s = (s1, s2)[k & 1]
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            outs.append(hm.align_merge((b1, b2)[k & 1]["raw"], p, (3, 2), 0, ap, stream=s))
    torch.cuda.synchronize()
    for k, o in enumerate(outs):
        assert torch.equal(o, (want1, want2)[k & 1])
    # captured into a graph and replayed on a new input
    raw = b1["raw"].clone()
    out = torch.empty_like(want1)
    cs = torch.cuda.Stream(dev)
    cs.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(cs):
        hm.align_merge(raw, p, (3, 2), 0, ap, out=out, stream=cs)  # workspace of this stream, outside capture
    cs.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        hm.align_merge(raw, p, (3, 2), 0, ap, out=out, stream=cs)
    raw.copy_(b2["raw"])
    out.fill_(-1.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, want2)


def test_one_call_rejects_mismatched_tiles(dev):
    b = burstgen.make_burst("tiny", seed=burstgen.SEED_BASE + 72, device=dev)
    with pytest.raises(ValueError):
        hm.align_merge(b["raw"], hm.MergeParams(tile=16), (1, 1), 0, hm.AlignParams(tile=32))
