"""Many streams of mixed sizes in one persistent launch (bayer_me_multi_stream):
every pair's MV field equals the single-pair search and the oracle bit for
bit, propagated features equal the float oracle bit for bit, and a second
call (cached CUDA graph, refreshed descriptor table) is exact too."""
import numpy as np
import pytest

import oracle
from paper_2508_05990_b300 import bayer_me as bm
from paper_2508_05990_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [(128, 160, 32, 8), (128, 160, 16, 4), (272, 480, 32, 8), (96, 64, 8, 16), (64, 96, 0, 8)]


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05990_b300 import build
    build.build()
    h = bm.Handle(0)
    yield h
    h.close()


def make(seed):
    streams = []
    for i, (H, W, C, s) in enumerate(SIZES):
        fr = synth.pan_clip(seed + i, H, W, n_frames=2, rect_size=(8, 48))
        q = {"np": fr, "ref": torch.from_numpy(fr[0]).cuda(), "cur": torch.from_numpy(fr[1]).cuda(),
             "mv": torch.empty((H // 16, W // 16, 2), dtype=torch.int32, device="cuda"), "stride": s}
        if C:
            f = synth.features(seed + 50 + i, C, H // s, W // s)[0]
            q.update(feat_np=f, feat=torch.from_numpy(f).cuda(), feat_out=torch.empty((C, H // s, W // s), device="cuda"))
        streams.append(q)
    return streams


@pytest.mark.parametrize("search_range", [32, 16])
def test_multi_stream_exact(handle, search_range):
    end = torch.zeros(len(SIZES), dtype=torch.int64, device="cuda")
    for call, seed in enumerate((300, 400)):
        streams = make(seed + search_range)
        sched = handle.multi_stream(streams, search_range, end_ns=end)
        torch.cuda.synchronize()
        assert sched in (40, 41, 80, 81)
        assert handle.sync_status() == bm.OK
        assert (end.cpu().numpy() > 0).all()
        for q in streams:
            single = handle.estimate(q["ref"], q["cur"], 16, search_range)
            torch.cuda.synchronize()
            assert torch.equal(q["mv"], single)
            want, _ = oracle.me_full(q["np"][0], q["np"][1], 16, search_range, even=True)
            got = bm.records_to_numpy(q["mv"])
            for k in ("dx", "dy", "sad"):
                np.testing.assert_array_equal(got[k], want[k])
            if "feat" in q:
                pw = oracle.propagate(q["feat_np"], want, 16, q["stride"], interp=oracle.BILINEAR)
                np.testing.assert_array_equal(q["feat_out"].cpu().numpy().view(np.uint32), pw.view(np.uint32))


def test_multi_stream_rejects_bad_sizes(handle):
    fr = torch.zeros((40, 64), dtype=torch.int16, device="cuda")
    mv = torch.empty((2, 4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(bm.BayerError):
        handle.multi_stream([{"ref": fr, "cur": fr, "mv": mv}], 32)  # H not a multiple of 16
