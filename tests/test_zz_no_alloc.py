"""The allocation-free coarse-to-fine entry point (bayer_me_estimate_c2f_noalloc).

Some callers cannot call cudaMalloc once they are running (a real-time frame
loop, or a host that fixes its device-memory budget at start-up), so the
library offers a coarse-to-fine search whose scratch is a static 1 MiB device
array instead of handle workspace.  This checks, through the C ABI, that two
calls in a row give exactly the fields the handle-based entry point gives on
the same inputs (motion vectors are integers: bit-exact), that the second
call's RAW three-level field also equals the CPU oracle's, that a run of calls
leaves the device's free memory unchanged, and that a request too large for
the static scratch is refused without running.

The file is named to be collected last, so a stop-at-first-failure run has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2508_05990_b300 import bayer_me as bm
from paper_2508_05990_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05990_b300 import build
    build.build()
    h = bm.Handle(0)
    yield h
    h.close()


def _pairs(seed, H, W, n):
    frames = synth.pan_clip(seed, H, W, n_frames=n + 1)
    return torch.from_numpy(frames).cuda()


def test_noalloc_matches_handle_path_on_two_calls(handle):
    H, W = 720, 960
    d = _pairs(70, H, W, 2)
    # call 1: EVEN phase, standard setting, 2 pairs batched
    want1 = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, phase=bm.PHASE_EVEN, batch=2,
                               ref_batch_stride=H * W, cur_batch_stride=H * W)
    got1 = bm.estimate_c2f_noalloc(d, d[1:], phase=bm.PHASE_EVEN, batch=2, ref_batch_stride=H * W,
                                   cur_batch_stride=H * W)
    # call 2: other frames, RAW phase, three levels (the scratch keeps call 1's contents)
    e = _pairs(71, H, W, 1)
    setting = bm.C2FSetting((64, 32, 16), ((8, 8), (4, 4), (2, 1)))
    want2 = handle.estimate_ex(e[0], e[1], mode=bm.MODE_C2F, phase=bm.PHASE_RAW, c2f=setting)
    got2 = bm.estimate_c2f_noalloc(e[0], e[1], c2f=setting, phase=bm.PHASE_RAW)
    torch.cuda.synchronize()
    assert torch.equal(got1, want1)
    assert torch.equal(got2, want2)
    assert handle.sync_status() == bm.OK
    # the RAW three-level field against the oracle directly
    fr = e.cpu().numpy()
    want, _ = oracle.me_c2f(fr[0], fr[1], setting.levels, setting.stages, even=False)
    g = bm.records_to_numpy(got2[0])
    for k in ("dx", "dy", "sad"):
        np.testing.assert_array_equal(g[k], want[k])


def test_noalloc_leaves_free_memory_unchanged(handle):
    """After a first call (address look-up, kernels loaded), further calls with
    a preallocated output take no device memory: the device's free memory is
    the same before and after a run of them."""
    H, W = 720, 960
    d = _pairs(72, H, W, 2)
    out = torch.empty((2, H // 32 + 1, W // 32, 2), dtype=torch.int32, device="cuda")
    kw = dict(phase=bm.PHASE_EVEN, batch=2, ref_batch_stride=H * W, cur_batch_stride=H * W, out=out)
    bm.estimate_c2f_noalloc(d, d[1:], **kw)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        bm.estimate_c2f_noalloc(d, d[1:], **kw)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    want = handle.estimate_ex(d, d[1:], mode=bm.MODE_C2F, phase=bm.PHASE_EVEN, batch=2, ref_batch_stride=H * W,
                              cur_batch_stride=H * W)
    torch.cuda.synchronize()
    assert torch.equal(out, want)


def test_noalloc_rejects_requests_beyond_the_scratch(handle):
    # 4 levels at 4K: the level-16 intermediate field is 240 x 135 records per
    # pair; 8 pairs need 2 x 259200 records > 131072 (1 MiB of 8-byte records)
    H, W = 2160, 3840
    f = torch.zeros((H, W), dtype=torch.int16, device="cuda")
    setting = bm.C2FSetting((64, 32, 16, 8), ((8, 8), (4, 4), (2, 1)))
    out = torch.empty((8, H // 8, W // 8, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(bm.BayerError) as err:
        bm.estimate_c2f_noalloc(f, f, c2f=setting, batch=8, out=out)
    assert err.value.status == bm.ERR_UNSUPPORTED
