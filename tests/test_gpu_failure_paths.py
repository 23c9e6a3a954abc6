"""Failure paths without a GPU fault.

* Device: the bounded mbarrier wait that every tensor-core kernel uses runs out
  when nothing arrives, records BAYER_ERR_TIMEOUT in the handle's status word,
  and the kernel finishes; the context stays usable and the status is read
  and cleared by bayer_me_sync_status.  With the arrival the wait succeeds.
* Host: a workspace allocation that fails (simulated by the test hook)
  returns BAYER_ERR_OOM and launches nothing; the next call allocates and
  gives the oracle's result.
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


def test_bounded_wait_times_out_and_context_survives(handle):
    assert handle.sync_status() == bm.OK
    handle.selftest_wait(arrive=True, limit=1000)
    assert handle.sync_status() == bm.OK
    handle.selftest_wait(arrive=False, limit=2000)
    assert handle.sync_status() == bm.ERR_TIMEOUT
    assert handle.sync_status() == bm.OK  # read and cleared
    # the context is intact: a search right after gives the oracle's field
    f0, f1, _ = synth.planted_pair(1000)
    mv = handle.estimate(torch.from_numpy(f0).cuda(), torch.from_numpy(f1).cuda(), 16, 16)
    want, _ = oracle.me_full(f0, f1, 16, 16, even=True)
    got = bm.records_to_numpy(mv)
    for k in ("dx", "dy", "sad"):
        np.testing.assert_array_equal(got[k], want[k])


def test_simulated_allocation_failure():
    """A fresh handle (no workspace yet): the C2F search needs the handle's
    scratch for its intermediate level."""
    h = bm.Handle(0)
    try:
        frames = synth.pan_clip(31, 128, 192, n_frames=2)
        d = torch.from_numpy(frames.view(np.int16)).cuda()
        h.debug_fail_allocs(1)
        with pytest.raises(bm.BayerError) as err:
            h.estimate_ex(d[0], d[1], mode=bm.MODE_C2F)
        assert err.value.status == bm.ERR_OOM
        out = h.estimate_ex(d[0], d[1], mode=bm.MODE_C2F)
        torch.cuda.synchronize()
        assert h.sync_status() == bm.OK
        want, _ = oracle.me_c2f(frames[0], frames[1], [64, 32], [(8, 8), (4, 4), (2, 1)], even=True)
        got = bm.records_to_numpy(out[0])
        for k in ("dx", "dy", "sad"):
            np.testing.assert_array_equal(got[k], want[k])
    finally:
        h.close()
