"""Checkpoint/resume of the proposal-network trainer (host logic, CPU only):
an interrupted run resumed from its checkpoint ends in exactly the state of an
uninterrupted run, and the cosine schedule spans lr0 -> lr_min."""
import numpy as np

from paper_2508_05990_b300.train_proposal import Trainer, cosine_lr


def make(ckpt, state):
    def step_fn(idx, lr, step):
        g = np.sin(np.asarray(idx, np.float64).sum() + step)
        state["w"] = state["w"] - lr * g * np.arange(1, 5)
        state["m"] = 0.9 * state["m"] + g
        return float(g * g)

    def get_state():
        return {k: v.copy() for k, v in state.items()}

    def set_state(st):
        state.update({k: np.asarray(v, np.float64).copy() for k, v in st.items()})

    return Trainer(40, 8, 6, 1e-2, 1e-4, step_fn, get_state, set_state, ckpt=ckpt, seed=3, log=lambda s: None)


def test_resume_equals_uninterrupted(tmp_path):
    s1 = {"w": np.zeros(4), "m": np.zeros(4)}
    make(None, s1).run()
    s2 = {"w": np.zeros(4), "m": np.zeros(4)}
    ck = str(tmp_path / "ck.pt")
    t = make(ck, s2)
    t.run(stop_after_epoch=2)
    s3 = {"w": np.full(4, 99.0), "m": np.full(4, 99.0)}  # a fresh process: state comes from the checkpoint
    t2 = make(ck, s3)
    assert t2.resume() and t2.epoch == 2 and t2.step == 10
    hist = t2.run()
    assert len(hist) == 6
    np.testing.assert_array_equal(s3["w"], s1["w"])
    np.testing.assert_array_equal(s3["m"], s1["m"])


def test_cosine_schedule_endpoints():
    assert cosine_lr(0, 100, 1e-4, 1e-6) == 1e-4
    assert abs(cosine_lr(99, 100, 1e-4, 1e-6) - 1e-6) < 1e-18
    vals = [cosine_lr(s, 100, 1e-4, 1e-6) for s in range(100)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))
