"""Train the learned MV-proposal network on the GPU and evaluate the
learned-seeded search.

    python -m paper_2508_05990_b300.train_proposal [--epochs 100] [--pairs 2000] ...

Recipe: the paper's recipe for its own learned module (Sec. 4.1 "Training
Details": AdamW, cosine decay to 1e-6, batch 16, 100 epochs) with two changes
for a network trained from scratch rather than on top of a trained base model:
a starting learning rate of 1e-3 instead of 1e-4 (at 1e-4 the confidence head
never leaves "fall back everywhere" within 100 epochs), and a weight w on the
unreachable class of the confidence loss, so that a confidence >= 0.5 means
the +-4 refine reaches the exhaustive-search optimum with probability
>= w/(1+w).  Held-out results with 4000 training pairs: w = 10: 26.5 %
fallback, 0.21 % SAD regret; w = 5: 20.3 %, 0.53 %; w = 3: 17.6 %, 0.75 %
(w = 1 with 2000 pairs: 2.6 % regret).  Default: w = 5.  Data: 1080p synthetic clips (the scene generator of synth.py, seeds
10^6 + k for training and 2*10^6 + k for evaluation, 7 pairs per 8-frame clip);
labels are the exhaustive +-32 EVEN search of each pair, computed by the
library's own kernel.  Every forward, backward and optimizer step runs in the
library's kernels (bayer_cnn_loss_grad, bayer_cnn_adamw); this module only
schedules them.

Checkpoints (torch.save of plain tensors: float32 weights, AdamW moments,
step, epoch, permutation RNG state) are written after every epoch and resumed
from automatically.  The final weights are written as an .npz of the flat
float32 parameter vector.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

H, W, T = 1088, 1920, 8
BLOCK, RANGE = 16, 32
TRAIN_SEED, EVAL_SEED = 1_000_000, 2_000_000
DEFAULT_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "proposal_1080p_r32.npz")


def cosine_lr(step: int, total: int, lr0: float, lr_min: float) -> float:
    """Cosine decay from lr0 (step 0) to lr_min (last step)."""
    if total <= 1:
        return lr0
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * step / (total - 1)))


def _clip(seed):
    from paper_2508_05990_b300 import synth
    return synth.pan_clip(seed, H, W, n_frames=T)


def make_clips(base_seed: int, n_clips: int, workers: int) -> np.ndarray:
    """[n_clips, T, H, W] uint16, generated in a spawn-started process pool."""
    import multiprocessing as mp
    seeds = [base_seed + k for k in range(n_clips)]
    if workers <= 1:
        return np.stack([_clip(s) for s in seeds])
    with mp.get_context("spawn").Pool(workers) as pool:
        return np.stack(pool.map(_clip, seeds, chunksize=1))


class Trainer:
    """Epoch loop with checkpoint/resume.  ``step_fn(indices, lr, step) -> loss``
    performs one optimizer step on the given pair indices; ``get_state`` /
    ``set_state`` move the model and optimizer state to and from a dict of
    numpy arrays."""

    def __init__(self, n_items, batch, epochs, lr0, lr_min, step_fn, get_state, set_state, ckpt=None, seed=0,
                 log=print):
        self.n_items, self.batch, self.epochs = n_items, batch, epochs
        self.lr0, self.lr_min = lr0, lr_min
        self.step_fn, self.get_state, self.set_state = step_fn, get_state, set_state
        self.ckpt, self.log = ckpt, log
        self.steps_per_epoch = n_items // batch
        self.total = self.steps_per_epoch * epochs
        self.rng = np.random.default_rng(seed)
        self.step = 0
        self.epoch = 0
        self.history = []

    def save(self):
        if not self.ckpt:
            return
        import torch
        st = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in self.get_state().items()}
        st["step"] = torch.tensor(self.step)
        st["epoch"] = torch.tensor(self.epoch)
        st["rng"] = json.dumps(self.rng.bit_generator.state)
        st["history"] = json.dumps(self.history)
        tmp = self.ckpt + ".tmp"
        torch.save(st, tmp)
        os.replace(tmp, self.ckpt)

    def resume(self) -> bool:
        if not self.ckpt or not os.path.exists(self.ckpt):
            return False
        import torch
        st = torch.load(self.ckpt, weights_only=False)
        self.step = int(st.pop("step"))
        self.epoch = int(st.pop("epoch"))
        self.rng.bit_generator.state = json.loads(st.pop("rng"))
        self.history = json.loads(st.pop("history"))
        self.set_state({k: v.numpy() for k, v in st.items()})
        return True

    def run(self, stop_after_epoch=None):
        while self.epoch < self.epochs:
            perm = self.rng.permutation(self.n_items)
            t0 = time.perf_counter()
            losses = []
            for s in range(self.steps_per_epoch):
                idx = perm[s * self.batch:(s + 1) * self.batch]
                lr = cosine_lr(self.step, self.total, self.lr0, self.lr_min)
                self.step += 1
                losses.append(self.step_fn(idx, lr, self.step))
            self.epoch += 1
            rec = {"epoch": self.epoch, "loss": float(np.mean([float(l) for l in losses])),
                   "seconds": time.perf_counter() - t0}
            self.history.append(rec)
            self.log(json.dumps(rec))
            self.save()
            if stop_after_epoch is not None and self.epoch >= stop_after_epoch:
                break
        return self.history


def evaluate(handle, clips_d, labels_d, w_bf16, thresh=0.5, reps=20, n_pairs=None):
    """Learned-seeded vs exhaustive search on the first n_pairs pairs of the
    clips (all of them by default): fallback rate, SAD regret, and frames/s of
    both (7 pairs per launch)."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    n_clips = clips_d.shape[0]
    if n_pairs is None:
        n_pairs = n_clips * (T - 1)
    hb, wb = H // BLOCK, W // BLOCK
    out = torch.empty((T - 1, hb, wb, 2), dtype=torch.int32, device="cuda")
    fb = torch.empty((T - 1, hb, wb), dtype=torch.uint8, device="cuda")
    sad_full = sad_seed = 0
    n_fb = n_blk = 0
    rel_sum = 0.0
    kw = dict(batch=T - 1, ref_batch_stride=H * W, cur_batch_stride=H * W)
    for c in range(n_clips):
        k = min(T - 1, n_pairs - c * (T - 1))  # this clip's pairs that count
        if k <= 0:
            break
        d = clips_d[c]
        handle.estimate_learned(d, d[1:], w_bf16, RANGE, thresh, out=out, fallback=fb, **kw)
        full = labels_d[c]
        s_seed = bm.records_to_numpy(out[:k])["sad"].astype(np.int64)
        s_full = bm.records_to_numpy(full[:k])["sad"].astype(np.int64)
        sad_full += int(s_full.sum())
        sad_seed += int(s_seed.sum())
        rel_sum += float(((s_seed - s_full) / np.maximum(s_full, 1)).sum())
        n_fb += int(fb[:k].sum().item())
        n_blk += fb[:k].numel()
    # timing: one clip, both searches, CUDA events
    d = clips_d[0]
    full_out = torch.empty_like(out)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(3):
        handle.estimate_ex(d, d[1:], search_range=RANGE, out=full_out, **kw)
        handle.estimate_learned(d, d[1:], w_bf16, RANGE, thresh, out=out, **kw)
    torch.cuda.synchronize()
    ev[0].record()
    for _ in range(reps):
        handle.estimate_ex(d, d[1:], search_range=RANGE, out=full_out, **kw)
    ev[1].record()
    ev[2].record()
    for _ in range(reps):
        handle.estimate_learned(d, d[1:], w_bf16, RANGE, thresh, out=out, **kw)
    ev[3].record()
    torch.cuda.synchronize()
    ms_full = ev[0].elapsed_time(ev[1]) / reps
    ms_seed = ev[2].elapsed_time(ev[3]) / reps
    return {"pairs": min(n_pairs, n_clips * (T - 1)), "fallback_rate": n_fb / n_blk,
            "sad_regret": (sad_seed - sad_full) / sad_full, "mean_block_rel_regret": rel_sum / n_blk,
            "me_ms_per_7_pairs_full": ms_full, "me_ms_per_7_pairs_learned": ms_seed,
            "me_speedup": ms_full / ms_seed}


def label_clips(handle, clips_d):
    """Exhaustive +-32 EVEN search of every pair: [n_clips, 7, h, w, 2] int32."""
    import torch
    n = clips_d.shape[0]
    labels = torch.empty((n, T - 1, H // BLOCK, W // BLOCK, 2), dtype=torch.int32, device="cuda")
    for c in range(n):
        d = clips_d[c]
        handle.estimate_ex(d, d[1:], search_range=RANGE, batch=T - 1, ref_batch_stride=H * W, cur_batch_stride=H * W,
                           out=labels[c])
    return labels


def upload_and_label(handle, train_np, eval_np):
    """Frames to the GPU (int16 views of the 12-bit uint16 samples, bit-identical;
    torch indexes int16 on the GPU) and exhaustive-search labels for every pair."""
    import torch
    train_d = torch.from_numpy(train_np.view(np.int16)).cuda()
    eval_d = torch.from_numpy(eval_np.view(np.int16)).cuda()
    return train_d, eval_d, label_clips(handle, train_d), label_clips(handle, eval_d)


def train(handle, train_d, train_lab, n_items, epochs=100, batch=16, lr=1e-3, lr_min=1e-6, weight_decay=0.01,
          neg_weight=5.0, seed=7, ckpt=None, init_theta=None, log=print):
    """AdamW training of the proposal network on the library's kernels.
    Returns (float32 master weights, bf16 copy, Trainer)."""
    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import synth
    theta = init_theta if init_theta is not None else synth.he_normal_params(seed, bm.CNN_SHAPES)
    w = torch.from_numpy(np.asarray(theta, np.float32).copy()).cuda()
    wb = bm.to_bf16_bits(w).contiguous()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    grad = torch.empty_like(w)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    ref_b = torch.empty((batch, H, W), dtype=train_d.dtype, device="cuda")
    cur_b = torch.empty_like(ref_b)
    lab_b = torch.empty((batch, H // BLOCK, W // BLOCK, 2), dtype=torch.int32, device="cuda")

    def step_fn(idx, lr_now, step):
        ii = torch.from_numpy(np.asarray(idx, np.int64)).cuda()
        clip, t = ii // (T - 1), ii % (T - 1)
        ref_b.copy_(train_d[clip, t])
        cur_b.copy_(train_d[clip, t + 1])
        lab_b.copy_(train_lab[clip, t])
        handle.cnn_loss_grad(ref_b, cur_b, wb, lab_b, RANGE, batch=len(idx), ref_batch_stride=H * W,
                             cur_batch_stride=H * W, grad=grad, loss=loss, neg_weight=neg_weight)
        handle.cnn_adamw(w, wb, grad, m, v, step, lr_now, weight_decay=weight_decay)
        return loss

    def get_state():
        return {"w": w.cpu().numpy(), "m": m.cpu().numpy(), "v": v.cpu().numpy()}

    def set_state(st):
        w.copy_(torch.from_numpy(st["w"]))
        m.copy_(torch.from_numpy(st["m"]))
        v.copy_(torch.from_numpy(st["v"]))
        wb.copy_(bm.to_bf16_bits(w))

    tr = Trainer(n_items, batch, epochs, lr, lr_min, step_fn, get_state, set_state, ckpt=ckpt, seed=seed, log=log)
    tr.resumed = tr.resume()
    tr.run()
    torch.cuda.synchronize()
    return w, wb, tr


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--pairs", type=int, default=4000)
    ap.add_argument("--eval-pairs", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--lr-min", type=float, default=1e-6)
    ap.add_argument("--weight-decay", type=float, default=0.01)
    ap.add_argument("--neg-weight", type=float, default=5.0, help="BCE weight of the unreachable class")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--ckpt", default=None, help="checkpoint path (resumed if present)")
    ap.add_argument("--out", default=DEFAULT_WEIGHTS, help="final float32 weights (.npz)")
    ap.add_argument("--report", default=None, help="JSON report path")
    ap.add_argument("--init", default=None, help="start from these weights (.npz) instead of He-normal")
    args = ap.parse_args(argv)

    n_train_clips = -(-args.pairs // (T - 1))
    n_eval_clips = -(-args.eval_pairs // (T - 1))
    t0 = time.perf_counter()
    train_np = make_clips(TRAIN_SEED, n_train_clips, args.workers)  # before any CUDA call
    eval_np = make_clips(EVAL_SEED, n_eval_clips, args.workers)
    t_gen = time.perf_counter() - t0

    import torch
    from paper_2508_05990_b300 import bayer_me as bm
    from paper_2508_05990_b300 import build
    build.build()
    handle = bm.Handle(0)
    t1 = time.perf_counter()
    train_d, eval_d, train_lab, eval_lab = upload_and_label(handle, train_np, eval_np)
    del train_np, eval_np
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t1
    n_items = min(args.pairs, n_train_clips * (T - 1))
    init = np.load(args.init)["theta"].astype(np.float32) if args.init else None
    before = None
    if init is None:
        from paper_2508_05990_b300 import synth
        w0 = torch.from_numpy(synth.he_normal_params(args.seed, bm.CNN_SHAPES)).cuda()
        before = evaluate(handle, eval_d, eval_lab, bm.to_bf16_bits(w0).contiguous(), n_pairs=args.eval_pairs)
    t2 = time.perf_counter()
    w, wb, tr = train(handle, train_d, train_lab, n_items, args.epochs, args.batch, args.lr, args.lr_min,
                      args.weight_decay, args.neg_weight, args.seed, args.ckpt, init,
                      log=lambda s: print(s, flush=True))
    t_train = time.perf_counter() - t2
    after = evaluate(handle, eval_d, eval_lab, wb, n_pairs=args.eval_pairs)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, theta=w.cpu().numpy(), range=RANGE, block=BLOCK)
    report = {"train_pairs": n_items, "eval_pairs": after["pairs"], "epochs": args.epochs,
              "batch": args.batch, "lr": args.lr, "lr_min": args.lr_min, "weight_decay": args.weight_decay,
              "neg_weight": args.neg_weight, "seconds": {"generate": t_gen, "label": t_label, "train": t_train},
              "resumed": tr.resumed, "history": tr.history, "eval_untrained": before, "eval_trained": after,
              "weights": args.out}
    text = json.dumps(report, indent=1)
    print(text)
    if args.report:
        with open(args.report, "w") as f:
            f.write(text)
    handle.close()


if __name__ == "__main__":
    main()
