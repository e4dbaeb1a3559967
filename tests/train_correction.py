"""Train the learned correction for the trace workload and store its weights.

    python tests/train_correction.py [--out paper_1810_13132_gb300/weights/correction_trace.npz]

Training data: (features, exact cardinality) pairs that the CPU oracle
generates on trace-shaped traffic (Zipf 1.05, 10% in-slice repeats, k = 30,
g = 256, 31 slices; oracle/learned.py) at 1/16 and 1/32 of the trace's pairs,
hosts, top cardinality and pool -- the same load per register as the full
trace -- seeds 1000 and up.  Evaluation: held-out seeds 0..3 at 1/16.
Training runs on the GPU with the library's own kernels (vbdr_mlp_train).
The output holds the FP32 parameters, nmax (the largest plain estimate seen
in training; larger ones keep the plain estimate) and the evaluation summary.
This script lives with the tests because it runs the oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_1810_13132_gb300", "weights",
                                                  "correction_trace.npz"))
    ap.add_argument("--runs16", type=int, default=24)
    ap.add_argument("--runs32", type=int, default=16)
    ap.add_argument("--eval-runs", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--processes", type=int, default=max(1, min(16, os.cpu_count() or 1)))
    a = ap.parse_args()

    from oracle import learned
    t0 = time.time()
    parts = []
    if a.runs16:
        parts.append(learned.training_set(range(1000, 1000 + a.runs16), scale=16,
                                          processes=a.processes))
    if a.runs32:
        parts.append(learned.training_set(range(2000, 2000 + a.runs32), scale=32,
                                          processes=a.processes))
    X = np.concatenate([p[0] for p in parts])
    n_plain = np.concatenate([p[1] for p in parts])
    card = np.concatenate([p[2] for p in parts])
    Xe, pe, ce = learned.training_set(range(a.eval_runs), scale=16, processes=a.processes)
    t_data = time.time() - t0

    import torch
    from paper_1810_13132_gb300 import Mlp, live_features
    torch.cuda.set_device(0)
    perm = np.random.default_rng(0).permutation(card.size)
    Xd = torch.from_numpy(live_features(X[perm]).astype(np.float32)).to(torch.bfloat16).cuda()
    y = (np.log1p(card) - np.log1p(n_plain))[perm].astype(np.float32)
    yd = torch.from_numpy(y).cuda()
    m = Mlp(seed=11)
    t1 = time.time()
    losses = m.train(Xd, yd, epochs=a.epochs, batch=4096, lr=2e-3, weight_decay=1e-4)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    params, _ = m.get_params()
    nmax = float(n_plain.max())

    Xed = torch.from_numpy(live_features(Xe).astype(np.float32)).to(torch.bfloat16).cuda()
    delta = m.forward(Xed).cpu().numpy().astype(np.float64)
    corr = np.where(pe > nmax, pe, learned.correct(pe, delta))

    def stats(est):
        rel = np.abs(est - ce) / ce
        out = {"mre": float(rel.mean())}
        for name, mask in (("p99_card_lt_1e3", ce < 1e3), ("p99_card_gt_1e4", ce > 1e4)):
            if mask.any():
                out[name] = float(np.quantile(rel[mask], 0.99))
        return out

    summary = {"train_samples": int(card.size), "eval_samples": int(ce.size),
               "epochs": a.epochs, "final_loss": float(losses[-1]), "first_loss": float(losses[0]),
               "plain": stats(pe), "learned": stats(corr), "nmax": nmax,
               "data_s": round(t_data, 1), "train_s": round(t_train, 1),
               "scales": {"16": a.runs16, "32": a.runs32}}
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    np.savez(a.out, params=params.astype(np.float32), nmax=np.float32(nmax),
             summary=json.dumps(summary))
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
