"""Train the compact learned correction for the trace workload and store it.

    python tests/train_correction_compact.py [--out paper_1810_13132_gb300/weights/correction_compact_trace.npz]

The compact network (oracle/learned.py: ten inputs -- the counts of register
values 0..3 over g and the six noise and estimate inputs of the full feature
row -- two GELU layers of 16) runs inside the planned estimate's kernel.
Training data: the same oracle runs on trace-shaped traffic as
train_correction.py (Zipf 1.05, 10% in-slice repeats, k = 30, g = 256, at
1/16 and 1/32 of the trace, seeds 1000 and up; held-out seeds 0..3 at 1/16
for evaluation).  Training runs on the CPU in plain PyTorch (AdamW, mean
squared error of delta against ln(1 + c) - ln(1 + n_plain)); the evaluation
uses the FP64 reference network.  The output holds the FP32 parameters (the
layout of learned.C_SIZES), nmax (the largest plain estimate seen in
training; larger ones keep the plain estimate) and the evaluation summary.
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


def train(Xc: np.ndarray, y: np.ndarray, epochs: int, seed: int = 0) -> np.ndarray:
    """FP32 parameters of the compact network fitted to (Xc, y)."""
    import torch
    from oracle import learned
    torch.manual_seed(seed)
    H = learned.C_HID
    net = torch.nn.Sequential(torch.nn.Linear(learned.C_IN, H), torch.nn.GELU(approximate="tanh"),
                              torch.nn.Linear(H, H), torch.nn.GELU(approximate="tanh"),
                              torch.nn.Linear(H, 1))
    opt = torch.optim.AdamW(net.parameters(), lr=2e-3, weight_decay=1e-4)
    A = torch.from_numpy(Xc.astype(np.float32))
    t = torch.from_numpy(y.astype(np.float32))
    n = A.shape[0]
    for _ in range(epochs):
        perm = torch.randperm(n)
        for i in range(0, n, 4096):
            idx = perm[i:i + 4096]
            opt.zero_grad()
            loss = ((net(A[idx]).squeeze(1) - t[idx]) ** 2).mean()
            loss.backward()
            opt.step()
    l1, l2, l3 = net[0], net[2], net[4]
    parts = [l1.weight, l1.bias, l2.weight, l2.bias, l3.weight.reshape(-1), l3.bias]
    theta = np.concatenate([p.detach().numpy().reshape(-1) for p in parts]).astype(np.float32)
    assert theta.size == learned.C_N_PARAMS
    return theta


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_1810_13132_gb300", "weights",
                                                  "correction_compact_trace.npz"))
    ap.add_argument("--runs16", type=int, default=24)
    ap.add_argument("--runs32", type=int, default=16)
    ap.add_argument("--eval-runs", type=int, default=4)
    ap.add_argument("--epochs", type=int, default=20)
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

    y = np.log1p(card) - np.log1p(n_plain)
    t1 = time.time()
    theta = train(learned.compact_features(X), y, a.epochs)
    t_train = time.time() - t1
    nmax = float(n_plain.max())
    delta = learned.compact_forward(theta, learned.compact_features(Xe))
    corr = np.where(pe > nmax, pe, learned.correct(pe, delta))

    def stats(est):
        rel = np.abs(est - ce) / ce
        out = {"mre": float(rel.mean())}
        for name, mask in (("p99_card_lt_1e3", ce < 1e3), ("p99_card_gt_1e4", ce > 1e4)):
            if mask.any():
                out[name] = float(np.quantile(rel[mask], 0.99))
        return out

    summary = {"train_samples": int(card.size), "eval_samples": int(ce.size),
               "epochs": a.epochs, "plain": stats(pe), "compact": stats(corr), "nmax": nmax,
               "data_s": round(t_data, 1), "train_s": round(t_train, 1),
               "scales": {"16": a.runs16, "32": a.runs32}}
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    np.savez(a.out, params=theta, nmax=np.float32(nmax), summary=json.dumps(summary))
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
