"""Learned warm start for lid-driven cavities.

The steady lid-driven cavity of Sec. 4.3 is reached from rest after a long
transient.  This module trains the library's U-Net (WarmStartNet) to predict
the steady (P - P0, u, v) of a cavity from its Reynolds number, seeds the
MDF-LBM with f = f^eq(P, u) of the prediction (the initialisation rule of
Sec. 4 applied to a non-rest state), and lets the solver iterate to the
same residual as a start from rest.  Training data are steady fields the
batched solver itself produces.  Every numerical step runs in the library's
kernels; this module only moves arrays and sequences calls.

    python -m paper_2108_08591_gb300.warmstart [--side 256] [--n-train 256] [--n-test 64]
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from typing import List, Sequence, Tuple

import numpy as np

from . import CavityBatch, WarmStartNet

CIN, COUT = 16, 16  # padded input / output channels of the network
RE_SCALE = 1000.0


def input_planes(N: int, Re: float, U: float) -> np.ndarray:
    """Network input of one cavity, [N][N][CIN] float32 (row = y, column = x):
    Re / 1000, U / 0.1, x, y of the node centres (j + 1/2)/N, a lid-row
    indicator and a wall-adjacent indicator; the other channels are zero."""
    x = np.zeros((N, N, CIN), np.float32)
    c = (np.arange(N, dtype=np.float32) + 0.5) / N
    x[..., 0] = Re / RE_SCALE
    x[..., 1] = U / 0.1
    x[..., 2] = c[None, :]
    x[..., 3] = c[:, None]
    x[N - 1, :, 4] = 1.0
    x[0, :, 5] = x[N - 1, :, 5] = 1.0
    x[:, 0, 5] = x[:, N - 1, 5] = 1.0
    return x


def targets(P: np.ndarray, u: np.ndarray, N: int, U: float) -> np.ndarray:
    """[N][N][3] float32: (P - 1)/U^2, u/U, v/U."""
    t = np.empty((N, N, 3), np.float32)
    t[..., 0] = ((P - 1.0) / (U * U)).reshape(N, N)
    t[..., 1] = (u[0] / U).reshape(N, N)
    t[..., 2] = (u[1] / U).reshape(N, N)
    return t


def draw_cases(n: int, seed: int, re_range: Tuple[float, float]) -> List[float]:
    import synth
    rng = synth.SplitMix64(seed)
    return [re_range[0] + (re_range[1] - re_range[0]) * rng.uniform() for _ in range(n)]


def solve(N: int, Res: Sequence[float], U: float, tol: float, max_steps: int, check_every: int,
          seeds=None, stream=None, neq: bool = False):
    """Run cavities of side N to the residual `tol`; `seeds` (optional) is a
    list of (P, u) host arrays for a warm start, seeded as f^eq(P, u), plus
    the non-equilibrium part of grad u with `neq`.  Returns (batch, steps,
    status, residual, seconds) with the solve timed by CUDA events."""
    import torch
    if stream is None:
        stream = torch.cuda.Stream()
    b = CavityBatch([N] * len(Res), list(Res), lid_speed=U, stream=stream)
    if seeds is not None:
        for c, (P, u) in enumerate(seeds):
            b.init(c, P, u, neq=neq)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    steps, status, res = b.run(tol=tol, max_steps=max_steps, check_every=check_every)
    e1.record(stream)
    torch.cuda.synchronize()
    return b, steps, status, res, e0.elapsed_time(e1) / 1e3


def dataset(N: int, Res: Sequence[float], U: float, tol: float, max_steps: int, check_every: int):
    """Steady fields of the given cavities (converged ones only)."""
    b, steps, status, res, secs = solve(N, Res, U, tol, max_steps, check_every)
    X, T, kept = [], [], []
    for c, Re in enumerate(Res):
        if status[c] != 0:
            continue
        f = b.fields_host(c, ("P", "u"))
        X.append(input_planes(N, Re, U))
        T.append(targets(f["P"], f["u"], N, U))
        kept.append(c)
    b.close()
    return np.stack(X), np.stack(T), kept, steps, status, secs


def train(net: WarmStartNet, X, T, epochs: int, batch: int, lr: float, seed: int = 0,
          log_every: int = 0):
    """Adam on minibatches (SplitMix64 shuffles); X, T CUDA float32 tensors."""
    import synth
    import torch
    n = X.shape[0]
    rng = synth.SplitMix64(seed)
    losses = []
    step = 0
    total = epochs * max(1, n // batch)
    for ep in range(epochs):
        order = sorted(range(n), key=lambda _: rng.uniform())
        for k in range(0, n - batch + 1, batch):
            idx = torch.tensor(order[k:k + batch], device=X.device)
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))  # cosine decay
            want = log_every and (step % log_every == 0)
            loss = net.train_step(X.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous(),
                                  rate, want_loss=bool(want))
            if want:
                losses.append((step, loss))
            step += 1
    return losses


def predict(net: WarmStartNet, X, N: int, U: float):
    """Network prediction as solver seeds: list of (P [N^2], u [2][N^2])."""
    import torch
    out = []
    for k in range(0, X.shape[0], net.max_batch):
        y = net.forward(X[k:k + net.max_batch].contiguous())
        torch.cuda.synchronize()
        y = y[..., :3].double().cpu().numpy()
        for s in range(y.shape[0]):
            P = 1.0 + U * U * y[s, ..., 0].reshape(-1)
            u = np.stack([U * y[s, ..., 1].reshape(-1), U * y[s, ..., 2].reshape(-1)])
            out.append((np.ascontiguousarray(P), np.ascontiguousarray(u)))
    return out


def study(side: int, n_train: int, n_test: int, U: float, re_range, tol: float, max_steps: int,
          check_every: int, epochs: int, channels, batch: int, lr: float, seed: int = 2108):
    """Cold vs learned-warm time to steady state on held-out cavities."""
    import torch
    t0 = time.perf_counter()
    re_train = draw_cases(n_train, seed, re_range)
    re_test = draw_cases(n_test, seed + 1, re_range)
    Xtr, Ttr, kept, st_tr, stat_tr, gen_s = dataset(side, re_train, U, tol, max_steps, check_every)
    Xd, Td = torch.from_numpy(Xtr).cuda(), torch.from_numpy(Ttr).cuda()
    net = WarmStartNet(side, side, channels, cin=CIN, cout=COUT, cout_used=3, max_batch=batch, seed=seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter()
    losses = train(net, Xd, Td, epochs, batch, lr, seed=seed, log_every=50)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t_train
    # held-out: cold start, then warm start from the prediction
    Xte = torch.from_numpy(np.stack([input_planes(side, Re, U) for Re in re_test])).cuda()
    torch.cuda.synchronize()
    t_inf = time.perf_counter()
    seeds = predict(net, Xte, side, U)
    infer_s = time.perf_counter() - t_inf
    bc, st_c, stat_c, _, cold_s = solve(side, re_test, U, tol, max_steps, check_every)
    bw, st_w, stat_w, _, warm_s = solve(side, re_test, U, tol, max_steps, check_every, seeds=seeds)
    bn, st_n, stat_n, _, warm_ne_s = solve(side, re_test, U, tol, max_steps, check_every, seeds=seeds,
                                           neq=True)
    bn.close()
    both = [c for c in range(n_test) if stat_c[c] == 0 and stat_w[c] == 0]
    all3 = [c for c in both if stat_n[c] == 0]
    err_final, err_pred = [], []
    for c in both:
        fc = bc.fields_host(c, ("P", "u"))
        fw = bw.fields_host(c, ("P", "u"))
        err_final.append(np.linalg.norm(fw["u"] - fc["u"]) / np.linalg.norm(fc["u"]))
        err_pred.append(np.linalg.norm(seeds[c][1] - fc["u"]) / np.linalg.norm(fc["u"]))
    bc.close()
    bw.close()
    net.close()
    return {
        "side": side, "lid_speed": U, "re_range": list(re_range), "tol": tol,
        "n_train_drawn": n_train, "n_train_converged": len(kept), "n_test": n_test,
        "n_test_converged_both": len(both), "datagen_s": gen_s, "train_s": train_s,
        "epochs": epochs, "final_loss": losses[-1][1] if losses else None,
        "loss_curve": losses[:: max(1, len(losses) // 10)],
        "cold_steps_mean": float(np.mean([st_c[c] for c in both])) if both else None,
        "warm_steps_mean": float(np.mean([st_w[c] for c in both])) if both else None,
        "cold_s": cold_s, "warm_s": warm_s + infer_s, "infer_s": infer_s,
        "warm_neq_steps_mean": float(np.mean([st_n[c] for c in all3])) if all3 else None,
        "warm_neq_s": warm_ne_s + infer_s, "n_test_converged_neq": len(all3),
        "speedup_time": cold_s / (warm_s + infer_s),
        "speedup_steps": (float(np.mean([st_c[c] for c in both])) / float(np.mean([st_w[c] for c in both])))
        if both else None,
        "pred_err_u_mean": float(np.mean(err_pred)) if err_pred else None,
        "final_warm_vs_cold_u_max": float(np.max(err_final)) if err_final else None,
        "wall_s": time.perf_counter() - t0,
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=256)
    ap.add_argument("--n-train", type=int, default=256)
    ap.add_argument("--n-test", type=int, default=64)
    ap.add_argument("--lid", type=float, default=0.1)
    ap.add_argument("--re-min", type=float, default=100.0)
    ap.add_argument("--re-max", type=float, default=1000.0)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-steps", type=int, default=2_000_000)
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--channels", type=str, default="32,64,128,256")
    args = ap.parse_args(argv)
    r = study(args.side, args.n_train, args.n_test, args.lid, (args.re_min, args.re_max), args.tol,
              args.max_steps, args.check_every, args.epochs,
              tuple(int(c) for c in args.channels.split(",")), args.batch, args.lr)
    print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
