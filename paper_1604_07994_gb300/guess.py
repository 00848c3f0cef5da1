"""Learned initial guess: training-set generation, training and evaluation (orchestration only).

Every numerical step runs in libsdx: the batched multigrid solves that produce the training
data (sdx_batch_solve), the feature and target maps (sdx_guess_features / sdx_guess_target),
the network's tensor-core forward and backward passes and Adam (sdx_net_train), and the
prediction (sdx_guess_predict).  This module only loops over instances and moves pointers.

The zero-guess multigrid stays the reference: a solve from the predicted iterate runs to the same
absolute residual ||b - K x|| <= rtol ||b|| as the solve from zero, so the network can only
save iterations, never accuracy.
"""
from __future__ import annotations

import time

import numpy as np

from . import sdx
from . import workloads as W


def training_set(count: int, n: int = 64, seed: int = 7000, batch: int = 48, rtol: float = 1e-8,
                 log10_contrast=(0.0, 4.0)):
    """`count` seeded instances at n^3 cells (1-4 boxes on the n/8 lattice, contrast
    log-uniform in 10^log10_contrast, Gaussian-blob forcing), solved by the batched FP32-refined
    multigrid to rtol.  Returns device tensors X [count, n^3, 16] (BF16) and T [count, n^3, 16]
    (FP32), and a dict of timings / iteration counts."""
    import torch
    X = torch.empty((count, n ** 3, 16), dtype=torch.bfloat16, device="cuda")
    T = torch.empty((count, n ** 3, 16), dtype=torch.float32, device="cuda")
    its, t_setup, t_solve = [], 0.0, 0.0
    for c0 in range(0, count, batch):
        ids = list(range(c0, min(count, c0 + batch)))
        probs = [W.random_instance(n, n // 8, seed + k, n // 8, log10_contrast=log10_contrast, forcing="blobs")
                 for k in ids]
        t0 = time.perf_counter()
        B = sdx.Batch(probs, prec=sdx.PREC_FP32_REFINED, coarse_form="sym", autotune=False)
        bs, xs, fss, hs = [], [], [], []
        for k, p in zip(ids, probs):
            H = B.instance(k - c0)
            f = torch.from_numpy(p.nodal_forcing().ravel()).cuda()
            b = torch.zeros(4 * p.nodes, dtype=torch.float64, device="cuda")
            H.sdx_rhs(f, b)
            fss.append(sdx.sdx_guess_features(H, f, X[k]))
            bs.append(b)
            xs.append(torch.zeros_like(b))
            hs.append(H)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st = B.sdx_batch_solve(bs, xs, rtol=rtol, maxit=400, restart=30)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        for k, H, x, fs in zip(ids, hs, xs, fss):
            sdx.sdx_guess_target(H, x, fs, T[k])
        torch.cuda.synchronize()
        its += [s["iterations"] for s in st]
        t_setup += t1 - t0
        t_solve += t2 - t1
        B.close()
    return X, T, {"instances": count, "n": n, "setup_s": t_setup, "solve_s": t_solve,
                  "iterations_mean": float(np.mean(its)), "iterations_max": int(np.max(its))}


def train(net, X, T, epochs: int = 20, batch: int = 8, lr: float = 2e-3, seed: int = 0):
    """Adam on mini-batches; returns the per-epoch mean loss and the wall time."""
    import torch
    count, V, _ = X.shape
    n = round(V ** (1.0 / 3.0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = net.train(n, count, X, T, epochs=epochs, batch=batch, lr=lr, seed=seed)
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def evaluate(net, problems, rtol: float = 1e-8, coarse_form="sym", prec=sdx.PREC_FP64, restart: int = 30,
             smooth_steps=(4,)):
    """Solve every problem from zero and from the network's guess (same absolute tolerance).
    The guess is refined by `s` Uzawa smoothing steps and a residual-minimising scaling
    (sdx_guess_refine) for every s in smooth_steps.  Returns per-instance iterations, times (a
    guess's time includes prediction and refinement) and the initial relative residuals."""
    import torch
    out = []
    for p in problems:
        H = sdx.Hierarchy.from_problem(p, form="tr", coarse_form=coarse_form, prec=prec)
        f = torch.from_numpy(p.nodal_forcing().ravel()).cuda()
        b = torch.zeros(4 * p.nodes, dtype=torch.float64, device="cuda")
        H.sdx_rhs(f, b)
        x = torch.zeros_like(b)
        H.sdx_solve(b, x, rtol=rtol, maxit=400, outer=sdx.OUTER_FGMRES, restart=restart)  # warm-up
        net.predict(H, f, x)
        torch.cuda.synchronize()
        res = {}
        xstar = None
        for mode in ["zero"] + [f"guess_s{k}" for k in smooth_steps]:
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            err0 = None
            if mode != "zero":
                net.predict(H, f, x)
                sdx.sdx_guess_refine(H, b, x, int(mode[len("guess_s"):]))
                torch.cuda.synchronize()
                t_pred = time.perf_counter() - t0
                d = x - xstar  # error of the start against the zero-start solution
                d[3 * p.nodes:] -= d[3 * p.nodes:].mean()
                err0 = float(d.norm() / xstar.norm())
                t0 = time.perf_counter() - t_pred
            st = H.sdx_solve(b, x, rtol=rtol, maxit=400, outer=sdx.OUTER_FGMRES, restart=restart)
            torch.cuda.synchronize()
            res[mode] = {"iterations": st["iterations"], "seconds": time.perf_counter() - t0,
                         "initial_rel_res": st["res0"] / st["bnorm"], "final_rel_res": st["res"] / st["bnorm"],
                         "initial_rel_error": 1.0 if mode == "zero" else err0}
            if mode == "zero":
                xstar = x.clone()
        out.append({"name": p.name, "n": p.n, "contrast": float(p.mu.max() / p.mu.min()), **res})
        H.close()
    return out
