"""Training of the learned Sinkhorn warm start on duals the method generates.

The network (dd_mlp_* in the C ABI) predicts, for a composite cell with a full
8 x 8 X block, the correction r of the cell's affine dual that initialises the
cell's Sinkhorn solve (DD_WARM_MLP). Its training data are produced by the
library itself: hybrid runs (Alg. 3) on seeded synthetic problems with
DD_FLAG_COLLECT, which records each cell's network inputs before its solve and
the converged dual (as r) after it. Training runs on the GPU through the
library's own forward / backward / Adam kernels; this module only orders the
calls (data collection, batch order, learning-rate schedule) and stores the
result.

    python -m paper_2405_09400_gb300.warmstart --out weights.npz

Parameters are stored as one flat float32 vector (the layout of dd_mlp_*),
weights rounded to BF16, with the training settings beside them.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import DD_FLAG_COLLECT, DD_MLP_NIN, DD_MLP_NHID, DD_MLP_NOUT, DD_MLP_NPARAMS, DD_WARM_PREV, MLP, DomDec

PKG = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(PKG, "weights", "warm_mlp_dd256.npz")
DIMS = (DD_MLP_NIN, DD_MLP_NHID, DD_MLP_NHID, DD_MLP_NHID, DD_MLP_NOUT)


def layer_slices():
    out, o = [], 0
    for l in range(len(DIMS) - 1):
        k, n = DIMS[l], DIMS[l + 1]
        out.append((slice(o, o + n * k), slice(o + n * k, o + n * k + n), n, k))
        o += n * k + n
    assert o == DD_MLP_NPARAMS
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights (SiLU), zero biases, a small last layer."""
    rng = np.random.default_rng(seed)
    p = np.zeros(DD_MLP_NPARAMS, dtype=np.float32)
    sl = layer_slices()
    for l, (ws, _, n, k) in enumerate(sl):
        std = math.sqrt(2.0 / k) * (0.1 if l == len(sl) - 1 else 1.0)
        p[ws] = rng.normal(0.0, std, n * k).astype(np.float32)
    return p


def round_bf16(p: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), kept as float32."""
    u = np.ascontiguousarray(p, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def save_params(path, params, meta):
    p = np.array(params, dtype=np.float32)
    for ws, _, _, _ in layer_slices():
        p[ws] = round_bf16(p[ws])
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.savez_compressed(path, params=p, meta=json.dumps(meta))


def load_params(path=WEIGHTS):
    with np.load(path) as z:
        return np.array(z["params"], dtype=np.float32), json.loads(str(z["meta"]))


def collect(seeds, iters, workload="dd256", tol=1e-5, max_iter=20000, log=None):
    """Hybrid runs from the KR coupling on each seed pair; every half-iteration's
    (inputs, targets) rows, on the device."""
    import torch

    import synth

    X, T = [], []
    for k in seeds:
        mu, nu, eps, p = synth.workload(workload, k)
        boxes = synth.boxes_from_coupling(mu.shape, p["s"], *synth.knothe_rosenblatt(mu, nu))
        g = DomDec(mu, nu, eps, p["s"], boxes=boxes, tol=tol, max_iter=max_iter, warm=DD_WARM_PREV,
                   flags=DD_FLAG_COLLECT)
        for _ in range(iters):
            for part in (0, 1):
                g.iterate(part)
                f, t = g.collect(part)
                X.append(f)
                T.append(t)
            g.flow_update()
        g.close()
        if log:
            log(f"collected seed {k}: {sum(x.shape[0] for x in X)} rows")
    return torch.cat(X), torch.cat(T)


def train(X, T, Xv=None, Tv=None, epochs=30, batch=4096, lr=2e-3, lr_end=2e-5, aux_weight=0.01, seed=0, log=None):
    """Adam on the weighted squared error (weight 1 on the 64 dual outputs,
    aux_weight on the 256 auxiliary ones), targets scaled per group to unit
    RMS during training; the scales are folded into the last layer."""
    import torch

    dev = X.device
    sa = float(T[:, :64].pow(2).mean().sqrt())
    sb = float(T[:, 64:].pow(2).mean().sqrt())
    scale = torch.ones(DD_MLP_NOUT, device=dev)
    scale[:64] = sa
    scale[64:] = sb
    Ts = (T / scale).contiguous()
    Tvs = (Tv / scale).contiguous() if Tv is not None else None
    w = torch.full((DD_MLP_NOUT,), aux_weight, dtype=torch.float32, device=dev)
    w[:64] = 1.0
    n = X.shape[0]
    batch = min(batch, n)
    net = MLP(batch)
    net.set_params(init_params(seed))
    steps_per = n // batch
    total = epochs * steps_per
    gen = torch.Generator().manual_seed(seed)
    hist = []
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(device=dev, dtype=torch.int32)
        tr = 0.0
        for b in range(steps_per):
            lr_t = lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * step / total))
            want = b == steps_per - 1
            l = net.train_step(X, Ts, perm[b * batch:(b + 1) * batch], w, lr_t, want_loss=want)
            if want:
                tr = l
            step += 1
        val = None
        if Xv is not None:
            val = evaluate(net, Xv, Tvs, batch)
        hist.append(dict(epoch=ep, train=tr, val=val, s=time.perf_counter() - t0))
        if log:
            log(f"epoch {ep}: train {tr:.5f} val {val} ({time.perf_counter() - t0:.1f} s)")
    p = net.get_params()
    net.close()
    ws, bs, _, _ = layer_slices()[-1]
    W4 = p[ws].reshape(DD_MLP_NOUT, DD_MLP_NHID)
    sc = scale.cpu().numpy().astype(np.float32)
    W4 *= sc[:, None]
    p[ws] = W4.reshape(-1)
    p[bs] *= sc
    return p, dict(history=hist, scale_alpha=sa, scale_aux=sb)


def evaluate(net, X, T, batch):
    """Fraction of the variance left unexplained, per output group (dual r,
    auxiliary), over all rows (forward passes only)."""
    se = [0.0, 0.0]
    for i in range(0, X.shape[0], batch):
        y = net.forward(X[i:i + batch])
        d = y - T[i:i + batch]
        se[0] += float((d[:, :64] ** 2).sum())
        se[1] += float((d[:, 64:] ** 2).sum())
    return [round(se[0] / float((T[:, :64] ** 2).sum()), 5), round(se[1] / float((T[:, 64:] ** 2).sum()), 5)]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--train-seeds", default="100-124")
    ap.add_argument("--val-seeds", default="125-126")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-7, help="cell tolerance of the data-generating runs")
    ap.add_argument("--aux-weight", type=float, default=0.01)
    a = ap.parse_args(argv)

    def rng(sp):
        lo, hi = (int(x) for x in sp.split("-"))
        return list(range(lo, hi + 1))

    def log(msg):
        print(msg, file=sys.stderr, flush=True)

    t0 = time.perf_counter()
    X, T = collect(rng(a.train_seeds), a.iters, tol=a.tol, log=log)
    Xv, Tv = collect(rng(a.val_seeds), a.iters, tol=a.tol, log=log)
    t_data = time.perf_counter() - t0
    p, info = train(X, T, Xv, Tv, epochs=a.epochs, batch=a.batch, lr=a.lr, aux_weight=a.aux_weight, seed=a.seed,
                    log=log)
    meta = dict(workload="dd256", train_seeds=a.train_seeds, val_seeds=a.val_seeds, iters=a.iters, tol=a.tol,
                rows=int(X.shape[0]), epochs=a.epochs, batch=a.batch, lr=a.lr, aux_weight=a.aux_weight,
                seed=a.seed, data_s=round(t_data, 2), **info)
    save_params(a.out, p, meta)
    log(f"saved {a.out}: {X.shape[0]} rows, data {t_data:.1f} s, final val (unexplained r, aux) "
        f"{info['history'][-1]['val']}")


if __name__ == "__main__":
    main()
