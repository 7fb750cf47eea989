"""Train the warm-start U-Net on pressure increments produced by the plain
solver, and compare the learned warm start with the plain one.

Training data (the recipe of the learned warm start): LES runs on a
128 x 128 x 64 grid (dx = 4 m, the same physics and building statistics as
the 256 x 256 x 128 workload, other building seeds), each step's
right-hand side b, previous pressure p_prev and converged pressure p
(relative residual 1e-6), cut into 64^3 crops.  Input channels
[b dx^2 / s, p_prev / s], target (p - p_prev) / s, s = dx^2 rms(b) over the
crop.  Everything runs through the C ABI (les_*, unet_*); the samples stay
in device memory.

    python -m paper_1711_04471_gb300.train_unet --out weights.npy
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np


def generate(nseeds=16, steps=50, spinup=10, crops=6, shape=(128, 128, 64), crop=64, dx=4.0, base_seed=2000,
             log=print):
    """Return (X, T) CUDA tensors of shape (n, crop, crop, crop, 2) and (n, crop, crop, crop)."""
    import torch

    from . import inputs
    from .les import LES
    nx, ny, nz = shape
    X, T = [], []
    t0 = time.time()
    for sd in range(nseeds):
        solid = inputs.les_buildings(nx, ny, nz, dx=dx, seed=inputs.derive_seed(base_seed, sd))
        rng = inputs.SplitMix64(inputs.derive_seed(base_seed + 1, sd))
        with LES(nx, ny, nz, solid, check_every=50, max_iter=200000) as les:
            les.step(spinup, stats=False)
            for _ in range(steps):
                p_prev = les.get("p")[1:-1, 1:-1, 1:-1]
                les.step(1, stats=False)
                b = les.get("b")[1:-1, 1:-1, 1:-1].astype(np.float64)
                p = les.get("p")[1:-1, 1:-1, 1:-1]
                off = rng.uniform(3 * crops)
                for c in range(crops):
                    z0 = int(off[3 * c] * (nz - crop + 1))
                    y0 = int(off[3 * c + 1] * (ny - crop + 1))
                    x0 = int(off[3 * c + 2] * (nx - crop + 1))
                    sl = (slice(z0, z0 + crop), slice(y0, y0 + crop), slice(x0, x0 + crop))
                    bb, pp, pn = b[sl], p_prev[sl], p[sl]
                    s = dx * dx * math.sqrt(float(np.mean(bb * bb)))
                    if not s > 0:
                        continue
                    x = np.stack([bb * dx * dx / s, pp / s], axis=-1).astype(np.float32)
                    t = ((pn - pp) / s).astype(np.float32)
                    X.append(torch.from_numpy(x).cuda())
                    T.append(torch.from_numpy(t).cuda())
        log(f"seed {sd}: {len(X)} samples, {time.time() - t0:.0f} s")
    return torch.stack(X), torch.stack(T)


def train(net, X, T, iters=3000, batch=4, lr=1e-3, val_frac=0.05, seed=0, log=print):
    """Adam with cosine decay on random minibatches; returns a summary dict."""
    import torch
    n = X.shape[0]
    nval = max(1, int(n * val_frac))
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    val, tr = perm[:nval], perm[nval:]

    def val_loss():
        tot, base = 0.0, 0.0
        for k in range(0, nval, batch):
            idx = torch.as_tensor(val[k:k + batch], device=X.device)
            xb, tb = X[idx].contiguous(), T[idx].contiguous()
            y = net.forward(xb)
            tot += float(((y - tb) ** 2).sum())
            base += float((tb ** 2).sum())
        return tot / base   # relative to the zero-increment predictor (the plain warm start)

    hist = []
    t0 = time.time()
    for it in range(iters):
        idx = torch.as_tensor(rng.choice(tr, size=batch, replace=False), device=X.device)
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        loss = net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr_t)
        hist.append(loss)
        if (it + 1) % max(1, iters // 10) == 0:
            log(f"iter {it + 1}: train loss {np.mean(hist[-50:]):.4e}, val rel {val_loss():.4f}, "
                f"{time.time() - t0:.0f} s")
    return dict(train_loss=float(np.mean(hist[-50:])), val_rel=val_loss(), seconds=time.time() - t0,
                samples=int(n), iters=iters, batch=batch)


def compare_warm_starts(net, shape=(256, 256, 128), seed=1003, spinup=20, steps=10, log=print, **les_kw):
    """Paired comparison on the same states: from each state of a plain run,
    one step with the previous-pressure warm start and one with the network,
    both to the same tolerance.  Returns per-step iterations and times."""
    from . import inputs
    from .les import LES
    nx, ny, nz = shape
    solid = inputs.les_buildings(nx, ny, nz, dx=4.0, seed=seed)
    names = ("u", "v", "w", "p", "fuo", "fvo", "fwo", "gu", "gv", "gw")
    rows = []
    with LES(nx, ny, nz, solid, **les_kw) as ref, LES(nx, ny, nz, solid, **les_kw) as trial:
        ref.step(spinup, stats=False)
        trial.set_warm_start(net)
        for k in range(steps):
            state = {n: ref.get(n) for n in names}
            count = ref.step_count
            for n in names:
                trial.set(n, state[n])
            trial.step_count = count
            a = ref.step(1)[0]
            b = trial.step(1)[0]
            rows.append(dict(plain_iters=a["iters"], nn_iters=b["iters"],
                             plain_ms=a["ms_predictor"] + a["ms_solve"],
                             nn_ms=b["ms_predictor"] + b["ms_guess"] + b["ms_solve"], nn_guess_ms=b["ms_guess"],
                             plain_res=a["rel_res"], nn_res=b["rel_res"]))
            log(f"step {count}: plain {a['iters']} it {rows[-1]['plain_ms']:.0f} ms | "
                f"nn {b['iters']} it {rows[-1]['nn_ms']:.0f} ms (guess {b['ms_guess']:.1f} ms)")
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--crops", type=int, default=6)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--init-seed", type=int, default=0)
    args = ap.parse_args()
    from . import build
    build()
    from .unet import UNet
    X, T = generate(args.seeds, args.steps, crops=args.crops)
    print(f"data: {tuple(X.shape)} inputs, target rms {float(T.pow(2).mean().sqrt()):.3e}", flush=True)
    with UNet(seed=args.init_seed) as net:
        summary = train(net, X, T, iters=args.iters, batch=args.batch, lr=args.lr)
        print(summary, flush=True)
        np.save(args.out, net.get_params())


if __name__ == "__main__":
    main()
