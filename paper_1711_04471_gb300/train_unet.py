"""Train the warm-start U-Net on pressure increments produced by the plain
solver, and compare the learned warm start with the plain one.

Training data (the recipe of the learned warm start): LES runs on the
256 x 256 x 128 workload grid (dx = 4 m, 20 % building cover) with other
building seeds than the evaluation runs, over the stage of the run that is
evaluated (steps 2-201; --start steps before the first pair, of which all
but the last are solved to a looser tolerance).  From each step the
solve's previous pressure p_prev, right-hand side b and converged pressure
p (relative residual 1e-6) give one pair on the grid coarsened by f:

    input   warm_start_features(p_prev, b)            (coarse residual and pressure)
    target  block mean of (p - p_prev) / s             (s from the same call)

The map from (b, p_prev) to p - p_prev = A^-1 (b - A p_prev) is linear and
commutes with translations and reflections in y (periodic) and with a sign
change, so each solved step also yields the pairs of its copies shifted by
multiples of f and mirrored (32 pairs per step at f = 16, formed from the
coarse tensors by augment), and any linear combination of pairs is a pair
(mixed_batch draws the training batches that way).
Everything runs through the C ABI (les_*, warm_start_*, unet_*); the samples
stay in device memory.

The committed weights come from 56 runs of base seed 5000 (k = 0..55; the
last one held out for validation), each 200 solved steps after one solved
start-up step: 11,000 training pairs, 352,000 with the shifted and
mirrored copies.  The runs used the previously committed weights (trained
the same way on 28 runs) as their warm start, which only shortens the
solves: every target is the solver's pressure at the 1e-6 residual.  One
call generates the pairs and trains (about 24 minutes of generation and 4
of training on one GB300; the pairs stay in device memory):

    python -m paper_1711_04471_gb300.train_unet --seeds 56 --base-seed 5000 --steps 200 --start 1 \
        --gen-weights previous_weights.npy --iters 150000 --out weights.npy
"""
from __future__ import annotations

import argparse
import math
import time

import numpy as np


def _block_mean(a, f):
    nz, ny, nx = a.shape
    return a.reshape(nz // f, f, ny // f, f, nx // f, f).mean(axis=(1, 3, 5))


def pair_from_step(p_prev, b, p_new, dx, f):
    """Coarse input (D/f, H/f, W/f, 2), target (D/f, H/f, W/f) and scale s of
    one solved step (CUDA float32 tensors, float), or None when the residual
    is 0.  p_prev, p_new: host float64 interiors; b: host float32 interior."""
    import torch

    from .les import warm_start_features
    x, s = warm_start_features(torch.from_numpy(np.ascontiguousarray(p_prev)).cuda(),
                               torch.from_numpy(np.ascontiguousarray(b)).cuda(), dx, f)
    if not s > 0:
        return None
    t = torch.from_numpy((_block_mean(p_new - p_prev, f) / s).astype(np.float32)).cuda()
    return x, t, s


def augment(X, T, S, mirror=True):
    """Copies shifted by every multiple of f in y and mirrored in y.  Such
    shifts and mirrors move whole f-blocks, so the copies' inputs and targets
    are the coarse tensors rolled and flipped."""
    import torch
    xs, ts = [], []
    for flip in ([False, True] if mirror else [False]):
        xf, tf = (X.flip(2), T.flip(2)) if flip else (X, T)
        for o in range(T.shape[2]):
            xs.append(torch.roll(xf, o, 2))
            ts.append(torch.roll(tf, o, 2))
    k = len(xs)
    return torch.cat(xs).contiguous(), torch.cat(ts).contiguous(), S.repeat(k)


def mixed_batch(X, T, S, idx_a, idx_b, gen):
    """Training batch of random linear combinations of solved pairs.

    With u = s x[..., 0] (the coarse residual times (f dx)^2) and v = s t
    (the coarse increment), alpha u_a + beta u_b and alpha v_a + beta v_b are
    again a residual and its increment (the map is linear); the pair is
    renormalised by s' = rms(u).  The pressure channel is taken from a
    third, unrelated sample: the increment is fixed by the residual alone,
    so the network must not learn to read it from the previous pressure."""
    import torch
    n = idx_a.numel()
    ab = torch.randn((2, n), generator=gen, device="cpu")
    ab[1] *= (torch.rand(n, generator=gen) < 0.5).float()   # half the batch: one pair, random sign and scale
    ab = ab.to(X.device)
    sa, sb = S[idx_a].view(n, 1, 1, 1), S[idx_b].view(n, 1, 1, 1)
    u = ab[0].view(n, 1, 1, 1) * sa * X[idx_a, ..., 0] + ab[1].view(n, 1, 1, 1) * sb * X[idx_b, ..., 0]
    v = ab[0].view(n, 1, 1, 1) * sa * T[idx_a] + ab[1].view(n, 1, 1, 1) * sb * T[idx_b]
    r = u.pow(2).mean(dim=(1, 2, 3), keepdim=True).sqrt().clamp_min(1e-30)
    idx_c = torch.randint(0, X.shape[0], (n,), generator=gen, device="cpu").to(X.device)
    x = torch.stack([u / r, X[idx_c, ..., 1]], dim=-1)
    return x.contiguous(), (v / r).contiguous()


def generate(nseeds=8, steps=32, start=17, shape=(256, 256, 128), dx=4.0, f=16, base_seed=2000, spinup_tol=1e-4,
             log=print, first_seed=0, net=None):
    """Per-seed (X, T, S) CUDA tensors of the solved steps, X (n, D/f, H/f,
    W/f, 2), T (n, D/f, H/f, W/f), S (n,) FP32 scales, for the building
    seeds derive_seed(base_seed, k), k = first_seed .. first_seed + nseeds - 1.
    The first start - 1 steps solve to spinup_tol (they only bring the flow
    to the stage that is evaluated), the next one to 1e-6 so that p_prev of
    the first pair is a converged pressure.  With net, the runs use it as
    their warm start: the solves reach the same 1e-6 residual sooner, and
    the target is still the solver's converged pressure."""
    import torch

    from . import inputs
    from .les import LES
    nx, ny, nz = shape
    out = []
    t0 = time.time()
    iters = []
    for sd in range(first_seed, first_seed + nseeds):
        solid = inputs.les_buildings(nx, ny, nz, dx=dx, seed=inputs.derive_seed(base_seed, sd))
        X, T, S = [], [], []
        with LES(nx, ny, nz, solid, dx=dx, check_every=50, max_iter=200000) as les:
            if net is not None:
                les.set_warm_start(net)
            if start > 1:
                les.set_solver(tol=spinup_tol)
                les.step(start - 1, stats=False)
                les.set_solver(tol=1e-6)
            if start > 0:
                les.step(1, stats=False)
            p_prev = les.get("p")[1:-1, 1:-1, 1:-1].copy()
            for _ in range(steps):
                st = les.step(1)[0]
                iters.append(st["iters"])
                b = les.get("b")[1:-1, 1:-1, 1:-1].copy()
                p_new = les.get("p")[1:-1, 1:-1, 1:-1].copy()
                pr = pair_from_step(p_prev, b, p_new, dx, f)
                if pr is not None:
                    X.append(pr[0])
                    T.append(pr[1])
                    S.append(pr[2])
                p_prev = p_new
        out.append((torch.stack(X), torch.stack(T), torch.tensor(S, dtype=torch.float32, device="cuda")))
        log(f"seed {sd}: {len(X)} steps, mean SOR iterations {np.mean(iters):.0f}, {time.time() - t0:.0f} s")
    return out


def slow_mode_error(y, t):
    """Median relative error of the amplitude of the slowest SOR mode
    (quarter cosine along x, constant in y and z) of prediction y vs target t,
    both (n, D, H, W) CUDA tensors."""
    import torch
    W = t.shape[-1]
    x = torch.arange(W, device=t.device, dtype=torch.float64) + 0.5
    phi = torch.cos(math.pi * x / (2 * W))
    a_t = (t.double().mean(dim=(1, 2)) * phi).sum(-1)
    a_y = (y.double().mean(dim=(1, 2)) * phi).sum(-1)
    return float(((a_y - a_t).abs() / a_t.abs().clamp_min(1e-30)).median())


def train(net, Xtr, Ttr, Str, Xval, Tval, iters=10000, batch=32, lr=1e-3, seed=0, log=print):
    """Adam with cosine decay on mixed minibatches (mixed_batch); returns a
    summary dict.  val_rel is the error energy relative to the zero
    increment (the plain warm start's coarse error) on held-out pairs."""
    import torch
    n = Xtr.shape[0]
    gen = torch.Generator().manual_seed(seed)

    def evaluate():
        ys = []
        for k in range(0, Xval.shape[0], batch):
            ys.append(net.forward(Xval[k:k + batch].contiguous()))
        y = torch.cat(ys)
        rel = float(((y - Tval) ** 2).sum() / (Tval ** 2).sum())
        return rel, slow_mode_error(y, Tval)

    hist = []
    t0 = time.time()
    for it in range(iters):
        ia = torch.randint(0, n, (batch,), generator=gen).to(Xtr.device)
        ib = torch.randint(0, n, (batch,), generator=gen).to(Xtr.device)
        x, t = mixed_batch(Xtr, Ttr, Str, ia, ib, gen)
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        hist.append(net.train_step(x, t, lr_t))
        if (it + 1) % max(1, iters // 10) == 0:
            rel, slow = evaluate()
            log(f"iter {it + 1}: train loss {np.mean(hist[-100:]):.4e}, val rel {rel:.4f}, "
                f"slow-mode err {slow:.4f}, {time.time() - t0:.0f} s")
    rel, slow = evaluate()
    return dict(train_loss=float(np.mean(hist[-100:])), val_rel=rel, val_slow_mode_err=slow,
                seconds=time.time() - t0, samples=int(n), val_samples=int(Xval.shape[0]), iters=iters, batch=batch)


def compare_warm_starts(net, shape=(256, 256, 128), seed=1003, spinup=20, steps=10, log=print, spinup_tol=None,
                        **les_kw):
    """Paired comparison on the same states: from each state of a plain run,
    one step with the previous-pressure warm start and one with the network,
    both to the same tolerance.  Returns per-step iterations and times.
    spinup_tol: tolerance of all spin-up steps but the last (None: the
    solver's own); the last one always solves to the solver's tolerance, so
    that the first compared step starts from a converged pressure."""
    from . import inputs
    from .les import LES
    nx, ny, nz = shape
    solid = inputs.les_buildings(nx, ny, nz, dx=4.0, seed=seed)
    rows = []
    with LES(nx, ny, nz, solid, **les_kw) as ref, LES(nx, ny, nz, solid, **les_kw) as trial:
        if spinup_tol is not None and spinup > 1:
            tol = ref.params.tol
            ref.set_solver(tol=spinup_tol)
            ref.step(spinup - 1, stats=False)
            ref.set_solver(tol=tol)
            ref.step(1, stats=False)
        else:
            ref.step(spinup, stats=False)
        trial.set_warm_start(net)
        for k in range(steps):
            state = ref.get_state()
            count = state["step"]
            trial.set_state(state)
            a = ref.step(1)[0]
            b = trial.step(1)[0]
            rows.append(dict(plain_iters=a["iters"], nn_iters=b["iters"],
                             plain_ms=a["ms_predictor"] + a["ms_solve"],
                             nn_ms=b["ms_predictor"] + b["ms_guess"] + b["ms_solve"], nn_guess_ms=b["ms_guess"],
                             plain_res=a["rel_res"], nn_res=b["rel_res"]))
            log(f"step {count}: plain {a['iters']} it {rows[-1]['plain_ms']:.0f} ms | "
                f"nn {b['iters']} it {rows[-1]['nn_ms']:.0f} ms (guess {b['ms_guess']:.2f} ms)")
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", type=int, default=8, help="LES runs (building seeds); the last one is held out")
    ap.add_argument("--steps", type=int, default=32, help="solved steps per run")
    ap.add_argument("--start", type=int, default=17, help="steps before the first pair")
    ap.add_argument("--factor", type=int, default=16)
    ap.add_argument("--data", nargs="+", help="load the solved pairs from these .npz files (in order; the last "
                                               "run of the last file is held out) instead of running the LES")
    ap.add_argument("--base-seed", type=int, default=2000, help="building seeds of the generated runs: "
                                                                 "derive_seed(base, k)")
    ap.add_argument("--first-seed", type=int, default=0, help="first k of the generated runs")
    ap.add_argument("--gen-weights", help="network weights used as the warm start while generating the runs")
    ap.add_argument("--save-data", help="write the solved pairs to this .npz")
    ap.add_argument("--iters", type=int, default=60000)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--compare-steps", type=int, default=0, help="paired evaluation steps after training")
    args = ap.parse_args()
    import torch

    from . import build
    build()
    from .unet import UNet
    if args.data:
        data = []
        for path in args.data:
            z = np.load(path)
            data += [tuple(torch.from_numpy(z[f"{a}{k}"]).cuda() for a in "xts") for k in range(int(z["nseeds"]))]
    else:
        gen_net = None
        if args.gen_weights:
            gen_net = UNet(seed=0)
            gen_net.set_params(np.load(args.gen_weights))
        data = generate(args.seeds, args.steps, start=args.start, f=args.factor, base_seed=args.base_seed,
                        first_seed=args.first_seed, net=gen_net)
        if gen_net is not None:
            gen_net.close()
    if args.save_data:
        arrs = {"nseeds": np.array(len(data))}
        for k, (x, t, s) in enumerate(data):
            arrs[f"x{k}"], arrs[f"t{k}"], arrs[f"s{k}"] = x.cpu().numpy(), t.cpu().numpy(), s.cpu().numpy()
        np.savez_compressed(args.save_data, **arrs)
        if args.iters == 0:
            return
    Xtr, Ttr, Str = augment(torch.cat([d[0] for d in data[:-1]]), torch.cat([d[1] for d in data[:-1]]),
                            torch.cat([d[2] for d in data[:-1]]))
    Xval, Tval, _ = data[-1]
    print(f"data: {tuple(Xtr.shape)} train (shifted and mirrored), {tuple(Xval.shape)} held out, "
          f"target rms {float(Ttr.pow(2).mean().sqrt()):.3e}", flush=True)
    with UNet(seed=args.init_seed) as net:
        summary = train(net, Xtr, Ttr, Str, Xval, Tval, iters=args.iters, batch=args.batch, lr=args.lr)
        print(summary, flush=True)
        np.save(args.out, net.get_params())
        if args.compare_steps:
            rows = compare_warm_starts(net, steps=args.compare_steps)
            pi = np.mean([r["plain_iters"] for r in rows])
            ni = np.mean([r["nn_iters"] for r in rows])
            print(f"paired: plain {pi:.0f} it, learned {ni:.0f} it", flush=True)


if __name__ == "__main__":
    main()
