"""Learned warm start for the Newton-Krylov registration.

Pipeline (all compute on the GPU through the C ABI):
  1. seeded synthetic pairs (``synth.ellipses_pair``) at n x n;
  2. targets = the plain zero-start solver's converged velocities
     (H1, incompressible, beta_v = 1e-3, nt = 16, relative gradient 1e-2),
     computed with the batch executor (``reg_executor_solve``);
  3. training of the 8-layer convolutional network (``reg_net_train_step``,
     Adam, mini-batches) on (m_T, m_R) -> v;
  4. calibration of the output scale s (warm start s P G net(x)): the s with
     the fewest mean Hessian matvecs on validation pairs drawn from the
     training distribution (seeds disjoint from training and held-out pairs);
  5. evaluation on held-out pairs: the same solve from v_0 = 0 and from the
     scaled prediction (``opts.warm_start = 1``; the stopping test keeps
     g_ref = g(0), so both starts target the same absolute gradient).
The weights are saved as .npy with the calibrated scale in a .json beside them.

Usage (GPU):  python -m paper_1503_00757_gb300.warmstart --train 20000 --test 1000
              python -m paper_1503_00757_gb300.warmstart --eval-only --init weights.npy
"""
import argparse
import json
import math
import os
import time

import numpy as np

N_DEFAULT, NT, BETA, VMAX = 256, 16, 1e-3, 0.098
TRAIN_SEED, TEST_SEED = 5_000_000, 6_000_000
VAL_SEED = 5_500_000  # training distribution, disjoint from the training and held-out seeds


def make_images(n, seeds, vmax=VMAX, workers=1):
    """Image pairs (len(seeds), 2, n, n) of ``synth.ellipses_pair`` (workers > 1: spawned process pool)."""
    from . import synth
    seeds = list(seeds)
    x = np.empty((len(seeds), 2, n, n), dtype=np.float32)
    for i, (mT, mR) in enumerate(synth.ellipses_images([(n, s, vmax) for s in seeds], workers)):
        x[i, 0], x[i, 1] = mT, mR
    return x


def solve_all(images, executor, opts, v0=None, chunk=64):
    """Solve every pair (zero start, or warm start from v0); returns (v, stats, seconds)."""
    import torch
    n = images.shape[-1]
    B = images.shape[0]
    v_out = torch.empty((B, 2, n, n), dtype=torch.float32, device="cuda")
    stats = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(0, B, chunk):
        e = min(B, s + chunk)
        pairs = []
        for i in range(s, e):
            img = torch.from_numpy(images[i]).cuda()
            v = v_out[i]
            if v0 is not None:
                v.copy_(v0[i])
            pairs.append(dict(mT=img[0].contiguous(), mR=img[1].contiguous(), v=v, nt=NT, regnorm=1, beta=BETA,
                              gamma=math.inf, shear=0.0))
        _, st = executor.solve(pairs, opts, check=False)
        stats.extend(st)
    torch.cuda.synchronize()
    return v_out, stats, time.perf_counter() - t0


def train(net, images, targets, epochs, batch, lr, seed=0, log=None):
    import torch
    rng = np.random.default_rng(seed)
    B = images.shape[0]
    x_all = torch.from_numpy(images).cuda()
    losses = []
    for ep in range(epochs):
        perm = rng.permutation(B)
        tot = 0.0
        nb = 0
        for s in range(0, B - batch + 1, batch):
            idx = torch.from_numpy(perm[s:s + batch]).cuda()
            xb = x_all.index_select(0, idx).contiguous()
            tb = targets.index_select(0, idx).contiguous()
            tot += net.train_step(xb, tb, lr * (0.5 ** (ep // max(1, epochs // 3))))
            nb += 1
        losses.append(tot / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
    return losses


def predict(net, images, batch):
    import torch
    B, _, n, _ = images.shape
    out = torch.empty((B, 2, n, n), dtype=torch.float32, device="cuda")
    for s in range(0, B, batch):
        e = min(B, s + batch)
        xb = torch.from_numpy(images[s:e]).cuda().contiguous()
        net.forward(xb, out[s:e])
    torch.cuda.synchronize()
    return out


def summarize(stats, seconds):
    ok = [s for s in stats if s["rc"] == 0]
    return {"pairs": len(stats), "converged": len(ok),
            "newton_mean": float(np.mean([s["n_newton"] for s in stats])),
            "matvec_mean": float(np.mean([s["n_mv"] for s in stats])),
            "gnorm_rel_max": float(max(s["gnorm_rel"] for s in stats)),
            "seconds": seconds, "registrations_per_s": len(stats) / seconds}


CHANNELS = (2, 32, 32, 32, 32, 32, 32, 32, 2)


def he_init(seed, channels=CHANNELS):
    """Initial network parameters: W ~ N(0, 2 / (9 Cin)) per layer (He), b = 0, as a list of
    (W (Cout, Cin, 3, 3), b (Cout,)) in the layout reg_net_set_params flattens."""
    rng = np.random.default_rng(seed)
    return [(rng.standard_normal((cout, cin, 3, 3)) * np.sqrt(2.0 / (9.0 * cin)), np.zeros(cout))
            for cin, cout in zip(channels[:-1], channels[1:])]


def calibrate_scale(net, images, executor, scales, batch, log=None):
    """Output scale s of the warm start s P G net(x) with the fewest mean Hessian matvecs on
    the given (validation) pairs; ties go to the larger s.  Returns (s, table)."""
    from .binding import default_opts
    wopts = default_opts(tol=1e-2, maxit_newton=50, warm_start=1)
    table = {}
    for sc in scales:
        net.set_output_scale(sc)
        v0 = predict(net, images, batch)
        _, st, sec = solve_all(images, executor, wopts, v0=v0)
        table[sc] = summarize(st, sec)
        if log:
            log(f"scale {sc}: {table[sc]}")
    net.set_output_scale(1.0)
    best = min(sorted(table, reverse=True), key=lambda sc: table[sc]["matvec_mean"])
    return best, table


def main():
    import torch
    from .binding import Executor, Net, default_opts, flatten_params

    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--val", type=int, default=128, help="validation pairs (training distribution) for the scale")
    ap.add_argument("--test", type=int, default=1000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--scales", default="0.5,0.6,0.7,0.8,0.9,1.0")
    ap.add_argument("--init", default=None, help="initial parameters (.npy, flat FP32); default: He initialisation")
    ap.add_argument("--eval-only", action="store_true", help="no training: calibrate and evaluate --init")
    ap.add_argument("--out", default="warmstart.json")
    ap.add_argument("--weights", default="warmstart_weights.npy")
    args = ap.parse_args()
    log = lambda m: print(m, flush=True)
    n = args.n
    opts = default_opts(tol=1e-2, maxit_newton=50)
    ex = Executor(args.workers)
    t = time.perf_counter()
    nproc = max(1, min(16, os.cpu_count() or 1))
    x_te = make_images(n, range(TEST_SEED, TEST_SEED + args.test), workers=nproc)
    x_va = make_images(n, range(VAL_SEED, VAL_SEED + args.val), workers=nproc)
    net = Net(n, n, args.batch)
    if args.init:
        p0 = torch.from_numpy(np.load(args.init).astype(np.float32)).cuda()
    else:
        p0 = torch.tensor(flatten_params(he_init(1)), dtype=torch.float32, device="cuda")
    net.set_params(p0)
    res = {"n": n, "nt": NT, "beta_v": BETA, "test_pairs": args.test, "val_pairs": args.val}
    if not args.eval_only:
        x_tr = make_images(n, range(TRAIN_SEED, TRAIN_SEED + args.train), workers=nproc)
        log(f"images: {time.perf_counter() - t:.1f} s")
        v_tr, st_tr, sec_tr = solve_all(x_tr, ex, opts)
        log(f"targets: {sec_tr:.1f} s, {summarize(st_tr, sec_tr)}")
        keep = [i for i, s in enumerate(st_tr) if s["rc"] == 0]
        x_tr = x_tr[keep]
        v_tr = v_tr[torch.tensor(keep, device="cuda")].contiguous()
        t = time.perf_counter()
        losses = train(net, x_tr, v_tr, args.epochs, args.batch, args.lr, log=log)
        res.update({"train_pairs": len(keep), "epochs": args.epochs, "batch": args.batch,
                    "train_seconds": time.perf_counter() - t, "loss_first": losses[0], "loss_last": losses[-1]})
    # output scale on validation pairs, then zero vs warm start on the held-out pairs
    scales = [float(x) for x in args.scales.split(",")]
    best, table = calibrate_scale(net, x_va, ex, scales, args.batch, log=log)
    res["output_scale"] = best
    res["calibration"] = {str(k): v for k, v in table.items()}
    v_zero, st_zero, sec_zero = solve_all(x_te, ex, opts)
    res["zero_start"] = summarize(st_zero, sec_zero)
    wopts = default_opts(tol=1e-2, maxit_newton=50, warm_start=1)
    for key, sc in (("warm_start_unscaled", 1.0), ("warm_start", best)):
        net.set_output_scale(sc)
        torch.cuda.synchronize()
        t = time.perf_counter()
        v_pred = predict(net, x_te, args.batch)
        pred_s = time.perf_counter() - t
        _, st_warm, sec_warm = solve_all(x_te, ex, wopts, v0=v_pred)
        res[key] = summarize(st_warm, sec_warm + pred_s)
        res[key]["predict_seconds"] = pred_s
        res[key]["output_scale"] = sc
        if sc == 1.0:
            rel = ((v_pred - v_zero).flatten(1).norm(dim=1) / v_zero.flatten(1).norm(dim=1).clamp_min(1e-30))
            res["prediction_rel_error_mean"] = float(rel.mean())
    net.set_output_scale(1.0)
    log(json.dumps(res))
    os.makedirs(os.path.dirname(args.out) or ".", exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    p = torch.empty(net.nparams, device="cuda")
    net.get_params(p)
    np.save(args.weights, p.cpu().numpy())
    with open(os.path.splitext(args.weights)[0] + ".json", "w") as f:
        json.dump({"output_scale": best, "calibration": res["calibration"],
                   "validation_seeds": [VAL_SEED, VAL_SEED + args.val]}, f, indent=1)
    net.close()
    ex.close()


if __name__ == "__main__":
    main()
