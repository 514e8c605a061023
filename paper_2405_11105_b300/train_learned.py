"""Train the learned cutoff rule for a workload and save its parameters.

    python -m paper_2405_11105_b300.train_learned --packets 400 --out weights.npy

Packets come from the seeded synthetic generator (recipe drawn per packet:
vessel count, width, Doppler step, tissue-to-blood ratio, motion amplitude),
generated on the host cores in worker processes; every window of every packet
gives one (capped-sweep spectrum, converged method-1 cutoff) pair through the
library on the GPU (learned.collect), and the network trains on the GPU.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _gen(args):
    import synth
    recipe_name, seed = args
    return generate_one(getattr(synth, recipe_name), seed)


def generate_one(recipe, seed):
    from synth import generate_packet
    return generate_packet(recipe, seed=seed)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--recipe", default="LEARNED_384x256x128")
    ap.add_argument("--windows", type=int, nargs=2, default=[16, 16])
    ap.add_argument("--packets", type=int, default=400)
    ap.add_argument("--test-packets", type=int, default=8)
    ap.add_argument("--fast-sweeps", type=int, default=2)
    ap.add_argument("--hidden", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed0", type=int, default=10000)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)

    import synth
    recipe = getattr(synth, a.recipe)
    wz, wx = a.windows
    seeds = list(range(a.seed0, a.seed0 + a.packets))
    test_seeds = list(range(a.seed0 + 10 * a.packets, a.seed0 + 10 * a.packets + a.test_packets))
    workers = a.workers or max(1, (os.cpu_count() or 2) - 1)
    # the pool starts (spawn) before the first CUDA call of this process
    pool = mp.get_context("spawn").Pool(workers)
    jobs = pool.imap(_gen, [(a.recipe, s) for s in seeds + test_seeds], chunksize=1)

    import torch
    from paper_2405_11105_b300 import learned
    t0 = time.time()
    full, fast = learned.make_plans(recipe.nz, recipe.nx, recipe.nt, wz, wx, a.fast_sweeps)
    Xs, Ks, test = [], [], []
    for i, iq in enumerate(jobs):
        if i < len(seeds):
            X, K = learned.collect([iq], full, fast, wz, wx)
            Xs.append(X)
            Ks.append(K)
        else:
            test.append(iq)
    pool.close()
    X, K = np.concatenate(Xs), np.concatenate(Ks)
    t1 = time.time()
    losses = []
    net = learned.train(X, K, recipe.nt, hidden=a.hidden, epochs=a.epochs, batch=a.batch, lr=a.lr,
                        log=lambda e, l: losses.append(l))
    torch.cuda.synchronize()
    t2 = time.time()
    Xt, Kt = learned.collect(test, full, fast, wz, wx)
    acc, pred = learned.accuracy(net, Xt, Kt)
    np.save(a.out, net.params())
    meta = {"recipe": a.recipe, "windows": [wz, wx], "nt": recipe.nt, "hidden": a.hidden,
            "fast_sweeps": a.fast_sweeps, "train_subsets": int(X.shape[0]), "epochs": a.epochs,
            "final_loss": losses[-1], "heldout_subsets": int(Xt.shape[0]), "heldout_exact_acc": acc,
            "heldout_within1": float(np.mean(np.abs(pred - Kt) <= 1)),
            "data_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1)}
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))
    return 0


if __name__ == "__main__":
    sys.exit(main())
