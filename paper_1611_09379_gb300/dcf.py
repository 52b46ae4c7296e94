"""Learned density compensation for the least-squares INUFFT (M > N).

The weights w_j of the weighted normal equations A^H W A c = A^H W g make
A^H W A close to the identity, so CG needs fewer iterations.  A small network
(``MLP``: 8 log neighbour spacings -> 64 -> 64 -> 1) predicts them per point;
it is trained on the GPU with the library's own forward/backward kernels on
weights computed for generated point sets by the fixed-point solver of
``dcf_targets`` (the Frobenius-optimal equations sum_j |D_N(y_i-y_j)|^2 w_j = N,
solved with positive weights).  Features are scale free, so a network trained
at small N, M serves any N, M with the same oversampling and distribution.
"""
from __future__ import annotations

import os

import numpy as np

from . import MLP, dcf_features_sorted, dcf_targets

WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dcf_mlp.f32")


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal hidden weights, zero biases, output bias with softplus(b3) = 1."""
    rng = np.random.Generator(np.random.Philox(seed))
    W1 = rng.standard_normal((64, 8)) * np.sqrt(2.0 / 8)
    W2 = rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    W3 = rng.standard_normal(64) * np.sqrt(1.0 / 64)
    b3 = np.log(np.e - 1.0)
    return np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), W3, [b3]]).astype(np.float32)


def training_data(point_sets: np.ndarray, N: int, iters: int = 100):
    """(features float32 [S*M, 8], targets float32 [S*M]) on the GPU for S point
    sets [S, M] in [0, 2 pi)."""
    import torch
    y = torch.from_numpy(np.sort(np.asarray(point_sets, np.float64), axis=1)).cuda()
    return dcf_features_sorted(y), dcf_targets(y, N, iters)


def train(feat, target, epochs: int = 40, lr: float = 3e-3, batch: int = 32768, seed: int = 0,
          params=None):
    """Train a fresh network (or continue from ``params``) with Adam; returns
    (mlp, per-epoch mean losses)."""
    import torch
    mlp = MLP(init_params(seed) if params is None else params)
    n = feat.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        tot, cnt = 0.0, 0
        for a in range(0, n, batch):
            idx = perm[a:a + batch]
            lr_ep = lr * (0.5 * (1 + np.cos(np.pi * ep / epochs)))  # cosine decay
            loss = mlp.train_step(feat[idx].contiguous(), target[idx].contiguous(), float(lr_ep),
                                  want_loss=True)
            tot += loss * idx.numel()
            cnt += idx.numel()
        losses.append(tot / cnt)
    return mlp, losses


def weights(plan, mlp):
    """Learned weights of a plan's points, mean 1, float32 CUDA tensor [M]
    (original order); features, inference and scaling run in the library."""
    return plan.dcf_weights(mlp)


def save(mlp, path: str = WEIGHTS_PATH):
    mlp.get_params().astype("<f4").tofile(path)


def load(path: str = WEIGHTS_PATH):
    return MLP(np.fromfile(path, dtype="<f4"))


def main(argv=None):
    """Train the shipped network: 10k point sets of the 1:100 contrast family
    at N = 256, M = 1024 (drawn with the repository's seeded generator module
    ``workloads``), targets from 100 fixed-point steps, 40 epochs of Adam;
    weights written to WEIGHTS_PATH."""
    import argparse
    import sys
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads
    sets = np.stack([workloads.points("contrast", 1024, seed=1000 + i) for i in range(a.sets)])
    feat, target = training_data(sets, 256)
    mlp, losses = train(feat, target, epochs=a.epochs)
    save(mlp, a.out)
    print("losses", [round(x, 4) for x in losses])


if __name__ == "__main__":
    main()
