"""Threshold ("machine precision") error eps_th(N) of the straightforward
method, the paper's experiment of Sec. 3.1: g = K f with the matrix K of
Eq. p4 evaluated in plain binary64, for f = 1 (exact answer g = 1), on M = N
uniform random points; eps(N) = max_j |g_j - 1|.  A second column compares
the straightforward method with the compensated oracle for random real
f_k in [0, 1] (the paper's second check).  Then a least-squares line
log2 eps_th = a + b log2 N, and the truncation numbers Eq. 18.2 gives at
eps = eps_th(N) with l_max = max(2, log2 N - 5) (Sec. 3.2, Fig. comp6's
p_th, q_th).

Test infrastructure: calls only the oracle; writes
tests/golden/eps_threshold_straightforward.txt.  Run:
    python -m oracle.eps_threshold [--lmax-log2 20] [--targets 1024]
"""
from __future__ import annotations

import argparse
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(ROOT, "tests", "golden", "eps_threshold_straightforward.txt")


def truncation_numbers(eps: float, L: int):
    """(l_max, p, q) of Eq. 18.2 (fraction 10/(3 pi eps), reading c5) at the
    paper's depth l_max = max(2, L - 5)."""
    lmax = max(2, L - 5)
    r = 10.0 / (3.0 * math.pi * eps)
    q = max(2, math.ceil(0.5 * math.log2(r)))
    p = max(4, math.ceil(1.0 + math.log(r) / math.log(3.0) + lmax / math.log2(3.0)))
    return lmax, p, q


def measure(L: int, targets: int):
    sys.path.insert(0, ROOT)
    import oracle
    import workloads
    N = 1 << L
    y = workloads.points("uniform", N, seed=500 + L)
    idx = workloads.sample_index(N, targets, seed=L)
    g1 = oracle.kernel_fwd_plain(np.ones(N, complex), y, idx)
    e1 = float(np.abs(g1 - 1.0).max())
    f = workloads.rng(600 + L).random(N).astype(complex)
    gp = oracle.kernel_fwd_plain(f, y, idx)
    gc = oracle.kernel_fwd(f, y, idx)
    er = float(np.abs(gp - gc).max())
    return N, idx.size, e1, er


def fit(rows, lo: int = 6):
    L = np.array([math.log2(r[0]) for r in rows if r[0] >= (1 << lo)])
    e = np.array([math.log2(r[2]) for r in rows if r[0] >= (1 << lo)])
    b, a = np.polyfit(L, e, 1)
    return float(a), float(b)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--lmax-log2", type=int, default=20)
    ap.add_argument("--targets", type=int, default=1024)
    args = ap.parse_args(argv)
    rows = [measure(L, args.targets) for L in range(3, args.lmax_log2 + 1)]
    a, b = fit(rows)
    lines = [
        "# Threshold error of the straightforward method (Sec. 3.1): K of Eq. p4 in plain",
        "# binary64 times f = 1 on M = N uniform points (seed 500 + log2 N), max over the",
        "# sampled targets (all when N <= targets); err_rand = max |plain - compensated| for",
        "# random real f in [0, 1].  Written by oracle/eps_threshold.py.",
        f"# fit log2 eps_th = a + b log2 N over N >= 64: a = {a:.6f} b = {b:.6f}",
        "# p_th, q_th: Eq. 18.2 at eps = fitted eps_th(N), l_max = max(2, log2 N - 5)",
        "# N targets eps_f1 err_rand eps_th_fit lmax p_th q_th",
    ]
    for N, nt, e1, er in rows:
        L = int(math.log2(N))
        eth = 2.0 ** (a + b * L)
        lmax, p, q = truncation_numbers(eth, L)
        lines.append(f"{N} {nt} {e1:.6e} {er:.6e} {eth:.6e} {lmax} {p} {q}")
    with open(OUT, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
