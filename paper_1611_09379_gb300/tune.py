"""Autotuner front end: the library's empirical parameter search
(nufft_autotune) plus a persistent table of its results.

The search itself runs in the library (timed through the exec calls, the
accuracy checked against the FP64 FMM at eps = 1e-15).  This module keys the
result by the problem class -- N, M, eps, precision, element type, batch,
the timed operations and a caller-supplied tag for the point distribution --
and keeps it in a JSON table, so a plan for the same class can be made with
the tuned parameters without searching again.

Table location: the ``path`` argument, else the environment variable
NUFFT_TUNE_CACHE; with neither, nothing is stored.
"""
from __future__ import annotations

import ctypes
import json
import os
import time

from . import (FP64, IO_C64, OP_ADJ, OP_FWD, OP_INV, Params, Plan, TuneTrial, _check, _dev_ptr,
               _lib, _P, _stream_handle, _torch)

ENV = "NUFFT_TUNE_CACHE"
_OPS = {"fwd": OP_FWD, "adj": OP_ADJ, "inv": OP_INV}


def ops_mask(ops) -> int:
    """'fwd+inv' / ('fwd', 'adj') / an int mask -> the NUFFT_OP_* mask."""
    if isinstance(ops, int):
        return ops
    if isinstance(ops, str):
        ops = ops.split("+")
    m = 0
    for o in ops:
        m |= _OPS[o]
    return m


def key(N: int, M: int, eps: float, prec: int, io: str, batch: int, ops, tag: str = "") -> str:
    return f"N={N} M={M} eps={eps:.3e} prec={prec} io={io} batch={batch} ops={ops_mask(ops)} tag={tag}"


def load_table(path: str | None = None) -> dict:
    path = path or os.environ.get(ENV)
    if not path or not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def save_table(table: dict, path: str | None = None) -> None:
    path = path or os.environ.get(ENV)
    if not path:
        return
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _pdict(p: Params) -> dict:
    return {"lmax": p.lmax, "p": p.p, "q": p.q, "batch": p.batch, "tc_level": p.tc_level,
            "tc_near": p.tc_near}


def autotune(N: int, y, eps: float, prec: int = FP64, io: str = "c128", batch: int = 1,
             ops="fwd", reps: int = 5, tag: str = "", path: str | None = None,
             use_table: bool = True, stream=None) -> dict:
    """Tuned parameters for the plan (N, y, eps, prec, io, batch) and the exec
    sequence ``ops``.  Returns {"params", "trials", "seconds", "key",
    "from_table"}; the table is consulted first and updated after a search."""
    torch = _torch()
    M = int(y.numel())
    k = key(N, M, eps, prec, io, batch, ops, tag)
    table = load_table(path) if use_table else {}
    if use_table and k in table:
        ent = dict(table[k])
        ent["from_table"] = True
        ent["key"] = k
        return ent
    flags = IO_C64 if io == "c64" else 0
    best = Params()
    cap = 64
    trials = (TuneTrial * cap)()
    n = ctypes.c_int(0)
    yp = _dev_ptr(y, torch.float64, M, "y")
    t0 = time.perf_counter()
    _check(_lib.nufft_autotune(N, M, yp, eps, prec, flags, batch, ops_mask(ops), reps,
                               ctypes.byref(best), trials, cap, ctypes.byref(n),
                               _stream_handle(stream)), "nufft_autotune")
    secs = time.perf_counter() - t0
    log = [{"params": _pdict(t.params), "ms": t.ms, "err": t.err, "accepted": bool(t.accepted)}
           for t in trials[:min(n.value, cap)]]
    ent = {"params": _pdict(best), "trials": log, "seconds": secs}
    if use_table:
        table = load_table(path)
        table[k] = ent
        save_table(table, path)
    ent = dict(ent)
    ent["from_table"] = False
    ent["key"] = k
    return ent


def tuned_plan(N: int, y, eps: float, prec: int = FP64, io: str = "c128", batch: int = 1,
               ops="fwd", tag: str = "", path: str | None = None, stream=None) -> Plan:
    """A plan made with the tuned parameters (searching first if the table
    has no entry for this problem class)."""
    ent = autotune(N, y, eps, prec=prec, io=io, batch=batch, ops=ops, tag=tag, path=path,
                   stream=stream)
    p = ent["params"]
    return Plan(N, y, eps=eps, prec=prec, io=io, inverse=bool(ops_mask(ops) & OP_INV),
                lmax=p["lmax"], p=p["p"], q=p["q"], batch=batch, tc_level=p["tc_level"],
                tc_near=p.get("tc_near", 0), stream=stream)
