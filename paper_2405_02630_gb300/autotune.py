"""Autotuner front end: picks the pipeline configuration of the pair kernels (sites
per chunk, stages in flight, and a whole or a quarter tile of pairs per CTA) per
(device, reps, precision, qubit-count bucket) and remembers it across processes.

The timing itself is native (qsvm_autotune in libqsvm times every configuration
with CUDA events on the caller's data); this module only keys, stores and
re-applies the winner.  The cache lives in $QSVM_AUTOTUNE_CACHE, else
$XDG_CACHE_HOME/qsvm_gb300/autotune.json, else ~/.cache/qsvm_gb300/autotune.json.
"""
from __future__ import annotations

import json
import os

from . import qsvm


def cache_path() -> str:
    p = os.environ.get("QSVM_AUTOTUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "qsvm_gb300", "autotune.json")


def n_bucket(n_qubits: int) -> int:
    """Qubit counts are bucketed by powers of two (the tile work scales with n)."""
    b = 1
    while b < n_qubits:
        b *= 2
    return b


def _key(reps: int, precision, n_qubits: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    prec = qsvm._prec(precision)
    return f"{p.name}|sm{p.multi_processor_count}|reps{reps}|prec{prec}|n{n_bucket(n_qubits)}"


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict):
    path = cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(mps, n_points: int, n_qubits: int, reps: int, precision, K, stream=None, save: bool = True) -> dict:
    """Times every configuration on this Gram (K is overwritten), selects the fastest."""
    best, ms = qsvm.qsvm_autotune(mps, n_points, n_qubits, reps, precision, K, stream=stream)
    rec = {"config": best, "ms": ms, "n_points": n_points,
           "shape": qsvm.qsvm_config_info(best, reps, precision),
           "cta": qsvm.qsvm_config_tile(best, reps, precision)}
    if save:
        d = _load()
        d[_key(reps, precision, n_qubits)] = rec
        _store(d)
    return rec


def apply_cached(reps: int, precision, n_qubits: int) -> int:
    """Selects the cached winner for this key, if any; returns it (or -1)."""
    rec = _load().get(_key(reps, precision, n_qubits))
    idx = int(rec["config"]) if rec else -1
    qsvm.qsvm_set_config(reps, precision, idx)
    return idx
