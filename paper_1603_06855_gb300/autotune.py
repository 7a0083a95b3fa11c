"""Measured choice of the batch's concurrency: the number of designs evaluated at once (workers)
and the number of concurrent k groups inside each mixed-form design (kgroups).

For a batch signature (the GPU's name and SM count, the precision, and the multiset of (lattice, N,
k-points, bands) of the designs), tune() times one evaluation of the batch (set_designs, bands and
the all-band weighted gap_and_grad) for every candidate after one untimed pass, keeps the fastest,
and records all measurements in a JSON file (by default $PC_AUTOTUNE_RECORD, else
~/.cache/paper_1603_06855_gb300/autotune.json).  choose() returns the recorded choice, tuning first
when the signature has none."""
from __future__ import annotations

import hashlib
import json
import os
import time

CANDIDATES = ((1, 0), (2, 0), (4, 0), (8, 0), (4, 1), (8, 1), (16, 1))


def record_path() -> str:
    return os.environ.get("PC_AUTOTUNE_RECORD",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_1603_06855_gb300", "autotune.json"))


def signature(designs, precision: int, gpu: str, sms: int) -> str:
    items = sorted((w.lattice, (2 * w.M + 1) ** 3, int(len(w.Q)), int(w.nbands)) for w in designs)
    text = json.dumps({"gpu": gpu, "sms": sms, "precision": int(precision), "designs": items}, sort_keys=True)
    return hashlib.sha256(text.encode()).hexdigest()[:24]


def load_record(path: str | None = None) -> dict:
    path = path or record_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_record(rec: dict, path: str | None = None) -> None:
    path = path or record_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(rec, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(timings: dict) -> tuple[int, int]:
    """The candidate with the shortest time (ties: fewer workers, then fewer k groups)."""
    best = min(timings.items(), key=lambda kv: (kv[1], tuple(int(v) for v in kv[0].split(","))))
    w, g = (int(v) for v in best[0].split(","))
    return w, g


def tune(designs, precision: int, rhos, measure, gpu: str, sms: int, candidates=CANDIDATES,
         path: str | None = None) -> dict:
    """measure(designs, precision, rhos, workers, kgroups) -> seconds of one timed evaluation.
    Records {signature: {"choice": [w, g], "seconds": {"w,g": t}}} and returns that entry."""
    timings = {}
    for w, g in candidates:
        timings[f"{w},{g}"] = float(measure(designs, precision, rhos, w, g))
    w, g = pick(timings)
    rec = load_record(path)
    entry = {"choice": [w, g], "seconds": timings, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    rec[signature(designs, precision, gpu, sms)] = entry
    save_record(rec, path)
    return entry


def choose(designs, precision: int, rhos, measure, gpu: str, sms: int, path: str | None = None,
           candidates=CANDIDATES) -> tuple[int, int]:
    rec = load_record(path)
    entry = rec.get(signature(designs, precision, gpu, sms))
    if entry is None:
        entry = tune(designs, precision, rhos, measure, gpu, sms, candidates, path)
    return tuple(entry["choice"])


def measure_batch(designs, precision: int, rhos, workers: int, kgroups: int) -> float:
    """One untimed and one timed evaluation of the batch on the current CUDA device."""
    import torch

    from .solver import BatchSolver
    from . import binding as B
    bs = BatchSolver(designs, precision, workers=workers, kgroups=kgroups)
    wts = [torch.full((len(w.Q), w.nbands), 1.0 / (len(w.Q) * w.nbands), dtype=torch.float64) for w in designs]
    for i in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bs.set_designs(rhos)
        bs.bands()
        bs.gap_and_grad(mode=B.PC_GRAD_ALLBANDS, weights=wts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    bs.close()
    return dt
