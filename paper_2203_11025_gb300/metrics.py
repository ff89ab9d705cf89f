"""Solver metrics the paper reports (host side, from a solve's per-right-hand-side results).

Eq. 4.1 defines the convergence factor rho = (||r_T|| / ||r_0||)^(1/T) over T iterations;
with x0 = 0, ||r_0|| = ||b|| and ||r_T|| / ||r_0|| is the relative residual a solve
returns.  The paper's T is the number of iterations for a 10^6 reduction; a solve run to
another tolerance gives rho the same way, and the iterations for a 10^6 reduction follow
from it.  `JsonlLog` keeps a run's solve records (iterations, residuals, factors, time per
iteration) and training-epoch lines in a JSON-lines file.
"""
from __future__ import annotations

import math


def convergence_factor(relres: float, iters: int) -> float | None:
    """rho of one right-hand side (Eq. 4.1); None when no iteration ran or relres is not a
    positive finite number."""
    if iters <= 0 or not (relres > 0.0) or math.isinf(relres):
        return None
    return relres ** (1.0 / iters)


def iterations_for_reduction(rho: float, reduction: float = 1e6) -> int | None:
    """Iterations T with rho^T <= 1 / reduction (the paper's T for reduction = 10^6)."""
    if rho is None or not (0.0 < rho < 1.0):
        return None
    return math.ceil(math.log(reduction) / -math.log(rho) - 1e-12)


def summary(relres, iters) -> dict:
    """Worst (largest) and mean rho over the right-hand sides of one solve, and T for a 10^6
    reduction at the worst rho."""
    rhos = [r for r in (convergence_factor(a, b) for a, b in zip(relres, iters)) if r is not None]
    if not rhos:
        return {"rho_max": None, "rho_mean": None, "T_1e6": None}
    worst = max(rhos)
    return {"rho_max": worst, "rho_mean": sum(rhos) / len(rhos), "T_1e6": iterations_for_reduction(worst)}


def solve_record(label: str, info: dict, seconds: float | None = None) -> dict:
    """One JSON-ready record of a solve: per-right-hand-side iterations and relative
    residuals, Eq. 4.1 factors, and (given the wall time) time per iteration."""
    rec = {"kind": "solve", "label": label, "status": info.get("status"), "iters": list(info["iters"]),
           "relres": [float(r) for r in info["relres"]], **summary(info["relres"], info["iters"])}
    if info.get("fallbacks"):
        rec["fallbacks"] = info["fallbacks"]
    if seconds is not None:
        rec["seconds"] = seconds
        its = max(info["iters"]) if info["iters"] else 0
        rec["ms_per_iteration"] = 1e3 * seconds / its if its else None
    return rec


class JsonlLog:
    """Append-only JSON-lines log (one record per line, wall-clock stamped): solve records,
    training epochs (train.train's `log` callback takes `epoch`), anything JSON-serialisable."""

    def __init__(self, path: str):
        self.path = path

    def write(self, record: dict) -> None:
        import json
        import time
        with open(self.path, "a") as f:
            f.write(json.dumps({"t": time.time(), **record}) + "\n")

    def solve(self, label: str, info: dict, seconds: float | None = None) -> None:
        self.write(solve_record(label, info, seconds))

    def epoch(self, message: str) -> None:
        self.write({"kind": "train", "message": message})


def read_jsonl(path: str) -> list:
    import json
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]
