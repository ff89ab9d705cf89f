"""Host-side solver metrics: the convergence factor of Eq. 4.1 and the iterations for a
10^6 reduction, against their definitions and the oracle's FGMRES history."""
import math

import numpy as np

from oracle import helmholtz as H
from paper_2203_11025_gb300 import metrics as M
from paper_2203_11025_gb300 import synth


def test_convergence_factor_closed_forms():
    assert M.convergence_factor(1e-6, 10) == 1e-6 ** 0.1
    assert abs(M.convergence_factor(0.5 ** 7, 7) - 0.5) < 1e-15
    assert M.convergence_factor(1e-7, 0) is None
    assert M.convergence_factor(float("nan"), 10) is None
    assert M.convergence_factor(0.0, 10) is None
    assert M.iterations_for_reduction(0.1) == 6          # 0.1^6 = 1e-6 exactly: six iterations
    assert M.iterations_for_reduction(0.5) == math.ceil(math.log2(1e6))
    assert M.iterations_for_reduction(1.0) is None and M.iterations_for_reduction(None) is None
    s = M.summary([1e-8, 1e-7, float("nan")], [20, 10, 5])
    assert s["rho_max"] == 1e-8 ** 0.05 and s["T_1e6"] == M.iterations_for_reduction(1e-8 ** 0.05)   # 20 its
    assert abs(s["rho_mean"] - (1e-8 ** 0.05 + 1e-7 ** 0.1) / 2) < 1e-15


def test_matches_the_oracle_solve():
    """rho from (relres, iters) equals the oracle's Eq. 4.1 on its own residual history, and
    T for 10^6 brackets the first history entry below 1e-6 of the start."""
    n = 32
    k2 = synth.grf_kappa2(n, n, 5, sigma=3.0).astype(np.float64)
    prob = H.Problem(k2, omega=synth.omega_for(n), h=1.0 / n, abc_width=8, levels=3)
    b = synth.complex_normal(6, (n, n))
    res = H.fgmres(prob.A, H.precond_v(prob), b, tol=1e-7, maxit=500)
    relres = res.true_history[-1] / res.true_history[0]
    rho = M.convergence_factor(relres, res.iters)
    assert abs(rho - H.convergence_factor(res.true_history[0], res.true_history[-1], res.iters)) < 1e-14
    assert 0.0 < rho < 1.0 and rho ** res.iters <= 1e-7 * (1 + 1e-9)
    assert M.iterations_for_reduction(rho) <= res.iters


def test_jsonl_log_round_trip(tmp_path):
    path = str(tmp_path / "run.jsonl")
    log = M.JsonlLog(path)
    info = {"status": 0, "iters": [35, 30], "relres": [9e-8, 8e-8], "fallbacks": 0}
    log.solve("M_VU", info, seconds=0.021)
    log.epoch("epoch 0 lr 1.00e-03 loss 12.5")
    recs = M.read_jsonl(path)
    assert [r["kind"] for r in recs] == ["solve", "train"]
    s = recs[0]
    assert s["label"] == "M_VU" and s["iters"] == [35, 30] and "fallbacks" not in s
    assert abs(s["rho_max"] - max(9e-8 ** (1 / 35), 8e-8 ** (1 / 30))) < 1e-15
    assert abs(s["ms_per_iteration"] - 21.0 / 35) < 1e-12 and s["t"] > 0
