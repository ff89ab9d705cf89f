"""Benchmark: seconds for FGMRES(10) to reach an FP64-verified relative residual of 1e-7 with
the U-Net + shifted-Laplacian preconditioner (M_VU, Eq. 3.4), against plain SL (M_V) on the
same GPU and inputs: 2048 x 2048 grid, 16 point sources, one Gaussian-random-field medium,
the network mini-retrained on that medium (Sec. 3.5).

Metric (one JSON line, rank 0): value = seconds per M_VU solve of the 16 right-hand sides.
The same line reports M_V's solve time with the same number of timed steps, FGMRES
iterations, convergence factors (Eq. 4.1), the 1024^2 x 16 and 256^2 x 8 cases (fewer timed
steps each), the tensor roofline of the U-Net convolutions and the HBM roofline of the
stencil and Arnoldi kernels, end-to-end time through the C ABI with host buffers, and the
FP64 CPU oracle on a bounded sample.

Networks (outside every timed region; time reported separately): a base network trained
on Eq. 3.8-3.9 pairs of one random 256^2 medium (not a benchmark medium), saved with
unet_save, then for each case loaded with unet_load and mini-retrained on pairs of that
case's medium (Sec. 3.5) -- the medium the case then solves on.  The general network of
Sec. 3.4.1 (pairs of 16 random media) is trained too and reported on a medium it never saw;
with this training budget (1024 pairs; the paper used 20k) it transfers worse than the
single-medium base, so the base of the mini-retrained networks is the latter.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--grid n --nrhs k] [--no-extras] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle (numpy) on the host cores on a bounded sample of
the same workload: per step one FGMRES iteration with M_V on one right-hand side, scaled
by the iteration count and the right-hand sides of the GPU's M_V solve of this problem.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 2048
NRHS = 16
TOL = 1e-7
RESTART = 10
METRIC = "s to FP64 rel-res 1e-7 & FGMRES iters, U-Net+SL vs plain SL on 1 GB300; HBM %"
EXTRAS = ((1024, 16), (256, 8))   # reported in config, fewer timed steps
EXTRA_STEPS = 3
E2E_STEPS = 2
# base network: TRAIN_PAIRS Eq. 3.8-3.9 pairs of one random 256^2 medium (seed BASE_SEED)
BASE_GRID = 256
BASE_SEED = 10 ** 6 + 500
TRAIN_PAIRS = 1024
TRAIN_EPOCHS = 96
TRAIN_LR = 1e-3          # constant; measured fastest at this size (3e-3 stalls; Sec. 4 starts at 1e-4)
TRAIN_BATCH = 16
# general network: Eq. 3.8-3.9 pairs of TRAIN_MEDIA random 256^2 media (seeds 10^6 + k)
TRAIN_MEDIA = 16
TRAIN_PAIRS_PER_MEDIUM = 64
# mini-retraining on the case's medium (Sec. 3.5: a few hundred pairs, a few hundred steps)
RETRAIN_PAIRS = 300
RETRAIN_EPOCHS = 20
RETRAIN_LR = 5e-4
# encoder-solver case (Sec. 3.3): 512^2, 16 point sources + 16 complex Gaussian right-hand
# sides; the pair trained jointly on ES_PAIRS pairs of the case's medium
ES_GRID = 512
ES_POINTS = 16
ES_GAUSS = 16
ES_PAIRS = 512
ES_EPOCHS = 40
# M_V iterations of the GPU solve of the default problem (2048^2, 16 point sources, medium
# seed 1000, FP32 Krylov vectors): the reference arm scales its per-iteration sample by it
M_V_ITERS_DEFAULT = 4664
# DRAM bytes (read + write) of the 20 tensor-core convolution launches of one U-Net forward on
# 4 x 1024^2 pixels (ncu dram__bytes_read.sum + dram__bytes_write.sum: 1.190 GB), per level-0
# pixel; scaled by pixels to a forward of the benchmark's chunk
CONV_DRAM_BYTES_PER_PIXEL = 1189817344 / (4 * 1024 * 1024)


def workload(n: int, nrhs: int) -> str:
    return (f"{n}x{n} grid, h=1/{n}, omega=0.2*pi*{n}, GRF medium (sigma 8, kappa in [0.25,1]), 16-cell "
            f"quadratic absorbing layer, {nrhs} random point sources; FGMRES({RESTART}) + M_VU (U-Net 4 levels "
            f"32..256 ch, BF16 tcgen05 convs, then SL V-cycle 3 levels V(1,1) w=0.8, coarse GMRES(10)), tol {TOL}; "
            f"network trained {TRAIN_EPOCHS} epochs on {TRAIN_PAIRS} pairs of one random {BASE_GRID}x{BASE_GRID} "
            f"medium, mini-retrained {RETRAIN_EPOCHS} epochs on {RETRAIN_PAIRS} pairs of the benchmark medium")


def max_batch(n: int, want: int) -> int:
    """Largest power-of-two batch <= want within the U-Net's limit B*n*n*64 < 2^31."""
    bs = want
    while bs > 1 and bs * n * n * 64 >= 1 << 31:
        bs //= 2
    return bs


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (the job's wall time when
    every rank solves its own problem: replicas, no data exchange); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def build_problem(rank: int, n: int = None, nrhs: int = None):
    import numpy as np
    from paper_2203_11025_gb300 import synth
    n = N_GRID if n is None else n
    nrhs = NRHS if nrhs is None else nrhs
    k2 = synth.grf_kappa2(n, n, synth.medium_seed(rank))
    pos = synth.source_positions(n, n, nrhs, synth.rhs_seed(rank), 16)
    b = synth.point_sources(n, n, pos, 1.0 / n)
    return k2, b.astype(np.complex128)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


_CPU_USE = [0.0, 0.0]   # process CPU seconds and wall seconds of the timed oracle runs


def oracle_cores() -> float:
    """Threads the timed oracle runs kept busy on average (CPU time / wall time: numpy's
    BLAS may use several host cores)."""
    return round(_CPU_USE[0] / _CPU_USE[1], 1) if _CPU_USE[1] > 0 else 1.0


def cpu_reference_step(k2, b, rhs_index: int, maxit: int):
    """Oracle solve (FP64 numpy, plain SL preconditioner) of one right-hand side, at most
    maxit iterations; (s, iters)."""
    import numpy as np
    from oracle import helmholtz as H
    n = k2.shape[0]
    prob = H.Problem(k2.astype(np.float64), omega=0.2 * np.pi * n, h=1.0 / n, abc_width=16)
    t0, c0 = time.perf_counter(), time.process_time()
    res = H.fgmres(prob.A, H.precond_v(prob), b[rhs_index], m=RESTART, tol=TOL, maxit=maxit)
    wall = time.perf_counter() - t0
    _CPU_USE[0] += time.process_time() - c0
    _CPU_USE[1] += wall
    return wall, res.iters


def run_reference(args):
    """The FP64 numpy oracle on the host cores, on the benchmark workload.  Bounded steps:
    each step times one FGMRES(10) iteration with M_V on one right-hand side and scales it
    to the solve (seconds per iteration x M_V's iteration count x right-hand sides).  The
    oracle's own U-Net forward (FP64 loop nests) would make its M_VU iteration ~20x its M_V
    iteration at 2048^2, so the timed oracle path is its faster one."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    k2, b = build_problem(0)
    iters = M_V_ITERS_DEFAULT if (N_GRID, NRHS) == (2048, 16) else None
    if iters is None:   # other sizes: the oracle's own M_V count on one right-hand side (small grids only)
        _, iters = cpu_reference_step(k2, b, 0, maxit=20000)
    times = []
    for s in range(args.warmup + args.steps):
        t, it = cpu_reference_step(k2, b, s % NRHS, maxit=1)
        if s >= args.warmup:
            times.append(t / max(it, 1) * iters * NRHS)
    v = statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(N_GRID, NRHS), "precond": "M_V (the oracle's faster preconditioner)",
                       "nrhs": NRHS, "grid": N_GRID},
            "cpu_baseline": {"value": v, "unit": "s", "cores": oracle_cores(), "kind": "oracle",
                             "sample": f"per step one FGMRES({RESTART}) iteration of one right-hand side by the FP64 "
                                       f"numpy oracle with M_V, scaled by {iters} iterations x {NRHS} right-hand "
                                       f"sides (the GPU's M_V iteration count for this problem)"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def train_base(lib, rank):
    """The base network: Eq. 3.8-3.9 pairs of one random 256^2 medium, MSE loss (Eq. 3.7),
    Adam (the paper's single-model recipe on a medium no case solves on)."""
    import torch
    from paper_2203_11025_gb300 import synth
    from paper_2203_11025_gb300 import train as T
    hz = lib.Helmholtz(torch.from_numpy(synth.grf_kappa2(BASE_GRID, BASE_GRID, BASE_SEED + rank)).cuda())
    t0 = time.perf_counter()
    pairs = hz.gen_pairs(TRAIN_PAIRS, 5151 + rank, 10)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=7 + rank)
    t0 = time.perf_counter()
    hist = T.train(hz, net, pairs=pairs, epochs=TRAIN_EPOCHS, batch=TRAIN_BATCH, lr=TRAIN_LR, seed=11 + rank)
    torch.cuda.synchronize()
    info = {"pairs": TRAIN_PAIRS, "grid": BASE_GRID, "medium_seed": BASE_SEED + rank, "epochs": TRAIN_EPOCHS,
            "lr": TRAIN_LR, "batch": TRAIN_BATCH, "gen_s": round(t_gen, 2),
            "train_s": round(time.perf_counter() - t0, 2), "loss_first": round(hist[0], 1),
            "loss_last": round(hist[-1], 1)}
    hz.close()
    return net, info


def general_case(lib, dev, rank):
    """The general network on a medium it never saw (the 256^2 x 8 case's problem): M_VU
    against M_V iterations and solve times, no retraining."""
    import torch
    gnet, ginfo = train_general(lib, rank)
    k2, b = build_problem(rank, 256, 8)
    hz = lib.Helmholtz(torch.from_numpy(k2).to(dev))
    bd = torch.from_numpy(b).to(dev)
    out = {"training": ginfo}
    for name, pc, nt in (("M_V", lib.HELM_PREC_V, None), ("M_VU", lib.HELM_PREC_VU, gnet)):
        hz.fgmres(bd, precond=pc, net=nt, tol=TOL, maxit=20000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = hz.fgmres(bd, precond=pc, net=nt, tol=TOL, maxit=20000)
        torch.cuda.synchronize()
        out.setdefault("fgmres_iters", {})[name] = info["iters_max"]
        out.setdefault("solve_s", {})[name] = time.perf_counter() - t0
        assert info["status"] == 0 and info["relres_max"] <= TOL, (name, info)
    out["medium"] = "the 256x256x8 case's medium (not among the 16 training media)"
    hz.close()
    gnet.close()
    return out


def encoder_solver_case(lib, dev, rank):
    """The encoder-solver pair of Sec. 3.3 (512^2 unknowns, 32 right-hand sides): the encoder
    U-Net maps the medium to context features once per medium, the solver U-Net (with those
    features at every level) is the M_VU network.  Both are trained jointly (Eq. 3.7, Adam) on
    Eq. 3.8-3.9 pairs of the case's medium; FGMRES with M_VU against M_V, iterations and solve
    times."""
    import numpy as np
    import torch
    from paper_2203_11025_gb300 import synth
    from paper_2203_11025_gb300 import train as T
    n = ES_GRID
    k2 = synth.grf_kappa2(n, n, synth.medium_seed(rank))
    pos = synth.source_positions(n, n, ES_POINTS, synth.rhs_seed(rank), 16)
    b = np.concatenate([synth.point_sources(n, n, pos, 1.0 / n),
                        synth.gaussian_rhs(n, n, ES_GAUSS, 2003 + rank)]).astype(np.complex128)
    hz = lib.Helmholtz(torch.from_numpy(k2).to(dev))
    bd = torch.from_numpy(b).to(dev)
    t0 = time.perf_counter()
    pairs = hz.gen_pairs(ES_PAIRS, 4242 + rank, 10)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    enc = lib.UNet(kind=lib.UNET_ENCODER, seed=1 + rank)
    sol = lib.UNet(kind=lib.UNET_SOLVER, seed=2 + rank)
    sol.attach_encoder(enc)
    t0 = time.perf_counter()
    hist = T.train(hz, sol, pairs=pairs, epochs=ES_EPOCHS, batch=TRAIN_BATCH, lr=TRAIN_LR, seed=11 + rank)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del pairs
    held = hz.gen_pairs(16, 9100 + rank, 10)       # pairs the training never saw
    rel = T.relative_error(hz, sol, held, 16)
    del held
    sol.encode(hz)            # context features of this medium, once
    out = {"grid": n, "rhs": {"point_sources": ES_POINTS, "complex_gaussian": ES_GAUSS},
           "training": {"pairs": ES_PAIRS, "epochs": ES_EPOCHS, "lr": TRAIN_LR, "batch": TRAIN_BATCH,
                        "gen_s": round(t_gen, 2), "train_s": round(t_train, 2), "loss_first": round(hist[0], 1),
                        "loss_last": round(hist[-1], 1), "relative_error_heldout": round(rel, 3)}}
    for name, pc, nt in (("M_V", lib.HELM_PREC_V, None), ("M_VU", lib.HELM_PREC_VU, sol)):
        hz.fgmres(bd, precond=pc, net=nt, tol=TOL, maxit=20000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info = hz.fgmres(bd, precond=pc, net=nt, tol=TOL, maxit=20000)
        torch.cuda.synchronize()
        out.setdefault("solve_s", {})[name] = time.perf_counter() - t0
        out.setdefault("fgmres_iters_max", {})[name] = info["iters_max"]
        its = info["iters"]
        out.setdefault("fgmres_iters_mean", {})[name] = {
            "point_sources": float(np.mean(its[:ES_POINTS])), "complex_gaussian": float(np.mean(its[ES_POINTS:]))}
        assert info["status"] == 0 and info["relres_max"] <= TOL, (name, info)
    out["precond"] = "encoder-solver M_VU (solver U-Net with the encoder's context features, then the V-cycle)"
    hz.close()
    sol.close()
    enc.close()
    return out


def train_general(lib, rank):
    """The general network (Sec. 3.4.1 / 4): Eq. 3.8-3.9 pairs generated by the library's
    SL-FGMRES on TRAIN_MEDIA random media, MSE loss (Eq. 3.7), Adam; returns (net, info)."""
    import torch
    from paper_2203_11025_gb300 import synth
    from paper_2203_11025_gb300 import train as T
    t0 = time.perf_counter()
    media = []
    for k in range(TRAIN_MEDIA):
        hz = lib.Helmholtz(torch.from_numpy(synth.grf_kappa2(BASE_GRID, BASE_GRID, 10 ** 6 + 97 * rank + k)).cuda())
        media.append((hz, hz.gen_pairs(TRAIN_PAIRS_PER_MEDIUM, 4000 + 97 * rank + k, 10)))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=7 + rank)
    t0 = time.perf_counter()
    hist = T.train_media(media, net, epochs=TRAIN_EPOCHS, batch=TRAIN_BATCH, lr=TRAIN_LR, seed=11 + rank)
    torch.cuda.synchronize()
    info = {"media": TRAIN_MEDIA, "pairs": TRAIN_MEDIA * TRAIN_PAIRS_PER_MEDIUM, "grid": BASE_GRID,
            "epochs": TRAIN_EPOCHS, "lr": TRAIN_LR, "batch": TRAIN_BATCH, "gen_s": round(t_gen, 2),
            "train_s": round(time.perf_counter() - t0, 2), "loss_first": round(hist[0], 1),
            "loss_last": round(hist[-1], 1)}
    for hz, _ in media:
        hz.close()
    return net, info


def retrain(lib, hz, base_path, n, rank):
    """Load the general network and mini-retrain it on pairs of hz's medium (Sec. 3.5)."""
    import torch
    from paper_2203_11025_gb300 import train as T
    net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=0)
    net.load(base_path)
    t0 = time.perf_counter()
    ch = max(1, (1 << 26) // (n * n))      # the pair generator's FGMRES basis scales with the count
    parts = [hz.gen_pairs(min(ch, RETRAIN_PAIRS - i), 7777 + 1000 * rank + i, 10)
             for i in range(0, RETRAIN_PAIRS, ch)]
    rp = (torch.cat([p[0] for p in parts]), torch.cat([p[1] for p in parts]))
    del parts
    bs = max_batch(n, 16)
    hist = T.train(hz, net, pairs=rp, epochs=RETRAIN_EPOCHS, batch=bs, lr=RETRAIN_LR, seed=5 + rank)
    torch.cuda.synchronize()
    del rp
    nh = max_batch(n, 16)
    held = hz.gen_pairs(nh, 9100 + rank, 10)
    info = {"pairs": RETRAIN_PAIRS, "epochs": RETRAIN_EPOCHS, "lr": RETRAIN_LR, "batch": bs,
            "s": round(time.perf_counter() - t0, 2), "loss_last": round(hist[-1], 1),
            "relative_error_heldout": round(T.relative_error(hz, net, held, nh), 3)}
    return net, info


class Case:
    """One problem: its handle, right-hand sides, networks and timed solves."""

    def __init__(self, lib, dev, rank, n, nrhs, base_path):
        import torch
        self.lib, self.n, self.nrhs = lib, n, nrhs
        self.k2, self.b = build_problem(rank, n, nrhs)
        self.hz = lib.Helmholtz(torch.from_numpy(self.k2).to(dev))
        self.net, self.tinfo = retrain(lib, self.hz, base_path, n, rank)
        self.bd = torch.from_numpy(self.b).to(dev)
        self.x = torch.zeros_like(self.bd)
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.P = {"M_VU": (lib.HELM_PREC_VU, self.net), "M_V": (lib.HELM_PREC_V, None)}
        if n <= 256:
            self.P["M_JU"] = (lib.HELM_PREC_JU, self.net)
        # M_JU (a comparison column) may stall on some right-hand sides: capped, converged count reported
        self.maxit = {"M_VU": 20000, "M_V": 20000, "M_JU": 3000}
        self.converged, self.last_info = {}, {}

    def solve(self, name):
        pc, nt = self.P[name]
        _, info = self.hz.fgmres(self.bd, self.x, precond=pc, net=nt, tol=TOL, maxit=self.maxit[name],
                                 restart=RESTART, flags=self.lib.HELM_FLAG_X0_ZERO)
        return info

    def timed(self, name, steps):
        import torch
        stream = torch.cuda.current_stream()
        tot, its, launches = 0.0, [], []
        for _ in range(steps):
            self.flush.fill_(1.0)                    # L2 flush between timed steps (256 MB write)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = self.solve(name)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
            its.append(info["iters_max"])
            launches.append(info["launches"])
            self.converged[name] = int(sum(r <= TOL for r in info["relres"]))
            self.last_info[name] = info
            if name != "M_JU":
                assert info["status"] == 0 and info["relres_max"] <= TOL, (name, info)
        return tot / steps, max(its), int(sum(launches))

    def summary(self, steps):
        """Solve times and iterations of every preconditioner (steps timed solves each)."""
        from paper_2203_11025_gb300 import metrics
        for name in self.P:
            self.solve(name)
        out = {"solve_s": {}, "fgmres_iters": {}}
        for name in self.P:
            ms, it, _ = self.timed(name, steps)
            out["solve_s"][name] = ms / 1e3
            out["fgmres_iters"][name] = it
        out["speedup_vs_plain_sl"] = out["solve_s"]["M_V"] / out["solve_s"]["M_VU"]
        out["converged_rhs"] = dict(self.converged)
        out["convergence_factor"] = {k: metrics.summary(v["relres"], v["iters"]) for k, v in self.last_info.items()}
        out["timed_steps"] = steps
        out["training"] = self.tinfo
        return out


C4_SIZES = (256, 384, 512, 768, 1024)
C4_PROBLEMS = 64
C4_RPP = 4


def c4_case(lib, dev, rank, base_path):
    """64 independent problems, grid sizes drawn (seeded) from {256, 384, 512, 768, 1024}^2,
    each with its own random medium and 4 point sources, M_VU with the base network:
    one fgmres_solve_batch call (one handle per size holding its problems' media, one
    network handle per size) against the same problems solved one by one (a handle each).
    Setup and graph capture are outside both timed regions."""
    import numpy as np
    import torch
    from paper_2203_11025_gb300 import synth
    u = synth.uniform01(8800 + rank, C4_PROBLEMS)
    sizes = [C4_SIZES[min(int(v * len(C4_SIZES)), len(C4_SIZES) - 1)] for v in u]
    groups = {}
    for p, n in enumerate(sizes):
        groups.setdefault(n, []).append(p)
    handles, nets, bs, meta = [], [], [], []
    for n, probs in sorted(groups.items()):
        k2 = np.stack([synth.grf_kappa2(n, n, 5000 + 100 * rank + p) for p in probs])
        hz = lib.Helmholtz(torch.from_numpy(k2).to(dev), rpp=C4_RPP)
        b = np.concatenate([synth.point_sources(n, n, synth.source_positions(n, n, C4_RPP, 6000 + 100 * rank + p, 16),
                                                1.0 / n) for p in probs])
        net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=0)
        net.load(base_path)
        handles.append(hz)
        nets.append(net)
        bs.append(torch.from_numpy(b).to(dev))
        meta.append((n, probs, k2, b))
    lib.fgmres_batch(handles, bs, precond=lib.HELM_PREC_VU, nets=nets, tol=TOL, maxit=20000)   # tune, capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, infos = lib.fgmres_batch(handles, bs, precond=lib.HELM_PREC_VU, nets=nets, tol=TOL, maxit=20000)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    for inf in infos:
        assert inf["status"] == 0 and inf["relres_max"] <= TOL, inf
    # the same problems one by one, one handle each (created, warmed and captured untimed)
    t_seq, seq_iters = 0.0, {}
    for (n, probs, k2, b), net in zip(meta, nets):
        for q, p in enumerate(probs):
            hz1 = lib.Helmholtz(torch.from_numpy(k2[q]).to(dev))
            b1 = torch.from_numpy(b[q * C4_RPP:(q + 1) * C4_RPP]).to(dev)
            hz1.fgmres(b1, precond=lib.HELM_PREC_VU, net=net, tol=TOL, maxit=20000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, inf1 = hz1.fgmres(b1, precond=lib.HELM_PREC_VU, net=net, tol=TOL, maxit=20000)
            torch.cuda.synchronize()
            t_seq += time.perf_counter() - t0
            seq_iters[n] = max(seq_iters.get(n, 0), inf1["iters_max"])
            hz1.close()
    out = {"problems": C4_PROBLEMS, "rhs_per_problem": C4_RPP,
           "problems_per_size": {f"{n}x{n}": len(probs) for n, probs, _, _ in meta},
           "batched_s": t_batch, "sequential_s": t_seq, "speedup_batched": t_seq / t_batch,
           "fgmres_iters_max": {f"{m[0]}x{m[0]}": inf["iters_max"] for m, inf in zip(meta, infos)},
           "sequential_iters_max": {f"{n}x{n}": v for n, v in seq_iters.items()},
           "precond": "M_VU, the base network (no retraining: every problem has its own random medium)",
           "timing": "host wall clock around one call, device synchronised on both sides"}
    for hz in handles:
        hz.close()
    for net in nets:
        net.close()
    return out


def hbm_kernels(hz, nrhs, hbm_peak):
    """Algorithmic GB/s of the HBM-bound kernels at the case's size (helm_time_kernel: CUDA
    events around back-to-back launches on the FP32 workspace)."""
    names = {0: "k_apply (y = A x)", 1: "k_resid_restrict_m (residual + full weighting)",
             2: "k_prolong_jacobi_m (prolongation + correction + Jacobi)", 3: "k_arnoldi_update2 (CGS update)",
             6: "k_arnoldi_project2 (A z + inner products)"}
    out = {}
    for k, nm in names.items():
        ms, nb = hz.time_kernel(k, nrhs, reps=20)
        gbs = nb / (ms * 1e-3) / 1e9
        out[nm] = {"launch_ms": ms, "bytes_per_launch": nb, "achieved": gbs, "frac": gbs / hbm_peak}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2203_11025_gb300 import lib
    from paper_2203_11025_gb300 import metrics

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    base, binfo = train_base(lib, rank)
    tmp = tempfile.mkdtemp(prefix="helm_bench_")
    base_path = os.path.join(tmp, f"base_rank{rank}.ckpt")
    base.save(base_path, {"kind": "base network", **binfo})
    base.close()

    case = Case(lib, dev, rank, N_GRID, NRHS, base_path)
    for name in case.P:
        for _ in range(max(1, args.warmup if name == "M_VU" else 1)):
            case.solve(name)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.profiler.start()     # profiler range (ncu --profile-from-start off) = the timed M_VU solves
    ms, it_vu, launches = case.timed("M_VU", args.steps)
    torch.cuda.profiler.stop()
    barrier()
    ck = clocks.stop()
    ms_v, it_v, _ = case.timed("M_V", args.steps)
    ms_ju, it_ju = None, None
    if "M_JU" in case.P:
        ms_ju, it_ju, _ = case.timed("M_JU", args.steps)
    ms, ms_v = max_over_ranks([ms, ms_v], dev)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    bh = torch.from_numpy(case.b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    flags = lib.HELM_FLAG_HOST_IO | lib.HELM_FLAG_X0_ZERO
    case.hz.fgmres(bh, xh, precond=lib.HELM_PREC_VU, net=case.net, tol=TOL, maxit=20000, restart=RESTART, flags=flags)
    barrier()
    e2e = []
    for _ in range(min(args.steps, E2E_STEPS)):
        case.flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        case.hz.fgmres(bh, xh, precond=lib.HELM_PREC_VU, net=case.net, tol=TOL, maxit=20000, restart=RESTART,
                       flags=flags)
        e2e.append(time.perf_counter() - t0)
    e2e_s = statistics.mean(e2e)

    # rooflines at the benchmark's size: the U-Net convolution layers (tensor) and the
    # stencil / Arnoldi kernels (HBM); the preconditioner's last forward set the layer geometry
    hbm_peak, tc_peak, peak_kind = peaks()
    names = net_layer_names(case.net)
    layers = []
    for li in range(len(names)):
        lms, fl, tc = case.net.time_layer(li, reps=10)
        layers.append((lms, fl, tc, names[li]))
    tot_conv_ms = sum(l[0] for l in layers)
    top = max(layers, key=lambda l: l[0])
    tc_layers = [l for l in layers if l[2] in (1, 2)]     # tensor-core kernels (TMA or cp.async fed)
    tc_ms = sum(l[0] for l in tc_layers)
    tc_fl = sum(l[1] for l in tc_layers)
    hbm = hbm_kernels(case.hz, NRHS, hbm_peak)
    dom = max(hbm.items(), key=lambda kv: kv[1]["launch_ms"])
    tiles = {f"level{l}": {"resid_restrict": case.hz.tile_choice(0, l, NRHS),
                           "prolong_jacobi": case.hz.tile_choice(1, l, NRHS)} for l in range(2)}

    extras = {}
    if not args.no_extras:
        for (n, k) in EXTRAS:
            if (n, k) == (N_GRID, NRHS):
                continue
            c2 = Case(lib, dev, rank, n, k, base_path)
            extras[f"{n}x{n}x{k}"] = c2.summary(min(args.steps, EXTRA_STEPS))
            c2.hz.close()
            c2.net.close()
        extras["general_network_unseen_256x256x8"] = general_case(lib, dev, rank)
        extras["batched_uneven_64"] = c4_case(lib, dev, rank, base_path)
        extras["encoder_solver_512x512x32"] = encoder_solver_case(lib, dev, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t1, it1 = cpu_reference_step(case.k2, case.b, 0, maxit=RESTART)
        cpu = {"value": t1 / it1 * it_v * NRHS, "unit": "s", "cores": oracle_cores(), "kind": "oracle",
               "sample": f"extrapolated: one FGMRES({RESTART}) restart cycle of right-hand side 0 with M_V by the "
                         f"FP64 numpy oracle ({t1:.1f} s, {it1} iterations), x {it_v}/{it1} iterations x {NRHS} "
                         f"right-hand sides"}
    if rank == 0:
        achieved = tc_fl / (tc_ms * 1e-3) / 1e12
        chunk = max_batch(N_GRID, NRHS)
        traffic = (CONV_DRAM_BYTES_PER_PIXEL * chunk * N_GRID * N_GRID) if CONV_DRAM_BYTES_PER_PIXEL else None
        line = {
            "metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "c32+f64 Krylov, bf16 U-Net", "data": "synthetic",
            "config": {"workload": workload(N_GRID, NRHS), "precond": "M_VU", "nrhs": NRHS, "grid": N_GRID,
                       "fgmres_iters": {"M_VU": it_vu, "M_V": it_v, **({"M_JU": it_ju} if it_ju else {})},
                       "converged_rhs": case.converged, "maxit": case.maxit,
                       "convergence_factor": {k: metrics.summary(v["relres"], v["iters"])
                                              for k, v in case.last_info.items()},
                       "solve_s": {"M_VU": ms / 1e3, "M_V": ms_v / 1e3,
                                   **({"M_JU": ms_ju / 1e3} if ms_ju else {})},
                       "speedup_vs_plain_sl": ms_v / ms,
                       "training": {"base": binfo, "mini_retraining": case.tinfo},
                       "other_cases": extras,
                       "tile_tuner": tiles,
                       "l2": "flushed between timed steps (256 MB write)",
                       "graph": "one CUDA graph per restart cycle",
                       "network_chunk": chunk},
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(case.b.nbytes),
                    "d2h_bytes_per_step": int(case.b.nbytes), "steps": len(e2e)},
            "roofline": {"bound": "tensor", "kernel": "k_conv_tma / k_conv_tma_reuse (tcgen05 implicit-GEMM "
                                                      "convolutions: all tensor-core layers of one U-Net forward)",
                         "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s", "frac": achieved / tc_peak,
                         "traffic": traffic,
                         "traffic_scope": (f"DRAM bytes of the 20 convolution launches of one forward of {chunk} "
                                           f"images, scaled by pixels from an ncu capture at 4 x 1024^2")
                         if traffic else "not captured for the current kernels",
                         "peak_kind": peak_kind + " bf16 burst", "forward_images": chunk,
                         "layer_ms_total": tot_conv_ms, "top_layer": {"name": top[3], "ms": top[0],
                                                                      "tflops": top[1] / top[0] / 1e9}},
            "roofline_hbm": {"bound": "hbm", "kernel": dom[0], "achieved": dom[1]["achieved"], "peak": hbm_peak,
                             "unit": "GB/s", "frac": dom[1]["frac"], "bytes_per_launch": dom[1]["bytes_per_launch"],
                             "launch_ms": dom[1]["launch_ms"], "kernels": hbm},
            "cpu_baseline": cpu,
            "clocks": ck,
            "gpu_launches": launches,
        }
        print(json.dumps(line), flush=True)
    case.hz.close()
    if world > 1:
        dist.destroy_process_group()


def net_layer_names(net):
    """Convolution layers in the library's layer order (include/unet.h)."""
    w = [net.cfg.widths[i] for i in range(net.cfg.levels)]
    names = []
    for l in range(1, len(w) + 1):
        names.append(f"down{l}")
        for r in range(net.cfg.coarse_resnets if l == len(w) else 1):
            names += [f"res{l}.{r}.k1", f"res{l}.{r}.k2"]
    for l in range(len(w), 0, -1):
        names.append(f"up{l}")
    return names


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the 1024^2 and 256^2 cases")
    ap.add_argument("--grid", type=int, default=2048, help="grid size n (n x n)")
    ap.add_argument("--nrhs", type=int, default=16, help="right-hand sides")
    args = ap.parse_args()
    global N_GRID, NRHS
    N_GRID, NRHS = args.grid, args.nrhs
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
