"""Small, self-contained GPU cases for profiling single kernels (ncu), e.g.

  python -m paper_2203_11025_gb300.profcase unet 256 8     # one U-Net forward, 8 images of 256^2
  python -m paper_2203_11025_gb300.profcase coarse 256 8   # one coarsest-grid solve (fine grid 256^2, 8 RHS)
  python -m paper_2203_11025_gb300.profcase hbm 2048 16    # per-launch time and GB/s of the HBM-bound kernels
  python -m paper_2203_11025_gb300.profcase layers 256 8   # per-layer times of the U-Net forward
  python -m paper_2203_11025_gb300.profcase mvu 256 8      # one FGMRES(10) restart cycle with M_VU
                                                           # (profiler range = that cycle)
  python -m paper_2203_11025_gb300.profcase mv 256 8       # the same with the plain SL V-cycle (M_V)
  python -m paper_2203_11025_gb300.profcase train 256 16   # one training step (forward, MSE, backward,
                                                           # Adam; profiler range = that step)
  python -m paper_2203_11025_gb300.profcase sweep 256 16   # block FGMRES + M_V: block iterations and time
                                                           # for block sizes 1..16 and restarts 5, 10, 20
  python -m paper_2203_11025_gb300.profcase block 256 8    # one block FGMRES(10) cycle with M_V
  python -m paper_2203_11025_gb300.profcase resloss 256 16 # the residual loss of a batch of 16
  python -m paper_2203_11025_gb300.profcase variants 1024 8 # stencil-kernel times and the M_V solve per
                                                           # boundary mode and stencil

Inputs are seeded and synthetic; nothing here checks results (the tests do).
"""
from __future__ import annotations

import sys


def main(argv):
    import numpy as np
    import torch

    from paper_2203_11025_gb300 import lib, synth
    what = argv[1] if len(argv) > 1 else "unet"
    n = int(argv[2]) if len(argv) > 2 else 256
    b = int(argv[3]) if len(argv) > 3 else 8
    if what in ("unet", "layers"):
        net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=1)
        x = torch.from_numpy(np.random.default_rng(0).standard_normal((b, n, n, 4)).astype(np.float32)).cuda()
        net.forward(x)
        torch.cuda.synchronize()
        if what == "layers":
            names = []
            w = [net.cfg.widths[i] for i in range(net.cfg.levels)]
            for l in range(1, len(w) + 1):
                names.append(f"down{l}")
                for r in range(net.cfg.coarse_resnets if l == len(w) else 1):
                    names += [f"res{l}.{r}.k1", f"res{l}.{r}.k2"]
            names += [f"up{l}" for l in range(len(w), 0, -1)]
            tot = 0.0
            for i, nm in enumerate(names):
                ms, fl, tc = net.time_layer(i, reps=10)
                tot += ms
                kind = {3: "direct", 2: "tma-tc", 1: "cpasync-tc"}.get(tc, "cuda-core")
                print(f"{nm:12s} {ms * 1e3:8.1f} us {fl / ms / 1e9:7.1f} TFLOP/s {kind}")
            print(f"total {tot * 1e3:.1f} us")
    elif what == "hbm":
        # per-launch device time and algorithmic bandwidth of the HBM-bound kernels
        # (helm_time_kernel: 0 apply, 1 residual + restriction, 2 prolongation + Jacobi,
        # 3 Arnoldi update sweep at j = 4, 6 projection sweep at j = 4; 4 V-cycle, 5 coarsest solve)
        import json
        k2 = synth.grf_kappa2(n, n, 1000)
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
        rec = {"n": n, "nrhs": b}
        for kern in (0, 1, 2, 3, 6, 4, 5):
            ms, by = hz.time_kernel(kern, b, reps=10)
            rec[str(kern)] = {"us": round(ms * 1e3, 1), "GB/s": round(by / ms / 1e6, 0) if by else None}
        print(json.dumps(rec))
    elif what == "coarse":
        k2 = synth.grf_kappa2(n, n, 1000)
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
        ms, _ = hz.time_kernel(5, b, reps=3)
        print(f"coarse solve {ms * 1e3:.1f} us")
    elif what in ("mvu", "mv"):
        k2 = synth.grf_kappa2(n, n, synth.medium_seed(0))
        pos = synth.source_positions(n, n, b, synth.rhs_seed(0), 16)
        rhs = torch.from_numpy(synth.point_sources(n, n, pos, 1.0 / n).astype(np.complex128)).cuda()
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
        net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=1) if what == "mvu" else None
        pc = lib.HELM_PREC_VU if what == "mvu" else lib.HELM_PREC_V
        x = torch.zeros_like(rhs)
        for _ in range(2):   # warm-up: workspaces, graphs
            hz.fgmres(rhs, x, precond=pc, net=net, tol=1e-7, maxit=10, restart=10, flags=lib.HELM_FLAG_X0_ZERO)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        hz.fgmres(rhs, x, precond=pc, net=net, tol=1e-7, maxit=10, restart=10, flags=lib.HELM_FLAG_X0_ZERO)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif what == "train":
        from paper_2203_11025_gb300 import train as T
        k2 = synth.grf_kappa2(n, n, synth.medium_seed(0))
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
        net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=1)
        r, e = hz.gen_pairs(b, 5151, 10)
        idx, coef = next(T.batches(np.random.default_rng(0), b, b, 2))
        x, t = hz.make_batch(r, e, idx, coef)

        def step():
            net.zero_grad()
            out = net.forward(x, train=True)
            _, g = net.mse(out, t)
            net.backward(g)
            net.adam_step(lr=1e-4)
        step()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    elif what == "block":
        k2 = synth.grf_kappa2(n, n, synth.medium_seed(0))
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
        pos = synth.source_positions(n, n, b, synth.rhs_seed(0), 16)
        rhs = torch.from_numpy(synth.point_sources(n, n, pos, 1.0 / n).astype(np.complex128)).cuda()
        hz.fgmres(rhs, tol=1e-7, maxit=10, block=True)
    elif what == "resloss":
        k2 = synth.grf_kappa2(n, n, synth.medium_seed(0))
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
        rng = np.random.default_rng(0)
        y = torch.from_numpy(rng.standard_normal((b, n, n, 2)).astype(np.float32)).cuda()
        x = torch.from_numpy(rng.standard_normal((b, n, n, 4)).astype(np.float32)).cuda()
        for _ in range(2):
            hz.residual_loss(y, x)
        torch.cuda.synchronize()
    elif what == "sweep":
        # the influence of the block size and of the Krylov subspace size (Sec. 4): block
        # FGMRES(m) with M_V on the first `bs` of b point sources, and independent FGMRES
        import json
        k2 = synth.grf_kappa2(n, n, synth.medium_seed(0))
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
        pos = synth.source_positions(n, n, b, synth.rhs_seed(0), 16)
        rhs = torch.from_numpy(synth.point_sources(n, n, pos, 1.0 / n).astype(np.complex128)).cuda()
        for m in (5, 10, 20):
            bs = 1
            while bs <= b:
                for block in (True, False):
                    if (not block and bs != b) or (block and (m + 1) * bs * bs > 4608):
                        continue
                    sub = rhs[:bs].contiguous()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    _, info = hz.fgmres(sub, tol=1e-7, maxit=20000, restart=m, block=block)
                    e1.record()
                    e1.synchronize()
                    print(json.dumps({"restart": m, "rhs": bs, "block": block, "iters": info["iters_max"],
                                      "ms": round(e0.elapsed_time(e1), 2), "relres_max": info["relres_max"]}))
                bs *= 2
    elif what == "variants":
        # boundary modes and stencils side by side: per-launch time and algorithmic GB/s of
        # the stencil kernels (helm_time_kernel 0-3) and the M_V solve of b point sources
        import json
        k2 = torch.from_numpy(synth.grf_kappa2(n, n, synth.medium_seed(0))).cuda()
        pos = synth.source_positions(n, n, b, synth.rhs_seed(0), 16)
        rhs = torch.from_numpy(synth.point_sources(n, n, pos, 1.0 / n).astype(np.complex128)).cuda()
        for bc, st in ((lib.HELM_BC_DIRICHLET, lib.HELM_STENCIL_5PT), (lib.HELM_BC_REFLECT, lib.HELM_STENCIL_5PT),
                       (lib.HELM_BC_REPLICATE, lib.HELM_STENCIL_5PT),
                       (lib.HELM_BC_DIRICHLET, lib.HELM_STENCIL_COMPACT4)):
            hz = lib.Helmholtz(k2, bc=bc, stencil=st)
            rec = {"bc": bc, "stencil": st}
            for kern in range(4):
                ms, nbytes = hz.time_kernel(kern, b, reps=50)
                rec[f"kernel{kern}_us"] = round(ms * 1e3, 2)
                rec[f"kernel{kern}_gbs"] = round(nbytes / (ms * 1e-3) / 1e9, 1) if nbytes else None
            hz.fgmres(rhs, tol=1e-7, maxit=20000)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, info = hz.fgmres(rhs, tol=1e-7, maxit=20000)
            e1.record()
            e1.synchronize()
            rec.update({"mv_ms": round(e0.elapsed_time(e1), 2), "mv_iters": info["iters_max"]})
            print(json.dumps(rec), flush=True)
            hz.close()
    else:
        raise SystemExit(f"unknown case {what}")


if __name__ == "__main__":
    main(sys.argv)
