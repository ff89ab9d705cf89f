"""Thin Python binding of libhelm's C ABI (include/helm.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Functions keep the C names; `Helmholtz` bundles a handle for convenience.
Vectors are torch tensors on the GPU (complex64 -> HELM_C32, complex128 ->
HELM_C64), contiguous, shaped (nrhs, ny, nx) or (ny, nx).  Loading fails
loudly if the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhelm.so")

HELM_OK, HELM_MAXIT = 0, 1
HELM_EINVAL, HELM_ECUDA, HELM_ENAN, HELM_ENOMEM, HELM_EUNSUPPORTED = -1, -2, -3, -5, -6
HELM_OP_A, HELM_OP_M = 0, 1
HELM_C32, HELM_C64 = 0, 1
HELM_PREC_NONE, HELM_PREC_V, HELM_PREC_JU, HELM_PREC_VU = 0, 1, 2, 3
HELM_FLAG_X0_ZERO, HELM_FLAG_HOST_IO, HELM_FLAG_NO_GRAPH, HELM_FLAG_FP64 = 1, 2, 4, 8
HELM_FLAG_FALLBACK_V = 16
HELM_DESC_MULTIKERNEL_COARSE, HELM_DESC_SINGLE_CTA_COARSE = 1, 2
HELM_BC_DIRICHLET, HELM_BC_REFLECT, HELM_BC_REPLICATE = 0, 1, 2
HELM_STENCIL_5PT, HELM_STENCIL_COMPACT4 = 0, 1
HELM_OP_RHS = 2

# Every symbol include/helm.h declares (checked by the CPU test suite).
ABI_SYMBOLS = [
    "helm_desc_default", "helm_setup", "helm_destroy", "helm_last_error", "helm_level_shape",
    "helm_level_kappa2", "helm_apply", "helm_residual", "helm_jacobi", "helm_restrict",
    "helm_prolong_add", "helm_coarse_solve", "sl_vcycle", "fgmres_solve", "bfgmres_solve", "helm_time_kernel",
    "helm_coarse_solve_static", "helm_tile_choice", "helm_set_tile_choice", "helm_setup_media",
    "fgmres_solve_batch",
    # include/unet.h
    "unet_cfg_default", "unet_create", "unet_destroy", "unet_sizes", "unet_set_params", "unet_get_params",
    "unet_set_bn_stats", "unet_get_bn_stats", "unet_get_grads", "unet_zero_grad", "unet_forward", "unet_backward",
    "unet_mse", "unet_adam_step", "unet_attach_encoder", "unet_encode", "unet_precond", "helm_gen_pairs",
    "unet_make_batch", "unet_status", "unet_time_layer", "unet_residual_loss", "unet_wait_probe",
    "unet_train_step", "unet_save", "unet_load",
]
UNET_FLAG_SIMT, UNET_FLAG_NO_TMA = 1, 2
UNET_STANDALONE, UNET_ENCODER, UNET_SOLVER = 0, 1, 2


class helm_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("h", ctypes.c_double), ("omega", ctypes.c_double),
                ("beta", ctypes.c_double), ("abc_width", ctypes.c_int), ("abc_gamma_max", ctypes.c_double),
                ("levels", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("jacobi_w", ctypes.c_double), ("coarse_its", ctypes.c_int), ("flags", ctypes.c_int),
                ("bc", ctypes.c_int), ("stencil", ctypes.c_int)]


class unet_cfg(ctypes.Structure):
    _fields_ = [("in_ch", ctypes.c_int), ("out_ch", ctypes.c_int), ("levels", ctypes.c_int),
                ("coarse_resnets", ctypes.c_int), ("widths", ctypes.c_int * 8), ("context", ctypes.c_int * 9),
                ("flags", ctypes.c_int)]


class unet_train_opts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("loss", ctypes.c_int)]


UNET_LOSS_MSE, UNET_LOSS_RESIDUAL = 0, 1


class fgmres_opts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("tol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("flags", ctypes.c_int)]


class fgmres_result(ctypes.Structure):
    _fields_ = [("iters_max", ctypes.c_int), ("cycles", ctypes.c_int), ("relres_max", ctypes.c_double),
                ("status", ctypes.c_int), ("iters", ctypes.POINTER(ctypes.c_int)),
                ("relres", ctypes.POINTER(ctypes.c_double)), ("launches", ctypes.c_longlong),
                ("fallbacks", ctypes.c_int)]


_lib = None


def load():
    """Open libhelm.so (once).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libhelm.so not built at {LIB_PATH}; run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "helm_desc_default": (I, [ctypes.POINTER(helm_desc), I, I]),
        "helm_setup": (I, [ctypes.POINTER(helm_desc), P, P, ctypes.POINTER(P)]),
        "helm_setup_media": (I, [ctypes.POINTER(helm_desc), P, I, I, P, ctypes.POINTER(P)]),
        "fgmres_solve_batch": (I, [I, P, I, P, P, P, P, ctypes.POINTER(fgmres_opts), P, P]),
        "helm_destroy": (None, [P]),
        "helm_last_error": (ctypes.c_char_p, []),
        "helm_level_shape": (I, [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "helm_level_kappa2": (I, [P, I, P]),
        "helm_apply": (I, [P, I, I, P, P, I, I, P]),
        "helm_residual": (I, [P, I, I, P, P, P, I, I, P]),
        "helm_jacobi": (I, [P, I, I, P, P, P, I, I, P]),
        "helm_restrict": (I, [P, I, P, P, I, I, P]),
        "helm_prolong_add": (I, [P, I, P, P, I, I, P]),
        "helm_coarse_solve": (I, [P, P, P, I, I, P]),
        "sl_vcycle": (I, [P, P, P, I, I, I, P]),
        "fgmres_solve": (I, [P, I, P, P, P, I, ctypes.POINTER(fgmres_opts), ctypes.POINTER(fgmres_result), P]),
        "bfgmres_solve": (I, [P, I, P, P, P, I, ctypes.POINTER(fgmres_opts), ctypes.POINTER(fgmres_result), P]),
        "helm_time_kernel": (I, [P, I, I, I, P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(D)]),
        "helm_coarse_solve_static": (I, [I, I, D, D, D, I, D, P, P, P, I, I, P]),
        "helm_tile_choice": (I, [P, I, I, I, ctypes.POINTER(I)]),
        "helm_set_tile_choice": (I, [P, I, I, I, I]),
        "unet_cfg_default": (I, [ctypes.POINTER(unet_cfg), I]),
        "unet_create": (I, [ctypes.POINTER(unet_cfg), ctypes.c_ulonglong, ctypes.POINTER(P)]),
        "unet_destroy": (None, [P]),
        "unet_sizes": (I, [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
        "unet_set_params": (I, [P, P, ctypes.c_longlong]),
        "unet_get_params": (I, [P, P, ctypes.c_longlong]),
        "unet_set_bn_stats": (I, [P, P, ctypes.c_longlong]),
        "unet_get_bn_stats": (I, [P, P, ctypes.c_longlong]),
        "unet_get_grads": (I, [P, P, ctypes.c_longlong]),
        "unet_zero_grad": (I, [P, P]),
        "unet_forward": (I, [P, P, P, I, I, I, I, P]),
        "unet_backward": (I, [P, P, P, P]),
        "unet_mse": (I, [P, P, ctypes.c_longlong, I, P, P, P]),
        "unet_residual_loss": (I, [P, P, P, I, P, P, P]),
        "unet_adam_step": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, P]),
        "unet_attach_encoder": (I, [P, P]),
        "unet_encode": (I, [P, P, I, P]),
        "unet_precond": (I, [P, P, I, P, P, I, I, P]),
        "helm_gen_pairs": (I, [P, I, ctypes.c_ulonglong, I, P, P, P]),
        "unet_make_batch": (I, [P, P, P, I, I, I, P, P, P, P, P]),
        "unet_status": (I, [P, ctypes.POINTER(I)]),
        "unet_wait_probe": (I, [P, ctypes.c_longlong, I, P]),
        "unet_train_step": (I, [P, P, P, P, I, ctypes.POINTER(unet_train_opts), P, P]),
        "unet_save": (I, [P, ctypes.c_char_p, ctypes.c_char_p]),
        "unet_load": (I, [P, ctypes.c_char_p]),
        "unet_time_layer": (I, [P, I, I, P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(D), ctypes.POINTER(I)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class HelmError(RuntimeError):
    def __init__(self, code, where):
        msg = load().helm_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def _check(code, where, ok=(HELM_OK,)):
    if code not in ok:
        raise HelmError(code, where)
    return code


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _dtype(t):
    import torch
    if t.dtype == torch.complex64:
        return HELM_C32
    if t.dtype == torch.complex128:
        return HELM_C64
    raise TypeError(f"vectors must be complex64 or complex128, got {t.dtype}")


def _nrhs(t, ny, nx):
    if t.dim() == 2:
        return 1
    if t.dim() == 3 and tuple(t.shape[1:]) == (ny, nx):
        return t.shape[0]
    raise ValueError(f"vector shape {tuple(t.shape)} does not match grid ({ny}, {nx})")


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


# ---------------------------------------------------------------- thin C-named calls
def helm_desc_default(nx, ny=None):
    d = helm_desc()
    _check(load().helm_desc_default(ctypes.byref(d), nx, ny or nx), "helm_desc_default")
    return d


def helm_setup(desc, kappa2, stream=None):
    h = ctypes.c_void_p()
    _check(load().helm_setup(ctypes.byref(desc), _ptr(kappa2), _stream(stream), ctypes.byref(h)), "helm_setup")
    return h


def helm_destroy(h):
    load().helm_destroy(h)


def helm_coarse_solve_static(nx, ny, h, omega, beta, abc_width, gamma_max, kappa2, f, x, nrhs, m=10, stream=None):
    """The allocation-free coarsest-grid solve (see include/helm.h); tensors on the GPU."""
    _check(load().helm_coarse_solve_static(nx, ny, h, omega, beta, abc_width, gamma_max, _ptr(kappa2), _ptr(f),
                                           _ptr(x), nrhs, m, _stream(stream)), "helm_coarse_solve_static")
    return x


_NAMED = {
    "bc": {"dirichlet": HELM_BC_DIRICHLET, "reflect": HELM_BC_REFLECT, "replicate": HELM_BC_REPLICATE},
    "stencil": {"5pt": HELM_STENCIL_5PT, "compact4": HELM_STENCIL_COMPACT4},
}


def desc_value(field: str, value):
    """A helm_desc field value; `bc` and `stencil` also accept their names
    ("dirichlet", "reflect", "replicate"; "5pt", "compact4")."""
    if isinstance(value, str):
        names = _NAMED.get(field)
        if names is None or value not in names:
            raise ValueError(f"unknown value {value!r} for helm_desc.{field}")
        return names[value]
    return value


class Helmholtz:
    """A solver handle: medium kappa^2 (float32 CUDA tensor [ny, nx]) plus desc.  A tensor
    [nmedia, ny, nx] with rpp makes a batch handle of one grid size (helm_setup_media):
    right-hand side r is solved on medium r // rpp."""

    def __init__(self, kappa2, desc=None, rpp=0, **overrides):
        import torch
        if kappa2.dtype != torch.float32 or not kappa2.is_cuda:
            raise TypeError("kappa2 must be a float32 CUDA tensor")
        ny, nx = kappa2.shape[-2:]
        self.nmedia = kappa2.shape[0] if kappa2.dim() == 3 else 1
        self.rpp = rpp if self.nmedia > 1 else 0
        self.desc = desc if desc is not None else helm_desc_default(nx, ny)
        for k, v in overrides.items():
            setattr(self.desc, k, desc_value(k, v))
        self.kappa2 = kappa2.contiguous()
        self.lib = load()
        if self.nmedia == 1:
            self.h = helm_setup(self.desc, self.kappa2)
        else:
            h = ctypes.c_void_p()
            _check(self.lib.helm_setup_media(ctypes.byref(self.desc), _ptr(self.kappa2), self.nmedia, self.rpp, None,
                                             ctypes.byref(h)), "helm_setup_media")
            self.h = h

    def close(self):
        if self.h:
            helm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level_shape(self, level):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.helm_level_shape(self.h, level, ctypes.byref(nx), ctypes.byref(ny)), "helm_level_shape")
        return ny.value, nx.value

    def level_kappa2(self, level):
        import torch
        ny, nx = self.level_shape(level)
        out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
        _check(self.lib.helm_level_kappa2(self.h, level, _ptr(out)), "helm_level_kappa2")
        torch.cuda.synchronize()
        return out

    def _vec(self, t, level=0):
        ny, nx = self.level_shape(level)
        if not t.is_contiguous():
            raise ValueError("vectors must be contiguous")
        return _nrhs(t, ny, nx), _dtype(t)

    def apply(self, x, op=HELM_OP_A, level=0, out=None, stream=None):
        import torch
        n, dt = self._vec(x, level)
        y = torch.empty_like(x) if out is None else out
        _check(self.lib.helm_apply(self.h, op, level, _ptr(x), _ptr(y), n, dt, _stream(stream)), "helm_apply")
        return y

    def residual(self, b, x, op=HELM_OP_A, level=0, out=None, stream=None):
        import torch
        n, dt = self._vec(x, level)
        r = torch.empty_like(x) if out is None else out
        _check(self.lib.helm_residual(self.h, op, level, _ptr(b), _ptr(x), _ptr(r), n, dt, _stream(stream)),
               "helm_residual")
        return r

    def jacobi(self, b, x_in=None, op=HELM_OP_M, level=0, out=None, stream=None):
        import torch
        n, dt = self._vec(b, level)
        y = torch.empty_like(b) if out is None else out
        _check(self.lib.helm_jacobi(self.h, op, level, _ptr(b), _ptr(x_in), _ptr(y), n, dt, _stream(stream)),
               "helm_jacobi")
        return y

    def restrict(self, fine, level=0, out=None, stream=None):
        import torch
        n, dt = self._vec(fine, level)
        ny, nx = self.level_shape(level + 1)
        c = torch.empty((fine.shape[0], ny, nx) if fine.dim() == 3 else (ny, nx), dtype=fine.dtype,
                        device=fine.device) if out is None else out
        _check(self.lib.helm_restrict(self.h, level, _ptr(fine), _ptr(c), n, dt, _stream(stream)), "helm_restrict")
        return c

    def prolong_add(self, coarse, fine, level=0, stream=None):
        n, dt = self._vec(fine, level)
        _check(self.lib.helm_prolong_add(self.h, level, _ptr(coarse), _ptr(fine), n, dt, _stream(stream)),
               "helm_prolong_add")
        return fine

    def coarse_solve(self, f, out=None, stream=None):
        import torch
        n, dt = self._vec(f, self.desc.levels - 1)
        x = torch.empty_like(f) if out is None else out
        _check(self.lib.helm_coarse_solve(self.h, _ptr(f), _ptr(x), n, dt, _stream(stream)), "helm_coarse_solve")
        return x

    def vcycle(self, f, x=None, stream=None):
        import torch
        n, dt = self._vec(f, 0)
        zero = x is None
        if zero:
            x = torch.empty_like(f)
        _check(self.lib.sl_vcycle(self.h, _ptr(f), _ptr(x), n, dt, 1 if zero else 0, _stream(stream)), "sl_vcycle")
        return x

    def time_kernel(self, kernel, nrhs, reps=20, stream=None):
        """Mean device ms per launch and algorithmic bytes per launch of an internal kernel."""
        ms, nbytes = ctypes.c_float(), ctypes.c_double()
        _check(self.lib.helm_time_kernel(self.h, kernel, nrhs, reps, _stream(stream), ctypes.byref(ms),
                                         ctypes.byref(nbytes)), "helm_time_kernel")
        return ms.value, nbytes.value

    def tile_choice(self, kernel, level, nrhs):
        """Segment height the tile tuner chose for fused cycle kernel 0 (residual + restriction)
        or 1 (prolongation + Jacobi) of `level` at nrhs right-hand sides (0: not tuned)."""
        v = ctypes.c_int()
        _check(self.lib.helm_tile_choice(self.h, kernel, level, nrhs, ctypes.byref(v)), "helm_tile_choice")
        return v.value

    def set_tile_choice(self, kernel, level, nrhs, seg):
        _check(self.lib.helm_set_tile_choice(self.h, kernel, level, nrhs, seg), "helm_set_tile_choice")

    def gen_pairs(self, count, seed, kmax=10, stream=None):
        """Training pairs (r, e) of Eq. 3.8-3.9 (complex128 CUDA tensors [count, ny, nx])."""
        import torch
        ny, nx = self.level_shape(0)
        r = torch.empty(count, ny, nx, dtype=torch.complex128, device="cuda")
        e = torch.empty_like(r)
        _check(self.lib.helm_gen_pairs(self.h, count, seed, kmax, _ptr(r), _ptr(e), _stream(stream)),
               "helm_gen_pairs")
        return r, e

    def make_batch(self, r, e, idx, coef, stream=None):
        """Network inputs and targets for samples mixing pairs idx [count, nmix] with complex
        coefficients coef [count, nmix] (numpy); r, e: complex128 CUDA pairs."""
        import numpy as np
        import torch
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        coef = np.ascontiguousarray(coef, dtype=np.complex128)
        count, nmix = idx.shape
        ny, nx = self.level_shape(0)
        x = torch.empty(count, ny, nx, 4, dtype=torch.float32, device="cuda")
        t = torch.empty(count, ny, nx, 2, dtype=torch.float32, device="cuda")
        _check(self.lib.unet_make_batch(self.h, _ptr(r), _ptr(e), r.shape[0], count, nmix, idx.ctypes.data,
                                        coef.ctypes.data, _ptr(x), _ptr(t), _stream(stream)), "unet_make_batch")
        return x, t

    def residual_loss(self, out, x, stream=None):
        """Unsupervised residual loss of network outputs out [B, ny, nx, 2] for inputs x
        [B, ny, nx, 4] on this medium; returns (loss tensor [1] on device, gout)."""
        import torch
        gout = torch.empty_like(out)
        loss = torch.empty(1, dtype=torch.float32, device=out.device)
        _check(self.lib.unet_residual_loss(self.h, _ptr(out), _ptr(x.contiguous()), out.shape[0], _ptr(gout),
                                           _ptr(loss), _stream(stream)), "unet_residual_loss")
        return loss, gout

    def unet_precond(self, net, r, kind=HELM_PREC_VU, out=None, stream=None):
        import torch
        n, dt = self._vec(r, 0)
        e = torch.empty_like(r) if out is None else out
        _check(self.lib.unet_precond(self.h, net.handle, kind, _ptr(r), _ptr(e), n, dt, _stream(stream)),
               "unet_precond")
        return e

    def fgmres(self, b, x=None, precond=HELM_PREC_V, net=None, restart=10, tol=1e-7, maxit=5000, flags=0,
               stream=None, block=False):
        """Solve A x = b (complex128 tensors, CUDA or pinned host with HELM_FLAG_HOST_IO).
        block=True: block FGMRES (one Krylov space for all right-hand sides, <= 16 of them).
        Returns (x, info dict)."""
        import torch
        ny, nx = self.level_shape(0)
        n = _nrhs(b, ny, nx)
        if b.dtype != torch.complex128:
            raise TypeError("b must be complex128")
        if x is None:
            x = torch.zeros_like(b)
            flags |= HELM_FLAG_X0_ZERO
        opts = fgmres_opts(restart, tol, maxit, flags)
        iters = (ctypes.c_int * n)()
        relres = (ctypes.c_double * n)()
        res = fgmres_result(0, 0, 0.0, 0, iters, relres, 0)
        netp = net.handle if net is not None and hasattr(net, "handle") else net
        solve = self.lib.bfgmres_solve if block else self.lib.fgmres_solve
        code = solve(self.h, precond, netp, _ptr(b), _ptr(x), n, ctypes.byref(opts), ctypes.byref(res),
                     _stream(stream))
        _check(code, "bfgmres_solve" if block else "fgmres_solve", ok=(HELM_OK, HELM_MAXIT))
        return x, {"status": code, "iters": list(iters), "relres": list(relres), "iters_max": res.iters_max,
                   "relres_max": res.relres_max, "cycles": res.cycles, "launches": res.launches,
                   "fallbacks": res.fallbacks}


def fgmres_batch(handles, bs, precond=HELM_PREC_V, nets=None, restart=10, tol=1e-7, maxit=5000, xs=None,
                 stream=None):
    """Solve the problems of several handles (e.g. one per grid size) in one call
    (fgmres_solve_batch): bs[i] complex128 CUDA tensors [nrhs_i, ny_i, nx_i]; nets: one
    network per handle for the U-Net preconditioners.  Returns (xs, infos)."""
    import torch
    nh = len(handles)
    if xs is None:
        xs = [torch.zeros_like(b) for b in bs]
    flags = HELM_FLAG_X0_ZERO
    opts = fgmres_opts(restart, tol, maxit, flags)
    H = (ctypes.c_void_p * nh)(*[hz.h.value if hasattr(hz.h, "value") else hz.h for hz in handles])
    B = (ctypes.c_void_p * nh)(*[b.data_ptr() for b in bs])
    X = (ctypes.c_void_p * nh)(*[x.data_ptr() for x in xs])
    nr = [int(b.shape[0]) for b in bs]
    NR = (ctypes.c_int * nh)(*nr)
    NETS = None
    if nets is not None:
        NETS = (ctypes.c_void_p * nh)(*[n.handle.value if hasattr(n.handle, "value") else n.handle for n in nets])
    its = [(ctypes.c_int * k)() for k in nr]
    rel = [(ctypes.c_double * k)() for k in nr]
    RES = (fgmres_result * nh)(*[fgmres_result(0, 0, 0.0, 0, its[i], rel[i], 0) for i in range(nh)])
    code = load().fgmres_solve_batch(nh, H, precond, NETS, B, X, NR, ctypes.byref(opts), RES, _stream(stream))
    _check(code, "fgmres_solve_batch", ok=(HELM_OK, HELM_MAXIT))
    infos = [{"status": RES[i].status, "iters": list(its[i]), "relres": list(rel[i]), "iters_max": RES[i].iters_max,
              "relres_max": RES[i].relres_max, "cycles": RES[i].cycles, "launches": RES[i].launches}
             for i in range(nh)]
    return xs, infos


def unet_cfg_default(kind=UNET_STANDALONE):
    c = unet_cfg()
    _check(load().unet_cfg_default(ctypes.byref(c), kind), "unet_cfg_default")
    return c


class UNet:
    """A U-Net of libhelm (include/unet.h): weights live on the GPU."""

    def __init__(self, cfg=None, seed=0, kind=UNET_STANDALONE):
        self.lib = load()
        self.cfg = cfg if cfg is not None else unet_cfg_default(kind)
        h = ctypes.c_void_p()
        _check(self.lib.unet_create(ctypes.byref(self.cfg), seed, ctypes.byref(h)), "unet_create")
        self.handle = h
        npar, nbn = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self.lib.unet_sizes(h, ctypes.byref(npar), ctypes.byref(nbn)), "unet_sizes")
        self.n_params, self.n_bn = npar.value, nbn.value
        self.encoder = None

    def close(self):
        if self.handle:
            self.lib.unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(self.lib.unet_set_params(self.handle, a.ctypes.data, a.size), "unet_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.n_params, np.float32)
        _check(self.lib.unet_get_params(self.handle, a.ctypes.data, a.size), "unet_get_params")
        return a

    def set_bn_stats(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(self.lib.unet_set_bn_stats(self.handle, a.ctypes.data, a.size), "unet_set_bn_stats")

    def get_bn_stats(self):
        import numpy as np
        a = np.empty(self.n_bn, np.float32)
        _check(self.lib.unet_get_bn_stats(self.handle, a.ctypes.data, a.size), "unet_get_bn_stats")
        return a

    def get_grads(self):
        import numpy as np
        import torch
        torch.cuda.synchronize()
        a = np.empty(self.n_params, np.float32)
        _check(self.lib.unet_get_grads(self.handle, a.ctypes.data, a.size), "unet_get_grads")
        return a

    def status(self):
        """Synchronise; True if a tensor-core kernel recorded an expired wait (then cleared)."""
        f = ctypes.c_int()
        _check(self.lib.unet_status(self.handle, ctypes.byref(f)), "unet_status")
        return bool(f.value)

    def wait_probe(self, rounds, arrive=False, stream=None):
        """Launch the failure-detection probe: a bounded mbarrier wait that expires
        (arrive=False, recorded for status()) or completes (arrive=True)."""
        _check(self.lib.unet_wait_probe(self.handle, int(rounds), 1 if arrive else 0, _stream(stream)),
               "unet_wait_probe")

    def time_layer(self, layer, reps=20, stream=None):
        """(ms per repetition, flops, kernel: 3 direct CUDA-core, 2 TMA tensor core, 1 cp.async tensor core,
        0 generic CUDA-core)
        of convolution `layer` in its inference form."""
        ms, fl, tc = ctypes.c_float(), ctypes.c_double(), ctypes.c_int()
        _check(self.lib.unet_time_layer(self.handle, layer, reps, _stream(stream), ctypes.byref(ms), ctypes.byref(fl),
                                        ctypes.byref(tc)), "unet_time_layer")
        return ms.value, fl.value, int(tc.value)

    def zero_grad(self, stream=None):
        _check(self.lib.unet_zero_grad(self.handle, _stream(stream)), "unet_zero_grad")

    def attach_encoder(self, enc):
        _check(self.lib.unet_attach_encoder(self.handle, enc.handle if enc else None), "unet_attach_encoder")
        self.encoder = enc

    def encode(self, hz, train=False, stream=None):
        _check(self.lib.unet_encode(self.handle, hz.h, 1 if train else 0, _stream(stream)), "unet_encode")

    def forward(self, x, train=False, stream=None):
        """x: float32 CUDA tensor [B, ny, nx, in_ch]; returns float32 [B, ny, nx, out_ch]."""
        import torch
        B, ny, nx, _ = x.shape
        out = torch.empty(B, ny, nx, self.cfg.out_ch, dtype=torch.float32, device=x.device)
        _check(self.lib.unet_forward(self.handle, _ptr(x.contiguous()), _ptr(out), B, ny, nx, 1 if train else 0,
                                     _stream(stream)), "unet_forward")
        return out

    def backward(self, gout, want_gx=False, stream=None):
        import torch
        gx = None
        if want_gx:
            B, ny, nx, _ = gout.shape
            gx = torch.empty(B, ny, nx, self.cfg.in_ch, dtype=torch.float32, device=gout.device)
        _check(self.lib.unet_backward(self.handle, _ptr(gout.contiguous()), _ptr(gx), _stream(stream)),
               "unet_backward")
        return gx

    def mse(self, out, target, stream=None):
        """MSE of Eq. 3.7; returns (loss tensor [1] on device, gout)."""
        import torch
        gout = torch.empty_like(out)
        loss = torch.empty(1, dtype=torch.float32, device=out.device)
        _check(self.lib.unet_mse(_ptr(out), _ptr(target.contiguous()), out.numel(), out.shape[0], _ptr(gout),
                                 _ptr(loss), _stream(stream)), "unet_mse")
        return loss, gout

    def train_step(self, hz, x, target=None, lr=1e-4, loss="error", b1=0.9, b2=0.999, eps=1e-8, stream=None):
        """One training step through the C ABI (encoder forward if attached, forward, loss,
        backward, Adam); loss "error" (Eq. 3.7, needs target) or "residual".  Returns the
        loss as a one-element device tensor."""
        import torch
        if loss not in ("error", "residual"):
            raise ValueError(f"unknown loss {loss!r}")
        opts = unet_train_opts(lr, b1, b2, eps, UNET_LOSS_MSE if loss == "error" else UNET_LOSS_RESIDUAL)
        lv = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(self.lib.unet_train_step(self.handle, hz.h, _ptr(x.contiguous()),
                                        _ptr(target.contiguous()) if target is not None else None, x.shape[0],
                                        ctypes.byref(opts), _ptr(lv), _stream(stream)), "unet_train_step")
        return lv

    def save(self, path, meta=None):
        """Write the weights and BatchNorm statistics to `path` (unet_save); meta: a dict
        stored as JSON in the header."""
        import json
        m = json.dumps(meta or {}, sort_keys=True).encode()
        _check(self.lib.unet_save(self.handle, os.fsencode(path), m), "unet_save")

    def load(self, path):
        """Restore weights and BatchNorm statistics from `path` (unet_load); the file's
        configuration must equal this network's."""
        _check(self.lib.unet_load(self.handle, os.fsencode(path)), "unet_load")

    def adam_step(self, lr=1e-4, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        _check(self.lib.unet_adam_step(self.handle, lr, b1, b2, eps, _stream(stream)), "unet_adam_step")
