"""FP64 CPU oracle: Helmholtz operator, shifted-Laplacian V-cycle, GMRES, FGMRES.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the GPU path computes.  Only tests/, the smoke check and the
benchmark's CPU-baseline/reference legs may import it; the product path never
does, and it shares no code with the CUDA library.

All arithmetic is complex128 / float64.  Arrays are (..., ny, nx), row-major,
unknown (iy, ix) at node index (iy, ix); values outside the grid are zero
(zero padding of size 1 = Dirichlet, Sec. 2.4); Level.bc = "reflect" or "replicate"
pads the operator's stencil by reflection or replication instead (Neumann, Sec. 2.4),
while the transfer kernels of Eq. 2.9 keep their zero padding.

Readings of points the paper leaves open:
  * A = L - w^2 k^2 (1 - g i) with L the 5-point negative Laplacian (Eq. 2.1,
    2.2); the shifted Laplacian is M = L - w^2 k^2 (1 - (g + beta) i)
    (Eq. 2.4 with alpha = 1, the shift added to the attenuation).
  * Absorbing layer: g(d) = g_max (1 - d/W)^2 for d < W cells from the nearest
    edge (d = 0 on the outermost unknown), 0 inside; on level l the width is
    W >> l.
  * Coarse operators: rediscretisation on H = 2h with k^2 restricted by full
    weighting, renormalised by the in-domain weight sum.
  * Coarsest solve: GMRES(m) with x0 = 0, right-preconditioned by the
    diagonal (Jacobi) of the coarsest operator, exactly m Arnoldi steps (fewer
    only on breakdown), no relaxation on that level.
  * Prolongation: the transposed stride-2 convolution with output size n
    (Eq. 2.9), so that R = P^T / 4 exactly.
  * Neumann padding: "reflect" mirrors about the boundary node (ghost u_-1 = u_1),
    "replicate" copies it (ghost u_-1 = u_0); every level carries the mode.
  * Higher-order operator (Level.order = 4): the compact fourth-order 9-point
    scheme, K u = L9 u - (1/12) M5 (m u) with right-hand side (1/12) M5 f (derived
    with the definitions below), rediscretised on every level.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Eq. 2.9: full-weighting (restriction) and bilinear (prolongation) kernels.
K_RESTRICT = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], dtype=np.float64) / 16.0
K_PROLONG = np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], dtype=np.float64) / 4.0


# ----------------------------------------------------------------------------
# Medium, absorbing layer, levels
# ----------------------------------------------------------------------------
def abc_gamma(ny: int, nx: int, width: int, gamma_max: float = 1.0) -> np.ndarray:
    """Absorbing-layer attenuation g(x) (Eq. 2.1; the layer of Sec. 4)."""
    iy = np.arange(ny)[:, None]
    ix = np.arange(nx)[None, :]
    d = np.minimum(np.minimum(iy, ny - 1 - iy), np.minimum(ix, nx - 1 - ix)).astype(np.float64)
    g = np.zeros((ny, nx))
    if width > 0:
        inside = d < width
        g[inside] = gamma_max * (1.0 - d[inside] / width) ** 2
    return g


@dataclass
class Level:
    """One grid of the hierarchy: the data that define A or M on it."""
    ny: int
    nx: int
    h: float
    omega: float
    kappa2: np.ndarray          # (ny, nx) float64
    gamma: np.ndarray           # (ny, nx) float64
    beta: float = 0.0           # shift of the operator (0 -> A, 0.5 -> M)
    bc: str = "dirichlet"       # stencil padding: "dirichlet" (zero), "reflect" or "replicate"
    order: int = 2              # 2: 5-point stencil (Eq. 2.2); 4: compact 9-point scheme

    def with_shift(self, beta: float) -> "Level":
        return Level(self.ny, self.nx, self.h, self.omega, self.kappa2, self.gamma, beta, self.bc, self.order)


@dataclass
class Problem:
    """Fine-grid problem description (Sec. 2.1, 4): grid, frequency, medium, layer."""
    kappa2: np.ndarray
    omega: float
    h: float
    abc_width: int = 16
    gamma_max: float = 1.0
    beta: float = 0.5
    levels: int = 3
    nu1: int = 1
    nu2: int = 1
    jacobi_w: float = 0.8
    coarse_its: int = 10
    bc: str = "dirichlet"
    order: int = 2
    hierarchy: list = field(default_factory=list)

    def __post_init__(self):
        self.kappa2 = np.asarray(self.kappa2, dtype=np.float64)
        ny, nx = self.kappa2.shape
        k2 = self.kappa2
        for l in range(self.levels):
            if l > 0:
                k2 = coarsen_kappa2(k2)
            lny, lnx = ny >> l, nx >> l
            g = abc_gamma(lny, lnx, self.abc_width >> l, self.gamma_max)
            self.hierarchy.append(Level(lny, lnx, self.h * (1 << l), self.omega, k2, g, self.beta, self.bc,
                                        self.order))

    @property
    def A(self) -> Level:
        """The Helmholtz operator on the fine grid (no shift)."""
        return self.hierarchy[0].with_shift(0.0)

    @property
    def M(self) -> Level:
        """The shifted-Laplacian operator on the fine grid."""
        return self.hierarchy[0]


# ----------------------------------------------------------------------------
# Operators (Eq. 2.2, 2.4), Jacobi
# ----------------------------------------------------------------------------
def _center(lv: Level) -> np.ndarray:
    """Centre weight of the stencil: 4/h^2 - w^2 k^2 (1 - (g + beta) i)."""
    return 4.0 / lv.h ** 2 - lv.omega ** 2 * lv.kappa2 * (1.0 - (lv.gamma + lv.beta) * 1j)


def _ghost(i: int, n: int, bc: str):
    """Node whose value a neighbour index i outside 0..n-1 takes (None: zero), for the
    padding of the stencil's convolution (Sec. 2.4: zero padding = Dirichlet; reflection
    or replication padding = Neumann)."""
    if 0 <= i < n:
        return i
    if bc == "reflect":
        return 1 if i < 0 else n - 2
    if bc == "replicate":
        return 0 if i < 0 else n - 1
    return None


# Compact fourth-order scheme (the higher-order operators Sec. 2.4 says the convolution
# form carries over to).  For -Lap u = g the compact fourth-order difference is
#   (1/(6h^2)) [-1 -4 -1; -4 20 -4; -1 -4 -1] u = (1/12) [0 1 0; 1 8 1; 0 1 0] g,
# and the Helmholtz equation is that with g = f + m u, m = w^2 k^2 (1 - (g + beta) i):
#   K u = L9 u - (1/12) M5 (m u),   right-hand side (1/12) M5 f.
LAP9 = np.array([[-1.0, -4.0, -1.0], [-4.0, 20.0, -4.0], [-1.0, -4.0, -1.0]]) / 6.0   # times 1/h^2
MASS5 = np.array([[0.0, 1.0, 0.0], [1.0, 8.0, 1.0], [0.0, 1.0, 0.0]]) / 12.0


def _mass(lv: Level) -> np.ndarray:
    """m = w^2 k^2 (1 - (g + beta) i), the mass term of Eq. 2.2 / 2.4."""
    return lv.omega ** 2 * lv.kappa2 * (1.0 - (lv.gamma + lv.beta) * 1j)


def _pad(lv: Level, u: np.ndarray) -> np.ndarray:
    mode = {"dirichlet": "constant", "reflect": "reflect", "replicate": "edge"}[lv.bc]
    return np.pad(u, [(0, 0)] * (u.ndim - 2) + [(1, 1), (1, 1)], mode=mode)


def _conv3(p: np.ndarray, w: np.ndarray) -> np.ndarray:
    """sum_{a,b} w[a+1, b+1] p(i+a, j+b) over the interior of a 1-padded array."""
    ny, nx = p.shape[-2] - 2, p.shape[-1] - 2
    out = np.zeros(p.shape[:-2] + (ny, nx), dtype=p.dtype)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            if w[a + 1, b + 1] != 0.0:
                out += w[a + 1, b + 1] * p[..., 1 + a:1 + a + ny, 1 + b:1 + b + nx]
    return out


def _apply_compact4(lv: Level, u: np.ndarray) -> np.ndarray:
    return _conv3(_pad(lv, u), LAP9) / lv.h ** 2 - _conv3(_pad(lv, _mass(lv) * u), MASS5)


def rhs_weight(lv: Level, f: np.ndarray) -> np.ndarray:
    """Right-hand side of the discrete equation for a source f: f itself for the 5-point
    scheme, (1/12) M5 f for the compact fourth-order one."""
    return f if lv.order == 2 else _conv3(_pad(lv, f), MASS5)


def _diagonal_compact4(lv: Level) -> np.ndarray:
    """Diagonal of the compact operator: every stencil entry whose (padded) neighbour is
    the node itself (the centre; also folded ghosts under replication)."""
    m = _mass(lv)
    d = np.zeros((lv.ny, lv.nx), dtype=np.complex128)
    iy = np.arange(lv.ny)[:, None]
    ix = np.arange(lv.nx)[None, :]
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            gy = np.array([_ghost(i + a, lv.ny, lv.bc) for i in range(lv.ny)], dtype=object)[:, None]
            gx = np.array([_ghost(j + b, lv.nx, lv.bc) for j in range(lv.nx)], dtype=object)[None, :]
            self_ = (gy == iy) & (gx == ix)
            d = d + self_ * (LAP9[a + 1, b + 1] / lv.h ** 2 - MASS5[a + 1, b + 1] * m)
    return d


def diagonal(lv: Level) -> np.ndarray:
    """Diagonal of the operator: the centre weight, less 1/h^2 for every neighbour that
    replication padding maps back onto the node itself."""
    if lv.order == 4:
        return _diagonal_compact4(lv)
    d = _center(lv)
    if lv.bc == "replicate":
        iy = np.arange(lv.ny)[:, None]
        ix = np.arange(lv.nx)[None, :]
        edges = (iy == 0).astype(float) + (iy == lv.ny - 1) + (ix == 0) + (ix == lv.nx - 1)
        d = d - edges / lv.h ** 2
    return d


def apply_op(lv: Level, u: np.ndarray) -> np.ndarray:
    """y = K u for the 5-point stencil of Eq. 2.2 (with shift beta), or the compact
    fourth-order scheme when lv.order == 4; neighbours outside the grid are zero
    (Dirichlet) or taken by reflection / replication (Neumann)."""
    if lv.order == 4:
        return _apply_compact4(lv, u)
    if lv.bc == "dirichlet":
        up = np.zeros_like(u)
        up[..., 1:, :] += u[..., :-1, :]
        up[..., :-1, :] += u[..., 1:, :]
        up[..., :, 1:] += u[..., :, :-1]
        up[..., :, :-1] += u[..., :, 1:]
    else:
        mode = {"reflect": "reflect", "replicate": "edge"}[lv.bc]
        pw = [(0, 0)] * (u.ndim - 2) + [(1, 1), (1, 1)]
        p = np.pad(u, pw, mode=mode)
        up = p[..., :-2, 1:-1] + p[..., 2:, 1:-1] + p[..., 1:-1, :-2] + p[..., 1:-1, 2:]
    return _center(lv) * u - up / lv.h ** 2


def apply_op_T(lv: Level, u: np.ndarray) -> np.ndarray:
    """y = K^T u.  K = C - (1/h^2) S P, with P the padding (grid -> grid plus one ghost
    layer), S the sum of the four neighbours read from the padded array and C the centre
    weight, so K^T = C - (1/h^2) P^T S^T: scatter every value to its four neighbours on
    the padded array, then fold each ghost back onto the node it copies.  Zero padding
    and replication give a symmetric K; reflection does not."""
    if lv.order != 2:
        raise NotImplementedError("transpose of the compact fourth-order operator")
    if lv.bc == "dirichlet":
        return apply_op(lv, u)
    ny, nx = u.shape[-2:]
    q = np.zeros(u.shape[:-2] + (ny + 2, nx + 2), dtype=np.result_type(u, np.complex128))
    q[..., 0:ny, 1:-1] += u        # value at node (i, j) -> padded (i - 1, j)
    q[..., 2:, 1:-1] += u          #                      -> padded (i + 1, j)
    q[..., 1:-1, 0:nx] += u
    q[..., 1:-1, 2:] += u
    src_lo, src_hi = (1, -2) if lv.bc == "reflect" else (0, -1)   # node a ghost copies
    t = q[..., :, 1:-1].copy()     # fold the ghost columns (padded 0 and nx + 1)
    t[..., :, src_lo] += q[..., :, 0]
    t[..., :, src_hi] += q[..., :, -1]
    s = t[..., 1:-1, :].copy()     # fold the ghost rows
    s[..., src_lo, :] += t[..., 0, :]
    s[..., src_hi, :] += t[..., -1, :]
    return _center(lv) * u - s / lv.h ** 2


def residual(lv: Level, f: np.ndarray, u: np.ndarray) -> np.ndarray:
    return f - apply_op(lv, u)


def jacobi(lv: Level, u: np.ndarray, f: np.ndarray, w: float) -> np.ndarray:
    """One damped Jacobi sweep: u + w D^-1 (f - K u)."""
    return u + w * (f - apply_op(lv, u)) / diagonal(lv)


def assemble_dense(lv: Level) -> np.ndarray:
    """Dense matrix of the operator, assembled node by node from the stencil (Eq. 2.2,
    or the compact fourth-order scheme), ghost neighbours mapped to the nodes they copy."""
    ny, nx = lv.ny, lv.nx
    n = ny * nx
    K = np.zeros((n, n), dtype=np.complex128)
    if lv.order == 4:
        m = _mass(lv)
        for iy in range(ny):
            for ix in range(nx):
                p = iy * nx + ix
                for a in (-1, 0, 1):
                    for b in (-1, 0, 1):
                        gy, gx = _ghost(iy + a, ny, lv.bc), _ghost(ix + b, nx, lv.bc)
                        if gy is None or gx is None:
                            continue
                        K[p, gy * nx + gx] += LAP9[a + 1, b + 1] / lv.h ** 2 - MASS5[a + 1, b + 1] * m[gy, gx]
        return K
    c = _center(lv)
    off = -1.0 / lv.h ** 2
    for iy in range(ny):
        for ix in range(nx):
            p = iy * nx + ix
            K[p, p] += c[iy, ix]
            for dy, dx in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                jy, jx = iy + dy, ix + dx
                if 0 <= jy < ny and 0 <= jx < nx:
                    K[p, jy * nx + jx] += off
                    continue
                gy, gx = _ghost(jy, ny, lv.bc), _ghost(jx, nx, lv.bc)
                if gy is not None and gx is not None:
                    K[p, gy * nx + gx] += off
    return K


# ----------------------------------------------------------------------------
# Transfer operators (Eq. 2.9): stride-2 convolution, zero padding 1
# ----------------------------------------------------------------------------
def restrict_fw(r: np.ndarray) -> np.ndarray:
    """Full weighting: r_H(I,J) = sum_{a,b} K_R[a,b] r_h(2I+a, 2J+b), a,b in {-1,0,1}."""
    ny, nx = r.shape[-2:]
    pad = np.zeros(r.shape[:-2] + (ny + 2, nx + 2), dtype=r.dtype)
    pad[..., 1:-1, 1:-1] = r
    out = np.zeros(r.shape[:-2] + (ny // 2, nx // 2), dtype=r.dtype)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            out += K_RESTRICT[a + 1, b + 1] * pad[..., 1 + a:1 + a + ny - 1:2, 1 + b:1 + b + nx - 1:2]
    return out


def prolong_bilinear(e: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Bilinear prolongation as the transposed stride-2 convolution (output ny x nx):
    out(2I+a, 2J+b) += K_P[a,b] e(I,J), contributions landing outside dropped."""
    nY, nX = e.shape[-2:]
    pad = np.zeros(e.shape[:-2] + (ny + 2, nx + 2), dtype=e.dtype)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            pad[..., 1 + a:1 + a + 2 * nY:2, 1 + b:1 + b + 2 * nX:2] += K_PROLONG[a + 1, b + 1] * e
    return pad[..., 1:ny + 1, 1:nx + 1]


def coarsen_kappa2(k2: np.ndarray) -> np.ndarray:
    """Coarse-grid medium: full weighting of k^2 divided by the in-domain weight sum."""
    return restrict_fw(k2) / restrict_fw(np.ones_like(k2))


# ----------------------------------------------------------------------------
# Givens rotations and small least squares (used by GMRES and FGMRES)
# ----------------------------------------------------------------------------
def givens(a: complex, b: complex):
    """Rotation (c real, s complex) with [c s; -conj(s) c] [a; b] = [r; 0]."""
    if b == 0:
        return 1.0, 0.0j, a
    if a == 0:
        return 0.0, 1.0 + 0.0j, b
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    phase = a / abs(a)
    s = phase * np.conj(b) / t
    return c, s, phase * t


def back_substitute(R: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Solve the k x k upper triangular system R y = g."""
    k = R.shape[0]
    y = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:k] @ y[i + 1:k]) / R[i, i]
    return y


class ArnoldiLS:
    """Hessenberg least-squares state updated column by column with Givens rotations."""

    def __init__(self, m: int, beta: float):
        self.H = np.zeros((m + 1, m), dtype=np.complex128)    # rotated (upper triangular part)
        self.Hraw = np.zeros((m + 1, m), dtype=np.complex128)  # the Arnoldi Hessenberg itself
        self.cs = np.zeros(m)
        self.sn = np.zeros(m, dtype=np.complex128)
        self.g = np.zeros(m + 1, dtype=np.complex128)
        self.g[0] = beta
        self.k = 0

    def add_column(self, h: np.ndarray) -> float:
        """Append Hessenberg column j (length j+2); return the residual estimate |g_{j+1}|."""
        j = self.k
        self.Hraw[:j + 2, j] = h
        col = h.astype(np.complex128).copy()
        for i in range(j):
            c, s = self.cs[i], self.sn[i]
            t = c * col[i] + s * col[i + 1]
            col[i + 1] = -np.conj(s) * col[i] + c * col[i + 1]
            col[i] = t
        c, s, r = givens(col[j], col[j + 1])
        self.cs[j], self.sn[j] = c, s
        col[j], col[j + 1] = r, 0.0
        self.H[:j + 2, j] = col
        self.g[j + 1] = -np.conj(s) * self.g[j]
        self.g[j] = c * self.g[j]
        self.k = j + 1
        return abs(self.g[j + 1])

    def solve(self) -> np.ndarray:
        k = self.k
        return back_substitute(self.H[:k, :k], self.g[:k])


def _dot(u: np.ndarray, v: np.ndarray) -> complex:
    """<u, v> = u^H v."""
    return complex(np.vdot(u.ravel(), v.ravel()))


def _norm(u: np.ndarray) -> float:
    return float(np.sqrt(np.vdot(u.ravel(), u.ravel()).real))


# ----------------------------------------------------------------------------
# Coarsest-grid GMRES(m) with diagonal right preconditioning (Sec. 2.4, 4)
# ----------------------------------------------------------------------------
def gmres_jacobi(lv: Level, f: np.ndarray, m: int = 10, breakdown: float = 0.0) -> np.ndarray:
    """m steps of GMRES on K D^-1 y = f from y0 = 0, x = D^-1 y (single right-hand side)."""
    dinv = 1.0 / diagonal(lv)
    beta = _norm(f)
    if beta == 0.0:
        return np.zeros_like(f)
    V = [f / beta]
    ls = ArnoldiLS(m, beta)
    for j in range(m):
        w = apply_op(lv, dinv * V[j])
        h = np.zeros(j + 2, dtype=np.complex128)
        for i in range(j + 1):                 # modified Gram-Schmidt
            h[i] = _dot(V[i], w)
            w = w - h[i] * V[i]
        h[j + 1] = _norm(w)
        ls.add_column(h)
        if h[j + 1].real <= breakdown * beta:  # happy breakdown: the space is invariant
            break
        V.append(w / h[j + 1].real)
    y = ls.solve()
    u = np.zeros_like(f)
    for i in range(ls.k):
        u = u + y[i] * V[i]
    return dinv * u


def coarse_direct(lv: Level, f: np.ndarray) -> np.ndarray:
    """Exact coarsest solve by the oracle's own dense LU (test mode of Alg. 1)."""
    K = assemble_dense(lv)
    return lu_solve(K, f.ravel()).reshape(f.shape)


# ----------------------------------------------------------------------------
# V-cycle (Alg. 1) on the shifted Laplacian hierarchy
# ----------------------------------------------------------------------------
def vcycle(prob: Problem, f: np.ndarray, v: np.ndarray | None = None, level: int = 0,
           coarse: str = "gmres") -> np.ndarray:
    """v <- V-cycle(v, f) for one right-hand side (ny, nx), Alg. 1 with nu1/nu2 damped
    Jacobi sweeps, full weighting, bilinear prolongation, recursion to the coarsest level."""
    lv = prob.hierarchy[level]
    if v is None:
        v = np.zeros_like(f)
    if level == len(prob.hierarchy) - 1:
        if coarse == "direct":
            return coarse_direct(lv, f)
        return gmres_jacobi(lv, f, prob.coarse_its)
    for _ in range(prob.nu1):
        v = jacobi(lv, v, f, prob.jacobi_w)
    fc = restrict_fw(residual(lv, f, v))
    vc = vcycle(prob, fc, None, level + 1, coarse)
    v = v + prolong_bilinear(vc, lv.ny, lv.nx)
    for _ in range(prob.nu2):
        v = jacobi(lv, v, f, prob.jacobi_w)
    return v


def precond_v(prob: Problem):
    """M_V: one SL V-cycle from a zero guess (Sec. 4)."""
    return lambda r: vcycle(prob, r)


# ----------------------------------------------------------------------------
# Restarted flexible GMRES(m), right preconditioned (Eq. 2.5; Saad 1993)
# ----------------------------------------------------------------------------
@dataclass
class FgmresResult:
    x: np.ndarray
    iters: int
    relres: float               # final true relative residual ||b - A x|| / ||b||
    converged: bool
    history: list               # (iteration, relative residual estimate) per step
    true_history: list          # true relative residual at each restart


def fgmres(A: Level, precond, b: np.ndarray, x0: np.ndarray | None = None, m: int = 10,
           tol: float = 1e-7, maxit: int = 2000) -> FgmresResult:
    """Solve A x = b (one right-hand side) with restarted FGMRES(m).

    Each cycle starts from the true residual r = b - A x; Arnoldi uses modified
    Gram-Schmidt on w = A z_j with z_j = precond(v_j); the cycle ends after m
    steps or when the Givens residual estimate drops to tol*||b||; then
    x += Z y.  Converged when the true relative residual is <= tol."""
    x = np.zeros_like(b) if x0 is None else x0.astype(np.complex128).copy()
    bnorm = _norm(b)
    if bnorm == 0.0:
        return FgmresResult(np.zeros_like(b), 0, 0.0, True, [], [0.0])
    iters = 0
    history, true_history = [], []
    while True:
        r = b - apply_op(A, x)
        beta = _norm(r)
        true_history.append(beta / bnorm)
        if beta / bnorm <= tol:
            return FgmresResult(x, iters, beta / bnorm, True, history, true_history)
        if iters >= maxit:
            return FgmresResult(x, iters, beta / bnorm, False, history, true_history)
        V = [r / beta]
        Z = []
        ls = ArnoldiLS(m, beta)
        for j in range(m):
            z = precond(V[j])
            Z.append(z)
            w = apply_op(A, z)
            h = np.zeros(j + 2, dtype=np.complex128)
            for i in range(j + 1):
                h[i] = _dot(V[i], w)
                w = w - h[i] * V[i]
            h[j + 1] = _norm(w)
            est = ls.add_column(h)
            iters += 1
            history.append((iters, est / bnorm))
            if est / bnorm <= tol or h[j + 1].real == 0.0 or iters >= maxit:
                break
            V.append(w / h[j + 1].real)
        y = ls.solve()
        for i in range(ls.k):
            x = x + y[i] * Z[i]


@dataclass
class BlockFgmresResult:
    X: np.ndarray               # (p, ny, nx) solutions
    iters: int                  # block iterations (each applies the preconditioner to p vectors)
    relres: np.ndarray          # (p,) final true relative residuals
    converged: bool
    true_history: list          # largest true relative residual at each restart
    estimates: list             # per block iteration: the p least-squares residual estimates / ||b_k||


def block_fgmres(A: Level, precond, B: np.ndarray, X0: np.ndarray | None = None, m: int = 10,
                 tol: float = 1e-7, maxit: int = 2000) -> BlockFgmresResult:
    """Block flexible GMRES(m) for the p right-hand sides B (p, ny, nx): one block
    Krylov space shared by all of them (the CPU solver of Sec. 4, after Calandra et al.).

    Each cycle: R = B - A X = V_1 S (thin QR); for j = 1..m: Z_j = precond(V_j), column
    by column; W = A Z_j; block modified Gram-Schmidt H_ij = V_i^H W, W -= V_i H_ij
    (i = 1..j); thin QR W = V_{j+1} H_{j+1,j}.  The least-squares problem
    min_Y ||E_1 S - Hbar_j Y||_F gives each column's residual estimate; the cycle ends
    after m block steps or when every estimate is <= tol ||b_k||; then X += [Z_1..Z_j] Y.
    Converged when every true relative residual is <= tol."""
    p = B.shape[0]
    shape = B.shape[1:]
    n = int(np.prod(shape))
    X = np.zeros_like(B, dtype=np.complex128) if X0 is None else X0.astype(np.complex128).copy()
    bn = np.array([_norm(B[k]) for k in range(p)])
    bn[bn == 0.0] = 1.0
    iters = 0
    true_history, estimates = [], []
    while True:
        R = B - apply_op(A, X)
        rr = np.array([_norm(R[k]) for k in range(p)]) / bn
        true_history.append(float(rr.max()))
        if rr.max() <= tol:
            return BlockFgmresResult(X, iters, rr, True, true_history, estimates)
        if iters >= maxit:
            return BlockFgmresResult(X, iters, rr, False, true_history, estimates)
        V1, S = np.linalg.qr(R.reshape(p, n).T)
        Vs, Zs = [V1], []
        Hbar = np.zeros(((m + 1) * p, m * p), dtype=np.complex128)
        Y = None
        for j in range(m):
            Zj = np.stack([precond(Vs[j][:, c].reshape(shape)).ravel() for c in range(p)], axis=1)
            Zs.append(Zj)
            W = np.stack([apply_op(A, Zj[:, c].reshape(shape)).ravel() for c in range(p)], axis=1)
            for i in range(j + 1):
                Hij = Vs[i].conj().T @ W
                W = W - Vs[i] @ Hij
                Hbar[i * p:(i + 1) * p, j * p:(j + 1) * p] = Hij
            Vn, Hn = np.linalg.qr(W)
            Hbar[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = Hn
            iters += 1
            k = j + 1
            E = np.zeros(((k + 1) * p, p), dtype=np.complex128)
            E[:p] = S
            Hk = Hbar[:(k + 1) * p, :k * p]
            Y = np.linalg.lstsq(Hk, E, rcond=None)[0]
            est = np.linalg.norm(E - Hk @ Y, axis=0) / bn
            estimates.append(est)
            if est.max() <= tol or iters >= maxit:
                break
            Vs.append(Vn)
        X = X + (np.concatenate(Zs, axis=1) @ Y).T.reshape(p, *shape)


def convergence_factor(history_true0: float, final: float, iters: int) -> float:
    """Eq. 4.1: rho = (||r_T|| / ||r_0||)^(1/T)."""
    if iters <= 0:
        return 0.0
    return (final / history_true0) ** (1.0 / iters)


# ----------------------------------------------------------------------------
# Dense LU with partial pivoting (test-mode coarse solve and the 16x16 pin)
# ----------------------------------------------------------------------------
def lu_solve(K: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Gaussian elimination with row partial pivoting, then two triangular solves."""
    a = np.array(K, dtype=np.complex128)
    n = a.shape[0]
    piv = np.arange(n)
    for k in range(n - 1):
        p = k + int(np.argmax(np.abs(a[k:, k])))
        if p != k:
            a[[k, p]] = a[[p, k]]
            piv[[k, p]] = piv[[p, k]]
        a[k + 1:, k] /= a[k, k]
        a[k + 1:, k + 1:] -= np.outer(a[k + 1:, k], a[k, k + 1:])
    y = np.array(f, dtype=np.complex128)[piv]
    for i in range(n):                       # L y = P f (unit lower)
        y[i] -= a[i, :i] @ y[:i]
    x = np.zeros(n, dtype=np.complex128)
    for i in range(n - 1, -1, -1):           # U x = y
        x[i] = (y[i] - a[i, i + 1:] @ x[i + 1:]) / a[i, i]
    return x
