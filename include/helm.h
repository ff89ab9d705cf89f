/*
 * libhelm — preconditioned Krylov solver for the 2D heterogeneous Helmholtz
 * equation on one GB300 GPU (sm_103a), after Azulay & Treister,
 * "Multigrid-augmented deep learning preconditioners for the Helmholtz
 * equation" (arXiv 2203.11025).
 *
 *   -Lap u - w^2 k(x)^2 (1 - g(x) i) u = f    on [0,1]^2        (Eq. 2.1)
 *
 * discretised by the 5-point stencil of Eq. 2.2 on an nx-by-ny grid of
 * unknowns with spacing h and zero (Dirichlet) values outside the grid; g is
 * an absorbing layer (quadratic profile, width abc_width cells, peak
 * abc_gamma_max).  The shifted Laplacian M replaces (1 - g i) by
 * (1 - (g + beta) i) (Eq. 2.4, alpha = 1).  helm_desc.bc selects Neumann
 * boundaries by reflection or replication padding instead, and
 * helm_desc.stencil the compact fourth-order 9-point scheme (Sec. 2.4).
 *
 * Conventions for every entry point
 *   - Vectors are complex, interleaved (re, im), row-major [rhs][y][x];
 *     dtype HELM_C32 = float2 elements, HELM_C64 = double2 elements.
 *   - Pointers are DEVICE pointers owned by the caller unless a flag says
 *     otherwise; the library never frees them.  kappa2 is float32 [y][x].
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued on it; calls return without synchronising except where noted.
 *   - Return value: 0 (HELM_OK) on success, > 0 a non-fatal outcome, < 0 an
 *     error; helm_last_error() gives a message (thread-local).  No exception
 *     crosses this boundary.  On error nothing is guaranteed about outputs.
 *   - Grid sizes: nx and ny divisible by 2^(levels-1).
 */
#ifndef HELM_H
#define HELM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct helm_ctx* helm_t;
typedef void* helm_stream_t;

enum {
  HELM_OK = 0,
  HELM_MAXIT = 1,          /* FGMRES stopped at maxit before reaching tol      */
  HELM_EINVAL = -1,        /* bad argument                                     */
  HELM_ECUDA = -2,         /* a CUDA call failed (message has the CUDA error)  */
  HELM_ENAN = -3,          /* a non-finite residual was met                    */
  HELM_ENOMEM = -5,        /* device allocation failed                         */
  HELM_EUNSUPPORTED = -6   /* feature not built for this configuration         */
};
enum { HELM_OP_A = 0, HELM_OP_M = 1,        /* Helmholtz A (Eq. 2.2) / shifted M (Eq. 2.4) */
       HELM_OP_RHS = 2 };                    /* right-hand side of a source (helm_apply only) */
enum { HELM_C32 = 0, HELM_C64 = 1 };
enum { HELM_PREC_NONE = 0, HELM_PREC_V = 1, HELM_PREC_JU = 2, HELM_PREC_VU = 3 };

/* Problem and multigrid description (Sec. 2.1, 2.2, 4). */
typedef struct {
  int nx, ny;              /* unknowns per row / per column                    */
  double h;                /* mesh width                                       */
  double omega;            /* angular frequency                                */
  double beta;             /* SL shift (Sec. 4: 0.5)                           */
  int abc_width;           /* absorbing layer width in fine cells (>= 0)       */
  double abc_gamma_max;    /* layer attenuation on the outermost unknowns      */
  int levels;              /* V-cycle levels incl. the coarsest (Sec. 4: 3)    */
  int nu1, nu2;            /* pre/post damped-Jacobi sweeps (Sec. 4: 1, 1)     */
  double jacobi_w;         /* Jacobi damping (Sec. 4: 0.8)                     */
  int coarse_its;          /* GMRES steps on the coarsest grid (Sec. 4: 10)   */
  int flags;               /* HELM_DESC_* implementation switches (0 = default) */
  int bc;                  /* HELM_BC_* boundary condition (0 = Dirichlet)     */
  int stencil;             /* HELM_STENCIL_* discretisation (0 = 5-point)      */
} helm_desc;
/* Discretisations.  5PT is Eq. 2.2.  COMPACT4 is the compact fourth-order 9-point
 * scheme, one of the higher-order operators that Sec. 2.4 says the convolution form
 * admits: with m = w^2 k^2 (1 - (g + beta) i),
 *   K u = (1/(6h^2)) [-1 -4 -1; -4 20 -4; -1 -4 -1] u - (1/12) [0 1 0; 1 8 1; 0 1 0] (m u),
 * and the discrete equation for a source f is K u = (1/12) [0 1 0; 1 8 1; 0 1 0] f
 * (helm_apply with HELM_OP_RHS computes that right-hand side).  Every level
 * rediscretises with the same scheme.  COMPACT4 needs HELM_BC_DIRICHLET. */
enum { HELM_STENCIL_5PT = 0, HELM_STENCIL_COMPACT4 = 1 };
/* Boundary conditions (Sec. 2.4: the 5-point stencil applied as a convolution,
 * whose padding sets the boundary).  DIRICHLET pads with zeros; REFLECT mirrors
 * about the boundary node (ghost u_-1 = u_1) and REPLICATE copies it (ghost
 * u_-1 = u_0), both Neumann conditions.  The mode holds on every level of the
 * hierarchy; the transfer operators of Eq. 2.9 keep zero padding.  REFLECT
 * needs every level at least 2 nodes wide in each direction. */
enum { HELM_BC_DIRICHLET = 0, HELM_BC_REFLECT = 1, HELM_BC_REPLICATE = 2 };
/* Coarsest-GMRES implementation switches (default: a thread-block cluster per
 * right-hand side with the Krylov basis in distributed shared memory when the
 * grid fits, else one CTA per right-hand side when the grid fits in one CTA's
 * shared memory, else one launch per Arnoldi pass); for cross-checking. */
enum { HELM_DESC_MULTIKERNEL_COARSE = 1, HELM_DESC_SINGLE_CTA_COARSE = 2 };

/* Fill `d` with the paper's defaults (Sec. 4) for an n-by-n grid, h = 1/n,
 * omega from max(omega k h) = 2 pi / 10 with max k = 1 (Sec. 2.1), a 16-cell
 * quadratic layer with peak 1.  Returns HELM_EINVAL if d is NULL. */
int helm_desc_default(helm_desc* d, int nx, int ny);

/* Build the level hierarchy: copies kappa2 (device, float32 [ny][nx]) and
 * derives coarse media by full weighting renormalised at the edges
 * (rediscretisation on H = 2h, Sec. 2.2).  Synchronises `stream` before
 * returning.  The handle owns all workspace; free it with helm_destroy. */
int helm_setup(const helm_desc* desc, const float* kappa2, helm_stream_t stream, helm_t* out);
void helm_destroy(helm_t h);
const char* helm_last_error(void);

/* A batch of problems of one grid size, each with its own medium (Sec. 4 solves problems
 * on many random media; no counterpart for the batching itself): kappa2 is device float32
 * [nmedia][ny][nx], and right-hand side r of every call on the handle is solved on medium
 * r / rpp (callers order right-hand sides by medium, rpp of them per medium; at most
 * nmedia * rpp per call).  The level hierarchy holds every medium's coarse media, and every
 * operator kernel picks each right-hand side's medium, so one launch per level serves the
 * whole batch.  helm_setup is helm_setup_media with one medium (rpp ignored).  Block FGMRES,
 * the pair generator, training and the encoder-solver pair need a handle of one medium
 * (HELM_EUNSUPPORTED). */
int helm_setup_media(const helm_desc* desc, const float* kappa2, int nmedia, int rpp, helm_stream_t stream,
                     helm_t* out);

/* Level sizes of the multigrid hierarchy (Sec. 2.2: H = 2h per level; level 0 = fine grid).
 * HELM_EINVAL for a level outside 0..levels-1. */
int helm_level_shape(helm_t h, int level, int* nx, int* ny);
/* Copy the level's kappa^2 (the rediscretised medium of Sec. 2.2; float64, [ny][nx]) into
 * a caller-owned device buffer. */
int helm_level_kappa2(helm_t h, int level, double* out);

/* y = K x on `level`, K = A (op HELM_OP_A) or M (HELM_OP_M), Eq. 2.2 / 2.4; with
 * op HELM_OP_RHS, y = the discrete right-hand side of the source x (x itself for the
 * 5-point stencil, (1/12) [0 1 0; 1 8 1; 0 1 0] x for COMPACT4).  y must not alias x
 * (HELM_EINVAL).  An op outside these is HELM_EINVAL (helm_residual and helm_jacobi
 * take A or M). */
int helm_apply(helm_t h, int op, int level, const void* x, void* y, int nrhs, int dtype, helm_stream_t stream);
/* r = b - K x (Eq. 2.2 / 2.4; op HELM_OP_A or HELM_OP_M); r must not alias b or x
 * (HELM_EINVAL). */
int helm_residual(helm_t h, int op, int level, const void* b, const void* x, void* r, int nrhs, int dtype,
                  helm_stream_t stream);
/* One damped Jacobi sweep x_out = x_in + w D^-1 (b - K x_in) (Sec. 4, w = desc.jacobi_w);
 * x_in NULL means a zero guess.  x_out must not alias x_in. */
int helm_jacobi(helm_t h, int op, int level, const void* b, const void* x_in, void* x_out, int nrhs, int dtype,
                helm_stream_t stream);
/* Full-weighting restriction (Eq. 2.9) from `level` to level+1. */
int helm_restrict(helm_t h, int level, const void* fine, void* coarse, int nrhs, int dtype, helm_stream_t stream);
/* fine += P coarse: bilinear prolongation (Eq. 2.9, transposed stride-2 conv) from level+1 to `level`. */
int helm_prolong_add(helm_t h, int level, const void* coarse, void* fine, int nrhs, int dtype,
                     helm_stream_t stream);
/* Coarsest-grid solve: desc.coarse_its GMRES steps with diagonal (Jacobi)
 * right preconditioning from x = 0 on M of the coarsest level (Sec. 2.4, 4). */
int helm_coarse_solve(helm_t h, const void* f, void* x, int nrhs, int dtype, helm_stream_t stream);

/* One shifted-Laplacian V-cycle on M (Alg. 1): x <- V-cycle(x, f) with nu1/nu2
 * damped-Jacobi sweeps, full weighting, bilinear prolongation and the coarsest
 * GMRES solve.  x_is_zero != 0 ignores the content of x (zero guess, as in M_V).
 * f and x must not alias. */
int sl_vcycle(helm_t h, const void* f, void* x, int nrhs, int dtype, int x_is_zero, helm_stream_t stream);

/* Restarted flexible GMRES (Sec. 2.2 and 4: FGMRES(m), right preconditioned,
 * Eq. 2.5), one independent Krylov process per right-hand side. */
enum {
  HELM_FLAG_X0_ZERO = 1,   /* start from x = 0 (x content ignored)              */
  HELM_FLAG_HOST_IO = 2,   /* b and x are HOST pointers (copied in and out)      */
  HELM_FLAG_NO_GRAPH = 4,  /* launch kernels directly instead of a CUDA graph    */
  HELM_FLAG_FP64 = 8,      /* FP64 Krylov vectors and preconditioner (checking)  */
  HELM_FLAG_FALLBACK_V = 16 /* U-Net preconditioners (fgmres_solve only): every
                              right-hand side that ends above tol (the iteration
                              cap, or a non-finite residual) is solved again with
                              plain M_V, from its iterate (from zero if that is
                              not finite), with the same restart, tol and maxit */
};
typedef struct {
  int restart;             /* m (Sec. 4: 10), 1..32                             */
  double tol;              /* stop when ||b - A x|| / ||b|| <= tol in FP64       */
  int maxit;               /* cap on inner iterations per right-hand side        */
  int flags;               /* HELM_FLAG_*                                        */
} fgmres_opts;
typedef struct {
  int iters_max;           /* iterations of the slowest right-hand side          */
  int cycles;              /* restart cycles run                                 */
  double relres_max;       /* max over right-hand sides of the FP64 true relres  */
  int status;              /* HELM_OK, HELM_MAXIT or HELM_ENAN                   */
  int* iters;              /* optional host array [nrhs], may be NULL            */
  double* relres;          /* optional host array [nrhs], may be NULL            */
  long long launches;      /* kernels this library launched for the solve (-1 if
                              not counted: HELM_FLAG_NO_GRAPH)                  */
  int fallbacks;           /* right-hand sides re-solved with M_V under
                              HELM_FLAG_FALLBACK_V (their iters count both
                              solves; relres and status are the M_V solve's)    */
} fgmres_result;

/* Solve A x = b (Eq. 2.5, FGMRES(m) of Sec. 2.2 and 4) for nrhs right-hand sides, each
 * with its own Krylov space.  b, x: complex FP64 ([rhs][y][x]),
 * device pointers unless HELM_FLAG_HOST_IO.  x holds x0 on entry (unless
 * HELM_FLAG_X0_ZERO) and the solution on return.  precond: HELM_PREC_V
 * (one SL V-cycle, M_V), HELM_PREC_NONE, or a U-Net preconditioner (needs
 * `net`, see unet.h).  Blocks the calling thread until the solve ends
 * (the host reads a convergence flag once per restart). */
int fgmres_solve(helm_t h, int precond, void* net, const void* b, void* x, int nrhs, const fgmres_opts* opts,
                 fgmres_result* result, helm_stream_t stream);

/* Problems of uneven grid sizes in one call (no counterpart in the paper): nh handles, one
 * per grid size (each may hold many media, helm_setup_media), with right-hand sides b[i] and
 * solutions x[i] (device, complex FP64, nrhs[i] each).  Each handle's restart cycle is one
 * CUDA graph on the handle's own stream; the calling thread interleaves the handles, so the
 * size classes run concurrently on the GPU.  U-Net preconditioners take one network handle
 * per solver handle in nets[i] (a network keeps one activation workspace per grid; copy the
 * weights with unet_get_params / unet_set_params or unet_save / unet_load); nets may be NULL
 * for HELM_PREC_V / NONE.  opts as for fgmres_solve without HOST_IO, FP64, FALLBACK_V or
 * NO_GRAPH (HELM_EUNSUPPORTED).  results: nh entries or NULL.  Returns the worst status.
 * Blocks the calling thread until every handle is done. */
int fgmres_solve_batch(int nh, helm_t* handles, int precond, void* const* nets, const void* const* b, void* const* x,
                       const int* nrhs, const fgmres_opts* opts, fgmres_result* results, helm_stream_t stream);

/* Block flexible GMRES(m) (the CPU solver of Sec. 4): one block Krylov space for all
 * nrhs right-hand sides (block size p = nrhs <= 16, (restart + 1) p^2 <= 4608).  Each
 * cycle: R = b - A x in FP64 = V_1 S; per block step Z_j = M(V_j) on the p vectors,
 * W = A Z_j, block classical Gram-Schmidt applied twice against V_1..V_j, W = V_{j+1}
 * H_{j+1,j} by Cholesky QR applied twice; the least-squares problem runs on the host in
 * FP64 and ends the cycle when every right-hand side's estimate is <= tol (or after
 * `restart` block steps); then x += Z Y.  Same arguments, flags and results as
 * fgmres_solve; iterations are block iterations (equal for every right-hand side), and
 * result->launches is -1.  Synchronises with the host at every block step. */
int bfgmres_solve(helm_t h, int precond, void* net, const void* b, void* x, int nrhs, const fgmres_opts* opts,
                  fgmres_result* result, helm_stream_t stream);

/* Measurement hook (no counterpart in the paper): launch one of the solver's
 * internal kernels `reps` times back to back on `stream` over the FP32
 * workspace of nrhs right-hand sides (fine grid) and return the mean device
 * time per launch in *ms (CUDA events on `stream`) and the kernel's
 * algorithmic bytes per launch in *bytes.  Workspace contents are overwritten.
 *   kernel 0: operator apply y = A x            (20 B per point)
 *   kernel 1: fused residual + full weighting   (8+4 B read per fine point + 8 B per coarse point)
 *   kernel 2: fused prolongation + Jacobi       (8+4+8 B per fine point + 8 B per coarse point)
 *   kernel 3: Arnoldi update sweep at step 4, w -= sum c_i v_i over 5 basis vectors
 *                                                (56 B per point)
 *   kernel 4: one whole V-cycle (M_V)            (bytes: not reported, 0)
 *   kernel 5: the coarsest-grid GMRES solve      (bytes: not reported, 0)
 *   kernel 6: Arnoldi projection sweep at step 4, w = A z with the 5 inner products
 *             <v_i, w> and ||w||^2               (60 B per point)               */
int helm_time_kernel(helm_t h, int kernel, int nrhs, int reps, helm_stream_t stream, float* ms, double* bytes);

/* Tile tuner report (no counterpart in the paper): the segment height the tuner chose
 * for a fused cycle kernel of `level` (kernel 0: residual + full weighting to level+1;
 * kernel 1: prolongation + correction + Jacobi from level+1) with nrhs right-hand sides:
 * 4, 8, 16 or 32 rows of the FP32 column-strip form, -1 for the shared-memory tile form,
 * 0 if not tuned yet (the launch then picks by occupancy).  fgmres_solve tunes every level
 * once per nrhs before it captures its first cycle, timing each candidate on the
 * handle's workspace.  HELM_EINVAL for a level without a coarser one. */
int helm_tile_choice(helm_t h, int kernel, int level, int nrhs, int* seg);
/* Set that choice instead of the tuner (seg as above; 0 forgets it, so that the next
 * fgmres_solve tunes again).  Also used by the tests to run every tile form.  Drops the
 * handle's captured cycles.  HELM_EINVAL for other values. */
int helm_set_tile_choice(helm_t h, int kernel, int level, int nrhs, int seg);

/* Coarsest-grid GMRES solve that allocates nothing (no counterpart in the
 * paper; the arithmetic is helm_coarse_solve's one-launch kernel).  Some
 * callers cannot call cudaMalloc: code that runs while a CUDA graph is being
 * captured, real-time loops that must not trigger the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree, and hosts whose memory budget is
 * fixed up front.  The operator is the 5-point stencil with Dirichlet
 * boundaries.  They pass the coarse problem itself -- nx x ny grid, mesh
 * width h, omega, shift beta, layer width (in this grid's cells) and peak,
 * kappa2 (device float32 [ny][nx]) -- and complex64 right-hand sides f and
 * outputs x ([nrhs][ny][nx], device, distinct); the Krylov basis lives in a
 * file-scope device array of 2^20 complex64 values (8 MiB), which every GPU
 * that loads the library holds until the process exits.
 *   Limits: (m + 1) * nrhs * nx * ny <= 2^20 and nx * ny * 8 <= 160 KiB, else
 *   HELM_EINVAL with a message; 1 <= m <= 32.
 *   The first call on a device looks up that array's device address
 *   (cudaGetSymbolAddress) with the device current; make that first call
 *   before any stream capture.  Every call shares the one array: calls that
 *   overlap on the GPU (different streams, or concurrent host threads) race
 *   and must be ordered by the caller.  The array keeps the last call's
 *   contents; nothing in it needs to start at zero (each basis vector is
 *   written before it is read). */
int helm_coarse_solve_static(int nx, int ny, double h, double omega, double beta, int abc_width, double gamma_max,
                             const float* kappa2, const void* f, void* x, int nrhs, int m, helm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
