// Internal declarations of libhelm: device helpers shared by the kernel files
// and the host-side launchers the solver driver calls.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace helm {

template <typename T> struct vec2;
template <> struct vec2<float> { typedef float2 type; };
template <> struct vec2<double> { typedef double2 type; };

// ---------------------------------------------------------------------------
// Operator description passed by value to every stencil kernel.
// K = (1/h^2)(5-point negative Laplacian) - w^2 k^2 (1 - (g + beta) i),
// g the quadratic absorbing-layer profile of width abc_w on this level
// (Eq. 2.1, 2.2; Eq. 2.4 with alpha = 1 for the shifted operator).
// Boundary (Sec. 2.4, the stencil as a convolution and its padding): bc 0 pads
// with zeros (Dirichlet); bc 1 reflects about the boundary node (ghost u_-1 =
// u_1), so the inward neighbour of a boundary node couples twice; bc 2
// replicates the boundary node (ghost u_-1 = u_0), which folds that coupling
// into the diagonal: -1/h^2 per boundary side.  Both are Neumann conditions.
// Stencil: order 2 is the 5-point scheme above; order 4 the compact fourth-order
// 9-point scheme (the higher-order operators the convolution form of Sec. 2.4
// admits): with m = w^2 k^2 (1 - (g + beta) i),
//   K u = (1/(6h^2)) [-1 -4 -1; -4 20 -4; -1 -4 -1] u - (1/12) [0 1 0; 1 8 1; 0 1 0] (m u),
// the compact fourth-order Laplacian with the mass term weighted like its right-hand
// side; Dirichlet boundaries only.
// ---------------------------------------------------------------------------
enum { kBcDirichlet = 0, kBcReflect = 1, kBcReplicate = 2 };

template <typename T> struct Op {
  int nx, ny, abc_w, bc, order;
  T inv_h2, h2, omega2, gmax, beta;
  T inv_w;      // 1 / abc_w (0 without a layer)
  const T* k2;  // kappa^2 on this level, [ny][nx] (with rpp > 0: [medium][ny][nx])
  int rpp;      // right-hand sides per medium: right-hand side r uses medium r / rpp (0: one medium)
};

// Per-level storage owned by the handle.
struct Level {
  int nx, ny, abc_w, bc, order;
  double h;
  float* k2f;   // kappa^2 (float32), [medium][ny][nx]
  double* k2d;  // kappa^2 (float64), [medium][ny][nx]
  int rpp;      // right-hand sides per medium (0: one medium shared by every right-hand side)
};

template <typename T>
inline Op<T> make_op(const Level& L, double omega, double gmax, double beta) {
  Op<T> op;
  op.nx = L.nx; op.ny = L.ny; op.abc_w = L.abc_w; op.bc = L.bc; op.order = L.order;
  op.h2 = (T)(L.h * L.h);
  op.inv_h2 = (T)(1.0 / (L.h * L.h));
  op.omega2 = (T)(omega * omega);
  op.gmax = (T)gmax;
  op.beta = (T)beta;
  op.inv_w = L.abc_w > 0 ? (T)(1.0 / L.abc_w) : T(0);
  op.k2 = nullptr;
  op.rpp = L.rpp;
  return op;
}
template <> inline Op<float> make_op<float>(const Level& L, double omega, double gmax, double beta) {
  Op<float> op;
  op.nx = L.nx; op.ny = L.ny; op.abc_w = L.abc_w; op.bc = L.bc; op.order = L.order;
  op.h2 = (float)(L.h * L.h);
  op.inv_h2 = (float)(1.0 / (L.h * L.h));
  op.omega2 = (float)(omega * omega);
  op.gmax = (float)gmax; op.beta = (float)beta; op.k2 = L.k2f;
  op.inv_w = L.abc_w > 0 ? (float)(1.0 / L.abc_w) : 0.f;
  op.rpp = L.rpp;
  return op;
}
template <> inline Op<double> make_op<double>(const Level& L, double omega, double gmax, double beta) {
  Op<double> op;
  op.nx = L.nx; op.ny = L.ny; op.abc_w = L.abc_w; op.bc = L.bc; op.order = L.order;
  op.h2 = L.h * L.h;
  op.inv_h2 = 1.0 / (L.h * L.h);
  op.omega2 = omega * omega;
  op.gmax = gmax; op.beta = beta; op.k2 = L.k2d;
  op.inv_w = L.abc_w > 0 ? 1.0 / L.abc_w : 0.0;
  op.rpp = L.rpp;
  return op;
}

#ifdef __CUDACC__
// Problems that share a grid but not a medium (a batch of one size class): right-hand side
// r is solved on medium r / rpp.  Every operator kernel calls this with its right-hand side.
template <typename T> __device__ __forceinline__ void select_medium(Op<T>& op, int rhs) {
  if (op.rpp > 0) op.k2 += (size_t)(rhs / op.rpp) * op.nx * op.ny;
}

template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { T2 r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { T2 r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename T2, typename T> __device__ __forceinline__ T2 cscale(T2 a, T s) { T2 r; r.x = a.x * s; r.y = a.y * s; return r; }
template <typename T2> __device__ __forceinline__ T2 czero() { T2 r; r.x = 0; r.y = 0; return r; }
template <typename T2> __device__ __forceinline__ T2 cinv(T2 a) {
  auto d = a.x * a.x + a.y * a.y;
  T2 r; r.x = a.x / d; r.y = -a.y / d; return r;
}

// Absorbing-layer attenuation g at node (x, y): g_max (1 - d/W)^2 for d < W,
// d the distance in cells to the nearest edge (0 on the outermost unknowns).
template <typename T> __device__ __forceinline__ T gamma_at(const Op<T>& op, int x, int y) {
  int d = min(min(x, op.nx - 1 - x), min(y, op.ny - 1 - y));
  if (d >= op.abc_w) return T(0);
  T t = T(1) - T(d) * op.inv_w;
  return t * t * op.gmax;
}

// Diagonal of K at (x, y) for a stored kappa^2 value k2: 4/h^2 - w^2 k^2 + i w^2 k^2 (g +
// beta), less 1/h^2 per boundary side under replication padding; (20/6)/h^2 - (8/12) m for
// the compact scheme.  BC and ORD as template arguments fix the boundary mode and the
// stencil at compile time (-1: read them from op).
template <int BC = -1, int ORD = -1, typename T>
__device__ __forceinline__ typename vec2<T>::type diag_k2(const Op<T>& op, int x, int y, T k2) {
  const int order = ORD >= 0 ? ORD : op.order;
  const int bc = BC >= 0 ? BC : op.bc;
  T wk = op.omega2 * k2;
  typename vec2<T>::type d;
  if (order == 4) {
    const T wm = wk * T(8) / T(12);
    d.x = T(20) / T(6) * op.inv_h2 - wm;
    d.y = wm * (gamma_at(op, x, y) + op.beta);
    return d;
  }
  T c = T(4);
  if (bc == kBcReplicate)
    c -= T((x == 0) + (x == op.nx - 1) + (y == 0) + (y == op.ny - 1));
  d.x = c * op.inv_h2 - wk;
  d.y = wk * (gamma_at(op, x, y) + op.beta);
  return d;
}
template <int BC = -1, int ORD = -1, typename T>
__device__ __forceinline__ typename vec2<T>::type diag_at(const Op<T>& op, int x, int y) {
  return diag_k2<BC, ORD>(op, x, y, op.k2[(size_t)y * op.nx + x]);
}

// 1 / d for a complex d with one reciprocal of |d|^2 (FP32: the intrinsic reciprocal).
template <typename T2> __device__ __forceinline__ T2 crecip(T2 a);
template <> __device__ __forceinline__ float2 crecip<float2>(float2 a) {
  const float r = __frcp_rn(a.x * a.x + a.y * a.y);
  return make_float2(a.x * r, -a.y * r);
}
template <> __device__ __forceinline__ double2 crecip<double2>(double2 a) {
  const double r = 1.0 / (a.x * a.x + a.y * a.y);
  return make_double2(a.x * r, -a.y * r);
}

// The part of the neighbour sum that reflection padding adds at a boundary node:
// the inward neighbour once more per boundary side.  l, r, d, u are the values at
// (x-1, y), (x+1, y), (x, y-1), (x, y+1) (zero outside the grid); grids are at
// least 2 nodes wide under reflection, so the inward neighbour always exists.
template <int BC = -1, typename T, typename T2>
__device__ __forceinline__ T2 reflect_extra(const Op<T>& op, int x, int y, T2 l, T2 r, T2 d, T2 u) {
  T2 e = czero<T2>();
  if ((BC >= 0 ? BC : op.bc) != kBcReflect) return e;
  if (x == 0) e = cadd(e, r); else if (x == op.nx - 1) e = cadd(e, l);
  if (y == 0) e = cadd(e, u); else if (y == op.ny - 1) e = cadd(e, d);
  return e;
}

// m u at (x, y): w^2 k^2 (1 - (g + beta) i) u.
template <typename T, typename T2>
__device__ __forceinline__ T2 mass_times(const Op<T>& op, int x, int y, T2 u) {
  const T wk = op.omega2 * op.k2[(size_t)y * op.nx + x];
  T2 m;
  m.x = wk;
  m.y = -wk * (gamma_at(op, x, y) + op.beta);
  return cmul(m, u);
}

// Off-diagonal part s of K at (x, y) in the form K u = D u - s / h^2, with at(dx, dy)
// the value at (x + dx, y + dy), called only for nodes inside the grid.  ORD 2 (5-point):
// the four neighbours (plus the reflection term); ORD 4 (compact scheme): (4 edges +
// corners) / 6 + (h^2 / 12) sum over the edges of m_q u_q.  The order is a template
// parameter so that the 5-point kernels carry none of the 9-point registers; launchers
// pick the instantiation from op.order.
template <int ORD, int BC = -1, typename T, typename F>
__device__ __forceinline__ typename vec2<T>::type stencil_sum(const Op<T>& op, int x, int y, F at) {
  typedef typename vec2<T>::type T2;
  const bool xl = x > 0, xr = x < op.nx - 1, yd = y > 0, yu = y < op.ny - 1;
  const T2 l = xl ? at(-1, 0) : czero<T2>();
  const T2 rt = xr ? at(1, 0) : czero<T2>();
  const T2 dn = yd ? at(0, -1) : czero<T2>();
  const T2 up = yu ? at(0, 1) : czero<T2>();
  const T2 e = cadd(cadd(l, rt), cadd(dn, up));
  if (ORD != 4) return cadd(e, reflect_extra<BC>(op, x, y, l, rt, dn, up));
  T2 c = czero<T2>();
  if (yd && xl) c = cadd(c, at(-1, -1));
  if (yd && xr) c = cadd(c, at(1, -1));
  if (yu && xl) c = cadd(c, at(-1, 1));
  if (yu && xr) c = cadd(c, at(1, 1));
  T2 mq = czero<T2>();
  if (xl) mq = cadd(mq, mass_times(op, x - 1, y, l));
  if (xr) mq = cadd(mq, mass_times(op, x + 1, y, rt));
  if (yd) mq = cadd(mq, mass_times(op, x, y - 1, dn));
  if (yu) mq = cadd(mq, mass_times(op, x, y + 1, up));
  T2 s = cscale(cadd(cscale(e, T(4)), c), T(1) / T(6));
  return cadd(s, cscale(mq, op.h2 / T(12)));
}
#endif

// Block sizes shared by launchers.
constexpr int kVecThreads = 256;

// ---------------------------------------------------------------------------
// Launchers (stencil.cu).  All vectors are complex, interleaved, [rhs][y][x];
// `active` (nullable) holds one int per right-hand side: 0 = skip it.
// ---------------------------------------------------------------------------
template <typename T> void launch_apply(const Op<T>& op, const void* x, const void* b, void* y, int nrhs,
                                        const int* active, cudaStream_t s);
// y = (1/12) [0 1 0; 1 8 1; 0 1 0] x (the compact scheme's right-hand side); y != x.
template <typename T> void launch_rhs_weight(const Op<T>& op, const void* x, void* y, int nrhs, cudaStream_t s);
template <typename T> void launch_jacobi(const Op<T>& op, T w, const void* f, const void* x_in, void* x_out,
                                         int nrhs, const int* active, cudaStream_t s);
template <typename T> void launch_restrict(int nx, int ny, const void* rf, void* rc, int nrhs,
                                           const int* active, cudaStream_t s);
template <typename T> void launch_prolong_add(int nxc, int nyc, int nx, int ny, const void* ec, void* xf,
                                              int nrhs, const int* active, cudaStream_t s);
// The fused cycle kernels.  seg: the segment height of the FP32 column-strip form (4, 8,
// 16 or 32 rows; 0 = pick by occupancy), or -1 for the shared-memory tile form; FP64,
// the compact scheme and pointers that are not 16-byte aligned always take the tile form.
template <typename T> void launch_resid_restrict(const Op<T>& fine, T w, const void* f, const void* v,
                                                 void* fc, int nrhs, const int* active, cudaStream_t s,
                                                 int seg = 0);
template <typename T> void launch_prolong_jacobi(const Op<T>& fine, T w, const void* f, const void* v,
                                                 bool implicit_v, const void* ec, int nxc, int nyc, void* out,
                                                 int nrhs, const int* active, cudaStream_t s, int seg = 0);
void launch_coarsen_kappa2(const double* k2d_fine, int nx, int ny, double* k2d_coarse, float* k2f_coarse,
                           cudaStream_t s);
void launch_widen_kappa2(const float* k2f, double* k2d, size_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Krylov machinery (krylov.cu).  One Arnoldi process per right-hand side,
// batched; reductions accumulate per thread in T, per block and across blocks
// in FP64; the last block to finish a reduction writes the result (and, for
// the norm, performs the Givens update) so no extra launch is needed.
// ---------------------------------------------------------------------------
struct ArnoldiState {      // device arrays, per right-hand side
  double2* H;              // [nrhs][m+1][m] Hessenberg (raw), complex FP64
  double2* R;              // [nrhs][m+1][m] rotated Hessenberg
  double* cs;              // [nrhs][m]
  double2* sn;             // [nrhs][m]
  double2* g;              // [nrhs][m+1]
  double2* y;              // [nrhs][m]
  double* beta;            // [nrhs]   initial residual norm of the cycle
  int* active;             // [nrhs]   1 while Arnoldi runs in this cycle
  int* k;                  // [nrhs]   steps taken in this cycle
  int* kmax;               // [nrhs]   steps allowed in this cycle
  double* est;             // [nrhs]   latest residual estimate |g_k|
  double* tol_abs;         // [nrhs]   stop when |g_k| <= tol_abs (0: run m steps)
  double2* part;           // [nrhs][nbmax] block partials
  int* counter;            // [nrhs]   arrival tickets of the last-block reduction
  int nbmax;
  int m;
  // classical Gram-Schmidt Arnoldi (launch_arnoldi)
  double2* proj;           // [nrhs][kProjMax] coefficients of the pending projection
  double2* mpart;          // [nrhs][kProjMax + 1][mcap] block partials of the multi-value reductions
  int mcap;                // block capacity of mpart (>= every nb used with this state)
};
constexpr int kProjMax = 32;   // longest Arnoldi column (restart length) the projections handle

struct SolveState {         // FGMRES, per right-hand side, device
  double* bnorm;
  double* relres;
  int* done;                // converged (or failed) for good
  int* iters;
  int* status;              // 0 running/converged, 1 max iterations, -3 non-finite
  const int* maxit_rhs;     // per right-hand-side iteration cap, or null (use the global one)
};

int vec_blocks(size_t N, int nrhs, int nsm);

// Start of a cycle from f: beta = ||f||, g_0 = beta, active = gate && beta > 0,
// then v_0 = f / beta (two launches).
template <typename T> void launch_start(const void* f, void* v0, size_t N, int nrhs, ArnoldiState& st, int nb,
                                        const int* gate, cudaStream_t s);
// w = K z (or K D^-1 z) and h_{0j} = <v_0, w>.
template <typename T> void launch_apply_dot(const Op<T>& op, bool diag_precond, const void* z, void* w,
                                            const void* v0, int nrhs, ArnoldiState& st, int j, int nb,
                                            cudaStream_t s);
// MGS pass i (1 <= i <= j+1): w -= h_{i-1,j} v_{i-1}; then h_{ij} = <v_i, w> (i <= j)
// or h_{j+1,j} = ||w|| followed by the Givens update and the stopping test (i = j+1).
template <typename T> void launch_mgs(const void* V, size_t vstride, void* w, size_t N, int nrhs, int j, int i,
                                      ArnoldiState& st, int nb, cudaStream_t s);
template <typename T> void launch_normalize(void* w, size_t N, int nrhs, int j, ArnoldiState& st, int nb,
                                            cudaStream_t s);
// Arnoldi step j by classical Gram-Schmidt applied twice (three sweeps instead of MGS's
// j + 3): w = K z (or K D^-1 z) written to V slot j+1, column j of the Hessenberg matrix,
// the Givens step and, if j + 1 < m, v_{j+1} = w / h_{j+1,j} in place.  V: [slot][rhs][N]
// with slots vstride elements apart.
template <typename T> void launch_arnoldi(const Op<T>& op, bool diag_precond, const void* z, void* V, size_t vstride,
                                          int nrhs, ArnoldiState& st, int j, int m, int nb, cudaStream_t s);
// One sweep of launch_arnoldi alone (timing hook): which 0 = the projection sweep
// (w = K z and the j + 2 reductions), 1 = the update sweep (w -= sum_i c_i v_i, i <= j).
template <typename T> void launch_arnoldi_sweep(int which, const Op<T>& op, const void* z, void* V, size_t vstride,
                                                int nrhs, ArnoldiState& st, int j, int nb, cudaStream_t s);
// y = R^-1 g per right-hand side; iters (nullable) += steps taken.
void launch_backsolve(ArnoldiState& st, int nrhs, int* iters, cudaStream_t s);
// out = (D^-1) sum_i y_i V_i over the k steps of each right-hand side (0 if k = 0);
// right-hand sides with gate == 0 are skipped.
template <typename T> void launch_combine(const void* V, size_t vstride, size_t N, int nrhs, ArnoldiState& st,
                                          const Op<T>* dinv_op, void* out, const int* gate, int nb,
                                          cudaStream_t s);

// Coarsest GMRES(m) in one launch (coarse.cu); false (nothing launched) if the grid does
// not fit or the kernel's shared-memory opt-in failed on this device.  launch_err
// (nullable) receives the launch's own result (or the opt-in failure).
template <typename T> bool launch_coarse_gmres_fused(const Op<T>& op, const void* f, void* out, void* V,
                                                     size_t vstride, int nrhs, int m, const int* gate,
                                                     cudaStream_t s, cudaError_t* launch_err = nullptr);

// Coarsest GMRES(m) on one thread-block cluster per right-hand side (coarse_cluster.cu);
// false if the grid does not fit (C <= 16 CTAs of <= 1024 points, basis in shared memory).
template <typename T> bool launch_coarse_gmres_cluster(const Op<T>& op, const void* f, void* out, int nrhs, int m,
                                                       const int* gate, void* gbasis, size_t vstride, cudaStream_t s);

// FGMRES (outer solver)
void launch_bnorm(const double2* b, size_t N, int nrhs, SolveState& ss, ArnoldiState& st, int nb, double tol,
                  cudaStream_t s);
template <typename T> void launch_true_residual(const Op<double>& A, const double2* b, const double2* x, void* r0,
                                                int nrhs, SolveState& ss, ArnoldiState& st, int nb, int maxit,
                                                cudaStream_t s);
template <typename T> void launch_scale_v0(void* v0, size_t N, int nrhs, ArnoldiState& st, int nb, cudaStream_t s);
template <typename T> void launch_update_x(const void* Z, size_t vstride, size_t N, int nrhs, ArnoldiState& st,
                                           double2* x, int nb, cudaStream_t s);

// Block kernels (block.cu) of block FGMRES.  Vectors [vector][point], `stride` apart.
// out[i * p + k] = sum over N points of conj(U_i) W_k (q x p, FP64), via block_gram_parts(nsm)
// per-CTA partials in `part` (q * p each); returns -1 if p > 16 or q * p > 4608.
int block_gram_parts(int nsm);
template <typename T2>
int block_gram(const T2* U, size_t ustride, int q, const T2* W, size_t wstride, int p, size_t N, double2* part,
               double2* out, int nsm, cudaStream_t s);
// out_k (+)= sum_i in_i C[i * p + k] (C device FP64, q x p); in may equal out when q == p.
template <typename TI, typename TO>
int block_combine(const TI* in, size_t istride, int q, const double2* C, TO* out, size_t ostride, int p, size_t N,
                  bool accumulate, int nsm, cudaStream_t s);

}  // namespace helm
