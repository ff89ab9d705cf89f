// Batched Arnoldi / GMRES / FGMRES kernels.
//
// GMRES(m) on the coarsest grid (Sec. 2.4 and 4: diagonal-Jacobi right
// preconditioning, x0 = 0) and restarted FGMRES(m) for A M^-1 u = g (Eq. 2.5;
// the flexible variant of Saad 1993 that the paper cites) share this code:
// modified Gram-Schmidt Arnoldi, complex Givens rotations on the Hessenberg
// matrix, back substitution, x += Z y.
//
// Precision: vectors are stored in T (float for the solver); every inner
// product and norm is accumulated per thread in T over four elements, then in
// FP64 across threads and blocks; the Hessenberg matrix, rotations and the
// least-squares solution are FP64; the FGMRES iterate x and the true residual
// b - A x at each restart are FP64.
//
// A reduction's blocks write their partial sums; the last block to arrive (an
// atomic ticket) adds them in a fixed order, so results are deterministic and
// no separate reduction launch is needed.
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int NT = 256;
constexpr int MMAX = 32;   // largest supported restart length

__device__ __forceinline__ double2 d2(double x, double y) { double2 r; r.x = x; r.y = y; return r; }
__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return d2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dmul(double2 a, double2 b) { return d2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 dconj(double2 a) { return d2(a.x, -a.y); }
__device__ __forceinline__ double dabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 dscale(double2 a, double s) { return d2(a.x * s, a.y * s); }

// Sum over a 256-thread block; the total is valid in thread 0.  Threads and
// warps add in T (FP64 throughput is scarce on this part); the 8 warp totals
// are added in FP64.
template <typename T>
__device__ double2 block_sum(T ax, T ay) {
  __shared__ double2 sm[NT / 32];
  __syncthreads();  // protects sm against a previous use
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_down_sync(0xffffffffu, ax, o);
    ay += __shfl_down_sync(0xffffffffu, ay, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sm[warp] = d2((double)ax, (double)ay);
  __syncthreads();
  double2 v = d2(0, 0);
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) { v.x += sm[i].x; v.y += sm[i].y; }
  return v;
}

// Publish this block's total; returns true in every thread of the last block to
// arrive, with the grand total (fixed summation order) in thread 0's `total`.
__device__ bool finish_reduction(double2 block_total, double2* part, int* counter, int nb, double2& total) {
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = block_total;
    __threadfence();
    int t = atomicAdd(counter, 1);
    s_last = (t == nb - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double ax = 0, ay = 0;
  for (int i = threadIdx.x; i < nb; i += NT) { double2 p = __ldcg(part + i); ax += p.x; ay += p.y; }
  total = block_sum<double>(ax, ay);
  if (threadIdx.x == 0) *counter = 0;
  return true;
}

// Complex Givens rotation (c real, s complex): [c s; -conj(s) c] [a; b] = [r; 0].
__device__ void givens(double2 a, double2 b, double& c, double2& s, double2& r) {
  double aa = dabs(a), bb = dabs(b);
  if (bb == 0.0) { c = 1.0; s = d2(0, 0); r = a; return; }
  if (aa == 0.0) { c = 0.0; s = d2(1, 0); r = b; return; }
  double t = hypot(aa, bb);
  c = aa / t;
  double2 phase = dscale(a, 1.0 / aa);
  s = dscale(dmul(phase, dconj(b)), 1.0 / t);
  r = dscale(phase, t);
}

// Column j of the Hessenberg matrix is complete: rotate it, extend the rotation
// sequence, update g and decide whether this right-hand side stops.
__device__ void givens_step(const ArnoldiState& st, int rhs, int j) {
  const int m = st.m;
  const double2* Hc = st.H + (size_t)rhs * (m + 1) * m;
  double2* R = st.R + (size_t)rhs * (m + 1) * m;
  double* cs = st.cs + (size_t)rhs * m;
  double2* sn = st.sn + (size_t)rhs * m;
  double2* g = st.g + (size_t)rhs * (m + 1);
  double2 col[MMAX + 1];
  for (int i = 0; i <= j + 1; ++i) col[i] = Hc[i * m + j];
  for (int i = 0; i < j; ++i) {
    double2 t = dadd(dscale(col[i], cs[i]), dmul(sn[i], col[i + 1]));
    col[i + 1] = dadd(dscale(dmul(dconj(sn[i]), col[i]), -1.0), dscale(col[i + 1], cs[i]));
    col[i] = t;
  }
  double c; double2 s, r;
  givens(col[j], col[j + 1], c, s, r);
  cs[j] = c; sn[j] = s;
  col[j] = r; col[j + 1] = d2(0, 0);
  for (int i = 0; i <= j; ++i) R[i * m + j] = col[i];
  double2 gj = g[j];
  g[j + 1] = dscale(dmul(dconj(s), gj), -1.0);
  g[j] = dscale(gj, c);
  double est = dabs(g[j + 1]);
  bool stop = !(est > st.tol_abs[rhs]) || Hc[(j + 1) * m + j].x == 0.0 || j + 1 >= st.kmax[rhs];
  st.k[rhs] = j + 1;
  st.est[rhs] = est;
  if (stop) st.active[rhs] = 0;
}

template <typename T, typename T2>
__device__ __forceinline__ void cdot_acc(T& ax, T& ay, T2 a, T2 b) {  // conj(a) * b
  ax += a.x * b.x + a.y * b.y;
  ay += a.x * b.y - a.y * b.x;
}

// ---------------------------------------------------------------------------
// beta = ||f||, g_0 = beta, step counters reset, active = gate && beta > 0.
template <typename T>
__global__ void __launch_bounds__(NT) k_norm_start(const typename vec2<T>::type* __restrict__ f, size_t N,
                                                   ArnoldiState st, int nb, const int* gate) {
  const int rhs = blockIdx.y;
  if (gate && !gate[rhs]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) { st.active[rhs] = 0; st.k[rhs] = 0; }
    return;
  }
  const typename vec2<T>::type* fr = f + (size_t)rhs * N;
  T acc = 0;
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < N; e += (size_t)nb * NT) {
    auto v = fr[e];
    acc += v.x * v.x + v.y * v.y;
  }
  double2 bt = block_sum<T>(acc, T(0)), tot;
  if (finish_reduction(bt, st.part + (size_t)rhs * st.nbmax, st.counter + rhs, nb, tot) && threadIdx.x == 0) {
    double beta = sqrt(tot.x);
    st.beta[rhs] = beta;
    st.g[(size_t)rhs * (st.m + 1)] = d2(beta, 0);
    st.k[rhs] = 0;
    st.kmax[rhs] = st.m;
    st.active[rhs] = (beta > 0.0 && isfinite(beta)) ? 1 : 0;
  }
}

// v0 = f / beta for active right-hand sides.
template <typename T>
__global__ void __launch_bounds__(NT) k_scale(const typename vec2<T>::type* __restrict__ f,
                                              typename vec2<T>::type* __restrict__ v0, size_t N, ArnoldiState st,
                                              int nb) {
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const T inv = (T)(1.0 / st.beta[rhs]);
  const size_t off = (size_t)rhs * N;
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < N; e += (size_t)nb * NT)
    v0[off + e] = cscale(f[off + e], inv);
}

// w = K z (diag_precond: w = K D^-1 z), then h_{0j} = <v_0, w>.
template <typename T, int ORD>
__global__ void __launch_bounds__(NT) k_apply_dot(Op<T> op, int diag_precond, const typename vec2<T>::type* __restrict__ z,
                                                  typename vec2<T>::type* __restrict__ w,
                                                  const typename vec2<T>::type* __restrict__ v0, ArnoldiState st,
                                                  int j, int nb) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny, off = (size_t)rhs * N;
  const T2* zr = z + off;
  T ax = 0, ay = 0;
  for (size_t p = (size_t)blockIdx.x * NT + threadIdx.x; p < N; p += (size_t)nb * NT) {
    const int y = (int)(p / nx), x = (int)(p - (size_t)y * nx);
    T2 c, s;
    if (diag_precond) {
      c = cmul(zr[p], cinv(diag_at(op, x, y)));
      s = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) {
        return cmul(zr[(ptrdiff_t)p + (ptrdiff_t)dy * nx + dx], cinv(diag_at(op, x + dx, y + dy)));
      });
    } else {
      c = zr[p];
      s = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) { return zr[(ptrdiff_t)p + (ptrdiff_t)dy * nx + dx]; });
    }
    T2 r = cmul(diag_at(op, x, y), c);
    r.x -= s.x * op.inv_h2;
    r.y -= s.y * op.inv_h2;
    w[off + p] = r;
    cdot_acc(ax, ay, v0[off + p], r);
  }
  double2 bt = block_sum<T>(ax, ay), tot;
  if (finish_reduction(bt, st.part + (size_t)rhs * st.nbmax, st.counter + rhs, nb, tot) && threadIdx.x == 0)
    st.H[(size_t)rhs * (st.m + 1) * st.m + j] = tot;  // row 0, column j
}

// MGS pass i of step j: w -= h_{i-1,j} v_{i-1}; then h_{ij} = <v_i, w> (i <= j) or,
// for i = j + 1, h_{j+1,j} = ||w|| and the Givens step.
template <typename T>
__global__ void __launch_bounds__(NT) k_mgs(const typename vec2<T>::type* __restrict__ V, size_t vstride,
                                            typename vec2<T>::type* __restrict__ w, size_t N, int j, int i,
                                            ArnoldiState st, int nb) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const int m = st.m;
  const double2 h = st.H[(size_t)rhs * (m + 1) * m + (size_t)(i - 1) * m + j];
  const T hx = (T)h.x, hy = (T)h.y;
  const size_t off = (size_t)rhs * N;
  const T2* vp = V + (size_t)(i - 1) * vstride + off;
  const T2* vn = (i <= j) ? V + (size_t)i * vstride + off : nullptr;
  T2* wr = w + off;
  T ax = 0, ay = 0;
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < N; e += (size_t)nb * NT) {
    T2 a = vp[e], wv = wr[e];
    wv.x -= hx * a.x - hy * a.y;
    wv.y -= hx * a.y + hy * a.x;
    wr[e] = wv;
    if (vn) cdot_acc(ax, ay, vn[e], wv);
    else ax += wv.x * wv.x + wv.y * wv.y;
  }
  double2 bt = block_sum<T>(ax, ay), tot;
  if (finish_reduction(bt, st.part + (size_t)rhs * st.nbmax, st.counter + rhs, nb, tot) && threadIdx.x == 0) {
    double2* Hr = st.H + (size_t)rhs * (m + 1) * m;
    if (vn) {
      Hr[(size_t)i * m + j] = tot;
    } else {
      Hr[(size_t)(j + 1) * m + j] = d2(sqrt(tot.x), 0);
      givens_step(st, rhs, j);
    }
  }
}

// v_{j+1} = w / h_{j+1,j} for right-hand sides that continue.
template <typename T>
__global__ void __launch_bounds__(NT) k_normalize(typename vec2<T>::type* __restrict__ w, size_t N, int j,
                                                  ArnoldiState st, int nb) {
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const double nrm = st.H[(size_t)rhs * (st.m + 1) * st.m + (size_t)(j + 1) * st.m + j].x;
  const T inv = (T)(1.0 / nrm);
  const size_t off = (size_t)rhs * N;
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < N; e += (size_t)nb * NT) w[off + e] = cscale(w[off + e], inv);
}

// y = R^-1 g over the k steps taken (one thread per right-hand side).
__global__ void k_backsolve(ArnoldiState st, int nrhs, int* iters) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  const int m = st.m, k = st.k[rhs];
  const double2* R = st.R + (size_t)rhs * (m + 1) * m;
  const double2* g = st.g + (size_t)rhs * (m + 1);
  double2* y = st.y + (size_t)rhs * m;
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int l = i + 1; l < k; ++l) {
      double2 t = dmul(R[i * m + l], y[l]);
      acc.x -= t.x; acc.y -= t.y;
    }
    double2 d = R[i * m + i];
    double dd = d.x * d.x + d.y * d.y;
    y[i] = d2((acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd);
  }
  if (iters) iters[rhs] += k;
}

// out = (D^-1) sum_{i<k} y_i V_i ; zero when no step was taken.
template <typename T>
__global__ void __launch_bounds__(NT) k_combine(const typename vec2<T>::type* __restrict__ V, size_t vstride,
                                                size_t N, ArnoldiState st, Op<T> dop, int use_dinv,
                                                typename vec2<T>::type* __restrict__ out, const int* gate, int nb) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.y;
  if (gate && !gate[rhs]) return;
  const int m = st.m, k = st.k[rhs];
  __shared__ T2 ys[MMAX];
  if (threadIdx.x < k) {
    double2 yv = st.y[(size_t)rhs * m + threadIdx.x];
    ys[threadIdx.x].x = (T)yv.x; ys[threadIdx.x].y = (T)yv.y;
  }
  __syncthreads();
  const size_t off = (size_t)rhs * N;
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < N; e += (size_t)nb * NT) {
    T2 acc = czero<T2>();
    for (int i = 0; i < k; ++i) acc = cadd(acc, cmul(ys[i], V[(size_t)i * vstride + off + e]));
    if (use_dinv && k > 0) {
      const int y = (int)(e / dop.nx), x = (int)(e - (size_t)y * dop.nx);
      acc = cmul(acc, cinv(diag_at(dop, x, y)));
    }
    out[off + e] = acc;
  }
}

// ---------------------------------------------------------------------------
// FGMRES: ||b||, the FP64 true residual at each restart, x += Z y.
__global__ void __launch_bounds__(NT) k_bnorm(const double2* __restrict__ b, size_t N, SolveState ss,
                                              ArnoldiState st, int nb, double tol) {
  const int rhs = blockIdx.y;
  const double2* br = b + (size_t)rhs * N;
  double acc = 0;
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < N; e += (size_t)nb * NT) {
    double2 v = br[e];
    acc += v.x * v.x + v.y * v.y;
  }
  double2 bt = block_sum<double>(acc, 0.0), tot;
  if (finish_reduction(bt, st.part + (size_t)rhs * st.nbmax, st.counter + rhs, nb, tot) && threadIdx.x == 0) {
    double bn = sqrt(tot.x);
    ss.bnorm[rhs] = bn;
    st.tol_abs[rhs] = tol * bn;
    ss.iters[rhs] = 0;
    ss.relres[rhs] = 0.0;
    ss.status[rhs] = isfinite(bn) ? 0 : -3;
    ss.done[rhs] = (bn == 0.0 || !isfinite(bn)) ? 1 : 0;
    st.active[rhs] = 0;
    st.k[rhs] = 0;
  }
}

// r0 = b - A x in FP64 (stored as T in v0 slot); beta = ||r0||; decides convergence.
template <typename T, int ORD>
__global__ void __launch_bounds__(NT) k_true_residual(Op<double> A, const double2* __restrict__ b,
                                                      const double2* __restrict__ x,
                                                      typename vec2<T>::type* __restrict__ r0, SolveState ss,
                                                      ArnoldiState st, int nb, int maxit) {
  const int rhs = blockIdx.y;
  if (ss.done[rhs]) return;
  const int nx = A.nx, ny = A.ny;
  const size_t N = (size_t)nx * ny, off = (size_t)rhs * N;
  const double2* xr = x + off;
  double acc = 0;
  for (size_t p = (size_t)blockIdx.x * NT + threadIdx.x; p < N; p += (size_t)nb * NT) {
    const int y = (int)(p / nx), xx = (int)(p - (size_t)y * nx);
    const double2 s = stencil_sum<ORD>(A, xx, y, [&](int dx, int dy) { return xr[(ptrdiff_t)p + (ptrdiff_t)dy * nx + dx]; });
    double2 ax = dmul(diag_at(A, xx, y), xr[p]);
    double2 bb = b[off + p];
    double2 r = d2(bb.x - (ax.x - s.x * A.inv_h2), bb.y - (ax.y - s.y * A.inv_h2));
    typename vec2<T>::type rt;
    rt.x = (T)r.x; rt.y = (T)r.y;
    r0[off + p] = rt;
    acc += r.x * r.x + r.y * r.y;
  }
  double2 bt = block_sum<double>(acc, 0.0), tot;
  if (finish_reduction(bt, st.part + (size_t)rhs * st.nbmax, st.counter + rhs, nb, tot) && threadIdx.x == 0) {
    double beta = sqrt(tot.x);
    ss.relres[rhs] = beta / ss.bnorm[rhs];
    st.k[rhs] = 0;
    if (ss.maxit_rhs) maxit = ss.maxit_rhs[rhs];
    if (!isfinite(beta)) {
      ss.done[rhs] = 1; ss.status[rhs] = -3; st.active[rhs] = 0;
    } else if (beta <= st.tol_abs[rhs]) {
      ss.done[rhs] = 1; ss.status[rhs] = 0; st.active[rhs] = 0;
    } else if (ss.iters[rhs] >= maxit) {
      ss.done[rhs] = 1; ss.status[rhs] = 1; st.active[rhs] = 0;
    } else {
      st.active[rhs] = 1;
      st.beta[rhs] = beta;
      st.g[(size_t)rhs * (st.m + 1)] = d2(beta, 0);
      st.kmax[rhs] = min(st.m, maxit - ss.iters[rhs]);
    }
  }
}

// x += sum_{i<k} y_i Z_i (accumulated in T, added to the FP64 iterate).
template <typename T>
__global__ void __launch_bounds__(NT) k_update_x(const typename vec2<T>::type* __restrict__ Z, size_t vstride,
                                                 size_t N, ArnoldiState st, double2* __restrict__ x, int nb) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.y;
  const int m = st.m, k = st.k[rhs];
  if (k == 0) return;
  __shared__ T2 ys[MMAX];
  if (threadIdx.x < k) {
    double2 yv = st.y[(size_t)rhs * m + threadIdx.x];
    ys[threadIdx.x].x = (T)yv.x; ys[threadIdx.x].y = (T)yv.y;
  }
  __syncthreads();
  const size_t off = (size_t)rhs * N;
  for (size_t e = (size_t)blockIdx.x * NT + threadIdx.x; e < N; e += (size_t)nb * NT) {
    T2 acc = czero<T2>();
    for (int i = 0; i < k; ++i) acc = cadd(acc, cmul(ys[i], Z[(size_t)i * vstride + off + e]));
    double2 xv = x[off + e];
    xv.x += (double)acc.x; xv.y += (double)acc.y;
    x[off + e] = xv;
  }
}

}  // namespace

int vec_blocks(size_t N, int nrhs, int nsm) {
  size_t want = (size_t)(nsm * 8 + nrhs - 1) / (size_t)nrhs;  // about one wave of 256-thread blocks
  size_t cap = (N + (size_t)NT * 4 - 1) / ((size_t)NT * 4);     // at least 4 elements per thread
  size_t nb = want < cap ? want : cap;
  if (nb < 1) nb = 1;
  if (nb > 4096) nb = 4096;
  return (int)nb;
}

template <typename T>
void launch_start(const void* f, void* v0, size_t N, int nrhs, ArnoldiState& st, int nb, const int* gate,
                  cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_norm_start<T><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)f, N, st, nb, gate);
  k_scale<T><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)f, (T2*)v0, N, st, nb);
}
template <typename T>
void launch_apply_dot(const Op<T>& op, bool diag_precond, const void* z, void* w, const void* v0, int nrhs,
                      ArnoldiState& st, int j, int nb, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  auto k = op.order == 4 ? k_apply_dot<T, 4> : k_apply_dot<T, 2>;
  k<<<dim3(nb, nrhs), NT, 0, s>>>(op, diag_precond ? 1 : 0, (const T2*)z, (T2*)w, (const T2*)v0, st, j, nb);
}
template <typename T>
void launch_mgs(const void* V, size_t vstride, void* w, size_t N, int nrhs, int j, int i, ArnoldiState& st, int nb,
                cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_mgs<T><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)V, vstride, (T2*)w, N, j, i, st, nb);
}
template <typename T>
void launch_normalize(void* w, size_t N, int nrhs, int j, ArnoldiState& st, int nb, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_normalize<T><<<dim3(nb, nrhs), NT, 0, s>>>((T2*)w, N, j, st, nb);
}
void launch_backsolve(ArnoldiState& st, int nrhs, int* iters, cudaStream_t s) {
  k_backsolve<<<(nrhs + 63) / 64, 64, 0, s>>>(st, nrhs, iters);
}
template <typename T>
void launch_combine(const void* V, size_t vstride, size_t N, int nrhs, ArnoldiState& st, const Op<T>* dinv_op,
                    void* out, const int* gate, int nb, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  Op<T> dop{};
  if (dinv_op) dop = *dinv_op;
  k_combine<T><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)V, vstride, N, st, dop, dinv_op ? 1 : 0, (T2*)out, gate, nb);
}
void launch_bnorm(const double2* b, size_t N, int nrhs, SolveState& ss, ArnoldiState& st, int nb, double tol,
                  cudaStream_t s) {
  k_bnorm<<<dim3(nb, nrhs), NT, 0, s>>>(b, N, ss, st, nb, tol);
}
template <typename T>
void launch_true_residual(const Op<double>& A, const double2* b, const double2* x, void* r0, int nrhs,
                          SolveState& ss, ArnoldiState& st, int nb, int maxit, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  auto k = A.order == 4 ? k_true_residual<T, 4> : k_true_residual<T, 2>;
  k<<<dim3(nb, nrhs), NT, 0, s>>>(A, b, x, (T2*)r0, ss, st, nb, maxit);
}
template <typename T>
void launch_scale_v0(void* v0, size_t N, int nrhs, ArnoldiState& st, int nb, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_scale<T><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)v0, (T2*)v0, N, st, nb);
}
template <typename T>
void launch_update_x(const void* Z, size_t vstride, size_t N, int nrhs, ArnoldiState& st, double2* x, int nb,
                     cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_update_x<T><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)Z, vstride, N, st, x, nb);
}

#define INST(T)                                                                                                  \
  template void launch_start<T>(const void*, void*, size_t, int, ArnoldiState&, int, const int*, cudaStream_t); \
  template void launch_apply_dot<T>(const Op<T>&, bool, const void*, void*, const void*, int, ArnoldiState&,    \
                                    int, int, cudaStream_t);                                                    \
  template void launch_mgs<T>(const void*, size_t, void*, size_t, int, int, int, ArnoldiState&, int,            \
                              cudaStream_t);                                                                    \
  template void launch_normalize<T>(void*, size_t, int, int, ArnoldiState&, int, cudaStream_t);                 \
  template void launch_combine<T>(const void*, size_t, size_t, int, ArnoldiState&, const Op<T>*, void*,        \
                                  const int*, int, cudaStream_t);                                               \
  template void launch_true_residual<T>(const Op<double>&, const double2*, const double2*, void*, int,          \
                                        SolveState&, ArnoldiState&, int, int, cudaStream_t);                    \
  template void launch_scale_v0<T>(void*, size_t, int, ArnoldiState&, int, cudaStream_t);                       \
  template void launch_update_x<T>(const void*, size_t, size_t, int, ArnoldiState&, double2*, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace helm
