// Batched Arnoldi / GMRES / FGMRES kernels.
//
// GMRES(m) on the coarsest grid (Sec. 2.4 and 4: diagonal-Jacobi right
// preconditioning, x0 = 0) and restarted FGMRES(m) for A M^-1 u = g (Eq. 2.5;
// the flexible variant of Saad 1993 that the paper cites) share this code:
// Arnoldi by classical Gram-Schmidt applied twice (launch_arnoldi; the modified
// Gram-Schmidt kernels remain for the block and timing paths), complex Givens
// rotations on the Hessenberg matrix, back substitution, x += Z y.
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
#include <cstdint>
#include <type_traits>

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
  select_medium(op, rhs);
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

// ---------------------------------------------------------------------------
// Arnoldi step by classical Gram-Schmidt applied twice (CGS2).
//
// MGS orthogonalises w against v_0..v_j one vector per sweep (j + 1 sweeps over w and
// one more to normalise).  CGS takes every projection coefficient from one sweep and
// subtracts them in the next; applied twice it keeps the basis as orthogonal as MGS
// does ("twice is enough": Giraud, Langou, Rozloznik 2005), whereas a single CGS pass
// loses orthogonality geometrically in FP32 when most of w lies in the basis (as it
// does with a good preconditioner):
//   A  w = K z;  c_i = <v_i, w>                                  (one sweep, also the operator)
//   B  w' = w - sum c_i v_i;  d_i = <v_i, w'>;  ||w'||^2         (one sweep)
//   C  v_{j+1} = (w' - sum d_i v_i) / nu,  nu^2 = ||w'||^2 - sum |d_i|^2
// Column j of the Hessenberg matrix is c + d with h_{j+1,j} = nu.  The second
// coefficients are small, so nu^2 by Pythagoras has no cancellation.  In exact
// arithmetic this is MGS's Arnoldi process.  Every reduction is deterministic (fixed
// order over blocks); the last block of sweep B completes column j and runs the Givens
// step; sweep C is skipped after the last step of a cycle.
// ---------------------------------------------------------------------------

// Reduce per-thread values over the block and publish this block's totals to mpart;
// returns true in every thread of the last block to arrive, which then holds the grand
// totals (fixed order) in tot[].  Values 0..j are reduced, and with with_norm also the
// value in slot NV - 1 (it lands in tot[j + 1]).
template <int NV, typename T>
__device__ bool reduce_many(T (&ax)[NV], T (&ay)[NV], int j, bool with_norm, const ArnoldiState& st, int rhs,
                            int nb, double2* tot) {
  __shared__ double2 sm[NT / 32][NV];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nv = j + 1 + (with_norm ? 1 : 0);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v <= j || (with_norm && v == NV - 1)) {
      T x = ax[v], y = ay[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
      }
      if (lane == 0) sm[warp][v <= j ? v : j + 1] = d2((double)x, (double)y);
    }
  }
  __syncthreads();
  double2* base = st.mpart + (size_t)rhs * (kProjMax + 1) * st.mcap;
  if (threadIdx.x < nv) {
    double2 acc = d2(0, 0);
    for (int w = 0; w < NT / 32; ++w) acc = dadd(acc, sm[w][threadIdx.x]);
    base[(size_t)threadIdx.x * st.mcap + blockIdx.x] = acc;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(st.counter + rhs, 1) == nb - 1);
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int v = warp; v < nv; v += NT / 32) {
    double x = 0, y = 0;
    for (int b = lane; b < nb; b += 32) {
      const double2 q = __ldcg(base + (size_t)v * st.mcap + b);
      x += q.x;
      y += q.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane == 0) tot[v] = d2(x, y);
  }
  __syncthreads();
  if (threadIdx.x == 0) st.counter[rhs] = 0;
  return true;
}

// Sweep A: w = K z (diag_precond: K D^-1 z), c_i = <v_i, w> for i <= j.
template <typename T, int ORD, int JB>
__global__ void __launch_bounds__(NT) k_arnoldi_project(Op<T> op, int diag_precond,
                                                        const typename vec2<T>::type* __restrict__ z,
                                                        const typename vec2<T>::type* __restrict__ V, size_t vstride,
                                                        typename vec2<T>::type* __restrict__ wbase, ArnoldiState st,
                                                        int j, int nb) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.y;
  select_medium(op, rhs);
  if (!st.active[rhs]) return;
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny, off = (size_t)rhs * N;
  const T2* zr = z + off;
  T2* w = wbase + off;
  T ax[JB], ay[JB];
#pragma unroll
  for (int i = 0; i < JB; ++i) { ax[i] = 0; ay[i] = 0; }
  for (size_t p = (size_t)blockIdx.x * NT + threadIdx.x; p < N; p += (size_t)nb * NT) {
    const int y = (int)(p / nx), x = (int)(p - (size_t)y * nx);
    T2 c, sn;
    if (diag_precond) {
      c = cmul(zr[p], crecip(diag_at(op, x, y)));
      sn = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) {
        return cmul(zr[(ptrdiff_t)p + (ptrdiff_t)dy * nx + dx], crecip(diag_at(op, x + dx, y + dy)));
      });
    } else {
      c = zr[p];
      sn = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) { return zr[(ptrdiff_t)p + (ptrdiff_t)dy * nx + dx]; });
    }
    T2 r = cmul(diag_at(op, x, y), c);
    r.x -= sn.x * op.inv_h2;
    r.y -= sn.y * op.inv_h2;
    w[p] = r;
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) cdot_acc(ax[i], ay[i], V[(size_t)i * vstride + off + p], r);
  }
  __shared__ double2 tot[JB + 1];
  if (!reduce_many<JB, T>(ax, ay, j, false, st, rhs, nb, tot) || threadIdx.x != 0) return;
  const int m = st.m;
  double2* Hc = st.H + (size_t)rhs * (m + 1) * m;
  double2* proj = st.proj + (size_t)rhs * kProjMax;
  for (int i = 0; i <= j; ++i) {
    Hc[(size_t)i * m + j] = tot[i];
    proj[i] = tot[i];
  }
}

// Sweep B: w' = w - sum_{i<=j} c_i v_i (written back when write_next), d_i = <v_i, w'>,
// ||w'||^2; the last block completes column j and runs the Givens step.
// only_update: the subtraction alone, written back, no reductions (timing hook).
template <typename T, int JB>
__global__ void __launch_bounds__(NT) k_arnoldi_update(const typename vec2<T>::type* __restrict__ V, size_t vstride,
                                                       typename vec2<T>::type* __restrict__ wbase, size_t N,
                                                       ArnoldiState st, int j, int nb, int write_next,
                                                       int only_update) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const int m = st.m;
  __shared__ T2 cf[JB];
  if (threadIdx.x <= j && threadIdx.x < JB) {
    const double2 q = st.proj[(size_t)rhs * kProjMax + threadIdx.x];
    cf[threadIdx.x].x = (T)q.x;
    cf[threadIdx.x].y = (T)q.y;
  }
  __syncthreads();
  const size_t off = (size_t)rhs * N;
  T2* w = wbase + off;
  T ax[JB + 1], ay[JB + 1];
#pragma unroll
  for (int i = 0; i <= JB; ++i) { ax[i] = 0; ay[i] = 0; }
  for (size_t p = (size_t)blockIdx.x * NT + threadIdx.x; p < N; p += (size_t)nb * NT) {
    T2 wv = w[p];
    T2 vv[JB];
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) {
        vv[i] = V[(size_t)i * vstride + off + p];
        wv = csub(wv, cmul(cf[i], vv[i]));
      }
    if (write_next || only_update) w[p] = wv;
    if (!only_update) {
#pragma unroll
      for (int i = 0; i < JB; ++i)
        if (i <= j) cdot_acc(ax[i], ay[i], vv[i], wv);
      ax[JB] += wv.x * wv.x + wv.y * wv.y;
    }
  }
  if (only_update) return;
  __shared__ double2 tot[JB + 2];
  if (!reduce_many<JB + 1, T>(ax, ay, j, true, st, rhs, nb, tot) || threadIdx.x != 0) return;
  double2* Hw = st.H + (size_t)rhs * (m + 1) * m;
  double2* proj = st.proj + (size_t)rhs * kProjMax;
  double s = 0.0;
  for (int i = 0; i <= j; ++i) {
    Hw[(size_t)i * m + j] = dadd(Hw[(size_t)i * m + j], tot[i]);
    proj[i] = tot[i];
    s += tot[i].x * tot[i].x + tot[i].y * tot[i].y;
  }
  const double nu2 = tot[j + 1].x - s;
  Hw[(size_t)(j + 1) * m + j] = d2(nu2 > 0.0 ? sqrt(nu2) : 0.0, 0);
  givens_step(st, rhs, j);
}

// Sweep C: v_{j+1} = (w' - sum d_i v_i) / h_{j+1,j} for right-hand sides that continue.
template <typename T, int JB>
__global__ void __launch_bounds__(NT) k_arnoldi_finish(const typename vec2<T>::type* __restrict__ V, size_t vstride,
                                                       typename vec2<T>::type* __restrict__ wbase, size_t N,
                                                       ArnoldiState st, int j, int nb) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const int m = st.m;
  __shared__ T2 cf[JB];
  if (threadIdx.x <= j && threadIdx.x < JB) {
    const double2 q = st.proj[(size_t)rhs * kProjMax + threadIdx.x];
    cf[threadIdx.x].x = (T)q.x;
    cf[threadIdx.x].y = (T)q.y;
  }
  __syncthreads();
  const T inv = (T)(1.0 / st.H[(size_t)rhs * (m + 1) * m + (size_t)(j + 1) * m + j].x);
  const size_t off = (size_t)rhs * N;
  T2* w = wbase + off;
  for (size_t p = (size_t)blockIdx.x * NT + threadIdx.x; p < N; p += (size_t)nb * NT) {
    T2 wv = w[p];
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) wv = csub(wv, cmul(cf[i], V[(size_t)i * vstride + off + p]));
    w[p] = cscale(wv, inv);
  }
}

// ---------------------------------------------------------------------------
// FP32 forms of the three CGS2 sweeps for the 5-point operator: each thread takes two
// consecutive nodes per visit (16-byte loads and stores; nx even, so a pair never
// crosses a row), which halves the load instructions and doubles the bytes in flight.
// Same arithmetic as the generic kernels above.
// ---------------------------------------------------------------------------
struct F2x2 { float2 a, b; };
__device__ __forceinline__ F2x2 ldp(const float2* p) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  return {make_float2(q.x, q.y), make_float2(q.z, q.w)};
}
__device__ __forceinline__ void stp(float2* p, F2x2 v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}

// DIAG: w = K D^-1 z (the coarsest GMRES's right preconditioning), i.e. w = z - s(u) / h^2
// with u = D^-1 z at the neighbours (D u = z at the node itself).
template <int BC, int JB, bool DIAG>
__global__ void __launch_bounds__(NT) k_arnoldi_project2(Op<float> op, const float2* __restrict__ z,
                                                         const float2* __restrict__ V, size_t vstride,
                                                         float2* __restrict__ wbase, ArnoldiState st, int j, int nb) {
  const int rhs = blockIdx.y;
  select_medium(op, rhs);
  if (!st.active[rhs]) return;
  const int nx = op.nx, ny = op.ny;
  const unsigned N = (unsigned)nx * (unsigned)ny, half = N / 2;
  const size_t off = (size_t)rhs * N;
  const float2* zr = z + off;
  float2* w = wbase + off;
  float ax[JB], ay[JB];
#pragma unroll
  for (int i = 0; i < JB; ++i) { ax[i] = 0; ay[i] = 0; }
  for (unsigned q = blockIdx.x * NT + threadIdx.x; q < half; q += (unsigned)nb * NT) {
    const unsigned p = 2 * q;
    const int y = (int)(p / (unsigned)nx), x = (int)(p - (unsigned)y * nx);
    const F2x2 c = ldp(zr + p);
    F2x2 dn = y > 0 ? ldp(zr + p - nx) : F2x2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    F2x2 up = y < ny - 1 ? ldp(zr + p + nx) : F2x2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float2 lf = x > 0 ? zr[p - 1] : make_float2(0.f, 0.f);
    float2 rt = x + 2 < nx ? zr[p + 2] : make_float2(0.f, 0.f);
    const float2 kk = *reinterpret_cast<const float2*>(op.k2 + p);
    F2x2 r;
    if (DIAG) {
      // u = D^-1 z on the neighbours and on the pair itself (each node's own diagonal)
      auto u_at = [&](float2 v, int xx, int yy) {
        return cmul(v, crecip(diag_k2<BC, 2>(op, xx, yy, op.k2[(size_t)yy * nx + xx])));
      };
      if (y > 0) { dn.a = u_at(dn.a, x, y - 1); dn.b = u_at(dn.b, x + 1, y - 1); }
      if (y < ny - 1) { up.a = u_at(up.a, x, y + 1); up.b = u_at(up.b, x + 1, y + 1); }
      if (x > 0) lf = u_at(lf, x - 1, y);
      if (x + 2 < nx) rt = u_at(rt, x + 2, y);
      const float2 ua = cmul(c.a, crecip(diag_k2<BC, 2>(op, x, y, kk.x)));
      const float2 ub = cmul(c.b, crecip(diag_k2<BC, 2>(op, x + 1, y, kk.y)));
      const float2 sa = stencil_sum<2, BC>(op, x, y, [&](int dx, int dy) {
        return dx < 0 ? lf : dx > 0 ? ub : dy < 0 ? dn.a : up.a;
      });
      const float2 sb = stencil_sum<2, BC>(op, x + 1, y, [&](int dx, int dy) {
        return dx < 0 ? ua : dx > 0 ? rt : dy < 0 ? dn.b : up.b;
      });
      r.a = make_float2(c.a.x - sa.x * op.inv_h2, c.a.y - sa.y * op.inv_h2);
      r.b = make_float2(c.b.x - sb.x * op.inv_h2, c.b.y - sb.y * op.inv_h2);
    } else {
      const float2 s = stencil_sum<2, BC>(op, x, y, [&](int dx, int dy) {
        return dx < 0 ? lf : dx > 0 ? c.b : dy < 0 ? dn.a : up.a;
      });
      r.a = cmul(diag_k2<BC, 2>(op, x, y, kk.x), c.a);
      r.a.x -= s.x * op.inv_h2;
      r.a.y -= s.y * op.inv_h2;
      const float2 s1 = stencil_sum<2, BC>(op, x + 1, y, [&](int dx, int dy) {
        return dx < 0 ? c.a : dx > 0 ? rt : dy < 0 ? dn.b : up.b;
      });
      r.b = cmul(diag_k2<BC, 2>(op, x + 1, y, kk.y), c.b);
      r.b.x -= s1.x * op.inv_h2;
      r.b.y -= s1.y * op.inv_h2;
    }
    stp(w + p, r);
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) {
        const F2x2 vi = ldp(V + (size_t)i * vstride + off + p);
        cdot_acc(ax[i], ay[i], vi.a, r.a);
        cdot_acc(ax[i], ay[i], vi.b, r.b);
      }
  }
  __shared__ double2 tot[JB + 1];
  if (!reduce_many<JB, float>(ax, ay, j, false, st, rhs, nb, tot) || threadIdx.x != 0) return;
  const int m = st.m;
  double2* Hc = st.H + (size_t)rhs * (m + 1) * m;
  double2* proj = st.proj + (size_t)rhs * kProjMax;
  for (int i = 0; i <= j; ++i) {
    Hc[(size_t)i * m + j] = tot[i];
    proj[i] = tot[i];
  }
}

template <int JB>
__device__ __forceinline__ void arnoldi_update2(const float2* __restrict__ V, size_t vstride,
                                                        float2* __restrict__ wbase, unsigned N, ArnoldiState st, int j,
                                                        int nb, int write_next, int only_update) {
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const int m = st.m;
  __shared__ float2 cf[JB];
  if (threadIdx.x <= j && threadIdx.x < JB) {
    const double2 q = st.proj[(size_t)rhs * kProjMax + threadIdx.x];
    cf[threadIdx.x] = make_float2((float)q.x, (float)q.y);
  }
  __syncthreads();
  const size_t off = (size_t)rhs * N;
  float2* w = wbase + off;
  float ax[JB + 1], ay[JB + 1];
#pragma unroll
  for (int i = 0; i <= JB; ++i) { ax[i] = 0; ay[i] = 0; }
  const unsigned half = N / 2;
  for (unsigned q = blockIdx.x * NT + threadIdx.x; q < half; q += (unsigned)nb * NT) {
    const unsigned p = 2 * q;
    F2x2 wv = ldp(w + p);
    F2x2 vv[JB];
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) {
        vv[i] = ldp(V + (size_t)i * vstride + off + p);
        wv.a = csub(wv.a, cmul(cf[i], vv[i].a));
        wv.b = csub(wv.b, cmul(cf[i], vv[i].b));
      }
    if (write_next || only_update) stp(w + p, wv);
    if (!only_update) {
#pragma unroll
      for (int i = 0; i < JB; ++i)
        if (i <= j) {
          cdot_acc(ax[i], ay[i], vv[i].a, wv.a);
          cdot_acc(ax[i], ay[i], vv[i].b, wv.b);
        }
      ax[JB] += wv.a.x * wv.a.x + wv.a.y * wv.a.y + wv.b.x * wv.b.x + wv.b.y * wv.b.y;
    }
  }
  if (only_update) return;
  __shared__ double2 tot[JB + 2];
  if (!reduce_many<JB + 1, float>(ax, ay, j, true, st, rhs, nb, tot) || threadIdx.x != 0) return;
  double2* Hw = st.H + (size_t)rhs * (m + 1) * m;
  double2* proj = st.proj + (size_t)rhs * kProjMax;
  double s = 0.0;
  for (int i = 0; i <= j; ++i) {
    Hw[(size_t)i * m + j] = dadd(Hw[(size_t)i * m + j], tot[i]);
    proj[i] = tot[i];
    s += tot[i].x * tot[i].x + tot[i].y * tot[i].y;
  }
  const double nu2 = tot[j + 1].x - s;
  Hw[(size_t)(j + 1) * m + j] = d2(nu2 > 0.0 ? sqrt(nu2) : 0.0, 0);
  givens_step(st, rhs, j);
}

template <int JB>
__global__ void __launch_bounds__(NT) k_arnoldi_update2(const float2* __restrict__ V, size_t vstride,
                                                        float2* __restrict__ wbase, unsigned N, ArnoldiState st, int j,
                                                        int nb, int write_next, int only_update) {
  arnoldi_update2<JB>(V, vstride, wbase, N, st, j, nb, write_next, only_update);
}
// The same sweep held to 80 registers (three blocks per SM instead of two at 5-8 basis
// vectors): more bytes in flight on the fine grid's long vectors (852 -> 720 us at
// 2048^2 x 16, j = 4); the coarsest solve's short vectors measured slower that way (fewer,
// unevenly filled waves), and at 1-4 vectors the free form already uses 60 registers.
template <int JB>
__global__ void __launch_bounds__(NT, 3) k_arnoldi_update2_occ(const float2* __restrict__ V, size_t vstride,
                                                               float2* __restrict__ wbase, unsigned N, ArnoldiState st,
                                                               int j, int nb, int write_next, int only_update) {
  arnoldi_update2<JB>(V, vstride, wbase, N, st, j, nb, write_next, only_update);
}

template <int JB>
__global__ void __launch_bounds__(NT) k_arnoldi_finish2(const float2* __restrict__ V, size_t vstride,
                                                        float2* __restrict__ wbase, unsigned N, ArnoldiState st, int j,
                                                        int nb) {
  const int rhs = blockIdx.y;
  if (!st.active[rhs]) return;
  const int m = st.m;
  __shared__ float2 cf[JB];
  if (threadIdx.x <= j && threadIdx.x < JB) {
    const double2 q = st.proj[(size_t)rhs * kProjMax + threadIdx.x];
    cf[threadIdx.x] = make_float2((float)q.x, (float)q.y);
  }
  __syncthreads();
  const float inv = (float)(1.0 / st.H[(size_t)rhs * (m + 1) * m + (size_t)(j + 1) * m + j].x);
  const size_t off = (size_t)rhs * N;
  float2* w = wbase + off;
  const unsigned half = N / 2;
  for (unsigned q = blockIdx.x * NT + threadIdx.x; q < half; q += (unsigned)nb * NT) {
    const unsigned p = 2 * q;
    F2x2 wv = ldp(w + p);
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) {
        const F2x2 vi = ldp(V + (size_t)i * vstride + off + p);
        wv.a = csub(wv.a, cmul(cf[i], vi.a));
        wv.b = csub(wv.b, cmul(cf[i], vi.b));
      }
    wv.a = cscale(wv.a, inv);
    wv.b = cscale(wv.b, inv);
    stp(w + p, wv);
  }
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
  if (use_dinv) select_medium(dop, rhs);
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
  select_medium(A, rhs);
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
namespace {
// Basis-length bucket of an Arnoldi column with j + 1 coefficients.
template <typename F> void with_jb(int j, F f) {
  if (j < 4) f(std::integral_constant<int, 4>());
  else if (j < 8) f(std::integral_constant<int, 8>());
  else if (j < 12) f(std::integral_constant<int, 12>());
  else if (j < 16) f(std::integral_constant<int, 16>());
  else if (j < 24) f(std::integral_constant<int, 24>());
  else f(std::integral_constant<int, 32>());
}
}  // namespace

// The pair kernels apply: FP32, the 5-point stencil, no diagonal scaling, an even point
// count and 16-byte aligned vectors.
template <typename T>
bool use_pairs(const Op<T>& op, bool diag_precond, const void* z, const void* V, size_t vstride) {
  const size_t N = (size_t)op.nx * op.ny;
  (void)diag_precond;
  return sizeof(T) == 4 && op.order == 2 && (op.nx % 2) == 0 && N < (1u << 31) &&
         (vstride % 2) == 0 && (!z || ((uintptr_t)z & 15u) == 0) && ((uintptr_t)V & 15u) == 0;
}
template <typename F> void with_bc(int bc, F f) {
  if (bc == kBcReflect) f(std::integral_constant<int, kBcReflect>());
  else if (bc == kBcReplicate) f(std::integral_constant<int, kBcReplicate>());
  else f(std::integral_constant<int, kBcDirichlet>());
}

template <typename T>
void launch_arnoldi(const Op<T>& op, bool diag_precond, const void* z, void* V, size_t vstride, int nrhs,
                    ArnoldiState& st, int j, int m, int nb, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  const size_t N = (size_t)op.nx * op.ny;
  const int write_next = j + 1 < m ? 1 : 0;
  if (use_pairs(op, diag_precond, z, V, vstride)) {
    const Op<float>& opf = reinterpret_cast<const Op<float>&>(op);
    float2* w = (float2*)V + (size_t)(j + 1) * vstride;
    with_jb(j, [&](auto jb) {
      constexpr int JB = decltype(jb)::value;
      with_bc(op.bc, [&](auto bc) {
        if (diag_precond)
          k_arnoldi_project2<decltype(bc)::value, JB, true><<<dim3(nb, nrhs), NT, 0, s>>>(
              opf, (const float2*)z, (const float2*)V, vstride, w, st, j, nb);
        else
          k_arnoldi_project2<decltype(bc)::value, JB, false><<<dim3(nb, nrhs), NT, 0, s>>>(
              opf, (const float2*)z, (const float2*)V, vstride, w, st, j, nb);
      });
      bool occ = false;
      if constexpr (JB == 8) {
        occ = !diag_precond;
        if (occ)
          k_arnoldi_update2_occ<JB><<<dim3(nb, nrhs), NT, 0, s>>>((const float2*)V, vstride, w, (unsigned)N, st, j,
                                                                  nb, write_next, 0);
      }
      if (!occ)
        k_arnoldi_update2<JB><<<dim3(nb, nrhs), NT, 0, s>>>((const float2*)V, vstride, w, (unsigned)N, st, j, nb,
                                                            write_next, 0);
      if (write_next)
        k_arnoldi_finish2<JB><<<dim3(nb, nrhs), NT, 0, s>>>((const float2*)V, vstride, w, (unsigned)N, st, j, nb);
    });
    return;
  }
  with_jb(j, [&](auto jb) {
    constexpr int JB = decltype(jb)::value;
    T2* w = (T2*)V + (size_t)(j + 1) * vstride;
    auto ka = op.order == 4 ? k_arnoldi_project<T, 4, JB> : k_arnoldi_project<T, 2, JB>;
    ka<<<dim3(nb, nrhs), NT, 0, s>>>(op, diag_precond ? 1 : 0, (const T2*)z, (const T2*)V, vstride, w, st, j, nb);
    k_arnoldi_update<T, JB><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)V, vstride, w, N, st, j, nb, write_next, 0);
    if (write_next) k_arnoldi_finish<T, JB><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)V, vstride, w, N, st, j, nb);
  });
}

template <typename T>
void launch_arnoldi_sweep(int which, const Op<T>& op, const void* z, void* V, size_t vstride, int nrhs,
                          ArnoldiState& st, int j, int nb, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  const size_t N = (size_t)op.nx * op.ny;
  T2* w = (T2*)V + (size_t)(j + 1) * vstride;
  const bool pairs = use_pairs(op, false, z, V, vstride);
  with_jb(j, [&](auto jb) {
    constexpr int JB = decltype(jb)::value;
    if (pairs) {
      const Op<float>& opf = reinterpret_cast<const Op<float>&>(op);
      if (which == 0)
        with_bc(op.bc, [&](auto bc) {
          k_arnoldi_project2<decltype(bc)::value, JB, false><<<dim3(nb, nrhs), NT, 0, s>>>(
              opf, (const float2*)z, (const float2*)V, vstride, (float2*)w, st, j, nb);
        });
      else
        if constexpr (JB == 8)
          k_arnoldi_update2_occ<JB><<<dim3(nb, nrhs), NT, 0, s>>>((const float2*)V, vstride, (float2*)w, (unsigned)N,
                                                                  st, j, nb, 0, 1);
        else
          k_arnoldi_update2<JB><<<dim3(nb, nrhs), NT, 0, s>>>((const float2*)V, vstride, (float2*)w, (unsigned)N, st,
                                                              j, nb, 0, 1);
    } else if (which == 0) {
      auto ka = op.order == 4 ? k_arnoldi_project<T, 4, JB> : k_arnoldi_project<T, 2, JB>;
      ka<<<dim3(nb, nrhs), NT, 0, s>>>(op, 0, (const T2*)z, (const T2*)V, vstride, w, st, j, nb);
    } else {
      k_arnoldi_update<T, JB><<<dim3(nb, nrhs), NT, 0, s>>>((const T2*)V, vstride, w, N, st, j, nb, 0, 1);
    }
  });
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
  template void launch_arnoldi<T>(const Op<T>&, bool, const void*, void*, size_t, int, ArnoldiState&, int, int, \
                                  int, cudaStream_t);                                                           \
  template void launch_arnoldi_sweep<T>(int, const Op<T>&, const void*, void*, size_t, int, ArnoldiState&, int,  \
                                        int, cudaStream_t);                                                     \
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
