// Stencil kernels of the shifted-Laplacian multigrid cycle:
//   * operator apply / residual     (Eq. 2.2, 2.4)
//   * damped Jacobi sweep           (Sec. 4: w = 0.8, one pre and one post sweep)
//   * full-weighting restriction and bilinear prolongation (Eq. 2.9), as
//     stride-2 convolution / transposed convolution with zero padding 1
//   * fused cycle kernels:
//       resid_restrict:  f_c = R (f - K v), with v = w D^-1 f computed in the
//                        tile when the level starts from a zero guess
//       prolong_jacobi:  out = J(v + P e_c, f), the coarse-grid correction
//                        followed by the post-smoothing sweep
// Every kernel is templated on the real type T (float for the solver, double
// for FP64 verification runs).  Layout: complex interleaved, [rhs][y][x].
#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int BX = 32, BY = 8;  // 256 threads, one point (fine or coarse) per thread

template <int ORD, typename T>
__device__ __forceinline__ typename vec2<T>::type apply_at(const Op<T>& op, const typename vec2<T>::type* u,
                                                           int x, int y) {
  typedef typename vec2<T>::type T2;
  size_t p = (size_t)y * op.nx + x;
  T2 c = u[p];
  const T2 s = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) { return u[(ptrdiff_t)p + (ptrdiff_t)dy * op.nx + dx]; });
  T2 d = diag_at(op, x, y);
  T2 r = cmul(d, c);
  r.x -= s.x * op.inv_h2;
  r.y -= s.y * op.inv_h2;
  return r;
}

// y = K x  (b == nullptr)   or   y = b - K x
template <typename T, int ORD>
__global__ void __launch_bounds__(256) k_apply(Op<T> op, const typename vec2<T>::type* __restrict__ x,
                                               const typename vec2<T>::type* __restrict__ b,
                                               typename vec2<T>::type* __restrict__ y, const int* active) {
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const int ix = blockIdx.x * BX + threadIdx.x, iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= op.nx || iy >= op.ny) return;
  const size_t N = (size_t)op.nx * op.ny, off = (size_t)rhs * N, p = (size_t)iy * op.nx + ix;
  auto ku = apply_at<ORD>(op, x + off, ix, iy);
  if (b) ku = csub(b[off + p], ku);
  y[off + p] = ku;
}

// Right-hand side of the compact fourth-order scheme for a source x:
// y = (1/12) [0 1 0; 1 8 1; 0 1 0] x, zero outside the grid.
template <typename T>
__global__ void __launch_bounds__(256) k_rhs_weight(int nx, int ny, const typename vec2<T>::type* __restrict__ x,
                                                    typename vec2<T>::type* __restrict__ y) {
  typedef typename vec2<T>::type T2;
  const int ix = blockIdx.x * BX + threadIdx.x, iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= nx || iy >= ny) return;
  const size_t off = (size_t)blockIdx.z * nx * ny, p = off + (size_t)iy * nx + ix;
  T2 e = czero<T2>();
  if (ix > 0) e = cadd(e, x[p - 1]);
  if (ix < nx - 1) e = cadd(e, x[p + 1]);
  if (iy > 0) e = cadd(e, x[p - nx]);
  if (iy < ny - 1) e = cadd(e, x[p + nx]);
  y[p] = cscale(cadd(cscale(x[p], T(8)), e), T(1) / T(12));
}

// x_out = x_in + w D^-1 (f - K x_in);   x_in == nullptr means a zero guess: x_out = w D^-1 f
template <typename T, int ORD>
__global__ void __launch_bounds__(256) k_jacobi(Op<T> op, T w, const typename vec2<T>::type* __restrict__ f,
                                                const typename vec2<T>::type* __restrict__ xin,
                                                typename vec2<T>::type* __restrict__ xout, const int* active) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const int ix = blockIdx.x * BX + threadIdx.x, iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= op.nx || iy >= op.ny) return;
  const size_t N = (size_t)op.nx * op.ny, off = (size_t)rhs * N, p = (size_t)iy * op.nx + ix;
  T2 r = f[off + p];
  if (xin) r = csub(r, apply_at<ORD>(op, xin + off, ix, iy));
  T2 c = cscale(cmul(r, cinv(diag_at(op, ix, iy))), w);
  if (xin) c = cadd(c, xin[off + p]);
  xout[off + p] = c;
}

// Full weighting: rc(I,J) = sum_{a,b in -1..1} (1/16)[1 2 1]_a [1 2 1]_b rf(2I+a, 2J+b)
template <typename T>
__global__ void __launch_bounds__(256) k_restrict(int nx, int ny, const typename vec2<T>::type* __restrict__ rf,
                                                  typename vec2<T>::type* __restrict__ rc, const int* active) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const int nxc = nx / 2, nyc = ny / 2;
  const int J = blockIdx.x * BX + threadIdx.x, I = blockIdx.y * BY + threadIdx.y;
  if (J >= nxc || I >= nyc) return;
  const T2* src = rf + (size_t)rhs * nx * ny;
  T2 acc = czero<T2>();
  for (int a = -1; a <= 1; ++a) {
    int y = 2 * I + a;
    if (y < 0 || y >= ny) continue;
    T wy = (a == 0) ? T(2) : T(1);
    for (int b = -1; b <= 1; ++b) {
      int x = 2 * J + b;
      if (x < 0 || x >= nx) continue;
      T wgt = wy * ((b == 0) ? T(2) : T(1)) * T(0.0625);
      T2 v = src[(size_t)y * nx + x];
      acc.x += wgt * v.x;
      acc.y += wgt * v.y;
    }
  }
  rc[(size_t)rhs * nxc * nyc + (size_t)I * nxc + J] = acc;
}

// (P e)(i, j): transposed stride-2 convolution with (1/4)[1 2 1; 2 4 2; 1 2 1]
template <typename T>
__device__ __forceinline__ typename vec2<T>::type prolong_at(const typename vec2<T>::type* ec, int nxc, int nyc,
                                                             int i, int j) {
  typedef typename vec2<T>::type T2;
  int I0, I1, J0, J1;
  T wy0, wy1, wx0, wx1;
  if ((i & 1) == 0) { I0 = i >> 1; I1 = -1; wy0 = T(1); wy1 = T(0); }
  else { I0 = i >> 1; I1 = (i >> 1) + 1; wy0 = T(0.5); wy1 = T(0.5); if (I1 >= nyc) I1 = -1; }
  if ((j & 1) == 0) { J0 = j >> 1; J1 = -1; wx0 = T(1); wx1 = T(0); }
  else { J0 = j >> 1; J1 = (j >> 1) + 1; wx0 = T(0.5); wx1 = T(0.5); if (J1 >= nxc) J1 = -1; }
  T2 acc = czero<T2>();
  if (I0 < nyc) {
    const T2* row = ec + (size_t)I0 * nxc;
    if (J0 < nxc) { T2 v = row[J0]; acc.x += wy0 * wx0 * v.x; acc.y += wy0 * wx0 * v.y; }
    if (J1 >= 0) { T2 v = row[J1]; acc.x += wy0 * wx1 * v.x; acc.y += wy0 * wx1 * v.y; }
  }
  if (I1 >= 0) {
    const T2* row = ec + (size_t)I1 * nxc;
    if (J0 < nxc) { T2 v = row[J0]; acc.x += wy1 * wx0 * v.x; acc.y += wy1 * wx0 * v.y; }
    if (J1 >= 0) { T2 v = row[J1]; acc.x += wy1 * wx1 * v.x; acc.y += wy1 * wx1 * v.y; }
  }
  return acc;
}

// xf += P ec
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(int nxc, int nyc, int nx, int ny,
                                                     const typename vec2<T>::type* __restrict__ ec,
                                                     typename vec2<T>::type* __restrict__ xf, const int* active) {
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const int j = blockIdx.x * BX + threadIdx.x, i = blockIdx.y * BY + threadIdx.y;
  if (j >= nx || i >= ny) return;
  auto add = prolong_at<T>(ec + (size_t)rhs * nxc * nyc, nxc, nyc, i, j);
  size_t p = (size_t)rhs * nx * ny + (size_t)i * nx + j;
  auto v = xf[p];
  v.x += add.x; v.y += add.y;
  xf[p] = v;
}

// ---------------------------------------------------------------------------
// Fused: f_c = R (f - K v) over a coarse tile of BY x BX points.
// v == nullptr: v = w D^-1 f (one Jacobi sweep from a zero guess), computed in
// shared memory for the tile plus a 2-node halo, never written to memory.
// ---------------------------------------------------------------------------
constexpr int RR_Y = 2 * BY + 3, RR_X = 2 * BX + 3;  // v region (fine), halo 2
constexpr int RI_Y = 2 * BY + 1, RI_X = 2 * BX + 1;  // residual region, halo 1

template <typename T, int ORD>
__global__ void __launch_bounds__(256) k_resid_restrict(Op<T> op, T w, const typename vec2<T>::type* __restrict__ f,
                                                        const typename vec2<T>::type* __restrict__ v,
                                                        typename vec2<T>::type* __restrict__ fc,
                                                        const int* active) {
  typedef typename vec2<T>::type T2;
  __shared__ T2 s_v[RR_Y][RR_X];
  __shared__ T2 s_r[RI_Y][RI_X];
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const int nx = op.nx, ny = op.ny, nxc = nx / 2, nyc = ny / 2;
  const size_t N = (size_t)nx * ny;
  const T2* fr = f + (size_t)rhs * N;
  const T2* vr = v ? v + (size_t)rhs * N : nullptr;
  const int I0 = blockIdx.y * BY, J0 = blockIdx.x * BX;
  const int fy0 = 2 * I0 - 2, fx0 = 2 * J0 - 2;
  const int tid = threadIdx.y * BX + threadIdx.x;
  // 1) v on the region, f on the inner (residual) region
  for (int q = tid; q < RR_Y * RR_X; q += BX * BY) {
    int ry = q / RR_X, rx = q - ry * RR_X;
    int y = fy0 + ry, x = fx0 + rx;
    T2 vv = czero<T2>(), ff = czero<T2>();
    if (y >= 0 && y < ny && x >= 0 && x < nx) {
      size_t p = (size_t)y * nx + x;
      ff = fr[p];
      vv = vr ? vr[p] : cscale(cmul(ff, cinv(diag_at(op, x, y))), w);
    }
    s_v[ry][rx] = vv;
    if (ry >= 1 && ry <= RI_Y && rx >= 1 && rx <= RI_X) s_r[ry - 1][rx - 1] = ff;
  }
  __syncthreads();
  // 2) r = f - K v on the inner region (zero outside the grid)
  for (int q = tid; q < RI_Y * RI_X; q += BX * BY) {
    int ry = q / RI_X, rx = q - ry * RI_X;
    int y = fy0 + 1 + ry, x = fx0 + 1 + rx;
    if (y >= 0 && y < ny && x >= 0 && x < nx) {
      int sy = ry + 1, sx = rx + 1;
      T2 c = s_v[sy][sx];
      // neighbours inside the grid, from the tile (boundary terms in stencil_sum / diag_at)
      const T2 s = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) { return s_v[sy + dy][sx + dx]; });
      T2 kv = cmul(diag_at(op, x, y), c);
      kv.x -= s.x * op.inv_h2;
      kv.y -= s.y * op.inv_h2;
      s_r[ry][rx] = csub(s_r[ry][rx], kv);
    }
  }
  __syncthreads();
  // 3) full weighting
  const int I = I0 + threadIdx.y, J = J0 + threadIdx.x;
  if (I < nyc && J < nxc) {
    const int cy = 2 * threadIdx.y + 1, cx = 2 * threadIdx.x + 1;
    T2 acc = czero<T2>();
#pragma unroll
    for (int a = -1; a <= 1; ++a) {
      T wy = (a == 0) ? T(2) : T(1);
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        T wgt = wy * ((b == 0) ? T(2) : T(1)) * T(0.0625);
        T2 r = s_r[cy + a][cx + b];
        acc.x += wgt * r.x;
        acc.y += wgt * r.y;
      }
    }
    fc[(size_t)rhs * nxc * nyc + (size_t)I * nxc + J] = acc;
  }
}

// ---------------------------------------------------------------------------
// Fused: out = x + w D^-1 (f - K x) with x = v + P e_c, on a fine BY x BX tile.
// v == nullptr: v = w D^-1 f when implicit_v (the pre-smoothing result from a
// zero guess), else v = 0.
// ---------------------------------------------------------------------------
template <typename T, int ORD>
__global__ void __launch_bounds__(256) k_prolong_jacobi(Op<T> op, T w, const typename vec2<T>::type* __restrict__ f,
                                                        const typename vec2<T>::type* __restrict__ v,
                                                        int implicit_v, const typename vec2<T>::type* __restrict__ ec,
                                                        int nxc, int nyc, typename vec2<T>::type* __restrict__ out,
                                                        const int* active) {
  typedef typename vec2<T>::type T2;
  __shared__ T2 s_x[BY + 2][BX + 2];
  const int rhs = blockIdx.z;
  if (active && !active[rhs]) return;
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const T2* fr = f + (size_t)rhs * N;
  const T2* vr = v ? v + (size_t)rhs * N : nullptr;
  const T2* er = ec + (size_t)rhs * nxc * nyc;
  const int y0 = blockIdx.y * BY - 1, x0 = blockIdx.x * BX - 1;
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int q = tid; q < (BY + 2) * (BX + 2); q += BX * BY) {
    int ry = q / (BX + 2), rx = q - ry * (BX + 2);
    int y = y0 + ry, x = x0 + rx;
    T2 xv = czero<T2>();
    if (y >= 0 && y < ny && x >= 0 && x < nx) {
      size_t p = (size_t)y * nx + x;
      T2 base = vr ? vr[p] : (implicit_v ? cscale(cmul(fr[p], cinv(diag_at(op, x, y))), w) : czero<T2>());
      xv = cadd(base, prolong_at<T>(er, nxc, nyc, y, x));
    }
    s_x[ry][rx] = xv;
  }
  __syncthreads();
  const int y = blockIdx.y * BY + threadIdx.y, x = blockIdx.x * BX + threadIdx.x;
  if (y < ny && x < nx) {
    const int sy = threadIdx.y + 1, sx = threadIdx.x + 1;
    T2 c = s_x[sy][sx];
    const T2 s = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) { return s_x[sy + dy][sx + dx]; });
    T2 d = diag_at(op, x, y);
    T2 kx = cmul(d, c);
    kx.x -= s.x * op.inv_h2;
    kx.y -= s.y * op.inv_h2;
    size_t p = (size_t)y * nx + x;
    T2 r = csub(fr[p], kx);
    out[(size_t)rhs * N + p] = cadd(c, cscale(cmul(r, cinv(d)), w));
  }
}

// Coarse medium: full weighting of k^2 renormalised by the in-domain weights.
__global__ void k_coarsen_kappa2(const double* __restrict__ k2f, int nx, int ny, double* __restrict__ k2d_c,
                                 float* __restrict__ k2f_c) {
  const int nxc = nx / 2, nyc = ny / 2;
  const int J = blockIdx.x * BX + threadIdx.x, I = blockIdx.y * BY + threadIdx.y;
  if (J >= nxc || I >= nyc) return;
  double acc = 0.0, wsum = 0.0;
  for (int a = -1; a <= 1; ++a) {
    int y = 2 * I + a;
    if (y < 0 || y >= ny) continue;
    double wy = (a == 0) ? 2.0 : 1.0;
    for (int b = -1; b <= 1; ++b) {
      int x = 2 * J + b;
      if (x < 0 || x >= nx) continue;
      double wgt = wy * ((b == 0) ? 2.0 : 1.0) / 16.0;
      acc += wgt * k2f[(size_t)y * nx + x];
      wsum += wgt;
    }
  }
  double c = acc / wsum;
  k2d_c[(size_t)I * nxc + J] = c;
  k2f_c[(size_t)I * nxc + J] = (float)c;
}

__global__ void k_widen(const float* __restrict__ a, double* __restrict__ b, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

inline dim3 grid2(int nx, int ny, int nrhs) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY, nrhs); }

}  // namespace

template <typename T>
void launch_apply(const Op<T>& op, const void* x, const void* b, void* y, int nrhs, const int* active, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  auto k = op.order == 4 ? k_apply<T, 4> : k_apply<T, 2>;
  k<<<grid2(op.nx, op.ny, nrhs), dim3(BX, BY), 0, s>>>(op, (const T2*)x, (const T2*)b, (T2*)y, active);
}
template <typename T>
void launch_rhs_weight(const Op<T>& op, const void* x, void* y, int nrhs, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_rhs_weight<T><<<grid2(op.nx, op.ny, nrhs), dim3(BX, BY), 0, s>>>(op.nx, op.ny, (const T2*)x, (T2*)y);
}
template <typename T>
void launch_jacobi(const Op<T>& op, T w, const void* f, const void* x_in, void* x_out, int nrhs, const int* active,
                   cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  auto k = op.order == 4 ? k_jacobi<T, 4> : k_jacobi<T, 2>;
  k<<<grid2(op.nx, op.ny, nrhs), dim3(BX, BY), 0, s>>>(op, w, (const T2*)f, (const T2*)x_in, (T2*)x_out, active);
}
template <typename T>
void launch_restrict(int nx, int ny, const void* rf, void* rc, int nrhs, const int* active, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_restrict<T><<<grid2(nx / 2, ny / 2, nrhs), dim3(BX, BY), 0, s>>>(nx, ny, (const T2*)rf, (T2*)rc, active);
}
template <typename T>
void launch_prolong_add(int nxc, int nyc, int nx, int ny, const void* ec, void* xf, int nrhs, const int* active,
                        cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  k_prolong_add<T><<<grid2(nx, ny, nrhs), dim3(BX, BY), 0, s>>>(nxc, nyc, nx, ny, (const T2*)ec, (T2*)xf, active);
}
template <typename T>
void launch_resid_restrict(const Op<T>& fine, T w, const void* f, const void* v, void* fc, int nrhs,
                           const int* active, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  auto k = fine.order == 4 ? k_resid_restrict<T, 4> : k_resid_restrict<T, 2>;
  k<<<grid2(fine.nx / 2, fine.ny / 2, nrhs), dim3(BX, BY), 0, s>>>(fine, w, (const T2*)f, (const T2*)v, (T2*)fc,
                                                                   active);
}
template <typename T>
void launch_prolong_jacobi(const Op<T>& fine, T w, const void* f, const void* v, bool implicit_v, const void* ec,
                           int nxc, int nyc, void* out, int nrhs, const int* active, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  auto k = fine.order == 4 ? k_prolong_jacobi<T, 4> : k_prolong_jacobi<T, 2>;
  k<<<grid2(fine.nx, fine.ny, nrhs), dim3(BX, BY), 0, s>>>(fine, w, (const T2*)f, (const T2*)v, implicit_v ? 1 : 0,
                                                           (const T2*)ec, nxc, nyc, (T2*)out, active);
}
void launch_coarsen_kappa2(const double* k2d_fine, int nx, int ny, double* k2d_coarse, float* k2f_coarse,
                           cudaStream_t s) {
  k_coarsen_kappa2<<<grid2(nx / 2, ny / 2, 1), dim3(BX, BY), 0, s>>>(k2d_fine, nx, ny, k2d_coarse, k2f_coarse);
}
void launch_widen_kappa2(const float* k2f, double* k2d, size_t n, cudaStream_t s) {
  k_widen<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(k2f, k2d, n);
}

#define INST(T)                                                                                                 \
  template void launch_apply<T>(const Op<T>&, const void*, const void*, void*, int, const int*, cudaStream_t); \
  template void launch_rhs_weight<T>(const Op<T>&, const void*, void*, int, cudaStream_t);                    \
  template void launch_jacobi<T>(const Op<T>&, T, const void*, const void*, void*, int, const int*,            \
                                 cudaStream_t);                                                               \
  template void launch_restrict<T>(int, int, const void*, void*, int, const int*, cudaStream_t);              \
  template void launch_prolong_add<T>(int, int, int, int, const void*, void*, int, const int*, cudaStream_t);  \
  template void launch_resid_restrict<T>(const Op<T>&, T, const void*, const void*, void*, int, const int*,    \
                                         cudaStream_t);                                                       \
  template void launch_prolong_jacobi<T>(const Op<T>&, T, const void*, const void*, bool, const void*, int,   \
                                         int, void*, int, const int*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace helm
