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
#include <cstdint>
#include <type_traits>

#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int BX = 32, BY = 8;  // 256 threads

// Boundary mode and stencil order as template arguments: every operator kernel is
// instantiated for the 5-point stencil with each boundary mode and for the compact
// scheme (Dirichlet), so no runtime branch on either remains in the inner loops.
template <int O, int B> struct Kind { static constexpr int ORD = O, BC = B; };
template <typename F> void with_kind(int order, int bc, F f) {
  if (order == 4) f(Kind<4, kBcDirichlet>());
  else if (bc == kBcReflect) f(Kind<2, kBcReflect>());
  else if (bc == kBcReplicate) f(Kind<2, kBcReplicate>());
  else f(Kind<2, kBcDirichlet>());
}

template <int ORD, int BC, typename T>
__device__ __forceinline__ typename vec2<T>::type apply_at(const Op<T>& op, const typename vec2<T>::type* u,
                                                           int x, int y) {
  typedef typename vec2<T>::type T2;
  size_t p = (size_t)y * op.nx + x;
  T2 c = u[p];
  const T2 s = stencil_sum<ORD, BC>(op, x, y, [&](int dx, int dy) { return u[(ptrdiff_t)p + (ptrdiff_t)dy * op.nx + dx]; });
  T2 d = diag_at<BC, ORD>(op, x, y);
  T2 r = cmul(d, c);
  r.x -= s.x * op.inv_h2;
  r.y -= s.y * op.inv_h2;
  return r;
}

// y = K x  (b == nullptr)   or   y = b - K x
template <typename T, int ORD, int BC>
__global__ void __launch_bounds__(256) k_apply(Op<T> op, const typename vec2<T>::type* __restrict__ x,
                                               const typename vec2<T>::type* __restrict__ b,
                                               typename vec2<T>::type* __restrict__ y, const int* active) {
  const int rhs = blockIdx.z;
  select_medium(op, rhs);
  if (active && !active[rhs]) return;
  const int ix = blockIdx.x * BX + threadIdx.x, iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= op.nx || iy >= op.ny) return;
  const size_t N = (size_t)op.nx * op.ny, off = (size_t)rhs * N, p = (size_t)iy * op.nx + ix;
  auto ku = apply_at<ORD, BC>(op, x + off, ix, iy);
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
template <typename T, int ORD, int BC>
__global__ void __launch_bounds__(256) k_jacobi(Op<T> op, T w, const typename vec2<T>::type* __restrict__ f,
                                                const typename vec2<T>::type* __restrict__ xin,
                                                typename vec2<T>::type* __restrict__ xout, const int* active) {
  typedef typename vec2<T>::type T2;
  const int rhs = blockIdx.z;
  select_medium(op, rhs);
  if (active && !active[rhs]) return;
  const int ix = blockIdx.x * BX + threadIdx.x, iy = blockIdx.y * BY + threadIdx.y;
  if (ix >= op.nx || iy >= op.ny) return;
  const size_t N = (size_t)op.nx * op.ny, off = (size_t)rhs * N, p = (size_t)iy * op.nx + ix;
  T2 r = f[off + p];
  if (xin) r = csub(r, apply_at<ORD, BC>(op, xin + off, ix, iy));
  T2 c = cscale(cmul(r, crecip(diag_at<BC, ORD>(op, ix, iy))), w);
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
// Fused: f_c = R (f - K v) over a coarse tile of (BY RPT) x BX points.
// v == nullptr: v = w D^-1 f (one Jacobi sweep from a zero guess), computed in
// shared memory for the tile plus a 2-node halo, never written to memory.
// Shared memory: v on the fine region (halo 2), f and kappa^2 on the residual region
// (halo 1); the residual overwrites f.  Each fine node's diagonal is formed twice
// (for v and for the residual) from kappa^2 without a division; D^-1 costs one
// reciprocal.  RPT (coarse rows per thread) sets the tile height.
// ---------------------------------------------------------------------------
template <typename T, int ORD, int BC, int RPT>
__global__ void __launch_bounds__(256) k_resid_restrict(Op<T> op, T w, const typename vec2<T>::type* __restrict__ f,
                                                        const typename vec2<T>::type* __restrict__ v,
                                                        typename vec2<T>::type* __restrict__ fc,
                                                        const int* active) {
  typedef typename vec2<T>::type T2;
  constexpr int TY = BY * RPT;                     // coarse rows per tile
  constexpr int RY = 2 * TY + 3, RX = 2 * BX + 3;  // v region (fine), halo 2
  constexpr int IY = 2 * TY + 1, IX = 2 * BX + 1;  // residual region, halo 1
  __shared__ T2 s_v[RY][RX];
  __shared__ T2 s_r[IY][IX];
  __shared__ T s_k[IY][IX];
  const int rhs = blockIdx.z;
  select_medium(op, rhs);
  if (active && !active[rhs]) return;
  const int nx = op.nx, ny = op.ny, nxc = nx / 2, nyc = ny / 2;
  const size_t N = (size_t)nx * ny;
  const T2* fr = f + (size_t)rhs * N;
  const T2* vr = v ? v + (size_t)rhs * N : nullptr;
  const int I0 = blockIdx.y * TY, J0 = blockIdx.x * BX;
  const int fy0 = 2 * I0 - 2, fx0 = 2 * J0 - 2;
  const int tid = threadIdx.y * BX + threadIdx.x;
  // 1) v on the region; f and kappa^2 on the inner (residual) region
  for (int q = tid; q < RY * RX; q += BX * BY) {
    const int ry = q / RX, rx = q - ry * RX;
    const int y = fy0 + ry, x = fx0 + rx;
    T2 vv = czero<T2>(), ff = czero<T2>();
    T kk = T(0);
    if (y >= 0 && y < ny && x >= 0 && x < nx) {
      const size_t p = (size_t)y * nx + x;
      ff = fr[p];
      kk = op.k2[p];
      vv = vr ? vr[p] : cscale(cmul(ff, crecip(diag_k2<BC, ORD>(op, x, y, kk))), w);
    }
    s_v[ry][rx] = vv;
    if (ry >= 1 && ry <= IY && rx >= 1 && rx <= IX) {
      s_r[ry - 1][rx - 1] = ff;
      s_k[ry - 1][rx - 1] = kk;
    }
  }
  __syncthreads();
  // 2) r = f - K v on the inner region (zero outside the grid)
  for (int q = tid; q < IY * IX; q += BX * BY) {
    const int ry = q / IX, rx = q - ry * IX;
    const int y = fy0 + 1 + ry, x = fx0 + 1 + rx;
    if (y >= 0 && y < ny && x >= 0 && x < nx) {
      const int sy = ry + 1, sx = rx + 1;
      const T2 s = stencil_sum<ORD, BC>(op, x, y, [&](int dx, int dy) { return s_v[sy + dy][sx + dx]; });
      T2 kv = cmul(diag_k2<BC, ORD>(op, x, y, s_k[ry][rx]), s_v[sy][sx]);
      kv.x -= s.x * op.inv_h2;
      kv.y -= s.y * op.inv_h2;
      s_r[ry][rx] = csub(s_r[ry][rx], kv);
    }
  }
  __syncthreads();
  // 3) full weighting
  const int J = J0 + threadIdx.x;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int ty = threadIdx.y + k * BY, I = I0 + ty;
    if (I < nyc && J < nxc) {
      const int cy = 2 * ty + 1, cx = 2 * threadIdx.x + 1;
      T2 acc = czero<T2>();
#pragma unroll
      for (int a = -1; a <= 1; ++a) {
        const T wy = (a == 0) ? T(2) : T(1);
#pragma unroll
        for (int b = -1; b <= 1; ++b) {
          const T wgt = wy * ((b == 0) ? T(2) : T(1)) * T(0.0625);
          const T2 r = s_r[cy + a][cx + b];
          acc.x += wgt * r.x;
          acc.y += wgt * r.y;
        }
      }
      fc[(size_t)rhs * nxc * nyc + (size_t)I * nxc + J] = acc;
    }
  }
}

// ---------------------------------------------------------------------------
// Fused: out = x + w D^-1 (f - K x) with x = v + P e_c, on a fine (BY RPT) x BX tile.
// v == nullptr: v = w D^-1 f when implicit_v (the pre-smoothing result from a
// zero guess), else v = 0.  x on the tile plus a 1-node halo in shared memory; f
// and kappa^2 of the tile's own nodes too.
// ---------------------------------------------------------------------------
template <typename T, int ORD, int BC, int RPT>
__global__ void __launch_bounds__(256) k_prolong_jacobi(Op<T> op, T w, const typename vec2<T>::type* __restrict__ f,
                                                        const typename vec2<T>::type* __restrict__ v,
                                                        int implicit_v, const typename vec2<T>::type* __restrict__ ec,
                                                        int nxc, int nyc, typename vec2<T>::type* __restrict__ out,
                                                        const int* active) {
  typedef typename vec2<T>::type T2;
  constexpr int TY = BY * RPT;
  __shared__ T2 s_x[TY + 2][BX + 2];
  __shared__ T2 s_f[TY][BX];
  __shared__ T s_k[TY][BX];
  const int rhs = blockIdx.z;
  select_medium(op, rhs);
  if (active && !active[rhs]) return;
  const int nx = op.nx, ny = op.ny;
  const size_t N = (size_t)nx * ny;
  const T2* fr = f + (size_t)rhs * N;
  const T2* vr = v ? v + (size_t)rhs * N : nullptr;
  const T2* er = ec + (size_t)rhs * nxc * nyc;
  const int y0 = blockIdx.y * TY - 1, x0 = blockIdx.x * BX - 1;
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int q = tid; q < (TY + 2) * (BX + 2); q += BX * BY) {
    const int ry = q / (BX + 2), rx = q - ry * (BX + 2);
    const int y = y0 + ry, x = x0 + rx;
    T2 xv = czero<T2>();
    if (y >= 0 && y < ny && x >= 0 && x < nx) {
      const size_t p = (size_t)y * nx + x;
      const bool inner = ry >= 1 && ry <= TY && rx >= 1 && rx <= BX;
      T2 ff = czero<T2>();
      T kk = T(0);
      if (implicit_v || inner) ff = fr[p];
      if (implicit_v || inner) kk = op.k2[p];
      const T2 base = vr ? vr[p]
                         : (implicit_v ? cscale(cmul(ff, crecip(diag_k2<BC, ORD>(op, x, y, kk))), w) : czero<T2>());
      xv = cadd(base, prolong_at<T>(er, nxc, nyc, y, x));
      if (inner) {
        s_f[ry - 1][rx - 1] = ff;
        s_k[ry - 1][rx - 1] = kk;
      }
    }
    s_x[ry][rx] = xv;
  }
  __syncthreads();
  const int x = blockIdx.x * BX + threadIdx.x;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int ty = threadIdx.y + k * BY, y = blockIdx.y * TY + ty;
    if (y < ny && x < nx) {
      const int sy = ty + 1, sx = threadIdx.x + 1;
      const T2 c = s_x[sy][sx];
      const T2 s = stencil_sum<ORD, BC>(op, x, y, [&](int dx, int dy) { return s_x[sy + dy][sx + dx]; });
      const T2 d = diag_k2<BC, ORD>(op, x, y, s_k[ty][threadIdx.x]);
      T2 kx = cmul(d, c);
      kx.x -= s.x * op.inv_h2;
      kx.y -= s.y * op.inv_h2;
      const T2 r = csub(s_f[ty][threadIdx.x], kx);
      out[(size_t)rhs * N + (size_t)y * nx + x] = cadd(c, cscale(cmul(r, crecip(d)), w));
    }
  }
}

// ---------------------------------------------------------------------------
// Column-strip ("marching") forms of the two fused cycle kernels, FP32, 5-point
// stencil.  A warp holds 64 consecutive fine columns (two per lane, 16-byte loads)
// and walks down the rows of its segment, keeping the rows the stencil needs in
// registers: left and right neighbours come from the adjacent lanes by shuffles,
// those above and below from the previous and next rows.  No shared memory, no
// block barrier, and each node's diagonal and Jacobi value are formed once.  The
// strip's outer lanes 0 and 31 only supply the halo: a strip produces 60 fine
// columns (30 coarse ones), strips start every 60 fine columns, and a segment
// recomputes 2-3 halo rows.  The segment height (TI coarse rows for the
// restriction, TY fine rows for the prolongation) trades that row halo against
// the number of warps; the launchers take it from the tile tuner.
// ---------------------------------------------------------------------------
constexpr int kStripW = 60;          // fine columns a strip produces
constexpr int kStripWarps = 4;       // warps (strips) per block

struct CPair { float2 a, b; };       // complex values of columns c0 and c0 + 1

__device__ __forceinline__ CPair cp_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ void st_pair(float2* p, CPair v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.a.x, v.a.y, v.b.x, v.b.y);
}
__device__ __forceinline__ float2 shfl_up1(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_dn1(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}
// w f / D with one approximate reciprocal of |D|^2 (2 ulp; the FP32 stencils' tolerance is 1e-5).
__device__ __forceinline__ float2 jacobi_from_zero(float2 f, float2 d, float w) {
  const float r = __fdividef(w, d.x * d.x + d.y * d.y);
  return make_float2((f.x * d.x + f.y * d.y) * r, (f.y * d.x - f.x * d.y) * r);
}
// K u at (x, y) = D u - s / h^2 from the node's value c and its four neighbours.
template <int BC>
__device__ __forceinline__ float2 op_at(const Op<float>& op, int x, int y, float2 d, float2 c, float2 l, float2 r,
                                        float2 dn, float2 up) {
  const float2 s = stencil_sum<2, BC>(op, x, y, [&](int dx, int dy) {
    return dx < 0 ? l : dx > 0 ? r : dy < 0 ? dn : up;
  });
  float2 k = cmul(d, c);
  k.x -= s.x * op.inv_h2;
  k.y -= s.y * op.inv_h2;
  return k;
}

// Rows of a strip away from every boundary and the absorbing layer: there g = 0, no
// neighbour is outside the grid and no boundary mode applies, so the diagonal and the
// stencil take their plain forms (for the strip of 64 columns from xs; the test is uniform
// over a warp).  strip_interior_cols: the strip's columns qualify (tested once per strip);
// strip_interior_row: row y does (from the kernel parameters, no registers held);
// strip_interior: both, tested per row.
__device__ __forceinline__ int interior_margin(const Op<float>& op) { return op.abc_w > 1 ? op.abc_w : 1; }
__device__ __forceinline__ bool strip_interior_cols(const Op<float>& op, int xs) {
  return xs >= interior_margin(op) && xs + 63 < op.nx - interior_margin(op);
}
__device__ __forceinline__ bool strip_interior_row(const Op<float>& op, int y) {
  return y >= interior_margin(op) && y < op.ny - interior_margin(op);
}
__device__ __forceinline__ bool strip_interior(const Op<float>& op, int xs, int y) {
  const int A = interior_margin(op);
  return y >= A && y < op.ny - A && xs >= A && xs + 63 < op.nx - A;
}
__device__ __forceinline__ float2 diag_plain(const Op<float>& op, float k2) {
  const float wk = op.omega2 * k2;
  return make_float2(4.f * op.inv_h2 - wk, wk * op.beta);
}
__device__ __forceinline__ float2 op_plain(const Op<float>& op, float2 d, float2 c, float2 l, float2 r, float2 dn,
                                           float2 up) {
  float2 k = cmul(d, c);
  const float2 s = cadd(cadd(l, r), cadd(dn, up));   // the general form's summation order
  k.x -= s.x * op.inv_h2;
  k.y -= s.y * op.inv_h2;
  return k;
}

// Row staging: each lane copies its own two columns of the rows ahead into a per-warp ring
// in shared memory with cp.async (zero-filled outside the grid) and reads them back when
// the walk reaches them, so that kRing - 1 rows per warp are in flight instead of the one
// a register prefetch allows.  A lane reads only the slots it wrote itself, so the
// group wait orders everything and no barrier is needed; a slot is refilled one row
// after it was read.
constexpr int kRing = 4;
__device__ __forceinline__ void row_cp16(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void row_cp8(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 8 : 0) : "memory");
}
__device__ __forceinline__ void row_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void row_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(kRing - 2) : "memory"); }
__device__ __forceinline__ CPair cp_of(float4 q) { return {make_float2(q.x, q.y), make_float2(q.z, q.w)}; }

// f_c = R (f - K v) (v == nullptr: v = w D^-1 f) for coarse rows [I0, I0 + TI) of one strip;
// HAS_V: v is given.
template <int BC, int TI, bool HAS_V>
__global__ void __launch_bounds__(32 * kStripWarps, 8) k_resid_restrict_m(Op<float> op, float w,
                                                                     const float2* __restrict__ f,
                                                                     const float2* __restrict__ v,
                                                                     float2* __restrict__ fc, const int* active,
                                                                     int nstrips) {
  constexpr int R = 2 * TI + 3;                  // fine rows 2 I0 - 2 .. 2 I0 + 2 TI
  __shared__ float4 s_f[kStripWarps][kRing][32];
  __shared__ float2 s_k[kStripWarps][kRing][32];
  __shared__ float4 s_v[HAS_V ? kStripWarps : 1][kRing][32];
  const int rhs = blockIdx.z;
  select_medium(op, rhs);
  if (active && !active[rhs]) return;
  const int wi = threadIdx.x >> 5;
  const int strip = blockIdx.x * kStripWarps + wi;
  if (strip >= nstrips) return;                  // uniform per warp
  const int lane = threadIdx.x & 31;
  const int nx = op.nx, ny = op.ny, nxc = nx >> 1, nyc = ny >> 1;
  const int xs = strip * kStripW - 2;              // first column of the strip
  const int c0 = xs + 2 * lane;                    // even
  const bool colin = c0 >= 0 && c0 < nx;           // both columns in or both out (nx even)
  const size_t N = (size_t)nx * ny;
  const float2* fr = f + (size_t)rhs * N;
  const float2* vr = HAS_V ? v + (size_t)rhs * N : nullptr;
  const int I0 = blockIdx.y * TI;
  const int ys = 2 * I0 - 2;                       // fine row of ring index 0
  const bool incols = strip_interior_cols(op, xs);
  auto issue = [&](int i) {
    if (i < R) {
      const int yy = ys + i, sl = i % kRing;
      const bool ok = colin && yy >= 0 && yy < ny;
      const int p = ok ? yy * nx + c0 : 0;         // one right-hand side holds < 2^31 nodes
      row_cp16(&s_f[wi][sl][lane], fr + p, ok);
      row_cp8(&s_k[wi][sl][lane], op.k2 + p, ok);
      if (HAS_V) row_cp16(&s_v[HAS_V ? wi : 0][sl][lane], vr + p, ok);
    }
    row_commit();
  };
  // ring row i: f, v (or w D^-1 f), the diagonal of both columns and whether the row is
  // interior (strip_interior_cols and strip_interior_row)
  auto take = [&](int i, CPair& ff, CPair& vv, CPair& dd, bool& in) {
    row_wait();
    const int yy = ys + i, sl = i % kRing;
    ff = cp_of(s_f[wi][sl][lane]);
    const float2 k = s_k[wi][sl][lane];
    vv = HAS_V ? cp_of(s_v[HAS_V ? wi : 0][sl][lane]) : cp_zero();
    dd = cp_zero();
    in = incols && strip_interior_row(op, yy);
    if (colin && yy >= 0 && yy < ny) {
      if (in) {
        dd.a = diag_plain(op, k.x);
        dd.b = diag_plain(op, k.y);
      } else {
        dd.a = diag_k2<BC, 2>(op, c0, yy, k.x);
        dd.b = diag_k2<BC, 2>(op, c0 + 1, yy, k.y);
      }
      if (!HAS_V) {
        vv.a = jacobi_from_zero(ff.a, dd.a, w);
        vv.b = jacobi_from_zero(ff.b, dd.b, w);
      }
    }
    issue(i + kRing - 1);
  };
#pragma unroll
  for (int i = 0; i < kRing - 1; ++i) issue(i);
  CPair vm = cp_zero(), v0, d0, f0, vp, dp, fp, ra = cp_zero(), rb = cp_zero();
  bool in0, inp;
  take(0, f0, v0, d0, in0);
  float2* fco = fc + (size_t)rhs * nxc * nyc;
#pragma unroll 4
  for (int i = 1; i < R; ++i) {
    take(i, fp, vp, dp, inp);
    const int y = ys + i - 1;                      // the row whose residual is formed
    if (i >= 2) {
      const float2 lft = shfl_up1(v0.b), rgt = shfl_dn1(v0.a);
      CPair rc = cp_zero();
      if (in0) {
        rc.a = csub(f0.a, op_plain(op, d0.a, v0.a, lft, v0.b, vm.a, vp.a));
        rc.b = csub(f0.b, op_plain(op, d0.b, v0.b, v0.a, rgt, vm.b, vp.b));
      } else if (colin && y >= 0 && y < ny) {
        rc.a = csub(f0.a, op_at<BC>(op, c0, y, d0.a, v0.a, lft, v0.b, vm.a, vp.a));
        rc.b = csub(f0.b, op_at<BC>(op, c0 + 1, y, d0.b, v0.b, v0.a, rgt, vm.b, vp.b));
      }
      if ((y & 1) && y >= 2 * I0 + 1) {          // coarse row (y - 1) / 2 is complete
        CPair rv;
        rv.a = cadd(cadd(ra.a, rc.a), cscale(rb.a, 2.f));
        rv.b = cadd(cadd(ra.b, rc.b), cscale(rb.b, 2.f));
        const float2 left = shfl_up1(rv.b);
        const int I = (y - 1) >> 1, J = c0 >> 1;
        if (lane >= 1 && lane <= 30 && I < nyc && J < nxc)
          fco[(size_t)I * nxc + J] = cscale(cadd(cadd(left, rv.b), cscale(rv.a, 2.f)), 0.0625f);
      }
      ra = rb;
      rb = rc;
    }
    vm = v0; v0 = vp; f0 = fp; d0 = dp; in0 = inp;
  }
}

// out = x + w D^-1 (f - K x), x = v + P e_c (v == nullptr: v = w D^-1 f if implicit_v,
// else 0), for fine rows [Y0, Y0 + TY) of one strip; HAS_V: v is given.
template <int BC, int TY, bool HAS_V>
__global__ void __launch_bounds__(32 * kStripWarps, 8) k_prolong_jacobi_m(Op<float> op, float w,
                                                                     const float2* __restrict__ f,
                                                                     const float2* __restrict__ v, int implicit_v,
                                                                     const float2* __restrict__ ec, int nxc, int nyc,
                                                                     float2* __restrict__ out, const int* active,
                                                                     int nstrips) {
  constexpr int R = TY + 2;                      // fine rows Y0 - 1 .. Y0 + TY
  __shared__ float4 s_f[kStripWarps][kRing][32];
  __shared__ float2 s_k[kStripWarps][kRing][32];
  __shared__ float4 s_v[HAS_V ? kStripWarps : 1][kRing][32];
  __shared__ float2 s_e[kStripWarps][kRing][33];   // coarse row entered at an even fine row
  const int rhs = blockIdx.z;
  select_medium(op, rhs);
  if (active && !active[rhs]) return;
  const int wi = threadIdx.x >> 5;
  const int strip = blockIdx.x * kStripWarps + wi;
  if (strip >= nstrips) return;
  const int lane = threadIdx.x & 31;
  const int nx = op.nx, ny = op.ny;
  const int xs = strip * kStripW - 2;
  const int c0 = xs + 2 * lane;
  const bool colin = c0 >= 0 && c0 < nx;
  const int J = c0 >> 1;                           // coarse column of c0 (c0 + 1 lies between J and J + 1)
  const size_t N = (size_t)nx * ny;
  const float2* fr = f + (size_t)rhs * N;
  const float2* vr = HAS_V ? v + (size_t)rhs * N : nullptr;
  const float2* er = ec + (size_t)rhs * nxc * nyc;
  const int Y0 = blockIdx.y * TY, ys = Y0 - 1;
  // coarse row I at columns J (every lane) and J + 1 of lane 31, zero outside the coarse grid
  auto ec_cp = [&](int I, float2* dst) {
    const bool rin = I >= 0 && I < nyc;
    const bool ok0 = rin && J >= 0 && J < nxc, ok1 = rin && J + 1 < nxc;
    row_cp8(dst + lane, er + (ok0 ? (size_t)I * nxc + J : 0), ok0);
    if (lane == 31) row_cp8(dst + 32, er + (ok1 ? (size_t)I * nxc + J + 1 : 0), ok1);
  };
  auto issue = [&](int i) {
    if (i < R) {
      const int yy = ys + i, sl = i % kRing;
      const bool ok = colin && yy >= 0 && yy < ny;
      const size_t p = ok ? (size_t)yy * nx + c0 : 0;
      row_cp8(&s_k[wi][sl][lane], op.k2 + p, ok);
      const bool fok = ok && (implicit_v || (yy >= Y0 && yy < Y0 + TY));
      row_cp16(&s_f[wi][sl][lane], fr + (fok ? p : 0), fok);
      if (HAS_V) row_cp16(&s_v[HAS_V ? wi : 0][sl][lane], vr + p, ok);
      if (i > 0 && !(yy & 1)) ec_cp((yy >> 1) + 1, &s_e[wi][sl][0]);
    }
    row_commit();
  };
  float2 elo0, elo1, ehi0, ehi1;
  {
    // the two coarse rows around the first fine row, read directly
    auto ec_row = [&](int I, float2& e0, float2& e1) {
      const bool rin = I >= 0 && I < nyc;
      e0 = (rin && J >= 0 && J < nxc) ? er[(size_t)I * nxc + J] : make_float2(0.f, 0.f);
      e1 = shfl_dn1(e0);
      if (lane == 31) e1 = (rin && J + 1 < nxc) ? er[(size_t)I * nxc + J + 1] : make_float2(0.f, 0.f);
    };
    ec_row(ys >> 1, elo0, elo1);
    ec_row((ys >> 1) + 1, ehi0, ehi1);
  }
#pragma unroll
  for (int i = 0; i < kRing - 1; ++i) issue(i);
  CPair xm = cp_zero(), x0 = cp_zero(), f0 = cp_zero(), d0 = cp_zero();
  bool in0 = false;
  float2* o = out + (size_t)rhs * N;
#pragma unroll 4
  for (int i = 0; i < R; ++i) {
    row_wait();
    const int yy = ys + i, sl = i % kRing;
    const CPair fq = cp_of(s_f[wi][sl][lane]);
    const float2 kq = s_k[wi][sl][lane];
    const CPair vq = HAS_V ? cp_of(s_v[HAS_V ? wi : 0][sl][lane]) : cp_zero();
    if (i > 0 && !(yy & 1)) {                     // entering coarse row yy / 2
      elo0 = ehi0; elo1 = ehi1;
      ehi0 = s_e[wi][sl][lane];
      ehi1 = shfl_dn1(ehi0);
      if (lane == 31) ehi1 = s_e[wi][sl][32];
    }
    issue(i + kRing - 1);
    CPair xp = cp_zero(), dp = cp_zero();
    const bool inp = strip_interior(op, xs, yy);
    if (colin && yy >= 0 && yy < ny) {
      if (inp) {
        dp.a = diag_plain(op, kq.x);
        dp.b = diag_plain(op, kq.y);
      } else {
        dp.a = diag_k2<BC, 2>(op, c0, yy, kq.x);
        dp.b = diag_k2<BC, 2>(op, c0 + 1, yy, kq.y);
      }
      CPair base = vq;
      if (!HAS_V && implicit_v) { base.a = jacobi_from_zero(fq.a, dp.a, w); base.b = jacobi_from_zero(fq.b, dp.b, w); }
      // P e_c: even rows take coarse row yy / 2, odd rows the mean of two coarse rows;
      // column c0 = 2J takes coarse column J, column c0 + 1 the mean of J and J + 1
      float2 e0 = elo0, e1 = elo1;
      if (yy & 1) { e0 = cscale(cadd(elo0, ehi0), 0.5f); e1 = cscale(cadd(elo1, ehi1), 0.5f); }
      xp.a = cadd(base.a, e0);
      xp.b = cadd(base.b, cscale(cadd(e0, e1), 0.5f));
    }
    if (i >= 2) {
      const int y = yy - 1;
      const float2 lft = shfl_up1(x0.b), rgt = shfl_dn1(x0.a);
      if (colin && lane >= 1 && lane <= 30 && y < ny) {
        const bool in = in0;
        const float2 ka = in ? op_plain(op, d0.a, x0.a, lft, x0.b, xm.a, xp.a)
                             : op_at<BC>(op, c0, y, d0.a, x0.a, lft, x0.b, xm.a, xp.a);
        const float2 kb = in ? op_plain(op, d0.b, x0.b, x0.a, rgt, xm.b, xp.b)
                             : op_at<BC>(op, c0 + 1, y, d0.b, x0.b, x0.a, rgt, xm.b, xp.b);
        CPair r;
        r.a = cadd(x0.a, jacobi_from_zero(csub(f0.a, ka), d0.a, w));
        r.b = cadd(x0.b, jacobi_from_zero(csub(f0.b, kb), d0.b, w));
        st_pair(o + (size_t)y * nx + c0, r);
      }
    }
    xm = x0; x0 = xp; f0 = fq; d0 = dp; in0 = inp;
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
  with_kind(op.order, op.bc, [&](auto kd) {
    k_apply<T, decltype(kd)::ORD, decltype(kd)::BC><<<grid2(op.nx, op.ny, nrhs), dim3(BX, BY), 0, s>>>(
        op, (const T2*)x, (const T2*)b, (T2*)y, active);
  });
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
  with_kind(op.order, op.bc, [&](auto kd) {
    k_jacobi<T, decltype(kd)::ORD, decltype(kd)::BC><<<grid2(op.nx, op.ny, nrhs), dim3(BX, BY), 0, s>>>(
        op, w, (const T2*)f, (const T2*)x_in, (T2*)x_out, active);
  });
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

// Rows per thread of the fused cycle kernels: taller tiles share their halo over more
// nodes (FP64 keeps one row: its tiles would not fit in static shared memory).
template <typename T> constexpr int fused_rpt() { return sizeof(T) == 4 ? 2 : 1; }

// Segment heights the marching kernels are built for.
template <typename F> bool with_seg(int seg, F f) {
  switch (seg) {
    case 4: f(std::integral_constant<int, 4>()); return true;
    case 8: f(std::integral_constant<int, 8>()); return true;
    case 16: f(std::integral_constant<int, 16>()); return true;
    case 32: f(std::integral_constant<int, 32>()); return true;
    default: return false;
  }
}
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Segment height for a marching launch: the chosen one if it is built, else the
// tallest that still gives about 16 warps per SM.
int march_seg(int chosen, int strips, int rows, int nrhs) {
  if (chosen == 4 || chosen == 8 || chosen == 16 || chosen == 32) return chosen;
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long want = 16ll * (nsm > 0 ? nsm : 148);
  for (int seg : {32, 16, 8})
    if ((long long)strips * ((rows + seg - 1) / seg) * nrhs >= want) return seg;
  return 4;
}

template <typename T>
void launch_resid_restrict(const Op<T>& fine, T w, const void* f, const void* v, void* fc, int nrhs,
                           const int* active, cudaStream_t s, int seg) {
  typedef typename vec2<T>::type T2;
  if (sizeof(T) == 4 && fine.order == 2 && seg >= 0 && aligned16(f) && (!v || aligned16(v))) {
    const Op<float>& op = reinterpret_cast<const Op<float>&>(fine);
    const int nstrips = (fine.nx / 2 + kStripW / 2 - 1) / (kStripW / 2);
    const int ti = march_seg(seg, nstrips, fine.ny / 2, nrhs);
    with_kind(2, fine.bc, [&](auto kd) {
      constexpr int BCk = decltype(kd)::BC;
      with_seg(ti, [&](auto tv) {
        constexpr int TI = decltype(tv)::value;
        const dim3 grid((nstrips + kStripWarps - 1) / kStripWarps, (fine.ny / 2 + TI - 1) / TI, nrhs);
        if (v)
          k_resid_restrict_m<BCk, TI, true><<<grid, 32 * kStripWarps, 0, s>>>(
              op, (float)w, (const float2*)f, (const float2*)v, (float2*)fc, active, nstrips);
        else
          k_resid_restrict_m<BCk, TI, false><<<grid, 32 * kStripWarps, 0, s>>>(
              op, (float)w, (const float2*)f, nullptr, (float2*)fc, active, nstrips);
      });
    });
    return;
  }
  constexpr int RPT = fused_rpt<T>();
  with_kind(fine.order, fine.bc, [&](auto kd) {
    const dim3 grid((fine.nx / 2 + BX - 1) / BX, (fine.ny / 2 + BY * RPT - 1) / (BY * RPT), nrhs);
    k_resid_restrict<T, decltype(kd)::ORD, decltype(kd)::BC, RPT><<<grid, dim3(BX, BY), 0, s>>>(
        fine, w, (const T2*)f, (const T2*)v, (T2*)fc, active);
  });
}
template <typename T>
void launch_prolong_jacobi(const Op<T>& fine, T w, const void* f, const void* v, bool implicit_v, const void* ec,
                           int nxc, int nyc, void* out, int nrhs, const int* active, cudaStream_t s, int seg) {
  typedef typename vec2<T>::type T2;
  if (sizeof(T) == 4 && fine.order == 2 && seg >= 0 && aligned16(f) && aligned16(out) && (!v || aligned16(v))) {
    const Op<float>& op = reinterpret_cast<const Op<float>&>(fine);
    const int nstrips = (fine.nx + kStripW - 1) / kStripW;
    const int ty = march_seg(seg, nstrips, fine.ny, nrhs);
    with_kind(2, fine.bc, [&](auto kd) {
      constexpr int BCk = decltype(kd)::BC;
      with_seg(ty, [&](auto tv) {
        constexpr int TY = decltype(tv)::value;
        const dim3 grid((nstrips + kStripWarps - 1) / kStripWarps, (fine.ny + TY - 1) / TY, nrhs);
        if (v)
          k_prolong_jacobi_m<BCk, TY, true><<<grid, 32 * kStripWarps, 0, s>>>(
              op, (float)w, (const float2*)f, (const float2*)v, 0, (const float2*)ec, nxc, nyc, (float2*)out,
              active, nstrips);
        else
          k_prolong_jacobi_m<BCk, TY, false><<<grid, 32 * kStripWarps, 0, s>>>(
              op, (float)w, (const float2*)f, nullptr, implicit_v ? 1 : 0, (const float2*)ec, nxc, nyc,
              (float2*)out, active, nstrips);
      });
    });
    return;
  }
  constexpr int RPT = fused_rpt<T>();
  with_kind(fine.order, fine.bc, [&](auto kd) {
    const dim3 grid((fine.nx + BX - 1) / BX, (fine.ny + BY * RPT - 1) / (BY * RPT), nrhs);
    k_prolong_jacobi<T, decltype(kd)::ORD, decltype(kd)::BC, RPT><<<grid, dim3(BX, BY), 0, s>>>(
        fine, w, (const T2*)f, (const T2*)v, implicit_v ? 1 : 0, (const T2*)ec, nxc, nyc, (T2*)out, active);
  });
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
                                         cudaStream_t, int);                                                  \
  template void launch_prolong_jacobi<T>(const Op<T>&, T, const void*, const void*, bool, const void*, int,   \
                                         int, void*, int, const int*, cudaStream_t, int);
INST(float)
INST(double)
#undef INST

}  // namespace helm
