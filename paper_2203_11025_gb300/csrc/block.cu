// Block kernels of block flexible GMRES (the CPU solver of Sec. 4, one Krylov space for
// all right-hand sides): the Gram matrix U^H W of two sets of complex vectors, and the
// combination Out (+)= In C with a small dense coefficient matrix C.  Vectors are
// [vector][point] complex, `stride` elements apart.
//
// Gram: every CTA walks a contiguous range of points in tiles of kTile points staged in
// shared memory; thread t owns pair t mod (q p) (and more pairs when q p > 256) and, when
// q p < 256, one of 256 / (q p) interleaved slices of each tile; it sums conj(u_i) w_k over
// its part of a tile in FP32 and adds that into FP64 accumulators (FP64 is a small
// fraction of the FP32 rate on this GPU).  The slices of a pair are added in shared memory
// in a fixed order, and the per-CTA partials by a second kernel, one warp per pair.  Combine: one thread per point holds the p outputs in registers and streams the
// q inputs of that point, so in-place use (Out == In, q == p) is safe.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "helm_internal.cuh"

namespace helm {

namespace {

constexpr int kTile = 32;      // points per shared-memory tile
constexpr int kGramThreads = 256;
constexpr int kMaxPairs = 18;  // (i, k) pairs per thread at most: q p <= 18 * 256 (m = p = 16: 4352)
constexpr int kRow = kTile + 1; // padded tile row (spreads the k-strided reads over the banks)
constexpr int kMaxP = 16;      // block size at most

template <typename T2> struct Real;
template <> struct Real<float2> { typedef float type; };
template <> struct Real<double2> { typedef double type; };

template <typename T2>
__global__ void __launch_bounds__(kGramThreads) k_bgram_partial(const T2* __restrict__ U, size_t ustride, int q,
                                                                const T2* __restrict__ W, size_t wstride, int p,
                                                                size_t N, double2* __restrict__ part) {
  typedef typename Real<T2>::type R;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T2* su = reinterpret_cast<T2*>(sm_raw);          // [q][kRow]
  T2* sw = su + (size_t)q * kRow;                   // [p][kRow]
  const int npair = q * p;
  const int nsl = npair >= kGramThreads ? 1 : kGramThreads / npair;   // tile slices per pair
  const int sl = npair >= kGramThreads ? 0 : (int)threadIdx.x / npair;
  const int tpr = npair >= kGramThreads ? (int)threadIdx.x : (int)threadIdx.x - sl * npair;
  const size_t per = (N + gridDim.x - 1) / gridDim.x;
  const size_t n0 = (size_t)blockIdx.x * per, n1 = n0 + per < N ? n0 + per : N;
  double ax[kMaxPairs], ay[kMaxPairs];
#pragma unroll
  for (int t = 0; t < kMaxPairs; ++t) { ax[t] = 0.0; ay[t] = 0.0; }
  for (size_t t0 = n0; t0 < n1; t0 += kTile) {
    const int len = (int)(n1 - t0 < (size_t)kTile ? n1 - t0 : (size_t)kTile);
    __syncthreads();
    for (int e = threadIdx.x; e < q * kTile; e += blockDim.x) {
      const int i = e / kTile, j = e - i * kTile;
      su[i * kRow + j] = j < len ? U[(size_t)i * ustride + t0 + j] : T2{0, 0};
    }
    for (int e = threadIdx.x; e < p * kTile; e += blockDim.x) {
      const int k = e / kTile, j = e - k * kTile;
      sw[k * kRow + j] = j < len ? W[(size_t)k * wstride + t0 + j] : T2{0, 0};
    }
    __syncthreads();
    if (sl < nsl) {
#pragma unroll
      for (int t = 0; t < kMaxPairs; ++t) {
        const int pr = tpr + t * kGramThreads;
        if (pr >= npair) break;
        const int i = pr / p, k = pr - i * p;
        const T2* a = su + (size_t)i * kRow;
        const T2* b = sw + (size_t)k * kRow;
        R sx = 0, sy = 0;
        for (int j = sl; j < kTile; j += nsl) {   // conj(a) * b
          sx += a[j].x * b[j].x + a[j].y * b[j].y;
          sy += a[j].x * b[j].y - a[j].y * b[j].x;
        }
        ax[t] += (double)sx;
        ay[t] += (double)sy;
      }
    }
  }
  if (nsl == 1) {
#pragma unroll
    for (int t = 0; t < kMaxPairs; ++t) {
      const int pr = tpr + t * kGramThreads;
      if (pr >= npair) break;
      part[(size_t)blockIdx.x * npair + pr] = make_double2(ax[t], ay[t]);
    }
    return;
  }
  // slices of one pair (npair < 256): add them in slice order through shared memory
  __syncthreads();
  double2* red = reinterpret_cast<double2*>(sm_raw);   // [nsl][npair], reuses the tiles
  if (sl < nsl) red[sl * npair + tpr] = make_double2(ax[0], ay[0]);
  __syncthreads();
  if ((int)threadIdx.x < npair) {
    double x = 0.0, y = 0.0;
    for (int q2 = 0; q2 < nsl; ++q2) {
      x += red[q2 * npair + threadIdx.x].x;
      y += red[q2 * npair + threadIdx.x].y;
    }
    part[(size_t)blockIdx.x * npair + threadIdx.x] = make_double2(x, y);
  }
}

// One warp per pair: lanes take every 32nd partial, then a fixed shuffle tree.
__global__ void k_bgram_reduce(const double2* __restrict__ part, int nparts, int npair, double2* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int pr = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; pr < npair; pr += (gridDim.x * blockDim.x) >> 5) {
    double x = 0.0, y = 0.0;
    for (int b = lane; b < nparts; b += 32) {
      const double2 v = part[(size_t)b * npair + pr];
      x += v.x;
      y += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) out[pr] = make_double2(x, y);
  }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(256) k_bcombine(const TI* in, size_t istride, int q,   // may alias out
                                                  const double2* __restrict__ C, TO* out, size_t ostride, int p,
                                                  size_t N, int accumulate) {
  typedef typename Real<TO>::type R;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  TO* sc = reinterpret_cast<TO*>(sm_raw);   // [q][p], in the output precision
  for (int e = threadIdx.x; e < q * p; e += blockDim.x) {
    sc[e].x = (R)C[e].x;
    sc[e].y = (R)C[e].y;
  }
  __syncthreads();
  for (size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    R ox[kMaxP], oy[kMaxP];
#pragma unroll
    for (int k = 0; k < kMaxP; ++k) { ox[k] = 0; oy[k] = 0; }
    for (int i = 0; i < q; ++i) {
      const TI v = in[(size_t)i * istride + n];
      const R vx = (R)v.x, vy = (R)v.y;
#pragma unroll
      for (int k = 0; k < kMaxP; ++k) {
        if (k >= p) break;
        const TO c = sc[i * p + k];
        ox[k] += vx * c.x - vy * c.y;
        oy[k] += vx * c.y + vy * c.x;
      }
    }
#pragma unroll
    for (int k = 0; k < kMaxP; ++k) {
      if (k >= p) break;
      TO o = accumulate ? out[(size_t)k * ostride + n] : TO{0, 0};
      o.x += ox[k];
      o.y += oy[k];
      out[(size_t)k * ostride + n] = o;
    }
  }
}

}  // namespace

int block_gram_parts(int nsm) { return 2 * nsm; }

template <typename T2>
int block_gram(const T2* U, size_t ustride, int q, const T2* W, size_t wstride, int p, size_t N, double2* part,
               double2* out, int nsm, cudaStream_t s) {
  if (q < 1 || p < 1 || p > kMaxP || q * p > kMaxPairs * kGramThreads) return -1;
  const int nparts = block_gram_parts(nsm);
  // the tiles, and the slice sums of the pairs (<= 256 double2) that reuse them
  const size_t smem = std::max((size_t)(q + p) * kRow * sizeof(T2), (size_t)kGramThreads * sizeof(double2));
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_bgram_partial<T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  k_bgram_partial<T2><<<nparts, kGramThreads, smem, s>>>(U, ustride, q, W, wstride, p, N, part);
  k_bgram_reduce<<<(q * p + 7) / 8, 256, 0, s>>>(part, nparts, q * p, out);
  return 0;
}
template int block_gram<float2>(const float2*, size_t, int, const float2*, size_t, int, size_t, double2*, double2*, int,
                                cudaStream_t);
template int block_gram<double2>(const double2*, size_t, int, const double2*, size_t, int, size_t, double2*, double2*,
                                 int, cudaStream_t);

template <typename TI, typename TO>
int block_combine(const TI* in, size_t istride, int q, const double2* C, TO* out, size_t ostride, int p, size_t N,
                  bool accumulate, int nsm, cudaStream_t s) {
  if (q < 1 || p < 1 || p > kMaxP) return -1;
  const size_t smem = (size_t)q * p * sizeof(double2);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_bcombine<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  const unsigned grid = (unsigned)std::min<size_t>((N + 255) / 256, (size_t)nsm * 8);
  k_bcombine<TI, TO><<<grid, 256, smem, s>>>(in, istride, q, C, out, ostride, p, N, accumulate ? 1 : 0);
  return 0;
}
template int block_combine<float2, float2>(const float2*, size_t, int, const double2*, float2*, size_t, int, size_t,
                                           bool, int, cudaStream_t);
template int block_combine<double2, double2>(const double2*, size_t, int, const double2*, double2*, size_t, int,
                                             size_t, bool, int, cudaStream_t);
template int block_combine<float2, double2>(const float2*, size_t, int, const double2*, double2*, size_t, int, size_t,
                                            bool, int, cudaStream_t);
template int block_combine<double2, float2>(const double2*, size_t, int, const double2*, float2*, size_t, int, size_t,
                                            bool, int, cudaStream_t);

}  // namespace helm
