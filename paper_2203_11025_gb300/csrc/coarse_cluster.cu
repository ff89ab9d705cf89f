// Coarsest-grid GMRES(m) of the SL V-cycle on a thread-block cluster per
// right-hand side (Sec. 2.4 and 4: diagonal-Jacobi right preconditioning,
// x0 = 0, m steps).
//
// The grid's rows are split over the C CTAs of a cluster (C <= 16); every CTA
// keeps its rows of the whole Krylov basis in shared memory, so the cluster's
// distributed shared memory holds the basis and no basis vector touches L2.
// Stencil halos (one row above and below) and inner-product partials are read
// from neighbouring CTAs through DSMEM after a hardware cluster barrier.
//
// Orthogonalisation is classical Gram-Schmidt applied twice (CGS2): per
// Arnoldi step one batched reduction for <v_i, w> (i <= j), the update, a
// second batched reduction for the re-orthogonalisation coefficients together
// with ||w||^2, and ||w - V h2||^2 = ||w||^2 - ||h2||^2 (V orthonormal).  In
// exact arithmetic this is the same Arnoldi process as modified Gram-Schmidt;
// CGS2 needs 2 reductions per step instead of j + 2.
//
// The matrix-vector product uses u = D^-1 v_j:  (M D^-1 v)(p) = v(p) - (1/h^2)
// * sum of u over the neighbours of p.  All arithmetic, reductions, the
// Hessenberg matrix and the Givens least-squares solve included, is in the
// Krylov type T (FP64 is a small fraction of FP32 throughput on this GPU);
// reductions run per thread, per warp, across warps and across CTAs in a
// fixed order, so every CTA of a cluster computes the identical Hessenberg
// matrix and solves the small least-squares problem redundantly.  Only
// barriers (block and cluster) are used; no CTA spins on memory written by
// another.
#include <cooperative_groups.h>

#include "devonce.cuh"
#include "helm_internal.cuh"

namespace cg = cooperative_groups;

namespace helm {

namespace {

constexpr int KT = 256;        // threads per CTA
constexpr int KMAX = 32;       // largest restart length

template <typename T>
__device__ __forceinline__ typename vec2<T>::type zz(T x, T y) {
  typename vec2<T>::type r;
  r.x = x; r.y = y;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 zmul2(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
__device__ __forceinline__ float hyp(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double hyp(double a, double b) { return hypot(a, b); }

template <typename T, int NT>
struct ClusterRed {
  typedef typename vec2<T>::type T2;
  T2 wsum[NT / 32][KMAX + 2];   // per-warp partials
  T2 csum[2][KMAX + 2];         // this CTA's totals, double-buffered across reductions
};

// Sum K complex values over the cluster: `vals(k, x, y)` gives this thread's partial
// of value k (already summed over its points).  Result, identical in every CTA, in out[k].
// Values are reduced two at a time so that the two shuffle chains overlap.
template <typename T, int MK, int NT, typename F>
__device__ __forceinline__ void cluster_reduce(cg::cluster_group& cl, ClusterRed<T, NT>& R, int buf, int K, F vals,
                                               typename vec2<T>::type* out) {
  typedef typename vec2<T>::type T2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = 0; k < K; k += 2) {
    T x0, y0, x1 = 0, y1 = 0;
    vals(k, x0, y0);
    if (k + 1 < K) vals(k + 1, x1, y1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x0 += __shfl_xor_sync(0xffffffffu, x0, o);
      y0 += __shfl_xor_sync(0xffffffffu, y0, o);
      x1 += __shfl_xor_sync(0xffffffffu, x1, o);
      y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    }
    if (lane == 0) {
      R.wsum[warp][k] = zz<T>(x0, y0);
      if (k + 1 < K) R.wsum[warp][k + 1] = zz<T>(x1, y1);
    }
  }
  __syncthreads();
  if (threadIdx.x < K) {
    T2 t = zz<T>(0, 0);
    for (int w = 0; w < NT / 32; ++w) { t.x += R.wsum[w][threadIdx.x].x; t.y += R.wsum[w][threadIdx.x].y; }
    R.csum[buf][threadIdx.x] = t;
  }
  cl.sync();
  if (threadIdx.x < K) {
    T2 t = zz<T>(0, 0);
    const int C = (int)cl.num_blocks();
    for (int r = 0; r < C; ++r) {
      const ClusterRed<T, NT>* rem = cl.map_shared_rank(&R, r);
      const T2 v = rem->csum[buf][threadIdx.x];
      t.x += v.x; t.y += v.y;
    }
    out[threadIdx.x] = t;
  }
  __syncthreads();
}

// NT threads per CTA; GB: the Krylov basis lives in global memory (gV, vectors vstride
// apart, [vector][rhs][point]), for grids whose basis does not fit in the cluster's
// shared memory; the halo vector u and D^-1 stay in shared memory.
template <typename T, int PPT, int MK, int NT, bool GB>
__global__ void __launch_bounds__(NT) k_coarse_cluster(Op<T> op, const typename vec2<T>::type* __restrict__ f,
                                                       typename vec2<T>::type* __restrict__ out, int m, int rows,
                                                       const int* gate, typename vec2<T>::type* gV, size_t vstride,
                                                       int di_smem) {
  typedef typename vec2<T>::type T2;
  constexpr int KT = NT;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int rhs = blockIdx.y;
  select_medium(op, rhs);
  if (gate && !gate[rhs]) return;                      // uniform over the cluster
  const int nx = op.nx, ny = op.ny, N = nx * ny;
  const int NP = rows * nx;                            // points of this CTA
  const int p0 = rank * NP;                            // first global point
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* Vs = reinterpret_cast<T2*>(smem_raw);            // [(m+1)][NP] (shared-memory basis)
  T2* U = GB ? Vs : Vs + (size_t)(m + 1) * NP;         // u = D^-1 v_j, [NP]
  T2* DI = U + NP;                                     // D^-1, [NP] (both layouts)
  // basis vector i of this CTA's points
  auto Vp = [&](int i) -> T2* {
    return GB ? gV + (size_t)i * vstride + (size_t)rhs * N + p0 : Vs + (size_t)i * NP;
  };
  // this thread's points: column and CTA-local row, computed once (kept in registers up to
  // 8 points per thread; beyond that they would spill, and are recomputed instead)
  constexpr bool kKeep = PPT <= 8;
  int qxs[kKeep ? PPT : 1], qys[kKeep ? PPT : 1];
#pragma unroll
  for (int q = 0; q < (kKeep ? PPT : 0); ++q) {
    const int lp = threadIdx.x + q * NT;
    qys[q] = lp / nx;
    qxs[q] = lp - qys[q] * nx;
  }
  auto qy = [&](int q) { return kKeep ? qys[q] : (int)(threadIdx.x + q * NT) / nx; };
  auto qx = [&](int q) { return kKeep ? qxs[q] : (int)(threadIdx.x + q * NT) - qy(q) * nx; };
  // D^-1: kept in shared memory when it fits (di_smem), else formed again when needed
  auto dinv = [&](int q, int lp) -> T2 {
    return di_smem ? DI[lp] : crecip(diag_at(op, qx(q), rank * rows + qy(q)));
  };
  __shared__ ClusterRed<T, NT> R;
  __shared__ T2 H[(KMAX + 1) * KMAX];
  __shared__ T2 hv[KMAX + 2];
  __shared__ T2 ys[KMAX];
  __shared__ T2 gg[KMAX + 1];
  __shared__ T2 snn[KMAX];
  __shared__ T css[KMAX];
  __shared__ int s_k;
  const int tid = threadIdx.x;
  const T2* fr = f + (size_t)rhs * N + p0;
  int buf = 0;

  T2 w[PPT];
  // D^-1 for own points; beta = ||f||
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int lp = tid + q * KT;
    if (lp < NP) {
      if (di_smem) DI[lp] = crecip(diag_at(op, qx(q), rank * rows + qy(q)));
      w[q] = fr[lp];
    } else {
      w[q] = czero<T2>();
    }
  }
  cluster_reduce<T, MK, NT>(cl, R, buf, 1, [&](int, T& a, T& b) {
    a = 0; b = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) a += w[q].x * w[q].x + w[q].y * w[q].y;
  }, hv);
  buf ^= 1;
  const T beta = sqrt(hv[0].x);
  T2* outr = out + (size_t)rhs * N + p0;
  if (!(beta > (T)0)) {
    T2 zv = czero<T2>();
    if (beta != beta) { zv.x = beta; zv.y = beta; }
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int lp = tid + q * KT;
      if (lp < NP) outr[lp] = zv;
    }
    cl.sync();   // no CTA leaves while others may still read its shared memory
    return;
  }
  {
    const T inv = (T)1 / beta;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int lp = tid + q * KT;
      if (lp < NP) Vp(0)[lp] = cscale(w[q], inv);
    }
  }
  const T ih2 = op.inv_h2;
  int k = 0;
  for (int j = 0; j < m; ++j) {
    const T2* vj = Vp(j);
    // u = D^-1 v_j, then halo exchange
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int lp = tid + q * KT;
      if (lp < NP) U[lp] = cmul(vj[lp], dinv(q, lp));
    }
    cl.sync();
    const T2* Uup = rank > 0 ? cl.map_shared_rank(U, rank - 1) : nullptr;       // row above: its last row
    const T2* Udn = rank < C - 1 ? cl.map_shared_rank(U, rank + 1) : nullptr;   // row below: its first row
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int lp = tid + q * KT;
      if (lp >= NP) continue;
      const int ly = qy(q), x = qx(q);
      // rows beyond this CTA's come from the neighbours' shared memory; stencil_sum asks for
      // them only inside the grid, where those neighbours exist
      const T2 s = stencil_sum<2>(op, x, rank * rows + ly, [&](int dx, int dy) -> T2 {
        const int yy = ly + dy, xx = x + dx;
        if (yy < 0) return Uup[(rows - 1) * nx + xx];
        if (yy >= rows) return Udn[xx];
        return U[yy * nx + xx];
      });
      T2 r = vj[lp];
      r.x -= s.x * ih2;
      r.y -= s.y * ih2;
      w[q] = r;
    }
    // CGS pass 1: h1_i = <v_i, w>
    cluster_reduce<T, MK, NT>(cl, R, buf, j + 1, [&](int i, T& a, T& b) {
      a = 0; b = 0;
      const T2* vi = Vp(i);
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int lp = tid + q * KT;
        if (lp < NP) { T2 v = vi[lp]; a += v.x * w[q].x + v.y * w[q].y; b += v.x * w[q].y - v.y * w[q].x; }
      }
    }, hv);
    buf ^= 1;
    if (tid <= j) H[tid * m + j] = hv[tid];
    for (int i = 0; i <= j; ++i) {
      const T hx = hv[i].x, hy = hv[i].y;
      const T2* vi = Vp(i);
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int lp = tid + q * KT;
        if (lp < NP) { T2 v = vi[lp]; w[q].x -= hx * v.x - hy * v.y; w[q].y -= hx * v.y + hy * v.x; }
      }
    }
    __syncthreads();   // hv is rewritten by the next reduction
    // CGS pass 2: h2_i = <v_i, w> and ||w||^2 in one reduction (value j+1)
    cluster_reduce<T, MK, NT>(cl, R, buf, j + 2, [&](int i, T& a, T& b) {
      a = 0; b = 0;
      if (i <= j) {
        const T2* vi = Vp(i);
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          const int lp = tid + q * KT;
          if (lp < NP) { T2 v = vi[lp]; a += v.x * w[q].x + v.y * w[q].y; b += v.x * w[q].y - v.y * w[q].x; }
        }
      } else {
#pragma unroll
        for (int q = 0; q < PPT; ++q) a += w[q].x * w[q].x + w[q].y * w[q].y;
      }
    }, hv);
    buf ^= 1;
    T nn = hv[j + 1].x;
    for (int i = 0; i <= j; ++i) nn -= hv[i].x * hv[i].x + hv[i].y * hv[i].y;
    const T nrm = sqrt(nn > (T)0 ? nn : (T)0);
    if (tid <= j) { T2 a = H[tid * m + j]; H[tid * m + j] = zz<T>(a.x + hv[tid].x, a.y + hv[tid].y); }
    if (tid == 0) H[(j + 1) * m + j] = zz<T>(nrm, 0);
    for (int i = 0; i <= j; ++i) {
      const T hx = hv[i].x, hy = hv[i].y;
      const T2* vi = Vp(i);
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int lp = tid + q * KT;
        if (lp < NP) { T2 v = vi[lp]; w[q].x -= hx * v.x - hy * v.y; w[q].y -= hx * v.y + hy * v.x; }
      }
    }
    k = j + 1;
    if (nrm == (T)0) break;                            // happy breakdown (identical in every CTA)
    if (j + 1 < m) {
      const T inv = (T)1 / nrm;
      T2* vn = Vp(j + 1);
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int lp = tid + q * KT;
        if (lp < NP) vn[lp] = cscale(w[q], inv);
      }
    }
    __syncthreads();
  }
  // least squares by Givens rotations (thread 0 of every CTA, identical inputs)
  if (tid == 0) {
    gg[0] = zz<T>(beta, 0);
    for (int j = 0; j < k; ++j) {
      for (int i = 0; i < j; ++i) {
        const T2 a = H[i * m + j], b = H[(i + 1) * m + j];
        const T2 t = zz<T>(css[i] * a.x + (snn[i].x * b.x - snn[i].y * b.y),
                           css[i] * a.y + (snn[i].x * b.y + snn[i].y * b.x));
        const T2 cj = zmul2(zz<T>(snn[i].x, -snn[i].y), a);
        H[(i + 1) * m + j] = zz<T>(-cj.x + css[i] * b.x, -cj.y + css[i] * b.y);
        H[i * m + j] = t;
      }
      const T2 a = H[j * m + j], b = H[(j + 1) * m + j];
      const T aa = hyp(a.x, a.y), bb = hyp(b.x, b.y);
      T c;
      T2 sv, r;
      if (bb == (T)0) { c = 1; sv = zz<T>(0, 0); r = a; }
      else if (aa == (T)0) { c = 0; sv = zz<T>(1, 0); r = b; }
      else {
        const T t = hyp(aa, bb);
        c = aa / t;
        const T2 ph = zz<T>(a.x / aa, a.y / aa);
        sv = zmul2(ph, zz<T>(b.x / t, -b.y / t));
        r = zz<T>(ph.x * t, ph.y * t);
      }
      css[j] = c; snn[j] = sv;
      H[j * m + j] = r;
      H[(j + 1) * m + j] = zz<T>(0, 0);
      const T2 gj = gg[j], sg = zmul2(zz<T>(sv.x, -sv.y), gj);
      gg[j + 1] = zz<T>(-sg.x, -sg.y);
      gg[j] = zz<T>(c * gj.x, c * gj.y);
    }
    for (int i = k - 1; i >= 0; --i) {
      T2 a = gg[i];
      for (int l = i + 1; l < k; ++l) { const T2 t = zmul2(H[i * m + l], ys[l]); a.x -= t.x; a.y -= t.y; }
      const T2 d = H[i * m + i];
      const T dd = d.x * d.x + d.y * d.y;
      ys[i] = zz<T>((a.x * d.x + a.y * d.y) / dd, (a.y * d.x - a.x * d.y) / dd);
    }
    s_k = k;
  }
  __syncthreads();
  const int kk = s_k;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int lp = tid + q * KT;
    if (lp >= NP) continue;
    T2 a = czero<T2>();
    for (int i = 0; i < kk; ++i) a = cadd(a, cmul(ys[i], Vp(i)[lp]));
    outr[lp] = cmul(a, dinv(q, lp));
  }
  cl.sync();   // keep shared memory alive until every CTA is done with remote reads
}

template <typename T, int PPT, int MK, int NT, bool GB>
bool launch_cluster(const Op<T>& op, const void* f, void* out, int nrhs, int m, const int* gate, int C, int rows,
                    size_t smem, void* gV, size_t vstride, cudaStream_t s, int di_smem = 1) {
  typedef typename vec2<T>::type T2;
  auto kern = k_coarse_cluster<T, PPT, MK, NT, GB>;
  // kernel attributes hold per device: set once on each device
  static DeviceOnce once;
  const bool ok = device_once(once, [&]() -> long long {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return 1;
  }, 0) == 1;
  if (!ok) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, nrhs, 1);
  cfg.blockDim = dim3(NT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, op, (const T2*)f, (T2*)out, m, rows, gate, (T2*)gV, vstride, di_smem) ==
         cudaSuccess;
}

}  // namespace

// Cluster geometry.  Shared-memory basis: rows per CTA so that each CTA holds <= 1024
// points (256 threads), C <= 16, and the CTA's basis fits in shared memory.  Otherwise,
// with a global basis gV (vectors vstride apart, [vector][rhs][point]): 1024 threads per
// CTA, C chosen so that the clusters of all right-hand sides fit in one wave, and only
// u (one vector) in shared memory.  Returns false if the grid fits neither.
template <typename T>
bool launch_coarse_gmres_cluster(const Op<T>& op, const void* f, void* out, int nrhs, int m, const int* gate,
                                 void* gV, size_t vstride, cudaStream_t s) {
  typedef typename vec2<T>::type T2;
  const int nx = op.nx, ny = op.ny;
  // 5-point stencil only: the compact scheme's coarsest solve takes the one-CTA or the
  // multi-kernel path
  if (op.order != 2 || m > KMAX || nx > 1024 || m + 2 > 34) return false;
  int C = 0, rows = 0;
  for (int target : {2 * KT, 4 * KT}) {       // prefer <= 2 points per thread (more SMs per solve)
    for (int c = 1; c <= 16 && !C; c *= 2) {
      if (ny % c) break;
      if ((long long)(ny / c) * nx <= target) { C = c; rows = ny / c; }
    }
    if (C) break;
  }
  if (C) {
    const int NP = rows * nx;
    const size_t smem = ((size_t)(m + 1) + 2) * NP * sizeof(T2);
    if (smem <= 180 * 1024) {
      const int ppt = (NP + KT - 1) / KT;
      if (m + 2 <= 12) {
        if (ppt <= 1) return launch_cluster<T, 1, 12, KT, false>(op, f, out, nrhs, m, gate, C, rows, smem, nullptr, 0, s);
        if (ppt <= 2) return launch_cluster<T, 2, 12, KT, false>(op, f, out, nrhs, m, gate, C, rows, smem, nullptr, 0, s);
        return launch_cluster<T, 4, 12, KT, false>(op, f, out, nrhs, m, gate, C, rows, smem, nullptr, 0, s);
      }
      if (ppt <= 1) return launch_cluster<T, 1, 34, KT, false>(op, f, out, nrhs, m, gate, C, rows, smem, nullptr, 0, s);
      if (ppt <= 2) return launch_cluster<T, 2, 34, KT, false>(op, f, out, nrhs, m, gate, C, rows, smem, nullptr, 0, s);
      return launch_cluster<T, 4, 34, KT, false>(op, f, out, nrhs, m, gate, C, rows, smem, nullptr, 0, s);
    }
  }
  // global basis: clusters of C CTAs x 1024 threads, C * nrhs <= 152 where possible
  if (!gV || m + 2 > 12) return false;
  constexpr int NTG = 1024;
  C = 16;
  while (C > 2 && (C * nrhs > 152 || ny % C)) C /= 2;
  if (ny % C) return false;
  rows = ny / C;
  const int NP = rows * nx;
  // u in shared memory, and D^-1 beside it when both fit
  const int di = (size_t)2 * NP * sizeof(T2) <= 180 * 1024 ? 1 : 0;
  const size_t smem = (size_t)(1 + di) * NP * sizeof(T2);
  if (smem > 180 * 1024) return false;
  const int ppt = (NP + NTG - 1) / NTG;
  if (ppt <= 4) return launch_cluster<T, 4, 12, NTG, true>(op, f, out, nrhs, m, gate, C, rows, smem, gV, vstride, s, di);
  if (ppt <= 8) return launch_cluster<T, 8, 12, NTG, true>(op, f, out, nrhs, m, gate, C, rows, smem, gV, vstride, s, di);
  if (ppt <= 16)
    return launch_cluster<T, 16, 12, NTG, true>(op, f, out, nrhs, m, gate, C, rows, smem, gV, vstride, s, di);
  return false;
}

template bool launch_coarse_gmres_cluster<float>(const Op<float>&, const void*, void*, int, int, const int*, void*,
                                                 size_t, cudaStream_t);
template bool launch_coarse_gmres_cluster<double>(const Op<double>&, const void*, void*, int, int, const int*, void*,
                                                  size_t, cudaStream_t);

}  // namespace helm
