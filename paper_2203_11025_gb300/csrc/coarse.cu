// Coarsest-grid solve of the SL V-cycle in ONE launch: m steps of GMRES with
// diagonal (Jacobi) right preconditioning from x = 0 on M of the coarsest
// level (Sec. 2.4 and 4; the "solve directly" line of Alg. 1 is replaced by
// GMRES(10) as the paper's experiments do).
//
// One 1024-thread CTA per right-hand side.  Each thread owns a fixed set of
// grid points (p = tid + 1024 q), keeps its part of the Arnoldi vector w in
// shared memory, and reads the basis vectors (stored in global memory, L2
// resident at these sizes) for the stencil neighbours and the Gram-Schmidt
// passes.  Modified Gram-Schmidt and the Givens least-squares solve follow the
// multi-kernel path exactly; inner products are accumulated per thread in T
// and across the block in FP64, in a fixed order (deterministic).  Only block
// barriers are used: no inter-CTA waiting.
#include <mutex>
#include <string>

#include "../../include/helm.h"
#include "devonce.cuh"
#include "helm_internal.cuh"

namespace helm {

void set_error(const std::string& s);

namespace {

constexpr int CT = 1024;
constexpr int CMAX = 32;

__device__ __forceinline__ double2 z2(double x, double y) { double2 r; r.x = x; r.y = y; return r; }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return z2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// Sum over the block, returned to every thread (fixed summation order).  The
// per-thread and per-warp sums stay in T (FP64 throughput is scarce on this
// part); the 32 warp totals are added in FP64 by one warp and broadcast.
template <typename T>
__device__ __forceinline__ double2 block_allsum(T ax, T ay, double2* red, double2* bcast) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, o);
    ay += __shfl_xor_sync(0xffffffffu, ay, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = z2((double)ax, (double)ay);
  __syncthreads();
  if (warp == 0) {
    double2 v = red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    if (lane == 0) *bcast = v;
  }
  __syncthreads();
  return *bcast;
}

template <typename T>
__device__ __forceinline__ typename vec2<T>::type scaled_by_dinv(const Op<T>& op, const typename vec2<T>::type* v,
                                                                 int x, int y) {
  return cmul(v[(size_t)y * op.nx + x], cinv(diag_at(op, x, y)));
}

template <typename T, int ORD>
__global__ void __launch_bounds__(CT) k_coarse_gmres(Op<T> op, const typename vec2<T>::type* __restrict__ f,
                                                     typename vec2<T>::type* __restrict__ out,
                                                     typename vec2<T>::type* __restrict__ Vg, size_t vstride, int m,
                                                     const int* gate) {
  typedef typename vec2<T>::type T2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* w = reinterpret_cast<T2*>(smem_raw);
  __shared__ double2 red[CT / 32];
  __shared__ double2 bcast;
  __shared__ double2 Hs[(CMAX + 1) * CMAX];
  __shared__ double2 ys[CMAX];
  __shared__ double2 g[CMAX + 1];
  __shared__ double2 sn[CMAX];
  __shared__ double cs[CMAX];
  __shared__ int s_k;
  const int rhs = blockIdx.x;
  select_medium(op, rhs);
  if (gate && !gate[rhs]) return;
  const int nx = op.nx, ny = op.ny, N = nx * ny, tid = threadIdx.x;
  const size_t off = (size_t)rhs * N;
  const T2* fr = f + off;
  T2* outr = out + off;

  // beta = ||f||, v_0 = f / beta
  T nb = 0;
  for (int p = tid; p < N; p += CT) { T2 v = fr[p]; nb += v.x * v.x + v.y * v.y; }
  const double beta = sqrt(block_allsum(nb, T(0), red, &bcast).x);
  if (!(beta > 0.0)) {                                 // zero (or non-finite) right-hand side
    T2 zv = czero<T2>();
    if (beta != beta) { zv.x = beta; zv.y = beta; }    // propagate NaN
    for (int p = tid; p < N; p += CT) outr[p] = zv;
    return;
  }
  {
    const T inv = (T)(1.0 / beta);
    T2* v0 = Vg + off;
    for (int p = tid; p < N; p += CT) v0[p] = cscale(fr[p], inv);
  }
  int k = 0;
  for (int j = 0; j < m; ++j) {
    __syncthreads();                                   // v_j complete
    const T2* vj = Vg + (size_t)j * vstride + off;
    // w = M D^-1 v_j
    for (int p = tid; p < N; p += CT) {
      const int y = p / nx, x = p - y * nx;
      T2 c = scaled_by_dinv(op, vj, x, y);
      const T2 s = stencil_sum<ORD>(op, x, y, [&](int dx, int dy) { return scaled_by_dinv(op, vj, x + dx, y + dy); });
      T2 r = cmul(diag_at(op, x, y), c);
      r.x -= s.x * op.inv_h2;
      r.y -= s.y * op.inv_h2;
      w[p] = r;
    }
    // modified Gram-Schmidt: each thread touches only its own points of w
    for (int i = 0; i <= j; ++i) {
      const T2* vi = Vg + (size_t)i * vstride + off;
      T ax = 0, ay = 0;
      for (int p = tid; p < N; p += CT) {
        T2 a = vi[p], b = w[p];
        ax += a.x * b.x + a.y * b.y;
        ay += a.x * b.y - a.y * b.x;
      }
      const double2 h = block_allsum(ax, ay, red, &bcast);
      if (tid == 0) Hs[i * m + j] = h;
      const T hx = (T)h.x, hy = (T)h.y;
      for (int p = tid; p < N; p += CT) {
        T2 a = vi[p], b = w[p];
        b.x -= hx * a.x - hy * a.y;
        b.y -= hx * a.y + hy * a.x;
        w[p] = b;
      }
    }
    T nn = 0;
    for (int p = tid; p < N; p += CT) { T2 b = w[p]; nn += b.x * b.x + b.y * b.y; }
    const double nrm = sqrt(block_allsum(nn, T(0), red, &bcast).x);
    if (tid == 0) Hs[(j + 1) * m + j] = z2(nrm, 0.0);
    k = j + 1;
    if (nrm == 0.0) break;                             // happy breakdown (uniform across the block)
    if (j + 1 < m) {
      const T inv = (T)(1.0 / nrm);
      T2* vn = Vg + (size_t)(j + 1) * vstride + off;
      for (int p = tid; p < N; p += CT) vn[p] = cscale(w[p], inv);
    }
  }
  __syncthreads();
  // least squares min ||beta e1 - H y|| by Givens rotations, in place in Hs (one thread)
  if (tid == 0) {
    g[0] = z2(beta, 0.0);
    for (int j = 0; j < k; ++j) {
      for (int i = 0; i < j; ++i) {
        double2 a = Hs[i * m + j], b = Hs[(i + 1) * m + j];
        double2 t = z2(cs[i] * a.x + (sn[i].x * b.x - sn[i].y * b.y), cs[i] * a.y + (sn[i].x * b.y + sn[i].y * b.x));
        double2 cj = zmul(z2(sn[i].x, -sn[i].y), a);
        Hs[(i + 1) * m + j] = z2(-cj.x + cs[i] * b.x, -cj.y + cs[i] * b.y);
        Hs[i * m + j] = t;
      }
      double2 a = Hs[j * m + j], b = Hs[(j + 1) * m + j];
      double aa = hypot(a.x, a.y), bb = hypot(b.x, b.y), c;
      double2 sv, r;
      if (bb == 0.0) { c = 1.0; sv = z2(0, 0); r = a; }
      else if (aa == 0.0) { c = 0.0; sv = z2(1, 0); r = b; }
      else {
        double t = hypot(aa, bb);
        c = aa / t;
        double2 ph = z2(a.x / aa, a.y / aa);
        sv = zmul(ph, z2(b.x / t, -b.y / t));
        r = z2(ph.x * t, ph.y * t);
      }
      cs[j] = c; sn[j] = sv;
      Hs[j * m + j] = r;
      Hs[(j + 1) * m + j] = z2(0, 0);
      double2 gj = g[j], sg = zmul(z2(sv.x, -sv.y), gj);
      g[j + 1] = z2(-sg.x, -sg.y);
      g[j] = z2(c * gj.x, c * gj.y);
    }
    for (int i = k - 1; i >= 0; --i) {
      double2 a = g[i];
      for (int l = i + 1; l < k; ++l) { double2 t = zmul(Hs[i * m + l], ys[l]); a.x -= t.x; a.y -= t.y; }
      double2 d = Hs[i * m + i];
      double dd = d.x * d.x + d.y * d.y;
      ys[i] = z2((a.x * d.x + a.y * d.y) / dd, (a.y * d.x - a.x * d.y) / dd);
    }
    s_k = k;
  }
  __syncthreads();
  // x = D^-1 sum_i y_i v_i
  const int kk = s_k;
  for (int p = tid; p < N; p += CT) {
    T2 a = czero<T2>();
    for (int i = 0; i < kk; ++i) {
      T2 yi;
      yi.x = (T)ys[i].x; yi.y = (T)ys[i].y;
      a = cadd(a, cmul(yi, Vg[(size_t)i * vstride + off + p]));
    }
    const int y = p / nx, x = p - y * nx;
    outr[p] = cmul(a, cinv(diag_at(op, x, y)));
  }
}

}  // namespace

template <typename T>
bool launch_coarse_gmres_fused(const Op<T>& op, const void* f, void* out, void* V, size_t vstride, int nrhs, int m,
                               const int* gate, cudaStream_t s, cudaError_t* launch_err) {
  typedef typename vec2<T>::type T2;
  if (launch_err) *launch_err = cudaSuccess;
  const size_t smem = (size_t)op.nx * op.ny * sizeof(T2);
  if (m > CMAX || smem > 160 * 1024) return false;
  // the shared-memory opt-in is a per-device attribute: raised once on each device
  static DeviceOnce once2, once4;
  auto k = op.order == 4 ? k_coarse_gmres<T, 4> : k_coarse_gmres<T, 2>;
  if (!set_dynamic_smem(op.order == 4 ? once4 : once2, k, 160 * 1024)) {
    if (launch_err) *launch_err = cudaErrorInvalidValue;
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nrhs, 1, 1);
  cfg.blockDim = dim3(CT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k, op, (const T2*)f, (T2*)out, (T2*)V, vstride, m, gate);
  if (launch_err) *launch_err = e;
  return true;
}

// ---------------------------------------------------------------------------
// Allocation-free entry point: the coarsest-grid GMRES solve with its Krylov
// basis in a file-scope device array instead of a handle's workspace.
// ---------------------------------------------------------------------------
namespace {

// 2^20 complex float = 8 MiB, held by every GPU that loads the library until exit.
constexpr size_t kStaticBasisElems = (size_t)1 << 20;
__device__ __align__(256) float2 g_static_basis[kStaticBasisElems];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

}  // namespace

template bool launch_coarse_gmres_fused<float>(const Op<float>&, const void*, void*, void*, size_t, int, int,
                                               const int*, cudaStream_t, cudaError_t*);
template bool launch_coarse_gmres_fused<double>(const Op<double>&, const void*, void*, void*, size_t, int, int,
                                                const int*, cudaStream_t, cudaError_t*);

}  // namespace helm

extern "C" int helm_coarse_solve_static(int nx, int ny, double h, double omega, double beta, int abc_width,
                                        double gamma_max, const float* kappa2, const void* f, void* x, int nrhs,
                                        int m, helm_stream_t stream) {
  if (nx <= 0 || ny <= 0 || nrhs < 1 || m < 1 || m > 32 || !(h > 0) || abc_width < 0 || !kappa2 || !f || !x) {
    helm::set_error("helm_coarse_solve_static: bad arguments");
    return HELM_EINVAL;
  }
  {
    // f is read by every block while others write x: the byte ranges must not meet
    const size_t bytes = (size_t)nrhs * (size_t)nx * (size_t)ny * sizeof(float2);
    const uintptr_t fa = (uintptr_t)f, xa = (uintptr_t)x;
    if (fa < xa + bytes && xa < fa + bytes) {
      helm::set_error("helm_coarse_solve_static: f and x overlap");
      return HELM_EINVAL;
    }
  }
  const size_t need = (size_t)(m + 1) * (size_t)nrhs * (size_t)nx * (size_t)ny;
  if (need > helm::kStaticBasisElems) {
    helm::set_error("helm_coarse_solve_static: (m+1)*nrhs*nx*ny = " + std::to_string(need) +
                    " complex values exceed the static scratch of " + std::to_string(helm::kStaticBasisElems));
    return HELM_EINVAL;
  }
  if ((size_t)nx * ny * sizeof(float2) > 160 * 1024) {
    helm::set_error("helm_coarse_solve_static: grid larger than the one-launch kernel's shared memory (160 KiB)");
    return HELM_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= helm::kMaxDevices) {
    helm::set_error("helm_coarse_solve_static: no usable current device");
    return HELM_ECUDA;
  }
  void* basis = nullptr;
  {
    std::lock_guard<std::mutex> lk(helm::g_static_mu);
    if (!helm::g_static_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, helm::g_static_basis);
      if (e != cudaSuccess) {
        helm::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return HELM_ECUDA;
      }
      helm::g_static_ptr[dev] = p;
    }
    basis = helm::g_static_ptr[dev];
  }
  helm::Op<float> op;
  op.nx = nx; op.ny = ny; op.abc_w = abc_width; op.bc = helm::kBcDirichlet; op.order = 2;
  op.inv_h2 = (float)(1.0 / (h * h));
  op.h2 = (float)(h * h);
  op.omega2 = (float)(omega * omega);
  op.gmax = (float)gamma_max;
  op.beta = (float)beta;
  op.inv_w = abc_width > 0 ? (float)(1.0 / abc_width) : 0.f;
  op.k2 = kappa2;
  op.rpp = 0;
  cudaError_t le = cudaSuccess;
  const bool launched = helm::launch_coarse_gmres_fused<float>(op, f, x, basis, (size_t)nrhs * nx * ny, nrhs, m,
                                                               nullptr, (cudaStream_t)stream, &le);
  if (!launched) {
    // the sizes were checked above, so only the shared-memory opt-in can have failed
    helm::set_error("helm_coarse_solve_static: raising the kernel's shared-memory limit failed on this device");
    return HELM_ECUDA;
  }
  if (le != cudaSuccess) {   // this launch's own result (an earlier, unrelated error is left pending)
    helm::set_error(std::string("helm_coarse_solve_static launch: ") + cudaGetErrorString(le));
    return HELM_ECUDA;
  }
  return HELM_OK;
}
