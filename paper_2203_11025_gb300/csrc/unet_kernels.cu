// Kernels of the U-Net preconditioner (Sec. 3.1-3.4): implicit-GEMM
// convolutions (5x5 stride-2, 3x3 stride-1, 5x5 stride-2 transposed) with their
// data and weight gradients, BatchNorm, eLU, the MSE loss and Adam.
//
// Layouts: activations NHWC (pixel-major, channels contiguous) in BF16, raw
// convolution outputs and all gradients in FP32; weights [tap][cin][cout]
// (tap = ky * k + kx) as FP32 masters with BF16 working copies.  Channel
// concatenations (skip connections, encoder context) are never materialised:
// a convolution reads up to two sources and writes into a channel slice.
#include <cuda_bf16.h>

#include <algorithm>

#include "devonce.cuh"
#include "unet_internal.cuh"

namespace helm {

namespace {

__device__ __forceinline__ float bf(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float elu_f(float x) { return x > 0.f ? x : expm1f(x); }
__device__ __forceinline__ float elu_grad(float x) { return x > 0.f ? 1.f : expf(x); }

// Input pixel feeding output pixel (oy, ox) through tap (ky, kx); false if padding.
__device__ __forceinline__ bool gather_pos(const ConvArgs& a, int oy, int ox, int ky, int kx, int& iy, int& ix) {
  if (!a.transposed) {
    iy = oy * a.stride + ky - a.pad;
    ix = ox * a.stride + kx - a.pad;
  } else {  // out[s*i + t - p] += W[t] in[i]  =>  i = (o + p - t) / s when divisible
    int ny = oy + a.pad - ky, nx = ox + a.pad - kx;
    if (ny < 0 || nx < 0 || ny % a.stride || nx % a.stride) return false;
    iy = ny / a.stride;
    ix = nx / a.stride;
  }
  return iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
}

__device__ __forceinline__ float load_src(const void* p, int f32, size_t idx) {
  return f32 ? ((const float*)p)[idx] : bf(((const __nv_bfloat16*)p)[idx]);
}

// Input element (pixel spix of image b, concatenated channel ci); the second source
// may be shared by every image of the batch (bcast1).
__device__ __forceinline__ float load_in(const ConvArgs& a, size_t spix, size_t plane, int ci) {
  float v = ci < a.c0 ? load_src(a.in0, a.in_f32, spix * a.ld0 + ci)
                      : load_src(a.in1, a.in_f32, (a.bcast1 ? spix % plane : spix) * a.ld1 + (ci - a.c0));
  return a.in_act ? elu_f(v) : v;
}

// out[m][co] = sum_{tap, ci} in(m, tap, ci) W[tap][ci][co] (+ bias, + residual);
// 64 pixels x 64 channels per block, K staged through shared memory in chunks of 16.
__global__ void __launch_bounds__(256) k_conv_simt(ConvArgs a) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int M = a.B * a.Ho * a.Wo;
  const int Cin = a.c0 + a.c1;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int tid = threadIdx.x, tm = tid & 15, tn = tid >> 4;
  const int lp = tid & 63, lk = (tid >> 6) * 4;
  const int pm = m0 + lp;
  const bool pvalid = pm < M;
  int pb = 0, poy = 0, pox = 0;
  if (pvalid) {
    pb = pm / (a.Ho * a.Wo);
    int r = pm - pb * a.Ho * a.Wo;
    poy = r / a.Wo;
    pox = r - poy * a.Wo;
  }
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int taps = a.k * a.k;
  for (int tap = 0; tap < taps; ++tap) {
    const int ky = tap / a.k, kx = tap - ky * a.k;
    int iy = 0, ix = 0;
    const bool v = pvalid && gather_pos(a, poy, pox, ky, kx, iy, ix);
    const size_t spix = ((size_t)pb * a.Hi + iy) * a.Wi + ix;
    for (int cb = 0; cb < Cin; cb += 16) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int ci = cb + lk + q;
        As[lk + q][lp] = (v && ci < Cin) ? load_in(a, spix, (size_t)a.Hi * a.Wi, ci) : 0.f;
        const int co = n0 + lp;
        Bs[lk + q][lp] = (ci < Cin && co < a.Cout) ? bf(a.W[tap * a.wst + ci * a.wsk + co * a.wsn]) : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        float av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { av[i] = As[kk][tm * 4 + i]; bv[i] = Bs[kk][tn * 4 + i]; }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tm * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int co = n0 + tn * 4 + j;
      if (co >= a.Cout) continue;
      float val = acc[i][j];
      if (a.bias) val += a.bias[co];
      if (a.res) val += bf(a.res[(size_t)m * a.ldr + co]);
      a.out[(size_t)m * a.ldo + co] = val;
    }
  }
}

// Thin convolution (few output channels, or few input channels): one thread per
// output pixel computes all Cout <= 32 outputs; the weights sit in shared memory
// as float; transposed stride-2 convolutions visit only the taps of the pixel's
// output phase.
template <int CO>
__global__ void __launch_bounds__(128) k_conv_thin(ConvArgs a) {
  extern __shared__ float wsm[];   // [taps][Cin][CO]
  const int Cin = a.c0 + a.c1;
  const int taps = a.k * a.k;
  for (int i = threadIdx.x; i < taps * Cin * CO; i += blockDim.x) {
    const int co = i % CO, r = i / CO;
    const int ci = r % Cin, tap = r / Cin;
    wsm[i] = co < a.Cout ? bf(a.W[tap * a.wst + ci * a.wsk + co * a.wsn]) : 0.f;
  }
  __syncthreads();
  const int M = a.B * a.Ho * a.Wo;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int b = m / (a.Ho * a.Wo);
  const int rr = m - b * a.Ho * a.Wo;
  const int oy = rr / a.Wo, ox = rr - oy * a.Wo;
  float acc[CO];
#pragma unroll
  for (int j = 0; j < CO; ++j) acc[j] = 0.f;
  const size_t plane = (size_t)a.Hi * a.Wi;
  int ky0 = 0, kx0 = 0, dk = 1;
  if (a.transposed) { ky0 = (oy + a.pad) % a.stride; kx0 = (ox + a.pad) % a.stride; dk = a.stride; }
  for (int ky = ky0; ky < a.k; ky += dk) {
    for (int kx = kx0; kx < a.k; kx += dk) {
      int iy, ix;
      if (!gather_pos(a, oy, ox, ky, kx, iy, ix)) continue;
      const size_t sp = ((size_t)b * a.Hi + iy) * a.Wi + ix;
      const float* wt = wsm + (size_t)(ky * a.k + kx) * Cin * CO;
      for (int ci = 0; ci < Cin; ++ci) {
        const float v = load_in(a, sp, plane, ci);
#pragma unroll
        for (int j = 0; j < CO; ++j) acc[j] = fmaf(v, wt[ci * CO + j], acc[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < CO; ++j) {
    if (j >= a.Cout) break;
    float val = acc[j];
    if (a.bias) val += a.bias[j];
    if (a.res) val += bf(a.res[(size_t)m * a.ldr + j]);
    a.out[(size_t)m * a.ldo + j] = val;
  }
}

// gW[tap][ci][co] += sum_m in(m, tap, ci) G[m][co] over a chunk of output pixels.
__global__ void __launch_bounds__(256) k_wgrad_simt(ConvArgs a, const float* __restrict__ G, int ldg,
                                                    float* __restrict__ gW, int chunk) {
  __shared__ float As[32][33];
  __shared__ float Gs[32][33];
  const int M = a.B * a.Ho * a.Wo;
  const int Cin = a.c0 + a.c1;
  const int nci = (Cin + 31) / 32, nco = (a.Cout + 31) / 32;
  int t = blockIdx.x;
  const int cot = t % nco; t /= nco;
  const int cit = t % nci; t /= nci;
  const int tap = t;
  const int ky = tap / a.k, kx = tap - ky * a.k;
  const int mbeg = blockIdx.y * chunk, mend = min(M, mbeg + chunk);
  const int tid = threadIdx.x;
  const int ti = tid & 15, tj = tid >> 4;    // 2x2 outputs each: ci = 2*ti.., co = 2*tj..
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int mb = mbeg; mb < mend; mb += 32) {
    for (int q = tid; q < 32 * 32; q += 256) {
      const int pr = q >> 5, c = q & 31;
      const int m = mb + pr;
      float av = 0.f, gv = 0.f;
      if (m < mend) {
        const int b = m / (a.Ho * a.Wo);
        const int r = m - b * a.Ho * a.Wo;
        const int oy = r / a.Wo, ox = r - (r / a.Wo) * a.Wo;
        int iy, ix;
        const int ci = cit * 32 + c;
        if (ci < Cin && gather_pos(a, oy, ox, ky, kx, iy, ix))
          av = load_in(a, ((size_t)b * a.Hi + iy) * a.Wi + ix, (size_t)a.Hi * a.Wi, ci);
        const int co = cot * 32 + c;
        if (co < a.Cout) gv = G[(size_t)m * ldg + co];
      }
      As[pr][c] = av;
      Gs[pr][c] = gv;
    }
    __syncthreads();
#pragma unroll 8
    for (int pr = 0; pr < 32; ++pr) {
      const float a0 = As[pr][2 * ti], a1 = As[pr][2 * ti + 1];
      const float g0 = Gs[pr][2 * tj], g1 = Gs[pr][2 * tj + 1];
      acc[0][0] = fmaf(a0, g0, acc[0][0]);
      acc[0][1] = fmaf(a0, g1, acc[0][1]);
      acc[1][0] = fmaf(a1, g0, acc[1][0]);
      acc[1][1] = fmaf(a1, g1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int ci = cit * 32 + 2 * ti + i, co = cot * 32 + 2 * tj + j;
      if (ci < Cin && co < a.Cout) atomicAdd(&gW[(size_t)tap * Cin * a.Cout + (size_t)ci * a.Cout + co], acc[i][j]);
    }
}

// Per-channel partial sums over a pixel range: mode 0 sum(z), mode 1 sum((z - mean)^2).
__global__ void __launch_bounds__(256) k_chan_partial(const float* __restrict__ z, int ld, int C, int M,
                                                      const double* __restrict__ mean, int mode,
                                                      float* __restrict__ part) {
  // blockDim 256 = 8 rows x 32 channels; grid (ceil(C/32), nblk)
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int r = threadIdx.x >> 5;
  float s = 0.f;
  if (c < C) {
    const float mu = mode ? (float)mean[c] : 0.f;
    for (int m = blockIdx.y * 8 + r; m < M; m += gridDim.y * 8) {
      float v = z[(size_t)m * ld + c] - mu;
      s += mode ? v * v : v;
    }
  }
  __shared__ float sm[8][33];
  sm[r][threadIdx.x & 31] = s;
  __syncthreads();
  if (r == 0 && c < C) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += sm[i][threadIdx.x];
    part[(size_t)blockIdx.y * C + c] = t;
  }
}

// Sum of the nblk partials part[b * stride + off] of one channel by one warp: FP32 per
// lane, FP64 across lanes (the result is in every lane).
__device__ __forceinline__ double warp_partials(const float* __restrict__ part, int nblk, size_t stride, size_t off) {
  const int lane = threadIdx.x & 31;
  float t = 0.f;
  for (int b = lane; b < nblk; b += 32) t += part[(size_t)b * stride + off];
  double d = t;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  return d;
}

// One warp per channel (blockDim 128: four channels per block).
__global__ void k_chan_finalize(const float* __restrict__ part, int nblk, int C, double scale,
                                double* __restrict__ out) {
  const int c = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (c >= C) return;
  const double s = warp_partials(part, nblk, C, c);
  if ((threadIdx.x & 31) == 0) out[c] = s * scale;
}

// scale = gamma / sqrt(var + eps), shift = beta - mean * scale; running-stat update.
__global__ void k_bn_coeffs(const double* __restrict__ mean, const double* __restrict__ var,
                            const float* __restrict__ gamma, const float* __restrict__ beta, int C,
                            float* __restrict__ scale, float* __restrict__ shift, float* __restrict__ rmean,
                            float* __restrict__ rvar, int update_running, double unbias, float momentum) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const double rs = 1.0 / sqrt(var[c] + (double)kBnEps);
  const double sc = (double)gamma[c] * rs;
  scale[c] = (float)sc;
  shift[c] = (float)((double)beta[c] - mean[c] * sc);
  if (update_running) {
    rmean[c] = (float)((1.0 - momentum) * rmean[c] + momentum * mean[c]);
    rvar[c] = (float)((1.0 - momentum) * rvar[c] + momentum * var[c] * unbias);
  }
}

// Inference coefficients from running statistics.
__global__ void k_bn_coeffs_eval(const float* __restrict__ rmean, const float* __restrict__ rvar,
                                 const float* __restrict__ gamma, const float* __restrict__ beta, int C,
                                 float* __restrict__ scale, float* __restrict__ shift) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const float sc = gamma[c] / sqrtf(rvar[c] + kBnEps);
  scale[c] = sc;
  shift[c] = beta[c] - rmean[c] * sc;
}

// y = act(z * scale + shift) -> BF16 slice of an NHWC tensor.
__global__ void k_bn_act(const float* __restrict__ z, int ldz, int C, int M, const float* __restrict__ scale,
                         const float* __restrict__ shift, int act, __nv_bfloat16* __restrict__ y, int ldy) {
  const size_t n = (size_t)M * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t m = i / C;
    const int c = (int)(i - m * C);
    float v = z[m * ldz + c] * scale[c] + shift[c];
    if (act) v = elu_f(v);
    y[m * ldy + c] = __float2bfloat16_rn(v);
  }
}

// BatchNorm backward, pass 1: gy = g (* eLU'(y) if act); partial sums of gy and gy * xhat.
__global__ void __launch_bounds__(256) k_bn_bwd_partial(const float* __restrict__ g, int ldg,
                                                        const float* __restrict__ z, int ldz, int C, int M,
                                                        const double* __restrict__ mean, const double* __restrict__ var,
                                                        const float* __restrict__ scale,
                                                        const float* __restrict__ shift, int act,
                                                        float* __restrict__ part) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int r = threadIdx.x >> 5;
  float s1 = 0.f, s2 = 0.f;
  if (c < C) {
    const float mu = (float)mean[c], rs = (float)(1.0 / sqrt(var[c] + (double)kBnEps));
    for (int m = blockIdx.y * 8 + r; m < M; m += gridDim.y * 8) {
      const float zz = z[(size_t)m * ldz + c];
      float gy = g[(size_t)m * ldg + c];
      if (act) gy *= elu_grad(zz * scale[c] + shift[c]);
      s1 += gy;
      s2 += gy * (zz - mu) * rs;
    }
  }
  __shared__ float sm1[8][33], sm2[8][33];
  sm1[r][threadIdx.x & 31] = s1;
  sm2[r][threadIdx.x & 31] = s2;
  __syncthreads();
  if (r == 0 && c < C) {
    float t1 = 0.f, t2 = 0.f;
    for (int i = 0; i < 8; ++i) { t1 += sm1[i][threadIdx.x]; t2 += sm2[i][threadIdx.x]; }
    part[((size_t)blockIdx.y * C + c) * 2] = t1;
    part[((size_t)blockIdx.y * C + c) * 2 + 1] = t2;
  }
}

// Per-channel totals (gamma, beta gradients) and the FP32 coefficients of pass 2:
// coef[c] = {gamma rstd, s1 / M, s2 / M, mean, rstd}.
__global__ void k_bn_bwd_finalize(const float* __restrict__ part, int nblk, int C, int M,
                                  const double* __restrict__ mean, const double* __restrict__ var,
                                  const float* __restrict__ gamma, float* __restrict__ coef,
                                  float* __restrict__ ggamma, float* __restrict__ gbeta) {
  const int c = blockIdx.x * 4 + (threadIdx.x >> 5);   // one warp per channel
  if (c >= C) return;
  const double s1 = warp_partials(part, nblk, 2 * (size_t)C, 2 * (size_t)c);
  const double s2 = warp_partials(part, nblk, 2 * (size_t)C, 2 * (size_t)c + 1);
  if ((threadIdx.x & 31) != 0) return;
  gbeta[c] += (float)s1;
  ggamma[c] += (float)s2;
  const double rs = 1.0 / sqrt(var[c] + (double)kBnEps);
  coef[5 * c] = (float)(gamma[c] * rs);
  coef[5 * c + 1] = (float)(s1 / M);
  coef[5 * c + 2] = (float)(s2 / M);
  coef[5 * c + 3] = (float)mean[c];
  coef[5 * c + 4] = (float)rs;
}

// BatchNorm backward, pass 2: gz = gamma rstd (gy - s1/M - xhat s2/M), FP32 throughout.
__global__ void k_bn_bwd_apply(const float* __restrict__ g, int ldg, const float* __restrict__ z, int ldz, int C,
                               int M, const float* __restrict__ coef, const float* __restrict__ scale,
                               const float* __restrict__ shift, int act, float* __restrict__ gz, int ldo) {
  const size_t n = (size_t)M * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t m = i / C;
    const int c = (int)(i - m * C);
    const float zz = z[m * ldz + c];
    float gy = g[m * ldg + c];
    if (act) gy *= elu_grad(zz * scale[c] + shift[c]);
    const float* k = coef + 5 * c;
    const float xhat = (zz - k[3]) * k[4];
    gz[m * ldo + c] = k[0] * (gy - k[1] - xhat * k[2]);
  }
}

// g *= eLU'(u) for an input that passed through eLU on load (u in BF16).
__global__ void k_elu_bwd(float* __restrict__ g, int ldg, const __nv_bfloat16* __restrict__ u, int ldu, int C, int M,
                          size_t plane) {
  const size_t n = (size_t)M * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t m = i / C;
    const int c = (int)(i - m * C);
    g[m * ldg + c] *= elu_grad(bf(u[(plane ? m % plane : m) * ldu + c]));
  }
}

// dst (slice) += src (slice), FP32.
__global__ void k_add_slice(float* __restrict__ dst, int ldd, const float* __restrict__ src, int lds, int C, int M) {
  const size_t n = (size_t)M * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t m = i / C;
    const int c = (int)(i - m * C);
    dst[m * ldd + c] += src[m * lds + c];
  }
}

// FP32 -> BF16 slice copy.
__global__ void k_to_bf16(const float* __restrict__ src, int lds, __nv_bfloat16* __restrict__ dst, int ldd, int C,
                          int M) {
  const size_t n = (size_t)M * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t m = i / C;
    const int c = (int)(i - m * C);
    dst[m * ldd + c] = __float2bfloat16_rn(src[m * lds + c]);
  }
}

// MSE loss (Eq. 3.7): loss = sum (out - tgt)^2 / B; gout = 2 (out - tgt) / B.
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ tgt, size_t n, int B,
                      float* __restrict__ gout, float* __restrict__ part) {
  float s = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = out[i] - tgt[i];
    gout[i] = 2.f * d / B;
    s += d * d;
  }
  __shared__ float sm[256];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_sum_partials(const float* __restrict__ part, int n, int B, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    *loss = (float)(s / B);
  }
}

// Boundary terms of h^2 A for the residual loss (Sec. 2.4's padding modes: bc 0 zero,
// 1 reflection, 2 replication).  Centre weight: 4, less one per boundary side under
// replication.  Reflection adds the inward neighbour once more at a boundary node, so
// A is not symmetric there; its transpose instead adds, at the inward neighbour of a
// boundary node, that boundary node once more.
__device__ __forceinline__ float resloss_centre(int bc, int ix, int iy, int nx, int ny) {
  return bc == 2 ? 4.f - (float)((ix == 0) + (ix == nx - 1) + (iy == 0) + (iy == ny - 1)) : 4.f;
}
__device__ __forceinline__ float2 resloss_reflect(const float2* v, size_t i, int ix, int iy, int nx, int ny,
                                                  bool transpose) {
  float2 e = make_float2(0.f, 0.f);
  const int lo = transpose ? 1 : 0, hi = transpose ? 2 : 1;   // node at which the extra term enters
  // forward: at x = 0 add x + 1, at x = nx - 1 add x - 1; transpose: at x = 1 add x - 1,
  // at x = nx - 2 add x + 1 (likewise in y)
  if (ix == lo) { const float2 a = v[transpose ? i - 1 : i + 1]; e.x += a.x; e.y += a.y; }
  if (ix == nx - hi) { const float2 a = v[transpose ? i + 1 : i - 1]; e.x += a.x; e.y += a.y; }
  if (iy == lo) { const float2 a = v[transpose ? i - nx : i + nx]; e.x += a.x; e.y += a.y; }
  if (iy == ny - hi) { const float2 a = v[transpose ? i + nx : i - nx]; e.x += a.x; e.y += a.y; }
  return e;
}

// Unsupervised residual loss (the Remark following Eq. 3.7) on network outputs y
// [B][ny][nx][2] (units e / s) and inputs x [B][ny][nx][4] (channels 0, 1 = h^2 r / s):
//   rho = h^2 A y - x_r,  (h^2 A y)_p = 4 y_p - (sum of the 4 neighbours, zero outside)
//                                      - c kappa2_p (1 - i gamma_p) y_p,  c = h^2 omega^2,
// with the boundary terms above.  Per-block sums of |rho|^2 go to part.
__global__ void __launch_bounds__(256) k_resloss_rho(const float2* __restrict__ y, const float* __restrict__ x,
                                                     int B, int ny, int nx, float c, const float* __restrict__ k2,
                                                     const float* __restrict__ gam, int bc, float2* __restrict__ rho,
                                                     float* __restrict__ part) {
  const size_t N = (size_t)nx * ny, M = N * B;
  float s = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i % N;
    const int iy = (int)(p / nx), ix = (int)(p - (size_t)iy * nx);
    const float2 v = y[i];
    float2 nb = make_float2(0.f, 0.f);
    if (ix > 0) { nb.x += y[i - 1].x; nb.y += y[i - 1].y; }
    if (ix < nx - 1) { nb.x += y[i + 1].x; nb.y += y[i + 1].y; }
    if (iy > 0) { nb.x += y[i - nx].x; nb.y += y[i - nx].y; }
    if (iy < ny - 1) { nb.x += y[i + nx].x; nb.y += y[i + nx].y; }
    if (bc == 1) { const float2 e = resloss_reflect(y, i, ix, iy, nx, ny, false); nb.x += e.x; nb.y += e.y; }
    const float cw = resloss_centre(bc, ix, iy, nx, ny);
    const float d = c * k2[p], g = gam[p];
    // -d (1 - i g)(a + i b) = -d (a + g b) - i d (b - g a)
    const float rx = cw * v.x - nb.x - d * (v.x + g * v.y) - x[i * 4];
    const float ry = cw * v.y - nb.y - d * (v.y - g * v.x) - x[i * 4 + 1];
    rho[i] = make_float2(rx, ry);
    s += rx * rx + ry * ry;
  }
  __shared__ float sm[256];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

// d loss / d (Re y, Im y) = (2 / B) conj(h^2 A^T conj(rho)) = (2 / B) h^2 A^H rho: the
// stencil of A^T (A itself but for reflection's boundary terms) with the diagonal's
// imaginary part negated.
__global__ void __launch_bounds__(256) k_resloss_grad(const float2* __restrict__ rho, int B, int ny, int nx, float c,
                                                      const float* __restrict__ k2, const float* __restrict__ gam,
                                                      int bc, float2* __restrict__ gout) {
  const size_t N = (size_t)nx * ny, M = N * B;
  const float sc = 2.f / B;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i % N;
    const int iy = (int)(p / nx), ix = (int)(p - (size_t)iy * nx);
    const float2 v = rho[i];
    float2 nb = make_float2(0.f, 0.f);
    if (ix > 0) { nb.x += rho[i - 1].x; nb.y += rho[i - 1].y; }
    if (ix < nx - 1) { nb.x += rho[i + 1].x; nb.y += rho[i + 1].y; }
    if (iy > 0) { nb.x += rho[i - nx].x; nb.y += rho[i - nx].y; }
    if (iy < ny - 1) { nb.x += rho[i + nx].x; nb.y += rho[i + nx].y; }
    if (bc == 1) { const float2 e = resloss_reflect(rho, i, ix, iy, nx, ny, true); nb.x += e.x; nb.y += e.y; }
    const float cw = resloss_centre(bc, ix, iy, nx, ny);
    const float d = c * k2[p], g = gam[p];
    // -d (1 + i g)(a + i b) = -d (a - g b) - i d (b + g a)
    gout[i] = make_float2(sc * (cw * v.x - nb.x - d * (v.x - g * v.y)), sc * (cw * v.y - nb.y - d * (v.y + g * v.x)));
  }
}

// Adam (Kingma & Ba) with bias correction on the flat FP32 parameter vector.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ s, __nv_bfloat16* __restrict__ d, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    d[i] = __float2bfloat16_rn(s[i]);
}

// Network input from complex residuals (Sec. 3.4): channels (Re, Im) of h^2 r / s with
// s = RMS(h^2 r) per sample, then kappa^2 and gamma.  Two passes over many blocks:
// per-block partial sums of |r|^2, then every block of the writer sums its sample's
// partials (one warp, fixed order) and writes the BF16 input.  kInBlocks blocks per sample:
// enough loads in flight for these HBM-bound sweeps at a few samples per pass (64 blocks
// per sample left them at about 1 TB/s).
constexpr int kInBlocks = 256;

template <typename T2>
__global__ void __launch_bounds__(256) k_input_partial(const T2* __restrict__ r, int N, float* __restrict__ part,
                                                       const int* gate) {
  const int b = blockIdx.y;
  if (gate && !gate[b]) return;
  const T2* rb = r + (size_t)b * N;
  float s = 0.f;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    T2 v = rb[p];
    s += (float)(v.x * v.x + v.y * v.y);
  }
  __shared__ float sm[256];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[b * kInBlocks + blockIdx.x] = sm[0];
}

// Offset of channel 0 of pixel (b, y, x) in the space-to-depth layout of a 4-channel
// image: [b][y / 2][x / 2][(y % 2) * 2 + x % 2][4] (16 channels per 2x2 block).
__device__ __forceinline__ size_t s2d_off(int b, int y, int x, int ny, int nx) {
  return ((((size_t)b * (ny >> 1) + (y >> 1)) * (nx >> 1) + (x >> 1)) * 4 + ((y & 1) * 2 + (x & 1))) * 4;
}

// S2D: x holds the space-to-depth layout (nx columns per image row, 4 channels), else
// ldx-channel pixels with channels 4.. zeroed.
template <typename T2, bool S2D>
__global__ void __launch_bounds__(256) k_input_write(const T2* __restrict__ r, int N, int nx, double h2,
                                                     const float* __restrict__ k2, const float* __restrict__ gam,
                                                     const float* __restrict__ part, __nv_bfloat16* __restrict__ x,
                                                     int ldx, float* __restrict__ sc, const int* gate, int rpp, int b0) {
  const int b = blockIdx.y;
  if (gate && !gate[b]) return;
  if (rpp > 0) k2 += (size_t)((b0 + b) / rpp) * N;   // this right-hand side's medium (a batch of problems)
  __shared__ float s_scale;
  if (threadIdx.x < 32) {
    // lane l adds partials l, l + 32, ...; then a fixed shuffle tree
    double t = 0.0;
    for (int i = threadIdx.x; i < kInBlocks; i += 32) t += part[b * kInBlocks + i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) {
      const float rms = (float)(sqrt(t / N) * h2);
      s_scale = rms > 0.f ? rms : 1.f;
      if (blockIdx.x == 0) sc[b] = s_scale;
    }
  }
  __syncthreads();
  const float f = (float)h2 / s_scale;
  const T2* rb = r + (size_t)b * N;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    T2 v = rb[p];
    if (S2D) {
      const int y = p / nx, xx = p - y * nx;
      __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(x + s2d_off(b, y, xx, N / nx, nx));
      o[0] = __floats2bfloat162_rn((float)v.x * f, (float)v.y * f);
      o[1] = __floats2bfloat162_rn(k2[p], gam[p]);
      continue;
    }
    __nv_bfloat16* o = x + ((size_t)b * N + p) * ldx;
    o[0] = __float2bfloat16_rn((float)v.x * f);
    o[1] = __float2bfloat16_rn((float)v.y * f);
    o[2] = __float2bfloat16_rn(k2[p]);
    o[3] = __float2bfloat16_rn(gam[p]);
    for (int c = 4; c < ldx; ++c) o[c] = __float2bfloat16_rn(0.f);
  }
}

// FP32 [M][lds] (4 channels) into the space-to-depth BF16 layout.
__global__ void k_to_bf16_s2d(const float* __restrict__ src, int lds, __nv_bfloat16* __restrict__ dst, int B,
                              int ny, int nx) {
  const size_t M = (size_t)B * ny * nx;
  for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(m % nx);
    const size_t r = m / nx;
    const int y = (int)(r % ny), b = (int)(r / ny);
    const float* q = src + m * lds;
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(dst + s2d_off(b, y, x, ny, nx));
    o[0] = __floats2bfloat162_rn(q[0], q[1]);
    o[1] = __floats2bfloat162_rn(q[2], q[3]);
  }
}

// Space-to-depth BF16 layout back to ldd-channel pixels (channels 4.. zeroed).
__global__ void k_s2d_to_std(const __nv_bfloat16* __restrict__ xs, __nv_bfloat16* __restrict__ dst, int ldd, int B,
                             int ny, int nx) {
  const size_t M = (size_t)B * ny * nx;
  for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(m % nx);
    const size_t r = m / nx;
    const int y = (int)(r % ny), b = (int)(r / ny);
    const __nv_bfloat16* q = xs + s2d_off(b, y, x, ny, nx);
    __nv_bfloat16* o = dst + m * ldd;
    for (int c = 0; c < ldd; ++c) o[c] = c < 4 ? q[c] : __float2bfloat16_rn(0.f);
  }
}

// e = s (out_0 + i out_1), optionally added to e.
template <typename T2>
__global__ void k_write_output(const float* __restrict__ out, int ny, int nx, const float* __restrict__ sc,
                               T2* __restrict__ e, int add, const int* gate) {
  const int b = blockIdx.y;
  if (gate && !gate[b]) return;
  const int N = nx * ny;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
    const float* o = out + ((size_t)b * N + p) * 2;
    T2 v = e[(size_t)b * N + p];
    const float s = sc[b];
    if (add) { v.x += o[0] * s; v.y += o[1] * s; }
    else { v.x = o[0] * s; v.y = o[1] * s; }
    e[(size_t)b * N + p] = v;
  }
}

__global__ void k_gamma_field(int ny, int nx, int width, float gmax, float* __restrict__ g) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx * ny) return;
  const int y = p / nx, x = p - y * nx;
  const int d = min(min(x, nx - 1 - x), min(y, ny - 1 - y));
  float v = 0.f;
  if (d < width) { float t = 1.f - (float)d / (float)width; v = gmax * t * t; }
  g[p] = v;
}

__global__ void k_chan_finalize_add(const float* __restrict__ part, int nblk, int C, float* __restrict__ dst) {
  const int c = blockIdx.x * 4 + (threadIdx.x >> 5);   // one warp per channel
  if (c >= C) return;
  const double s = warp_partials(part, nblk, C, c);
  if ((threadIdx.x & 31) == 0) dst[c] += (float)s;
}

// dst[p][c] (+)= sum_b src[b][p][c]: gradient of a tensor shared by the whole batch.
__global__ void k_batch_sum(const float* __restrict__ src, int lds, int B, size_t P, int C,
                            float* __restrict__ dst, int ldd, int accumulate) {
  const size_t n = P * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / C;
    const int c = (int)(i - p * C);
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += src[((size_t)b * P + p) * lds + c];
    if (accumulate) dst[p * ldd + c] += s;
    else dst[p * ldd + c] = s;
  }
}

// SplitMix64 (Steele, Lea & Flood 2014): output for stream `seed` at counter i.
__device__ __forceinline__ unsigned long long splitmix(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long i) {
  return ((double)(splitmix(seed, i) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// x[j][p] ~ CN(0,1): Box-Muller on the uniform pair (2p, 2p+1) of stream seed + 1 + j.
__global__ void k_complex_normal(unsigned long long seed, int count, size_t N, double2* __restrict__ x) {
  const int j = blockIdx.y;
  const unsigned long long sj = seed + 1ull + (unsigned long long)j;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
    const double u1 = u01(sj, 2 * p), u2 = u01(sj, 2 * p + 1);
    const double rad = sqrt(-2.0 * log(u1)) * 0.70710678118654752440;
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    x[(size_t)j * N + p] = make_double2(rad * cs, rad * sn);
  }
}

// Training batch (Sec. 3.4): sample i mixes pairs idx[i][q] with complex
// coefficients coef[i][q] (augmentation by linear combinations), then
// x = [Re, Im](h^2 r' / s), kappa^2, gamma and target = [Re, Im](e' / s),
// s = RMS(h^2 r').
__global__ void __launch_bounds__(256) k_make_batch(const double2* __restrict__ r, const double2* __restrict__ e,
                                                    size_t N, const int* __restrict__ idx,
                                                    const double2* __restrict__ coef, int nmix, double h2,
                                                    const float* __restrict__ k2, const float* __restrict__ gam,
                                                    float* __restrict__ x, float* __restrict__ tgt) {
  const int i = blockIdx.x;
  const int* id = idx + (size_t)i * nmix;
  const double2* cf = coef + (size_t)i * nmix;
  float acc = 0.f;
  for (size_t p = threadIdx.x; p < N; p += blockDim.x) {
    double rx = 0.0, ry = 0.0;
    for (int q = 0; q < nmix; ++q) {
      const double2 v = r[(size_t)id[q] * N + p], c = cf[q];
      rx += c.x * v.x - c.y * v.y;
      ry += c.x * v.y + c.y * v.x;
    }
    acc += (float)(rx * rx + ry * ry);
  }
  __shared__ float sm[256];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  const double rms = sqrt((double)sm[0] / (double)N) * h2;
  const double sc = rms > 0.0 ? rms : 1.0;
  for (size_t p = threadIdx.x; p < N; p += blockDim.x) {
    double rx = 0.0, ry = 0.0, ex = 0.0, ey = 0.0;
    for (int q = 0; q < nmix; ++q) {
      const double2 v = r[(size_t)id[q] * N + p], w = e[(size_t)id[q] * N + p], c = cf[q];
      rx += c.x * v.x - c.y * v.y;
      ry += c.x * v.y + c.y * v.x;
      ex += c.x * w.x - c.y * w.y;
      ey += c.x * w.y + c.y * w.x;
    }
    float* xo = x + ((size_t)i * N + p) * 4;
    xo[0] = (float)(rx * h2 / sc);
    xo[1] = (float)(ry * h2 / sc);
    xo[2] = k2[p];
    xo[3] = gam[p];
    float* to = tgt + ((size_t)i * N + p) * 2;
    to[0] = (float)(ex / sc);
    to[1] = (float)(ey / sc);
  }
}

// WT[co][tap * cin + ci] = P[(tap * cin + ci) * cout + co] (BF16).
__global__ void k_weights_kmajor(const float* __restrict__ P, __nv_bfloat16* __restrict__ WT, int K, int cout) {
  const size_t n = (size_t)K * cout;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t co = i / K, k = i - co * K;
    WT[i] = __float2bfloat16_rn(P[k * cout + co]);
  }
}

__global__ void k_elu_copy(const __nv_bfloat16* __restrict__ src, int lds, int C, size_t M,
                           __nv_bfloat16* __restrict__ dst, int ldd) {
  const size_t n = M * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t m = i / C;
    const int c = (int)(i - m * C);
    dst[m * ldd + c] = __float2bfloat16_rn(elu_f(bf(src[m * lds + c])));
  }
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace

void weights_kmajor(const float* P, __nv_bfloat16* WT, int taps, int cin, int cout, cudaStream_t s) {
  k_weights_kmajor<<<grid_for((size_t)taps * cin * cout), 256, 0, s>>>(P, WT, taps * cin, cout);
}

void elu_copy_bf16(const __nv_bfloat16* src, int lds, int C, size_t M, __nv_bfloat16* dst, int ldd, cudaStream_t s) {
  k_elu_copy<<<grid_for(M * C), 256, 0, s>>>(src, lds, C, M, dst, ldd);
}

bool conv_thin(const ConvArgs& a, cudaStream_t s) {
  const int Cin = a.c0 + a.c1;
  const size_t wbytes = (size_t)a.k * a.k * Cin * 4;
  const int M = a.B * a.Ho * a.Wo;
  const int grid = (M + 127) / 128;
  if (a.Cout <= 2 && wbytes * 2 <= 96 * 1024) {
    static DeviceOnce once2;   // per-device kernel attribute
    if (!set_dynamic_smem(once2, k_conv_thin<2>, 96 * 1024)) return false;
    k_conv_thin<2><<<grid, 128, wbytes * 2, s>>>(a);
    return true;
  }
  if (Cin <= 8 && a.Cout <= 32 && wbytes * 32 <= 96 * 1024) {
    static DeviceOnce once32;
    if (!set_dynamic_smem(once32, k_conv_thin<32>, 96 * 1024)) return false;
    k_conv_thin<32><<<grid, 128, wbytes * 32, s>>>(a);
    return true;
  }
  return false;
}

void conv_forward(const ConvArgs& a, cudaStream_t s) {
  if (conv_thin(a, s)) return;
  const int M = a.B * a.Ho * a.Wo;
  dim3 grid((M + 63) / 64, (a.Cout + 63) / 64);
  k_conv_simt<<<grid, 256, 0, s>>>(a);
}

void conv_wgrad(const ConvArgs& a, const float* G, int ldg, float* gW, cudaStream_t s) {
  const int M = a.B * a.Ho * a.Wo;
  const int Cin = a.c0 + a.c1;
  const int tiles = a.k * a.k * ((Cin + 31) / 32) * ((a.Cout + 31) / 32);
  int chunk = 2048;
  int nchunk = (M + chunk - 1) / chunk;
  while (nchunk > 1 && (long long)tiles * nchunk > 4096) { chunk *= 2; nchunk = (M + chunk - 1) / chunk; }
  k_wgrad_simt<<<dim3(tiles, nchunk), 256, 0, s>>>(a, G, ldg, gW, chunk);
}

void bn_batch_stats(const float* z, int ldz, int C, int M, double* mean, double* var, float* part, int nblk,
                    cudaStream_t s) {
  k_chan_partial<<<dim3((C + 31) / 32, nblk), 256, 0, s>>>(z, ldz, C, M, nullptr, 0, part);
  k_chan_finalize<<<(C + 3) / 4, 128, 0, s>>>(part, nblk, C, 1.0 / M, mean);
  k_chan_partial<<<dim3((C + 31) / 32, nblk), 256, 0, s>>>(z, ldz, C, M, mean, 1, part);
  k_chan_finalize<<<(C + 3) / 4, 128, 0, s>>>(part, nblk, C, 1.0 / M, var);
}

void bn_coeffs(const double* mean, const double* var, const float* gamma, const float* beta, int C, float* scale,
               float* shift, float* rmean, float* rvar, bool update, int M, cudaStream_t s) {
  k_bn_coeffs<<<(C + 127) / 128, 128, 0, s>>>(mean, var, gamma, beta, C, scale, shift, rmean, rvar, update ? 1 : 0,
                                              M > 1 ? (double)M / (M - 1) : 1.0, kBnMomentum);
}

void bn_coeffs_eval(const float* rmean, const float* rvar, const float* gamma, const float* beta, int C,
                    float* scale, float* shift, cudaStream_t s) {
  k_bn_coeffs_eval<<<(C + 127) / 128, 128, 0, s>>>(rmean, rvar, gamma, beta, C, scale, shift);
}

void bn_act(const float* z, int ldz, int C, int M, const float* scale, const float* shift, bool act,
            __nv_bfloat16* y, int ldy, cudaStream_t s) {
  k_bn_act<<<grid_for((size_t)M * C), 256, 0, s>>>(z, ldz, C, M, scale, shift, act ? 1 : 0, y, ldy);
}

void bn_backward(const float* g, int ldg, const float* z, int ldz, int C, int M, const double* mean, const double* var,
                 const float* scale, const float* shift, bool act, const float* gamma, float* ggamma, float* gbeta,
                 float* part, int nblk, float* coef, float* gz, int ldo, cudaStream_t s) {
  k_bn_bwd_partial<<<dim3((C + 31) / 32, nblk), 256, 0, s>>>(g, ldg, z, ldz, C, M, mean, var, scale, shift,
                                                            act ? 1 : 0, part);
  k_bn_bwd_finalize<<<(C + 3) / 4, 128, 0, s>>>(part, nblk, C, M, mean, var, gamma, coef, ggamma, gbeta);
  k_bn_bwd_apply<<<grid_for((size_t)M * C), 256, 0, s>>>(g, ldg, z, ldz, C, M, coef, scale, shift, act ? 1 : 0, gz,
                                                         ldo);
}

void elu_backward_inplace(float* g, int ldg, const __nv_bfloat16* u, int ldu, int C, int M, size_t plane,
                          cudaStream_t s) {
  k_elu_bwd<<<grid_for((size_t)M * C), 256, 0, s>>>(g, ldg, u, ldu, C, M, plane);
}

void add_slice(float* dst, int ldd, const float* src, int lds, int C, int M, cudaStream_t s) {
  k_add_slice<<<grid_for((size_t)M * C), 256, 0, s>>>(dst, ldd, src, lds, C, M);
}

void to_bf16_slice(const float* src, int lds, __nv_bfloat16* dst, int ldd, int C, int M, cudaStream_t s) {
  k_to_bf16<<<grid_for((size_t)M * C), 256, 0, s>>>(src, lds, dst, ldd, C, M);
}

void mse_loss(const float* out, const float* tgt, size_t n, int B, float* gout, float* part, float* loss,
              cudaStream_t s) {
  const int nb = 256;
  k_mse<<<nb, 256, 0, s>>>(out, tgt, n, B, gout, part);
  k_sum_partials<<<1, 32, 0, s>>>(part, nb, B, loss);
}

void residual_loss(const float* y, const float* x, int B, int ny, int nx, float c, const float* k2, const float* gam,
                   int bc, float* rho, float* gout, float* part, float* loss, cudaStream_t s) {
  const int nb = 256;
  k_resloss_rho<<<nb, 256, 0, s>>>((const float2*)y, x, B, ny, nx, c, k2, gam, bc, (float2*)rho, part);
  k_sum_partials<<<1, 32, 0, s>>>(part, nb, B, loss);
  k_resloss_grad<<<grid_for((size_t)B * ny * nx), 256, 0, s>>>((const float2*)rho, B, ny, nx, c, k2, gam, bc,
                                                               (float2*)gout);
}

void adam_update(float* p, const float* g, float* m1, float* m2, size_t n, float lr, float b1, float b2, float eps,
                 int t, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  k_adam<<<grid_for(n), 256, 0, s>>>(p, g, m1, m2, n, lr, b1, b2, eps, c1, c2);
}

void f32_to_bf16(const float* src, __nv_bfloat16* dst, size_t n, cudaStream_t s) {
  k_f32_to_bf16<<<grid_for(n), 256, 0, s>>>(src, dst, n);
}

void make_input(const void* r, bool fp64, int B, int ny, int nx, double h, const float* k2, const float* gam,
                __nv_bfloat16* x, int ldx, float* sc, float* part, const int* gate, cudaStream_t s, bool s2d, int rpp,
                int b0) {
  const int N = nx * ny;
  const dim3 grid(kInBlocks, B);
  if (fp64) {
    k_input_partial<double2><<<grid, 256, 0, s>>>((const double2*)r, N, part, gate);
    if (s2d)
      k_input_write<double2, true><<<grid, 256, 0, s>>>((const double2*)r, N, nx, h * h, k2, gam, part, x, ldx, sc,
                                                        gate, rpp, b0);
    else
      k_input_write<double2, false><<<grid, 256, 0, s>>>((const double2*)r, N, nx, h * h, k2, gam, part, x, ldx, sc,
                                                         gate, rpp, b0);
  } else {
    k_input_partial<float2><<<grid, 256, 0, s>>>((const float2*)r, N, part, gate);
    if (s2d)
      k_input_write<float2, true><<<grid, 256, 0, s>>>((const float2*)r, N, nx, h * h, k2, gam, part, x, ldx, sc,
                                                       gate, rpp, b0);
    else
      k_input_write<float2, false><<<grid, 256, 0, s>>>((const float2*)r, N, nx, h * h, k2, gam, part, x, ldx, sc,
                                                        gate, rpp, b0);
  }
}

void to_bf16_s2d(const float* src, int lds, __nv_bfloat16* dst, int B, int ny, int nx, cudaStream_t s) {
  k_to_bf16_s2d<<<grid_for((size_t)B * ny * nx), 256, 0, s>>>(src, lds, dst, B, ny, nx);
}

void s2d_to_std(const __nv_bfloat16* xs, __nv_bfloat16* dst, int ldd, int B, int ny, int nx, cudaStream_t s) {
  k_s2d_to_std<<<grid_for((size_t)B * ny * nx), 256, 0, s>>>(xs, dst, ldd, B, ny, nx);
}

void write_output(const float* out, bool fp64, int B, int ny, int nx, const float* sc, void* e, bool add,
                  const int* gate, cudaStream_t s) {
  dim3 grid((nx * ny + 255) / 256 > 1024 ? 1024 : (nx * ny + 255) / 256, B);
  if (fp64) k_write_output<double2><<<grid, 256, 0, s>>>(out, ny, nx, sc, (double2*)e, add ? 1 : 0, gate);
  else k_write_output<float2><<<grid, 256, 0, s>>>(out, ny, nx, sc, (float2*)e, add ? 1 : 0, gate);
}

void chan_sum_add(const float* g, int ld, int C, int M, float* dst, float* part, int nblk, cudaStream_t s) {
  k_chan_partial<<<dim3((C + 31) / 32, nblk), 256, 0, s>>>(g, ld, C, M, nullptr, 0, part);
  k_chan_finalize_add<<<(C + 3) / 4, 128, 0, s>>>(part, nblk, C, dst);
}

void batch_sum(const float* src, int lds, int B, size_t P, int C, float* dst, int ldd, bool accumulate,
               cudaStream_t s) {
  k_batch_sum<<<grid_for(P * C), 256, 0, s>>>(src, lds, B, P, C, dst, ldd, accumulate ? 1 : 0);
}

void complex_normal(unsigned long long seed, int count, size_t N, double2* x, cudaStream_t s) {
  dim3 grid((unsigned)std::min<size_t>((N + 255) / 256, 1024), count);
  k_complex_normal<<<grid, 256, 0, s>>>(seed, count, N, x);
}

void make_batch(const double2* r, const double2* e, size_t N, int count, const int* idx, const double2* coef, int nmix,
                double h, const float* k2, const float* gam, float* x, float* tgt, cudaStream_t s) {
  k_make_batch<<<count, 256, 0, s>>>(r, e, N, idx, coef, nmix, h * h, k2, gam, x, tgt);
}

void gamma_field(int ny, int nx, int width, float gmax, float* g, cudaStream_t s) {
  k_gamma_field<<<(nx * ny + 255) / 256, 256, 0, s>>>(ny, nx, width, gmax, g);
}

}  // namespace helm
