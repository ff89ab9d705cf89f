// Direct convolutions on CUDA cores for the two U-Net layers whose channel counts
// leave an MMA tile mostly empty (Sec. 3.1, Fig. 2): the first down convolution
// (5x5, stride 2, from the 4-channel network input) and the last up convolution
// (transposed 5x5, stride 2, to the 2-channel output).  On the tensor cores these
// pad K to 64 (input) or N to 16 (output) and run at a few percent of the MMA rate.
//
// Both kernels stage one output tile's input window and all weights in shared
// memory as FP32 and accumulate in FP32 registers:
//   k_down_small: 32x16 output pixels per block, two pixels (rows ty, ty + 16)
//     and all output channels (<= 32) per thread; the input window is
//     pixel-major with the channels of a pixel contiguous (float4 loads).
//   k_up_small: 16x16 output pixels per block; each warp serves one output phase
//     (oy mod 2, ox mod 2), so the taps it visits -- and the weights it reads --
//     are uniform across the warp; the input window is channel-major; the eLU of
//     the inputs is applied while staging.
// Outputs: FP32 (+ bias, + residual), or BatchNorm (scale, shift) and eLU fused
// into BF16 as in the tensor-core epilogue.
#include <cuda_bf16.h>

#include <cstdint>

#include "unet_internal.cuh"

namespace helm {

namespace {

constexpr int TS = 16;   // output tile edge

__device__ __forceinline__ float bfv(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float elu_s(float x) { return x > 0.f ? x : expm1f(x); }

// ---------------------------------------------------------------------------
// 5x5 stride-2 convolution from <= 8 input channels (one source) to <= CO outputs.
// Tile: DY x TS output pixels; thread (ty, tx) computes rows ty and ty + TS, so every
// weight read from shared memory feeds two pixels.
constexpr int DY = 2 * TS;

template <int CIP, int CO>
__global__ void __launch_bounds__(256) k_down_small(ConvArgs a) {
  constexpr int K = 5, S = 2;
  constexpr int IW = (TS - 1) * S + K;          // 35 input columns
  constexpr int IH = (DY - 1) * S + K;          // 67 input rows
  extern __shared__ __align__(16) float sm[];
  float* sIn = sm;                               // [IH][IW][CIP]
  float* sW = sIn + IH * IW * CIP;               // [K*K][CIP][CO]
  const int tid = threadIdx.x;
  const int tilesx = (a.Wo + TS - 1) / TS;
  const int ox0 = (blockIdx.x % tilesx) * TS, oy0 = (blockIdx.x / tilesx) * DY;
  const int b = blockIdx.y;
  const int ix0 = ox0 * S - a.pad, iy0 = oy0 * S - a.pad;
  for (int i = tid; i < K * K * CIP * CO; i += 256) {
    const int co = i % CO, r = i / CO, ci = r % CIP, tap = r / CIP;
    sW[i] = (ci < a.c0 && co < a.Cout) ? bfv(a.W[tap * a.wst + ci * a.wsk + co * a.wsn]) : 0.f;
  }
  const __nv_bfloat16* in = (const __nv_bfloat16*)a.in0;
  const bool v16 = (a.ld0 % 8 == 0) && !((uintptr_t)in & 15);   // one 16-byte load per pixel
  for (int i = tid; i < IH * IW; i += 256) {
    const int r = i / IW, c = i - r * IW;
    const int gy = iy0 + r, gx = ix0 + c;
    float* d = sIn + i * CIP;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (gy >= 0 && gy < a.Hi && gx >= 0 && gx < a.Wi) {
      const __nv_bfloat16* src = in + (((size_t)b * a.Hi + gy) * a.Wi + gx) * a.ld0;
      if (v16) {
        const uint4 q = *reinterpret_cast<const uint4*>(src);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float2 t = __bfloat1622float2(h[k]);
          v[2 * k] = t.x; v[2 * k + 1] = t.y;
        }
      } else {
#pragma unroll
        for (int ci = 0; ci < 8; ++ci)
          if (ci < a.c0) v[ci] = bfv(src[ci]);
      }
    }
#pragma unroll
    for (int ci = 0; ci < CIP; ++ci) {
      float x = ci < a.c0 ? v[ci] : 0.f;          // channels past c0 are never read as data
      if (a.in_act) x = elu_s(x);
      d[ci] = x;
    }
  }
  __syncthreads();
  const int ty = tid / TS, tx = tid - ty * TS;
  float acc0[CO], acc1[CO];
#pragma unroll
  for (int j = 0; j < CO; ++j) { acc0[j] = 0.f; acc1[j] = 0.f; }
#pragma unroll 1
  for (int ky = 0; ky < K; ++ky) {
#pragma unroll 1
    for (int kx = 0; kx < K; ++kx) {
      const float* ip0 = sIn + ((ty * S + ky) * IW + tx * S + kx) * CIP;
      const float* ip1 = ip0 + TS * S * IW * CIP;   // row ty + TS
      const float* wp = sW + (ky * K + kx) * CIP * CO;
#pragma unroll
      for (int c4 = 0; c4 < CIP; c4 += 4) {
        const float4 u0 = *reinterpret_cast<const float4*>(ip0 + c4);
        const float4 u1 = *reinterpret_cast<const float4*>(ip1 + c4);
        const float x0[4] = {u0.x, u0.y, u0.z, u0.w}, x1[4] = {u1.x, u1.y, u1.z, u1.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4* w4 = reinterpret_cast<const float4*>(wp + (c4 + q) * CO);
#pragma unroll
          for (int j = 0; j < CO / 4; ++j) {
            const float4 w = w4[j];
            acc0[4 * j] = fmaf(x0[q], w.x, acc0[4 * j]);
            acc0[4 * j + 1] = fmaf(x0[q], w.y, acc0[4 * j + 1]);
            acc0[4 * j + 2] = fmaf(x0[q], w.z, acc0[4 * j + 2]);
            acc0[4 * j + 3] = fmaf(x0[q], w.w, acc0[4 * j + 3]);
            acc1[4 * j] = fmaf(x1[q], w.x, acc1[4 * j]);
            acc1[4 * j + 1] = fmaf(x1[q], w.y, acc1[4 * j + 1]);
            acc1[4 * j + 2] = fmaf(x1[q], w.z, acc1[4 * j + 2]);
            acc1[4 * j + 3] = fmaf(x1[q], w.w, acc1[4 * j + 3]);
          }
        }
      }
    }
  }
  const int ox = ox0 + tx;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int oy = oy0 + ty + h * TS;
    if (oy >= a.Ho || ox >= a.Wo) continue;
    const float* acc = h ? acc1 : acc0;
    const size_t pix = ((size_t)b * a.Ho + oy) * a.Wo + ox;
#pragma unroll
    for (int j = 0; j < CO; ++j) {
      if (j >= a.Cout) break;
      float v = acc[j];
      if (a.bias) v += a.bias[j];
      if (a.res) v += bfv(a.res[pix * a.ldr + j]);
      if (a.ybf) {
        if (a.scale) v = v * a.scale[j] + a.shift[j];
        if (a.ep_act) v = elu_s(v);
        a.ybf[pix * a.ldy + j] = __float2bfloat16_rn(v);
      } else {
        a.out[pix * a.ldo + j] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Transposed 5x5 stride-2 convolution (out[2 i + t - pad] += W[t] in[i]) from up to
// two BF16 sources (the second possibly shared by the batch) to <= CO outputs.
constexpr int UW = TS / 2 + 2;   // input window edge: 10
constexpr int UR = UW + 1;       // padded row stride of a channel plane

template <int CO>
__global__ void __launch_bounds__(256) k_up_small(ConvArgs a) {
  constexpr int K = 5;
  extern __shared__ __align__(16) float sm[];
  const int Cin = a.c0 + a.c1;
  float* sIn = sm;                               // [Cin][UW][UR]
  float* sW = sIn + (size_t)Cin * UW * UR;       // [K*K][Cin][CO]
  const int tid = threadIdx.x;
  const int tilesx = (a.Wo + TS - 1) / TS;
  const int ox0 = (blockIdx.x % tilesx) * TS, oy0 = (blockIdx.x / tilesx) * TS;
  const int b = blockIdx.y;
  const int ix0 = ox0 / 2 - 1, iy0 = oy0 / 2 - 1;   // window origin (tile origins are even)
  for (int i = tid; i < K * K * Cin * CO; i += 256) {
    const int co = i % CO, r = i / CO, ci = r % Cin, tap = r / Cin;
    sW[i] = co < a.Cout ? bfv(a.W[tap * a.wst + ci * a.wsk + co * a.wsn]) : 0.f;
  }
  const __nv_bfloat16* in0 = (const __nv_bfloat16*)a.in0;
  const __nv_bfloat16* in1 = (const __nv_bfloat16*)a.in1;
  const size_t plane = (size_t)a.Hi * a.Wi;
  for (int i = tid; i < UW * UW * Cin; i += 256) {
    const int ci = i % Cin, p = i / Cin;        // channel fastest: coalesced reads along a pixel row
    const int r = p / UW, c = p - r * UW;
    const int gy = iy0 + r, gx = ix0 + c;
    float v = 0.f;
    if (gy >= 0 && gy < a.Hi && gx >= 0 && gx < a.Wi) {
      const size_t sp = ((size_t)b * a.Hi + gy) * a.Wi + gx;
      v = ci < a.c0 ? bfv(in0[sp * a.ld0 + ci])
                    : bfv(in1[(a.bcast1 ? sp % plane : sp) * a.ld1 + (ci - a.c0)]);
      if (a.in_act) v = elu_s(v);
    }
    sIn[((size_t)ci * UW + r) * UR + c] = v;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int ph = warp & 3, py = ph >> 1, px = ph & 1;
  const int idx = (warp >> 2) * 32 + lane;     // 0..63 within the phase's 8x8 grid
  const int qy = idx >> 3, qx = idx & 7;
  const int oy = oy0 + 2 * qy + py, ox = ox0 + 2 * qx + px;
  float acc[CO];
#pragma unroll
  for (int j = 0; j < CO; ++j) acc[j] = 0.f;
  // taps of this phase: (oy + pad - ky) even; local window row = qy + (py + pad - ky) / 2 + 1
  const int ky0 = (py + a.pad) & 1, kx0 = (px + a.pad) & 1;
#pragma unroll 1
  for (int ky = ky0; ky < K; ky += 2) {
    const int ly = qy + (py + a.pad - ky) / 2 + 1;
#pragma unroll 1
    for (int kx = kx0; kx < K; kx += 2) {
      const int lx = qx + (px + a.pad - kx) / 2 + 1;
      const float* ip = sIn + (size_t)ly * UR + lx;
      const float* wp = sW + (size_t)(ky * K + kx) * Cin * CO;
#pragma unroll 4
      for (int ci = 0; ci < Cin; ++ci) {
        const float v = ip[(size_t)ci * UW * UR];
#pragma unroll
        for (int j = 0; j < CO; ++j) acc[j] = fmaf(v, wp[ci * CO + j], acc[j]);
      }
    }
  }
  if (oy >= a.Ho || ox >= a.Wo) return;
  const size_t pix = ((size_t)b * a.Ho + oy) * a.Wo + ox;
#pragma unroll
  for (int j = 0; j < CO; ++j) {
    if (j >= a.Cout) break;
    float v = acc[j];
    if (a.bias) v += a.bias[j];
    if (a.res) v += bfv(a.res[pix * a.ldr + j]);
    if (a.ybf) {
      if (a.scale) v = v * a.scale[j] + a.shift[j];
      if (a.ep_act) v = elu_s(v);
      a.ybf[pix * a.ldy + j] = __float2bfloat16_rn(v);
    } else {
      a.out[pix * a.ldo + j] = v;
    }
  }
}

template <typename Kern>
bool launch_small(Kern kern, const ConvArgs& a, size_t smem, int tile_h, cudaStream_t s) {
  if (smem > 48 * 1024 && cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                              cudaSuccess)
    return false;
  const dim3 grid(((a.Wo + TS - 1) / TS) * ((a.Ho + tile_h - 1) / tile_h), a.B);
  kern<<<grid, 256, smem, s>>>(a);
  return true;
}

}  // namespace

bool conv_small_eligible(const ConvArgs& a) {
  if (a.in_f32 || a.k != 5 || a.stride != 2 || a.pad != 2) return false;
  if (!a.transposed) return !a.in1 && a.c0 <= 8 && a.Cout <= 32 && a.Ho * 2 <= a.Hi + 1 && a.Wo * 2 <= a.Wi + 1;
  // transposed: even output size 2 Hi x 2 Wi (tile origins even), few outputs.  Measured
  // slower than the TMA tensor-core path at 64 input channels (one shared-memory load
  // per two FMAs), so it serves only inputs the TMA path does not take.
  return a.Cout <= 4 && a.Ho == 2 * a.Hi && a.Wo == 2 * a.Wi && (a.c0 + (a.in1 ? a.c1 : 0)) <= 128 &&
         (a.ld0 % 8 || (a.in1 && a.ld1 % 8));
}

bool conv_forward_small(const ConvArgs& a, cudaStream_t s) {
  if (!conv_small_eligible(a)) return false;
  if (!a.transposed) {
    constexpr int IW = (TS - 1) * 2 + 5, IH = (DY - 1) * 2 + 5;
    if (a.c0 <= 4) {
      const size_t smem = sizeof(float) * ((size_t)IH * IW * 4 + 25 * 4 * 32);
      return launch_small(k_down_small<4, 32>, a, smem, DY, s);
    }
    const size_t smem = sizeof(float) * ((size_t)IH * IW * 8 + 25 * 8 * 32);
    return launch_small(k_down_small<8, 32>, a, smem, DY, s);
  }
  const int Cin = a.c0 + (a.in1 ? a.c1 : 0);
  ConvArgs b = a;
  if (!a.in1) b.c1 = 0;
  const size_t smem = sizeof(float) * ((size_t)Cin * UW * UR + (size_t)25 * Cin * (a.Cout <= 2 ? 2 : 4));
  if (a.Cout <= 2) return launch_small(k_up_small<2>, b, smem, TS, s);
  return launch_small(k_up_small<4>, b, smem, TS, s);
}

}  // namespace helm
