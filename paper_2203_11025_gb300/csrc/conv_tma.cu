// Tensor-core implicit-GEMM convolution fed by TMA (sm_103a).
//
// A CTA computes a tile of 128 output pixels (a BX x BY x BB box of one or more
// images; for transposed stride-2 convolutions a box of one output phase) times
// Cout (<= 256, rounded up to 16).  The reduction runs over K-blocks = (tap,
// 64-channel chunk of one input source); for each K-block one TMA load brings
// the input box at the tap's offset -- element stride 2 for stride-2
// convolutions, zero fill outside the image (the convolution's padding) -- in
// the 128-byte-swizzled K-major layout the MMA reads, and one TMA load brings
// the matching weight tile from a padded K-major copy [cout][tap][chunks*64].
// Warp 4 issues the TMA loads (mbarrier expect_tx), warp 5 issues
// tcgen05.mma (M = 128, K = 16 x 4 per block) and commits each stage back to
// the producer; warps 0-3 read the FP32 accumulator from tensor memory and
// apply bias / residual / BatchNorm / eLU.  All waits are bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "unet_internal.cuh"

namespace helm {

namespace {

constexpr int TM = 128;
constexpr int TK = 64;
constexpr int NST = 4;
constexpr int NTHR = 192;          // warps 0-3 epilogue, 4 TMA, 5 MMA
constexpr long long kWait = 1ll << 24;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint32_t a, int c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(c) : "memory");
}
__device__ __forceinline__ bool mb_try(uint32_t a, uint32_t par) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(a), "r"(par)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint32_t a, uint32_t par) {
  for (long long i = 0; i < kWait; ++i)
    if (mb_try(a, par)) return true;
  return false;
}
__device__ __forceinline__ void mb_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ uint64_t desc128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

struct TmaArgs {
  int B, Ho, Wo, Cout, NT;
  int k, stride, pad, transposed;
  int BX, BY, BB;                 // output tile (pixels of the output or phase grid)
  int tx, ty;                     // tiles along x and y
  int nch0, nch1;                 // 64-channel chunks per source
  int bcast1;                     // source 1 is one image shared by the batch
  int kpad;                       // padded K per tap = 64 (nch0 + nch1)
  float* out; int ldo;
  const float* bias;
  const __nv_bfloat16* res; int ldr;
  const float* scale; const float* shift; int act;
  __nv_bfloat16* ybf; int ldy;
  int* err;
};

__global__ void __launch_bounds__(NTHR, 1) k_conv_tma(const __grid_constant__ CUtensorMap mA0,
                                                      const __grid_constant__ CUtensorMap mA1,
                                                      const __grid_constant__ CUtensorMap mB, TmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[NST], empty[NST], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = a.NT, n0 = blockIdx.y * a.NT;
  const int py = a.transposed ? (blockIdx.z >> 1) : 0, px = a.transposed ? (blockIdx.z & 1) : 0;
  int ky0 = 0, kx0 = 0, dk = 1;
  if (a.transposed) { ky0 = (py + a.pad) & 1; kx0 = (px + a.pad) & 1; dk = 2; }
  const int nty = (a.k - ky0 + dk - 1) / dk, ntx = (a.k - kx0 + dk - 1) / dk;
  const int nchk = a.nch0 + a.nch1;
  const int nkb = nty * ntx * nchk;
  // tile origin in the output (or phase) grid
  int t = blockIdx.x;
  const int tix = t % a.tx; t /= a.tx;
  const int tiy = t % a.ty; t /= a.ty;
  const int x0 = tix * a.BX, y0 = tiy * a.BY, b0 = t * a.BB;

  const uint32_t base = (su32(smem) + 1023u) & ~1023u;
  const uint32_t a_bytes = TM * 128, b_bytes = (uint32_t)N * 128, stage = a_bytes + b_bytes;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) { mb_init(su32(&full[s]), 1); mb_init(su32(&empty[s]), 1); }
    mb_init(su32(&done), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 4) {
    if ((tid & 31) == 0) {
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NST;
        const uint32_t use = (uint32_t)(kb / NST);
        if (kb >= NST && !mb_wait(su32(&empty[s]), (use - 1) & 1u)) { ok = false; break; }
        const int tap = kb / nchk, ch = kb - tap * nchk;
        const int ty = tap / ntx, tx = tap - ty * ntx;
        const int ky = ky0 + dk * ty, kx = kx0 + dk * tx;
        int ix, iy;
        if (!a.transposed) { ix = x0 * a.stride + kx - a.pad; iy = y0 * a.stride + ky - a.pad; }
        else { ix = x0 + (px + a.pad - kx) / 2; iy = y0 + (py + a.pad - ky) / 2; }
        const uint32_t sA = base + (uint32_t)s * stage, sB = sA + a_bytes;
        mb_expect_tx(su32(&full[s]), stage);
        if (ch < a.nch0) tma_load_4d(sA, &mA0, ch * TK, ix, iy, b0, su32(&full[s]));
        else tma_load_4d(sA, &mA1, (ch - a.nch0) * TK, ix, iy, a.bcast1 ? 0 : b0, su32(&full[s]));
        tma_load_2d(sB, &mB, (ky * a.k + kx) * a.kpad + ch * TK, n0, su32(&full[s]));
      }
      if (!ok) atomicExch(&s_fail, 1);
    }
  } else if (warp == 5) {
    if ((tid & 31) == 0) {
      const uint32_t id = idesc(N);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % NST;
        if (!mb_wait(su32(&full[s]), (uint32_t)(kb / NST) & 1u)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t sA = base + (uint32_t)s * stage;
        const uint64_t da = desc128(sA), db = desc128(sA + a_bytes);
#pragma unroll
        for (int k4 = 0; k4 < TK / 16; ++k4) {
          const uint32_t acc = (kb > 0 || k4 > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(da + (uint64_t)(2 * k4)), "l"(db + (uint64_t)(2 * k4)), "r"(id), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         su32(&empty[s]))
                     : "memory");
      }
      if (!ok) atomicExch(&s_fail, 1);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&done))
                   : "memory");
    }
  } else {
    // epilogue: warps 0-3, tile row = tid
    const bool fin = mb_wait(su32(&done), 0);
    if (!fin) atomicExch(&s_fail, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int m = tid;
    const int bb = m / (a.BY * a.BX), rr = m - bb * a.BY * a.BX, by = rr / a.BX, bx = rr - by * a.BX;
    const int b = b0 + bb, qy = y0 + by, qx = x0 + bx;
    const int oy = a.transposed ? 2 * qy + py : qy, ox = a.transposed ? 2 * qx + px : qx;
    const bool rv = fin && b < a.B && oy < a.Ho && ox < a.Wo;
    const size_t pix = ((size_t)b * a.Ho + oy) * a.Wo + ox;
    if (fin) {
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (rv) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int co = n0 + c0 + j;
            if (co >= a.Cout) break;
            float f = __uint_as_float(v[j]);
            if (a.bias) f += a.bias[co];
            if (a.res) f += __bfloat162float(a.res[pix * a.ldr + co]);
            if (a.ybf) {
              if (a.scale) f = f * a.scale[co] + a.shift[co];
              if (a.act) f = f > 0.f ? f : expm1f(f);
              a.ybf[pix * a.ldy + co] = __float2bfloat16_rn(f);
            } else {
              a.out[pix * a.ldo + co] = f;
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_fail && a.err) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

bool get_encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  return g_encode != nullptr;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// 4-D map over an NHWC BF16 source slice: (channels, x, y, image), box (64, BX*s, BY*s, BB).
bool encode_act(CUtensorMap* m, const void* ptr, int C, int ld, int W, int H, int B, int BX, int BY, int BB, int es) {
  if (((uintptr_t)ptr & 15) || (ld * 2) % 16) return false;
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * W, (cuuint64_t)ld * 2 * W * H};
  cuuint32_t box[4] = {64, (cuuint32_t)(BX * es), (cuuint32_t)(BY * es), (cuuint32_t)BB};
  cuuint32_t estr[4] = {1, (cuuint32_t)es, (cuuint32_t)es, 1};
  if (box[1] > 256 || box[2] > 256) return false;
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_w(CUtensorMap* m, const void* ptr, int K, int cout, int NT) {
  if (((uintptr_t)ptr & 15) || (K * 2) % 16) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)cout};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)NT};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

__global__ void k_weights_padded(const float* __restrict__ P, __nv_bfloat16* __restrict__ WP, int taps, int c0, int c1,
                                 int cout, int kpad, int off1) {
  const size_t n = (size_t)cout * taps * kpad;
  const int cin = c0 + c1;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % kpad);
    const size_t r = i / kpad;
    const int tap = (int)(r % taps), co = (int)(r / taps);
    int ci = -1;
    if (k < c0) ci = k;
    else if (k >= off1 && k < off1 + c1) ci = c0 + (k - off1);
    WP[i] = __float2bfloat16_rn(ci >= 0 ? P[((size_t)tap * cin + ci) * cout + co] : 0.f);
  }
}

}  // namespace

size_t conv_tma_weight_elems(int k, int c0, int c1, int cout) {
  const int kpad = 64 * ((c0 + 63) / 64 + (c1 + 63) / 64);
  return (size_t)cout * k * k * kpad;
}

void conv_tma_weights(const float* P, __nv_bfloat16* WP, int k, int c0, int c1, int cout, cudaStream_t s) {
  const int nch0 = (c0 + 63) / 64;
  const int kpad = 64 * (nch0 + (c1 + 63) / 64);
  const size_t n = (size_t)cout * k * k * kpad;
  k_weights_padded<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(P, WP, k * k, c0, c1, cout, kpad,
                                                                                     64 * nch0);
}

// Launch if the convolution fits the TMA path; false otherwise (caller falls back).
bool conv_forward_tma(const ConvArgs& c, int* err, cudaStream_t s) {
  if (!c.WP || c.in_f32 || c.in_act || c.Cout > 256) return false;
  if (c.transposed && c.stride != 2) return false;
  if (!c.transposed && c.stride != 1 && c.stride != 2) return false;
  if (c.c0 % 8 || (c.in1 && c.c1 % 8)) return false;
  if (!get_encoder()) return false;
  const int Wq = c.transposed ? c.Wo / 2 : c.Wo, Hq = c.transposed ? c.Ho / 2 : c.Ho;
  if (!pow2(Wq) || !pow2(Hq) || (c.transposed && (c.Wo % 2 || c.Ho % 2))) return false;
  const int BX = Wq < 128 ? Wq : 128;
  const int BY = Hq < 128 / BX ? Hq : 128 / BX;
  const int BB = 128 / (BX * BY);
  if (c.in1 && c.bcast1 && BB > 1) return false;
  const int es = c.transposed ? 1 : c.stride;
  CUtensorMap mA0, mA1, mB;
  if (!encode_act(&mA0, c.in0, c.c0, c.ld0, c.Wi, c.Hi, c.B, BX, BY, BB, es)) return false;
  if (c.in1) {
    if (!encode_act(&mA1, c.in1, c.c1, c.ld1, c.Wi, c.Hi, c.bcast1 ? 1 : c.B, BX, BY, BB, es)) return false;
  } else {
    mA1 = mA0;
  }
  TmaArgs a;
  a.B = c.B; a.Ho = c.Ho; a.Wo = c.Wo; a.Cout = c.Cout;
  a.NT = ((c.Cout + 15) / 16) * 16;
  a.k = c.k; a.stride = c.stride; a.pad = c.pad; a.transposed = c.transposed;
  a.BX = BX; a.BY = BY; a.BB = BB;
  a.tx = Wq / BX; a.ty = Hq / BY;
  a.nch0 = (c.c0 + 63) / 64;
  a.nch1 = c.in1 ? (c.c1 + 63) / 64 : 0;
  a.bcast1 = (c.in1 && c.bcast1) ? 1 : 0;
  a.kpad = 64 * (a.nch0 + a.nch1);
  if (!encode_w(&mB, c.WP, c.k * c.k * a.kpad, c.Cout, a.NT)) return false;
  a.out = c.out; a.ldo = c.ldo; a.bias = c.bias; a.res = c.res; a.ldr = c.ldr;
  a.scale = c.scale; a.shift = c.shift; a.act = c.ep_act; a.ybf = c.ybf; a.ldy = c.ldy;
  a.err = err;
  const size_t smem = (size_t)NST * (TM * 128 + (size_t)a.NT * 128) + 1024;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_conv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, NST * (TM * 128 + 256 * 128) + 1024);
    configured = true;
  }
  const int tb = (c.B + BB - 1) / BB;
  k_conv_tma<<<dim3(a.tx * a.ty * tb, 1, c.transposed ? 4 : 1), NTHR, smem, s>>>(mA0, mA1, mB, a);
  return true;
}

}  // namespace helm
