// Tensor-core implicit-GEMM convolution for sm_103a (5th-generation tensor
// cores: tcgen05.mma with the accumulator in tensor memory).
//
// One CTA computes a 128-pixel x Cout tile (Cout <= 256, a multiple of 16):
//   D[128][Cout] = sum over K-blocks of A[128][64] * B[64][Cout]
// A = im2col gather of the NHWC BF16 input (zero-filled padding), B = the
// K-major BF16 weights WT[cout][tap * Cin + ci].  Each K-block (64 BF16 = one
// 128-byte row) is staged with cp.async into shared memory in the canonical
// K-major 128-byte-swizzled layout (16-byte chunk c of row r stored at chunk
// c ^ (r % 8)), four pipeline stages; one thread issues four
// tcgen05.mma.kind::f16 (M = 128, K = 16 each) per K-block and commits them to
// the stage's mbarrier, which frees the stage for the next loads.  The
// epilogue reads the FP32 accumulator back with tcgen05.ld (warp w owns TMEM
// lanes 32w..32w+31 = tile rows) and applies bias / residual.
//
// Transposed stride-2 convolutions run per output phase (oy % 2, ox % 2): only
// the taps with matching parity contribute (9, 6, 6 or 4 of 25), so no MMA
// work is spent on structural zeros.
//
// Every mbarrier wait is bounded; on expiry the kernel records an error code,
// still waits (bounded) for its copies, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cstdint>

#include "devonce.cuh"
#include "unet_internal.cuh"

namespace helm {

namespace {

constexpr int TM = 128;           // pixels per tile (MMA M)
constexpr int TK = 64;            // K elements per stage (128 bytes of BF16)
constexpr int NSTAGE = 4;
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t a, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; returns false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(a, parity)) return true;
  return false;
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);        // start address
  d |= (uint64_t)1u << 16;                         // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024u >> 4) << 32;               // stride byte offset
  d |= (uint64_t)1u << 46;                         // descriptor version (tcgen05)
  d |= (uint64_t)2u << 61;                         // swizzle mode: 128 B
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

struct TcArgs {
  const __nv_bfloat16* in0; int c0, ld0;
  const __nv_bfloat16* in1; int c1, ld1; int bcast1;
  int B, Hi, Wi, Ho, Wo, Cout;
  int k, stride, pad, transposed;
  const __nv_bfloat16* WT; int ktot;     // [Cout][k*k*Cin]
  float* out; int ldo;
  const float* bias;
  const __nv_bfloat16* res; int ldr;
  const float* scale; const float* shift; int act;   // fused inference BatchNorm (+ eLU), or null
  __nv_bfloat16* ybf; int ldy;                         // BF16 destination of the fused epilogue
  int NT;                                              // output channels per CTA (blockIdx.y selects the chunk)
  int* err;
};

// Output pixel of tile row r (phase-aware for transposed convolutions).
__device__ __forceinline__ bool tile_pixel(const TcArgs& a, int m, int py, int px, int& b, int& oy, int& ox) {
  if (!a.transposed) {
    const int M = a.B * a.Ho * a.Wo;
    if (m >= M) return false;
    b = m / (a.Ho * a.Wo);
    const int r = m - b * a.Ho * a.Wo;
    oy = r / a.Wo;
    ox = r - oy * a.Wo;
    return true;
  }
  const int Hq = (a.Ho - py + 1) / 2, Wq = (a.Wo - px + 1) / 2;
  const int M = a.B * Hq * Wq;
  if (m >= M) return false;
  b = m / (Hq * Wq);
  const int r = m - b * Hq * Wq;
  const int qy = r / Wq;
  oy = 2 * qy + py;
  ox = 2 * (r - qy * Wq) + px;
  return true;
}

constexpr int NPROD = 128;        // producer / epilogue threads (warps 0-3)
constexpr int NTHREADS = NPROD + 32;  // + one MMA warp
constexpr int LAG = NSTAGE - 2;   // cp.async groups a producer keeps in flight before signalling

__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a) : "memory");
}

// Warp-specialised implicit-GEMM convolution: warps 0-3 gather A (one tile row =
// output pixel per thread) and B with cp.async into the stage buffers and arrive
// on full[s]; warp 4 waits on full[s], issues the MMAs and commits them to
// empty[s]; after the last K-block warps 0-3 drain the accumulator (epilogue).
__global__ void __launch_bounds__(NTHREADS, 1) k_conv_tc(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ int tab[1664];        // per 8-channel K chunk: ci | (dy + 128) << 16 | (dx + 128) << 24

  const int N = a.NT;
  const int n0 = blockIdx.y * a.NT;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Cin = a.c0 + a.c1;
  const int py = a.transposed ? (blockIdx.z >> 1) : 0, px = a.transposed ? (blockIdx.z & 1) : 0;
  int ky0 = 0, kx0 = 0, dk = 1;
  if (a.transposed) { ky0 = (py + a.pad) & 1; kx0 = (px + a.pad) & 1; dk = 2; }
  const int nty = (a.k - ky0 + dk - 1) / dk, ntx = (a.k - kx0 + dk - 1) / dk;
  const int ktot_phase = nty * ntx * Cin;
  const int nkb = (ktot_phase + TK - 1) / TK;
  const int nchunk = ktot_phase / 8;

  const uint32_t base = (smem_u32(smem) + 1023u) & ~1023u;
  const uint32_t a_bytes = TM * 128, b_bytes = (uint32_t)N * 128;
  const uint32_t stage_bytes = a_bytes + b_bytes;

  // tap table: input offset of each K chunk relative to the pixel's base coordinate
  for (int q = tid; q < nchunk; q += NTHREADS) {
    const int kidx = q * 8;
    const int t = kidx / Cin, ci = kidx - t * Cin;
    const int ty = t / ntx, tx = t - ty * ntx;
    const int ky = ky0 + dk * ty, kx = kx0 + dk * tx;
    int dy, dx;
    if (!a.transposed) { dy = ky - a.pad; dx = kx - a.pad; }
    else { dy = (py + a.pad - ky) / 2; dx = (px + a.pad - kx) / 2; }   // exact: parity matches
    tab[q] = ci | ((dy + 128) << 16) | ((dx + 128) << 24);
  }
  if (tid == 0) {
    for (int st = 0; st < NSTAGE; ++st) {
      mbar_init(smem_u32(&full[st]), NPROD);
      mbar_init(smem_u32(&empty[st]), 1);
    }
    mbar_init(smem_u32(&done), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const uint32_t ncols = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp < 4) {
    // ---------------- producers ----------------
    int pb = 0, poy = 0, pox = 0;
    const bool prow = tile_pixel(a, blockIdx.x * TM + tid, py, px, pb, poy, pox);
    const int by = a.transposed ? (poy - py) / 2 : poy * a.stride;   // base input coordinate
    const int bx = a.transposed ? (pox - px) / 2 : pox * a.stride;
    const size_t plane = (size_t)a.Hi * a.Wi;
    const size_t img = (size_t)pb * plane;
    bool ok = true;
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int st = kb % NSTAGE;
      const uint32_t use = (uint32_t)(kb / NSTAGE);
      if (kb >= NSTAGE && !mbar_wait(smem_u32(&empty[st]), (use - 1) & 1u)) { ok = false; break; }
      const uint32_t sA = base + (uint32_t)st * stage_bytes;
      const uint32_t sB = sA + a_bytes;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int q = kb * 8 + c;
        bool v = prow && q < nchunk;
        const void* src = a.in0;
        if (v) {
          const int e = tab[q];
          const int ci = e & 0xFFFF, iy = by + ((e >> 16) & 0xFF) - 128, ix = bx + ((e >> 24) & 0xFF) - 128;
          v = iy >= 0 && iy < a.Hi && ix >= 0 && ix < a.Wi;
          if (v) {
            const size_t sp = img + (size_t)iy * a.Wi + ix;
            src = ci < a.c0 ? (const void*)(a.in0 + sp * a.ld0 + ci)
                            : (const void*)(a.in1 + (a.bcast1 ? sp % plane : sp) * a.ld1 + (ci - a.c0));
          }
        }
        cp_async16(sA + (uint32_t)tid * 128u + (uint32_t)((c ^ (tid & 7)) << 4), src, v);
      }
      for (int co = tid; co < N; co += NPROD) {
        const bool rowv = n0 + co < a.Cout;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int q = kb * 8 + c;
          bool v = rowv && q < nchunk;
          const void* src = a.WT;
          if (v) {   // tap from the table entry: ky = dy + pad (conv) or py + pad - 2 dy (transposed)
            const int e = tab[q];
            const int ci = e & 0xFFFF, dy = ((e >> 16) & 0xFF) - 128, dx = ((e >> 24) & 0xFF) - 128;
            const int ky = a.transposed ? py + a.pad - 2 * dy : dy + a.pad;
            const int kx = a.transposed ? px + a.pad - 2 * dx : dx + a.pad;
            src = a.WT + (size_t)(n0 + co) * a.ktot + (size_t)(ky * a.k + kx) * Cin + ci;
          }
          cp_async16(sB + (uint32_t)co * 128u + (uint32_t)((c ^ (co & 7)) << 4), src, v);
        }
      }
      cp_async_commit();
      if (kb >= LAG) {
        cp_async_wait<LAG>();
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive(smem_u32(&full[(kb - LAG) % NSTAGE]));
      }
    }
    cp_async_wait<0>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    if (ok) {
      for (int kb = nkb > LAG ? nkb - LAG : 0; kb < nkb; ++kb) mbar_arrive(smem_u32(&full[kb % NSTAGE]));
    } else {
      atomicExch(&s_fail, 1);
    }
    // ---------------- epilogue ----------------
    const bool fin = mbar_wait(smem_u32(&done), 0);
    if (!fin) atomicExch(&s_fail, 1);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (fin && ok) {
      int b = 0, oy = 0, ox = 0;
      const bool rv = tile_pixel(a, blockIdx.x * TM + tid, py, px, b, oy, ox);
      const size_t pix = ((size_t)b * a.Ho + oy) * a.Wo + ox;
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
  } else if (tid == NPROD) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = idesc_bf16(N);
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      const int st = kb % NSTAGE;
      const uint32_t use = (uint32_t)(kb / NSTAGE);
      if (!mbar_wait(smem_u32(&full[st]), use & 1u)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t sA = base + (uint32_t)st * stage_bytes;
      const uint64_t da = sw128_desc(sA), db = sw128_desc(sA + a_bytes);
#pragma unroll
      for (int k4 = 0; k4 < TK / 16; ++k4) {
        const uint32_t acc = (kb > 0 || k4 > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da + (uint64_t)(2 * k4)), "l"(db + (uint64_t)(2 * k4)), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&empty[st]))
                   : "memory");
    }
    if (!ok) atomicExch(&s_fail, 1);
    // `done` completes when every MMA issued above has retired
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(&done))
                 : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_fail && a.err) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

}  // namespace

bool conv_tc_eligible(const ConvArgs& a) {
  if (a.in_f32 || a.in_act || !a.WT) return false;
  if (a.c0 % 8 || a.c1 % 8 || a.ld0 % 8 || (a.in1 && a.ld1 % 8)) return false;
  if (a.Cout < 1 || a.Cout > 256) return false;
  if (a.transposed && a.stride != 2) return false;
  if ((long long)a.k * a.k * (a.c0 + (a.in1 ? a.c1 : 0)) / 8 > 1664) return false;   // tap-table capacity
  return true;
}

size_t conv_tc_smem(int nt) { return (size_t)NSTAGE * (TM * 128 + (size_t)nt * 128) + 1024; }

void conv_forward_tc(const ConvArgs& c, int* err, cudaStream_t s) {
  TcArgs a;
  a.in0 = (const __nv_bfloat16*)c.in0; a.c0 = c.c0; a.ld0 = c.ld0;
  a.in1 = (const __nv_bfloat16*)c.in1; a.c1 = c.in1 ? c.c1 : 0; a.ld1 = c.ld1; a.bcast1 = c.bcast1;
  a.B = c.B; a.Hi = c.Hi; a.Wi = c.Wi; a.Ho = c.Ho; a.Wo = c.Wo; a.Cout = c.Cout;
  a.k = c.k; a.stride = c.stride; a.pad = c.pad; a.transposed = c.transposed;
  a.WT = c.WT; a.ktot = c.k * c.k * (c.c0 + (c.in1 ? c.c1 : 0));
  a.out = c.out; a.ldo = c.ldo; a.bias = c.bias; a.res = c.res; a.ldr = c.ldr;
  a.scale = c.scale; a.shift = c.shift; a.act = c.ep_act; a.ybf = c.ybf; a.ldy = c.ldy;
  a.err = err;
  // one output-channel tile of the full width (rounded up to the MMA's 16)
  const int M = c.transposed ? c.B * ((c.Ho + 1) / 2) * ((c.Wo + 1) / 2) : c.B * c.Ho * c.Wo;
  const int nt = ((c.Cout + 15) / 16) * 16;
  a.NT = nt;
  const int nchunk = (c.Cout + nt - 1) / nt;
  const size_t smem = conv_tc_smem(nt);
  static DeviceOnce once;   // the opt-in is a per-device kernel attribute
  set_dynamic_smem(once, k_conv_tc, (int)conv_tc_smem(256));
  if (!c.transposed) {
    k_conv_tc<<<dim3((M + TM - 1) / TM, nchunk, 1), NTHREADS, smem, s>>>(a);
  } else {
    k_conv_tc<<<dim3((M + TM - 1) / TM, nchunk, 4), NTHREADS, smem, s>>>(a);
  }
}

}  // namespace helm
