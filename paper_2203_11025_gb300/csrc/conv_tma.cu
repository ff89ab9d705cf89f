// Tensor-core implicit-GEMM convolution fed by TMA (sm_103a).
//
// Work item: a tile of 128 output pixels (a BX x BY x BB box of one or more
// images; for transposed stride-2 convolutions a box of one output phase) times
// Cout (<= 256, rounded up to 16), reduced over one range of K-blocks = (tap,
// 64-channel chunk of one input source).  For each K-block one TMA load brings
// the input box at the tap's offset -- element stride 2 for stride-2
// convolutions, zero fill outside the image (the convolution's padding) and
// past the real channels -- in the 128-byte-swizzled K-major layout the MMA
// reads, and one TMA load brings the matching weight tile from a padded K-major
// copy [cout][tap][chunks*64].
//
// The kernel is persistent (one or two CTAs per SM, items strided by the grid).
// Warp 4 issues the TMA loads into a ring of 4-8 stages (mbarrier expect_tx)
// without stopping at item boundaries; warp 5 issues tcgen05.mma (M = 128,
// K = 16 x 4 per block) into one of two TMEM accumulators and commits each
// stage back to the producer; warps 0-3 read the finished accumulator and
// apply bias / residual / BatchNorm / eLU while the next item accumulates in
// the other buffer.  Convolutions with too few tiles to fill the GPU split K
// across items: each split stores its partial tile to its own FP32 slice and a
// second kernel adds the slices and applies the epilogue.  Eight epilogue warps
// (two column groups per TMEM lane quadrant) take per-channel constants from
// shared memory.  All waits are bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <functional>
#include <mutex>
#include <unordered_map>
#include <utility>

#include "devonce.cuh"
#include "fdiv.h"
#include "pdl.cuh"
#include "unet_internal.cuh"

namespace helm {

namespace {

constexpr int TM = 128;
constexpr bool kSplitFixupInKernel = false;
constexpr int MAXST = 12;          // stage ring capacity (the host picks nst <= MAXST)
constexpr int NEPI = 8;                  // epilogue warps: 2 groups (alternate tiles) x 4 TMEM lane quadrants
constexpr int NACC = 4;                  // TMEM accumulator buffers at most (the host picks nacc <= NACC)
constexpr int WPROD = NEPI, WMMA = NEPI + 1;
constexpr int NTHR = 32 * (NEPI + 2);    // + the TMA producer warp and the MMA warp
constexpr long long kWait = 1ll << 24;       // try_wait rounds before a wait gives up (seconds at most)
constexpr long long kWaitSleep = 1ll << 23;  // sleeping polls before an epilogue wait gives up (~1 s)

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint32_t a, int c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(a), "r"(c) : "memory");
}
__device__ __forceinline__ bool mb_test(uint32_t a, uint32_t par) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(a), "r"(par)
               : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mb_try(uint32_t a, uint32_t par) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(a), "r"(par)
               : "memory");
  return ok != 0;
}
// Critical-path waits (TMA producer, MMA issuer): try_wait suspends the thread in
// hardware until the phase completes, so a waiting warp takes no issue slots.
__device__ __forceinline__ bool mb_wait(uint32_t a, uint32_t par, long long bound = kWait) {
  for (long long i = 0; i < bound; ++i)
    if (mb_try(a, par)) return true;
  return false;
}
// Epilogue waits (an item's whole MMA time): poll with a sleep in between, so that
// the epilogue warps leave the issue slots to the producer and MMA threads.
__device__ __forceinline__ bool mb_wait_sleep(uint32_t a, uint32_t par) {
  for (long long i = 0; i < kWaitSleep; ++i) {
    if (mb_test(a, par)) return true;
    __nanosleep(128);
  }
  return false;
}
__device__ __forceinline__ void mb_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a), "r"(bytes)
               : "memory");
}
// Failure-detection probe: one thread waits, through the pipeline's bounded wait, on an
// mbarrier that expects one arrival.  With arrive = 0 nothing arrives, the wait gives up
// after `rounds` polls and the failure is recorded in err exactly as the convolution
// kernels record an expired wait; with arrive = 1 the thread arrives first and the wait
// succeeds.  Either way the kernel returns.
__global__ void k_wait_probe(int* err, long long rounds, int arrive) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t a = su32(&bar);
  mb_init(a, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  if (arrive) asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(a) : "memory");
  if (!mb_wait(a, 0, rounds) && err) atomicExch(err, 1);
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
// Shared-memory descriptor of a K-major operand whose rows (one pixel or one output
// column) hold tk = 16, 32 or 64 BF16 channels: rows of 32, 64 or 128 bytes written by
// TMA with the matching swizzle, 8-row groups 8 rows apart (stride byte offset), layout
// type SWIZZLE_32B (6), SWIZZLE_64B (4) or SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t desc_k(uint32_t saddr, int tk) {
  const uint32_t row = 2u * (uint32_t)tk;
  const uint64_t lay = tk == 64 ? 2u : (tk == 32 ? 4u : 6u);
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)((8u * row) >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= lay << 61;
  return d;
}
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// One tcgen05.mma (M = 128, kind::f16, D in TMEM at d) of K-step descriptors da, db;
// accumulate: add into D (else overwrite it).
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t da, uint64_t db, uint32_t id, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(da), "l"(db), "r"(id), "r"(accumulate)
      : "memory");
}

// The MMAs of one stage as straight-line code (a single thread issues an MMA in far fewer
// cycles when no branch separates it from the previous one): NJ taps x NK4 K-steps of 16,
// tap j reading A at a0 + j * astep and B at w0 + j * wstep (byte offsets may be negative
// as unsigned wrap-around).  acc0: the first MMA accumulates (else it starts D).
template <int NJ, int NK4>
__device__ __forceinline__ void mma_taps(uint32_t d, uint32_t a0, uint32_t astep, uint32_t w0, uint32_t wstep, int tk,
                                         uint32_t id, uint32_t acc0) {
#pragma unroll
  for (int j = 0; j < NJ; ++j) {
    const uint64_t da = desc_k(a0 + (uint32_t)j * astep, tk), db = desc_k(w0 + (uint32_t)j * wstep, tk);
#pragma unroll
    for (int k4 = 0; k4 < NK4; ++k4)
      mma_f16(d, da + (uint64_t)(2 * k4), db + (uint64_t)(2 * k4), id, (j == 0 && k4 == 0) ? acc0 : 1u);
  }
}
template <int NJ>
__device__ __forceinline__ void mma_taps_k(int nk4, uint32_t d, uint32_t a0, uint32_t astep, uint32_t w0,
                                           uint32_t wstep, int tk, uint32_t id, uint32_t acc0) {
  switch (nk4) {
    case 1: mma_taps<NJ, 1>(d, a0, astep, w0, wstep, tk, id, acc0); break;
    case 2: mma_taps<NJ, 2>(d, a0, astep, w0, wstep, tk, id, acc0); break;
    case 3: mma_taps<NJ, 3>(d, a0, astep, w0, wstep, tk, id, acc0); break;
    default: mma_taps<NJ, 4>(d, a0, astep, w0, wstep, tk, id, acc0); break;
  }
}

// NB consecutive K-blocks of a stage (K-block b's A and B kstep bytes after K-block b - 1's),
// NK4 K-steps each, as straight-line code.
template <int NB, int NK4>
__device__ __forceinline__ void mma_kblocks(uint32_t d, uint32_t a0, uint32_t b0, uint32_t kstep, int tk, uint32_t id,
                                            uint32_t acc0) {
#pragma unroll
  for (int b = 0; b < NB; ++b)
    mma_taps<1, NK4>(d, a0 + (uint32_t)b * kstep, 0u, b0 + (uint32_t)b * kstep, 0u, tk, id, b == 0 ? acc0 : 1u);
}
__device__ __forceinline__ void mma_kblocks_n(int nb, int nk4, uint32_t d, uint32_t a0, uint32_t b0, uint32_t kstep,
                                              int tk, uint32_t id, uint32_t acc0) {
#define HELM_KB(NB, NK)                                                          \
  if (nb == (NB) && nk4 == (NK)) { mma_kblocks<NB, NK>(d, a0, b0, kstep, tk, id, acc0); return; }
  HELM_KB(2, 4) HELM_KB(3, 4) HELM_KB(2, 2) HELM_KB(3, 2)
#undef HELM_KB
  for (int b = 0; b < nb; ++b)
    mma_taps_k<1>(nk4, d, a0 + (uint32_t)b * kstep, 0u, b0 + (uint32_t)b * kstep, 0u, tk, id, b == 0 ? acc0 : 1u);
}

// Low and high words of desc_k: the high word depends only on tk, the low word holds the
// shared-memory address (16-byte units), so taps and K-steps step the low word alone.
__device__ __forceinline__ uint32_t desc_lo(uint32_t saddr) { return ((saddr >> 4) & 0x3FFFu) | (1u << 16); }
__device__ __forceinline__ uint32_t desc_hi(int tk) {
  const uint32_t lay = tk == 64 ? 2u : (tk == 32 ? 4u : 6u);
  return ((8u * 2u * (uint32_t)tk) >> 4) | (1u << 14) | (lay << 29);
}
__device__ __forceinline__ void mma_lo(uint32_t d, uint32_t alo, uint32_t blo, uint32_t hi, uint32_t id,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b64 da, db;\n setp.ne.b32 p, %5, 0;\n mov.b64 da, {%1, %3};\n"
      " mov.b64 db, {%2, %3};\n tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %4, p;\n}\n" ::"r"(d),
      "r"(alo), "r"(blo), "r"(hi), "r"(id), "r"(accumulate)
      : "memory");
}
// NX boxes x NJ taps x NK4 K-steps from low descriptor words: box x, tap j, step k reads A at
// alo + x * xs + j * as + 2 k and B at blo + x * wxs + j * ws + 2 k (steps in 16-byte units,
// two's complement for negative ones).
template <int NX, int NJ, int NK4>
__device__ __forceinline__ void mma_lo_boxes(uint32_t d, uint32_t alo, uint32_t as, uint32_t xs, uint32_t blo,
                                             uint32_t ws, uint32_t wxs, uint32_t hi, uint32_t id, uint32_t acc0) {
#pragma unroll
  for (int x = 0; x < NX; ++x)
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
      for (int k = 0; k < NK4; ++k)
        mma_lo(d, alo + (uint32_t)x * xs + (uint32_t)j * as + 2u * k,
               blo + (uint32_t)x * wxs + (uint32_t)j * ws + 2u * k, hi, id, (x == 0 && j == 0 && k == 0) ? acc0 : 1u);
}
// Shape code of a stage: nx | nj << 4 | nk4 << 8.  Instantiated shapes issue as one block.
__device__ __forceinline__ bool mma_lo_shape(uint32_t shape, uint32_t d, uint32_t alo, uint32_t as, uint32_t xs,
                                             uint32_t blo, uint32_t ws, uint32_t wxs, uint32_t hi, uint32_t id,
                                             uint32_t acc0) {
#define HELM_SHAPE(NX, NJ, NK)                                            \
  case (NX) | ((NJ) << 4) | ((NK) << 8):                                  \
    mma_lo_boxes<NX, NJ, NK>(d, alo, as, xs, blo, ws, wxs, hi, id, acc0); \
    return true;
  switch (shape) {
    HELM_SHAPE(3, 3, 1) HELM_SHAPE(3, 3, 2) HELM_SHAPE(3, 3, 4)   // 3x3 stride 1
    HELM_SHAPE(5, 3, 1) HELM_SHAPE(5, 3, 2) HELM_SHAPE(5, 3, 4)   // 5x5 stride 2, even rows
    HELM_SHAPE(5, 2, 1) HELM_SHAPE(5, 2, 2) HELM_SHAPE(5, 2, 4)   // 5x5 stride 2, odd rows
    HELM_SHAPE(3, 2, 1) HELM_SHAPE(3, 2, 2) HELM_SHAPE(3, 2, 4)   // transposed phases
    HELM_SHAPE(2, 3, 1) HELM_SHAPE(2, 3, 2) HELM_SHAPE(2, 3, 4)
    HELM_SHAPE(2, 2, 1) HELM_SHAPE(2, 2, 2) HELM_SHAPE(2, 2, 4)
    HELM_SHAPE(1, 3, 1) HELM_SHAPE(1, 3, 2) HELM_SHAPE(1, 3, 4)   // one box per stage
    HELM_SHAPE(1, 2, 1) HELM_SHAPE(1, 2, 2) HELM_SHAPE(1, 2, 4)
    default: return false;
  }
#undef HELM_SHAPE
}

struct TmaArgs {
  int B, Ho, Wo, Cout, NT;
  int k, stride, pad, transposed;
  int BX, BY, BB;                 // output tile (pixels of the output or phase grid)
  int tx, ty, tb;                 // tiles along x, y and images
  int nch0, nch1;                 // tk-channel chunks per source
  int c0, c1;                     // real channels per source (MMAs skip the zero-filled K)
  int shuf, cr;                   // sub-pixel output: column n = phase * cr + channel, pixel (2y + py, 2x + px)
  int bcast1;                     // source 1 is one image shared by the batch
  int ksplit;                     // K-block ranges per tile; > 1: FP32 atomic accumulation
  int nitems;                     // tiles x phases x ksplit
  int nst;                        // pipeline stages (<= MAXST)
  int colsz;                      // TMEM columns of one accumulator (power of two >= 32)
  int vec;                        // every row pointer of out / ybf / res / part is 16-byte aligned
  int kpad;                       // padded K per tap = tk (nch0 + nch1)
  int tk;                         // channels per K-chunk (stage row): 16, 32 or 64
  int nacc;                       // TMEM accumulator buffers (2 or 4; item i uses buffer i % nacc)
  int kps;                        // general kernel: K-blocks per stage (> 1 only when every chunk is full)
  int epig;                       // epilogue: 1 = warp groups on alternate items, 0 = on alternate columns
  float* out; int ldo;
  const float* bias;
  const __nv_bfloat16* res; int ldr;
  const float* scale; const float* shift; int act;
  __nv_bfloat16* ybf; int ldy;
  __nv_bfloat16* y2; int ldy2;    // optional: eLU of the BF16 result as well (next layer's activated input)
  // split-K: split s stores its partial sums to part + s * slice ([pixels][Cout], FP32);
  // the last split of a tile to finish (ticket cnt[tile]) adds the slices and applies the
  // epilogue, and puts the ticket back to 0 (cnt null: k_splitk_finish does it instead)
  float* part; size_t slice;
  int* cnt;
  int* err;
  FDiv f_tile, f_tx, f_ty, f_ks;  // tx * ty * tb, tx, ty, ksplit
  FDiv f_ns;                      // nst (stage ring position and phase of K-block g)
  int lg_nacc;                    // log2(nacc)
};

// The divisors decode() uses, from the filled-in tile counts.
void set_fdivs(TmaArgs& a) {
  a.f_tile = make_fdiv((uint32_t)(a.tx * a.ty * a.tb));
  a.f_tx = make_fdiv((uint32_t)a.tx);
  a.f_ty = make_fdiv((uint32_t)a.ty);
  a.f_ks = make_fdiv((uint32_t)a.ksplit);
  a.f_ns = make_fdiv((uint32_t)a.nst);
  a.lg_nacc = a.nacc == 4 ? 2 : (a.nacc == 2 ? 1 : 0);
}

// eLU for BF16 results: exp(x) - 1 with the fast exponential (absolute error ~1e-7,
// far below the BF16 rounding of the stored value; expm1f made the epilogue issue-bound).
__device__ __forceinline__ float elu_bf(float x) { return x > 0.f ? x : __expf(x) - 1.f; }

// One work item: an output tile of one phase, reduced over one K range.
struct Item {
  int x0, y0, b0, py, px, ky0, kx0, dk, ntx, nchk, kbeg, nkb, split;
};

__device__ __forceinline__ Item decode(const TmaArgs& a, int w) {
  const int r = fdiv(a.f_tile, w);
  int t = w - r * (int)a.f_tile.d;
  const int z = a.transposed ? (r & 3) : 0, ys = a.transposed ? (r >> 2) : r;
  Item it;
  it.py = a.transposed ? (z >> 1) : 0;
  it.px = a.transposed ? (z & 1) : 0;
  it.ky0 = 0; it.kx0 = 0; it.dk = 1;
  if (a.transposed) { it.ky0 = (it.py + a.pad) & 1; it.kx0 = (it.px + a.pad) & 1; it.dk = 2; }
  const int nty = (a.k - it.ky0 + it.dk - 1) / it.dk;
  it.ntx = (a.k - it.kx0 + it.dk - 1) / it.dk;
  it.nchk = a.nch0 + a.nch1;
  const int nkb_all = nty * it.ntx * it.nchk;
  // balanced K ranges; the host keeps ksplit <= nkb_all, so nkb >= 1
  it.kbeg = fdiv(a.f_ks, ys * nkb_all);
  it.nkb = fdiv(a.f_ks, (ys + 1) * nkb_all) - it.kbeg;
  it.split = ys;
  const int t1 = fdiv(a.f_tx, t), tix = t - t1 * a.tx;
  t = t1;
  const int t2 = fdiv(a.f_ty, t), tiy = t - t2 * a.ty;
  t = t2;
  it.x0 = tix * a.BX; it.y0 = tiy * a.BY; it.b0 = t * a.BB;
  return it;
}

__device__ __forceinline__ bool failed(const volatile int* f) { return *f != 0; }

// OR of a predicate over the epilogue warps that share an item: all 8 (named barrier 1),
// or with alt the 4 of group g (named barrier 1 + g).  A uniform decision among them.
__device__ __forceinline__ bool epi_any(bool p, int g, bool alt) {
  uint32_t r;
  if (!alt)
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "n"(NEPI * 32)
        : "memory");
  else if (g == 0)
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "n"(NEPI / 2 * 32)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 2, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)p), "n"(NEPI / 2 * 32)
        : "memory");
  return r != 0;
}

// Per-column epilogue constants: with BatchNorm (BF16 results) y = (acc + bias + res) *
// scale + shift = acc * mul + add + res * mul with mul = scale and add = bias * scale +
// shift; without it mul = 1 and add = bias.  One FMA per value (two with a residual).
__device__ __forceinline__ void epi_constants(const TmaArgs& a, float* s_mul, float* s_add) {
  const bool bn = a.ybf && a.scale;
  for (int c = threadIdx.x; c < a.Cout && c < 256; c += blockDim.x) {
    const int ch = a.shuf ? c % a.cr : c;   // per column (sub-pixel: the column's channel)
    const float m = bn ? a.scale[ch] : 1.f;
    s_mul[c] = m;
    s_add[c] = (a.bias ? a.bias[ch] : 0.f) * m + (bn ? a.shift[ch] : 0.f);
  }
}

// Bias, residual, BatchNorm and eLU on 16 consecutive columns [cb, cb + 16) of one pixel,
// then the store (BF16 y, or FP32 out).  km / ka: the per-column constants in shared memory.
__device__ __forceinline__ void finish16(const TmaArgs& a, float* f, size_t pix, int cb, int sc, bool add_lin,
                                         const uint4* r4, const float* km, const float* ka) {
  // cb: first column (per-column constants), sc: first channel of the stored pixel
  if (cb + 16 <= a.Cout && a.vec) {
    if (add_lin) {
      const float4* m4 = reinterpret_cast<const float4*>(km + cb);
      const float4* a4 = reinterpret_cast<const float4*>(ka + cb);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 m = m4[q], c = a4[q];
        f[4 * q] = fmaf(f[4 * q], m.x, c.x);
        f[4 * q + 1] = fmaf(f[4 * q + 1], m.y, c.y);
        f[4 * q + 2] = fmaf(f[4 * q + 2], m.z, c.z);
        f[4 * q + 3] = fmaf(f[4 * q + 3], m.w, c.w);
      }
      if (a.res) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const __nv_bfloat162* r2 = reinterpret_cast<const __nv_bfloat162*>(&r4[h]);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float2 rf = __bfloat1622float2(r2[j]);
            const int i = 8 * h + 2 * j;
            f[i] = fmaf(rf.x, km[cb + i], f[i]);
            f[i + 1] = fmaf(rf.y, km[cb + i + 1], f[i + 1]);
          }
        }
      }
    }
    if (a.ybf) {
      if (a.act) {
#pragma unroll
        for (int j = 0; j < 16; ++j) f[j] = elu_bf(f[j]);
      }
      uint4 o4[2];
      __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(o4);
#pragma unroll
      for (int j = 0; j < 8; ++j) o2[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
      uint4* yp = reinterpret_cast<uint4*>(a.ybf + pix * a.ldy + sc);
      yp[0] = o4[0];
      yp[1] = o4[1];
      if (a.y2) {
        // eLU of the value as stored (rounded to BF16), as the consumer would compute it
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float2 t = __bfloat1622float2(o2[j]);
          o2[j] = __floats2bfloat162_rn(elu_bf(t.x), elu_bf(t.y));
        }
        uint4* zp = reinterpret_cast<uint4*>(a.y2 + pix * a.ldy2 + sc);
        zp[0] = o4[0];
        zp[1] = o4[1];
      }
    } else {
      float4* op = reinterpret_cast<float4*>(a.out + pix * a.ldo + sc);
#pragma unroll
      for (int q = 0; q < 4; ++q) op[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int co = cb + j, so = sc + j;
    if (co >= a.Cout) break;
    float g = f[j];
    if (add_lin) {
      g = fmaf(g, km[co], ka[co]);
      if (a.res) g = fmaf(__bfloat162float(a.res[pix * a.ldr + so]), km[co], g);
    }
    if (a.ybf) {
      if (a.act) g = elu_bf(g);
      const __nv_bfloat16 gb = __float2bfloat16_rn(g);
      a.ybf[pix * a.ldy + so] = gb;
      if (a.y2) {
        const float t = __bfloat162float(gb);
        a.y2[pix * a.ldy2 + so] = __float2bfloat16_rn(elu_bf(t));
      }
    } else {
      a.out[pix * a.ldo + so] = g;
    }
  }
}

// One value of column n stored as channel sc of pixel pix (constants and eLU as finish16).
__device__ __forceinline__ void finish1(const TmaArgs& a, float g, size_t pix, int n, int sc, const float* km,
                                        const float* ka) {
  g = fmaf(g, km[n], ka[n]);
  if (a.ybf) {
    if (a.act) g = elu_bf(g);
    const __nv_bfloat16 gb = __float2bfloat16_rn(g);
    a.ybf[pix * a.ldy + sc] = gb;
    if (a.y2) a.y2[pix * a.ldy2 + sc] = __float2bfloat16_rn(elu_bf(__bfloat162float(gb)));
  } else {
    a.out[pix * a.ldo + sc] = g;
  }
}

// Barrier of the epilogue warps that share an item (ids and counts as in epi_any).
__device__ __forceinline__ void epi_sync(int g, bool alt) {
  if (!alt) asm volatile("bar.sync 1, %0;\n" ::"n"(NEPI * 32) : "memory");
  else if (g == 0) asm volatile("bar.sync 1, %0;\n" ::"n"(NEPI / 2 * 32) : "memory");
  else asm volatile("bar.sync 2, %0;\n" ::"n"(NEPI / 2 * 32) : "memory");
}

// The epilogue of columns [c0, c0 + 16) of pixel pix of an item (non-split layout rules:
// plain, or the sub-pixel scatter of transposed layers), from accumulated values f.
__device__ __forceinline__ void finish_chunk(const TmaArgs& a, float* f, size_t pix, int b, int oy, int ox, int c0,
                                             const uint4* rc, const float* km, const float* ka) {
  if (!a.shuf) {
    finish16(a, f, pix, c0, c0, true, rc, km, ka);
  } else if (a.cr % 16 == 0) {
    // sub-pixel: the chunk is one phase's channels [co0, co0 + 16)
    const int ph = c0 / a.cr, co0 = c0 - ph * a.cr;
    const size_t opix = ((size_t)b * (2 * a.Ho) + 2 * oy + (ph >> 1)) * (2 * a.Wo) + 2 * ox + (ph & 1);
    finish16(a, f, opix, c0, co0, true, rc, km, ka);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = c0 + j;
      if (n >= a.Cout) break;
      const int ph = n / a.cr, co = n - ph * a.cr;
      const size_t opix = ((size_t)b * (2 * a.Ho) + 2 * oy + (ph >> 1)) * (2 * a.Wo) + 2 * ox + (ph & 1);
      finish1(a, f[j], opix, n, co, km, ka);
    }
  }
}

// Start reading 16 consecutive TMEM columns of this warp's 32 lanes (32x32b shape: thread t
// gets lane t); complete with tcgen05.wait::ld before using v.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// Wait for the outstanding TMEM reads; v is tied to the wait so that no use of it can be
// scheduled before the wait.
__device__ __forceinline__ void tmem_wait16(uint32_t (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                 "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}

// Epilogue warps (0 .. NEPI-1) of both convolution kernels: drain TMEM accumulator
// buffer i % nacc of item i into the destination, then hand the buffer back.  Warp w reads
// TMEM lanes 32 (w % 4) .. + 31 (the tile rows it may access).  With a.epig warps 0-3 take
// the CTA's even items and warps 4-7 the odd ones, every column each (two narrow tiles
// drain at a time); otherwise group w / 4 takes the 16-column chunks w / 4, w / 4 + 2, ...
// of every item (wide tiles).
__device__ __forceinline__ void conv_epilogue(const TmaArgs& a, uint32_t tmem, uint64_t* tfull, uint64_t* tempty,
                                              int* s_fail, const float* km, const float* ka) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.NT;
  volatile int* fail = s_fail;
  const int q4 = warp & 3, grp = warp >> 2;
  const int m = q4 * 32 + lane;
  const int bb = m / (a.BY * a.BX), rr = m - bb * a.BY * a.BX, by = rr / a.BX, bx = rr - by * a.BX;
  const bool alt = a.epig != 0;
  const int cfirst = alt ? 0 : 16 * grp, cstep = alt ? 16 : 32;
  const int istep = alt ? 2 : 1;
  int li = alt ? grp : 0;
  for (int w = blockIdx.x + (alt ? grp : 0) * gridDim.x; w < a.nitems; w += istep * gridDim.x, li += istep) {
    if (epi_any(failed(fail), grp, alt)) break;
    const Item it = decode(a, w);
    const int acc = li & (a.nacc - 1);
    const bool ok = mb_wait(su32(&tfull[acc]), (uint32_t)(li >> a.lg_nacc) & 1u);
    if (epi_any(!ok, grp, alt)) { atomicExch(s_fail, 1); break; }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int b = it.b0 + bb, qy = it.y0 + by, qx = it.x0 + bx;
    const int oy = a.transposed ? 2 * qy + it.py : qy, ox = a.transposed ? 2 * qx + it.px : qx;
    const bool rv = it.nkb > 0 && b < a.B && oy < a.Ho && ox < a.Wo;
    const size_t pix = ((size_t)b * a.Ho + oy) * a.Wo + ox;
    // residual of the next chunk is requested before the current chunk's TMEM read
    const bool pre = rv && a.ksplit <= 1 && a.res && a.vec;
    uint4 rn[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
    if (pre && cfirst + 16 <= a.Cout) {
      const uint4* rp = reinterpret_cast<const uint4*>(a.res + pix * a.ldr + cfirst);
      rn[0] = rp[0]; rn[1] = rp[1];
    }
    // TMEM columns of chunk c0 for this warp's lane quadrant; the next chunk's read is
    // issued before the current chunk is finished, so its latency overlaps that work
    const uint32_t trow = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(acc * a.colsz);
    for (int c0 = cfirst; c0 < N; c0 += cstep) {
      uint32_t v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
      const uint4 rc[2] = {rn[0], rn[1]};
      if (pre && c0 + cstep + 16 <= a.Cout) {
        const uint4* rp = reinterpret_cast<const uint4*>(a.res + pix * a.ldr + c0 + cstep);
        rn[0] = rp[0]; rn[1] = rp[1];
      }
      tmem_wait16(v);
      float f[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) f[j] = __uint_as_float(v[j]);
      if (!rv) continue;
      if (a.ksplit > 1) {
        // partial sums of this K range into the split's slice (plain stores)
        float* dst = a.part + (size_t)it.split * a.slice + pix * a.Cout + c0;
        if (c0 + 16 <= a.Cout && a.vec) {
          float4* op = reinterpret_cast<float4*>(dst);
#pragma unroll
          for (int q = 0; q < 4; ++q) op[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < a.Cout) dst[j] = f[j];
        }
      } else {
        finish_chunk(a, f, pix, b, oy, ox, c0, rc, km, ka);
      }
    }
    // accumulator read: hand buffer acc back to the MMA warp
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(&tempty[acc])) : "memory");
    if (a.ksplit > 1 && a.cnt) {
      // split-K fix-up: the last split of this tile to store its partial sums adds every
      // split's slice and applies the epilogue (no separate finishing launch)
      __shared__ int s_last[2];
      __threadfence();                                   // this thread's partial sums, device-wide
      epi_sync(grp, alt);
      const int tile = w % (a.tx * a.ty * a.tb * (a.transposed ? 4 : 1));
      if ((warp & 3) == 0 && lane == 0 && (alt || grp == 0))
        s_last[grp] = atomicAdd(a.cnt + tile, 1) == a.ksplit - 1;
      epi_sync(grp, alt);
      if (s_last[alt ? grp : 0]) {
        __threadfence();
        for (int c0 = cfirst; c0 < N && rv; c0 += cstep) {
          float f[16];
          const float* src = a.part + pix * a.Cout + c0;
          if (c0 + 16 <= a.Cout && a.vec) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float4 t = __ldcg(reinterpret_cast<const float4*>(src) + q);
              for (int sp = 1; sp < a.ksplit; ++sp) {
                const float4 u = __ldcg(reinterpret_cast<const float4*>(src + (size_t)sp * a.slice) + q);
                t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
              }
              f[4 * q] = t.x; f[4 * q + 1] = t.y; f[4 * q + 2] = t.z; f[4 * q + 3] = t.w;
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              f[j] = 0.f;
              if (c0 + j < a.Cout)
                for (int sp = 0; sp < a.ksplit; ++sp) f[j] += __ldcg(src + (size_t)sp * a.slice + j);
            }
          }
          uint4 rc[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
          if (a.res && a.vec && c0 + 16 <= a.Cout) {
            const uint4* rp = reinterpret_cast<const uint4*>(a.res + pix * a.ldr + c0);
            rc[0] = rp[0]; rc[1] = rp[1];
          }
          finish_chunk(a, f, pix, b, oy, ox, c0, rc, km, ka);
        }
        if ((warp & 3) == 0 && lane == 0 && (alt || grp == 0)) a.cnt[tile] = 0;   // ready for the next launch
      }
    }
  }
}

// Persistent: CTA c takes items c, c + gridDim.x, ...  The producer warp streams
// K-blocks through the stage ring across item boundaries, the MMA warp accumulates
// item i in TMEM buffer i & 1, the epilogue warps drain buffer i & 1 while the MMAs
// of item i + 1 run.
// (two CTAs per SM for N <= 64 need <= 102 registers per thread at 320 threads)
// GROUPED: a.kps K-blocks per stage (the instantiation without it keeps the one-K-block loops
// only: the widest layers, which never group, measured 7 % slower with both in one kernel).
template <bool GROUPED>
__global__ void __launch_bounds__(NTHR, 2) k_conv_tma(const __grid_constant__ CUtensorMap mA0,
                                                    const __grid_constant__ CUtensorMap mA1,
                                                    const __grid_constant__ CUtensorMap mB, TmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[MAXST], empty[MAXST], tfull[NACC], tempty[NACC], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ __align__(16) float s_mul[256], s_add[256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.NT, NS = a.nst;

  const uint32_t base = (su32(smem) + 1023u) & ~1023u;
  const int TK = a.tk;
  // a stage holds kps K-blocks, each an A box followed by its B tile
  const uint32_t a_bytes = TM * 2 * TK, b_bytes = (uint32_t)N * 2 * TK, kbytes = a_bytes + b_bytes;
  const uint32_t stage = GROUPED ? kbytes * (uint32_t)a.kps : kbytes;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) { mb_init(su32(&full[s]), 1); mb_init(su32(&empty[s]), 1); }
    for (int q = 0; q < a.nacc; ++q) {
      mb_init(su32(&tfull[q]), 1);
      mb_init(su32(&tempty[q]), a.epig ? NEPI / 2 : NEPI);   // lane 0 of each draining warp
    }
    mb_init(su32(&drain), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const uint32_t ncols = (uint32_t)a.nacc * (uint32_t)a.colsz;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_slot)),
        "r"(ncols)
        : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // everything above overlaps the previous kernel; global memory is read from here on
  griddep_wait();
  griddep_launch();
  epi_constants(a, s_mul, s_add);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* fail = &s_fail;

  if (warp == WPROD) {
    if (lane == 0) {
      uint32_t g = 0;   // K-blocks issued by this CTA
      for (int w = blockIdx.x; w < a.nitems && !failed(fail); w += gridDim.x) {
        const Item it = decode(a, w);
        bool ok = true;
        // K-block kbeg + kb = (tap ty * ntx + tx, chunk ch), stepped without divisions
        int ch = it.kbeg % it.nchk, tap = it.kbeg / it.nchk;
        int ty = tap / it.ntx, tx = tap - ty * it.ntx;
        // one K-block per stage (the producer is on the critical path of the widest layers:
        // its loop stays minimal there)
        if constexpr (!GROUPED) {
          for (int kb = 0; kb < it.nkb; ++kb, ++g) {
            const uint32_t use = (uint32_t)fdiv(a.f_ns, (int)g);
            const int s = (int)(g - use * (uint32_t)NS);
            if (g >= (uint32_t)NS && !mb_wait(su32(&empty[s]), (use - 1) & 1u)) { ok = false; break; }
            const int ky = it.ky0 + it.dk * ty, kx = it.kx0 + it.dk * tx;
            int ix, iy;
            if (!a.transposed) { ix = it.x0 * a.stride + kx - a.pad; iy = it.y0 * a.stride + ky - a.pad; }
            else { ix = it.x0 + (it.px + a.pad - kx) / 2; iy = it.y0 + (it.py + a.pad - ky) / 2; }
            const uint32_t sA = base + (uint32_t)s * stage, sB = sA + a_bytes;
            mb_expect_tx(su32(&full[s]), kbytes);
            if (ch < a.nch0) tma_load_4d(sA, &mA0, ch * TK, ix, iy, it.b0, su32(&full[s]));
            else tma_load_4d(sA, &mA1, (ch - a.nch0) * TK, ix, iy, a.bcast1 ? 0 : it.b0, su32(&full[s]));
            tma_load_2d(sB, &mB, (ky * a.k + kx) * a.kpad + ch * TK, 0, su32(&full[s]));
            if (++ch == it.nchk) {
              ch = 0;
              if (++tx == it.ntx) { tx = 0; ++ty; }
            }
          }
        } else {
          for (int kb = 0; kb < it.nkb; ++g) {
            const uint32_t use = (uint32_t)fdiv(a.f_ns, (int)g);
            const int s = (int)(g - use * (uint32_t)NS);
            if (g >= (uint32_t)NS && !mb_wait(su32(&empty[s]), (use - 1) & 1u)) { ok = false; break; }
            const int nb = min(a.kps, it.nkb - kb);
            const uint32_t sA0 = base + (uint32_t)s * stage;
            mb_expect_tx(su32(&full[s]), kbytes * (uint32_t)nb);
            for (int b = 0; b < nb; ++b, ++kb) {
              const int ky = it.ky0 + it.dk * ty, kx = it.kx0 + it.dk * tx;
              int ix, iy;
              if (!a.transposed) { ix = it.x0 * a.stride + kx - a.pad; iy = it.y0 * a.stride + ky - a.pad; }
              else { ix = it.x0 + (it.px + a.pad - kx) / 2; iy = it.y0 + (it.py + a.pad - ky) / 2; }
              const uint32_t sA = sA0 + (uint32_t)b * kbytes, sB = sA + a_bytes;
              if (ch < a.nch0) tma_load_4d(sA, &mA0, ch * TK, ix, iy, it.b0, su32(&full[s]));
              else tma_load_4d(sA, &mA1, (ch - a.nch0) * TK, ix, iy, a.bcast1 ? 0 : it.b0, su32(&full[s]));
              tma_load_2d(sB, &mB, (ky * a.k + kx) * a.kpad + ch * TK, 0, su32(&full[s]));
              if (++ch == it.nchk) {
                ch = 0;
                if (++tx == it.ntx) { tx = 0; ++ty; }
              }
            }
          }
        }
        if (!ok) { atomicExch(&s_fail, 1); break; }
      }
      // let the loads still in flight land before the CTA can exit (bounded)
      for (uint32_t j = g > (uint32_t)NS ? g - (uint32_t)NS : 0u; j < g; ++j)
        mb_wait(su32(&full[j % (uint32_t)NS]), (j / (uint32_t)NS) & 1u);
    }
  } else if (warp == WMMA) {
    if (lane == 0) {
      const uint32_t id = idesc(N);
      uint32_t g = 0;
      int li = 0;
      for (int w = blockIdx.x; w < a.nitems && !failed(fail); w += gridDim.x, ++li) {
        const Item it = decode(a, w);
        const int acc = li & (a.nacc - 1);
        const uint32_t use = (uint32_t)(li >> a.lg_nacc);
        if (li >= a.nacc && !mb_wait(su32(&tempty[acc]), (use - 1) & 1u)) { atomicExch(&s_fail, 1); break; }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(acc * a.colsz);
        bool ok = true;
        int kch = it.kbeg % it.nchk;   // chunk of K-block kbeg + kb, stepped below
        for (int kb = 0; kb < it.nkb; ++g) {
          const uint32_t use = (uint32_t)fdiv(a.f_ns, (int)g);
          const int s = (int)(g - use * (uint32_t)NS);
          if (!mb_wait(su32(&full[s]), use & 1u)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t sA = base + (uint32_t)s * stage;
          const uint32_t acc0 = kb > 0 ? 1u : 0u;
          if constexpr (GROUPED) {
            // every chunk full: TK / 16 K-steps per K-block, the stage's K-blocks as one block
            const int nb = min(a.kps, it.nkb - kb);
            mma_kblocks_n(nb, TK / 16, d, sA, sA + a_bytes, kbytes, TK, id, acc0);
            kb += nb;
          } else {
            // K-steps of 16 that hold real channels (the rest of a chunk is zero fill)
            const int cval = kch < a.nch0 ? min(TK, a.c0 - kch * TK) : min(TK, a.c1 - (kch - a.nch0) * TK);
            const int nk4 = (cval + 15) / 16;
            mma_taps_k<1>(nk4, d, sA, 0u, sA + a_bytes, 0u, TK, id, acc0);
            kch = kch + 1 == it.nchk ? 0 : kch + 1;
            ++kb;
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              su32(&empty[s]))
              : "memory");
        }
        if (!ok) { atomicExch(&s_fail, 1); break; }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            su32(&tfull[acc]))
            : "memory");
      }
      // every MMA issued above completes before tensor memory is released (bounded)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&drain))
          : "memory");
      mb_wait(su32(&drain), 0);
    }
  } else {
    conv_epilogue(a, tmem, tfull, tempty, &s_fail, s_mul, s_add);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_fail && a.err) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// Column-reuse variant, for layers whose whole padded weight copy fits in shared
// memory next to the stage ring (one 128-pixel tile of BX x BY pixels, BX in {8, 16}):
// the weights are loaded once per CTA, and per (x-tap, channel chunk) one TMA box of
// (BY + nyt - 1) rows of BX pixels serves every y-tap of that column -- y-tap j is the
// box from row j * BX on, i.e. BX * 2 tk bytes further, a whole number of 8-row
// swizzle atoms.  Stride-2 convolutions split their y-taps into even and odd classes
// (element stride 2 along y); transposed stride-2 convolutions use their phase's taps.
// A stage holds the boxes of every x-tap of one (channel chunk, class) when two such stages
// fit, else one box.  The producer writes, per stage slot, what the MMA thread needs (the
// low descriptor words of A and B, the stage's shape, whether it starts or ends an item),
// so the single MMA-issuing thread only waits, reads that record and issues the stage's
// MMAs (x-taps x y-taps x K-steps, 18 for a 3x3 layer of 32 channels) as one straight-line
// block: its own instruction latency, not the tensor pipe, bounded these layers.
struct ReuseArgs {
  int nyt;        // y-taps one box serves at most (box height BY + nyt - 1)
  int nxt;        // x-taps (boxes) one stage holds at most
  int bres;       // bytes of the resident weights (all taps x chunks, NT rows each)
};

__global__ void __launch_bounds__(NTHR, 2) k_conv_tma_reuse(const __grid_constant__ CUtensorMap mA,
                                                            const __grid_constant__ CUtensorMap mB, TmaArgs a,
                                                            ReuseArgs r) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[MAXST], empty[MAXST], tfull[NACC], tempty[NACC], drain, wres;
  // per stage slot, written by the producer before it arms the slot: low descriptor words of
  // A and B, shape code | flags << 16 (1: first stage of an item, 2: last)
  __shared__ uint4 sdesc[MAXST];
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  __shared__ __align__(16) float s_mul[256], s_add[256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.NT, NS = a.nst;
  const uint32_t wbase = (su32(smem) + 1023u) & ~1023u;          // resident weights
  const uint32_t base = wbase + (((uint32_t)r.bres + 1023u) & ~1023u);
  const int TK = a.tk;
  const uint32_t box = (uint32_t)((a.BY + r.nyt - 1) * a.BX * 2 * TK);   // one x-tap's input box
  const uint32_t stage = box * (uint32_t)r.nxt;
  const uint32_t wtile = (uint32_t)N * 2 * TK;                    // one (tap, chunk) weight tile
  const int nch = a.nch0;
  if (tid == 0) {
    for (int q = 0; q < NS; ++q) { mb_init(su32(&full[q]), 1); mb_init(su32(&empty[q]), 1); }
    for (int q = 0; q < a.nacc; ++q) {
      mb_init(su32(&tfull[q]), 1);
      mb_init(su32(&tempty[q]), a.epig ? NEPI / 2 : NEPI);   // lane 0 of each draining warp
    }
    mb_init(su32(&drain), 1);
    mb_init(su32(&wres), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const uint32_t ncols = (uint32_t)a.nacc * (uint32_t)a.colsz;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  // everything above overlaps the previous kernel; global memory is read from here on
  griddep_wait();
  griddep_launch();
  epi_constants(a, s_mul, s_add);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* fail = &s_fail;
  const bool tr = a.transposed != 0;
  const int ncls = (!tr && a.stride == 2) ? 2 : 1;

  if (warp == WPROD) {
    if (lane == 0) {
      // the weights, once
      mb_expect_tx(su32(&wres), (uint32_t)r.bres);
      for (int tap = 0; tap < a.k * a.k; ++tap)
        for (int ch = 0; ch < nch; ++ch)
          tma_load_2d(wbase + (uint32_t)(tap * nch + ch) * wtile, &mB, tap * a.kpad + ch * TK, 0, su32(&wres));
      uint32_t g = 0;
      for (int w = blockIdx.x; w < a.nitems && !failed(fail); w += gridDim.x) {
        const Item it = decode(a, w);
        const int nxt = tr ? it.ntx : a.k;
        const int nty = tr ? (a.k - it.ky0 + 1) / 2 : 0;
        bool ok = true;
        const int kx0 = tr ? it.kx0 : 0, dkx = tr ? 2 : 1;
        for (int ch = 0; ch < nch && ok; ++ch)
          for (int cls = 0; cls < ncls && ok; ++cls)
            for (int xg = 0; xg < nxt; xg += r.nxt, ++g) {
              const int nx = min(r.nxt, nxt - xg);
              const uint32_t use = (uint32_t)fdiv(a.f_ns, (int)g);
              const int s = (int)(g - use * (uint32_t)NS);
              if (g >= (uint32_t)NS && !mb_wait(su32(&empty[s]), (use - 1) & 1u)) { ok = false; break; }
              const uint32_t sA = base + (uint32_t)s * stage;
              // what the MMA thread needs for this stage: box x = x-tap kx0 + dkx (xg + x), its
              // y-taps j = 0 .. nj-1 (ky = ky0 + dky j) at box row j * BX (transposed: reversed)
              {
                const int nk4 = (min(TK, a.c0 - ch * TK) + 15) / 16;   // K-steps with real channels
                const int nj = tr ? nty : (a.stride == 1 ? a.k : (a.k - cls + 1) / 2);
                const int ky0 = tr ? it.ky0 : (a.stride == 1 ? 0 : cls);
                const uint32_t a0 = tr ? sA + (uint32_t)(nty - 1) * (uint32_t)(a.BX * 2 * TK) : sA;
                const uint32_t w0 = wbase + (uint32_t)((ky0 * a.k + kx0 + dkx * xg) * nch + ch) * wtile;
                const uint32_t flags = (ch == 0 && cls == 0 && xg == 0 ? 1u : 0u) |
                                       (ch == nch - 1 && cls == ncls - 1 && xg + r.nxt >= nxt ? 2u : 0u);
                sdesc[s] = make_uint4(desc_lo(a0), desc_lo(w0),
                                      (uint32_t)nx | ((uint32_t)nj << 4) | ((uint32_t)nk4 << 8) | (flags << 16), 0u);
              }
              mb_expect_tx(su32(&full[s]), box * (uint32_t)nx);
              for (int x = 0; x < nx; ++x) {
                const int xt = xg + x;
                int ix, iy;
                if (!tr) {
                  ix = it.x0 * a.stride + xt - a.pad;
                  iy = a.stride == 1 ? it.y0 - a.pad : 2 * it.y0 + cls - a.pad;
                } else {
                  const int kx = it.kx0 + 2 * xt;
                  ix = it.x0 + (it.px + a.pad - kx) / 2;
                  iy = it.y0 + (it.py + a.pad - it.ky0) / 2 - (nty - 1);
                }
                tma_load_4d(sA + (uint32_t)x * box, &mA, ch * TK, ix, iy, it.b0, su32(&full[s]));
              }
            }
        if (!ok) { atomicExch(&s_fail, 1); break; }
      }
      for (uint32_t j = g > (uint32_t)NS ? g - (uint32_t)NS : 0u; j < g; ++j)
        mb_wait(su32(&full[j % (uint32_t)NS]), (j / (uint32_t)NS) & 1u);
      mb_wait(su32(&wres), 0);
    }
  } else if (warp == WMMA) {
    if (lane == 0) {
      // one pass per stage, from the producer's stage records: wait for the stage, on an
      // item's first stage also for its accumulator, issue the stage's MMAs as one block,
      // release the stage, and on an item's last stage hand the accumulator to the epilogue
      const uint32_t id = idesc(N), hi = desc_hi(TK);
      const uint32_t rows = (uint32_t)(a.BX * 2 * TK) >> 4;           // one box row, 16-byte units
      const uint32_t as = tr ? 0u - rows : rows, xs = box >> 4;
      const int dky = a.stride == 1 && !tr ? 1 : 2, dkx = tr ? 2 : 1;
      const uint32_t ws = ((uint32_t)(dky * a.k * nch) * wtile) >> 4, wxs = ((uint32_t)(dkx * nch) * wtile) >> 4;
      const int items = (int)blockIdx.x < a.nitems ? (a.nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
      const bool wok = mb_wait(su32(&wres), 0);
      if (!wok) atomicExch(&s_fail, 1);
      uint32_t g = 0;
      int li = 0;
      uint32_t d = tmem;
      while (wok && li < items && !failed(fail)) {
        const uint32_t use = (uint32_t)fdiv(a.f_ns, (int)g);
        const int s = (int)(g - use * (uint32_t)NS);
        if (!mb_wait(su32(&full[s]), use & 1u)) { atomicExch(&s_fail, 1); break; }
        const uint4 q = sdesc[s];
        const uint32_t flags = q.z >> 16, shape = q.z & 0xFFFFu;
        const int acc = li & (a.nacc - 1);
        if (flags & 1u) {
          if (li >= a.nacc && !mb_wait(su32(&tempty[acc]), (uint32_t)((li >> a.lg_nacc) - 1) & 1u)) {
            atomicExch(&s_fail, 1);
            break;
          }
          d = tmem + (uint32_t)(acc * a.colsz);
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t acc0 = (flags & 1u) ? 0u : 1u;
        if (!mma_lo_shape(shape, d, q.x, as, xs, q.y, ws, wxs, hi, id, acc0)) {
          const int nx = (int)(shape & 15u), nj = (int)((shape >> 4) & 15u), nk4 = (int)(shape >> 8);
          for (int x = 0; x < nx; ++x)
            for (int j = 0; j < nj; ++j)
              for (int k = 0; k < nk4; ++k)
                mma_lo(d, q.x + (uint32_t)x * xs + (uint32_t)j * as + 2u * k,
                       q.y + (uint32_t)x * wxs + (uint32_t)j * ws + 2u * k, hi, id,
                       (x == 0 && j == 0 && k == 0) ? acc0 : 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         su32(&empty[s]))
                     : "memory");
        if (flags & 2u) {
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           su32(&tfull[acc]))
                       : "memory");
          ++li;
        }
        ++g;
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&drain))
                   : "memory");
      mb_wait(su32(&drain), 0);
    }
  } else {
    conv_epilogue(a, tmem, tfull, tempty, &s_fail, s_mul, s_add);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_fail && a.err) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// Split-K epilogue: y[p][c] = act(BN(sum_s part[s][p][c] + bias[c] + res[p][c])), four
// channels per thread (Cout % 4 == 0), BF16 into y or FP32 into out.
__global__ void __launch_bounds__(256) k_splitk_finish(TmaArgs a, int M) {
  griddep_wait();
  griddep_launch();
  const int C4 = a.Cout / 4;
  const size_t n = (size_t)M * C4;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t p = i / C4;
    const int c = (int)(i - p * C4) * 4;
    float4 t = __ldcg(reinterpret_cast<const float4*>(a.part + p * a.Cout + c));
    for (int sp = 1; sp < a.ksplit; ++sp) {
      const float4 u = __ldcg(reinterpret_cast<const float4*>(a.part + (size_t)sp * a.slice + p * a.Cout + c));
      t.x += u.x; t.y += u.y; t.z += u.z; t.w += u.w;
    }
    float f[4] = {t.x, t.y, t.z, t.w};
    const int cc = a.shuf ? c % a.cr : c;   // channel of the column (sub-pixel: within its phase)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (a.bias) f[j] += a.bias[cc + j];
      if (a.res) f[j] += __bfloat162float(a.res[p * a.ldr + c + j]);
      if (a.ybf) {
        if (a.scale) f[j] = f[j] * a.scale[cc + j] + a.shift[cc + j];
        if (a.act) f[j] = elu_bf(f[j]);
      }
    }
    // destination pixel and channel of column c + j (sub-pixel: phase scatter)
    size_t q = p;
    int sc = c;
    if (a.shuf) {
      const int ph = c / a.cr;   // cr % 4 == 0: the four columns share the phase
      const size_t wq = (size_t)a.Wo, hq = (size_t)a.Ho;
      const size_t bq = p / (hq * wq), rq = p - bq * hq * wq, yq = rq / wq, xq = rq - yq * wq;
      q = (bq * 2 * hq + 2 * yq + (ph >> 1)) * (2 * wq) + 2 * xq + (ph & 1);
      sc = c - ph * a.cr;
    }
    if (a.ybf) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16 yb = __float2bfloat16_rn(f[j]);
        a.ybf[q * a.ldy + sc + j] = yb;
        if (a.y2) {
          const float t = __bfloat162float(yb);
          a.y2[q * a.ldy2 + sc + j] = __float2bfloat16_rn(elu_bf(t));
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) a.out[q * a.ldo + sc + j] = f[j];
    }
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

CUtensorMapSwizzle swizzle_for(int tk) {
  return tk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (tk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
}

// 4-D map over an NHWC BF16 source slice: (channels, x, y, image), box (tk, BX*s, BY*s, BB).
bool encode_act(CUtensorMap* m, const void* ptr, int C, int ld, int W, int H, int B, int BX, int BY, int BB, int es,
                int tk) {
  if (((uintptr_t)ptr & 15) || (ld * 2) % 16) return false;
  cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
  cuuint64_t strides[3] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 2 * W, (cuuint64_t)ld * 2 * W * H};
  cuuint32_t box[4] = {(cuuint32_t)tk, (cuuint32_t)(BX * es), (cuuint32_t)(BY * es), (cuuint32_t)BB};
  cuuint32_t estr[4] = {1, (cuuint32_t)es, (cuuint32_t)es, 1};
  if (box[1] > 256 || box[2] > 256) return false;
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(tk), CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_w(CUtensorMap* m, const void* ptr, int K, int cout, int NT, int tk) {
  if (((uintptr_t)ptr & 15) || (K * 2) % 16) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)cout};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {(cuuint32_t)tk, (cuuint32_t)NT};
  cuuint32_t estr[2] = {1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle_for(tk), CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
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

// Adjoint copy for data gradients: the convolution of dL/dy with W^T, as a forward
// convolution with Cin' = cout inputs and Cout' = cin outputs:
// WPA[ci][tap'][kpad'] = W[tap][ci][co] (co < cout), tap = taps - 1 - tap' when flipped.
__global__ void k_weights_adjoint(const float* __restrict__ P, __nv_bfloat16* __restrict__ WPA, int taps, int cin,
                                  int cout, int kpad, int flip) {
  const size_t n = (size_t)cin * taps * kpad;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int co = (int)(i % kpad);
    const size_t r = i / kpad;
    const int tp = (int)(r % taps), ci = (int)(r / taps);
    const int tap = flip ? taps - 1 - tp : tp;
    WPA[i] = __float2bfloat16_rn(co < cout ? P[((size_t)tap * cin + ci) * cout + co] : 0.f);
  }
}

// Sub-pixel copy of a transposed 5x5 stride-2 (pad 2) convolution: a 3x3 stride-1
// convolution over the input grid with 4 * cout outputs, column n = (2 py + px) * cout + co:
// WS[n][(dy + 1) * 3 + dx + 1][chunked ci] = W[py + 2 - 2 dy][px + 2 - 2 dx][ci][co], zero
// where the tap falls outside the 5x5 kernel.  Chunks as the padded copy (c0, then c1).
__global__ void k_weights_subpixel(const float* __restrict__ P, __nv_bfloat16* __restrict__ WS, int c0, int c1,
                                   int cout, int kpad, int off1) {
  const int cin = c0 + c1;
  const size_t n = (size_t)4 * cout * 9 * kpad;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % kpad);
    const size_t r = i / kpad;
    const int t3 = (int)(r % 9), col = (int)(r / 9);
    const int ph = col / cout, co = col - ph * cout, py = ph >> 1, px = ph & 1;
    const int dy = t3 / 3 - 1, dx = t3 % 3 - 1;
    const int ky = py + 2 - 2 * dy, kx = px + 2 - 2 * dx;
    int ci = -1;
    if (k < c0) ci = k;
    else if (k >= off1 && k < off1 + c1) ci = c0 + (k - off1);
    float v = 0.f;
    if (ci >= 0 && ky >= 0 && ky < 5 && kx >= 0 && kx < 5) v = P[((size_t)(ky * 5 + kx) * cin + ci) * cout + co];
    WS[i] = __float2bfloat16_rn(v);
  }
}

// Space-to-depth form of the 5x5 stride-2 input convolution (pad 2) from cin <= 4
// channels: on the grid of 2x2 input blocks it is a 3x3 stride-1 convolution (pad 1)
// whose input pixel holds the block's 4 cin values, channel (dy * 2 + dx) * cin + c.
// Block tap (by, bx) and sub-pixel (dy, dx) meet the original tap (2 by + dy, 2 bx + dx);
// taps 5 of that 6x6 footprint are zero.  WD[co][t3][k] (K-major, 16 channels per tap).
__global__ void k_weights_s2d_in(const float* __restrict__ P, __nv_bfloat16* __restrict__ WD, int cin, int cout) {
  const size_t n = (size_t)cout * 9 * 16;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % 16);
    const size_t r = i / 16;
    const int t3 = (int)(r % 9), co = (int)(r / 9);
    const int sub = k / cin, c = k - sub * cin;
    const int ky = 2 * (t3 / 3) + (sub >> 1), kx = 2 * (t3 % 3) + (sub & 1);
    float v = 0.f;
    if (sub < 4 && ky < 5 && kx < 5) v = P[((size_t)(ky * 5 + kx) * cin + c) * cout + co];
    WD[i] = __float2bfloat16_rn(v);
  }
}

}  // namespace

size_t conv_tma_weight_s2d_elems(int cout) { return (size_t)cout * 9 * 16; }

void conv_tma_weights_s2d_in(const float* P, __nv_bfloat16* WD, int cin, int cout, cudaStream_t s) {
  const size_t n = conv_tma_weight_s2d_elems(cout);
  k_weights_s2d_in<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(P, WD, cin, cout);
}

// Channels per K-chunk (one stage row per pixel) of a layer with sources of c0 and c1
// channels: the narrowest of 16, 32, 64 that holds the wider source, so that narrow
// layers stage no zero-filled channels (rows of 32, 64 or 128 bytes, swizzled to match).
// The padded weight copies and the launchers both follow this rule.
static int conv_tk(int c0, int c1) {
  const int m = std::max(c0, c1);
  return m <= 16 ? 16 : (m <= 32 ? 32 : 64);
}

// Padded K per tap of a two-source layer: each source in whole tk-channel chunks.
static int kpad_of(int c0, int c1) {
  const int tk = conv_tk(c0, c1);
  return tk * ((c0 + tk - 1) / tk + (c1 + tk - 1) / tk);
}

size_t conv_tma_weight_sub_elems(int c0, int c1, int cout) { return (size_t)4 * cout * 9 * kpad_of(c0, c1); }

void conv_tma_weights_subpixel(const float* P, __nv_bfloat16* WS, int c0, int c1, int cout, cudaStream_t s) {
  const int tk = conv_tk(c0, c1);
  const int kpad = kpad_of(c0, c1);
  const size_t n = (size_t)4 * cout * 9 * kpad;
  k_weights_subpixel<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(P, WS, c0, c1, cout, kpad,
                                                                                      tk * ((c0 + tk - 1) / tk));
}

size_t conv_tma_weight_adj_elems(int k, int cin, int cout) { return (size_t)cin * k * k * kpad_of(cout, 0); }

void conv_tma_weights_adjoint(const float* P, __nv_bfloat16* WPA, int k, int cin, int cout, bool flip,
                              cudaStream_t s) {
  const int kpad = kpad_of(cout, 0);
  const size_t n = (size_t)cin * k * k * kpad;
  k_weights_adjoint<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(P, WPA, k * k, cin, cout, kpad,
                                                                                     flip ? 1 : 0);
}

size_t conv_tma_weight_elems(int k, int c0, int c1, int cout) { return (size_t)cout * k * k * kpad_of(c0, c1); }

void conv_tma_weights(const float* P, __nv_bfloat16* WP, int k, int c0, int c1, int cout, cudaStream_t s) {
  const int tk = conv_tk(c0, c1);
  const int kpad = kpad_of(c0, c1);
  const size_t n = (size_t)cout * k * k * kpad;
  k_weights_padded<<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(P, WP, k * k, c0, c1, cout, kpad,
                                                                                     tk * ((c0 + tk - 1) / tk));
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cache[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = n > 0 ? n : 1;
  }
  return cache[dev];
}

// Encoded tensor maps, keyed by every argument of the encoding (a map only holds the
// address and the geometry, so a hit is valid whatever happened to the buffer since).
struct MapKey {
  const void* p;
  int v[10];
  bool operator==(const MapKey& o) const {
    if (p != o.p) return false;
    for (int i = 0; i < 10; ++i)
      if (v[i] != o.v[i]) return false;
    return true;
  }
};
struct MapKeyHash {
  size_t operator()(const MapKey& k) const {
    size_t h = std::hash<const void*>()(k.p);
    for (int i = 0; i < 10; ++i) h = h * 1000003u ^ (size_t)(unsigned)k.v[i];
    return h;
  }
};
std::mutex g_maps_mu;
std::unordered_map<MapKey, CUtensorMap, MapKeyHash> g_maps;

template <typename F>
bool cached_map(const MapKey& key, CUtensorMap* out, F encode) {
  {
    std::lock_guard<std::mutex> lk(g_maps_mu);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) { *out = it->second; return true; }
  }
  if (!encode(out)) return false;
  std::lock_guard<std::mutex> lk(g_maps_mu);
  if (g_maps.size() > 4096) g_maps.clear();
  g_maps.emplace(key, *out);
  return true;
}
int ctas_per_sm(int nt) { return nt <= 64 ? 2 : 1; }

// K split for convolutions whose pixel tiles leave most SMs idle (1 = none).
int conv_tma_split(const ConvArgs& c) {
  const int Wq = c.transposed ? c.Wo / 2 : c.Wo, Hq = c.transposed ? c.Ho / 2 : c.Ho;
  // partial sums go to FP32 slices of the split scratch (capacity splitcnt_n floats)
  if (!pow2(Wq) || !pow2(Hq) || !c.splitbuf || c.Cout % 4 || (c.shuffle && c.cr % 4)) return 1;
  const int BX = Wq < 128 ? Wq : 128;
  const int BY = Hq < 128 / BX ? Hq : 128 / BX;
  const int BB = 128 / (BX * BY);
  const int tiles = (Wq / BX) * (Hq / BY) * ((c.B + BB - 1) / BB) * (c.transposed ? 4 : 1);
  const long long outsz = (long long)c.B * c.Ho * c.Wo * c.Cout;
  const int taps = c.transposed ? (c.k * c.k + 3) / 4 : c.k * c.k;
  const int c1 = c.in1 ? c.c1 : 0, tk = conv_tk(c.c0, c1);
  const int nkb = taps * ((c.c0 + tk - 1) / tk + (c1 + tk - 1) / tk);
  const int slots = sm_count() * ctas_per_sm(((c.Cout + 15) / 16) * 16);
  int sp = 1;
  while (tiles * sp * 2 <= slots && nkb / (sp * 2) >= 4 && sp < 16 && outsz * sp * 2 <= c.splitcnt_n) sp *= 2;
  return sp;
}

// The column-reuse kernel for a layer that qualifies (single source, N <= 64, all
// weights plus >= 2 stages in shared memory, tile width 8 or 16); false otherwise.
bool launch_reuse(const ConvArgs& c, int* err, cudaStream_t s) {
  if (c.in1 || c.Cout > 64) return false;
  const bool tr = c.transposed != 0;
  if (tr ? (c.k != 5 || c.pad != 2) : !((c.k == 3 && c.stride == 1 && c.pad == 1) || (c.k == 5 && c.stride == 2 && c.pad == 2)))
    return false;
  const int Wq = tr ? c.Wo / 2 : c.Wo, Hq = tr ? c.Ho / 2 : c.Ho;
  if (!pow2(Wq) || !pow2(Hq) || Wq < 8) return false;
  const int BX = Wq < 16 ? Wq : 16, BY = 128 / BX;
  if (Hq < BY || (tr && (c.Wo % 2 || c.Ho % 2))) return false;
  const int NT = ((c.Cout + 15) / 16) * 16;
  const int nyt = (!tr && c.stride == 1) ? c.k : (c.k + 1) / 2;
  const int es = (!tr && c.stride == 2) ? 2 : 1;
  const int nxt_all = tr ? (c.k + 1) / 2 : c.k;
  // Configuration, first that fits: (1) two CTAs per SM (two MMA-issuing threads), stages
  // of every x-tap box of a (chunk, class) -- the stage's MMAs issue as one block; (2) the
  // same with 32-channel chunks (half the box and stage), where the padded weight layout is
  // the same; (3) one CTA per SM with merged stages (the whole shared memory for resident
  // weights, e.g. 64 -> 64 channels); (4) two CTAs, one box per stage.
  const int tk0 = conv_tk(c.c0, 0);
  const int kpad0 = tk0 * ((c.c0 + tk0 - 1) / tk0);
  int tk = 0, per_sm = 0, nxt = 0;
  auto fits = [&](int t, int ps, int nx, int min_st) {
    const int nc = (c.c0 + t - 1) / t;
    if (t * nc != kpad0) return false;
    const size_t br = ((size_t)c.k * c.k * nc * NT * 2 * t + 1023) / 1024 * 1024;
    const size_t st = (size_t)(BY + nyt - 1) * BX * 2 * t * nx;
    const size_t bud = (size_t)228 * 1024 / ps - 7 * 1024;
    if (br + (size_t)min_st * st > bud) return false;
    tk = t; per_sm = ps; nxt = nx;
    return true;
  };
  if (!fits(tk0, 2, nxt_all, 2) && !(tk0 == 64 && fits(32, 2, nxt_all, 2)) && !fits(tk0, 1, nxt_all, 2) &&
      !fits(tk0, 2, 1, 3))
    return false;
  const int nch = (c.c0 + tk - 1) / tk;
  const size_t bres = (size_t)c.k * c.k * nch * NT * 2 * tk;
  const size_t bres_al = (bres + 1023) / 1024 * 1024;
  const size_t stage = (size_t)(BY + nyt - 1) * BX * 2 * tk * nxt;
  const size_t budget = (size_t)228 * 1024 / per_sm - 7 * 1024;
  const int nst = (int)std::min<size_t>(MAXST, (budget - bres_al) / stage);
  const size_t smem = 1024 + bres_al + (size_t)nst * stage;
  static DeviceOnce once;   // per-device opt-in (kernel attributes hold per device)
  const long long max_dyn = opt_in_dynamic_smem(once, k_conv_tma_reuse);
  if ((long long)smem > max_dyn) return false;
  // input boxes: BX x (BY + nyt - 1) pixels of tk channels, element stride es
  CUtensorMap mA, mB;
  {
    const MapKey key{c.in0, {4 + 16 * tk, c.c0, c.ld0, c.Wi, c.Hi, c.B, BX, BY + nyt - 1, es, 0}};
    if (!cached_map(key, &mA, [&](CUtensorMap* o) {
          return encode_act(o, c.in0, c.c0, c.ld0, c.Wi, c.Hi, c.B, BX, BY + nyt - 1, 1, es, tk);
        }))
      return false;
  }
  const int kpad = tk * nch;
  {
    const int K = c.k * c.k * kpad;
    const MapKey key{c.WP, {1 + 16 * tk, K, c.Cout, NT, 0, 0, 0, 0, 0, 0}};
    if (!cached_map(key, &mB, [&](CUtensorMap* o) { return encode_w(o, c.WP, K, c.Cout, NT, tk); })) return false;
  }
  TmaArgs a{};
  a.B = c.B; a.Ho = c.Ho; a.Wo = c.Wo; a.Cout = c.Cout; a.NT = NT;
  a.k = c.k; a.stride = c.stride; a.pad = c.pad; a.transposed = c.transposed;
  a.BX = BX; a.BY = BY; a.BB = 1;
  a.tx = Wq / BX; a.ty = Hq / BY; a.tb = c.B;
  a.nch0 = nch; a.nch1 = 0; a.bcast1 = 0;
  a.c0 = c.c0; a.c1 = 0;
  a.shuf = c.shuffle; a.cr = c.cr;
  a.ksplit = 1;
  a.nitems = a.tx * a.ty * a.tb * (tr ? 4 : 1);
  a.nst = nst;
  a.colsz = NT <= 32 ? 32 : 64;
  a.nacc = NACC;                                     // 4 x <= 64 columns per CTA, two CTAs per SM
  a.kps = 1;
  a.epig = 1;
  a.kpad = kpad;
  a.tk = tk;
  a.out = c.out; a.ldo = c.ldo; a.bias = c.bias; a.res = c.res; a.ldr = c.ldr;
  a.scale = c.scale; a.shift = c.shift; a.act = c.ep_act; a.ybf = c.ybf; a.ldy = c.ldy;
  a.y2 = c.ybf ? c.y2 : nullptr; a.ldy2 = c.ldy2;
  a.part = nullptr; a.slice = 0;
  a.err = err;
  a.vec = ((c.ldo % 4 == 0) && !((uintptr_t)c.out & 15) && (c.ldy % 8 == 0) && !((uintptr_t)c.ybf & 15) &&
           (!a.y2 || ((c.ldy2 % 8 == 0) && !((uintptr_t)a.y2 & 15))) &&
           (!c.res || ((c.ldr % 8 == 0) && !((uintptr_t)c.res & 15)))) ? 1 : 0;
  ReuseArgs r;
  r.nyt = nyt;
  r.nxt = nxt;
  r.bres = (int)bres;
  const int grid = std::min(a.nitems, sm_count() * per_sm);
  set_fdivs(a);
  launch_pdl(k_conv_tma_reuse, dim3(grid), dim3(NTHR), smem, s, mA, mB, a, r);
  return true;
}

const char* g_tma_reject = "";
const char* conv_tma_last_reject() { return g_tma_reject; }

bool conv_wait_probe(int* err, long long rounds, int arrive, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(err, rounds, arrive);
  return cudaGetLastError() == cudaSuccess;
}

bool conv_forward_tma(const ConvArgs& c, int* err, cudaStream_t s) {
#define TMA_REJECT(why) do { g_tma_reject = why; return false; } while (0)
  if (!c.WP) TMA_REJECT("no padded weights");
  if (c.in_f32 || c.in_act || c.Cout > 256) TMA_REJECT("fp32 or activated input, or Cout > 256");
  if (c.transposed && c.stride != 2) TMA_REJECT("transposed stride");
  if (!c.transposed && c.stride != 1 && c.stride != 2) TMA_REJECT("stride");
  if (c.ld0 % 8 || (c.in1 && c.ld1 % 8)) TMA_REJECT("row stride");   // TMA zero-fills channels past c0 / c1
  if (!get_encoder()) TMA_REJECT("no tensor-map encoder");
  if (launch_reuse(c, err, s)) {
    g_tma_reject = "";
    return true;
  }
  const int Wq = c.transposed ? c.Wo / 2 : c.Wo, Hq = c.transposed ? c.Ho / 2 : c.Ho;
  if (!pow2(Wq) || !pow2(Hq) || (c.transposed && (c.Wo % 2 || c.Ho % 2))) TMA_REJECT("grid not a power of two");
  const int BX = Wq < 128 ? Wq : 128;
  const int BY = Hq < 128 / BX ? Hq : 128 / BX;
  const int BB = 128 / (BX * BY);
  if (c.in1 && c.bcast1 && BB > 1) TMA_REJECT("broadcast source with several images per tile");
  const int es = c.transposed ? 1 : c.stride;
  const int tk = conv_tk(c.c0, c.in1 ? c.c1 : 0);
  CUtensorMap mA0, mA1, mB;
  auto act_map = [&](CUtensorMap* m, const void* p, int C, int ld, int nb) {
    const MapKey key{p, {16 * tk, C, ld, c.Wi, c.Hi, nb, BX, BY, BB, es}};
    return cached_map(key, m,
                      [&](CUtensorMap* o) { return encode_act(o, p, C, ld, c.Wi, c.Hi, nb, BX, BY, BB, es, tk); });
  };
  if (!act_map(&mA0, c.in0, c.c0, c.ld0, c.B)) TMA_REJECT("source 0 map");
  if (c.in1) {
    if (!act_map(&mA1, c.in1, c.c1, c.ld1, c.bcast1 ? 1 : c.B)) TMA_REJECT("source 1 map");
  } else {
    mA1 = mA0;
  }
  TmaArgs a;
  a.B = c.B; a.Ho = c.Ho; a.Wo = c.Wo; a.Cout = c.Cout;
  a.NT = ((c.Cout + 15) / 16) * 16;
  a.k = c.k; a.stride = c.stride; a.pad = c.pad; a.transposed = c.transposed;
  a.BX = BX; a.BY = BY; a.BB = BB;
  a.tx = Wq / BX; a.ty = Hq / BY;
  a.tk = tk;
  a.nch0 = (c.c0 + tk - 1) / tk;
  a.nch1 = c.in1 ? (c.c1 + tk - 1) / tk : 0;
  a.c0 = c.c0;
  a.c1 = c.in1 ? c.c1 : 0;
  a.shuf = c.shuffle; a.cr = c.cr;
  a.bcast1 = (c.in1 && c.bcast1) ? 1 : 0;
  a.ksplit = conv_tma_split(c);
  a.kpad = tk * (a.nch0 + a.nch1);
  {
    const int K = c.k * c.k * a.kpad;
    const MapKey key{c.WP, {1 + 16 * tk, K, c.Cout, a.NT, 0, 0, 0, 0, 0, 0}};
    if (!cached_map(key, &mB, [&](CUtensorMap* o) { return encode_w(o, c.WP, K, c.Cout, a.NT, tk); }))
      TMA_REJECT("weight map");
  }
  a.out = c.out; a.ldo = c.ldo; a.bias = c.bias; a.res = c.res; a.ldr = c.ldr;
  a.scale = c.scale; a.shift = c.shift; a.act = c.ep_act; a.ybf = c.ybf; a.ldy = c.ldy;
  a.y2 = c.ybf ? c.y2 : nullptr; a.ldy2 = c.ldy2;
  a.err = err;
  a.part = a.ksplit > 1 ? c.splitbuf : nullptr;
  // in-kernel split-K fix-up (the last split of a tile adds the slices): measured slower than
  // the finishing launch on the level-3/4 layers (one CTA per tile reads every slice), so off
  a.cnt = (kSplitFixupInKernel && a.ksplit > 1 && c.splitcnt &&
           a.tx * a.ty * a.tb * (c.transposed ? 4 : 1) <= kSplitTickets) ? c.splitcnt : nullptr;
  a.slice = (size_t)c.B * c.Ho * c.Wo * c.Cout;
  a.vec = ((c.ldo % 4 == 0) && !((uintptr_t)c.out & 15) && (c.ldy % 8 == 0) && !((uintptr_t)c.ybf & 15) &&
           (!a.y2 || ((c.ldy2 % 8 == 0) && !((uintptr_t)a.y2 & 15))) &&
           (!c.res || ((c.ldr % 8 == 0) && !((uintptr_t)c.res & 15))) &&
           (!a.part || (c.Cout % 4 == 0 && !((uintptr_t)a.part & 15)))) ? 1 : 0;
  const int nph = c.transposed ? 4 : 1;
  a.tb = (c.B + BB - 1) / BB;
  a.nitems = a.tx * a.ty * a.tb * nph * a.ksplit;
  a.colsz = a.NT <= 32 ? 32 : (a.NT <= 64 ? 64 : (a.NT <= 128 ? 128 : 256));
  // accumulator buffers within the 512 TMEM columns of the SM's CTAs
  a.nacc = NACC * a.colsz * ctas_per_sm(a.NT) <= 512 ? NACC : 2;
  // narrow tiles drain two at a time (measured faster up to 64 columns, slower at 256)
  a.epig = a.NT <= 64 ? 1 : 0;
  // stage ring sized to the shared memory left per CTA (228 KB per SM; per CTA 1 KB
  // reserved, 4 KB of static barriers and epilogue constants, 1 KB alignment slack, 1 KB
  // margin): 4-8 stages
  const int per_sm = ctas_per_sm(a.NT);
  const size_t kbytes = ((size_t)TM + a.NT) * 2 * tk;
  const size_t budget = (size_t)228 * 1024 / per_sm - 7 * 1024;
  // K-blocks per stage when every chunk is full (the MMA thread then issues them as one
  // block behind one wait and one commit): as many (up to 3) as leave three stages
  a.kps = 1;
  if (c.c0 % tk == 0 && (!c.in1 || c.c1 % tk == 0))
    for (int k = 3; k >= 2; --k)
      if (budget / (kbytes * k) >= 3) { a.kps = k; break; }
  const size_t stage = kbytes * a.kps;
  a.nst = (int)std::min<size_t>(MAXST, budget / stage);
  if (a.nst < 2) TMA_REJECT("shared memory");
  const size_t smem = (size_t)a.nst * stage + 1024;
  // dynamic shared memory opt-in: the per-block limit less the kernel's static barriers
  static DeviceOnce once;   // per-device opt-in (kernel attributes hold per device)
  static DeviceOnce once_g;
  const long long max_dyn = a.kps > 1 ? opt_in_dynamic_smem(once_g, k_conv_tma<true>)
                                      : opt_in_dynamic_smem(once, k_conv_tma<false>);
  if ((long long)smem > max_dyn) TMA_REJECT("shared memory");
  const int grid = std::min(a.nitems, sm_count() * per_sm);
  set_fdivs(a);
  if (a.kps > 1) launch_pdl(k_conv_tma<true>, dim3(grid), dim3(NTHR), smem, s, mA0, mA1, mB, a);
  else launch_pdl(k_conv_tma<false>, dim3(grid), dim3(NTHR), smem, s, mA0, mA1, mB, a);
  if (a.ksplit > 1 && !a.cnt) {
    const int M = c.B * c.Ho * c.Wo;
    const size_t n4 = (size_t)M * (c.Cout / 4);
    launch_pdl(k_splitk_finish, dim3((unsigned)std::min<size_t>((n4 + 255) / 256, (size_t)sm_count() * 8)), dim3(256),
               0, s, a, M);
  }
  g_tma_reject = "";
  return true;
#undef TMA_REJECT
}

// ===========================================================================
// Weight gradients on the tensor cores:
//   dW[tap][ci][co] = sum over pixels p of X_tap(p)[ci] * G(p)[co]
// as a GEMM with M = 128 input channels, N = Cout (padded to 64), K = 64-pixel
// blocks.  Both operands come from the NHWC tensors as TMA boxes {64 channels,
// 64 pixels}, i.e. MN-major (channels contiguous) in shared memory; the tap's
// offset, the stride and the transposed convolution's output parity are box
// coordinates and element strides on the pixel dimensions.  Items (tap, channel
// block, pixel chunk) run on a persistent grid; each adds its FP32 tile into dW
// with vector atomics.
// ===========================================================================
namespace {

constexpr int WG_THR = 192;   // warps 0-3 epilogue, 4 TMA, 5 MMA

struct WgArgs {
  int k, pad, kind;           // kind 0: 5x5 stride 2, 1: stride 1, 2: transposed stride 2
  int B, tx, ty, bx, by;      // K grid: tx * ty blocks of bx x by pixels per image
  int cin, cout, mblk, NT;    // 128-channel blocks of cin; N = Cout padded to 64
  int cin_tot;                // input channels of the whole layer (rows of one tap in gW)
  int nchunks, nitems, nst, colsz;
  uint32_t lbo, sbo;          // MN-major descriptor strides (bytes)
  int vec;                    // gW rows 16-byte aligned (float4 atomics)
  float* gW;
  // deterministic sums: item (tap, block, chunk) stores its tile to part + chunk * pstride
  // ([tap][cin][cout]) and a second launch adds the chunks in order; null: vector atomics
  float* part;
  size_t pstride;
  int* err;
};

__device__ __forceinline__ uint64_t desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}
// kind::f16, FP32 accumulate, BF16 A and B, both MN-major (transpose bits 15, 16)
__host__ __device__ constexpr uint32_t idesc_mn(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

struct WgItem { int tap, mb, kb0, nkb, chunk; };

__device__ __forceinline__ WgItem wg_decode(const WgArgs& a, int w) {
  WgItem it;
  const int chunk = w % a.nchunks, r = w / a.nchunks;
  it.mb = r % a.mblk;
  it.tap = r / a.mblk;
  const int KB = a.B * a.tx * a.ty;
  it.kb0 = (int)((long long)chunk * KB / a.nchunks);
  it.nkb = (int)((long long)(chunk + 1) * KB / a.nchunks) - it.kb0;
  it.chunk = chunk;
  return it;
}

__global__ void __launch_bounds__(WG_THR, 1) k_wgrad_tma(const __grid_constant__ CUtensorMap mX,
                                                         const __grid_constant__ CUtensorMap mG, WgArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[MAXST], empty[MAXST], tfull[2], tempty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int N = a.NT, NS = a.nst;
  const uint32_t base = (su32(smem) + 1023u) & ~1023u;
  const uint32_t a_bytes = 2 * 8192, b_bytes = (uint32_t)(N / 64) * 8192, stage = a_bytes + b_bytes;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) { mb_init(su32(&full[s]), 1); mb_init(su32(&empty[s]), 1); }
    for (int q = 0; q < 2; ++q) { mb_init(su32(&tfull[q]), 1); mb_init(su32(&tempty[q]), 4); }
    mb_init(su32(&drain), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  const uint32_t ncols = 2u * (uint32_t)a.colsz;
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
  volatile int* fail = &s_fail;
  const int kbi = a.tx * a.ty;   // K-blocks per image

  if (warp == 4) {
    if (lane == 0) {
      uint32_t g = 0;
      for (int w = blockIdx.x; w < a.nitems && !failed(fail); w += gridDim.x) {
        const WgItem it = wg_decode(a, w);
        const int ky = it.tap / a.k, kx = it.tap - ky * a.k;
        bool ok = true;
        for (int kb = 0; kb < it.nkb; ++kb, ++g) {
          const int s = (int)(g % (uint32_t)NS);
          const uint32_t use = g / (uint32_t)NS;
          if (g >= (uint32_t)NS && !mb_wait(su32(&empty[s]), (use - 1) & 1u)) { ok = false; break; }
          const int kg = it.kb0 + kb;
          const int b = kg / kbi, r = kg - b * kbi, tyi = r / a.tx, txi = r - tyi * a.tx;
          const int x0 = txi * a.bx, y0 = tyi * a.by;
          int xx, xy, gx, gy;   // box origins of X and G (TMA coordinates of the pixel dims)
          if (a.kind == 1) { xx = x0 + kx - a.pad; xy = y0 + ky - a.pad; gx = x0; gy = y0; }
          else if (a.kind == 0) { xx = 2 * x0 + kx - a.pad; xy = 2 * y0 + ky - a.pad; gx = x0; gy = y0; }
          else { xx = x0; xy = y0; gx = 2 * x0 + kx - a.pad; gy = 2 * y0 + ky - a.pad; }
          const uint32_t sA = base + (uint32_t)s * stage, sB = sA + a_bytes;
          mb_expect_tx(su32(&full[s]), stage);
          tma_load_4d(sA, &mX, it.mb * 128, xx, xy, b, su32(&full[s]));
          tma_load_4d(sA + 8192, &mX, it.mb * 128 + 64, xx, xy, b, su32(&full[s]));
          for (int nb = 0; nb < N / 64; ++nb) tma_load_4d(sB + nb * 8192, &mG, nb * 64, gx, gy, b, su32(&full[s]));
        }
        if (!ok) { atomicExch(&s_fail, 1); break; }
      }
      for (uint32_t j = g > (uint32_t)NS ? g - (uint32_t)NS : 0u; j < g; ++j)
        mb_wait(su32(&full[j % (uint32_t)NS]), (j / (uint32_t)NS) & 1u);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t id = idesc_mn(128, N);
      uint32_t g = 0;
      int li = 0;
      for (int w = blockIdx.x; w < a.nitems && !failed(fail); w += gridDim.x, ++li) {
        const WgItem it = wg_decode(a, w);
        const int acc = li & 1;
        if (li >= 2 && !mb_wait(su32(&tempty[acc]), (uint32_t)((li >> 1) - 1) & 1u)) { atomicExch(&s_fail, 1); break; }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(acc * a.colsz);
        bool ok = true;
        for (int kb = 0; kb < it.nkb; ++kb, ++g) {
          const int s = (int)(g % (uint32_t)NS);
          if (!mb_wait(su32(&full[s]), (g / (uint32_t)NS) & 1u)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t sA = base + (uint32_t)s * stage, sB = sA + a_bytes;
#pragma unroll
          for (int k4 = 0; k4 < 4; ++k4) {   // 16 pixels (two 8-row groups) per MMA
            const uint64_t da = desc_mn(sA + (uint32_t)k4 * 2048u, a.lbo, a.sbo);
            const uint64_t db = desc_mn(sB + (uint32_t)k4 * 2048u, a.lbo, a.sbo);
            const uint32_t accum = (kb > 0 || k4 > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                "l"(da), "l"(db), "r"(id), "r"(accum)
                : "memory");
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           su32(&empty[s]))
                       : "memory");
        }
        if (!ok) { atomicExch(&s_fail, 1); break; }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         su32(&tfull[acc]))
                     : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&drain))
                   : "memory");
      mb_wait(su32(&drain), 0);
    }
  } else {
    // epilogue: row m = input channel mb * 128 + m, columns = output channels
    int li = 0;
    for (int w = blockIdx.x; w < a.nitems; w += gridDim.x, ++li) {
      if (failed(fail)) break;
      const WgItem it = wg_decode(a, w);
      const int acc = li & 1;
      if (!mb_wait_sleep(su32(&tfull[acc]), (uint32_t)(li >> 1) & 1u)) { atomicExch(&s_fail, 1); break; }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int ci = it.mb * 128 + warp * 32 + lane;
      float* row = a.gW + ((size_t)it.tap * a.cin_tot + ci) * a.cout;
      const bool vec = a.vec != 0;
      for (int c0 = 0; c0 < N && c0 < a.cout; c0 += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * a.colsz + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (ci >= a.cin) continue;
        if (a.part) {
          // this chunk's tile, plain stores (zero when the chunk holds no K-blocks)
          float* prow = a.part + (size_t)it.chunk * a.pstride + ((size_t)it.tap * a.cin + ci) * a.cout;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < a.cout) prow[c0 + j] = it.nkb > 0 ? __uint_as_float(v[j]) : 0.f;
          continue;
        }
        if (it.nkb <= 0) continue;
        if (vec && c0 + 16 <= a.cout) {
          float4* op = reinterpret_cast<float4*>(row + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            atomicAdd(op + q, make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                          __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3])));
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < a.cout) atomicAdd(row + c0 + j, __uint_as_float(v[j]));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(&tempty[acc])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (tid == 0 && s_fail && a.err) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// gW[(tap * cin_tot + ci) * cout + co] += sum over chunks c = 0, 1, ... (in this order) of
// part[c * pstride + (tap * cin + ci) * cout + co].
__global__ void k_wgrad_reduce(const float* __restrict__ part, size_t pstride, int nchunks, int taps, int cin,
                               int cout, int cin_tot, float* __restrict__ gW) {
  const size_t n = (size_t)taps * cin * cout;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float t = 0.f;
    for (int c = 0; c < nchunks; ++c) t += part[(size_t)c * pstride + e];
    const size_t tap = e / ((size_t)cin * cout), r = e - tap * cin * cout;
    gW[(tap * cin_tot) * cout + r] += t;
  }
}

// MN-major descriptor strides: (LBO, SBO) = (channel-atom stride, 8-pixel-group stride)
// when wg_desc_order == 0, swapped otherwise.
int g_wg_desc_order = 0;

}  // namespace

void conv_wgrad_tma_set_desc_order(int order) { g_wg_desc_order = order; }

// dW += weight gradient of the forward convolution c (single BF16 source, no on-load
// activation) from g = dL/dy (BF16 [pixels][Cout], ld ldg).  False: not eligible.
bool conv_wgrad_tma(const ConvArgs& c, const __nv_bfloat16* g, int ldg, float* gW, int* err, cudaStream_t s,
                    int cin_total, bool launch, float* scratch, size_t scratch_cap) {
  if (c.in1 || c.in_act || c.in_f32 || c.Cout > 256 || c.ld0 % 8 || ldg % 8) return false;
  if (c.k != 3 && c.k != 5) return false;
  if (!get_encoder()) return false;
  const int kind = c.transposed ? 2 : (c.stride == 2 ? 0 : 1);
  if (kind == 1 && c.stride != 1) return false;
  // K grid: output pixels (kinds 0, 1) or input pixels (transposed)
  const int Wk = kind == 2 ? c.Wi : c.Wo, Hk = kind == 2 ? c.Hi : c.Ho;
  if (!pow2(Wk) || !pow2(Hk) || Wk * Hk < 64) return false;
  if (kind == 2 && (c.Wo != 2 * c.Wi || c.Ho != 2 * c.Hi)) return false;
  WgArgs a;
  a.k = c.k; a.pad = c.pad; a.kind = kind; a.B = c.B;
  a.bx = Wk < 64 ? Wk : 64;
  a.by = 64 / a.bx;
  a.tx = Wk / a.bx; a.ty = Hk / a.by;
  a.cin = c.c0; a.cout = c.Cout;
  a.cin_tot = cin_total > 0 ? cin_total : c.c0;
  a.mblk = (c.c0 + 127) / 128;
  a.NT = 64 * ((c.Cout + 63) / 64);
  a.colsz = a.NT <= 64 ? 64 : (a.NT <= 128 ? 128 : 256);
  const int taps = c.k * c.k;
  const int KB = c.B * a.tx * a.ty;
  const int per_sm = a.NT <= 64 ? 2 : 1;
  const int slots = sm_count() * per_sm;
  int nch = (2 * slots + taps * a.mblk - 1) / (taps * a.mblk);
  nch = std::max(1, std::min(nch, KB / 8 > 0 ? KB / 8 : 1));
  a.nchunks = nch;
  a.nitems = taps * a.mblk * nch;
  a.lbo = g_wg_desc_order == 0 ? 8192u : 1024u;
  a.sbo = g_wg_desc_order == 0 ? 1024u : 8192u;
  a.gW = gW;
  a.err = err;
  a.vec = (c.Cout % 4 == 0 && !((uintptr_t)gW & 15)) ? 1 : 0;
  // the ring, 1 KB alignment slack and 16 KB past the last stage (descriptor strides
  // reach at most 16 KB beyond a stage's start whichever field carries which stride)
  const size_t stage = 2 * 8192 + (size_t)(a.NT / 64) * 8192;
  const size_t budget = (size_t)228 * 1024 / per_sm - 21 * 1024;
  a.nst = (int)std::min<size_t>(MAXST, budget / stage);
  if (a.nst < 2) return false;
  const size_t smem = (size_t)a.nst * stage + 1024 + 16 * 1024;
  static DeviceOnce once;   // per-device opt-in (kernel attributes hold per device)
  const long long max_dyn = opt_in_dynamic_smem(once, k_wgrad_tma);
  if ((long long)smem > max_dyn) return false;
  // X: box {64 channels, bx (x es), by (x es), 1}; G likewise (element stride 2 on G for
  // transposed convolutions, on X for stride-2 ones)
  const int ex = kind == 0 ? 2 : 1, eg = kind == 2 ? 2 : 1;
  CUtensorMap mX, mG;
  {
    const MapKey key{c.in0, {2, c.c0, c.ld0, c.Wi, c.Hi, c.B, a.bx, a.by, ex, 0}};
    if (!cached_map(key, &mX, [&](CUtensorMap* o) {
          return encode_act(o, c.in0, c.c0, c.ld0, c.Wi, c.Hi, c.B, a.bx, a.by, 1, ex, 64);
        }))
      return false;
  }
  {
    const MapKey key{g, {3, c.Cout, ldg, c.Wo, c.Ho, c.B, a.bx, a.by, eg, 0}};
    if (!cached_map(key, &mG, [&](CUtensorMap* o) {
          return encode_act(o, g, c.Cout, ldg, c.Wo, c.Ho, c.B, a.bx, a.by, 1, eg, 64);
        }))
      return false;
  }
  if (!launch) return true;
  // deterministic sums when the scratch holds every chunk's tiles
  const size_t pstride = (size_t)taps * c.c0 * c.Cout;
  a.part = scratch && (size_t)a.nchunks * pstride <= scratch_cap ? scratch : nullptr;
  a.pstride = pstride;
  const int grid = std::min(a.nitems, slots);
  k_wgrad_tma<<<grid, WG_THR, smem, s>>>(mX, mG, a);
  if (a.part) {
    const int rb = (int)std::min<size_t>((pstride + 255) / 256, (size_t)sm_count() * 8);
    k_wgrad_reduce<<<rb, 256, 0, s>>>(a.part, pstride, a.nchunks, taps, c.c0, c.Cout, a.cin_tot, gW);
  }
  return true;
}

}  // namespace helm
