// Internal declarations of the U-Net kernels (unet_kernels.cu) used by the
// network executor (unet.cu).  Not part of the ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstddef>

namespace helm {

constexpr float kBnEps = 1e-5f;
constexpr float kBnMomentum = 0.1f;

// One convolution as an implicit GEMM: rows = output pixels, columns = output
// channels, reduction over taps x input channels.  The input is the channel
// concatenation of two sources (in1 may be null); in_f32 selects FP32 sources
// (gradients) instead of BF16 (activations); in_act applies eLU on load.
// Weight element (tap, ci, co) sits at W[tap * wst + ci * wsk + co * wsn].
struct ConvArgs {
  const void* in0; int c0, ld0;
  const void* in1; int c1, ld1;
  int bcast1;                        // in1 is one image shared by the whole batch
  int in_f32, in_act;
  int B, Hi, Wi, Ho, Wo, Cout;
  int k, stride, pad, transposed;
  const __nv_bfloat16* W; long long wst, wsk, wsn;
  const __nv_bfloat16* WT;           // K-major copy [cout][tap * cin + ci] for the tensor-core path, or null
  const __nv_bfloat16* WP;           // padded K-major copy [cout][tap][64-channel chunks] for the TMA path, or null
  float* out; int ldo;
  const float* bias;                 // per output channel, may be null
  const __nv_bfloat16* res; int ldr; // residual added to the output, may be null
  // fused inference BatchNorm epilogue (tensor-core path only): y = act((conv + res) * scale + shift)
  const float* scale; const float* shift; int ep_act;
  __nv_bfloat16* ybf; int ldy;       // BF16 destination; when set, `out` is not written
  __nv_bfloat16* y2; int ldy2;       // optional second BF16 destination: eLU of what ybf receives (TMA path)
  // split-K scratch of the TMA path: splitcnt_n floats for the FP32 partial-sum slices
  // (null: not split)
  float* splitbuf; int* splitcnt; long long splitcnt_n;   // splitcnt: kSplitTickets zeroed tickets
  // sub-pixel form of a transposed 5x5 stride-2 convolution (TMA path): the weights
  // [4 cout][3x3][chunks]; with shuffle = 1 the arguments describe the 3x3 convolution
  // over the input grid with Cout = 4 cr columns scattered to the 2x output
  const __nv_bfloat16* WS; int shuffle, cr;
};

void conv_forward(const ConvArgs& a, cudaStream_t s);
// CUDA-core direct convolutions (conv_small.cu) for the 5x5 stride-2 layer from <= 8
// input channels and the transposed 5x5 stride-2 layer to <= 4 outputs.
bool conv_small_eligible(const ConvArgs& a);
bool conv_forward_small(const ConvArgs& a, cudaStream_t s);
// Tensor-core path (conv_tc.cu): eligible when inputs are BF16 without on-load
// activation, channel counts are multiples of 8, Cout a multiple of 16 (<= 256).
bool conv_tc_eligible(const ConvArgs& a);
void conv_forward_tc(const ConvArgs& a, int* err, cudaStream_t s);
void weights_kmajor(const float* P, __nv_bfloat16* WT, int taps, int cin, int cout, cudaStream_t s);
// TMA-fed tensor-core path (conv_tma.cu); false if the convolution does not fit it.
// Tickets of the split-K fix-up (one per output tile and phase of a launch).
constexpr int kSplitTickets = 4096;
bool conv_forward_tma(const ConvArgs& a, int* err, cudaStream_t s);
// One-thread kernel that waits on an mbarrier through the convolution pipeline's bounded
// wait (at most `rounds` polls); without an arrival the wait expires and err records it.
bool conv_wait_probe(int* err, long long rounds, int arrive, cudaStream_t s);
int conv_tma_split(const ConvArgs& a);
// adjoint (data-gradient) weight copies for the TMA path: [cin][tap][64-chunks of cout],
// taps reversed for stride-1 convolutions
size_t conv_tma_weight_adj_elems(int k, int cin, int cout);
size_t conv_tma_weight_s2d_elems(int cout);
// Space-to-depth copy WD of a 5x5 stride-2 input convolution from cin <= 4 channels:
// 3x3 stride-1 taps over 2x2 input blocks of 4 * cin channels (K padded to 64).
void conv_tma_weights_s2d_in(const float* P, __nv_bfloat16* WD, int cin, int cout, cudaStream_t s);
size_t conv_tma_weight_sub_elems(int c0, int c1, int cout);
void conv_tma_weights_subpixel(const float* P, __nv_bfloat16* WS, int c0, int c1, int cout, cudaStream_t s);
// weight gradient on the tensor cores (TMA path): gW += dW of the forward convolution a
// (one BF16 source, no on-load activation) from g = dL/dy, BF16 [pixels][Cout] with ld ldg
// Weight gradient of source 0 of a (a.in1 must be null) added into gW on the tensor cores;
// cin_total: input channels of the whole layer (rows of one tap in gW; 0: a.c0), so that a
// second source's gradient can start at gW + c0 * Cout.  launch = false only checks that the
// layer qualifies.  Returns false (nothing launched) when it does not.  scratch (capacity
// scratch_cap floats): when it holds every pixel chunk's tile, the chunks are summed in a
// fixed order by a second launch (bit-reproducible gradients); else with atomics.
bool conv_wgrad_tma(const ConvArgs& a, const __nv_bfloat16* g, int ldg, float* gW, int* err, cudaStream_t s,
                    int cin_total = 0, bool launch = true, float* scratch = nullptr, size_t scratch_cap = 0);
void conv_wgrad_tma_set_desc_order(int order);
void conv_tma_weights_adjoint(const float* P, __nv_bfloat16* WPA, int k, int cin, int cout, bool flip, cudaStream_t s);
const char* conv_tma_last_reject();      // why the last conv_forward_tma call declined ("" if it launched)   // > 1: the TMA path splits K (FP32 atomics, no fused epilogue)
size_t conv_tma_weight_elems(int k, int c0, int c1, int cout);
void conv_tma_weights(const float* P, __nv_bfloat16* WP, int k, int c0, int c1, int cout, cudaStream_t s);
void elu_copy_bf16(const __nv_bfloat16* src, int lds, int C, size_t M, __nv_bfloat16* dst, int ldd, cudaStream_t s);
void conv_wgrad(const ConvArgs& a, const float* G, int ldg, float* gW, cudaStream_t s);
void bn_batch_stats(const float* z, int ldz, int C, int M, double* mean, double* var, float* part, int nblk,
                    cudaStream_t s);
void bn_coeffs(const double* mean, const double* var, const float* gamma, const float* beta, int C, float* scale,
               float* shift, float* rmean, float* rvar, bool update, int M, cudaStream_t s);
void bn_coeffs_eval(const float* rmean, const float* rvar, const float* gamma, const float* beta, int C,
                    float* scale, float* shift, cudaStream_t s);
void bn_act(const float* z, int ldz, int C, int M, const float* scale, const float* shift, bool act,
            __nv_bfloat16* y, int ldy, cudaStream_t s);
void bn_backward(const float* g, int ldg, const float* z, int ldz, int C, int M, const double* mean, const double* var,
                 const float* scale, const float* shift, bool act, const float* gamma, float* ggamma, float* gbeta,
                 float* part, int nblk, float* coef, float* gz, int ldo, cudaStream_t s);
// g *= eLU'(u); plane != 0: u is one image of `plane` pixels shared by the batch.
void elu_backward_inplace(float* g, int ldg, const __nv_bfloat16* u, int ldu, int C, int M, size_t plane,
                          cudaStream_t s);
void add_slice(float* dst, int ldd, const float* src, int lds, int C, int M, cudaStream_t s);
void to_bf16_slice(const float* src, int lds, __nv_bfloat16* dst, int ldd, int C, int M, cudaStream_t s);
void mse_loss(const float* out, const float* tgt, size_t n, int B, float* gout, float* part, float* loss,
              cudaStream_t s);
// Residual loss sum |h^2 A y - x_r|^2 / B and its gradient (float2 outputs y, inputs x with
// 4 channels); rho: scratch of B*ny*nx float2; part: 256 floats; c = h^2 omega^2; bc the
// boundary mode (0 zero, 1 reflection, 2 replication padding; 1 needs nx, ny >= 2).
void residual_loss(const float* y, const float* x, int B, int ny, int nx, float c, const float* k2, const float* gam,
                   int bc, float* rho, float* gout, float* part, float* loss, cudaStream_t s);
void adam_update(float* p, const float* g, float* m1, float* m2, size_t n, float lr, float b1, float b2, float eps,
                 int t, cudaStream_t s);
void f32_to_bf16(const float* src, __nv_bfloat16* dst, size_t n, cudaStream_t s);
// Network input (Sec. 3.4): Re r, Im r divided by rms(r), kappa^2, gamma; s2d: into the
// space-to-depth layout [b][y/2][x/2][2x2 block][4] (ny, nx even), else ldx-channel pixels.
void make_input(const void* r, bool fp64, int B, int ny, int nx, double h, const float* k2, const float* gam,
                __nv_bfloat16* x, int ldx, float* sc, float* part, const int* gate, cudaStream_t s, bool s2d, int rpp = 0,
                int b0 = 0);
// FP32 4-channel pixels [M][lds] into the space-to-depth BF16 layout, and that layout back to
// ldd-channel pixels (channels past 4 zeroed).
void to_bf16_s2d(const float* src, int lds, __nv_bfloat16* dst, int B, int ny, int nx, cudaStream_t s);
void s2d_to_std(const __nv_bfloat16* xs, __nv_bfloat16* dst, int ldd, int B, int ny, int nx, cudaStream_t s);
void write_output(const float* out, bool fp64, int B, int ny, int nx, const float* sc, void* e, bool add,
                  const int* gate, cudaStream_t s);
void gamma_field(int ny, int nx, int width, float gmax, float* g, cudaStream_t s);
void chan_sum_add(const float* g, int ld, int C, int M, float* dst, float* part, int nblk, cudaStream_t s);
void batch_sum(const float* src, int lds, int B, size_t P, int C, float* dst, int ldd, bool accumulate,
               cudaStream_t s);
void complex_normal(unsigned long long seed, int count, size_t N, double2* x, cudaStream_t s);
void make_batch(const double2* r, const double2* e, size_t N, int count, const int* idx, const double2* coef, int nmix,
                double h, const float* k2, const float* gam, float* x, float* tgt, cudaStream_t s);

}  // namespace helm
