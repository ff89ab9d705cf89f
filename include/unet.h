/*
 * U-Net preconditioners of libhelm (Azulay & Treister, arXiv 2203.11025,
 * Sec. 3): the network itself, its training (MSE loss of Eq. 3.7, Adam), the
 * encoder-solver pair (Sec. 3.3) and the preconditioners M_JU (Alg. 2) and
 * M_VU (Eq. 3.4).
 *
 * Network (Sec. 3.1): down levels x_l = eLU(BN(R_l x_{l-1})) with R_l a 5x5
 * stride-2 convolution doubling the channels (Eq. 3.1), a ResNet block
 * eLU(BN(x + K2 eLU(BN(K1 x)))) per level and `coarse_resnets` at the coarsest
 * (Eq. 3.2); up levels u <- cat(BN(P_l eLU(u)), x_{l-1}) with P_l a 5x5
 * stride-2 transposed convolution (Eq. 3.3); the last up layer maps to
 * out_ch channels with a bias.  Channel widths are configurable (the paper's
 * figure with them is lost; default 32, 64, 128, 256).
 *
 * Conventions: activations NHWC float32 at this boundary ([B][ny][nx][ch]),
 * BF16 inside with FP32 accumulation; parameters travel as one flat float32
 * HOST array: every convolution weight in layer order as [ky][kx][cin][cout],
 * then the output bias, then (gamma, beta) of every BatchNorm in layer order.
 * Layer order: down1, res1.0.k1, res1.0.k2, down2, ..., downL, resL.0.k1, ...,
 * upL, ..., up2, up1; BatchNorms: down1.bn, res1.0.bn1, res1.0.bn2, ..., upL.bn,
 * ..., up2.bn.  Return codes and helm_last_error() as in helm.h.
 */
#ifndef HELM_UNET_H
#define HELM_UNET_H

#include "helm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct unet_ctx* unet_t;

typedef struct {
  int in_ch;               /* 4 for a solver (Re r, Im r, kappa^2, gamma), 2 for an encoder */
  int out_ch;              /* 2 for a solver (Re e, Im e); encoder: channels of f^(0)       */
  int levels;              /* down/up levels (default 4)                                    */
  int coarse_resnets;      /* ResNet blocks at the coarsest level (Sec. 3.1: 3)             */
  int widths[8];           /* channels per level (default 32, 64, 128, 256)                 */
  int context[9];          /* solver with encoder: channels of f^(0..levels), else all 0    */
  int flags;               /* UNET_FLAG_*                                                   */
} unet_cfg;
/* Implementation switches (cross-checking; same arithmetic up to summation order):
 * UNET_FLAG_SIMT runs every convolution on CUDA cores (FP32 FMA); UNET_FLAG_NO_TMA
 * keeps the tcgen05 kernel but stages operands with cp.async instead of TMA. */
enum { UNET_FLAG_SIMT = 1, UNET_FLAG_NO_TMA = 2 };

enum { UNET_STANDALONE = 0, UNET_ENCODER = 1, UNET_SOLVER = 2 };

/* Defaults of the given kind: the U-Net of Sec. 3.1 (Eq. 3.1-3.3; 4 levels, 32-256
 * channels, 3 ResNet blocks at the coarsest level), the encoder of Sec. 3.3, or the solver
 * with context channels (Eq. 3.5; `context` filled for the default encoder).  HELM_EINVAL
 * for a NULL cfg; a kind other than UNET_ENCODER or UNET_SOLVER gives the standalone net. */
int unet_cfg_default(unet_cfg* cfg, int kind);
/* Create the network of cfg (Sec. 3.1; Eq. 3.5 with context channels) with He-normal
 * weights drawn from `seed` (SplitMix64 + Box-Muller; the paper gives no initialisation),
 * BN gamma 1, beta 0, running mean 0, var 1.  The handle owns its device memory; free it
 * with unet_destroy.  HELM_EINVAL for a bad cfg; an error code (message in
 * helm_last_error) if a device allocation fails. */
int unet_create(const unet_cfg* cfg, unsigned long long seed, unet_t* out);
void unet_destroy(unet_t net);
/* Network state (no counterpart in the paper: access for checkpoints and tests).  Sizes
 * of the flat FP32 parameter vector (convolution weights [ky][kx][cin][cout] layer by layer,
 * the output bias, then BN gamma/beta per layer) and of the BN running-stat vector (means
 * then variances).  set/get copy between that layout and caller-owned HOST arrays of exactly
 * n elements (HELM_EINVAL otherwise); set also refreshes the BF16 working copies.  The
 * copies are synchronous. */
int unet_sizes(unet_t net, long long* n_params, long long* n_bn);
int unet_set_params(unet_t net, const float* host, long long n);
int unet_get_params(unet_t net, float* host, long long n);
int unet_set_bn_stats(unet_t net, const float* host, long long n);
int unet_get_bn_stats(unet_t net, float* host, long long n);
/* Failure detection (no counterpart in the paper): synchronise and report a failure
 * recorded by a tensor-core kernel (a bounded wait that expired): *failed = 0 if none.
 * Clears the record. */
int unet_status(unet_t net, int* failed);
/* Failure-detection probe (no counterpart in the paper; for tests): one GPU thread waits,
 * through the same bounded mbarrier wait the tensor-core kernels use, on a barrier that
 * expects one arrival.  arrive = 0: nothing arrives, the wait gives up after `rounds`
 * polls (1 <= rounds <= 2^20, well under a second) and records the failure that
 * unet_status then reports; arrive = 1: the thread arrives first and nothing is recorded.
 * The kernel returns either way; the context stays usable.  Asynchronous on `stream`. */
int unet_wait_probe(unet_t net, long long rounds, int arrive, helm_stream_t stream);
/* Parameter gradients of the training loss (Sec. 3.4, Eq. 3.7) accumulated since the last
 * unet_zero_grad, in the flat parameter layout, into a HOST array of n elements. */
int unet_get_grads(unet_t net, float* host, long long n);
int unet_zero_grad(unet_t net, helm_stream_t stream);

/* Forward pass (Eq. 3.1-3.3; Eq. 3.5 for a solver with context) on x (device float32
 * [B][ny][nx][in_ch]) into out (device float32
 * [B][ny][nx][out_ch]).  train != 0 uses batch statistics, updates the running
 * statistics and keeps what unet_backward needs.  A solver with context reads
 * the features of its attached encoder's last forward (unet_attach_encoder).
 * ny, nx must be multiples of 2^levels; B*ny*nx*2*widths[0] must stay below 2^31
 * (HELM_EUNSUPPORTED otherwise, also from unet_precond and the U-Net preconditioned
 * solves). */
int unet_forward(unet_t net, const float* x, float* out, int B, int ny, int nx, int train, helm_stream_t stream);
/* Backward of the last train-mode forward (the gradients of Sec. 3.4's training) for the
 * loss sum(gout * out): adds
 * parameter gradients; writes d loss / d x into gx if not null (device float32
 * like x).  A solver with an attached encoder also back-propagates into the
 * encoder (whose own last forward must be train-mode). */
int unet_backward(unet_t net, const float* gout, float* gx, helm_stream_t stream);
/* MSE loss of Eq. 3.7 between out and target (device float32, n elements, B
 * samples): writes gout = d loss / d out (device) and the loss into *loss_dev. */
int unet_mse(const float* out, const float* target, long long n, int B, float* gout, float* loss_dev,
             helm_stream_t stream);
/* One training step (Sec. 3.4; the paper trains with Adam on the loss of Eq. 3.7): with an
 * attached encoder, the encoder's train-mode forward on the medium of h (the pair is
 * trained jointly); then zeroed gradients, the train-mode forward on x (device float32
 * [B][ny][nx][in_ch], h's fine grid, e.g. from unet_make_batch), the loss, the backward
 * pass and one Adam step on every parameter.  opt->loss selects the MSE of Eq. 3.7 against
 * target (device float32 [B][ny][nx][out_ch]) or the unsupervised residual loss of the
 * Remark following Eq. 3.7 (target unused, may be NULL).  The loss value goes to
 * loss_dev (device float, nullable).  Asynchronous on `stream`; the network keeps the
 * output-gradient buffer it needs (allocated on the first call of a size). */
enum { UNET_LOSS_MSE = 0, UNET_LOSS_RESIDUAL = 1 };
typedef struct {
  float lr, beta1, beta2, eps;   /* Adam: learning rate (Sec. 4: 1e-4), moment decays, epsilon */
  int loss;                      /* UNET_LOSS_MSE or UNET_LOSS_RESIDUAL                       */
} unet_train_opts;
int unet_train_step(unet_t net, helm_t h, const float* x, const float* target, int B, const unet_train_opts* opt,
                    float* loss_dev, helm_stream_t stream);

/* Network checkpoints (no counterpart in the paper: persistence of the trained state).
 * unet_save writes the FP32 master weights and the BatchNorm running statistics of net
 * (device state, read back synchronously) to the file `path`: 8-byte magic "HLMUNET1",
 * uint32 header length, a JSON header {"cfg": the unet_cfg fields, "crc32": CRC-32 of the
 * payload, "meta": meta_json (one JSON object, NULL for {}), "n_bn", "n_params",
 * "version": 1}, zero padding to 16 bytes, then float32 weights (flat order above) and
 * float32 BN means and variances.  unet_load restores such a file into net, which must
 * have the same configuration; a bad magic, version, size, CRC or configuration is
 * HELM_EINVAL with a message, and net is then unchanged.  Adam moments are not stored. */
int unet_save(unet_t net, const char* path, const char* meta_json);
int unet_load(unet_t net, const char* path);

/* Unsupervised residual loss (the Remark following Eq. 3.7) on the medium of h: with
 * the network output y (device float32 [B][ny][nx][2], units e / s) and its input x
 * (device float32 [B][ny][nx][4] as unet_make_batch writes it, channels 0, 1 = h^2 r / s),
 *   rho = h^2 A (y0 + i y1) - (x0 + i x1),  loss = sum |rho|^2 / B,
 * gout = d loss / d y = (2 / B) conj(h^2 A^T conj(rho)) (device, like y; must differ from
 * out; A^T = A but for reflection boundaries), A with the boundary mode of h; the loss
 * goes to *loss_dev.  Allocates its scratch stream-ordered.  HELM_EUNSUPPORTED for a
 * handle with the compact fourth-order stencil. */
int unet_residual_loss(helm_t h, const float* out, const float* x, int B, float* gout, float* loss_dev,
                       helm_stream_t stream);
/* One Adam step (Sec. 3.4 and 4: the paper trains with Adam), bias-corrected, on every
 * parameter of net (and of its attached encoder), from the accumulated gradients. */
int unet_adam_step(unet_t net, float lr, float beta1, float beta2, float eps, helm_stream_t stream);

/* Attach an encoder (Sec. 3.3) to a solver net built with context channels (Eq. 3.5);
 * detach with NULL.  HELM_EINVAL if the encoder's feature channels do not match. */
int unet_attach_encoder(unet_t solver, unet_t encoder);
/* Run the attached encoder on the medium of h (kappa^2 and the layer
 * attenuation of the fine grid, batch 1) and keep its features for the
 * solver: once per medium at solve time (Sec. 3.3, train = 0), or before each
 * solver training step when the pair is trained jointly (train = 1). */
int unet_encode(unet_t solver, helm_t h, int train, helm_stream_t stream);

/* Preconditioner application e = M(r) with the U-Net in inference mode:
 *   HELM_PREC_JU: Alg. 2 (Jacobi on A from 0, U-Net on the new residual, Jacobi)
 *   HELM_PREC_VU: Eq. 3.4 (V-cycle on M started from U-Net(r))
 * The network sees [Re, Im](h^2 r / s), kappa^2, gamma with s = RMS(h^2 r) per
 * right-hand side and its output is scaled back by s.  r, e: complex [nrhs][ny][nx],
 * device, dtype HELM_C32 or HELM_C64; r and e must differ. */
int unet_precond(helm_t h, unet_t net, int kind, const void* r, void* e, int nrhs, int dtype,
                 helm_stream_t stream);

/* Training batch from generated pairs (Sec. 3.4): sample i mixes the pairs
 * idx[i][q] (q < nmix) with complex coefficients coef[i][q] = (re, im) (the
 * paper's augmentation by linear combinations; nmix = 1, coef 1 = no mixing),
 * r' = sum coef r[idx], e' likewise, then writes the network input
 * x[i] = [Re, Im](h^2 r' / s), kappa^2, gamma and the target [Re, Im](e' / s),
 * s = RMS(h^2 r').  r, e: device complex128 [npairs][ny][nx]; idx (int) and
 * coef (double pairs) are HOST arrays [count][nmix]; x: device float32
 * [count][ny][nx][4]; target: device float32 [count][ny][nx][2].  Synchronises. */
int unet_make_batch(helm_t h, const void* r, const void* e, int npairs, int count, int nmix, const int* idx,
                    const double* coef, float* x, float* target, helm_stream_t stream);

/* Measurement hook (no counterpart in the paper): time one convolution layer
 * (index in layer order) of the last forward's geometry, in its inference form
 * (BatchNorm and eLU applied as the forward applies them): `reps` repetitions
 * captured in one CUDA graph on an internal stream and replayed, timed with CUDA
 * events (device time without host launch overhead; `stream` runs the warm-up);
 * *ms = mean device time per repetition (all launches
 * of the layer), *flops = 2 * MACs of the layer (structural zeros of transposed
 * convolutions excluded), *tc = the convolution kernel that ran: 3 direct
 * CUDA-core kernel for thin layers, 2 TMA-fed tensor core, 1 cp.async-fed tensor
 * core, 0 generic CUDA-core kernel.  Needs a prior
 * unet_forward of that shape; overwrites that layer's activation buffer. */
int unet_time_layer(unet_t net, int layer, int reps, helm_stream_t stream, float* ms, double* flops, int* tc);

/* Training pairs of Eq. 3.8-3.9 on the medium of h: x ~ CN(0,1) per node and
 * k ~ U{1..kmax} per pair from SplitMix64(seed) (counter layout in synth.py),
 * b = A x, x~ = k FGMRES(m)+M_V iterations from 0, r = b - A x~, e = x - x~.
 * r, e: device complex128 [count][ny][nx]. */
int helm_gen_pairs(helm_t h, int count, unsigned long long seed, int kmax, void* r, void* e, helm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HELM_UNET_H */
