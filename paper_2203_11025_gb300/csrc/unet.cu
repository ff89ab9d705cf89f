// U-Net executor and C ABI (include/unet.h): network layout in the order of
// Sec. 3.1 (Eq. 3.1-3.3), encoder-solver context (Sec. 3.3, Eq. 3.5),
// train/inference forward, full backward, Adam (Sec. 3.4), and the
// preconditioners M_JU (Alg. 2) and M_VU (Eq. 3.4).
#include <cuda_bf16.h>

#include <atomic>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/helm.h"
#include "../../include/unet.h"
#include "devonce.cuh"
#include "helm_internal.cuh"
#include "unet_api.h"
#include "unet_internal.cuh"

namespace helm {
void set_error(const std::string& s);
}
using namespace helm;

#define UCHECK(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      return HELM_ECUDA;                                                               \
    }                                                                                  \
  } while (0)
#define UTRY(call)         \
  do {                     \
    int r_ = (call);       \
    if (r_ < 0) return r_; \
  } while (0)

namespace {

struct ConvL {
  std::string name;
  int kind;                 // 0 down (5x5 stride 2), 1 same (3x3), 2 up (5x5 stride-2 transposed)
  int k, cin, cout;
  size_t woff;              // offset in the flat parameter vector
  int c0, c1;               // input split: main source, encoder context
  size_t wpoff;             // offset of the padded weight copy (TMA path)
  size_t wpaoff;            // offset of the padded adjoint copy (data gradients on the TMA path)
  size_t wsoff;             // offset of the sub-pixel copy (transposed layers with 4 cout <= 256), or SIZE_MAX
};
struct BnL { std::string name; int c; size_t goff; size_t soff; };

// A device arena of float-aligned pieces.
struct DevArena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  template <typename T> T* take(size_t n) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + n * sizeof(T);
    return base ? (T*)(base + off) : nullptr;
  }
};

}  // namespace

struct unet_ctx {
  unet_cfg cfg{};
  int L = 0;
  // identity of the buffers a captured solve cycle references: a process-unique id and
  // the generation of the workspace (bumped on every reallocation)
  unsigned long long uid = 0, ws_gen = 0;
  std::vector<ConvL> convs;
  std::vector<BnL> bns;
  size_t bias_off = 0, nparams = 0, nbn = 0;
  float *P = nullptr, *G = nullptr, *M1 = nullptr, *M2 = nullptr, *rstats = nullptr;
  __nv_bfloat16* Wb = nullptr;
  __nv_bfloat16* WTb = nullptr;                    // K-major weight copies (tensor-core path)
  __nv_bfloat16* WPb = nullptr;                    // padded K-major weight copies (TMA path)
  size_t nwp = 0;
  __nv_bfloat16* WPAb = nullptr;                   // padded adjoint copies (data gradients, TMA path)
  size_t nwpa = 0;
  __nv_bfloat16* WSb = nullptr;                    // sub-pixel copies of transposed layers (TMA path)
  size_t nws = 0;
  __nv_bfloat16* WDb = nullptr;                    // space-to-depth copy of a 4-channel input layer
  __nv_bfloat16* gbf = nullptr;                    // BF16 copy of a layer's output gradient
  float* gsum = nullptr;                           // batch sum of a layer's output gradient (one image)
  __nv_bfloat16* gsum_bf = nullptr;                // its BF16 copy
  bool use_tma = true;
  int* d_err = nullptr;                            // failure record of the tensor-core kernel
  bool use_tc = true;
  float *bn_scale = nullptr, *bn_shift = nullptr;
  double *bn_mean = nullptr, *bn_var = nullptr;
  float *ev_scale = nullptr, *ev_shift = nullptr;  // inference BN coefficients from running statistics
  bool ev_dirty = true;
  int adam_t = 0;
  float* gout = nullptr;                           // output gradient of unet_train_step (+1 spare float)
  size_t gout_n = 0;
  unet_ctx* encoder = nullptr;
  bool is_encoder = false;                         // attached to a solver: keep a BF16 copy of the output
  float* splitbuf = nullptr;                       // split-K partial-sum slices (TMA path)
  int* splitcnt = nullptr;
  long long splitcnt_n = 0;                        // floats in splitbuf
  int last_path = 0;   // kernel of the last convolution: 3 CUDA-core direct, 2 TMA, 1 cp.async, 0 generic SIMT
  bool last_train = false;
  // activation workspace for (B, ny, nx)
  int B = 0, ny = 0, nx = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  __nv_bfloat16* x_in = nullptr;
  __nv_bfloat16* xs2d = nullptr;                   // inference input in the space-to-depth layout
  bool xs2d_valid = false;                         // the last input was written there (not to x_in)
  std::vector<float*> zdown;                       // [l] raw down conv output
  std::vector<__nv_bfloat16*> h0;                  // [l] after down BN + eLU
  std::vector<std::vector<float*>> t1, sres;       // [l][r] raw ResNet convs (s includes the residual)
  std::vector<std::vector<__nv_bfloat16*>> a1, hres;
  std::vector<__nv_bfloat16*> cat;                 // [l] (1..L-1): [zn of up l+1 | skip h_l]
  __nv_bfloat16* hL = nullptr;                     // coarsest output
  std::vector<float*> zup;                         // [l] (2..L) raw up conv output at level l-1
  std::vector<__nv_bfloat16*> uact, fact;          // eLU'd up-conv inputs (tensor-core path)
  std::vector<char> uact_ok;                       // uact[l] holds the last forward's eLU'd input
  float* out = nullptr;                            // final output (FP32)
  __nv_bfloat16* out_bf = nullptr;                 // BF16 copy (encoder feature f^(0))
  // backward buffers
  std::vector<float*> gU, gzup, gD, gzd, gfeat;
  std::vector<std::vector<float*>> gS, gA1, gT1, gH2;
  float* part = nullptr;                           // reduction partials
  float* bncoef = nullptr;                         // per-channel BatchNorm backward coefficients
  int nblk = 1024;                                 // pixel blocks of the per-channel reductions
  // preconditioner scratch
  float *xin32 = nullptr, *scale = nullptr;
  void* tmp_e = nullptr;
  size_t tmp_e_bytes = 0;
};

namespace {

// Row stride of the network input and output copies: padded to 8 channels so that
// rows are 16-byte aligned (the TMA path zero-fills the channels past the real ones).
int xin_ld(const unet_ctx* n) { return (n->cfg.in_ch + 7) / 8 * 8; }
// Row stride of the BF16 copy of a layer's output gradient (channels past cout unused).
int gbf_ld(int cout) { return (cout + 7) / 8 * 8; }
int out_ld(const unet_ctx* n) { return (n->cfg.out_ch + 7) / 8 * 8; }

int level_ch_in(const unet_ctx* n, int l) {  // channels of the down-conv source at level l-1
  return l == 1 ? n->cfg.in_ch : n->cfg.widths[l - 2];
}

void build_layout(unet_ctx* n) {
  const unet_cfg& c = n->cfg;
  const int L = c.levels;
  n->L = L;
  size_t off = 0, soff = 0;
  size_t wpo = 0, wpao = 0, wso = 0;
  auto conv = [&](const std::string& nm, int kind, int k, int ci, int co, int c1) {
    const bool sub = kind == 2 && k == 5 && 4 * co <= 256;
    n->convs.push_back({nm, kind, k, ci, co, off, ci - c1, c1, wpo, wpao, sub ? wso : SIZE_MAX});
    off += (size_t)k * k * ci * co;
    wpo += conv_tma_weight_elems(k, ci - c1, c1, co);
    wpao += conv_tma_weight_adj_elems(k, ci, co);
    if (sub) wso += conv_tma_weight_sub_elems(ci - c1, c1, co);
  };
  std::vector<std::pair<std::string, int>> bnl;
  int cin = c.in_ch;
  for (int l = 1; l <= L; ++l) {
    const int w = c.widths[l - 1];
    conv("down" + std::to_string(l), 0, 5, cin + c.context[l - 1], w, c.context[l - 1]);
    bnl.push_back({"down" + std::to_string(l) + ".bn", w});
    const int nres = l == L ? c.coarse_resnets : 1;
    for (int r = 0; r < nres; ++r) {
      std::string pre = "res" + std::to_string(l) + "." + std::to_string(r);
      conv(pre + ".k1", 1, 3, w, w, 0);
      bnl.push_back({pre + ".bn1", w});
      conv(pre + ".k2", 1, 3, w, w, 0);
      bnl.push_back({pre + ".bn2", w});
    }
    cin = w;
  }
  int ucin = c.widths[L - 1];
  for (int l = L; l >= 2; --l) {
    const int co = c.widths[l - 2];
    conv("up" + std::to_string(l), 2, 5, ucin + c.context[l], co, c.context[l]);
    bnl.push_back({"up" + std::to_string(l) + ".bn", co});
    ucin = 2 * co;
  }
  conv("up1", 2, 5, ucin + c.context[1], c.out_ch, c.context[1]);
  n->nwp = wpo;
  n->nwpa = wpao;
  n->nws = wso;
  n->bias_off = off;
  off += c.out_ch;
  for (auto& b : bnl) {
    n->bns.push_back({b.first, b.second, off, soff});
    off += 2 * (size_t)b.second;
    soff += b.second;
  }
  n->nparams = off;
  n->nbn = soff;
}

const ConvL& conv_of(const unet_ctx* n, const std::string& nm) {
  for (auto& c : n->convs)
    if (c.name == nm) return c;
  return n->convs[0];
}
const BnL& bn_of(const unet_ctx* n, const std::string& nm) {
  for (auto& b : n->bns)
    if (b.name == nm) return b;
  return n->bns[0];
}

void free_ws(unet_ctx* n) {
  if (n->ws) cudaFree(n->ws);
  n->ws = nullptr;
  n->ws_bytes = 0;
  n->B = n->ny = n->nx = 0;
}

// Carve every activation and gradient buffer for (B, ny, nx); base == null measures.
void carve(unet_ctx* n, DevArena& a, int B, int ny, int nx) {
  const unet_cfg& c = n->cfg;
  const int L = n->L;
  auto M = [&](int l) { return (size_t)B * (ny >> l) * (nx >> l); };
  const int* w = c.widths;
  n->x_in = a.take<__nv_bfloat16>(M(0) * xin_ld(n));
  n->xs2d = c.in_ch == 4 ? a.take<__nv_bfloat16>(M(0) * 4) : nullptr;
  n->xs2d_valid = false;
  n->zdown.assign(L + 1, nullptr); n->h0.assign(L + 1, nullptr);
  n->t1.assign(L + 1, {}); n->sres.assign(L + 1, {}); n->a1.assign(L + 1, {}); n->hres.assign(L + 1, {});
  n->cat.assign(L + 1, nullptr); n->zup.assign(L + 1, nullptr);
  n->gU.assign(L + 1, nullptr); n->gzup.assign(L + 1, nullptr); n->gD.assign(L + 1, nullptr);
  n->gzd.assign(L + 1, nullptr); n->gfeat.assign(L + 1, nullptr);
  n->gS.assign(L + 1, {}); n->gA1.assign(L + 1, {}); n->gT1.assign(L + 1, {}); n->gH2.assign(L + 1, {});
  for (int l = 1; l <= L; ++l) {
    const size_t m = M(l);
    const int nres = l == L ? c.coarse_resnets : 1;
    n->zdown[l] = a.take<float>(m * w[l - 1]);
    n->h0[l] = a.take<__nv_bfloat16>(m * w[l - 1]);
    for (int r = 0; r < nres; ++r) {
      n->t1[l].push_back(a.take<float>(m * w[l - 1]));
      n->sres[l].push_back(a.take<float>(m * w[l - 1]));
      n->a1[l].push_back(a.take<__nv_bfloat16>(m * w[l - 1]));
      n->hres[l].push_back(a.take<__nv_bfloat16>(m * w[l - 1]));
      n->gS[l].push_back(a.take<float>(m * w[l - 1]));
      n->gA1[l].push_back(a.take<float>(m * w[l - 1]));
      n->gT1[l].push_back(a.take<float>(m * w[l - 1]));
      n->gH2[l].push_back(a.take<float>(m * w[l - 1]));
    }
    if (l < L) n->cat[l] = a.take<__nv_bfloat16>(m * 2 * w[l - 1]);
    if (l >= 2) {
      n->zup[l] = a.take<float>(M(l - 1) * w[l - 2]);
      n->gzup[l] = a.take<float>(M(l - 1) * w[l - 2]);
    }
    const int cu = (l == L) ? w[L - 1] : 2 * w[l - 1];
    n->gU[l] = a.take<float>(m * (cu + c.context[l]));
    n->gD[l] = a.take<float>(M(l - 1) * (level_ch_in(n, l) + c.context[l - 1]));
    n->gzd[l] = a.take<float>(m * w[l - 1]);
  }
  for (int l = 0; l <= L; ++l)
    if (c.context[l]) n->gfeat[l] = a.take<float>(M(l) * c.context[l]);
  n->uact.assign(L + 1, nullptr);
  n->fact.assign(L + 1, nullptr);
  for (int l = 1; l <= L; ++l) {
    const int cu = (l == L) ? w[L - 1] : 2 * w[l - 1];
    n->uact[l] = a.take<__nv_bfloat16>(M(l) * cu);
    if (c.context[l]) n->fact[l] = a.take<__nv_bfloat16>(M(l) * c.context[l]);
  }
  n->hL = a.take<__nv_bfloat16>(M(L) * w[L - 1]);
  n->out = a.take<float>(M(0) * c.out_ch);
  n->out_bf = a.take<__nv_bfloat16>(M(0) * out_ld(n));
  {
    // split-K partial sums: room for 4x the largest convolution output (splits only
    // run on layers with few pixels, whose outputs are small)
    size_t smax = 0;
    for (int l = 1; l <= L; ++l) {
      smax = std::max(smax, M(l) * (size_t)w[l - 1]);
      smax = std::max(smax, M(l - 1) * (size_t)(l >= 2 ? w[l - 2] : c.out_ch));
    }
    n->splitcnt_n = (long long)(4 * smax);
    n->splitbuf = a.take<float>((size_t)n->splitcnt_n);
    n->splitcnt = a.take<int>(kSplitTickets);   // zeroed with the workspace; each fix-up puts its ticket back
    n->gbf = a.take<__nv_bfloat16>(std::max(smax, M(0) * (size_t)gbf_ld(c.out_ch)));
    n->gsum = nullptr;
    n->gsum_bf = nullptr;
    bool ctx = false;
    for (int l = 0; l <= L; ++l) ctx = ctx || c.context[l] != 0;
    if (ctx) {
      // per-image output gradients (broadcast context sources: their weight gradient is
      // the correlation of the one feature image with the batch sum of the gradient)
      const size_t per = std::max(smax / (size_t)B, (M(0) / (size_t)B) * (size_t)gbf_ld(c.out_ch));
      n->gsum = a.take<float>(per);
      n->gsum_bf = a.take<__nv_bfloat16>(per);
    }
  }
  n->part = a.take<float>((size_t)n->nblk * 2 * 512 + 1024);
  n->bncoef = a.take<float>(5 * 512);
  n->xin32 = a.take<float>(M(0) * c.in_ch);
  n->scale = a.take<float>((size_t)B + 8);
}

// Not every kernel forms element offsets in 64-bit arithmetic: the widest tensor (twice the
// first level's width at full resolution) stays below 2^31 elements.
bool batch_fits(const unet_ctx* n, int B, int ny, int nx) {
  return (long long)B * ny * nx * 2 * n->cfg.widths[0] < (1ll << 31);
}

// Images per network pass when a preconditioner applies the U-Net to nrhs right-hand sides:
// the largest divisor of nrhs within the size limit (0 if not even one image fits).
int apply_chunk(const unet_ctx* n, int nrhs, int ny, int nx) {
  for (int c = nrhs; c >= 1; --c)
    if (nrhs % c == 0 && batch_fits(n, c, ny, nx)) return c;
  return 0;
}

int ensure_ws(unet_ctx* n, int B, int ny, int nx) {
  if (n->ws && n->B == B && n->ny == ny && n->nx == nx) return HELM_OK;
  if (!batch_fits(n, B, ny, nx)) {
    set_error("U-Net batch too large: B*ny*nx*" + std::to_string(2 * n->cfg.widths[0]) + " must stay below 2^31");
    return HELM_EUNSUPPORTED;
  }
  free_ws(n);
  DevArena m;
  carve(n, m, B, ny, nx);
  const size_t bytes = m.used + 1024;
  if (cudaMalloc(&n->ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("U-Net workspace allocation failed (" + std::to_string(bytes) + " bytes)");
    return HELM_ENOMEM;
  }
  n->ws_bytes = bytes;
  ++n->ws_gen;
  DevArena a{(char*)n->ws, bytes, 0};
  carve(n, a, B, ny, nx);
  n->B = B; n->ny = ny; n->nx = nx;
  UCHECK(cudaMemset(n->ws, 0, bytes));
  return HELM_OK;
}

// A source tensor for a convolution input.
struct Src { const void* p; int c, ld; bool bcast; };

// Context feature f^(l) of the attached encoder (BF16 source), or empty.
Src feat_of(const unet_ctx* n, int l) {
  const unet_ctx* e = n->encoder;
  if (!e || !n->cfg.context[l]) return {nullptr, 0, 0, false};
  const bool bc = (e->B == 1 && n->B > 1);
  const int L = e->L;
  if (l == 0) return {e->out_bf, e->cfg.out_ch, out_ld(e), bc};
  if (l == L) return {e->hL, e->cfg.widths[L - 1], e->cfg.widths[L - 1], bc};
  return {e->cat[l], e->cfg.widths[l - 1], 2 * e->cfg.widths[l - 1], bc};
}

ConvArgs conv_args(const unet_ctx* n, const ConvL& cl, Src a, Src b, bool act, int Hi, int Wi, float* out, int ldo) {
  ConvArgs c{};
  c.in0 = a.p; c.c0 = a.c; c.ld0 = a.ld;
  c.in1 = b.p; c.c1 = b.p ? b.c : 0; c.ld1 = b.ld; c.bcast1 = b.bcast ? 1 : 0;
  c.in_f32 = 0; c.in_act = act ? 1 : 0;
  c.B = n->B; c.Hi = Hi; c.Wi = Wi;
  c.k = cl.k;
  if (cl.kind == 0) { c.stride = 2; c.pad = 2; c.transposed = 0; c.Ho = Hi / 2; c.Wo = Wi / 2; }
  else if (cl.kind == 1) { c.stride = 1; c.pad = 1; c.transposed = 0; c.Ho = Hi; c.Wo = Wi; }
  else { c.stride = 2; c.pad = 2; c.transposed = 1; c.Ho = 2 * Hi; c.Wo = 2 * Wi; }
  c.Cout = cl.cout;
  c.W = n->Wb + cl.woff;
  c.wst = (long long)cl.cin * cl.cout; c.wsk = cl.cout; c.wsn = 1;
  c.WT = n->WTb + cl.woff;
  // the padded copy matches the layer's fixed (main, context) split
  c.WP = (a.c == cl.c0 && (b.p ? b.c : 0) == cl.c1) ? n->WPb + cl.wpoff : nullptr;
  c.WS = (c.WP && cl.wsoff != SIZE_MAX) ? n->WSb + cl.wsoff : nullptr;
  c.out = out; c.ldo = ldo;
  c.splitbuf = n->splitbuf; c.splitcnt = n->splitcnt; c.splitcnt_n = n->splitcnt_n;
  return c;
}

// The sub-pixel form of a transposed 5x5 stride-2 convolution: the 3x3 stride-1
// convolution over the input grid whose 4 Cout columns are the output phases.
ConvArgs subpixel_args(const ConvArgs& a) {
  ConvArgs c = a;
  c.k = 3; c.stride = 1; c.pad = 1; c.transposed = 0;
  c.Ho = a.Hi; c.Wo = a.Wi;
  c.Cout = 4 * a.Cout;
  c.WP = a.WS;
  c.shuffle = 1; c.cr = a.Cout;
  return c;
}

// The TMA kernel on the sub-pixel form when the layer has one (fewer, wider MMAs).
bool try_subpixel(unet_ctx* n, const ConvArgs& a, cudaStream_t s) {
  if (!(n->use_tc && n->use_tma && a.WS && a.transposed && a.k == 5 && a.pad == 2 && !a.in_act && !a.in_f32 &&
        a.Ho == 2 * a.Hi && a.Wo == 2 * a.Wi && !a.res))
    return false;
  return conv_forward_tma(subpixel_args(a), n->d_err, s);
}

// Inference inputs go to the space-to-depth layout when the input layer can run there:
// 4 input channels, no encoder context, the TMA tensor-core path.
bool s2d_input(const unet_ctx* n) {
  const int hx = n->nx / 2, hy = n->ny / 2;   // the TMA kernel tiles power-of-two grids
  return n->WDb && n->xs2d && n->use_tc && n->use_tma && hx > 0 && hy > 0 && !(hx & (hx - 1)) && !(hy & (hy - 1));
}

// The 5x5 stride-2 input layer as a 3x3 stride-1 convolution over 2x2 input blocks of
// 16 channels (one K-step per tap on the tensor cores instead of CUDA-core FMAs).
bool try_s2d_input(unet_ctx* n, const ConvArgs& a, cudaStream_t s) {
  if (a.in1 || a.transposed || a.k != 5 || a.stride != 2 || a.pad != 2 || a.c0 != 4 || a.in_act || a.in_f32 ||
      a.Hi != 2 * a.Ho || a.Wi != 2 * a.Wo)
    return false;
  ConvArgs c = a;
  c.in0 = n->xs2d; c.c0 = 16; c.ld0 = 16;
  c.Hi = a.Ho; c.Wi = a.Wo;
  c.k = 3; c.stride = 1; c.pad = 1;
  c.WP = n->WDb; c.WS = nullptr;
  return conv_forward_tma(c, n->d_err, s);
}

void run_conv(unet_ctx* n, const ConvArgs& a, cudaStream_t s) {
  if (try_subpixel(n, a, s)) { n->last_path = 2; return; }
  if (n->use_tc && conv_forward_small(a, s)) { n->last_path = 3; return; }   // 4-channel input layer
  if (n->use_tc && n->use_tma && conv_forward_tma(a, n->d_err, s)) { n->last_path = 2; return; }
  if (n->use_tc && conv_tc_eligible(a)) { conv_forward_tc(a, n->d_err, s); n->last_path = 1; }
  else { conv_forward(a, s); n->last_path = 0; }
}

// Data gradient of a convolution: the adjoint geometry with transposed weights.
ConvArgs dgrad_args(const unet_ctx* n, const ConvL& cl, const float* g, int ldg, int Hg, int Wg, float* out, int ldo) {
  ConvArgs c{};
  c.in0 = g; c.c0 = cl.cout; c.ld0 = ldg; c.in1 = nullptr; c.c1 = 0;
  c.in_f32 = 1; c.in_act = 0;
  c.B = n->B; c.Hi = Hg; c.Wi = Wg; c.k = cl.k;
  if (cl.kind == 0) { c.stride = 2; c.pad = 2; c.transposed = 1; c.Ho = 2 * Hg; c.Wo = 2 * Wg; }
  else if (cl.kind == 1) { c.stride = 1; c.pad = 1; c.transposed = 1; c.Ho = Hg; c.Wo = Wg; }
  else { c.stride = 2; c.pad = 2; c.transposed = 0; c.Ho = Hg / 2; c.Wo = Wg / 2; }
  c.Cout = cl.cin;
  c.W = n->Wb + cl.woff;
  c.wst = (long long)cl.cin * cl.cout; c.wsk = 1; c.wsn = cl.cout;
  c.out = out; c.ldo = ldo;
  return c;
}

// Data gradient dL/dx of convolution cl from g = dL/dy (FP32, ld ldg, grid Hg x Wg): on
// the TMA tensor-core path as a forward convolution of a BF16 copy of g with the
// adjoint weights (3x3 stride 1: taps reversed; 5x5 stride 2: transposed stride 2;
// transposed 5x5: stride 2), else on the generic kernel.
void run_dgrad(unet_ctx* n, const ConvL& cl, const float* g, int ldg, int Hg, int Wg, float* out, int ldo,
               cudaStream_t s, bool have_gbf = false) {
  if (n->use_tc && n->use_tma) {
    const int Mg = n->B * Hg * Wg;
    ConvArgs c{};
    c.in0 = n->gbf; c.c0 = cl.cout; c.ld0 = gbf_ld(cl.cout); c.in1 = nullptr; c.c1 = 0;
    c.B = n->B; c.Hi = Hg; c.Wi = Wg; c.k = cl.k;
    if (cl.kind == 0) { c.stride = 2; c.pad = 2; c.transposed = 1; c.Ho = 2 * Hg; c.Wo = 2 * Wg; }
    else if (cl.kind == 1) { c.stride = 1; c.pad = 1; c.transposed = 0; c.Ho = Hg; c.Wo = Wg; }
    else { c.stride = 2; c.pad = 2; c.transposed = 0; c.Ho = Hg / 2; c.Wo = Wg / 2; }
    c.Cout = cl.cin;
    c.WP = n->WPAb + cl.wpaoff;
    c.out = out; c.ldo = ldo;
    c.splitbuf = n->splitbuf; c.splitcnt = n->splitcnt; c.splitcnt_n = n->splitcnt_n;
    if (!have_gbf) to_bf16_slice(g, ldg, n->gbf, gbf_ld(cl.cout), cl.cout, Mg, s);
    if (conv_forward_tma(c, n->d_err, s)) return;
  }
  conv_forward(dgrad_args(n, cl, g, ldg, Hg, Wg, out, ldo), s);
}

// Weight gradient gW += dW of the forward convolution fa from g = dL/dy (FP32, ld ldg)
// and, when dx is set, the data gradient into dx: both from one BF16 copy of g on the
// tensor-core path.  `act_src`: the materialised eLU copy of fa's input, if any.
// Weight gradient of a two-source convolution (input channels [0, c0) from in0, [c0, c0 +
// c1) from the context source in1) on the tensor cores: one GEMM per source into its rows
// of gW.  A broadcast context source (one image for the batch) correlates with the batch
// sum of g.  eLU'd inputs need their materialised copies (act0, act1).  Launches nothing
// and returns false unless both parts qualify.
bool wgrad_two_sources(unet_ctx* n, const ConvL& cl, const ConvArgs& fa, const float* g, int ldg, float* gW, int Hg,
                       int Wg, const __nv_bfloat16* act0, const __nv_bfloat16* act1, cudaStream_t s) {
  if (fa.in_act && (!act0 || !act1)) return false;
  if (fa.bcast1 && (!n->gsum || !n->gsum_bf)) return false;
  const int cin = fa.c0 + fa.c1, ldgb = gbf_ld(cl.cout);
  ConvArgs t0 = fa;
  t0.in1 = nullptr; t0.c1 = 0; t0.bcast1 = 0;
  if (fa.in_act) { t0.in0 = act0; t0.ld0 = fa.c0; t0.in_act = 0; }
  ConvArgs t1 = fa;
  t1.in0 = fa.in1; t1.c0 = fa.c1; t1.ld0 = fa.ld1; t1.in1 = nullptr; t1.c1 = 0; t1.bcast1 = 0;
  if (fa.in_act) { t1.in0 = act1; t1.ld0 = fa.c1; t1.in_act = 0; }
  const __nv_bfloat16* g1 = n->gbf;
  if (fa.bcast1) { t1.B = 1; g1 = n->gsum_bf; }
  if (!conv_wgrad_tma(t0, n->gbf, ldgb, gW, n->d_err, s, cin, false) ||
      !conv_wgrad_tma(t1, g1, ldgb, gW + (size_t)fa.c0 * cl.cout, n->d_err, s, cin, false))
    return false;
  if (fa.bcast1) {
    const size_t P = (size_t)Hg * Wg;
    batch_sum(g, ldg, n->B, P, cl.cout, n->gsum, cl.cout, false, s);
    to_bf16_slice(n->gsum, cl.cout, n->gsum_bf, ldgb, cl.cout, (int)P, s);
  }
  conv_wgrad_tma(t0, n->gbf, ldgb, gW, n->d_err, s, cin, true, n->splitbuf, (size_t)n->splitcnt_n);
  conv_wgrad_tma(t1, g1, ldgb, gW + (size_t)fa.c0 * cl.cout, n->d_err, s, cin, true, n->splitbuf,
                 (size_t)n->splitcnt_n);
  return true;
}

void backprop_conv(unet_ctx* n, const ConvL& cl, ConvArgs fa, const float* g, int ldg, float* gW, int Hg, int Wg,
                   float* dx, int lddx, cudaStream_t s, const __nv_bfloat16* act_src = nullptr,
                   const __nv_bfloat16* act_ctx = nullptr) {
  bool have = false;
  if (n->use_tc && n->use_tma) {
    to_bf16_slice(g, ldg, n->gbf, gbf_ld(cl.cout), cl.cout, n->B * Hg * Wg, s);
    have = true;
    ConvArgs t = fa;
    if (t.in_act && act_src && !t.in1) { t.in0 = act_src; t.ld0 = t.c0; t.in_act = 0; }
    const bool done = fa.in1 ? wgrad_two_sources(n, cl, fa, g, ldg, gW, Hg, Wg, act_src, act_ctx, s)
                             : conv_wgrad_tma(t, n->gbf, gbf_ld(cl.cout), gW, n->d_err, s, 0, true, n->splitbuf,
                                              (size_t)n->splitcnt_n);
    if (!done) conv_wgrad(fa, g, ldg, gW, s);
  } else {
    conv_wgrad(fa, g, ldg, gW, s);
  }
  if (dx) run_dgrad(n, cl, g, ldg, Hg, Wg, dx, lddx, s, have);
}

void ensure_eval_coeffs(unet_ctx* n, cudaStream_t s);

// BatchNorm (train: batch statistics, running update; eval: running statistics),
// then optional eLU, into a BF16 slice.
void run_bn(unet_ctx* n, const std::string& nm, const float* z, int ldz, int M, bool act, __nv_bfloat16* y, int ldy,
            bool train, cudaStream_t s) {
  const BnL& b = bn_of(n, nm);
  float* gamma = n->P + b.goff;
  float* beta = gamma + b.c;
  float* sc = n->bn_scale + b.soff;
  float* sh = n->bn_shift + b.soff;
  float* rm = n->rstats + b.soff;
  float* rv = n->rstats + n->nbn + b.soff;
  if (train) {
    bn_batch_stats(z, ldz, b.c, M, n->bn_mean + b.soff, n->bn_var + b.soff, n->part, n->nblk, s);
    bn_coeffs(n->bn_mean + b.soff, n->bn_var + b.soff, gamma, beta, b.c, sc, sh, rm, rv, true, M, s);
  } else {
    ensure_eval_coeffs(n, s);
    sc = n->ev_scale + b.soff;
    sh = n->ev_shift + b.soff;
  }
  bn_act(z, ldz, b.c, M, sc, sh, act, y, ldy, s);
}

void run_bn_bwd(unet_ctx* n, const std::string& nm, const float* g, int ldg, const float* z, int ldz, int M, bool act,
                float* gz, int ldo, cudaStream_t s) {
  const BnL& b = bn_of(n, nm);
  bn_backward(g, ldg, z, ldz, b.c, M, n->bn_mean + b.soff, n->bn_var + b.soff, n->bn_scale + b.soff,
              n->bn_shift + b.soff, act, n->P + b.goff, n->G + b.goff, n->G + b.goff + b.c, n->part, n->nblk,
              n->bncoef, gz, ldo, s);
}

void ensure_eval_coeffs(unet_ctx* n, cudaStream_t s) {
  if (!n->ev_dirty) return;
  for (auto& b : n->bns)
    bn_coeffs_eval(n->rstats + b.soff, n->rstats + n->nbn + b.soff, n->P + b.goff, n->P + b.goff + b.c, b.c,
                   n->ev_scale + b.soff, n->ev_shift + b.soff, s);
  n->ev_dirty = false;
}

// Convolution followed by BatchNorm (+ eLU) into a BF16 slice.  At inference on the
// tensor-core path the normalisation is applied in the convolution's epilogue.
void conv_bn(unet_ctx* n, ConvArgs a, const std::string& bn, bool act, __nv_bfloat16* y, int ldy, int M, bool train,
             cudaStream_t s, __nv_bfloat16* y2 = nullptr, int ldy2 = 0) {
  // inference: BatchNorm and eLU fused into the convolution's epilogue; y2 (optional):
  // eLU of y, the activated input of the next up convolution (written by the TMA
  // epilogue, else copied)
  if (!train && n->use_tc) {
    ConvArgs f = a;
    const BnL& b = bn_of(n, bn);
    ensure_eval_coeffs(n, s);
    f.scale = n->ev_scale + b.soff;
    f.shift = n->ev_shift + b.soff;
    f.ep_act = act ? 1 : 0;
    f.ybf = y;
    f.ldy = ldy;
    f.y2 = y2;
    f.ldy2 = ldy2;
    bool done = false, wrote2 = false;
    if (a.in0 == n->x_in && n->xs2d_valid) {
      if (try_s2d_input(n, f, s)) { n->last_path = 2; done = wrote2 = true; }
      else { s2d_to_std(n->xs2d, n->x_in, xin_ld(n), n->B, n->ny, n->nx, s); n->xs2d_valid = false; }
    }
    if (done) {
    } else if (try_subpixel(n, f, s)) { n->last_path = 2; done = wrote2 = true; }
    else if (conv_forward_small(f, s)) { n->last_path = 3; done = true; }   // measured faster than TMA here
    else if (n->use_tma && conv_forward_tma(f, n->d_err, s)) { n->last_path = 2; done = wrote2 = true; }
    else if (conv_tc_eligible(f)) {
      conv_forward_tc(f, n->d_err, s);
      n->last_path = 1;
      done = true;
    }
    if (done) {
      if (y2 && !wrote2) elu_copy_bf16(y, ldy, a.Cout, (size_t)M, y2, ldy2, s);
      return;
    }
  }
  if (a.in0 == n->x_in && n->xs2d_valid) {
    s2d_to_std(n->xs2d, n->x_in, xin_ld(n), n->B, n->ny, n->nx, s);
    n->xs2d_valid = false;
  }
  run_conv(n, a, s);
  run_bn(n, bn, a.out, a.ldo, M, act, y, ldy, train, s);
  if (y2) elu_copy_bf16(y, ldy, a.Cout, (size_t)M, y2, ldy2, s);
}

// Materialise eLU of an up convolution's inputs for the tensor-core gather.
ConvArgs act_inputs(unet_ctx* n, ConvArgs a, int l, const Src& u, const Src& f, int H, int W, int M, cudaStream_t s) {
  if (!n->use_tc || conv_small_eligible(a)) return a;   // the direct kernel applies eLU while staging
  ConvArgs t = a;
  t.in_act = 0;
  if (!conv_tc_eligible(t)) return a;
  elu_copy_bf16((const __nv_bfloat16*)u.p, u.ld, u.c, (size_t)M, n->uact[l], u.c, s);
  if ((int)n->uact_ok.size() > l) n->uact_ok[l] = 1;
  t.in0 = n->uact[l];
  t.ld0 = u.c;
  if (f.p) {
    const size_t fm = f.bcast ? (size_t)H * W : (size_t)M;
    elu_copy_bf16((const __nv_bfloat16*)f.p, f.ld, f.c, fm, n->fact[l], f.c, s);
    t.in1 = n->fact[l];
    t.ld1 = f.c;
  }
  return t;
}

int forward_impl(unet_ctx* n, bool train, cudaStream_t s) {
  const unet_cfg& c = n->cfg;
  const int L = n->L;
  n->uact_ok.assign(L + 1, 0);
  // inference: epilogues write the eLU'd inputs of the up convolutions (levels without
  // encoder context; with context those levels keep the explicit copy)
  const bool direct = !train && n->use_tc;
  const int* w = c.widths;
  auto hw = [&](int l, int& H, int& W) { H = n->ny >> l; W = n->nx >> l; };
  auto M = [&](int l) { return n->B * (n->ny >> l) * (n->nx >> l); };
  for (int l = 1; l <= L; ++l) {
    int H, W;
    hw(l - 1, H, W);
    Src src = l == 1 ? Src{n->x_in, c.in_ch, xin_ld(n), false} : Src{n->cat[l - 1] + w[l - 2], w[l - 2], 2 * w[l - 2], false};
    const ConvL& dl = conv_of(n, "down" + std::to_string(l));
    ConvArgs a = conv_args(n, dl, src, feat_of(n, l - 1), false, H, W, n->zdown[l], w[l - 1]);
    conv_bn(n, a, "down" + std::to_string(l) + ".bn", true, n->h0[l], w[l - 1], M(l), train, s);
    const __nv_bfloat16* h = n->h0[l];
    int ldh = w[l - 1];
    const int nres = l == L ? c.coarse_resnets : 1;
    int Hl, Wl;
    hw(l, Hl, Wl);
    for (int r = 0; r < nres; ++r) {
      const std::string pre = "res" + std::to_string(l) + "." + std::to_string(r);
      ConvArgs k1 = conv_args(n, conv_of(n, pre + ".k1"), Src{h, w[l - 1], ldh, false}, Src{nullptr, 0, 0, false},
                              false, Hl, Wl, n->t1[l][r], w[l - 1]);
      conv_bn(n, k1, pre + ".bn1", true, n->a1[l][r], w[l - 1], M(l), train, s);
      ConvArgs k2 = conv_args(n, conv_of(n, pre + ".k2"), Src{n->a1[l][r], w[l - 1], w[l - 1], false},
                              Src{nullptr, 0, 0, false}, false, Hl, Wl, n->sres[l][r], w[l - 1]);
      k2.res = h; k2.ldr = ldh;
      __nv_bfloat16* dst;
      int ldd;
      if (r == nres - 1 && l < L) { dst = n->cat[l] + w[l - 1]; ldd = 2 * w[l - 1]; }
      else if (r == nres - 1) { dst = n->hL; ldd = w[L - 1]; }
      else { dst = n->hres[l][r]; ldd = w[l - 1]; }
      // inference without context at this level: also the eLU'd copy the up convolution reads
      __nv_bfloat16* d2 = nullptr;
      if (direct && r == nres - 1) d2 = l < L ? n->uact[l] + w[l - 1] : n->uact[L];
      conv_bn(n, k2, pre + ".bn2", true, dst, ldd, M(l), train, s, d2, ldd);
      h = dst;
      ldh = ldd;
    }
  }
  // up convolutions read eLU(u): the eLU'd copy written by the producing epilogues
  // (inference without context), else materialised here
  auto up_args = [&](const ConvL& ul, int l, const Src& u, const Src& f, int H, int W, float* out, int ldo) {
    if (direct && !f.p) {
      n->uact_ok[l] = 1;
      return conv_args(n, ul, Src{n->uact[l], u.c, u.c, false}, f, false, H, W, out, ldo);
    }
    ConvArgs a = conv_args(n, ul, u, f, true, H, W, out, ldo);
    return act_inputs(n, a, l, u, f, H, W, M(l), s);   // the tensor-core gather copies raw bytes
  };
  Src u{n->hL, w[L - 1], w[L - 1], false};
  for (int l = L; l >= 2; --l) {
    int H, W;
    hw(l, H, W);
    const ConvL& ul = conv_of(n, "up" + std::to_string(l));
    Src f = feat_of(n, l);
    ConvArgs a = up_args(ul, l, u, f, H, W, n->zup[l], w[l - 2]);
    conv_bn(n, a, "up" + std::to_string(l) + ".bn", false, n->cat[l - 1], 2 * w[l - 2], M(l - 1), train, s,
            direct ? n->uact[l - 1] : nullptr, 2 * w[l - 2]);
    u = Src{n->cat[l - 1], 2 * w[l - 2], 2 * w[l - 2], false};
  }
  {
    int H, W;
    hw(1, H, W);
    Src f = feat_of(n, 1);
    ConvArgs a = up_args(conv_of(n, "up1"), 1, u, f, H, W, n->out, c.out_ch);
    a.bias = n->P + n->bias_off;
    run_conv(n, a, s);
    if (n->is_encoder) to_bf16_slice(n->out, c.out_ch, n->out_bf, out_ld(n), c.out_ch, M(0), s);
  }
  n->last_train = train;
  if (train) n->ev_dirty = true;   // running statistics moved
  UCHECK(cudaGetLastError());
  return HELM_OK;
}

// Backward of the last train forward.  gout: d/d out (ld out_ch).  g_own: gradients
// arriving on this net's own features (encoder), else null.  gx: input gradient or null.
int backward_impl(unet_ctx* n, const float* gout, float* const* g_own, float* gx, cudaStream_t s) {
  const unet_cfg& c = n->cfg;
  const int L = n->L;
  const int* w = c.widths;
  auto hw = [&](int l, int& H, int& W) { H = n->ny >> l; W = n->nx >> l; };
  auto M = [&](int l) { return n->B * (n->ny >> l) * (n->nx >> l); };
  for (int l = 0; l <= L; ++l)
    if (n->gfeat[l]) UCHECK(cudaMemsetAsync(n->gfeat[l], 0, (size_t)M(l) * c.context[l] * 4, s));
  // final layer
  chan_sum_add(gout, c.out_ch, c.out_ch, M(0), n->G + n->bias_off, n->part, n->nblk, s);
  {
    const ConvL& cl = conv_of(n, "up1");
    int H, W;
    hw(1, H, W);
    Src u = L > 1 ? Src{n->cat[1], 2 * w[0], 2 * w[0], false} : Src{n->hL, w[0], w[0], false};
    ConvArgs fa = conv_args(n, cl, u, feat_of(n, 1), true, H, W, nullptr, 0);
    const int cu = u.c, ldU = cu + c.context[1];
    backprop_conv(n, cl, fa, gout, c.out_ch, n->G + cl.woff, n->ny, n->nx, n->gU[1], ldU, s,
                  n->uact_ok[1] ? n->uact[1] : nullptr, n->uact_ok[1] ? n->fact[1] : nullptr);
    elu_backward_inplace(n->gU[1], ldU, (const __nv_bfloat16*)u.p, u.ld, cu, M(1), 0, s);
    if (c.context[1]) {
      Src f = feat_of(n, 1);
      elu_backward_inplace(n->gU[1] + cu, ldU, (const __nv_bfloat16*)f.p, f.ld, f.c, M(1),
                           f.bcast ? (size_t)H * W : 0, s);
      add_slice(n->gfeat[1], c.context[1], n->gU[1] + cu, ldU, c.context[1], M(1), s);
    }
  }
  // up levels 2..L
  for (int l = 2; l <= L; ++l) {
    const int cz = w[l - 2];
    const int ldin = 2 * cz + c.context[l - 1];   // ld of gU[l-1]
    float* gzn = n->gU[l - 1];
    if (g_own && g_own[l - 1]) add_slice(gzn, ldin, g_own[l - 1], cz, cz, M(l - 1), s);
    run_bn_bwd(n, "up" + std::to_string(l) + ".bn", gzn, ldin, n->zup[l], cz, M(l - 1), false, n->gzup[l], cz, s);
    const ConvL& cl = conv_of(n, "up" + std::to_string(l));
    int H, W;
    hw(l, H, W);
    Src u = (l == L) ? Src{n->hL, w[L - 1], w[L - 1], false} : Src{n->cat[l], 2 * w[l - 1], 2 * w[l - 1], false};
    ConvArgs fa = conv_args(n, cl, u, feat_of(n, l), true, H, W, nullptr, 0);
    const int ldU = u.c + c.context[l];
    int Hg, Wg;
    hw(l - 1, Hg, Wg);
    backprop_conv(n, cl, fa, n->gzup[l], cz, n->G + cl.woff, Hg, Wg, n->gU[l], ldU, s,
                  n->uact_ok[l] ? n->uact[l] : nullptr, n->uact_ok[l] ? n->fact[l] : nullptr);
    elu_backward_inplace(n->gU[l], ldU, (const __nv_bfloat16*)u.p, u.ld, u.c, M(l), 0, s);
    if (c.context[l]) {
      Src f = feat_of(n, l);
      elu_backward_inplace(n->gU[l] + u.c, ldU, (const __nv_bfloat16*)f.p, f.ld, f.c, M(l), f.bcast ? (size_t)H * W : 0,
                           s);
      add_slice(n->gfeat[l], c.context[l], n->gU[l] + u.c, ldU, c.context[l], M(l), s);
    }
  }
  // down path
  float* gh = n->gU[L];
  int ldgh = w[L - 1] + c.context[L];
  if (g_own && g_own[L]) add_slice(gh, ldgh, g_own[L], w[L - 1], w[L - 1], M(L), s);
  for (int l = L; l >= 1; --l) {
    const int cw = w[l - 1];
    if (l < L) {
      // gradient on h_l = skip part of gU[l] + first cw channels of the down l+1 data gradient
      const int ldU = 2 * cw + c.context[l];
      gh = n->gU[l] + cw;
      ldgh = ldU;
      add_slice(gh, ldgh, n->gD[l + 1], cw + c.context[l], cw, M(l), s);
    }
    const int nres = l == L ? c.coarse_resnets : 1;
    int Hl, Wl;
    hw(l, Hl, Wl);
    for (int r = nres - 1; r >= 0; --r) {
      const std::string pre = "res" + std::to_string(l) + "." + std::to_string(r);
      const __nv_bfloat16* hin = r == 0 ? n->h0[l] : n->hres[l][r - 1];
      run_bn_bwd(n, pre + ".bn2", gh, ldgh, n->sres[l][r], cw, M(l), true, n->gS[l][r], cw, s);
      const ConvL& k2 = conv_of(n, pre + ".k2");
      ConvArgs fa2 = conv_args(n, k2, Src{n->a1[l][r], cw, cw, false}, Src{nullptr, 0, 0, false}, false, Hl, Wl, nullptr, 0);
      backprop_conv(n, k2, fa2, n->gS[l][r], cw, n->G + k2.woff, Hl, Wl, n->gA1[l][r], cw, s);
      run_bn_bwd(n, pre + ".bn1", n->gA1[l][r], cw, n->t1[l][r], cw, M(l), true, n->gT1[l][r], cw, s);
      const ConvL& k1 = conv_of(n, pre + ".k1");
      ConvArgs fa1 = conv_args(n, k1, Src{hin, cw, cw, false}, Src{nullptr, 0, 0, false}, false, Hl, Wl, nullptr, 0);
      backprop_conv(n, k1, fa1, n->gT1[l][r], cw, n->G + k1.woff, Hl, Wl, n->gH2[l][r], cw, s);
      add_slice(n->gH2[l][r], cw, n->gS[l][r], cw, cw, M(l), s);   // identity branch
      gh = n->gH2[l][r];
      ldgh = cw;
    }
    run_bn_bwd(n, "down" + std::to_string(l) + ".bn", gh, ldgh, n->zdown[l], cw, M(l), true, n->gzd[l], cw, s);
    const ConvL& dl = conv_of(n, "down" + std::to_string(l));
    int H, W;
    hw(l - 1, H, W);
    Src src = l == 1 ? Src{n->x_in, c.in_ch, xin_ld(n), false} : Src{n->cat[l - 1] + w[l - 2], w[l - 2], 2 * w[l - 2], false};
    ConvArgs fa = conv_args(n, dl, src, feat_of(n, l - 1), false, H, W, nullptr, 0);
    const int ldD = src.c + c.context[l - 1];
    backprop_conv(n, dl, fa, n->gzd[l], cw, n->G + dl.woff, Hl, Wl, n->gD[l], ldD, s);
    if (c.context[l - 1]) add_slice(n->gfeat[l - 1], c.context[l - 1], n->gD[l] + src.c, ldD, c.context[l - 1], M(l - 1), s);
    if (l == 1 && gx) UCHECK(cudaMemcpy2DAsync(gx, c.in_ch * 4, n->gD[1], ldD * 4, c.in_ch * 4, M(0),
                                                cudaMemcpyDeviceToDevice, s));
  }
  UCHECK(cudaGetLastError());
  return HELM_OK;
}

// The context feature gradients of a solver, reduced to the encoder's batch, then
// the encoder's backward.
int backward_encoder(unet_ctx* solver, cudaStream_t s) {
  unet_ctx* e = solver->encoder;
  if (!e) return HELM_OK;
  if (!e->last_train) { set_error("encoder's last forward was not train-mode"); return HELM_EINVAL; }
  const int L = e->L;
  std::vector<float*> g_own(L + 1, nullptr);
  // reuse the encoder's gfeat-free scratch: zdown-sized gradient buffers are not needed; use gU/gD of the
  // encoder? They are overwritten by its own backward.  Reduce into dedicated buffers instead.
  static_assert(sizeof(float) == 4, "");
  std::vector<float*> bufs;
  for (int l = 0; l <= L; ++l) {
    const size_t P = (size_t)(e->ny >> l) * (e->nx >> l);
    const int C = solver->cfg.context[l];
    float* d = nullptr;
    UCHECK(cudaMallocAsync(&d, P * e->B * C * 4, s));
    bufs.push_back(d);
    if (e->B == solver->B) UCHECK(cudaMemcpyAsync(d, solver->gfeat[l], P * e->B * C * 4, cudaMemcpyDeviceToDevice, s));
    else batch_sum(solver->gfeat[l], C, solver->B, P, C, d, C, false, s);
    g_own[l] = d;
  }
  // f^(0) is the encoder output: its gradient is the encoder's gout
  int r = backward_impl(e, g_own[0], g_own.data(), nullptr, s);
  for (float* d : bufs) cudaFreeAsync(d, s);
  return r;
}

void refresh_bf16(unet_ctx* n, cudaStream_t s) {
  f32_to_bf16(n->P, n->Wb, n->nparams, s);
  for (auto& cl : n->convs) {
    weights_kmajor(n->P + cl.woff, n->WTb + cl.woff, cl.k * cl.k, cl.cin, cl.cout, s);
    conv_tma_weights(n->P + cl.woff, n->WPb + cl.wpoff, cl.k, cl.c0, cl.c1, cl.cout, s);
    conv_tma_weights_adjoint(n->P + cl.woff, n->WPAb + cl.wpaoff, cl.k, cl.cin, cl.cout, cl.kind == 1, s);
    if (cl.wsoff != SIZE_MAX) conv_tma_weights_subpixel(n->P + cl.woff, n->WSb + cl.wsoff, cl.c0, cl.c1, cl.cout, s);
  }
  if (n->WDb) {
    const ConvL& d1 = conv_of(n, "down1");
    conv_tma_weights_s2d_in(n->P + d1.woff, n->WDb, d1.cin, d1.cout, s);
  }
}

}  // namespace

// ===========================================================================
// helm-side bridge: U-Net preconditioners inside FGMRES
// ===========================================================================
namespace helm {
// defined in solver.cu
int vcycle_public(helm_ctx* c, const void* f, const void* v_in, void* out, int nrhs, int real_bytes, const int* gate,
                  cudaStream_t s);
int jacobi_public(helm_ctx* c, int op, const void* f, const void* x_in, void* x_out, int nrhs, int real_bytes,
                  const int* gate, cudaStream_t s);
int residual_public(helm_ctx* c, int op, const void* b, const void* x, void* r, int nrhs, int real_bytes,
                    const int* gate, cudaStream_t s);
void helm_geometry(helm_ctx* c, int* nx, int* ny, double* h, int* abc_w, double* gmax, const float** k2f,
                   const float** gam);
void* helm_scratch(helm_ctx* c, int real_bytes, int which, int nrhs);
double helm_omega(helm_ctx* c);
int helm_media(helm_ctx* c, int* rpp);
int helm_bc(helm_ctx* c);
int helm_stencil(helm_ctx* c);
}  // namespace helm

// e = U-Net(r) (inference), with the network input built on the fly.
static int unet_apply(helm_ctx* hc, unet_ctx* n, const void* r, void* e, bool add, int nrhs, int real_bytes,
                      const int* gate, cudaStream_t s) {
  int nx, ny, abc_w;
  double h, gmax;
  const float *k2f, *gam;
  helm_geometry(hc, &nx, &ny, &h, &abc_w, &gmax, &k2f, &gam);
  const int div = 1 << n->L;
  if (nx % div || ny % div) { set_error("grid not divisible by 2^levels of the U-Net"); return HELM_EINVAL; }
  if (n->cfg.in_ch != 4 || n->cfg.out_ch != 2) { set_error("preconditioner net needs 4 inputs, 2 outputs"); return HELM_EINVAL; }
  const int cb = apply_chunk(n, nrhs, ny, nx);
  if (cb == 0) { set_error("grid too large for one U-Net image"); return HELM_EUNSUPPORTED; }
  int rpp = 0;
  if (helm_media(hc, &rpp) > 1 && n->encoder) {
    set_error("the encoder-solver pair runs on a handle of one medium");
    return HELM_EUNSUPPORTED;
  }
  if (n->ws == nullptr || n->B != cb || n->ny != ny || n->nx != nx) {
    cudaStreamCaptureStatus cs;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) { set_error("U-Net workspace not prepared before capture"); return HELM_EINVAL; }
    UTRY(ensure_ws(n, cb, ny, nx));
  }
  // right-hand sides in chunks of cb images (one chunk unless the size limit splits them)
  const size_t vec_bytes = (size_t)nx * ny * 2 * real_bytes;
  for (int c0 = 0; c0 < nrhs; c0 += cb) {
    const void* rc = (const char*)r + c0 * vec_bytes;
    void* ec = (char*)e + c0 * vec_bytes;
    const int* gc = gate ? gate + c0 : nullptr;
    const bool s2d = s2d_input(n);
    make_input(rc, real_bytes == 8, cb, ny, nx, h, k2f, gam, s2d ? n->xs2d : n->x_in, xin_ld(n), n->scale, n->part,
               gc, s, s2d, rpp, c0);
    n->xs2d_valid = s2d;
    UTRY(forward_impl(n, false, s));
    write_output(n->out, real_bytes == 8, cb, ny, nx, n->scale, ec, add, gc, s);
  }
  UCHECK(cudaGetLastError());
  return HELM_OK;
}

int unet_precond_impl(helm_ctx* hc, void* netp, int kind, const void* v, void* z, int nrhs, int real_bytes,
                      const int* gate, cudaStream_t s) {
  unet_ctx* n = (unet_ctx*)netp;
  if (!n) { set_error("null net"); return HELM_EINVAL; }
  if (n->cfg.context[0] && !n->encoder) { set_error("solver net needs an attached, encoded encoder"); return HELM_EINVAL; }
  if (kind == HELM_PREC_VU) {
    // Eq. 3.4: e = V-cycle(e0 = U-Net(r), r)
    void* e0 = helm_scratch(hc, real_bytes, 0, nrhs);
    if (!e0) return HELM_ENOMEM;
    UTRY(unet_apply(hc, n, v, e0, false, nrhs, real_bytes, gate, s));
    return vcycle_public(hc, v, e0, z, nrhs, real_bytes, gate, s);
  }
  if (kind == HELM_PREC_JU) {
    // Alg. 2: e1 = Jacobi(0, r); e2 = e1 + U-Net(r - A e1); e = Jacobi(e2, r)   (Jacobi on A)
    void* e1 = helm_scratch(hc, real_bytes, 0, nrhs);
    void* rr = helm_scratch(hc, real_bytes, 1, nrhs);
    if (!e1 || !rr) return HELM_ENOMEM;
    UTRY(jacobi_public(hc, HELM_OP_A, v, nullptr, e1, nrhs, real_bytes, gate, s));
    UTRY(residual_public(hc, HELM_OP_A, v, e1, rr, nrhs, real_bytes, gate, s));
    UTRY(unet_apply(hc, n, rr, e1, true, nrhs, real_bytes, gate, s));
    return jacobi_public(hc, HELM_OP_A, v, e1, z, nrhs, real_bytes, gate, s);
  }
  set_error("unknown U-Net preconditioner kind");
  return HELM_EINVAL;
}

void unet_release_ctx(helm_ctx*) {}

void unet_graph_ids(void* netp, unsigned long long ids[4]) {
  const unet_ctx* n = (const unet_ctx*)netp;
  ids[0] = n ? n->uid : 0;
  ids[1] = n ? n->ws_gen : 0;
  ids[2] = (n && n->encoder) ? n->encoder->uid : 0;
  ids[3] = (n && n->encoder) ? n->encoder->ws_gen : 0;
}

int unet_prepare_impl(helm_ctx* hc, void* netp, int nrhs) {
  unet_ctx* n = (unet_ctx*)netp;
  if (!n) { set_error("null net"); return HELM_EINVAL; }
  int nx, ny, abc_w;
  double h, gmax;
  const float *k2f, *gam;
  helm_geometry(hc, &nx, &ny, &h, &abc_w, &gmax, &k2f, &gam);
  const int cb = apply_chunk(n, nrhs, ny, nx);
  if (cb == 0) { set_error("grid too large for one U-Net image"); return HELM_EUNSUPPORTED; }
  UTRY(ensure_ws(n, cb, ny, nx));
  ensure_eval_coeffs(n, 0);
  if (n->encoder) ensure_eval_coeffs(n->encoder, 0);
  UCHECK(cudaDeviceSynchronize());
  return HELM_OK;
}

// ===========================================================================
// C ABI
// ===========================================================================
void unet_cfg_of(unet_t n, unet_cfg* cfg) {
  if (n && cfg) *cfg = n->cfg;
}

extern "C" {

int unet_cfg_default(unet_cfg* cfg, int kind) {
  if (!cfg) { set_error("null cfg"); return HELM_EINVAL; }
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->levels = 4;
  cfg->coarse_resnets = 3;
  const int wd[4] = {32, 64, 128, 256};
  for (int i = 0; i < 4; ++i) cfg->widths[i] = wd[i];
  if (kind == UNET_ENCODER) { cfg->in_ch = 2; cfg->out_ch = 4; }
  else { cfg->in_ch = 4; cfg->out_ch = 2; }
  if (kind == UNET_SOLVER) {
    cfg->context[0] = 4;
    for (int l = 1; l < 4; ++l) cfg->context[l] = wd[l - 1];
    cfg->context[4] = wd[3];
  }
  return HELM_OK;
}

int unet_create(const unet_cfg* cfg, unsigned long long seed, unet_t* out) {
  if (!cfg || !out) { set_error("null argument"); return HELM_EINVAL; }
  if (cfg->levels < 1 || cfg->levels > 8 || cfg->in_ch < 1 || cfg->out_ch < 1 || cfg->coarse_resnets < 1) {
    set_error("bad U-Net configuration");
    return HELM_EINVAL;
  }
  for (int l = 0; l < cfg->levels; ++l)
    if (cfg->widths[l] < 1 || cfg->widths[l] > 512) { set_error("bad width"); return HELM_EINVAL; }
  static std::atomic<unsigned long long> next_uid{1};
  unet_ctx* n = new unet_ctx();
  n->uid = next_uid++;
  n->cfg = *cfg;
  build_layout(n);
  const size_t np = n->nparams, nb = n->nbn;
  UCHECK(cudaMalloc(&n->P, np * 4));
  UCHECK(cudaMalloc(&n->G, np * 4));
  UCHECK(cudaMalloc(&n->M1, np * 4));
  UCHECK(cudaMalloc(&n->M2, np * 4));
  UCHECK(cudaMalloc(&n->Wb, np * 2));
  UCHECK(cudaMalloc(&n->WTb, np * 2));
  UCHECK(cudaMalloc(&n->WPb, n->nwp * 2));
  UCHECK(cudaMalloc(&n->WPAb, n->nwpa * 2));
  UCHECK(cudaMalloc(&n->WSb, std::max<size_t>(n->nws, 1) * 2));
  if (cfg->in_ch == 4 && cfg->context[0] == 0)
    UCHECK(cudaMalloc(&n->WDb, conv_tma_weight_s2d_elems(cfg->widths[0]) * 2));
  UCHECK(cudaMalloc(&n->d_err, sizeof(int)));
  UCHECK(cudaMemset(n->d_err, 0, sizeof(int)));
  n->use_tc = !(cfg->flags & UNET_FLAG_SIMT);
  n->use_tma = !(cfg->flags & UNET_FLAG_NO_TMA);
  UCHECK(cudaMalloc(&n->rstats, 2 * nb * 4));
  UCHECK(cudaMalloc(&n->bn_scale, nb * 4));
  UCHECK(cudaMalloc(&n->bn_shift, nb * 4));
  UCHECK(cudaMalloc(&n->bn_mean, nb * 8));
  UCHECK(cudaMalloc(&n->ev_scale, nb * 4));
  UCHECK(cudaMalloc(&n->ev_shift, nb * 4));
  UCHECK(cudaMalloc(&n->bn_var, nb * 8));
  UCHECK(cudaMemset(n->G, 0, np * 4));
  UCHECK(cudaMemset(n->M1, 0, np * 4));
  UCHECK(cudaMemset(n->M2, 0, np * 4));
  // He-normal weights from SplitMix64 + Box-Muller (layer i uses stream seed*1000+i,
  // as the oracle's init_params), BN gamma 1 / beta 0, running mean 0 / var 1.
  std::vector<float> hp(np, 0.f);
  for (size_t i = 0; i < n->convs.size(); ++i) {
    const ConvL& cl = n->convs[i];
    const size_t cnt = (size_t)cl.k * cl.k * cl.cin * cl.cout;
    const double stdv = std::sqrt(2.0 / (cl.k * cl.k * cl.cin));
    const unsigned long long st = seed * 1000ull + i;
    auto sm = [&](unsigned long long idx) {
      unsigned long long z = st + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (size_t q = 0; q < cnt; q += 2) {
      const double u1 = sm(q), u2 = sm(q + 1);
      const double rad = std::sqrt(-2.0 * std::log(u1));
      hp[cl.woff + q] = (float)(rad * std::cos(2.0 * M_PI * u2) * stdv);
      if (q + 1 < cnt) hp[cl.woff + q + 1] = (float)(rad * std::sin(2.0 * M_PI * u2) * stdv);
    }
  }
  for (auto& b : n->bns)
    for (int c = 0; c < b.c; ++c) hp[b.goff + c] = 1.f;
  UCHECK(cudaMemcpy(n->P, hp.data(), np * 4, cudaMemcpyHostToDevice));
  std::vector<float> rs(2 * nb, 0.f);
  std::fill(rs.begin() + nb, rs.end(), 1.f);
  UCHECK(cudaMemcpy(n->rstats, rs.data(), 2 * nb * 4, cudaMemcpyHostToDevice));
  refresh_bf16(n, 0);
  UCHECK(cudaDeviceSynchronize());
  *out = n;
  return HELM_OK;
}

void unet_destroy(unet_t n) {
  if (!n) return;
  cudaDeviceSynchronize();
  free_ws(n);
  for (void* p : {(void*)n->P, (void*)n->G, (void*)n->M1, (void*)n->M2, (void*)n->Wb, (void*)n->WTb, (void*)n->WPb, (void*)n->WPAb, (void*)n->WSb, (void*)n->WDb,
                  (void*)n->d_err, (void*)n->rstats,
                  (void*)n->bn_scale, (void*)n->bn_shift, (void*)n->bn_mean, (void*)n->bn_var, (void*)n->ev_scale,
                  (void*)n->ev_shift, n->tmp_e, (void*)n->gout})
    if (p) cudaFree(p);
  delete n;
}

int unet_sizes(unet_t n, long long* np, long long* nb) {
  if (!n) { set_error("null net"); return HELM_EINVAL; }
  if (np) *np = (long long)n->nparams;
  if (nb) *nb = 2 * (long long)n->nbn;
  return HELM_OK;
}

int unet_set_params(unet_t n, const float* host, long long cnt) {
  if (!n || !host || cnt != (long long)n->nparams) { set_error("bad parameter vector"); return HELM_EINVAL; }
  UCHECK(cudaMemcpy(n->P, host, cnt * 4, cudaMemcpyHostToDevice));
  refresh_bf16(n, 0);
  n->ev_dirty = true;
  UCHECK(cudaDeviceSynchronize());
  return HELM_OK;
}
int unet_get_params(unet_t n, float* host, long long cnt) {
  if (!n || !host || cnt != (long long)n->nparams) { set_error("bad parameter vector"); return HELM_EINVAL; }
  UCHECK(cudaMemcpy(host, n->P, cnt * 4, cudaMemcpyDeviceToHost));
  return HELM_OK;
}
int unet_set_bn_stats(unet_t n, const float* host, long long cnt) {
  if (!n || !host || cnt != 2 * (long long)n->nbn) { set_error("bad BN vector"); return HELM_EINVAL; }
  UCHECK(cudaMemcpy(n->rstats, host, cnt * 4, cudaMemcpyHostToDevice));
  n->ev_dirty = true;
  return HELM_OK;
}
int unet_get_bn_stats(unet_t n, float* host, long long cnt) {
  if (!n || !host || cnt != 2 * (long long)n->nbn) { set_error("bad BN vector"); return HELM_EINVAL; }
  UCHECK(cudaMemcpy(host, n->rstats, cnt * 4, cudaMemcpyDeviceToHost));
  return HELM_OK;
}
int unet_time_layer(unet_t n, int layer, int reps, helm_stream_t stream, float* ms, double* flops, int* tc) {
  if (!n || !ms || !flops || !tc || reps < 1 || layer < 0 || layer >= (int)n->convs.size() || !n->ws) {
    set_error("bad arguments (a forward must run first)");
    return HELM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const ConvL& cl = n->convs[layer];
  const unet_cfg& c = n->cfg;
  const int* w = c.widths;
  const int L = n->L;
  // reconstruct the layer's geometry from its name (inputs are whatever the buffers hold)
  int lvl = 0;
  if (cl.name.rfind("down", 0) == 0) lvl = std::stoi(cl.name.substr(4));
  else if (cl.name.rfind("res", 0) == 0) lvl = std::stoi(cl.name.substr(3, cl.name.find('.') - 3));
  else lvl = std::stoi(cl.name.substr(2));
  int H = 0, W = 0;
  ConvArgs a{};
  if (cl.kind == 0) {
    H = n->ny >> (lvl - 1); W = n->nx >> (lvl - 1);
    Src src = lvl == 1 ? Src{n->x_in, c.in_ch, xin_ld(n), false} : Src{n->cat[lvl - 1] + w[lvl - 2], w[lvl - 2], 2 * w[lvl - 2], false};
    a = conv_args(n, cl, src, feat_of(n, lvl - 1), false, H, W, n->zdown[lvl], w[lvl - 1]);
  } else if (cl.kind == 1) {
    H = n->ny >> lvl; W = n->nx >> lvl;
    a = conv_args(n, cl, Src{n->h0[lvl], w[lvl - 1], w[lvl - 1], false}, Src{nullptr, 0, 0, false}, false, H, W,
                  n->t1[lvl][0], w[lvl - 1]);
  } else {
    H = n->ny >> lvl; W = n->nx >> lvl;
    // the forward's sources (eLU on load), then the same materialisation decision
    const Src u = lvl == L ? Src{n->hL, w[L - 1], w[L - 1], false}
                           : Src{n->cat[lvl], 2 * w[lvl - 1], 2 * w[lvl - 1], false};
    const Src f = feat_of(n, lvl);
    a = conv_args(n, cl, u, f, true, H, W, lvl >= 2 ? n->zup[lvl] : n->out, lvl >= 2 ? w[lvl - 2] : c.out_ch);
    if (lvl == 1) a.bias = n->P + n->bias_off;
    a = act_inputs(n, a, lvl, u, f, H, W, n->B * H * W, s);
  }
  const double taps_eff = cl.kind == 2 ? (double)cl.k * cl.k / 4.0 : (double)cl.k * cl.k;
  *flops = 2.0 * (double)n->B * a.Ho * a.Wo * taps_eff * cl.cin * cl.cout;
  // the inference form of the layer: BatchNorm (+ eLU) into BF16 as the forward does it
  // (this overwrites the layer's activation buffer; the next forward rewrites it)
  const int Ml = n->B * a.Ho * a.Wo;
  auto launch = [&](cudaStream_t st) {
    if (cl.kind == 0) conv_bn(n, a, cl.name + ".bn", true, n->h0[lvl], w[lvl - 1], Ml, false, st);
    else if (cl.kind == 1) {
      const bool second = cl.name.compare(cl.name.size() - 2, 2, "k2") == 0;
      conv_bn(n, a, cl.name.substr(0, cl.name.size() - 2) + (second ? "bn2" : "bn1"), true, n->a1[lvl][0],
              w[lvl - 1], Ml, false, st);
    } else if (lvl >= 2) {
      conv_bn(n, a, cl.name + ".bn", false, n->cat[lvl - 1], 2 * w[lvl - 2], Ml, false, st);
    } else {
      run_conv(n, a, st);
    }
  };
  launch(s);  // warm-up (also settles the inference BatchNorm coefficients)
  *tc = n->last_path;
  UCHECK(cudaStreamSynchronize(s));
  // device time without host launch overhead: the repetitions replay as one CUDA graph
  cudaStream_t cs = nullptr;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float t = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int r = 0; r < reps; ++r) launch(cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, cs);   // warm replay
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, cs);
  if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  if (cs) cudaStreamDestroy(cs);
  UCHECK(e);
  *ms = t / reps;
  UCHECK(cudaGetLastError());
  return HELM_OK;
}

int unet_status(unet_t n, int* failed) {
  if (!n || !failed) { set_error("bad arguments"); return HELM_EINVAL; }
  UCHECK(cudaDeviceSynchronize());
  UCHECK(cudaMemcpy(failed, n->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  UCHECK(cudaMemset(n->d_err, 0, sizeof(int)));
  // a kernel that gave up may have left split-K tickets taken
  if (*failed && n->splitcnt) UCHECK(cudaMemset(n->splitcnt, 0, kSplitTickets * sizeof(int)));
  return HELM_OK;
}

int unet_wait_probe(unet_t n, long long rounds, int arrive, helm_stream_t stream) {
  if (!n || rounds < 1 || rounds > (1ll << 20) || (arrive != 0 && arrive != 1)) {
    set_error("unet_wait_probe: bad arguments (1 <= rounds <= 2^20, arrive 0 or 1)");
    return HELM_EINVAL;
  }
  if (!conv_wait_probe(n->d_err, rounds, arrive, (cudaStream_t)stream)) {
    set_error("unet_wait_probe: launch failed");
    return HELM_ECUDA;
  }
  return HELM_OK;
}

int unet_train_step(unet_t n, helm_t h, const float* x, const float* target, int B, const unet_train_opts* opt,
                    float* loss_dev, helm_stream_t stream) {
  if (!n || !h || !x || !opt || B < 1 || (opt->loss != UNET_LOSS_MSE && opt->loss != UNET_LOSS_RESIDUAL) ||
      (opt->loss == UNET_LOSS_MSE && !target) || !(opt->lr > 0.f)) {
    set_error("unet_train_step: bad arguments");
    return HELM_EINVAL;
  }
  int nx, ny, abc_w;
  double hh, gmax;
  const float *k2f, *gam;
  helm_geometry(h, &nx, &ny, &hh, &abc_w, &gmax, &k2f, &gam);
  if (helm_media(h, nullptr) > 1) {
    set_error("this entry point needs a handle of one medium (helm_setup)");
    return HELM_EUNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (n->encoder) UTRY(unet_encode(n, h, 1, stream));
  UTRY(unet_zero_grad(n, stream));
  UTRY(unet_forward(n, x, nullptr, B, ny, nx, 1, stream));
  const size_t nout = (size_t)B * ny * nx * n->cfg.out_ch;
  if (n->gout_n < nout) {
    if (n->gout) cudaFree(n->gout);
    n->gout = nullptr;
    n->gout_n = 0;
    UCHECK(cudaMalloc(&n->gout, nout * sizeof(float) + 256));
    n->gout_n = nout;
  }
  float* loss = loss_dev ? loss_dev : n->gout + nout;   // the spare float past the gradient
  if (opt->loss == UNET_LOSS_MSE) UTRY(unet_mse(n->out, target, (long long)nout, B, n->gout, loss, stream));
  else UTRY(unet_residual_loss(h, n->out, x, B, n->gout, loss, stream));
  UTRY(unet_backward(n, n->gout, nullptr, stream));
  UTRY(unet_adam_step(n, opt->lr, opt->beta1, opt->beta2, opt->eps, stream));
  (void)s;
  return HELM_OK;
}

int unet_get_grads(unet_t n, float* host, long long cnt) {
  if (!n || !host || cnt != (long long)n->nparams) { set_error("bad gradient vector"); return HELM_EINVAL; }
  UCHECK(cudaMemcpy(host, n->G, cnt * 4, cudaMemcpyDeviceToHost));
  return HELM_OK;
}
int unet_zero_grad(unet_t n, helm_stream_t stream) {
  if (!n) { set_error("null net"); return HELM_EINVAL; }
  UCHECK(cudaMemsetAsync(n->G, 0, n->nparams * 4, (cudaStream_t)stream));
  if (n->encoder) UCHECK(cudaMemsetAsync(n->encoder->G, 0, n->encoder->nparams * 4, (cudaStream_t)stream));
  return HELM_OK;
}

int unet_forward(unet_t n, const float* x, float* out, int B, int ny, int nx, int train, helm_stream_t stream) {
  if (!n || !x || B < 1) { set_error("bad arguments"); return HELM_EINVAL; }
  const int div = 1 << n->L;
  if (ny % div || nx % div || ny <= 0 || nx <= 0) { set_error("ny, nx must be positive multiples of 2^levels"); return HELM_EINVAL; }
  if (n->cfg.context[0]) {
    if (!n->encoder || !n->encoder->ws) { set_error("solver net needs an attached encoder that has run"); return HELM_EINVAL; }
    if (n->encoder->ny != ny || n->encoder->nx != nx || (n->encoder->B != 1 && n->encoder->B != B)) {
      set_error("encoder features do not match the solver input");
      return HELM_EINVAL;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  UTRY(ensure_ws(n, B, ny, nx));
  if (!train && s2d_input(n)) {
    to_bf16_s2d(x, n->cfg.in_ch, n->xs2d, B, ny, nx, s);
    n->xs2d_valid = true;
  } else {
    to_bf16_slice(x, n->cfg.in_ch, n->x_in, xin_ld(n), n->cfg.in_ch, B * ny * nx, s);
    n->xs2d_valid = false;
  }
  UTRY(forward_impl(n, train != 0, s));
  if (out) UCHECK(cudaMemcpyAsync(out, n->out, (size_t)B * ny * nx * n->cfg.out_ch * 4, cudaMemcpyDeviceToDevice, s));
  return HELM_OK;
}

int unet_backward(unet_t n, const float* gout, float* gx, helm_stream_t stream) {
  if (!n || !gout) { set_error("bad arguments"); return HELM_EINVAL; }
  if (!n->last_train) { set_error("backward needs a train-mode forward first"); return HELM_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  UTRY(backward_impl(n, gout, nullptr, gx, s));
  if (n->encoder) UTRY(backward_encoder(n, s));
  return HELM_OK;
}

int unet_mse(const float* out, const float* target, long long cnt, int B, float* gout, float* loss_dev,
             helm_stream_t stream) {
  if (!out || !target || !gout || !loss_dev || cnt <= 0 || B < 1) { set_error("bad arguments"); return HELM_EINVAL; }
  // reduction scratch: one buffer per device (a device pointer is valid on its own device only)
  static DeviceOnce once;
  float* part = (float*)(uintptr_t)device_once(once, []() -> long long {
    void* p = nullptr;
    if (cudaMalloc(&p, 256 * 4) != cudaSuccess) { cudaGetLastError(); return 0; }
    return (long long)(uintptr_t)p;
  }, 0);
  if (!part) { set_error("unet_mse: scratch allocation failed"); return HELM_ENOMEM; }
  mse_loss(out, target, (size_t)cnt, B, gout, part, loss_dev, (cudaStream_t)stream);
  UCHECK(cudaGetLastError());
  return HELM_OK;
}

int unet_adam_step(unet_t n, float lr, float b1, float b2, float eps, helm_stream_t stream) {
  if (!n) { set_error("null net"); return HELM_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  for (unet_ctx* m : {n, n->encoder}) {
    if (!m) continue;
    m->adam_t += 1;
    adam_update(m->P, m->G, m->M1, m->M2, m->nparams, lr, b1, b2, eps, m->adam_t, s);
    refresh_bf16(m, s);
    m->ev_dirty = true;
  }
  UCHECK(cudaGetLastError());
  return HELM_OK;
}

int unet_attach_encoder(unet_t solver, unet_t encoder) {
  if (!solver) { set_error("null solver"); return HELM_EINVAL; }
  if (encoder) {
    for (int l = 0; l <= solver->L; ++l) {
      int need = solver->cfg.context[l], have;
      if (l == 0) have = encoder->cfg.out_ch;
      else if (l == encoder->L) have = encoder->cfg.widths[l - 1];
      else have = encoder->cfg.widths[l - 1];
      if (encoder->L != solver->L || need != have) { set_error("encoder features do not match solver context"); return HELM_EINVAL; }
    }
  }
  solver->encoder = encoder;
  if (encoder) encoder->is_encoder = true;
  return HELM_OK;
}

int unet_encode(unet_t solver, helm_t h, int train, helm_stream_t stream) {
  if (!solver || !solver->encoder || !h) { set_error("solver with an attached encoder and a handle needed"); return HELM_EINVAL; }
  unet_ctx* e = solver->encoder;
  int nx, ny, abc_w;
  double hh, gmax;
  const float *k2f, *gam;
  helm_geometry(h, &nx, &ny, &hh, &abc_w, &gmax, &k2f, &gam);
  if (helm_media(h, nullptr) > 1) { set_error("the encoder runs on a handle of one medium"); return HELM_EUNSUPPORTED; }
  if (e->cfg.in_ch != 2) { set_error("encoder must take 2 inputs (kappa^2, gamma)"); return HELM_EINVAL; }
  cudaStream_t s = (cudaStream_t)stream;
  UTRY(ensure_ws(e, 1, ny, nx));
  float* med = e->xin32;  // [ny*nx][2] float32 staging
  UCHECK(cudaMemcpy2DAsync(med, 8, k2f, 4, 4, (size_t)nx * ny, cudaMemcpyDeviceToDevice, s));
  UCHECK(cudaMemcpy2DAsync(med + 1, 8, gam, 4, 4, (size_t)nx * ny, cudaMemcpyDeviceToDevice, s));
  to_bf16_slice(med, 2, e->x_in, xin_ld(e), 2, nx * ny, s);
  e->xs2d_valid = false;
  return forward_impl(e, train != 0, s);
}

int unet_make_batch(helm_t h, const void* r, const void* e, int npairs, int count, int nmix, const int* idx,
                    const double* coef, float* x, float* target, helm_stream_t stream) {
  if (!h || !r || !e || !idx || !coef || !x || !target || count < 1 || nmix < 1 || npairs < 1) {
    set_error("bad arguments");
    return HELM_EINVAL;
  }
  for (long long q = 0; q < (long long)count * nmix; ++q)
    if (idx[q] < 0 || idx[q] >= npairs) { set_error("pair index out of range"); return HELM_EINVAL; }
  int nx, ny, abc_w;
  double hh, gmax;
  const float *k2f, *gam;
  helm_geometry(h, &nx, &ny, &hh, &abc_w, &gmax, &k2f, &gam);
  if (helm_media(h, nullptr) > 1) {
    set_error("this entry point needs a handle of one medium (helm_setup)");
    return HELM_EUNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nq = (size_t)count * nmix;
  int* d_idx = nullptr;
  double2* d_coef = nullptr;
  UCHECK(cudaMallocAsync(&d_idx, nq * sizeof(int), s));
  UCHECK(cudaMallocAsync(&d_coef, nq * sizeof(double2), s));
  UCHECK(cudaMemcpyAsync(d_idx, idx, nq * sizeof(int), cudaMemcpyHostToDevice, s));
  UCHECK(cudaMemcpyAsync(d_coef, coef, nq * sizeof(double2), cudaMemcpyHostToDevice, s));
  make_batch((const double2*)r, (const double2*)e, (size_t)nx * ny, count, d_idx, d_coef, nmix, hh, k2f, gam, x, target, s);
  cudaFreeAsync(d_idx, s);
  cudaFreeAsync(d_coef, s);
  UCHECK(cudaGetLastError());
  UCHECK(cudaStreamSynchronize(s));   // the host arrays may be released by the caller
  return HELM_OK;
}

int unet_residual_loss(helm_t h, const float* out, const float* x, int B, float* gout, float* loss_dev,
                       helm_stream_t stream) {
  if (!h || !out || !x || !gout || !loss_dev || B < 1 || out == gout) {
    set_error("bad arguments");
    return HELM_EINVAL;
  }
  if (helm_stencil(h) != HELM_STENCIL_5PT) {
    set_error("the residual loss is built for the 5-point stencil only");
    return HELM_EUNSUPPORTED;
  }
  int nx, ny, abc_w;
  double hh, gmax;
  const float *k2f, *gam;
  helm_geometry(h, &nx, &ny, &hh, &abc_w, &gmax, &k2f, &gam);
  if (helm_media(h, nullptr) > 1) {
    set_error("this entry point needs a handle of one medium (helm_setup)");
    return HELM_EUNSUPPORTED;
  }
  const double om = helm_omega(h);
  cudaStream_t s = (cudaStream_t)stream;
  float *rho = nullptr, *part = nullptr;
  UCHECK(cudaMallocAsync(&rho, (size_t)B * nx * ny * 2 * sizeof(float), s));
  UCHECK(cudaMallocAsync(&part, 256 * sizeof(float), s));
  residual_loss(out, x, B, ny, nx, (float)(hh * hh * om * om), k2f, gam, helm_bc(h), rho, gout, part, loss_dev, s);
  cudaFreeAsync(rho, s);
  cudaFreeAsync(part, s);
  UCHECK(cudaGetLastError());
  return HELM_OK;
}

int unet_precond(helm_t h, unet_t net, int kind, const void* r, void* e, int nrhs, int dtype, helm_stream_t stream) {
  if (!h || !net || !r || !e || r == e || nrhs < 1 || (dtype != HELM_C32 && dtype != HELM_C64)) {
    set_error("bad arguments");
    return HELM_EINVAL;
  }
  return unet_precond_impl(h, net, kind, r, e, nrhs, dtype == HELM_C32 ? 4 : 8, nullptr, (cudaStream_t)stream);
}

}  // extern "C"
