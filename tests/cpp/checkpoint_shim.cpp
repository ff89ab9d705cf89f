// The library's checkpoint reader and writer (paper_2203_11025_gb300/csrc/checkpoint.cu,
// host code only) compiled on the CPU with the host compiler, over a stand-in network
// whose weights and BatchNorm statistics are host arrays: the unet_* accessors the
// checkpoint code calls are defined here instead of by the GPU library.
#include <string>
#include <vector>

#include "checkpoint.cu"

struct unet_ctx {
  unet_cfg cfg;
  std::vector<float> params, bn;
};

namespace helm {
static std::string g_shim_err;
void set_error(const std::string& s) { g_shim_err = s; }
}  // namespace helm

void unet_cfg_of(unet_t n, unet_cfg* cfg) { *cfg = n->cfg; }

extern "C" {

int unet_sizes(unet_t n, long long* np, long long* nb) {
  *np = (long long)n->params.size();
  *nb = (long long)n->bn.size();
  return HELM_OK;
}
int unet_get_params(unet_t n, float* host, long long cnt) {
  if (cnt != (long long)n->params.size()) return HELM_EINVAL;
  std::copy(n->params.begin(), n->params.end(), host);
  return HELM_OK;
}
int unet_set_params(unet_t n, const float* host, long long cnt) {
  if (cnt != (long long)n->params.size()) return HELM_EINVAL;
  std::copy(host, host + cnt, n->params.begin());
  return HELM_OK;
}
int unet_get_bn_stats(unet_t n, float* host, long long cnt) {
  if (cnt != (long long)n->bn.size()) return HELM_EINVAL;
  std::copy(n->bn.begin(), n->bn.end(), host);
  return HELM_OK;
}
int unet_set_bn_stats(unet_t n, const float* host, long long cnt) {
  if (cnt != (long long)n->bn.size()) return HELM_EINVAL;
  std::copy(host, host + cnt, n->bn.begin());
  return HELM_OK;
}

// A stand-in network: cfg, n_params weights and n_bn statistics copied from the arrays.
unet_t shim_new(const unet_cfg* cfg, const float* params, long long np, const float* bn, long long nb) {
  unet_ctx* n = new unet_ctx;
  n->cfg = *cfg;
  n->params.assign(params, params + np);
  n->bn.assign(bn, bn + nb);
  return n;
}
void shim_free(unet_t n) { delete n; }
const char* shim_error() { return helm::g_shim_err.c_str(); }

}  // extern "C"
