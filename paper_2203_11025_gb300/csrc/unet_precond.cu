// U-Net preconditioners M_JU (Alg. 2) and M_VU (Eq. 3.4).
#include <string>

#include "../../include/helm.h"
#include "unet_api.h"

namespace helm { void set_error(const std::string& s); }

int unet_precond_impl(helm_ctx*, void*, int, const void*, void*, int, int, const int*, cudaStream_t) {
  helm::set_error("U-Net preconditioners are not available in this build");
  return HELM_EUNSUPPORTED;
}
void unet_release_ctx(helm_ctx*) {}
