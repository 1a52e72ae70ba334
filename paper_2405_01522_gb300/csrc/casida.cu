// Tamm-Dancoff Casida calls of the C ABI (work in progress: not yet available).
#include "../../include/rsx.h"
#include "api_internal.cuh"

using namespace rsx;

extern "C" {

int rsx_casida_K(rsx_ctx* c, const void*, int, const void*, int, double*, void*) {
  if (!c) return RSX_EINVAL;
  return set_error(c, RSX_EUNSUPPORTED, "casida_K not available in this build");
}

int rsx_casida_Kd(rsx_ctx* c, const void*, int, const void*, int, double*, void*) {
  if (!c) return RSX_EINVAL;
  return set_error(c, RSX_EUNSUPPORTED, "casida_Kd not available in this build");
}

int rsx_casida_solve(rsx_ctx* c, const double*, int, const double*, int, const double*, const double*, double,
                     int, double*, double*, void*) {
  if (!c) return RSX_EINVAL;
  return set_error(c, RSX_EUNSUPPORTED, "casida_solve not available in this build");
}

}  // extern "C"
