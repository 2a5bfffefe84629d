// World-space fit and parameter backward (temporary: not yet implemented).
#include "srn_fit.h"

namespace srn {
cudaError_t fit_scratch_alloc(FitScratch& s, const NetDev&, int max_points) {
  memset(&s, 0, sizeof(s));
  s.max_points = max_points;
  return cudaSuccess;
}
void fit_scratch_free(FitScratch& s) { memset(&s, 0, sizeof(s)); }
cudaError_t launch_backward(FitScratch&, const NetDev&, const float*, int, float, const float*, float*, float*, float*,
                            cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_fit_step(FitScratch&, const NetDev&, const FitArgs&, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace srn
