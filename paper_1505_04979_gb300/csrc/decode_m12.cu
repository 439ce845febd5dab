// Decode kernels for N = 4096 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_m12(const LaunchReq& q) { return launch_decode<12>(q); }
}  // namespace polarbp
