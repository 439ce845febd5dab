// Decode kernels for N = 2048 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_m11(const LaunchReq& q) { return launch_decode<11>(q); }
}  // namespace polarbp
