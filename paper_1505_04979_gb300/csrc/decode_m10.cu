// Decode kernels for N = 1024 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_m10(const LaunchReq& q) { return launch_decode<10>(q); }
}  // namespace polarbp
