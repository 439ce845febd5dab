// Decode kernels for N = 512 (instantiations of bp_decode.cuh).
#include "bp_decode.cuh"

namespace polarbp {
cudaError_t launch_m9(const LaunchReq& q) { return launch_decode<9>(q); }
}  // namespace polarbp
