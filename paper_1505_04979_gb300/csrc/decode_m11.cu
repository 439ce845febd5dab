// Decode kernels for N = 2048 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_m11(const LaunchReq& q) { return launch_decode_pipe<11>(q); }
}  // namespace polarbp
