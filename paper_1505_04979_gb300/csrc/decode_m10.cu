// Decode kernels for N = 1024 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_m10(const LaunchReq& q) { return launch_decode_pipe<10>(q); }
}  // namespace polarbp
