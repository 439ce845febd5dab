// Decode kernels for N = 4096 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_m12(const LaunchReq& q) { return launch_decode_pipe<12>(q); }
}  // namespace polarbp
