// Decode kernels for N = 512 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_m9(const LaunchReq& q) { return launch_decode_pipe<9>(q); }
}  // namespace polarbp
