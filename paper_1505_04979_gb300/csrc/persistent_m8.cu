// Persistent decode kernels for N = 256 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_persistent_m8(const SegLaunch& q) { return launch_persistent_pipe<8>(q); }
}  // namespace polarbp
