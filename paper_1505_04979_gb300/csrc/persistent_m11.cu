// Persistent decode kernels for N = 2048 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_persistent_m11(const SegLaunch& q) { return launch_persistent_pipe<11>(q); }
}  // namespace polarbp
