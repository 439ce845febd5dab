// Persistent decode kernels for N = 1024 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_persistent_m10(const SegLaunch& q) { return launch_persistent_pipe<10>(q); }
}  // namespace polarbp
