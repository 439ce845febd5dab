// Persistent decode kernels for N = 4096 (instantiations of bp_decode.cuh and bp_pipe.cuh).
#include "bp_pipe.cuh"

namespace polarbp {
cudaError_t launch_persistent_m12(const SegLaunch& q) { return launch_persistent_pipe<12>(q); }
}  // namespace polarbp
