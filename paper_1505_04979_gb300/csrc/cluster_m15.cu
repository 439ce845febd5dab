// Decode kernels for N = 32768: clusters of 8 thread blocks (instantiations of bp_cluster.cuh).
#include "bp_cluster.cuh"

namespace polarbp {
cudaError_t launch_m15(const LaunchReq& q) { return launch_cluster<3>(q); }
}  // namespace polarbp
