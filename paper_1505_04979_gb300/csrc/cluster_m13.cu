// Decode kernels for N = 8192: clusters of 2 thread blocks (instantiations of bp_cluster.cuh).
#include "bp_cluster.cuh"

namespace polarbp {
cudaError_t launch_m13(const LaunchReq& q) { return launch_cluster<1>(q); }
}  // namespace polarbp
