// One-launch mixed-stream decoder whose longest code length is 2^12 (bp_mixed.cuh).
#include "bp_mixed.cuh"

namespace polarbp {
cudaError_t launch_mixed_m12(const MixedArgs& a, int stop_mode, int freeze_mode, int sms, cudaStream_t s)
{
    return launch_mixed<12>(a, stop_mode, freeze_mode, sms, s);
}
}  // namespace polarbp
