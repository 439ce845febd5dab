// checked.cuh -- the shared-memory redzones of the checked build.
//
// Compiled with -DPOLARBP_CHECKED (paper_1505_04979_gb300.build.build(checked=True),
// library libpolarbp_checked.so), every shared-memory layout of the decoders
// puts a redzone of kRedzone bytes before its first region and after each
// region.  A decode fills its redzones with a pattern before its first store
// and compares them once all of its threads are past their last store; a
// changed word means a store left its region.  The decode then sets bit 1 of
// the code's status word and records, in the words after it, the number of
// changed words, the first redzone that held one and its byte offset in the
// layout; polarbp_get_status reports it as POLARBP_ERR_CHECK.  Nothing is
// skipped or clamped: the redzone absorbs the stray store, so the decode runs
// on, and its results are those of the default build unless a store did leave
// its region.
//
// In the default build kRedzone is 0, every layout offset is the one written
// without redzones, and the fill and the comparison compile to nothing.
#pragma once

#include <cstddef>
#include <cstdint>

namespace polarbp {

#ifdef POLARBP_CHECKED
constexpr bool kChecked = true;
constexpr size_t kRedzone = 256;  // bytes; a multiple of 16, so the layouts keep their alignment
#else
constexpr bool kChecked = false;
constexpr size_t kRedzone = 0;
#endif

constexpr uint32_t kRedzoneWord = 0x5a3cc3a5u;

// status word layout: [0] flags (bit 0 non-finite LLR, bit 1 redzone written),
// [1] changed words, [2] (layout id << 8) | zone index of the first, [3] its byte offset
constexpr int kStatusWords = 4;
constexpr unsigned kStatusRedzone = 2u;

// Layout ids of the record, one per layout struct: SmemLayout (zones 0..10),
// the buffers PipeLayout adds (zones 0..1), those CLayout adds (zones 0..9).
enum : int { kLayoutBlock = 1, kLayoutPipe = 2, kLayoutCluster = 3 };

// Fill (FILL) or compare the redzone that starts at byte `off` of `base`, with the
// threads [tid, tid + stride, ...); `zone` identifies it in the record.
template <bool FILL>
__device__ __forceinline__ void redzone_pass(unsigned char* base, size_t off, int layout, int zone,
                                             unsigned int* status, int tid, int stride)
{
    if constexpr (kRedzone > 0) {
        uint32_t* w = reinterpret_cast<uint32_t*>(base + off);
        for (int i = tid; i < (int)(kRedzone / 4); i += stride) {
            if constexpr (FILL) {
                w[i] = kRedzoneWord;
            } else if (w[i] != kRedzoneWord) {
                if (atomicAdd(status + 1, 1u) == 0u) {
                    status[2] = (unsigned)((layout << 8) | zone);
                    status[3] = (unsigned)(off + 4 * (size_t)i);
                }
                atomicOr(status, kStatusRedzone);
            }
        }
    }
}

}  // namespace polarbp
