// bp_mixed.cuh -- one persistent launch over a mixed stream of code lengths
// N = 256 .. 4096 (the same decode as polarbp_decode, per codeword).
//
// Method: arXiv 1505.04979, Eq. (1) (Sec. II-A), the CSFG freezing of Sec. III
// and the G-matrix stop; each codeword is decoded by decode_codeword of
// bp_decode.cuh (or, for N = 4096 with freezing, decode_pipe_codeword of
// bp_pipe.cuh) and retires at its own stop.
//
// Shape.  The launch is specialised on the longest length 2^MT in the stream.
// A block has Geo<MT>::BLOCK threads and 8800 x 2^(MT-8) bytes of shared
// memory.  It drains the device queues longest first: the whole block takes
// codewords of length 2^MT one at a time; once that queue is empty it splits
// into 2 groups for length 2^(MT-1), each of those into 2 for 2^(MT-2), and so
// on down to N = 256 (one warp per codeword).  A group of length 2^M owns the
// slice 8800 x 2^(M-8) of its index; that slice holds SmemLayout<M> and is the
// union of the slices of the two groups it splits into, so a group moves on to
// the next length as soon as its own pops fail, whatever the rest of the block
// does.  Barriers: the block barrier for the top length, named barriers
// 1 + (2^d - 2) + g for the groups g of depth d = MT - M in 1..3 (disjoint, since
// groups of different depths run at once), warp synchronisation for N = 256.
// With freezing and N = 4096 on top, the block has one warp more and decodes the
// N = 4096 codewords pipelined (a checker warp beside the 16 sweep warps, the
// named barriers of bp_pipe.cuh, every one complete before the block barrier
// that ends the length); that warp idles through the shorter lengths.
#pragma once

#include "bp_pipe.cuh"

namespace polarbp {

// bytes of shared memory per N = 256 group (the checked build's redzones need 11 x 256 more)
constexpr int kMixedSlice8 = kChecked ? 8800 + 3072 : 8800;

template <int MT, bool FREEZE>
struct MixedTop {
    static constexpr bool PIPE = FREEZE && MT == 12;  // the top length runs pipelined
    static constexpr int THREADS = PIPE ? PipeGeo<MT>::THREADS : Geo<MT>::BLOCK;
    static constexpr int SLICES = kMixedSlice8 << (MT - 8);
    static constexpr int PBYTES = PIPE ? (int)PipeLayout<MT>::bytes : 0;
    static constexpr int SMEM = PBYTES > SLICES ? PBYTES : SLICES;
    // blocks per SM the kernel is compiled for: 640 threads per SM, the one-length kernels' bound
    // (the tighter bound they take for N = 1024 with freezing spills the shorter lengths' decoders)
    static constexpr int MIN_BLOCKS = (640 / THREADS) < 1 ? 1 : (640 / THREADS);
};

template <int MT, int M>
struct MixedShape {
    static constexpr int BLOCK = Geo<M>::BLOCK;
    static constexpr int CPC = Geo<MT>::BLOCK / BLOCK;
    static constexpr int SLICE = kMixedSlice8 << (M - 8);
    static constexpr int BAR0 = CPC - 2;  // group_sync's named barrier is 1 + BAR0 + g
    static_assert(BLOCK * CPC == Geo<MT>::BLOCK && SLICE * CPC == (kMixedSlice8 << (MT - 8)), "groups tile the block");
    static_assert(SLICE % 32 == 0 && (size_t)SLICE >= SmemLayout<M>::bytes, "a group's slice holds its decoder");
    static_assert(CPC == 1 || BLOCK == 32 || BAR0 + CPC <= 15, "named barriers 1..15");
};

struct MixedArgs {
    SegArgs seg[5];  // index M - 8; total 0 when the stream has no codeword of that length
};

// Drain the queue of length 2^M with this thread's group; returns once the group's pops fail and
// every thread of the group is past its last codeword (the group's slice is then free).
template <int MT, int M, bool GSTOP, bool FREEZE>
__device__ __forceinline__ void mixed_drain(const SegArgs& a, unsigned char* smem_raw)
{
    using SH = MixedShape<MT, M>;
    constexpr int N = Geo<M>::N, BLOCK = SH::BLOCK, CPC = SH::CPC;
    if (a.total == 0) return;
    if (threadIdx.x >= Geo<MT>::BLOCK) return;  // the pipelined top length's checker warp
    const int grp = threadIdx.x / BLOCK;
    const int tid = threadIdx.x % BLOCK;
    const int bar = SH::BAR0 + grp;
    unsigned char* smem = smem_raw + grp * SH::SLICE;
    int* qslot = reinterpret_cast<int*>(smem + SmemLayout<M>::off_Ctl) + CTL_Q;
    for (;;) {
        group_sync<BLOCK, CPC>(bar);  // the previous codeword's readers are done with the slice
        if (tid == 0) *qslot = atomicAdd(a.queue, 1);
        group_sync<BLOCK, CPC>(bar);
        const int q = *qslot;
        if (q >= a.total) break;
        int sg = 0;
        while (sg + 1 < a.nseg && q >= a.start[sg + 1]) ++sg;
        const long long r = q - a.start[sg];
        const CwIO io{a.llr[sg] + r * N,
                      a.frozen_words[sg],
                      a.u_hat[sg] + r * N,
                      a.iters[sg] ? a.iters[sg] + r : nullptr,
                      a.pe[sg] ? a.pe[sg] + r : nullptr,
                      nullptr,
                      nullptr,
                      nullptr,
                      a.bitrev[sg]};
        decode_codeword<M, GSTOP, FREEZE, false, CPC>(io, a.max_iter, a.alpha, a.status[sg], smem, tid, bar);
    }
    group_sync<BLOCK, CPC>(bar);  // every thread of the group has read its last pop
}

// The top length pipelined (bp_pipe.cuh): the whole block takes one codeword at a time.
template <int MT, bool GSTOP>
__device__ __forceinline__ void mixed_drain_pipe(const SegArgs& a, unsigned char* smem_raw)
{
    constexpr int N = Geo<MT>::N;
    if (a.total == 0) return;
    Smem<MT> sm(smem_raw);
    int* qslot = sm.ctl + CTL_Q;
    for (;;) {
        __syncthreads();  // the previous codeword's readers are done with shared memory
        if (threadIdx.x == 0) *qslot = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = *qslot;
        if (q >= a.total) break;
        int sg = 0;
        while (sg + 1 < a.nseg && q >= a.start[sg + 1]) ++sg;
        const long long r = q - a.start[sg];
        const CwIO io{a.llr[sg] + r * N,
                      a.frozen_words[sg],
                      a.u_hat[sg] + r * N,
                      a.iters[sg] ? a.iters[sg] + r : nullptr,
                      a.pe[sg] ? a.pe[sg] + r : nullptr,
                      nullptr,
                      nullptr,
                      nullptr,
                      a.bitrev[sg]};
        __syncthreads();  // every thread has read the popped index before the decode reuses the slot
        decode_pipe_codeword_call<MT, GSTOP>(io, a.max_iter, a.alpha, a.status[sg], smem_raw);
    }
    __syncthreads();  // the shorter lengths reuse the shared memory
}

template <int MT, int M, bool GSTOP, bool FREEZE>
__device__ __forceinline__ void mixed_drain_down(const MixedArgs& a, unsigned char* smem_raw)
{
    if constexpr (M == MT && MixedTop<MT, FREEZE>::PIPE) mixed_drain_pipe<MT, GSTOP>(a.seg[M - 8], smem_raw);
    else mixed_drain<MT, M, GSTOP, FREEZE>(a.seg[M - 8], smem_raw);
    if constexpr (M > 8) mixed_drain_down<MT, M - 1, GSTOP, FREEZE>(a, smem_raw);
}

template <int MT, bool GSTOP, bool FREEZE>
__global__ void __launch_bounds__(MixedTop<MT, FREEZE>::THREADS, MixedTop<MT, FREEZE>::MIN_BLOCKS)
    bp_decode_mixed(MixedArgs a)
{
    extern __shared__ __align__(32) unsigned char smem_raw[];
    mixed_drain_down<MT, MT, GSTOP, FREEZE>(a, smem_raw);
}

template <int MT, bool GSTOP, bool FREEZE>
cudaError_t launch_mixed_one(const MixedArgs& args, int sms, cudaStream_t stream)
{
    auto kern = bp_decode_mixed<MT, GSTOP, FREEZE>;
    constexpr int threads = MixedTop<MT, FREEZE>::THREADS, smem = MixedTop<MT, FREEZE>::SMEM;
    // blocks per SM, per device, set with the shared-memory attribute on the device's first launch
    constexpr int kDevices = 64;
    static std::atomic<int> blocks_per_sm[kDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevices) return cudaErrorInvalidDevice;
    int bps = blocks_per_sm[dev].load(std::memory_order_acquire);
    if (bps == 0) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem);
        if (e != cudaSuccess) return e;
        bps = b > 0 ? b : 1;
        blocks_per_sm[dev].store(bps, std::memory_order_release);
    }
    // no more blocks than the work can fill: a block holds 2^(MT-M) codewords of length 2^M
    long long work = 0;
    for (int k = 0; k <= MT - 8; ++k) {
        const int per_block = 1 << (MT - 8 - k);
        work += (args.seg[k].total + per_block - 1) / per_block;
    }
    long long grid = (long long)bps * sms;
    if (grid > work) grid = work;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, threads, smem, stream>>>(args);
    return cudaGetLastError();
}

template <int MT>
cudaError_t launch_mixed(const MixedArgs& args, int stop_mode, int freeze_mode, int sms, cudaStream_t stream)
{
    const bool g = stop_mode != 0, f = freeze_mode != 0;
    if (g && f) return launch_mixed_one<MT, true, true>(args, sms, stream);
    if (g) return launch_mixed_one<MT, true, false>(args, sms, stream);
    if (f) return launch_mixed_one<MT, false, true>(args, sms, stream);
    return launch_mixed_one<MT, false, false>(args, sms, stream);
}

}  // namespace polarbp
