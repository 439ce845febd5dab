// bp_decode.cuh -- min-sum BP decoding of polar codes with the G-matrix stop
// and connected-sub-factor-graph (CSFG) freezing, one codeword per thread block.
//
// Method: arXiv 1505.04979.  Eq. (1) (Sec. II-A) is the PE update; Sec. III and
// Eqs. (2)-(4) define the CSFG check, the freezing order and the +-inf feedback;
// Sec. IV defines the PE-update count.
//
// Layout of one decode (N = 2^M, node columns c = 0..M, column 0 = channel side):
//   * Each worker thread owns EL = 8 elements (all N when N < 8).  The M PE
//     stages are grouped into phases of up to three stages; in phase p a thread
//     owns the 8 indices that differ in the phase's three "register bits", so
//     those stages run entirely in registers (a radix-8 butterfly).
//   * L columns that are read and written inside one phase live in registers
//     for the whole decode.  The column between two phases (c = 3, 6, 9, ...)
//     lives in shared memory, as does the R column when it changes owner at a
//     phase boundary (double-buffered, one barrier per boundary).
//   * R is updated in place: stage s turns R[s] into R[s+1] pairwise.
//   * Freezing state is a single integer P: the covered source positions always
//     form the prefix [0, P) (the checked CSFG is the first uncovered one of its
//     stage and covered CSFGs never shrink), so "level-s CSFG of index a is
//     covered" is  a < (P >> (M-s)) << (M-s).
//   * The sweep records hard decisions of the R columns the checks need; after
//     the sweep one warp runs the checks of stages 1..M in order, the G-matrix
//     test and the termination decision.  Running the checks after the sweep
//     gives the same messages as running each right after its stage: a check at
//     stage j only reads R[j], only changes L[j] (and enclosing CSFGs' L) of
//     blocks it covers, and those messages are next read in the following
//     iteration; PEs it would have skipped in the rest of the sweep only write
//     messages of covered CSFGs, which nothing reads again.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "checked.cuh"

namespace polarbp {

constexpr uint32_t kFull = 0xffffffffu;

template <int M_>
struct Geo {
    static constexpr int M = M_;
    static constexpr int N = 1 << M;
    static constexpr int RB = M < 3 ? M : 3;   // register bits per thread
    static constexpr int EL = 1 << RB;         // elements per thread
    static constexpr int T = N / EL;           // worker threads
    static constexpr int NP = (M + 2) / 3;     // phases
    static constexpr int BLOCK = T < 32 ? 32 : T;
    static constexpr int NW = N < 32 ? 1 : N / 32;  // 32-bit words of an N-bit vector
    static constexpr int NB = (M - 1) / 3;          // shared-memory L columns
    static constexpr int MIN_BLOCKS = (640 / BLOCK) < 1 ? 1 : (640 / BLOCK);
    // Blocks per SM the kernels are compiled for (the register bound is 65536 / (blocks x BLOCK)).
    // The freezing kernels spend much of an iteration in one warp (the CSFG walk), so more
    // resident blocks hide more of it: at N = 1024 six blocks of 128 threads (80 registers, no
    // spills) measured 4-6 % faster than five.  At N = 256..2048 otherwise, and for the kernels
    // without freezing, the 640-thread bound measured as fast or faster.
    __host__ __device__ static constexpr int min_blocks(bool freeze) { return (freeze && M == 10) ? 6 : MIN_BLOCKS; }

    __host__ __device__ static constexpr int s0(int p) { return 3 * p; }
    __host__ __device__ static constexpr int cnt(int p) { return (M - 3 * p) < 3 ? (M - 3 * p) : 3; }
    __host__ __device__ static constexpr int lo(int p) { return (p == NP - 1) ? 0 : (M - 3 - 3 * p); }
    __host__ __device__ static constexpr bool is_boundary(int c) { return c > 0 && c < M && (c % 3) == 0; }
    // column M (the source side) lives in shared memory, see Smem::Lm
    __host__ __device__ static constexpr bool is_reg(int c) { return c > 0 && c < M && !is_boundary(c); }
    __host__ __device__ static constexpr int bslot(int c) { return c / 3 - 1; }
    __host__ __device__ static constexpr int rslot(int c)
    {
        int r = 0;
        for (int x = 1; x < c; ++x) r += is_reg(x) ? 1 : 0;
        return r;
    }
    static constexpr int NR = M - NB - 1;          // register columns (1..M-1 less the boundaries)
    static constexpr int NRA = NR > 0 ? NR : 1;    // their array extent
    // Shared-memory layout of the buffers at the boundary between phases b and
    // b+1: entry i sits at i + (i >> padsh(b)).  The shift minimises bank
    // conflicts of the two phases' access patterns (found by enumerating them);
    // with any shift the address of element e of a thread is a per-thread base
    // plus a compile-time offset, so no address arithmetic is spent per access.
    __host__ __device__ static constexpr int padsh(int b)
    {
        return M <= 7 ? 2 : (M <= 9 ? 3 : (b == 0 ? 5 : 3));
    }
    static constexpr int BUF = N + (N >> (M <= 7 ? 2 : 3)) + 4;  // floats per padded buffer
    // hard-decision snapshots: one byte per worker thread per column (bit e =
    // decision on the thread's element e), rows of >= 32 bytes, 32-byte aligned
    static constexpr int HDS = T < 32 ? 32 : T;
    static constexpr int RW = NW < 32 ? 1 : NW / 32;              // words per lane of an N-bit vector
    __host__ __device__ static constexpr int owner(int c) { return (c / 3) < (NP - 1) ? (c / 3) : (NP - 1); }
};

// Global index of element e of thread t in phase PH's mapping: the phase's
// register bits come from e, the other bits (ascending) from t.
template <int M, int PH>
__device__ __forceinline__ int elem_index(int t, int e)
{
    constexpr int lo = Geo<M>::lo(PH);
    constexpr int RB = Geo<M>::RB;
    return (t & ((1 << lo) - 1)) | (e << lo) | ((t >> lo) << (lo + RB));
}

template <int SH>
__host__ __device__ __forceinline__ constexpr int padded(int i) { return i + (i >> SH); }

// Padded address of element e of thread t in phase PH's mapping, for a buffer
// with pad shift SH: the thread part and the element part add up.
template <int M, int PH, int SH>
__device__ __forceinline__ int padded_base(int t)
{
    constexpr int lo = Geo<M>::lo(PH);
    constexpr int RB = Geo<M>::RB;
    const int b = (t & ((1 << lo) - 1)) | ((t >> lo) << (lo + RB));
    return b + (b >> SH);
}
template <int M, int PH, int SH>
__host__ __device__ __forceinline__ constexpr int padded_off(int e)
{
    return (e << Geo<M>::lo(PH)) + ((e << Geo<M>::lo(PH)) >> SH);
}

// alpha * sign(x) sign(y) min(|x|, |y|)  (Eq. (1)).  The magnitude is exact,
// the product by alpha rounds once.  The sign is that of the product x * y,
// whose IEEE sign is the xor of the operands' signs; it is computed on the FMA
// pipe, which leaves the (half-rate) integer/logic pipe two instructions per
// term instead of three.  The one exception, 0 * inf = NaN, only occurs when
// the magnitude is 0, so it can change nothing but the sign of a zero result,
// and the sign of a zero never reaches a nonzero message or a decision.
__device__ __forceinline__ float fms(float x, float y, float alpha)
{
    const float mag = __fmul_rn(alpha, fminf(fabsf(x), fabsf(y)));
    const float p = __fmul_rn(x, y);
    return __uint_as_float(__float_as_uint(mag) | (__float_as_uint(p) & 0x80000000u));
}

struct DecodeArgs {
    const float* llr;
    const uint32_t* frozen_words;  // NW words, bit i of word i/32 = frozen[i]
    uint8_t* u_hat;
    int32_t* iters;
    int64_t* pe;
    unsigned int* status;
    float* trace_L;
    float* trace_R;
    int32_t* trace_P;
    int batch;
    int max_iter;
    float alpha;
    int bitrev;  // 1: the codeword positions arrive in bit-reversed order (channel position i carries x[rev(i)])
};

// Pointers of one codeword (trace pointers already offset to the codeword).
struct CwIO {
    const float* llr;              // [N]
    const uint32_t* frozen_words;  // ceil(N/32) words
    uint8_t* u_hat;                // [N]
    int32_t* iters;                // one entry, or NULL
    int64_t* pe;                   // one entry, or NULL
    float* trace_L;                // [max_iter][M+1][N], or NULL
    float* trace_R;
    int32_t* trace_P;              // [max_iter]
    int bitrev;                    // 1: llr[i] belongs to code position rev(i) (bit reversal of m bits)
};

enum : int { CTL_P = 0, CTL_DONE = 1, CTL_EVENT = 2, CTL_Q = 3, CTL_PE = 4, CTL_EV = 8 };

// Barrier of the CPC-way group of threads that decodes one codeword: the whole
// block when it decodes one codeword, a warp when the group is a warp, else a
// named barrier per group (ids 1..CPC; id 0 is __syncthreads).
template <int BLOCK, int CPC>
__device__ __forceinline__ void group_sync(int grp)
{
    if constexpr (CPC == 1) {
        __syncthreads();
    } else if constexpr (BLOCK == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(BLOCK) : "memory");
    }
}

// Byte offsets of one decode's shared memory.  RZ is the redzone of the checked
// build (0 otherwise): one before the first region and one after each region.
template <int M>
struct SmemLayout {
    using G = Geo<M>;
    static constexpr int N = G::N, NW = G::NW;
    static constexpr size_t RZ = kRedzone;
    static constexpr size_t off_Lb = RZ;
    static constexpr size_t end_Lb = off_Lb + sizeof(float) * G::NB * G::BUF;
    static constexpr size_t off_Rx = end_Lb + RZ;
    static constexpr size_t end_Rx = off_Rx + sizeof(float) * (G::NP > 1 ? 2 : 0) * G::BUF;
    static constexpr size_t off_Llr = (end_Rx + RZ + 15) / 16 * 16;
    static constexpr size_t end_Llr = off_Llr + sizeof(float) * G::N;
    static constexpr size_t off_U = end_Llr + RZ;
    static constexpr size_t end_U = off_U + sizeof(uint32_t) * NW;
    static constexpr size_t off_Fz = end_U + RZ;
    static constexpr size_t end_Fz = off_Fz + sizeof(uint32_t) * NW;
    static constexpr size_t off_Xf = end_Fz + RZ;
    static constexpr size_t end_Xf = off_Xf + sizeof(uint32_t) * (M + 1) * NW;
    static constexpr size_t off_Ctl = (end_Xf + RZ + 15) / 16 * 16;
    static constexpr int CTL_INTS = CTL_EV + 2 * (M + 1);
    static constexpr size_t end_Ctl = off_Ctl + sizeof(int) * CTL_INTS;
    static constexpr size_t off_Hd = (end_Ctl + RZ + 15) / 16 * 16;
    static constexpr size_t hd_bytes = (size_t)(M + 1) * G::HDS;
    static constexpr size_t end_Hd = off_Hd + hd_bytes;
    // two NW-word buffers for the encoding of the channel-side decisions
    static constexpr size_t off_Ge = (end_Hd + RZ + 15) / 16 * 16;
    static constexpr size_t end_Ge = off_Ge + 2 * sizeof(uint32_t) * NW;
    // column M in natural order; 32-byte aligned so each thread's 8 entries load as two float4
    static constexpr size_t off_Lm = (end_Ge + RZ + 31) / 32 * 32;
    static constexpr size_t end_Lm = off_Lm + sizeof(float) * N;
    static constexpr size_t bytes = (end_Lm + RZ + 15) / 16 * 16;
    // redzone k starts at zone(k) (k = 0: before Lb; k >= 1: after the k-th region)
    static constexpr int ZONES = 11;
    __host__ __device__ static constexpr size_t zone(int k)
    {
        return k == 0 ? 0 : k == 1 ? end_Lb : k == 2 ? end_Rx : k == 3 ? end_Llr : k == 4 ? end_U : k == 5 ? end_Fz
             : k == 6 ? end_Xf : k == 7 ? end_Ctl : k == 8 ? end_Hd : k == 9 ? end_Ge : end_Lm;
    }
};

// Fill (FILL) or compare the redzones of a SmemLayout<M> at base.
template <int M, bool FILL>
__device__ __forceinline__ void redzones(unsigned char* base, unsigned int* status, int tid, int stride)
{
    if constexpr (kChecked) {
#pragma unroll 1
        for (int k = 0; k < SmemLayout<M>::ZONES; ++k)
            redzone_pass<FILL>(base, SmemLayout<M>::zone(k), kLayoutBlock, k, status, tid, stride);
    }
}

template <int M>
struct Smem {
    float* Lb;
    float* Rx;
    float* llr;     // channel LLRs, [EL][T] (element e of thread t at e * T + t)
    uint32_t* U;    // stored source bits of covered positions
    uint32_t* Fz;   // frozen mask
    uint32_t* Xf;   // [(M+1)][NW] hard decisions of the latest feedback event per column
    int* ctl;
    uint8_t* hd;    // [(M+1)][HDS] hard-decision snapshots (one byte per thread)
    float* L0;      // column 0 of a sweep that is the lower part of a larger code (else unused)
    uint32_t* Ge;   // [2][NW] encoding of HD(R[0] + L[0]), built during the sweep
    float* Lm;      // [N] column M: the prior (+inf frozen, 0 otherwise) and the stage-M feedback
    __device__ __forceinline__ explicit Smem(unsigned char* base)
    {
        L0 = nullptr;
        using L = SmemLayout<M>;
        Ge = reinterpret_cast<uint32_t*>(base + L::off_Ge);
        Lm = reinterpret_cast<float*>(base + L::off_Lm);
        Lb = reinterpret_cast<float*>(base + L::off_Lb);
        Rx = reinterpret_cast<float*>(base + L::off_Rx);
        llr = reinterpret_cast<float*>(base + L::off_Llr);
        U = reinterpret_cast<uint32_t*>(base + L::off_U);
        Fz = reinterpret_cast<uint32_t*>(base + L::off_Fz);
        Xf = reinterpret_cast<uint32_t*>(base + L::off_Xf);
        ctl = reinterpret_cast<int*>(base + L::off_Ctl);
        hd = base + L::off_Hd;
    }
    __device__ __forceinline__ long long* pe_acc() { return reinterpret_cast<long long*>(ctl + CTL_PE); }
    __device__ __forceinline__ int* ev_lo() { return ctl + CTL_EV; }
    __device__ __forceinline__ int* ev_hi() { return ctl + CTL_EV + (M + 1); }
};

__device__ __forceinline__ uint32_t bit_of(const uint32_t* words, int i) { return (words[i >> 5] >> (i & 31)) & 1u; }

// ---------------------------------------------------------------------------
// warp-level bit-vector helpers for the checks
// A CSFG of S positions (S a power of two) is held by the checker warp as
// packed words: word w = 32 r + lane when S >= 32, else bits [0, S) of v[0] in
// every lane.  Sizes are run-time values so the checker's code stays small.
// ---------------------------------------------------------------------------
// four 0/1 bytes of a word -> 4 bits (byte k -> bit k)
__device__ __forceinline__ uint32_t nib4(uint32_t w) { return (w * 0x01020408u) >> 24; }

__device__ __forceinline__ uint32_t xmask(int h)
{
    return h == 1 ? 0x55555555u : h == 2 ? 0x33333333u : h == 4 ? 0x0F0F0F0Fu : h == 8 ? 0x00FF00FFu : 0x0000FFFFu;
}

__device__ __forceinline__ uint32_t low_mask(int S) { return S >= 32 ? 0xffffffffu : ((1u << S) - 1u); }

// bit e of each of four bytes -> 4 bits (byte k -> bit k)
__device__ __forceinline__ uint32_t nib_bit(uint32_t v, int e) { return (((v >> e) & 0x01010101u) * 0x01020408u) >> 24; }

// Decisions of positions [i0, i0 + 32) (i0 a multiple of 32), in natural
// order, from a snapshot row written in a phase whose register bits start at
// bit lo: byte t holds, in bit e, the decision on element e of thread t, i.e.
// on position (t & (2^lo - 1)) | e << lo | (t >> lo) << (lo + 3).  The
// positions of one word come from 32, 16, 8 or 4 consecutive bytes depending
// on lo.
__device__ __forceinline__ uint32_t hd_word(const uint8_t* row, int lo, int i0)
{
    if (lo == 0) return *reinterpret_cast<const uint32_t*>(row + (i0 >> 3));
    if (lo >= 5) {
        const int t0 = (i0 & ((1 << lo) - 1)) | ((i0 >> (lo + 3)) << lo);
        const int e = (i0 >> lo) & 7;
        const uint4 a = *reinterpret_cast<const uint4*>(row + t0);
        const uint4 b = *reinterpret_cast<const uint4*>(row + t0 + 16);
        return nib_bit(a.x, e) | (nib_bit(a.y, e) << 4) | (nib_bit(a.z, e) << 8) | (nib_bit(a.w, e) << 12) |
               (nib_bit(b.x, e) << 16) | (nib_bit(b.y, e) << 20) | (nib_bit(b.z, e) << 24) | (nib_bit(b.w, e) << 28);
    }
    if (lo == 4) {
        const int t0 = (i0 >> 7) << 4;
        const int e = (i0 >> 4) & 7;
        const uint4 a = *reinterpret_cast<const uint4*>(row + t0);
        const uint32_t l = nib_bit(a.x, e) | (nib_bit(a.y, e) << 4) | (nib_bit(a.z, e) << 8) | (nib_bit(a.w, e) << 12);
        const uint32_t h = nib_bit(a.x, e + 1) | (nib_bit(a.y, e + 1) << 4) | (nib_bit(a.z, e + 1) << 8) |
                           (nib_bit(a.w, e + 1) << 12);
        return l | (h << 16);
    }
    if (lo == 3) {
        const int t0 = (i0 >> 6) << 3;
        const int e = (i0 >> 3) & 7;
        const uint2 a = *reinterpret_cast<const uint2*>(row + t0);
        uint32_t w = 0;
#pragma unroll
        for (int d = 0; d < 4; ++d) w |= (nib_bit(a.x, e + d) | (nib_bit(a.y, e + d) << 4)) << (8 * d);
        return w;
    }
    const uint32_t v = *reinterpret_cast<const uint32_t*>(row + ((i0 >> 5) << 2));
    uint32_t w = 0;
    if (lo == 2) {
#pragma unroll
        for (int e = 0; e < 8; ++e) w |= nib_bit(v, e) << (4 * e);
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const uint32_t n = nib_bit(v, e);
            w |= ((n & 3u) << (2 * e)) | ((n >> 2) << (16 + 2 * e));
        }
    }
    return w;
}

// register-bit base of the phase that writes the snapshot of column c
// (column 0: stage 0's channel-side decisions; column c >= 1: R[c] after stage c-1)
template <int M>
__device__ __forceinline__ int snap_lo(int c)
{
    const int ph = c == 0 ? 0 : (c - 1) / 3;
    return (ph == Geo<M>::NP - 1) ? 0 : (M - 3 - 3 * ph);
}

// Codes of N >= 256 (every phase has whole warps) store the snapshot rows of the
// phases with register bits from bit lo >= 1 as raw ballots (raw_word below) and
// the last phase's rows (lo = 0) as one byte per thread, which is natural order;
// smaller codes keep one byte per thread and gather with hd_word.
template <int M>
__host__ __device__ constexpr bool natural_rows()
{
    return M >= 8;
}

// Decisions of positions [i0, i0 + 32) (i0 a multiple of 32) from a raw ballot
// row: word 8 k + e holds, in bit l, the decision on element e of thread 32 k + l
// of a phase whose register bits start at bit lo >= 1, i.e. on position
// p = (t & (2^lo - 1)) | e << lo | (t >> lo) << (lo + 3), t = 32 k + l.  For
// lo <= 4 the warp is k = p >> 8.
__device__ __forceinline__ uint32_t raw_word(const uint32_t* row, int lo, int i0)
{
    const int q = i0 >> 5;
    if (lo >= 5) {
        // the lanes of a warp hold 32 consecutive positions of each element: one ballot
        const int k = ((i0 & ((1 << lo) - 1)) >> 5) | ((i0 >> (lo + 3)) << (lo - 5));
        return row[8 * k + ((i0 >> lo) & 7)];
    }
    const uint32_t* r = row + 8 * (i0 >> 8);
    if (lo == 4) {
        // positions b < 16 / b >= 16 of the word: elements 2 (q & 3) and + 1, lanes 16 h ..
        const int e = 2 * (q & 3), h = (q >> 2) & 1;
        return __byte_perm(r[e], r[e + 1], h ? 0x7632u : 0x5410u);
    }
    if (lo == 3) {
        // elements 4 (q & 1) .. + 3, byte g of each
        const int e = 4 * (q & 1);
        const uint32_t g = (q >> 1) & 3, sel = g | ((4u + g) << 4);
        return __byte_perm(__byte_perm(r[e], r[e + 1], sel), __byte_perm(r[e + 2], r[e + 3], sel), 0x5410u);
    }
    // lo = 2, 1: nibble g = q & 7 (lanes 4 g .. 4 g + 3) of each of the 8 elements
    const int g4 = 4 * (q & 7);
    uint32_t n[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) n[e] = (r[e] >> g4) & 0xFu;
    const uint32_t x = n[0] | (n[1] << 4) | (n[2] << 8) | (n[3] << 12) | (n[4] << 16) | (n[5] << 20) |
                       (n[6] << 24) | (n[7] << 28);  // position bits 0-1: lane bits 0-1, bits 2-4: element
    if (lo == 2) return x;
    // lo = 1: lane bit 0 is position bit 0, lane bit 1 position bit 4, the element bits 1-3
    uint32_t a = x & 0x33333333u, b = (x >> 2) & 0x33333333u;
    a = (a | (a >> 2)) & 0x0F0F0F0Fu;
    b = (b | (b >> 2)) & 0x0F0F0F0Fu;
    a = (a | (a >> 4)) & 0x00FF00FFu;
    b = (b | (b >> 4)) & 0x00FF00FFu;
    a = (a | (a >> 8)) & 0x0000FFFFu;
    b = (b | (b >> 8)) & 0x0000FFFFu;
    return a | (b << 16);
}

// Decisions of positions [i0, i0 + 32) of snapshot column c.
template <int M>
__device__ __forceinline__ uint32_t snap_word(const uint8_t* hd, int c, int i0)
{
    const uint8_t* row = hd + c * Geo<M>::HDS;
    if constexpr (natural_rows<M>()) {
        const int lo = snap_lo<M>(c);
        if (lo == 0) return reinterpret_cast<const uint32_t*>(row)[i0 >> 5];
        return raw_word(reinterpret_cast<const uint32_t*>(row), lo, i0);
    } else {
        return hd_word(row, snap_lo<M>(c), i0);
    }
}

template <int RW>
__device__ __forceinline__ void packed_load(const uint32_t* words, int base, int S, uint32_t (&v)[RW], int lane)
{
    if (S >= 32) {
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int w = 32 * r + lane;
            v[r] = (w < (S >> 5)) ? words[(base >> 5) + w] : 0u;
        }
    } else {
        v[0] = (words[base >> 5] >> (base & 31)) & low_mask(S);
#pragma unroll
        for (int r = 1; r < RW; ++r) v[r] = 0u;
    }
}

template <int RW>
__device__ __forceinline__ void packed_store(uint32_t* words, int base, int S, const uint32_t (&v)[RW], int lane)
{
    if (S >= 32) {
#pragma unroll
        for (int r = 0; r < RW; ++r) {
            const int w = 32 * r + lane;
            if (w < (S >> 5)) words[(base >> 5) + w] = v[r];
        }
    } else if (lane == 0) {
        const uint32_t mask = low_mask(S) << (base & 31);
        uint32_t* p = words + (base >> 5);
        *p = (*p & ~mask) | ((v[0] << (base & 31)) & mask);
    }
}

// v <- v . F^{(x) log2 S}: for every bit h of the position, entries with bit h
// clear absorb (xor) the entry with bit h set.
template <int RW>
__device__ __forceinline__ void polar_xform(uint32_t (&v)[RW], int S, int lane)
{
    const int inw = S < 32 ? S : 32;
#pragma unroll 1
    for (int h = 1; h < inw; h <<= 1) {
        const uint32_t mk = xmask(h);
#pragma unroll
        for (int r = 0; r < RW; ++r) v[r] ^= (v[r] >> h) & mk;
    }
    const int W = S >> 5;
#pragma unroll 1
    for (int d = 1; d < W; d <<= 1) {
        if (d < 32) {
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                const uint32_t y = __shfl_xor_sync(kFull, v[r], d);
                if (!(lane & d)) v[r] ^= y;
            }
        } else {
            const int dr = d >> 5;
#pragma unroll
            for (int r = 0; r < RW; ++r) {
                if (!(r & dr) && r + dr < RW) v[r] ^= v[r + dr];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// checker warp
// ---------------------------------------------------------------------------
// Record the feedback event [lo, hi) on column J.  Under reading B a column can
// take several events in one iteration; they are consecutive CSFGs (P only
// grows, and by steps no larger than the column's CSFGs), so the range grows.
template <int M>
__device__ __forceinline__ void note_event(Smem<M>& sm, int J, int lo, int hi, int lane, bool multi = false)
{
    if (lane == 0) {
        if (!multi || !(sm.ctl[CTL_EVENT] & (1 << J))) sm.ev_lo()[J] = lo;
        sm.ev_hi()[J] = hi;
        sm.ctl[CTL_EVENT] |= 1 << J;
    }
}

// After a freeze that ended at P on stage J, freeze every enclosing CSFG that
// has become fully covered: its hard decision is its stored source bits
// re-encoded (the +-inf messages its own PEs would emit).
template <int M>
__device__ __forceinline__ void propagate(Smem<M>& sm, int P, int J, int lane, bool multi = false)
{
    constexpr int N = Geo<M>::N, NW = Geo<M>::NW, RW = Geo<M>::RW;
#pragma unroll 1
    for (int jp = J - 1; jp >= 1; --jp) {
        const int Sp = N >> jp;
        if (P & (Sp - 1)) break;
        const int bp = P - Sp;
        // F^{(x)k} = [[F', 0], [F', F']]: the encoding of (u_left, u_right) is
        // (x_left ^ x_right, x_right), the halves' own encodings being their
        // stage-(jp+1) decisions.
        const uint32_t* xc = sm.Xf + (jp + 1) * NW;
        uint32_t* xo = sm.Xf + jp * NW;
        if (Sp >= 64) {
            const int hw = Sp >> 6;
            for (int w = lane; w < 2 * hw; w += 32) {
                const int ww = (bp >> 5) + w;
                xo[ww] = w < hw ? (xc[ww] ^ xc[ww + hw]) : xc[ww];
            }
        } else if (lane == 0) {
            const int h = Sp >> 1, off = bp & 31;
            const uint32_t x = xc[bp >> 5];
            const uint32_t v = x ^ ((x >> h) & (((1u << h) - 1u) << off));
            const uint32_t mk = low_mask(Sp) << off;
            xo[bp >> 5] = (xo[bp >> 5] & ~mk) | (v & mk);
        }
        note_event(sm, jp, bp, P, lane, multi);
        __syncwarp();
    }
}

// Speculative check of every stage's frontier CSFG under the covered prefix P0
// of the start of the iteration, all stages at once.  CSFGs of >= 32 positions
// are laid out word by word over the warp's lanes (stage j's words in an aligned
// group of 2^(M-5-j) slots), so one sequence of shifts and lane shuffles applies
// Eq. (3) to all of them; every smaller CSFG is handled whole by one lane.  The
// result stays valid for stage j unless a shallower stage froze earlier in the
// same iteration (the frontier then moved); resolve() re-checks those.
template <int M>
struct Spec {
    static constexpr int N = 1 << M;
    static constexpr int TW = N >= 64 ? N / 32 - 1 : 0;  // words of all CSFGs with >= 32 positions
    static constexpr int R = TW > 0 ? (TW + 31) / 32 : 1;
    static constexpr int JB = M - 5;                    // stages 1..JB have CSFGs of >= 32 positions
    static constexpr int JS0 = JB >= 1 ? JB + 1 : 1;    // first stage with smaller CSFGs
    static constexpr int NS = M - JS0 + 1;              // number of such stages (<= 5)
    uint32_t x[R], u[R];  // Eq. (2) decisions and Eq. (3) source words of this lane's slots
    int lvl[R], w[R];     // stage (0 = unused slot) and word-in-CSFG of each slot
    uint32_t xs, us;      // the small CSFG this lane holds (lane < NS)
    int fail;             // bit j: the speculative check of stage j fails Eq. (4)
};

// Lane-constant part of the speculative check: the stage and word of each of
// the lane's slots, and which of the cross-word butterfly steps apply to it.
template <int M>
struct SpecSlots {
    int lvl[Spec<M>::R];
    int w[Spec<M>::R];
    unsigned xm[Spec<M>::R];  // bit q: step d = 2^q xors in the partner word
};

template <int M>
__device__ __forceinline__ void spec_slots(SpecSlots<M>& ss, int lane)
{
    using SP = Spec<M>;
    constexpr int N = 1 << M;
#pragma unroll
    for (int r = 0; r < SP::R; ++r) {
        const int sl = 32 * r + lane;
        ss.lvl[r] = 0;
        ss.w[r] = 0;
        ss.xm[r] = 0u;
        if (sl < SP::TW) {
            const int lw = 31 - __clz(N / 32 - sl - 1);  // log2 of the stage's word count
            const int wi = sl - (N / 32 - (2 << lw));
            ss.lvl[r] = M - 5 - lw;
            ss.w[r] = wi;
            const int W = 1 << lw;
#pragma unroll
            for (int q = 0; (1 << q) < N / 64; ++q)
                if (W > (1 << q) && !(wi & (1 << q))) ss.xm[r] |= 1u << q;
        }
    }
}

template <int M, bool SMALL = true>
__device__ __forceinline__ void speculate(Smem<M>& sm, Spec<M>& sp, const SpecSlots<M>& ss, int P0, int jmin, int lane)
{
    using SP = Spec<M>;
    constexpr int N = 1 << M;
    unsigned bad_levels = 0;
    if constexpr (SP::TW > 0) if (jmin <= SP::JB) {
        int base[SP::R];
#pragma unroll
        for (int r = 0; r < SP::R; ++r) {
            sp.lvl[r] = ss.lvl[r];
            sp.w[r] = ss.w[r];
            sp.x[r] = 0u;
            base[r] = 0;
            if (ss.lvl[r]) {
                const int j = ss.lvl[r];
                base[r] = (P0 >> (M - j)) << (M - j);
                sp.x[r] = snap_word<M>(sm.hd, j, base[r] + 32 * ss.w[r]);
            }
            uint32_t v = sp.x[r];
#pragma unroll
            for (int h = 1; h < 32; h <<= 1) v ^= (v >> h) & xmask(h);
            sp.u[r] = v;
        }
#pragma unroll
        for (int q = 0; (1 << q) < N / 64; ++q) {
            const int d = 1 << q;
            if (d < 32) {
#pragma unroll
                for (int r = 0; r < SP::R; ++r) {
                    const uint32_t y = __shfl_xor_sync(kFull, sp.u[r], d);
                    if (ss.xm[r] & (1u << q)) sp.u[r] ^= y;
                }
            } else {
                const int dr = d / 32;
#pragma unroll
                for (int r = 0; r < SP::R; ++r) {
                    if ((r & dr) || r + dr >= SP::R) continue;
                    if (ss.xm[r] & (1u << q)) sp.u[r] ^= sp.u[r + dr];
                }
            }
        }
#pragma unroll
        for (int r = 0; r < SP::R; ++r) {
            unsigned flag = 0;
            if (ss.lvl[r] && (sp.u[r] & sm.Fz[(base[r] >> 5) + ss.w[r]])) flag = 1u << ss.lvl[r];
            bad_levels |= __reduce_or_sync(kFull, flag);
        }
    }
    if constexpr (SMALL) {
        unsigned flag = 0;
        sp.xs = sp.us = 0u;
        if (lane < SP::NS && SP::JS0 + lane >= jmin) {
            const int j = SP::JS0 + lane;
            const int S = N >> j;
            const int base = (P0 >> (M - j)) << (M - j);
            const uint32_t mk = low_mask(S);
            const uint32_t xv = (snap_word<M>(sm.hd, j, base & ~31) >> (base & 31)) & mk;
            uint32_t v = xv;
#pragma unroll
            for (int h = 1; h < 16; h <<= 1) v ^= (v >> h) & xmask(h);  // steps >= S act on zero bits
            sp.xs = xv;
            sp.us = v;
            if (v & (sm.Fz[base >> 5] >> (base & 31)) & mk) flag = 1u << j;
        }
        bad_levels |= __reduce_or_sync(kFull, flag);
    }
    sp.fail = (int)bad_levels;
}

// Stages 1..M in order (the checks depend on each other through P).  All
// stages at or below jmin are checked speculatively against the current
// frontier; the first stage that passes is committed (its CSFG frozen, P moved
// to the CSFG's end, enclosing CSFGs completed), which moves the frontier of
// every deeper stage, so those are checked again from there.  Stages before
// the first pass failed against the frontier they would have seen.  Returns
// the PE updates of the iteration (Sec. IV count; stage s runs the PEs outside
// covered CSFGs given P after the check of stage s).
// MULTI selects reading B (a variant): after a CSFG of stage J freezes, the next
// round checks stage J again from the new frontier, on the same R[J].
template <int M, bool MULTI>
__device__ __forceinline__ int resolve(Smem<M>& sm, int& P, int lane)
{
    constexpr bool multi = MULTI;
    using SP = Spec<M>;
    constexpr int N = Geo<M>::N, NW = Geo<M>::NW;
    int jmin = 1;
    int Ps = P;  // lane s (1 <= s < M): P seen by stage s, i.e. after the last commit at a stage <= s
    SpecSlots<M> ss;
    spec_slots<M>(ss, lane);
#pragma unroll 1
    while (P < N && jmin <= M) {
        Spec<M> sp;
        speculate<M>(sm, sp, ss, P, jmin, lane);
        const unsigned wanted = ((2u << M) - 1u) & ~((1u << jmin) - 1u);
        const unsigned pass = ~(unsigned)sp.fail & wanted;
        if (!pass) break;
        const int J = __ffs(pass) - 1;
        const int S = N >> J;
        const int cand = (P >> (M - J)) << (M - J);
        if (J <= SP::JB) {
#pragma unroll
            for (int r = 0; r < SP::R; ++r) {
                if (sp.lvl[r] == J) {
                    sm.U[(cand >> 5) + sp.w[r]] = sp.u[r];
                    sm.Xf[J * NW + (cand >> 5) + sp.w[r]] = sp.x[r];
                }
            }
        } else if (lane == J - SP::JS0) {
            const uint32_t mk = low_mask(S) << (cand & 31);
            uint32_t* pu = sm.U + (cand >> 5);
            uint32_t* px = sm.Xf + J * NW + (cand >> 5);
            *pu = (*pu & ~mk) | ((sp.us << (cand & 31)) & mk);
            *px = (*px & ~mk) | ((sp.xs << (cand & 31)) & mk);
            // a stage-M CSFG is one position; its feedback goes straight to column M
            if (J == M) sm.Lm[cand] = (sp.xs & 1u) ? -INFINITY : INFINITY;
        }
        if (J < M) note_event(sm, J, cand, cand + S, lane, multi);
        P = cand + S;
        __syncwarp();
        propagate<M>(sm, P, J, lane, multi);
        if (lane >= J) Ps = P;
        jmin = multi ? J : J + 1;  // reading B checks the next CSFG of the same stage, on the same R[J]
    }
    const int pe = (lane >= 1 && lane < M) ? (N - ((Ps >> (M - lane)) << (M - lane))) >> 1 : 0;
    return (int)__reduce_add_sync(kFull, (unsigned)pe) + (N >> 1);
}

// G-matrix stop for N >= 256.  F^{(x)M} is its own inverse over GF(2), so
// u_hat . F^{(x)M} == HD(R[0] + L[0]) holds exactly when u_hat equals the
// encoding of HD(R[0] + L[0]).  That encoding does not depend on the freezes
// of the iteration, so the sweep builds it (genc_step) from stage 0 on, spread
// over every warp, and the test after the freezes is a word-by-word comparison.
template <int M>
__host__ __device__ constexpr int genc_steps()
{
    return (M - 8 + 1) / 2;  // radix-4 steps over the word-index bits above the warp's 8 words
}

template <int M, int PH>
__device__ __forceinline__ void genc_step(Smem<M>& sm, int tid)
{
    static_assert(genc_steps<M>() <= Geo<M>::NP - 2, "one radix-4 step per phase boundary after the first");
    constexpr int NW = Geo<M>::NW;
    constexpr int LNW = M - 5;  // log2 NW
    if constexpr (PH == 1) {
        // each warp: 8 words, in-word butterflies, then across the 8 lanes
        const int lane = tid & 31, w = 8 * (tid >> 5) + (lane & 7);
        uint32_t v = snap_word<M>(sm.hd, 0, 32 * w);
#pragma unroll
        for (int h = 1; h < 32; h <<= 1) v ^= (v >> h) & xmask(h);
#pragma unroll
        for (int d = 1; d < 8; d <<= 1) {
            const uint32_t y = __shfl_xor_sync(kFull, v, d);
            if (!(lane & d)) v ^= y;
        }
        if (lane < 8) sm.Ge[w] = v;
    } else if constexpr (PH >= 2 && PH - 2 < genc_steps<M>()) {
        // word-index bits b and b + 1 (b = 3 + 2 (PH - 2)), ping-pong between the two buffers
        constexpr int b = 3 + 2 * (PH - 2);
        constexpr bool two = b + 1 < LNW;
        const uint32_t* src = sm.Ge + ((PH - 2) & 1) * NW;
        uint32_t* dst = sm.Ge + ((PH - 1) & 1) * NW;
        if (tid < NW) {
            const int w = tid;
            uint32_t v = src[w];
            const bool c1 = !(w & (1 << b));
            if (c1) v ^= src[w | (1 << b)];
            if constexpr (two) {
                const bool c2 = !(w & (1 << (b + 1)));
                if (c2) v ^= src[w | (2 << b)];
                if (c1 && c2) v ^= src[w | (3 << b)];
            }
            dst[w] = v;
        }
    }
}

template <int M>
__device__ __forceinline__ bool gmatrix_ok_pre(Smem<M>& sm, int P, int lane)
{
    constexpr int NW = Geo<M>::NW, RW = Geo<M>::RW;
    const uint32_t* enc = sm.Ge + (genc_steps<M>() & 1) * NW;
    bool same = true;
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int w = 32 * r + lane;
        if (w < NW) {
            uint32_t cov;
            if (P >= 32 * (w + 1)) cov = kFull;
            else if (P <= 32 * w) cov = 0u;
            else cov = (1u << (P - 32 * w)) - 1u;
            const uint32_t u = (sm.U[w] & cov) | (snap_word<M>(sm.hd, M, 32 * w) & ~sm.Fz[w] & ~cov);
            same &= u == enc[w];
        }
    }
    return __all_sync(kFull, same);
}

// G-matrix stop: u_hat . F^{(x)M} == HD(R[0] + L[0]).
template <int M>
__device__ __forceinline__ bool gmatrix_ok(Smem<M>& sm, int P, int lane)
{
    constexpr int N = Geo<M>::N, NW = Geo<M>::NW, RW = Geo<M>::RW, HDS = Geo<M>::HDS;
    uint32_t u[RW], x[RW];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int w = 32 * r + lane;
        const bool in = (N >= 32) ? (w < NW) : (lane == 0);
        u[r] = in ? snap_word<M>(sm.hd, M, 32 * w) & low_mask(N) : 0u;
        x[r] = in ? snap_word<M>(sm.hd, 0, 32 * w) & low_mask(N) : 0u;
        if (N < 32) {
            u[r] = __shfl_sync(kFull, u[r], 0);
            x[r] = __shfl_sync(kFull, x[r], 0);
        }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
        const int w = (N >= 32) ? 32 * r + lane : 0;
        uint32_t cov;
        if (P >= 32 * (w + 1)) cov = kFull;
        else if (P <= 32 * w) cov = 0u;
        else cov = (1u << (P - 32 * w)) - 1u;
        const uint32_t us = (w < NW) ? sm.U[w] : 0u;
        const uint32_t fz = (w < NW) ? sm.Fz[w] : 0u;
        u[r] = (us & cov) | (u[r] & ~fz & ~cov);
    }
    polar_xform<RW>(u, N, lane);
    bool same = true;
    const uint32_t valid = low_mask(N);
#pragma unroll
    for (int r = 0; r < RW; ++r) same &= ((u[r] ^ x[r]) & valid) == 0u;
    return __all_sync(kFull, same);
}

// Stages 1..M in order under reading A for codes of N >= 256 (natural-order
// snapshot rows); the same freezes, stored bits, feedback events and PE count as
// resolve<M, false>, with less serial work.
//  * Stages 1..M-6 (CSFGs of >= 64 positions) are checked speculatively at the
//    frontier as in resolve.  They rarely pass, so this is usually one round.
//  * Stages M-5..M (CSFGs of <= 32 positions).  With the frontier P at the end of
//    the large stages, every CSFG these stages can check lies in the two words
//    w0 = P / 32 and w0 + 1: the stage-(M-5) CSFG is word w0 itself, and the
//    freezes of the deeper stages add up to less than 32 positions.  Twelve lanes
//    evaluate Eqs. (2)-(4) for every aligned CSFG of their stage in one of those
//    words at once (the transform of Eq. (3) acts on each aligned block of a word
//    independently, and a fold of the failing bits gives one pass bit per CSFG),
//    then every lane runs the six-stage chain on the pass bits in registers.
//  * Only the first freeze of an iteration can complete enclosing CSFGs (it ends
//    at a multiple of its own size; each later freeze adds a smaller power of
//    two), so propagate() runs once.
template <int M>
__device__ __forceinline__ int resolve_fast(Smem<M>& sm, int& P, int lane)
{
    using SP = Spec<M>;
    constexpr int N = Geo<M>::N, NW = Geo<M>::NW;
    constexpr int JB = M - 6;  // stages with CSFGs of >= 64 positions
    constexpr int JS = M - 5;  // first stage with CSFGs of <= 32 positions
    static_assert(natural_rows<M>() && JB >= 2 && SP::JB == JB + 1, "codes of N >= 256");
    int Ps = P;  // lane s (1 <= s < M): P after the check of stage s
    bool first = true;
    int jmin = 1;
    {
        SpecSlots<M> ss;
        spec_slots<M>(ss, lane);
#pragma unroll 1
        while (jmin <= JB && P < N) {
            Spec<M> sp;
            speculate<M, false>(sm, sp, ss, P, jmin, lane);
            const unsigned wanted = ((2u << JB) - 1u) & ~((1u << jmin) - 1u);
            const unsigned pass = ~(unsigned)sp.fail & wanted;
            if (!pass) break;
            const int J = __ffs(pass) - 1;
            const int cand = (P >> (M - J)) << (M - J);
#pragma unroll
            for (int r = 0; r < SP::R; ++r) {
                if (sp.lvl[r] == J) {
                    sm.U[(cand >> 5) + sp.w[r]] = sp.u[r];
                    sm.Xf[J * NW + (cand >> 5) + sp.w[r]] = sp.x[r];
                }
            }
            note_event(sm, J, cand, cand + (N >> J), lane);
            P = cand + (N >> J);
            __syncwarp();
            propagate<M>(sm, P, J, lane);
            if (lane >= J) Ps = P;
            first = false;
            jmin = J + 1;
        }
    }
    if (P < N) {
        const int w0 = P >> 5;
        // lane l < 12: stage JS + l/2 on word w0 + (l & 1)
        const int jl = JS + (lane >> 1);
        const int wl = w0 + (lane & 1);
        const int Sl = N >> (jl < M ? jl : M);
        uint32_t x = 0u, u = 0u, pw = 0u;
        if (lane < 12 && wl < NW) {
            x = snap_word<M>(sm.hd, jl, 32 * wl);
            u = x;
#pragma unroll
            for (int h = 1; h < 32; h <<= 1)
                if (h < Sl) u ^= (u >> h) & xmask(h);
            uint32_t bad = u & sm.Fz[wl];
#pragma unroll
            for (int h = 1; h < 32; h <<= 1)
                if (h < Sl) bad |= bad >> h;
            // bits at the first position of every aligned block of Sl positions
            const uint32_t starts = Sl == 1 ? 0xffffffffu : Sl == 2 ? 0x55555555u : Sl == 4 ? 0x11111111u
                                  : Sl == 8 ? 0x01010101u : Sl == 16 ? 0x00010001u : 0x00000001u;
            pw = ~bad & starts;
        }
        uint32_t pa[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) pa[i] = __shfl_sync(kFull, pw, i);
        unsigned frz = 0u;  // bit jj: stage JS + jj froze
        int mybs = 0;       // start of the CSFG frozen at this lane's stage
#pragma unroll
        for (int jj = 0; jj < 6; ++jj) {
            const int S = N >> (JS + jj);
            if (P < N) {
                const int bs = P & ~(S - 1);
                const int off = bs - 32 * w0;  // 0 <= off < 64
                const uint32_t word = off < 32 ? pa[2 * jj] : pa[2 * jj + 1];
                if ((word >> (off & 31)) & 1u) {
                    frz |= 1u << jj;
                    if ((lane >> 1) == jj) mybs = bs;
                    P = bs + S;
                    if (lane >= JS + jj) Ps = P;
                }
            }
        }
        if (frz) {
            // stored bits and feedback decisions of the frozen CSFGs; several can share a
            // word of U, so U's two words are merged across lanes first
            uint32_t mk = 0u;
            if (lane < 12 && ((frz >> (lane >> 1)) & 1u) && (mybs >> 5) == wl)
                mk = low_mask(Sl) << (mybs & 31);
            const uint32_t ue = __reduce_or_sync(kFull, (lane & 1) ? 0u : mk);
            const uint32_t uo = __reduce_or_sync(kFull, (lane & 1) ? mk : 0u);
            const uint32_t ve = __reduce_or_sync(kFull, (lane & 1) ? 0u : (u & mk));
            const uint32_t vo = __reduce_or_sync(kFull, (lane & 1) ? (u & mk) : 0u);
            if (lane < 2 && w0 + lane < NW) {
                const uint32_t m2 = lane ? uo : ue, v2 = lane ? vo : ve;
                if (m2) sm.U[w0 + lane] = (sm.U[w0 + lane] & ~m2) | v2;
            }
            if (mk) {
                uint32_t* px = sm.Xf + jl * NW + wl;
                *px = (*px & ~mk) | (x & mk);
                if (jl == M) sm.Lm[mybs] = (x >> (mybs & 31)) & 1u ? -INFINITY : INFINITY;
                else {
                    sm.ev_lo()[jl] = mybs;
                    sm.ev_hi()[jl] = mybs + Sl;
                }
            }
            if (lane == 0) sm.ctl[CTL_EVENT] |= (int)((frz << JS) & ~(1u << M));
            __syncwarp();
            if (first) {
                const int jf = JS + __ffs(frz) - 1;
                const int Sf = N >> jf;
                const int bf = __shfl_sync(kFull, mybs, 2 * (jf - JS));
                propagate<M>(sm, bf + Sf, jf, lane);
            }
        }
    }
    const int pe = (lane >= 1 && lane < M) ? (N - ((Ps >> (M - lane)) << (M - lane))) >> 1 : 0;
    return (int)__reduce_add_sync(kFull, (unsigned)pe) + (N >> 1);
}

template <int M, bool GSTOP, bool FREEZE, bool MULTI>
__device__ __forceinline__ void checker(unsigned char* smem_base, int lane)
{
    constexpr int N = Geo<M>::N;
    Smem<M> sm(smem_base);
    if (lane <= M) {
        sm.ev_lo()[lane] = 0;
        sm.ev_hi()[lane] = 0;
    }
    if (lane == 0) sm.ctl[CTL_EVENT] = 0;
    __syncwarp();
    int P = sm.ctl[CTL_P];
    int pe_it = N >> 1;  // stage 0 always runs
    if constexpr (FREEZE) {
        if constexpr (natural_rows<M>() && !MULTI) pe_it = resolve_fast<M>(sm, P, lane);
        else pe_it = resolve<M, MULTI>(sm, P, lane);
    } else {
        pe_it = M * (N >> 1);
    }
    bool done = FREEZE && (P >= N);
    if constexpr (GSTOP) {
        if constexpr (natural_rows<M>()) {
            if (!done) done = gmatrix_ok_pre<M>(sm, P, lane);
        } else {
            if (!done) done = gmatrix_ok<M>(sm, P, lane);
        }
    }
    __syncwarp();
    if (lane == 0) {
        sm.ctl[CTL_P] = P;
        sm.ctl[CTL_DONE] = done ? 1 : 0;
        *sm.pe_acc() += pe_it;
    }
}

// ---------------------------------------------------------------------------
// the sweep
// ---------------------------------------------------------------------------
template <int M>
struct Regs {
    float R[Geo<M>::EL];
    float Lr[Geo<M>::NRA][Geo<M>::EL];
};

// L of column C at element e of the running phase PH.  Boundary column C is
// the buffer of boundary C/3 - 1 (between phases C/3 - 1 and C/3).
template <int M, int PH, int C>
__device__ __forceinline__ float load_L(Regs<M>& rg, Smem<M>& sm, int e, int pb)
{
    using G = Geo<M>;
    if constexpr (G::is_boundary(C)) {
        constexpr int SH = G::padsh(G::bslot(C));
        return sm.Lb[G::bslot(C) * G::BUF + pb + padded_off<M, PH, SH>(e)];
    } else {
        static_assert(C < M, "column M is read from shared memory by run_stage");
        return rg.Lr[G::rslot(C)][e];
    }
}

// Store L of column C; with keep set (the PE lies in a covered CSFG) the old
// value, possibly a +-inf freeze feedback, stays.  Covered PEs are still
// evaluated: their R outputs are never read again, and evaluating them keeps
// the sweep free of branches.  Column 0 is not stored unless the sweep is the
// lower part of a larger code (XC > 0 upper stages run elsewhere): then it is
// the column those stages read, kept in natural order in sm.L0 (phase 0 maps
// element e of thread t to position e * T + t, passed here as pb = t).
template <int M, int PH, int C, int XC = 0>
__device__ __forceinline__ void store_L(Regs<M>& rg, Smem<M>& sm, int e, int pb, float v, bool keep)
{
    using G = Geo<M>;
    if constexpr (C == 0) {
        if constexpr (XC > 0) {
            static_assert(PH == 0 && G::NP > 1, "column 0 is written in phase 0");
            if (!keep) sm.L0[e * G::T + pb] = v;
        } else {
            (void)rg; (void)sm; (void)e; (void)pb; (void)v; (void)keep;
        }
    } else if constexpr (G::is_boundary(C)) {
        constexpr int SH = G::padsh(G::bslot(C));
        if (!keep) sm.Lb[G::bslot(C) * G::BUF + pb + padded_off<M, PH, SH>(e)] = v;
    } else {
        rg.Lr[G::rslot(C)][e] = keep ? rg.Lr[G::rslot(C)][e] : v;
    }
}

// Snapshot rows: the hard decisions of one column, written by the phase PH that
// computes it.  For N >= 256 the phases with register bits from bit lo >= 1
// write raw ballots (raw_word reads them): one ballot of the warp's decisions
// per element, the warp's 8 words stored by its lane 0 as two 16-byte stores.
// The last phase (lo = 0) and smaller codes write one byte per thread (bit e =
// element e), which for lo = 0 is natural order.
template <int M, int PH>
__host__ __device__ constexpr bool raw_row()
{
    return natural_rows<M>() && Geo<M>::lo(PH) >= 1;
}

template <int M, int PH>
__device__ __forceinline__ void snap_row_raw(uint8_t* row, const uint32_t (&b)[8], int tid)
{
    static_assert(raw_row<M, PH>(), "raw ballot rows only");
    if ((tid & 31) == 0) {
        uint4* d = reinterpret_cast<uint4*>(row + 32 * (tid >> 5));
        d[0] = make_uint4(b[0], b[1], b[2], b[3]);
        d[1] = make_uint4(b[4], b[5], b[6], b[7]);
    }
}

template <int M, int PH>
__device__ __forceinline__ void snap_row(uint8_t* row, uint32_t byte, int tid)
{
    static_assert(!raw_row<M, PH>(), "byte rows only");
    row[tid] = (uint8_t)byte;
}

// Stage s of phase PH.  With XC > 0 the sweep is the lower M stages of a code
// of M + XC stages (stage s here is stage s + XC there): P0 is then the covered
// prefix within this part, stage 0 may be covered, its L column is stored, the
// channel-side decisions are taken elsewhere and trace columns are N << XC apart.
// KEEP (default: FREEZE) protects the L outputs of covered PEs with keep-selects;
// the pipelined decoder (bp_pipe.cuh) keeps covered CSFGs at a fixed point of
// Eq. (1) instead and runs every PE unguarded.
template <int M, int PH, int Q, bool GSTOP, bool FREEZE, bool TRACE, int XC = 0, bool KEEP = FREEZE>
__device__ __forceinline__ void run_stage(Regs<M>& rg, Smem<M>& sm, int tid, int P0, float alpha, const CwIO& a,
                                          long long trace_base)
{
    using G = Geo<M>;
    constexpr int N = G::N, EL = G::EL;
    constexpr int s = G::s0(PH) + Q;
    constexpr int b = M - 1 - s;
    constexpr int k = b - G::lo(PH);
    constexpr bool snap = FREEZE || (GSTOP && s == M - 1);
    constexpr long long TSTRIDE = (long long)N << XC;
    const int thr = (s + XC == 0 || !KEEP) ? 0 : ((P0 >> (M - s)) << (M - s));
    uint32_t xbyte = 0;  // stage 0: decisions on R[0] + L[0] (G-matrix stop)
    uint32_t xb[8];      // the same as ballots, for rows built from ballots
    // padded bases for the boundary columns read (s+1) and written (s) here
    const int pb_in = G::is_boundary(s + 1) ? padded_base<M, PH, G::padsh(G::bslot(s + 1))>(tid) : 0;
    // column M: this thread's entries, which the last phase (register bits from bit 0) holds
    // at consecutive positions
    float lm[EL];
    if constexpr (s + 1 == M) {
        static_assert(G::lo(PH) == 0, "stage M-1 runs in the last phase");
        const int i0 = elem_index<M, PH>(tid, 0);
        if constexpr (EL == 8) {
            const float4 q0 = reinterpret_cast<const float4*>(sm.Lm + i0)[0];
            const float4 q1 = reinterpret_cast<const float4*>(sm.Lm + i0)[1];
            lm[0] = q0.x; lm[1] = q0.y; lm[2] = q0.z; lm[3] = q0.w;
            lm[4] = q1.x; lm[5] = q1.y; lm[6] = q1.z; lm[7] = q1.w;
        } else {
#pragma unroll
            for (int e = 0; e < EL; ++e) lm[e] = sm.Lm[i0 + e];
        }
    }
    const int pb_out = G::is_boundary(s) ? padded_base<M, PH, G::padsh(G::bslot(s))>(tid) : (s == 0 ? tid : 0);
#pragma unroll
    for (int e = 0; e < EL; ++e) {
        if (e & (1 << k)) continue;
        const int e2 = e | (1 << k);
        const int ia = elem_index<M, PH>(tid, e);
        const int ib = ia + (1 << b);
        const bool covered = KEEP && s + XC > 0 && ia < thr;  // PE inside a covered CSFG
        float La, Lb;
        if constexpr (s + 1 == M) {
            La = lm[e];
            Lb = lm[e2];
        } else {
            La = load_L<M, PH, s + 1>(rg, sm, e, pb_in);
            Lb = load_L<M, PH, s + 1>(rg, sm, e2, pb_in);
        }
        const float Ra = rg.R[e];
        const float Rb = rg.R[e2];
        const float t = __fadd_rn(Lb, Rb);
        const float g = fms(La, Ra, alpha);
        const float nLa = fms(La, t, alpha);
        const float nLb = __fadd_rn(Lb, g);
        const float nRa = fms(Ra, t, alpha);
        const float nRb = __fadd_rn(Rb, g);
        store_L<M, PH, s, XC>(rg, sm, e, pb_out, nLa, covered);
        store_L<M, PH, s, XC>(rg, sm, e2, pb_out, nLb, covered);
        if constexpr (s == 0 && GSTOP && XC == 0) {
            if constexpr (raw_row<M, PH>()) {
                xb[e] = __ballot_sync(kFull, __fadd_rn(Ra, nLa) < 0.f);
                xb[e2] = __ballot_sync(kFull, __fadd_rn(Rb, nLb) < 0.f);
            } else {
                xbyte |= (__fadd_rn(Ra, nLa) < 0.f ? 1u : 0u) << e;
                xbyte |= (__fadd_rn(Rb, nLb) < 0.f ? 1u : 0u) << e2;
            }
        }
        if constexpr (s == 0 && TRACE && XC == 0) {
            a.trace_L[trace_base + ia] = nLa;
            a.trace_L[trace_base + ib] = nLb;
        }
        rg.R[e] = nRa;
        rg.R[e2] = nRb;
    }
    if constexpr (s == 0 && GSTOP && XC == 0) {
        if constexpr (raw_row<M, PH>()) snap_row_raw<M, PH>(sm.hd, xb, tid);
        else snap_row<M, PH>(sm.hd, xbyte, tid);
    }
    if constexpr (snap) {
        if constexpr (raw_row<M, PH>()) {
            uint32_t b[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) b[e] = __ballot_sync(kFull, rg.R[e] < 0.f);
            snap_row_raw<M, PH>(sm.hd + (s + 1) * G::HDS, b, tid);
        } else {
            uint32_t byte = 0;
#pragma unroll
            for (int e = 0; e < EL; ++e) byte |= (rg.R[e] < 0.f ? 1u : 0u) << e;
            snap_row<M, PH>(sm.hd + (s + 1) * G::HDS, byte, tid);
        }
    }
    if constexpr (TRACE) {
#pragma unroll
        for (int e = 0; e < EL; ++e)
            a.trace_R[trace_base + (long long)(s + 1) * TSTRIDE + elem_index<M, PH>(tid, e)] = rg.R[e];
    }
    if constexpr (Q + 1 < G::cnt(PH))
        run_stage<M, PH, Q + 1, GSTOP, FREEZE, TRACE, XC, KEEP>(rg, sm, tid, P0, alpha, a, trace_base);
}

template <int M, int PH, bool GSTOP, bool FREEZE, bool TRACE, int CPC, int XC = 0>
__device__ __forceinline__ void run_phase(Regs<M>& rg, Smem<M>& sm, int tid, bool worker, int P0, float alpha,
                                          const CwIO& a, long long trace_base, int grp)
{
    using G = Geo<M>;
    constexpr int N = G::N, EL = G::EL;
    if constexpr (PH > 0) {
        if (worker) {
            constexpr int SH = G::padsh(PH - 1);
            const int pb = padded_base<M, PH, SH>(tid);
#pragma unroll
            for (int e = 0; e < EL; ++e) rg.R[e] = sm.Rx[((PH - 1) & 1) * G::BUF + pb + padded_off<M, PH, SH>(e)];
        }
        if constexpr (GSTOP && XC == 0 && natural_rows<M>()) genc_step<M, PH>(sm, tid);
    }
    if (worker) run_stage<M, PH, 0, GSTOP, FREEZE, TRACE, XC>(rg, sm, tid, P0, alpha, a, trace_base);
    if constexpr (PH + 1 < G::NP) {
        if (worker) {
            constexpr int SH = G::padsh(PH);
            const int pb = padded_base<M, PH, SH>(tid);
#pragma unroll
            for (int e = 0; e < EL; ++e) sm.Rx[(PH & 1) * G::BUF + pb + padded_off<M, PH, SH>(e)] = rg.R[e];
        }
        group_sync<G::BLOCK, CPC>(grp);
        run_phase<M, PH + 1, GSTOP, FREEZE, TRACE, CPC, XC>(rg, sm, tid, worker, P0, alpha, a, trace_base, grp);
    }
}

// Fix L of the columns that received a freeze event to (-1)^x_hat * inf.  Every
// thread rewrites only entries it reads itself in the next iteration: register
// columns in their owner phase's mapping, shared-memory columns in the mapping of
// the phase that reads them (stage C-1).  No barrier is needed.
template <int M, int C>
__device__ __forceinline__ void apply_column(Regs<M>& rg, Smem<M>& sm, int tid)
{
    using G = Geo<M>;
    {
        {
            const int lo = sm.ev_lo()[C], hi = sm.ev_hi()[C];
            const uint32_t* xf = sm.Xf + C * G::NW;
            constexpr int PH = G::is_boundary(C) ? (C - 1) / 3 : G::owner(C);
            constexpr int SH = G::is_boundary(C) ? G::padsh(G::bslot(C)) : 5;
            // element e of this thread sits at i0 + (e << LO); elements [e1, e2) lie in [lo, hi)
            constexpr int LO = G::lo(PH);
            const int i0 = elem_index<M, PH>(tid, 0);
            const int e1 = min(G::EL, max(0, (lo - i0 + (1 << LO) - 1) >> LO));
            const int e2 = min(G::EL, max(0, (hi - i0 + (1 << LO) - 1) >> LO));
            if (e1 < e2) {
                // the thread's decisions, bit e for element e: its positions lie in one aligned
                // segment of 8 << LO positions, i.e. in one word for LO <= 2
                uint32_t bits = 0;
                if constexpr (LO >= 5) {
#pragma unroll
                    for (int e = 0; e < G::EL; ++e)
                        bits |= ((xf[(i0 >> 5) + (e << (LO - 5))] >> (i0 & 31)) & 1u) << e;
                } else if constexpr (LO <= 2) {
                    const uint32_t w = xf[i0 >> 5] >> (i0 & 31);
#pragma unroll
                    for (int e = 0; e < G::EL; ++e) bits |= ((w >> (e << LO)) & 1u) << e;
                } else {
#pragma unroll
                    for (int q = 0; q < (G::EL << LO) / 32; ++q) {
                        const uint32_t w = xf[(i0 >> 5) + q] >> (i0 & 31);
#pragma unroll
                        for (int e = 0; e < G::EL; ++e)
                            if (((e << LO) >> 5) == q) bits |= ((w >> ((e << LO) & 31)) & 1u) << e;
                    }
                }
                // elements [e1, e2) take (-1)^bit inf
                const uint32_t m8 = (0xffu >> (8 - e2)) & ~((1u << e1) - 1u);
                const int pb = padded_base<M, PH, SH>(tid);
#pragma unroll
                for (int e = 0; e < G::EL; ++e) {
                    const float v = __uint_as_float(0x7f800000u | ((bits << (31 - e)) & 0x80000000u));
                    const bool in = (m8 >> e) & 1u;
                    if constexpr (C == M) {
                        if (in) sm.Lm[i0 + (e << LO)] = v;
                    } else if constexpr (G::is_boundary(C)) {
                        if (in) sm.Lb[G::bslot(C) * G::BUF + pb + padded_off<M, PH, SH>(e)] = v;
                    } else {
                        rg.Lr[G::rslot(C)][e] = in ? v : rg.Lr[G::rslot(C)][e];
                    }
                }
            }
        }
    }
}

template <int M, int C>
__device__ __forceinline__ void apply_events(Regs<M>& rg, Smem<M>& sm, int tid, int mask)
{
    if constexpr (C <= M) {
        if (mask & (1 << C)) apply_column<M, C>(rg, sm, tid);
        apply_events<M, C + 1>(rg, sm, tid, mask);
    }
}

template <int M, int C, int XC = 0>
__device__ __forceinline__ void trace_L_columns(Regs<M>& rg, Smem<M>& sm, int tid, bool worker, const CwIO& a,
                                                long long trace_base)
{
    using G = Geo<M>;
    constexpr long long TSTRIDE = (long long)G::N << XC;
    if constexpr (C <= M) {
        if constexpr (C == M) {
            for (int i = tid; i < G::N; i += G::BLOCK) a.trace_L[trace_base + C * TSTRIDE + i] = sm.Lm[i];
        } else if constexpr (G::is_boundary(C)) {
            constexpr int SH = G::padsh(G::bslot(C));
            for (int i = tid; i < G::N; i += G::BLOCK)
                a.trace_L[trace_base + C * TSTRIDE + i] = sm.Lb[G::bslot(C) * G::BUF + padded<SH>(i)];
        } else if (worker) {
#pragma unroll
            for (int e = 0; e < G::EL; ++e)
                a.trace_L[trace_base + C * TSTRIDE + elem_index<M, G::owner(C)>(tid, e)] = rg.Lr[G::rslot(C)][e];
        }
        trace_L_columns<M, C + 1, XC>(rg, sm, tid, worker, a, trace_base);
    }
}

// Stage the channel LLRs of one codeword into shared memory in phase 0's
// element-major layout (element e of worker t at e * T + t).  With N >= 8 and a
// 16-byte aligned row in natural order the row is read with 16-byte loads,
// thread i taking positions 4i .. 4i+3, and scattered; otherwise element by
// element (gathered through the bit reversal when the code has it).  Returns
// false if a loaded value is not finite.  The caller synchronises before the
// values are read.
template <int M>
__device__ __forceinline__ bool stage_llr(float* dst, const float* llr, int tid, int nthreads, int bitrev)
{
    using G = Geo<M>;
    constexpr int N = G::N, T = G::T, lo0 = G::lo(0);
    bool finite = true;
    if constexpr (N >= 8) {
        if (!bitrev && (reinterpret_cast<uintptr_t>(llr) & 15u) == 0) {
            for (int i = tid; i < N / 4; i += nthreads) {
                const float4 v = reinterpret_cast<const float4*>(llr)[i];
                finite &= isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int p = 4 * i + k;
                    const int t = (p & ((1 << lo0) - 1)) | ((p >> (lo0 + G::RB)) << lo0);
                    dst[((p >> lo0) & (G::EL - 1)) * T + t] = vv[k];
                }
            }
            return finite;
        }
    }
    for (int p = tid; p < N; p += nthreads) {
        // bit-reversed order: code position p was received at channel position rev(p)
        const float v = llr[bitrev ? (int)(__brev((unsigned)p) >> (32 - M)) : p];
        finite &= isfinite(v);
        const int t = (p & ((1 << lo0) - 1)) | ((p >> (lo0 + G::RB)) << lo0);
        dst[((p >> lo0) & (G::EL - 1)) * T + t] = v;
    }
    return finite;
}

// Decode one codeword with the BLOCK threads of group grp (tid = thread index in
// the group) on the group's shared memory smem_raw.
template <int M, bool GSTOP, bool FREEZE, bool TRACE, int CPC, bool MULTI = false>
__device__ __forceinline__ void decode_codeword(const CwIO& a, int max_iter, float alpha, unsigned int* status,
                                                unsigned char* smem_raw, int tid, int grp)
{
    using G = Geo<M>;
    constexpr int N = G::N, EL = G::EL, T = G::T, NW = G::NW;
    Smem<M> sm(smem_raw);
    const int lane = tid & 31;
    const bool worker = tid < T;

    redzones<M, true>(smem_raw, status, tid, G::BLOCK);
    for (int w = tid; w < NW; w += G::BLOCK) {
        sm.Fz[w] = a.frozen_words[w];
        sm.U[w] = 0u;
    }
    for (int i = tid; i < G::NB * G::BUF; i += G::BLOCK) sm.Lb[i] = 0.f;
    // source-side prior (reading: +inf on frozen positions, 0 elsewhere)
    for (int i = tid; i < N; i += G::BLOCK) sm.Lm[i] = ((a.frozen_words[i >> 5] >> (i & 31)) & 1u) ? INFINITY : 0.f;
    {
        uint32_t* hd32 = reinterpret_cast<uint32_t*>(sm.hd);
        for (int i = tid; i < (int)(SmemLayout<M>::hd_bytes / 4); i += G::BLOCK) hd32[i] = 0u;
    }
    if (tid == 0) {
        sm.ctl[CTL_P] = 0;
        sm.ctl[CTL_DONE] = 0;
        sm.ctl[CTL_EVENT] = 0;
        *sm.pe_acc() = 0;
    }
    if (!stage_llr<M>(sm.llr, a.llr, tid, G::BLOCK, a.bitrev)) atomicOr(status, 1u);
    group_sync<G::BLOCK, CPC>(grp);

    Regs<M> rg;
    if (worker) {
#pragma unroll
        for (int c = 0; c < G::NRA; ++c)
#pragma unroll
            for (int e = 0; e < EL; ++e) rg.Lr[c][e] = 0.f;
    }

    int it = 1;
    for (; it <= max_iter; ++it) {
        const int P0 = sm.ctl[CTL_P];
        const long long trace_base = TRACE ? (long long)(it - 1) * (M + 1) * N : 0;
        if (worker) {
#pragma unroll
            for (int e = 0; e < EL; ++e) rg.R[e] = sm.llr[e * T + tid];
            if constexpr (TRACE) {
#pragma unroll
                for (int e = 0; e < EL; ++e) a.trace_R[trace_base + elem_index<M, 0>(tid, e)] = rg.R[e];
            }
        }
        run_phase<M, 0, GSTOP, FREEZE, TRACE, CPC>(rg, sm, tid, worker, P0, alpha, a, trace_base, grp);
        group_sync<G::BLOCK, CPC>(grp);
        bool done = false;
        if constexpr (GSTOP || FREEZE) {
            if (tid < 32) checker<M, GSTOP, FREEZE, MULTI>(smem_raw, lane);
            group_sync<G::BLOCK, CPC>(grp);
            done = sm.ctl[CTL_DONE] != 0;
            if constexpr (FREEZE) {
                const int mask = sm.ctl[CTL_EVENT];
                if (mask && worker) apply_events<M, 1>(rg, sm, tid, mask);
            }
        }
        if constexpr (TRACE) {
            group_sync<G::BLOCK, CPC>(grp);
            trace_L_columns<M, 1>(rg, sm, tid, worker, a, trace_base);
            if (tid == 0) a.trace_P[it - 1] = sm.ctl[CTL_P];
        }
        if (done) break;
    }
    const int iters = it <= max_iter ? it : max_iter;

    // output: stored bits on covered positions, HD(R[M]) elsewhere, 0 on frozen
    if (worker) {
        const int P = sm.ctl[CTL_P];
        // HD(R[M]) of the last sweep: the snapshot byte when one is kept, else R itself
        uint32_t hdM = 0;
        if constexpr (GSTOP || FREEZE) {
            hdM = sm.hd[M * G::HDS + tid];
        } else {
#pragma unroll
            for (int e = 0; e < EL; ++e) hdM |= (rg.R[e] < 0.f ? 1u : 0u) << e;
        }
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const int i = elem_index<M, G::NP - 1>(tid, e);
            uint8_t bit;
            if (i < P) bit = (uint8_t)bit_of(sm.U, i);
            else bit = bit_of(sm.Fz, i) ? 0 : (uint8_t)((hdM >> e) & 1u);
            a.u_hat[i] = bit;
        }
    }
    if (tid == 0) {
        if (a.iters) *a.iters = iters;
        if (a.pe) *a.pe = (GSTOP || FREEZE) ? *sm.pe_acc() : (long long)iters * M * (N >> 1);
    }
    if constexpr (kChecked) {
        group_sync<G::BLOCK, CPC>(grp);  // every store of this decode is done
        redzones<M, false>(smem_raw, status, tid, G::BLOCK);
    }
}

// One codeword per block, grid = batch.  MULTI: freezing under reading B.
template <int M, bool GSTOP, bool FREEZE, bool TRACE, bool MULTI = false>
__global__ void __launch_bounds__(Geo<M>::BLOCK, Geo<M>::min_blocks(FREEZE)) bp_decode_kernel(DecodeArgs a)
{
    constexpr int N = Geo<M>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long cw = blockIdx.x;
    const long long tb = TRACE ? cw * a.max_iter * (long long)(M + 1) * N : 0;
    const CwIO io{a.llr + cw * N,
                  a.frozen_words,
                  a.u_hat + cw * N,
                  a.iters ? a.iters + cw : nullptr,
                  a.pe ? a.pe + cw : nullptr,
                  TRACE ? a.trace_L + tb : nullptr,
                  TRACE ? a.trace_R + tb : nullptr,
                  TRACE ? a.trace_P + cw * a.max_iter : nullptr,
                  a.bitrev};
    decode_codeword<M, GSTOP, FREEZE, TRACE, 1, MULTI>(io, a.max_iter, a.alpha, a.status, smem_raw, threadIdx.x, 0);
}

// Persistent decoding of a queue of codewords split in segments (one code per
// segment, all of length N = 2^M): CPC groups of threads per block, each group
// takes the next codeword from a device counter, decodes it and retires it at
// its own stop, then takes the next, until the queue is empty.
constexpr int kMaxSeg = 8;
struct SegArgs {
    int nseg;
    int total;
    int* queue;  // device counter, zero at launch
    int max_iter;
    float alpha;
    int start[kMaxSeg + 1];  // first queue index of each segment; start[nseg] = total
    unsigned int* status[kMaxSeg];  // the status word of each segment's code
    const float* llr[kMaxSeg];
    const uint32_t* frozen_words[kMaxSeg];
    uint8_t* u_hat[kMaxSeg];
    int32_t* iters[kMaxSeg];
    int64_t* pe[kMaxSeg];
    int bitrev[kMaxSeg];  // per segment: its code's positions arrive in bit-reversed order
};

template <int M, int CPC>
struct PersistentShape {
    static constexpr int THREADS = Geo<M>::BLOCK * CPC;
    static constexpr int MIN_BLOCKS = (640 / THREADS) < 1 ? 1 : (640 / THREADS);
    // one codeword per block: the bound of bp_decode_kernel
    static constexpr int min_blocks(bool freeze) { return CPC == 1 ? Geo<M>::min_blocks(freeze) : MIN_BLOCKS; }
};

template <int M, bool GSTOP, bool FREEZE, int CPC>
__global__ void __launch_bounds__(PersistentShape<M, CPC>::THREADS, PersistentShape<M, CPC>::min_blocks(FREEZE))
    bp_decode_persistent(SegArgs a)
{
    using G = Geo<M>;
    constexpr int N = G::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int grp = threadIdx.x / G::BLOCK;
    const int tid = threadIdx.x % G::BLOCK;
    unsigned char* smem = smem_raw + grp * SmemLayout<M>::bytes;
    int* qslot = reinterpret_cast<int*>(smem + SmemLayout<M>::off_Ctl) + CTL_Q;
    for (;;) {
        group_sync<G::BLOCK, CPC>(grp);  // the previous codeword's readers are done with smem
        if (tid == 0) *qslot = atomicAdd(a.queue, 1);
        group_sync<G::BLOCK, CPC>(grp);
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
        decode_codeword<M, GSTOP, FREEZE, false, CPC>(io, a.max_iter, a.alpha, a.status[sg], smem, tid, grp);
    }
}


struct LaunchReq {
    DecodeArgs args;
    int stop_mode;
    int freeze_mode;
    bool trace;
    bool pipelined = true;  // freezing at N = 256 .. 4096: the checker-warp mapping (bp_pipe.cuh)
    cudaStream_t stream;
};

template <int M, bool GSTOP, bool FREEZE, bool TRACE, bool MULTI = false>
cudaError_t launch_one(const LaunchReq& q)
{
    auto kern = bp_decode_kernel<M, GSTOP, FREEZE, TRACE, MULTI>;
    constexpr size_t smem = SmemLayout<M>::bytes;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<q.args.batch, Geo<M>::BLOCK, smem, q.stream>>>(q.args);
    return cudaGetLastError();
}

template <int M>
cudaError_t launch_decode(const LaunchReq& q)
{
    const bool g = q.stop_mode != 0, f = q.freeze_mode != 0;
    if (q.freeze_mode == 2) {  // reading B
        if (q.trace) return g ? launch_one<M, true, true, true, true>(q) : launch_one<M, false, true, true, true>(q);
        return g ? launch_one<M, true, true, false, true>(q) : launch_one<M, false, true, false, true>(q);
    }
    if (q.trace) {
        if (g && f) return launch_one<M, true, true, true>(q);
        if (g) return launch_one<M, true, false, true>(q);
        if (f) return launch_one<M, false, true, true>(q);
        return launch_one<M, false, false, true>(q);
    }
    if (g && f) return launch_one<M, true, true, false>(q);
    if (g) return launch_one<M, true, false, false>(q);
    if (f) return launch_one<M, false, true, false>(q);
    return launch_one<M, false, false, false>(q);
}


// ---------------------------------------------------------------------------
// persistent launches
// ---------------------------------------------------------------------------
struct SegLaunch {
    SegArgs args;
    int stop_mode;
    int freeze_mode;
    int cpc;
    bool pipelined = true;  // freezing at N = 256 .. 4096 with cpc 1: the checker-warp mapping (bp_pipe.cuh)
    int sms;
    cudaStream_t stream;
};

template <int M, int CPC>
constexpr bool persistent_fits()
{
    return PersistentShape<M, CPC>::THREADS <= 512 && SmemLayout<M>::bytes * CPC <= 200 * 1024;
}

template <int M, bool GSTOP, bool FREEZE, int CPC>
cudaError_t launch_persistent_one(const SegLaunch& q)
{
    auto kern = bp_decode_persistent<M, GSTOP, FREEZE, CPC>;
    constexpr size_t smem = SmemLayout<M>::bytes * CPC;
    constexpr int threads = PersistentShape<M, CPC>::THREADS;
    // Blocks per SM, one value per device and instantiation, set with the kernel's
    // shared-memory attribute on the device's first launch.  Host threads that race
    // on the first launch compute and store the same value.
    constexpr int kDevices = 64;
    static std::atomic<int> blocks_per_sm[kDevices];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kDevices) return cudaErrorInvalidDevice;
    int bps = blocks_per_sm[dev].load(std::memory_order_acquire);
    if (bps == 0) {
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, threads, smem);
        if (e != cudaSuccess) return e;
        bps = b > 0 ? b : 1;
        blocks_per_sm[dev].store(bps, std::memory_order_release);
    }
    long long grid = (long long)bps * q.sms;
    const long long need = (q.args.total + CPC - 1) / CPC;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, threads, smem, q.stream>>>(q.args);
    return cudaGetLastError();
}

template <int M, int CPC>
cudaError_t launch_persistent_cpc(const SegLaunch& q)
{
    if constexpr (!persistent_fits<M, CPC>()) {
        (void)q;
        return cudaErrorInvalidConfiguration;
    } else {
        const bool g = q.stop_mode != 0, f = q.freeze_mode != 0;
        if (g && f) return launch_persistent_one<M, true, true, CPC>(q);
        if (g) return launch_persistent_one<M, true, false, CPC>(q);
        if (f) return launch_persistent_one<M, false, true, CPC>(q);
        return launch_persistent_one<M, false, false, CPC>(q);
    }
}

template <int M>
bool persistent_supported_m(int cpc)
{
    return cpc == 1 ? persistent_fits<M, 1>() : cpc == 2 ? persistent_fits<M, 2>() : cpc == 4 ? persistent_fits<M, 4>() : false;
}

inline bool persistent_supported(int m, int cpc)
{
    switch (m) {
    case 8: return persistent_supported_m<8>(cpc);
    case 9: return persistent_supported_m<9>(cpc);
    case 10: return persistent_supported_m<10>(cpc);
    case 11: return persistent_supported_m<11>(cpc);
    case 12: return persistent_supported_m<12>(cpc);
    default: return false;
    }
}

template <int M>
cudaError_t launch_persistent(const SegLaunch& q)
{
    switch (q.cpc) {
    case 1: return launch_persistent_cpc<M, 1>(q);
    case 2: return launch_persistent_cpc<M, 2>(q);
    case 4: return launch_persistent_cpc<M, 4>(q);
    default: return cudaErrorInvalidConfiguration;
    }
}

}  // namespace polarbp
