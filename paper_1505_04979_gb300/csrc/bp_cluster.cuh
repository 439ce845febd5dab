// bp_cluster.cuh -- min-sum BP decoding of long polar codes (N = 2^(12+XC),
// 8192 <= N <= 32768) by a thread-block cluster of C = 2^XC blocks, with the
// G-matrix stop and CSFG freezing.
//
// Method: arXiv 1505.04979.  Eq. (1) (Sec. II-A) is the PE update; Sec. III and
// Eqs. (2)-(4) define the CSFG check, the freezing order and the +-inf feedback;
// Sec. IV defines the PE-update count.
//
// Partition.  Block r of the cluster owns positions [r n, (r+1) n), n = 4096, of
// every node column.  PE stage s pairs a with a + 2^(M-1-s): stages 0..XC-1 pair
// positions of two blocks (rank bit XC-1-s), stages XC..M-1 stay inside a block.
//   * Cross stages.  Each block computes the Eq. (1) outputs of its own
//     positions: the a side L[s][a] = f(L[s+1][a], L[s+1][b] + R[s][b]) and
//     R[s+1][a] = f(R[s][a], L[s+1][b] + R[s][b]); the b side L[s][b] =
//     L[s+1][b] + f(L[s+1][a], R[s][a]) and R[s+1][b] = R[s][b] + f(...).  The
//     partner's L[s+1] and R[s] are read from its shared memory (distributed
//     shared memory, plain loads); one cluster barrier follows each cross stage.
//     Both sides evaluate the shared terms with the same operands, so the
//     messages are those of a single sweep.
//   * Lower stages.  The sweep of bp_decode.cuh for a 4096-point code, run on
//     the block's part: its column 0 is column XC here, stored in shared memory
//     because the partner reads it in cross stage XC-1.
//   * Columns 1..XC of L live in shared memory in natural order (the cross
//     stages and phase 0 of the lower sweep both map element e of thread t to
//     position e * 512 + t).
// Checks (after the sweep, as in bp_decode.cuh).  The covered positions are a
// prefix [0, P) of the code.  Every block evaluates Eqs. (2)-(4) for all CSFGs
// of the stages inside its part (one warp per stage) and publishes a bit per
// CSFG; for the stages whose CSFGs span blocks it publishes the Eq. (3)
// transform of its part, and the partners combine the transforms (the
// transform of a vector split over blocks is, per block, the xor of the
// transforms of the blocks whose rank contains its rank bitwise).  The G-matrix
// test is combined the same way.  After a cluster barrier every block runs the
// same walk over stages 1..M (the first uncovered CSFG of each stage, in order)
// on the published bits, so all blocks reach the same P, events and stop
// decision without a further exchange.  Iterations that freeze a CSFG take a
// slower path with two more cluster barriers (feedback of enclosing CSFGs that
// span blocks, and the G-matrix test on the new prefix).
#pragma once

#include <cooperative_groups.h>

#include "bp_decode.cuh"

namespace polarbp {

namespace cg = cooperative_groups;

template <int XC>
struct CGeo {
    static constexpr int ML = 12;           // stages inside one block
    static constexpr int M = ML + XC;       // stages of the code
    static constexpr int N = 1 << M;
    static constexpr int C = 1 << XC;       // blocks per cluster
    static constexpr int n = 1 << ML;       // positions per block
    static constexpr int T = n / 8;         // threads per block
    static constexpr int NWL = n / 32;      // 32-bit words of a block's part of an N-bit vector
    static constexpr int NWARP = T / 32;
    static constexpr int FBW = 260;         // words of the per-stage CSFG failure bitmaps
};

// First word of the failure bitmap of local stage jl (1..12): one bit per CSFG.
__host__ __device__ constexpr int fail_word0(int jl) { return jl <= 5 ? jl - 1 : (1 << (jl - 5)) + 3; }

enum : int {
    CC_P = 0,
    CC_DONE = 1,
    CC_FLAGS = 2,   // bit j (1..XC): this block's part of stage j's CSFG fails Eq. (4); bit 31: G test mismatch
    CC_FLAGS2 = 3,  // bit 0: G test mismatch on the prefix after this iteration's freezes
    CC_EVMASK = 4,  // stages with a freeze event this iteration
    CC_EVDIR = 5,   // of those, the ones whose CSFG passed its own check (others complete by enclosure)
    CC_EVLO = 8,    // [16] event ranges, code positions
    CC_EVHI = 24,   // [16]
    CC_FLC = 40,    // [16] flag words of the cluster's blocks (walker scratch)
    CC_PE = 56,     // long long PE-update count
    CC_INTS = 60
};

template <int XC>
struct CLayout {
    using G = CGeo<XC>;
    static constexpr size_t RZ = kRedzone;  // redzone after each region (checked build only)
    static constexpr size_t off_Lx = SmemLayout<12>::bytes;                     // [XC][n] L columns 1..XC
    static constexpr size_t end_Lx = off_Lx + sizeof(float) * XC * G::n;
    static constexpr size_t off_LlrP = end_Lx + RZ;                             // partner's channel LLRs
    static constexpr size_t end_LlrP = off_LlrP + sizeof(float) * G::n;
    static constexpr size_t off_Xw = end_LlrP + RZ;                             // [XC+1][NWL] decisions
    static constexpr size_t end_Xw = off_Xw + 4 * (XC + 1) * G::NWL;
    static constexpr size_t off_V = end_Xw + RZ;                                // [XC][NWL] Eq. (3) of the part
    static constexpr size_t end_V = off_V + 4 * XC * G::NWL;
    static constexpr size_t off_Uc = end_V + RZ;                                // [XC][NWL] combined Eq. (3)
    static constexpr size_t end_Uc = off_Uc + 4 * XC * G::NWL;
    static constexpr size_t off_XfX = end_Uc + RZ;                              // [XC][NWL] feedback decisions
    static constexpr size_t end_XfX = off_XfX + 4 * XC * G::NWL;
    static constexpr size_t off_Wg = end_XfX + RZ;                              // [NWL] u_hat transform
    static constexpr size_t end_Wg = off_Wg + 4 * G::NWL;
    static constexpr size_t off_UE = end_Wg + RZ;                               // [NWL] stored bits transform
    static constexpr size_t end_UE = off_UE + 4 * G::NWL;
    static constexpr size_t off_Fb = end_UE + RZ;                               // [FBW] failure bitmaps
    static constexpr size_t end_Fb = off_Fb + 4 * G::FBW;
    static constexpr size_t off_Cc = end_Fb + RZ;
    static constexpr size_t end_Cc = off_Cc + 4 * CC_INTS;
    static constexpr size_t bytes = end_Cc + RZ;
    static constexpr int ZONES = 10;
    __host__ __device__ static constexpr size_t zone(int k)
    {
        return k == 0 ? end_Lx : k == 1 ? end_LlrP : k == 2 ? end_Xw : k == 3 ? end_V : k == 4 ? end_Uc
             : k == 5 ? end_XfX : k == 6 ? end_Wg : k == 7 ? end_UE : k == 8 ? end_Fb : end_Cc;
    }
};

// Fill (FILL) or compare every redzone of a CLayout<XC> at base.
template <int XC, bool FILL>
__device__ __forceinline__ void cluster_redzones(unsigned char* base, unsigned int* status, int tid, int stride)
{
    if constexpr (kChecked) {
        redzones<12, FILL>(base, status, tid, stride);
#pragma unroll 1
        for (int k = 0; k < CLayout<XC>::ZONES; ++k)
            redzone_pass<FILL>(base, CLayout<XC>::zone(k), kLayoutCluster, k, status, tid, stride);
    }
}

template <int XC>
struct CSmem {
    using G = CGeo<XC>;
    using L = CLayout<XC>;
    float* Lx;
    float* LlrP;
    uint32_t* Xw;
    uint32_t* V;
    uint32_t* Uc;
    uint32_t* XfX;
    uint32_t* Wg;
    uint32_t* UE;
    uint32_t* Fb;
    int* cc;
    __device__ __forceinline__ explicit CSmem(unsigned char* base)
    {
        Lx = reinterpret_cast<float*>(base + L::off_Lx);
        LlrP = reinterpret_cast<float*>(base + L::off_LlrP);
        Xw = reinterpret_cast<uint32_t*>(base + L::off_Xw);
        V = reinterpret_cast<uint32_t*>(base + L::off_V);
        Uc = reinterpret_cast<uint32_t*>(base + L::off_Uc);
        XfX = reinterpret_cast<uint32_t*>(base + L::off_XfX);
        Wg = reinterpret_cast<uint32_t*>(base + L::off_Wg);
        UE = reinterpret_cast<uint32_t*>(base + L::off_UE);
        Fb = reinterpret_cast<uint32_t*>(base + L::off_Fb);
        cc = reinterpret_cast<int*>(base + L::off_Cc);
    }
    __device__ __forceinline__ float* Lcol(int c) { return Lx + (c - 1) * G::n; }  // c = 1..XC
    __device__ __forceinline__ uint32_t* xw(int c) { return Xw + c * G::NWL; }     // c = 0..XC
    __device__ __forceinline__ uint32_t* v(int j) { return V + (j - 1) * G::NWL; } // j = 1..XC
    __device__ __forceinline__ uint32_t* uc(int j) { return Uc + (j - 1) * G::NWL; }
    __device__ __forceinline__ uint32_t* xfx(int j) { return XfX + (j - 1) * G::NWL; }
    __device__ __forceinline__ long long* pe_acc() { return reinterpret_cast<long long*>(cc + CC_PE); }
};

// bit k*S of f -> bit k (S a power of two below 32)
__device__ __forceinline__ uint32_t compact_every(uint32_t f, int S)
{
    uint32_t c = 0;
#pragma unroll 1
    for (int k = 0; k < 32 / S; ++k) c |= ((f >> (k * S)) & 1u) << k;
    return c;
}

// v <- v . F^{(x) log2 S} on each aligned run of S positions of a 4096-bit
// vector held as four words per lane (word 32 q + lane): for every bit h of
// the position, entries with bit h clear absorb (xor) the entry with bit h set.
__device__ __forceinline__ void xform4(uint32_t (&v)[4], int S, int lane)
{
    const int inw = S < 32 ? S : 32;
#pragma unroll 1
    for (int h = 1; h < inw; h <<= 1) {
        const uint32_t mk = xmask(h);
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] ^= (v[q] >> h) & mk;
    }
    const int W = S >> 5;
#pragma unroll 1
    for (int d = 1; d < W && d < 32; d <<= 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t y = __shfl_xor_sync(kFull, v[q], d);
            if (!(lane & d)) v[q] ^= y;
        }
    }
    if (W > 32) {
        v[0] ^= v[1];
        v[2] ^= v[3];
    }
    if (W > 64) {
        v[0] ^= v[2];
        v[1] ^= v[3];
    }
}

// Distributed shared memory: the 32-bit cluster address of a local shared-memory
// object in block `rank` (mapa), and plain loads from such addresses.  The asm is
// volatile with a memory clobber so that no load moves across a cluster barrier
// and no mapped address is hoisted into a long-lived register.
__device__ __forceinline__ uint32_t peer_addr(const void* local, int rank)
{
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(a)
                 : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
    return a;
}
__device__ __forceinline__ uint32_t ld_peer_u32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ float ld_peer_f32(uint32_t addr)
{
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// Word w of the xor of the arrays `arr` of the blocks r | x, x ranging over the
// subsets of the low `bits` rank bits that are clear in r: block r's part of the
// Eq. (3) transform of a vector spanning those 2^bits blocks.  The loop is
// unrolled over every possible x so that the remote loads are in flight together.
template <int XC>
__device__ __forceinline__ uint32_t xor_supersets(cg::cluster_group& cl, uint32_t* arr, int r, int bits, int w)
{
    uint32_t out = arr[w];
    const int free = ((1 << bits) - 1) & ~r;
#pragma unroll
    for (int x = 1; x < (1 << XC); ++x) {
        if ((x & ~free) == 0) out ^= ld_peer_u32(peer_addr(arr + w, r | x));
    }
    return out;
}

// Warp: Eqs. (2)-(4) for every CSFG of local stage jl (1..12) of this block's
// part; bit k of the stage's bitmap = CSFG k fails Eq. (4).
template <int XC>
__device__ __forceinline__ void local_stage_checks(Smem<12>& sm, CSmem<XC>& cs, int jl, int lane)
{
    const int S = 1 << (12 - jl);
    uint32_t u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = snap_word<12>(sm.hd, jl, 32 * (32 * q + lane));
    xform4(u, S, lane);
    uint32_t bad[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) bad[q] = u[q] & sm.Fz[32 * q + lane];
    uint32_t* fb = cs.Fb + fail_word0(jl);
    if (S >= 32) {
        const int W = S >> 5;  // words per CSFG
        uint32_t bb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) bb[q] = __ballot_sync(kFull, bad[q] != 0u);
        if (W > 32) {  // two CSFGs of 64 words (stage 1 only)
            if (lane == 0) fb[0] = ((bb[0] | bb[1]) ? 1u : 0u) | ((bb[2] | bb[3]) ? 2u : 0u);
        } else {
            const int nb = 32 / W;
            uint32_t mine = 0u;  // lane w < (bitmap words) assembles bitmap word w
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t f = bb[q];
#pragma unroll 1
                for (int h = 1; h < W; h <<= 1) f |= f >> h;
                const uint32_t c = __ballot_sync(kFull, lane < nb && ((f >> (lane * W)) & 1u));
                const int first = 32 * q / W;  // first CSFG of this group of 32 words
                if ((first >> 5) == lane) mine |= c << (first & 31);
            }
            const int nwords = (128 / W + 31) / 32;
            if (lane < nwords) fb[lane] = mine;
        }
    } else {
        // S < 32: 32/S CSFGs per word; S consecutive words fill one bitmap word
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t f = bad[q];
#pragma unroll 1
            for (int h = 1; h < S; h <<= 1) f |= f >> h;
            uint32_t c = S == 1 ? f : compact_every(f, S);
            const int w = 32 * q + lane;
            c <<= (w % S) * (32 / S);
#pragma unroll 1
            for (int d = 1; d < S; d <<= 1) c |= __shfl_xor_sync(kFull, c, d);
            if ((w % S) == 0) fb[w / S] = c;
        }
    }
}

// Warp: this block's part of u_hat on the prefix P (stored bits on covered
// positions, HD(R[M]) elsewhere, 0 on frozen positions), Eq. (3)-transformed
// over the part, into dst.
template <int XC>
__device__ __forceinline__ void uhat_transform(Smem<12>& sm, int Ploc, uint32_t* dst, int lane)
{
    uint32_t u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int w = 32 * q + lane;
        uint32_t cov;
        if (Ploc >= 32 * (w + 1)) cov = kFull;
        else if (Ploc <= 32 * w) cov = 0u;
        else cov = (1u << (Ploc - 32 * w)) - 1u;
        const uint32_t hdm = snap_word<12>(sm.hd, 12, 32 * w);
        u[q] = (sm.U[w] & cov) | (hdm & ~sm.Fz[w] & ~cov);
    }
    xform4(u, 4096, lane);
#pragma unroll
    for (int q = 0; q < 4; ++q) dst[32 * q + lane] = u[q];
}

// One codeword per cluster; block r of the cluster owns positions [r n, (r+1) n).
template <int XC, bool GSTOP, bool FREEZE, bool TRACE>
__global__ void __launch_bounds__(512, 1) bp_decode_cluster(DecodeArgs a)
{
    using G = CGeo<XC>;
    using GL = Geo<12>;
    constexpr int M = G::M, N = G::N, n = G::n, T = G::T, NWL = G::NWL, EL = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const long long cw = blockIdx.x / G::C;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Smem<12> sm(smem_raw);
    CSmem<XC> cs(smem_raw);
    sm.L0 = cs.Lcol(XC);
    const int base = r * n;  // first code position of this block's part
    cluster_redzones<XC, true>(smem_raw, a.status, tid, T);

    const float* llr = a.llr + cw * N;
    const long long tb0 = TRACE ? cw * a.max_iter * (long long)(M + 1) * N : 0;
    // pointers of the lower sweep: columns XC.., positions base..
    const CwIO io{llr + base,
                  a.frozen_words + (base >> 5),
                  a.u_hat + cw * N + base,
                  nullptr,
                  nullptr,
                  TRACE ? a.trace_L + tb0 + (long long)XC * N + base : nullptr,
                  TRACE ? a.trace_R + tb0 + (long long)XC * N + base : nullptr,
                  nullptr,
                  0};

    // ---- initial state
    for (int w = tid; w < NWL; w += T) {
        sm.Fz[w] = a.frozen_words[(base >> 5) + w];
        sm.U[w] = 0u;
    }
    for (int i = tid; i < GL::NB * GL::BUF; i += T) sm.Lb[i] = 0.f;
    for (int i = tid; i < XC * n; i += T) cs.Lx[i] = 0.f;
    {
        uint32_t* hd32 = reinterpret_cast<uint32_t*>(sm.hd);
        for (int i = tid; i < (int)(SmemLayout<12>::hd_bytes / 4); i += T) hd32[i] = 0u;
    }
    if (tid == 0) {
        cs.cc[CC_P] = 0;
        cs.cc[CC_DONE] = 0;
        cs.cc[CC_FLAGS] = 0;
        cs.cc[CC_FLAGS2] = 0;
        *cs.pe_acc() = 0;
    }
    Regs<12> rg;
    {
        const int p0 = r ^ (1 << (XC - 1));  // stage-0 partner
        bool finite = true;
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const int i = e * T + tid;
            // bit-reversed order: code position q was received at channel position rev(q)
            const int q0 = base + i, q1 = p0 * n + i;
            const float v = llr[a.bitrev ? (int)(__brev((unsigned)q0) >> (32 - M)) : q0];
            finite &= isfinite(v);
            sm.llr[i] = v;
            cs.LlrP[i] = llr[a.bitrev ? (int)(__brev((unsigned)q1) >> (32 - M)) : q1];
        }
        if (!finite) atomicOr(a.status, 1u);
#pragma unroll
        for (int c = 0; c < GL::NRA; ++c)
#pragma unroll
            for (int e = 0; e < EL; ++e) rg.Lr[c][e] = 0.f;
        __syncthreads();
        // source-side prior: +inf on frozen positions, 0 elsewhere (column 12 is in shared memory)
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const int i = elem_index<12, GL::NP - 1>(tid, e);
            sm.Lm[i] = bit_of(sm.Fz, i) ? INFINITY : 0.f;
        }
    }
    cl.sync();  // every block of the cluster has started and initialised

    int it = 1;
    for (; it <= a.max_iter; ++it) {
        const int P0 = cs.cc[CC_P];
        const int Ploc0 = min(max(P0 - base, 0), n);
        const long long tb = TRACE ? (long long)(it - 1) * (M + 1) * N : 0;
#pragma unroll
        for (int e = 0; e < EL; ++e) rg.R[e] = sm.llr[e * T + tid];
        if constexpr (TRACE) {
#pragma unroll
            for (int e = 0; e < EL; ++e) a.trace_R[tb0 + tb + base + e * T + tid] = rg.R[e];
        }

        // ---- cross stages 0..XC-1
#pragma unroll
        for (int s = 0; s < XC; ++s) {
            const int bitp = XC - 1 - s;
            const int pr = r ^ (1 << bitp);
            const bool aside = ((r >> bitp) & 1) == 0;
            const float* Lown = cs.Lcol(s + 1);
            const uint32_t Lpeer = peer_addr(cs.Lcol(s + 1) + tid, pr);
            const uint32_t Rpeer = peer_addr(sm.Rx + (s & 1) * GL::BUF + tid, pr);
            // the CSFG of stage s holding this block spans blocks [(r >> (XC-s)) << (XC-s), ...)
            const bool covered = FREEZE && s > 0 && ((((r >> (XC - s)) + 1) << (M - s)) <= P0);
            uint32_t xbits = 0;
            // all loads first: the partner's columns are remote, so every load of the
            // stage is issued before the first use (stores below may not be reordered
            // above loads of possibly the same memory, which would serialise them)
            float Lov[EL], Lpv[EL], Rpv[EL];
#pragma unroll
            for (int e = 0; e < EL; ++e) {
                const int i = e * T + tid;
                Lpv[e] = ld_peer_f32(Lpeer + 4 * e * T);
                Rpv[e] = s == 0 ? cs.LlrP[i] : ld_peer_f32(Rpeer + 4 * e * T);
                Lov[e] = Lown[i];
            }
#pragma unroll
            for (int e = 0; e < EL; ++e) {
                const int i = e * T + tid;
                const float Lo = Lov[e], Lp = Lpv[e], Ro = rg.R[e], Rp = Rpv[e];
                float nL, nR;
                if (aside) {
                    const float t = __fadd_rn(Lp, Rp);
                    nL = fms(Lo, t, a.alpha);
                    nR = fms(Ro, t, a.alpha);
                } else {
                    const float g = fms(Lp, Rp, a.alpha);
                    nL = __fadd_rn(Lo, g);
                    nR = __fadd_rn(Ro, g);
                }
                if (s > 0 && !covered) cs.Lcol(s)[i] = nL;
                if (s == 0 && GSTOP) xbits |= (__fadd_rn(Ro, nL) < 0.f ? 1u : 0u) << e;
                if constexpr (TRACE) {
                    if (s == 0) a.trace_L[tb0 + tb + base + i] = nL;
                    a.trace_R[tb0 + tb + (long long)(s + 1) * N + base + i] = nR;
                }
                rg.R[e] = nR;
            }
            if (s == 0 && GSTOP) {
#pragma unroll
                for (int e = 0; e < EL; ++e) {
                    const uint32_t wv = __ballot_sync(kFull, (xbits >> e) & 1u);
                    if (lane == 0) cs.xw(0)[16 * e + warp] = wv;
                }
            }
            if (FREEZE) {
#pragma unroll
                for (int e = 0; e < EL; ++e) {
                    const uint32_t wv = __ballot_sync(kFull, rg.R[e] < 0.f);
                    if (lane == 0) cs.xw(s + 1)[16 * e + warp] = wv;
                }
            }
            if (s + 1 < XC) {
#pragma unroll
                for (int e = 0; e < EL; ++e) sm.Rx[((s + 1) & 1) * GL::BUF + e * T + tid] = rg.R[e];
            }
            cl.sync();
            if (s == 0 && tid == 0) {
                // every block has finished reading the flags of the previous iteration
                cs.cc[CC_FLAGS] = 0;
                cs.cc[CC_FLAGS2] = 0;
            }
        }

        // ---- stages XC..M-1 inside the block
        run_phase<12, 0, GSTOP, FREEZE, TRACE, 1, XC>(rg, sm, tid, true, Ploc0, a.alpha, io, tb, 0);
        __syncthreads();

        bool done = false;
        if constexpr (GSTOP || FREEZE) {
            // ---- C1: per-block checks, published
            if (FREEZE && warp < 12) local_stage_checks<XC>(sm, cs, warp + 1, lane);
            if (FREEZE && warp >= 12 && warp < 12 + XC) {
                const int j = warp - 11;
                uint32_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = cs.xw(j)[32 * q + lane];
                xform4(v, 4096, lane);
                bool bad = false;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    cs.v(j)[32 * q + lane] = v[q];
                    bad |= (v[q] & sm.Fz[32 * q + lane]) != 0u;
                }
                if (j == XC && __any_sync(kFull, bad) && lane == 0) atomicOr(&cs.cc[CC_FLAGS], 1 << XC);
            }
            if (GSTOP && warp == 12 + XC) uhat_transform<XC>(sm, Ploc0, cs.Wg, lane);
            cl.sync();  // B1
            // ---- C2: combine the parts of CSFGs and of the G test that span blocks;
            // four warps per task, one word per lane
            {
                constexpr int NX = FREEZE ? XC - 1 : 0;  // stages 1..XC-1
                const int task = warp >> 2, w = 32 * (warp & 3) + lane;
                if (task < NX) {
                    const int j = task + 1;
                    const uint32_t u = xor_supersets<XC>(cl, cs.v(j), r, XC - j, w);
                    cs.uc(j)[w] = u;
                    if (__any_sync(kFull, (u & sm.Fz[w]) != 0u) && lane == 0) atomicOr(&cs.cc[CC_FLAGS], 1 << j);
                } else if (GSTOP && task == NX) {
                    const uint32_t x = xor_supersets<XC>(cl, cs.Wg, r, XC, w);
                    if (__any_sync(kFull, x != cs.xw(0)[w]) && lane == 0)
                        atomicOr(&cs.cc[CC_FLAGS], (int)0x80000000u);
                }
            }
            cl.sync();  // B2
            // ---- C3: the walk over stages 1..M, identical in every block
            if (warp == 0) {
                int* flc = cs.cc + CC_FLC;
                if (lane < G::C) flc[lane] = (int)ld_peer_u32(peer_addr(cs.cc + CC_FLAGS, lane));
                __syncwarp();
                int P = P0;
                int Ps = P;
                int evmask = 0, evdir = 0;
                int pe_it = N >> 1;
                if constexpr (FREEZE) {
                    int jmin = 1;
#pragma unroll 1
                    while (P < N && jmin <= M) {
                        const int j = lane + 1;
                        bool pass = false;
                        if (j >= jmin && j <= M) {
                            bool fail;
                            if (j < XC) {
                                const int k = P >> (M - j);
                                const int r0 = k << (XC - j), cnt = 1 << (XC - j);
                                int f = 0;
                                for (int q = 0; q < cnt; ++q) f |= flc[r0 + q];
                                fail = (f >> j) & 1;
                            } else if (j == XC) {
                                fail = (flc[P >> (M - XC)] >> XC) & 1;
                            } else {
                                const int owner = P >> (M - XC);
                                const int jl = j - XC;
                                const int kl = (P & (n - 1)) >> (12 - jl);
                                const uint32_t fw = ld_peer_u32(peer_addr(cs.Fb + fail_word0(jl) + (kl >> 5), owner));
                                fail = (fw >> (kl & 31)) & 1u;
                            }
                            pass = !fail;
                        }
                        const unsigned pm = __ballot_sync(kFull, pass);
                        if (!pm) break;
                        const int J = __ffs(pm);  // stage of the first passing check
                        const int S = N >> J;
                        const int cand = (P >> (M - J)) << (M - J);
                        P = cand + S;
                        evmask |= 1 << J;
                        evdir |= 1 << J;
                        if (lane == 0) {
                            cs.cc[CC_EVLO + J] = cand;
                            cs.cc[CC_EVHI + J] = P;
                        }
                        // enclosing CSFGs completed by this freeze
#pragma unroll 1
                        for (int jp = J - 1; jp >= 1; --jp) {
                            const int Sp = N >> jp;
                            if (P & (Sp - 1)) break;
                            evmask |= 1 << jp;
                            if (lane == 0) {
                                cs.cc[CC_EVLO + jp] = P - Sp;
                                cs.cc[CC_EVHI + jp] = P;
                            }
                        }
                        if (lane >= J) Ps = P;
                        jmin = J + 1;
                    }
                    const int pe = (lane >= 1 && lane < M) ? (N - ((Ps >> (M - lane)) << (M - lane))) >> 1 : 0;
                    pe_it = (int)__reduce_add_sync(kFull, (unsigned)pe) + (N >> 1);
                } else {
                    pe_it = M * (N >> 1);
                }
                bool dn = FREEZE && P >= N;
                if (GSTOP && !dn && evmask == 0) {
                    int f = 0;
                    for (int q = 0; q < G::C; ++q) f |= flc[q];
                    dn = (f & (int)0x80000000u) == 0;
                }
                if (lane == 0) {
                    cs.cc[CC_P] = P;
                    cs.cc[CC_DONE] = dn ? 1 : 0;
                    cs.cc[CC_EVMASK] = evmask;
                    cs.cc[CC_EVDIR] = evdir;
                    *cs.pe_acc() += pe_it;
                }
            }
            __syncthreads();
            done = cs.cc[CC_DONE] != 0;
            if constexpr (FREEZE) {
                const int evmask = cs.cc[CC_EVMASK];
                if (evmask) {
                    // ---- slow path: apply this iteration's freezes
                    const int evdir = cs.cc[CC_EVDIR];
                    const int P = cs.cc[CC_P];
                    // E1: CSFGs that passed their check: stored bits and feedback decisions
                    if (warp < M && ((evdir >> (warp + 1)) & 1)) {
                        const int J = warp + 1;
                        const int lo = cs.cc[CC_EVLO + J], hi = cs.cc[CC_EVHI + J];
                        if (lo < base + n && hi > base) {
                            if (J > XC) {
                                const int jl = J - XC, S = hi - lo, llo = lo - base;
                                uint32_t x[4], u[4];
                                if (S >= 32) {
#pragma unroll
                                    for (int q = 0; q < 4; ++q) {
                                        const int w = 32 * q + lane;
                                        x[q] = (w < (S >> 5))
                                                   ? snap_word<12>(sm.hd, jl, llo + 32 * w)
                                                   : 0u;
                                    }
                                } else {
                                    x[0] = (snap_word<12>(sm.hd, jl, llo & ~31) >> (llo & 31)) &
                                           low_mask(S);
                                    x[1] = x[2] = x[3] = 0u;
                                }
#pragma unroll
                                for (int q = 0; q < 4; ++q) u[q] = x[q];
                                xform4(u, S, lane);
                                // CSFGs of several stages may end in one word of U: runs shorter than a
                                // word are or-ed in (their bits are still 0: a position is stored once)
                                if (S >= 32) {
                                    packed_store<4>(sm.U, llo, S, u, lane);
                                } else if (lane == 0) {
                                    atomicOr(&sm.U[llo >> 5], (u[0] & low_mask(S)) << (llo & 31));
                                }
                                packed_store<4>(sm.Xf + jl * GL::NW, llo, S, x, lane);
                                if (lane == 0) {
                                    sm.ev_lo()[jl] = llo;
                                    sm.ev_hi()[jl] = llo + S;
                                }
                            } else {
                                const uint32_t* src = J == XC ? cs.v(XC) : cs.uc(J);
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    sm.U[32 * q + lane] = src[32 * q + lane];
                                    cs.xfx(J)[32 * q + lane] = cs.xw(J)[32 * q + lane];
                                }
                            }
                        }
                    }
                    __syncthreads();
                    // E2: enclosing CSFGs inside the block; transforms for the exchange
                    const int evenc = evmask & ~evdir;
                    if (warp < M && ((evenc >> (warp + 1)) & 1)) {
                        const int J = warp + 1;
                        const int lo = cs.cc[CC_EVLO + J], hi = cs.cc[CC_EVHI + J];
                        if (J >= XC && lo < base + n && hi > base) {
                            const int S = hi - lo, llo = lo - base;
                            uint32_t v[4];
                            packed_load<4>(sm.U, llo, S, v, lane);
                            xform4(v, S, lane);
                            if (J > XC) {
                                const int jl = J - XC;
                                packed_store<4>(sm.Xf + jl * GL::NW, llo, S, v, lane);
                                if (lane == 0) {
                                    sm.ev_lo()[jl] = llo;
                                    sm.ev_hi()[jl] = llo + S;
                                }
                            } else {
#pragma unroll
                                for (int q = 0; q < 4; ++q) cs.xfx(XC)[32 * q + lane] = v[q];
                            }
                        }
                    }
                    if (warp == G::NWARP - 1) {
                        if (evenc & ((1 << XC) - 2)) {  // an enclosing CSFG spans blocks
                            uint32_t v[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) v[q] = sm.U[32 * q + lane];
                            xform4(v, 4096, lane);
#pragma unroll
                            for (int q = 0; q < 4; ++q) cs.UE[32 * q + lane] = v[q];
                        }
                        if (GSTOP && P < N) uhat_transform<XC>(sm, min(max(P - base, 0), n), cs.Wg, lane);
                    }
                    cl.sync();  // E-barrier 1
                    // E3: enclosing CSFGs spanning blocks; G test on the new prefix
                    {
                        const int task = warp >> 2, w = 32 * (warp & 3) + lane;
                        if (task < XC - 1) {
                            const int J = task + 1;
                            const int lo = cs.cc[CC_EVLO + J], hi = cs.cc[CC_EVHI + J];
                            if (((evenc >> J) & 1) && lo < base + n && hi > base)
                                cs.xfx(J)[w] = xor_supersets<XC>(cl, cs.UE, r, XC - J, w);
                        } else if (GSTOP && P < N && task == XC - 1) {
                            const uint32_t x = xor_supersets<XC>(cl, cs.Wg, r, XC, w);
                            if (__any_sync(kFull, x != cs.xw(0)[w]) && lane == 0) atomicOr(&cs.cc[CC_FLAGS2], 1);
                        }
                    }
                    __syncthreads();
                    // feedback (-1)^x_hat * inf on every frozen CSFG's own L column
                    int lmask = 0;  // local stages 1..12 with an event inside this block's part
#pragma unroll 1
                    for (int J = XC + 1; J <= M; ++J) {
                        if (((evmask >> J) & 1) && cs.cc[CC_EVLO + J] < base + n && cs.cc[CC_EVHI + J] > base)
                            lmask |= 1 << (J - XC);
                    }
                    if (lmask) apply_events<12, 1>(rg, sm, tid, lmask);
#pragma unroll 1
                    for (int J = 1; J <= XC; ++J) {
                        if (!((evmask >> J) & 1)) continue;
                        const int lo = cs.cc[CC_EVLO + J], hi = cs.cc[CC_EVHI + J];
                        if (!(lo < base + n && hi > base)) continue;
                        const uint32_t* xf = cs.xfx(J);
#pragma unroll
                        for (int e = 0; e < EL; ++e) {
                            const int i = e * T + tid;
                            cs.Lcol(J)[i] = bit_of(xf, i) ? -INFINITY : INFINITY;
                        }
                    }
                    cl.sync();  // E-barrier 2: feedback visible to the partners
                    if (GSTOP && P < N) {
                        if (warp == 0) {
                            const int f = lane < G::C ? (int)ld_peer_u32(peer_addr(cs.cc + CC_FLAGS2, lane)) : 0;
                            const bool any = __any_sync(kFull, f != 0);
                            if (lane == 0) cs.cc[CC_DONE] = any ? 0 : 1;
                        }
                        __syncthreads();
                        done = cs.cc[CC_DONE] != 0;
                    }
                }
            }
        } else {
            cl.sync();  // column XC written by the lower sweep is read by the partner next
        }
        if constexpr (TRACE) {
            __syncthreads();
            trace_L_columns<12, 1, XC>(rg, sm, tid, true, io, tb);
#pragma unroll 1
            for (int c = 1; c <= XC; ++c)
                for (int i = tid; i < n; i += T) a.trace_L[tb0 + tb + (long long)c * N + base + i] = cs.Lcol(c)[i];
            if (tid == 0 && r == 0) a.trace_P[cw * a.max_iter + it - 1] = cs.cc[CC_P];
        }
        if (done) break;
    }
    const int iters = it <= a.max_iter ? it : a.max_iter;
    cl.sync();  // no block leaves while a partner may still read its shared memory

    // output: stored bits on covered positions, HD(R[M]) elsewhere, 0 on frozen
    {
        const int Ploc = min(max(cs.cc[CC_P] - base, 0), n);
        uint32_t hdM = 0;
        if constexpr (GSTOP || FREEZE) {
            hdM = sm.hd[12 * GL::HDS + tid];
        } else {
#pragma unroll
            for (int e = 0; e < EL; ++e) hdM |= (rg.R[e] < 0.f ? 1u : 0u) << e;
        }
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const int i = elem_index<12, GL::NP - 1>(tid, e);
            uint8_t bit;
            if (i < Ploc) bit = (uint8_t)bit_of(sm.U, i);
            else bit = bit_of(sm.Fz, i) ? 0 : (uint8_t)((hdM >> e) & 1u);
            io.u_hat[i] = bit;
        }
    }
    if (tid == 0 && r == 0) {
        if (a.iters) a.iters[cw] = iters;
        if (a.pe) a.pe[cw] = (GSTOP || FREEZE) ? *cs.pe_acc() : (long long)iters * M * (N >> 1);
    }
    // every shared-memory store of the cluster precedes its last barrier
    cluster_redzones<XC, false>(smem_raw, a.status, tid, T);
}

template <int XC, bool GSTOP, bool FREEZE, bool TRACE>
cudaError_t launch_cluster_one(const LaunchReq& q)
{
    auto kern = bp_decode_cluster<XC, GSTOP, FREEZE, TRACE>;
    constexpr size_t smem = CLayout<XC>::bytes;
    static_assert(smem <= 227 * 1024, "cluster layout exceeds the shared memory of one block");
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)q.args.batch * CGeo<XC>::C, 1, 1);
    cfg.blockDim = dim3(CGeo<XC>::T, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = q.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CGeo<XC>::C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, q.args);
}

template <int XC>
cudaError_t launch_cluster(const LaunchReq& q)
{
    const bool g = q.stop_mode != 0, f = q.freeze_mode != 0;
    if (q.trace) {
        if (g && f) return launch_cluster_one<XC, true, true, true>(q);
        if (g) return launch_cluster_one<XC, true, false, true>(q);
        if (f) return launch_cluster_one<XC, false, true, true>(q);
        return launch_cluster_one<XC, false, false, true>(q);
    }
    if (g && f) return launch_cluster_one<XC, true, true, false>(q);
    if (g) return launch_cluster_one<XC, true, false, false>(q);
    if (f) return launch_cluster_one<XC, false, true, false>(q);
    return launch_cluster_one<XC, false, false, false>(q);
}

}  // namespace polarbp
