// bp_pipe.cuh -- pipelined min-sum BP decoding of polar codes with the G-matrix
// stop and CSFG freezing (reading A), N = 256 .. 4096, one codeword per block.
//
// Method: arXiv 1505.04979, Eq. (1) (Sec. II-A), the CSFG check, freezing order
// and +-inf feedback of Sec. III (Eqs. (2)-(4)), the PE count of Sec. IV.  The
// decisions, stored bits, iteration counts and PE counts are those of
// bp_decode_kernel (bp_decode.cuh); only the schedule of the work differs.
//
// Schedule.  The block has the sweep's worker threads plus one checker warp.  The
// checker runs the CSFG walk of iteration t (the checks of stages 1..M, the
// freezes, the feedback, the G-matrix test) while the workers already sweep
// iteration t+1.  Phase p of sweep t+1 starts once the checker has released it
// (named barrier REL_p), i.e. once every feedback value that phase reads is in
// place; the checker releases phase 0 early when walk t cannot change the
// columns phase 0 reads.  The hard-decision snapshots and the encoding of the
// channel-side decisions are double-buffered by iteration parity, so sweep t+1
// writes one buffer while walk t reads the other.  When walk t decides to stop,
// the partial sweep t+1 is discarded: the outputs come from iteration t's state.
//
// Frozen CSFGs as fixed points.  A covered CSFG B of stage j keeps, in every
// column c = j..M, the +-inf messages of its stored source bits encoded through
// stages M-1 .. c (column M holds (-1)^u inf, column j the feedback
// (-1)^x_hat inf of Sec. III).  With those inputs every PE inside B reproduces
// its own L outputs exactly -- f(+-inf, +-inf) = +-inf with the product's sign,
// and +-inf plus a finite value stays +-inf -- while its R outputs stay finite
// and are read only inside B.  So the sweep runs every PE unguarded and needs
// neither the covered prefix nor keep-selects; a freeze writes its CSFG's
// columns j..M once, a completed enclosing CSFG its root column.  The L
// messages read from outside covered CSFGs are the same as with skipped PEs.
#pragma once

#include "bp_decode.cuh"

namespace polarbp {

// Named barriers: 0 is __syncthreads; REL_p = kBarRel + p (checker releases phase
// p of the next sweep); kBarSwept (workers: sweep done, snapshots written).
constexpr int kBarRel = 1;
constexpr int kBarSwept = 6;

__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int M>
struct PipeGeo {
    static constexpr int WORKERS = Geo<M>::BLOCK;
    static constexpr int THREADS = WORKERS + 32;
    static constexpr int MIN_BLOCKS = (800 / THREADS) < 1 ? 1 : (800 / THREADS);
};

// Shared memory: the one-block decoder's layout plus a second snapshot buffer and
// a second pair of G-encoding buffers (iteration parity 1).
template <int M>
struct PipeLayout {
    using L = SmemLayout<M>;
    static constexpr size_t off_hd1 = (L::bytes + 31) / 32 * 32;
    static constexpr size_t end_hd1 = off_hd1 + L::hd_bytes;
    static constexpr size_t off_ge1 = (end_hd1 + L::RZ + 15) / 16 * 16;
    static constexpr size_t end_ge1 = off_ge1 + 2 * sizeof(uint32_t) * Geo<M>::NW;
    static constexpr size_t bytes = (end_ge1 + L::RZ + 15) / 16 * 16;
};

// Fill (FILL) or compare every redzone of a PipeLayout<M> at base.
template <int M, bool FILL>
__device__ __forceinline__ void pipe_redzones(unsigned char* base, unsigned int* status, int tid, int stride)
{
    if constexpr (kChecked) {
        redzones<M, FILL>(base, status, tid, stride);
        redzone_pass<FILL>(base, PipeLayout<M>::end_hd1, kLayoutPipe, 0, status, tid, stride);
        redzone_pass<FILL>(base, PipeLayout<M>::end_ge1, kLayoutPipe, 1, status, tid, stride);
    }
}

template <int M>
__device__ __forceinline__ void pipe_buffers(Smem<M>& sm, unsigned char* base, int it)
{
    using L = SmemLayout<M>;
    using PL = PipeLayout<M>;
    sm.hd = base + ((it & 1) ? PL::off_hd1 : L::off_Hd);
    sm.Ge = reinterpret_cast<uint32_t*>(base + ((it & 1) ? PL::off_ge1 : L::off_Ge));
}

// -inf / +inf of a decision bit written into column C (shared-memory columns only:
// the boundary columns and column M) at natural position i.
template <int M>
__device__ __forceinline__ void put_smem_L(Smem<M>& sm, int C, int i, uint32_t bit)
{
    using G = Geo<M>;
    const float v = bit ? -INFINITY : INFINITY;
    if (C == M) {
        sm.Lm[i] = v;
    } else {
        // the padding shift of boundary b (see Geo::padsh), at run time
        const int b = C / 3 - 1;
        const int sh = M <= 7 ? 2 : (M <= 9 ? 3 : (b == 0 ? 5 : 3));
        sm.Lb[b * G::BUF + i + (i >> sh)] = v;
    }
}

__device__ __forceinline__ bool smem_column(int M, int C) { return C == M || (C > 0 && C < M && C % 3 == 0); }

// Record the feedback range [lo, hi) of register column C for the workers.  The
// CSFGs an iteration freezes are consecutive, so the ranges of one column grow.
template <int M>
__device__ __forceinline__ void note_reg_event(Smem<M>& sm, int C, int lo, int hi, int lane)
{
    if (lane == 0) {
        if (!(sm.ctl[CTL_EVENT] & (1 << C))) sm.ev_lo()[C] = lo;
        sm.ev_hi()[C] = hi;
        sm.ctl[CTL_EVENT] |= 1 << C;
    }
}

// Freeze a CSFG of 64 or more positions (rare): stage j, positions [bs, bs + S);
// Xf[j] over the CSFG already holds its decisions.  Column by column, the words of
// the CSFG are spread over the lanes.
template <int M>
__device__ __forceinline__ void freeze_big_fp(Smem<M>& sm, int j, int bs, int lane)
{
    constexpr int N = Geo<M>::N, NW = Geo<M>::NW;
    const int S = N >> j;
    const int w0 = bs >> 5, nw = S >> 5;
#pragma unroll 1
    for (int c = j; c <= M; ++c) {
        __syncwarp();
        const uint32_t* xc = sm.Xf + c * NW;
        if (smem_column(M, c)) {
            for (int i = lane; i < S; i += 32) put_smem_L<M>(sm, c, bs + i, (xc[(bs + i) >> 5] >> ((bs + i) & 31)) & 1u);
        } else {
            note_reg_event<M>(sm, c, bs, bs + S, lane);
        }
        if (c < M) {
            const int h = N >> (c + 1);
            uint32_t* xn = sm.Xf + (c + 1) * NW;
            for (int q = lane; q < nw; q += 32) {
                uint32_t v = xc[w0 + q];
                if (h >= 32) {
                    const int d = h >> 5;
                    if (!(q & d)) v ^= xc[w0 + q + d];
                } else {
                    v ^= (v >> h) & xmask(h);
                }
                xn[w0 + q] = v;
            }
        } else {
            for (int q = lane; q < nw; q += 32) sm.U[w0 + q] = xc[w0 + q];
        }
    }
    __syncwarp();
}

// After the first freeze of an iteration ended at P (stage J), complete every
// enclosing CSFG that is now fully covered: its decisions are the xor of its
// halves' (F^{(x)k} = [[F', 0], [F', F']]), written to its root column only (its
// deeper columns already hold its halves' fixed points).
template <int M>
__device__ __forceinline__ void complete_fp(Smem<M>& sm, int P, int J, int lane)
{
    constexpr int N = Geo<M>::N, NW = Geo<M>::NW;
#pragma unroll 1
    for (int jp = J - 1; jp >= 1; --jp) {
        const int Sp = N >> jp;
        if (P & (Sp - 1)) break;
        const int bp = P - Sp;
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
        __syncwarp();
        if (smem_column(M, jp)) {
            for (int i = lane; i < Sp; i += 32) put_smem_L<M>(sm, jp, bp + i, (xo[(bp + i) >> 5] >> ((bp + i) & 31)) & 1u);
        } else {
            note_reg_event<M>(sm, jp, bp, P, lane);
        }
        __syncwarp();
    }
}


// Release phases [released, upto) of the next sweep (warp-uniform).
template <int M>
__device__ __forceinline__ void release_upto(int& released, int upto)
{
    if (upto > released) {
        __syncwarp();
        __threadfence_block();
#pragma unroll
        for (int p = 0; p < Geo<M>::NP; ++p)
            if (p >= released && p < upto) bar_arrive(kBarRel + p, PipeGeo<M>::THREADS);
        released = upto;
    }
}

// The CSFG walk of one iteration (stages 1..M in order, reading A): the same
// checks, freezes and PE count as resolve_fast (bp_decode.cuh), with fixed-point
// commits.  Returns the iteration's PE updates (Sec. IV).  `ss` is the
// lane-constant slot layout of the speculative check (spec_slots).
// `released` counts the phases of the next sweep released so far.  Phase 0 goes
// before the small stages are checked when no freeze and no completion of this
// walk can reach the columns it reads (1..3): no CSFG of >= 64 positions froze,
// stages M-5.. only write columns >= M-5 >= 4, and the first freeze ends at most
// at 32 w0 + 64, so it completes a stage-3 CSFG only if a multiple of N/8 lies in
// (P, 32 w0 + 64].  Once the freezes are known, the phases that read only
// columns below every column still to be written go; the rest but the last after
// the commits.  The last phase waits for the stop decision (the workers must
// learn it at a release at the latest).
//
// The CSFGs of <= 32 positions that freeze in one iteration lie in the two words
// w0, w0 + 1 and are committed together: lane 2 (c - M + 5) + k holds column c on
// word w0 + k.  Column c of every CSFG of stage j <= c frozen now is the new
// stored bits encoded through the butterflies of stages M-1 .. c (steps 1 .. S_c/2,
// which stay inside each aligned CSFG of stage <= c); the columns of one stage
// cover the union of those CSFGs, a contiguous range.  The enclosing CSFGs of
// <= 32 positions that the first freeze completes join that commit (their root
// column is the same encoding of their stored bits); larger ones go through
// complete_fp.  The kernel is bound by instruction fetch as much as by issue, so
// the walk keeps one copy of each rare path.
template <int M>
__device__ __forceinline__ int walk_pipe(Smem<M>& sm, const SpecSlots<M>& ss, int& P, int lane, int& released)
{
    using SP = Spec<M>;
    constexpr int N = Geo<M>::N, NW = Geo<M>::NW;
    constexpr int JB = M - 6;  // stages with CSFGs of >= 64 positions
    constexpr int JS = M - 5;  // first stage with CSFGs of <= 32 positions
    static_assert(natural_rows<M>() && JB >= 2 && SP::JB == JB + 1, "codes of N >= 256");
    int Ps = P;  // lane s (1 <= s < M): P after the check of stage s
    bool first = true;
    int jmin = 1;
    int jf = 0, p1 = 0;  // stage and end of the iteration's first freeze
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
        for (int r = 0; r < SP::R; ++r)
            if (sp.lvl[r] == J) sm.Xf[J * NW + (cand >> 5) + sp.w[r]] = sp.x[r];
        freeze_big_fp<M>(sm, J, cand, lane);
        P = cand + (N >> J);
        if (first) {
            jf = J;
            p1 = P;
        }
        if (lane >= J) Ps = P;
        first = false;
        jmin = J + 1;
    }
    if (P < N) {
        const int w0 = P >> 5;
        if constexpr (M >= 9) {
            constexpr int S3 = N >> 3;
            if (first && (((32 * w0 + 64) & ~(S3 - 1)) <= P)) release_upto<M>(released, 1);
        }
        // lane l < 12: stage (and column) jl = JS + l/2 on word wl = w0 + (l & 1)
        const int jl = JS + (lane >> 1);
        const int wl = w0 + (lane & 1);
        const bool act = lane < 12 && wl < NW;
        const int Sl = N >> (jl < M ? jl : M);
        uint32_t u = 0u, pw = 0u;
        if (act) {
            const uint32_t x = snap_word<M>(sm.hd, jl, 32 * wl);
            u = x;
#pragma unroll
            for (int h = 1; h < 32; h <<= 1)
                if (h < Sl) u ^= (u >> h) & xmask(h);
            uint32_t bad = u & sm.Fz[wl];
#pragma unroll
            for (int h = 1; h < 32; h <<= 1)
                if (h < Sl) bad |= bad >> h;
            pw = ~bad;  // bit k S: CSFG k of the word passes (the chain reads block starts only)
        }
        uint32_t pa[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) pa[i] = __shfl_sync(kFull, pw, i);
        unsigned frz = 0u;  // bit jj: stage JS + jj froze
        int js = 0;         // stage of the first small freeze
        uint32_t mk = 0u;   // this lane's stage: the frozen CSFG's bits in word wl
#pragma unroll
        for (int jj = 0; jj < 6; ++jj) {
            const int S = N >> (JS + jj);
            if (P < N) {
                const int bs = P & ~(S - 1);
                const int off = bs - 32 * w0;  // 0 <= off < 64
                const uint32_t word = off < 32 ? pa[2 * jj] : pa[2 * jj + 1];
                if ((word >> (off & 31)) & 1u) {
                    if (!frz) {
                        js = JS + jj;
                        if (first) {
                            jf = js;
                            p1 = bs + S;
                        }
                    }
                    frz |= 1u << jj;
                    if ((lane >> 1) == jj && (bs >> 5) == wl) mk = low_mask(S) << (bs & 31);
                    P = bs + S;
                    if (lane >= JS + jj) Ps = P;
                }
            }
        }
        int cmin = M + 1;
        if (first) {
            // every column this walk still writes is >= cmin: the stage of the first freeze,
            // or of the last CSFG it completes; release the phases that read only columns
            // below it (phase p reads columns 3p+1 .. 3p+3), all but the last one
            if (frz) {
                cmin = js;
                while (cmin > 1 && !(p1 & ((N >> (cmin - 1)) - 1))) --cmin;
            }
            const int pr = cmin >= 4 ? (cmin - 4) / 3 + 1 : 0;
            release_upto<M>(released, pr < Geo<M>::NP - 1 ? pr : Geo<M>::NP - 1);
        }
        if (frz) {
            // new stored bits of the two words
            const uint32_t m_e = __reduce_or_sync(kFull, (lane & 1) ? 0u : mk);
            const uint32_t m_o = __reduce_or_sync(kFull, (lane & 1) ? mk : 0u);
            const uint32_t v_e = __reduce_or_sync(kFull, (lane & 1) ? 0u : (u & mk));
            const uint32_t v_o = __reduce_or_sync(kFull, (lane & 1) ? (u & mk) : 0u);
            const uint32_t mw = (lane & 1) ? m_o : m_e;
            uint32_t un = 0u;
            if (act) un = (sm.U[wl] & ~mw) | ((lane & 1) ? v_o : v_e);
            __syncwarp();
            if (lane < 2 && mw) sm.U[wl] = un;
            // the enclosing CSFGs of <= 32 positions the first freeze completes (stages cmin ..
            // js-1, each ending at p1, in word (p1-1)/32): their root columns take the encoding
            // of their stored bits like the frozen CSFGs' columns do
            uint32_t mkp = 0u;
            if (first && act && jl < js && jl >= cmin && ((p1 - 1) >> 5) == wl) {
                const int Sp = N >> jl;
                mkp = low_mask(Sp) << ((p1 - Sp) & 31);
            }
            // column jl: the CSFGs of stages <= jl frozen or completed now (prefix-or over the stages)
            uint32_t mc = mk | mkp, t;
            t = __shfl_up_sync(kFull, mc, 2);  if (lane >= 2) mc |= t;
            t = __shfl_up_sync(kFull, mc, 4);  if (lane >= 4) mc |= t;
            t = __shfl_up_sync(kFull, mc, 8);  if (lane >= 8) mc |= t;
            if (!act) mc = 0u;
            uint32_t xc = un;  // encode through stages M-1 .. jl: steps 1 .. S_jl / 2
#pragma unroll
            for (int h = 1; h < 32; h <<= 1)
                if (h < Sl) xc ^= (xc >> h) & xmask(h);
            if (mc) {
                uint32_t* px = sm.Xf + jl * NW + wl;
                *px = (*px & ~mc) | (xc & mc);
            }
            // register columns: their range [lo, hi) for the workers
            const uint32_t mc1 = __shfl_down_sync(kFull, mc, 1);
            bool ev = false;
            if (act && !(lane & 1) && !smem_column(M, jl) && (mc | mc1)) {
                const unsigned long long m64 = (unsigned long long)mc | ((unsigned long long)mc1 << 32);
                const int lo = 32 * w0 + __ffsll((long long)m64) - 1;
                // a CSFG of >= 64 positions frozen earlier in this iteration starts the range
                if (!(sm.ctl[CTL_EVENT] & (1 << jl))) sm.ev_lo()[jl] = lo;
                sm.ev_hi()[jl] = 32 * w0 + 64 - __clzll((long long)m64);
                ev = true;
            }
            const unsigned evm = __reduce_or_sync(kFull, ev ? (1u << jl) : 0u);
            if (lane == 0) sm.ctl[CTL_EVENT] |= (int)evm;
            // shared-memory columns (the boundary columns and column M): one position per lane
            const int nk = P > 32 * (w0 + 1) ? 2 : 1;  // a frozen CSFG reaches word w0 + 1
            const int c0 = (first && cmin < js) ? (cmin > JS ? cmin : JS) : js;
#pragma unroll 1
            for (int c = c0; c <= M; ++c) {
                if (!smem_column(M, c)) continue;
                for (int k = 0; k < nk; ++k) {
                    const int src = 2 * (c - JS) + k;
                    const uint32_t m = __shfl_sync(kFull, mc, src);
                    const uint32_t xv = __shfl_sync(kFull, xc, src);
                    if ((m >> lane) & 1u) put_smem_L<M>(sm, c, 32 * (w0 + k) + lane, (xv >> lane) & 1u);
                }
            }
            __syncwarp();
        }
    }
    // the enclosing CSFGs the iteration's first freeze completes (later freezes of the same
    // iteration add less than its size, so they complete none): after a freeze of <= 32
    // positions the commit above took those of stages >= M-5, the rest go here
    {
        const int jc = (first && jf > JS) ? JS : jf;
        if (jc > 1 && !(p1 & ((N >> (jc - 1)) - 1))) complete_fp<M>(sm, p1, jc, lane);
    }
    // every feedback value is in place: all phases but the last (which waits for the stop decision)
    release_upto<M>(released, Geo<M>::NP - 1);
    const int pe = (lane >= 1 && lane < M) ? (N - ((Ps >> (M - lane)) << (M - lane))) >> 1 : 0;
    return (int)__reduce_add_sync(kFull, (unsigned)pe) + (N >> 1);
}

// Phase PH of a worker's sweep: wait for the checker's release, stop if the
// checker has decided to (consuming the releases of the remaining phases), write
// the feedback of this phase's register columns, then the phase's stages with
// their snapshots (no keep-selects: covered CSFGs are fixed points).
template <int M, int PH, bool GSTOP>
__device__ __forceinline__ bool sweep_pipe(Regs<M>& rg, Smem<M>& sm, int tid, float alpha, const CwIO& a)
{
    using G = Geo<M>;
    constexpr int EL = G::EL, THREADS = PipeGeo<M>::THREADS;
    bar_sync(kBarRel + PH, THREADS);
    if (*reinterpret_cast<volatile int*>(&sm.ctl[CTL_DONE])) {
#pragma unroll
        for (int q = PH + 1; q < G::NP; ++q) bar_sync(kBarRel + q, THREADS);
        return false;
    }
    {
        const int mask = *reinterpret_cast<volatile int*>(&sm.ctl[CTL_EVENT]);
        constexpr int C1 = 3 * PH + 1, C2 = 3 * PH + 2;
        if constexpr (G::is_reg(C1) && G::owner(C1) == PH)
            if (mask & (1 << C1)) apply_column<M, C1>(rg, sm, tid);
        if constexpr (G::is_reg(C2) && G::owner(C2) == PH)
            if (mask & (1 << C2)) apply_column<M, C2>(rg, sm, tid);
    }
    if constexpr (PH > 0) {
        constexpr int SH = G::padsh(PH - 1);
        const int pb = padded_base<M, PH, SH>(tid);
#pragma unroll
        for (int e = 0; e < EL; ++e) rg.R[e] = sm.Rx[((PH - 1) & 1) * G::BUF + pb + padded_off<M, PH, SH>(e)];
        if constexpr (GSTOP) genc_step<M, PH>(sm, tid);
    }
    run_stage<M, PH, 0, GSTOP, true, false, 0, false>(rg, sm, tid, 0, alpha, a, 0);
    if constexpr (PH + 1 < G::NP) {
        constexpr int SH = G::padsh(PH);
        const int pb = padded_base<M, PH, SH>(tid);
#pragma unroll
        for (int e = 0; e < EL; ++e) sm.Rx[(PH & 1) * G::BUF + pb + padded_off<M, PH, SH>(e)] = rg.R[e];
        return sweep_pipe<M, PH + 1, GSTOP>(rg, sm, tid, alpha, a);
    } else {
        return true;
    }
}

// Decode one codeword with the whole block (Geo<M>::BLOCK workers and one
// checker warp) on the block's shared memory smem_raw.  Every named barrier the
// call uses is complete when it returns, so a block may decode codewords back
// to back (after a block barrier).
template <int M, bool GSTOP>
__device__ __forceinline__ void decode_pipe_codeword(const CwIO& a, int max_iter, float alpha, unsigned int* status,
                                                     unsigned char* smem_raw)
{
    using G = Geo<M>;
    constexpr int N = G::N, EL = G::EL, T = G::T, NW = G::NW, NP = G::NP;
    constexpr int WORKERS = PipeGeo<M>::WORKERS, THREADS = PipeGeo<M>::THREADS;
    static_assert(natural_rows<M>() && T == WORKERS, "codes of N >= 256");
    const int tid = threadIdx.x;
    Smem<M> sm(smem_raw);

    pipe_redzones<M, true>(smem_raw, status, tid, THREADS);
    for (int w = tid; w < NW; w += THREADS) {
        sm.Fz[w] = a.frozen_words[w];
        sm.U[w] = 0u;
    }
    for (int i = tid; i < G::NB * G::BUF; i += THREADS) sm.Lb[i] = 0.f;
    // source-side prior (reading: +inf on frozen positions, 0 elsewhere)
    for (int i = tid; i < N; i += THREADS) sm.Lm[i] = ((a.frozen_words[i >> 5] >> (i & 31)) & 1u) ? INFINITY : 0.f;
    for (int b = 0; b < 2; ++b) {
        pipe_buffers<M>(sm, smem_raw, b);
        uint32_t* hd32 = reinterpret_cast<uint32_t*>(sm.hd);
        for (int i = tid; i < (int)(SmemLayout<M>::hd_bytes / 4); i += THREADS) hd32[i] = 0u;
    }
    if (tid == 0) {
        sm.ctl[CTL_P] = 0;
        sm.ctl[CTL_DONE] = 0;
        sm.ctl[CTL_EVENT] = 0;
        sm.ctl[CTL_Q] = 1;
        *sm.pe_acc() = 0;
    }
    if (!stage_llr<M>(sm.llr, a.llr, tid, THREADS, a.bitrev)) atomicOr(status, 1u);
    __syncthreads();

    if (tid < WORKERS) {
        Regs<M> rg;
#pragma unroll
        for (int c = 0; c < G::NRA; ++c)
#pragma unroll
            for (int e = 0; e < EL; ++e) rg.Lr[c][e] = 0.f;
        for (int it = 1;; ++it) {
            pipe_buffers<M>(sm, smem_raw, it);
#pragma unroll
            for (int e = 0; e < EL; ++e) rg.R[e] = sm.llr[e * T + tid];
            if (!sweep_pipe<M, 0, GSTOP>(rg, sm, tid, alpha, a)) break;
            __threadfence_block();
            bar_arrive(kBarSwept, THREADS);
        }
    } else {
        const int lane = tid - WORKERS;
#pragma unroll
        for (int p = 0; p < NP; ++p) bar_arrive(kBarRel + p, THREADS);  // sweep 1 reads the start state
        int P = 0, t = 1;
        long long pe = 0;
        SpecSlots<M> ss;
        spec_slots<M>(ss, lane);
        for (;; ++t) {
            bar_sync(kBarSwept, THREADS);
            pipe_buffers<M>(sm, smem_raw, t);
            if (lane == 0) {
                sm.ctl[CTL_EVENT] = 0;
                if (t >= max_iter) sm.ctl[CTL_DONE] = 1;  // the iteration cap: no further sweep
            }
            __syncwarp();
            int released = 0;
            pe += walk_pipe<M>(sm, ss, P, lane, released);
            bool done = (P >= N) || t >= max_iter;
            if constexpr (GSTOP) {
                if (!done) done = gmatrix_ok_pre<M>(sm, P, lane);
            }
            if (done && lane == 0) sm.ctl[CTL_DONE] = 1;
            release_upto<M>(released, NP);
            if (done) break;
        }
        if (lane == 0) {
            sm.ctl[CTL_P] = P;
            sm.ctl[CTL_Q] = t;
            *sm.pe_acc() = pe;
        }
    }
    __syncthreads();

    // output: stored bits on covered positions, HD(R[M]) of the last iteration elsewhere, 0 on frozen
    const int iters = sm.ctl[CTL_Q];
    pipe_buffers<M>(sm, smem_raw, iters);
    if (tid < WORKERS) {
        const int P = sm.ctl[CTL_P];
        const uint32_t hdM = sm.hd[M * G::HDS + tid];
#pragma unroll
        for (int e = 0; e < EL; ++e) {
            const int i = elem_index<M, NP - 1>(tid, e);
            uint8_t bit;
            if (i < P) bit = (uint8_t)bit_of(sm.U, i);
            else bit = bit_of(sm.Fz, i) ? 0 : (uint8_t)((hdM >> e) & 1u);
            a.u_hat[i] = bit;
        }
    }
    if (tid == 0) {
        if (a.iters) *a.iters = iters;
        if (a.pe) *a.pe = *sm.pe_acc();
    }
    if constexpr (kChecked) {
        __syncthreads();  // every store of this decode is done
        pipe_redzones<M, false>(smem_raw, status, tid, THREADS);
    }
}

// One codeword per block.
template <int M, bool GSTOP>
__global__ void __launch_bounds__(PipeGeo<M>::THREADS, PipeGeo<M>::MIN_BLOCKS) bp_decode_pipe_kernel(DecodeArgs args)
{
    constexpr int N = Geo<M>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long long cw = blockIdx.x;
    const CwIO a{args.llr + cw * N, args.frozen_words, args.u_hat + cw * N, args.iters ? args.iters + cw : nullptr,
                 args.pe ? args.pe + cw : nullptr, nullptr, nullptr, nullptr, args.bitrev};
    decode_pipe_codeword<M, GSTOP>(a, args.max_iter, args.alpha, args.status, smem_raw);
}

// The per-codeword decode as one out-of-line function, for the persistent kernels:
// at N = 1024 a loop around the inlined body compiles to code 9 % slower than one
// block per codeword (more instructions, more instruction-fetch stalls); called,
// 2 %.  At N = 4096 the inlined loop is the faster of the two (26.8 against 27.3 ms
// per 16,384 codewords at 2.5 dB), so the persistent kernel inlines it there.
template <int M, bool GSTOP>
__device__ __noinline__ void decode_pipe_codeword_call(const CwIO a, int max_iter, float alpha, unsigned int* status,
                                                       unsigned char* smem_raw)
{
    decode_pipe_codeword<M, GSTOP>(a, max_iter, alpha, status, smem_raw);
}

// Persistent form: each block takes the next codeword from the device counter,
// decodes it pipelined and retires it at its own stop, until the queue is empty.
template <int M, bool GSTOP>
__global__ void __launch_bounds__(PipeGeo<M>::THREADS, PipeGeo<M>::MIN_BLOCKS) bp_decode_pipe_persistent(SegArgs a)
{
    constexpr int N = Geo<M>::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<M> sm(smem_raw);
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
        if constexpr (M == 12) decode_pipe_codeword<M, GSTOP>(io, a.max_iter, a.alpha, a.status[sg], smem_raw);
        else decode_pipe_codeword_call<M, GSTOP>(io, a.max_iter, a.alpha, a.status[sg], smem_raw);
    }
}

template <int M, bool GSTOP>
cudaError_t launch_pipe(const DecodeArgs& args, cudaStream_t stream)
{
    auto kern = bp_decode_pipe_kernel<M, GSTOP>;
    constexpr size_t smem = PipeLayout<M>::bytes;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<args.batch, PipeGeo<M>::THREADS, smem, stream>>>(args);
    return cudaGetLastError();
}

// Decode launches of one code length: G-stop + freezing and freezing alone
// (reading A, without message planes) run pipelined for N = 256 .. 4096 unless
// the code asks for the one-block mapping, the rest on bp_decode_kernel.
template <int M>
cudaError_t launch_decode_pipe(const LaunchReq& q)
{
    if constexpr (M >= 8 && M <= 12) {
        if (q.freeze_mode == 1 && !q.trace && q.pipelined)
            return q.stop_mode ? launch_pipe<M, true>(q.args, q.stream) : launch_pipe<M, false>(q.args, q.stream);
    }
    return launch_decode<M>(q);
}

template <int M, bool GSTOP>
cudaError_t launch_pipe_persistent(const SegLaunch& q)
{
    auto kern = bp_decode_pipe_persistent<M, GSTOP>;
    constexpr size_t smem = PipeLayout<M>::bytes;
    constexpr int threads = PipeGeo<M>::THREADS;
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
    if (grid > q.args.total) grid = q.args.total;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, threads, smem, q.stream>>>(q.args);
    return cudaGetLastError();
}

// Persistent launches of one code length: the pipelined mapping for freezing
// (reading A) at N = 256 .. 4096 with one codeword per block, unless the code
// asks for the one-block mapping; otherwise bp_decode_persistent.
template <int M>
cudaError_t launch_persistent_pipe(const SegLaunch& q)
{
    if constexpr (M >= 8 && M <= 12) {
        if (q.freeze_mode == 1 && q.pipelined && q.cpc == 1)
            return q.stop_mode ? launch_pipe_persistent<M, true>(q) : launch_pipe_persistent<M, false>(q);
    }
    return launch_persistent<M>(q);
}

}  // namespace polarbp
