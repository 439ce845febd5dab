// Compile-time checks of the decoders' shared-memory layouts, built by
// tests/test_layouts_cpu.py with and without -DPOLARBP_CHECKED (nothing runs).
//
// Both builds: regions are in increasing order, every redzone (kRedzone bytes
// at zone(k)) ends before the next region starts, the vector-loaded regions
// keep their alignment, and every layout fits one block's shared memory.
// Default build only: the redzones are empty and the byte counts are the
// dynamic shared memory the ncu captures report for these kernels
// (36,448 B for the pipelined N = 1024 kernel, 215,008 B for the N = 32768
// cluster kernel).
#include "bp_decode.cuh"
#include "bp_pipe.cuh"
#include "bp_cluster.cuh"
#include "bp_mixed.cuh"

using namespace polarbp;

template <int M>
constexpr bool block_layout_ok()
{
    using L = SmemLayout<M>;
    constexpr size_t next[L::ZONES] = {L::off_Lb, L::off_Rx, L::off_Llr, L::off_U,  L::off_Fz, L::off_Xf,
                                       L::off_Ctl, L::off_Hd, L::off_Ge, L::off_Lm, L::bytes};
    for (int k = 0; k < L::ZONES; ++k) {
        if (L::zone(k) + kRedzone > next[k]) return false;
        if (L::zone(k) % 4 != 0) return false;
        if (k > 0 && next[k] < next[k - 1]) return false;
    }
    return L::off_Llr % 16 == 0 && L::off_Ctl % 16 == 0 && L::off_Hd % 16 == 0 && L::off_Ge % 16 == 0 &&
           L::off_Lm % 32 == 0 && L::bytes % 16 == 0 && L::bytes <= 227 * 1024;
}

template <int M>
constexpr bool pipe_layout_ok()
{
    using P = PipeLayout<M>;
    return SmemLayout<M>::bytes <= P::off_hd1 && P::off_hd1 % 32 == 0 && P::end_hd1 + kRedzone <= P::off_ge1 &&
           P::off_ge1 % 16 == 0 && P::end_ge1 + kRedzone <= P::bytes && P::bytes <= 227 * 1024;
}

template <int XC>
constexpr bool cluster_layout_ok()
{
    using L = CLayout<XC>;
    constexpr size_t next[L::ZONES] = {L::off_LlrP, L::off_Xw, L::off_V,  L::off_Uc, L::off_XfX,
                                       L::off_Wg,   L::off_UE, L::off_Fb, L::off_Cc, L::bytes};
    if (L::off_Lx != SmemLayout<12>::bytes) return false;
    for (int k = 0; k < L::ZONES; ++k)
        if (L::zone(k) + kRedzone > next[k] || L::zone(k) % 4 != 0) return false;
    return L::bytes <= 227 * 1024;
}

static_assert(block_layout_ok<1>() && block_layout_ok<2>() && block_layout_ok<3>() && block_layout_ok<4>() &&
                  block_layout_ok<5>() && block_layout_ok<6>() && block_layout_ok<7>() && block_layout_ok<8>() &&
                  block_layout_ok<9>() && block_layout_ok<10>() && block_layout_ok<11>() && block_layout_ok<12>(),
              "one-block layouts");
static_assert(pipe_layout_ok<8>() && pipe_layout_ok<9>() && pipe_layout_ok<10>() && pipe_layout_ok<11>() &&
                  pipe_layout_ok<12>(),
              "pipelined layouts");
static_assert(cluster_layout_ok<1>() && cluster_layout_ok<2>() && cluster_layout_ok<3>(), "cluster layouts");
static_assert(MixedTop<12, true>::SMEM <= 227 * 1024 && MixedTop<12, false>::SMEM <= 227 * 1024, "mixed kernel");

#ifndef POLARBP_CHECKED
static_assert(kRedzone == 0 && !kChecked, "the default build has no redzones");
static_assert(SmemLayout<10>::bytes == 34784, "N = 1024 one-block layout");
static_assert(PipeLayout<10>::bytes == 36448, "N = 1024 pipelined layout (ncu: 36.448 KB dynamic shared memory)");
static_assert(PipeLayout<12>::bytes == 148192, "N = 4096 pipelined layout");
static_assert(CLayout<3>::bytes == 215008, "N = 32768 cluster layout (ncu: 215.008 KB dynamic shared memory)");
#else
static_assert(kRedzone == 256 && kChecked, "the checked build's redzones");
#endif
