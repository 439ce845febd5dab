// flood.cu -- BP decoding of polar codes under the true flooding schedule.
//
// The paper's decoder (Sec. II-A) activates the PEs stage by stage from left
// to right, so a stage reads R of the current iteration and L of the previous
// one (Eq. (1)).  Under flooding every PE of every stage reads both L and R from
// the previous iteration and all of them update together.  The PE is Eq. (1)'s
// with the same operand order; R[0] is the channel, L[m] the prior (+inf on
// frozen positions, 0 elsewhere) and interior messages start at 0.  Stop: fixed
// iterations or the G-matrix test (u_hat . F^{(x)m} == HD(R[0] + L[0])).  There
// is no CSFG freezing: its order of checks (Sec. III) is defined on the sweep.
//
// One block per codeword, one thread per PE index p (N/2 threads, at least 32).
// In every iteration a thread evaluates PE p of every stage from the planes in
// shared memory, keeps the 4 m outputs in registers, and writes them after a
// barrier; a second barrier ends the iteration.  Planes: L and R, (m+1) x N
// binary32 each, 8 (m+1) N bytes (88 KB at N = 1024, 2 blocks per SM).
#include <cmath>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "polarbp.h"
#include "bp_decode.cuh"

namespace {

struct FloodArgs {
    const float* llr;              // [batch][N]
    const uint32_t* frozen_words;  // ceil(N/32) words
    uint8_t* u_hat;                // [batch][N]
    int32_t* iters;                // [batch] or NULL
    int64_t* pe;                   // [batch] or NULL
    unsigned int* status;
    float* trace_L;                // [batch][max_iter][m+1][N] or NULL
    float* trace_R;
    int max_iter;
    float alpha;
    int gstop;
};

__device__ __forceinline__ bool frozen_at(const uint32_t* w, int i) { return (w[i >> 5] >> (i & 31)) & 1u; }

// G-matrix test on the planes: the source word (0 on frozen positions,
// HD(R[m] + L[m]) elsewhere) re-encoded with F^{(x)m} against HD(R[0] + L[0]).
// Words are built with ballots by all warps, then warp 0 applies the transform
// (in-word butterflies, then across lanes) and compares.
template <int M>
__device__ bool flood_gtest(const float* L, const float* R, const uint32_t* fz, uint32_t* wu, uint32_t* wx, int* flag)
{
    constexpr int N = 1 << M, NW = N < 32 ? 1 : N / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int q = warp; q < NW; q += nwarps) {
        const int i = 32 * q + lane;
        const bool in = i < N;
        const bool ub = in && !frozen_at(fz, i) && __fadd_rn(R[M * N + i], L[M * N + i]) < 0.f;
        const bool xb = in && __fadd_rn(R[i], L[i]) < 0.f;
        const uint32_t bu = __ballot_sync(polarbp::kFull, ub);
        const uint32_t bx = __ballot_sync(polarbp::kFull, xb);
        if (lane == 0) {
            wu[q] = bu;
            wx[q] = bx;
        }
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < NW ? wu[lane] : 0u;
        const uint32_t x = lane < NW ? wx[lane] : 0u;
#pragma unroll
        for (int h = 1; h < 32; h <<= 1) v ^= (v >> h) & polarbp::xmask(h);
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_xor_sync(polarbp::kFull, v, d);
            if (d < NW && !(lane & d)) v ^= y;
        }
        const bool same = __all_sync(polarbp::kFull, lane >= NW || v == x);
        if (lane == 0) *flag = same ? 1 : 0;
    }
    __syncthreads();
    return *flag != 0;
}

template <int M>
__global__ void __launch_bounds__((1 << M) / 2 < 32 ? 32 : (1 << M) / 2) flood_kernel(FloodArgs a)
{
    constexpr int N = 1 << M, H = N / 2;
    extern __shared__ __align__(16) float planes[];
    float* L = planes;            // [(M+1)][N]
    float* R = planes + (M + 1) * N;
    __shared__ uint32_t wu[N < 32 ? 1 : N / 32], wx[N < 32 ? 1 : N / 32];
    __shared__ int flag;
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long cw = blockIdx.x;
    const float* llr = a.llr + cw * N;
    const uint32_t* fz = a.frozen_words;

    bool finite = true;
    for (int i = tid; i < (M + 1) * N; i += nt) {
        const int c = i / N, j = i - c * N;
        float l = 0.f, r = 0.f;
        if (c == M) l = frozen_at(fz, j) ? INFINITY : 0.f;
        if (c == 0) {
            r = llr[j];
            finite &= isfinite(r);
        }
        L[i] = l;
        R[i] = r;
    }
    if (!finite) atomicOr(a.status, 1u);
    __syncthreads();

    // this thread's PE at every stage: pair (ia, ib = ia + 2^(M-1-s))
    const int p = tid;
    const float alpha = a.alpha;
    int it = 1;
    for (; it <= a.max_iter; ++it) {
        float o[M][4];
        if (p < H) {
#pragma unroll
            for (int s = 0; s < M; ++s) {
                const int k = M - 1 - s, h = 1 << k;
                const int ia = ((p >> k) << (k + 1)) | (p & (h - 1)), ib = ia + h;
                const float La = L[(s + 1) * N + ia], Lb = L[(s + 1) * N + ib];
                const float Ra = R[s * N + ia], Rb = R[s * N + ib];
                const float t = __fadd_rn(Lb, Rb);
                const float g = polarbp::fms(La, Ra, alpha);
                o[s][0] = polarbp::fms(La, t, alpha);
                o[s][1] = __fadd_rn(Lb, g);
                o[s][2] = polarbp::fms(Ra, t, alpha);
                o[s][3] = __fadd_rn(Rb, g);
            }
        }
        __syncthreads();
        if (p < H) {
#pragma unroll
            for (int s = 0; s < M; ++s) {
                const int k = M - 1 - s, h = 1 << k;
                const int ia = ((p >> k) << (k + 1)) | (p & (h - 1)), ib = ia + h;
                L[s * N + ia] = o[s][0];
                L[s * N + ib] = o[s][1];
                R[(s + 1) * N + ia] = o[s][2];
                R[(s + 1) * N + ib] = o[s][3];
            }
        }
        __syncthreads();
        if (a.trace_L) {
            const long long base = (cw * a.max_iter + (it - 1)) * (long long)((M + 1) * N);
            for (int i = tid; i < (M + 1) * N; i += nt) {
                a.trace_L[base + i] = L[i];
                a.trace_R[base + i] = R[i];
            }
        }
        if (a.gstop && flood_gtest<M>(L, R, fz, wu, wx, &flag)) break;
    }
    const int iters = it <= a.max_iter ? it : a.max_iter;
    for (int i = tid; i < N; i += nt)
        a.u_hat[cw * N + i] = (!frozen_at(fz, i) && __fadd_rn(R[M * N + i], L[M * N + i]) < 0.f) ? 1 : 0;
    if (tid == 0) {
        if (a.iters) a.iters[cw] = iters;
        if (a.pe) a.pe[cw] = (long long)iters * M * H;
    }
}

template <int M>
cudaError_t launch_flood(const FloodArgs& a, int batch, cudaStream_t s)
{
    constexpr int N = 1 << M;
    const size_t smem = 2 * (size_t)(M + 1) * N * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(flood_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = N / 2 < 32 ? 32 : N / 2;
    flood_kernel<M><<<batch, threads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// host side (declared in include/polarbp.h)
// ---------------------------------------------------------------------------
struct polarbp_code;  // opaque here: the accessors below come from polarbp_api.cu
extern "C" int polarbp_code_info(const polarbp_code* code, int* N, int* K, int* m);
namespace polarbp_internal {
const uint32_t* frozen_words(const polarbp_code* c);
unsigned int* status_word(const polarbp_code* c);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int check_device(const polarbp_code* c);
int bit_reversed(const polarbp_code* c);
}  // namespace polarbp_internal

extern "C" {

int polarbp_decode_flooding(const polarbp_code* code, const float* llr, int batch, int max_iter, float scale,
                            int stop_mode, uint8_t* u_hat, int32_t* iterations, int64_t* pe_updates, float* trace_L,
                            float* trace_R, void* stream)
{
    using namespace polarbp_internal;
    if (!code) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (max_iter < 1) return fail(POLARBP_ERR_ARG, "max_iter must be >= 1");
    if (!(scale > 0.f) || !std::isfinite(scale)) return fail(POLARBP_ERR_ARG, "scale must be finite and > 0");
    if (stop_mode != POLARBP_STOP_NONE && stop_mode != POLARBP_STOP_GMATRIX)
        return fail(POLARBP_ERR_ARG, "unknown stop_mode");
    if ((trace_L == nullptr) != (trace_R == nullptr)) return fail(POLARBP_ERR_ARG, "give both trace planes or neither");
    int m = 0;
    polarbp_code_info(code, nullptr, nullptr, &m);
    if (m > 10) return fail(POLARBP_ERR_UNSUPPORTED, "the flooding schedule supports N <= 1024");
    if (batch == 0) return POLARBP_OK;
    if (!llr || !u_hat) return fail(POLARBP_ERR_ARG, "llr and u_hat must be device pointers");
    if (bit_reversed(code)) return fail(POLARBP_ERR_UNSUPPORTED, "this decoder variant takes codewords in natural order only (see polarbp_set_bit_reversed)");
    int rc = check_device(code);
    if (rc != POLARBP_OK) return rc;
    FloodArgs a;
    a.llr = llr;
    a.frozen_words = frozen_words(code);
    a.u_hat = u_hat;
    a.iters = iterations;
    a.pe = pe_updates;
    a.status = status_word(code);
    a.trace_L = trace_L;
    a.trace_R = trace_R;
    a.max_iter = max_iter;
    a.alpha = scale;
    a.gstop = stop_mode == POLARBP_STOP_GMATRIX;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (m) {
    case 1: e = launch_flood<1>(a, batch, s); break;
    case 2: e = launch_flood<2>(a, batch, s); break;
    case 3: e = launch_flood<3>(a, batch, s); break;
    case 4: e = launch_flood<4>(a, batch, s); break;
    case 5: e = launch_flood<5>(a, batch, s); break;
    case 6: e = launch_flood<6>(a, batch, s); break;
    case 7: e = launch_flood<7>(a, batch, s); break;
    case 8: e = launch_flood<8>(a, batch, s); break;
    case 9: e = launch_flood<9>(a, batch, s); break;
    default: e = launch_flood<10>(a, batch, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "flooding decode launch");
    return POLARBP_OK;
}

}  // extern "C"
