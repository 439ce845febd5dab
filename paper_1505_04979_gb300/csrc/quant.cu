// quant.cu -- BP decoding of polar codes with quantised (16-bit saturating
// integer) messages, a variant for fixed-point hardware, which Sec. V names as
// future work.
//
// Schedule and PE are Eq. (1) as the main decoder reads it: one left-to-right
// sweep per iteration, R of this iteration and L of the previous one.
// Messages are integers in [-QMAX, QMAX], QMAX = 32767:
//   channel   q = clamp(rint(llr * 2^F), -QMAX, QMAX)   (round half to even)
//   sums      clamped to [-QMAX, QMAX]; +-QMAX plays the part of +-inf
//   scaling   alpha = A / 16, f(x, y) = sign(x) sign(y) ((A min(|x|, |y|) + 8) >> 4)
//   prior     L[m] = +QMAX on frozen positions, 0 elsewhere; interior at 0
// Stop (fixed iterations or the G-matrix test), output and PE count are those
// of the main decoder without freezing.  Every value is an exact integer.
//
// One block per codeword, one thread per PE index (N/2 threads, at least 32),
// the L and R planes in shared memory as int16 (4 (m+1) N bytes, half the
// bytes of binary32 planes), one barrier after each stage.
#include <cmath>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "polarbp.h"
#include "bp_decode.cuh"

namespace {

constexpr int QMAX = 32767;

struct QArgs {
    const float* llr;              // [batch][N]
    const uint32_t* frozen_words;  // ceil(N/32) words
    uint8_t* u_hat;                // [batch][N]
    int32_t* iters;                // [batch] or NULL
    int64_t* pe;                   // [batch] or NULL
    unsigned int* status;
    int16_t* trace_L;              // [batch][max_iter][m+1][N] or NULL
    int16_t* trace_R;
    int max_iter;
    int A;                         // alpha = A / 16
    int F;                         // fractional bits of the channel values
    int gstop;
};

__device__ __forceinline__ bool qfrozen(const uint32_t* w, int i) { return (w[i >> 5] >> (i & 31)) & 1u; }
__device__ __forceinline__ int qsat(int v) { return min(max(v, -QMAX), QMAX); }
__device__ __forceinline__ int qf(int A, int x, int y)
{
    const int mag = (A * min(abs(x), abs(y)) + 8) >> 4;
    return ((x < 0) != (y < 0)) ? -mag : mag;
}

// G-matrix test on the integer planes: the source word (0 on frozen positions,
// HD(R[m] + L[m]) elsewhere) re-encoded with F^{(x)m} against HD(R[0] + L[0]).
// Clamping a sum keeps its sign, so the decisions use the plain sums.
template <int M>
__device__ bool qgtest(const int16_t* L, const int16_t* R, const uint32_t* fz, uint32_t* wu, uint32_t* wx, int* flag)
{
    constexpr int N = 1 << M, NW = N < 32 ? 1 : N / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int q = warp; q < NW; q += nwarps) {
        const int i = 32 * q + lane;
        const bool in = i < N;
        const bool ub = in && !qfrozen(fz, i) && (int)R[M * N + i] + (int)L[M * N + i] < 0;
        const bool xb = in && (int)R[i] + (int)L[i] < 0;
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
__global__ void __launch_bounds__((1 << M) / 2 < 32 ? 32 : (1 << M) / 2) qsweep_kernel(QArgs a)
{
    constexpr int N = 1 << M, H = N / 2;
    extern __shared__ __align__(16) int16_t qplanes[];
    int16_t* L = qplanes;  // [(M+1)][N]
    int16_t* R = qplanes + (M + 1) * N;
    __shared__ uint32_t wu[N < 32 ? 1 : N / 32], wx[N < 32 ? 1 : N / 32];
    __shared__ int flag;
    const int tid = threadIdx.x, nt = blockDim.x;
    const long long cw = blockIdx.x;
    const float* llr = a.llr + cw * N;
    const uint32_t* fz = a.frozen_words;
    const float scale = (float)(1 << a.F);

    bool finite = true;
    for (int i = tid; i < (M + 1) * N; i += nt) {
        const int c = i / N, j = i - c * N;
        int l = 0, r = 0;
        if (c == M) l = qfrozen(fz, j) ? QMAX : 0;
        if (c == 0) {
            const float v = llr[j];
            finite &= isfinite(v);
            r = qsat(__float2int_rn(v * scale));  // saturating conversion, round half to even
        }
        L[i] = (int16_t)l;
        R[i] = (int16_t)r;
    }
    if (!finite) atomicOr(a.status, 1u);
    __syncthreads();

    const int p = tid;
    const int A = a.A;
    int it = 1;
    for (; it <= a.max_iter; ++it) {
#pragma unroll
        for (int s = 0; s < M; ++s) {
            if (p < H) {
                const int k = M - 1 - s, h = 1 << k;
                const int ia = ((p >> k) << (k + 1)) | (p & (h - 1)), ib = ia + h;
                const int La = L[(s + 1) * N + ia], Lb = L[(s + 1) * N + ib];
                const int Ra = R[s * N + ia], Rb = R[s * N + ib];
                const int t = qsat(Lb + Rb);
                const int g = qf(A, La, Ra);
                L[s * N + ia] = (int16_t)qf(A, La, t);
                L[s * N + ib] = (int16_t)qsat(Lb + g);
                R[(s + 1) * N + ia] = (int16_t)qf(A, Ra, t);
                R[(s + 1) * N + ib] = (int16_t)qsat(Rb + g);
            }
            __syncthreads();
        }
        if (a.trace_L) {
            const long long base = (cw * a.max_iter + (it - 1)) * (long long)((M + 1) * N);
            for (int i = tid; i < (M + 1) * N; i += nt) {
                a.trace_L[base + i] = L[i];
                a.trace_R[base + i] = R[i];
            }
        }
        if (a.gstop && qgtest<M>(L, R, fz, wu, wx, &flag)) break;
    }
    const int iters = it <= a.max_iter ? it : a.max_iter;
    for (int i = tid; i < N; i += nt)
        a.u_hat[cw * N + i] = (!qfrozen(fz, i) && (int)R[M * N + i] + (int)L[M * N + i] < 0) ? 1 : 0;
    if (tid == 0) {
        if (a.iters) a.iters[cw] = iters;
        if (a.pe) a.pe[cw] = (long long)iters * M * H;
    }
}

template <int M>
cudaError_t launch_q(const QArgs& a, int batch, cudaStream_t s)
{
    constexpr int N = 1 << M;
    const size_t smem = 2 * (size_t)(M + 1) * N * sizeof(int16_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(qsweep_kernel<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = N / 2 < 32 ? 32 : N / 2;
    qsweep_kernel<M><<<batch, threads, smem, s>>>(a);
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

int polarbp_decode_quantized(const polarbp_code* code, const float* llr, int batch, int max_iter, int alpha_16,
                             int frac_bits, int stop_mode, uint8_t* u_hat, int32_t* iterations,
                             int64_t* pe_updates, int16_t* trace_L, int16_t* trace_R, void* stream)
{
    using namespace polarbp_internal;
    if (!code) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (max_iter < 1) return fail(POLARBP_ERR_ARG, "max_iter must be >= 1");
    if (alpha_16 < 1 || alpha_16 > 16) return fail(POLARBP_ERR_ARG, "alpha_16 must be in 1..16");
    if (frac_bits < 0 || frac_bits > 8) return fail(POLARBP_ERR_ARG, "frac_bits must be in 0..8");
    if (stop_mode != POLARBP_STOP_NONE && stop_mode != POLARBP_STOP_GMATRIX)
        return fail(POLARBP_ERR_ARG, "unknown stop_mode");
    if ((trace_L == nullptr) != (trace_R == nullptr)) return fail(POLARBP_ERR_ARG, "give both trace planes or neither");
    int m = 0;
    polarbp_code_info(code, nullptr, nullptr, &m);
    if (m > 10) return fail(POLARBP_ERR_UNSUPPORTED, "quantised messages support N <= 1024");
    if (batch == 0) return POLARBP_OK;
    if (!llr || !u_hat) return fail(POLARBP_ERR_ARG, "llr and u_hat must be device pointers");
    if (bit_reversed(code)) return fail(POLARBP_ERR_UNSUPPORTED, "this decoder variant takes codewords in natural order only (see polarbp_set_bit_reversed)");
    int rc = check_device(code);
    if (rc != POLARBP_OK) return rc;
    QArgs a;
    a.llr = llr;
    a.frozen_words = frozen_words(code);
    a.u_hat = u_hat;
    a.iters = iterations;
    a.pe = pe_updates;
    a.status = status_word(code);
    a.trace_L = trace_L;
    a.trace_R = trace_R;
    a.max_iter = max_iter;
    a.A = alpha_16;
    a.F = frac_bits;
    a.gstop = stop_mode == POLARBP_STOP_GMATRIX;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (m) {
    case 1: e = launch_q<1>(a, batch, s); break;
    case 2: e = launch_q<2>(a, batch, s); break;
    case 3: e = launch_q<3>(a, batch, s); break;
    case 4: e = launch_q<4>(a, batch, s); break;
    case 5: e = launch_q<5>(a, batch, s); break;
    case 6: e = launch_q<6>(a, batch, s); break;
    case 7: e = launch_q<7>(a, batch, s); break;
    case 8: e = launch_q<8>(a, batch, s); break;
    case 9: e = launch_q<9>(a, batch, s); break;
    default: e = launch_q<10>(a, batch, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "quantised decode launch");
    return POLARBP_OK;
}

}  // extern "C"
