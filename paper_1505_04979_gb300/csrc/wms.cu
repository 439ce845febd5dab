// wms.cu -- weighted min-sum BP forward / adjoint for learning per-PE scalings.
//
// The decoder is Eq. (1) (Sec. II-A) with the min-sum scaling alpha replaced by
// one weight per (iteration t, stage s, PE p), T unrolled iterations, no stop
// and no freezing.  PE p of stage s pairs a and a + h (h = 2^(m-1-s)) with
// p = (a >> (m-s)) h + (a mod h); weight (t, s, p) sits at
// w[(t m + s) N/2 + p].  The soft output of position i is R[m][i] + L[m][i]
// after the last iteration (+inf on frozen positions, the prior).
//
// Gradient of f_w(x, y) = w h(x, y), h = sign(x) sign(y) min(|x|, |y|):
// df/dw = h; when |x| <= |y| (ties to the first argument) df/dx = w sign(y),
// df/dy = 0, else df/dx = 0, df/dy = w sign(x).  Messages that are +-inf
// (built from the frozen prior) do not change with any weight or input: no
// adjoint flows into or out of them and they add nothing to a weight's
// gradient.
//
// One block of N/2 threads (at least 32) per codeword, one PE per thread per
// stage, all message planes in shared memory; the forward checkpoints L and R
// after every iteration to the caller's workspace, the adjoint reads them back
// in reverse order and writes one gradient partial per codeword, which two
// more kernels sum over the batch in a fixed order (chunks of codewords, then
// the chunks).
#include <cmath>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "polarbp.h"

namespace {

struct WmsShape {
    int N, m, T;
    size_t plane;  // (m+1) N
};

__device__ __forceinline__ float wsgn(float v) { return (float)((v > 0.f) - (v < 0.f)); }

// w * sign(x) sign(y) min(|x|, |y|): exact magnitude, one rounding for the product
__device__ __forceinline__ float wmin(float w, float x, float y)
{
    const float mag = __fmul_rn(w, fminf(fabsf(x), fabsf(y)));
    const uint32_t s = (__float_as_uint(x) ^ __float_as_uint(y)) & 0x80000000u;
    return __uint_as_float(__float_as_uint(mag) | s);
}

__device__ __forceinline__ float hval(float x, float y)
{
    return wsgn(x) * wsgn(y) * fminf(fabsf(x), fabsf(y));
}

__device__ __forceinline__ int pair_a(int m, int s, int p)
{
    const int h = 1 << (m - 1 - s);
    return (p / h) * 2 * h + (p % h);
}

// checkpoints: [batch][T][2][(m+1)][N]: L after iteration t, then R after iteration t
__global__ void wms_forward_kernel(const float* __restrict__ llr, const uint32_t* __restrict__ frozen_words,
                                   const float* __restrict__ w, int N, int m, int T, float* __restrict__ out,
                                   float* __restrict__ ckpt)
{
    extern __shared__ __align__(16) float sh[];
    float* L = sh;                        // (m+1) N
    float* R = sh + (size_t)(m + 1) * N;  // (m+1) N
    const long long cw = blockIdx.x;
    const int plane = (m + 1) * N;
    for (int k = threadIdx.x; k < plane; k += blockDim.x) {
        const int c = k / N, i = k % N;
        L[k] = (c == m) ? (((frozen_words[i >> 5] >> (i & 31)) & 1u) ? INFINITY : 0.f) : 0.f;
        R[k] = 0.f;
    }
    __syncthreads();
    const int p = threadIdx.x;
    for (int t = 0; t < T; ++t) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) R[i] = llr[cw * N + i];
        __syncthreads();
        for (int s = 0; s < m; ++s) {
            if (p < N / 2) {
                const int h = 1 << (m - 1 - s);
                const int a = pair_a(m, s, p), b = a + h;
                const float wt = __ldg(w + ((size_t)t * m + s) * (N / 2) + p);
                const float La = L[(s + 1) * N + a], Lb = L[(s + 1) * N + b];
                const float Ra = R[s * N + a], Rb = R[s * N + b];
                const float tt = __fadd_rn(Lb, Rb);
                const float g = wmin(wt, La, Ra);
                L[s * N + a] = wmin(wt, La, tt);
                L[s * N + b] = __fadd_rn(Lb, g);
                R[(s + 1) * N + a] = wmin(wt, Ra, tt);
                R[(s + 1) * N + b] = __fadd_rn(Rb, g);
            }
            __syncthreads();
        }
        // checkpoint: both planes with 16-byte stores ((m+1) N is a multiple of 4)
        float4* dst = reinterpret_cast<float4*>(ckpt + ((size_t)cw * T + t) * 2 * plane);
        const float4* L4 = reinterpret_cast<const float4*>(L);
        const float4* R4 = reinterpret_cast<const float4*>(R);
        for (int k = threadIdx.x; k < plane / 4; k += blockDim.x) {
            dst[k] = L4[k];
            dst[plane / 4 + k] = R4[k];
        }
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) out[cw * N + i] = __fadd_rn(R[m * N + i], L[m * N + i]);
}

// Every product and sum of the adjoint is rounded on its own (no fused
// multiply-add): the adjoint is binary32 arithmetic operation by operation, in
// the chain-rule order written below.
__device__ __forceinline__ void acc(float* slot, float value, float g)
{
    if (!isinf(value)) *slot = __fadd_rn(*slot, g);
}

// partials: [batch][T m N/2]
__global__ void wms_backward_kernel(const float* __restrict__ llr, const uint32_t* __restrict__ frozen_words,
                                    const float* __restrict__ w, int N, int m, int T, const float* __restrict__ ckpt,
                                    const float* __restrict__ dout, float* __restrict__ partial,
                                    float* __restrict__ dllr)
{
    extern __shared__ float sh[];
    const int plane = (m + 1) * N;
    float* dL = sh;            // adjoint of the L state after the current iteration
    float* dLp = sh + plane;   // adjoint of the L state before it
    float* dR = sh + 2 * plane;
    const long long cw = blockIdx.x;
    for (int k = threadIdx.x; k < plane; k += blockDim.x) {
        dL[k] = 0.f;
    }
    float dl_acc[4] = {0.f, 0.f, 0.f, 0.f};  // dllr of positions threadIdx.x + j blockDim.x (N <= 4 blockDim.x)
    __syncthreads();
    const int p = threadIdx.x;
    const size_t W = (size_t)T * m * (N / 2);
    for (int t = T - 1; t >= 0; --t) {
        const float* Rc = ckpt + ((size_t)cw * T + t) * 2 * plane + plane;                   // R^t
        // L^{t-1}; before iteration 1 it is the prior (+inf on frozen positions of column m, else 0)
        const float* Lp = t > 0 ? ckpt + ((size_t)cw * T + (t - 1)) * 2 * plane : nullptr;
        for (int k = threadIdx.x; k < plane; k += blockDim.x) {
            dR[k] = 0.f;
            dLp[k] = 0.f;
        }
        __syncthreads();
        if (t == T - 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) acc(&dR[m * N + i], Rc[m * N + i], dout[cw * N + i]);
        }
        __syncthreads();
        for (int s = m - 1; s >= 0; --s) {
            if (p < N / 2) {
                const int h = 1 << (m - 1 - s);
                const int a = pair_a(m, s, p), b = a + h;
                const size_t widx = ((size_t)t * m + s) * (N / 2) + p;
                const float wt = __ldg(w + widx);
                float La = 0.f, Lb = 0.f;
                if (Lp) {
                    La = Lp[(s + 1) * N + a];
                    Lb = Lp[(s + 1) * N + b];
                } else if (s + 1 == m) {
                    La = ((frozen_words[a >> 5] >> (a & 31)) & 1u) ? INFINITY : 0.f;
                    Lb = ((frozen_words[b >> 5] >> (b & 31)) & 1u) ? INFINITY : 0.f;
                }
                const float Ra = Rc[s * N + a], Rb = Rc[s * N + b];
                const float tt = __fadd_rn(Lb, Rb);
                const float g = wmin(wt, La, Ra);
                // the stage's forward outputs, recomputed from its inputs exactly as the
                // forward formed them (only their infinities matter here)
                const float oLa = wmin(wt, La, tt), oLb = __fadd_rn(Lb, g);
                const float oRa = wmin(wt, Ra, tt), oRb = __fadd_rn(Rb, g);
                const float gLa = (s >= 1 && !isinf(oLa)) ? dL[s * N + a] : 0.f;
                const float gLb = (s >= 1 && !isinf(oLb)) ? dL[s * N + b] : 0.f;
                const float gRa = isinf(oRa) ? 0.f : dR[(s + 1) * N + a];
                const float gRb = isinf(oRb) ? 0.f : dR[(s + 1) * N + b];
                float dg = 0.f, dt = 0.f, dw = 0.f;
                acc(&dR[s * N + b], Rb, gRb);
                if (!isinf(g)) dg = __fadd_rn(dg, gRb);
                acc(&dLp[(s + 1) * N + b], Lb, gLb);
                if (!isinf(oLb)) dg = __fadd_rn(dg, gLb);
                if (!isinf(oRa) && gRa != 0.f) {
                    if (fabsf(Ra) <= fabsf(tt)) acc(&dR[s * N + a], Ra, __fmul_rn(__fmul_rn(gRa, wt), wsgn(tt)));
                    else if (!isinf(tt)) dt = __fadd_rn(dt, __fmul_rn(__fmul_rn(gRa, wt), wsgn(Ra)));
                    dw = __fadd_rn(dw, __fmul_rn(gRa, hval(Ra, tt)));
                }
                if (!isinf(oLa) && gLa != 0.f) {
                    if (fabsf(La) <= fabsf(tt)) acc(&dLp[(s + 1) * N + a], La, __fmul_rn(__fmul_rn(gLa, wt), wsgn(tt)));
                    else if (!isinf(tt)) dt = __fadd_rn(dt, __fmul_rn(__fmul_rn(gLa, wt), wsgn(La)));
                    dw = __fadd_rn(dw, __fmul_rn(gLa, hval(La, tt)));
                }
                if (!isinf(g) && dg != 0.f) {
                    if (fabsf(La) <= fabsf(Ra)) acc(&dLp[(s + 1) * N + a], La, __fmul_rn(__fmul_rn(dg, wt), wsgn(Ra)));
                    else acc(&dR[s * N + a], Ra, __fmul_rn(__fmul_rn(dg, wt), wsgn(La)));
                    dw = __fadd_rn(dw, __fmul_rn(dg, hval(La, Ra)));
                }
                if (!isinf(tt)) {
                    acc(&dLp[(s + 1) * N + b], Lb, dt);
                    acc(&dR[s * N + b], Rb, dt);
                }
                partial[(size_t)cw * W + widx] = dw;
            }
            __syncthreads();
        }
        for (int j = 0; j < 4; ++j) {
            const int i = threadIdx.x + j * blockDim.x;
            if (i < N) dl_acc[j] = __fadd_rn(dl_acc[j], dR[i]);
        }
        __syncthreads();
        float* tmp = dL;
        dL = dLp;
        dLp = tmp;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            dL[m * N + i] = 0.f;
            dL[i] = 0.f;
        }
        __syncthreads();
    }
    for (int j = 0; j < 4; ++j) {
        const int i = threadIdx.x + j * blockDim.x;
        if (i < N) dllr[cw * N + i] = dl_acc[j];
    }
}

// Deterministic batch sum of the per-codeword gradient partials, in two fixed
// passes: chunk[q][k] = sum of partial[c][k] over the kReduceChunk codewords of
// chunk q in codeword order (grid: weight tiles x chunks), then dw[k] = sum of
// chunk[q][k] in chunk order.
constexpr int kReduceChunk = 64;

__global__ void wms_reduce_chunks_kernel(const float* __restrict__ partial, int batch, size_t W,
                                         float* __restrict__ chunk)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (k >= W) return;
    const int c0 = q * kReduceChunk, c1 = min(batch, c0 + kReduceChunk);
    float acc_v = 0.f;
#pragma unroll 8
    for (int c = c0; c < c1; ++c) acc_v = __fadd_rn(acc_v, partial[(size_t)c * W + k]);
    chunk[(size_t)q * W + k] = acc_v;
}

__global__ void wms_reduce_kernel(const float* __restrict__ chunk, int nchunks, size_t W, float* __restrict__ dw)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= W) return;
    float acc_v = 0.f;
    for (int q = 0; q < nchunks; ++q) acc_v = __fadd_rn(acc_v, chunk[(size_t)q * W + k]);
    dw[k] = acc_v;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// ---------------------------------------------------------------------------
// host side (declared in include/polarbp.h)
// ---------------------------------------------------------------------------
struct polarbp_code;  // opaque here: the accessors below come from polarbp_api.cu
extern "C" int polarbp_code_info(const polarbp_code* code, int* N, int* K, int* m);
namespace polarbp_internal {
const uint32_t* frozen_words(const polarbp_code* c);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
int check_device(const polarbp_code* c);
int bit_reversed(const polarbp_code* c);
}  // namespace polarbp_internal

namespace {
struct WmsLayout {
    size_t ckpt, partial, chunk, total;
};
WmsLayout wms_layout(int N, int m, int batch, int T)
{
    WmsLayout l;
    const size_t W = (size_t)T * m * (N / 2);
    const size_t nchunks = ((size_t)batch + kReduceChunk - 1) / kReduceChunk;
    l.ckpt = 0;
    l.partial = align256((size_t)batch * T * 2 * (m + 1) * N * sizeof(float));
    l.chunk = align256(l.partial + (size_t)batch * W * sizeof(float));
    l.total = align256(l.chunk + nchunks * W * sizeof(float));
    return l;
}

int wms_args(const polarbp_code* c, int batch, int T, int* N, int* m)
{
    using namespace polarbp_internal;
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (T < 1) return fail(POLARBP_ERR_ARG, "iterations must be >= 1");
    polarbp_code_info(c, N, nullptr, m);
    if (*m > 10) return fail(POLARBP_ERR_UNSUPPORTED, "weighted min-sum supports N <= 1024");
    if (bit_reversed(c)) return fail(POLARBP_ERR_UNSUPPORTED, "this decoder variant takes codewords in natural order only (see polarbp_set_bit_reversed)");
    return POLARBP_OK;
}
}  // namespace

extern "C" {

size_t polarbp_wms_workspace(const polarbp_code* code, int batch, int iterations)
{
    int N = 0, m = 0;
    if (!code || batch < 0 || iterations < 1) return 0;
    polarbp_code_info(code, &N, nullptr, &m);
    return wms_layout(N, m, batch, iterations).total;
}

int polarbp_wms_forward(const polarbp_code* code, const float* llr, int batch, int iterations, const float* weights,
                        float* out, void* workspace, size_t workspace_bytes, void* stream)
{
    using namespace polarbp_internal;
    int N = 0, m = 0;
    int rc = wms_args(code, batch, iterations, &N, &m);
    if (rc != POLARBP_OK) return rc;
    if (batch == 0) return POLARBP_OK;
    if (!llr || !weights || !out) return fail(POLARBP_ERR_ARG, "llr, weights and out must be device pointers");
    const WmsLayout l = wms_layout(N, m, batch, iterations);
    if (!workspace || workspace_bytes < l.total) return fail(POLARBP_ERR_ARG, "workspace too small");
    rc = check_device(code);
    if (rc != POLARBP_OK) return rc;
    const int threads = N / 2 < 32 ? 32 : N / 2;
    const size_t smem = 2 * (size_t)(m + 1) * N * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(wms_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "wms forward attribute");
    }
    float* ckpt = reinterpret_cast<float*>(static_cast<char*>(workspace) + l.ckpt);
    wms_forward_kernel<<<batch, threads, smem, static_cast<cudaStream_t>(stream)>>>(
        llr, frozen_words(code), weights, N, m, iterations, out, ckpt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wms forward launch");
    return POLARBP_OK;
}

int polarbp_wms_backward(const polarbp_code* code, const float* llr, int batch, int iterations, const float* weights,
                         const float* dout, float* dweights, float* dllr, void* workspace, size_t workspace_bytes,
                         void* stream)
{
    using namespace polarbp_internal;
    int N = 0, m = 0;
    int rc = wms_args(code, batch, iterations, &N, &m);
    if (rc != POLARBP_OK) return rc;
    if (!weights || !dweights) return fail(POLARBP_ERR_ARG, "weights and dweights must be device pointers");
    const size_t W = (size_t)iterations * m * (N / 2);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (batch == 0) {
        cudaError_t e = cudaMemsetAsync(dweights, 0, W * sizeof(float), s);
        return e == cudaSuccess ? POLARBP_OK : cuda_fail(e, "wms backward");
    }
    if (!llr || !dout || !dllr) return fail(POLARBP_ERR_ARG, "llr, dout and dllr must be device pointers");
    const WmsLayout l = wms_layout(N, m, batch, iterations);
    if (!workspace || workspace_bytes < l.total) return fail(POLARBP_ERR_ARG, "workspace too small");
    rc = check_device(code);
    if (rc != POLARBP_OK) return rc;
    const int threads = N / 2 < 32 ? 32 : N / 2;
    const size_t smem = 3 * (size_t)(m + 1) * N * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(wms_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "wms backward attribute");
    }
    const float* ckpt = reinterpret_cast<const float*>(static_cast<const char*>(workspace) + l.ckpt);
    float* partial = reinterpret_cast<float*>(static_cast<char*>(workspace) + l.partial);
    wms_backward_kernel<<<batch, threads, smem, s>>>(llr, frozen_words(code), weights, N, m, iterations, ckpt, dout,
                                                     partial, dllr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wms backward launch");
    float* chunk = reinterpret_cast<float*>(static_cast<char*>(workspace) + l.chunk);
    const int nchunks = (batch + kReduceChunk - 1) / kReduceChunk;
    wms_reduce_chunks_kernel<<<dim3((unsigned)((W + 255) / 256), (unsigned)nchunks), 256, 0, s>>>(partial, batch, W,
                                                                                                  chunk);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wms reduce launch");
    wms_reduce_kernel<<<(unsigned)((W + 255) / 256), 256, 0, s>>>(chunk, nchunks, W, dweights);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wms reduce launch");
    return POLARBP_OK;
}

}  // extern "C"
