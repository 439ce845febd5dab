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
// stage, all message planes in shared memory.  Checkpoint interval k = 1: the
// forward stores both planes after every iteration and the adjoint reads them
// back.  k > 1: the forward stores only the state one iteration hands to the
// next, L columns 1..m-1 (R is rebuilt from the channel LLRs every iteration,
// L[m] is the prior, L[0] is read by nothing), after iterations k-1, 2k-1, ...;
// the adjoint runs the segments [jk, jk+k) last to first, reloads the
// checkpoint before the segment, recomputes the segment's L states in shared
// memory with the forward's own arithmetic and rebuilds each iteration's R plane
// from its L state when that iteration's adjoint runs.  Every recomputed message
// equals the forward's bit for bit, so the gradients do not depend on k; k
// trades workspace (and HBM traffic) for recomputation.  The adjoint writes one
// gradient partial per codeword, which two more kernels sum over the batch in
// a fixed order (chunks of codewords, then the chunks).
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

// One forward iteration t on the planes L (in place) and R, Eq. (1) with weight (t, s, p).
__device__ __forceinline__ void wms_iteration(float* L, float* R, const float* __restrict__ llr_cw,
                                              const float* __restrict__ w, int N, int m, int t)
{
    const int p = threadIdx.x;
    for (int i = threadIdx.x; i < N; i += blockDim.x) R[i] = llr_cw[i];
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
}

// The R plane of iteration t from the L state before it (Lp, read only): the R
// half of wms_iteration, the same operations in the same order.
__device__ __forceinline__ void wms_rebuild_R(const float* Lp, float* R, const float* __restrict__ llr_cw,
                                              const float* __restrict__ w, int N, int m, int t)
{
    const int p = threadIdx.x;
    for (int i = threadIdx.x; i < N; i += blockDim.x) R[i] = llr_cw[i];
    __syncthreads();
    for (int s = 0; s < m; ++s) {
        if (p < N / 2) {
            const int h = 1 << (m - 1 - s);
            const int a = pair_a(m, s, p), b = a + h;
            const float wt = __ldg(w + ((size_t)t * m + s) * (N / 2) + p);
            const float La = Lp[(s + 1) * N + a], Lb = Lp[(s + 1) * N + b];
            const float Ra = R[s * N + a], Rb = R[s * N + b];
            const float tt = __fadd_rn(Lb, Rb);
            const float g = wmin(wt, La, Ra);
            R[(s + 1) * N + a] = wmin(wt, Ra, tt);
            R[(s + 1) * N + b] = __fadd_rn(Rb, g);
        }
        __syncthreads();
    }
}

// The L state before iteration 0: the prior on column m (+inf frozen, 0 else), 0 elsewhere.
__device__ __forceinline__ void wms_initial_L(float* L, const uint32_t* __restrict__ frozen_words, int N, int m)
{
    const int plane = (m + 1) * N;
    for (int k = threadIdx.x; k < plane; k += blockDim.x) {
        const int c = k / N, i = k % N;
        L[k] = (c == m) ? (((frozen_words[i >> 5] >> (i & 31)) & 1u) ? INFINITY : 0.f) : 0.f;
    }
}

// Checkpoints.  k = 1: [batch][T][2][(m+1) N], the L and R planes after iteration t.
// k > 1: [batch][(T-1)/k][(m-1) N], checkpoint j = L columns 1..m-1 after iteration (j+1) k - 1.
__global__ void wms_forward_kernel(const float* __restrict__ llr, const uint32_t* __restrict__ frozen_words,
                                   const float* __restrict__ w, int N, int m, int T, int k, float* __restrict__ out,
                                   float* __restrict__ ckpt)
{
    extern __shared__ __align__(16) float sh[];
    float* L = sh;                        // (m+1) N
    float* R = sh + (size_t)(m + 1) * N;  // (m+1) N
    const long long cw = blockIdx.x;
    const int NC = (T - 1) / k;           // checkpoints per codeword
    const int cols = (m - 1) * N;         // L columns 1..m-1
    wms_initial_L(L, frozen_words, N, m);
    __syncthreads();
    const int plane = (m + 1) * N;
    for (int t = 0; t < T; ++t) {
        wms_iteration(L, R, llr + cw * N, w, N, m, t);
        if (k == 1) {  // both planes with 16-byte stores ((m+1) N is a multiple of 4)
            float4* dst = reinterpret_cast<float4*>(ckpt + ((size_t)cw * T + t) * 2 * plane);
            const float4* L4 = reinterpret_cast<const float4*>(L);
            const float4* R4 = reinterpret_cast<const float4*>(R);
            for (int q = threadIdx.x; q < plane / 4; q += blockDim.x) {
                dst[q] = L4[q];
                dst[plane / 4 + q] = R4[q];
            }
        } else if ((t + 1) % k == 0 && t + 1 < T) {
            float* dst = ckpt + ((size_t)cw * NC + (t + 1) / k - 1) * cols;
            if ((cols & 3) == 0) {  // 16-byte stores (N >= 4)
                float4* d4 = reinterpret_cast<float4*>(dst);
                const float4* s4 = reinterpret_cast<const float4*>(L + N);
                for (int q = threadIdx.x; q < cols / 4; q += blockDim.x) d4[q] = s4[q];
            } else {
                for (int q = threadIdx.x; q < cols; q += blockDim.x) dst[q] = L[N + q];
            }
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

// The adjoint of iteration t (its stages last to first), given the L state before
// it (Lp; NULL for t = 0: the prior) and its R plane (Rc).  dL holds the adjoint
// of the L state after iteration t and becomes that of the state before it.
// partials: [batch][T m N/2].
__device__ __forceinline__ void wms_backward_iteration(const float* Lp, const float* Rc, float*& dL, float*& dLp,
                                                       float* dR, const uint32_t* __restrict__ frozen_words,
                                                       const float* __restrict__ w, int N, int m, int T, int t,
                                                       const float* __restrict__ dout_cw, float* __restrict__ partial_cw,
                                                       float (&dl_acc)[4])
{
    const int plane = (m + 1) * N;
    const int p = threadIdx.x;
    for (int q = threadIdx.x; q < plane; q += blockDim.x) {
        dR[q] = 0.f;
        dLp[q] = 0.f;
    }
    __syncthreads();
    if (t == T - 1) {
        for (int i = threadIdx.x; i < N; i += blockDim.x) acc(&dR[m * N + i], Rc[m * N + i], dout_cw[i]);
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
            partial_cw[widx] = dw;
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

// k = 1: the L and R planes of every iteration come from the checkpoints.
// Shared memory: dL, dLp, dR, (m+1) N floats each.
__global__ void wms_backward_kernel(const float* __restrict__ llr, const uint32_t* __restrict__ frozen_words,
                                    const float* __restrict__ w, int N, int m, int T, const float* __restrict__ ckpt,
                                    const float* __restrict__ dout, float* __restrict__ partial,
                                    float* __restrict__ dllr)
{
    extern __shared__ __align__(16) float sh[];
    const int plane = (m + 1) * N;
    float* dL = sh;
    float* dLp = sh + plane;
    float* dR = sh + 2 * plane;
    const long long cw = blockIdx.x;
    const size_t W = (size_t)T * m * (N / 2);
    for (int q = threadIdx.x; q < plane; q += blockDim.x) dL[q] = 0.f;
    float dl_acc[4] = {0.f, 0.f, 0.f, 0.f};  // dllr of positions threadIdx.x + j blockDim.x (N <= 4 blockDim.x)
    __syncthreads();
    for (int t = T - 1; t >= 0; --t) {
        const float* Rc = ckpt + ((size_t)cw * T + t) * 2 * plane + plane;                // R^t
        const float* Lp = t > 0 ? ckpt + ((size_t)cw * T + (t - 1)) * 2 * plane : nullptr;  // L^{t-1}
        wms_backward_iteration(Lp, Rc, dL, dLp, dR, frozen_words, w, N, m, T, t, dout + cw * N, partial + cw * W,
                               dl_acc);
    }
    for (int j = 0; j < 4; ++j) {
        const int i = threadIdx.x + j * blockDim.x;
        if (i < N) dllr[cw * N + i] = dl_acc[j];
    }
}

// k > 1: segments [t0, t0 + k) last to first, their L states recomputed from the checkpoint
// before them, each iteration's R plane rebuilt when its adjoint runs.  Shared memory: dL,
// dLp, dR, the R plane, then k L planes (Ls + i: the state before iteration t0 + i),
// (m+1) N floats each.
__global__ void wms_backward_seg_kernel(const float* __restrict__ llr, const uint32_t* __restrict__ frozen_words,
                                        const float* __restrict__ w, int N, int m, int T, int k,
                                        const float* __restrict__ ckpt, const float* __restrict__ dout,
                                        float* __restrict__ partial, float* __restrict__ dllr)
{
    extern __shared__ __align__(16) float sh[];
    const int plane = (m + 1) * N;
    float* dL = sh;
    float* dLp = sh + plane;
    float* dR = sh + 2 * plane;
    float* Rc = sh + 3 * plane;
    float* Ls = sh + 4 * plane;
    const long long cw = blockIdx.x;
    const float* llr_cw = llr + cw * N;
    const size_t W = (size_t)T * m * (N / 2);
    const int NC = (T - 1) / k;
    const int cols = (m - 1) * N;
    for (int q = threadIdx.x; q < plane; q += blockDim.x) dL[q] = 0.f;
    float dl_acc[4] = {0.f, 0.f, 0.f, 0.f};
    __syncthreads();
    for (int seg = (T - 1) / k; seg >= 0; --seg) {
        const int t0 = seg * k, len = min(T, t0 + k) - t0;
        // the L state before the segment: the prior, or the checkpoint after iteration t0 - 1
        wms_initial_L(Ls, frozen_words, N, m);
        __syncthreads();
        if (seg > 0) {
            const float* src = ckpt + ((size_t)cw * NC + seg - 1) * cols;
            for (int q = threadIdx.x; q < cols; q += blockDim.x) Ls[N + q] = src[q];
        }
        __syncthreads();
        // the segment's later L states with the forward's arithmetic (Rc is scratch here)
        for (int i = 1; i < len; ++i) {
            float* Li = Ls + (size_t)i * plane;
            for (int q = threadIdx.x; q < plane; q += blockDim.x) Li[q] = Li[q - plane];
            __syncthreads();
            wms_iteration(Li, Rc, llr_cw, w, N, m, t0 + i - 1);
        }
        for (int i = len - 1; i >= 0; --i) {
            const float* Lp = Ls + (size_t)i * plane;
            wms_rebuild_R(Lp, Rc, llr_cw, w, N, m, t0 + i);
            wms_backward_iteration(Lp, Rc, dL, dLp, dR, frozen_words, w, N, m, T, t0 + i, dout + cw * N,
                                   partial + cw * W, dl_acc);
        }
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
// k: the checkpoint interval, already clamped to [1, T]
WmsLayout wms_layout(int N, int m, int batch, int T, int k)
{
    WmsLayout l;
    const size_t W = (size_t)T * m * (N / 2);
    const size_t nchunks = ((size_t)batch + kReduceChunk - 1) / kReduceChunk;
    const size_t NC = (size_t)(T - 1) / k;
    const size_t ckpt_floats = k == 1 ? (size_t)T * 2 * (m + 1) * N : NC * (m - 1) * N;
    l.ckpt = 0;
    l.partial = align256((size_t)batch * ckpt_floats * sizeof(float));
    l.chunk = align256(l.partial + (size_t)batch * W * sizeof(float));
    l.total = align256(l.chunk + nchunks * W * sizeof(float));
    return l;
}

constexpr size_t kMaxBlockSmem = 227 * 1024;

size_t backward_smem(int N, int m, int k) { return (size_t)(k == 1 ? 3 : 4 + k) * (m + 1) * N * sizeof(float); }

// Checks the arguments; *k becomes the effective checkpoint interval min(k, T).
int wms_args(const polarbp_code* c, int batch, int T, int* k, int* N, int* m)
{
    using namespace polarbp_internal;
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (T < 1) return fail(POLARBP_ERR_ARG, "iterations must be >= 1");
    if (*k < 1) return fail(POLARBP_ERR_ARG, "checkpoint interval must be >= 1");
    if (*k > T) *k = T;
    polarbp_code_info(c, N, nullptr, m);
    if (*m > 10) return fail(POLARBP_ERR_UNSUPPORTED, "weighted min-sum supports N <= 1024");
    if (bit_reversed(c)) return fail(POLARBP_ERR_UNSUPPORTED, "this decoder variant takes codewords in natural order only (see polarbp_set_bit_reversed)");
    if (backward_smem(*N, *m, *k) > kMaxBlockSmem)
        return fail(POLARBP_ERR_UNSUPPORTED, "checkpoint interval too long for this code length (shared memory of the adjoint)");
    return POLARBP_OK;
}
}  // namespace

extern "C" {

size_t polarbp_wms_workspace(const polarbp_code* code, int batch, int iterations, int checkpoint_every)
{
    int N = 0, m = 0;
    if (!code || batch < 0 || iterations < 1 || checkpoint_every < 1) return 0;
    polarbp_code_info(code, &N, nullptr, &m);
    return wms_layout(N, m, batch, iterations, checkpoint_every < iterations ? checkpoint_every : iterations).total;
}

int polarbp_wms_forward(const polarbp_code* code, const float* llr, int batch, int iterations, int checkpoint_every,
                        const float* weights, float* out, void* workspace, size_t workspace_bytes, void* stream)
{
    using namespace polarbp_internal;
    int N = 0, m = 0, k = checkpoint_every;
    int rc = wms_args(code, batch, iterations, &k, &N, &m);
    if (rc != POLARBP_OK) return rc;
    if (batch == 0) return POLARBP_OK;
    if (!llr || !weights || !out) return fail(POLARBP_ERR_ARG, "llr, weights and out must be device pointers");
    const WmsLayout l = wms_layout(N, m, batch, iterations, k);
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
        llr, frozen_words(code), weights, N, m, iterations, k, out, ckpt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "wms forward launch");
    return POLARBP_OK;
}

int polarbp_wms_backward(const polarbp_code* code, const float* llr, int batch, int iterations, int checkpoint_every,
                         const float* weights, const float* dout, float* dweights, float* dllr, void* workspace,
                         size_t workspace_bytes, void* stream)
{
    using namespace polarbp_internal;
    int N = 0, m = 0, k = checkpoint_every;
    int rc = wms_args(code, batch, iterations, &k, &N, &m);
    if (rc != POLARBP_OK) return rc;
    if (!weights || !dweights) return fail(POLARBP_ERR_ARG, "weights and dweights must be device pointers");
    const size_t W = (size_t)iterations * m * (N / 2);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (batch == 0) {
        cudaError_t e = cudaMemsetAsync(dweights, 0, W * sizeof(float), s);
        return e == cudaSuccess ? POLARBP_OK : cuda_fail(e, "wms backward");
    }
    if (!llr || !dout || !dllr) return fail(POLARBP_ERR_ARG, "llr, dout and dllr must be device pointers");
    const WmsLayout l = wms_layout(N, m, batch, iterations, k);
    if (!workspace || workspace_bytes < l.total) return fail(POLARBP_ERR_ARG, "workspace too small");
    rc = check_device(code);
    if (rc != POLARBP_OK) return rc;
    const int threads = N / 2 < 32 ? 32 : N / 2;
    const size_t smem = backward_smem(N, m, k);
    auto kern = k == 1 ? (void*)wms_backward_kernel : (void*)wms_backward_seg_kernel;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "wms backward attribute");
    }
    const float* ckpt = reinterpret_cast<const float*>(static_cast<const char*>(workspace) + l.ckpt);
    float* partial = reinterpret_cast<float*>(static_cast<char*>(workspace) + l.partial);
    if (k == 1)
        wms_backward_kernel<<<batch, threads, smem, s>>>(llr, frozen_words(code), weights, N, m, iterations, ckpt,
                                                         dout, partial, dllr);
    else
        wms_backward_seg_kernel<<<batch, threads, smem, s>>>(llr, frozen_words(code), weights, N, m, iterations, k,
                                                             ckpt, dout, partial, dllr);
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
