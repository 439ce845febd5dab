// polarbp_api.cu -- host side of the C ABI declared in include/polarbp.h:
// argument checking, code construction (Sec. II), the encoder kernel and the
// dispatch of the decode kernels in bp_decode.cuh.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "polarbp.h"
#include "bp_decode.cuh"
#include "bp_mixed.cuh"

constexpr int kPipe = 3;  // streams of polarbp_decode_host's copy/decode pipeline

struct polarbp_code {
    int N = 0, K = 0, m = 0;
    int device = 0;
    std::vector<uint8_t> frozen;
    uint32_t* d_frozen = nullptr;  // ceil(N/32) words, bit i = frozen[i]
    unsigned int* d_status = nullptr;
    int cpc = 1;  // codewords per block of the persistent launch
    int mapping = POLARBP_MAP_PIPELINED;  // thread mapping when freezing at N = 256 .. 4096 (set by construct)
    int bitrev = 0;  // 1: channel position i carries code position rev(i) (Arikan's B_N)
    // polarbp_decode_host's pipeline, created with the handle so that the call
    // itself creates nothing; `pipe_lock` serialises enqueueing on them
    cudaStream_t pipe[kPipe] = {};
    cudaEvent_t pipe_start = nullptr;
    cudaEvent_t pipe_done[kPipe] = {};
    mutable std::mutex pipe_lock;
};

// decode kernels, one translation unit per code length (compiled in parallel)
namespace polarbp {
cudaError_t launch_m1(const LaunchReq&);
cudaError_t launch_m2(const LaunchReq&);
cudaError_t launch_m3(const LaunchReq&);
cudaError_t launch_m4(const LaunchReq&);
cudaError_t launch_m5(const LaunchReq&);
cudaError_t launch_m6(const LaunchReq&);
cudaError_t launch_m7(const LaunchReq&);
cudaError_t launch_m8(const LaunchReq&);
cudaError_t launch_m9(const LaunchReq&);
cudaError_t launch_m10(const LaunchReq&);
cudaError_t launch_m11(const LaunchReq&);
cudaError_t launch_m12(const LaunchReq&);
cudaError_t launch_m13(const LaunchReq&);  // thread-block clusters (bp_cluster.cuh)
cudaError_t launch_m14(const LaunchReq&);
cudaError_t launch_m15(const LaunchReq&);
cudaError_t launch_persistent_m8(const SegLaunch&);
cudaError_t launch_persistent_m9(const SegLaunch&);
cudaError_t launch_persistent_m10(const SegLaunch&);
cudaError_t launch_persistent_m11(const SegLaunch&);
cudaError_t launch_persistent_m12(const SegLaunch&);
cudaError_t launch_mixed_m8(const MixedArgs&, int, int, int, cudaStream_t);  // one launch, longest N = 2^m (bp_mixed.cuh)
cudaError_t launch_mixed_m9(const MixedArgs&, int, int, int, cudaStream_t);
cudaError_t launch_mixed_m10(const MixedArgs&, int, int, int, cudaStream_t);
cudaError_t launch_mixed_m11(const MixedArgs&, int, int, int, cudaStream_t);
cudaError_t launch_mixed_m12(const MixedArgs&, int, int, int, cudaStream_t);
}  // namespace polarbp

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return POLARBP_ERR_CUDA;
}

int exact_log2(int n)
{
    if (n < 1) return -1;
    int m = 0;
    while ((1 << m) < n) ++m;
    return (1 << m) == n ? m : -1;
}

// Frozen set of an (N, K) code from the Bhattacharyya parameters of a binary
// erasure channel with erasure probability z0 (the paper leaves the
// construction open).  Position i's synthetic channel is obtained by splitting
// z0 m times, the bits of i from the most significant one down choosing the
// worse (2z - z^2, bit 0) or the better (z^2, bit 1) half; the pair
// (ln z, ln(1 - z)) is tracked so neither tail saturates.  The N - K positions
// with the largest z are frozen; among equal z the smaller index counts as the
// less reliable.
void bec_frozen_set(int N, int m, int K, double z0, std::vector<uint8_t>& frozen)
{
    std::vector<std::pair<double, int>> order(N);
    for (int i = 0; i < N; ++i) {
        double lz = std::log(z0), lw = std::log1p(-z0);  // ln z, ln(1 - z)
        for (int b = m - 1; b >= 0; --b) {
            if ((i >> b) & 1) {
                const double lw_next = lw + std::log1p(std::exp(lz));
                lz = 2.0 * lz;
                lw = lw_next;
            } else {
                const double lz_next = lz + std::log1p(std::exp(lw));
                lw = 2.0 * lw;
                lz = lz_next;
            }
        }
        order[i] = {lz - lw, i};
    }
    std::sort(order.begin(), order.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
        if (a.first != b.first) return a.first < b.first;
        return a.second > b.second;
    });
    frozen.assign(N, 1);
    for (int k = 0; k < K; ++k) frozen[order[k].second] = 0;
}

int check_device(const polarbp_code* c)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != c->device) return fail(POLARBP_ERR_ARG, "code handle belongs to another device");
    return POLARBP_OK;
}

// x = u F^{(x)m}: one block per codeword, the N bits in shared memory, one
// butterfly pass per index bit (v[c] ^= v[c + h] for c with bit h clear).
__global__ void encode_kernel(const uint8_t* __restrict__ u, uint8_t* __restrict__ x, int N, int m, int bitrev)
{
    extern __shared__ uint8_t buf[];
    const long long cw = blockIdx.x;
    for (int i = threadIdx.x; i < N; i += blockDim.x) buf[i] = u[cw * N + i] & 1u;
    __syncthreads();
    for (int b = 0; b < m; ++b) {
        const int h = 1 << b;
        for (int c = threadIdx.x; c < N; c += blockDim.x)
            if (!(c & h)) buf[c] ^= buf[c + h];
        __syncthreads();
    }
    // bit-reversed order: channel position i carries code position rev(i)
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        x[cw * N + i] = buf[bitrev ? (int)(__brev((unsigned)i) >> (32 - m)) : i];
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// the key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t philox_word(uint64_t seed, uint64_t cw, uint32_t stream, uint32_t w)
{
    const uint4 o = philox4x32_10(make_uint4(w >> 2, (uint32_t)cw, (uint32_t)(cw >> 32), stream), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    const uint32_t q = w & 3u;
    return q == 0 ? o.x : q == 1 ? o.y : q == 2 ? o.z : o.w;
}

// One block per codeword: source bits, encoder (as encode_kernel), BPSK + AWGN.
__global__ void awgn_kernel(const uint32_t* __restrict__ frozen_words, int N, int m, uint64_t seed, uint64_t first,
                            float sigma_all, const float* __restrict__ ebn0_per_cw, float rate, int bitrev,
                            uint8_t* __restrict__ u_out, float* __restrict__ llr)
{
    extern __shared__ uint8_t bits[];
    const long long b = blockIdx.x;
    const uint64_t cw = first + (uint64_t)b;
    // per-codeword Eb/N0: sigma^2 = 1 / (2 R 10^(Eb/N0 / 10))
    const float sigma = ebn0_per_cw ? sqrtf(1.f / (2.f * rate * exp10f(ebn0_per_cw[b] * 0.1f))) : sigma_all;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const uint32_t word = philox_word(seed, cw, 1u, (uint32_t)(i >> 5));
        const uint32_t fz = (frozen_words[i >> 5] >> (i & 31)) & 1u;
        const uint8_t ui = fz ? 0 : (uint8_t)((word >> (i & 31)) & 1u);
        bits[i] = ui;
        if (u_out) u_out[b * N + i] = ui;
    }
    __syncthreads();
    for (int s = 0; s < m; ++s) {
        const int h = 1 << s;
        for (int c = threadIdx.x; c < N; c += blockDim.x)
            if (!(c & h)) bits[c] ^= bits[c + h];
        __syncthreads();
    }
    const float scale = 2.f / (sigma * sigma);
    for (int p = threadIdx.x; p < (N + 1) / 2; p += blockDim.x) {
        const uint32_t w0 = philox_word(seed, cw, 2u, (uint32_t)(2 * p));
        const uint32_t w1 = philox_word(seed, cw, 2u, (uint32_t)(2 * p + 1));
        const float u1 = ((float)w0 + 1.0f) * 2.3283064365386963e-10f;  // (w0 + 1) / 2^32
        const float u2 = (float)w1 * 2.3283064365386963e-10f;
        const float r = sqrtf(-2.f * logf(u1));
        float sn, cs;
        sincospif(2.f * u2, &sn, &cs);
        // channel positions i0, i1 carry code positions rev(i0), rev(i1) in bit-reversed order
        const int i0 = 2 * p, i1 = 2 * p + 1;
        const int c0 = bitrev ? (int)(__brev((unsigned)i0) >> (32 - m)) : i0;
        const int c1 = bitrev ? (int)(__brev((unsigned)i1) >> (32 - m)) : i1;
        llr[b * N + i0] = scale * ((1.f - 2.f * bits[c0]) + sigma * r * cs);
        if (i1 < N) llr[b * N + i1] = scale * ((1.f - 2.f * bits[c1]) + sigma * r * sn);
    }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct HostLayout {
    size_t llr, u_hat, iters, pe, total;
};

HostLayout host_layout(int N, int batch)
{
    HostLayout h;
    size_t b = (size_t)batch;
    h.llr = 0;
    h.u_hat = align256(h.llr + b * N * sizeof(float));
    h.iters = align256(h.u_hat + b * N);
    h.pe = align256(h.iters + b * sizeof(int32_t));
    h.total = align256(h.pe + b * sizeof(int64_t));
    return h;
}

// The decode parameters that do not depend on the buffers.  The host entry
// points check them before they enqueue any copy, so that an argument error
// never leaves a copy from the caller's host buffer in flight.
int decode_params_check(const polarbp_code* c, int batch, int max_iter, float scale, int stop_mode, int freeze_mode)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (max_iter < 1) return fail(POLARBP_ERR_ARG, "max_iter must be >= 1");
    if (!(scale > 0.f) || !std::isfinite(scale)) return fail(POLARBP_ERR_ARG, "scale must be finite and > 0");
    if (stop_mode != POLARBP_STOP_NONE && stop_mode != POLARBP_STOP_GMATRIX)
        return fail(POLARBP_ERR_ARG, "unknown stop_mode");
    if (freeze_mode != POLARBP_FREEZE_OFF && freeze_mode != POLARBP_FREEZE_CSFG &&
        freeze_mode != POLARBP_FREEZE_CSFG_MULTI)
        return fail(POLARBP_ERR_ARG, "unknown freeze_mode");
    if (freeze_mode == POLARBP_FREEZE_CSFG_MULTI && c->m > 12)
        return fail(POLARBP_ERR_UNSUPPORTED, "POLARBP_FREEZE_CSFG_MULTI supports N <= 4096");
    if (c->m > 15) return fail(POLARBP_ERR_UNSUPPORTED, "decode supports N <= 32768");
    return POLARBP_OK;
}

int decode_impl(const polarbp_code* c, const float* llr, int batch, int max_iter, float scale, int stop_mode,
                int freeze_mode, uint8_t* u_hat, int32_t* iterations, int64_t* pe_updates, float* trace_L,
                float* trace_R, int32_t* trace_P, bool trace, void* stream)
{
    {
        const int rc = decode_params_check(c, batch, max_iter, scale, stop_mode, freeze_mode);
        if (rc != POLARBP_OK) return rc;
    }
    if (batch == 0) return POLARBP_OK;
    if (!llr || !u_hat) return fail(POLARBP_ERR_ARG, "llr and u_hat must be device pointers");
    if (trace && (!trace_L || !trace_R || !trace_P)) return fail(POLARBP_ERR_ARG, "trace buffers must be given");
    int rc = check_device(c);
    if (rc != POLARBP_OK) return rc;

    polarbp::LaunchReq q;
    q.args.llr = llr;
    q.args.frozen_words = c->d_frozen;
    q.args.u_hat = u_hat;
    q.args.iters = iterations;
    q.args.pe = pe_updates;
    q.args.status = c->d_status;
    q.args.trace_L = trace_L;
    q.args.trace_R = trace_R;
    q.args.trace_P = trace_P;
    q.args.batch = batch;
    q.args.max_iter = max_iter;
    q.args.alpha = scale;
    q.args.bitrev = c->bitrev;
    q.stop_mode = stop_mode;
    q.freeze_mode = freeze_mode;
    q.trace = trace;
    q.pipelined = c->mapping == POLARBP_MAP_PIPELINED;
    q.stream = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (c->m) {
    case 1: e = polarbp::launch_m1(q); break;
    case 2: e = polarbp::launch_m2(q); break;
    case 3: e = polarbp::launch_m3(q); break;
    case 4: e = polarbp::launch_m4(q); break;
    case 5: e = polarbp::launch_m5(q); break;
    case 6: e = polarbp::launch_m6(q); break;
    case 7: e = polarbp::launch_m7(q); break;
    case 8: e = polarbp::launch_m8(q); break;
    case 9: e = polarbp::launch_m9(q); break;
    case 10: e = polarbp::launch_m10(q); break;
    case 11: e = polarbp::launch_m11(q); break;
    case 12: e = polarbp::launch_m12(q); break;
    case 13: e = polarbp::launch_m13(q); break;
    case 14: e = polarbp::launch_m14(q); break;
    default: e = polarbp::launch_m15(q); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    return POLARBP_OK;
}

// Side streams and events for the concurrent persistent launches of
// polarbp_decode_segments, created once per device.
constexpr int kSegWorkspace = 256;
constexpr int kSideStreams = 4;
struct SideResources {
    bool ready = false;
    int sms = 0;
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kSideStreams] = {};
};
std::mutex g_side_mutex;
SideResources g_side[64];

int side_resources(SideResources** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(POLARBP_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_side_mutex);
    SideResources& r = g_side[dev];
    if (!r.ready) {
        e = cudaDeviceGetAttribute(&r.sms, cudaDevAttrMultiProcessorCount, dev);
        for (int k = 0; e == cudaSuccess && k < kSideStreams; ++k) {
            e = cudaStreamCreateWithFlags(&r.side[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.join[k], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            // undo a partial creation so that the next call starts clean
            for (int k = 0; k < kSideStreams; ++k) {
                if (r.side[k]) cudaStreamDestroy(r.side[k]);
                if (r.join[k]) cudaEventDestroy(r.join[k]);
                r.side[k] = nullptr;
                r.join[k] = nullptr;
            }
            if (r.fork) cudaEventDestroy(r.fork);
            r.fork = nullptr;
            return cuda_fail(e, "side stream creation");
        }
        r.ready = true;
    }
    *out = &r;
    return POLARBP_OK;
}

cudaError_t launch_persistent_m(int m, const polarbp::SegLaunch& q)
{
    switch (m) {
    case 8: return polarbp::launch_persistent_m8(q);
    case 9: return polarbp::launch_persistent_m9(q);
    case 10: return polarbp::launch_persistent_m10(q);
    case 11: return polarbp::launch_persistent_m11(q);
    case 12: return polarbp::launch_persistent_m12(q);
    default: return cudaErrorInvalidValue;
    }
}

// Staging area of polarbp_decode_host_noalloc: a fixed device array that is
// part of the library image, so the entry point never allocates.  Host code
// must not pass the symbol itself to a kernel or copy (on the host it names a
// host-side stand-in); it uses the device address looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[POLARBP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kMaxDevices] = {};

int noalloc_scratch_address(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(POLARBP_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the built-in scratch");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return POLARBP_OK;
}


int first_of_length(const polarbp_segment* segs, int nseg, int m)
{
    for (int k = 0; k < nseg; ++k)
        if (segs[k].count > 0 && segs[k].code->m == m) return k;
    return 0;
}

// Checks the arguments of the mixed-stream entry points and groups the runs by
// code length: args[m] (m = 8 .. 12) lists the runs of length 2^m in call order,
// their queue counter at workspace + m; total 0 when the stream has none.
// per_length: the runs are decoded by one persistent launch per length, whose
// codewords-per-block setting must be admissible.
int group_segments(const polarbp_segment* segs, int nseg, int max_iter, float scale, int stop_mode, int freeze_mode,
                   void* workspace, size_t workspace_bytes, bool per_length, polarbp::SegArgs* args)
{
    if (nseg < 0 || (nseg > 0 && !segs)) return fail(POLARBP_ERR_ARG, "bad segment list");
    if (max_iter < 1) return fail(POLARBP_ERR_ARG, "max_iter must be >= 1");
    if (!(scale > 0.f) || !std::isfinite(scale)) return fail(POLARBP_ERR_ARG, "scale must be finite and > 0");
    if (stop_mode != POLARBP_STOP_NONE && stop_mode != POLARBP_STOP_GMATRIX)
        return fail(POLARBP_ERR_ARG, "unknown stop_mode");
    if (freeze_mode != POLARBP_FREEZE_OFF && freeze_mode != POLARBP_FREEZE_CSFG)
        return fail(POLARBP_ERR_ARG, "unknown freeze_mode");
    if (!workspace || workspace_bytes < (size_t)kSegWorkspace) return fail(POLARBP_ERR_ARG, "workspace too small");
    std::vector<int> by_m[13];
    for (int k = 0; k < nseg; ++k) {
        const polarbp_segment& g = segs[k];
        if (!g.code) return fail(POLARBP_ERR_ARG, "segment without a code");
        if (g.code->m < 8 || g.code->m > 12)
            return fail(POLARBP_ERR_UNSUPPORTED, "segments support N from 256 to 4096");
        if (g.count < 0) return fail(POLARBP_ERR_ARG, "segment count must be >= 0");
        if (g.count == 0) continue;
        if (!g.llr || !g.u_hat) return fail(POLARBP_ERR_ARG, "segment llr and u_hat must be device pointers");
        int rc = check_device(g.code);
        if (rc != POLARBP_OK) return rc;
        by_m[g.code->m].push_back(k);
    }
    for (int m = 0; m <= 12; ++m) {
        polarbp::SegArgs& q = args[m];
        q = polarbp::SegArgs{};
        q.queue = static_cast<int*>(workspace) + m;
        q.max_iter = max_iter;
        q.alpha = scale;
        if (by_m[m].empty()) continue;
        if ((int)by_m[m].size() > polarbp::kMaxSeg) return fail(POLARBP_ERR_ARG, "at most 8 segments per code length");
        long long total = 0;
        for (int k : by_m[m]) total += segs[k].count;
        if (total > 0x7fffffffLL) return fail(POLARBP_ERR_ARG, "too many codewords of one length");
        if (per_length && !polarbp::persistent_supported(m, segs[by_m[m][0]].code->cpc))
            return fail(POLARBP_ERR_UNSUPPORTED, "codewords per block");
        q.nseg = (int)by_m[m].size();
        int start = 0;
        for (int j = 0; j < q.nseg; ++j) {
            const polarbp_segment& sg = segs[by_m[m][j]];
            q.start[j] = start;
            q.llr[j] = sg.llr;
            q.frozen_words[j] = sg.code->d_frozen;
            q.status[j] = sg.code->d_status;
            q.u_hat[j] = sg.u_hat;
            q.iters[j] = sg.iterations;
            q.pe[j] = sg.pe_updates;
            q.bitrev[j] = sg.code->bitrev;
            start += sg.count;
        }
        q.start[q.nseg] = start;
        q.total = start;
    }
    return POLARBP_OK;
}

}  // namespace

// accessors shared with the other translation units of the library
namespace polarbp_internal {
const uint32_t* frozen_words(const polarbp_code* c) { return c->d_frozen; }
unsigned int* status_word(const polarbp_code* c) { return c->d_status; }
int fail(int code, const std::string& msg) { return ::fail(code, msg); }
int cuda_fail(cudaError_t e, const char* what) { return ::cuda_fail(e, what); }
int check_device(const polarbp_code* c) { return ::check_device(c); }
int bit_reversed(const polarbp_code* c) { return c->bitrev; }
}  // namespace polarbp_internal

// Free everything a code handle owns (any member may still be unset).
static void release(polarbp_code* c)
{
    if (c->d_frozen) cudaFree(c->d_frozen);
    if (c->d_status) cudaFree(c->d_status);
    for (int i = 0; i < kPipe; ++i) {
        if (c->pipe[i]) cudaStreamDestroy(c->pipe[i]);
        if (c->pipe_done[i]) cudaEventDestroy(c->pipe_done[i]);
    }
    if (c->pipe_start) cudaEventDestroy(c->pipe_start);
    delete c;
}

extern "C" {

int polarbp_construct(int N, int K, const uint8_t* frozen_mask, double z0, polarbp_code** out)
{
    if (!out) return fail(POLARBP_ERR_ARG, "out is NULL");
    *out = nullptr;
    const int m = exact_log2(N);
    if (m < 1 || N > 32768) return fail(POLARBP_ERR_ARG, "N must be a power of two in [2, 32768]");
    if (K < 0 || K > N) return fail(POLARBP_ERR_ARG, "K must be in [0, N]");
    polarbp_code* c = new (std::nothrow) polarbp_code;
    if (!c) return fail(POLARBP_ERR_NOMEM, "out of host memory");
    c->N = N;
    c->K = K;
    c->m = m;
    // default thread mapping: pipelined where it measured faster (N >= 1024; at N = 256 its
    // checker warp is as large as the one-warp sweep and the block mapping is 1.3x faster)
    c->mapping = m >= 10 ? POLARBP_MAP_PIPELINED : POLARBP_MAP_BLOCK;
    if (frozen_mask) {
        c->frozen.assign(frozen_mask, frozen_mask + N);
        int nf = 0;
        for (int i = 0; i < N; ++i) {
            if (c->frozen[i] > 1) {
                delete c;
                return fail(POLARBP_ERR_ARG, "frozen_mask entries must be 0 or 1");
            }
            nf += c->frozen[i];
        }
        if (nf != N - K) {
            delete c;
            return fail(POLARBP_ERR_ARG, "frozen_mask popcount must equal N - K");
        }
    } else {
        if (!(z0 > 0.0 && z0 < 1.0)) {
            delete c;
            return fail(POLARBP_ERR_ARG, "z0 must be in (0, 1)");
        }
        bec_frozen_set(N, m, K, z0, c->frozen);
    }
    const int nw = (N + 31) / 32;
    std::vector<uint32_t> words(nw, 0u);
    for (int i = 0; i < N; ++i)
        if (c->frozen[i]) words[i >> 5] |= 1u << (i & 31);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_frozen, nw * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(c->d_frozen, words.data(), nw * sizeof(uint32_t), cudaMemcpyHostToDevice);
    // status words: flags, then the checked build's redzone record
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, polarbp::kStatusWords * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, polarbp::kStatusWords * sizeof(unsigned int));
    for (int i = 0; i < kPipe && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&c->pipe[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->pipe_done[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->pipe_start, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int rc = (e == cudaErrorMemoryAllocation) ? fail(POLARBP_ERR_NOMEM, "device allocation failed")
                                                  : cuda_fail(e, "construct");
        release(c);
        return rc;
    }
    *out = c;
    return POLARBP_OK;
}

int polarbp_frozen_set(int N, int K, double z0, uint8_t* frozen_mask)
{
    const int m = exact_log2(N);
    if (m < 1 || N > 32768) return fail(POLARBP_ERR_ARG, "N must be a power of two in [2, 32768]");
    if (K < 0 || K > N) return fail(POLARBP_ERR_ARG, "K must be in [0, N]");
    if (!(z0 > 0.0 && z0 < 1.0)) return fail(POLARBP_ERR_ARG, "z0 must be in (0, 1)");
    if (!frozen_mask) return fail(POLARBP_ERR_ARG, "frozen_mask is NULL");
    std::vector<uint8_t> f;
    bec_frozen_set(N, m, K, z0, f);
    std::memcpy(frozen_mask, f.data(), (size_t)N);
    return POLARBP_OK;
}

void polarbp_destroy(polarbp_code* c)
{
    if (!c) return;
    // drain the handle's device, which need not be the caller's current one
    const int dev = c->device;
    int cur = -1;
    const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != dev;
    if (other) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    release(c);
    if (other) cudaSetDevice(cur);
}

int polarbp_code_info(const polarbp_code* c, int* N, int* K, int* m)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (N) *N = c->N;
    if (K) *K = c->K;
    if (m) *m = c->m;
    return POLARBP_OK;
}

int polarbp_set_bit_reversed(polarbp_code* c, int on)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (on != 0 && on != 1) return fail(POLARBP_ERR_ARG, "on must be 0 or 1");
    c->bitrev = on;
    return POLARBP_OK;
}

int polarbp_get_bit_reversed(const polarbp_code* c, int* on)
{
    if (!c || !on) return fail(POLARBP_ERR_ARG, "NULL argument");
    *on = c->bitrev;
    return POLARBP_OK;
}

int polarbp_get_frozen_mask(const polarbp_code* c, uint8_t* frozen_mask)
{
    if (!c || !frozen_mask) return fail(POLARBP_ERR_ARG, "NULL argument");
    std::memcpy(frozen_mask, c->frozen.data(), (size_t)c->N);
    return POLARBP_OK;
}

int polarbp_encode(const polarbp_code* c, const uint8_t* u, uint8_t* x, int batch, void* stream)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (batch == 0) return POLARBP_OK;
    if (!u || !x || u == x) return fail(POLARBP_ERR_ARG, "u and x must be distinct device pointers");
    int rc = check_device(c);
    if (rc != POLARBP_OK) return rc;
    const int threads = c->N < 256 ? (c->N < 32 ? 32 : c->N) : 256;
    encode_kernel<<<batch, threads, c->N, static_cast<cudaStream_t>(stream)>>>(u, x, c->N, c->m, c->bitrev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "encode launch");
    return POLARBP_OK;
}

int polarbp_decode(const polarbp_code* c, const float* llr, int batch, int max_iter, float scale, int stop_mode,
                   int freeze_mode, uint8_t* u_hat, int32_t* iterations, int64_t* pe_updates, void* stream)
{
    return decode_impl(c, llr, batch, max_iter, scale, stop_mode, freeze_mode, u_hat, iterations, pe_updates,
                       nullptr, nullptr, nullptr, false, stream);
}

int polarbp_decode_trace(const polarbp_code* c, const float* llr, int batch, int max_iter, float scale,
                         int stop_mode, int freeze_mode, uint8_t* u_hat, int32_t* iterations, int64_t* pe_updates,
                         float* trace_L, float* trace_R, int32_t* trace_P, void* stream)
{
    return decode_impl(c, llr, batch, max_iter, scale, stop_mode, freeze_mode, u_hat, iterations, pe_updates,
                       trace_L, trace_R, trace_P, true, stream);
}

size_t polarbp_decode_host_workspace(const polarbp_code* c, int batch)
{
    if (!c || batch < 0) return 0;
    return host_layout(c->N, batch).total;
}

int polarbp_decode_host(const polarbp_code* c, const float* llr, int batch, int max_iter, float scale,
                        int stop_mode, int freeze_mode, uint8_t* u_hat, int32_t* iterations, int64_t* pe_updates,
                        void* workspace, size_t workspace_bytes, void* stream)
{
    {
        const int rc = decode_params_check(c, batch, max_iter, scale, stop_mode, freeze_mode);
        if (rc != POLARBP_OK) return rc;
    }
    if (batch == 0) return POLARBP_OK;
    if (!llr || !u_hat) return fail(POLARBP_ERR_ARG, "llr and u_hat must be host pointers");
    const HostLayout h = host_layout(c->N, batch);
    if (!workspace || workspace_bytes < h.total) return fail(POLARBP_ERR_ARG, "workspace too small");
    {
        const int rc = check_device(c);
        if (rc != POLARBP_OK) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(workspace);
    float* d_llr = reinterpret_cast<float*>(ws + h.llr);
    uint8_t* d_u = reinterpret_cast<uint8_t*>(ws + h.u_hat);
    int32_t* d_it = reinterpret_cast<int32_t*>(ws + h.iters);
    int64_t* d_pe = reinterpret_cast<int64_t*>(ws + h.pe);
    // Codewords are independent, so a large batch runs as a pipeline of chunks
    // of about 64 MiB of LLRs, dealt round-robin to the handle's streams: the
    // upload of one chunk, the decode of another and the download of a third
    // overlap (the copy engines and the SMs work at once).  A batch of fewer
    // than two chunks runs as one upload, decode and download on `stream`.
    const int N = c->N;
    const int cb = (int)std::max<size_t>(1, ((size_t)64 << 20) / ((size_t)N * sizeof(float)));
    const bool piped = batch >= 2 * cb;
    std::unique_lock<std::mutex> lock(c->pipe_lock, std::defer_lock);
    cudaError_t e = cudaSuccess;
    // Once a copy is enqueued, every error return first waits for the streams
    // used so far, so that no copy from or to the caller's host buffers is left
    // in flight when the call returns.
    auto drain = [&](int rc) {
        if (piped)
            for (int i = 0; i < kPipe; ++i) cudaStreamSynchronize(c->pipe[i]);
        cudaStreamSynchronize(s);
        return rc;
    };
    if (piped) {
        lock.lock();
        e = cudaEventRecord(c->pipe_start, s);
        for (int i = 0; i < kPipe && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(c->pipe[i], c->pipe_start, 0);
        if (e != cudaSuccess) return cuda_fail(e, "decode_host pipeline");
    }
    for (int k = 0, off = 0; off < batch; ++k, off += (piped ? cb : batch)) {
        const int nb = piped ? std::min(cb, batch - off) : batch;
        cudaStream_t st = piped ? c->pipe[k % kPipe] : s;
        const size_t o = (size_t)off * N, n = (size_t)nb * N;
        e = cudaMemcpyAsync(d_llr + o, llr + o, n * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return drain(cuda_fail(e, "llr upload"));
        int rc = decode_impl(c, d_llr + o, nb, max_iter, scale, stop_mode, freeze_mode, d_u + o, d_it + off, d_pe + off,
                             nullptr, nullptr, nullptr, false, st);
        if (rc != POLARBP_OK) return drain(rc);
        e = cudaMemcpyAsync(u_hat + o, d_u + o, n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && iterations)
            e = cudaMemcpyAsync(iterations + off, d_it + off, (size_t)nb * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && pe_updates)
            e = cudaMemcpyAsync(pe_updates + off, d_pe + off, (size_t)nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return drain(cuda_fail(e, "decode_host copies"));
    }
    if (piped) {
        for (int i = 0; i < kPipe && e == cudaSuccess; ++i) {
            e = cudaEventRecord(c->pipe_done[i], c->pipe[i]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->pipe_done[i], 0);
        }
        if (e != cudaSuccess) return drain(cuda_fail(e, "decode_host pipeline"));
        lock.unlock();
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "decode_host copies");
    return POLARBP_OK;
}

int polarbp_awgn(const polarbp_code* c, uint64_t seed, uint64_t first_codeword, int batch, float ebn0_db, uint8_t* u,
                 float* llr, void* stream)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (c->K < 1) return fail(POLARBP_ERR_ARG, "the channel needs K >= 1 (rate > 0)");
    if (!std::isfinite(ebn0_db)) return fail(POLARBP_ERR_ARG, "ebn0_db must be finite");
    if (batch == 0) return POLARBP_OK;
    if (!llr) return fail(POLARBP_ERR_ARG, "llr must be a device pointer");
    int rc = check_device(c);
    if (rc != POLARBP_OK) return rc;
    const double rate = (double)c->K / (double)c->N;
    const float sigma = (float)std::sqrt(1.0 / (2.0 * rate * std::pow(10.0, ebn0_db / 10.0)));
    const int threads = c->N < 256 ? (c->N < 32 ? 32 : c->N) : 256;
    awgn_kernel<<<batch, threads, c->N, static_cast<cudaStream_t>(stream)>>>(c->d_frozen, c->N, c->m, seed,
                                                                             first_codeword, sigma, nullptr, 0.f,
                                                                             c->bitrev, u, llr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "awgn launch");
    return POLARBP_OK;
}

int polarbp_decode_host_noalloc(const polarbp_code* c, const float* llr, int batch, int max_iter, float scale,
                                int stop_mode, int freeze_mode, uint8_t* u_hat, int32_t* iterations,
                                int64_t* pe_updates, void* stream)
{
    {
        const int rc = decode_params_check(c, batch, max_iter, scale, stop_mode, freeze_mode);
        if (rc != POLARBP_OK) return rc;
    }
    if (batch == 0) return POLARBP_OK;
    {
        // the scratch address below is looked up on the current device: it must be the handle's
        const int rc = check_device(c);
        if (rc != POLARBP_OK) return rc;
    }
    const size_t need = host_layout(c->N, batch).total;
    if (need > POLARBP_NOALLOC_SCRATCH_BYTES) {
        size_t fit = 0;
        size_t lo = 1, hi = (size_t)batch;
        while (lo <= hi) {  // largest batch whose staging fits the array
            const size_t mid = (lo + hi) / 2;
            if (host_layout(c->N, (int)mid).total <= POLARBP_NOALLOC_SCRATCH_BYTES) {
                fit = mid;
                lo = mid + 1;
            } else {
                hi = mid - 1;
            }
        }
        return fail(POLARBP_ERR_ARG, "batch too large for the built-in 16 MiB scratch: at most " +
                                         std::to_string(fit) + " codewords of length " + std::to_string(c->N) +
                                         " per call");
    }
    void* ws = nullptr;
    int rc = noalloc_scratch_address(&ws);
    if (rc != POLARBP_OK) return rc;
    return polarbp_decode_host(c, llr, batch, max_iter, scale, stop_mode, freeze_mode, u_hat, iterations, pe_updates,
                               ws, POLARBP_NOALLOC_SCRATCH_BYTES, stream);
}

size_t polarbp_decode_segments_workspace(void) { return kSegWorkspace; }

int polarbp_set_codewords_per_block(polarbp_code* c, int cpc)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (!polarbp::persistent_supported(c->m, cpc))
        return fail(POLARBP_ERR_UNSUPPORTED, "codewords per block not admissible for this code length");
    c->cpc = cpc;
    return POLARBP_OK;
}

int polarbp_get_codewords_per_block(const polarbp_code* c, int* cpc)
{
    if (!c || !cpc) return fail(POLARBP_ERR_ARG, "NULL argument");
    *cpc = c->cpc;
    return POLARBP_OK;
}

int polarbp_set_thread_mapping(polarbp_code* c, int mapping)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (mapping != POLARBP_MAP_PIPELINED && mapping != POLARBP_MAP_BLOCK)
        return fail(POLARBP_ERR_ARG, "unknown thread mapping");
    c->mapping = mapping;
    return POLARBP_OK;
}

int polarbp_get_thread_mapping(const polarbp_code* c, int* mapping)
{
    if (!c || !mapping) return fail(POLARBP_ERR_ARG, "NULL argument");
    *mapping = c->mapping;
    return POLARBP_OK;
}

int polarbp_decode_segments(const polarbp_segment* segs, int nseg, int max_iter, float scale, int stop_mode,
                            int freeze_mode, void* workspace, size_t workspace_bytes, void* stream)
{
    polarbp::SegArgs args[13];
    int rc = group_segments(segs, nseg, max_iter, scale, stop_mode, freeze_mode, workspace, workspace_bytes, true, args);
    if (rc != POLARBP_OK) return rc;
    SideResources* side = nullptr;
    rc = side_resources(&side);
    if (rc != POLARBP_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(workspace, 0, kSegWorkspace, s);
    if (e != cudaSuccess) return cuda_fail(e, "segment counters");
    std::vector<int> ms;
    for (int m = 8; m <= 12; ++m)
        if (args[m].total > 0) ms.push_back(m);
    if (ms.empty()) return POLARBP_OK;
    if (ms.size() > 1) {
        e = cudaEventRecord(side->fork, s);
        for (size_t g = 1; e == cudaSuccess && g < ms.size(); ++g) e = cudaStreamWaitEvent(side->side[g - 1], side->fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "stream fork");
    }
    for (size_t g = 0; g < ms.size(); ++g) {
        const int m = ms[g];
        polarbp::SegLaunch q{};
        q.args = args[m];
        q.stop_mode = stop_mode;
        q.freeze_mode = freeze_mode;
        const polarbp_code* c0 = segs[first_of_length(segs, nseg, m)].code;
        q.cpc = c0->cpc;
        q.pipelined = c0->mapping == POLARBP_MAP_PIPELINED;
        q.sms = side->sms;
        q.stream = g == 0 ? s : side->side[g - 1];
        e = launch_persistent_m(m, q);
        if (e != cudaSuccess) return cuda_fail(e, "persistent decode launch");
    }
    for (size_t g = 1; g < ms.size(); ++g) {
        e = cudaEventRecord(side->join[g - 1], side->side[g - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, side->join[g - 1], 0);
        if (e != cudaSuccess) return cuda_fail(e, "stream join");
    }
    return POLARBP_OK;
}

int polarbp_decode_mixed(const polarbp_segment* segs, int nseg, int max_iter, float scale, int stop_mode,
                         int freeze_mode, void* workspace, size_t workspace_bytes, void* stream)
{
    polarbp::MixedArgs a{};
    polarbp::SegArgs args[13];
    int rc = group_segments(segs, nseg, max_iter, scale, stop_mode, freeze_mode, workspace, workspace_bytes, false, args);
    if (rc != POLARBP_OK) return rc;
    int top = 0;
    for (int m = 8; m <= 12; ++m) {
        a.seg[m - 8] = args[m];
        if (args[m].total > 0) top = m;
    }
    SideResources* side = nullptr;
    rc = side_resources(&side);
    if (rc != POLARBP_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(workspace, 0, kSegWorkspace, s);
    if (e != cudaSuccess) return cuda_fail(e, "segment counters");
    if (top == 0) return POLARBP_OK;
    switch (top) {
    case 8: e = polarbp::launch_mixed_m8(a, stop_mode, freeze_mode, side->sms, s); break;
    case 9: e = polarbp::launch_mixed_m9(a, stop_mode, freeze_mode, side->sms, s); break;
    case 10: e = polarbp::launch_mixed_m10(a, stop_mode, freeze_mode, side->sms, s); break;
    case 11: e = polarbp::launch_mixed_m11(a, stop_mode, freeze_mode, side->sms, s); break;
    default: e = polarbp::launch_mixed_m12(a, stop_mode, freeze_mode, side->sms, s); break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "mixed decode launch");
    return POLARBP_OK;
}

int polarbp_autotune(polarbp_code* c, int max_iter, float scale, int stop_mode, int freeze_mode, void* stream)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (c->m < 8 || c->m > 12) return fail(POLARBP_ERR_UNSUPPORTED, "autotune supports N from 256 to 4096");
    if (c->K < 1) return fail(POLARBP_ERR_ARG, "autotune needs K >= 1");
    const int B = std::max(2048, std::min(65536, (1 << 23) >> c->m));
    const size_t n = (size_t)B * c->N;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* d_llr = nullptr;
    uint8_t* d_u = nullptr;
    void* ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&d_llr, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d_u, n);
    if (e == cudaSuccess) e = cudaMalloc(&ws, kSegWorkspace);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int rc = POLARBP_OK;
    if (e != cudaSuccess) rc = (e == cudaErrorMemoryAllocation) ? fail(POLARBP_ERR_NOMEM, "autotune buffers")
                                                                 : cuda_fail(e, "autotune setup");
    const int keep = c->cpc, keep_map = c->mapping;
    int best = keep, best_map = keep_map;
    float best_ms = 3.4e38f;
    if (rc == POLARBP_OK) rc = polarbp_awgn(c, 1, 0, B, 2.5f, nullptr, d_llr, stream);
    // candidates (mapping, codewords per block); the pipelined mapping exists for freezing
    // (reading A) at N = 256 .. 4096 with one codeword per block
    const bool pipe_ok = freeze_mode == POLARBP_FREEZE_CSFG && c->m <= 12;
    const std::pair<int, int> cands[] = {{POLARBP_MAP_PIPELINED, 1}, {POLARBP_MAP_BLOCK, 1}, {POLARBP_MAP_BLOCK, 2},
                                         {POLARBP_MAP_BLOCK, 4}};
    for (const auto& cand : cands) {
        const int map = cand.first, cpc = cand.second;
        if (rc != POLARBP_OK) break;
        if (map == POLARBP_MAP_PIPELINED && !pipe_ok) continue;
        if (!polarbp::persistent_supported(c->m, cpc)) continue;
        c->cpc = cpc;
        c->mapping = map;
        polarbp_segment sg{c, d_llr, d_u, nullptr, nullptr, B};
        rc = polarbp_decode_segments(&sg, 1, max_iter, scale, stop_mode, freeze_mode, ws, kSegWorkspace, stream);
        if (rc != POLARBP_OK) break;
        e = cudaEventRecord(e0, s);
        for (int rep = 0; e == cudaSuccess && rep < 3; ++rep) {
            rc = polarbp_decode_segments(&sg, 1, max_iter, scale, stop_mode, freeze_mode, ws, kSegWorkspace, stream);
            if (rc != POLARBP_OK) break;
        }
        if (rc != POLARBP_OK) break;
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "autotune timing");
            break;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = cpc;
            best_map = map;
        }
    }
    c->cpc = rc == POLARBP_OK ? best : keep;
    c->mapping = rc == POLARBP_OK ? best_map : keep_map;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_llr);
    cudaFree(d_u);
    cudaFree(ws);
    return rc;
}

int polarbp_awgn_ebn0(const polarbp_code* c, uint64_t seed, uint64_t first_codeword, int batch, const float* ebn0_db,
                      uint8_t* u, float* llr, void* stream)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    if (batch < 0) return fail(POLARBP_ERR_ARG, "batch must be >= 0");
    if (c->K < 1) return fail(POLARBP_ERR_ARG, "the channel needs K >= 1 (rate > 0)");
    if (batch == 0) return POLARBP_OK;
    if (!llr || !ebn0_db) return fail(POLARBP_ERR_ARG, "llr and ebn0_db must be device pointers");
    int rc = check_device(c);
    if (rc != POLARBP_OK) return rc;
    const int threads = c->N < 256 ? (c->N < 32 ? 32 : c->N) : 256;
    awgn_kernel<<<batch, threads, c->N, static_cast<cudaStream_t>(stream)>>>(
        c->d_frozen, c->N, c->m, seed, first_codeword, 0.f, ebn0_db, (float)c->K / (float)c->N, c->bitrev, u, llr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "awgn launch");
    return POLARBP_OK;
}

int polarbp_get_status(const polarbp_code* c, void* stream)
{
    if (!c) return fail(POLARBP_ERR_ARG, "code handle is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned int h[polarbp::kStatusWords] = {};
    cudaError_t e = cudaMemcpyAsync(h, c->d_status, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof h, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "get_status");
    if (h[0] & polarbp::kStatusRedzone) {
        static const char* const layouts[] = {"?", "SmemLayout", "PipeLayout", "CLayout"};
        const unsigned lay = h[2] >> 8;
        return fail(POLARBP_ERR_CHECK, std::to_string(h[1]) + " redzone words changed; first in " +
                                           layouts[lay < 4 ? lay : 0] + " redzone " + std::to_string(h[2] & 0xffu) +
                                           " at byte " + std::to_string(h[3]));
    }
    if (h[0] & 1u) return fail(POLARBP_ERR_NONFINITE, "a decode saw a non-finite channel LLR");
    return POLARBP_OK;
}

const char* polarbp_last_error(void) { return g_last_error.c_str(); }

const char* polarbp_version(void) { return polarbp::kChecked ? "polarbp 0.1 (sm_103a) checked" : "polarbp 0.1 (sm_103a)"; }

}  // extern "C"
