/*
 * polarbp.h -- C ABI of the GB300 belief-propagation polar decoder.
 *
 * Method: S. M. Abbas, Y. Fan, J. Chen, C.-Y. Tsui, "Low Complexity Belief
 * Propagation Polar Code Decoder", arXiv 1505.04979.
 *
 * Conventions shared by every entry point:
 *   - N = 2^m code length, K information bits; the frozen set A^c has N-K
 *     positions (Sec. II).
 *   - Device pointers are CUDA global-memory pointers the caller allocated on
 *     the current device; the library never frees them.  Host pointers are
 *     plain host memory (pinned memory makes the copies asynchronous).
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Device-side work is asynchronous on that stream unless an entry
 *     point says it synchronises.
 *   - Every call returns a polarbp_status; nothing throws across the ABI.  The
 *     message of the last failure on the calling thread is in
 *     polarbp_last_error().
 *   - Layouts are row-major: [batch][N] for per-position arrays, [batch] for
 *     per-codeword scalars.  Bits are one byte each (0 or 1).
 */
#ifndef POLARBP_H
#define POLARBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum polarbp_status {
    POLARBP_OK = 0,
    POLARBP_ERR_ARG = 1,         /* an argument is out of range or NULL where not allowed */
    POLARBP_ERR_NONFINITE = 2,   /* a decode saw a NaN or infinite channel LLR */
    POLARBP_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    POLARBP_ERR_TIMEOUT = 4,     /* reserved for a device-side bounded wait; no kernel of the library
                                    spins on a flag (work queues use atomics, the cluster decoder
                                    hardware cluster barriers), so no call returns it */
    POLARBP_ERR_NOMEM = 5,       /* a library allocation failed */
    POLARBP_ERR_UNSUPPORTED = 6, /* valid arguments the library has no kernel for */
    POLARBP_ERR_CHECK = 7        /* checked build only: a decode stored into a shared-memory
                                    redzone, i.e. outside the region it meant (polarbp_get_status) */
} polarbp_status;

typedef enum polarbp_stop_mode {
    POLARBP_STOP_NONE = 0,    /* run exactly max_iter iterations (baseline BP)            */
    POLARBP_STOP_GMATRIX = 1  /* stop once u_hat G == x_hat (the G-matrix early stop, Sec. I) */
} polarbp_stop_mode;

typedef enum polarbp_freeze_mode {
    POLARBP_FREEZE_OFF = 0,        /* every PE of every stage runs every iteration */
    POLARBP_FREEZE_CSFG = 1,       /* connected-sub-factor-graph freezing, Sec. III */
    POLARBP_FREEZE_CSFG_MULTI = 2  /* a variant reading of Sec. III: checks continue along a stage */
} polarbp_freeze_mode;

/* How the threads of a block share one codeword's work when freezing
 * (POLARBP_FREEZE_CSFG) at N = 256 .. 4096.  Decisions, iteration and PE counts
 * are the same under both; only the schedule differs. */
typedef enum polarbp_thread_mapping {
    POLARBP_MAP_PIPELINED = 0,  /* N/8 sweep threads plus one checker warp that runs the CSFG
                                   checks of iteration t while the sweep runs iteration t+1
                                   (one codeword per block); the default for N >= 1024 */
    POLARBP_MAP_BLOCK = 1       /* N/8 threads that sweep, then one of their warps checks while
                                   the others wait (1, 2 or 4 codewords per block); the default
                                   below N = 1024 */
} polarbp_thread_mapping;

/* Opaque code handle: the frozen set plus its device-side tables.  Owned by the
 * library; create with polarbp_construct, release with polarbp_destroy. */
typedef struct polarbp_code polarbp_code;

/*
 * polarbp_construct -- build an (N, K) polar code (Sec. II).
 *   N            code length, a power of two, 2 <= N <= 32768.
 *   K            number of information bits, 0 <= K <= N.
 *   frozen_mask  host array of N bytes, 1 = frozen, or NULL.  With NULL the
 *                frozen set is the N-K least reliable synthetic channels of a
 *                binary erasure channel with erasure probability z0 (the
 *                Bhattacharyya recursion; the paper does not state its
 *                construction).  When given, its popcount must be N-K.
 *   z0           erasure probability in (0, 1); ignored when frozen_mask != NULL.
 *   out          receives the handle.
 * Allocates the handle and a few KB of device memory on the current device,
 * and creates three non-blocking CUDA streams and four events there for
 * polarbp_decode_host's pipeline.
 * Errors: POLARBP_ERR_ARG, POLARBP_ERR_NOMEM, POLARBP_ERR_CUDA.
 */
int polarbp_construct(int N, int K, const uint8_t* frozen_mask, double z0, polarbp_code** out);

/*
 * polarbp_frozen_set -- host-only: the frozen set polarbp_construct builds when
 * it is given no mask (N-K least reliable BEC(z0) synthetic channels, Sec. II).
 * frozen_mask receives N bytes (1 = frozen).  Touches no GPU.
 * Errors: POLARBP_ERR_ARG.
 */
int polarbp_frozen_set(int N, int K, double z0, uint8_t* frozen_mask);

/* polarbp_destroy -- release a handle (NULL is ignored).  Synchronises the
 * handle's device (making it current for the call and restoring the caller's
 * device afterwards) before freeing its tables, streams and events. */
void polarbp_destroy(polarbp_code* code);

/* polarbp_code_info -- N, K and m = log2 N of a handle (any out pointer may be NULL). */
int polarbp_code_info(const polarbp_code* code, int* N, int* K, int* m);

/*
 * polarbp_set_bit_reversed -- codeword order of a code handle (Sec. II; Arikan's
 * generator B_N F^{(x)m}).  With on = 1 the codeword positions travel in
 * bit-reversed order: channel position i carries code position rev(i), the
 * m-bit reversal of i, i.e. x = u B_N F^{(x)m} = (u F^{(x)m}) B_N, since B_N
 * commutes with F^{(x)m}.  The frozen set, the source bits u_hat and every
 * decoding result keep the natural source order; polarbp_encode writes x in
 * channel order, polarbp_awgn sends channel order, and polarbp_decode (all its
 * forms, polarbp_decode_host and polarbp_decode_segments) reads LLRs in channel
 * order.  The variant decoders (polarbp_decode_flooding, polarbp_decode_quantized,
 * polarbp_wms_*) reject such a handle with POLARBP_ERR_UNSUPPORTED.  Default 0
 * (natural order, the paper's Fig. 1).  Not to be changed while work that uses
 * the handle is in flight.
 * Errors: POLARBP_ERR_ARG (NULL handle, on not 0 or 1).
 */
int polarbp_set_bit_reversed(polarbp_code* code, int on);
/* polarbp_get_bit_reversed -- the handle's codeword order (0 natural, 1 bit-reversed). */
int polarbp_get_bit_reversed(const polarbp_code* code, int* on);

/* polarbp_get_frozen_mask -- copy the frozen set to a host array of N bytes (1 = frozen). */
int polarbp_get_frozen_mask(const polarbp_code* code, uint8_t* frozen_mask);

/*
 * polarbp_encode -- x = u F^{(x)m} over GF(2), natural index order (Sec. II, Fig. 1).
 *   u  device [batch][N] source bits (frozen positions are not forced to 0).
 *   x  device [batch][N] codeword bits; may not alias u.
 * Errors: POLARBP_ERR_ARG, POLARBP_ERR_CUDA.
 */
int polarbp_encode(const polarbp_code* code, const uint8_t* u, uint8_t* x, int batch, void* stream);

/*
 * polarbp_decode -- scaled min-sum belief-propagation decoding on the m-stage
 * factor graph (Sec. II-A, Eq. (1)): one left-to-right sweep of PE stages per
 * iteration, R messages of the current and L messages of the previous
 * iteration, L initialised to 0 inside the graph and to the prior (+inf on
 * frozen positions, 0 elsewhere) on the source side.
 *   llr          device [batch][N] channel LLRs, log P(x=0)/P(x=1), binary32.
 *   batch        number of codewords, >= 0 (0 is a no-op).
 *   max_iter     iteration cap, >= 1.
 *   scale        the min-sum scaling alpha (0.9375 in Sec. IV), finite and > 0.
 *   stop_mode    POLARBP_STOP_NONE or POLARBP_STOP_GMATRIX: after every
 *                iteration, stop when u_hat . F^{(x)m} equals HD(R + L) on the
 *                channel side; u_hat takes HD(R + L) on the source side, 0 on
 *                frozen positions and the stored decision on frozen CSFGs.
 *   freeze_mode  POLARBP_FREEZE_OFF or POLARBP_FREEZE_CSFG (Sec. III): after PE
 *                stage j-1 the first not-yet-covered CSFG of stage j is checked
 *                with Eqs. (2)-(4); when it passes, its decision is stored, its
 *                right-to-left messages are fixed to (-1)^x_hat * inf, and its
 *                PEs are skipped from then on.  A CSFG whose two halves are
 *                covered is frozen too.  Decoding ends once every position is
 *                covered, at the G-matrix stop, or at max_iter.
 *                POLARBP_FREEZE_CSFG_MULTI reads Sec. III's "move to the next
 *                stage" as coming only after a failing check: a CSFG that passes
 *                is frozen and the next CSFG of the same stage is checked at
 *                once, on the same R, until one fails.  It is a variant for
 *                comparison: a CSFG checked before its left neighbours' feedback
 *                has reached it misses the successive-cancellation-like
 *                decision reading A gives it, and FER rises 13- to 160-fold
 *                at 2.5-3.5 dB on the (1024,512) code;
 *                N <= 4096, polarbp_decode and polarbp_decode_trace only.
 *   u_hat        device [batch][N] decoded source bits (0 on frozen positions).
 *   iterations   device [batch] int32 iterations run, or NULL.
 *   pe_updates   device [batch] int64 PE updates executed, counted as in
 *                Sec. IV (each active PE of each iteration counts once), or NULL.
 * Supported N: 2..32768.  Up to 4096 one thread block decodes a codeword with
 * every message on chip; 8192, 16384 and 32768 run one codeword per cluster of
 * 2, 4 or 8 thread blocks, each holding 4096 positions of every message column
 * and reading its partners' columns through distributed shared memory.
 * A NaN or infinite LLR is recorded in the handle's status word; read it with
 * polarbp_get_status.  Errors: POLARBP_ERR_ARG, POLARBP_ERR_UNSUPPORTED,
 * POLARBP_ERR_CUDA (launch failure).
 */
int polarbp_decode(const polarbp_code* code, const float* llr, int batch, int max_iter, float scale,
                   int stop_mode, int freeze_mode, uint8_t* u_hat, int32_t* iterations, int64_t* pe_updates,
                   void* stream);

/*
 * polarbp_decode_trace -- polarbp_decode plus the message planes after every
 * iteration, for checking against a reference implementation.  Same
 * arguments, plus device buffers:
 *   trace_L, trace_R  [batch][max_iter][m+1][N] binary32: L and R of node
 *                     columns 0..m (column 0 = channel side) at the end of each
 *                     iteration.  Entries inside covered CSFGs are unspecified.
 *                     Iterations after the stop are left untouched.
 *   trace_P           [batch][max_iter] int32: length of the covered prefix of
 *                     source positions at the end of each iteration.
 * Slow (every message goes to global memory); N <= 32768.
 */
int polarbp_decode_trace(const polarbp_code* code, const float* llr, int batch, int max_iter, float scale,
                         int stop_mode, int freeze_mode, uint8_t* u_hat, int32_t* iterations,
                         int64_t* pe_updates, float* trace_L, float* trace_R, int32_t* trace_P, void* stream);

/*
 * polarbp_decode_flooding -- BP decoding under the true flooding schedule, a
 * variant beside the left-to-right sweep of Eq. (1) (Sec. II-A): in every
 * iteration every PE of every stage takes both its L and its R inputs from
 * the previous iteration, and all PEs update together.  The PE update, the
 * scaling, the prior (+inf on frozen positions, 0 elsewhere), the zero start
 * of interior messages, the G-matrix stop and the output are those of
 * polarbp_decode without freezing; CSFG freezing (Sec. III) is defined on the
 * sweep and is not offered here.
 *   llr, batch, max_iter, scale, u_hat, iterations, pe_updates
 *                    as polarbp_decode (device buffers; iterations and
 *                    pe_updates may be NULL; pe_updates = iterations m N/2).
 *   stop_mode        POLARBP_STOP_NONE or POLARBP_STOP_GMATRIX.
 *   trace_L, trace_R NULL, or both [batch][max_iter][m+1][N] binary32 device
 *                    buffers receiving the planes after every iteration
 *                    (iterations after the stop are left untouched).
 * N <= 1024 (the planes of one codeword, 8 (m+1) N bytes, sit in shared
 * memory); larger codes return POLARBP_ERR_UNSUPPORTED.  Non-finite LLRs are
 * recorded in the status word.  Errors: POLARBP_ERR_ARG,
 * POLARBP_ERR_UNSUPPORTED, POLARBP_ERR_CUDA.
 */
int polarbp_decode_flooding(const polarbp_code* code, const float* llr, int batch, int max_iter, float scale,
                            int stop_mode, uint8_t* u_hat, int32_t* iterations, int64_t* pe_updates,
                            float* trace_L, float* trace_R, void* stream);

/*
 * polarbp_decode_quantized -- BP decoding with quantised messages, a variant
 * for fixed-point hardware (Sec. V names a VLSI architecture as future work).
 * Eq. (1) under the sweep schedule of polarbp_decode, without freezing, with
 * 16-bit saturating integer messages in [-32767, 32767]:
 *   channel values  q = clamp(rint(llr * 2^frac_bits)), round half to even;
 *   sums            clamped to the range, whose ends stand for +-inf;
 *   scaling         alpha = alpha_16 / 16, f(x, y) =
 *                   sign(x) sign(y) ((alpha_16 min(|x|, |y|) + 8) >> 4);
 *   prior           +32767 on frozen positions, 0 elsewhere.
 *   llr, batch, max_iter, stop_mode, u_hat, iterations, pe_updates
 *                    as polarbp_decode (stop_mode NONE or GMATRIX;
 *                    pe_updates = iterations m N/2).
 *   alpha_16         1..16 (15 gives the paper's 0.9375).
 *   frac_bits        0..8 fractional bits of the channel values.
 *   trace_L, trace_R NULL, or both [batch][max_iter][m+1][N] int16 device
 *                    buffers receiving the planes after every iteration.
 * N <= 1024 (the int16 planes of a codeword, 4 (m+1) N bytes, sit in shared
 * memory).  Every value is an exact integer.  Non-finite LLRs are recorded in
 * the status word.  Errors: POLARBP_ERR_ARG, POLARBP_ERR_UNSUPPORTED,
 * POLARBP_ERR_CUDA.
 */
int polarbp_decode_quantized(const polarbp_code* code, const float* llr, int batch, int max_iter, int alpha_16,
                             int frac_bits, int stop_mode, uint8_t* u_hat, int32_t* iterations,
                             int64_t* pe_updates, int16_t* trace_L, int16_t* trace_R, void* stream);

/*
 * polarbp_decode_host_workspace -- bytes of device workspace polarbp_decode_host
 * needs for `batch` codewords (256-byte aligned sub-buffers).
 */
size_t polarbp_decode_host_workspace(const polarbp_code* code, int batch);

/*
 * polarbp_decode_host -- end-to-end decode from host buffers: copies llr to
 * the device workspace, decodes as polarbp_decode, copies u_hat, iterations
 * and pe_updates back, and synchronises `stream` before returning.
 *   llr, u_hat, iterations, pe_updates  host arrays with the layouts above
 *                                       (iterations / pe_updates may be NULL);
 *                                       page-locked (pinned) memory lets the
 *                                       copies overlap the decode.
 *   workspace        device buffer of at least
 *                    polarbp_decode_host_workspace(code, batch) bytes.
 * A batch of at least two chunks of 64 MiB of LLRs (32,768 codewords at
 * N = 1024) runs as a pipeline on the handle's three streams: each chunk is
 * uploaded, decoded and downloaded on one of them, so copies in both
 * directions overlap the decode of other chunks.  The streams start after the
 * work already queued on `stream`, and `stream` waits for them before the
 * call synchronises it.  Host threads that share a handle are serialised
 * while they queue a pipeline.  Smaller batches run as one upload, decode and
 * download on `stream`.  Results do not depend on the path.
 * The call allocates nothing.  Errors as polarbp_decode.
 */
int polarbp_decode_host(const polarbp_code* code, const float* llr, int batch, int max_iter, float scale,
                        int stop_mode, int freeze_mode, uint8_t* u_hat, int32_t* iterations,
                        int64_t* pe_updates, void* workspace, size_t workspace_bytes, void* stream);

/*
 * polarbp_awgn -- seeded synthetic channel input on the device: the setting of
 * Sec. IV (BPSK over AWGN).  For codeword c = first_codeword + b (b < batch):
 * uniform source bits (0 on frozen positions), x = u F^{(x)m}, BPSK 0 -> +1,
 * 1 -> -1, Gaussian noise of variance sigma^2 = 1 / (2 (K/N) 10^(EbN0/10)),
 * LLR = 2 y / sigma^2 in binary32.  Random words come from Philox4x32-10
 * (Salmon et al., SC'11) with key = seed and counter = (block, c low 32 bits,
 * c high 32 bits, stream), stream 1 for source bits (bit i = bit i%32 of word
 * i/32) and stream 2 for noise (Box-Muller on words 2p, 2p+1 for positions 2p,
 * 2p+1), so any codeword can be regenerated on its own.
 *   u    device [batch][N] source bits, or NULL.
 *   llr  device [batch][N] channel LLRs.
 * Requires K >= 1.  Errors: POLARBP_ERR_ARG, POLARBP_ERR_CUDA.
 */
int polarbp_awgn(const polarbp_code* code, uint64_t seed, uint64_t first_codeword, int batch, float ebn0_db,
                 uint8_t* u, float* llr, void* stream);

/*
 * polarbp_decode_host_noalloc -- polarbp_decode_host without a caller-supplied
 * workspace, for callers that may not allocate device memory: real-time
 * receive chains that forbid cudaMalloc once running (it can synchronise the
 * device and take milliseconds), and plug-ins whose host application owns all
 * device memory.  The paper has no counterpart; this is a deployment variant.
 *
 * The staging buffers live in one fixed array of POLARBP_NOALLOC_SCRATCH_BYTES
 * in device global memory, part of this library; every GPU that loads the
 * library holds it until the process exits.  The call allocates nothing.
 *   Arguments and results are those of polarbp_decode_host (host arrays).
 *   batch must satisfy polarbp_decode_host_workspace(code, batch) <=
 *   POLARBP_NOALLOC_SCRATCH_BYTES (about 3,200 codewords at N = 1024);
 *   larger batches return POLARBP_ERR_ARG with the limit in the message.
 * The current device must be the handle's (POLARBP_ERR_ARG otherwise, before
 * anything is enqueued).  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and keeps it
 * for the life of the process; make that first call before any stream capture.
 * cudaDeviceReset invalidates that address together with every code handle of
 * the device: after a reset, call nothing in this library on that device.  All
 * calls share the one array and leave the last call's contents in it; nothing
 * in it needs to start at zero (each call writes every byte it reads).  Calls
 * that overlap on the GPU -- on different streams or host threads at the same
 * time on the same device -- race on the array: serialise them.  Synchronises
 * `stream` before returning.
 */
#define POLARBP_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int polarbp_decode_host_noalloc(const polarbp_code* code, const float* llr, int batch, int max_iter, float scale,
                                int stop_mode, int freeze_mode, uint8_t* u_hat, int32_t* iterations,
                                int64_t* pe_updates, void* stream);

/*
 * A run of codewords that share one code, for polarbp_decode_segments.
 *   code        code of every codeword of the run; N >= 256.
 *   llr         device [count][N] channel LLRs.
 *   u_hat       device [count][N] decoded source bits.
 *   iterations  device [count] int32, or NULL; pe_updates device [count] int64, or NULL.
 */
typedef struct polarbp_segment {
    const polarbp_code* code;
    const float* llr;
    uint8_t* u_hat;
    int32_t* iterations;
    int64_t* pe_updates;
    int count;
} polarbp_segment;

/* polarbp_decode_segments_workspace -- device workspace bytes polarbp_decode_segments needs (queue counters). */
size_t polarbp_decode_segments_workspace(void);

/*
 * polarbp_decode_segments -- decode a mixed stream of codewords of different
 * lengths and rates (the same decode as polarbp_decode, per codeword) with one
 * persistent launch per code length.  Each block holds the code's
 * codewords-per-block groups of threads; a group takes the next codeword from
 * a device counter, stops it at its own G-matrix stop or freeze completion,
 * then takes the next, so codewords retire independently.  The launches for
 * different lengths run concurrently on library-owned side streams joined back
 * to `stream`; the whole call may be captured into a CUDA graph (call it once
 * uncaptured first: the first call per kernel sets attributes and queries
 * occupancy).
 *   segs, nseg   runs of codewords; at most 8 runs per code length, N in {256 .. 4096}.
 *   workspace    device buffer of polarbp_decode_segments_workspace() bytes
 *                (counters; zeroed by the call).  Calls sharing a workspace must
 *                not overlap on the GPU.
 * A non-finite LLR sets the status word of its own segment's code (read with
 * polarbp_get_status on that code).
 * Errors: POLARBP_ERR_ARG, POLARBP_ERR_UNSUPPORTED (N < 256 or > 4096), POLARBP_ERR_CUDA.
 */
int polarbp_decode_segments(const polarbp_segment* segs, int nseg, int max_iter, float scale, int stop_mode,
                            int freeze_mode, void* workspace, size_t workspace_bytes, void* stream);

/*
 * polarbp_decode_mixed -- the decode of polarbp_decode_segments (Eq. (1) of Sec.
 * II-A per codeword, G-matrix stop, CSFG freezing of Sec. III) in ONE persistent
 * launch over every code length of the stream.  A block has the thread count of
 * the longest length present (N/8 threads, at least a warp) and drains the
 * per-length device queues longest first; when a length's queue is empty, each
 * group of threads splits into two groups that take codewords of half that
 * length in the two halves of its shared memory, down to one warp per N = 256
 * codeword.  Codewords retire at their own stop, independently of the others.
 * With freezing and N = 4096 the longest length, the block has one warp more and
 * decodes the N = 4096 codewords pipelined (a checker warp beside the sweep);
 * every other length runs in the block mapping.  The codewords-per-block and
 * thread-mapping settings of the codes are not used.  The call may be
 * captured into a CUDA graph after one uncaptured call (the first call per
 * kernel sets attributes and queries occupancy).
 *   segs, nseg, max_iter, scale, stop_mode, freeze_mode: as polarbp_decode_segments
 *                (at most 8 runs per code length, N in {256 .. 4096}).
 *   workspace    device buffer of polarbp_decode_segments_workspace() bytes
 *                (counters; zeroed by the call, on `stream`).  Calls sharing a
 *                workspace must not overlap on the GPU.
 *   stream       the launch's stream; nothing runs on other streams.
 * Output and iteration / PE counts are those of polarbp_decode, codeword by
 * codeword; a non-finite LLR sets the status word of its own segment's code.
 * Errors: POLARBP_ERR_ARG, POLARBP_ERR_UNSUPPORTED (N < 256 or > 4096), POLARBP_ERR_CUDA.
 */
int polarbp_decode_mixed(const polarbp_segment* segs, int nseg, int max_iter, float scale, int stop_mode,
                         int freeze_mode, void* workspace, size_t workspace_bytes, void* stream);

/* polarbp_set_codewords_per_block / polarbp_get_codewords_per_block -- codewords
 * decoded side by side by one block of the persistent launch (1, 2 or 4, as
 * thread and shared-memory limits allow for the code length). */
int polarbp_set_codewords_per_block(polarbp_code* code, int codewords_per_block);
int polarbp_get_codewords_per_block(const polarbp_code* code, int* codewords_per_block);

/* polarbp_set_thread_mapping / polarbp_get_thread_mapping -- the thread mapping
 * (polarbp_thread_mapping) that polarbp_decode, polarbp_decode_host and
 * polarbp_decode_segments use for this code when freezing at N = 256 .. 4096.
 * The pipelined mapping holds one codeword per block: with codewords per block
 * above 1 the persistent launch takes the block mapping.  polarbp_decode_mixed
 * does not use this setting (it fixes the mapping per length).  Errors:
 * POLARBP_ERR_ARG (NULL handle, unknown mapping). */
int polarbp_set_thread_mapping(polarbp_code* code, int mapping);
int polarbp_get_thread_mapping(const polarbp_code* code, int* mapping);

/*
 * polarbp_autotune -- time the persistent decode of a synthetic batch
 * (BPSK/AWGN at 2.5 dB, about 8M LLRs) for every admissible thread mapping and
 * codewords-per-block value with the given decode settings (the pipelined
 * mapping with one codeword per block, and the block mapping with 1, 2 or 4,
 * as the code length admits) and keep the fastest pair in the handle.
 * Allocates and frees temporary device memory; synchronises `stream`.  The
 * handle's settings change while it runs: decode nothing with this handle from
 * another thread meanwhile.  On an error the previous settings are restored.
 * Errors: POLARBP_ERR_ARG (K = 0), POLARBP_ERR_UNSUPPORTED, POLARBP_ERR_NOMEM, POLARBP_ERR_CUDA.
 */
int polarbp_autotune(polarbp_code* code, int max_iter, float scale, int stop_mode, int freeze_mode, void* stream);

/*
 * polarbp_awgn_ebn0 -- polarbp_awgn with one Eb/N0 per codeword:
 *   ebn0_db  device [batch] float, the Eb/N0 (dB) of codeword first_codeword + b.
 * The noise words and source bits are those of polarbp_awgn.
 */
int polarbp_awgn_ebn0(const polarbp_code* code, uint64_t seed, uint64_t first_codeword, int batch,
                      const float* ebn0_db, uint8_t* u, float* llr, void* stream);

/*
 * Weighted min-sum (trainable scalings).  Eq. (1) with alpha replaced by one
 * weight per (iteration t, stage s, PE p), `iterations` unrolled iterations
 * with the schedule of polarbp_decode, no stop and no freezing.  PE p of stage
 * s pairs positions a and a + 2^(m-1-s), p = (a >> (m-s)) 2^(m-1-s) +
 * (a mod 2^(m-1-s)).  Supported N: 2 .. 1024.
 *   weights   device [iterations][m][N/2] float, weight (t, s, p) at (t m + s) N/2 + p.
 *   out       device [batch][N] soft outputs R[m] + L[m] after the last
 *             iteration (+inf on frozen positions: the prior).
 *   checkpoint_every  k >= 1.  k = 1: the forward stores both message planes
 *             after every iteration and the backward reads them back.  k > 1:
 *             the forward stores only the state one iteration hands to the next
 *             (L columns 1..m-1) after iterations k-1, 2k-1, ...; the backward
 *             recomputes the iterations in between in shared memory with the
 *             forward's arithmetic.  The results do not depend on k; k trades
 *             workspace for recomputation.  k above `iterations` acts as
 *             `iterations`.  With k > 1 the backward holds 4 + k message planes
 *             of (m+1) N floats per block: k up to 52 at N = 128, 21 at N = 256,
 *             7 at N = 512, 1 at N = 1024 (POLARBP_ERR_UNSUPPORTED beyond).  The
 *             forward and the backward of one batch take the same k.
 *   workspace device buffer of polarbp_wms_workspace(code, batch, iterations,
 *             checkpoint_every) bytes: the forward writes its checkpoints there
 *             and the backward of the same batch reads them; keep it unchanged
 *             between the two.
 */
size_t polarbp_wms_workspace(const polarbp_code* code, int batch, int iterations, int checkpoint_every);
int polarbp_wms_forward(const polarbp_code* code, const float* llr, int batch, int iterations, int checkpoint_every,
                        const float* weights, float* out, void* workspace, size_t workspace_bytes, void* stream);

/*
 * polarbp_wms_backward -- gradients of a loss through polarbp_wms_forward.
 *   dout      device [batch][N]: dLoss/d out (entries at frozen positions are ignored).
 *   dweights  device [iterations][m][N/2]: dLoss/d weights, summed over the batch
 *             in codeword order (overwritten).
 *   dllr      device [batch][N]: dLoss/d llr (overwritten).
 * min is differentiated towards its smaller argument (ties: the first), sign
 * as a constant; +-inf messages (built from the frozen prior) are constants.
 */
int polarbp_wms_backward(const polarbp_code* code, const float* llr, int batch, int iterations, int checkpoint_every,
                         const float* weights, const float* dout, float* dweights, float* dllr, void* workspace,
                         size_t workspace_bytes, void* stream);

/*
 * polarbp_get_status -- read and clear the handle's device status words.  Waits
 * for `stream`.  Returns POLARBP_ERR_NONFINITE when a decode since the last
 * call saw a non-finite LLR, else POLARBP_OK (or POLARBP_ERR_CUDA).
 * In the checked build (compiled with POLARBP_CHECKED; polarbp_version then
 * ends in "checked"), the shared memory of every decode of polarbp_decode,
 * _trace, _host, _segments and _mixed has a 256-byte redzone before its first
 * region and after each region, filled before the decode's first store and
 * compared after its last; a changed redzone word makes this call return
 * POLARBP_ERR_CHECK (before POLARBP_ERR_NONFINITE), with a message that gives
 * the number of changed words and the layout, redzone and byte offset of the
 * first.  The default build has no redzones and never returns it.
 */
int polarbp_get_status(const polarbp_code* code, void* stream);

/* polarbp_last_error -- message of the calling thread's last failure ("" if none). */
const char* polarbp_last_error(void);

/* polarbp_version -- library version string ("... checked" for the checked build). */
const char* polarbp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* POLARBP_H */
