/*
 * polar_oracle.c -- plain, slow CPU oracle for belief-propagation (BP)
 * decoding of polar codes with the G-matrix early stop and the paper's
 * connected-sub-factor-graph (CSFG) freezing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The GPU library shares no
 * code, header, table or helper with it.
 *
 * Paper: S. M. Abbas, Y. Fan, J. Chen, C.-Y. Tsui, "Low Complexity Belief
 * Propagation Polar Code Decoder", arXiv 1505.04979.
 *
 *   code, frozen set, x = u F^{(x)m} .......... Sec. II
 *   factor graph, min-sum PE update ............ Sec. II-A, Eq. (1)
 *   CSFG, freezing order ....................... Sec. III
 *   hard decision / inverse / frozen test ...... Sec. III, Eqs. (2)-(4), Lemma 1
 *   +-infinity feedback of a frozen CSFG ....... Sec. III (equation after Lemma 1)
 *   computation count .......................... Sec. IV
 *
 * Index conventions (0-based).  Node columns c = 0..m; column 0 is the channel
 * side (the paper's stage 1) and column m the source side (the paper's stage
 * m+1).  PE stage s = 0..m-1 joins columns s and s+1 (the paper's stage
 * j = s+1) and pairs node a with node b = a + 2^(m-1-s).  Level j = 1..m holds
 * the 2^j CSFGs of the paper's stage j, each of size 2^(m-j); CSFG k of level
 * j covers source indices [k 2^(m-j), (k+1) 2^(m-j)) and is fed by R[j].
 *
 * Readings of the paper that this file fixes (the kernels follow the same
 * readings):
 *   R1  one left-to-right sweep per iteration; R from this iteration, L from
 *       the previous one, exactly as Eq. (1) is written (Sec. II-A).
 *   R2  interior L messages start at 0; L[m] is the prior: +inf on frozen
 *       positions, 0 on information positions.
 *   R3  level j is checked right after PE stage j-1 (it consumes R[j]), and
 *       only its first CSFG that is not yet covered is checked, once per
 *       iteration (Sec. III; Fig. 5 captions).  Reading B, offered as a
 *       variant (freeze = 2), keeps checking along the level, on the same
 *       R[j], while the checks pass.
 *   R4  a CSFG is "covered" when it, or a CSFG containing it, is frozen.  A
 *       CSFG whose two halves are both covered is frozen at that moment, with
 *       the hard decision obtained by re-encoding the stored source bits of
 *       its range (the +-inf messages its own PEs would emit).
 *   R5  the PEs of stage s >= 1 inside a covered level-s CSFG are skipped and
 *       not counted; stage 0 always runs.
 *   R6  Eq. (2) maps values >= 0 (including -0) to 0.
 *   R7  G-matrix stop: u_hat (stored bits on covered indices, HD(R[m]+L[m])
 *       elsewhere, 0 on frozen indices) re-encoded must equal HD(R[0]+L[0]).
 *   R8  freeze-only decoding ends when every index is covered; the output is
 *       the stored bits on covered indices and HD(R[m]+L[m]) elsewhere.
 *
 * Precision.  By default every message is an IEEE double.  With fp32 != 0
 * every arithmetic result is rounded to binary32 right after it is formed,
 * which reproduces single-precision arithmetic operation by operation (sums of
 * two binary32 values are exact or correctly rounded once in binary64, and
 * rounding binary64 to binary32 after a single add or multiply is innocuous);
 * this lets hard decisions be compared in the precision a GPU kernel uses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOMEM (-2)
#define ORC_ERR_PREFIX (-3)
#define ORC_ERR_NAN (-4)

static int ilog2_exact(int n)
{
    int m = 0;
    if (n < 1) return -1;
    while ((1 << m) < n) ++m;
    return ((1 << m) == n) ? m : -1;
}

/* ------------------------------------------------------------------------ */
/* Sec. II: frozen set.  The paper does not say how the reliable positions   */
/* are found; the Bhattacharyya recursion of a binary erasure channel with    */
/* erasure probability z0 is used.  A channel with parameter z splits into    */
/* a worse one, 2z - z^2, and a better one, z^2; after m splits, position i   */
/* carries the channel whose split decisions are the bits of i read from the  */
/* most significant bit (first split) to the least significant (last split),  */
/* 0 = worse, 1 = better.  The recursion runs on (ln z, ln(1 - z)) so that    */
/* neither tail rounds to 0 or 1:                                             */
/*   worse:  ln z' = ln z + log1p(1 - z),   ln(1 - z') = 2 ln(1 - z)           */
/*   better: ln z' = 2 ln z,                ln(1 - z') = ln(1 - z) + log1p(z)  */
/* ------------------------------------------------------------------------ */
int orc_bec_lnz(int N, double z0, double* ln_z, double* ln_1mz)
{
    int m = ilog2_exact(N);
    if (m < 0 || !(z0 > 0.0 && z0 < 1.0) || !ln_z || !ln_1mz) return ORC_ERR_ARG;
    ln_z[0] = log(z0);
    ln_1mz[0] = log1p(-z0);
    for (int level = 0; level < m; ++level) {
        int count = 1 << level;
        /* walk backwards so that entry k is read before 2k and 2k+1 are written */
        for (int k = count - 1; k >= 0; --k) {
            double a = ln_z[k], b = ln_1mz[k];
            double worse_a = a + log1p(exp(b));
            double worse_b = 2.0 * b;
            double better_a = 2.0 * a;
            double better_b = b + log1p(exp(a));
            ln_z[2 * k] = worse_a;
            ln_1mz[2 * k] = worse_b;
            ln_z[2 * k + 1] = better_a;
            ln_1mz[2 * k + 1] = better_b;
        }
    }
    return ORC_OK;
}

typedef struct {
    double logit;
    int index;
} rank_t;

static int rank_cmp(const void* pa, const void* pb)
{
    const rank_t* a = (const rank_t*)pa;
    const rank_t* b = (const rank_t*)pb;
    if (a->logit < b->logit) return -1;
    if (a->logit > b->logit) return 1;
    /* equal reliability: the larger index counts as the more reliable one */
    return (a->index > b->index) ? -1 : (a->index < b->index);
}

/* frozen[i] = 1 for the N-K least reliable positions (largest z). */
int orc_bec_frozen(int N, int K, double z0, uint8_t* frozen)
{
    int m = ilog2_exact(N);
    if (m < 0 || K < 0 || K > N || !frozen) return ORC_ERR_ARG;
    double* a = (double*)malloc(sizeof(double) * (size_t)N);
    double* b = (double*)malloc(sizeof(double) * (size_t)N);
    rank_t* r = (rank_t*)malloc(sizeof(rank_t) * (size_t)N);
    if (!a || !b || !r) {
        free(a);
        free(b);
        free(r);
        return ORC_ERR_NOMEM;
    }
    int rc = orc_bec_lnz(N, z0, a, b);
    if (rc == ORC_OK) {
        for (int i = 0; i < N; ++i) {
            r[i].logit = a[i] - b[i]; /* ln(z / (1 - z)), increasing in z */
            r[i].index = i;
        }
        qsort(r, (size_t)N, sizeof(rank_t), rank_cmp);
        for (int i = 0; i < N; ++i) frozen[i] = 1;
        for (int i = 0; i < K; ++i) frozen[r[i].index] = 0;
    }
    free(a);
    free(b);
    free(r);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Sec. II, Eq. (3): out = in . F^{(x)k} over GF(2), n = 2^k.                 */
/* F^{(x)k} = [[F^{(x)k-1}, 0], [F^{(x)k-1}, F^{(x)k-1}]], so a row vector     */
/* [p, q] maps to [(p xor q) F^{(x)k-1}, q F^{(x)k-1}].  scratch needs n bytes.*/
/* ------------------------------------------------------------------------ */
static void polar_transform(const uint8_t* in, uint8_t* out, int n, uint8_t* scratch)
{
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    int h = n / 2;
    uint8_t* tmp = scratch;
    for (int i = 0; i < h; ++i) tmp[i] = (uint8_t)(in[i] ^ in[i + h]);
    polar_transform(tmp, out, h, scratch + h);
    polar_transform(in + h, out + h, h, scratch + h);
}

int orc_encode(int N, const uint8_t* u, uint8_t* x)
{
    if (ilog2_exact(N) < 0 || !u || !x) return ORC_ERR_ARG;
    uint8_t* scratch = (uint8_t*)malloc((size_t)N);
    uint8_t* in = (uint8_t*)malloc((size_t)N);
    if (!scratch || !in) {
        free(scratch);
        free(in);
        return ORC_ERR_NOMEM;
    }
    for (int i = 0; i < N; ++i) in[i] = (uint8_t)(u[i] & 1);
    polar_transform(in, x, N, scratch);
    free(scratch);
    free(in);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Eqs. (2)-(4) on one CSFG of size S with inputs Rin (Lemma 1: when this     */
/* returns 1, uh is the maximum-likelihood source word of the constituent     */
/* code).  xh, uh get S bytes; scratch needs S bytes.                         */
/* ------------------------------------------------------------------------ */
int orc_csfg_check(int S, const double* Rin, const uint8_t* frozen_sub, uint8_t* xh, uint8_t* uh,
                   uint8_t* scratch)
{
    for (int i = 0; i < S; ++i) xh[i] = (Rin[i] < 0.0) ? 1 : 0; /* Eq. (2) */
    polar_transform(xh, uh, S, scratch);                           /* Eq. (3) */
    for (int i = 0; i < S; ++i)
        if (frozen_sub[i] && uh[i]) return 0; /* Eq. (4) fails */
    return 1;
}

/* public wrapper with its own scratch, for the brute-force Lemma 1 test */
int orc_csfg_check_ext(int S, const double* Rin, const uint8_t* frozen_sub, uint8_t* xh, uint8_t* uh)
{
    if (ilog2_exact(S) < 0) return ORC_ERR_ARG;
    uint8_t* scratch = (uint8_t*)malloc((size_t)S);
    if (!scratch) return ORC_ERR_NOMEM;
    int r = orc_csfg_check(S, Rin, frozen_sub, xh, uh, scratch);
    free(scratch);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Decoder                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int N, m;
    int fp32;
    double alpha;
    const uint8_t* frozen;
    double* L;          /* (m+1) x N */
    double* R;          /* (m+1) x N */
    uint8_t* blk;       /* per-level frozen flags: level j block k at blk[(1<<j) + k] */
    uint8_t* ustore;    /* decided source bits of covered indices */
    uint8_t* xh;        /* N */
    uint8_t* uh;        /* N */
    uint8_t* scratch;   /* N */
    uint8_t* ubits;     /* N */
    uint8_t* xbits;     /* N */
    int64_t pe;
    double margin;
    int nan_seen;
    int rule;           /* freeze-check variant (orc_decode_rule_batch): 0 = Eqs. (2)-(4) on R */
    double theta;       /* reliability threshold of rule 2 */
    double* rl;         /* N: the messages Eq. (2) decides on under rule 1 */
} dec_t;

#define LM(d, c, i) ((d)->L[(size_t)(c) * (size_t)(d)->N + (size_t)(i)])
#define RM(d, c, i) ((d)->R[(size_t)(c) * (size_t)(d)->N + (size_t)(i)])

static double rnd(const dec_t* d, double v) { return d->fp32 ? (double)(float)v : v; }

static double sgn(double v) { return (double)((v > 0.0) - (v < 0.0)); }

/* scaled min-sum: alpha sign(x) sign(y) min(|x|, |y|)   (Eq. (1)) */
static double fms(const dec_t* d, double x, double y)
{
    return rnd(d, d->alpha * sgn(x) * sgn(y) * fmin(fabs(x), fabs(y)));
}

static void note_margin(dec_t* d, double v)
{
    double a = fabs(v);
    if (a < d->margin) d->margin = a;
}

/* A CSFG is covered when it or one of the CSFGs that contain it is frozen. */
static int covered(const dec_t* d, int j, int k)
{
    for (int jj = j; jj >= 1; --jj) {
        if (d->blk[(1 << jj) + (k >> (j - jj))]) return 1;
    }
    return 0;
}

static int index_covered(const dec_t* d, int i) { return covered(d, d->m, i); }

/* Length of the covered prefix; returns -1 when the covered set is not a prefix. */
static int covered_prefix(const dec_t* d)
{
    int P = 0;
    while (P < d->N && index_covered(d, P)) ++P;
    for (int i = P; i < d->N; ++i)
        if (index_covered(d, i)) return -1;
    return P;
}

/* Fix the feedback of a frozen CSFG: L[j][block] = (-1)^xh * inf. */
static void set_feedback(dec_t* d, int j, int base, int S, const uint8_t* xh)
{
    for (int i = 0; i < S; ++i) LM(d, j, base + i) = xh[i] ? -INFINITY : INFINITY;
}

/* Freeze CSFG (j, k) with hard decision xh and source word uh, then freeze every
 * enclosing CSFG whose two halves have become covered (reading R4). */
static void freeze_block(dec_t* d, int j, int k, const uint8_t* xh, const uint8_t* uh)
{
    int S = d->N >> j;
    int base = k * S;
    d->blk[(1 << j) + k] = 1;
    memcpy(d->ustore + base, uh, (size_t)S);
    set_feedback(d, j, base, S, xh);
    while (j > 1) {
        int sib = k ^ 1;
        if (!covered(d, j, sib)) break;
        j -= 1;
        k >>= 1;
        S = d->N >> j;
        base = k * S;
        d->blk[(1 << j) + k] = 1;
        /* the hard decision of the parent is its stored source bits re-encoded */
        polar_transform(d->ustore + base, d->xbits, S, d->scratch);
        set_feedback(d, j, base, S, d->xbits);
    }
}

/* Check the first uncovered CSFG of level j (reading R3).  With multi set
 * (reading B, a variant) a CSFG that passes is frozen and the next one of the
 * same level is checked at once, on the same R[j], until one fails or the
 * level is covered. */
static void check_level(dec_t* d, int j, int multi)
{
    int S = d->N >> j;
    int nblk = 1 << j;
    for (;;) {
        int k = 0;
        while (k < nblk && covered(d, j, k)) ++k;
        if (k == nblk) return;
        int base = k * S;
        const double* Rin = &RM(d, j, base);
        for (int i = 0; i < S; ++i) note_margin(d, Rin[i]);
        if (d->rule == 1) {
            /* variant: Eq. (2) on the a-posteriori message R + L of the CSFG's input node */
            for (int i = 0; i < S; ++i) d->rl[i] = rnd(d, Rin[i] + LM(d, j, base + i));
            Rin = d->rl;
        } else if (d->rule == 2) {
            /* variant: Eqs. (2)-(4), and only when every input is at least theta in magnitude */
            int weak = 0;
            for (int i = 0; i < S; ++i) weak |= fabs(Rin[i]) < d->theta;
            if (weak) return;
        }
        if (!orc_csfg_check(S, Rin, d->frozen + base, d->xh, d->uh, d->scratch)) return;
        freeze_block(d, j, k, d->xh, d->uh);
        if (!multi) return;
    }
}

/* PE stage s (Eq. (1)), skipping PEs inside covered CSFGs (reading R5). */
static void pe_stage(dec_t* d, int s)
{
    const int N = d->N, m = d->m;
    const int h = 1 << (m - 1 - s);
    for (int a = 0; a < N; ++a) {
        if (a & h) continue;
        if (s >= 1 && covered(d, s, a >> (m - s))) continue;
        const int b = a + h;
        const double La = LM(d, s + 1, a); /* L^{t-1}_{i,j+1}       */
        const double Lb = LM(d, s + 1, b); /* L^{t-1}_{i+2^(m-j),j+1} */
        const double Ra = RM(d, s, a);     /* R^t_{i,j}             */
        const double Rb = RM(d, s, b);     /* R^t_{i+2^(m-j),j}     */
        const double t = rnd(d, Lb + Rb);
        const double g = fms(d, La, Ra);
        const double nLa = fms(d, La, t);
        const double nLb = rnd(d, Lb + g);
        const double nRa = fms(d, Ra, t);
        const double nRb = rnd(d, Rb + g);
        if (isnan(nLa) || isnan(nLb) || isnan(nRa) || isnan(nRb)) d->nan_seen = 1;
        LM(d, s, a) = nLa;
        LM(d, s, b) = nLb;
        RM(d, s + 1, a) = nRa;
        RM(d, s + 1, b) = nRb;
        d->pe += 1;
    }
}

/* source-side decision for index i (readings R7, R8) */
static uint8_t source_bit(dec_t* d, int i, int use_store)
{
    if (use_store && index_covered(d, i)) return d->ustore[i];
    if (d->frozen[i]) return 0;
    double v = rnd(d, RM(d, d->m, i) + LM(d, d->m, i));
    note_margin(d, v);
    return (v < 0.0) ? 1 : 0;
}

/* G-matrix stop (reading R7): u_hat . G == HD(R[0] + L[0]) */
static int gmatrix_stop(dec_t* d, int use_store)
{
    const int N = d->N;
    for (int i = 0; i < N; ++i) d->ubits[i] = source_bit(d, i, use_store);
    polar_transform(d->ubits, d->uh, N, d->scratch);
    int same = 1;
    for (int i = 0; i < N; ++i) {
        double v = rnd(d, RM(d, 0, i) + LM(d, 0, i));
        note_margin(d, v);
        uint8_t x = (v < 0.0) ? 1 : 0;
        if (x != d->uh[i]) same = 0;
    }
    return same;
}

/*
 * Decode one codeword.
 *   llr        N channel LLRs, log P(x=0)/P(x=1), as binary32
 *   stop_mode  0 = fixed iterations, 1 = G-matrix stop
 *   freeze     0 = off, 1 = CSFG freezing (reading R3: one check per level per
 *              iteration), 2 = CSFG freezing under reading B (a variant: at
 *              each level, checks continue along the level while they pass)
 *   u_hat      N output bytes (0/1)
 *   iters      iterations executed; pe = PE updates executed (Sec. IV count)
 *   margin     smallest |value| a hard decision was taken on (may be NULL)
 *   cover      length of the covered prefix at the end (may be NULL)
 *   trace_L, trace_R   optional max_iter x (m+1) x N planes after each iteration
 *   trace_P    optional max_iter entries: covered-prefix length after each iteration
 *   trace_pe   optional max_iter entries: PE updates in each iteration
 * Returns ORC_OK, or a negative error code.
 */
static int decode_one(int N, const uint8_t* frozen, const float* llr, int max_iter, double alpha, int stop_mode,
                      int freeze, int fp32, uint8_t* u_hat, int32_t* iters, int64_t* pe, double* margin,
                      int32_t* cover, double* trace_L, double* trace_R, int32_t* trace_P, int64_t* trace_pe,
                      int rule, double theta);

int orc_decode(int N, const uint8_t* frozen, const float* llr, int max_iter, double alpha, int stop_mode,
               int freeze, int fp32, uint8_t* u_hat, int32_t* iters, int64_t* pe, double* margin, int32_t* cover,
               double* trace_L, double* trace_R, int32_t* trace_P, int64_t* trace_pe)
{
    return decode_one(N, frozen, llr, max_iter, alpha, stop_mode, freeze, fp32, u_hat, iters, pe, margin, cover,
                      trace_L, trace_R, trace_P, trace_pe, 0, 0.0);
}

static int decode_one(int N, const uint8_t* frozen, const float* llr, int max_iter, double alpha, int stop_mode,
                      int freeze, int fp32, uint8_t* u_hat, int32_t* iters, int64_t* pe, double* margin,
                      int32_t* cover, double* trace_L, double* trace_R, int32_t* trace_P, int64_t* trace_pe,
                      int rule, double theta)
{
    int m = ilog2_exact(N);
    if (m < 1 || !frozen || !llr || max_iter < 1 || !(alpha > 0.0) || !u_hat) return ORC_ERR_ARG;
    dec_t d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.m = m;
    d.fp32 = fp32;
    d.alpha = fp32 ? (double)(float)alpha : alpha;
    d.frozen = frozen;
    d.margin = INFINITY;
    size_t planes = (size_t)(m + 1) * (size_t)N;
    d.L = (double*)calloc(planes, sizeof(double));
    d.R = (double*)calloc(planes, sizeof(double));
    d.blk = (uint8_t*)calloc((size_t)2 * (size_t)N, 1);
    d.ustore = (uint8_t*)calloc((size_t)N, 1);
    d.xh = (uint8_t*)malloc((size_t)N);
    d.uh = (uint8_t*)malloc((size_t)N);
    d.scratch = (uint8_t*)malloc((size_t)N);
    d.ubits = (uint8_t*)malloc((size_t)N);
    d.xbits = (uint8_t*)malloc((size_t)N);
    d.rl = (double*)malloc(sizeof(double) * (size_t)N);
    d.rule = rule;
    d.theta = theta;
    int rc = ORC_OK;
    if (!d.L || !d.R || !d.blk || !d.ustore || !d.xh || !d.uh || !d.scratch || !d.ubits || !d.xbits || !d.rl) {
        rc = ORC_ERR_NOMEM;
        goto out;
    }
    /* reading R2: prior on the source side, zero elsewhere */
    for (int i = 0; i < N; ++i) LM(&d, m, i) = frozen[i] ? INFINITY : 0.0;

    int done = 0, t_done = max_iter;
    for (int t = 1; t <= max_iter && !done; ++t) {
        int64_t pe_before = d.pe;
        for (int i = 0; i < N; ++i) RM(&d, 0, i) = (double)llr[i];
        for (int s = 0; s < m; ++s) {
            if (freeze && s >= 1) {
                check_level(&d, s, freeze == 2);
                if (covered_prefix(&d) == N) {
                    done = 1;
                    break;
                }
            }
            pe_stage(&d, s);
        }
        if (!done && freeze) {
            check_level(&d, m, freeze == 2);
            if (covered_prefix(&d) == N) done = 1;
        }
        if (!done && stop_mode == 1) {
            if (gmatrix_stop(&d, freeze)) done = 1;
        }
        int P = covered_prefix(&d);
        if (P < 0) {
            rc = ORC_ERR_PREFIX;
            goto out;
        }
        if (d.nan_seen) {
            rc = ORC_ERR_NAN;
            goto out;
        }
        if (trace_L) memcpy(trace_L + (size_t)(t - 1) * planes, d.L, planes * sizeof(double));
        if (trace_R) memcpy(trace_R + (size_t)(t - 1) * planes, d.R, planes * sizeof(double));
        if (trace_P) trace_P[t - 1] = P;
        if (trace_pe) trace_pe[t - 1] = d.pe - pe_before;
        if (done) t_done = t;
    }
    for (int i = 0; i < N; ++i) u_hat[i] = source_bit(&d, i, freeze);
    if (iters) *iters = t_done;
    if (pe) *pe = d.pe;
    if (margin) *margin = d.margin;
    if (cover) *cover = covered_prefix(&d);
out:
    free(d.L);
    free(d.R);
    free(d.blk);
    free(d.ustore);
    free(d.xh);
    free(d.uh);
    free(d.scratch);
    free(d.ubits);
    free(d.xbits);
    free(d.rl);
    return rc;
}

/*
 * orc_decode_rule_batch -- reading A (freeze = 1) with a variant of the CSFG
 * check, for the comparison of freezing rules the paper leaves open (Sec. III):
 *   rule 0  Eqs. (2)-(4) on R (the reading every other entry point uses);
 *   rule 1  Eq. (2) on R + L at the CSFG's input node instead of R;
 *   rule 2  Eqs. (2)-(4) on R, and only when every |R| of the CSFG is >= theta.
 * Other arguments as orc_decode_batch (no margins, no cover).
 */
int orc_decode_rule_batch(int N, const uint8_t* frozen, const float* llr, int batch, int max_iter, double alpha,
                          int stop_mode, int rule, double theta, int fp32, int nthreads, uint8_t* u_hat,
                          int32_t* iters, int64_t* pe)
{
    if (batch < 0 || rule < 0 || rule > 2 || !(theta >= 0.0)) return ORC_ERR_ARG;
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int c = 0; c < batch; ++c) {
        int r = decode_one(N, frozen, llr + (size_t)c * (size_t)N, max_iter, alpha, stop_mode, 1, fp32,
                           u_hat + (size_t)c * (size_t)N, iters ? iters + c : NULL, pe ? pe + c : NULL, NULL, NULL,
                           NULL, NULL, NULL, NULL, rule, theta);
        if (r != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (err == ORC_OK) err = r;
            }
        }
    }
    (void)nthreads;
    return err;
}

/*
 * True flooding schedule, a variant beside the sweep of Eq. (1).  The paper
 * activates the PEs stage by stage from left to right (Sec. II-A), so R comes
 * from the current iteration and L from the previous one.  Under flooding,
 * every PE of every stage takes both its L and its R inputs from iteration
 * t-1, and all PEs update together.  Column 0's R (the channel) and column m's
 * L (the prior) are constant.  Messages start as in R2: interior L and R at 0.
 * The PE is Eq. (1)'s, with the same operand order.  There is no CSFG freezing:
 * its order of checks is defined on the sweep.  Stop modes, the output and the
 * PE count (m N/2 per iteration) are those of the sweep without freezing.
 */
int orc_decode_flood(int N, const uint8_t* frozen, const float* llr, int max_iter, double alpha, int stop_mode,
                     int fp32, uint8_t* u_hat, int32_t* iters, int64_t* pe, double* margin, double* trace_L,
                     double* trace_R)
{
    int m = ilog2_exact(N);
    if (m < 1 || !frozen || !llr || max_iter < 1 || !(alpha > 0.0) || !u_hat) return ORC_ERR_ARG;
    dec_t d;
    memset(&d, 0, sizeof d);
    d.N = N;
    d.m = m;
    d.fp32 = fp32;
    d.alpha = fp32 ? (double)(float)alpha : alpha;
    d.frozen = frozen;
    d.margin = INFINITY;
    size_t planes = (size_t)(m + 1) * (size_t)N;
    d.L = (double*)calloc(planes, sizeof(double));
    d.R = (double*)calloc(planes, sizeof(double));
    double* Ln = (double*)calloc(planes, sizeof(double));
    double* Rn = (double*)calloc(planes, sizeof(double));
    d.uh = (uint8_t*)malloc((size_t)N);
    d.scratch = (uint8_t*)malloc((size_t)N);
    d.ubits = (uint8_t*)malloc((size_t)N);
    int rc = ORC_OK;
    if (!d.L || !d.R || !Ln || !Rn || !d.uh || !d.scratch || !d.ubits) {
        rc = ORC_ERR_NOMEM;
        goto out;
    }
    for (int i = 0; i < N; ++i) {
        LM(&d, m, i) = frozen[i] ? INFINITY : 0.0; /* reading R2 */
        RM(&d, 0, i) = (double)llr[i];
    }
    int done = 0, t_done = max_iter;
    for (int t = 1; t <= max_iter && !done; ++t) {
        memcpy(Ln, d.L, planes * sizeof(double)); /* keeps L[m], the prior */
        memcpy(Rn, d.R, planes * sizeof(double)); /* keeps R[0], the channel */
        for (int s = 0; s < m; ++s) {
            const int h = 1 << (m - 1 - s);
            for (int a = 0; a < N; ++a) {
                if (a & h) continue;
                const int b = a + h;
                const double La = LM(&d, s + 1, a); /* L^{t-1}_{i,j+1}        */
                const double Lb = LM(&d, s + 1, b); /* L^{t-1}_{i+2^(m-j),j+1} */
                const double Ra = RM(&d, s, a);     /* R^{t-1}_{i,j}          */
                const double Rb = RM(&d, s, b);     /* R^{t-1}_{i+2^(m-j),j}  */
                const double tt = rnd(&d, Lb + Rb);
                const double g = fms(&d, La, Ra);
                const double nLa = fms(&d, La, tt);
                const double nLb = rnd(&d, Lb + g);
                const double nRa = fms(&d, Ra, tt);
                const double nRb = rnd(&d, Rb + g);
                if (isnan(nLa) || isnan(nLb) || isnan(nRa) || isnan(nRb)) d.nan_seen = 1;
                Ln[(size_t)s * N + a] = nLa;
                Ln[(size_t)s * N + b] = nLb;
                Rn[(size_t)(s + 1) * N + a] = nRa;
                Rn[(size_t)(s + 1) * N + b] = nRb;
                d.pe += 1;
            }
        }
        memcpy(d.L, Ln, planes * sizeof(double));
        memcpy(d.R, Rn, planes * sizeof(double));
        if (d.nan_seen) {
            rc = ORC_ERR_NAN;
            goto out;
        }
        if (stop_mode == 1 && gmatrix_stop(&d, 0)) done = 1;
        if (trace_L) memcpy(trace_L + (size_t)(t - 1) * planes, d.L, planes * sizeof(double));
        if (trace_R) memcpy(trace_R + (size_t)(t - 1) * planes, d.R, planes * sizeof(double));
        if (done) t_done = t;
    }
    for (int i = 0; i < N; ++i) u_hat[i] = source_bit(&d, i, 0);
    if (iters) *iters = t_done;
    if (pe) *pe = d.pe;
    if (margin) *margin = d.margin;
out:
    free(d.L);
    free(d.R);
    free(Ln);
    free(Rn);
    free(d.uh);
    free(d.scratch);
    free(d.ubits);
    return rc;
}

int orc_decode_flood_batch(int N, const uint8_t* frozen, const float* llr, int batch, int max_iter, double alpha,
                           int stop_mode, int fp32, int nthreads, uint8_t* u_hat, int32_t* iters, int64_t* pe,
                           double* margin)
{
    if (batch < 0) return ORC_ERR_ARG;
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int c = 0; c < batch; ++c) {
        int r = orc_decode_flood(N, frozen, llr + (size_t)c * (size_t)N, max_iter, alpha, stop_mode, fp32,
                                 u_hat + (size_t)c * (size_t)N, iters ? iters + c : NULL, pe ? pe + c : NULL,
                                 margin ? margin + c : NULL, NULL, NULL);
        if (r != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (err == ORC_OK) err = r;
            }
        }
    }
    (void)nthreads;
    return err;
}

/* Decode `batch` codewords (llr is batch x N), threaded over codewords when the
 * file is built with OpenMP.  nthreads <= 0 uses the OpenMP default.  Returns
 * the first nonzero error code met, else ORC_OK. */
int orc_decode_batch(int N, const uint8_t* frozen, const float* llr, int batch, int max_iter, double alpha,
                     int stop_mode, int freeze, int fp32, int nthreads, uint8_t* u_hat, int32_t* iters,
                     int64_t* pe, double* margin, int32_t* cover)
{
    if (batch < 0) return ORC_ERR_ARG;
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int c = 0; c < batch; ++c) {
        int r = orc_decode(N, frozen, llr + (size_t)c * (size_t)N, max_iter, alpha, stop_mode, freeze, fp32,
                           u_hat + (size_t)c * (size_t)N, iters ? iters + c : NULL, pe ? pe + c : NULL,
                           margin ? margin + c : NULL, cover ? cover + c : NULL, NULL, NULL, NULL, NULL);
        if (r != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (err == ORC_OK) err = r;
            }
        }
    }
    (void)nthreads;
    return err;
}

/*
 * Successive-cancellation (SC) decoding on the same code (Sec. III compares a
 * frozen CSFG's decision with SC decoding of its constituent code).  With
 * x = u F^{(x)m} in natural order, a block of S positions with channel LLRs
 * lam splits into halves: its first half of u sees x1 = x_left ^ x_right, with
 * LLRs f(lam[t], lam[t + S/2]); once that half is decided (its encoding x1),
 * the second half sees x2 = x_right = x_left ^ x1, with LLRs
 * lam[t + S/2] + (1 - 2 x1[t]) lam[t]; the block's encoding is (x1 ^ x2, x2).
 * A frozen position decides 0, an information position HD(LLR) (values >= 0
 * decide 0).  f is the exact box-plus (exact != 0), 2 atanh(tanh(a/2) tanh(b/2)),
 * or its min-sum approximation sign(a) sign(b) min(|a|, |b|).  FP64.  The exact
 * f is evaluated as written while min(|a|, |b|) < 4 (tanh is not saturated
 * there, and tiny results keep their relative precision), else as
 *   sign(a) sign(b) min(|a|, |b|) + log(1 + e^-|a+b|) - log(1 + e^-|a-b|),
 * the same function, whose correction terms are then small (no cancellation).
 */
static double sc_f(int exact, double a, double b)
{
    const double mn = fmin(fabs(a), fabs(b));
    if (!exact) return sgn(a) * sgn(b) * mn;
    if (mn < 4.0) return 2.0 * atanh(tanh(0.5 * a) * tanh(0.5 * b));
    return sgn(a) * sgn(b) * mn + log1p(exp(-fabs(a + b))) - log1p(exp(-fabs(a - b)));
}

/* Decode the block of S positions starting at source index `base` from LLRs
 * lam[0..S); writes u_hat[base..base+S) and the block's encoding x[0..S).
 * work holds at least 2 S doubles. */
static void sc_node(int S, int base, const double* lam, const uint8_t* frozen, int exact, uint8_t* u_hat,
                    uint8_t* x, double* work)
{
    if (S == 1) {
        uint8_t b = frozen[base] ? 0 : (lam[0] < 0.0 ? 1 : 0);
        u_hat[base] = b;
        x[0] = b;
        return;
    }
    const int h = S / 2;
    double* child = work;   /* h LLRs for the child being decoded */
    double* rest = work + h; /* scratch for the child's own recursion */
    for (int t = 0; t < h; ++t) child[t] = sc_f(exact, lam[t], lam[t + h]);
    sc_node(h, base, child, frozen, exact, u_hat, x, rest);
    for (int t = 0; t < h; ++t) child[t] = lam[t + h] + (1.0 - 2.0 * (double)x[t]) * lam[t];
    sc_node(h, base + h, child, frozen, exact, u_hat, x + h, rest);
    for (int t = 0; t < h; ++t) x[t] ^= x[t + h];
}

int orc_sc_decode(int N, const uint8_t* frozen, const float* llr, int exact, uint8_t* u_hat)
{
    int m = ilog2_exact(N);
    if (m < 0 || !frozen || !llr || !u_hat) return ORC_ERR_ARG;
    double* lam = (double*)malloc(sizeof(double) * (size_t)N);
    double* work = (double*)malloc(sizeof(double) * (size_t)(2 * N + 2));
    uint8_t* x = (uint8_t*)malloc((size_t)N);
    int rc = ORC_OK;
    if (!lam || !work || !x) {
        rc = ORC_ERR_NOMEM;
    } else {
        for (int i = 0; i < N; ++i) lam[i] = (double)llr[i];
        sc_node(N, 0, lam, frozen, exact, u_hat, x, work);
    }
    free(lam);
    free(work);
    free(x);
    return rc;
}

int orc_sc_decode_batch(int N, const uint8_t* frozen, const float* llr, int batch, int exact, int nthreads,
                        uint8_t* u_hat)
{
    if (batch < 0) return ORC_ERR_ARG;
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
#endif
    for (int c = 0; c < batch; ++c) {
        int r = orc_sc_decode(N, frozen, llr + (size_t)c * (size_t)N, exact, u_hat + (size_t)c * (size_t)N);
        if (r != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (err == ORC_OK) err = r;
            }
        }
    }
    (void)nthreads;
    return err;
}

/*
 * Quantised messages (a variant for fixed-point hardware, which Sec. V names as
 * future work): Eq. (1) under the sweep schedule of R1 with 16-bit saturating
 * integer messages.
 *   quantisation   q = clamp(rint(llr * 2^F), -QMAX, QMAX), QMAX = 32767
 *   saturation     every sum is clamped to [-QMAX, QMAX]; +-QMAX plays +-inf
 *   scaling        alpha = A / 16 (A in 1..16), f(x, y) = sign(x) sign(y) ((A min(|x|, |y|) + 8) >> 4),
 *                  the scaled magnitude rounded to the nearest integer (ties up)
 *   prior          L[m] = +QMAX on frozen positions, 0 elsewhere; interior messages start at 0
 * Stop, output and PE count are those of the sweep without freezing.  Every
 * value is an exact integer, so a GPU kernel reproduces it bit for bit.
 */
#define QMAX 32767

static int32_t q_sat(int64_t v) { return (int32_t)(v > QMAX ? QMAX : (v < -QMAX ? -QMAX : v)); }

static int32_t q_f(int A, int32_t x, int32_t y)
{
    const int32_t ax = x < 0 ? -x : x, ay = y < 0 ? -y : y;
    const int32_t mag = ((int32_t)A * (ax < ay ? ax : ay) + 8) >> 4; /* rounded to nearest, ties up */
    return ((x < 0) != (y < 0)) ? -mag : mag;
}

int orc_decode_q(int N, const uint8_t* frozen, const float* llr, int max_iter, int A, int F, int stop_mode,
                 uint8_t* u_hat, int32_t* iters, int64_t* pe, int32_t* trace_L, int32_t* trace_R)
{
    int m = ilog2_exact(N);
    if (m < 1 || !frozen || !llr || max_iter < 1 || A < 1 || A > 16 || F < 0 || F > 8 || !u_hat) return ORC_ERR_ARG;
    size_t planes = (size_t)(m + 1) * (size_t)N;
    int32_t* L = (int32_t*)calloc(planes, sizeof(int32_t));
    int32_t* R = (int32_t*)calloc(planes, sizeof(int32_t));
    uint8_t* ub = (uint8_t*)malloc((size_t)N);
    uint8_t* xb = (uint8_t*)malloc((size_t)N);
    uint8_t* sc = (uint8_t*)malloc((size_t)N);
    int rc = ORC_OK;
    if (!L || !R || !ub || !xb || !sc) {
        rc = ORC_ERR_NOMEM;
        goto out;
    }
    for (int i = 0; i < N; ++i) {
        double v = rint((double)llr[i] * ldexp(1.0, F));
        R[i] = q_sat((int64_t)fmax(fmin(v, 1e9), -1e9));
        L[(size_t)m * N + i] = frozen[i] ? QMAX : 0;
    }
    int t_done = max_iter;
    int64_t count = 0;
    for (int t = 1; t <= max_iter; ++t) {
        for (int s = 0; s < m; ++s) {
            const int h = 1 << (m - 1 - s);
            for (int a = 0; a < N; ++a) {
                if (a & h) continue;
                const int b = a + h;
                const int32_t La = L[(size_t)(s + 1) * N + a], Lb = L[(size_t)(s + 1) * N + b];
                const int32_t Ra = R[(size_t)s * N + a], Rb = R[(size_t)s * N + b];
                const int32_t tt = q_sat((int64_t)Lb + Rb);
                const int32_t g = q_f(A, La, Ra);
                L[(size_t)s * N + a] = q_f(A, La, tt);
                L[(size_t)s * N + b] = q_sat((int64_t)Lb + g);
                R[(size_t)(s + 1) * N + a] = q_f(A, Ra, tt);
                R[(size_t)(s + 1) * N + b] = q_sat((int64_t)Rb + g);
                count += 1;
            }
        }
        if (trace_L) memcpy(trace_L + (size_t)(t - 1) * planes, L, planes * sizeof(int32_t));
        if (trace_R) memcpy(trace_R + (size_t)(t - 1) * planes, R, planes * sizeof(int32_t));
        if (stop_mode == 1) {
            for (int i = 0; i < N; ++i)
                ub[i] = frozen[i] ? 0 : (q_sat((int64_t)R[(size_t)m * N + i] + L[(size_t)m * N + i]) < 0);
            polar_transform(ub, xb, N, sc);
            int same = 1;
            for (int i = 0; i < N; ++i)
                if ((q_sat((int64_t)R[i] + L[i]) < 0) != xb[i]) same = 0;
            if (same) {
                t_done = t;
                break;
            }
        }
    }
    for (int i = 0; i < N; ++i)
        u_hat[i] = frozen[i] ? 0 : (q_sat((int64_t)R[(size_t)m * N + i] + L[(size_t)m * N + i]) < 0);
    if (iters) *iters = t_done;
    if (pe) *pe = count;
out:
    free(L);
    free(R);
    free(ub);
    free(xb);
    free(sc);
    return rc;
}

int orc_decode_q_batch(int N, const uint8_t* frozen, const float* llr, int batch, int max_iter, int A, int F,
                       int stop_mode, int nthreads, uint8_t* u_hat, int32_t* iters, int64_t* pe)
{
    if (batch < 0) return ORC_ERR_ARG;
    int err = ORC_OK;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int c = 0; c < batch; ++c) {
        int r = orc_decode_q(N, frozen, llr + (size_t)c * (size_t)N, max_iter, A, F, stop_mode,
                             u_hat + (size_t)c * (size_t)N, iters ? iters + c : NULL, pe ? pe + c : NULL, NULL, NULL);
        if (r != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            {
                if (err == ORC_OK) err = r;
            }
        }
    }
    (void)nthreads;
    return err;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Weighted min-sum: Eq. (1) with the scaling alpha replaced by one weight    */
/* per (iteration t, stage s, PE p), T unrolled iterations, no stop and no    */
/* freezing.  PE p of stage s pairs a and a + h (h = 2^(m-1-s)), p counting   */
/* the pairs in increasing a:  p = (a >> (m-s)) * h + (a mod h).  Weight      */
/* (t, s, p) sits at w[(t*m + s)*(N/2) + p].  The soft output of position i   */
/* is R[m][i] + L[m][i] after the last iteration.                             */
/*                                                                            */
/* Gradient.  f_w(x, y) = w h(x, y), h = sign(x) sign(y) min(|x|, |y|):       */
/*   df/dw = h;  when |x| <= |y| (ties to the first argument) df/dx =         */
/*   w sign(y), df/dy = 0, else df/dx = 0, df/dy = w sign(x).  Messages that  */
/*   are +-inf (made from the frozen prior) do not change with any weight or  */
/*   input: no adjoint flows into or out of them and they add nothing to a    */
/*   weight's gradient.                                                       */
/* ------------------------------------------------------------------------ */
static double r32(int fp32, double v) { return fp32 ? (double)(float)v : v; }

static double wms_f(int fp32, double w, double x, double y)
{
    double v = w * sgn(x) * sgn(y) * fmin(fabs(x), fabs(y));
    return fp32 ? (double)(float)v : v;
}

static int wms_pair_index(int m, int s, int a)
{
    const int h = 1 << (m - 1 - s);
    return ((a >> (m - s)) * h) + (a & (h - 1));
}

/* planes_L / planes_R: (T+1) x (m+1) x N; index 0 = before iteration 1 (L), then after each iteration */
static int wms_run(int N, int m, const uint8_t* frozen, const float* llr, int T, const double* w, int fp32,
                   double* planes_L, double* planes_R)
{
    const size_t P = (size_t)(m + 1) * (size_t)N;
    double* L = planes_L;
    double* R = planes_R;
    for (size_t k = 0; k < P; ++k) L[k] = 0.0, R[k] = 0.0;
    for (int i = 0; i < N; ++i) L[(size_t)m * N + i] = frozen[i] ? INFINITY : 0.0;
    for (int t = 1; t <= T; ++t) {
        double* Lc = planes_L + (size_t)t * P;
        double* Rc = planes_R + (size_t)t * P;
        memcpy(Lc, planes_L + (size_t)(t - 1) * P, P * sizeof(double));
        for (int i = 0; i < N; ++i) Rc[i] = (double)llr[i];
        for (int s = 0; s < m; ++s) {
            const int h = 1 << (m - 1 - s);
            for (int a = 0; a < N; ++a) {
                if (a & h) continue;
                const int b = a + h;
                const double wt = fp32 ? (double)(float)w[((size_t)(t - 1) * m + s) * (N / 2) + wms_pair_index(m, s, a)]
                                       : w[((size_t)(t - 1) * m + s) * (N / 2) + wms_pair_index(m, s, a)];
                const double La = Lc[(size_t)(s + 1) * N + a], Lb = Lc[(size_t)(s + 1) * N + b];
                const double Ra = Rc[(size_t)s * N + a], Rb = Rc[(size_t)s * N + b];
                double tt = Lb + Rb;
                if (fp32) tt = (double)(float)tt;
                const double g = wms_f(fp32, wt, La, Ra);
                double nLb = Lb + g, nRb = Rb + g;
                if (fp32) nLb = (double)(float)nLb, nRb = (double)(float)nRb;
                Lc[(size_t)s * N + a] = wms_f(fp32, wt, La, tt);
                Lc[(size_t)s * N + b] = nLb;
                Rc[(size_t)(s + 1) * N + a] = wms_f(fp32, wt, Ra, tt);
                Rc[(size_t)(s + 1) * N + b] = nRb;
                if (isnan(tt) || isnan(g)) return ORC_ERR_NAN;
            }
        }
    }
    (void)L;
    (void)R;
    return ORC_OK;
}

/*
 * orc_wms_forward -- weighted min-sum decode of one codeword.
 *   w         T*m*(N/2) weights (layout above), doubles
 *   out       N soft outputs R[m][i] + L[m][i] after iteration T
 *   trace_L, trace_R  optional T x (m+1) x N planes after each iteration
 */
int orc_wms_forward(int N, const uint8_t* frozen, const float* llr, int T, const double* w, int fp32, double* out,
                    double* trace_L, double* trace_R)
{
    const int m = ilog2_exact(N);
    if (m < 1 || T < 1 || !frozen || !llr || !w || !out) return ORC_ERR_ARG;
    const size_t P = (size_t)(m + 1) * (size_t)N;
    double* pl = (double*)malloc(sizeof(double) * P * (size_t)(T + 1));
    double* pr = (double*)malloc(sizeof(double) * P * (size_t)(T + 1));
    if (!pl || !pr) {
        free(pl);
        free(pr);
        return ORC_ERR_NOMEM;
    }
    int rc = wms_run(N, m, frozen, llr, T, w, fp32, pl, pr);
    if (rc == ORC_OK) {
        const double* Lf = pl + (size_t)T * P;
        const double* Rf = pr + (size_t)T * P;
        for (int i = 0; i < N; ++i) {
            double v = Rf[(size_t)m * N + i] + Lf[(size_t)m * N + i];
            out[i] = fp32 ? (double)(float)v : v;
        }
        if (trace_L) memcpy(trace_L, pl + P, sizeof(double) * P * (size_t)T);
        if (trace_R) memcpy(trace_R, pr + P, sizeof(double) * P * (size_t)T);
    }
    free(pl);
    free(pr);
    return rc;
}

/* derivative of f_w(x, y) with respect to x and y (ties to the first argument) */
static void wms_df(double w, double x, double y, double* dx, double* dy)
{
    if (fabs(x) <= fabs(y)) {
        *dx = w * sgn(y);
        *dy = 0.0;
    } else {
        *dx = 0.0;
        *dy = w * sgn(x);
    }
}

/* accumulate into an adjoint slot unless the message it belongs to is +-inf;
   with fp32 the sum is rounded to binary32, like every other operation */
static void wms_acc(int fp32, double* slot, double value, double g)
{
    if (!isinf(value)) *slot = r32(fp32, *slot + g);
}

/*
 * orc_wms_backward -- gradient of a loss through orc_wms_forward.
 *   dout   N values dLoss/d out[i]
 *   fp32   0: FP64 throughout.  1: the forward of orc_wms_forward's fp32 mode,
 *          and every product and sum of the adjoint rounded to binary32 (the
 *          weights and dout are taken as binary32 values).  The adjoint is the
 *          same chain rule in the same order either way: stages m-1 .. 0 of
 *          iterations T .. 1, PEs in increasing a, and within a PE the outputs
 *          R[s+1][b], L[s][b], R[s+1][a], L[s][a], then g and t.
 *   dw     T*m*(N/2) gradient of the weights (overwritten)
 *   dllr   N gradient of the channel LLRs (overwritten)
 */
int orc_wms_backward(int N, const uint8_t* frozen, const float* llr, int T, const double* w, const double* dout,
                     int fp32, double* dw, double* dllr)
{
    const int m = ilog2_exact(N);
    if (m < 1 || T < 1 || !frozen || !llr || !w || !dout || !dw || !dllr) return ORC_ERR_ARG;
    const size_t P = (size_t)(m + 1) * (size_t)N;
    double* pl = (double*)malloc(sizeof(double) * P * (size_t)(T + 1));
    double* pr = (double*)malloc(sizeof(double) * P * (size_t)(T + 1));
    double* dL = (double*)calloc(P, sizeof(double)); /* adjoint of the L state after the current iteration */
    double* dLp = (double*)calloc(P, sizeof(double)); /* adjoint of the L state before it */
    double* dR = (double*)calloc(P, sizeof(double));
    int rc = (pl && pr && dL && dLp && dR) ? ORC_OK : ORC_ERR_NOMEM;
    if (rc == ORC_OK) rc = wms_run(N, m, frozen, llr, T, w, fp32, pl, pr);
    if (rc == ORC_OK) {
        for (size_t k = 0; k < (size_t)T * (size_t)m * (size_t)(N / 2); ++k) dw[k] = 0.0;
        for (int i = 0; i < N; ++i) dllr[i] = 0.0;
        /* the soft output R[m] + L[m] of the last iteration; L[m] is the constant prior */
        for (int i = 0; i < N; ++i) dL[(size_t)m * N + i] = 0.0;
        for (int t = T; t >= 1; --t) {
            const double* Lp = pl + (size_t)(t - 1) * P; /* L^{t-1}: PE inputs */
            const double* Lc = pl + (size_t)t * P;       /* L^t:     PE outputs */
            const double* Rc = pr + (size_t)t * P;       /* R^t */
            for (size_t k = 0; k < P; ++k) dR[k] = 0.0, dLp[k] = 0.0;
            if (t == T)
                for (int i = 0; i < N; ++i) wms_acc(fp32, &dR[(size_t)m * N + i], Rc[(size_t)m * N + i], r32(fp32, dout[i]));
            /* the L state of columns m (prior) and 0 (read by nothing) carries no adjoint */
            for (int s = m - 1; s >= 0; --s) {
                const int h = 1 << (m - 1 - s);
                for (int a = 0; a < N; ++a) {
                    if (a & h) continue;
                    const int b = a + h;
                    const size_t widx = ((size_t)(t - 1) * m + s) * (N / 2) + wms_pair_index(m, s, a);
                    const double wt = r32(fp32, w[widx]);
                    const double La = Lp[(size_t)(s + 1) * N + a], Lb = Lp[(size_t)(s + 1) * N + b];
                    const double Ra = Rc[(size_t)s * N + a], Rb = Rc[(size_t)s * N + b];
                    const double tt = r32(fp32, Lb + Rb);
                    const double g = wms_f(fp32, wt, La, Ra);
                    /* adjoints of the four outputs (zero for +-inf outputs) */
                    const double oLa = Lc[(size_t)s * N + a], oLb = Lc[(size_t)s * N + b];
                    const double oRa = Rc[(size_t)(s + 1) * N + a], oRb = Rc[(size_t)(s + 1) * N + b];
                    const double gLa = (s >= 1 && !isinf(oLa)) ? dL[(size_t)s * N + a] : 0.0;
                    const double gLb = (s >= 1 && !isinf(oLb)) ? dL[(size_t)s * N + b] : 0.0;
                    const double gRa = isinf(oRa) ? 0.0 : dR[(size_t)(s + 1) * N + a];
                    const double gRb = isinf(oRb) ? 0.0 : dR[(size_t)(s + 1) * N + b];
                    double dg = 0.0, dt = 0.0, dx, dy;
                    /* R[s+1][b] = Rb + g ; L[s][b] = Lb + g */
                    wms_acc(fp32, &dR[(size_t)s * N + b], Rb, gRb);
                    if (!isinf(g)) dg = r32(fp32, dg + gRb);
                    wms_acc(fp32, &dLp[(size_t)(s + 1) * N + b], Lb, gLb);
                    if (!isinf(oLb)) dg = r32(fp32, dg + gLb);
                    /* R[s+1][a] = f(Ra, t) */
                    if (!isinf(oRa) && gRa != 0.0) {
                        wms_df(wt, Ra, tt, &dx, &dy);
                        wms_acc(fp32, &dR[(size_t)s * N + a], Ra, r32(fp32, gRa * dx));
                        if (!isinf(tt)) dt = r32(fp32, dt + r32(fp32, gRa * dy));
                        dw[widx] = r32(fp32, dw[widx] + r32(fp32, gRa * (sgn(Ra) * sgn(tt) * fmin(fabs(Ra), fabs(tt)))));
                    }
                    /* L[s][a] = f(La, t) */
                    if (!isinf(oLa) && gLa != 0.0) {
                        wms_df(wt, La, tt, &dx, &dy);
                        wms_acc(fp32, &dLp[(size_t)(s + 1) * N + a], La, r32(fp32, gLa * dx));
                        if (!isinf(tt)) dt = r32(fp32, dt + r32(fp32, gLa * dy));
                        dw[widx] = r32(fp32, dw[widx] + r32(fp32, gLa * (sgn(La) * sgn(tt) * fmin(fabs(La), fabs(tt)))));
                    }
                    /* g = f(La, Ra) */
                    if (!isinf(g) && dg != 0.0) {
                        wms_df(wt, La, Ra, &dx, &dy);
                        wms_acc(fp32, &dLp[(size_t)(s + 1) * N + a], La, r32(fp32, dg * dx));
                        wms_acc(fp32, &dR[(size_t)s * N + a], Ra, r32(fp32, dg * dy));
                        dw[widx] = r32(fp32, dw[widx] + r32(fp32, dg * (sgn(La) * sgn(Ra) * fmin(fabs(La), fabs(Ra)))));
                    }
                    /* t = Lb + Rb */
                    if (!isinf(tt)) {
                        wms_acc(fp32, &dLp[(size_t)(s + 1) * N + b], Lb, dt);
                        wms_acc(fp32, &dR[(size_t)s * N + b], Rb, dt);
                    }
                }
            }
            for (int i = 0; i < N; ++i) dllr[i] = r32(fp32, dllr[i] + dR[i]);
            /* the L state before iteration t: columns 1..m-1 carry over; iteration 1 reads the start state */
            double* tmp = dL;
            dL = dLp;
            dLp = tmp;
            for (int i = 0; i < N; ++i) dL[(size_t)m * N + i] = 0.0, dL[i] = 0.0;
        }
    }
    free(pl);
    free(pr);
    free(dL);
    free(dLp);
    free(dR);
    return rc;
}
