/*
 * hb_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * Householder-aligned permutation test (Ehara, "Accurate and Efficient
 * Statistical Testing for Word Semantic Breadth", ACL 2026).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call this file.  The
 * product library never links it and shares no code, header, table or helper
 * with it.  Numeric status codes and enum values are restated here by
 * convention, not included.
 *
 * What it computes, in the order of Algorithm 1:
 *   step 1  sample means x_bar, y_bar and mean directions mu_x, mu_y   (Sec. 3.1)
 *   step 2  Householder axis u = (mu_x - mu_y)/||mu_x - mu_y||         (Sec. 3.1, axis eq.)
 *   step 3  x' = x - 2 u (u^T x) for every x of the reflected cloud     (Eq. householder_fast)
 *   step 4  observed statistic T_obs                                     (Eqs. r, v, tobs)
 *   step 5  B relabellings of the pooled Z = X' u Y, exceedance count    (Sec. 3.1, fixed-space test)
 *   step 6  p = (1 + count)/(B + 1)                                     (Eq. pvalue)
 *
 * Arithmetic conventions (the readings of the paper this file fixes):
 *  - Inputs are FP32 or BF16 bit patterns.  Every input/Z value v is widened
 *    to an exact fixed-point integer v * 2^87 held in a signed 128-bit
 *    integer; values with |v| < 2^-64 are taken as 0 (they lie far below any
 *    resolution the statistic has).  Column sums and group sums are therefore
 *    exact and independent of summation order; each exact sum is rounded once
 *    to FP64 (round-to-nearest-even).
 *  - Every other floating-point step is IEEE binary64 with round-to-nearest-
 *    even.  Dot products and squared norms are sequential fused multiply-add
 *    chains over j = 0..d-1.  The file must be compiled with
 *    -ffp-contract=off so that the compiler adds no fusions of its own.
 *  - The reflected rows are rounded once to the input storage type (FP32 or
 *    BF16, round-to-nearest-even): the paper runs its group-sum GEMM on data
 *    held in half precision (Sec. 3.2, practical note (1)), and the pooled
 *    set Z is fixed after alignment (Sec. 3.1, fixed-space permutation).
 *  - The reflection is skipped (H = I) when ||mu_x - mu_y|| <= 2^-27
 *    (the paper applies it only "if mu_x != mu_y").
 *  - The concentration map g_d is the approximation of Banerjee et al.
 *    (JMLR 2005), g_d(r) = r (d - r^2)/(1 - r^2); the paper only says it uses
 *    "the same estimator as in prior work" (Sec. 3.1, Eq. v).
 *  - Labels: HB-LABEL-v1.  Philox4x32-10 (Salmon et al., SC'11) with key
 *    (seed_lo, seed_hi) and counter (i/4, b_lo, stream, b_hi); word i mod 4
 *    serves position i; sequential selection sampling (Knuth, TAOCP vol. 2,
 *    Sec. 3.4.2, Algorithm S) puts position i in group 1 iff
 *    floor(w_i * (N - i) / 2^32) < n - (ones so far).  Exactly n ones.
 *  - Exceedance: two-sided |T_b| >= |T_obs| by default (ties count, Eq.
 *    pvalue uses >=); one-sided ">=" and "<=" are selectable.  For the
 *    log-volume statistic the decision is DEFINED by cross-multiplying the
 *    positive g values (g2_b * g1_o >= g2_o * g1_b for T_b >= T_obs, and the
 *    larger-times-smaller form for |T|), each product rounded once in FP64.
 *    In exact arithmetic this equals comparing the logarithms; with the two
 *    rounded products it can differ from a comparison of rounded logarithms
 *    only when the two sides agree to about one ulp, and it keeps structural
 *    ties (the complement split of n = m, where the products are equal
 *    exactly) and uses only correctly-rounded IEEE operations, so every
 *    implementation that follows it reaches the same decision.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

/* status codes (same numbering as the public C ABI, restated) */
enum { HBO_OK = 0, HBO_ERR_INVALID_ARG = 1, HBO_ERR_DEGENERATE = 2 };
/* storage types */
enum { HBO_F32 = 0, HBO_BF16 = 1 };
/* statistics */
enum { HBO_STAT_LOGVOL_VMF = 0, HBO_STAT_ONE_MINUS_R2 = 1, HBO_STAT_MEAN_COSDIST = 2 };
/* alternatives */
enum { HBO_ALT_TWO_SIDED = 0, HBO_ALT_GREATER = 1, HBO_ALT_LESS = 2 };

typedef struct {
    uint64_t seed;
    uint32_t stream;
    int64_t B;
    int32_t stat;
    int32_t alt;
    int32_t align;        /* 1 = Householder alignment, 0 = naive test   */
    int32_t reflect_side; /* 0 = reflect X (paper), 1 = reflect Y        */
    int32_t exhaustive;   /* 1 = all C(N, n) splits in colex order       */
} hbo_opts;

typedef struct {
    double p;
    int64_t count;
    int64_t B_eff;
    double T_obs;
    double r_x;
    double r_y;
    int32_t reflection_skipped;
    int32_t status;
} hbo_result;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from its published definition (Salmon, Moraes, Dror and    */
/* Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11).              */
/* ------------------------------------------------------------------------ */
void hbo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u; /* Weyl increments */
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One label row of HB-LABEL-v1: bit i of row = 1 iff position i is in group 1. */
static void label_row(uint64_t seed, uint32_t stream, int64_t n, int64_t N, int64_t b, uint32_t *row)
{
    int64_t W = (N + 31) / 32;
    memset(row, 0, (size_t)W * sizeof(uint32_t));
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t words[4] = {0, 0, 0, 0};
    int64_t ones = 0;
    for (int64_t i = 0; i < N; ++i) {
        if ((i & 3) == 0) {
            uint32_t ctr[4] = {(uint32_t)(i >> 2), (uint32_t)b, stream, (uint32_t)((uint64_t)b >> 32)};
            hbo_philox4x32_10(ctr, key, words);
        }
        uint64_t remaining = (uint64_t)(N - i);          /* N - i positions left      */
        uint64_t needed = (uint64_t)(n - ones);          /* ones still to place       */
        uint64_t scaled = ((uint64_t)words[i & 3] * remaining) >> 32; /* in [0, N - i) */
        if (scaled < needed) {
            row[i >> 5] |= 1u << (i & 31);
            ++ones;
        }
    }
}

void hbo_labels(uint64_t seed, uint32_t stream, int64_t n, int64_t N, int64_t b0, int64_t count, uint32_t *bits)
{
    int64_t W = (N + 31) / 32;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k)
        label_row(seed, stream, n, N, b0 + k, bits + k * W);
}

/* Number of n-subsets of N, exact in 64 bits for N <= 62. */
int64_t hbo_binomial(int64_t N, int64_t n)
{
    if (n < 0 || n > N) return 0;
    if (n > N - n) n = N - n;
    uint64_t c = 1;
    for (int64_t k = 1; k <= n; ++k) c = c * (uint64_t)(N - n + k) / (uint64_t)k;
    return (int64_t)c;
}

/* All n-subsets of {0..N-1} in colex order (increasing bit-mask value),
 * enumerated with Gosper's next-combination step.  N <= 30. */
void hbo_labels_exhaustive(int64_t n, int64_t N, uint32_t *bits)
{
    int64_t C = hbo_binomial(N, n);
    uint64_t mask = (n == 0) ? 0 : ((1ull << n) - 1ull);
    for (int64_t b = 0; b < C; ++b) {
        bits[b] = (uint32_t)mask;
        if (mask == 0) break;
        uint64_t low = mask & (~mask + 1ull);
        uint64_t ripple = mask + low;
        uint64_t ones = ((ripple ^ mask) >> 2) / low;
        mask = ripple | ones;
    }
}

/* ------------------------------------------------------------------------ */
/* Exact widening and rounding.                                              */
/* ------------------------------------------------------------------------ */
static uint32_t storage_to_f32bits(const void *base, int dtype, int64_t idx)
{
    if (dtype == HBO_F32) return ((const uint32_t *)base)[idx];
    return (uint32_t)((const uint16_t *)base)[idx] << 16;
}

static double f32bits_to_f64(uint32_t b)
{
    float f;
    memcpy(&f, &b, sizeof f);
    return (double)f;
}

/* v * 2^87 as an exact integer; |v| < 2^-64 gives 0. */
static i128 fixed_from_f32bits(uint32_t b)
{
    uint32_t e = (b >> 23) & 0xffu;
    if (e < 63u) return 0;
    uint32_t mant = (b & 0x7fffffu) | 0x800000u;
    i128 m = (i128)mant << (e - 63u);
    return (b >> 31) ? -m : m;
}

static double fixed_to_f64(i128 v) { return ldexp((double)v, -87); }

/* Round x once to a binary format with p significand bits and minimum normal
 * exponent emin, round-to-nearest-even (IEEE 754 "roundTiesToEven"). */
static double round_to_format(double x, int p, int emin)
{
    if (x == 0.0 || !isfinite(x)) return x;
    double a = fabs(x);
    int e = ilogb(a);
    if (e < emin) e = emin;
    double quantum = ldexp(1.0, e - (p - 1));
    double r = nearbyint(a / quantum) * quantum;
    return copysign(r, x);
}

static void store_rounded(void *base, int dtype, int64_t idx, double x)
{
    if (dtype == HBO_F32) {
        double r = round_to_format(x, 24, -126);
        float f = (float)r; /* exact: r is an FP32 value */
        uint32_t b;
        memcpy(&b, &f, sizeof b);
        ((uint32_t *)base)[idx] = b;
    } else {
        double r = round_to_format(x, 8, -126);
        float f = (float)r; /* exact: every BF16 value is an FP32 value */
        uint32_t b;
        memcpy(&b, &f, sizeof b);
        ((uint16_t *)base)[idx] = (uint16_t)(b >> 16);
    }
}

static int valid_value(uint32_t f32bits)
{
    uint32_t e = (f32bits >> 23) & 0xffu;
    if (e == 0xffu) return 0;            /* inf or nan */
    return e < 127u + 4u;                /* |v| < 16   */
}

/* ------------------------------------------------------------------------ */
/* Steps 1-3: mean directions, Householder axis, reflection.                 */
/* ------------------------------------------------------------------------ */
/* rows (ptr, count) of one cloud; returns exact column sums rounded to FP64 */
static void column_sums(const void *base, int dtype, int64_t rows, int64_t d, double *out)
{
    i128 *acc = (i128 *)calloc((size_t)d, sizeof(i128));
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < d; ++j) acc[j] += fixed_from_f32bits(storage_to_f32bits(base, dtype, i * d + j));
    for (int64_t j = 0; j < d; ++j) out[j] = fixed_to_f64(acc[j]);
    free(acc);
}

static double sq_norm(const double *v, int64_t d)
{
    double acc = 0.0;
    for (int64_t j = 0; j < d; ++j) acc = fma(v[j], v[j], acc);
    return acc;
}

/*
 * Z_out  : [n+m][d] in the storage type; rows 0..n-1 come from X, n..N-1 from Y.
 * u_out  : [d] FP64 axis (zeros when the reflection is skipped), nullable.
 * zf64   : [n+m][d] FP64 values before the storage rounding, nullable.
 * Returns a status code.
 */
int hbo_align(const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int dtype, int align, int reflect_side,
              void *Z_out, double *u_out, double *zf64, int32_t *skipped)
{
    if (n < 1 || m < 1 || d < 1 || (dtype != HBO_F32 && dtype != HBO_BF16)) return HBO_ERR_INVALID_ARG;
    for (int64_t k = 0; k < n * d; ++k)
        if (!valid_value(storage_to_f32bits(X, dtype, k))) return HBO_ERR_INVALID_ARG;
    for (int64_t k = 0; k < m * d; ++k)
        if (!valid_value(storage_to_f32bits(Y, dtype, k))) return HBO_ERR_INVALID_ARG;

    double *xbar = (double *)malloc(sizeof(double) * (size_t)d);
    double *ybar = (double *)malloc(sizeof(double) * (size_t)d);
    double *u = (double *)calloc((size_t)d, sizeof(double));
    int status = HBO_OK;
    int skip = 1;

    if (align) {
        /* step 1: x_bar = (1/n) sum x_i, mu_x = x_bar/||x_bar||; likewise for Y */
        column_sums(X, dtype, n, d, xbar);
        column_sums(Y, dtype, m, d, ybar);
        for (int64_t j = 0; j < d; ++j) {
            xbar[j] = xbar[j] / (double)n;
            ybar[j] = ybar[j] / (double)m;
        }
        double nx = sqrt(sq_norm(xbar, d));
        double ny = sqrt(sq_norm(ybar, d));
        if (!(nx > 0.0) || !(ny > 0.0)) {
            status = HBO_ERR_DEGENERATE;
        } else {
            /* step 2: u = (mu_x - mu_y)/||mu_x - mu_y|| */
            double *v = (double *)malloc(sizeof(double) * (size_t)d);
            for (int64_t j = 0; j < d; ++j) v[j] = xbar[j] / nx - ybar[j] / ny;
            double nv = sqrt(sq_norm(v, d));
            if (nv > 0x1p-27) {
                skip = 0;
                for (int64_t j = 0; j < d; ++j) u[j] = v[j] / nv;
            }
            free(v);
        }
    }
    if (status == HBO_OK) {
        int64_t N = n + m;
        for (int64_t i = 0; i < N; ++i) {
            int from_x = i < n;
            const void *src = from_x ? X : Y;
            int64_t row = from_x ? i : i - n;
            int reflect = !skip && (from_x ? reflect_side == 0 : reflect_side == 1);
            if (!reflect) {
                for (int64_t j = 0; j < d; ++j) {
                    uint32_t b = storage_to_f32bits(src, dtype, row * d + j);
                    if (dtype == HBO_F32) ((uint32_t *)Z_out)[i * d + j] = b;
                    else ((uint16_t *)Z_out)[i * d + j] = (uint16_t)(b >> 16);
                    if (zf64) zf64[i * d + j] = f32bits_to_f64(b);
                }
                continue;
            }
            /* step 3: c = u^T x, then x' = x - 2 c u, one rounding per element */
            double c = 0.0;
            for (int64_t j = 0; j < d; ++j)
                c = fma(u[j], f32bits_to_f64(storage_to_f32bits(src, dtype, row * d + j)), c);
            for (int64_t j = 0; j < d; ++j) {
                double x = f32bits_to_f64(storage_to_f32bits(src, dtype, row * d + j));
                double xr = fma(-2.0 * c, u[j], x);
                if (zf64) zf64[i * d + j] = xr;
                store_rounded(Z_out, dtype, i * d + j, xr);
            }
        }
    }
    if (u_out) memcpy(u_out, u, sizeof(double) * (size_t)d);
    if (skipped) *skipped = skip;
    free(xbar);
    free(ybar);
    free(u);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Steps 4-6: statistic, exceedance count, p-value.                          */
/* ------------------------------------------------------------------------ */
/* Per-group value A from q = ||group sum||^2 and the group size:
 *   LOGVOL_VMF  : A = g_d(r) with r = ||sum||/n_g  (T = log A2 - log A1)
 *   ONE_MINUS_R2: A = 1 - r^2                       (T = A1 - A2)
 *   MEAN_COSDIST: A = (n_g^2 - q)/(n_g (n_g - 1))   (T = A1 - A2) */
static double group_value(int stat, double q, double ng, double d)
{
    double ng2 = ng * ng;
    if (stat == HBO_STAT_LOGVOL_VMF) {
        double rr = q / ng2;
        double r = sqrt(rr);
        double den = 1.0 - rr;
        if (!(den > 0.0)) return INFINITY;
        return (r * (d - rr)) / den;
    }
    if (stat == HBO_STAT_ONE_MINUS_R2) return 1.0 - q / ng2;
    return (ng2 - q) / (ng * (ng - 1.0));
}

static double stat_T(int stat, double A1, double A2)
{
    if (stat == HBO_STAT_LOGVOL_VMF) return log(A2) - log(A1);
    return A1 - A2;
}

/* exceedance decision of permutation b against the observed split o */
static int exceeds(int stat, int alt, double A1b, double A2b, double A1o, double A2o)
{
    if (stat == HBO_STAT_LOGVOL_VMF) {
        if (alt == HBO_ALT_GREATER) return A2b * A1o >= A2o * A1b;
        if (alt == HBO_ALT_LESS) return A2b * A1o <= A2o * A1b;
        double hib = A1b > A2b ? A1b : A2b, lob = A1b > A2b ? A2b : A1b;
        double hio = A1o > A2o ? A1o : A2o, loo = A1o > A2o ? A2o : A1o;
        return hib * loo >= hio * lob;
    }
    double Tb = A1b - A2b, To = A1o - A2o;
    if (alt == HBO_ALT_GREATER) return Tb >= To;
    if (alt == HBO_ALT_LESS) return Tb <= To;
    return fabs(Tb) >= fabs(To);
}

/* Exact group sums of Z (fixed point) for the split in `row` (bit i = group 1),
 * each group summed directly over its own members, then q1, q2 in FP64. */
static void split_q(const i128 *zfx, int64_t N, int64_t d, const uint32_t *row, i128 *s1, i128 *s2, double *q1,
                    double *q2)
{
    memset(s1, 0, sizeof(i128) * (size_t)d);
    memset(s2, 0, sizeof(i128) * (size_t)d);
    for (int64_t i = 0; i < N; ++i) {
        i128 *dst = ((row[i >> 5] >> (i & 31)) & 1u) ? s1 : s2;
        const i128 *zi = zfx + i * d;
        for (int64_t j = 0; j < d; ++j) dst[j] += zi[j];
    }
    double a1 = 0.0, a2 = 0.0;
    for (int64_t j = 0; j < d; ++j) {
        double v1 = fixed_to_f64(s1[j]);
        double v2 = fixed_to_f64(s2[j]);
        a1 = fma(v1, v1, a1);
        a2 = fma(v2, v2, a2);
    }
    *q1 = a1;
    *q2 = a2;
}

typedef struct {
    i128 *zfx;         /* [N][d] exact Z */
    int64_t n, m, N, d;
    double A1o, A2o;   /* observed per-group values */
    double To;
} prepared;

static int prepare(const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int dtype, const hbo_opts *o,
                   prepared *P, hbo_result *res, void *Z_keep)
{
    memset(res, 0, sizeof *res);
    if (n < 2 || m < 2) { res->status = HBO_ERR_DEGENERATE; return res->status; }
    if (o->stat < 0 || o->stat > 2 || o->alt < 0 || o->alt > 2 || (o->reflect_side != 0 && o->reflect_side != 1)) {
        res->status = HBO_ERR_INVALID_ARG;
        return res->status;
    }
    int64_t N = n + m;
    size_t esz = dtype == HBO_F32 ? 4 : 2;
    void *Z = Z_keep ? Z_keep : malloc((size_t)N * (size_t)d * esz);
    int32_t skipped = 0;
    int st = hbo_align(X, n, Y, m, d, dtype, o->align, o->reflect_side, Z, NULL, NULL, &skipped);
    if (st != HBO_OK) {
        if (!Z_keep) free(Z);
        res->status = st;
        return st;
    }
    P->zfx = (i128 *)malloc(sizeof(i128) * (size_t)N * (size_t)d);
    for (int64_t k = 0; k < N * d; ++k) P->zfx[k] = fixed_from_f32bits(storage_to_f32bits(Z, dtype, k));
    if (!Z_keep) free(Z);
    P->n = n; P->m = m; P->N = N; P->d = d;

    /* step 4: the observed split is rows 0..n-1 against rows n..N-1 */
    int64_t W = (N + 31) / 32;
    uint32_t *row = (uint32_t *)calloc((size_t)W, sizeof(uint32_t));
    for (int64_t i = 0; i < n; ++i) row[i >> 5] |= 1u << (i & 31);
    i128 *s1 = (i128 *)malloc(sizeof(i128) * (size_t)d), *s2 = (i128 *)malloc(sizeof(i128) * (size_t)d);
    double q1, q2;
    split_q(P->zfx, N, d, row, s1, s2, &q1, &q2);
    free(row); free(s1); free(s2);
    P->A1o = group_value(o->stat, q1, (double)n, (double)d);
    P->A2o = group_value(o->stat, q2, (double)m, (double)d);
    P->To = stat_T(o->stat, P->A1o, P->A2o);
    res->T_obs = P->To;
    res->r_x = sqrt(q1 / ((double)n * (double)n));
    res->r_y = sqrt(q2 / ((double)m * (double)m));
    res->reflection_skipped = skipped;
    if (o->stat == HBO_STAT_LOGVOL_VMF && (!(q1 > 0.0) || !(q2 > 0.0) || !isfinite(P->A1o) || !isfinite(P->A2o))) {
        free(P->zfx);
        P->zfx = NULL;
        res->status = HBO_ERR_DEGENERATE;
        return res->status;
    }
    return HBO_OK;
}

/*
 * Full test of one pair.  T_out (nullable) receives T_b for b = 0..B_eff-1
 * and exceed_out (nullable) the per-b decisions.
 */
int hbo_perm_test(const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int dtype, const hbo_opts *o,
                  hbo_result *res, double *T_out, uint8_t *exceed_out)
{
    prepared P;
    memset(&P, 0, sizeof P);
    if (prepare(X, n, Y, m, d, dtype, o, &P, res, NULL) != HBO_OK) return res->status;
    int64_t N = P.N, W = (N + 31) / 32;
    int64_t Beff;
    uint32_t *all = NULL;
    if (o->exhaustive) {
        if (N > 30) { free(P.zfx); res->status = HBO_ERR_INVALID_ARG; return res->status; }
        Beff = hbo_binomial(N, n);
        all = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)Beff);
        hbo_labels_exhaustive(n, N, all);
    } else {
        if (o->B < 1) { free(P.zfx); res->status = HBO_ERR_INVALID_ARG; return res->status; }
        Beff = o->B;
    }
    int64_t count = 0;
#pragma omp parallel reduction(+ : count)
    {
        uint32_t *row = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)W);
        i128 *s1 = (i128 *)malloc(sizeof(i128) * (size_t)d), *s2 = (i128 *)malloc(sizeof(i128) * (size_t)d);
#pragma omp for schedule(dynamic, 16)
        for (int64_t b = 0; b < Beff; ++b) {
            if (o->exhaustive) row[0] = all[b];
            else label_row(o->seed, o->stream, n, N, b, row);
            double q1, q2;
            split_q(P.zfx, N, d, row, s1, s2, &q1, &q2);
            double A1 = group_value(o->stat, q1, (double)n, (double)d);
            double A2 = group_value(o->stat, q2, (double)m, (double)d);
            int e = exceeds(o->stat, o->alt, A1, A2, P.A1o, P.A2o);
            count += e;
            if (T_out) T_out[b] = stat_T(o->stat, A1, A2);
            if (exceed_out) exceed_out[b] = (uint8_t)e;
        }
        free(row); free(s1); free(s2);
    }
    free(all);
    free(P.zfx);
    res->count = count;
    res->B_eff = Beff;
    if (o->exhaustive) res->p = (double)count / (double)Beff;
    else res->p = (double)(1 + count) / (double)(Beff + 1);
    res->status = HBO_OK;
    return HBO_OK;
}

/* T_b and decisions for a list of permutation indices only (sampled checks
 * at sizes where the full loop would take too long). */
int hbo_perm_stats(const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int dtype, const hbo_opts *o,
                   const int64_t *b_list, int64_t nb, hbo_result *res, double *T_out, uint8_t *exceed_out,
                   double *q_out /* nullable [nb][2] */)
{
    prepared P;
    memset(&P, 0, sizeof P);
    if (prepare(X, n, Y, m, d, dtype, o, &P, res, NULL) != HBO_OK) return res->status;
    int64_t N = P.N, W = (N + 31) / 32;
#pragma omp parallel
    {
        uint32_t *row = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)W);
        i128 *s1 = (i128 *)malloc(sizeof(i128) * (size_t)d), *s2 = (i128 *)malloc(sizeof(i128) * (size_t)d);
#pragma omp for schedule(dynamic, 1)
        for (int64_t k = 0; k < nb; ++k) {
            label_row(o->seed, o->stream, n, N, b_list[k], row);
            double q1, q2;
            split_q(P.zfx, N, d, row, s1, s2, &q1, &q2);
            double A1 = group_value(o->stat, q1, (double)n, (double)d);
            double A2 = group_value(o->stat, q2, (double)m, (double)d);
            if (T_out) T_out[k] = stat_T(o->stat, A1, A2);
            if (exceed_out) exceed_out[k] = (uint8_t)exceeds(o->stat, o->alt, A1, A2, P.A1o, P.A2o);
            if (q_out) { q_out[2 * k] = q1; q_out[2 * k + 1] = q2; }
        }
        free(row); free(s1); free(s2);
    }
    free(P.zfx);
    res->status = HBO_OK;
    return HBO_OK;
}

/* Several pairs packed back to back (pair p: n[p] rows of X then m[p] rows of Y). */
int hbo_perm_test_batched(int64_t P, const void *XY, const int64_t *n, const int64_t *m, int64_t d, int dtype,
                          const hbo_opts *o, hbo_result *out)
{
    size_t esz = dtype == HBO_F32 ? 4 : 2;
    const char *base = (const char *)XY;
    int worst = HBO_OK;
    for (int64_t p = 0; p < P; ++p) {
        const char *x = base;
        const char *y = base + (size_t)n[p] * (size_t)d * esz;
        int st = hbo_perm_test(x, n[p], y, m[p], d, dtype, o, &out[p], NULL, NULL);
        if (st != HBO_OK && worst == HBO_OK) worst = st;
        base = y + (size_t)m[p] * (size_t)d * esz;
    }
    return worst;
}

/* Exposed for pins: exact fixed-point widening of one FP32 pattern (as two
 * 64-bit halves) and the FP64 rounding of an exact value. */
void hbo_fixed_from_f32bits(uint32_t bits, int64_t *hi, uint64_t *lo)
{
    i128 v = fixed_from_f32bits(bits);
    *hi = (int64_t)(v >> 64);
    *lo = (uint64_t)v;
}

double hbo_round_to_bf16(double x) { return round_to_format(x, 8, -126); }
double hbo_round_to_f32(double x) { return round_to_format(x, 24, -126); }
