// hb_internal.cuh -- device helpers and launch metadata shared by the hbperm
// kernels (sm_103a).  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hb {

typedef __int128 i128;
typedef unsigned __int128 u128;

enum : int32_t { ST_OK = 0, ST_INVALID = 1, ST_DEGENERATE = 2, ST_TIMEOUT = 5 };
enum : int32_t { DT_F32 = 0, DT_BF16 = 1 };
enum : int32_t { STAT_LOGVOL = 0, STAT_R2 = 1, STAT_COSDIST = 2 };
enum : int32_t { ALT_TWO = 0, ALT_GREATER = 1, ALT_LESS = 2 };

// Per-pair launch metadata, built on the host.
struct PairMeta {
    const void *X;      // device pointer to n rows
    const void *Y;      // device pointer to m rows
    int64_t z_row;      // first row of this pair in Z (rows padded to 64)
    int64_t lab_off;    // first word of this pair's label block [W][B_pad]
    int64_t B;          // relabellings (C(N, n) when exhaustive)
    int64_t T_off;      // offset of this pair's T_b values in T_out, -1 = none
    int64_t g_off;      // tensor-core path: first entry of this pair's list of relabellings (B_pad entries)
    int32_t n, m, N, N_pad;
    int32_t W;          // 32-bit label words per relabelling
    int32_t B_pad;      // B rounded up to the relabellings of a work item
    int32_t chunk0;     // first row chunk of this pair (X side then Y side)
    int32_t nchunk_x;   // row chunks of the X side
    int32_t nchunk_y;   // row chunks of the Y side
    int32_t pad_;
};

// A chunk of at most CHUNK_ROWS consecutive rows of one side of one pair.
constexpr int CHUNK_ROWS = 128;
struct RowChunk {
    int32_t pair;
    int32_t side;   // 0 = rows of X (group 1 of the observed split), 1 = rows of Y
    int32_t row0;   // first row within the side
    int32_t nrows;
};

// Per-pair state written by the device.
struct PairState {
    int32_t status;
    int32_t skipped;
    double A1o, A2o, To;     // observed per-group values and T_obs (FP64, exact path)
    double rx, ry;
    float tnorm;             // ||t|| (FP32) for the error band
    float sumc2;             // sum_j c_j^2 of the per-column band constants (all slices)
    unsigned long long count;
    unsigned long long rechecked;
    unsigned int band_max_bits;  // float bits of the largest band (atomicMax)
    float sumc2_1;           // sum_j c1_j^2 (tensor-core path, BF16: the single-slice pass)
    unsigned int n_gather;   // relabellings the single-slice pass left to the two-slice pass
    int32_t pad_;
};

// Per-column constants of one pair for the fast paths.
struct ColConst {
    float q_hi;   // scale of the first slice: 2^(E-8) (FP32 storage); 1 (BF16: slices hold values); 0.5 plain
    float t;      // column total of Z, rounded to FP32
    float c;      // band constant: residual sum of all slices (tensor cores) or gamma_K * sum|z| (plain)
    float c1;     // BF16 tensor-core path: residual sum of the first slice alone
};

// Shared launch options (flattened hb_opts).
struct RunOpts {
    uint64_t seed;
    uint32_t stream;
    int32_t stat, alt, align, reflect_side, exhaustive, path;
    int32_t d, d_pad, dtype, slices;
    int32_t want_T;
    int32_t cw;      // z-columns per tensor-core tile of one slice (128 BF16, 64 FP32; half when narrow; 96 with am)
    int32_t cg;      // tensor-core path: 1 = one CTA per MMA, 2 = CTA pairs (M = 256)
    int32_t nacc;    // accumulator columns of a tensor-core tile: slices * cw
    int32_t s1_max;  // BF16 tensor-core path: pairs with N <= s1_max take the single-slice pass first
    int32_t am;      // BF16 on CTA pairs: the A operand in TMEM (192-column accumulators) instead of shared memory
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// ---------------------------------------------------------------------------
// Values and the exact 2^-87 fixed-point grid.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t load_f32bits(const void *base, int dtype, int64_t idx)
{
    if (dtype == DT_F32) return __ldg(reinterpret_cast<const uint32_t *>(base) + idx);
    return uint32_t(__ldg(reinterpret_cast<const unsigned short *>(base) + idx)) << 16;
}

// finite and |v| < 16
__device__ __forceinline__ bool valid_f32bits(uint32_t b)
{
    return ((b >> 23) & 0xffu) < 131u;
}

// v * 2^87 exactly; |v| < 2^-64 gives 0.
__device__ __forceinline__ i128 fixed_from_f32bits(uint32_t b)
{
    const uint32_t e = (b >> 23) & 0xffu;
    if (e < 63u) return 0;
    const uint64_t mant = (b & 0x7fffffu) | 0x800000u;
    const uint32_t sh = e - 63u;
    u128 m = (u128)mant << sh;
    return (b >> 31) ? -(i128)m : (i128)m;
}

// Exact sums on the same 2^-87 grid, cheaper: values within 55 binades below
// a column bound 2^E are accumulated as integers of unit 2^(E-55) in 64 bits
// (at most 2^55 each, so 128 of them cannot overflow); the rare smaller values
// go through the 128-bit path.  Flushing below 2^-64 is unchanged.
struct WinAcc {
    int64_t acc;
    i128 slow;
    int eb;    // biased FP32 exponent of the window: E + 95 (256 = no window)
    int sh;    // shift from the window unit to the 2^-87 grid: E + 32
    __device__ __forceinline__ void init(int E)
    {
        acc = 0;
        slow = 0;
        if (E + 32 >= 0 && E <= 120) {
            eb = E + 95;
            sh = E + 32;
        } else {
            eb = 256;
            sh = 0;
        }
    }
    __device__ __forceinline__ void add(uint32_t b)
    {
        const int e = (int)((b >> 23) & 0xffu);
        if (e < 63) return;  // |v| < 2^-64 counts as 0
        const int s = e - eb;
        if (s >= 0) {
            const int64_t v = (int64_t)((b & 0x7fffffu) | 0x800000u) << s;
            acc += (b >> 31) ? -v : v;
        } else {
            slow += fixed_from_f32bits(b);
        }
    }
    // moves the 64-bit part into the 128-bit total (call at least every 128 adds)
    __device__ __forceinline__ void flush()
    {
        slow += (i128)acc << sh;
        acc = 0;
    }
    __device__ __forceinline__ i128 total()
    {
        flush();
        return slow;
    }
};

// E with |v| < 2^E for every value of a column whose maximum magnitude has
// FP32 bit pattern maxbits (0 for an all-zero column).
__device__ __forceinline__ int col_bound_exp(unsigned int maxbits)
{
    if (maxbits == 0u) return -200;
    return (int)((maxbits >> 23) & 0xffu) - 126;
}

// ---------------------------------------------------------------------------
// BF16 storage, tensor-core path: the two slices of one column of one pair.
// Both are grids of powers of two that keep every FP32 accumulator of the
// group-sum GEMM exact.  With L1 >= sum_i |z_i| over the pair's N tokens and
// g = 2^eg, eg = ceil(log2 L1) - 23, the first slice k_i g = z_i rounded to
// the grid g satisfies sum_i |k_i g| < L1 + N g/2 < 2^24 g, so every partial
// sum of any subset is a multiple of g below 2^24 g: an exact FP32 value.  A
// BF16 z_i whose last bit is >= g is its own first slice; smaller ones round
// to a multiple of g of at most 8 significant bits, so the first slice is a
// BF16 value too.  The second slice k2_i g2 = (z_i - k_i g) rounded to
// g2 = g 2^(ceil(log2 N) - 23) has the same property (the residuals of the
// first slice sum to at most N g/2 <= 2^22 g2) and at most 8 significant bits.
// What both leave out, z_i - k_i g - k2_i g2, is nonzero only for values below
// 2^7 g2 with bits under g2, and enters the error band.  Values below 2^-64
// count as 0 (the oracle's rule) and are flushed before the split.
// ---------------------------------------------------------------------------
struct L1Grid {
    int eg, eg2;   // exponents of g and g2
    bool split;    // false: both slices 0 and the residual is the value
    float g, inv_g, g2, inv_g2;
};

// l1fx = ceil(L1 * 2^40) (0: every value of the column is 0); N = tokens of the pair
__device__ __forceinline__ L1Grid l1_grid(unsigned long long l1fx, int N)
{
    L1Grid G;
    const int cl = l1fx <= 1ull ? 0 : 64 - __clzll((long long)(l1fx - 1ull));  // ceil(log2 l1fx)
    const int cn = N <= 1 ? 0 : 32 - __clz(N - 1);                               // ceil(log2 N)
    G.eg = cl - 40 - 23;
    G.eg2 = G.eg + cn - 23;
    // exact integer totals need g2 on the 2^-87 grid (g2 >= 2^-87, a normal float)
    G.split = l1fx != 0ull && G.eg2 >= -87;
    if (G.split) {
        G.g = __int_as_float((G.eg + 127) << 23);
        G.inv_g = __int_as_float((127 - G.eg) << 23);
        G.g2 = __int_as_float((G.eg2 + 127) << 23);
        G.inv_g2 = __int_as_float((127 - G.eg2) << 23);
    } else {
        G.g = G.inv_g = G.g2 = G.inv_g2 = 0.0f;
    }
    return G;
}

// The exact split z = k g + k2 g2 + r2 (r1 = z - k g); every step is exact in FP32.
__device__ __forceinline__ void l1_split(float z, const L1Grid &G, float &k, float &k2, float &r1, float &r2)
{
    if (((__float_as_uint(z) >> 23) & 0xffu) < 63u) z = 0.0f;  // |z| < 2^-64 counts as 0
    k = rintf(__fmul_rn(z, G.inv_g));
    r1 = __fmaf_rn(-k, G.g, z);
    k2 = rintf(__fmul_rn(r1, G.inv_g2));
    r2 = __fmaf_rn(-k2, G.g2, r1);
}

__device__ __forceinline__ double pow2d(int e)  // 2^e for -1022 <= e <= 1023
{
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Exact integer -> FP64, round-to-nearest-even.
__device__ __forceinline__ double i128_to_f64_rn(i128 v)
{
    if (v == 0) return 0.0;
    const bool neg = v < 0;
    const u128 a = neg ? (u128)0 - (u128)v : (u128)v;
    const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
    const int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    double r;
    if (msb <= 52) {
        r = __ull2double_rn(lo);  // exact
    } else {
        const int sh = msb - 52;
        uint64_t top = (uint64_t)(a >> sh);
        const u128 rem = a & (((u128)1 << sh) - 1);
        const u128 half = (u128)1 << (sh - 1);
        if (rem > half || (rem == half && (top & 1ull))) top += 1ull;
        r = __dmul_rn(__ull2double_rn(top), pow2d(sh));  // both exact
    }
    return neg ? -r : r;
}

__device__ __forceinline__ double fixed_to_f64(i128 v)
{
    return __dmul_rn(i128_to_f64_rn(v), pow2d(-87));
}

__device__ __forceinline__ double f32bits_to_f64(uint32_t b)
{
    return (double)__uint_as_float(b);
}

// Right shift with round-to-nearest-even, s >= 1.
__device__ __forceinline__ uint64_t rshift_rne(uint64_t v, int s)
{
    if (s >= 64) return 0ull;  // v < 2^53 here, so v / 2^s < 1/2
    const uint64_t q = v >> s;
    const uint64_t rem = v & ((1ull << s) - 1ull);
    const uint64_t half = 1ull << (s - 1);
    return (rem > half || (rem == half && (q & 1ull))) ? q + 1ull : q;
}

// FP64 -> BF16 bit pattern, one rounding to nearest-even (finite input).
__device__ __forceinline__ uint16_t f64_to_bf16_rn(double x)
{
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint16_t sign = (uint16_t)((b >> 48) & 0x8000u);
    const int ebits = (int)((b >> 52) & 0x7ff);
    if (ebits == 0) return sign;  // zero or below 2^-1022: rounds to zero in BF16
    const int e = ebits - 1023;
    const uint64_t sig = (b & ((1ull << 52) - 1ull)) | (1ull << 52);
    if (e >= -126) {
        uint64_t s8 = rshift_rne(sig, 45);  // 8 significant bits, may round up to 256
        int ee = e;
        if (s8 == 256ull) {
            s8 = 128ull;
            ++ee;
        }
        if (ee > 127) return (uint16_t)(sign | 0x7f80u);
        return (uint16_t)(sign | (uint16_t)((ee + 127) << 7) | (uint16_t)(s8 & 0x7fu));
    }
    // subnormal BF16: value / 2^-133 = sig * 2^(e + 81)
    const uint64_t k = rshift_rne(sig, -(e + 81));
    return (uint16_t)(sign | (uint16_t)k);  // k == 128 encodes the smallest normal
}

// BF16 bits of a normal or subnormal FP32 value, round to nearest even (the
// same result as f64_to_bf16_rn of the exactly widened value).
__device__ __forceinline__ unsigned short f32_to_bf16_rn_bits(float f)
{
    const uint32_t b = __float_as_uint(f);
    return (unsigned short)((b + 0x7fffu + ((b >> 16) & 1u)) >> 16);
}

// Exact FP32 -> FP64 widening built from the bit fields (normal values);
// zero, subnormals, infinities and NaN take the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const uint64_t db = ((uint64_t)(b & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                        ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)db);
}

// ---------------------------------------------------------------------------
// Exact-path statistic (FP64, correctly rounded operations only).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double group_value_f64(int stat, double q, double ng, double d)
{
    const double ng2 = __dmul_rn(ng, ng);
    if (stat == STAT_LOGVOL) {
        const double rr = __ddiv_rn(q, ng2);
        const double r = __dsqrt_rn(rr);
        const double den = __dsub_rn(1.0, rr);
        if (!(den > 0.0)) return __longlong_as_double(0x7ff0000000000000ll);
        return __ddiv_rn(__dmul_rn(r, __dsub_rn(d, rr)), den);
    }
    if (stat == STAT_R2) return __dsub_rn(1.0, __ddiv_rn(q, ng2));
    return __ddiv_rn(__dsub_rn(ng2, q), __dmul_rn(ng, __dsub_rn(ng, 1.0)));
}

__device__ __forceinline__ double stat_T_f64(int stat, double A1, double A2)
{
    if (stat == STAT_LOGVOL) return __dsub_rn(log(A2), log(A1));
    return __dsub_rn(A1, A2);
}

__device__ __forceinline__ int exceeds_f64(int stat, int alt, double A1b, double A2b, double A1o, double A2o)
{
    if (stat == STAT_LOGVOL) {
        if (alt == ALT_GREATER) return __dmul_rn(A2b, A1o) >= __dmul_rn(A2o, A1b);
        if (alt == ALT_LESS) return __dmul_rn(A2b, A1o) <= __dmul_rn(A2o, A1b);
        const double hib = A1b > A2b ? A1b : A2b, lob = A1b > A2b ? A2b : A1b;
        const double hio = A1o > A2o ? A1o : A2o, loo = A1o > A2o ? A2o : A1o;
        return __dmul_rn(hib, loo) >= __dmul_rn(hio, lob);
    }
    const double Tb = __dsub_rn(A1b, A2b), To = __dsub_rn(A1o, A2o);
    if (alt == ALT_GREATER) return Tb >= To;
    if (alt == ALT_LESS) return Tb <= To;
    return fabs(Tb) >= fabs(To);
}

// ---------------------------------------------------------------------------
// Fast-path decision with a rigorous error band (FP32).
//   q1, q2   : approximate squared group-sum norms
//   dq1, dq2 : bounds on |q_hat - q| (exact q of the relabelling)
// Returns +1 (exceeds), 0 (does not), -1 (inside the band: decide exactly).
// ---------------------------------------------------------------------------
constexpr float U32 = 5.9604645e-8f;  // 2^-24

__device__ __forceinline__ float logvol_phi_band(float q, float dq, float ng, float d, float *phi)
{
    // phi = log g(r), r = sqrt(q)/ng.  |dphi/dq| <= h(r)/(2q) with
    // h(r) = 1 + 2 r^2/(1 - r^2) an upper bound of d log g / d log r.
    const float ng2 = ng * ng;
    const float rr = q / ng2;
    const float r = sqrtf(rr);
    const float den = 1.0f - rr;
    const float g = r * (d - rr) / den;
    *phi = logf(g);
    const float qlo = q - dq, qhi = q + dq;
    const float rrhi = qhi / ng2;
    if (!(qlo > 0.0f) || !(rrhi < 0.999f) || !(den > 0.0f) || !(g > 0.0f)) return INFINITY;
    const float h = 1.0f + 2.0f * rrhi / (1.0f - rrhi);
    const float lin = h * dq / (2.0f * qlo);
    // FP32 evaluation of phi(q_hat): rr (2 roundings), sqrt, d - rr, 1 - rr (its
    // error amplified by rr/(1 - rr)), product and quotient give a relative
    // error of g below (7 + 2 rr/(1 - rr)) u; logf adds at most 1 ulp of phi.
    const float ev = 1.1f * U32 * (7.0f + 2.0f * rrhi / (1.0f - rrhi)) + 2.2f * U32 * fabsf(*phi);
    return lin + ev;
}

__device__ __forceinline__ int fast_decide(int stat, int alt, float d, float n, float m, float q1, float q2, float dq1,
                                           float dq2, float To, float *T_hat, float *band)
{
    float T, eps;
    if (stat == STAT_LOGVOL) {
        float p1, p2;
        const float e1 = logvol_phi_band(q1, dq1, n, d, &p1);
        const float e2 = logvol_phi_band(q2, dq2, m, d, &p2);
        T = p2 - p1;
        eps = e1 + e2 + U32 * fabsf(T);
    } else if (stat == STAT_R2) {
        const float a = q1 / (n * n), b = q2 / (m * m);
        T = b - a;
        eps = dq1 / (n * n) + dq2 / (m * m) + 3.0f * U32 * (a + b + fabsf(T));
    } else {
        const float a = (n * n - q1) / (n * (n - 1.0f)), b = (m * m - q2) / (m * (m - 1.0f));
        T = a - b;
        eps = dq1 / (n * (n - 1.0f)) + dq2 / (m * (m - 1.0f)) +
              8.0f * U32 * ((n * n + q1) / (n * (n - 1.0f)) + (m * m + q2) / (m * (m - 1.0f)) + fabsf(T));
    }
    float D;
    if (alt == ALT_GREATER) D = T - To;
    else if (alt == ALT_LESS) D = To - T;
    else D = fabsf(T) - fabsf(To);
    // rounding of To to FP32 and of the subtraction; a factor 1.5 covers the
    // second-order terms the first-order bounds above leave out
    eps = 1.5f * (eps + 2.0f * U32 * (fabsf(T) + fabsf(To))) + 1e-30f;
    *T_hat = T;
    *band = eps;
    if (!(eps < INFINITY) || D != D) return -1;
    if (D > eps) return 1;
    if (D < -eps) return 0;
    return -1;
}

// Bound on |q_hat - q| given the accumulated terms (see the design notes):
//   E    = sum_j |sigma_hat_j| c_j      (first-order term of the per-column bounds)
//   q    = q_hat of this group, qa/qb = both groups, tnorm = ||t||,
//   sumc2 = sum_j c_j^2, chain = rounding-chain length of the q accumulation.
__device__ __forceinline__ float q_bound(float E, float q, float q1, float q2, float tnorm, float sumc2, float chain)
{
    // per column: |sigma_hat_g - sigma_g| <= c_j + u (|t_j| + |s1_j| + |s2_j| + |s_g,j|) (1 + 2u),
    // so 2 sum_j |sigma_hat_g| e_j <= 2E + 2.01 u (s (||t|| + s1 + s2) + q) by Cauchy-Schwarz
    const float s = sqrtf(q), s1 = sqrtf(q1), s2 = sqrtf(q2);
    const float first = 2.0f * E * (1.0f + (chain + 8.0f) * U32) + 2.01f * U32 * (s * (tnorm + s1 + s2) + q);
    const float second = 2.0f * sumc2 + 10.0f * U32 * U32 * (tnorm * tnorm + q1 + q2 + q);
    return (first + second + chain * U32 * q) * (1.0f + 1e-4f);
}

// A relabelling whose fast-path decision fell inside its error band.
struct alignas(8) RecheckItem {
    int32_t pair;
    uint32_t b;
};

__device__ __forceinline__ void push_recheck(RecheckItem *list, unsigned int *n_items, unsigned int cap,
                                             unsigned int *overflow, int p, uint32_t b)
{
    const unsigned int k = atomicAdd(n_items, 1u);
    if (k < cap) list[k] = RecheckItem{p, b};
    else atomicExch(overflow, 1u);
}

// Per-pair result copied back to the host.
struct PairOut {
    double p;
    int64_t count;
    int64_t B_eff;
    double T_obs, r_x, r_y;
    int32_t skipped, status;
    int64_t rechecked;
    double band_max;
};

// Packed FP32 pairs (f32x2): two independent IEEE single-precision
// operations, round to nearest, in one instruction; the low word is the
// first element.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// upward-rounded forms (rigorous bounds)
__device__ __forceinline__ f2_t f2_add_ru(f2_t a, f2_t b)
{
    f2_t d;
    asm("add.rp.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_mul_ru(f2_t a, f2_t b)
{
    f2_t d;
    asm("mul.rp.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2_fma_ru(f2_t a, f2_t b, f2_t c)
{
    f2_t d;
    asm("fma.rp.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2_splat(float a) { return f2_pack(a, a); }
__device__ __forceinline__ f2_t f2_abs(f2_t a) { return a & 0x7FFFFFFF7FFFFFFFull; }

// Iteration cap of every bounded device spin-wait.
constexpr long long SPIN_LIMIT = 1ll << 26;

}  // namespace hb
