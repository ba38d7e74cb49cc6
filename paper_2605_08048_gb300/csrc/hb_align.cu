// hb_align.cu -- steps 1-4 of Algorithm 1 on the device.
//
//   k_colsum_partial / k_colsum_reduce : exact column sums of X and Y
//       (Sec. 3.1: x_bar = (1/n) sum x_i), inputs validated on the way
//   k_axis   : mean directions, v = mu_x - mu_y, u = v/||v|| in FP64
//       (Sec. 3.1 axis equation; skipped when ||v|| <= 2^-27)
//   k_reflect: x' = x - 2u(u^T x) per row (Eq. householder_fast), defined as
//       the FP64 sequential dot then one FMA per element, rounded once to the
//       storage type (BF16 storage: evaluated in compensated FP32 with a
//       rigorous bound, the FP64 steps deciding what the bound cannot); the
//       other cloud is copied; column maxima for the fixed-point scales of
//       the mixed path
//   k_zstats_partial / k_zstats_tok / k_zstats_reduce : exact column totals t
//       of Z and the group-1 sums of the observed split, the band constants,
//       and (tensor-core path) the slices of Z in token-contiguous rows for
//       the tensor-core B operand: two grid slices of the values for BF16
//       storage (l1_split), three fixed-point slices for FP32 storage
//   k_tobs   : observed statistic T_obs from the exact sums (Eq. tobs)
//
// The FP64 arithmetic uses explicit __d*_rn / __fma_rn intrinsics so that no
// contraction or reassociation changes a result.
#include <algorithm>

#include "hb_launch.cuh"

namespace hb {

// ---------------------------------------------------------------------------
// Column sums of the inputs (exact), one block per row chunk.  When every row
// starts on a 16-byte boundary, thread g sums the 16-byte column group g
// (VE = 8 BF16 or 4 FP32 columns) over the chunk's rows with vector loads,
// several rows in flight; otherwise one column per thread.  Exact sums do not
// depend on the order, so both give the same totals.
// ---------------------------------------------------------------------------
// BF16 input: each value v splits exactly into h = v rounded to the 2^-12 grid
// and l = v - h.  For a valid |v| < 16 the h of <= 128 rows sum to < 2^11 on
// the 2^-12 grid and every l of a value >= 2^-21 is a multiple of 2^-28 below
// 2^-13, so both FP32 running sums are exact; values below 2^-21 (rare) are
// added exactly one by one (|v| < 2^-64 counts as 0).  Invalid values show as
// a non-finite sum or a maximum magnitude >= 16.
__device__ __noinline__ i128 colsum_tiny_bf16(const uint4 *src, int64_t stride, int nrows, int e)
{
    i128 acc = 0;
    for (int r = 0; r < nrows; ++r) {
        const uint4 v = __ldg(src + r * stride);
        const uint32_t w = (e >> 1) == 0 ? v.x : (e >> 1) == 1 ? v.y : (e >> 1) == 2 ? v.z : v.w;
        const uint32_t b = (e & 1) ? (w & 0xffff0000u) : (w << 16);
        if (((b >> 23) & 0xffu) < 127u - 21u) acc += fixed_from_f32bits(b);
    }
    return acc;
}

__device__ __forceinline__ void colsum_bf16(const void *base, const RowChunk &ch, int d, i128 *out, bool &ok)
{
    const int groups = d / 8;
    const float M = 3072.0f;  // 1.5 * 2^11: (v + M) - M rounds v to the 2^-12 grid for |v| < 2^10
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        float sh[8], sl[8], amax = 0.0f;
        uint32_t tiny = 0u;
#pragma unroll
        for (int e = 0; e < 8; ++e) sh[e] = sl[e] = 0.0f;
        const uint4 *src = reinterpret_cast<const uint4 *>(base) + ((int64_t)ch.row0 * d) / 8 + g;
        const int64_t stride = d / 8;
#pragma unroll 4
        for (int r = 0; r < ch.nrows; ++r) {
            const uint4 v = __ldg(src + r * stride);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const uint32_t b = (e & 1) ? (w[e >> 1] & 0xffff0000u) : (w[e >> 1] << 16);
                const float x = __uint_as_float(b);
                const float h = __fsub_rn(__fadd_rn(x, M), M);
                sh[e] = __fadd_rn(sh[e], h);
                sl[e] = __fadd_rn(sl[e], __fsub_rn(x, h));
                amax = fmaxf(amax, fabsf(x));
                // 0 < |v| < 2^-21 (the wrap-around of |b| - 1 leaves zeros out)
                tiny |= ((b & 0x7fffffffu) - 1u < (106u << 23) - 1u) ? (1u << e) : 0u;
            }
        }
        ok &= amax < 16.0f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            // tiny values took part in the FP32 sums: remove them exactly by recomputing the
            // column from scratch in that (rare) case
            ok &= isfinite(sh[e]) && isfinite(sl[e]);
            if ((tiny >> e) & 1u) {
                i128 acc = colsum_tiny_bf16(src, stride, ch.nrows, e);
                // the values >= 2^-21, exactly: their split sums without the tiny ones
                float h2 = 0.0f, l2 = 0.0f;
                for (int r = 0; r < ch.nrows; ++r) {
                    const uint4 v = __ldg(src + r * stride);
                    const uint32_t w = (e >> 1) == 0 ? v.x : (e >> 1) == 1 ? v.y : (e >> 1) == 2 ? v.z : v.w;
                    const uint32_t b = (e & 1) ? (w & 0xffff0000u) : (w << 16);
                    if (((b >> 23) & 0xffu) < 127u - 21u) continue;
                    const float x = __uint_as_float(b);
                    const float h = __fsub_rn(__fadd_rn(x, M), M);
                    h2 = __fadd_rn(h2, h);
                    l2 = __fadd_rn(l2, __fsub_rn(x, h));
                }
                out[g * 8 + e] = acc + fixed_from_f32bits(__float_as_uint(h2)) + fixed_from_f32bits(__float_as_uint(l2));
            } else {
                out[g * 8 + e] = fixed_from_f32bits(__float_as_uint(sh[e])) + fixed_from_f32bits(__float_as_uint(sl[e]));
            }
        }
    }
}

template <int DT>
__device__ __forceinline__ void colsum_vec(const void *base, const RowChunk &ch, int d, i128 *out, bool &ok)
{
    constexpr int VE = DT == DT_BF16 ? 8 : 4;
    const int groups = d / VE;
    for (int g = threadIdx.x; g < groups; g += blockDim.x) {
        WinAcc wa[VE];
#pragma unroll
        for (int e = 0; e < VE; ++e) wa[e].init(4);  // valid inputs satisfy |v| < 2^4
        const uint4 *src = reinterpret_cast<const uint4 *>(base) + ((int64_t)ch.row0 * d) / VE + g;
        const int64_t stride = d / VE;
#pragma unroll 4
        for (int r = 0; r < ch.nrows; ++r) {
            const uint4 v = __ldg(src + r * stride);
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < VE; ++e) {
                const uint32_t b = DT == DT_BF16 ? ((e & 1) ? (w[e >> 1] & 0xffff0000u) : (w[e >> 1] << 16)) : w[e];
                ok &= valid_f32bits(b);
                wa[e].add(b);
            }
        }
#pragma unroll
        for (int e = 0; e < VE; ++e) out[g * VE + e] = wa[e].total();
    }
}

__global__ void k_colsum_partial(const PairMeta *__restrict__ meta, const RowChunk *__restrict__ chunks, int c0,
                                 int d, int dtype, i128 *__restrict__ part, int *__restrict__ bad)
{
    const int ci = c0 + (int)blockIdx.x;  // chunk index
    const RowChunk ch = chunks[ci];
    const PairMeta pm = meta[ch.pair];
    const void *base = ch.side ? pm.Y : pm.X;
    const int esz = dtype == DT_F32 ? 4 : 2;
    bool ok = true;
    i128 *out = part + (int64_t)ci * d;
    if ((d * esz) % 16 == 0 && ((uintptr_t)base & 15u) == 0) {
        if (dtype == DT_F32) colsum_vec<DT_F32>(base, ch, d, out, ok);
        else colsum_bf16(base, ch, d, out, ok);
    } else {
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            WinAcc wa;
            wa.init(4);  // valid inputs satisfy |v| < 2^4
            for (int r = 0; r < ch.nrows; ++r) {
                const uint32_t b = load_f32bits(base, dtype, (int64_t)(ch.row0 + r) * d + j);
                ok &= valid_f32bits(b);
                wa.add(b);
            }
            out[j] = wa.total();
        }
    }
    if (!ok) atomicOr(bad + ch.pair, 1);
}

// s[(p*2 + side)*d + j] = sum over the chunks of (p, side), pairs p0 .. p1-1
__global__ void k_colsum_reduce(const PairMeta *__restrict__ meta, int p0, int p1, int d,
                                const i128 *__restrict__ part, i128 *__restrict__ s)
{
    const int64_t idx = (int64_t)p0 * 2 * d + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)p1 * 2 * d) return;
    const int j = (int)(idx % d);
    const int ps = (int)(idx / d);
    const int p = ps >> 1, side = ps & 1;
    const PairMeta pm = meta[p];
    const int c0 = pm.chunk0 + (side ? pm.nchunk_x : 0);
    const int nc = side ? pm.nchunk_y : pm.nchunk_x;
    i128 acc = 0;
    for (int c = 0; c < nc; ++c) acc += part[(int64_t)(c0 + c) * d + j];
    s[idx] = acc;
}

// ---------------------------------------------------------------------------
// Axis: one block of 64 threads per pair (p0 + block); dynamic smem 2*d doubles.
// ---------------------------------------------------------------------------
__global__ void k_axis(const PairMeta *__restrict__ meta, int p0, const RunOpts o, const i128 *__restrict__ s,
                       const int *__restrict__ bad, PairState *__restrict__ st, double *__restrict__ u)
{
    extern __shared__ double sm_axis[];
    const int p = p0 + (int)blockIdx.x;
    const PairMeta pm = meta[p];
    const int d = o.d;
    double *xb = sm_axis, *yb = sm_axis + d;
    __shared__ double nrm[3];
    __shared__ int skip;
    if (threadIdx.x == 0) {
        // bad: bit 0 = an input value is non-finite or |v| >= 16 (set on the device),
        //      bit 1 = n < 2 or m < 2 (set by the host)
        st[p].status = (bad[p] & 1) ? ST_INVALID : (bad[p] & 2) ? ST_DEGENERATE : ST_OK;
        st[p].skipped = 1;
        st[p].count = 0ull;
        st[p].rechecked = 0ull;
        st[p].band_max_bits = 0u;
        st[p].n_gather = 0u;
        skip = 1;
    }
    __syncthreads();
    const bool do_align = o.align && !bad[p];
    if (!do_align) {
        for (int j = threadIdx.x; j < d; j += blockDim.x) u[(int64_t)p * d + j] = 0.0;
        return;
    }
    const i128 *sx = s + (int64_t)(2 * p) * d, *sy = sx + d;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        xb[j] = __ddiv_rn(fixed_to_f64(sx[j]), (double)pm.n);
        yb[j] = __ddiv_rn(fixed_to_f64(sy[j]), (double)pm.m);
    }
    __syncthreads();
    // ||x_bar||^2 and ||y_bar||^2: sequential FMA chains in index order
    if (threadIdx.x == 0 || threadIdx.x == 32) {
        const double *v = threadIdx.x ? yb : xb;
        double acc = 0.0;
        for (int j = 0; j < d; ++j) acc = __fma_rn(v[j], v[j], acc);
        nrm[threadIdx.x ? 1 : 0] = __dsqrt_rn(acc);
    }
    __syncthreads();
    const double nx = nrm[0], ny = nrm[1];
    if (!(nx > 0.0) || !(ny > 0.0)) {
        if (threadIdx.x == 0) st[p].status = ST_DEGENERATE;
        for (int j = threadIdx.x; j < d; j += blockDim.x) u[(int64_t)p * d + j] = 0.0;
        return;
    }
    for (int j = threadIdx.x; j < d; j += blockDim.x) xb[j] = __dsub_rn(__ddiv_rn(xb[j], nx), __ddiv_rn(yb[j], ny));
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int j = 0; j < d; ++j) acc = __fma_rn(xb[j], xb[j], acc);
        const double nv = __dsqrt_rn(acc);
        nrm[2] = nv;
        skip = !(nv > 0x1p-27);
        st[p].skipped = skip;
    }
    __syncthreads();
    const double nv = nrm[2];
    for (int j = threadIdx.x; j < d; j += blockDim.x) u[(int64_t)p * d + j] = skip ? 0.0 : __ddiv_rn(xb[j], nv);
}

// ---------------------------------------------------------------------------
// Reflection / copy into Z, one block (128 threads) per row chunk.
// ---------------------------------------------------------------------------
constexpr int RT = 32;  // columns per smem tile of the dot-product phase

template <int DT>
__device__ __forceinline__ void store_z(void *Z, int64_t idx, double v)
{
    if (DT == DT_F32) reinterpret_cast<float *>(Z)[idx] = __double2float_rn(v);
    else reinterpret_cast<unsigned short *>(Z)[idx] = f64_to_bf16_rn(v);
}

// BF16 storage, one step j of the compensated FP32 dot product u^T x of a row:
// u_j = uh + ul + e_j with |e_j| <= 2^-48 |u_j|; exact products uh x = p + e;
// the partial sums of p by TwoSum, their errors, e and ul x summed by a second
// TwoSum level; fa = sum |p| rounded up.
__device__ __forceinline__ void dot_step(float x, float uh, float ul, float &fs, float &fc, float &fcc, float &fa)
{
    const float p = __fmul_rn(uh, x);
    const float e = __fmaf_rn(uh, x, -p);
    const float q = __fmul_rn(ul, x);
    const float s1 = __fadd_rn(fs, p), bp = __fsub_rn(s1, fs);
    const float err = __fadd_rn(__fsub_rn(fs, __fsub_rn(s1, bp)), __fsub_rn(p, bp));
    fs = s1;
    const float wv = __fadd_rn(__fadd_rn(err, e), q);
    const float c1 = __fadd_rn(fc, wv), bw = __fsub_rn(c1, fc);
    fcc = __fadd_rn(fcc, __fadd_rn(__fsub_rn(fc, __fsub_rn(c1, bw)), __fsub_rn(wv, bw)));
    fc = c1;
    fa = __fadd_ru(fa, fabsf(p));
}

// a = -2 (ah + al) with ah + al = fs + (fc + fcc) (TwoSum); its distance to
// -2 c_chain is at most dl = 2 delta:
//   delta = A (2^-45 (d + 8) + 2 (d 2^-24)^3) + 2^-100, A = sum |uh x| (rounded up)
// which covers the FP32 roundings of the second level, the first-level error
// sums, the dropped ul x and e_j terms, |c_chain - u^T x| <= d 2^-53 sum |u x|,
// and products below the normal range
__device__ __forceinline__ void dot_finish(float fs, float fc, float fcc, float fa, int d, float &ah2, float &al2,
                                           float &dl)
{
    const float t = __fadd_rn(fc, fcc);
    const float ah = __fadd_rn(fs, t), bt = __fsub_rn(ah, fs);
    const float al = __fadd_rn(__fsub_rn(fs, __fsub_rn(ah, bt)), __fsub_rn(t, bt));
    const float dd = (float)d;
    const float g3 = __fmul_ru(dd, 0x1p-24f);
    const float K = __fadd_ru(__fmul_ru(__fadd_ru(dd, 8.0f), 0x1p-45f), __fmul_ru(2.0f, __fmul_ru(g3, __fmul_ru(g3, g3))));
    ah2 = -2.0f * ah;
    al2 = -2.0f * al;
    dl = __fmul_ru(2.0f, __fmaf_ru(fa, K, 0x1p-100f));
}

// BF16 storage, one reflected element v = fl64(a u_j + x), a = -2 c_chain,
// from the compensated values: x + (ah + al)(uh + ul) = S + yl = V + t up to
// 2^-44 (|x| + |P|), plus |u_j| dl for the distance of ah + al to a and
// 2^-52 |v| for the FP64 rounding (E).  With m the BF16 midpoint in |V|'s
// interval, |v| - m = (|V| - m) +- t +- E and |V| - m is exact: outside +-E
// (and with E + |t| under a quarter step) the sign decides the rounding
// (sure = true); otherwise (or for tiny V) the caller decides with the FP64
// chain and expression.
__device__ __forceinline__ unsigned short reflect_bf16_fast(float x, float ah, float al, float dl, float uh, float ul,
                                                            float auh, bool &sure)
{
    const float P = __fmul_rn(ah, uh), Pe = __fmaf_rn(ah, uh, -P);
    const float cross = __fmaf_rn(ah, ul, __fmul_rn(al, uh));
    const float S = __fadd_rn(x, P), bp = __fsub_rn(S, x);
    const float Se = __fadd_rn(__fsub_rn(x, __fsub_rn(S, bp)), __fsub_rn(P, bp));
    const float yl = __fadd_rn(Se, __fadd_rn(Pe, cross));
    // S + yl renormalised (TwoSum) to V + t with |t| <= 2^-24 |V|: under cancellation
    // yl can span several BF16 steps of the result
    const float V = __fadd_rn(S, yl), bv = __fsub_rn(V, S);
    const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(V, bv)), __fsub_rn(yl, bv));
    const float E = __fmaf_ru(__fadd_ru(fabsf(x), fabsf(P)), 0x1p-43f, __fmaf_ru(auh, __fmul_ru(dl, 1.01f), 0x1p-100f));
    const float aV = fabsf(V);
    const uint32_t tr = __float_as_uint(aV) & 0xffff0000u;
    const float dist = __fadd_rn(__fsub_rn(aV, __uint_as_float(tr | 0x8000u)), V < 0.0f ? -t : t);
    // a quarter of V's BF16 step: |v| stays between the neighbouring midpoints
    const float q4 = __uint_as_float((__float_as_uint(aV) & 0x7f800000u) - (9u << 23));
    sure = aV >= 0x1p-100f && fabsf(dist) > __fmul_ru(E, 1.0001f) && __fadd_ru(E, fabsf(t)) < q4;
    return (unsigned short)(((__float_as_uint(V) & 0x80000000u) | (tr + (dist > 0.0f ? 0x10000u : 0u))) >> 16);
}

// Two elements of one row (columns e, e + 1; xw holds their BF16 values, the
// lower column in the low half) with the operations of reflect_bf16_fast on
// packed FP32 pairs: each half rounds exactly as the scalar form, so the
// results and the `sure` decisions are the scalar ones.  Row constants: ah2,
// nah2 = -ah2, al2 (splat), dl101 = dl * 1.01 rounded up; column pairs uh2,
// ul2 and auh2 = |uh2|.  -P is not formed: fma(-ah, uh, P) = -Pe exactly, and
// cross + Pe = cross - (-Pe).
__device__ __forceinline__ uint32_t reflect_bf16_fast2(uint32_t xw, f2_t ah2, f2_t nah2, f2_t al2, f2_t dl101,
                                                       f2_t uh2, f2_t ul2, f2_t auh2, bool &sure0, bool &sure1)
{
    const f2_t x2 = f2_pack(__uint_as_float(xw << 16), __uint_as_float(xw & 0xffff0000u));
    const f2_t P = f2_mul(ah2, uh2), nPe = f2_fma(nah2, uh2, P);
    const f2_t cross = f2_fma(ah2, ul2, f2_mul(al2, uh2));
    const f2_t S = f2_add(x2, P), bp = f2_sub(S, x2);
    const f2_t Se = f2_add(f2_sub(x2, f2_sub(S, bp)), f2_sub(P, bp));
    const f2_t yl = f2_add(Se, f2_sub(cross, nPe));
    const f2_t V = f2_add(S, yl), bv = f2_sub(V, S);
    const f2_t t = f2_add(f2_sub(S, f2_sub(V, bv)), f2_sub(yl, bv));
    const f2_t K = f2_fma_ru(auh2, dl101, f2_splat(0x1p-100f));
    const f2_t E = f2_fma_ru(f2_add_ru(f2_abs(x2), f2_abs(P)), f2_splat(0x1p-43f), K);
    const f2_t aV = f2_abs(V);
    // per element: the truncated BF16 pattern, the midpoint above it, t signed like V
    const uint32_t av0 = (uint32_t)aV, av1 = (uint32_t)(aV >> 32);
    const uint32_t tr0 = av0 & 0xffff0000u, tr1 = av1 & 0xffff0000u;
    const f2_t mid = ((f2_t)(tr1 | 0x8000u) << 32) | (tr0 | 0x8000u);
    const f2_t ts = t ^ (V & 0x8000000080000000ull);
    const f2_t dist = f2_add(f2_sub(aV, mid), ts);
    const f2_t Eq = f2_mul_ru(E, f2_splat(1.0001f)), Et = f2_add_ru(E, f2_abs(t));
    float d0, d1, e0, e1, q0, q1;
    f2_unpack(dist, d0, d1);
    f2_unpack(Eq, e0, e1);
    f2_unpack(Et, q0, q1);
    // a quarter of V's BF16 step: |v| stays between the neighbouring midpoints
    const float s0 = __uint_as_float((av0 & 0x7f800000u) - (9u << 23)), s1 = __uint_as_float((av1 & 0x7f800000u) - (9u << 23));
    sure0 = __uint_as_float(av0) >= 0x1p-100f && fabsf(d0) > e0 && q0 < s0;
    sure1 = __uint_as_float(av1) >= 0x1p-100f && fabsf(d1) > e1 && q1 < s1;
    const uint32_t v0 = (uint32_t)V, v1 = (uint32_t)(V >> 32);
    const uint32_t z0 = ((v0 & 0x80000000u) | (tr0 + (d0 > 0.0f ? 0x10000u : 0u))) >> 16;
    const uint32_t z1 = ((v1 & 0x80000000u) | (tr1 + (d1 > 0.0f ? 0x10000u : 0u))) >> 16;
    return z0 | (z1 << 16);
}

// The exact FP64 dot product c = u^T x_r of the reference, a sequential FMA
// chain over j = 0..d-1, for the rare elements a BF16-storage reflection cannot
// decide from its compensated FP32 evaluation; -2c is kept in shared memory.
template <int DT>
__device__ __noinline__ double reflect_chain(const void *src, int64_t row, int d, const double *up)
{
    double c = 0.0;
    for (int j = 0; j < d; ++j)
        c = __fma_rn(up[j], f32_to_f64(__uint_as_float(load_f32bits(src, DT, row * d + j))), c);
    return -2.0 * c;  // exact scaling by -2
}

template <int DT>
__global__ void __launch_bounds__(128, 8) k_reflect(const PairMeta *__restrict__ meta, const RowChunk *__restrict__ chunks,
                                                 int c0, const RunOpts o, const PairState *__restrict__ st,
                                                 const double *__restrict__ u, void *__restrict__ Z,
                                                 unsigned int *__restrict__ colmax,
                                                 unsigned long long *__restrict__ colL1)
{
    __shared__ float xs[CHUNK_ROWS][RT + 1];
    __shared__ double us[RT];
    __shared__ float uh_s[RT], ul_s[RT];
    __shared__ double cs[CHUNK_ROWS];      // FP32 storage: -2c per row; BF16: -2c of fallback rows
    __shared__ float ah_s[CHUNK_ROWS], al_s[CHUNK_ROWS], dl_s[CHUNK_ROWS];
    __shared__ int chain_s[CHUNK_ROWS];    // BF16: cs[r] holds the exact -2c
    const RowChunk ch = chunks[c0 + (int)blockIdx.x];
    const PairMeta pm = meta[ch.pair];
    if (st[ch.pair].status != ST_OK) return;
    const int d = o.d;
    const void *src = ch.side ? pm.Y : pm.X;
    const int64_t zrow0 = pm.z_row + (ch.side ? pm.n : 0) + ch.row0;
    const bool reflect = !st[ch.pair].skipped && (ch.side == o.reflect_side);
    const double *up = u + (int64_t)ch.pair * d;

    if (reflect) {
        // FP32 storage: c_r = u^T x_r as the sequential FP64 FMA chain.  BF16 storage:
        // a compensated FP32 dot product instead (u_j = uh + ul + e_j with |e_j| <=
        // 2^-48 |u_j|; exact products uh x = p + e; the partial sums of p by TwoSum,
        // their errors, e and ul x summed by a second TwoSum level), with a rigorous
        // bound of its distance to the FP64 chain (one thread per row)
        double c = 0.0;
        float fs = 0.0f, fc = 0.0f, fcc = 0.0f, fa = 0.0f;
        for (int j0 = 0; j0 < d; j0 += RT) {
            const int w = min(RT, d - j0);
            // loads in batches of eight in flight before their stores (blockDim.x == 128)
            constexpr int PER = CHUNK_ROWS * RT / 128, LB = 8;
#pragma unroll 1
            for (int k0 = 0; k0 < PER; k0 += LB) {
                uint32_t xv[LB];
#pragma unroll
                for (int k = 0; k < LB; ++k) {
                    const int t = threadIdx.x + 128 * (k0 + k), r = t / RT, jj = t % RT;
                    xv[k] = (r < ch.nrows && jj < w) ? load_f32bits(src, DT, (int64_t)(ch.row0 + r) * d + j0 + jj)
                                                      : 0u;
                }
#pragma unroll
                for (int k = 0; k < LB; ++k) {
                    const int t = threadIdx.x + 128 * (k0 + k);
                    xs[t / RT][t % RT] = __uint_as_float(xv[k]);
                }
            }
            if (threadIdx.x < RT) {
                const double uu = threadIdx.x < w ? up[j0 + threadIdx.x] : 0.0;
                us[threadIdx.x] = uu;
                const float h = __double2float_rn(uu);
                uh_s[threadIdx.x] = h;
                ul_s[threadIdx.x] = __double2float_rn(__dsub_rn(uu, (double)h));
            }
            __syncthreads();
            if (threadIdx.x < ch.nrows) {
                const int r = threadIdx.x;
                if (DT == DT_F32) {
                    for (int jj = 0; jj < w; ++jj) c = __fma_rn(us[jj], f32_to_f64(xs[r][jj]), c);
                } else {
                    for (int jj = 0; jj < w; ++jj) dot_step(xs[r][jj], uh_s[jj], ul_s[jj], fs, fc, fcc, fa);
                }
            }
            __syncthreads();
        }
        const int r = threadIdx.x;
        if (DT == DT_F32) {
            cs[r] = -2.0 * c;  // exact scaling by -2
        } else {
            dot_finish(fs, fc, fcc, fa, d, ah_s[r], al_s[r], dl_s[r]);
            chain_s[r] = 0;
        }
        __syncthreads();
    }
    // element pass: z = fl_storage(fma(-2c, u_j, x)) or a copy
    constexpr int RB = 8;  // rows whose loads are issued together
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double uj = reflect ? up[j] : 0.0;
        const float uh = __double2float_rn(uj), ul = __double2float_rn(__dsub_rn(uj, (double)uh));
        const float auh = fabsf(uh);
        float mx = 0.0f, l1 = 0.0f;  // column maximum and sum of |z| (rounded up) over the chunk
        for (int rb = 0; rb < ch.nrows; rb += RB) {
        uint32_t xv[RB];
#pragma unroll
        for (int k = 0; k < RB; ++k)
            xv[k] = rb + k < ch.nrows ? load_f32bits(src, DT, (int64_t)(ch.row0 + rb + k) * d + j) : 0u;
#pragma unroll
        for (int k = 0; k < RB; ++k) {
            const int r = rb + k;
            if (r >= ch.nrows) break;
            const int64_t zi = (zrow0 + r) * d + j;
            const uint32_t xb = xv[k];
            float zf;
            if (reflect && DT == DT_BF16) {
                bool sure;
                unsigned short zb = reflect_bf16_fast(__uint_as_float(xb), ah_s[r], al_s[r], dl_s[r], uh, ul, auh, sure);
                if (!sure) {
                    if (!((volatile int *)chain_s)[r]) {  // another column's thread may be here too
                        ((volatile double *)cs)[r] = reflect_chain<DT>(src, ch.row0 + r, d, up);
                        __threadfence_block();
                        ((volatile int *)chain_s)[r] = 1;
                    }
                    zb = f64_to_bf16_rn(__fma_rn(((volatile double *)cs)[r], uj, f32_to_f64(__uint_as_float(xb))));
                }
                reinterpret_cast<unsigned short *>(Z)[zi] = zb;
                zf = __uint_as_float((uint32_t)zb << 16);
            } else if (reflect) {
                const double zv = __fma_rn(cs[r], uj, (double)__uint_as_float(xb));
                store_z<DT>(Z, zi, zv);
                zf = (DT == DT_F32) ? __double2float_rn(zv) : __uint_as_float((uint32_t)f64_to_bf16_rn(zv) << 16);
            } else {
                if (DT == DT_F32) reinterpret_cast<uint32_t *>(Z)[zi] = xb;
                else reinterpret_cast<unsigned short *>(Z)[zi] = (unsigned short)(xb >> 16);
                zf = __uint_as_float(xb);
            }
            mx = fmaxf(mx, fabsf(zf));
            l1 = __fadd_ru(l1, fabsf(zf));
        }
        }
        if (colmax) atomicMax(colmax + (int64_t)ch.pair * o.d_pad + j, __float_as_uint(mx));
        // an upper bound of the column's L1 norm in units of 2^-40 (integer atomics:
        // exact and order-free, so the slice grids do not depend on the schedule)
        if (colL1) atomicAdd(colL1 + (int64_t)ch.pair * o.d_pad + j, __float2ull_ru(__fmul_rn(l1, 0x1p40f)));
    }
}

// ---------------------------------------------------------------------------
// The same reflection for BF16 storage with d a multiple of 8, d <= 1024 and
// 16-byte aligned rows: the same arithmetic per row and per element, with
// 16-byte loads and stores and the next loads in flight while the current
// ones are consumed.  Dot products: tiles of 128 rows x 32 columns staged in
// shared memory (two buffers; the next tile is loaded into registers during
// the current tile's steps), one row per thread in column order.  Element
// pass: thread g owns the 8-column group g for every row of the chunk (its
// u values, maxima and L1 sums stay in registers), four rows per batch with
// the next batch in flight.
// ---------------------------------------------------------------------------
// The rare element the compensated evaluation cannot decide: the row's FP64
// chain (computed once per row by whichever thread needs it first) and the
// FP64 expression.  Out of line, so the unrolled element loop stays small.
__device__ __noinline__ uint32_t reflect_v_fallback(const void *src, int row, int r, int d, const double *up, int j,
                                                    uint32_t xb, double *cs, int *chain_s)
{
    if (!((volatile int *)chain_s)[r]) {  // another column's thread may be here too
        ((volatile double *)cs)[r] = reflect_chain<DT_BF16>(src, row, d, up);
        __threadfence_block();
        ((volatile int *)chain_s)[r] = 1;
    }
    return f64_to_bf16_rn(__fma_rn(((volatile double *)cs)[r], up[j], f32_to_f64(__uint_as_float(xb))));
}

constexpr int RV_T = 32;               // columns per dot-product tile
constexpr int RV_Q = RV_T / 8;         // 16-byte pieces per tile row
constexpr int RV_RB = 4;               // rows per element-pass batch

__global__ void __launch_bounds__(128, 4) k_reflect_v(const PairMeta *__restrict__ meta,
                                                     const RowChunk *__restrict__ chunks, int c0, const RunOpts o,
                                                     const PairState *__restrict__ st, const double *__restrict__ u,
                                                     void *__restrict__ Z, unsigned int *__restrict__ colmax,
                                                     unsigned long long *__restrict__ colL1)
{
    __shared__ uint4 xt[2][CHUNK_ROWS][RV_Q + 1];  // +1: conflict-free row reads
    __shared__ float uh_s[1024], ul_s[1024];
    __shared__ double cs[CHUNK_ROWS];
    __shared__ float ah_s[CHUNK_ROWS], al_s[CHUNK_ROWS], dl_s[CHUNK_ROWS];
    __shared__ int chain_s[CHUNK_ROWS];
    const RowChunk ch = chunks[c0 + (int)blockIdx.x];
    const PairMeta pm = meta[ch.pair];
    if (st[ch.pair].status != ST_OK) return;
    const int d = o.d, G = d / 8, t = threadIdx.x;
    const uint4 *src = reinterpret_cast<const uint4 *>(ch.side ? pm.Y : pm.X) + (int64_t)ch.row0 * G;
    uint4 *dst = reinterpret_cast<uint4 *>(Z) + (pm.z_row + (ch.side ? pm.n : 0) + ch.row0) * (int64_t)G;
    const bool reflect = !st[ch.pair].skipped && (ch.side == o.reflect_side);
    const double *up = u + (int64_t)ch.pair * d;
    const int nr = ch.nrows;

    if (reflect) {
        for (int j = t; j < d; j += blockDim.x) {
            const double uu = up[j];
            const float h = __double2float_rn(uu);
            uh_s[j] = h;
            ul_s[j] = __double2float_rn(__dsub_rn(uu, (double)h));
        }
        // piece k = t + 128 i of a tile: row k / RV_Q, 8-column piece k % RV_Q
        const int ntile = (d + RV_T - 1) / RV_T;
        uint4 pre[RV_Q];
        auto load_tile = [&](int tt) {
#pragma unroll
            for (int i = 0; i < RV_Q; ++i) {
                const int k = t + 128 * i, r = k / RV_Q, q = k % RV_Q, g = tt * RV_Q + q;
                pre[i] = (r < nr && g < G) ? __ldg(src + (int64_t)r * G + g) : make_uint4(0u, 0u, 0u, 0u);
            }
        };
        load_tile(0);
        float fs = 0.0f, fc = 0.0f, fcc = 0.0f, fa = 0.0f;
        for (int tt = 0; tt < ntile; ++tt) {
            uint4 (*buf)[RV_Q + 1] = xt[tt & 1];
#pragma unroll
            for (int i = 0; i < RV_Q; ++i) {
                const int k = t + 128 * i;
                buf[k / RV_Q][k % RV_Q] = pre[i];
            }
            __syncthreads();  // the tile is in; uh_s/ul_s too (first tile)
            if (tt + 1 < ntile) load_tile(tt + 1);
            if (t < nr) {
                const int j0 = tt * RV_T, w = min(RV_T, d - j0);
                for (int q = 0; q < w / 8; ++q) {
                    const uint4 v = buf[t][q];
                    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float x = __uint_as_float((e & 1) ? (wv[e >> 1] & 0xffff0000u) : (wv[e >> 1] << 16));
                        const int j = j0 + 8 * q + e;
                        dot_step(x, uh_s[j], ul_s[j], fs, fc, fcc, fa);
                    }
                }
            }
        }
        if (t < nr) {
            dot_finish(fs, fc, fcc, fa, d, ah_s[t], al_s[t], dl_s[t]);
            chain_s[t] = 0;
        }
        __syncthreads();
    }

    // element pass: thread g < G owns columns 8g .. 8g + 7, two at a time on packed
    // FP32 pairs (reflect_bf16_fast2)
    if (t < G) {
        f2_t uh2[4], ul2[4], auh2[4];
        float mx[8], l1[8];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = 8 * t + 2 * h;
            uh2[h] = reflect ? f2_pack(uh_s[j], uh_s[j + 1]) : 0ull;
            ul2[h] = reflect ? f2_pack(ul_s[j], ul_s[j + 1]) : 0ull;
            auh2[h] = f2_abs(uh2[h]);
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) mx[e] = l1[e] = 0.0f;
        uint4 cur[RV_RB], nxt[RV_RB];
#pragma unroll
        for (int k = 0; k < RV_RB; ++k) cur[k] = k < nr ? __ldg(src + (int64_t)k * G + t) : make_uint4(0u, 0u, 0u, 0u);
        for (int rb = 0; rb < nr; rb += RV_RB) {
#pragma unroll
            for (int k = 0; k < RV_RB; ++k) {
                const int r = rb + RV_RB + k;
                nxt[k] = r < nr ? __ldg(src + (int64_t)r * G + t) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int k = 0; k < RV_RB; ++k) {
                const int r = rb + k;
                if (r >= nr) break;
                const uint32_t wv[4] = {cur[k].x, cur[k].y, cur[k].z, cur[k].w};
                uint32_t ow[4];
                f2_t ah2 = 0ull, nah2 = 0ull, al2 = 0ull, dl101 = 0ull;
                if (reflect) {
                    ah2 = f2_splat(ah_s[r]);
                    nah2 = f2_splat(-ah_s[r]);
                    al2 = f2_splat(al_s[r]);
                    dl101 = f2_splat(__fmul_ru(dl_s[r], 1.01f));
                }
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    uint32_t zw = wv[h];  // the unreflected side keeps its values
                    if (reflect) {
                        bool s0, s1;
                        zw = reflect_bf16_fast2(wv[h], ah2, nah2, al2, dl101, uh2[h], ul2[h], auh2[h], s0, s1);
                        if (!s0)
                            zw = (zw & 0xffff0000u) | reflect_v_fallback(ch.side ? pm.Y : pm.X, ch.row0 + r, r, d, up,
                                                                         8 * t + 2 * h, wv[h] << 16, cs, chain_s);
                        if (!s1)
                            zw = (zw & 0xffffu) | (reflect_v_fallback(ch.side ? pm.Y : pm.X, ch.row0 + r, r, d, up,
                                                                      8 * t + 2 * h + 1, wv[h] & 0xffff0000u, cs,
                                                                      chain_s)
                                                   << 16);
                    }
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const int e = 2 * h + s2;
                        const float zf = __uint_as_float(s2 ? (zw & 0xffff0000u) : (zw << 16));
                        mx[e] = fmaxf(mx[e], fabsf(zf));
                        l1[e] = __fadd_ru(l1[e], fabsf(zf));
                    }
                    ow[h] = zw;
                }
                dst[(int64_t)r * G + t] = make_uint4(ow[0], ow[1], ow[2], ow[3]);
            }
#pragma unroll
            for (int k = 0; k < RV_RB; ++k) cur[k] = nxt[k];
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int64_t ci = (int64_t)ch.pair * o.d_pad + 8 * t + e;
            if (colmax) atomicMax(colmax + ci, __float_as_uint(mx[e]));
            if (colL1) atomicAdd(colL1 + ci, __float2ull_ru(__fmul_rn(l1[e], 0x1p40f)));
        }
    }
}

// ---------------------------------------------------------------------------
// Z statistics and fixed-point slices, one block (256 threads) per row chunk.
// ---------------------------------------------------------------------------

// scale exponent E of column j: max |z| < 2^E; q_hi = 2^(E-8)
__device__ __forceinline__ float qhi_from_max(unsigned int maxbits)
{
    const int e = (int)((maxbits >> 23) & 0xffu);
    if (maxbits == 0u) return 1.0f;
    const int E = e - 126;
    return ldexpf(1.0f, E - 8);
}

// Exact hi/lo(/lo2) split of z on its column's fixed-point grid: every step
// is exact in FP32; `res` is what the slices leave out.  |z| < 256 q_hi, so
// |hi| <= 256; the lower slices use grids 512x finer, so |lo|, |lo2| <= 256.
// Integers of magnitude <= 256 are exact in BF16.
__device__ __forceinline__ void fixed_split(float z, float qh, int S, float &hi, float &lo, float &lo2, float &res)
{
    const float ql = qh * (1.0f / 512.0f), ql2 = ql * (1.0f / 512.0f);
    if (qh <= 1.0f && qh >= 0x1p-100f) {
        // scaling by the exact reciprocal 2^-k (k >= 0) is exact, as the quotient is
        const float inv = __int_as_float((254 - ((__float_as_int(qh) >> 23) & 0xff)) << 23);
        hi = rintf(__fmul_rn(z, inv));
        const float w = __fsub_rn(z, __fmul_rn(hi, qh));
        lo = rintf(__fmul_rn(w, inv * 512.0f));
        res = __fsub_rn(w, __fmul_rn(lo, ql));
        lo2 = 0.0f;
        if (S == 3) {
            lo2 = rintf(__fmul_rn(res, inv * 262144.0f));
            res = __fsub_rn(res, __fmul_rn(lo2, ql2));
        }
        return;
    }
    hi = rintf(z / qh);
    const float w = __fsub_rn(z, __fmul_rn(hi, qh));
    lo = rintf(w / ql);
    res = __fsub_rn(w, __fmul_rn(lo, ql));
    lo2 = 0.0f;
    if (S == 3) {
        lo2 = rintf(res / ql2);
        res = __fsub_rn(res, __fmul_rn(lo2, ql2));
    }
}

// The slice matrix holds slice s of column j in row s * d_pad + j, over the
// token positions of all pairs side by side (each pair from its z_row), in
// blocks of 64 tokens: block k holds every row's tokens 64k .. 64k + 63
// (128 bytes a row), so that one TMA box (64 tokens x up to 128 rows) is one
// contiguous piece and a pair's slices one contiguous range, whatever the
// batch size (rows of all pairs' tokens would put every row of a box on its
// own memory page).
__device__ __forceinline__ int64_t slice_row(int j, int s, int d_pad) { return (int64_t)s * d_pad + j; }
__device__ __forceinline__ int64_t zq_index(int64_t t, int64_t row, int64_t zq_rows)
{
    return ((t >> 6) * zq_rows + row) * 64 + (t & 63);
}
// BF16 grid slices also interleave the two halves of every 32-token group of
// a pair: pair token t sits at position slice_pos(t) = 32 (t / 32) +
// 2 (t % 16) + (t / 16) % 2, i.e. the order 0, 16, 1, 17, ..., 15, 31.  The
// GEMM sums over positions, so any order serves; this one puts tokens j and
// j + 16 into one 32-bit word of the K dimension, which are bits j and j + 16
// of a label word: two operations expand a word, with no bit shuffle.  FP32
// fixed-point slices keep the token order.
__device__ __forceinline__ int64_t slice_pos(int64_t t) { return (t & ~(int64_t)31) | ((t & 15) << 1) | ((t >> 4) & 1); }

// One block (256 threads) per row chunk, tiles of ZS_T columns.  Phase A:
// thread (column, 16-row part) reads its values (coalesced across columns),
// adds them exactly to the column totals, splits each once into its slices
// (staged transposed in shared memory) and sums the residuals; phase B stores
// the slices token-contiguous.  FP32 storage: three fixed-point slices of
// the column's scale; BF16 storage: the two grid slices (l1_split).
constexpr int ZS_T = 32;
constexpr int ZS_PARTS = 256 / ZS_T;               // 8 parts of 16 rows
constexpr int ZS_ROWS = CHUNK_ROWS / ZS_PARTS;     // 16

template <int DT>
__global__ void __launch_bounds__(256) k_zstats_partial(const PairMeta *__restrict__ meta,
                                                        const RowChunk *__restrict__ chunks, int c0,
                                                        const RunOpts o,
                                                        const PairState *__restrict__ st, const void *__restrict__ Z,
                                                        const unsigned int *__restrict__ colmax,
                                                        const unsigned long long *__restrict__ colL1,
                                                        i128 *__restrict__ tpart, float *__restrict__ cpart,
                                                        float *__restrict__ cpart1,
                                                        unsigned short *__restrict__ zq)
{
    __shared__ unsigned short sq[3][ZS_T][CHUNK_ROWS + 2];
    __shared__ i128 acc_s[ZS_PARTS][ZS_T];
    __shared__ float cacc_s[ZS_PARTS][ZS_T], cacc1_s[ZS_PARTS][ZS_T];
    const int ci = c0 + (int)blockIdx.x;  // chunk index
    const RowChunk ch = chunks[ci];
    const PairMeta pm = meta[ch.pair];
    if (st[ch.pair].status != ST_OK) return;
    const int d = o.d;
    const int64_t tok0 = (ch.side ? pm.n : 0) + ch.row0;  // token index within the pair
    const int64_t zrow0 = pm.z_row + tok0;
    const bool mixed = (o.path == 0);
    const int S = o.slices;
    // the last chunk of the pair also zero-fills the padded tokens of the slices
    const bool last = ch.side == 1 && ch.row0 + ch.nrows == pm.m;
    const int npad = last ? pm.N_pad - pm.N : 0;
    const int jj = threadIdx.x % ZS_T, part = threadIdx.x / ZS_T;

    for (int j0 = 0; j0 < d; j0 += ZS_T) {
        const int j = j0 + jj;
        const unsigned int mb = j < d ? colmax[(int64_t)ch.pair * o.d_pad + j] : 0u;
        const float qh = qhi_from_max(mb);
        L1Grid G{};
        if (mixed && DT == DT_BF16) G = l1_grid(j < d ? colL1[(int64_t)ch.pair * o.d_pad + j] : 0ull, pm.N);
        WinAcc wa;
        wa.init(col_bound_exp(mb));
        float cacc = 0.0f, cacc1 = 0.0f;
        const int r0 = part * ZS_ROWS, nr = max(0, min(ch.nrows - r0, ZS_ROWS));
        // this thread's values first (all loads in flight), then the arithmetic
        uint32_t bv[ZS_ROWS];
#pragma unroll
        for (int k = 0; k < ZS_ROWS; ++k) bv[k] = (k < nr && j < d) ? load_f32bits(Z, DT, (zrow0 + r0 + k) * d + j) : 0u;
#pragma unroll
        for (int k = 0; k < ZS_ROWS; ++k) {
            if (k >= nr) break;
            const int r = r0 + k;
            const uint32_t b = bv[k];
            wa.add(b);
            const float z = __uint_as_float(b);
            if (mixed && DT == DT_BF16) {
                float k1, k2, r1, r2;
                l1_split(z, G, k1, k2, r1, r2);
                cacc = __fadd_ru(cacc, fabsf(r2));
                cacc1 = __fadd_ru(cacc1, fabsf(r1));
                // k1 g and k2 g2 have at most 8 significant bits: BF16 exactly
                sq[0][jj][r] = (unsigned short)(__float_as_uint(__fmul_rn(k1, G.g)) >> 16);
                sq[1][jj][r] = (unsigned short)(__float_as_uint(__fmul_rn(k2, G.g2)) >> 16);
            } else if (mixed) {
                float hi, lo, lo2, res;
                fixed_split(z, qh, S, hi, lo, lo2, res);
                cacc = __fadd_ru(cacc, fabsf(res));
                sq[0][jj][r] = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
                sq[1][jj][r] = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
                if (S == 3) sq[2][jj][r] = __bfloat16_as_ushort(__float2bfloat16_rn(lo2));
            } else {
                cacc = __fadd_ru(cacc, fabsf(z));
            }
        }
        acc_s[part][jj] = wa.total();
        cacc_s[part][jj] = cacc;
        cacc1_s[part][jj] = cacc1;
        __syncthreads();
        if (mixed) {
            // warp per column, lanes along tokens: token-contiguous stores
            const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
            for (int c = wp; c < ZS_T && j0 + c < d; c += (int)(blockDim.x >> 5)) {
                for (int s = 0; s < S; ++s) {
                    const int64_t row = slice_row(j0 + c, s, o.d_pad), zr = (int64_t)S * o.d_pad;
                    if (DT == DT_BF16) {
                        for (int r = ln; r < ch.nrows; r += 32)
                            zq[zq_index(pm.z_row + slice_pos(tok0 + r), row, zr)] = sq[s][c][r];
                        for (int k = ln; k < npad; k += 32) zq[zq_index(pm.z_row + slice_pos(pm.N + k), row, zr)] = 0;
                    } else {
                        for (int r = ln; r < ch.nrows; r += 32) zq[zq_index(pm.z_row + tok0 + r, row, zr)] = sq[s][c][r];
                        for (int k = ln; k < npad; k += 32) zq[zq_index(pm.z_row + pm.N + k, row, zr)] = 0;
                    }
                }
            }
        }
        if (threadIdx.x < ZS_T && j0 + threadIdx.x < d) {
            i128 a = 0;
            float c = 0.0f, c1 = 0.0f;
            for (int q = 0; q < ZS_PARTS; ++q) {
                a += acc_s[q][threadIdx.x];
                c = __fadd_ru(c, cacc_s[q][threadIdx.x]);
                c1 = __fadd_ru(c1, cacc1_s[q][threadIdx.x]);
            }
            tpart[(int64_t)ci * d + j0 + threadIdx.x] = a;
            cpart[(int64_t)ci * d + j0 + threadIdx.x] = c;
            cpart1[(int64_t)ci * d + j0 + threadIdx.x] = c1;
        }
        __syncthreads();
    }
}

// The same outputs for the tensor-core path on BF16 storage with d a
// multiple of 8, with lanes along tokens.  Warp w takes the 8-column groups
// w, w + 8, ... ; the chunk lies in a window of four 32-token groups that
// starts g = tok0 mod 32 tokens before it (the host keeps g + nrows <= 128),
// and lane l takes the window's tokens 32 (l / 8) + {2k, 2k + 1, 2k + 16,
// 2k + 17}, k = l % 8, whose slice positions 32 (l / 8) + 4k .. + 3 are
// contiguous (slice_pos), so that a lane's four values of one slice column
// leave in one aligned 8-byte store.  The column
// total is k_sum g + k2_sum g2 (integer warp sums of the slice multiples)
// plus the rare nonzero second residuals added exactly out of line (columns
// outside the split range add every value exactly, with the oracle's rule
// that |v| < 2^-64 counts as 0), so every chunk total is the exact sum of its
// values.
__device__ __forceinline__ i128 warp_sum_i128(i128 v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const u128 u = (u128)v;
        const uint32_t w0 = __shfl_xor_sync(0xffffffffu, (uint32_t)u, off);
        const uint32_t w1 = __shfl_xor_sync(0xffffffffu, (uint32_t)(u >> 32), off);
        const uint32_t w2 = __shfl_xor_sync(0xffffffffu, (uint32_t)(u >> 64), off);
        const uint32_t w3 = __shfl_xor_sync(0xffffffffu, (uint32_t)(u >> 96), off);
        v += (i128)(((u128)w3 << 96) | ((u128)w2 << 64) | ((u128)w1 << 32) | (u128)w0);
    }
    return v;
}

__device__ __forceinline__ float warp_sum_ru(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Exact fixed-point value (unit 2^-87) of a second residual: a nonzero
// residual of a value z >= 2^-64 is a multiple of z's last bit, so >= 2^-71
// and a multiple of 2^-87 (the right shift below drops only zero bits).
__device__ __forceinline__ i128 fixed_from_residual(uint32_t b)
{
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u) return 0;
    const uint64_t mant = (b & 0x7fffffu) | 0x800000u;
    const u128 m = e >= 63u ? (u128)mant << (e - 63u) : (u128)(mant >> min(63u - e, 63u));
    return (b >> 31) ? -(i128)m : (i128)m;
}

// The exact part of one column of a warp's 128 positions, called by the whole
// warp (out of line: rare): split columns add their second residuals, the
// others every value (|v| < 2^-64 counts as 0).
__device__ __noinline__ i128 zs_slow_column(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, bool high,
                                            unsigned int okm, const L1Grid G)
{
    i128 sl = 0;
    const uint32_t ws[4] = {w0, w1, w2, w3};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (!((okm >> i) & 1u)) continue;
        const uint32_t bb = high ? (ws[i] & 0xffff0000u) : (ws[i] << 16);
        if (!G.split) {
            sl += fixed_from_f32bits(bb);
        } else {
            float k, k2, r1, r2;
            l1_split(__uint_as_float(bb), G, k, k2, r1, r2);
            if (r2 != 0.0f) sl += fixed_from_residual(__float_as_uint(r2));
        }
    }
    return warp_sum_i128(sl);
}

__global__ void __launch_bounds__(256, 3) k_zstats_tok(const PairMeta *__restrict__ meta,
                                                    const RowChunk *__restrict__ chunks, int c0, const RunOpts o,
                                                    const PairState *__restrict__ st, const uint4 *__restrict__ Z,
                                                    const unsigned long long *__restrict__ colL1,
                                                    i128 *__restrict__ tpart, float *__restrict__ cpart,
                                                    float *__restrict__ cpart1,
                                                    unsigned short *__restrict__ zq)
{
    const int ci = c0 + (int)blockIdx.x;  // chunk index
    const RowChunk ch = chunks[ci];
    const PairMeta pm = meta[ch.pair];
    if (st[ch.pair].status != ST_OK) return;
    const int d = o.d, d_pad = o.d_pad;
    const int64_t tok0 = (ch.side ? pm.n : 0) + ch.row0;  // token index within the pair
    const int g = (int)(tok0 & 31);
    const bool last = ch.side == 1 && ch.row0 + ch.nrows == pm.m;
    const int npad = last ? pm.N_pad - pm.N : 0;
    const int wp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    // chunk rows of the lane's four tokens 2k, 2k + 1, 2k + 16, 2k + 17 of its group
    const int wb = 32 * (ln >> 3) + 2 * (ln & 7) - g;
    const int rbi[4] = {wb, wb + 1, wb + 16, wb + 17};
    bool ok[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) ok[i] = rbi[i] >= 0 && rbi[i] < ch.nrows;
    const bool full = ok[0] && ok[1] && ok[2] && ok[3];
    const unsigned int okm = (ok[0] ? 1u : 0u) | (ok[1] ? 2u : 0u) | (ok[2] ? 4u : 0u) | (ok[3] ? 8u : 0u);
    // position of the lane's first value (token 2k; then 2k + 16, 2k + 1, 2k + 17)
    const int64_t tq = pm.z_row + tok0 - g + 32 * (ln >> 3) + 4 * (ln & 7);
    const unsigned long long *cl = colL1 + (int64_t)ch.pair * d_pad;
    const int d16 = d / 8;  // 16-byte units per row
    // row of the chunk's first token in 16-byte units; only rows with ok[i] are read
    const int64_t zr = (pm.z_row + tok0) * d16;
    const int64_t zrows = 2 * (int64_t)d_pad;      // rows of the slice matrix (two BF16 grid slices)
    const int64_t lo_off = (int64_t)d_pad * 64;     // second slice: d_pad rows further in the token block

    for (int c8 = wp; c8 < d16; c8 += 8) {
        const int j = 8 * c8;
        uint4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = ok[i] ? __ldg(Z + zr + (int64_t)rbi[i] * d16 + c8) : make_uint4(0u, 0u, 0u, 0u);
        unsigned short *dh = zq + zq_index(tq, j, zrows);  // the lane's 4 positions lie in one 64-token block
        // lane e < 8 keeps column j + e's reductions
        int my_ik = 0, my_ik2 = 0, my_eg = 0, my_eg2 = 0;
        bool my_split = false;
        i128 my_slow = 0;
        float my_c = 0.0f, my_c1 = 0.0f;
        const ulonglong2 l01 = __ldg(reinterpret_cast<const ulonglong2 *>(cl + j));
        const ulonglong2 l23 = __ldg(reinterpret_cast<const ulonglong2 *>(cl + j) + 1);
        const ulonglong2 l45 = __ldg(reinterpret_cast<const ulonglong2 *>(cl + j) + 2);
        const ulonglong2 l67 = __ldg(reinterpret_cast<const ulonglong2 *>(cl + j) + 3);
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const unsigned long long lb = e == 0 ? l01.x : e == 1 ? l01.y : e == 2 ? l23.x : e == 3 ? l23.y
                                        : e == 4 ? l45.x : e == 5 ? l45.y : e == 6 ? l67.x : l67.y;
            const L1Grid G = l1_grid(lb, pm.N);
            float kf[4], k2f[4];
            // the slice multiples k, k2 are integers whose magnitudes over all of the
            // pair's tokens sum to less than 2^24 (l1_grid), so FP32 sums of any of them
            // are exact; one conversion per lane instead of one per value
            float fk = 0.0f, fk2 = 0.0f;
            float ra1 = 0.0f, ra2 = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t wd = (e >> 1) == 0 ? v[i].x : (e >> 1) == 1 ? v[i].y : (e >> 1) == 2 ? v[i].z : v[i].w;
                const float z = __uint_as_float((e & 1) ? (wd & 0xffff0000u) : (wd << 16));  // 0 where !ok
                float r1, r2;
                l1_split(z, G, kf[i], k2f[i], r1, r2);
                fk += kf[i];
                fk2 += k2f[i];
                ra1 = __fadd_ru(ra1, fabsf(r1));
                ra2 = __fadd_ru(ra2, fabsf(r2));  // 0 iff every second residual is 0
                kf[i] = __fmul_rn(kf[i], G.g);    // the slice values (exact)
                k2f[i] = __fmul_rn(k2f[i], G.g2);
            }
            const int sk = __float2int_rz(fk), sk2 = __float2int_rz(fk2);
            // the slice values have at most 8 significant bits: the high halves of
            // their FP32 bits are their BF16 bits; positions in the order of tokens
            // 2k, 2k + 16, 2k + 1, 2k + 17 (values 0, 2, 1, 3)
            const uint32_t hp0 = __byte_perm(__float_as_uint(kf[0]), __float_as_uint(kf[2]), 0x7632);
            const uint32_t hp1 = __byte_perm(__float_as_uint(kf[1]), __float_as_uint(kf[3]), 0x7632);
            const uint32_t lp0 = __byte_perm(__float_as_uint(k2f[0]), __float_as_uint(k2f[2]), 0x7632);
            const uint32_t lp1 = __byte_perm(__float_as_uint(k2f[1]), __float_as_uint(k2f[3]), 0x7632);
            unsigned short *dl = dh + lo_off;
            if (full) {
                *reinterpret_cast<uint2 *>(dh) = make_uint2(hp0, hp1);
                *reinterpret_cast<uint2 *>(dl) = make_uint2(lp0, lp1);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (ok[(q >> 1) | ((q & 1) << 1)]) {  // position q holds value 0, 2, 1, 3
                        const uint32_t hp = q < 2 ? hp0 : hp1, lp = q < 2 ? lp0 : lp1;
                        dh[q] = (unsigned short)((q & 1) ? hp >> 16 : hp);
                        dl[q] = (unsigned short)((q & 1) ? lp >> 16 : lp);
                    }
            }
            dh += 64;  // the next row of the block
            const int ik = __reduce_add_sync(0xffffffffu, sk);
            const int ik2 = __reduce_add_sync(0xffffffffu, sk2);
            const float c1 = __any_sync(0xffffffffu, ra1 != 0.0f) ? warp_sum_ru(ra1) : 0.0f;
            float c2 = 0.0f;
            i128 slow = 0;
            if (__any_sync(0xffffffffu, !G.split || ra2 != 0.0f)) {
                c2 = warp_sum_ru(ra2);
                const uint32_t w0 = (e >> 1) == 0 ? v[0].x : (e >> 1) == 1 ? v[0].y : (e >> 1) == 2 ? v[0].z : v[0].w;
                const uint32_t w1 = (e >> 1) == 0 ? v[1].x : (e >> 1) == 1 ? v[1].y : (e >> 1) == 2 ? v[1].z : v[1].w;
                const uint32_t w2 = (e >> 1) == 0 ? v[2].x : (e >> 1) == 1 ? v[2].y : (e >> 1) == 2 ? v[2].z : v[2].w;
                const uint32_t w3 = (e >> 1) == 0 ? v[3].x : (e >> 1) == 1 ? v[3].y : (e >> 1) == 2 ? v[3].z : v[3].w;
                slow = zs_slow_column(w0, w1, w2, w3, (e & 1) != 0, okm, G);
            }
            if (ln == e) {
                my_ik = ik;
                my_ik2 = ik2;
                my_eg = G.eg;
                my_eg2 = G.eg2;
                my_split = G.split;
                my_slow = slow;
                my_c = c2;
                my_c1 = c1;
            }
        }
        if (ln < 8) {
            i128 tot = my_slow;
            if (my_split) tot += ((i128)my_ik << (my_eg + 87)) + ((i128)my_ik2 << (my_eg2 + 87));
            tpart[(int64_t)ci * d + j + ln] = tot;
            cpart[(int64_t)ci * d + j + ln] = my_c;
            cpart1[(int64_t)ci * d + j + ln] = my_c1;
        }
        // the last chunk of the pair also zero-fills the padded tokens of the slices
        for (int k = ln; k < 16 * npad; k += 32) {
            const int e = k / (2 * npad), s = (k / npad) & 1, t = k % npad;
            zq[zq_index(pm.z_row + slice_pos(pm.N + t), slice_row(j + e, s, d_pad), zrows)] = 0;
        }
    }
}

// Per (pair, column) of pairs p0 .. p1-1: exact totals, observed group-1 sums,
// band constants.
__global__ void k_zstats_reduce(const PairMeta *__restrict__ meta, int p0, int p1, const RunOpts o,
                                const PairState *__restrict__ st, const unsigned int *__restrict__ colmax,
                                const i128 *__restrict__ tpart, const float *__restrict__ cpart,
                                const float *__restrict__ cpart1, i128 *__restrict__ t_ex, i128 *__restrict__ s1o,
                                ColConst *__restrict__ cc, float *__restrict__ ct)
{
    const int d = o.d;
    const int64_t idx = (int64_t)p0 * o.d_pad + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)p1 * o.d_pad) return;
    const int p = (int)(idx / o.d_pad), j = (int)(idx % o.d_pad);
    const PairMeta pm = meta[p];
    ColConst c{0.0f, 0.0f, 0.0f, 0.0f};
    if (j >= d || st[p].status != ST_OK) {
        cc[idx] = c;
        ct[idx] = 0.0f;
        if (j < d) {
            t_ex[(int64_t)p * d + j] = 0;
            s1o[(int64_t)p * d + j] = 0;
        }
        return;
    }
    i128 a = 0, ax = 0;
    float csum = 0.0f, csum1 = 0.0f;
    for (int k = 0; k < pm.nchunk_x + pm.nchunk_y; ++k) {
        const int64_t q = (int64_t)(pm.chunk0 + k) * d + j;
        a += tpart[q];
        if (k < pm.nchunk_x) ax += tpart[q];
        csum = __fadd_ru(csum, cpart[q]);
        if (o.path == 0 && o.dtype == DT_BF16) csum1 = __fadd_ru(csum1, cpart1[q]);
    }
    t_ex[(int64_t)p * d + j] = a;
    s1o[(int64_t)p * d + j] = ax;
    c.t = __double2float_rn(fixed_to_f64(a));
    if (o.path == 0) {
        // FP32 storage: fixed-point slices of scale 2^(E-8); BF16: the slices hold values
        c.q_hi = o.dtype == DT_BF16 ? 1.0f : qhi_from_max(colmax[idx]);
        c.c = csum;    // sum of |residuals| of all slices
        c.c1 = csum1;  // BF16: sum of |residuals| of the first slice alone
    } else {
        // sequential FP32 accumulation over K = N_pad tokens: gamma_K = K u / (1 - K u)
        const float K = (float)pm.N_pad;
        const float gam = __fdiv_ru(K * U32, 1.0f - K * U32);
        c.q_hi = 0.5f;
        c.c = __fmul_ru(gam, csum);
    }
    cc[idx] = c;
    ct[idx] = c.t;
}

// ---------------------------------------------------------------------------
// Observed statistic, one block of 64 threads per pair (p0 + block); dynamic
// smem 2*d doubles.
// ---------------------------------------------------------------------------
__global__ void k_tobs(const PairMeta *__restrict__ meta, int p0, const RunOpts o, const i128 *__restrict__ t_ex,
                       const i128 *__restrict__ s1o, const ColConst *__restrict__ cc, PairState *__restrict__ st)
{
    extern __shared__ double sm_tobs[];
    const int p = p0 + (int)blockIdx.x;
    if (st[p].status != ST_OK) return;
    const PairMeta pm = meta[p];
    const int d = o.d;
    double *a = sm_tobs, *b = sm_tobs + d;
    __shared__ double q[2];
    __shared__ float red[3][64];
    float tn = 0.0f, c2 = 0.0f, c21 = 0.0f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const i128 x = s1o[(int64_t)p * d + j];
        a[j] = fixed_to_f64(x);
        b[j] = fixed_to_f64(t_ex[(int64_t)p * d + j] - x);
        const ColConst c = cc[(int64_t)p * o.d_pad + j];
        tn = fmaf(c.t, c.t, tn);
        c2 = __fmaf_ru(c.c, c.c, c2);
        c21 = __fmaf_ru(c.c1, c.c1, c21);
    }
    red[0][threadIdx.x] = tn;
    red[1][threadIdx.x] = c2;
    red[2][threadIdx.x] = c21;
    __syncthreads();
    if (threadIdx.x == 0 || threadIdx.x == 32) {
        const double *v = threadIdx.x ? b : a;
        double acc = 0.0;
        for (int j = 0; j < d; ++j) acc = __fma_rn(v[j], v[j], acc);
        q[threadIdx.x ? 1 : 0] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float T = 0.0f, C = 0.0f, C1 = 0.0f;
        for (int k = 0; k < 64; ++k) {
            T += red[0][k];
            C = __fadd_ru(C, red[1][k]);
            C1 = __fadd_ru(C1, red[2][k]);
        }
        const double n = (double)pm.n, m = (double)pm.m, dd = (double)d;
        const double A1 = group_value_f64(o.stat, q[0], n, dd);
        const double A2 = group_value_f64(o.stat, q[1], m, dd);
        PairState &s = st[p];
        s.A1o = A1;
        s.A2o = A2;
        s.To = stat_T_f64(o.stat, A1, A2);
        s.rx = __dsqrt_rn(__ddiv_rn(q[0], __dmul_rn(n, n)));
        s.ry = __dsqrt_rn(__ddiv_rn(q[1], __dmul_rn(m, m)));
        s.tnorm = sqrtf(T) * (1.0f + 1e-4f);
        s.sumc2 = C * (1.0f + 1e-4f);
        s.sumc2_1 = C1 * (1.0f + 1e-4f);
        if (o.stat == STAT_LOGVOL &&
            (!(q[0] > 0.0) || !(q[1] > 0.0) || !(A1 < INFINITY) || !(A2 < INFINITY)))
            s.status = ST_DEGENERATE;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline unsigned cdiv_(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

void launch_colsum(const PairMeta *meta, const RowChunk *chunks, const PairSpan &sp, int d, int dtype, i128 *part,
                   i128 *s, int *bad, cudaStream_t st)
{
    if (sp.c1 <= sp.c0 || sp.p1 <= sp.p0) return;
    // one thread per 16-byte column group when rows can be 16-byte aligned, else per column
    const int esz = dtype == DT_F32 ? 4 : 2, groups = (d * esz) % 16 == 0 ? d * esz / 16 : d;
    const int threads = std::min(256, std::max(32, (groups + 31) / 32 * 32));
    k_colsum_partial<<<sp.c1 - sp.c0, threads, 0, st>>>(meta, chunks, sp.c0, d, dtype, part, bad);
    k_colsum_reduce<<<cdiv_((int64_t)(sp.p1 - sp.p0) * 2 * d, 256), 256, 0, st>>>(meta, sp.p0, sp.p1, d, part, s);
}

void launch_axis(const PairMeta *meta, const PairSpan &sp, const RunOpts &o, const i128 *s, const int *bad,
                 PairState *pst, double *u, cudaStream_t st)
{
    if (sp.p1 <= sp.p0) return;
    k_axis<<<sp.p1 - sp.p0, 64, 2 * sizeof(double) * o.d, st>>>(meta, sp.p0, o, s, bad, pst, u);
}

void launch_reflect(const PairMeta *meta, const RowChunk *chunks, const PairSpan &sp, const RunOpts &o,
                    const PairState *pst, const double *u, void *Z, unsigned int *colmax,
                    unsigned long long *colL1, bool vec16, cudaStream_t st)
{
    if (sp.c1 <= sp.c0) return;
    const unsigned nc = (unsigned)(sp.c1 - sp.c0);
    if (o.dtype == DT_F32) k_reflect<DT_F32><<<nc, 128, 0, st>>>(meta, chunks, sp.c0, o, pst, u, Z, colmax, colL1);
    else if (vec16 && o.d % 8 == 0 && o.d <= 1024)
        k_reflect_v<<<nc, 128, 0, st>>>(meta, chunks, sp.c0, o, pst, u, Z, colmax, colL1);
    else k_reflect<DT_BF16><<<nc, 128, 0, st>>>(meta, chunks, sp.c0, o, pst, u, Z, colmax, colL1);
}

void launch_zstats(const PairMeta *meta, const RowChunk *chunks, const PairSpan &sp, const RunOpts &o,
                   const PairState *pst, const void *Z, const unsigned int *colmax,
                   const unsigned long long *colL1, i128 *tpart, float *cpart, float *cpart1, unsigned short *zq,
                   i128 *t_ex, i128 *s1o, ColConst *cc, float *ct, bool tok_layout, cudaStream_t st)
{
    if (sp.c1 <= sp.c0 || sp.p1 <= sp.p0) return;
    const unsigned nc = (unsigned)(sp.c1 - sp.c0);
    if (o.dtype == DT_F32)
        k_zstats_partial<DT_F32><<<nc, 256, 0, st>>>(meta, chunks, sp.c0, o, pst, Z, colmax, colL1, tpart, cpart,
                                                     cpart1, zq);
    else if (tok_layout)
        k_zstats_tok<<<nc, 256, 0, st>>>(meta, chunks, sp.c0, o, pst, static_cast<const uint4 *>(Z), colL1, tpart,
                                         cpart, cpart1, zq);
    else
        k_zstats_partial<DT_BF16><<<nc, 256, 0, st>>>(meta, chunks, sp.c0, o, pst, Z, colmax, colL1, tpart, cpart,
                                                      cpart1, zq);
    k_zstats_reduce<<<cdiv_((int64_t)(sp.p1 - sp.p0) * o.d_pad, 256), 256, 0, st>>>(
        meta, sp.p0, sp.p1, o, pst, colmax, tpart, cpart, cpart1, t_ex, s1o, cc, ct);
}

void launch_tobs(const PairMeta *meta, const PairSpan &sp, const RunOpts &o, const i128 *t_ex, const i128 *s1o,
                 const ColConst *cc, PairState *pst, cudaStream_t st)
{
    if (sp.p1 <= sp.p0) return;
    k_tobs<<<sp.p1 - sp.p0, 64, 2 * sizeof(double) * o.d, st>>>(meta, sp.p0, o, t_ex, s1o, cc, pst);
}

void set_align_attributes()
{
    // the reflection's shared-memory tiles: keep the largest carveout so that the
    // register limit, not shared memory, decides how many blocks an SM holds
    cudaFuncSetAttribute(k_reflect_v, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_axis, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_tobs, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace hb
