// hb_recheck.cu -- exact re-decision of the relabellings that fell inside
// their error band (both fast paths), and the per-pair p-value (Eq. pvalue).
//
// For relabelling b of pair p the group-1 sum is recomputed exactly on the
// 2^-87 fixed-point grid from the stored Z and the stored label bits,
// sigma_2 = t - sigma_1 exactly (Sec. 3.2: the two group sums add up to t),
// each coordinate is rounded once to FP64, the squared norms are sequential
// FMA chains over j = 0..d-1, and the decision uses only correctly rounded
// IEEE operations -- the same arithmetic as the FP64 CPU oracle.  The exact
// sums come from k_recheck_rows (BF16 storage, d a multiple of 8, d <= 1024:
// listed selected rows, 16-byte loads) or else from k_recheck_sums.
#include "hb_launch.cuh"

namespace hb {

// Stage 1: exact group sums of a batch of rechecked relabellings.  Block
// (item, 256-column slice); each thread owns one column and, per 32-row label
// word, issues the loads of the selected rows before consuming any.
template <int DT>
__global__ void __launch_bounds__(256) k_recheck_sums(const PairMeta *__restrict__ meta, const RunOpts o,
                                                      const void *__restrict__ Z, const i128 *__restrict__ t_ex,
                                                      const unsigned int *__restrict__ colmax,
                                                      const uint32_t *__restrict__ bits,
                                                      const RecheckItem *__restrict__ list,
                                                      const unsigned int *__restrict__ n_items, unsigned int cap,
                                                      unsigned int batch0, double *__restrict__ sums)
{
    extern __shared__ uint32_t sm_bits[];
    const unsigned int total = min(*n_items, cap);
    const unsigned int it = batch0 + blockIdx.x;
    if (it >= total) return;
    const int d = o.d;
    const RecheckItem item = list[it];
    const PairMeta pm = meta[item.pair];
    for (int w = threadIdx.x; w < pm.W; w += blockDim.x) sm_bits[w] = bits[pm.lab_off + (int64_t)w * pm.B_pad + item.b];
    __syncthreads();
    const int j = blockIdx.y * blockDim.x + threadIdx.x;
    if (j >= d) return;
    WinAcc wa;
    wa.init(col_bound_exp(colmax[(int64_t)item.pair * o.d_pad + j]));
    for (int w = 0; w < pm.W; ++w) {
        const uint32_t word = sm_bits[w];
        if (word == 0u) continue;
        const int64_t base = (pm.z_row + (int64_t)w * 32) * d + j;
        // two halves of 16 rows: their loads are issued before any is consumed
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int kk = 16 * h + k;
                v[k] = 0u;
                if ((word >> kk) & 1u)
                    v[k] = (DT == DT_F32) ? __ldg(reinterpret_cast<const uint32_t *>(Z) + base + (int64_t)kk * d)
                                          : (uint32_t)__ldg(reinterpret_cast<const unsigned short *>(Z) + base +
                                                            (int64_t)kk * d)
                                                << 16;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) wa.add(v[k]);
        }
        wa.flush();
    }
    const i128 acc = wa.total();
    double *out = sums + (int64_t)blockIdx.x * 2 * d;
    out[j] = fixed_to_f64(acc);
    out[d + j] = fixed_to_f64(t_ex[(int64_t)item.pair * d + j] - acc);
}

// The same sums for BF16 storage, d a multiple of 8 and d <= 1024, one block
// per item.  Warp 0 lists the selected rows of a window of up to RC_WIN_WORDS
// label words in shared memory; thread t < G = d/8 sums the 16-byte column
// group t (8 columns) over the listed rows of even index, thread G + t over
// those of odd index (four loads in flight each), and after the last window
// the two exact halves are added through shared memory.
constexpr int RC_WIN_WORDS = 256;  // 8192 rows per window
constexpr int RC_MAX_G = 128;      // d <= 1024

__global__ void __launch_bounds__(256) k_recheck_rows(const PairMeta *__restrict__ meta, const RunOpts o,
                                                      const uint4 *__restrict__ Z, const i128 *__restrict__ t_ex,
                                                      const unsigned int *__restrict__ colmax,
                                                      const uint32_t *__restrict__ bits,
                                                      const RecheckItem *__restrict__ list,
                                                      const unsigned int *__restrict__ n_items, unsigned int cap,
                                                      unsigned int batch0, double *__restrict__ sums)
{
    __shared__ uint16_t rows[RC_WIN_WORDS * 32];
    __shared__ i128 half1[RC_MAX_G * 8];
    __shared__ int nsel;
    const unsigned int total = min(*n_items, cap);
    const unsigned int it = batch0 + blockIdx.x;
    if (it >= total) return;
    const int d = o.d, G = d / 8;
    const RecheckItem item = list[it];
    const PairMeta pm = meta[item.pair];
    const int lane = threadIdx.x & 31;
    const int h = (int)threadIdx.x >= G ? 1 : 0, gg = (int)threadIdx.x - h * G;
    const bool live = gg < G;  // blockDim.x may exceed 2G (whole warps)
    // exact sums: each value splits into h on the 2^-12 grid and l = v - h on the 2^-28
    // grid, summed in FP32 (exact for up to 128 values of |v| < 16), folded into 128-bit
    // totals every 128 values; values below 2^-21 go to the 128-bit total directly
    // (|v| < 2^-64 counts as 0)
    const float M = 3072.0f;  // (v + M) - M rounds v to the 2^-12 grid
    float sh[8], sl[8];
    i128 tot[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        sh[e] = sl[e] = 0.0f;
        tot[e] = 0;
    }
    int cnt = 0;
    for (int w0 = 0; w0 < pm.W; w0 += RC_WIN_WORDS) {
        const int nw = min(RC_WIN_WORDS, pm.W - w0);
        __syncthreads();  // the previous window's list is consumed
        if (threadIdx.x < 32) {
            int base = 0;
            for (int k0 = 0; k0 < nw; k0 += 32) {
                const int k = k0 + lane;
                uint32_t word = k < nw ? bits[pm.lab_off + (int64_t)(w0 + k) * pm.B_pad + item.b] : 0u;
                const int c = __popc(word);
                int incl = c;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += t;
                }
                int pos = base + incl - c;
                while (word) {
                    rows[pos++] = (uint16_t)(k * 32 + __ffs(word) - 1);
                    word &= word - 1u;
                }
                base += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) nsel = base;
        }
        __syncthreads();
        const int ns = nsel;
        if (!live) continue;
        const uint4 *zp = Z + (pm.z_row + (int64_t)w0 * 32) * G + gg;
        for (int r0 = h; r0 < ns; r0 += 8) {
            uint4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                v[k] = r0 + 2 * k < ns ? __ldg(zp + (int64_t)rows[r0 + 2 * k] * G) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t wv[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t b = (e & 1) ? (wv[e >> 1] & 0xffff0000u) : (wv[e >> 1] << 16);
                    float x = __uint_as_float(b);
                    if ((b & 0x7fffffffu) - 1u < (106u << 23) - 1u) {  // 0 < |v| < 2^-21: rare
                        tot[e] += fixed_from_f32bits(b);
                        x = 0.0f;
                    }
                    const float h = __fsub_rn(__fadd_rn(x, M), M);
                    sh[e] = __fadd_rn(sh[e], h);
                    sl[e] = __fadd_rn(sl[e], __fsub_rn(x, h));
                }
            }
            if ((++cnt & 31) == 0) {  // every 128 values per column
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    tot[e] += fixed_from_f32bits(__float_as_uint(sh[e])) + fixed_from_f32bits(__float_as_uint(sl[e]));
                    sh[e] = sl[e] = 0.0f;
                }
            }
        }
    }
    i128 acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
        acc[e] = tot[e] + fixed_from_f32bits(__float_as_uint(sh[e])) + fixed_from_f32bits(__float_as_uint(sl[e]));
    if (live && h == 1) {
#pragma unroll
        for (int e = 0; e < 8; ++e) half1[gg * 8 + e] = acc[e];
    }
    __syncthreads();
    if (live && h == 0) {
        double *out = sums + (int64_t)blockIdx.x * 2 * d;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int j = 8 * gg + e;
            const i128 a = acc[e] + half1[gg * 8 + e];
            out[j] = fixed_to_f64(a);
            out[d + j] = fixed_to_f64(t_ex[(int64_t)item.pair * d + j] - a);
        }
    }
}

// Stage 2: squared norms as sequential FMA chains over j = 0..d-1 (two
// threads per item, one per group, all items in flight together), then the
// exact decision with correctly rounded IEEE operations only.
__global__ void k_recheck_decide(const PairMeta *__restrict__ meta, const RunOpts o, PairState *__restrict__ st,
                                 const RecheckItem *__restrict__ list, const unsigned int *__restrict__ n_items,
                                 unsigned int cap, unsigned int batch0, unsigned int batch,
                                 const double *__restrict__ sums, float *__restrict__ T_out)
{
    const unsigned int total = min(*n_items, cap);
    const unsigned int t = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned int k = t >> 1, g = t & 1u;
    const unsigned int it = batch0 + k;
    const bool live = k < batch && it < total;
    const int d = o.d;
    double q = 0.0;
    if (live) {
        const double *v = sums + (int64_t)k * 2 * d + (int64_t)g * d;
        for (int j = 0; j < d; ++j) q = __fma_rn(v[j], v[j], q);
    }
    const double q2 = __shfl_down_sync(0xffffffffu, q, 1);
    if (!live || g != 0u) return;
    const RecheckItem item = list[it];
    const PairMeta pm = meta[item.pair];
    const PairState s = st[item.pair];
    const double A1 = group_value_f64(o.stat, q, (double)pm.n, (double)d);
    const double A2 = group_value_f64(o.stat, q2, (double)pm.m, (double)d);
    if (exceeds_f64(o.stat, o.alt, A1, A2, s.A1o, s.A2o)) atomicAdd(&st[item.pair].count, 1ull);
    atomicAdd(&st[item.pair].rechecked, 1ull);
    if (T_out && pm.T_off >= 0) T_out[pm.T_off + item.b] = (float)stat_T_f64(o.stat, A1, A2);
}

// p = (1 + count)/(B + 1), or count/C(N, n) when every split is enumerated.
__global__ void k_finalize(const PairMeta *__restrict__ meta, int P, const RunOpts o, const PairState *__restrict__ st,
                           PairOut *__restrict__ out)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const PairMeta pm = meta[p];
    const PairState s = st[p];
    PairOut r;
    r.status = s.status;
    r.skipped = s.skipped;
    r.B_eff = pm.B;
    r.count = (int64_t)s.count;
    r.rechecked = (int64_t)s.rechecked;
    r.band_max = (double)__uint_as_float(s.band_max_bits);
    if (s.status == ST_OK) {
        r.T_obs = s.To;
        r.r_x = s.rx;
        r.r_y = s.ry;
        r.p = o.exhaustive ? __ddiv_rn((double)r.count, (double)pm.B)
                           : __ddiv_rn((double)(r.count + 1), (double)(pm.B + 1));
    } else {
        r.T_obs = r.r_x = r.r_y = 0.0;
        r.p = 0.0;
        r.count = 0;
    }
    out[p] = r;
}

void launch_recheck(unsigned int cap, unsigned int batch, int max_W, const PairMeta *meta, const RunOpts &o,
                    PairState *pst, const void *Z, const i128 *t_ex, const unsigned int *colmax, const uint32_t *bits,
                    const RecheckItem *list, const unsigned int *n_items, double *sums, float *T_out,
                    cudaStream_t st)
{
    // batches up to the list capacity; batches past the actual count exit at once
    const size_t smem = sizeof(uint32_t) * (size_t)max_W;
    const dim3 g1(batch, (unsigned)((o.d + 255) / 256));
    const bool rows_path = o.dtype == DT_BF16 && o.d % 8 == 0 && o.d <= 8 * RC_MAX_G;
    const unsigned int rthreads = (unsigned)(((2 * (o.d / 8) + 31) / 32) * 32);
    for (unsigned int b0 = 0; b0 < cap; b0 += batch) {
        if (rows_path)
            k_recheck_rows<<<batch, rthreads, 0, st>>>(meta, o, static_cast<const uint4 *>(Z), t_ex, colmax, bits,
                                                       list, n_items, cap, b0, sums);
        else if (o.dtype == DT_F32)
            k_recheck_sums<DT_F32><<<g1, 256, smem, st>>>(meta, o, Z, t_ex, colmax, bits, list, n_items, cap, b0,
                                                          sums);
        else
            k_recheck_sums<DT_BF16><<<g1, 256, smem, st>>>(meta, o, Z, t_ex, colmax, bits, list, n_items, cap, b0,
                                                           sums);
        k_recheck_decide<<<(2 * batch + 127) / 128, 128, 0, st>>>(meta, o, pst, list, n_items, cap, b0, batch, sums,
                                                                 T_out);
    }
}

void launch_finalize(const PairMeta *meta, int P, const RunOpts &o, const PairState *pst, PairOut *out,
                     cudaStream_t st)
{
    k_finalize<<<(unsigned)((P + 127) / 128), 128, 0, st>>>(meta, P, o, pst, out);
}

void set_kernel_attributes()
{
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_recheck_sums<DT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_recheck_sums<DT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    set_align_attributes();
}

}  // namespace hb
