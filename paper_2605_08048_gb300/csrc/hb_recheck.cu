// hb_recheck.cu -- exact re-decision of the relabellings that fell inside
// their error band (both fast paths), and the per-pair p-value (Eq. pvalue).
//
// For relabelling b of pair p the group-1 sum is recomputed exactly on the
// 2^-87 fixed-point grid from the stored Z and the stored label bits,
// sigma_2 = t - sigma_1 exactly (Sec. 3.2: the two group sums add up to t),
// each coordinate is rounded once to FP64, the squared norms are sequential
// FMA chains over j = 0..d-1, and the decision uses only correctly rounded
// IEEE operations -- the same arithmetic as the FP64 CPU oracle.
#include "hb_launch.cuh"

namespace hb {

template <int DT>
__global__ void __launch_bounds__(256) k_recheck(const PairMeta *__restrict__ meta, const RunOpts o,
                                                 PairState *__restrict__ st, const void *__restrict__ Z,
                                                 const i128 *__restrict__ t_ex, const uint32_t *__restrict__ bits,
                                                 const RecheckItem *__restrict__ list,
                                                 const unsigned int *__restrict__ n_items, unsigned int cap,
                                                 double *__restrict__ scratch, float *__restrict__ T_out)
{
    extern __shared__ uint32_t sm_bits[];
    __shared__ double q[2];
    const int d = o.d;
    const unsigned int total = min(*n_items, cap);
    double *s1 = scratch + (int64_t)blockIdx.x * 2 * d, *s2 = s1 + d;
    for (unsigned int it = blockIdx.x; it < total; it += gridDim.x) {
        const RecheckItem item = list[it];
        const PairMeta pm = meta[item.pair];
        for (int w = threadIdx.x; w < pm.W; w += blockDim.x)
            sm_bits[w] = bits[pm.lab_off + (int64_t)w * pm.B_pad + item.b];
        __syncthreads();
        // exact group-1 sums: up to RC columns per thread per pass; for each
        // 32-row label word the 32 predicated loads of a column are issued
        // before any is consumed (loads of unselected rows are skipped)
        constexpr int RC = 4;
        for (int j0 = 0; j0 < d; j0 += RC * (int)blockDim.x) {
            i128 acc[RC];
#pragma unroll
            for (int c = 0; c < RC; ++c) acc[c] = 0;
            for (int w = 0; w < pm.W; ++w) {
                const uint32_t word = sm_bits[w];
                if (word == 0u) continue;
                const unsigned short *rowp16 = nullptr;
                const uint32_t *rowp32 = nullptr;
                const int64_t base = (pm.z_row + (int64_t)w * 32) * d;
                if (DT == DT_F32) rowp32 = reinterpret_cast<const uint32_t *>(Z) + base;
                else rowp16 = reinterpret_cast<const unsigned short *>(Z) + base;
#pragma unroll
                for (int c = 0; c < RC; ++c) {
                    const int j = j0 + c * (int)blockDim.x + (int)threadIdx.x;
                    if (j >= d) break;
                    uint32_t v[32];
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        v[k] = 0u;
                        if ((word >> k) & 1u)
                            v[k] = (DT == DT_F32) ? __ldg(rowp32 + (int64_t)k * d + j)
                                                  : (uint32_t)__ldg(rowp16 + (int64_t)k * d + j) << 16;
                    }
#pragma unroll
                    for (int k = 0; k < 32; ++k) acc[c] += fixed_from_f32bits(v[k]);
                }
            }
#pragma unroll
            for (int c = 0; c < RC; ++c) {
                const int j = j0 + c * (int)blockDim.x + (int)threadIdx.x;
                if (j < d) {
                    s1[j] = fixed_to_f64(acc[c]);
                    s2[j] = fixed_to_f64(t_ex[(int64_t)item.pair * d + j] - acc[c]);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 || threadIdx.x == 32) {
            const double *v = threadIdx.x ? s2 : s1;
            double a = 0.0;
            for (int j = 0; j < d; ++j) a = __fma_rn(v[j], v[j], a);
            q[threadIdx.x ? 1 : 0] = a;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const PairState s = st[item.pair];
            const double A1 = group_value_f64(o.stat, q[0], (double)pm.n, (double)d);
            const double A2 = group_value_f64(o.stat, q[1], (double)pm.m, (double)d);
            const int e = exceeds_f64(o.stat, o.alt, A1, A2, s.A1o, s.A2o);
            if (e) atomicAdd(&st[item.pair].count, 1ull);
            atomicAdd(&st[item.pair].rechecked, 1ull);
            if (T_out && pm.T_off >= 0) T_out[pm.T_off + item.b] = (float)stat_T_f64(o.stat, A1, A2);
        }
        __syncthreads();
    }
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

void launch_recheck(int grid, size_t smem, const PairMeta *meta, const RunOpts &o, PairState *pst, const void *Z,
                    const i128 *t_ex, const uint32_t *bits, const RecheckItem *list, const unsigned int *n_items,
                    unsigned int cap, double *scratch, float *T_out, cudaStream_t st)
{
    if (o.dtype == DT_F32)
        k_recheck<DT_F32><<<grid, 256, smem, st>>>(meta, o, pst, Z, t_ex, bits, list, n_items, cap, scratch, T_out);
    else
        k_recheck<DT_BF16><<<grid, 256, smem, st>>>(meta, o, pst, Z, t_ex, bits, list, n_items, cap, scratch, T_out);
}

void launch_finalize(const PairMeta *meta, int P, const RunOpts &o, const PairState *pst, PairOut *out,
                     cudaStream_t st)
{
    k_finalize<<<(unsigned)((P + 127) / 128), 128, 0, st>>>(meta, P, o, pst, out);
}

void set_kernel_attributes()
{
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_recheck<DT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_recheck<DT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    set_align_attributes();
}

}  // namespace hb
