// hb_plain.cu -- the plain FP32 path: Algorithm 2 of the paper taken
// literally.  Signs s_i = +1 (group 1) / -1 (group 2), U = S Z with an FP32
// SIMT GEMM (Eq. gemm), sigma_1 = (t + U)/2, sigma_2 = (t - U)/2, then the
// statistic of every relabelling in an FP32 epilogue (Algorithm 2, "recover
// group sums" and "compute test statistic").  Each decision carries a
// rigorous error band; relabellings inside it are re-decided exactly by
// k_recheck, so the count equals the exact one.
//
// One CTA (256 threads) owns 128 relabellings of one pair and sweeps all d
// columns in tiles of 128; each thread accumulates an 8 x 8 block of U over
// the tokens (K) in chunks of 16, so per token chunk it issues 64 FMAs for 4
// 16-byte shared loads.
#include "hb_launch.cuh"

namespace hb {

constexpr int PT_M = 128;  // relabellings per CTA
constexpr int PT_N = 128;  // columns per tile
constexpr int PT_K = 16;   // tokens per chunk

template <int DT>
__global__ void __launch_bounds__(256) k_plain_gemm(const PairMeta *__restrict__ meta, const RunOpts o,
                                                    PairState *__restrict__ st, const void *__restrict__ Z,
                                                    const ColConst *__restrict__ cc, const uint32_t *__restrict__ bits,
                                                    RecheckItem *__restrict__ list, unsigned int *__restrict__ n_items,
                                                    unsigned int cap, unsigned int *__restrict__ overflow,
                                                    float *__restrict__ T_out, int pair0)
{
    __shared__ __align__(16) float Ss[PT_K][PT_M];
    __shared__ __align__(16) float Zs[PT_K][PT_N];
    __shared__ float ts[PT_N], cs[PT_N];

    const int p = pair0 + blockIdx.y;
    const PairMeta pm = meta[p];
    const int tile = blockIdx.x;
    if (tile * PT_M >= pm.B_pad || st[p].status != ST_OK) return;
    const int d = o.d;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t b0 = (int64_t)tile * PT_M;

    float q1[8], q2[8], e1[8], e2[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) q1[i] = q2[i] = e1[i] = e2[i] = 0.0f;

    for (int j0 = 0; j0 < d; j0 += PT_N) {
        __syncthreads();  // the previous tile's epilogue has finished reading ts/cs
        if (tid < PT_N) {
            const int j = j0 + tid;
            const ColConst c = j < d ? cc[(int64_t)p * o.d_pad + j] : ColConst{0.f, 0.f, 0.f, 0.f};
            ts[tid] = c.t;
            cs[tid] = c.c;
        }
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[i][k] = 0.0f;

        for (int k0 = 0; k0 < pm.N; k0 += PT_K) {
            __syncthreads();
            if (tid < PT_M) {
                // signs of 16 tokens for relabelling b0 + tid
                const uint32_t w = bits[pm.lab_off + (int64_t)(k0 >> 5) * pm.B_pad + b0 + tid];
                const uint32_t h = (w >> (k0 & 16)) & 0xffffu;
#pragma unroll
                for (int kk = 0; kk < PT_K; ++kk) Ss[kk][tid] = ((h >> kk) & 1u) ? 1.0f : -1.0f;
            } else {
                const int c = tid - PT_M;
                const int j = j0 + c;
#pragma unroll 4
                for (int kk = 0; kk < PT_K; ++kk) {
                    const int tok = k0 + kk;
                    float v = 0.0f;
                    if (tok < pm.N && j < d)
                        v = __uint_as_float(load_f32bits(Z, DT, (pm.z_row + tok) * (int64_t)d + j));
                    Zs[kk][c] = v;
                }
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < PT_K; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&Ss[kk][ty * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&Ss[kk][64 + ty * 4]);
                const float4 z0 = *reinterpret_cast<const float4 *>(&Zs[kk][tx * 4]);
                const float4 z1 = *reinterpret_cast<const float4 *>(&Zs[kk][64 + tx * 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float z[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int k = 0; k < 8; ++k) acc[i][k] = fmaf(a[i], z[k], acc[i][k]);
            }
        }
        // epilogue of this column tile: sigma_1,2 = (t +- U)/2 and the band terms
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float pq1 = 0.f, pq2 = 0.f, pe1 = 0.f, pe2 = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = (k < 4) ? tx * 4 + k : 64 + tx * 4 + (k - 4);
                const float t = ts[c], cj = cs[c];
                const float s1 = (t + acc[i][k]) * 0.5f;
                const float s2 = (t - acc[i][k]) * 0.5f;
                pq1 = fmaf(s1, s1, pq1);
                pq2 = fmaf(s2, s2, pq2);
                pe1 = fmaf(fabsf(s1), cj, pe1);
                pe2 = fmaf(fabsf(s2), cj, pe2);
            }
            q1[i] += pq1;
            q2[i] += pq2;
            e1[i] += pe1;
            e2[i] += pe2;
        }
    }
    // reduce over the 16 column groups (tx) of each relabelling: lanes differ in bits 0..3
#pragma unroll
    for (int i = 0; i < 8; ++i) {
#pragma unroll
        for (int off = 1; off < 16; off <<= 1) {
            q1[i] += __shfl_xor_sync(0xffffffffu, q1[i], off);
            q2[i] += __shfl_xor_sync(0xffffffffu, q2[i], off);
            e1[i] += __shfl_xor_sync(0xffffffffu, e1[i], off);
            e2[i] += __shfl_xor_sync(0xffffffffu, e2[i], off);
        }
    }
    if (tx != 0) return;
    const PairState s = st[p];
    const float To = (float)s.To;
    const float chain = 24.0f + (float)((d + PT_N - 1) / PT_N);
    unsigned int nex = 0;
    float bmax = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
        const int64_t b = b0 + r;
        if (b >= pm.B) continue;
        const float dq1 = q_bound(e1[i], q1[i], q1[i], q2[i], s.tnorm, s.sumc2, chain);
        const float dq2 = q_bound(e2[i], q2[i], q1[i], q2[i], s.tnorm, s.sumc2, chain);
        float T, band;
        const int dec = fast_decide(o.stat, o.alt, (float)d, (float)pm.n, (float)pm.m, q1[i], q2[i], dq1, dq2, To,
                                    &T, &band);
        if (dec == 1) ++nex;
        else if (dec < 0) push_recheck(list, n_items, cap, overflow, p, (uint32_t)b);
        if (band < INFINITY) bmax = fmaxf(bmax, band);
        if (T_out && pm.T_off >= 0) T_out[pm.T_off + b] = T;
    }
    if (nex) atomicAdd(&st[p].count, (unsigned long long)nex);
    atomicMax(&st[p].band_max_bits, __float_as_uint(bmax));
}

void launch_plain(const PairMeta *meta, int P, int max_Bpad, const RunOpts &o, PairState *pst, const void *Z,
                  const ColConst *cc, const uint32_t *bits, RecheckItem *list, unsigned int *n_items,
                  unsigned int cap, unsigned int *overflow, float *T_out, cudaStream_t st)
{
    for (int p0 = 0; p0 < P; p0 += 65535) {
        const dim3 g((unsigned)((max_Bpad + PT_M - 1) / PT_M), (unsigned)min(65535, P - p0));
        if (o.dtype == DT_F32)
            k_plain_gemm<DT_F32><<<g, 256, 0, st>>>(meta, o, pst, Z, cc, bits, list, n_items, cap, overflow, T_out,
                                                     p0);
        else
            k_plain_gemm<DT_BF16><<<g, 256, 0, st>>>(meta, o, pst, Z, cc, bits, list, n_items, cap, overflow, T_out,
                                                      p0);
    }
}

}  // namespace hb
