// hb_triage.cu -- kernels of the learned triage (an addition of this library;
// the paper has no learned part): per-pair features, the 19 -> 256 -> 256 -> 9 MLP that
// predicts null quantiles of |T| (forward, backward, pinball loss, Adam),
// null-quantile targets from the method's own relabellings, and the
// predicted p used to route pairs.
//
// Features of a pair: log n, log m, log(d * lambda_k) for the 16 Ritz values
// lambda_k of the pooled scatter Z^T Z / N after RITZ_ITERS block subspace
// iterations (V <- orth(Z^T Z V / N), Cholesky-QR)
// from a fixed Philox start block, and 10 * T_obs.
#include <math.h>

#include <algorithm>

#include "hb_launch.cuh"

namespace hb {

constexpr int RK = 16;          // Ritz block size
constexpr int RITZ_ITERS = 2;
constexpr int MLP_IN = 19, MLP_H = 256, MLP_OUT = 9;

// ---------------------------------------------------------------------------
// block reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float block_sum(float v, float *red)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    float s = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];  // same order in every thread
    return s;
}

// ---------------------------------------------------------------------------
// Ritz values of Z^T Z / N, one CTA (256 threads, 8 warps) per pair, FP32
// SIMT (FP32 rows; BF16 rows take k_ritz_mma below, which keeps the same
// chunk loop and replaces the FMAs of both contractions by MMAs).
//
// One pass W = Z^T (Z V) streams Z through shared memory in chunks of R rows
// (cp.async double buffer).  Per chunk: (1) P = Zc V (R x 16): warp w takes
// the w-th eighth of the columns j, lane (rq, cg) rows rq + 8i and columns
// 4cg..4cg+3, then the 8 warp partials are summed; (2) W += Zc^T P: thread t
// owns rows j = t + 256u of W, kept in registers for the whole pass.
// Between passes W goes to shared memory (over both chunk buffers, which hold
// at least d x 16 floats) for the orthonormalisation V = W R^-1 (Cholesky-QR
// of W^T W = R^T R).  Chunks of 8 FP32 rows keep the shared memory of a CTA
// near 110 KB and its registers at 128, so that two pairs' CTAs share an SM
// and one's barriers and serial steps overlap the other's streaming.
// dynamic smem: Zc[2][R][ZS] (input element type), V[dp][16], part[8][R][16],
// Pm[R][16]  (dp = d rounded up to 32, ZS = dp + 16 bytes of padding)
// ---------------------------------------------------------------------------
template <int DT> struct RitzTile;
template <> struct RitzTile<DT_BF16> {
    static constexpr int R = 16, ES = 2, PAD = 8;
    __device__ __forceinline__ static void load4(const unsigned char *row, int j, float *z)
    {
        const uint2 w = *reinterpret_cast<const uint2 *>(row + 2 * j);
        z[0] = __uint_as_float(w.x << 16);
        z[1] = __uint_as_float(w.x & 0xffff0000u);
        z[2] = __uint_as_float(w.y << 16);
        z[3] = __uint_as_float(w.y & 0xffff0000u);
    }
    __device__ __forceinline__ static float load1(const unsigned char *row, int j)
    {
        return __uint_as_float((uint32_t)reinterpret_cast<const unsigned short *>(row)[j] << 16);
    }
};
template <> struct RitzTile<DT_F32> {
    static constexpr int R = 8, ES = 4, PAD = 4;
    __device__ __forceinline__ static void load4(const unsigned char *row, int j, float *z)
    {
        const float4 w = *reinterpret_cast<const float4 *>(row + 4 * j);
        z[0] = w.x;
        z[1] = w.y;
        z[2] = w.z;
        z[3] = w.w;
    }
    __device__ __forceinline__ static float load1(const unsigned char *row, int j)
    {
        return reinterpret_cast<const float *>(row)[j];
    }
};

__device__ __forceinline__ int ritz_dp(int d) { return (d + 31) & ~31; }

template <int DT>
__host__ __device__ __forceinline__ size_t ritz_zc_bytes(int d)
{
    return (size_t)RitzTile<DT>::R * (size_t)(((d + 31) & ~31) + RitzTile<DT>::PAD) * RitzTile<DT>::ES;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// stage rows [r0, r0 + ROWS) of the pair into a chunk buffer of row stride ZS
// elements (rows past N read as zero)
template <int DT, int ROWS>
__device__ __forceinline__ void ritz_stage(unsigned char *buf, const void *Z, int64_t z_row, int r0, int N, int d,
                                           int ZS, bool vec)
{
    constexpr int ES = RitzTile<DT>::ES;
    const unsigned char *src = reinterpret_cast<const unsigned char *>(Z);
    if (vec) {  // rows of d elements are a whole number of 16-byte pieces
        const int per_row = d * ES / 16;
        for (int t = threadIdx.x; t < ROWS * per_row; t += blockDim.x) {
            const int r = t / per_row, q = t - r * per_row;
            const bool in = r0 + r < N;
            const unsigned char *g = in ? src + ((z_row + r0 + r) * (int64_t)d * ES + (int64_t)q * 16) : src;
            cp_async16(buf + (size_t)r * ZS * ES + q * 16, g, in ? 16 : 0);
        }
        cp_async_commit();
    } else {
        for (int t = threadIdx.x; t < ROWS * d; t += blockDim.x) {
            const int r = t / d, j = t - r * d;
            const bool in = r0 + r < N;
            const uint32_t bits = in ? load_f32bits(Z, DT, (z_row + r0 + r) * (int64_t)d + j) : 0u;
            if (DT == DT_BF16)
                reinterpret_cast<unsigned short *>(buf)[(size_t)r * ZS + j] = (unsigned short)(bits >> 16);
            else
                reinterpret_cast<uint32_t *>(buf)[(size_t)r * ZS + j] = bits;
        }
    }
}

// the same for BF16 rows of a whole number of 16-byte pieces (per_row of
// them), walking this thread's (row, piece) pairs by additions: (r, q) of item
// t + k blockDim follows from that of item t (r0q, q0) and the step (dr, dq)
__device__ __forceinline__ void ritz_stage_vec(unsigned char *buf, const unsigned char *src_row0, int rows_left,
                                               int per_row, int ZS2, int64_t row_bytes, int r, int q, int dr, int dq,
                                               int rows)
{
    for (; r < rows; r += dr, q += dq) {
        if (q >= per_row) {
            q -= per_row;
            ++r;
            if (r >= rows) break;
        }
        const bool in = r < rows_left;
        const unsigned char *g = in ? src_row0 + r * row_bytes + q * 16 : src_row0;
        cp_async16(buf + r * ZS2 + q * 16, g, in ? 16 : 0);
    }
    cp_async_commit();
}

// Cholesky-QR factor of W [d][16] (shared memory, 256 threads): G = W^T W =
// R^T R, Rinv = R^-1 (upper triangular).  The Gram entries take one thread
// each; the factorisation runs in warp 0 with lane c (lanes 16-31 repeat
// lanes 0-15) holding column c of G in registers: right-looking Cholesky
// (step k: r_kk = sqrt(G_kk), R_kc = G_kc / r_kk, G_ic -= R_ki R_kc for
// i > k, R_ki taken from lane i), then R goes to Hm and lane c solves
// R x = e_c by back substitution for column c of R^-1.  Ends with a barrier.
__device__ void ritz_rinv(const float *Wsm, int d, float (*Hm)[RK], float (*Rinv)[RK])
{
    const int tid = threadIdx.x;
    {
        const int a = tid >> 4, bb = tid & 15;  // one Gram entry per thread
        float g0 = 0.f, g1 = 0.f;
        int j = 0;
        for (; j + 1 < d; j += 2) {
            g0 = fmaf(Wsm[j * RK + a], Wsm[j * RK + bb], g0);
            g1 = fmaf(Wsm[(j + 1) * RK + a], Wsm[(j + 1) * RK + bb], g1);
        }
        if (j < d) g0 = fmaf(Wsm[j * RK + a], Wsm[j * RK + bb], g0);
        Hm[a][bb] = g0 + g1;
    }
    __syncthreads();
    if (tid < 32) {
        const int c = tid & 15;
        float gc[RK];
#pragma unroll
        for (int i = 0; i < RK; ++i) gc[i] = Hm[i][c];
#pragma unroll
        for (int k = 0; k < RK; ++k) {
            const float rkk = sqrtf(fmaxf(__shfl_sync(0xffffffffu, gc[k], k), 1e-30f));
            const float rkc = c > k ? gc[k] / rkk : (c == k ? rkk : 0.f);  // R[k][c]
            gc[k] = rkc;
#pragma unroll
            for (int i = k + 1; i < RK; ++i) gc[i] = fmaf(-__shfl_sync(0xffffffffu, rkc, i), rkc, gc[i]);
        }
        __syncwarp();  // every lane has read G
        if (tid < 16)
#pragma unroll
            for (int i = 0; i < RK; ++i) Hm[i][c] = gc[i];
        __syncwarp();
        float x[RK];
#pragma unroll
        for (int i = RK - 1; i >= 0; --i) {
            float t = 0.f;
#pragma unroll
            for (int k = i + 1; k < RK; ++k) t = fmaf(Hm[i][k], x[k], t);
            x[i] = i > c ? 0.f : (i == c ? 1.0f / Hm[i][i] : -t / Hm[i][i]);
        }
        if (tid < 16)
#pragma unroll
            for (int i = 0; i < RK; ++i) Rinv[i][c] = x[i];
    }
    __syncthreads();
}

// Eigenvalues of the 16 x 16 Rayleigh-Ritz matrix in Hm, by warp 0 (the
// calling warp): symmetrise, then parallel cyclic Jacobi (round-robin order:
// 15 rounds of 8 disjoint rotations per sweep) until the off-diagonal part is
// negligible relative to the diagonal; lam[0..15] in descending order.
__device__ void ritz_jacobi(float (*Hm)[RK], float *lam)
{
    __shared__ float jc[8], js[8];
    __shared__ int ja[8], jb[8];
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < RK * RK; e += 32) {
        const int a = e >> 4, b = e & 15;
        if (a < b) Hm[a][b] = Hm[b][a] = 0.5f * (Hm[a][b] + Hm[b][a]);
    }
    __syncwarp();
    for (int sweep = 0; sweep < 20; ++sweep) {
        float off = 0.f, dg = 0.f;
        for (int e = lane; e < RK * RK; e += 32) {
            const int a = e >> 4, b = e & 15;
            const float h = Hm[a][b];
            if (a < b) off += h * h;
            if (a == b) dg += h * h;
        }
#pragma unroll
        for (int s = 16; s; s >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, s);
            dg += __shfl_xor_sync(0xffffffffu, dg, s);
        }
        if (off <= 1e-13f * dg || off < 1e-30f) break;
        for (int k = 0; k < RK - 1; ++k) {
            if (lane < 8) {
                int a, b;
                if (lane == 0) {
                    a = k;
                    b = RK - 1;
                } else {
                    a = (k + lane) % (RK - 1);
                    b = (k - lane + RK - 1) % (RK - 1);
                }
                if (a > b) {
                    const int tmp = a;
                    a = b;
                    b = tmp;
                }
                const float hab = Hm[a][b];
                float c = 1.f, s = 0.f;
                if (fabsf(hab) > 1e-30f) {
                    const float theta = 0.5f * (Hm[b][b] - Hm[a][a]) / hab;
                    const float t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
                    c = rsqrtf(t * t + 1.0f);
                    s = t * c;
                }
                ja[lane] = a;
                jb[lane] = b;
                jc[lane] = c;
                js[lane] = s;
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // columns a, b of every row
                const int task = lane + 32 * q, i = task >> 4, row = task & 15;
                const int a = ja[i], b = jb[i];
                const float c = jc[i], s = js[i];
                const float hka = Hm[row][a], hkb = Hm[row][b];
                Hm[row][a] = c * hka - s * hkb;
                Hm[row][b] = s * hka + c * hkb;
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // rows a, b of every column
                const int task = lane + 32 * q, i = task >> 4, col = task & 15;
                const int a = ja[i], b = jb[i];
                const float c = jc[i], s = js[i];
                const float hak = Hm[a][col], hbk = Hm[b][col];
                Hm[a][col] = c * hak - s * hbk;
                Hm[b][col] = s * hak + c * hbk;
            }
            __syncwarp();
        }
    }
    if (lane == 0) {
        float ev[RK];
        for (int a = 0; a < RK; ++a) ev[a] = Hm[a][a];
        for (int a = 1; a < RK; ++a)  // insertion sort, descending
            for (int b = a; b > 0 && ev[b] > ev[b - 1]; --b) {
                const float tmp = ev[b];
                ev[b] = ev[b - 1];
                ev[b - 1] = tmp;
            }
        for (int a = 0; a < RK; ++a) lam[a] = ev[a];
    }
}

template <int DT, int JU>
__global__ void __launch_bounds__(256, 2) k_ritz(const PairMeta *__restrict__ meta, const RunOpts o,
                                                 const PairState *__restrict__ st, const void *__restrict__ Z,
                                                 float *__restrict__ lam_out)
{
    using TT = RitzTile<DT>;
    constexpr int R = TT::R, RI = R / 8;
    extern __shared__ __align__(16) unsigned char sm_ritz[];
    __shared__ float Hm[RK][RK];
    __shared__ float Rinv[RK][RK];
    const int p = blockIdx.x;
    if (st[p].status != ST_OK) {
        if (threadIdx.x < RK) lam_out[p * RK + threadIdx.x] = 0.f;
        return;
    }
    const PairMeta pm = meta[p];
    const int d = o.d, N = pm.N, dp = ritz_dp(d), ZS = dp + TT::PAD;
    const size_t zc_bytes = ritz_zc_bytes<DT>(d);
    unsigned char *Zc[2] = {sm_ritz, sm_ritz + zc_bytes};
    float *V = reinterpret_cast<float *>(sm_ritz + 2 * zc_bytes);
    float *part = V + (size_t)dp * RK;
    float *Pm = part + 8 * R * RK;
    float *Wsm = reinterpret_cast<float *>(Zc[0]);  // W between passes, [d][16], over both chunk buffers
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, rq = lane >> 2, cg = lane & 3;
    const bool vec = (d * TT::ES) % 16 == 0;

    // zero everything once: padding columns of the chunk buffers and V rows >= d stay zero
    for (size_t t = tid; t < (2 * zc_bytes) / 4 + (size_t)dp * RK; t += blockDim.x)
        reinterpret_cast<float *>(sm_ritz)[t] = 0.f;
    __syncthreads();
    // fixed start block: (w >> 8) / 2^24 - 1/2, w = Philox(j, c, 0x5EED, 0; key 0, 0) word 0
    for (int t = tid; t < d * RK; t += blockDim.x) {
        const int j = t >> 4, c = t & 15;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)c, 0x5EEDu, 0u), 0u, 0u);
        Wsm[t] = (float)(r.x >> 8) * (1.0f / 16777216.0f) - 0.5f;
    }
    __syncthreads();
    const int nch = (N + R - 1) / R;
    const float invN = 1.0f / (float)N;
    for (int iter = 0; iter <= RITZ_ITERS; ++iter) {
        // ---- V = orth(W): G = W^T W = R^T R (Cholesky), V = W R^-1 ----
        ritz_rinv(Wsm, d, Hm, Rinv);
        for (int t = tid; t < d * RK; t += blockDim.x) {
            const int j = t >> 4, c = t & 15;
            float v = 0.f;
            for (int k = 0; k <= c; ++k) v = fmaf(Wsm[j * RK + k], Rinv[k][c], v);
            V[t] = v;
        }
        __syncthreads();
        // the W staging overwrote the padding columns [d, dp) of both chunk buffers
        if (dp != d)
            for (int t = tid; t < 2 * R * (dp - d); t += blockDim.x) {
                const int r = t / (dp - d), j = d + t % (dp - d);  // r < 2R: rows of Zc[0] then Zc[1]
                if (DT == DT_BF16) reinterpret_cast<unsigned short *>(Zc[0])[(size_t)r * ZS + j] = 0;
                else reinterpret_cast<float *>(Zc[0])[(size_t)r * ZS + j] = 0.f;
            }
        __syncthreads();

        // ---- one pass: W = Z^T (Z V) / N ----
        float Wacc[JU][RK];
#pragma unroll
        for (int u = 0; u < JU; ++u)
#pragma unroll
            for (int c = 0; c < RK; ++c) Wacc[u][c] = 0.f;
        ritz_stage<DT, R>(Zc[0], Z, pm.z_row, 0, N, d, ZS, vec);
        for (int ch = 0; ch < nch; ++ch) {
            if (vec) cp_async_wait_all();
            __syncthreads();  // chunk ch landed; everyone is done with chunk ch - 1
            if (ch + 1 < nch) ritz_stage<DT, R>(Zc[(ch + 1) & 1], Z, pm.z_row, (ch + 1) * R, N, d, ZS, vec);
            const unsigned char *zc = Zc[ch & 1];
            // (1) warp partial of P = Zc V over columns [w dp/8, (w+1) dp/8)
            {
                float acc[RI][4];
#pragma unroll
                for (int i = 0; i < RI; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
                const int j0 = w * (dp >> 3), j1 = j0 + (dp >> 3);
#pragma unroll 2
                for (int j = j0; j < j1; j += 4) {
                    float z[RI][4];
#pragma unroll
                    for (int i = 0; i < RI; ++i) TT::load4(zc + (size_t)(rq + 8 * i) * ZS * TT::ES, j, z[i]);
                    float4 v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = *reinterpret_cast<const float4 *>(V + (j + q) * RK + 4 * cg);
#pragma unroll
                    for (int i = 0; i < RI; ++i)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            acc[i][0] = fmaf(z[i][q], v[q].x, acc[i][0]);
                            acc[i][1] = fmaf(z[i][q], v[q].y, acc[i][1]);
                            acc[i][2] = fmaf(z[i][q], v[q].z, acc[i][2]);
                            acc[i][3] = fmaf(z[i][q], v[q].w, acc[i][3]);
                        }
                }
#pragma unroll
                for (int i = 0; i < RI; ++i)
                    *reinterpret_cast<float4 *>(part + ((size_t)w * R + rq + 8 * i) * RK + 4 * cg) =
                        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
            }
            __syncthreads();
            for (int e = tid; e < R * RK; e += blockDim.x) {
                float s = 0.f;
#pragma unroll
                for (int ww = 0; ww < 8; ++ww) s += part[ww * R * RK + e];
                Pm[e] = s;
            }
            __syncthreads();
            // (2) W += Zc^T P for the rows j = tid + 256 u this thread owns
#pragma unroll 4
            for (int r = 0; r < R; ++r) {
                const float4 p0 = *reinterpret_cast<const float4 *>(Pm + r * RK);
                const float4 p1 = *reinterpret_cast<const float4 *>(Pm + r * RK + 4);
                const float4 p2 = *reinterpret_cast<const float4 *>(Pm + r * RK + 8);
                const float4 p3 = *reinterpret_cast<const float4 *>(Pm + r * RK + 12);
                const unsigned char *row = zc + (size_t)r * ZS * TT::ES;
#pragma unroll
                for (int u = 0; u < JU; ++u) {
                    const int j = tid + 256 * u;
                    const float z = j < d ? TT::load1(row, j) : 0.f;
                    const float pv[RK] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w,
                                          p2.x, p2.y, p2.z, p2.w, p3.x, p3.y, p3.z, p3.w};
#pragma unroll
                    for (int c = 0; c < RK; ++c) Wacc[u][c] = fmaf(z, pv[c], Wacc[u][c]);
                }
            }
        }
        __syncthreads();  // all reads of the chunk buffers done
#pragma unroll
        for (int u = 0; u < JU; ++u) {
            const int j = tid + 256 * u;
            if (j < d)
#pragma unroll
                for (int c = 0; c < RK; c += 4)
                    *reinterpret_cast<float4 *>(Wsm + j * RK + c) =
                        make_float4(Wacc[u][c] * invN, Wacc[u][c + 1] * invN, Wacc[u][c + 2] * invN,
                                    Wacc[u][c + 3] * invN);
        }
        __syncthreads();
    }
    // Rayleigh-Ritz: H = V^T W (V orthonormal, W = S V), one entry per thread
    {
        const int a = tid >> 4, bb = tid & 15;
        float h0 = 0.f, h1 = 0.f;
        int j = 0;
        for (; j + 1 < d; j += 2) {
            h0 = fmaf(V[j * RK + a], Wsm[j * RK + bb], h0);
            h1 = fmaf(V[(j + 1) * RK + a], Wsm[(j + 1) * RK + bb], h1);
        }
        if (j < d) h0 = fmaf(V[j * RK + a], Wsm[j * RK + bb], h0);
        Hm[a][bb] = h0 + h1;
    }
    __syncthreads();
    if (w == 0) ritz_jacobi(Hm, lam_out + (size_t)p * RK);
}

// ---------------------------------------------------------------------------
// BF16 Ritz values on the warp-level tensor-core MMA (mma.sync m16n8k16, BF16
// operands, FP32 accumulation), one CTA (256 threads, 8 warps) per pair.
//
// The contraction is skinny (16 columns), so the MMA's role is to take the
// 2 x 16 FMAs of every element of Z off the FP32 pipe; tcgen05 tiles
// (128 rows x N >= 16, operands through shared-memory descriptors) would
// read the same operands at no higher rate for N = 16.  Z is exact in BF16;
// the other factor of each product (V in P = Zc V, P in W += Zc^T P) is split
// into a BF16 pair x = hi + lo, hi = rn(x), lo = rn(x - hi), which carries
// about 16 significant bits, and both halves go through the MMA into the same
// FP32 accumulator.  Chunks of 16 rows; warp w owns the K range (columns of
// Z) [128 w KS / 8 ... ) in P = Zc V (its partial tile is summed with the
// others through shared memory) and the same rows of W, kept in registers for
// the whole pass.  dpm = d rounded up to 128 (= 128 KS); columns [d, dpm) of
// the chunk buffers and of V stay zero.
// dynamic smem: Zc[2][16][ZS] BF16, Vh/Vl[16][ZS] BF16 (V transposed),
// part[8][16][16] FP32, Ph/Pl[16][24] BF16  (ZS = dpm + 8)
// ---------------------------------------------------------------------------
constexpr int RM_R = 16;   // rows per chunk
constexpr int RM_PS = 24;  // row stride of the P tiles in BF16 elements (48 B: ldmatrix rows on distinct banks)

__host__ __device__ __forceinline__ int ritz_dpm(int d) { return (d + 127) & ~127; }

__host__ __device__ __forceinline__ size_t ritz_mma_smem(int d)
{
    const size_t zs = (size_t)ritz_dpm(d) + 8;
    return 2 * RM_R * zs * 2 + 2 * RK * zs * 2 + sizeof(float) * 8 * RM_R * RK + 2 * RM_R * RM_PS * 2;
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr)
                 : "memory");
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr)
                 : "memory");
}

// c += A (16 x 16, row) B (16 x 8, col), BF16 operands, FP32 accumulator
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};\n"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void bf16_split(float x, unsigned short &hi, unsigned short &lo)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
}

__device__ __forceinline__ float bf16_bits_to_float(unsigned short b) { return __uint_as_float((uint32_t)b << 16); }

template <int KS>
__global__ void __launch_bounds__(256, 2) k_ritz_mma(const PairMeta *__restrict__ meta, const RunOpts o,
                                                     const PairState *__restrict__ st, const void *__restrict__ Z,
                                                     float *__restrict__ lam_out)
{
    constexpr int dpm = 128 * KS, ZS = dpm + 8;
    constexpr size_t zc_bytes = (size_t)RM_R * ZS * 2;
    extern __shared__ __align__(16) unsigned char sm_ritz[];
    __shared__ float Hm[RK][RK];
    __shared__ float Rinv[RK][RK];
    const int p = blockIdx.x;
    if (st[p].status != ST_OK) {
        if (threadIdx.x < RK) lam_out[p * RK + threadIdx.x] = 0.f;
        return;
    }
    const PairMeta pm = meta[p];
    const int d = o.d, N = pm.N;
    unsigned char *Zc[2] = {sm_ritz, sm_ritz + zc_bytes};
    unsigned short *Vh = reinterpret_cast<unsigned short *>(sm_ritz + 2 * zc_bytes);
    unsigned short *Vl = Vh + (size_t)RK * ZS;
    float *part = reinterpret_cast<float *>(Vl + (size_t)RK * ZS);
    unsigned short *Ph = reinterpret_cast<unsigned short *>(part + 8 * RM_R * RK);
    unsigned short *Pl = Ph + RM_R * RM_PS;
    float *Wsm = reinterpret_cast<float *>(Zc[0]);  // W between passes, [d][16], over both chunk buffers
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, g = lane >> 2, tig = lane & 3;
    const int li = lane >> 3, lr = lane & 7;  // ldmatrix: this lane's matrix and row
    const bool vec = (d * 2) % 16 == 0;
    // staging walk of this thread (vector rows): item tid + 256 k is row r, piece q
    const int per_row = d / 8, st_dr = 256 / per_row, st_dq = 256 % per_row;
    const int st_r = tid / per_row, st_q = tid % per_row;
    const int64_t row_bytes = (int64_t)d * 2;
    const unsigned char *zrow0 = reinterpret_cast<const unsigned char *>(Z) + pm.z_row * row_bytes;
    const uint32_t zc_s0 = (uint32_t)__cvta_generic_to_shared(Zc[0]);
    const uint32_t vh_s = (uint32_t)__cvta_generic_to_shared(Vh), vl_s = (uint32_t)__cvta_generic_to_shared(Vl);
    const uint32_t ph_s = (uint32_t)__cvta_generic_to_shared(Ph), pl_s = (uint32_t)__cvta_generic_to_shared(Pl);

    // zero the chunk buffers and V once: columns [d, dpm) of V stay zero
    for (size_t t = tid; t < (2 * zc_bytes + 2 * (size_t)RK * ZS * 2) / 4; t += blockDim.x)
        reinterpret_cast<float *>(sm_ritz)[t] = 0.f;
    __syncthreads();
    // fixed start block: (w >> 8) / 2^24 - 1/2, w = Philox(j, c, 0x5EED, 0; key 0, 0) word 0
    for (int t = tid; t < d * RK; t += blockDim.x) {
        const int j = t >> 4, c = t & 15;
        const uint4 r = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)c, 0x5EEDu, 0u), 0u, 0u);
        Wsm[t] = (float)(r.x >> 8) * (1.0f / 16777216.0f) - 0.5f;
    }
    __syncthreads();
    const int nch = (N + RM_R - 1) / RM_R;
    const float invN = 1.0f / (float)N;
    for (int iter = 0; iter <= RITZ_ITERS; ++iter) {
        // ---- V = orth(W) = W R^-1, stored transposed as BF16 pairs ----
        ritz_rinv(Wsm, d, Hm, Rinv);
        for (int t = tid; t < d * RK; t += blockDim.x) {
            const int j = t >> 4, c = t & 15;
            float v = 0.f;
            for (int k = 0; k <= c; ++k) v = fmaf(Wsm[j * RK + k], Rinv[k][c], v);
            bf16_split(v, Vh[c * ZS + j], Vl[c * ZS + j]);
        }
        __syncthreads();
        // the W staging overwrote columns [d, dpm) of the chunk rows
        if (dpm != d)
            for (int t = tid; t < 2 * RM_R * (dpm - d); t += blockDim.x) {
                const int r = t / (dpm - d), j = d + t % (dpm - d);  // r < 32: rows of Zc[0] then Zc[1]
                reinterpret_cast<unsigned short *>(Zc[0])[(size_t)r * ZS + j] = 0;
            }
        __syncthreads();

        // ---- one pass: W = Z^T (Z V) / N ----
        float wacc[KS][2][4];
#pragma unroll
        for (int m = 0; m < KS; ++m)
#pragma unroll
            for (int n = 0; n < 2; ++n)
#pragma unroll
                for (int q = 0; q < 4; ++q) wacc[m][n][q] = 0.f;
        if (vec) ritz_stage_vec(Zc[0], zrow0, N, per_row, ZS * 2, row_bytes, st_r, st_q, st_dr, st_dq, RM_R);
        else ritz_stage<DT_BF16, RM_R>(Zc[0], Z, pm.z_row, 0, N, d, ZS, vec);
        for (int ch = 0; ch < nch; ++ch) {
            if (vec) cp_async_wait_all();
            __syncthreads();  // chunk ch landed; everyone is done with chunk ch - 1 and the P tiles
            if (ch + 1 < nch) {
                const int r0 = (ch + 1) * RM_R;
                if (vec)
                    ritz_stage_vec(Zc[(ch + 1) & 1], zrow0 + r0 * row_bytes, N - r0, per_row, ZS * 2, row_bytes,
                                   st_r, st_q, st_dr, st_dq, RM_R);
                else
                    ritz_stage<DT_BF16, RM_R>(Zc[(ch + 1) & 1], Z, pm.z_row, r0, N, d, ZS, vec);
            }
            const uint32_t zs = zc_s0 + (uint32_t)((ch & 1) * zc_bytes);
            // (1) this warp's partial of P = Zc V over its K range
            {
                float pacc[4][4];  // n-tile 0 hi, lo, n-tile 1 hi, lo: four independent MMA chains
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 4; ++q) pacc[i][q] = 0.f;
#pragma unroll
                for (int ks = 0; ks < KS; ++ks) {
                    const int k0 = (w * KS + ks) * 16;
                    uint32_t a[4], bh[4], bl[4];
                    // A = Zc[0:16, k0:k0+16]: matrices (rows 0-7 | 8-15) x (cols k0 | k0 + 8)
                    ldsm_x4(zs + (uint32_t)((((li & 1) * 8 + lr) * ZS + k0 + (li >> 1) * 8) * 2), a);
                    // B = V[k0:k0+16, 0:16] from V^T: matrices (n 0-7 | 8-15) x (k0 | k0 + 8)
                    const uint32_t vo = (uint32_t)((((li >> 1) * 8 + lr) * ZS + k0 + (li & 1) * 8) * 2);
                    ldsm_x4(vh_s + vo, bh);
                    ldsm_x4(vl_s + vo, bl);
                    mma_bf16_16816(pacc[0], a, bh[0], bh[1]);
                    mma_bf16_16816(pacc[1], a, bl[0], bl[1]);
                    mma_bf16_16816(pacc[2], a, bh[2], bh[3]);
                    mma_bf16_16816(pacc[3], a, bl[2], bl[3]);
                }
                // partial tile, columns of rows with bit 1 of the row set swapped by 8 halves (rows g and
                // g + 2 would share banks): stored at col ^ 8 ((row >> 1) & 1)
                float *pw = part + w * (RM_R * RK);
                const int sw = ((g >> 1) & 1) << 3;  // rows g and g + 8 have the same swap
#pragma unroll
                for (int n = 0; n < 2; ++n) {
                    const int c = (n * 8 + 2 * tig) ^ sw;
                    *reinterpret_cast<float2 *>(pw + g * RK + c) =
                        make_float2(pacc[2 * n][0] + pacc[2 * n + 1][0], pacc[2 * n][1] + pacc[2 * n + 1][1]);
                    *reinterpret_cast<float2 *>(pw + (g + 8) * RK + c) =
                        make_float2(pacc[2 * n][2] + pacc[2 * n + 1][2], pacc[2 * n][3] + pacc[2 * n + 1][3]);
                }
            }
            __syncthreads();
            {  // P = sum of the 8 partials (one entry per thread), as a BF16 pair
                const int r = tid >> 4, c = tid & 15, e = r * RK + (c ^ (((r >> 1) & 1) << 3));
                float s = 0.f;
#pragma unroll
                for (int ww = 0; ww < 8; ++ww) s += part[ww * RM_R * RK + e];
                bf16_split(s, Ph[r * RM_PS + c], Pl[r * RM_PS + c]);
            }
            __syncthreads();
            // (2) W += Zc^T P for this warp's rows of W
            uint32_t bh[4], bl[4];
            {  // B = P[0:16, 0:16]: matrices (t 0-7 | 8-15) x (n 0-7 | 8-15), transposed on load
                const uint32_t po = (uint32_t)((((li & 1) * 8 + lr) * RM_PS + (li >> 1) * 8) * 2);
                ldsm_x4_t(ph_s + po, bh);
                ldsm_x4_t(pl_s + po, bl);
            }
#pragma unroll
            for (int mt = 0; mt < KS; ++mt) {
                const int j0 = (w * KS + mt) * 16;
                uint32_t a[4];
                // A = Zc^T[j0:j0+16, 0:16]: matrices (j0 | j0 + 8) x (t 0-7 | 8-15), transposed on load
                ldsm_x4_t(zs + (uint32_t)((((li >> 1) * 8 + lr) * ZS + j0 + (li & 1) * 8) * 2), a);
                mma_bf16_16816(wacc[mt][0], a, bh[0], bh[1]);
                mma_bf16_16816(wacc[mt][0], a, bl[0], bl[1]);
                mma_bf16_16816(wacc[mt][1], a, bh[2], bh[3]);
                mma_bf16_16816(wacc[mt][1], a, bl[2], bl[3]);
            }
        }
        __syncthreads();  // all reads of the chunk buffers done
#pragma unroll
        for (int mt = 0; mt < KS; ++mt) {
            const int j = (w * KS + mt) * 16 + g;
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                const int c = n * 8 + 2 * tig;
                if (j < d)
                    *reinterpret_cast<float2 *>(Wsm + j * RK + c) =
                        make_float2(wacc[mt][n][0] * invN, wacc[mt][n][1] * invN);
                if (j + 8 < d)
                    *reinterpret_cast<float2 *>(Wsm + (j + 8) * RK + c) =
                        make_float2(wacc[mt][n][2] * invN, wacc[mt][n][3] * invN);
            }
        }
        __syncthreads();
    }
    // Rayleigh-Ritz: H = V^T W (V orthonormal, W = S V), one entry per thread
    {
        const int a = tid >> 4, bb = tid & 15;
        float h0 = 0.f, h1 = 0.f;
        for (int j = 0; j < d; ++j) {
            h0 = fmaf(bf16_bits_to_float(Vh[a * ZS + j]), Wsm[j * RK + bb], h0);
            h1 = fmaf(bf16_bits_to_float(Vl[a * ZS + j]), Wsm[j * RK + bb], h1);
        }
        Hm[a][bb] = h0 + h1;
    }
    __syncthreads();
    if (w == 0) ritz_jacobi(Hm, lam_out + (size_t)p * RK);
}

__global__ void k_features_pack(const PairMeta *__restrict__ meta, int P, const RunOpts o,
                                const PairState *__restrict__ st, const float *__restrict__ lam,
                                float *__restrict__ feat, double *__restrict__ tobs)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const PairMeta pm = meta[p];
    const bool ok = st[p].status == ST_OK;
    float *f = feat + (int64_t)p * MLP_IN;
    f[0] = logf((float)pm.n);
    f[1] = logf((float)pm.m);
    for (int k = 0; k < RK; ++k) f[2 + k] = ok ? logf(fmaxf(lam[p * RK + k] * (float)o.d, 1e-12f)) : 0.f;
    f[18] = ok ? (float)(10.0 * st[p].To) : 0.f;
    if (tobs) tobs[p] = ok ? st[p].To : 0.0;
}

// ---------------------------------------------------------------------------
// Tiled SIMT GEMM for the MLP: C[M][N] (=|+=) A[M][K] B[K][N] with strided
// operands (so transposes are free), FP32 accumulation.  64 x 64 tiles,
// 256 threads, 4 x 4 outputs per thread.
// Epilogue: 0 store, 1 store(acc + bias[n]) with optional ReLU,
//           2 store acc * (mask[m][n] > 0)
// ---------------------------------------------------------------------------
struct Mat {
    const void *ptr;
    int64_t rs, cs;  // element strides of (row, col)
    int bf16;        // 1 = BF16 elements
    __device__ __forceinline__ float at(int64_t r, int64_t c) const
    {
        const int64_t i = r * rs + c * cs;
        if (bf16) return __uint_as_float((uint32_t)reinterpret_cast<const unsigned short *>(ptr)[i] << 16);
        return reinterpret_cast<const float *>(ptr)[i];
    }
};

__global__ void __launch_bounds__(256) k_mlp_gemm(int M, int N, int K, Mat A, Mat B, float *__restrict__ C, int64_t ldc,
                                                  int mode, const float *__restrict__ bias, int relu,
                                                  const float *__restrict__ mask, int64_t ldm, int kchunk)
{
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int k_begin = blockIdx.z * kchunk, k_end = min(K, k_begin + kchunk);
    float acc[4][4] = {};
    for (int k0 = k_begin; k0 < k_end; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int kk = t / 64, i = t % 64;
            const int k = k0 + kk;
            As[kk][i] = (m0 + i < M && k < k_end) ? A.at(m0 + i, k) : 0.f;
            Bs[kk][i] = (n0 + i < N && k < k_end) ? B.at(k, n0 + i) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][ty * 4 + u];
                b[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
    float *Cz = C + (int64_t)blockIdx.z * (int64_t)M * ldc;  // split-K partials are stacked
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int m = m0 + ty * 4 + u;
        if (m >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int n = n0 + tx * 4 + v;
            if (n >= N) continue;
            float x = acc[u][v];
            if (mode == 1) {
                x += bias ? bias[n] : 0.f;
                if (relu) x = fmaxf(x, 0.f);
            } else if (mode == 2) {
                x = mask[(int64_t)m * ldm + n] > 0.f ? x : 0.f;
            }
            Cz[(int64_t)m * ldc + n] = x;
        }
    }
}

// out[i] = sum_z part[z][i] (fixed order)
__global__ void k_sum_partials(const float *__restrict__ part, int nz, int64_t n, float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int z = 0; z < nz; ++z) s += part[(int64_t)z * n + i];
    out[i] = s;
}

// db[n] = sum_m D[m][n] in fixed order, one thread per column
__global__ void k_colsum_f32(const float *__restrict__ D, int M, int N, float *__restrict__ db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += D[(int64_t)m * N + n];
    db[n] = s;
}

// h = relu(a) in place copy
__global__ void k_relu(const float *__restrict__ a, float *__restrict__ h, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) h[i] = fmaxf(a[i], 0.f);
}

// pinball loss and its gradient; per-block loss partials
__global__ void k_pinball(const float *__restrict__ y, const float *__restrict__ target, int P,
                          float *__restrict__ dy, float *__restrict__ loss_part)
{
    const float lv[MLP_OUT] = {0.5f, 0.8f, 0.9f, 0.95f, 0.975f, 0.99f, 0.995f, 0.998f, 0.999f};
    __shared__ float red[8];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < (int64_t)P * MLP_OUT) {
        const float tau = lv[i % MLP_OUT];
        const float u = target[i] - y[i];
        l = u >= 0.f ? tau * u : (tau - 1.0f) * u;
        dy[i] = -(u >= 0.f ? tau : tau - 1.0f) / ((float)P * (float)MLP_OUT);
    }
    const float s = block_sum(l, red);
    if (threadIdx.x == 0) loss_part[blockIdx.x] = s;
}

__global__ void k_loss_final(const float *__restrict__ part, int nb, int P, float *__restrict__ loss)
{
    if (threadIdx.x || blockIdx.x) return;
    float s = 0.f;
    for (int k = 0; k < nb; ++k) s += part[k];
    *loss = s / ((float)P * (float)MLP_OUT);
}

// Adam (Kingma and Ba, 2015) and the BF16 copy of the parameters
__global__ void k_adam(float *__restrict__ w, unsigned short *__restrict__ wh, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wh[i] = __bfloat16_as_ushort(__float2bfloat16_rn(wi));
}

__global__ void k_to_bf16(const float *__restrict__ w, unsigned short *__restrict__ wh, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) wh[i] = __bfloat16_as_ushort(__float2bfloat16_rn(w[i]));
}

// ---------------------------------------------------------------------------
// null quantiles of |T_b| per pair: bitonic sort in shared memory
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_null_quantiles(const PairMeta *__restrict__ meta, const float *__restrict__ T,
                                                          const PairState *__restrict__ st, float scale,
                                                          float *__restrict__ q_out)
{
    extern __shared__ float sv[];
    const double lv[MLP_OUT] = {0.5, 0.8, 0.9, 0.95, 0.975, 0.99, 0.995, 0.998, 0.999};
    const int p = blockIdx.x;
    const PairMeta pm = meta[p];
    const int B = (int)pm.B;
    int L = 1;
    while (L < B) L <<= 1;
    for (int i = threadIdx.x; i < L; i += blockDim.x) sv[i] = i < B ? fabsf(T[pm.T_off + i]) : INFINITY;
    __syncthreads();
    for (int k = 2; k <= L; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < L; i += blockDim.x) {
                const int x = i ^ j;
                if (x > i) {
                    const bool up = (i & k) == 0;
                    const float a = sv[i], b = sv[x];
                    if ((a > b) == up) {
                        sv[i] = b;
                        sv[x] = a;
                    }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x < MLP_OUT) {
        // the ceil(level * B)-th smallest value (level * B evaluated in FP64)
        const int64_t k = (int64_t)ceil(lv[threadIdx.x] * (double)B) - 1;
        const bool ok = st[p].status == ST_OK;
        q_out[p * MLP_OUT + threadIdx.x] = ok ? scale * sv[max((int64_t)0, k)] : 0.f;
    }
}

// predicted p from predicted (scaled) quantiles and |T_obs| (see the oracle's definition)
__global__ void k_predict_p(int P, const float *__restrict__ q_scaled, float scale, const double *__restrict__ tobs,
                            float *__restrict__ p_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const double lv[MLP_OUT] = {0.5, 0.8, 0.9, 0.95, 0.975, 0.99, 0.995, 0.998, 0.999};
    double q[MLP_OUT];
    double run = -1e300;
    for (int k = 0; k < MLP_OUT; ++k) {
        run = fmax(run, (double)q_scaled[(int64_t)i * MLP_OUT + k] / (double)scale);
        q[k] = run;
    }
    const double t = fabs(tobs[i]);
    double F;
    if (t <= q[0]) {
        F = lv[0] * (q[0] > 0 ? t / q[0] : 1.0);
    } else if (t >= q[MLP_OUT - 1]) {
        const double span = fmax(q[MLP_OUT - 1] - q[MLP_OUT - 2], 1e-12);
        F = lv[MLP_OUT - 1] + (1.0 - lv[MLP_OUT - 1]) * fmin(1.0, (t - q[MLP_OUT - 1]) / span);
        F = fmin(F, 1.0 - 1e-4);
    } else {
        int k = 0;
        while (k < MLP_OUT - 2 && q[k + 1] <= t) ++k;
        const double w = (t - q[k]) / fmax(q[k + 1] - q[k], 1e-12);
        F = lv[k] + w * (lv[k + 1] - lv[k]);
    }
    p_out[i] = (float)(1.0 - F);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int DT>
static size_t ritz_smem(int d)
{
    const size_t dp = (size_t)((d + 31) & ~31);
    return 2 * ritz_zc_bytes<DT>(d) + sizeof(float) * (dp * RK + 8 * RitzTile<DT>::R * RK + RitzTile<DT>::R * RK);
}

template <int DT, int JU>
static void launch_ritz(const PairMeta *meta, int P, const RunOpts &o, const PairState *st, const void *Z, float *lam,
                        cudaStream_t s)
{
    const size_t smem = ritz_smem<DT>(o.d);
    cudaFuncSetAttribute(k_ritz<DT, JU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ritz<DT, JU><<<P, 256, smem, s>>>(meta, o, st, Z, lam);
}

template <int DT>
static void launch_ritz_ju(const PairMeta *meta, int P, const RunOpts &o, const PairState *st, const void *Z,
                           float *lam, cudaStream_t s)
{
    switch ((o.d + 255) / 256) {  // rows of W per thread; d <= 1024 is checked by the caller
    case 1: launch_ritz<DT, 1>(meta, P, o, st, Z, lam, s); break;
    case 2: launch_ritz<DT, 2>(meta, P, o, st, Z, lam, s); break;
    case 3: launch_ritz<DT, 3>(meta, P, o, st, Z, lam, s); break;
    default: launch_ritz<DT, 4>(meta, P, o, st, Z, lam, s); break;
    }
}

template <int KS>
static void launch_ritz_mma(const PairMeta *meta, int P, const RunOpts &o, const PairState *st, const void *Z,
                            float *lam, cudaStream_t s)
{
    const size_t smem = ritz_mma_smem(o.d);
    cudaFuncSetAttribute(k_ritz_mma<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ritz_mma<KS><<<P, 256, smem, s>>>(meta, o, st, Z, lam);
}

void launch_features(const PairMeta *meta, int P, const RunOpts &o, const PairState *st, const void *Z, float *lam,
                     float *feat, double *tobs, cudaStream_t s)
{
    if (o.dtype == DT_F32) {
        launch_ritz_ju<DT_F32>(meta, P, o, st, Z, lam, s);
    } else {
        switch (ritz_dpm(o.d) / 128) {  // K steps of 16 per warp; d <= 1024 is checked by the caller
        case 1: launch_ritz_mma<1>(meta, P, o, st, Z, lam, s); break;
        case 2: launch_ritz_mma<2>(meta, P, o, st, Z, lam, s); break;
        case 3: launch_ritz_mma<3>(meta, P, o, st, Z, lam, s); break;
        case 4: launch_ritz_mma<4>(meta, P, o, st, Z, lam, s); break;
        case 5: launch_ritz_mma<5>(meta, P, o, st, Z, lam, s); break;
        case 6: launch_ritz_mma<6>(meta, P, o, st, Z, lam, s); break;
        case 7: launch_ritz_mma<7>(meta, P, o, st, Z, lam, s); break;
        default: launch_ritz_mma<8>(meta, P, o, st, Z, lam, s); break;
        }
    }
    k_features_pack<<<(P + 127) / 128, 128, 0, s>>>(meta, P, o, st, lam, feat, tobs);
}

void launch_null_quantiles(const PairMeta *meta, int P, int max_B, const float *T, const PairState *st, float scale,
                           float *q_out, cudaStream_t s)
{
    int L = 1;
    while (L < max_B) L <<= 1;
    const size_t smem = sizeof(float) * (size_t)L;
    cudaFuncSetAttribute(k_null_quantiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_null_quantiles<<<P, 1024, smem, s>>>(meta, T, st, scale, q_out);
}

static void gemm(int M, int N, int K, Mat A, Mat B, float *C, int64_t ldc, int mode, const float *bias, int relu,
                 const float *mask, int64_t ldm, cudaStream_t s, int splitk = 1, int kchunk = 0)
{
    if (kchunk <= 0) kchunk = K;
    const dim3 g((N + 63) / 64, (M + 63) / 64, splitk);
    k_mlp_gemm<<<g, 256, 0, s>>>(M, N, K, A, B, C, ldc, mode, bias, relu, mask, ldm, kchunk);
}

// parameter offsets: W1[19][256], b1, W2[256][256], b2, W3[256][9], b3
struct MlpOffsets {
    int64_t W1 = 0, b1 = MLP_IN * MLP_H, W2 = b1 + MLP_H, b2 = W2 + MLP_H * MLP_H, W3 = b2 + MLP_H,
            b3 = W3 + MLP_H * MLP_OUT, total = b3 + MLP_OUT;
};

int64_t mlp_param_count() { return MlpOffsets().total; }

// workspace floats: a1, h1, a2, h2 [P][256], y [P][9], dy [P][9], da2, da1 [P][256], partials
int64_t mlp_work_floats(int P)
{
    const int64_t splitk = std::max<int64_t>(1, (P + 4095) / 4096);
    const int64_t nb = ((int64_t)P * MLP_OUT + 255) / 256;
    return (int64_t)P * (6 * MLP_H + 2 * MLP_OUT) + (nb + 64) / 64 * 64 + splitk * (int64_t)MLP_H * MLP_H;
}

void mlp_forward(const float *params, const unsigned short *wh, int P, const float *feat, float *work, float *y_out,
                 cudaStream_t s)
{
    const MlpOffsets O;
    float *a1 = work, *h1 = a1 + (int64_t)P * MLP_H, *a2 = h1 + (int64_t)P * MLP_H, *h2 = a2 + (int64_t)P * MLP_H;
    const Mat F{feat, MLP_IN, 1, 0};
    gemm(P, MLP_H, MLP_IN, F, Mat{wh + O.W1, MLP_H, 1, 1}, a1, MLP_H, 1, params + O.b1, 0, nullptr, 0, s);
    k_relu<<<(unsigned)(((int64_t)P * MLP_H + 255) / 256), 256, 0, s>>>(a1, h1, (int64_t)P * MLP_H);
    gemm(P, MLP_H, MLP_H, Mat{h1, MLP_H, 1, 0}, Mat{wh + O.W2, MLP_H, 1, 1}, a2, MLP_H, 1, params + O.b2, 0,
         nullptr, 0, s);
    k_relu<<<(unsigned)(((int64_t)P * MLP_H + 255) / 256), 256, 0, s>>>(a2, h2, (int64_t)P * MLP_H);
    gemm(P, MLP_OUT, MLP_H, Mat{h2, MLP_H, 1, 0}, Mat{wh + O.W3, MLP_OUT, 1, 1}, y_out, MLP_OUT, 1, params + O.b3,
         0, nullptr, 0, s);
}

// gradient of the mean pinball loss; the forward must have run on `work`
void mlp_backward(const float *params, const unsigned short *wh, int P, const float *feat, const float *target,
                  float *work, float *grad, float *loss, cudaStream_t s)
{
    (void)params;  // the backward multiplies by the BF16 weights `wh` the forward used
    const MlpOffsets O;
    float *a1 = work, *h1 = a1 + (int64_t)P * MLP_H, *a2 = h1 + (int64_t)P * MLP_H, *h2 = a2 + (int64_t)P * MLP_H;
    float *y = h2 + (int64_t)P * MLP_H, *dy = y + (int64_t)P * MLP_OUT;
    float *da2 = dy + (int64_t)P * MLP_OUT, *da1 = da2 + (int64_t)P * MLP_H, *part = da1 + (int64_t)P * MLP_H;
    const int nb = (int)(((int64_t)P * MLP_OUT + 255) / 256);
    float *lpart = part;
    float *gpart = part + ((int64_t)nb + 64) / 64 * 64;
    k_pinball<<<nb, 256, 0, s>>>(y, target, P, dy, lpart);
    k_loss_final<<<1, 32, 0, s>>>(lpart, nb, P, loss);
    const int splitk = std::max(1, (P + 4095) / 4096);
    const int kch = (P + splitk - 1) / splitk;
    auto wgrad = [&](int M, int N, const float *Xin, int64_t ldx, const float *D, int64_t ldd, float *out) {
        // out[M][N] = Xin^T D over the P rows, split along P, partials summed in order
        gemm(M, N, P, Mat{Xin, 1, ldx, 0}, Mat{D, ldd, 1, 0}, gpart, N, 0, nullptr, 0, nullptr, 0, s, splitk,
             (kch + 15) / 16 * 16);
        k_sum_partials<<<(unsigned)(((int64_t)M * N + 255) / 256), 256, 0, s>>>(gpart, splitk, (int64_t)M * N, out);
    };
    // layer 3
    wgrad(MLP_H, MLP_OUT, h2, MLP_H, dy, MLP_OUT, grad + O.W3);
    k_colsum_f32<<<1, 32, 0, s>>>(dy, P, MLP_OUT, grad + O.b3);
    // da2 = (dy W3^T) * (a2 > 0)
    gemm(P, MLP_H, MLP_OUT, Mat{dy, MLP_OUT, 1, 0}, Mat{wh + O.W3, 1, MLP_OUT, 1}, da2, MLP_H, 2, nullptr, 0, a2,
         MLP_H, s);
    wgrad(MLP_H, MLP_H, h1, MLP_H, da2, MLP_H, grad + O.W2);
    k_colsum_f32<<<(MLP_H + 127) / 128, 128, 0, s>>>(da2, P, MLP_H, grad + O.b2);
    // da1 = (da2 W2^T) * (a1 > 0)
    gemm(P, MLP_H, MLP_H, Mat{da2, MLP_H, 1, 0}, Mat{wh + O.W2, 1, MLP_H, 1}, da1, MLP_H, 2, nullptr, 0, a1, MLP_H,
         s);
    wgrad(MLP_IN, MLP_H, feat, MLP_IN, da1, MLP_H, grad + O.W1);
    k_colsum_f32<<<(MLP_H + 127) / 128, 128, 0, s>>>(da1, P, MLP_H, grad + O.b1);
}

void mlp_adam(float *params, unsigned short *wh, const float *grad, float *m, float *v, float lr, int64_t t,
              cudaStream_t s)
{
    const int64_t n = mlp_param_count();
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, wh, grad, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
}

void mlp_to_bf16(const float *params, unsigned short *wh, cudaStream_t s)
{
    const int64_t n = mlp_param_count();
    k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(params, wh, n);
}

void launch_predict_p(int P, const float *q_scaled, float scale, const double *tobs, float *p_out, cudaStream_t s)
{
    k_predict_p<<<(P + 127) / 128, 128, 0, s>>>(P, q_scaled, scale, tobs, p_out);
}

}  // namespace hb
