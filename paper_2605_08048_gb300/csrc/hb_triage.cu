// hb_triage.cu -- kernels of the learned triage (a task component; the paper
// has no learned part): per-pair features, the 19 -> 256 -> 256 -> 9 MLP that
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
// Ritz values of Z^T Z / N, one CTA (256 threads, 8 warps) per pair.
//
// One pass W = Z^T (Z V) streams Z through shared memory in chunks of R rows
// (cp.async double buffer).  Per chunk: (1) P = Zc V (R x 16): warp w takes
// the w-th eighth of the columns j, lane (rq, cg) rows rq + 8i and columns
// 4cg..4cg+3, then the 8 warp partials are summed; (2) W += Zc^T P: thread t
// owns rows j = t + 256u of W, kept in registers for the whole pass.
// Between passes W goes to shared memory (over both chunk buffers, which hold
// at least d x 16 floats) for the orthonormalisation V = W R^-1 (Cholesky-QR
// of W^T W = R^T R).  Chunks of 16 (BF16) or 8 (FP32) rows keep the shared
// memory of a CTA near 110 KB and its registers at 128, so that two pairs'
// CTAs share an SM and one's barriers and serial steps overlap the other's
// streaming.
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

// stage rows [r0, r0 + R) of the pair into a chunk buffer (rows past N read as zero)
template <int DT>
__device__ __forceinline__ void ritz_stage(unsigned char *buf, const void *Z, int64_t z_row, int r0, int N, int d,
                                           bool vec)
{
    using TT = RitzTile<DT>;
    const int ZS = ritz_dp(d) + TT::PAD;
    const unsigned char *src = reinterpret_cast<const unsigned char *>(Z);
    if (vec) {  // rows of d elements are a whole number of 16-byte pieces
        const int per_row = d * TT::ES / 16;
        for (int t = threadIdx.x; t < TT::R * per_row; t += blockDim.x) {
            const int r = t / per_row, q = t - r * per_row;
            const bool in = r0 + r < N;
            const unsigned char *g = in ? src + ((z_row + r0 + r) * (int64_t)d * TT::ES + (int64_t)q * 16) : src;
            cp_async16(buf + (size_t)r * ZS * TT::ES + q * 16, g, in ? 16 : 0);
        }
        cp_async_commit();
    } else {
        for (int t = threadIdx.x; t < TT::R * d; t += blockDim.x) {
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
    __shared__ float jc[8], js[8];
    __shared__ int ja[8], jb[8];
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
        if (tid == 0) {
            float Rm[RK][RK];
            for (int i = 0; i < RK; ++i)
                for (int k = 0; k < RK; ++k) Rm[i][k] = 0.f;
            for (int k = 0; k < RK; ++k) {  // G = R^T R, R upper triangular
                float s = Hm[k][k];
                for (int i = 0; i < k; ++i) s -= Rm[i][k] * Rm[i][k];
                const float rkk = sqrtf(fmaxf(s, 1e-30f));
                Rm[k][k] = rkk;
                for (int c = k + 1; c < RK; ++c) {
                    float t = Hm[k][c];
                    for (int i = 0; i < k; ++i) t -= Rm[i][k] * Rm[i][c];
                    Rm[k][c] = t / rkk;
                }
            }
            for (int c = RK - 1; c >= 0; --c) {  // R^-1, upper triangular
                for (int i = 0; i < RK; ++i) Rinv[i][c] = 0.f;
                Rinv[c][c] = 1.0f / Rm[c][c];
                for (int i = c - 1; i >= 0; --i) {
                    float t = 0.f;
                    for (int k = i + 1; k <= c; ++k) t += Rm[i][k] * Rinv[k][c];
                    Rinv[i][c] = -t / Rm[i][i];
                }
            }
        }
        __syncthreads();
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
        ritz_stage<DT>(Zc[0], Z, pm.z_row, 0, N, d, vec);
        for (int ch = 0; ch < nch; ++ch) {
            if (vec) cp_async_wait_all();
            __syncthreads();  // chunk ch landed; everyone is done with chunk ch - 1
            if (ch + 1 < nch) ritz_stage<DT>(Zc[(ch + 1) & 1], Z, pm.z_row, (ch + 1) * R, N, d, vec);
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
    if (w != 0) return;
    // warp 0: symmetrise, then parallel cyclic Jacobi (round-robin order: 15
    // rounds of 8 disjoint rotations per sweep) until the off-diagonal part is
    // negligible relative to the diagonal
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
        for (int a = 0; a < RK; ++a) lam_out[p * RK + a] = ev[a];
    }
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

void launch_features(const PairMeta *meta, int P, const RunOpts &o, const PairState *st, const void *Z, float *lam,
                     float *feat, double *tobs, cudaStream_t s)
{
    if (o.dtype == DT_F32) launch_ritz_ju<DT_F32>(meta, P, o, st, Z, lam, s);
    else launch_ritz_ju<DT_BF16>(meta, P, o, st, Z, lam, s);
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
