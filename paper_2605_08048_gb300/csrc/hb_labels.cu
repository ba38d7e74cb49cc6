// hb_labels.cu -- HB-LABEL-v1 label draws (the sign matrix S of Sec. 3.2,
// "Vectorized formulation with sign matrices", with bit 1 = group 1).
//
// Philox4x32-10 with key (seed_lo, seed_hi) and counter (i/4, b_lo, stream,
// b_hi); word i%4 serves position i.  Sequential selection sampling (Knuth,
// TAOCP vol. 2, Sec. 3.4.2, Algorithm S): position i joins group 1 iff
// mulhi32(w_i, N - i) < n - (ones so far), which places exactly n ones.
// One thread walks one relabelling b; the walk is inherently sequential in
// i, and the B relabellings give the parallelism.
#include "hb_launch.cuh"

namespace hb {

// Walks relabelling b and hands each finished 32-bit word to `emit(w, word)`.
template <typename Emit>
__device__ __forceinline__ void walk_labels(uint64_t seed, uint32_t stream, int n, int N, uint64_t b, Emit emit)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint32_t blo = (uint32_t)b, bhi = (uint32_t)(b >> 32);
    uint32_t need = (uint32_t)n;
    uint32_t word = 0;
    int i = 0;
    for (; i < N; i += 4) {
        if (need == 0u) break;                       // the rest is group 2
        if (need == (uint32_t)(N - i)) break;        // the rest is group 1
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(i >> 2), blo, stream, bhi), k0, k1);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int pos = i + k;
            if (pos < N) {
                const uint32_t take = __umulhi(ws[k], (uint32_t)(N - pos)) < need;
                word |= take << (pos & 31);
                need -= take;
            }
        }
        if ((i & 31) == 28 || i + 4 >= N) {
            emit(i >> 5, word);
            word = 0;
        }
    }
    if (i < N) {
        // forced tail from position i (i is a multiple of 4): all ones or all zeros
        const bool ones = need != 0u;
        for (int pos = i; pos < N; ++pos) {
            if (ones) word |= 1u << (pos & 31);
            if ((pos & 31) == 31 || pos + 1 == N) {
                emit(pos >> 5, word);
                word = 0;
            }
        }
    }
}

// Row-major [count][W] output (the public hb_perm_labels layout).
__global__ void k_labels_rows(uint64_t seed, uint32_t stream, int n, int N, int64_t b0, int64_t count, uint32_t *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int W = (N + 31) >> 5;
    uint32_t *row = out + k * W;
    for (int w = 0; w < W; ++w) row[w] = 0u;
    walk_labels(seed, stream, n, N, (uint64_t)(b0 + k), [&](int w, uint32_t v) { row[w] = v; });
}

// Pipeline layout: per pair, [W][B_pad] with the relabelling index fastest
// (coalesced stores here, coalesced 128-relabelling tile loads in the GEMMs).
// Grid: x over 128-relabelling tiles, y over pairs.
__global__ void k_labels_pipeline(const PairMeta *__restrict__ meta, const PairState *__restrict__ st, uint64_t seed,
                                  uint32_t stream, uint32_t *__restrict__ bits, int pair0)
{
    const int p = pair0 + blockIdx.y;
    const PairMeta pm = meta[p];
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= pm.B_pad) return;
    uint32_t *col = bits + pm.lab_off + b;
    // labels depend only on (seed, stream, b, n, N), never on the data, so this
    // kernel runs concurrently with the alignment stages (st is not read)
    (void)st;
    if (b >= pm.B) {
        for (int w = 0; w < pm.W; ++w) col[(int64_t)w * pm.B_pad] = 0u;
        return;
    }
    // the walk emits every word 0..W-1 exactly once
    walk_labels(seed, stream, pm.n, pm.N, (uint64_t)b, [&](int w, uint32_t v) { col[(int64_t)w * pm.B_pad] = v; });
}

// Exhaustive mode: relabelling b is the b-th n-subset of {0..N-1} in colex
// order, unranked in the combinatorial number system (b = sum_k C(c_k, k)).
__global__ void k_labels_exhaustive(const PairMeta *__restrict__ meta, uint32_t *__restrict__ bits, int pair0)
{
    __shared__ long long binom[25][25];
    for (int t = threadIdx.x; t < 25 * 25; t += blockDim.x) {
        const int a = t / 25, k = t % 25;
        long long c = 0;
        if (k <= a) {
            c = 1;
            for (int i = 1; i <= k; ++i) c = c * (a - k + i) / i;
        }
        binom[a][k] = c;
    }
    __syncthreads();
    const int p = pair0 + blockIdx.y;
    const PairMeta pm = meta[p];
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= pm.B_pad) return;
    uint32_t mask = 0u;
    if (b < pm.B) {
        long long rem = b;
        int c = pm.N;
        for (int k = pm.n; k >= 1; --k) {
            c = c - 1;
            while (c >= k && binom[c][k] > rem) --c;  // largest c with C(c, k) <= rem
            if (c < k - 1) c = k - 1;
            rem -= (c >= k) ? binom[c][k] : 0;
            mask |= 1u << c;
        }
    }
    bits[pm.lab_off + b] = mask;  // W == 1 for N <= 24
}

void launch_labels_rows(uint64_t seed, uint32_t stream, int n, int N, int64_t b0, int64_t count, uint32_t *out,
                        cudaStream_t st)
{
    k_labels_rows<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(seed, stream, n, N, b0, count, out);
}

void launch_labels_pipeline(const PairMeta *meta, const PairState *pst, int P, int max_Bpad, const RunOpts &o,
                            uint32_t *bits, cudaStream_t st)
{
    for (int p0 = 0; p0 < P; p0 += 65535) {
        const dim3 g((unsigned)((max_Bpad + 127) / 128), (unsigned)min(65535, P - p0));
        if (o.exhaustive) k_labels_exhaustive<<<g, 128, 0, st>>>(meta, bits, p0);
        else k_labels_pipeline<<<g, 128, 0, st>>>(meta, pst, o.seed, o.stream, bits, p0);
    }
}

}  // namespace hb
