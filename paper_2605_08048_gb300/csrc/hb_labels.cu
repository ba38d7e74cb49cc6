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

constexpr uint32_t PH_M0 = 0xD2511F53u, PH_M1 = 0xCD9E8D57u;

// Everything of Philox4x32-10 that depends only on (seed, stream): the ten
// round keys and the round-0 product of the counter word `stream`.  Built on
// the host and passed as a kernel parameter, so it costs no registers.
struct LabelKeys {
    uint32_t rk0[10], rk1[10];
    uint32_t hi_s, lo_s;  // mulhi / mullo of PH_M1 and stream
};

static LabelKeys label_keys(uint64_t seed, uint32_t stream)
{
    LabelKeys k;
    k.rk0[0] = (uint32_t)seed;
    k.rk1[0] = (uint32_t)(seed >> 32);
    for (int r = 1; r < 10; ++r) {
        k.rk0[r] = k.rk0[r - 1] + 0x9E3779B9u;
        k.rk1[r] = k.rk1[r - 1] + 0xBB67AE85u;
    }
    const uint64_t prod = (uint64_t)PH_M1 * stream;
    k.hi_s = (uint32_t)(prod >> 32);
    k.lo_s = (uint32_t)prod;
    return k;
}

// a * b + c (mod 2^32) as one integer multiply-add
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// Walks relabelling b and hands each finished 32-bit word to `emit(w, word)`,
// words in increasing order, each exactly once.  Each group of four positions
// costs the counter multiply of round 0 and nine full rounds.
template <typename Emit>
__device__ __forceinline__ void walk_labels(const LabelKeys &K, int n, int N, uint64_t b, Emit emit)
{
    constexpr uint32_t M0 = PH_M0, M1 = PH_M1;
    const uint32_t blo = (uint32_t)b, bhi = (uint32_t)(b >> 32);
    const uint32_t y0 = K.hi_s ^ blo ^ K.rk0[0];  // round-0 outputs that do not
    const uint32_t y1 = K.lo_s;                   // depend on the position
    const uint32_t *rk0 = K.rk0, *rk1 = K.rk1;
    auto draw = [&](uint32_t q) {
        uint4 c = make_uint4(y0, y1, __umulhi(M0, q) ^ bhi ^ rk1[0], M0 * q);
#pragma unroll
        for (int r = 1; r < 10; ++r) {
            // one widening multiply gives both halves of each product
            const uint64_t p0 = (uint64_t)M0 * c.x, p1 = (uint64_t)M1 * c.z;
            const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
            const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
            c = make_uint4(hi1 ^ c.y ^ rk0[r], lo1, hi0 ^ c.w ^ rk1[r], lo0);
        }
        return c;
    };
    uint32_t need = (uint32_t)n;
    uint32_t word = 0;
    int i = 0;
    bool forced = false;  // the rest is all group 2 (need = 0) or all group 1
    // full words of 32 positions: eight groups of four, the forced test once per word
    for (; i + 32 <= N; i += 32) {
        if (need == 0u || need == (uint32_t)(N - i)) {
            forced = true;
            break;
        }
        uint32_t rem = (uint32_t)(N - i);
        uint32_t wd = 0;
        // the bookkeeping of each decision (need -= t, wd += t 2^k) as integer
        // multiply-adds, which run on the multiply pipe beside the logic pipe that
        // the Philox rounds' XORs and the comparisons keep busy
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            const uint4 w = draw((uint32_t)((i >> 2) + g));
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t t = __umulhi(ws[k], rem - (uint32_t)k) < need;
                need = imad(t, 0xffffffffu, need);
                wd = imad(t, 1u << (4 * g + k), wd);
            }
            rem -= 4u;
        }
        emit(i >> 5, wd);
    }
    // full groups of four positions of the last, partial word
    for (; !forced && i + 4 <= N; i += 4) {
        if (need == 0u || need == (uint32_t)(N - i)) {
            forced = true;
            break;
        }
        const uint4 w = draw((uint32_t)(i >> 2));
        const uint32_t rem = (uint32_t)(N - i);
        const uint32_t t0 = __umulhi(w.x, rem) < need;
        need -= t0;
        const uint32_t t1 = __umulhi(w.y, rem - 1u) < need;
        need -= t1;
        const uint32_t t2 = __umulhi(w.z, rem - 2u) < need;
        need -= t2;
        const uint32_t t3 = __umulhi(w.w, rem - 3u) < need;
        need -= t3;
        word |= (t0 | (t1 << 1) | (t2 << 2) | (t3 << 3)) << (i & 31);
        if ((i & 31) == 28 || i + 4 == N) {
            emit(i >> 5, word);
            word = 0;
        }
    }
    // a last partial group of 1-3 positions
    if (!forced && i < N) {
        if (need == 0u || need == (uint32_t)(N - i)) {
            forced = true;
        } else {
            const uint4 w = draw((uint32_t)(i >> 2));
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int pos = i + k;
                if (pos < N) {
                    const uint32_t take = __umulhi(ws[k], (uint32_t)(N - pos)) < need;
                    word |= take << (pos & 31);
                    need -= take;
                }
            }
            emit(i >> 5, word);
            return;
        }
    }
    if (forced) {
        // forced tail from position i (a multiple of 4), a word at a time
        const bool ones = need != 0u;
        int pos = i;
        while (pos < N) {
            const int wend = min(N, (pos | 31) + 1);
            const int len = wend - pos;
            if (ones) word |= (len == 32 ? ~0u : ((1u << len) - 1u)) << (pos & 31);
            emit(pos >> 5, word);
            word = 0;
            pos = wend;
        }
    }
}

// Row-major [count][W] output (the public hb_perm_labels layout).
__global__ void k_labels_rows(const __grid_constant__ LabelKeys K, int n, int N, int64_t b0, int64_t count,
                              uint32_t *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int W = (N + 31) >> 5;
    uint32_t *row = out + k * W;
    for (int w = 0; w < W; ++w) row[w] = 0u;
    walk_labels(K, n, N, (uint64_t)(b0 + k), [&](int w, uint32_t v) { row[w] = v; });
}

// Pipeline layout: per pair, [W][B_pad] with the relabelling index fastest
// (coalesced stores here, coalesced 128-relabelling tile loads in the GEMMs).
// Grid: x over 128-relabelling tiles, y over pairs order[pair0 + y] (or pair
// pair0 + y when order is null).
__global__ void __launch_bounds__(128, 16) k_labels_pipeline(const PairMeta *__restrict__ meta,
                                                              const PairState *__restrict__ st,
                                                              const __grid_constant__ LabelKeys K,
                                                              uint32_t *__restrict__ bits, const int *__restrict__ order,
                                                              int pair0)
{
    const int p = order ? order[pair0 + blockIdx.y] : pair0 + (int)blockIdx.y;
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
    walk_labels(K, pm.n, pm.N, (uint64_t)b, [&](int w, uint32_t v) { col[(int64_t)w * pm.B_pad] = v; });
}

// Exhaustive mode: relabelling b is the b-th n-subset of {0..N-1} in colex
// order, unranked in the combinatorial number system (b = sum_k C(c_k, k)).
__global__ void k_labels_exhaustive(const PairMeta *__restrict__ meta, uint32_t *__restrict__ bits,
                                    const int *__restrict__ order, int pair0)
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
    const int p = order ? order[pair0 + blockIdx.y] : pair0 + (int)blockIdx.y;
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
    k_labels_rows<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(label_keys(seed, stream), n, N, b0, count, out);
}

void launch_labels_pipeline(const PairMeta *meta, const PairState *pst, const int *order, int p_begin, int p_end,
                            int max_Bpad, const RunOpts &o, uint32_t *bits, cudaStream_t st)
{
    for (int p0 = p_begin; p0 < p_end; p0 += 65535) {
        const dim3 g((unsigned)((max_Bpad + 127) / 128), (unsigned)min(65535, p_end - p0));
        if (o.exhaustive) k_labels_exhaustive<<<g, 128, 0, st>>>(meta, bits, order, p0);
        else k_labels_pipeline<<<g, 128, 0, st>>>(meta, pst, label_keys(o.seed, o.stream), bits, order, p0);
    }
}

}  // namespace hb
