// hb_mixed.cu -- group sums of all relabellings on the tcgen05 tensor cores
// (Sec. 3.2, Eq. gemm: "a single GEMM call"), with the statistic, the error
// band and the exceedance count fused into the epilogue (Algorithm 2).
//
// GEMM: D[b, a] = sum_i L[b, i] * Zs[i, a]
//   A = labels L (128 relabellings x 64 tokens per stage), 0/1 in BF16,
//       expanded from the packed label bits by the producer warps straight
//       into the 128-byte-swizzled K-major shared-memory layout;
//   B = slices of Z (tokens contiguous), loaded by TMA with 128-byte swizzle
//       in boxes of up to 128 slice rows (one or two per stage for BF16);
//   D = FP32 accumulators in TMEM, 128 lanes x nacc columns (nacc = slices x
//       z-columns of the tile), two buffers so the epilogue of one column tile
//       overlaps the MMAs of the next.
// Every FP32 accumulator holds an exact sum: BF16 storage uses the grid
// slices of l1_split (every partial sum is a multiple of the column's grid
// below 2^24 grid units), FP32 storage three fixed-point slices of magnitude
// <= 256 (|D| <= 256 * 65536 = 2^24).  The group sums are therefore exact up
// to the residual of the slices used, which the error band carries as a
// per-column bound.
//
// Work items (pair, tile group, mode):
//   MODE_FULL   every slice (BF16: 2, FP32: 3), relabellings of the tiles;
//               in-band relabellings go to the exact recheck;
//   MODE_SINGLE BF16 only: the first grid slice alone (half the MMAs and
//               half the B bytes); the band carries that slice's residual,
//               and in-band relabellings are listed for MODE_GATHER;
//   MODE_GATHER every slice, for the relabellings MODE_SINGLE listed (a
//               tile's rows are gathered from the pair's list).
// Each relabelling is decided once: by the single-slice pass when it falls
// outside that pass's band, else by the two-slice pass, else exactly.
//
// Warp roles (448 threads, one CTA per SM, persistent over work items):
//   warps 0-3  epilogue: TMEM -> registers, sigma_1 = sum_s k_s D_s,
//              sigma_2 = t - sigma_1, squared norms, band (its first-order
//              term by Cauchy-Schwarz from the column bounds' norm), decision
//   warp  4    TMA producer of the B tiles
//   warp  5    MMA issuer (one elected lane; with CTA pairs (CG = 2) the even
//              CTA's, whose barriers count both CTAs' operands)
//   warps 6-13 A producers (label bits -> BF16 0/1 tiles): warp 6 + i
//              expands rows 32*(i%4) .. +31, tokens 32*(i/4) .. +31 (one
//              label word) of every stage
// The kernel is capped at 96 registers a thread (launch bound; the epilogue
// reads 16 TMEM columns at a time), leaving room for the label draws, which
// run beside it on another stream.
// Variants: CG = 2 (tcgen05 cta_group::2 on CTA pairs, M = 256, each CTA
// loading half of every B tile: the default route, half the B bytes per SM of
// single CTAs) and CG = 1 (single CTAs, each loading its own B tiles; also the
// gathered pass).  No copy is multicast.  AM = 1 (CTA pairs, BF16) keeps the
// A operand in TMEM instead: the producer warps write it with tcgen05.st
// (warp w reaches TMEM lanes 32 (w % 4) .. +31) and the accumulator tiles
// shrink to 192 columns to make room for four 64-token A stages; shared
// memory then holds only B, in eight stages.
// Every mbarrier wait is bounded (wall-clock limit, a launch parameter); on
// expiry the kernel raises the timeout flag, drains its own copies and MMAs,
// frees TMEM and returns, and the host reports HB_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <string>

#include "hb_launch.cuh"

namespace hb {

constexpr int MX_M = 128;            // relabellings per tile (TMEM lanes)
constexpr int MX_K = 64;             // tokens of one 128-byte swizzle atom of BF16 (a stage holds 1 or 2)
constexpr int MX_PF = 6;             // label-word prefetch distance of the A producers (stages)
constexpr int MX_A_BYTES = MX_M * MX_K * 2;       // 16 KB: the A tile of one atom
constexpr int MX_NACC = 256;         // accumulator columns of one TMEM buffer
constexpr int MX_NACC_TA = 192;      // the same with the A operand in TMEM (CTA pairs, BF16)
constexpr int MX_BOXR_MIN = 32;      // slice rows per TMA box: at least this, at most 128
constexpr int MX_APROD = 8;          // A-producer warps (two per row block, one label word each)
constexpr int MX_THREADS = 192 + 32 * MX_APROD;
// The launch bound names more threads than a CTA has, which caps the kernel at
// 96 registers a thread (65536 / 576 rounded down): the SM then keeps about a
// third of its registers free for the label draws, which run beside the GEMM
// on another stream and finish under it instead of in the gaps between its
// launches.
constexpr int MX_BOUND_THREADS = 576;
static_assert(MX_BOUND_THREADS >= MX_THREADS, "launch bound");
constexpr int MX_TMEM_COLS = 512;    // two accumulator buffers of MX_NACC columns
constexpr int MX_STAGE_AREA = 192 * 1024;  // CG = 1: 4 stages of 48 KB; CG = 2: 6 of 32 KB
constexpr int MX_BAR_OFF = MX_STAGE_AREA;
constexpr int MX_CONST_OFF = MX_BAR_OFF + 512;
constexpr int MX_SMEM = 1024 + MX_CONST_OFF + 4 * 4 * MX_NACC * 4;  // per epilogue warp: two tiles' t and q_hi

struct MixedParams {
    const PairMeta *meta;
    RunOpts o;
    PairState *st;
    const ColConst *cc;
    const float *ct;                 // column totals t, [pair][d_pad], zero past d
    const uint32_t *bits;
    const WorkItem *items;
    int n_work;                      // items, or -1: read *n_work_dev
    const unsigned int *n_work_dev;  // device item count (the gathered pass)
    uint32_t *glist;                 // per pair (from g_off, B_pad entries): relabellings left by MODE_SINGLE
    RecheckItem *list;
    unsigned int *n_items;
    unsigned int cap;
    unsigned int *overflow;
    unsigned int *timeout;
    float *T_out;
    uint64_t wait_ns;                // wall-clock limit of every barrier wait
    int withhold;                    // test hook: CTA 0 withholds one A-stage arrival (the waits run out)
    int box_rows;                    // slice rows of one TMA box (divides every tile's z-columns)
};

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Bounded wait for the phase with the given parity.  Returns false when the
// wall-clock limit (limit_ns) expired here or another thread already raised
// the flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned int *timeout, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*(volatile unsigned int *)timeout) return false;
            if (globaltimer() - t0 > limit_ns) {
                atomicExch(timeout, 1u);
                return false;
            }
        }
    }
}

// the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// arrive on an mbarrier of another CTA without a release: for signals that
// publish no memory writes (TMEM stores the thread has waited for, ordered by
// tcgen05.fence::before_thread_sync), where a cluster-scope release would cost
// about a microsecond
__device__ __forceinline__ void mbar_arrive_remote_relaxed(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// The slice matrix as a 3-D tensor: 64 tokens (128 bytes, the innermost
// coordinate, always 0 here), rows, 64-token blocks.  A box is 64 tokens x
// box_rows rows of one block.
__device__ __forceinline__ void tma_load_rows(uint32_t dst, const CUtensorMap *map, int y, int kb, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(0), "r"(y), "r"(kb), "r"(bar)
        : "memory");
}

// CTA pairs: a tile into this CTA's shared memory whose completion is counted
// on an mbarrier of the pair's even CTA (bar: shared::cluster address)
__device__ __forceinline__ void tma_load_rows_pair(uint32_t dst, const CUtensorMap *map, int y, int kb, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(0), "r"(y), "r"(kb), "r"(bar)
        : "memory");
}

// A whole warp waits for a barrier phase: lane 0 polls (one shared-memory
// access per poll instead of 32) and the warp takes its outcome; __syncwarp
// orders the other lanes' later accesses after lane 0's acquire.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, unsigned int *timeout, uint64_t limit_ns)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, timeout, limit_ns);
    ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    __syncwarp();
    return ok;
}

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// 4- and 16-byte asynchronous copies global -> shared (cp.async), and their groups
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM management: with CG = 2 one warp of each CTA of the pair performs the
// allocation (same offset, same columns) collectively, and both CTAs receive
// the same address.
template <int CG>
__device__ __forceinline__ void tmem_alloc(uint32_t holder, uint32_t ncols)
{
    if (CG == 2)
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder), "r"(ncols)
                     : "memory");
    else
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(holder), "r"(ncols)
                     : "memory");
}
template <int CG>
__device__ __forceinline__ void tmem_relinquish()
{
    if (CG == 2) asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    else asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int CG>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    if (CG == 2)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T across the CTA pair (M = 256: each CTA's
// shared memory holds its 128 rows of A and its half of the N columns of B at
// the same offsets; each CTA's TMEM receives its 128 rows of D).  Issued by the
// even CTA of the pair only.
__device__ __forceinline__ void umma_bf16_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                               uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T across the CTA pair: as umma_bf16_pair,
// with each CTA's 128 rows of A in its own TMEM (row = lane, two BF16 values
// of consecutive k per 32-bit column, the lower k in the low half).
__device__ __forceinline__ void umma_bf16_pair_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                                  uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrives (once the pair's prior MMAs complete) on the mbarrier at offset
// `bar` in every CTA of ctaMask.
__device__ __forceinline__ void umma_commit_pair_mc(uint32_t bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     bar),
                 "h"(mask)
                 : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 16 consecutive TMEM columns of this thread's lane from 16 registers
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address, 16-byte units
    d |= (uint64_t)1u << 16;                   // leading-dimension offset (unused with 128B swizzle)
    d |= (uint64_t)(1024u >> 4) << 32;         // stride-dimension offset: 1024 bytes
    d |= (uint64_t)1u << 46;                   // descriptor version (tcgen05)
    d |= (uint64_t)2u << 61;                   // swizzle mode: 128 bytes
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ __forceinline__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}


// The even-indexed bits of w to bits 0..15 and the odd-indexed ones to bits
// 16..31, in order (four delta swaps: 2 <-> 1 within nibbles, then 2-bit,
// nibble and byte fields).
__device__ __forceinline__ uint32_t unshuffle32(uint32_t x)
{
    uint32_t t;
    t = (x ^ (x >> 1)) & 0x22222222u;
    x ^= t ^ (t << 1);
    t = (x ^ (x >> 2)) & 0x0C0C0C0Cu;
    x ^= t ^ (t << 2);
    t = (x ^ (x >> 4)) & 0x00F000F0u;
    x ^= t ^ (t << 4);
    t = (x ^ (x >> 8)) & 0x0000FF00u;
    x ^= t ^ (t << 8);
    return x;
}

// One label word (32 tokens) -> 16 words of two BF16 labels 0.0 / 1.0, the
// K positions 2j (low half) and 2j + 1 (high half) of the word's 32 slice
// positions in word j.  BF16 grid slices hold tokens j and j + 16 there (the
// slices interleave the halves of every 32-token group), i.e. bits j and
// j + 16 of w; FP32 fixed-point slices hold tokens 2j and 2j + 1, which
// unshuffle32 moves to bits j and j + 16.  Word j is then those two bits
// times 0x3F80 (BF16 1.0) in each half; as 0x3F80 = 127 * 2^7, for j < 8 the
// shift folds into the multiplier.
template <int DT>
__device__ __forceinline__ void expand_word(uint32_t w, uint32_t (&v)[16])
{
    const uint32_t x = DT == DT_BF16 ? w : unshuffle32(w), x8 = x >> 8;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        v[j] = (x & (0x00010001u << j)) * (0x3F80u >> j);
        v[j + 8] = (x8 & (0x00010001u << j)) * (0x3F80u >> j);
    }
}

// What every role of a CTA needs to know about one work item; every role
// computes it the same way and skips the same items.
struct ItemInfo {
    int p;         // pair
    int mode;      // MODE_FULL, MODE_SINGLE or MODE_GATHER
    int S, cw, C;  // slices, z-columns per tile, column tiles
    int KC;        // 64-token K chunks
    int64_t row0;  // first relabelling (tiles) or list index (gathered) of this CTA's 128 rows
    int64_t nrow;  // relabellings (tiles: B) or list length (gathered)
    bool skip;
};

template <int DT, int KS>
__device__ __forceinline__ ItemInfo item_info(const MixedParams &P, const WorkItem &w, int CL, int sub)
{
    ItemInfo I;
    I.p = w.pair;
    I.mode = w.mode;
    const PairMeta &pm = P.meta[w.pair];
    const PairState &st = P.st[w.pair];
    I.S = w.mode == MODE_SINGLE ? 1 : (DT == DT_BF16 ? 2 : 3);
    I.cw = P.o.nacc / I.S;
    I.C = (P.o.d + I.cw - 1) / I.cw;
    // stages of KS tokens; with two atoms per stage the second atom of the last
    // stage may lie past the pair's tokens: its labels are 0, so it adds nothing
    I.KC = (pm.N_pad + KS - 1) / KS;
    I.row0 = ((int64_t)w.tile * CL + sub) * MX_M;
    I.nrow = w.mode == MODE_GATHER ? (int64_t)st.n_gather : pm.B;
    // uniform over the cluster: the item's first row decides
    I.skip = st.status != ST_OK || (int64_t)w.tile * CL * MX_M >= I.nrow;
    return I;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <int CG, int DT, int AM>
__global__ void __launch_bounds__(MX_BOUND_THREADS, 1) k_mixed(const __grid_constant__ CUtensorMap tmap, const MixedParams P)
{
    static_assert(AM == 0 || (CG == 2 && DT == DT_BF16), "A in TMEM: CTA pairs on BF16 slices");
    constexpr int CL = CG;  // CTAs per work item (a cluster of two for CTA pairs)
    // stages: AT swizzle atoms of 64 tokens, each an A tile (16 KB) and this CTA's
    // B rows (up to 256 x 128 B for single CTAs, 128 x 128 B for CTA pairs).  CTA
    // pairs take two atoms per stage (eight MMAs per barrier handshake, which halves
    // the handshakes' cost) in three stages of 64 KB; single CTAs one atom in four
    // stages of 48 KB
    // With the A operand in TMEM (AM = 1: CTA pairs, 192 accumulator columns)
    // shared memory holds only the B halves, 2 x 96 rows x 128 B a stage, in
    // eight stages; the A tiles of four 64-token atoms sit in TMEM columns
    // 384..511 behind the two accumulator buffers.
    constexpr int AT = CG == 2 ? 2 : 1;
    constexpr int KS = AT * MX_K;                  // tokens per stage
    constexpr int A_BYTES = AM ? 0 : AT * MX_A_BYTES;
    constexpr int STAGE = AM ? 24 * 1024 : (CG == 2 ? 64 * 1024 : 48 * 1024);
    constexpr int NS = AM ? 8 : (CG == 2 ? 3 : 4);
    constexpr int NSA = 4;                                   // AM: A stages (one atom each) in TMEM
    constexpr uint32_t ACCS = AM ? MX_NACC_TA : MX_NACC;     // TMEM columns of one accumulator buffer
    constexpr uint32_t ACOL = 2 * ACCS;                      // AM: TMEM column of A stage 0
    static_assert(NS * STAGE <= MX_STAGE_AREA, "stage layout");
    static_assert(!AM || ACOL + NSA * (MX_K / 2) <= MX_TMEM_COLS, "TMEM columns");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + MX_BAR_OFF;
    // full(s): the stage's A tile (one arrival per producer warp) and B tile (the TMA
    // thread's expect_tx arrival and the copies' bytes) are in place; with CTA pairs
    // the even CTA's barrier counts both CTAs' producer warps and B halves (the odd
    // CTA's barrier is unused)
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (2 * NS + s); };
    auto acc_full = [&](int b) { return bar0 + 8u * (3 * NS + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (3 * NS + 2 + b); };
    const uint32_t drain = bar0 + 8u * (3 * NS + 4);
    // AM: A stage sa is in TMEM (every producer warp of both CTAs has arrived;
    // on the even CTA) / free again (the MMAs reading it completed; both CTAs)
    auto afull = [&](int sa) { return bar0 + 8u * (NS + sa); };
    auto aempty = [&](int sa) { return bar0 + 8u * (3 * NS + 5 + sa); };
    static_assert(8 * (4 * NS + 5) + 4 <= MX_CONST_OFF - MX_BAR_OFF, "barrier block");
    uint32_t *tmem_holder = (uint32_t *)(smem + MX_BAR_OFF + 8 * (4 * NS + 5));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RunOpts &o = P.o;
    const uint64_t lim = P.wait_ns;
    const int nacc = o.nacc;
    const uint32_t crank = CL > 1 ? cluster_ctarank() : 0u;
    const int cid = (int)blockIdx.x / CL, ncl = (int)gridDim.x / CL;
    const bool leader = CG == 1 || (crank & 1u) == 0u;  // issues the MMAs (CG = 2: the even CTA)
    const uint16_t pair_mask = (uint16_t)((CG == 2 ? 3u : 1u) << (crank & ~(uint32_t)(CG - 1)));
    const int n_work = P.n_work >= 0 ? P.n_work : (int)*P.n_work_dev;
    const int sub = (int)crank;  // this CTA's 128-row tile within the item's CL tiles

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full(s), AM || !leader ? 1 : CG * MX_APROD + 1);
            mbar_init(empty(s), 1);  // the MMA commit (CG = 2: the pair's commit reaches both CTAs)
            if (AM && s < NSA) {
                mbar_init(afull(s), 2 * MX_APROD);
                mbar_init(aempty(s), 1);
            }
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(acc_full(b), 1);
            mbar_init(acc_empty(b), 4 * CG);  // the epilogue warps of every CTA sharing the accumulator
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc<CG>(smem_u32(tmem_holder), MX_TMEM_COLS);
        tmem_relinquish<CG>();
    }
    // every barrier of both CTAs of a pair is initialised before any copy or commit reaches it
    tc_fence_before();
    if (CL > 1) cluster_sync();
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 4) {
        // ---------------- TMA producer: B tiles (Z slices) ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            long long issued = 0;
            bool ok = true;
            // this CTA's share of a tile's nacc rows: all (CG = 1) or one half, in boxes
            // of box_rows slice rows (a box never straddles two slices)
            const int r_begin = CG == 2 ? (int)(crank & 1u) * (nacc / 2) : 0, r_cnt = nacc / CG;
            const int br = P.box_rows, nb = r_cnt / br;
            for (int it = cid; it < n_work && ok; it += ncl) {
                const ItemInfo I = item_info<DT, KS>(P, P.items[it], CL, sub);
                if (I.skip) continue;
                const PairMeta &pm = P.meta[I.p];
                // slice row of each box in column tile 0 (tile c adds c * cw)
                int yb[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int a = r_begin + k * br;
                    yb[k] = k < nb ? (a / I.cw) * o.d_pad + a % I.cw : 0;
                }
                for (int c = 0; c < I.C && ok; ++c) {
                    for (int kc = 0; kc < I.KC; ++kc) {
                        if (!mbar_wait(empty(stage), phase ^ 1u, P.timeout, lim)) {
                            ok = false;
                            break;
                        }
                        const int x0 = (int)(pm.z_row + kc * KS);
                        const uint32_t bdst = sbase + stage * STAGE + A_BYTES;
                        if (CG == 1) {
                            mbar_arrive_expect_tx(full(stage), (uint32_t)(AT * r_cnt) * 128u);
                        } else if (leader) {
                            // each CTA of the pair loads its half into its own shared memory and
                            // the even CTA's barrier counts both halves
                            mbar_arrive_expect_tx(full(stage), (uint32_t)(AT * nacc) * 128u);
                        }
                        const uint32_t bar = CG == 1 ? full(stage) : mapa_rank(full(stage), crank & ~1u);
#pragma unroll
                        for (int a = 0; a < AT; ++a) {
                            const uint32_t adst = bdst + (uint32_t)(a * r_cnt) * 128u;  // atom a's rows
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                if (k >= nb) break;
                                // (a pair's tokens start at a multiple of 64: block x0 / 64 + a)
                                if (CG == 1) tma_load_rows(adst + (uint32_t)(k * br) * 128u, &tmap, yb[k] + c * I.cw,
                                                           (x0 >> 6) + a, bar);
                                else tma_load_rows_pair(adst + (uint32_t)(k * br) * 128u, &tmap, yb[k] + c * I.cw,
                                                        (x0 >> 6) + a, bar);
                            }
                        }
                        ++issued;
                        if (++stage == NS) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            // wait for this thread's copies still in flight (bounded); an odd CTA's
            // copies complete on the even CTA's barriers, which its MMA thread drains
            const int inflight = CG == 2 && !leader ? 0 : (int)std::min<long long>(issued, NS);
            for (int k = 1; k <= inflight; ++k) {
                int s = stage - k;
                uint32_t ph = phase;
                if (s < 0) {
                    s += NS;
                    ph ^= 1u;
                }
                unsigned int dummy = 0;
                mbar_wait(full(s), ph, ok ? P.timeout : &dummy, lim);
            }
        }
    } else if (warp == 5 && !leader) {
        // CG = 2, odd CTA: no MMA issuer (its producers and copies report to the even
        // CTA's barriers directly)
    } else if (warp == 5 && AM) {
        // ---------------- MMA issuer, A in TMEM ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(MX_M * CG, nacc);
            const uint32_t dhi = (uint32_t)(sw128_desc(sbase) >> 32);
            const uint32_t blo0 = (uint32_t)sw128_desc(sbase);
            constexpr uint32_t STEP = STAGE >> 4;
            const uint32_t BAOFF = (uint32_t)(nacc / CG) * 8u;  // one atom of this CTA's B rows, 16-byte units
            int stage = 0, sa = 0, abuf = 0;
            uint32_t phase = 0, aph = 0, aphase = 0, blo = blo0;
            bool ok = true;
            for (int it = cid; it < n_work && ok; it += ncl) {
                const ItemInfo I = item_info<DT, KS>(P, P.items[it], CL, sub);
                if (I.skip) continue;
                for (int c = 0; c < I.C && ok; ++c) {
                    if (!mbar_wait(acc_empty(abuf), aphase ^ 1u, P.timeout, lim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + (uint32_t)abuf * ACCS;
                    for (int kc = 0; kc < I.KC && ok; ++kc) {
                        if (!mbar_wait(full(stage), phase, P.timeout, lim)) {
                            ok = false;
                            break;
                        }
#pragma unroll
                        for (int a = 0; a < AT; ++a) {
                            // both CTAs' A tiles of this atom (the odd CTA's producers arrive once
                            // their TMEM stores are complete; the fence below orders the MMAs after)
                            if (!mbar_wait(afull(sa), aph, P.timeout, lim)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t at = tmem + ACOL + (uint32_t)sa * (MX_K / 2);
#pragma unroll
                            for (int kk = 0; kk < MX_K / 16; ++kk) {
                                const uint64_t bd = ((uint64_t)dhi << 32) | (blo + a * BAOFF + 2u * kk);
                                umma_bf16_pair_ta(dt, at + 8u * kk, bd, idesc, (kc | a | kk) != 0 ? 1u : 0u);
                            }
                            umma_commit_pair_mc(aempty(sa), pair_mask);  // this A stage is free in both CTAs
                            if (++sa == NSA) {
                                sa = 0;
                                aph ^= 1u;
                            }
                        }
                        if (!ok) break;
                        umma_commit_pair_mc(empty(stage), pair_mask);  // this B stage is free in both CTAs
                        blo += STEP;
                        if (++stage == NS) {
                            stage = 0;
                            phase ^= 1u;
                            blo = blo0;
                        }
                    }
                    if (!ok) break;
                    umma_commit_pair_mc(acc_full(abuf), pair_mask);  // both CTAs' epilogues
                    abuf ^= 1;
                    if (abuf == 0) aphase ^= 1u;
                }
            }
            umma_commit_pair_mc(drain, (uint16_t)(1u << crank));
            unsigned int dummy = 0;
            mbar_wait(drain, 0, ok ? P.timeout : &dummy, lim);
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(MX_M * CG, nacc);
            // shared-memory descriptors: the high word is the same for every operand,
            // the low word holds the start address (16-byte units) and the leading
            // byte offset; stage s starts at sbase + s * STAGE and K step k adds 32
            // bytes, so each MMA's descriptors are two integer adds away
            const uint32_t dhi = (uint32_t)(sw128_desc(sbase) >> 32);
            const uint32_t alo0 = (uint32_t)sw128_desc(sbase);
            constexpr uint32_t STEP = STAGE >> 4, BOFF = A_BYTES >> 4, AOFF = MX_A_BYTES >> 4;
            const uint32_t BAOFF = (uint32_t)(nacc / CG) * 8u;  // one atom of this CTA's B rows, 16-byte units
            int stage = 0, abuf = 0;
            uint32_t phase = 0, aphase = 0, alo = alo0;
            bool ok = true;
            for (int it = cid; it < n_work && ok; it += ncl) {
                const ItemInfo I = item_info<DT, KS>(P, P.items[it], CL, sub);
                if (I.skip) continue;
                for (int c = 0; c < I.C && ok; ++c) {
                    if (!mbar_wait(acc_empty(abuf), aphase ^ 1u, P.timeout, lim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + (uint32_t)abuf * MX_NACC;
                    for (int kc = 0; kc < I.KC; ++kc) {
                        if (!mbar_wait(full(stage), phase, P.timeout, lim)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int k = 0; k < KS / 16; ++k) {
                            const uint32_t a = (uint32_t)(k >> 2), kk = (uint32_t)(k & 3);
                            const uint64_t ad = ((uint64_t)dhi << 32) | (alo + a * AOFF + 2u * kk);
                            const uint64_t bd = ((uint64_t)dhi << 32) | (alo + BOFF + a * BAOFF + 2u * kk);
                            if (CG == 2) umma_bf16_pair(dt, ad, bd, idesc, (kc | k) != 0 ? 1u : 0u);
                            else umma_bf16(dt, ad, bd, idesc, (kc | k) != 0 ? 1u : 0u);
                        }
                        if (CG == 2) umma_commit_pair_mc(empty(stage), pair_mask);  // frees this slot in both CTAs
                        else umma_commit(empty(stage));
                        alo += STEP;
                        if (++stage == NS) {
                            stage = 0;
                            phase ^= 1u;
                            alo = alo0;
                        }
                    }
                    if (!ok) break;
                    if (CG == 2) umma_commit_pair_mc(acc_full(abuf), pair_mask);  // both CTAs' epilogues
                    else umma_commit(acc_full(abuf));
                    abuf ^= 1;
                    if (abuf == 0) aphase ^= 1u;
                }
            }
            // all MMAs issued by this thread have completed once `drain` flips
            if (CG == 2) umma_commit_pair_mc(drain, (uint16_t)(1u << crank));
            else umma_commit(drain);
            unsigned int dummy = 0;
            mbar_wait(drain, 0, ok ? P.timeout : &dummy, lim);
        }
    } else if (warp >= 6) {
        // ---------------- A producers: label bits -> BF16 0/1 ----------------
        const int pi = warp - 6;
        // relabelling row of the tile, 0..127 (AM: the TMEM lane quarter this warp may
        // access is warp % 4)
        const int r = AM ? (warp & 3) * 32 + lane : (pi & 3) * 32 + lane;
        const int half = pi >> 2;            // the 32-token half of each atom this warp fills
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        bool withheld = false;
        for (int it = cid; it < n_work && ok; it += ncl) {
            const ItemInfo I = item_info<DT, KS>(P, P.items[it], CL, sub);
            if (I.skip) continue;
            const PairMeta &pm = P.meta[I.p];
            // this row's relabelling: the tile's row, or the listed one (gathered pass)
            const int64_t idx = I.row0 + r;
            const bool valid = idx < I.nrow;
            const int64_t b = !valid ? 0 : I.mode == MODE_GATHER ? (int64_t)P.glist[pm.g_off + idx] : idx;
            const uint32_t *lab = P.bits + pm.lab_off + b;
            const int nW = pm.W;             // (in registers: the asm statements below clobber memory)
            const int64_t nBp = pm.B_pad;
            // this warp's label word of 64-token atom q of the pair (identical for every
            // column tile)
            const int QA = I.KC * AT;  // atoms of a column tile
            auto word = [&](int q) {
                const int w0 = 2 * q + half;
                return valid && w0 < nW ? __ldg(lab + (int64_t)w0 * nBp) : 0u;
            };
            // loads run MX_PF atoms ahead of the expansion (a register ring, wrapping
            // across column tiles), which covers the DRAM latency
            uint32_t rw[MX_PF];
            int knext = 0;  // atom of the next load
#pragma unroll
            for (int i = 0; i < MX_PF; ++i) {
                rw[i] = word(knext);
                if (++knext == QA) knext = 0;
            }
            if (AM) {
                // one atom per A stage: this warp's label word of the atom, expanded to 16
                // TMEM columns of two BF16 labels (tokens 2j, 2j + 1 of the word in column j)
                const uint32_t trow = tmem + ((uint32_t)(r & ~31) << 16) + ACOL + (uint32_t)half * 16u;
                for (int q = 0; q < I.C * QA && ok; ++q) {
                    // the MMAs that read this stage are complete (their commit flipped the
                    // barrier): the stores below cannot overtake them, so no
                    // tcgen05.fence::after_thread_sync is needed (it costs about 200
                    // clocks here)
                    if (!warp_wait(aempty(stage), phase ^ 1u, P.timeout, lim)) {
                        ok = false;
                        break;
                    }
                    uint32_t v[16];
                    expand_word<DT>(rw[0], v);
#pragma unroll
                    for (int i = 0; i + 1 < MX_PF; ++i) rw[i] = rw[i + 1];
                    rw[MX_PF - 1] = word(knext);
                    if (++knext == QA) knext = 0;
                    tmem_st16(trow + (uint32_t)stage * (MX_K / 2), v);
                    tmem_st_wait();
                    tc_fence_before();
                    __syncwarp();
                    const bool hold = P.withhold && !withheld && blockIdx.x == 0 && pi == 0;
                    withheld |= hold;
                    if (lane == 0 && !hold) {
                        if (leader) mbar_arrive(afull(stage));
                        else mbar_arrive_remote_relaxed(mapa_rank(afull(stage), crank - 1u));
                    }
                    if (++stage == NSA) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                continue;
            }
            for (int c = 0; c < I.C && ok; ++c) {
                for (int kc = 0; kc < I.KC; ++kc) {
                    // warp-uniform outcome, so the __syncwarp below is always complete
                    if (!warp_wait(empty(stage), phase ^ 1u, P.timeout, lim)) {
                        ok = false;
                        break;
                    }
#pragma unroll
                    for (int a = 0; a < AT; ++a) {
                        uint8_t *row = smem + stage * STAGE + a * MX_A_BYTES + r * 128;
                        const uint32_t wd = rw[0];
#pragma unroll
                        for (int i = 0; i + 1 < MX_PF; ++i) rw[i] = rw[i + 1];
                        rw[MX_PF - 1] = word(knext);
                        if (++knext == QA) knext = 0;
                        uint32_t v[16];
                        expand_word<DT>(wd, v);
#pragma unroll
                        for (int cl = 0; cl < 4; ++cl) {
                            const int ch = 4 * half + cl;  // 16-byte chunk of the row: 8 tokens
                            *(uint4 *)(row + ((ch ^ (r & 7)) << 4)) =
                                make_uint4(v[4 * cl], v[4 * cl + 1], v[4 * cl + 2], v[4 * cl + 3]);
                        }
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    // test hook: CTA 0's first producer warp withholds its first arrival, so
                    // the MMA thread's wait for that stage runs out
                    const bool hold = P.withhold && !withheld && blockIdx.x == 0 && pi == 0;
                    withheld |= hold;
                    // the odd CTA's warps arrive on the even CTA's barrier without a release:
                    // their stores are visible to the async proxy (the fence above), and the
                    // tensor core reading them is this SM's own
                    if (lane == 0 && !hold) {
                        if (leader) mbar_arrive(full(stage));
                        else mbar_arrive_remote_relaxed(mapa_rank(full(stage), crank - 1u));
                    }
                    if (++stage == NS) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else {
        // ---------------- epilogue (warps 0-3 = TMEM lanes 0-127) ----------------
        const int r = threadIdx.x;  // TMEM lane = relabelling row
        // this warp's column constants (totals t and, FP32 storage, slice scales
        // q_hi) of two tiles: the current one and the next, fetched by cp.async
        // while the current one is waited for and consumed
        float *const cbase = (float *)(smem + MX_CONST_OFF) + warp * 4 * MX_NACC;
        auto fetch = [&](int p, int c, int cw, int buf) {
            float *t = cbase + buf * 2 * MX_NACC;
            // totals: 16-byte copies of the contiguous array, which is zero past d (a
            // tile never reaches past d_pad); FP32 storage also the slice scales
            const float *src = P.ct + (int64_t)p * o.d_pad + c * cw;
            for (int k = lane; k < cw / 4; k += 32) cp_async16(t + 4 * k, src + 4 * k);
            if (DT == DT_F32) {
                for (int jj = lane; jj < cw; jj += 32) {
                    const int j = c * cw + jj;
                    if (j < o.d) cp_async4(t + MX_NACC + jj, &P.cc[(int64_t)p * o.d_pad + j].q_hi);
                    else t[MX_NACC + jj] = 0.f;
                }
            }
            cp_async_commit();
        };
        auto next_item = [&](int from, ItemInfo &J) {
            for (int k = from; k < n_work; k += ncl) {
                J = item_info<DT, KS>(P, P.items[k], CL, sub);
                if (!J.skip) return k;
            }
            return n_work;
        };
        int abuf = 0, cb = 0;
        uint32_t aphase = 0;
        bool ok = true;
        // rounding chain of each squared norm: 4 FMAs per interleaved accumulator,
        // 2 combining adds, up to 16 chunk adds per tile, then exact-enough FP64
        // across tiles and one final rounding to FP32
        const float chain = 29.0f;
        ItemInfo I;
        int it = next_item(cid, I);
        if (it < n_work) fetch(I.p, 0, I.cw, 0);
        for (; it < n_work && ok;) {
            ItemInfo NI;
            const int nit = next_item(it + ncl, NI);
            const int p = I.p;
            const PairMeta &pm = P.meta[p];
            const bool single = I.mode == MODE_SINGLE;
            const int nch = I.cw / 16;
            double Q1 = 0.0, Q2 = 0.0;
            for (int c = 0; c < I.C; ++c) {
                // every lane is done with the other buffer (the previous tile): fetch the
                // next tile's constants into it, then wait for this tile's (all copy
                // groups but the newest; an empty group keeps the count uniform)
                __syncwarp();
                if (c + 1 < I.C) fetch(p, c + 1, I.cw, cb ^ 1);
                else if (nit < n_work) fetch(NI.p, 0, NI.cw, cb ^ 1);
                else cp_async_commit();
                cp_async_wait1();
                __syncwarp();
                const float *tt = cbase + cb * 2 * MX_NACC, *qq = tt + MX_NACC;
                cb ^= 1;
                if (!warp_wait(acc_full(abuf), aphase, P.timeout, lim)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)abuf * ACCS;
                float pq1[4] = {0.f, 0.f, 0.f, 0.f}, pq2[4] = {0.f, 0.f, 0.f, 0.f};
                float tq1 = 0.f, tq2 = 0.f;
                // per column: sigma_1, sigma_2 = t - sigma_1 and both squares; the band's
                // first-order term comes from ||sigma_g|| ||c|| (Cauchy-Schwarz) below, so
                // no per-column band work is needed
                auto column = [&](int i, float s1, float t) {
                    const float s2 = t - s1;
                    pq1[i & 3] = fmaf(s1, s1, pq1[i & 3]);
                    pq2[i & 3] = fmaf(s2, s2, pq2[i & 3]);
                };
                auto fold = [&]() {
                    tq1 += (pq1[0] + pq1[1]) + (pq1[2] + pq1[3]);
                    tq2 += (pq2[0] + pq2[1]) + (pq2[2] + pq2[3]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) pq1[q] = pq2[q] = 0.f;
                };
                if (DT == DT_BF16 && I.S == 1) {
                    // the single-slice pass (the hot path): the slice holds values, so
                    // sigma_1 = D exactly; the next chunk's TMEM load is in flight while
                    // this one is consumed.  The same operations as `column` and `fold`,
                    // two columns per instruction: accumulator pair a holds pq[0], pq[1],
                    // pair b pq[2], pq[3]
                    f2_t p1a = 0ull, p1b = 0ull, p2a = 0ull, p2b = 0ull;
                    auto chunk = [&](const uint32_t (&dv)[16], int c0) {
#pragma unroll
                        for (int i = 0; i < 16; i += 4) {
                            const float4 t4 = *(const float4 *)(tt + c0 + i);
                            const f2_t sa = f2_pack(__uint_as_float(dv[i]), __uint_as_float(dv[i + 1]));
                            const f2_t sb = f2_pack(__uint_as_float(dv[i + 2]), __uint_as_float(dv[i + 3]));
                            const f2_t ra = f2_sub(f2_pack(t4.x, t4.y), sa), rb = f2_sub(f2_pack(t4.z, t4.w), sb);
                            p1a = f2_fma(sa, sa, p1a);
                            p1b = f2_fma(sb, sb, p1b);
                            p2a = f2_fma(ra, ra, p2a);
                            p2b = f2_fma(rb, rb, p2b);
                        }
                        float x0, x1, x2, x3;
                        f2_unpack(p1a, x0, x1);
                        f2_unpack(p1b, x2, x3);
                        tq1 += (x0 + x1) + (x2 + x3);
                        f2_unpack(p2a, x0, x1);
                        f2_unpack(p2b, x2, x3);
                        tq2 += (x0 + x1) + (x2 + x3);
                        p1a = p1b = p2a = p2b = 0ull;
                    };
                    uint32_t da[16], db[16];
                    tmem_ld16(tb, da);
                    tmem_ld_wait();
#pragma unroll 1
                    for (int ch = 0; ch < nch; ch += 2) {
                        tmem_ld16(tb + (ch + 1) * 16, db);  // nch is even
                        chunk(da, ch * 16);
                        tmem_ld_wait();
                        if (ch + 2 < nch) tmem_ld16(tb + (ch + 2) * 16, da);
                        chunk(db, (ch + 1) * 16);
                        tmem_ld_wait();
                    }
                } else {
                    // every slice: sigma_1 = D_0 + D_1 (BF16 grid slices hold values; one
                    // rounding) or q_hi (D_0 + D_1/2^9 + D_2/2^18) for the fixed-point slices
                    // of FP32 storage (exact products, one rounding per added slice)
#pragma unroll 1
                    for (int ch = 0; ch < nch; ++ch) {
                        uint32_t d0[16], d1[16], d2[16];
                        tmem_ld16(tb + ch * 16, d0);
                        tmem_ld16(tb + I.cw + ch * 16, d1);
                        if (DT == DT_F32) tmem_ld16(tb + 2 * I.cw + ch * 16, d2);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float2 k = make_float2(qq[ch * 16 + i], tt[ch * 16 + i]);
                            float s1;
                            if (DT == DT_BF16) {
                                s1 = __fadd_rn(__uint_as_float(d0[i]), __uint_as_float(d1[i]));
                            } else {
                                s1 = __fmul_rn(__uint_as_float(d0[i]), k.x);
                                s1 = __fmaf_rn(__uint_as_float(d1[i]), k.x * (1.0f / 512.0f), s1);
                                s1 = __fmaf_rn(__uint_as_float(d2[i]), k.x * (1.0f / 262144.0f), s1);
                            }
                            column(i, s1, k.y);
                        }
                        fold();
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (leader) mbar_arrive(acc_empty(abuf));
                    // the even CTA reuses it (its loads are complete: no release needed)
                    else mbar_arrive_remote_relaxed(mapa_rank(acc_empty(abuf), crank - 1u));
                }
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1u;
                Q1 += (double)tq1;
                Q2 += (double)tq2;
            }
            if (!ok) break;
            const float q1 = (float)Q1, q2 = (float)Q2;
            // decision for this row's relabelling
            const int64_t idx = I.row0 + r;
            int dec = -2;
            float T = 0.f, band = 0.f;
            if (idx < I.nrow) {
                const int64_t b = I.mode == MODE_GATHER ? (int64_t)P.glist[pm.g_off + idx] : idx;
                const PairState &s = P.st[p];
                const float sc2 = single ? s.sumc2_1 : s.sumc2;
                // sum_j |sigma_g,j| c_j <= ||sigma_g|| ||c||, with ||sigma_g||^2 <= q_g (1 + chain u)
                const float ec = 1.0f + (chain + 4.0f) * U32;
                const float e1 = __fmul_ru(__fsqrt_ru(__fmul_ru(q1, sc2)), ec);
                const float e2 = __fmul_ru(__fsqrt_ru(__fmul_ru(q2, sc2)), ec);
                const float dq1 = q_bound(e1, q1, q1, q2, s.tnorm, sc2, chain);
                const float dq2 = q_bound(e2, q2, q1, q2, s.tnorm, sc2, chain);
                dec = fast_decide(o.stat, o.alt, (float)o.d, (float)pm.n, (float)pm.m, q1, q2, dq1, dq2,
                                  (float)s.To, &T, &band);
                if (dec < 0) {
                    if (single) P.glist[pm.g_off + atomicAdd(&P.st[p].n_gather, 1u)] = (uint32_t)b;
                    else push_recheck(P.list, P.n_items, P.cap, P.overflow, p, (uint32_t)b);
                }
                if (P.T_out && pm.T_off >= 0) P.T_out[pm.T_off + b] = T;
            }
            const unsigned int ex = __ballot_sync(0xffffffffu, dec == 1);
            float bm = (dec >= -1 && band < INFINITY) ? band : 0.f;
#pragma unroll
            for (int off = 16; off; off >>= 1) bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, off));
            if (lane == 0) {
                if (ex) atomicAdd(&P.st[p].count, (unsigned long long)__popc(ex));
                atomicMax(&P.st[p].band_max_bits, __float_as_uint(bm));
            }
            it = nit;
            I = NI;
        }
        cp_async_wait0();  // no copy into this CTA's shared memory outlives the loop
    }

    // no CTA leaves while a peer may still copy into its shared memory or
    // arrive on its barriers (every role above drained its own copies and MMAs)
    tc_fence_before();
    if (CL > 1) cluster_sync();
    else __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc<CG>(tmem, MX_TMEM_COLS);
    }
}

// ---------------------------------------------------------------------------
// the gathered pass: one work item per 128 listed relabellings of a pair
// ---------------------------------------------------------------------------
// Single block: per pair of order[q0 .. q1) (order null: pairs q0 .. q1) the
// listed count n_gather, items in that order.
__global__ void k_gather_items(const PairState *__restrict__ st, const int *__restrict__ order, int q0, int q1,
                               WorkItem *__restrict__ items, unsigned int *__restrict__ n_items)
{
    __shared__ unsigned int warp_tot[32];
    __shared__ unsigned int base_s;
    if (threadIdx.x == 0) base_s = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)blockDim.x >> 5;
    for (int k0 = q0; k0 < q1; k0 += (int)blockDim.x) {
        const int k = k0 + (int)threadIdx.x;
        const int p = k < q1 ? (order ? order[k] : k) : 0;
        const unsigned int cnt = k < q1 && st[p].status == ST_OK ? (st[p].n_gather + MX_M - 1) / MX_M : 0u;
        unsigned int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            unsigned int v = lane < nw ? warp_tot[lane] : 0u, w = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned int t = __shfl_up_sync(0xffffffffu, w, off);
                if (lane >= off) w += t;
            }
            if (lane < nw) warp_tot[lane] = w - v;  // exclusive
        }
        __syncthreads();
        const unsigned int at = base_s + warp_tot[wid] + incl - cnt;
        for (unsigned int t = 0; t < cnt; ++t) items[at + t] = WorkItem{p, (int32_t)t, MODE_GATHER};
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base_s = at + cnt;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_items = base_s;
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode(std::string &err)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn) return fn;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        err = "cuTensorMapEncodeTiled is not available";
        return nullptr;
    }
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    return fn;
}

typedef void (*MixedKernel)(const CUtensorMap, const MixedParams);

// am: CTA pairs on BF16 slices with the A operand in TMEM
static MixedKernel pick_kernel(int dtype, int cg, bool am)
{
    if (dtype == DT_BF16) return cg == 2 ? (am ? k_mixed<2, DT_BF16, 1> : k_mixed<2, DT_BF16, 0>) : k_mixed<1, DT_BF16, 0>;
    return cg == 2 ? k_mixed<2, DT_F32, 0> : k_mixed<1, DT_F32, 0>;
}

cudaError_t launch_mixed(const MixedArgs &a, cudaStream_t s, std::string &err)
{
    if (a.n_work == 0) return cudaSuccess;
    const int S = a.o.slices, nacc = a.o.nacc;
    if (!((a.o.dtype == DT_BF16 && S == 2) || (a.o.dtype == DT_F32 && S == 3))) {
        err = "unsupported slice count";
        return cudaErrorInvalidValue;
    }
    const int CGv = a.o.cg == 2 ? 2 : 1;
    const bool am = a.o.am && a.o.dtype == DT_BF16 && CGv == 2;
    if (nacc > MX_NACC || nacc % (MX_BOXR_MIN * CGv) != 0 || nacc % S != 0 || (nacc / S) % MX_BOXR_MIN != 0 ||
        (am && nacc != MX_NACC_TA)) {
        err = "unsupported column tile width";
        return cudaErrorInvalidValue;
    }
    // the largest box (a multiple of 8 rows: whole 1 KB swizzle groups) that divides
    // both a slice's z-columns of a tile and this CTA's share of the tile, at most
    // 128 rows (at most 8 boxes per stage)
    int br = 128;
    while ((nacc / S) % br != 0 || (nacc / CGv) % br != 0) br -= 8;
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode(err);
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    // the slice matrix in 64-token blocks: (64 tokens, zq_rows rows, zq_ld / 64 blocks)
    const cuuint64_t gdim[3] = {(cuuint64_t)MX_K, (cuuint64_t)a.zq_rows, (cuuint64_t)(a.zq_ld / MX_K)};
    const cuuint64_t gstride[2] = {(cuuint64_t)MX_K * 2, (cuuint64_t)a.zq_rows * MX_K * 2};
    const cuuint32_t box[3] = {(cuuint32_t)MX_K, (cuuint32_t)br, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)a.zq, gdim, gstride, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")";
        return cudaErrorInvalidValue;
    }
    MixedParams prm;
    prm.meta = a.meta;
    prm.o = a.o;
    prm.st = a.st;
    prm.cc = a.cc;
    prm.ct = a.ct;
    prm.bits = a.bits;
    prm.items = a.items;
    prm.n_work = a.n_work;
    prm.n_work_dev = a.n_work_dev;
    prm.glist = a.glist;
    prm.list = a.list;
    prm.n_items = a.n_items;
    prm.cap = a.cap;
    prm.overflow = a.overflow;
    prm.timeout = a.timeout;
    prm.T_out = a.T_out;
    prm.wait_ns = a.wait_ns;
    prm.withhold = a.withhold;
    prm.box_rows = br;
    const MixedKernel kern = pick_kernel(a.o.dtype, CGv, am);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MX_SMEM);
    if (e != cudaSuccess) return e;
    const int CL = CGv;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(MX_THREADS, 1, 1);
    cfg.dynamicSmemBytes = MX_SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // persistent: as many clusters as can be resident at once
    cfg.gridDim = dim3(CL * (unsigned)std::max(1, a.sms / CL), 1, 1);
    int max_clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&max_clusters, (const void *)kern, &cfg);
    if (e != cudaSuccess || max_clusters < 1) {
        cudaGetLastError();
        max_clusters = std::max(1, a.sms / CL);
    }
    // a device item count (n_work < 0) is not known here: launch every resident cluster
    const int clusters = a.n_work > 0 ? std::max(1, std::min(a.n_work, max_clusters)) : max_clusters;
    cfg.gridDim = dim3((unsigned)(clusters * CL), 1, 1);
    e = cudaLaunchKernelEx(&cfg, kern, map, prm);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

void launch_gather_items(const PairState *st, const int *order, int p0, int p1, WorkItem *items,
                         unsigned int *n_items, cudaStream_t s)
{
    k_gather_items<<<1, 1024, 0, s>>>(st, order, p0, p1, items, n_items);
}

}  // namespace hb
