// hb_mixed.cu -- group sums of all relabellings on the tcgen05 tensor cores
// (Sec. 3.2, Eq. gemm: "a single GEMM call"), with the statistic, the error
// band and the exceedance count fused into the epilogue (Algorithm 2).
//
// GEMM: D[b, c] = sum_i L[b, i] * Zs[i, c]
//   A = labels L (128 relabellings x 64 tokens per stage), 0/1 in BF16,
//       expanded from the packed label bits by the producer warps straight
//       into the 128-byte-swizzled K-major shared-memory layout;
//   B = the fixed-point slices of Z (hi, lo[, lo2] of `cw` columns, tokens
//       contiguous), loaded by TMA with 128-byte swizzle;
//   D = FP32 accumulators in TMEM, 128 lanes x (S*cw) columns, two buffers so
//       the epilogue of one column tile overlaps the MMAs of the next.
// Every slice value is an integer of magnitude <= 256 and every label is 0
// or 1, so each FP32 accumulator holds an exact integer (|D| <= 256 * 65536 =
// 2^24): the group sums are exact up to the residual of the slices, which the
// error band carries as a per-column bound.
//
// Warp roles (448 threads, one CTA per SM, persistent over work items):
//   warps 0-3  epilogue: TMEM -> registers, sigma_1 = sum_s q_s D_s,
//              sigma_2 = t - sigma_1, squared norms, band, decision
//   warp  4    TMA producer of the B tiles
//   warp  5    MMA issuer (one elected lane); with CTA pairs (CG = 2) the odd
//              CTA's warp 5 relays its A readiness to the even CTA instead
//   warps 6-13 A producers (label bits -> BF16 0/1 tiles): warp 6 + i
//              expands rows 32*(i%4) .. +31, tokens 32*(i/4) .. +31 (one
//              label word) of every stage (with MX_APROD = 4, both words)
// The kernel is capped at 96 registers a thread (launch bound; the epilogue
// reads 16 TMEM columns at a time), leaving room for the label draws, which
// run beside it on another stream.
// CG = 2 (HB_PATH_MIXED_2SM): the CTAs of each pair of the cluster (ranks 2k,
// 2k+1) run tcgen05 cta_group::2 MMAs with M = 256; each holds its 128 rows of
// A and half of the N columns of every B tile, so each SM receives half the B
// bytes.  It is exact like the rest but not faster on GB300 at this tile
// shape: shared-memory operand reads, not B ingress, bound both variants.
// Every mbarrier wait is bounded (wall-clock limit); on expiry the kernel
// raises the timeout flag, drains its own copies and MMAs, frees TMEM and
// returns, and the host reports HB_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <string>

#include "hb_launch.cuh"

namespace hb {

constexpr int MX_M = 128;            // relabellings per tile (TMEM lanes)
constexpr int MX_K = 64;             // tokens per stage (one 128-byte swizzle atom of BF16)
constexpr int MX_NS = 4;             // pipeline stages
constexpr int MX_PF = 6;             // label-word prefetch distance of the A producers (stages)
constexpr int MX_A_BYTES = MX_M * MX_K * 2;       // 16 KB
constexpr int MX_STAGE_BYTES = 48 * 1024;         // A + up to 256 B-rows x 128 B
constexpr int MX_APROD = 8;         // A-producer warps (8: two per row block, one label word each; or 4)
static_assert(MX_APROD == 8 || MX_APROD == 4, "four or eight A producers");
constexpr int MX_THREADS = 192 + 32 * MX_APROD;
// The launch bound names more threads than a CTA has, which caps the kernel at
// 96 registers a thread (65536 / 576 rounded down): the SM then keeps about a
// third of its registers free for the label draws, which run beside the GEMM
// on another stream and finish under it instead of in the gaps between its
// launches.
constexpr int MX_BOUND_THREADS = 576;
static_assert(MX_BOUND_THREADS >= MX_THREADS, "launch bound");
constexpr int MX_TMEM_COLS = 512;    // two accumulator buffers of 256 columns
constexpr int MX_BAR_OFF = MX_NS * MX_STAGE_BYTES;
constexpr int MX_CONST_OFF = MX_BAR_OFF + 256;
constexpr int MX_SMEM = 1024 + MX_CONST_OFF + 4 * 128 * 16;  // per-epilogue-warp column constants
constexpr unsigned long long MX_WAIT_NS = 4000000000ull;  // 4 s per wait

struct MixedParams {
    const PairMeta *meta;
    RunOpts o;
    PairState *st;
    const ColConst *cc;
    const uint32_t *bits;
    const WorkItem *items;
    int n_work;
    RecheckItem *list;
    unsigned int *n_items;
    unsigned int cap;
    unsigned int *overflow;
    unsigned int *timeout;
    float *T_out;
};

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
// wall-clock limit expired here or another thread already raised the flag.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned int *timeout)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*(volatile unsigned int *)timeout) return false;
            if (globaltimer() - t0 > MX_WAIT_NS) {
                atomicExch(timeout, 1u);
                return false;
            }
        }
    }
}

// try_wait with acquire at cluster scope: for barriers a peer CTA arrives on
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0u;
}

// bounded wait as mbar_wait, with cluster-scope acquire
__device__ __forceinline__ bool mbar_wait_cluster(uint32_t bar, uint32_t parity, unsigned int *timeout)
{
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 255u) == 0u) {
            if (*(volatile unsigned int *)timeout) return false;
            if (globaltimer() - t0 > MX_WAIT_NS) {
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

// arrive, with release at cluster scope, on an mbarrier of another CTA
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// CTA pairs: a tile into this CTA's shared memory whose completion is counted
// on an mbarrier of the pair's even CTA (bar: shared::cluster address)
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// The same tile into the shared memory of every CTA in ctaMask (same offset),
// completing bytes on each destination CTA's mbarrier at offset `bar`.
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar,
                                               uint16_t mask)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster "
        "[%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar), "h"(mask)
        : "memory");
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

// Arrives (once the prior MMAs complete) on the mbarrier at offset `bar` in
// every CTA of ctaMask.
__device__ __forceinline__ void umma_commit_mc(uint32_t bar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
                     bar),
                 "h"(mask)
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
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// two labels (bits 0, 1 of b) -> two BF16 values 0.0 / 1.0 packed in 32 bits
__device__ __forceinline__ uint32_t expand2(uint32_t b)
{
    return ((b & 1u) ? 0x3F80u : 0u) | ((b & 2u) ? 0x3F800000u : 0u);
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <int S, int CW, int CG>
__global__ void __launch_bounds__(MX_BOUND_THREADS, 1) k_mixed(const __grid_constant__ CUtensorMap tmap, const MixedParams P)
{
    // CW z-columns per column tile: 128 (wide) or 64 (narrow) for two slices,
    // 64 or 32 for three.  CG = 2: CTA pairs (ranks 2k, 2k+1) run M = 256 MMAs,
    // each CTA holding NACC/2 rows of every B tile.
    constexpr int NACC = S * CW;  // accumulator columns of one buffer
    static_assert(NACC <= 256 && CW % 32 == 0 && NACC % 16 == 0, "column tile");
    static_assert(CG == 1 || (CG == 2 && NACC % 16 == 0 && MIXED_CLUSTER % 2 == 0), "CTA pairs");
    constexpr int BR = NACC / CG;                  // B rows of a stage in this CTA
    constexpr uint32_t B_BYTES = (uint32_t)BR * 128u;
    // stages: A (16 KB) + this CTA's B rows; CTA pairs hold half the B rows, so
    // the same shared memory holds six stages instead of four
    constexpr int STAGE = CG == 2 ? 32 * 1024 : MX_STAGE_BYTES;
    constexpr int NS = CG == 2 ? 6 : MX_NS;
    static_assert(NS * STAGE <= MX_BAR_OFF && MX_A_BYTES + (int)B_BYTES <= STAGE, "stage layout");
    // CG = 2: the odd CTA reports its A stages to the even one in groups of RG
    // (a cluster-scope release costs about as much as a stage's MMAs, so one per
    // group rather than per stage); the even CTA waits at the first stage of each
    // group
    constexpr int RG = CG == 2 ? 3 : 1;
    static_assert(NS % RG == 0 && NS >= 2 * RG, "relay groups");

    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = sbase + MX_BAR_OFF;
    auto full_a = [&](int s) { return bar0 + 8u * s; };
    auto full_b = [&](int s) { return bar0 + 8u * (NS + s); };
    auto empty = [&](int s) { return bar0 + 8u * (2 * NS + s); };
    auto acc_full = [&](int b) { return bar0 + 8u * (3 * NS + b); };
    auto acc_empty = [&](int b) { return bar0 + 8u * (3 * NS + 2 + b); };
    const uint32_t drain = bar0 + 8u * (3 * NS + 4);
    // CG = 2, even CTA: the odd CTA's A tiles of stages s .. s + RG - 1 are in place
    auto peer_ready = [&](int s) { return bar0 + 8u * (3 * NS + 5 + s); };
    static_assert(8 * (4 * NS + 5) + 4 <= 256, "barrier block");
    uint32_t *tmem_holder = (uint32_t *)(smem + MX_BAR_OFF + 8 * (4 * NS + 5));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const RunOpts &o = P.o;
    const int C = o.d_pad / CW;
    // cluster: CTA `crank` of cluster `cid` owns tile (group * MIXED_CLUSTER + crank)
    const uint32_t crank = cluster_ctarank();
    const int cid = (int)blockIdx.x / MIXED_CLUSTER, ncl = (int)gridDim.x / MIXED_CLUSTER;
    constexpr uint16_t CMASK = (uint16_t)((1u << MIXED_CLUSTER) - 1u);
    const bool leader = CG == 1 || (crank & 1u) == 0u;  // issues the MMAs (CG = 2: the even CTA)
    const uint16_t pair_mask = (uint16_t)((CG == 2 ? 3u : 1u) << (crank & ~(uint32_t)(CG - 1)));

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full_a(s), MX_APROD);
            mbar_init(full_b(s), 1);
            mbar_init(empty(s), CG == 2 ? 1 : MIXED_CLUSTER);  // CG = 2: the pair's commit; else one per CTA
            mbar_init(peer_ready(s), 1);
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
    // every barrier of every CTA is initialised before any multicast copy or commit
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 4) {
        // ---------------- TMA producer: B tiles (Z slices) ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            long long issued = 0;
            bool ok = true;
            for (int it = cid; it < P.n_work && ok; it += ncl) {
                const WorkItem w = P.items[it];
                if (P.st[w.pair].status != ST_OK) continue;
                const PairMeta &pm = P.meta[w.pair];
                const int KC = pm.N_pad / MX_K;
                for (int c = 0; c < C && ok; ++c) {
                    for (int kc = 0; kc < KC; ++kc) {
                        if (!mbar_wait(empty(stage), phase ^ 1u, P.timeout)) {
                            ok = false;
                            break;
                        }
                        // every CTA expects its rows of the tile; the cluster's first CTA (per
                        // half, with CTA pairs) fetches them once from L2 and multicasts them
                        // (the slot is free in every destination: `empty` counts one commit
                        // from every MMA-issuing CTA)
                        if (CG == 1) {
                            mbar_arrive_expect_tx(full_b(stage), B_BYTES);
                            if (crank == 0)
                                tma_load_2d_mc(sbase + stage * STAGE + MX_A_BYTES, &tmap, (int)(pm.z_row + kc * MX_K),
                                               c * NACC, full_b(stage), CMASK);
                        } else {
                            // each CTA of the pair loads its half into its own shared memory and
                            // the even CTA's barrier counts both halves
                            if (leader) mbar_arrive_expect_tx(full_b(stage), 2u * B_BYTES);
                            tma_load_2d_pair(sbase + stage * STAGE + MX_A_BYTES, &tmap, (int)(pm.z_row + kc * MX_K),
                                             c * NACC + (int)(crank & 1u) * BR, mapa_rank(full_b(stage), crank & ~1u));
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
                mbar_wait(full_b(s), ph, ok ? P.timeout : &dummy);
            }
        }
    } else if (warp == 5 && !leader) {
        // ---------------- CG = 2, odd CTA: tells the even CTA when its A tiles are in ----------------
        // (its B halves are counted on the even CTA's barriers by the copies themselves)
        if (lane == 0) {
            const uint32_t rank0 = crank - 1u;
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            int pending = -1;  // first stage of a group not reported yet
            for (int it = cid; it < P.n_work && ok; it += ncl) {
                const WorkItem w = P.items[it];
                if (P.st[w.pair].status != ST_OK) continue;
                const PairMeta &pm = P.meta[w.pair];
                const int KC = pm.N_pad / MX_K;
                for (int c = 0; c < C && ok; ++c) {
                    for (int kc = 0; kc < KC; ++kc) {
                        if (!mbar_wait(full_a(stage), phase, P.timeout)) {
                            ok = false;
                            break;
                        }
                        if (stage % RG == 0) pending = stage;
                        if (stage % RG == RG - 1) {
                            mbar_arrive_remote(mapa_rank(peer_ready(pending), rank0));
                            pending = -1;
                        }
                        if (++stage == NS) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
            }
            // the last group may be short: its stages are all in
            if (ok && pending >= 0) mbar_arrive_remote(mapa_rank(peer_ready(pending), rank0));
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(MX_M * CG, NACC);
            int stage = 0, abuf = 0;
            uint32_t phase = 0, aphase = 0;
            bool ok = true;
            for (int it = cid; it < P.n_work && ok; it += ncl) {
                const WorkItem w = P.items[it];
                if (P.st[w.pair].status != ST_OK) continue;
                const PairMeta &pm = P.meta[w.pair];
                const int KC = pm.N_pad / MX_K;
                for (int c = 0; c < C && ok; ++c) {
                    if (!mbar_wait(acc_empty(abuf), aphase ^ 1u, P.timeout)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem + (uint32_t)abuf * 256u;
                    for (int kc = 0; kc < KC; ++kc) {
                        if (!mbar_wait(full_a(stage), phase, P.timeout) || !mbar_wait(full_b(stage), phase, P.timeout) ||
                            (CG == 2 && stage % RG == 0 && !mbar_wait_cluster(peer_ready(stage), phase, P.timeout))) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t a0 = sbase + stage * STAGE, b0 = a0 + MX_A_BYTES;
                        if (CG == 2) {
#pragma unroll
                            for (int k = 0; k < MX_K / 16; ++k)
                                umma_bf16_pair(dt, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), idesc,
                                               (kc | k) != 0 ? 1u : 0u);
                            umma_commit_pair_mc(empty(stage), pair_mask);  // frees this slot in both CTAs
                        } else {
#pragma unroll
                            for (int k = 0; k < MX_K / 16; ++k)
                                umma_bf16(dt, sw128_desc(a0 + 32u * k), sw128_desc(b0 + 32u * k), idesc,
                                          (kc | k) != 0 ? 1u : 0u);
                            umma_commit_mc(empty(stage), CMASK);  // frees this slot in every CTA's view
                        }
                        if (++stage == NS) {
                            stage = 0;
                            phase ^= 1u;
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
            mbar_wait(drain, 0, ok ? P.timeout : &dummy);
        }
    } else if (warp >= 6) {
        // ---------------- A producers: label bits -> BF16 0/1 ----------------
        const int pi = warp - 6;
        const int r = (pi & 3) * 32 + lane;  // relabelling row of the tile, 0..127
        // with eight producers a warp fills one 32-token half of each stage, with
        // four it fills both
        constexpr int HALVES = 8 / MX_APROD;
        const int half0 = MX_APROD == 8 ? (pi >> 2) : 0;
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        for (int it = cid; it < P.n_work && ok; it += ncl) {
            const WorkItem w = P.items[it];
            if (P.st[w.pair].status != ST_OK) continue;
            const PairMeta &pm = P.meta[w.pair];
            const int KC = pm.N_pad / MX_K;
            const int tile = w.tile * MIXED_CLUSTER + (int)crank;
            const uint32_t *lab = P.bits + pm.lab_off + (int64_t)tile * MX_M + r;
            // this warp's label word of K-chunk kc and half h (identical for every column tile)
            auto word = [&](int kc, int h) {
                const int w0 = 2 * kc + half0 + h;
                return w0 < pm.W ? __ldg(lab + (int64_t)w0 * pm.B_pad) : 0u;
            };
            // loads run MX_PF stages ahead of the expansion (a register ring,
            // wrapping across column tiles), which covers the DRAM latency
            uint32_t rw[HALVES][MX_PF];
            int knext = 0;  // K-chunk of the next load
#pragma unroll
            for (int i = 0; i < MX_PF; ++i) {
#pragma unroll
                for (int h = 0; h < HALVES; ++h) rw[h][i] = word(knext, h);
                if (++knext == KC) knext = 0;
            }
            for (int c = 0; c < C && ok; ++c) {
                for (int kc = 0; kc < KC; ++kc) {
                    // warp-uniform outcome, so the __syncwarp below is always complete
                    if (!__all_sync(0xffffffffu, mbar_wait(empty(stage), phase ^ 1u, P.timeout))) {
                        ok = false;
                        break;
                    }
                    uint8_t *row = smem + stage * STAGE + r * 128;
#pragma unroll
                    for (int h = 0; h < HALVES; ++h) {
                        const uint32_t wd = rw[h][0];
#pragma unroll
                        for (int i = 0; i + 1 < MX_PF; ++i) rw[h][i] = rw[h][i + 1];
                        rw[h][MX_PF - 1] = word(knext, h);
                        const int half = half0 + h;
#pragma unroll
                        for (int cl = 0; cl < 4; ++cl) {
                            const int ch = 4 * half + cl;  // 16-byte chunk of the row: 8 tokens
                            const uint32_t b8 = (wd >> (cl * 8)) & 0xffu;
                            uint4 v;
                            v.x = expand2(b8);
                            v.y = expand2(b8 >> 2);
                            v.z = expand2(b8 >> 4);
                            v.w = expand2(b8 >> 6);
                            *(uint4 *)(row + ((ch ^ (r & 7)) << 4)) = v;
                        }
                    }
                    if (++knext == KC) knext = 0;
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(full_a(stage));
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
        float4 *consts = (float4 *)(smem + MX_CONST_OFF) + warp * 128;
        int abuf = 0;
        uint32_t aphase = 0;
        bool ok = true;
        // rounding chain of each squared norm: 8 FMAs per interleaved accumulator,
        // 2 combining adds, 4 chunk adds per tile, then exact-enough FP64 across
        // tiles and one final rounding to FP32
        const float chain = 17.0f;
        for (int it = cid; it < P.n_work && ok; it += ncl) {
            const WorkItem w = P.items[it];
            const int p = w.pair;
            if (P.st[p].status != ST_OK) continue;
            const PairMeta &pm = P.meta[p];
            double Q1 = 0.0, Q2 = 0.0, E1 = 0.0, E2 = 0.0;
            for (int c = 0; c < C; ++c) {
                float tq1 = 0.f, tq2 = 0.f, te1 = 0.f, te2 = 0.f;
                // this warp's copy of the tile's column constants (no cross-warp barrier)
                __syncwarp();
                for (int jj = lane; jj < CW; jj += 32) {
                    const ColConst k = P.cc[(int64_t)p * o.d_pad + c * CW + jj];
                    consts[jj] = make_float4(k.q_hi, k.t, k.c, 0.f);
                }
                __syncwarp();
                if (!__all_sync(0xffffffffu, mbar_wait(acc_full(abuf), aphase, P.timeout))) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)abuf * 256u;
                // 16 accumulator columns per TMEM load keep the epilogue within the
                // kernel's register budget (the label draws run beside the GEMM in
                // the registers it leaves free)
#pragma unroll 1
                for (int ch = 0; ch < CW / 16; ++ch) {
                    uint32_t dh[16], dl[16], dl2[16];
                    tmem_ld16(tb + ch * 16, dh);
                    tmem_ld16(tb + CW + ch * 16, dl);
                    if (S == 3) tmem_ld16(tb + 2 * CW + ch * 16, dl2);
                    tmem_ld_wait();
                    float pq1[4] = {0.f, 0.f, 0.f, 0.f}, pq2[4] = {0.f, 0.f, 0.f, 0.f};
                    float pe1[4] = {0.f, 0.f, 0.f, 0.f}, pe2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float4 k = consts[ch * 16 + i];
                        // sigma_1 = q_hi*D_hi + q_lo*D_lo (+ q_lo2*D_lo2): exact products, one rounding each
                        float s1 = __fmul_rn(__uint_as_float(dh[i]), k.x);
                        s1 = __fmaf_rn(__uint_as_float(dl[i]), k.x * (1.0f / 512.0f), s1);
                        if (S == 3) s1 = __fmaf_rn(__uint_as_float(dl2[i]), k.x * (1.0f / 262144.0f), s1);
                        const float s2 = k.y - s1;
                        pq1[i & 3] = fmaf(s1, s1, pq1[i & 3]);
                        pq2[i & 3] = fmaf(s2, s2, pq2[i & 3]);
                        pe1[i & 3] = fmaf(fabsf(s1), k.z, pe1[i & 3]);
                        pe2[i & 3] = fmaf(fabsf(s2), k.z, pe2[i & 3]);
                    }
                    tq1 += (pq1[0] + pq1[1]) + (pq1[2] + pq1[3]);
                    tq2 += (pq2[0] + pq2[1]) + (pq2[2] + pq2[3]);
                    te1 += (pe1[0] + pe1[1]) + (pe1[2] + pe1[3]);
                    te2 += (pe2[0] + pe2[1]) + (pe2[2] + pe2[3]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (leader) mbar_arrive(acc_empty(abuf));
                    else mbar_arrive_remote(mapa_rank(acc_empty(abuf), crank - 1u));  // the even CTA reuses it
                }
                abuf ^= 1;
                if (abuf == 0) aphase ^= 1u;
                Q1 += (double)tq1;
                Q2 += (double)tq2;
                E1 += (double)te1;
                E2 += (double)te2;
            }
            if (!ok) break;
            const float q1 = (float)Q1, q2 = (float)Q2, e1 = (float)E1, e2 = (float)E2;
            // decision for relabelling b of this tile
            const int64_t b = (int64_t)(w.tile * MIXED_CLUSTER + (int)crank) * MX_M + r;
            int dec = -2;
            float T = 0.f, band = 0.f;
            if (b < pm.B) {
                const PairState &s = P.st[p];
                const float dq1 = q_bound(e1, q1, q1, q2, s.tnorm, s.sumc2, chain);
                const float dq2 = q_bound(e2, q2, q1, q2, s.tnorm, s.sumc2, chain);
                dec = fast_decide(o.stat, o.alt, (float)o.d, (float)pm.n, (float)pm.m, q1, q2, dq1, dq2,
                                  (float)s.To, &T, &band);
                if (dec < 0) push_recheck(P.list, P.n_items, P.cap, P.overflow, p, (uint32_t)b);
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
        }
    }

    // no CTA leaves while a peer may still multicast into its shared memory or
    // arrive on its barriers (every role above drained its own copies and MMAs)
    tc_fence_before();
    cluster_sync();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc<CG>(tmem, MX_TMEM_COLS);
    }
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

cudaError_t launch_mixed(const MixedArgs &a, cudaStream_t s, std::string &err)
{
    if (a.n_work == 0) return cudaSuccess;
    const int S = a.o.slices;
    if (S != 2 && S != 3) {
        err = "unsupported slice count";
        return cudaErrorInvalidValue;
    }
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode(err);
    if (!enc) return cudaErrorNotSupported;
    const int CGv = a.o.cg == 2 ? 2 : 1;
    const int nacc = S * a.o.cw / CGv;  // B rows of one CTA's share of a tile
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)a.zq_ld, (cuuint64_t)a.zq_rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)a.zq_ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)MX_K, (cuuint32_t)nacc};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)a.zq, gdim, gstride, box, estr,
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
    prm.bits = a.bits;
    prm.items = a.items;
    prm.n_work = a.n_work;
    prm.list = a.list;
    prm.n_items = a.n_items;
    prm.cap = a.cap;
    prm.overflow = a.overflow;
    prm.timeout = a.timeout;
    prm.T_out = a.T_out;
    void (*kern)(const CUtensorMap, const MixedParams) = nullptr;
    if (CGv == 2) kern = S == 2 && a.o.cw == 128 ? k_mixed<2, 128, 2> : S == 3 && a.o.cw == 64 ? k_mixed<3, 64, 2> : nullptr;
    else if (S == 2) kern = a.o.cw == 128 ? k_mixed<2, 128, 1> : a.o.cw == 64 ? k_mixed<2, 64, 1> : nullptr;
    else kern = a.o.cw == 64 ? k_mixed<3, 64, 1> : a.o.cw == 32 ? k_mixed<3, 32, 1> : nullptr;
    if (!kern) {
        err = "unsupported column tile width";
        return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MX_SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = MIXED_CLUSTER;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(MX_THREADS, 1, 1);
    cfg.dynamicSmemBytes = MX_SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // persistent: as many clusters as can be resident at once
    cfg.gridDim = dim3(MIXED_CLUSTER * (unsigned)std::max(1, a.sms / MIXED_CLUSTER), 1, 1);
    int max_clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&max_clusters, (const void *)kern, &cfg);
    if (e != cudaSuccess || max_clusters < 1) {
        cudaGetLastError();
        max_clusters = std::max(1, a.sms / MIXED_CLUSTER);
    }
    const int clusters = std::max(1, std::min(a.n_work, max_clusters));
    cfg.gridDim = dim3((unsigned)(clusters * MIXED_CLUSTER), 1, 1);
    e = cudaLaunchKernelEx(&cfg, kern, map, prm);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace hb
