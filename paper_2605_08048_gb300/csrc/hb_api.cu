// hb_api.cu -- the C ABI (include/hbperm.h): argument checking, per-pair
// metadata, the device workspace, and the launch sequence of one test batch:
//
//   colsum -> axis -> reflect -> zstats -> tobs -> labels -> GEMM+epilogue
//          -> exact recheck -> finalize -> one device-to-host copy
//
// Everything between the metadata upload and the result download runs on the
// caller's stream with no host round trip.  Host input is copied in pieces of
// whole pairs, and colsum .. tobs run per piece as the pieces arrive.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hb_launch.cuh"
#include "hbperm.h"

using namespace hb;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static hb_status fail(hb_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(HB_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" const char *hb_last_error(void) { return g_err.c_str(); }

struct hb_ctx;
extern "C" hb_status hb_ctx_set_timing(hb_ctx *c, int32_t enable);
extern "C" hb_status hb_ctx_stage_times(hb_ctx *c, float *ms_out, int32_t *n_launches);

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
namespace {
constexpr int LABEL_CHUNKS = 4;  // label-draw chunks of a mixed-path call
// device counters of a call: [0] recheck items, [1] overflow, [2] timeout,
// [3 + c] work items of chunk c's gathered pass
constexpr int N_COUNTERS = 3 + LABEL_CHUNKS;
constexpr int ALIGN_PIECES = 8;  // pieces of the host-to-device input copy, aligned as they arrive
}

struct hb_ctx {
    int device = 0;
    int sms = 0;
    void *ws = nullptr;
    size_t ws_cap = 0;
    void *stage = nullptr;  // pinned host staging
    size_t stage_cap = 0;
    cudaEvent_t stage_done = nullptr;
    bool attrs_set = false;
    // tracing: events between the stages of the last call
    bool timing = false;
    bool last_timed = false;
    cudaEvent_t tev[7] = {};
    cudaEvent_t gev[4 * LABEL_CHUNKS] = {};  // around each chunk's GEMM launch and its gathered pass
    float last_ms[7] = {};
    int last_launches = 0;
    // Streams of a call: the caller's stream forks into `main` (highest
    // priority) and joins back at the end; the label draws, which depend on no
    // data, run on `side` (lowest priority) and fill the SMs the alignment
    // kernels leave free instead of holding them back.
    cudaStream_t main = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, enter = nullptr, leave = nullptr;
    cudaEvent_t lab_ev[LABEL_CHUNKS] = {};  // label chunk c drawn
    // host input: the copy runs on `copy`, piece by piece, beside the
    // alignment of the pieces already copied
    cudaStream_t copy = nullptr;
    cudaEvent_t cp_ev[ALIGN_PIECES] = {};  // input piece k copied
    // route table of HB_PATH_AUTO, per size bucket (hb_autotune)
    int32_t route[HB_ROUTE_BUCKETS];
    bool tuned = false;
    // relabelling statistics of hb_null_quantiles
    void *tbuf = nullptr;
    size_t tbuf_cap = 0;
    // options (hb_ctx_set_option)
    uint64_t wait_ns = 4000000000ull;  // limit of every device barrier wait
    int32_t s1_max = 65536;            // BF16: pairs with n + m <= s1_max start with the single-slice pass
    int32_t withhold = 0;              // test hook: the next tensor-core call withholds one barrier arrival
    int32_t a_tmem = 0;                // CTA pairs on BF16: the A operand in TMEM
};

extern "C" void hb_ctx_destroy(hb_ctx *c);

static bool create_events(cudaEvent_t *ev, int n)
{
    for (int k = 0; k < n; ++k)
        if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
}

static void mark(hb_ctx *c, int k, cudaStream_t s)
{
    if (c->timing) cudaEventRecord(c->tev[k], s);
}

extern "C" hb_status hb_ctx_create(hb_ctx **out, int device)
{
    if (!out) return fail(HB_ERR_INVALID_ARG, "ctx pointer is NULL");
    int count = 0;
    CK(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(HB_ERR_INVALID_ARG, "device %d out of range", device);
    CK(cudaSetDevice(device));
    hb_ctx *c = new hb_ctx();
    c->device = device;
    for (int k = 0; k < HB_ROUTE_BUCKETS; ++k) c->route[k] = k <= 10 ? HB_PATH_MIXED_2SM : HB_PATH_FP32_PLAIN;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->enter, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->leave, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->main, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
        !create_events(c->lab_ev, LABEL_CHUNKS) || !create_events(c->cp_ev, ALIGN_PIECES) ||
        cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_least) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking) != cudaSuccess) {
        hb_ctx_destroy(c);
        return fail(HB_ERR_CUDA, "stream or event creation failed");
    }
    *out = c;
    g_err.clear();
    return HB_OK;
}

extern "C" void hb_ctx_destroy(hb_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stage_done) {
        cudaEventSynchronize(c->stage_done);
        cudaEventDestroy(c->stage_done);
    }
    for (int k = 0; k < 7; ++k)
        if (c->tev[k]) cudaEventDestroy(c->tev[k]);
    for (cudaEvent_t e : c->gev)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t q : {c->main, c->side, c->copy})
        if (q) {
            cudaStreamSynchronize(q);
            cudaStreamDestroy(q);
        }
    for (cudaEvent_t e : {c->fork, c->join, c->enter, c->leave})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->lab_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->cp_ev)
        if (e) cudaEventDestroy(e);
    if (c->tbuf) cudaFree(c->tbuf);
    if (c->ws) cudaFree(c->ws);
    if (c->stage) cudaFreeHost(c->stage);
    delete c;
}

static hb_status ensure_ws(hb_ctx *c, size_t bytes)
{
    if (bytes <= c->ws_cap) return HB_OK;
    if (c->ws) {
        cudaDeviceSynchronize();
        cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_cap = 0;
    }
    const size_t want = bytes + (bytes >> 3);
    if (cudaMalloc(&c->ws, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(HB_ERR_OOM, "device workspace of %zu bytes could not be allocated", want);
    }
    c->ws_cap = want;
    return HB_OK;
}

static hb_status ensure_stage(hb_ctx *c, size_t bytes)
{
    if (c->stage_done) cudaEventSynchronize(c->stage_done);  // previous upload finished reading it
    if (bytes <= c->stage_cap) return HB_OK;
    if (c->stage) cudaFreeHost(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    const size_t want = std::max<size_t>(bytes * 2, 1 << 20);
    if (cudaMallocHost(&c->stage, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(HB_ERR_OOM, "pinned staging of %zu bytes could not be allocated", want);
    }
    c->stage_cap = want;
    return HB_OK;
}

static void set_attrs(hb_ctx *c)
{
    if (c->attrs_set) return;
    set_kernel_attributes();
    c->attrs_set = true;
}

// ---------------------------------------------------------------------------
// workspace carving
// ---------------------------------------------------------------------------
struct Carve {
    char *base;
    size_t off = 0;
    explicit Carve(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

static int64_t binom64(int64_t N, int64_t k)
{
    if (k < 0 || k > N) return 0;
    if (k > N - k) k = N - k;
    int64_t c = 1;
    for (int64_t i = 1; i <= k; ++i) c = c * (N - k + i) / i;
    return c;
}

static inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Context options a plan is built with (defaults without a context).
struct CtxOpts {
    uint64_t wait_ns = 4000000000ull;
    int32_t s1_max = 65536;
    int32_t withhold = 0;
    int32_t a_tmem = 0;
};

static CtxOpts ctx_opts(const hb_ctx *c)
{
    CtxOpts k;
    k.wait_ns = c->wait_ns;
    k.s1_max = c->s1_max;
    k.withhold = c->withhold;
    k.a_tmem = c->a_tmem;
    return k;
}

struct Plan {
    int P;
    RunOpts o;
    CtxOpts k;
    int cl = 1;       // tensor-core path: CTAs per work item (2 for CTA pairs)
    int n_single = 0; // work items of the single-slice pass
    int64_t total_gl = 0;  // entries of the relabelling lists of the gathered pass
    std::vector<PairMeta> meta;
    std::vector<RowChunk> chunks;
    std::vector<int> init_bad;
    std::vector<WorkItem> items;  // (pair, 128-relabelling tile), costliest pairs first
    int64_t total_rows_pad = 0, total_label_words = 0, total_B = 0;
    int max_Bpad = 0, max_W = 0, max_N = 0;
    // mixed path: pairs in the items' order, cut into nlc chunks of label work
    // (a smaller first one, the rest even); chunk c is pairs order[lc_pair[c] .. lc_pair[c+1]) and
    // items [lc_item[c], lc_item[c+1]), so its GEMM can start as soon as its
    // labels are drawn while the next chunk's labels are still being drawn
    std::vector<int> order;
    int nlc = 0;
    int lc_pair[LABEL_CHUNKS + 1] = {};
    int lc_item[LABEL_CHUNKS + 1] = {};
    // the gathered pass of chunk c: its work list starts at lc_gi[c] (room for every
    // listed relabelling of the chunk's pairs), and it runs if the chunk has
    // single-slice items
    int lc_gi[LABEL_CHUNKS + 1] = {};
    bool lc_single[LABEL_CHUNKS] = {};
};

// every pair's X and Y rows and the rows of Z start on 16-byte boundaries
static bool rows_16b_aligned(const Plan &pl, const void *Z)
{
    const size_t row = (size_t)pl.o.d * (pl.o.dtype == HB_F32 ? 4 : 2);
    if (row % 16 != 0 || ((uintptr_t)Z & 15u) != 0) return false;
    for (const PairMeta &pm : pl.meta)
        if ((((uintptr_t)pm.X | (uintptr_t)pm.Y) & 15u) != 0) return false;
    return true;
}

static hb_status validate_common(int64_t d, int32_t dtype)
{
    if (d < 1 || d > 8192) return fail(HB_ERR_INVALID_ARG, "d = %lld outside [1, 8192]", (long long)d);
    if (dtype != HB_F32 && dtype != HB_BF16) return fail(HB_ERR_INVALID_ARG, "dtype %d unknown", dtype);
    return HB_OK;
}

static hb_status validate_opts(const hb_opts *op)
{
    if (!op) return fail(HB_ERR_INVALID_ARG, "opts is NULL");
    if (op->stat < 0 || op->stat > 2) return fail(HB_ERR_INVALID_ARG, "stat %d unknown", op->stat);
    if (op->alt < 0 || op->alt > 2) return fail(HB_ERR_INVALID_ARG, "alt %d unknown", op->alt);
    if (op->reflect_side != 0 && op->reflect_side != 1)
        return fail(HB_ERR_INVALID_ARG, "reflect_side %d unknown", op->reflect_side);
    if (op->path < HB_PATH_MIXED || op->path > HB_PATH_MIXED_2SM)
        return fail(HB_ERR_INVALID_ARG, "path %d unknown", op->path);
    if (!op->exhaustive && (op->B < 1 || op->B > 0x7fffffffLL))
        return fail(HB_ERR_INVALID_ARG, "B = %lld outside [1, 2^31)", (long long)op->B);
    return HB_OK;
}

// Builds the per-pair metadata.  X/Y pointers filled by the caller.
// size bucket of a pair: 0 for N <= 64, k for 2^(k+5) < N <= 2^(k+6)
static int route_bucket(int64_t N)
{
    int k = 0;
    while (k < HB_ROUTE_BUCKETS - 1 && ((int64_t)64 << k) < N) ++k;
    return k;
}

static int32_t route_for(const hb_ctx *c, int64_t N)
{
    if (N > 65536) return HB_PATH_FP32_PLAIN;  // the only route for large pairs
    return c->route[route_bucket(N)];
}

// One route for a whole batch under HB_PATH_AUTO (plans and the triage calls):
// the SIMT path if any pair needs it, else the route of the bucket holding
// most of the batch's rows.
static int32_t route_for_batch(const hb_ctx *c, int64_t P, const int64_t *n, const int64_t *m)
{
    int64_t rows[5] = {0, 0, 0, 0, 0};
    for (int64_t p = 0; p < P; ++p) {
        const int32_t r = route_for(c, n[p] + m[p]);
        if (r == HB_PATH_FP32_PLAIN && n[p] + m[p] > 65536) return HB_PATH_FP32_PLAIN;
        rows[r] += n[p] + m[p];
    }
    int32_t best = HB_PATH_MIXED_2SM;
    for (int32_t r = 0; r < 5; ++r)
        if (r != HB_PATH_AUTO && rows[r] > rows[best]) best = r;
    return best;
}

static hb_status make_plan(Plan &pl, int64_t P, const int64_t *n, const int64_t *m, int64_t d, int32_t dtype,
                           const hb_opts &op, bool align_only, bool want_T, const CtxOpts &k = CtxOpts())
{
    pl.P = (int)P;
    pl.k = k;
    RunOpts &o = pl.o;
    memset(&o, 0, sizeof o);
    o.seed = op.seed;
    o.stream = op.stream;
    o.stat = op.stat;
    o.alt = op.alt;
    o.align = op.align ? 1 : 0;
    o.reflect_side = op.reflect_side;
    o.exhaustive = op.exhaustive ? 1 : 0;
    // HB_PATH_AUTO is resolved by the caller; the narrow tensor-core route is
    // the mixed path with half-width column tiles
    const bool narrow = op.path == HB_PATH_MIXED_NARROW, two_sm = op.path == HB_PATH_MIXED_2SM;
    o.path = align_only ? 1 : (narrow || two_sm ? HB_PATH_MIXED : op.path);
    o.cg = two_sm && !align_only ? 2 : 1;
    o.d = (int)d;
    o.dtype = dtype;
    o.want_T = want_T ? 1 : 0;
    if (o.path == HB_PATH_MIXED) {
        // accumulator tiles of nacc columns: BF16 two grid slices of cw columns (the
        // single-slice pass covers 2 cw columns per tile), FP32 three fixed-point slices
        o.slices = dtype == HB_F32 ? 3 : 2;
        // (CTA pairs on BF16 with the A operand in TMEM: 96, so that the two
        // 192-column accumulators leave TMEM room for it)
        o.am = o.slices == 2 && two_sm && k.a_tmem ? 1 : 0;
        o.cw = o.am ? 96 : (o.slices == 2 ? 128 : 64) >> (narrow ? 1 : 0);
        o.nacc = o.slices * o.cw;
        o.d_pad = (int)rup(d, dtype == HB_F32 ? o.cw : 2 * o.cw);
        o.s1_max = dtype == HB_F32 ? 0 : k.s1_max;
        pl.cl = o.cg == 2 ? 2 : 1;
    } else {
        o.slices = 0;
        o.cw = 128;
        o.nacc = 0;
        o.d_pad = (int)d;
    }
    pl.meta.resize(P);
    pl.init_bad.assign(P, 0);
    pl.chunks.clear();
    int64_t zrow = 0, lab = 0, tb = 0;
    for (int64_t p = 0; p < P; ++p) {
        const int64_t np = n[p], mp = m[p];
        if (np < 1 || mp < 1) return fail(HB_ERR_INVALID_ARG, "pair %lld: n = %lld, m = %lld", (long long)p,
                                          (long long)np, (long long)mp);
        const int64_t N = np + mp;
        if (N > (1 << 20)) return fail(HB_ERR_UNSUPPORTED, "pair %lld: n + m = %lld > 2^20", (long long)p, (long long)N);
        if (!align_only && o.path == HB_PATH_MIXED && N > 65536)
            return fail(HB_ERR_UNSUPPORTED, "pair %lld: the mixed path needs n + m <= 65536", (long long)p);
        if (!align_only && op.exhaustive && N > 24)
            return fail(HB_ERR_UNSUPPORTED, "pair %lld: exhaustive mode needs n + m <= 24", (long long)p);
        PairMeta &pm = pl.meta[p];
        memset(&pm, 0, sizeof pm);
        pm.n = (int)np;
        pm.m = (int)mp;
        pm.N = (int)N;
        pm.N_pad = (int)rup(N, 64);
        pm.z_row = zrow;
        zrow += pm.N_pad;
        pm.W = (int)((N + 31) / 32);
        if (!align_only) {
            pm.B = op.exhaustive ? binom64(N, np) : op.B;
            // the tensor-core path works on groups of cl tiles of 128 relabellings
            pm.B_pad = (int)rup(pm.B, o.path == HB_PATH_MIXED ? 128 * pl.cl : 128);
            pm.lab_off = lab;
            lab += (int64_t)pm.W * pm.B_pad;
            pm.g_off = pl.total_gl;
            pl.total_gl += pm.B_pad;
            pm.T_off = want_T ? tb : -1;
            tb += pm.B;
            if (np < 2 || mp < 2) pl.init_bad[p] = 2;
        }
        pm.chunk0 = (int)pl.chunks.size();
        for (int64_t r = 0; r < np; r += CHUNK_ROWS)
            pl.chunks.push_back(RowChunk{(int)p, 0, (int)r, (int)std::min<int64_t>(CHUNK_ROWS, np - r)});
        pm.nchunk_x = (int)pl.chunks.size() - pm.chunk0;
        // the first Y chunk ends where token n + rows is a multiple of 32: every
        // chunk then starts at a token index t with (t mod 32) + rows <= 128
        for (int64_t r = 0; r < mp;) {
            const int64_t rows = std::min<int64_t>(r == 0 ? CHUNK_ROWS - (np & 31) : CHUNK_ROWS, mp - r);
            pl.chunks.push_back(RowChunk{(int)p, 1, (int)r, (int)rows});
            r += rows;
        }
        pm.nchunk_y = (int)pl.chunks.size() - pm.chunk0 - pm.nchunk_x;
        pl.max_Bpad = std::max(pl.max_Bpad, pm.B_pad);
        pl.max_W = std::max(pl.max_W, pm.W);
        pl.max_N = std::max(pl.max_N, pm.N);
    }
    pl.total_rows_pad = zrow;
    pl.total_label_words = lab;
    pl.total_B = tb;
    pl.items.clear();
    pl.n_single = 0;
    if (!align_only && o.path == HB_PATH_MIXED) {
        std::vector<int> order(P);
        for (int64_t p = 0; p < P; ++p) order[p] = (int)p;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return pl.meta[a].N_pad > pl.meta[b].N_pad; });
        // BF16 pairs up to s1_max tokens start with the single-slice pass (the two-slice
        // pass then runs on the relabellings it leaves in its band); larger ones, whose
        // single-slice band is wide, and FP32 input take every slice at once
        for (int p : order)
            if (pl.init_bad[p] == 0) {
                const int mode = pl.meta[p].N <= o.s1_max ? MODE_SINGLE : MODE_FULL;
                for (int g = 0; g < pl.meta[p].B_pad / (128 * pl.cl); ++g) pl.items.push_back(WorkItem{p, g, mode});
                if (mode == MODE_SINGLE) pl.n_single += pl.meta[p].B_pad / (128 * pl.cl);
            }
        // label chunks in the same order
        pl.order = order;
        int64_t total = 0;
        for (int p : order) total += (int64_t)pl.meta[p].W * pl.meta[p].B_pad;
        int cuts[LABEL_CHUNKS + 1];
        cuts[0] = 0;
        int64_t acc = 0;
        int i = 0;
        for (int c = 1; c < LABEL_CHUNKS; ++c) {
            // the first chunk is smaller (16 % of the label work), so that it is drawn
            // by the time the alignment stages end; the rest is split evenly and drawn
            // beside the GEMM of the chunks before it
            const int64_t first = total * 16 / 100;
            const int64_t target = first + (total - first) * (c - 1) / (LABEL_CHUNKS - 1);
            while (i < (int)P && acc < target) {
                acc += (int64_t)pl.meta[order[i]].W * pl.meta[order[i]].B_pad;
                ++i;
            }
            cuts[c] = i;
        }
        cuts[LABEL_CHUNKS] = (int)P;
        pl.nlc = 0;
        pl.lc_pair[0] = 0;
        for (int c = 1; c <= LABEL_CHUNKS; ++c)
            if (cuts[c] > pl.lc_pair[pl.nlc]) pl.lc_pair[++pl.nlc] = cuts[c];
        // item boundaries: items follow `order`, so count the items of each chunk's pairs
        int it = 0, gi = 0;
        pl.lc_item[0] = 0;
        pl.lc_gi[0] = 0;
        for (int c = 0; c < pl.nlc; ++c) {
            pl.lc_single[c] = false;
            for (int k = pl.lc_pair[c]; k < pl.lc_pair[c + 1]; ++k) {
                const int p = order[k];
                if (pl.init_bad[p] == 0) {
                    it += pl.meta[p].B_pad / (128 * pl.cl);
                    if (pl.meta[p].N <= o.s1_max) pl.lc_single[c] = true;
                }
                gi += pl.meta[p].B_pad / 128 + 1;
            }
            pl.lc_item[c + 1] = it;
            pl.lc_gi[c + 1] = gi;
        }
    }
    return HB_OK;
}

// Device buffers of one run.
struct Bufs {
    PairMeta *meta;
    RowChunk *chunks;
    int *bad;
    PairState *st;
    i128 *part;
    i128 *s;
    double *u;
    void *Z;
    unsigned int *colmax;
    unsigned long long *colL1;  // tensor-core path, BF16: column L1 bounds (units of 2^-40)
    float *cpart, *cpart1;
    i128 *t_ex, *s1o;
    ColConst *cc;
    float *ct;
    unsigned short *zq;
    uint32_t *bits;
    RecheckItem *list;
    unsigned int *counters;  // [0] recheck items, [1] overflow, [2] timeout
    double *scratch;
    PairOut *out;
    void *xy;
    WorkItem *items;
    uint32_t *glist;   // BF16 tensor-core path: relabellings left by the single-slice pass
    WorkItem *gitems;  // and the gathered pass's work list
    int *order;  // mixed path: pairs in the items' order
    float *lam;  // Ritz values [P][16] (features mode)
};

static size_t carve(Carve &cv, Bufs &b, const Plan &pl, bool align_only, bool own_Z, size_t xy_bytes,
                    unsigned int cap, int rgrid)
{
    const int P = pl.P;
    const int d = pl.o.d;
    const size_t nch = pl.chunks.size();
    const size_t esz = pl.o.dtype == HB_F32 ? 4 : 2;
    b.meta = cv.take<PairMeta>(P);
    b.chunks = cv.take<RowChunk>(nch);
    b.bad = cv.take<int>(P);
    b.st = cv.take<PairState>(P);
    b.part = cv.take<i128>(nch * d);
    b.s = cv.take<i128>((size_t)P * 2 * d);
    b.u = cv.take<double>((size_t)P * d);
    b.Z = own_Z ? (void *)cv.take<char>((size_t)pl.total_rows_pad * d * esz) : nullptr;
    b.colmax = cv.take<unsigned int>((size_t)P * pl.o.d_pad);
    b.xy = xy_bytes ? (void *)cv.take<char>(xy_bytes) : nullptr;
    const bool grid_slices = !align_only && pl.o.path == HB_PATH_MIXED && pl.o.dtype == HB_BF16;
    b.colL1 = grid_slices ? cv.take<unsigned long long>((size_t)P * pl.o.d_pad) : nullptr;
    b.glist = grid_slices && pl.n_single ? cv.take<uint32_t>((size_t)pl.total_gl) : nullptr;
    b.gitems = grid_slices && pl.n_single ? cv.take<WorkItem>((size_t)(pl.total_gl / 128 + P)) : nullptr;
    if (!align_only) {
        b.cpart = cv.take<float>(nch * d);
        b.cpart1 = cv.take<float>(nch * d);
        b.t_ex = cv.take<i128>((size_t)P * d);
        b.s1o = cv.take<i128>((size_t)P * d);
        b.cc = cv.take<ColConst>((size_t)P * pl.o.d_pad);
        b.ct = cv.take<float>((size_t)P * pl.o.d_pad);
        b.zq = pl.o.path == HB_PATH_MIXED
                   ? cv.take<unsigned short>((size_t)pl.o.slices * pl.o.d_pad * pl.total_rows_pad)
                   : nullptr;
        b.bits = cv.take<uint32_t>(pl.total_label_words);
        b.list = cv.take<RecheckItem>(cap);
        b.counters = cv.take<unsigned int>(N_COUNTERS);
        b.scratch = cv.take<double>((size_t)rgrid * 2 * d);
        b.out = cv.take<PairOut>(P);
        b.items = pl.o.path == HB_PATH_MIXED ? cv.take<WorkItem>(pl.items.size()) : nullptr;
        b.order = pl.o.path == HB_PATH_MIXED ? cv.take<int>(pl.order.size()) : nullptr;
        b.lam = cv.take<float>((size_t)P * 16);
    }
    return cv.off;
}


// The whole launch sequence.  Xp/Yp: device pointers per pair.
// Optional outputs of the triage entry points.
struct TriageOut {
    float *feat = nullptr;   // features mode: steps 1-4 only, then [P][19] features
    double *tobs = nullptr;  // features mode: T_obs per pair
    float *quant = nullptr;  // null-quantile mode: [P][9] quantiles of |T_b| (x100), T_out required
};

// Handles a call's device stages are enqueued with.
struct Exec {
    cudaStream_t s, side;    // main stream; the label draws run on `side`
    cudaEvent_t fork, join;  // side-stream fork/join
    cudaEvent_t *tev;        // 7 stage events, or nullptr
    int sms;
    bool capture = false;    // enqueued under stream capture (events become graph nodes)
    cudaEvent_t *lab_ev = nullptr;  // LABEL_CHUNKS events: label chunk c drawn (mixed path)
    cudaEvent_t *gev = nullptr;     // 2 * LABEL_CHUNKS timing events around the GEMM launches, or nullptr
    cudaStream_t copy = nullptr;    // host input: stream of the piecewise input copy (else one copy on s)
    cudaEvent_t *cp_ev = nullptr;   // ALIGN_PIECES events: input piece k copied
};

static void xrec(const Exec &ex, cudaEvent_t e)
{
    cudaEventRecordWithFlags(e, ex.s, ex.capture ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Sum of the GEMM launch durations of the last call (the stage above also
// holds the waits for later label chunks).
static float gemm_ms(const Plan &pl, const cudaEvent_t *gev)
{
    float total = 0.f;
    const int nl = std::max(pl.nlc, 1);
    for (int k = 0; k < 2 * nl; ++k) {
        // launch k / 2 of chunk k / 2: its single-slice (or full) GEMM, then its gathered pass,
        // which runs only after a single-slice pass
        if ((k & 1) && !(pl.nlc ? pl.lc_single[k / 2] : pl.n_single > 0)) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, gev[2 * k], gev[2 * k + 1]) == cudaSuccess) total += ms;
        else cudaGetLastError();  // not recorded: leave no sticky error for the next call
    }
    return total;
}

// Cuts the pairs into at most `pieces` ranges of whole pairs with about equal
// input rows (every range holds at least one pair); returns the number of
// ranges.
static int piece_spans(const Plan &pl, int pieces, PairSpan *sp)
{
    const int P = pl.P, nch = (int)pl.chunks.size();
    int64_t total = 0;
    for (int p = 0; p < P; ++p) total += pl.meta[p].N;
    int n = 0, p = 0;
    int64_t acc = 0;
    for (int k = 0; k < pieces && p < P; ++k) {
        const int64_t target = total * (k + 1) / pieces;
        const int p0 = p;
        do {
            acc += pl.meta[p].N;
            ++p;
        } while (p < P && acc < target);
        sp[n++] = PairSpan{p0, p, pl.meta[p0].chunk0, p < P ? pl.meta[p].chunk0 : nch};
    }
    return n;
}

// Kernel launches of one test call: colsum (2) + axis + reflect + zstats (2) +
// tobs (per input piece when the input comes from the host) + label draws +
// GEMM + recheck (2 per batch) + finalize.
static int launch_count(const Plan &pl, unsigned int cap, int rgrid, bool host_input)
{
    PairSpan sp[ALIGN_PIECES];
    const int pieces = host_input ? piece_spans(pl, ALIGN_PIECES, sp) : 1;
    const bool mixed = pl.o.path == HB_PATH_MIXED;
    const int pchunks = (pl.P + 65534) / 65535;
    int labels = pchunks, gemm = pchunks;
    if (mixed) {
        labels = 0;
        for (int c = 0; c < pl.nlc; ++c) labels += (pl.lc_pair[c + 1] - pl.lc_pair[c] + 65534) / 65535;
        gemm = 0;
        for (int c = 0; c < pl.nlc; ++c) gemm += pl.lc_item[c + 1] > pl.lc_item[c] ? 1 : 0;
    }
    if (mixed && pl.n_single) {
        // each chunk's gathered pass: its work list and its GEMM
        if (pl.nlc == 0) gemm += 2;
        for (int c = 0; c < pl.nlc; ++c) gemm += pl.lc_single[c] ? 2 : 0;
    }
    return 7 * pieces + 1 + labels + gemm + 2 * (int)((cap + rgrid - 1) / rgrid);
}

static void xmark(const Exec &ex, int k)
{
    if (ex.tev) cudaEventRecordWithFlags(ex.tev[k], ex.s, ex.capture ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Every device stage of a permutation test after the metadata upload: label
// draws (side stream), steps 1-5 of the path, finalize and the copy of the
// counters (host_out + 0) and per-pair results (host_out + 64) to pinned host
// memory.  Nothing here synchronises the host, so a stream capture of this
// function is a CUDA graph of the whole call.
static hb_status enqueue_test(const Exec &ex, const Plan &pl, const Bufs &b, void *Z, const void *xy_host,
                              size_t xy_bytes, float *T_out, const TriageOut *tri, unsigned int cap, int rgrid,
                              void *host_out)
{
    const bool features = tri && tri->feat;
    const cudaStream_t s = ex.s;
    const int P = pl.P;
    const RunOpts &o = pl.o;
    const int d = o.d;
    const bool mixed = o.path == HB_PATH_MIXED;
    const bool chunked = mixed && !features && pl.nlc > 0;
    CK(cudaEventRecord(ex.fork, s));
    if (!features) {
        // labels on the side stream from here on, concurrently with steps 1-4 and,
        // chunk by chunk, with the GEMM of the chunks drawn before
        CK(cudaStreamWaitEvent(ex.side, ex.fork, 0));
        if (chunked) {
            for (int c = 0; c < pl.nlc; ++c) {
                launch_labels_pipeline(b.meta, b.st, b.order, pl.lc_pair[c], pl.lc_pair[c + 1], pl.max_Bpad, o, b.bits,
                                       ex.side);
                CK(cudaEventRecord(ex.lab_ev[c], ex.side));
            }
        } else {
            launch_labels_pipeline(b.meta, b.st, nullptr, 0, P, pl.max_Bpad, o, b.bits, ex.side);
        }
        CK(cudaEventRecord(ex.join, ex.side));
    }
    CK(cudaMemsetAsync(b.colmax, 0, sizeof(unsigned int) * P * o.d_pad, s));
    if (b.colL1) CK(cudaMemsetAsync(b.colL1, 0, sizeof(unsigned long long) * P * o.d_pad, s));
    CK(cudaMemsetAsync(b.counters, 0, N_COUNTERS * sizeof(unsigned int), s));
    if (mixed && o.d_pad != d)
        CK(cudaMemsetAsync(b.zq, 0, sizeof(unsigned short) * (size_t)o.slices * o.d_pad * pl.total_rows_pad, s));

    // Host input is copied in pieces of whole pairs on the copy stream, and
    // steps 1-4 of the pairs of piece k run as soon as its bytes are in, beside
    // the copy of the pieces after it.  Every step before the GEMM works pair
    // by pair, so the pieces give the same results as one pass over all pairs.
    PairSpan spans[ALIGN_PIECES];
    int pieces = 1;
    spans[0] = PairSpan{0, P, 0, (int)pl.chunks.size()};
    if (xy_host && ex.copy) {
        pieces = piece_spans(pl, ALIGN_PIECES, spans);
        CK(cudaStreamWaitEvent(ex.copy, ex.fork, 0));
        for (int k = 0; k < pieces; ++k) {
            const size_t lo = (size_t)((const char *)pl.meta[spans[k].p0].X - (const char *)b.xy);
            const size_t hi = spans[k].p1 < P ? (size_t)((const char *)pl.meta[spans[k].p1].X - (const char *)b.xy)
                                              : xy_bytes;
            CK(cudaMemcpyAsync((char *)b.xy + lo, (const char *)xy_host + lo, hi - lo, cudaMemcpyHostToDevice,
                               ex.copy));
            CK(cudaEventRecord(ex.cp_ev[k], ex.copy));
        }
    } else if (xy_host) {
        CK(cudaMemcpyAsync(b.xy, xy_host, xy_bytes, cudaMemcpyHostToDevice, s));
    }
    // lanes-along-tokens slices: tensor-core path, BF16 grid slices, 16-byte rows
    const bool tok_layout = mixed && o.dtype == HB_BF16 && d % 8 == 0;
    const int64_t zq_ld = pl.total_rows_pad;
    xmark(ex, 0);
    for (int k = 0; k < pieces; ++k) {
        const PairSpan &sp = spans[k];
        if (pieces > 1) CK(cudaStreamWaitEvent(s, ex.cp_ev[k], 0));
        // steps 1-3 (column maxima feed the slice scales and the exact-sum windows)
        launch_colsum(b.meta, b.chunks, sp, d, o.dtype, b.part, b.s, b.bad, s);
        launch_axis(b.meta, sp, o, b.s, b.bad, b.st, b.u, s);
        launch_reflect(b.meta, b.chunks, sp, o, b.st, b.u, Z, b.colmax, features ? nullptr : b.colL1,
                       rows_16b_aligned(pl, Z), s);
        CK(cudaGetLastError());
        // step 4: Z statistics, fixed-point slices, T_obs
        if (pieces == 1) xmark(ex, 1);
        launch_zstats(b.meta, b.chunks, sp, o, b.st, Z, b.colmax, b.colL1, b.part, b.cpart, b.cpart1, b.zq,
                      b.t_ex, b.s1o, b.cc, b.ct, tok_layout, s);
        launch_tobs(b.meta, sp, o, b.t_ex, b.s1o, b.cc, b.st, s);
        CK(cudaGetLastError());
    }
    if (pieces > 1) xmark(ex, 1);  // piecewise: the "align" stage holds steps 1-4 and the copy

    if (features) {
        xmark(ex, 2);
        xmark(ex, 3);
        launch_features(b.meta, P, o, b.st, Z, b.lam, tri->feat, tri->tobs, s);
        xmark(ex, 4);
    } else {
        // step 5: labels, group sums + statistic + band, exact recheck
        xmark(ex, 2);
        CK(cudaStreamWaitEvent(s, chunked ? ex.lab_ev[0] : ex.join, 0));  // the "labels" stage: the part not hidden
        xmark(ex, 3);
        CK(cudaGetLastError());
        if (mixed) {
            MixedArgs ma{};
            ma.meta = b.meta;
            ma.P = P;
            ma.o = o;
            ma.st = b.st;
            ma.cc = b.cc;
            ma.ct = b.ct;
            ma.bits = b.bits;
            ma.zq = b.zq;
            ma.zq_ld = zq_ld;
            ma.zq_rows = (int64_t)o.slices * o.d_pad;
            ma.n_work_dev = nullptr;
            ma.glist = b.glist;
            ma.list = b.list;
            ma.n_items = b.counters;
            ma.cap = cap;
            ma.overflow = b.counters + 1;
            ma.timeout = b.counters + 2;
            ma.T_out = T_out;
            ma.wait_ns = pl.k.wait_ns;
            ma.withhold = pl.k.withhold;
            ma.sms = ex.sms;
            const int nl = std::max(pl.nlc, 1);
            for (int c = 0; c < nl; ++c) {
                if (c > 0) CK(cudaStreamWaitEvent(s, ex.lab_ev[c], 0));
                ma.items = b.items + (pl.nlc ? pl.lc_item[c] : 0);
                ma.n_work = pl.nlc ? pl.lc_item[c + 1] - pl.lc_item[c] : (int)pl.items.size();
                std::string err;
                if (ex.gev) xrec(ex, ex.gev[4 * c]);
                cudaError_t e = launch_mixed(ma, s, err);
                if (ex.gev) xrec(ex, ex.gev[4 * c + 1]);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return fail(e == cudaErrorNotSupported ? HB_ERR_UNSUPPORTED : HB_ERR_CUDA,
                                "mixed path launch failed: %s (%s)", cudaGetErrorString(e), err.c_str());
                }
                if (!(pl.nlc ? pl.lc_single[c] : pl.n_single > 0)) continue;
                // the chunk's gathered pass: every slice for the relabellings its single-slice
                // pass left inside its band, in single CTAs (128 listed relabellings per
                // item); it runs while the next chunk's labels are still being drawn
                const int q0 = pl.nlc ? pl.lc_pair[c] : 0, q1 = pl.nlc ? pl.lc_pair[c + 1] : P;
                WorkItem *gi = b.gitems + (pl.nlc ? pl.lc_gi[c] : 0);
                launch_gather_items(b.st, pl.nlc ? b.order : nullptr, q0, q1, gi, b.counters + 3 + c, s);
                MixedArgs mg = ma;
                mg.o.cg = 1;
                mg.withhold = 0;
                mg.items = gi;
                mg.n_work = -1;
                mg.n_work_dev = b.counters + 3 + c;
                if (ex.gev) xrec(ex, ex.gev[4 * c + 2]);
                e = launch_mixed(mg, s, err);
                if (ex.gev) xrec(ex, ex.gev[4 * c + 3]);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return fail(e == cudaErrorNotSupported ? HB_ERR_UNSUPPORTED : HB_ERR_CUDA,
                                "mixed path launch failed: %s (%s)", cudaGetErrorString(e), err.c_str());
                }
            }
            CK(cudaStreamWaitEvent(s, ex.join, 0));  // every side-stream launch joined
        } else {
            if (ex.gev) xrec(ex, ex.gev[0]);
            launch_plain(b.meta, P, pl.max_Bpad, o, b.st, Z, b.cc, b.bits, b.list, b.counters, cap, b.counters + 1,
                         T_out, s);
            if (ex.gev) xrec(ex, ex.gev[1]);
        }
        CK(cudaGetLastError());
        xmark(ex, 4);
        launch_recheck(cap, (unsigned int)rgrid, pl.max_W, b.meta, o, b.st, Z, b.t_ex, b.colmax, b.bits, b.list,
                       b.counters, b.scratch, T_out, s);
    }
    xmark(ex, 5);
    launch_finalize(b.meta, P, o, b.st, b.out, s);
    if (tri && tri->quant) {
        int64_t maxB = 1;
        for (int p = 0; p < P; ++p) maxB = std::max<int64_t>(maxB, pl.meta[p].B);
        launch_null_quantiles(b.meta, P, (int)maxB, T_out, b.st, 100.0f, tri->quant, s);
    }
    CK(cudaGetLastError());

    // one copy back: results and the counters
    char *h = (char *)host_out;
    CK(cudaMemcpyAsync(h, b.counters, 4 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h + 64, b.out, sizeof(PairOut) * P, cudaMemcpyDeviceToHost, s));
    xmark(ex, 6);
    return HB_OK;
}

static hb_status run_on(hb_ctx *c, Plan &pl, const void *xy_host, size_t xy_bytes, const int64_t *xy_row_off,
                        bool align_only, void *Z_out, double *u_out, int32_t *skipped_out, float *T_out,
                        cudaStream_t s, std::vector<PairOut> &out, const TriageOut *tri)
{
    set_attrs(c);
    const int P = pl.P;
    const RunOpts o = pl.o;
    const int d = o.d;
    const size_t esz = o.dtype == HB_F32 ? 4 : 2;
    const bool mixed = !align_only && o.path == HB_PATH_MIXED;
    unsigned int cap = (unsigned int)std::min<int64_t>(
        (int64_t)1 << 30, (mixed ? pl.total_B / 256 : pl.total_B / 16) + 4096);

    for (int attempt = 0; attempt < 3; ++attempt) {
        // recheck batch: items whose exact sums share the scratch at once (<= 256 MB of FP64)
        const int rgrid = (int)std::max<int64_t>(
            1, std::min<int64_t>(cap, (int64_t)(256u << 20) / (int64_t)(2 * sizeof(double) * pl.o.d)));
        Bufs b{};
        Carve plan_cv(nullptr);
        const size_t need = carve(plan_cv, b, pl, align_only, Z_out == nullptr, xy_bytes, cap, rgrid);
        hb_status hs = ensure_ws(c, need);
        if (hs != HB_OK) return hs;
        Carve cv(c->ws);
        carve(cv, b, pl, align_only, Z_out == nullptr, xy_bytes, cap, rgrid);
        void *Z = Z_out ? Z_out : b.Z;

        // pair pointers into the device copy of host input (copied below, after
        // the label draws are forked: they need only the metadata)
        if (xy_host) {
            for (int p = 0; p < P; ++p) {
                pl.meta[p].X = (const char *)b.xy + (size_t)xy_row_off[p] * d * esz;
                pl.meta[p].Y = (const char *)pl.meta[p].X + (size_t)pl.meta[p].n * d * esz;
            }
        }
        // metadata upload through pinned staging
        const size_t mbytes = sizeof(PairMeta) * P, cbytes = sizeof(RowChunk) * pl.chunks.size(),
                     bbytes = sizeof(int) * P, ibytes = mixed ? sizeof(WorkItem) * pl.items.size() : 0,
                     obytes = mixed ? sizeof(int) * pl.order.size() : 0;
        hs = ensure_stage(c, std::max(mbytes + cbytes + bbytes + ibytes + obytes, sizeof(PairOut) * P) + 64);
        if (hs != HB_OK) return hs;
        char *hs_ = (char *)c->stage;
        memcpy(hs_, pl.meta.data(), mbytes);
        memcpy(hs_ + mbytes, pl.chunks.data(), cbytes);
        memcpy(hs_ + mbytes + cbytes, pl.init_bad.data(), bbytes);
        CK(cudaMemcpyAsync(b.meta, hs_, mbytes, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(b.chunks, hs_ + mbytes, cbytes, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(b.bad, hs_ + mbytes + cbytes, bbytes, cudaMemcpyHostToDevice, s));
        if (ibytes) {
            memcpy(hs_ + mbytes + cbytes + bbytes, pl.items.data(), ibytes);
            CK(cudaMemcpyAsync(b.items, hs_ + mbytes + cbytes + bbytes, ibytes, cudaMemcpyHostToDevice, s));
        }
        if (obytes) {
            memcpy(hs_ + mbytes + cbytes + bbytes + ibytes, pl.order.data(), obytes);
            CK(cudaMemcpyAsync(b.order, hs_ + mbytes + cbytes + bbytes + ibytes, obytes, cudaMemcpyHostToDevice, s));
        }
        CK(cudaEventRecord(c->stage_done, s));
        if (align_only) {
            if (xy_host) CK(cudaMemcpyAsync(b.xy, xy_host, xy_bytes, cudaMemcpyHostToDevice, s));
            const PairSpan all{0, P, 0, (int)pl.chunks.size()};
            mark(c, 0, s);
            launch_colsum(b.meta, b.chunks, all, d, o.dtype, b.part, b.s, b.bad, s);
            launch_axis(b.meta, all, o, b.s, b.bad, b.st, b.u, s);
            launch_reflect(b.meta, b.chunks, all, o, b.st, b.u, Z, nullptr, nullptr, rows_16b_aligned(pl, Z), s);
            CK(cudaGetLastError());
            if (u_out) CK(cudaMemcpyAsync(u_out, b.u, sizeof(double) * d, cudaMemcpyDeviceToDevice, s));
            if (skipped_out) {
                PairState hst;
                CK(cudaMemcpyAsync(&hst, b.st, sizeof hst, cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                if (hst.status != ST_OK)
                    return fail((hb_status)hst.status, "alignment failed (status %d)", hst.status);
                *skipped_out = hst.skipped;
            }
            return HB_OK;
        }
        // results come back through the same pinned staging (after the metadata copies)
        Exec ex{s, c->side, c->fork, c->join, c->timing ? c->tev : nullptr, c->sms};
        ex.lab_ev = c->lab_ev;
        ex.gev = c->timing && !tri ? c->gev : nullptr;
        ex.copy = c->copy;
        ex.cp_ev = c->cp_ev;
        hs = enqueue_test(ex, pl, b, Z, xy_host, xy_bytes, T_out, tri, cap, rgrid, c->stage);
        if (hs != HB_OK) {
            // a failed enqueue may leave the label draws or the input copy running
            // on their own streams: let them end before the caller reuses the input
            // buffer or the context reuses the workspace
            cudaStreamSynchronize(c->side);
            cudaStreamSynchronize(c->copy);
            cudaGetLastError();
            return hs;
        }
        char *h = (char *)c->stage;
        CK(cudaStreamSynchronize(s));
        const unsigned int *cnt = (const unsigned int *)h;
        if (cnt[2]) return fail(HB_ERR_TIMEOUT, "a bounded device wait expired in the mixed path");
        if (cnt[1]) {
            cap = (unsigned int)std::min<int64_t>((int64_t)1 << 30, pl.total_B + 64);
            continue;  // recheck list overflowed: rerun with room for every relabelling
        }
        out.assign((PairOut *)(h + 64), (PairOut *)(h + 64) + P);
        c->last_timed = c->timing;
        if (c->timing) {
            for (int k = 0; k < 6; ++k) cudaEventElapsedTime(&c->last_ms[k], c->tev[k], c->tev[k + 1]);
            c->last_ms[6] = tri ? 0.f : gemm_ms(pl, c->gev);
        }
        c->last_launches = launch_count(pl, cap, rgrid, xy_host != nullptr);
        return HB_OK;
    }
    return fail(HB_ERR_CUDA, "recheck list kept overflowing");
}

// One call: fork the caller's stream into the context's main stream, run,
// join back (also on failure), so that work the caller queues afterwards sees
// every output.
static hb_status run(hb_ctx *c, Plan &pl, const void *xy_host, size_t xy_bytes, const int64_t *xy_row_off,
                     bool align_only, void *Z_out, double *u_out, int32_t *skipped_out, float *T_out,
                     cudaStream_t user, std::vector<PairOut> &out, const TriageOut *tri = nullptr)
{
    CK(cudaEventRecord(c->enter, user));
    CK(cudaStreamWaitEvent(c->main, c->enter, 0));
    const hb_status hs = run_on(c, pl, xy_host, xy_bytes, xy_row_off, align_only, Z_out, u_out, skipped_out, T_out,
                                c->main, out, tri);
    if (!align_only && pl.o.path == HB_PATH_MIXED) c->withhold = 0;  // the test hook acts on one call
    CK(cudaEventRecord(c->leave, c->main));
    CK(cudaStreamWaitEvent(user, c->leave, 0));
    return hs;
}

static void fill_result(const PairOut &r, hb_result *o)
{
    o->p = r.p;
    o->count = r.count;
    o->B_eff = r.B_eff;
    o->T_obs = r.T_obs;
    o->r_x = r.r_x;
    o->r_y = r.r_y;
    o->reflection_skipped = r.skipped;
    o->status = r.status;
    o->n_rechecked = r.rechecked;
    o->band_max = r.band_max;
}

// ---------------------------------------------------------------------------
// entry points
// ---------------------------------------------------------------------------
extern "C" hb_status hb_perm_labels(uint64_t seed, uint32_t stream_id, int64_t n, int64_t N, int64_t b0,
                                    int64_t count, uint32_t *bits_out, void *stream)
{
    if (N < 1 || N > (1 << 20) || n < 0 || n > N || b0 < 0 || count < 0 || b0 + count > ((int64_t)1 << 40))
        return fail(HB_ERR_INVALID_ARG, "bad label request n=%lld N=%lld b0=%lld count=%lld", (long long)n,
                    (long long)N, (long long)b0, (long long)count);
    if (count == 0) return HB_OK;
    if (!bits_out) return fail(HB_ERR_INVALID_ARG, "bits_out is NULL");
    launch_labels_rows(seed, stream_id, (int)n, (int)N, b0, count, bits_out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return HB_OK;
}

extern "C" hb_status hb_align(hb_ctx *c, const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int32_t dtype,
                              int32_t align, int32_t reflect_side, void *Z_out, double *u_out, int32_t *skipped,
                              void *stream)
{
    if (!c) return fail(HB_ERR_INVALID_ARG, "ctx is NULL");
    if (!X || !Y || !Z_out) return fail(HB_ERR_INVALID_ARG, "X, Y and Z_out must be non-NULL");
    hb_status hs = validate_common(d, dtype);
    if (hs != HB_OK) return hs;
    if (reflect_side != 0 && reflect_side != 1) return fail(HB_ERR_INVALID_ARG, "reflect_side %d", reflect_side);
    CK(cudaSetDevice(c->device));
    hb_opts op{};
    op.align = align;
    op.reflect_side = reflect_side;
    op.path = HB_PATH_FP32_PLAIN;
    op.B = 1;
    Plan pl;
    hs = make_plan(pl, 1, &n, &m, d, dtype, op, true, false);
    if (hs != HB_OK) return hs;
    pl.meta[0].X = X;
    pl.meta[0].Y = Y;
    std::vector<PairOut> out;
    return run(c, pl, nullptr, 0, nullptr, true, Z_out, u_out, skipped, nullptr, (cudaStream_t)stream, out);
}

extern "C" hb_status hb_perm_test(hb_ctx *c, const void *X, int64_t n, const void *Y, int64_t m, int64_t d,
                                  int32_t dtype, const hb_opts *opts, hb_result *res, float *T_out, void *stream)
{
    if (!c) return fail(HB_ERR_INVALID_ARG, "ctx is NULL");
    if (!X || !Y || !res) return fail(HB_ERR_INVALID_ARG, "X, Y and out must be non-NULL");
    hb_status hs = validate_common(d, dtype);
    if (hs != HB_OK) return hs;
    hs = validate_opts(opts);
    if (hs != HB_OK) return hs;
    memset(res, 0, sizeof *res);
    if (n < 2 || m < 2) {
        res->status = HB_ERR_DEGENERATE;
        return fail(HB_ERR_DEGENERATE, "n = %lld and m = %lld must both be >= 2", (long long)n, (long long)m);
    }
    CK(cudaSetDevice(c->device));
    hb_opts op = *opts;
    if (op.path == HB_PATH_AUTO) op.path = route_for(c, n + m);
    Plan pl;
    hs = make_plan(pl, 1, &n, &m, d, dtype, op, false, T_out != nullptr, ctx_opts(c));
    if (hs != HB_OK) return hs;
    pl.meta[0].X = X;
    pl.meta[0].Y = Y;
    std::vector<PairOut> out;
    hs = run(c, pl, nullptr, 0, nullptr, false, nullptr, nullptr, nullptr, T_out, (cudaStream_t)stream, out);
    if (hs != HB_OK) return hs;
    fill_result(out[0], res);
    if (out[0].status != HB_OK) return fail((hb_status)out[0].status, "test failed with status %d", out[0].status);
    g_err.clear();
    return HB_OK;
}

// HB_PATH_AUTO over pairs that take different routes: one run per route on
// the pairs of that route (XY staged on the device once if it is host memory).
static hb_status batched_routes(hb_ctx *c, int64_t P, const void *XY, const int64_t *n, const int64_t *m, int64_t d,
                                int32_t dtype, hb_opts op, const std::vector<int64_t> (&sel)[5], hb_result *res,
                                cudaStream_t s)
{
    const size_t esz = dtype == HB_F32 ? 4 : 2;
    std::vector<int64_t> off(P + 1, 0);
    for (int64_t p = 0; p < P; ++p) off[p + 1] = off[p] + n[p] + m[p];
    const size_t xy_bytes = (size_t)off[P] * d * esz;
    cudaPointerAttributes attr{};
    const cudaError_t ae = cudaPointerGetAttributes(&attr, XY);
    if (ae != cudaSuccess) cudaGetLastError();
    const bool on_device = ae == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    void *tmp = nullptr;
    const char *base = (const char *)XY;
    if (!on_device) {
        if (cudaMalloc(&tmp, xy_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(HB_ERR_OOM, "device copy of the input (%zu bytes)", xy_bytes);
        }
        if (cudaMemcpyAsync(tmp, XY, xy_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaFree(tmp);
            return fail(HB_ERR_CUDA, "copy of the input failed");
        }
        base = (const char *)tmp;
    }
    hb_status hs = HB_OK, first = HB_OK;
    for (int r = 0; r < 5 && hs == HB_OK; ++r) {
        const std::vector<int64_t> &ix = sel[r];
        if (ix.empty()) continue;
        const int64_t S = (int64_t)ix.size();
        std::vector<int64_t> ns(S), ms(S);
        for (int64_t i = 0; i < S; ++i) {
            ns[i] = n[ix[i]];
            ms[i] = m[ix[i]];
        }
        op.path = r;
        Plan pl;
        hs = make_plan(pl, S, ns.data(), ms.data(), d, dtype, op, false, false, ctx_opts(c));
        if (hs != HB_OK) break;
        for (int64_t i = 0; i < S; ++i) {
            pl.meta[i].X = base + (size_t)off[ix[i]] * d * esz;
            pl.meta[i].Y = (const char *)pl.meta[i].X + (size_t)ns[i] * d * esz;
        }
        std::vector<PairOut> out;
        hs = run(c, pl, nullptr, 0, nullptr, false, nullptr, nullptr, nullptr, nullptr, s, out);
        if (hs != HB_OK) break;
        for (int64_t i = 0; i < S; ++i) {
            fill_result(out[i], &res[ix[i]]);
            if (out[i].status != HB_OK && first == HB_OK) first = (hb_status)out[i].status;
        }
    }
    if (tmp) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
    }
    if (hs != HB_OK) return hs;
    if (first != HB_OK) return fail(first, "at least one pair failed (first status %d)", first);
    g_err.clear();
    return HB_OK;
}

extern "C" hb_status hb_perm_test_batched(hb_ctx *c, int64_t P, const void *XY, const int64_t *n, const int64_t *m,
                                          int64_t d, int32_t dtype, const hb_opts *opts, hb_result *res, void *stream)
{
    if (!c) return fail(HB_ERR_INVALID_ARG, "ctx is NULL");
    if (P < 1 || P > (1 << 24)) return fail(HB_ERR_INVALID_ARG, "P = %lld", (long long)P);
    if (!XY || !n || !m || !res) return fail(HB_ERR_INVALID_ARG, "XY, n, m and out must be non-NULL");
    hb_status hs = validate_common(d, dtype);
    if (hs != HB_OK) return hs;
    hs = validate_opts(opts);
    if (hs != HB_OK) return hs;
    CK(cudaSetDevice(c->device));
    hb_opts op = *opts;
    if (op.path == HB_PATH_AUTO) {
        std::vector<int64_t> sel[5];
        for (int64_t p = 0; p < P; ++p) sel[route_for(c, n[p] + m[p])].push_back(p);
        int used = 0, only = HB_PATH_MIXED;
        for (int r = 0; r < 5; ++r)
            if (!sel[r].empty()) {
                ++used;
                only = r;
            }
        if (used > 1) return batched_routes(c, P, XY, n, m, d, dtype, op, sel, res, (cudaStream_t)stream);
        op.path = only;
    }
    Plan pl;
    hs = make_plan(pl, P, n, m, d, dtype, op, false, false, ctx_opts(c));
    if (hs != HB_OK) return hs;
    const size_t esz = dtype == HB_F32 ? 4 : 2;
    std::vector<int64_t> off(P + 1, 0);
    for (int64_t p = 0; p < P; ++p) off[p + 1] = off[p] + n[p] + m[p];
    cudaPointerAttributes attr{};
    const cudaError_t ae = cudaPointerGetAttributes(&attr, XY);
    if (ae != cudaSuccess) cudaGetLastError();
    const bool on_device = ae == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    const size_t xy_bytes = (size_t)off[P] * d * esz;
    for (int64_t p = 0; p < P; ++p) {
        pl.meta[p].X = (const char *)XY + (size_t)off[p] * d * esz;
        pl.meta[p].Y = (const char *)pl.meta[p].X + (size_t)n[p] * d * esz;
    }
    std::vector<PairOut> out;
    hs = run(c, pl, on_device ? nullptr : XY, on_device ? 0 : xy_bytes, off.data(), false, nullptr, nullptr, nullptr,
             nullptr, (cudaStream_t)stream, out);
    if (hs != HB_OK) return hs;
    hb_status first = HB_OK;
    for (int64_t p = 0; p < P; ++p) {
        fill_result(out[p], &res[p]);
        if (out[p].status != HB_OK && first == HB_OK) first = (hb_status)out[p].status;
    }
    if (first != HB_OK) return fail(first, "at least one pair failed (first status %d)", first);
    g_err.clear();
    return HB_OK;
}

// ---------------------------------------------------------------------------
// planned batches: the device stages of one batch shape as a CUDA graph
// ---------------------------------------------------------------------------
struct hb_plan {
    hb_ctx *c = nullptr;
    Plan pl;
    hb_opts opts{};
    std::vector<int64_t> n, m, off;
    int64_t d = 0;
    int32_t dtype = 0;
    size_t esz = 2, xy_bytes = 0, res_bytes = 0, mbytes = 0;
    unsigned int cap = 0;
    int rgrid = 1;
    Bufs b{};
    void *ws = nullptr;
    void *xy_dev = nullptr;       // device copy of host input
    char *host = nullptr;         // pinned: [counters + results][pair metadata]
    const void *bound = nullptr;  // input the uploaded pair pointers refer to
    cudaStream_t cs = nullptr, side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaEvent_t lab_ev[LABEL_CHUNKS] = {};
    cudaEvent_t tev[7] = {};
    cudaEvent_t gev[4 * LABEL_CHUNKS] = {};
    bool timed = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;
};

extern "C" void hb_plan_destroy(hb_plan *q)
{
    if (!q) return;
    if (q->c) cudaSetDevice(q->c->device);
    for (cudaStream_t st : {q->cs, q->side})
        if (st) cudaStreamSynchronize(st);
    if (q->exec) cudaGraphExecDestroy(q->exec);
    if (q->graph) cudaGraphDestroy(q->graph);
    for (cudaStream_t st : {q->cs, q->side})
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : {q->fork, q->join})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : q->lab_ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : q->tev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : q->gev)
        if (e) cudaEventDestroy(e);
    if (q->ws) cudaFree(q->ws);
    if (q->xy_dev) cudaFree(q->xy_dev);
    if (q->host) cudaFreeHost(q->host);
    delete q;
}

extern "C" hb_status hb_plan_layout(int64_t P, const int64_t *n, const int64_t *m, int64_t d, int32_t dtype,
                                    const hb_opts *opts, hb_layout_counts *counts, int32_t *chunks, int32_t *pieces,
                                    int32_t *label_chunks, int32_t *items, int32_t *order)
{
    if (P < 1 || P > (1 << 24)) return fail(HB_ERR_INVALID_ARG, "P = %lld", (long long)P);
    if (!n || !m || !counts) return fail(HB_ERR_INVALID_ARG, "n, m and counts must be non-NULL");
    hb_status hs = validate_common(d, dtype);
    if (hs != HB_OK) return hs;
    hs = validate_opts(opts);
    if (hs != HB_OK) return hs;
    if (opts->path == HB_PATH_AUTO) return fail(HB_ERR_INVALID_ARG, "HB_PATH_AUTO needs a context's route table");
    Plan pl;
    hs = make_plan(pl, P, n, m, d, dtype, *opts, false, false);
    if (hs != HB_OK) return hs;
    PairSpan sp[ALIGN_PIECES];
    const int np = piece_spans(pl, ALIGN_PIECES, sp);
    counts->n_chunks = (int32_t)pl.chunks.size();
    counts->n_pieces = np;
    counts->n_label_chunks = pl.nlc;
    counts->n_items = pl.o.path == HB_PATH_MIXED ? (int32_t)pl.items.size() : 0;
    if (chunks)
        for (size_t k = 0; k < pl.chunks.size(); ++k) {
            const RowChunk &c = pl.chunks[k];
            int32_t *r = chunks + 4 * k;
            r[0] = c.pair;
            r[1] = c.side;
            r[2] = c.row0;
            r[3] = c.nrows;
        }
    if (pieces)
        for (int k = 0; k < np; ++k) {
            int32_t *r = pieces + 4 * k;
            r[0] = sp[k].p0;
            r[1] = sp[k].p1;
            r[2] = sp[k].c0;
            r[3] = sp[k].c1;
        }
    if (label_chunks)
        for (int k = 0; k <= pl.nlc; ++k) {
            label_chunks[2 * k] = pl.lc_pair[k];
            label_chunks[2 * k + 1] = pl.lc_item[k];
        }
    if (items && counts->n_items)
        for (size_t k = 0; k < pl.items.size(); ++k) {
            items[3 * k] = pl.items[k].pair;
            items[3 * k + 1] = pl.items[k].tile;
            items[3 * k + 2] = pl.items[k].mode;
        }
    // the pair order exists on every tensor-core path, also when no pair has work items
    if (order && pl.o.path == HB_PATH_MIXED)
        for (size_t k = 0; k < pl.order.size(); ++k) order[k] = pl.order[k];
    g_err.clear();
    return HB_OK;
}

static hb_status plan_build(hb_plan *q, int64_t P)
{
    hb_ctx *c = q->c;
    Plan &pl = q->pl;
    CtxOpts k = ctx_opts(c);
    k.withhold = 0;  // a graph replays every call: the one-call test hook does not apply
    hb_status hs = make_plan(pl, P, q->n.data(), q->m.data(), q->d, q->dtype, q->opts, false, false, k);
    if (hs != HB_OK) return hs;
    const bool mixed = pl.o.path == HB_PATH_MIXED;
    q->esz = q->dtype == HB_F32 ? 4 : 2;
    q->off.assign(P + 1, 0);
    for (int64_t p = 0; p < P; ++p) q->off[p + 1] = q->off[p] + q->n[p] + q->m[p];
    q->xy_bytes = (size_t)q->off[P] * q->d * q->esz;
    q->cap = (unsigned int)std::min<int64_t>((int64_t)1 << 30, (mixed ? pl.total_B / 256 : pl.total_B / 16) + 4096);
    q->rgrid = (int)std::max<int64_t>(
        1, std::min<int64_t>(q->cap, (int64_t)(256u << 20) / (int64_t)(2 * sizeof(double) * pl.o.d)));

    // own workspace and pinned staging
    Carve probe(nullptr);
    const size_t need = carve(probe, q->b, pl, false, true, 0, q->cap, q->rgrid);
    if (cudaMalloc(&q->ws, need) != cudaSuccess) {
        cudaGetLastError();
        q->ws = nullptr;
        return fail(HB_ERR_OOM, "plan workspace of %zu bytes", need);
    }
    Carve cv(q->ws);
    carve(cv, q->b, pl, false, true, 0, q->cap, q->rgrid);
    q->mbytes = sizeof(PairMeta) * P;
    const size_t cbytes = sizeof(RowChunk) * pl.chunks.size(), bbytes = sizeof(int) * P,
                 ibytes = mixed ? sizeof(WorkItem) * pl.items.size() : 0,
                 obytes = mixed ? sizeof(int) * pl.order.size() : 0;
    q->res_bytes = (64 + sizeof(PairOut) * P + 255) & ~(size_t)255;
    const size_t host_bytes = q->res_bytes + std::max(q->mbytes, cbytes + bbytes + ibytes + obytes) + 64;
    if (cudaMallocHost((void **)&q->host, host_bytes) != cudaSuccess) {
        cudaGetLastError();
        q->host = nullptr;
        return fail(HB_ERR_OOM, "plan staging of %zu bytes", host_bytes);
    }

    int prio_least = 0, prio_greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    CK(cudaStreamCreateWithPriority(&q->cs, cudaStreamNonBlocking, prio_greatest));
    CK(cudaStreamCreateWithPriority(&q->side, cudaStreamNonBlocking, prio_least));
    CK(cudaEventCreateWithFlags(&q->fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&q->join, cudaEventDisableTiming));
    if (!create_events(q->lab_ev, LABEL_CHUNKS)) return fail(HB_ERR_CUDA, "event creation failed");
    q->timed = c->timing;
    if (q->timed) {
        for (cudaEvent_t &e : q->tev) CK(cudaEventCreate(&e));
        for (cudaEvent_t &e : q->gev) CK(cudaEventCreate(&e));
    }

    // the metadata that does not depend on the input address, once
    char *h = q->host + q->res_bytes;
    memcpy(h, pl.chunks.data(), cbytes);
    memcpy(h + cbytes, pl.init_bad.data(), bbytes);
    if (ibytes) memcpy(h + cbytes + bbytes, pl.items.data(), ibytes);
    if (obytes) memcpy(h + cbytes + bbytes + ibytes, pl.order.data(), obytes);
    CK(cudaMemcpyAsync(q->b.chunks, h, cbytes, cudaMemcpyHostToDevice, q->cs));
    CK(cudaMemcpyAsync(q->b.bad, h + cbytes, bbytes, cudaMemcpyHostToDevice, q->cs));
    if (ibytes) CK(cudaMemcpyAsync(q->b.items, h + cbytes + bbytes, ibytes, cudaMemcpyHostToDevice, q->cs));
    if (obytes) CK(cudaMemcpyAsync(q->b.order, h + cbytes + bbytes + ibytes, obytes, cudaMemcpyHostToDevice, q->cs));
    CK(cudaStreamSynchronize(q->cs));

    // capture every device stage of the call
    CK(cudaStreamBeginCapture(q->cs, cudaStreamCaptureModeRelaxed));
    Exec ex{q->cs, q->side, q->fork, q->join, q->timed ? q->tev : nullptr, c->sms};
    ex.capture = true;
    ex.lab_ev = q->lab_ev;
    ex.gev = q->timed ? q->gev : nullptr;
    hs = enqueue_test(ex, pl, q->b, q->b.Z, nullptr, 0, nullptr, nullptr, q->cap, q->rgrid, q->host);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(q->cs, &g);
    if (hs != HB_OK) {
        if (g) cudaGraphDestroy(g);
        return hs;
    }
    if (ce != cudaSuccess || !g) return fail(HB_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    q->graph = g;
    CK(cudaGraphInstantiateWithFlags(&q->exec, g, cudaGraphInstantiateFlagUseNodePriority));
    q->launches = launch_count(pl, q->cap, q->rgrid, false);
    return HB_OK;
}

extern "C" hb_status hb_plan_create(hb_ctx *c, int64_t P, const int64_t *n, const int64_t *m, int64_t d,
                                    int32_t dtype, const hb_opts *opts, hb_plan **out)
{
    if (!c || !out) return fail(HB_ERR_INVALID_ARG, "ctx and plan must be non-NULL");
    *out = nullptr;
    if (P < 1 || P > (1 << 24)) return fail(HB_ERR_INVALID_ARG, "P = %lld", (long long)P);
    if (!n || !m || !opts) return fail(HB_ERR_INVALID_ARG, "n, m and opts must be non-NULL");
    hb_status hs = validate_common(d, dtype);
    if (hs != HB_OK) return hs;
    hs = validate_opts(opts);
    if (hs != HB_OK) return hs;
    CK(cudaSetDevice(c->device));
    set_attrs(c);
    hb_plan *q = new hb_plan();
    q->c = c;
    q->opts = *opts;
    q->d = d;
    q->dtype = dtype;
    q->n.assign(n, n + P);
    q->m.assign(m, m + P);
    if (q->opts.path == HB_PATH_AUTO) q->opts.path = route_for_batch(c, P, n, m);
    hs = plan_build(q, P);
    if (hs != HB_OK) {
        const std::string msg = g_err;
        hb_plan_destroy(q);
        g_err = msg;
        return hs;
    }
    *out = q;
    g_err.clear();
    return HB_OK;
}

extern "C" hb_status hb_plan_execute(hb_plan *q, const void *XY, hb_result *res, void *stream)
{
    if (!q || !XY || !res) return fail(HB_ERR_INVALID_ARG, "plan, XY and out must be non-NULL");
    hb_ctx *c = q->c;
    CK(cudaSetDevice(c->device));
    const cudaStream_t user = (cudaStream_t)stream;
    const int64_t P = q->pl.P;
    cudaPointerAttributes attr{};
    const cudaError_t ae = cudaPointerGetAttributes(&attr, XY);
    if (ae != cudaSuccess) cudaGetLastError();
    const bool on_device = ae == cudaSuccess && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    const void *src = XY;
    if (!on_device) {
        if (!q->xy_dev && cudaMalloc(&q->xy_dev, q->xy_bytes) != cudaSuccess) {
            cudaGetLastError();
            q->xy_dev = nullptr;
            return fail(HB_ERR_OOM, "plan input buffer of %zu bytes", q->xy_bytes);
        }
        CK(cudaMemcpyAsync(q->xy_dev, XY, q->xy_bytes, cudaMemcpyHostToDevice, user));
        src = q->xy_dev;
    }
    if (src != q->bound) {
        for (int64_t p = 0; p < P; ++p) {
            q->pl.meta[p].X = (const char *)src + (size_t)q->off[p] * q->d * q->esz;
            q->pl.meta[p].Y = (const char *)q->pl.meta[p].X + (size_t)q->n[p] * q->d * q->esz;
        }
        char *h = q->host + q->res_bytes;
        memcpy(h, q->pl.meta.data(), q->mbytes);
        CK(cudaMemcpyAsync(q->b.meta, h, q->mbytes, cudaMemcpyHostToDevice, user));
        q->bound = src;
    }
    CK(cudaGraphLaunch(q->exec, user));
    CK(cudaStreamSynchronize(user));
    const unsigned int *cnt = (const unsigned int *)q->host;
    if (cnt[2]) return fail(HB_ERR_TIMEOUT, "a bounded device wait expired in the mixed path");
    if (cnt[1])  // recheck list outgrew the planned capacity: the unplanned path sizes it anew
        return hb_perm_test_batched(c, P, XY, q->n.data(), q->m.data(), q->d, q->dtype, &q->opts, res, stream);
    const PairOut *outp = (const PairOut *)(q->host + 64);
    hb_status first = HB_OK;
    for (int64_t p = 0; p < P; ++p) {
        fill_result(outp[p], &res[p]);
        if (outp[p].status != HB_OK && first == HB_OK) first = (hb_status)outp[p].status;
    }
    c->last_timed = q->timed;
    if (q->timed)
        for (int k = 0; k < 6; ++k) cudaEventElapsedTime(&c->last_ms[k], q->tev[k], q->tev[k + 1]);
    if (q->timed) c->last_ms[6] = gemm_ms(q->pl, q->gev);
    c->last_launches = q->launches;
    if (first != HB_OK) return fail(first, "at least one pair failed (first status %d)", first);
    g_err.clear();
    return HB_OK;
}

// ---------------------------------------------------------------------------
// route tuning
// ---------------------------------------------------------------------------
// Synthetic unit-norm rows for timing the routes: entry j of row r is a
// Philox uniform in [-1/2, 1/2) (counter (j, r, 0x7D5E, 0), key (seed, 0)),
// plus 0.3 on coordinate 0 (a common mean direction); the row is normalised
// in FP32 and stored as dtype (BF16 round-to-nearest-even).
__global__ void k_tune_rows(void *out, int64_t rows, int d, int dtype, uint32_t seed)
{
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= rows) return;
    auto val = [&](int j) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)r, 0x7D5Eu, 0u), seed, 0u);
        return (float)(w.x >> 8) * (1.0f / 16777216.0f) - 0.5f + (j == 0 ? 0.3f : 0.0f);
    };
    float ss = 0.f;
    for (int j = 0; j < d; ++j) {
        const float v = val(j);
        ss = fmaf(v, v, ss);
    }
    const float inv = 1.0f / sqrtf(ss);
    for (int j = 0; j < d; ++j) {
        const float v = val(j) * inv;
        if (dtype == HB_F32) {
            reinterpret_cast<float *>(out)[r * d + j] = v;
        } else {
            uint32_t u = __float_as_uint(v);
            u += 0x7FFFu + ((u >> 16) & 1u);
            reinterpret_cast<unsigned short *>(out)[r * d + j] = (unsigned short)(u >> 16);
        }
    }
}

extern "C" hb_status hb_route(hb_ctx *c, int64_t N, int32_t *path_out)
{
    if (!c || !path_out) return fail(HB_ERR_INVALID_ARG, "ctx and path_out must be non-NULL");
    if (N < 2 || N > (1 << 20)) return fail(HB_ERR_INVALID_ARG, "N = %lld outside [2, 2^20]", (long long)N);
    *path_out = route_for(c, N);
    g_err.clear();
    return HB_OK;
}

extern "C" hb_status hb_autotune(hb_ctx *c, int64_t d, int32_t dtype, const hb_opts *opts, int64_t max_N,
                                 float *ms_out)
{
    if (!c) return fail(HB_ERR_INVALID_ARG, "ctx is NULL");
    hb_status hs = validate_common(d, dtype);
    if (hs != HB_OK) return hs;
    hs = validate_opts(opts);
    if (hs != HB_OK) return hs;
    if (opts->exhaustive) return fail(HB_ERR_INVALID_ARG, "route tuning needs sampled relabellings");
    CK(cudaSetDevice(c->device));
    constexpr int NR = 4;
    const int32_t paths[NR] = {HB_PATH_MIXED, HB_PATH_MIXED_NARROW, HB_PATH_FP32_PLAIN, HB_PATH_MIXED_2SM};
    if (ms_out)
        for (int k = 0; k < HB_ROUTE_BUCKETS * NR; ++k) ms_out[k] = -1.0f;
    const int64_t rows = (int64_t)1 << 18;
    const size_t esz = dtype == HB_F32 ? 4 : 2;
    void *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)rows * d * esz) != cudaSuccess) {
        cudaGetLastError();
        return fail(HB_ERR_OOM, "tuning buffer of %zu bytes", (size_t)rows * d * esz);
    }
    cudaStream_t s = nullptr;
    k_tune_rows<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(buf, rows, (int)d, dtype, 0x5EEDu);
    hs = cudaGetLastError() == cudaSuccess ? HB_OK : fail(HB_ERR_CUDA, "tuning data kernel failed");
    hb_opts op = *opts;
    op.B = std::min<int64_t>(opts->B, 1023);
    const int64_t top = std::min<int64_t>(std::max<int64_t>(max_N, 64), 65536);
    std::vector<hb_result> res;
    for (int k = 0; hs == HB_OK && k < HB_ROUTE_BUCKETS && ((int64_t)64 << k) <= top; ++k) {
        const int64_t N = (int64_t)64 << k, P = std::max<int64_t>(1, rows / N);
        std::vector<int64_t> n(P, N / 2), m(P, N - N / 2);
        res.assign(P, hb_result{});
        float best = 0.f;
        int32_t best_path = HB_PATH_MIXED;
        for (int r = 0; r < NR && hs == HB_OK; ++r) {
            op.path = paths[r];
            float ms = 0.f;
            for (int rep = 0; rep < 2 && hs == HB_OK; ++rep) {  // the second run is timed
                const auto t0 = std::chrono::steady_clock::now();
                hs = hb_perm_test_batched(c, P, buf, n.data(), m.data(), d, dtype, &op, res.data(), s);
                ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
            }
            if (hs != HB_OK) break;
            if (ms_out) ms_out[k * NR + r] = ms;
            if (r == 0 || ms < best) {
                best = ms;
                best_path = paths[r];
            }
        }
        if (hs == HB_OK) c->route[k] = best_path;
    }
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (hs != HB_OK) return hs;
    c->tuned = true;
    g_err.clear();
    return HB_OK;
}

extern "C" hb_status hb_ctx_set_timing(hb_ctx *c, int32_t enable)
{
    if (!c) return fail(HB_ERR_INVALID_ARG, "ctx is NULL");
    if (enable && !c->tev[0]) {
        CK(cudaSetDevice(c->device));
        for (int k = 0; k < 7; ++k) CK(cudaEventCreate(&c->tev[k]));
        for (cudaEvent_t &e : c->gev) CK(cudaEventCreate(&e));
    }
    c->timing = enable != 0;
    return HB_OK;
}

extern "C" hb_status hb_ctx_stage_times(hb_ctx *c, float *ms_out, int32_t *n_launches)
{
    if (!c || !ms_out) return fail(HB_ERR_INVALID_ARG, "ctx and ms_out must be non-NULL");
    if (!c->last_timed) return fail(HB_ERR_INVALID_ARG, "timing was not enabled for the last call");
    for (int k = 0; k < 7; ++k) ms_out[k] = c->last_ms[k];
    if (n_launches) *n_launches = c->last_launches;
    return HB_OK;
}

extern "C" hb_status hb_ctx_set_option(hb_ctx *c, int32_t option, int64_t value)
{
    if (!c) return fail(HB_ERR_INVALID_ARG, "ctx is NULL");
    switch (option) {
    case HB_OPT_WAIT_LIMIT_NS:
        if (value < 1000 || value > 60000000000ll)
            return fail(HB_ERR_INVALID_ARG, "wait limit %lld ns outside [1 us, 60 s]", (long long)value);
        c->wait_ns = (uint64_t)value;
        break;
    case HB_OPT_SINGLE_SLICE_MAX_N:
        if (value < 0 || value > 65536) return fail(HB_ERR_INVALID_ARG, "single-slice limit %lld", (long long)value);
        c->s1_max = (int32_t)value;
        break;
    case HB_OPT_TEST_WITHHOLD_ARRIVAL:
        c->withhold = value != 0;
        break;
    case HB_OPT_A_OPERAND_TMEM:
        c->a_tmem = value != 0;
        break;
    default:
        return fail(HB_ERR_INVALID_ARG, "option %d unknown", option);
    }
    g_err.clear();
    return HB_OK;
}

void hb_internal_set_error(const char *msg) { g_err = msg ? msg : ""; }

// ---------------------------------------------------------------------------
// learned triage
// ---------------------------------------------------------------------------
static hb_status batched_common(hb_ctx *c, int64_t P, const void *XY, const int64_t *n, const int64_t *m, int64_t d,
                                int32_t dtype, const hb_opts *opts, hb_result *res, float *T_out,
                                const TriageOut *tri, bool features, void *stream)
{
    if (!c) return fail(HB_ERR_INVALID_ARG, "ctx is NULL");
    if (P < 1 || P > (1 << 24)) return fail(HB_ERR_INVALID_ARG, "P = %lld", (long long)P);
    if (!XY || !n || !m || !res) return fail(HB_ERR_INVALID_ARG, "XY, n, m and out must be non-NULL");
    hb_status hs = validate_common(d, dtype);
    if (hs != HB_OK) return hs;
    hs = validate_opts(opts);
    if (hs != HB_OK) return hs;
    CK(cudaSetDevice(c->device));
    hb_opts op = *opts;
    if (op.path == HB_PATH_AUTO) op.path = route_for_batch(c, P, n, m);
    if (features) {
        op.path = HB_PATH_FP32_PLAIN;  // no slices needed
        op.B = 1;
        op.exhaustive = 0;
    }
    Plan pl;
    hs = make_plan(pl, P, n, m, d, dtype, op, false, T_out != nullptr, ctx_opts(c));
    if (hs != HB_OK) return hs;
    const size_t esz = dtype == HB_F32 ? 4 : 2;
    int64_t off = 0;
    for (int64_t p = 0; p < P; ++p) {
        pl.meta[p].X = (const char *)XY + (size_t)off * d * esz;
        pl.meta[p].Y = (const char *)pl.meta[p].X + (size_t)n[p] * d * esz;
        off += n[p] + m[p];
    }
    std::vector<PairOut> out;
    hs = run(c, pl, nullptr, 0, nullptr, false, nullptr, nullptr, nullptr, T_out, (cudaStream_t)stream, out, tri);
    if (hs != HB_OK) return hs;
    for (int64_t p = 0; p < P; ++p) fill_result(out[p], &res[p]);
    g_err.clear();
    return HB_OK;
}

extern "C" hb_status hb_triage_features(hb_ctx *c, int64_t P, const void *XY, const int64_t *n, const int64_t *m,
                                        int64_t d, int32_t dtype, const hb_opts *opts, float *feat_out,
                                        double *tobs_out, hb_result *out, void *stream)
{
    if (!feat_out) return fail(HB_ERR_INVALID_ARG, "feat_out is NULL");
    if (d > 1024) return fail(HB_ERR_UNSUPPORTED, "triage features need d <= 1024");
    TriageOut tri;
    tri.feat = feat_out;
    tri.tobs = tobs_out;
    return batched_common(c, P, XY, n, m, d, dtype, opts, out, nullptr, &tri, true, stream);
}

extern "C" hb_status hb_null_quantiles(hb_ctx *c, int64_t P, const void *XY, const int64_t *n, const int64_t *m,
                                       int64_t d, int32_t dtype, const hb_opts *opts, float *quant_out,
                                       hb_result *out, void *stream)
{
    if (!c || !quant_out || !opts) return fail(HB_ERR_INVALID_ARG, "ctx, opts and quant_out must be non-NULL");
    if (P < 1) return fail(HB_ERR_INVALID_ARG, "P = %lld", (long long)P);
    if (opts->exhaustive || opts->B > 32768) return fail(HB_ERR_UNSUPPORTED, "null quantiles need B <= 32768");
    const size_t need = sizeof(float) * (size_t)P * (size_t)std::max<int64_t>(1, opts->B);
    if (need > c->tbuf_cap) {
        if (c->tbuf) cudaFree(c->tbuf);
        c->tbuf = nullptr;
        c->tbuf_cap = 0;
        if (cudaMalloc(&c->tbuf, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(HB_ERR_OOM, "T buffer of %zu bytes could not be allocated", need);
        }
        c->tbuf_cap = need;
    }
    TriageOut tri;
    tri.quant = quant_out;
    return batched_common(c, P, XY, n, m, d, dtype, opts, out, (float *)c->tbuf, &tri, false, stream);
}

extern "C" int64_t hb_mlp_param_count(void) { return mlp_param_count(); }

static bool mlp_ok(const hb_mlp *net)
{
    return net && net->params && net->params_bf16 && net->grad && net->adam_m && net->adam_v;
}

extern "C" hb_status hb_mlp_sync(const hb_mlp *net, void *stream)
{
    if (!net || !net->params || !net->params_bf16) return fail(HB_ERR_INVALID_ARG, "net is incomplete");
    mlp_to_bf16(net->params, net->params_bf16, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return HB_OK;
}

extern "C" hb_status hb_mlp_forward(hb_ctx *c, const hb_mlp *net, int64_t P, const float *feat, float *out,
                                    void *stream)
{
    if (!c || !net || !net->params || !net->params_bf16 || !feat || !out || P < 1 || P > (1 << 22))
        return fail(HB_ERR_INVALID_ARG, "bad hb_mlp_forward arguments");
    CK(cudaSetDevice(c->device));
    hb_status hs = ensure_ws(c, sizeof(float) * (size_t)mlp_work_floats((int)P));
    if (hs != HB_OK) return hs;
    mlp_forward(net->params, net->params_bf16, (int)P, feat, (float *)c->ws, out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return HB_OK;
}

extern "C" hb_status hb_mlp_grad(hb_ctx *c, const hb_mlp *net, int64_t P, const float *feat, const float *target,
                                 float *loss, void *stream)
{
    if (!c || !mlp_ok(net) || !feat || !target || !loss || P < 1 || P > (1 << 22))
        return fail(HB_ERR_INVALID_ARG, "bad hb_mlp_grad arguments");
    CK(cudaSetDevice(c->device));
    hb_status hs = ensure_ws(c, sizeof(float) * (size_t)mlp_work_floats((int)P));
    if (hs != HB_OK) return hs;
    float *work = (float *)c->ws;
    float *y = work + (int64_t)P * 256 * 4;  // after a1, h1, a2, h2
    mlp_forward(net->params, net->params_bf16, (int)P, feat, work, y, (cudaStream_t)stream);
    mlp_backward(net->params, net->params_bf16, (int)P, feat, target, work, net->grad, loss, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return HB_OK;
}

extern "C" hb_status hb_mlp_adam(const hb_mlp *net, float lr, int64_t t, void *stream)
{
    if (!mlp_ok(net) || t < 1) return fail(HB_ERR_INVALID_ARG, "bad hb_mlp_adam arguments");
    mlp_adam(net->params, net->params_bf16, net->grad, net->adam_m, net->adam_v, lr, t, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return HB_OK;
}

extern "C" hb_status hb_triage_predict_p(int64_t P, const float *quant, const double *tobs, float *p_out,
                                         void *stream)
{
    if (P < 1 || !quant || !tobs || !p_out) return fail(HB_ERR_INVALID_ARG, "bad hb_triage_predict_p arguments");
    launch_predict_p((int)P, quant, 100.0f, tobs, p_out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return HB_OK;
}
