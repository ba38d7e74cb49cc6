// hb_noalloc.cu -- hb_align_noalloc: the alignment stage (steps 1-3 of the
// test) for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc -- a host application
// whose device memory is entirely reserved by its own pool allocator (for
// example a framework's caching allocator holding most of HBM), or a
// latency-critical pipeline that cannot accept cudaMalloc's implicit device
// synchronisation.  hb_align gets its scratch from an hb_ctx workspace that the
// library allocates on demand; this entry point takes all of its scratch from
// one fixed array in device global memory instead and allocates nothing.
//
// The scratch array is a file-scope static __device__ array of
// NOALLOC_SCRATCH_BYTES (2 MiB).  Every GPU that loads the library holds it
// until the process exits.  All calls share it and it keeps the contents of
// the last call: the set-up kernel below clears what must start at zero, and
// calls that overlap on the GPU (different streams, different host threads)
// race on it.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress, with
// that device current; that first call should therefore come before any
// stream capture.
#include <cstring>
#include <mutex>

#include "hb_launch.cuh"
#include "hbperm.h"

namespace hb {

constexpr size_t NOALLOC_SCRATCH_BYTES = 2u << 20;
constexpr int NOALLOC_MAX_D = 1024;
constexpr int NOALLOC_MAX_ROWS = 8192;  // n + m

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Layout of the scratch for one pair (offsets 256-byte aligned).
struct NoallocLayout {
    size_t meta, chunks, bad, st, part, s, u, total;
    NoallocLayout(int nch, int d)
    {
        size_t off = 0;
        auto take = [&](size_t bytes) {
            off = (off + 255) & ~(size_t)255;
            const size_t at = off;
            off += bytes;
            return at;
        };
        meta = take(sizeof(PairMeta));
        chunks = take(sizeof(RowChunk) * (size_t)nch);
        bad = take(sizeof(int));
        st = take(sizeof(PairState));
        part = take(sizeof(i128) * (size_t)nch * d);
        s = take(sizeof(i128) * 2 * (size_t)d);
        u = take(sizeof(double) * (size_t)d);
        total = off;
    }
};

// Writes the pair metadata and the row-chunk table into the scratch and
// clears the input-validity flag (the scratch keeps the previous call's data).
__global__ void k_noalloc_setup(PairMeta pm, int nch_x, int nch_y, size_t off_meta, size_t off_chunks, size_t off_bad)
{
    PairMeta *meta = reinterpret_cast<PairMeta *>(g_noalloc_scratch + off_meta);
    RowChunk *chunks = reinterpret_cast<RowChunk *>(g_noalloc_scratch + off_chunks);
    int *bad = reinterpret_cast<int *>(g_noalloc_scratch + off_bad);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *meta = pm;
        *bad = 0;
    }
    if (t < nch_x) chunks[t] = RowChunk{0, 0, t * CHUNK_ROWS, min(CHUNK_ROWS, pm.n - t * CHUNK_ROWS)};
    else if (t < nch_x + nch_y) {
        const int k = t - nch_x;
        chunks[t] = RowChunk{0, 1, k * CHUNK_ROWS, min(CHUNK_ROWS, pm.m - k * CHUNK_ROWS)};
    }
}

static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[64] = {};

}  // namespace hb

using namespace hb;

// sets the message hb_last_error() returns (hb_api.cu)
void hb_internal_set_error(const char *msg);

extern "C" hb_status hb_align_noalloc(const void *X, int64_t n, const void *Y, int64_t m, int64_t d, int32_t dtype,
                                      int32_t align, int32_t reflect_side, void *Z_out, double *u_out,
                                      int32_t *skipped, void *stream)
{
    // every return sets the message hb_last_error() reports (cleared on success)
    auto err = [](hb_status st, const char *msg) {
        hb_internal_set_error(msg);
        return st;
    };
    if (!X || !Y || !Z_out) return err(HB_ERR_INVALID_ARG, "hb_align_noalloc: X, Y and Z_out must be non-NULL");
    if (dtype != HB_F32 && dtype != HB_BF16) return err(HB_ERR_INVALID_ARG, "hb_align_noalloc: dtype unknown");
    if (reflect_side != 0 && reflect_side != 1)
        return err(HB_ERR_INVALID_ARG, "hb_align_noalloc: reflect_side must be 0 or 1");
    if (n < 1 || m < 1 || d < 1) return err(HB_ERR_INVALID_ARG, "hb_align_noalloc: n, m and d must be >= 1");
    if (d > NOALLOC_MAX_D || n + m > NOALLOC_MAX_ROWS)
        return err(HB_ERR_UNSUPPORTED,
                   "hb_align_noalloc: needs d <= 1024 and n + m <= 8192 (fixed 2 MiB device scratch)");
    const int nch_x = (int)((n + CHUNK_ROWS - 1) / CHUNK_ROWS), nch_y = (int)((m + CHUNK_ROWS - 1) / CHUNK_ROWS);
    const NoallocLayout L(nch_x + nch_y, (int)d);
    if (L.total > NOALLOC_SCRATCH_BYTES)
        return err(HB_ERR_UNSUPPORTED, "hb_align_noalloc: the request does not fit the 2 MiB device scratch");

    // once per device, with that device current: the array's device address
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return err(HB_ERR_CUDA, "hb_align_noalloc: cudaGetDevice failed or the device index is >= 64");
    }
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return err(HB_ERR_CUDA, "hb_align_noalloc: cudaGetSymbolAddress of the scratch array failed");
            }
            g_noalloc_ptr[dev] = (unsigned char *)p;
        }
        base = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;

    PairMeta pm;
    memset(&pm, 0, sizeof pm);
    pm.X = X;
    pm.Y = Y;
    pm.n = (int)n;
    pm.m = (int)m;
    pm.N = (int)(n + m);
    pm.N_pad = (int)(((n + m) + 63) / 64 * 64);
    pm.W = (int)((n + m + 31) / 32);
    pm.T_off = -1;
    pm.chunk0 = 0;
    pm.nchunk_x = nch_x;
    pm.nchunk_y = nch_y;
    RunOpts o;
    memset(&o, 0, sizeof o);
    o.align = align ? 1 : 0;
    o.reflect_side = reflect_side;
    o.path = HB_PATH_FP32_PLAIN;
    o.d = (int)d;
    o.d_pad = (int)d;
    o.dtype = dtype;
    o.cw = 128;

    const int nch = nch_x + nch_y;
    PairMeta *meta = (PairMeta *)(base + L.meta);
    RowChunk *chunks = (RowChunk *)(base + L.chunks);
    int *bad = (int *)(base + L.bad);
    PairState *st = (PairState *)(base + L.st);
    i128 *part = (i128 *)(base + L.part);
    i128 *sums = (i128 *)(base + L.s);
    double *u = (double *)(base + L.u);

    k_noalloc_setup<<<(nch + 127) / 128, 128, 0, s>>>(pm, nch_x, nch_y, L.meta, L.chunks, L.bad);
    const PairSpan all{0, 1, 0, nch};
    launch_colsum(meta, chunks, all, (int)d, dtype, part, sums, bad, s);
    launch_axis(meta, all, o, sums, bad, st, u, s);
    const bool vec16 = (d * (dtype == HB_F32 ? 4 : 2)) % 16 == 0 &&
                       (((uintptr_t)X | (uintptr_t)Y | (uintptr_t)Z_out) & 15u) == 0;
    launch_reflect(meta, chunks, all, o, st, u, Z_out, nullptr, nullptr, vec16, s);
    if (cudaGetLastError() != cudaSuccess) return err(HB_ERR_CUDA, "hb_align_noalloc: a kernel launch failed");
    if (u_out && cudaMemcpyAsync(u_out, u, sizeof(double) * (size_t)d, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return err(HB_ERR_CUDA, "hb_align_noalloc: copy of u failed");
    }
    if (skipped) {
        PairState hst;
        if (cudaMemcpyAsync(&hst, st, sizeof hst, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return err(HB_ERR_CUDA, "hb_align_noalloc: reading the alignment status failed");
        }
        if (hst.status != ST_OK) return err((hb_status)hst.status, "hb_align_noalloc: alignment failed (invalid or degenerate input)");
        *skipped = hst.skipped;
    }
    hb_internal_set_error("");
    return HB_OK;
}
