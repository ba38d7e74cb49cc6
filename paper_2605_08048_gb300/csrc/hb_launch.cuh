// hb_launch.cuh -- host-side launchers of the hbperm kernels (one per kernel
// family; each lives in the translation unit that defines its kernels).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "hb_internal.cuh"

namespace hb {
// A contiguous range of pairs, p0 .. p1-1, and of their row chunks, c0 .. c1-1
// (the chunks of a pair follow one another, pair by pair).  The alignment and
// Z-statistics launchers work on one range, so a call can align the pairs
// whose input has arrived while the rest is still being copied.
struct PairSpan {
    int p0, p1;
    int c0, c1;
};
void launch_colsum(const PairMeta *meta, const RowChunk *chunks, const PairSpan &sp, int d, int dtype, i128 *part,
                   i128 *s, int *bad, cudaStream_t st);
void launch_axis(const PairMeta *meta, const PairSpan &sp, const RunOpts &o, const i128 *s, const int *bad,
                 PairState *pst, double *u, cudaStream_t st);
// vec16: every pair's X, Y and Z rows start on 16-byte boundaries (BF16 with
// d % 8 == 0 and d <= 1024 then takes the 16-byte kernel)
void launch_reflect(const PairMeta *meta, const RowChunk *chunks, const PairSpan &sp, const RunOpts &o,
                    const PairState *pst, const double *u, void *Z, unsigned int *colmax,
                    unsigned long long *colL1, bool vec16, cudaStream_t st);
void launch_zstats(const PairMeta *meta, const RowChunk *chunks, const PairSpan &sp, const RunOpts &o,
                   const PairState *pst, const void *Z, const unsigned int *colmax,
                   const unsigned long long *colL1, i128 *tpart, float *cpart, float *cpart1, unsigned short *zq,
                   i128 *t_ex, i128 *s1o, ColConst *cc, float *ct, bool tok_layout, cudaStream_t st);
void launch_tobs(const PairMeta *meta, const PairSpan &sp, const RunOpts &o, const i128 *t_ex, const i128 *s1o,
                 const ColConst *cc, PairState *pst, cudaStream_t st);
void launch_labels_rows(uint64_t seed, uint32_t stream, int n, int N, int64_t b0, int64_t count, uint32_t *out,
                        cudaStream_t st);
void launch_labels_pipeline(const PairMeta *meta, const PairState *pst, const int *order, int p_begin, int p_end,
                            int max_Bpad, const RunOpts &o, uint32_t *bits, cudaStream_t st);
void launch_plain(const PairMeta *meta, int P, int max_Bpad, const RunOpts &o, PairState *pst, const void *Z,
                  const ColConst *cc, const uint32_t *bits, RecheckItem *list, unsigned int *n_items,
                  unsigned int cap, unsigned int *overflow, float *T_out, cudaStream_t st);
void launch_recheck(unsigned int cap, unsigned int batch, int max_W, const PairMeta *meta, const RunOpts &o,
                    PairState *pst, const void *Z, const i128 *t_ex, const unsigned int *colmax, const uint32_t *bits,
                    const RecheckItem *list, const unsigned int *n_items, double *sums, float *T_out,
                    cudaStream_t st);
void launch_finalize(const PairMeta *meta, int P, const RunOpts &o, const PairState *pst, PairOut *out,
                     cudaStream_t st);
// tensor-core path (hb_mixed.cu)
// A work item is one 128-relabelling tile for single CTAs and two consecutive
// tiles of one pair for CTA pairs (tcgen05 cta_group::2).
enum : int32_t { MODE_FULL = 0, MODE_SINGLE = 1, MODE_GATHER = 2 };
struct WorkItem {
    int32_t pair;
    int32_t tile;  // group of (cluster size) consecutive 128-row tiles of the pair's relabellings or list
    int32_t mode;  // MODE_FULL, MODE_SINGLE (BF16: first slice only) or MODE_GATHER (listed relabellings)
};
struct MixedArgs {
    const PairMeta *meta;
    int P;
    RunOpts o;
    PairState *st;
    const ColConst *cc;
    const float *ct;  // column totals t alone, [pair][d_pad] (zero past d)
    const uint32_t *bits;
    const unsigned short *zq;
    int64_t zq_ld;    // token positions of the slice matrix (a multiple of 64)
    int64_t zq_rows;  // slice rows
    const WorkItem *items;
    int n_work;                      // >= 0: items; < 0: the count is *n_work_dev (written on the device)
    const unsigned int *n_work_dev;
    uint32_t *glist;                 // relabellings MODE_SINGLE leaves to MODE_GATHER (per pair from g_off)
    RecheckItem *list;
    unsigned int *n_items;
    unsigned int cap;
    unsigned int *overflow;
    unsigned int *timeout;
    float *T_out;
    uint64_t wait_ns;                // wall-clock limit of every device barrier wait
    int withhold;                    // test hook: one barrier arrival withheld (the wait runs out)
    int sms;
};
// the gathered pass's work list: ceil(n_gather / 128) items per pair, *n_items of them
// work items of the gathered pass for pairs order[p0 .. p1) (order null: p0 .. p1)
void launch_gather_items(const PairState *st, const int *order, int p0, int p1, WorkItem *items,
                         unsigned int *n_items, cudaStream_t s);
cudaError_t launch_mixed(const MixedArgs &a, cudaStream_t s, std::string &err);

// learned triage (hb_triage.cu)
void launch_features(const PairMeta *meta, int P, const RunOpts &o, const PairState *st, const void *Z, float *lam,
                     float *feat, double *tobs, cudaStream_t s);
void launch_null_quantiles(const PairMeta *meta, int P, int max_B, const float *T, const PairState *st, float scale,
                           float *q_out, cudaStream_t s);
int64_t mlp_param_count();
int64_t mlp_work_floats(int P);
void mlp_forward(const float *params, const unsigned short *wh, int P, const float *feat, float *work, float *y_out,
                 cudaStream_t s);
void mlp_backward(const float *params, const unsigned short *wh, int P, const float *feat, const float *target,
                  float *work, float *grad, float *loss, cudaStream_t s);
void mlp_adam(float *params, unsigned short *wh, const float *grad, float *m, float *v, float lr, int64_t t,
              cudaStream_t s);
void mlp_to_bf16(const float *params, unsigned short *wh, cudaStream_t s);
void launch_predict_p(int P, const float *q_scaled, float scale, const double *tobs, float *p_out, cudaStream_t s);

void set_kernel_attributes();
void set_align_attributes();
}  // namespace hb
