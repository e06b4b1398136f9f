// Internal declarations shared by the host API and the kernels of libabea.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/abea.h"

namespace abea {

// Per-read descriptor, built on the host for every batch (thesis Sec. "Data
// array serialisation": one flat array per kind of data plus per-read
// offsets into each).
struct ReadDesc {
    int64_t ev_off;     // first event of the read in the events array
    int64_t seq_off;    // first base of the read in the bases array
    int64_t kc_off;     // first k-mer cache entry (float4 units)
    int64_t tr_off;     // first trace word (uint32 units); one record of rec_words per band
    int64_t mv_off;     // first per-band move byte (used only when all 32 lanes hold the band)
    int64_t pair_off;   // first output pair (int2 units)
    int32_t n_e;        // events
    int32_t n_k;        // k-mers
    int32_t pair_cap;   // output pair capacity
    int32_t host_bad;   // rejected on the host (counts, scalings)
    // transition constants, FP64 rounded once; lp_stay_step = lp_stay - lp_step (the scores are
    // carried as S + lp_step, so the stay transition adds lp_stay - lp_step)
    float lp_skip, lp_stay_step, lp_step, lp_trim;
    // read-model scaling, FP64; log_var_step = ln(var) - lp_step (folds lp_step into the k-mer
    // cache's emission constant)
    double scale, shift, inv_var, log_var_step;
};
static_assert(sizeof(ReadDesc) == 112, "descriptor layout");

// Per model row: mean, sqrt(1/2)/stdv, ln(1/sqrt(2 pi)) - ln(stdv) and stdv, FP64.
struct ModelRow {
    double mu;
    double a0;
    double c0;
    double sd;          // the stdv as given
};

// Band-record geometry for a band width W: C offsets per lane, L lanes,
// W' = C*L >= W physical offsets (mixed: W' > W), full: L == 32 (no lane
// above the band); cg offsets per lane when a block's warps share one read
// (0: never); rec_words uint32 words of trace reserved per band (the larger
// record of the two modes).
struct Geometry {
    int C, L, Wp, rec_words, cg;
    bool mixed, full;
};
Geometry geometry_for(int W);

struct AlignArgs {
    const ReadDesc *rd;
    const int32_t *order;      // reads in processing order (longest first)
    const int32_t *flags;      // nonzero: bad input found on the device
    int32_t n;
    int32_t W;
    int32_t L;
    const float *events;
    const uint8_t *seq;
    const float4 *kc;
    uint32_t *trace;
    uint8_t *moves;            // per band: 1 if it moved by one k-mer (only when full)
    int32_t *pairs;            // int32 pairs, (event, k-mer)
    abea_result *res;
    int32_t *queue;            // work counter, zeroed before the launch
    int32_t n_group;           // order[0 .. n_group-1] run in block mode (one read per block)
};

// Launchers (return cudaError_t as int).
int launch_prep(const ReadDesc *rd, int32_t n, const uint8_t *seq, const float *events,
                const ModelRow *model, int k, float4 *kc, int32_t *flags, void *stream);
int launch_align(const AlignArgs &a, const Geometry &g, int grid, void *stream);
// model_f: the model's level mean and stdv as floats, one float2 per k-mer rank.
// The batch's bases are seq[seq_lo .. seq_hi); ranks: scratch of one int2 per
// base; total_slots = pair_off[n] - pair_off[0].
int launch_eventalign(const int64_t *meta, int32_t n, int64_t total_slots, const uint8_t *seq, int64_t seq_lo,
                      int64_t seq_hi, int2 *ranks, const float *events, const abea_scalings *sc, const abea_result *res, const int32_t *pairs,
                      const int32_t *ref_pos, const uint8_t *ref, int64_t ref_len, const float2 *model_f, int k,
                      int scale_events, abea_eventalign_row *rows, void *stream);
// Read summaries (meta as for eventalign: seq_off, ev_off, pair_off, n+1 each).
int launch_summary(const int64_t *meta, int32_t n, int k, const abea_result *res, const int32_t *pairs,
                   abea_read_summary *out, void *stream);
// Event detection runs over tiles of kEventTile positions (a read of len
// samples has ceil(len / kEventTile) tiles; tile_off is their prefix over the
// reads, tile_read the read of each tile).  scratch holds event_tile_bytes()
// per tile.  Three launches.
constexpr int kEventTile = 4096;
size_t event_tile_bytes();
int launch_events(const int64_t *raw_off, const int64_t *ev_off, const int64_t *tile_off, const int32_t *tile_read,
                  int32_t n, int64_t n_tiles, const int16_t *raw, const abea_calib *calib, int window, float tau2,
                  void *scratch, abea_event *out, int32_t *n_ev, void *stream);
int launch_f32_from_i64(const int64_t *in, int64_t n, float *out, void *stream);
int launch_f32_from_f64(const double *in, int64_t n, float *out, void *stream);
int launch_scalings(const int64_t *d_seq_off, const int64_t *d_ev_off, int32_t n, const uint8_t *seq,
                    const float *events, const float2 *model_f, int k, abea_scalings *out, int32_t *status,
                    void *stream);
int align_grid_size(const Geometry &g, int device);

constexpr double kDefaultBlockTheta = 1.0;

// How many of the longest reads (order[0..], longest first) run in block
// mode: those with more than theta times the bands each warp of the launch
// would get if the batch were spread evenly, at most one per block.
int group_count(const ReadDesc *rd, const int32_t *order, int32_t n, const Geometry &g, int grid, double theta);
// Blocks to launch for n reads of which n_group run in block mode (at most grid).
int align_launch_grid(int32_t n, int n_group, int grid);

// Context internals used by the serving loop.
int context_model(const abea_ctx *c, int *k, const float **mean, const float **stdv);
int context_device(const abea_ctx *c);
size_t context_budget(const abea_ctx *c);
void *context_stream(const abea_ctx *c);
// Device bytes a read of n_e events and seq_len bases with pair_cap pairs needs in a batch.
size_t request_bytes(const abea_ctx *c, int W, int64_t n_e, int64_t seq_len, int64_t pair_cap);
// abea_align_packed for one wave whose host buffers are all page-locked (the
// caller guarantees it), enqueued on the context's own stream without waiting;
// ABEA_ERR_NOMEM if the batch exceeds the context's budget.  The buffers must
// stay valid until the stream has passed the copies back.
int align_packed_async(abea_ctx *c, int32_t n, int W, const char *seq, const int64_t *seq_off, const float *events,
                       const int64_t *ev_off, const abea_scalings *sc, abea_result *out, int32_t *pairs,
                       const int64_t *pair_off);

}  // namespace abea
