/*
 * abea.h -- C ABI of the GB300-native Adaptive Banded Event Alignment library.
 *
 * The problem (H. Gamaarachchi, PhD thesis, UNSW 2020, Ch.5, Alg.
 * adaptivebandedcpu): given a read's base sequence `ref`, a k-mer pore model
 * and the read's detected events, align the events to the read's k-mers with
 * an adaptively banded dynamic program and return the alignment as a list of
 * {event index, k-mer index} pairs.  The library adds the per-read score of
 * that alignment.
 *
 * Conventions shared by every call:
 *   - Return value: ABEA_OK (0) or a negative ABEA_ERR_* code; no exception
 *     crosses the ABI.  abea_strerror() names a code.
 *   - Per-read outcome: abea_result.status, one of ABEA_READ_*.
 *   - Host pointers are owned by the caller and only read (or, for outputs,
 *     written) during the call.  Device pointers (the *_device call) are
 *     borrowed for the duration of the call's work on the given stream.
 *   - The context owns every device allocation it makes; it copies the model.
 *     A context is not thread-safe: use one context per host thread.
 *   - Indices are 0-based.  Pairs are (event, k-mer) int32 pairs in
 *     ascending order.  A k-mer's model row is its rank over A,C,G,T with
 *     the first base most significant (A=0, C=1, G=2, T=3).
 *   - Band width W: 2 <= W <= 256.
 *   - Scores are FP32.  Events are FP32 event means in pA (the thesis's
 *     Alg. adaptivebandedcpucomputelog uses only the mean of an event).
 */
#ifndef ABEA_H
#define ABEA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define ABEA_OK 0
#define ABEA_ERR_ARG (-1)        /* invalid argument (null pointer, bad size, W out of range, k mismatch) */
#define ABEA_ERR_CAPACITY (-2)   /* an output buffer is too small (abea_align: required pairs in out->n_pairs) */
#define ABEA_ERR_NOMEM (-3)      /* a device or pinned-host allocation failed, or the memory budget is too small */
#define ABEA_ERR_CUDA (-4)       /* a CUDA runtime call failed */
#define ABEA_ERR_TIMEOUT (-5)    /* a bounded device wait gave up */
#define ABEA_ERR_NO_MODEL (-6)   /* no pore model set */

/* Per-read status. */
#define ABEA_READ_OK 0           /* aligned */
#define ABEA_READ_FAIL_NO_END 1  /* no band reached the last k-mer with a finite score */
#define ABEA_READ_BAD_INPUT 2    /* non-ACGT base, non-finite event, var <= 0, no events, or seq shorter than k */
#define ABEA_READ_CAPACITY 3     /* the read's pair capacity is smaller than its alignment (n_pairs = required) */

/* Per-read status of abea_estimate_scalings. */
#define ABEA_SCALE_OK 0          /* scale and shift from the moments */
#define ABEA_SCALE_DEGENERATE 1  /* fewer than 2 events or a zero variance: scale 1, shift = mean difference */
#define ABEA_SCALE_BAD_INPUT 2   /* no events or k-mers, non-ACGT base or non-finite event: scale 1, shift 0 */

typedef struct abea_ctx abea_ctx;

/* Read-model scaling (thesis Sec. ABEA, "read-model scaling"): the model
 * mean of every k-mer becomes mean*scale + shift; its stdv becomes
 * stdv*var.  var = 1 is the thesis's two-parameter scaling exactly. */
typedef struct {
    float scale, shift, var;
} abea_scalings;

/* One read on the host: event means, bases ('A','C','G','T'), scalings.
 * n_kmers = seq_len - k + 1. */
typedef struct {
    const float *ev_mean;
    int32_t n_events;
    const char *seq;
    int32_t seq_len;
    abea_scalings sc;
} abea_read;

/* Per-read result.
 * score  : FP32 score of the alignment: the best S(e, n_k-1) + (n_e-1-e)*ln(1/100),
 *          -inf when status != OK.
 * e_end  : event of that end cell.
 * cells  : in-matrix band cells filled for this read (the throughput unit). */
typedef struct {
    float score;
    int32_t status;
    int32_t n_pairs;
    int32_t e_end;
    int64_t cells;
} abea_result;

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the
 * device memory the context may hold for batch work (0 = 90 % of the free
 * memory at creation).  Batches whose working set exceeds the budget are
 * run in several waves that reuse the same buffers (thesis Sec. "Heuristic
 * based memory pre-allocation": memory is allocated once and reused).
 * On error *ctx is NULL. */
int abea_create(abea_ctx **ctx, int device, size_t mem_budget_bytes);

/* Release every device and pinned allocation of the context. NULL is a no-op. */
void abea_destroy(abea_ctx *ctx);

/* Human-readable name of a return code. */
const char *abea_strerror(int code);

/* Set the pore model (thesis Sec. "Methylation calling": a table of all 4^k
 * k-mers with a mean level and a standard deviation).  level_mean and
 * level_stdv are host arrays of 4^k floats, copied.  1 <= k <= 12; every
 * stdv must be finite and > 0 and every mean finite (else ABEA_ERR_ARG). */
int abea_set_model(abea_ctx *ctx, int k, const float *level_mean, const float *level_stdv);

/* Align one read, synchronously.  pairs: host int32[2*cap].  If the
 * alignment has more than cap pairs, returns ABEA_ERR_CAPACITY with the
 * required count in out->n_pairs.  cap = n_events + n_kmers - 1 always
 * suffices. */
int abea_align(abea_ctx *ctx, const abea_read *read, int W, abea_result *out,
               int32_t *pairs, int32_t cap);

/* Align n reads given as abea_read records (host memory).  out: host
 * abea_result[n].  pairs: host int32[2*pair_off[n]]; read i's pairs go to
 * pairs[2*pair_off[i] .. 2*pair_off[i+1]) and its capacity is
 * pair_off[i+1]-pair_off[i] pairs.  Host-to-device copies, kernels and the
 * device-to-host copy are issued on cuda_stream (a cudaStream_t, or NULL for
 * the context's own stream); the call returns after the results are on the
 * host. */
int abea_align_batch(abea_ctx *ctx, const abea_read *reads, int32_t n, int W,
                     abea_result *out, int32_t *pairs, const int64_t *pair_off, void *cuda_stream);

/* As abea_align_batch, with the reads packed on the host as structures of
 * arrays: read i's bases are seq[seq_off[i] .. seq_off[i+1]), its events
 * events[ev_off[i] .. ev_off[i+1]), its scalings sc[i]. */
int abea_align_packed(abea_ctx *ctx, int32_t n, int W,
                      const char *seq, const int64_t *seq_off,
                      const float *events, const int64_t *ev_off, const abea_scalings *sc,
                      abea_result *out, int32_t *pairs, const int64_t *pair_off, void *cuda_stream);

/* Align n reads whose bulk data is already in device memory.  The offsets
 * and scalings are host arrays (as in abea_align_packed); d_seq (bases),
 * d_events, d_out (abea_result[n]) and d_pairs (int32[2*pair_off[n]]) are
 * device pointers.  All work is enqueued on cuda_stream and the call
 * returns without waiting for it; the outputs are valid once the stream
 * reaches that point.  The batch must fit the memory budget in one wave
 * (else ABEA_ERR_NOMEM). */
int abea_align_batch_device(abea_ctx *ctx, int32_t n, int W,
                            const uint8_t *d_seq, const int64_t *seq_off,
                            const float *d_events, const int64_t *ev_off, const abea_scalings *sc,
                            abea_result *d_out, int32_t *d_pairs, const int64_t *pair_off,
                            void *cuda_stream);

/* Launch statistics accumulated since the previous call of this function
 * (or since the context was created): the number of kernel launches the
 * batch calls issued, and the summed device time of their core-kernel
 * launches in milliseconds, measured with CUDA events recorded on each
 * call's stream immediately around the core kernel.  Waits for those events;
 * then resets both counters.  Up to 4096 core-kernel launches are timed
 * between two calls (later ones are folded into the last slot). */
int abea_last_launch_stats(abea_ctx *ctx, int32_t *n_launches, float *align_kernel_ms);

/* eventalign rows (f5c's eventalign: events aligned to reference k-mers; the
 * thesis gives no record format).  For every read i with d_results[i].status
 * == ABEA_READ_OK, its d_results[i].n_pairs pairs (event e, read k-mer j) at
 * d_pairs + 2*pair_off[i] become records d_rows[pair_off[i] + t]:
 *   ref_pos    reference position of k-mer j's first base, d_ref_pos[seq_off[i] + j]
 *              (the read's base-space alignment: one int32 per read base, -1 for an insertion),
 *   ref_rank   rank of d_ref[ref_pos .. ref_pos+k) (-1 if unaligned, past ref_len or not ACGT),
 *   model_rank rank of the read k-mer,
 *   default:       level = x_e, model_mean = mu*scale + shift, model_stdv = sigma*var;
 *   scale_events:  level = (x_e - shift)/scale, model_mean = mu, model_stdv = sigma*var/scale;
 *   z = (level - model_mean) / model_stdv (FP32, one operation at a time in that order).
 * Rows of other reads and past n_pairs are not written.  d_* are device
 * pointers (d_seq, d_events, d_results, d_pairs as given to and returned by
 * abea_align_batch_device), seq_off, ev_off, sc and pair_off host arrays;
 * uses ctx's model; enqueued on cuda_stream. */
typedef struct {
    int32_t read, event, kmer, ref_pos, ref_rank, model_rank;
    float level, model_mean, model_stdv, z;
} abea_eventalign_row;
int abea_eventalign(abea_ctx *ctx, int32_t n, const uint8_t *d_seq, const int64_t *seq_off,
                    const float *d_events, const int64_t *ev_off, const abea_scalings *sc,
                    const abea_result *d_results, const int32_t *d_pairs, const int64_t *pair_off,
                    const int32_t *d_ref_pos, const uint8_t *d_ref, int64_t ref_len, int scale_events,
                    abea_eventalign_row *d_rows, void *cuda_stream);

/* Per-read summary of an alignment, for eventalign's consumers (f5c's
 * eventalign lists a --summary option, "summarise the alignment of each
 * read", with no format; the fields below are a reading).  From a read's
 * result and its pairs (event e, k-mer j), ascending:
 *   first_event, last_event  events of the first and last pair (-1 if none);
 *                            the first_event leading and n_events-1-last_event
 *                            trailing events are trimmed;
 *   stays    pairs whose event follows the previous pair's on the same k-mer
 *            (e+1, j): an extra event on one k-mer;
 *   skips    pairs whose k-mer follows the previous pair's with the same
 *            event (e, j+1): a k-mer entered without an event of its own;
 *   events_aligned = n_pairs - skips (distinct events in the pairs);
 *   score_per_event = score / n_events;
 *   flags: ABEA_QC_NOT_ALIGNED (status is not ABEA_READ_OK), ABEA_QC_TRIMMED
 *   (more than half of the events trimmed), ABEA_QC_SKIPS (skips above a fifth
 *   of the k-mers), ABEA_QC_LOW_SCORE (score_per_event below -10). */
#define ABEA_QC_NOT_ALIGNED 1
#define ABEA_QC_TRIMMED 2
#define ABEA_QC_SKIPS 4
#define ABEA_QC_LOW_SCORE 8
typedef struct {
    int32_t read, status, n_events, n_kmers, n_pairs;
    int32_t first_event, last_event, events_aligned, stays, skips;
    float score, score_per_event;
    int32_t flags;
} abea_read_summary;
/* Summaries of reads 0..n-1 from the device results and pairs of
 * abea_align_batch_device (d_results, d_pairs at 2*pair_off[i]); ev_off,
 * seq_off and pair_off are host arrays, k the model's k (n_kmers = bases - k
 * + 1); d_out: n device records.  Enqueued on cuda_stream (one warp per
 * read). */
int abea_summarise(abea_ctx *ctx, int32_t n, const int64_t *seq_off, const int64_t *ev_off,
                   const abea_result *d_results, const int32_t *d_pairs, const int64_t *pair_off,
                   abea_read_summary *d_out, void *cuda_stream);

/* Tab-separated text of eventalign rows (host arrays), one line per row:
 *   read event kmer ref_pos ref_kmer model_kmer level model_mean model_stdv z
 * k-mers as bases (lexicographic ranks over ACGT, first base most
 * significant; "NNN..." for ref_rank -1), level, model_mean and model_stdv
 * with 2 decimals, z with 3 (printf "%.2f" / "%.3f").  With header, a first
 * line of the column names.  Writes at most cap bytes to buf (NUL
 * terminated when cap > 0) and the full length (without the NUL) to
 * *needed; ABEA_ERR_CAPACITY if it did not fit.  No CUDA call. */
int abea_eventalign_tsv(const abea_eventalign_row *rows, int64_t n_rows, int k, int header, char *buf,
                        size_t cap, size_t *needed);
/* Tab-separated text of read summaries (host array), one line per read:
 *   read status n_events n_kmers n_pairs first_event last_event events_aligned stays skips score
 *   score_per_event flags
 * scores with 3 decimals; otherwise as abea_eventalign_tsv. */
int abea_summary_tsv(const abea_read_summary *s, int32_t n, int header, char *buf, size_t cap, size_t *needed);

/* Event detection: raw signal -> events (thesis Sec. "Methylation calling":
 * the raw signal is segmented at sudden level changes, each segment an event
 * with the mean, standard deviation and duration of its samples; the thesis
 * gives no detector).  Two-window t-test: at sample position i of a read with
 * exact window sums S_L, S_R (of x[i-window, i) and x[i, i+window)) and
 * Q_L, Q_R of the squares, t2 = float(window*(S_R-S_L)^2) /
 * float(window*(Q_L+Q_R) - S_L^2 - S_R^2) (+inf for a zero denominator and a
 * nonzero numerator), 0 where a window leaves the read.  Position i >= 1
 * starts an event when t2 >= tau2 and t2 is the maximum within
 * window-1 positions on each side (ties to the earliest).  Each event:
 * mean = float(S)/L, stdv = sqrt(max(float(Q)/L - mean^2, 0)) (FP32, in that
 * order), both in pA: (mean + offset) * pa_per_unit, stdv * pa_per_unit.
 * Starts are at least `window` samples apart, so a read of L samples has at
 * most L/window + 1 events.  window in [2, 8]; defaults 3 and 2.0 give about
 * 1.7 events per k-mer on the synthetic signals (the thesis reports 1.5-2.5).
 * d_raw (int16 samples), d_events (event_off[n] entries) and d_n_events
 * (int32[n]) are device pointers; raw_off, calib and event_off host arrays.
 * d_n_events[i] is read i's event count; only its first
 * event_off[i+1]-event_off[i] events are written. */
typedef struct { float mean, stdv; int32_t start, length; } abea_event;   /* pA, pA, samples, samples */
typedef struct { float offset, pa_per_unit; } abea_calib;                 /* pA = (raw + offset) * pa_per_unit */
int abea_detect_events(abea_ctx *ctx, int32_t n, const int16_t *d_raw, const int64_t *raw_off,
                       const abea_calib *calib, int window, float tau2, abea_event *d_events,
                       const int64_t *event_off, int32_t *d_n_events, void *cuda_stream);

/* The integer-to-float rounding that event detection uses for its sums and
 * t2 terms: d_out[j] = the float nearest to d_in[j], ties to even
 * (|d_in[j]| < 2^63), formed from integer operations.  Exposed so that it can
 * be checked against the platform's own conversion.  d_in (int64[n]) and
 * d_out (float[n]) are device pointers; enqueued on cuda_stream.  Returns
 * ABEA_ERR_ARG for n < 0 or a null pointer with n > 0. */
int abea_f32_from_i64(const int64_t *d_in, int64_t n, float *d_out, void *cuda_stream);

/* The double-to-float rounding that the pre-kernel uses for the k-mer
 * cache's FP64 operands: d_out[j] = the float nearest to d_in[j], ties to
 * even, formed from integer operations where the result is a normal float
 * (the FP64 pipe's conversion otherwise).  Exposed so that it can be checked
 * against the platform's own conversion.  d_in (double[n]) and d_out
 * (float[n]) are device pointers; enqueued on cuda_stream.  Returns
 * ABEA_ERR_ARG for n < 0 or a null pointer with n > 0. */
int abea_f32_from_f64(const double *d_in, int64_t n, float *d_out, void *cuda_stream);

/* Per-read scalings by the method of moments (thesis Sec. "Read-model
 * scaling": shift and scale are estimated per read before ABEA, which then
 * uses mu * scale + shift; the thesis gives no formula).  For read i, with
 * m_e, v_e the mean and population variance of its event means and m_m, v_m
 * those of the model level means (ctx's model) along its k-mers:
 *   d_out[i] = { scale = sqrt(v_e / v_m), shift = m_e - scale * m_m, var = 1 },
 * d_status[i] = ABEA_SCALE_OK; degenerate and rejected reads as the
 * ABEA_SCALE_* codes say.  The sums carry about 48 significant bits (error-
 * free FP32 pairs), the moments and the square root are FP64, and each
 * result is within one float ulp of the FP64 definition rounded once.  Bulk data
 * as in abea_align_batch_device: d_seq, d_events, d_out (abea_scalings[n])
 * and d_status (int32[n]) are device pointers, seq_off and ev_off host
 * arrays; enqueued on cuda_stream without waiting. */
int abea_estimate_scalings(abea_ctx *ctx, int32_t n, const uint8_t *d_seq, const int64_t *seq_off,
                           const float *d_events, const int64_t *ev_off, abea_scalings *d_out,
                           int32_t *d_status, void *cuda_stream);

/* Scheduling of long reads (the paper has no counterpart; results do not
 * depend on it).  Within one core-kernel launch a read normally occupies one
 * warp; a read with more than theta times the bands that each warp of the
 * launch would get if the batch were spread evenly is instead shared by the
 * four warps of one block (at most one such read per block, longest first),
 * so that it does not set the batch's makespan.  theta <= 0 disables this;
 * the default is 1.0.  Band widths that do not split over four warps
 * (W < 32, W not a multiple of 4, or W / 4 not a multiple of 1 or 2 with
 * at most 31 lanes) always run one read per warp.  Returns ABEA_ERR_ARG for
 * a NaN theta. */
int abea_set_block_mode(abea_ctx *ctx, double theta);

/* Launch-geometry autotuner (the paper has no counterpart; results do not
 * depend on it).  The per-read choice couples three knobs: a read runs
 * either in per-warp mode (4 reads per CTA, one warp each; L = ceil(W/C)
 * threads per band; a trace record of 2C words per band) or in block mode
 * (1 read per CTA; its 4 warps share each band, 4 x L' threads; a record of
 * 4 x 2C' words).  abea_autotune times both modes on a caller's sample of
 * reads (host arrays as for abea_align_packed) for each length bucket of
 * bands per read: [0, 4096), [4096, 16384), [16384, 65536), [65536, inf)
 * (bands = events + k-mers + 1), two runs per mode after a warm-up, keeping
 * the faster of each (device time of the core kernels).  Block mode is then
 * used from the shortest bucket upward where it keeps winning: later batch
 * calls of ctx at band width W run reads with at least that many bands in
 * block mode (at most one per CTA, longest first) and the others per warp,
 * instead of abea_set_block_mode's rule; abea_set_block_mode clears the
 * tuning.  Writes one abea_tune_choice per bucket the sample populates (at
 * most cap) and their number to *n_out.  W's without block mode (see
 * abea_set_block_mode) tune to per-warp mode without running it. */
typedef struct {
    int32_t W;
    int32_t min_bands, max_bands;   /* bucket: min_bands <= bands < max_bands (max_bands -1: unbounded) */
    int32_t sample_reads;           /* the sample's reads in the bucket */
    int32_t reads_per_cta;          /* chosen: 4 (per-warp mode) or 1 (block mode) */
    int32_t threads_per_band;       /* chosen: L, or 4 x L' in block mode */
    int32_t record_words;           /* chosen traceback layout: trace words per band */
    float gcups_per_warp;           /* measured on the bucket's sample reads */
    float gcups_block;              /* measured (0: block mode not available) */
} abea_tune_choice;
int abea_autotune(abea_ctx *ctx, int W, int32_t n, const char *seq, const int64_t *seq_off, const float *events,
                  const int64_t *ev_off, const abea_scalings *sc, abea_tune_choice *out, int32_t cap,
                  int32_t *n_out);

/* Serving loop (the paper has no counterpart: it aligns files batch by
 * batch).  Requests (one read each) are admitted one at a time and aligned
 * in micro-batches while earlier ones are still running:
 *
 *   abea_server_start(ctx, &cfg, &srv);
 *   abea_server_submit(srv, &read, &ticket);          (any host thread)
 *   abea_server_poll(srv, ticket, wait_us, &res, pairs, cap, &latency_us);
 *   abea_server_stop(srv);
 *
 * A worker thread closes a micro-batch when it holds max_batch_reads
 * requests or max_wait_us after its first request arrived, whichever comes
 * first (short reads and longer ones batch apart, see short_bases), and runs
 * it on one of batches_in_flight internal contexts (each
 * with its own stream and page-locked staging) on ctx's device, with ctx's
 * model; each internal context gets 1/batches_in_flight of ctx's memory
 * budget, and a micro-batch stays within it.  Results equal those of
 * abea_align for the same read (the kernels do not depend on the batch).
 * ctx must stay alive (and its model unchanged) until abea_server_stop. */
typedef struct abea_server abea_server;
typedef struct {
    int W;                     /* band width of every request (2..256) */
    int32_t max_batch_reads;   /* 0: 256 */
    int32_t max_wait_us;       /* 0: 200; a micro-batch waits at most this long for more requests */
    int32_t batches_in_flight; /* 0: 3 */
    int32_t max_requests;      /* 0: 65536; requests submitted and not yet polled to completion */
    double block_theta;        /* per micro-batch, as abea_set_block_mode (<= 0: off) */
    int32_t short_bases;       /* 0: 1000; reads of at most this many bases queue and batch apart, go
                                  first and may use every context, longer ones leave one context free
                                  for them; < 0: one queue for all */
} abea_server_cfg;

/* Returns ABEA_ERR_NO_MODEL if ctx has no model, ABEA_ERR_ARG for a bad cfg. */
int abea_server_start(abea_ctx *ctx, const abea_server_cfg *cfg, abea_server **out);

/* Copies the read (events, bases, scalings) and queues it; *ticket names it
 * for abea_server_poll.  ABEA_ERR_CAPACITY: max_requests are outstanding
 * (poll some, then retry).  ABEA_ERR_NOMEM: the read alone exceeds an
 * internal context's memory budget.  ABEA_ERR_ARG: bad read or the server
 * is stopping.  Thread-safe. */
int abea_server_submit(abea_server *srv, const abea_read *read, int64_t *ticket);

/* Waits up to wait_us microseconds (0: no wait) for the request to finish.
 * ABEA_OK: *out holds its result, its pairs (out->n_pairs of them, event
 * and k-mer index, ascending) are in pairs[0 .. 2*n_pairs), *latency_us (if
 * not NULL) is the time from submission to the result being in host
 * memory, and the ticket is retired.  ABEA_ERR_TIMEOUT: not finished yet.
 * ABEA_ERR_CAPACITY: finished but cap < out->n_pairs; *out is filled and
 * the ticket stays valid for another poll.  ABEA_ERR_ARG: unknown or
 * retired ticket.  ABEA_ERR_CUDA: its micro-batch failed on the device.
 * Thread-safe; one poller per ticket. */
int abea_server_poll(abea_server *srv, int64_t ticket, int32_t wait_us, abea_result *out, int32_t *pairs,
                     int32_t cap, double *latency_us);

/* Finishes the queued and running requests, stops the worker and frees
 * everything (unpolled results are dropped). */
int abea_server_stop(abea_server *srv);

/* The paper has no counterpart to this call.  abea_align_batch_device without
 * any memory allocation, for callers that cannot call cudaMalloc: for
 * example a plugin inside a host application that already holds (nearly)
 * all device memory in its own pool, or a latency-critical path on which
 * cudaMalloc/cudaFree, which may synchronise the device, are not allowed.
 * No context is needed: the pore model (k <= 7, 4^k host floats each) is
 * passed with every call, and all working memory (model rows, per-read
 * descriptors, k-mer cache, trace) comes from one 64 MiB device array
 * compiled into the library.  A device holds the array from the moment the
 * library's device code is loaded there until the process exits; under
 * CUDA's lazy module loading (the default) that is the first call of this
 * function on the device, so make that first call before the host
 * application fills the device's memory (or set CUDA_MODULE_LOADING=EAGER);
 * if the device has no room for the array then, the call returns
 * ABEA_ERR_NOMEM.  Inputs, outputs, offsets and scalings are as in
 * abea_align_batch_device; the work runs on the current device, on
 * cuda_stream.  The model rows and descriptors are copied from pageable
 * host buffers, which CUDA may stage by first synchronising with the stream:
 * the call can wait for earlier work on its own stream, never for other
 * streams, and returns without waiting for its own kernels.
 * Returns ABEA_ERR_NOMEM, before issuing any work, when n > 16384 or the
 * batch's working set exceeds the 64 MiB array (at W = 100 about 0.33 B per
 * band cell plus 16 B per k-mer and 120 B per read).
 * Every call reuses the same array: calls whose work overlaps on the GPU
 * (different streams) race and must not be made; issue them one after
 * another on one stream.  A lock serialises calls from several host threads.
 * The first call on a device looks up the array's device address, so make it
 * before any stream capture. */
int abea_align_batch_device_noalloc(int k, const float *level_mean, const float *level_stdv,
                                    int32_t n, int W,
                                    const uint8_t *d_seq, const int64_t *seq_off,
                                    const float *d_events, const int64_t *ev_off, const abea_scalings *sc,
                                    abea_result *d_out, int32_t *d_pairs, const int64_t *pair_off,
                                    void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* ABEA_H */
