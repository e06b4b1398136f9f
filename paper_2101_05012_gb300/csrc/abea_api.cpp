// Host side of libabea: the C ABI of include/abea.h.
//
// A batch call (thesis Alg. a:exec and Alg. a:memalloc) serialises the reads
// into flat arrays with per-read offsets (Sec. "Data array serialisation"),
// copies them to the device, runs the pre-kernel (k-mer cache, input checks)
// and the core kernel (band loop, end cell, backtrack), and copies the
// results back.  Device buffers are allocated once per context and reused,
// growing only when a batch needs more (Sec. "Heuristic based memory
// pre-allocation"); when a batch needs more than the context's memory budget
// it is split into waves that reuse the same buffers.  Unlike the thesis,
// no read is sent to the CPU: reads are processed longest first by a
// persistent kernel, which takes the place of the CPU/GPU split of
// Sec. "Heterogeneous processing".
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "abea_internal.h"

using abea::AlignArgs;
using abea::Geometry;
using abea::ModelRow;
using abea::ReadDesc;

namespace {

constexpr double kLogInvSqrt2Pi = -0.91893853320467274178;   // ln(1/sqrt(2 pi))
constexpr double kSqrtHalf = 0.70710678118654752440;         // sqrt(1/2)
constexpr int kMaxTimed = 4096;                              // timed launches kept between stats calls

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct abea_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    size_t budget = 0;
    size_t held = 0;            // bytes of device buffers currently allocated from the pool
    int k = 0;
    DevBuf model, model_f;             // model rows; level mean and stdv as float2
    DevBuf rd, order, flags, kc, trace, moves, queue, offs, ev_meta, ev_bits, ea_meta, ea_ranks;
    DevBuf events, seq, res, pairs;   // staging of the host-memory calls
    HostBuf h_rd, h_order, h_events, h_seq, h_res, h_pairs, h_offs, h_ev_meta, h_ea_meta;
    cudaEvent_t t0 = nullptr, t1 = nullptr, upload_done = nullptr, batch_done = nullptr;
    std::vector<cudaEvent_t> wave_t0, wave_t1;   // one pair per timed core-kernel launch
    int32_t n_timed = 0;                        // pairs recorded since the last stats call
    int32_t last_launches = 0;                  // kernel launches since the last stats call
    std::vector<float> h_mean, h_stdv;          // the model as set (host copy)
    int grid[9][2][2][3] = {};
    double block_theta = abea::kDefaultBlockTheta;   // block mode for reads above theta x the even share
    int tune_W = 0;                             // band width abea_autotune tuned (0: none)
    int64_t tune_block_min_bands = -1;          // tuned: reads with at least this many bands in block mode
    cudaMemPool_t pool = nullptr;               // the working buffers (stream-ordered: growing one never
                                                // synchronises the device)
};

namespace {

int cuda_err(cudaError_t e)
{
    if (e == cudaSuccess) return ABEA_OK;
    cudaGetLastError();
    return ABEA_ERR_CUDA;
}

// Grow a working buffer, in stream order on st (the stream is already ordered
// after every earlier use of the buffer).
int ensure_dev(abea_ctx *c, DevBuf &b, size_t bytes, cudaStream_t st)
{
    if (bytes <= b.cap) return ABEA_OK;
    size_t want = std::max(bytes, b.cap + b.cap / 4);
    want = (want + 255) & ~size_t(255);
    if (b.p) {
        cudaFreeAsync(b.p, st);
        c->held -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    if (cudaMallocFromPoolAsync(&b.p, want, c->pool, st) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMallocFromPoolAsync(&b.p, bytes, c->pool, st) != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return ABEA_ERR_NOMEM;
        }
        want = bytes;
    }
    b.cap = want;
    c->held += want;
    return ABEA_OK;
}

int ensure_host(HostBuf &b, size_t bytes)
{
    if (bytes <= b.cap) return ABEA_OK;
    size_t want = std::max(bytes, b.cap + b.cap / 4);
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    if (cudaMallocHost(&b.p, want) != cudaSuccess) {
        cudaGetLastError();
        return ABEA_ERR_NOMEM;
    }
    b.cap = want;
    return ABEA_OK;
}

// Return a working buffer to the context's pool in stream order on st (no
// device-wide synchronisation, unlike cudaFree).
void free_dev(DevBuf &b, cudaStream_t st)
{
    if (b.p) cudaFreeAsync(b.p, st);
    b.p = nullptr;
    b.cap = 0;
}

void free_host(HostBuf &b)
{
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
}

cudaStream_t pick_stream(abea_ctx *c, void *s) { return s ? (cudaStream_t)s : c->own_stream; }

// Per-read footprint in device memory (k-mer cache entries, trace words, move bytes).
struct Footprint {
    size_t kc, trace, moves;
};

Footprint footprint(int64_t n_e, int64_t n_k, const Geometry &g)
{
    const int64_t bands = n_e + n_k + 1;
    Footprint f;
    f.kc = (size_t)std::max<int64_t>(n_k, 0);
    f.trace = (size_t)(bands * g.rec_words);
    f.moves = g.full ? (size_t)((bands + 15) / 16 * 16) : 0;
    return f;
}

// Build the descriptors of reads `ids` (indices into the caller's arrays).
// ev_base/seq_base: offsets of the first event/base of each read in the
// arrays the kernels will read; pair_base/pair_cap likewise for the pairs.
int plan_reads(const abea_ctx *c, const Geometry &g, const std::vector<int32_t> &ids,
               const int64_t *seq_off, const int64_t *ev_off, const abea_scalings *sc,
               const std::vector<int64_t> &seq_base, const std::vector<int64_t> &ev_base,
               const std::vector<int64_t> &pair_base, const std::vector<int32_t> &pair_cap,
               ReadDesc *rd, int32_t *order, Footprint &total)
{
    total = Footprint{0, 0, 0};
    const size_t n = ids.size();
    for (size_t t = 0; t < n; t++) {
        const int32_t i = ids[t];
        const int64_t n_e = ev_off[i + 1] - ev_off[i];
        const int64_t seq_len = seq_off[i + 1] - seq_off[i];
        const int64_t n_k = seq_len - c->k + 1;
        ReadDesc d;
        std::memset(&d, 0, sizeof(d));
        const abea_scalings s = sc[i];
        bool bad = n_e < 1 || n_k < 1 || n_e > (1LL << 30) || n_k > (1LL << 30) ||
                   !std::isfinite(s.scale) || !std::isfinite(s.shift) || !std::isfinite(s.var) || !(s.var > 0.0f);
        d.ev_off = ev_base[t];
        d.seq_off = seq_base[t];
        d.pair_off = pair_base[t];
        d.pair_cap = pair_cap[t];
        d.host_bad = bad ? 1 : 0;
        if (!bad) {
            d.n_e = (int32_t)n_e;
            d.n_k = (int32_t)n_k;
            // transition constants (thesis Alg. adaptivebandedcpucompute), FP64 then rounded once
            const double epk = (double)n_e / (double)n_k;
            const double lp_skip = std::log(1e-10);
            const double lp_stay = std::log(1.0 - 1.0 / (epk + 1.0));
            const double lp_step = std::log(1.0 - std::exp(lp_skip) - std::exp(lp_stay));
            const double lp_trim = std::log(1.0 / 100.0);
            d.lp_skip = (float)lp_skip;
            d.lp_stay_step = (float)(lp_stay - lp_step);
            d.lp_step = (float)lp_step;
            d.lp_trim = (float)lp_trim;
            d.scale = (double)s.scale;
            d.shift = (double)s.shift;
            d.inv_var = 1.0 / (double)s.var;
            d.log_var_step = std::log((double)s.var) - lp_step;
            const Footprint f = footprint(n_e, n_k, g);
            d.kc_off = (int64_t)total.kc;
            d.tr_off = (int64_t)total.trace;
            d.mv_off = (int64_t)total.moves;
            total.kc += f.kc;
            total.trace += f.trace;
            total.moves += f.moves;
        }
        rd[t] = d;
    }
    // longest reads first; host-rejected reads last
    std::vector<int64_t> key(n);
    for (size_t t = 0; t < n; t++) key[t] = rd[t].host_bad ? -1 : (int64_t)rd[t].n_e + rd[t].n_k;
    std::vector<int32_t> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return key[a] > key[b]; });
    std::memcpy(order, ord.data(), n * sizeof(int32_t));
    return ABEA_OK;
}

// Device bytes one wave of `n` reads holds besides its inputs/outputs.
size_t work_bytes(size_t n, const Footprint &f)
{
    return n * (sizeof(ReadDesc) + 2 * sizeof(int32_t)) + f.kc * 16 + f.trace * 4 + f.moves + 256;
}

// Enqueue prep + align for one planned wave whose descriptors/order are in
// host pinned memory h_rd/h_order and whose inputs/outputs are device arrays.
int run_wave(abea_ctx *c, const Geometry &g, int32_t n, const Footprint &f, const ReadDesc *h_rd,
             const int32_t *h_order, const uint8_t *d_seq, const float *d_events, abea_result *d_res,
             int32_t *d_pairs, int W, cudaStream_t st)
{
    int rc;
    if ((rc = ensure_dev(c, c->rd, (size_t)n * sizeof(ReadDesc), st))) return rc;
    if ((rc = ensure_dev(c, c->order, (size_t)n * sizeof(int32_t), st))) return rc;
    if ((rc = ensure_dev(c, c->flags, (size_t)n * sizeof(int32_t), st))) return rc;
    if ((rc = ensure_dev(c, c->kc, std::max<size_t>(f.kc, 1) * 16, st))) return rc;
    if ((rc = ensure_dev(c, c->trace, std::max<size_t>(f.trace, 4) * 4, st))) return rc;
    if ((rc = ensure_dev(c, c->moves, std::max<size_t>(f.moves, 16), st))) return rc;
    if ((rc = ensure_dev(c, c->queue, 256, st))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->rd.p, h_rd, (size_t)n * sizeof(ReadDesc), cudaMemcpyHostToDevice, st))))
        return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->order.p, h_order, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st))))
        return rc;
    if ((rc = cuda_err(cudaEventRecord(c->upload_done, st)))) return rc;
    if ((rc = cuda_err(cudaMemsetAsync(c->queue.p, 0, sizeof(int32_t), st)))) return rc;
    if ((rc = cuda_err((cudaError_t)abea::launch_prep((const ReadDesc *)c->rd.p, n, d_seq, d_events,
                                                       (const ModelRow *)c->model.p, c->k, (float4 *)c->kc.p,
                                                       (int32_t *)c->flags.p, st))))
        return rc;
    c->last_launches++;
    int &grid = c->grid[g.C][g.mixed ? 1 : 0][g.full ? 1 : 0][g.cg];
    if (grid <= 0) grid = abea::align_grid_size(g, c->device);
    if (grid <= 0) return ABEA_ERR_CUDA;
    int n_group;
    if (c->tune_W == W) {                       // tuned: block mode for the reads of the tuned length buckets
        n_group = 0;
        if (g.cg > 0)
            while (n_group < n && n_group < grid && !h_rd[h_order[n_group]].host_bad &&
                   (int64_t)h_rd[h_order[n_group]].n_e + h_rd[h_order[n_group]].n_k + 1 >= c->tune_block_min_bands)
                n_group++;
    } else {
        n_group = abea::group_count(h_rd, h_order, n, g, grid, c->block_theta);
    }
    AlignArgs a;
    a.rd = (const ReadDesc *)c->rd.p;
    a.order = (const int32_t *)c->order.p;
    a.flags = (const int32_t *)c->flags.p;
    a.n = n;
    a.W = W;
    a.L = g.L;
    a.events = d_events;
    a.seq = d_seq;
    a.kc = (const float4 *)c->kc.p;
    a.trace = (uint32_t *)c->trace.p;
    a.moves = (uint8_t *)c->moves.p;
    a.pairs = d_pairs;
    a.res = d_res;
    a.queue = (int32_t *)c->queue.p;
    a.n_group = n_group;
    const int wave = std::min<int>(c->n_timed, kMaxTimed - 1);   // past the cap the last slot is reused
    while ((int)c->wave_t0.size() <= wave) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return ABEA_ERR_CUDA;
        c->wave_t0.push_back(e0);
        c->wave_t1.push_back(e1);
    }
    if ((rc = cuda_err(cudaEventRecord(c->wave_t0[wave], st)))) return rc;
    const int launch_grid = abea::align_launch_grid(n, n_group, grid);
    if ((rc = cuda_err((cudaError_t)abea::launch_align(a, g, launch_grid, st)))) return rc;
    c->last_launches++;
    if ((rc = cuda_err(cudaEventRecord(c->wave_t1[wave], st)))) return rc;
    if (c->n_timed < kMaxTimed) c->n_timed++;
    return ABEA_OK;
}

int check_common(abea_ctx *c, int W)
{
    if (!c) return ABEA_ERR_ARG;
    if (c->k <= 0) return ABEA_ERR_NO_MODEL;
    if (W < 2 || W > 256) return ABEA_ERR_ARG;
    return ABEA_OK;
}

// Make `st` wait for the previous batch of this context (buffers are reused).
int order_after_previous(abea_ctx *c, cudaStream_t st)
{
    return cuda_err(cudaStreamWaitEvent(st, c->batch_done, 0));
}

bool is_page_locked(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

// One wave whose host buffers are all page-locked: copy straight from and
// to the caller's arrays (no staging copy on the host).
int packed_direct(abea_ctx *c, const Geometry &g, int32_t n, int W, const char *seq, const int64_t *seq_off,
                  const float *events, const int64_t *ev_off, const abea_scalings *sc, abea_result *out,
                  int32_t *pairs, const int64_t *pair_off, cudaStream_t st, bool wait = true)
{
    int rc;
    const int64_t ns = seq_off[n] - seq_off[0], ne = ev_off[n] - ev_off[0], np = pair_off[n] - pair_off[0];
    if ((rc = cuda_err(cudaEventSynchronize(c->upload_done)))) return rc;
    if ((rc = ensure_host(c->h_rd, (size_t)n * sizeof(ReadDesc)))) return rc;
    if ((rc = ensure_host(c->h_order, (size_t)n * sizeof(int32_t)))) return rc;
    std::vector<int32_t> ids(n);
    std::iota(ids.begin(), ids.end(), 0);
    std::vector<int64_t> sb(n), eb(n), pb(n);
    std::vector<int32_t> pc(n);
    for (int32_t i = 0; i < n; i++) {
        sb[i] = seq_off[i] - seq_off[0];
        eb[i] = ev_off[i] - ev_off[0];
        pb[i] = pair_off[i] - pair_off[0];
        pc[i] = (int32_t)(pair_off[i + 1] - pair_off[i]);
    }
    Footprint f;
    plan_reads(c, g, ids, seq_off, ev_off, sc, sb, eb, pb, pc, (ReadDesc *)c->h_rd.p, (int32_t *)c->h_order.p, f);
    if ((rc = ensure_dev(c, c->seq, std::max<int64_t>(ns, 1), st))) return rc;
    if ((rc = ensure_dev(c, c->events, std::max<int64_t>(ne, 1) * 4, st))) return rc;
    if ((rc = ensure_dev(c, c->res, (size_t)n * sizeof(abea_result), st))) return rc;
    if ((rc = ensure_dev(c, c->pairs, std::max<int64_t>(np, 1) * 8, st))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->seq.p, seq + seq_off[0], (size_t)ns, cudaMemcpyHostToDevice, st)))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->events.p, events + ev_off[0], 4 * (size_t)ne, cudaMemcpyHostToDevice, st))))
        return rc;
    rc = run_wave(c, g, n, f, (const ReadDesc *)c->h_rd.p, (const int32_t *)c->h_order.p, (const uint8_t *)c->seq.p,
                  (const float *)c->events.p, (abea_result *)c->res.p, (int32_t *)c->pairs.p, W, st);
    if (rc) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(out, c->res.p, (size_t)n * sizeof(abea_result), cudaMemcpyDeviceToHost, st))))
        return rc;
    if (np > 0 && (rc = cuda_err(cudaMemcpyAsync(pairs + 2 * pair_off[0], c->pairs.p, 8 * (size_t)np,
                                                 cudaMemcpyDeviceToHost, st))))
        return rc;
    if (wait && (rc = cuda_err(cudaStreamSynchronize(st)))) return rc;
    return cuda_err(cudaEventRecord(c->batch_done, st));
}

// Device bytes one read needs in a wave (working set plus its inputs and outputs).
size_t read_bytes(const abea_ctx *c, const Geometry &g, int64_t n_e, int64_t seq_len, int64_t pair_cap)
{
    const int64_t n_k = seq_len - c->k + 1;
    const Footprint f = footprint(std::max<int64_t>(n_e, 0), std::max<int64_t>(n_k, 0), g);
    return work_bytes(1, f) + (size_t)seq_len + 4 * (size_t)std::max<int64_t>(n_e, 0) + 8 * (size_t)pair_cap +
           sizeof(abea_result);
}

// Bounded text output of the TSV writers: writes what fits (always NUL
// terminated when cap > 0) and counts the full length.
struct TextOut {
    char *buf;
    size_t cap;
    size_t len = 0;
    void put(const char *s)
    {
        const size_t l = std::strlen(s);
        if (len < cap) {
            const size_t room = cap - len - 1;
            std::memcpy(buf + len, s, std::min(room, l));
        }
        len += l;
    }
    template <class... A>
    void printf(const char *fmt, A... a)
    {
        char line[512];
        const int l = std::snprintf(line, sizeof(line), fmt, a...);
        if (l > 0) put(line);
    }
    int finish(size_t *needed)
    {
        if (cap > 0) buf[std::min(len, cap - 1)] = '\0';
        *needed = len;
        return len < cap ? ABEA_OK : ABEA_ERR_CAPACITY;
    }
};

// k-mer of lexicographic rank r over ACGT (first base most significant); "NNN.." for a negative rank.
void kmer_text(int32_t r, int k, char *out)
{
    for (int t = k - 1; t >= 0; t--) {
        out[t] = r < 0 ? 'N' : "ACGT"[r & 3];
        if (r >= 0) r >>= 2;
    }
    out[k] = '\0';
}

}  // namespace

extern "C" {

const char *abea_strerror(int code)
{
    switch (code) {
    case ABEA_OK: return "ok";
    case ABEA_ERR_ARG: return "invalid argument";
    case ABEA_ERR_CAPACITY: return "output capacity too small";
    case ABEA_ERR_NOMEM: return "out of memory or memory budget too small";
    case ABEA_ERR_CUDA: return "CUDA runtime error";
    case ABEA_ERR_TIMEOUT: return "bounded device wait timed out";
    case ABEA_ERR_NO_MODEL: return "no pore model set";
    default: return "unknown error";
    }
}

int abea_create(abea_ctx **out, int device, size_t mem_budget_bytes)
{
    if (!out) return ABEA_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return ABEA_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return ABEA_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    abea_ctx *c = new (std::nothrow) abea_ctx();
    if (!c) return ABEA_ERR_NOMEM;
    c->device = device;
    if (cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&c->t0) != cudaSuccess || cudaEventCreate(&c->t1) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->upload_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->batch_done, cudaEventDisableTiming) != cudaSuccess) {
        abea_destroy(c);
        return cuda_err(cudaErrorUnknown);
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        abea_destroy(c);
        return cuda_err(cudaErrorUnknown);
    }
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    uint64_t keep = ~(uint64_t)0;                     // keep freed memory for the next growth
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        cudaGetLastError();
        abea_destroy(c);
        return ABEA_ERR_CUDA;
    }
    c->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)(0.9 * (double)free_b);
    cudaEventRecord(c->batch_done, c->own_stream);
    *out = c;
    return ABEA_OK;
}

void abea_destroy(abea_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    // wait for this context's own work only (its last batch, on whichever stream it ran), never for
    // other contexts or other streams of the device
    if (c->batch_done) cudaEventSynchronize(c->batch_done);
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    DevBuf *dev[] = {&c->model, &c->model_f, &c->rd, &c->order, &c->flags, &c->kc, &c->trace, &c->moves,
                     &c->queue, &c->events, &c->seq, &c->res, &c->pairs, &c->offs, &c->ev_meta, &c->ev_bits,
                     &c->ea_meta, &c->ea_ranks};
    for (DevBuf *b : dev) free_dev(*b, c->own_stream);
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    HostBuf *host[] = {&c->h_rd, &c->h_order, &c->h_events, &c->h_seq, &c->h_res, &c->h_pairs, &c->h_offs,
                       &c->h_ev_meta, &c->h_ea_meta};
    for (HostBuf *b : host) free_host(*b);
    for (cudaEvent_t e : c->wave_t0) cudaEventDestroy(e);
    for (cudaEvent_t e : c->wave_t1) cudaEventDestroy(e);
    if (c->t0) cudaEventDestroy(c->t0);
    if (c->t1) cudaEventDestroy(c->t1);
    if (c->upload_done) cudaEventDestroy(c->upload_done);
    if (c->batch_done) cudaEventDestroy(c->batch_done);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->pool) cudaMemPoolDestroy(c->pool);
    cudaGetLastError();
    delete c;
}

int abea_set_model(abea_ctx *c, int k, const float *level_mean, const float *level_stdv)
{
    if (!c || !level_mean || !level_stdv || k < 1 || k > 12) return ABEA_ERR_ARG;
    const size_t rows = (size_t)1 << (2 * k);
    std::vector<ModelRow> m(rows);
    for (size_t r = 0; r < rows; r++) {
        const float mu = level_mean[r], sd = level_stdv[r];
        if (!std::isfinite(mu) || !std::isfinite(sd) || !(sd > 0.0f)) return ABEA_ERR_ARG;
        m[r].mu = (double)mu;
        m[r].a0 = kSqrtHalf / (double)sd;
        m[r].c0 = kLogInvSqrt2Pi - std::log((double)sd);
        m[r].sd = (double)sd;
    }
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    // The model rows may still be read by this context's last batch (on whichever stream it ran):
    // wait for that batch only, then replace them on the context's own stream.  Nothing here waits
    // for other contexts or streams of the device (no cudaDeviceSynchronize, no cudaFree, no copy
    // on the legacy default stream).
    if (cudaEventSynchronize(c->batch_done) != cudaSuccess) return cuda_err(cudaErrorUnknown);
    cudaStream_t st = c->own_stream;
    std::vector<float2> mf(rows);
    for (size_t r = 0; r < rows; r++) mf[r] = make_float2(level_mean[r], level_stdv[r]);
    int rc;
    if ((rc = ensure_dev(c, c->model, rows * sizeof(ModelRow), st))) return rc;
    if ((rc = ensure_dev(c, c->model_f, rows * sizeof(float2), st))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->model.p, m.data(), rows * sizeof(ModelRow), cudaMemcpyHostToDevice, st))))
        return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->model_f.p, mf.data(), rows * sizeof(float2), cudaMemcpyHostToDevice, st))))
        return rc;
    // the host copies above read m and mf, which go out of scope on return
    if ((rc = cuda_err(cudaStreamSynchronize(st)))) return rc;
    if ((rc = cuda_err(cudaEventRecord(c->batch_done, st)))) return rc;
    c->k = k;
    c->h_mean.assign(level_mean, level_mean + rows);
    c->h_stdv.assign(level_stdv, level_stdv + rows);
    return ABEA_OK;
}

int abea_align_batch_device(abea_ctx *c, int32_t n, int W, const uint8_t *d_seq, const int64_t *seq_off,
                            const float *d_events, const int64_t *ev_off, const abea_scalings *sc,
                            abea_result *d_out, int32_t *d_pairs, const int64_t *pair_off, void *cuda_stream)
{
    int rc = check_common(c, W);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!seq_off || !ev_off || !sc || !pair_off || !d_out))) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    if (!d_seq || !d_events || (!d_pairs && pair_off[n] > 0)) return ABEA_ERR_ARG;
    for (int32_t i = 0; i < n; i++)
        if (seq_off[i + 1] < seq_off[i] || ev_off[i + 1] < ev_off[i] || pair_off[i + 1] < pair_off[i] ||
            pair_off[i + 1] - pair_off[i] > INT32_MAX)
            return ABEA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    const Geometry g = abea::geometry_for(W);
    cudaStream_t st = pick_stream(c, cuda_stream);
    if ((rc = order_after_previous(c, st))) return rc;
    // the pinned descriptor staging may still feed the previous upload
    if ((rc = cuda_err(cudaEventSynchronize(c->upload_done)))) return rc;
    if ((rc = ensure_host(c->h_rd, (size_t)n * sizeof(ReadDesc)))) return rc;
    if ((rc = ensure_host(c->h_order, (size_t)n * sizeof(int32_t)))) return rc;
    std::vector<int32_t> ids(n);
    std::iota(ids.begin(), ids.end(), 0);
    std::vector<int64_t> sb(seq_off, seq_off + n), eb(ev_off, ev_off + n), pb(pair_off, pair_off + n);
    std::vector<int32_t> pc(n);
    for (int32_t i = 0; i < n; i++) pc[i] = (int32_t)(pair_off[i + 1] - pair_off[i]);
    Footprint f;
    plan_reads(c, g, ids, seq_off, ev_off, sc, sb, eb, pb, pc, (ReadDesc *)c->h_rd.p, (int32_t *)c->h_order.p, f);
    if (work_bytes((size_t)n, f) > c->budget) return ABEA_ERR_NOMEM;
    rc = run_wave(c, g, n, f, (const ReadDesc *)c->h_rd.p, (const int32_t *)c->h_order.p, d_seq, d_events, d_out,
                  d_pairs, W, st);
    if (rc) return rc;
    return cuda_err(cudaEventRecord(c->batch_done, st));
}

int abea_align_packed(abea_ctx *c, int32_t n, int W, const char *seq, const int64_t *seq_off, const float *events,
                      const int64_t *ev_off, const abea_scalings *sc, abea_result *out, int32_t *pairs,
                      const int64_t *pair_off, void *cuda_stream)
{
    int rc = check_common(c, W);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!seq || !seq_off || !events || !ev_off || !sc || !out || !pair_off))) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    if (!pairs && pair_off[n] > pair_off[0]) return ABEA_ERR_ARG;
    for (int32_t i = 0; i < n; i++)
        if (seq_off[i + 1] < seq_off[i] || ev_off[i + 1] < ev_off[i] || pair_off[i + 1] < pair_off[i] ||
            pair_off[i + 1] - pair_off[i] > INT32_MAX)
            return ABEA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    const Geometry g = abea::geometry_for(W);
    cudaStream_t st = pick_stream(c, cuda_stream);
    if ((rc = order_after_previous(c, st))) return rc;

    // waves: reads in decreasing length, each wave within the memory budget
    std::vector<int32_t> all(n);
    std::iota(all.begin(), all.end(), 0);
    auto len = [&](int32_t i) { return (ev_off[i + 1] - ev_off[i]) + (seq_off[i + 1] - seq_off[i]); };
    std::stable_sort(all.begin(), all.end(), [&](int32_t a, int32_t b) { return len(a) > len(b); });
    std::vector<std::vector<int32_t>> waves;
    {
        std::vector<int32_t> cur;
        size_t cur_bytes = 0;
        for (int32_t i : all) {
            const size_t bytes = read_bytes(c, g, ev_off[i + 1] - ev_off[i], seq_off[i + 1] - seq_off[i],
                                            pair_off[i + 1] - pair_off[i]);
            if (bytes > c->budget) return ABEA_ERR_NOMEM;
            if (!cur.empty() && cur_bytes + bytes > c->budget) {
                waves.push_back(cur);
                cur.clear();
                cur_bytes = 0;
            }
            cur.push_back(i);
            cur_bytes += bytes;
        }
        if (!cur.empty()) waves.push_back(cur);
    }
    if (waves.size() == 1 && is_page_locked(seq) && is_page_locked(events) && is_page_locked(out) &&
        (pair_off[n] == pair_off[0] || is_page_locked(pairs)))
        return packed_direct(c, g, n, W, seq, seq_off, events, ev_off, sc, out, pairs, pair_off, st);
    for (const std::vector<int32_t> &ids : waves) {
        const int32_t m = (int32_t)ids.size();
        // gather the wave's inputs into pinned staging
        std::vector<int64_t> sb(m), eb(m), pb(m);
        std::vector<int32_t> pc(m);
        int64_t ns = 0, ne = 0, np = 0;
        for (int32_t t = 0; t < m; t++) {
            const int32_t i = ids[t];
            sb[t] = ns;
            eb[t] = ne;
            pb[t] = np;
            pc[t] = (int32_t)(pair_off[i + 1] - pair_off[i]);
            ns += seq_off[i + 1] - seq_off[i];
            ne += ev_off[i + 1] - ev_off[i];
            np += pc[t];
        }
        if ((rc = cuda_err(cudaEventSynchronize(c->upload_done)))) return rc;
        if ((rc = ensure_host(c->h_seq, std::max<int64_t>(ns, 1)))) return rc;
        if ((rc = ensure_host(c->h_events, std::max<int64_t>(ne, 1) * 4))) return rc;
        if ((rc = ensure_host(c->h_rd, (size_t)m * sizeof(ReadDesc)))) return rc;
        if ((rc = ensure_host(c->h_order, (size_t)m * sizeof(int32_t)))) return rc;
        if ((rc = ensure_host(c->h_res, (size_t)m * sizeof(abea_result)))) return rc;
        if ((rc = ensure_host(c->h_pairs, std::max<int64_t>(np, 1) * 8))) return rc;
        for (int32_t t = 0; t < m; t++) {
            const int32_t i = ids[t];
            std::memcpy((char *)c->h_seq.p + sb[t], seq + seq_off[i], (size_t)(seq_off[i + 1] - seq_off[i]));
            std::memcpy((float *)c->h_events.p + eb[t], events + ev_off[i], 4 * (size_t)(ev_off[i + 1] - ev_off[i]));
        }
        std::vector<int64_t> s_off(m + 1), e_off(m + 1);
        std::vector<abea_scalings> wsc(m);
        for (int32_t t = 0; t < m; t++) {
            s_off[t] = sb[t];
            e_off[t] = eb[t];
            wsc[t] = sc[ids[t]];
        }
        s_off[m] = ns;
        e_off[m] = ne;
        std::vector<int32_t> loc(m);
        std::iota(loc.begin(), loc.end(), 0);
        Footprint f;
        plan_reads(c, g, loc, s_off.data(), e_off.data(), wsc.data(), sb, eb, pb, pc, (ReadDesc *)c->h_rd.p,
                   (int32_t *)c->h_order.p, f);
        if ((rc = ensure_dev(c, c->seq, std::max<int64_t>(ns, 1), st))) return rc;
        if ((rc = ensure_dev(c, c->events, std::max<int64_t>(ne, 1) * 4, st))) return rc;
        if ((rc = ensure_dev(c, c->res, (size_t)m * sizeof(abea_result), st))) return rc;
        if ((rc = ensure_dev(c, c->pairs, std::max<int64_t>(np, 1) * 8, st))) return rc;
        if ((rc = cuda_err(cudaMemcpyAsync(c->seq.p, c->h_seq.p, (size_t)ns, cudaMemcpyHostToDevice, st)))) return rc;
        if ((rc = cuda_err(cudaMemcpyAsync(c->events.p, c->h_events.p, 4 * (size_t)ne, cudaMemcpyHostToDevice, st))))
            return rc;
        rc = run_wave(c, g, m, f, (const ReadDesc *)c->h_rd.p, (const int32_t *)c->h_order.p,
                      (const uint8_t *)c->seq.p, (const float *)c->events.p, (abea_result *)c->res.p,
                      (int32_t *)c->pairs.p, W, st);
        if (rc) return rc;
        if ((rc = cuda_err(cudaMemcpyAsync(c->h_res.p, c->res.p, (size_t)m * sizeof(abea_result),
                                           cudaMemcpyDeviceToHost, st))))
            return rc;
        if (np > 0 && (rc = cuda_err(cudaMemcpyAsync(c->h_pairs.p, c->pairs.p, 8 * (size_t)np,
                                                     cudaMemcpyDeviceToHost, st))))
            return rc;
        if ((rc = cuda_err(cudaStreamSynchronize(st)))) return rc;
        const abea_result *hr = (const abea_result *)c->h_res.p;
        for (int32_t t = 0; t < m; t++) {
            const int32_t i = ids[t];
            out[i] = hr[t];
            const int32_t cnt = std::min<int32_t>(hr[t].n_pairs, pc[t]);
            if (hr[t].status == ABEA_READ_OK && cnt > 0)
                std::memcpy(pairs + 2 * pair_off[i], (const int32_t *)c->h_pairs.p + 2 * pb[t], 8 * (size_t)cnt);
        }
    }
    return cuda_err(cudaEventRecord(c->batch_done, st));
}

int abea_align_batch(abea_ctx *c, const abea_read *reads, int32_t n, int W, abea_result *out, int32_t *pairs,
                     const int64_t *pair_off, void *cuda_stream)
{
    if (!c || n < 0 || (n > 0 && (!reads || !out || !pair_off))) return ABEA_ERR_ARG;
    std::vector<int64_t> so(n + 1, 0), eo(n + 1, 0);
    for (int32_t i = 0; i < n; i++) {
        if (reads[i].n_events < 0 || reads[i].seq_len < 0) return ABEA_ERR_ARG;
        if ((reads[i].n_events > 0 && !reads[i].ev_mean) || (reads[i].seq_len > 0 && !reads[i].seq)) return ABEA_ERR_ARG;
        so[i + 1] = so[i] + reads[i].seq_len;
        eo[i + 1] = eo[i] + reads[i].n_events;
    }
    std::vector<char> s((size_t)std::max<int64_t>(so[n], 1));
    std::vector<float> e((size_t)std::max<int64_t>(eo[n], 1));
    std::vector<abea_scalings> sc(std::max<int32_t>(n, 1));
    for (int32_t i = 0; i < n; i++) {
        if (reads[i].seq_len) std::memcpy(s.data() + so[i], reads[i].seq, (size_t)reads[i].seq_len);
        if (reads[i].n_events) std::memcpy(e.data() + eo[i], reads[i].ev_mean, 4 * (size_t)reads[i].n_events);
        sc[i] = reads[i].sc;
    }
    return abea_align_packed(c, n, W, s.data(), so.data(), e.data(), eo.data(), sc.data(), out, pairs, pair_off,
                             cuda_stream);
}

int abea_align(abea_ctx *c, const abea_read *read, int W, abea_result *out, int32_t *pairs, int32_t cap)
{
    if (!c || !read || !out || cap < 0 || (cap > 0 && !pairs)) return ABEA_ERR_ARG;
    const int64_t po[2] = {0, cap};
    int rc = abea_align_batch(c, read, 1, W, out, pairs, po, nullptr);
    if (rc) return rc;
    if (out->status == ABEA_READ_CAPACITY) return ABEA_ERR_CAPACITY;
    return ABEA_OK;
}

int abea_eventalign(abea_ctx *c, int32_t n, const uint8_t *d_seq, const int64_t *seq_off, const float *d_events,
                    const int64_t *ev_off, const abea_scalings *sc, const abea_result *d_results,
                    const int32_t *d_pairs, const int64_t *pair_off, const int32_t *d_ref_pos, const uint8_t *d_ref,
                    int64_t ref_len, int scale_events, abea_eventalign_row *d_rows, void *cuda_stream)
{
    if (!c) return ABEA_ERR_ARG;
    if (c->k <= 0) return ABEA_ERR_NO_MODEL;
    if (n < 0 || ref_len < 0) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    if (!d_seq || !seq_off || !d_events || !ev_off || !sc || !d_results || !d_pairs || !pair_off || !d_ref_pos ||
        (!d_ref && ref_len > 0) || !d_rows)
        return ABEA_ERR_ARG;
    for (int32_t i = 0; i < n; i++)
        if (seq_off[i + 1] < seq_off[i] || ev_off[i + 1] < ev_off[i] || pair_off[i + 1] < pair_off[i] ||
            !(sc[i].scale != 0.0f) || !std::isfinite(sc[i].scale))
            return ABEA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    cudaStream_t st = pick_stream(c, cuda_stream);
    int rc;
    if ((rc = order_after_previous(c, st))) return rc;
    const size_t m = (size_t)(n + 1);
    const size_t bytes = 3 * m * sizeof(int64_t) + (size_t)n * sizeof(abea_scalings);
    if ((rc = cuda_err(cudaEventSynchronize(c->upload_done)))) return rc;
    if ((rc = ensure_host(c->h_ea_meta, bytes))) return rc;
    int64_t *h = (int64_t *)c->h_ea_meta.p;
    std::memcpy(h, seq_off, m * sizeof(int64_t));
    std::memcpy(h + m, ev_off, m * sizeof(int64_t));
    std::memcpy(h + 2 * m, pair_off, m * sizeof(int64_t));
    std::memcpy(h + 3 * m, sc, (size_t)n * sizeof(abea_scalings));
    if ((rc = ensure_dev(c, c->ea_meta, bytes, st))) return rc;
    if ((rc = ensure_dev(c, c->ea_ranks, std::max<int64_t>(seq_off[n] - seq_off[0], 1) * sizeof(int2), st))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->ea_meta.p, h, bytes, cudaMemcpyHostToDevice, st)))) return rc;
    if ((rc = cuda_err(cudaEventRecord(c->upload_done, st)))) return rc;
    const int64_t *d_meta = (const int64_t *)c->ea_meta.p;
    if ((rc = cuda_err((cudaError_t)abea::launch_eventalign(
             d_meta, n, pair_off[n] - pair_off[0], d_seq, seq_off[0], seq_off[n], (int2 *)c->ea_ranks.p, d_events,
             (const abea_scalings *)(d_meta + 3 * m), d_results, d_pairs, d_ref_pos, d_ref, ref_len,
             (const float2 *)c->model_f.p, c->k, scale_events ? 1 : 0, d_rows, st))))
        return rc;
    c->last_launches += 2;
    return cuda_err(cudaEventRecord(c->batch_done, st));
}

int abea_summarise(abea_ctx *c, int32_t n, const int64_t *seq_off, const int64_t *ev_off,
                   const abea_result *d_results, const int32_t *d_pairs, const int64_t *pair_off,
                   abea_read_summary *d_out, void *cuda_stream)
{
    if (!c) return ABEA_ERR_ARG;
    if (c->k <= 0) return ABEA_ERR_NO_MODEL;
    if (n < 0) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    if (!seq_off || !ev_off || !pair_off || !d_results || !d_out || (!d_pairs && pair_off[n] > pair_off[0]))
        return ABEA_ERR_ARG;
    for (int32_t i = 0; i < n; i++)
        if (seq_off[i + 1] < seq_off[i] || ev_off[i + 1] < ev_off[i] || pair_off[i + 1] < pair_off[i])
            return ABEA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    cudaStream_t st = pick_stream(c, cuda_stream);
    int rc;
    if ((rc = order_after_previous(c, st))) return rc;
    const size_t m = (size_t)(n + 1);
    const size_t bytes = 3 * m * sizeof(int64_t);
    if ((rc = cuda_err(cudaEventSynchronize(c->upload_done)))) return rc;
    if ((rc = ensure_host(c->h_ea_meta, bytes))) return rc;
    int64_t *h = (int64_t *)c->h_ea_meta.p;
    std::memcpy(h, seq_off, m * sizeof(int64_t));
    std::memcpy(h + m, ev_off, m * sizeof(int64_t));
    std::memcpy(h + 2 * m, pair_off, m * sizeof(int64_t));
    if ((rc = ensure_dev(c, c->ea_meta, bytes, st))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->ea_meta.p, h, bytes, cudaMemcpyHostToDevice, st)))) return rc;
    if ((rc = cuda_err(cudaEventRecord(c->upload_done, st)))) return rc;
    if ((rc = cuda_err((cudaError_t)abea::launch_summary((const int64_t *)c->ea_meta.p, n, c->k, d_results, d_pairs,
                                                          d_out, st))))
        return rc;
    c->last_launches++;
    return cuda_err(cudaEventRecord(c->batch_done, st));
}

int abea_eventalign_tsv(const abea_eventalign_row *rows, int64_t n_rows, int k, int header, char *buf, size_t cap,
                        size_t *needed)
{
    if (n_rows < 0 || k < 1 || k > 15 || (n_rows > 0 && !rows) || (cap > 0 && !buf) || !needed) return ABEA_ERR_ARG;
    TextOut o{buf, cap};
    if (header) o.put("read\tevent\tkmer\tref_pos\tref_kmer\tmodel_kmer\tlevel\tmodel_mean\tmodel_stdv\tz\n");
    char rk[16], mk[16];
    for (int64_t t = 0; t < n_rows; t++) {
        const abea_eventalign_row &r = rows[t];
        kmer_text(r.ref_rank, k, rk);
        kmer_text(r.model_rank, k, mk);
        o.printf("%d\t%d\t%d\t%d\t%s\t%s\t%.2f\t%.2f\t%.2f\t%.3f\n", r.read, r.event, r.kmer, r.ref_pos, rk, mk,
                 (double)r.level, (double)r.model_mean, (double)r.model_stdv, (double)r.z);
    }
    return o.finish(needed);
}

int abea_summary_tsv(const abea_read_summary *s, int32_t n, int header, char *buf, size_t cap, size_t *needed)
{
    if (n < 0 || (n > 0 && !s) || (cap > 0 && !buf) || !needed) return ABEA_ERR_ARG;
    TextOut o{buf, cap};
    if (header)
        o.put("read\tstatus\tn_events\tn_kmers\tn_pairs\tfirst_event\tlast_event\tevents_aligned\tstays\tskips"
              "\tscore\tscore_per_event\tflags\n");
    for (int32_t i = 0; i < n; i++) {
        const abea_read_summary &r = s[i];
        o.printf("%d\t%d\t%d\t%d\t%d\t%d\t%d\t%d\t%d\t%d\t%.3f\t%.3f\t%d\n", r.read, r.status, r.n_events,
                 r.n_kmers, r.n_pairs, r.first_event, r.last_event, r.events_aligned, r.stays, r.skips,
                 (double)r.score, (double)r.score_per_event, r.flags);
    }
    return o.finish(needed);
}

int abea_detect_events(abea_ctx *c, int32_t n, const int16_t *d_raw, const int64_t *raw_off,
                       const abea_calib *calib, int window, float tau2, abea_event *d_events,
                       const int64_t *event_off, int32_t *d_n_events, void *cuda_stream)
{
    if (!c) return ABEA_ERR_ARG;
    if (n < 0 || window < 2 || window > 8 || !std::isfinite(tau2) || tau2 < 0.0f) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    if (!d_raw || !raw_off || !calib || !event_off || !d_n_events || (!d_events && event_off[n] > event_off[0]))
        return ABEA_ERR_ARG;
    for (int32_t i = 0; i < n; i++)
        if (raw_off[i + 1] < raw_off[i] || raw_off[i + 1] - raw_off[i] > INT32_MAX / 2 ||
            event_off[i + 1] < event_off[i] || !std::isfinite(calib[i].offset) || !std::isfinite(calib[i].pa_per_unit))
            return ABEA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    cudaStream_t st = pick_stream(c, cuda_stream);
    int rc;
    if ((rc = order_after_previous(c, st))) return rc;
    // the reads' positions in tiles of kEventTile (ceil(len / kEventTile) per read); the metadata
    // holds the offsets of samples, events and tiles, the calibrations and each tile's read
    const size_t m = (size_t)(n + 1);
    int64_t n_tiles = 0;
    for (int32_t i = 0; i < n; i++) n_tiles += (raw_off[i + 1] - raw_off[i] + abea::kEventTile - 1) / abea::kEventTile;
    if (n_tiles > INT32_MAX) return ABEA_ERR_ARG;
    const size_t meta_bytes = 3 * m * sizeof(int64_t) + (size_t)n * sizeof(abea_calib) + (size_t)n_tiles * 4;
    if ((rc = cuda_err(cudaEventSynchronize(c->upload_done)))) return rc;
    if ((rc = ensure_host(c->h_ev_meta, meta_bytes))) return rc;
    int64_t *h_raw_off = (int64_t *)c->h_ev_meta.p, *h_ev_off = h_raw_off + m, *h_tile_off = h_ev_off + m;
    abea_calib *h_cal = (abea_calib *)(h_tile_off + m);
    int32_t *h_tile_read = (int32_t *)(h_cal + n);
    h_tile_off[0] = 0;
    for (int32_t i = 0; i < n; i++) {
        const int64_t tiles = (raw_off[i + 1] - raw_off[i] + abea::kEventTile - 1) / abea::kEventTile;
        h_raw_off[i] = raw_off[i] - raw_off[0];
        h_ev_off[i] = event_off[i] - event_off[0];
        h_tile_off[i + 1] = h_tile_off[i] + tiles;
        for (int64_t t = h_tile_off[i]; t < h_tile_off[i + 1]; t++) h_tile_read[t] = i;
        h_cal[i] = calib[i];
    }
    h_raw_off[n] = raw_off[n] - raw_off[0];
    h_ev_off[n] = event_off[n] - event_off[0];
    if ((rc = ensure_dev(c, c->ev_meta, meta_bytes, st))) return rc;
    if ((rc = ensure_dev(c, c->ev_bits, std::max<int64_t>(n_tiles, 1) * abea::event_tile_bytes(), st))) return rc;
    if ((rc = cuda_err(cudaMemcpyAsync(c->ev_meta.p, h_raw_off, meta_bytes, cudaMemcpyHostToDevice, st)))) return rc;
    if ((rc = cuda_err(cudaEventRecord(c->upload_done, st)))) return rc;
    const int64_t *d_meta = (const int64_t *)c->ev_meta.p;
    const abea_calib *d_cal = (const abea_calib *)(d_meta + 3 * m);
    if ((rc = cuda_err((cudaError_t)abea::launch_events(d_meta, d_meta + m, d_meta + 2 * m,
                                                         (const int32_t *)(d_cal + n), n, n_tiles,
                                                         d_raw + raw_off[0], d_cal, window, tau2, c->ev_bits.p,
                                                         d_events + event_off[0], d_n_events, st))))
        return rc;
    c->last_launches += n_tiles > 0 ? 3 : 1;
    return cuda_err(cudaEventRecord(c->batch_done, st));
}

int abea_f32_from_i64(const int64_t *d_in, int64_t n, float *d_out, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!d_in || !d_out))) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    return cuda_err((cudaError_t)abea::launch_f32_from_i64(d_in, n, d_out, cuda_stream));
}

int abea_f32_from_f64(const double *d_in, int64_t n, float *d_out, void *cuda_stream)
{
    if (n < 0 || (n > 0 && (!d_in || !d_out))) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    return cuda_err((cudaError_t)abea::launch_f32_from_f64(d_in, n, d_out, cuda_stream));
}

int abea_estimate_scalings(abea_ctx *c, int32_t n, const uint8_t *d_seq, const int64_t *seq_off,
                           const float *d_events, const int64_t *ev_off, abea_scalings *d_out, int32_t *d_status,
                           void *cuda_stream)
{
    if (!c) return ABEA_ERR_ARG;
    if (c->k <= 0) return ABEA_ERR_NO_MODEL;
    if (n < 0 || (n > 0 && (!seq_off || !ev_off || !d_out || !d_status || !d_seq || !d_events))) return ABEA_ERR_ARG;
    if (n == 0) return ABEA_OK;
    for (int32_t i = 0; i < n; i++)
        if (seq_off[i + 1] < seq_off[i] || ev_off[i + 1] < ev_off[i] || seq_off[i + 1] - seq_off[i] > INT32_MAX ||
            ev_off[i + 1] - ev_off[i] > INT32_MAX)
            return ABEA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    cudaStream_t st = pick_stream(c, cuda_stream);
    int rc;
    if ((rc = order_after_previous(c, st))) return rc;
    // the offsets go through page-locked staging (free once its previous upload is done)
    if ((rc = cuda_err(cudaEventSynchronize(c->upload_done)))) return rc;
    const size_t bytes = 2 * (size_t)(n + 1) * sizeof(int64_t);
    if ((rc = ensure_host(c->h_offs, bytes))) return rc;
    if ((rc = ensure_dev(c, c->offs, bytes, st))) return rc;
    int64_t *h = (int64_t *)c->h_offs.p;
    std::memcpy(h, seq_off, (size_t)(n + 1) * sizeof(int64_t));
    std::memcpy(h + n + 1, ev_off, (size_t)(n + 1) * sizeof(int64_t));
    if ((rc = cuda_err(cudaMemcpyAsync(c->offs.p, h, bytes, cudaMemcpyHostToDevice, st)))) return rc;
    if ((rc = cuda_err(cudaEventRecord(c->upload_done, st)))) return rc;
    const int64_t *d_off = (const int64_t *)c->offs.p;
    if ((rc = cuda_err((cudaError_t)abea::launch_scalings(d_off, d_off + n + 1, n, d_seq, d_events,
                                                           (const float2 *)c->model_f.p, c->k, d_out, d_status,
                                                           st))))
        return rc;
    c->last_launches++;
    return cuda_err(cudaEventRecord(c->batch_done, st));
}

int abea_set_block_mode(abea_ctx *c, double theta)
{
    if (!c || std::isnan(theta)) return ABEA_ERR_ARG;
    c->block_theta = theta;
    c->tune_W = 0;
    return ABEA_OK;
}

int abea_autotune(abea_ctx *c, int W, int32_t n, const char *seq, const int64_t *seq_off, const float *events,
                  const int64_t *ev_off, const abea_scalings *sc, abea_tune_choice *out, int32_t cap, int32_t *n_out)
{
    int rc = check_common(c, W);
    if (rc) return rc;
    if (n < 0 || (n > 0 && (!seq || !seq_off || !events || !ev_off || !sc)) || cap < 0 || (cap > 0 && !out) || !n_out)
        return ABEA_ERR_ARG;
    *n_out = 0;
    const Geometry g = abea::geometry_for(W);
    const int64_t bounds[5] = {0, 4096, 16384, 65536, INT64_MAX};
    const double saved_theta = c->block_theta;
    c->tune_W = 0;                              // time the two modes, not the old choice
    bool block_wins[4] = {false, false, false, false};
    bool populated[4] = {false, false, false, false};
    int32_t n_choices = 0;
    for (int bk = 0; bk < 4; bk++) {
        // the bucket's sample reads, packed
        std::vector<char> s;
        std::vector<float> e;
        std::vector<int64_t> so(1, 0), eo(1, 0), po(1, 0);
        std::vector<abea_scalings> sv;
        for (int32_t i = 0; i < n; i++) {
            const int64_t ne = ev_off[i + 1] - ev_off[i], nb = seq_off[i + 1] - seq_off[i];
            const int64_t bands = ne + (nb - c->k + 1) + 1;
            if (ne < 1 || nb < c->k || bands < bounds[bk] || bands >= bounds[bk + 1]) continue;
            s.insert(s.end(), seq + seq_off[i], seq + seq_off[i + 1]);
            e.insert(e.end(), events + ev_off[i], events + ev_off[i + 1]);
            so.push_back((int64_t)s.size());
            eo.push_back((int64_t)e.size());
            po.push_back(po.back() + ne + (nb - c->k + 1));
            sv.push_back(sc[i]);
        }
        const int32_t m = (int32_t)sv.size();
        if (m == 0) continue;
        populated[bk] = true;
        std::vector<abea_result> res(m);
        std::vector<int32_t> pairs((size_t)std::max<int64_t>(po.back(), 1) * 2);
        float rate[2] = {0.0f, 0.0f};
        for (int mode = 0; mode < 2; mode++) {
            if (mode == 1 && g.cg == 0) break;
            c->block_theta = mode == 0 ? 0.0 : 1e-300;   // 1e-300: every read above any share (one per CTA)
            float best = 0.0f;
            for (int rep = 0; rep < 3; rep++) {
                abea_last_launch_stats(c, nullptr, nullptr);
                if ((rc = abea_align_packed(c, m, W, s.data(), so.data(), e.data(), eo.data(), sv.data(), res.data(),
                                            pairs.data(), po.data(), nullptr))) {
                    c->block_theta = saved_theta;
                    return rc;
                }
                float ms = 0.0f;
                if ((rc = abea_last_launch_stats(c, nullptr, &ms))) {
                    c->block_theta = saved_theta;
                    return rc;
                }
                double cells = 0.0;
                for (int32_t t = 0; t < m; t++) cells += (double)res[t].cells;
                const float gcups = ms > 0.0f ? (float)(cells / ((double)ms * 1e6)) : 0.0f;
                if (rep > 0) best = std::max(best, gcups);   // rep 0 warms up
            }
            rate[mode] = best;
        }
        block_wins[bk] = g.cg > 0 && rate[1] > rate[0];
        if (n_choices < cap) {
            abea_tune_choice &o = out[n_choices];
            o.W = W;
            o.min_bands = (int32_t)bounds[bk];
            o.max_bands = bk == 3 ? -1 : (int32_t)bounds[bk + 1];
            o.sample_reads = m;
            o.reads_per_cta = block_wins[bk] ? 1 : 4;
            o.threads_per_band = block_wins[bk] ? (W / 4 / std::max(g.cg, 1)) * 4 : g.L;
            o.record_words = g.rec_words;
            o.gcups_per_warp = rate[0];
            o.gcups_block = rate[1];
        }
        n_choices++;
    }
    // block mode from the shortest populated bucket upward where it keeps winning
    int64_t min_bands = INT64_MAX;
    for (int bk = 3; bk >= 0; bk--) {
        if (!populated[bk]) continue;
        if (!block_wins[bk]) break;
        min_bands = bounds[bk];
    }
    for (int32_t t = 0; t < std::min(n_choices, cap); t++) {   // report what later batches will do
        const bool blk = out[t].min_bands >= min_bands;
        out[t].reads_per_cta = blk ? 1 : 4;
        out[t].threads_per_band = blk ? (W / 4 / std::max(g.cg, 1)) * 4 : g.L;
    }
    c->block_theta = saved_theta;
    c->tune_W = W;
    c->tune_block_min_bands = min_bands;
    *n_out = std::min(n_choices, cap);
    return ABEA_OK;
}

int abea_last_launch_stats(abea_ctx *c, int32_t *n_launches, float *align_kernel_ms)
{
    if (!c) return ABEA_ERR_ARG;
    float total = 0.0f;
    int rc = ABEA_OK;
    for (int w = 0; w < c->n_timed; w++) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(c->wave_t1[w]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, c->wave_t0[w], c->wave_t1[w]);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = ABEA_ERR_CUDA;
            break;
        }
        total += ms;
    }
    if (n_launches) *n_launches = c->last_launches;
    if (align_kernel_ms) *align_kernel_ms = total;
    c->n_timed = 0;
    c->last_launches = 0;
    return rc;
}

}  // extern "C"

// Internal entry points of the serving loop (abea_internal.h).
namespace abea {

int context_model(const abea_ctx *c, int *k, const float **mean, const float **stdv)
{
    if (!c || c->k <= 0) return ABEA_ERR_NO_MODEL;
    *k = c->k;
    *mean = c->h_mean.data();
    *stdv = c->h_stdv.data();
    return ABEA_OK;
}

int context_device(const abea_ctx *c) { return c->device; }

size_t context_budget(const abea_ctx *c) { return c->budget; }

void *context_stream(const abea_ctx *c) { return (void *)c->own_stream; }

size_t request_bytes(const abea_ctx *c, int W, int64_t n_e, int64_t seq_len, int64_t pair_cap)
{
    return read_bytes(c, geometry_for(W), n_e, seq_len, pair_cap);
}

int align_packed_async(abea_ctx *c, int32_t n, int W, const char *seq, const int64_t *seq_off, const float *events,
                       const int64_t *ev_off, const abea_scalings *sc, abea_result *out, int32_t *pairs,
                       const int64_t *pair_off)
{
    int rc = check_common(c, W);
    if (rc) return rc;
    if (n <= 0 || !seq || !seq_off || !events || !ev_off || !sc || !out || !pair_off || !pairs) return ABEA_ERR_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_err(cudaErrorInvalidDevice);
    const Geometry g = geometry_for(W);
    size_t bytes = 0;
    for (int32_t i = 0; i < n; i++)
        bytes += read_bytes(c, g, ev_off[i + 1] - ev_off[i], seq_off[i + 1] - seq_off[i], pair_off[i + 1] - pair_off[i]);
    if (bytes > c->budget) return ABEA_ERR_NOMEM;
    cudaStream_t st = c->own_stream;
    if ((rc = order_after_previous(c, st))) return rc;
    return packed_direct(c, g, n, W, seq, seq_off, events, ev_off, sc, out, pairs, pair_off, st, false);
}

}  // namespace abea
