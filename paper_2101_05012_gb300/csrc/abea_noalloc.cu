// abea_align_batch_device_noalloc: the batch alignment of
// abea_align_batch_device, for callers that must not allocate memory.
//
// Who needs it: code that cannot call cudaMalloc, for example a plugin
// running inside a host application that has already reserved (nearly) all
// device memory in its own pool, or a latency-critical path on which
// cudaMalloc/cudaFree, which may synchronise the device, are not allowed.
// Such a caller passes its inputs and outputs as before; everything else the
// kernels need lives in one file-scope device array of fixed size
// (kScratchBytes), held on a device from the moment the library's device
// code is loaded there until the process exits.  With CUDA's lazy module
// loading (the default since CUDA 12.2) that moment is the first call of
// this function on the device, whose symbol lookup loads the module: make
// that first call before the host application fills its memory pool (or set
// CUDA_MODULE_LOADING=EAGER, which loads it with the library).  If the
// device has no room left for the array then, the call fails with
// ABEA_ERR_NOMEM.  The host side uses only static buffers as well.
//
// Limits and sharing: the scratch holds the model rows, the per-read
// descriptors and the kernels' working set (k-mer cache and trace, about
// 0.33 B per band cell at W = 100); a batch that does not fit is rejected
// with ABEA_ERR_NOMEM before any work is issued.  Every call uses the same
// array and leaves its contents behind; the call clears what must start at
// zero.  Calls whose work overlaps on the GPU (two streams, or two host
// threads issuing on different streams) race on the array: issue them one
// after another on one stream.  On the host, a lock serialises the calls
// (the static host buffers are filled under it), so entering from two host
// threads is safe as such; only the device array is shared.  The model rows,
// descriptors and order are copied from those pageable static buffers; CUDA
// may stage such a copy by first synchronising with the stream, so the call
// can wait for earlier work on its own stream (never for other streams).
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (with that device current), so make that first call
// before any stream capture.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "abea_internal.h"

using abea::AlignArgs;
using abea::Geometry;
using abea::ModelRow;
using abea::ReadDesc;

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;   // 64 MiB of device scratch per GPU
constexpr int kMaxReads = 16384;                     // reads per call
constexpr int kMaxK = 7;                             // model rows: 4^7 at most
constexpr int kMaxDevices = 64;
constexpr double kLogInvSqrt2Pi = -0.91893853320467274178;   // ln(1/sqrt(2 pi))
constexpr double kSqrtHalf = 0.70710678118654752440;         // sqrt(1/2)

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host-side buffers (static: no heap allocation on this path).
ModelRow s_rows[size_t(1) << (2 * kMaxK)];
ReadDesc s_desc[kMaxReads];
int32_t s_order[kMaxReads];
int64_t s_key[kMaxReads];
unsigned char *s_scratch[kMaxDevices];               // device address of g_scratch, per device
int s_grid[kMaxDevices][9][2][2][3];
std::mutex s_setup;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on `device` (current), looked up once.
// On failure *no_room tells whether the device had no memory left for it.
unsigned char *scratch_for(int device, bool *no_room)
{
    *no_room = false;
    std::lock_guard<std::mutex> lock(s_setup);
    if (!s_scratch[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *no_room = e == cudaErrorMemoryAllocation;
            return nullptr;
        }
        s_scratch[device] = (unsigned char *)p;
    }
    return s_scratch[device];
}

}  // namespace

extern "C" int abea_align_batch_device_noalloc(int k, const float *level_mean, const float *level_stdv,
                                               int32_t n, int W, const uint8_t *d_seq, const int64_t *seq_off,
                                               const float *d_events, const int64_t *ev_off,
                                               const abea_scalings *sc, abea_result *d_out, int32_t *d_pairs,
                                               const int64_t *pair_off, void *cuda_stream)
{
    if (k < 1 || k > kMaxK || !level_mean || !level_stdv || W < 2 || W > 256 || n < 0) return ABEA_ERR_ARG;
    if (n > kMaxReads) return ABEA_ERR_NOMEM;
    if (n == 0) return ABEA_OK;
    if (!seq_off || !ev_off || !sc || !pair_off || !d_out || !d_seq || !d_events ||
        (!d_pairs && pair_off[n] > pair_off[0]))
        return ABEA_ERR_ARG;
    for (int32_t i = 0; i < n; i++)
        if (seq_off[i + 1] < seq_off[i] || ev_off[i + 1] < ev_off[i] || pair_off[i + 1] < pair_off[i] ||
            pair_off[i + 1] - pair_off[i] > INT32_MAX)
            return ABEA_ERR_ARG;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
        cudaGetLastError();
        return ABEA_ERR_CUDA;
    }
    const Geometry g = abea::geometry_for(W);
    const size_t rows = size_t(1) << (2 * k);

    // working set: model rows, descriptors, order, flags, queue, k-mer cache, trace, moves
    size_t kc = 0, tr = 0, mv = 0;
    for (int32_t i = 0; i < n; i++) {
        const int64_t n_e = ev_off[i + 1] - ev_off[i];
        const int64_t n_k = (seq_off[i + 1] - seq_off[i]) - k + 1;
        if (n_e < 1 || n_k < 1) continue;
        const int64_t bands = n_e + n_k + 1;
        kc += (size_t)n_k;
        tr += (size_t)(bands * g.rec_words);
        mv += g.full ? (size_t)((bands + 15) / 16 * 16) : 0;
    }
    const size_t off_rows = 0;
    const size_t off_desc = align256(off_rows + rows * sizeof(ModelRow));
    const size_t off_order = align256(off_desc + (size_t)n * sizeof(ReadDesc));
    const size_t off_flags = align256(off_order + (size_t)n * sizeof(int32_t));
    const size_t off_queue = align256(off_flags + (size_t)n * sizeof(int32_t));
    const size_t off_kc = align256(off_queue + 256);
    const size_t off_tr = align256(off_kc + kc * 16);
    const size_t off_mv = align256(off_tr + tr * 4);
    const size_t total = align256(off_mv + mv);
    if (total > kScratchBytes) return ABEA_ERR_NOMEM;

    bool no_room = false;
    unsigned char *base = scratch_for(device, &no_room);
    if (!base) return no_room ? ABEA_ERR_NOMEM : ABEA_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    std::lock_guard<std::mutex> lock(s_setup);   // the static host buffers below are shared
    for (size_t r = 0; r < rows; r++) {
        const float mu = level_mean[r], sd = level_stdv[r];
        if (!std::isfinite(mu) || !std::isfinite(sd) || !(sd > 0.0f)) return ABEA_ERR_ARG;
        s_rows[r].mu = (double)mu;
        s_rows[r].a0 = kSqrtHalf / (double)sd;
        s_rows[r].c0 = kLogInvSqrt2Pi - std::log((double)sd);
        s_rows[r].sd = (double)sd;
    }
    size_t ckc = 0, ctr = 0, cmv = 0;
    for (int32_t i = 0; i < n; i++) {
        ReadDesc &d = s_desc[i];
        std::memset(&d, 0, sizeof(d));
        const int64_t n_e = ev_off[i + 1] - ev_off[i];
        const int64_t n_k = (seq_off[i + 1] - seq_off[i]) - k + 1;
        const abea_scalings s = sc[i];
        const bool bad = n_e < 1 || n_k < 1 || !std::isfinite(s.scale) || !std::isfinite(s.shift) ||
                         !std::isfinite(s.var) || !(s.var > 0.0f);
        d.ev_off = ev_off[i];
        d.seq_off = seq_off[i];
        d.pair_off = pair_off[i];
        d.pair_cap = (int32_t)(pair_off[i + 1] - pair_off[i]);
        d.host_bad = bad ? 1 : 0;
        if (!bad) {
            d.n_e = (int32_t)n_e;
            d.n_k = (int32_t)n_k;
            const double epk = (double)n_e / (double)n_k;
            const double lp_skip = std::log(1e-10);
            const double lp_stay = std::log(1.0 - 1.0 / (epk + 1.0));
            const double lp_step = std::log(1.0 - std::exp(lp_skip) - std::exp(lp_stay));
            d.lp_skip = (float)lp_skip;
            d.lp_stay_step = (float)(lp_stay - lp_step);
            d.lp_step = (float)lp_step;
            d.lp_trim = (float)std::log(1.0 / 100.0);
            d.scale = (double)s.scale;
            d.shift = (double)s.shift;
            d.inv_var = 1.0 / (double)s.var;
            d.log_var_step = std::log((double)s.var) - lp_step;
            const int64_t bands = n_e + n_k + 1;
            d.kc_off = (int64_t)ckc;
            d.tr_off = (int64_t)ctr;
            d.mv_off = (int64_t)cmv;
            ckc += (size_t)n_k;
            ctr += (size_t)(bands * g.rec_words);
            cmv += g.full ? (size_t)((bands + 15) / 16 * 16) : 0;
        }
        s_order[i] = i;
        s_key[i] = bad ? -1 : n_e + n_k;
    }
    std::sort(s_order, s_order + n, [](int32_t a, int32_t b) {   // longest first, then by index
        return s_key[a] != s_key[b] ? s_key[a] > s_key[b] : a < b;
    });

    // pageable sources: each copy has read the host buffer by the time it returns
    if (cudaMemcpyAsync(base + off_rows, s_rows, rows * sizeof(ModelRow), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(base + off_desc, s_desc, (size_t)n * sizeof(ReadDesc), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(base + off_order, s_order, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(base + off_queue, 0, sizeof(int32_t), st) != cudaSuccess) {
        cudaGetLastError();
        return ABEA_ERR_CUDA;
    }
    int rc = abea::launch_prep((const ReadDesc *)(base + off_desc), n, d_seq, d_events,
                               (const ModelRow *)(base + off_rows), k, (float4 *)(base + off_kc),
                               (int32_t *)(base + off_flags), st);
    if (rc != cudaSuccess) return ABEA_ERR_CUDA;
    int &grid = s_grid[device][g.C][g.mixed ? 1 : 0][g.full ? 1 : 0][g.cg];
    if (grid <= 0) grid = abea::align_grid_size(g, device);
    if (grid <= 0) return ABEA_ERR_CUDA;
    const int n_group = abea::group_count(s_desc, s_order, n, g, grid, abea::kDefaultBlockTheta);
    AlignArgs a;
    a.rd = (const ReadDesc *)(base + off_desc);
    a.order = (const int32_t *)(base + off_order);
    a.flags = (const int32_t *)(base + off_flags);
    a.n = n;
    a.W = W;
    a.L = g.L;
    a.events = d_events;
    a.seq = d_seq;
    a.kc = (const float4 *)(base + off_kc);
    a.trace = (uint32_t *)(base + off_tr);
    a.moves = (uint8_t *)(base + off_mv);
    a.pairs = d_pairs;
    a.res = d_out;
    a.queue = (int32_t *)(base + off_queue);
    a.n_group = n_group;
    rc = abea::launch_align(a, g, abea::align_launch_grid(n, n_group, grid), st);
    return rc == cudaSuccess ? ABEA_OK : ABEA_ERR_CUDA;
}
