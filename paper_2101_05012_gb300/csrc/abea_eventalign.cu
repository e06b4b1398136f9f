// eventalign rows: each aligned (event, read k-mer) pair of ABEA becomes a
// record with the k-mer's reference position and reference k-mer (through the
// read's base-space alignment), the event level, the scaled model mean and
// standard deviation of the read k-mer and the standardised level.
//
// The thesis lists eventalign as aligning a read's events to reference
// k-mers (f5c's command line; --scale-events scales the events to the model
// instead of the model to the events) and gives no record format; this file
// takes the plain reading:
//   default:       level = x,                  mean = mu*scale + shift, stdv = sigma*var
//   scale_events:  level = (x - shift)/scale,  mean = mu,              stdv = sigma*var/scale
//   z = (level - mean) / stdv
// every step one FP32 operation in that order; ref_pos is the reference
// position of the k-mer's first base (-1 for an inserted read base) and
// ref_rank the rank of ref[ref_pos : ref_pos+k] (-1 if unaligned, past the
// reference end or not ACGT).
//
// Two launches: the k-mer ranks of every read position (read and reference),
// then the rows.  Per row: 8 B of pair, 4 B of event, 4 B of reference
// position, 8 B of ranks, a model entry (shared memory for k <= 6) and 40 B
// of record.
#include <algorithm>

#include "abea_internal.h"

namespace abea {

namespace {

constexpr int kThreads = 256;

// c is one of A C G T: c - 'A' is 0, 2, 6 or 19.
__device__ __forceinline__ bool is_base(unsigned c)
{
    const unsigned d = c - 'A';
    return d < 32u && ((0x80045u >> d) & 1u);
}

// 2-bit code of an ACGT base: ((c >> 1) ^ (c >> 2)) & 3 maps A C G T to 0 1 2 3.
__device__ __forceinline__ unsigned base_code(unsigned c) { return ((c >> 1) ^ (c >> 2)) & 3u; }

constexpr int kPasses = 8;                         // passes of 256 per chunk
constexpr int kChunk = kThreads * kPasses;         // positions or pair slots per chunk

// The last i with off[i] <= x (off ascending, off[0] <= x < off[n]).
__device__ __forceinline__ int find_read(const int64_t *off, int n, int64_t x)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Rank of the k bases at s (A C G T = 0 1 2 3, the first base most
// significant); -1 if one of them is not A, C, G or T.  code[c]: the 2-bit
// code of byte c, or 4 if c is not a base.
__device__ __forceinline__ int rank_of(const uint8_t *s, int k, const uint8_t *code)
{
    unsigned r = 0, bad = 0;
    for (int j = 0; j < k; j++) {
        const unsigned c = code[s[j]];
        bad |= c;
        r = (r << 2) | (c & 3u);
    }
    return (bad & 4u) ? -1 : (int)r;
}

// Launch 1: for every k-mer start q of an aligned read, the rank of the read's
// k-mer and of the reference k-mer at ref_pos[q] (-1 if unaligned, past the
// reference end or not ACGT), into ranks[seq_off[i] - seq_lo + q].  The grid
// runs over chunks of 2,048 bases of the batch, each warp 256 of them, one
// position per lane and pass, so that a warp's loads cover consecutive bases.
__global__ void __launch_bounds__(kThreads) eventalign_ranks_kernel(const int64_t *meta, int32_t n, int64_t n_chunks,
                                                                  const uint8_t *seq, int64_t seq_lo,
                                                                  const abea_result *res, const int32_t *ref_pos,
                                                                  const uint8_t *ref, int64_t ref_len, int k,
                                                                  int2 *ranks)
{
    __shared__ uint8_t code[256];
    for (int c = threadIdx.x; c < 256; c += kThreads) code[c] = is_base((unsigned)c) ? (uint8_t)base_code(c) : 4;
    __syncthreads();
    const int64_t *seq_off = meta;
    const int64_t end = seq_off[n];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        // warp w takes positions c0 + 256 w .. c0 + 256 w + 255, 32 per pass
        const int64_t w0 = seq_lo + c * kChunk + (int64_t)kThreads * warp;
        if (w0 >= end) continue;
        int rd = __shfl_sync(0xffffffffu, lane == 0 ? find_read(seq_off, n, w0) : 0, 0), cur = -1;
        bool ok = false;
        int64_t last = 0;                          // the read's last k-mer start + 1
        for (int j = 0; j < kPasses; j++) {
            const int64_t g = w0 + 32 * j + lane;
            if (g >= end) break;
            while (g >= seq_off[rd + 1]) rd++;
            if (rd != cur) {
                cur = rd;
                ok = res[rd].status == ABEA_READ_OK;
                last = seq_off[rd + 1] - k + 1;
            }
            if (!ok || g >= last) continue;
            const int pos = ref_pos[g];
            const int rr = (pos >= 0 && (int64_t)pos + k <= ref_len) ? rank_of(ref + pos, k, code) : -1;
            ranks[g - seq_lo] = make_int2(rank_of(seq + g, k, code), rr);
        }
    }
}

constexpr int kRowWords = (int)(sizeof(abea_eventalign_row) / 4);
constexpr int kSmemModelRanks = 4096;              // models up to k = 6 sit in shared memory
static_assert(sizeof(abea_eventalign_row) == 40, "row layout");

// Launch 2.  The grid runs over chunks of 2,048 pair slots of the whole
// batch (the slots of read i are pair_off[i] .. pair_off[i+1]); a block takes
// chunks in turn, each warp 256 consecutive slots of a chunk, 32 per pass.
// Each warp forms its 32 slots' rows in its own shared-memory stage and
// writes the valid ones as consecutive words, so that a store covers whole
// lines.  SMEM_MODEL: the model's (mean, stdv) table is copied into shared
// memory once per block.
template <bool SMEM_MODEL, bool WORD8>
__global__ void __launch_bounds__(kThreads, 5) eventalign_kernel(const int64_t *meta, int32_t n, int64_t n_chunks,
                                                            int64_t seq_lo, const float *events,
                                                            const abea_scalings *sc, const abea_result *res,
                                                            const int32_t *pairs, const int32_t *ref_pos,
                                                            const int2 *ranks, const float2 *model_f, int k,
                                                            int scale_events, abea_eventalign_row *rows)
{
    __shared__ float2 smodel[SMEM_MODEL ? kSmemModelRanks : 1];
    __shared__ __align__(16) abea_eventalign_row stage[kThreads];
    const int64_t *seq_off = meta, *ev_off = meta + (n + 1), *pair_off = meta + 2 * (n + 1);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (SMEM_MODEL) {
        for (int r = t; r < (1 << (2 * k)); r += kThreads) smodel[r] = model_f[r];
        __syncthreads();
    }
    const float2 *mdl = SMEM_MODEL ? smodel : model_f;
    abea_eventalign_row *my_stage = stage + 32 * warp;
    const int64_t end = pair_off[n];
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        // warp w takes slots c0 + 256 w .. c0 + 256 w + 255, 32 per pass
        const int64_t w0 = pair_off[0] + c * kChunk + (int64_t)kThreads * warp;
        if (w0 >= end) continue;
        int rd = __shfl_sync(0xffffffffu, lane == 0 ? find_read(pair_off, n, w0) : 0, 0), cur = -1;
        int np = 0;
        bool ok = false;
        int64_t p0 = 0;
        const int2 *rk = nullptr;
        const int32_t *rp = nullptr;
        const float *ev = nullptr;
        abea_scalings s{};
        for (int j = 0; j < kPasses; j++) {
            const int64_t wfirst = w0 + 32 * j;                              // the pass's first slot
            if (wfirst >= end) break;                                        // whole warps
            const int64_t slot = wfirst + lane;
            bool valid = false;
            if (slot < end) {
                while (slot >= pair_off[rd + 1]) rd++;
                if (rd != cur) {
                    cur = rd;
                    const abea_result r = res[rd];
                    ok = r.status == ABEA_READ_OK;
                    np = r.n_pairs;
                    p0 = pair_off[rd];
                    rk = ranks + (seq_off[rd] - seq_lo);
                    rp = ref_pos + seq_off[rd];
                    ev = events + ev_off[rd];
                    s = sc[rd];
                }
                const int64_t q = slot - p0;
                if (ok && q < np) {
                    valid = true;
                    const int2 p = reinterpret_cast<const int2 *>(pairs)[slot];
                    const float x = ev[p.x];
                    const int pos = rp[p.y];
                    const int2 rank = rk[p.y];
                    const int mr = rank.x, rr = rank.y;   // mr >= 0: the read aligned, so its bases are ACGT
                    const float2 row = mdl[mr < 0 ? 0 : mr];
                    const float mu = row.x, sd = row.y;
                    float level, mean, stdv;
                    if (scale_events) {
                        level = __fdiv_rn(__fsub_rn(x, s.shift), s.scale);
                        mean = mu;
                        stdv = __fdiv_rn(__fmul_rn(sd, s.var), s.scale);
                    } else {
                        level = x;
                        mean = __fadd_rn(__fmul_rn(mu, s.scale), s.shift);
                        stdv = __fmul_rn(sd, s.var);
                    }
                    abea_eventalign_row o;
                    o.read = rd;
                    o.event = p.x;
                    o.kmer = p.y;
                    o.ref_pos = pos;
                    o.ref_rank = rr;
                    o.model_rank = mr;
                    o.level = level;
                    o.model_mean = mean;
                    o.model_stdv = stdv;
                    o.z = __fdiv_rn(__fsub_rn(level, mean), stdv);
                    my_stage[lane] = o;
                }
            }
            const unsigned vb = __ballot_sync(0xffffffffu, valid);
            __syncwarp();
            // the warp's rows out as consecutive words (8 or 4 bytes), valid rows only
            if (WORD8) {
                const uint2 *src = reinterpret_cast<const uint2 *>(my_stage);
                uint2 *dst = reinterpret_cast<uint2 *>(rows + wfirst);
#pragma unroll
                for (int m = 0; m < kRowWords / 2; m++) {
                    const int w = lane + 32 * m, row = w / (kRowWords / 2);
                    if ((vb >> row) & 1u) dst[w] = src[w];
                }
            } else {
                const unsigned *src = reinterpret_cast<const unsigned *>(my_stage);
                unsigned *dst = reinterpret_cast<unsigned *>(rows + wfirst);
#pragma unroll
                for (int m = 0; m < kRowWords; m++) {
                    const int w = lane + 32 * m, row = w / kRowWords;
                    if ((vb >> row) & 1u) dst[w] = src[w];
                }
            }
            __syncwarp();
        }
    }
}

// Read summaries: one warp per read (grid-stride); the lanes count stays and
// skips over consecutive pairs, lane 0 writes the record.
__global__ void __launch_bounds__(kThreads) summary_kernel(const int64_t *__restrict__ meta, int32_t n, int k,
                                                           const abea_result *__restrict__ res,
                                                           const int32_t *__restrict__ pairs,
                                                           abea_read_summary *__restrict__ out)
{
    const int64_t *seq_off = meta, *ev_off = meta + (n + 1), *pair_off = meta + 2 * (n + 1);
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
        const abea_result r = res[i];
        const int32_t n_e = (int32_t)(ev_off[i + 1] - ev_off[i]);
        const int32_t n_k = (int32_t)(seq_off[i + 1] - seq_off[i]) - k + 1;
        const bool ok = r.status == ABEA_READ_OK;
        const int32_t np = ok ? r.n_pairs : 0;
        const int2 *p = reinterpret_cast<const int2 *>(pairs) + pair_off[i];
        int stays = 0, skips = 0;
        for (int32_t t = 1 + lane; t < np; t += 32) {
            const int2 a = p[t - 1], b = p[t];
            stays += (b.x == a.x + 1 && b.y == a.y) ? 1 : 0;
            skips += (b.x == a.x && b.y == a.y + 1) ? 1 : 0;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            stays += __shfl_xor_sync(0xffffffffu, stays, off);
            skips += __shfl_xor_sync(0xffffffffu, skips, off);
        }
        if (lane == 0) {
            abea_read_summary s;
            s.read = i;
            s.status = r.status;
            s.n_events = n_e;
            s.n_kmers = n_k;
            s.n_pairs = np;
            s.first_event = np > 0 ? p[0].x : -1;
            s.last_event = np > 0 ? p[np - 1].x : -1;
            s.stays = stays;
            s.skips = skips;
            s.events_aligned = np - skips;
            s.score = r.score;
            s.score_per_event = n_e > 0 ? __fdiv_rn(r.score, (float)n_e) : 0.0f;
            int flags = 0;
            if (!ok) {
                flags = ABEA_QC_NOT_ALIGNED;
            } else {
                if (2 * (s.first_event + (n_e - 1 - s.last_event)) > n_e) flags |= ABEA_QC_TRIMMED;
                if (5 * skips > n_k) flags |= ABEA_QC_SKIPS;
                if (s.score_per_event < -10.0f) flags |= ABEA_QC_LOW_SCORE;
            }
            s.flags = flags;
            out[i] = s;
        }
    }
}

}  // namespace

int launch_summary(const int64_t *meta, int32_t n, int k, const abea_result *res, const int32_t *pairs,
                   abea_read_summary *out, void *stream)
{
    if (n <= 0) return (int)cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    const int64_t blocks = ((int64_t)n + kThreads / 32 - 1) / (kThreads / 32);
    summary_kernel<<<(unsigned)std::min<int64_t>(blocks, (int64_t)sms * 8), kThreads, 0, (cudaStream_t)stream>>>(
        meta, n, k, res, pairs, out);
    return (int)cudaGetLastError();
}

int launch_eventalign(const int64_t *meta, int32_t n, int64_t total_slots, const uint8_t *seq, int64_t seq_lo,
                      int64_t seq_hi, int2 *ranks, const float *events, const abea_scalings *sc, const abea_result *res, const int32_t *pairs,
                      const int32_t *ref_pos, const uint8_t *ref, int64_t ref_len, const float2 *model_f, int k,
                      int scale_events, abea_eventalign_row *rows, void *stream)
{
    if (n <= 0 || total_slots <= 0) return (int)cudaSuccess;
    if (k < 1 || k > 12) return (int)cudaErrorInvalidValue;
    const int64_t n_chunks = (total_slots + kChunk - 1) / kChunk;
    const bool smem_model = (1 << (2 * k)) <= kSmemModelRanks;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    // resident blocks per SM: 5 with the 43 KB of shared memory of the model copy, else 8
    const unsigned grid = (unsigned)std::min<int64_t>(n_chunks, (int64_t)sms * (smem_model ? 5 : 8));
    const bool word8 = ((uintptr_t)rows & 7) == 0;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n_bases = seq_hi - seq_lo, rank_chunks = (n_bases + kChunk - 1) / kChunk;
    if (rank_chunks > 0)
        eventalign_ranks_kernel<<<(unsigned)std::min<int64_t>(rank_chunks, (int64_t)sms * 8), kThreads, 0, st>>>(
            meta, n, rank_chunks, seq, seq_lo, res, ref_pos, ref, ref_len, k, ranks);
#define ABEA_EA_LAUNCH(sm_, w8_) \
    eventalign_kernel<sm_, w8_><<<grid, kThreads, 0, st>>>(meta, n, n_chunks, seq_lo, events, sc, res, pairs, ref_pos, \
                                                           ranks, model_f, k, scale_events, rows)
    if (smem_model) {
        if (word8) ABEA_EA_LAUNCH(true, true);
        else ABEA_EA_LAUNCH(true, false);
    } else {
        if (word8) ABEA_EA_LAUNCH(false, true);
        else ABEA_EA_LAUNCH(false, false);
    }
#undef ABEA_EA_LAUNCH
    return (int)cudaGetLastError();
}

}  // namespace abea
