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
// One block per read; the threads take its pairs in turn.  Gather-bound: per
// pair 8 B of pair, 4 B of event, a model row (L2), the read's and the
// reference's k bases (L1) and 40 B of record.
#include "abea_internal.h"

namespace abea {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int rank_of(const uint8_t *s, int k)
{
    int r = 0;
    for (int j = 0; j < k; j++) {
        const unsigned c = s[j];
        const unsigned d = c - 'A';
        if (!(d < 32u && ((0x80045u >> d) & 1u))) return -1;   // A C G T only
        r = 4 * r + (int)(((c >> 1) ^ (c >> 2)) & 3u);
    }
    return r;
}

__global__ void __launch_bounds__(kThreads) eventalign_kernel(const int64_t *meta, int32_t n, const uint8_t *seq,
                                                            const float *events, const abea_scalings *sc,
                                                            const abea_result *res, const int32_t *pairs,
                                                            const int32_t *ref_pos, const uint8_t *ref,
                                                            int64_t ref_len, const ModelRow *model, int k,
                                                            int scale_events, abea_eventalign_row *rows)
{
    const int i = blockIdx.x;
    if (i >= n) return;
    const int64_t *seq_off = meta, *ev_off = meta + (n + 1), *pair_off = meta + 2 * (n + 1);
    const abea_result r = res[i];
    if (r.status != ABEA_READ_OK) return;
    const int np = r.n_pairs;
    const uint8_t *sq = seq + seq_off[i];
    const int32_t *rp = ref_pos + seq_off[i];
    const float *ev = events + ev_off[i];
    const int2 *pr = reinterpret_cast<const int2 *>(pairs) + pair_off[i];
    abea_eventalign_row *out = rows + pair_off[i];
    const abea_scalings s = sc[i];
    for (int t = threadIdx.x; t < np; t += kThreads) {
        const int2 p = pr[t];
        const float x = ev[p.x];
        const int mr = rank_of(sq + p.y, k);     // a valid k-mer: the read aligned
        const ModelRow row = model[mr < 0 ? 0 : mr];
        const float mu = (float)row.mu, sd = (float)row.sd;   // exact: the model is FP32
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
        const int pos = rp[p.y];
        const int rr = (pos >= 0 && (int64_t)pos + k <= ref_len) ? rank_of(ref + pos, k) : -1;
        abea_eventalign_row o;
        o.read = i;
        o.event = p.x;
        o.kmer = p.y;
        o.ref_pos = pos;
        o.ref_rank = rr;
        o.model_rank = mr;
        o.level = level;
        o.model_mean = mean;
        o.model_stdv = stdv;
        o.z = __fdiv_rn(__fsub_rn(level, mean), stdv);
        out[t] = o;
    }
}

}  // namespace

int launch_eventalign(const int64_t *meta, int32_t n, const uint8_t *seq, const float *events,
                      const abea_scalings *sc, const abea_result *res, const int32_t *pairs, const int32_t *ref_pos,
                      const uint8_t *ref, int64_t ref_len, const ModelRow *model, int k, int scale_events,
                      abea_eventalign_row *rows, void *stream)
{
    if (n <= 0) return (int)cudaSuccess;
    eventalign_kernel<<<n, kThreads, 0, (cudaStream_t)stream>>>(meta, n, seq, events, sc, res, pairs, ref_pos, ref,
                                                               ref_len, model, k, scale_events, rows);
    return (int)cudaGetLastError();
}

}  // namespace abea
