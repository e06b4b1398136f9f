// Event detection: a read's raw signal (int16 ADC samples) -> events (mean,
// standard deviation and duration of the samples between level changes).
//
// The thesis (Sec. "Methylation calling") defines event detection as this
// segmentation but gives no detector.  This file takes a two-window t-test
// reading, every decision in integers or in one fixed FP32 order:
//   at position i (w <= i <= n-w), with exact sums S_L, S_R of x[i-w:i] and
//   x[i:i+w] and Q_L, Q_R of their squares,
//     N = w (S_R - S_L)^2,  D = w (Q_L + Q_R) - S_L^2 - S_R^2,
//     t2_i = float(N) / float(D)  (+inf if D = 0 < N, 0 if N = 0),
//   (the squared Welch statistic of the two windows, population variances);
//   t2 = 0 at the other positions.  Position i >= 1 starts an event when
//   t2_i >= tau2, t2_i > t2_j for j in [i-w+1, i-1] and t2_i >= t2_j for
//   j in [i+1, i+w-1] (a local maximum, ties to the earliest).  An event of L
//   samples with exact sums S, Q has mean = float(S) / L,
//   var = float(Q) / L - mean^2, stdv = sqrt(max(var, 0)), reported in pA as
//   (mean + offset) * per_unit and stdv * per_unit.
//
// One block per read.  Pass 1: each thread takes a 32-aligned chunk of
// positions, rolls the window sums over the chunk and w-1 positions on each
// side, keeps the last 2w-1 values of t2 in registers to decide its
// positions, and writes one bit per position.  A block scan of the chunks'
// event counts and sample sums gives each thread its first event index and
// prefix sums.  Pass 2: each thread rolls the prefix sums over its chunk and
// records (prefix sums, position) at each event start; then every event's
// statistics come from two consecutive records.
#include "abea_internal.h"

namespace abea {

namespace {

constexpr int kThreads = 256;

struct Bound {
    long long S, Q;    // sums of the samples (and squares) before the event's first sample
    int pos, pad;
};

__device__ __forceinline__ int xg(const int16_t *x, long long p, long long n)
{
    return (p >= 0 && p < n) ? (int)x[p] : 0;
}

// Exclusive block scan of (a, b, c); returns the block totals in *tot.
__device__ __forceinline__ void block_scan3(long long &a, long long &b, long long &c, long long *tot,
                                            long long (*sh)[3])
{
    const int t = threadIdx.x;
    sh[t][0] = a;
    sh[t][1] = b;
    sh[t][2] = c;
    __syncthreads();
    // Hillis-Steele over kThreads entries (log2(256) = 8 rounds)
    for (int off = 1; off < kThreads; off <<= 1) {
        long long v0 = 0, v1 = 0, v2 = 0;
        if (t >= off) {
            v0 = sh[t - off][0];
            v1 = sh[t - off][1];
            v2 = sh[t - off][2];
        }
        __syncthreads();
        sh[t][0] += v0;
        sh[t][1] += v1;
        sh[t][2] += v2;
        __syncthreads();
    }
    tot[0] = sh[kThreads - 1][0];
    tot[1] = sh[kThreads - 1][1];
    tot[2] = sh[kThreads - 1][2];
    a = sh[t][0] - a;
    b = sh[t][1] - b;
    c = sh[t][2] - c;
    __syncthreads();
}

template <int W>
__global__ void __launch_bounds__(kThreads) events_kernel(const int64_t *raw_off, const int16_t *raw,
                                                        const abea_calib *calib, float tau2, uint32_t *bits,
                                                        const int64_t *bits_off, Bound *bnd, const int64_t *bnd_off,
                                                        abea_event *out, const int64_t *ev_off, int32_t *n_ev)
{
    __shared__ long long sh[kThreads][3];
    const int i = blockIdx.x;
    const long long n = raw_off[i + 1] - raw_off[i];
    const int16_t *x = raw + raw_off[i];
    uint32_t *bw = bits + bits_off[i];
    Bound *rec = bnd + bnd_off[i];
    const long long chunk = (((n + kThreads - 1) / kThreads) + 31) / 32 * 32;
    const long long a = (long long)threadIdx.x * chunk;
    const long long b = (a + chunk < n) ? a + chunk : n;

    // pass 1: t2 and event starts over [a, b).  The samples x[p-W .. p+W] sit in a register
    // ring (one load per step); the window sums roll in 32 bits (|S| < 2^19) and the sums of
    // squares in 64 bits (each step adds the 32-bit difference of two squares).
    long long cnt = 0, csum = 0, csq = 0;
    if (a < b) {
        float ring[2 * W - 1];                 // t2 at p-2W+2 .. p
#pragma unroll
        for (int r = 0; r < 2 * W - 1; r++) ring[r] = -1.0f;
        int xs[2 * W + 1];                     // x[p-W .. p+W] (0 outside the read)
        long long p = a - (W - 1);
#pragma unroll
        for (int q = 0; q < 2 * W + 1; q++) xs[q] = xg(x, p - W + q, n);
        int SL = 0, SR = 0;
        long long QL = 0, QR = 0;
#pragma unroll
        for (int q = 0; q < W; q++) {
            SL += xs[q];
            QL += xs[q] * xs[q];
            SR += xs[W + q];
            QR += xs[W + q] * xs[W + q];
        }
        uint32_t word = 0;
        int ccount = 0;
        long long cs = 0;
        const long long p_end = b + W - 1;
        for (; p < p_end; p++) {
            float t2 = -1.0f;                  // outside the read
            if (p >= 0 && p < n) {
                t2 = 0.0f;
                if (p >= W && p <= n - W) {
                    const int d = SR - SL;
                    const long long N = (long long)W * ((long long)d * d);
                    const long long D = (long long)W * (QL + QR) - (long long)SL * SL - (long long)SR * SR;
                    if (D == 0) t2 = (N > 0) ? __int_as_float(0x7f800000) : 0.0f;
                    else t2 = __fdiv_rn(__ll2float_rn(N), __ll2float_rn(D));
                }
            }
#pragma unroll
            for (int r = 0; r < 2 * W - 2; r++) ring[r] = ring[r + 1];
            ring[2 * W - 2] = t2;
            const long long c = p - (W - 1);   // ring[W-1] holds t2_c
            if (c >= a) {                      // c < b holds for every p < p_end
                const float v = ring[W - 1];
                bool start = (c >= 1) && (v >= tau2);
#pragma unroll
                for (int r = 0; r < W - 1; r++) start = start && !(ring[r] >= v);
#pragma unroll
                for (int r = W; r < 2 * W - 1; r++) start = start && !(ring[r] > v);
                const int bit = (int)((c - a) & 31);
                word |= (start ? 1u : 0u) << bit;
                ccount += start ? 1 : 0;
                const int xv = xs[1];          // x[c] = x[p-W+1]
                cs += xv;
                csq += xv * xv;
                if (bit == 31 || c == b - 1) {
                    bw[c >> 5] = word;
                    word = 0;
                }
            }
            // roll to p+1: x[p] leaves the right window for the left, x[p-W] leaves, x[p+W] enters
            const int in_r = xg(x, p + W + 1, n);
            const int x_p = xs[W], out_l = xs[0], new_r = xs[2 * W];
            SL += x_p - out_l;
            QL += x_p * x_p - out_l * out_l;
            SR += new_r - x_p;
            QR += new_r * new_r - x_p * x_p;
#pragma unroll
            for (int q = 0; q < 2 * W; q++) xs[q] = xs[q + 1];
            xs[2 * W] = in_r;
        }
        cnt = ccount;
        csum = cs;
    }
    long long tot[3];
    block_scan3(cnt, csum, csq, tot, sh);      // cnt, csum, csq become this chunk's exclusive prefixes
    const long long n_events = (n > 0) ? tot[0] + 1 : 0;

    // pass 2: the record of every event start (index 0: position 0), and a final record at n
    if (threadIdx.x == 0 && n > 0) {
        rec[0] = Bound{0, 0, 0, 0};
        rec[n_events] = Bound{tot[1], tot[2], (int)n, 0};
    }
    if (a < b) {
        long long e = cnt + 1, S = csum, Q = csq;
        for (long long c0 = a; c0 < b; c0 += 32) {
            uint32_t word = bw[c0 >> 5];
            const int m = (b - c0 < 32) ? (int)(b - c0) : 32;
            for (int j = 0; j < m; j++) {
                if ((word >> j) & 1u) rec[e++] = Bound{S, Q, (int)(c0 + j), 0};
                const int xv = x[c0 + j];
                S += xv;
                Q += xv * xv;
            }
        }
    }
    __syncthreads();
    const int64_t cap = ev_off[i + 1] - ev_off[i];
    const float offset = calib[i].offset, per_unit = calib[i].pa_per_unit;
    for (long long e = threadIdx.x; e < n_events && e < cap; e += kThreads) {
        const Bound r0 = rec[e], r1 = rec[e + 1];
        const int L = r1.pos - r0.pos;
        const float fL = __int2float_rn(L);
        const float mean = __fdiv_rn(__ll2float_rn(r1.S - r0.S), fL);
        const float var = __fsub_rn(__fdiv_rn(__ll2float_rn(r1.Q - r0.Q), fL), __fmul_rn(mean, mean));
        const float stdv = __fsqrt_rn(var > 0.0f ? var : 0.0f);
        abea_event ev;
        ev.mean = __fmul_rn(__fadd_rn(mean, offset), per_unit);
        ev.stdv = __fmul_rn(stdv, per_unit);
        ev.start = r0.pos;
        ev.length = L;
        out[ev_off[i] + e] = ev;
    }
    if (threadIdx.x == 0) n_ev[i] = (int32_t)n_events;
}

template <int W>
int launch_w(const int64_t *raw_off, int32_t n, const int16_t *raw, const abea_calib *calib, float tau2,
             uint32_t *bits, const int64_t *bits_off, void *bnd, const int64_t *bnd_off, abea_event *out,
             const int64_t *ev_off, int32_t *n_ev, void *stream)
{
    events_kernel<W><<<n, kThreads, 0, (cudaStream_t)stream>>>(raw_off, raw, calib, tau2, bits, bits_off,
                                                               (Bound *)bnd, bnd_off, out, ev_off, n_ev);
    return (int)cudaGetLastError();
}

}  // namespace

size_t event_record_bytes() { return sizeof(Bound); }

int launch_events(const int64_t *raw_off, int32_t n, const int16_t *raw, const abea_calib *calib, int window,
                  float tau2, uint32_t *bits, const int64_t *bits_off, void *bnd, const int64_t *bnd_off,
                  abea_event *out, const int64_t *ev_off, int32_t *n_ev, void *stream)
{
    if (n <= 0) return (int)cudaSuccess;
    switch (window) {
    case 2: return launch_w<2>(raw_off, n, raw, calib, tau2, bits, bits_off, bnd, bnd_off, out, ev_off, n_ev, stream);
    case 3: return launch_w<3>(raw_off, n, raw, calib, tau2, bits, bits_off, bnd, bnd_off, out, ev_off, n_ev, stream);
    case 4: return launch_w<4>(raw_off, n, raw, calib, tau2, bits, bits_off, bnd, bnd_off, out, ev_off, n_ev, stream);
    case 5: return launch_w<5>(raw_off, n, raw, calib, tau2, bits, bits_off, bnd, bnd_off, out, ev_off, n_ev, stream);
    case 6: return launch_w<6>(raw_off, n, raw, calib, tau2, bits, bits_off, bnd, bnd_off, out, ev_off, n_ev, stream);
    case 7: return launch_w<7>(raw_off, n, raw, calib, tau2, bits, bits_off, bnd, bnd_off, out, ev_off, n_ev, stream);
    case 8: return launch_w<8>(raw_off, n, raw, calib, tau2, bits, bits_off, bnd, bnd_off, out, ev_off, n_ev, stream);
    default: return (int)cudaErrorInvalidValue;
    }
}

}  // namespace abea
