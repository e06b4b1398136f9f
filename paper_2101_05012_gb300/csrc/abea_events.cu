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
// The grid runs over tiles of kEventTile positions of all reads at once, so a
// long read takes as many blocks as its length needs.  Three launches:
//   1. per tile: the samples around the tile into shared memory; t2 of the
//      tile's positions and of w-1 on each side; one start bit per position
//      (a warp vote per 32 positions); the tile's summary: its starts, the
//      sums of its samples, its last start and the sums before that start;
//   2. per read (one warp): an exclusive scan of the tile summaries gives
//      each tile the starts, the sums and the last start before it
//      (position 0 counts as the first start); the read's event count;
//   3. per tile: each thread takes 16 consecutive positions; a block scan
//      gives every start its index and the sums before it; the starts'
//      records go to shared memory, and each thread then makes every 256th
//      event of the tile from two consecutive records (the event closed by
//      the tile's first start opens at the last start before the tile; the
//      read's last tile also closes the final event at the end of the read).
// No block waits for another.
#include <algorithm>

#include "abea_internal.h"

namespace abea {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kPer = kEventTile / kThreads;    // positions per thread in launch 3
constexpr int kWords = kEventTile / 32;        // start-bit words per tile
static_assert(kPer == 16, "launch 3 reads one 16-bit half of a start word per thread");

// A run of positions [u, v): its starts, the sums of its samples (and their
// squares), and its last start with the sums of the run's samples before it.
struct Run {
    long long S, Q, S_last, Q_last;
    int cnt, has, last, pad;
};

// float(v) rounded to nearest, ties to even, from integer operations (the
// IEEE 754 rule written out): the 24 leading significant bits are kept, the
// dropped bits round them.  The platform's 64-bit integer conversion runs on
// the FP64 pipe, a small fraction of GB300's throughput, and two of them per
// position bound the t2 pass.
__device__ __forceinline__ float f32_from_u64(unsigned long long v)
{
    if (v == 0) return 0.0f;
    const int e = 63 - __clzll(v);                 // v in [2^e, 2^(e+1))
    unsigned m;                                    // significand, [2^23, 2^24]
    if (e <= 23) {
        m = (unsigned)v << (23 - e);
    } else {
        const int drop = e - 23;                   // 1 .. 40
        m = (unsigned)(v >> drop);
        const unsigned long long rem = v & ((1ull << drop) - 1ull), half = 1ull << (drop - 1);
        m += (rem > half || (rem == half && (m & 1u))) ? 1u : 0u;
    }
    // exponent field 127 + e holds the implicit bit: adding m (with its 2^23) to
    // (126 + e) << 23 gives the right bits, a carry to 2^24 included
    return __uint_as_float(((unsigned)(126 + e) << 23) + m);
}

// The same rounding for v < 2^44 (the t2 terms: N <= 8 (2^19)^2, D <= 8 * 16 * 2^30):
// v = h 2^21 + l with h, l < 2^23, both exact in float, and one fused
// multiply-add rounds h 2^21 + l once.
__device__ __forceinline__ float f32_from_u44(unsigned long long v)
{
    const unsigned h = (unsigned)(v >> 21), l = (unsigned)v & 0x1fffffu;
    const float fh = __fsub_rn(__uint_as_float(0x4b000000u | h), 8388608.0f);   // 2^23 + h - 2^23
    const float fl = __fsub_rn(__uint_as_float(0x4b000000u | l), 8388608.0f);
    return __fmaf_rn(fh, 2097152.0f, fl);
}

__device__ __forceinline__ float f32_from_i64(long long v)
{
    const float f = f32_from_u64(v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v);
    return v < 0 ? -f : f;
}

__device__ __forceinline__ Run run_empty() { return Run{0, 0, 0, 0, 0, 0, 0, 0}; }

// [u, w) from [u, v) and [v, w).
__device__ __forceinline__ Run combine(const Run &x, const Run &y)
{
    Run r;
    r.S = x.S + y.S;
    r.Q = x.Q + y.Q;
    r.cnt = x.cnt + y.cnt;
    r.has = x.has | y.has;
    r.last = y.has ? y.last : x.last;
    r.S_last = y.has ? x.S + y.S_last : x.S_last;
    r.Q_last = y.has ? x.Q + y.Q_last : x.Q_last;
    r.pad = 0;
    return r;
}

__device__ __forceinline__ Run shfl_run(const Run &x, int src)
{
    Run r;
    r.S = __shfl_sync(kFull, x.S, src);
    r.Q = __shfl_sync(kFull, x.Q, src);
    r.S_last = __shfl_sync(kFull, x.S_last, src);
    r.Q_last = __shfl_sync(kFull, x.Q_last, src);
    r.cnt = __shfl_sync(kFull, x.cnt, src);
    r.has = __shfl_sync(kFull, x.has, src);
    r.last = __shfl_sync(kFull, x.last, src);
    r.pad = 0;
    return r;
}

__device__ __forceinline__ Run shfl_up_run(const Run &x, int d)
{
    Run r;
    r.S = __shfl_up_sync(kFull, x.S, d);
    r.Q = __shfl_up_sync(kFull, x.Q, d);
    r.S_last = __shfl_up_sync(kFull, x.S_last, d);
    r.Q_last = __shfl_up_sync(kFull, x.Q_last, d);
    r.cnt = __shfl_up_sync(kFull, x.cnt, d);
    r.has = __shfl_up_sync(kFull, x.has, d);
    r.last = __shfl_up_sync(kFull, x.last, d);
    r.pad = 0;
    return r;
}

// Inclusive scan over the warp's lanes in lane order.
__device__ __forceinline__ Run warp_scan(Run x, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const Run y = shfl_up_run(x, d);
        if (lane >= d) x = combine(y, x);
    }
    return x;
}

// Sums over the block (long long), then the result in every thread.
template <int N>
__device__ __forceinline__ void block_sum(long long (&v)[N], long long (*sh)[N])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < N; j++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[j] += __shfl_xor_sync(kFull, v[j], off);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < N; j++) sh[warp][j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < N; j++) {
        v[j] = 0;
        for (int w = 0; w < kWarpsPerBlock; w++) v[j] += sh[w][j];
    }
    __syncthreads();
}

// Shared-memory index of element q of an array padded with one word after
// every 16: a thread's 16 consecutive elements and a warp's 32 consecutive
// elements both fall in distinct banks.
__device__ __forceinline__ int pad16(int q) { return q + (q >> 4); }

// t2 at position p of a read of n samples from the exact sums of its two
// windows (-1 outside the read, 0 where a window leaves it).
template <int W>
__device__ __forceinline__ float t2_value(int p, int n, int SL, int SR, long long QL, long long QR)
{
    if (p < 0 || p >= n) return -1.0f;
    if (p < W || p > n - W) return 0.0f;
    const int d = SR - SL;
    const long long N = (long long)W * ((long long)d * d);
    const long long D = (long long)W * (QL + QR) - (long long)SL * SL - (long long)SR * SR;
    if (D == 0) return (N > 0) ? __int_as_float(0x7f800000) : 0.0f;
    return __fdiv_rn(f32_from_u44((unsigned long long)N), f32_from_u44((unsigned long long)D));
}

// Launch 1.  Shared memory: the samples x[a-2W+1 .. a+T+2W-2] (0 outside the
// read) and t2 at a-W+1 .. a+T+W-2 (-1 outside the read), a = the tile's
// first position, both padded.  Thread t forms t2 at positions a + 16t ..
// a + 16t + 15, rolling the four window sums from registers, then decides the
// same positions from the t2 values around them.
template <int W>
__global__ void __launch_bounds__(kThreads, 6) event_tiles_kernel(const int64_t *raw_off, const int64_t *tile_off,
                                                             const int32_t *tile_read, const int16_t *raw,
                                                             float tau2, uint32_t *bits, Run *tsum)
{
    constexpr int XH = 2 * W - 1;                 // samples kept before the tile
    constexpr int NT = kEventTile + 2 * W - 2;    // t2s[q] = t2 at a - (W-1) + q
    constexpr int NX = kEventTile + 4 * W - 2;    // xs[q] = x[a - XH + q]
    constexpr int NV = kPer + 2 * W - 1;          // samples behind a thread's 16 t2 values
    __shared__ int xs[NX + NX / 16 + 1];
    __shared__ float t2s[NT + NT / 16 + 1];
    __shared__ long long red[kWarpsPerBlock][3];
    __shared__ int redl[kWarpsPerBlock];
    const long long tile = blockIdx.x;
    const int i = tile_read[tile];
    const int n = (int)(raw_off[i + 1] - raw_off[i]);          // < 2^30 samples per read
    const int a = (int)(tile - tile_off[i]) * kEventTile;
    const int16_t *x = raw + raw_off[i];
    const int t = threadIdx.x;
    for (int q = t; q < NX; q += kThreads) {
        const int p = a - XH + q;
        xs[pad16(q)] = (p >= 0 && p < n) ? (int)x[p] : 0;
    }
    __syncthreads();
    // t2 at index q (position a - (W-1) + q): left window xs[q .. q+W-1], right window xs[q+W .. q+2W-1].
    // Thread t takes q = 16t + W-1 .. 16t + W+14, the positions it decides below, rolling the sums;
    // the first and the last thread add the W-1 values on either side.
    {
        int xv[NV];
#pragma unroll
        for (int u = 0; u < NV; u++) {
            constexpr int o = W - 1;
            xv[u] = xs[17 * t + (o + u) + ((o + u) >> 4)];   // pad16(16 t + o + u)
        }
        // |x| <= 2^15: a square fits in 32 bits
        auto sq = [&](int u) { return xv[u] * xv[u]; };
        int SL = 0, SR = 0;
        long long QL = 0, QR = 0;
#pragma unroll
        for (int u = 0; u < W; u++) {
            SL += xv[u];
            SR += xv[W + u];
            QL += sq(u);
            QR += sq(W + u);
        }
#pragma unroll
        for (int j = 0; j < kPer; j++) {
            constexpr int o = W - 1;
            t2s[17 * t + (o + j) + ((o + j) >> 4)] = t2_value<W>(a + kPer * t + j, n, SL, SR, QL, QR);
            if (j + 1 < kPer) {                                // roll to the next position
                SL += xv[j + W] - xv[j];
                SR += xv[j + 2 * W] - xv[j + W];
                const int mid = sq(j + W);
                QL += mid - sq(j);
                QR += sq(j + 2 * W) - mid;
            }
        }
        if (t == 0 || t == kThreads - 1) {
            const int q0 = (t == 0) ? 0 : kEventTile + W - 1;
            for (int q = q0; q < q0 + W - 1; q++) {
                int sl = 0, sr = 0;
                long long ql = 0, qr = 0;
                for (int u = 0; u < W; u++) {
                    const int l = xs[pad16(q + u)], r = xs[pad16(q + W + u)];
                    sl += l;
                    sr += r;
                    ql += l * l;
                    qr += r * r;
                }
                t2s[pad16(q)] = t2_value<W>(a - (W - 1) + q, n, sl, sr, ql, qr);
            }
        }
    }
    __syncthreads();
    // starts: thread t decides positions a + 16t .. a + 16t + 15 from t2 at 16t .. 16t + 15 + 2W - 2
    // (t2s indices) held in registers; two threads' 16 bits form one word
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NR = kPer + 2 * W - 2;
    float tv[NR];
#pragma unroll
    for (int u = 0; u < NR; u++) tv[u] = t2s[17 * t + u + (u >> 4)];      // pad16(16 t + u), u < 32
    int xv[kPer];
    long long S = 0, Q = 0;
    unsigned mask = 0;
#pragma unroll
    for (int j = 0; j < kPer; j++) {
        const int c = a + kPer * t + j;
        xv[j] = xs[17 * t + (j + XH) + ((j + XH) >> 4)];                   // pad16(16 t + j + XH)
        S += xv[j];                                                         // 0 past the read
        Q += xv[j] * xv[j];
        const float v = tv[j + W - 1];
        bool start = (c >= 1) && (c < n) && (v >= tau2);
#pragma unroll
        for (int u = 1; u < W; u++) start = start && !(tv[j + W - 1 - u] >= v) && !(tv[j + W - 1 + u] > v);
        mask |= (start ? 1u : 0u) << j;
    }
    const unsigned up = __shfl_down_sync(kFull, mask, 1);
    if ((t & 1) == 0) bits[tile * kWords + (t >> 1)] = mask | (up << 16);
    const int mylast = mask ? kPer * t + 31 - __clz(mask) : -1;
    int last = mylast;                                                      // the tile's last start (tile-relative)
    long long tot[3] = {__popc(mask), S, Q};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) last = max(last, __shfl_xor_sync(kFull, last, off));
    if (lane == 0) redl[warp] = last;
    block_sum<3>(tot, red);                        // its barriers also publish redl
    for (int w = 0; w < kWarpsPerBlock; w++) last = max(last, redl[w]);
    // the sums of the tile's samples before its last start
    long long before[2] = {0, 0};
    if (last >= 0) {
        if (kPer * t + kPer <= last) {
            before[0] = S;
            before[1] = Q;
        } else {
#pragma unroll
            for (int j = 0; j < kPer; j++)
                if (kPer * t + j < last) {
                    before[0] += xv[j];
                    before[1] += xv[j] * xv[j];
                }
        }
    }
    block_sum<2>(before, reinterpret_cast<long long(*)[2]>(red));
    if (threadIdx.x == 0)
        tsum[tile] = Run{tot[1], tot[2], before[0], before[1], (int)tot[0], last >= 0 ? 1 : 0,
                         last >= 0 ? a + last : 0, 0};
}

// Launch 2: one warp per read.  tpre[t] = the run from the read's position 0
// to tile t's first position, with position 0 as a start (cnt counts the
// starts from position 1 on).
__global__ void __launch_bounds__(kThreads) event_scan_kernel(const int64_t *raw_off, const int64_t *tile_off,
                                                            int32_t n_reads, const Run *tsum, Run *tpre,
                                                            int32_t *n_ev)
{
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (i >= n_reads) return;                      // whole warps
    const long long t0 = tile_off[i], t1 = tile_off[i + 1];
    Run carry = Run{0, 0, 0, 0, 0, 1, 0, 0};
    for (long long base = t0; base < t1; base += 32) {
        const long long t = base + lane;
        const Run v = (t < t1) ? tsum[t] : run_empty();
        const Run inc = warp_scan(v, lane);
        Run exc = shfl_up_run(inc, 1);
        if (lane == 0) exc = run_empty();
        if (t < t1) tpre[t] = combine(carry, exc);
        carry = combine(carry, shfl_run(inc, 31));
    }
    if (lane == 0) n_ev[i] = (raw_off[i + 1] > raw_off[i]) ? carry.cnt + 1 : 0;
}

__device__ __forceinline__ abea_event make_event(long long S, long long Q, int start, int L, float offset,
                                                 float per_unit)
{
    const float fL = f32_from_u64((unsigned long long)L);
    const float mean = __fdiv_rn(f32_from_i64(S), fL);
    const float var = __fsub_rn(__fdiv_rn(f32_from_u64((unsigned long long)Q), fL), __fmul_rn(mean, mean));
    const float stdv = __fsqrt_rn(var > 0.0f ? var : 0.0f);
    abea_event ev;
    ev.mean = __fmul_rn(__fadd_rn(mean, offset), per_unit);
    ev.stdv = __fmul_rn(stdv, per_unit);
    ev.start = start;
    ev.length = L;
    return ev;
}

// Exclusive sums over the block's threads in thread order (c, S, Q), and the
// block's totals.
__device__ __forceinline__ void block_exclusive3(int &c, long long &S, long long &Q, int &ct, long long &St,
                                                 long long &Qt, long long (*sh)[3])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ic = c;
    long long iS = S, iQ = Q;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int yc = __shfl_up_sync(kFull, ic, d);
        const long long yS = __shfl_up_sync(kFull, iS, d), yQ = __shfl_up_sync(kFull, iQ, d);
        if (lane >= d) {
            ic += yc;
            iS += yS;
            iQ += yQ;
        }
    }
    if (lane == 31) {
        sh[warp][0] = ic;
        sh[warp][1] = iS;
        sh[warp][2] = iQ;
    }
    __syncthreads();
    long long pc = 0, pS = 0, pQ = 0;
    ct = 0;
    St = Qt = 0;
    for (int w = 0; w < kWarpsPerBlock; w++) {
        if (w == warp) {
            pc = ct;
            pS = St;
            pQ = Qt;
        }
        ct += (int)sh[w][0];
        St += sh[w][1];
        Qt += sh[w][2];
    }
    c = (int)pc + ic - c;
    S = pS + iS - S;
    Q = pQ + iQ - Q;
}

// A start inside a tile: its position and the sums of the tile's samples
// before it.
struct Rec {
    int pos, S;                                    // |S| <= 4096 * 2^15
    long long Q;
};
constexpr int kMaxRec = kEventTile / 2;            // starts lie >= w >= 2 apart
constexpr int kXsWords = kEventTile + kEventTile / 16;
constexpr int kEmitSmem = (kXsWords * 4 > kMaxRec * (int)sizeof(Rec)) ? kXsWords * 4 : kMaxRec * (int)sizeof(Rec);

// Launch 3.  The tile's samples go to shared memory (padded), thread t keeps
// positions a + 16t .. a + 16t + 15 in registers; a block scan gives each
// thread its first start's index and the sums before its positions; the
// starts' records replace the samples in shared memory; then thread t makes
// events t, t + 256, ... of the tile: event e runs from record e-1 (the last
// start before the tile for e = 0) to record e (the end of the read after the
// read's last record).
__global__ void __launch_bounds__(kThreads, 6) event_emit_kernel(const int64_t *raw_off, const int64_t *tile_off,
                                                            const int32_t *tile_read, const int64_t *ev_off,
                                                            const int16_t *raw, const abea_calib *calib,
                                                            const uint32_t *bits, const Run *tpre, abea_event *out)
{
    __shared__ __align__(16) unsigned char smem[kEmitSmem];
    __shared__ long long sh[kWarpsPerBlock][3];
    int *xs = reinterpret_cast<int *>(smem);
    Rec *rec = reinterpret_cast<Rec *>(smem);
    const long long tile = blockIdx.x;
    const int i = tile_read[tile];
    const int n = (int)(raw_off[i + 1] - raw_off[i]);
    const int a = (int)(tile - tile_off[i]) * kEventTile;
    const int16_t *x = raw + raw_off[i];
    for (int q = threadIdx.x; q < kEventTile; q += kThreads) xs[pad16(q)] = (a + q < n) ? (int)x[a + q] : 0;
    const int t = threadIdx.x;
    const uint32_t m16 = (bits[tile * kWords + (t >> 1)] >> (16 * (t & 1))) & 0xffffu;
    __syncthreads();
    int xv[kPer];
    long long S = 0, Q = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        xv[k] = xs[17 * t + k];                    // pad16(16 t + k)
        S += xv[k];
        Q += xv[k] * xv[k];
    }
    int c = __popc(m16), ct;
    long long St, Qt;
    block_exclusive3(c, S, Q, ct, St, Qt, sh);     // its barrier ends the reads of xs
    int sr = (int)S;
    long long qr = Q;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        if ((m16 >> k) & 1u) {
            if (c < kMaxRec) rec[c] = Rec{a + 16 * t + k, sr, qr};
            c++;
        }
        sr += xv[k];
        qr += xv[k] * xv[k];
    }
    __syncthreads();
    const Run pre = tpre[tile];
    const long long cap = ev_off[i + 1] - ev_off[i];
    abea_event *o = out + ev_off[i];
    const float offset = calib[i].offset, per_unit = calib[i].pa_per_unit;
    const int nrec = min(ct, kMaxRec);
    const int n_out = nrec + ((a + kEventTile >= n) ? 1 : 0);
    for (int e = t; e < n_out; e += kThreads) {
        int p0, p1;
        long long S0, Q0, S1, Q1;
        if (e == 0) {
            p0 = pre.last;
            S0 = pre.S_last;
            Q0 = pre.Q_last;
        } else {
            const Rec r = rec[e - 1];
            p0 = r.pos;
            S0 = pre.S + r.S;
            Q0 = pre.Q + r.Q;
        }
        if (e < nrec) {
            const Rec r = rec[e];
            p1 = r.pos;
            S1 = pre.S + r.S;
            Q1 = pre.Q + r.Q;
        } else {                                   // the end of the read
            p1 = n;
            S1 = pre.S + St;
            Q1 = pre.Q + Qt;
        }
        const long long m = pre.cnt + e;
        if (m < cap) o[m] = make_event(S1 - S0, Q1 - Q0, p0, p1 - p0, offset, per_unit);
    }
}

template <int W>
int launch_w(const int64_t *raw_off, const int64_t *ev_off, const int64_t *tile_off, const int32_t *tile_read,
             int32_t n, int64_t n_tiles, const int16_t *raw, const abea_calib *calib, float tau2, void *scratch,
             abea_event *out, int32_t *n_ev, cudaStream_t st)
{
    uint32_t *bits = (uint32_t *)scratch;
    Run *tsum = (Run *)(bits + (size_t)n_tiles * kWords);
    Run *tpre = tsum + n_tiles;
    if (n_tiles > 0)
        event_tiles_kernel<W><<<(unsigned)n_tiles, kThreads, 0, st>>>(raw_off, tile_off, tile_read, raw, tau2, bits,
                                                                      tsum);
    event_scan_kernel<<<(n + kWarpsPerBlock - 1) / kWarpsPerBlock, kThreads, 0, st>>>(raw_off, tile_off, n, tsum,
                                                                                       tpre, n_ev);
    if (n_tiles > 0)
        event_emit_kernel<<<(unsigned)n_tiles, kThreads, 0, st>>>(raw_off, tile_off, tile_read, ev_off, raw, calib,
                                                                  bits, tpre, out);
    return (int)cudaGetLastError();
}

__global__ void f32_from_i64_kernel(const long long *in, long long n, float *out)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        out[j] = f32_from_i64(in[j]);
}

}  // namespace

int launch_f32_from_i64(const int64_t *in, int64_t n, float *out, void *stream)
{
    if (n <= 0) return (int)cudaSuccess;
    const long long blocks = std::min<long long>((n + kThreads - 1) / kThreads, 152 * 8);
    f32_from_i64_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>((const long long *)in, n, out);
    return (int)cudaGetLastError();
}

size_t event_tile_bytes() { return (size_t)kWords * 4 + 2 * sizeof(Run); }

int launch_events(const int64_t *raw_off, const int64_t *ev_off, const int64_t *tile_off, const int32_t *tile_read,
                  int32_t n, int64_t n_tiles, const int16_t *raw, const abea_calib *calib, int window, float tau2,
                  void *scratch, abea_event *out, int32_t *n_ev, void *stream)
{
    if (n <= 0) return (int)cudaSuccess;
    if (n_tiles < 0 || n_tiles > 0x7fffffff) return (int)cudaErrorInvalidValue;
    cudaStream_t st = (cudaStream_t)stream;
#define ABEA_EVENTS_W(w_) \
    case w_: return launch_w<w_>(raw_off, ev_off, tile_off, tile_read, n, n_tiles, raw, calib, tau2, scratch, out, n_ev, st)
    switch (window) {
        ABEA_EVENTS_W(2);
        ABEA_EVENTS_W(3);
        ABEA_EVENTS_W(4);
        ABEA_EVENTS_W(5);
        ABEA_EVENTS_W(6);
        ABEA_EVENTS_W(7);
        ABEA_EVENTS_W(8);
    default: return (int)cudaErrorInvalidValue;
    }
#undef ABEA_EVENTS_W
}

}  // namespace abea
