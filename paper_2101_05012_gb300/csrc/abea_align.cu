// Core kernel: adaptive banded event alignment of a batch of reads, one warp
// per read, the band held in registers.
//
// What it computes (thesis Ch.5):
//   Alg. adaptivebandedcpu        band initialisation, the band loop with the
//                                 Suzuki-Kasahara move, the band fill, backtrack
//   Alg. adaptivebandedcpucompute the D/U/L cell score and its direction
//   Alg. adaptivebandedcpucomputelog  the Gaussian emission (operands from the
//                                 k-mer cache built by the pre-kernel)
//   Sec. ABEA "trim states"       leading events via the k = -1 column,
//                                 trailing events via the end-cell rule
//
// Band b holds the cells with e + k = b - 2.  Offset j of band b is the cell
// (ll_e - j, ll_k + j): offset 0 is the band's max-event end, offset W-1 its
// max-k-mer end.  Band 0 puts the origin (-1,-1) at offset W/2; band 1 is
// band 0 moved by one event and holds the trim cell (0,-1).  Each later band
// moves by one k-mer when S_{b-1}[0] < S_{b-1}[W-1] (the better end is the
// k-mer end), else by one event; when both ends are -inf the moves alternate
// (a k-mer move on odd b).
//
// GB300 mapping (this differs from the thesis's one-block-per-read design
// with three shared-memory bands and four __syncthreads per band):
//   - one warp per read; lane l owns the C consecutive offsets
//     [C*l, C*l + C) of every band; L = ceil(W/C) lanes are live;
//   - the previous two bands, the events and the k-mer operands of the
//     lane's offsets live in registers.  A band move shifts either the k-mer
//     operands (k-mer move) or the events (event move) by one offset; the
//     one value that crosses a lane boundary travels by __shfl_*_sync.  The
//     value entering at the band end comes from a warp-wide prefetch window
//     (lane i holds the i-th next event / k-mer entry, with the following 32
//     already in flight), so no band waits on global memory;
//   - the neighbours of a cell are a +-0/1 offset shift of the previous one
//     or two bands, selected by the last two moves; the four cases are
//     compiled separately so every register index is static;
//   - the direction of every cell is two predicates (U over D; L over the
//     max), gathered across the warp by __ballot_sync into 2C words per band
//     and stored by lane 0 (2 bits per cell), plus the band's offset-0 event
//     index (4 B); no score array is ever written;
//   - cells outside the matrix need no per-cell test: a missing event reads
//     +inf and a missing k-mer reads (a=1, b=0, c=-inf), which make the
//     emission -inf; the only cells this leaves finite lie beyond the last
//     k-mer, which no in-matrix cell reads, and the band-move decision
//     clamps those to -inf;
//   - bands whose W offsets all lie in the matrix run a lean loop (no trim,
//     end or bound checks); the rest run the same step with those checks;
//   - after the last band the same warp picks the end cell and walks the
//     trace back: the records of 32 bands at a time sit in the lanes'
//     registers (the next 32 in flight), each step takes its two trace words
//     and the next bands' ll_e by shuffle, and the pairs are gathered across
//     the lanes and stored 32 at a time.
//
// All FP32 arithmetic uses explicitly rounded intrinsics, so no operation is
// fused or reordered: the scores equal those of the FP32 canonical form
//   z = fmaf(x, a, b); E = fmaf(-z, z, c);
//   d = diag + lp_step; u = up + lp_stay; m = (u > d) ? u : d; s = m + E;
//   l = left + lp_skip; S = (l > s) ? l : s
// (max(diag+lp_step+E, up+lp_stay+E) = max(diag+lp_step, up+lp_stay) + E
// because rounding is monotone).
#include <climits>

#include "abea_internal.h"

namespace abea {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }
__device__ __forceinline__ float pos_inf() { return __int_as_float(0x7f800000); }

struct Consts {
    float lp_skip, lp_stay, lp_step, lp_trim;
};

__device__ __forceinline__ float cell(float up, float left, float diag, float x, float a, float b, float c,
                                      const Consts &cs, bool &p0, bool &p1)
{
    const float z = __fmaf_rn(x, a, b);
    const float em = __fmaf_rn(-z, z, c);
    const float d = __fadd_rn(diag, cs.lp_step);
    const float u = __fadd_rn(up, cs.lp_stay);
    p0 = u > d;
    const float m = p0 ? u : d;
    const float s = __fadd_rn(m, em);
    const float l = __fadd_rn(left, cs.lp_skip);
    p1 = l > s;
    return p1 ? l : s;
}

__device__ __forceinline__ float4 kmer_operands(const float4 *kc, int k, int n_k)
{
    if ((unsigned)k < (unsigned)n_k) return kc[k];
    return make_float4(1.0f, 0.0f, neg_inf(), 0.0f);
}

__device__ __forceinline__ float event_value(const float *ev, int e, int n_e)
{
    return ((unsigned)e < (unsigned)n_e) ? ev[e] : pos_inf();
}

// Lane state other than the two score bands.
template <int C>
struct Lane {
    float X[C], A[C], B[C], Cc[C];   // operands of the lane's offsets
    float qprev;                     // boundary value of the previous band's shifted view
    bool kprev;                      // previous move advanced the k-mer
    int ll_e, ll_k;                  // offset-0 cell of the last computed band
    float xnext;                     // event entering at offset 0 on the next event move
    float4 knext;                    // k-mer operands entering at offset W'-1 on the next k-mer move
    float ev_cur, ev_nxt;            // prefetch window: event ev_base + lane, and 32 further
    int ev_base;
    float4 kc_cur, kc_nxt;           // prefetch window: k-mer kc_base + lane, and 32 further
    int kc_base;
    int b;                           // next band to compute
    int re, rk;                      // steady-loop budgets: event / k-mer moves left
    double frame;                    // total shift applied to the scores so far (see renormalise)
    double best;                     // best end candidate seen by this lane (unshifted)
    int best_e;
    long long cells;
};

struct ReadCtx {
    const float *ev;
    const float4 *kc;
    uint32_t *tr;
    int32_t *lle;
    int n_e, n_k, W, Wp, L, lane;
    bool first_lane, last_lane;
    unsigned dead_mask;              // slots of this lane beyond offset W-1
    Consts cs;
};

// Band b from S_{b-1} (P) and S_{b-2} (PP); S_b is written into PP.
// KM: this band moves by one k-mer; KP: the previous band did.
template <int C, bool KM, bool KP>
__device__ __forceinline__ void band_fill(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C],
                                          bool (&p0)[C], bool (&p1)[C])
{
    // operands of band b
    if (KM) {
        const float sa = __shfl_down_sync(kFull, s.A[0], 1);
        const float sb = __shfl_down_sync(kFull, s.B[0], 1);
        const float sc = __shfl_down_sync(kFull, s.Cc[0], 1);
#pragma unroll
        for (int i = 0; i < C - 1; i++) {
            s.A[i] = s.A[i + 1];
            s.B[i] = s.B[i + 1];
            s.Cc[i] = s.Cc[i + 1];
        }
        s.A[C - 1] = r.last_lane ? s.knext.x : sa;
        s.B[C - 1] = r.last_lane ? s.knext.y : sb;
        s.Cc[C - 1] = r.last_lane ? s.knext.z : sc;
    } else {
        const float sx = __shfl_up_sync(kFull, s.X[C - 1], 1);
#pragma unroll
        for (int i = C - 1; i > 0; i--) s.X[i] = s.X[i - 1];
        s.X[0] = r.first_lane ? s.xnext : sx;
    }
    // Q[t] = S_{b-1}[C*lane + t - 1 + KM], t = 0..C: left of slot i is Q[i], up is Q[i+1]
    float qb;
    if (KM) {
        qb = __shfl_down_sync(kFull, P[0], 1);
        if (r.last_lane) qb = neg_inf();
    } else {
        qb = __shfl_up_sync(kFull, P[C - 1], 1);
        if (r.first_lane) qb = neg_inf();
    }
    float S[C];
#pragma unroll
    for (int i = 0; i < C; i++) {
        const float left = KM ? P[i] : (i == 0 ? qb : P[i > 0 ? i - 1 : 0]);
        const float up = KM ? (i == C - 1 ? qb : P[i < C - 1 ? i + 1 : 0]) : P[i];
        // diag = previous band's Q at t = i + KM
        const int t = i + (KM ? 1 : 0);
        float diag;
        if (KP) diag = (t == C) ? s.qprev : PP[t < C ? t : 0];
        else diag = (t == 0) ? s.qprev : PP[t > 0 ? t - 1 : 0];
        S[i] = cell(up, left, diag, s.X[i], s.A[i], s.B[i], s.Cc[i], r.cs, p0[i], p1[i]);
    }
#pragma unroll
    for (int i = 0; i < C; i++) PP[i] = S[i];
    s.qprev = qb;
}

template <int C>
__device__ __forceinline__ void band_fill_dispatch(bool K, Lane<C> &s, const ReadCtx &r, float (&P)[C],
                                                   float (&PP)[C], bool (&p0)[C], bool (&p1)[C])
{
    if (K) {
        if (s.kprev) band_fill<C, true, true>(s, r, P, PP, p0, p1);
        else band_fill<C, true, false>(s, r, P, PP, p0, p1);
    } else {
        if (s.kprev) band_fill<C, false, true>(s, r, P, PP, p0, p1);
        else band_fill<C, false, false>(s, r, P, PP, p0, p1);
    }
}

// The value of S_{b-1} at offset W-1.
template <int C, bool MIXED>
__device__ __forceinline__ float far_end(const ReadCtx &r, const float (&P)[C])
{
    if (!MIXED) return __shfl_sync(kFull, P[C - 1], r.L - 1);
    const int j = r.W - 1, slot = j % C;
    float v = P[0];
#pragma unroll
    for (int i = 1; i < C; i++)
        if (slot == i) v = P[i];
    return __shfl_sync(kFull, v, j / C);
}

// Every 64th band of the lean loop, the band just computed and the one before
// (both wholly in the matrix) are shifted up by R, a multiple of 1024 no
// larger in magnitude than their maximum.  Each shifted value is exactly
// representable, so the shift decides nothing by itself; it keeps the running
// scores small so that later FP32 additions round at a fine ulp instead of
// drifting on long reads.  The total shift is kept in FP64 and added back to
// the end score.  The FP32 oracle applies the same shifts at the same bands.
constexpr int kRenormPeriod = 64;

template <int C>
__device__ __forceinline__ void renormalise(Lane<C> &s, const ReadCtx &r, float (&Sb)[C], float (&Sb1)[C])
{
    float m = neg_inf();
    if (r.lane < r.L) {
#pragma unroll
        for (int i = 0; i < C; i++)
            if (!((r.dead_mask >> i) & 1u)) m = fmaxf(m, fmaxf(Sb[i], Sb1[i]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, off));
    if (m <= -2048.0f) {
        const float R = -1024.0f * floorf(__fmul_rn(-m, 1.0f / 1024.0f));
#pragma unroll
        for (int i = 0; i < C; i++) {
            Sb[i] = __fsub_rn(Sb[i], R);
            Sb1[i] = __fsub_rn(Sb1[i], R);
        }
        s.qprev = __fsub_rn(s.qprev, R);
        s.frame += (double)R;
    }
}

// Next injected event (index e) from the prefetch window; e never skips ahead
// of the window by more than one step.
template <int C>
__device__ __forceinline__ void next_event(Lane<C> &s, const ReadCtx &r, int e)
{
    int idx = e - s.ev_base;
    if (idx >= 32) {
        s.ev_cur = s.ev_nxt;
        s.ev_base += 32;
        idx -= 32;
        s.ev_nxt = event_value(r.ev, s.ev_base + 32 + r.lane, r.n_e);
    }
    s.xnext = __shfl_sync(kFull, s.ev_cur, idx);
}

template <int C>
__device__ __forceinline__ void next_kmer(Lane<C> &s, const ReadCtx &r, int k)
{
    int idx = k - s.kc_base;
    if (idx >= 32) {
        s.kc_cur = s.kc_nxt;
        s.kc_base += 32;
        idx -= 32;
        s.kc_nxt = kmer_operands(r.kc, s.kc_base + 32 + r.lane, r.n_k);
    }
    s.knext.x = __shfl_sync(kFull, s.kc_cur.x, idx);
    s.knext.y = __shfl_sync(kFull, s.kc_cur.y, idx);
    s.knext.z = __shfl_sync(kFull, s.kc_cur.z, idx);
}

// One band: decision, fill, (checks), trace record, bookkeeping.
// GENERAL: the band may touch the matrix edges (trim column, end cells,
// cells outside the matrix); otherwise every offset of band b-1 and b lies
// in the matrix.
template <int C, bool MIXED, bool GENERAL>
__device__ __forceinline__ void band_step(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C])
{
    const int b = s.b;
    float lo = __shfl_sync(kFull, P[0], 0);
    float hi = far_end<C, MIXED>(r, P);
    bool K;
    if (GENERAL) {
        // cells beyond the last k-mer are not -inf in registers; clamp the ends
        if (s.ll_k >= r.n_k) lo = neg_inf();
        if (s.ll_k + r.W - 1 >= r.n_k) hi = neg_inf();
        K = (lo == neg_inf() && hi == neg_inf()) ? ((b & 1) != 0) : (lo < hi);
    } else {
        K = lo < hi;
    }
    bool p0[C], p1[C];
    band_fill_dispatch<C>(K, s, r, P, PP, p0, p1);
    if (!GENERAL && (b % kRenormPeriod) == 0) renormalise<C>(s, r, PP, P);
    s.kprev = K;
    if (K) {
        s.ll_k++;
        s.rk--;
    } else {
        s.ll_e++;
        s.re--;
    }
    if (MIXED) {
#pragma unroll
        for (int i = 0; i < C; i++)
            if (r.dead_mask & (1u << i)) PP[i] = neg_inf();
    }
    if (GENERAL) {
        // trim state: the cell (e,-1) scores (e+1)*lp_trim
        if (s.ll_k < 0) {
            const int jt = -1 - s.ll_k;
            const int e = s.ll_e - jt;
            const float v = (e >= 0 && e < r.n_e) ? __fmul_rn((float)(e + 1), r.cs.lp_trim) : neg_inf();
#pragma unroll
            for (int i = 0; i < C; i++)
                if (C * r.lane + i == jt) PP[i] = v;
        }
        // end cell candidates: (e, n_k-1) plus the n_e-1-e trailing events trimmed
        const int jend = r.n_k - 1 - s.ll_k;
        if (jend >= 0 && jend < r.W) {
            const int e = s.ll_e - jend;
            if (e >= 0 && e < r.n_e) {
#pragma unroll
                for (int i = 0; i < C; i++) {
                    if (C * r.lane + i == jend) {
                        const float rel = __fadd_rn(PP[i], __fmul_rn((float)(r.n_e - 1 - e), r.cs.lp_trim));
                        const double cand = s.frame + (double)rel;
                        if (cand > s.best) {
                            s.best = cand;
                            s.best_e = e;
                        }
                    }
                }
            }
        }
        // in-matrix cells of this band
        int jlo = max(0, max(s.ll_e - r.n_e + 1, -s.ll_k));
        int jhi = min(r.W, min(s.ll_e + 1, r.n_k - s.ll_k));
        s.cells += max(0, jhi - jlo);
    } else {
        s.cells += r.W;
    }
    // trace: 2 bits per cell as 2C ballots; one move byte per band
    uint32_t w[2 * C];
#pragma unroll
    for (int i = 0; i < C; i++) {
        w[2 * i] = __ballot_sync(kFull, p0[i]);
        w[2 * i + 1] = __ballot_sync(kFull, p1[i]);
    }
    if (r.lane == 0) {
        constexpr int R = (2 * C + 3) / 4 * 4;
        uint4 *dst = reinterpret_cast<uint4 *>(r.tr + (size_t)b * R);
#pragma unroll
        for (int q = 0; q < R / 4; q++) {
            uint4 v;
            v.x = (4 * q + 0 < 2 * C) ? w[(4 * q + 0) % (2 * C)] : 0u;
            v.y = (4 * q + 1 < 2 * C) ? w[(4 * q + 1) % (2 * C)] : 0u;
            v.z = (4 * q + 2 < 2 * C) ? w[(4 * q + 2) % (2 * C)] : 0u;
            v.w = (4 * q + 3 < 2 * C) ? w[(4 * q + 3) % (2 * C)] : 0u;
            dst[q] = v;
        }
        r.lle[b] = s.ll_e;
    }
    // the operand the next move of this kind will inject
    if (K) next_kmer(s, r, s.ll_k + r.Wp);
    else next_event(s, r, s.ll_e + 1);
    s.b = b + 1;
}

template <int C>
__device__ __forceinline__ void swap_bands(float (&P)[C], float (&PP)[C])
{
#pragma unroll
    for (int i = 0; i < C; i++) {
        const float t = P[i];
        P[i] = PP[i];
        PP[i] = t;
    }
}

template <int C>
__device__ __forceinline__ bool steady_ok(Lane<C> &s, const ReadCtx &r)
{
    // bands b-1 and b both lie in the matrix whichever move b makes
    // (the k-mer budget keeps the end column k = n_k-1 out of band b)
    s.re = r.n_e - 1 - s.ll_e;
    s.rk = r.n_k - r.W - 1 - s.ll_k;
    return s.ll_e >= r.W - 1 && s.ll_k >= 0 && s.re > 0 && s.rk > 0;
}

// Trace records of bands top-lane (lane 0 = band top), with the ll_e of the
// two bands below each.
template <int C>
struct Chunk {
    static constexpr int R = (2 * C + 3) / 4 * 4;
    uint32_t rec[R];
    int l1, l2;
};

template <int C>
__device__ __forceinline__ void load_chunk(const ReadCtx &r, int top, Chunk<C> &c)
{
    const int mb = top - r.lane;
    if (mb >= 2) {                        // bands 0 and 1 hold no matrix cell and are never visited
        const uint4 *src = reinterpret_cast<const uint4 *>(r.tr + (size_t)mb * Chunk<C>::R);
#pragma unroll
        for (int q = 0; q < Chunk<C>::R / 4; q++) {
            const uint4 v = src[q];
            c.rec[4 * q] = v.x;
            c.rec[4 * q + 1] = v.y;
            c.rec[4 * q + 2] = v.z;
            c.rec[4 * q + 3] = v.w;
        }
        c.l1 = r.lle[mb - 1];
        c.l2 = r.lle[mb - 2];
    }
}

// Walk the trace from (e_end, n_k-1) until an index leaves the matrix,
// writing pair t of the walk to out[cap-1-t] (t < cap).  Returns 0, or -1
// if a traced cell lies outside its band (cannot happen); n = pairs walked.
template <int C>
__device__ int backtrack(const ReadCtx &r, int e_end, int2 *out, int cap, int &n_out)
{
    const int lane = r.lane;
    int e = e_end, k = r.n_k - 1;
    int bb = e + k + 2;
    int le = r.lle[bb];
    int top = bb;
    Chunk<C> cur, nxt;
    load_chunk<C>(r, top, cur);
    load_chunk<C>(r, top - 32, nxt);
    int n = 0;
    int2 mine = make_int2(0, 0);
    int status = 0;
    while (e >= 0 && k >= 0) {
        if (bb < top - 31) {
            cur = nxt;
            top -= 32;
            load_chunk<C>(r, top - 32, nxt);
        }
        const int src = top - bb;
        const int j = le - e;
        if (j < 0 || j >= r.W) {
            status = -1;
            break;
        }
        const int slot = j % C;
        const unsigned bit = (unsigned)(j / C);
        uint32_t s0 = cur.rec[0], s1 = cur.rec[1];
#pragma unroll
        for (int i = 1; i < C; i++) {
            if (slot == i) {
                s0 = cur.rec[2 * i];
                s1 = cur.rec[2 * i + 1];
            }
        }
        const uint32_t w0 = __shfl_sync(kFull, s0, src);
        const uint32_t w1 = __shfl_sync(kFull, s1, src);
        const int lm1 = __shfl_sync(kFull, cur.l1, src);
        const int lm2 = __shfl_sync(kFull, cur.l2, src);
        if (lane == (n & 31)) mine = make_int2(e, k);
        n++;
        if ((n & 31) == 0) {                    // pairs n-32 .. n-1 -> out[cap-n .. cap-n+31], descending
            const int t = n - 32 + lane;
            if (t < cap) out[cap - 1 - t] = mine;
        }
        if ((w1 >> bit) & 1u) {                 // L
            k--;
            bb--;
            le = lm1;
        } else if ((w0 >> bit) & 1u) {          // U
            e--;
            bb--;
            le = lm1;
        } else {                                // D
            e--;
            k--;
            bb -= 2;
            le = lm2;
        }
    }
    const int rest = n & 31;
    if (rest) {
        const int t = n - rest + lane;
        if (lane < rest && t < cap) out[cap - 1 - t] = mine;
    }
    n_out = n;
    return status;
}

template <int C, bool MIXED>
__device__ void align_read(const AlignArgs &a, const ReadDesc &d, int rid, int lane)
{
    ReadCtx r;
    r.ev = a.events + d.ev_off;
    r.kc = a.kc + d.kc_off;
    r.tr = a.trace + d.tr_off;
    r.lle = a.lle + d.ll_off;
    r.n_e = d.n_e;
    r.n_k = d.n_k;
    r.W = a.W;
    r.L = a.L;
    r.Wp = C * a.L;
    r.lane = lane;
    r.first_lane = lane == 0;
    r.last_lane = lane == a.L - 1;
    r.dead_mask = 0;
#pragma unroll
    for (int i = 0; i < C; i++)
        if (C * lane + i >= a.W) r.dead_mask |= 1u << i;
    r.cs = Consts{d.lp_skip, d.lp_stay, d.lp_step, d.lp_trim};

    const int W = a.W, half = W / 2;
    Lane<C> s;
    float P[C], PP[C];
    // bands 0 and 1: the origin (-1,-1) at offset W/2 of band 0 (score 0);
    // band 1 = band 0 moved by one event, the trim cell (0,-1) at offset W/2.
    s.ll_e = half;
    s.ll_k = -1 - half;
#pragma unroll
    for (int i = 0; i < C; i++) {
        const int j = C * lane + i;
        PP[i] = (j == half) ? 0.0f : neg_inf();
        P[i] = (j == half) ? d.lp_trim : neg_inf();
        s.X[i] = event_value(r.ev, s.ll_e - j, r.n_e);
        const float4 q = kmer_operands(r.kc, s.ll_k + j, r.n_k);
        s.A[i] = q.x;
        s.B[i] = q.y;
        s.Cc[i] = q.z;
    }
    // band 1's shifted view of band 0 (band 1 moved by one event)
    s.qprev = __shfl_up_sync(kFull, PP[C - 1], 1);
    if (r.first_lane) s.qprev = neg_inf();
    s.kprev = false;
    s.ev_base = s.ll_e + 1;
    s.ev_cur = event_value(r.ev, s.ev_base + lane, r.n_e);
    s.ev_nxt = event_value(r.ev, s.ev_base + 32 + lane, r.n_e);
    s.kc_base = s.ll_k + r.Wp;
    s.kc_cur = kmer_operands(r.kc, s.kc_base + lane, r.n_k);
    s.kc_nxt = kmer_operands(r.kc, s.kc_base + 32 + lane, r.n_k);
    next_event(s, r, s.ll_e + 1);
    next_kmer(s, r, s.ll_k + r.Wp);
    s.b = 2;
    s.frame = 0.0;
    s.best = -(double)pos_inf();
    s.best_e = INT_MAX;
    s.cells = 0;
    if (lane == 0) {
        r.lle[0] = half - 1;
        r.lle[1] = half;
    }

    const int b_end = r.n_e + r.n_k;
    while (s.b <= b_end) {
        if (steady_ok(s, r)) {
            for (;;) {
                band_step<C, MIXED, false>(s, r, P, PP);     // S_b in PP
                if (!(s.re > 0 && s.rk > 0)) {
                    swap_bands(P, PP);
                    break;
                }
                band_step<C, MIXED, false>(s, r, PP, P);     // S_b in P
                if (!(s.re > 0 && s.rk > 0)) break;
            }
        } else {
            band_step<C, MIXED, true>(s, r, P, PP);
            swap_bands(P, PP);
        }
    }

    // end cell: max score, then smallest event (the first maximum in event order)
    double best = s.best;
    int best_e = s.best_e;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(kFull, best, off);
        const int oe = __shfl_xor_sync(kFull, best_e, off);
        if (ob > best || (ob == best && oe < best_e)) {
            best = ob;
            best_e = oe;
        }
    }
    long long cells = s.cells;   // identical in every lane

    int status = ABEA_READ_OK;
    int n = 0;
    int2 *out = reinterpret_cast<int2 *>(a.pairs) + d.pair_off;
    const int cap = d.pair_cap;
    if (best == -(double)pos_inf()) {
        status = ABEA_READ_FAIL_NO_END;
    } else {
        __syncwarp();                         // lane 0's trace and ll_e stores are visible to the warp
        status = backtrack<C>(r, best_e, out, cap, n);
        if (status == ABEA_READ_OK && n <= cap) {
            __syncwarp();
            for (int base = 0; base < n; base += 32) {   // move pairs to the front, ascending
                const int t = base + lane;
                int2 v = make_int2(0, 0);
                if (t < n) v = out[cap - n + t];
                __syncwarp();
                if (t < n) out[t] = v;
                __syncwarp();
            }
        } else if (status == ABEA_READ_OK) {
            status = ABEA_READ_CAPACITY;
        } else {
            status = ABEA_READ_FAIL_NO_END;   // internal inconsistency, reported as no alignment
            n = 0;
        }
    }
    if (lane == 0) {
        abea_result res;
        res.score = (status == ABEA_READ_OK || status == ABEA_READ_CAPACITY) ? __double2float_rn(best) : neg_inf();
        res.status = status;
        res.n_pairs = (status == ABEA_READ_FAIL_NO_END) ? 0 : n;
        res.e_end = (status == ABEA_READ_FAIL_NO_END) ? -1 : best_e;
        res.cells = cells;
        a.res[rid] = res;
    }
}

template <int C, bool MIXED>
__global__ void __launch_bounds__(128) align_kernel(const AlignArgs a)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(a.queue, 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= a.n) break;
        const int rid = a.order[q];
        const ReadDesc d = a.rd[rid];
        if (d.host_bad || a.flags[rid]) {
            if (lane == 0) {
                abea_result res;
                res.score = neg_inf();
                res.status = ABEA_READ_BAD_INPUT;
                res.n_pairs = 0;
                res.e_end = -1;
                res.cells = 0;
                a.res[rid] = res;
            }
            continue;
        }
        align_read<C, MIXED>(a, d, rid, lane);
    }
}

template <int C, bool MIXED>
int launch_c(const AlignArgs &a, int grid, void *stream)
{
    align_kernel<C, MIXED><<<grid, 128, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

template <int C, bool MIXED>
int grid_c(int device)
{
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, align_kernel<C, MIXED>, 128, 0);
    if (e != cudaSuccess || per_sm < 1) return -1;
    return sms * per_sm;
}

}  // namespace

Geometry geometry_for(int W)
{
    Geometry g{};
    const int cmin = (W + 31) / 32;
    int C = cmin;
    for (int c = cmin; c <= 8; c++) {
        if (W % c == 0) {
            C = c;
            break;
        }
    }
    g.C = C;
    g.L = (W + C - 1) / C;
    g.Wp = C * g.L;
    g.mixed = g.Wp != W;
    g.rec_words = (2 * C + 3) / 4 * 4;
    return g;
}

#define ABEA_FOR_EACH_C(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

int launch_align(const AlignArgs &a, int C, bool mixed, int grid, void *stream)
{
#define X(c)                                                                       \
    if (C == c) return mixed ? launch_c<c, true>(a, grid, stream) : launch_c<c, false>(a, grid, stream);
    ABEA_FOR_EACH_C(X)
#undef X
    return (int)cudaErrorInvalidValue;
}

int align_grid_size(int C, bool mixed, int device)
{
#define X(c)                                                                       \
    if (C == c) return mixed ? grid_c<c, true>(device) : grid_c<c, false>(device);
    ABEA_FOR_EACH_C(X)
#undef X
    return -1;
}

}  // namespace abea
