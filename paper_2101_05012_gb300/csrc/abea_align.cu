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
//     [C*l, C*l + C) of every band; L = ceil(W/C) lanes are live.  The lanes
//     above hold -inf scores and "no k-mer" operands (and an lp_skip of
//     -inf), so they are the -inf edge of the band without any per-band test;
//   - the previous band, the band before it (as the view the previous band
//     read it through) and the events and k-mer operands of the lane's
//     offsets live in registers.  A band move shifts either the k-mer
//     operands (k-mer move) or the events (event move) by one offset; the one
//     value that crosses a lane boundary travels by __shfl_*_sync.  The value
//     entering at the band end comes from a per-warp ring in shared memory,
//     refilled by cp.async once per run of bands;
//   - the neighbours of a cell are a +-0/1 offset shift of the previous band
//     (left, up) and of the stored view of the band before it (diagonal),
//     selected by the band's own move only; the two cases are compiled
//     separately so every register index is static;
//   - the move of band b+1 is decided at the end of band b (two shuffles of
//     its end cells), so the decision overlaps band b's bookkeeping;
//   - the direction of every cell is two predicates (U over D; L over the
//     max), gathered by __ballot_sync into 2C words per band and stored by
//     the warp in one wide store (2 bits per cell); the band's move rides in
//     bit 31 of its first word (lane 31 lies above the band); no score array
//     is ever written;
//   - cells outside the matrix need no per-cell test: a missing event reads
//     +inf and a missing k-mer reads (a=1, b=0, c=-inf), which make the
//     emission -inf; the only cells this leaves finite lie beyond the last
//     k-mer, which no in-matrix cell reads, and the band-move decision
//     clamps those to -inf;
//   - runs of bands whose W offsets all lie in the matrix go through a lean
//     loop controlled by one counter (no trim, end or bound checks); the rest
//     run the same step with those checks;
//   - after the last band the trace is walked back: the records of 32 bands
//     at a time are copied to shared memory with cp.async, two chunks ahead
//     of the walk; each step reads its two trace bits there and the band
//     moves give each band's position.  A warp walks its reads two at a
//     time, half a warp each, while the queue lasts (a read's walk waits for
//     the warp's next read), and one at a time with the whole warp in the
//     queue's tail.

// All FP32 arithmetic uses explicitly rounded intrinsics, so no operation is
// fused or reordered: the scores equal those of the FP32 canonical form,
// in which every cell carries T = S + lp_step (S the recurrence's score):
//   z = fmaf(x, a, b); E' = fmaf(-z, z, c'), c' = c + lp_step (E' = E + lp_step);
//   d = diag; u = up + (lp_stay - lp_step); m = (u > d) ? u : d; s = m + E';
//   l = left + lp_skip; T = (l > s) ? l : s
// (in exact arithmetic T_d = S_diag + lp_step + E + lp_step = T_diag + E',
// T_u = T_up + (lp_stay - lp_step) + E', T_l = T_left + lp_skip; and
// max(d + E', u + E') = max(d, u) + E' because rounding is monotone).  The
// origin scores lp_step, the trim column (e+1)*lp_trim + lp_step, and the
// end score subtracts lp_step in FP64.  Plus the exact renormalisation below.
#include <algorithm>
#include <climits>

#include "abea_internal.h"

namespace abea {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;          // warps per block
constexpr int kChunk = 32;         // bands per backtrack chunk
constexpr int kRenormPeriod = 64;

// Dynamic shared memory of the core kernel: the walk's record rings (one per
// warp), then the block-mode exchange state.  Declared once so that every
// function, including the out-of-line block mode, addresses it as shared.
extern __shared__ __align__(16) uint32_t abea_smem[];

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }
__device__ __forceinline__ float pos_inf() { return __int_as_float(0x7f800000); }

struct Consts {
    float lp_skip, lp_stay_step, lp_step, lp_trim;   // lp_stay_step = lp_stay - lp_step
};

// One cell in the T = S + lp_step form (c includes lp_step).
__device__ __forceinline__ float cell(float up, float left, float diag, float x, float a, float b, float c,
                                      float lp_stay_step, float lp_skip, bool &p0, bool &p1)
{
    const float z = __fmaf_rn(x, a, b);
    const float em = __fmaf_rn(-z, z, c);
    const float d = diag;
    const float u = __fadd_rn(up, lp_stay_step);
    p0 = u > d;
    const float m = p0 ? u : d;
    const float s = __fadd_rn(m, em);
    const float l = __fadd_rn(left, lp_skip);
    p1 = l > s;
    return p1 ? l : s;
}

__device__ __forceinline__ float4 no_kmer() { return make_float4(1.0f, 0.0f, neg_inf(), 0.0f); }

__device__ __forceinline__ float4 kmer_operands(const float4 *kc, int k, int n_k)
{
    if ((unsigned)k < (unsigned)n_k) return kc[k];
    return no_kmer();
}

__device__ __forceinline__ float event_value(const float *ev, int e, int n_e)
{
    return ((unsigned)e < (unsigned)n_e) ? ev[e] : pos_inf();
}

template <int C>
struct Rec {
    static constexpr int R = (2 * C + 3) / 4 * 4;   // trace words per band
};

// State of a read that the lean loop never touches.  Kept per lane in shared
// memory rather than registers, so that the lean loop's live registers fit
// the occupancy it runs at: it is read and written only by bands run with
// checks, by the renormalisation and at the end of the read.
struct Cold {
    double frame;                    // total renormalisation shift so far
    double best;                     // best end candidate seen by this lane (unshifted)
    long long cells;                 // in-matrix cells of bands run with checks
    long long lean_bands;            // bands run by the lean loop (W cells each)
    int best_e, best_le;
};

// Lane state other than the two score bands.
template <int C>
struct Lane {
    float X[C], A[C], B[C], Cc[C];   // operands of the lane's offsets
    float qprev;                     // boundary value of the previous band's shifted view
    float nb_lo, nb_hi;              // block mode: S_b of the neighbour warps at offsets off0-1 and off0+W'
    bool kprev;                      // the last band moved by one k-mer
    bool knext;                      // the next band moves by one k-mer (decided)
    int ll_e, ll_k;                  // offset-0 cell of the last computed band
    float xin;                       // event entering at offset 0 on the next event move
    float4 kin;                      // k-mer operands entering at offset W'-1 on the next k-mer move
    float ev_cur, ev_nxt;            // prefetch window: event ev_base + lane, and 32 further
    int ev_base;
    float4 kc_cur, kc_nxt;           // prefetch window: k-mer kc_base + lane, and 32 further
    int kc_base;
    int b;                           // next band to compute
    Cold *cold;                      // the read's state the lean loop never touches
};

struct ReadCtx {
    const float *ev;
    const float4 *kc;
    uint32_t *tr;
    uint8_t *mv;                     // per-band move bytes (only when no lane lies above the band)
    int n_e, n_k, W, Wp, L, lane, src_up;
    bool first_lane, last_lane, lane31;
    unsigned dead_mask;              // slots of this lane beyond offset W-1
    float lsk;                       // lp_skip; -inf above the band
    Consts cs;
    // block mode (the block's warps share one read; warp gw owns offsets
    // [off0, off0 + W') of every band, W' = W / kWarps)
    int off0, gw;
    float2 *xch;                     // [2][kWarps] band edges (S at off0, S at off0+W'-1), by band parity
    float *rx;                       // [kWarps] renormalisation maxima
};

// Band b from S_{b-1} (P) and S_{b-2} (PP); S_b is written into PP and its
// trace words into w.  KM: this band moves by one k-mer; KP: the previous
// band did.  FULLW: all 32 lanes are live (no lane above the band).
template <int C, bool KM, bool KP, bool FULLW, bool GROUP>
__device__ __forceinline__ void band_fill(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C],
                                          uint32_t (&w)[2 * C])
{
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
        s.A[C - 1] = r.last_lane ? s.kin.x : sa;
        s.B[C - 1] = r.last_lane ? s.kin.y : sb;
        s.Cc[C - 1] = r.last_lane ? s.kin.z : sc;
    } else {
        const float sx = __shfl_sync(kFull, s.X[C - 1], r.src_up);
#pragma unroll
        for (int i = C - 1; i > 0; i--) s.X[i] = s.X[i - 1];
        s.X[0] = r.first_lane ? s.xin : sx;
    }
    // Q[t] = S_{b-1}[C*lane + t - 1 + KM], t = 0..C: left of slot i is Q[i],
    // up is Q[i+1].  Across the band's edges the neighbour lane is a lane
    // above the band (all -inf), unless FULLW; in block mode the value across
    // the warp's edge comes from the neighbour warp.
    float qb;
    if (KM) {
        qb = __shfl_down_sync(kFull, P[0], 1);
        if (FULLW && r.last_lane) qb = neg_inf();
        if (GROUP && r.last_lane) qb = s.nb_hi;
    } else {
        qb = __shfl_sync(kFull, P[C - 1], r.src_up);
        if (FULLW && r.first_lane) qb = neg_inf();
        if (GROUP && r.first_lane) qb = s.nb_lo;
    }
    float S[C];
#pragma unroll
    for (int i = 0; i < C; i++) {
        const float left = KM ? P[i] : (i == 0 ? qb : P[i > 0 ? i - 1 : 0]);
        const float up = KM ? (i == C - 1 ? qb : P[i < C - 1 ? i + 1 : 0]) : P[i];
        const int t = i + (KM ? 1 : 0);      // diag = the previous band's Q at t
        float diag;
        if (KP) diag = (t == C) ? s.qprev : PP[t < C ? t : 0];
        else diag = (t == 0) ? s.qprev : PP[t > 0 ? t - 1 : 0];
        bool p0, p1;
        S[i] = cell(up, left, diag, s.X[i], s.A[i], s.B[i], s.Cc[i], r.cs.lp_stay_step, r.lsk, p0, p1);
        if (!FULLW && i == 0) p0 = r.lane31 ? KM : p0;     // the band's move, bit 31 of word 0
        w[2 * i] = __ballot_sync(kFull, p0);
        w[2 * i + 1] = __ballot_sync(kFull, p1);
    }
#pragma unroll
    for (int i = 0; i < C; i++) PP[i] = S[i];
    s.qprev = qb;
}

template <int C, bool FULLW, bool GROUP>
__device__ __forceinline__ void band_fill_dispatch(bool K, Lane<C> &s, const ReadCtx &r, float (&P)[C],
                                                   float (&PP)[C], uint32_t (&w)[2 * C])
{
    if (K) {
        if (s.kprev) band_fill<C, true, true, FULLW, GROUP>(s, r, P, PP, w);
        else band_fill<C, true, false, FULLW, GROUP>(s, r, P, PP, w);
    } else {
        if (s.kprev) band_fill<C, false, true, FULLW, GROUP>(s, r, P, PP, w);
        else band_fill<C, false, false, FULLW, GROUP>(s, r, P, PP, w);
    }
}

// Block mode: barrier over the block's warps (all of them share the read).
__device__ __forceinline__ void group_sync() { asm volatile("bar.sync 1, %0;\n" ::"n"(kWarps * 32) : "memory"); }

// Block mode: publish band b's edge cells (S = S_b), wait for the other warps,
// then read the band's end cells (offsets 0 and W-1) and the neighbour
// warps' edges for the next band.  Slots alternate by band parity, so one
// barrier per band suffices: a slot is rewritten two bands later, after
// every warp has passed the barrier that follows its reads.
template <int C>
__device__ __forceinline__ void group_exchange(Lane<C> &s, const ReadCtx &r, int b, const float (&S)[C], float &lo,
                                               float &hi)
{
    float2 *x = r.xch + (b & 1) * kWarps;
    if (r.first_lane) x[r.gw].x = S[0];
    if (r.last_lane) x[r.gw].y = S[C - 1];
    group_sync();
    lo = x[0].x;
    hi = x[kWarps - 1].y;
    s.nb_lo = (r.gw > 0) ? x[r.gw > 0 ? r.gw - 1 : 0].y : neg_inf();
    s.nb_hi = (r.gw < kWarps - 1) ? x[r.gw < kWarps - 1 ? r.gw + 1 : 0].x : neg_inf();
}

// The value of a band at offset W-1.
template <int C, bool MIXED, int N>
__device__ __forceinline__ float far_end(const ReadCtx &r, const float (&S)[N])
{
    if (!MIXED) return __shfl_sync(kFull, S[C - 1], r.L - 1);
    const int j = r.W - 1, slot = j % C;
    float v = S[0];
#pragma unroll
    for (int i = 1; i < C; i++)
        if (slot == i) v = S[i];
    return __shfl_sync(kFull, v, j / C);
}

// Exact renormalisation.  After the lean loop's bands with b % 64 == 0, the
// band just computed and the one before (both wholly in the matrix) are
// shifted up by R, a multiple of 1024 no larger in magnitude than their
// maximum (only when that maximum is <= -2048).  Each shifted value is
// exactly representable, so the shift decides nothing by itself; it keeps the
// running scores small so that later FP32 additions round at a fine ulp
// instead of drifting on long reads.  The total shift is kept in FP64 and
// added back to the end score.  The FP32 oracle applies the same shifts.
template <int C, bool GROUP>
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
    if (GROUP) {                       // the maximum over the whole band
        if (r.first_lane) r.rx[r.gw] = m;
        group_sync();
#pragma unroll
        for (int g = 0; g < kWarps; g++) m = fmaxf(m, r.rx[g]);
    }
    if (m <= -2048.0f) {
        const float R = -1024.0f * floorf(__fmul_rn(-m, 1.0f / 1024.0f));
#pragma unroll
        for (int i = 0; i < C; i++) {
            Sb[i] = __fsub_rn(Sb[i], R);
            Sb1[i] = __fsub_rn(Sb1[i], R);
        }
        s.qprev = __fsub_rn(s.qprev, R);
        if (GROUP) {                   // the neighbours' edges of S_b, shifted by their own warps too
            s.nb_lo = __fsub_rn(s.nb_lo, R);
            s.nb_hi = __fsub_rn(s.nb_hi, R);
        }
        s.cold->frame += (double)R;
    }
}

// Event injected at offset 0 by the next event move (index e), from the
// prefetch window; successive calls advance e by one.
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
    s.xin = __shfl_sync(kFull, s.ev_cur, idx);
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
    s.kin.x = __shfl_sync(kFull, s.kc_cur.x, idx);
    s.kin.y = __shfl_sync(kFull, s.kc_cur.y, idx);
    s.kin.z = __shfl_sync(kFull, s.kc_cur.z, idx);
}

// The move of band b+1 from band b's end cells (S = S_b, s.b = b).
// GENERAL: band b may reach beyond the last k-mer, whose cells are not -inf
// in registers.
// The move rule on band b's end cells lo = S_b[0], hi = S_b[W-1] (s.b = b):
// cells beyond the last k-mer count as -inf; both -inf: a k-mer move on odd
// bands.
template <int C>
__device__ __forceinline__ bool general_move(const Lane<C> &s, const ReadCtx &r, float lo, float hi)
{
    if (s.ll_k >= r.n_k) lo = neg_inf();
    if (s.ll_k + r.W - 1 >= r.n_k) hi = neg_inf();
    return (lo == neg_inf() && hi == neg_inf()) ? (((s.b + 1) & 1) != 0) : (lo < hi);
}

template <int C, bool MIXED, bool GENERAL>
__device__ __forceinline__ void decide_next(Lane<C> &s, const ReadCtx &r, const float (&S)[C])
{
    float lo = __shfl_sync(kFull, S[0], 0);
    float hi = far_end<C, MIXED>(r, S);
    const bool k = GENERAL ? general_move<C>(s, r, lo, hi) : (lo < hi);
    s.knext = __all_sync(kFull, k);
}

// The warp writes band b's trace record (R words): every lane holds the same
// words and stores them to the same address, which costs no more than one
// lane's store and no predicate (measured 0.5 % faster than a store by lane 0
// alone).  256-bit stores when R is a multiple of 8 words (records then start
// on 32-byte boundaries), else 128-bit.
template <int C>
__device__ __forceinline__ void store_record(const ReadCtx &r, int b, const uint32_t (&w)[2 * C])
{
    constexpr int R = Rec<C>::R;
    uint32_t v[R];
#pragma unroll
    for (int q = 0; q < R; q++) v[q] = (q < 2 * C) ? w[q < 2 * C ? q : 0] : 0u;
    uint32_t *dst = r.tr + (size_t)b * R;
    if (R % 8 == 0) {
#pragma unroll
        for (int q = 0; q < R / 8; q++)
            asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"l"(dst + 8 * q),
                         "r"(v[8 * q]), "r"(v[8 * q + 1]), "r"(v[8 * q + 2]), "r"(v[8 * q + 3]), "r"(v[8 * q + 4]),
                         "r"(v[8 * q + 5]), "r"(v[8 * q + 6]), "r"(v[8 * q + 7])
                         : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < R / 4; q++)
            asm volatile("st.global.v4.b32 [%0], {%1,%2,%3,%4};\n" ::"l"(dst + 4 * q), "r"(v[4 * q]),
                         "r"(v[4 * q + 1]), "r"(v[4 * q + 2]), "r"(v[4 * q + 3])
                         : "memory");
    }
}

// Block mode: lane 0 of warp gw writes its 2C words of band b's record
// (words [2C*gw, 2C*gw + 2C) of a record of kWarps*2C words).
template <int C>
__device__ __forceinline__ void store_record_group(const ReadCtx &r, int b, const uint32_t (&w)[2 * C])
{
    constexpr int RG = 2 * C * kWarps;
    uint32_t *dst = r.tr + (size_t)b * RG + 2 * C * r.gw;
#pragma unroll
    for (int q = 0; q < C; q++)
        asm volatile("{\n .reg .pred p;\n setp.eq.u32 p, %3, 0;\n"
                     " @p st.global.v2.b32 [%0], {%1,%2};\n}\n" ::"l"(dst + 2 * q),
                     "r"(w[2 * q]), "r"(w[2 * q + 1]), "r"(r.lane)
                     : "memory");
}

// One band b = s.b: fill with the decided move, checks (GENERAL), trace
// record, decision for band b+1, prefetch.
template <int C, bool MIXED, bool FULLW, bool GENERAL, bool GROUP>
__device__ __forceinline__ void band_step(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C])
{
    const int b = s.b;
    const bool K = s.knext;
    uint32_t w[2 * C];
    band_fill_dispatch<C, FULLW, GROUP>(K, s, r, P, PP, w);
    s.kprev = K;
    if (K) s.ll_k++;
    else s.ll_e++;
    if (MIXED) {
#pragma unroll
        for (int i = 0; i < C; i++)
            if (r.dead_mask & (1u << i)) PP[i] = neg_inf();
    }
    if (GENERAL) {
        // trim state: the cell (e,-1) scores (e+1)*lp_trim (+ lp_step in the T form)
        if (s.ll_k < 0) {
            const int jt = -1 - s.ll_k;
            const int e = s.ll_e - jt;
            const float v = (e >= 0 && e < r.n_e) ? __fadd_rn(__fmul_rn((float)(e + 1), r.cs.lp_trim), r.cs.lp_step)
                                                   : neg_inf();
#pragma unroll
            for (int i = 0; i < C; i++)
                if ((GROUP ? r.off0 : 0) + C * r.lane + i == jt && (!GROUP || r.lane < r.L)) PP[i] = v;
        }
        // end cell candidates: (e, n_k-1) plus the n_e-1-e trailing events trimmed
        const int jend = r.n_k - 1 - s.ll_k;
        if (jend >= 0 && jend < r.W) {
            const int e = s.ll_e - jend;
            if (e >= 0 && e < r.n_e) {
#pragma unroll
                for (int i = 0; i < C; i++) {
                    if ((GROUP ? r.off0 : 0) + C * r.lane + i == jend && (!GROUP || r.lane < r.L)) {
                        const float rel = __fadd_rn(PP[i], __fmul_rn((float)(r.n_e - 1 - e), r.cs.lp_trim));
                        const double cand = s.cold->frame + (double)rel;
                        if (cand > s.cold->best) {
                            s.cold->best = cand;
                            s.cold->best_e = e;
                            s.cold->best_le = s.ll_e;
                        }
                    }
                }
            }
        }
        const int jlo = max(0, max(s.ll_e - r.n_e + 1, -s.ll_k));
        const int jhi = min(r.W, min(s.ll_e + 1, r.n_k - s.ll_k));
        s.cold->cells += max(0, jhi - jlo);
    }
    if (GROUP) {
        float lo, hi;
        group_exchange<C>(s, r, b, PP, lo, hi);
        s.knext = GENERAL ? general_move<C>(s, r, lo, hi) : (lo < hi);
        store_record_group<C>(r, b, w);
        if (K) next_kmer(s, r, s.ll_k + r.off0 + r.Wp);
        else next_event(s, r, s.ll_e + 1 - r.off0);
    } else {
        decide_next<C, MIXED, GENERAL>(s, r, PP);
        store_record<C>(r, b, w);
        if (FULLW && r.lane == 0) r.mv[b] = K ? 1 : 0;
        if (K) next_kmer(s, r, s.ll_k + r.Wp);
        else next_event(s, r, s.ll_e + 1);
    }
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

// Bands the lean loop may run from here whichever way they move: band b-1
// and every band of the run lie wholly in the matrix and miss the end
// column.  0 if band b-1 itself does not qualify.
template <class LaneT>
__device__ __forceinline__ int lean_run(const LaneT &s, const ReadCtx &r)
{
    if (s.ll_e < r.W - 1 || s.ll_k < 0) return 0;
    const int re = r.n_e - 1 - s.ll_e;          // event moves before offset 0 leaves the matrix
    const int rk = r.n_k - r.W - 1 - s.ll_k;    // k-mer moves before the band meets the end column
    return max(0, min(re, rk));
}

// One band of the lean loop (band b-1 and band b lie wholly in the matrix
// and miss the end column), with the move known at compile time.  The move of
// band b+1 is decided from S_b at offsets 0 and W-1 once the whole band is
// formed.  (Forming those two cells ahead of the band, from the lane's own
// registers, shortens one band's critical path but adds two cells' work to
// every lane; with four or five resident blocks per SM the extra issue slots
// cost more than the latency they hide.)
template <int C, bool MIXED, bool FULLW, bool KM, bool KP, bool GROUP>
__device__ __forceinline__ void lean_band(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C])
{
    const int b = s.b;
    if (GROUP) {                       // block mode: the end cells come through shared memory
        uint32_t w[2 * C];
        band_fill<C, KM, KP, false, true>(s, r, P, PP, w);
        if (KM) s.ll_k++;
        else s.ll_e++;
        float lo, hi;
        group_exchange<C>(s, r, b, PP, lo, hi);
        s.knext = lo < hi;
        store_record_group<C>(r, b, w);
        if (KM) next_kmer(s, r, s.ll_k + r.off0 + r.Wp);
        else next_event(s, r, s.ll_e + 1 - r.off0);
        s.b = b + 1;
        return;
    }
    uint32_t w[2 * C];
    band_fill<C, KM, KP, FULLW, false>(s, r, P, PP, w);
    if (MIXED) {
#pragma unroll
        for (int i = 0; i < C; i++)
            if (r.dead_mask & (1u << i)) PP[i] = neg_inf();
    }
    if (KM) s.ll_k++;
    else s.ll_e++;
    const float lo = __shfl_sync(kFull, PP[0], 0);
    const float hi = far_end<C, MIXED>(r, PP);
    s.knext = __all_sync(kFull, lo < hi);
    store_record<C>(r, b, w);
    if (FULLW && r.lane == 0) r.mv[b] = KM ? 1 : 0;
    if (KM) next_kmer(s, r, s.ll_k + r.Wp);
    else next_event(s, r, s.ll_e + 1);
    s.b = b + 1;
}

// m lean bands (m >= 1) as a state machine over (which array holds S_{b-1},
// previous move); each state branches once, on the decided move.  On exit
// P holds the last band and PP the one before.
template <int C, bool MIXED, bool FULLW, bool GROUP>
__device__ __forceinline__ void lean_loop(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C], int m)
{
    if (s.kprev) goto p0_k1;
    goto p0_k0;
p0_k0:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, false, GROUP>(s, r, P, PP);
        if (--m == 0) goto out1_k1;
        goto p1_k1;
    }
    lean_band<C, MIXED, FULLW, false, false, GROUP>(s, r, P, PP);
    if (--m == 0) goto out1_k0;
    goto p1_k0;
p0_k1:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, true, GROUP>(s, r, P, PP);
        if (--m == 0) goto out1_k1;
        goto p1_k1;
    }
    lean_band<C, MIXED, FULLW, false, true, GROUP>(s, r, P, PP);
    if (--m == 0) goto out1_k0;
    goto p1_k0;
p1_k0:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, false, GROUP>(s, r, PP, P);
        if (--m == 0) goto out0_k1;
        goto p0_k1;
    }
    lean_band<C, MIXED, FULLW, false, false, GROUP>(s, r, PP, P);
    if (--m == 0) goto out0_k0;
    goto p0_k0;
p1_k1:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, true, GROUP>(s, r, PP, P);
        if (--m == 0) goto out0_k1;
        goto p0_k1;
    }
    lean_band<C, MIXED, FULLW, false, true, GROUP>(s, r, PP, P);
    if (--m == 0) goto out0_k0;
    goto p0_k0;
out1_k0:
    swap_bands(P, PP);
    s.kprev = false;
    return;
out1_k1:
    swap_bands(P, PP);
    s.kprev = true;
    return;
out0_k0:
    s.kprev = false;
    return;
out0_k1:
    s.kprev = true;
    return;
}

template <int C, bool MIXED, bool FULLW, bool GROUP>
__device__ __forceinline__ void band_loop(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C])
{
    const int b_end = r.n_e + r.n_k;
    while (s.b <= b_end) {
        int n = lean_run(s, r);
        if (n > 0) {
            s.cold->lean_bands += n;
            while (n > 0) {
                // run up to the next band with b % 64 == 0, then renormalise
                const int to_renorm = (kRenormPeriod - (s.b % kRenormPeriod)) % kRenormPeriod + 1;
                const int m = min(n, to_renorm);
                n -= m;
                lean_loop<C, MIXED, FULLW, GROUP>(s, r, P, PP, m);
                if (((s.b - 1) % kRenormPeriod) == 0) renormalise<C, GROUP>(s, r, P, PP);
            }
        } else {
            band_step<C, MIXED, FULLW, true, GROUP>(s, r, P, PP);
            swap_bands(P, PP);
        }
    }
}

// ---------------------------------------------------------------------------
// Backtrack.

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copy the trace records (R words each) of bands top-lane (lane = 0..31)
// into buf.
template <int R>
__device__ __forceinline__ void chunk_copy(const ReadCtx &r, int top, uint32_t *buf)
{
    const int mb = top - r.lane;
    if (mb >= 2) {                         // bands 0 and 1 hold no matrix cell
        const uint32_t *src = r.tr + (size_t)mb * R;
        uint32_t *dst = buf + r.lane * R;
#pragma unroll
        for (int q = 0; q < R / 4; q++) cp_async16(dst + 4 * q, src + 4 * q);
    }
    cp_async_commit();
}

// Bit l set: band top-l moved by one event.
template <int R, bool FULLW>
__device__ __forceinline__ unsigned chunk_event_moves(const ReadCtx &r, int top, const uint32_t *buf)
{
    const int mb = top - r.lane;
    bool kmove = false;
    if (mb >= 2) kmove = FULLW ? (r.mv[mb] != 0) : (((buf[r.lane * R] >> 31) & 1u) != 0);
    return __ballot_sync(kFull, mb >= 2 && !kmove);
}

// Walk the trace from (e_end, n_k-1) (whose band has offset-0 event le_end)
// until an index leaves the matrix; pair t of the walk goes to out[cap-1-t]
// (t < cap).  Returns 0, or -1 if a traced cell lies outside its band (cannot
// happen); n_out = pairs walked.  The records of 96 bands sit in a
// shared-memory ring of three 32-band chunks, the next two always on their
// way (cp.async).  Within a chunk a step is one shared-memory load, a few
// bit operations and one shared-memory store of the step's cell into the
// stage (32 pairs, the same value from every lane): the band moves of this
// chunk and the next sit in two words (one funnel shift gives the two that a
// step needs).  At the end of each chunk the warp writes the chunk's pairs
// from the stage at once, lane t the t-th.
// Record layout: per-warp mode, offset j is bit j/C of word pair j%C of a
// record of R words; block mode (GROUP), offset j = gw*W' + C*lane + i is
// bit lane of word pair gw*C + i, W' = wg (wg_magic = ceil(2^32 / wg)).
template <int C, int R, bool FULLW, bool GROUP>
__device__ int backtrack(const ReadCtx &r, uint32_t *bufs, int2 *stage, int e_end, int le_end, int2 *out, int cap,
                         int &n_out, unsigned wg = 1, unsigned wg_magic = 0)
{
    constexpr int RING = 3 * kChunk;
    int e = e_end, k = r.n_k - 1;
    int top = e + k + 2;               // band held in ring slot `base`
    int base = 0;
    chunk_copy<R>(r, top, bufs);
    chunk_copy<R>(r, top - kChunk, bufs + kChunk * R);
    chunk_copy<R>(r, top - 2 * kChunk, bufs + 2 * kChunk * R);
    cp_async_wait<1>();
    __syncwarp();
    // bit i: band top-i (em_lo) or top-32-i (em_hi) moved by one event
    unsigned em_lo = chunk_event_moves<R, FULLW>(r, top, bufs);
    unsigned em_hi = chunk_event_moves<R, FULLW>(r, top - kChunk, bufs + kChunk * R);
    int le = le_end;
    int off = 0;                       // the current cell's band is top - off
    int n = 0;                         // pairs walked before the current chunk
    bool bad = false;
    for (;;) {
        const uint32_t *rec = bufs + base * R;
        int2 *sp = stage;
        // One step of the walk.  A cell outside its band (it cannot happen) is noted at the end of
        // each chunk from the offset of the cell the walk continues from; the load index stays inside
        // the record either way.
        auto step = [&]() {
            const int j = le - e;
            unsigned pair, bit;
            if (GROUP) {
                const unsigned ju = ((unsigned)j >= (unsigned)r.W) ? 0u : (unsigned)j;   // inside the record
                const unsigned gq = __umulhi(ju, wg_magic);                           // ju / wg
                const unsigned jj = ju - gq * wg;
                pair = gq * C + jj % C;
                bit = jj / C;
            } else {
                pair = (unsigned)j % C;
                bit = (unsigned)j / C;
            }
            const uint2 w = *reinterpret_cast<const uint2 *>(rec + off * R + 2 * pair);
            const unsigned l = (w.y >> bit) & 1u;
            const unsigned d = (((w.x >> bit) | l) & 1u) ^ 1u;      // D: neither L nor U
            const unsigned ev = __funnelshift_r(em_lo, em_hi, off);  // bit 0: band top-off, bit 1: the one below
            le -= (int)((ev & 1u) + ((ev >> 1) & d));
            *sp++ = make_int2(e, k);
            e += (int)l - 1;                                         // U or D: e-1
            k -= (int)(l + d);                                       // L or D: k-1 (L and D exclusive)
            off += 1 + (int)d;
        };
        while (off <= kChunk - 4 && e >= 1 && k >= 1) {      // two steps stay in the chunk and the matrix
            step();
            step();
        }
        while (off < kChunk && (e | k) >= 0) step();         // at most 32 steps in all per chunk
        bad |= (unsigned)(le - e) >= (unsigned)r.W && (e | k) >= 0;
        const int nb = (int)(sp - stage);
        __syncwarp();
        if (r.lane < nb) {             // the chunk's pairs, one per lane
            const int t = n + r.lane;
            if (t < cap) out[cap - 1 - t] = stage[r.lane];
        }
        n += nb;
        if ((e | k) < 0 || bad) break;
        // the walk enters the next chunk
        __syncwarp();
        const int freed = base;
        top -= kChunk;
        off -= kChunk;
        base += kChunk;
        base -= (base >= RING) ? RING : 0;
        em_lo = em_hi;
        cp_async_wait<0>();
        __syncwarp();
        int nxt = base + kChunk;
        nxt -= (nxt >= RING) ? RING : 0;
        em_hi = chunk_event_moves<R, FULLW>(r, top - kChunk, bufs + nxt * R);
        chunk_copy<R>(r, top - 2 * kChunk, bufs + freed * R);
    }
    cp_async_wait<0>();
    __syncwarp();
    n_out = n;
    return bad ? -1 : 0;
}

// ---------------------------------------------------------------------------

// Pairs (cap - n .. cap-1 of out) moved to the front, ascending, by the
// `width` lanes of `mask` (lane index `lane` among them), 4*width pairs at a
// time: the four loads of a lane are in flight together.  Ascending blocks
// with all loads before the stores are safe however the two ranges overlap
// (a store never reaches a pair a later block still has to load).
__device__ __forceinline__ void compact_pairs(int2 *out, int cap, int n, int lane, int width = 32,
                                              unsigned mask = 0xffffffffu)
{
    __syncwarp(mask);
    for (int base = 0; base < n; base += 4 * width) {
        int2 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int t = base + u * width + lane;
            v[u] = (t < n) ? out[cap - n + t] : make_int2(0, 0);
        }
        __syncwarp(mask);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int t = base + u * width + lane;
            if (t < n) out[t] = v[u];
        }
        __syncwarp(mask);
    }
}

// ---------------------------------------------------------------------------
// Per-warp mode: two walks at once.
//
// A warp walks the reads it aligned two at a time, half a warp each: lanes
// 0-15 walk one read and lanes 16-31 the other, so every instruction of the
// walk's dependent chain serves two reads.  The walk of a read waits in
// shared memory (a WalkJob) until the warp has finished the bands of its
// next read.  The halves run their chunks in step (the same iteration of the
// chunk loop); a half whose walk has ended idles until the other's ends.

// What the walk of one read needs, from its band loop to its walk.
struct WalkJob {
    double best;                     // the end cell's score (T form, renormalisation frame included)
    long long cells;
    const uint32_t *tr;              // the read's trace records
    const uint8_t *mv;               // its per-band move bytes (all 32 lanes live)
    int2 *out;                       // its pair slot
    int rid, best_e, best_le, n_k, cap;
    float lp_step;
};

// Copy the records of bands top-t (t = 0..31) into buf, lanes hl and hl+16
// of a half each copying one band's record (nothing when !live).
template <int R>
__device__ __forceinline__ void chunk_copy2(const uint32_t *tr, int top, uint32_t *buf, int hl, bool live)
{
#pragma unroll
    for (int rep = 0; rep < 2; rep++) {
        const int t = hl + 16 * rep;
        const int mb = top - t;
        if (live && mb >= 2) {         // bands 0 and 1 hold no matrix cell
            const uint32_t *src = tr + (size_t)mb * R;
            uint32_t *dst = buf + t * R;
#pragma unroll
            for (int q = 0; q < R / 4; q++) cp_async16(dst + 4 * q, src + 4 * q);
        }
    }
    cp_async_commit();
}

// Bit t: band top-t moved by one event (this half's chunk).  Both halves call
// it in step (two ballots over the warp).
template <int R, bool FULLW>
__device__ __forceinline__ unsigned chunk_event_moves2(const uint8_t *mv, int top, const uint32_t *buf, int h, int hl,
                                                       bool live)
{
    bool em[2];
#pragma unroll
    for (int rep = 0; rep < 2; rep++) {
        const int t = hl + 16 * rep;
        const int mb = top - t;
        bool kmove = false;
        if (live && mb >= 2) kmove = FULLW ? (mv[mb] != 0) : (((buf[t * R] >> 31) & 1u) != 0);
        em[rep] = live && mb >= 2 && !kmove;
    }
    const unsigned b0 = __ballot_sync(kFull, em[0]) >> (16 * h);
    const unsigned b1 = __ballot_sync(kFull, em[1]) >> (16 * h);
    return (b0 & 0xffffu) | ((b1 & 0xffffu) << 16);
}

// Walk the job at byte offset ja of the kernel's shared memory with lanes
// 0-15 and the job at jb (-1: none) with lanes 16-31, each as backtrack does
// for one read (pairs from the end of the read's slot, then moved to the
// front), and write both results.  The two rings of 3*kChunk records of R
// words start at word bufs, the two stages of kChunk pairs at byte stages.
// Out of line: called once per two reads, and its registers then do not
// weigh on the band loop's allocation; its shared-memory addresses are
// offsets into the kernel's shared array, so its loads and stores stay
// shared-memory ones.
template <int C, int R, bool FULLW>
__device__ __noinline__ void walk2(int ja, int jb, int W, int bufs, int stages, abea_result *res, int lane)
{
    constexpr int RING = 3 * kChunk;
    const int h = lane >> 4, hl = lane & 15;
    const unsigned hmask = 0xffffu << (16 * h);
    const bool live = (h == 0) || (jb >= 0);
    const WalkJob &j = *reinterpret_cast<const WalkJob *>(reinterpret_cast<const char *>(abea_smem) +
                                                          ((h == 0 || jb < 0) ? ja : jb));
    uint32_t *ring = abea_smem + bufs + h * RING * R;
    int2 *stage = reinterpret_cast<int2 *>(reinterpret_cast<char *>(abea_smem) + stages) + h * kChunk;
    const uint32_t *tr = j.tr;
    const uint8_t *mv = j.mv;
    int2 *out = j.out;
    const int cap = j.cap;
    int e = j.best_e, k = j.n_k - 1;
    int top = e + k + 2;               // band held in ring slot `base`
    int base = 0;
    chunk_copy2<R>(tr, top, ring, hl, live);
    chunk_copy2<R>(tr, top - kChunk, ring + kChunk * R, hl, live);
    chunk_copy2<R>(tr, top - 2 * kChunk, ring + 2 * kChunk * R, hl, live);
    cp_async_wait<1>();
    __syncwarp();
    // bit i: band top-i (em_lo) or top-32-i (em_hi) moved by one event
    unsigned em_lo = chunk_event_moves2<R, FULLW>(mv, top, ring, h, hl, live);
    unsigned em_hi = chunk_event_moves2<R, FULLW>(mv, top - kChunk, ring + kChunk * R, h, hl, live);
    int le = j.best_le;
    int off = 0;                       // the current cell's band is top - off
    int n = 0;                         // pairs walked before the current chunk
    bool bad = false;
    bool done = !live;                 // this half's walk has ended
    for (;;) {
        const uint32_t *rec = ring + base * R;
        int2 *sp = stage;
        // One step, as in backtrack (per-warp record layout).
        auto step = [&]() {
            const int j2 = le - e;
            const unsigned pair = (unsigned)j2 % C, bit = (unsigned)j2 / C;
            const uint2 w = *reinterpret_cast<const uint2 *>(rec + off * R + 2 * pair);
            const unsigned l = (w.y >> bit) & 1u;
            const unsigned d = (((w.x >> bit) | l) & 1u) ^ 1u;      // D: neither L nor U
            const unsigned ev = __funnelshift_r(em_lo, em_hi, off);  // bit 0: band top-off, bit 1: the one below
            le -= (int)((ev & 1u) + ((ev >> 1) & d));
            *sp++ = make_int2(e, k);
            e += (int)l - 1;                                         // U or D: e-1
            k -= (int)(l + d);                                       // L or D: k-1 (L and D exclusive)
            off += 1 + (int)d;
        };
        if (!done) {
            while (off <= kChunk - 4 && e >= 1 && k >= 1) {      // two steps stay in the chunk and the matrix
                step();
                step();
            }
            while (off < kChunk && (e | k) >= 0) step();         // at most 32 steps in all per chunk
            bad |= (unsigned)(le - e) >= (unsigned)W && (e | k) >= 0;
        }
        const int nb = (int)(sp - stage);
        __syncwarp();
        for (int t = hl; t < nb; t += 16)                         // the chunk's pairs, two per lane at most
            if (n + t < cap) out[cap - 1 - (n + t)] = stage[t];
        n += nb;
        if (!done && ((e | k) < 0 || bad)) done = true;
        if (__all_sync(kFull, done)) break;
        // both halves enter their next chunk
        __syncwarp();
        const int freed = base;
        top -= kChunk;
        off -= kChunk;
        base += kChunk;
        base -= (base >= RING) ? RING : 0;
        em_lo = em_hi;
        cp_async_wait<0>();
        __syncwarp();
        int nxt = base + kChunk;
        nxt -= (nxt >= RING) ? RING : 0;
        em_hi = chunk_event_moves2<R, FULLW>(mv, top - kChunk, ring + nxt * R, h, hl, !done);
        chunk_copy2<R>(tr, top - 2 * kChunk, ring + freed * R, hl, !done);
    }
    cp_async_wait<0>();
    __syncwarp();
    if (!live) return;
    int status = ABEA_READ_OK;
    if (bad) {
        status = ABEA_READ_FAIL_NO_END;   // internal inconsistency, reported as no alignment
        n = 0;
    } else if (n > cap) {
        status = ABEA_READ_CAPACITY;
    } else {                          // pairs (cap - n .. cap-1) moved to the front, ascending, by the half
        compact_pairs(out, cap, n, hl, 16, hmask);
    }
    if (hl == 0) {
        abea_result rr;
        rr.score = (status == ABEA_READ_OK || status == ABEA_READ_CAPACITY)
                       ? __double2float_rn(j.best - (double)j.lp_step)   // S = T - lp_step
                       : neg_inf();
        rr.status = status;
        rr.n_pairs = (status == ABEA_READ_FAIL_NO_END) ? 0 : n;
        rr.e_end = (status == ABEA_READ_FAIL_NO_END) ? -1 : j.best_e;
        rr.cells = j.cells;
        res[j.rid] = rr;
    }
}

// One read's walk with the whole warp (backtrack), for a read walked alone.
template <int C, int R, bool FULLW>
__device__ __noinline__ void walk1(int ja, int W, int bufs, int stages, abea_result *res, int lane)
{
    const WalkJob &j = *reinterpret_cast<const WalkJob *>(reinterpret_cast<const char *>(abea_smem) + ja);
    ReadCtx r;
    r.tr = const_cast<uint32_t *>(j.tr);
    r.mv = const_cast<uint8_t *>(j.mv);
    r.n_k = j.n_k;
    r.W = W;
    r.lane = lane;
    int n = 0;
    int status = ABEA_READ_OK;
    const int rc = backtrack<C, R, FULLW, false>(r, abea_smem + bufs,
                                                 reinterpret_cast<int2 *>(reinterpret_cast<char *>(abea_smem) + stages),
                                                 j.best_e, j.best_le, j.out, j.cap, n);
    if (rc != 0) {
        status = ABEA_READ_FAIL_NO_END;   // internal inconsistency, reported as no alignment
        n = 0;
    } else if (n > j.cap) {
        status = ABEA_READ_CAPACITY;
    } else {
        compact_pairs(j.out, j.cap, n, lane);
    }
    if (lane == 0) {
        abea_result rr;
        rr.score = (status == ABEA_READ_OK || status == ABEA_READ_CAPACITY)
                       ? __double2float_rn(j.best - (double)j.lp_step)   // S = T - lp_step
                       : neg_inf();
        rr.status = status;
        rr.n_pairs = (status == ABEA_READ_FAIL_NO_END) ? 0 : n;
        rr.e_end = (status == ABEA_READ_FAIL_NO_END) ? -1 : j.best_e;
        rr.cells = j.cells;
        res[j.rid] = rr;
    }
}

// ---------------------------------------------------------------------------
// Per-warp mode.
//
// Scores: P[0..C-1] holds S_{b-1} at the lane's offsets; H holds band b-1's
// view of S_{b-2} (the C+1 values that band b-1 took its left and up
// neighbours from: Q[t] = S_{b-2}[C*lane + t - 1 + KM_{b-1}], t = 0..C),
// stored rotated, H[m] = Q[(m + 1) mod (C+1)].  Band b's diagonal neighbour
// of slot i is Q[i + KM_b], so it is read at an index fixed by band b's own
// move; S_b is written over H, and P becomes the next band's H: in place
// after an event move (H = {P[0..C-1], boundary}), rotated by one register
// after a k-mer move.  The band loop is unrolled by four (the two arrays
// alternate roles), with one branch per band on its move.  A compact loop
// keeps the code of the hot path small enough for the instruction caches
// (state machines over more than a handful of band variants ran slower,
// fetch-bound, although they executed fewer instructions).
//
// The event and k-mer operands entering the band come from two rings in
// shared memory per warp (128 events, 128 k-mer cache entries), filled 32
// at a time by cp.async at the start of each run of at most 64 bands, so
// that each band takes its entering operand with one shared-memory load.  K-mer k
// sits in slot (k - W') mod 128 and event e in slot (e - 1) mod 128: the
// operands entering on the next move are then at slots ll_k and ll_e.

constexpr int kRing = 128;        // entries per operand ring
constexpr int kRingAhead = 96;    // entries requested past the next entering one at each run start
// bands per run at most: every entry a run consumes was requested at an earlier run start and has
// landed at this one's (kRun <= kRingAhead); runs also end at the renormalisation bands (every 64),
// so 64 makes one run per renormalisation period (1.1 % faster than 32)
constexpr int kRun = 64;

struct WRings {
    float4 k[kRing];              // k-mer cache entries (a, b, c)
    float e[kRing];               // events
};

template <int C>
struct WLane {
    float X[C], A[C], B[C], Cc[C];   // operands of the lane's offsets
    bool knext;                      // the next band moves by one k-mer (decided)
    int ll_e, ll_k;                  // offset-0 cell of the last computed band
    int b;                           // next band to compute
    float xin;                       // event entering at offset 0 on the next event move
    float4 kin;                      // k-mer operands entering at offset W'-1 on the next k-mer move
    WRings *ring;
    int k_req, e_req;                // ring entries requested so far (exclusive ends)
    Cold *cold;                      // the read's state the band loop never touches
};

// Request ring entries up to kRingAhead past the next entering k-mer and
// event (one commit group).  Entries beyond the read hold "no k-mer" and
// +inf.  Entries consumed before the next call were requested by an earlier
// call; the caller waits for those (wring_wait) first.
template <int C>
__device__ __forceinline__ void wring_refill(WLane<C> &s, const ReadCtx &r)
{
    const int k_next = s.ll_k + r.Wp, e_next = s.ll_e + 1;
    while (s.k_req < k_next + kRingAhead) {
        const int k = s.k_req + r.lane;
        float4 *dst = s.ring->k + ((k - r.Wp) & (kRing - 1));
        if ((unsigned)k < (unsigned)r.n_k) cp_async16(dst, r.kc + k);
        else *dst = no_kmer();
        s.k_req += 32;
    }
    while (s.e_req < e_next + kRingAhead) {
        const int e = s.e_req + r.lane;
        float *dst = s.ring->e + ((e - 1) & (kRing - 1));
        if ((unsigned)e < (unsigned)r.n_e) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(r.ev + e) : "memory");
        } else {
            *dst = pos_inf();
        }
        s.e_req += 32;
    }
    cp_async_commit();
}

// All requested ring entries have landed and are visible to the warp.
__device__ __forceinline__ void wring_wait()
{
    cp_async_wait<0>();
    __syncwarp();
}

// The operands entering on the next k-mer move (k-mer ll_k + W', ring slot ll_k) and event move
// (event ll_e + 1, ring slot ll_e).
template <int C>
__device__ __forceinline__ void wnext_kmer(WLane<C> &s, const ReadCtx &)
{
    s.kin = s.ring->k[s.ll_k & (kRing - 1)];
}
template <int C>
__device__ __forceinline__ void wnext_event(WLane<C> &s)
{
    s.xin = s.ring->e[s.ll_e & (kRing - 1)];
}

// Band b from S_{b-1} (P[0..C-1]) and band b-1's view of S_{b-2} (H);
// S_b is written into H[0..C-1] and its trace words into w, and P becomes
// band b's view of S_{b-1} (the next band's H).  KM: this band moves by one
// k-mer.  FULLW: all 32 lanes are live (no lane above the band).
template <int C, bool KM, bool FULLW>
__device__ __forceinline__ void wband_fill(WLane<C> &s, const ReadCtx &r, float (&P)[C + 1], float (&H)[C + 1],
                                           uint32_t (&w)[2 * C])
{
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
        s.A[C - 1] = r.last_lane ? s.kin.x : sa;
        s.B[C - 1] = r.last_lane ? s.kin.y : sb;
        s.Cc[C - 1] = r.last_lane ? s.kin.z : sc;
    } else {
        const float sx = __shfl_sync(kFull, s.X[C - 1], r.src_up);
#pragma unroll
        for (int i = C - 1; i > 0; i--) s.X[i] = s.X[i - 1];
        s.X[0] = r.first_lane ? s.xin : sx;
    }
    // Q[t] = S_{b-1}[C*lane + t - 1 + KM], t = 0..C: left of slot i is Q[i], up is Q[i+1]; the
    // one value from a neighbour lane is qb (Q[C] after a k-mer move, Q[0] after an event move).
    float qb;
    if (KM) {
        qb = __shfl_down_sync(kFull, P[0], 1);
        if (FULLW && r.last_lane) qb = neg_inf();
    } else {
        qb = __shfl_sync(kFull, P[C - 1], r.src_up);
        if (FULLW && r.first_lane) qb = neg_inf();
    }
    // the slots in descending order: slot i writes H[i] after slot i+1 has read it (event move)
#pragma unroll
    for (int i = C - 1; i >= 0; i--) {
        const float left = KM ? P[i] : (i == 0 ? qb : P[i > 0 ? i - 1 : 0]);
        const float up = KM ? (i == C - 1 ? qb : P[i < C - 1 ? i + 1 : 0]) : P[i];
        // diag = band b-1's Q at t = i + KM, stored at H[(t + C) mod (C+1)]
        const float diag = KM ? H[i] : H[i == 0 ? C : i - 1];
        bool p0, p1;
        H[i] = cell(up, left, diag, s.X[i], s.A[i], s.B[i], s.Cc[i], r.cs.lp_stay_step, r.lsk, p0, p1);
        w[2 * i] = __ballot_sync(kFull, p0);
        w[2 * i + 1] = __ballot_sync(kFull, p1);
    }
    // the band's move in bit 31 of word 0: lane 31 lies above the band unless all 32 lanes are
    // live, so its bits are 0 (its cells are -inf)
    if (!FULLW && KM) w[0] |= 0x80000000u;
    // P becomes this band's Q, rotated: P[m] = Q[(m + 1) mod (C+1)]
    if (KM) {                           // Q = {P[0..C-1], qb}
        const float q0 = P[0];
#pragma unroll
        for (int m = 0; m < C - 1; m++) P[m] = P[m + 1];
        P[C - 1] = qb;
        P[C] = q0;
    } else {                            // Q = {qb, P[0..C-1]}: P[0..C-1] stay
        P[C] = qb;
    }
}

template <int C, bool MIXED>
__device__ __forceinline__ void wkill_dead(const ReadCtx &r, float (&S)[C + 1])
{
    if constexpr (MIXED) {
#pragma unroll
        for (int i = 0; i < C; i++)
            if (r.dead_mask & (1u << i)) S[i] = neg_inf();
    }
}

// One band of a lean run (band b-1 and band b lie wholly in the matrix and
// miss the end column).  S_b ends in H, band b's view of S_{b-1} in P.  The
// move of band b+1 compares two values every lane received from the same
// lanes, so every lane takes the same decision without a vote.
template <int C, bool MIXED, bool FULLW, bool KM>
__device__ __forceinline__ void wlean_band(WLane<C> &s, const ReadCtx &r, float (&P)[C + 1], float (&H)[C + 1])
{
    const int b = s.b;
    uint32_t w[2 * C];
    wband_fill<C, KM, FULLW>(s, r, P, H, w);
    wkill_dead<C, MIXED>(r, H);
    if (KM) s.ll_k++;
    else s.ll_e++;
    const float lo = __shfl_sync(kFull, H[0], 0);
    const float hi = far_end<C, MIXED>(r, H);
    s.knext = lo < hi;
    store_record<C>(r, b, w);
    if (FULLW && r.lane == 0) r.mv[b] = KM ? 1 : 0;
    if (KM) wnext_kmer(s, r);
    else wnext_event(s);
    s.b = b + 1;
}

// m lean bands (m >= 1), four per iteration and one test of the count per
// iteration (measured 1.2 % faster than two per iteration); a count that is
// not a multiple of four enters the loop body at the band that leaves the
// last band in P, with the arrays swapped first where that band reads them
// the other way round.  On exit P holds the last band and H the view of the
// one before.
template <int C, bool MIXED, bool FULLW>
__device__ __forceinline__ void wlean_run(WLane<C> &s, const ReadCtx &r, float (&P)[C + 1], float (&H)[C + 1], int m)
{
    int t = (m + 3) >> 2;              // fourth bands to run
    switch (m & 3) {
    case 1:
        swap_bands(P, H);
        goto b4;
    case 2:
        goto b3;
    case 3:
        swap_bands(P, H);
        goto b2;
    default:
        break;
    }
    for (;;) {
        if (s.knext) wlean_band<C, MIXED, FULLW, true>(s, r, P, H);
        else wlean_band<C, MIXED, FULLW, false>(s, r, P, H);
    b2:
        if (s.knext) wlean_band<C, MIXED, FULLW, true>(s, r, H, P);
        else wlean_band<C, MIXED, FULLW, false>(s, r, H, P);
    b3:
        if (s.knext) wlean_band<C, MIXED, FULLW, true>(s, r, P, H);
        else wlean_band<C, MIXED, FULLW, false>(s, r, P, H);
    b4:
        if (s.knext) wlean_band<C, MIXED, FULLW, true>(s, r, H, P);
        else wlean_band<C, MIXED, FULLW, false>(s, r, H, P);
        if (--t == 0) return;
    }
}

// One band b = s.b with every check (trim cell, end cell, cell count, bounds
// of the move).  As wlean_band: S_b ends in H, band b's view of S_{b-1} in P.
template <int C, bool MIXED, bool FULLW>
__device__ __forceinline__ void wband_step(WLane<C> &s, const ReadCtx &r, float (&P)[C + 1], float (&H)[C + 1])
{
    const int b = s.b;
    const bool K = s.knext;
    uint32_t w[2 * C];
    if (K) wband_fill<C, true, FULLW>(s, r, P, H, w);
    else wband_fill<C, false, FULLW>(s, r, P, H, w);
    if (K) s.ll_k++;
    else s.ll_e++;
    wkill_dead<C, MIXED>(r, H);
    // trim state: the cell (e,-1) scores (e+1)*lp_trim (+ lp_step in the T form)
    if (s.ll_k < 0) {
        const int jt = -1 - s.ll_k;
        const int e = s.ll_e - jt;
        const float v = (e >= 0 && e < r.n_e) ? __fadd_rn(__fmul_rn((float)(e + 1), r.cs.lp_trim), r.cs.lp_step)
                                                   : neg_inf();
#pragma unroll
        for (int i = 0; i < C; i++)
            if (C * r.lane + i == jt) H[i] = v;
    }
    // end cell candidates: (e, n_k-1) plus the n_e-1-e trailing events trimmed
    const int jend = r.n_k - 1 - s.ll_k;
    if (jend >= 0 && jend < r.W) {
        const int e = s.ll_e - jend;
        if (e >= 0 && e < r.n_e) {
#pragma unroll
            for (int i = 0; i < C; i++) {
                if (C * r.lane + i == jend) {
                    const float rel = __fadd_rn(H[i], __fmul_rn((float)(r.n_e - 1 - e), r.cs.lp_trim));
                    const double cand = s.cold->frame + (double)rel;
                    if (cand > s.cold->best) {
                        s.cold->best = cand;
                        s.cold->best_e = e;
                        s.cold->best_le = s.ll_e;
                    }
                }
            }
        }
    }
    const int jlo = max(0, max(s.ll_e - r.n_e + 1, -s.ll_k));
    const int jhi = min(r.W, min(s.ll_e + 1, r.n_k - s.ll_k));
    s.cold->cells += max(0, jhi - jlo);
    // the move of band b+1: cells beyond the last k-mer count as -inf; both ends -inf: a k-mer
    // move on odd bands
    float lo = __shfl_sync(kFull, H[0], 0);
    float hi = far_end<C, MIXED>(r, H);
    if (s.ll_k >= r.n_k) lo = neg_inf();
    if (s.ll_k + r.W - 1 >= r.n_k) hi = neg_inf();
    const bool kn = (lo == neg_inf() && hi == neg_inf()) ? (((b + 1) & 1) != 0) : (lo < hi);
    s.knext = __all_sync(kFull, kn);
    store_record<C>(r, b, w);
    if (FULLW && r.lane == 0) r.mv[b] = K ? 1 : 0;
    if (K) wnext_kmer(s, r);
    else wnext_event(s);
    s.b = b + 1;
}

// Exact renormalisation after a lean band with b % 64 == 0 (see
// renormalise): P[0..C-1] = S_b and H = band b's view of S_{b-1}, both bands
// wholly in the matrix.  The view holds S_{b-1} at the lane's offsets and
// one value of a neighbour lane's, so its maximum over the warp is S_{b-1}'s;
// lanes above the band and masked slots hold -inf.
template <int C>
__device__ __forceinline__ void wrenormalise(WLane<C> &s, const ReadCtx &r, float (&P)[C + 1], float (&H)[C + 1])
{
    float m = H[C];
#pragma unroll
    for (int i = 0; i < C; i++) m = fmaxf(m, fmaxf(P[i], H[i]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, off));
    if (m <= -2048.0f) {
        const float R = -1024.0f * floorf(__fmul_rn(-m, 1.0f / 1024.0f));
#pragma unroll
        for (int i = 0; i < C; i++) P[i] = __fsub_rn(P[i], R);
#pragma unroll
        for (int i = 0; i <= C; i++) H[i] = __fsub_rn(H[i], R);
        s.cold->frame += (double)R;
    }
}

template <int C, bool MIXED, bool FULLW>
__device__ __forceinline__ void wband_loop(WLane<C> &s, const ReadCtx &r, float (&P)[C + 1], float (&H)[C + 1])
{
    const int b_end = r.n_e + r.n_k;
    while (s.b <= b_end) {
        wring_wait();                 // the entries this run consumes were requested before
        wring_refill(s, r);
        const int n = min(lean_run(s, r), kRun);
        if (n > 0) {
            // up to the next band with b % 64 == 0, then renormalise
            const int to_renorm = (kRenormPeriod - (s.b % kRenormPeriod)) % kRenormPeriod + 1;
            const int m = min(n, to_renorm);
            s.cold->lean_bands += m;
            wlean_run<C, MIXED, FULLW>(s, r, P, H, m);
            if (((s.b - 1) % kRenormPeriod) == 0) wrenormalise<C>(s, r, P, H);
        } else {
            wband_step<C, MIXED, FULLW>(s, r, P, H);
            swap_bands(P, H);
        }
    }
    cp_async_wait<0>();
}

// The bands and the end cell of one read.  A read with an end cell leaves
// its walk in *job (filled by lane 0) and returns true; otherwise its result
// is written here and it returns false.
template <int C, bool MIXED, bool FULLW>
__device__ bool align_read(const AlignArgs &a, const ReadDesc &d, int rid, int lane, Cold &cold, WRings *rings,
                           WalkJob *job)
{
    ReadCtx r;
    r.ev = a.events + d.ev_off;
    r.kc = a.kc + d.kc_off;
    r.tr = a.trace + d.tr_off;
    r.mv = a.moves + d.mv_off;
    r.n_e = d.n_e;
    r.n_k = d.n_k;
    r.W = a.W;
    r.L = a.L;
    r.Wp = C * a.L;
    r.lane = lane;
    r.src_up = (lane + 31) & 31;
    r.first_lane = lane == 0;
    r.last_lane = lane == a.L - 1;
    r.lane31 = lane == 31;
    r.dead_mask = 0;
#pragma unroll
    for (int i = 0; i < C; i++)
        if (C * lane + i >= a.W) r.dead_mask |= 1u << i;
    r.cs = Consts{d.lp_skip, d.lp_stay_step, d.lp_step, d.lp_trim};
    const bool above = lane >= a.L;                 // a lane above the band
    r.lsk = above ? neg_inf() : d.lp_skip;

    const int W = a.W, half = W / 2;
    WLane<C> s;
    float P[C + 1], H[C + 1];
    // bands 0 and 1: the origin (-1,-1) at offset W/2 of band 0 (score 0);
    // band 1 = band 0 moved by one event, the trim cell (0,-1) at offset W/2.
    s.ll_e = half;
    s.ll_k = -1 - half;
#pragma unroll
    for (int i = 0; i < C; i++) {
        const int j = C * lane + i;
        H[i] = (j == half) ? d.lp_step : neg_inf();                        // origin: S = 0
        P[i] = (j == half) ? __fadd_rn(d.lp_trim, d.lp_step) : neg_inf();  // (0,-1): S = lp_trim
        s.X[i] = event_value(r.ev, s.ll_e - j, r.n_e);
        const float4 q = above ? no_kmer() : kmer_operands(r.kc, s.ll_k + j, r.n_k);
        s.A[i] = q.x;
        s.B[i] = q.y;
        s.Cc[i] = q.z;
    }
    P[C] = neg_inf();
    // band 1's view of band 0 (band 1 moved by one event): Q = {boundary, S_0[0..C-1]}
    H[C] = __shfl_sync(kFull, H[C - 1], r.src_up);
    if (r.first_lane) H[C] = neg_inf();
    s.ring = rings;
    s.k_req = s.ll_k + r.Wp;
    s.e_req = s.ll_e + 1;
    __syncwarp();                 // the warp's previous read has finished with the rings
    wring_refill(s, r);
    wring_wait();
    wnext_event(s);
    wnext_kmer(s, r);
    {                             // the move of band 2 from band 1 (only its trim cell can be finite)
        float lo = __shfl_sync(kFull, P[0], 0);
        float hi = far_end<C, MIXED>(r, P);
        if (s.ll_k >= r.n_k) lo = neg_inf();
        if (s.ll_k + r.W - 1 >= r.n_k) hi = neg_inf();
        s.knext = __all_sync(kFull, (lo == neg_inf() && hi == neg_inf()) ? false : (lo < hi));
    }
    s.b = 2;
    s.cold = &cold;
    cold.frame = 0.0;
    cold.best = -(double)pos_inf();
    cold.best_e = INT_MAX;
    cold.best_le = 0;
    cold.cells = 0;
    cold.lean_bands = 0;

    wband_loop<C, MIXED, FULLW>(s, r, P, H);

    // end cell: max score, then smallest event (the first maximum in event order)
    double best = cold.best;
    int best_e = cold.best_e, best_le = cold.best_le;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(kFull, best, off);
        const int oe = __shfl_xor_sync(kFull, best_e, off);
        const int ol = __shfl_xor_sync(kFull, best_le, off);
        if (ob > best || (ob == best && oe < best_e)) {
            best = ob;
            best_e = oe;
            best_le = ol;
        }
    }
    const long long cells = cold.cells + cold.lean_bands * (long long)W;   // identical in every lane

    if (best == -(double)pos_inf()) {
        if (lane == 0) {
            abea_result res;
            res.score = neg_inf();
            res.status = ABEA_READ_FAIL_NO_END;
            res.n_pairs = 0;
            res.e_end = -1;
            res.cells = cells;
            a.res[rid] = res;
        }
        return false;
    }
    if (lane == 0) {
        job->best = best;
        job->cells = cells;
        job->tr = r.tr;
        job->mv = r.mv;
        job->out = reinterpret_cast<int2 *>(a.pairs) + d.pair_off;
        job->rid = rid;
        job->best_e = best_e;
        job->best_le = best_le;
        job->n_k = d.n_k;
        job->cap = d.pair_cap;
        job->lp_step = d.lp_step;
    }
    __syncwarp();                             // the job and the read's trace stores are visible to the warp
    return true;
}

// Shared state of block mode.
struct GroupShared {
    int2 stage[kChunk];                  // the walk's pairs of one chunk
    float2 xch[2][kWarps];
    float rx[kWarps];
    double best[kWarps];
    int best_e[kWarps], best_le[kWarps];
};

// Block mode: the kWarps warps of the block align one read together (a long
// one, so that it does not set the batch's makespan).  Warp gw owns offsets
// [gw*W', gw*W' + W') of every band, W' = W / kWarps = C * L'; the two cells
// next to a warp's edge and the band's two end cells come through shared
// memory after each band (one barrier).  Every warp runs the same bands in
// the same order: the moves are read by all of them from the same shared
// values, so they all pass the same barriers.  Warp 0 then walks the trace
// alone; the other warps return to per-warp work.  Record: kWarps*2C words
// per band.  Results equal those of the per-warp mode bit for bit (same
// cells, same operations).
// Out of line: inlined into the kernel, this code slows the per-warp loop by
// about a fifth under full load (measured).  Its shared memory sits in the
// kernel's dynamic shared memory: the exchange state at word gs_words, warp
// 0's record ring (at least 3*kChunk*RG words) for the walk.
template <int C>
__device__ __noinline__ void align_read_group(const AlignArgs &a, const ReadDesc &d, int rid, int warp, int lane,
                                              int gs_words)
{
    constexpr int RG = 2 * C * kWarps;
    GroupShared &gs = *reinterpret_cast<GroupShared *>(abea_smem + gs_words);
    uint32_t *bt_bufs = abea_smem;                                 // warp 0's ring serves the walk
    const int W = a.W, Wg = W / kWarps, Lg = Wg / C, half = W / 2;
    ReadCtx r;
    r.ev = a.events + d.ev_off;
    r.kc = a.kc + d.kc_off;
    r.tr = a.trace + d.tr_off;
    r.mv = a.moves + d.mv_off;
    r.n_e = d.n_e;
    r.n_k = d.n_k;
    r.W = W;
    r.L = Lg;
    r.Wp = Wg;
    r.lane = lane;
    r.src_up = (lane + 31) & 31;
    r.first_lane = lane == 0;
    r.last_lane = lane == Lg - 1;
    r.lane31 = lane == 31;
    r.dead_mask = 0;
#pragma unroll
    for (int i = 0; i < C; i++)
        if (C * lane + i >= Wg) r.dead_mask |= 1u << i;
    r.cs = Consts{d.lp_skip, d.lp_stay_step, d.lp_step, d.lp_trim};
    const bool live = lane < Lg;
    r.lsk = live ? d.lp_skip : neg_inf();
    r.off0 = warp * Wg;
    r.gw = warp;
    r.xch = &gs.xch[0][0];
    r.rx = gs.rx;

    Lane<C> s;
    float P[C], PP[C];
    const float t_origin = d.lp_step, t_trim0 = __fadd_rn(d.lp_trim, d.lp_step);   // T = S + lp_step
    s.ll_e = half;
    s.ll_k = -1 - half;
#pragma unroll
    for (int i = 0; i < C; i++) {
        const int j = r.off0 + C * lane + i;
        PP[i] = (live && j == half) ? t_origin : neg_inf();
        P[i] = (live && j == half) ? t_trim0 : neg_inf();
        s.X[i] = event_value(r.ev, s.ll_e - j, r.n_e);
        const float4 q = live ? kmer_operands(r.kc, s.ll_k + j, r.n_k) : no_kmer();
        s.A[i] = q.x;
        s.B[i] = q.y;
        s.Cc[i] = q.z;
    }
    // band 1's shifted view of band 0 (S_0 one offset below the lane's first slot)
    s.qprev = (live && r.off0 + C * lane - 1 == half) ? t_origin : neg_inf();
    // the neighbour warps' edges of band 1 (its only finite cell is at offset W/2)
    s.nb_lo = (warp > 0 && r.off0 - 1 == half) ? t_trim0 : neg_inf();
    s.nb_hi = (warp < kWarps - 1 && r.off0 + Wg == half) ? t_trim0 : neg_inf();
    s.kprev = false;
    s.ev_base = s.ll_e + 1 - r.off0;
    s.ev_cur = event_value(r.ev, s.ev_base + lane, r.n_e);
    s.ev_nxt = event_value(r.ev, s.ev_base + 32 + lane, r.n_e);
    s.kc_base = s.ll_k + r.off0 + Wg;
    s.kc_cur = kmer_operands(r.kc, s.kc_base + lane, r.n_k);
    s.kc_nxt = kmer_operands(r.kc, s.kc_base + 32 + lane, r.n_k);
    next_event(s, r, s.ll_e + 1 - r.off0);
    next_kmer(s, r, s.ll_k + r.off0 + Wg);
    s.b = 1;
    s.knext = general_move<C>(s, r, (half == 0) ? t_trim0 : neg_inf(), (half == W - 1) ? t_trim0 : neg_inf());
    s.b = 2;
    Cold cold;
    s.cold = &cold;
    cold.frame = 0.0;
    cold.best = -(double)pos_inf();
    cold.best_e = INT_MAX;
    cold.best_le = 0;
    cold.cells = 0;
    cold.lean_bands = 0;

    band_loop<C, false, false, true>(s, r, P, PP);

    double best = cold.best;
    int best_e = cold.best_e, best_le = cold.best_le;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_xor_sync(kFull, best, off);
        const int oe = __shfl_xor_sync(kFull, best_e, off);
        const int ol = __shfl_xor_sync(kFull, best_le, off);
        if (ob > best || (ob == best && oe < best_e)) {
            best = ob;
            best_e = oe;
            best_le = ol;
        }
    }
    if (lane == 0) {
        gs.best[warp] = best;
        gs.best_e[warp] = best_e;
        gs.best_le[warp] = best_le;
    }
    __threadfence();                      // this warp's trace records, before warp 0 reads them
    group_sync();
    if (warp != 0) return;
#pragma unroll
    for (int g = 1; g < kWarps; g++) {
        const double ob = gs.best[g];
        const int oe = gs.best_e[g];
        if (ob > best || (ob == best && oe < best_e)) {
            best = ob;
            best_e = oe;
            best_le = gs.best_le[g];
        }
    }
    const long long cells = cold.cells + cold.lean_bands * (long long)W;

    int status = ABEA_READ_OK;
    int n = 0;
    int2 *out = reinterpret_cast<int2 *>(a.pairs) + d.pair_off;
    const int cap = d.pair_cap;
    if (best == -(double)pos_inf()) {
        status = ABEA_READ_FAIL_NO_END;
    } else {
        const unsigned magic = 0xffffffffu / (unsigned)Wg + 1u;
        const int rc = backtrack<C, RG, false, true>(r, bt_bufs, gs.stage, best_e, best_le, out, cap, n, (unsigned)Wg,
                                                     magic);
        if (rc != 0) {
            status = ABEA_READ_FAIL_NO_END;
            n = 0;
        } else if (n > cap) {
            status = ABEA_READ_CAPACITY;
        } else {
            compact_pairs(out, cap, n, lane);
        }
    }
    if (lane == 0) {
        abea_result res;
        res.score = (status == ABEA_READ_OK || status == ABEA_READ_CAPACITY)
                        ? __double2float_rn(best - (double)d.lp_step)    // S = T - lp_step
                        : neg_inf();
        res.status = status;
        res.n_pairs = (status == ABEA_READ_FAIL_NO_END) ? 0 : n;
        res.e_end = (status == ABEA_READ_FAIL_NO_END) ? -1 : best_e;
        res.cells = cells;
        a.res[rid] = res;
    }
}

// Dynamic shared memory layout for per-warp C and block-mode CG: per warp
// the two walk rings of 3*kChunk records of R words (one per half-warp; in
// block mode warp 0's region holds the one ring of 3*kChunk block records),
// the block-mode exchange state, one Cold per thread, one WRings per warp,
// two WalkJobs per warp.
template <int C, int CG>
struct Smem {
    static constexpr int WALK_WORDS = 2 * 3 * kChunk * Rec<C>::R;     // per warp
    static_assert(CG == 0 || 3 * kChunk * 2 * CG * kWarps <= WALK_WORDS, "block-mode ring fits warp 0's region");
    static constexpr int GS_WORDS = kWarps * WALK_WORDS;
    static constexpr size_t GS_BYTES = CG > 0 ? (sizeof(GroupShared) + 15) / 16 * 16 : 0;
    static constexpr size_t COLD_OFF = 4 * (size_t)GS_WORDS + GS_BYTES;   // one Cold per thread
    static constexpr size_t RING_OFF = COLD_OFF + kWarps * 32 * sizeof(Cold); // one WRings per warp
    static constexpr size_t JOB_OFF = (RING_OFF + kWarps * sizeof(WRings) + 15) / 16 * 16;   // two WalkJobs per warp
    static constexpr size_t BYTES = JOB_OFF + kWarps * 2 * sizeof(WalkJob);
};

// Persistent kernel.  Blocks 0 .. n_group-1 first align reads order[0 ..
// n_group-1] in block mode (CG offsets per lane); then every warp takes reads
// order[n_group ..] one at a time from the shared counter, and walks them two
// at a time (walk2) or, in the queue's tail, one at a time (walk1).
// Blocks per SM the register budget is set for: 5 where the band fits in at
// most 96 registers without spilling much (C <= 2, and C = 4 with 25 lanes:
// 5 ran 3 % faster than 4 blocks at W = 100; 6, 7 and 8 ran no faster or
// spilled in the band loop), 4 for the rest up to C = 5, 3 for C >= 6
// (168 registers; 10 % faster than 2 blocks at W = 200).
template <int C, bool MIXED, bool FULLW>
struct Occupancy {
    static constexpr int blocks = (C >= 6) ? 3 : (C <= 2 || (C == 4 && !MIXED && !FULLW)) ? 5 : 4;
};

template <int C, bool MIXED, bool FULLW, int CG>
__global__ void __launch_bounds__(kWarps * 32, Occupancy<C, MIXED, FULLW>::blocks) align_kernel(const AlignArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    Cold &cold = reinterpret_cast<Cold *>(reinterpret_cast<char *>(abea_smem) + Smem<C, CG>::COLD_OFF)[threadIdx.x];
    WRings *rings = reinterpret_cast<WRings *>(reinterpret_cast<char *>(abea_smem) + Smem<C, CG>::RING_OFF) + warp;
    WalkJob *jobs = reinterpret_cast<WalkJob *>(reinterpret_cast<char *>(abea_smem) + Smem<C, CG>::JOB_OFF) + 2 * warp;
    // walk2's shared-memory operands as offsets: the jobs, the rings, the stages (the operand ring
    // is idle while the warp walks)
    const int job_off = (int)(Smem<C, CG>::JOB_OFF + 2 * warp * sizeof(WalkJob));
    const int bt_off = warp * Smem<C, CG>::WALK_WORDS;
    const int stage_off = (int)(Smem<C, CG>::RING_OFF + warp * sizeof(WRings));
    if (CG > 0 && (int)blockIdx.x < a.n_group) {
        const int rid = a.order[blockIdx.x];
        const ReadDesc d = a.rd[rid];
        if (d.host_bad || a.flags[rid]) {
            if (threadIdx.x == 0) {
                abea_result res;
                res.score = neg_inf();
                res.status = ABEA_READ_BAD_INPUT;
                res.n_pairs = 0;
                res.e_end = -1;
                res.cells = 0;
                a.res[rid] = res;
            }
        } else {
            align_read_group<(CG > 0 ? CG : 1)>(a, d, rid, warp, lane, Smem<C, CG>::GS_WORDS);
        }
        __syncwarp();
    }
    bool pending = false;              // jobs[cur ^ 1] holds a walk waiting for the next read's
    int cur = 0;
    for (;;) {
        int q = 0;
        if (lane == 0) q = atomicAdd(a.queue, 1);
        q = __shfl_sync(kFull, q, 0) + a.n_group;
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
        // The walk of a read waits for the warp's next read, and the two are walked together, while
        // the queue holds at least one more read per warp; in the queue's tail a read is walked at
        // once, so that no read's result waits for another read's bands there.
        if (align_read<C, MIXED, FULLW>(a, d, rid, lane, cold, rings, jobs + cur)) {
            if (pending) {
                walk2<C, Rec<C>::R, FULLW>(job_off + (cur ^ 1) * (int)sizeof(WalkJob), job_off + cur * (int)sizeof(WalkJob),
                                           a.W, bt_off, stage_off, a.res, lane);
                pending = false;
            } else if (q + (int)gridDim.x * kWarps < a.n) {
                pending = true;
                cur ^= 1;
            } else {
                walk1<C, Rec<C>::R, FULLW>(job_off + cur * (int)sizeof(WalkJob), a.W, bt_off, stage_off, a.res, lane);
            }
        }
        __syncwarp();
    }
    if (pending) walk1<C, Rec<C>::R, FULLW>(job_off + (cur ^ 1) * (int)sizeof(WalkJob), a.W, bt_off, stage_off, a.res, lane);
}

// Dynamic shared memory above the 48 KB default needs the kernel's opt-in
// (the wide geometries' two walk rings per warp).
template <int C, bool MIXED, bool FULLW, int CG>
cudaError_t opt_in_smem()
{
    if (Smem<C, CG>::BYTES <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(align_kernel<C, MIXED, FULLW, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Smem<C, CG>::BYTES);
}

template <int C, bool MIXED, bool FULLW, int CG>
int launch_c(const AlignArgs &a, int grid, void *stream)
{
    const cudaError_t e = opt_in_smem<C, MIXED, FULLW, CG>();
    if (e != cudaSuccess) return (int)e;
    align_kernel<C, MIXED, FULLW, CG><<<grid, kWarps * 32, Smem<C, CG>::BYTES, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

template <int C, bool MIXED, bool FULLW, int CG>
int grid_c(int device)
{
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return -1;
    e = opt_in_smem<C, MIXED, FULLW, CG>();
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, align_kernel<C, MIXED, FULLW, CG>, kWarps * 32,
                                                      Smem<C, CG>::BYTES);
    if (e != cudaSuccess || per_sm < 1) return -1;
    return sms * per_sm;
}

// Offsets per lane in block mode for band width W (0: no block mode): W
// splits evenly over the block's warps, W' = W / kWarps, and W' = c * L'
// with L' <= 31 lanes (lane 31 stays above the band and carries the move
// bit), c = 1 or 2.  Narrow bands (W < 32) gain nothing from it.
int group_offsets_per_lane(int W)
{
    if (W < 32 || W % kWarps != 0) return 0;
    const int Wg = W / kWarps;
    for (int c = 1; c <= 2; c++)
        if (Wg % c == 0 && Wg / c <= 31) return c;
    return 0;
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
    g.full = g.L == 32;
    g.cg = group_offsets_per_lane(W);
    g.rec_words = std::max((2 * C + 3) / 4 * 4, 2 * g.cg * kWarps);
    return g;
}

int group_count(const ReadDesc *rd, const int32_t *order, int32_t n, const Geometry &g, int grid, double theta)
{
    if (g.cg == 0 || n <= 0 || grid <= 0 || !(theta > 0.0)) return 0;
    double total = 0.0;
    for (int32_t t = 0; t < n; t++)
        if (!rd[t].host_bad) total += (double)rd[t].n_e + rd[t].n_k + 1;
    const double slots = (double)std::min<int64_t>((int64_t)grid, (n + kWarps - 1) / kWarps) * kWarps;
    const double limit = theta * total / slots;
    int m = 0;
    while (m < n && m < grid) {
        const ReadDesc &d = rd[order[m]];
        if (d.host_bad || (double)d.n_e + d.n_k + 1 <= limit) break;
        m++;
    }
    return m;
}

int align_launch_grid(int32_t n, int n_group, int grid)
{
    const int64_t want = (int64_t)n_group + (n - n_group + kWarps - 1) / kWarps;
    return (int)std::max<int64_t>(1, std::min<int64_t>(grid, want));
}

// Instantiated geometries: every (C, mixed, full, block-mode C) that
// geometry_for gives for 2 <= W <= 256.
#define ABEA_FOR_EACH_GEOMETRY(X)                                                                  \
    X(1, false, false, 0) X(1, false, true, 1) X(2, false, false, 0) X(2, false, false, 1)         \
    X(2, false, true, 1) X(2, true, false, 0) X(3, false, false, 0) X(3, false, false, 1)          \
    X(3, false, true, 1) X(3, true, false, 0) X(3, true, true, 0) X(4, false, false, 1)            \
    X(4, false, true, 2) X(4, true, false, 0) X(4, true, true, 0) X(5, false, false, 0)            \
    X(5, false, true, 2) X(5, true, false, 0) X(5, true, true, 0) X(6, false, false, 0)            \
    X(6, false, false, 2) X(6, false, true, 2) X(6, true, false, 0) X(6, true, true, 0)            \
    X(7, false, false, 0) X(7, false, true, 2) X(7, true, false, 0) X(7, true, true, 0)            \
    X(8, false, false, 2) X(8, false, true, 0) X(8, true, false, 0) X(8, true, true, 0)

int launch_align(const AlignArgs &args, const Geometry &g, int grid, void *stream)
{
    AlignArgs a = args;
    a.n_group = std::max(0, std::min(std::min(a.n_group, a.n), grid));
    if (g.cg == 0) a.n_group = 0;
#define X(c_, m_, f_, g_)                                                                          \
    if (g.C == c_ && g.mixed == m_ && g.full == f_ && g.cg == g_) return launch_c<c_, m_, f_, g_>(a, grid, stream);
    ABEA_FOR_EACH_GEOMETRY(X)
#undef X
    return (int)cudaErrorInvalidValue;
}

int align_grid_size(const Geometry &g, int device)
{
#define X(c_, m_, f_, g_)                                                                          \
    if (g.C == c_ && g.mixed == m_ && g.full == f_ && g.cg == g_) return grid_c<c_, m_, f_, g_>(device);
    ABEA_FOR_EACH_GEOMETRY(X)
#undef X
    return -1;
}

}  // namespace abea
