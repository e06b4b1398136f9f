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
//   - the previous two bands, the events and the k-mer operands of the
//     lane's offsets live in registers.  A band move shifts either the k-mer
//     operands (k-mer move) or the events (event move) by one offset; the one
//     value that crosses a lane boundary travels by __shfl_*_sync.  The value
//     entering at the band end comes from a warp-wide prefetch window (lane i
//     holds the i-th next event / k-mer entry, the following 32 in flight);
//   - the neighbours of a cell are a +-0/1 offset shift of the previous one
//     or two bands, selected by the last two moves; the four cases are
//     compiled separately so every register index is static;
//   - the move of band b+1 is decided at the end of band b (two shuffles of
//     its end cells), so the decision overlaps band b's bookkeeping;
//   - the direction of every cell is two predicates (U over D; L over the
//     max), gathered by __ballot_sync into 2C words per band and stored by
//     lane 0 (2 bits per cell); the band's move rides in bit 31 of its first
//     word (lane 31 lies above the band); no score array is ever written;
//   - cells outside the matrix need no per-cell test: a missing event reads
//     +inf and a missing k-mer reads (a=1, b=0, c=-inf), which make the
//     emission -inf; the only cells this leaves finite lie beyond the last
//     k-mer, which no in-matrix cell reads, and the band-move decision
//     clamps those to -inf;
//   - runs of bands whose W offsets all lie in the matrix go through a lean
//     loop controlled by one counter (no trim, end or bound checks); the rest
//     run the same step with those checks;
//   - after the last band the same warp walks the trace back: the records of
//     32 bands at a time are copied to shared memory with cp.async, two
//     chunks ahead of the walk; each step reads its two trace words there and
//     the band moves give each band's position; the pairs are gathered across
//     the lanes and stored 32 at a time.
//
// All FP32 arithmetic uses explicitly rounded intrinsics, so no operation is
// fused or reordered: the scores equal those of the FP32 canonical form
//   z = fmaf(x, a, b); E = fmaf(-z, z, c);
//   d = diag + lp_step; u = up + lp_stay; m = (u > d) ? u : d; s = m + E;
//   l = left + lp_skip; S = (l > s) ? l : s
// (max(diag+lp_step+E, up+lp_stay+E) = max(diag+lp_step, up+lp_stay) + E
// because rounding is monotone), plus the exact renormalisation below.
#include <climits>

#include "abea_internal.h"

namespace abea {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = 4;          // warps per block
constexpr int kChunk = 32;         // bands per backtrack chunk
constexpr int kRenormPeriod = 64;

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }
__device__ __forceinline__ float pos_inf() { return __int_as_float(0x7f800000); }

struct Consts {
    float lp_skip, lp_stay, lp_step, lp_trim;
};

__device__ __forceinline__ float cell(float up, float left, float diag, float x, float a, float b, float c,
                                      float lp_step, float lp_stay, float lp_skip, bool &p0, bool &p1)
{
    const float z = __fmaf_rn(x, a, b);
    const float em = __fmaf_rn(-z, z, c);
    const float d = __fadd_rn(diag, lp_step);
    const float u = __fadd_rn(up, lp_stay);
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

// Lane state other than the two score bands.
template <int C>
struct Lane {
    float X[C], A[C], B[C], Cc[C];   // operands of the lane's offsets
    float qprev;                     // boundary value of the previous band's shifted view
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
    double frame;                    // total renormalisation shift so far
    double best;                     // best end candidate seen by this lane (unshifted)
    int best_e, best_le;
    long long cells;                 // in-matrix cells of bands run with checks
    long long lean_bands;            // bands run by the lean loop (W cells each)
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
};

// Band b from S_{b-1} (P) and S_{b-2} (PP); S_b is written into PP and its
// trace words into w.  KM: this band moves by one k-mer; KP: the previous
// band did.  FULLW: all 32 lanes are live (no lane above the band).
template <int C, bool KM, bool KP, bool FULLW>
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
    // above the band (all -inf), unless FULLW.
    float qb;
    if (KM) {
        qb = __shfl_down_sync(kFull, P[0], 1);
        if (FULLW && r.last_lane) qb = neg_inf();
    } else {
        qb = __shfl_sync(kFull, P[C - 1], r.src_up);
        if (FULLW && r.first_lane) qb = neg_inf();
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
        S[i] = cell(up, left, diag, s.X[i], s.A[i], s.B[i], s.Cc[i], r.cs.lp_step, r.cs.lp_stay, r.lsk, p0, p1);
        if (!FULLW && i == 0) p0 = r.lane31 ? KM : p0;     // the band's move, bit 31 of word 0
        w[2 * i] = __ballot_sync(kFull, p0);
        w[2 * i + 1] = __ballot_sync(kFull, p1);
    }
#pragma unroll
    for (int i = 0; i < C; i++) PP[i] = S[i];
    s.qprev = qb;
}

template <int C, bool FULLW>
__device__ __forceinline__ void band_fill_dispatch(bool K, Lane<C> &s, const ReadCtx &r, float (&P)[C],
                                                   float (&PP)[C], uint32_t (&w)[2 * C])
{
    if (K) {
        if (s.kprev) band_fill<C, true, true, FULLW>(s, r, P, PP, w);
        else band_fill<C, true, false, FULLW>(s, r, P, PP, w);
    } else {
        if (s.kprev) band_fill<C, false, true, FULLW>(s, r, P, PP, w);
        else band_fill<C, false, false, FULLW>(s, r, P, PP, w);
    }
}

// The value of a band at offset W-1.
template <int C, bool MIXED>
__device__ __forceinline__ float far_end(const ReadCtx &r, const float (&S)[C])
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
template <int C, bool MIXED, bool GENERAL>
__device__ __forceinline__ void decide_next(Lane<C> &s, const ReadCtx &r, const float (&S)[C])
{
    float lo = __shfl_sync(kFull, S[0], 0);
    float hi = far_end<C, MIXED>(r, S);
    bool k;
    if (GENERAL) {
        if (s.ll_k >= r.n_k) lo = neg_inf();
        if (s.ll_k + r.W - 1 >= r.n_k) hi = neg_inf();
        k = (lo == neg_inf() && hi == neg_inf()) ? (((s.b + 1) & 1) != 0) : (lo < hi);
    } else {
        k = lo < hi;
    }
    s.knext = __all_sync(kFull, k);
}

// Lane 0 writes band b's trace record (R words, all lanes hold the same w);
// predicated, no branch.  256-bit stores when R is a multiple of 8 words
// (records then start on 32-byte boundaries), else 128-bit.
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
            asm volatile("{\n .reg .pred p;\n setp.eq.u32 p, %9, 0;\n"
                         " @p st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n}\n" ::"l"(dst + 8 * q),
                         "r"(v[8 * q]), "r"(v[8 * q + 1]), "r"(v[8 * q + 2]), "r"(v[8 * q + 3]), "r"(v[8 * q + 4]),
                         "r"(v[8 * q + 5]), "r"(v[8 * q + 6]), "r"(v[8 * q + 7]), "r"(r.lane)
                         : "memory");
    } else {
#pragma unroll
        for (int q = 0; q < R / 4; q++)
            asm volatile("{\n .reg .pred p;\n setp.eq.u32 p, %5, 0;\n"
                         " @p st.global.v4.b32 [%0], {%1,%2,%3,%4};\n}\n" ::"l"(dst + 4 * q), "r"(v[4 * q]),
                         "r"(v[4 * q + 1]), "r"(v[4 * q + 2]), "r"(v[4 * q + 3]), "r"(r.lane)
                         : "memory");
    }
}

// One band b = s.b: fill with the decided move, checks (GENERAL), trace
// record, decision for band b+1, prefetch.
template <int C, bool MIXED, bool FULLW, bool GENERAL>
__device__ __forceinline__ void band_step(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C])
{
    const int b = s.b;
    const bool K = s.knext;
    uint32_t w[2 * C];
    band_fill_dispatch<C, FULLW>(K, s, r, P, PP, w);
    s.kprev = K;
    if (K) s.ll_k++;
    else s.ll_e++;
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
                            s.best_le = s.ll_e;
                        }
                    }
                }
            }
        }
        const int jlo = max(0, max(s.ll_e - r.n_e + 1, -s.ll_k));
        const int jhi = min(r.W, min(s.ll_e + 1, r.n_k - s.ll_k));
        s.cells += max(0, jhi - jlo);
    }
    decide_next<C, MIXED, GENERAL>(s, r, PP);
    store_record<C>(r, b, w);
    if (FULLW && r.lane == 0) r.mv[b] = K ? 1 : 0;
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

// Bands the lean loop may run from here whichever way they move: band b-1
// and every band of the run lie wholly in the matrix and miss the end
// column.  0 if band b-1 itself does not qualify.
template <int C>
__device__ __forceinline__ int lean_run(const Lane<C> &s, const ReadCtx &r)
{
    if (s.ll_e < r.W - 1 || s.ll_k < 0) return 0;
    const int re = r.n_e - 1 - s.ll_e;          // event moves before offset 0 leaves the matrix
    const int rk = r.n_k - r.W - 1 - s.ll_k;    // k-mer moves before the band meets the end column
    return max(0, min(re, rk));
}

// One band of the lean loop (band b-1 and band b lie wholly in the matrix
// and miss the end column), with the move known at compile time.  The move of
// band b+1 needs S_b at offsets 0 and W-1.  Those two cells have no
// neighbour across a lane edge (the lane below offset 0 and the lane above
// offset W-1 lie outside the band), so they are formed from the lane's own
// registers and the injected operand, and their shuffles are issued before
// the rest of the band; the same values come out of the full band, so the
// decision is unchanged.
template <int C, bool MIXED, bool FULLW, bool KM, bool KP>
__device__ __forceinline__ void lean_band(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C])
{
    const int b = s.b;
    float lo_src, hi_src;
    if (!MIXED) {
        const float lp_step = r.cs.lp_step, lp_stay = r.cs.lp_stay, lsk = r.lsk;
        // offset 0 (lane 0, slot 0)
        {
            const float x = KM ? s.X[0] : s.xin;
            const float a = KM ? s.A[C > 1 ? 1 : 0] : s.A[0];
            const float bb = KM ? s.B[C > 1 ? 1 : 0] : s.B[0];
            const float c = KM ? s.Cc[C > 1 ? 1 : 0] : s.Cc[0];
            const float up = KM ? P[C > 1 ? 1 : 0] : P[0];
            const float left = KM ? P[0] : neg_inf();
            const int t = KM ? 1 : 0;
            const float diag = KP ? (t == C ? s.qprev : PP[t < C ? t : 0]) : (t == 0 ? s.qprev : PP[t > 0 ? t - 1 : 0]);
            bool q0, q1;
            lo_src = (KM && C == 1) ? 0.0f : cell(up, left, diag, x, a, bb, c, lp_step, lp_stay, lsk, q0, q1);
        }
        // offset W-1 (lane L-1, slot C-1)
        {
            const float x = KM ? s.X[C - 1] : s.X[C > 1 ? C - 2 : 0];
            const float a = KM ? s.kin.x : s.A[C - 1];
            const float bb = KM ? s.kin.y : s.B[C - 1];
            const float c = KM ? s.kin.z : s.Cc[C - 1];
            const float up = KM ? neg_inf() : P[C - 1];
            const float left = KM ? P[C - 1] : P[C > 1 ? C - 2 : 0];
            const int t = C - 1 + (KM ? 1 : 0);
            const float diag = KP ? (t == C ? s.qprev : PP[t < C ? t : 0]) : (t == 0 ? s.qprev : PP[t > 0 ? t - 1 : 0]);
            bool q0, q1;
            hi_src = (!KM && C == 1) ? 0.0f : cell(up, left, diag, x, a, bb, c, lp_step, lp_stay, lsk, q0, q1);
        }
    }
    uint32_t w[2 * C];
    band_fill<C, KM, KP, FULLW>(s, r, P, PP, w);
    if (MIXED) {
#pragma unroll
        for (int i = 0; i < C; i++)
            if (r.dead_mask & (1u << i)) PP[i] = neg_inf();
    }
    if (MIXED || C == 1) {
        lo_src = PP[0];
        hi_src = PP[C - 1];
    }
    if (KM) s.ll_k++;
    else s.ll_e++;
    float lo = __shfl_sync(kFull, lo_src, 0);
    float hi;
    if (MIXED) hi = far_end<C, MIXED>(r, PP);
    else hi = __shfl_sync(kFull, hi_src, r.L - 1);
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
template <int C, bool MIXED, bool FULLW>
__device__ __forceinline__ void lean_loop(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C], int m)
{
    if (s.kprev) goto p0_k1;
    goto p0_k0;
p0_k0:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, false>(s, r, P, PP);
        if (--m == 0) goto out1_k1;
        goto p1_k1;
    }
    lean_band<C, MIXED, FULLW, false, false>(s, r, P, PP);
    if (--m == 0) goto out1_k0;
    goto p1_k0;
p0_k1:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, true>(s, r, P, PP);
        if (--m == 0) goto out1_k1;
        goto p1_k1;
    }
    lean_band<C, MIXED, FULLW, false, true>(s, r, P, PP);
    if (--m == 0) goto out1_k0;
    goto p1_k0;
p1_k0:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, false>(s, r, PP, P);
        if (--m == 0) goto out0_k1;
        goto p0_k1;
    }
    lean_band<C, MIXED, FULLW, false, false>(s, r, PP, P);
    if (--m == 0) goto out0_k0;
    goto p0_k0;
p1_k1:
    if (s.knext) {
        lean_band<C, MIXED, FULLW, true, true>(s, r, PP, P);
        if (--m == 0) goto out0_k1;
        goto p0_k1;
    }
    lean_band<C, MIXED, FULLW, false, true>(s, r, PP, P);
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

template <int C, bool MIXED, bool FULLW>
__device__ __forceinline__ void band_loop(Lane<C> &s, const ReadCtx &r, float (&P)[C], float (&PP)[C])
{
    const int b_end = r.n_e + r.n_k;
    while (s.b <= b_end) {
        int n = lean_run(s, r);
        if (n > 0) {
            s.lean_bands += n;
            while (n > 0) {
                // run up to the next band with b % 64 == 0, then renormalise
                const int to_renorm = (kRenormPeriod - (s.b % kRenormPeriod)) % kRenormPeriod + 1;
                const int m = min(n, to_renorm);
                n -= m;
                lean_loop<C, MIXED, FULLW>(s, r, P, PP, m);
                if (((s.b - 1) % kRenormPeriod) == 0) renormalise<C>(s, r, P, PP);
            }
        } else {
            band_step<C, MIXED, FULLW, true>(s, r, P, PP);
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

// Copy the trace records of bands top-lane (lane = 0..31) into buf.
template <int C>
__device__ __forceinline__ void chunk_copy(const ReadCtx &r, int top, uint32_t *buf)
{
    constexpr int R = Rec<C>::R;
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
template <int C, bool FULLW>
__device__ __forceinline__ unsigned chunk_event_moves(const ReadCtx &r, int top, const uint32_t *buf)
{
    constexpr int R = Rec<C>::R;
    const int mb = top - r.lane;
    bool kmove = false;
    if (mb >= 2) kmove = FULLW ? (r.mv[mb] != 0) : (((buf[r.lane * R] >> 31) & 1u) != 0);
    return __ballot_sync(kFull, mb >= 2 && !kmove);
}

// Walk the trace from (e_end, n_k-1) (whose band has offset-0 event le_end)
// until an index leaves the matrix; lane 0 writes pair t of the walk to
// out[cap-1-t] (t < cap).  Returns 0, or -1 if a traced cell lies outside
// its band (cannot happen); n_out = pairs walked.  The records of 96 bands
// sit in a shared-memory ring of three 32-band chunks, the next two always
// on their way (cp.async); the band moves of the current and next chunk are
// kept as one 64-bit word, so a step needs one shared-memory load.
template <int C, bool FULLW>
__device__ int backtrack(const ReadCtx &r, uint32_t *bufs, int e_end, int le_end, int2 *out, int cap, int &n_out)
{
    constexpr int R = Rec<C>::R;
    constexpr int RING = 3 * kChunk;
    int e = e_end, k = r.n_k - 1;
    int top = e + k + 2;               // band held in ring slot `base`
    int base = 0;
    chunk_copy<C>(r, top, bufs);
    chunk_copy<C>(r, top - kChunk, bufs + kChunk * R);
    chunk_copy<C>(r, top - 2 * kChunk, bufs + 2 * kChunk * R);
    cp_async_wait<1>();
    __syncwarp();
    // bit i: band top-i moved by one event
    unsigned long long em = (unsigned long long)chunk_event_moves<C, FULLW>(r, top, bufs) |
                            ((unsigned long long)chunk_event_moves<C, FULLW>(r, top - kChunk, bufs + kChunk * R)
                             << 32);
    const bool writer = r.lane == 0;
    int le = le_end;
    int off = 0;                       // the current cell's band is top - off
    int n = 0;
    unsigned bad = 0;
    while (((e | k) >= 0) && !bad) {
        const int j = le - e;
        bad = (unsigned)j >= (unsigned)r.W ? 1u : 0u;
        int p = base + off;
        p -= (p >= RING) ? RING : 0;
        const uint2 w = *reinterpret_cast<const uint2 *>(bufs + p * R + 2 * ((unsigned)j % C));
        const unsigned bit = (unsigned)j / C;
        if (writer && n < cap) out[cap - 1 - n] = make_int2(e, k);
        n++;
        const unsigned l = (w.y >> bit) & 1u;
        const unsigned d = ((w.x >> bit) & 1u | l) ^ 1u;          // D: neither L nor U
        const unsigned ev = (unsigned)(em >> off);                 // bit 0: band bb, bit 1: band bb-1
        le -= (int)((ev & 1u) + ((ev >> 1) & d));
        e -= (int)(l ^ 1u);                                        // U or D
        k -= (int)(l | d);                                         // L or D
        off += 1 + (int)d;
        if (off >= kChunk) {           // the walk enters the next chunk
            __syncwarp();
            const int freed = base;
            top -= kChunk;
            off -= kChunk;
            base += kChunk;
            base -= (base >= RING) ? RING : 0;
            em >>= 32;
            cp_async_wait<0>();
            __syncwarp();
            int nxt = base + kChunk;
            nxt -= (nxt >= RING) ? RING : 0;
            em |= (unsigned long long)chunk_event_moves<C, FULLW>(r, top - kChunk, bufs + nxt * R) << 32;
            chunk_copy<C>(r, top - 2 * kChunk, bufs + freed * R);
        }
    }
    cp_async_wait<0>();
    __syncwarp();
    n_out = n;
    return bad ? -1 : 0;
}

// ---------------------------------------------------------------------------

template <int C, bool MIXED, bool FULLW>
__device__ void align_read(const AlignArgs &a, const ReadDesc &d, int rid, int lane, uint32_t *bt_bufs)
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
    r.cs = Consts{d.lp_skip, d.lp_stay, d.lp_step, d.lp_trim};
    const bool above = lane >= a.L;                 // a lane above the band
    r.lsk = above ? neg_inf() : d.lp_skip;

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
        const float4 q = above ? no_kmer() : kmer_operands(r.kc, s.ll_k + j, r.n_k);
        s.A[i] = q.x;
        s.B[i] = q.y;
        s.Cc[i] = q.z;
    }
    // band 1's shifted view of band 0 (band 1 moved by one event)
    s.qprev = __shfl_sync(kFull, PP[C - 1], r.src_up);
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
    s.b = 1;
    decide_next<C, MIXED, true>(s, r, P);          // the move of band 2
    s.b = 2;
    s.frame = 0.0;
    s.best = -(double)pos_inf();
    s.best_e = INT_MAX;
    s.best_le = 0;
    s.cells = 0;
    s.lean_bands = 0;

    band_loop<C, MIXED, FULLW>(s, r, P, PP);

    // end cell: max score, then smallest event (the first maximum in event order)
    double best = s.best;
    int best_e = s.best_e, best_le = s.best_le;
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
    const long long cells = s.cells + s.lean_bands * (long long)W;   // identical in every lane

    int status = ABEA_READ_OK;
    int n = 0;
    int2 *out = reinterpret_cast<int2 *>(a.pairs) + d.pair_off;
    const int cap = d.pair_cap;
    if (best == -(double)pos_inf()) {
        status = ABEA_READ_FAIL_NO_END;
    } else {
        __syncwarp();                         // lane 0's trace stores are visible to the warp
        const int rc = backtrack<C, FULLW>(r, bt_bufs, best_e, best_le, out, cap, n);
        if (rc != 0) {
            status = ABEA_READ_FAIL_NO_END;   // internal inconsistency, reported as no alignment
            n = 0;
        } else if (n > cap) {
            status = ABEA_READ_CAPACITY;
        } else {
            __syncwarp();
            for (int base = 0; base < n; base += 32) {   // move the pairs to the front, ascending
                const int t = base + lane;
                int2 v = make_int2(0, 0);
                if (t < n) v = out[cap - n + t];
                __syncwarp();
                if (t < n) out[t] = v;
                __syncwarp();
            }
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

template <int C, bool MIXED, bool FULLW>
__global__ void __launch_bounds__(kWarps * 32, (C >= 6) ? 2 : 4) align_kernel(const AlignArgs a)
{
    constexpr int R = Rec<C>::R;
    __shared__ __align__(16) uint32_t bt[kWarps][3 * kChunk * R];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
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
        align_read<C, MIXED, FULLW>(a, d, rid, lane, bt[warp]);
        __syncwarp();
    }
}

template <int C, bool MIXED, bool FULLW>
int launch_c(const AlignArgs &a, int grid, void *stream)
{
    align_kernel<C, MIXED, FULLW><<<grid, kWarps * 32, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

template <int C, bool MIXED, bool FULLW>
int grid_c(int device)
{
    int sms = 0, per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return -1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, align_kernel<C, MIXED, FULLW>, kWarps * 32, 0);
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
    g.full = g.L == 32;
    g.rec_words = (2 * C + 3) / 4 * 4;
    return g;
}

#define ABEA_FOR_EACH_C(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8)

int launch_align(const AlignArgs &a, const Geometry &g, int grid, void *stream)
{
#define X(c)                                                                                      \
    if (g.C == c) {                                                                               \
        if (g.mixed)                                                                              \
            return g.full ? launch_c<c, true, true>(a, grid, stream) : launch_c<c, true, false>(a, grid, stream); \
        return g.full ? launch_c<c, false, true>(a, grid, stream) : launch_c<c, false, false>(a, grid, stream);   \
    }
    ABEA_FOR_EACH_C(X)
#undef X
    return (int)cudaErrorInvalidValue;
}

int align_grid_size(const Geometry &g, int device)
{
#define X(c)                                                                                      \
    if (g.C == c) {                                                                               \
        if (g.mixed) return g.full ? grid_c<c, true, true>(device) : grid_c<c, true, false>(device); \
        return g.full ? grid_c<c, false, true>(device) : grid_c<c, false, false>(device);         \
    }
    ABEA_FOR_EACH_C(X)
#undef X
    return -1;
}

}  // namespace abea
