/*
 * abea_oracle.c -- plain CPU oracle of Adaptive Banded Event Alignment (ABEA).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only tests/,
 * __graft_entry__.smoke() and bench.py's CPU-baseline leg may build, load or
 * run it; the library's product path never does.  It shares no code with the
 * CUDA path.
 *
 * The file is compiled twice:
 *   (default)          FP64 scoring, the paper's formulas written out;
 *   -DORACLE_F32       FP32 scoring in the canonical single-precision form
 *                      that the GPU path also uses (see cell_score below),
 *                      so that both make every max/argmax decision on the
 *                      same FP32 values.  In this form every cell carries
 *                      T = S + lp_step (S the paper's score), which makes
 *                      the diagonal candidate T_diag itself; the reported
 *                      score subtracts lp_step again in FP64.
 * Build with -ffp-contract=off: no multiply-add may be fused unless written
 * as fma()/fmaf().
 *
 * What it follows (H. Gamaarachchi, PhD thesis, UNSW 2020, Ch.5):
 *   Alg. adaptivebandedcpu         band initialisation, band loop, move, fill, backtrack
 *   Alg. adaptivebandedcpucompute  the transition constants and the D/U/L cell score
 *   Alg. adaptivebandedcpucomputelog  the Gaussian log-likelihood emission
 *   Sec. ABEA, read-model scaling  mu <- mean*scale + shift
 *   Sec. ABEA, trim states         leading/trailing events may stay unaligned
 * Readings where the paper is silent or garbled (A1-A14 in the design notes):
 *   epsilon = 1e-10 (the printed "1^{-10}");  lp_trim = ln(1/100);
 *   ll_0 = (W/2-1, -1-W/2), ll_1 = ll_0 + one event;  bands 0..n_e+n_k;
 *   move: advance the k-mer iff S[0] < S[W-1], alternate by band parity when
 *   both are -inf;  max ties prefer D, then U, then L;  end cell = first
 *   maximum of S(e, n_k-1) + (n_e-1-e)*lp_trim;  sigma' = var*sigma.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#ifdef ORACLE_F32
typedef float real;
#define NAME(x) x##_f32
#else
typedef double real;
#define NAME(x) x##_f64
#endif

#define ST_OK 0
#define ST_FAIL_NO_END 1
#define ST_BAD_INPUT 2
#define ST_CAPACITY 3
#define ST_NOMEM 4
#define ST_INTERNAL 5

#define TR_D 0
#define TR_U 1
#define TR_L 2

/* FP32 only: every RENORM_PERIOD bands, while the band and the one before
 * lie wholly in the matrix, all their scores are shifted up by R, a multiple
 * of 1024 no larger in magnitude than their maximum (reading A13).  The
 * shift is exact (each difference is representable), so it changes no
 * decision by itself; it keeps the running scores small, so that later FP32
 * additions round at a fine ulp instead of drifting on long reads.  The
 * shift applied so far is carried in FP64 and added back to the end score. */
#define RENORM_PERIOD 64
#define RENORM_BELOW (-2048.0f)

/* ln(1/sqrt(2*pi)) and sqrt(1/2), to 20 digits. */
#define LOG_INV_SQRT_2PI (-0.91893853320467274178)
#define SQRT_HALF 0.70710678118654752440

/* ---------------------------------------------------------------------- */
/* Inputs shared by both precisions (defined once, in the FP64 build).     */

#ifndef ORACLE_F32
/* k-mer rank: lexicographic over A,C,G,T with the first base most
 * significant (reading A11: the thesis only says there are 4^k k-mers).
 * Returns 0, or -1 if a base is not one of ACGT. */
int oracle_kmer_ranks(const char *seq, int32_t seq_len, int32_t k, int32_t *ranks)
{
    int32_t n_k = seq_len - k + 1;
    for (int32_t i = 0; i < n_k; i++) {
        int32_t r = 0;
        for (int32_t t = 0; t < k; t++) {
            int c;
            switch (seq[i + t]) {
            case 'A': c = 0; break;
            case 'C': c = 1; break;
            case 'G': c = 2; break;
            case 'T': c = 3; break;
            default: return -1;
            }
            r = r * 4 + c;
        }
        ranks[i] = r;
    }
    return 0;
}

/* Transition constants of Alg. adaptivebandedcpucompute, in FP64:
 * out = {lp_skip, lp_stay, lp_step, lp_trim}. */
void oracle_constants(int32_t n_events, int32_t n_kmers, double *out)
{
    double events_per_kmer = (double)n_events / (double)n_kmers;
    double epsilon = 1e-10;
    double lp_skip = log(epsilon);
    double lp_stay = log(1.0 - 1.0 / (events_per_kmer + 1.0));
    double lp_step = log(1.0 - exp(lp_skip) - exp(lp_stay));
    double lp_trim = log(1.0 / 100.0);
    out[0] = lp_skip;
    out[1] = lp_stay;
    out[2] = lp_step;
    out[3] = lp_trim;
}
#endif

int oracle_kmer_ranks(const char *seq, int32_t seq_len, int32_t k, int32_t *ranks);
void oracle_constants(int32_t n_events, int32_t n_kmers, double *out);

/* ---------------------------------------------------------------------- */
/* Emission (Alg. adaptivebandedcpucomputelog with read-model scaling).    */

typedef struct {
    real lp_skip, lp_stay, lp_step, lp_trim;
#ifdef ORACLE_F32
    float lp_stay_step;        /* lp_stay - lp_step, FP64 rounded once */
    float *a, *b, *c;          /* per k-mer of the read, see emission() */
#else
    double *mu, *sigma;        /* per k-mer of the read: scaled mean, scaled stdv */
#endif
} read_params;

#ifdef ORACLE_F32
/* FP32 canonical form.  With sigma' = var*sigma and z = (x - mu')/sigma',
 *   lp = ln(1/sqrt(2pi)) - ln(sigma') - z^2/2
 *      = c - z'^2,   z' = z/sqrt(2) = x*a + b,
 *   a = sqrt(1/2)/sigma',  b = -mu'*a,  c = ln(1/sqrt(2pi)) - ln(sigma').
 * The FP32 form returns lp + lp_step (the diagonal transition folded in, see
 * cell_score).  a, b, c are computed per k-mer in FP64 and rounded once:
 *   a = (sqrt(1/2)/sigma) * (1/var),  b = -(mu' * a_fp64),
 *   c = (ln(1/sqrt(2pi)) - ln(sigma)) - (ln(var) - lp_step),
 *   mu' = scale*mean + shift.
 * Then two fused multiply-adds: z' = fmaf(x, a, b), lp = fmaf(-z', z', c). */
static inline float emission(const read_params *p, float x, int32_t k)
{
    float z = fmaf(x, p->a[k], p->b[k]);
    return fmaf(-z, z, p->c[k]);
}
#else
static inline double emission(const read_params *p, float x, int32_t k)
{
    double z = ((double)x - p->mu[k]) / p->sigma[k];
    return LOG_INV_SQRT_2PI - log(p->sigma[k]) - 0.5 * z * z;
}
#endif

/* ---------------------------------------------------------------------- */
/* Cell score (Alg. adaptivebandedcpucompute).                              */

/* margin: winner minus runner-up of the three candidates (+inf when the
 * runner-up is -inf).  FP64 build only uses it for the near-tie record. */
static inline real cell_score(const read_params *p, real up, real left, real diag,
                              real lp_emission, uint8_t *dir, double *margin)
{
#ifdef ORACLE_F32
    /* Every score is carried as T = S + lp_step, and lp_emission here is the
     * emission plus lp_step.  Then, in exact arithmetic,
     *   T_d = S_diag + lp_step + E + lp_step = T_diag + lp_emission,
     *   T_u = S_up + lp_stay + E + lp_step = (T_up + (lp_stay - lp_step)) + lp_emission,
     *   T_l = S_left + lp_skip + lp_step = T_left + lp_skip,
     * and the diagonal candidate needs no addition.  T_d and T_u share
     * lp_emission, so max(T_d, T_u) = max(T_diag, T_up + (lp_stay - lp_step))
     * + lp_emission; rounding is monotone, so this equals the max of the two
     * separately rounded FP32 sums, and the direction is taken before the
     * emission is added (D on ties). */
    real d = diag;
    real u = up + p->lp_stay_step;
    real m;
    uint8_t t;
    if (u > d) { m = u; t = TR_U; } else { m = d; t = TR_D; }
    real s = m + lp_emission;
    real l = left + p->lp_skip;
    if (l > s) { s = l; t = TR_L; }
    *dir = t;
    (void)margin;
    return s;
#else
    real score_d = diag + p->lp_step + lp_emission;
    real score_u = up + p->lp_stay + lp_emission;
    real score_l = left + p->lp_skip;
    real s = score_d;
    uint8_t t = TR_D;
    if (score_u > s) { s = score_u; t = TR_U; }
    if (score_l > s) { s = score_l; t = TR_L; }
    *dir = t;
    if (margin) {
        real second;
        if (t == TR_D) second = fmax(score_u, score_l);
        else if (t == TR_U) second = fmax(score_d, score_l);
        else second = fmax(score_d, score_u);
        *margin = (second == -INFINITY) ? INFINITY : (double)(s - second);
    }
    return s;
#endif
}

/* ---------------------------------------------------------------------- */
/* Per-read set-up shared by the banded and the full DP.                   */

static int setup_read(const float *model_mean, const float *model_stdv, int32_t k,
                      const char *seq, int32_t seq_len, const float *events, int32_t n_events,
                      float scale, float shift, float var, read_params *p, int32_t **ranks_out)
{
    *ranks_out = NULL;
    memset(p, 0, sizeof(*p));
    if (k < 1 || k > 15 || seq_len < k || n_events < 1) return ST_BAD_INPUT;
    if (!isfinite(scale) || !isfinite(shift) || !isfinite(var) || !(var > 0.0f)) return ST_BAD_INPUT;
    for (int32_t e = 0; e < n_events; e++)
        if (!isfinite(events[e])) return ST_BAD_INPUT;
    int32_t n_k = seq_len - k + 1;
    int32_t *ranks = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_k);
    if (!ranks) return ST_NOMEM;
    if (oracle_kmer_ranks(seq, seq_len, k, ranks) != 0) { free(ranks); return ST_BAD_INPUT; }
    for (int32_t i = 0; i < n_k; i++) {
        float m = model_mean[ranks[i]], s = model_stdv[ranks[i]];
        if (!isfinite(m) || !isfinite(s) || !(s > 0.0f)) { free(ranks); return ST_BAD_INPUT; }
    }
    double c[4];
    oracle_constants(n_events, n_k, c);
    p->lp_skip = (real)c[0];
    p->lp_stay = (real)c[1];
    p->lp_step = (real)c[2];
    p->lp_trim = (real)c[3];
#ifdef ORACLE_F32
    p->a = (float *)malloc(sizeof(float) * (size_t)n_k);
    p->b = (float *)malloc(sizeof(float) * (size_t)n_k);
    p->c = (float *)malloc(sizeof(float) * (size_t)n_k);
    if (!p->a || !p->b || !p->c) { free(ranks); return ST_NOMEM; }
    p->lp_stay_step = (float)(c[1] - c[2]);
    double dscale = scale, dshift = shift, dvar = var;
    double inv_var = 1.0 / dvar, log_var_step = log(dvar) - c[2];
    for (int32_t i = 0; i < n_k; i++) {
        double mean = model_mean[ranks[i]], sd = model_stdv[ranks[i]];
        double mu_p = dscale * mean + dshift;
        double a = (SQRT_HALF / sd) * inv_var;
        p->a[i] = (float)a;
        p->b[i] = (float)(-(mu_p * a));
        p->c[i] = (float)((LOG_INV_SQRT_2PI - log(sd)) - log_var_step);
    }
#else
    p->mu = (double *)malloc(sizeof(double) * (size_t)n_k);
    p->sigma = (double *)malloc(sizeof(double) * (size_t)n_k);
    if (!p->mu || !p->sigma) { free(ranks); return ST_NOMEM; }
    for (int32_t i = 0; i < n_k; i++) {
        p->mu[i] = (double)model_mean[ranks[i]] * (double)scale + (double)shift;
        p->sigma[i] = (double)model_stdv[ranks[i]] * (double)var;
    }
#endif
    *ranks_out = ranks;
    return ST_OK;
}

static void free_read(read_params *p, int32_t *ranks)
{
#ifdef ORACLE_F32
    free(p->a); free(p->b); free(p->c);
#else
    free(p->mu); free(p->sigma);
#endif
    free(ranks);
}

/* ---------------------------------------------------------------------- */
/* Banded ABEA (Alg. adaptivebandedcpu).                                    */

typedef struct {
    double score;          /* best end score (A12), -inf if none */
    int32_t status;
    int32_t n_pairs;       /* pairs written (or required, on ST_CAPACITY) */
    int32_t e_end;         /* event of the end cell */
    int64_t cells;         /* in-matrix cells filled (the throughput unit) */
    double min_margin;     /* FP64 near-tie record (A15), +inf if none */
} oracle_result;

/*
 * One read.  pairs: int32[2*cap] (event, k-mer) in ascending order.
 * Optional debug outputs (may be NULL): ll_out int32[2*n_bands] holding
 * (event, k-mer) of each band's offset-0 cell, and band_scores
 * real[n_bands*W].
 */
int NAME(oracle_abea)(const float *model_mean, const float *model_stdv, int32_t k,
                      const char *seq, int32_t seq_len, const float *events, int32_t n_events,
                      float scale, float shift, float var, int32_t W,
                      int32_t *pairs, int32_t cap, oracle_result *res,
                      int32_t *ll_out, real *band_scores)
{
    res->score = -INFINITY;
    res->status = ST_BAD_INPUT;
    res->n_pairs = 0;
    res->e_end = -1;
    res->cells = 0;
    res->min_margin = INFINITY;
    if (W < 2) return ST_BAD_INPUT;

    read_params p;
    int32_t *ranks;
    int st = setup_read(model_mean, model_stdv, k, seq, seq_len, events, n_events,
                        scale, shift, var, &p, &ranks);
    if (st != ST_OK) { free_read(&p, ranks); res->status = st; return st; }

    const int32_t n_e = n_events, n_k = seq_len - k + 1;
    const int64_t n_bands = (int64_t)n_e + n_k + 1;    /* bands 0..n_e+n_k (A4) */
    real *S = (real *)malloc(sizeof(real) * (size_t)(n_bands * W));
    uint8_t *T = (uint8_t *)malloc((size_t)(n_bands * W));
    int32_t *ll_e = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_bands);
    int32_t *ll_k = (int32_t *)malloc(sizeof(int32_t) * (size_t)n_bands);
#ifndef ORACLE_F32
    float *M = (float *)malloc(sizeof(float) * (size_t)(n_bands * W));   /* cell margins */
#endif
    if (!S || !T || !ll_e || !ll_k
#ifndef ORACLE_F32
        || !M
#endif
    ) {
        free(S); free(T); free(ll_e); free(ll_k);
#ifndef ORACLE_F32
        free(M);
#endif
        free_read(&p, ranks);
        res->status = ST_NOMEM;
        return ST_NOMEM;
    }
    for (int64_t i = 0; i < n_bands * W; i++) {
        S[i] = -INFINITY;
        T[i] = TR_D;
#ifndef ORACLE_F32
        M[i] = INFINITY;
#endif
    }
    double min_margin = INFINITY;
    double *band_frame = (double *)calloc((size_t)n_bands, sizeof(double));   /* shift of each band's scores */
    double frame = 0.0;
    if (!band_frame) { res->status = ST_NOMEM; free(S); free(T); free(ll_e); free(ll_k);
#ifndef ORACLE_F32
        free(M);
#endif
        free_read(&p, ranks); return ST_NOMEM; }

    /* Band b holds the cells with e + k = b - 2; offset j of band b is the
     * cell (ll_e[b] - j, ll_k[b] + j).  Offset 0 is the band's max-event end,
     * offset W-1 its max-k-mer end. */
#define SCORE(b, j) S[(int64_t)(b) * W + (j)]
#define TRACE(b, j) T[(int64_t)(b) * W + (j)]

    /* initialise_first_two_bands: band 0 is placed so that the origin
     * (-1,-1) sits at offset W/2 (score 0); band 1 is band 0 moved by one
     * event, and holds the first trim cell (0,-1). */
    const int32_t half = W / 2;
    ll_e[0] = half - 1;
    ll_k[0] = -1 - half;
    ll_e[1] = ll_e[0] + 1;
    ll_k[1] = ll_k[0];
    SCORE(0, half) = 0;
    SCORE(1, ll_e[1] - 0) = p.lp_trim;          /* cell (0,-1) */
    TRACE(1, ll_e[1] - 0) = TR_U;
#ifdef ORACLE_F32
    SCORE(0, half) += p.lp_step;                /* T = S + lp_step */
    SCORE(1, ll_e[1] - 0) += p.lp_step;
#endif

    for (int64_t b = 2; b < n_bands; b++) {
        /* suzuki_kasahara_rule on the previous band's two end cells */
        real lower_left = SCORE(b - 1, 0);
        real upper_right = SCORE(b - 1, W - 1);
        int advance_kmer;
        if (lower_left == -INFINITY && upper_right == -INFINITY) {
            advance_kmer = (int)(b & 1);
        } else {
            advance_kmer = lower_left < upper_right;
#ifndef ORACLE_F32
            if (lower_left != -INFINITY && upper_right != -INFINITY) {
                double mg = fabs((double)lower_left - (double)upper_right);
                if (mg < min_margin) min_margin = mg;
            }
#endif
        }
        if (advance_kmer) {          /* move along the k-mer axis */
            ll_e[b] = ll_e[b - 1];
            ll_k[b] = ll_k[b - 1] + 1;
        } else {                     /* move along the event axis */
            ll_e[b] = ll_e[b - 1] + 1;
            ll_k[b] = ll_k[b - 1];
        }

        /* trim state: the cell (e,-1) scores (e+1)*lp_trim */
        int32_t jt = -1 - ll_k[b];
        if (jt >= 0 && jt < W) {
            int32_t e = ll_e[b] - jt;
            if (e >= 0 && e < n_e) {
                SCORE(b, jt) = (real)(e + 1) * p.lp_trim;
#ifdef ORACLE_F32
                SCORE(b, jt) += p.lp_step;
#endif
                TRACE(b, jt) = TR_U;
            }
        }

        /* fill the cells of band b that lie in the matrix */
        for (int32_t j = 0; j < W; j++) {
            int32_t e = ll_e[b] - j, kk = ll_k[b] + j;
            if (e < 0 || e >= n_e || kk < 0 || kk >= n_k) continue;
            int32_t j_up = ll_e[b - 1] - (e - 1);        /* (e-1, k)   in band b-1 */
            int32_t j_left = (kk - 1) - ll_k[b - 1];      /* (e, k-1)   in band b-1 */
            int32_t j_diag = (kk - 1) - ll_k[b - 2];      /* (e-1, k-1) in band b-2 */
            real up = (j_up >= 0 && j_up < W) ? SCORE(b - 1, j_up) : -INFINITY;
            real left = (j_left >= 0 && j_left < W) ? SCORE(b - 1, j_left) : -INFINITY;
            real diag = (j_diag >= 0 && j_diag < W) ? SCORE(b - 2, j_diag) : -INFINITY;
            real lp_emission = emission(&p, events[e], kk);
            uint8_t dir;
#ifdef ORACLE_F32
            SCORE(b, j) = cell_score(&p, up, left, diag, lp_emission, &dir, NULL);
#else
            double mg;
            SCORE(b, j) = cell_score(&p, up, left, diag, lp_emission, &dir, &mg);
            M[(int64_t)b * W + j] = (float)mg;
#endif
            TRACE(b, j) = dir;
            res->cells++;
        }
#ifdef ORACLE_F32
        if (b % RENORM_PERIOD == 0 && ll_e[b - 1] >= W - 1 && ll_k[b - 1] >= 0 &&
            ll_e[b - 1] + 1 < n_e && ll_k[b - 1] + W + 1 < n_k) {
            float top = -INFINITY;
            for (int32_t j = 0; j < W; j++) {
                top = fmaxf(top, SCORE(b, j));
                top = fmaxf(top, SCORE(b - 1, j));
            }
            if (top <= RENORM_BELOW) {
                float R = -1024.0f * floorf(-top / 1024.0f);
                for (int32_t j = 0; j < W; j++) {
                    SCORE(b, j) -= R;
                    SCORE(b - 1, j) -= R;
                }
                frame += (double)R;
            }
        }
#endif
        band_frame[b] = frame;
    }

    /* end cell (A12): over events e, the cell (e, n_k-1) in band e+n_k+1;
     * the remaining n_e-1-e events are trimmed at lp_trim each. */
    double best = -INFINITY, second = -INFINITY;
    int32_t e_best = -1;
    for (int32_t e = 0; e < n_e; e++) {
        int64_t b = (int64_t)e + n_k + 1;
        int32_t j = ll_e[b] - e;
        if (j < 0 || j >= W) continue;
        double cand = band_frame[b] + (double)(SCORE(b, j) + (real)(n_e - 1 - e) * p.lp_trim);
        if (cand > best) { second = best; best = cand; e_best = e; }
        else if (cand > second) second = cand;
    }
#ifndef ORACLE_F32
    if (best != -INFINITY && second != -INFINITY && best - second < min_margin)
        min_margin = best - second;
#endif
#ifdef ORACLE_F32
    res->score = (double)(float)(best - (double)p.lp_step);   /* S = T - lp_step, in FP64 */
#else
    res->score = best;
#endif
    res->e_end = e_best;

    if (best == -INFINITY) {
        res->status = ST_FAIL_NO_END;
    } else {
        /* backtrack from (e_best, n_k-1) until an index leaves the matrix */
        int32_t e = e_best, kk = n_k - 1, n = 0;
        int overflow = 0;
        while (e >= 0 && kk >= 0) {
            int64_t b = (int64_t)e + kk + 2;
            int32_t j = ll_e[b] - e;
            if (j < 0 || j >= W) { res->status = ST_INTERNAL; overflow = 2; break; } /* cannot happen */
            if (n < cap) { pairs[2 * n] = e; pairs[2 * n + 1] = kk; }
            else overflow = 1;
            n++;
#ifndef ORACLE_F32
            float mg = M[b * W + j];
            if (mg < min_margin) min_margin = mg;
#endif
            uint8_t t = TRACE(b, j);
            if (t == TR_D) { e--; kk--; }
            else if (t == TR_U) { e--; }
            else { kk--; }
        }
        if (overflow == 2) {
            n = 0;
        } else if (overflow) {
            res->status = ST_CAPACITY;
        } else {
            for (int32_t i = 0; i < n / 2; i++) {          /* ascending order */
                int32_t te = pairs[2 * i], tk = pairs[2 * i + 1];
                pairs[2 * i] = pairs[2 * (n - 1 - i)];
                pairs[2 * i + 1] = pairs[2 * (n - 1 - i) + 1];
                pairs[2 * (n - 1 - i)] = te;
                pairs[2 * (n - 1 - i) + 1] = tk;
            }
            res->status = ST_OK;
        }
        res->n_pairs = n;
    }
    res->min_margin = min_margin;

    if (ll_out)
        for (int64_t b = 0; b < n_bands; b++) { ll_out[2 * b] = ll_e[b]; ll_out[2 * b + 1] = ll_k[b]; }
    if (band_scores) memcpy(band_scores, S, sizeof(real) * (size_t)(n_bands * W));
#undef SCORE
#undef TRACE
    free(band_frame);
    free(S); free(T); free(ll_e); free(ll_k);
#ifndef ORACLE_F32
    free(M);
#endif
    free_read(&p, ranks);
    return res->status;
}

/* ---------------------------------------------------------------------- */
/* Unbanded DP over the whole augmented matrix [-1,n_e) x [-1,n_k), with   */
/* the same recurrence, trim column, end rule and backtrack.  With a band  */
/* wide enough to hold every cell, banded ABEA must reproduce it.          */

int NAME(oracle_full_dp)(const float *model_mean, const float *model_stdv, int32_t k,
                         const char *seq, int32_t seq_len, const float *events, int32_t n_events,
                         float scale, float shift, float var,
                         int32_t *pairs, int32_t cap, oracle_result *res)
{
    res->score = -INFINITY;
    res->status = ST_BAD_INPUT;
    res->n_pairs = 0;
    res->e_end = -1;
    res->cells = 0;
    res->min_margin = INFINITY;
    read_params p;
    int32_t *ranks;
    int st = setup_read(model_mean, model_stdv, k, seq, seq_len, events, n_events,
                        scale, shift, var, &p, &ranks);
    if (st != ST_OK) { free_read(&p, ranks); res->status = st; return st; }
    const int32_t n_e = n_events, n_k = seq_len - k + 1;
    const int64_t R = n_e + 1, C = n_k + 1;            /* row e+1, column k+1 */
    real *S = (real *)malloc(sizeof(real) * (size_t)(R * C));
    uint8_t *T = (uint8_t *)malloc((size_t)(R * C));
    if (!S || !T) { free(S); free(T); free_read(&p, ranks); res->status = ST_NOMEM; return ST_NOMEM; }
#define FS(e, kk) S[((int64_t)(e) + 1) * C + (kk) + 1]
#define FT(e, kk) T[((int64_t)(e) + 1) * C + (kk) + 1]
    for (int64_t i = 0; i < R * C; i++) { S[i] = -INFINITY; T[i] = TR_D; }
    FS(-1, -1) = 0;
    for (int32_t e = 0; e < n_e; e++) { FS(e, -1) = (real)(e + 1) * p.lp_trim; FT(e, -1) = TR_U; }
#ifdef ORACLE_F32
    FS(-1, -1) += p.lp_step;                    /* T = S + lp_step */
    for (int32_t e = 0; e < n_e; e++) FS(e, -1) += p.lp_step;
#endif
    for (int32_t e = 0; e < n_e; e++)
        for (int32_t kk = 0; kk < n_k; kk++) {
            uint8_t dir;
            FS(e, kk) = cell_score(&p, FS(e - 1, kk), FS(e, kk - 1), FS(e - 1, kk - 1),
                                   emission(&p, events[e], kk), &dir, NULL);
            FT(e, kk) = dir;
            res->cells++;
        }
    real best = -INFINITY;
    int32_t e_best = -1;
    for (int32_t e = 0; e < n_e; e++) {
        real cand = FS(e, n_k - 1) + (real)(n_e - 1 - e) * p.lp_trim;
        if (cand > best) { best = cand; e_best = e; }
    }
#ifdef ORACLE_F32
    res->score = (double)(float)((double)best - (double)p.lp_step);   /* S = T - lp_step, in FP64 */
#else
    res->score = best;
#endif
    res->e_end = e_best;
    if (best == -INFINITY) {
        res->status = ST_FAIL_NO_END;
    } else {
        int32_t e = e_best, kk = n_k - 1, n = 0;
        while (e >= 0 && kk >= 0) {
            if (n < cap) { pairs[2 * n] = e; pairs[2 * n + 1] = kk; }
            n++;
            uint8_t t = FT(e, kk);
            if (t == TR_D) { e--; kk--; }
            else if (t == TR_U) { e--; }
            else { kk--; }
        }
        if (n > cap) {
            res->status = ST_CAPACITY;
        } else {
            for (int32_t i = 0; i < n / 2; i++) {
                int32_t te = pairs[2 * i], tk = pairs[2 * i + 1];
                pairs[2 * i] = pairs[2 * (n - 1 - i)];
                pairs[2 * i + 1] = pairs[2 * (n - 1 - i) + 1];
                pairs[2 * (n - 1 - i)] = te;
                pairs[2 * (n - 1 - i) + 1] = tk;
            }
            res->status = ST_OK;
        }
        res->n_pairs = n;
    }
#undef FS
#undef FT
    free(S); free(T);
    free_read(&p, ranks);
    return res->status;
}

/* ---------------------------------------------------------------------- */
/* A batch of reads over n_threads POSIX threads (reads taken one at a     */
/* time from a shared counter).  Used for whole-batch parity and for the   */
/* CPU baseline timing.  Arrays are packed: read i's bases are             */
/* seq[seq_off[i]..seq_off[i+1]), its events events[ev_off[i]..), its      */
/* pairs pairs[2*pair_off[i]..2*pair_off[i+1]).                            */

typedef struct {
    const float *model_mean, *model_stdv;
    int32_t k, W;
    const char *seq;
    const int64_t *seq_off;
    const float *events;
    const int64_t *ev_off;
    const float *scalings;
    int32_t *pairs;
    const int64_t *pair_off;
    oracle_result *res;
    int32_t n;
    volatile int32_t next;
    pthread_mutex_t lock;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&j->lock);
        int32_t i = j->next++;
        pthread_mutex_unlock(&j->lock);
        if (i >= j->n) break;
        NAME(oracle_abea)(j->model_mean, j->model_stdv, j->k,
                          j->seq + j->seq_off[i], (int32_t)(j->seq_off[i + 1] - j->seq_off[i]),
                          j->events + j->ev_off[i], (int32_t)(j->ev_off[i + 1] - j->ev_off[i]),
                          j->scalings[3 * i], j->scalings[3 * i + 1], j->scalings[3 * i + 2], j->W,
                          j->pairs + 2 * j->pair_off[i], (int32_t)(j->pair_off[i + 1] - j->pair_off[i]),
                          &j->res[i], NULL, NULL);
    }
    return NULL;
}

int NAME(oracle_abea_batch)(const float *model_mean, const float *model_stdv, int32_t k, int32_t W,
                            int32_t n, const char *seq, const int64_t *seq_off,
                            const float *events, const int64_t *ev_off, const float *scalings,
                            int32_t *pairs, const int64_t *pair_off, oracle_result *res,
                            int32_t n_threads)
{
    batch_job j;
    j.model_mean = model_mean; j.model_stdv = model_stdv; j.k = k; j.W = W;
    j.seq = seq; j.seq_off = seq_off; j.events = events; j.ev_off = ev_off;
    j.scalings = scalings; j.pairs = pairs; j.pair_off = pair_off; j.res = res;
    j.n = n; j.next = 0;
    pthread_mutex_init(&j.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    int started = 0;
    for (int t = 0; t < n_threads; t++)
        if (pthread_create(&th[t], NULL, batch_worker, &j) == 0) started++;
        else break;
    if (started == 0) batch_worker(&j);
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&j.lock);
    return 0;
}
