// Per-read scaling estimate (method of moments): the shift and scale that
// ABEA applies to the pore model (thesis Sec. "Read-model scaling": the model
// means become mu * scale + shift, both estimated per read before ABEA).
//
// The thesis names the method but not its formula; this file takes the plain
// reading: match the first two moments (population mean and variance) of the
// read's event means to those of the model level means along the read's
// k-mer sequence,
//   scale = sqrt(v_e / v_m),  shift = m_e - scale * m_m,  var = 1.
// A read with fewer than two events or a zero variance is degenerate
// (scale 1, shift m_e - m_m); a read without events or k-mers, with a base
// outside ACGT or a non-finite event is rejected (scale 1, shift 0).
//
// One block per read, one pass over its events and bases.  FP64 arithmetic
// is slow on this GPU, so each thread sums in FP32 without losing bits: a
// running sum is a pair (hi, lo) of floats, each addition an error-free
// TwoSum (Knuth: hi + x = s + err exactly) whose error goes into lo, and each
// square an error-free product (p = x*x, fma(x, x, -p) = its rounding error).
// The pairs (about 48 significant bits) merge the same way across the block
// and only the block's sums are widened to FP64; the variance is
// E[x^2] - E[x]^2 in FP64 (the cancellation costs a
// few bits of 53).  The results agree with the two-pass FP64 definition to
// within a float rounding.
#include "abea_internal.h"

namespace abea {

namespace {

constexpr int kThreads = 256;

// 2-bit code of an ACGT base, branch-free: ((c >> 1) ^ (c >> 2)) & 3 maps the
// ASCII codes of A C G T to 0 1 2 3.
__device__ __forceinline__ unsigned base_code(unsigned c) { return ((c >> 1) ^ (c >> 2)) & 3u; }

// c is one of A C G T: c - 'A' is 0, 2, 6 or 19.
__device__ __forceinline__ bool is_base(unsigned c)
{
    const unsigned d = c - 'A';
    return d < 32u && ((0x80045u >> d) & 1u);
}

// A float sum carried as hi + lo.
struct DSum {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float s = __fadd_rn(hi, x);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    __device__ __forceinline__ void add_square(float x)
    {
        const float p = __fmul_rn(x, x);
        const float pe = __fmaf_rn(x, x, -p);
        add(p);
        lo = __fadd_rn(lo, pe);
    }
    // this + o, error-free on the hi parts
    __device__ __forceinline__ void merge(const DSum &o)
    {
        add(o.hi);
        lo = __fadd_rn(lo, o.lo);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// The sum over the block of every thread's pair, as a double in every thread:
// the pairs merge in FP32 (a warp tree, then the warps' results in order), and
// only the block's result is widened.
__device__ __forceinline__ double block_sum(DSum v, float2 *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        DSum w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v.merge(w);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();                        // red is free again
    if (lane == 0) red[warp] = make_float2(v.hi, v.lo);
    __syncthreads();
    DSum s;
#pragma unroll
    for (int w = 0; w < kThreads / 32; w++) {
        DSum t;
        t.hi = red[w].x;
        t.lo = red[w].y;
        s.merge(t);
    }
    return s.value();
}

__global__ void __launch_bounds__(kThreads) scalings_kernel(const int64_t *seq_off, const int64_t *ev_off, int32_t n,
                                                          const uint8_t *seq, const float *events,
                                                          const float2 *model_f, int k, abea_scalings *out,
                                                          int32_t *status)
{
    __shared__ float2 red[kThreads / 32];
    const int i = blockIdx.x;
    if (i >= n) return;
    const int64_t n_e = ev_off[i + 1] - ev_off[i];
    const int64_t n_k = (seq_off[i + 1] - seq_off[i]) - k + 1;
    const float *ev = events + ev_off[i];
    const uint8_t *sq = seq + seq_off[i];
    int bad = (n_e < 1 || n_k < 1) ? 1 : 0;

    DSum se, qe, sm, qm;
    const int ne = (int)n_e, nk = (int)n_k;            // a read's counts fit 32 bits (checked on the host)
    for (int t = threadIdx.x; t < ne; t += kThreads) {
        const float x = ev[t];
        if (!isfinite(x)) bad = 1;
        se.add(x);
        qe.add_square(x);
    }
    // k-mers [a, b) of this thread, contiguous, ranks rolled forward one base at a time
    const int per = (nk + kThreads - 1) / kThreads;
    const int a = min(nk, (int)threadIdx.x * per), b = min(nk, a + per);
    if (a < b) {
        const unsigned mask = (k >= 16) ? 0xffffffffu : ((1u << (2 * k)) - 1u);
        unsigned r = 0;
        for (int j = 0; j < k - 1; j++) {
            const unsigned c = sq[a + j];
            if (!is_base(c)) bad = 1;
            r = (r << 2) | base_code(c);
        }
        for (int t = a; t < b; t++) {
            const unsigned c = sq[t + k - 1];
            if (!is_base(c)) bad = 1;
            r = ((r << 2) | base_code(c)) & mask;
            const float mu = model_f[r].x;
            sm.add(mu);
            qm.add_square(mu);
        }
    }
    bad = __syncthreads_or(bad);
    if (bad) se = qe = sm = qm = DSum();
    const double s_e = block_sum(se, red);
    const double q_e = block_sum(qe, red);
    const double s_m = block_sum(sm, red);
    const double q_m = block_sum(qm, red);
    if (threadIdx.x == 0) {
        abea_scalings s;
        s.var = 1.0f;
        int st;
        if (bad) {
            st = ABEA_SCALE_BAD_INPUT;
            s.scale = 1.0f;
            s.shift = 0.0f;
        } else {
            const double m_e = s_e / (double)n_e, m_m = s_m / (double)n_k;
            const double v_e = q_e / (double)n_e - m_e * m_e, v_m = q_m / (double)n_k - m_m * m_m;
            if (n_e < 2 || !(v_e > 0.0) || !(v_m > 0.0)) {
                st = ABEA_SCALE_DEGENERATE;
                s.scale = 1.0f;
                s.shift = (float)(m_e - m_m);
            } else {
                const double scale = sqrt(v_e / v_m);
                st = ABEA_SCALE_OK;
                s.scale = (float)scale;
                s.shift = (float)(m_e - scale * m_m);
            }
        }
        out[i] = s;
        status[i] = st;
    }
}

}  // namespace

int launch_scalings(const int64_t *d_seq_off, const int64_t *d_ev_off, int32_t n, const uint8_t *seq,
                    const float *events, const float2 *model_f, int k, abea_scalings *out, int32_t *status,
                    void *stream)
{
    if (n <= 0) return (int)cudaSuccess;
    scalings_kernel<<<n, kThreads, 0, (cudaStream_t)stream>>>(d_seq_off, d_ev_off, n, seq, events, model_f, k, out,
                                                              status);
    return (int)cudaGetLastError();
}

}  // namespace abea
