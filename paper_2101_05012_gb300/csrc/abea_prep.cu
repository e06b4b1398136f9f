// Pre-kernel: per-read k-mer cache and input checks.
//
// The thesis's pre-kernel (Alg. adaptivebandedcudapre) fills, for every read,
// a "kcache" holding the pore-model entry of each of the read's k-mers in
// read order, so that the core kernel reads the model sequentially instead of
// at random.  Here the cache entry is already the emission's per-k-mer
// operands, with the read-model scaling applied (thesis Sec. ABEA,
// read-model scaling): for sigma' = var*stdv and mu' = scale*mean + shift,
//   a = sqrt(1/2)/sigma',  b = -mu'*a,  c = ln(1/sqrt(2 pi)) - ln(sigma'),
// so that the emission of Alg. adaptivebandedcpucomputelog is
//   ln(1/sqrt(2 pi)) - ln(sigma') - ((x-mu')/sigma')^2/2 = c - (x*a + b)^2.
// The core kernel carries every score as S + lp_step, so its c also holds
// the read's lp_step (the diagonal transition): c = (ln(1/sqrt(2 pi)) -
// ln(stdv)) - (ln(var) - lp_step).  a, b, c are formed in FP64 (explicitly
// rounded operations, never fused) and rounded once to FP32.  The same kernel checks the read's bases and
// events and flags the read when one is invalid.
#include <algorithm>

#include "abea_internal.h"

namespace abea {

namespace {

__device__ __forceinline__ int base_code(uint8_t c)
{
    switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
    }
}

}  // namespace

// A double rounded to the nearest float (ties to even), as __double2float_rn
// gives it, with integer operations for results in the normal float range:
// on GB300 the conversion instruction runs on the FP64 pipe, which the
// pre-kernel's arithmetic already keeps busy.  Zero, subnormal and
// out-of-range inputs (and inf, NaN) take the conversion instruction.
__device__ float f32_from_f64(double v)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
    const int e = (int)((hi >> 20) & 0x7ffu);                      // biased FP64 exponent
    if (e < 1023 - 126 || e > 1023 + 127) return __double2float_rn(v);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);        // the top 23 of the 52 mantissa bits
    const unsigned rest = lo & 0x1fffffffu;                        // the 29 bits rounded away
    const unsigned half = 0x10000000u;
    const unsigned up = (rest > half || (rest == half && (m & 1u))) ? 1u : 0u;
    // a carry out of the mantissa moves into the exponent, and past the largest float to +-inf
    return __uint_as_float(((hi & 0x80000000u) | ((unsigned)(e - 1023 + 127) << 23) | m) + up);
}

namespace {

// One block per read.
__global__ void __launch_bounds__(256) prep_kernel(const ReadDesc *__restrict__ rd, int32_t n,
                                                   const uint8_t *__restrict__ seq,
                                                   const float *__restrict__ events,
                                                   const ModelRow *__restrict__ model, int k,
                                                   float4 *__restrict__ kc, int32_t *__restrict__ flags)
{
    const int r = blockIdx.x;
    if (r >= n) return;
    const ReadDesc d = rd[r];
    int bad = d.host_bad;
    if (!d.host_bad) {
        const uint8_t *s = seq + d.seq_off;
        float4 *out = kc + d.kc_off;
        for (int i = threadIdx.x; i < d.n_k; i += blockDim.x) {
            uint32_t rank = 0;
            bool ok = true;
            for (int t = 0; t < k; t++) {
                int c = base_code(s[i + t]);
                ok &= c >= 0;
                rank = rank * 4u + (uint32_t)(c & 3);
            }
            if (!ok) {
                bad = 1;
                out[i] = make_float4(1.0f, 0.0f, -__int_as_float(0x7f800000), 0.0f);
                continue;
            }
            const ModelRow m = model[rank];
            const double mu_p = __dadd_rn(__dmul_rn(d.scale, m.mu), d.shift);
            const double a = __dmul_rn(m.a0, d.inv_var);
            const double b = -__dmul_rn(mu_p, a);
            const double c = __dsub_rn(m.c0, d.log_var_step);
            out[i] = make_float4(f32_from_f64(a), f32_from_f64(b), f32_from_f64(c), 0.0f);
        }
        const float *ev = events + d.ev_off;
        for (int e = threadIdx.x; e < d.n_e; e += blockDim.x) {
            const float x = ev[e];
            if (!isfinite(x)) bad = 1;               // NaN or +-inf (every finite event is aligned)
        }
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) flags[r] = bad;
}

}  // namespace

namespace {

__global__ void __launch_bounds__(256) f32_from_f64_kernel(const double *in, long long n, float *out)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x)
        out[j] = f32_from_f64(in[j]);
}

}  // namespace

int launch_f32_from_f64(const double *in, int64_t n, float *out, void *stream)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    f32_from_f64_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(in, n, out);
    return (int)cudaGetLastError();
}

int launch_prep(const ReadDesc *rd, int32_t n, const uint8_t *seq, const float *events,
                const ModelRow *model, int k, float4 *kc, int32_t *flags, void *stream)
{
    if (n <= 0) return cudaSuccess;
    prep_kernel<<<n, 256, 0, (cudaStream_t)stream>>>(rd, n, seq, events, model, k, kc, flags);
    return (int)cudaGetLastError();
}

}  // namespace abea
