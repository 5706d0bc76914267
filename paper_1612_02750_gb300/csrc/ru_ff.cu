// ru_ff.cu -- the reliable update's operator in float-float arithmetic.
//
// A mixed-precision solve recomputes its residual r = b - A x from the FP64
// solution and the FP64 links every time the iterated residual has dropped
// by delta (reliable update).  In FP64 arithmetic the two Dslash passes of an
// update are bound by the GPU's FP64 rate (two FMAs per SM and clock: 288
// FMAs a site take about 2.6 times as long as the pass's HBM traffic).  The
// updates that cannot end the solve run here instead: every real is carried
// as an unevaluated sum hi + lo of two FP32 numbers (about 47 significant
// bits), on the FP32 pipes.
//
// * FP64 inputs are split as they are loaded, with integer instructions: hi
//   takes the leading 24 bits of the significand (truncated), lo the next 23;
//   the split is exact up to 2^-46 of the value.  Vectors are carried times
//   2^ff_k (about unit size a real, from ||b||^2): an exact rescaling that
//   keeps them far from FP32's range limits.
// * A product a b of two pairs is hi_a hi_b with its exact rounding error
//   (one FMA) plus the cross terms hi_a lo_b + lo_a hi_b; sums keep their
//   rounding error with the two-sum of Knuth (TAOCP vol. 2, 4.2.2) and
//   Moller, so that nothing is lost to the order of the terms.
// * The error of an update (measured: about 1e-13 of ||x|| + ||b||) enters
//   the next inner cycle's true residual.  At small mass ||x|| is many times
//   ||b||, so the kernel that folds the inner iterate into x (blas.cu,
//   accum_x_kernel) hands the update back to FP64 unless that error stays
//   below 1e-3 of the iterated residual that asked for it.  The update that
//   may accept convergence (asked for when the iterated residual meets tol,
//   or at maxiter) and the first one run in FP64, so the solve's stopping
//   test is always an FP64 true residual.
#include "qex_kernels.cuh"

namespace qex {

struct FF {
    float hi, lo;
};

// 256 threads a block, 3 blocks per SM (80 registers) without the Naik term,
// 2 with it (128 registers; 80 spill).  32^4, the update's two passes:
// 0.33 ms at 256 x 3 against 0.35 (256 x 2), 0.37-0.39 (128 x 4..8, 64 x 8).
constexpr int kFfBlock = 256;
template <bool NAIK>
struct FfMinBlocks {
    static constexpr int value = NAIK ? 2 : 3;
};

// Split bounds of one kind of input (links: scale 2^0; vectors: 2^ff_k).
struct FfSplit {
    uint32_t bias;  // added to (high word << 3): rebases the exponent, 1023 - 127 - k
    uint32_t tiny;  // |high word| below this: the value is taken as 0 (|d| 2^k < 2^-103)
    uint32_t huge;  // |high word| from this: NaN (|d| 2^k >= 2^127, Inf, NaN)
};

__host__ __device__ inline FfSplit ff_split_bounds(int k) {
    FfSplit s;
    s.bias = 0x40000000u + ((uint32_t)k << 23);
    s.tiny = (uint32_t)(920 - k) << 20;
    s.huge = (uint32_t)(1151 - k) << 20;
    return s;
}

// d 2^k = hi + lo + e with |e| < 2^-46 |d 2^k|.  The double's exponent field
// e11 and significand bits m[51..0]: hi has exponent e11 - 1023 + k and
// significand m[51..29] (the shift by 3 lines m[51..29] up with the float
// significand, and the bias rebases the low 9 exponent bits modulo 512, which
// is exact over the accepted range); lo = m[28..6] 2^(E - 46) with E hi's
// unbiased exponent, formed as (2^(E-23) (1 + m/2^23)) - 2^(E-23).
__device__ __forceinline__ FF split_d(double d, const FfSplit &sp) {
    const uint32_t H = (uint32_t)__double2hiint(d), L = (uint32_t)__double2loint(d);
    const uint32_t mag = H & 0x7FFFFFFFu;
    const uint32_t hb = (__funnelshift_l(L, H, 3) + sp.bias) | (H & 0x80000000u);
    const uint32_t es = (hb & 0xFF800000u) - (23u << 23);
    FF r;
    r.hi = __uint_as_float(hb);
    r.lo = __uint_as_float(es | ((L >> 6) & 0x7FFFFFu)) - __uint_as_float(es);
    if (mag < sp.tiny) r.hi = r.lo = 0.f;
    if (mag >= sp.huge) r.hi = r.lo = __uint_as_float(0x7FC00000u);
    return r;
}

// s + e = a + b exactly (no condition on the magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bv = s - a;
    e = (a - (s - bv)) + (b - bv);
}

__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// acc += a b (the lo lo product, below 2^-46 of the product, is dropped; acc
// is left unnormalised: hi the FP32 running sum, lo its collected errors).
__device__ __forceinline__ void ff_fma(FF &acc, FF a, FF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    float s, t;
    two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo = acc.lo + (t + e);
}

__device__ __forceinline__ FF ff_norm(FF a) {
    FF r;
    two_sum(a.hi, a.lo, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    float s, t;
    two_sum(a.hi, b.hi, s, t);
    return ff_norm(FF{s, t + (a.lo + b.lo)});
}

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    FF acc{0.f, 0.f};
    ff_fma(acc, a, b);
    return ff_norm(acc);
}

// A colour vector: re/im of colours 0..2 as v[2a], v[2a + 1].
struct FVec {
    FF v[6];
};

__device__ __forceinline__ FVec split_vec(const double *base, size_t vh, int i, const FfSplit &sp) {
    const Vec3<double> d = load_vec(base, vh, i);
    FVec r;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r.v[2 * a] = split_d(d.c[a].re, sp);
        r.v[2 * a + 1] = split_d(d.c[a].im, sp);
    }
    return r;
}

// Float-pair half field: colour a is a float4 plane (re.hi, re.lo, im.hi,
// im.lo) at offset a * vh.
__device__ __forceinline__ FVec load_ff(const float4 *base, size_t vh, int i) {
    FVec r;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float4 t = __ldg(base + a * vh + i);
        r.v[2 * a] = FF{t.x, t.y};
        r.v[2 * a + 1] = FF{t.z, t.w};
    }
    return r;
}

__device__ __forceinline__ void store_ff(float4 *base, size_t vh, int i, const FVec &f) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
        base[a * vh + i] = make_float4(f.v[2 * a].hi, f.v[2 * a].lo, f.v[2 * a + 1].hi, f.v[2 * a + 1].lo);
}

__device__ __forceinline__ FVec flip(const FVec &f, bool neg) {
    FVec r;
#pragma unroll
    for (int c = 0; c < 6; ++c) r.v[c] = neg ? ff_neg(f.v[c]) : f.v[c];
    return r;
}

// acc += U v (dag: U^+ v) for the FP64 link U, split entry by entry.
template <bool DAG>
__device__ __forceinline__ void ff_mv(FVec &acc, const Mat3<double> &u, const FVec &v, const FfSplit &sp) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int e = DAG ? 3 * b + a : 3 * a + b;
            const FF ur = split_d(u.e[e].re, sp), ui = split_d(u.e[e].im, sp);
            const FF vr = v.v[2 * b], vi = v.v[2 * b + 1];
            ff_fma(acc.v[2 * a], ur, vr);
            ff_fma(acc.v[2 * a + 1], ur, vi);
            if (DAG) {  // conj(u) v
                ff_fma(acc.v[2 * a], ui, vi);
                ff_fma(acc.v[2 * a + 1], ff_neg(ui), vr);
            } else {
                ff_fma(acc.v[2 * a], ff_neg(ui), vi);
                ff_fma(acc.v[2 * a + 1], ui, vr);
            }
        }
    }
}

struct FfParams {
    Geom g;
    const double *fat, *lng;
    FF c3, m2;
    const double *x;  // stage 1: at the neighbours; stage 2: q = x at the site
    const double *b;  // stage 2
    float4 *tmp;      // stage 1 output, stage 2 input
    float *r32;       // stage 2 output
    CgScalars *S;
    double *partials;
    unsigned int *counter;
    int cg, force;
};

// (D in)(x) at the i-th site of parity p, with the same terms, signs and
// links as the FP64 kernel (qex_dslash_site.cuh); the Naik terms are summed
// apart and multiplied by c3 once.
template <bool NAIK, typename In>
__device__ __forceinline__ FVec ff_site(const FfParams &P, int p, int i, const Site &s, const In &in) {
    const Geom &g = P.g;
    const size_t vh = (size_t)g.vh;
    const FfSplit lsp = ff_split_bounds(0);
    FVec acc, acc3;
#pragma unroll
    for (int c = 0; c < 6; ++c) acc.v[c] = acc3.v[c] = FF{0.f, 0.f};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const bool eta_neg = eta_bit(s, mu) != 0;
        {
            const int j = hop_index(g, s, mu, 1);
            const bool neg = eta_neg != (bc_bit_fwd(g, s, mu, 1) != 0);
            ff_mv<false>(acc, load_link(P.fat, vh, p, mu, i), flip(in(j), neg), lsp);
        }
        {
            const int j = hop_index(g, s, mu, -1);
            const bool neg = eta_neg == (bc_bit_bwd(g, s, mu, 1) != 0);
            ff_mv<true>(acc, load_link(P.fat, vh, 1 - p, mu, j), flip(in(j), neg), lsp);
        }
        if (NAIK) {
            {
                const int j = hop_index(g, s, mu, 3);
                const bool neg = eta_neg != (bc_bit_fwd(g, s, mu, 3) != 0);
                ff_mv<false>(acc3, load_link(P.lng, vh, p, mu, i), flip(in(j), neg), lsp);
            }
            {
                const int j = hop_index(g, s, mu, -3);
                const bool neg = eta_neg == (bc_bit_bwd(g, s, mu, 3) != 0);
                ff_mv<true>(acc3, load_link(P.lng, vh, 1 - p, mu, j), flip(in(j), neg), lsp);
            }
        }
    }
    if (NAIK) {
#pragma unroll
        for (int c = 0; c < 6; ++c) ff_fma(acc.v[c], P.c3, ff_norm(acc3.v[c]));
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) acc.v[c] = ff_norm(acc.v[c]);
    return acc;
}

// Stage 1: tmp = D_oe x (odd sites).  Stage 2: r = b - m^2 x + D_eo tmp on
// the even sites, r32 = r rounded to FP32, ||r32||^2 -> the CG scalars.
template <bool NAIK, int STAGE>
__global__ void __launch_bounds__(kFfBlock, FfMinBlocks<NAIK>::value) ru_ff_kernel(const FfParams P) {
    __shared__ double smem[32];
    __shared__ unsigned int is_last;
    pdl_trigger();
    pdl_wait();  // x64, tmp and S->ru_ff come from the kernels before (launched with programmatic dependence
                 // in the host-driven loops)
    CgScalars *S = P.S;
    if (!P.force && !S->ru_ff) return;  // uniform: an FP64 update
    const Geom &g = P.g;
    const size_t vh = (size_t)g.vh;
    const int k = S->ff_k;
    const FfSplit vsp = ff_split_bounds(k);
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.vh; i += gridDim.x * blockDim.x) {
        if constexpr (STAGE == 1) {
            const Site s = site_of(g, 1, i);
            const FVec d = ff_site<NAIK>(P, 1, i, s, [&](int j) { return split_vec(P.x, vh, j, vsp); });
            store_ff(P.tmp, vh, i, d);
        } else {
            const Site s = site_of(g, 0, i);
            const FVec d = ff_site<NAIK>(P, 0, i, s, [&](int j) { return load_ff(P.tmp, vh, j); });
            const FVec q = split_vec(P.x, vh, i, vsp), bv = split_vec(P.b, vh, i, vsp);
            const float unscale = __uint_as_float((uint32_t)(127 - k) << 23);  // 2^-k
            Vec3<float> r;
            float n2 = 0.f;  // of the scaled residual (about unit size a real): no FP32 overflow
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const FF o = ff_add(ff_add(bv.v[c], ff_neg(ff_mul(P.m2, q.v[c]))), d.v[c]);
                const float rs = o.hi + o.lo;
                if (c & 1)
                    r.c[c >> 1].im = rs * unscale;
                else
                    r.c[c >> 1].re = rs * unscale;
                n2 = fmaf(rs, rs, n2);
            }
            store_vec(P.r32, vh, i, r);
            part += (double)n2;
        }
    }
    if constexpr (STAGE == 2) {
        const double bs = block_sum(part, smem);
        if (threadIdx.x == 0) {
            P.partials[blockIdx.x] = bs;
            __threadfence();
            const unsigned int t = atomicAdd(P.counter, 1u);
            is_last = (t == gridDim.x - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        const double tot = ldexp(block_sum_partials(P.partials, gridDim.x, smem), -2 * k);
        if (threadIdx.x != 0) return;
        *P.counter = 0u;
        if (P.cg)
            take_true_residual(S, tot, false);
        else
            S->true_rr = tot;
    }
}

static FF ff_of(double d) {
    FF r;
    r.hi = (float)d;
    r.lo = (float)(d - (double)r.hi);
    return r;
}

template <bool NAIK, int STAGE>
static void launch_ff(qex_lattice *lat, const FfParams &P, cudaStream_t st) {
    int grid = blocks_for(lat->vh, kFfBlock);
    if (STAGE == 2) {  // persistent: each block pays the reduction's tail once
        static int n = 0;
        if (n == 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ru_ff_kernel<NAIK, STAGE>, kFfBlock, 0) !=
                          cudaSuccess)
            n = FfMinBlocks<NAIK>::value;
        if (n < 1) n = 1;
        const int persistent = sm_count() * (n < 16 ? n : 16);
        if (persistent < grid) grid = persistent;
    }
    launch_k(ru_ff_kernel<NAIK, STAGE>, dim3(grid), dim3(kFfBlock), 0, st, lat->pdl != 0, P);
}

qex_status launch_ru_ff(qex_lattice *lat, int stage, const double *fat64, const double *lng64, double c3,
                        double m2, const double *x64, const double *b64, void *tmp, float *r32, CgScalars *S,
                        bool cg, bool force, cudaStream_t st) {
    qex_status s = ensure_scratch(lat);
    if (s) return s;
    FfParams P;
    P.g = lat->geom;
    P.fat = fat64;
    P.lng = lng64;
    P.c3 = ff_of(c3);
    P.m2 = ff_of(m2);
    P.x = x64;
    P.b = b64;
    P.tmp = (float4 *)tmp;
    P.r32 = r32;
    P.S = S;
    P.partials = lat->partials;
    P.counter = lat->counter;
    P.cg = cg ? 1 : 0;
    P.force = force ? 1 : 0;
    const bool naik = lng64 != nullptr;
    if (stage == 1) {
        if (naik)
            launch_ff<true, 1>(lat, P, st);
        else
            launch_ff<false, 1>(lat, P, st);
    } else {
        if (naik)
            launch_ff<true, 2>(lat, P, st);
        else
            launch_ff<false, 2>(lat, P, st);
    }
    QEX_CHECK_LAUNCH("ru_ff_kernel");
    return QEX_OK;
}

}  // namespace qex
