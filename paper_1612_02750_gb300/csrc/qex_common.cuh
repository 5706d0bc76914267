// qex_common.cuh -- shared device/host helpers of libqex_gpu: lattice
// geometry (even-odd indexing, neighbours, staggered phases, boundary signs),
// internal field/link layouts, complex colour algebra, deterministic block
// reductions and the error plumbing of the C ABI.
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/qex_gpu.h"

#define QEX_HD __host__ __device__ __forceinline__

namespace qex {

// ----------------------------------------------------------------- errors

void set_error(const char *fmt, ...);
qex_status cuda_fail(cudaError_t e, const char *what);

#define QEX_CUDA(call)                                              \
    do {                                                            \
        cudaError_t _e = (call);                                    \
        if (_e != cudaSuccess) return ::qex::cuda_fail(_e, #call);  \
    } while (0)

void note_launch();

#define QEX_CHECK_LAUNCH(what)                                      \
    do {                                                            \
        cudaError_t _e = cudaGetLastError();                        \
        if (_e != cudaSuccess) return ::qex::cuda_fail(_e, what);   \
        ::qex::note_launch();                                       \
    } while (0)

// ------------------------------------------------------- fast division
// Division by a run-time invariant divisor d in [1, 2^31) through a
// multiply-high, exact for every 32-bit dividend (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Fig. 4.1).
struct FastDiv {
    uint32_t d, m;
    uint32_t s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;  // l = ceil(log2 d)
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

QEX_HD uint32_t fd_div(const FastDiv &f, uint32_t n) {
#ifdef __CUDA_ARCH__
    uint32_t t1 = __umulhi(f.m, n);
#else
    uint32_t t1 = (uint32_t)(((uint64_t)f.m * n) >> 32);
#endif
    return (t1 + ((n - t1) >> f.s1)) >> f.s2;
}

// ------------------------------------------------------------ geometry
// Site lex = x + Lx*(y + Ly*(z + Lz*t)).  Lx is even, so the sites of one
// parity are exactly the lex values {2i, 2i+1} with one member chosen by
// parity; i = lex >> 1 is their rank within the parity (the even-odd index).
struct Geom {
    int L[4];        // extents x, y, z, t
    int stride[4];   // lex strides 1, Lx, Lx*Ly, Lx*Ly*Lz
    int vh;          // V / 2
    int antiperiodic;
    FastDiv div_xh;  // Lx / 2
    FastDiv div_y;   // Ly
    FastDiv div_z;   // Lz
};

struct Site {
    int c[4];   // coordinates x, y, z, t
    int lex;
};

// Coordinates of the i-th site of parity p.
QEX_HD Site site_of(const Geom &g, int p, int i) {
    uint32_t r1 = fd_div(g.div_xh, (uint32_t)i);
    int xh = i - (int)r1 * (g.L[0] >> 1);
    uint32_t r2 = fd_div(g.div_y, r1);
    int y = (int)r1 - (int)r2 * g.L[1];
    uint32_t t = fd_div(g.div_z, r2);
    int z = (int)r2 - (int)t * g.L[2];
    int bit = (p + y + z + (int)t) & 1;
    Site s;
    s.c[0] = 2 * xh + bit;
    s.c[1] = y;
    s.c[2] = z;
    s.c[3] = (int)t;
    s.lex = 2 * i + bit;
    return s;
}

// Even-odd index (within the neighbour's parity) of site + k*mu_hat,
// 0 < |k| < L[mu] (a single periodic wrap).
QEX_HD int hop_index(const Geom &g, const Site &s, int mu, int k) {
    int c = s.c[mu] + k;
    int lex = s.lex + k * g.stride[mu];
    if (c >= g.L[mu]) lex -= g.L[mu] * g.stride[mu];
    if (c < 0) lex += g.L[mu] * g.stride[mu];
    return lex >> 1;
}

// Staggered phase eta_mu(x) as a 0/1 sign bit: (-1)^(x_0 + ... + x_{mu-1}).
QEX_HD int eta_bit(const Site &s, int mu) {
    int e = 0;
    for (int nu = 0; nu < mu; ++nu) e += s.c[nu];
    return e & 1;
}

// Antiperiodic-time sign bit of the k-step link leaving the site along +mu:
// set when mu = t and the hop crosses t = Lt-1 -> 0 (k < Lt, one crossing).
QEX_HD int bc_bit_fwd(const Geom &g, const Site &s, int mu, int k) {
    return (mu == 3 && g.antiperiodic && s.c[3] + k >= g.L[3]) ? 1 : 0;
}
// Sign bit of the k-step link arriving at the site from site - k*mu_hat.
QEX_HD int bc_bit_bwd(const Geom &g, const Site &s, int mu, int k) {
    return (mu == 3 && g.antiperiodic && s.c[3] - k < 0) ? 1 : 0;
}

Geom make_geom(const int dims[4], int antiperiodic);

// --------------------------------------------------------- layouts
// Internal link set: block (p, mu) holds the Vh links U_mu(x) of the sites x
// of parity p, as planes over sites.
//   F64: 9 planes of double2 (element c = 3a + b); block size 9*Vh double2.
//   F32: 4 planes of float4 (elements {0,1},{2,3},{4,5},{6,7}) then 1 plane
//        of float2 (element 8); block size 18*Vh floats.
// Half field (Vh sites of one parity):
//   F64: 3 planes of double2 (colour a);  F32: float4 plane (colours 0, 1)
//   then float2 plane (colour 2).
template <typename R> struct Cplx { R re, im; };

template <typename R> struct Vec3 { Cplx<R> c[3]; };
template <typename R> struct Mat3 { Cplx<R> e[9]; };

// Read-only loads of link data, which no other thread of a Dslash launch
// reads again: they do not allocate L1 lines (ld.global.nc.L1::no_allocate),
// which then stay with the neighbour vectors (read by up to eight sites each).
// 32^4 mixed solve: 21.65-21.76 -> 21.11 ms.  QEX_LINK_L1_NOALLOC=0 restores
// the plain read-only path.
#ifndef QEX_LINK_L1_NOALLOC
#define QEX_LINK_L1_NOALLOC 1
#endif
__device__ __forceinline__ uint4 ldg_link(const uint4 *p) {
#if QEX_LINK_L1_NOALLOC
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
#else
    return __ldg(p);
#endif
}
__device__ __forceinline__ uint2 ldg_link(const uint2 *p) {
#if QEX_LINK_L1_NOALLOC
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
#else
    return __ldg(p);
#endif
}
__device__ __forceinline__ float4 ldg_link(const float4 *p) {
    const uint4 v = ldg_link(reinterpret_cast<const uint4 *>(p));
    return make_float4(__uint_as_float(v.x), __uint_as_float(v.y), __uint_as_float(v.z), __uint_as_float(v.w));
}
__device__ __forceinline__ float2 ldg_link(const float2 *p) {
    const uint2 v = ldg_link(reinterpret_cast<const uint2 *>(p));
    return make_float2(__uint_as_float(v.x), __uint_as_float(v.y));
}
__device__ __forceinline__ double2 ldg_link(const double2 *p) {
    const uint4 v = ldg_link(reinterpret_cast<const uint4 *>(p));
    return make_double2(__hiloint2double((int)v.y, (int)v.x), __hiloint2double((int)v.w, (int)v.z));
}

__device__ __forceinline__ Mat3<double> load_link(const double *base, size_t vh, int p, int mu, int i) {
    const double2 *b = reinterpret_cast<const double2 *>(base) + (size_t)(p * 4 + mu) * 9 * vh + i;
    Mat3<double> m;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        double2 v = ldg_link(b + c * vh);
        m.e[c].re = v.x;
        m.e[c].im = v.y;
    }
    return m;
}

__device__ __forceinline__ Mat3<float> load_link(const float *base, size_t vh, int p, int mu, int i) {
    const float *blk = base + (size_t)(p * 4 + mu) * 18 * vh;
    const float4 *b4 = reinterpret_cast<const float4 *>(blk) + i;
    Mat3<float> m;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float4 v = ldg_link(b4 + q * vh);
        m.e[2 * q].re = v.x;
        m.e[2 * q].im = v.y;
        m.e[2 * q + 1].re = v.z;
        m.e[2 * q + 1].im = v.w;
    }
    float2 v = ldg_link(reinterpret_cast<const float2 *>(blk + 16 * vh) + i);
    m.e[8].re = v.x;
    m.e[8].im = v.y;
    return m;
}

// Third row of an SU(3) matrix from its first two: row2 = conj(row0 x row1).
template <typename R>
__host__ __device__ __forceinline__ void reconstruct_row2(Mat3<R> &m) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int k = (j + 1) % 3, l = (j + 2) % 3;
        const Cplx<R> a = m.e[k], b = m.e[3 + l], c = m.e[l], d = m.e[3 + k];
        R re = a.re * b.re - a.im * b.im;
        R im = a.re * b.im + a.im * b.re;
        re -= c.re * d.re - c.im * d.im;
        im -= c.re * d.im + c.im * d.re;
        m.e[6 + j].re = re;
        m.e[6 + j].im = -im;
    }
}

// Two-row FP32 link: block (p, mu) holds 3 float4 planes {e0,e1}, {e2,e3},
// {e4,e5}; block size 12*Vh floats.
__device__ __forceinline__ Mat3<float> load_link_r12(const float *base, size_t vh, int p, int mu, int i) {
    const float4 *b4 = reinterpret_cast<const float4 *>(base + (size_t)(p * 4 + mu) * 12 * vh) + i;
    Mat3<float> m;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float4 v = ldg_link(b4 + q * vh);
        m.e[2 * q].re = v.x;
        m.e[2 * q].im = v.y;
        m.e[2 * q + 1].re = v.z;
        m.e[2 * q + 1].im = v.w;
    }
    reconstruct_row2(m);
    return m;
}

// Two-row links in 16-bit fixed point: block (p, mu) holds a plane of 16-byte
// words (re/im of elements 0..3) then a plane of 8-byte words (elements 4,
// 5); block size 24*Vh bytes.  Each 32-bit word holds re in its low and im in
// its high 16 bits as offset binary, u = q + 32768 with q = round(32767 v).
//
// The kernels decode the integer q, not q/32767: the 16 bits placed under the
// exponent of 2^23 (one LOP3 or PRMT) give the float 2^23 + u exactly, and
// subtracting 2^23 + 2^15 leaves q exactly.  The matrix they hold is then
// 32767 U in rows 0, 1 and, rebuilt from those, 32767^2 U in row 2; the
// scale comes back once per output row in the sign factor of the hop
// (acc_mv_fix16, acc_mdv_fix16).
constexpr float kFix16Inv = 1.0f / 32767.0f;
constexpr float kFix16Inv2 = (float)(1.0 / (32767.0 * 32767.0));

__device__ __forceinline__ float fix16_lo(uint32_t w) {
    return __uint_as_float((w & 0xFFFFu) | 0x4B000000u) - 8421376.0f;
}
__device__ __forceinline__ float fix16_hi(uint32_t w) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7632)) - 8421376.0f;
}

// 32767 x (rows 0, 1) and 32767^2 x (row 2) of the stored link.
__device__ __forceinline__ Mat3<float> load_link_fix16(const float *base_f, size_t vh, int p, int mu, int i) {
    const char *blk = reinterpret_cast<const char *>(base_f) + (size_t)(p * 4 + mu) * 24 * vh;
    const uint4 a = ldg_link(reinterpret_cast<const uint4 *>(blk) + i);
    const uint2 b = ldg_link(reinterpret_cast<const uint2 *>(blk + 16 * vh) + i);
    const uint32_t w[6] = {a.x, a.y, a.z, a.w, b.x, b.y};
    Mat3<float> m;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        m.e[c].re = fix16_lo(w[c]);
        m.e[c].im = fix16_hi(w[c]);
    }
    reconstruct_row2(m);
    return m;
}

// Full 3x3 links in 16-bit fixed point with a per-link step (for links that
// are not unitary, e.g. the Naik long links): block (p, mu) holds two planes
// of 16-byte words (elements 0..3 and 4..7, one offset-binary re/im word per
// element as above) and a plane of 8-byte words (element 8, then the FP32
// step d); block size 40*Vh bytes.  Value = q * d.  Returns the integers q in
// m and the step in *d (the caller folds d into the hop's sign factor).
__device__ __forceinline__ Mat3<float> load_link_s16(const float *base_f, size_t vh, int p, int mu, int i, float *d) {
    const char *blk = reinterpret_cast<const char *>(base_f) + (size_t)(p * 4 + mu) * 40 * vh;
    const uint4 a = ldg_link(reinterpret_cast<const uint4 *>(blk) + i);
    const uint4 b = ldg_link(reinterpret_cast<const uint4 *>(blk + 16 * vh) + i);
    const uint2 c = ldg_link(reinterpret_cast<const uint2 *>(blk + 32 * vh) + i);
    const uint32_t w[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x};
    Mat3<float> m;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        m.e[k].re = fix16_lo(w[k]);
        m.e[k].im = fix16_hi(w[k]);
    }
    *d = __uint_as_float(c.y);
    return m;
}

__device__ __forceinline__ Vec3<double> load_vec(const double *base, size_t vh, int i) {
    const double2 *b = reinterpret_cast<const double2 *>(base) + i;
    Vec3<double> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double2 t = __ldg(b + a * vh);
        v.c[a].re = t.x;
        v.c[a].im = t.y;
    }
    return v;
}

__device__ __forceinline__ Vec3<float> load_vec(const float *base, size_t vh, int i) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(base) + i);
    float2 u = __ldg(reinterpret_cast<const float2 *>(base + 4 * vh) + i);
    Vec3<float> v;
    v.c[0].re = t.x;
    v.c[0].im = t.y;
    v.c[1].re = t.z;
    v.c[1].im = t.w;
    v.c[2].re = u.x;
    v.c[2].im = u.y;
    return v;
}

__device__ __forceinline__ void store_vec(double *base, size_t vh, int i, const Vec3<double> &v) {
    double2 *b = reinterpret_cast<double2 *>(base) + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) b[a * vh] = make_double2(v.c[a].re, v.c[a].im);
}

__device__ __forceinline__ void store_vec(float *base, size_t vh, int i, const Vec3<float> &v) {
    reinterpret_cast<float4 *>(base)[i] = make_float4(v.c[0].re, v.c[0].im, v.c[1].re, v.c[1].im);
    reinterpret_cast<float2 *>(base + 4 * vh)[i] = make_float2(v.c[2].re, v.c[2].im);
}

// ----------------------------------------------------- colour algebra
// acc += sgn * (M v), sgn = +1 or -1.
template <typename R>
__device__ __forceinline__ void acc_mv(Vec3<R> &acc, R sgn, const Mat3<R> &m, const Vec3<R> &v) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R re = m.e[3 * a].re * v.c[0].re;
        R im = m.e[3 * a].re * v.c[0].im;
        re = fma(-m.e[3 * a].im, v.c[0].im, re);
        im = fma(m.e[3 * a].im, v.c[0].re, im);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            re = fma(m.e[3 * a + b].re, v.c[b].re, re);
            re = fma(-m.e[3 * a + b].im, v.c[b].im, re);
            im = fma(m.e[3 * a + b].re, v.c[b].im, im);
            im = fma(m.e[3 * a + b].im, v.c[b].re, im);
        }
        acc.c[a].re = fma(sgn, re, acc.c[a].re);
        acc.c[a].im = fma(sgn, im, acc.c[a].im);
    }
}

// FP64 hops whose factor is +1 or -1 (the one-hop term): the sign goes into
// the input vector as an XOR of its sign bits (integer pipe) and the mat-vec
// accumulates straight into acc, 36 FP64 FMAs per hop instead of 42.
__device__ __forceinline__ Vec3<double> flip_sign(const Vec3<double> &v, bool neg) {
    const unsigned long long m = neg ? 0x8000000000000000ull : 0ull;
    Vec3<double> w;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        w.c[a].re = __longlong_as_double(__double_as_longlong(v.c[a].re) ^ m);
        w.c[a].im = __longlong_as_double(__double_as_longlong(v.c[a].im) ^ m);
    }
    return w;
}

// acc += (neg ? -1 : 1) * (M v)
__device__ __forceinline__ void acc_mv_unit(Vec3<double> &acc, bool neg, const Mat3<double> &m, const Vec3<double> &v) {
    const Vec3<double> w = flip_sign(v, neg);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            acc.c[a].re = fma(m.e[3 * a + b].re, w.c[b].re, acc.c[a].re);
            acc.c[a].re = fma(-m.e[3 * a + b].im, w.c[b].im, acc.c[a].re);
            acc.c[a].im = fma(m.e[3 * a + b].re, w.c[b].im, acc.c[a].im);
            acc.c[a].im = fma(m.e[3 * a + b].im, w.c[b].re, acc.c[a].im);
        }
    }
}

// acc += (neg ? -1 : 1) * (M^+ v)
__device__ __forceinline__ void acc_mdv_unit(Vec3<double> &acc, bool neg, const Mat3<double> &m,
                                             const Vec3<double> &v) {
    const Vec3<double> w = flip_sign(v, neg);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            acc.c[a].re = fma(m.e[3 * b + a].re, w.c[b].re, acc.c[a].re);
            acc.c[a].re = fma(m.e[3 * b + a].im, w.c[b].im, acc.c[a].re);
            acc.c[a].im = fma(m.e[3 * b + a].re, w.c[b].im, acc.c[a].im);
            acc.c[a].im = fma(-m.e[3 * b + a].im, w.c[b].re, acc.c[a].im);
        }
    }
}

// acc += sgn * (U v) for U held as load_link_fix16 returns it.
__device__ __forceinline__ void acc_mv_fix16(Vec3<float> &acc, float sgn, const Mat3<float> &m, const Vec3<float> &v) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float re = m.e[3 * a].re * v.c[0].re;
        float im = m.e[3 * a].re * v.c[0].im;
        re = fmaf(-m.e[3 * a].im, v.c[0].im, re);
        im = fmaf(m.e[3 * a].im, v.c[0].re, im);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            re = fmaf(m.e[3 * a + b].re, v.c[b].re, re);
            re = fmaf(-m.e[3 * a + b].im, v.c[b].im, re);
            im = fmaf(m.e[3 * a + b].re, v.c[b].im, im);
            im = fmaf(m.e[3 * a + b].im, v.c[b].re, im);
        }
        const float s = sgn * (a < 2 ? kFix16Inv : kFix16Inv2);
        acc.c[a].re = fmaf(s, re, acc.c[a].re);
        acc.c[a].im = fmaf(s, im, acc.c[a].im);
    }
}

// acc += sgn * (U^+ v) for U held as load_link_fix16 returns it: column a of
// U^+ mixes rows 0, 1 (scale 32767) with row 2 (scale 32767^2), so v_2 takes
// one factor 1/32767 first and the row sign the other.
__device__ __forceinline__ void acc_mdv_fix16(Vec3<float> &acc, float sgn, const Mat3<float> &m, const Vec3<float> &v) {
    Vec3<float> w = v;
    w.c[2].re *= kFix16Inv;
    w.c[2].im *= kFix16Inv;
    const float s = sgn * kFix16Inv;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float re = m.e[a].re * w.c[0].re;
        float im = m.e[a].re * w.c[0].im;
        re = fmaf(m.e[a].im, w.c[0].im, re);
        im = fmaf(-m.e[a].im, w.c[0].re, im);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            re = fmaf(m.e[3 * b + a].re, w.c[b].re, re);
            re = fmaf(m.e[3 * b + a].im, w.c[b].im, re);
            im = fmaf(m.e[3 * b + a].re, w.c[b].im, im);
            im = fmaf(-m.e[3 * b + a].im, w.c[b].re, im);
        }
        acc.c[a].re = fmaf(s, re, acc.c[a].re);
        acc.c[a].im = fmaf(s, im, acc.c[a].im);
    }
}

// acc += sgn * (M^+ v).
template <typename R>
__device__ __forceinline__ void acc_mdv(Vec3<R> &acc, R sgn, const Mat3<R> &m, const Vec3<R> &v) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R re = m.e[a].re * v.c[0].re;
        R im = m.e[a].re * v.c[0].im;
        re = fma(m.e[a].im, v.c[0].im, re);
        im = fma(-m.e[a].im, v.c[0].re, im);
#pragma unroll
        for (int b = 1; b < 3; ++b) {
            re = fma(m.e[3 * b + a].re, v.c[b].re, re);
            re = fma(m.e[3 * b + a].im, v.c[b].im, re);
            im = fma(m.e[3 * b + a].re, v.c[b].im, im);
            im = fma(-m.e[3 * b + a].im, v.c[b].re, im);
        }
        acc.c[a].re = fma(sgn, re, acc.c[a].re);
        acc.c[a].im = fma(sgn, im, acc.c[a].im);
    }
}

// --------------------------------------------------- block reductions
// Deterministic: a fixed shuffle tree within each warp, then warp 0 reduces
// the per-warp values in index order.  Requires blockDim.x % 32 == 0, <= 1024.
__device__ __forceinline__ double block_sum(double v, double *smem /* >= 32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[w] = v;
    __syncthreads();
    double s = 0;
    if (w == 0) {
        int nw = blockDim.x >> 5;
        s = lane < nw ? smem[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

// Sum of partial[0..n) by one block in a fixed order (valid in thread 0).
// Reads bypass L1 (the partials were written by other blocks).
__device__ __forceinline__ double block_sum_partials(const double *partial, int n, double *smem) {
    double s = 0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += __ldcg(partial + k);
    return block_sum(s, smem);
}

// ------------------------------------------- programmatic dependent launch
// A kernel launched with the programmatic-serialization attribute may start
// while its predecessor in the stream is still finishing: each kernel of the
// CG path lets the next one launch at once (pdl_trigger) and waits for its
// predecessors' completion and memory (pdl_wait) before it reads anything;
// for an ordinary launch both return at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl,
                     Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ------------------------------------------------------- lattice object
struct CgScalars;

// Launch shapes of one (precision, Naik) of a lattice, chosen by the
// autotuner (tune.cu); zeros mean the compiled defaults.
struct LaunchShape {
    int ds_block;    // threads per block of the non-reducing Dslash variants
    int red_block;   // threads per block of the reducing variants (0: defaults for both fields)
    int red_per_sm;  // their persistent grid, blocks per SM (0: one thread per site)
    int ds_waves;    // non-reducing grid capped at this many resident waves, sites
                     // taken grid-stride (0: one thread per site)
};

}  // namespace qex

struct qex_lattice {
    int dims[4];
    int antiperiodic;
    int64_t volume;
    int64_t vh;
    qex::Geom geom;
    int device;
    // scratch owned by the library
    double *partials;          // per-block partial sums (max over kernels)
    int partials_len;
    unsigned int *counter;     // last-block counters (zero between calls)
    double *red_out;           // small result area for reductions
    qex::CgScalars *scalars;   // CG state (device)
    qex::CgScalars *scalars_host;   // pinned mirror, readback slot 0
    qex::CgScalars *scalars_host2;  // pinned readback slot 1
    void *work;                // CG work vectors
    size_t work_bytes;
    void *host_work;           // staging of qex_cg_host
    size_t host_work_bytes;
    cudaStream_t copy_stream;  // qex_cg_host: host-to-device copies of the link slabs
    cudaEvent_t slab_ev[9];    // ... one event per slab, and one ordering event
    void *cg_graph;            // cached CUDA graph of the last CG solve
    void *batch_ctx;           // scratch of qex_cg_batch calls led by this lattice
    cudaEvent_t ev0, ev1;
    // autotuner state (tune.cu): per precision and Naik, and the BLAS grid
    qex::LaunchShape shape[5][2];  // [qex_prec][Naik]
    int tuned[5][2];           // 0 no, 1 measured, 2 from the cache, 3 defaults (QEX_TUNE=0)
    int blas_per_sm;           // 0: QEX_BLAS_BLOCKS_PER_SM
    int pdl;                   // CG kernels launch with programmatic dependent launch (set by qex_cg)
    int fused_blocks;          // grid of the last fused CG launch
    int batch_pin[2];          // qex_cg_batch_tune_set: blocks per SM, groups per item (0: not pinned)
    int batch_shape[3];        // shape of the last batch led by this lattice: blocks per SM, groups per item, source
};

namespace qex {

qex_status ensure_scratch(qex_lattice *lat);
qex_status ensure_work(qex_lattice *lat, size_t bytes);
// Tune (prec, Naik iff lng) of the lattice once, from the process cache or by
// measurement on the stream (skipped while the stream is capturing).
// tune_blas: also choose the BLAS grid from prec's vector-update kernel.
qex_status ensure_tuned(qex_lattice *lat, qex_prec prec, const void *fat, const void *lng, cudaStream_t st,
                        bool tune_blas);
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }
inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
qex_status check_lattice(const qex_lattice *lat);
qex_status check_prec(qex_prec prec);
inline bool is_f64(qex_prec p) { return p == QEX_F64; }

constexpr int kBlock = 256;  // threads per block of the site kernels
constexpr int kHostSlabs = 8;  // t-slabs of a link set in qex_cg_host (lattice::slab_ev holds one more)

// Dslash launch shape: threads per block and the minimum resident blocks per
// SM handed to __launch_bounds__ (which caps registers per thread).
#ifndef QEX_DSLASH_BLOCK
#define QEX_DSLASH_BLOCK 256
#endif
#ifndef QEX_DSLASH_MIN_BLOCKS
#define QEX_DSLASH_MIN_BLOCKS 4
#endif
#ifndef QEX_DSLASH_MIN_BLOCKS_F64
#define QEX_DSLASH_MIN_BLOCKS_F64 3
#endif
// Grid of the reducing Dslash variants: resident blocks per SM of their
// persistent grid (-1: the launch-bounds minimum; 0: one thread per site).
#ifndef QEX_REDUCE_BLOCKS_PER_SM
#define QEX_REDUCE_BLOCKS_PER_SM -1
#endif
// Cap of the streaming BLAS kernels' grid, in blocks per SM (0: no cap).
#ifndef QEX_BLAS_BLOCKS_PER_SM
#define QEX_BLAS_BLOCKS_PER_SM 4
#endif
constexpr int kDslashBlock = QEX_DSLASH_BLOCK;
constexpr int kDslashMinBlocks = QEX_DSLASH_MIN_BLOCKS;         // FP32 variants
constexpr int kDslashMinBlocksF64 = QEX_DSLASH_MIN_BLOCKS_F64;  // FP64 variants (ALU bound, no spills)
template <typename R> struct DslashMinBlocks { static constexpr int value = kDslashMinBlocks; };
template <> struct DslashMinBlocks<double> { static constexpr int value = kDslashMinBlocksF64; };

inline int blocks_for(int64_t n, int bs = kBlock) { return (int)((n + bs - 1) / bs); }

}  // namespace qex
