// pack.cu -- conversions between the canonical lexicographic layouts and the
// internal even-odd structure-of-arrays layouts, and FP64 <-> FP32 copies.
#include <type_traits>

#include "qex_kernels.cuh"

namespace qex {

// Write matrix m (18 reals, element c = 3a+b as re,im) into block (p,mu).
__device__ __forceinline__ void put_link(double *base, size_t vh, int blk, int i, const double *m) {
    double2 *b = reinterpret_cast<double2 *>(base) + (size_t)blk * 9 * vh + i;
#pragma unroll
    for (int c = 0; c < 9; ++c) b[c * vh] = make_double2(m[2 * c], m[2 * c + 1]);
}

__device__ __forceinline__ void put_link(float *base, size_t vh, int blk, int i, const double *m) {
    float *bb = base + (size_t)blk * 18 * vh;
    float4 *b4 = reinterpret_cast<float4 *>(bb) + i;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        b4[q * vh] = make_float4((float)m[4 * q], (float)m[4 * q + 1], (float)m[4 * q + 2], (float)m[4 * q + 3]);
    reinterpret_cast<float2 *>(bb + 16 * vh)[i] = make_float2((float)m[16], (float)m[17]);
}

__device__ __forceinline__ void get_link(const double *base, size_t vh, int blk, int i, double *m) {
    const double2 *b = reinterpret_cast<const double2 *>(base) + (size_t)blk * 9 * vh + i;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        double2 v = b[c * vh];
        m[2 * c] = v.x;
        m[2 * c + 1] = v.y;
    }
}

__device__ __forceinline__ void get_link(const float *base, size_t vh, int blk, int i, double *m) {
    const float *bb = base + (size_t)blk * 18 * vh;
    const float4 *b4 = reinterpret_cast<const float4 *>(bb) + i;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float4 v = b4[q * vh];
        m[4 * q] = v.x;
        m[4 * q + 1] = v.y;
        m[4 * q + 2] = v.z;
        m[4 * q + 3] = v.w;
    }
    float2 v = reinterpret_cast<const float2 *>(bb + 16 * vh)[i];
    m[16] = v.x;
    m[17] = v.y;
}

// Two-row FP32 links: rows 0 and 1 (elements 0..5) in 3 float4 planes.
struct R12 {
    float *p;
};
struct R12c {
    const float *p;
};

__device__ __forceinline__ void put_link(R12 base, size_t vh, int blk, int i, const double *m) {
    float4 *b4 = reinterpret_cast<float4 *>(base.p + (size_t)blk * 12 * vh) + i;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        b4[q * vh] = make_float4((float)m[4 * q], (float)m[4 * q + 1], (float)m[4 * q + 2], (float)m[4 * q + 3]);
}

// Reads the two stored rows and rebuilds the third in FP64.
__device__ __forceinline__ void get_link(R12c base, size_t vh, int blk, int i, double *m) {
    const float4 *b4 = reinterpret_cast<const float4 *>(base.p + (size_t)blk * 12 * vh) + i;
    Mat3<double> u;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float4 v = b4[q * vh];
        u.e[2 * q].re = v.x;
        u.e[2 * q].im = v.y;
        u.e[2 * q + 1].re = v.z;
        u.e[2 * q + 1].im = v.w;
    }
    reconstruct_row2(u);
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        m[2 * c] = u.e[c].re;
        m[2 * c + 1] = u.e[c].im;
    }
}

// Two-row links in 16-bit fixed point (q = round(v * 32767), v clamped to
// [-1, 1]), each re/im stored as the offset-binary u = q + 32768; elements
// 0..3 in a 16-byte word, 4..5 in an 8-byte word.
struct R12H {
    float *p;
};
struct R12Hc {
    const float *p;
};

// Rounding first and clamping the integer gives the same q as clamping v to
// [-1, 1] first (both are monotonic; the conversion saturates, and a NaN
// converts to INT_MIN, i.e. -32767 as with the clamp), with two FP64
// operations per real instead of four.
__device__ __forceinline__ int fix16_round(double x) {
    const int q = __double2int_rn(x);
    return q < -32767 ? -32767 : (q > 32767 ? 32767 : q);
}
__device__ __forceinline__ int fix16_q(double v) { return fix16_round(v * 32767.0); }

__device__ __forceinline__ uint32_t fix16_pair(double re, double im) {
    return (uint32_t)(fix16_q(re) + 32768) | ((uint32_t)(fix16_q(im) + 32768) << 16);
}

__device__ __forceinline__ double fix16_value(uint32_t w, bool hi) {
    const int q = (int)(hi ? (w >> 16) : (w & 0xFFFFu)) - 32768;
    return (double)q / 32767.0;
}

__device__ __forceinline__ void put_link(R12H base, size_t vh, int blk, int i, const double *m) {
    char *b = reinterpret_cast<char *>(base.p) + (size_t)blk * 24 * vh;
    reinterpret_cast<uint4 *>(b)[i] = make_uint4(fix16_pair(m[0], m[1]), fix16_pair(m[2], m[3]),
                                                 fix16_pair(m[4], m[5]), fix16_pair(m[6], m[7]));
    reinterpret_cast<uint2 *>(b + 16 * vh)[i] = make_uint2(fix16_pair(m[8], m[9]), fix16_pair(m[10], m[11]));
}

// Reads the two stored rows and rebuilds the third in FP64.
__device__ __forceinline__ void get_link(R12Hc base, size_t vh, int blk, int i, double *m) {
    const char *b = reinterpret_cast<const char *>(base.p) + (size_t)blk * 24 * vh;
    const uint4 a = reinterpret_cast<const uint4 *>(b)[i];
    const uint2 c = reinterpret_cast<const uint2 *>(b + 16 * vh)[i];
    const uint32_t w[6] = {a.x, a.y, a.z, a.w, c.x, c.y};
    Mat3<double> u;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        u.e[k].re = fix16_value(w[k], false);
        u.e[k].im = fix16_value(w[k], true);
    }
    reconstruct_row2(u);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        m[2 * k] = u.e[k].re;
        m[2 * k + 1] = u.e[k].im;
    }
}

// Full 3x3 links in 16-bit fixed point with a per-link FP32 step d: d is
// the largest |re| or |im| of the link over 32767, rounded up to FP32 (so
// every |v| / d <= 32767), and q = round(v * (1/d)) clamped to +-32767 (all
// zero for a zero link).  Elements 0..3 and 4..7 in two 16-byte words,
// element 8 and d in an 8-byte word.
struct S16 {
    float *p;
};
struct S16c {
    const float *p;
};

__device__ __forceinline__ void put_link(S16 base, size_t vh, int blk, int i, const double *m) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 18; ++k) s = fmax(s, fabs(m[k]));
    const float d = __double2float_ru(s / 32767.0);
    const double inv = d > 0.f ? 1.0 / (double)d : 0.0;
    uint32_t w[9];
#pragma unroll
    for (int k = 0; k < 9; ++k)
        w[k] = (uint32_t)(fix16_round(m[2 * k] * inv) + 32768) |
               ((uint32_t)(fix16_round(m[2 * k + 1] * inv) + 32768) << 16);
    char *b = reinterpret_cast<char *>(base.p) + (size_t)blk * 40 * vh;
    reinterpret_cast<uint4 *>(b)[i] = make_uint4(w[0], w[1], w[2], w[3]);
    reinterpret_cast<uint4 *>(b + 16 * vh)[i] = make_uint4(w[4], w[5], w[6], w[7]);
    reinterpret_cast<uint2 *>(b + 32 * vh)[i] = make_uint2(w[8], __float_as_uint(d));
}

__device__ __forceinline__ void get_link(S16c base, size_t vh, int blk, int i, double *m) {
    const char *b = reinterpret_cast<const char *>(base.p) + (size_t)blk * 40 * vh;
    const uint4 a = reinterpret_cast<const uint4 *>(b)[i];
    const uint4 c = reinterpret_cast<const uint4 *>(b + 16 * vh)[i];
    const uint2 e = reinterpret_cast<const uint2 *>(b + 32 * vh)[i];
    const uint32_t w[9] = {a.x, a.y, a.z, a.w, c.x, c.y, c.z, c.w, e.x};
    const double d = (double)__uint_as_float(e.y);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        m[2 * k] = (double)((int)(w[k] & 0xFFFFu) - 32768) * d;
        m[2 * k + 1] = (double)((int)(w[k] >> 16) - 32768) * d;
    }
}


__device__ __forceinline__ void put_vec(double *base, size_t vh, int i, const double *v) {
    double2 *b = reinterpret_cast<double2 *>(base) + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) b[a * vh] = make_double2(v[2 * a], v[2 * a + 1]);
}

__device__ __forceinline__ void put_vec(float *base, size_t vh, int i, const double *v) {
    reinterpret_cast<float4 *>(base)[i] = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
    reinterpret_cast<float2 *>(base + 4 * vh)[i] = make_float2((float)v[4], (float)v[5]);
}

__device__ __forceinline__ void get_vec(const double *base, size_t vh, int i, double *v) {
    const double2 *b = reinterpret_cast<const double2 *>(base) + i;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double2 t = b[a * vh];
        v[2 * a] = t.x;
        v[2 * a + 1] = t.y;
    }
}

__device__ __forceinline__ void get_vec(const float *base, size_t vh, int i, double *v) {
    float4 t = reinterpret_cast<const float4 *>(base)[i];
    float2 u = reinterpret_cast<const float2 *>(base + 4 * vh)[i];
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
    v[4] = u.x;
    v[5] = u.y;
}

// blockIdx.y = p*4 + mu; one thread per site of parity p.
template <typename R>
__global__ void pack_links_kernel(Geom g, const double *__restrict__ lex, R out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    int blk = blockIdx.y, p = blk >> 2, mu = blk & 3;
    Site s = site_of(g, p, i);
    const double *src = lex + ((size_t)s.lex * 4 + mu) * 18;
    double m[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) m[k] = src[k];
    put_link(out, g.vh, blk, i, m);
}

// The links of the internal indices [i0, i1) of both parities (a range of
// t-slices), written in FP64 and, unless R is void*, also in a second format:
// each canonical link is read once for both.
template <typename R>
__global__ void pack_links_range_kernel(Geom g, const double *__restrict__ lex, double *out64, R out2, int i0,
                                        int i1) {
    const int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= i1) return;
    const int blk = blockIdx.y, p = blk >> 2, mu = blk & 3;
    const Site s = site_of(g, p, i);
    const double *src = lex + ((size_t)s.lex * 4 + mu) * 18;
    double m[18];
#pragma unroll
    for (int k = 0; k < 18; ++k) m[k] = src[k];
    put_link(out64, g.vh, blk, i, m);
    if constexpr (!std::is_same<R, void *>::value) put_link(out2, g.vh, blk, i, m);
}

template <typename R>
__global__ void unpack_links_kernel(Geom g, R in, double *__restrict__ lex) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    int blk = blockIdx.y, p = blk >> 2, mu = blk & 3;
    Site s = site_of(g, p, i);
    double m[18];
    get_link(in, g.vh, blk, i, m);
    double *dst = lex + ((size_t)s.lex * 4 + mu) * 18;
#pragma unroll
    for (int k = 0; k < 18; ++k) dst[k] = m[k];
}

template <typename RI, typename RO>
__global__ void convert_links_kernel(int vh, RI in, RO out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    double m[18];
    get_link(in, vh, blockIdx.y, i, m);
    put_link(out, vh, blockIdx.y, i, m);
}

template <typename R>
__global__ void pack_field_kernel(Geom g, int p, const double *__restrict__ lex, R *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    Site s = site_of(g, p, i);
    const double *src = lex + (size_t)s.lex * 6;
    double v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = src[k];
    put_vec(out, g.vh, i, v);
}

template <typename R>
__global__ void unpack_field_kernel(Geom g, int p, const R *__restrict__ in, double *__restrict__ lex) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    Site s = site_of(g, p, i);
    double v[6];
    get_vec(in, g.vh, i, v);
    double *dst = lex + (size_t)s.lex * 6;
#pragma unroll
    for (int k = 0; k < 6; ++k) dst[k] = v[k];
}

template <typename RI, typename RO>
__global__ void convert_field_kernel(int vh, const RI *__restrict__ in, RO *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    double v[6];
    get_vec(in, vh, i, v);
    put_vec(out, vh, i, v);
}

static qex_status check_ptrs(const void *a, const void *b) {
    if (!a || !b) {
        set_error("field/link pointer is NULL");
        return QEX_ERR_ARG;
    }
    if (!aligned16(a) || !aligned16(b)) {
        set_error("field/link pointers must be 16-byte aligned");
        return QEX_ERR_ALIGN;
    }
    return QEX_OK;
}

template <typename RI>
static void convert_links_to(qex_prec to, int vh, RI in, void *out, dim3 grid, cudaStream_t s) {
    if (to == QEX_F64)
        convert_links_kernel<RI, double *><<<grid, kBlock, 0, s>>>(vh, in, (double *)out);
    else if (to == QEX_F32)
        convert_links_kernel<RI, float *><<<grid, kBlock, 0, s>>>(vh, in, (float *)out);
    else if (to == QEX_F32_R12)
        convert_links_kernel<RI, R12><<<grid, kBlock, 0, s>>>(vh, in, R12{(float *)out});
    else if (to == QEX_F32_R12H)
        convert_links_kernel<RI, R12H><<<grid, kBlock, 0, s>>>(vh, in, R12H{(float *)out});
    else
        convert_links_kernel<RI, S16><<<grid, kBlock, 0, s>>>(vh, in, S16{(float *)out});
}

// Pack the canonical links of internal indices [i0, i1) (both parities) into
// out64 (FP64) and, when out2 is given, into out2 in format `second` too.
qex_status launch_pack_links_range(qex_lattice *lat, const double *lex, void *out64, qex_prec second, void *out2,
                                   int i0, int i1, cudaStream_t s) {
    if (i1 <= i0) return QEX_OK;
    dim3 grid(blocks_for(i1 - i0), 8);
    double *o = (double *)out64;
    if (!out2)
        pack_links_range_kernel<void *><<<grid, kBlock, 0, s>>>(lat->geom, lex, o, nullptr, i0, i1);
    else if (second == QEX_F32)
        pack_links_range_kernel<float *><<<grid, kBlock, 0, s>>>(lat->geom, lex, o, (float *)out2, i0, i1);
    else if (second == QEX_F32_R12)
        pack_links_range_kernel<R12><<<grid, kBlock, 0, s>>>(lat->geom, lex, o, R12{(float *)out2}, i0, i1);
    else if (second == QEX_F32_R12H)
        pack_links_range_kernel<R12H><<<grid, kBlock, 0, s>>>(lat->geom, lex, o, R12H{(float *)out2}, i0, i1);
    else if (second == QEX_F32_S16)
        pack_links_range_kernel<S16><<<grid, kBlock, 0, s>>>(lat->geom, lex, o, S16{(float *)out2}, i0, i1);
    else {
        set_error("internal: no second link format %d", (int)second);
        return QEX_ERR_ARG;
    }
    QEX_CHECK_LAUNCH("pack_links_range_kernel");
    return QEX_OK;
}

}  // namespace qex

using namespace qex;

extern "C" {

qex_status qex_pack_links(const qex_lattice *lat, qex_prec prec, const double *lex_links, void *internal,
                          void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(prec)) || (st = check_ptrs(lex_links, internal))) return st;
    dim3 grid(blocks_for(lat->vh), 8);
    cudaStream_t s = as_stream(stream);
    if (prec == QEX_F64)
        pack_links_kernel<double *><<<grid, kBlock, 0, s>>>(lat->geom, lex_links, (double *)internal);
    else if (prec == QEX_F32)
        pack_links_kernel<float *><<<grid, kBlock, 0, s>>>(lat->geom, lex_links, (float *)internal);
    else if (prec == QEX_F32_R12)
        pack_links_kernel<R12><<<grid, kBlock, 0, s>>>(lat->geom, lex_links, R12{(float *)internal});
    else if (prec == QEX_F32_R12H)
        pack_links_kernel<R12H><<<grid, kBlock, 0, s>>>(lat->geom, lex_links, R12H{(float *)internal});
    else
        pack_links_kernel<S16><<<grid, kBlock, 0, s>>>(lat->geom, lex_links, S16{(float *)internal});
    QEX_CHECK_LAUNCH("pack_links_kernel");
    return QEX_OK;
}

qex_status qex_unpack_links(const qex_lattice *lat, qex_prec prec, const void *internal, double *lex_links,
                            void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(prec)) || (st = check_ptrs(lex_links, internal))) return st;
    dim3 grid(blocks_for(lat->vh), 8);
    cudaStream_t s = as_stream(stream);
    if (prec == QEX_F64)
        unpack_links_kernel<const double *><<<grid, kBlock, 0, s>>>(lat->geom, (const double *)internal, lex_links);
    else if (prec == QEX_F32)
        unpack_links_kernel<const float *><<<grid, kBlock, 0, s>>>(lat->geom, (const float *)internal, lex_links);
    else if (prec == QEX_F32_R12)
        unpack_links_kernel<R12c><<<grid, kBlock, 0, s>>>(lat->geom, R12c{(const float *)internal}, lex_links);
    else if (prec == QEX_F32_R12H)
        unpack_links_kernel<R12Hc><<<grid, kBlock, 0, s>>>(lat->geom, R12Hc{(const float *)internal}, lex_links);
    else
        unpack_links_kernel<S16c><<<grid, kBlock, 0, s>>>(lat->geom, S16c{(const float *)internal}, lex_links);
    QEX_CHECK_LAUNCH("unpack_links_kernel");
    return QEX_OK;
}

qex_status qex_pack_field(const qex_lattice *lat, qex_prec prec, int parity, const double *lex_field, void *half,
                          void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(prec)) || (st = check_ptrs(lex_field, half))) return st;
    if (parity != 0 && parity != 1) {
        set_error("parity must be 0 or 1");
        return QEX_ERR_ARG;
    }
    int nb = blocks_for(lat->vh);
    if (is_f64(prec))
        pack_field_kernel<double><<<nb, kBlock, 0, as_stream(stream)>>>(lat->geom, parity, lex_field, (double *)half);
    else
        pack_field_kernel<float><<<nb, kBlock, 0, as_stream(stream)>>>(lat->geom, parity, lex_field, (float *)half);
    QEX_CHECK_LAUNCH("pack_field_kernel");
    return QEX_OK;
}

qex_status qex_unpack_field(const qex_lattice *lat, qex_prec prec, int parity, const void *half, double *lex_field,
                            void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(prec)) || (st = check_ptrs(lex_field, half))) return st;
    if (parity != 0 && parity != 1) {
        set_error("parity must be 0 or 1");
        return QEX_ERR_ARG;
    }
    int nb = blocks_for(lat->vh);
    if (is_f64(prec))
        unpack_field_kernel<double>
            <<<nb, kBlock, 0, as_stream(stream)>>>(lat->geom, parity, (const double *)half, lex_field);
    else
        unpack_field_kernel<float>
            <<<nb, kBlock, 0, as_stream(stream)>>>(lat->geom, parity, (const float *)half, lex_field);
    QEX_CHECK_LAUNCH("unpack_field_kernel");
    return QEX_OK;
}

qex_status qex_pack_links_pair(const qex_lattice *lat, const double *lex_links, void *internal64, qex_prec second,
                               void *internal2, void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(second)) || (st = check_ptrs(lex_links, internal64)) ||
        (st = check_ptrs(internal2, internal64)))
        return st;
    if (second == QEX_F64) {
        set_error("the second link set of qex_pack_links_pair must be an FP32 format");
        return QEX_ERR_ARG;
    }
    return launch_pack_links_range(const_cast<qex_lattice *>(lat), lex_links, internal64, second, internal2, 0,
                                   (int)lat->vh, as_stream(stream));
}

qex_status qex_convert_links(const qex_lattice *lat, qex_prec from, const void *in, qex_prec to, void *out,
                             void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(from)) || (st = check_prec(to)) || (st = check_ptrs(in, out)))
        return st;
    dim3 grid(blocks_for(lat->vh), 8);
    cudaStream_t s = as_stream(stream);
    int vh = (int)lat->vh;
    if (from == QEX_F64)
        convert_links_to<const double *>(to, vh, (const double *)in, out, grid, s);
    else if (from == QEX_F32)
        convert_links_to<const float *>(to, vh, (const float *)in, out, grid, s);
    else if (from == QEX_F32_R12)
        convert_links_to<R12c>(to, vh, R12c{(const float *)in}, out, grid, s);
    else if (from == QEX_F32_R12H)
        convert_links_to<R12Hc>(to, vh, R12Hc{(const float *)in}, out, grid, s);
    else
        convert_links_to<S16c>(to, vh, S16c{(const float *)in}, out, grid, s);
    QEX_CHECK_LAUNCH("convert_links_kernel");
    return QEX_OK;
}

qex_status qex_convert_field(const qex_lattice *lat, qex_prec from, const void *in, qex_prec to, void *out,
                             void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(from)) || (st = check_prec(to)) || (st = check_ptrs(in, out)))
        return st;
    int nb = blocks_for(lat->vh);
    cudaStream_t s = as_stream(stream);
    int vh = (int)lat->vh;
    if (is_f64(from) && !is_f64(to))
        convert_field_kernel<double, float><<<nb, kBlock, 0, s>>>(vh, (const double *)in, (float *)out);
    else if (!is_f64(from) && is_f64(to))
        convert_field_kernel<float, double><<<nb, kBlock, 0, s>>>(vh, (const float *)in, (double *)out);
    else if (is_f64(from))
        convert_field_kernel<double, double><<<nb, kBlock, 0, s>>>(vh, (const double *)in, (double *)out);
    else
        convert_field_kernel<float, float><<<nb, kBlock, 0, s>>>(vh, (const float *)in, (float *)out);
    QEX_CHECK_LAUNCH("convert_field_kernel");
    return QEX_OK;
}

}  // extern "C"
