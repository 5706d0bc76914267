// qex_dslash_site.cuh -- the staggered operator's sum at one output site,
// shared by the single-field, multi-RHS and multi-lattice kernels.
#pragma once

#include <type_traits>

#include "qex_common.cuh"

namespace qex {

// Fat-link formats: 0 = full 3x3 in the field precision, 1 = FP32 two-row,
// 2 = 16-bit fixed-point two-row (third row rebuilt in registers, the matrix
// held scaled: see load_link_fix16), 3 = 16-bit fixed-point full 3x3 with a
// per-link step (load_link_s16).  Long links are full 3x3 in the field
// precision for formats 0 and 1, and 16-bit with a per-link step for 2 and 3.
template <typename R, int FMT>
__device__ __forceinline__ Mat3<R> load_fat(const R *base, size_t vh, int p, int mu, int i) {
    if constexpr (FMT == 1)
        return load_link_r12(base, vh, p, mu, i);
    else if constexpr (FMT == 2)
        return load_link_fix16(base, vh, p, mu, i);
    else
        return load_link(base, vh, p, mu, i);
}

// (D in_k)(x), k = 0..K-1, for the i-th site x (= s) of parity p:
//   sum_mu eta b U_mu(x) in(x+mu) - eta b U_mu(x-mu)^+ in(x-mu)
//   + c3 (the same with the long links and x +- 3mu)           [NAIK]
// `in(j, k)` returns the input vector of field k at index j of the other
// parity.  Each link is loaded and decoded once and applied to all K fields.
template <typename R, int FMT, bool NAIK, int K, typename In>
__device__ __forceinline__ void dslash_site_n(const Geom &g, const R *fat, const R *lng, R c3, int p, int i,
                                              const Site &s, const In &in, Vec3<R> (&acc)[K]) {
    const size_t vh = (size_t)g.vh;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[k].c[a].re = acc[k].c[a].im = R(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const R eta = eta_bit(s, mu) ? R(-1) : R(1);
        {   // + eta b U_mu(x) in(x + mu)
            const int j = hop_index(g, s, mu, 1);
            const R sg = bc_bit_fwd(g, s, mu, 1) ? -eta : eta;
            if constexpr (FMT == 3) {
                float d;
                const Mat3<R> u = load_link_s16(fat, vh, p, mu, i, &d);
#pragma unroll
                for (int k = 0; k < K; ++k) acc_mv(acc[k], sg * d, u, in(j, k));
            } else {
                const Mat3<R> u = load_fat<R, FMT>(fat, vh, p, mu, i);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if constexpr (FMT == 2)
                        acc_mv_fix16(acc[k], sg, u, in(j, k));
                    else if constexpr (std::is_same<R, double>::value)
                        acc_mv_unit(acc[k], sg < R(0), u, in(j, k));
                    else
                        acc_mv(acc[k], sg, u, in(j, k));
                }
            }
        }
        {   // - eta b U_mu(x - mu)^+ in(x - mu)
            const int j = hop_index(g, s, mu, -1);
            const R sg = bc_bit_bwd(g, s, mu, 1) ? eta : -eta;
            if constexpr (FMT == 3) {
                float d;
                const Mat3<R> u = load_link_s16(fat, vh, 1 - p, mu, j, &d);
#pragma unroll
                for (int k = 0; k < K; ++k) acc_mdv(acc[k], sg * d, u, in(j, k));
            } else {
                const Mat3<R> u = load_fat<R, FMT>(fat, vh, 1 - p, mu, j);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if constexpr (FMT == 2)
                        acc_mdv_fix16(acc[k], sg, u, in(j, k));
                    else if constexpr (std::is_same<R, double>::value)
                        acc_mdv_unit(acc[k], sg < R(0), u, in(j, k));
                    else
                        acc_mdv(acc[k], sg, u, in(j, k));
                }
            }
        }
        if (NAIK) {
            const R e3 = c3 * eta;
            {
                const int j = hop_index(g, s, mu, 3);
                const R sg = bc_bit_fwd(g, s, mu, 3) ? -e3 : e3;
                if constexpr (FMT >= 2) {
                    float d;
                    const Mat3<R> u = load_link_s16(lng, vh, p, mu, i, &d);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc_mv(acc[k], sg * d, u, in(j, k));
                } else {
                    const Mat3<R> u = load_link(lng, vh, p, mu, i);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc_mv(acc[k], sg, u, in(j, k));
                }
            }
            {
                const int j = hop_index(g, s, mu, -3);
                const R sg = bc_bit_bwd(g, s, mu, 3) ? e3 : -e3;
                if constexpr (FMT >= 2) {
                    float d;
                    const Mat3<R> u = load_link_s16(lng, vh, 1 - p, mu, j, &d);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc_mdv(acc[k], sg * d, u, in(j, k));
                } else {
                    const Mat3<R> u = load_link(lng, vh, 1 - p, mu, j);
#pragma unroll
                    for (int k = 0; k < K; ++k) acc_mdv(acc[k], sg, u, in(j, k));
                }
            }
        }
    }
}

// One field: (D in)(x), `in(j)` the input vector at index j.
template <typename R, int FMT, bool NAIK, typename In>
__device__ __forceinline__ Vec3<R> dslash_site(const Geom &g, const R *fat, const R *lng, R c3, int p, int i,
                                               const Site &s, const In &in) {
    Vec3<R> acc[1];
    dslash_site_n<R, FMT, NAIK, 1>(g, fat, lng, c3, p, i, s, [&](int j, int) { return in(j); }, acc);
    return acc[0];
}

// r + beta p at index j (the CG direction formed on the fly).
template <typename R>
__device__ __forceinline__ Vec3<R> axpy_vec(const R *r, const R *p, R beta, size_t vh, int j) {
    const Vec3<R> rv = load_vec(r, vh, j), pv = load_vec(p, vh, j);
    Vec3<R> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
        v.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
    }
    return v;
}

}  // namespace qex
