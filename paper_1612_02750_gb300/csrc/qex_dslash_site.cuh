// qex_dslash_site.cuh -- the staggered operator's sum at one output site,
// shared by the single-field, multi-RHS and multi-lattice kernels.
#pragma once

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

// (D in)(x) for the i-th site x (= s) of parity p:
//   sum_mu eta b U_mu(x) in(x+mu) - eta b U_mu(x-mu)^+ in(x-mu)
//   + c3 (the same with the long links and x +- 3mu)           [NAIK]
// `in(j)` returns the input vector at index j of the other parity.
template <typename R, int FMT, bool NAIK, typename In>
__device__ __forceinline__ Vec3<R> dslash_site(const Geom &g, const R *fat, const R *lng, R c3, int p, int i,
                                               const Site &s, const In &in) {
    const size_t vh = (size_t)g.vh;
    Vec3<R> acc;
#pragma unroll
    for (int a = 0; a < 3; ++a) acc.c[a].re = acc.c[a].im = R(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        const R eta = eta_bit(s, mu) ? R(-1) : R(1);
        {   // + eta b U_mu(x) in(x + mu)
            const int j = hop_index(g, s, mu, 1);
            if constexpr (FMT == 3) {
                float d;
                const Mat3<R> u = load_link_s16(fat, vh, p, mu, i, &d);
                acc_mv(acc, (bc_bit_fwd(g, s, mu, 1) ? -eta : eta) * d, u, in(j));
            } else {
                const Mat3<R> u = load_fat<R, FMT>(fat, vh, p, mu, i);
                if constexpr (FMT == 2)
                    acc_mv_fix16(acc, bc_bit_fwd(g, s, mu, 1) ? -eta : eta, u, in(j));
                else
                    acc_mv(acc, bc_bit_fwd(g, s, mu, 1) ? -eta : eta, u, in(j));
            }
        }
        {   // - eta b U_mu(x - mu)^+ in(x - mu)
            const int j = hop_index(g, s, mu, -1);
            if constexpr (FMT == 3) {
                float d;
                const Mat3<R> u = load_link_s16(fat, vh, 1 - p, mu, j, &d);
                acc_mdv(acc, (bc_bit_bwd(g, s, mu, 1) ? eta : -eta) * d, u, in(j));
            } else {
                const Mat3<R> u = load_fat<R, FMT>(fat, vh, 1 - p, mu, j);
                if constexpr (FMT == 2)
                    acc_mdv_fix16(acc, bc_bit_bwd(g, s, mu, 1) ? eta : -eta, u, in(j));
                else
                    acc_mdv(acc, bc_bit_bwd(g, s, mu, 1) ? eta : -eta, u, in(j));
            }
        }
        if (NAIK) {
            const R e3 = c3 * eta;
            {
                const int j = hop_index(g, s, mu, 3);
                if constexpr (FMT >= 2) {
                    float d;
                    const Mat3<R> u = load_link_s16(lng, vh, p, mu, i, &d);
                    acc_mv(acc, (bc_bit_fwd(g, s, mu, 3) ? -e3 : e3) * d, u, in(j));
                } else {
                    const Mat3<R> u = load_link(lng, vh, p, mu, i);
                    acc_mv(acc, bc_bit_fwd(g, s, mu, 3) ? -e3 : e3, u, in(j));
                }
            }
            {
                const int j = hop_index(g, s, mu, -3);
                if constexpr (FMT >= 2) {
                    float d;
                    const Mat3<R> u = load_link_s16(lng, vh, 1 - p, mu, j, &d);
                    acc_mdv(acc, (bc_bit_bwd(g, s, mu, 3) ? e3 : -e3) * d, u, in(j));
                } else {
                    const Mat3<R> u = load_link(lng, vh, 1 - p, mu, j);
                    acc_mdv(acc, bc_bit_bwd(g, s, mu, 3) ? e3 : -e3, u, in(j));
                }
            }
        }
    }
    return acc;
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
