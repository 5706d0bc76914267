// dslash_mrhs.cu -- the even-odd staggered operator applied to N right-hand
// sides at once, each link read from memory once for all of them, with the
// epilogues of the multi-RHS CG.
//
// Fields: N half fields back to back (field r starts at r * qex_field_bytes).
// A block covers 32 consecutive output sites (threadIdx.x) and up to eight
// groups of four right-hand sides (threadIdx.y, one warp each; more groups
// go to blockIdx.y); the warps of a block request the same link addresses at
// about the same time, so a link line comes from HBM once and is served to
// the other warps from L1/L2.  Per site the algorithmic traffic is the 8 (16
// with Naik) links once plus, per right-hand side, the input vector once and
// the output once.  The reducing epilogues run a persistent grid-stride loop
// and reduce per right-hand side in a fixed order (bit-reproducible).
#include "qex_kernels.cuh"

namespace qex {

constexpr int kMrhsSites = 32;  // output sites per block (one warp row)
constexpr int kMrhsGroup = 4;   // right-hand sides per thread
constexpr int kMrhsWarps = 8;   // right-hand-side groups per block (more go to blockIdx.y)

template <typename R, int FMT>
__device__ __forceinline__ Mat3<R> load_fat_m(const R *base, size_t vh, int p, int mu, int i) {
    if constexpr (FMT == 1)
        return load_link_r12(base, vh, p, mu, i);
    else
        return load_link(base, vh, p, mu, i);
}

template <typename R>
struct MParams {
    Geom g;
    const R *fat, *lng;
    R c3;
    int p, nrhs;
    const R *in;
    R *out;
    const R *q;
    const double *b;
    R m2;
    MrhsScalars *S;
    int check_halt;
    const R *r;
    R *pbuf0, *pbuf1;
    double *partials;
    unsigned int *counter;
};

template <typename R, int EPI>
__device__ __forceinline__ Vec3<R> mrhs_in(const MParams<R> &P, const R *pold, R beta, size_t off, size_t vh,
                                           int j) {
    if constexpr (EPI == EPI_PUPD) {
        const Vec3<R> rv = load_vec(P.r + off, vh, j), pv = load_vec(pold + off, vh, j);
        Vec3<R> v;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
            v.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
        }
        return v;
    } else {
        return load_vec(P.in + off, vh, j);
    }
}

template <typename R, int FMT, bool NAIK, int EPI>
__global__ void __launch_bounds__(kMrhsSites * kMrhsWarps) dslash_mrhs_kernel(const MParams<R> P) {
    __shared__ unsigned int is_last;
    MrhsScalars *S = P.S;
    if (P.check_halt && S->halt) return;  // uniform over the grid
    const int r0 = (blockIdx.y * blockDim.y + threadIdx.y) * kMrhsGroup;
    const Geom &g = P.g;
    const size_t vh = (size_t)g.vh;
    const size_t fstride = 6 * vh;  // reals per half field
    const int p = P.p;
    bool act[kMrhsGroup];
    R beta[kMrhsGroup];
#pragma unroll
    for (int k = 0; k < kMrhsGroup; ++k) {
        const int r = r0 + k;
        act[k] = r < P.nrhs && (S == nullptr || S->active[r]);
        beta[k] = (EPI == EPI_PUPD && act[k]) ? (R)S->beta[r] : R(0);
    }
    const R *pold = nullptr;
    R *pnew = nullptr;
    if (EPI == EPI_PUPD || EPI == EPI_NORMAL) {
        const int it = S->iter;
        pold = (it & 1) ? P.pbuf1 : P.pbuf0;
        pnew = (it & 1) ? P.pbuf0 : P.pbuf1;
    }
    double part[kMrhsGroup] = {0.0, 0.0, 0.0, 0.0};

    for (int i = blockIdx.x * kMrhsSites + threadIdx.x; i < g.vh; i += gridDim.x * kMrhsSites) {
        const Site s = site_of(g, p, i);
        Vec3<R> acc[kMrhsGroup];
#pragma unroll
        for (int k = 0; k < kMrhsGroup; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[k].c[a].re = acc[k].c[a].im = R(0);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const R eta = eta_bit(s, mu) ? R(-1) : R(1);
#pragma unroll
            for (int hop = 0; hop < (NAIK ? 4 : 2); ++hop) {
                const int k3 = hop >= 2 ? 3 : 1;
                const bool fwd = (hop & 1) == 0;
                const int j = hop_index(g, s, mu, fwd ? k3 : -k3);
                Mat3<R> u;
                if (hop >= 2)
                    u = load_link(P.lng, vh, fwd ? p : 1 - p, mu, fwd ? i : j);
                else
                    u = load_fat_m<R, FMT>(P.fat, vh, fwd ? p : 1 - p, mu, fwd ? i : j);
                const int bc = fwd ? bc_bit_fwd(g, s, mu, k3) : bc_bit_bwd(g, s, mu, k3);
                R sg = (bc ? -eta : eta) * (hop >= 2 ? P.c3 : R(1));
                if (!fwd) sg = -sg;
#pragma unroll
                for (int k = 0; k < kMrhsGroup; ++k) {
                    if (act[k]) {
                        const Vec3<R> v = mrhs_in<R, EPI>(P, pold, beta[k], (size_t)(r0 + k) * fstride, vh, j);
                        if (fwd)
                            acc_mv(acc[k], sg, u, v);
                        else
                            acc_mdv(acc[k], sg, u, v);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kMrhsGroup; ++k) {
            if (!act[k]) continue;
            const size_t off = (size_t)(r0 + k) * fstride;
            if constexpr (EPI == EPI_PLAIN) {
                store_vec(P.out + off, vh, i, acc[k]);
            } else if constexpr (EPI == EPI_PUPD) {
                store_vec(P.out + off, vh, i, acc[k]);
                store_vec(pnew + off, vh, i, mrhs_in<R, EPI>(P, pold, beta[k], off, vh, i));
            } else if constexpr (EPI == EPI_NORMAL) {
                const Vec3<R> qv = load_vec(pnew + off, vh, i);
                Vec3<R> o;
                R d = R(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o.c[a].re = fma(P.m2, qv.c[a].re, -acc[k].c[a].re);
                    o.c[a].im = fma(P.m2, qv.c[a].im, -acc[k].c[a].im);
                    d = fma(qv.c[a].re, o.c[a].re, d);
                    d = fma(qv.c[a].im, o.c[a].im, d);
                }
                store_vec(P.out + off, vh, i, o);
                part[k] += (double)d;
            } else {  // EPI_RESID, FP64: out = b - m^2 x + D in
                const Vec3<R> qv = load_vec(P.q + off, vh, i);
                const Vec3<double> bv = load_vec(P.b + off, vh, i);
                Vec3<R> o;
                double d = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o.c[a].re = (R)bv.c[a].re - fma(P.m2, qv.c[a].re, -acc[k].c[a].re);
                    o.c[a].im = (R)bv.c[a].im - fma(P.m2, qv.c[a].im, -acc[k].c[a].im);
                    d = fma((double)o.c[a].re, (double)o.c[a].re, d);
                    d = fma((double)o.c[a].im, (double)o.c[a].im, d);
                }
                store_vec(P.out + off, vh, i, o);
                part[k] += d;
            }
        }
    }
    if constexpr (EPI == EPI_PLAIN || EPI == EPI_PUPD) {
        return;
    } else {
        // per right-hand side: warp sum -> partials[blockIdx.x][r]; the last
        // block sums each r over blockIdx.x in a fixed order
#pragma unroll
        for (int k = 0; k < kMrhsGroup; ++k) {
            double v = part[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0 && r0 + k < P.nrhs) P.partials[(size_t)blockIdx.x * P.nrhs + r0 + k] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            __threadfence();
            const unsigned int t = atomicAdd(P.counter, 1u);
            is_last = (t == gridDim.x * gridDim.y - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        for (int r = threadIdx.y; r < P.nrhs; r += blockDim.y) {
            double v = 0.0;
            for (int bx = threadIdx.x; bx < (int)gridDim.x; bx += 32) v += __ldcg(P.partials + (size_t)bx * P.nrhs + r);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x != 0 || !S->active[r]) continue;
            if constexpr (EPI == EPI_NORMAL) {
                S->pAp[r] = v;
                if (!(v > 0.0) || !isfinite(v)) {
                    S->error = isfinite(v) ? 2 : 1;
                    S->halt = 1;
                } else {
                    S->alpha[r] = S->rr[r] / v;
                }
            } else {
                S->true_rr[r] = v;
                if (!isfinite(v)) {
                    S->error = 1;
                    S->halt = 1;
                    continue;
                }
                S->beta[r] = S->rr[r] > 0.0 ? v / S->rr[r] : 0.0;
                S->rr[r] = v;
                S->rmax2[r] = v;
                if (v <= S->stop2[r]) {
                    S->done[r] = 1;
                    S->active[r] = 0;
                }
            }
        }
        if constexpr (EPI == EPI_RESID) {
            __syncthreads();
            if (threadIdx.x == 0 && threadIdx.y == 0) {
                int n = 0;
                for (int r = 0; r < P.nrhs; ++r) n += S->active[r];
                S->nactive = n;
                S->need_ru = 0;
                S->reliable_updates += 1;
                S->halt = (n == 0 || S->iter >= S->maxiter || S->error) ? 1 : 0;
            }
        }
        if (threadIdx.x == 0 && threadIdx.y == 0) *P.counter = 0u;
    }
}

template <typename R, int FMT, bool NAIK, int EPI>
static void launch_m(const qex_lattice *lat, const MrhsArgs &a, cudaStream_t st) {
    MParams<R> P;
    P.g = lat->geom;
    P.fat = (const R *)a.fat;
    P.lng = (const R *)a.lng;
    P.c3 = (R)a.c3;
    P.p = a.out_parity;
    P.nrhs = a.nrhs;
    P.in = (const R *)a.in;
    P.out = (R *)a.out;
    P.q = (const R *)a.q;
    P.b = a.b;
    P.m2 = (R)a.m2;
    P.S = a.S;
    P.check_halt = (a.S && (EPI == EPI_PUPD || EPI == EPI_NORMAL)) ? 1 : 0;
    P.r = (const R *)a.r;
    P.pbuf0 = (R *)a.pbuf[0];
    P.pbuf1 = (R *)a.pbuf[1];
    P.partials = lat->partials;
    P.counter = lat->counter;
    const int groups = (a.nrhs + kMrhsGroup - 1) / kMrhsGroup;
    const int wy = groups < kMrhsWarps ? groups : kMrhsWarps;
    const int full = (int)((lat->vh + kMrhsSites - 1) / kMrhsSites);
    int gx = full;
    if (EPI == EPI_NORMAL || EPI == EPI_RESID) {  // persistent grid for the reducing variants
        const int cap = sm_count() * 4;
        gx = full < cap ? full : cap;
    }
    dim3 block(kMrhsSites, wy);
    dim3 grid(gx, (groups + wy - 1) / wy);
    dslash_mrhs_kernel<R, FMT, NAIK, EPI><<<grid, block, 0, st>>>(P);
}

template <typename R, int FMT, bool NAIK>
static void launch_m_epi(const qex_lattice *lat, const MrhsArgs &a, cudaStream_t st) {
    if (a.epi == EPI_PLAIN)
        launch_m<R, FMT, NAIK, EPI_PLAIN>(lat, a, st);
    else if (a.epi == EPI_PUPD)
        launch_m<R, FMT, NAIK, EPI_PUPD>(lat, a, st);
    else if (a.epi == EPI_NORMAL)
        launch_m<R, FMT, NAIK, EPI_NORMAL>(lat, a, st);
    else if constexpr (std::is_same<R, double>::value)
        launch_m<R, FMT, NAIK, EPI_RESID>(lat, a, st);
}

qex_status launch_dslash_mrhs(qex_lattice *lat, const MrhsArgs &a, cudaStream_t st) {
    if (a.epi == EPI_NORMAL || a.epi == EPI_RESID) {
        qex_status s = ensure_scratch(lat);
        if (s) return s;
        const size_t need = (size_t)(sm_count() * 4 + 1) * a.nrhs;
        if ((size_t)lat->partials_len < need) {
            set_error("internal: partials buffer too small for %d right-hand sides", a.nrhs);
            return QEX_ERR_ARG;
        }
    }
    if (a.prec == QEX_F64) {
        if (a.lng)
            launch_m_epi<double, 0, true>(lat, a, st);
        else
            launch_m_epi<double, 0, false>(lat, a, st);
    } else {
        if (a.epi == EPI_RESID) {
            set_error("the residual epilogue is FP64 only");
            return QEX_ERR_ARG;
        }
        if (a.prec == QEX_F32_R12) {
            if (a.lng)
                launch_m_epi<float, 1, true>(lat, a, st);
            else
                launch_m_epi<float, 1, false>(lat, a, st);
        } else {
            if (a.lng)
                launch_m_epi<float, 0, true>(lat, a, st);
            else
                launch_m_epi<float, 0, false>(lat, a, st);
        }
    }
    QEX_CHECK_LAUNCH("dslash_mrhs_kernel");
    return QEX_OK;
}

qex_status check_dslash_args(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                             const void *in, const void *out);

}  // namespace qex

using namespace qex;

extern "C" qex_status qex_dslash_mrhs(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                                      double c_naik, int out_parity, int nrhs, const void *in, void *out,
                                      void *stream) {
    qex_status st = check_dslash_args(lat, prec, fat, lng, in, out);
    if (st) return st;
    if (out_parity != 0 && out_parity != 1) {
        set_error("out_parity must be 0 or 1");
        return QEX_ERR_ARG;
    }
    if (nrhs < 1 || nrhs > QEX_MRHS_MAX) {
        set_error("nrhs must be in [1, %d] (got %d)", QEX_MRHS_MAX, nrhs);
        return QEX_ERR_ARG;
    }
    MrhsArgs a = {};
    a.prec = prec;
    a.fat = fat;
    a.lng = lng;
    a.c3 = c_naik;
    a.out_parity = out_parity;
    a.nrhs = nrhs;
    a.in = in;
    a.out = out;
    a.epi = EPI_PLAIN;
    return launch_dslash_mrhs(const_cast<qex_lattice *>(lat), a, as_stream(stream));
}
