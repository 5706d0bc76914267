// dslash_mrhs.cu -- the even-odd staggered operator applied to N right-hand
// sides at once, each link read from memory once for all of them, with the
// epilogues of the multi-RHS CG.
//
// Fields: N half fields back to back (field r starts at r * qex_field_bytes).
// Per site the algorithmic traffic is the 8 (16 with Naik) links once plus,
// per right-hand side, the input vector once and the output once.  The
// reducing epilogues run a persistent grid-stride loop and reduce per
// right-hand side in a fixed order (bit-reproducible).
#include "qex_dslash_site.cuh"
#include "qex_kernels.cuh"

namespace qex {

// Thread mapping: one output site per thread and a group of KR right-hand
// sides per thread (held in registers; KR by precision and epilogue, see
// MrhsShape): each link is loaded and decoded once per group and applied to
// all KR vectors.
// A block is 256 sites of one group; linear block b covers site block
// b / ngroups and group b % ngroups, so the blocks that reuse a link run back
// to back and find it in L2.
constexpr int kMrhsBlock = 256;  // threads (sites) per block
// Right-hand sides per thread (KR) and resident blocks per SM (MINB, the
// register cap) by precision and epilogue.  The plain Dslash keeps KR = 4 at 2
// blocks (128 registers: the four accumulators, the four input vectors of a
// hop and a decoded link; the four independent mat-vecs supply the
// instruction-level parallelism that the lower occupancy gives up).  The CG
// epilogues, which also gather the directions or read the q vectors, run
// faster at KR = 2 and 4 blocks (24^4, 16 sources: the batched mixed CG
// 0.42 s against 0.46 s); FP64 keeps KR = 2 at 2 blocks (it spills above).
#ifndef QEX_MRHS_KR_CG
#define QEX_MRHS_KR_CG 2
#endif
#ifndef QEX_MRHS_MIN_BLOCKS_CG
#define QEX_MRHS_MIN_BLOCKS_CG 4
#endif
template <typename R, int EPI>
struct MrhsShape {
    static constexpr int kr = EPI == EPI_PLAIN ? 4 : QEX_MRHS_KR_CG;
    static constexpr int minb = EPI == EPI_PLAIN ? 2 : QEX_MRHS_MIN_BLOCKS_CG;
};
template <int EPI>
struct MrhsShape<double, EPI> {
    static constexpr int kr = 2;
    static constexpr int minb = 2;
};
// the largest persistent grid times KR of any reducing variant (partials per launch)
constexpr int kMrhsMaxPartialsPerSm = 8;

template <typename R>
struct MParams {
    Geom g;
    const R *fat, *lng;
    R c3;
    int p, nrhs, ngroups;
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

template <typename R, int FMT, bool NAIK, int EPI>
__global__ void __launch_bounds__(kMrhsBlock, (MrhsShape<R, EPI>::minb)) dslash_mrhs_kernel(const MParams<R> P) {
    constexpr int KR = MrhsShape<R, EPI>::kr;
    __shared__ double wsum[kMrhsBlock / 32][KR];
    __shared__ unsigned int is_last;
    MrhsScalars *S = P.S;
    if (P.check_halt && S->halt) return;  // uniform over the grid
    const Geom &g = P.g;
    const size_t vh = (size_t)g.vh;
    const size_t fstride = 6 * vh;  // reals per half field
    const int p = P.p;
    const int nsb = (int)((vh + kMrhsBlock - 1) / kMrhsBlock);
    const int total = nsb * P.ngroups;
    const R *pold = nullptr;
    R *pnew = nullptr;
    if (EPI == EPI_PUPD || EPI == EPI_NORMAL) {
        const int it = S->iter;
        pold = (it & 1) ? P.pbuf1 : P.pbuf0;
        pnew = (it & 1) ? P.pbuf0 : P.pbuf1;
    }
    double part[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) part[k] = 0.0;
    // reducing launches have gridDim.x a multiple of ngroups: the group is fixed per block
    for (int bl = blockIdx.x; bl < total; bl += gridDim.x) {
        const int grp = bl % P.ngroups;
        const int i = (bl / P.ngroups) * kMrhsBlock + threadIdx.x;
        if (i >= g.vh) continue;
        bool act[KR];
        R beta[KR];
        size_t off[KR];
        bool any = false;
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int rh = grp * KR + k;  // uniform over the block
            act[k] = rh < P.nrhs && (S == nullptr || S->active[rh]);
            any |= act[k];
            off[k] = (size_t)(act[k] ? rh : 0) * fstride;
            beta[k] = (EPI == EPI_PUPD && act[k]) ? (R)S->beta[rh] : R(0);
        }
        if (!any) continue;
        const Site s = site_of(g, p, i);
        Vec3<R> acc[KR];
        dslash_site_n<R, FMT, NAIK, KR>(g, P.fat, P.lng, P.c3, p, i, s, [&](int j, int k) {
            Vec3<R> v;
            if (!act[k]) {
#pragma unroll
                for (int a = 0; a < 3; ++a) v.c[a].re = v.c[a].im = R(0);
            } else if constexpr (EPI == EPI_PUPD) {
                v = axpy_vec(P.r + off[k], pold + off[k], beta[k], vh, j);
            } else {
                v = load_vec(P.in + off[k], vh, j);
            }
            return v;
        }, acc);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            if (!act[k]) continue;
            if constexpr (EPI == EPI_PLAIN) {
                store_vec(P.out + off[k], vh, i, acc[k]);
            } else if constexpr (EPI == EPI_PUPD) {
                store_vec(P.out + off[k], vh, i, acc[k]);
                store_vec(pnew + off[k], vh, i, axpy_vec(P.r + off[k], pold + off[k], beta[k], vh, i));
            } else if constexpr (EPI == EPI_NORMAL) {
                const Vec3<R> qv = load_vec(pnew + off[k], vh, i);
                Vec3<R> o;
                R d = R(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o.c[a].re = fma(P.m2, qv.c[a].re, -acc[k].c[a].re);
                    o.c[a].im = fma(P.m2, qv.c[a].im, -acc[k].c[a].im);
                    d = fma(qv.c[a].re, o.c[a].re, d);
                    d = fma(qv.c[a].im, o.c[a].im, d);
                }
                store_vec(P.out + off[k], vh, i, o);
                part[k] += (double)d;
            } else {  // EPI_RESID, FP64: out = b - m^2 x + D in
                const Vec3<R> qv = load_vec(P.q + off[k], vh, i);
                const Vec3<double> bv = load_vec(P.b + off[k], vh, i);
                Vec3<R> o;
                double d = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o.c[a].re = (R)bv.c[a].re - fma(P.m2, qv.c[a].re, -acc[k].c[a].re);
                    o.c[a].im = (R)bv.c[a].im - fma(P.m2, qv.c[a].im, -acc[k].c[a].im);
                    d = fma((double)o.c[a].re, (double)o.c[a].re, d);
                    d = fma((double)o.c[a].im, (double)o.c[a].im, d);
                }
                store_vec(P.out + off[k], vh, i, o);
                part[k] += d;
            }
        }
    }
    if constexpr (EPI == EPI_PLAIN || EPI == EPI_PUPD) {
        return;
    } else {
        // per right-hand side of this block's group: a fixed shuffle tree in
        // each warp, then warps in order -> partials[blockIdx.x * KR + k]
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            double v = part[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) wsum[warp][k] = v;
        }
        __syncthreads();
        if (threadIdx.x < KR) {
            double t = 0.0;
            for (int w = 0; w < kMrhsBlock / 32; ++w) t += wsum[w][threadIdx.x];
            P.partials[(size_t)blockIdx.x * KR + threadIdx.x] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned int t = atomicAdd(P.counter, 1u);
            is_last = (t == gridDim.x - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        // right-hand side r = grp * KR + k lives in blocks bx = grp (mod ngroups)
        const int nw = kMrhsBlock / 32;
        for (int r = warp; r < P.nrhs; r += nw) {
            const int grp = r / KR, kk = r % KR;
            double t = 0.0;
            for (int bx = grp + lane * P.ngroups; bx < (int)gridDim.x; bx += 32 * P.ngroups)
                t += __ldcg(P.partials + (size_t)bx * KR + kk);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane != 0 || !S->active[r]) continue;
            if constexpr (EPI == EPI_NORMAL) {
                S->pAp[r] = t;
                if (!(t > 0.0) || !isfinite(t)) {
                    S->error = isfinite(t) ? 2 : 1;
                    S->halt = 1;
                } else {
                    S->alpha[r] = S->rr[r] / t;
                }
            } else {
                S->true_rr[r] = t;
                if (!isfinite(t)) {
                    S->error = 1;
                    S->halt = 1;
                    continue;
                }
                S->beta[r] = S->rr[r] > 0.0 ? t / S->rr[r] : 0.0;
                S->rr[r] = t;
                S->rmax2[r] = t;
                if (t <= S->stop2[r]) {
                    S->done[r] = 1;
                    S->active[r] = 0;
                }
            }
        }
        if constexpr (EPI == EPI_RESID) {
            __syncthreads();
            if (threadIdx.x == 0) {
                int n = 0;
                for (int r = 0; r < P.nrhs; ++r) n += S->active[r];
                S->nactive = n;
                S->need_ru = 0;
                S->ru_iter0 = S->iter;
                S->reliable_updates += 1;
                S->halt = (n == 0 || S->iter >= S->maxiter || S->error) ? 1 : 0;
            }
        }
        if (threadIdx.x == 0) *P.counter = 0u;
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
    constexpr int KR = MrhsShape<R, EPI>::kr;
    P.ngroups = (a.nrhs + KR - 1) / KR;
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
    const int nsb = (int)((lat->vh + kMrhsBlock - 1) / kMrhsBlock);
    const int total = nsb * P.ngroups;
    int gx = total;
    if (EPI == EPI_NORMAL || EPI == EPI_RESID) {  // persistent grid, a multiple of ngroups
        int cap = sm_count() * MrhsShape<R, EPI>::minb;
        cap -= cap % P.ngroups;
        if (cap < P.ngroups) cap = P.ngroups;
        gx = total < cap ? total : cap;
    }
    dslash_mrhs_kernel<R, FMT, NAIK, EPI><<<gx, kMrhsBlock, 0, st>>>(P);
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
        const size_t need = (size_t)(sm_count() + 1) * kMrhsMaxPartialsPerSm;
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
        } else if (a.prec == QEX_F32_R12H) {
            if (a.lng)
                launch_m_epi<float, 2, true>(lat, a, st);
            else
                launch_m_epi<float, 2, false>(lat, a, st);
        } else if (a.prec == QEX_F32_S16) {
            if (a.lng)
                launch_m_epi<float, 3, true>(lat, a, st);
            else
                launch_m_epi<float, 3, false>(lat, a, st);
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
