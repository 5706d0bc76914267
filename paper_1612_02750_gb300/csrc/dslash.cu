// dslash.cu -- the even-odd staggered operator D_{p,1-p} (one-hop term plus
// optional Naik three-hop term) and its CG epilogues.
//
// One thread per output site of parity p.  Per site the kernel reads the
// four forward links stored at the site, the four backward links stored at
// the neighbours x - mu (block 1-p of the link set), and the eight neighbour
// colour vectors of the input half field; with the Naik term the same again
// for the long links and the x +- 3mu neighbours.  Staggered phases and the
// antiperiodic time boundary are computed from the site coordinates; no phase
// is folded into the links.
#include <type_traits>
#include "qex_dslash_site.cuh"
#include "qex_kernels.cuh"

namespace qex {

template <typename R>
struct DsParams {
    Geom g;
    const R *fat;
    const R *lng;
    R c3;
    int p;              // output parity
    const R *in;
    R *out;
    const R *q;
    const double *b;
    R m2;
    CgScalars *S;
    int check_halt;
    const R *r;         // EPI_PUPD
    R *x;               // EPI_PUPD: iterate that takes the pending alpha p_old (NULL: none)
    R *pbuf0, *pbuf1;   // p ping-pong
    int psel;
    int skip_zero_x;
    int reverse;        // walk the sites from the last index down
    int skip_ff;
    double *partials;
    unsigned int *counter;
};

template <typename R, int FMT, bool NAIK, int EPI>
__global__ void __launch_bounds__(kDslashBlock, DslashMinBlocks<R>::value) dslash_kernel(const DsParams<R> P) {
    __shared__ double smem[32];
    __shared__ unsigned int is_last;
    pdl_trigger();
    pdl_wait();  // everything below may read what earlier kernels wrote
    if (P.check_halt && P.S->halt) return;  // uniform over the grid
    if (P.skip_ff && P.S->ru_ff) return;    // uniform: a float-float update
    // first residual from a zero initial guess: D x = 0 (uniform over the grid)
    const bool zero_x = P.skip_zero_x && !P.S->x_nonzero;
    if (EPI == EPI_PLAIN && zero_x) return;

    const Geom &g = P.g;
    const size_t vh = (size_t)g.vh;
    const int p = P.p;
    // direction buffers by iteration parity (read before any block can change it)
    const R *pold = nullptr;
    R *pnew = nullptr;
    R beta = R(0);
    const R *in = P.in;
    if (EPI == EPI_PLAIN && P.psel) in = (P.S->iters & 1) ? P.pbuf0 : P.pbuf1;  // the new direction
    R alpha = R(0);
    if constexpr (EPI == EPI_PUPD) {
        alpha = (R)P.S->alpha;
        const int it = P.S->iters;
        pold = (it & 1) ? P.pbuf1 : P.pbuf0;
        pnew = (it & 1) ? P.pbuf0 : P.pbuf1;
        beta = (R)P.S->beta;
    }
    double part = 0.0;
    // grid-stride over the sites: one pass per thread when the grid covers
    // the lattice, several when the launch is persistent (reducing variants)
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < g.vh; k += gridDim.x * blockDim.x) {
        const int i = P.reverse ? g.vh - 1 - k : k;
        const Site s = site_of(g, p, i);
        Vec3<R> acc;
        if (EPI == EPI_RESID && zero_x) {
#pragma unroll
            for (int a = 0; a < 3; ++a) acc.c[a].re = acc.c[a].im = R(0);
        } else {
            acc = dslash_site<R, FMT, NAIK>(g, P.fat, P.lng, P.c3, p, i, s, [&](int j) {
                if constexpr (EPI == EPI_PUPD)
                    return axpy_vec(P.r, pold, beta, vh, j);
                else
                    return load_vec(in, vh, j);
            });
        }
        if constexpr (EPI == EPI_PLAIN) {
            store_vec(P.out, vh, i, acc);
        } else if constexpr (EPI == EPI_PUPD) {
            store_vec(P.out, vh, i, acc);
            // this thread also owns index i of the other parity's direction,
            // and of the iterate, which takes the previous iteration's alpha p
            // (p_old read once for both; the same FMAs as axpy_vec)
            const Vec3<R> pv = load_vec(pold, vh, i), rv = load_vec(P.r, vh, i);
            Vec3<R> pn;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                pn.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
                pn.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
            }
            store_vec(pnew, vh, i, pn);
            if (P.x) {
                Vec3<R> xv = load_vec(P.x, vh, i);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    xv.c[a].re = fma(alpha, pv.c[a].re, xv.c[a].re);
                    xv.c[a].im = fma(alpha, pv.c[a].im, xv.c[a].im);
                }
                store_vec(P.x, vh, i, xv);
            }
        } else if constexpr (EPI == EPI_NORMAL) {
            // out = m^2 q - D in;  part = Re <q, out>
            const R *q = P.q;
            if (P.psel) q = (P.S->iters & 1) ? P.pbuf0 : P.pbuf1;  // the new direction
            const Vec3<R> qv = load_vec(q, vh, i);
            Vec3<R> o;
            R d = R(0);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o.c[a].re = fma(P.m2, qv.c[a].re, -acc.c[a].re);
                o.c[a].im = fma(P.m2, qv.c[a].im, -acc.c[a].im);
                d = fma(qv.c[a].re, o.c[a].re, d);
                d = fma(qv.c[a].im, o.c[a].im, d);
            }
            store_vec(P.out, vh, i, o);
            part += (double)d;
        } else {
            // out = b - m^2 q + D in;  part = ||out||^2   (FP64 only)
            const Vec3<R> qv = load_vec(P.q, vh, i);
            const Vec3<double> bv = load_vec(P.b, vh, i);
            Vec3<R> o;
            double d = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o.c[a].re = (R)bv.c[a].re - fma(P.m2, qv.c[a].re, -acc.c[a].re);
                o.c[a].im = (R)bv.c[a].im - fma(P.m2, qv.c[a].im, -acc.c[a].im);
                d = fma((double)o.c[a].re, (double)o.c[a].re, d);
                d = fma((double)o.c[a].im, (double)o.c[a].im, d);
            }
            store_vec(P.out, vh, i, o);
            part += d;
        }
    }
    if constexpr (EPI == EPI_PLAIN || EPI == EPI_PUPD) {
        return;
    } else {
        CgScalars *S = P.S;
        if (S == nullptr) return;  // uniform over the grid

        // Deterministic grid reduction: block sums -> partials; the last block
        // to finish sums the partials in index order and updates the CG scalars.
        const double bs = block_sum(part, smem);
        if (threadIdx.x == 0) {
            P.partials[blockIdx.x] = bs;
            __threadfence();
            unsigned int t = atomicAdd(P.counter, 1u);
            is_last = (t == gridDim.x - 1) ? 1u : 0u;
        }
        __syncthreads();
        if (!is_last) return;
        __threadfence();
        const double tot = block_sum_partials(P.partials, gridDim.x, smem);
        if (threadIdx.x != 0) return;
        *P.counter = 0u;
        if constexpr (EPI == EPI_NORMAL) {
            S->pAp = tot;
            if (!(tot > 0.0) || !isfinite(tot)) {
                S->error = isfinite(tot) ? 2 : 1;
                S->halt = 1;
            } else {
                S->alpha = S->rr / tot;
            }
        } else {
            // FP64 true residual: accept convergence, or continue with beta from it
            take_true_residual(S, tot, true);
        }
    }
}

// Shape of a Dslash launch: one thread per site, or, for the variants that
// end in a grid reduction, a persistent grid of as many blocks per SM as the
// launch bounds keep resident, so that each block pays the reduction's
// fence-and-atomic tail once.  The autotuner may replace the block size and
// the persistent grid per (precision, Naik) of the lattice, and may cap the
// other variants' grid at a few resident waves (min_blocks x kDslashBlock
// threads per SM each), each thread then taking ~1-2 sites grid-stride: on a
// launch of 3-4 waves this trims the partial last wave.
static void dslash_shape(const qex_lattice *lat, qex_prec prec, bool naik, bool reducing, int min_blocks, int *grid,
                         int *block) {
    const LaunchShape &sh = lat->shape[prec][naik ? 1 : 0];
    int per_sm = QEX_REDUCE_BLOCKS_PER_SM >= 0 ? QEX_REDUCE_BLOCKS_PER_SM : min_blocks;
    int b = kDslashBlock;
    if (sh.red_block > 0) {
        b = reducing ? sh.red_block : sh.ds_block;
        per_sm = sh.red_per_sm;
    }
    *block = b;
    const int full = blocks_for(lat->vh, b);
    *grid = full;
    if (reducing && per_sm > 0) {
        const int persistent = sm_count() * per_sm;
        if (persistent < full) *grid = persistent;
    }
    if (!reducing && sh.red_block > 0 && sh.ds_waves > 0) {
        const int capped = sm_count() * sh.ds_waves * (min_blocks * kDslashBlock / b);
        if (capped > 0 && capped < full) *grid = capped;
    }
}

template <typename R, int FMT, bool NAIK, int EPI>
static void launch_t(qex_lattice *lat, const DslashArgs &a, cudaStream_t st) {
    DsParams<R> P;
    P.g = lat->geom;
    P.fat = (const R *)a.fat;
    P.lng = (const R *)a.lng;
    P.c3 = (R)a.c3;
    P.p = a.out_parity;
    P.in = (const R *)a.in;
    P.out = (R *)a.out;
    P.q = (const R *)a.q;
    P.b = a.b;
    P.m2 = (R)a.m2;
    P.S = a.S;
    P.check_halt = a.check_halt;
    P.r = (const R *)a.r;
    P.x = (R *)a.x;
    P.pbuf0 = (R *)a.pbuf[0];
    P.pbuf1 = (R *)a.pbuf[1];
    P.psel = a.psel;
    P.skip_zero_x = a.skip_zero_x;
    P.reverse = a.reverse;
    P.skip_ff = a.skip_ff;
    P.partials = lat->partials;
    P.counter = lat->counter;
    int grid, block;
    dslash_shape(lat, a.prec, NAIK, EPI != EPI_PLAIN && EPI != EPI_PUPD && a.S != nullptr, DslashMinBlocks<R>::value,
                 &grid, &block);
    launch_k(dslash_kernel<R, FMT, NAIK, EPI>, dim3(grid), dim3(block), 0, st, lat->pdl != 0, P);
}

template <typename R, int FMT, bool NAIK>
static void launch_epi(qex_lattice *lat, const DslashArgs &a, cudaStream_t st) {
    if (a.epi == EPI_PLAIN)
        launch_t<R, FMT, NAIK, EPI_PLAIN>(lat, a, st);
    else if (a.epi == EPI_NORMAL)
        launch_t<R, FMT, NAIK, EPI_NORMAL>(lat, a, st);
    else if (a.epi == EPI_PUPD)
        launch_t<R, FMT, NAIK, EPI_PUPD>(lat, a, st);
    else if constexpr (std::is_same<R, double>::value)
        launch_t<R, FMT, NAIK, EPI_RESID>(lat, a, st);
}

qex_status launch_dslash(qex_lattice *lat, const DslashArgs &a, cudaStream_t st) {
    if (a.S) {
        qex_status s = ensure_scratch(lat);
        if (s) return s;
    }
    if (a.prec == QEX_F64) {
        if (a.lng)
            launch_epi<double, 0, true>(lat, a, st);
        else
            launch_epi<double, 0, false>(lat, a, st);
    } else {
        if (a.epi == EPI_RESID) {
            set_error("the residual epilogue is FP64 only");
            return QEX_ERR_ARG;
        }
        if (a.prec == QEX_F32_R12) {
            if (a.lng)
                launch_epi<float, 1, true>(lat, a, st);
            else
                launch_epi<float, 1, false>(lat, a, st);
        } else if (a.prec == QEX_F32_R12H) {
            if (a.lng)
                launch_epi<float, 2, true>(lat, a, st);
            else
                launch_epi<float, 2, false>(lat, a, st);
        } else if (a.prec == QEX_F32_S16) {
            if (a.lng)
                launch_epi<float, 3, true>(lat, a, st);
            else
                launch_epi<float, 3, false>(lat, a, st);
        } else {
            if (a.lng)
                launch_epi<float, 0, true>(lat, a, st);
            else
                launch_epi<float, 0, false>(lat, a, st);
        }
    }
    QEX_CHECK_LAUNCH("dslash_kernel");
    return QEX_OK;
}

qex_status check_dslash_args(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                             const void *in, const void *out) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(prec))) return st;
    if (!fat || !in || !out) {
        set_error("fat, in and out must not be NULL");
        return QEX_ERR_ARG;
    }
    if (!aligned16(fat) || !aligned16(in) || !aligned16(out) || (lng && !aligned16(lng))) {
        set_error("links and fields must be 16-byte aligned");
        return QEX_ERR_ALIGN;
    }
    if (in == out) {
        set_error("in and out must not alias");
        return QEX_ERR_ARG;
    }
    if (lng) {
        for (int mu = 0; mu < 4; ++mu)
            if (lat->dims[mu] < 4) {
                set_error("the Naik term needs every extent >= 4");
                return QEX_ERR_SHAPE;
            }
    }
    return QEX_OK;
}

}  // namespace qex

using namespace qex;

extern "C" {

qex_status qex_dslash(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng, double c_naik,
                      int out_parity, const void *in, void *out, void *stream) {
    qex_status st = check_dslash_args(lat, prec, fat, lng, in, out);
    if (st) return st;
    if (out_parity != 0 && out_parity != 1) {
        set_error("out_parity must be 0 or 1");
        return QEX_ERR_ARG;
    }
    qex_lattice *l = const_cast<qex_lattice *>(lat);
    if ((st = ensure_tuned(l, prec, fat, lng, as_stream(stream), false))) return st;
    DslashArgs a = {};
    a.prec = prec;
    a.fat = fat;
    a.lng = lng;
    a.c3 = c_naik;
    a.out_parity = out_parity;
    a.in = in;
    a.out = out;
    a.epi = EPI_PLAIN;
    return launch_dslash(l, a, as_stream(stream));
}

qex_status qex_normal_op(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng, double c_naik,
                         double mass, const void *in, void *out, void *tmp_odd, void *stream) {
    qex_status st = check_dslash_args(lat, prec, fat, lng, in, out);
    if (st) return st;
    if (!tmp_odd || !aligned16(tmp_odd) || tmp_odd == in || tmp_odd == out) {
        set_error("tmp_odd must be a separate, 16-byte aligned half field");
        return QEX_ERR_ARG;
    }
    qex_lattice *l = const_cast<qex_lattice *>(lat);
    cudaStream_t s = as_stream(stream);
    if ((st = ensure_tuned(l, prec, fat, lng, s, false))) return st;
    DslashArgs a = {};
    a.prec = prec;
    a.fat = fat;
    a.lng = lng;
    a.c3 = c_naik;
    a.out_parity = 1;
    a.in = in;
    a.out = tmp_odd;
    a.epi = EPI_PLAIN;
    if ((st = launch_dslash(l, a, s))) return st;
    // normal epilogue without CG state (S = NULL): no reduction is formed
    a.out_parity = 0;
    a.in = tmp_odd;
    a.out = out;
    a.epi = EPI_NORMAL;
    a.q = in;
    a.m2 = mass * mass;
    return launch_dslash(l, a, s);
}

}  // extern "C"
