// blas.cu -- fused CG vector updates and deterministic FP64 reductions.
//
// Grid-stride kernels over the Vh sites of one parity with a fixed grid per
// lattice (at most QEX_BLAS_BLOCKS_PER_SM blocks per SM), so the per-block partial sums -- and
// therefore every reduction -- come out bit-identical run to run.  Sums are
// formed per site in the vector precision and accumulated across sites in
// FP64.
#include "qex_kernels.cuh"

namespace qex {

// Block partial -> partials[]; the last block sums them in index order.
// Returns true in thread 0 of the last block, with *tot set.
__device__ __forceinline__ bool grid_sum(double part, double *partials, unsigned int *counter, double *smem,
                                         double *tot) {
    __shared__ unsigned int is_last;
    const double bs = block_sum(part, smem);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bs;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    const double s = block_sum_partials(partials, gridDim.x, smem);
    if (threadIdx.x != 0) return false;
    *counter = 0u;
    *tot = s;
    return true;
}

template <typename R>
__device__ __forceinline__ R norm2_site(const Vec3<R> &v) {
    R s = v.c[0].re * v.c[0].re;
    s = fma(v.c[0].im, v.c[0].im, s);
#pragma unroll
    for (int a = 1; a < 3; ++a) {
        s = fma(v.c[a].re, v.c[a].re, s);
        s = fma(v.c[a].im, v.c[a].im, s);
    }
    return s;
}

__device__ __forceinline__ void set_conditions(const GraphCtl &ctl, unsigned int loop, unsigned int ru) {
    if (ctl.active) {
        cudaGraphSetConditional(ctl.loop, loop);
        cudaGraphSetConditional(ctl.ru, ru);
    }
}

// x += alpha p_new (DO_X; otherwise the next iteration's first Dslash adds
// it); r -= alpha ap; ||r||^2 -> rr_new; then the CG scalar
// logic: continue (beta = rr_new / rr), or ask for a reliable update
// (iterated residual small enough, or the iteration cap reached), or stop
// on a NaN.  In the graph solve the last block also sets the loop and
// reliable-update conditions; a halted entry clears both.
template <typename R, bool DO_X>
__global__ void __launch_bounds__(kBlock)
update_xr_kernel(int vh, R *__restrict__ x, R *__restrict__ r, R *pbuf0, R *pbuf1, const R *__restrict__ ap,
                 CgScalars *S, double *partials, unsigned int *counter, const GraphCtl ctl) {
    __shared__ double smem[32];
    pdl_trigger();
    pdl_wait();
    if (S->halt) {
        // an earlier iteration of the same graph trip asked for a reliable
        // update (keep its conditions) or stopped on an error (end the loop)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned int ru = (S->need_ru && !S->error) ? 1u : 0u;
            set_conditions(ctl, ru, ru);
            S->idle_iters += 1;
        }
        return;
    }
    // fail-safe: stop unless the last block (which runs after this block's
    // fenced atomicAdd below) sets the conditions again
    if (blockIdx.x == 0 && threadIdx.x == 0) set_conditions(ctl, 0u, 0u);
    const R alpha = (R)S->alpha;
    const R *p = (S->iters & 1) ? pbuf0 : pbuf1;  // the new direction
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
        Vec3<R> rv = load_vec(r, vh, i);
        const Vec3<R> av = load_vec(ap, vh, i);
        if constexpr (DO_X) {
            Vec3<R> xv = load_vec(x, vh, i);
            const Vec3<R> pv = load_vec(p, vh, i);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xv.c[a].re = fma(alpha, pv.c[a].re, xv.c[a].re);
                xv.c[a].im = fma(alpha, pv.c[a].im, xv.c[a].im);
            }
            store_vec(x, vh, i, xv);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            rv.c[a].re = fma(-alpha, av.c[a].re, rv.c[a].re);
            rv.c[a].im = fma(-alpha, av.c[a].im, rv.c[a].im);
        }
        store_vec(r, vh, i, rv);
        part += (double)norm2_site(rv);
    }
    double rr_new;
    if (!grid_sum(part, partials, counter, smem, &rr_new)) return;
    S->iters += 1;
    S->trips += 1;
    if (!isfinite(rr_new)) {
        S->error = 1;
        S->halt = 1;
        set_conditions(ctl, 0u, 0u);
        return;
    }
    if (rr_new > S->rmax2) S->rmax2 = rr_new;
    const bool long_cycle = S->max_cycle > 0 && S->iters - S->ru_iter0 >= S->max_cycle;
    if (rr_new <= S->stop2 || rr_new < S->delta2 * S->rmax2 || S->iters >= S->maxiter || long_cycle) {
        // true residual next (reliable update / convergence check); rr keeps
        // the previous value so that beta is formed from the true one; an
        // update that cannot end the solve may run in float-float arithmetic
        S->ru_ff = (S->ff_ok && rr_new > S->stop2 && S->iters < S->maxiter) ? 1 : 0;
        S->rr_ru = rr_new;
        S->need_ru = 1;
        S->halt = 1;
        set_conditions(ctl, S->trips < S->maxiter + 4 ? 1u : 0u, 1u);
        return;
    }
    S->beta = rr_new / S->rr;
    S->rr = rr_new;
    set_conditions(ctl, S->trips < S->maxiter + 4 ? 1u : 0u, 0u);
}

// p_new = r + beta p_old, buffers by iteration parity
template <typename R>
__global__ void __launch_bounds__(kBlock)
update_p_kernel(int vh, const R *__restrict__ r, R *pbuf0, R *pbuf1, const CgScalars *S) {
    pdl_trigger();
    pdl_wait();
    if (S->halt) return;
    const int it = S->iters;
    const R *pold = (it & 1) ? pbuf1 : pbuf0;
    R *pnew = (it & 1) ? pbuf0 : pbuf1;
    const R beta = (R)S->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
        const Vec3<R> rv = load_vec(r, vh, i), pv = load_vec(pold, vh, i);
        Vec3<R> o;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o.c[a].re = fma(beta, pv.c[a].re, rv.c[a].re);
            o.c[a].im = fma(beta, pv.c[a].im, rv.c[a].im);
        }
        store_vec(pnew, vh, i, o);
    }
}

// Float-float error of a true residual, relative to sqrt(||x||^2 + ||b||^2):
// measured 0.7-1.2e-13 near the solution on Haar and exp(i a H) links, 4^4
// to 32^4, m = 0.005..0.05, with and without the Naik term.
constexpr double kFfErr = 2.5e-13;

// x64 += xh32 + alpha p (the iterate update the last iteration left pending,
// p = pbuf[iters & 1]; pbuf0 NULL: none); xh32 = 0.  When the update was asked
// for in float-float arithmetic, ||x64||^2 decides whether it may be: its
// error, kFfErr (||x|| + ||b||), has to stay below 1e-3 of the iterated
// residual that asked for it, since that error enters the next inner cycle's
// true residual (at small mass ||x|| is many times ||b||, and a cycle that
// reduces its residual slowly would otherwise meet the error again at every
// update); otherwise the FP64 kernels run it.
__global__ void __launch_bounds__(kBlock)
accum_x_kernel(int vh, double *__restrict__ x, float *__restrict__ xh, const float *pbuf0, const float *pbuf1,
               CgScalars *S, double *partials, unsigned int *counter) {
    __shared__ double smem[32];
    pdl_trigger();
    pdl_wait();
    const float *p = pbuf0 ? ((S->iters & 1) ? pbuf1 : pbuf0) : nullptr;
    const float alpha = p ? (float)S->alpha : 0.f;
    const bool ff = S->ru_ff != 0;  // uniform
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
        Vec3<double> xv = load_vec(x, vh, i);
        Vec3<float> hv = load_vec(xh, vh, i);
        if (p) {  // the same FP32 step the iteration would have taken
            const Vec3<float> pv = load_vec(p, vh, i);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                hv.c[a].re = fmaf(alpha, pv.c[a].re, hv.c[a].re);
                hv.c[a].im = fmaf(alpha, pv.c[a].im, hv.c[a].im);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xv.c[a].re += (double)hv.c[a].re;
            xv.c[a].im += (double)hv.c[a].im;
        }
        store_vec(x, vh, i, xv);
        if (ff) part += norm2_site(xv);
        Vec3<float> z;
#pragma unroll
        for (int a = 0; a < 3; ++a) z.c[a].re = z.c[a].im = 0.f;
        store_vec(xh, vh, i, z);
    }
    if (!ff) return;
    double xx;
    if (!grid_sum(part, partials, counter, smem, &xx)) return;
    if (!(kFfErr * kFfErr * (xx + S->bb) <= 1e-6 * S->rr_ru)) S->ru_ff = 0;
}

// End of a reliable update: r32 = (float) r64 (mixed precision only), and
// in the graph solve the loop condition from the flags the FP64 residual set.
__global__ void __launch_bounds__(kBlock)
finish_ru_kernel(int vh, const double *__restrict__ r64, float *__restrict__ r32, CgScalars *S,
                 const GraphCtl ctl) {
    pdl_trigger();
    pdl_wait();
    // nothing is pending for the iterate after a reliable update (no block
    // of this kernel reads alpha)
    if (blockIdx.x == 0 && threadIdx.x == 0) S->alpha = 0.0;
    if (r32 && !S->ru_ff) {  // a float-float update wrote r32 itself
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
            const Vec3<double> rd = load_vec(r64, vh, i);
            Vec3<float> rv;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                rv.c[a].re = (float)rd.c[a].re;
                rv.c[a].im = (float)rd.c[a].im;
            }
            store_vec(r32, vh, i, rv);
        }
    }
    if (ctl.active && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional(ctl.loop, (!S->halt && S->trips < S->maxiter + 4) ? 1u : 0u);
}

__global__ void __launch_bounds__(kBlock) any_nonzero_kernel(size_t n2, const double2 *__restrict__ f, int *flag) {
    pdl_trigger();
    pdl_wait();
    int nz = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (size_t)gridDim.x * blockDim.x) {
        const double2 v = __ldg(f + i);
        nz |= (v.x != 0.0 || v.y != 0.0) ? 1 : 0;  // NaN != 0
    }
    if (__syncthreads_or(nz) && threadIdx.x == 0) atomicOr(flag, 1);
}

template <typename R>
__global__ void __launch_bounds__(kBlock)
norm2_kernel(int vh, const R *__restrict__ f, double *out, CgScalars *S, double *partials, unsigned int *counter) {
    __shared__ double smem[32];
    pdl_trigger();
    pdl_wait();
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x)
        part += (double)norm2_site(load_vec(f, vh, i));
    double tot;
    if (!grid_sum(part, partials, counter, smem, &tot)) return;
    if (out) *out = tot;
    if (S) {
        S->bb = tot;
        S->stop2 = S->tol2 * tot;
        // float-float updates carry the vectors times 2^ff_k, about unit size a real
        int e = 0;
        if (tot > 0.0 && isfinite(tot)) frexp(sqrt(tot / (6.0 * vh)), &e);
        S->ff_k = e < -100 ? 100 : (e > 100 ? -100 : -e);
    }
}

template <typename R>
__global__ void __launch_bounds__(kBlock)
dot_kernel(int vh, const R *__restrict__ a, const R *__restrict__ b, double *out, double *partials,
           unsigned int *counter) {
    __shared__ double smem[32];
    __shared__ double re_tot;
    double pre = 0.0, pim = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
        const Vec3<R> av = load_vec(a, vh, i), bv = load_vec(b, vh, i);
        R re = R(0), im = R(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {  // conj(a) b
            re = fma(av.c[c].re, bv.c[c].re, re);
            re = fma(av.c[c].im, bv.c[c].im, re);
            im = fma(av.c[c].re, bv.c[c].im, im);
            im = fma(-av.c[c].im, bv.c[c].re, im);
        }
        pre += (double)re;
        pim += (double)im;
    }
    // two fixed-order grid sums over disjoint halves of the partials buffer
    double t0;
    unsigned int nb = gridDim.x;
    const double bre = block_sum(pre, smem);
    const double bim = block_sum(pim, smem);
    __shared__ unsigned int is_last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bre;
        partials[nb + blockIdx.x] = bim;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == nb - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    t0 = block_sum_partials(partials, nb, smem);
    if (threadIdx.x == 0) re_tot = t0;
    const double t1 = block_sum_partials(partials + nb, nb, smem);
    if (threadIdx.x != 0) return;
    *counter = 0u;
    out[0] = re_tot;
    out[1] = t1;
}

qex_status launch_update_xr(qex_lattice *lat, qex_prec prec, void *x, void *r, void *const pbuf[2], const void *ap,
                            CgScalars *S, const GraphCtl &ctl, cudaStream_t st) {
    int nb = blas_blocks(lat), vh = (int)lat->vh;
    if (prec == QEX_F64)
        launch_k(update_xr_kernel<double, true>, dim3(nb), dim3(kBlock), 0, st, lat->pdl != 0, vh, (double *)x,
                 (double *)r, (double *)pbuf[0], (double *)pbuf[1], (const double *)ap, S, lat->partials,
                 lat->counter, ctl);
    else if (x)
        launch_k(update_xr_kernel<float, true>, dim3(nb), dim3(kBlock), 0, st, lat->pdl != 0, vh, (float *)x,
                 (float *)r, (float *)pbuf[0], (float *)pbuf[1], (const float *)ap, S, lat->partials, lat->counter,
                 ctl);
    else
        launch_k(update_xr_kernel<float, false>, dim3(nb), dim3(kBlock), 0, st, lat->pdl != 0, vh, (float *)x,
                 (float *)r, (float *)pbuf[0], (float *)pbuf[1], (const float *)ap, S, lat->partials, lat->counter,
                 ctl);
    QEX_CHECK_LAUNCH("update_xr_kernel");
    return QEX_OK;
}

qex_status launch_update_p(qex_lattice *lat, qex_prec prec, const void *r, void *const pbuf[2], CgScalars *S,
                           cudaStream_t st) {
    int nb = blas_blocks(lat), vh = (int)lat->vh;
    if (prec == QEX_F64)
        launch_k(update_p_kernel<double>, dim3(nb), dim3(kBlock), 0, st, lat->pdl != 0, vh, (const double *)r,
                 (double *)pbuf[0], (double *)pbuf[1], (const CgScalars *)S);
    else
        launch_k(update_p_kernel<float>, dim3(nb), dim3(kBlock), 0, st, lat->pdl != 0, vh, (const float *)r,
                 (float *)pbuf[0], (float *)pbuf[1], (const CgScalars *)S);
    QEX_CHECK_LAUNCH("update_p_kernel");
    return QEX_OK;
}

qex_status launch_accum_x(qex_lattice *lat, double *x64, float *xh32, float *const pbuf[2], CgScalars *S,
                          cudaStream_t st) {
    launch_k(accum_x_kernel, dim3(blas_blocks(lat)), dim3(kBlock), 0, st, lat->pdl != 0, (int)lat->vh, x64, xh32,
             (const float *)(pbuf ? pbuf[0] : nullptr), (const float *)(pbuf ? pbuf[1] : nullptr), S, lat->partials,
             lat->counter);
    QEX_CHECK_LAUNCH("accum_x_kernel");
    return QEX_OK;
}

qex_status launch_finish_ru(qex_lattice *lat, const double *r64, float *r32, CgScalars *S, const GraphCtl &ctl,
                            cudaStream_t st) {
    launch_k(finish_ru_kernel, dim3(r32 ? blas_blocks(lat) : 1), dim3(kBlock), 0, st, lat->pdl != 0, (int)lat->vh, r64,
             r32, S, ctl);
    QEX_CHECK_LAUNCH("finish_ru_kernel");
    return QEX_OK;
}

qex_status launch_any_nonzero(qex_lattice *lat, const double *f, int *flag, cudaStream_t st) {
    any_nonzero_kernel<<<blas_blocks(lat), kBlock, 0, st>>>((size_t)lat->vh * 3, (const double2 *)f, flag);
    QEX_CHECK_LAUNCH("any_nonzero_kernel");
    return QEX_OK;
}

qex_status launch_norm2(qex_lattice *lat, qex_prec prec, const void *f, double *out, CgScalars *S, cudaStream_t st) {
    qex_status s = ensure_scratch(lat);
    if (s) return s;
    int nb = blas_blocks(lat), vh = (int)lat->vh;
    if (prec == QEX_F64)
        norm2_kernel<double><<<nb, kBlock, 0, st>>>(vh, (const double *)f, out, S, lat->partials, lat->counter);
    else
        norm2_kernel<float><<<nb, kBlock, 0, st>>>(vh, (const float *)f, out, S, lat->partials, lat->counter);
    QEX_CHECK_LAUNCH("norm2_kernel");
    return QEX_OK;
}

qex_status launch_dot(qex_lattice *lat, qex_prec prec, const void *a, const void *b, double *out, cudaStream_t st) {
    qex_status s = ensure_scratch(lat);
    if (s) return s;
    int nb = blas_blocks(lat), vh = (int)lat->vh;
    if (prec == QEX_F64)
        dot_kernel<double><<<nb, kBlock, 0, st>>>(vh, (const double *)a, (const double *)b, out, lat->partials,
                                                  lat->counter);
    else
        dot_kernel<float><<<nb, kBlock, 0, st>>>(vh, (const float *)a, (const float *)b, out, lat->partials,
                                                 lat->counter);
    QEX_CHECK_LAUNCH("dot_kernel");
    return QEX_OK;
}

}  // namespace qex

using namespace qex;

extern "C" {

qex_status qex_norm2(const qex_lattice *lat, qex_prec prec, const void *f, double *dev_out, void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(prec))) return st;
    if (!f || !dev_out) {
        set_error("field and dev_out must not be NULL");
        return QEX_ERR_ARG;
    }
    if (!aligned16(f)) {
        set_error("field must be 16-byte aligned");
        return QEX_ERR_ALIGN;
    }
    return launch_norm2(const_cast<qex_lattice *>(lat), prec, f, dev_out, nullptr, as_stream(stream));
}

qex_status qex_dot(const qex_lattice *lat, qex_prec prec, const void *a, const void *b, double *dev_out,
                   void *stream) {
    qex_status st;
    if ((st = check_lattice(lat)) || (st = check_prec(prec))) return st;
    if (!a || !b || !dev_out) {
        set_error("fields and dev_out must not be NULL");
        return QEX_ERR_ARG;
    }
    if (!aligned16(a) || !aligned16(b)) {
        set_error("fields must be 16-byte aligned");
        return QEX_ERR_ALIGN;
    }
    return launch_dot(const_cast<qex_lattice *>(lat), prec, a, b, dev_out, as_stream(stream));
}

}  // extern "C"
