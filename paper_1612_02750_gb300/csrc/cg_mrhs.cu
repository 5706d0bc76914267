// cg_mrhs.cu -- conjugate gradient on A = m^2 - D_eo D_oe for N right-hand
// sides at once (FP64, or FP32 inner with FP64 reliable updates).
//
// The N solves share every operator application (qex_dslash_mrhs reads each
// link once for all of them) and keep their own alpha, beta and residual
// norms.  They iterate in lockstep; a right-hand side whose FP64 true
// residual meets tol is frozen (its `active` flag drops) while the others go
// on.  A reliable update, requested by any active right-hand side, is done
// for all active ones: x += x_hat, r = b - A x in FP64, r_hat = (float) r,
// beta_r = ||r||^2 / rr_r with the previous iterated norm.  An iteration is
// three kernels (fused direction update + D_oe, normal operator with the
// per-RHS <p, Ap>, x/r update with the per-RHS norms); the host enqueues them
// in batches and reads the scalars once per batch.
#include <math.h>
#include <string.h>

#include "qex_kernels.cuh"

namespace qex {

qex_status check_dslash_args(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                             const void *in, const void *out);

// blockIdx.y = right-hand side.  x += alpha p_new; r -= alpha ap; ||r||^2;
// then, in the last block, the lockstep decision: if any active right-hand
// side asks for a reliable update (or the cap is reached), nobody advances
// rr/beta and the reliable update takes over; otherwise each advances.
template <typename R>
__global__ void __launch_bounds__(kBlock)
update_xr_mrhs_kernel(int vh, int nrhs, R *__restrict__ x, R *__restrict__ r, R *pbuf0, R *pbuf1,
                      const R *__restrict__ ap, MrhsScalars *S, double *partials, unsigned int *counter) {
    __shared__ double smem[32];
    __shared__ unsigned int is_last;
    __shared__ double rr_new[kMaxRhs];
    __shared__ int any_ru;
    if (S->halt) return;  // uniform
    const int rh = blockIdx.y;
    const size_t off = (size_t)rh * 6 * vh;
    double part = 0.0;
    if (S->active[rh]) {
        const R alpha = (R)S->alpha[rh];
        const R *p = ((S->iter & 1) ? pbuf0 : pbuf1) + off;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
            Vec3<R> xv = load_vec(x + off, vh, i), rv = load_vec(r + off, vh, i);
            const Vec3<R> pv = load_vec(p, vh, i), av = load_vec(ap + off, vh, i);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xv.c[a].re = fma(alpha, pv.c[a].re, xv.c[a].re);
                xv.c[a].im = fma(alpha, pv.c[a].im, xv.c[a].im);
                rv.c[a].re = fma(-alpha, av.c[a].re, rv.c[a].re);
                rv.c[a].im = fma(-alpha, av.c[a].im, rv.c[a].im);
                part += (double)(rv.c[a].re * rv.c[a].re + rv.c[a].im * rv.c[a].im);
            }
            store_vec(x + off, vh, i, xv);
            store_vec(r + off, vh, i, rv);
        }
    }
    const double bs = block_sum(part, smem);
    if (threadIdx.x == 0) {
        partials[(size_t)rh * gridDim.x + blockIdx.x] = bs;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x * gridDim.y - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (threadIdx.x == 0) any_ru = 0;
    __syncthreads();
    // one warp per right-hand side, fixed order over the blocks
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < nrhs; q += nw) {
        double v = 0.0;
        for (int bx = lane; bx < (int)gridDim.x; bx += 32) v += __ldcg(partials + (size_t)q * gridDim.x + bx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
            rr_new[q] = v;
            if (S->active[q]) {
                S->iters[q] += 1;
                if (!isfinite(v)) {
                    S->error = 1;
                    atomicOr(&any_ru, 1);
                } else {
                    if (v > S->rmax2[q]) S->rmax2[q] = v;
                    if (v <= S->stop2[q] || v < S->delta2 * S->rmax2[q]) atomicOr(&any_ru, 1);
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        S->iter += 1;
        *counter = 0u;
        if (S->error) {
            S->halt = 1;
        } else if (any_ru || S->iter >= S->maxiter ||
                   (S->max_cycle > 0 && S->iter - S->ru_iter0 >= S->max_cycle)) {
            S->need_ru = 1;
            S->halt = 1;
        } else {
            for (int q = 0; q < nrhs; ++q)
                if (S->active[q]) {
                    S->beta[q] = rr_new[q] / S->rr[q];
                    S->rr[q] = rr_new[q];
                }
        }
    }
}

// blockIdx.y = right-hand side: x64 += xh32, xh32 = 0 (active ones).
__global__ void __launch_bounds__(kBlock)
accum_x_mrhs_kernel(int vh, double *__restrict__ x, float *__restrict__ xh, const MrhsScalars *S) {
    const int rh = blockIdx.y;
    if (!S->active[rh]) return;
    const size_t off = (size_t)rh * 6 * vh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
        Vec3<double> xv = load_vec(x + off, vh, i);
        const Vec3<float> hv = load_vec(xh + off, vh, i);
        Vec3<float> z;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xv.c[a].re += (double)hv.c[a].re;
            xv.c[a].im += (double)hv.c[a].im;
            z.c[a].re = z.c[a].im = 0.f;
        }
        store_vec(x + off, vh, i, xv);
        store_vec(xh + off, vh, i, z);
    }
}

// blockIdx.y = right-hand side: r32 = (float) r64 (active ones).
__global__ void __launch_bounds__(kBlock)
lower_r_mrhs_kernel(int vh, const double *__restrict__ r64, float *__restrict__ r32, const MrhsScalars *S) {
    const int rh = blockIdx.y;
    if (!S->active[rh]) return;
    const size_t off = (size_t)rh * 6 * vh;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
        const Vec3<double> rd = load_vec(r64 + off, vh, i);
        Vec3<float> rv;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            rv.c[a].re = (float)rd.c[a].re;
            rv.c[a].im = (float)rd.c[a].im;
        }
        store_vec(r32 + off, vh, i, rv);
    }
}

// blockIdx.y = right-hand side: ||b_r||^2 -> bb, stop2; zero sources are
// solved at once (x = 0, done).
__global__ void __launch_bounds__(kBlock)
norm2_mrhs_kernel(int vh, int nrhs, const double *__restrict__ b, double *__restrict__ x, MrhsScalars *S,
                  double *partials, unsigned int *counter) {
    __shared__ double smem[32];
    __shared__ unsigned int is_last;
    const int rh = blockIdx.y;
    const size_t off = (size_t)rh * 6 * vh;
    double part = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < vh; i += gridDim.x * blockDim.x) {
        const Vec3<double> v = load_vec(b + off, vh, i);
#pragma unroll
        for (int a = 0; a < 3; ++a) part += v.c[a].re * v.c[a].re + v.c[a].im * v.c[a].im;
    }
    const double bs = block_sum(part, smem);
    if (threadIdx.x == 0) {
        partials[(size_t)rh * gridDim.x + blockIdx.x] = bs;
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x * gridDim.y - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = warp; q < nrhs; q += nw) {
        double v = 0.0;
        for (int bx = lane; bx < (int)gridDim.x; bx += 32) v += __ldcg(partials + (size_t)q * gridDim.x + bx);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
            S->bb[q] = v;
            S->stop2[q] = S->tol2 * v;
            if (!isfinite(v)) S->error = 1;
            if (v == 0.0) {  // zero source: x = 0 is exact
                S->active[q] = 0;
                S->done[q] = 1;
            }
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

static size_t align256m(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace qex

using namespace qex;

extern "C" qex_status qex_cg_mrhs(const qex_lattice *latc, qex_prec inner, const void *fat64, const void *lng64,
                                  const void *fat32, const void *lng32, double c_naik, double mass, int nrhs,
                                  const void *b64, void *x64, double tol, int maxiter, double delta, void *stream,
                                  qex_cg_stats *stats) {
    qex_status st;
    if ((st = check_lattice(latc)) || (st = check_prec(inner))) return st;
    if ((st = check_dslash_args(latc, QEX_F64, fat64, lng64, b64, x64))) return st;
    if (nrhs < 1 || nrhs > QEX_MRHS_MAX) {
        set_error("nrhs must be in [1, %d] (got %d)", QEX_MRHS_MAX, nrhs);
        return QEX_ERR_ARG;
    }
    const bool mixed = inner != QEX_F64;
    if (mixed && (!fat32 || !aligned16(fat32) || (lng64 && (!lng32 || !aligned16(lng32))))) {
        set_error("mixed precision needs aligned FP32 copies of the fat (and long) links");
        return QEX_ERR_ARG;
    }
    if (!(tol > 0.0) || maxiter < 0 || !(delta >= 0.0 && delta < 1.0)) {
        set_error("need tol > 0, maxiter >= 0 and 0 <= delta < 1");
        return QEX_ERR_ARG;
    }
    qex_lattice *lat = const_cast<qex_lattice *>(latc);
    if ((st = ensure_scratch(lat))) return st;
    const cudaStream_t s = as_stream(stream);
    const int vh = (int)lat->vh;
    // nrhs fields back to back, 6*vh reals apart (16-byte aligned: vh is even)
    const size_t f64 = align256m((size_t)vh * 48 * nrhs), f32 = align256m((size_t)vh * 24 * nrhs);
    // work: r64, tmp64 (+ p64 x2, ap64 in FP64 mode) | xh, r, p x2, ap, tmp (FP32 mode); scalars
    const size_t need = (mixed ? 2 * f64 + 6 * f32 : 5 * f64) + align256m(sizeof(MrhsScalars));
    if ((st = ensure_work(lat, need))) return st;
    char *w = (char *)lat->work;
    double *r64 = (double *)w;
    w += f64;
    double *tmp64 = (double *)w;
    w += f64;
    void *xi, *ri, *pb[2], *api, *tmpi;
    const size_t fi = mixed ? f32 : f64;
    if (mixed) {
        xi = w;
        w += fi;
        ri = w;
        w += fi;
    } else {
        xi = x64;
        ri = r64;
    }
    pb[0] = w;
    w += fi;
    pb[1] = w;
    w += fi;
    api = w;
    w += fi;
    if (mixed) {
        tmpi = w;
        w += fi;
    } else {
        tmpi = tmp64;
    }
    MrhsScalars *S = (MrhsScalars *)w;

    MrhsScalars init;
    memset(&init, 0, sizeof(init));
    init.nrhs = nrhs;
    init.tol2 = tol * tol;
    init.delta2 = mixed ? delta * delta : 0.0;
    init.max_cycle = ru_max_cycle(inner);
    init.maxiter = maxiter;
    for (int q = 0; q < nrhs; ++q) init.active[q] = 1;
    MrhsScalars *host = nullptr;
    QEX_CUDA(cudaMallocHost(&host, sizeof(MrhsScalars)));
    *host = init;
    cudaEvent_t t0, t1;
    QEX_CUDA(cudaEventCreate(&t0));
    QEX_CUDA(cudaEventCreate(&t1));
    QEX_CUDA(cudaEventRecord(t0, s));
    QEX_CUDA(cudaMemcpyAsync(S, host, sizeof(MrhsScalars), cudaMemcpyHostToDevice, s));
    const size_t fbytes = (size_t)nrhs * vh * (mixed ? 24 : 48);
    QEX_CUDA(cudaMemsetAsync(pb[0], 0, fbytes, s));
    QEX_CUDA(cudaMemsetAsync(pb[1], 0, fbytes, s));
    if (mixed) QEX_CUDA(cudaMemsetAsync(xi, 0, fbytes, s));
    const int nbb = blas_blocks(lat);
    dim3 bgrid(nbb, nrhs);
    norm2_mrhs_kernel<<<bgrid, kBlock, 0, s>>>(vh, nrhs, (const double *)b64, (double *)x64, S, lat->partials,
                                               lat->counter);
    QEX_CHECK_LAUNCH("norm2_mrhs_kernel");

    MrhsArgs a = {};
    a.nrhs = nrhs;
    a.c3 = c_naik;
    a.m2 = mass * mass;
    a.S = S;
    auto reliable_update = [&]() -> qex_status {
        if (mixed) {
            accum_x_mrhs_kernel<<<bgrid, kBlock, 0, s>>>(vh, (double *)x64, (float *)xi, S);
            QEX_CHECK_LAUNCH("accum_x_mrhs_kernel");
        }
        MrhsArgs d = a;
        d.prec = QEX_F64;
        d.fat = fat64;
        d.lng = lng64;
        d.out_parity = 1;
        d.in = x64;
        d.out = tmp64;
        d.epi = EPI_PLAIN;
        MrhsScalars *keep = d.S;
        d.S = nullptr;  // plain application over all fields (frozen ones are harmless)
        qex_status e;
        if ((e = launch_dslash_mrhs(lat, d, s))) return e;
        d.S = keep;
        d.out_parity = 0;
        d.in = tmp64;
        d.out = r64;
        d.epi = EPI_RESID;
        d.q = x64;
        d.b = (const double *)b64;
        if ((e = launch_dslash_mrhs(lat, d, s))) return e;
        if (mixed) {
            lower_r_mrhs_kernel<<<bgrid, kBlock, 0, s>>>(vh, r64, (float *)ri, S);
            QEX_CHECK_LAUNCH("lower_r_mrhs_kernel");
        }
        return QEX_OK;
    };
    auto iteration = [&]() -> qex_status {
        MrhsArgs d = a;
        d.prec = inner;
        d.fat = mixed ? fat32 : fat64;
        d.lng = mixed ? lng32 : lng64;
        d.pbuf[0] = pb[0];
        d.pbuf[1] = pb[1];
        d.out_parity = 1;
        d.r = ri;
        d.out = tmpi;
        d.epi = EPI_PUPD;
        qex_status e;
        if ((e = launch_dslash_mrhs(lat, d, s))) return e;
        d.out_parity = 0;
        d.in = tmpi;
        d.out = api;
        d.epi = EPI_NORMAL;
        if ((e = launch_dslash_mrhs(lat, d, s))) return e;
        if (mixed)
            update_xr_mrhs_kernel<float><<<bgrid, kBlock, 0, s>>>(vh, nrhs, (float *)xi, (float *)ri, (float *)pb[0],
                                                                  (float *)pb[1], (const float *)api, S,
                                                                  lat->partials, lat->counter);
        else
            update_xr_mrhs_kernel<double><<<bgrid, kBlock, 0, s>>>(vh, nrhs, (double *)xi, (double *)ri,
                                                                   (double *)pb[0], (double *)pb[1],
                                                                   (const double *)api, S, lat->partials,
                                                                   lat->counter);
        QEX_CHECK_LAUNCH("update_xr_mrhs_kernel");
        return QEX_OK;
    };
    auto fetch = [&]() -> qex_status {
        QEX_CUDA(cudaMemcpyAsync(host, S, sizeof(MrhsScalars), cudaMemcpyDeviceToHost, s));
        QEX_CUDA(cudaStreamSynchronize(s));
        return QEX_OK;
    };

    qex_status result = QEX_OK;
    if ((st = reliable_update()) || (st = fetch())) {
        cudaFreeHost(host);
        return st;
    }
    // zero sources: x = 0 exactly
    for (int q = 0; q < nrhs; ++q)
        if (host->bb[q] == 0.0) QEX_CUDA(cudaMemsetAsync((double *)x64 + (size_t)q * 6 * vh, 0, (size_t)vh * 48, s));
    const int batch = 8;
    while (!host->error && !host->halt) {
        for (int k = 0; k < batch; ++k)
            if ((st = iteration())) break;
        if (st || (st = fetch())) break;
        if (host->error || !host->need_ru) continue;
        if ((st = reliable_update()) || (st = fetch())) break;
    }
    QEX_CUDA(cudaEventRecord(t1, s));
    QEX_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (!st) {
        int all = 1;
        for (int q = 0; q < nrhs; ++q) all &= host->done[q];
        if (host->error) {
            set_error("NaN/Inf or CG breakdown in a multi-RHS solve");
            result = QEX_ERR_NAN;
        } else if (!all) {
            set_error("multi-RHS CG did not converge in %d iterations", maxiter);
            result = QEX_ERR_NOT_CONVERGED;
        }
        if (stats) {
            for (int q = 0; q < nrhs; ++q) {
                stats[q].iters = host->iters[q];
                stats[q].reliable_updates = host->reliable_updates > 0 ? host->reliable_updates - 1 : 0;
                stats[q].converged = host->done[q];
                stats[q].ff_updates = 0;
                stats[q].true_rel_resid = host->bb[q] > 0.0 ? sqrt(host->true_rr[q] / host->bb[q]) : 0.0;
                stats[q].time_ms = ms;
            }
        }
    } else {
        result = st;
    }
    cudaFreeHost(host);
    return result;
}
