// cg_fused.cu -- the mixed-precision CG iteration of a small lattice as one
// persistent kernel.
//
// On a small lattice (a few thousand even sites) each of the three kernels of
// an iteration does a few microseconds of work and the launch, the drain of
// the grid and the last-block reduction tail cost as much again.  Here one
// cooperative launch (every block resident) runs the inner iterations back to
// back:
//   1. tmp = D_oe (r + beta p_old) with p_new stored        grid barrier
//   2. A p_new = m^2 p_new - D_eo tmp, block sums of <p,Ap>  grid barrier
//      every block sums the block partials in the same fixed order -> alpha
//   3. x += alpha p_new, r -= alpha A p_new, block sums of ||r||^2
//                                                            grid barrier
//      every block sums them -> beta, or the request for a reliable update
// until a reliable update is due (or an error): then the kernel writes the CG
// scalars back and returns, the host runs the FP64 reliable update with the
// ordinary kernels, and launches it again.  The iterations are the ones the
// three-kernel form computes (the reductions sum the same per-site terms in
// another block grouping).
//
// Grid barriers: arrival counters (per group of 32 blocks, then across the
// groups) and a generation word, reset by the host before each launch; the
// last block to arrive bumps the generation.  A wait
// that lasts longer than a limit (clock64 cycles, about a second by default;
// the environment variable QEX_BARRIER_TIMEOUT_CYCLES sets another, which the
// tests use to make the limit run out) records a timeout in the error word
// and every block leaves at its next barrier, so a barrier can never hang the
// GPU; each block counts itself out on leaving, and the host then reports
// QEX_ERR_TIMEOUT with the count.
#include <math.h>
#include <stdlib.h>

#include "qex_dslash_site.cuh"
#include "qex_kernels.cuh"

namespace qex {

template <typename R>
struct FusedArgs {
    Geom g;
    const R *fat, *lng;
    R c3, m2;
    R *x, *r, *p0, *p1, *ap, *tmp;
    CgScalars *S;
    double *partials;            // 2 * gridDim.x
    unsigned int *bar_count;     // barrier counters: top at [0], group g at [(g + 1) * 32]
    unsigned int *bar_gen;       // barriers completed in this launch
    int *bar_err;                // nonzero: a barrier timed out
    unsigned int *exited;        // blocks that have left the kernel
    long long timeout_cycles;    // longest wait at a barrier
};

constexpr int kFusedBlock = 256;  // most threads per block (launch bounds)
#ifndef QEX_FUSED_BLOCK
#define QEX_FUSED_BLOCK 128  // threads per block of a launch (a sweep: 128 beats 256, 64, 32)
#endif
#ifndef QEX_FUSED_SPIN_NS
#define QEX_FUSED_SPIN_NS 0  // sleep between polls of a barrier (0: poll back to back)
#endif
constexpr long long kBarrierTimeoutCycles = 2000000000ll;  // default limit: about one second at 2 GHz

// Grid barrier number `gen + 1`; false if some block timed out (then every
// block leaves at its next barrier).  Two levels: a block arrives at the
// counter of its group of 32 blocks (each counter on its own 128-byte line);
// the last of a group arrives at the top counter, and the last of those bumps
// the generation.  Waiting blocks poll the generation with plain loads, so
// the arrivals' atomics meet no contention from the pollers.
constexpr int kBarrierGroup = 32;
constexpr int kBarrierStride = 32;  // unsigned words between counters (128 bytes)

__device__ __forceinline__ bool fused_barrier(unsigned int *counters, unsigned int *gen_word, int *err,
                                              unsigned int gen, long long timeout_cycles) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int grp = blockIdx.x / kBarrierGroup, ngroups = (gridDim.x + kBarrierGroup - 1) / kBarrierGroup;
        const unsigned int gsize = min((unsigned int)kBarrierGroup, gridDim.x - grp * kBarrierGroup);
        unsigned int *gc = counters + (size_t)(grp + 1) * kBarrierStride;
        bool last = false;
        if (atomicAdd(gc, 1u) == gsize - 1) {
            atomicExch(gc, 0u);
            if (atomicAdd(counters, 1u) == (unsigned int)ngroups - 1) {
                atomicExch(counters, 0u);
                __threadfence();
                atomicExch(gen_word, gen + 1);
                last = true;
            }
        }
        if (!last) {
            const volatile unsigned int *gv = gen_word;
            const volatile int *ev = err;
            const long long t0 = clock64();
            while (*gv != gen + 1) {
                if (*ev != 0) break;
                if (clock64() - t0 > timeout_cycles) {
                    atomicExch(err, 1);
                    break;
                }
                if (QEX_FUSED_SPIN_NS > 0) __nanosleep(QEX_FUSED_SPIN_NS);
            }
        }
        __threadfence();
        ok = *(const volatile int *)err == 0;
    }
    __syncthreads();
    return ok != 0;
}

// Vectors written by this kernel are read back in later phases of the same
// launch, so they are loaded through L2 (ld.global.cg), never through the
// read-only path that assumes data constant for the kernel's lifetime; only
// the links use that path.
__device__ __forceinline__ Vec3<float> load_vec_cg(const float *base, size_t vh, int i) {
    const float4 t = __ldcg(reinterpret_cast<const float4 *>(base) + i);
    const float2 u = __ldcg(reinterpret_cast<const float2 *>(base + 4 * vh) + i);
    Vec3<float> v;
    v.c[0].re = t.x;
    v.c[0].im = t.y;
    v.c[1].re = t.z;
    v.c[1].im = t.w;
    v.c[2].re = u.x;
    v.c[2].im = u.y;
    return v;
}

__device__ __forceinline__ Vec3<float> axpy_vec_cg(const float *r, const float *p, float beta, size_t vh, int j) {
    const Vec3<float> rv = load_vec_cg(r, vh, j), pv = load_vec_cg(p, vh, j);
    Vec3<float> v;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v.c[a].re = fmaf(beta, pv.c[a].re, rv.c[a].re);
        v.c[a].im = fmaf(beta, pv.c[a].im, rv.c[a].im);
    }
    return v;
}

// Sum of partials[0..n) in index order, returned to every thread of the block.
__device__ __forceinline__ double fused_total(const double *partials, int n, double *smem) {
    __shared__ double total;
    const double s = block_sum_partials(partials, n, smem);
    if (threadIdx.x == 0) total = s;
    __syncthreads();
    return total;
}

#ifndef QEX_FUSED_MIN_BLOCKS
#define QEX_FUSED_MIN_BLOCKS 2  // launch-bounds residency of 256-thread blocks (register cap)
#endif

// Loop state of the solve, identical in every block, kept in shared memory so
// that it holds no registers during the Dslash phases.
struct FusedState {
    double rr, beta, rmax2, alpha, pAp;
    double rr_ru;
    int iters, trips, need_ru, ru_ff, error;
};

template <typename R, int FMT, bool NAIK>
__device__ __forceinline__ void cg_fused_body(const FusedArgs<R> &A) {
    __shared__ double smem[32];
    __shared__ FusedState st;
    CgScalars *S = A.S;
    if (S->halt) return;  // uniform
    const Geom &g = A.g;
    const size_t vh = (size_t)g.vh;
    const int nb = gridDim.x;
    const int stride = nb * blockDim.x;
    if (threadIdx.x == 0) {
        st.rr = S->rr;
        st.beta = S->beta;
        st.rmax2 = S->rmax2;
        st.alpha = S->alpha;
        st.pAp = S->pAp;
        st.iters = S->iters;
        st.trips = S->trips;
        st.need_ru = 0;
        st.ru_ff = 0;
        st.error = 0;
    }
    __syncthreads();
    unsigned int gen = 0;
    for (;;) {
        const int it = st.iters;
        const R *pold = (it & 1) ? A.p1 : A.p0;
        R *pnew = (it & 1) ? A.p0 : A.p1;
        {   // 1. tmp = D_oe (r + beta p_old); p_new at the thread's own even index
            const R b = (R)st.beta;
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.vh; i += stride) {
                const Site s = site_of(g, 1, i);
                const Vec3<R> acc = dslash_site<R, FMT, NAIK>(g, A.fat, A.lng, A.c3, 1, i, s,
                                                              [&](int j) { return axpy_vec_cg(A.r, pold, b, vh, j); });
                store_vec(A.tmp, vh, i, acc);
                store_vec(pnew, vh, i, axpy_vec_cg(A.r, pold, b, vh, i));
            }
        }
        if (!fused_barrier(A.bar_count, A.bar_gen, A.bar_err, gen++, A.timeout_cycles)) return;
        {   // 2. A p_new = m^2 p_new - D_eo tmp; <p_new, A p_new>
            double part = 0.0;
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.vh; i += stride) {
                const Site s = site_of(g, 0, i);
                const Vec3<R> acc = dslash_site<R, FMT, NAIK>(
                    g, A.fat, A.lng, A.c3, 0, i, s, [&](int j) { return load_vec_cg(A.tmp, vh, j); });
                const Vec3<R> qv = load_vec_cg(pnew, vh, i);
                Vec3<R> o;
                R d = R(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o.c[a].re = fma(A.m2, qv.c[a].re, -acc.c[a].re);
                    o.c[a].im = fma(A.m2, qv.c[a].im, -acc.c[a].im);
                    d = fma(qv.c[a].re, o.c[a].re, d);
                    d = fma(qv.c[a].im, o.c[a].im, d);
                }
                store_vec(A.ap, vh, i, o);
                part += (double)d;
            }
            const double bs = block_sum(part, smem);
            if (threadIdx.x == 0) A.partials[blockIdx.x] = bs;
        }
        if (!fused_barrier(A.bar_count, A.bar_gen, A.bar_err, gen++, A.timeout_cycles)) return;
        {
            const double pAp = fused_total(A.partials, nb, smem);
            if (threadIdx.x == 0) {
                st.pAp = pAp;
                if (!(pAp > 0.0) || !isfinite(pAp))
                    st.error = isfinite(pAp) ? 2 : 1;
                else
                    st.alpha = st.rr / pAp;
            }
            __syncthreads();
            if (st.error) break;
        }
        {   // 3. x += alpha p_new; r -= alpha A p_new; ||r||^2
            const R al = (R)st.alpha;
            double part = 0.0;
            for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.vh; i += stride) {
                Vec3<R> xv = load_vec_cg(A.x, vh, i), rv = load_vec_cg(A.r, vh, i);
                const Vec3<R> pv = load_vec_cg(pnew, vh, i), av = load_vec_cg(A.ap, vh, i);
                R d = R(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    xv.c[a].re = fma(al, pv.c[a].re, xv.c[a].re);
                    xv.c[a].im = fma(al, pv.c[a].im, xv.c[a].im);
                    rv.c[a].re = fma(-al, av.c[a].re, rv.c[a].re);
                    rv.c[a].im = fma(-al, av.c[a].im, rv.c[a].im);
                    d = fma(rv.c[a].re, rv.c[a].re, d);
                    d = fma(rv.c[a].im, rv.c[a].im, d);
                }
                store_vec(A.x, vh, i, xv);
                store_vec(A.r, vh, i, rv);
                part += (double)d;
            }
            const double bs = block_sum(part, smem);
            if (threadIdx.x == 0) A.partials[nb + blockIdx.x] = bs;
        }
        if (!fused_barrier(A.bar_count, A.bar_gen, A.bar_err, gen++, A.timeout_cycles)) return;
        {
            const double rr_new = fused_total(A.partials + nb, nb, smem);
            if (threadIdx.x == 0) {
                st.iters += 1;
                st.trips += 1;
                if (!isfinite(rr_new)) {
                    st.error = 1;
                } else {
                    if (rr_new > st.rmax2) st.rmax2 = rr_new;
                    const bool long_cycle = S->max_cycle > 0 && st.iters - S->ru_iter0 >= S->max_cycle;
                    if (rr_new <= S->stop2 || rr_new < S->delta2 * st.rmax2 || st.iters >= S->maxiter || long_cycle) {
                        st.need_ru = 1;  // rr keeps its value: beta then comes from the true residual
                        st.ru_ff = (S->ff_ok && rr_new > S->stop2 && st.iters < S->maxiter) ? 1 : 0;
                        st.rr_ru = rr_new;
                    } else {
                        st.beta = rr_new / st.rr;
                        st.rr = rr_new;
                    }
                }
            }
            __syncthreads();
            if (st.error || st.need_ru) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S->rr = st.rr;
        S->beta = st.beta;
        S->rmax2 = st.rmax2;
        S->alpha = st.alpha;
        S->pAp = st.pAp;
        S->iters = st.iters;
        S->trips = st.trips;
        if (st.error) S->error = st.error;
        S->need_ru = st.need_ru;
        if (st.need_ru) {
            S->ru_ff = st.ru_ff;
            S->rr_ru = st.rr_ru;
        }
        S->halt = 1;
    }
}

template <typename R, int FMT, bool NAIK>
__global__ void __launch_bounds__(kFusedBlock, QEX_FUSED_MIN_BLOCKS) cg_fused_kernel(const FusedArgs<R> A) {
    cg_fused_body<R, FMT, NAIK>(A);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(A.exited, 1u);  // every way out of the body ends here
}

template <typename R, int FMT, bool NAIK>
static qex_status launch_fused_t(qex_lattice *lat, const FusedArgs<R> &A0, cudaStream_t st) {
    auto kernel = cg_fused_kernel<R, FMT, NAIK>;
    int per_sm = 0;
    const int block = QEX_FUSED_BLOCK;
    QEX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0));
    if (per_sm < 1) {
        set_error("the fused CG kernel does not fit on an SM");
        return QEX_ERR_CUDA;
    }
    const int want = blocks_for(lat->vh, block);
    const int cap = per_sm * sm_count();
    int nb = want < cap ? want : cap;
    // barrier words after the 2 nb partial sums in the lattice's partials
    // buffer: the top and group counters (128 bytes apart), then the
    // generation; the error word is counter[3] of the lattice scratch; all
    // fresh for every launch
    const int ngroups = (nb + kBarrierGroup - 1) / kBarrierGroup;
    const size_t bar_words = (size_t)(ngroups + 1) * kBarrierStride + kBarrierStride;
    const size_t need = 2 * (size_t)nb + (bar_words * sizeof(unsigned int) + sizeof(double) - 1) / sizeof(double) + 16;
    if ((size_t)lat->partials_len < need) {
        set_error("internal: partials buffer too small for the fused CG kernel");
        return QEX_ERR_ARG;
    }
    unsigned int *bar = reinterpret_cast<unsigned int *>(lat->partials + 2 * (size_t)nb + 16);
    QEX_CUDA(cudaMemsetAsync(bar, 0, bar_words * sizeof(unsigned int), st));
    QEX_CUDA(cudaMemsetAsync(lat->counter + 3, 0, 2 * sizeof(unsigned int), st));  // error word, exit count
    FusedArgs<R> A = A0;
    A.partials = lat->partials;
    A.bar_count = bar;
    A.bar_gen = bar + (size_t)(ngroups + 1) * kBarrierStride;
    A.bar_err = reinterpret_cast<int *>(lat->counter + 3);
    A.exited = lat->counter + 4;
    A.timeout_cycles = kBarrierTimeoutCycles;
    if (const char *e = getenv("QEX_BARRIER_TIMEOUT_CYCLES")) {
        const long long v = atoll(e);
        if (v > 0) A.timeout_cycles = v;
    }
    lat->fused_blocks = nb;
    void *args[] = {&A};
    QEX_CUDA(cudaLaunchCooperativeKernel((const void *)kernel, dim3(nb), dim3(block), args, 0, st));
    note_launch();
    return QEX_OK;
}

template <int FMT>
static qex_status launch_fused_n(qex_lattice *lat, const FusedArgs<float> &A, bool naik, cudaStream_t st) {
    return naik ? launch_fused_t<float, FMT, true>(lat, A, st) : launch_fused_t<float, FMT, false>(lat, A, st);
}

// One run of the fused iteration kernel (mixed precision only).
qex_status launch_cg_fused(qex_lattice *lat, qex_prec inner, const void *fat32, const void *lng32, double c3, double m2,
                           float *x, float *r, float *const p[2], float *ap, float *tmp, cudaStream_t st) {
    FusedArgs<float> A = {};
    A.g = lat->geom;
    A.fat = (const float *)fat32;
    A.lng = (const float *)lng32;
    A.c3 = (float)c3;
    A.m2 = (float)m2;
    A.x = x;
    A.r = r;
    A.p0 = p[0];
    A.p1 = p[1];
    A.ap = ap;
    A.tmp = tmp;
    A.S = lat->scalars;
    const bool naik = lng32 != nullptr;
    switch (inner) {
        case QEX_F32: return launch_fused_n<0>(lat, A, naik, st);
        case QEX_F32_R12: return launch_fused_n<1>(lat, A, naik, st);
        case QEX_F32_R12H: return launch_fused_n<2>(lat, A, naik, st);
        case QEX_F32_S16: return launch_fused_n<3>(lat, A, naik, st);
        default: set_error("the fused CG iteration is for mixed precision only"); return QEX_ERR_ARG;
    }
}

// Whether a barrier of the last fused run timed out (reads the error word),
// and how many of its blocks left the kernel.
qex_status fused_barrier_status(qex_lattice *lat, cudaStream_t st, int *timed_out, int *exited) {
    unsigned int v[2] = {0u, 0u};
    QEX_CUDA(cudaMemcpyAsync(v, lat->counter + 3, sizeof(v), cudaMemcpyDeviceToHost, st));
    QEX_CUDA(cudaStreamSynchronize(st));
    *timed_out = v[0] != 0;
    if (exited) *exited = (int)v[1];
    return QEX_OK;
}

}  // namespace qex
