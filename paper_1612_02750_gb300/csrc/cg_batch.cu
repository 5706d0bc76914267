// cg_batch.cu -- conjugate gradient on many independent lattices at once
// (different extents, masses and links), every launch covering a work list of
// (lattice, tile) items.
//
// Small lattices cannot fill the GPU on their own; batching them makes every
// kernel of an iteration one launch over the tiles of all running lattices.
// Each lattice keeps its own alpha, beta, norms and reliable-update state;
// the lattices iterate in lockstep (the lockstep count's parity selects the
// direction buffers).  The iteration kernels run a persistent grid over a
// device-resident list of the running lattices' tiles, which the reliable
// update recompacts whenever a lattice meets its FP64 true residual, so a
// finished lattice costs nothing afterwards.  A tile is `spt` groups of 256
// consecutive even-odd sites of one lattice (256 threads, one site per thread
// and group), and the persistent grid has `per_sm` resident blocks per SM;
// both are chosen per set of extents by timing the iteration's Dslash
// kernels at the start of the solve (or pinned, qex_cg_batch_tune_set).
// Reductions are per 256-site group, summed per lattice in group order by the
// last block, so the result is bit-identical for every shape.  By
// default the loop is one CUDA graph: a conditional WHILE node around the
// three iteration kernels and a conditional IF node holding the reliable
// update of the lattices that asked for one; QEX_CG_MODE=host drives the same
// kernels from the host in batches.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "qex_dslash_site.cuh"
#include "qex_kernels.cuh"

namespace qex {

constexpr int kTile = 256;  // sites per group (threads per block)
constexpr int kBatchMinBlocks = 3;  // resident blocks per SM of the iteration kernels (no spills at 85 registers)
constexpr int kMaxSpt = 4;          // groups per work item

struct LatDesc {
    Geom g;
    int tile0, ntiles;  // 256-site groups: first in the full group list, count
    const void *fat_in, *lng_in;  // inner-precision links
    const double *fat64, *lng64;
    const double *b;
    double *x64, *r64, *tmp64;
    void *xi, *ri, *p0, *p1, *api, *tmpi;  // inner-precision CG vectors
    double m2, c3;
};

struct BatchScalars {
    double rr[kMaxRhs], pAp[kMaxRhs], alpha[kMaxRhs], beta[kMaxRhs], bb[kMaxRhs], stop2[kMaxRhs],
        rmax2[kMaxRhs], true_rr[kMaxRhs];
    int active[kMaxRhs], done[kMaxRhs], need[kMaxRhs], iters[kMaxRhs];
    int alist[kMaxRhs];       // running lattices, in lattice order
    int astart[kMaxRhs + 1];  // their first group in the compacted group list; astart[nlist] = groups
    int bstart[kMaxRhs + 1];  // their first work item (spt groups) in the compacted list
    int ru_iter0[kMaxRhs];    // iters[l] at lattice l's last reliable update
    int spt;                  // groups per work item
    int nlist;
    int max_cycle;            // > 0: a reliable update also follows max_cycle iterations without one
    double tol2, delta2;
    int n, iter, maxiter, halt, error, any_need, nactive, reliable_updates, trips;
    int idle_iters;  // iterations whose update kernel found the batch halted
};

enum BatchRole {
    ROLE_K1 = 0,   // tmp = D_oe (r + beta p_old), p_new stored          (inner, running lattices)
    ROLE_K2 = 1,   // ap = m^2 p_new - D_eo tmp, <p_new, ap> -> alpha    (inner, running lattices)
    ROLE_RU1 = 2,  // tmp64 = D_oe x64                                   (FP64, lattices in a reliable update)
    ROLE_RU2 = 3   // r64 = b - m^2 x64 + D_eo tmp64, ||r64||^2 -> flags (FP64, lattices in a reliable update)
};

// Last index k with start[k] <= t (start sorted, start[0] = 0).
__device__ __forceinline__ int find_start(const int *start, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int lattice_of_full_tile(const LatDesc *d, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (d[mid].tile0 <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Rebuild the running-lattice list from the active flags (one thread).
__device__ __forceinline__ void compact_list(BatchScalars *S, const LatDesc *d, int n) {
    int k = 0, t = 0, w = 0;
    for (int l = 0; l < n; ++l)
        if (S->active[l]) {
            S->alist[k] = l;
            S->astart[k] = t;
            S->bstart[k] = w;
            t += d[l].ntiles;
            w += (d[l].ntiles + S->spt - 1) / S->spt;
            ++k;
        }
    S->nlist = k;
    S->astart[k] = t;
    S->bstart[k] = w;
}

__device__ __forceinline__ void set_conds(const GraphCtl &ctl, unsigned int loop, unsigned int ru) {
    if (ctl.active) {
        cudaGraphSetConditional(ctl.loop, loop);
        cudaGraphSetConditional(ctl.ru, ru);
    }
}

// After the per-tile partials of this launch are written: the last of the
// nblocks participating blocks sums each listed lattice's tiles in order
// (one warp per lattice) into tot[].
__device__ __forceinline__ bool last_block_totals(double *partials, unsigned int *counter, int nl, const int *start,
                                                  double *tot, unsigned int nblocks) {
    __shared__ unsigned int is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == nblocks - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < nl; k += nw) {
        double v = 0.0;
        for (int j = start[k] + lane; j < start[k + 1]; j += 32) v += __ldcg(partials + j);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) tot[k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

// Iteration Dslash kernels: persistent grid over the compacted tile list.
template <typename R, int FMT, bool NAIK, int ROLE>
__global__ void __launch_bounds__(kTile, kBatchMinBlocks)
batch_iter_dslash_kernel(const LatDesc *__restrict__ descs, BatchScalars *S, double *partials, unsigned int *counter) {
    __shared__ double smem[32];
    __shared__ double tot[kMaxRhs];
    if (S->halt) return;  // uniform over the grid
    const int nl = S->nlist;
    const int nitems = S->bstart[nl];
    const int spt = S->spt;
    const int it = S->iter;
    // blocks beyond the running work items leave at once (the last running
    // lattice can be a few items against a grid sized for all of them)
    const unsigned int nblk = nitems < (int)gridDim.x ? (unsigned int)nitems : gridDim.x;
    if (blockIdx.x >= nblk) return;
    for (int w = blockIdx.x; w < nitems; w += gridDim.x)
    for (int q = 0; q < spt; ++q) {
        const int k = find_start(S->bstart, nl, w);
        const int l = S->alist[k];
        const LatDesc &D = descs[l];
        const int grp = (w - S->bstart[k]) * spt + q;  // group within the lattice
        if (grp >= D.ntiles) break;                     // uniform over the block
        const int t = S->astart[k] + grp;               // group in the compacted list
        const Geom &g = D.g;
        const size_t vh = (size_t)g.vh;
        const int i = grp * kTile + threadIdx.x;
        const R *pold = (const R *)((it & 1) ? D.p1 : D.p0);
        R *pnew = (R *)((it & 1) ? D.p0 : D.p1);
        double part = 0.0;
        if (i < g.vh) {
            if constexpr (ROLE == ROLE_K1) {
                const Site s = site_of(g, 1, i);
                const R beta = (R)S->beta[l];
                const R *r = (const R *)D.ri;
                const Vec3<R> acc = dslash_site<R, FMT, NAIK>(g, (const R *)D.fat_in, (const R *)D.lng_in, (R)D.c3, 1,
                                                              i, s, [&](int j) { return axpy_vec(r, pold, beta, vh, j); });
                store_vec((R *)D.tmpi, vh, i, acc);
                store_vec(pnew, vh, i, axpy_vec(r, pold, beta, vh, i));
            } else {
                const Site s = site_of(g, 0, i);
                const R *tmp = (const R *)D.tmpi;
                const Vec3<R> acc = dslash_site<R, FMT, NAIK>(g, (const R *)D.fat_in, (const R *)D.lng_in, (R)D.c3, 0,
                                                              i, s, [&](int j) { return load_vec(tmp, vh, j); });
                const Vec3<R> qv = load_vec((const R *)pnew, vh, i);
                const R m2 = (R)D.m2;
                Vec3<R> o;
                R dd = R(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    o.c[a].re = fma(m2, qv.c[a].re, -acc.c[a].re);
                    o.c[a].im = fma(m2, qv.c[a].im, -acc.c[a].im);
                    dd = fma(qv.c[a].re, o.c[a].re, dd);
                    dd = fma(qv.c[a].im, o.c[a].im, dd);
                }
                store_vec((R *)D.api, vh, i, o);
                part = (double)dd;
            }
        }
        if constexpr (ROLE == ROLE_K2) {
            const double bs = block_sum(part, smem);
            if (threadIdx.x == 0) partials[t] = bs;
        }
    }
    if constexpr (ROLE == ROLE_K2) {
        if (!last_block_totals(partials, counter, nl, S->astart, tot, nblk)) return;
        if (threadIdx.x != 0) return;
        for (int k = 0; k < nl; ++k) {
            const int l = S->alist[k];
            const double v = tot[k];
            S->pAp[l] = v;
            if (!(v > 0.0) || !isfinite(v)) {
                S->error = isfinite(v) ? 2 : 1;
                S->halt = 1;
            } else {
                S->alpha[l] = S->rr[l] / v;
            }
        }
    }
}

// x += alpha p_new; r -= alpha ap; ||r||^2 per lattice, then the decisions
// and, in the graph solve, the loop and reliable-update conditions.
template <typename R>
__global__ void __launch_bounds__(kTile)
batch_update_kernel(const LatDesc *__restrict__ descs, BatchScalars *S, double *partials, unsigned int *counter,
                    const GraphCtl ctl) {
    __shared__ double smem[32];
    __shared__ double tot[kMaxRhs];
    if (S->halt) {
        // an earlier iteration of the same graph trip asked for a reliable
        // update (keep its conditions) or the batch stopped (end the loop)
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned int ru = (S->any_need && !S->error) ? 1u : 0u;
            set_conds(ctl, ru, ru);
            S->idle_iters += 1;
        }
        return;
    }
    // fail-safe: stop unless the last block sets the conditions again
    if (blockIdx.x == 0 && threadIdx.x == 0) set_conds(ctl, 0u, 0u);
    const int nl = S->nlist;
    const int nitems = S->bstart[nl];
    const int spt = S->spt;
    const unsigned int nblk = nitems < (int)gridDim.x ? (unsigned int)nitems : gridDim.x;
    if (blockIdx.x >= nblk) return;  // a running list is never empty here (an empty one halts)
    for (int w = blockIdx.x; w < nitems; w += gridDim.x)
    for (int q = 0; q < spt; ++q) {
        const int k = find_start(S->bstart, nl, w);
        const int l = S->alist[k];
        const LatDesc &D = descs[l];
        const int grp = (w - S->bstart[k]) * spt + q;
        if (grp >= D.ntiles) break;  // uniform over the block
        const int t = S->astart[k] + grp;
        const size_t vh = (size_t)D.g.vh;
        const int i = grp * kTile + threadIdx.x;
        double part = 0.0;
        if (i < D.g.vh) {
            const R alpha = (R)S->alpha[l];
            const R *p = (const R *)((S->iter & 1) ? D.p0 : D.p1);
            R *x = (R *)D.xi, *r = (R *)D.ri;
            Vec3<R> xv = load_vec(x, vh, i), rv = load_vec(r, vh, i);
            const Vec3<R> pv = load_vec(p, vh, i), av = load_vec((const R *)D.api, vh, i);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xv.c[a].re = fma(alpha, pv.c[a].re, xv.c[a].re);
                xv.c[a].im = fma(alpha, pv.c[a].im, xv.c[a].im);
                rv.c[a].re = fma(-alpha, av.c[a].re, rv.c[a].re);
                rv.c[a].im = fma(-alpha, av.c[a].im, rv.c[a].im);
                part += (double)(rv.c[a].re * rv.c[a].re + rv.c[a].im * rv.c[a].im);
            }
            store_vec(x, vh, i, xv);
            store_vec(r, vh, i, rv);
        }
        const double bs = block_sum(part, smem);
        if (threadIdx.x == 0) partials[t] = bs;
    }
    if (!last_block_totals(partials, counter, nl, S->astart, tot, nblk)) return;
    if (threadIdx.x != 0) return;
    S->iter += 1;
    S->trips += 1;
    int any = 0;
    for (int k = 0; k < nl; ++k) {
        const int l = S->alist[k];
        const double v = tot[k];
        S->iters[l] += 1;
        if (!isfinite(v)) {
            S->error = 1;
            continue;
        }
        if (v > S->rmax2[l]) S->rmax2[l] = v;
        if (v <= S->stop2[l] || v < S->delta2 * S->rmax2[l] || S->iter >= S->maxiter ||
            (S->max_cycle > 0 && S->iters[l] - S->ru_iter0[l] >= S->max_cycle)) {
            S->need[l] = 1;  // rr keeps its old value: beta comes from the true residual
            any = 1;
        } else {
            S->beta[l] = v / S->rr[l];
            S->rr[l] = v;
        }
    }
    S->any_need = any;
    S->halt = (any || S->error) ? 1 : 0;
    const unsigned int go = (!S->error && S->trips < S->maxiter + 4) ? 1u : 0u;
    set_conds(ctl, go, (go && any) ? 1u : 0u);
}

// Reliable update, FP64 Dslash over the full tile list (lattices with need set).
template <bool NAIK, int ROLE>
__global__ void __launch_bounds__(kTile, 3)
batch_ru_dslash_kernel(const LatDesc *__restrict__ descs, int n, BatchScalars *S, const int *need, double *partials,
                       unsigned int *counter) {
    __shared__ double smem[32];
    __shared__ double tot[kMaxRhs];
    __shared__ int ident[kMaxRhs + 1];
    const int l = lattice_of_full_tile(descs, n, blockIdx.x);
    const LatDesc &D = descs[l];
    const Geom &g = D.g;
    const size_t vh = (size_t)g.vh;
    const int i = (blockIdx.x - D.tile0) * kTile + threadIdx.x;
    double part = 0.0;
    if (need[l] && i < g.vh) {
        if constexpr (ROLE == ROLE_RU1) {
            const Site s = site_of(g, 1, i);
            const double *x = D.x64;
            store_vec(D.tmp64, vh, i, dslash_site<double, 0, NAIK>(g, D.fat64, D.lng64, D.c3, 1, i, s,
                                                                   [&](int j) { return load_vec(x, vh, j); }));
        } else {
            const Site s = site_of(g, 0, i);
            const double *tmp = D.tmp64;
            const Vec3<double> acc = dslash_site<double, 0, NAIK>(g, D.fat64, D.lng64, D.c3, 0, i, s,
                                                                  [&](int j) { return load_vec(tmp, vh, j); });
            const Vec3<double> xv = load_vec(D.x64, vh, i), bv = load_vec(D.b, vh, i);
            Vec3<double> o;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                o.c[a].re = bv.c[a].re - fma(D.m2, xv.c[a].re, -acc.c[a].re);
                o.c[a].im = bv.c[a].im - fma(D.m2, xv.c[a].im, -acc.c[a].im);
                part = fma(o.c[a].re, o.c[a].re, part);
                part = fma(o.c[a].im, o.c[a].im, part);
            }
            store_vec(D.r64, vh, i, o);
        }
    }
    if constexpr (ROLE == ROLE_RU2) {
        const double bs = block_sum(part, smem);
        if (threadIdx.x == 0) partials[blockIdx.x] = bs;
        if (threadIdx.x == 0)  // per-lattice tile ranges of the full list
            for (int k = 0; k <= n; ++k) ident[k] = k < n ? descs[k].tile0 : descs[n - 1].tile0 + descs[n - 1].ntiles;
        if (!last_block_totals(partials, counter, n, ident, tot, gridDim.x)) return;
        if (threadIdx.x != 0) return;
        for (int k = 0; k < n; ++k) {
            if (!need[k] || !S->need[k]) continue;
            const double v = tot[k];
            S->need[k] = 0;
            S->ru_iter0[k] = S->iters[k];
            S->true_rr[k] = v;
            if (!isfinite(v)) {
                S->error = 1;
                continue;
            }
            S->beta[k] = S->rr[k] > 0.0 ? v / S->rr[k] : 0.0;
            S->rr[k] = v;
            S->rmax2[k] = v;
            if (v <= S->stop2[k]) {
                S->done[k] = 1;
                S->active[k] = 0;
            }
        }
        compact_list(S, descs, n);
        S->nactive = S->nlist;
        S->any_need = 0;
        S->reliable_updates += 1;
        S->halt = (S->nlist == 0 || S->iter >= S->maxiter || S->error) ? 1 : 0;
    }
}

// Reliable-update vector steps over the full tile list (lattices in `need`):
// x64 += xh, xh = 0 before the FP64 residual; r_inner = (float) r64 after it.
template <int STEP>
__global__ void __launch_bounds__(kTile)
batch_ru_vectors_kernel(const LatDesc *__restrict__ descs, int n, const int *need) {
    const int l = lattice_of_full_tile(descs, n, blockIdx.x);
    if (!need[l]) return;
    const LatDesc &D = descs[l];
    const size_t vh = (size_t)D.g.vh;
    const int i = (blockIdx.x - D.tile0) * kTile + threadIdx.x;
    if (i >= D.g.vh) return;
    if (STEP == 0) {
        Vec3<double> xv = load_vec(D.x64, vh, i);
        const Vec3<float> hv = load_vec((const float *)D.xi, vh, i);
        Vec3<float> z;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xv.c[a].re += (double)hv.c[a].re;
            xv.c[a].im += (double)hv.c[a].im;
            z.c[a].re = z.c[a].im = 0.f;
        }
        store_vec(D.x64, vh, i, xv);
        store_vec((float *)D.xi, vh, i, z);
    } else {
        const Vec3<double> rd = load_vec(D.r64, vh, i);
        Vec3<float> rv;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            rv.c[a].re = (float)rd.c[a].re;
            rv.c[a].im = (float)rd.c[a].im;
        }
        store_vec((float *)D.ri, vh, i, rv);
    }
}

// End of a reliable update in the graph solve: the loop condition.
__global__ void batch_setcond_kernel(const BatchScalars *S, const GraphCtl ctl) {
    if (ctl.active && threadIdx.x == 0)
        cudaGraphSetConditional(ctl.loop, (!S->halt && S->trips < S->maxiter + 4) ? 1u : 0u);
}

// Snapshot of need[] for the update's vector steps (the residual clears it).
__global__ void batch_snap_kernel(const BatchScalars *S, int *need, int n) {
    if (threadIdx.x < n) need[threadIdx.x] = S->need[threadIdx.x];
}

// ||b||^2 per lattice (stop criterion); zero sources are solved (x = 0).
__global__ void __launch_bounds__(kTile)
batch_norm2_kernel(const LatDesc *__restrict__ descs, int n, BatchScalars *S, double *partials,
                   unsigned int *counter) {
    __shared__ double smem[32];
    __shared__ double tot[kMaxRhs];
    __shared__ int ident[kMaxRhs + 1];
    const int l = lattice_of_full_tile(descs, n, blockIdx.x);
    const LatDesc &D = descs[l];
    const size_t vh = (size_t)D.g.vh;
    const int i = (blockIdx.x - D.tile0) * kTile + threadIdx.x;
    double part = 0.0;
    if (i < D.g.vh) {
        const Vec3<double> v = load_vec(D.b, vh, i);
#pragma unroll
        for (int a = 0; a < 3; ++a) part += v.c[a].re * v.c[a].re + v.c[a].im * v.c[a].im;
    }
    const double bs = block_sum(part, smem);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bs;
        for (int k = 0; k <= n; ++k) ident[k] = k < n ? descs[k].tile0 : descs[n - 1].tile0 + descs[n - 1].ntiles;
    }
    if (!last_block_totals(partials, counter, n, ident, tot, gridDim.x)) return;
    if (threadIdx.x != 0) return;
    for (int k = 0; k < n; ++k) {
        S->bb[k] = tot[k];
        S->stop2[k] = S->tol2 * tot[k];
        if (!isfinite(tot[k])) S->error = 1;
        S->need[k] = 1;  // the first FP64 residual
        if (tot[k] == 0.0) {
            S->active[k] = 0;
            S->done[k] = 1;
            S->need[k] = 0;
        }
    }
}

// Batch scratch and cached graph, owned by the first item's lattice.
struct BatchCtx {
    LatDesc *descs;
    BatchScalars *S;
    BatchScalars *host;
    int *need_snap;
    double *partials;
    unsigned int *counter;
    int cap_tiles;
    // graph cache key and graph
    int g_n, g_tiles, g_naik, g_grid, g_spt;
    qex_prec g_inner;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

void free_batch_ctx(void *p) {
    BatchCtx *c = (BatchCtx *)p;
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    cudaFree(c->descs);
    cudaFree(c->S);
    cudaFreeHost(c->host);
    cudaFree(c->need_snap);
    cudaFree(c->partials);
    cudaFree(c->counter);
    delete c;
}

static size_t al256b(size_t n) { return (n + 255) & ~size_t(255); }

qex_status check_dslash_args(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                             const void *in, const void *out);

struct BatchLaunch {
    const BatchCtx *c;
    int n, total_tiles, iter_grid, spt;
    qex_prec inner;
    bool naik, mixed;
};

// Work items of a batch with `spt` groups per item, and the iteration grid
// of `per_sm` resident blocks per SM.
static int batch_items(const std::vector<LatDesc> &d, int spt) {
    int w = 0;
    for (const LatDesc &D : d) w += (D.ntiles + spt - 1) / spt;
    return w;
}

static int batch_grid(int items, int per_sm) {
    const int resident = sm_count() * per_sm;
    return items < resident ? items : resident;
}

// Set the groups per work item and rebuild the running list (one thread).
__global__ void batch_relist_kernel(BatchScalars *S, const LatDesc *__restrict__ descs, int n, int spt) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        S->spt = spt;
        compact_list(S, descs, n);
    }
}

// Launch shapes chosen per (SM count, extents and boundary of every lattice
// in order, inner precision, Naik), for the life of the process.
struct BatchShape {
    int per_sm, spt;
};
static std::map<std::string, BatchShape> g_batch_shapes;
static std::mutex g_batch_mu;

static std::string batch_key(int n, const qex_cg_item *items, qex_prec inner, bool naik) {
    std::string k = "sm" + std::to_string(sm_count()) + " prec" + std::to_string((int)inner) + " naik" +
                    std::to_string(naik ? 1 : 0);
    for (int i = 0; i < n; ++i) {
        const qex_lattice *l = items[i].lat;
        k += " " + std::to_string(l->dims[0]) + "x" + std::to_string(l->dims[1]) + "x" + std::to_string(l->dims[2]) +
             "x" + std::to_string(l->dims[3]) + (l->antiperiodic ? "a" : "p");
    }
    return k;
}

template <typename R, int FMT, bool NAIK>
static void launch_iter_t(const BatchLaunch &b, int role, cudaStream_t s) {
    if (role == ROLE_K1)
        batch_iter_dslash_kernel<R, FMT, NAIK, ROLE_K1><<<b.iter_grid, kTile, 0, s>>>(b.c->descs, b.c->S,
                                                                                       b.c->partials, b.c->counter);
    else
        batch_iter_dslash_kernel<R, FMT, NAIK, ROLE_K2><<<b.iter_grid, kTile, 0, s>>>(b.c->descs, b.c->S,
                                                                                       b.c->partials, b.c->counter);
}

template <typename R, int FMT>
static void launch_iter_n(const BatchLaunch &b, int role, cudaStream_t s) {
    if (b.naik)
        launch_iter_t<R, FMT, true>(b, role, s);
    else
        launch_iter_t<R, FMT, false>(b, role, s);
}

static void launch_iter_role(const BatchLaunch &b, int role, cudaStream_t s) {
    if (b.inner == QEX_F64)
        launch_iter_n<double, 0>(b, role, s);
    else if (b.inner == QEX_F32_R12)
        launch_iter_n<float, 1>(b, role, s);
    else if (b.inner == QEX_F32_R12H)
        launch_iter_n<float, 2>(b, role, s);
    else if (b.inner == QEX_F32_S16)
        launch_iter_n<float, 3>(b, role, s);
    else
        launch_iter_n<float, 0>(b, role, s);
}

static qex_status enqueue_iteration(const BatchLaunch &b, const GraphCtl &ctl, cudaStream_t s) {
    for (int role = ROLE_K1; role <= ROLE_K2; ++role) {
        launch_iter_role(b, role, s);
        QEX_CHECK_LAUNCH("batch_iter_dslash_kernel");
    }
    if (b.mixed)
        batch_update_kernel<float><<<b.iter_grid, kTile, 0, s>>>(b.c->descs, b.c->S, b.c->partials, b.c->counter, ctl);
    else
        batch_update_kernel<double><<<b.iter_grid, kTile, 0, s>>>(b.c->descs, b.c->S, b.c->partials, b.c->counter,
                                                                  ctl);
    QEX_CHECK_LAUNCH("batch_update_kernel");
    return QEX_OK;
}

static qex_status enqueue_reliable_update(const BatchLaunch &b, const GraphCtl &ctl, cudaStream_t s) {
    const BatchCtx *c = b.c;
    batch_snap_kernel<<<1, kMaxRhs, 0, s>>>(c->S, c->need_snap, b.n);
    QEX_CHECK_LAUNCH("batch_snap_kernel");
    if (b.mixed) {
        batch_ru_vectors_kernel<0><<<b.total_tiles, kTile, 0, s>>>(c->descs, b.n, c->need_snap);
        QEX_CHECK_LAUNCH("batch_ru_vectors_kernel");
    }
    if (b.naik) {
        batch_ru_dslash_kernel<true, ROLE_RU1><<<b.total_tiles, kTile, 0, s>>>(c->descs, b.n, c->S, c->need_snap,
                                                                             c->partials, c->counter);
        QEX_CHECK_LAUNCH("batch_ru_dslash_kernel");
        batch_ru_dslash_kernel<true, ROLE_RU2><<<b.total_tiles, kTile, 0, s>>>(c->descs, b.n, c->S, c->need_snap,
                                                                             c->partials, c->counter);
    } else {
        batch_ru_dslash_kernel<false, ROLE_RU1><<<b.total_tiles, kTile, 0, s>>>(c->descs, b.n, c->S, c->need_snap,
                                                                              c->partials, c->counter);
        QEX_CHECK_LAUNCH("batch_ru_dslash_kernel");
        batch_ru_dslash_kernel<false, ROLE_RU2><<<b.total_tiles, kTile, 0, s>>>(c->descs, b.n, c->S, c->need_snap,
                                                                              c->partials, c->counter);
    }
    QEX_CHECK_LAUNCH("batch_ru_dslash_kernel");
    if (b.mixed) {
        batch_ru_vectors_kernel<1><<<b.total_tiles, kTile, 0, s>>>(c->descs, b.n, c->need_snap);
        QEX_CHECK_LAUNCH("batch_ru_vectors_kernel");
    }
    if (ctl.active) {
        batch_setcond_kernel<<<1, 32, 0, s>>>(c->S, ctl);
        QEX_CHECK_LAUNCH("batch_setcond_kernel");
    }
    return QEX_OK;
}

static qex_status build_batch_graph(BatchCtx *c, const BatchLaunch &b) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->exec = nullptr;
    c->graph = nullptr;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaSuccess;
    qex_status st = QEX_OK;
    set_count_launches(false);
    do {
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) break;
        if ((e = cudaGraphCreate(&c->graph, 0))) break;
        GraphCtl ctl = {};
        ctl.active = 1;
        if ((e = cudaGraphConditionalHandleCreate(&ctl.loop, c->graph, 1, cudaGraphCondAssignDefault))) break;
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = ctl.loop;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode;
        if ((e = cudaGraphAddNode(&wnode, c->graph, nullptr, nullptr, 0, &wp))) break;
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        if ((e = cudaGraphConditionalHandleCreate(&ctl.ru, body, 0, 0))) break;
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
        for (int u = 0; u < QEX_GRAPH_UNROLL && !st; ++u) st = enqueue_iteration(b, ctl, cs);
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        cudaGraph_t capg = nullptr;
        cudaGraphNodeParams ip = {};
        cudaGraphNode_t inode = nullptr;
        if (!st) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &capg, &deps, nullptr, &ndeps);
        if (!st && !e) {
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = ctl.ru;
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            e = cudaGraphAddNode(&inode, capg, deps, nullptr, ndeps, &ip);
        }
        if (!st && !e)
            e = cudaStreamUpdateCaptureDependencies(cs, &inode, nullptr, 1, cudaStreamSetCaptureDependencies);
        cudaGraph_t captured = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
        if (st) break;
        if (e || (e = e2)) break;
        if ((e = cudaStreamBeginCaptureToGraph(cs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeRelaxed)))
            break;
        st = enqueue_reliable_update(b, ctl, cs);
        e2 = cudaStreamEndCapture(cs, &captured);
        if (st) break;
        if ((e = e2)) break;
        if ((e = cudaGraphInstantiate(&c->exec, c->graph, 0))) break;
    } while (0);
    set_count_launches(true);
    if (cs) cudaStreamDestroy(cs);
    if (st || e) {
        if (c->exec) cudaGraphExecDestroy(c->exec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->exec = nullptr;
        c->graph = nullptr;
        return st ? st : cuda_fail(e, "building the batched CG graph");
    }
    c->g_n = b.n;
    c->g_tiles = b.total_tiles;
    c->g_grid = b.iter_grid;
    c->g_spt = b.spt;
    c->g_naik = b.naik;
    c->g_inner = b.inner;
    return QEX_OK;
}

static bool batch_tuning_enabled() {
    const char *e = getenv("QEX_TUNE");
    return !(e && strcmp(e, "0") == 0);
}

// Time the two Dslash kernels of an iteration (both only overwrite scratch
// and the per-lattice alpha, so repeating them changes nothing the loop then
// computes) for every (blocks per SM, groups per item) candidate, each the
// least of three short batches; keep the fastest.  The running list is left
// built for the last candidate's items: the caller rebuilds it.
static qex_status tune_batch(const BatchLaunch &b0, const std::vector<LatDesc> &descs, cudaStream_t s,
                             BatchShape *best) {
    cudaEvent_t e0, e1;
    QEX_CUDA(cudaEventCreate(&e0));
    QEX_CUDA(cudaEventCreate(&e1));
    float best_us = 0.f;
    *best = BatchShape{kBatchMinBlocks, 1};
    qex_status st = QEX_OK;
    set_count_launches(false);
    for (int spt = 1; spt <= kMaxSpt && !st; spt *= 2)
        for (int per_sm = 1; per_sm <= kBatchMinBlocks && !st; ++per_sm) {
            BatchLaunch b = b0;
            b.spt = spt;
            b.iter_grid = batch_grid(batch_items(descs, spt), per_sm);
            batch_relist_kernel<<<1, 32, 0, s>>>(const_cast<BatchScalars *>(b.c->S), b.c->descs, b.n, spt);
            float cand = 0.f;
            for (int rep = 0; rep < 4 && !st; ++rep) {  // rep 0 warms up
                cudaEventRecord(e0, s);
                for (int k = 0; k < 4; ++k)
                    for (int role = ROLE_K1; role <= ROLE_K2; ++role) launch_iter_role(b, role, s);
                cudaEventRecord(e1, s);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaGetLastError();
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "timing a batch launch shape");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1 || (rep > 1 && ms * 250.f < cand)) cand = ms * 250.f;  // us per iteration
            }
            if (!st && (best_us == 0.f || cand < best_us)) {
                best_us = cand;
                *best = BatchShape{per_sm, spt};
            }
        }
    set_count_launches(true);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // namespace qex

using namespace qex;

extern "C" qex_status qex_cg_batch_tune_info(const qex_lattice *lead, int *out) {
    qex_status st;
    if ((st = check_lattice(lead))) return st;
    if (!out) {
        set_error("out must not be NULL");
        return QEX_ERR_ARG;
    }
    out[0] = lead->batch_shape[0] > 0 ? lead->batch_shape[0] : kBatchMinBlocks;
    out[1] = lead->batch_shape[1] > 0 ? lead->batch_shape[1] : 1;
    out[2] = lead->batch_shape[2];
    return QEX_OK;
}

extern "C" qex_status qex_cg_batch_tune_set(const qex_lattice *lead, int blocks_per_sm, int groups_per_item) {
    qex_status st;
    if ((st = check_lattice(lead))) return st;
    const bool unpin = blocks_per_sm == 0 && groups_per_item == 0;
    if (!unpin && (blocks_per_sm < 1 || blocks_per_sm > kBatchMinBlocks ||
                   (groups_per_item != 1 && groups_per_item != 2 && groups_per_item != 4))) {
        set_error("need 1 <= blocks_per_sm <= %d and groups_per_item 1, 2 or 4 (0, 0 unpins)", kBatchMinBlocks);
        return QEX_ERR_ARG;
    }
    qex_lattice *l = const_cast<qex_lattice *>(lead);
    l->batch_pin[0] = unpin ? 0 : blocks_per_sm;
    l->batch_pin[1] = unpin ? 0 : groups_per_item;
    return QEX_OK;
}

extern "C" qex_status qex_cg_batch(int n, const qex_cg_item *items, qex_prec inner, double tol, int maxiter,
                                   double delta, void *stream, qex_cg_stats *stats) {
    qex_status st;
    if (n < 1 || n > QEX_BATCH_MAX || !items) {
        set_error("need 1 <= n <= %d items", QEX_BATCH_MAX);
        return QEX_ERR_ARG;
    }
    if ((st = check_prec(inner))) return st;
    if (!(tol > 0.0) || maxiter < 0 || !(delta >= 0.0 && delta < 1.0)) {
        set_error("need tol > 0, maxiter >= 0 and 0 <= delta < 1");
        return QEX_ERR_ARG;
    }
    const bool mixed = inner != QEX_F64;
    const bool naik = items[0].lng64 != nullptr;
    int total_tiles = 0;
    for (int k = 0; k < n; ++k) {
        const qex_cg_item &it = items[k];
        if ((st = check_dslash_args(it.lat, QEX_F64, it.fat64, it.lng64, it.b64, it.x64))) return st;
        if ((it.lng64 != nullptr) != naik) {
            set_error("all batch items must agree on the Naik term");
            return QEX_ERR_ARG;
        }
        if (mixed && (!it.fat32 || !aligned16(it.fat32) || (naik && (!it.lng32 || !aligned16(it.lng32))))) {
            set_error("item %d: mixed precision needs aligned inner-precision links", k);
            return QEX_ERR_ARG;
        }
        for (int j = 0; j < k; ++j)
            if (items[j].lat == it.lat) {
                set_error("items %d and %d share a lattice object (each needs its own work vectors)", j, k);
                return QEX_ERR_ARG;
            }
        total_tiles += blocks_for(it.lat->vh, kTile);
    }
    const cudaStream_t s = as_stream(stream);
    qex_lattice *own = const_cast<qex_lattice *>(items[0].lat);
    const char *mode = getenv("QEX_CG_MODE");
    const bool use_graph = !(mode && strcmp(mode, "host") == 0);

    // per-lattice work vectors in each lattice's own work area
    std::vector<LatDesc> descs(n);
    int tile = 0;
    for (int k = 0; k < n; ++k) {
        const qex_cg_item &it = items[k];
        qex_lattice *lat = const_cast<qex_lattice *>(it.lat);
        const size_t f64 = al256b((size_t)lat->vh * 48), fi = al256b((size_t)lat->vh * (mixed ? 24 : 48));
        if ((st = ensure_work(lat, 2 * f64 + 6 * fi))) return st;
        char *w = (char *)lat->work;
        LatDesc &D = descs[k];
        memset(&D, 0, sizeof(D));
        D.g = lat->geom;
        D.tile0 = tile;
        D.ntiles = blocks_for(lat->vh, kTile);
        tile += D.ntiles;
        D.fat_in = mixed ? it.fat32 : it.fat64;
        D.lng_in = mixed ? it.lng32 : it.lng64;
        D.fat64 = (const double *)it.fat64;
        D.lng64 = (const double *)it.lng64;
        D.b = (const double *)it.b64;
        D.x64 = (double *)it.x64;
        D.r64 = (double *)w;
        w += f64;
        D.tmp64 = (double *)w;
        w += f64;
        if (mixed) {
            D.xi = w;
            w += fi;
            D.ri = w;
            w += fi;
        } else {
            D.xi = D.x64;
            D.ri = D.r64;
            w += 2 * fi;
        }
        D.p0 = w;
        w += fi;
        D.p1 = w;
        w += fi;
        D.api = w;
        w += fi;
        D.tmpi = mixed ? (void *)w : (void *)D.tmp64;
        D.m2 = it.mass * it.mass;
        D.c3 = it.c_naik;
    }

    // batch scratch on the first lattice
    BatchCtx *c = (BatchCtx *)own->batch_ctx;
    if (!c || c->cap_tiles < total_tiles) {
        if (c) {
            QEX_CUDA(cudaStreamSynchronize(s));
            free_batch_ctx(c);
            own->batch_ctx = nullptr;
        }
        c = new BatchCtx;
        memset(c, 0, sizeof(*c));
        c->cap_tiles = total_tiles;
        own->batch_ctx = c;
        QEX_CUDA(cudaMalloc(&c->descs, sizeof(LatDesc) * QEX_BATCH_MAX));
        QEX_CUDA(cudaMalloc(&c->S, sizeof(BatchScalars)));
        QEX_CUDA(cudaMallocHost(&c->host, sizeof(BatchScalars)));
        QEX_CUDA(cudaMalloc(&c->need_snap, sizeof(int) * QEX_BATCH_MAX));
        QEX_CUDA(cudaMalloc(&c->partials, sizeof(double) * total_tiles));
        QEX_CUDA(cudaMalloc(&c->counter, sizeof(unsigned int)));
        QEX_CUDA(cudaMemset(c->counter, 0, sizeof(unsigned int)));
    }
    BatchLaunch b;
    b.c = c;
    b.n = n;
    b.total_tiles = total_tiles;
    b.inner = inner;
    b.naik = naik;
    b.mixed = mixed;
    // launch shape: pinned on the lead lattice, from the process cache, the
    // compiled defaults (QEX_TUNE=0), or measured after the first residual
    const std::string key = batch_key(n, items, inner, naik);
    int per_sm = kBatchMinBlocks, spt = 1, source = 0;
    bool need_tune = false;
    if (own->batch_pin[0] > 0) {
        per_sm = own->batch_pin[0];
        spt = own->batch_pin[1];
        source = 4;
    } else if (!batch_tuning_enabled()) {
        source = 3;
    } else {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        auto it = g_batch_shapes.find(key);
        if (it != g_batch_shapes.end()) {
            per_sm = it->second.per_sm;
            spt = it->second.spt;
            source = 2;
        } else {
            need_tune = true;
        }
    }
    b.spt = spt;
    b.iter_grid = batch_grid(batch_items(descs, spt), per_sm);

    QEX_CUDA(cudaStreamSynchronize(s));  // the pinned slot is free
    BatchScalars *h = c->host;
    memset(h, 0, sizeof(*h));
    h->n = n;
    h->spt = spt;
    h->tol2 = tol * tol;
    h->delta2 = mixed ? delta * delta : 0.0;
    h->max_cycle = ru_max_cycle(inner);
    h->maxiter = maxiter;
    for (int k = 0; k < n; ++k) h->active[k] = 1;
    cudaEvent_t t0, t1;
    QEX_CUDA(cudaEventCreate(&t0));
    QEX_CUDA(cudaEventCreate(&t1));
    QEX_CUDA(cudaEventRecord(t0, s));
    QEX_CUDA(cudaMemcpyAsync(c->descs, descs.data(), sizeof(LatDesc) * n, cudaMemcpyHostToDevice, s));
    QEX_CUDA(cudaMemcpyAsync(c->S, h, sizeof(BatchScalars), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < n; ++k) {
        const size_t fb = (size_t)items[k].lat->vh * (mixed ? 24 : 48);
        QEX_CUDA(cudaMemsetAsync(descs[k].p0, 0, fb, s));
        QEX_CUDA(cudaMemsetAsync(descs[k].p1, 0, fb, s));
        if (mixed) QEX_CUDA(cudaMemsetAsync(descs[k].xi, 0, fb, s));
    }
    batch_norm2_kernel<<<total_tiles, kTile, 0, s>>>(c->descs, n, c->S, c->partials, c->counter);
    QEX_CHECK_LAUNCH("batch_norm2_kernel");
    const GraphCtl off = {};
    auto fetch = [&]() -> qex_status {
        QEX_CUDA(cudaMemcpyAsync(h, c->S, sizeof(BatchScalars), cudaMemcpyDeviceToHost, s));
        QEX_CUDA(cudaStreamSynchronize(s));
        return QEX_OK;
    };
    // the first FP64 residual of every lattice, outside the loop (it also
    // builds the running-lattice list)
    if ((st = enqueue_reliable_update(b, off, s)) || (st = fetch())) return st;
    for (int k = 0; k < n; ++k)  // zero sources: x = 0 exactly
        if (h->bb[k] == 0.0) QEX_CUDA(cudaMemsetAsync(items[k].x64, 0, (size_t)items[k].lat->vh * 48, s));
    bool relist = spt != h->spt;  // the list the first residual built is for another item size
    if (need_tune && !h->error && !h->halt) {
        BatchShape best;
        if ((st = tune_batch(b, descs, s, &best))) return st;
        per_sm = best.per_sm;
        spt = best.spt;
        source = 1;
        relist = true;  // the timing left the list built for its last candidate
        std::lock_guard<std::mutex> lk(g_batch_mu);
        g_batch_shapes[key] = best;
    }
    if (relist) {
        batch_relist_kernel<<<1, 32, 0, s>>>(c->S, c->descs, n, spt);
        QEX_CHECK_LAUNCH("batch_relist_kernel");
    }
    b.spt = spt;
    b.iter_grid = batch_grid(batch_items(descs, spt), per_sm);
    own->batch_shape[0] = per_sm;
    own->batch_shape[1] = spt;
    own->batch_shape[2] = source;
    if (use_graph && !h->error && !h->halt &&
        !(c->exec && c->g_n == n && c->g_tiles == total_tiles && c->g_naik == (int)naik && c->g_inner == inner &&
          c->g_grid == b.iter_grid && c->g_spt == spt)) {
        QEX_CUDA(cudaStreamSynchronize(s));
        if ((st = build_batch_graph(c, b))) return st;
    }
    if (!h->error && !h->halt) {
        if (use_graph) {
            QEX_CUDA(cudaGraphLaunch(c->exec, s));
            if ((st = fetch())) return st;
            note_launches(3ull * (unsigned long long)(h->trips + h->idle_iters) +
                          (mixed ? 6ull : 4ull) *
                              (unsigned long long)(h->reliable_updates > 1 ? h->reliable_updates - 1 : 0));
        } else {
            const int batch = 8;
            while (!st && !h->error && !h->halt) {
                for (int k = 0; k < batch && !st; ++k) st = enqueue_iteration(b, off, s);
                if (st || (st = fetch())) break;
                if (h->error || !h->any_need) continue;
                if ((st = enqueue_reliable_update(b, off, s)) || (st = fetch())) break;
            }
            if (st) return st;
        }
    }
    QEX_CUDA(cudaEventRecord(t1, s));
    QEX_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    int all = 1;
    for (int k = 0; k < n; ++k) all &= h->done[k];
    qex_status result = QEX_OK;
    if (h->error) {
        set_error("NaN/Inf or CG breakdown in a batched solve");
        result = QEX_ERR_NAN;
    } else if (!all) {
        set_error("batched CG: not every lattice converged in %d iterations", maxiter);
        result = QEX_ERR_NOT_CONVERGED;
    }
    if (stats)
        for (int k = 0; k < n; ++k) {
            stats[k].iters = h->iters[k];
            stats[k].reliable_updates = h->reliable_updates > 0 ? h->reliable_updates - 1 : 0;
            stats[k].converged = h->done[k];
            stats[k].ff_updates = 0;
            stats[k].true_rel_resid = h->bb[k] > 0.0 ? sqrt(h->true_rr[k] / h->bb[k]) : 0.0;
            stats[k].time_ms = ms;
        }
    return result;
}
