// cg.cu -- conjugate gradient on A = m^2 - D_eo D_oe (even sites): plain FP64
// and mixed precision with reliable updates.
//
// One iteration is three kernels (mixed precision) and reads nothing back:
//   1. p_new = r + beta p_old formed on the fly at every neighbour read,
//      tmp = D_oe p_new, and p_new stored (two p buffers, chosen by the parity
//      of the device-side iteration count; FP64 CG forms p_new in a separate
//      pass, because its Dslash is FP64-ALU bound);
//   2. A p_new = m^2 p_new - D_eo tmp with <p_new, A p_new> -> alpha;
//   3. x += alpha p_new, r -= alpha A p_new, ||r||^2 -> beta or a halt flag.
// In a mixed solve the iterate update of kernel 3 moves into the next
// iteration's kernel 1, which reads p_old at its own site anyway (kernel 3
// then moves r and A p only); a reliable update takes the pending alpha p
// itself and zeroes alpha.
// alpha, beta and the norms stay in device memory.  By default the whole
// solve runs as one CUDA graph: a conditional WHILE node around
// QEX_GRAPH_UNROLL iterations of the three kernels, followed inside the loop
// by a conditional IF node holding the reliable update (FP64 true residual);
// kernel 3 and the update's last kernel set the two conditions.  The loop ends when the true residual meets
// tol, on the iteration cap, or on a NaN, and in any case after maxiter + 4
// trips.  Setting QEX_CG_MODE=host instead enqueues batches of iterations
// from the host and runs the reliable updates between batches.  A mixed
// solve of a small lattice (Vh <= 32768, or QEX_CG_MODE=fused) runs its inner
// iterations as one persistent cooperative kernel instead (cg_fused.cu), with
// the reliable updates launched from the host in between.
//
// Mixed precision (inner = any FP32 format): x_hat, r_hat, p, A p live in FP32
// and the operator runs on FP32 links; when ||r_hat|| falls below delta times
// its largest value since the last update, or meets tol, x += x_hat (FP64),
// r = b - A x with the FP64 operator, r_hat = (float) r, and beta comes from
// the true ||r||^2; p is kept.  Convergence is only accepted on the FP64 true
// residual.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "qex_kernels.cuh"

namespace qex {

qex_status check_dslash_args(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                             const void *in, const void *out);
void set_count_launches(bool on);

static size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Largest half volume that the mixed solve runs as the fused persistent
// iteration by default (cg_fused.cu).
constexpr int64_t kFusedAutoMaxVh = 32768;

struct CgBuffers {
    double *r64, *tmp64, *p64[2], *ap64;
    float *xh32, *r32, *p32[2], *ap32, *tmp32;
};

static qex_status carve(qex_lattice *lat, bool mixed, CgBuffers &B) {
    size_t f64 = align256((size_t)lat->vh * 48), f32 = align256((size_t)lat->vh * 24);
    size_t need = mixed ? 2 * f64 + 6 * f32 : 5 * f64;
    qex_status st = ensure_work(lat, need);
    if (st) return st;
    char *w = (char *)lat->work;
    memset(&B, 0, sizeof(B));
    B.r64 = (double *)w;
    w += f64;
    B.tmp64 = (double *)w;
    w += f64;
    if (mixed) {
        float **f[] = {&B.xh32, &B.r32, &B.p32[0], &B.p32[1], &B.ap32, &B.tmp32};
        for (float **q : f) {
            *q = (float *)w;
            w += f32;
        }
    } else {
        double **d[] = {&B.p64[0], &B.p64[1], &B.ap64};
        for (double **q : d) {
            *q = (double *)w;
            w += f64;
        }
    }
    return QEX_OK;
}

struct Solve {
    qex_lattice *lat;
    bool mixed;
    qex_prec inner;
    const void *fat64, *lng64, *fat32, *lng32;
    double c3, m2;
    const double *b64;
    double *x64;
    bool defer_x;  // the FP32 iterate takes alpha p one iteration late, in kernel 1
    bool ff_ok;    // intermediate reliable updates in float-float arithmetic (ru_ff.cu)
    CgBuffers B;
};

// Reliable updates are FP64 (the true-residual recomputation of the mixed
// scheme); QEX_RU_FF=1 runs those that cannot end the solve in float-float
// arithmetic instead (ru_ff.cu), the stopping test staying FP64.
static bool ru_ff_enabled(bool mixed) {
    if (!mixed) return false;
    const char *e = getenv("QEX_RU_FF");
    return e && strcmp(e, "1") == 0;
}

#ifndef QEX_DEFER_X
#define QEX_DEFER_X 1
#endif
#ifndef QEX_REVERSE_SECOND
#define QEX_REVERSE_SECOND 1
#endif
// The normal-operator Dslash walks the sites downwards, meeting first the
// links the D_oe launch before it read last (still in L2).
static const bool reverse_second = QEX_REVERSE_SECOND != 0;

// Events recorded after each kernel of an iteration (profiling only).
struct Marks {
    cudaEvent_t *ev;  // one per kernel of the iteration, NULL: none
    int n;
};

static qex_status mark(const Marks *m, int k, cudaStream_t st) {
    if (m && m->ev && k < m->n) QEX_CUDA(cudaEventRecord(m->ev[k], st));
    return QEX_OK;
}

// One CG iteration in the inner precision, every kernel halt-checked.
// marks: an event recorded after each kernel (k = 0, 1, ...), or NULL.
static qex_status enqueue_iteration(Solve &s, const GraphCtl &ctl, cudaStream_t st, const Marks *marks = nullptr) {
    qex_lattice *lat = s.lat;
    CgScalars *S = lat->scalars;
    DslashArgs a = {};
    a.prec = s.inner;
    a.fat = s.mixed ? s.fat32 : s.fat64;
    a.lng = s.mixed ? s.lng32 : s.lng64;
    a.c3 = s.c3;
    a.S = S;
    a.check_halt = 1;
    void *tmp = s.mixed ? (void *)s.B.tmp32 : (void *)s.B.tmp64;
    void *ap = s.mixed ? (void *)s.B.ap32 : (void *)s.B.ap64;
    void *x = s.mixed ? (void *)s.B.xh32 : (void *)s.x64;
    void *r = s.mixed ? (void *)s.B.r32 : (void *)s.B.r64;
    void *pb[2] = {s.mixed ? (void *)s.B.p32[0] : (void *)s.B.p64[0],
                   s.mixed ? (void *)s.B.p32[1] : (void *)s.B.p64[1]};
    qex_status err;
    int k = 0;
    a.out_parity = 1;
    a.out = tmp;
    a.r = r;
    a.pbuf[0] = pb[0];
    a.pbuf[1] = pb[1];
    if (s.mixed) {
        // FP32: the direction update rides along the first Dslash (its few
        // extra FMAs per neighbour are free in a memory-bound kernel)
        a.epi = EPI_PUPD;
        if (s.defer_x) {
            a.x = x;
            x = nullptr;
        }
    } else {
        // FP64: the Dslash is FP64-ALU bound, so the update is its own
        // memory-bound pass instead of eight recomputations per site
        if ((err = launch_update_p(lat, a.prec, r, pb, S, st))) return err;
        if ((err = mark(marks, k++, st))) return err;
        a.epi = EPI_PLAIN;
        a.psel = 1;
    }
    if ((err = launch_dslash(lat, a, st))) return err;
    if ((err = mark(marks, k++, st))) return err;
    a.out_parity = 0;
    a.in = tmp;
    a.out = ap;
    a.epi = EPI_NORMAL;
    a.psel = 1;
    a.m2 = s.m2;
    a.reverse = reverse_second ? 1 : 0;
    if ((err = launch_dslash(lat, a, st))) return err;
    if ((err = mark(marks, k++, st))) return err;
    if ((err = launch_update_xr(lat, a.prec, x, r, pb, ap, S, ctl, st))) return err;
    return mark(marks, k, st);
}

// FP64 true residual r64 = b - A x64 (after folding x_hat into x64), then the
// inner residual from it.  `first`: the residual of the initial guess, whose
// two Dslash passes do nothing when every element of x is zero (checked just
// before).
static qex_status enqueue_reliable_update(Solve &s, const GraphCtl &ctl, cudaStream_t st, bool first = false) {
    qex_lattice *lat = s.lat;
    CgScalars *S = lat->scalars;
    qex_status err;
    if (s.mixed && (err = launch_accum_x(lat, s.x64, s.B.xh32, (s.defer_x && !first) ? s.B.p32 : nullptr, S, st)))
        return err;
    DslashArgs a = {};
    a.prec = QEX_F64;
    a.fat = s.fat64;
    a.lng = s.lng64;
    a.c3 = s.c3;
    a.out_parity = 1;
    a.in = s.x64;
    a.out = s.B.tmp64;
    a.epi = EPI_PLAIN;
    a.S = S;
    a.skip_zero_x = first ? 1 : 0;
    // the FP64 kernels and their float-float twins (an update the iterated
    // residual asks for before it meets tol): S->ru_ff lets one pair run
    const bool ff = s.mixed && !first && s.ff_ok;
    a.skip_ff = ff ? 1 : 0;
    if ((err = launch_dslash(lat, a, st))) return err;
    if (ff && (err = launch_ru_ff(lat, 1, (const double *)s.fat64, (const double *)s.lng64, s.c3, s.m2,
                                  (const double *)s.x64, nullptr, s.B.tmp64, nullptr, S, true, false, st)))
        return err;
    a.out_parity = 0;
    a.in = s.B.tmp64;
    a.out = s.B.r64;
    a.epi = EPI_RESID;
    a.q = s.x64;
    a.b = s.b64;
    a.m2 = s.m2;
    a.S = S;
    if ((err = launch_dslash(lat, a, st))) return err;
    if (ff && (err = launch_ru_ff(lat, 2, (const double *)s.fat64, (const double *)s.lng64, s.c3, s.m2,
                                  (const double *)s.x64, (const double *)s.b64, s.B.tmp64, s.B.r32, S, true, false,
                                  st)))
        return err;
    return launch_finish_ru(lat, s.B.r64, s.mixed ? s.B.r32 : nullptr, S, ctl, st);
}

static qex_status fetch_scalars(qex_lattice *lat, int slot, cudaStream_t st) {
    QEX_CUDA(cudaMemcpyAsync(slot ? lat->scalars_host2 : lat->scalars_host, lat->scalars, sizeof(CgScalars),
                             cudaMemcpyDeviceToHost, st));
    QEX_CUDA(cudaEventRecord(slot ? lat->ev1 : lat->ev0, st));
    return QEX_OK;
}

static qex_status wait_scalars(qex_lattice *lat, int slot) {
    QEX_CUDA(cudaEventSynchronize(slot ? lat->ev1 : lat->ev0));
    return QEX_OK;
}

// ------------------------------------------------------------- graph solve

// An instantiated solve graph, reusable while every pointer and constant
// baked into its kernels stays the same.
struct CgGraph {
    qex_prec inner;
    const void *fat64, *lng64, *fat32, *lng32;
    double c3, m2;
    const void *b64, *x64, *work;
    int pdl;  // kernels linked by programmatic dependencies
    bool ff_ok;  // the updates carry float-float twins
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    unsigned long long kernels_per_iter, kernels_per_ru;
};

static bool same_key(const CgGraph *g, const Solve &s) {
    return g && g->inner == s.inner && g->fat64 == s.fat64 && g->lng64 == s.lng64 && g->fat32 == s.fat32 &&
           g->lng32 == s.lng32 && g->c3 == s.c3 && g->m2 == s.m2 && g->b64 == s.b64 && g->x64 == s.x64 &&
           g->work == s.lat->work && g->pdl == s.lat->pdl && g->ff_ok == s.ff_ok;
}

static void drop_graph(CgGraph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

static qex_status build_graph(Solve &s, CgGraph **out) {
    *out = nullptr;
    CgGraph *G = new CgGraph;
    memset(G, 0, sizeof(*G));
    G->inner = s.inner;
    G->fat64 = s.fat64;
    G->lng64 = s.lng64;
    G->fat32 = s.fat32;
    G->lng32 = s.lng32;
    G->c3 = s.c3;
    G->m2 = s.m2;
    G->b64 = s.b64;
    G->x64 = s.x64;
    G->work = s.lat->work;
    G->pdl = s.lat->pdl;
    G->ff_ok = s.ff_ok;
    G->kernels_per_iter = s.mixed ? 3 : 4;
    G->kernels_per_ru = s.mixed ? (s.ff_ok ? 6 : 4) : 3;
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaSuccess;
    qex_status st = QEX_OK;
    set_count_launches(false);
    do {
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) break;
        if ((e = cudaGraphCreate(&G->graph, 0))) break;
        GraphCtl ctl = {};
        ctl.active = 1;
        if ((e = cudaGraphConditionalHandleCreate(&ctl.loop, G->graph, 1, cudaGraphCondAssignDefault))) break;
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = ctl.loop;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode;
        if ((e = cudaGraphAddNode(&wnode, G->graph, nullptr, nullptr, 0, &wp))) break;
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        if ((e = cudaGraphConditionalHandleCreate(&ctl.ru, body, 0, 0))) break;
        // loop body: the three iteration kernels, then IF (reliable update)
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed))) break;
        for (int u = 0; u < QEX_GRAPH_UNROLL && !st; ++u) st = enqueue_iteration(s, ctl, cs);
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
        // IF body: the reliable update
        if ((e = cudaStreamBeginCaptureToGraph(cs, ip.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeRelaxed)))
            break;
        st = enqueue_reliable_update(s, ctl, cs);
        e2 = cudaStreamEndCapture(cs, &captured);
        if (st) break;
        if ((e = e2)) break;
        if ((e = cudaGraphInstantiate(&G->exec, G->graph, 0))) break;
    } while (0);
    set_count_launches(true);
    if (cs) cudaStreamDestroy(cs);
    if (st || e) {
        drop_graph(G);
        if (!st) st = cuda_fail(e, "building the CG graph");
        return st;
    }
    *out = G;
    return QEX_OK;
}

void free_cg_graph(void *g) { drop_graph((CgGraph *)g); }

}  // namespace qex

using namespace qex;

extern "C" qex_status qex_cg(const qex_lattice *latc, qex_prec inner, const void *fat64, const void *lng64,
                             const void *fat32, const void *lng32, double c_naik, double mass, const void *b64,
                             void *x64, double tol, int maxiter, double delta, void *stream,
                             qex_cg_stats *stats) {
    qex_status st;
    if ((st = check_lattice(latc)) || (st = check_prec(inner))) return st;
    const bool mixed = inner != QEX_F64;
    if ((st = check_dslash_args(latc, QEX_F64, fat64, lng64, b64, x64))) return st;
    if (mixed) {
        if (!fat32 || !aligned16(fat32) || (lng64 && (!lng32 || !aligned16(lng32)))) {
            set_error("mixed precision needs aligned FP32 copies of the fat (and long) links");
            return QEX_ERR_ARG;
        }
    }
    if (!(tol > 0.0) || maxiter < 0 || !(delta >= 0.0 && delta < 1.0)) {
        set_error("need tol > 0, maxiter >= 0 and 0 <= delta < 1");
        return QEX_ERR_ARG;
    }
    qex_lattice *lat = const_cast<qex_lattice *>(latc);
    if ((st = ensure_scratch(lat))) return st;
    if (!lat->scalars_host2) QEX_CUDA(cudaMallocHost(&lat->scalars_host2, sizeof(CgScalars)));
    // small lattices default to the persistent fused iteration (1.15-1.3x
    // faster per iteration up to 16^4); QEX_CG_MODE=graph|host|fused forces
    const char *mode = getenv("QEX_CG_MODE");
    const bool use_fused = mixed && ((mode && strcmp(mode, "fused") == 0) || (!mode && lat->vh <= kFusedAutoMaxVh));
    const bool use_graph = !(mode && (strcmp(mode, "host") == 0 || use_fused));

    Solve s;
    s.lat = lat;
    s.mixed = mixed;
    s.ff_ok = ru_ff_enabled(mixed);
    s.inner = inner;
    s.fat64 = fat64;
    s.lng64 = lng64;
    s.fat32 = mixed ? fat32 : nullptr;
    s.lng32 = mixed ? lng32 : nullptr;
    s.c3 = c_naik;
    s.m2 = mass * mass;
    s.b64 = (const double *)b64;
    s.x64 = (double *)x64;
    s.defer_x = mixed && !use_fused && QEX_DEFER_X != 0;  // the fused kernel updates x itself
    const cudaStream_t cst = as_stream(stream);
    // launch shapes of the inner iteration and of the FP64 reliable updates,
    // before the graph bakes them in (the vector kernels keep their compiled
    // grid: timed alone on L2-resident scratch they favour grids that are
    // slower inside the solve)
    if ((st = ensure_tuned(lat, inner, mixed ? fat32 : fat64, mixed ? lng32 : lng64, cst, false))) return st;
    if (mixed && (st = ensure_tuned(lat, QEX_F64, fat64, lng64, cst, false))) return st;
    if ((st = carve(lat, mixed, s.B))) return st;
    // programmatic dependent launch: on for the host-driven loop (measured
    // 0.5 ms faster on the 32^4 workload), off in the graph solve (1.0 ms
    // slower with programmatic edges); QEX_PDL=1 or 0 forces either way, and a
    // graph with programmatic edges that cannot be built falls back to plain
    // launches
    struct PdlScope {
        qex_lattice *l;
        ~PdlScope() { l->pdl = 0; }
    } pdl_scope{lat};
    static bool pdl_graph_failed = false;  // a graph with programmatic edges could not be built once
    const char *pdl_env = getenv("QEX_PDL");
    if (pdl_env && (strcmp(pdl_env, "0") == 0 || strcmp(pdl_env, "1") == 0))
        lat->pdl = pdl_env[0] == '1' ? 1 : 0;
    else
        lat->pdl = use_graph ? 0 : 1;
    if (use_graph && pdl_graph_failed) lat->pdl = 0;
    if (use_graph && !same_key((CgGraph *)lat->cg_graph, s)) {
        QEX_CUDA(cudaStreamSynchronize(cst));
        drop_graph((CgGraph *)lat->cg_graph);
        lat->cg_graph = nullptr;
        CgGraph *G;
        st = build_graph(s, &G);
        if (st && lat->pdl) {
            cudaGetLastError();
            pdl_graph_failed = true;
            lat->pdl = 0;
            st = build_graph(s, &G);
        }
        if (st) return st;
        lat->cg_graph = G;
    }

    cudaEvent_t t0, t1;
    QEX_CUDA(cudaEventCreate(&t0));
    QEX_CUDA(cudaEventCreate(&t1));
    QEX_CUDA(cudaEventRecord(t0, cst));

    CgScalars init;
    memset(&init, 0, sizeof(init));
    init.tol2 = tol * tol;
    init.delta2 = mixed ? delta * delta : 0.0;
    init.max_cycle = ru_max_cycle(inner);
    init.ff_ok = s.ff_ok ? 1 : 0;
    init.maxiter = maxiter;
    CgScalars *h0 = lat->scalars_host, *h1 = lat->scalars_host2;
    QEX_CUDA(cudaStreamSynchronize(cst));  // the pinned slots are free
    *h0 = init;
    QEX_CUDA(cudaMemcpyAsync(lat->scalars, h0, sizeof(CgScalars), cudaMemcpyHostToDevice, cst));
    size_t fbytes = (size_t)lat->vh * (mixed ? 24 : 48);
    for (int k = 0; k < 2; ++k)
        QEX_CUDA(cudaMemsetAsync(mixed ? (void *)s.B.p32[k] : (void *)s.B.p64[k], 0, fbytes, cst));
    if (mixed) QEX_CUDA(cudaMemsetAsync(s.B.xh32, 0, fbytes, cst));
    const GraphCtl off = {};
    if ((st = launch_norm2(lat, QEX_F64, b64, nullptr, lat->scalars, cst))) return st;
    if ((st = launch_any_nonzero(lat, (const double *)x64, &lat->scalars->x_nonzero, cst))) return st;
    if ((st = enqueue_reliable_update(s, off, cst, true))) return st;
    if ((st = fetch_scalars(lat, 0, cst)) || (st = wait_scalars(lat, 0))) return st;

    qex_status result = QEX_OK;
    CgScalars cur = *h0;
    if (cur.bb == 0.0) {
        QEX_CUDA(cudaMemsetAsync(x64, 0, (size_t)lat->vh * 48, cst));
        cur.done = 1;
        cur.true_rr = 0.0;
    } else if (!isfinite(cur.bb) || cur.error) {
        set_error("NaN/Inf in the source or the initial residual");
        result = QEX_ERR_NAN;
    } else if (!cur.done && !cur.halt && use_graph) {
        CgGraph *G = (CgGraph *)lat->cg_graph;
        QEX_CUDA(cudaGraphLaunch(G->exec, cst));
        if ((st = fetch_scalars(lat, 0, cst)) || (st = wait_scalars(lat, 0))) return st;
        cur = *h0;
        const unsigned long long rus = cur.reliable_updates > 1 ? cur.reliable_updates - 1 : 0;
        note_launches(G->kernels_per_iter * (unsigned long long)(cur.trips + cur.idle_iters) +
                      G->kernels_per_ru * rus);
    } else if (!cur.done && !cur.halt && use_fused) {
        // persistent inner iterations, FP64 reliable updates in between
        while (!cur.done && !cur.error) {
            if ((st = launch_cg_fused(lat, inner, s.fat32, s.lng32, s.c3, s.m2, s.B.xh32, s.B.r32, s.B.p32, s.B.ap32,
                                      s.B.tmp32, cst)))
                return st;
            int timed_out = 0, exited = 0;
            if ((st = fused_barrier_status(lat, cst, &timed_out, &exited))) return st;
            if (timed_out) {
                set_error("fused CG: a grid barrier timed out (%d of %d blocks left the kernel)", exited,
                          lat->fused_blocks);
                result = QEX_ERR_TIMEOUT;
                break;
            }
            if ((st = fetch_scalars(lat, 0, cst)) || (st = wait_scalars(lat, 0))) return st;
            cur = *h0;
            if (cur.error || !cur.need_ru) break;
            if ((st = enqueue_reliable_update(s, off, cst))) return st;
            if ((st = fetch_scalars(lat, 0, cst)) || (st = wait_scalars(lat, 0))) return st;
            cur = *h0;
            if (!cur.done && !cur.error && cur.iters >= maxiter) break;
        }
    } else if (!cur.done && !cur.halt) {
        const int batch = 8;
        while (!cur.done && !cur.error) {
            // iterate until a kernel halts; slot k&1 holds the scalars after batch k
            int k = 0;
            for (int j = 0; j < batch; ++j)
                if ((st = enqueue_iteration(s, off, cst))) return st;
            if ((st = fetch_scalars(lat, 0, cst))) return st;
            for (;;) {
                for (int j = 0; j < batch; ++j)
                    if ((st = enqueue_iteration(s, off, cst))) return st;
                if ((st = fetch_scalars(lat, (k + 1) & 1, cst))) return st;
                if ((st = wait_scalars(lat, k & 1))) return st;
                cur = (k & 1) ? *h1 : *h0;
                ++k;
                if (cur.halt) break;
            }
            if ((st = wait_scalars(lat, k & 1))) return st;  // drain the queued batch
            cur = (k & 1) ? *h1 : *h0;
            if (cur.error || !cur.need_ru) break;
            if ((st = enqueue_reliable_update(s, off, cst))) return st;
            if ((st = fetch_scalars(lat, 0, cst)) || (st = wait_scalars(lat, 0))) return st;
            cur = *h0;
            if (!cur.done && !cur.error && cur.iters >= maxiter) break;
        }
    }
    if (result == QEX_OK && !cur.done) {
        if (cur.error) {
            set_error(cur.error == 2 ? "CG breakdown: <p, A p> <= 0" : "NaN/Inf in a CG reduction");
            result = QEX_ERR_NAN;
        } else if (cur.iters >= maxiter) {
            set_error("CG did not converge in %d iterations", maxiter);
            result = QEX_ERR_NOT_CONVERGED;
        } else {
            set_error("internal error: CG stopped without a reason (iters %d, trips %d)", cur.iters, cur.trips);
            result = QEX_ERR_ARG;
        }
    }
    QEX_CUDA(cudaEventRecord(t1, cst));
    QEX_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (stats) {
        stats->iters = cur.iters;
        stats->reliable_updates = cur.reliable_updates > 0 ? cur.reliable_updates - 1 : 0;
        stats->converged = cur.done;
        stats->ff_updates = cur.ff_updates;
        stats->true_rel_resid = cur.bb > 0.0 ? sqrt(cur.true_rr / cur.bb) : 0.0;
        stats->time_ms = ms;
    }
    return result;
}

// Device time of each kernel of the CG iteration, measured inside a solve:
// the same set-up as qex_cg (initial FP64 residual), then `iters` iterations
// of exactly the kernels the solve runs, in its order and with its launch
// shapes, enqueued back to back with an event after every kernel.  The stop
// test is disabled (tol 0, no reliable update before `iters`), so every
// timed kernel does its full work.
extern "C" qex_status qex_cg_profile(const qex_lattice *latc, qex_prec inner, const void *fat64, const void *lng64,
                                     const void *fat32, const void *lng32, double c_naik, double mass,
                                     const void *b64, void *x64, int iters, void *stream, double *ms_out,
                                     int *n_out) {
    qex_status st;
    if ((st = check_lattice(latc)) || (st = check_prec(inner))) return st;
    const bool mixed = inner != QEX_F64;
    if ((st = check_dslash_args(latc, QEX_F64, fat64, lng64, b64, x64))) return st;
    if (mixed && (!fat32 || !aligned16(fat32) || (lng64 && (!lng32 || !aligned16(lng32))))) {
        set_error("mixed precision needs aligned FP32 copies of the fat (and long) links");
        return QEX_ERR_ARG;
    }
    if (iters < 3 || iters > 10000 || !ms_out || !n_out) {
        set_error("need 3 <= iters <= 10000 and non-NULL ms_out, n_out");
        return QEX_ERR_ARG;
    }
    qex_lattice *lat = const_cast<qex_lattice *>(latc);
    if ((st = ensure_scratch(lat))) return st;
    Solve s;
    s.lat = lat;
    s.mixed = mixed;
    s.ff_ok = ru_ff_enabled(mixed);
    s.inner = inner;
    s.fat64 = fat64;
    s.lng64 = lng64;
    s.fat32 = mixed ? fat32 : nullptr;
    s.lng32 = mixed ? lng32 : nullptr;
    s.c3 = c_naik;
    s.m2 = mass * mass;
    s.b64 = (const double *)b64;
    s.x64 = (double *)x64;
    s.defer_x = mixed && QEX_DEFER_X != 0;
    const cudaStream_t cst = as_stream(stream);
    if ((st = ensure_tuned(lat, inner, mixed ? fat32 : fat64, mixed ? lng32 : lng64, cst, false))) return st;
    if (mixed && (st = ensure_tuned(lat, QEX_F64, fat64, lng64, cst, false))) return st;
    if ((st = carve(lat, mixed, s.B))) return st;
    lat->pdl = 0;  // an event between kernels would cut programmatic overlap anyway
    CgScalars init;
    memset(&init, 0, sizeof(init));
    init.tol2 = 0.0;    // never met: every iteration runs
    init.delta2 = 0.0;  // no reliable update
    init.maxiter = iters;
    QEX_CUDA(cudaStreamSynchronize(cst));
    *lat->scalars_host = init;
    QEX_CUDA(cudaMemcpyAsync(lat->scalars, lat->scalars_host, sizeof(CgScalars), cudaMemcpyHostToDevice, cst));
    const size_t fbytes = (size_t)lat->vh * (mixed ? 24 : 48);
    for (int k = 0; k < 2; ++k)
        QEX_CUDA(cudaMemsetAsync(mixed ? (void *)s.B.p32[k] : (void *)s.B.p64[k], 0, fbytes, cst));
    if (mixed) QEX_CUDA(cudaMemsetAsync(s.B.xh32, 0, fbytes, cst));
    const GraphCtl off = {};
    if ((st = launch_norm2(lat, QEX_F64, b64, nullptr, lat->scalars, cst))) return st;
    if ((st = launch_any_nonzero(lat, (const double *)x64, &lat->scalars->x_nonzero, cst))) return st;
    if ((st = enqueue_reliable_update(s, off, cst, true))) return st;
    if ((st = fetch_scalars(lat, 0, cst)) || (st = wait_scalars(lat, 0))) return st;
    if (!(lat->scalars_host->bb > 0.0) || !isfinite(lat->scalars_host->bb)) {
        set_error("qex_cg_profile needs a non-zero, finite source");
        return QEX_ERR_ARG;
    }
    const int nk = mixed ? 3 : 4;
    const int nev = iters * nk + 1;
    cudaEvent_t *ev = new cudaEvent_t[nev];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < nev && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e != cudaSuccess) --made;
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], cst);
    for (int it = 0; it < iters && e == cudaSuccess && !st; ++it) {
        Marks m = {ev + 1 + it * nk, nk};
        st = enqueue_iteration(s, off, cst, &m);
    }
    if (e == cudaSuccess && !st) e = cudaEventSynchronize(ev[nev - 1]);
    if (e == cudaSuccess && !st) {
        // average over all but the first two iterations
        for (int j = 0; j < nk; ++j) ms_out[j] = 0.0;
        for (int it = 2; it < iters; ++it)
            for (int j = 0; j < nk; ++j) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[it * nk + j], ev[it * nk + j + 1]);
                ms_out[j] += ms;
            }
        for (int j = 0; j < nk; ++j) ms_out[j] /= (iters - 2);
        *n_out = nk;
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    delete[] ev;
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "qex_cg_profile events");
    return QEX_OK;
}

// ------------------------------------------------------ true residual

// ||b - A x|| / ||b|| in FP64 or in the float-float arithmetic of the
// intermediate reliable updates, with the update's own kernels.
extern "C" qex_status qex_true_residual(const qex_lattice *latc, const void *fat64, const void *lng64, double c_naik,
                                        double mass, const void *b64, const void *x64, int arith, double *rel_resid,
                                        void *stream) {
    qex_status st;
    if ((st = check_lattice(latc))) return st;
    if ((st = check_dslash_args(latc, QEX_F64, fat64, lng64, b64, x64))) return st;
    if (!rel_resid || (arith != 0 && arith != 1)) {
        set_error("need rel_resid and arith 0 (FP64) or 1 (float-float)");
        return QEX_ERR_ARG;
    }
    qex_lattice *lat = const_cast<qex_lattice *>(latc);
    if ((st = ensure_scratch(lat))) return st;
    const size_t f64 = align256((size_t)lat->vh * 48);
    if ((st = ensure_work(lat, 2 * f64))) return st;
    char *w = (char *)lat->work;
    void *tmp = w, *r = w + f64;
    const cudaStream_t cst = as_stream(stream);
    CgScalars init;
    memset(&init, 0, sizeof(init));
    QEX_CUDA(cudaStreamSynchronize(cst));  // the pinned slot is free
    *lat->scalars_host = init;
    QEX_CUDA(cudaMemcpyAsync(lat->scalars, lat->scalars_host, sizeof(CgScalars), cudaMemcpyHostToDevice, cst));
    if ((st = launch_norm2(lat, QEX_F64, b64, nullptr, lat->scalars, cst))) return st;
    if (arith == 0) {
        DslashArgs a = {};
        a.prec = QEX_F64;
        a.fat = fat64;
        a.lng = lng64;
        a.c3 = c_naik;
        a.out_parity = 1;
        a.in = x64;
        a.out = tmp;
        a.epi = EPI_PLAIN;
        a.S = lat->scalars;
        if ((st = launch_dslash(lat, a, cst))) return st;
        a.out_parity = 0;
        a.in = tmp;
        a.out = r;
        a.epi = EPI_RESID;
        a.q = x64;
        a.b = (const double *)b64;
        a.m2 = mass * mass;
        if ((st = launch_dslash(lat, a, cst))) return st;
    } else {
        if ((st = launch_ru_ff(lat, 1, (const double *)fat64, (const double *)lng64, c_naik, mass * mass,
                               (const double *)x64, nullptr, tmp, nullptr, lat->scalars, false, true, cst)))
            return st;
        if ((st = launch_ru_ff(lat, 2, (const double *)fat64, (const double *)lng64, c_naik, mass * mass,
                               (const double *)x64, (const double *)b64, tmp, (float *)r, lat->scalars, false, true,
                               cst)))
            return st;
    }
    QEX_CUDA(cudaMemcpyAsync(lat->scalars_host, lat->scalars, sizeof(CgScalars), cudaMemcpyDeviceToHost, cst));
    QEX_CUDA(cudaStreamSynchronize(cst));
    const CgScalars &h = *lat->scalars_host;
    if (!isfinite(h.bb) || !isfinite(h.true_rr)) {
        set_error("NaN/Inf in the residual");
        return QEX_ERR_NAN;
    }
    *rel_resid = h.bb > 0.0 ? sqrt(h.true_rr / h.bb) : 0.0;
    return QEX_OK;
}
