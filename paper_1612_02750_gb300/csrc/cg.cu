// cg.cu -- conjugate gradient on A = m^2 - D_eo D_oe (even sites): plain FP64
// and mixed precision with reliable updates.
//
// The iteration keeps alpha, beta and the residual norms on the device: each
// iteration is four launches (D_oe p; A p with <p, A p>; x, r update with
// ||r||^2; p update) and none reads anything back.  The host enqueues batches
// of iterations and reads the scalars once per batch, double-buffered so that
// the next batch is already queued while the previous flags travel back.
// Once a kernel sets `halt` (convergence candidate, reliable update due,
// iteration cap, NaN), the remaining queued iteration kernels return at once.
//
// Mixed precision (inner = F32): x_hat, r_hat, p, A p live in FP32 and the
// operator runs on FP32 links; when ||r_hat|| falls below delta times its
// largest value since the last update, or meets tol, the host runs a reliable
// update: x += x_hat (FP64), r = b - A x with the FP64 operator, r_hat =
// (float) r, beta from the true ||r||^2, p kept.  Convergence is only ever
// accepted on the FP64 true residual.
#include <math.h>
#include <string.h>

#include "qex_kernels.cuh"

namespace qex {

qex_status check_dslash_args(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                             const void *in, const void *out);

static size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

struct CgBuffers {
    double *r64, *p64, *ap64, *tmp64;
    float *xh32, *r32, *p32, *ap32, *tmp32;
};

static qex_status carve(qex_lattice *lat, bool mixed, CgBuffers &B) {
    size_t f64 = align256((size_t)lat->vh * 48), f32 = align256((size_t)lat->vh * 24);
    size_t need = mixed ? 2 * f64 + 5 * f32 : 4 * f64;
    qex_status st = ensure_work(lat, need);
    if (st) return st;
    char *w = (char *)lat->work;
    memset(&B, 0, sizeof(B));
    B.r64 = (double *)w;
    w += f64;
    B.tmp64 = (double *)w;
    w += f64;
    if (mixed) {
        B.xh32 = (float *)w;
        w += f32;
        B.r32 = (float *)w;
        w += f32;
        B.p32 = (float *)w;
        w += f32;
        B.ap32 = (float *)w;
        w += f32;
        B.tmp32 = (float *)w;
    } else {
        B.p64 = (double *)w;
        w += f64;
        B.ap64 = (double *)w;
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
    CgBuffers B;
    cudaStream_t st;
};

// One CG iteration in the inner precision, every kernel halt-checked.
static qex_status enqueue_iteration(Solve &s) {
    qex_lattice *lat = s.lat;
    CgScalars *S = lat->scalars;
    DslashArgs a = {};
    a.prec = s.inner;
    a.fat = s.mixed ? s.fat32 : s.fat64;
    a.lng = s.mixed ? s.lng32 : s.lng64;
    a.c3 = s.c3;
    a.S = S;
    a.check_halt = 1;
    void *p = s.mixed ? (void *)s.B.p32 : (void *)s.B.p64;
    void *tmp = s.mixed ? (void *)s.B.tmp32 : (void *)s.B.tmp64;
    void *ap = s.mixed ? (void *)s.B.ap32 : (void *)s.B.ap64;
    void *x = s.mixed ? (void *)s.B.xh32 : (void *)s.x64;
    void *r = s.mixed ? (void *)s.B.r32 : (void *)s.B.r64;
    qex_status st;
    a.out_parity = 1;
    a.in = p;
    a.out = tmp;
    a.epi = EPI_PLAIN;
    if ((st = launch_dslash(lat, a, s.st))) return st;
    a.out_parity = 0;
    a.in = tmp;
    a.out = ap;
    a.epi = EPI_NORMAL;
    a.q = p;
    a.m2 = s.m2;
    if ((st = launch_dslash(lat, a, s.st))) return st;
    if ((st = launch_update_xr(lat, a.prec, x, r, p, ap, S, s.st))) return st;
    return launch_update_p(lat, a.prec, r, p, S, 1, s.st);
}

// FP64 true residual r64 = b - A x64 (after folding x_hat into x64), then the
// inner residual and search direction from it.
static qex_status enqueue_reliable_update(Solve &s) {
    qex_lattice *lat = s.lat;
    CgScalars *S = lat->scalars;
    qex_status st;
    if (s.mixed && (st = launch_accum_x(lat, s.x64, s.B.xh32, s.st))) return st;
    DslashArgs a = {};
    a.prec = QEX_F64;
    a.fat = s.fat64;
    a.lng = s.lng64;
    a.c3 = s.c3;
    a.out_parity = 1;
    a.in = s.x64;
    a.out = s.B.tmp64;
    a.epi = EPI_PLAIN;
    if ((st = launch_dslash(lat, a, s.st))) return st;
    a.out_parity = 0;
    a.in = s.B.tmp64;
    a.out = s.B.r64;
    a.epi = EPI_RESID;
    a.q = s.x64;
    a.b = s.b64;
    a.m2 = s.m2;
    a.S = S;
    if ((st = launch_dslash(lat, a, s.st))) return st;
    if (s.mixed) return launch_lower_r_update_p(lat, s.B.r64, s.B.r32, s.B.p32, S, s.st);
    return launch_update_p(lat, QEX_F64, s.B.r64, s.B.p64, S, 0, s.st);
}

static qex_status fetch_scalars(Solve &s, int slot) {
    QEX_CUDA(cudaMemcpyAsync(slot ? s.lat->scalars_host2 : s.lat->scalars_host, s.lat->scalars,
                             sizeof(CgScalars), cudaMemcpyDeviceToHost, s.st));
    QEX_CUDA(cudaEventRecord(slot ? s.lat->ev1 : s.lat->ev0, s.st));
    return QEX_OK;
}

static qex_status wait_scalars(Solve &s, int slot) {
    QEX_CUDA(cudaEventSynchronize(slot ? s.lat->ev1 : s.lat->ev0));
    return QEX_OK;
}

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
    // two pinned scalar slots for the double-buffered readback
    if (!lat->scalars_host2) QEX_CUDA(cudaMallocHost(&lat->scalars_host2, sizeof(CgScalars)));

    Solve s;
    s.lat = lat;
    s.mixed = mixed;
    s.inner = inner;
    s.fat64 = fat64;
    s.lng64 = lng64;
    s.fat32 = fat32;
    s.lng32 = mixed ? lng32 : nullptr;
    s.c3 = c_naik;
    s.m2 = mass * mass;
    s.b64 = (const double *)b64;
    s.x64 = (double *)x64;
    s.st = as_stream(stream);
    if ((st = carve(lat, mixed, s.B))) return st;

    cudaEvent_t t0, t1;
    QEX_CUDA(cudaEventCreate(&t0));
    QEX_CUDA(cudaEventCreate(&t1));
    QEX_CUDA(cudaEventRecord(t0, s.st));

    CgScalars init;
    memset(&init, 0, sizeof(init));
    init.tol2 = tol * tol;
    init.delta2 = mixed ? delta * delta : 0.0;
    init.maxiter = maxiter;
    CgScalars *h0 = lat->scalars_host, *h1 = lat->scalars_host2;
    QEX_CUDA(cudaStreamSynchronize(s.st));  // the pinned slots are free
    *h0 = init;
    QEX_CUDA(cudaMemcpyAsync(lat->scalars, h0, sizeof(CgScalars), cudaMemcpyHostToDevice, s.st));
    size_t fbytes = (size_t)lat->vh * (mixed ? 24 : 48);
    QEX_CUDA(cudaMemsetAsync(mixed ? (void *)s.B.p32 : (void *)s.B.p64, 0, fbytes, s.st));
    if (mixed) QEX_CUDA(cudaMemsetAsync(s.B.xh32, 0, fbytes, s.st));
    if ((st = launch_norm2(lat, QEX_F64, b64, nullptr, lat->scalars, s.st))) return st;
    if ((st = enqueue_reliable_update(s))) return st;
    QEX_CUDA(cudaMemcpyAsync(h0, lat->scalars, sizeof(CgScalars), cudaMemcpyDeviceToHost, s.st));
    QEX_CUDA(cudaStreamSynchronize(s.st));

    qex_status result = QEX_OK;
    CgScalars cur = *h0;
    if (cur.bb == 0.0) {
        QEX_CUDA(cudaMemsetAsync(x64, 0, (size_t)lat->vh * 48, s.st));
        cur.done = 1;
        cur.true_rr = 0.0;
    } else if (!isfinite(cur.bb) || cur.error) {
        set_error("NaN/Inf in the source or the initial residual");
        result = QEX_ERR_NAN;
    } else {
        const int batch = 8;
        while (!cur.done && !cur.error) {
            if (cur.halt) {
                if (cur.iters >= maxiter) {
                    set_error("CG did not converge in %d iterations", maxiter);
                    result = QEX_ERR_NOT_CONVERGED;
                    break;
                }
            }
            // iterate until a kernel halts; slot k&1 holds the scalars after batch k
            int k = 0;
            for (int j = 0; j < batch; ++j)
                if ((st = enqueue_iteration(s))) return st;
            if ((st = fetch_scalars(s, 0))) return st;
            for (;;) {
                for (int j = 0; j < batch; ++j)
                    if ((st = enqueue_iteration(s))) return st;
                if ((st = fetch_scalars(s, (k + 1) & 1))) return st;
                if ((st = wait_scalars(s, k & 1))) return st;
                cur = (k & 1) ? *h1 : *h0;
                ++k;
                if (cur.halt) break;
            }
            if ((st = wait_scalars(s, k & 1))) return st;  // drain the queued batch
            cur = (k & 1) ? *h1 : *h0;
            if (cur.error) break;
            if (!cur.need_ru) {  // halt without a cause: never set by the kernels
                set_error("internal error: CG halted without a reason");
                result = QEX_ERR_ARG;
                break;
            }
            if ((st = enqueue_reliable_update(s))) return st;
            if ((st = fetch_scalars(s, 0))) return st;
            if ((st = wait_scalars(s, 0))) return st;
            cur = *h0;
            if (!cur.done && !cur.error && cur.iters >= maxiter) {
                set_error("CG did not converge in %d iterations", maxiter);
                result = QEX_ERR_NOT_CONVERGED;
                break;
            }
        }
        if (cur.error && result == QEX_OK) {
            set_error(cur.error == 2 ? "CG breakdown: <p, A p> <= 0" : "NaN/Inf in a CG reduction");
            result = QEX_ERR_NAN;
        }
    }
    QEX_CUDA(cudaEventRecord(t1, s.st));
    QEX_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (stats) {
        stats->iters = cur.iters;
        stats->reliable_updates = cur.reliable_updates > 0 ? cur.reliable_updates - 1 : 0;
        stats->converged = cur.done;
        stats->reserved = 0;
        stats->true_rel_resid = cur.bb > 0.0 ? sqrt(cur.true_rr / cur.bb) : 0.0;
        stats->time_ms = ms;
    }
    return result;
}
