// qex_kernels.cuh -- device-resident CG state and the host launchers that the
// translation units of libqex_gpu share.
#pragma once

#include <cstdlib>

#include "qex_common.cuh"

namespace qex {

// CG scalars live in device memory so that an iteration needs no host round
// trip; the last block of each reducing kernel updates them (fixed-order sum
// of the per-block partials, so results are bit-reproducible).
struct CgScalars {
    double rr;        // ||r||^2 of the iterated residual (FP64 accumulation)
    double pAp;       // Re <p, A p>
    double alpha;     // rr / pAp
    double beta;      // rr_new / rr (used by the next direction update)
    double bb;        // ||b||^2
    double tol2;      // tol^2
    double stop2;     // tol^2 * bb
    double delta2;    // reliable-update threshold factor delta^2 (0: only at convergence)
    double rmax2;     // max ||r||^2 since the last reliable update
    double true_rr;   // ||b - A x||^2 from the last FP64 recomputation
    int max_cycle;    // > 0: a reliable update also follows max_cycle inner iterations without one
    int ru_iter0;     // iteration count at the last reliable update
    int ff_ok;        // intermediate reliable updates may run in float-float arithmetic (ru_ff.cu)
    int ru_ff;        // the pending reliable update runs in float-float arithmetic
    int ff_k;         // float-float updates carry the vectors times 2^ff_k (set with bb)
    double rr_ru;     // iterated ||r||^2 when the pending reliable update was asked for
    int ff_updates;   // reliable updates made in float-float arithmetic
    int idle_iters;   // iterations whose kernels found the solve halted (queued or graph-unrolled)
    int iters;        // completed iterations; its parity selects the current p buffer
    int maxiter;
    int done;         // true residual met tol
    int need_ru;      // iterated residual calls for an FP64 recomputation
    int halt;         // done | need_ru | error: iteration kernels return at once
    int error;        // 1: NaN/Inf in a reduction, 2: <p, Ap> <= 0
    int reliable_updates;
    int trips;        // executions of the update kernel (graph loop guard)
    int x_nonzero;    // the initial guess has an element != 0 (or NaN); 0: the first residual is b
};

// The CG scalars after a true residual ||b - A x||^2 = tot (last block of the
// residual kernel, one thread).  `may_accept`: the residual was computed in
// FP64 and may end the solve; a float-float one never does (the next update
// that the iterated residual asks for at tol is an FP64 one).
__device__ __forceinline__ void take_true_residual(CgScalars *S, double tot, bool may_accept) {
    S->true_rr = tot;
    S->reliable_updates += 1;
    if (!may_accept) S->ff_updates += 1;
    if (!isfinite(tot)) {
        S->error = 1;
        S->halt = 1;
        return;
    }
    S->ru_iter0 = S->iters;
    S->beta = S->rr > 0.0 ? tot / S->rr : 0.0;
    S->rr = tot;
    S->rmax2 = tot;
    S->need_ru = 0;
    S->done = (may_accept && tot <= S->stop2) ? 1 : 0;
    S->halt = (S->done || S->iters >= S->maxiter) ? 1 : 0;
}

// Reliable updates in float-float arithmetic (ru_ff.cu): `stage` 1 writes
// tmp = D_oe x64 (float pairs, 48 bytes a site), stage 2 r32 = b - m^2 x64 +
// D_eo tmp rounded to FP32 and ||r||^2 (cg: the CG scalars as an update,
// else only true_rr).  Unless `force`, both return at once when S->ru_ff is 0.
qex_status launch_ru_ff(qex_lattice *lat, int stage, const double *fat64, const double *lng64, double c3,
                        double m2, const double *x64, const double *b64, void *tmp, float *r32, CgScalars *S,
                        bool cg, bool force, cudaStream_t st);

// CG iterations per trip of a CUDA-graph solve's WHILE node (single lattice and batched).  Evaluating the loop and
// IF conditions costs a few microseconds a trip; the iterations after one
// that asks for a reliable update in the same trip find the solve halted and
// return at once.  32^4 solve: 20.87-20.91 ms (1), 20.44 (2), 19.82-19.83
// (4), 19.74-19.75 (8), the last two on a faster box.
#ifndef QEX_GRAPH_UNROLL
#define QEX_GRAPH_UNROLL 8
#endif

// Inner iterations after which a mixed-precision solve makes a reliable
// update even when the iterated residual has not yet dropped by delta.  Over
// a long cycle (thousands of iterations at small mass) the recursion residual
// of the inner precision drifts away from b - A x, and the iteration keeps
// reducing a residual that is no longer the true one; a bounded cycle resets
// it to the FP64 true residual often enough.  16-bit links (step 2^-15) drift
// faster than FP32 ones, hence the shorter cycle.  QEX_RU_CYCLE=<n> overrides
// both, 0 turns the bound off.
constexpr int kRuCycle16 = 100, kRuCycle32 = 500;
inline int ru_max_cycle(qex_prec inner) {
    if (inner == QEX_F64) return 0;
    const char *e = getenv("QEX_RU_CYCLE");
    if (!e || !*e) return (inner == QEX_F32_R12H || inner == QEX_F32_S16) ? kRuCycle16 : kRuCycle32;
    const int v = atoi(e);
    return v > 0 ? v : 0;
}

// Conditional-node handles of the CUDA-graph solve (active = 0 outside it).
// The loop never runs more than maxiter + 4 trips (CgScalars::trips).
struct GraphCtl {
    int active;
    cudaGraphConditionalHandle loop;  // while: run another iteration
    cudaGraphConditionalHandle ru;    // if: run a reliable update now
};

// Epilogues / variants of the Dslash kernel.
enum Epilogue {
    EPI_PLAIN = 0,   // out = D in
    EPI_NORMAL = 1,  // out = m^2 q - D in; Re<q, out> -> pAp, alpha   (CG: q = new p)
    EPI_RESID = 2,   // out = b - m^2 q + D in; ||out||^2 -> true_rr, flags (CG: q = x), FP64 only
    EPI_PUPD = 3     // in = r + beta p_old (formed on the fly), out = D in, p_new = r + beta p_old stored
};

struct DslashArgs {
    qex_prec prec;
    const void *fat;
    const void *lng;     // NULL: no Naik term
    double c3;
    int out_parity;
    const void *in;      // EPI_PLAIN / NORMAL / RESID
    void *out;
    int epi;
    const void *q;       // EPI_NORMAL / EPI_RESID (ignored when psel)
    const double *b;     // EPI_RESID (FP64 half field)
    double m2;
    CgScalars *S;        // EPI_NORMAL / EPI_RESID / halt check / buffer selection
    int check_halt;
    // CG direction ping-pong: p_old = pbuf[iters & 1], p_new = pbuf[(iters + 1) & 1]
    const void *r;       // EPI_PUPD
    void *x;             // EPI_PUPD: iterate that takes the pending alpha p_old (NULL: none)
    void *pbuf[2];       // EPI_PUPD, and EPI_PLAIN / EPI_NORMAL when psel
    int psel;            // EPI_PLAIN: in = p_new; EPI_NORMAL: q = p_new
    int reverse;         // visit the sites from the last index down (the second Dslash of a CG
                         // iteration meets the links the first one read last while they are in L2)
    int skip_zero_x;     // EPI_PLAIN / EPI_RESID of the first residual: unless S->x_nonzero,
                         // PLAIN writes nothing and RESID takes D in = 0 (r = b)
    int skip_ff;         // EPI_PLAIN / EPI_RESID of a mixed solve's update: return at once when
                         // S->ru_ff (the float-float kernels run it)
};

qex_status launch_dslash(qex_lattice *lat, const DslashArgs &a, cudaStream_t st);

// ------------------------------------------------------------ multi-RHS CG
// Per-right-hand-side CG scalars (all active right-hand sides iterate in
// lockstep; a converged one is frozen by its `active` flag).
constexpr int kMaxRhs = QEX_MRHS_MAX;
struct MrhsScalars {
    double rr[kMaxRhs], pAp[kMaxRhs], alpha[kMaxRhs], beta[kMaxRhs], bb[kMaxRhs], stop2[kMaxRhs],
        rmax2[kMaxRhs], true_rr[kMaxRhs];
    int active[kMaxRhs];   // still iterating
    int done[kMaxRhs];     // true residual met tol
    int iters[kMaxRhs];    // iterations while active
    double tol2, delta2;
    int nrhs;
    int iter;              // lockstep iteration count: its parity selects the p buffers
    int maxiter;
    int max_cycle;         // > 0: a reliable update also follows max_cycle iterations without one
    int ru_iter0;          // iter at the last reliable update
    int need_ru, halt, error;
    int reliable_updates;
    int nactive;
};

struct MrhsArgs {
    qex_prec prec;
    const void *fat, *lng;
    double c3;
    int out_parity;
    int nrhs;
    const void *in;       // EPI_PLAIN / EPI_NORMAL / EPI_RESID input fields
    void *out;
    int epi;
    const void *q;        // EPI_RESID: x fields
    const double *b;      // EPI_RESID: b fields (FP64)
    double m2;
    MrhsScalars *S;       // NULL: plain application, no masking
    const void *r;        // EPI_PUPD
    void *pbuf[2];        // EPI_PUPD / EPI_NORMAL (q = p_new)
};

qex_status launch_dslash_mrhs(qex_lattice *lat, const MrhsArgs &a, cudaStream_t st);

// x += alpha p_new (x NULL: left to the next iteration's first Dslash);
// r -= alpha ap; ||r||^2 -> S (rr, beta, flags); sets the graph conditions
// when ctl.active.
qex_status launch_update_xr(qex_lattice *lat, qex_prec prec, void *x, void *r, void *const pbuf[2],
                            const void *ap, CgScalars *S, const GraphCtl &ctl, cudaStream_t st);
// p_new = r + beta p_old with the buffers chosen by the iteration parity
// (halt-checked); the FP64 iteration's first kernel.
qex_status launch_update_p(qex_lattice *lat, qex_prec prec, const void *r, void *const pbuf[2], CgScalars *S,
                           cudaStream_t st);
// x64 += (double) xh32 + alpha p with p = pbuf[iters & 1] (the update the
// iteration left pending; pbuf NULL: none); xh32 = 0.
qex_status launch_accum_x(qex_lattice *lat, double *x64, float *xh32, float *const pbuf[2], CgScalars *S,
                          cudaStream_t st);
// r32 = (float) r64 (r32 may be NULL: only the graph condition is set),
// alpha = 0 (no pending iterate update after a reliable update); loop
// condition = !halt when ctl.active.
qex_status launch_finish_ru(qex_lattice *lat, const double *r64, float *r32, CgScalars *S, const GraphCtl &ctl,
                            cudaStream_t st);
// *flag |= (some element of the FP64 half field f is not zero; NaN counts).
qex_status launch_any_nonzero(qex_lattice *lat, const double *f, int *flag, cudaStream_t st);
// ||f||^2 -> *out (FP64, fixed order); if S, also S->bb and S->stop2.
qex_status launch_norm2(qex_lattice *lat, qex_prec prec, const void *f, double *out, CgScalars *S,
                        cudaStream_t st);
// <a, b> -> out[0..1].
qex_status launch_dot(qex_lattice *lat, qex_prec prec, const void *a, const void *b, double *out,
                      cudaStream_t st);

// The mixed-precision inner iteration of a small lattice as one persistent
// cooperative kernel (cg_fused.cu): runs iterations until a reliable update
// is due or an error, then writes the CG scalars back (halt set).
qex_status launch_cg_fused(qex_lattice *lat, qex_prec inner, const void *fat32, const void *lng32, double c3, double m2,
                           float *x, float *r, float *const p[2], float *ap, float *tmp, cudaStream_t st);
// Synchronises st and reports whether a grid barrier of the last fused run
// timed out, and how many of its blocks left the kernel (exited may be NULL).
qex_status fused_barrier_status(qex_lattice *lat, cudaStream_t st, int *timed_out, int *exited);

int blas_blocks(const qex_lattice *lat);
int sm_count();
void note_launches(unsigned long long n);
void set_count_launches(bool on);
void free_cg_graph(void *g);
void free_batch_ctx(void *c);

}  // namespace qex
