/*
 * qex_gpu.h -- C ABI of libqex_gpu.so: the even-odd staggered Dirac operator
 * (with optional Naik term), its normal operator and conjugate-gradient
 * solvers on one GB300 GPU (sm_103a).
 *
 * The paper (Jin & Osborn, "QEX: a framework for lattice field theories",
 * Sec. 4) names the workload -- the staggered Dirac operator with the Naik
 * term on SU(3) links, and single/double precision CG solvers for it
 * (benchmarked with one right-hand side, Fig. 1) -- without printing a
 * formula.  The operator implemented here is the standard one:
 *
 *   (D psi)(x) = sum_mu s_mu(x)   U_mu(x) psi(x+mu) - s_mu(x-mu)   U_mu(x-mu)^+ psi(x-mu)
 *         + c3 sum_mu s3_mu(x)  W_mu(x) psi(x+3mu) - s3_mu(x-3mu) W_mu(x-3mu)^+ psi(x-3mu)
 *
 *   s_mu(y)  = eta_mu(y) * (-1 if mu = t, time is antiperiodic and y_t = Lt-1)
 *   s3_mu(y) = eta_mu(y) * (-1 if mu = t, time is antiperiodic and y_t >= Lt-3)
 *   eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z)
 *
 * D flips site parity; D_eo (D_oe) is its block with even (odd) output.  The
 * solvers invert the normal operator A = m^2 - D_eo D_oe on even sites.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Extents dims = {Lx, Ly, Lz, Lt}: all even and >= 2; >= 4 when the Naik
 *   term is used.  V = Lx*Ly*Lz*Lt < 2^31, Vh = V/2.
 * - Site lex = x + Lx*(y + Ly*(z + Lz*t)); parity = (x+y+z+t) mod 2; the
 *   even-odd index of a site is parity*Vh + (lex >> 1).
 * - Canonical ("lex") layouts, interleaved complex double, device memory:
 *     links  [V][4][3][3]  (U_mu(x)_ab at ((lex*4 + mu)*3 + a)*3 + b)
 *     fields [V][3]
 * - Internal layouts (written by qex_pack_*; all other calls take these):
 *     links: per parity p, per direction mu, structure-of-arrays planes over
 *            the Vh sites of parity p.  F64: 9 planes of double2 (matrix
 *            element c = 3a+b); F32: 4 planes of float4 (elements 0-1, 2-3,
 *            4-5, 6-7) and 1 plane of float2 (element 8); F32_R12: 3 planes
 *            of float4 (elements 0-1, 2-3, 4-5: rows 0 and 1); F32_R12H: 1
 *            plane of 16-byte words (elements 0-3) and 1 plane of 8-byte
 *            words (elements 4-5), one 32-bit word per element: re in the
 *            low, im in the high 16 bits; F32_S16: 2 planes of 16-byte
 *            words (elements 0-3, 4-7) and 1 plane of 8-byte words (element
 *            8, then the FP32 step d).  Size qex_links_bytes().
 *     half field (the Vh sites of one parity): F64: 3 planes of double2
 *            (colour a); every FP32 precision: 1 plane of float4
 *            (colours 0,1) + 1 plane of float2 (colour 2).  Size
 *            qex_field_bytes().
 * - All field and link pointers are caller-owned DEVICE memory, 16-byte
 *   aligned; the library never frees them.  The library owns only the
 *   lattice object and its scratch (created lazily, freed by destroy).
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls are asynchronous on it unless stated otherwise.
 * - Every call checks its arguments before launching anything and returns a
 *   qex_status; nothing aborts or traps.  qex_last_error() gives the message
 *   of the calling thread's last failure.
 * - A lattice object is not thread-safe: one host thread per lattice at a
 *   time; its scratch is shared by all calls on it, so calls on one lattice
 *   must be ordered on one stream.
 */
#ifndef QEX_GPU_H
#define QEX_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QEX_OK = 0,
    QEX_ERR_ARG = 1,             /* null pointer, bad parity/direction/hop, bad tolerance */
    QEX_ERR_SHAPE = 2,           /* odd or too small extent, volume too large */
    QEX_ERR_ALIGN = 3,           /* pointer not 16-byte aligned */
    QEX_ERR_CUDA = 4,            /* a CUDA runtime call failed (message in qex_last_error) */
    QEX_ERR_NOT_CONVERGED = 5,   /* solver hit maxiter; the result so far is returned */
    QEX_ERR_TIMEOUT = 6,         /* a bounded device-side wait ran out */
    QEX_ERR_NAN = 7              /* NaN/Inf met in a reduction, or CG breakdown */
} qex_status;

/* Precisions.  QEX_F32_R12 means FP32 fields and FP32 fat links stored as
 * their first two rows only (12 reals); the third row is rebuilt in the
 * kernel as the complex conjugate of the cross product of the first two,
 * which is exact for SU(3) matrices only -- use it for unitary, unimodular
 * links.  QEX_F32_R12H is the same with each of the 12 reals stored as a
 * 16-bit fixed-point number (q = round(32767 v) in [-32767, 32767], stored
 * as the unsigned offset-binary q + 32768; value q / 32767; SU(3) entries
 * lie in [-1, 1]), quantisation error <= 1.5e-5 per real: an inner-solver format
 * (use it inside mixed-precision CG, whose FP64 reliable updates correct
 * it).  QEX_F32_S16 means FP32 fields and links of any kind (unitary or
 * not) as all 18 reals in 16-bit fixed point with a per-link FP32 step d =
 * (largest |re| or |im| of the link) / 32767 rounded up: q = round(v / d)
 * (computed as v * (1/d)), value q * d, error <= d / 2 per real.
 * Long (Naik) links have the format qex_long_links_prec(prec): QEX_F64 and
 * QEX_F32 keep their own; QEX_F32_R12 uses QEX_F32 (long links are not
 * unitary, so two-row storage does not apply); QEX_F32_R12H and QEX_F32_S16
 * use QEX_F32_S16. */
typedef enum { QEX_F64 = 0, QEX_F32 = 1, QEX_F32_R12 = 2, QEX_F32_R12H = 3, QEX_F32_S16 = 4 } qex_prec;

typedef struct qex_lattice qex_lattice; /* opaque, owned by the library */

typedef struct {
    int iters;               /* operator applications inside the CG iteration   */
    int reliable_updates;    /* FP64 true-residual recomputations (incl. final) */
    int converged;           /* 1 if the FP64 true residual met tol             */
    int ff_updates;          /* of these, made in float-float arithmetic          */
    double true_rel_resid;   /* ||b - A x|| / ||b||, recomputed in FP64         */
    double time_ms;          /* wall time of the solve on the stream            */
} qex_cg_stats;

/* ---------------------------------------------------------------- lattice */

/* Create a lattice of extents dims[4] = {Lx,Ly,Lz,Lt}; antiperiodic_t != 0
 * makes time antiperiodic for fermions.  Errors: QEX_ERR_ARG (null),
 * QEX_ERR_SHAPE (odd extent, extent < 2, V >= 2^31).
 * Paper: Sec. 4 (the lattice the staggered operator acts on; Fig. 1 runs the
 * solver on L^3 x T volumes).  Boundary condition and size limits are this
 * library's.
 */
qex_status qex_lattice_create(const int dims[4], int antiperiodic_t, qex_lattice **out);

/* Free the lattice and all scratch it owns (synchronises the device first).
 * NULL is accepted.
 * Paper: no counterpart (resource management of this library).
 */
qex_status qex_lattice_destroy(qex_lattice *lat);

/* Volume V and half volume Vh.
 * Paper: no counterpart.
 */
int64_t qex_volume(const qex_lattice *lat);
int64_t qex_half_volume(const qex_lattice *lat);

/* Even-odd index parity*Vh + (lex >> 1) of coord[4] = {x,y,z,t}
 * (host function; -1 on bad arguments).
 * Paper: no counterpart (the even-odd site order is this library's layout; the
 * paper describes QEX's data layout only in general terms, Sec. 3).
 */
int64_t qex_eo_index(const qex_lattice *lat, const int coord[4]);

/* Neighbour table: for the i-th site x of parity `parity` (i in [0,Vh)),
 * host_out[i] = index, within the opposite parity, of x + hop*mu_hat
 * (periodic wrap), hop in {+1,-1,+3,-3}.  Computed on the host with the same
 * index arithmetic the kernels use.  host_out holds Vh int32.
 * Paper: Sec. 4 names the operator whose hops these are (x +- mu, and x +- 3mu
 * for the Naik term); the table itself has no counterpart.
 */
qex_status qex_neighbor_table(const qex_lattice *lat, int parity, int mu, int hop, int32_t *host_out);

/* Same table written by a kernel into device memory dev_out (Vh int32).
 * Paper: as qex_neighbor_table.
 */
qex_status qex_neighbor_table_device(const qex_lattice *lat, int parity, int mu, int hop,
                                     int32_t *dev_out, void *stream);

/* ---------------------------------------------------------------- layout */

/* Bytes of one internal link set (4V links) and of one internal half field.
 * Paper: no counterpart (layout of this library).
 */
size_t qex_links_bytes(const qex_lattice *lat, qex_prec prec);
size_t qex_field_bytes(const qex_lattice *lat, qex_prec prec);

/* Format of the long (Naik) link set that an operator of precision prec
 * reads (see the precisions above); -1 for an unknown prec.
 * Paper: no counterpart (link formats of this library).
 */
int qex_long_links_prec(qex_prec prec);

/* Canonical lex links (complex double, [V][4][3][3]) -> internal links of
 * precision prec (F32 rounds to nearest).  lex_links and internal must not
 * overlap.
 * Paper: no counterpart (layout conversion).
 */
qex_status qex_pack_links(const qex_lattice *lat, qex_prec prec, const double *lex_links,
                          void *internal, void *stream);

/* Canonical lex links -> the internal F64 set (internal64) and a second set of
 * an FP32 precision (internal2, e.g. the inner links of a mixed solve: the
 * inner format for fat links, qex_long_links_prec(inner) for long links) in
 * one pass over lex_links; bit for bit what qex_pack_links to F64 followed by
 * qex_convert_links from F64 gives.  No buffer may overlap another.
 * Errors: QEX_ERR_ARG (NULL, second = QEX_F64 or unknown), QEX_ERR_ALIGN.
 * Paper: no counterpart (layout conversion).
 */
qex_status qex_pack_links_pair(const qex_lattice *lat, const double *lex_links, void *internal64,
                               qex_prec second, void *internal2, void *stream);

/* Internal links -> canonical lex links (complex double).
 * Paper: no counterpart (layout conversion).
 */
qex_status qex_unpack_links(const qex_lattice *lat, qex_prec prec, const void *internal,
                            double *lex_links, void *stream);

/* Sites of parity `parity` of a canonical full-lattice field ([V][3] complex
 * double) -> internal half field of precision prec.
 * Paper: no counterpart (layout conversion).
 */
qex_status qex_pack_field(const qex_lattice *lat, qex_prec prec, int parity, const double *lex_field,
                          void *half, void *stream);

/* Internal half field -> the parity-`parity` sites of a canonical field
 * (sites of the other parity are left untouched).
 * Paper: no counterpart (layout conversion).
 */
qex_status qex_unpack_field(const qex_lattice *lat, qex_prec prec, int parity, const void *half,
                            double *lex_field, void *stream);

/* Precision conversion of internal links or half fields (F64 -> F32 rounds
 * to nearest, F32 -> F64 is exact).  in and out must not overlap.
 * Paper: Sec. 4 runs the solver in single and double precision; the
 * conversions between this library's formats have no counterpart.
 */
qex_status qex_convert_links(const qex_lattice *lat, qex_prec from, const void *in, qex_prec to,
                             void *out, void *stream);
qex_status qex_convert_field(const qex_lattice *lat, qex_prec from, const void *in, qex_prec to,
                             void *out, void *stream);

/* ---------------------------------------------------------------- operator */

/* out = D_{p,1-p} in (p = out_parity): the staggered operator from the
 * parity-(1-p) half field `in` to the parity-p half field `out`.  fat: one
 * internal link set (U); lng: long links W for the Naik term, or NULL;
 * c_naik: the Naik coefficient c3 (ignored when lng is NULL).  in, out, fat,
 * lng share precision prec.  in and out must not overlap.
 * Paper: Sec. 4 (the Dirac operator of the staggered fermion action with the
 * Naik term); the paper prints no formula, the one implemented is written out
 * at the top of this header.
 */
qex_status qex_dslash(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                      double c_naik, int out_parity, const void *in, void *out, void *stream);

/* Largest number of right-hand sides of the multi-RHS calls. */
#define QEX_MRHS_MAX 64

/* Multi-RHS Dslash: out_r = D_{p,1-p} in_r for r = 0..nrhs-1, with each link
 * read from memory once for all right-hand sides (the paper benchmarks one
 * right-hand side, Fig. 1; batching them cuts the link traffic per vector by
 * nrhs).  `in` and `out` hold nrhs half fields back to back (field r starts
 * at r * qex_field_bytes(lat, prec)); they must not overlap.  1 <= nrhs <=
 * QEX_MRHS_MAX.  Other arguments and errors as qex_dslash.
 * Paper: Sec. 4 (the operator, as qex_dslash); several right-hand sides at once
 * are this library's extension of the one-vector benchmark of Fig. 1.
 */
qex_status qex_dslash_mrhs(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                           double c_naik, int out_parity, int nrhs, const void *in, void *out, void *stream);

/* out = (m^2 - D_eo D_oe) in on even sites; tmp_odd is a caller half field
 * (odd sites) that receives D_oe in.
 * Paper: Sec. 4 and Fig. 1 (the matrix the conjugate-gradient solver inverts);
 * the even-odd normal form m^2 - D_eo D_oe is this library's reading.
 */
qex_status qex_normal_op(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                         double c_naik, double mass, const void *in, void *out, void *tmp_odd,
                         void *stream);

/* Size of the static device scratch behind qex_normal_op_static (32 MiB). */
#define QEX_NORMAL_OP_STATIC_MAX_BYTES ((size_t)32 << 20)

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory.  qex_normal_op needs a caller-allocated
 * odd half field (tmp_odd) for D_oe in; callers running under an allocator
 * that forbids allocations outside its own pool, or on paths where the
 * device-wide synchronisation of cudaMalloc/cudaFree is not acceptable, may
 * have no way to provide one.  This variant computes the same
 * out = (m^2 - D_eo D_oe) in, but keeps D_oe in in a fixed array compiled
 * into the library (a file-scope __device__ array of
 * QEX_NORMAL_OP_STATIC_MAX_BYTES bytes), so it allocates nothing: no
 * cudaMalloc, cudaFree or allocating library routine.  The caller still
 * passes the links, `in` and `out` (device memory, as for qex_normal_op).
 * - Size limit: the intermediate half field, qex_field_bytes(lat, prec),
 *   must fit in QEX_NORMAL_OP_STATIC_MAX_BYTES (FP64: Vh <= 699,050 sites,
 *   e.g. 32^4; FP32: Vh <= 1,398,101 sites); larger lattices get
 *   QEX_ERR_SHAPE before anything is launched.
 * - Memory: every GPU that loads the library holds the array until the
 *   process exits.
 * - Set-up: the first call made with a given device current looks up the
 *   array's device address (cudaGetSymbolAddress) for that device, and so
 *   does the first call after the device's context changed (for example
 *   after cudaDeviceReset, which can move the array); make that first call
 *   before any stream capture.
 * - Launch shape: the call never runs the autotuner (which allocates); it
 *   uses the shapes the lattice already has, the compiled defaults on a
 *   lattice no other call has tuned.
 * - Sharing: every call on every lattice uses the same array, and it keeps
 *   the last call's contents (each call overwrites what it reads).  Calls
 *   whose kernels overlap on the GPU (different streams, or host threads
 *   without ordering) race on the array: order them on one stream. */
qex_status qex_normal_op_static(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                                double c_naik, double mass, const void *in, void *out, void *stream);

/* ||f||^2 of a half field, accumulated in FP64 in a fixed order
 * (bit-reproducible run to run); written to dev_out (one double, device).
 * Paper: Sec. 4 and Fig. 1 (the global sums of the conjugate-gradient solver).
 */
qex_status qex_norm2(const qex_lattice *lat, qex_prec prec, const void *f, double *dev_out,
                     void *stream);

/* <a, b> = sum conj(a) b over a half field, FP64 accumulation, fixed order;
 * dev_out receives {re, im} (two doubles, device).
 * Paper: Sec. 4 and Fig. 1 (the global sums of the conjugate-gradient solver).
 */
qex_status qex_dot(const qex_lattice *lat, qex_prec prec, const void *a, const void *b,
                   double *dev_out, void *stream);

/* ---------------------------------------------------------------- solvers */

/* Solve (m^2 - D_eo D_oe) x = b on even sites to a true relative residual
 * ||b - A x|| / ||b|| <= tol, computed in FP64.
 *
 * inner = QEX_F64: plain CG in FP64 on fat64/lng64.
 * inner = QEX_F32, QEX_F32_R12, QEX_F32_R12H or QEX_F32_S16: mixed precision: the CG
 *   iteration runs in FP32 on fat32/lng32 (fat32 in the `inner` link format,
 *   lng32 in qex_long_links_prec(inner); inner residual and iterate in FP32,
 *   all reductions in FP64);
 *   whenever the iterated residual norm drops below delta times its maximum
 *   since the last update (or meets tol), the FP64 solution is updated and the
 *   residual is recomputed in FP64 with fat64/lng64 (reliable update).
 *   A reliable update also follows any 100 inner iterations without one with
 *   16-bit links (QEX_F32_R12H, QEX_F32_S16) and any 500 with FP32 links: over
 *   longer cycles (small mass) the inner recursion residual drifts away from
 *   the true one and the solve stalls.  The environment variable
 *   QEX_RU_CYCLE = n sets another bound (0: none), read at each solve.
 *   The updates are FP64.  With the environment variable QEX_RU_FF = 1 (read
 *   at each solve) those asked for before the iterated residual meets tol
 *   (and before maxiter) run in float-float arithmetic (qex_true_residual,
 *   arith = 1) on the FP32 pipes instead, as long as their error stays below
 *   1e-3 of the residual; the first one and the one that may end the solve
 *   stay FP64, so convergence is always judged on an FP64 true residual.
 * b64, x64: F64 even half fields; x64 holds the initial guess on entry and the
 *   solution on return.  lng64/lng32 NULL = no Naik term.
 * Synchronises the stream before returning (fills stats, may be NULL).
 * Execution: one CUDA graph for the whole solve by default; for a mixed solve
 * with Vh <= 32768 the inner iterations run instead as one persistent
 * cooperative kernel between the reliable updates.  The environment variable
 * QEX_CG_MODE = graph | host | fused forces one of the three.
 * Returns QEX_ERR_NOT_CONVERGED after maxiter iterations (x64 holds the last
 * iterate), QEX_ERR_NAN on a NaN/Inf or a non-positive <p, A p>,
 * QEX_ERR_TIMEOUT if a grid barrier of the persistent kernel waited longer
 * than its limit (blocks not co-resident; the kernel returns instead of
 * waiting forever; the message says how many of its blocks left it).  The
 * limit is about a second (2e9 clock64 cycles); the environment variable
 * QEX_BARRIER_TIMEOUT_CYCLES sets another (read at each launch).
 * Paper: Sec. 4 (single and double precision conjugate-gradient solvers of the
 * staggered Dirac matrix) and Fig. 1 (one right-hand side); the mixed solve
 * with FP64 reliable updates is this library's combination of the two.
 */
qex_status qex_cg(const qex_lattice *lat, qex_prec inner, const void *fat64, const void *lng64,
                  const void *fat32, const void *lng32, double c_naik, double mass, const void *b64,
                  void *x64, double tol, int maxiter, double delta, void *stream,
                  qex_cg_stats *stats);

/* Device time of each kernel of the CG iteration, measured inside a solve
 * (profiling): the set-up of qex_cg (same arguments and link formats), then
 * `iters` iterations (3 <= iters <= 10000) of exactly the kernels qex_cg runs,
 * in its order and launch shapes and on the same buffers, with an event after
 * every kernel.  The stop test is disabled, so every kernel does its full
 * work; no reliable update runs.  ms_out (host, room for 4) receives each
 * kernel's average time in milliseconds over all but the first two
 * iterations, *n_out the number of kernels per iteration: 3 for a mixed solve
 * (direction update fused into D_oe, normal operator with <p, A p>, residual
 * update with ||r||^2), 4 for FP64 (direction update, D_oe, normal operator,
 * iterate and residual update).  b64 must be non-zero; x64 is the initial
 * guess and afterwards holds an intermediate iterate (FP64) or is unchanged
 * (mixed).  Synchronises the stream.  Errors as qex_cg, QEX_ERR_ARG for
 * iters out of range or a zero source.
 * Paper: no counterpart (measurement of the solver of Sec. 4 and Fig. 1). */
qex_status qex_cg_profile(const qex_lattice *lat, qex_prec inner, const void *fat64, const void *lng64,
                          const void *fat32, const void *lng32, double c_naik, double mass, const void *b64,
                          void *x64, int iters, void *stream, double *ms_out, int *n_out);

/* ||b - A x|| / ||b|| with A = m^2 - D_eo D_oe on the even sites, from F64
 * links (lng64 NULL = no Naik term) and F64 even half fields b64, x64, with
 * the kernels of a reliable update: arith = 0 in FP64, arith = 1 in the
 * float-float arithmetic of the intermediate updates (every real an
 * unevaluated sum of two FP32 numbers, about 47 significant bits; link
 * entries and b, x within 2^-100..2^100 of the root mean square of b's reals
 * are carried at full precision, smaller ones as zero).  rel_resid (host)
 * receives the result, 0 when b = 0.  Uses the lattice's work area and CG
 * scalars (not while a solve on the same lattice runs).  Synchronises the
 * stream.  Errors: as qex_dslash for the arguments, QEX_ERR_ARG (NULL
 * rel_resid, arith not 0 or 1), QEX_ERR_NAN (NaN/Inf in the result).
 * Paper: Sec. 4 (the solvers' stopping test, a relative true residual). */
qex_status qex_true_residual(const qex_lattice *lat, const void *fat64, const void *lng64, double c_naik,
                             double mass, const void *b64, const void *x64, int arith, double *rel_resid,
                             void *stream);

/* ---------------------------------------------------------------- force */

/* Fermion force of the pseudofermion action S = phi^+ A^{-1} phi,
 * A = m^2 - D_eo D_oe on even sites (the paper, Sec. 4, lists hybrid Monte
 * Carlo gauge generation, whose molecular dynamics needs this derivative).
 * Inputs: x_even = X = A^{-1} phi (F64 even half field, e.g. from qex_cg) and
 * y_odd = Y = D_oe X (F64 odd half field, e.g. from qex_dslash with
 * out_parity 1).  Since D is anti-Hermitian for any links,
 * dS = 2 Re sum_{x,mu} tr(dU_mu(x) G_mu(x)) with
 *   G_mu(x) =  s_mu(x) Y(x+mu) X(x)^+  (x even),
 *   G_mu(x) = -s_mu(x) X(x+mu) Y(x)^+  (x odd),
 * s_mu the staggered phase times the link's antiperiodic sign; for the long
 * links c_naik s3_mu and the x+3mu neighbours.  kind = 0 writes
 * F = 2 TA(U G) per link (traceless anti-Hermitian: dS/de along
 * U -> exp(i e w) U is sum i tr(w F)); kind = 1 writes 2 G^+, the gradient of
 * the real S with respect to the complex link entries (dS = Re sum
 * conj(2 G^+)_ab dU_ab).  out_fat (and out_lng when lng64 is given) receive
 * one internal F64 link set each (qex_unpack_links converts them).
 * Errors: QEX_ERR_ARG (NULL, bad kind), QEX_ERR_ALIGN, QEX_ERR_SHAPE (Naik on
 * an extent < 4). */
qex_status qex_force(const qex_lattice *lat, const void *fat64, const void *lng64, double c_naik,
                     const void *x_even, const void *y_odd, int kind, void *out_fat, void *out_lng, void *stream);

/* Multi-RHS CG: solves (m^2 - D_eo D_oe) x_r = b_r for r = 0..nrhs-1 with
 * every operator application shared (qex_dslash_mrhs), as qex_cg does for
 * one right-hand side.  b64, x64: nrhs F64 even half fields back to back;
 * x64 holds the initial guesses and receives the solutions.  The solves
 * iterate in lockstep; each stops (is frozen) when its own FP64 true residual
 * meets tol; a reliable update requested by any running one is done for all
 * running ones (the cycle bound of qex_cg counts lockstep iterations).  stats
 * (may be NULL) receives nrhs entries.  Synchronises the
 * stream.  Errors as qex_cg (QEX_ERR_NOT_CONVERGED if any right-hand side did
 * not converge).
 * Paper: extends the one-right-hand-side solver of Sec. 4 and Fig. 1.
 */
qex_status qex_cg_mrhs(const qex_lattice *lat, qex_prec inner, const void *fat64, const void *lng64,
                       const void *fat32, const void *lng32, double c_naik, double mass, int nrhs, const void *b64,
                       void *x64, double tol, int maxiter, double delta, void *stream, qex_cg_stats *stats);

/* Largest number of lattices in one qex_cg_batch call. */
#define QEX_BATCH_MAX 64

/* One problem of a batched solve: its own lattice object (not shared with
 * another item), links, mass, source and solution.  fat64/lng64: F64 link
 * sets; fat32/lng32: the inner-precision copies (fat32 in the `inner` link
 * format, lng32 in qex_long_links_prec(inner)) when inner != QEX_F64; lng64 NULL = no Naik
 * term (all items of a batch agree).  b64, x64: F64 even half fields, x64
 * holding the initial guess. */
typedef struct {
    const qex_lattice *lat;
    const void *fat64, *lng64;
    const void *fat32, *lng32;
    double c_naik;
    double mass;
    const void *b64;
    void *x64;
} qex_cg_item;

/* Batched CG over n independent lattices (different extents, links and
 * masses): every kernel of an iteration is one launch over a work list of
 * (lattice, tile) items of all running lattices, so small lattices share
 * the GPU (tile size and grid: qex_cg_batch_tune_info).  Each lattice has its own alpha, beta, residual norms,
 * reliable updates (with the cycle bound of qex_cg, counted in its own
 * iterations) and FP64 true-residual stop (tol, maxiter and delta are
 * common); the lattices iterate in lockstep and a converged one stops.  The
 * scratch of the batch (descriptors, scalars, per-tile partials) is owned by
 * items[0].lat; the CG vectors of each item live in its own lattice's work
 * area.  stats (may be NULL) receives n entries.  Synchronises the stream.
 * Errors as qex_cg; QEX_ERR_ARG also for 0 or more than QEX_BATCH_MAX items,
 * items sharing a lattice object, or items disagreeing on the Naik term.
 * Paper: extends the solver of Sec. 4 and Fig. 1 (run there one L^3 x T volume
 * at a time) to several lattices in one launch.
 */
qex_status qex_cg_batch(int n, const qex_cg_item *items, qex_prec inner, double tol, int maxiter, double delta,
                        void *stream, qex_cg_stats *stats);

/* Launch shape of the batched solver for batches led by lead (items[0].lat).
 * The iteration kernels run a persistent grid of out[0] resident blocks of
 * 256 threads per SM (1..3) over work items of out[1] groups of 256
 * consecutive sites of one lattice (1, 2 or 4).  Unless pinned
 * (qex_cg_batch_tune_set) or QEX_TUNE=0, the first qex_cg_batch call for a
 * (set of extents and boundaries in item order, inner precision, Naik) key
 * times the two Dslash kernels of an iteration for all nine (blocks per SM,
 * groups per item) pairs after the first FP64 residual and keeps the fastest
 * for the rest of the process.  Reductions are formed per 256-site group in a
 * fixed order, so every shape gives bit-identical results.  out[2]: where the
 * last batch's shape came from (0 none yet, 1 measured, 2 the process cache,
 * 3 defaults under QEX_TUNE=0, 4 pinned).  out is a host array of 3 ints.
 * Errors: QEX_ERR_ARG.
 * Paper: no counterpart (a GPU launch-configuration search). */
qex_status qex_cg_batch_tune_info(const qex_lattice *lead, int *out);

/* Pin the batch launch shape for batches led by lead: blocks_per_sm 1..3,
 * groups_per_item 1, 2 or 4; (0, 0) removes the pin.  Errors: QEX_ERR_ARG.
 * Paper: no counterpart. */
qex_status qex_cg_batch_tune_set(const qex_lattice *lead, int blocks_per_sm, int groups_per_item);

/* End-to-end solve from HOST memory (the call for users whose fields live
 * on the host).  host_fat (and host_lng, or NULL) are canonical complex-double
 * links [V][4][3][3]; host_b is a canonical complex-double field [V][3] whose
 * even sites are the source.  The call copies them to the device, packs them
 * (and rounds FP32 copies when inner is QEX_F32 or QEX_F32_R12), solves as qex_cg from
 * x0 = 0, and writes the solution to the even sites of host_x (canonical
 * [V][3]; its odd sites are set to zero).  Page-locked host buffers make the
 * copies asynchronous DMA.  Device staging (canonical and internal copies) is
 * owned by the lattice, allocated on first use and reused.  Synchronises the
 * stream.  Errors as qex_cg.
 * Paper: the solve of Sec. 4 and Fig. 1; the host-memory interface has no
 * counterpart.
 */
qex_status qex_cg_host(const qex_lattice *lat, qex_prec inner, const double *host_fat, const double *host_lng,
                       double c_naik, double mass, const double *host_b, double *host_x, double tol, int maxiter,
                       double delta, void *stream, qex_cg_stats *stats);

/* ---------------------------------------------------------- autotuner
 * Launch shapes (threads per block and grid) of the Dslash variants and of the
 * CG vector kernels.  The paper has no counterpart: this is a GPU launch-
 * configuration search.  For (lat, prec, Naik iff lng != NULL) qex_tune times,
 * with CUDA events on scratch fields it allocates and frees (about three half
 * fields), the plain Dslash at 256, 128 and 64 threads per block (one thread
 * per site, and a grid capped at two resident waves with the sites taken
 * grid-stride where that cap cuts the grid), the
 * normal-operator Dslash (which ends in a grid reduction) at a few block
 * sizes and grids, and the CG vector update with its grid capped at 2, 4, 8
 * or 16 blocks per SM; it keeps a shape only if it beats the compiled default
 * by more than 2 %, and stores the result in the lattice, in a per-process
 * cache keyed by (SM count, extents, boundary, prec, Naik) and, if the
 * environment variable QEX_TUNE_CACHE names a file, appends it there.
 * fat (and lng) are the link sets in prec's layout (read only).  The call
 * synchronises the stream.  Errors: QEX_ERR_ARG (null fat, or the stream is
 * being captured), QEX_ERR_ALIGN, QEX_ERR_SHAPE (Naik with an extent < 4),
 * QEX_ERR_CUDA.
 * qex_dslash, qex_normal_op and qex_cg tune the Dslash shapes (not the
 * vector-update grid, which only qex_tune measures) on their first uncaptured
 * call for a (prec, Naik) unless QEX_TUNE=0, taking the cache (file included)
 * when it holds the key.  Per-site results do not depend on the shape; FP64 sums
 * over blocks (CG reductions) are bit-reproducible for a given shape. */
qex_status qex_tune(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng, void *stream);

/* Launch shapes in use for (lat, prec, naik != 0): out[0] Dslash threads per
 * block, out[1] threads per block of the reducing Dslash variants, out[2] their
 * persistent grid in blocks per SM (0: one thread per site), out[3] the
 * vector kernels' grid cap in blocks per SM, out[4] where they came from (0
 * compiled defaults, not tuned yet; 1 measured; 2 cache; 3 defaults kept by
 * QEX_TUNE=0; 4 set by qex_tune_set), out[5] the non-reducing Dslash grid cap in resident waves (0:
 * one thread per site).  out is a host array of 6 ints.  Errors: QEX_ERR_ARG.
 * Paper: no counterpart.
 */
qex_status qex_tune_info(const qex_lattice *lat, qex_prec prec, int naik, int *out);

/* Pin the launch shapes of (lat, prec, naik != 0), the inverse of
 * qex_tune_info: in[0] Dslash threads per block, in[1] threads per block of
 * the reducing variants (both 64, 128 or 256), in[2] their persistent grid in
 * blocks per SM (0..16, 0: one thread per site), in[3] the vector kernels'
 * grid cap in blocks per SM (1..16; 0 leaves it), in[4] the non-reducing
 * Dslash grid cap in resident waves (0..8, 0: one thread per site).  The
 * shapes stay until the next qex_tune of the key (the automatic tuning of the
 * other calls does not replace them; qex_tune_info then reports source 4).
 * Use it to reproduce FP64 reduction bits across processes (they are fixed
 * for a given shape) or to run a chosen shape.  A cached CG graph of the
 * lattice is dropped (the device is synchronised first).  Errors:
 * QEX_ERR_ARG (NULL, a value out of range).
 * Paper: no counterpart. */
qex_status qex_tune_set(const qex_lattice *lat, qex_prec prec, int naik, const int *in);

/* Measured fused multiply-add rates of the current GPU, in GFLOP/s (2 flops
 * per FMA): *fp64_gflops (double) and *fp32_gflops (float, scalar FMA), from
 * fixed-trip FMA chains over several resident waves, timed with CUDA events
 * on `stream` (best of five bursts of a few ms; allocates and frees 512 KB of scratch;
 * synchronises the stream).  The FP64 rate bounds the FP64 Dslash on a GPU
 * whose FP64 units are few (GB300: about 1.2 TFLOP/s, 288 FP64 FMAs per site).
 * Errors: QEX_ERR_ARG (NULL), QEX_ERR_CUDA.
 * Paper: no counterpart (a measurement of the hardware). */
qex_status qex_fma_rates(double *fp64_gflops, double *fp32_gflops, void *stream);

/* Number of kernels this library has launched in the calling process so far
 * (monotone counter, for accounting of the kernels in a timed region).
 * Paper: no counterpart.
 */
uint64_t qex_launch_count(void);

/* Message of the calling thread's last failed call ("" if none).
 * Paper: no counterpart.
 */
const char *qex_last_error(void);

/* Library version string.
 * Paper: no counterpart.
 */
const char *qex_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QEX_GPU_H */
