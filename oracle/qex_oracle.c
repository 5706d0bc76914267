/*
 * qex_oracle.c -- plain FP64 CPU oracle for the staggered Dirac operator with
 * the Naik term, its even-odd normal operator, conjugate gradient and the
 * fermion force.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library; the product (CUDA) path
 * never does, and the two share no code, header or table.
 *
 * What it computes.  The paper (Sec. 4, "Current status and plans") names the
 * operator -- the staggered Dirac operator on SU(N) gauge links including the
 * Naik term -- and benchmarks a conjugate-gradient solver on it (Sec. 4 and
 * the caption of Fig. 1, one right-hand side, single and double precision).
 * It prints no formula, so the standard Kawamoto-Smit form is written out
 * here, literally, with lexicographic site loops and no even-odd layout:
 *
 *   (D psi)(x) = sum_mu eta_mu(x) b_mu(x,+1) U_mu(x) psi(x+mu)
 *              - sum_mu eta_mu(x-mu) b_mu(x-mu,+1) U_mu(x-mu)^+ psi(x-mu)
 *              + c3 sum_mu eta_mu(x) b_mu(x,+3) W_mu(x) psi(x+3mu)
 *              - c3 sum_mu eta_mu(x-3mu) b_mu(x-3mu,+3) W_mu(x-3mu)^+ psi(x-3mu)
 *
 *   eta_0 = 1, eta_1 = (-1)^x0, eta_2 = (-1)^(x0+x1), eta_3 = (-1)^(x0+x1+x2)
 *   b_mu(y,k) = (-1)^(number of times y_t + k wraps past Lt), for mu = t and
 *               antiperiodic time; 1 otherwise (the sign belongs to the link
 *               that leaves y by k steps)
 *
 * D_eo / D_oe are the parity blocks of D (it flips parity).  The normal
 * operator on even sites is A = m^2 - D_eo D_oe; it is Hermitian positive
 * definite because D is anti-Hermitian for any links.
 *
 * Layouts (complex double, C order): site lex = x0 + L0*(x1 + L1*(x2 + L2*x3));
 * links U[(lex*4 + mu)*9 + 3a + b]; fields psi[lex*3 + a]; full lattice always
 * (sites of the parity a function does not use are zero).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ geometry */

int64_t oracle_volume(const int L[4]) {
    return (int64_t)L[0] * L[1] * L[2] * L[3];
}

int64_t oracle_lex(const int L[4], const int x[4]) {
    return x[0] + (int64_t)L[0] * (x[1] + (int64_t)L[1] * (x[2] + (int64_t)L[2] * x[3]));
}

void oracle_coords(const int L[4], int64_t lex, int x[4]) {
    for (int mu = 0; mu < 4; ++mu) {
        x[mu] = (int)(lex % L[mu]);
        lex /= L[mu];
    }
}

int oracle_parity(const int x[4]) {
    return (x[0] + x[1] + x[2] + x[3]) % 2;
}

/* Coordinates of x + k mu_hat with periodic wrap (k may be negative). */
static void shifted(const int L[4], const int x[4], int mu, int k, int y[4]) {
    for (int nu = 0; nu < 4; ++nu) y[nu] = x[nu];
    int c = (x[mu] + k) % L[mu];
    if (c < 0) c += L[mu];
    y[mu] = c;
}

/* Staggered phase eta_mu(x) = (-1)^(sum of x_nu over nu < mu). */
int oracle_eta(int mu, const int x[4]) {
    int s = 0;
    for (int nu = 0; nu < mu; ++nu) s += x[nu];
    return (s % 2) ? -1 : 1;
}

/* Boundary sign carried by the link leaving y along mu by k > 0 steps:
 * with antiperiodic time, -1 for every crossing of the t boundary. */
int oracle_link_bc(const int L[4], int antiperiodic, int mu, const int y[4], int k) {
    if (!antiperiodic || mu != 3) return 1;
    int wraps = (y[3] + k) / L[3];
    return (wraps % 2) ? -1 : 1;
}

/* eo[lex] = parity * V/2 + (rank of the site among the sites of its parity,
 * counted in lexicographic order).  Built by plain enumeration. */
void oracle_eo_table(const int L[4], int32_t *eo) {
    int64_t V = oracle_volume(L);
    int64_t count[2] = {0, 0};
    int x[4];
    for (int64_t s = 0; s < V; ++s) {
        oracle_coords(L, s, x);
        int p = oracle_parity(x);
        eo[s] = (int32_t)(p * (V / 2) + count[p]);
        count[p]++;
    }
}

/* For the k-th site x of parity `parity` (lexicographic order), out[k] is the
 * rank, within its own parity, of the site x + hop*mu_hat. */
void oracle_neighbor_table(const int L[4], int parity, int mu, int hop, int32_t *out) {
    int64_t V = oracle_volume(L);
    int32_t *eo = (int32_t *)malloc(sizeof(int32_t) * V);
    oracle_eo_table(L, eo);
    int64_t k = 0;
    int x[4], y[4];
    for (int64_t s = 0; s < V; ++s) {
        oracle_coords(L, s, x);
        if (oracle_parity(x) != parity) continue;
        shifted(L, x, mu, hop, y);
        int64_t r = eo[oracle_lex(L, y)];
        out[k++] = (int32_t)(r % (V / 2));
    }
    free(eo);
}

/* -------------------------------------------------------------- colour algebra */

static const cplx *link_at(const cplx *U, int64_t lex, int mu) {
    return U + (lex * 4 + mu) * 9;
}

/* acc += s * M v */
static void add_mv(cplx acc[3], double s, const cplx *M, const cplx *v) {
    for (int a = 0; a < 3; ++a) {
        cplx t = 0;
        for (int b = 0; b < 3; ++b) t += M[3 * a + b] * v[b];
        acc[a] += s * t;
    }
}

/* acc += s * M^+ v */
static void add_mdagv(cplx acc[3], double s, const cplx *M, const cplx *v) {
    for (int a = 0; a < 3; ++a) {
        cplx t = 0;
        for (int b = 0; b < 3; ++b) t += conj(M[3 * b + a]) * v[b];
        acc[a] += s * t;
    }
}

/* ------------------------------------------------------------------ operator */

/* acc = (D in)(x) at the site of lexicographic index s (formula in the
 * header).  W may be NULL (no Naik term). */
static void dslash_at(const int L[4], int antiperiodic, const cplx *U, const cplx *W, double c3,
                      const cplx *in, int64_t s, cplx acc[3]) {
    int x[4], y[4];
    oracle_coords(L, s, x);
    acc[0] = acc[1] = acc[2] = 0;
    for (int mu = 0; mu < 4; ++mu) {
        /* forward one-hop: eta_mu(x) b U_mu(x) psi(x+mu) */
        shifted(L, x, mu, +1, y);
        add_mv(acc, oracle_eta(mu, x) * oracle_link_bc(L, antiperiodic, mu, x, 1),
               link_at(U, s, mu), in + 3 * oracle_lex(L, y));
        /* backward one-hop: -eta_mu(y) b U_mu(y)^+ psi(y), y = x - mu */
        shifted(L, x, mu, -1, y);
        int64_t ly = oracle_lex(L, y);
        add_mdagv(acc, -oracle_eta(mu, y) * oracle_link_bc(L, antiperiodic, mu, y, 1),
                  link_at(U, ly, mu), in + 3 * ly);
        if (W) {
            shifted(L, x, mu, +3, y);
            add_mv(acc, c3 * oracle_eta(mu, x) * oracle_link_bc(L, antiperiodic, mu, x, 3),
                   link_at(W, s, mu), in + 3 * oracle_lex(L, y));
            shifted(L, x, mu, -3, y);
            ly = oracle_lex(L, y);
            add_mdagv(acc, -c3 * oracle_eta(mu, y) * oracle_link_bc(L, antiperiodic, mu, y, 3),
                      link_at(W, ly, mu), in + 3 * ly);
        }
    }
}

/* out = D in on the full lattice.  `in` and `out` must not alias. */
void oracle_dslash(const int L[4], int antiperiodic, const cplx *U, const cplx *W, double c3,
                   const cplx *in, cplx *out) {
    int64_t V = oracle_volume(L);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; ++s) {
        cplx acc[3];
        dslash_at(L, antiperiodic, U, W, c3, in, s, acc);
        for (int a = 0; a < 3; ++a) out[3 * s + a] = acc[a];
    }
}

/* out[3k..3k+2] = (D in)(x_k) for the n sites of lexicographic index
 * sites[k] (the same sum as oracle_dslash, evaluated only there). */
void oracle_dslash_sites(const int L[4], int antiperiodic, const cplx *U, const cplx *W, double c3,
                         const cplx *in, const int64_t *sites, int64_t n, cplx *out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        cplx acc[3];
        dslash_at(L, antiperiodic, U, W, c3, in, sites[k], acc);
        for (int a = 0; a < 3; ++a) out[3 * k + a] = acc[a];
    }
}

/* Zero the colour vectors of every site whose parity is not `keep`. */
static void keep_parity(const int L[4], cplx *f, int keep) {
    int64_t V = oracle_volume(L);
    int x[4];
    for (int64_t s = 0; s < V; ++s) {
        oracle_coords(L, s, x);
        if (oracle_parity(x) != keep)
            for (int a = 0; a < 3; ++a) f[3 * s + a] = 0;
    }
}

/* out = D_{p,1-p} in: the input restricted to parity 1-p, the output read at
 * parity p (zero elsewhere). */
void oracle_dslash_parity(const int L[4], int antiperiodic, const cplx *U, const cplx *W,
                          double c3, int out_parity, const cplx *in, cplx *out) {
    int64_t V = oracle_volume(L);
    cplx *t = (cplx *)malloc(sizeof(cplx) * 3 * V);
    memcpy(t, in, sizeof(cplx) * 3 * V);
    keep_parity(L, t, 1 - out_parity);
    oracle_dslash(L, antiperiodic, U, W, c3, t, out);
    keep_parity(L, out, out_parity);
    free(t);
}

/* out = (m^2 - D_eo D_oe) in on even sites (odd sites of out are zero). */
void oracle_normal_op(const int L[4], int antiperiodic, const cplx *U, const cplx *W, double c3,
                      double mass, const cplx *in, cplx *out) {
    int64_t V = oracle_volume(L);
    cplx *odd = (cplx *)malloc(sizeof(cplx) * 3 * V);
    cplx *even = (cplx *)malloc(sizeof(cplx) * 3 * V);
    oracle_dslash_parity(L, antiperiodic, U, W, c3, 1, in, odd);   /* D_oe in   */
    oracle_dslash_parity(L, antiperiodic, U, W, c3, 0, odd, even); /* D_eo D_oe */
    cplx *in_e = odd; /* reuse as the even part of the input */
    memcpy(in_e, in, sizeof(cplx) * 3 * V);
    keep_parity(L, in_e, 0);
    for (int64_t i = 0; i < 3 * V; ++i) out[i] = mass * mass * in_e[i] - even[i];
    free(odd);
    free(even);
}

/* ------------------------------------------------------------- vector algebra */

static double norm2(int64_t n, const cplx *a) {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return s;
}

static cplx dot(int64_t n, const cplx *a, const cplx *b) {
    cplx s = 0;
    for (int64_t i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

/* ||b - A x|| / ||b|| on even sites. */
double oracle_true_residual(const int L[4], int antiperiodic, const cplx *U, const cplx *W,
                            double c3, double mass, const cplx *b, const cplx *x) {
    int64_t n = 3 * oracle_volume(L);
    cplx *ax = (cplx *)malloc(sizeof(cplx) * n);
    oracle_normal_op(L, antiperiodic, U, W, c3, mass, x, ax);
    cplx *be = (cplx *)malloc(sizeof(cplx) * n);
    memcpy(be, b, sizeof(cplx) * n);
    keep_parity(L, be, 0);
    for (int64_t i = 0; i < n; ++i) ax[i] = be[i] - ax[i];
    double r = sqrt(norm2(n, ax) / norm2(n, be));
    free(ax);
    free(be);
    return r;
}

/* Conjugate gradient (Hestenes-Stiefel) on A x = b, even sites.  x holds the
 * initial guess on entry.  Stops when the recursively updated residual meets
 * ||r|| <= tol ||b||; the true residual b - A x is then recomputed, and if it
 * does not meet tol the iteration restarts from it.  Returns 0 when converged,
 * 1 when maxiter was reached.  `iters` counts applications of A inside the
 * iteration (true-residual recomputations are not counted). */
int oracle_cg(const int L[4], int antiperiodic, const cplx *U, const cplx *W, double c3,
              double mass, const cplx *b, cplx *x, double tol, int maxiter, int *iters,
              double *true_rel) {
    int64_t n = 3 * oracle_volume(L);
    cplx *r = (cplx *)malloc(sizeof(cplx) * n);
    cplx *p = (cplx *)malloc(sizeof(cplx) * n);
    cplx *ap = (cplx *)malloc(sizeof(cplx) * n);
    cplx *be = (cplx *)malloc(sizeof(cplx) * n);
    memcpy(be, b, sizeof(cplx) * n);
    keep_parity(L, be, 0);
    keep_parity(L, x, 0);
    double bb = norm2(n, be);
    int k = 0, converged = 0;
    if (bb == 0) {
        memset(x, 0, sizeof(cplx) * n);
        converged = 1;
    } else {
        oracle_normal_op(L, antiperiodic, U, W, c3, mass, x, ap);
        for (int64_t i = 0; i < n; ++i) r[i] = be[i] - ap[i];
        memcpy(p, r, sizeof(cplx) * n);
        double rr = norm2(n, r);
        while (rr > tol * tol * bb && k < maxiter) {
            oracle_normal_op(L, antiperiodic, U, W, c3, mass, p, ap);
            double alpha = rr / creal(dot(n, p, ap));
            for (int64_t i = 0; i < n; ++i) {
                x[i] += alpha * p[i];
                r[i] -= alpha * ap[i];
            }
            double rr_new = norm2(n, r);
            ++k;
            if (rr_new <= tol * tol * bb) {
                /* recompute the true residual before accepting convergence */
                oracle_normal_op(L, antiperiodic, U, W, c3, mass, x, ap);
                for (int64_t i = 0; i < n; ++i) r[i] = be[i] - ap[i];
                rr_new = norm2(n, r);
                if (rr_new > tol * tol * bb) {
                    memcpy(p, r, sizeof(cplx) * n); /* restart from the true residual */
                    rr = rr_new;
                    continue;
                }
                rr = rr_new;
                break;
            }
            double beta = rr_new / rr;
            rr = rr_new;
            for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        }
        converged = rr <= tol * tol * bb;
    }
    if (iters) *iters = k;
    if (true_rel) *true_rel = bb == 0 ? 0 : oracle_true_residual(L, antiperiodic, U, W, c3, mass, b, x);
    free(r);
    free(p);
    free(ap);
    free(be);
    return converged ? 0 : 1;
}

/* ------------------------------------------------------------------ force */

/* Fermion force of S = phi^+ A^{-1} phi (A = m^2 - D_eo D_oe on even sites).
 * With X = A^{-1} phi on even sites and Y = D_oe X on odd sites,
 * dS = -X^+ dA X = 2 Re X^+ dD_eo Y = 2 Re sum_{x,mu} tr(dU_mu(x) G_mu(x)):
 * D is anti-Hermitian for any links, so X^+ D_eo = -(D_oe X)^+ and
 * dD_oe = -dD_eo^+.  Collecting the terms of dD_eo link by link:
 *   G_mu(x) =  s_mu(x) Y(x+mu) X(x)^+    for even x,
 *   G_mu(x) = -s_mu(x) X(x+mu) Y(x)^+    for odd x,
 * with s_mu the staggered phase times the boundary sign of that link, and
 * the same with c3 and the 3-hop neighbours for the long links.  Outputs,
 * per link (links layout, full lattice):
 *   kind 0:  F = 2 TA(U G), TA(M) = (M - M^+)/2 - tr(M - M^+)/6 (traceless
 *            anti-Hermitian part): dS/de along U -> exp(i e w) U is
 *            sum i tr(w F) for Hermitian traceless w;
 *   kind 1:  2 G^+ = 2 dS/d(conj U): for any complex dU,
 *            dS = Re sum conj(2 G^+)_ab dU_ab (the gradient convention of
 *            torch for a real loss of complex inputs).
 * X and Y are full-lattice fields (X on even sites, Y on odd sites; the
 * other sites are ignored).  W and out_long may be NULL. */
static void force_links(const int L[4], int antiperiodic, const cplx *U, double coef, int hop, const cplx *X,
                        const cplx *Y, int kind, cplx *out) {
    int64_t V = oracle_volume(L);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < V; ++s) {
        int x[4], y[4];
        oracle_coords(L, s, x);
        int even = oracle_parity(x) == 0;
        for (int mu = 0; mu < 4; ++mu) {
            shifted(L, x, mu, hop, y);
            int64_t ly = oracle_lex(L, y);
            double sgn = coef * oracle_eta(mu, x) * oracle_link_bc(L, antiperiodic, mu, x, hop);
            const cplx *a = even ? Y + 3 * ly : X + 3 * ly;   /* field at x + hop mu */
            const cplx *b = even ? X + 3 * s : Y + 3 * s;     /* field at x */
            if (!even) sgn = -sgn;
            cplx G[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) G[3 * i + j] = sgn * a[i] * conj(b[j]);
            cplx *o = out + (s * 4 + mu) * 9;
            if (kind == 1) {
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) o[3 * i + j] = 2.0 * conj(G[3 * j + i]);
                continue;
            }
            const cplx *u = link_at(U, s, mu);
            cplx M[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    cplx t = 0;
                    for (int k = 0; k < 3; ++k) t += u[3 * i + k] * G[3 * k + j];
                    M[3 * i + j] = t;
                }
            cplx tr = 0;
            for (int i = 0; i < 3; ++i) tr += M[4 * i] - conj(M[4 * i]);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    cplx ta = 0.5 * (M[3 * i + j] - conj(M[3 * j + i]));
                    if (i == j) ta -= tr / 6.0;
                    o[3 * i + j] = 2.0 * ta;
                }
        }
    }
}

void oracle_force(const int L[4], int antiperiodic, const cplx *U, const cplx *W, double c3, const cplx *X,
                  const cplx *Y, int kind, cplx *out_fat, cplx *out_long) {
    force_links(L, antiperiodic, U, 1.0, 1, X, Y, kind, out_fat);
    if (W && out_long) force_links(L, antiperiodic, W, c3, 3, X, Y, kind, out_long);
}

/* Number of OpenMP threads the site loops use (1 without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}

/* Threads of the later site loops (timing only; the results do not depend on
 * it, each site's sum being formed by one thread). */
void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
