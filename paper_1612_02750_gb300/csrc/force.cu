// force.cu -- fermion force of S = phi^+ A^{-1} phi, A = m^2 - D_eo D_oe.
//
// With X = A^{-1} phi (even sites) and Y = D_oe X (odd sites),
// dS = 2 Re sum_{x,mu} tr(dU_mu(x) G_mu(x)) where
//   G_mu(x) =  s_mu(x) Y(x+mu) X(x)^+   on even x,
//   G_mu(x) = -s_mu(x) X(x+mu) Y(x)^+   on odd x,
// s_mu the staggered phase times the link's antiperiodic sign; the long
// links take c3 and the x+3mu neighbours.  The kernel forms G for every link
// and writes either F = 2 TA(U G) (traceless anti-Hermitian part, the force
// along U -> exp(i e w) U) or 2 G^+ (the gradient with respect to the complex
// link entries) in the internal FP64 link layout.  One thread per link:
// blockIdx.y = parity * 4 + mu.
#include "qex_kernels.cuh"

namespace qex {

__global__ void __launch_bounds__(kBlock)
force_kernel(Geom g, const double *__restrict__ links, double coef, int hop, const double *__restrict__ X,
             const double *__restrict__ Y, int kind, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const int blk = blockIdx.y, p = blk >> 2, mu = blk & 3;
    const size_t vh = (size_t)g.vh;
    const Site s = site_of(g, p, i);
    const int j = hop_index(g, s, mu, hop);
    double sgn = coef * ((eta_bit(s, mu) ^ bc_bit_fwd(g, s, mu, hop)) ? -1.0 : 1.0);
    // even x: a = Y(x+hop mu), b = X(x); odd x: a = X(x+hop mu), b = Y(x), sign flipped
    Vec3<double> a, b;
    if (p == 0) {
        a = load_vec(Y, vh, j);
        b = load_vec(X, vh, i);
    } else {
        a = load_vec(X, vh, j);
        b = load_vec(Y, vh, i);
        sgn = -sgn;
    }
    Mat3<double> G;  // sgn * a b^+
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            G.e[3 * r + c].re = sgn * (a.c[r].re * b.c[c].re + a.c[r].im * b.c[c].im);
            G.e[3 * r + c].im = sgn * (a.c[r].im * b.c[c].re - a.c[r].re * b.c[c].im);
        }
    double2 *o = reinterpret_cast<double2 *>(out) + (size_t)blk * 9 * vh + i;
    if (kind == 1) {  // 2 G^+
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                o[(3 * r + c) * vh] = make_double2(2.0 * G.e[3 * c + r].re, -2.0 * G.e[3 * c + r].im);
        return;
    }
    const Mat3<double> u = load_link(links, vh, p, mu, i);
    Mat3<double> M;  // U G
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                re = fma(u.e[3 * r + k].re, G.e[3 * k + c].re, re);
                re = fma(-u.e[3 * r + k].im, G.e[3 * k + c].im, re);
                im = fma(u.e[3 * r + k].re, G.e[3 * k + c].im, im);
                im = fma(u.e[3 * r + k].im, G.e[3 * k + c].re, im);
            }
            M.e[3 * r + c].re = re;
            M.e[3 * r + c].im = im;
        }
    // 2 TA(M) = (M - M^+) - tr(M - M^+)/3; tr(M - M^+) = 2i Im tr M
    const double imtr = (M.e[0].im + M.e[4].im + M.e[8].im) / 3.0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double re = M.e[3 * r + c].re - M.e[3 * c + r].re;
            double im = M.e[3 * r + c].im + M.e[3 * c + r].im;
            if (r == c) im -= 2.0 * imtr;
            o[(3 * r + c) * vh] = make_double2(re, im);
        }
}

}  // namespace qex

using namespace qex;

extern "C" qex_status qex_force(const qex_lattice *lat, const void *fat64, const void *lng64, double c_naik,
                                const void *x_even, const void *y_odd, int kind, void *out_fat, void *out_lng,
                                void *stream) {
    qex_status st;
    if ((st = check_lattice(lat))) return st;
    if (!fat64 || !x_even || !y_odd || !out_fat || (lng64 && !out_lng)) {
        set_error("fat64, x_even, y_odd and out_fat (and out_lng with long links) must not be NULL");
        return QEX_ERR_ARG;
    }
    if (!aligned16(fat64) || !aligned16(x_even) || !aligned16(y_odd) || !aligned16(out_fat) ||
        (lng64 && (!aligned16(lng64) || !aligned16(out_lng)))) {
        set_error("links and fields must be 16-byte aligned");
        return QEX_ERR_ALIGN;
    }
    if (kind != 0 && kind != 1) {
        set_error("kind must be 0 (force 2 TA(U G)) or 1 (gradient 2 G^+)");
        return QEX_ERR_ARG;
    }
    if (lng64)
        for (int mu = 0; mu < 4; ++mu)
            if (lat->dims[mu] < 4) {
                set_error("the Naik term needs every extent >= 4");
                return QEX_ERR_SHAPE;
            }
    dim3 grid(blocks_for(lat->vh), 8);
    cudaStream_t s = as_stream(stream);
    force_kernel<<<grid, kBlock, 0, s>>>(lat->geom, (const double *)fat64, 1.0, 1, (const double *)x_even,
                                         (const double *)y_odd, kind, (double *)out_fat);
    QEX_CHECK_LAUNCH("force_kernel");
    if (lng64) {
        force_kernel<<<grid, kBlock, 0, s>>>(lat->geom, (const double *)lng64, c_naik, 3, (const double *)x_even,
                                             (const double *)y_odd, kind, (double *)out_lng);
        QEX_CHECK_LAUNCH("force_kernel");
    }
    return QEX_OK;
}
