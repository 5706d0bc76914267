// host_api.cu -- qex_cg_host: the whole path from host buffers (copy in,
// pack, convert, solve, unpack, copy out) in one call.
//
// The host link is the slow part (a few hundred GB/s against the HBM's
// several TB/s), so the links travel in slabs of t-slices on a copy stream,
// and each slab is packed -- into the FP64 set and the inner format at once,
// reading every canonical link once -- on the caller's stream as soon as it
// has landed, while the next slab is in flight.  Only the last slab's packing
// is left after the last copy.
#include <string.h>

#include "qex_kernels.cuh"

namespace qex {
qex_status launch_pack_links_range(qex_lattice *lat, const double *lex, void *out64, qex_prec second, void *out2,
                                   int i0, int i1, cudaStream_t s);
}

using namespace qex;

static size_t al256(size_t n) { return (n + 255) & ~size_t(255); }

// Copy one canonical link set (host) into d_lex slab by slab on the copy
// stream and pack each slab on s into out64 (FP64) and out2 (format second,
// or NULL).  `after` (recorded on s) orders the first copy after the caller's
// earlier work.
static qex_status copy_pack_links(qex_lattice *lat, const double *host, double *d_lex, void *out64, qex_prec second,
                                  void *out2, cudaEvent_t after, cudaStream_t s) {
    const int lt = lat->dims[3];
    const int nslab = lt < kHostSlabs ? lt : kHostSlabs;
    const size_t vs = (size_t)lat->dims[0] * lat->dims[1] * lat->dims[2];  // sites per t-slice (even)
    QEX_CUDA(cudaStreamWaitEvent(lat->copy_stream, after, 0));
    for (int k = 0; k < nslab; ++k) {
        const size_t t0 = (size_t)k * lt / nslab, t1 = (size_t)(k + 1) * lt / nslab;
        const size_t off = t0 * vs * 4 * 18;  // doubles
        QEX_CUDA(cudaMemcpyAsync(d_lex + off, host + off, (t1 - t0) * vs * 4 * 18 * sizeof(double),
                                 cudaMemcpyHostToDevice, lat->copy_stream));
        QEX_CUDA(cudaEventRecord(lat->slab_ev[k], lat->copy_stream));
        QEX_CUDA(cudaStreamWaitEvent(s, lat->slab_ev[k], 0));
        qex_status st = launch_pack_links_range(lat, d_lex, out64, second, out2, (int)(t0 * vs / 2),
                                                (int)(t1 * vs / 2), s);
        if (st) return st;
    }
    return QEX_OK;
}

extern "C" qex_status qex_cg_host(const qex_lattice *latc, qex_prec inner, const double *host_fat,
                                  const double *host_lng, double c_naik, double mass, const double *host_b,
                                  double *host_x, double tol, int maxiter, double delta, void *stream,
                                  qex_cg_stats *stats) {
    qex_status st;
    if ((st = check_lattice(latc)) || (st = check_prec(inner))) return st;
    if (!host_fat || !host_b || !host_x) {
        set_error("host_fat, host_b and host_x must not be NULL");
        return QEX_ERR_ARG;
    }
    qex_lattice *lat = const_cast<qex_lattice *>(latc);
    const bool naik = host_lng != nullptr;
    const bool mixed = inner != QEX_F64;
    const size_t lex_links = (size_t)lat->volume * 4 * 18 * sizeof(double);
    const size_t lex_field = (size_t)lat->volume * 6 * sizeof(double);
    const size_t l64 = qex_links_bytes(lat, QEX_F64), l32 = qex_links_bytes(lat, QEX_F32);  // >= R12 size
    const size_t f64 = qex_field_bytes(lat, QEX_F64);
    // staging: canonical links, canonical field, internal links (F64 [+F32]) x (fat [+long]), b, x
    const int nsets = naik ? 2 : 1;
    size_t need = al256(lex_links) + al256(lex_field) + nsets * (al256(l64) + (mixed ? al256(l32) : 0)) +
                  2 * al256(f64);
    if (lat->host_work_bytes < need) {
        if (lat->host_work) {
            QEX_CUDA(cudaDeviceSynchronize());
            QEX_CUDA(cudaFree(lat->host_work));
            lat->host_work = nullptr;
            lat->host_work_bytes = 0;
        }
        QEX_CUDA(cudaMalloc(&lat->host_work, need));
        lat->host_work_bytes = need;
    }
    char *w = (char *)lat->host_work;
    double *d_lex = (double *)w;
    w += al256(lex_links);
    double *d_field = (double *)w;
    w += al256(lex_field);
    void *fat64 = w;
    w += al256(l64);
    void *fat32 = nullptr, *lng64 = nullptr, *lng32 = nullptr;
    if (mixed) {
        fat32 = w;
        w += al256(l32);
    }
    if (naik) {
        lng64 = w;
        w += al256(l64);
        if (mixed) {
            lng32 = w;
            w += al256(l32);
        }
    }
    void *b64 = w;
    w += al256(f64);
    void *x64 = w;
    cudaStream_t s = as_stream(stream);

    if (!lat->copy_stream) {
        QEX_CUDA(cudaStreamCreateWithFlags(&lat->copy_stream, cudaStreamNonBlocking));
        for (int k = 0; k <= kHostSlabs; ++k)
            QEX_CUDA(cudaEventCreateWithFlags(&lat->slab_ev[k], cudaEventDisableTiming));
    }
    cudaEvent_t ready = lat->slab_ev[kHostSlabs];
    QEX_CUDA(cudaEventRecord(ready, s));
    if ((st = copy_pack_links(lat, host_fat, d_lex, fat64, inner, mixed ? fat32 : nullptr, ready, s))) return st;
    if (naik) {
        // d_lex is reused: the long links' copies wait for the fat links' packing
        QEX_CUDA(cudaEventRecord(ready, s));
        if ((st = copy_pack_links(lat, host_lng, d_lex, lng64, (qex_prec)qex_long_links_prec(inner),
                                  mixed ? lng32 : nullptr, ready, s)))
            return st;
    }
    QEX_CUDA(cudaMemcpyAsync(d_field, host_b, lex_field, cudaMemcpyHostToDevice, lat->copy_stream));
    QEX_CUDA(cudaEventRecord(ready, lat->copy_stream));
    QEX_CUDA(cudaStreamWaitEvent(s, ready, 0));
    if ((st = qex_pack_field(lat, QEX_F64, 0, d_field, b64, stream))) return st;
    QEX_CUDA(cudaMemsetAsync(x64, 0, f64, s));
    qex_status solve = qex_cg(lat, inner, fat64, lng64, fat32, lng32, c_naik, mass, b64, x64, tol, maxiter, delta,
                              stream, stats);
    if (solve != QEX_OK && solve != QEX_ERR_NOT_CONVERGED) return solve;
    QEX_CUDA(cudaMemsetAsync(d_field, 0, lex_field, s));
    if ((st = qex_unpack_field(lat, QEX_F64, 0, x64, d_field, stream))) return st;
    QEX_CUDA(cudaMemcpyAsync(host_x, d_field, lex_field, cudaMemcpyDeviceToHost, s));
    QEX_CUDA(cudaStreamSynchronize(s));
    if (solve != QEX_OK) set_error("CG did not converge in %d iterations", maxiter);
    return solve;
}
