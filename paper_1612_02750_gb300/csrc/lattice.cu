// lattice.cu -- lattice object, geometry, error plumbing, scratch and the
// neighbour-table entry points of libqex_gpu.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>

#include "qex_kernels.cuh"

namespace qex {

static thread_local char g_err[512] = "";
static std::atomic<unsigned long long> g_launches(0);

static thread_local bool g_count = true;  // off while a graph is being captured

void note_launch() {
    if (g_count) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void set_count_launches(bool on) { g_count = on; }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

qex_status cuda_fail(cudaError_t e, const char *what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return QEX_ERR_CUDA;
}

Geom make_geom(const int dims[4], int antiperiodic) {
    Geom g;
    for (int mu = 0; mu < 4; ++mu) g.L[mu] = dims[mu];
    g.stride[0] = 1;
    for (int mu = 1; mu < 4; ++mu) g.stride[mu] = g.stride[mu - 1] * dims[mu - 1];
    g.vh = (int)((int64_t)dims[0] * dims[1] * dims[2] * dims[3] / 2);
    g.antiperiodic = antiperiodic ? 1 : 0;
    g.div_xh = make_fastdiv((uint32_t)(dims[0] / 2));
    g.div_y = make_fastdiv((uint32_t)dims[1]);
    g.div_z = make_fastdiv((uint32_t)dims[2]);
    return g;
}

qex_status check_lattice(const qex_lattice *lat) {
    if (!lat) {
        set_error("lattice is NULL");
        return QEX_ERR_ARG;
    }
    return QEX_OK;
}

qex_status check_prec(qex_prec prec) {
    if (prec != QEX_F64 && prec != QEX_F32 && prec != QEX_F32_R12 && prec != QEX_F32_R12H && prec != QEX_F32_S16) {
        set_error("unknown precision %d", (int)prec);
        return QEX_ERR_ARG;
    }
    return QEX_OK;
}

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        sms = n;
    }
    return sms;
}

int blas_blocks(const qex_lattice *lat) {
    int want = blocks_for(lat->vh);
    const int per_sm = lat->blas_per_sm > 0 ? lat->blas_per_sm : QEX_BLAS_BLOCKS_PER_SM;
    if (per_sm <= 0) return want;
    int cap = sm_count() * per_sm;
    return want < cap ? want : cap;
}

// Scratch shared by every reducing kernel: per-block partials (two doubles
// per block of the largest grid), the last-block counter, a small result area
// and the CG scalars with their pinned host mirror.
qex_status ensure_scratch(qex_lattice *lat) {
    if (lat->partials) return QEX_OK;
    // the largest grids any launch shape of the autotuner can give
    int nb = blocks_for(lat->vh, 64);
    int nbb = sm_count() * 16;
    lat->partials_len = 2 * (nb > nbb ? nb : nbb);
    const int mrhs = (sm_count() * 8 + 1) * kMaxRhs;  // per-block, per-right-hand-side partials
    if (lat->partials_len < mrhs) lat->partials_len = mrhs;
    QEX_CUDA(cudaMalloc(&lat->partials, sizeof(double) * lat->partials_len));
    QEX_CUDA(cudaMalloc(&lat->counter, sizeof(unsigned int) * 8));
    QEX_CUDA(cudaMemset(lat->counter, 0, sizeof(unsigned int) * 8));
    QEX_CUDA(cudaMalloc(&lat->red_out, sizeof(double) * 8));
    QEX_CUDA(cudaMalloc(&lat->scalars, sizeof(CgScalars)));
    QEX_CUDA(cudaMallocHost(&lat->scalars_host, sizeof(CgScalars)));
    QEX_CUDA(cudaEventCreate(&lat->ev0));
    QEX_CUDA(cudaEventCreate(&lat->ev1));
    return QEX_OK;
}

qex_status ensure_work(qex_lattice *lat, size_t bytes) {
    if (lat->work_bytes >= bytes) return QEX_OK;
    if (lat->cg_graph) {  // its kernels point into the old buffer
        free_cg_graph(lat->cg_graph);
        lat->cg_graph = nullptr;
    }
    if (lat->work) {
        QEX_CUDA(cudaDeviceSynchronize());
        QEX_CUDA(cudaFree(lat->work));
        lat->work = nullptr;
        lat->work_bytes = 0;
    }
    QEX_CUDA(cudaMalloc(&lat->work, bytes));
    lat->work_bytes = bytes;
    return QEX_OK;
}

__global__ void neighbor_kernel(Geom g, int p, int mu, int hop, int32_t *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    Site s = site_of(g, p, i);
    out[i] = hop_index(g, s, mu, hop);
}

static qex_status check_hop(const qex_lattice *lat, int parity, int mu, int hop) {
    if (parity != 0 && parity != 1) {
        set_error("parity must be 0 or 1 (got %d)", parity);
        return QEX_ERR_ARG;
    }
    if (mu < 0 || mu > 3) {
        set_error("direction must be 0..3 (got %d)", mu);
        return QEX_ERR_ARG;
    }
    if (hop != 1 && hop != -1 && hop != 3 && hop != -3) {
        set_error("hop must be +-1 or +-3 (got %d)", hop);
        return QEX_ERR_ARG;
    }
    if ((hop == 3 || hop == -3) && lat->dims[mu] < 4) {
        set_error("a 3-hop needs extent >= 4 along direction %d", mu);
        return QEX_ERR_SHAPE;
    }
    return QEX_OK;
}

}  // namespace qex

using namespace qex;

extern "C" {

const char *qex_last_error(void) { return g_err; }

const char *qex_version(void) { return "qex_gpu 0.1 (sm_103a)"; }

uint64_t qex_launch_count(void) { return (uint64_t)g_launches.load(std::memory_order_relaxed); }

qex_status qex_lattice_create(const int dims[4], int antiperiodic_t, qex_lattice **out) {
    if (!dims || !out) {
        set_error("dims and out must not be NULL");
        return QEX_ERR_ARG;
    }
    *out = nullptr;
    int64_t v = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2 || dims[mu] % 2) {
            set_error("extent %d along direction %d must be even and >= 2", dims[mu], mu);
            return QEX_ERR_SHAPE;
        }
        v *= dims[mu];
    }
    if (v >= (int64_t(1) << 31)) {
        set_error("volume %lld too large (must be < 2^31)", (long long)v);
        return QEX_ERR_SHAPE;
    }
    qex_lattice *lat = new qex_lattice;
    memset(lat, 0, sizeof(*lat));
    for (int mu = 0; mu < 4; ++mu) lat->dims[mu] = dims[mu];
    lat->antiperiodic = antiperiodic_t ? 1 : 0;
    lat->volume = v;
    lat->vh = v / 2;
    lat->geom = make_geom(dims, lat->antiperiodic);
    cudaGetDevice(&lat->device);
    *out = lat;
    return QEX_OK;
}

qex_status qex_lattice_destroy(qex_lattice *lat) {
    if (!lat) return QEX_OK;
    qex_status st = QEX_OK;
    if (lat->partials || lat->work || lat->host_work || lat->batch_ctx) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "cudaDeviceSynchronize in destroy");
    }
    if (lat->partials) cudaFree(lat->partials);
    if (lat->counter) cudaFree(lat->counter);
    if (lat->red_out) cudaFree(lat->red_out);
    if (lat->scalars) cudaFree(lat->scalars);
    if (lat->scalars_host) cudaFreeHost(lat->scalars_host);
    if (lat->scalars_host2) cudaFreeHost(lat->scalars_host2);
    if (lat->work) cudaFree(lat->work);
    if (lat->host_work) cudaFree(lat->host_work);
    if (lat->cg_graph) free_cg_graph(lat->cg_graph);
    if (lat->batch_ctx) free_batch_ctx(lat->batch_ctx);
    if (lat->copy_stream) cudaStreamDestroy(lat->copy_stream);
    for (cudaEvent_t e : lat->slab_ev)
        if (e) cudaEventDestroy(e);
    if (lat->ev0) cudaEventDestroy(lat->ev0);
    if (lat->ev1) cudaEventDestroy(lat->ev1);
    delete lat;
    return st;
}

int64_t qex_volume(const qex_lattice *lat) { return lat ? lat->volume : -1; }

int64_t qex_half_volume(const qex_lattice *lat) { return lat ? lat->vh : -1; }

int64_t qex_eo_index(const qex_lattice *lat, const int coord[4]) {
    if (!lat || !coord) return -1;
    int64_t lex = 0, par = 0;
    for (int mu = 3; mu >= 0; --mu) {
        if (coord[mu] < 0 || coord[mu] >= lat->dims[mu]) return -1;
        lex = lex * lat->dims[mu] + coord[mu];
        par += coord[mu];
    }
    return (par & 1) * lat->vh + (lex >> 1);
}

qex_status qex_neighbor_table(const qex_lattice *lat, int parity, int mu, int hop, int32_t *host_out) {
    qex_status st = check_lattice(lat);
    if (st) return st;
    if (!host_out) {
        set_error("host_out is NULL");
        return QEX_ERR_ARG;
    }
    if ((st = check_hop(lat, parity, mu, hop))) return st;
    for (int i = 0; i < lat->geom.vh; ++i) {
        Site s = site_of(lat->geom, parity, i);
        host_out[i] = hop_index(lat->geom, s, mu, hop);
    }
    return QEX_OK;
}

qex_status qex_neighbor_table_device(const qex_lattice *lat, int parity, int mu, int hop,
                                     int32_t *dev_out, void *stream) {
    qex_status st = check_lattice(lat);
    if (st) return st;
    if (!dev_out) {
        set_error("dev_out is NULL");
        return QEX_ERR_ARG;
    }
    if ((st = check_hop(lat, parity, mu, hop))) return st;
    neighbor_kernel<<<blocks_for(lat->vh), kBlock, 0, as_stream(stream)>>>(lat->geom, parity, mu, hop, dev_out);
    QEX_CHECK_LAUNCH("neighbor_kernel");
    return QEX_OK;
}

size_t qex_links_bytes(const qex_lattice *lat, qex_prec prec) {
    if (!lat) return 0;
    if (prec == QEX_F32_R12) return (size_t)lat->volume * 4 * 12 * 4;
    if (prec == QEX_F32_R12H) return (size_t)lat->volume * 4 * 12 * 2;
    if (prec == QEX_F32_S16) return (size_t)lat->volume * 4 * 40;
    return (size_t)lat->volume * 4 * 18 * (prec == QEX_F64 ? 8 : 4);
}

int qex_long_links_prec(qex_prec prec) {
    switch (prec) {
        case QEX_F64: return QEX_F64;
        case QEX_F32:
        case QEX_F32_R12: return QEX_F32;
        case QEX_F32_R12H:
        case QEX_F32_S16: return QEX_F32_S16;
        default: return -1;
    }
}

size_t qex_field_bytes(const qex_lattice *lat, qex_prec prec) {
    if (!lat) return 0;
    return (size_t)lat->vh * 6 * (prec == QEX_F64 ? 8 : 4);
}

}  // extern "C"
