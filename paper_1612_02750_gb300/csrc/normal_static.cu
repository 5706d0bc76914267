// normal_static.cu -- qex_normal_op_static: the even-site normal operator
// (m^2 - D_eo D_oe) for callers that cannot allocate device memory.
//
// qex_normal_op needs an odd-parity half field for the intermediate D_oe in,
// which the caller must allocate.  Some callers cannot: code running under a
// memory allocator that forbids allocations outside its own pool, or paths
// where the implicit device-wide synchronisation of cudaMalloc/cudaFree is
// not acceptable.  This variant keeps that intermediate in a fixed
// file-scope device array instead, so the call allocates nothing; the caller
// still passes links, input and output.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (kStaticScratchBytes) until the process exits.  Host code
// must not pass the array's name to a kernel (on the host it is only a
// stand-in symbol); the device address is looked up with cudaGetSymbolAddress
// on the first call made with a device current, and again whenever the
// device's current CUDA context is not the one the address was taken in (a
// cudaDeviceReset destroys the context, and the array may come back at
// another address in the next one).  The context is identified by the
// driver's context id, reached through the runtime's driver entry-point
// query, so the library does not link the driver directly; without that
// query every call looks the address up again.
#include <mutex>

#include "qex_kernels.cuh"

namespace qex {

constexpr size_t kStaticScratchBytes = QEX_NORMAL_OP_STATIC_MAX_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_normal_scratch[kStaticScratchBytes];

struct ScratchSlot {
    void *ptr;                // device address of g_normal_scratch in that context
    unsigned long long ctx;   // driver id of the context it was taken in (0: none)
};
static ScratchSlot g_scratch[kMaxDevices];
static std::mutex g_scratch_mu;

qex_status check_dslash_args(const qex_lattice *lat, qex_prec prec, const void *fat, const void *lng,
                             const void *in, const void *out);

// Id of the calling thread's current driver context, 0 if there is none or
// the driver does not offer the two queries.  The function pointers are
// looked up once per process.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

static unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();  // a failed query leaves no sticky error behind
    });
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx) return 0;
    if (get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_normal_scratch on the current device, in its current
// context (looked up when the device has none cached for this context).
static qex_status static_scratch(void **out) {
    int dev = 0;
    QEX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond the %d supported by the static scratch", dev, kMaxDevices);
        return QEX_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    const unsigned long long ctx = current_context_id();
    ScratchSlot &slot = g_scratch[dev];
    if (!slot.ptr || ctx == 0 || slot.ctx != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_normal_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_normal_scratch)");
        if (!p) {
            set_error("cudaGetSymbolAddress returned NULL for the static scratch");
            return QEX_ERR_CUDA;
        }
        slot.ptr = p;
        // the lookup made the device's primary context current if no
        // context was: take the id again
        slot.ctx = ctx ? ctx : current_context_id();
    }
    *out = slot.ptr;
    return QEX_OK;
}

}  // namespace qex

using namespace qex;

extern "C" qex_status qex_normal_op_static(const qex_lattice *lat, qex_prec prec, const void *fat,
                                           const void *lng, double c_naik, double mass, const void *in, void *out,
                                           void *stream) {
    qex_status st = check_dslash_args(lat, prec, fat, lng, in, out);
    if (st) return st;
    const size_t need = qex_field_bytes(lat, prec);
    if (need > kStaticScratchBytes) {
        set_error("qex_normal_op_static: the intermediate half field needs %zu bytes, more than the %zu-byte "
                  "static scratch (use qex_normal_op with a caller-allocated tmp_odd)",
                  need, kStaticScratchBytes);
        return QEX_ERR_SHAPE;
    }
    void *tmp = nullptr;
    if ((st = static_scratch(&tmp))) return st;
    qex_lattice *l = const_cast<qex_lattice *>(lat);
    cudaStream_t s = as_stream(stream);
    // D_oe in -> scratch (fully overwritten, so nothing left by an earlier call is read)
    DslashArgs a = {};
    a.prec = prec;
    a.fat = fat;
    a.lng = lng;
    a.c3 = c_naik;
    a.out_parity = 1;
    a.in = in;
    a.out = tmp;
    a.epi = EPI_PLAIN;
    if ((st = launch_dslash(l, a, s))) return st;
    // out = m^2 in - D_eo scratch (no CG state: S = NULL, no reduction scratch)
    a.out_parity = 0;
    a.in = tmp;
    a.out = out;
    a.epi = EPI_NORMAL;
    a.q = in;
    a.m2 = mass * mass;
    return launch_dslash(l, a, s);
}
