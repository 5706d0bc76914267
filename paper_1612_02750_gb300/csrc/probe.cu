// probe.cu -- qex_fma_rates: the FP64 and FP32 fused multiply-add rates of
// the current GPU, the ceilings behind the FP64 Dslash (FP64-ALU bound on a
// GB300) and the issue-bound FP32 kernels.
//
// Every thread runs independent FMA chains (enough of them to cover the
// pipelines' latency) for a fixed trip count on a grid of several resident
// waves; the result is written so that nothing is optimised away.  The rate
// is 2 flops per FMA over the time between CUDA events on the stream, the
// best of five launches of about 5 ms each: a burst rate, like that of the
// sub-millisecond Dslash launches it bounds (a single 70 ms FP64 run read 12 %
// lower on a GB300).
#include "qex_kernels.cuh"

namespace qex {

constexpr int kChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) fma_probe_kernel(int trips, R a, R b, R *out) {
    R v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (R)(threadIdx.x + c);
    for (int t = 0; t < trips; ++t)
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    R s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == (R)-1.2345) out[blockIdx.x] = s;  // never true for these inputs; keeps the chains live
}

template <typename R>
static qex_status time_fma(int trips, cudaStream_t st, R *out, double *gflops) {
    int per_sm = 0;
    QEX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<R>, 256, 0));
    const int grid = sm_count() * (per_sm > 0 ? per_sm : 1) * 4;
    cudaEvent_t e0, e1;
    QEX_CUDA(cudaEventCreate(&e0));
    QEX_CUDA(cudaEventCreate(&e1));
    fma_probe_kernel<R><<<grid, 256, 0, st>>>(trips / 8, (R)0.999, (R)0.001, out);  // warm-up
    note_launch();
    cudaError_t e = cudaSuccess;
    float best = 0.f;
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        fma_probe_kernel<R><<<grid, 256, 0, st>>>(trips, (R)0.999, (R)0.001, out);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        if (e == cudaSuccess) {
            cudaEventElapsedTime(&ms, e0, e1);
            if (best == 0.f || ms < best) best = ms;
            note_launch();
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "fma_probe_kernel");
    *gflops = 2.0 * kChains * (double)trips * grid * 256 / (best * 1e-3) / 1e9;
    return QEX_OK;
}

}  // namespace qex

using namespace qex;

extern "C" qex_status qex_fma_rates(double *fp64_gflops, double *fp32_gflops, void *stream) {
    if (!fp64_gflops || !fp32_gflops) {
        set_error("fp64_gflops and fp32_gflops must not be NULL");
        return QEX_ERR_ARG;
    }
    cudaStream_t st = as_stream(stream);
    double *out = nullptr;
    QEX_CUDA(cudaMalloc(&out, sizeof(double) * 65536));
    qex_status s = time_fma<double>(320, st, out, fp64_gflops);
    if (!s) s = time_fma<float>(16384, st, reinterpret_cast<float *>(out), fp32_gflops);
    cudaFree(out);
    return s;
}
