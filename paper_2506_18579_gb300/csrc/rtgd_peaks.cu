// rtgd_peaks.cu -- ceilings of this GPU measured with kernels written here:
// FP32 and FP64 fused multiply-add issue rates and L2 read bandwidth.  The
// tracer is bound by FP32 issue (mixed path), FP64 issue (all-FP64 path) and,
// second, by sample gathers served from L1/L2, so its roofline fractions are
// taken against these three numbers.  The paper has no counterpart.
#include <cuda_runtime.h>

#include <cstring>

#include "rtgd.h"
#include "rtgd_internal.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (hides the FMA latency)

// Every thread runs kChains independent chains of `iters` FMAs; the chains
// depend on runtime values, so nothing folds.  One value per thread is
// written only if it equals an impossible sentinel (keeps the work live).
template <typename T>
__global__ void fma_kernel(T x, T y, int iters, T *sink) {
    T a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = a[i] * x + y;
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += a[i];
    if (s == (T)-1.2345e30) sink[0] = s;
}

// Grid-stride float4 reads of a buffer that fits in L2, `passes` times.
__global__ void l2_read_kernel(const float4 *__restrict__ buf, long long n4, int passes, float *sink) {
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += stride) {
            const float4 v = __ldcg(buf + i);  // cache in L2 only, bypass L1
            acc += v.x + v.y + v.z + v.w;
        }
    }
    if (acc == -1.2345e30f) sink[0] = acc;
}

template <typename T>
cudaError_t time_fma(int sms, int iters, double *flops_per_s, T *sink, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
    const int threads = 256, blocks = sms * 8;
    fma_kernel<T><<<blocks, threads, 0, st>>>((T)0.999999, (T)1e-7, iters / 8, sink);  // warm-up
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        fma_kernel<T><<<blocks, threads, 0, st>>>((T)0.999999, (T)1e-7, iters, sink);
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    *flops_per_s = 2.0 * kChains * (double)iters * blocks * threads / (best * 1e-3);
    return cudaGetLastError();
}

}  // namespace

extern "C" rt_err rt_measure_peaks(rt_peaks *out) {
    if (!out) return rtgd_set_error(RT_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return rtgd_set_error(RT_EUNSUPPORTED, "no CUDA device available");
    int dev = 0, sms = 0, clk_khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    out->sm_count = sms;
    out->max_sm_mhz = clk_khz / 1000.0;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    void *sink = nullptr, *buf = nullptr;
    const size_t l2_bytes = (size_t)48 << 20;  // 48 MiB: well inside L2, far beyond L1
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, 64);
    if (e == cudaSuccess) e = cudaMalloc(&buf, l2_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, l2_bytes, st);
    if (e == cudaSuccess) e = time_fma<float>(sms, 1 << 11, &out->fp32_fma_flops, (float *)sink, st, e0, e1);
    if (e == cudaSuccess) e = time_fma<double>(sms, 1 << 6, &out->fp64_fma_flops, (double *)sink, st, e0, e1);
    if (e == cudaSuccess) {
        const long long n4 = (long long)(l2_bytes / sizeof(float4));
        const int threads = 512, blocks = sms * 4, passes = 20;
        l2_read_kernel<<<blocks, threads, 0, st>>>((const float4 *)buf, n4, 2, (float *)sink);  // warm L2
        float best = 1e30f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            cudaEventRecord(e0, st);
            l2_read_kernel<<<blocks, threads, 0, st>>>((const float4 *)buf, n4, passes, (float *)sink);
            cudaEventRecord(e1, st);
            e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            if (ms > 0.0f && ms < best) best = ms;
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        out->l2_read_bytes_per_s = (double)l2_bytes * passes / (best * 1e-3);
    }
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return rtgd_set_error(RT_ECUDA, cudaGetErrorString(e));
    return RT_OK;
}
