// vg_peaks.cu -- throughput probes for the roofline denominators the
// measured-peaks file does not carry: FP32 FMA, the base-2 exponential unit,
// shared-memory loads and global float atomics (no counterpart in the paper).
#include "vg_internal.h"

namespace vgk {

constexpr int PROBE_CHAINS = 8;  // independent dependency chains per thread

__global__ void __launch_bounds__(256) probe_fma_kernel(float* out, int iters, float b, float c) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fmaf(a[j], b, c);
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) t += a[j];
    if (t == 1.2345e30f) out[blockIdx.x] = t;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) probe_ex2_kernel(float* out, int iters) {
    float a[PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (float)(threadIdx.x & 7) * 0.1f + 0.01f * j;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fast_exp2(-a[j]);  // stays in (0.5, 1]
    float t = 0.f;
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) t += a[j];
    if (t == 1.2345e30f) out[blockIdx.x] = t;
}

__global__ void __launch_bounds__(256) probe_smem_kernel(float* out, int iters) {
    __shared__ float4 s[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) s[i] = make_float4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    int k = threadIdx.x;
    for (int i = 0; i < iters; ++i) {
        const float4 v = s[k];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
        k = (k + 32) & 1023;  // each warp reads 32 consecutive float4: no bank conflicts
    }
    if (acc.x + acc.y + acc.z + acc.w == 1.2345e30f) out[blockIdx.x] = acc.x;
}

__global__ void __launch_bounds__(256) probe_atomic_kernel(float* buf, int iters, int contended) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // distinct: every thread its own address; contended: one address per warp
    float* p = contended ? buf + (tid >> 5) * 32 : buf + tid;
    for (int i = 0; i < iters; ++i) atomicAdd(p, 1.f);
}

}  // namespace vgk

using namespace vgk;

extern "C" vg_status vg_probe_peak(int32_t kind, int32_t iters, float* buf, int64_t buf_floats, int64_t* units,
                                   vg_stream stream) {
    if (!buf || !units || iters < 1 || kind < 0 || kind > 4)
        return set_error(VG_ERR_INVALID_ARG, "vg_probe_peak: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    const int64_t nthr = (int64_t)blocks * threads;
    if (buf_floats < nthr) return set_error(VG_ERR_INVALID_ARG, "vg_probe_peak: buffer smaller than the grid");
    count_launches(1);
    switch (kind) {
        case 0:
            probe_fma_kernel<<<blocks, threads, 0, st>>>(buf, iters, 0.9999f, 1e-4f);
            *units = nthr * iters * PROBE_CHAINS * 2;  // FLOP
            break;
        case 1:
            probe_ex2_kernel<<<blocks, threads, 0, st>>>(buf, iters);
            *units = nthr * iters * PROBE_CHAINS;  // exponentials
            break;
        case 2:
            probe_smem_kernel<<<blocks, threads, 0, st>>>(buf, iters);
            *units = nthr * iters * 16;  // bytes
            break;
        default:
            probe_atomic_kernel<<<blocks, threads, 0, st>>>(buf, iters, kind == 4);
            *units = nthr * iters;  // atomic operations
            break;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VG_OK : set_error(VG_ERR_CUDA, cudaGetErrorString(e));
}
