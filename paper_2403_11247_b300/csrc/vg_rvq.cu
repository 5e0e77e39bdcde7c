// vg_rvq.cu -- residual vector quantisation encode (Eq. 14, second line) and
// the codebook loss with its gradient (Eq. 15).
//
// One thread per item.  The codebooks (all stages) sit in shared memory; at
// stage s every thread scans the K codewords in order, so the warp reads the
// same codeword at the same time (a broadcast).  The argmin decisions follow
// a fixed FP32 order: l_hat summed in stage order, residual x - l_hat, and a
// codeword's distance is the sum over components, in order, of the rounded
// squares of the rounded differences (no fused multiply-add); the first
// minimum wins.  The loss and the codebook gradient accumulate per block
// (shared memory) and are added to the outputs once per block.
#include "vg_internal.h"

namespace vgk {

constexpr int RVQ_MAX_DIM = 16;

// the codeword scan of one stage: DP = the codeword stride in shared memory
// (4 for dim <= 4: one 16-byte load per codeword), first minimum wins
template <int DP>
__device__ __forceinline__ int rvq_argmin(const float* __restrict__ cs, int K, int dim, const float* r) {
    float best = INFINITY;
    int bk = 0;
    if (DP == 4) {
        const float4* c4 = reinterpret_cast<const float4*>(cs);
        const float r0 = r[0], r1 = dim > 1 ? r[1] : 0.f, r2 = dim > 2 ? r[2] : 0.f, r3 = dim > 3 ? r[3] : 0.f;
        for (int k = 0; k < K; ++k) {
            const float4 w = c4[k];
            // components beyond dim are padded with zeros on both sides: their terms are +0
            float d = __fmul_rn(__fsub_rn(w.x, r0), __fsub_rn(w.x, r0));
            d = __fadd_rn(d, __fmul_rn(__fsub_rn(w.y, r1), __fsub_rn(w.y, r1)));
            d = __fadd_rn(d, __fmul_rn(__fsub_rn(w.z, r2), __fsub_rn(w.z, r2)));
            d = __fadd_rn(d, __fmul_rn(__fsub_rn(w.w, r3), __fsub_rn(w.w, r3)));
            if (d < best) {
                best = d;
                bk = k;
            }
        }
    } else {
        for (int k = 0; k < K; ++k) {
            float d = 0.f;
            for (int c = 0; c < dim; ++c) {
                const float e = __fsub_rn(cs[k * DP + c], r[c]);
                d = __fadd_rn(d, __fmul_rn(e, e));
            }
            if (d < best) {
                best = d;
                bk = k;
            }
        }
    }
    return bk;
}

template <int DP>
__global__ void __launch_bounds__(256) rvq_encode_kernel(int dim, int L, int K, const float* __restrict__ cb,
                                                         const float* __restrict__ x, int64_t n,
                                                         uint8_t* __restrict__ idx, float* __restrict__ loss,
                                                         float* __restrict__ dcb, float scale) {
    extern __shared__ float4 s_mem4[];
    float* s_cb = reinterpret_cast<float*>(s_mem4);  // [L][K][DP], padded with zeros
    float* s_g = s_cb + (size_t)L * K * DP;          // [L][K][dim] gradient sums (when dcb)
    __shared__ float s_tmp[8];
    const int total = L * K * dim;
    for (int i = threadIdx.x; i < L * K * DP; i += blockDim.x) {
        const int c = i % DP, lk = i / DP;
        s_cb[i] = c < dim ? cb[(size_t)lk * dim + c] : 0.f;
    }
    if (dcb)
        for (int i = threadIdx.x; i < total; i += blockDim.x) s_g[i] = 0.f;
    __syncthreads();
    float acc = 0.f;
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item < n) {
        float xv[RVQ_MAX_DIM], lhat[RVQ_MAX_DIM], r[RVQ_MAX_DIM];
        for (int c = 0; c < dim; ++c) {
            xv[c] = x[item * dim + c];
            lhat[c] = 0.f;
        }
        for (int s = 0; s < L; ++s) {
            for (int c = 0; c < dim; ++c) r[c] = __fsub_rn(xv[c], lhat[c]);
            const float* cs = s_cb + (size_t)s * K * DP;
            const int bk = rvq_argmin<DP>(cs, K, dim, r);
            idx[(int64_t)s * n + item] = (uint8_t)bk;
            for (int c = 0; c < dim; ++c) {
                const float w = cs[bk * DP + c];
                const float e = w - r[c];  // the stop-gradient residual against the chosen codeword
                acc += e * e;
                if (dcb) atomicAdd(s_g + ((size_t)s * K + bk) * dim + c, 2.f * e);
                lhat[c] = __fadd_rn(lhat[c], w);
            }
        }
    }
    if (loss) {
        float v = acc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_tmp[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_tmp[w];
            if (t != 0.f) atomicAdd(loss, t * scale);
        }
    }
    if (dcb) {
        __syncthreads();
        for (int i = threadIdx.x; i < total; i += blockDim.x)
            if (s_g[i] != 0.f) atomicAdd(dcb + i, s_g[i] * scale);
    }
}

}  // namespace vgk

using namespace vgk;

extern "C" vg_status vg_rvq_encode(const vg_attr_group* g, int64_t n_items, const float* x, uint8_t* idx, float* loss,
                                   float* dcodebook, vg_stream stream) {
    if (!g || n_items < 0) return set_error(VG_ERR_INVALID_ARG, "vg_rvq_encode: null group or n < 0");
    if (g->stages < 1 || g->codewords < 1 || g->codewords > 256 || g->dim < 1 || g->dim > RVQ_MAX_DIM || !g->codebook)
        return set_error(VG_ERR_INVALID_ARG, "vg_rvq_encode: need 1 <= codewords <= 256, 1 <= dim <= 16 and a codebook");
    if (n_items > 0 && (!x || !idx)) return set_error(VG_ERR_INVALID_ARG, "vg_rvq_encode: null items or indices");
    const int L = g->stages, K = g->codewords, d = g->dim;
    const int DP = d <= 4 ? 4 : RVQ_MAX_DIM;  // codeword stride in shared memory
    const size_t cb_bytes = (size_t)L * K * d * sizeof(float);
    const size_t smem = (size_t)L * K * DP * sizeof(float) + (dcodebook ? cb_bytes : 0);
    if (smem > 200 * 1024) return set_error(VG_ERR_INVALID_ARG, "vg_rvq_encode: codebooks too large for shared memory");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (loss) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e == cudaSuccess && dcodebook) e = cudaMemsetAsync(dcodebook, 0, cb_bytes, st);
    if (e != cudaSuccess) return set_error(VG_ERR_CUDA, cudaGetErrorString(e));
    if (n_items == 0) return VG_OK;
    const float scale = 1.f / ((float)n_items * (float)K);
    const unsigned blocks = (unsigned)ceil_div(n_items, 256);
    count_launches(1);
    if (DP == 4) {
        e = allow_dynamic_smem((const void*)rvq_encode_kernel<4>, smem);
        if (e != cudaSuccess) return set_error(VG_ERR_CUDA, cudaGetErrorString(e));
        rvq_encode_kernel<4><<<blocks, 256, smem, st>>>(d, L, K, g->codebook, x, n_items, idx, loss, dcodebook, scale);
    } else {
        e = allow_dynamic_smem((const void*)rvq_encode_kernel<RVQ_MAX_DIM>, smem);
        if (e != cudaSuccess) return set_error(VG_ERR_CUDA, cudaGetErrorString(e));
        rvq_encode_kernel<RVQ_MAX_DIM><<<blocks, 256, smem, st>>>(d, L, K, g->codebook, x, n_items, idx, loss,
                                                                  dcodebook, scale);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? VG_OK : set_error(VG_ERR_CUDA, cudaGetErrorString(e));
}
