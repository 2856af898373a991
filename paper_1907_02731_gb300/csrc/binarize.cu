// binarize.cu -- the projection step of Alg. 1 (Step 3) and the final hard
// threshold (Sec. 4, "Binarization - Spectral vs Discrete space").
//
// After a few power steps in the continuous space the iterate is projected
// through a sigmoid onto an almost discrete space and the next step starts
// from that projection; after the last step a hard threshold gives the
// segmentation.  The paper gives no parameters; with u = x / max(x) (x >= 0
// by Perron-Frobenius, so u lies in [0, 1] whatever the scale of x):
//   projection   p = 1 / (1 + exp(-beta (u - tau))), then renormalised;
//   final mask   m = [u >= theta].
//
// Kernels:
//   vmax_stored_kernel  max of the stored iterate of one video (pitched, storage type)
//   project_kernel      p of every voxel, stored in place; FP64 block partials of p^2
//   project_finish      fixed-order sum of the partials (one block) -> the video's scale 1 / ||p||
//   vmax_f32_kernel     max of a contiguous FP32 array (the caller's x)
//   threshold_kernel    m = [x >= theta * max(x)] as bytes
// Maxima go through an order-preserving map of the float bits onto unsigned
// integers, so that atomicMax on the integers is a max on the floats.
#include "sfseg_launch.h"

namespace sfseg {

__device__ __forceinline__ float block_max(float v) {
    __shared__ float sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : -INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;   // valid in thread 0
}

template <typename TS>
__global__ void __launch_bounds__(256) vmax_stored_kernel(const __grid_constant__ ProjectParams P) {
    if (P.state[P.video].done) return;
    const VideoGeom g = P.g;
    const TS* Z = (const TS*)P.buf + g.off;
    float m = -INFINITY;
    for_each_voxel(g, [&](long long, long long o) { m = fmaxf(m, to_f(Z[o])); });
    m = block_max(m);
    if (threadIdx.x == 0) atomicMax(P.vmax_key, float_key(m));
}

template <typename TS>
__global__ void __launch_bounds__(256) project_kernel(const __grid_constant__ ProjectParams P) {
    const VideoGeom g = P.g;
    TS* Z = (TS*)P.buf + g.off;
    const float vmax = key_float(*P.vmax_key);
    float part = 0.f;
    if (!P.state[P.video].done && vmax > 0.f && isfinite(vmax)) {
        const float inv = 1.f / vmax;
        for_each_voxel(g, [&](long long, long long o) {
            const float u = to_f(Z[o]) * inv;
            const TS ps = from_f<TS>(1.f / (1.f + expf(-P.beta * (u - P.tau))));
            Z[o] = ps;
            const float pv = to_f(ps);
            part = fmaf(pv, pv, part);
        });
    }
    // FP32 per thread, FP64 per warp and block
    const float w = warp_sum(part);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
        P.partials[blockIdx.x] = s;
    }
}

__global__ void project_finish_kernel(const __grid_constant__ ProjectParams P) {
    const double s = block_sum_partials(P.partials, P.n_blocks);
    if (threadIdx.x != 0) return;
    VState* st = P.state + P.video;
    const float vmax = key_float(*P.vmax_key);
    *P.vmax_key = 0u;   // ready for the next projection
    if (st->done) return;
    if (!(vmax > 0.f) || !isfinite(vmax) || !(s > 0.0) || !isfinite(s)) {
        st->status = isfinite(vmax) && isfinite(s) ? 4 : 5;   // SFSEG_EZERONORM / SFSEG_ENONFINITE
        st->done = 1;
        return;
    }
    // the stored vector is the projection p; the next step reads x_hat = p / ||p||
    st->scale = 1.0 / sqrt(s);
}

__global__ void __launch_bounds__(256) vmax_f32_kernel(const float* x, long long n, unsigned* key) {
    float m = -INFINITY;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, x[i]);
    m = block_max(m);
    if (threadIdx.x == 0) atomicMax(key, float_key(m));
}

__global__ void __launch_bounds__(256) threshold_kernel(const float* x, long long n, const unsigned* key,
                                                        float theta, unsigned char* mask) {
    const float cut = theta * key_float(*key);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        mask[i] = (x[i] >= cut) ? 1 : 0;
}

template <typename TS>
static cudaError_t launch_project_t(const ProjectParams& P, cudaStream_t s) {
    vmax_stored_kernel<TS><<<P.n_blocks, 256, 0, s>>>(P);
    project_kernel<TS><<<P.n_blocks, 256, 0, s>>>(P);
    project_finish_kernel<<<1, 256, 0, s>>>(P);
    return cudaPeekAtLastError();
}

cudaError_t launch_project(int storage, const ProjectParams& P, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_project_t<float>(P, s);
        case 1: return launch_project_t<__nv_bfloat16>(P, s);
        case 2: return launch_project_t<__half>(P, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_threshold(const float* x, long long n, unsigned* key, float theta, unsigned char* mask,
                             int n_blocks, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(key, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    vmax_f32_kernel<<<n_blocks, 256, 0, s>>>(x, n, key);
    threshold_kernel<<<n_blocks, 256, 0, s>>>(x, n, key, theta, mask);
    return cudaPeekAtLastError();
}

}  // namespace sfseg
