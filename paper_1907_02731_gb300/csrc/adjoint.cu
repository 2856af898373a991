// adjoint.cu -- reverse mode of the unrolled, normalised power iteration.
//
// Forward step k (Eq. 4, Eq. 8): y_k = M x^k, x^{k+1} = y_k / ||y_k||, with
// M x = sp . K(sp . x) and K v = (1 - a f^2) G*v + 2 a f G*(f v) - a G*(f^2 v)
// (Eq. 6 / Eq. 7 times alpha).  Given g_{k+1} = dL/dx^{k+1}:
//   u_k      = (g_{k+1} - x^{k+1} (x^{k+1} . g_{k+1})) / ||y_k||   (normalisation)
//   g_k      = M^T u_k = M u_k                                    (M symmetric)
//   dL/dsp  += u_k . K(sp . x^k) + x^k . K(sp . u_k)
//   dL/df   += -2 a sp [u_k (f G*X - G*(f X)) + x^k (f G*U - G*(f U))],
//              U = sp . u_k, X = sp . x^k
// One launch of adjoint_kernel does all of this for one k: six channels
// (U, fU, f^2 U, X, fX, f^2 X) through the same separable Gaussian as the
// forward step (y-pass, x-pass in shared memory, t-ring), and the epilogue
// also reduces x^k . g_k, the dot product the next (earlier) step needs.
#include "sfseg_launch.h"

namespace sfseg {

constexpr int AJ_TX = 32, AJ_TY = 16, AJ_THREADS = 256, AJ_CH = 6;

__global__ void __launch_bounds__(AJ_THREADS) adjoint_kernel(const __grid_constant__ AdjParams P) {
    extern __shared__ __align__(16) float sm[];
    const WorkItem it = P.items[blockIdx.x];
    const VideoGeom g = P.geo[it.video];
    const int rt = P.rt, ry = P.ry, rx = P.rx;
    constexpr int TX = AJ_TX, TY = AJ_TY;
    const int TXH = TX + 2 * rx, TYH = TY + 2 * ry, NR = 2 * rt + 1;
    const int IN = TYH * TXH, YP = TY * TXH, RS = TY * TX;
    float* in6 = sm;                      // [6][TYH][TXH]
    float* yp6 = in6 + AJ_CH * IN;        // [6][TY][TXH]
    float* ring = yp6 + AJ_CH * YP;       // [NR][6][TY][TX]
    const float s_next = (float)*P.s_next, s_cur = (float)*P.s_cur;
    const float c = (float)*P.c_in, inv_ny = (float)(1.0 / *P.ny);
    const float alpha = P.alpha;
    const float* G1 = P.g_in + g.off;
    const float* X1 = P.x_next + g.off;
    const float* X0 = P.x_cur + g.off;
    const float* SP = P.sp + g.off;
    const float* F = P.f + g.off;
    float part = 0.f;
    double acc = 0.0;

    for (int tin = it.t0 - rt; tin < it.t1 + rt; ++tin) {
        if (tin >= 0 && tin < g.nf) {
            for (int idx = threadIdx.x; idx < IN; idx += blockDim.x) {
                const int ly = idx / TXH, lx = idx - ly * TXH;
                const int yy = it.y0 - ry + ly, xg = it.x0 - rx + lx;
                float v[AJ_CH] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (yy >= 0 && yy < g.h && xg >= 0 && xg < g.w) {
                    const long long o = (long long)tin * g.plane + (long long)yy * g.pitch + xg;
                    const float s = SP[o], fv = F[o];
                    const float u = (G1[o] - c * (s_next * X1[o])) * inv_ny;
                    const float U = s * u, X = s * (s_cur * X0[o]);
                    v[0] = U; v[1] = fv * U; v[2] = fv * v[1];
                    v[3] = X; v[4] = fv * X; v[5] = fv * v[4];
                }
#pragma unroll
                for (int ch = 0; ch < AJ_CH; ++ch) in6[ch * IN + idx] = v[ch];
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < YP; idx += blockDim.x) {
                const int oy = idx / TXH, lx = idx - oy * TXH;
                float a[AJ_CH] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int d = 0; d <= 2 * ry; ++d) {
                    const float gw = P.gy[d];
                    const int o = (oy + d) * TXH + lx;
#pragma unroll
                    for (int ch = 0; ch < AJ_CH; ++ch) a[ch] = fmaf(gw, in6[ch * IN + o], a[ch]);
                }
#pragma unroll
                for (int ch = 0; ch < AJ_CH; ++ch) yp6[ch * YP + idx] = a[ch];
            }
            __syncthreads();
            float* slot = ring + (size_t)(tin % NR) * AJ_CH * RS;
            for (int idx = threadIdx.x; idx < RS; idx += blockDim.x) {
                const int oy = idx / TX, ox = idx - oy * TX;
                float a[AJ_CH] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int d = 0; d <= 2 * rx; ++d) {
                    const float gw = P.gx[d];
                    const int o = oy * TXH + ox + d;
#pragma unroll
                    for (int ch = 0; ch < AJ_CH; ++ch) a[ch] = fmaf(gw, yp6[ch * YP + o], a[ch]);
                }
#pragma unroll
                for (int ch = 0; ch < AJ_CH; ++ch) slot[ch * RS + idx] = a[ch];
            }
            __syncthreads();
        }
        const int to = tin - rt;
        if (to >= it.t0 && to < it.t1) {
            for (int idx = threadIdx.x; idx < RS; idx += blockDim.x) {
                const int oy = idx / TX, ox = idx - oy * TX;
                const int yy = it.y0 + oy, xg = it.x0 + ox;
                if (yy >= g.h || xg >= g.w) continue;
                float C[AJ_CH] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int d = -rt; d <= rt; ++d) {
                    const int tp = to + d;
                    if (tp < 0 || tp >= g.nf) continue;
                    const float* sl = ring + (size_t)(tp % NR) * AJ_CH * RS;
                    const float gw = P.gt[d + rt];
#pragma unroll
                    for (int ch = 0; ch < AJ_CH; ++ch) C[ch] = fmaf(gw, sl[ch * RS + idx], C[ch]);
                }
                const long long o = (long long)to * g.plane + (long long)yy * g.pitch + xg;
                const float s = SP[o], fv = F[o];
                const float u = (G1[o] - c * (s_next * X1[o])) * inv_ny;
                const float x = s_cur * X0[o];
                const float af = alpha * fv;
                const float KU = fmaf(-af, fv, 1.f) * C[0] + 2.f * af * C[1] - alpha * C[2];
                const float KX = fmaf(-af, fv, 1.f) * C[3] + 2.f * af * C[4] - alpha * C[5];
                const float gk = s * KU;
                P.g_out[g.off + o] = gk;
                P.dsp[g.off + o] += fmaf(u, KX, x * KU);
                P.df[g.off + o] += -2.f * alpha * s * fmaf(u, fmaf(fv, C[3], -C[4]), x * fmaf(fv, C[0], -C[1]));
                part = fmaf(x, gk, part);
            }
            const float w = warp_sum(part);
            if ((threadIdx.x & 31) == 0) acc += (double)w;
            part = 0.f;
        }
    }
    __syncthreads();
    double* sh = reinterpret_cast<double*>(sm);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        P.partials[blockIdx.x] = s;
        __threadfence();
        const unsigned prev = atomicAdd(P.counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double tot = block_sum_partials(P.partials, (int)gridDim.x);
    if (threadIdx.x != 0) return;
    *P.c_out = tot;
    *P.counter = 0u;
}

// x . g over the volume (FP64 result in *out): scale_x * stored x, g pitched.
__global__ void __launch_bounds__(256) dot_kernel(const float* x, const double* scale_x, const float* gv,
                                                  VideoGeom g, double* partials, unsigned* counter,
                                                  double* out) {
    float part = 0.f;
    for_each_voxel(g, [&](long long, long long o) { part = fmaf(x[g.off + o], gv[g.off + o], part); });
    __shared__ double sh[32];
    __shared__ int s_last;
    const float w = warp_sum(part);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
        partials[blockIdx.x] = s;
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double tot = block_sum_partials(partials, (int)gridDim.x);
    if (threadIdx.x != 0) return;
    *out = tot * *scale_x;
    *counter = 0u;
}

// contiguous FP32 caller array <-> pitched internal FP32 volume, times a
// device scalar (nullable = 1).
__global__ void __launch_bounds__(256) pitch_copy_kernel(const float* src, float* dst, VideoGeom g,
                                                         int to_pitched, const double* scale) {
    const float sc = scale ? (float)*scale : 1.f;
    for_each_voxel(g, [&](long long i, long long o) {
        if (to_pitched) dst[g.off + o] = src[i] * sc;
        else dst[i] = src[g.off + o] * sc;
    });
}

// Per-video state for recomputing forward steps from a checkpoint.
// ---- reverse step on the specialised forward kernel (FP32):
// 1. uprep: u_k = (g_{k+1} - c x^{k+1}) / ||y_k||, c = x^{k+1}.g_{k+1}, into a
//    buffer the forward kernel reads;
// 2. the forward kernel on u with scale = gain = 1 gives g_k = M u_k and, as
//    its adjoint terms, K_U and F_U (the recompute of step k gave K_X, F_X of
//    the stored x^k, to be scaled by s_cur);
// 3. adj_combine: dL/dsp += u K_X s_cur + x K_U, dL/df += -2 alpha sp
//    (u F_X s_cur + x F_U), x = s_cur * stored x^k, and x^k.g_k for the next
//    (earlier) step, g_k = sp K_U.
// Both sweep the whole pitched volume with 16-byte accesses: the pad columns
// are zero in u, x and sp, so they contribute nothing (pitch is a multiple of
// 8 and every video starts 256-byte aligned).
__global__ void __launch_bounds__(256) uprep_kernel(const float* g_in, const float* x_next, const double* s_next,
                                                    const double* c, const double* ny, float* u_out,
                                                    VideoGeom g) {
    const long long n4 = (long long)g.nf * g.plane / 4;
    const float cs = (float)(*c * *s_next), inv = (float)(1.0 / *ny);
    const float4* G = reinterpret_cast<const float4*>(g_in + g.off);
    const float4* X = reinterpret_cast<const float4*>(x_next + g.off);
    float4* U = reinterpret_cast<float4*>(u_out + g.off);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 a = G[i], b = X[i];
        U[i] = make_float4((a.x - cs * b.x) * inv, (a.y - cs * b.y) * inv, (a.z - cs * b.z) * inv,
                           (a.w - cs * b.w) * inv);
    }
}

__global__ void __launch_bounds__(256) adj_combine_kernel(const __grid_constant__ AdjCombineParams P) {
    const VideoGeom g = P.g;
    const long long n4 = (long long)g.nf * g.plane / 4;
    const float s_cur = (float)*P.s_cur, m2a = -2.f * P.alpha;
    auto v4 = [&](const float* p) { return reinterpret_cast<const float4*>(p + g.off); };
    const float4 *U = v4(P.u), *X = v4(P.x_cur), *S = v4(P.sp), *KU = v4(P.ku), *FU = v4(P.fu),
                 *KX = v4(P.kx), *FX = v4(P.fx);
    float4* DS = reinterpret_cast<float4*>(P.dsp + g.off);
    float4* DF = reinterpret_cast<float4*>(P.df + g.off);
    float part = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 u4 = U[i], x4 = X[i], s4 = S[i], ku4 = KU[i], fu4 = FU[i], kx4 = KX[i], fx4 = FX[i];
        float4 ds = DS[i], df = DF[i];
        const float uu[4] = {u4.x, u4.y, u4.z, u4.w}, xx[4] = {x4.x, x4.y, x4.z, x4.w};
        const float ss[4] = {s4.x, s4.y, s4.z, s4.w}, kuv[4] = {ku4.x, ku4.y, ku4.z, ku4.w};
        const float fuv[4] = {fu4.x, fu4.y, fu4.z, fu4.w}, kxv[4] = {kx4.x, kx4.y, kx4.z, kx4.w};
        const float fxv[4] = {fx4.x, fx4.y, fx4.z, fx4.w};
        float dsv[4] = {ds.x, ds.y, ds.z, ds.w}, dfv[4] = {df.x, df.y, df.z, df.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float x = s_cur * xx[j];
            dsv[j] += fmaf(uu[j], s_cur * kxv[j], x * kuv[j]);
            dfv[j] += m2a * ss[j] * fmaf(uu[j], s_cur * fxv[j], x * fuv[j]);
            part = fmaf(x, ss[j] * kuv[j], part);          // x^k . g_k, g_k = sp K_U
        }
        DS[i] = make_float4(dsv[0], dsv[1], dsv[2], dsv[3]);
        DF[i] = make_float4(dfv[0], dfv[1], dfv[2], dfv[3]);
    }
    const float w = warp_sum(part);
    __shared__ double sh[32];
    __shared__ int s_last;
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b += sh[k];
        P.partials[blockIdx.x] = b;
        __threadfence();
        s_last = (atomicAdd(P.counter, 1u) + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double tot = block_sum_partials(P.partials, (int)gridDim.x);
    if (threadIdx.x == 0) {
        *P.c_out = tot;
        *P.counter = 0u;
    }
}

cudaError_t launch_uprep(const float* g_in, const float* x_next, const double* s_next, const double* c,
                         const double* ny, float* u_out, const VideoGeom& g, int blocks, cudaStream_t s) {
    uprep_kernel<<<blocks, 256, 0, s>>>(g_in, x_next, s_next, c, ny, u_out, g);
    return cudaPeekAtLastError();
}

cudaError_t launch_adj_combine(const AdjCombineParams& P, int blocks, cudaStream_t s) {
    adj_combine_kernel<<<blocks, 256, 0, s>>>(P);
    return cudaPeekAtLastError();
}

__global__ void set_state_kernel(VState* st, const double* scale, const double* gain, int iter) {
    VState s{};
    s.scale = *scale;
    s.gain = *gain;
    s.shift = 0.0;
    s.tol = 0.0;
    s.iter = iter;
    s.done = 0;
    s.status = 0;
    s.final_iter = -1;
    s.in_norm = 1.0;
    *st = s;
}

size_t adjoint_smem_bytes(int rt, int ry, int rx) {
    const int TXH = AJ_TX + 2 * rx, TYH = AJ_TY + 2 * ry, NR = 2 * rt + 1;
    const size_t floats = (size_t)AJ_CH * TYH * TXH + (size_t)AJ_CH * AJ_TY * TXH +
                          (size_t)NR * AJ_CH * AJ_TY * AJ_TX;
    return 4 * floats;
}

// The opt-in is a per-function attribute shared by every context, so it only
// ever grows to the largest tile requested so far; radii whose six-channel
// tile does not fit next to the kernel's static shared memory are refused.
cudaError_t setup_adjoint(int rt, int ry, int rx) {
    static int opted = 0;
    const size_t need = adjoint_smem_bytes(rt, ry, rx);
    if (need > (size_t)kMaxDynSmem - 1024) return cudaErrorInvalidValue;
    if ((int)need <= opted) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)need);
    if (e == cudaSuccess) opted = (int)need;
    return e;
}

cudaError_t launch_adjoint(const AdjParams& P, int n_items, cudaStream_t s) {
    adjoint_kernel<<<n_items, AJ_THREADS, adjoint_smem_bytes(P.rt, P.ry, P.rx), s>>>(P);
    return cudaPeekAtLastError();
}

cudaError_t launch_dot(const float* x, const double* scale_x, const float* gv, const VideoGeom& g,
                       double* partials, unsigned* counter, double* out, int blocks, cudaStream_t s) {
    dot_kernel<<<blocks, 256, 0, s>>>(x, scale_x, gv, g, partials, counter, out);
    return cudaPeekAtLastError();
}

cudaError_t launch_pitch_copy(const float* src, float* dst, const VideoGeom& g, int to_pitched,
                              const double* scale, cudaStream_t s) {
    const int blocks = prep_x_blocks(g.n);
    pitch_copy_kernel<<<blocks, 256, 0, s>>>(src, dst, g, to_pitched, scale);
    return cudaPeekAtLastError();
}

cudaError_t launch_set_state(VState* st, const double* scale, const double* gain, int iter,
                             cudaStream_t s) {
    set_state_kernel<<<1, 1, 0, s>>>(st, scale, gain, iter);
    return cudaPeekAtLastError();
}

}  // namespace sfseg
