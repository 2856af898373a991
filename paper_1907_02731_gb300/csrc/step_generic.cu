// step_generic.cu -- one power step y = M x_hat for any radii (Eq. 7).
//
// The step is the 3D-convolution form of Eq. 7 multiplied by alpha:
//   a0 = sp x_hat, a1 = f a0, a2 = f a1                     (point-wise, Eq. 7)
//   C_c = G * a_c,  G = g_t (x) g_y (x) g_x, zero padding     (3 convolutions)
//   y = sp [(1 - alpha f^2) C0 + 2 alpha f C1 - alpha C2]     (= M x_hat, Eq. 2)
// with the separable Gaussian applied as three 1D passes (Sec. 4: 3 x 7 x 7
// taps become 3 + 7 + 7).  Each CTA owns a 32 x 16 (x, y) tile of one video
// and streams the frames of its range: every input frame is loaded once with
// its spatial halo, filtered in y then x in shared memory, and kept in a ring
// of 2 rt + 1 filtered frames from which the t-pass and the combine emit the
// output frame t - rt.  Reductions for the norm and the Rayleigh quotient are
// FP32 per frame, FP64 across frames and CTAs.
//
// This kernel handles every radius up to the library limits and is the
// reference point for the specialised kernels; it favours simplicity.
#include "sfseg_common.cuh"
#include "sfseg_launch.h"

namespace sfseg {

constexpr int GT_TX = 32, GT_TY = 16, GT_THREADS = 256;

template <typename TS>
__global__ void __launch_bounds__(GT_THREADS)
step_generic_kernel(const __grid_constant__ StepParams P)
{
    extern __shared__ __align__(16) float sm[];
    const WorkItem it = P.items[blockIdx.x];
    const int v = it.video;
    VState* st = P.state + v;
    __shared__ int s_skip;
    __shared__ float s_scale, s_gain, s_shift;
    if (threadIdx.x == 0) {
        s_skip = st->done;
        s_scale = (float)st->scale;
        s_gain = (float)st->gain;
        s_shift = (float)st->shift;
    }
    __syncthreads();
    if (s_skip) return;

    const VideoGeom g = P.geo[v];
    const int rt = P.rt, ry = P.ry, rx = P.rx;
    constexpr int TX = GT_TX, TY = GT_TY;
    const int TXH = TX + 2 * rx, TYH = TY + 2 * ry, NR = 2 * rt + 1;
    const int IN = TYH * TXH, YP = TY * TXH, RS = TY * TX;
    float* in3 = sm;                 // [3][TYH][TXH]  a0, a1, a2 with halo
    float* yp = in3 + 3 * IN;        // [3][TY][TXH]   after the y-pass
    float* ring = yp + 3 * YP;       // [NR][3][TY][TX] after the x-pass
    const TS* X = (const TS*)P.x_in + g.off;
    const TS* SP = (const TS*)P.sp + g.off;
    const TS* F = (const TS*)P.f + g.off;
    TS* Z = P.z_out ? (TS*)P.z_out + g.off : nullptr;
    float* FO = P.final_out ? P.final_out[v] : nullptr;
    const float alpha = P.alpha, scale = s_scale, gain = s_gain, shift = s_shift;

    float part[kRed] = {0.f, 0.f, 0.f, 0.f};
    double acc[kRed] = {0.0, 0.0, 0.0, 0.0};

    for (int tin = it.t0 - rt; tin < it.t1 + rt; ++tin) {
        if (tin >= 0 && tin < g.nf) {
            // 1. load frame tin with halo; point-wise products (zero outside)
            for (int idx = threadIdx.x; idx < IN; idx += blockDim.x) {
                const int ly = idx / TXH, lx = idx - ly * TXH;
                const int yy = it.y0 - ry + ly, xg = it.x0 - rx + lx;
                float a0 = 0.f, a1 = 0.f, a2 = 0.f;
                if (yy >= 0 && yy < g.h && xg >= 0 && xg < g.w) {
                    const long long o = (long long)tin * g.plane + (long long)yy * g.pitch + xg;
                    const float xh = scale * to_f(X[o]);
                    const float s = to_f(SP[o]), fv = to_f(F[o]);
                    a0 = s * xh;
                    a1 = fv * a0;
                    a2 = fv * a1;
                }
                in3[idx] = a0;
                in3[IN + idx] = a1;
                in3[2 * IN + idx] = a2;
            }
            __syncthreads();
            // 2. y-pass over the TY output rows, all TXH columns
            for (int idx = threadIdx.x; idx < YP; idx += blockDim.x) {
                const int oy = idx / TXH, lx = idx - oy * TXH;
                float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                for (int d = 0; d <= 2 * ry; ++d) {
                    const float gw = P.gy[d];
                    const int o = (oy + d) * TXH + lx;
                    c0 = fmaf(gw, in3[o], c0);
                    c1 = fmaf(gw, in3[IN + o], c1);
                    c2 = fmaf(gw, in3[2 * IN + o], c2);
                }
                yp[idx] = c0;
                yp[YP + idx] = c1;
                yp[2 * YP + idx] = c2;
            }
            __syncthreads();
            // 3. x-pass into the ring slot of frame tin
            float* slot = ring + (size_t)(tin % NR) * 3 * RS;
            for (int idx = threadIdx.x; idx < RS; idx += blockDim.x) {
                const int oy = idx / TX, ox = idx - oy * TX;
                float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                for (int d = 0; d <= 2 * rx; ++d) {
                    const float gw = P.gx[d];
                    const int o = oy * TXH + ox + d;
                    c0 = fmaf(gw, yp[o], c0);
                    c1 = fmaf(gw, yp[YP + o], c1);
                    c2 = fmaf(gw, yp[2 * YP + o], c2);
                }
                slot[idx] = c0;
                slot[RS + idx] = c1;
                slot[2 * RS + idx] = c2;
            }
            __syncthreads();
        }
        // 4. t-pass + combine for output frame to = tin - rt
        const int to = tin - rt;
        if (to >= it.t0 && to < it.t1) {
            for (int idx = threadIdx.x; idx < RS; idx += blockDim.x) {
                const int oy = idx / TX, ox = idx - oy * TX;
                const int yy = it.y0 + oy, xg = it.x0 + ox;
                if (yy >= g.h || xg >= g.w) continue;
                float C0 = 0.f, C1 = 0.f, C2 = 0.f;
                for (int d = -rt; d <= rt; ++d) {
                    const int tp = to + d;
                    if (tp < 0 || tp >= g.nf) continue;
                    const float* sl = ring + (size_t)(tp % NR) * 3 * RS;
                    const float gw = P.gt[d + rt];
                    C0 = fmaf(gw, sl[idx], C0);
                    C1 = fmaf(gw, sl[RS + idx], C1);
                    C2 = fmaf(gw, sl[2 * RS + idx], C2);
                }
                const long long o = (long long)to * g.plane + (long long)yy * g.pitch + xg;
                const float s = to_f(SP[o]), fv = to_f(F[o]);
                const float xh = scale * to_f(X[o]);
                const float af = alpha * fv;
                const float inner = fmaf(-af, fv, 1.f) * C0 + 2.f * af * C1 - alpha * C2;
                float z = gain * (s * inner);
                if (FO) {
                    FO[((long long)to * g.h + yy) * g.w + xg] = z;
                } else if (Z) {
                    const TS zs = from_f<TS>(z);
                    Z[o] = zs;
                    z = to_f(zs);
                }
                part[0] = fmaf(z, z, part[0]);
                part[1] = fmaf(xh, z, part[1]);
                part[2] = fmaf(xh, xh, part[2]);
                const float dz = fmaf(-shift, xh, z);
                part[3] = fmaf(dz, dz, part[3]);
            }
            warp_flush(part, acc);
        }
    }
    __syncthreads();
    double* sh = reinterpret_cast<double*>(sm);   // stencil buffers are free now
    block_sum_lane0(acc, sh);
    if (threadIdx.x == 0)
        for (int c = 0; c < kRed; ++c) P.partials[(long long)blockIdx.x * kRed + c] = acc[c];
    arrive_and_finalize(P, v, sh);
}

size_t generic_smem_bytes(int rt, int ry, int rx) {
    const int TXH = GT_TX + 2 * rx, TYH = GT_TY + 2 * ry, NR = 2 * rt + 1;
    size_t floats = 3 * (size_t)TYH * TXH + 3 * (size_t)GT_TY * TXH + (size_t)NR * 3 * GT_TY * GT_TX;
    size_t red = (size_t)GT_THREADS * kRed * 2;   // doubles as floats for finalize
    return 4 * (floats > red ? floats : red);
}

void generic_tile(int* tx, int* ty) { *tx = GT_TX; *ty = GT_TY; }

// The dynamic shared-memory opt-in is set at context creation (not during a
// stream capture); the launch itself only enqueues.  The opt-in is a
// per-function attribute shared by every context in the process, so it is
// always set to the size of the largest supported radii: a later context with
// small radii must not lower the limit another context's launches rely on.
cudaError_t setup_step_generic(int, int, int) {
    const int smem = (int)generic_smem_bytes(kMaxRt, kMaxR, kMaxR);
    cudaError_t e = cudaFuncSetAttribute(step_generic_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_generic_kernel<__nv_bfloat16>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_generic_kernel<__half>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <typename TS>
static cudaError_t launch_generic_t(const StepParams& P, int n_items, cudaStream_t s) {
    const size_t smem = generic_smem_bytes(P.rt, P.ry, P.rx);
    step_generic_kernel<TS><<<n_items, GT_THREADS, smem, s>>>(P);
    return cudaPeekAtLastError();
}

cudaError_t launch_step_generic(int storage, const StepParams& P, int n_items, cudaStream_t s) {
    switch (storage) {
        case 0: return launch_generic_t<float>(P, n_items, s);
        case 1: return launch_generic_t<__nv_bfloat16>(P, n_items, s);
        case 2: return launch_generic_t<__half>(P, n_items, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace sfseg
