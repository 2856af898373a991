// step_generic.cu -- one power step y = M x_hat for any radii (Eq. 7, Eq. 9).
//
// The step is the 3D-convolution form of Eq. 7 multiplied by alpha, summed
// over the C pairwise channels of Eq. 9:
//   a = sp x_hat, b_c = f_c a (c < C), q = (sum_c f_c^2) a    (point-wise)
//   A = G * a, B_c = G * b_c, Q = G * q, G = g_t (x) g_y (x) g_x, zero padding
//   y = sp [(C - alpha sum_c f_c^2) A + 2 alpha sum_c f_c B_c - alpha Q]
// which is M x_hat for M_ij = sp_i sp_j sum_c [1 - alpha (f_ci - f_cj)^2] G_ij
// (Eq. 2 per channel); C + 2 convolutions.  For C = 1 this is
// y = sp [(1 - alpha f^2) A + 2 alpha f B - alpha Q], q = f (f a).
// The separable Gaussian is applied as three 1D passes (Sec. 4: 3 x 7 x 7
// taps become 3 + 7 + 7).  Each CTA owns a 32 x 16 (x, y) tile of one video
// and streams the frames of its range: every input frame is loaded once with
// its spatial halo, filtered in y then x in shared memory, and kept in a ring
// of 2 rt + 1 filtered frames from which the t-pass and the combine emit the
// output frame t - rt.  Reductions for the norm and the Rayleigh quotient are
// FP32 per frame, FP64 across frames and CTAs.
//
// This kernel handles every radius up to the library limits and every channel
// count up to kMaxChan (as far as the buffers fit in shared memory); it is the
// reference point for the specialised kernels and favours simplicity.
#include "sfseg_common.cuh"
#include "sfseg_launch.h"

namespace sfseg {

constexpr int GT_TX = 32, GT_TY = 16, GT_THREADS = 256;

template <typename TS, int NCH>
__global__ void __launch_bounds__(GT_THREADS)
step_generic_kernel(const __grid_constant__ StepParams P)
{
    constexpr int C = NCH - 2;       // pairwise feature channels
    extern __shared__ __align__(16) float sm[];
    const WorkItem it = P.items[blockIdx.x];
    const int v = it.video;
    if (!dbg_ok((int)blockIdx.x < P.n_items && v >= 0 && v < P.n_videos, kDbgSlot, blockIdx.x, v)) return;
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
    if (!dbg_ok(0 <= it.t0 && it.t0 < it.t1 && it.t1 <= g.nf && 0 <= it.x0 && it.x0 < g.w && 0 <= it.y0 &&
                    it.y0 < g.h && g.off + (long long)g.nf * g.plane <= P.total,
                kDbgSegment, blockIdx.x, ((long long)it.t0 << 32) | (unsigned)it.t1))
        return;
    const int rt = P.rt, ry = P.ry, rx = P.rx;
    constexpr int TX = GT_TX, TY = GT_TY;
    const int TXH = TX + 2 * rx, TYH = TY + 2 * ry, NR = 2 * rt + 1;
    const int IN = TYH * TXH, YP = TY * TXH, RS = TY * TX;
    float* inb = sm;                 // [NCH][TYH][TXH]  a, b_c, q with halo
    float* yp = inb + NCH * IN;      // [NCH][TY][TXH]   after the y-pass
    float* ring = yp + NCH * YP;     // [NR][NCH][TY][TX] after the x-pass
    const TS* X = (const TS*)P.x_in + g.off;
    const TS* SP = (const TS*)P.sp + g.off;
    const TS* F = (const TS*)P.f + g.off;     // channel c at F + c * fstride
    const long long fs = P.fstride;
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
                float ch[NCH];
#pragma unroll
                for (int k = 0; k < NCH; ++k) ch[k] = 0.f;
                if (yy >= 0 && yy < g.h && xg >= 0 && xg < g.w) {
                    const long long o = (long long)tin * g.plane + (long long)yy * g.pitch + xg;
                    const float xh = scale * to_f(X[o]);
                    ch[0] = to_f(SP[o]) * xh;
                    if (C == 1) {
                        const float fv = to_f(F[o]);
                        ch[1] = fv * ch[0];
                        ch[2] = fv * ch[1];
                    } else {
                        float fsq = 0.f;
#pragma unroll
                        for (int c = 0; c < C; ++c) {
                            const float fv = to_f(F[c * fs + o]);
                            ch[1 + c] = fv * ch[0];
                            fsq = fmaf(fv, fv, fsq);
                        }
                        ch[NCH - 1] = fsq * ch[0];
                    }
                }
#pragma unroll
                for (int k = 0; k < NCH; ++k) inb[k * IN + idx] = ch[k];
            }
            __syncthreads();
            // 2. y-pass over the TY output rows, all TXH columns
            for (int idx = threadIdx.x; idx < YP; idx += blockDim.x) {
                const int oy = idx / TXH, lx = idx - oy * TXH;
                float cs[NCH];
#pragma unroll
                for (int k = 0; k < NCH; ++k) cs[k] = 0.f;
                for (int d = 0; d <= 2 * ry; ++d) {
                    const float gw = P.gy[d];
                    const int o = (oy + d) * TXH + lx;
#pragma unroll
                    for (int k = 0; k < NCH; ++k) cs[k] = fmaf(gw, inb[k * IN + o], cs[k]);
                }
#pragma unroll
                for (int k = 0; k < NCH; ++k) yp[k * YP + idx] = cs[k];
            }
            __syncthreads();
            // 3. x-pass into the ring slot of frame tin
            float* slot = ring + (size_t)(tin % NR) * NCH * RS;
            for (int idx = threadIdx.x; idx < RS; idx += blockDim.x) {
                const int oy = idx / TX, ox = idx - oy * TX;
                float cs[NCH];
#pragma unroll
                for (int k = 0; k < NCH; ++k) cs[k] = 0.f;
                for (int d = 0; d <= 2 * rx; ++d) {
                    const float gw = P.gx[d];
                    const int o = oy * TXH + ox + d;
#pragma unroll
                    for (int k = 0; k < NCH; ++k) cs[k] = fmaf(gw, yp[k * YP + o], cs[k]);
                }
#pragma unroll
                for (int k = 0; k < NCH; ++k) slot[k * RS + idx] = cs[k];
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
                float cs[NCH];
#pragma unroll
                for (int k = 0; k < NCH; ++k) cs[k] = 0.f;
                for (int d = -rt; d <= rt; ++d) {
                    const int tp = to + d;
                    if (tp < 0 || tp >= g.nf) continue;
                    const float* sl = ring + (size_t)(tp % NR) * NCH * RS;
                    const float gw = P.gt[d + rt];
#pragma unroll
                    for (int k = 0; k < NCH; ++k) cs[k] = fmaf(gw, sl[k * RS + idx], cs[k]);
                }
                const long long o = (long long)to * g.plane + (long long)yy * g.pitch + xg;
                if (!dbg_ok(o < (long long)g.nf * g.plane, kDbgStore, o, g.nf)) continue;
                const float s = to_f(SP[o]);
                const float xh = scale * to_f(X[o]);
                float inner;
                if (C == 1) {
                    const float fv = to_f(F[o]);
                    const float af = alpha * fv;
                    inner = fmaf(-af, fv, 1.f) * cs[0] + 2.f * af * cs[1] - alpha * cs[2];
                } else {
                    float fsq = 0.f, fb = 0.f;
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        const float fv = to_f(F[c * fs + o]);
                        fsq = fmaf(fv, fv, fsq);
                        fb = fmaf(fv, cs[1 + c], fb);
                    }
                    inner = fmaf(-alpha, fsq, (float)C) * cs[0] + 2.f * alpha * fb - alpha * cs[NCH - 1];
                }
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

SFSEG_DEBUG_TU(generic)

size_t generic_smem_bytes(int rt, int ry, int rx, int nchan) {
    const size_t nch = (size_t)nchan + 2;
    const int TXH = GT_TX + 2 * rx, TYH = GT_TY + 2 * ry, NR = 2 * rt + 1;
    size_t floats = nch * ((size_t)TYH * TXH + (size_t)GT_TY * TXH + (size_t)NR * GT_TY * GT_TX);
    size_t red = (size_t)GT_THREADS * kRed * 2;   // doubles as floats for finalize
    return 4 * (floats > red ? floats : red);
}

void generic_tile(int* tx, int* ty) { *tx = GT_TX; *ty = GT_TY; }

// The dynamic shared-memory opt-in is set at context creation (not during a
// stream capture); the launch itself only enqueues.  The opt-in is a
// per-function attribute shared by every context in the process, so it is
// always set to the size of the largest supported radii: a later context with
// small radii must not lower the limit another context's launches rely on.
// Dynamic shared memory of the any-radius kernel is capped below the
// per-block opt-in limit, which also has to hold the kernel's static shared
// variables.
size_t generic_smem_cap() { return (size_t)kMaxDynSmem - 1024; }

template <int NCH>
static cudaError_t setup_generic_nch() {
    // the largest radii this channel count supports within the shared-memory limit
    size_t smem = generic_smem_bytes(kMaxRt, kMaxR, kMaxR, NCH - 2);
    if (smem > generic_smem_cap()) smem = generic_smem_cap();
    cudaError_t e = cudaFuncSetAttribute(step_generic_kernel<float, NCH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_generic_kernel<__nv_bfloat16, NCH>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_generic_kernel<__half, NCH>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

cudaError_t setup_step_generic(int, int, int) {
    cudaError_t e = setup_generic_nch<3>();
    if (e == cudaSuccess) e = setup_generic_nch<4>();
    if (e == cudaSuccess) e = setup_generic_nch<5>();
    if (e == cudaSuccess) e = setup_generic_nch<6>();
    return e;
}

template <typename TS>
static cudaError_t launch_generic_t(const StepParams& P, int n_items, cudaStream_t s) {
    const size_t smem = generic_smem_bytes(P.rt, P.ry, P.rx, P.nchan);
    switch (P.nchan) {
        case 1: step_generic_kernel<TS, 3><<<n_items, GT_THREADS, smem, s>>>(P); break;
        case 2: step_generic_kernel<TS, 4><<<n_items, GT_THREADS, smem, s>>>(P); break;
        case 3: step_generic_kernel<TS, 5><<<n_items, GT_THREADS, smem, s>>>(P); break;
        case 4: step_generic_kernel<TS, 6><<<n_items, GT_THREADS, smem, s>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
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
