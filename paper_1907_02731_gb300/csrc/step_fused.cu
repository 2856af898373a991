// step_fused.cu -- all K power steps of a context in one cooperative launch.
//
// Small volumes pay the fixed cost of a launch, a pipeline fill and a drain
// on every power step of the per-step kernels.  This kernel runs the whole
// iteration loop of Alg. 1 (Eq. 4 + Eq. 8) as one persistent grid, with two
// grid-wide barriers per step:
//
//   phase 1  per (video, 32 x 16 tile, frame) unit: the point-wise products
//            a0 = sp x, a1 = f a0, a2 = f a1 of the STORED iterate (the
//            deferred scale is linear and is applied in phase 2), then the
//            y and x passes of the separable Gaussian (Eq. 7, Sec. 4), into a
//            scratch of three FP32 channel volumes (L2-resident for the
//            volumes this kernel serves);
//   barrier
//   phase 2  per (video, frame, row chunk) unit: the t-pass over 2 rt + 1
//            scratch frames, the combine y = sp [(1 - a f^2) C0 + 2 a f C1
//            - a C2] with the scale and gain, the store (or the caller's FP32
//            buffer after the last step) and the FP32/FP64 partial sums of
//            z.z, x.z, x.x, |z - s x|^2, one FP64 record per CTA and video;
//   barrier
//   finalize CTA G - 1 - (v mod G) sums video v's records in a fixed order
//            and updates its scalars (Rayleigh quotient, residual, norm, next
//            scale and gain: the same finish_step as the per-step kernels),
//            while the other CTAs start the next phase 1 (which needs no
//            scalars); the next phase 2 reads them after the next barrier.
//
// Videos that converged (or failed) skip their phase-2 units (phase 1 filters
// them once more into the scratch, which nothing reads); when all have, every
// CTA leaves the loop together after the first barrier (they read the same
// settled scalars).  Each
// barrier wait is limited in time: a CTA that gives up raises a grid-wide
// abort flag, marks every video SFSEG_ETIMEOUT and returns; the other CTAs see
// the flag (or their own limit) and return too.  No trap, no unbounded wait.
#include <cuda_runtime.h>

#include "sfseg_common.cuh"
#include "sfseg_launch.h"

namespace sfseg {

constexpr int FU_TX = 32, FU_TY = 16, FU_THREADS = 256;
constexpr unsigned long long kFusedWaitNs = 1000000000ull;   // a barrier wait gives up after 1 s

__device__ __forceinline__ unsigned long long fu_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of the cooperative launch: a monotonic arrival count
// (zeroed before the launch).  Barrier b (0, 1, ...) completes when the count
// reaches (b + 1) G; arrival is a release add, the wait an acquire load, so a
// CTA sees every write the others made before arriving.  Returns false when
// the wait gave up (time limit, or the grid-wide abort flag raised by a CTA
// that gave up); `skip_arrive` (fault injection for tests) makes the CTA wait
// without arriving, so the barrier can never complete.
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ bool grid_barrier(unsigned* bar, unsigned n_ctas, unsigned& nb, bool skip_arrive) {
    __shared__ int s_ok;
    __syncthreads();   // the block's writes precede thread 0's release
    if (threadIdx.x == 0) {
        const volatile int* abort = reinterpret_cast<volatile int*>(bar + 2);
        const unsigned target = (nb + 1) * n_ctas;
        int ok = 1;
        if (!skip_arrive) red_release_add(bar, 1u);
        if (ld_acquire(bar) < target) {
            const unsigned long long t0 = fu_ns();
            unsigned i = 0;
            while (ld_acquire(bar) < target) {
                if (*abort) { ok = 0; break; }
                if ((++i & 31u) == 0u && fu_ns() - t0 > kFusedWaitNs) {
                    atomicExch(reinterpret_cast<int*>(bar + 2), 1);
                    ok = 0;
                    break;
                }
            }
        }
        nb += 1;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Phase-1 unit u of the grid -> video and (frame, tile) inside it.
__device__ __forceinline__ int unit_video(const int* begin, int n_videos, int u) {
    int lo = 0, hi = n_videos - 1;
    while (lo < hi) {   // last video whose first unit is <= u
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= u) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Finalize of video v after the step's phase 2 (run by one CTA per video):
// the video's run partials summed in a fixed order (strided per thread, then a
// halving tree in shared memory), then the norm / Rayleigh / residual update
// of finish_step.  A video that was already done skipped the step and is left
// alone.  Every thread of the block calls it; `red` holds blockDim * kRed
// doubles.
__device__ void fused_finalize(const StepParams& P, int v, double* red) {
    const int b = P.item_begin[v], e = P.item_begin[v + 1];
    double acc[kRed] = {0.0, 0.0, 0.0, 0.0};
    for (int i = b + (int)threadIdx.x; i < e; i += blockDim.x) {
        const long long id = P.vseg[i];
        for (int c = 0; c < kRed; ++c) acc[c] += __ldcg(&P.partials[id * kRed + c]);
    }
    for (int c = 0; c < kRed; ++c) red[c * blockDim.x + threadIdx.x] = acc[c];
    __syncthreads();
    for (int n = blockDim.x; n > 1;) {
        const int h = (n + 1) / 2;
        if ((int)threadIdx.x < n - h)
            for (int c = 0; c < kRed; ++c) red[c * blockDim.x + threadIdx.x] += red[c * blockDim.x + threadIdx.x + h];
        __syncthreads();
        n = h;
    }
    if (threadIdx.x == 0) {
        VState* st = P.state + v;
        if (!st->done) {
            double S[kRed];
            for (int c = 0; c < kRed; ++c) S[c] = red[c * blockDim.x];
            const int k = st->iter;
            double* row = (k < P.trace_cap) ? P.trace + ((long long)v * P.trace_cap + k) * 3 : nullptr;
            finish_step(st, row, S, P.geo[v].n, &P.rec);
        }
    }
    __syncthreads();   // red is reused
}

template <typename TS>
__global__ void __launch_bounds__(FU_THREADS)
step_fused_kernel(const __grid_constant__ FusedParams F) {
    const StepParams& P = F.S;
    extern __shared__ __align__(16) float sm[];
    const int rt = P.rt, ry = P.ry, rx = P.rx;
    const int TXH = FU_TX + 2 * rx, TYH = FU_TY + 2 * ry;
    const int IN = TYH * TXH, YP = FU_TY * TXH;
    float* inb = sm;              // [3][TYH][TXH] point-wise products with halo
    float* yp = inb + 3 * IN;     // [3][FU_TY][TXH] after the y-pass
    const unsigned G = gridDim.x;
    unsigned nb = 0;   // barriers passed
    __shared__ int s_all_done;
    __shared__ float s_sg, s_scale, s_shift;
    __shared__ int s_skip;
    const float alpha = P.alpha;

    for (int k = 0; k < F.n_steps; ++k) {
        const TS* X = (const TS*)((k & 1) ? F.buf1 : F.buf0);
        TS* Z = (TS*)((k & 1) ? F.buf0 : F.buf1);
        const bool final_step = F.final_mode && k == F.n_steps - 1;

        // ------------------------------------------------ phase 1: y, x passes
        // (videos that are done are filtered too -- the scratch of a finished
        // video is never read -- so that phase 1 waits on no scalar)
        for (int u = blockIdx.x; u < F.n_units1; u += G) {
            const int v = unit_video(F.unit1_begin, F.n_videos, u);
            const VideoGeom g = P.geo[v];
            if (!dbg_ok(g.off + (long long)g.nf * g.plane <= F.total, kDbgUnit, u, v)) continue;
            const int ntx = (g.w + FU_TX - 1) / FU_TX, nty = (g.h + FU_TY - 1) / FU_TY;
            const int local = u - F.unit1_begin[v];
            const int t = local / (ntx * nty), r = local - t * (ntx * nty);
            const int y0 = (r / ntx) * FU_TY, x0 = (r - (r / ntx) * ntx) * FU_TX;
            if (!dbg_ok(t < g.nf && y0 < g.h && x0 < g.w, kDbgUnit, u, t)) continue;   // uniform over the CTA
            const TS* Xv = X + g.off;
            const TS* SPv = (const TS*)P.sp + g.off;
            const TS* Fv = (const TS*)P.f + g.off;
            constexpr int UNR = 4;   // loads of UNR rounds in flight before the stores
            for (int base = 0; base < IN; base += UNR * FU_THREADS) {
                float xs[UNR], ss[UNR], fs[UNR];
#pragma unroll
                for (int j = 0; j < UNR; ++j) {
                    const int idx = base + j * FU_THREADS + (int)threadIdx.x;
                    const int ly = idx / TXH, lx = idx - ly * TXH;
                    const int yy = y0 - ry + ly, xx = x0 - rx + lx;
                    xs[j] = ss[j] = fs[j] = 0.f;
                    if (idx < IN && yy >= 0 && yy < g.h && xx >= 0 && xx < g.w) {
                        const long long o = (long long)t * g.plane + (long long)yy * g.pitch + xx;
                        // the iterate was written by other SMs in the previous
                        // step: read it through L2 (an L1 line may be stale)
                        xs[j] = to_f(__ldcg(Xv + o));
                        ss[j] = to_f(SPv[o]);
                        fs[j] = to_f(Fv[o]);
                    }
                }
#pragma unroll
                for (int j = 0; j < UNR; ++j) {
                    const int idx = base + j * FU_THREADS + (int)threadIdx.x;
                    if (idx < IN) {
                        const float a0 = ss[j] * xs[j], a1 = fs[j] * a0;
                        inb[idx] = a0;
                        inb[IN + idx] = a1;
                        inb[2 * IN + idx] = fs[j] * a1;
                    }
                }
            }
            __syncthreads();
            // y-pass: NO outputs per thread in flight, so their shared-memory
            // loads overlap (the tap loop has a run-time trip count)
            constexpr int NO = 4;
            for (int base = 0; base < YP; base += NO * FU_THREADS) {
                float c[NO][3];
                int oo[NO];
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    const int idx = min(base + j * FU_THREADS + (int)threadIdx.x, YP - 1);
                    const int oy = idx / TXH;
                    oo[j] = oy * TXH + (idx - oy * TXH);
                    c[j][0] = c[j][1] = c[j][2] = 0.f;
                }
#pragma unroll 2
                for (int d = 0; d <= 2 * ry; ++d) {
                    const float gw = P.gy[d];
#pragma unroll
                    for (int j = 0; j < NO; ++j) {
                        const int o = oo[j] + d * TXH;
                        c[j][0] = fmaf(gw, inb[o], c[j][0]);
                        c[j][1] = fmaf(gw, inb[IN + o], c[j][1]);
                        c[j][2] = fmaf(gw, inb[2 * IN + o], c[j][2]);
                    }
                }
#pragma unroll
                for (int j = 0; j < NO; ++j) {
                    const int idx = base + j * FU_THREADS + (int)threadIdx.x;
                    if (idx < YP) {
                        yp[idx] = c[j][0];
                        yp[YP + idx] = c[j][1];
                        yp[2 * YP + idx] = c[j][2];
                    }
                }
            }
            __syncthreads();
            // x-pass: the tile's FU_TY x FU_TX outputs, NX per thread
            float* pv = F.pvol + g.off;
            constexpr int NX = FU_TY * FU_TX / FU_THREADS;
            static_assert(NX * FU_THREADS == FU_TY * FU_TX, "x-pass outputs per thread");
            {
                float c[NX][3];
                int oo[NX];
#pragma unroll
                for (int j = 0; j < NX; ++j) {
                    const int idx = j * FU_THREADS + (int)threadIdx.x;
                    const int oy = idx / FU_TX;
                    oo[j] = oy * TXH + (idx - oy * FU_TX);
                    c[j][0] = c[j][1] = c[j][2] = 0.f;
                }
#pragma unroll 2
                for (int d = 0; d <= 2 * rx; ++d) {
                    const float gw = P.gx[d];
#pragma unroll
                    for (int j = 0; j < NX; ++j) {
                        const int o = oo[j] + d;
                        c[j][0] = fmaf(gw, yp[o], c[j][0]);
                        c[j][1] = fmaf(gw, yp[YP + o], c[j][1]);
                        c[j][2] = fmaf(gw, yp[2 * YP + o], c[j][2]);
                    }
                }
#pragma unroll
                for (int j = 0; j < NX; ++j) {
                    const int idx = j * FU_THREADS + (int)threadIdx.x;
                    const int oy = idx / FU_TX, ox = idx - oy * FU_TX;
                    const int yy = y0 + oy, xx = x0 + ox;
                    if (yy < g.h && xx < g.w) {
                        const long long o = (long long)t * g.plane + (long long)yy * g.pitch + xx;
                        pv[o] = c[j][0];
                        pv[F.total + o] = c[j][1];
                        pv[2 * F.total + o] = c[j][2];
                    }
                }
            }
            __syncthreads();   // inb / yp are reused by the next unit
        }
        if (!grid_barrier(F.bar, G, nb, P.inject_timeout && blockIdx.x == 0 && k == 0)) goto timed_out;

        // every CTA reads the same settled scalars (the finalize of the step
        // before ran ahead of its CTA's arrival at this barrier); with one
        // video they are kept for phase 2 as well
        if (threadIdx.x == 0) {
            int all = 1;
            for (int v = 0; v < F.n_videos; ++v) all &= __ldcg(&P.state[v].done);
            s_all_done = all;
            if (F.n_videos == 1) {
                const VState* st = P.state;
                const double sc = __ldcg(&st->scale);
                s_skip = all;
                s_scale = (float)sc;
                s_sg = (float)(sc * __ldcg(&st->gain));
                s_shift = (float)__ldcg(&st->shift);
            }
        }
        __syncthreads();
        if (s_all_done) break;

        // ------------------------------- phase 2: t-pass, combine, reductions
        {
            const int ib = P.cta_begin[blockIdx.x], ie = P.cta_begin[blockIdx.x + 1];
            for (int it = ib; it < ie; ++it) {
                const WorkItem item = P.items[it];
                const int v = item.video;
                if (!dbg_ok(it < P.n_items && v >= 0 && v < F.n_videos, kDbgSlot, it, v)) continue;
                __syncthreads();   // s_* of the previous item are no longer read
                if (threadIdx.x == 0 && F.n_videos > 1) {
                    const VState* st = P.state + v;
                    s_skip = __ldcg(&st->done);
                    const double sc = __ldcg(&st->scale);
                    s_scale = (float)sc;
                    s_sg = (float)(sc * __ldcg(&st->gain));
                    s_shift = (float)__ldcg(&st->shift);
                }
                __syncthreads();
                if (s_skip) continue;   // the whole CTA skips (shared flag)
                const VideoGeom g = P.geo[v];
                const int rows = fused_rows2(g.w);
                const int nchunk = (g.h + rows - 1) / rows;
                if (!dbg_ok(0 <= item.t0 && item.t0 <= item.t1 && item.t1 <= g.nf * nchunk, kDbgUnit, it,
                            item.t1))
                    continue;
                const TS* Xv = X + g.off;
                const TS* SPv = (const TS*)P.sp + g.off;
                const TS* Fv = (const TS*)P.f + g.off;
                const float* pv = F.pvol + g.off;
                TS* Zv = Z + g.off;
                float* FO = final_step ? P.final_out[v] : nullptr;
                const float scale = s_scale, sg = s_sg, shift = s_shift;
                float part[kRed] = {0.f, 0.f, 0.f, 0.f};
                // the warp's running sums of its flushed partials (one per unit,
                // a few per item) in FP32: FP64 adds on lane 0 cost ~0.3 us per
                // step on this GPU's FP64 units; the block sum is FP64
                float acc[kRed] = {0.f, 0.f, 0.f, 0.f};
                for (int un = item.t0; un < item.t1; ++un) {
                    const int t = un / nchunk, r0 = (un - t * nchunk) * rows;
                    const int nr = min(rows, g.h - r0);
                    for (int idx = threadIdx.x; idx < nr * g.w; idx += blockDim.x) {
                        const int yy = r0 + idx / g.w, xx = idx - (idx / g.w) * g.w;
                        const long long o = (long long)t * g.plane + (long long)yy * g.pitch + xx;
                        const float s = to_f(SPv[o]);
                        const float fv = to_f(Fv[o]);
                        const float xh = scale * to_f(__ldcg(Xv + o));
                        // temporal taps in groups of TG frames whose loads are
                        // issued together (taps past 2 rt or outside the video
                        // are predicated off)
                        constexpr int TG = 5;
                        float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                        for (int d0 = 0; d0 <= 2 * rt; d0 += TG) {
                            float q0[TG], q1[TG], q2[TG];
#pragma unroll
                            for (int j = 0; j < TG; ++j) {
                                const int d = d0 + j, tp = t - rt + d;
                                q0[j] = q1[j] = q2[j] = 0.f;
                                if (d <= 2 * rt && tp >= 0 && tp < g.nf) {
                                    const long long q = o + (long long)(d - rt) * g.plane;
                                    q0[j] = __ldcg(pv + q);
                                    q1[j] = __ldcg(pv + F.total + q);
                                    q2[j] = __ldcg(pv + 2 * F.total + q);
                                }
                            }
#pragma unroll
                            for (int j = 0; j < TG; ++j)
                                if (d0 + j <= 2 * rt) {
                                    const float gw = P.gt[d0 + j];
                                    c0 = fmaf(gw, q0[j], c0);
                                    c1 = fmaf(gw, q1[j], c1);
                                    c2 = fmaf(gw, q2[j], c2);
                                }
                        }
                        const float af = alpha * fv;
                        const float inner = fmaf(-af, fv, 1.f) * c0 + 2.f * af * c1 - alpha * c2;
                        float z = sg * (s * inner);
                        if (FO) {
                            FO[((long long)t * g.h + yy) * g.w + xx] = z;
                        } else {
                            const TS zs = from_f<TS>(z);
                            Zv[o] = zs;
                            z = to_f(zs);
                        }
                        part[0] = fmaf(z, z, part[0]);
                        part[1] = fmaf(xh, z, part[1]);
                        part[2] = fmaf(xh, xh, part[2]);
                        const float dz = fmaf(-shift, xh, z);
                        part[3] = fmaf(dz, dz, part[3]);
                    }
                    warp_flush(part, acc);   // at most ~rows * w / 256 terms per thread and unit
                }
                // the run's FP64 sums go to its item slot (reduced after the barrier)
                double* sh = reinterpret_cast<double*>(sm);
                double run[kRed];
                for (int c = 0; c < kRed; ++c) run[c] = (double)acc[c];
                block_sum_lane0(run, sh);
                if (threadIdx.x == 0)
                    for (int c = 0; c < kRed; ++c) P.partials[(long long)it * kRed + c] = run[c];
            }
        }
        if (!grid_barrier(F.bar, G, nb, false)) goto timed_out;
        // finalize: CTA G - 1 - (v mod G) updates video v -- the last CTAs,
        // which have no phase-1 unit when the grid has a spare CTA per video,
        // so the update overlaps the other CTAs' next phase 1 (which needs no
        // scalars); the next phase 2 starts after the next barrier
        for (int v = (int)G - 1 - (int)blockIdx.x; v < F.n_videos; v += G)
            fused_finalize(P, v, reinterpret_cast<double*>(sm));
    }
    return;

timed_out:
    if (threadIdx.x == 0)
        for (int v = 0; v < F.n_videos; ++v) {
            atomicExch(&P.state[v].status, 6);   // SFSEG_ETIMEOUT
            P.state[v].done = 1;
        }
}

SFSEG_DEBUG_TU(fused)

size_t fused_smem_bytes(int ry, int rx) {
    const size_t TXH = FU_TX + 2 * rx, TYH = FU_TY + 2 * ry;
    size_t floats = 3 * (TYH * TXH + (size_t)FU_TY * TXH);
    const size_t red = (size_t)FU_THREADS * kRed * 2;   // finalize scratch (doubles as floats)
    if (floats < red) floats = red;
    return 4 * floats;
}

void fused_tile(int* tx, int* ty, int* threads) {
    *tx = FU_TX;
    *ty = FU_TY;
    *threads = FU_THREADS;
}

static const void* fused_fn(int storage) {
    switch (storage) {
        case 0: return (const void*)step_fused_kernel<float>;
        case 1: return (const void*)step_fused_kernel<__nv_bfloat16>;
        case 2: return (const void*)step_fused_kernel<__half>;
    }
    return nullptr;
}

// Opt in to the shared memory of the largest radii (a per-function attribute
// shared by every context, as for the any-radius kernel), and return how many
// CTAs of this kernel can be resident at once on the current device (the
// cooperative launch needs all of them resident).
cudaError_t setup_step_fused(int storage, int ry, int rx, int* max_ctas) {
    const void* fn = fused_fn(storage);
    if (!fn) return cudaErrorInvalidValue;
    const size_t cap = fused_smem_bytes(kMaxR, kMaxR);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, FU_THREADS, fused_smem_bytes(ry, rx));
    if (e != cudaSuccess) return e;
    *max_ctas = coop ? sms * per_sm : 0;
    return cudaSuccess;
}

cudaError_t launch_step_fused(int storage, const FusedParams& F, int n_ctas, cudaStream_t s) {
    const void* fn = fused_fn(storage);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<FusedParams*>(&F)};
    return cudaLaunchCooperativeKernel(fn, dim3(n_ctas), dim3(FU_THREADS), args,
                                       fused_smem_bytes(F.S.ry, F.S.rx), s);
}

}  // namespace sfseg
