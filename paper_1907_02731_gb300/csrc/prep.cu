// prep.cu -- per-call set-up and finish kernels.
//
// prep_features: caller FP32 S and F (contiguous) -> internal pitched storage,
//   sp = S^p (the unary term of Eq. 1, computed with powf), once per video.
// prep_x:        caller FP32 x0 -> internal stored iterate, with the FP64
//   norm ||x0|| that sets the first scale (x_hat_0 = x0 / ||x0||).
// finish:        the unit-norm result x^K = scale * z into the caller's FP32
//   buffer (Eq. 8 applied to the last step's output).
#include "sfseg_launch.h"

namespace sfseg {

template <typename TS>
__global__ void __launch_bounds__(256) prep_features_kernel(const __grid_constant__ PrepFeatParams P) {
    const VideoGeom g = P.g;
    const long long n = g.n;
    TS* SPo = (TS*)P.sp_out + g.off;
    TS* Fo = (TS*)P.f_out + g.off;
    int bad = 0;
    float fmin[kMaxChan], fmax[kMaxChan];   // range of the stored f per channel
#pragma unroll
    for (int c = 0; c < kMaxChan; ++c) {
        fmin[c] = INFINITY;
        fmax[c] = -INFINITY;
    }
    auto track = [&](int c, float v) {
#pragma unroll
        for (int k = 0; k < kMaxChan; ++k)
            if (k == c) {
                fmin[k] = fminf(fmin[k], v);
                fmax[k] = fmaxf(fmax[k], v);
            }
    };
    auto one = [&](long long i, long long o) {
        const float s = P.s[i];
        const float sp = P.s_is_sp ? s : powf(s, P.p);
        bad |= !isfinite(s) | !isfinite(sp);
        SPo[o] = from_f<TS>(sp);
        for (int c = 0; c < P.nchan; ++c) {
            const float fv = P.f[c * n + i];
            bad |= !isfinite(fv);
            Fo[c * P.chan_stride + o] = from_f<TS>(fv);
            track(c, to_f(from_f<TS>(fv)));
        }
    };
    if (aligned8(P.s) && aligned8(P.f) && pair_batch_ok(g)) {
        constexpr int U = 4;
        for_each_pair_batch<U>(g, [&](const long long (&i)[U], const long long (&o)[U], const bool (&ok)[U]) {
            float2 s[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) s[u] = *reinterpret_cast<const float2*>(P.s + i[u]);
            // with S = F (one array) the F loads below hit the lines just read;
            // the channel loop is unrolled so that each channel's range lives
            // in registers
#pragma unroll
            for (int c = 0; c < kMaxChan; ++c) {
                if (c >= P.nchan) break;
                float2 fv[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (ok[u]) fv[u] = *reinterpret_cast<const float2*>(P.f + c * n + i[u]);
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (ok[u]) {
                        bad |= !isfinite(fv[u].x) | !isfinite(fv[u].y);
                        store_pair<TS>(Fo + c * P.chan_stride + o[u], fv[u].x, fv[u].y);
                        const float f0 = to_f(from_f<TS>(fv[u].x)), f1 = to_f(from_f<TS>(fv[u].y));
                        fmin[c] = fminf(fmin[c], fminf(f0, f1));
                        fmax[c] = fmaxf(fmax[c], fmaxf(f0, f1));
                    }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) {
                    const float sp0 = P.s_is_sp ? s[u].x : powf(s[u].x, P.p);
                    const float sp1 = P.s_is_sp ? s[u].y : powf(s[u].y, P.p);
                    bad |= !isfinite(s[u].x) | !isfinite(s[u].y) | !isfinite(sp0) | !isfinite(sp1);
                    store_pair<TS>(SPo + o[u], sp0, sp1);
                }
        });
    } else {
        for_each_voxel(g, one);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(P.bad, 1);
    // range of f per channel: warp, then block, then one atomic per block
    __shared__ float s_min[kMaxChan][8], s_max[kMaxChan][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < kMaxChan; ++c) {
        float lo = fmin[c], hi = fmax[c];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
        }
        if (lane == 0) {
            s_min[c][warp] = lo;
            s_max[c][warp] = hi;
        }
    }
    __syncthreads();
    if (threadIdx.x < P.nchan && P.fmin_key) {
        const int c = threadIdx.x;
        float lo = INFINITY, hi = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            lo = fminf(lo, s_min[c][w]);
            hi = fmaxf(hi, s_max[c][w]);
        }
        atomicMin(&P.fmin_key[c], float_key(lo));
        atomicMax(&P.fmax_key[c], float_key(hi));
    }
}

template <typename TS>
__global__ void __launch_bounds__(256) prep_x_kernel(const __grid_constant__ PrepXParams P) {
    const VideoGeom g = P.g;
    TS* Xo = (TS*)P.x_out + g.off;
    float part = 0.f;
    int bad = 0;
    if (P.ext_sum) {   // slab: store every frame, count only [norm_t0, norm_t1) in the norm
        const long long hw = (long long)g.h * g.w;
        for_each_voxel(g, [&](long long i, long long o) {
            const TS xs = from_f<TS>(P.x[i]);
            const float xv = to_f(xs);
            const long long t = i / hw;
            Xo[o] = xs;
            if (t >= P.norm_t0 && t < P.norm_t1) {
                bad |= !isfinite(xv);
                part = fmaf(xv, xv, part);
            }
        });
    } else if (aligned8(P.x) && pair_batch_ok(g)) {
        constexpr int U = 4;
        for_each_pair_batch<U>(g, [&](const long long (&i)[U], const long long (&o)[U], const bool (&ok)[U]) {
            float2 xv[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) xv[u] = *reinterpret_cast<const float2*>(P.x + i[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) {
                    const float x0 = to_f(from_f<TS>(xv[u].x)), x1 = to_f(from_f<TS>(xv[u].y));   // as stored
                    bad |= !isfinite(x0) | !isfinite(x1);
                    store_pair<TS>(Xo + o[u], xv[u].x, xv[u].y);
                    part = fmaf(x0, x0, part);
                    part = fmaf(x1, x1, part);
                }
        });
    } else {
        for_each_voxel(g, [&](long long i, long long o) {
            const TS xs = from_f<TS>(P.x[i]);
            const float xv = to_f(xs);
            bad |= !isfinite(xv);
            Xo[o] = xs;
            part = fmaf(xv, xv, part);
        });
    }
    bad = __syncthreads_or(bad);
    __shared__ double sh[32];
    __shared__ int s_last;
    const float w = warp_sum(part);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)w;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
        P.partials[blockIdx.x] = bad ? __longlong_as_double(0x7ff8000000000000LL) : s;
        __threadfence();
        const unsigned prev = atomicAdd(P.counter, 1u);
        s_last = (prev + 1u == gridDim.x);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const double xx = block_sum_partials(P.partials, (int)gridDim.x);
    if (threadIdx.x != 0) return;
    *P.counter = 0u;
    if (P.ext_sum) {
        *P.ext_sum = xx;   // NaN when a stored value was not finite
        return;
    }
    VState st;
    st.tol = P.tol;
    st.iter = 0;
    st.final_iter = -1;
    st.shift = 0.0;
    st.status = 0;
    st.done = 0;
    st.in_norm = (isfinite(xx) && xx > 0.0) ? sqrt(xx) : 1.0;
    const int bad_feat = P.bad_features ? *(volatile const int*)P.bad_features : 0;
    if (P.raw) {
        st.in_norm = 1.0;
        st.scale = 1.0;
        st.gain = 1.0;
        if (!isfinite(xx) || bad_feat) { st.status = 5; st.done = 1; }
    } else {
        st.gain = P.gain0;
        if (!isfinite(xx) || bad_feat) { st.status = 5; st.done = 1; st.scale = 0.0; }
        else if (!(xx > 0.0)) { st.status = 4; st.done = 1; st.scale = 0.0; }
        else st.scale = 1.0 / sqrt(xx);
    }
    if (P.rec_scale0) *P.rec_scale0 = st.scale;
    P.state[P.video] = st;
}

template <typename TS>
__global__ void __launch_bounds__(256) finish_kernel(const __grid_constant__ FinishParams P) {
    const VideoGeom g = P.g;
    const VState st = P.state[P.video];
    const long long n = g.n;
    const bool in_place = (st.status == 0 && st.iter == P.final_iter);
    const float sc = (float)st.scale;
    const TS* src = (const TS*)((st.iter & 1) ? P.buf1 : P.buf0) + g.off;
    if (in_place) {
        const bool vec = ((unsigned long long)P.out & 15ull) == 0;
        const long long n4 = vec ? n / 4 : 0;
        float4* o4 = reinterpret_cast<float4*>(P.out);
        const long long stride = (long long)gridDim.x * blockDim.x;
        constexpr int U = 4;   // U float4 loads in flight per thread before the stores
        for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n4; j += U * stride) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j + u * stride < n4) v[u] = o4[j + u * stride];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (j + u * stride < n4) {
                    v[u].x *= sc; v[u].y *= sc; v[u].z *= sc; v[u].w *= sc;
                    o4[j + u * stride] = v[u];
                }
        }
        for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride)
            P.out[i] = P.out[i] * sc;
    } else if (aligned8(P.out) && pair_batch_ok(g)) {
        constexpr int U = 4;
        for_each_pair_batch<U>(g, [&](const long long (&i)[U], const long long (&o)[U], const bool (&ok)[U]) {
            float2 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u]) v[u] = load_pair<TS>(src + o[u]);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (ok[u])
                    *reinterpret_cast<float2*>(P.out + i[u]) =
                        make_float2((float)(st.scale * (double)v[u].x), (float)(st.scale * (double)v[u].y));
        });
    } else {
        for_each_voxel(g, [&](long long i, long long o) { P.out[i] = (float)(st.scale * (double)to_f(src[o])); });
    }
}

__global__ void set_ptrs_kernel(float** dst, const __grid_constant__ PtrPack pk) {
    const int i = threadIdx.x;
    if (i < pk.n) dst[pk.base + i] = pk.p[i];
}

static int grid_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return (int)b;
}

int prep_x_blocks(long long n) { return grid_for(n); }

cudaError_t launch_prep_features(int storage, const PrepFeatParams& P, cudaStream_t s) {
    const int b = grid_for(P.g.n);
    switch (storage) {
        case 0: prep_features_kernel<float><<<b, 256, 0, s>>>(P); break;
        case 1: prep_features_kernel<__nv_bfloat16><<<b, 256, 0, s>>>(P); break;
        case 2: prep_features_kernel<__half><<<b, 256, 0, s>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaPeekAtLastError();
}

cudaError_t launch_prep_x(int storage, const PrepXParams& P, int blocks, cudaStream_t s) {
    switch (storage) {
        case 0: prep_x_kernel<float><<<blocks, 256, 0, s>>>(P); break;
        case 1: prep_x_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(P); break;
        case 2: prep_x_kernel<__half><<<blocks, 256, 0, s>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaPeekAtLastError();
}

cudaError_t launch_finish(int storage, const FinishParams& P, cudaStream_t s) {
    const int b = grid_for(P.g.n);
    switch (storage) {
        case 0: finish_kernel<float><<<b, 256, 0, s>>>(P); break;
        case 1: finish_kernel<__nv_bfloat16><<<b, 256, 0, s>>>(P); break;
        case 2: finish_kernel<__half><<<b, 256, 0, s>>>(P); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaPeekAtLastError();
}

// Slab scalars (one thread).  mode 0: the start of the iteration from the
// global sum of x0^2, as the tail of prep_x; mode 1: the step's global sums
// through the same finish_step as every other path.
__global__ void slab_state_kernel(VState* st, const double* sums, int mode, double gain0,
                                  long long n_video, double* trace, int trace_cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (mode == 0) {
        const double xx = sums[0];
        VState v;
        v.tol = 0.0;
        v.iter = 0;
        v.final_iter = -1;
        v.shift = 0.0;
        v.status = 0;
        v.done = 0;
        v.gain = gain0;
        v.in_norm = (isfinite(xx) && xx > 0.0) ? sqrt(xx) : 1.0;
        if (!isfinite(xx)) { v.status = 5; v.done = 1; v.scale = 0.0; }
        else if (!(xx > 0.0)) { v.status = 4; v.done = 1; v.scale = 0.0; }
        else v.scale = 1.0 / sqrt(xx);
        *st = v;
        return;
    }
    if (st->done) return;
    double S[kRed];
    for (int c = 0; c < kRed; ++c) S[c] = sums[c];
    const int k = st->iter;
    finish_step(st, k < trace_cap ? trace + 3ll * k : nullptr, S, n_video, nullptr);
}

cudaError_t launch_slab_state(VState* st, const double* sums, int mode, double gain0, long long n_video,
                              double* trace, int trace_cap, cudaStream_t s) {
    slab_state_kernel<<<1, 32, 0, s>>>(st, sums, mode, gain0, n_video, trace, trace_cap);
    return cudaPeekAtLastError();
}

cudaError_t launch_set_ptrs(float** dst, float* const* src, int n, cudaStream_t s) {
    for (int base = 0; base < n; base += PtrPack::kMax) {
        PtrPack pk;
        pk.base = base;
        pk.n = (n - base < PtrPack::kMax) ? n - base : PtrPack::kMax;
        for (int i = 0; i < pk.n; ++i) pk.p[i] = src[base + i];
        set_ptrs_kernel<<<1, PtrPack::kMax, 0, s>>>(dst, pk);
        cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace sfseg
