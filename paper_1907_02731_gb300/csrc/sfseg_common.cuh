// sfseg_common.cuh -- types and device helpers shared by the SFSeg kernels.
//
// Internal layout in HBM (one packed allocation per array, all videos of a
// context back to back, each video 256-byte aligned):
//   sp, f, x_a, x_b : [nf][h][pitch] in the storage type, pitch = w rounded
//                     up to 8 elements (16-byte rows for FP32, BF16 and FP16),
//                     the pad columns are zero and never read as data.
// The iterate is stored unnormalised: x_hat = scale * x_stored (deferred
// normalisation, Eq. 8), and each step stores z = gain * M x_hat with a
// power-of-two gain that keeps the stored values near RMS 1 (FP16 range).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sfseg {

constexpr int kMaxR = 16;       // largest spatial radius
constexpr int kMaxRt = 8;       // largest temporal radius
constexpr int kRed = 4;         // reductions per step: z.z, xh.z, xh.xh, |z - s xh|^2
constexpr int kMaxDynSmem = 232448;   // dynamic shared memory per block (227 KB)
constexpr int kMaxChan = 4;           // pairwise feature channels (Eq. 9) of the step kernels
// TMA descriptors per video: sp, f channel 0, x_a, x_b, f channels 1 .. kMaxChan - 1
constexpr int kMapsPerVideo = 3 + kMaxChan;

// Per-step record of the forward pass for the adjoint (per video, nullable):
// scale[k] turns the stored iterate of step k into the unit-norm x^k (k = 0..K),
// gain[k] is the gain step k stored with, ny[k] = ||M x^k|| with unit-norm x^k.
struct Record {
    double* scale;
    double* gain;
    double* ny;
};

struct VideoGeom {
    int nf, h, w, pitch;        // pitch in elements
    long long plane;            // h * pitch
    long long off;              // element offset of this video in the packed arrays
    long long n;                // nf * h * w (voxels)
};

// Per-video device state, updated by the last CTA of each step (finalize).
struct VState {
    double scale;               // x_hat = scale * stored iterate
    double gain;                // the step stores z = gain * (M x_hat)
    double shift;               // gain * r_{k-1}: shift of the residual sum
    double tol;                 // early-stop tolerance on rho/r (0 = off)
    int iter;                   // completed steps
    int done;                   // 1: converged or failed, later steps skip
    int status;                 // sfseg_status of the device-side checks
    int final_iter;             // step count whose output went to the caller buffer
    double in_norm;             // ||x^k|| of the caller's scale: ||x0|| before step 0, then 1
};

// One CTA's share of a step: a (x0, y0) tile of one video over frames [t0, t1).
struct WorkItem {
    int video, x0, y0, t0, t1;
    int pad[3];
};

struct StepParams {
    const void* x_in;           // packed stored iterate (storage type)
    void* z_out;                // packed output (storage type), or null
    float* const* final_out;    // per-video contiguous FP32 output, or null
    const void* sp;
    const void* f;
    const VideoGeom* geo;
    VState* state;
    const WorkItem* items;
    const int* item_begin;      // [n_videos + 1]: video v's items are vseg[b[v] .. b[v+1])
    const int* vseg;            // item ids grouped by video (null: identity)
    double* partials;           // [n_items][kRed]
    unsigned* counters;         // [n_videos]
    double* trace;              // [n_videos][trace_cap][3]: r_k, rho_k, ||M x_hat||
    int trace_cap;
    int n_items;
    float alpha;
    int rt, ry, rx;
    float gt[2 * kMaxRt + 1];
    float gy[2 * kMaxR + 1];
    float gx[2 * kMaxR + 1];
    // specialised kernel only
    float2 gt2[2 * kMaxRt + 1];  // each tap twice, the paired operand of the packed FMAs
    float2 gy2[2 * kMaxR + 1];
    float2 gx2[2 * kMaxR + 1];  // (g, -2 g): the x-pass of the (a, b) pair yields (C0, -2 C1), exactly
    const void* maps;           // [n_videos][4] CUtensorMap: sp, f, x_a, x_b (global memory)
    int x_sel;                  // 0: the input iterate is x_a, 1: x_b
    const int* cta_begin;       // [n_ctas + 1]: segments of CTA c are [cta_begin[c], cta_begin[c+1])
    Record rec;                 // forward record (single video), or all null
    // Appended last: inserting them before the fields above shifts the tap
    // pairs the packed FMAs read from the constant bank and costs the
    // specialised step about 3% (measured).
    int nchan;                  // pairwise feature channels C (Eq. 9); f holds C volumes
    long long fstride;          // elements between consecutive channel volumes of f
    // specialised kernel, FP32 only: per-voxel terms the adjoint needs, pitched
    // like the iterate (null = not written): the bracket K = C0 - alpha (f^2 C0
    // - 2 f C1 + C2) with y = scale * gain * sp * K, and F = f C0 - C1
    float* aux_k;
    float* aux_f;
    // test aid (sfseg_debug_inject_timeout): the first x-pass warp of every CTA
    // waits once on a barrier nothing arrives on, so the step gives up
    int inject_timeout;
    // specialised kernel, several channels (Eq. 9) as one pass per channel:
    // the pass reads channel f_chan; acc_in (or null) holds the partial sum of
    // the earlier passes, added before the store; no_reduce skips the
    // reductions and the arrival (every pass but the last)
    int f_chan;
    const void* acc_in;
    int no_reduce;
    // one rank's slab of a video split along t: the step's FP64 sums (of the
    // slab's own frames) go to ext_sums[v * kRed ..] instead of updating the
    // video's scalars; the caller sums them over the ranks and applies them
    // with a separate finalize (null = normal finalize)
    double* ext_sums;
    // sizes the bounds checks of the debug build compare against
    int n_videos;
    long long total;            // packed elements per volume array
};

// ------------------------------------------------------ debug build checks
// Compiled with SFSEG_DEBUG (libsfseg_debug.so), kernels check segment and
// item ranges, TMA box coordinates and workspace offsets before using them.
// A failed check counts the violation, keeps the first one's code and two
// values in a device word of its translation unit, and the caller skips the
// access (no trap); sfseg_debug_status reads and clears the words.  In the
// normal build dbg_ok is the constant true and the checks compile away.
enum DebugCode {
    kDbgSegment = 1,    // a work item outside its video (frames, tile origin, video index)
    kDbgTma = 2,        // a TMA box coordinate misaligned or outside the volume's frames
    kDbgStore = 3,      // an offset outside the packed workspace or the caller's buffer
    kDbgSlot = 4,       // a partials / item slot outside its array
    kDbgUnit = 5        // a fused-kernel unit outside its plan
};
#ifdef SFSEG_DEBUG
static __device__ unsigned long long g_dbg[4];   // count, first code, first values (one per translation unit)
__device__ __forceinline__ bool dbg_ok(bool ok, int code, long long a, long long b) {
    if (!ok && atomicAdd(&g_dbg[0], 1ull) == 0ull) {
        g_dbg[1] = (unsigned long long)code;
        g_dbg[2] = (unsigned long long)a;
        g_dbg[3] = (unsigned long long)b;
    }
    return ok;
}
// host: copy this translation unit's words to out[4] and clear them
#define SFSEG_DEBUG_TU(name)                                                        \
    void sfseg_debug_take_##name(unsigned long long* out) {                         \
        cudaMemcpyFromSymbol(out, g_dbg, sizeof(g_dbg));                            \
        const unsigned long long z[4] = {0, 0, 0, 0};                               \
        cudaMemcpyToSymbol(g_dbg, z, sizeof(z));                                    \
    }
#else
__device__ __forceinline__ bool dbg_ok(bool ok, int, long long, long long) { return true; }
#define SFSEG_DEBUG_TU(name)                                                        \
    void sfseg_debug_take_##name(unsigned long long* out) {                         \
        for (int i = 0; i < 4; ++i) out[i] = 0;                                     \
    }
#endif

// ---------------------------------------------------------------- storage
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }

// ------------------------------------------------------------ traversal
// Visits every voxel of one video once: the grid's blocks take the rows
// r = t h + y in turn and their threads the columns, so the contiguous index
// (t h + y) w + x and the pitched offset t plane + y pitch + x (without
// g.off) cost one 32-bit division per row, not two 64-bit ones per voxel.
template <typename Fn>
__device__ __forceinline__ void for_each_voxel(const VideoGeom& g, Fn&& fn) {
    const int rows = g.nf * g.h;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const int t = r / g.h, y = r - t * g.h;
        const long long src = (long long)r * g.w;
        const long long dst = (long long)t * g.plane + (long long)y * g.pitch;
        for (int x = threadIdx.x; x < g.w; x += blockDim.x) fn(src + x, dst + x);
    }
}

__device__ __forceinline__ bool aligned8(const void* p) { return ((unsigned long long)p & 7ull) == 0; }

// Column pairs of one video (w even) U at a time per thread: pair k covers
// the contiguous index i = 2k and the pitched offset o of row r = k / (w/2)
// (one 32-bit division per pair).  The grid strides over the pairs and a
// thread takes k0, k0 + S, ..., k0 + (U-1) S (S = the grid's threads), so each
// u is a coalesced sweep and a kernel can issue its U loads before any store
// (U x 8 bytes in flight per thread and array: enough to cover the HBM
// latency with eight 256-thread blocks per SM).  fn(i, o, ok) gets the U
// offsets and which of them lie inside the video.
template <int U, typename Fn>
__device__ __forceinline__ void for_each_pair_batch(const VideoGeom& g, Fn&& fn) {
    const unsigned npairs = (unsigned)(g.n >> 1), hw = (unsigned)(g.w >> 1);
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < npairs; k0 += U * stride) {
        long long i[U], o[U];
        bool ok[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned k = k0 + (unsigned)u * stride;
            ok[u] = k < npairs && k >= k0;   // (k >= k0: no wrap-around)
            const unsigned r = k / hw;
            i[u] = 2ll * k;
            o[u] = (long long)r * g.pitch + 2ll * (k - r * hw);
        }
        fn(i, o, ok);
    }
}

// Whether for_each_pair_batch covers the video: even rows and a pair count
// that fits its 32-bit indices.
__device__ __forceinline__ bool pair_batch_ok(const VideoGeom& g) {
    return (g.w & 1) == 0 && (g.n >> 1) + 8ll * gridDim.x * blockDim.x < (1ll << 32);
}

// two adjacent values of a storage array (8 / 4 / 4 bytes, aligned)
template <typename T> __device__ __forceinline__ void store_pair(T* p, float a, float b);
template <> __device__ __forceinline__ void store_pair<float>(float* p, float a, float b) {
    *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
template <> __device__ __forceinline__ void store_pair<__nv_bfloat16>(__nv_bfloat16* p, float a, float b) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(a, b);
}
template <> __device__ __forceinline__ void store_pair<__half>(__half* p, float a, float b) {
    *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a, b);
}
template <typename T> __device__ __forceinline__ float2 load_pair(const T* p);
template <> __device__ __forceinline__ float2 load_pair<float>(const float* p) {
    return *reinterpret_cast<const float2*>(p);
}
template <> __device__ __forceinline__ float2 load_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}
template <> __device__ __forceinline__ float2 load_pair<__half>(const __half* p) {
    return __half22float2(*reinterpret_cast<const __half2*>(p));
}

// Order-preserving map of float bits onto unsigned integers: atomicMax /
// atomicMin on the keys are max / min on the floats (key 0 is below every
// float, 0xffffffff above).
__device__ __forceinline__ unsigned float_key(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// ------------------------------------------------------------ reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adds the warp's FP32 partials into lane 0's accumulators (FP64, or FP32
// where a caller keeps only a few dozen flushes per accumulator) and clears them.
template <typename A>
__device__ __forceinline__ void warp_flush(float (&p)[kRed], A (&acc)[kRed]) {
#pragma unroll
    for (int c = 0; c < kRed; ++c) {
        float s = warp_sum(p[c]);
        if ((threadIdx.x & 31) == 0) acc[c] += (A)s;
        p[c] = 0.f;
    }
}

// Fixed-order FP64 sum of n per-block partials (read through L2, written by
// other blocks of the grid before their arrival), by the whole block: each
// thread sums a strided subset, then halving folds in shared memory.  Every
// thread of the block calls it (blockDim.x <= 256) and gets the sum.
__device__ inline double block_sum_partials(const double* partials, int n) {
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += __ldcg(&partials[b]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int m = blockDim.x; m > 1;) {
        const int h = (m + 1) / 2;
        if ((int)threadIdx.x < m - h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
        m = h;
    }
    const double tot = red[0];
    __syncthreads();   // red may be reused
    return tot;
}

// Block-wide FP64 sum of lane-0 accumulators, result valid in thread 0.
// Fixed order (deterministic).  `sh` must hold kRed * (blockDim/32) doubles.
__device__ __forceinline__ void block_sum_lane0(double (&acc)[kRed], double* sh) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < kRed; ++c) sh[warp * kRed + c] = acc[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < kRed; ++c) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w * kRed + c];
            acc[c] = s;
        }
    }
    __syncthreads();
}

// Power-of-two helpers for the gain by the FP64 exponent bits (integer
// operations only: FP64 division, square roots and transcendental functions
// are slow on this GPU and sit on the critical path of every power step).
// 1 / v for v = 2^e in the normal range (exact).
__device__ __forceinline__ double pow2_recip(double v) {
    const long long ex = (__double_as_longlong(v) >> 52) & 0x7ff;
    return __longlong_as_double((2046ll - ex) << 52);
}
// e with |log2(v) - e| <= 1/2 for a finite v > 0: the binary exponent, one
// more when the mantissa exceeds sqrt(2).
__device__ __forceinline__ int pow2_exponent_near(double v) {
    const long long b = __double_as_longlong(v);
    int e = (int)((b >> 52) & 0x7ff) - 1023;
    if ((b & 0xfffffffffffffll) > 0x6a09e667f3bccll) e += 1;
    return e;
}
// 2^e, e clamped to the normal range
__device__ __forceinline__ double pow2(int e) {
    e = e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
    return __longlong_as_double((long long)(1023 + e) << 52);
}

// The step's scalar update (Eq. 3 Rayleigh quotient, residual, Eq. 8 norm),
// from the FP64 sums S = (z.z, xh.z, xh.xh, |z - shift xh|^2) of video v.
// Runs in one thread.  One FP64 division, one reciprocal square root and one
// square root; the gain (a power of two, so that the stored z has RMS ~ 1 in
// every storage type) is chosen from exponent bits.  The gain only rescales
// the stored iterate by an exact power of two, which the next scale undoes.
__device__ inline void finish_step(VState* st, double* trace_row, const double (&S)[kRed],
                                   long long n_vox, const Record* rec = nullptr) {
    const double zz = S[0], xz = S[1], xx = S[2], dd = S[3];
    const double gain = st->gain, sig = st->shift;
    if (!(isfinite(zz) && isfinite(xz) && isfinite(xx) && isfinite(dd))) {
        st->status = 5;   // SFSEG_ENONFINITE
        st->done = 1;
        return;
    }
    if (!(zz > 0.0) || !(xx > 0.0)) {
        st->status = 4;   // SFSEG_EZERONORM
        st->done = 1;
        return;
    }
    const double ig = pow2_recip(gain);
    const double rxx = 1.0 / xx;
    const double rsz = rsqrt(zz);                // 1 / ||z||
    const double ny = zz * rsz * ig;             // ||M x_hat||, x_hat of unit norm
    const double rz = xz * rxx;                  // Rayleigh quotient of z = gain * M x_hat
    const double r = rz * ig;
    // ||z - rz xh||^2 = ||z - sig xh||^2 - (rz - sig)^2 xh.xh  (exact identity)
    double e = dd - (rz - sig) * (rz - sig) * xx;
    if (e < 0.0) e = 0.0;
    const double rho = sqrt(e * rxx) * ig;
    if (trace_row) {
        trace_row[0] = r;
        trace_row[1] = rho;
        trace_row[2] = ny * st->in_norm;        // ||M x^k|| at the caller's scale of x^k
    }
    st->in_norm = 1.0;
    if (rec && rec->scale) {
        rec->gain[st->iter] = gain;
        rec->ny[st->iter] = ny;
        rec->scale[st->iter + 1] = rsz;
    }
    st->scale = rsz;
    // next gain ~ sqrt(n xh.xh) / ny; its square is n xx (rsz gain)^2
    const double q = rsz * gain;
    st->gain = pow2(pow2_exponent_near((double)n_vox * xx * q * q) >> 1);
    st->shift = st->gain * r;
    st->iter += 1;
    if (st->tol > 0.0 && rho < st->tol * fabs(r)) st->done = 1;
}

// After a CTA of video v stored the FP64 partials of n_arrive of the video's
// items (thread 0), the last CTA of that video to arrive reduces all of them
// (fixed order) and runs finish_step.  No CTA ever waits on another: the last
// one does the work.
__device__ inline void arrive_and_finalize(const StepParams& P, int v, double* sh,
                                           unsigned n_arrive = 1u) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned cnt = (unsigned)(P.item_begin[v + 1] - P.item_begin[v]);
        const unsigned prev = atomicAdd(&P.counters[v], n_arrive);
        s_last = (prev + n_arrive == cnt);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int b = P.item_begin[v], e = P.item_begin[v + 1];
    double acc[kRed] = {0.0, 0.0, 0.0, 0.0};
    for (int i = b + (int)threadIdx.x; i < e; i += blockDim.x)
        for (int c = 0; c < kRed; ++c) {
            const long long id = P.vseg ? P.vseg[i] : i;
            acc[c] += __ldcg(&P.partials[id * kRed + c]);
        }
    // tree over threads in shared memory (fixed order)
    double* red = sh;   // blockDim * kRed doubles
    for (int c = 0; c < kRed; ++c) red[c * blockDim.x + threadIdx.x] = acc[c];
    __syncthreads();
    // halving folds; an odd count keeps its middle element for the next fold,
    // so any block size works (for a power of two this is the plain tree)
    for (int n = blockDim.x; n > 1;) {
        const int h = (n + 1) / 2;
        if ((int)threadIdx.x < n - h)
            for (int c = 0; c < kRed; ++c)
                red[c * blockDim.x + threadIdx.x] += red[c * blockDim.x + threadIdx.x + h];
        __syncthreads();
        n = h;
    }
    if (threadIdx.x == 0 && P.ext_sums) {
        for (int c = 0; c < kRed; ++c) P.ext_sums[(long long)v * kRed + c] = red[c * blockDim.x];
        P.counters[v] = 0u;
    } else if (threadIdx.x == 0) {
        double S[kRed];
        for (int c = 0; c < kRed; ++c) S[c] = red[c * blockDim.x];
        VState* st = P.state + v;
        const int k = st->iter;
        double* row = (k < P.trace_cap) ? P.trace + ((long long)v * P.trace_cap + k) * 3 : nullptr;
        finish_step(st, row, S, P.geo[v].n, &P.rec);
        P.counters[v] = 0u;
    }
}

}  // namespace sfseg
