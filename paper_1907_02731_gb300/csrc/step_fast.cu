// step_fast.cu -- the power step y = M x_hat (Eq. 7 x alpha) for the common
// radii, specialised at compile time.
//
// Work decomposition.  A video is cut into 112 x 12 (x, y) tiles; one unit is
// one output frame of one tile.  Persistent CTAs (one of 512 threads per SM)
// first stream one whole tile each, all in step (frame t of neighbouring
// tiles is loaded at about the same time, so the halo rows one CTA loads are
// still in L2 for the next); the remaining tiles' units are then split into
// equal contiguous ranges.  A range is a list of segments (tile, frames
// [ta, tb)); a segment that starts or ends inside a video recomputes the
// 2 RT boundary frames' spatial passes.
//
// Per segment the CTA streams frames, with two warp roles that overlap:
//   load    one thread issues three TMA 3D box loads (x, sp, f) of the tile
//           plus its halo (128 x (12 + 2 RY)) into a ring of RT + NYB + LA
//           shared-memory stages (zero fill outside the volume = the zero
//           padding of Eq. 7's convolutions), LA frames ahead (1 for FP32
//           storage, 2 for 2-byte storage), completion on
//           an mbarrier per stage;
//   y-pass  warps 0..3 ("A"): a task is a column pair x 6 output rows;
//           a0 = sp x, a1 = f a0, a2 = f a1 and the vertical taps in
//           registers, every channel packed over the column pair (FMUL2 /
//           FFMA2); (a0, a1) are stored interleaved per column in a swizzled
//           plane, a2 in its own plane, in NYB buffers (2 for FP32
//           storage, 4 for 2-byte storage); FULL mbarrier;
//   x-pass  warps 4..15 ("B"): warp w owns output row w - 4, lanes 0..27 four
//           output columns each, windows read straight from shared memory;
//           (a0, a1) filtered with packed FMAs (a1's taps carry the factor
//           -2 of the combine, exact in binary), a2 with scalar ones;
//   t-pass  each thread keeps 2 RT + 1 partial sums per voxel and channel in
//           registers; the frame loop is unrolled over the ring phase so the
//           slot roles are fixed registers;
//   combine y = sp [(1 - a f^2) C0 + 2 a f C1 - a C2] for frame t - RT, with
//           the deferred scale and gain; 16-byte stores; FP32 partial sums of
//           z.z, x.z, x.x, |z - s x|^2 per thread over at most 16 frames
//           (packed over voxel pairs with FP32 storage), flushed into a
//           running sum per warp (FP32 with FP32 storage, else FP64); EMPTY
//           mbarrier back to the y-pass warps.
// With 2-byte storage the y-pass takes sp x as a mixed-precision FMA of the
// 2-byte operands (exact in FP32).
// Consecutive segments of one video on a CTA form a run with one FP64 block
// reduction and one arrival; the last CTA of each video to arrive reduces the
// partials and updates the video's scalars (no CTA waits on another).
// Variants (template flags): AUX also stores the per-voxel terms the adjoint
// needs; MC runs several pairwise channels (Eq. 9) as one pass per channel,
// each adding to the partial sum in the output buffer.  Every device wait is
// limited in time and gives up when another warp of the CTA has; a CTA that
// gives up drains its loads, records SFSEG_ETIMEOUT and leaves.
#include <cuda.h>

#include <type_traits>

#include "sfseg_common.cuh"
#include "sfseg_launch.h"

namespace sfseg {
namespace fast {

constexpr int TX = 112, TY = 12, XPAD = 8, BOXW = TX + 2 * XPAD, YBW = BOXW;
constexpr int NA_WARPS = 4;                   // warps running the loads and the y-pass
constexpr int NT = 32 * (NA_WARPS + TY);      // plus one x-pass/combine warp per tile row
constexpr unsigned long long kWaitNs = 1000000000ull;   // a device-side wait gives up after 1 s

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of `parity` to complete, for at most kWaitNs; with an
// abort flag, also give up as soon as another warp of the CTA has raised it.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, const volatile int* abort = nullptr) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort && *abort) return false;
        if ((i & 63u) == 63u && global_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, unsigned bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <typename TS> struct Vec4;
template <> struct Vec4<float> {
    __device__ static void load(const float* p, float (&v)[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ static void store(float* p, const float (&v)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4<__nv_bfloat16> {
    __device__ static void load(const __nv_bfloat16* p, float (&v)[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
    }
    __device__ static void store(__nv_bfloat16* p, const float (&v)[4]) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<unsigned*>(&a);
        q.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};
template <> struct Vec4<__half> {
    __device__ static void load(const __half* p, float (&v)[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const float2 fa = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        const float2 fb = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        v[0] = fa.x; v[1] = fa.y; v[2] = fb.x; v[3] = fb.y;
    }
    __device__ static void store(__half* p, const float (&v)[4]) {
        __half2 a = __floats2half2_rn(v[0], v[1]);
        __half2 b = __floats2half2_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<unsigned*>(&a);
        q.y = *reinterpret_cast<unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};

template <typename TS> struct Ld2;
// b0 = sp * x for a column pair of the y-pass.  The product of two BF16 or
// FP16 values is exact in FP32, so the mixed-precision FMA (2-byte operands,
// FP32 addend and result; the addend -0 keeps the product's sign of zero)
// gives the same value as converting both operands and multiplying in FP32,
// without the four conversions (measured: 207.6 -> 201.0 us per step for
// BF16 storage at 854x480x72, bit-identical iterates).
template <typename TS> struct Prod2;
template <> struct Prod2<float> {
    __device__ static float2 get(const float* sp, const float* x) {
        return __fmul2_rn(*reinterpret_cast<const float2*>(sp), *reinterpret_cast<const float2*>(x));
    }
};
template <> struct Prod2<__nv_bfloat16> {
    __device__ static float2 get(const __nv_bfloat16* sp, const __nv_bfloat16* x) {
        const unsigned us = *reinterpret_cast<const unsigned*>(sp), ux = *reinterpret_cast<const unsigned*>(x);
        float lo, hi;
        asm("{\n .reg .b16 s0, s1, x0, x1;\n mov.b32 {s0, s1}, %2;\n mov.b32 {x0, x1}, %3;\n"
            " fma.rn.f32.bf16 %0, s0, x0, %4;\n fma.rn.f32.bf16 %1, s1, x1, %4;\n}"
            : "=f"(lo), "=f"(hi) : "r"(us), "r"(ux), "f"(-0.0f));
        return make_float2(lo, hi);
    }
};
template <> struct Prod2<__half> {
    __device__ static float2 get(const __half* sp, const __half* x) {
        const unsigned us = *reinterpret_cast<const unsigned*>(sp), ux = *reinterpret_cast<const unsigned*>(x);
        float lo, hi;
        asm("{\n .reg .b16 s0, s1, x0, x1;\n mov.b32 {s0, s1}, %2;\n mov.b32 {x0, x1}, %3;\n"
            " fma.rn.f32.f16 %0, s0, x0, %4;\n fma.rn.f32.f16 %1, s1, x1, %4;\n}"
            : "=f"(lo), "=f"(hi) : "r"(us), "r"(ux), "f"(-0.0f));
        return make_float2(lo, hi);
    }
};
template <> struct Ld2<float> {
    __device__ static float2 get(const float* p) { return *reinterpret_cast<const float2*>(p); }
};
template <> struct Ld2<__nv_bfloat16> {
    __device__ static float2 get(const __nv_bfloat16* p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
};
template <> struct Ld2<__half> {
    __device__ static float2 get(const __half* p) {
        return __half22float2(*reinterpret_cast<const __half2*>(p));
    }
};

template <int RT, int RY, int RX, typename TS>
struct Cfg {
    static constexpr int RXE = (RX + 1) & ~1;                 // x halo rounded to a column pair
    static constexpr int NPAIR = (TX + 2 * RXE) / 2;          // y-pass column pairs
    static constexpr int NGRP = NA_WARPS * 32 / NPAIR;        // row groups of the y-pass
    static constexpr int NTA = NGRP * NPAIR;                  // y-pass tasks: pair x TROWS rows
    static constexpr int TROWS = TY / NGRP;                   // output rows per y-pass task
    static constexpr int SC0 = XPAD - RXE;                    // first y-pass stage column
    static constexpr int ROWS = TY + 2 * RY;                  // input rows per tile
    static constexpr int IN_ROWS = TROWS + 2 * RY;            // input rows per task
    static constexpr int NR = 2 * RT + 1;                     // temporal taps
    // y-pass output buffers: the x-pass warps may trail the y-pass by NYB - 1
    // frames (with 2-byte storage the stages are small enough for four)
    static constexpr int NYB = sizeof(TS) == 4 ? 2 : 4;
    // frames of TMA lookahead: the 2-byte stages leave room for two (measured
    // at 854x480x72, BF16: 201.0 -> 193.9 us per step; FP32 gains nothing
    // from a second frame and has no room for it)
    static constexpr int LA = sizeof(TS) == 4 ? 1 : 2;
    static constexpr int NS = RT + NYB + LA;                  // stages (see the stage-reuse note)
    static constexpr int BOX_BYTES = ROWS * BOXW * (int)sizeof(TS);
    static constexpr int ARR = (BOX_BYTES + 127) / 128 * 128; // one array of a stage
    static constexpr int STAGE = 3 * ARR;
    static constexpr int YBC = TY * YBW * 4;                  // one channel of one Yb buffer
    static constexpr int YB = 3 * YBC;                        // one Yb buffer (3 channels)
    static constexpr int NBAR = NS + 2 * NYB;                 // stages, FULL[NYB], EMPTY[NYB]
    static constexpr int SMEM = NS * STAGE + NYB * YB + NBAR * 8 + 128;
    static_assert(NTA <= NA_WARPS * 32 && TY % NGRP == 0, "y-pass tasks must tile the rows");
    static_assert(RX <= XPAD && SC0 >= 0, "x radius exceeds the halo pad");
    static_assert(NS * STAGE >= NT * kRed * 8, "finalize scratch must fit in the stages");
        static_assert(SMEM <= 232448, "shared memory per block");
};

constexpr int NB_WARPS = NT / 32 - NA_WARPS;   // x-pass / temporal / combine warps

// Packed (f32x2) and scalar multiply-add under one name, so that the temporal
// ring code serves the paired (a, b) channels and the single c channel.
__device__ __forceinline__ float2 pmul(float2 a, float2 g) { return __fmul2_rn(a, g); }
__device__ __forceinline__ float2 pfma(float2 a, float2 g, float2 c) { return __ffma2_rn(a, g, c); }
__device__ __forceinline__ float pmul(float a, float g) { return a * g; }
__device__ __forceinline__ float pfma(float a, float g, float c) { return fmaf(a, g, c); }

// Temporal taps of one channel (or channel pair) for ring phase U: frame tin
// feeds outputs tin - RT + k with weight g_t(RT - k) (constant-bank operand);
// slot (U - RT + k) mod NR holds output tin - RT + k.  Returns the finished
// output (slot of k = 0) in c.
template <int U, int RT, typename V>
__device__ __forceinline__ void tpass(V (&ring)[2 * RT + 1][4], const V (&p)[4], const V* gt,
                                      V (&c)[4]) {
    constexpr int NR = 2 * RT + 1;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int slot = ((U - RT + k) % NR + NR) % NR;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (k == NR - 1) ring[slot][i] = pmul(p[i], gt[k]);
            else ring[slot][i] = pfma(p[i], gt[k], ring[slot][i]);
        }
    }
    constexpr int slot0 = ((U - RT) % NR + NR) % NR;
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = ring[slot0][i];
}

// The (a, b) plane of a Yb row is 64 chunks of 16 bytes (two columns each);
// chunk k is stored at k ^ ((k >> 3) & 1), so that the x-pass windows (lane
// stride two chunks) fall in eight distinct bank groups per 8-lane phase.
__device__ __forceinline__ int ab_chunk(int k) { return k ^ ((k >> 3) & 1); }

// x-pass of one Yb row.  Channels a and b are interleaved in Yb ((a, b) per
// column, 8 bytes), so one packed FMA filters both; channel c has its own
// plane.  Lane l's outputs are Yb columns XPAD + 4l .. +3; the input windows
// are read straight from shared memory with aligned 16-byte loads; the taps
// are constant-bank operands (paired for the packed FMAs).
template <int RX>
__device__ __forceinline__ void xpass_abc(const float* row_ab, const float* row_c, int lane,
                                          const float2* gx2, const float* gx, float2 (&pab)[4],
                                          float (&pc)[4]) {
    {
        constexpr int W0 = (XPAD - RX) & ~1;                 // first window column (even)
        constexpr int SH = XPAD - RX - W0;                   // offset of column -RX in the window
        constexpr int NQ = (SH + 4 + 2 * RX + 1) / 2;        // 16-byte loads (2 columns each)
        static_assert(4 * 27 + W0 + 2 * NQ <= YBW && YBW % 16 == 0,
                      "(a, b) window of the last output lane exceeds the row");
        float2 w[2 * NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(row_ab + 4 * ab_chunk(2 * lane + W0 / 2 + q));
            w[2 * q] = make_float2(v.x, v.y);
            w[2 * q + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 a = __fmul2_rn(w[SH + i], gx2[0]);
#pragma unroll
            for (int d = 1; d <= 2 * RX; ++d) a = __ffma2_rn(w[SH + i + d], gx2[d], a);
            pab[i] = a;
        }
    }
    {
        constexpr int W0 = (XPAD - RX) & ~3;                 // first window column (multiple of 4)
        constexpr int SH = XPAD - RX - W0;
        constexpr int NQ = (SH + 4 + 2 * RX + 3) / 4;        // 16-byte loads (4 columns each)
        static_assert(4 * 27 + W0 + 4 * NQ <= YBW, "c window of the last output lane exceeds the row");
        float w[4 * NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(row_c + 4 * lane + W0 + 4 * q);
            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float a = w[SH + i] * gx[0];
#pragma unroll
            for (int d = 1; d <= 2 * RX; ++d) a = fmaf(w[SH + i + d], gx[d], a);
            pc[i] = a;
        }
    }
}

// Warp roles.  Warps 0..3 ("A"): the elected thread issues the TMA loads LA
// frames ahead; all of them run the y-pass of frame p into Yb[vc % NYB] (vc
// counts the valid frames of the segment), then each A warp arrives once on
// the FULL mbarrier of that buffer.  Warps 4.. ("B", one output row each):
// each waits on FULL on its own (the B warps are not coupled to each other),
// x-pass and temporal ring of the three channels, combine of frame p - RT
// (its x, sp, f from the frame's stage), store, then arrives once on EMPTY.
// A waits until all B warps have arrived on EMPTY of a buffer before refilling
// it, so A runs at most NYB frames ahead of B's completed work.
// Stage reuse: with NS = RT + NYB + LA stages and loads LA frames ahead, the
// load of frame p + LA (issued at frame p, after A's EMPTY wait) overwrites
// frame p - RT - NYB, whose last reader (B's combine of that frame, at B's
// frame p - NYB) arrived on EMPTY before A passed that wait.
template <int RT, int RY, int RX, typename TS, bool AUX, bool MC>
__global__ void __launch_bounds__(NT, 1) step_fast_kernel(const __grid_constant__ StepParams P) {
    using C = Cfg<RT, RY, RX, TS>;
    constexpr int NR = C::NR, NS = C::NS;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stages = smem;
    float* yb = reinterpret_cast<float*>(smem + NS * C::STAGE);        // [2][3][TY][YBW]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + NS * C::STAGE + C::NYB * C::YB);
    __shared__ float s_scale, s_gain, s_shift;
    __shared__ int s_skip, s_abort;
    __shared__ __align__(8) unsigned long long s_never;   // an mbarrier nothing arrives on (fault injection)

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool is_a = warp < NA_WARPS;
    const int brow = warp - NA_WARPS;            // B: output row of the tile
    const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P.maps);

    unsigned long long* full = bars + NS;       // [2], NA_WARPS arrivals per phase
    unsigned long long* empty = bars + NS + C::NYB;  // [NYB], NB_WARPS arrivals per phase
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
        for (int b = 0; b < C::NYB; ++b) {
            mbar_init(smem_u32(&full[b]), NA_WARPS);
            mbar_init(smem_u32(&empty[b]), NB_WARPS);
        }
        mbar_init(smem_u32(&s_never), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    // a wait that gave up: the step fails with SFSEG_ETIMEOUT and every other
    // wait of the CTA gives up at once (the loads in flight are still drained)
    auto give_up = [&](int v) {
        s_abort = 1;
        atomicExch(&P.state[v].status, 6);
        P.state[v].done = 1;
    };
    __syncthreads();
    // bit b: parity of the first FULL / EMPTY completion of buffer b in the
    // current segment; use n of buffer b completes phase base ^ (n & 1)
    unsigned fullbase = 0, emptybase = 0;
    // bit s: parity of the first completion of stage s in the current segment.
    // Inside a segment the valid frames p_first, p_first + 1, ... use stage
    // p % NS in turn, so frame p completes phase segphase[s] ^ ((p - p_first) / NS).
    unsigned segphase = 0;
    unsigned owed = 0, owed_par = 0;   // (thread 0) loads issued and not yet waited for

    // Consecutive segments of one video form a run: the video's scalars are
    // read once per run (they cannot change before every segment of the video
    // has arrived), the sums accumulate over the run, and the run arrives
    // once, counting all its segments.  Each x-pass warp adds its flushed FP32
    // partials (one per 16 frames, a few dozen per run) into a running sum:
    // FP32 with FP32 storage -- FP64 adds sit on the warp's critical chain and
    // FP64 is slow on this GPU (measured at 854x480x72: 194.7 -> 188.2 us per
    // step, iterates within 1e-7) -- and FP64 with 2-byte storage and in the
    // variant that stores the adjoint terms, where the FP32 form measured
    // slower; the block and everything above sum in FP64.
    const int seg_b = P.cta_begin[blockIdx.x], seg_e = P.cta_begin[blockIdx.x + 1];
    using WAcc = typename std::conditional<std::is_same<TS, float>::value && !AUX, float, double>::type;
    WAcc acc[kRed] = {0, 0, 0, 0};
    int run_v = -1, run_first = seg_b;
    for (int sg = seg_b; sg < seg_e; ++sg) {
        const WorkItem it = P.items[sg];
        const int v = it.video;
        if (!dbg_ok(sg < P.n_items && v >= 0 && v < P.n_videos, kDbgSlot, sg, v)) continue;
        if (v != run_v) {
            __syncthreads();   // every thread has read the previous run's scalars
            if (tid == 0) {
                const VState* st = P.state + v;
                s_skip = st->done;
                s_scale = (float)st->scale;
                s_gain = (float)st->gain;
                s_shift = (float)(st->shift * st->scale);
            }
            __syncthreads();
            run_v = v;
            run_first = sg;
        }
        if (s_skip) continue;
        const VideoGeom g = P.geo[v];
        const int ta = it.t0, tb = it.t1, x0 = it.x0, y0 = it.y0;
        // (uniform over the CTA: every thread skips the same segment)
        if (!dbg_ok(0 <= ta && ta < tb && tb <= g.nf && 0 <= x0 && x0 < g.w && 0 <= y0 && y0 < g.h,
                    kDbgSegment, sg, ((long long)ta << 32) | (unsigned)tb))
            continue;
        if (!dbg_ok(((x0 - XPAD) * (int)sizeof(TS)) % 16 == 0 && g.off + (long long)g.nf * g.plane <= P.total,
                    kDbgTma, x0, g.off))
            continue;
        const int t_end = tb + RT;
        const int p_first = max(ta - RT, 0), p_last = min(t_end, g.nf);   // valid frames [p_first, p_last)
        const int n_valid = p_last - p_first;
        auto parity = [&](int p) -> unsigned {
            return ((segphase >> (p % NS)) ^ (unsigned)((p - p_first) / NS)) & 1u;
        };

        if (is_a) {
            // ============================ A: loads + y-pass ====================
            const CUtensorMap* map_sp = maps + kMapsPerVideo * v + 0;
            const CUtensorMap* map_f = maps + kMapsPerVideo * v + ((!MC || P.f_chan == 0) ? 1 : 3 + P.f_chan);
            const CUtensorMap* map_x = maps + kMapsPerVideo * v + 2 + P.x_sel;
            auto issue = [&](int p) {
                const int s = p % NS;
                const unsigned bar = smem_u32(&bars[s]);
                unsigned char* st = stages + s * C::STAGE;
                mbar_expect_tx(bar, 3u * C::BOX_BYTES);
                tma_load_3d(smem_u32(st), map_x, bar, x0 - XPAD, y0 - RY, p);
                tma_load_3d(smem_u32(st + C::ARR), map_sp, bar, x0 - XPAD, y0 - RY, p);
                tma_load_3d(smem_u32(st + 2 * C::ARR), map_f, bar, x0 - XPAD, y0 - RY, p);
                owed |= 1u << s;
                owed_par = (owed_par & ~(1u << s)) | (parity(p) << s);
            };
            const int a_h = tid / C::NPAIR, a_p = tid - a_h * C::NPAIR;
            const int a_sc = C::SC0 + 2 * a_p;
            const bool a_task = tid < C::NTA;
            const float2* gy2 = P.gy2;
            if (tid == 0)
                for (int q = 0; q < C::LA && q < n_valid; ++q) issue(p_first + q);
            for (int vc = 0; vc < n_valid; ++vc) {
                const int p = p_first + vc;
                const int b = (int)((unsigned)vc % C::NYB);
                const unsigned n = (unsigned)vc / C::NYB;
                if (n >= 1 && !mbar_wait(smem_u32(&empty[b]), ((emptybase >> b) ^ (n - 1)) & 1u, &s_abort))
                    give_up(v);
                if (tid == 0 && !s_abort && vc + C::LA < n_valid) issue(p + C::LA);
                const int s = p % NS;
                if (mbar_wait(smem_u32(&bars[s]), parity(p), &s_abort)) owed &= ~(1u << s);
                else give_up(v);   // the load stays owed: drained before the CTA leaves
                if (a_task) {
                    const unsigned char* st = stages + s * C::STAGE;
                    const int r0 = a_h * C::TROWS;
                    const TS* sx = reinterpret_cast<const TS*>(st) + r0 * BOXW + a_sc;
                    const TS* ssp = reinterpret_cast<const TS*>(st + C::ARR) + r0 * BOXW + a_sc;
                    const TS* sf = reinterpret_cast<const TS*>(st + 2 * C::ARR) + r0 * BOXW + a_sc;
                    float2 q0[C::TROWS], q1[C::TROWS], q2[C::TROWS];
#pragma unroll
                    for (int i = 0; i < C::IN_ROWS; ++i) {
                        const float2 fv = Ld2<TS>::get(sf + i * BOXW);
                        const float2 b0 = Prod2<TS>::get(ssp + i * BOXW, sx + i * BOXW);
                        const float2 b1 = __fmul2_rn(fv, b0);
                        const float2 b2 = __fmul2_rn(fv, b1);
#pragma unroll
                        for (int o = 0; o < C::TROWS; ++o) {
                            const int d = i - o;
                            if (d == 0) {              // first tap of output row o
                                q0[o] = __fmul2_rn(b0, gy2[0]);
                                q1[o] = __fmul2_rn(b1, gy2[0]);
                                q2[o] = __fmul2_rn(b2, gy2[0]);
                            } else if (d > 0 && d <= 2 * RY) {
                                q0[o] = __ffma2_rn(b0, gy2[d], q0[o]);
                                q1[o] = __ffma2_rn(b1, gy2[d], q1[o]);
                                q2[o] = __ffma2_rn(b2, gy2[d], q2[o]);
                            }
                        }
                    }
                    // Yb buffer: (a, b) interleaved plane [TY][YBW][2] (chunks swizzled), then the c plane [TY][YBW]
                    float* yc = yb + b * 3 * TY * YBW;
#pragma unroll
                    for (int o = 0; o < C::TROWS; ++o) {
                        const int r = (r0 + o) * YBW;
                        *reinterpret_cast<float4*>(yc + 2 * r + 4 * ab_chunk(a_sc / 2)) =
                            make_float4(q0[o].x, q1[o].x, q0[o].y, q1[o].y);
                        *reinterpret_cast<float2*>(yc + 2 * TY * YBW + r + a_sc) = q2[o];
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&full[b]));
            }
        } else {
            // ================= B: x-pass, temporal ring, combine ==============
            const float sg_s = s_scale * s_gain;     // deferred scale and gain
            const float alpha = P.alpha, shift = s_shift;
            const bool out_lane = lane < 28;
            TS* Z = P.z_out ? (TS*)P.z_out + g.off : nullptr;
            float* FO = P.final_out ? P.final_out[v] : nullptr;
            const int yy = y0 + brow;
            const int xg = x0 + 4 * lane;
            const bool st_ok = out_lane && yy < g.h;
            bool st_ok_dbg = true;   // the debug build's store check (always true otherwise)

            float2 rab[NR][4];   // temporal ring of the (a, b) pair
            float rc[NR][4];     // temporal ring of c
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    rab[k][i] = make_float2(0.f, 0.f);
                    rc[k][i] = 0.f;
                }
            float part[kRed] = {0.f, 0.f, 0.f, 0.f};
            // FP32 storage, 11x11x5: the four per-voxel sums run as packed FMAs
            // over voxel pairs (x: voxels 0, 2; y: 1, 3), folded at each flush
            // (measured 188.3 -> 186.4 us per step at 854x480x72); with 2-byte
            // storage, at 9x9x5 (the 24-video batch: 114.3 -> 116.9 ms) and in
            // the adjoint-term variant the scalar form measured faster or
            // spilled less
            constexpr bool kPairSums = std::is_same<TS, float>::value && !AUX && RX == 5;
            float2 pp[kRed];
#pragma unroll
            for (int c = 0; c < kRed; ++c) pp[c] = make_float2(0.f, 0.f);
            const float2 nshift2 = make_float2(-s_shift, -s_shift);
            auto fold_pairs = [&]() {
                if (kPairSums)
#pragma unroll
                    for (int c = 0; c < kRed; ++c) {
                        part[c] = pp[c].x + pp[c].y;
                        pp[c] = make_float2(0.f, 0.f);
                    }
            };
            int flush = 0;
            int vc = 0;
            int tin = ta - RT;
            int so_next = ta % NS;                                   // stage of the next output frame
            TS* zp = Z ? Z + (long long)ta * g.plane + (long long)yy * g.pitch + xg : nullptr;
            // One input frame tin; U = (tin - (ta - RT)) mod NR is the ring phase,
            // a compile-time constant, so the ring slots are fixed registers.
            auto frame = [&](auto phase) {
                constexpr int U = decltype(phase)::value;
                const bool valid = (tin >= 0 && tin < g.nf);
                const int b = (int)((unsigned)vc % C::NYB);
                float2 pab[4];
                float pc[4];
                if (valid) {
                    if (P.inject_timeout && brow == 0 && vc == 0 &&
                        !mbar_wait(smem_u32(&s_never), 0u, &s_abort))
                        give_up(v);
                    if (!mbar_wait(smem_u32(&full[b]), ((fullbase >> b) ^ ((unsigned)vc / C::NYB)) & 1u, &s_abort))
                        give_up(v);
                    const float* yc = yb + b * 3 * TY * YBW;
                    // lanes 28..31 have no outputs: give them lane 27's window so
                    // every read stays inside the row
                    xpass_abc<RX>(yc + 2 * brow * YBW, yc + (2 * TY + brow) * YBW, out_lane ? lane : 27,
                                  P.gx2, P.gx, pab, pc);
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        pab[i] = make_float2(0.f, 0.f);
                        pc[i] = 0.f;
                    }
                }
                float2 cab[4];
                float c2[4];
                tpass<U, RT>(rab, pab, P.gt2, cab);
                tpass<U, RT>(rc, pc, P.gt, c2);
                const int o = tin - RT;
                if (o >= ta && o < tb) {
                    // The load of frame o completed before A's y-pass of o (A waited
                    // on the stage's mbarrier), and A's FULL arrival for o happened
                    // after that wait; this warp has since observed FULL of o and of
                    // the RT frames after it, so the load's bytes are visible here.
                    const int so = so_next;
                    so_next = (so_next + 1 == NS) ? 0 : so_next + 1;
                    const unsigned char* st = stages + so * C::STAGE;
                    const int off = (brow + RY) * BOXW + XPAD + 4 * lane;
                    float xs[4], sps[4], fs[4], z[4];
                    Vec4<TS>::load(reinterpret_cast<const TS*>(st) + off, xs);
                    Vec4<TS>::load(reinterpret_cast<const TS*>(st + C::ARR) + off, sps);
                    Vec4<TS>::load(reinterpret_cast<const TS*>(st + 2 * C::ARR) + off, fs);
                    float ak[4], af[4];   // adjoint terms (AUX only)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        // scale and gain applied here; t1 = f C0 - 2 C1
                        const float t1 = fmaf(fs[i], cab[i].x, cab[i].y);   // cab[i].y = -2 C1
                        const float t2 = fmaf(fs[i], t1, c2[i]);
                        const float kb = fmaf(-alpha, t2, cab[i].x);
                        z[i] = (sg_s * sps[i]) * kb;
                        if (AUX) {
                            ak[i] = kb;
                            af[i] = fmaf(-0.5f, cab[i].y, t1);   // f C0 - C1
                        }
                    }
                    if (MC && P.acc_in && st_ok && xg < g.pitch) {   // earlier channels' passes (Eq. 9 sums them)
                        float zp[4];
                        Vec4<TS>::load((const TS*)P.acc_in + g.off + (long long)o * g.plane +
                                           (long long)yy * g.pitch + xg,
                                       zp);
#pragma unroll
                        for (int i = 0; i < 4; ++i) z[i] += zp[i];
                    }
                    if (AUX && P.aux_k && st_ok && xg < g.pitch) {
                        const long long ao = g.off + (long long)o * g.plane + (long long)yy * g.pitch + xg;
                        Vec4<float>::store(P.aux_k + ao, ak);
                        Vec4<float>::store(P.aux_f + ao, af);
                    }
                    const long long zoff = (long long)o * g.plane + (long long)yy * g.pitch + xg;
                    if (st_ok && xg < g.pitch &&   // the lanes that store
                        !dbg_ok(zoff + 3 < (long long)g.nf * g.plane, kDbgStore, zoff, g.nf))
                        st_ok_dbg = false;
                    if (st_ok && st_ok_dbg) {
                        if (FO) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (xg + i < g.w) FO[((long long)o * g.h + yy) * g.w + xg + i] = z[i];
                        } else if (Z && xg < g.pitch) {
                            if (!std::is_same<TS, float>::value) {
#pragma unroll
                                for (int i = 0; i < 4; ++i) z[i] = to_f(from_f<TS>(z[i]));
                            }
                            Vec4<TS>::store(zp, z);
                        }
                    }
                    if (out_lane && !(MC && P.no_reduce)) {
                        if (kPairSums) {
#pragma unroll
                            for (int i = 0; i < 4; i += 2) {
                                const float2 z2 = make_float2(z[i], z[i + 1]), x2 = make_float2(xs[i], xs[i + 1]);
                                pp[0] = __ffma2_rn(z2, z2, pp[0]);
                                pp[1] = __ffma2_rn(x2, z2, pp[1]);
                                pp[2] = __ffma2_rn(x2, x2, pp[2]);
                                const float2 d2 = __ffma2_rn(nshift2, x2, z2);
                                pp[3] = __ffma2_rn(d2, d2, pp[3]);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                part[0] = fmaf(z[i], z[i], part[0]);
                                part[1] = fmaf(xs[i], z[i], part[1]);
                                part[2] = fmaf(xs[i], xs[i], part[2]);
                                const float dz = fmaf(-shift, xs[i], z[i]);
                                part[3] = fmaf(dz, dz, part[3]);
                            }
                        }
                    }
                    if (zp) zp += g.plane;
                    if (++flush == 16) {          // at most 64 FP32 terms per lane
                        flush = 0;
                        fold_pairs();
                        warp_flush(part, acc);
                    }
                }
                if (valid) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&empty[b]));
                    ++vc;
                }
                ++tin;
            };
            using I0 = std::integral_constant<int, 0>;
            using I1 = std::integral_constant<int, 1 % NR>;
            using I2 = std::integral_constant<int, 2 % NR>;
            using I3 = std::integral_constant<int, 3 % NR>;
            using I4 = std::integral_constant<int, 4 % NR>;
            static_assert(NR == 5 || NR == 3, "the phase unroll covers 2 RT + 1 = 3 or 5");
            while (tin < t_end) {
                frame(I0{});
                if (tin >= t_end) break;
                frame(I1{});
                if (tin >= t_end) break;
                frame(I2{});
                if (NR == 3 || tin >= t_end) continue;
                frame(I3{});
                if (tin >= t_end) break;
                frame(I4{});
            }
            fold_pairs();
            warp_flush(part, acc);
        }
        __syncthreads();
        if (s_abort) {
            // wait (bounded, ignoring the abort flag) for loads still in flight
            // into this CTA's stages
            if (tid == 0)
                for (int s = 0; s < NS; ++s)
                    if (owed & (1u << s)) (void)mbar_wait(smem_u32(&bars[s]), (owed_par >> s) & 1u);
            __syncthreads();
            return;
        }
        // buffer b was used ceil((n_valid - b) / NYB) times: FULL and EMPTY advanced
        for (int b = 0; b < C::NYB; ++b) {
            const unsigned uses = (unsigned)((n_valid - b + C::NYB - 1) / C::NYB);
            fullbase ^= (uses & 1u) << b;
            emptybase ^= (uses & 1u) << b;
        }
        // every valid frame of the segment completed one phase of its stage
        for (int s = 0; s < NS; ++s) {
            const int j = ((s - p_first) % NS + NS) % NS;        // first frame index on stage s
            const int cnt = (j < n_valid) ? (n_valid - 1 - j) / NS + 1 : 0;
            segphase ^= (unsigned)(cnt & 1) << s;
        }
        if (!(MC && P.no_reduce) && (sg + 1 == seg_e || P.items[sg + 1].video != v)) {
            // end of the run: its sum goes to the slot of its last segment, the
            // other segments' slots get zeros, and the run arrives once
            const double sc = (double)s_scale;
            double run[kRed];
            for (int c = 0; c < kRed; ++c) run[c] = (double)acc[c];
            run[1] *= sc;
            run[2] *= sc * sc;
            double* sh = reinterpret_cast<double*>(stages);
            block_sum_lane0(run, sh);
            if (tid == 0) {
                for (int q = run_first; q < sg; ++q)
                    for (int c = 0; c < kRed; ++c) P.partials[(long long)q * kRed + c] = 0.0;
                for (int c = 0; c < kRed; ++c) P.partials[(long long)sg * kRed + c] = run[c];
            }
            arrive_and_finalize(P, v, sh, (unsigned)(sg - run_first + 1));
            for (int c = 0; c < kRed; ++c) acc[c] = 0;
        }
        fence_proxy_async();   // generic writes to the stages precede the next TMA writes
        __syncthreads();
    }
}

}  // namespace fast

SFSEG_DEBUG_TU(fast)

// --------------------------------------------------------------- host side
struct FastEntry {
    int rt, ry, rx, storage;
    bool aux, mc;
    const void* fn;
    int smem;
};

// per radii: FP32 / BF16 / FP16; FP32 with the adjoint terms; FP32 channel passes
#define SFSEG_FAST(RT, RY, RX)                                                                         \
    {RT, RY, RX, 0, false, false, (const void*)fast::step_fast_kernel<RT, RY, RX, float, false, false>, \
     fast::Cfg<RT, RY, RX, float>::SMEM},                                                               \
    {RT, RY, RX, 1, false, false,                                                                       \
     (const void*)fast::step_fast_kernel<RT, RY, RX, __nv_bfloat16, false, false>,                      \
     fast::Cfg<RT, RY, RX, __nv_bfloat16>::SMEM},                                                       \
    {RT, RY, RX, 2, false, false, (const void*)fast::step_fast_kernel<RT, RY, RX, __half, false, false>, \
     fast::Cfg<RT, RY, RX, __half>::SMEM},                                                              \
    {RT, RY, RX, 0, true, false, (const void*)fast::step_fast_kernel<RT, RY, RX, float, true, false>,   \
     fast::Cfg<RT, RY, RX, float>::SMEM},                                                               \
    {RT, RY, RX, 0, false, true, (const void*)fast::step_fast_kernel<RT, RY, RX, float, false, true>,   \
     fast::Cfg<RT, RY, RX, float>::SMEM}

static const FastEntry kFast[] = {
    SFSEG_FAST(2, 5, 5),   // 11x11x5 Gaussian
    SFSEG_FAST(2, 4, 4),   // 9x9x5
};

static const FastEntry* find_fast(int rt, int ry, int rx, int storage, bool aux = false, bool mc = false) {
    for (const FastEntry& e : kFast)
        if (e.rt == rt && e.ry == ry && e.rx == rx && e.storage == storage && e.aux == aux && e.mc == mc)
            return &e;
    return nullptr;
}

bool fast_available(int rt, int ry, int rx, int storage) {
    return find_fast(rt, ry, rx, storage) != nullptr;
}

void fast_tile(int* tx, int* ty, int* threads) {
    *tx = fast::TX;
    *ty = fast::TY;
    *threads = fast::NT;
}

void fast_box(int ry, int* box_w, int* box_h, int* x_pad) {
    *box_w = fast::BOXW;
    *box_h = fast::TY + 2 * ry;
    *x_pad = fast::XPAD;
}

cudaError_t setup_step_fast(int rt, int ry, int rx, int storage) {
    const FastEntry* e = find_fast(rt, ry, rx, storage);
    if (!e) return cudaErrorInvalidValue;
    cudaError_t r = cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem);
    const FastEntry* ea = find_fast(rt, ry, rx, storage, true);          // adjoint terms (FP32)
    if (r == cudaSuccess && ea)
        r = cudaFuncSetAttribute(ea->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ea->smem);
    const FastEntry* em = find_fast(rt, ry, rx, storage, false, true);   // channel passes (FP32)
    if (r == cudaSuccess && em)
        r = cudaFuncSetAttribute(em->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, em->smem);
    return r;
}

cudaError_t launch_step_fast(int storage, const StepParams& P, int n_ctas, cudaStream_t s) {
    const FastEntry* e = find_fast(P.rt, P.ry, P.rx, storage, P.aux_k != nullptr, P.nchan > 1);
    if (!e) return cudaErrorInvalidValue;
    void* args[] = {const_cast<StepParams*>(&P)};
    return cudaLaunchKernel(e->fn, dim3(n_ctas), dim3(fast::NT), args, (size_t)e->smem, s);
}

}  // namespace sfseg
