// step_fast.cu -- the power step y = M x_hat (Eq. 7 x alpha) for the common
// radii, specialised at compile time.
//
// Work decomposition.  A video is cut into 112 x 16 (x, y) tiles; one unit is
// one output frame of one tile.  Persistent CTAs (one of 512 threads per SM)
// first stream one whole tile each, all in step (frame t of neighbouring
// tiles is loaded at about the same time, so the halo rows one CTA loads are
// still in L2 for the next); the remaining tiles' units are then split into
// equal contiguous ranges.  A range is a list of segments (tile, frames
// [ta, tb)); a segment that starts or ends inside a video recomputes the
// 2 RT boundary frames' spatial passes.
//
// Per segment the CTA streams frames.  For each input frame:
//   load    one thread issues three TMA 3D box loads (x, sp, f) of the tile
//           plus its halo (128 x (16 + 2 RY)) into a ring of RT + 2 shared-
//           memory stages (zero fill outside the volume = the zero padding of
//           Eq. 7's convolutions), one frame ahead, completion on an mbarrier;
//   y-pass  warps 0..7: a task is a column pair x 4 output rows; a0 = sp x,
//           a1 = f a0, a2 = f a1 and the vertical taps in registers, every
//           channel packed over the column pair (FMUL2 / FFMA2);
//   x-pass  warp w owns output row w; lanes 0..27 own 4 output columns each,
//           lanes 28..31 hold the 2 x 4 halo columns, so every halo value
//           comes from one shuffle with a source lane fixed per thread;
//   t-pass  each thread keeps 2 RT + 1 partial sums per voxel and channel in
//           registers; the slot roles are static per ring phase (a switch on
//           the phase selects one of 2 RT + 1 specialisations);
//   combine y = sp [(1 - a f^2) C0 + 2 a f C1 - a C2] for frame t - RT, with
//           the deferred scale and gain folded into the temporal taps;
//           16-byte stores, FP32 partial sums of z.z, x.z, x.x, |z - s x|^2
//           per thread, FP64 per warp and per segment.
// The last CTA of each video to finish reduces the per-segment partials and
// updates the video's scalars (no CTA waits on another).  Every mbarrier wait
// is bounded; on timeout the CTA records SFSEG_ETIMEOUT and stops.
#include <cuda.h>

#include <type_traits>

#include "sfseg_common.cuh"
#include "sfseg_launch.h"

namespace sfseg {
namespace fast {

constexpr int TX = 112, TY = 12, NT = 512, XPAD = 8, BOXW = TX + 2 * XPAD, YBW = BOXW;
constexpr int NA_WARPS = 4;                   // warps running the loads and the y-pass
constexpr long kWaitTries = 1L << 24;         // bounded mbarrier wait

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
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (long i = 0; i < kWaitTries; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
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
    static constexpr int NTA = 2 * NPAIR;                     // y-pass tasks: pair x 6 rows
    static constexpr int TROWS = TY / 2;                      // output rows per y-pass task
    static constexpr int SC0 = XPAD - RXE;                    // first y-pass stage column
    static constexpr int ROWS = TY + 2 * RY;                  // input rows per tile
    static constexpr int IN_ROWS = TROWS + 2 * RY;            // input rows per task
    static constexpr int NR = 2 * RT + 1;                     // temporal taps
    static constexpr int NS = RT + 3;                         // stages (see the stage-reuse note)
    static constexpr int BOX_BYTES = ROWS * BOXW * (int)sizeof(TS);
    static constexpr int ARR = (BOX_BYTES + 127) / 128 * 128; // one array of a stage
    static constexpr int STAGE = 3 * ARR;
    static constexpr int YBC = TY * YBW * 4;                  // one channel of one Yb buffer
    static constexpr int YB = 3 * YBC;                        // one Yb buffer (3 channels)
    static constexpr int NBAR = NS + 4;                       // stages, FULL[2], EMPTY[2]
    static constexpr int SMEM = NS * STAGE + 2 * YB + NBAR * 8 + 128;
    static_assert(NTA <= NA_WARPS * 32, "y-pass tasks exceed the y-pass warps");
    static_assert(RX <= XPAD && SC0 >= 0, "x radius exceeds the halo pad");
    static_assert(NS * STAGE >= NT * kRed * 8, "finalize scratch must fit in the stages");
    static_assert(NR <= 5, "the ring-phase switch covers 2 RT + 1 <= 5");
    static_assert(SMEM <= 232448, "shared memory per block");
};

// Lane that owns quad q of a Yb row: quads 2..29 are the output lanes 0..27,
// quads 0, 1 (left halo) and 30, 31 (right halo) belong to lanes 28..31.
__device__ __forceinline__ int quad_owner(int q) {
    return q < 2 ? 28 + q : (q < 30 ? q - 2 : q);
}

constexpr int NB_WARPS = NT / 32 - NA_WARPS;   // x-pass / temporal / combine warps

// Temporal taps of one channel for ring phase U: frame tin feeds outputs
// tin - RT + k with weight g_t(RT - k) (constant-bank operand); slot
// (U - RT + k) mod NR holds output tin - RT + k.  Returns the finished
// output (slot of k = 0) in c.
template <int U, int RT>
__device__ __forceinline__ void tpass(float (&ring)[2 * RT + 1][4], const float (&p)[4],
                                      const float* gt, float (&c)[4]) {
    constexpr int NR = 2 * RT + 1;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int slot = ((U - RT + k) % NR + NR) % NR;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (k == NR - 1) ring[slot][i] = p[i] * gt[k];
            else ring[slot][i] = fmaf(p[i], gt[k], ring[slot][i]);
        }
    }
    constexpr int slot0 = ((U - RT) % NR + NR) % NR;
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = ring[slot0][i];
}

template <int RT>
__device__ __forceinline__ void tpass_phase(int u, float (&ring)[2 * RT + 1][4], const float (&p)[4],
                                            const float* gt, float (&c)[4]) {
    constexpr int NR = 2 * RT + 1;
    switch (u) {
        case 0: tpass<0, RT>(ring, p, gt, c); break;
        case 1: tpass<1 % NR, RT>(ring, p, gt, c); break;
        case 2: tpass<2 % NR, RT>(ring, p, gt, c); break;
        case 3: tpass<3 % NR, RT>(ring, p, gt, c); break;
        default: tpass<4 % NR, RT>(ring, p, gt, c); break;
    }
}

// x-pass of the three channels of one Yb row (channel planes TY * YBW apart):
// lane l's outputs are Yb columns XPAD + 4l .. +3; its 4 + 2 RX input window
// is read straight from shared memory with aligned 16-byte loads; taps as
// constant-bank FMA operands.
template <int RX>
__device__ __forceinline__ void xpass3(const float* row, int lane, const float* gx, float (&p0)[4],
                                       float (&p1)[4], float (&p2)[4]) {
    constexpr int W0 = (XPAD - RX) & ~3;                    // aligned window start (column)
    constexpr int NQ = (XPAD + 4 + RX - W0 + 3) / 4;        // float4 loads per channel
    static_assert(4 * 27 + W0 + 4 * NQ <= YBW, "x window of the last output lane exceeds the row");
    constexpr int SH = XPAD - RX - W0;                      // offset of column -RX in the window
    float w[3][4 * NQ];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float4 v = *reinterpret_cast<const float4*>(row + ch * TY * YBW + 4 * lane + W0 + 4 * q);
            w[ch][4 * q] = v.x; w[ch][4 * q + 1] = v.y; w[ch][4 * q + 2] = v.z; w[ch][4 * q + 3] = v.w;
        }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int d = 0; d <= 2 * RX; ++d) {
            a0 = fmaf(w[0][SH + i + d], gx[d], a0);
            a1 = fmaf(w[1][SH + i + d], gx[d], a1);
            a2 = fmaf(w[2][SH + i + d], gx[d], a2);
        }
        p0[i] = a0;
        p1[i] = a1;
        p2[i] = a2;
    }
}

// x-pass of one channel of one Yb row: lane owns quad own_q; the halo comes
// from the lanes owning the neighbour quads (one shuffle per value).
template <int RX>
__device__ __forceinline__ void xpass(const float* row, int own_q, int src_m2, int src_m1, int src_p1,
                                      int src_p2, const float* gx, float (&out)[4]) {
    float o[4];
    {
        const float4 q = *reinterpret_cast<const float4*>(row + 4 * own_q);
        o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
    }
    float w[4 + 2 * RX];
#pragma unroll
    for (int c = -RX; c < 4 + RX; ++c) {
        if (c >= 0 && c < 4) {
            w[c + RX] = o[c];
        } else {
            const int qo = (c < 0) ? -((3 - c) / 4) : c / 4;   // floor(c / 4)
            const int e = c - 4 * qo;
            const int src = qo == -2 ? src_m2 : qo == -1 ? src_m1 : qo == 1 ? src_p1 : src_p2;
            w[c + RX] = __shfl_sync(0xffffffffu, o[e], src);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float acc = 0.f;
#pragma unroll
        for (int d = 0; d <= 2 * RX; ++d) acc = fmaf(w[i + d], gx[d], acc);
        out[i] = acc;
    }
}

// Warp roles.  Warps 0..3 ("A"): the elected thread issues the TMA loads one
// frame ahead; all of them run the y-pass of frame p into Yb[vc % 2] (vc
// counts the valid frames of the segment), then each A warp arrives once on
// the FULL mbarrier of that buffer.  Warps 4..15 ("B", one output row each):
// each waits on FULL on its own (the B warps are not coupled to each other),
// x-pass and temporal ring of the three channels, combine of frame p - RT
// (its x, sp, f from the frame's stage), store, then arrives once on EMPTY.
// A waits until all B warps have arrived on EMPTY of a buffer before refilling
// it, so A runs at most two frames ahead of B's completed work.
// Stage reuse: with NS = RT + 3 stages and loads one frame ahead, the load of
// frame p + 1 overwrites frame p - RT - 2, whose last reader (B's combine of
// that frame, at B's frame p - 2) arrived on EMPTY before A passes its wait
// at frame p.
template <int RT, int RY, int RX, typename TS>
__global__ void __launch_bounds__(NT, 1) step_fast_kernel(const __grid_constant__ StepParams P) {
    using C = Cfg<RT, RY, RX, TS>;
    constexpr int NR = C::NR, NS = C::NS;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* stages = smem;
    float* yb = reinterpret_cast<float*>(smem + NS * C::STAGE);        // [2][3][TY][YBW]
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + NS * C::STAGE + 2 * C::YB);
    __shared__ float s_scale, s_gain, s_shift;
    __shared__ int s_skip, s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool is_a = warp < NA_WARPS;
    const int brow = warp - NA_WARPS;            // B: output row of the tile
    const CUtensorMap* maps = reinterpret_cast<const CUtensorMap*>(P.maps);

    unsigned long long* full = bars + NS;       // [2], NA_WARPS arrivals per phase
    unsigned long long* empty = bars + NS + 2;  // [2], NB_WARPS arrivals per phase
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(smem_u32(&bars[s]), 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&full[b]), NA_WARPS);
            mbar_init(smem_u32(&empty[b]), NB_WARPS);
        }
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    // bit b: parity of the first FULL / EMPTY completion of buffer b in the
    // current segment; use n of buffer b completes phase base ^ (n & 1)
    unsigned fullbase = 0, emptybase = 0;
    // bit s: parity of the first completion of stage s in the current segment.
    // Inside a segment the valid frames p_first, p_first + 1, ... use stage
    // p % NS in turn, so frame p completes phase segphase[s] ^ ((p - p_first) / NS).
    unsigned segphase = 0;
    unsigned owed = 0, owed_par = 0;   // (thread 0) loads issued and not yet waited for

    const int seg_b = P.cta_begin[blockIdx.x], seg_e = P.cta_begin[blockIdx.x + 1];
    for (int sg = seg_b; sg < seg_e; ++sg) {
        const WorkItem it = P.items[sg];
        const int v = it.video;
        __syncthreads();   // every thread has read the previous segment's scalars
        if (tid == 0) {
            const VState* st = P.state + v;
            s_skip = st->done;
            s_scale = (float)st->scale;
            s_gain = (float)st->gain;
            s_shift = (float)(st->shift * st->scale);
        }
        __syncthreads();
        if (s_skip) continue;
        const VideoGeom g = P.geo[v];
        const int ta = it.t0, tb = it.t1, x0 = it.x0, y0 = it.y0;
        const int t_end = tb + RT;
        const int p_first = max(ta - RT, 0), p_last = min(t_end, g.nf);   // valid frames [p_first, p_last)
        const int n_valid = p_last - p_first;
        auto parity = [&](int p) -> unsigned {
            return ((segphase >> (p % NS)) ^ (unsigned)((p - p_first) / NS)) & 1u;
        };
        double acc[kRed] = {0.0, 0.0, 0.0, 0.0};

        if (is_a) {
            // ============================ A: loads + y-pass ====================
            const CUtensorMap* map_sp = maps + 4 * v + 0;
            const CUtensorMap* map_f = maps + 4 * v + 1;
            const CUtensorMap* map_x = maps + 4 * v + 2 + P.x_sel;
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
            float2 gy2[2 * RY + 1];
#pragma unroll
            for (int d = 0; d <= 2 * RY; ++d) gy2[d] = make_float2(P.gy[d], P.gy[d]);
            if (tid == 0 && n_valid > 0) issue(p_first);
            for (int vc = 0; vc < n_valid; ++vc) {
                const int p = p_first + vc;
                const int b = vc & 1;
                const unsigned n = (unsigned)(vc >> 1);
                if (n >= 1 && !mbar_wait(smem_u32(&empty[b]), ((emptybase >> b) ^ (n - 1)) & 1u)) s_abort = 1;
                if (tid == 0 && vc + 1 < n_valid) issue(p + 1);
                const int s = p % NS;
                if (!mbar_wait(smem_u32(&bars[s]), parity(p))) {
                    s_abort = 1;
                    atomicExch(&P.state[v].status, 6);
                    P.state[v].done = 1;
                }
                owed &= ~(1u << s);
                if (a_task) {
                    const unsigned char* st = stages + s * C::STAGE;
                    const int r0 = a_h * C::TROWS;
                    const TS* sx = reinterpret_cast<const TS*>(st) + r0 * BOXW + a_sc;
                    const TS* ssp = reinterpret_cast<const TS*>(st + C::ARR) + r0 * BOXW + a_sc;
                    const TS* sf = reinterpret_cast<const TS*>(st + 2 * C::ARR) + r0 * BOXW + a_sc;
                    float2 q0[C::TROWS], q1[C::TROWS], q2[C::TROWS];
#pragma unroll
                    for (int o = 0; o < C::TROWS; ++o) {
                        q0[o] = make_float2(0.f, 0.f);
                        q1[o] = make_float2(0.f, 0.f);
                        q2[o] = make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int i = 0; i < C::IN_ROWS; ++i) {
                        const float2 xv = Ld2<TS>::get(sx + i * BOXW);
                        const float2 sv = Ld2<TS>::get(ssp + i * BOXW);
                        const float2 fv = Ld2<TS>::get(sf + i * BOXW);
                        const float2 b0 = __fmul2_rn(sv, xv);
                        const float2 b1 = __fmul2_rn(fv, b0);
                        const float2 b2 = __fmul2_rn(fv, b1);
#pragma unroll
                        for (int o = 0; o < C::TROWS; ++o) {
                            const int d = i - o;
                            if (d >= 0 && d <= 2 * RY) {
                                q0[o] = __ffma2_rn(b0, gy2[d], q0[o]);
                                q1[o] = __ffma2_rn(b1, gy2[d], q1[o]);
                                q2[o] = __ffma2_rn(b2, gy2[d], q2[o]);
                            }
                        }
                    }
                    float* yc = yb + b * 3 * TY * YBW;
#pragma unroll
                    for (int o = 0; o < C::TROWS; ++o) {
                        const int r = (r0 + o) * YBW + a_sc;
                        *reinterpret_cast<float2*>(yc + r) = q0[o];
                        *reinterpret_cast<float2*>(yc + TY * YBW + r) = q1[o];
                        *reinterpret_cast<float2*>(yc + 2 * TY * YBW + r) = q2[o];
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&full[b]));
            }
        } else {
            // ================= B: x-pass, temporal ring, combine ==============
            const float sg_s = s_scale * s_gain;     // deferred scale and gain
            const float alpha = P.alpha, shift = s_shift;
            const int own_q = lane < 28 ? lane + 2 : (lane < 30 ? lane - 28 : lane);
            const int src_m2 = quad_owner(max(own_q - 2, 0)), src_m1 = quad_owner(max(own_q - 1, 0));
            const int src_p1 = quad_owner(min(own_q + 1, 31)), src_p2 = quad_owner(min(own_q + 2, 31));
            const bool out_lane = lane < 28;
            TS* Z = P.z_out ? (TS*)P.z_out + g.off : nullptr;
            float* FO = P.final_out ? P.final_out[v] : nullptr;
            const int yy = y0 + brow;
            const int xg = x0 + 4 * lane;
            const bool st_ok = out_lane && yy < g.h;

            float r0[NR][4], r1[NR][4], r2[NR][4];   // temporal rings, one per channel
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int i = 0; i < 4; ++i) r0[k][i] = r1[k][i] = r2[k][i] = 0.f;
            float part[kRed] = {0.f, 0.f, 0.f, 0.f};
            int u = 0;             // ring phase of frame tin: (tin - (ta - RT)) mod NR
            int flush = 0;
            int vc = 0;
            for (int tin = ta - RT; tin < t_end; ++tin) {
                const bool valid = (tin >= 0 && tin < g.nf);
                const int b = vc & 1;
                float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
                float p2[4] = {0.f, 0.f, 0.f, 0.f};
                if (valid) {
                    if (!mbar_wait(smem_u32(&full[b]), ((fullbase >> b) ^ (unsigned)(vc >> 1)) & 1u))
                        s_abort = 1;
                    const float* row = yb + (b * 3 * TY + brow) * YBW;
                    // lanes 28..31 have no outputs: give them lane 27's window so
                    // every read stays inside the row (columns <= XPAD + 4*27 + 4 + RX)
                    xpass3<RX>(row, out_lane ? lane : 27, P.gx, p0, p1, p2);
                }
                float c0[4], c1[4], c2[4];
                tpass_phase<RT>(u, r0, p0, P.gt, c0);
                tpass_phase<RT>(u, r1, p1, P.gt, c1);
                tpass_phase<RT>(u, r2, p2, P.gt, c2);
                u = (u == NR - 1) ? 0 : u + 1;
                const int o = tin - RT;
                if (o >= ta && o < tb) {
                    const int so = o % NS;
                    // the frame's load completed long ago (A waited for it); this
                    // wait returns at once and orders the reads after the load
                    (void)mbar_wait(smem_u32(&bars[so]), parity(o));
                    const unsigned char* st = stages + so * C::STAGE;
                    const int off = (brow + RY) * BOXW + XPAD + 4 * lane;
                    float xs[4], sps[4], fs[4], z[4];
                    Vec4<TS>::load(reinterpret_cast<const TS*>(st) + off, xs);
                    Vec4<TS>::load(reinterpret_cast<const TS*>(st + C::ARR) + off, sps);
                    Vec4<TS>::load(reinterpret_cast<const TS*>(st + 2 * C::ARR) + off, fs);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        // scale and gain applied here; t1 = f C0 - 2 C1
                        const float t1 = fmaf(fs[i], c0[i], -2.f * c1[i]);
                        const float t2 = fmaf(fs[i], t1, c2[i]);
                        z[i] = (sg_s * sps[i]) * fmaf(-alpha, t2, c0[i]);
                    }
                    if (st_ok) {
                        if (FO) {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (xg + i < g.w) FO[((long long)o * g.h + yy) * g.w + xg + i] = z[i];
                        } else if (Z && xg < g.pitch) {
                            if (!std::is_same<TS, float>::value) {
#pragma unroll
                                for (int i = 0; i < 4; ++i) z[i] = to_f(from_f<TS>(z[i]));
                            }
                            Vec4<TS>::store(Z + (long long)o * g.plane + (long long)yy * g.pitch + xg, z);
                        }
                    }
                    if (out_lane) {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            part[0] = fmaf(z[i], z[i], part[0]);
                            part[1] = fmaf(xs[i], z[i], part[1]);
                            part[2] = fmaf(xs[i], xs[i], part[2]);
                            const float dz = fmaf(-shift, xs[i], z[i]);
                            part[3] = fmaf(dz, dz, part[3]);
                        }
                    }
                    if (++flush == 8) {
                        flush = 0;
                        warp_flush(part, acc);
                    }
                }
                if (valid) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&empty[b]));
                    ++vc;
                }
            }
            warp_flush(part, acc);
        }
        __syncthreads();
        if (s_abort) {
            // wait (bounded) for loads still in flight into this CTA's stages
            if (tid == 0)
                for (int s = 0; s < NS; ++s)
                    if (owed & (1u << s)) (void)mbar_wait(smem_u32(&bars[s]), (owed_par >> s) & 1u);
            __syncthreads();
            return;
        }
        // buffer b was used (n_valid + 1 - b) / 2 times: FULL and EMPTY advanced
        for (int b = 0; b < 2; ++b) {
            const unsigned uses = (unsigned)((n_valid + 1 - b) / 2);
            fullbase ^= (uses & 1u) << b;
            emptybase ^= (uses & 1u) << b;
        }
        // every valid frame of the segment completed one phase of its stage
        for (int s = 0; s < NS; ++s) {
            const int j = ((s - p_first) % NS + NS) % NS;        // first frame index on stage s
            const int cnt = (j < n_valid) ? (n_valid - 1 - j) / NS + 1 : 0;
            segphase ^= (unsigned)(cnt & 1) << s;
        }
        {
            const double sc = (double)s_scale;
            acc[1] *= sc;
            acc[2] *= sc * sc;
        }
        double* sh = reinterpret_cast<double*>(stages);
        block_sum_lane0(acc, sh);
        if (tid == 0)
            for (int c = 0; c < kRed; ++c) P.partials[(long long)sg * kRed + c] = acc[c];
        arrive_and_finalize(P, v, sh);
        fence_proxy_async();   // generic writes to the stages precede the next TMA writes
        __syncthreads();
    }
}

}  // namespace fast

// --------------------------------------------------------------- host side
struct FastEntry {
    int rt, ry, rx, storage;
    const void* fn;
    int smem;
};

#define SFSEG_FAST(RT, RY, RX)                                                                    \
    {RT, RY, RX, 0, (const void*)fast::step_fast_kernel<RT, RY, RX, float>,                     \
     fast::Cfg<RT, RY, RX, float>::SMEM},                                                          \
    {RT, RY, RX, 1, (const void*)fast::step_fast_kernel<RT, RY, RX, __nv_bfloat16>,             \
     fast::Cfg<RT, RY, RX, __nv_bfloat16>::SMEM},                                                  \
    {RT, RY, RX, 2, (const void*)fast::step_fast_kernel<RT, RY, RX, __half>,                    \
     fast::Cfg<RT, RY, RX, __half>::SMEM}

static const FastEntry kFast[] = {
    SFSEG_FAST(2, 5, 5),   // 11x11x5 Gaussian
    SFSEG_FAST(2, 4, 4),   // 9x9x5
};

static const FastEntry* find_fast(int rt, int ry, int rx, int storage) {
    for (const FastEntry& e : kFast)
        if (e.rt == rt && e.ry == ry && e.rx == rx && e.storage == storage) return &e;
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
    return cudaFuncSetAttribute(e->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem);
}

cudaError_t launch_step_fast(int storage, const StepParams& P, int n_ctas, cudaStream_t s) {
    const FastEntry* e = find_fast(P.rt, P.ry, P.rx, storage);
    if (!e) return cudaErrorInvalidValue;
    void* args[] = {const_cast<StepParams*>(&P)};
    return cudaLaunchKernel(e->fn, dim3(n_ctas), dim3(fast::NT), args, (size_t)e->smem, s);
}

}  // namespace sfseg
