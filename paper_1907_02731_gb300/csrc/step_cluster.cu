// step_cluster.cu -- all K power steps of one small video inside one
// thread-block cluster, the whole video resident in shared memory.
//
// For volumes of a few hundred thousand voxels the per-step kernels and the
// fused cooperative launch are bound by latency: every step pays its
// grid-wide synchronisation and the round trips of its operands through L2.
// Here one cluster of up to 16 CTAs (one 16 x TH spatial tile each, all
// frames) keeps sp, f and the iterate in shared memory for the whole call of
// Alg. 1 (Eq. 4 + Eq. 8), and per step:
//
//   halo     warps 1..15 fetch the halo ring of each frame's extended tile
//            (RY rows above and below, RX columns left and right) from the
//            neighbouring CTAs' tile buffers through distributed shared memory
//            (zero outside the video: the zero padding of Eq. 7's
//            convolutions); the interior is the tile's own iterate, written by
//            the previous step's combine;
//   y, x     per (frame, 8-row chunk) task, one warp (tasks from a shared
//            counter): the point-wise products a0 = sp x, a1 = f a0,
//            a2 = f a1 and the y-pass with the lanes on the extended columns
//            and the rows unrolled (Eq. 7, Sec. 4), then the x-pass from a
//            warp-private row buffer; C0 and C1 travel as packed pairs;
//   t, comb  per tile column and frame range, one thread: the temporal taps as
//            a register ring, the combine y = sp [(1 - a f^2) C0 + 2 a f C1 -
//            a C2] with the deferred scale and gain, the stored (rounded)
//            iterate into the other of two tile buffers and into the extended
//            tile's interior, the sums z.z, xh.z, xh.xh, |z - s xh|^2 in FP32
//            trees over lanes and warps: one record per CTA;
//   barrier  one cluster barrier; then warp 0 of every CTA fetches the 16
//            records, sums them in a fixed FP64 tree and runs the scalar
//            update (finish_step of the other paths) on the CTA's copy of the
//            video's state -- while warps 1..15 already assemble the next halo
//            and start the next y/x tasks, which need no scalar -- so all CTAs
//            hold bitwise-identical scalars and take the same branch; rank 0
//            writes the trace row.
//
// Waits: the only waits between CTAs are cluster barriers, which every CTA
// reaches on the same control flow (its decisions come from the identical
// scalars); there is no spin-wait.  A final cluster barrier keeps every CTA's
// shared memory alive until the last remote read.  At the end rank 0 writes
// the state back and each CTA writes its tile of the result: the last step's
// FP32 output into the caller's buffer (final mode) or the stored iterate of
// the last completed step into the ping-pong buffer finish_kernel reads.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "sfseg_common.cuh"
#include "sfseg_launch.h"

namespace sfseg {
namespace cgc = cooperative_groups;

namespace clu {

constexpr int TW = 16;                 // tile width (interior columns per CTA)
constexpr int RC = 8;                  // output rows per y-pass task
constexpr int NTH = 512;               // threads per CTA
constexpr int NWARP = NTH / 32;
static_assert(RC * (TW / 4) == 32, "x-pass: one lane per (row, 4-column group) of a task");

template <int RT, int RY, int RX>
struct Cfg {
    static constexpr int EW = TW + 2 * RX;                 // extended columns (y-pass lanes)
    static constexpr int NQ = (4 + 2 * RX + 3) / 4;        // float4 loads of an x-pass window
    // row stride of the y-pass output rows: holds the last group's window and
    // is an odd number of 16-byte chunks (the 8 rows a load phase touches fall
    // in 8 distinct bank groups)
    static constexpr int YW0 = TW - 4 + 4 * NQ;
    static constexpr int YW = ((YW0 / 4) & 1) ? YW0 : YW0 + 4;
    static constexpr int PW = TW + 4;                      // row stride of the C2 planes (5 chunks)
    // channels C0 and C1 travel as interleaved pairs (packed FMAs): the
    // x-pass window of 4 outputs is NQ2 16-byte loads of two column pairs; row
    // strides in pairs, an odd number of 16-byte chunks
    static constexpr int NQ2 = (4 + 2 * RX + 1) / 2;
    static constexpr int YW20 = (EW > TW - 4 + 2 * NQ2 ? EW : TW - 4 + 2 * NQ2);
    static constexpr int YW2 = (((YW20 + 1) / 2) & 1) ? (YW20 + 1) / 2 * 2 : (YW20 + 1) / 2 * 2 + 2;
    static constexpr int PW2 = TW + 2;
    static constexpr int NR = 2 * RT + 1;
    static_assert(EW <= 32, "the extended tile row must fit the lanes of a warp");
    static_assert(YW >= EW, "y-pass rows hold the extended columns");
    static_assert(((YW2 / 2) & 1) && ((PW2 / 2) & 1) && YW2 >= EW, "pair strides");
};

// Shared-memory layout (floats) for nf frames and tile height th.
struct Layout {
    int eh, ew, yw, pw, yw2, pw2;
    long long spe, fe, xe, zt0, zt1, pv01, pv2, yrow, total;
};
struct Strides {
    int yw, pw, yw2, pw2;
};
__host__ __device__ inline Layout layout(int nf, int th, int ry, int rx, Strides S) {
    Layout L;
    L.eh = th + 2 * ry;
    L.ew = TW + 2 * rx;
    L.yw = S.yw;
    L.pw = S.pw;
    L.yw2 = S.yw2;
    L.pw2 = S.pw2;
    // every array starts on a 16-byte boundary (float4 access)
    const long long ext = ((long long)nf * L.eh * L.ew + 3) & ~3ll;
    const long long tile = (long long)nf * th * TW;
    L.spe = 0;
    L.fe = L.spe + ext;
    L.xe = L.fe + ext;
    L.zt0 = L.xe + ext;
    L.zt1 = L.zt0 + tile;
    L.pv01 = L.zt1 + tile;                                 // [nf][th][pw2] (C0, C1) pairs
    L.pv2 = L.pv01 + 2ll * nf * th * L.pw2;                // [nf][th][pw] C2
    L.yrow = L.pv2 + (long long)nf * th * L.pw;            // per warp: [RC][yw2] pairs, [RC][yw]
    L.total = L.yrow + (long long)NWARP * RC * (2 * L.yw2 + L.yw);
    L.total = (L.total + 3) & ~3ll;
    return L;
}
// bytes: the float arrays and the two record slots [2][kRed] (doubles)
inline size_t smem_bytes(int nf, int th, int ry, int rx, Strides S) {
    const Layout L = layout(nf, th, ry, rx, S);
    return sizeof(float) * (size_t)L.total + sizeof(double) * 2 * kRed;
}

// Barrier `id` among n threads of the CTA (a multiple of 32); arrive marks
// this warp's arrival without waiting (producer side of the same barrier).
__device__ __forceinline__ void named_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Calls f(integral_constant<0>), f(<1>), ... in order while they return true.
template <typename F, int... I>
__device__ __forceinline__ bool phase_round(F&& f, std::integer_sequence<int, I...>) {
    return (f(std::integral_constant<int, I>{}) && ...);
}

template <int RT, int RY, int RX, typename TS>
__global__ void __launch_bounds__(NTH, 1) step_cluster_kernel(const __grid_constant__ ClusterParams C) {
    using Q = Cfg<RT, RY, RX>;
    constexpr int NR = Q::NR, EW = Q::EW;
    const StepParams& P = C.S;
    cgc::cluster_group cluster = cgc::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int ncta = (int)cluster.num_blocks();
    extern __shared__ __align__(16) float sm[];
    const VideoGeom g = P.geo[0];
    const int nf = g.nf, th = C.th;
    const Layout L = layout(nf, th, RY, RX, Strides{Q::YW, Q::PW, Q::YW2, Q::PW2});
    float* spe = sm + L.spe;
    float* fe = sm + L.fe;
    float* xe = sm + L.xe;
    float2* pv01 = reinterpret_cast<float2*>(sm + L.pv01);
    float* pv2 = sm + L.pv2;
    double* slots = reinterpret_cast<double*>(sm + L.total);   // [2][kRed]
    __shared__ VState s_st;
    __shared__ float s_scale, s_sg, s_shift;
    __shared__ int s_done, s_task;
    __shared__ float s_wsum[NWARP * kRed];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = rank % C.tiles_x, ty = rank / C.tiles_x;
    const int x0 = tx * TW, y0 = ty * th;
    const int eh = L.eh;
    const long long tile = (long long)nf * th * TW;
    const TS* SPg = (const TS*)P.sp + g.off;
    const TS* Fg = (const TS*)P.f + g.off;
    const TS* X0 = (const TS*)C.buf0 + g.off;

    // ------------------------------------------------------------ set-up
    // sp and f over the extended tile (zero outside the video), the stored x0
    // over the tile (zero outside), the video's scalars
    {
        // one extended row (t, ey) per warp and round, lane = extended column,
        // SU rows' loads in flight before their stores; x0 on the tile rows
        constexpr int SU = 4;
        const int xx = x0 - RX + lane;
        const bool xin = lane < EW && xx >= 0 && xx < g.w;
        const bool own = xin && lane >= RX && lane < RX + TW;
        const int nrow = nf * eh;
        for (int r0 = warp; r0 < nrow; r0 += NWARP * SU) {
            float s[SU], f[SU], x[SU];
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                const int r = r0 + u * NWARP;
                const int t = r / eh, ey = r - t * eh, yy = y0 - RY + ey;
                s[u] = f[u] = x[u] = 0.f;
                if (r < nrow && xin && yy >= 0 && yy < g.h) {
                    const long long o = (long long)t * g.plane + (long long)yy * g.pitch + xx;
                    s[u] = to_f(SPg[o]);
                    f[u] = to_f(Fg[o]);
                    if (own && ey >= RY && ey < RY + th) x[u] = to_f(X0[o]);
                }
            }
#pragma unroll
            for (int u = 0; u < SU; ++u) {
                const int r = r0 + u * NWARP;
                if (r < nrow && lane < EW) {
                    spe[r * EW + lane] = s[u];
                    fe[r * EW + lane] = f[u];
                    xe[r * EW + lane] = x[u];   // the tile's own x0; the halo is assembled per step
                    const int t = r / eh, ey = r - t * eh;
                    if (lane >= RX && lane < RX + TW && ey >= RY && ey < RY + th)
                        sm[L.zt0 + (t * th + ey - RY) * TW + lane - RX] = x[u];
                }
            }
        }
    }
    if (tid == 0) {
        s_st = P.state[0];
        s_task = 0;
    }
    cluster.sync();   // every tile's x0 is in place before the first remote read

    const float alpha = P.alpha;
    // warp 0 publishes the scalars of the next step: after step kk's records
    // are in place it fetches all of them (lane q: CTA q's record, one round
    // trip), sums them in a fixed tree order in FP64 and runs the scalar
    // update on the CTA's copy of the state (lane 0)
    auto publish = [&](int kk) {
        if (kk >= 0) {
            double v[kRed];
#pragma unroll
            for (int c = 0; c < kRed; ++c) v[c] = 0.0;
            if (lane < ncta) {
                const double* sq = lane == rank ? slots : cluster.map_shared_rank(slots, lane);
#pragma unroll
                for (int c = 0; c < kRed; ++c) v[c] = sq[(kk & 1) * kRed + c];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int c = 0; c < kRed; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], off);
            if (lane == 0) {
                const int it = s_st.iter;
                double* row = (rank == 0 && it < P.trace_cap) ? P.trace + (long long)it * 3 : nullptr;
                finish_step(&s_st, row, v, g.n, nullptr);
            }
        }
        if (lane == 0) {
            s_done = s_st.done;
            s_scale = (float)s_st.scale;
            s_sg = (float)(s_st.scale * s_st.gain);
            s_shift = (float)s_st.shift;
        }
        __syncwarp();
    };

    int k = 0;
    bool stopped = false;
    for (; k < C.n_steps; ++k) {
        const float* zin = sm + ((k & 1) ? L.zt1 : L.zt0);
        float* zout = sm + ((k & 1) ? L.zt0 : L.zt1);
        const bool final_step = C.final_mode && k == C.n_steps - 1;

        if (warp == 0) {
            // the update of step k - 1 overlaps the other warps' halo assembly
            // and first y/x tasks of step k (which need no scalar)
            publish(k - 1);
            named_sync(2, NTH);   // the assembly of every other warp is complete
        } else {
            // ------------------------------------------- halo assembly
            // warps 1..15 fetch the halo ring of the extended tile (the
            // interior holds the tile's own iterate, written by the previous
            // step's combine): per frame RY rows above and below (all
            // extended columns) and RX columns left and right of the tile
            // rows; HU elements' loads (remote) before their stores.  The
            // owner of a halo voxel is a neighbouring tile (halo < tile), so
            // no division by the tile size.
            constexpr int HU = 8, NWK = NWARP - 1;
            constexpr int NTOP = RY * EW, NSIDE = RX;   // per frame: 2 NTOP + 2 th NSIDE
            const int nh = 2 * NTOP + 2 * th * NSIDE, ntot = nf * nh;
            // i / nh = umulhi(i, inv_nh): exact for nh >= 2 and i < 2^16
            const unsigned inv_nh = 0xffffffffu / (unsigned)nh + 1u;
            const int wt = tid - 32;
            for (int i0 = wt; i0 < ntot; i0 += NWK * 32 * HU) {
                float v[HU];
                int dst[HU];
#pragma unroll
                for (int u = 0; u < HU; ++u) {
                    const int i = i0 + u * NWK * 32;
                    const int t = (int)__umulhi((unsigned)i, inv_nh), j = i - t * nh;
                    int ey, ex;
                    if (j < NTOP) {
                        ey = j / EW; ex = j - ey * EW;
                    } else if (j < 2 * NTOP) {
                        const int j2 = j - NTOP;
                        ey = RY + th + j2 / EW; ex = j2 - (j2 / EW) * EW;
                    } else {
                        const int j3 = j - 2 * NTOP;
                        const int side = j3 >= th * NSIDE ? 1 : 0, j4 = j3 - side * th * NSIDE;
                        ey = RY + j4 / NSIDE;
                        ex = side * (RX + TW) + (j4 - (j4 / NSIDE) * NSIDE);
                    }
                    const int yy = y0 - RY + ey, xx = x0 - RX + ex;
                    dst[u] = (t * eh + ey) * EW + ex;
                    v[u] = 0.f;
                    if (i < ntot && yy >= 0 && yy < g.h && xx >= 0 && xx < g.w) {
                        const int oty = ty + (yy >= y0 + th ? 1 : 0) - (yy < y0 ? 1 : 0);
                        const int otx = tx + (xx >= x0 + TW ? 1 : 0) - (xx < x0 ? 1 : 0);
                        const int owner = oty * C.tiles_x + otx;
                        const int o = (t * th + (yy - oty * th)) * TW + (xx - otx * TW);
                        if (dbg_ok(owner >= 0 && owner < ncta && owner != rank && t < nf, kDbgSlot, owner, ncta))
                            v[u] = cluster.map_shared_rank(zin, owner)[o];
                    }
                }
#pragma unroll
                for (int u = 0; u < HU; ++u)
                    if (i0 + u * NWK * 32 < ntot) xe[dst[u]] = v[u];
            }
            named_arrive(2, NTH);
            named_sync(1, NTH - 32);   // xe is complete for the y/x tasks
        }

        // ------------------------------------------------- y and x passes
        // tasks (frame, 8-row chunk) from a shared counter: warp 0 takes its
        // share once its update is done
        {
            float2* yr01 = reinterpret_cast<float2*>(sm + L.yrow + (long long)warp * RC * (2 * Q::YW2 + Q::YW));
            float* yr2 = reinterpret_cast<float*>(yr01 + RC * Q::YW2);
            const int nchunk = th / RC, ntask = nf * nchunk;
            for (;;) {
                int task = 0;
                if (lane == 0) task = atomicAdd(&s_task, 1);
                task = __shfl_sync(0xffffffffu, task, 0);
                if (task >= ntask) break;
                const int t = task / nchunk, c = task - t * nchunk;
                if (lane < EW) {
                    const int b = (t * eh + c * RC) * EW + lane;
                    float2 acc01[RC];
                    float acc2[RC];
#pragma unroll
                    for (int i = 0; i < RC + 2 * RY; ++i) {
                        const float a0 = spe[b + i * EW] * xe[b + i * EW];
                        const float fv = fe[b + i * EW];
                        const float a1 = fv * a0, a2 = fv * a1;
                        const float2 a01 = make_float2(a0, a1);
#pragma unroll
                        for (int j = 0; j < RC; ++j) {
                            const int d = i - j;
                            if (d == 0) {
                                acc01[j] = __fmul2_rn(a01, P.gy2[0]);
                                acc2[j] = P.gy[0] * a2;
                            } else if (d > 0 && d <= 2 * RY) {
                                acc01[j] = __ffma2_rn(a01, P.gy2[d], acc01[j]);
                                acc2[j] = fmaf(P.gy[d], a2, acc2[j]);
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < RC; ++j) {
                        yr01[j * Q::YW2 + lane] = acc01[j];
                        yr2[j * Q::YW + lane] = acc2[j];
                    }
                }
                __syncwarp();
                {
                    const int gi = lane >> 3, j = lane & 7;   // 4-column group, row of the task
                    // (C0, -2 C1) with the pair taps (g, -2 g): the factor is exact
                    {
                        const float2* row = yr01 + j * Q::YW2 + 4 * gi;
                        float2 w[2 * Q::NQ2];
#pragma unroll
                        for (int q = 0; q < Q::NQ2; ++q) {
                            const float4 v = *reinterpret_cast<const float4*>(row + 2 * q);
                            w[2 * q] = make_float2(v.x, v.y);
                            w[2 * q + 1] = make_float2(v.z, v.w);
                        }
                        float2 o[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float2 a = __fmul2_rn(w[i], P.gx2[0]);
#pragma unroll
                            for (int d = 1; d <= 2 * RX; ++d) a = __ffma2_rn(w[i + d], P.gx2[d], a);
                            o[i] = a;
                        }
                        float4* dst = reinterpret_cast<float4*>(pv01 + (t * th + c * RC + j) * Q::PW2 + 4 * gi);
                        dst[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
                        dst[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
                    }
                    {
                        const float* row = yr2 + j * Q::YW + 4 * gi;
                        float w[4 * Q::NQ];
#pragma unroll
                        for (int q = 0; q < Q::NQ; ++q) {
                            const float4 v = *reinterpret_cast<const float4*>(row + 4 * q);
                            w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w;
                        }
                        float o[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            float a = P.gx[0] * w[i];
#pragma unroll
                            for (int d = 1; d <= 2 * RX; ++d) a = fmaf(P.gx[d], w[i + d], a);
                            o[i] = a;
                        }
                        float* dst = pv2 + (t * th + c * RC + j) * Q::PW + 4 * gi;
                        *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
                    }
                }
                __syncwarp();   // the row buffer is rewritten by the warp's next task
            }
        }
        __syncthreads();
        if (s_done) {   // identical in every CTA: the update of step k - 1 ended the iteration
            stopped = true;
            break;
        }

        // --------------------------- t-pass, combine, store, reductions
        {
            if (tid == 0) s_task = 0;   // every warp has left the task loop
            const float scale = s_scale, sg = s_sg, shift = s_shift;
            const int ncol = th * TW;
            const int fg_n = NTH / ncol > 0 ? (NTH / ncol < nf ? NTH / ncol : nf) : 1;
            float part[kRed] = {0.f, 0.f, 0.f, 0.f};
            float* FO = final_step ? P.final_out[0] : nullptr;
            const int plane01 = th * Q::PW2, plane2 = th * Q::PW;
            for (int idx = tid; idx < ncol * fg_n; idx += NTH) {
                const int fgi = idx / ncol, col = idx - fgi * ncol;
                const int ly = col / TW, lx = col - ly * TW;
                const int yy = y0 + ly, xx = x0 + lx;
                const bool in_vid = yy < g.h && xx < g.w;
                const int ta = fgi * nf / fg_n, tb = (fgi + 1) * nf / fg_n;
                const float2* pc01 = pv01 + ly * Q::PW2 + lx;    // + t plane01
                const float* pc2 = pv2 + ly * Q::PW + lx;        // + t plane2
                const int e0 = (ly + RY) * EW + lx + RX;         // + t eh EW
                float2 ring01[NR];
                float ring2[NR];
#pragma unroll
                for (int s = 0; s < NR; ++s) {
                    ring01[s] = make_float2(0.f, 0.f);
                    ring2[s] = 0.f;
                }
                int tin = ta - RT;
                const int t_end = tb + RT;
                auto frame = [&](auto phase) -> bool {
                    constexpr int U = decltype(phase)::value;
                    if (tin >= t_end) return false;
                    float2 p01 = make_float2(0.f, 0.f);
                    float p2 = 0.f;
                    if (tin >= 0 && tin < nf) {
                        p01 = pc01[tin * plane01];
                        p2 = pc2[tin * plane2];
                    }
                    // input frame tin is tap d = 2 RT - m of output tin - RT + m
                    // (the first of its taps when m = 2 RT); slot (U - RT + m)
                    // mod NR holds that output
#pragma unroll
                    for (int m = 0; m < NR; ++m) {
                        const int slot = ((U - RT + m) % NR + NR) % NR;
                        if (m == NR - 1) {
                            ring01[slot] = __fmul2_rn(p01, P.gt2[NR - 1 - m]);
                            ring2[slot] = P.gt[NR - 1 - m] * p2;
                        } else {
                            ring01[slot] = __ffma2_rn(p01, P.gt2[NR - 1 - m], ring01[slot]);
                            ring2[slot] = fmaf(P.gt[NR - 1 - m], p2, ring2[slot]);
                        }
                    }
                    constexpr int s0 = ((U - RT) % NR + NR) % NR;   // output tin - RT is complete
                    const int o = tin - RT;
                    if (o >= ta && o < tb && in_vid) {
                        const float c0 = ring01[s0].x, c1m2 = ring01[s0].y, c2 = ring2[s0];   // c1m2 = -2 C1
                        const int e = o * eh * EW + e0;
                        const float s = spe[e], fv = fe[e];
                        const int zo = o * th * TW + col;
                        const float xh = scale * zin[zo];
                        const float af = alpha * fv;
                        const float inner = fmaf(-af, c1m2, fmaf(-af, fv, 1.f) * c0) - alpha * c2;
                        float z = sg * (s * inner);
                        if (FO) {
                            FO[((long long)o * g.h + yy) * g.w + xx] = z;
                        } else {
                            z = to_f(from_f<TS>(z));
                            zout[zo] = z;   // for the neighbours' halos
                            xe[e] = z;      // the next step's own interior (phase 1 is done)
                        }
                        part[0] = fmaf(z, z, part[0]);
                        part[1] = fmaf(xh, z, part[1]);
                        part[2] = fmaf(xh, xh, part[2]);
                        const float dz = fmaf(-shift, xh, z);
                        part[3] = fmaf(dz, dz, part[3]);
                    }
                    ++tin;
                    return true;
                };
                while (phase_round(frame, std::make_integer_sequence<int, NR>{})) {
                }
            }
            // the CTA's record: FP32 trees over lanes, then over warps (FP64
            // is slow on this GPU and the CTA holds a few thousand voxels);
            // the records of all CTAs are summed in FP64
#pragma unroll
            for (int c = 0; c < kRed; ++c) {
                const float w = warp_sum(part[c]);
                if (lane == 0) s_wsum[warp * kRed + c] = w;
            }
            __syncthreads();
            if (warp == 0) {
#pragma unroll
                for (int c = 0; c < kRed; ++c) {
                    const float w = warp_sum(lane < NWARP ? s_wsum[lane * kRed + c] : 0.f);
                    if (lane == 0) slots[(k & 1) * kRed + c] = (double)w;
                }
            }
        }
        cluster.sync();   // every tile's z and record are in place
    }
    if (!stopped && warp == 0) publish(k - 1);   // the update of the last step
    cluster.sync();   // no CTA leaves while another may still read its shared memory

    // ------------------------------------------------------------ results
    const VState st = s_st;
    if (rank == 0 && tid == 0) P.state[0] = st;
    const bool in_caller = C.final_mode && st.status == 0 && st.iter == C.n_steps;
    if (!in_caller) {
        // the stored iterate of the last completed step, where finish_kernel
        // looks for it
        const float* z = sm + ((st.iter & 1) ? L.zt1 : L.zt0);
        TS* Xo = (TS*)((st.iter & 1) ? C.buf1 : const_cast<void*>(C.buf0)) + g.off;
        for (long long i = tid; i < tile; i += NTH) {
            const int t = (int)(i / (th * TW)), r = (int)(i - (long long)t * th * TW);
            const int ly = r / TW, lx = r - ly * TW;
            const int yy = y0 + ly, xx = x0 + lx;
            if (yy < g.h && xx < g.w) Xo[(long long)t * g.plane + (long long)yy * g.pitch + xx] = from_f<TS>(z[i]);
        }
    }
}

template <int RT, int RY, int RX>
struct Inst {
    static const void* fn(int storage) {
        switch (storage) {
            case 0: return (const void*)step_cluster_kernel<RT, RY, RX, float>;
            case 1: return (const void*)step_cluster_kernel<RT, RY, RX, __nv_bfloat16>;
            case 2: return (const void*)step_cluster_kernel<RT, RY, RX, __half>;
        }
        return nullptr;
    }
    static clu::Strides strides() {
        using Q = Cfg<RT, RY, RX>;
        return clu::Strides{Q::YW, Q::PW, Q::YW2, Q::PW2};
    }
};

// the radii the cluster kernel is compiled for: (rt, ry, rx)
static bool lookup(int rt, int ry, int rx, int storage, const void** fn, Strides* st) {
#define SFSEG_CLU(A, B, D)                                        \
    if (rt == A && ry == B && rx == D) {                          \
        *fn = Inst<A, B, D>::fn(storage);                         \
        *st = Inst<A, B, D>::strides();                           \
        return *fn != nullptr;                                    \
    }
    SFSEG_CLU(3, 3, 3)
    SFSEG_CLU(2, 5, 5)
    SFSEG_CLU(2, 4, 4)
#undef SFSEG_CLU
    return false;
}

}  // namespace clu

SFSEG_DEBUG_TU(cluster)

// Plan of the cluster launch for one video (nf, h, w): 16-column tiles of
// th rows (a multiple of 8), the largest number of CTAs that is at most the
// device's cluster limit and whose shared memory fits; the launch
// configuration is checked with the occupancy API (the cluster must be
// schedulable).  Returns false when the video does not qualify.
bool plan_step_cluster(int storage, int rt, int ry, int rx, int nf, int h, int w, ClusterPlan* out) {
    const void* fn = nullptr;
    clu::Strides st{};
    if (!clu::lookup(rt, ry, rx, storage, &fn, &st)) return false;
    if (nf < 1 || h < 1 || w < 1) return false;
    int dev = 0, smem_optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return false;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int tiles_x = (w + clu::TW - 1) / clu::TW;
    ClusterPlan best{};
    bool found = false;
    for (int th = clu::RC; th <= 64; th += clu::RC) {
        const int tiles_y = (h + th - 1) / th;
        const int n = tiles_x * tiles_y;
        if (n > 16) continue;
        // the kernel's 32-bit reciprocal divisions need indices below 2^16
        const long long nh = 2ll * ry * (clu::TW + 2 * rx) + 2ll * th * rx;
        if ((long long)nf * nh + 8 * clu::NTH >= 65536 || (long long)nf * (th + 2 * ry) >= 65536) continue;
        const size_t bytes = clu::smem_bytes(nf, th, ry, rx, st);
        if (bytes + 1024 > (size_t)smem_optin) continue;   // plus the static shared variables
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(n);
        cfg.blockDim = dim3(clu::NTH);
        cfg.dynamicSmemBytes = bytes;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = n;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (clusters < 1) continue;
        if (!found || n > best.n_ctas) {
            best.n_ctas = n;
            best.tiles_x = tiles_x;
            best.th = th;
            best.smem = bytes;
            found = true;
        }
    }
    if (found) *out = best;
    return found;
}

cudaError_t launch_step_cluster(int storage, const ClusterParams& C, const ClusterPlan& plan, cudaStream_t s) {
    const void* fn = nullptr;
    clu::Strides st{};
    if (!clu::lookup(C.S.rt, C.S.ry, C.S.rx, storage, &fn, &st)) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(plan.n_ctas);
    cfg.blockDim = dim3(clu::NTH);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = plan.n_ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void* args[] = {const_cast<ClusterParams*>(&C)};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace sfseg
