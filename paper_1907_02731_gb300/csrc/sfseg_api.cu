// sfseg_api.cu -- the C-ABI of include/sfseg.h: context, validation, the
// iteration loop (replayed as a CUDA graph) and host-side bookkeeping.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include <nvtx3/nvToolsExt.h>

#include "sfseg.h"
#include "sfseg_launch.h"

// NVTX range around a public entry point (a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

using namespace sfseg;

struct sfseg_ctx {
    sfseg_params prm{};
    int nv = 0;
    bool batched = false;
    std::vector<VideoGeom> geo;
    long long total = 0;        // packed elements per volume array
    size_t elt = 4;
    // device workspace (owned)
    void* sp = nullptr;
    void* f = nullptr;
    void* xa = nullptr;
    void* xb = nullptr;
    VideoGeom* d_geo = nullptr;
    VState* d_state = nullptr;
    WorkItem* d_items = nullptr;
    int* d_item_begin = nullptr;
    double* d_partials = nullptr;
    unsigned* d_counters = nullptr;
    double* d_prep_partials = nullptr;
    unsigned* d_prep_counter = nullptr;
    int* d_bad = nullptr;
    double* d_trace = nullptr;
    int trace_cap = 0;
    float** d_out = nullptr;
    int n_items = 0;
    // specialised kernel: balanced segment lists and TMA descriptors
    bool fast = false;
    int n_ctas = 0;
    int* d_cta_begin = nullptr;
    int* d_vseg = nullptr;
    CUtensorMap* d_maps = nullptr;
    // generic tile plan (always built): the adjoint and its forward recompute
    WorkItem* d_gitems = nullptr;
    int* d_gitem_begin = nullptr;
    double* d_gpartials = nullptr;
    int g_n_items = 0;
    // forward record and adjoint workspace (allocated on first use)
    int rec_cap = 0;            // steps the record arrays hold
    double* d_rec = nullptr;    // [3][rec_cap + 1]: scale, gain, ny
    double* d_rrec = nullptr;   // the same for the backward's recompute
    int ckpt_cap = 0;
    void* d_ckpt = nullptr;     // [ckpt_cap] volumes: x^{j C} (and x^K last)
    // binarisation scratch (allocated on first use): 2 max keys + block partials
    unsigned char* d_bin = nullptr;
    // reverse step on the specialised kernel: scratch state, constants, partials
    unsigned char* d_adj_misc = nullptr;
    // test aid: step launches still to run with an injected device-side timeout
    int inject_steps = 0;
    // range of the loaded f per video and channel: float keys [nv][kMaxChan]
    unsigned* d_fmin = nullptr;
    unsigned* d_fmax = nullptr;
    void* d_adj = nullptr;      // [C + 4] volumes: recompute ring, g ping-pong, dsp, df
    int adj_cap = 0;
    double* d_adjc = nullptr;   // [2] dot products
    double* d_adj_partials = nullptr;
    unsigned* d_adj_counter = nullptr;
    bool recorded = false;
    int rec_K = 0;
    // step path of power_iterate: per-step specialised / per-step any-radius /
    // all steps in one cooperative launch (step_fused.cu)
    int path = SFSEG_PATH_FAST;
    bool tune_pending = false;  // SFSEG_AUTOTUNE: choose the path at the first power_iterate
    double tuned_us[4] = {-1.0, -1.0, -1.0, -1.0};   // measured us per step of each path (-1: not timed)
    // cluster path (step_cluster.cu): one small video resident in one cluster
    bool cluster_ok = false;
    ClusterPlan cplan{};
    // fused path: phase-2 runs, barrier words, scratch (allocated on first use)
    bool fused_ok = false;      // the context can run the fused kernel
    int fused_max = 0;          // co-resident CTAs of the fused kernel on this device
    int fused_ctas = 0;         // CTAs of the fused launch (the plan below is built for it)
    int fused_n_units1 = 0;
    int fused_n_items = 0;
    int* d_fu1 = nullptr;       // [nv + 1] phase-1 unit prefix
    WorkItem* d_fitems = nullptr;
    int* d_fcta_begin = nullptr;
    int* d_fitem_begin = nullptr;
    int* d_fvseg = nullptr;
    double* d_fpartials = nullptr;
    unsigned* d_fbar = nullptr; // [3]
    float* d_pvol = nullptr;    // 3 FP32 volumes
    // slab of a video split along t (sfseg_create_slab): own output frames
    // [own_lo, own_hi) of the context's volume, the voxel count of the whole
    // video (the gain rule), steps completed (parity of the stored iterate)
    bool slab = false;
    int own_lo = 0, own_hi = 0;
    long long video_voxels = 0;
    int slab_k = 0;
    float* slab_final = nullptr;   // the caller buffer the last slab step wrote in FP32
    std::vector<int> item_begin;
    // host-side
    float gt[2 * kMaxRt + 1], gy[2 * kMaxR + 1], gx[2 * kMaxR + 1];
    double gsum = 1.0;
    cudaStream_t cap_stream = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
    bool features = false;
    cudaStream_t last_stream = nullptr;
    long long launches = 0;
    std::string err;
};

static thread_local std::string g_create_err;

static sfseg_status fail(sfseg_ctx* c, sfseg_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_err = buf;
    return st;
}

#define CUDA_OR(ctx, call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? SFSEG_ENOMEM : SFSEG_ECUDA, \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

static sfseg_status validate(const sfseg_params* p) {
    if (!p) return fail(nullptr, SFSEG_EINVAL, "params is NULL");
    if (p->rt < 0 || p->rt > kMaxRt || p->ry < 0 || p->ry > kMaxR || p->rx < 0 || p->rx > kMaxR)
        return fail(nullptr, SFSEG_EINVAL, "radii (rt,ry,rx)=(%d,%d,%d) outside [0,%d]x[0,%d]x[0,%d]",
                    p->rt, p->ry, p->rx, kMaxRt, kMaxR, kMaxR);
    if (!finite_pos(p->sigma_t) || !finite_pos(p->sigma_y) || !finite_pos(p->sigma_x))
        return fail(nullptr, SFSEG_EINVAL, "sigmas must be finite and > 0");
    if (!std::isfinite(p->alpha) || p->alpha < 0.0)
        return fail(nullptr, SFSEG_EINVAL, "alpha must be finite and >= 0");
    if (!std::isfinite(p->p) || p->p < 0.0)
        return fail(nullptr, SFSEG_EINVAL, "p must be finite and >= 0");
    if (p->storage < 0 || p->storage > 2)
        return fail(nullptr, SFSEG_EINVAL, "storage %d is not an sfseg_dtype", p->storage);
    if (p->flags & ~(SFSEG_S_IS_SP | SFSEG_NO_GRAPH | SFSEG_RECORD | SFSEG_GENERIC | SFSEG_FUSED |
                     SFSEG_AUTOTUNE | SFSEG_CLUSTER))
        return fail(nullptr, SFSEG_EINVAL, "flags 0x%x: unknown bits", (unsigned)p->flags);
    if ((p->flags & SFSEG_CLUSTER) && (p->flags & (SFSEG_GENERIC | SFSEG_FUSED | SFSEG_AUTOTUNE)))
        return fail(nullptr, SFSEG_EINVAL, "SFSEG_CLUSTER excludes SFSEG_GENERIC, SFSEG_FUSED and SFSEG_AUTOTUNE");
    if ((p->flags & SFSEG_CLUSTER) && (p->flags & SFSEG_RECORD))
        return fail(nullptr, SFSEG_EUNSUPPORTED, "SFSEG_RECORD runs the per-step kernel (no SFSEG_CLUSTER)");
    if ((p->flags & SFSEG_CLUSTER) && p->nchan != 1)
        return fail(nullptr, SFSEG_EUNSUPPORTED, "the cluster kernel runs one channel (nchan = 1)");
    if ((p->flags & SFSEG_FUSED) && (p->flags & (SFSEG_GENERIC | SFSEG_AUTOTUNE)))
        return fail(nullptr, SFSEG_EINVAL, "SFSEG_FUSED excludes SFSEG_GENERIC and SFSEG_AUTOTUNE");
    if ((p->flags & (SFSEG_FUSED | SFSEG_AUTOTUNE)) && (p->flags & SFSEG_RECORD))
        return fail(nullptr, SFSEG_EUNSUPPORTED,
                    "SFSEG_RECORD runs the per-step kernel (no SFSEG_FUSED / SFSEG_AUTOTUNE)");
    if ((p->flags & SFSEG_FUSED) && p->nchan != 1)
        return fail(nullptr, SFSEG_EUNSUPPORTED, "the fused kernel runs one channel (nchan = 1)");
    if (p->nchan < 1 || p->nchan > 8)
        return fail(nullptr, SFSEG_EINVAL, "nchan %d outside [1, 8]", p->nchan);
    if (p->nchan > kMaxChan)
        return fail(nullptr, SFSEG_EUNSUPPORTED, "nchan %d: at most %d channels are built", p->nchan, kMaxChan);
    if (generic_smem_bytes(p->rt, p->ry, p->rx, p->nchan) > generic_smem_cap())
        return fail(nullptr, SFSEG_EUNSUPPORTED,
                    "nchan %d with radii (%d,%d,%d): the step's buffers exceed shared memory", p->nchan,
                    p->rt, p->ry, p->rx);
    if (p->ckpt_every < 0) return fail(nullptr, SFSEG_EINVAL, "ckpt_every must be >= 0");
    return SFSEG_OK;
}

namespace sfseg {
sfseg_status validate_params(const sfseg_params* p) { return validate(p); }
void set_global_error(const char* msg) { g_create_err = msg ? msg : ""; }
}  // namespace sfseg

static void free_ctx(sfseg_ctx* c) {
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
    void* ptrs[] = {c->sp, c->f, c->xa, c->xb, c->d_geo, c->d_state, c->d_items, c->d_item_begin,
                    c->d_partials, c->d_counters, c->d_prep_partials, c->d_prep_counter, c->d_bad,
                    c->d_trace, c->d_out, c->d_cta_begin, c->d_vseg, c->d_maps,
                    c->d_gitems, c->d_gitem_begin, c->d_gpartials, c->d_rec, c->d_rrec,
                    c->d_ckpt, c->d_adj, c->d_adjc, c->d_adj_partials, c->d_adj_counter, c->d_bin,
                    c->d_adj_misc, c->d_fmin, c->d_fmax, c->d_fu1, c->d_fitems, c->d_fcta_begin,
                    c->d_fitem_begin, c->d_fvseg, c->d_fpartials, c->d_fbar, c->d_pvol};
    for (void* p : ptrs) if (p) cudaFree(p);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

static void host_taps(int r, double sigma, float* g, double* sum) {
    double s = 0.0;
    for (int d = -r; d <= r; ++d) {
        const double v = std::exp(-(double)d * d / (2.0 * sigma * sigma));
        g[d + r] = (float)v;
        s += (double)(float)v;
    }
    *sum *= s;
}

// Work decomposition of the specialised kernel.  Units = output frames of
// (video, tile) pairs.  n_ctas = min(sms, units / 8).  Per video, while at
// least n_ctas of its tiles remain, a round gives CTA c one whole tile (all
// CTAs stream their tiles in step, so the halo rows one CTA loads are still
// in L2 when its neighbours need them); the units of every video's last
// < n_ctas tiles are laid end to end and cut into n_ctas equal contiguous
// ranges.  Outputs: segments
// ordered by CTA, cta_begin, and per-video segment id lists (vseg /
// item_begin) for the finalize.
static void build_segments(const std::vector<VideoGeom>& geo, int sms, std::vector<WorkItem>* items,
                           std::vector<int>* item_begin, std::vector<int>* cta_begin,
                           std::vector<int>* vseg, int f_lo = 0, int f_hi = -1) {
    // output frames [f_lo, f_hi) of every video (f_hi < 0: all frames); a
    // slab of a video split along t computes its own frames only
    int tx, ty, nt;
    fast_tile(&tx, &ty, &nt);
    struct Tile { int v, x0, y0, nf; };
    auto fr0 = [&](const VideoGeom& g) { return f_lo < g.nf ? f_lo : g.nf; };
    auto fr1 = [&](const VideoGeom& g) { return f_hi < 0 || f_hi > g.nf ? g.nf : f_hi; };
    long long U = 0;
    for (const VideoGeom& g : geo)
        U += (long long)(fr1(g) - fr0(g)) * ((g.w + tx - 1) / tx) * ((g.h + ty - 1) / ty);
    long long n = U / 8;                      // at least ~8 output frames per CTA
    if (n > sms) n = sms;
    if (n < 1) n = 1;
    // whole-tile rounds per video (every tile of a round has the same frame
    // count, so each round adds the same work to every CTA); leftovers of all
    // videos go to the even split
    std::vector<std::vector<WorkItem>> per(n);
    std::vector<Tile> tiles;   // leftovers
    for (int v = 0; v < (int)geo.size(); ++v) {
        const VideoGeom& g = geo[v];
        std::vector<Tile> tv;
        for (int y0 = 0; y0 < g.h; y0 += ty)
            for (int x0 = 0; x0 < g.w; x0 += tx) tv.push_back({v, x0, y0, fr1(g) - fr0(g)});
        const size_t whole = tv.size() / (size_t)n * (size_t)n;
        for (size_t k = 0; k < whole; ++k) {
            WorkItem it{};
            it.video = v;
            it.x0 = tv[k].x0;
            it.y0 = tv[k].y0;
            it.t0 = fr0(g);
            it.t1 = fr1(g);
            per[k % n].push_back(it);
        }
        tiles.insert(tiles.end(), tv.begin() + whole, tv.end());
    }
    long long U2 = 0;
    for (const Tile& t : tiles) U2 += t.nf;
    long long pos = 0, cur = 0;
    for (size_t k = 0; k < tiles.size(); ++k) {
        const long long end_tile = pos + tiles[k].nf;
        long long t = pos;
        while (t < end_tile) {
            while (cur + 1 < n && U2 * (cur + 1) / n <= t) ++cur;
            const long long cut = U2 * (cur + 1) / n;
            const long long e = end_tile < cut ? end_tile : cut;
            WorkItem it{};
            it.video = tiles[k].v;
            it.x0 = tiles[k].x0;
            it.y0 = tiles[k].y0;
            it.t0 = fr0(geo[tiles[k].v]) + (int)(t - pos);
            it.t1 = fr0(geo[tiles[k].v]) + (int)(e - pos);
            per[cur].push_back(it);
            t = e;
        }
        pos = end_tile;
    }
    cta_begin->assign(n + 1, 0);
    for (long long c = 0; c < n; ++c) {
        (*cta_begin)[c] = (int)items->size();
        items->insert(items->end(), per[c].begin(), per[c].end());
    }
    (*cta_begin)[n] = (int)items->size();
    vseg->clear();
    item_begin->clear();
    for (int v = 0; v < (int)geo.size(); ++v) {
        item_begin->push_back((int)vseg->size());
        for (int i = 0; i < (int)items->size(); ++i)
            if ((*items)[i].video == v) vseg->push_back(i);
    }
    item_begin->push_back((int)vseg->size());
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// One 3D tiled descriptor per (video, array): dims (w, h, nf) so the TMA box
// reads zeros outside the volume, row/plane strides of the pitched layout.
static const char* encode_maps(sfseg_ctx* c, CUtensorMap* maps) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return "cuTensorMapEncodeTiled unavailable";
    int bw, bh, xpad;
    fast_box(c->prm.ry, &bw, &bh, &xpad);
    const CUtensorMapDataType dt = c->prm.storage == SFSEG_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : c->prm.storage == SFSEG_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                                  : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    void* arrays[kMapsPerVideo] = {c->sp, c->f, c->xa, c->xb};
    for (int ch = 1; ch < c->prm.nchan; ++ch) arrays[3 + ch] = (char*)c->f + (size_t)ch * c->total * c->elt;
    const int n_arrays = 3 + c->prm.nchan;
    for (int v = 0; v < c->nv; ++v) {
        const VideoGeom& g = c->geo[v];
        cuuint64_t gdim[3] = {(cuuint64_t)g.w, (cuuint64_t)g.h, (cuuint64_t)g.nf};
        cuuint64_t gstr[2] = {(cuuint64_t)g.pitch * c->elt, (cuuint64_t)g.plane * c->elt};
        cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1u};
        cuuint32_t est[3] = {1u, 1u, 1u};
        for (int a = 0; a < n_arrays; ++a) {
            void* base = (char*)arrays[a] + (size_t)g.off * c->elt;
            CUresult r = enc(&maps[kMapsPerVideo * v + a], dt, 3, base, gdim, gstr, box, est,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return "cuTensorMapEncodeTiled failed";
        }
    }
    return nullptr;
}

// Work plan of the fused kernel for G CTAs.  Phase 1: per video, frames x
// 32x16 tiles (unit1_begin = prefix over videos; CTAs stride over them).
// Phase 2: per video, frames x chunks of fused_rows2(w) rows, laid end to end
// over all videos and cut into G equal contiguous ranges; a range's units of
// one video form one item (a run that arrives once at the finalize).
struct FusedPlan {
    std::vector<int> unit1_begin;
    std::vector<WorkItem> items;
    std::vector<int> cta_begin, item_begin, vseg;
};

static long long fused_units2(const VideoGeom& g) {
    const int rows = fused_rows2(g.w);
    return (long long)g.nf * ((g.h + rows - 1) / rows);
}

static void build_fused_plan(const std::vector<VideoGeom>& geo, int G, FusedPlan* fp) {
    int tx, ty, nt;
    fused_tile(&tx, &ty, &nt);
    fp->unit1_begin.assign(1, 0);
    for (const VideoGeom& g : geo)
        fp->unit1_begin.push_back(fp->unit1_begin.back() +
                                  g.nf * ((g.h + ty - 1) / ty) * ((g.w + tx - 1) / tx));
    std::vector<long long> u2b(1, 0);
    for (const VideoGeom& g : geo) u2b.push_back(u2b.back() + fused_units2(g));
    const long long U2 = u2b.back();
    fp->items.clear();
    fp->cta_begin.assign(G + 1, 0);
    int v = 0;
    for (int c = 0; c < G; ++c) {
        fp->cta_begin[c] = (int)fp->items.size();
        long long a = U2 * c / G;
        const long long b = U2 * (c + 1) / G;
        while (a < b) {
            while (u2b[v + 1] <= a) ++v;
            const long long e = b < u2b[v + 1] ? b : u2b[v + 1];
            WorkItem it{};
            it.video = v;
            it.t0 = (int)(a - u2b[v]);
            it.t1 = (int)(e - u2b[v]);
            fp->items.push_back(it);
            a = e;
        }
    }
    fp->cta_begin[G] = (int)fp->items.size();
    fp->vseg.clear();
    fp->item_begin.clear();
    for (int w = 0; w < (int)geo.size(); ++w) {
        fp->item_begin.push_back((int)fp->vseg.size());
        for (int i = 0; i < (int)fp->items.size(); ++i)
            if (fp->items[i].video == w) fp->vseg.push_back(i);
    }
    fp->item_begin.push_back((int)fp->vseg.size());
}

// CTAs worth launching: one per phase-1 unit plus one spare per video (the
// last CTAs run the videos' scalar updates while the others filter the next
// step), or one per phase-2 unit if more; no more than the resident maximum.
static int fused_default_ctas(const sfseg_ctx* c) {
    int tx, ty, nt;
    fused_tile(&tx, &ty, &nt);
    long long u1 = 0, u2 = 0;
    for (const VideoGeom& g : c->geo) {
        u1 += (long long)g.nf * ((g.h + ty - 1) / ty) * ((g.w + tx - 1) / tx);
        u2 += fused_units2(g);
    }
    u1 += c->nv;
    long long n = u1 > u2 ? u1 : u2;
    if (n > c->fused_max) n = c->fused_max;
    return n < 1 ? 1 : (int)n;
}

// Upload the fused plan for G CTAs (host-synchronous; never during a capture).
static cudaError_t upload_fused_plan(sfseg_ctx* c, int G) {
    FusedPlan fp;
    build_fused_plan(c->geo, G, &fp);
    cudaError_t e = cudaMemcpy(c->d_fu1, fp.unit1_begin.data(), sizeof(int) * fp.unit1_begin.size(),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_fitems, fp.items.data(), sizeof(WorkItem) * fp.items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_fcta_begin, fp.cta_begin.data(), sizeof(int) * fp.cta_begin.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_fitem_begin, fp.item_begin.data(), sizeof(int) * fp.item_begin.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !fp.vseg.empty())
        e = cudaMemcpy(c->d_fvseg, fp.vseg.data(), sizeof(int) * fp.vseg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        c->fused_ctas = G;
        c->fused_n_units1 = fp.unit1_begin.back();
        c->fused_n_items = (int)fp.items.size();
    }
    return e;
}

static sfseg_status create_impl(const sfseg_params* prm, int nv, const int32_t* dims, bool batched,
                                sfseg_ctx** out, int f_lo = 0, int f_hi = -1) {
    if (!out) return fail(nullptr, SFSEG_EINVAL, "out is NULL");
    *out = nullptr;
    sfseg_status st = validate(prm);
    if (st != SFSEG_OK) return st;
    if (nv < 1) return fail(nullptr, SFSEG_EINVAL, "n_videos must be >= 1");
    for (int v = 0; v < nv; ++v)
        if (dims[3 * v] < 1 || dims[3 * v + 1] < 1 || dims[3 * v + 2] < 1)
            return fail(nullptr, SFSEG_EINVAL, "video %d: dims (%d,%d,%d) must be >= 1", v,
                        dims[3 * v], dims[3 * v + 1], dims[3 * v + 2]);
    sfseg_ctx* c = new sfseg_ctx();
    c->prm = *prm;
    c->nv = nv;
    c->batched = batched;
    c->elt = prm->storage == SFSEG_F32 ? 4 : 2;
    const long long align = 256 / (long long)c->elt;
    long long off = 0;
    for (int v = 0; v < nv; ++v) {
        VideoGeom g;
        g.nf = dims[3 * v];
        g.h = dims[3 * v + 1];
        g.w = dims[3 * v + 2];
        g.pitch = (g.w + 7) / 8 * 8;
        g.plane = (long long)g.h * g.pitch;
        g.off = off;
        g.n = (long long)g.nf * g.h * g.w;
        off += (g.nf * g.plane + align - 1) / align * align;
        c->geo.push_back(g);
    }
    // several channels run as one pass per channel, with FP32 partial sums
    c->fast = !(prm->flags & SFSEG_GENERIC) && (prm->nchan == 1 || prm->storage == SFSEG_F32) &&
              fast_available(prm->rt, prm->ry, prm->rx, prm->storage);
    std::vector<WorkItem> items;
    std::vector<int> cta_begin, vseg;
    if (c->fast) {
        int sms = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
        build_segments(c->geo, sms, &items, &c->item_begin, &cta_begin, &vseg, f_lo, f_hi);
        c->n_ctas = (int)cta_begin.size() - 1;
    }
    std::vector<WorkItem> gitems;
    std::vector<int> gitem_begin;
    {
        int tx, ty;
        generic_tile(&tx, &ty);
        for (int v = 0; v < nv; ++v) {
            const VideoGeom& g = c->geo[v];
            gitem_begin.push_back((int)gitems.size());
            for (int y0 = 0; y0 < g.h; y0 += ty)
                for (int x0 = 0; x0 < g.w; x0 += tx) {
                    WorkItem it{};
                    it.video = v;
                    it.x0 = x0;
                    it.y0 = y0;
                    it.t0 = f_lo;
                    it.t1 = f_hi < 0 ? g.nf : f_hi;
                    gitems.push_back(it);
                }
        }
        gitem_begin.push_back((int)gitems.size());
        c->g_n_items = (int)gitems.size();
    }
    if (!c->fast) {
        int tx, ty;
        generic_tile(&tx, &ty);
        for (int v = 0; v < nv; ++v) {
            const VideoGeom& g = c->geo[v];
            c->item_begin.push_back((int)items.size());
            for (int y0 = 0; y0 < g.h; y0 += ty)
                for (int x0 = 0; x0 < g.w; x0 += tx) {
                    WorkItem it{};
                    it.video = v;
                    it.x0 = x0;
                    it.y0 = y0;
                    it.t0 = f_lo;
                    it.t1 = f_hi < 0 ? g.nf : f_hi;
                    items.push_back(it);
                }
        }
        c->item_begin.push_back((int)items.size());
    }
    c->total = off;
    c->n_items = (int)items.size();
    c->gsum = 1.0;
    host_taps(prm->rt, prm->sigma_t, c->gt, &c->gsum);
    host_taps(prm->ry, prm->sigma_y, c->gy, &c->gsum);
    host_taps(prm->rx, prm->sigma_x, c->gx, &c->gsum);

#define ALLOC(ptr, bytes)                                                                 \
    do {                                                                                  \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                             \
        if (e_ != cudaSuccess) {                                                          \
            fail(nullptr, SFSEG_ENOMEM, "cudaMalloc(%zu): %s", (size_t)(bytes),           \
                 cudaGetErrorString(e_));                                                 \
            free_ctx(c);                                                                  \
            return SFSEG_ENOMEM;                                                          \
        }                                                                                 \
    } while (0)
    const size_t vol = (size_t)c->total * c->elt;
    ALLOC(c->sp, vol);
    ALLOC(c->f, vol * prm->nchan);
    ALLOC(c->xa, vol);
    ALLOC(c->xb, vol);
    ALLOC(c->d_geo, sizeof(VideoGeom) * nv);
    ALLOC(c->d_state, sizeof(VState) * nv);
    ALLOC(c->d_items, sizeof(WorkItem) * items.size());
    ALLOC(c->d_item_begin, sizeof(int) * (nv + 1));
    ALLOC(c->d_partials, sizeof(double) * kRed * items.size());
    ALLOC(c->d_counters, sizeof(unsigned) * nv);
    ALLOC(c->d_prep_partials, sizeof(double) * prep_x_blocks(1LL << 40));
    ALLOC(c->d_prep_counter, sizeof(unsigned));
    ALLOC(c->d_bad, sizeof(int));
    ALLOC(c->d_out, sizeof(float*) * nv);
    ALLOC(c->d_fmin, sizeof(unsigned) * kMaxChan * nv);
    ALLOC(c->d_fmax, sizeof(unsigned) * kMaxChan * nv);
    ALLOC(c->d_gitems, sizeof(WorkItem) * gitems.size());
    ALLOC(c->d_gitem_begin, sizeof(int) * gitem_begin.size());
    ALLOC(c->d_gpartials, sizeof(double) * kRed * gitems.size());
    if (c->fast) {
        ALLOC(c->d_cta_begin, sizeof(int) * cta_begin.size());
        ALLOC(c->d_vseg, sizeof(int) * (vseg.size() + 1));
        ALLOC(c->d_maps, sizeof(CUtensorMap) * kMapsPerVideo * nv);
    }
#undef ALLOC
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemset(c->sp, 0, vol);
    if (e == cudaSuccess) e = cudaMemset(c->f, 0, vol * prm->nchan);
    if (e == cudaSuccess) e = cudaMemset(c->xa, 0, vol);
    if (e == cudaSuccess) e = cudaMemset(c->xb, 0, vol);
    if (e == cudaSuccess) e = cudaMemset(c->d_state, 0, sizeof(VState) * nv);
    if (e == cudaSuccess) e = cudaMemset(c->d_counters, 0, sizeof(unsigned) * nv);
    if (e == cudaSuccess) e = cudaMemset(c->d_prep_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(c->d_bad, 0, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_geo, c->geo.data(), sizeof(VideoGeom) * nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_items, items.data(), sizeof(WorkItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_item_begin, c->item_begin.data(), sizeof(int) * (nv + 1),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_gitems, gitems.data(), sizeof(WorkItem) * gitems.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_gitem_begin, gitem_begin.data(), sizeof(int) * gitem_begin.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = setup_step_generic(prm->rt, prm->ry, prm->rx);
    if (e == cudaSuccess && prm->nchan == 1 && !(prm->flags & SFSEG_RECORD) && f_lo == 0 && f_hi < 0) {
        // fused path: its plan arrays hold the largest plan (one item per CTA
        // and video boundary); the scratch volumes are allocated on first use
        e = setup_step_fused(prm->storage, prm->ry, prm->rx, &c->fused_max);
        if (e == cudaSuccess && c->fused_max > 0) {
            const size_t cap = (size_t)c->fused_max + nv;
            e = cudaMalloc((void**)&c->d_fu1, sizeof(int) * (nv + 1));
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_fitems, sizeof(WorkItem) * cap);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_fcta_begin, sizeof(int) * (c->fused_max + 1));
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_fitem_begin, sizeof(int) * (nv + 1));
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_fvseg, sizeof(int) * cap);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_fpartials, sizeof(double) * kRed * cap);
            if (e == cudaSuccess) e = cudaMalloc((void**)&c->d_fbar, sizeof(unsigned) * 3);
            if (e == cudaSuccess) e = upload_fused_plan(c, fused_default_ctas(c));
            if (e == cudaSuccess) c->fused_ok = true;
        }
    }
    if (e == cudaSuccess && nv == 1 && prm->nchan == 1 && !(prm->flags & SFSEG_RECORD) && f_lo == 0 && f_hi < 0)
        c->cluster_ok = plan_step_cluster(prm->storage, prm->rt, prm->ry, prm->rx, c->geo[0].nf, c->geo[0].h,
                                          c->geo[0].w, &c->cplan);
    c->path = c->fast ? SFSEG_PATH_FAST : SFSEG_PATH_GENERIC;
    if (e == cudaSuccess && (prm->flags & SFSEG_CLUSTER)) {
        if (!c->cluster_ok) {
            fail(nullptr, SFSEG_EUNSUPPORTED,
                 "SFSEG_CLUSTER: needs one video, radii (3,3,3), (2,5,5) or (2,4,4), at most 16 tiles of 16 "
                 "columns whose frames fit one CTA's shared memory, and a device that schedules the cluster");
            free_ctx(c);
            return SFSEG_EUNSUPPORTED;
        }
        c->path = SFSEG_PATH_CLUSTER;
    }
    if (e == cudaSuccess && (prm->flags & SFSEG_FUSED)) {
        if (!c->fused_ok) {
            fail(nullptr, SFSEG_EUNSUPPORTED, "SFSEG_FUSED: this device has no cooperative launch");
            free_ctx(c);
            return SFSEG_EUNSUPPORTED;
        }
        c->path = SFSEG_PATH_FUSED;
    }
    c->tune_pending = (prm->flags & SFSEG_AUTOTUNE) != 0;
    if (e == cudaSuccess && c->fast) {
        e = setup_step_fast(prm->rt, prm->ry, prm->rx, prm->storage);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_cta_begin, cta_begin.data(), sizeof(int) * cta_begin.size(),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !vseg.empty())
            e = cudaMemcpy(c->d_vseg, vseg.data(), sizeof(int) * vseg.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            std::vector<CUtensorMap> maps(kMapsPerVideo * (size_t)nv);
            const char* why = encode_maps(c, maps.data());
            if (why) {
                fail(nullptr, SFSEG_ECUDA, "tensor map: %s", why);
                free_ctx(c);
                return SFSEG_ECUDA;
            }
            e = cudaMemcpy(c->d_maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                           cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        fail(nullptr, SFSEG_ECUDA, "context set-up: %s", cudaGetErrorString(e));
        free_ctx(c);
        return SFSEG_ECUDA;
    }
    *out = c;
    return SFSEG_OK;
}

static sfseg_status ensure_trace(sfseg_ctx* c, int K) {
    if (K <= c->trace_cap) return SFSEG_OK;
    int cap = c->trace_cap ? c->trace_cap : 64;
    while (cap < K) cap *= 2;
    double* t = nullptr;
    CUDA_OR(c, cudaDeviceSynchronize());
    CUDA_OR(c, cudaMalloc((void**)&t, sizeof(double) * 3 * (size_t)cap * c->nv));
    CUDA_OR(c, cudaMemset(t, 0, sizeof(double) * 3 * (size_t)cap * c->nv));
    if (c->d_trace) cudaFree(c->d_trace);
    c->d_trace = t;
    c->trace_cap = cap;
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);   // they captured the old pointer
    c->graphs.clear();
    return SFSEG_OK;
}

static StepParams step_params(sfseg_ctx* c, int k, bool final_out, bool store,
                              bool record = false) {
    StepParams P{};
    P.x_in = (k & 1) ? c->xb : c->xa;
    P.z_out = (store && !final_out) ? ((k & 1) ? c->xa : c->xb) : nullptr;
    P.final_out = final_out ? c->d_out : nullptr;
    P.sp = c->sp;
    P.f = c->f;
    P.geo = c->d_geo;
    P.state = c->d_state;
    P.items = c->d_items;
    P.item_begin = c->d_item_begin;
    P.partials = c->d_partials;
    P.counters = c->d_counters;
    P.trace = c->d_trace;
    P.trace_cap = c->trace_cap;
    P.n_items = c->n_items;
    P.alpha = (float)c->prm.alpha;
    P.rt = c->prm.rt;
    P.ry = c->prm.ry;
    P.rx = c->prm.rx;
    memcpy(P.gt, c->gt, sizeof c->gt);
    memcpy(P.gy, c->gy, sizeof c->gy);
    memcpy(P.gx, c->gx, sizeof c->gx);
    P.nchan = c->prm.nchan;
    P.fstride = c->total;
    P.n_videos = c->nv;
    P.total = c->total;
    for (int d = 0; d < 2 * kMaxRt + 1; ++d) P.gt2[d] = make_float2(P.gt[d], P.gt[d]);
    for (int d = 0; d < 2 * kMaxR + 1; ++d) {
        P.gy2[d] = make_float2(P.gy[d], P.gy[d]);
        P.gx2[d] = make_float2(P.gx[d], -2.f * P.gx[d]);   // channel b carries -2 (exact)
    }
    P.maps = c->d_maps;
    P.x_sel = k & 1;
    P.cta_begin = c->d_cta_begin;
    P.vseg = c->d_vseg;
    if (record && c->d_rec) {
        P.rec.scale = c->d_rec;
        P.rec.gain = c->d_rec + (c->rec_cap + 1);
        P.rec.ny = c->d_rec + 2 * (c->rec_cap + 1);
    }
    return P;
}

static cudaError_t launch_step(sfseg_ctx* c, int k, bool final_out, bool store, cudaStream_t s,
                               bool record = false, double* ext_sums = nullptr) {
    StepParams P = step_params(c, k, final_out, store, record);
    P.ext_sums = ext_sums;
    if (c->inject_steps > 0) {
        P.inject_timeout = 1;
        c->inject_steps -= 1;
    }
    c->launches += 1;
    const bool fast = c->fast && c->path != SFSEG_PATH_GENERIC;
    if (!fast) {   // the any-radius kernel on its own tile plan
        P.items = c->d_gitems;
        P.item_begin = c->d_gitem_begin;
        P.partials = c->d_gpartials;
        P.vseg = nullptr;
        P.n_items = c->g_n_items;
        return launch_step_generic(c->prm.storage, P, c->g_n_items, s);
    }
    if (c->prm.nchan > 1) {
        // Eq. 9 as one pass per channel: every pass adds its M_c x to the
        // partial sum in the step's output buffer; the last pass also reduces
        // (and writes the caller's buffer in final mode)
        void* zbuf = (k & 1) ? c->xa : c->xb;
        const int C = c->prm.nchan;
        for (int ch = 0; ch < C; ++ch) {
            StepParams Q = P;
            Q.f_chan = ch;
            Q.acc_in = ch > 0 ? zbuf : nullptr;
            Q.no_reduce = ch < C - 1 ? 1 : 0;
            if (ch < C - 1) {
                Q.z_out = zbuf;
                Q.final_out = nullptr;
            }
            if (ch < C - 1 && Q.inject_timeout) Q.inject_timeout = 0;
            cudaError_t e = launch_step_fast(c->prm.storage, Q, c->n_ctas, s);
            if (e != cudaSuccess) return e;
        }
        c->launches += C - 1;
        return cudaSuccess;
    }
    return launch_step_fast(c->prm.storage, P, c->n_ctas, s);
}

// All n power steps of a call in one cooperative launch (step_fused.cu).  The
// last step writes the caller's FP32 buffers when final_mode is set (the
// pointer table d_out must hold them).
static sfseg_status run_fused(sfseg_ctx* c, int n, bool final_mode, cudaStream_t s) {
    if (n <= 0) return SFSEG_OK;
    if (!c->d_pvol)
        CUDA_OR(c, cudaMalloc((void**)&c->d_pvol, sizeof(float) * 3 * (size_t)c->total));
    FusedParams F{};
    F.S = step_params(c, 0, final_mode, true);
    F.S.items = c->d_fitems;
    F.S.cta_begin = c->d_fcta_begin;
    F.S.item_begin = c->d_fitem_begin;
    F.S.vseg = c->d_fvseg;
    F.S.partials = c->d_fpartials;
    F.S.n_items = c->fused_n_items;
    if (c->inject_steps > 0) {
        F.S.inject_timeout = 1;
        c->inject_steps = 0;
    }
    F.buf0 = c->xa;
    F.buf1 = c->xb;
    F.pvol = c->d_pvol;
    F.total = c->total;
    F.unit1_begin = c->d_fu1;
    F.n_units1 = c->fused_n_units1;
    F.n_videos = c->nv;
    F.n_steps = n;
    F.final_mode = final_mode ? 1 : 0;
    F.bar = c->d_fbar;
    CUDA_OR(c, cudaMemsetAsync(c->d_fbar, 0, sizeof(unsigned) * 3, s));
    CUDA_OR(c, launch_step_fused(c->prm.storage, F, c->fused_ctas, s));
    c->launches += 1;
    return SFSEG_OK;
}

// All n power steps of a call in one cluster launch (step_cluster.cu); the
// last step writes the caller's FP32 buffer when final_mode is set.
static sfseg_status run_cluster(sfseg_ctx* c, int n, bool final_mode, cudaStream_t s) {
    if (n <= 0) return SFSEG_OK;
    ClusterParams C{};
    C.S = step_params(c, 0, final_mode, true);
    C.buf0 = c->xa;
    C.buf1 = c->xb;
    C.n_steps = n;
    C.final_mode = final_mode ? 1 : 0;
    C.tiles_x = c->cplan.tiles_x;
    C.th = c->cplan.th;
    CUDA_OR(c, launch_step_cluster(c->prm.storage, C, c->cplan, s));
    c->launches += 1;
    return SFSEG_OK;
}

// Steps [0, n) that store into the internal ping-pong buffers: one CUDA
// graph per n, captured on the context's own stream and replayed on the
// caller's stream.
static sfseg_status run_steps(sfseg_ctx* c, int n, cudaStream_t s) {
    if (n <= 0) return SFSEG_OK;
    if ((c->prm.flags & SFSEG_NO_GRAPH) || c->inject_steps > 0) {   // an injection is never captured
        for (int k = 0; k < n; ++k) CUDA_OR(c, launch_step(c, k, false, true, s));
        return SFSEG_OK;
    }
    auto it = c->graphs.find(n);
    if (it == c->graphs.end()) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const long long before = c->launches;
        CUDA_OR(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = cudaSuccess;
        for (int k = 0; k < n && le == cudaSuccess; ++k) le = launch_step(c, k, false, true, c->cap_stream);
        cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
        c->launches = before;
        if (le != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(c, SFSEG_ECUDA, "graph capture: %s / %s", cudaGetErrorString(le),
                        cudaGetErrorString(ee));
        }
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return fail(c, SFSEG_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
        if (c->graphs.size() >= 16) {
            cudaGraphExecDestroy(c->graphs.begin()->second);
            c->graphs.erase(c->graphs.begin());
        }
        it = c->graphs.emplace(n, exec).first;
    }
    CUDA_OR(c, cudaGraphLaunch(it->second, s));
    c->launches += n;
    return SFSEG_OK;
}

static sfseg_status load_features_impl(sfseg_ctx* c, const float* const* d_s, const float* const* d_f,
                                       cudaStream_t s) {
    for (int v = 0; v < c->nv; ++v)
        if (!d_s[v] || !d_f[v]) return fail(c, SFSEG_EINVAL, "video %d: NULL feature pointer", v);
    CUDA_OR(c, cudaMemsetAsync(c->d_bad, 0, sizeof(int), s));
    for (int v = 0; v < c->nv; ++v) {
        PrepFeatParams P{};
        P.s = d_s[v];
        P.f = d_f[v];
        P.sp_out = c->sp;
        P.f_out = c->f;
        P.chan_stride = c->total;
        P.g = c->geo[v];
        P.nchan = c->prm.nchan;
        P.p = (float)c->prm.p;
        P.s_is_sp = (c->prm.flags & SFSEG_S_IS_SP) ? 1 : 0;
        P.bad = c->d_bad;
        P.fmin_key = c->d_fmin + kMaxChan * v;
        P.fmax_key = c->d_fmax + kMaxChan * v;
        CUDA_OR(c, cudaMemsetAsync(P.fmin_key, 0xff, sizeof(unsigned) * kMaxChan, s));
        CUDA_OR(c, cudaMemsetAsync(P.fmax_key, 0, sizeof(unsigned) * kMaxChan, s));
        CUDA_OR(c, launch_prep_features(c->prm.storage, P, s));
        c->launches += 1;
    }
    c->features = true;
    return SFSEG_OK;
}

static sfseg_status prep_x(sfseg_ctx* c, int v, const float* d_x, bool raw, double tol, cudaStream_t s,
                           double* rec_scale0 = nullptr, double* ext_sum = nullptr) {
    PrepXParams P{};
    P.ext_sum = ext_sum;
    P.norm_t0 = c->own_lo;
    P.norm_t1 = c->own_hi;
    P.rec_scale0 = rec_scale0;
    P.x = d_x;
    P.x_out = c->xa;
    P.g = c->geo[v];
    P.video = v;
    P.raw = raw ? 1 : 0;
    P.gain0 = std::exp2(std::rint(std::log2(std::sqrt((double)c->geo[v].n) / c->gsum)));
    P.tol = tol;
    P.bad_features = c->d_bad;
    P.state = c->d_state;
    P.partials = c->d_prep_partials;
    P.counter = c->d_prep_counter;
    // a step whose CTAs gave up (SFSEG_ETIMEOUT) left its arrival count
    // unfinished: every call starts the video's count from zero
    CUDA_OR(c, cudaMemsetAsync(c->d_counters + v, 0, sizeof(unsigned), s));
    CUDA_OR(c, launch_prep_x(c->prm.storage, P, prep_x_blocks(c->geo[v].n), s));
    c->launches += 1;
    return SFSEG_OK;
}

static sfseg_status device_status(sfseg_ctx* c, cudaStream_t s, std::vector<VState>* out) {
    std::vector<VState> st(c->nv);
    CUDA_OR(c, cudaStreamSynchronize(s));
    CUDA_OR(c, cudaMemcpy(st.data(), c->d_state, sizeof(VState) * c->nv, cudaMemcpyDeviceToHost));
    if (out) *out = st;
    for (int v = 0; v < c->nv; ++v)
        if (st[v].status != 0)
            return fail(c, (sfseg_status)st[v].status, "video %d: %s at step %d", v,
                        sfseg_status_string((sfseg_status)st[v].status), st[v].iter);
    return SFSEG_OK;
}

static size_t vol_bytes(const sfseg_ctx* c) { return (size_t)c->total * c->elt; }

static sfseg_status ensure_record(sfseg_ctx* c, int K) {
    const int C = c->prm.ckpt_every > 0 ? c->prm.ckpt_every : 8;
    const int nck = (K + C - 1) / C + 1;
    if (K > c->rec_cap) {
        CUDA_OR(c, cudaDeviceSynchronize());
        if (c->d_rec) cudaFree(c->d_rec);
        if (c->d_rrec) cudaFree(c->d_rrec);
        c->d_rec = c->d_rrec = nullptr;
        c->rec_cap = 0;
        CUDA_OR(c, cudaMalloc((void**)&c->d_rec, sizeof(double) * 3 * (K + 1)));
        CUDA_OR(c, cudaMalloc((void**)&c->d_rrec, sizeof(double) * 3 * (K + 1)));
        c->rec_cap = K;
    }
    if (nck > c->ckpt_cap) {
        CUDA_OR(c, cudaDeviceSynchronize());
        if (c->d_ckpt) cudaFree(c->d_ckpt);
        c->d_ckpt = nullptr;
        c->ckpt_cap = 0;
        CUDA_OR(c, cudaMalloc(&c->d_ckpt, vol_bytes(c) * nck));
        c->ckpt_cap = nck;
    }
    return SFSEG_OK;
}

static void* ckpt_ptr(sfseg_ctx* c, int j) { return (char*)c->d_ckpt + vol_bytes(c) * (size_t)j; }

// Forward pass that keeps what the adjoint needs: the scale, gain and norm
// of every step, and the stored iterate every C steps (and the last one).
static sfseg_status iterate_record(sfseg_ctx* c, const float* d_x_in, float* d_x, int K,
                                   cudaStream_t s) {
    const int C = c->prm.ckpt_every > 0 ? c->prm.ckpt_every : 8;
    sfseg_status st = ensure_record(c, K > 0 ? K : 1);
    if (st != SFSEG_OK) return st;
    c->recorded = false;
    st = prep_x(c, 0, d_x_in, false, 0.0, s, c->d_rec);
    if (st != SFSEG_OK) return st;
    const size_t vb = vol_bytes(c);
    CUDA_OR(c, cudaMemcpyAsync(ckpt_ptr(c, 0), c->xa, vb, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < K; ++k) {
        CUDA_OR(c, launch_step(c, k, false, true, s, true));
        const int k1 = k + 1;
        if (k1 % C == 0 || k1 == K) {
            const void* src = (k1 & 1) ? c->xb : c->xa;
            CUDA_OR(c, cudaMemcpyAsync(ckpt_ptr(c, (k1 + C - 1) / C), src, vb, cudaMemcpyDeviceToDevice, s));
        }
    }
    FinishParams F{};
    F.out = d_x;
    F.buf0 = c->xa;
    F.buf1 = c->xb;
    F.g = c->geo[0];
    F.state = c->d_state;
    F.video = 0;
    F.final_iter = -1;
    CUDA_OR(c, launch_finish(c->prm.storage, F, s));
    c->launches += 1;
    c->last_stream = s;
    c->recorded = true;
    c->rec_K = K;
    return SFSEG_OK;
}

// ------------------------------------------------------------- autotuner
// SFSEG_AUTOTUNE: at the first power_iterate the context times every step path
// it can run on its own features and x0 (the per-step specialised kernel, the
// per-step any-radius kernel, and the fused launch with the default, half and
// quarter CTA count when the volume is small enough for its scratch to stay in
// L2), and keeps the fastest.  The choice is cached per (video shapes, radii,
// storage, channels, device) for the process, so later contexts of the same
// shape class skip the timing.  Every candidate computes the same operator;
// results differ only in summation order.
static constexpr long long kFusedTuneMaxVoxels = 8ll << 20;   // scratch 3 x 4 B x N <= 96 MiB
static constexpr int kTuneSteps = 6;

struct TuneChoice { int path, ctas; double us[4]; };
static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune_cache;

static std::string tune_key(const sfseg_ctx* c) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::string k = std::to_string(dev) + ":" + std::to_string(c->prm.rt) + "," + std::to_string(c->prm.ry) +
                    "," + std::to_string(c->prm.rx) + ":" + std::to_string(c->prm.storage) + ":" +
                    std::to_string(c->prm.nchan) + ":" + std::to_string(c->fast ? 1 : 0);
    for (const VideoGeom& g : c->geo)
        k += ":" + std::to_string(g.nf) + "x" + std::to_string(g.h) + "x" + std::to_string(g.w);
    return k;
}

static void drop_graphs(sfseg_ctx* c) {   // captured graphs belong to the path they were taken on
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

static sfseg_status set_path(sfseg_ctx* c, int path, int ctas) {
    if (path != c->path) drop_graphs(c);
    c->path = path;
    if (path == SFSEG_PATH_FUSED && ctas != c->fused_ctas) CUDA_OR(c, upload_fused_plan(c, ctas));
    return SFSEG_OK;
}

static sfseg_status autotune(sfseg_ctx* c, const float* const* d_x_in, cudaStream_t s) {
    c->tune_pending = false;
    const std::string key = tune_key(c);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            memcpy(c->tuned_us, it->second.us, sizeof c->tuned_us);
            return set_path(c, it->second.path, it->second.ctas);
        }
    }
    struct Cand { int path, ctas; };
    std::vector<Cand> cands;
    if (c->fast) cands.push_back({SFSEG_PATH_FAST, 0});
    cands.push_back({SFSEG_PATH_GENERIC, 0});
    if (c->cluster_ok) cands.push_back({SFSEG_PATH_CLUSTER, 0});
    if (c->fused_ok && c->total <= kFusedTuneMaxVoxels) {
        const int g0 = fused_default_ctas(c);
        for (int g : {g0, (g0 + 1) / 2, (g0 + 3) / 4})
            if (g >= 1 && (cands.back().path != SFSEG_PATH_FUSED || cands.back().ctas != g))
                cands.push_back({SFSEG_PATH_FUSED, g});
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_OR(c, cudaEventCreate(&e0));
    CUDA_OR(c, cudaEventCreate(&e1));
    double best = 1e300;
    Cand pick = cands[0];
    double us_path[4] = {-1.0, -1.0, -1.0, -1.0};
    sfseg_status st = SFSEG_OK;
    for (const Cand& cd : cands) {
        if ((st = set_path(c, cd.path, cd.ctas)) != SFSEG_OK) break;
        double us = 0.0;
        for (int rep = 0; rep < 2 && st == SFSEG_OK; ++rep) {   // rep 0 warms up (graph capture, scratch)
            cudaEventRecord(e0, s);
            for (int v = 0; v < c->nv && st == SFSEG_OK; ++v) st = prep_x(c, v, d_x_in[v], false, 0.0, s);
            if (st != SFSEG_OK) break;
            st = cd.path == SFSEG_PATH_FUSED     ? run_fused(c, kTuneSteps, false, s)
                 : cd.path == SFSEG_PATH_CLUSTER ? run_cluster(c, kTuneSteps, false, s)
                                                 : run_steps(c, kTuneSteps, s);
            if (st != SFSEG_OK) break;
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = fail(c, SFSEG_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
                break;
            }
            us = 1000.0 * ms / kTuneSteps;
        }
        if (st != SFSEG_OK) break;
        if (us_path[cd.path] < 0.0 || us < us_path[cd.path]) us_path[cd.path] = us;
        if (us < best) {
            best = us;
            pick = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SFSEG_OK) return st;
    memcpy(c->tuned_us, us_path, sizeof us_path);
    st = set_path(c, pick.path, pick.ctas);
    if (st != SFSEG_OK) return st;
    drop_graphs(c);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneChoice tc{pick.path, pick.ctas, {us_path[0], us_path[1], us_path[2], us_path[3]}};
    g_tune_cache[key] = tc;
    return SFSEG_OK;
}

static sfseg_status iterate_impl(sfseg_ctx* c, const float* const* d_x_in, float* const* d_x,
                                 int K, double tol, int32_t* iters_done, cudaStream_t s) {
    if (K < 0) return fail(c, SFSEG_EINVAL, "n_iters must be >= 0");
    if (!std::isfinite(tol) || tol < 0.0) return fail(c, SFSEG_EINVAL, "tol must be finite and >= 0");
    if (!c->features) return fail(c, SFSEG_ESTATE, "no features loaded");
    for (int v = 0; v < c->nv; ++v)
        if (!d_x[v]) return fail(c, SFSEG_EINVAL, "video %d: NULL x pointer", v);
    sfseg_status st = ensure_trace(c, K > 0 ? K : 1);
    if (st != SFSEG_OK) return st;
    if (c->prm.flags & SFSEG_RECORD) {
        if (c->nv != 1 || c->prm.storage != SFSEG_F32 || tol != 0.0 || c->prm.nchan != 1)
            return fail(c, SFSEG_EUNSUPPORTED,
                        "recording for the adjoint needs one video, FP32 storage, one channel, tol = 0");
        st = iterate_record(c, d_x_in[0], d_x[0], K, s);
        if (st == SFSEG_OK && iters_done) {
            std::vector<VState> vs;
            st = device_status(c, s, &vs);
            *iters_done = vs[0].iter;
        }
        return st;
    }
    c->recorded = false;
    if (c->tune_pending) {
        st = autotune(c, d_x_in, s);
        if (st != SFSEG_OK) return st;
    }
    for (int v = 0; v < c->nv; ++v) {
        st = prep_x(c, v, d_x_in[v], false, tol, s);
        if (st != SFSEG_OK) return st;
    }
    const bool final_mode = (K > 0 && tol == 0.0);
    if (c->path == SFSEG_PATH_FUSED || c->path == SFSEG_PATH_CLUSTER) {
        if (final_mode) {
            CUDA_OR(c, launch_set_ptrs(c->d_out, d_x, c->nv, s));
            c->launches += 1;
        }
        st = c->path == SFSEG_PATH_FUSED ? run_fused(c, K, final_mode, s) : run_cluster(c, K, final_mode, s);
        if (st != SFSEG_OK) return st;
    } else {
        st = run_steps(c, final_mode ? K - 1 : K, s);
        if (st != SFSEG_OK) return st;
        if (final_mode) {
            CUDA_OR(c, launch_set_ptrs(c->d_out, d_x, c->nv, s));
            CUDA_OR(c, launch_step(c, K - 1, true, true, s));
            c->launches += 1;   // set_ptrs
        }
    }
    for (int v = 0; v < c->nv; ++v) {
        FinishParams F{};
        F.out = d_x[v];
        F.buf0 = c->xa;
        F.buf1 = c->xb;
        F.g = c->geo[v];
        F.state = c->d_state;
        F.video = v;
        F.final_iter = final_mode ? K : -1;
        CUDA_OR(c, launch_finish(c->prm.storage, F, s));
        c->launches += 1;
    }
    c->last_stream = s;
    if (iters_done) {
        std::vector<VState> vs;
        st = device_status(c, s, &vs);
        *iters_done = vs[0].iter;
        return st;
    }
    return SFSEG_OK;
}

// per translation unit: the debug build's violation words (zeros otherwise)
namespace sfseg {
void sfseg_debug_take_fast(unsigned long long* out);
void sfseg_debug_take_generic(unsigned long long* out);
void sfseg_debug_take_fused(unsigned long long* out);
void sfseg_debug_take_cluster(unsigned long long* out);
}  // namespace sfseg

// ======================================================================= C-ABI
extern "C" {

int32_t sfseg_debug_build(void) {
#ifdef SFSEG_DEBUG
    return 1;
#else
    return 0;
#endif
}

sfseg_status sfseg_debug_status(int64_t* count, int32_t* code, int64_t* a, int64_t* b) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(nullptr, SFSEG_ECUDA, "debug status: %s", cudaGetErrorString(e));
    unsigned long long n = 0, first[3] = {0, 0, 0};
    void (*take[])(unsigned long long*) = {sfseg_debug_take_fast, sfseg_debug_take_generic,
                                           sfseg_debug_take_fused, sfseg_debug_take_cluster};
    for (auto fn : take) {
        unsigned long long w[4];
        fn(w);
        if (w[0] && !n) memcpy(first, w + 1, sizeof first);
        n += w[0];
    }
    if (count) *count = (int64_t)n;
    if (code) *code = (int32_t)first[0];
    if (a) *a = (int64_t)first[1];
    if (b) *b = (int64_t)first[2];
    return SFSEG_OK;
}

void sfseg_default_params(sfseg_params* p, int32_t nf, int32_t h, int32_t w) {
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->nf = nf;
    p->h = h;
    p->w = w;
    p->rt = 2;
    p->ry = 5;
    p->rx = 5;
    p->sigma_t = 1.5;
    p->sigma_y = 3.0;
    p->sigma_x = 3.0;
    p->alpha = 1.0;
    p->p = 0.1;
    p->storage = SFSEG_F32;
    p->flags = 0;
    p->nchan = 1;
    p->ckpt_every = 8;
}

sfseg_status sfseg_create(const sfseg_params* prm, sfseg_ctx** out) {
    if (!prm) return fail(nullptr, SFSEG_EINVAL, "params is NULL");
    int32_t dims[3] = {prm->nf, prm->h, prm->w};
    return create_impl(prm, 1, dims, false, out);
}

sfseg_status sfseg_create_batched(const sfseg_params* prm, int32_t n_videos, const int32_t* dims,
                                  sfseg_ctx** out) {
    if (!dims) return fail(nullptr, SFSEG_EINVAL, "dims is NULL");
    return create_impl(prm, n_videos, dims, true, out);
}

void sfseg_destroy(sfseg_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx(ctx);
}

sfseg_status sfseg_load_features(sfseg_ctx* c, const float* d_s, const float* d_f, void* stream) {
    NvtxRange nvtx_range("sfseg_load_features");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (c->batched) return fail(c, SFSEG_EINVAL, "batched context: use sfseg_load_features_batched");
    return load_features_impl(c, &d_s, &d_f, (cudaStream_t)stream);
}

sfseg_status sfseg_load_features_batched(sfseg_ctx* c, const float* const* d_s,
                                         const float* const* d_f, void* stream) {
    NvtxRange nvtx_range("sfseg_load_features_batched");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (!d_s || !d_f) return fail(c, SFSEG_EINVAL, "NULL pointer array");
    return load_features_impl(c, d_s, d_f, (cudaStream_t)stream);
}

sfseg_status sfseg_power_iterate(sfseg_ctx* c, const float* d_s, const float* d_f, float* d_x,
                                 int32_t n_iters, double tol, int32_t* iters_done, void* stream) {
    NvtxRange nvtx_range("sfseg_power_iterate");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (c->batched) return fail(c, SFSEG_EINVAL, "batched context: use sfseg_power_iterate_batched");
    cudaStream_t s = (cudaStream_t)stream;
    if ((d_s == nullptr) != (d_f == nullptr))
        return fail(c, SFSEG_EINVAL, "pass both d_s and d_f, or neither");
    if (d_s) {
        sfseg_status st = load_features_impl(c, &d_s, &d_f, s);
        if (st != SFSEG_OK) return st;
    }
    const float* xin = d_x;
    return iterate_impl(c, &xin, &d_x, n_iters, tol, iters_done, s);
}

void sfseg_default_binarize(sfseg_binarize* b) {
    if (!b) return;
    b->k0 = 3;
    b->reserved = 0;
    b->beta = 10.0;
    b->tau = 0.5;
    b->theta = 0.5;
}

static constexpr int kBinBlocks = 1216;   // 8 blocks of 256 threads per SM on 152 SMs

sfseg_status sfseg_power_iterate_binarized(sfseg_ctx* c, const float* d_s, const float* d_f,
                                           float* d_x, int32_t n_iters, const sfseg_binarize* b,
                                           uint8_t* d_mask, void* stream) {
    NvtxRange nvtx_range("sfseg_power_iterate_binarized");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (c->batched) return fail(c, SFSEG_EINVAL, "binarisation takes a single-video context");
    if (!b) return fail(c, SFSEG_EINVAL, "schedule is NULL");
    if (b->k0 < 1 || !std::isfinite(b->beta) || b->beta < 0.0 || !std::isfinite(b->tau) ||
        !std::isfinite(b->theta))
        return fail(c, SFSEG_EINVAL, "schedule: k0 >= 1, beta finite >= 0, tau and theta finite");
    if (n_iters < 1) return fail(c, SFSEG_EINVAL, "n_iters must be >= 1");
    if (!d_x) return fail(c, SFSEG_EINVAL, "d_x is NULL");
    if (c->prm.flags & SFSEG_RECORD)
        return fail(c, SFSEG_EUNSUPPORTED, "binarisation does not record for the adjoint");
    cudaStream_t s = (cudaStream_t)stream;
    if ((d_s == nullptr) != (d_f == nullptr))
        return fail(c, SFSEG_EINVAL, "pass both d_s and d_f, or neither");
    if (d_s) {
        sfseg_status st = load_features_impl(c, &d_s, &d_f, s);
        if (st != SFSEG_OK) return st;
    }
    if (!c->features) return fail(c, SFSEG_ESTATE, "no features loaded");
    sfseg_status st = ensure_trace(c, n_iters);
    if (st != SFSEG_OK) return st;
    if (!c->d_bin) {
        const size_t bytes = 16 + sizeof(double) * kBinBlocks;
        CUDA_OR(c, cudaMalloc((void**)&c->d_bin, bytes));
        CUDA_OR(c, cudaMemset(c->d_bin, 0, bytes));
    }
    unsigned* keys = reinterpret_cast<unsigned*>(c->d_bin);
    double* partials = reinterpret_cast<double*>(c->d_bin + 16);
    c->recorded = false;
    st = prep_x(c, 0, d_x, false, 0.0, s);
    if (st != SFSEG_OK) return st;
    const VideoGeom& g = c->geo[0];
    const int nblk = (int)std::min<long long>(kBinBlocks, (g.n + 255) / 256);
    const int K = n_iters;
    for (int k = 0; k < K; ++k) {
        if (k == K - 1) {
            CUDA_OR(c, launch_set_ptrs(c->d_out, &d_x, 1, s));
            c->launches += 1;
            CUDA_OR(c, launch_step(c, k, true, true, s));
        } else {
            CUDA_OR(c, launch_step(c, k, false, true, s));
        }
        if (k + 1 < K && k + 1 >= b->k0) {   // Alg. 1 Step 3 after step k + 1 (1-based)
            ProjectParams P{};
            P.buf = ((k + 1) & 1) ? c->xb : c->xa;   // where step k stored its output
            P.g = g;
            P.state = c->d_state;
            P.video = 0;
            P.beta = (float)b->beta;
            P.tau = (float)b->tau;
            P.vmax_key = keys;
            P.partials = partials;
            P.n_blocks = nblk;
            CUDA_OR(c, launch_project(c->prm.storage, P, s));
            c->launches += 3;
        }
    }
    FinishParams F{};
    F.out = d_x;
    F.buf0 = c->xa;
    F.buf1 = c->xb;
    F.g = g;
    F.state = c->d_state;
    F.video = 0;
    F.final_iter = K;
    CUDA_OR(c, launch_finish(c->prm.storage, F, s));
    c->launches += 1;
    if (d_mask) {
        CUDA_OR(c, launch_threshold(d_x, g.n, keys + 1, (float)b->theta, d_mask, nblk, s));
        c->launches += 2;
    }
    c->last_stream = s;
    return SFSEG_OK;
}

sfseg_status sfseg_power_iterate_batched(sfseg_ctx* c, const float* const* d_s,
                                         const float* const* d_f, float* const* d_x,
                                         int32_t n_iters, void* stream) {
    NvtxRange nvtx_range("sfseg_power_iterate_batched");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (!d_x) return fail(c, SFSEG_EINVAL, "d_x is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if ((d_s == nullptr) != (d_f == nullptr))
        return fail(c, SFSEG_EINVAL, "pass both d_s and d_f, or neither");
    if (d_s) {
        sfseg_status st = load_features_impl(c, d_s, d_f, s);
        if (st != SFSEG_OK) return st;
    }
    std::vector<const float*> xin(d_x, d_x + c->nv);
    return iterate_impl(c, xin.data(), d_x, n_iters, 0.0, nullptr, s);
}

sfseg_status sfseg_rayleigh(sfseg_ctx* c, const float* d_x, double* lambda, double* residual,
                            void* stream) {
    NvtxRange nvtx_range("sfseg_rayleigh");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (c->batched) return fail(c, SFSEG_EINVAL, "rayleigh needs a single-video context");
    if (!d_x) return fail(c, SFSEG_EINVAL, "d_x is NULL");
    if (!c->features) return fail(c, SFSEG_ESTATE, "no features loaded");
    cudaStream_t s = (cudaStream_t)stream;
    sfseg_status st = ensure_trace(c, 1);
    if (st != SFSEG_OK) return st;
    st = prep_x(c, 0, d_x, false, 0.0, s);
    if (st != SFSEG_OK) return st;
    CUDA_OR(c, launch_step(c, 0, false, false, s));
    st = device_status(c, s, nullptr);
    if (st != SFSEG_OK) return st;
    double row[3];
    CUDA_OR(c, cudaMemcpy(row, c->d_trace, sizeof row, cudaMemcpyDeviceToHost));
    if (lambda) *lambda = row[0];
    if (residual) *residual = row[1];
    c->last_stream = s;
    return SFSEG_OK;
}

sfseg_status sfseg_apply(sfseg_ctx* c, const float* d_x, float* d_y, void* stream) {
    NvtxRange nvtx_range("sfseg_apply");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (c->batched) return fail(c, SFSEG_EINVAL, "apply needs a single-video context");
    if (!d_x || !d_y) return fail(c, SFSEG_EINVAL, "NULL pointer");
    if (d_x == d_y) return fail(c, SFSEG_EINVAL, "d_x and d_y may not alias");
    if (!c->features) return fail(c, SFSEG_ESTATE, "no features loaded");
    cudaStream_t s = (cudaStream_t)stream;
    sfseg_status st = ensure_trace(c, 1);
    if (st != SFSEG_OK) return st;
    st = prep_x(c, 0, d_x, true, 0.0, s);
    if (st != SFSEG_OK) return st;
    CUDA_OR(c, launch_set_ptrs(c->d_out, &d_y, 1, s));
    CUDA_OR(c, launch_step(c, 0, true, true, s));
    c->launches += 1;
    c->last_stream = s;
    return SFSEG_OK;
}

int32_t sfseg_get_trace(sfseg_ctx* c, int32_t video, double* rayleigh, double* residual,
                        double* norms, int32_t cap) {
    if (!c) return -1;
    if (video < 0 || video >= c->nv || cap < 0) {
        fail(c, SFSEG_EINVAL, "bad video index or capacity");
        return -1;
    }
    if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) {
        fail(c, SFSEG_ECUDA, "stream synchronise failed");
        return -1;
    }
    VState st;
    if (cudaMemcpy(&st, c->d_state + video, sizeof st, cudaMemcpyDeviceToHost) != cudaSuccess) {
        fail(c, SFSEG_ECUDA, "state copy failed");
        return -1;
    }
    int n = st.iter < c->trace_cap ? st.iter : c->trace_cap;
    if (n > cap) n = cap;
    if (n > 0) {
        std::vector<double> rows(3 * (size_t)n);
        if (cudaMemcpy(rows.data(), c->d_trace + 3 * (size_t)video * c->trace_cap,
                       sizeof(double) * 3 * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
            fail(c, SFSEG_ECUDA, "trace copy failed");
            return -1;
        }
        for (int k = 0; k < n; ++k) {
            if (rayleigh) rayleigh[k] = rows[3 * k];
            if (residual) residual[k] = rows[3 * k + 1];
            if (norms) norms[k] = rows[3 * k + 2];
        }
    }
    return n;
}

sfseg_status sfseg_adjoint(sfseg_ctx* c, const float* d_gx, float* d_gsp, float* d_gf,
                           float* d_gx0, void* stream) {
    NvtxRange nvtx_range("sfseg_adjoint");
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (!d_gx) return fail(c, SFSEG_EINVAL, "d_gx is NULL");
    if (!c->recorded) return fail(c, SFSEG_ESTATE, "no recorded forward (create with SFSEG_RECORD)");
    if (c->rec_K < 1) return fail(c, SFSEG_EUNSUPPORTED, "the recorded forward has no step");
    cudaStream_t s = (cudaStream_t)stream;
    const int K = c->rec_K;
    const int C = c->prm.ckpt_every > 0 ? c->prm.ckpt_every : 8;
    const int nseg = (K + C - 1) / C;
    const VideoGeom& g = c->geo[0];
    const size_t vb = vol_bytes(c);
    if (setup_adjoint(c->prm.rt, c->prm.ry, c->prm.rx) != cudaSuccess)
        return fail(c, SFSEG_EUNSUPPORTED, "radii too large for the adjoint tile");
    // volumes: recomputed iterates [C], g ping-pong [2], dL/dsp, dL/df; on the
    // specialised path also K_X, F_X of every recomputed step [2C], K_U, F_U
    const int nvol = c->fast ? 3 * C + 6 : C + 4;
    if (c->adj_cap < nvol) {
        CUDA_OR(c, cudaDeviceSynchronize());
        if (c->d_adj) cudaFree(c->d_adj);
        c->d_adj = nullptr;
        c->adj_cap = 0;
        CUDA_OR(c, cudaMalloc(&c->d_adj, vb * nvol));
        c->adj_cap = nvol;
    }
    constexpr int kAdjBlocks = 1216;
    if (c->fast && !c->d_adj_misc) {
        const size_t bytes = 256 + sizeof(double) * kAdjBlocks;
        CUDA_OR(c, cudaMalloc((void**)&c->d_adj_misc, bytes));
        CUDA_OR(c, cudaMemset(c->d_adj_misc, 0, bytes));
        const double ones[2] = {1.0, 1.0};
        CUDA_OR(c, cudaMemcpy(c->d_adj_misc + 128, ones, sizeof ones, cudaMemcpyHostToDevice));
    }
    if (!c->d_adjc) {
        CUDA_OR(c, cudaMalloc((void**)&c->d_adjc, sizeof(double) * 2));
        CUDA_OR(c, cudaMalloc((void**)&c->d_adj_partials, sizeof(double) * c->g_n_items));
        CUDA_OR(c, cudaMalloc((void**)&c->d_adj_counter, sizeof(unsigned)));
        CUDA_OR(c, cudaMemset(c->d_adj_counter, 0, sizeof(unsigned)));
    }
    auto vol = [&](int j) { return (float*)((char*)c->d_adj + vb * (size_t)j); };
    float* gb[2] = {vol(C), vol(C + 1)};
    float* dsp = vol(C + 2);
    float* df = vol(C + 3);
    const double* rscale = c->d_rec;
    const double* rgain = c->d_rec + (c->rec_cap + 1);
    const double* rny = c->d_rec + 2 * (c->rec_cap + 1);
    double* qscale = c->d_rrec;   // scales of the recomputed iterates
    CUDA_OR(c, cudaMemsetAsync(c->d_adj, 0, vb * nvol, s));
    CUDA_OR(c, launch_pitch_copy(d_gx, gb[0], g, 1, nullptr, s));
    CUDA_OR(c, launch_dot((const float*)ckpt_ptr(c, nseg), rscale + K, gb[0], g, c->d_prep_partials,
                          c->d_prep_counter, c->d_adjc, prep_x_blocks(g.n), s));
    c->launches += 2;
    int cur = 0, cpar = 0;
    for (int m = nseg - 1; m >= 0; --m) {
        const int k0 = m * C, k1 = (k0 + C < K) ? k0 + C : K;
        // recompute x^{k0+1} .. x^{k1-1} from the checkpoint with the step kernel
        // of the forward: the specialised one reproduces the recorded iterates
        // bit for bit (same kernel, plan and operands); it runs through the
        // context's ping-pong buffers (they carry the TMA descriptors) and each
        // output is copied to its adjoint volume
        if (c->fast) {
            // every step of the segment, the last one for its adjoint terms only
            CUDA_OR(c, launch_set_state(c->d_state, rscale + k0, rgain + k0, k0, s));
            c->launches += 1;
            CUDA_OR(c, cudaMemcpyAsync(c->xa, ckpt_ptr(c, m), vb, cudaMemcpyDeviceToDevice, s));
            for (int k = k0; k < k1; ++k) {
                const int i = k - k0;
                StepParams P = step_params(c, i, false, true);   // reads buffer i & 1
                P.trace = nullptr;
                P.trace_cap = 0;
                P.rec.scale = qscale;
                P.rec.gain = qscale + (c->rec_cap + 1);
                P.rec.ny = qscale + 2 * (c->rec_cap + 1);
                P.aux_k = vol(C + 4 + i);
                P.aux_f = vol(2 * C + 4 + i);
                CUDA_OR(c, launch_step_fast(c->prm.storage, P, c->n_ctas, s));
                c->launches += 1;
                if (k + 1 < k1)
                    CUDA_OR(c, cudaMemcpyAsync(vol(i + 1), ((i + 1) & 1) ? c->xb : c->xa, vb,
                                               cudaMemcpyDeviceToDevice, s));
            }
            VState* ustate = reinterpret_cast<VState*>(c->d_adj_misc);
            const double* one = reinterpret_cast<const double*>(c->d_adj_misc + 128);
            unsigned* cnt = reinterpret_cast<unsigned*>(c->d_adj_misc + 192);
            double* part = reinterpret_cast<double*>(c->d_adj_misc + 256);
            float* ku = vol(3 * C + 4);
            float* fu = vol(3 * C + 5);
            const int nblk = (int)std::min<long long>(kAdjBlocks, (g.n + 255) / 256);
            for (int k = k1 - 1; k >= k0; --k) {
                const float* x_next = (k + 1 == k1) ? (const float*)ckpt_ptr(c, m + 1) : vol(k + 1 - k0);
                const double* s_next = (k + 1 == k1) ? rscale + k1 : qscale + k + 1;
                const float* x_cur = (k == k0) ? (const float*)ckpt_ptr(c, m) : vol(k - k0);
                const double* s_cur = (k == k0) ? rscale + k0 : qscale + k;
                // u_k into the forward kernel's input buffer
                CUDA_OR(c, launch_uprep(gb[cur], x_next, s_next, c->d_adjc + cpar, rny + k, (float*)c->xa, g,
                                        nblk, s));
                // g_k = M u_k, with K_U and F_U
                CUDA_OR(c, launch_set_state(ustate, one, one + 1, 0, s));
                StepParams P = step_params(c, 0, false, true);
                P.z_out = gb[1 - cur];
                P.state = ustate;
                P.trace = nullptr;
                P.trace_cap = 0;
                P.aux_k = ku;
                P.aux_f = fu;
                CUDA_OR(c, launch_step_fast(c->prm.storage, P, c->n_ctas, s));
                AdjCombineParams Q{};
                Q.u = (const float*)c->xa;
                Q.x_cur = x_cur;
                Q.sp = (const float*)c->sp;
                Q.ku = ku;
                Q.fu = fu;
                Q.kx = vol(C + 4 + (k - k0));
                Q.fx = vol(2 * C + 4 + (k - k0));
                Q.dsp = dsp;
                Q.df = df;
                Q.s_cur = s_cur;
                Q.c_out = c->d_adjc + (1 - cpar);
                Q.partials = part;
                Q.counter = cnt;
                Q.g = g;
                Q.alpha = (float)c->prm.alpha;
                CUDA_OR(c, launch_adj_combine(Q, nblk, s));
                c->launches += 4;
                cur = 1 - cur;
                cpar = 1 - cpar;
            }
            continue;
        } else if (k1 - k0 > 1) {
            CUDA_OR(c, launch_set_state(c->d_state, rscale + k0, rgain + k0, k0, s));
            c->launches += 1;
            for (int k = k0; k < k1 - 1; ++k) {
                StepParams P = step_params(c, 0, false, true);
                P.x_in = (k == k0) ? ckpt_ptr(c, m) : (void*)vol(k - k0);
                P.z_out = vol(k - k0 + 1);
                P.items = c->d_gitems;
                P.item_begin = c->d_gitem_begin;
                P.vseg = nullptr;
                P.partials = c->d_gpartials;
                P.n_items = c->g_n_items;
                P.trace = nullptr;
                P.trace_cap = 0;
                P.rec.scale = qscale;
                P.rec.gain = qscale + (c->rec_cap + 1);
                P.rec.ny = qscale + 2 * (c->rec_cap + 1);
                CUDA_OR(c, launch_step_generic(c->prm.storage, P, c->g_n_items, s));
                c->launches += 1;
            }
        }
        for (int k = k1 - 1; k >= k0; --k) {
            AdjParams A{};
            A.g_in = gb[cur];
            A.g_out = gb[1 - cur];
            A.x_next = (k + 1 == k1) ? (const float*)ckpt_ptr(c, m + 1) : vol(k + 1 - k0);
            A.s_next = (k + 1 == k1) ? rscale + k1 : qscale + k + 1;
            A.x_cur = (k == k0) ? (const float*)ckpt_ptr(c, m) : vol(k - k0);
            A.s_cur = (k == k0) ? rscale + k0 : qscale + k;
            A.ny = rny + k;
            A.c_in = c->d_adjc + cpar;
            A.c_out = c->d_adjc + (1 - cpar);
            A.sp = (const float*)c->sp;
            A.f = (const float*)c->f;
            A.dsp = dsp;
            A.df = df;
            A.geo = c->d_geo;
            A.items = c->d_gitems;
            A.partials = c->d_adj_partials;
            A.counter = c->d_adj_counter;
            A.alpha = (float)c->prm.alpha;
            A.rt = c->prm.rt;
            A.ry = c->prm.ry;
            A.rx = c->prm.rx;
            memcpy(A.gt, c->gt, sizeof c->gt);
            memcpy(A.gy, c->gy, sizeof c->gy);
            memcpy(A.gx, c->gx, sizeof c->gx);
            CUDA_OR(c, launch_adjoint(A, c->g_n_items, s));
            c->launches += 1;
            cur = 1 - cur;
            cpar = 1 - cpar;
        }
    }
    // dL/dx0 = g_0 / ||x0|| (x^0 was the normalised x0); dL/dsp, dL/df
    if (d_gx0) CUDA_OR(c, launch_pitch_copy(gb[cur], d_gx0, g, 0, rscale + 0, s));
    if (d_gsp) CUDA_OR(c, launch_pitch_copy(dsp, d_gsp, g, 0, nullptr, s));
    if (d_gf) CUDA_OR(c, launch_pitch_copy(df, d_gf, g, 0, nullptr, s));
    c->launches += 3;
    c->last_stream = s;
    return SFSEG_OK;
}

// key of a float as kept on the device (float_key), decoded on the host
static float key_to_float(unsigned k) {
    const unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float v;
    memcpy(&v, &b, sizeof v);
    return v;
}

sfseg_status sfseg_get_warnings(sfseg_ctx* c, int32_t* flags) {
    if (!c || !flags) return fail(c, SFSEG_EINVAL, "ctx and flags must be non-NULL");
    *flags = 0;
    if (!c->features) return SFSEG_OK;
    CUDA_OR(c, cudaDeviceSynchronize());   // the load may have run on any stream
    std::vector<unsigned> lo((size_t)kMaxChan * c->nv), hi((size_t)kMaxChan * c->nv);
    CUDA_OR(c, cudaMemcpy(lo.data(), c->d_fmin, sizeof(unsigned) * lo.size(), cudaMemcpyDeviceToHost));
    CUDA_OR(c, cudaMemcpy(hi.data(), c->d_fmax, sizeof(unsigned) * hi.size(), cudaMemcpyDeviceToHost));
    for (int v = 0; v < c->nv; ++v)
        for (int ch = 0; ch < c->prm.nchan; ++ch) {
            const double r = (double)key_to_float(hi[kMaxChan * v + ch]) - key_to_float(lo[kMaxChan * v + ch]);
            if (c->prm.alpha * r * r > 1.0) *flags |= SFSEG_WARN_NEGATIVE_M;
        }
    return SFSEG_OK;
}

sfseg_status sfseg_debug_inject_timeout(sfseg_ctx* c, int32_t n_steps) {
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (n_steps < 0) return fail(c, SFSEG_EINVAL, "n_steps must be >= 0");
    if (c->path == SFSEG_PATH_CLUSTER)
        return fail(c, SFSEG_EUNSUPPORTED, "the cluster launch has no timed wait to inject into");
    if (!c->fast && c->path != SFSEG_PATH_FUSED)
        return fail(c, SFSEG_EUNSUPPORTED,
                    "timeouts exist only in the specialised step kernel and the fused launch");
    c->inject_steps = n_steps;
    return SFSEG_OK;
}

sfseg_status sfseg_sync_status(sfseg_ctx* c) {
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    return device_status(c, c->last_stream, nullptr);
}

const char* sfseg_last_error(const sfseg_ctx* c) {
    return c ? c->err.c_str() : g_create_err.c_str();
}

const char* sfseg_status_string(sfseg_status st) {
    switch (st) {
        case SFSEG_OK: return "SFSEG_OK";
        case SFSEG_EINVAL: return "SFSEG_EINVAL";
        case SFSEG_ENOMEM: return "SFSEG_ENOMEM";
        case SFSEG_ECUDA: return "SFSEG_ECUDA";
        case SFSEG_EZERONORM: return "SFSEG_EZERONORM";
        case SFSEG_ENONFINITE: return "SFSEG_ENONFINITE";
        case SFSEG_ETIMEOUT: return "SFSEG_ETIMEOUT";
        case SFSEG_EUNSUPPORTED: return "SFSEG_EUNSUPPORTED";
        case SFSEG_ESTATE: return "SFSEG_ESTATE";
    }
    return "SFSEG_UNKNOWN";
}

int64_t sfseg_launch_count(const sfseg_ctx* c) { return c ? c->launches : 0; }

// ------------------------------------------------ video split along t (slabs)
sfseg_status sfseg_create_slab(const sfseg_params* prm, int32_t own_lo, int32_t own_hi,
                               int64_t video_voxels, sfseg_ctx** out) {
    if (!prm) return fail(nullptr, SFSEG_EINVAL, "params is NULL");
    if (out) *out = nullptr;
    sfseg_status st = validate(prm);
    if (st != SFSEG_OK) return st;
    if (prm->flags & (SFSEG_FUSED | SFSEG_AUTOTUNE | SFSEG_RECORD | SFSEG_CLUSTER))
        return fail(nullptr, SFSEG_EUNSUPPORTED,
                    "a slab runs the per-step kernels (no FUSED, AUTOTUNE, RECORD, CLUSTER)");
    if (own_lo < 0 || own_hi > prm->nf || own_lo >= own_hi)
        return fail(nullptr, SFSEG_EINVAL, "own frames [%d, %d) outside the slab's %d frames", own_lo, own_hi,
                    prm->nf);
    if (own_lo > prm->rt || prm->nf - own_hi > prm->rt)
        return fail(nullptr, SFSEG_EINVAL, "halo of %d and %d frames exceeds rt = %d", own_lo, prm->nf - own_hi,
                    prm->rt);
    if ((own_lo > 0 || own_hi < prm->nf) && own_hi - own_lo < prm->rt)
        return fail(nullptr, SFSEG_EINVAL, "%d own frames: a slab with neighbours owns at least rt = %d",
                    own_hi - own_lo, prm->rt);
    const long long own_vox = (long long)(own_hi - own_lo) * prm->h * prm->w;
    if (video_voxels < own_vox)
        return fail(nullptr, SFSEG_EINVAL, "video_voxels %lld < the slab's own %lld", (long long)video_voxels,
                    own_vox);
    int32_t dims[3] = {prm->nf, prm->h, prm->w};
    st = create_impl(prm, 1, dims, false, out, own_lo, own_hi);
    if (st != SFSEG_OK) return st;
    sfseg_ctx* c = *out;
    c->slab = true;
    c->own_lo = own_lo;
    c->own_hi = own_hi;
    c->video_voxels = video_voxels;
    return SFSEG_OK;
}

static sfseg_status slab_ok(sfseg_ctx* c) {
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (!c->slab) return fail(c, SFSEG_EINVAL, "not a slab context (sfseg_create_slab)");
    if (!c->features) return fail(c, SFSEG_ESTATE, "no features loaded");
    return SFSEG_OK;
}

sfseg_status sfseg_slab_start(sfseg_ctx* c, const float* d_x0, int32_t n_iters, double* d_part,
                              void* stream) {
    NvtxRange nvtx_range("sfseg_slab_start");
    sfseg_status st = slab_ok(c);
    if (st != SFSEG_OK) return st;
    if (!d_x0 || !d_part) return fail(c, SFSEG_EINVAL, "NULL pointer");
    if (n_iters < 0) return fail(c, SFSEG_EINVAL, "n_iters must be >= 0");
    if ((st = ensure_trace(c, n_iters > 0 ? n_iters : 1)) != SFSEG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = prep_x(c, 0, d_x0, false, 0.0, s, nullptr, d_part);
    if (st != SFSEG_OK) return st;
    c->slab_k = 0;
    c->recorded = false;
    c->last_stream = s;
    return SFSEG_OK;
}

sfseg_status sfseg_slab_set_norm(sfseg_ctx* c, const double* d_sumsq, void* stream) {
    sfseg_status st = slab_ok(c);
    if (st != SFSEG_OK) return st;
    if (!d_sumsq) return fail(c, SFSEG_EINVAL, "d_sumsq is NULL");
    const double gain0 = std::exp2(std::rint(std::log2(std::sqrt((double)c->video_voxels) / c->gsum)));
    CUDA_OR(c, launch_slab_state(c->d_state, d_sumsq, 0, gain0, c->video_voxels, c->d_trace, c->trace_cap,
                                 (cudaStream_t)stream));
    c->launches += 1;
    return SFSEG_OK;
}

sfseg_status sfseg_slab_step(sfseg_ctx* c, double* d_part, float* d_x_final, void* stream) {
    NvtxRange nvtx_range("sfseg_slab_step");
    sfseg_status st = slab_ok(c);
    if (st != SFSEG_OK) return st;
    if (!d_part) return fail(c, SFSEG_EINVAL, "d_part is NULL");
    if (c->slab_k >= c->trace_cap) return fail(c, SFSEG_EINVAL, "more steps than sfseg_slab_start's n_iters");
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_OR(c, cudaMemsetAsync(d_part, 0, sizeof(double) * kRed, s));   // a skipped (done) step sums to 0
    c->slab_final = d_x_final;
    if (d_x_final) {
        // the kernel writes frame t of the slab at [(t * h + y) * w + x] of
        // the pointer table's entry: offset it so the own frames land at 0
        const VideoGeom& g = c->geo[0];
        float* base = d_x_final - (long long)c->own_lo * g.h * g.w;
        CUDA_OR(c, launch_set_ptrs(c->d_out, &base, 1, s));
        c->launches += 1;
    }
    CUDA_OR(c, launch_step(c, c->slab_k, d_x_final != nullptr, true, s, false, d_part));
    c->slab_k += 1;
    c->last_stream = s;
    return SFSEG_OK;
}

sfseg_status sfseg_slab_finish_step(sfseg_ctx* c, const double* d_sums, void* stream) {
    sfseg_status st = slab_ok(c);
    if (st != SFSEG_OK) return st;
    if (!d_sums) return fail(c, SFSEG_EINVAL, "d_sums is NULL");
    CUDA_OR(c, launch_slab_state(c->d_state, d_sums, 1, 0.0, c->video_voxels, c->d_trace, c->trace_cap,
                                 (cudaStream_t)stream));
    c->launches += 1;
    return SFSEG_OK;
}

int64_t sfseg_slab_halo_bytes(const sfseg_ctx* c, int32_t side, int32_t dir) {
    if (!c || !c->slab || side < 0 || side > 1 || dir < 0 || dir > 1) return -1;
    const VideoGeom& g = c->geo[0];
    const long long frames = dir == 0 ? c->prm.rt : (side == 0 ? c->own_lo : g.nf - c->own_hi);
    return frames * g.plane * (long long)c->elt;
}

sfseg_status sfseg_slab_halo(sfseg_ctx* c, int32_t side, int32_t dir, void* d_buf, void* stream) {
    sfseg_status st = slab_ok(c);
    if (st != SFSEG_OK) return st;
    if (!d_buf) return fail(c, SFSEG_EINVAL, "d_buf is NULL");
    if (side < 0 || side > 1 || dir < 0 || dir > 1) return fail(c, SFSEG_EINVAL, "side and dir are 0 or 1");
    const VideoGeom& g = c->geo[0];
    const long long bytes = sfseg_slab_halo_bytes(c, side, dir);
    if (bytes == 0) return SFSEG_OK;
    // the stored iterate the next step reads
    char* buf = (char*)((c->slab_k & 1) ? c->xb : c->xa) + (size_t)g.off * c->elt;
    const long long pb = g.plane * (long long)c->elt;
    const int rt = c->prm.rt;
    char* frames = dir == 0 ? buf + (side == 0 ? c->own_lo : c->own_hi - rt) * pb
                            : buf + (side == 0 ? 0 : c->own_hi) * pb;
    if (dir == 0)
        CUDA_OR(c, cudaMemcpyAsync(d_buf, frames, (size_t)bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    else
        CUDA_OR(c, cudaMemcpyAsync(frames, d_buf, (size_t)bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SFSEG_OK;
}

sfseg_status sfseg_slab_output(sfseg_ctx* c, float* d_x, void* stream) {
    sfseg_status st = slab_ok(c);
    if (st != SFSEG_OK) return st;
    if (!d_x) return fail(c, SFSEG_EINVAL, "d_x is NULL");
    FinishParams F{};
    F.out = d_x;
    F.buf0 = c->xa;
    F.buf1 = c->xb;
    F.g = c->geo[0];
    F.g.nf = c->own_hi - c->own_lo;
    F.g.off += (long long)c->own_lo * F.g.plane;
    F.g.n = (long long)F.g.nf * F.g.h * F.g.w;
    F.state = c->d_state;
    F.video = 0;
    // the last step wrote its FP32 output into d_x: scale it in place (if
    // that step completed; otherwise the stored iterate of the last one that did)
    F.final_iter = (d_x == c->slab_final) ? c->slab_k : -1;
    CUDA_OR(c, launch_finish(c->prm.storage, F, (cudaStream_t)stream));
    c->launches += 1;
    c->last_stream = (cudaStream_t)stream;
    return SFSEG_OK;
}

sfseg_status sfseg_get_path(const sfseg_ctx* c, int32_t* path, int32_t* fused_ctas, double* us_per_step) {
    if (!c) return fail(nullptr, SFSEG_EINVAL, "ctx is NULL");
    if (path) *path = c->path;
    if (fused_ctas)
        *fused_ctas = c->path == SFSEG_PATH_FUSED ? c->fused_ctas
                      : c->path == SFSEG_PATH_CLUSTER ? c->cplan.n_ctas : 0;
    if (us_per_step) memcpy(us_per_step, c->tuned_us, sizeof c->tuned_us);
    return SFSEG_OK;
}

int32_t sfseg_plan_segments(int32_t n_videos, const int32_t* dims, int32_t n_sms,
                            int32_t* segments, int32_t seg_cap, int32_t* cta_begin,
                            int32_t cta_cap) {
    if (n_videos < 1 || !dims || n_sms < 1) {
        fail(nullptr, SFSEG_EINVAL, "plan: bad arguments");
        return -1;
    }
    std::vector<VideoGeom> geo;
    for (int v = 0; v < n_videos; ++v) {
        if (dims[3 * v] < 1 || dims[3 * v + 1] < 1 || dims[3 * v + 2] < 1) {
            fail(nullptr, SFSEG_EINVAL, "plan: video %d has an empty dimension", v);
            return -1;
        }
        VideoGeom g{};
        g.nf = dims[3 * v];
        g.h = dims[3 * v + 1];
        g.w = dims[3 * v + 2];
        geo.push_back(g);
    }
    std::vector<WorkItem> items;
    std::vector<int> ib, cb, vs;
    build_segments(geo, n_sms, &items, &ib, &cb, &vs);
    if (segments)
        for (int i = 0; i < (int)items.size() && i < seg_cap; ++i) {
            segments[5 * i + 0] = items[i].video;
            segments[5 * i + 1] = items[i].x0;
            segments[5 * i + 2] = items[i].y0;
            segments[5 * i + 3] = items[i].t0;
            segments[5 * i + 4] = items[i].t1;
        }
    if (cta_begin)
        for (int i = 0; i < (int)cb.size() && i < cta_cap; ++i) cta_begin[i] = cb[i];
    return (int32_t)items.size();
}

}  // extern "C"
