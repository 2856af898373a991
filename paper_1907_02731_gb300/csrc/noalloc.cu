// noalloc.cu -- power iteration for callers that cannot allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not
// wanted -- inside a region being captured into a larger CUDA graph (an
// allocation there breaks or serialises the capture), real-time paths with
// a fixed memory budget (cudaMalloc can block every stream on the device and
// can fail under memory pressure), and plug-ins hosted by a framework that owns
// all device memory through its own allocator.  sfseg_create() allocates the
// context's workspace with cudaMalloc, so those callers cannot use it.
//
// This entry point takes its workspace from one file-scope device array of
// fixed size instead, and calls no allocating routine.  The caller still owns
// and passes the inputs and the output.  What that costs:
//   * every GPU that loads the library holds the array (kScratchBytes) until
//     the process exits;
//   * volumes are limited to what fits in it (about 2 million voxels in
//     FP32 storage, twice that in BF16/FP16); larger requests fail with
//     SFSEG_EINVAL before anything is launched;
//   * all calls share the one array: calls that overlap on the GPU (two
//     streams, or two host threads) race and corrupt each other.  Serialise
//     them on one stream.
// The first call on each device looks up the array's device address (and the
// driver may load the library's device code then); make that first call
// before any stream capture begins.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "sfseg.h"
#include "sfseg_launch.h"

namespace {

using namespace sfseg;

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB per GPU
constexpr int kTraceCap = 1024;                       // trace rows kept per call
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// Items of the generic step kernel for one video: one CTA per (x, y) tile,
// each streaming every frame.  Written on the device (no host staging).
__global__ void noalloc_init_kernel(VideoGeom g, VideoGeom* geo, WorkItem* items, int* item_begin,
                                    int tiles_x, int n_items, int tx, int ty) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        geo[0] = g;
        item_begin[0] = 0;
        item_begin[1] = n_items;
    }
    if (i < n_items) {
        WorkItem it{};
        it.video = 0;
        it.x0 = (i % tiles_x) * tx;
        it.y0 = (i / tiles_x) * ty;
        it.t0 = 0;
        it.t1 = g.nf;
        items[i] = it;
    }
}

// Device address of g_scratch on the current device, looked up once.
sfseg_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_global_error(cudaGetErrorString(e));
        return SFSEG_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_global_error("no-alloc path: device index out of range");
        return SFSEG_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_global_error(cudaGetErrorString(e));
            return SFSEG_ECUDA;
        }
        e = setup_step_generic(kMaxRt, kMaxR, kMaxR);
        if (e != cudaSuccess) {
            set_global_error(cudaGetErrorString(e));
            return SFSEG_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SFSEG_OK;
}

}  // namespace

extern "C" sfseg_status sfseg_power_iterate_noalloc(const sfseg_params* prm, const float* d_s,
                                                    const float* d_f, float* d_x, int32_t n_iters,
                                                    double* d_trace, void* stream) {
    sfseg_status st = validate_params(prm);
    if (st != SFSEG_OK) return st;
    if (prm->nchan != 1) {
        set_global_error("no-alloc path: one pairwise channel only");
        return SFSEG_EUNSUPPORTED;
    }
    if (!d_s || !d_f || !d_x) {
        set_global_error("no-alloc path: d_s, d_f and d_x must be non-NULL");
        return SFSEG_EINVAL;
    }
    if (n_iters < 1) {
        set_global_error("no-alloc path: n_iters must be >= 1");
        return SFSEG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t elt = prm->storage == SFSEG_F32 ? 4 : 2;
    VideoGeom g;
    g.nf = prm->nf;
    g.h = prm->h;
    g.w = prm->w;
    g.pitch = (g.w + 7) / 8 * 8;
    g.plane = (long long)g.h * g.pitch;
    g.off = 0;
    g.n = (long long)g.nf * g.h * g.w;
    int tx, ty;
    generic_tile(&tx, &ty);
    const int tiles_x = (g.w + tx - 1) / tx, tiles_y = (g.h + ty - 1) / ty;
    const long long n_items_ll = (long long)tiles_x * tiles_y;
    const size_t vol = up256((size_t)g.nf * (size_t)g.plane * elt);
    const int prep_blocks = prep_x_blocks(g.n);

    // carve the scratch array: [header | prep partials | trace | items | partials | 4 volumes]
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += up256(bytes); return o; };
    const size_t o_geo = take(sizeof(VideoGeom));
    const size_t o_state = take(sizeof(VState));
    const size_t o_ib = take(2 * sizeof(int));
    const size_t o_cnt = take(sizeof(unsigned));
    const size_t o_pcnt = take(sizeof(unsigned));
    const size_t o_bad = take(sizeof(int));
    const size_t o_out = take(sizeof(float*));
    const size_t zero_end = off;                       // bytes [0, zero_end) start at zero
    const size_t o_pp = take(sizeof(double) * prep_blocks);
    const size_t o_trace = take(sizeof(double) * 3 * kTraceCap);
    const size_t o_items = take(sizeof(WorkItem) * (size_t)n_items_ll);
    const size_t o_part = take(sizeof(double) * kRed * (size_t)n_items_ll);
    const size_t o_sp = take(vol), o_f = take(vol), o_xa = take(vol), o_xb = take(vol);
    if (off > kScratchBytes || (long long)g.nf * g.plane > (1LL << 40)) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "no-alloc path: a %dx%dx%d volume needs %zu bytes of workspace; "
                 "the fixed array holds %zu (use sfseg_create for larger volumes)",
                 g.nf, g.h, g.w, off, kScratchBytes);
        set_global_error(msg);
        return SFSEG_EINVAL;
    }
    void* base = nullptr;
    st = scratch_address(&base);
    if (st != SFSEG_OK) return st;
    unsigned char* B = (unsigned char*)base;

    StepParams P{};
    P.sp = B + o_sp;
    P.f = B + o_f;
    P.nchan = 1;
    P.geo = (const VideoGeom*)(B + o_geo);
    P.state = (VState*)(B + o_state);
    P.items = (const WorkItem*)(B + o_items);
    P.item_begin = (const int*)(B + o_ib);
    P.partials = (double*)(B + o_part);
    P.counters = (unsigned*)(B + o_cnt);
    P.trace = (double*)(B + o_trace);
    P.trace_cap = kTraceCap;
    P.n_items = (int)n_items_ll;
    P.alpha = (float)prm->alpha;
    P.rt = prm->rt;
    P.ry = prm->ry;
    P.rx = prm->rx;
    double gsum = 1.0;
    {
        const int radii[3] = {prm->rt, prm->ry, prm->rx};
        const double sig[3] = {prm->sigma_t, prm->sigma_y, prm->sigma_x};
        float* taps[3] = {P.gt, P.gy, P.gx};
        for (int a = 0; a < 3; ++a) {
            double sum = 0.0;
            for (int d = -radii[a]; d <= radii[a]; ++d) {
                const float v = (float)std::exp(-(double)d * d / (2.0 * sig[a] * sig[a]));
                taps[a][d + radii[a]] = v;
                sum += (double)v;
            }
            gsum *= sum;
        }
    }

#define NA_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) {                                       \
            set_global_error(cudaGetErrorString(e_));                  \
            return SFSEG_ECUDA;                                        \
        }                                                              \
    } while (0)

    // The array keeps the previous call's contents: reset the counters and flags.
    NA_CUDA(cudaMemsetAsync(B, 0, zero_end, s));
    noalloc_init_kernel<<<(int)((n_items_ll + 255) / 256), 256, 0, s>>>(
        g, (VideoGeom*)(B + o_geo), (WorkItem*)(B + o_items), (int*)(B + o_ib), tiles_x,
        (int)n_items_ll, tx, ty);
    NA_CUDA(cudaPeekAtLastError());

    PrepFeatParams F{};
    F.s = d_s;
    F.f = d_f;
    F.sp_out = B + o_sp;
    F.f_out = B + o_f;
    F.chan_stride = 0;
    F.g = g;
    F.nchan = 1;
    F.p = (float)prm->p;
    F.s_is_sp = (prm->flags & SFSEG_S_IS_SP) ? 1 : 0;
    F.bad = (int*)(B + o_bad);
    NA_CUDA(launch_prep_features(prm->storage, F, s));

    PrepXParams X{};
    X.x = d_x;
    X.x_out = B + o_xa;
    X.g = g;
    X.video = 0;
    X.raw = 0;
    X.gain0 = std::exp2(std::rint(std::log2(std::sqrt((double)g.n) / gsum)));
    X.tol = 0.0;
    X.bad_features = (const int*)(B + o_bad);
    X.state = P.state;
    X.partials = (double*)(B + o_pp);
    X.counter = (unsigned*)(B + o_pcnt);
    NA_CUDA(launch_prep_x(prm->storage, X, prep_blocks, s));

    for (int k = 0; k < n_iters; ++k) {
        const bool last = (k == n_iters - 1);
        P.x_in = (k & 1) ? B + o_xb : B + o_xa;
        P.z_out = last ? nullptr : ((k & 1) ? B + o_xa : B + o_xb);
        P.final_out = last ? (float* const*)(B + o_out) : nullptr;
        if (last) NA_CUDA(launch_set_ptrs((float**)(B + o_out), &d_x, 1, s));
        NA_CUDA(launch_step_generic(prm->storage, P, (int)n_items_ll, s));
    }
    FinishParams Fin{};
    Fin.out = d_x;
    Fin.buf0 = B + o_xa;
    Fin.buf1 = B + o_xb;
    Fin.g = g;
    Fin.state = P.state;
    Fin.video = 0;
    Fin.final_iter = n_iters;
    NA_CUDA(launch_finish(prm->storage, Fin, s));
    if (d_trace) {
        const int rows = n_iters < kTraceCap ? n_iters : kTraceCap;
        NA_CUDA(cudaMemcpyAsync(d_trace, B + o_trace, sizeof(double) * 3 * rows,
                                cudaMemcpyDeviceToDevice, s));
    }
#undef NA_CUDA
    return SFSEG_OK;
}
