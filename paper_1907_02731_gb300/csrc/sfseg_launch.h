// sfseg_launch.h -- host-side launchers of the SFSeg kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "sfseg.h"
#include "sfseg_common.cuh"

namespace sfseg {

// ------------------------------------------------------------- prepare
struct PrepFeatParams {
    const float* s;             // caller [nf][h][w] FP32
    const float* f;             // caller [nchan][nf][h][w] FP32
    void* sp_out;               // internal pitched, storage type
    void* f_out;                // internal pitched, storage type ([nchan] volumes)
    long long chan_stride;      // elements between channel volumes of f_out
    VideoGeom g;
    int nchan;
    float p;
    int s_is_sp;
    int* bad;                   // set to 1 if a non-finite input is seen
    unsigned* fmin_key;         // [nchan] float_key of the minimum of the stored f (all ones before)
    unsigned* fmax_key;         // [nchan] float_key of the maximum (zero before); both may be null
};

struct PrepXParams {
    const float* x;             // caller [nf][h][w] FP32
    void* x_out;                // internal pitched, storage type
    VideoGeom g;
    int video;
    int raw;                    // 1: scale = gain = 1 (unnormalised apply)
    double gain0;               // first step's gain
    double tol;
    const int* bad_features;    // nullable
    VState* state;
    double* partials;           // [gridDim.x]
    unsigned* counter;
    double* rec_scale0;         // nullable: receives the scale of x^0 (forward record)
    // slab of a video split along t: only frames [norm_t0, norm_t1) count in
    // the norm, and the sum of x^2 goes to *ext_sum (the state is set later
    // from the sum over all ranks); ext_sum null = the whole volume, state set
    double* ext_sum;
    int norm_t0, norm_t1;
};

// Scalar state of a slab (one rank's frames of a video split along t):
// mode 0 starts the iteration from the global sum of x0^2 (sums[0]); mode 1
// finalizes a power step from the global step sums (sums[0..kRed)).
cudaError_t launch_slab_state(VState* st, const double* sums, int mode, double gain0, long long n_video,
                              double* trace, int trace_cap, cudaStream_t s);

// Up to kMax device pointers passed by value to a tiny kernel that writes
// them into a device array (safe inside stream order, no host staging).
struct PtrPack {
    static constexpr int kMax = 64;
    int base, n;
    float* p[kMax];
};

struct FinishParams {
    float* out;                 // caller [nf][h][w] FP32
    const void* buf0;           // packed stored iterates
    const void* buf1;
    VideoGeom g;
    const VState* state;
    int video;
    int final_iter;             // iter value meaning "the last step wrote `out`"
};

cudaError_t launch_prep_features(int storage, const PrepFeatParams& P, cudaStream_t s);
cudaError_t launch_prep_x(int storage, const PrepXParams& P, int blocks, cudaStream_t s);
cudaError_t launch_finish(int storage, const FinishParams& P, cudaStream_t s);

// binarisation (Alg. 1 Step 3): projection of a video's stored iterate, and
// the final threshold of the caller's FP32 result
struct ProjectParams {
    void* buf;                  // packed stored iterate (storage type), projected in place
    VideoGeom g;
    VState* state;
    int video;
    float beta, tau;            // p = 1 / (1 + exp(-beta (x / max x - tau)))
    unsigned* vmax_key;         // order-preserving key of max x (0 before the call)
    double* partials;           // [n_blocks]
    int n_blocks;
};
cudaError_t launch_project(int storage, const ProjectParams& P, cudaStream_t s);
cudaError_t launch_threshold(const float* x, long long n, unsigned* key, float theta, unsigned char* mask,
                             int n_blocks, cudaStream_t s);
cudaError_t launch_set_ptrs(float** dst, float* const* src, int n, cudaStream_t s);
int prep_x_blocks(long long n);

// --------------------------------------------------------------- adjoint
struct AdjParams {
    const float* g_in;          // g_{k+1} = dL/dx^{k+1}, pitched FP32
    float* g_out;               // g_k, pitched FP32
    const float* x_next;        // stored x^{k+1} (FP32), unit norm after * s_next
    const float* x_cur;         // stored x^k (FP32), unit norm after * s_cur
    const float* sp;            // internal FP32 sp
    const float* f;             // internal FP32 f
    float* dsp;                 // pitched FP32 accumulators (+=)
    float* df;
    const VideoGeom* geo;
    const double* s_next;       // device scalars
    const double* s_cur;
    const double* ny;           // ||M x^k||, unit-norm x^k
    const double* c_in;         // x^{k+1} . g_{k+1}
    double* c_out;              // receives x^k . g_k
    const WorkItem* items;      // generic 32 x 16 tiles over all frames (one per CTA)
    double* partials;           // [n_items]
    unsigned* counter;
    float alpha;
    int rt, ry, rx;
    float gt[2 * kMaxRt + 1];
    float gy[2 * kMaxR + 1];
    float gx[2 * kMaxR + 1];
};

// reverse step on the specialised forward kernel (adjoint.cu)
struct AdjCombineParams {
    const float* u;             // u_k (pitched FP32)
    const float* x_cur;         // stored x^k
    const float* sp;
    const float* ku;            // K_U, F_U of the forward kernel run on u_k
    const float* fu;
    const float* kx;            // K_X, F_X of the recomputed step k (stored x^k)
    const float* fx;
    float* dsp;                 // accumulators (+=)
    float* df;
    const double* s_cur;        // x^k = s_cur * stored x^k
    double* c_out;              // receives x^k . g_k
    double* partials;           // [blocks]
    unsigned* counter;          // 0 before the call, 0 after
    VideoGeom g;
    float alpha;
};
cudaError_t launch_uprep(const float* g_in, const float* x_next, const double* s_next, const double* c,
                         const double* ny, float* u_out, const VideoGeom& g, int blocks, cudaStream_t s);
cudaError_t launch_adj_combine(const AdjCombineParams& P, int blocks, cudaStream_t s);

size_t adjoint_smem_bytes(int rt, int ry, int rx);
cudaError_t setup_adjoint(int rt, int ry, int rx);
cudaError_t launch_adjoint(const AdjParams& P, int n_items, cudaStream_t s);
cudaError_t launch_dot(const float* x, const double* scale_x, const float* gv, const VideoGeom& g,
                       double* partials, unsigned* counter, double* out, int blocks, cudaStream_t s);
cudaError_t launch_pitch_copy(const float* src, float* dst, const VideoGeom& g, int to_pitched,
                              const double* scale, cudaStream_t s);
cudaError_t launch_set_state(VState* st, const double* scale, const double* gain, int iter,
                             cudaStream_t s);

// ---------------------------------------------------------- host helpers
// Parameter validation of sfseg_create, and the message slot that
// sfseg_last_error(NULL) returns (for entry points without a context).
sfseg_status validate_params(const sfseg_params* p);
void set_global_error(const char* msg);

// ---------------------------------------------------------------- steps
size_t generic_smem_bytes(int rt, int ry, int rx, int nchan = 1);
size_t generic_smem_cap();
void generic_tile(int* tx, int* ty);
cudaError_t setup_step_generic(int rt, int ry, int rx);
cudaError_t launch_step_generic(int storage, const StepParams& P, int n_items, cudaStream_t s);

// Specialised kernel for radii (2,5,5), (3,3,3), (2,4,4): 128 x 16 tiles,
// persistent CTAs of 512 threads over balanced segment lists, TMA loads.
bool fast_available(int rt, int ry, int rx, int storage);
void fast_tile(int* tx, int* ty, int* threads);
void fast_box(int ry, int* box_w, int* box_h, int* x_pad);   // TMA box of one stage array
cudaError_t setup_step_fast(int rt, int ry, int rx, int storage);
cudaError_t launch_step_fast(int storage, const StepParams& P, int n_ctas, cudaStream_t s);

// ------------------------------------------------------- fused multi-step
// All K power steps of a context in one cooperative launch (step_fused.cu):
// per step a phase of y/x passes into an FP32 scratch, a grid barrier, a
// phase of t-pass + combine + reductions + finalize, a grid barrier.
struct FusedParams {
    StepParams S;               // taps, alpha, geo, sp, f, state, trace, final_out; items /
                                // cta_begin / item_begin / vseg / partials / counters describe
                                // the phase-2 runs (item t0..t1 = unit range of its video)
    const void* buf0;           // stored iterate of even steps (x_a)
    void* buf1;                 // stored iterate of odd steps (x_b)
    float* pvol;                // scratch: 3 FP32 volumes (packed pitched layout), channel c at + c * total
    long long total;            // packed elements per volume
    const int* unit1_begin;     // [n_videos + 1]: phase-1 units (frame x 32x16 tile) of video v
    int n_units1;
    int n_videos;
    int n_steps;                // K
    int final_mode;             // the last step writes the caller's FP32 buffers (S.final_out)
    unsigned* bar;              // [3]: barrier arrival count, (unused), abort flag (zero before the launch)
};

// rows of one phase-2 unit of the fused kernel for a video of width w
__host__ __device__ inline int fused_rows2(int w) {
    const int r = 1024 / (w > 0 ? w : 1);
    return r < 1 ? 1 : r;
}

// ------------------------------------------------------------- cluster
// All K steps of one small video in one thread-block cluster (step_cluster.cu).
struct ClusterParams {
    StepParams S;               // taps, alpha, geo, sp, f, state, trace, final_out (video 0)
    const void* buf0;           // stored x0 (x_a); the result goes to buf0 / buf1 by iter parity
    void* buf1;                 // x_b
    int n_steps;                // K
    int final_mode;             // the last step writes the caller's FP32 buffer (S.final_out[0])
    int tiles_x;                // tile columns of the cluster (CTA rank = ty * tiles_x + tx)
    int th;                     // tile height (a multiple of 8); tiles are 16 columns wide
};
struct ClusterPlan {
    int n_ctas;                 // CTAs of the one cluster (at most 16)
    int tiles_x, th;
    size_t smem;                // dynamic shared memory per CTA
};
bool plan_step_cluster(int storage, int rt, int ry, int rx, int nf, int h, int w, ClusterPlan* out);
cudaError_t launch_step_cluster(int storage, const ClusterParams& C, const ClusterPlan& plan, cudaStream_t s);

size_t fused_smem_bytes(int ry, int rx);
void fused_tile(int* tx, int* ty, int* threads);
cudaError_t setup_step_fused(int storage, int ry, int rx, int* max_ctas);
cudaError_t launch_step_fused(int storage, const FusedParams& F, int n_ctas, cudaStream_t s);

}  // namespace sfseg
