// Library-internal state shared by the C-ABI translation units: device
// buffers, the context, and the per-frame view of the buffers that one
// render / backward pass reads and writes.
#pragma once

#include <cstdarg>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/facert.h"
#include "kernels.cuh"

namespace fr {

// Device buffer owned by the context.
template <class T> struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  void free_() { if (p) cudaFree(p); p = nullptr; n = 0; }
  cudaError_t alloc(size_t count) {
    free_();
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e == cudaSuccess) n = count;
    return e;
  }
};

struct DevBVH {
  DBuf<float4> nodes, cones;
  DBuf<int> leaf_first, leaf_count, leaf_parent, leaf_slot, node_parent, node_slot, counter;
  int n_nodes = 0, n_leaves = 0;
};

}  // namespace fr

using fr::DBuf;
using fr::DevBVH;
using fr::Light;
using fr::CS;

constexpr int NCOUNT = fr::CNT_TOTAL;   // work counters: 6 per render kernel
constexpr int NPHASE = 8;    // timed phases
enum { PH_GEOMETRY = 0, PH_FORWARD, PH_INTERIOR, PH_PEDGE, PH_SEDGE, PH_ADJOINT, PH_LOSS, PH_SEDGE_ADD };

struct fr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  fr_config cfg;
  std::string err;
  std::vector<Light> lights;
  // mesh
  int V = 0, F = 0, E = 0;
  bool have_mesh = false, have_bases = false;
  uint64_t generation = 0;   // counts mesh and basis uploads (a batch is tied to one)
  DBuf<float> mean, uv;
  DBuf<int4> tris, edges_canon, edges_leaf;
  DBuf<int> vf_off, vf_idx, tri_perm, edge_id_leaf;
  DevBVH tbvh, ebvh;
  // the edge hierarchy collapsed to 4 children per node (fixed topology) and
  // the gather table of its child slots from the binary one
  int n4 = 0;
  DBuf<int4> e4codes;
  DBuf<int2> e4src;
  DBuf<float2> e4boxes;
  DBuf<float4> e4cones;
  // bases
  int K_id = 0, K_exp = 0, K_alb = 0;
  DBuf<float> BidT, BexpT, alb_mean, BalbT;
  // per-render state
  DBuf<float4> X, Xm, alb, nrm, ng, tv, epack;
  DBuf<int> sil, n_sil, block_count, err_flag;
  DBuf<unsigned long long> counters;
  bool counters_on = false;
  // device limits (fr_set_limits)
  int max_steps = fr::DEFAULT_MAX_STEPS;
  int wait_limit = fr::DEFAULT_WAIT_LIMIT;
  uint64_t launches = 0;
  // per-phase timing (fr_set_timing): geometry, forward, interior, primary
  // edges, shadow edges, adjoint, loss
  bool timing_on = false, events_made = false;
  cudaEvent_t ev[NPHASE][2];
  bool phase_used[NPHASE] = {false};
  // NVTX ranges around the host-side enqueue of each phase (a profiler that
  // records NVTX shows them; otherwise they cost a few nanoseconds).  A
  // phase left open by an error return is closed when it is entered again.
  bool nvtx_open[NPHASE] = {false};
  void mark(int phase, int end) {
    static const char* const names[NPHASE] = {"facert geometry", "facert forward", "facert interior",
                                              "facert primary edges", "facert shadow-edge search", "facert adjoint",
                                              "facert loss", "facert shadow-edge contributions"};
    if (nvtx_open[phase]) { nvtxRangePop(); nvtx_open[phase] = false; }
    if (!end) { nvtxRangePushA(names[phase]); nvtx_open[phase] = true; }
    if (!timing_on) return;
    cudaEventRecord(ev[phase][end], stream);
    if (end) phase_used[phase] = true;
  }
  // gradient accumulators
  DBuf<float4> dX, dN, dA, gs;
  DBuf<float> dXm, dC, dL;
  DBuf<int2> hits;        // primary hit per tiled sample (backward)
  DBuf<int2> picks;       // shadow-edge pick per (light, tiled sample): (candidates, leaf slot)
  DBuf<float> aov_scratch;  // mean luminance per pixel (feature output, atomic path)
  DBuf<float> dimg;       // dE_data/d image of fr_step when the caller passes none
  // denoiser: FP32 master weights, Adam moments, gradients, training scratch
  DBuf<float> mlp_w, mlp_m, mlp_v, mlp_g, mlp_scratch;
  bool have_mlp = false;
  int mlp_steps = 0;
  int n_params() const { return K_id + K_exp + K_alb + CS * CS + 6 + 3 * cfg.n_lights; }
  int off_cspec() const { return K_id + K_exp + K_alb; }
  int off_pose() const { return off_cspec() + CS * CS; }
  int off_lights() const { return off_pose() + 6; }
};

namespace fr {

// Buffers of one frame: posed mesh, BVH boxes (topology from the context),
// packed edges, camera silhouettes and the per-vertex gradient accumulators.
// The single-image entry points use the context's own buffers
// (main_view); a batch gives every frame its own.
struct FrameView {
  float4 *X, *Xm, *alb, *nrm, *ng, *tv, *epack;
  float4 *tnodes, *tcones, *enodes, *econes;
  float2* e4boxes;         // 4-wide edge hierarchy: child boxes and cones
  float4* e4cones;
  int *tcounter, *ecounter;
  int *sil, *n_sil, *block_count;
  float4 *dX, *dN, *dA, *gs;
  float *dXm, *dC, *dL;
};

FrameView main_view(fr_ctx* c);
int fail(fr_ctx* c, int code, const char* fmt, ...);
GeoArgs geo_args(fr_ctx* c, const FrameView& v);
Cam make_cam(const fr_ctx* c, int W, int H);
int prepare_geometry(fr_ctx* ctx, const float* theta, const FrameView& v);
int silhouettes(fr_ctx* ctx, const FrameView& v);
RenderArgs render_args(fr_ctx* c, const float* theta, const fr_render_opts* o, const FrameView& v);
// Geometry adjoint: dN -> dX, R^T, pose gradient, transposed basis
// contractions, specular-map and light accumulators -> grad (added).
// with_alb = 0 leaves the albedo term (dA) out.
int adjoint(fr_ctx* ctx, const float* theta, const FrameView& v, double* grad, bool with_alb);
inline unsigned grid_for(long long threads, int block) { return (unsigned)((threads + block - 1) / block); }

}  // namespace fr

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? FR_ERR_OOM : FR_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                          \
  } while (0)

#define CKL()                                                                                 \
  do {                                                                                        \
    ++ctx->launches;                                                                          \
    cudaError_t e_ = cudaGetLastError();                                                      \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, FR_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

