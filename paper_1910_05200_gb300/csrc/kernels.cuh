// Kernel argument structures and declarations of the facert CUDA kernels.
#pragma once

#include "common.cuh"

namespace fr {

struct GeoArgs {
  int V, F, K_id, K_exp, K_alb, off_pose;
  const float* mean;      // [3V]
  const float* BidT;      // [K_id][3V]
  const float* BexpT;     // [K_exp][3V]
  const float* alb_mean;  // [3V]
  const float* BalbT;     // [K_alb][3V]
  const int4* tris;       // [F]
  const int* tri_perm;    // leaf slot -> face id
  const int* vf_off;      // [V+1] vertex -> incident faces (CSR)
  const int* vf_idx;
  float4* X;              // posed vertices
  float4* Xm;             // model-space vertices
  float4* alb;            // albedo
  float4* nrm;            // unit vertex normals, w = 1/|sum|
  float4* ng;             // decision-form face normals
  float4* tv;             // leaf-ordered triangle vertices
};

struct RefitArgs {
  int n_leaves;
  const int* leaf_first;
  const int* leaf_count;
  const int* leaf_parent;
  const int* leaf_slot;
  const int* node_parent;
  const int* node_slot;
  int* counter;           // [n_nodes], zeroed before the launch
  float4* nodes;
  int is_edge;
  const float4* tv;       // triangles (is_edge = 0)
  const int4* edges;      // leaf-ordered edges (is_edge = 1)
  const float4* X;
  const float4* pack;     // packed edge records (is_edge = 1): face normals for the cones
  float4* cones;          // [n_nodes * 2] normal cone per child slot (is_edge = 1)
};

struct SilArgs {
  int E;
  const int4* edges;      // canonical order (v0, v1, f0, f1)
  const int4* tris;
  const float4* ng;
  const float4* X;
  V3 cam_o;
  int* block_count;
  int* sil;
  int* n_sil;
};

struct EdgeBVH {
  BVHView bvh;
  const int4* edges;      // leaf-ordered (v0, v1, f0, f1)
  const int* edge_id;     // leaf slot -> canonical edge id
  const float4* pack;     // leaf-ordered packed records, 6 float4 per edge
  const int4* verts;      // same as edges (v0, v1 read by the adjoint)
  const float4* cones;    // [n_nodes * 2] normal cones of the faces below each child
  // the same hierarchy collapsed to 4 children per node (grandchildren of a
  // binary node become its children), searched by the shadow-edge pass
  const int4* codes4;     // [n4] child codes: leaf code, 4-wide node index or EMPTY_CHILD
  const float2* boxes4;   // [n4 * 12] child c: lo.xy | lo.z, hi.x | hi.yz at float2 12k + 3c
  const float4* cones4;   // [n4 * 8] child c at 8k + 2c: normal cone (axis, cos of the half-angle
                          // grown by 2e-3; -1 from pi/2 on), then the bounding sphere of its box
                          // (centre, radius)
};

struct RenderArgs {
  int W, H, spp;
  uint32_t seed, iter;
  int n_lights;
  float side, eps_pedge, eps_sedge, tmin, kappa;
  Brdf brdf;
  Cam cam;
  Light lights[MAX_LIGHTS];
  Mesh mesh;
  EdgeBVH ebvh;
  const float4* nrm;
  const float4* alb;
  const float2* uv;
  const float* cspec;     // theta + off_cspec
  const float* lights_dev;// theta + off_lights
  const int* sil;         // camera silhouette edges
  const int* n_sil;
  const int4* edges_canon;
  int* err;
  float* aov_scratch;     // [W*H] mean luminance for the atomic AOV path
  unsigned long long* counters;  // [CNT_TOTAL] or null: CNT_PER_KERNEL per kernel (fwd, interior, pedge, sedge)
};

struct GradBufs {
  float4* dX;             // [V]
  float4* dN;             // [V]
  float4* dA;             // [V]
  float* dC;              // [1024]
  float* dL;              // [3N]
  const float* d_image;   // [H*W*3]
  int2* hits;             // per tiled sample: (face or -1, t bits), written by k_bwd_interior or k_step_fwd
};

// One frame of a batch: the render arguments and gradient buffers of that
// frame plus its image, adjoint, target and loss slots (device table).
struct BatchFrame {
  RenderArgs a;           // a.iter is replaced by *BatchArgs::iter
  GradBufs gb;            // gb.d_image is this frame's adjoint; gb.hits its samples' primary hits, in the
                          // sample order of the launch mode (8x8 tiles phased, tile items persistent)
  float* image;           // [H*W*3]
  float* d_image;         // [H*W*3], written by the frame's tile items
  const float* target;    // [H*W*3]
  const uint8_t* mask;    // [H*W] or null
  double* loss;           // E_data of the frame (added)
  int tiles_x, n_tiles;
  long long n_pedge;      // primary-edge samples: W*H*spp
};

// Work items of the persistent kernel, in queue order: tile items (frame,
// tile), then shadow-edge items (frame | SEDGE_ITEM, chunk << SEDGE_LIGHT_BITS
// | light) light-major within each frame, then primary-edge items (frame |
// PEDGE_ITEM, chunk); frames in the same order in each group.
constexpr int PEDGE_ITEM = 1 << 30;
constexpr int SEDGE_ITEM = 1 << 29;
constexpr int SEDGE_LIGHT_BITS = 5;
constexpr int SEDGE_LIGHTS = 1 << SEDGE_LIGHT_BITS;
static_assert(MAX_LIGHTS <= SEDGE_LIGHTS, "a light index must fit the shadow-edge item's light bits");
// Samples per shadow-edge item and per primary-edge item (multiples of 32).
// Short items keep the warps that run at the same time on one light of one
// frame and leave a short tail; on 32 frames of the full face, 32 samples
// beat 64, 128, 256 and 1024 for both kinds.
constexpr int BATCH_SEDGE_CHUNK = 32;
constexpr int BATCH_PEDGE_CHUNK = 32;
// Default spin limit of an edge item waiting for its frame's tiles
// (__nanosleep(256) per try: about a second); fr_set_limits changes it.
constexpr int DEFAULT_WAIT_LIMIT = 1 << 22;

struct BatchArgs {
  const BatchFrame* frames;
  const int2* items;
  int n_items;
  int tile_w, tile_h;     // pixels per tile item
  int pedge_chunk;        // edge samples per primary-edge item
  int sedge_chunk;        // camera samples per shadow-edge item (a multiple of 32)
  int* queue;             // next item, zeroed before the launch
  int* tiles_done;        // [n_frames], zeroed before the launch
  const uint32_t* iter;
  int* err;
  unsigned long long* counters;  // [CNT_TOTAL] or null, same layout as the single-image kernels
  int max_steps;          // traversal step cap of every frame
  int wait_limit;         // tries of an edge item waiting for its frame's tiles
};

// Phase kernels of a batch (one launch per phase for all frames): block b of
// the launch belongs to the frame f with block_start[f] <= b <
// block_start[f + 1]; frames are laid out one after another so that the
// blocks of one frame run together and its structures stay in L2.
struct PhaseArgs {
  const BatchFrame* frames;
  const int* block_start;   // [n_frames + 1]
  int n_frames;
  const uint32_t* iter;
  int* err;
  unsigned long long* counters;  // [CNT_TOTAL] or null
  int max_steps;            // traversal step cap of every frame
  int2* picks;              // shadow-edge picks, one per thread of the shadow-edge launches
};

// Per-warp slice of k_batch_step's dynamic shared memory: the arguments of
// the frame the warp works on and its light-gradient accumulator.
struct BatchWarpState {
  RenderArgs a;
  GradBufs g;
  float sL[3 * MAX_LIGHTS];
};
// Dynamic shared memory of k_batch_step: the block's specular-map
// accumulator, then one BatchWarpState per warp.
FR_HOST_DEV inline size_t batch_smem_head() { return (sizeof(float) * CS * CS + 15) & ~(size_t)15; }
FR_HOST_DEV inline size_t batch_smem_bytes(int block) {
  return batch_smem_head() + (size_t)(block / 32) * sizeof(BatchWarpState);
}

// forward + loss + interior adjoint (spp dividing 256), blocks of 256 threads
// over each frame's samples in 8x8-tile order; writes gb.hits for the
// shadow-edge phase
__global__ void k_batch_fwd(PhaseArgs p);
// shadow edges: per frame n_lights x (that frame's forward blocks), light-major;
// the search and pick (3 or 4 resident blocks per SM), then the contributions
__global__ void k_batch_sedge3(PhaseArgs p);
__global__ void k_batch_sedge4(PhaseArgs p);
__global__ void k_batch_sedge_add(PhaseArgs p);
// primary edges: blocks of 256 over each frame's W*H*spp edge samples
__global__ void k_batch_pedge(PhaseArgs p);
__global__ void k_batch_step2(BatchArgs b);
__global__ void k_batch_step3(BatchArgs b);
__global__ void k_batch_step4(BatchArgs b);
__global__ void k_batch_gather_theta(int n_frames, int P, int K_id, int K_exp, int K_alb, int n_light_vals,
                                     const float* __restrict__ ts, const float* __restrict__ tf,
                                     float* __restrict__ theta);
__global__ void k_batch_reduce(int n_frames, int P, int K_id, int K_exp, int K_alb, int n_light_vals,
                               const float* __restrict__ theta, const double* __restrict__ grad_full,
                               const double* __restrict__ loss_frames, int prior, const float* __restrict__ m, float w1,
                               float w2, double* __restrict__ grad_s, double* __restrict__ grad_f,
                               double* __restrict__ loss);

__global__ void k_geometry(GeoArgs g, const float* __restrict__ theta);
__global__ void k_faces(GeoArgs g);
__global__ void k_pack_edges(int E, const int4* __restrict__ edges_leaf, const int* __restrict__ edge_id,
                             const int4* __restrict__ tris, const float4* __restrict__ X,
                             const float4* __restrict__ ng, float4* __restrict__ pack);
__global__ void k_vertex_normals(GeoArgs g);
__global__ void k_refit(RefitArgs r);
// Boxes and cones of the 4-wide edge hierarchy from the refitted binary one:
// slot i takes (binary node, slot) src[i]; src.x < 0 marks an empty slot.
__global__ void k_gather4(int n_slots, const int2* __restrict__ src, const float4* __restrict__ nodes,
                          const float4* __restrict__ cones, float2* __restrict__ boxes4, float4* __restrict__ cones4);
__global__ void k_silhouette_flags(SilArgs s);
__global__ void k_silhouette_scan(SilArgs s, int nblocks);
__global__ void k_silhouette_scatter(SilArgs s);
__global__ void k_normals_bwd_vertex(GeoArgs g, const float4* __restrict__ dN, float4* __restrict__ gs);
__global__ void k_normals_bwd_gather(GeoArgs g, const float4* __restrict__ gs, float4* __restrict__ dX);
__global__ void k_pose_bwd(GeoArgs g, const float* __restrict__ theta, const float4* __restrict__ dX,
                           float* __restrict__ dXm, double* __restrict__ grad);
// k_geometry: vertices per block, column groups, threads per block;
// k_basis_T: slices per basis row (grid (K, BASIS_SLICES)).
constexpr int GEO_VERTS = 32, GEO_KSPLIT = 4, GEO_THREADS = 3 * GEO_VERTS * GEO_KSPLIT, BASIS_SLICES = 16;
__global__ void k_basis_T(const float* __restrict__ BT, int K, int n, const float* __restrict__ y,
                          const float4* __restrict__ y4, double* __restrict__ grad, int out_off);
__global__ void k_add_small(const float* __restrict__ src, int n, double* __restrict__ grad, int off);

__global__ void k_render_fwd(RenderArgs a, float* __restrict__ image);
__global__ void k_render_fwd_aov(RenderArgs a, float* __restrict__ image, float* __restrict__ aov);
__global__ void k_aov_finish(int n_pix, float* __restrict__ aov, const float* __restrict__ meanY);
__global__ void k_bwd_interior(RenderArgs a, GradBufs gb);
// Outputs and loss inputs of the fused single-image step (k_step_fwd).
struct StepBufs {
  float* image;           // [H*W*3]
  float* d_image;         // [H*W*3] dE_data/d image, read by the edge passes
  const float* target;    // [H*W*3]
  const uint8_t* mask;    // [H*W] or null
  double* loss;           // E_data is added
  int interior;           // run the interior adjoint
};
__global__ void k_step_fwd(RenderArgs a, GradBufs gb, StepBufs sb);
__global__ void k_bwd_pedge(RenderArgs a, GradBufs gb);
// Shading points per thread of the single-image shadow-edge search (a warp's
// 32 NS samples share one walk of the edge hierarchy): 2 from 256 x 256
// pixels up, 1 below.  Two points per lane halve the walks but widen the
// group, which pays only where pixels are small: on the full face at
// 256 x 256 x 16 the search takes 7.14 ms with 2 against 7.33 ms with 1,
// at 128 x 128 (pixels twice the size) 4.81 against 4.10 ms.
constexpr long long SEDGE_NS2_MIN_PIXELS = 256 * 256;
// Shadow edges: the search and pick per (light, sample), stored in picks
// [n_lights * tiled samples] as (candidates, leaf slot); then the boundary
// contributions of the picks.
__global__ void k_bwd_sedge(RenderArgs a, GradBufs gb, int2* __restrict__ picks);     // two points per lane
__global__ void k_bwd_sedge_1(RenderArgs a, GradBufs gb, int2* __restrict__ picks);   // one point per lane
__global__ void k_bwd_sedge_add(RenderArgs a, GradBufs gb, const int2* __restrict__ picks);

__global__ void k_loss_data(int n_pix, const float* __restrict__ image, const float* __restrict__ target,
                            const uint8_t* __restrict__ mask, double* __restrict__ loss, float* __restrict__ d_image);
__global__ void k_loss_reg(const float* __restrict__ theta, int n_prior, int off_lights, int n_light_vals,
                           int prior, const float* __restrict__ m, float w1, float w2, double* __restrict__ loss,
                           double* __restrict__ grad);

// m of E_light (Eq. 1) for light value i = 3 j + c of the n lights l[3n]:
// prior 0 the caller's m (zero when null), 1 the mean of the lights in
// channel c, 2 the mean of light j's channels.  FP64, summed in index order.
__device__ inline double light_prior_mean(const float* __restrict__ l, int n, int prior,
                                          const float* __restrict__ m, int i) {
  if (prior == 1) {
    const int c = i % 3;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += (double)l[3 * k + c];
    return s / (double)n;
  }
  if (prior == 2) {
    const int j = i / 3;
    return ((double)l[3 * j] + (double)l[3 * j + 1] + (double)l[3 * j + 2]) / 3.0;
  }
  return m ? (double)m[i] : 0.0;
}

// denoiser (denoise.cu)
__global__ void k_mlp_infer(int n_pix, const float* __restrict__ w, const float* __restrict__ aov,
                            float* __restrict__ out, const float* __restrict__ d_out, float* __restrict__ d_rgb);
__global__ void k_mlp_train_tc(int n_pix, const float* __restrict__ w, const float* __restrict__ aov,
                               const float* __restrict__ target, float* __restrict__ scratch, double* __restrict__ loss);
__global__ void k_mlp_wgrad(int n_pix, const float* __restrict__ scratch, int g_off, int h_off, int N, int K, int Kw,
                            float* __restrict__ dW, float* __restrict__ db, int chunk);
__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2);
__global__ void k_adam_theta(int n, float* __restrict__ theta, const double* __restrict__ grad,
                             float* __restrict__ m, float* __restrict__ v, const float* __restrict__ lr, float c1,
                             float c2, int off_cspec, int n_cspec, int off_lights);
int mlp_n_weights();
size_t mlp_smem_bytes();
int mlp_train_stride();
void mlp_layer_offsets(int* off);

// Pixel order: 8x8 tiles, row-major tiles, Z-order within a tile (bits of
// the in-tile index interleave x and y), so that any aligned run of 2^k
// pixels -- the pixels of one warp's samples -- is a compact block (4x2 at 4
// spp, 2x2 at 8 spp): the warp-wide shadow-edge search works on a small
// group of shading points.  Returns false for pixels outside the image.
FR_DEV bool tile_pixel(int idx, int W, int H, int& px, int& py) {
  int tiles_x = (W + 7) >> 3;
  int tile = idx >> 6, in = idx & 63;
  int tx = tile % tiles_x, ty = tile / tiles_x;
  int ix = (in & 1) | ((in >> 1) & 2) | ((in >> 2) & 4);
  int iy = ((in >> 1) & 1) | ((in >> 2) & 2) | ((in >> 3) & 4);
  px = (tx << 3) + ix;
  py = (ty << 3) + iy;
  return px < W && py < H;
}
FR_DEV int tiled_pixel_count(int W, int H) { return ((W + 7) >> 3) * ((H + 7) >> 3) * 64; }

}  // namespace fr
