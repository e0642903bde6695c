// C-ABI of batched frames (declared in include/facert.h): per-frame buffers,
// the work queue of the persistent kernel, the CUDA graph of one step and
// the autotuner of the kernel's launch configuration.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "context.cuh"

using namespace fr;

namespace fr {
__global__ void k_set_u32(uint32_t* p, uint32_t v) { *p = v; }
}  // namespace fr

struct fr_batch {
  fr_ctx* ctx = nullptr;
  int nF = 0, spp = 0, P = 0, Ps = 0, Pf = 0;
  std::vector<fr_frame> frames;
  std::vector<long long> pix_off;      // first packed pixel of each frame
  long long n_pix = 0;
  int nt_nodes = 0, ne_nodes = 0, nb_sil = 0;
  // per-frame buffers, frame f at offset f * (per-frame size)
  DBuf<float4> X, Xm, nrm, ng, tv, epack, tnodes, tcones, enodes, econes, e4cones, dX, dN, gs;
  DBuf<float2> e4boxes;
  DBuf<int> tcounter, ecounter, sil, n_sil, block_count;
  DBuf<float> dXm, dL;
  // shared by the frames: albedo and its adjoint, specular-map adjoint
  DBuf<float4> alb, dA;
  DBuf<float> dC;
  // inputs and outputs of a step
  DBuf<float> theta_s, theta_f, theta, targets, images, d_images, m;
  DBuf<uint8_t> masks;
  bool have_targets = false, have_masks = false;
  DBuf<double> grad_full, loss_frames, loss, grad_s, grad_f;
  // persistent kernel
  DBuf<BatchFrame> dframes;
  DBuf<int2> items, hits, picks;
  DBuf<int> queue, tiles_done, bs_fwd, bs_sedge, bs_pedge;
  int nb_fwd = 0, nb_sedge = 0, nb_pedge = 0;
  std::vector<long long> hit_off;      // first hit slot of each frame
  DBuf<uint32_t> iter_dev;
  int n_items = 0;
  fr_tile_config cfg{8, 8, 256, 4, 0, 0.0f};
  bool configured = false;
  // graph of one step
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false, g_counters = false;
  float g_w1 = 0.0f, g_w2 = 0.0f;
  int g_max_steps = 0, g_wait_limit = 0;     // device limits the graph was captured with
  uint64_t kernels_per_step = 0;
  int n_sms = 0;
  int occ = 0;             // blocks per SM of the configured kernel
  uint64_t generation = 0; // the context's mesh and bases this batch was sized for
};

namespace {

FrameView frame_view(fr_batch* b, int f) {
  const fr_ctx* c = b->ctx;
  const size_t V = c->V, F = c->F, E = c->E;
  FrameView v;
  v.X = b->X.p + f * V; v.Xm = b->Xm.p + f * V; v.nrm = b->nrm.p + f * V; v.ng = b->ng.p + f * F;
  v.tv = b->tv.p + f * 3 * F; v.epack = b->epack.p + f * 6 * E;
  v.alb = b->alb.p;
  v.tnodes = b->tnodes.p + (size_t)f * 4 * b->nt_nodes; v.tcones = b->tcones.p + (size_t)f * 2 * b->nt_nodes;
  v.enodes = b->enodes.p + (size_t)f * 4 * b->ne_nodes; v.econes = b->econes.p + (size_t)f * 2 * b->ne_nodes;
  v.e4boxes = b->e4boxes.p + (size_t)f * 12 * c->n4; v.e4cones = b->e4cones.p + (size_t)f * 8 * c->n4;
  v.tcounter = b->tcounter.p + (size_t)f * b->nt_nodes; v.ecounter = b->ecounter.p + (size_t)f * b->ne_nodes;
  v.sil = b->sil.p + f * E; v.n_sil = b->n_sil.p + f; v.block_count = b->block_count.p + (size_t)f * b->nb_sil;
  v.dX = b->dX.p + f * V; v.dN = b->dN.p + f * V; v.dA = b->dA.p; v.gs = b->gs.p + f * V;
  v.dXm = b->dXm.p + f * 3 * V; v.dC = b->dC.p; v.dL = b->dL.p + (size_t)f * 3 * MAX_LIGHTS;
  return v;
}

size_t smem_of(const fr_batch*, const fr_tile_config& c) { return batch_smem_bytes(c.block); }

void (*kernel_of(int min_blocks))(BatchArgs) {
  switch (min_blocks) {
    case 2: return k_batch_step2;
    case 3: return k_batch_step3;
    case 4: return k_batch_step4;
    default: return nullptr;
  }
}

// Does the configuration fit the device?  Sets the kernel's dynamic shared
// memory limit as a side effect.  *blocks_per_sm receives the occupancy.
int check_config(fr_batch* b, const fr_tile_config& c, int* blocks_per_sm) {
  fr_ctx* ctx = b->ctx;
  if (c.fused != 0 && c.fused != 1) return fail(ctx, FR_ERR_INVALID_ARG, "fused must be 0 or 1");
  if (!c.fused) {
    if (256 % b->spp) return fail(ctx, FR_ERR_INVALID_ARG, "the phased launches need spp dividing 256");
    if (c.min_blocks != 3 && c.min_blocks != 4)
      return fail(ctx, FR_ERR_INVALID_ARG, "phased: min_blocks must be 3 or 4, got %d", c.min_blocks);
    *blocks_per_sm = c.min_blocks;
    return FR_OK;
  }
  if (c.tile_w < 1 || c.tile_h < 1 || c.tile_w > 64 || c.tile_h > 64)
    return fail(ctx, FR_ERR_INVALID_ARG, "tile %dx%d: sides must be in [1, 64]", c.tile_w, c.tile_h);
  if (c.block < 32 || c.block > 256 || c.block % 32)
    return fail(ctx, FR_ERR_INVALID_ARG, "block must be a multiple of 32 in [32, 256], got %d", c.block);
  auto kern = kernel_of(c.min_blocks);
  if (!kern) return fail(ctx, FR_ERR_INVALID_ARG, "min_blocks must be 2, 3 or 4, got %d", c.min_blocks);
  int dev_max = 0;
  CK(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  size_t sm = smem_of(b, c);
  if (sm > (size_t)dev_max) return fail(ctx, FR_ERR_INVALID_ARG, "tile needs %zu bytes of shared memory", sm);
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int occ = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, c.block, sm));
  if (occ < 1) return fail(ctx, FR_ERR_INVALID_ARG, "configuration does not fit an SM");
  *blocks_per_sm = occ;
  return FR_OK;
}

// The persistent kernel's work items (encoding in kernels.cuh): all tile
// items, then the shadow-edge items light-major within each frame, then the
// primary-edge items.  Frames with more pixels come first in each group:
// their items start early and the tail of the queue holds small items.
// Returns FR_OK, FR_ERR_INVALID_ARG when the list does not fit its encoding
// or FR_ERR_OOM when host memory for it runs out, with *why set.
int plan_items(const fr_frame* frames, int nF, int spp, int tw, int th, int n_lights, std::vector<int2>& items,
               const char** why) {
  items.clear();
  std::vector<int> order(nF);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (long long)frames[x].W * frames[x].H > (long long)frames[y].W * frames[y].H;
  });
  auto n_tiles = [&](int f) {
    return (long long)((frames[f].W + tw - 1) / tw) * ((frames[f].H + th - 1) / th);
  };
  long long total = 0;
  for (int f = 0; f < nF; ++f) {
    const long long nc = (n_tiles(f) * tw * th * spp + BATCH_SEDGE_CHUNK - 1) / BATCH_SEDGE_CHUNK;
    const long long np = ((long long)frames[f].W * frames[f].H * spp + BATCH_PEDGE_CHUNK - 1) / BATCH_PEDGE_CHUNK;
    if (n_tiles(f) > INT32_MAX || nc >= (1LL << (30 - SEDGE_LIGHT_BITS)) || np > INT32_MAX) {
      *why = "frame too large for one launch";
      return FR_ERR_INVALID_ARG;
    }
    total += n_tiles(f) + nc * n_lights + np;
  }
  if (total > INT32_MAX / 2) {
    *why = "too many work items";
    return FR_ERR_INVALID_ARG;
  }
  try {
    items.reserve((size_t)total);
  } catch (const std::bad_alloc&) {
    *why = "out of host memory for the work items";
    return FR_ERR_OOM;
  }
  for (int f : order)
    for (long long t = 0; t < n_tiles(f); ++t) items.push_back(make_int2(f, (int)t));
  for (int f : order) {
    const long long nc = (n_tiles(f) * tw * th * spp + BATCH_SEDGE_CHUNK - 1) / BATCH_SEDGE_CHUNK;
    for (int j = 0; j < n_lights; ++j)
      for (long long k = 0; k < nc; ++k) items.push_back(make_int2(f | SEDGE_ITEM, (int)(k << SEDGE_LIGHT_BITS) | j));
  }
  for (int f : order) {
    const long long np = ((long long)frames[f].W * frames[f].H * spp + BATCH_PEDGE_CHUNK - 1) / BATCH_PEDGE_CHUNK;
    for (long long k = 0; k < np; ++k) items.push_back(make_int2(f | PEDGE_ITEM, (int)k));
  }
  return FR_OK;
}

// Frame table and work items for the current configuration (host -> device,
// synchronous: never inside a capture).
int configure(fr_batch* b) {
  fr_ctx* ctx = b->ctx;
  const fr_tile_config& c = b->cfg;
  std::vector<BatchFrame> tab(b->nF);
  std::vector<int2> items;       // the persistent kernel's; the phased launches take none
  // primary hits, per frame in the sample order of the launch mode: 8x8
  // tiles (phased) or the tile items' order (persistent); each frame's slots
  // start on a 128-byte line
  long long nh = 0;
  for (int f = 0; f < b->nF; ++f) {
    const fr_frame& q = b->frames[f];
    b->hit_off[f] = nh;
    const long long n = c.fused ? (long long)((q.W + c.tile_w - 1) / c.tile_w) * ((q.H + c.tile_h - 1) / c.tile_h) *
                                      c.tile_w * c.tile_h * b->spp
                                : (long long)((q.W + 7) / 8) * ((q.H + 7) / 8) * 64 * b->spp;
    nh += (n + 15) & ~15LL;
  }
  if (c.fused || 256 % b->spp == 0)
    if (b->hits.n < (size_t)nh) CK(b->hits.alloc((size_t)nh));
  for (int f = 0; f < b->nF; ++f) {
    const fr_frame& fr_ = b->frames[f];
    fr_render_opts o{fr_.W, fr_.H, b->spp, fr_.seed, 0u, 0};
    FrameView v = frame_view(b, f);
    BatchFrame& T = tab[f];
    T.a = render_args(ctx, b->theta.p + (size_t)f * b->P, &o, v);
    T.a.counters = nullptr;
    T.gb.dX = v.dX; T.gb.dN = v.dN; T.gb.dA = v.dA; T.gb.dC = v.dC; T.gb.dL = v.dL;
    T.gb.d_image = b->d_images.p + 3 * b->pix_off[f];
    T.gb.hits = b->hits.p + b->hit_off[f];
    T.image = b->images.p + 3 * b->pix_off[f];
    T.d_image = b->d_images.p + 3 * b->pix_off[f];
    T.target = b->targets.p + 3 * b->pix_off[f];
    T.mask = b->have_masks ? b->masks.p + b->pix_off[f] : nullptr;
    T.loss = b->loss_frames.p + f;
    T.tiles_x = (fr_.W + c.tile_w - 1) / c.tile_w;
    T.n_tiles = T.tiles_x * ((fr_.H + c.tile_h - 1) / c.tile_h);
    T.n_pedge = (long long)fr_.W * fr_.H * b->spp;
  }
  if (c.fused) {
    const char* why = "";
    const int rc = plan_items(b->frames.data(), b->nF, b->spp, c.tile_w, c.tile_h, ctx->cfg.n_lights, items, &why);
    if (rc) return fail(ctx, rc, "%s", why);
  }
  // block tables of the phased launches (256 threads per block)
  std::vector<int> sf(b->nF + 1), ss(b->nF + 1), sp(b->nF + 1);
  long long nf = 0, ns = 0, np = 0;
  for (int f = 0; f < b->nF; ++f) {
    const fr_frame& q = b->frames[f];
    long long tiled = (long long)((q.W + 7) / 8) * ((q.H + 7) / 8) * 64 * b->spp;
    sf[f] = (int)nf; ss[f] = (int)ns; sp[f] = (int)np;
    nf += (tiled + 255) / 256;
    ns += (tiled + 255) / 256 * ctx->cfg.n_lights;
    np += ((long long)q.W * q.H * b->spp + 255) / 256;
    if (ns > INT32_MAX) return fail(ctx, FR_ERR_INVALID_ARG, "batch too large for one launch");
  }
  sf[b->nF] = (int)nf; ss[b->nF] = (int)ns; sp[b->nF] = (int)np;
  b->nb_fwd = (int)nf; b->nb_sedge = (int)ns; b->nb_pedge = (int)np;
  // one shadow-edge pick per thread of the phased shadow-edge launches
  const size_t n_picks = 256 % b->spp == 0 ? (size_t)ns * 256 : 0;
  if (b->picks.n != n_picks) CK(b->picks.alloc(n_picks));
  b->n_items = (int)items.size();
  CK(cudaStreamSynchronize(ctx->stream));
  CK(b->dframes.alloc(tab.size()));
  CK(b->items.alloc(items.size()));
  CK(cudaMemcpy(b->dframes.p, tab.data(), sizeof(BatchFrame) * tab.size(), cudaMemcpyHostToDevice));
  if (!items.empty()) CK(cudaMemcpy(b->items.p, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice));
  CK(b->bs_fwd.alloc(b->nF + 1));
  CK(b->bs_sedge.alloc(b->nF + 1));
  CK(b->bs_pedge.alloc(b->nF + 1));
  CK(cudaMemcpy(b->bs_fwd.p, sf.data(), sizeof(int) * sf.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->bs_sedge.p, ss.data(), sizeof(int) * ss.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->bs_pedge.p, sp.data(), sizeof(int) * sp.size(), cudaMemcpyHostToDevice));
  b->configured = true;
  return FR_OK;
}

// The work of one step, enqueued on ctx->stream (captured into the graph).
int enqueue_step(fr_batch* b, float w1, float w2) {
  fr_ctx* ctx = b->ctx;
  cudaStream_t s = ctx->stream;
  const int nF = b->nF, P = b->P;
  const size_t V = ctx->V;
  const int nlv = 3 * ctx->cfg.n_lights;
  long long nth = (long long)nF * P;
  k_batch_gather_theta<<<grid_for(nth, 256), 256, 0, s>>>(nF, P, ctx->K_id, ctx->K_exp, ctx->K_alb, nlv,
                                                          b->theta_s.p, b->theta_f.p, b->theta.p);
  CKL();
  CK(cudaMemsetAsync(b->grad_full.p, 0, sizeof(double) * nth, s));
  CK(cudaMemsetAsync(b->loss_frames.p, 0, sizeof(double) * nF, s));
  CK(cudaMemsetAsync(b->queue.p, 0, sizeof(int), s));
  CK(cudaMemsetAsync(b->tiles_done.p, 0, sizeof(int) * nF, s));
  CK(cudaMemsetAsync(b->dA.p, 0, sizeof(float4) * V, s));
  CK(cudaMemsetAsync(b->dC.p, 0, sizeof(float) * CS * CS, s));
  CK(cudaMemsetAsync(b->dX.p, 0, sizeof(float4) * V * nF, s));
  CK(cudaMemsetAsync(b->dN.p, 0, sizeof(float4) * V * nF, s));
  CK(cudaMemsetAsync(b->dL.p, 0, sizeof(float) * 3 * MAX_LIGHTS * nF, s));
  for (int f = 0; f < nF; ++f) {
    FrameView v = frame_view(b, f);
    if (f > 0) v.alb = nullptr;        // albedo (delta shared) is computed once
    int rc = prepare_geometry(ctx, b->theta.p + (size_t)f * P, v);
    if (rc) return rc;
    rc = silhouettes(ctx, v);
    if (rc) return rc;
  }
  unsigned long long* counters = ctx->counters_on ? ctx->counters.p : nullptr;
  if (counters) CK(cudaMemsetAsync(counters, 0, NCOUNT * sizeof(unsigned long long), s));
  if (b->cfg.fused) {
    BatchArgs a;
    a.frames = b->dframes.p; a.items = b->items.p; a.n_items = b->n_items;
    a.tile_w = b->cfg.tile_w; a.tile_h = b->cfg.tile_h; a.pedge_chunk = BATCH_PEDGE_CHUNK;
    a.sedge_chunk = BATCH_SEDGE_CHUNK;
    a.queue = b->queue.p; a.tiles_done = b->tiles_done.p; a.iter = b->iter_dev.p; a.err = ctx->err_flag.p;
    a.counters = counters;
    a.max_steps = ctx->max_steps; a.wait_limit = ctx->wait_limit;
    int grid = (int)std::min<long long>((long long)b->occ * b->n_sms, b->n_items);
    kernel_of(b->cfg.min_blocks)<<<grid, b->cfg.block, smem_of(b, b->cfg), s>>>(a);
    CKL();
  } else {
    PhaseArgs pa;
    pa.frames = b->dframes.p; pa.n_frames = nF; pa.iter = b->iter_dev.p; pa.err = ctx->err_flag.p;
    pa.counters = counters;
    pa.max_steps = ctx->max_steps;
    pa.picks = nullptr;
    pa.block_start = b->bs_fwd.p;
    k_batch_fwd<<<b->nb_fwd, 256, 0, s>>>(pa);
    CKL();
    pa.block_start = b->bs_sedge.p;
    pa.picks = b->picks.p;
    if (b->cfg.min_blocks == 3) k_batch_sedge3<<<b->nb_sedge, 256, 0, s>>>(pa);
    else k_batch_sedge4<<<b->nb_sedge, 256, 0, s>>>(pa);
    CKL();
    k_batch_sedge_add<<<b->nb_sedge, 256, 0, s>>>(pa);
    CKL();
    pa.block_start = b->bs_pedge.p;
    k_batch_pedge<<<b->nb_pedge, 256, 0, s>>>(pa);
    CKL();
  }
  for (int f = 0; f < nF; ++f) {
    FrameView v = frame_view(b, f);
    if (f > 0) v.dC = nullptr;          // specular map (shared) is added once
    int rc = adjoint(ctx, b->theta.p + (size_t)f * P, v, b->grad_full.p + (size_t)f * P, f == 0);
    if (rc) return rc;
  }
  long long nout = b->Ps + (long long)nF * b->Pf;
  k_batch_reduce<<<grid_for(nout, 256), 256, 0, s>>>(nF, P, ctx->K_id, ctx->K_exp, ctx->K_alb, nlv, b->theta.p,
                                                    b->grad_full.p, b->loss_frames.p,
                                                    ctx->cfg.light_prior, b->m.p,
                                                    w1, w2, b->grad_s.p, b->grad_f.p, b->loss.p);
  CKL();
  return FR_OK;
}

int capture(fr_batch* b, float w1, float w2) {
  fr_ctx* ctx = b->ctx;
  if (b->exec) {
    CK(cudaStreamSynchronize(ctx->stream));   // the old graph may still run
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->graph_ok = false;
  if (!b->configured) {
    int rc = configure(b);
    if (rc) return rc;
  }
  int rc = check_config(b, b->cfg, &b->occ);   // attributes and occupancy outside the capture
  if (rc) return rc;
  cudaStream_t saved = ctx->stream;
  uint64_t launches0 = ctx->launches;
  CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  ctx->stream = b->cap_stream;
  rc = enqueue_step(b, w1, w2);
  ctx->stream = saved;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
  b->kernels_per_step = ctx->launches - launches0;
  ctx->launches = launches0;
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return fail(ctx, FR_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(ctx, FR_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
  b->graph_ok = true;
  b->g_w1 = w1; b->g_w2 = w2; b->g_counters = ctx->counters_on;
  b->g_max_steps = ctx->max_steps; b->g_wait_limit = ctx->wait_limit;
  return FR_OK;
}

// Copy the parameters in, set iter, launch the graph (capturing it first
// when needed).
int launch_step(fr_batch* b, const float* ts, const float* tf, float w1, float w2, uint32_t iter) {
  fr_ctx* ctx = b->ctx;
  if (b->generation != ctx->generation)
    return fail(ctx, FR_ERR_NOT_READY, "the mesh or bases changed after this batch was created: create a new batch");
  if (!b->have_targets) return fail(ctx, FR_ERR_NOT_READY, "fr_batch_set_targets first");
  if (!ts || !tf) return fail(ctx, FR_ERR_INVALID_ARG, "theta_shared or theta_frames is null");
  if (!b->graph_ok || w1 != b->g_w1 || w2 != b->g_w2 || ctx->counters_on != b->g_counters ||
      ctx->max_steps != b->g_max_steps || ctx->wait_limit != b->g_wait_limit) {
    int rc = capture(b, w1, w2);
    if (rc) return rc;
  }
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(b->theta_s.p, ts, sizeof(float) * b->Ps, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(b->theta_f.p, tf, sizeof(float) * (size_t)b->nF * b->Pf, cudaMemcpyDeviceToDevice, s));
  k_set_u32<<<1, 1, 0, s>>>(b->iter_dev.p, iter);
  CKL();
  CK(cudaGraphLaunch(b->exec, s));
  ctx->launches += b->kernels_per_step;
  return FR_OK;
}

}  // namespace

extern "C" {

int32_t fr_batch_n_shared(const fr_ctx* ctx) { return ctx ? ctx->K_id + ctx->K_alb + CS * CS : FR_ERR_INVALID_ARG; }
int32_t fr_batch_n_frame(const fr_ctx* ctx) { return ctx ? ctx->K_exp + 6 + 3 * ctx->cfg.n_lights : FR_ERR_INVALID_ARG; }

int fr_batch_plan(const fr_frame* frames, int32_t n_frames, int32_t spp, int32_t tile_w, int32_t tile_h,
                  int32_t n_lights, int32_t* items, int64_t cap, int64_t* n_out) {
  if (!frames || n_frames < 1 || n_frames > 4096 || !n_out || cap < 0 || (cap > 0 && !items))
    return FR_ERR_INVALID_ARG;
  if (spp < 1 || (spp < 32 && 32 % spp) || (spp > 32 && spp % 32)) return FR_ERR_INVALID_ARG;
  if (tile_w < 1 || tile_h < 1 || tile_w > 64 || tile_h > 64 || n_lights < 1 || n_lights > MAX_LIGHTS)
    return FR_ERR_INVALID_ARG;
  for (int f = 0; f < n_frames; ++f) {
    const fr_frame& q = frames[f];
    if (q.W < 1 || q.H < 1 || (long long)q.W * q.H > (1LL << 26) || (long long)q.W * q.H * spp > (1LL << 31) - 1)
      return FR_ERR_INVALID_ARG;
  }
  std::vector<int2> v;
  const char* why = "";
  const int rc = plan_items(frames, n_frames, spp, tile_w, tile_h, n_lights, v, &why);
  if (rc) return rc;
  *n_out = (int64_t)v.size();
  const size_t n = std::min<size_t>(v.size(), (size_t)cap);
  for (size_t i = 0; i < n; ++i) { items[2 * i] = v[i].x; items[2 * i + 1] = v[i].y; }
  return FR_OK;
}

int fr_batch_create(fr_ctx* ctx, const fr_frame* frames, int32_t n_frames, int32_t spp, fr_batch** out) {
  if (!ctx || !out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctx->have_mesh || !ctx->have_bases) return fail(ctx, FR_ERR_NOT_READY, "mesh and bases must be uploaded first");
  if (!frames || n_frames < 1 || n_frames > 4096) return fail(ctx, FR_ERR_INVALID_ARG, "frames or n_frames");
  if (spp < 1 || (spp < 32 && 32 % spp) || (spp > 32 && spp % 32))
    return fail(ctx, FR_ERR_INVALID_ARG, "batched spp must divide 32 or be a multiple of 32, got %d", spp);
  long long n_pix = 0;
  for (int f = 0; f < n_frames; ++f) {
    const fr_frame& q = frames[f];
    if (q.W < 1 || q.H < 1 || (long long)q.W * q.H > (1LL << 26) || (long long)q.W * q.H * spp > (1LL << 31) - 1)
      return fail(ctx, FR_ERR_INVALID_ARG, "frame %d: size %dx%d at %d spp out of range", f, q.W, q.H, spp);
    n_pix += (long long)q.W * q.H;
  }
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  fr_batch* b = new fr_batch();
  b->ctx = ctx;
  b->generation = ctx->generation;
  b->nF = n_frames; b->spp = spp;
  if (256 % spp) b->cfg = fr_tile_config{4, 4, 256, 2, 1, 0.0f};   // the phased launches need spp dividing 256
  b->P = ctx->n_params(); b->Ps = fr_batch_n_shared(ctx); b->Pf = fr_batch_n_frame(ctx);
  b->frames.assign(frames, frames + n_frames);
  b->pix_off.resize(n_frames);
  long long off = 0;
  for (int f = 0; f < n_frames; ++f) { b->pix_off[f] = off; off += (long long)frames[f].W * frames[f].H; }
  b->n_pix = n_pix;
  b->nt_nodes = ctx->tbvh.n_nodes; b->ne_nodes = ctx->ebvh.n_nodes; b->nb_sil = (ctx->E + 255) / 256;
  const size_t nF = n_frames, V = ctx->V, F = ctx->F, E = ctx->E;
  auto cleanup = [&](int code) { fr_batch_destroy(b); return code; };
#define BK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return cleanup(fail(ctx, e_ == cudaErrorMemoryAllocation ? FR_ERR_OOM : FR_ERR_CUDA, "%s: %s", #call, \
                          cudaGetErrorString(e_)));                                \
  } while (0)
  BK(b->X.alloc(nF * V)); BK(b->Xm.alloc(nF * V)); BK(b->nrm.alloc(nF * V)); BK(b->ng.alloc(nF * F));
  BK(b->tv.alloc(nF * 3 * F)); BK(b->epack.alloc(nF * 6 * E));
  BK(b->tnodes.alloc(nF * 4 * b->nt_nodes)); BK(b->tcones.alloc(nF * 2 * b->nt_nodes));
  BK(b->enodes.alloc(nF * 4 * b->ne_nodes)); BK(b->econes.alloc(nF * 2 * b->ne_nodes));
  BK(b->e4boxes.alloc(nF * 12 * (size_t)ctx->n4)); BK(b->e4cones.alloc(nF * 8 * (size_t)ctx->n4));
  BK(b->tcounter.alloc(nF * b->nt_nodes)); BK(b->ecounter.alloc(nF * b->ne_nodes));
  BK(b->sil.alloc(nF * E)); BK(b->n_sil.alloc(nF)); BK(b->block_count.alloc(nF * b->nb_sil));
  BK(b->dX.alloc(nF * V)); BK(b->dN.alloc(nF * V)); BK(b->gs.alloc(nF * V));
  BK(b->dXm.alloc(nF * 3 * V)); BK(b->dL.alloc(nF * 3 * MAX_LIGHTS));
  BK(b->alb.alloc(V)); BK(b->dA.alloc(V)); BK(b->dC.alloc(CS * CS));
  BK(b->theta_s.alloc(b->Ps)); BK(b->theta_f.alloc(nF * b->Pf)); BK(b->theta.alloc(nF * b->P));
  BK(b->targets.alloc(3 * (size_t)n_pix)); BK(b->images.alloc(3 * (size_t)n_pix));
  BK(b->d_images.alloc(3 * (size_t)n_pix)); BK(b->m.alloc(3 * MAX_LIGHTS));
  BK(b->masks.alloc((size_t)n_pix));
  BK(b->grad_full.alloc(nF * b->P)); BK(b->loss_frames.alloc(nF)); BK(b->loss.alloc(1));
  BK(b->grad_s.alloc(b->Ps)); BK(b->grad_f.alloc(nF * b->Pf));
  BK(b->queue.alloc(1)); BK(b->tiles_done.alloc(nF)); BK(b->iter_dev.alloc(1));
  // primary hits: sized for the launch mode when a configuration is set up
  b->hit_off.resize(n_frames);
  // BVH boxes start as the context's (child codes and empty children are
  // fixed by the topology; refits rewrite the rest)
  for (size_t f = 0; f < nF; ++f) {
    BK(cudaMemcpy(b->tnodes.p + f * 4 * b->nt_nodes, ctx->tbvh.nodes.p, sizeof(float4) * 4 * b->nt_nodes,
                  cudaMemcpyDeviceToDevice));
    BK(cudaMemcpy(b->tcones.p + f * 2 * b->nt_nodes, ctx->tbvh.cones.p, sizeof(float4) * 2 * b->nt_nodes,
                  cudaMemcpyDeviceToDevice));
    BK(cudaMemcpy(b->enodes.p + f * 4 * b->ne_nodes, ctx->ebvh.nodes.p, sizeof(float4) * 4 * b->ne_nodes,
                  cudaMemcpyDeviceToDevice));
    BK(cudaMemcpy(b->econes.p + f * 2 * b->ne_nodes, ctx->ebvh.cones.p, sizeof(float4) * 2 * b->ne_nodes,
                  cudaMemcpyDeviceToDevice));
  }
  BK(cudaMemset(b->m.p, 0, sizeof(float) * 3 * MAX_LIGHTS));
  BK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  BK(cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, ctx->device));
  BK(cudaDeviceSynchronize());
#undef BK
  *out = b;
  return FR_OK;
}

void fr_batch_destroy(fr_batch* b) {
  if (!b) return;
  cudaSetDevice(b->ctx->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (DBuf<float4>* p : {&b->X, &b->Xm, &b->nrm, &b->ng, &b->tv, &b->epack, &b->tnodes, &b->tcones, &b->enodes,
                          &b->econes, &b->e4cones, &b->dX, &b->dN, &b->gs, &b->alb, &b->dA})
    p->free_();
  for (DBuf<int>* p : {&b->tcounter, &b->ecounter, &b->sil, &b->n_sil, &b->block_count, &b->queue, &b->tiles_done})
    p->free_();
  for (DBuf<float>* p : {&b->dXm, &b->dL, &b->dC, &b->theta_s, &b->theta_f, &b->theta, &b->targets, &b->images,
                         &b->d_images, &b->m})
    p->free_();
  for (DBuf<double>* p : {&b->grad_full, &b->loss_frames, &b->loss, &b->grad_s, &b->grad_f}) p->free_();
  b->e4boxes.free_();
  b->masks.free_(); b->dframes.free_(); b->items.free_(); b->hits.free_(); b->picks.free_(); b->iter_dev.free_();
  b->bs_fwd.free_(); b->bs_sedge.free_(); b->bs_pedge.free_();
  delete b;
}

int fr_batch_set_targets(fr_batch* b, const float* targets, const uint8_t* masks, const float* m) {
  if (!b) return FR_ERR_INVALID_ARG;
  fr_ctx* ctx = b->ctx;
  if (!targets) return fail(ctx, FR_ERR_INVALID_ARG, "targets is null");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  CK(cudaMemcpyAsync(b->targets.p, targets, sizeof(float) * 3 * b->n_pix, cudaMemcpyDeviceToDevice, s));
  if (masks) CK(cudaMemcpyAsync(b->masks.p, masks, (size_t)b->n_pix, cudaMemcpyDeviceToDevice, s));
  // the captured graph always reads the batch's own m: zero stands for "no m"
  if (m) CK(cudaMemcpyAsync(b->m.p, m, sizeof(float) * 3 * ctx->cfg.n_lights, cudaMemcpyDeviceToDevice, s));
  else CK(cudaMemsetAsync(b->m.p, 0, sizeof(float) * 3 * MAX_LIGHTS, s));
  bool masks_now = masks != nullptr;
  if (masks_now != b->have_masks || !b->have_targets) {
    b->have_masks = masks_now;
    b->configured = false;            // the frame table records the mask pointers
    b->graph_ok = false;
  }
  b->have_targets = true;
  return FR_OK;
}

int fr_batch_step(fr_batch* b, const float* theta_shared, const float* theta_frames, float w1, float w2,
                  uint32_t iter, double* loss, double* grad_shared, double* grad_frames, float* images) {
  if (!b) return FR_ERR_INVALID_ARG;
  fr_ctx* ctx = b->ctx;
  CK(cudaSetDevice(ctx->device));
  int rc = launch_step(b, theta_shared, theta_frames, w1, w2, iter);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  if (loss) CK(cudaMemcpyAsync(loss, b->loss.p, sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (grad_shared) CK(cudaMemcpyAsync(grad_shared, b->grad_s.p, sizeof(double) * b->Ps, cudaMemcpyDeviceToDevice, s));
  if (grad_frames)
    CK(cudaMemcpyAsync(grad_frames, b->grad_f.p, sizeof(double) * (size_t)b->nF * b->Pf, cudaMemcpyDeviceToDevice, s));
  if (images) CK(cudaMemcpyAsync(images, b->images.p, sizeof(float) * 3 * b->n_pix, cudaMemcpyDeviceToDevice, s));
  return FR_OK;
}

int fr_batch_get_config(const fr_batch* b, fr_tile_config* out) {
  if (!b || !out) return FR_ERR_INVALID_ARG;
  *out = b->cfg;
  return FR_OK;
}

int fr_batch_set_config(fr_batch* b, const fr_tile_config* cfg) {
  if (!b || !cfg) return FR_ERR_INVALID_ARG;
  fr_ctx* ctx = b->ctx;
  CK(cudaSetDevice(ctx->device));
  int occ = 0;
  int rc = check_config(b, *cfg, &occ);
  if (rc) return rc;
  b->cfg = *cfg;
  b->configured = false;
  b->graph_ok = false;
  return FR_OK;
}

int fr_batch_autotune(fr_batch* b, const float* theta_shared, const float* theta_frames, int32_t reps,
                      fr_tile_config* table, int32_t cap, int32_t* n_out) {
  if (!b) return FR_ERR_INVALID_ARG;
  fr_ctx* ctx = b->ctx;
  if (reps < 1 || (cap > 0 && !table)) return fail(ctx, FR_ERR_INVALID_ARG, "reps >= 1 and a table of cap entries");
  CK(cudaSetDevice(ctx->device));
  const fr_tile_config cands[6] = {{8, 8, 256, 3, 0, 0.0f}, {8, 8, 256, 4, 0, 0.0f}, {2, 2, 256, 2, 1, 0.0f},
                                   {2, 2, 256, 4, 1, 0.0f}, {4, 4, 256, 2, 1, 0.0f}, {4, 4, 256, 4, 1, 0.0f}};
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const fr_tile_config saved = b->cfg;
  fr_tile_config best{0, 0, 0, 0, 0, 0.0f};
  int n = 0, rc = FR_OK;
  const float w1 = b->graph_ok ? b->g_w1 : 0.0f, w2 = b->graph_ok ? b->g_w2 : 0.0f;
  for (fr_tile_config c : cands) {
    int occ = 0;
    if (check_config(b, c, &occ) != FR_OK) continue;    // does not fit: skipped
    b->cfg = c;
    b->configured = false;
    b->graph_ok = false;
    rc = launch_step(b, theta_shared, theta_frames, w1, w2, 0u);       // capture + warm-up
    if (rc) goto out;
    if (cudaEventRecord(e0, ctx->stream) != cudaSuccess) { rc = fail(ctx, FR_ERR_CUDA, "event record"); goto out; }
    for (int r = 0; r < reps; ++r) {
      rc = launch_step(b, theta_shared, theta_frames, w1, w2, (uint32_t)(r + 1));
      if (rc) goto out;
    }
    if (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = fail(ctx, FR_ERR_CUDA, "event timing");
      goto out;
    }
    cudaEventElapsedTime(&c.ms, e0, e1);
    c.ms /= (float)reps;
    if (n < cap) table[n] = c;
    ++n;
    if (best.block == 0 || c.ms < best.ms) best = c;
  }
out:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_out) *n_out = n;
  b->cfg = rc == FR_OK && best.block ? best : saved;
  b->configured = false;
  b->graph_ok = false;
  return rc;
}

}  // extern "C"
