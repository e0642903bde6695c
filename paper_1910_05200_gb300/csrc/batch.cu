// Batched render + loss + backward of many frames in one persistent launch.
//
// Frames share identity, albedo and the specular map and differ in
// expression, pose and lights (a video of one face, or several crops); each
// has its own crop size.  The launch is a work queue served by warps: every
// warp takes items on its own (no block-wide barrier while items remain, so
// a warp with cheap samples never waits for one with costly samples).  The
// queue holds three kinds of item, in this order:
//   tile items       a tile of one frame, taken 32 samples at a time: forward
//                    samples, the pixel means (image), the photo-consistency
//                    loss and its adjoint d_image = 2 mask (image - target)
//                    (Eq. 1 of the Optimization paragraph, per pixel), then the
//                    interior adjoint of the same samples with their primary
//                    hits and the shadow decisions of the lights that are on
//                    still in registers (no re-trace when spp divides 32).
//                    Each sample's primary hit goes to the frame's hit array.
//   shadow-edge items  (frame, light, chunk of samples): the shadow-boundary
//                    term of one light for consecutive samples of the frame,
//                    from the stored hits and d_image.  The items of one
//                    light of one frame follow each other in the queue, so
//                    the warps that run at the same time search the edge
//                    hierarchy towards the same light, as the light-major
//                    shadow-edge launches of the single-image path do.
//   primary-edge items  a chunk of one frame's primary-edge samples; they
//                    read d_image anywhere in the frame.
// Each kind of item runs in a function of its own, out of line, and so do
// the shadow-edge search and contribution: each is register-allocated on its
// own within the kernel's budget (inlined into the kernel they spilled more
// and ran slower).
// Edge items wait until all tile items of their frame have published their
// hits and d_image.  All tile items come before all edge items in the queue
// and a warp only takes an item when it is running, so every tile item an
// edge item waits for is held by a running warp that does not wait: the
// wait ends.  It is bounded all the same (BatchArgs::wait_limit,
// fr_set_limits; ERR_WAIT on expiry).
//
// Samples, decisions and per-sample arithmetic are those of the single-image
// kernels (same device functions, same Philox keys, the same warp-cooperative
// traversals), so a frame's image equals the single-image render of the same
// frame up to FP32 rounding (the same formulas compiled in another kernel may
// contract multiply-adds differently) and its gradient differs only in that
// and the order of floating-point atomic additions.  spp a multiple of 32 takes each pixel in
// two passes (radiance, then the interior adjoint with the primary hit traced again).
#include "render_device.cuh"

namespace fr {

namespace {

using WarpState = BatchWarpState;

FR_DEV void flush_lights(WarpState& w, int lane) {
  for (int i = lane; i < 3 * MAX_LIGHTS; i += 32)
    if (w.sL[i] != 0.0f) { atomicAdd(&w.g.dL[i], w.sL[i]); w.sL[i] = 0.0f; }
  __syncwarp();
}

// Loss and adjoint of pixel pix from its mean I: image and d_image written
// when `write`, E_data added to lacc.  Returns d_image.
FR_DEV V3 pixel_loss(const BatchFrame& F, size_t pix, V3 I, bool write, double& lacc) {
  bool in = F.mask ? F.mask[pix] != 0 : true;
  float Iv[3] = {I.x, I.y, I.z}, dv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double diff = (double)Iv[c] - (double)F.target[3 * pix + c];
    if (in && write) lacc += diff * diff;
    dv[c] = in ? (float)(2.0 * diff) : 0.0f;
    if (write) {
      F.image[3 * pix + c] = Iv[c];
      F.d_image[3 * pix + c] = dv[c];
    }
  }
  return V3{dv[0], dv[1], dv[2]};
}

FR_DEV bool nonzero(V3 v) { return v.x != 0.0f || v.y != 0.0f || v.z != 0.0f; }

// A tile item, spp dividing 32: chunks of 32 consecutive samples hold whole
// pixels, so each pixel's mean is a shuffle reduction within the warp.
__device__ __noinline__ void tile_small(WarpState& w, const BatchFrame& F, float* sC, int tile, int tw, int th,
                                        double& lacc, unsigned long long* cnt) {
  const RenderArgs& a = w.a;
  const int spp = a.spp, lane = threadIdx.x & 31;
  const int tx = tile % F.tiles_x, ty = tile / F.tiles_x;
  const int nS = tw * th * spp;
  int2* hits = F.gb.hits + (long long)tile * nS;
  const float inv = 1.0f / (float)spp;
  for (int c0 = 0; c0 < nS; c0 += 32) {
    int k = c0 + lane;
    int ip = k / spp, s = k - ip * spp;
    int px = tx * tw + ip % tw, py = ty * th + ip / tw;
    bool valid = k < nS && px < a.W && py < a.H;
    int2 hit = make_int2(-1, 0);
    uint32_t pix = 0, vis = 0u;
    const V3 d = valid ? sample_dir(a, px, py, s, pix) : V3{0, 0, -1};
    const V3 L = radiance(a, a.cam.o, d, TAG_LIGHT, pix, (uint32_t)s, cnt, nullptr, &hit, &vis, valid);
    if (!valid) { hit = make_int2(-1, 0); vis = 0u; }
    float v0 = L.x, v1 = L.y, v2 = L.z;
    for (int off = spp >> 1; off > 0; off >>= 1) {
      v0 += __shfl_xor_sync(0xffffffffu, v0, off);
      v1 += __shfl_xor_sync(0xffffffffu, v1, off);
      v2 += __shfl_xor_sync(0xffffffffu, v2, off);
    }
    V3 dv{0, 0, 0};
    if (valid) dv = pixel_loss(F, pix, V3{v0 * inv, v1 * inv, v2 * inv}, s == 0, lacc);
    const bool adj = valid && hit.x >= 0 && nonzero(dv);
    if (k < nS) hits[k] = adj ? hit : make_int2(-1, 0);
    // warp-collective: every lane takes part
    interior_sample(a, w.g, sC, w.sL, pix, s, d, hit.x, __int_as_float(hit.y), dv,
                    cnt ? cnt + CNT_INTERIOR : nullptr, &vis, adj);
  }
}

// A tile item, spp a multiple of 32: one pixel at a time, its samples in
// chunks of 32; pass 1 sums the radiance, pass 2 runs the interior adjoint.
__device__ __noinline__ void tile_large(WarpState& w, const BatchFrame& F, float* sC, int tile, int tw, int th,
                                        double& lacc, unsigned long long* cnt) {
  const RenderArgs& a = w.a;
  const int spp = a.spp, lane = threadIdx.x & 31;
  const int tx = tile % F.tiles_x, ty = tile / F.tiles_x;
  int2* hits = F.gb.hits + (long long)tile * tw * th * spp;
  for (int ip = 0; ip < tw * th; ++ip) {
    int px = tx * tw + ip % tw, py = ty * th + ip / tw;
    int2* hp = hits + (long long)ip * spp;
    if (!(px < a.W && py < a.H)) {                               // uniform
      for (int s = lane; s < spp; s += 32) hp[s] = make_int2(-1, 0);
      continue;
    }
    V3 acc{0, 0, 0};
    uint32_t pix = 0;
    for (int s = lane; s < spp; s += 32) {
      V3 d = sample_dir(a, px, py, s, pix);
      acc += radiance(a, a.cam.o, d, TAG_LIGHT, pix, (uint32_t)s, cnt);
    }
    for (int off = 16; off > 0; off >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, off);
    }
    const float inv = 1.0f / (float)spp;
    V3 dv = pixel_loss(F, (size_t)py * a.W + px, acc * inv, lane == 0, lacc);
    if (!nonzero(dv)) {                                          // uniform
      for (int s = lane; s < spp; s += 32) hp[s] = make_int2(-1, 0);
      continue;
    }
    for (int s = lane; s < spp; s += 32) {
      V3 d = sample_dir(a, px, py, s, pix);
      float t = 0.0f;
      int f = closest_hit_warp(a.mesh, true, a.cam.o, d, t, a.err, cnt ? cnt + CNT_INTERIOR : nullptr);
      hp[s] = f >= 0 ? make_int2(f, __float_as_int(t)) : make_int2(-1, 0);
      interior_sample(a, w.g, sC, w.sL, pix, s, d, f, t, dv, cnt ? cnt + CNT_INTERIOR : nullptr, nullptr, f >= 0);
    }
  }
}

// The search and the contribution of a shadow-edge item, out of line: each
// is register-allocated on its own, within the kernel's budget.
__device__ __noinline__ Pick sedge_pick(const RenderArgs& a, bool valid, V3 x32, int f, int j, uint32_t pix, int s,
                                        unsigned long long* cnt) {
  return pick_light_warp(a, valid, x32, f, j, pix, s, cnt);
}
__device__ __noinline__ void sedge_add(const RenderArgs& a, const GradBufs& gb, int j, Pick P, V3 d, V3 x32, int f,
                                       int flip, uint32_t pix, int s, V3 wrgb, unsigned long long* cnt, bool active) {
  sedge_contribution(a, gb, j, P.n, P.slot, d, x32, f, flip, pix, s, wrgb, cnt, active);
}

// A shadow-edge item: light j for the samples [k0, k0 + len) of the frame,
// in the tile items' sample order, 32 at a time (the same warps of samples
// as the tile items).
__device__ __noinline__ void sedge_item(const WarpState& w, const BatchFrame& F, int j, long long k0, int len, int tw,
                                        int th, unsigned long long* cnt) {
  const RenderArgs& a = w.a;
  const int spp = a.spp, lane = threadIdx.x & 31;
  const int per_tile = tw * th * spp;
  const long long n = (long long)F.n_tiles * per_tile;
  const float inv = 1.0f / (float)spp;
  for (int c = 0; c < len && k0 + c < n; c += 32) {              // uniform
    const long long k = k0 + c + lane;
    const int2 hit = k < n ? F.gb.hits[k] : make_int2(-1, 0);
    const bool valid = hit.x >= 0;
    V3 d{0, 0, -1}, x32{0, 0, 0}, wrgb{0, 0, 0};
    uint32_t pix = 0;
    int flip = 1, s = 0;
    if (valid) {
      const int tile = (int)(k / per_tile), r = (int)(k - (long long)tile * per_tile), ip = r / spp;
      s = r - ip * spp;
      const int px = (tile % F.tiles_x) * tw + ip % tw, py = (tile / F.tiles_x) * th + ip / tw;
      d = sample_dir(a, px, py, s, pix);
      flip = face_flip(a.mesh, hit.x, d);
      x32 = hit_point(a.cam.o, d, __int_as_float(hit.y));
      const float* dI = F.d_image + 3 * (size_t)pix;
      wrgb = V3{dI[0], dI[1], dI[2]} * inv;
    }
    // warp-collective: every lane takes part
    const Pick P = sedge_pick(a, valid, x32, hit.x, j, pix, s, cnt ? cnt + CNT_SEDGE : nullptr);
    if (__any_sync(0xffffffffu, valid && P.n > 0))                 // uniform
      sedge_add(a, w.g, j, P, d, x32, hit.x, flip, pix, s, wrgb, cnt ? cnt + CNT_SEDGE : nullptr, valid && P.n > 0);
  }
}

// A primary-edge item: edge samples [base, base + len) of the frame.
__device__ __noinline__ void pedge_item(const WarpState& w, const BatchFrame& F, long long base, int len,
                                        unsigned long long* cnt) {
  for (int k = threadIdx.x & 31; k < len; k += 32) {
    const long long t = base + k;
    pedge_sample(w.a, w.g, t, cnt, t < F.n_pedge);              // warp-collective
  }
}

// Bounded wait of an edge item until every tile item of frame fi has
// published its hits and d_image.  Returns false when the wait ran out
// (ERR_WAIT set; the item is skipped).
FR_DEV bool wait_tiles(const BatchArgs& b, const BatchFrame& F, int fi) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    const volatile int* done = b.tiles_done + fi;
    int tries = 0;
    while (*done < F.n_tiles) {
      if (++tries > b.wait_limit) { atomicOr(b.err, ERR_WAIT); ok = 0; break; }
      __nanosleep(256);
    }
    __threadfence();
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

}  // namespace

FR_DEV void batch_step_body(const BatchArgs& b) {
  extern __shared__ __align__(16) unsigned char smem[];
  float* sC = reinterpret_cast<float*>(smem);                       // [CS*CS], shared by the block's warps
  WarpState* ws = reinterpret_cast<WarpState*>(smem + batch_smem_head());
  const int lane = threadIdx.x & 31;
  WarpState& w = ws[threadIdx.x >> 5];
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x) sC[i] = 0.0f;
  for (int i = lane; i < 3 * MAX_LIGHTS; i += 32) w.sL[i] = 0.0f;
  __syncthreads();
  int cur = -1;
  while (true) {
    int item = 0;
    if (lane == 0) item = atomicAdd(b.queue, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= b.n_items) break;
    const int2 it = b.items[item];
    const bool is_pedge = (it.x & PEDGE_ITEM) != 0, is_sedge = (it.x & SEDGE_ITEM) != 0;
    const int fi = it.x & ~(PEDGE_ITEM | SEDGE_ITEM);
    const BatchFrame& F = b.frames[fi];
    if (fi != cur) {
      if (cur >= 0) flush_lights(w, lane);
      const int* src = reinterpret_cast<const int*>(&F.a);
      int* dst = reinterpret_cast<int*>(&w.a);
      for (int i = lane; i < (int)(sizeof(RenderArgs) / 4); i += 32) dst[i] = src[i];
      const int* gsrc = reinterpret_cast<const int*>(&F.gb);
      int* gdst = reinterpret_cast<int*>(&w.g);
      for (int i = lane; i < (int)(sizeof(GradBufs) / 4); i += 32) gdst[i] = gsrc[i];
      __syncwarp();
      if (lane == 0) { w.a.iter = *b.iter; w.a.counters = b.counters; w.a.err = b.err; w.a.mesh.max_steps = b.max_steps; }
      __syncwarp();
      cur = fi;
    }
    if (!is_pedge && !is_sedge) {
      double lacc = 0.0;
      if (w.a.spp <= 32) tile_small(w, F, sC, it.y, b.tile_w, b.tile_h, lacc, b.counters);
      else tile_large(w, F, sC, it.y, b.tile_w, b.tile_h, lacc, b.counters);
      for (int off = 16; off > 0; off >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, off);
      // publish the tile's hits and d_image to the frame's edge items
      __threadfence();
      __syncwarp();
      if (lane == 0) {
        atomicAdd(F.loss, lacc);
        atomicAdd(b.tiles_done + fi, 1);
      }
      continue;
    }
    if (is_sedge) {
      const int j = it.y & (SEDGE_LIGHTS - 1);
      if (!light_on(w.a, j)) continue;                             // uniform: no wait for a light that is off
      if (!wait_tiles(b, F, fi)) continue;
      sedge_item(w, F, j, (long long)(it.y >> SEDGE_LIGHT_BITS) * b.sedge_chunk, b.sedge_chunk, b.tile_w,
                 b.tile_h, b.counters);
      continue;
    }
    if (!wait_tiles(b, F, fi)) continue;
    pedge_item(w, F, (long long)it.y * b.pedge_chunk, b.pedge_chunk, b.counters ? b.counters + CNT_PEDGE : nullptr);
  }
  if (cur >= 0) flush_lights(w, lane);
  __syncthreads();
  float* dC = b.frames[0].gb.dC;                 // the specular map is shared by the frames
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x)
    if (sC[i] != 0.0f) atomicAdd(&dC[i], sC[i]);
}

// ---------------------------------------------------------------------------
// Phase kernels

namespace {

// Frame of block b (binary search over block_start) and its arguments copied
// to shared memory.
FR_DEV int phase_frame(const PhaseArgs& p, unsigned char* a_raw, unsigned char* g_raw) {
  __shared__ int s_f;
  if (threadIdx.x == 0) {
    int lo = 0, hi = p.n_frames - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (p.block_start[mid] <= b) lo = mid; else hi = mid - 1;
    }
    s_f = lo;
  }
  __syncthreads();
  const int f = s_f;
  const BatchFrame& F = p.frames[f];
  const int* src = reinterpret_cast<const int*>(&F.a);
  for (int i = threadIdx.x; i < (int)(sizeof(RenderArgs) / 4); i += blockDim.x) reinterpret_cast<int*>(a_raw)[i] = src[i];
  const int* gsrc = reinterpret_cast<const int*>(&F.gb);
  for (int i = threadIdx.x; i < (int)(sizeof(GradBufs) / 4); i += blockDim.x) reinterpret_cast<int*>(g_raw)[i] = gsrc[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    RenderArgs& a = *reinterpret_cast<RenderArgs*>(a_raw);
    a.iter = *p.iter;
    a.counters = p.counters;
    a.err = p.err;
    a.mesh.max_steps = p.max_steps;
  }
  __syncthreads();
  return f;
}

}  // namespace

__global__ void __launch_bounds__(256, 3) k_batch_fwd(PhaseArgs p) {
  __shared__ __align__(16) unsigned char a_raw[sizeof(RenderArgs)];
  __shared__ __align__(16) unsigned char g_raw[sizeof(GradBufs)];
  __shared__ float sC[CS * CS];
  __shared__ float sL[3 * MAX_LIGHTS];
  __shared__ double red[8];
  const int f = phase_frame(p, a_raw, g_raw);
  const RenderArgs& a = *reinterpret_cast<const RenderArgs*>(a_raw);
  const GradBufs& g = *reinterpret_cast<const GradBufs*>(g_raw);
  const BatchFrame& F = p.frames[f];
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x) sC[i] = 0.0f;
  for (int i = threadIdx.x; i < 3 * MAX_LIGHTS; i += blockDim.x) sL[i] = 0.0f;
  __syncthreads();
  const int spp = a.spp;
  const long long tid = (long long)(blockIdx.x - p.block_start[f]) * blockDim.x + threadIdx.x;
  const long long total = (long long)tiled_pixel_count(a.W, a.H) * spp;
  int ip = (int)(tid / spp), s = (int)(tid - (long long)ip * spp);
  int px = 0, py = 0;
  bool valid = tid < total && tile_pixel(ip, a.W, a.H, px, py);
  unsigned long long* cnt = p.counters;
  V3 L{0, 0, 0}, d{0, 0, -1};
  int2 hit = make_int2(-1, 0);
  uint32_t pix = 0, vis = 0u;
  if (valid) d = sample_dir(a, px, py, s, pix);
  L = radiance(a, a.cam.o, d, TAG_LIGHT, pix, (uint32_t)s, cnt, nullptr, &hit, &vis, valid);
  if (!valid) { hit = make_int2(-1, 0); vis = 0u; }
  float v0 = L.x, v1 = L.y, v2 = L.z;
  for (int off = (spp < 32 ? spp : 32) >> 1; off > 0; off >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, off);
    v1 += __shfl_xor_sync(0xffffffffu, v1, off);
    v2 += __shfl_xor_sync(0xffffffffu, v2, off);
  }
  if (spp > 32) {                      // uniform: the pixel spans spp / 32 warps of this block
    __shared__ float wsum[8][3];
    const int w = threadIdx.x >> 5, nw = spp >> 5, w0 = w - w % nw;
    if ((threadIdx.x & 31) == 0) { wsum[w][0] = v0; wsum[w][1] = v1; wsum[w][2] = v2; }
    __syncthreads();
    v0 = 0.0f; v1 = 0.0f; v2 = 0.0f;
    for (int k = 0; k < nw; ++k) { v0 += wsum[w0 + k][0]; v1 += wsum[w0 + k][1]; v2 += wsum[w0 + k][2]; }
  }
  const float inv = 1.0f / (float)spp;
  double lacc = 0.0;
  V3 dv{0, 0, 0};
  if (valid) dv = pixel_loss(F, pix, V3{v0 * inv, v1 * inv, v2 * inv}, s == 0, lacc);
  bool adj = valid && hit.x >= 0 && (dv.x != 0.0f || dv.y != 0.0f || dv.z != 0.0f);
  if (tid < total) g.hits[tid] = adj ? hit : make_int2(-1, 0);
  interior_sample(a, g, sC, sL, pix, s, d, hit.x, __int_as_float(hit.y), dv, cnt ? cnt + CNT_INTERIOR : nullptr,
                        &vis, adj);
  for (int off = 16; off > 0; off >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    if (sum != 0.0) atomicAdd(F.loss, sum);
  }
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x)
    if (sC[i] != 0.0f) atomicAdd(&g.dC[i], sC[i]);
  for (int i = threadIdx.x; i < 3 * a.n_lights; i += blockDim.x)
    if (sL[i] != 0.0f) atomicAdd(&g.dL[i], sL[i]);
}

// The shading point of one thread of the batch's shadow-edge launches: the
// frame's blocks hold its lights one after another, one thread per tiled
// camera sample of the frame.
struct BatchSedgeSample {
  int j;                // light
  bool valid;           // the sample hit the face
  int fh, flip, s;
  uint32_t pix;
  V3 d, x32;
};

FR_DEV BatchSedgeSample batch_sedge_sample(const PhaseArgs& p, int f, const RenderArgs& a, const GradBufs& gb) {
  BatchSedgeSample q;
  const int nb = (p.block_start[f + 1] - p.block_start[f]) / a.n_lights;   // blocks per light
  const int local = (int)blockIdx.x - p.block_start[f];
  q.j = local / nb;
  const int spp = a.spp;
  const long long tid = (long long)(local - q.j * nb) * blockDim.x + threadIdx.x;
  const long long total = (long long)tiled_pixel_count(a.W, a.H) * spp;
  const int2 hit = tid < total ? gb.hits[tid] : make_int2(-1, 0);
  q.fh = hit.x;
  q.valid = tid < total && q.fh >= 0;
  const int ip = (int)(tid / spp);
  q.s = (int)(tid - (long long)ip * spp);
  q.pix = 0;
  q.flip = 1;
  q.d = V3{0, 0, -1};
  q.x32 = V3{0, 0, 0};
  if (q.valid) {
    int px = 0, py = 0;
    tile_pixel(ip, a.W, a.H, px, py);
    q.d = sample_dir(a, px, py, q.s, q.pix);
    q.flip = face_flip(a.mesh, q.fh, q.d);
    q.x32 = hit_point(a.cam.o, q.d, __int_as_float(hit.y));
  }
  return q;
}

// First launch: the search and pick of every (frame, light, sample), stored
// in p.picks at the thread's global index.
FR_DEV void batch_sedge_pick_body(const PhaseArgs& p) {
  __shared__ __align__(16) unsigned char a_raw[sizeof(RenderArgs)];
  __shared__ __align__(16) unsigned char g_raw[sizeof(GradBufs)];
  const int f = phase_frame(p, a_raw, g_raw);
  const RenderArgs& a = *reinterpret_cast<const RenderArgs*>(a_raw);
  const GradBufs& gb = *reinterpret_cast<const GradBufs*>(g_raw);
  const int nb = (p.block_start[f + 1] - p.block_start[f]) / a.n_lights;
  if (!light_on(a, ((int)blockIdx.x - p.block_start[f]) / nb)) return;   // uniform over the block
  const BatchSedgeSample q = batch_sedge_sample(p, f, a, gb);
  const Pick P = pick_light_warp(a, q.valid, q.x32, q.fh, q.j, q.pix, q.s,
                                 p.counters ? p.counters + CNT_SEDGE : nullptr);
  p.picks[(long long)blockIdx.x * blockDim.x + threadIdx.x] = make_int2(q.valid ? P.n : 0, P.slot);
}

// Second launch: the boundary contribution of each pick.
FR_DEV void batch_sedge_add_body(const PhaseArgs& p) {
  __shared__ __align__(16) unsigned char a_raw[sizeof(RenderArgs)];
  __shared__ __align__(16) unsigned char g_raw[sizeof(GradBufs)];
  const int f = phase_frame(p, a_raw, g_raw);
  const RenderArgs& a = *reinterpret_cast<const RenderArgs*>(a_raw);
  const GradBufs& gb = *reinterpret_cast<const GradBufs*>(g_raw);
  const int nb = (p.block_start[f + 1] - p.block_start[f]) / a.n_lights;
  if (!light_on(a, ((int)blockIdx.x - p.block_start[f]) / nb)) return;
  const int2 pk = p.picks[(long long)blockIdx.x * blockDim.x + threadIdx.x];
  if (!__any_sync(0xffffffffu, pk.x > 0)) return;          // uniform over the warp
  const BatchSedgeSample q = batch_sedge_sample(p, f, a, gb);
  V3 wrgb{0, 0, 0};
  if (q.valid) {
    const float* dI = gb.d_image + 3 * (size_t)q.pix;
    wrgb = V3{dI[0], dI[1], dI[2]} * (1.0f / (float)a.spp);
  }
  sedge_contribution(a, gb, q.j, pk.x, pk.y, q.d, q.x32, q.fh, q.flip, q.pix, q.s, wrgb,
                           p.counters ? p.counters + CNT_SEDGE : nullptr, q.valid && pk.x > 0);
}

__global__ void __launch_bounds__(256, 3) k_batch_sedge3(PhaseArgs p) { batch_sedge_pick_body(p); }
__global__ void __launch_bounds__(256, 4) k_batch_sedge4(PhaseArgs p) { batch_sedge_pick_body(p); }
__global__ void __launch_bounds__(256, 4) k_batch_sedge_add(PhaseArgs p) { batch_sedge_add_body(p); }

__global__ void __launch_bounds__(256, 4) k_batch_pedge(PhaseArgs p) {
  __shared__ __align__(16) unsigned char a_raw[sizeof(RenderArgs)];
  __shared__ __align__(16) unsigned char g_raw[sizeof(GradBufs)];
  const int f = phase_frame(p, a_raw, g_raw);
  const RenderArgs& a = *reinterpret_cast<const RenderArgs*>(a_raw);
  const GradBufs& gb = *reinterpret_cast<const GradBufs*>(g_raw);
  long long tid = (long long)(blockIdx.x - p.block_start[f]) * blockDim.x + threadIdx.x;
  // every lane takes part in the warp-cooperative traversals
  pedge_sample(a, gb, tid, p.counters ? p.counters + CNT_PEDGE : nullptr, tid < (long long)a.W * a.H * a.spp);
}

// The persistent kernel at three register budgets (launch bounds of 256
// threads and 2, 3 or 4 resident blocks per SM); the autotuner picks one.
__global__ void __launch_bounds__(256, 2) k_batch_step2(BatchArgs b) { batch_step_body(b); }
__global__ void __launch_bounds__(256, 3) k_batch_step3(BatchArgs b) { batch_step_body(b); }
__global__ void __launch_bounds__(256, 4) k_batch_step4(BatchArgs b) { batch_step_body(b); }

// theta[f] = (alpha, beta_f, delta, c_spec, pose_f, lights_f) from the shared
// vector (alpha, delta, c_spec) and the frame vectors (beta, pose, lights).
__global__ void k_batch_gather_theta(int n_frames, int P, int K_id, int K_exp, int K_alb, int n_light_vals,
                                     const float* __restrict__ ts, const float* __restrict__ tf,
                                     float* __restrict__ theta) {
  const int Pf = K_exp + 6 + n_light_vals;
  const int off_d = K_id + K_exp, off_c = off_d + K_alb, off_p = off_c + CS * CS;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)n_frames * P;
       idx += (long long)gridDim.x * blockDim.x) {
    int f = (int)(idx / P), i = (int)(idx - (long long)f * P);
    const float* fr_ = tf + (size_t)f * Pf;
    float v;
    if (i < K_id) v = ts[i];
    else if (i < off_d) v = fr_[i - K_id];
    else if (i < off_p) v = ts[K_id + (i - off_d)];
    else v = fr_[K_exp + (i - off_p)];
    theta[idx] = v;
  }
}

// Shared and per-frame gradients from the per-frame full gradients, plus the
// prior and light terms of Eq. 1 counted once per parameter:
//   loss = sum_f E_data,f + w1 (|alpha|^2 + |delta|^2 + sum_f |beta_f|^2)
//          + w2 sum_f sum_j |l_fj - m_j|^2,
// m_j the caller's (prior 0) or following frame f's lights (prior 1, 2).
// One thread per output; block 0 also reduces the loss.
__global__ void k_batch_reduce(int n_frames, int P, int K_id, int K_exp, int K_alb, int n_light_vals,
                               const float* __restrict__ theta, const double* __restrict__ grad_full,
                               const double* __restrict__ loss_frames, int prior, const float* __restrict__ m, float w1,
                               float w2, double* __restrict__ grad_s, double* __restrict__ grad_f,
                               double* __restrict__ loss) {
  const int Ps = K_id + K_alb + CS * CS, Pf = K_exp + 6 + n_light_vals;
  const int off_d = K_id + K_exp, off_c = off_d + K_alb, off_p = off_c + CS * CS, off_l = off_p + 6;
  const long long n_out = Ps + (long long)n_frames * Pf;
  const long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o < Ps) {
    int i = (int)o;
    int full = i < K_id ? i : off_d + (i - K_id);
    double sum = 0.0;
    for (int f = 0; f < n_frames; ++f) sum += grad_full[(size_t)f * P + full];
    if (full < off_d + K_alb) sum += 2.0 * (double)w1 * (double)theta[full];   // alpha, delta (frame 0 copy)
    grad_s[i] = sum;
  } else if (o < n_out) {
    int f = (int)((o - Ps) / Pf), i = (int)((o - Ps) - (long long)f * Pf);
    int full = i < K_exp ? K_id + i : off_p + (i - K_exp);
    const float* th = theta + (size_t)f * P;
    double v = grad_full[(size_t)f * P + full];
    if (full < off_d) v += 2.0 * (double)w1 * (double)th[full];
    if (full >= off_l)
      v += 2.0 * (double)w2 * ((double)th[full] - light_prior_mean(th + off_l, n_light_vals / 3, prior, m, full - off_l));
    grad_f[(size_t)f * Pf + i] = v;
  }
  if (blockIdx.x == 0) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int f = threadIdx.x; f < n_frames; f += blockDim.x) acc += loss_frames[f];
    for (int i = threadIdx.x; i < K_id; i += blockDim.x) acc += (double)w1 * (double)theta[i] * (double)theta[i];
    for (int i = threadIdx.x; i < K_alb; i += blockDim.x) {
      double t = theta[off_d + i];
      acc += (double)w1 * t * t;
    }
    for (int f = 0; f < n_frames; ++f) {
      const float* th = theta + (size_t)f * P;
      for (int i = threadIdx.x; i < K_exp; i += blockDim.x) acc += (double)w1 * (double)th[K_id + i] * (double)th[K_id + i];
      for (int i = threadIdx.x; i < n_light_vals; i += blockDim.x) {
        double dd = (double)th[off_l + i] - light_prior_mean(th + off_l, n_light_vals / 3, prior, m, i);
        acc += (double)w2 * dd * dd;
      }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      *loss = s;
    }
  }
}

}  // namespace fr
