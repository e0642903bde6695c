// Monte-Carlo render of the light stage and its gradient.
//
// Forward (Optimization paragraph, p^T = F(f_r, l_j, alpha, beta, R, t)):
// one thread per (pixel, sample): jittered camera ray, closest hit, one
// uniform point on every light that is on, a shadow ray for self-shadows,
// Cook-Torrance shading (Face Modeling paragraph).
//
// Backward (Face Modeling paragraph: backpropagation through Li et al.'s
// differentiable ray tracer): every intersection is recomputed with the same
// samples.  Three kernels add into per-vertex and per-parameter FP32
// accumulators:
//   k_bwd_interior  exact derivative of each sample's estimate with its
//                   decisions held fixed (all lights, for dL/dl_j);
//   k_bwd_pedge     primary-visibility edge sampling: W*H*spp samples placed
//                   systematically (one random offset) along the camera
//                   silhouette edges taken together, radiance differenced
//                   across the edge;
//   k_bwd_sedge     shadow-boundary edge sampling: per camera sample and light
//                   that is on, one edge picked uniformly (minimum Philox key)
//                   among the edges that are silhouettes seen from the shading
//                   point and whose central projection crosses the light square.
#include "render_device.cuh"

namespace fr {

// AOV = true also writes the denoiser features aov[14 * pixel + k]:
// 0-2 noisy RGB, 3-5 shading normal, 6-8 diffuse albedo, 9 specular albedo,
// 10 depth, 11 visible-light fraction, 12 variance over spp of the
// luminance (r+g+b)/3, 13 coverage (fraction of samples that hit), all means
// over the pixel's samples (misses count as zero).
template <bool AOV>
FR_DEV void render_fwd_body(const RenderArgs& a, float* __restrict__ image, float* __restrict__ aov) {
  const int spp = a.spp;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)tiled_pixel_count(a.W, a.H) * spp;
  int ip = (int)(tid / spp), s = (int)(tid - (long long)ip * spp);
  int px = 0, py = 0;
  bool valid = tid < total && tile_pixel(ip, a.W, a.H, px, py);
  unsigned long long* cnt = a.counters;      // forward: counters 0..3
  constexpr int NV = AOV ? 15 : 3;           // RGB (+ 11 features + squared luminance)
  float v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0f;
  uint32_t pix = 0;
  {
    // every lane takes part in the warp-cooperative traversal
    V3 d = valid ? sample_dir(a, px, py, s, pix) : V3{0, 0, -1};
    SampleAux aux{V3{0, 0, 0}, V3{0, 0, 0}, 0.0f, 0.0f, 0.0f, 0.0f};
    V3 L = radiance(a, a.cam.o, d, TAG_LIGHT, pix, (uint32_t)s, cnt, AOV ? &aux : nullptr, nullptr, nullptr,
                          valid);
    v[0] = L.x; v[1] = L.y; v[2] = L.z;
    if (AOV) {
      v[3] = aux.n.x; v[4] = aux.n.y; v[5] = aux.n.z;
      v[6] = aux.rho.x; v[7] = aux.rho.y; v[8] = aux.rho.z;
      v[9] = aux.cs; v[10] = aux.depth; v[11] = aux.vis;
      float Y = (L.x + L.y + L.z) * (1.0f / 3.0f);
      v[12] = Y * Y;
      v[13] = aux.hit;
      v[14] = Y;
    }
  }
  const float inv = 1.0f / (float)spp;
  bool shuffle = spp <= 32 && (32 % spp) == 0;
  if (shuffle) {
    for (int off = spp >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
    }
    if (!(valid && s == 0)) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) image[3 * pix + k] = v[k] * inv;
    if (AOV) {
      float* o = aov + 14 * (size_t)pix;
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = v[k] * inv;
      float mY = v[14] * inv;
      o[12] = fmaxf(0.0f, v[12] * inv - mY * mY);
      o[13] = v[13] * inv;
    }
  } else if (valid) {
#pragma unroll
    for (int k = 0; k < 3; ++k) atomicAdd(&image[3 * pix + k], v[k] * inv);
    if (AOV) {
      // the caller finishes the variance (aux[12] holds E[Y^2], scratch E[Y]) in k_aov_finish
      float* o = aov + 14 * (size_t)pix;
#pragma unroll
      for (int k = 0; k < 12; ++k) atomicAdd(&o[k], v[k] * inv);
      atomicAdd(&o[12], v[12] * inv);
      atomicAdd(&o[13], v[13] * inv);
      atomicAdd(&a.aov_scratch[pix], v[14] * inv);
    }
  }
}

__global__ void __launch_bounds__(256, 4) k_render_fwd(RenderArgs a, float* __restrict__ image) {
  render_fwd_body<false>(a, image, nullptr);
}

__global__ void __launch_bounds__(256) k_render_fwd_aov(RenderArgs a, float* __restrict__ image,
                                                        float* __restrict__ aov) {
  render_fwd_body<true>(a, image, aov);
}

// Variance of the luminance for the atomic path: E[Y^2] - E[Y]^2.
__global__ void k_aov_finish(int n_pix, float* __restrict__ aov, const float* __restrict__ meanY) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pix) return;
  float m = meanY[p];
  aov[14 * (size_t)p + 12] = fmaxf(0.0f, aov[14 * (size_t)p + 12] - m * m);
}

__global__ void __launch_bounds__(256, 3) k_bwd_interior(RenderArgs a, GradBufs gb) {
  __shared__ float sC[CS * CS];
  __shared__ float sL[3 * MAX_LIGHTS];
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x) sC[i] = 0.0f;
  for (int i = threadIdx.x; i < 3 * MAX_LIGHTS; i += blockDim.x) sL[i] = 0.0f;
  __syncthreads();
  const int spp = a.spp;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)tiled_pixel_count(a.W, a.H) * spp;
  int ip = (int)(tid / spp), s = (int)(tid - (long long)ip * spp);
  int px = 0, py = 0;
  unsigned long long* cnt = a.counters ? a.counters + CNT_INTERIOR : nullptr;
  bool in_image = tid < total && tile_pixel(ip, a.W, a.H, px, py);
  if (tid < total && !in_image && gb.hits) gb.hits[tid] = make_int2(-1, 0);
  {
    // every lane takes part in the warp-cooperative traversals
    uint32_t pix = 0;
    V3 d{0, 0, -1}, dimg{0, 0, 0};
    if (in_image) {
      d = sample_dir(a, px, py, s, pix);
      const float* dI = gb.d_image + 3 * (size_t)pix;
      dimg = V3{dI[0], dI[1], dI[2]};
    }
    const bool want = in_image && (dimg.x != 0.0f || dimg.y != 0.0f || dimg.z != 0.0f);
    float t = 0.0f;
    int f = closest_hit_warp(a.mesh, want, a.cam.o, d, t, a.err, cnt);
    if (!want) { f = -1; t = 0.0f; }
    if (in_image && gb.hits) gb.hits[tid] = make_int2(f, __float_as_int(t));
    interior_sample(a, gb, sC, sL, pix, s, d, f, t, dimg, cnt, nullptr, f >= 0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x)
    if (sC[i] != 0.0f) atomicAdd(&gb.dC[i], sC[i]);
  for (int i = threadIdx.x; i < 3 * a.n_lights; i += blockDim.x)
    if (sL[i] != 0.0f) atomicAdd(&gb.dL[i], sL[i]);
}

// Fused render, data term and interior adjoint of one optimisation step
// (Eq. 1), for spp dividing 256 (blocks of 256 threads) so that a pixel's
// samples lie in one block: the pixel's mean is a shuffle reduction (plus a
// shared-memory sum over its spp / 32 warps when spp > 32), its adjoint
// 2 mask (image - target) is known in the block that rendered it, and each
// sample's interior adjoint starts from the same primary hit and the shadow
// decisions of the lights that are on (only lights that are off trace shadow
// rays again).  For spp dividing 32 the image equals k_render_fwd's and the
// adjoint k_loss_data's up to FP32 rounding (the compiler contracts the two
// kernels' shading into FMAs differently); the hits written for the edge
// passes are the same decisions as k_bwd_interior's.
__global__ void __launch_bounds__(256, 5) k_step_fwd(RenderArgs a, GradBufs gb, StepBufs sb) {
  __shared__ float sC[CS * CS];
  __shared__ float sL[3 * MAX_LIGHTS];
  __shared__ double red[8];
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x) sC[i] = 0.0f;
  for (int i = threadIdx.x; i < 3 * MAX_LIGHTS; i += blockDim.x) sL[i] = 0.0f;
  __syncthreads();
  const int spp = a.spp;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)tiled_pixel_count(a.W, a.H) * spp;
  const int ip = (int)(tid / spp), s = (int)(tid - (long long)ip * spp);
  int px = 0, py = 0;
  const bool valid = tid < total && tile_pixel(ip, a.W, a.H, px, py);
  unsigned long long* cnt = a.counters;
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
  float dv[3] = {0.0f, 0.0f, 0.0f};
  if (valid) {
    const float I[3] = {v0 * inv, v1 * inv, v2 * inv};
    const bool in = sb.mask ? sb.mask[pix] != 0 : true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double diff = (double)I[c] - (double)sb.target[3 * (size_t)pix + c];
      if (in && s == 0) lacc += diff * diff;
      dv[c] = in ? (float)(2.0 * diff) : 0.0f;
      if (s == 0) {
        sb.image[3 * (size_t)pix + c] = I[c];
        sb.d_image[3 * (size_t)pix + c] = dv[c];
      }
    }
  }
  const bool adj = valid && hit.x >= 0 && (dv[0] != 0.0f || dv[1] != 0.0f || dv[2] != 0.0f);
  if (tid < total && gb.hits) gb.hits[tid] = adj ? hit : make_int2(-1, 0);
  if (sb.interior)                     // uniform
    interior_sample(a, gb, sC, sL, pix, s, d, hit.x, __int_as_float(hit.y), V3{dv[0], dv[1], dv[2]},
                          cnt ? cnt + CNT_INTERIOR : nullptr, &vis, adj);
  for (int off = 16; off > 0; off >>= 1) lacc += __shfl_xor_sync(0xffffffffu, lacc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
    if (sum != 0.0) atomicAdd(sb.loss, sum);
  }
  for (int i = threadIdx.x; i < CS * CS; i += blockDim.x)
    if (sC[i] != 0.0f) atomicAdd(&gb.dC[i], sC[i]);
  for (int i = threadIdx.x; i < 3 * a.n_lights; i += blockDim.x)
    if (sL[i] != 0.0f) atomicAdd(&gb.dL[i], sL[i]);
}

__global__ void __launch_bounds__(256, 4) k_bwd_pedge(RenderArgs a, GradBufs gb) {
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  // every lane takes part in the warp-cooperative traversals
  pedge_sample(a, gb, tid, a.counters ? a.counters + CNT_PEDGE : nullptr, tid < (long long)a.W * a.H * a.spp);
}

// The shading point of one thread of the shadow-edge kernels: one thread per
// (light, tiled camera sample), light-major (blockIdx.y is the light).  The
// primary hit comes from the interior pass of the same backward call
// (gb.hits).
struct SedgeSample {
  long long tid, total;
  bool valid;           // the sample hit the face
  int f, flip, s;
  uint32_t pix;
  V3 d, x32;
};

FR_DEV SedgeSample sedge_sample(const RenderArgs& a, const GradBufs& gb, long long tid) {
  SedgeSample q;
  const int spp = a.spp;
  q.tid = tid;
  q.total = (long long)tiled_pixel_count(a.W, a.H) * spp;
  const int2 hit = q.tid < q.total ? gb.hits[q.tid] : make_int2(-1, 0);
  q.f = hit.x;
  q.valid = q.tid < q.total && q.f >= 0;
  const int ip = (int)(q.tid / spp);
  q.s = (int)(q.tid - (long long)ip * spp);
  q.pix = 0;
  q.flip = 1;
  q.d = V3{0, 0, -1};
  q.x32 = V3{0, 0, 0};
  if (q.valid) {
    int px = 0, py = 0;
    tile_pixel(ip, a.W, a.H, px, py);
    q.d = sample_dir(a, px, py, q.s, q.pix);
    q.flip = face_flip(a.mesh, q.f, q.d);
    q.x32 = hit_point(a.cam.o, q.d, __int_as_float(hit.y));
  }
  return q;
}

// Shadow-edge term, first kernel: the candidate search and pick of every
// (light, camera sample) (pick_light_warp_n), stored in picks[j * total +
// sample] as (number of candidates, leaf slot of the pick).  A warp serves
// one light and 32 NS neighbouring samples (lane l holds samples 32 NS w +
// 32 q + l), which share one walk, so the search stays coherent, and warps
// of lights that are off retire at once.  Every lane reaches the
// warp-cooperative search; samples without a shading point take part with
// valid = false.
template <int NS>
FR_DEV void bwd_sedge_body(const RenderArgs& a, const GradBufs& gb, int2* __restrict__ picks) {
  const int j = blockIdx.y;
  if (!light_on(a, j)) return;                 // uniform over the block
  const int lane = threadIdx.x & 31;
  const long long wbase = ((long long)blockIdx.x * blockDim.x + (threadIdx.x - lane)) * NS;
  SedgeSample qs[NS];
  SedgePoint pt[NS];
#pragma unroll
  for (int qi = 0; qi < NS; ++qi) {
    qs[qi] = sedge_sample(a, gb, wbase + 32 * qi + lane);
    pt[qi] = SedgePoint{qs[qi].valid, qs[qi].x32, qs[qi].f, qs[qi].pix, qs[qi].s};
  }
  Pick P[NS];
  pick_light_warp_n<NS>(a, pt, j, a.counters ? a.counters + CNT_SEDGE : nullptr, P);
#pragma unroll
  for (int qi = 0; qi < NS; ++qi)
    if (qs[qi].tid < qs[qi].total)
      picks[j * qs[qi].total + qs[qi].tid] = make_int2(qs[qi].valid ? P[qi].n : 0, P[qi].slot);
}
// two points per lane (images of 256 x 256 pixels and more), one point
__global__ void __launch_bounds__(256, 4) k_bwd_sedge(RenderArgs a, GradBufs gb, int2* __restrict__ picks) {
  bwd_sedge_body<2>(a, gb, picks);
}
__global__ void __launch_bounds__(256, 4) k_bwd_sedge_1(RenderArgs a, GradBufs gb, int2* __restrict__ picks) {
  bwd_sedge_body<1>(a, gb, picks);
}

// Shadow-edge term, second kernel: the boundary contribution of each pick
// (sedge_contribution), in the same thread layout; warps without a pick
// retire at once.  Apart from the search, each kernel has the registers to
// itself: fused into one kernel the two spilled and ran 8 % slower.
__global__ void __launch_bounds__(256, 4) k_bwd_sedge_add(RenderArgs a, GradBufs gb,
                                                          const int2* __restrict__ picks) {
  const int j = blockIdx.y;
  if (!light_on(a, j)) return;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)tiled_pixel_count(a.W, a.H) * a.spp;
  const int2 p = tid < total ? picks[j * total + tid] : make_int2(0, -1);
  if (!__any_sync(0xffffffffu, p.x > 0)) return;          // uniform over the warp
  const SedgeSample q = sedge_sample(a, gb, tid);
  V3 wrgb{0, 0, 0};
  if (q.valid) {
    const float* dI = gb.d_image + 3 * (size_t)q.pix;
    wrgb = V3{dI[0], dI[1], dI[2]} * (1.0f / (float)a.spp);
  }
  sedge_contribution(a, gb, j, p.x, p.y, q.d, q.x32, q.f, q.flip, q.pix, q.s, wrgb,
                           a.counters ? a.counters + CNT_SEDGE : nullptr, q.valid && p.x > 0);
}

}  // namespace fr
