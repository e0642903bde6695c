/*
 * facert: differentiable ray-traced rendering of a morphable face inside a
 * virtual light stage, and its gradient, on one GB300 GPU.
 *
 * Method: Dib et al., "Face Reflectance and Geometry Modeling via
 * Differentiable Ray Tracing" (CVMP 2019).
 *   - Face Modeling paragraph: N = 20 fixed square area lights on the
 *     vertices of an isotropically sampled hemisphere, pointing at the origin;
 *     parameters l_j in R^3 (light off = 0), identity alpha in R^80,
 *     expression beta in R^90, pose [R t] in R^6, albedo coefficients
 *     delta in R^80, a 32x32 grey specular map c_spec; Cook-Torrance
 *     reflectance f_r = k_d f_lambert + k_s f_ct on vertex normals
 *     n_i(alpha, beta, R, t).
 *   - Optimization paragraph, Eq. 1: argmin E_data + w1 E_prior + w2 E_light
 *     with E_data = sum_i |p_i^T - p_i^R|^2, E_light = sum_j |l_j - m_j|^2,
 *     p^T = F(f_r, l_j, alpha, beta, R, t) the Monte-Carlo estimator of the
 *     lighting equation; gradients by backpropagation through the
 *     differentiable ray tracer of Li et al. 2018 (edge sampling).
 *
 * Conventions for every entry point:
 *   - Returns FR_OK (0) or a negative FR_ERR_* code; never throws.  The
 *     context keeps a message for the last failure (fr_last_error).
 *   - Pointers documented "device" must be CUDA device memory of the
 *     context's device; pointers documented "host" are host memory read
 *     before the call returns.  The library owns the context and its copies
 *     of the mesh, bases and acceleration structures; the caller owns every
 *     buffer it passes.
 *   - Work is enqueued asynchronously on the context stream (fr_set_stream;
 *     default: the legacy default stream).  Calls on one context must not
 *     overlap: the context's scratch buffers are shared.
 *   - The packed parameter vector theta (FP32, device) has the layout
 *       alpha[K_id] | beta[K_exp] | delta[K_alb] | c_spec[32*32] (row v,
 *       column u) | pose[6] = (rx, ry, rz, tx, ty, tz) | lights[20*3] (RGB)
 *     with R = Rz(rz) Ry(ry) Rx(rx) in radians; P = fr_n_params(ctx).
 *   - Images are H x W x 3 FP32, row-major, pixel (px, py) at index
 *     3*(py*W + px), py = 0 at the top.
 *   - The phases of each call (geometry, forward, interior, primary edges,
 *     shadow-edge search, shadow-edge contributions, adjoint, loss) are
 *     marked as NVTX ranges named "facert <phase>" around their host-side
 *     enqueue.
 */
#ifndef FACERT_H
#define FACERT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FR_OK 0
#define FR_ERR_INVALID_ARG (-1)   /* null pointer, bad size or value */
#define FR_ERR_SHAPE (-2)         /* mesh/basis sizes inconsistent, non-manifold mesh */
#define FR_ERR_CUDA (-3)          /* a CUDA runtime call failed */
#define FR_ERR_OOM (-4)           /* device allocation failed */
#define FR_ERR_DEVICE_LIMIT (-5)  /* a traversal stack or step limit was hit on the device */
#define FR_ERR_NOT_READY (-6)     /* mesh or bases not uploaded yet */

typedef struct fr_ctx fr_ctx;

/* Scene constants.  The paper fixes only N = 20 and the parameter sizes; the
 * remaining values are one reading of the Face Modeling paragraph (pinhole
 * camera at (0, 0, d_cam) looking down -z, square lights of side light_side
 * at distance light_radius, Beckmann roughness beckmann_m).  eps_pedge
 * (pixels) and eps_sedge (light-plane units) are the offsets at which edge
 * samples evaluate the two sides of a visibility boundary; shadow rays
 * accept hits with segment parameter in (shadow_tmin, 1 - shadow_tmin);
 * clip_kappa is the minimum height of an occluder point above the shading
 * point, measured along the light direction. */
typedef struct fr_config {
  float tan_half_fov;
  float d_cam;
  float light_radius;
  float light_side;
  float beckmann_m;
  float eps_pedge;
  float eps_sedge;
  float shadow_tmin;
  float clip_kappa;
  int32_t n_lights;  /* 1..32 */
  /* Readings of what the paper leaves open:
   * brdf_model 0 = Beckmann D with the Cook-Torrance V-cavity G, 1 = GGX D
   * with the separable Smith G (beckmann_m is then GGX alpha);
   * fresnel 0 = F folded into c_spec, 1 = Schlick F with c_spec as the
   * reflectance at normal incidence;
   * light_layout 0 = Fibonacci points on the hemisphere, 1 = the 20 upper
   * vertices of a once-subdivided icosahedron (needs n_lights = 20);
   * light_prior selects m_j of E_light (Eq. 1 names it the j-th light's mean
   * intensity without saying over what): 0 = the caller's m (fr_loss, fr_batch_set_targets), 1 = the mean
   * of the lights, per channel, m_jc = (1/N) sum_k l_kc, 2 = the light's own
   * channel mean, m_jc = (l_jr + l_jg + l_jb) / 3.  In 1 and 2 m follows the
   * lights and the gradient is taken through it (it reduces to
   * 2 w2 (l_jc - m_jc), the deviations summing to zero). */
  int32_t brdf_model;
  int32_t fresnel;
  int32_t light_layout;
  int32_t light_prior;
} fr_config;

/* Fill *cfg with the library defaults (tan_half_fov 0.275, d_cam 4,
 * light_radius 3, light_side 0.6, beckmann_m 0.3, eps_pedge 1e-3,
 * eps_sedge 2e-4, shadow_tmin 1e-4, clip_kappa 1e-5, n_lights 20,
 * brdf_model 0, fresnel 0, light_layout 0, light_prior 0). */
void fr_default_config(fr_config* cfg);

/* Per-call render options.  Samples are drawn from Philox4x32-10 keyed by
 * (seed, iter); W, H >= 1, spp >= 1.  terms selects the gradient terms of
 * fr_render_backward: 1 interior, 2 primary-visibility edges, 4 shadow
 * edges (0 = all). */
typedef struct fr_render_opts {
  int32_t W, H, spp;
  uint32_t seed, iter;
  int32_t terms;
} fr_render_opts;

/* Create a context on CUDA device `device`.  *out receives the context. */
int fr_create(fr_ctx** out, const fr_config* cfg, int32_t device);
void fr_destroy(fr_ctx* ctx);
/* Stream (a cudaStream_t) on which all later work of this context runs. */
int fr_set_stream(fr_ctx* ctx, void* stream);
const char* fr_last_error(const fr_ctx* ctx);
const char* fr_strerror(int32_t code);

/* Topology and mean shape (host pointers).  mean[V*3] FP32 (mu of the
 * morphable model), tris[F*3] int32 counter-clockwise seen from outside,
 * uv[V*2] FP32 specular-map coordinates in [0,1]^2.  Builds the edge list,
 * the vertex-face adjacency and the two bounding-volume hierarchies (over
 * triangles and over edges) from the mean shape; they are refitted on every
 * render.  Fails with FR_ERR_SHAPE on an edge shared by more than two
 * triangles or an out-of-range index. */
int fr_upload_mesh(fr_ctx* ctx, const float* mean, int32_t V, const int32_t* tris, int32_t F,
                   const float* uv);

/* Morphable bases (host pointers, row-major, row 3v+c = coordinate c of
 * vertex v): B_id[3V*K_id], B_exp[3V*K_exp], alb_mean[3V], B_alb[3V*K_alb].
 * Face Modeling paragraph: X = mu + B_id alpha + B_exp beta, albedo =
 * alb_mean + B_alb delta.  Must follow fr_upload_mesh. */
int fr_upload_bases(fr_ctx* ctx, const float* B_id, int32_t K_id, const float* B_exp, int32_t K_exp,
                    const float* alb_mean, const float* B_alb, int32_t K_alb);

/* Number of parameters P of theta for the uploaded bases. */
int32_t fr_n_params(const fr_ctx* ctx);

/* Forward render (Optimization paragraph: p^T = F(...), the Monte-Carlo
 * estimator of the lighting equation).  theta[P] device; image[H*W*3]
 * device, overwritten with the mean over spp of the per-sample radiance:
 * one jittered camera ray per sample, one uniform point per light that is
 * on, a shadow ray for self-shadows, Cook-Torrance shading.  Lights with
 * l_j = 0 are skipped.  aov[H*W*14] device or NULL: per-pixel denoiser
 * features (means over the pixel's samples, misses counting as zero):
 * 0-2 noisy RGB, 3-5 shading normal, 6-8 diffuse albedo, 9 specular albedo,
 * 10 distance to the camera / d_cam, 11 fraction of the lit lights that are
 * visible, 12 variance over samples of the luminance (r+g+b)/3, 13 fraction
 * of samples that hit the face.  Returns FR_ERR_NOT_READY before both
 * uploads. */
int fr_render(fr_ctx* ctx, const float* theta, const fr_render_opts* opts, float* image, float* aov);

/* Gradient of <d_image, image(theta)> with respect to theta (Face Modeling
 * paragraph: backpropagation through the differentiable ray tracer).  Uses
 * the same samples as fr_render with the same opts, recomputes every
 * intersection (no path storage) and adds the edge-sampling terms of Li et
 * al. 2018 for primary visibility and for shadow boundaries on the lights.
 * d_image[H*W*3] FP32 device; grad[P] FP64 device, overwritten
 * (accumulate = 0) or added to (accumulate = 1).  The context grows its
 * device scratch on demand (fr_step likewise): 8 B per camera sample for the
 * primary hits and 8 B per (light, sample) for the shadow-edge picks, 168 MB
 * at 256 x 256 x 16 spp with 20 lights; FR_ERR_OOM if that fails. */
int fr_render_backward(fr_ctx* ctx, const float* theta, const fr_render_opts* opts, const float* d_image,
                       double* grad, int32_t accumulate);

/* Eq. 1: loss = E_data + w1 E_prior + w2 E_light with
 *   E_data  = sum over pixels with mask != 0 of |image - target|^2,
 *   E_prior = |alpha|^2 + |beta|^2 + |delta|^2 (the statistical prior; the
 *             landmark term needs detected landmarks and is not computed),
 *   E_light = sum_j |l_j - m_j|^2, j = 1..N, m_j as fr_config.light_prior
 *             selects.
 * theta[P], image/target[H*W*3] FP32 device; mask[H*W] uint8 device or NULL
 * (all pixels); m[3N] FP32 device or NULL (zero), read only when
 * light_prior is 0; loss: one FP64 device
 * scalar, overwritten; d_image[H*W*3] FP32 device or NULL, overwritten with
 * dE_data/d image; grad[P] FP64 device or NULL: the gradient of
 * w1 E_prior + w2 E_light is ADDED to it. */
int fr_loss(fr_ctx* ctx, const float* theta, int32_t W, int32_t H, const float* image, const float* target,
            const uint8_t* mask, const float* m, float w1, float w2, double* loss, float* d_image,
            double* grad);

/* One step of the optimisation (Eq. 1 and its gradient) in one call: the
 * render of fr_render, the loss of fr_loss and the gradient of both,
 *   grad = d(E_data + w1 E_prior + w2 E_light)/d theta (overwritten),
 * all terms of fr_render_backward unless opts->terms selects some.
 * theta[P], target[H*W*3] FP32 device; mask[H*W] uint8 device or NULL; m
 * as fr_loss; image[H*W*3] FP32 device (written); d_image[H*W*3] FP32
 * device (written with dE_data/d image) or NULL (a context buffer is used);
 * loss: one FP64 device scalar (overwritten); grad[P] FP64 device.
 * Results equal those of fr_render, fr_loss and fr_render_backward with the
 * same opts: the same samples and decisions, values up to FP32 rounding
 * (the same formulas compiled in another kernel) and the order of
 * floating-point additions.  When spp divides 256 the render,
 * the data term's adjoint and the interior adjoint run as one kernel (a
 * pixel's samples lie in one block of 256 threads): each sample's interior
 * adjoint reuses its primary hit and the shadow decisions of the lights that
 * are on; the geometry is prepared once.  Other spp run the three calls in
 * sequence.  Timings (fr_get_timings): the
 * fused kernel is the forward phase. */
int fr_step(fr_ctx* ctx, const float* theta, const fr_render_opts* opts, const float* target, const uint8_t* mask,
            const float* m, float w1, float w2, float* image, float* d_image, double* loss, double* grad);

/* Geometry stage alone (Face Modeling paragraph), for inspection and tests:
 * posed vertices X[V*3] FP32, unit vertex normals N[V*3] FP32 and albedo
 * A[V*3] FP32, all device (any may be NULL).  Returns the number of camera
 * silhouette edges (>= 0) or an error. */
int fr_geometry(fr_ctx* ctx, const float* theta, float* X, float* N, float* A);

/* fr_geometry for callers that must not allocate device memory during the
 * call (their allocator owns the device, their memory budget is fixed at
 * start-up, or they cannot afford the synchronisation an allocation may
 * cause).  The paper has no counterpart: this is a deployment variant.
 * Same outputs and return value as fr_geometry; the camera-silhouette
 * compaction keeps its scratch (one int per 256 edges) in a static device
 * array of 4096 ints, so meshes with more than 1,048,576 edges are rejected
 * with FR_ERR_INVALID_ARG.  The array is shared by every call on a device and
 * kept until the process exits; calls whose GPU work overlaps race on it.
 * The first call on a device looks up the array's device address (set-up);
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: after cudaDeviceReset (or any other reset of the
 * device's primary context) it is stale, so do not call this entry point on
 * that device again.  Calls no cudaMalloc or cudaFree. */
int fr_geometry_noalloc(fr_ctx* ctx, const float* theta, float* X, float* N, float* A);

/* Camera-silhouette edges found by the last geometry preparation on this
 * context (any call that renders, differentiates or returns geometry): their
 * canonical edge ids in increasing order, written to out[cap] (host; the
 * first cap of them).  Canonical edges are the mesh's edges sorted by
 * (smaller vertex, larger vertex).  Returns their number (which may exceed
 * cap) after a stream synchronisation.  For inspection and tests. */
int fr_silhouettes(fr_ctx* ctx, int32_t* out, int32_t cap);

/* Per-vertex position gradient of the last fr_render_backward on this
 * context (after the normals adjoint, before the pose and basis
 * contractions): dX[V*3] FP32 device.  For inspection and tests. */
int fr_vertex_grad(fr_ctx* ctx, float* dX);

/* Light stage frames (host, out[n_lights*12]: centre, e1, e2, direction). */
int fr_light_stage(const fr_ctx* ctx, float* out);

/* Wait for the context stream; returns FR_ERR_DEVICE_LIMIT (and clears the
 * flag) if a kernel hit its traversal stack or step limit since the last
 * fr_sync, FR_ERR_CUDA if the stream reported an error, else FR_OK. */
int fr_sync(fr_ctx* ctx);

/* Device-side limits of this context's later calls (a robustness guard with
 * no counterpart in the paper).
 *   max_steps (>= 1): node visits one traversal of a hierarchy may make
 *     before it stops and raises FR_ERR_DEVICE_LIMIT at the next fr_sync
 *     (default 65536; a valid hierarchy needs a few hundred);
 *   wait_limit (>= 0): tries (about 256 ns apart) an edge work item
 *     (shadow or primary edges) of the persistent batch kernel waits for its
 *     frame's tiles before it skips its samples and raises
 *     FR_ERR_DEVICE_LIMIT (default 4194304, about a second).
 * A call that stops at a limit leaves its outputs incomplete; the context
 * stays usable.  FR_ERR_INVALID_ARG for values out of range. */
int fr_set_limits(fr_ctx* ctx, int32_t max_steps, int32_t wait_limit);

/* Work counts of the last fr_render / fr_render_backward call (or batch
 * step), read back after a stream synchronisation.  out[24]: six counts
 * (BVH nodes visited by rays, triangle tests, nodes of the 4-wide edge
 * hierarchy visited -- once per warp, the search being warp-wide --, exact
 * silhouette tests of (shading point, edge) pairs, clip tests of pairs that
 * passed the silhouette and adjacency tests, leaf edges classified against
 * the box of a warp's shading points -- once per warp) for each of the
 * forward, interior, primary-edge and shadow-edge kernels, in that order.
 * Collected only when enabled with fr_set_counters(ctx, 1). */
int fr_set_counters(fr_ctx* ctx, int32_t enable);
int fr_get_counters(fr_ctx* ctx, uint64_t* out);

/* Per-phase device time (CUDA events on the context stream) of the most
 * recent call containing each phase, in ms: out[8] = geometry (morphable
 * model, normals, refits, silhouettes), forward render, interior adjoint,
 * primary edges, shadow-edge search and pick, normal/geometry adjoint, loss,
 * shadow-edge contributions.  Events are
 * recorded only while enabled with fr_set_timing(ctx, 1); fr_get_timings
 * synchronises the stream.  A phase not run since enabling reads 0. */
int fr_set_timing(fr_ctx* ctx, int32_t enable);
int fr_get_timings(fr_ctx* ctx, float* out);

/* Per-pixel MLP denoiser (motivated by the Results and Conclusion paragraph:
 * few samples give a noisy render, many samples a slow optimisation).
 * y = rgb + cov s_out (W4 h3 + b4), h_l = relu(W_l h_{l-1} + b_l),
 * h_0 = (t(x) - mu) * is, 14 -> 64 -> 64 -> 64 -> 3 over the fr_render
 * features (t: feature 12 enters as its square root; mu, is, s_out fixed
 * standardisation constants that training leaves unchanged; cov = feature
 * 13, so pixels the face does not cover pass through); FP16 weights
 * and activations on the tensor cores, FP32 accumulation.  Master weights
 * are FP32, packed W1[64][14] b1[64] W2[64][64] b2[64] W3[64][64] b3[64]
 * W4[3][64] b4[3] mu[14] is[14] s_out (fr_denoiser_n_weights() = 9504). */
int32_t fr_denoiser_n_weights(void);
/* Copy weights in (host w[n]); resets the Adam state.  Allocates the
 * denoiser's buffers on first use. */
int fr_denoiser_set_weights(fr_ctx* ctx, const float* w, int32_t n);
int fr_denoiser_get_weights(fr_ctx* ctx, float* w, int32_t n);
/* Inference on n_pix pixels: aov[n_pix*14] device features, out[n_pix*3]
 * device.  With d_out[n_pix*3] (device, the adjoint of out), also writes
 * d_rgb[n_pix*3] = J^T d_out, J = dy/d(noisy rgb), the image-space adjoint
 * to hand to fr_render_backward (other features are held constant). */
int fr_denoise(fr_ctx* ctx, const float* aov, int32_t n_pix, float* out, const float* d_out, float* d_rgb);
/* One Adam step (lr, beta 0.9/0.999, eps 1e-8) on the mean over pixels of
 * |y - target|^2; target[n_pix*3] device; loss: one FP64 device scalar
 * (the loss before the step). */
int fr_denoiser_train_step(fr_ctx* ctx, const float* aov, const float* target, int32_t n_pix, float lr,
                           double* loss);
/* Gradient of the last training step (host g[n]), for tests. */
int fr_denoiser_get_grad(fr_ctx* ctx, float* g, int32_t n);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected with step >= 1)
 * on theta[P] (FP32, device) from grad[P] (FP64, device), with moment
 * buffers m[P], v[P] (FP32, device, zero before the first step) and
 * per-parameter learning rates lr[P] (FP32, device; 0 freezes a parameter,
 * which is how the staged schedule of the Optimization paragraph selects
 * the groups it optimises).  Afterwards lights are clamped to >= 0 and
 * specular texels to [0, 1]. */
int fr_adam_step(fr_ctx* ctx, float* theta, const double* grad, float* m, float* v, const float* lr, int32_t step);

/* Number of kernels this context has launched since it was created (a
 * replayed batch graph counts its kernel nodes on every replay). */
uint64_t fr_launch_count(const fr_ctx* ctx);

/* Roofline denominators of this library's kernels, measured on `device`
 * (a measurement utility with no counterpart in the paper: the render and
 * its gradient are FP32 ALU work on data resident in L2).
 *   fp32_tflops (host, written): best FP32 FMA throughput of the CUDA cores,
 *     2 FLOP per FMA, over five timed runs of independent FMA chains on
 *     every SM (TFLOP/s);
 *   l2_read_gbs (host, written): best streaming read bandwidth of a 32 MiB
 *     buffer resident in L2, loads that bypass L1 (GB/s);
 *   sm_count (host, written, may be NULL): multiprocessors of the device.
 * Allocates 32 MiB of device memory for the duration of the call, on its
 * own stream, and frees it.  FR_ERR_CUDA for a bad device or a failed
 * runtime call, FR_ERR_OOM if the buffer cannot be allocated. */
int fr_probe_peaks(int32_t device, double* fp32_tflops, double* l2_read_gbs, int32_t* sm_count);

/* ---------------------------------------------------------------------------
 * Batched frames.  Several frames of one face (a video, or crops of uneven
 * size) fitted together: Eq. 1 of the Optimization paragraph summed over
 * frames, with identity alpha, albedo delta and specular map c_spec shared
 * and expression beta, pose and lights per frame.  One step renders every
 * frame, takes the loss and its gradient with respect to all parameters:
 *   loss = sum_f E_data,f + w1 (|alpha|^2 + |delta|^2 + sum_f |beta_f|^2)
 *          + w2 sum_f sum_j |l_fj - m_j|^2.
 * The paper fits single images; batching is this library's extension (the
 * per-frame arithmetic is that of fr_render / fr_loss / fr_render_backward,
 * with the same samples for equal (seed, iter)).
 *
 * A step is one CUDA graph: per-frame geometry and refits, the render +
 * loss + backward of all frames (three launches over all frames, or one
 * persistent launch: fr_tile_config), and the per-frame geometry adjoints.
 * The launch configuration comes from fr_batch_autotune or
 * fr_batch_set_config.
 *
 * Layouts (all device, FP32 unless stated):
 *   theta_shared[Ps] = alpha[K_id] | delta[K_alb] | c_spec[32*32],
 *   theta_frames[F][Pf] = beta[K_exp] | pose[6] | lights[3N],
 *   Ps = fr_batch_n_shared(ctx), Pf = fr_batch_n_frame(ctx);
 *   images, targets: the frames' H_f x W_f x 3 images one after another in
 *   frame order (frame f starts at pixel sum_{g<f} W_g H_g);
 *   masks: the same packing of H_f x W_f uint8.
 * ------------------------------------------------------------------------- */
typedef struct fr_batch fr_batch;

/* One frame: crop size and the seed of its samples. */
typedef struct fr_frame {
  int32_t W, H;
  uint32_t seed;
} fr_frame;

/* Launch configuration of a step's render + loss + backward.
 *   fused = 0 (phased, the default): three launches, each over all frames
 *     in frame order -- forward + loss + interior adjoint, shadow edges
 *     (light-major within a frame), primary edges; blocks of 256 threads;
 *     min_blocks 3 or 4 is the register budget of the shadow-edge kernel
 *     (65536 / (256 * min_blocks) registers per thread); tile_w, tile_h and
 *     block are ignored (8x8 tiles).  Needs spp dividing 256 (a pixel's
 *     samples in one block of 256 threads; the default for such spp).
 *   fused = 1: one persistent launch whose warps take work items from a
 *     queue: tiles of tile_w x tile_h pixels (sides 1..64) that run forward,
 *     loss and interior terms together, then chunks of camera samples for
 *     one light's shadow-edge term (light-major within each frame), then
 *     chunks of primary-edge samples; block threads (a multiple of 32 up to
 *     256);
 *     min_blocks 2, 3 or 4 is the kernel's register budget.
 * ms is the time of one step measured by fr_batch_autotune (0 otherwise). */
typedef struct fr_tile_config {
  int32_t tile_w, tile_h, block, min_blocks, fused;
  float ms;
} fr_tile_config;

/* Ps = K_id + K_alb + 32*32, the length of theta_shared and grad_shared, and
 * Pf = K_exp + 6 + 3N, the length of one frame's theta_frames and
 * grad_frames row, for the context's bases and lights (FR_ERR_INVALID_ARG
 * for a null context). */
int32_t fr_batch_n_shared(const fr_ctx* ctx);
int32_t fr_batch_n_frame(const fr_ctx* ctx);

/* The work-item list of the persistent launch (fused = 1) for frames
 * [n_frames] at spp with tiles of tile_w x tile_h pixels and n_lights
 * lights, in queue order.  Host only: no context, no GPU.  Item i is
 * (items[2i], items[2i+1]) = (x, y):
 *   x = f (frame index): a tile item, y = its tile (row-major, tiles of
 *     the frame's W x H pixels);
 *   x = f | 1 << 29: a shadow-edge item, y = k << 5 | j: light j, samples
 *     [32 k, 32 k + 32) of the frame's samples in tile order (tile, then
 *     pixel row-major within the tile, then sample);
 *   x = f | 1 << 30: a primary-edge item, y = k: the frame's primary-edge
 *     samples [32 k, 32 k + 32).
 * All tile items come first, then the shadow-edge items (light-major within
 * each frame), then the primary-edge items; frames with more pixels first
 * within each group.  Writes min(cap, length) items (cap >= 0; items may be
 * NULL when cap = 0) and the length to *n_out.  FR_ERR_INVALID_ARG for the
 * arguments fr_batch_create or fr_batch_set_config refuses, or for a list
 * beyond the queue's range; FR_ERR_OOM when host memory for the list runs
 * out. */
int fr_batch_plan(const fr_frame* frames, int32_t n_frames, int32_t spp, int32_t tile_w, int32_t tile_h,
                  int32_t n_lights, int32_t* items, int64_t cap, int64_t* n_out);

/* Create a batch of frames[n_frames] (host array; 1..4096 frames, each
 * with W, H >= 1, W H <= 2^26 and W H spp < 2^31) at spp samples per pixel
 * (dividing 32, or a multiple of 32) on a context with mesh and bases
 * uploaded.  Allocates every per-frame buffer the steps use (about 30 MB per
 * frame for a 35,709-vertex mesh, plus the images); the buffers that depend
 * on the launch configuration (primary hits, shadow-edge picks, the
 * persistent launch's work list) are sized at the first step with that
 * configuration.  *out receives the batch; it must be destroyed
 * (fr_batch_destroy; NULL is ignored) before its context.  The batch is
 * sized for the context's current mesh and bases: after a later
 * fr_upload_mesh or fr_upload_bases, fr_batch_step and fr_batch_autotune
 * fail with FR_ERR_NOT_READY (create a new batch).  FR_ERR_NOT_READY before
 * the mesh and bases are uploaded, FR_ERR_INVALID_ARG for sizes out of
 * range, FR_ERR_OOM when device memory runs out (nothing is kept). */
int fr_batch_create(fr_ctx* ctx, const fr_frame* frames, int32_t n_frames, int32_t spp, fr_batch** out);
void fr_batch_destroy(fr_batch* b);

/* Targets (packed images), masks (packed uint8, or NULL for all pixels) and
 * the light prior m[3N] (or NULL for zero; used only when the context's
 * light_prior is 0): copied into the batch (device to
 * device, on the context stream) and used by every later step. */
int fr_batch_set_targets(fr_batch* b, const float* targets, const uint8_t* masks, const float* m);

/* One step for parameters (theta_shared, theta_frames) and sample stream
 * iter.  Outputs (device, each may be NULL): loss (one FP64), grad_shared[Ps]
 * and grad_frames[F][Pf] (FP64, overwritten), images (packed, FP32).
 * Enqueued on the context stream; the first step with a configuration or
 * weights (w1, w2) not seen before captures the graph.  A device-side
 * traversal limit or an edge item's wait that expired is reported by the
 * next fr_sync (FR_ERR_DEVICE_LIMIT). */
int fr_batch_step(fr_batch* b, const float* theta_shared, const float* theta_frames, float w1, float w2,
                  uint32_t iter, double* loss, double* grad_shared, double* grad_frames, float* images);

/* Autotuner: time one step (mean of `reps` graph replays after one warm-up
 * replay, CUDA events on the context stream) for every candidate launch
 * configuration that fits the device and the batch, keep the fastest, and
 * return the table (host, up to cap entries; *n_out receives the count).
 * Candidates: phased with min_blocks 3 and 4; fused with tiles 2x2 and 4x4,
 * blocks of 256 and min_blocks 2 and 4.  Results do not depend on the
 * configuration beyond the order of floating-point atomic additions (and,
 * for spp a multiple of 32, the order of the pixel sums). */
int fr_batch_autotune(fr_batch* b, const float* theta_shared, const float* theta_frames, int32_t reps,
                      fr_tile_config* table, int32_t cap, int32_t* n_out);
int fr_batch_get_config(const fr_batch* b, fr_tile_config* out);
/* Set the configuration by hand (FR_ERR_INVALID_ARG if it does not fit). */
int fr_batch_set_config(fr_batch* b, const fr_tile_config* cfg);

#ifdef __cplusplus
}
#endif

#endif /* FACERT_H */
