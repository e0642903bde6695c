// C-ABI of the facert library (declared in include/facert.h): context,
// uploads, acceleration-structure build, and the render / backward / loss
// entry points, each a fixed sequence of kernel launches on the context
// stream.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "context.cuh"

using namespace fr;

namespace {

// Edges per leaf of the edge hierarchy (the most a leaf code holds).  A node
// visit of the warp-wide search is a dependent round trip to memory, while
// the edges of a leaf load independently: measured on the full face,
// leaves of 8 edges beat 6, 4, 2 and 1.
constexpr int EDGE_LEAF = 8;
// Triangles per leaf of the triangle hierarchy.  The warp-cooperative walk
// tests a leaf's triangles for every lane whose box test passed, so small
// leaves pay: on the full face at 256x256x16, leaves of 1 / 2 / 3 / 4 / 6 /
// 8 triangles gave steps of 16.90 / 16.42 / 16.43 / 16.73 / 17.15 / 17.87 ms.
constexpr int TRI_LEAF = 2;

// Binary BVH in the device layout of common.cuh plus the refit topology.
struct HostBVH {
  std::vector<float4> nodes;          // 4 per node
  std::vector<int> perm;              // leaf slot -> primitive id
  std::vector<int> leaf_first, leaf_count, leaf_parent, leaf_slot;
  std::vector<int> node_parent, node_slot;
};

struct Box {
  float lo[3], hi[3];
  void reset() { for (int i = 0; i < 3; ++i) { lo[i] = 3e38f; hi[i] = -3e38f; } }
  void grow(const float* p) { for (int i = 0; i < 3; ++i) { lo[i] = std::min(lo[i], p[i]); hi[i] = std::max(hi[i], p[i]); } }
  void grow(const Box& b) { for (int i = 0; i < 3; ++i) { lo[i] = std::min(lo[i], b.lo[i]); hi[i] = std::max(hi[i], b.hi[i]); } }
  float area() const {
    float d[3];
    for (int i = 0; i < 3; ++i) d[i] = std::max(0.0f, hi[i] - lo[i]);
    return 2.0f * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0]);
  }
};

// Binned surface-area-heuristic build (12 bins per axis, leaves of at most
// `leaf` primitives, 1..8).
struct Builder {
  const std::vector<Box>& boxes;
  std::vector<float> cen;            // [n*3]
  std::vector<int>& perm;
  HostBVH& out;
  static constexpr int BINS = 12;
  const int LEAF;
  Builder(const std::vector<Box>& b, HostBVH& o, int leaf) : boxes(b), perm(o.perm), out(o), LEAF(leaf) {
    size_t n = b.size();
    cen.resize(3 * n);
    perm.resize(n);
    for (size_t i = 0; i < n; ++i) {
      perm[i] = (int)i;
      for (int k = 0; k < 3; ++k) cen[3 * i + k] = 0.5f * (b[i].lo[k] + b[i].hi[k]);
    }
  }
  int new_node(int parent, int slot) {
    int id = (int)out.node_parent.size();
    out.node_parent.push_back(parent);
    out.node_slot.push_back(slot);
    for (int i = 0; i < 4; ++i) out.nodes.push_back(make_float4(0, 0, 0, 0));
    return id;
  }
  void set_child(int node, int slot, int code) {
    int* c = reinterpret_cast<int*>(&out.nodes[4 * node + 3]);
    c[slot] = code;
  }
  void empty_box(int node, int slot) {
    float* N = reinterpret_cast<float*>(&out.nodes[4 * node]);
    int o = slot ? 6 : 0;
    N[o] = N[o + 1] = N[o + 2] = 3e38f;
    N[o + 3] = N[o + 4] = N[o + 5] = -3e38f;
  }
  int make_leaf(int b, int e, int parent, int slot) {
    int id = (int)out.leaf_first.size();
    out.leaf_first.push_back(b);
    out.leaf_count.push_back(e - b);
    out.leaf_parent.push_back(parent);
    out.leaf_slot.push_back(slot);
    (void)id;
    return ~((b << 3) | (e - b - 1));
  }
  // returns the split position in perm (b < m < e)
  int split(int b, int e) {
    Box cb;
    cb.reset();
    for (int i = b; i < e; ++i) cb.grow(&cen[3 * perm[i]]);
    float best = 3e38f;
    int best_axis = -1, best_bin = -1;
    for (int ax = 0; ax < 3; ++ax) {
      float ext = cb.hi[ax] - cb.lo[ax];
      if (!(ext > 0)) continue;
      Box bb[BINS];
      int cnt[BINS] = {0};
      for (int k = 0; k < BINS; ++k) bb[k].reset();
      for (int i = b; i < e; ++i) {
        int k = std::min(BINS - 1, (int)((cen[3 * perm[i] + ax] - cb.lo[ax]) / ext * BINS));
        cnt[k]++;
        bb[k].grow(boxes[perm[i]]);
      }
      float la[BINS], ra[BINS];
      int lc[BINS], rc[BINS];
      Box acc;
      acc.reset();
      int c = 0;
      for (int k = 0; k < BINS; ++k) { acc.grow(bb[k]); c += cnt[k]; la[k] = acc.area(); lc[k] = c; }
      acc.reset();
      c = 0;
      for (int k = BINS - 1; k >= 0; --k) { acc.grow(bb[k]); c += cnt[k]; ra[k] = acc.area(); rc[k] = c; }
      for (int k = 0; k < BINS - 1; ++k) {
        if (lc[k] == 0 || rc[k + 1] == 0) continue;
        float cost = la[k] * lc[k] + ra[k + 1] * rc[k + 1];
        if (cost < best) { best = cost; best_axis = ax; best_bin = k; }
      }
    }
    int m = -1;
    if (best_axis >= 0) {
      float ext = cb.hi[best_axis] - cb.lo[best_axis];
      auto mid = std::partition(perm.begin() + b, perm.begin() + e, [&](int p) {
        int k = std::min(BINS - 1, (int)((cen[3 * p + best_axis] - cb.lo[best_axis]) / ext * BINS));
        return k <= best_bin;
      });
      m = (int)(mid - perm.begin());
    }
    if (m <= b || m >= e) {   // degenerate: median split along the largest extent
      int ax = 0;
      for (int k = 1; k < 3; ++k) if (cb.hi[k] - cb.lo[k] > cb.hi[ax] - cb.lo[ax]) ax = k;
      m = (b + e) / 2;
      std::nth_element(perm.begin() + b, perm.begin() + m, perm.begin() + e,
                       [&](int p, int q) { return cen[3 * p + ax] < cen[3 * q + ax]; });
    }
    return m;
  }
  // Build the subtree over perm[b, e) hanging below (parent, slot).
  int build(int b, int e, int parent, int slot) {
    if (e - b <= LEAF) return make_leaf(b, e, parent, slot);
    int m = split(b, e);
    int id = new_node(parent, slot);
    int c0 = build(b, m, id, 0);
    set_child(id, 0, c0);
    int c1 = build(m, e, id, 1);
    set_child(id, 1, c1);
    return id;
  }
  void run() {
    int n = (int)boxes.size();
    int root = new_node(-1, 0);
    if (n <= LEAF) {
      set_child(root, 0, make_leaf(0, n, root, 0));
      set_child(root, 1, EMPTY_CHILD);
      empty_box(root, 1);
      return;
    }
    int m = split(0, n);
    set_child(root, 0, build(0, m, root, 0));
    set_child(root, 1, build(m, n, root, 1));
  }
};

}  // namespace

namespace fr {

int fail(fr_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

}  // namespace fr

namespace {

template <class T> cudaError_t upload(DBuf<T>& b, const T* h, size_t n, cudaStream_t s) {
  cudaError_t e = b.alloc(n);
  if (e != cudaSuccess || n == 0) return e;
  e = cudaMemcpyAsync(b.p, h, n * sizeof(T), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

// Unit directions of the light stage (Face Modeling paragraph: lights on an
// isotropically sampled hemisphere, the camera side z >= 0).
//   layout 0: Fibonacci points, z_k = (k + 1/2)/n, azimuth k pi (3 - sqrt 5);
//   layout 1 (n = 20): the 42 vertices of a once-subdivided icosahedron
//     (vertices (0, +-1, +-phi) and cyclic, plus the normalised edge
//     midpoints), turned about x so that the axis (0, 1, phi^2) becomes +z;
//     the 20 strictly above z = 0, by height (descending) then azimuth
//     (components below 1e-12 set to zero first).
std::vector<std::array<double, 3>> light_dirs(int n, int layout) {
  std::vector<std::array<double, 3>> d;
  if (layout == 0) {
    const double ga = 3.14159265358979323846 * (3.0 - std::sqrt(5.0));
    for (int k = 0; k < n; ++k) {
      double z = (k + 0.5) / n, r = std::sqrt(1.0 - z * z), ph = k * ga;
      d.push_back({r * std::cos(ph), r * std::sin(ph), z});
    }
    return d;
  }
  const double phi = 0.5 * (1.0 + std::sqrt(5.0));
  std::vector<std::array<double, 3>> v;
  for (int a = -1; a <= 1; a += 2)
    for (int b = -1; b <= 1; b += 2) {
      v.push_back({0.0, (double)a, b * phi});
      v.push_back({(double)a, b * phi, 0.0});
      v.push_back({b * phi, 0.0, (double)a});
    }
  const double edge2 = 4.0;                  // squared edge length of this icosahedron
  std::vector<std::array<double, 3>> all;
  auto unit = [](std::array<double, 3> p) {
    double l = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    return std::array<double, 3>{p[0] / l, p[1] / l, p[2] / l};
  };
  for (auto& p : v) all.push_back(unit(p));
  for (size_t i = 0; i < v.size(); ++i)
    for (size_t j = i + 1; j < v.size(); ++j) {
      double dx = v[i][0] - v[j][0], dy = v[i][1] - v[j][1], dz = v[i][2] - v[j][2];
      if (std::fabs(dx * dx + dy * dy + dz * dz - edge2) < 1e-9)
        all.push_back(unit({v[i][0] + v[j][0], v[i][1] + v[j][1], v[i][2] + v[j][2]}));
    }
  const double th = std::atan2(1.0, phi * phi), ct = std::cos(th), st = std::sin(th);
  for (auto& p : all) {
    std::array<double, 3> q{p[0], p[1] * ct - p[2] * st, p[1] * st + p[2] * ct};
    for (double& x : q)
      if (std::fabs(x) < 1e-12) x = 0.0;        // exact zeros: symmetric directions sort alike
    if (q[2] > 1e-9) d.push_back(q);
  }
  std::sort(d.begin(), d.end(), [](const std::array<double, 3>& x, const std::array<double, 3>& y) {
    if (std::fabs(x[2] - y[2]) > 1e-9) return x[2] > y[2];
    return std::atan2(x[1], x[0]) < std::atan2(y[1], y[0]);
  });
  return d;
}

// Light stage: square quads of side light_side centred at radius * d_k,
// facing the origin; in-plane axes e1 = normalize(+y x d), e2 = d x e1.
std::vector<Light> make_lights(int n, double radius, int layout) {
  std::vector<std::array<double, 3>> D = light_dirs(n, layout);
  std::vector<Light> L(n);
  for (int k = 0; k < n && k < (int)D.size(); ++k) {
    const double* d = D[k].data();
    double e1[3] = {d[2], 0.0, -d[0]};
    double n1 = std::sqrt(e1[0] * e1[0] + e1[2] * e1[2]);
    e1[0] /= n1; e1[2] /= n1;
    double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2], d[0] * e1[1] - d[1] * e1[0]};
    L[k].c = V3{(float)(radius * d[0]), (float)(radius * d[1]), (float)(radius * d[2])};
    L[k].e1 = V3{(float)e1[0], (float)e1[1], (float)e1[2]};
    L[k].e2 = V3{(float)e2[0], (float)e2[1], (float)e2[2]};
    L[k].dl = V3{(float)d[0], (float)d[1], (float)d[2]};
  }
  return L;
}

// Collapse a binary hierarchy to 4 children per node: the children of a
// 4-wide node are the grandchildren of its binary node through internal
// children, and the leaf children themselves.  codes4[k] holds the child
// codes (leaf code, 4-wide node index, or EMPTY_CHILD); src4[4k + c] the
// binary (node, slot) whose box and cone child c takes, (-1, -1) if empty.
// A box that fails a conservative test also fails for everything below it,
// so the 4-wide search visits the same leaves as the binary one.
void collapse4(const HostBVH& h, std::vector<int4>& codes4, std::vector<int2>& src4) {
  const int nb = (int)(h.nodes.size() / 4);
  auto code = [&](int n, int s) { return reinterpret_cast<const int*>(&h.nodes[4 * n + 3])[s]; };
  std::vector<int> to4(nb, -1), order{0};
  to4[0] = 0;
  codes4.assign(1, make_int4(EMPTY_CHILD, EMPTY_CHILD, EMPTY_CHILD, EMPTY_CHILD));
  src4.assign(4, make_int2(-1, -1));
  for (size_t q = 0; q < order.size(); ++q) {
    const int n = order[q], k = to4[n];
    int cc[4] = {EMPTY_CHILD, EMPTY_CHILD, EMPTY_CHILD, EMPTY_CHILD};
    int2 ss[4] = {make_int2(-1, -1), make_int2(-1, -1), make_int2(-1, -1), make_int2(-1, -1)};
    int used = 0;
    auto add = [&](int c, int sn, int sl) {
      if (!leaf_child(c)) {
        to4[c] = (int)codes4.size();
        codes4.push_back(make_int4(EMPTY_CHILD, EMPTY_CHILD, EMPTY_CHILD, EMPTY_CHILD));
        src4.resize(src4.size() + 4, make_int2(-1, -1));
        order.push_back(c);
        c = to4[c];
      }
      cc[used] = c;
      ss[used] = make_int2(sn, sl);
      ++used;
    };
    for (int s = 0; s < 2; ++s) {
      int c = code(n, s);
      if (c == EMPTY_CHILD) continue;
      if (leaf_child(c)) { add(c, n, s); continue; }
      for (int s2 = 0; s2 < 2; ++s2) {
        int c2 = code(c, s2);
        if (c2 != EMPTY_CHILD) add(c2, c, s2);
      }
    }
    codes4[k] = make_int4(cc[0], cc[1], cc[2], cc[3]);
    for (int c = 0; c < 4; ++c) src4[4 * k + c] = ss[c];
  }
}

int upload_bvh(fr_ctx* ctx, const HostBVH& h, DevBVH& d) {
  d.n_nodes = (int)(h.nodes.size() / 4);
  d.n_leaves = (int)h.leaf_first.size();
  CK(upload(d.nodes, h.nodes.data(), h.nodes.size(), ctx->stream));
  CK(upload(d.leaf_first, h.leaf_first.data(), h.leaf_first.size(), ctx->stream));
  CK(upload(d.leaf_count, h.leaf_count.data(), h.leaf_count.size(), ctx->stream));
  CK(upload(d.leaf_parent, h.leaf_parent.data(), h.leaf_parent.size(), ctx->stream));
  CK(upload(d.leaf_slot, h.leaf_slot.data(), h.leaf_slot.size(), ctx->stream));
  CK(upload(d.node_parent, h.node_parent.data(), h.node_parent.size(), ctx->stream));
  CK(upload(d.node_slot, h.node_slot.data(), h.node_slot.size(), ctx->stream));
  CK(d.counter.alloc(d.n_nodes));
  {
    std::vector<float4> full(2 * (size_t)d.n_nodes, make_float4(0, 0, 1, CONE_FULL));
    CK(upload(d.cones, full.data(), full.size(), ctx->stream));
  }
  return FR_OK;
}

}  // namespace

namespace fr {

FrameView main_view(fr_ctx* c) {
  FrameView v;
  v.X = c->X.p; v.Xm = c->Xm.p; v.alb = c->alb.p; v.nrm = c->nrm.p; v.ng = c->ng.p; v.tv = c->tv.p;
  v.epack = c->epack.p;
  v.tnodes = c->tbvh.nodes.p; v.tcones = c->tbvh.cones.p; v.tcounter = c->tbvh.counter.p;
  v.enodes = c->ebvh.nodes.p; v.econes = c->ebvh.cones.p; v.ecounter = c->ebvh.counter.p;
  v.e4boxes = c->e4boxes.p; v.e4cones = c->e4cones.p;
  v.sil = c->sil.p; v.n_sil = c->n_sil.p; v.block_count = c->block_count.p;
  v.dX = c->dX.p; v.dN = c->dN.p; v.dA = c->dA.p; v.gs = c->gs.p;
  v.dXm = c->dXm.p; v.dC = c->dC.p; v.dL = c->dL.p;
  return v;
}

GeoArgs geo_args(fr_ctx* c, const FrameView& v) {
  GeoArgs g;
  g.V = c->V; g.F = c->F; g.K_id = c->K_id; g.K_exp = c->K_exp; g.K_alb = c->K_alb; g.off_pose = c->off_pose();
  g.mean = c->mean.p; g.BidT = c->BidT.p; g.BexpT = c->BexpT.p; g.alb_mean = c->alb_mean.p; g.BalbT = c->BalbT.p;
  g.tris = c->tris.p; g.tri_perm = c->tri_perm.p; g.vf_off = c->vf_off.p; g.vf_idx = c->vf_idx.p;
  g.X = v.X; g.Xm = v.Xm; g.alb = v.alb; g.nrm = v.nrm; g.ng = v.ng; g.tv = v.tv;
  return g;
}

Cam make_cam(const fr_ctx* c, int W, int H) {
  Cam cam;
  cam.o = V3{0.0f, 0.0f, c->cfg.d_cam};
  cam.k = (float)(2.0 * (double)c->cfg.tan_half_fov / (double)H);
  cam.cx = (float)((double)c->cfg.tan_half_fov * (double)W / (double)H);
  cam.cy = c->cfg.tan_half_fov;
  cam.dcam = c->cfg.d_cam;
  return cam;
}

// Bottom-up refit of one BVH's boxes (topology b, boxes in nodes / cones).
static int refit(fr_ctx* ctx, const DevBVH& b, float4* nodes, float4* cones, int* counter, bool is_edge,
                 const FrameView& v) {
  if (b.n_leaves == 0) return FR_OK;
  CK(cudaMemsetAsync(counter, 0, sizeof(int) * b.n_nodes, ctx->stream));
  RefitArgs r;
  r.n_leaves = b.n_leaves;
  r.leaf_first = b.leaf_first.p; r.leaf_count = b.leaf_count.p; r.leaf_parent = b.leaf_parent.p;
  r.leaf_slot = b.leaf_slot.p; r.node_parent = b.node_parent.p; r.node_slot = b.node_slot.p;
  r.counter = counter; r.nodes = nodes; r.is_edge = is_edge ? 1 : 0;
  r.tv = v.tv; r.edges = ctx->edges_leaf.p; r.X = v.X;
  r.pack = v.epack; r.cones = cones;
  k_refit<<<(b.n_leaves + 255) / 256, 256, 0, ctx->stream>>>(r);
  CKL();
  return FR_OK;
}

// Geometry, normals, packed edges and refits for theta.
int prepare_geometry(fr_ctx* ctx, const float* theta, const FrameView& v) {
  if (!ctx->have_mesh || !ctx->have_bases) return fail(ctx, FR_ERR_NOT_READY, "mesh and bases must be uploaded first");
  if (!theta) return fail(ctx, FR_ERR_INVALID_ARG, "theta is null");
  GeoArgs g = geo_args(ctx, v);
  cudaStream_t s = ctx->stream;
  k_geometry<<<(ctx->V + GEO_VERTS - 1) / GEO_VERTS, GEO_THREADS, 0, s>>>(g, theta);
  CKL();
  k_faces<<<(ctx->F + 255) / 256, 256, 0, s>>>(g);
  CKL();
  k_vertex_normals<<<(ctx->V + 255) / 256, 256, 0, s>>>(g);
  CKL();
  k_pack_edges<<<(ctx->E + 255) / 256, 256, 0, s>>>(ctx->E, ctx->edges_leaf.p, ctx->edge_id_leaf.p, ctx->tris.p,
                                                     v.X, v.ng, v.epack);
  CKL();
  int rc = refit(ctx, ctx->tbvh, v.tnodes, v.tcones, v.tcounter, false, v);
  if (rc) return rc;
  rc = refit(ctx, ctx->ebvh, v.enodes, v.econes, v.ecounter, true, v);
  if (rc) return rc;
  if (ctx->n4 > 0) {
    k_gather4<<<(4 * ctx->n4 + 255) / 256, 256, 0, s>>>(4 * ctx->n4, ctx->e4src.p, v.enodes, v.econes, v.e4boxes,
                                                          v.e4cones);
    CKL();
  }
  return FR_OK;
}

// Order-preserving list of camera-silhouette edges; block_count is the
// compaction's scratch (one int per 256 edges).
int silhouettes(fr_ctx* ctx, const FrameView& v) {
  cudaStream_t s = ctx->stream;
  SilArgs sa;
  sa.E = ctx->E; sa.edges = ctx->edges_canon.p; sa.tris = ctx->tris.p; sa.ng = v.ng; sa.X = v.X;
  sa.cam_o = V3{0.0f, 0.0f, ctx->cfg.d_cam};
  sa.block_count = v.block_count; sa.sil = v.sil; sa.n_sil = v.n_sil;
  int nb = (ctx->E + 255) / 256;
  k_silhouette_flags<<<nb, 256, 0, s>>>(sa);
  CKL();
  k_silhouette_scan<<<1, 1024, 0, s>>>(sa, nb);
  CKL();
  k_silhouette_scatter<<<nb, 256, 0, s>>>(sa);
  CKL();
  return FR_OK;
}

RenderArgs render_args(fr_ctx* c, const float* theta, const fr_render_opts* o, const FrameView& v) {
  RenderArgs a;
  a.W = o->W; a.H = o->H; a.spp = o->spp; a.seed = o->seed; a.iter = o->iter;
  a.n_lights = c->cfg.n_lights;
  a.side = c->cfg.light_side; a.eps_pedge = c->cfg.eps_pedge;
  a.brdf = Brdf{c->cfg.beckmann_m, c->cfg.brdf_model, c->cfg.fresnel};
  a.eps_sedge = c->cfg.eps_sedge; a.tmin = c->cfg.shadow_tmin; a.kappa = c->cfg.clip_kappa;
  a.cam = make_cam(c, o->W, o->H);
  for (int j = 0; j < c->cfg.n_lights; ++j) a.lights[j] = c->lights[j];
  a.mesh.X = v.X; a.mesh.ng = v.ng; a.mesh.tris = c->tris.p; a.mesh.tv = v.tv;
  a.mesh.bvh.nodes = v.tnodes; a.mesh.bvh.n_nodes = c->tbvh.n_nodes;
  a.mesh.max_steps = c->max_steps;
  a.ebvh.bvh.nodes = v.enodes; a.ebvh.bvh.n_nodes = c->ebvh.n_nodes;
  a.ebvh.edges = c->edges_leaf.p; a.ebvh.edge_id = c->edge_id_leaf.p;
  a.ebvh.pack = v.epack; a.ebvh.verts = c->edges_leaf.p; a.ebvh.cones = v.econes;
  a.ebvh.codes4 = c->e4codes.p; a.ebvh.boxes4 = v.e4boxes; a.ebvh.cones4 = v.e4cones;
  a.nrm = v.nrm; a.alb = v.alb; a.uv = reinterpret_cast<const float2*>(c->uv.p);
  a.cspec = theta + c->off_cspec(); a.lights_dev = theta + c->off_lights();
  a.sil = v.sil; a.n_sil = v.n_sil; a.edges_canon = c->edges_canon.p;
  a.err = c->err_flag.p;
  a.aov_scratch = nullptr;
  a.counters = c->counters_on ? c->counters.p : nullptr;
  return a;
}

int adjoint(fr_ctx* ctx, const float* theta, const FrameView& v, double* grad, bool with_alb) {
  cudaStream_t s = ctx->stream;
  const int V = ctx->V;
  GeoArgs g = geo_args(ctx, v);
  k_normals_bwd_vertex<<<(V + 255) / 256, 256, 0, s>>>(g, v.dN, v.gs);
  CKL();
  k_normals_bwd_gather<<<(V + 255) / 256, 256, 0, s>>>(g, v.gs, v.dX);
  CKL();
  k_pose_bwd<<<152, 256, 0, s>>>(g, theta, v.dX, v.dXm, grad);
  CKL();
  const int n3 = 3 * V;
  if (ctx->K_id) {
    k_basis_T<<<dim3(ctx->K_id, BASIS_SLICES), 256, 0, s>>>(ctx->BidT.p, ctx->K_id, n3, v.dXm, nullptr, grad, 0);
    CKL();
  }
  if (ctx->K_exp) {
    k_basis_T<<<dim3(ctx->K_exp, BASIS_SLICES), 256, 0, s>>>(ctx->BexpT.p, ctx->K_exp, n3, v.dXm, nullptr, grad,
                                                            ctx->K_id);
    CKL();
  }
  if (ctx->K_alb && with_alb) {
    k_basis_T<<<dim3(ctx->K_alb, BASIS_SLICES), 256, 0, s>>>(ctx->BalbT.p, ctx->K_alb, n3, nullptr, v.dA, grad,
                                                            ctx->K_id + ctx->K_exp);
    CKL();
  }
  if (v.dC) {
    k_add_small<<<(CS * CS + 255) / 256, 256, 0, s>>>(v.dC, CS * CS, grad, ctx->off_cspec());
    CKL();
  }
  k_add_small<<<1, 128, 0, s>>>(v.dL, 3 * ctx->cfg.n_lights, grad, ctx->off_lights());
  CKL();
  return FR_OK;
}

}  // namespace fr

namespace {

// Geometry, normals, refits and camera silhouettes for theta (context buffers).
int prepare(fr_ctx* ctx, const float* theta, int W, int H) {
  ctx->mark(PH_GEOMETRY, 0);
  FrameView v = main_view(ctx);
  int rc = prepare_geometry(ctx, theta, v);
  if (rc) return rc;
  (void)W; (void)H;
  rc = silhouettes(ctx, v);
  ctx->mark(PH_GEOMETRY, 1);
  return rc;
}

// Copy the geometry outputs of the last prepare and return the silhouette count.
int geometry_outputs(fr_ctx* ctx, float* X, float* N, float* A) {
  const int V = ctx->V;
  cudaStream_t s = ctx->stream;
  if (X) CK(cudaMemcpy2DAsync(X, 3 * sizeof(float), ctx->X.p, sizeof(float4), 3 * sizeof(float), V, cudaMemcpyDeviceToDevice, s));
  if (N) CK(cudaMemcpy2DAsync(N, 3 * sizeof(float), ctx->nrm.p, sizeof(float4), 3 * sizeof(float), V, cudaMemcpyDeviceToDevice, s));
  if (A) CK(cudaMemcpy2DAsync(A, 3 * sizeof(float), ctx->alb.p, sizeof(float4), 3 * sizeof(float), V, cudaMemcpyDeviceToDevice, s));
  int nsil = 0;
  CK(cudaMemcpyAsync(&nsil, ctx->n_sil.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return nsil;
}

int check_opts(fr_ctx* ctx, const fr_render_opts* o) {
  if (!o) return fail(ctx, FR_ERR_INVALID_ARG, "opts is null");
  if (o->W < 1 || o->H < 1 || o->spp < 1) return fail(ctx, FR_ERR_INVALID_ARG, "W, H, spp must be >= 1");
  if ((long long)o->W * o->H > (1LL << 26) || (long long)o->W * o->H * o->spp > (1LL << 31) - 1)
    return fail(ctx, FR_ERR_INVALID_ARG, "image or sample count too large");
  return FR_OK;
}

// The backward after its interior pass: primary-visibility and shadow edge
// passes, then the normal/geometry adjoint added into grad.
int edges_and_adjoint(fr_ctx* ctx, const float* theta, const fr_render_opts* opts, const RenderArgs& a,
                      const GradBufs& gb, int terms, double* grad) {
  cudaStream_t s = ctx->stream;
  long long tiled = (long long)(((opts->W + 7) / 8) * ((opts->H + 7) / 8)) * 64 * opts->spp;
  if (terms & TERM_PEDGE) {
    ctx->mark(PH_PEDGE, 0);
    k_bwd_pedge<<<grid_for((long long)opts->W * opts->H * opts->spp, 256), 256, 0, s>>>(a, gb);
    CKL();
    ctx->mark(PH_PEDGE, 1);
  }
  if (terms & TERM_SEDGE) {
    dim3 grid(grid_for(tiled, 256), ctx->cfg.n_lights);
    ctx->mark(PH_SEDGE, 0);
    const size_t n_picks = (size_t)tiled * ctx->cfg.n_lights;
    if (ctx->picks.n < n_picks) CK(ctx->picks.alloc(n_picks));
    // the search takes one or two samples per thread, by the image's size
    if ((long long)opts->W * opts->H >= SEDGE_NS2_MIN_PIXELS)
      k_bwd_sedge<<<dim3(grid_for(tiled, 512), ctx->cfg.n_lights), 256, 0, s>>>(a, gb, ctx->picks.p);
    else
      k_bwd_sedge_1<<<dim3(grid_for(tiled, 256), ctx->cfg.n_lights), 256, 0, s>>>(a, gb, ctx->picks.p);
    CKL();
    ctx->mark(PH_SEDGE, 1);
    ctx->mark(PH_SEDGE_ADD, 0);
    k_bwd_sedge_add<<<grid, 256, 0, s>>>(a, gb, ctx->picks.p);
    CKL();
    ctx->mark(PH_SEDGE_ADD, 1);
  }
  ctx->mark(PH_ADJOINT, 0);
  int rc = adjoint(ctx, theta, main_view(ctx), grad, true);
  if (rc) return rc;
  ctx->mark(PH_ADJOINT, 1);
  return FR_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

void fr_default_config(fr_config* c) {
  if (!c) return;
  c->tan_half_fov = 0.275f; c->d_cam = 4.0f; c->light_radius = 3.0f; c->light_side = 0.6f; c->beckmann_m = 0.3f;
  c->eps_pedge = 1e-3f; c->eps_sedge = 2e-4f; c->shadow_tmin = 1e-4f; c->clip_kappa = 1e-5f; c->n_lights = 20;
  c->brdf_model = 0; c->fresnel = 0; c->light_layout = 0; c->light_prior = 0;
}

const char* fr_strerror(int32_t code) {
  switch (code) {
    case FR_OK: return "ok";
    case FR_ERR_INVALID_ARG: return "invalid argument";
    case FR_ERR_SHAPE: return "inconsistent shapes";
    case FR_ERR_CUDA: return "CUDA error";
    case FR_ERR_OOM: return "out of device memory";
    case FR_ERR_DEVICE_LIMIT: return "device traversal limit reached";
    case FR_ERR_NOT_READY: return "mesh or bases not uploaded";
    default: return "unknown error";
  }
}

const char* fr_last_error(const fr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int fr_create(fr_ctx** out, const fr_config* cfg, int32_t device) {
  fr_ctx* ctx = nullptr;
  if (!out) return FR_ERR_INVALID_ARG;
  *out = nullptr;
  fr_config c;
  if (cfg) c = *cfg; else fr_default_config(&c);
  if (c.n_lights < 1 || c.n_lights > MAX_LIGHTS) return FR_ERR_INVALID_ARG;
  if (!(c.light_side > 0) || !(c.d_cam > 0) || !(c.tan_half_fov > 0) || !(c.beckmann_m > 0)) return FR_ERR_INVALID_ARG;
  if (c.brdf_model < 0 || c.brdf_model > 1 || c.fresnel < 0 || c.fresnel > 1 || c.light_layout < 0 ||
      c.light_layout > 1 || (c.light_layout == 1 && c.n_lights != 20) || c.light_prior < 0 || c.light_prior > 2)
    return FR_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FR_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return FR_ERR_CUDA;
  ctx = new fr_ctx();
  ctx->device = device;
  ctx->cfg = c;
  ctx->lights = make_lights(c.n_lights, c.light_radius, c.light_layout);
  if (ctx->err_flag.alloc(1) != cudaSuccess || ctx->counters.alloc(NCOUNT) != cudaSuccess ||
      ctx->n_sil.alloc(1) != cudaSuccess) {
    delete ctx;
    return FR_ERR_OOM;
  }
  cudaMemset(ctx->err_flag.p, 0, sizeof(int));
  cudaMemset(ctx->counters.p, 0, NCOUNT * sizeof(unsigned long long));
  cudaMemset(ctx->n_sil.p, 0, sizeof(int));
  if (cudaDeviceSynchronize() != cudaSuccess) { delete ctx; return FR_ERR_CUDA; }
  *out = ctx;
  return FR_OK;
}

void fr_destroy(fr_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  ctx->mean.free_(); ctx->uv.free_(); ctx->tris.free_(); ctx->edges_canon.free_(); ctx->edges_leaf.free_();
  ctx->vf_off.free_(); ctx->vf_idx.free_(); ctx->tri_perm.free_(); ctx->edge_id_leaf.free_();
  for (DevBVH* b : {&ctx->tbvh, &ctx->ebvh}) {
    b->nodes.free_(); b->cones.free_(); b->leaf_first.free_(); b->leaf_count.free_(); b->leaf_parent.free_(); b->leaf_slot.free_();
    b->node_parent.free_(); b->node_slot.free_(); b->counter.free_();
  }
  ctx->BidT.free_(); ctx->BexpT.free_(); ctx->alb_mean.free_(); ctx->BalbT.free_();
  ctx->X.free_(); ctx->Xm.free_(); ctx->alb.free_(); ctx->nrm.free_(); ctx->ng.free_(); ctx->tv.free_();
  ctx->epack.free_();
  ctx->e4codes.free_(); ctx->e4src.free_(); ctx->e4boxes.free_(); ctx->e4cones.free_();
  ctx->sil.free_(); ctx->n_sil.free_(); ctx->block_count.free_(); ctx->err_flag.free_(); ctx->counters.free_();
  ctx->dX.free_(); ctx->dN.free_(); ctx->dA.free_(); ctx->gs.free_(); ctx->dXm.free_(); ctx->dC.free_(); ctx->dL.free_();
  ctx->hits.free_(); ctx->picks.free_(); ctx->aov_scratch.free_(); ctx->dimg.free_();
  ctx->mlp_w.free_(); ctx->mlp_m.free_(); ctx->mlp_v.free_(); ctx->mlp_g.free_(); ctx->mlp_scratch.free_();
  if (ctx->events_made)
    for (int i = 0; i < NPHASE; ++i) { cudaEventDestroy(ctx->ev[i][0]); cudaEventDestroy(ctx->ev[i][1]); }
  delete ctx;
}

int fr_set_stream(fr_ctx* ctx, void* stream) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return FR_OK;
}

int fr_upload_mesh(fr_ctx* ctx, const float* mean, int32_t V, const int32_t* tris, int32_t F, const float* uv) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (!mean || !tris || !uv || V < 3 || F < 1) return fail(ctx, FR_ERR_INVALID_ARG, "mesh arrays null or too small");
  if (F > (1 << 27) || V > (1 << 27)) return fail(ctx, FR_ERR_INVALID_ARG, "mesh too large");
  CK(cudaSetDevice(ctx->device));
  for (int i = 0; i < 3 * F; ++i)
    if (tris[i] < 0 || tris[i] >= V) return fail(ctx, FR_ERR_SHAPE, "triangle index %d out of range", tris[i]);
  // canonical edges: sorted by (min vertex, max vertex); f0 < f1, f1 = -1 on the boundary
  std::vector<std::array<int, 3>> he;
  he.reserve(3 * (size_t)F);
  for (int f = 0; f < F; ++f)
    for (int k = 0; k < 3; ++k) {
      int a = tris[3 * f + k], b = tris[3 * f + (k + 1) % 3];
      if (a == b) return fail(ctx, FR_ERR_SHAPE, "degenerate triangle %d", f);
      he.push_back({std::min(a, b), std::max(a, b), f});
    }
  std::sort(he.begin(), he.end());
  std::vector<int4> edges;
  for (size_t i = 0; i < he.size();) {
    size_t j = i;
    while (j < he.size() && he[j][0] == he[i][0] && he[j][1] == he[i][1]) ++j;
    if (j - i > 2) return fail(ctx, FR_ERR_SHAPE, "edge (%d,%d) shared by %d triangles", he[i][0], he[i][1], (int)(j - i));
    edges.push_back(make_int4(he[i][0], he[i][1], he[i][2], j - i == 2 ? he[i + 1][2] : -1));
    i = j;
  }
  const int E = (int)edges.size();
  // vertex -> face CSR
  std::vector<int> vf_off(V + 1, 0), vf_idx(3 * (size_t)F);
  for (int i = 0; i < 3 * F; ++i) vf_off[tris[i] + 1]++;
  for (int v = 0; v < V; ++v) vf_off[v + 1] += vf_off[v];
  {
    std::vector<int> pos(vf_off.begin(), vf_off.end() - 1);
    for (int f = 0; f < F; ++f)
      for (int k = 0; k < 3; ++k) vf_idx[pos[tris[3 * f + k]]++] = f;
  }
  // BVHs over the mean shape
  std::vector<Box> tb(F), eb(E);
  for (int f = 0; f < F; ++f) {
    tb[f].reset();
    for (int k = 0; k < 3; ++k) tb[f].grow(&mean[3 * tris[3 * f + k]]);
  }
  for (int e = 0; e < E; ++e) {
    eb[e].reset();
    eb[e].grow(&mean[3 * edges[e].x]);
    eb[e].grow(&mean[3 * edges[e].y]);
  }
  HostBVH ht, he2;
  { Builder b(tb, ht, TRI_LEAF); b.run(); }
  { Builder b(eb, he2, EDGE_LEAF); b.run(); }
  std::vector<int4> tris4(F), edges_leaf(E);
  for (int f = 0; f < F; ++f) tris4[f] = make_int4(tris[3 * f], tris[3 * f + 1], tris[3 * f + 2], 0);
  for (int i = 0; i < E; ++i) edges_leaf[i] = edges[he2.perm[i]];
  cudaStream_t s = ctx->stream;
  CK(upload(ctx->mean, mean, 3 * (size_t)V, s));
  CK(upload(ctx->uv, uv, 2 * (size_t)V, s));
  CK(upload(ctx->tris, tris4.data(), F, s));
  CK(upload(ctx->edges_canon, edges.data(), E, s));
  CK(upload(ctx->edges_leaf, edges_leaf.data(), E, s));
  CK(upload(ctx->edge_id_leaf, he2.perm.data(), E, s));
  CK(upload(ctx->tri_perm, ht.perm.data(), F, s));
  CK(upload(ctx->vf_off, vf_off.data(), V + 1, s));
  CK(upload(ctx->vf_idx, vf_idx.data(), 3 * (size_t)F, s));
  int rc = upload_bvh(ctx, ht, ctx->tbvh);
  if (rc) return rc;
  rc = upload_bvh(ctx, he2, ctx->ebvh);
  if (rc) return rc;
  {
    std::vector<int4> codes4;
    std::vector<int2> src4;
    collapse4(he2, codes4, src4);
    ctx->n4 = (int)codes4.size();
    CK(upload(ctx->e4codes, codes4.data(), codes4.size(), s));
    CK(upload(ctx->e4src, src4.data(), src4.size(), s));
    CK(ctx->e4boxes.alloc(12 * codes4.size()));
    CK(ctx->e4cones.alloc(8 * codes4.size()));
  }
  ctx->V = V; ctx->F = F; ctx->E = E;
  ++ctx->generation;
  CK(ctx->X.alloc(V)); CK(ctx->Xm.alloc(V)); CK(ctx->alb.alloc(V)); CK(ctx->nrm.alloc(V));
  CK(ctx->ng.alloc(F)); CK(ctx->tv.alloc(3 * (size_t)F)); CK(ctx->epack.alloc(6 * (size_t)E));
  CK(ctx->sil.alloc(E)); CK(ctx->block_count.alloc((E + 255) / 256));
  CK(ctx->dX.alloc(V)); CK(ctx->dN.alloc(V)); CK(ctx->dA.alloc(V)); CK(ctx->gs.alloc(V));
  CK(ctx->dXm.alloc(3 * (size_t)V)); CK(ctx->dC.alloc(CS * CS)); CK(ctx->dL.alloc(3 * MAX_LIGHTS));
  ctx->have_mesh = true;
  ctx->have_bases = false;
  return FR_OK;
}

int fr_upload_bases(fr_ctx* ctx, const float* B_id, int32_t K_id, const float* B_exp, int32_t K_exp,
                    const float* alb_mean, const float* B_alb, int32_t K_alb) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (!ctx->have_mesh) return fail(ctx, FR_ERR_NOT_READY, "upload the mesh first");
  if (K_id < 0 || K_exp < 0 || K_alb < 0 || K_id + K_exp + K_alb > 512)
    return fail(ctx, FR_ERR_INVALID_ARG, "basis sizes must be >= 0 with K_id + K_exp + K_alb <= 512");
  if (!alb_mean || (K_id && !B_id) || (K_exp && !B_exp) || (K_alb && !B_alb))
    return fail(ctx, FR_ERR_INVALID_ARG, "basis pointer is null");
  CK(cudaSetDevice(ctx->device));
  const size_t n3 = 3 * (size_t)ctx->V;
  auto transpose = [&](const float* B, int K) {
    std::vector<float> T((size_t)K * n3);
    for (size_t i = 0; i < n3; ++i)
      for (int k = 0; k < K; ++k) T[(size_t)k * n3 + i] = B[i * K + k];
    return T;
  };
  std::vector<float> t;
  t = transpose(B_id, K_id);
  CK(upload(ctx->BidT, t.data(), t.size(), ctx->stream));
  t = transpose(B_exp, K_exp);
  CK(upload(ctx->BexpT, t.data(), t.size(), ctx->stream));
  t = transpose(B_alb, K_alb);
  CK(upload(ctx->BalbT, t.data(), t.size(), ctx->stream));
  CK(upload(ctx->alb_mean, alb_mean, n3, ctx->stream));
  ctx->K_id = K_id; ctx->K_exp = K_exp; ctx->K_alb = K_alb;
  ctx->have_bases = true;
  ++ctx->generation;
  return FR_OK;
}

int32_t fr_n_params(const fr_ctx* ctx) { return ctx ? ctx->n_params() : FR_ERR_INVALID_ARG; }

int fr_render(fr_ctx* ctx, const float* theta, const fr_render_opts* opts, float* image, float* aov) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  int rc = check_opts(ctx, opts);
  if (rc) return rc;
  if (!image) return fail(ctx, FR_ERR_INVALID_ARG, "image is null");
  CK(cudaSetDevice(ctx->device));
  rc = prepare(ctx, theta, opts->W, opts->H);
  if (rc) return rc;
  RenderArgs a = render_args(ctx, theta, opts, main_view(ctx));
  if (ctx->counters_on)
    CK(cudaMemsetAsync(ctx->counters.p + CNT_FWD, 0, CNT_PER_KERNEL * sizeof(unsigned long long), ctx->stream));
  bool shuffle = opts->spp <= 32 && (32 % opts->spp) == 0;
  const size_t npix = (size_t)opts->W * opts->H;
  if (!shuffle) CK(cudaMemsetAsync(image, 0, sizeof(float) * 3 * npix, ctx->stream));
  if (aov && !shuffle) {
    if (ctx->aov_scratch.n < npix) CK(ctx->aov_scratch.alloc(npix));
    CK(cudaMemsetAsync(aov, 0, sizeof(float) * 14 * npix, ctx->stream));
    CK(cudaMemsetAsync(ctx->aov_scratch.p, 0, sizeof(float) * npix, ctx->stream));
    a.aov_scratch = ctx->aov_scratch.p;
  }
  long long threads = (long long)(((opts->W + 7) / 8) * ((opts->H + 7) / 8)) * 64 * opts->spp;
  ctx->mark(PH_FORWARD, 0);
  if (aov) k_render_fwd_aov<<<grid_for(threads, 256), 256, 0, ctx->stream>>>(a, image, aov);
  else k_render_fwd<<<grid_for(threads, 256), 256, 0, ctx->stream>>>(a, image);
  CKL();
  if (aov && !shuffle) {
    k_aov_finish<<<grid_for((long long)npix, 256), 256, 0, ctx->stream>>>((int)npix, aov, ctx->aov_scratch.p);
    CKL();
  }
  ctx->mark(PH_FORWARD, 1);
  return FR_OK;
}

int fr_render_backward(fr_ctx* ctx, const float* theta, const fr_render_opts* opts, const float* d_image,
                       double* grad, int32_t accumulate) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  int rc = check_opts(ctx, opts);
  if (rc) return rc;
  if (!d_image || !grad) return fail(ctx, FR_ERR_INVALID_ARG, "d_image or grad is null");
  CK(cudaSetDevice(ctx->device));
  rc = prepare(ctx, theta, opts->W, opts->H);
  if (rc) return rc;
  cudaStream_t s = ctx->stream;
  const int V = ctx->V;
  if (!accumulate) CK(cudaMemsetAsync(grad, 0, sizeof(double) * ctx->n_params(), s));
  CK(cudaMemsetAsync(ctx->dX.p, 0, sizeof(float4) * V, s));
  CK(cudaMemsetAsync(ctx->dN.p, 0, sizeof(float4) * V, s));
  CK(cudaMemsetAsync(ctx->dA.p, 0, sizeof(float4) * V, s));
  CK(cudaMemsetAsync(ctx->dC.p, 0, sizeof(float) * CS * CS, s));
  CK(cudaMemsetAsync(ctx->dL.p, 0, sizeof(float) * 3 * MAX_LIGHTS, s));
  if (ctx->counters_on)
    CK(cudaMemsetAsync(ctx->counters.p + CNT_INTERIOR, 0, (CNT_TOTAL - CNT_INTERIOR) * sizeof(unsigned long long), s));
  RenderArgs a = render_args(ctx, theta, opts, main_view(ctx));
  const int terms = opts->terms ? opts->terms : (TERM_INTERIOR | TERM_PEDGE | TERM_SEDGE);
  long long tiled = (long long)(((opts->W + 7) / 8) * ((opts->H + 7) / 8)) * 64 * opts->spp;
  if ((terms & TERM_SEDGE) && ctx->hits.n < (size_t)tiled) CK(ctx->hits.alloc(tiled));
  GradBufs gb;
  gb.dX = ctx->dX.p; gb.dN = ctx->dN.p; gb.dA = ctx->dA.p; gb.dC = ctx->dC.p; gb.dL = ctx->dL.p;
  gb.d_image = d_image;
  gb.hits = (terms & TERM_SEDGE) ? ctx->hits.p : nullptr;
  // The interior pass finds each sample's primary hit; the shadow-edge pass reuses it.
  if (terms & (TERM_INTERIOR | TERM_SEDGE)) {
    RenderArgs ai = a;
    if (!(terms & TERM_INTERIOR)) { ai.n_lights = 0; }   // hits only
    ctx->mark(PH_INTERIOR, 0);
    k_bwd_interior<<<grid_for(tiled, 256), 256, 0, s>>>(ai, gb);
    CKL();
    ctx->mark(PH_INTERIOR, 1);
  }
  return edges_and_adjoint(ctx, theta, opts, a, gb, terms, grad);
}

int fr_loss(fr_ctx* ctx, const float* theta, int32_t W, int32_t H, const float* image, const float* target,
            const uint8_t* mask, const float* m, float w1, float w2, double* loss, float* d_image, double* grad) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (!theta || !image || !target || !loss || W < 1 || H < 1)
    return fail(ctx, FR_ERR_INVALID_ARG, "loss: null pointer or bad size");
  if (!ctx->have_bases) return fail(ctx, FR_ERR_NOT_READY, "bases not uploaded");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  ctx->mark(PH_LOSS, 0);
  CK(cudaMemsetAsync(loss, 0, sizeof(double), s));
  int n = W * H;
  int blocks = std::min((n + 255) / 256, 4 * 152);
  k_loss_data<<<blocks, 256, 0, s>>>(n, image, target, mask, loss, d_image);
  CKL();
  k_loss_reg<<<1, 256, 0, s>>>(theta, ctx->K_id + ctx->K_exp + ctx->K_alb, ctx->off_lights(), 3 * ctx->cfg.n_lights,
                               ctx->cfg.light_prior, m, w1, w2, loss, grad);
  CKL();
  ctx->mark(PH_LOSS, 1);
  return FR_OK;
}

int fr_step(fr_ctx* ctx, const float* theta, const fr_render_opts* opts, const float* target, const uint8_t* mask,
            const float* m, float w1, float w2, float* image, float* d_image, double* loss, double* grad) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  int rc = check_opts(ctx, opts);
  if (rc) return rc;
  if (!theta || !target || !image || !loss || !grad)
    return fail(ctx, FR_ERR_INVALID_ARG, "step: theta, target, image, loss or grad is null");
  if (!ctx->have_bases) return fail(ctx, FR_ERR_NOT_READY, "bases not uploaded");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const size_t npix = (size_t)opts->W * opts->H;
  if (!d_image) {
    if (ctx->dimg.n < 3 * npix) CK(ctx->dimg.alloc(3 * npix));
    d_image = ctx->dimg.p;
  }
  const int n_prior = ctx->K_id + ctx->K_exp + ctx->K_alb, nlv = 3 * ctx->cfg.n_lights;
  if (256 % opts->spp != 0) {
    // a pixel's samples span several blocks: the three calls in sequence,
    // then the prior and light terms' gradient (their value is in *loss)
    rc = fr_render(ctx, theta, opts, image, nullptr);
    if (!rc) rc = fr_loss(ctx, theta, opts->W, opts->H, image, target, mask, m, w1, w2, loss, d_image, nullptr);
    if (!rc) rc = fr_render_backward(ctx, theta, opts, d_image, grad, 0);
    if (rc) return rc;
    k_loss_reg<<<1, 256, 0, s>>>(theta, n_prior, ctx->off_lights(), nlv, ctx->cfg.light_prior, m, w1, w2, nullptr,
                                 grad);
    CKL();
    return FR_OK;
  }
  rc = prepare(ctx, theta, opts->W, opts->H);
  if (rc) return rc;
  const int V = ctx->V;
  CK(cudaMemsetAsync(grad, 0, sizeof(double) * ctx->n_params(), s));
  CK(cudaMemsetAsync(loss, 0, sizeof(double), s));
  CK(cudaMemsetAsync(ctx->dX.p, 0, sizeof(float4) * V, s));
  CK(cudaMemsetAsync(ctx->dN.p, 0, sizeof(float4) * V, s));
  CK(cudaMemsetAsync(ctx->dA.p, 0, sizeof(float4) * V, s));
  CK(cudaMemsetAsync(ctx->dC.p, 0, sizeof(float) * CS * CS, s));
  CK(cudaMemsetAsync(ctx->dL.p, 0, sizeof(float) * 3 * MAX_LIGHTS, s));
  if (ctx->counters_on) CK(cudaMemsetAsync(ctx->counters.p, 0, CNT_TOTAL * sizeof(unsigned long long), s));
  RenderArgs a = render_args(ctx, theta, opts, main_view(ctx));
  const int terms = opts->terms ? opts->terms : (TERM_INTERIOR | TERM_PEDGE | TERM_SEDGE);
  long long tiled = (long long)(((opts->W + 7) / 8) * ((opts->H + 7) / 8)) * 64 * opts->spp;
  if ((terms & TERM_SEDGE) && ctx->hits.n < (size_t)tiled) CK(ctx->hits.alloc(tiled));
  GradBufs gb;
  gb.dX = ctx->dX.p; gb.dN = ctx->dN.p; gb.dA = ctx->dA.p; gb.dC = ctx->dC.p; gb.dL = ctx->dL.p;
  gb.d_image = d_image;
  gb.hits = (terms & TERM_SEDGE) ? ctx->hits.p : nullptr;
  StepBufs sb;
  sb.image = image; sb.d_image = d_image; sb.target = target; sb.mask = mask; sb.loss = loss;
  sb.interior = (terms & TERM_INTERIOR) ? 1 : 0;
  ctx->mark(PH_FORWARD, 0);
  k_step_fwd<<<grid_for(tiled, 256), 256, 0, s>>>(a, gb, sb);
  CKL();
  ctx->mark(PH_FORWARD, 1);
  rc = edges_and_adjoint(ctx, theta, opts, a, gb, terms, grad);
  if (rc) return rc;
  ctx->mark(PH_LOSS, 0);
  k_loss_reg<<<1, 256, 0, s>>>(theta, n_prior, ctx->off_lights(), nlv, ctx->cfg.light_prior, m, w1, w2, loss, grad);
  CKL();
  ctx->mark(PH_LOSS, 1);
  return FR_OK;
}

int fr_geometry(fr_ctx* ctx, const float* theta, float* X, float* N, float* A) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  int rc = prepare(ctx, theta, 1, 1);
  if (rc) return rc;
  return geometry_outputs(ctx, X, N, A);
}

int fr_vertex_grad(fr_ctx* ctx, float* dX) {
  if (!ctx || !dX) return FR_ERR_INVALID_ARG;
  if (!ctx->have_mesh) return fail(ctx, FR_ERR_NOT_READY, "mesh not uploaded");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpy2DAsync(dX, 3 * sizeof(float), ctx->dX.p, sizeof(float4), 3 * sizeof(float), ctx->V,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  return FR_OK;
}

int fr_light_stage(const fr_ctx* ctx, float* out) {
  if (!ctx || !out) return FR_ERR_INVALID_ARG;
  for (int k = 0; k < ctx->cfg.n_lights; ++k) {
    const Light& L = ctx->lights[k];
    float v[12] = {L.c.x, L.c.y, L.c.z, L.e1.x, L.e1.y, L.e1.z, L.e2.x, L.e2.y, L.e2.z, L.dl.x, L.dl.y, L.dl.z};
    std::memcpy(out + 12 * k, v, sizeof v);
  }
  return FR_OK;
}

int fr_set_counters(fr_ctx* ctx, int32_t enable) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  ctx->counters_on = enable != 0;
  return FR_OK;
}

int fr_get_counters(fr_ctx* ctx, uint64_t* out) {
  if (!ctx || !out) return FR_ERR_INVALID_ARG;
  unsigned long long c[NCOUNT];
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(c, ctx->counters.p, sizeof c, cudaMemcpyDeviceToHost));
  for (int i = 0; i < NCOUNT; ++i) out[i] = c[i];
  return FR_OK;
}

int fr_set_timing(fr_ctx* ctx, int32_t enable) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  if (enable && !ctx->events_made) {
    for (int i = 0; i < NPHASE; ++i) {
      CK(cudaEventCreate(&ctx->ev[i][0]));
      CK(cudaEventCreate(&ctx->ev[i][1]));
    }
    ctx->events_made = true;
  }
  ctx->timing_on = enable != 0;
  for (int i = 0; i < NPHASE; ++i) ctx->phase_used[i] = false;
  return FR_OK;
}

int fr_get_timings(fr_ctx* ctx, float* ms) {
  if (!ctx || !ms) return FR_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < NPHASE; ++i) {
    ms[i] = 0.0f;
    if (ctx->events_made && ctx->phase_used[i]) CK(cudaEventElapsedTime(&ms[i], ctx->ev[i][0], ctx->ev[i][1]));
  }
  return FR_OK;
}

uint64_t fr_launch_count(const fr_ctx* ctx) { return ctx ? ctx->launches : 0; }

// ---------------------------------------------------------------------------
// Denoiser

int32_t fr_denoiser_n_weights(void) { return mlp_n_weights(); }

int fr_denoiser_set_weights(fr_ctx* ctx, const float* w, int32_t n) {
  if (!ctx || !w) return FR_ERR_INVALID_ARG;
  if (n != mlp_n_weights()) return fail(ctx, FR_ERR_SHAPE, "denoiser has %d weights, got %d", mlp_n_weights(), n);
  CK(cudaSetDevice(ctx->device));
  if (!ctx->have_mlp) {
    CK(ctx->mlp_w.alloc(n)); CK(ctx->mlp_m.alloc(n)); CK(ctx->mlp_v.alloc(n)); CK(ctx->mlp_g.alloc(n));
    static bool attr_done[64] = {false};
    if (ctx->device < 64 && !attr_done[ctx->device]) {
      CK(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes()));
      CK(cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_smem_bytes()));
      CK(cudaFuncSetAttribute(k_mlp_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 4));
      attr_done[ctx->device] = true;
    }
  }
  CK(cudaMemcpyAsync(ctx->mlp_w.p, w, sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->mlp_m.p, 0, sizeof(float) * n, ctx->stream));
  CK(cudaMemsetAsync(ctx->mlp_v.p, 0, sizeof(float) * n, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_mlp = true;
  ctx->mlp_steps = 0;
  return FR_OK;
}

int fr_denoiser_get_weights(fr_ctx* ctx, float* w, int32_t n) {
  if (!ctx || !w) return FR_ERR_INVALID_ARG;
  if (!ctx->have_mlp) return fail(ctx, FR_ERR_NOT_READY, "denoiser weights not set");
  if (n != mlp_n_weights()) return fail(ctx, FR_ERR_SHAPE, "denoiser has %d weights, got %d", mlp_n_weights(), n);
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpyAsync(w, ctx->mlp_w.p, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FR_OK;
}

int fr_denoise(fr_ctx* ctx, const float* aov, int32_t n_pix, float* out, const float* d_out, float* d_rgb) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (!ctx->have_mlp) return fail(ctx, FR_ERR_NOT_READY, "denoiser weights not set");
  if (!aov || !out || n_pix < 1 || (d_out && !d_rgb)) return fail(ctx, FR_ERR_INVALID_ARG, "fr_denoise arguments");
  CK(cudaSetDevice(ctx->device));
  int blocks = (n_pix + 127) / 128;
  k_mlp_infer<<<blocks, 256, mlp_smem_bytes(), ctx->stream>>>(n_pix, ctx->mlp_w.p, aov, out, d_out, d_rgb);
  CKL();
  return FR_OK;
}

int fr_denoiser_train_step(fr_ctx* ctx, const float* aov, const float* target, int32_t n_pix, float lr,
                           double* loss) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (!ctx->have_mlp) return fail(ctx, FR_ERR_NOT_READY, "denoiser weights not set");
  if (!aov || !target || !loss || n_pix < 1 || !(lr > 0)) return fail(ctx, FR_ERR_INVALID_ARG, "train_step arguments");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const int stride = mlp_train_stride();
  if (ctx->mlp_scratch.n < (size_t)n_pix * stride) CK(ctx->mlp_scratch.alloc((size_t)n_pix * stride));
  const int NW = mlp_n_weights();
  CK(cudaMemsetAsync(ctx->mlp_g.p, 0, sizeof(float) * NW, s));
  CK(cudaMemsetAsync(loss, 0, sizeof(double), s));
  k_mlp_train_tc<<<(n_pix + 127) / 128, 256, mlp_smem_bytes(), s>>>(n_pix, ctx->mlp_w.p, aov, target,
                                                                    ctx->mlp_scratch.p, loss);
  CKL();
  int off[8];
  mlp_layer_offsets(off);
  // scratch offsets: h0 0, h1 16, h2 80, h3 144, g1 208, g2 272, g3 336, g4 400
  const int chunk = 128;
  const int nb = (n_pix + chunk - 1) / chunk;
  struct L { int g, h, N, K, Kw, w, b; } layers[4] = {
      {208, 0, 64, 16, 14, off[0], off[1]}, {272, 16, 64, 64, 64, off[2], off[3]},
      {336, 80, 64, 64, 64, off[4], off[5]}, {400, 144, 3, 64, 64, off[6], off[7]}};
  for (const L& l : layers) {
    size_t sm = sizeof(float) * chunk * (l.N + l.K);
    k_mlp_wgrad<<<nb, 256, sm, s>>>(n_pix, ctx->mlp_scratch.p, l.g, l.h, l.N, l.K, l.Kw, ctx->mlp_g.p + l.w,
                                    ctx->mlp_g.p + l.b, chunk);
    CKL();
  }
  ctx->mlp_steps++;
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = (float)(1.0 - std::pow((double)b1, (double)ctx->mlp_steps));
  float c2 = (float)(1.0 - std::pow((double)b2, (double)ctx->mlp_steps));
  k_adam<<<(NW + 255) / 256, 256, 0, s>>>(NW, ctx->mlp_w.p, ctx->mlp_g.p, ctx->mlp_m.p, ctx->mlp_v.p, lr, b1, b2,
                                          1e-8f, c1, c2);
  CKL();
  return FR_OK;
}

int fr_adam_step(fr_ctx* ctx, float* theta, const double* grad, float* m, float* v, const float* lr, int32_t step) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (!ctx->have_bases) return fail(ctx, FR_ERR_NOT_READY, "bases not uploaded");
  if (!theta || !grad || !m || !v || !lr || step < 1) return fail(ctx, FR_ERR_INVALID_ARG, "fr_adam_step arguments");
  CK(cudaSetDevice(ctx->device));
  const int P = ctx->n_params();
  float c1 = (float)(1.0 - std::pow(0.9, (double)step)), c2 = (float)(1.0 - std::pow(0.999, (double)step));
  k_adam_theta<<<(P + 255) / 256, 256, 0, ctx->stream>>>(P, theta, grad, m, v, lr, c1, c2, ctx->off_cspec(), CS * CS,
                                                         ctx->off_lights());
  CKL();
  return FR_OK;
}

// Gradient of the last training step (for tests), host copy.
int fr_denoiser_get_grad(fr_ctx* ctx, float* g, int32_t n) {
  if (!ctx || !g) return FR_ERR_INVALID_ARG;
  if (!ctx->have_mlp || n != mlp_n_weights()) return fail(ctx, FR_ERR_SHAPE, "denoiser gradient size");
  CK(cudaSetDevice(ctx->device));
  CK(cudaMemcpyAsync(g, ctx->mlp_g.p, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return FR_OK;
}

// ---------------------------------------------------------------------------
// Geometry stage without device allocation.
//
// Some callers cannot call cudaMalloc while they run this library: a
// framework whose caching allocator owns all device memory and forbids
// allocations behind its back, a fixed-budget deployment that reserves every
// byte at start-up, or a latency-critical loop that must not pay the implicit
// device synchronisation cudaMalloc/cudaFree may trigger.  For them the
// camera-silhouette compaction keeps its per-block counts in the file-scope
// array below instead of a context buffer.  The array exists once per device
// that loads the library and lives until the process exits; every call on
// that device shares it, and each call overwrites every count it reads before
// reading it, so nothing has to be cleared between calls.  Two calls whose
// work overlaps on the GPU (different contexts on different streams of the
// same device) race on it.

constexpr int NOALLOC_MAX_SIL_BLOCKS = 4096;   // 16 KiB: up to 4096 * 256 = 1,048,576 edges
static __device__ __align__(256) int g_noalloc_sil_blocks[NOALLOC_MAX_SIL_BLOCKS];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
int* g_noalloc_sil_ptr[NOALLOC_MAX_DEVICES];   // device address of the array, per device
std::mutex g_noalloc_mu;

// In host code the array's name only stands in for the symbol; its device
// address comes from the runtime, once per device, with that device current.
int noalloc_scratch(fr_ctx* ctx, int** out) {
  if (ctx->device < 0 || ctx->device >= NOALLOC_MAX_DEVICES)
    return fail(ctx, FR_ERR_INVALID_ARG, "device %d beyond the %d devices supported", ctx->device, NOALLOC_MAX_DEVICES);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_sil_ptr[ctx->device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_sil_blocks);
    if (e != cudaSuccess || !p)
      return fail(ctx, FR_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(e));
    g_noalloc_sil_ptr[ctx->device] = static_cast<int*>(p);
  }
  *out = g_noalloc_sil_ptr[ctx->device];
  return FR_OK;
}
}  // namespace

int fr_geometry_noalloc(fr_ctx* ctx, const float* theta, float* X, float* N, float* A) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  int nb = (ctx->E + 255) / 256;
  if (nb > NOALLOC_MAX_SIL_BLOCKS)
    return fail(ctx, FR_ERR_INVALID_ARG, "fr_geometry_noalloc supports at most %d mesh edges (mesh has %d)",
                NOALLOC_MAX_SIL_BLOCKS * 256, ctx->E);
  CK(cudaSetDevice(ctx->device));
  int* scratch = nullptr;
  int rc = noalloc_scratch(ctx, &scratch);
  if (rc) return rc;
  FrameView v = main_view(ctx);
  rc = prepare_geometry(ctx, theta, v);
  if (rc) return rc;
  v.block_count = scratch;
  rc = silhouettes(ctx, v);
  if (rc) return rc;
  return geometry_outputs(ctx, X, N, A);
}

int fr_silhouettes(fr_ctx* ctx, int32_t* out, int32_t cap) {
  if (!ctx || cap < 0 || (cap > 0 && !out)) return FR_ERR_INVALID_ARG;
  if (!ctx->have_mesh) return fail(ctx, FR_ERR_NOT_READY, "mesh not uploaded");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  int n = 0;
  CK(cudaMemcpy(&n, ctx->n_sil.p, sizeof(int), cudaMemcpyDeviceToHost));
  const int k = std::min(n, (int)cap);
  if (k > 0) CK(cudaMemcpy(out, ctx->sil.p, sizeof(int) * (size_t)k, cudaMemcpyDeviceToHost));
  return n;
}

int fr_set_limits(fr_ctx* ctx, int32_t max_steps, int32_t wait_limit) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  if (max_steps < 1 || wait_limit < 0)
    return fail(ctx, FR_ERR_INVALID_ARG, "limits: max_steps must be >= 1 and wait_limit >= 0");
  ctx->max_steps = max_steps;
  ctx->wait_limit = wait_limit;
  return FR_OK;
}

// Wait for the context stream and report device-side limit hits (traversal
// stack overflow or step cap) raised since the last call, clearing the flag.
int fr_sync(fr_ctx* ctx) {
  if (!ctx) return FR_ERR_INVALID_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  int flag = 0;
  CK(cudaMemcpy(&flag, ctx->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    CK(cudaMemset(ctx->err_flag.p, 0, sizeof(int)));
    return fail(ctx, FR_ERR_DEVICE_LIMIT, "device traversal limit reached (flags 0x%x)", flag);
  }
  return FR_OK;
}

}  // extern "C"
