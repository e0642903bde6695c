// Geometry stage and its adjoint (Face Modeling paragraph):
//   X_model = mu + B_id alpha + B_exp beta, X = R(r) X_model + t,
//   albedo = mu_a + B_alb delta, area-weighted unit vertex normals,
// face normals in decision form, refit of the triangle and edge BVHs, and the
// list of camera-silhouette edges.  Backward: normals adjoint, R^T, the
// transposed basis contractions and the pose gradient.
#include "kernels.cuh"

namespace fr {

// Rotation R = Rz Ry Rx (row-major) and its derivatives dR/dr_m.
__device__ void rotation(const float* pose, double* R) {
  double cx = cos((double)pose[0]), sx = sin((double)pose[0]);
  double cy = cos((double)pose[1]), sy = sin((double)pose[1]);
  double cz = cos((double)pose[2]), sz = sin((double)pose[2]);
  R[0] = cz * cy; R[1] = cz * sy * sx - sz * cx; R[2] = cz * sy * cx + sz * sx;
  R[3] = sz * cy; R[4] = sz * sy * sx + cz * cx; R[5] = sz * sy * cx - cz * sx;
  R[6] = -sy;     R[7] = cy * sx;                R[8] = cy * cx;
}

__device__ void rotation_grad(const float* pose, float* dR /*[3][9]*/) {
  float cx = cosf(pose[0]), sx = sinf(pose[0]);
  float cy = cosf(pose[1]), sy = sinf(pose[1]);
  float cz = cosf(pose[2]), sz = sinf(pose[2]);
  // d/drx
  float* A = dR;
  A[0] = 0; A[1] = cz * sy * cx + sz * sx; A[2] = -cz * sy * sx + sz * cx;
  A[3] = 0; A[4] = sz * sy * cx - cz * sx; A[5] = -sz * sy * sx - cz * cx;
  A[6] = 0; A[7] = cy * cx;                A[8] = -cy * sx;
  // d/dry
  float* B = dR + 9;
  B[0] = -cz * sy; B[1] = cz * cy * sx; B[2] = cz * cy * cx;
  B[3] = -sz * sy; B[4] = sz * cy * sx; B[5] = sz * cy * cx;
  B[6] = -cy;      B[7] = -sy * sx;     B[8] = -sy * cx;
  // d/drz
  float* Cc = dR + 18;
  Cc[0] = -sz * cy; Cc[1] = -sz * sy * sx - cz * cx; Cc[2] = -sz * sy * cx + cz * sx;
  Cc[3] = cz * cy;  Cc[4] = cz * sy * sx - sz * cx;  Cc[5] = cz * sy * cx + sz * sx;
  Cc[6] = 0;        Cc[7] = 0;                       Cc[8] = 0;
}

// Positions accumulate in FP64 so that their FP32 rounding is (up to a tie
// at a rounding boundary) independent of summation order; albedo
// accumulates in FP32.  Bases are stored transposed, [K][3V].  A block
// covers GEO_VERTS vertices, i.e. 3 * GEO_VERTS coordinates i = 3 v + c, with
// GEO_KSPLIT groups of three warps: group q sums the q-th quarter of the
// basis columns for every coordinate of the block (reads coalesced along
// i).  The quarters' partial sums meet in shared memory in a fixed order;
// then one thread per vertex applies the pose.
__global__ void __launch_bounds__(GEO_THREADS) k_geometry(GeoArgs g, const float* __restrict__ theta) {
  __shared__ double R[9];
  __shared__ float coef[512];
  __shared__ double sx[GEO_KSPLIT][3 * GEO_VERTS];
  __shared__ float sa[GEO_KSPLIT][3 * GEO_VERTS];
  const int K1 = g.K_id, K2 = g.K_exp, K3 = g.K_alb;
  if (threadIdx.x == 0) rotation(theta + g.off_pose, R);
  for (int i = threadIdx.x; i < K1 + K2 + K3; i += blockDim.x) coef[i] = theta[i];
  __syncthreads();
  const int n3 = 3 * g.V;
  const int q = threadIdx.x / (3 * GEO_VERTS), ii = threadIdx.x - q * (3 * GEO_VERTS);
  const int i = 3 * GEO_VERTS * blockIdx.x + ii;
  double x = 0.0;
  float al = 0.0f;
  if (i < n3) {
    const int KG = K1 + K2, cg = (KG + GEO_KSPLIT - 1) / GEO_KSPLIT, ca = (K3 + GEO_KSPLIT - 1) / GEO_KSPLIT;
    const int k1 = min(KG, (q + 1) * cg);
    for (int k = q * cg; k < k1; ++k) {
      const float* B = k < K1 ? g.BidT + (size_t)k * n3 : g.BexpT + (size_t)(k - K1) * n3;
      x += (double)B[i] * (double)coef[k];
    }
    if (g.alb) {             // null: albedo kept from another frame of a batch
      const int a1 = min(K3, (q + 1) * ca);
      for (int k = q * ca; k < a1; ++k) al += g.BalbT[(size_t)k * n3 + i] * coef[K1 + K2 + k];
    }
  }
  sx[q][ii] = x;
  sa[q][ii] = al;
  __syncthreads();
  if (q == 0 && i < n3) {
    double xm = (double)g.mean[i];
    float a = g.alb ? g.alb_mean[i] : 0.0f;
#pragma unroll
    for (int r = 0; r < GEO_KSPLIT; ++r) { xm += sx[r][ii]; a += sa[r][ii]; }
    sx[0][ii] = xm;
    sa[0][ii] = a;
  }
  __syncthreads();
  const int v = GEO_VERTS * blockIdx.x + threadIdx.x;
  if (threadIdx.x >= GEO_VERTS || v >= g.V) return;
  const double* xm = &sx[0][3 * threadIdx.x];
  const float* a = &sa[0][3 * threadIdx.x];
  const float* t = theta + g.off_pose + 3;
  float X[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double xw = R[3 * c] * xm[0] + R[3 * c + 1] * xm[1] + R[3 * c + 2] * xm[2] + (double)t[c];
    X[c] = (float)xw;
  }
  g.X[v] = make_float4(X[0], X[1], X[2], 0.0f);
  g.Xm[v] = make_float4((float)xm[0], (float)xm[1], (float)xm[2], 0.0f);
  if (g.alb) g.alb[v] = make_float4(a[0], a[1], a[2], 0.0f);
}

// Face normals in decision form and the leaf-ordered triangle array.
__global__ void k_faces(GeoArgs g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;   // leaf-order slot
  if (i >= g.F) return;
  int f = g.tri_perm[i];
  int4 t = g.tris[f];
  float4 p0 = g.X[t.x], p1 = g.X[t.y], p2 = g.X[t.z];
  V3 a = v3(p0), b = v3(p1), c = v3(p2);
  V3 n = cross3r(sub3r(b, a), sub3r(c, a));
  g.ng[f] = make_float4(n.x, n.y, n.z, 0.0f);
  g.tv[3 * i] = make_float4(a.x, a.y, a.z, __int_as_float(f));
  g.tv[3 * i + 1] = make_float4(b.x, b.y, b.z, 0.0f);
  g.tv[3 * i + 2] = make_float4(c.x, c.y, c.z, 0.0f);
}

// Packed per-edge records for the shadow-edge search (edge-BVH leaf order):
// endpoints, ids, and for each adjacent face its decision-form normal and
// first vertex, so that a leaf test reads one 96-byte record.
__global__ void k_pack_edges(int E, const int4* __restrict__ edges_leaf, const int* __restrict__ edge_id,
                             const int4* __restrict__ tris, const float4* __restrict__ X,
                             const float4* __restrict__ ng, float4* __restrict__ pack) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E) return;
  int4 e = edges_leaf[i];
  float4 a = X[e.x], b = X[e.y];
  float4 n0 = ng[e.z];
  float4 p0 = X[tris[e.z].x];
  float4 n1 = make_float4(0, 0, 0, 0), p1 = make_float4(0, 0, 0, 0);
  if (e.w >= 0) { n1 = ng[e.w]; p1 = X[tris[e.w].x]; }
  float4* R = pack + 6 * (size_t)i;
  R[0] = make_float4(a.x, a.y, a.z, __int_as_float(edge_id[i]));
  R[1] = make_float4(b.x, b.y, b.z, __int_as_float(e.z));
  R[2] = make_float4(n0.x, n0.y, n0.z, __int_as_float(e.w));
  R[3] = make_float4(p0.x, p0.y, p0.z, 0.0f);
  R[4] = make_float4(n1.x, n1.y, n1.z, 0.0f);
  R[5] = make_float4(p1.x, p1.y, p1.z, 0.0f);
}

// Unit vertex normals: gather the face cross products around each vertex.
__global__ void k_vertex_normals(GeoArgs g) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.V) return;
  V3 s{0, 0, 0};
  for (int k = g.vf_off[v]; k < g.vf_off[v + 1]; ++k) {
    int4 t = g.tris[g.vf_idx[k]];
    V3 a = v3(g.X[t.x]), b = v3(g.X[t.y]), c = v3(g.X[t.z]);
    s += cross(b - a, c - a);
  }
  float l2 = dot(s, s);
  float inv = l2 > 0.0f ? rsqrtf(l2) : 0.0f;
  g.nrm[v] = make_float4(s.x * inv, s.y * inv, s.z * inv, inv);
}

// Pad a box so that FP32 rounding in the slab test can never reject a ray
// that the watertight triangle test accepts.
__device__ __forceinline__ void pad_box(V3& lo, V3& hi) {
  const float r = 1e-6f, a = 1e-5f;
  lo.x -= a + r * fabsf(lo.x); lo.y -= a + r * fabsf(lo.y); lo.z -= a + r * fabsf(lo.z);
  hi.x += a + r * fabsf(hi.x); hi.y += a + r * fabsf(hi.y); hi.z += a + r * fabsf(hi.z);
}

__device__ __forceinline__ void write_slot(float4* nodes, int node, int slot, V3 lo, V3 hi) {
  float* N = reinterpret_cast<float*>(nodes + 4 * node);
  int o = slot ? 6 : 0;
  N[o + 0] = lo.x; N[o + 1] = lo.y; N[o + 2] = lo.z; N[o + 3] = hi.x; N[o + 4] = hi.y; N[o + 5] = hi.z;
}

__global__ void k_gather4(int n_slots, const int2* __restrict__ src, const float4* __restrict__ nodes,
                          const float4* __restrict__ cones, float2* __restrict__ boxes4, float4* __restrict__ cones4) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_slots) return;
  int2 sr = src[i];
  float b[6] = {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f};
  float4 cn = make_float4(0.0f, 0.0f, 1.0f, -1.0f);
  float4 sp = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  if (sr.x >= 0) {
    const float* N = reinterpret_cast<const float*>(nodes + 4 * sr.x) + 6 * sr.y;
    for (int k = 0; k < 6; ++k) b[k] = N[k];
    cn = cones[2 * sr.x + sr.y];
    // the search's cone test takes cos(theta + 2e-3), the half-angle grown
    // for rounding; a cone of pi/2 or more can prune nothing (-1)
    const float th = cn.w + 2e-3f;
    cn.w = th < 0.5f * PI_F ? cosf(th) : -1.0f;
    // bounding sphere of the box, grown for rounding
    const V3 lo{b[0], b[1], b[2]}, hi{b[3], b[4], b[5]};
    const V3 c = (lo + hi) * 0.5f;
    sp = make_float4(c.x, c.y, c.z, len((hi - lo) * 0.5f) * 1.0001f + 1e-6f);
  }
  float2* B = boxes4 + 3 * i;
  B[0] = make_float2(b[0], b[1]);
  B[1] = make_float2(b[2], b[3]);
  B[2] = make_float2(b[4], b[5]);
  cones4[2 * i] = cn;
  cones4[2 * i + 1] = sp;
}

// Bottom-up refit: one thread per leaf; the second child to arrive at a node
// computes the node's box and carries on upward.
// Normal cone of the faces adjacent to the edges of one leaf; boundary edges
// make it full (they are silhouettes from any side).
__device__ float4 leaf_cone(const float4* pack, int first, int cnt) {
  V3 n[8];
  int m = 0;
  bool full = false;
  for (int k = 0; k < cnt; ++k) {
    const float4* R = pack + 6 * (first + k);
    float4 n0 = R[2];
    n[m++] = normalize(v3(n0));
    if (__float_as_int(n0.w) < 0) full = true;
    else n[m++] = normalize(v3(R[4]));
  }
  V3 sum{0, 0, 0};
  for (int k = 0; k < m; ++k) sum += n[k];
  float l2 = dot(sum, sum);
  if (full || !(l2 > 1e-12f)) return make_float4(0, 0, 1, CONE_FULL);
  V3 ax = sum * rsqrtf(l2);
  float th = 0.0f;
  for (int k = 0; k < m; ++k) th = fmaxf(th, acosf(fminf(1.0f, fmaxf(-1.0f, dot(ax, n[k])))));
  return make_float4(ax.x, ax.y, ax.z, th * 1.0001f + 1e-4f);
}

__global__ void k_refit(RefitArgs r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r.n_leaves) return;
  int first = r.leaf_first[i], cnt = r.leaf_count[i];
  V3 lo{3e38f, 3e38f, 3e38f}, hi{-3e38f, -3e38f, -3e38f};
  for (int k = 0; k < cnt; ++k) {
    int s = first + k;
    for (int q = 0; q < 2 + (r.is_edge ? 0 : 1); ++q) {
      V3 p;
      if (r.is_edge) {
        int4 e = r.edges[s];
        p = v3(r.X[q == 0 ? e.x : e.y]);
      } else {
        p = v3(r.tv[3 * s + q]);
      }
      lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
      hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
    }
  }
  pad_box(lo, hi);
  float4 cone = r.is_edge ? leaf_cone(r.pack, first, cnt) : make_float4(0, 0, 1, CONE_FULL);
  int node = r.leaf_parent[i], slot = r.leaf_slot[i];
  while (node >= 0) {
    write_slot(r.nodes, node, slot, lo, hi);
    if (r.is_edge) r.cones[2 * node + slot] = cone;
    __threadfence();
    int prev = atomicAdd(&r.counter[node], 1);
    if (prev == 0) return;          // the sibling finishes this node
    __threadfence();
    const float* N = reinterpret_cast<const float*>(r.nodes + 4 * node);
    volatile const float* Nv = N;
    V3 l0{Nv[0], Nv[1], Nv[2]}, h0{Nv[3], Nv[4], Nv[5]}, l1{Nv[6], Nv[7], Nv[8]}, h1{Nv[9], Nv[10], Nv[11]};
    lo = V3{fminf(l0.x, l1.x), fminf(l0.y, l1.y), fminf(l0.z, l1.z)};
    hi = V3{fmaxf(h0.x, h1.x), fmaxf(h0.y, h1.y), fmaxf(h0.z, h1.z)};
    if (r.is_edge) {
      volatile const float* C = reinterpret_cast<const float*>(r.cones + 2 * node);
      cone = cone_merge(make_float4(C[0], C[1], C[2], C[3]), make_float4(C[4], C[5], C[6], C[7]));
    }
    slot = r.node_slot[node];
    node = r.node_parent[node];
  }
}

// Camera silhouette flags (decision form) and per-block counts.
__global__ void k_silhouette_flags(SilArgs s) {
  __shared__ int warp_cnt[32];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int flag = 0;
  if (e < s.E) {
    int4 E = s.edges[e];   // v0, v1, f0, f1 in canonical edge order
    if (E.w < 0) {
      flag = 1;
    } else {
      float4 n0 = s.ng[E.z], n1 = s.ng[E.w];
      V3 w0 = sub3r(s.cam_o, v3(s.X[s.tris[E.z].x]));
      V3 w1 = sub3r(s.cam_o, v3(s.X[s.tris[E.w].x]));
      float s0 = dot3r(v3(n0), w0), s1 = dot3r(v3(n1), w1);
      flag = ((s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f)) ? 1 : 0;
    }
  }
  unsigned m = __ballot_sync(0xffffffffu, flag);
  if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) c += warp_cnt[w];
    s.block_count[blockIdx.x] = c;
  }
}

// Exclusive scan of the per-block counts (one block) and the total.
__global__ void k_silhouette_scan(SilArgs s, int nblocks) {
  __shared__ int buf[1024];
  int carry = 0;
  for (int base = 0; base < nblocks; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < nblocks ? s.block_count[i] : 0;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int t = threadIdx.x >= off ? buf[threadIdx.x - off] : 0;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nblocks) s.block_count[i] = carry + buf[threadIdx.x] - v;
    int tot = buf[1023];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) *s.n_sil = carry;
}

// Order-preserving compaction of the flagged edges.
__global__ void k_silhouette_scatter(SilArgs s) {
  __shared__ int warp_off[32];
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int flag = 0;
  if (e < s.E) {
    int4 E = s.edges[e];
    if (E.w < 0) {
      flag = 1;
    } else {
      float4 n0 = s.ng[E.z], n1 = s.ng[E.w];
      V3 w0 = sub3r(s.cam_o, v3(s.X[s.tris[E.z].x]));
      V3 w1 = sub3r(s.cam_o, v3(s.X[s.tris[E.w].x]));
      float s0 = dot3r(v3(n0), w0), s1 = dot3r(v3(n1), w1);
      flag = ((s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f)) ? 1 : 0;
    }
  }
  unsigned m = __ballot_sync(0xffffffffu, flag);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) warp_off[w] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { int t = warp_off[k]; warp_off[k] = c; c += t; }
  }
  __syncthreads();
  if (flag) {
    int pos = s.block_count[blockIdx.x] + warp_off[w] + __popc(m & ((1u << lane) - 1u));
    s.sil[pos] = e;
  }
}

// ---------------------------------------------------------------------------
// Backward

// dN (unit normals) -> gradient of the unnormalised normal sum, per vertex.
__global__ void k_normals_bwd_vertex(GeoArgs g, const float4* __restrict__ dN, float4* __restrict__ gs) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.V) return;
  float4 n = g.nrm[v];
  float4 d = dN[v];
  float dd = n.x * d.x + n.y * d.y + n.z * d.z;
  float inv = n.w;
  gs[v] = make_float4((d.x - dd * n.x) * inv, (d.y - dd * n.y) * inv, (d.z - dd * n.z) * inv, 0.0f);
}

// Per vertex, gather the adjoint of every incident face's cross product.
__global__ void k_normals_bwd_gather(GeoArgs g, const float4* __restrict__ gs, float4* __restrict__ dX) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.V) return;
  V3 acc{0, 0, 0};
  for (int k = g.vf_off[v]; k < g.vf_off[v + 1]; ++k) {
    int4 t = g.tris[g.vf_idx[k]];
    V3 P0 = v3(g.X[t.x]), P1 = v3(g.X[t.y]), P2 = v3(g.X[t.z]);
    V3 gc = v3(gs[t.x]) + v3(gs[t.y]) + v3(gs[t.z]);
    V3 e1 = P1 - P0, e2 = P2 - P0;
    V3 ge1 = cross(e2, gc), ge2 = cross(gc, e1);
    if (t.x == v) acc -= ge1 + ge2;
    if (t.y == v) acc += ge1;
    if (t.z == v) acc += ge2;
  }
  float4 o = dX[v];
  dX[v] = make_float4(o.x + acc.x, o.y + acc.y, o.z + acc.z, 0.0f);
}

// dX -> dX_model = R^T dX (FP32, [3V] flat) and the pose gradient.
__global__ void k_pose_bwd(GeoArgs g, const float* __restrict__ theta, const float4* __restrict__ dX,
                           float* __restrict__ dXm, double* __restrict__ grad) {
  __shared__ float R[9];
  __shared__ float dR[27];
  __shared__ double red[6][32];
  if (threadIdx.x == 0) {
    double Rd[9];
    rotation(theta + g.off_pose, Rd);
    for (int i = 0; i < 9; ++i) R[i] = (float)Rd[i];
    rotation_grad(theta + g.off_pose, dR);
  }
  __syncthreads();
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.V; v += gridDim.x * blockDim.x) {
    float4 d = dX[v];
    float4 xm = g.Xm[v];
    for (int c = 0; c < 3; ++c) dXm[3 * v + c] = R[c] * d.x + R[3 + c] * d.y + R[6 + c] * d.z;
    acc[3] += d.x; acc[4] += d.y; acc[5] += d.z;
    for (int mm = 0; mm < 3; ++mm) {
      const float* A = dR + 9 * mm;
      float r0 = A[0] * xm.x + A[1] * xm.y + A[2] * xm.z;
      float r1 = A[3] * xm.x + A[4] * xm.y + A[5] * xm.z;
      float r2 = A[6] * xm.x + A[7] * xm.y + A[8] * xm.z;
      acc[mm] += (double)(d.x * r0 + d.y * r1 + d.z * r2);
    }
  }
  for (int q = 0; q < 6; ++q) {
    double v = acc[q];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[threadIdx.x][w];
    atomicAdd(&grad[g.off_pose + threadIdx.x], s);
  }
}

// Transposed basis contraction: grad[out_off + k] += sum_i B^T[k][i] * y[i].
// Grid (K, BASIS_SLICES): block (k, s) sums the s-th slice of row k (FP32 per
// thread, FP64 across the block) and adds it with one FP64 atomic, so that
// K * BASIS_SLICES blocks stream the basis.
__global__ void k_basis_T(const float* __restrict__ BT, int K, int n, const float* __restrict__ y,
                          const float4* __restrict__ y4, double* __restrict__ grad, int out_off) {
  __shared__ double red[32];
  const int k = blockIdx.x;
  if (k >= K) return;
  const int chunk = (n + (int)gridDim.y - 1) / (int)gridDim.y;
  const int i0 = (int)blockIdx.y * chunk, i1 = min(n, i0 + chunk);
  const float* row = BT + (size_t)k * n;
  float acc = 0.0f;
  if (y) {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += row[i] * y[i];
  } else {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      float4 q = y4[i / 3];
      int c = i - 3 * (i / 3);
      acc += row[i] * (c == 0 ? q.x : (c == 1 ? q.y : q.z));
    }
  }
  double v = acc;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(&grad[out_off + k], s);
  }
}

// FP32 accumulators (c_spec texels, lights) -> FP64 gradient.
__global__ void k_add_small(const float* __restrict__ src, int n, double* __restrict__ grad, int off) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) grad[off + i] += (double)src[i];
}

}  // namespace fr
