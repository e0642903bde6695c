// Device helpers shared by the facert kernels.
//
// Decision arithmetic.  Every discrete decision of the renderer (which
// triangle a ray hits, whether a shadow ray is blocked, whether an edge is a
// silhouette or can cast a shadow onto a light, which pixel an edge sample
// lands in) is computed in FP32 with explicitly rounded intrinsics
// (__fmul_rn, __fadd_rn, ...), which the compiler never fuses into FMAs.  The
// order of operations of each predicate is part of its definition, so the
// decisions are reproducible by any IEEE FP32 implementation of the same
// formula.  Values (radiance, derivatives) use ordinary FP32 arithmetic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define FR_DEV __device__ __forceinline__
#define FR_HOST_DEV __host__ __device__

namespace fr {

constexpr int CS = 32;              // specular map resolution
constexpr int MAX_LIGHTS = 32;
constexpr float PI_F = 3.14159265358979323846f;

// Stream tags of the Philox counter word 2 (tag << 8 | light).
enum { TAG_CAMERA = 0, TAG_LIGHT = 1, TAG_PEDGE = 2, TAG_PEDGE_LIGHT = 3, TAG_SEDGE_POINT = 4,
       TAG_SEDGE_PICK = 5, TAG_PEDGE_OFFSET = 6 };
enum { TERM_INTERIOR = 1, TERM_PEDGE = 2, TERM_SEDGE = 4 };
enum { ERR_STACK = 1, ERR_STEPS = 2, ERR_WAIT = 4 };   // device error flags
// Work counters (fr_set_counters): 6 per render kernel, in the order forward,
// interior adjoint, primary edges, shadow edges; within a kernel: BVH node
// visits of rays, triangle tests, edge-hierarchy node visits (once per warp),
// exact silhouette tests of (shading point, edge) pairs, clip tests (pairs
// that passed the silhouette and adjacency tests), and leaf edges classified
// against the box of a warp's shading points (once per warp).
enum { CNT_PER_KERNEL = 6, CNT_FWD = 0, CNT_INTERIOR = 6, CNT_PEDGE = 12, CNT_SEDGE = 18, CNT_TOTAL = 24 };

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
struct U4 { uint32_t x, y, z, w; };

FR_DEV U4 philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}
// 24-bit uniform in [0, 1), exact in FP32.
FR_DEV float unitf(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// small vector type (values)
struct V3 { float x, y, z; };
FR_DEV V3 v3(float x, float y, float z) { return V3{x, y, z}; }
FR_DEV V3 v3(float4 a) { return V3{a.x, a.y, a.z}; }
FR_DEV V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
FR_DEV V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
FR_DEV V3 operator-(V3 a) { return V3{-a.x, -a.y, -a.z}; }
FR_DEV V3 operator*(V3 a, float s) { return V3{a.x * s, a.y * s, a.z * s}; }
FR_DEV V3 operator*(float s, V3 a) { return V3{a.x * s, a.y * s, a.z * s}; }
FR_DEV V3& operator+=(V3& a, V3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
FR_DEV V3& operator-=(V3& a, V3 b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; return a; }
FR_DEV float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
FR_DEV V3 cross(V3 a, V3 b) { return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
FR_DEV float len(V3 a) { return sqrtf(dot(a, a)); }
FR_DEV V3 normalize(V3 a) { return a * rsqrtf(dot(a, a)); }

// ---------------------------------------------------------------------------
// exactly rounded decision arithmetic
FR_DEV float dot3r(V3 a, V3 b) {
  float p = __fmul_rn(a.x, b.x);
  p = __fadd_rn(p, __fmul_rn(a.y, b.y));
  p = __fadd_rn(p, __fmul_rn(a.z, b.z));
  return p;
}
FR_DEV V3 sub3r(V3 a, V3 b) { return V3{__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z)}; }
FR_DEV V3 cross3r(V3 a, V3 b) {
  return V3{__fsub_rn(__fmul_rn(a.y, b.z), __fmul_rn(a.z, b.y)),
            __fsub_rn(__fmul_rn(a.z, b.x), __fmul_rn(a.x, b.z)),
            __fsub_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x))};
}
FR_DEV float comp(V3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2(1), 2013).
struct RayPre { int kx, ky, kz; float Sx, Sy, Sz; V3 o; };

FR_DEV RayPre ray_pre(V3 o, V3 d) {
  RayPre r;
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  int kx = kz + 1; if (kx == 3) kx = 0;
  int ky = kx + 1; if (ky == 3) ky = 0;
  float dz = comp(d, kz);
  if (dz < 0.0f) { int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  r.Sx = __fdiv_rn(comp(d, kx), dz);
  r.Sy = __fdiv_rn(comp(d, ky), dz);
  r.Sz = __fdiv_rn(1.0f, dz);
  r.o = o;
  return r;
}

// Line/triangle crossing; writes the ray parameter t (unrestricted).
FR_DEV bool tri_hit(const RayPre& r, V3 v0, V3 v1, V3 v2, float& t) {
  V3 A = sub3r(v0, r.o), B = sub3r(v1, r.o), C = sub3r(v2, r.o);
  float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
  float Ax = __fsub_rn(comp(A, r.kx), __fmul_rn(r.Sx, Akz)), Ay = __fsub_rn(comp(A, r.ky), __fmul_rn(r.Sy, Akz));
  float Bx = __fsub_rn(comp(B, r.kx), __fmul_rn(r.Sx, Bkz)), By = __fsub_rn(comp(B, r.ky), __fmul_rn(r.Sy, Bkz));
  float Cx = __fsub_rn(comp(C, r.kx), __fmul_rn(r.Sx, Ckz)), Cy = __fsub_rn(comp(C, r.ky), __fmul_rn(r.Sy, Ckz));
  float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
  float Vv = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
  float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
  if (U == 0.0f || Vv == 0.0f || W == 0.0f) {
    U = (float)__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx));
    Vv = (float)__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx));
    W = (float)__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax));
  }
  if ((U < 0.0f || Vv < 0.0f || W < 0.0f) && (U > 0.0f || Vv > 0.0f || W > 0.0f)) return false;
  float det = __fadd_rn(__fadd_rn(U, Vv), W);
  if (det == 0.0f) return false;
  float T = __fmul_rn(U, __fmul_rn(r.Sz, Akz));
  T = __fadd_rn(T, __fmul_rn(Vv, __fmul_rn(r.Sz, Bkz)));
  T = __fadd_rn(T, __fmul_rn(W, __fmul_rn(r.Sz, Ckz)));
  t = __fdiv_rn(T, det);
  return true;
}

// ---------------------------------------------------------------------------
// Scene-level constants passed by value to kernels.
struct Light { V3 c, e1, e2, dl; };

struct Cam {
  V3 o;
  float k, cx, cy, dcam;
};

FR_DEV V3 camera_dir(const Cam& c, float sx, float sy) {
  return V3{__fsub_rn(__fmul_rn(sx, c.k), c.cx), __fsub_rn(c.cy, __fmul_rn(sy, c.k)), -1.0f};
}
FR_DEV V3 hit_point(V3 o, V3 d, float t) {
  return V3{__fadd_rn(o.x, __fmul_rn(t, d.x)), __fadd_rn(o.y, __fmul_rn(t, d.y)), __fadd_rn(o.z, __fmul_rn(t, d.z))};
}
FR_DEV V3 light_point(const Light& L, float side, float u2, float u3) {
  float a = __fmul_rn(__fsub_rn(u2, 0.5f), side), b = __fmul_rn(__fsub_rn(u3, 0.5f), side);
  return V3{__fadd_rn(__fadd_rn(L.c.x, __fmul_rn(a, L.e1.x)), __fmul_rn(b, L.e2.x)),
            __fadd_rn(__fadd_rn(L.c.y, __fmul_rn(a, L.e1.y)), __fmul_rn(b, L.e2.y)),
            __fadd_rn(__fadd_rn(L.c.z, __fmul_rn(a, L.e1.z)), __fmul_rn(b, L.e2.z))};
}
FR_DEV void project(const Cam& c, V3 p, float& sx, float& sy) {
  float q = __fsub_rn(c.dcam, p.z);
  float X = __fdiv_rn(p.x, q), Y = __fdiv_rn(p.y, q);
  sx = __fdiv_rn(__fadd_rn(X, c.cx), c.k);
  sy = __fdiv_rn(__fsub_rn(c.cy, Y), c.k);
}

// ---------------------------------------------------------------------------
// Bounding-volume hierarchy (binary; both child boxes stored in the parent).
// Node = 4 float4: (lo0.xyz, hi0.x) (hi0.yz, lo1.xy) (lo1.z, hi1.xyz) (child0, child1, -, -).
// child >= 0: internal node index; child < 0: leaf, ~child = first << 3 | (count - 1).
struct BVHView {
  const float4* nodes;   // [n_nodes * 4]
  int n_nodes;
};

// Normal cone (axis.xyz, half-angle in radians; >= pi means "any direction").
constexpr float CONE_FULL = 4.0f;

FR_DEV float4 cone_merge(float4 c1, float4 c2) {
  if (c1.w >= PI_F || c2.w >= PI_F) return make_float4(0, 0, 1, CONE_FULL);
  float d = c1.x * c2.x + c1.y * c2.y + c1.z * c2.z;
  float w = acosf(fminf(1.0f, fmaxf(-1.0f, d)));
  if (w + c2.w <= c1.w) return c1;
  if (w + c1.w <= c2.w) return c2;
  float th = 0.5f * (w + c1.w + c2.w);
  if (th >= PI_F) return make_float4(0, 0, 1, CONE_FULL);
  float rot = th - c1.w;             // rotate axis 1 toward axis 2 by rot
  float ax = c1.x, ay = c1.y, az = c1.z;
  if (w > 1e-6f) {
    float is = 1.0f / sinf(w), s1 = sinf(w - rot) * is, s2 = sinf(rot) * is;
    ax = c1.x * s1 + c2.x * s2; ay = c1.y * s1 + c2.y * s2; az = c1.z * s1 + c2.z * s2;
    float in = rsqrtf(ax * ax + ay * ay + az * az);
    ax *= in; ay *= in; az *= in;
  }
  return make_float4(ax, ay, az, th * 1.0001f + 1e-5f);   // slack for rounding
}

// Child code of an absent child (root of a hierarchy with a single leaf).
constexpr int EMPTY_CHILD = (int)0x80000000;
FR_HOST_DEV inline bool leaf_child(int c) { return c < 0; }
FR_DEV int leaf_first(int c) { return (~c) >> 3; }
FR_DEV int leaf_count(int c) { return ((~c) & 7) + 1; }

// Slab test of a ray against a box, one FMA per slab plane: t = lo * inv -
// oi with oi = o * inv.  Its rounding differs from (lo - o) * inv by about
// ulp(o inv), below the boxes' padding (pad_box: 1e-5 absolute) for scenes
// within 100 m of the origin.  NaN-safe: fminf/fmaxf drop NaN operands,
// which only widens the accepted interval (a ray parallel to an axis, inv =
// +-inf, may give NaN slab values for that axis, which then reject nothing).
FR_DEV V3 ray_oi(V3 o, V3 inv) { return V3{o.x * inv.x, o.y * inv.y, o.z * inv.z}; }
FR_DEV bool box_hit(V3 lo, V3 hi, V3 oi, V3 inv, float tmin, float tmax, float& tenter) {
  float tx0 = fmaf(lo.x, inv.x, -oi.x), tx1 = fmaf(hi.x, inv.x, -oi.x);
  float ty0 = fmaf(lo.y, inv.y, -oi.y), ty1 = fmaf(hi.y, inv.y, -oi.y);
  float tz0 = fmaf(lo.z, inv.z, -oi.z), tz1 = fmaf(hi.z, inv.z, -oi.z);
  float t0 = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
  float t1 = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  tenter = t0;
  return t0 <= t1;
}

// Node visits per traversal before the error flag is raised (default of
// fr_set_limits; a traversal of a valid hierarchy needs far fewer).
constexpr int DEFAULT_MAX_STEPS = 1 << 16;

struct Mesh {
  const float4* X;      // posed vertices [V] (w unused)
  const float4* ng;     // FP32 face normals [F] (decision form)
  const int4* tris;     // [F] (v0, v1, v2, -)
  const float4* tv;     // triangle vertices in BVH leaf order [F*3]; tv[3i].w = original face id bits
  BVHView bvh;
  int max_steps;        // node visits per traversal before ERR_STEPS
};

// ---------------------------------------------------------------------------
// Warp-cooperative traversal.  The 32 lanes of a warp trace their own rays
// through one shared walk of the hierarchy: a child is entered when any lane
// that is still searching hits its box (one ballot per child), each lane
// tests a leaf's triangles only if its own box test passed, and the walk
// ends when its stack is empty or no lane is searching.  Every lane ends with
// the result of its own ray (the closest hit with ties to the smaller face
// index, or whether any face crosses the segment), because a lane visits
// every node its own walk would visit and a decision taken on a triangle
// does not depend on the order in which triangles are tested.  Lanes
// without a ray take part with active = false.  All 32 lanes of the warp
// must call these functions together.
//
// The stack is warp-uniform and lives in registers: entry k in register k / 32
// of lane k % 32.
constexpr int WSTACK = 64;
struct WStack { int r0, r1, sp; };
FR_DEV void wpush(WStack& s, int v, int lane) {
  if (s.sp < 32) { if (lane == s.sp) s.r0 = v; }
  else if (lane == s.sp - 32) s.r1 = v;
  ++s.sp;
}
FR_DEV int wpop(WStack& s) {
  --s.sp;
  return s.sp < 32 ? __shfl_sync(0xffffffffu, s.r0, s.sp) : __shfl_sync(0xffffffffu, s.r1, s.sp - 32);
}

FR_DEV int closest_hit_warp(const Mesh& m, bool active, V3 o, V3 d, float& t_best, int* err,
                            unsigned long long* cnt) {
  const int lane = threadIdx.x & 31;
  RayPre rp = ray_pre(o, d);
  V3 inv = V3{1.0f / d.x, 1.0f / d.y, 1.0f / d.z};
  const V3 oi = ray_oi(o, inv);
  int best = -1;
  t_best = __int_as_float(0x7f800000);
  unsigned nvis = 0, ntri = 0;       // per walk; widened when added to the counters
  if (m.bvh.n_nodes == 0 || !__any_sync(0xffffffffu, active)) return -1;
  WStack st{0, 0, 0};
  int node = 0, steps = 0;
  while (true) {
    if (++steps > m.max_steps) { if (active) atomicOr(err, ERR_STEPS); break; }
    if (active) ++nvis;
    const float4* N = m.bvh.nodes + 4 * node;
    const float4 a = N[0], b = N[1], c = N[2];
    const int4 ch = *reinterpret_cast<const int4*>(N + 3);
    float te0 = 0.0f, te1 = 0.0f;
    const bool h0 = active && box_hit(V3{a.x, a.y, a.z}, V3{a.w, b.x, b.y}, oi, inv, 0.0f, t_best, te0);
    const bool h1 = active && box_hit(V3{b.z, b.w, c.x}, V3{c.y, c.z, c.w}, oi, inv, 0.0f, t_best, te1);
    const unsigned m0 = __ballot_sync(0xffffffffu, h0), m1 = __ballot_sync(0xffffffffu, h1);
    const unsigned mf = __ballot_sync(0xffffffffu, h0 && h1 && te1 < te0);
    // near child first, by the vote of the lanes that hit both
    const bool swap = 2 * __popc(mf) > __popc(m0 & m1);
    int next = -1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const bool second = (k == 1) != swap;                  // child slot taken at this step
      const int c2 = second ? ch.y : ch.x;
      const bool h = second ? h1 : h0;
      if ((second ? m1 : m0) == 0u || c2 == EMPTY_CHILD) continue;
      if (leaf_child(c2)) {
        const int f0 = leaf_first(c2), n = leaf_count(c2);
        for (int i = 0; i < n; ++i) {
          const float4* T = m.tv + 3 * (f0 + i);
          const float4 p0 = T[0], p1 = T[1], p2 = T[2];
          if (!h) continue;
          const int fid = __float_as_int(p0.w);
          float tt;
          ++ntri;
          if (tri_hit(rp, V3{p0.x, p0.y, p0.z}, V3{p1.x, p1.y, p1.z}, V3{p2.x, p2.y, p2.z}, tt) && tt > 0.0f) {
            if (tt < t_best || (tt == t_best && fid < best)) { t_best = tt; best = fid; }
          }
        }
      } else if (next < 0) {
        next = c2;
      } else {
        if (st.sp >= WSTACK) { if (active) atomicOr(err, ERR_STACK); goto done; }
        wpush(st, c2, lane);
      }
    }
    if (next >= 0) { node = next; continue; }
    if (st.sp == 0) break;
    node = wpop(st);
  }
done:
  if (cnt && active) { atomicAdd(cnt, (unsigned long long)nvis); atomicAdd(cnt + 1, (unsigned long long)ntri); }
  return best;
}

// Any face other than `skip` crossed by x + t w, t in (tlo, thi)?  A lane
// stops searching at its first hit; the walk ends when no lane searches.
// Kept out of line: the kernels call it from several light loops, and one
// copy of the walk keeps their code within the instruction cache (measured:
// the fused render + interior kernel 5.36 -> 4.07 ms on the full workload).
static __device__ __noinline__ bool occluded_warp(const Mesh& m, bool active, V3 x, V3 w, int skip, float tlo, float thi, int* err,
                          unsigned long long* cnt) {
  const int lane = threadIdx.x & 31;
  RayPre rp = ray_pre(x, w);
  V3 inv = V3{1.0f / w.x, 1.0f / w.y, 1.0f / w.z};
  const V3 oi = ray_oi(x, inv);
  bool hit = false, live = active;
  unsigned nvis = 0, ntri = 0;       // per walk; widened when added to the counters
  if (m.bvh.n_nodes == 0 || !__any_sync(0xffffffffu, live)) return false;
  WStack st{0, 0, 0};
  int node = 0, steps = 0;
  while (true) {
    if (++steps > m.max_steps) { if (live) atomicOr(err, ERR_STEPS); break; }
    if (live) ++nvis;
    const float4* N = m.bvh.nodes + 4 * node;
    const float4 a = N[0], b = N[1], c = N[2];
    const int4 ch = *reinterpret_cast<const int4*>(N + 3);
    float te0, te1;
    const bool h0 = live && box_hit(V3{a.x, a.y, a.z}, V3{a.w, b.x, b.y}, oi, inv, 0.0f, thi, te0);
    const bool h1 = live && box_hit(V3{b.z, b.w, c.x}, V3{c.y, c.z, c.w}, oi, inv, 0.0f, thi, te1);
    const unsigned m0 = __ballot_sync(0xffffffffu, h0), m1 = __ballot_sync(0xffffffffu, h1);
    int next = -1;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int c2 = k ? ch.y : ch.x;
      const bool h = k ? h1 : h0;
      if ((k ? m1 : m0) == 0u || c2 == EMPTY_CHILD) continue;
      if (leaf_child(c2)) {
        const int f0 = leaf_first(c2), n = leaf_count(c2);
        for (int i = 0; i < n; ++i) {
          const float4* T = m.tv + 3 * (f0 + i);
          const float4 p0 = T[0], p1 = T[1], p2 = T[2];
          if (!(h && live)) continue;
          if (__float_as_int(p0.w) == skip) continue;
          float tt;
          ++ntri;
          if (tri_hit(rp, V3{p0.x, p0.y, p0.z}, V3{p1.x, p1.y, p1.z}, V3{p2.x, p2.y, p2.z}, tt) && tt > tlo &&
              tt < thi) {
            hit = true;
            live = false;
          }
        }
      } else if (next < 0) {
        next = c2;
      } else {
        if (st.sp >= WSTACK) { if (live) atomicOr(err, ERR_STACK); goto done; }
        wpush(st, c2, lane);
      }
    }
    if (!__any_sync(0xffffffffu, live)) break;
    if (next >= 0) { node = next; continue; }
    if (st.sp == 0) break;
    node = wpop(st);
  }
done:
  if (cnt && active) { atomicAdd(cnt, (unsigned long long)nvis); atomicAdd(cnt + 1, (unsigned long long)ntri); }
  return hit;
}

FR_DEV int face_flip(const Mesh& m, int f, V3 d) {
  float4 n = m.ng[f];
  return dot3r(V3{n.x, n.y, n.z}, d) > 0.0f ? -1 : 1;
}

// Does face f (>= 0; -1 gives false) cross the segment of rp, t in (tlo,
// thi)?  The any-hit walk's own test on the same vertices (tv holds each
// face's vertices in the order of tris).
FR_DEV bool face_blocks(const Mesh& m, int f, const RayPre& rp, float tlo, float thi) {
  if (f < 0) return false;
  const int4 t = m.tris[f];
  float tt;
  return tri_hit(rp, v3(m.X[t.x]), v3(m.X[t.y]), v3(m.X[t.z]), tt) && tt > tlo && tt < thi;
}

// Visibility of light point y from hit point x on face f seen from side
// `flip`, for a whole warp (occluded_warp); lanes with active = false take
// part and get false.
FR_DEV bool visible_warp(const Mesh& m, bool active, V3 x, V3 y, int f, int flip, float tmin, int* err,
                         unsigned long long* cnt) {
  V3 w = sub3r(y, x);
  bool gate = false;
  if (active) {
    float4 n = m.ng[f];
    float g = dot3r(V3{n.x, n.y, n.z}, w);
    gate = flip > 0 ? g > 0.0f : g < 0.0f;
  }
  return !occluded_warp(m, gate, x, w, f, tmin, __fsub_rn(1.0f, tmin), err, cnt) && gate;
}

// ---------------------------------------------------------------------------
// Surface at a hit (values).
struct Surf {
  V3 x, ns, wo, rho;
  float b0, b1, b2;
  float u, v;
  float inv_nlen;   // 1 / |interpolated normal|
  V3 nraw;          // interpolated (unnormalised, unflipped) normal
  int flip;
};

// Bilinear specular-map lookup with clamp to edge, texel centres at (k+0.5)/32.
FR_DEV float cspec_lookup(const float* C, float u, float v, int* idx, float* w, float& fu, float& fv) {
  float su = u * (float)CS - 0.5f, sv = v * (float)CS - 0.5f;
  float fu0 = floorf(su), fv0 = floorf(sv);
  fu = su - fu0; fv = sv - fv0;
  int iu = (int)fu0, iv = (int)fv0;
  int iu0 = min(max(iu, 0), CS - 1), iu1 = min(max(iu + 1, 0), CS - 1);
  int iv0 = min(max(iv, 0), CS - 1), iv1 = min(max(iv + 1, 0), CS - 1);
  idx[0] = iv0 * CS + iu0; idx[1] = iv0 * CS + iu1; idx[2] = iv1 * CS + iu0; idx[3] = iv1 * CS + iu1;
  w[0] = (1.0f - fu) * (1.0f - fv); w[1] = fu * (1.0f - fv); w[2] = (1.0f - fu) * fv; w[3] = fu * fv;
  return w[0] * C[idx[0]] + w[1] * C[idx[1]] + w[2] * C[idx[2]] + w[3] * C[idx[3]];
}

// Shading of one light: returns h = l (x) f_r cos_x cos_y / d^2 (RGB) and, if
// requested, the pieces the adjoint needs.
struct ShadeOut {
  V3 h;       // RGB integrand
  float geo;  // cos_x cos_y / d^2
  float spec; // specular factor before c_s
  bool active;
};

// BRDF readings (the Face Modeling paragraph names Cook-Torrance without its
// terms): model 0 = Beckmann D with the Cook-Torrance V-cavity G, model 1 =
// GGX (Trowbridge-Reitz) D with the separable Smith G of GGX; fresnel 0 =
// F folded into c_spec, 1 = Schlick's F with c_spec as the reflectance at
// normal incidence.  m is the roughness (Beckmann m, or GGX alpha).
struct Brdf {
  float m;
  int model, fresnel;
};

// Reciprocal for value arithmetic (radiance and derivatives, never a
// decision): the hardware's approximate reciprocal, within 2 ulp for the
// normal-range arguments of the shading formulas.  The formulas below divide
// through these reciprocals, a few per light instead of one exact division
// per quotient.
FR_DEV float rcp(float x) { return __fdividef(1.0f, x); }

// Smith masking of GGX for one direction at cos c: 2c / (c + sqrt(a2 + (1 - a2) c^2)).
FR_DEV float smith_g1_ggx(float c, float a2, float& r) {
  r = sqrtf(a2 + (1.0f - a2) * c * c);
  return 2.0f * c * rcp(c + r);
}

FR_DEV ShadeOut shade_light(const Surf& S, float cs, V3 l, V3 y, V3 dl, const Brdf& b) {
  ShadeOut o;
  o.active = false;
  o.h = V3{0, 0, 0};
  o.geo = 0; o.spec = 0;
  V3 w = y - S.x;
  float d2 = dot(w, w);
  const float ir = rsqrtf(d2);
  V3 wi = w * ir;
  float ci = dot(S.ns, wi);
  if (!(ci > 0.0f)) return o;
  float cy = dot(dl, wi);
  if (!(cy > 0.0f)) return o;
  float co = dot(S.ns, S.wo);
  float spec = 0.0f, F = cs;
  if (co > 0.0f) {
    V3 h = normalize(wi + S.wo);
    float ch = dot(S.ns, h), oh = dot(S.wo, h);   // both > 0: wi and wo lie on the side of ns
    float ch2 = ch * ch;
    const float m = b.m, a2 = m * m, ia2 = rcp(a2);
    float D, G;
    if (b.model == 0) {
      const float ich2 = rcp(ch2);
      const float tan2 = (1.0f - ch2) * ich2;
      D = __expf(-tan2 * ia2) * ((1.0f / PI_F) * ia2 * ich2 * ich2);
      G = fminf(1.0f, 2.0f * ch * rcp(oh) * fminf(co, ci));
    } else {
      float t = ch2 * (a2 - 1.0f) + 1.0f, ri, ro;
      const float it = rcp(t);
      D = a2 * (1.0f / PI_F) * it * it;
      G = smith_g1_ggx(ci, a2, ri) * smith_g1_ggx(co, a2, ro);
    }
    spec = D * G * rcp(4.0f * ci * co);
    if (b.fresnel) {
      float q = 1.0f - oh, q2 = q * q;
      F = cs + (1.0f - cs) * q2 * q2 * q;
    }
  }
  float geo = ci * cy * (ir * ir);
  float sp = F * spec;
  o.h = V3{l.x * (S.rho.x * (1.0f / PI_F) + sp) * geo, l.y * (S.rho.y * (1.0f / PI_F) + sp) * geo,
           l.z * (S.rho.z * (1.0f / PI_F) + sp) * geo};
  o.geo = geo;
  o.spec = spec;
  o.active = true;
  return o;
}

}  // namespace fr
