// Device functions of the Monte-Carlo render and its gradient, shared by the
// single-image kernels (render.cu) and the batched persistent kernel
// (batch.cu).
#pragma once

#include "kernels.cuh"

namespace fr {

FR_DEV Surf surface(const RenderArgs& a, int f, V3 o, V3 d, int flip) {
  int4 t = a.mesh.tris[f];
  V3 P0 = v3(a.mesh.X[t.x]), P1 = v3(a.mesh.X[t.y]), P2 = v3(a.mesh.X[t.z]);
  V3 e1 = P1 - P0, e2 = P2 - P0, s = o - P0;
  V3 pv = cross(d, e2);
  float inv = 1.0f / dot(e1, pv);
  V3 qv = cross(s, e1);
  Surf S;
  S.b1 = dot(s, pv) * inv;
  S.b2 = dot(d, qv) * inv;
  S.b0 = 1.0f - S.b1 - S.b2;
  // hit point from the barycentrics: its error is relative to the triangle,
  // not to the camera distance
  S.x = P0 + e1 * S.b1 + e2 * S.b2;
  V3 N0 = v3(a.nrm[t.x]), N1 = v3(a.nrm[t.y]), N2 = v3(a.nrm[t.z]);
  S.nraw = N0 * S.b0 + N1 * S.b1 + N2 * S.b2;
  S.inv_nlen = rsqrtf(dot(S.nraw, S.nraw));
  S.ns = S.nraw * (S.inv_nlen * (float)flip);
  S.wo = normalize(-d);
  V3 A0 = v3(a.alb[t.x]), A1 = v3(a.alb[t.y]), A2 = v3(a.alb[t.z]);
  S.rho = A0 * S.b0 + A1 * S.b1 + A2 * S.b2;
  float2 u0 = a.uv[t.x], u1 = a.uv[t.y], u2 = a.uv[t.z];
  S.u = S.b0 * u0.x + S.b1 * u1.x + S.b2 * u2.x;
  S.v = S.b0 * u0.y + S.b1 * u1.y + S.b2 * u2.y;
  S.flip = flip;
  return S;
}

FR_DEV V3 light_rgb(const RenderArgs& a, int j) {
  const float* l = a.lights_dev + 3 * j;
  return V3{__ldg(l), __ldg(l + 1), __ldg(l + 2)};
}
// A light is off when all three channels are exactly zero.
FR_DEV bool light_on(const RenderArgs& a, int j) {
  V3 l = light_rgb(a, j);
  return l.x != 0.0f || l.y != 0.0f || l.z != 0.0f;
}

// Per-sample auxiliary features for the denoiser (means over spp are taken
// by the caller): shading normal, diffuse albedo, specular albedo, distance
// to the camera / d_cam, fraction of lit lights that are visible, hit flag.
struct SampleAux {
  V3 n, rho;
  float cs, depth, vis, hit;
};

// One-sample radiance along a camera ray, lights that are on only.
// hit (optional) receives the primary hit: face (or -1) and the bits of t;
// vis (optional) bit j = light j is on and its light point is visible.
// All 32 lanes of the warp call together (warp-cooperative traversal,
// common.cuh); lanes without a ray pass active = false and get 0.
FR_DEV V3 radiance(const RenderArgs& a, V3 o, V3 d, int tag, uint32_t c0, uint32_t c1, unsigned long long* cnt,
                   SampleAux* aux = nullptr, int2* hit = nullptr, uint32_t* vis = nullptr, bool active = true) {
  float t;
  int f;
  f = closest_hit_warp(a.mesh, active, o, d, t, a.err, cnt);
  if (hit) *hit = make_int2(f, __float_as_int(t));
  if (vis) *vis = 0u;
  const bool lit = f >= 0;
  int flip = 1;
  V3 x32{0, 0, 0};
  Surf S;
  float cs = 0.0f;
  if (lit) {
    flip = face_flip(a.mesh, f, d);
    x32 = hit_point(o, d, t);
    S = surface(a, f, o, d, flip);
    int idx[4];
    float w[4], fu, fv;
    cs = cspec_lookup(a.cspec, S.u, S.v, idx, w, fu, fv);
  }
  V3 L{0, 0, 0};
  const float area = a.side * a.side;
  int n_on = 0, n_vis = 0;
  for (int j = 0; j < a.n_lights; ++j) {
    if (!light_on(a, j)) continue;
    ++n_on;
    U4 q = philox(a.seed, a.iter, c0, c1, (uint32_t)(tag << 8 | j), 0);
    V3 y = light_point(a.lights[j], a.side, unitf(q.x), unitf(q.y));
    bool seen;
    seen = visible_warp(a.mesh, lit, x32, y, f, flip, a.tmin, a.err, cnt);
    if (!seen) continue;
    ++n_vis;
    if (vis) *vis |= 1u << j;
    ShadeOut sh = shade_light(S, cs, light_rgb(a, j), y, a.lights[j].dl, a.brdf);
    L += sh.h * area;
  }
  if (aux && lit) {
    aux->n = S.ns; aux->rho = S.rho; aux->cs = cs;
    aux->depth = t * len(d) / a.cam.dcam;
    aux->vis = n_on ? (float)n_vis / (float)n_on : 0.0f;
    aux->hit = 1.0f;
  }
  return L;
}

// Camera ray of sample s of pixel (px, py).
FR_DEV V3 sample_dir(const RenderArgs& a, int px, int py, int s, uint32_t& pix) {
  pix = (uint32_t)(py * a.W + px);
  U4 q = philox(a.seed, a.iter, pix, (uint32_t)s, (uint32_t)(TAG_CAMERA << 8), 0);
  float sx = __fadd_rn((float)px, unitf(q.x));
  float sy = __fadd_rn((float)py, unitf(q.y));
  return camera_dir(a.cam, sx, sy);
}




// ---------------------------------------------------------------------------
// Interior adjoint

// Reverse-mode of shade_light for one light.  G = adjoint RGB times area/spp.
FR_DEV void shade_light_bwd(const Surf& S, float cs, V3 l, V3 y, V3 dl, const Brdf& bd, V3 G, V3& g_x, V3& g_ns,
                            V3& g_rho, float& g_cs, V3& g_l) {
  V3 w = y - S.x;
  float d2 = dot(w, w);
  float ir = rsqrtf(d2);
  const float id2 = ir * ir;                 // 1 / d2
  V3 wi = w * ir;
  float ci = dot(S.ns, wi);
  if (!(ci > 0.0f)) return;
  float cy = dot(dl, wi);
  if (!(cy > 0.0f)) return;
  float co = dot(S.ns, S.wo);
  const float m = bd.m, a2 = m * m, ia2 = rcp(a2);
  float spec = 0.0f, D = 0.0f, Gf = 0.0f, ch = 0.0f, oh = 0.0f, g1 = 0.0f, g2 = 0.0f, ihl = 1.0f;
  float ich = 0.0f, ioh = 0.0f, ik4 = 0.0f, it = 1.0f;
  float G1i = 1.0f, G1o = 1.0f, ri = 1.0f, ro = 1.0f, F = cs, q = 0.0f, q4 = 0.0f;
  int branch = 0;
  V3 h{0, 0, 0};
  if (co > 0.0f) {
    V3 hv = wi + S.wo;
    ihl = rsqrtf(dot(hv, hv));               // 1 / |wi + wo|
    h = hv * ihl;
    ch = dot(S.ns, h);                       // ch, oh > 0: wi and wo lie on the side of ns
    oh = dot(S.wo, h);
    ich = rcp(ch);
    ioh = rcp(oh);
    float ch2 = ch * ch;
    if (bd.model == 0) {
      const float ich2 = ich * ich;
      float tan2 = (1.0f - ch2) * ich2;
      D = __expf(-tan2 * ia2) * ((1.0f / PI_F) * ia2 * ich2 * ich2);
      g1 = 2.0f * ch * co * ioh;
      g2 = 2.0f * ch * ci * ioh;
      float inner = g1 <= g2 ? g1 : g2;
      if (1.0f <= inner) { Gf = 1.0f; branch = 0; }
      else { Gf = inner; branch = g1 <= g2 ? 1 : 2; }
    } else {
      float t = ch2 * (a2 - 1.0f) + 1.0f;
      it = rcp(t);
      D = a2 * (1.0f / PI_F) * it * it;
      G1i = smith_g1_ggx(ci, a2, ri);
      G1o = smith_g1_ggx(co, a2, ro);
      Gf = G1i * G1o;
    }
    ik4 = rcp(4.0f * ci * co);
    spec = D * Gf * ik4;
    if (bd.fresnel) {
      q = 1.0f - oh;
      float q2 = q * q;
      q4 = q2 * q2;
      F = cs + (1.0f - cs) * q4 * q;
    }
  }
  float geo = ci * cy * id2;
  const float ip = 1.0f / PI_F;
  const float sp = F * spec;
  V3 Fr{S.rho.x * ip + sp, S.rho.y * ip + sp, S.rho.z * ip + sp};
  g_l += V3{G.x * Fr.x * geo, G.y * Fr.y * geo, G.z * Fr.z * geo};
  V3 s{G.x * l.x, G.y * l.y, G.z * l.z};
  g_rho += s * (geo * ip);
  float Ssum = (s.x + s.y + s.z) * geo;
  // sp = F spec with F = c_s (folded) or c_s + (1 - c_s) q^5, q = 1 - oh
  g_cs += Ssum * spec * (bd.fresnel ? 1.0f - q4 * q : 1.0f);
  float d_spec = Ssum * F;
  float d_geo = s.x * Fr.x + s.y * Fr.y + s.z * Fr.z;
  float d_ci = d_geo * cy * id2;
  float d_cy = d_geo * ci * id2;
  float d_d2 = -d_geo * geo * id2;
  float d_co = 0.0f;
  V3 d_ns{0, 0, 0}, d_wi{0, 0, 0};
  if (co > 0.0f && Ssum != 0.0f) {
    float d_D = d_spec * Gf * ik4, d_G = d_spec * D * ik4;
    // spec / ci = D Gf / (4 ci^2 co) and spec / co likewise
    d_ci -= d_spec * spec * (4.0f * co * ik4);
    d_co -= d_spec * spec * (4.0f * ci * ik4);
    float d_ch = 0.0f, d_oh = bd.fresnel ? -5.0f * Ssum * spec * (1.0f - cs) * q4 : 0.0f;
    if (bd.model == 0) {
      if (branch == 1) { d_ch += d_G * 2.0f * co * ioh; d_co += d_G * 2.0f * ch * ioh; d_oh -= d_G * g1 * ioh; }
      else if (branch == 2) { d_ch += d_G * 2.0f * ci * ioh; d_ci += d_G * 2.0f * ch * ioh; d_oh -= d_G * g2 * ioh; }
      d_ch += d_D * D * (2.0f * ia2 * ich * ich * ich - 4.0f * ich);
    } else {
      // Smith: dG1/dc = 2 a2 / (r (c + r)^2); GGX: dD/dch = -4 D ch (a2 - 1) / t
      d_ci += d_G * G1o * 2.0f * a2 * rcp(ri * (ci + ri) * (ci + ri));
      d_co += d_G * G1i * 2.0f * a2 * rcp(ro * (co + ro) * (co + ro));
      d_ch += d_D * D * (-4.0f * ch * (a2 - 1.0f) * it);
    }
    d_ns += h * d_ch;
    V3 d_h = S.ns * d_ch + S.wo * d_oh;
    d_wi += (d_h - h * dot(d_h, h)) * ihl;
  }
  d_ns += wi * d_ci + S.wo * d_co;
  d_wi += S.ns * d_ci + dl * d_cy;
  V3 d_w = (d_wi - wi * dot(d_wi, wi)) * ir + w * (2.0f * d_d2);
  g_x -= d_w;
  g_ns += d_ns;
}

FR_DEV void atomic_add3(float4* p, V3 v) {
  atomicAdd(p, make_float4(v.x, v.y, v.z, 0.0f));
}

// Adjoint of the hit point x = o + t d with respect to the hit triangle's
// vertices (ray fixed), plus barycentric adjoints g_b1, g_b2 (b0 = 1-b1-b2
// already folded in).  Scatters b_k * lambda into dX.
FR_DEV void cross64(const double* a, const double* b, double* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

// Hit point of the ray (o, d) on face f in FP64 (Moller-Trumbore on the FP32
// vertices): accurate along the surface even for grazing rays.
FR_DEV void hit_point64(const RenderArgs& a, int f, V3 o, V3 d, double* x) {
  int4 t = a.mesh.tris[f];
  float4 p0 = a.mesh.X[t.x], p1 = a.mesh.X[t.y], p2 = a.mesh.X[t.z];
  double e1[3] = {(double)p1.x - p0.x, (double)p1.y - p0.y, (double)p1.z - p0.z};
  double e2[3] = {(double)p2.x - p0.x, (double)p2.y - p0.y, (double)p2.z - p0.z};
  double dd[3] = {d.x, d.y, d.z};
  double s[3] = {(double)o.x - p0.x, (double)o.y - p0.y, (double)o.z - p0.z};
  double pv[3], qv[3];
  cross64(dd, e2, pv);
  cross64(s, e1, qv);
  double inv = 1.0 / (e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2]);
  double b1 = (s[0] * pv[0] + s[1] * pv[1] + s[2] * pv[2]) * inv;
  double b2 = (dd[0] * qv[0] + dd[1] * qv[1] + dd[2] * qv[2]) * inv;
  x[0] = (double)p0.x + b1 * e1[0] + b2 * e2[0];
  x[1] = (double)p0.y + b1 * e1[1] + b2 * e2[1];
  x[2] = (double)p0.z + b1 * e1[2] + b2 * e2[2];
}

// The 3x3 solve is ill-conditioned for grazing hits (det -> 0), so it runs in
// FP64 (a few dozen operations per sample).
FR_DEV void hit_adjoint(const RenderArgs& a, int f, V3 d, const Surf& S, V3 g_x, float g_b1, float g_b2,
                        float4* dX) {
  int4 t = a.mesh.tris[f];
  float4 p0 = a.mesh.X[t.x], p1 = a.mesh.X[t.y], p2 = a.mesh.X[t.z];
  double e1x = (double)p1.x - p0.x, e1y = (double)p1.y - p0.y, e1z = (double)p1.z - p0.z;
  double e2x = (double)p2.x - p0.x, e2y = (double)p2.y - p0.y, e2z = (double)p2.z - p0.z;
  double dx = d.x, dy = d.y, dz = d.z;
  double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  double det = dx * nx + dy * ny + dz * nz;
  double gt = (double)g_x.x * dx + (double)g_x.y * dy + (double)g_x.z * dz;
  double b1 = g_b1, b2 = g_b2;
  // lambda = (n g_t + (d x e2) g_b1 + (e1 x d) g_b2) / det
  double lx = nx * gt + (dy * e2z - dz * e2y) * b1 + (e1y * dz - e1z * dy) * b2;
  double ly = ny * gt + (dz * e2x - dx * e2z) * b1 + (e1z * dx - e1x * dz) * b2;
  double lz = nz * gt + (dx * e2y - dy * e2x) * b1 + (e1x * dy - e1y * dx) * b2;
  double inv = 1.0 / det;
  V3 lam{(float)(lx * inv), (float)(ly * inv), (float)(lz * inv)};
  atomic_add3(dX + t.x, lam * S.b0);
  atomic_add3(dX + t.y, lam * S.b1);
  atomic_add3(dX + t.z, lam * S.b2);
}

// Interior adjoint of one camera sample with primary hit (f, t) on ray d:
// every light (for dL/dl_j), shading, normals, albedo, specular map and the
// hit point, with the sample's decisions held fixed.  sC and sL are the
// block's shared accumulators of the specular-map and light gradients.
// vis (optional): the forward's visibility bits of this sample (radiance
// with the light tag): lights that are on take their shadow decision from
// it, the others trace their shadow ray.
// All 32 lanes call together; lanes without a sample pass active = false.
FR_DEV void interior_sample(const RenderArgs& a, const GradBufs& gb, float* sC, float* sL, uint32_t pix, int s,
                            V3 d, int f, float t, V3 dimg, unsigned long long* cnt, const uint32_t* vis = nullptr,
                            bool active = true) {
  const int spp = a.spp;
  int flip = 1;
  V3 x32{0, 0, 0};
  Surf S;
  int idx[4] = {0, 0, 0, 0};
  float w[4] = {0, 0, 0, 0}, fu = 0.0f, fv = 0.0f;
  float cs = 0.0f;
  if (active) {
    flip = face_flip(a.mesh, f, d);
    x32 = hit_point(a.cam.o, d, t);
    S = surface(a, f, a.cam.o, d, flip);
    cs = cspec_lookup(a.cspec, S.u, S.v, idx, w, fu, fv);
  }
  const float scale = a.side * a.side / (float)spp;
  V3 G = dimg * scale;
  V3 g_x{0, 0, 0}, g_ns{0, 0, 0}, g_rho{0, 0, 0};
  float g_cs = 0.0f;
  for (int j = 0; j < a.n_lights; ++j) {
    U4 q = philox(a.seed, a.iter, pix, (uint32_t)s, (uint32_t)(TAG_LIGHT << 8 | j), 0);
    V3 y = light_point(a.lights[j], a.side, unitf(q.x), unitf(q.y));
    bool seen;
    if (vis && light_on(a, j)) seen = active && ((*vis >> j) & 1u) != 0u;
    else seen = visible_warp(a.mesh, active, x32, y, f, flip, a.tmin, a.err, cnt);
    if (!seen) continue;
    V3 g_l{0, 0, 0};
    shade_light_bwd(S, cs, light_rgb(a, j), y, a.lights[j].dl, a.brdf, G, g_x, g_ns, g_rho, g_cs, g_l);
    atomicAdd(&sL[3 * j], g_l.x);
    atomicAdd(&sL[3 * j + 1], g_l.y);
    atomicAdd(&sL[3 * j + 2], g_l.z);
  }
  if (!active) return;
  int4 tri = a.mesh.tris[f];
  // shading normal: ns = flip * n / |n|
  V3 nh = S.nraw * S.inv_nlen;
  V3 dnh = g_ns * (float)flip;
  V3 g_n = (dnh - nh * dot(nh, dnh)) * S.inv_nlen;
  V3 N0 = v3(a.nrm[tri.x]), N1 = v3(a.nrm[tri.y]), N2 = v3(a.nrm[tri.z]);
  V3 A0 = v3(a.alb[tri.x]), A1 = v3(a.alb[tri.y]), A2 = v3(a.alb[tri.z]);
  atomic_add3(gb.dN + tri.x, g_n * S.b0);
  atomic_add3(gb.dN + tri.y, g_n * S.b1);
  atomic_add3(gb.dN + tri.z, g_n * S.b2);
  atomic_add3(gb.dA + tri.x, g_rho * S.b0);
  atomic_add3(gb.dA + tri.y, g_rho * S.b1);
  atomic_add3(gb.dA + tri.z, g_rho * S.b2);
  float gb0 = dot(N0, g_n) + dot(A0, g_rho);
  float gb1 = dot(N1, g_n) + dot(A1, g_rho);
  float gb2 = dot(N2, g_n) + dot(A2, g_rho);
  // specular map
  if (g_cs != 0.0f) {
    for (int k = 0; k < 4; ++k) atomicAdd(&sC[idx[k]], w[k] * g_cs);
    const float* C = a.cspec;
    float C0 = C[idx[0]], C1 = C[idx[1]], C2 = C[idx[2]], C3 = C[idx[3]];
    float dfu = g_cs * (-(1.0f - fv) * C0 + (1.0f - fv) * C1 - fv * C2 + fv * C3);
    float dfv = g_cs * (-(1.0f - fu) * C0 - fu * C1 + (1.0f - fu) * C2 + fu * C3);
    float du = dfu * (float)CS, dv = dfv * (float)CS;
    float2 u0 = a.uv[tri.x], u1 = a.uv[tri.y], u2 = a.uv[tri.z];
    gb0 += u0.x * du + u0.y * dv;
    gb1 += u1.x * du + u1.y * dv;
    gb2 += u2.x * du + u2.y * dv;
  }
  hit_adjoint(a, f, d, S, g_x, gb1 - gb0, gb2 - gb0, gb.dX);
}


// ---------------------------------------------------------------------------
// Primary-visibility edges

// Edge sample tid (Philox keys: pixel tid / spp, sample tid % spp) of the
// primary-visibility term.  d_image is read through L2 (__ldcg): in the batched launch another
// block of the same launch wrote it.
// All 32 lanes call together; lanes without a sample pass active = false.
FR_DEV void pedge_sample(const RenderArgs& a, const GradBufs& gb, long long tid, unsigned long long* cnt,
                         bool active = true) {
  const int nS = *a.n_sil;
  if (nS <= 0) return;                          // uniform
  if (!active) tid = 0;
  uint32_t pix = (uint32_t)(tid / a.spp);
  int s = (int)(tid - (long long)pix * a.spp);
  // Systematic sampling of the silhouette edges taken as one interval
  // [0, nS) (edge k = [k, k + 1)): sample tid at z = (tid + xi0) nS / N with
  // one uniform offset xi0 per launch, formed in FP64 (add, multiply, divide);
  // (nS / N) sum f(z) is an unbiased estimate of the edge integrals, and
  // neighbouring threads walk along one edge (coherent rays).
  U4 q0 = philox(a.seed, a.iter, 0u, 0u, (uint32_t)(TAG_PEDGE_OFFSET << 8), 0);
  const double xi0 = (double)q0.x * 2.3283064365386963e-10;            // 2^-32
  const double n_s = (double)((long long)a.W * a.H * a.spp);
  const double zt = __ddiv_rn(__dmul_rn(__dadd_rn((double)tid, xi0), (double)nS), n_s);
  int k = (int)floor(zt);
  if (k > nS - 1) k = nS - 1;
  float u = __double2float_rn(__dsub_rn(zt, (double)k));
  int4 E = a.edges_canon[a.sil[k]];
  V3 A = v3(a.mesh.X[E.x]), B = v3(a.mesh.X[E.y]);
  float ax, ay, bx, by;
  project(a.cam, A, ax, ay);
  project(a.cam, B, bx, by);
  float ex = __fsub_rn(bx, ax), ey = __fsub_rn(by, ay);
  float mx = __fadd_rn(ax, __fmul_rn(u, ex)), my = __fadd_rn(ay, __fmul_rn(u, ey));
  float fx = floorf(mx), fy = floorf(my);
  bool ok = active && fx >= 0.0f && fx < (float)a.W && fy >= 0.0f && fy < (float)a.H;
  V3 dimg{0, 0, 0};
  if (ok) {
    const float* dI = gb.d_image + 3 * ((size_t)(int)fy * a.W + (int)fx);
    dimg = V3{__ldcg(dI), __ldcg(dI + 1), __ldcg(dI + 2)};
  }
  ok = ok && !(dimg.x == 0.0f && dimg.y == 0.0f && dimg.z == 0.0f);
  float L2 = __fmul_rn(ex, ex);
  L2 = __fadd_rn(L2, __fmul_rn(ey, ey));
  float Ln = __fsqrt_rn(L2);
  ok = ok && Ln != 0.0f;
  if (!ok) Ln = 1.0f;
  float nx = __fdiv_rn(-ey, Ln), ny = __fdiv_rn(ex, Ln);
  float e = a.eps_pedge;
  V3 dp = camera_dir(a.cam, __fadd_rn(mx, __fmul_rn(e, nx)), __fadd_rn(my, __fmul_rn(e, ny)));
  V3 dm = camera_dir(a.cam, __fsub_rn(mx, __fmul_rn(e, nx)), __fsub_rn(my, __fmul_rn(e, ny)));
  V3 fp = radiance(a, a.cam.o, dp, TAG_PEDGE_LIGHT, pix, (uint32_t)s, cnt, nullptr, nullptr, nullptr, ok);
  V3 fm = radiance(a, a.cam.o, dm, TAG_PEDGE_LIGHT, pix, (uint32_t)s, cnt, nullptr, nullptr, nullptr, ok);
  if (!ok) return;
  float delta = dot(dimg, fm - fp);
  if (delta == 0.0f) return;
  float w = delta * (float)nS / ((float)a.W * (float)a.H * (float)a.spp);
  const float kc = a.cam.k;
  // screen edge vector from 3D differences (accurate for short edges)
  float qa = a.cam.dcam - A.z, qb = a.cam.dcam - B.z;
  V3 BA = B - A;
  float iq = 1.0f / (qa * qb * kc);
  float evx = (BA.x * qa + A.x * BA.z) * iq;
  float evy = -(BA.y * qa + A.y * BA.z) * iq;
  float gmx = -evy * w, gmy = evx * w;     // w * R90(e)
  // adjoint of the screen projection for each endpoint
  {
    float c = 1.0f - u;
    float gx = gmx * c, gy = gmy * c;
    atomic_add3(gb.dX + E.x, V3{gx / (kc * qa), -gy / (kc * qa), (gx * A.x - gy * A.y) / (kc * qa * qa)});
  }
  {
    float gx = gmx * u, gy = gmy * u;
    atomic_add3(gb.dX + E.y, V3{gx / (kc * qb), -gy / (kc * qb), (gx * B.x - gy * B.y) / (kc * qb * qb)});
  }
}


// ---------------------------------------------------------------------------
// Shadow-boundary edges

// Clip the edge parameter interval to the part whose central projection from
// x lands in the light square (decision form).
FR_DEV bool shadow_clip(V3 A, V3 B, V3 x, const Light& L, float hs, float kappa, float& t0, float& t1) {
  V3 xc = sub3r(x, L.c);
  float al1 = dot3r(xc, L.e1), al2 = dot3r(xc, L.e2);
  float D = -dot3r(xc, L.dl);
  float ca[5], cb[5];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    V3 q = sub3r(e == 0 ? A : B, x);
    float h = dot3r(q, L.dl), s1 = dot3r(q, L.e1), s2 = dot3r(q, L.e2);
    float n1 = __fadd_rn(__fmul_rn(al1, h), __fmul_rn(s1, D));
    float n2 = __fadd_rn(__fmul_rn(al2, h), __fmul_rn(s2, D));
    float hh = __fmul_rn(hs, h);
    float* cc = e == 0 ? ca : cb;
    cc[0] = __fsub_rn(h, kappa);
    cc[1] = __fsub_rn(hh, n1);
    cc[2] = __fadd_rn(hh, n1);
    cc[3] = __fsub_rn(hh, n2);
    cc[4] = __fadd_rn(hh, n2);
  }
  float lo = 0.0f, hi = 1.0f;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    float p = ca[k], r = cb[k];
    if (p < 0.0f && r < 0.0f) return false;
    if (p < 0.0f) { float rr = __fdiv_rn(p, __fsub_rn(p, r)); if (rr > lo) lo = rr; }
    else if (r < 0.0f) { float rr = __fdiv_rn(p, __fsub_rn(p, r)); if (rr < hi) hi = rr; }
  }
  t0 = lo; t1 = hi;
  return lo < hi;
}

FR_DEV V3 edge_proj(V3 A, V3 B, V3 x, const Light& L, float D, float tau) {
  V3 p{__fadd_rn(A.x, __fmul_rn(tau, __fsub_rn(B.x, A.x))), __fadd_rn(A.y, __fmul_rn(tau, __fsub_rn(B.y, A.y))),
       __fadd_rn(A.z, __fmul_rn(tau, __fsub_rn(B.z, A.z)))};
  V3 q = sub3r(p, x);
  float h = dot3r(q, L.dl);
  float f = __fdiv_rn(D, h);
  return V3{__fadd_rn(x.x, __fmul_rn(f, q.x)), __fadd_rn(x.y, __fmul_rn(f, q.y)), __fadd_rn(x.z, __fmul_rn(f, q.z))};
}

// Packed edge record (6 float4 per edge, edge-BVH leaf order), written per
// render by k_pack_edges:
//   [0] a.xyz, canonical edge id   [1] b.xyz, f0   [2] n0.xyz, f1
//   [3] V0(f0).xyz                 [4] n1.xyz      [5] V0(f1).xyz
// n = decision-form face normal, V0 = first vertex of the face.

// Candidate search for one (shading point, light): traverse the edge BVH,
// keeping a child when (1) its box reaches the pyramid from x through the
// light square (4 side planes and the plane in front of x, with margins) and
// (2) its normal cone does not prove every face below it is seen from the
// same side (no silhouette possible).  Both tests are conservative; the leaf
// test (silhouette + clip, decision form) decides.  The candidate with the
// minimum Philox key is kept, so the pick does not depend on the order of
// enumeration.
struct Pick {
  int n;        // number of candidates
  int id;       // canonical id of the pick
  int slot;     // its leaf slot in the packed array
};

// Silhouette seen from x (decision form) with the edge's face planes in
// registers and without branches.
FR_DEV bool silhouette_regs(V3 n0, V3 p0, V3 n1, V3 p1, bool boundary, V3 x) {
  const float s0 = dot3r(n0, sub3r(x, p0));
  const float s1 = dot3r(n1, sub3r(x, p1));
  const bool two = (s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f);
  return boundary ? s0 != 0.0f : two;
}

// Sign of the decision form dot3r(n, sub3r(x, p)) over every x of the box
// [lo, hi]: +1 or -1 when it is proven to have that sign for all of them,
// 0 otherwise.  With u = 2^-24, sub3r and dot3r put at most four roundings
// on each term, so the computed value differs from the exact n.(x - p) by at
// most gamma_4 T, gamma_4 = 4u / (1 - 4u) < 2.4e-7 and
// T = sum_i |n_i| max(|lo_i - p_i|, |hi_i - p_i|).  The exact extremes over
// the box lie at the corners selected by the signs of n, and their FP32
// evaluation here carries the same bound; the margin 1e-6 T (more than
// 2 gamma_4 T, with room for the rounding of T itself), plus 1e-30 for
// products that flush to zero, proves the sign.  NaN or infinite data give 0.
FR_DEV int plane_sign_over_box(V3 n, V3 p, V3 lo, V3 hi) {
  const V3 cmin{n.x > 0.0f ? lo.x : hi.x, n.y > 0.0f ? lo.y : hi.y, n.z > 0.0f ? lo.z : hi.z};
  const V3 cmax{n.x > 0.0f ? hi.x : lo.x, n.y > 0.0f ? hi.y : lo.y, n.z > 0.0f ? hi.z : lo.z};
  const float smin = dot(n, cmin - p), smax = dot(n, cmax - p);
  const float T = fabsf(n.x) * fmaxf(fabsf(lo.x - p.x), fabsf(hi.x - p.x)) +
                  fabsf(n.y) * fmaxf(fabsf(lo.y - p.y), fabsf(hi.y - p.y)) +
                  fabsf(n.z) * fmaxf(fabsf(lo.z - p.z), fabsf(hi.z - p.z));
  const float m = 1e-6f * T + 1e-30f;
  return smin > m ? 1 : (smax < -m ? -1 : 0);
}

// One (shading point, edge) pair whose silhouette test has passed: the
// adjacency test (an edge of the hit face itself is no occluder), the clip
// against the light's pyramid and, for a candidate, its pick key.
FR_DEV void sedge_consider(const RenderArgs& a, const Light& L, float hs, int j, uint32_t pix, int s, V3 x,
                           int hitf, int slot, Pick& P, uint32_t& bestkey, unsigned& nclip) {
  const float4* R = a.ebvh.pack + 6 * slot;
  const float4 r1 = R[1];
  const int f0 = __float_as_int(r1.w), f1 = __float_as_int(R[2].w);
  if (f0 == hitf || f1 == hitf) return;
  const float4 r0 = R[0];
  float t0, t1;
  ++nclip;
  if (!shadow_clip(v3(r0), v3(r1), x, L, hs, a.kappa, t0, t1)) return;
  const int id = __float_as_int(r0.w);
  const uint32_t key = philox(a.seed, a.iter, pix, (uint32_t)s, (uint32_t)(TAG_SEDGE_PICK << 8 | j), (uint32_t)id).x;
  ++P.n;
  if (P.id < 0 || key < bestkey || (key == bestkey && id < P.id)) {
    bestkey = key; P.id = id; P.slot = slot;
  }
}

// Warps per block that the search's shared scratch serves: every kernel that
// calls it runs blocks of at most 256 threads.
constexpr int SEDGE_WARPS = 8;

// A lane's shading point for the search.
struct SedgePoint {
  bool valid;      // the sample hit the face
  V3 x;            // hit point (FP32)
  int hitf;        // hit face
  uint32_t pix;    // pixel and sample index: the pick's Philox key
  int s;
};

// The search runs warp-cooperatively.  Each lane holds NS shading points
// (NS = 1 or 2); the warp's group, its 32 NS points, shares one light and
// (light-major order) neighbouring samples, so the warp walks the edge BVH
// once with tests that hold for every point of the group's bounding sphere
// (centre rc, radius rr): the pyramid from any x in the sphere lies in the
// pyramid from rc dilated by rr, and a face seen from any x in the sphere
// is judged with the node's sphere grown by rr.  Control flow is uniform
// across the warp.  Points without a shading point (valid = false) still
// take part in the walk.
//
// The edges of the leaves that a node keeps are spread over the lanes, one
// edge per lane.  An edge whose two faces are proven to face the same way
// from every point of the box of the group's shading points
// (plane_sign_over_box) is no silhouette from any of them and is dropped;
// the others are queued.  Every 32 queued edges (and at the end) the warp
// runs the exact decision-form silhouette test of each queued edge, held by
// one lane, against each valid shading point in turn, and one ballot per
// shading point hands the lane that holds it the mask of its passing edges.
// The decisions are those of the per-pair test, so the candidate set, its
// size and the pick are unchanged; only the work to find them is smaller.
template <int NS>
FR_DEV void pick_light_warp_n(const RenderArgs& a, const SedgePoint (&q)[NS], int j, unsigned long long* cnt,
                              Pick (&P)[NS]) {
  __shared__ int sQ[SEDGE_WARPS][64];
  const Light& L = a.lights[j];
  const float hs = __fmul_rn(0.5f, a.side);
  uint32_t bestkey[NS];
#pragma unroll
  for (int qi = 0; qi < NS; ++qi) { P[qi].n = 0; P[qi].id = -1; P[qi].slot = -1; bestkey[qi] = 0xffffffffu; }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= SEDGE_WARPS) { if (lane == 0) atomicOr(a.err, ERR_STACK); return; }   // uniform over the warp
  // group bounding box -> sphere
  V3 lo_x{3e38f, 3e38f, 3e38f}, hi_x{-3e38f, -3e38f, -3e38f};
#pragma unroll
  for (int qi = 0; qi < NS; ++qi) {
    if (!q[qi].valid) continue;
    lo_x = V3{fminf(lo_x.x, q[qi].x.x), fminf(lo_x.y, q[qi].x.y), fminf(lo_x.z, q[qi].x.z)};
    hi_x = V3{fmaxf(hi_x.x, q[qi].x.x), fmaxf(hi_x.y, q[qi].x.y), fmaxf(hi_x.z, q[qi].x.z)};
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo_x.x = fminf(lo_x.x, __shfl_xor_sync(0xffffffffu, lo_x.x, off));
    lo_x.y = fminf(lo_x.y, __shfl_xor_sync(0xffffffffu, lo_x.y, off));
    lo_x.z = fminf(lo_x.z, __shfl_xor_sync(0xffffffffu, lo_x.z, off));
    hi_x.x = fmaxf(hi_x.x, __shfl_xor_sync(0xffffffffu, hi_x.x, off));
    hi_x.y = fmaxf(hi_x.y, __shfl_xor_sync(0xffffffffu, hi_x.y, off));
    hi_x.z = fmaxf(hi_x.z, __shfl_xor_sync(0xffffffffu, hi_x.z, off));
  }
  if (!(lo_x.x <= hi_x.x) || a.ebvh.bvh.n_nodes == 0) return;   // no valid point
  const V3 rc = (lo_x + hi_x) * 0.5f;
  const float rr = len((hi_x - lo_x) * 0.5f) * 1.0001f + 1e-6f;
  unsigned vm[NS];
#pragma unroll
  for (int qi = 0; qi < NS; ++qi) vm[qi] = __ballot_sync(0xffffffffu, q[qi].valid);
  // The search walks the 4-wide edge hierarchy; its node test is spread over
  // lanes 0..23: lane 6c + t holds test t of child c -- t = 0 the normal
  // cone, t = 1 the front plane, t = 2..5 side plane t - 2 of the pyramid
  // from rc through the light square, each dilated by the group radius rr.
  // Every test but the cone has the form dot(n, p - rc) >= -m with p the
  // box corner furthest along n.  A child is kept when its six lanes pass
  // (one ballot).
  const int tc = lane < 24 ? lane / 6 : 0, tt = lane < 24 ? lane - 6 * tc : 6;
  V3 pn{0, 0, 0};
  float pm = 0.0f;
  if (tt == 1) {
    pn = L.dl;
    pm = rr + 1e-4f - a.kappa;
  } else if (tt >= 2 && tt <= 5) {
    // light-square corners in the order (-,-), (+,-), (+,+), (-,+)
    const int k0 = tt - 2, k1 = (k0 + 1) & 3;
    const float u0 = (k0 == 1 || k0 == 2) ? hs : -hs, v0 = k0 >= 2 ? hs : -hs;
    const float u1 = (k1 == 1 || k1 == 2) ? hs : -hs, v1 = k1 >= 2 ? hs : -hs;
    V3 Qa = L.c + L.e1 * u0 + L.e2 * v0 - rc;
    V3 Qb = L.c + L.e1 * u1 + L.e2 * v1 - rc;
    V3 n = cross(Qa, Qb);
    if (dot(n, L.c - rc) < 0.0f) n = -n;
    pn = n;
    pm = (1e-4f + rr) * len(n);     // margin + dilation by the group radius
  }
  unsigned nvis = 0, ntest = 0, nclass = 0, nclip = 0;   // per search; widened when added to the counters
  int node = 0, steps = 0, qn = 0;
  bool failed = false;
  WStack wst{0, 0, 0};
  while (true) {
    if (++steps > a.mesh.max_steps) { atomicOr(a.err, ERR_STEPS); failed = true; break; }
    ++nvis;
    const int4 ch = a.ebvh.codes4[node];
    bool pass = true;
    if (tt < 6) {
      const int code_c = tc == 0 ? ch.x : (tc == 1 ? ch.y : (tc == 2 ? ch.z : ch.w));
      if (code_c == EMPTY_CHILD) {
        pass = false;
      } else if (tt == 0) {
        // With v from the child's bounding sphere (radius grown by rr) to
        // rc, beta the sphere's angular radius seen from rc and theta the
        // cone's grown half-angle (cn.w = cos theta, or -1 when theta >=
        // pi/2): every face below is seen from the same side by every point
        // of the group when theta + beta < pi/2 and the angle between v and
        // the axis differs from pi/2 by more than theta + beta.  Scaled by
        // |v|: q = |v| cos beta, rb = |v| sin beta.
        const float4* C = a.ebvh.cones4 + 2 * (4 * node + tc);
        const float4 cn = C[0];
        if (cn.w > 0.0f) {
          const float4 sp = C[1];     // bounding sphere of the child's box
          const float rb = sp.w + rr;
          const V3 v = rc - v3(sp);
          const float e2 = dot(v, v) - rb * rb;
          if (e2 > 0.0f) {
            const float q = e2 * rsqrtf(e2);
            const float s2 = 1.0f - cn.w * cn.w;        // >= 4e-6: theta >= 2e-3
            const float sT = s2 * rsqrtf(s2);
            if (q * cn.w > rb * sT) {
              const float lim = rb * cn.w + q * sT;     // |v| sin(theta + beta)
              const float c = dot(v, v3(cn));
              if (c > lim || c < -lim) pass = false;
            }
          }
        }
      } else {
        const float2* B = a.ebvh.boxes4 + 12 * node + 3 * tc;
        const float2 q0 = B[0], q1 = B[1], q2 = B[2];
        const V3 lo{q0.x, q0.y, q1.x}, hi{q1.y, q2.x, q2.y};
        V3 p{pn.x > 0 ? hi.x : lo.x, pn.y > 0 ? hi.y : lo.y, pn.z > 0 ? hi.z : lo.z};
        pass = dot(pn, p - rc) >= -pm;
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, pass);
    int next = -1, nl = 0, myslot = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (((m >> (6 * k)) & 0x3fu) != 0x3fu) continue;
      const int c2 = k == 0 ? ch.x : (k == 1 ? ch.y : (k == 2 ? ch.z : ch.w));
      if (leaf_child(c2)) {
        // leaves hold at most 8 edges, so a node's leaf edges fit the warp
        const int n = leaf_count(c2);
        if (lane >= nl && lane < nl + n) myslot = leaf_first(c2) + (lane - nl);
        nl += n;
      } else if (next < 0) {
        next = c2;
      } else {
        if (wst.sp >= WSTACK) { atomicOr(a.err, ERR_STACK); failed = true; break; }
        wpush(wst, c2, lane);
      }
    }
    if (failed) break;
    if (nl > 0) {
      if (lane == 0) nclass += nl;
      bool keep = false;     // a silhouette from some point of the box is possible
      if (myslot >= 0) {
        const float4* R = a.ebvh.pack + 6 * myslot;
        const float4 r2 = R[2], r3 = R[3];
        keep = true;
        if (__float_as_int(r2.w) >= 0) {
          const float4 r4 = R[4], r5 = R[5];
          const int c0 = plane_sign_over_box(v3(r2), v3(r3), lo_x, hi_x);
          const int c1 = plane_sign_over_box(v3(r4), v3(r5), lo_x, hi_x);
          keep = c0 == 0 || c0 != c1;
        }
      }
      const unsigned mk = __ballot_sync(0xffffffffu, keep);
      if (keep) sQ[w][qn + __popc(mk & ((1u << lane) - 1u))] = myslot;
      qn += __popc(mk);
      __syncwarp();
    }
    bool finished = false;
    if (next >= 0) node = next;
    else if (wst.sp == 0) finished = true;
    else node = wpop(wst);
    // Every 32 queued edges, and what is left at the end: the exact test of
    // each queued edge, held by one lane, against each valid lane's shading
    // point in turn; one ballot per shading point hands that lane the mask
    // of its passing edges, which it then takes through sedge_consider.
#pragma unroll 1
    while (qn >= 32 || (finished && qn > 0)) {
      const int nq = qn < 32 ? qn : 32;
      const bool has = lane < nq;
      const int slot = has ? sQ[w][lane] : 0;
      const float4* R = a.ebvh.pack + 6 * slot;
      const float4 r2 = R[2], r3 = R[3], r4 = R[4], r5 = R[5];
      const bool bnd = __float_as_int(r2.w) < 0;
      unsigned mine[NS];
#pragma unroll
      for (int qi = 0; qi < NS; ++qi) {
        mine[qi] = 0;
#pragma unroll 1
        for (unsigned r = vm[qi]; r != 0; r &= r - 1) {
          const int k = __ffs(r) - 1;
          const V3 xk{__shfl_sync(0xffffffffu, q[qi].x.x, k), __shfl_sync(0xffffffffu, q[qi].x.y, k),
                      __shfl_sync(0xffffffffu, q[qi].x.z, k)};
          const bool sil = has && silhouette_regs(v3(r2), v3(r3), v3(r4), v3(r5), bnd, xk);
          const unsigned b = __ballot_sync(0xffffffffu, sil);
          if (lane == k) mine[qi] = b;
        }
        if (lane == 0) ntest += (unsigned)nq * __popc(vm[qi]);
      }
#pragma unroll
      for (int qi = 0; qi < NS; ++qi) {
#pragma unroll 1
        while (mine[qi] != 0) {
          const int e = __ffs(mine[qi]) - 1;
          mine[qi] &= mine[qi] - 1;
          sedge_consider(a, L, hs, j, q[qi].pix, q[qi].s, q[qi].x, q[qi].hitf, sQ[w][e], P[qi], bestkey[qi], nclip);
        }
      }
      __syncwarp();
      const int rest = qn - nq;
      const int v = lane < rest ? sQ[w][32 + lane] : 0;
      __syncwarp();
      if (lane < rest) sQ[w][lane] = v;
      __syncwarp();
      qn = rest;
    }
    if (finished) break;
  }
  if (cnt) {                          // one set of atomics per warp
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nclip += __shfl_xor_sync(0xffffffffu, nclip, off);
    if (lane == 0) {
      atomicAdd(cnt + 2, (unsigned long long)nvis); atomicAdd(cnt + 3, (unsigned long long)ntest);
      atomicAdd(cnt + 4, (unsigned long long)nclip); atomicAdd(cnt + 5, (unsigned long long)nclass);
    }
  }
}

// One shading point per lane.
FR_DEV Pick pick_light_warp(const RenderArgs& a, bool valid, V3 x, int hitf, int j, uint32_t pix, int s,
                            unsigned long long* cnt) {
  const SedgePoint q[1] = {{valid, x, hitf, pix, s}};
  Pick P[1];
  pick_light_warp_n<1>(a, q, j, cnt, P);
  return P[0];
}

// Boundary term of one light given its pick: sample the clipped edge,
// difference the integrand across the projected edge, scatter the adjoint.
// All 32 lanes call together; lanes without a pick pass active = false.
FR_DEV void sedge_contribution(const RenderArgs& a, const GradBufs& gb, int j, int n_cand, int slot, V3 d, V3 x32,
                               int f, int flip, uint32_t pix, int s, V3 wrgb, unsigned long long* cnt,
                               bool active = true) {
  const Light& L = a.lights[j];
  const float hs = __fmul_rn(0.5f, a.side);
  if (!active) slot = 0;
  const float4* R = a.ebvh.pack + 6 * slot;
  float4 r0 = R[0], r1 = R[1];
  V3 A = v3(r0), B = v3(r1);
  int4 ev = a.ebvh.verts[slot];
  int v0 = ev.x, v1 = ev.y;
  float t0, t1;
  shadow_clip(A, B, x32, L, hs, a.kappa, t0, t1);
  U4 q = philox(a.seed, a.iter, pix, (uint32_t)s, (uint32_t)(TAG_SEDGE_POINT << 8 | j), 0);
  float u = unitf(q.x);
  float tau = __fadd_rn(t0, __fmul_rn(u, __fsub_rn(t1, t0)));
  float Dd = -dot3r(sub3r(x32, L.c), L.dl);
  V3 y = edge_proj(A, B, x32, L, Dd, tau);
  V3 y0 = edge_proj(A, B, x32, L, Dd, t0);
  V3 y1 = edge_proj(A, B, x32, L, Dd, t1);
  V3 nv = cross3r(L.dl, sub3r(y1, y0));
  float nl = __fsqrt_rn(dot3r(nv, nv));
  bool ok = active && nl != 0.0f;
  if (!ok) nl = 1.0f;
  nv = V3{__fdiv_rn(nv.x, nl), __fdiv_rn(nv.y, nl), __fdiv_rn(nv.z, nl)};
  const float e = a.eps_sedge;
  V3 yp{__fadd_rn(y.x, __fmul_rn(e, nv.x)), __fadd_rn(y.y, __fmul_rn(e, nv.y)), __fadd_rn(y.z, __fmul_rn(e, nv.z))};
  V3 ym{__fsub_rn(y.x, __fmul_rn(e, nv.x)), __fsub_rn(y.y, __fmul_rn(e, nv.y)), __fsub_rn(y.z, __fmul_rn(e, nv.z))};
  // visible_warp for both light points, with one shortcut: they straddle
  // the picked edge's shadow line, so the segment toward the shadowed one
  // usually ends on one of the edge's two faces.  Testing those first
  // settles it without a walk; an any-hit decision does not depend on
  // which blocking face is found, and neither face is the hit face (the
  // pick excludes adjacent edges).
  const int fa = __float_as_int(r1.w), fb = __float_as_int(R[2].w);
  const float thi = __fsub_rn(1.0f, a.tmin);
  const V3 wp = sub3r(yp, x32), wm = sub3r(ym, x32);
  bool gate_p = false, gate_m = false, bp = false, bm = false;
  if (ok) {
    const float4 n = a.mesh.ng[f];
    const V3 nn{n.x, n.y, n.z};
    const float sp = dot3r(nn, wp), sm = dot3r(nn, wm);
    gate_p = flip > 0 ? sp > 0.0f : sp < 0.0f;
    gate_m = flip > 0 ? sm > 0.0f : sm < 0.0f;
    if (gate_p) {
      const RayPre rp = ray_pre(x32, wp);
      bp = face_blocks(a.mesh, fa, rp, a.tmin, thi) || face_blocks(a.mesh, fb, rp, a.tmin, thi);
    }
    if (gate_m) {
      const RayPre rp = ray_pre(x32, wm);
      bm = face_blocks(a.mesh, fa, rp, a.tmin, thi) || face_blocks(a.mesh, fb, rp, a.tmin, thi);
    }
  }
  const bool op = occluded_warp(a.mesh, gate_p && !bp, x32, wp, f, a.tmin, thi, a.err, cnt);
  const bool om = occluded_warp(a.mesh, gate_m && !bm, x32, wm, f, a.tmin, thi, a.err, cnt);
  const bool vp = gate_p && !bp && !op;
  const bool vm = gate_m && !bm && !om;
  if (!ok || vp == vm) return;
  Surf S = surface(a, f, a.cam.o, d, flip);
  int idx[4];
  float w4[4], fu, fv;
  float cs = cspec_lookup(a.cspec, S.u, S.v, idx, w4, fu, fv);
  V3 l = light_rgb(a, j);
  V3 gp{0, 0, 0}, gm{0, 0, 0};
  if (vp) gp = shade_light(S, cs, l, yp, L.dl, a.brdf).h;
  if (vm) gm = shade_light(S, cs, l, ym, L.dl, a.brdf).h;
  float delta = dot(wrgb, gm - gp);
  if (delta == 0.0f) return;
  float w = delta * (float)n_cand * (t1 - t0);
  // Adjoint of the boundary point y(tau) = x + q D/h on the light plane,
  // q = p - x, p = A + tau (B - A), h = q.dl, D = (c - x).dl.  With
  // u = B - A and K = (dl x (q x u)) x q, the normal velocity of the
  // boundary times its length element gives
  //   dE/dp = w (D/h^2)^2 K,   dE/dx = w (1 - D/h) (D/h^3) K.
  // For an occluder close to the shading point these factors amplify any
  // error in x, and x itself is ill-conditioned at grazing hits, so this
  // (rare: only where the two sides differ) step runs in FP64.
  double x64[3];
  hit_point64(a, f, a.cam.o, d, x64);
  double ue[3] = {(double)B.x - A.x, (double)B.y - A.y, (double)B.z - A.z};
  double qv[3] = {((double)A.x - x64[0]) + ue[0] * tau, ((double)A.y - x64[1]) + ue[1] * tau,
                  ((double)A.z - x64[2]) + ue[2] * tau};
  double dl[3] = {L.dl.x, L.dl.y, L.dl.z};
  double h = qv[0] * dl[0] + qv[1] * dl[1] + qv[2] * dl[2];
  double D = ((double)L.c.x - x64[0]) * dl[0] + ((double)L.c.y - x64[1]) * dl[1] + ((double)L.c.z - x64[2]) * dl[2];
  double Dh2 = D / (h * h);
  double c1[3], c2[3], K[3];
  cross64(qv, ue, c1);
  cross64(dl, c1, c2);
  cross64(c2, qv, K);
  double sp = (double)w * Dh2 * Dh2, sx = (double)w * (1.0 - D / h) * (Dh2 / h);
  V3 g_p{(float)(K[0] * sp), (float)(K[1] * sp), (float)(K[2] * sp)};
  V3 gx{(float)(K[0] * sx), (float)(K[1] * sx), (float)(K[2] * sx)};
  atomic_add3(gb.dX + v0, g_p * (1.0f - tau));
  atomic_add3(gb.dX + v1, g_p * tau);
  hit_adjoint(a, f, d, S, gx, 0.0f, 0.0f, gb.dX);
}

}  // namespace fr
