// CPU oracle for the differentiable light-stage face renderer.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
// call this file: only tests/, the smoke check and the bench's CPU-baseline
// leg use it.  It shares no code with the CUDA library.
//
// What it computes (Dib et al., "Face Reflectance and Geometry Modeling via
// Differentiable Ray Tracing", Face Modeling and Optimization paragraphs):
//   * morphable geometry  X = R(r) (mu + B_id alpha + B_exp beta) + t,
//     albedo a = mu_a + B_alb delta                       (Face Modeling)
//   * area-weighted vertex normals n_i(alpha, beta, R, t) (Face Modeling)
//   * a virtual light stage of N = 20 square area lights on the vertices of an
//     isotropically sampled hemisphere, pointing at the origin (Face Modeling)
//   * the Monte-Carlo estimator F of the lighting equation with self-shadows
//     and the Cook-Torrance BRDF f_r = k_d f_lambert + k_s f_ct  (Eq. 1 text)
//   * its gradient: the interior derivative plus Li et al.'s edge-sampling
//     terms for primary visibility and for shadow boundaries on the lights
//   * the loss E_data + w1 E_prior + w2 E_light                     (Eq. 1)
//
// Precision rule.  Every value is FP64.  Every discrete decision (which
// triangle a ray hits, whether a shadow ray is blocked, whether an edge is a
// silhouette or can shadow a light, which pixel an edge sample lands in) is
// taken in FP32 from FP32 inputs with one fixed order of operations, so that a
// kernel computing in FP32 reaches the same integer decisions.  Sample
// positions (camera jitter points, light points, edge points and their
// offsets) are therefore FP32 values; the estimator is evaluated at them in
// FP64.  Build with -ffp-contract=off so no multiply-add is fused.
//
// Derivatives are forward-mode dual numbers over the same templated value
// code, so each derivative is the exact derivative of the value code.
//
// Readings of points the paper leaves open:
// pinhole camera at (0,0,d_cam) looking down -z; light k at Fibonacci
// direction z_k = (k+0.5)/N, phi_k = k*pi*(3-sqrt5), square of side s_L at
// radius R_L; Beckmann D with m = 0.3, V-cavity G, F folded into c_spec;
// R = Rz Ry Rx; E_prior = |alpha|^2 + |beta|^2 + |delta|^2 (statistical part);
// m_j of E_light given by the caller.
// The configuration also selects the alternatives: GGX D with Smith masking,
// Schlick's F, an icosphere dome of lights, and m_j as the mean of the lights
// per channel or as light j's channel mean.

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with a Weyl key
// schedule.
struct U4 { uint32_t v[4]; };

U4 philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0;
    uint64_t p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  U4 r; r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
  return r;
}

// 24-bit uniform in [0,1): exact in FP32 and FP64.
inline float unitf(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// Stream tags of the third counter word (tag << 8 | light).
enum { TAG_CAMERA = 0, TAG_LIGHT = 1, TAG_PEDGE = 2, TAG_PEDGE_LIGHT = 3,
       TAG_SEDGE_POINT = 4, TAG_SEDGE_PICK = 5, TAG_PEDGE_OFFSET = 6 };

// ---------------------------------------------------------------------------
// Dual numbers: value plus N partial derivatives.
template <int N> struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  static Dual var(double x, int i) { Dual r(x); r.d[i] = 1.0; return r; }
};
template <int N> Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) { Dual<N> r(a.v + b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) { Dual<N> r(a.v - b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> Dual<N> operator-(const Dual<N>& a) { Dual<N> r(-a.v); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) { Dual<N> r(a.v * b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) { Dual<N> r(a.v / b.v); double ib = 1.0 / b.v; for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib; return r; }
template <int N> Dual<N> operator+(const Dual<N>& a, double b) { Dual<N> r = a; r.v += b; return r; }
template <int N> Dual<N> operator+(double b, const Dual<N>& a) { return a + b; }
template <int N> Dual<N> operator-(const Dual<N>& a, double b) { Dual<N> r = a; r.v -= b; return r; }
template <int N> Dual<N> operator-(double b, const Dual<N>& a) { Dual<N> r = -a; r.v += b; return r; }
template <int N> Dual<N> operator*(const Dual<N>& a, double b) { Dual<N> r(a.v * b); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b; return r; }
template <int N> Dual<N> operator*(double b, const Dual<N>& a) { return a * b; }
template <int N> Dual<N> operator/(const Dual<N>& a, double b) { return a * (1.0 / b); }
template <int N> Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> Dual<N> sqrt(const Dual<N>& a) { Dual<N> r(std::sqrt(a.v)); double k = 0.5 / r.v; for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * k; return r; }
template <int N> Dual<N> exp(const Dual<N>& a) { Dual<N> r(std::exp(a.v)); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * r.v; return r; }

inline double val(double x) { return x; }
template <int N> double val(const Dual<N>& x) { return x.v; }
inline double sqrt(double x) { return std::sqrt(x); }
inline double exp(double x) { return std::exp(x); }
template <class T> T tmin(const T& a, const T& b) { return val(a) <= val(b) ? a : b; }

template <class T> struct V3 {
  T x, y, z;
  V3() : x(0.0), y(0.0), z(0.0) {}
  V3(const T& a, const T& b, const T& c) : x(a), y(b), z(c) {}
};
template <class T> V3<T> operator+(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> V3<T> operator-(const V3<T>& a, const V3<T>& b) { return V3<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T, class S> V3<T> operator*(const V3<T>& a, const S& s) { return V3<T>(a.x * s, a.y * s, a.z * s); }
template <class T, class S> V3<T> operator/(const V3<T>& a, const S& s) { return V3<T>(a.x / s, a.y / s, a.z / s); }
template <class T> T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return V3<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class T> V3<T> normalize(const V3<T>& a) { return a / sqrt(dot(a, a)); }
template <class T> V3<T> lift(const V3<double>& a) { return V3<T>(T(a.x), T(a.y), T(a.z)); }
inline V3<double> widen(const float* p) { return V3<double>(p[0], p[1], p[2]); }

// ---------------------------------------------------------------------------
// Inputs (mirrors of the ctypes structures in oracle/oracle.py).
struct OracleConfig {
  int32_t W, H, spp;
  uint32_t seed, iter;
  float tan_half_fov, d_cam, light_radius, light_side, beckmann_m;
  float eps_pedge, eps_sedge, shadow_tmin, clip_kappa;
  int32_t n_lights, shade_mode, n_threads, terms;
  int32_t value_mesh;   // 0: values on the FP64 posed mesh; 1: on the posed mesh rounded to FP32
  int32_t brdf_model;   // 0 Beckmann D + Cook-Torrance V-cavity G; 1 GGX D + separable Smith G
  int32_t fresnel;      // 0 F folded into c_spec; 1 Schlick F with c_spec as normal-incidence reflectance
  int32_t light_layout; // 0 Fibonacci hemisphere; 1 upper 20 vertices of a once-subdivided icosahedron
  int32_t light_prior;  // m_j of E_light: 0 given; 1 mean of the lights per channel; 2 light j's channel mean
};
struct OracleScene {
  int32_t V, F, K_id, K_exp, K_alb;
  const float* mean;      // [V*3]
  const int32_t* tris;    // [F*3]
  const float* uv;        // [V*2]
  const float* B_id;      // [3V*K_id]
  const float* B_exp;     // [3V*K_exp]
  const float* alb_mean;  // [3V]
  const float* B_alb;     // [3V*K_alb]
};

constexpr int CS = 32;             // c_spec resolution
constexpr double PI = 3.14159265358979323846;
enum { SHADE_FULL = 0, SHADE_FLAT = 1 };
enum { TERM_INTERIOR = 1, TERM_PEDGE = 2, TERM_SEDGE = 4 };

struct Layout {
  int alpha, beta, delta, cspec, pose, lights, total;
  Layout(const OracleScene& s, int nl) {
    alpha = 0; beta = s.K_id; delta = beta + s.K_exp; cspec = delta + s.K_alb;
    pose = cspec + CS * CS; lights = pose + 6; total = lights + 3 * nl;
  }
};

struct Light {           // one square area light; float frame is the definition
  float c[3], e1[3], e2[3], dl[3];   // centre, in-plane axes, unit direction from origin
};

// Light directions on the hemisphere z >= 0 (camera side).
// Layout 0: Fibonacci points, height (k + 1/2)/n, azimuth k times the golden
// angle pi (3 - sqrt 5).  Layout 1 (20 lights): the icosahedron with vertices
// the cyclic permutations of (0, +-1, +-phi), once subdivided (unit vertices
// plus the unit midpoints of its 30 edges: 42 directions), rotated about the
// x axis so that (0, 1, phi^2) points along +z; the 20 directions strictly
// above the horizon, ordered by height (descending) and then azimuth; a
// component below 1e-12 counts as exactly zero.
std::vector<std::array<double, 3>> stage_directions(int n, int layout) {
  std::vector<std::array<double, 3>> out;
  if (layout != 1) {
    const double golden = PI * (3.0 - std::sqrt(5.0));
    for (int k = 0; k < n; ++k) {
      double z = (k + 0.5) / n, rho = std::sqrt(1.0 - z * z);
      out.push_back({rho * std::cos(k * golden), rho * std::sin(k * golden), z});
    }
    return out;
  }
  const double g = (1.0 + std::sqrt(5.0)) / 2.0, s = 1.0 / std::sqrt(1.0 + g * g);
  const double ico[12][3] = {{0, 1, g}, {0, -1, g}, {0, 1, -g}, {0, -1, -g}, {1, g, 0}, {-1, g, 0},
                             {1, -g, 0}, {-1, -g, 0}, {g, 0, 1}, {-g, 0, 1}, {g, 0, -1}, {-g, 0, -1}};
  std::vector<std::array<double, 3>> dirs;
  for (auto& v : ico) dirs.push_back({v[0] * s, v[1] * s, v[2] * s});
  // neighbours on the unit icosahedron have cosine 1/sqrt(5)
  for (int i = 0; i < 12; ++i)
    for (int j = i + 1; j < 12; ++j) {
      double c = dirs[i][0] * dirs[j][0] + dirs[i][1] * dirs[j][1] + dirs[i][2] * dirs[j][2];
      if (std::fabs(c - 1.0 / std::sqrt(5.0)) > 1e-9) continue;
      double m[3] = {dirs[i][0] + dirs[j][0], dirs[i][1] + dirs[j][1], dirs[i][2] + dirs[j][2]};
      double l = std::sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
      dirs.push_back({m[0] / l, m[1] / l, m[2] / l});
    }
  const double ang = std::atan2(1.0, g * g);
  const double Rm[3][3] = {{1, 0, 0}, {0, std::cos(ang), -std::sin(ang)}, {0, std::sin(ang), std::cos(ang)}};
  for (auto& d : dirs) {
    std::array<double, 3> r{};
    for (int i = 0; i < 3; ++i) {
      r[i] = Rm[i][0] * d[0] + Rm[i][1] * d[1] + Rm[i][2] * d[2];
      if (std::fabs(r[i]) < 1e-12) r[i] = 0.0;   // round-off zeros made exact, so ties order alike
    }
    if (r[2] > 1e-9) out.push_back(r);
  }
  std::stable_sort(out.begin(), out.end(), [](const std::array<double, 3>& p, const std::array<double, 3>& q) {
    if (std::fabs(p[2] - q[2]) > 1e-9) return p[2] > q[2];
    return std::atan2(p[1], p[0]) < std::atan2(q[1], q[0]);
  });
  out.resize(n);
  return out;
}

// Light stage: one square per direction, centred at radius * d and facing
// the origin; e1 = normalize(+y x d), e2 = d x e1.
std::vector<Light> light_stage(int n, double radius, int layout) {
  std::vector<std::array<double, 3>> dirs = stage_directions(n, layout);
  std::vector<Light> L(n);
  for (int k = 0; k < n; ++k) {
    const double* d = dirs[k].data();
    // e1 = normalize(up x d) with up = +y; e2 = d x e1
    double e1[3] = {d[2], 0.0, -d[0]};
    double n1 = std::sqrt(e1[0] * e1[0] + e1[2] * e1[2]);
    e1[0] /= n1; e1[2] /= n1;
    double e2[3] = {d[1] * e1[2] - d[2] * e1[1], d[2] * e1[0] - d[0] * e1[2], d[0] * e1[1] - d[1] * e1[0]};
    for (int i = 0; i < 3; ++i) {
      L[k].c[i] = (float)(radius * d[i]);
      L[k].e1[i] = (float)e1[i];
      L[k].e2[i] = (float)e2[i];
      L[k].dl[i] = (float)d[i];
    }
  }
  return L;
}

// ---------------------------------------------------------------------------
// FP32 decision predicates (fixed operation order, no fused multiply-add).
inline float dot3f(const float* a, const float* b) {
  float p = a[0] * b[0];
  p = p + a[1] * b[1];
  p = p + a[2] * b[2];
  return p;
}
inline void sub3f(const float* a, const float* b, float* r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
inline void cross3f(const float* a, const float* b, float* r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2(1) 2013): shear
// the ray onto +z, evaluate the three 2D edge functions, recompute them in
// double when one is exactly zero.
struct RayPre { int kx, ky, kz; float Sx, Sy, Sz; float o[3]; };
inline RayPre ray_pre(const float* o, const float* d) {
  RayPre r;
  float ax = std::fabs(d[0]), ay = std::fabs(d[1]), az = std::fabs(d[2]);
  int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
  int kx = kz + 1; if (kx == 3) kx = 0;
  int ky = kx + 1; if (ky == 3) ky = 0;
  if (d[kz] < 0.0f) std::swap(kx, ky);
  r.kx = kx; r.ky = ky; r.kz = kz;
  r.Sx = d[kx] / d[kz];
  r.Sy = d[ky] / d[kz];
  r.Sz = 1.0f / d[kz];
  r.o[0] = o[0]; r.o[1] = o[1]; r.o[2] = o[2];
  return r;
}
// Returns true and t if the ray's line crosses the triangle (t unrestricted).
inline bool tri_hit32(const RayPre& r, const float* v0, const float* v1, const float* v2, float& t) {
  float A[3], B[3], C[3];
  sub3f(v0, r.o, A); sub3f(v1, r.o, B); sub3f(v2, r.o, C);
  float Ax = A[r.kx] - r.Sx * A[r.kz], Ay = A[r.ky] - r.Sy * A[r.kz];
  float Bx = B[r.kx] - r.Sx * B[r.kz], By = B[r.ky] - r.Sy * B[r.kz];
  float Cx = C[r.kx] - r.Sx * C[r.kz], Cy = C[r.ky] - r.Sy * C[r.kz];
  float U = Cx * By - Cy * Bx;
  float Vv = Ax * Cy - Ay * Cx;
  float W = Bx * Ay - By * Ax;
  if (U == 0.0f || Vv == 0.0f || W == 0.0f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    Vv = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.0f || Vv < 0.0f || W < 0.0f) && (U > 0.0f || Vv > 0.0f || W > 0.0f)) return false;
  float det = U + Vv;
  det = det + W;
  if (det == 0.0f) return false;
  float Az = r.Sz * A[r.kz], Bz = r.Sz * B[r.kz], Cz = r.Sz * C[r.kz];
  float T = U * Az;
  T = T + Vv * Bz;
  T = T + W * Cz;
  t = T / det;
  return true;
}

// ---------------------------------------------------------------------------
// Per-render state.
struct Edge { int32_t v0, v1, f0, f1; };   // v0 < v1; f0 < f1, f1 = -1 on the boundary

struct Render {
  const OracleConfig* cfg;
  const OracleScene* sc;
  const float* theta;
  Layout lay;
  int V, F, NL;
  std::vector<double> Xm;      // model-space vertices [V*3]
  std::vector<double> X;       // posed vertices used for values [V*3]
  std::vector<double> X64;     // posed vertices in FP64, before any rounding
  std::vector<float> X32;      // posed vertices rounded to FP32 (decisions)
  std::vector<double> alb;     // albedo [V*3]
  std::vector<double> nrm;     // unit vertex normals [V*3]
  std::vector<double> nsum;    // unnormalised vertex normal sums [V*3]
  std::vector<float> ng32;     // FP32 face normals [F*3] (decisions)
  std::vector<Edge> edges;
  std::vector<int32_t> sil;    // camera silhouette edges in index order
  std::vector<Light> lights;
  double R[9];
  float cam_o[3], cam_k, cam_cx, cam_cy;
  Render(const OracleConfig* c, const OracleScene* s, const float* th)
      : cfg(c), sc(s), theta(th), lay(*s, c->n_lights) {}

  const float* lightrgb(int j) const { return theta + lay.lights + 3 * j; }
  bool light_on(int j) const { const float* l = lightrgb(j); return l[0] != 0.0f || l[1] != 0.0f || l[2] != 0.0f; }
  const float* v32(int v) const { return &X32[3 * v]; }
  V3<double> v64(int v) const { return V3<double>(X[3 * v], X[3 * v + 1], X[3 * v + 2]); }
};

// R = Rz(rz) Ry(ry) Rx(rx), generic in the scalar type.
template <class T> void rotation(const T& rx, const T& ry, const T& rz, T* R) {
  T cx = T(std::cos(val(rx))), sx = T(std::sin(val(rx)));
  T cy = T(std::cos(val(ry))), sy = T(std::sin(val(ry)));
  T cz = T(std::cos(val(rz))), sz = T(std::sin(val(rz)));
  (void)cx; (void)sx; (void)cy; (void)sy; (void)cz; (void)sz;
  R[0] = cz * cy; R[1] = cz * sy * sx - sz * cx; R[2] = cz * sy * cx + sz * sx;
  R[3] = sz * cy; R[4] = sz * sy * sx + cz * cx; R[5] = sz * sy * cx - cz * sx;
  R[6] = -sy;     R[7] = cy * sx;                R[8] = cy * cx;
}
// Dual-aware sin/cos for the rotation derivative.
template <int N> Dual<N> dsin(const Dual<N>& a) { Dual<N> r(std::sin(a.v)); double c = std::cos(a.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * c; return r; }
template <int N> Dual<N> dcos(const Dual<N>& a) { Dual<N> r(std::cos(a.v)); double s = -std::sin(a.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * s; return r; }
template <int N> void rotation_dual(const Dual<N>& rx, const Dual<N>& ry, const Dual<N>& rz, Dual<N>* R) {
  Dual<N> cx = dcos(rx), sx = dsin(rx), cy = dcos(ry), sy = dsin(ry), cz = dcos(rz), sz = dsin(rz);
  R[0] = cz * cy; R[1] = cz * sy * sx - sz * cx; R[2] = cz * sy * cx + sz * sx;
  R[3] = sz * cy; R[4] = sz * sy * sx + cz * cx; R[5] = sz * sy * cx - cz * sx;
  R[6] = -sy;     R[7] = cy * sx;                R[8] = cy * cx;
}

int build_edges(Render& r) {
  const int F = r.F;
  std::vector<std::array<int32_t, 3>> he;   // (vmin, vmax, face)
  he.reserve(3 * F);
  for (int f = 0; f < F; ++f)
    for (int k = 0; k < 3; ++k) {
      int a = r.sc->tris[3 * f + k], b = r.sc->tris[3 * f + (k + 1) % 3];
      he.push_back({std::min(a, b), std::max(a, b), f});
    }
  std::sort(he.begin(), he.end());
  r.edges.clear();
  for (size_t i = 0; i < he.size();) {
    size_t j = i;
    while (j < he.size() && he[j][0] == he[i][0] && he[j][1] == he[i][1]) ++j;
    if (j - i > 2) return -2;            // non-manifold edge
    Edge e{he[i][0], he[i][1], he[i][2], (j - i == 2) ? he[i + 1][2] : -1};
    r.edges.push_back(e);
    i = j;
  }
  return 0;
}

// Morphable geometry, pose, albedo, normals (Face Modeling paragraph).
int prepare(Render& r) {
  const OracleScene& s = *r.sc;
  r.V = s.V; r.F = s.F; r.NL = r.cfg->n_lights;
  const int V = r.V, n3 = 3 * V;
  const float* al = r.theta + r.lay.alpha;
  const float* be = r.theta + r.lay.beta;
  const float* de = r.theta + r.lay.delta;
  const float* po = r.theta + r.lay.pose;
  r.Xm.assign(n3, 0.0); r.X.assign(n3, 0.0); r.X64.assign(n3, 0.0); r.X32.assign(n3, 0.0f); r.alb.assign(n3, 0.0);
  for (int i = 0; i < n3; ++i) {
    double x = s.mean[i];
    for (int k = 0; k < s.K_id; ++k) x += (double)s.B_id[(size_t)i * s.K_id + k] * al[k];
    for (int k = 0; k < s.K_exp; ++k) x += (double)s.B_exp[(size_t)i * s.K_exp + k] * be[k];
    r.Xm[i] = x;
    double a = s.alb_mean[i];
    for (int k = 0; k < s.K_alb; ++k) a += (double)s.B_alb[(size_t)i * s.K_alb + k] * de[k];
    r.alb[i] = a;
  }
  rotation<double>(po[0], po[1], po[2], r.R);
  for (int v = 0; v < V; ++v)
    for (int c = 0; c < 3; ++c) {
      double x = r.R[3 * c] * r.Xm[3 * v] + r.R[3 * c + 1] * r.Xm[3 * v + 1] + r.R[3 * c + 2] * r.Xm[3 * v + 2] + po[3 + c];
      r.X64[3 * v + c] = x;
      r.X32[3 * v + c] = (float)x;
      r.X[3 * v + c] = r.cfg->value_mesh ? (double)(float)x : x;
    }
  // FP32 face normals for decisions; FP64 area-weighted vertex normals for values.
  r.ng32.assign(3 * r.F, 0.0f);
  r.nsum.assign(n3, 0.0);
  for (int f = 0; f < r.F; ++f) {
    const int32_t* t = &s.tris[3 * f];
    float e1[3], e2[3];
    sub3f(r.v32(t[1]), r.v32(t[0]), e1);
    sub3f(r.v32(t[2]), r.v32(t[0]), e2);
    cross3f(e1, e2, &r.ng32[3 * f]);
    V3<double> c = cross(r.v64(t[1]) - r.v64(t[0]), r.v64(t[2]) - r.v64(t[0]));
    for (int k = 0; k < 3; ++k) {
      r.nsum[3 * t[k]] += c.x; r.nsum[3 * t[k] + 1] += c.y; r.nsum[3 * t[k] + 2] += c.z;
    }
  }
  r.nrm.assign(n3, 0.0);
  for (int v = 0; v < V; ++v) {
    double n = std::sqrt(r.nsum[3 * v] * r.nsum[3 * v] + r.nsum[3 * v + 1] * r.nsum[3 * v + 1] + r.nsum[3 * v + 2] * r.nsum[3 * v + 2]);
    if (n > 0) for (int c = 0; c < 3; ++c) r.nrm[3 * v + c] = r.nsum[3 * v + c] / n;
  }
  int rc = build_edges(r);
  if (rc) return rc;
  r.lights = light_stage(r.NL, r.cfg->light_radius, r.cfg->light_layout);
  // Camera: pinhole at (0,0,d_cam) looking down -z, square pixels.
  const OracleConfig& c = *r.cfg;
  r.cam_o[0] = 0.0f; r.cam_o[1] = 0.0f; r.cam_o[2] = c.d_cam;
  r.cam_k = (float)(2.0 * (double)c.tan_half_fov / (double)c.H);
  r.cam_cx = (float)((double)c.tan_half_fov * (double)c.W / (double)c.H);
  r.cam_cy = c.tan_half_fov;
  // Camera silhouettes: faces on opposite sides of the camera, or boundary edges.
  r.sil.clear();
  for (int e = 0; e < (int)r.edges.size(); ++e) {
    const Edge& E = r.edges[e];
    if (E.f1 < 0) { r.sil.push_back(e); continue; }
    float w0[3], w1[3];
    sub3f(r.cam_o, r.v32(s.tris[3 * E.f0]), w0);
    sub3f(r.cam_o, r.v32(s.tris[3 * E.f1]), w1);
    float s0 = dot3f(&r.ng32[3 * E.f0], w0), s1 = dot3f(&r.ng32[3 * E.f1], w1);
    if ((s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f)) r.sil.push_back(e);
  }
  return 0;
}

// Camera ray direction through screen point (sx, sy) in pixel units.
inline void camera_dir(const Render& r, float sx, float sy, float* d) {
  d[0] = sx * r.cam_k - r.cam_cx;
  d[1] = r.cam_cy - sy * r.cam_k;
  d[2] = -1.0f;
}

struct Hit { int f; float t; };

Hit closest_hit(const Render& r, const float* o, const float* d) {
  RayPre rp = ray_pre(o, d);
  Hit h{-1, 0.0f};
  for (int f = 0; f < r.F; ++f) {
    const int32_t* t = &r.sc->tris[3 * f];
    float tt;
    if (!tri_hit32(rp, r.v32(t[0]), r.v32(t[1]), r.v32(t[2]), tt)) continue;
    if (!(tt > 0.0f)) continue;
    if (h.f < 0 || tt < h.t) { h.f = f; h.t = tt; }   // ascending f: ties keep the smaller index
  }
  return h;
}

// Any triangle other than `skip` crossing the segment x + t w, t in (tmin, 1 - tmin)?
bool occluded(const Render& r, const float* x, const float* w, int skip) {
  RayPre rp = ray_pre(x, w);
  const float tlo = r.cfg->shadow_tmin, thi = 1.0f - r.cfg->shadow_tmin;
  for (int f = 0; f < r.F; ++f) {
    if (f == skip) continue;
    const int32_t* t = &r.sc->tris[3 * f];
    float tt;
    if (!tri_hit32(rp, r.v32(t[0]), r.v32(t[1]), r.v32(t[2]), tt)) continue;
    if (tt > tlo && tt < thi) return true;
  }
  return false;
}

inline void hit_point32(const float* o, const float* d, float t, float* x) {
  x[0] = o[0] + t * d[0]; x[1] = o[1] + t * d[1]; x[2] = o[2] + t * d[2];
}

inline void light_point32(const Light& L, float s, float u2, float u3, float* y) {
  float a = (u2 - 0.5f) * s, b = (u3 - 0.5f) * s;
  for (int i = 0; i < 3; ++i) { float p = L.c[i] + a * L.e1[i]; y[i] = p + b * L.e2[i]; }
}

// Visibility of light point y from hit point x on face f viewed from side `flip`.
bool visible(const Render& r, const float* x, const float* y, int f, int flip) {
  float w[3];
  sub3f(y, x, w);
  float g = dot3f(&r.ng32[3 * f], w);
  bool gate = flip > 0 ? g > 0.0f : g < 0.0f;
  if (!gate) return false;
  return !occluded(r, x, w, f);
}

// ---------------------------------------------------------------------------
// Shading (FP64 or dual).

// Hit-point quantities on face f for a fixed ray, generic in T: the vertex
// positions, vertex normals and albedos are supplied as T so that derivatives
// can be taken with respect to any of them.
template <class T> struct Surf {
  V3<T> x, ns, wo, rho;
  T b0, b1, b2;
  double u, v;   // interpolated specular-map coordinates (value)
  T uvu, uvv;
};

template <class T>
Surf<T> surface(const V3<double>& o, const V3<double>& d, const V3<T>* P, const V3<T>* Nv,
                const V3<T>* Av, const float* uv0, const float* uv1, const float* uv2, int flip) {
  // Moller-Trumbore solve of o + t d = P0 + b1 (P1-P0) + b2 (P2-P0).
  V3<T> e1 = P[1] - P[0], e2 = P[2] - P[0];
  V3<T> dd = lift<T>(d), s = lift<T>(o) - P[0];
  V3<T> pv = cross(dd, e2);
  T det = dot(e1, pv);
  T b1 = dot(s, pv) / det;
  V3<T> qv = cross(s, e1);
  T b2 = dot(dd, qv) / det;
  T t = dot(e2, qv) / det;
  Surf<T> S;
  S.b1 = b1; S.b2 = b2; S.b0 = T(1.0) - b1 - b2;
  S.x = lift<T>(o) + dd * t;
  V3<T> n = Nv[0] * S.b0 + Nv[1] * b1 + Nv[2] * b2;
  S.ns = normalize(n) * T((double)flip);
  S.wo = normalize(lift<T>(o) - S.x);
  S.rho = Av[0] * S.b0 + Av[1] * b1 + Av[2] * b2;
  S.uvu = S.b0 * (double)uv0[0] + b1 * (double)uv1[0] + b2 * (double)uv2[0];
  S.uvv = S.b0 * (double)uv0[1] + b1 * (double)uv1[1] + b2 * (double)uv2[1];
  S.u = val(S.uvu); S.v = val(S.uvv);
  return S;
}

// Bilinear lookup of the 32x32 specular map at (u, v), texel centres at
// (k + 0.5) / 32, clamp to edge.  Returns the four texel indices and weights.
template <class T> void bilinear(const T& u, const T& v, int* idx, T* w) {
  T su = u * (double)CS - 0.5, sv = v * (double)CS - 0.5;
  double fu0 = std::floor(val(su)), fv0 = std::floor(val(sv));
  T fu = su - fu0, fv = sv - fv0;
  int iu = (int)fu0, iv = (int)fv0;
  int iu0 = std::min(std::max(iu, 0), CS - 1), iu1 = std::min(std::max(iu + 1, 0), CS - 1);
  int iv0 = std::min(std::max(iv, 0), CS - 1), iv1 = std::min(std::max(iv + 1, 0), CS - 1);
  idx[0] = iv0 * CS + iu0; idx[1] = iv0 * CS + iu1; idx[2] = iv1 * CS + iu0; idx[3] = iv1 * CS + iu1;
  w[0] = (T(1.0) - fu) * (T(1.0) - fv); w[1] = fu * (T(1.0) - fv);
  w[2] = (T(1.0) - fu) * fv;            w[3] = fu * fv;
}

// Unshadowed integrand of one light at light point y, without the light's area:
// h = l (x) f_r(wi, wo) cos_x cos_y / d^2   (RGB).
// Reflectance readings (the Face Modeling paragraph names Cook-Torrance
// without its terms): roughness m; model 0 = Beckmann distribution
// exp(-tan^2/m^2) / (pi m^2 cos^4) with the V-cavity masking
// min(1, 2 (n.h)(n.wo)/(wo.h), 2 (n.h)(n.wi)/(wo.h)); model 1 = GGX
// distribution a^2 / (pi ((n.h)^2 (a^2 - 1) + 1)^2), a = m, with Smith
// masking G1(wi) G1(wo), G1(c) = 2c / (c + sqrt(a^2 + (1 - a^2) c^2));
// fresnel 0: the specular term is scaled by c_spec; fresnel 1: by Schlick's
// c_spec + (1 - c_spec)(1 - wo.h)^5.
struct Brdf {
  double m;
  int model, fresnel;
};
inline Brdf brdf_of(const OracleConfig& c) { return Brdf{(double)c.beckmann_m, c.brdf_model, c.fresnel}; }

template <class T>
V3<T> light_integrand(const V3<T>& x, const V3<T>& ns, const V3<T>& wo, const V3<T>& rho, const T& cs,
                      const V3<T>& l, const V3<double>& y, const V3<double>& dl, const Brdf& b) {
  V3<T> w = lift<T>(y) - x;
  T d2 = dot(w, w);
  V3<T> wi = w / sqrt(d2);
  T ci = dot(ns, wi);
  if (!(val(ci) > 0.0)) return V3<T>();
  T cy = dot(lift<T>(dl), wi);
  if (!(val(cy) > 0.0)) return V3<T>();
  T co = dot(ns, wo);
  T spec(0.0), F = cs;
  if (val(co) > 0.0) {
    V3<T> h = normalize(wi + wo);
    T ch = dot(ns, h), oh = dot(wo, h);
    T ch2 = ch * ch;
    const double m = b.m;
    T D, G;
    if (b.model == 0) {
      T tan2 = (T(1.0) - ch2) / ch2;
      D = exp(-tan2 / (m * m)) / (PI * m * m * ch2 * ch2);
      G = tmin(T(1.0), tmin(T(2.0) * ch * co / oh, T(2.0) * ch * ci / oh));
    } else {
      const double a2 = m * m;
      T den = ch2 * (a2 - 1.0) + T(1.0);
      D = T(a2) / (PI * den * den);
      T gi = T(2.0) * ci / (ci + sqrt(T(a2) + (1.0 - a2) * ci * ci));
      T go = T(2.0) * co / (co + sqrt(T(a2) + (1.0 - a2) * co * co));
      G = gi * go;
    }
    spec = D * G / (T(4.0) * ci * co);
    if (b.fresnel) {
      T q = T(1.0) - oh;
      F = cs + (T(1.0) - cs) * (q * q * q * q * q);
    }
  }
  T geo = ci * cy / d2;
  T sp = F * spec;
  return V3<T>(l.x * (rho.x / PI + sp) * geo, l.y * (rho.y / PI + sp) * geo, l.z * (rho.z / PI + sp) * geo);
}

// Gather helpers.
inline V3<double> nrm_of(const Render& r, int v) { return V3<double>(r.nrm[3 * v], r.nrm[3 * v + 1], r.nrm[3 * v + 2]); }
inline V3<double> alb_of(const Render& r, int v) { return V3<double>(r.alb[3 * v], r.alb[3 * v + 1], r.alb[3 * v + 2]); }

inline int face_flip(const Render& r, int f, const float* d) {
  return dot3f(&r.ng32[3 * f], d) > 0.0f ? -1 : 1;
}

Surf<double> surface_value(const Render& r, int f, const float* o, const float* d, int flip) {
  const int32_t* t = &r.sc->tris[3 * f];
  V3<double> P[3], N[3], A[3];
  for (int k = 0; k < 3; ++k) { P[k] = r.v64(t[k]); N[k] = nrm_of(r, t[k]); A[k] = alb_of(r, t[k]); }
  return surface<double>(widen(o), widen(d), P, N, A, &r.sc->uv[2 * t[0]], &r.sc->uv[2 * t[1]], &r.sc->uv[2 * t[2]], flip);
}

double cspec_value(const Render& r, double u, double v) {
  int idx[4]; double w[4];
  bilinear<double>(u, v, idx, w);
  const float* C = r.theta + r.lay.cspec;
  return w[0] * C[idx[0]] + w[1] * C[idx[1]] + w[2] * C[idx[2]] + w[3] * C[idx[3]];
}

// Auxiliary per-sample features (denoiser inputs): shading normal, diffuse
// albedo, specular albedo, distance / d_cam, fraction of lit lights visible.
struct Aux { double n[3], rho[3], cs, depth, vis, hit; };

// One-sample radiance along a camera ray (all lights that are on), using
// light samples from stream `tag` keyed by (c0, c1).  Also returns a decision
// signature and, optionally, the auxiliary features.
V3<double> radiance(const Render& r, const float* o, const float* d, int tag, uint32_t c0, uint32_t c1,
                    uint64_t* sig, Aux* aux = nullptr) {
  Hit h = closest_hit(r, o, d);
  if (sig) *sig = *sig * 1000003u + (uint64_t)(h.f + 1);
  if (h.f < 0) return V3<double>();
  if (r.cfg->shade_mode == SHADE_FLAT) return V3<double>(1.0, 1.0, 1.0);
  int flip = face_flip(r, h.f, d);
  float x32[3];
  hit_point32(o, d, h.t, x32);
  Surf<double> S = surface_value(r, h.f, o, d, flip);
  double cs = cspec_value(r, S.u, S.v);
  V3<double> L;
  const double area = (double)r.cfg->light_side * (double)r.cfg->light_side;
  int n_on = 0, n_vis = 0;
  for (int j = 0; j < r.NL; ++j) {
    if (!r.light_on(j)) continue;
    ++n_on;
    U4 q = philox(r.cfg->seed, r.cfg->iter, c0, c1, (uint32_t)(tag << 8 | j), 0);
    float y32[3];
    light_point32(r.lights[j], r.cfg->light_side, unitf(q.v[0]), unitf(q.v[1]), y32);
    bool vis = visible(r, x32, y32, h.f, flip);
    if (sig) *sig = *sig * 31u + (vis ? 1u : 0u);
    if (!vis) continue;
    ++n_vis;
    const float* l = r.lightrgb(j);
    V3<double> hv = light_integrand<double>(S.x, S.ns, S.wo, S.rho, cs, V3<double>(l[0], l[1], l[2]),
                                            widen(y32), widen(r.lights[j].dl), brdf_of(*r.cfg));
    L = L + hv * area;
  }
  if (aux) {
    aux->n[0] = S.ns.x; aux->n[1] = S.ns.y; aux->n[2] = S.ns.z;
    aux->rho[0] = S.rho.x; aux->rho[1] = S.rho.y; aux->rho[2] = S.rho.z;
    aux->cs = cs;
    V3<double> dd = widen(d);
    aux->depth = (double)h.t * std::sqrt(dot(dd, dd)) / (double)r.cfg->d_cam;
    aux->vis = n_on ? (double)n_vis / n_on : 0.0;
    aux->hit = 1.0;
  }
  return L;
}

inline void sample_ray(const Render& r, int px, int py, int s, float* d, uint32_t* pix) {
  uint32_t p = (uint32_t)(py * r.cfg->W + px);
  U4 q = philox(r.cfg->seed, r.cfg->iter, p, (uint32_t)s, (uint32_t)(TAG_CAMERA << 8), 0);
  float sx = (float)px + unitf(q.v[0]);
  float sy = (float)py + unitf(q.v[1]);
  camera_dir(r, sx, sy, d);
  *pix = p;
}

template <class F> void parallel_for(int n, int threads, F fn) {
  if (threads <= 1 || n < 2) { for (int i = 0; i < n; ++i) fn(i, 0); return; }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < threads; ++t)
    th.emplace_back([&, t]() {
      for (;;) {
        int i = next.fetch_add(1);
        if (i >= n) break;
        fn(i, t);
      }
    });
  for (auto& t : th) t.join();
}

int nthreads(const OracleConfig* c) {
  if (c->n_threads > 0) return c->n_threads;
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

// ---------------------------------------------------------------------------
// Backward.

// Per-thread FP64 accumulators.  Next to every sum the oracle keeps its L1
// mass (the sum of the absolute values of the contributions, propagated
// through the adjoints with absolute Jacobians): the size against which the
// rounding error of any other evaluation order or precision is measured.
struct Grad {
  std::vector<double> dX, dN, dA, dC, dL;
  std::vector<double> aX, aN, aA, aC, aL;   // L1 masses
  void init(int V, int NL) {
    dX.assign(3 * V, 0); dN.assign(3 * V, 0); dA.assign(3 * V, 0); dC.assign(CS * CS, 0); dL.assign(3 * NL, 0);
    aX.assign(3 * V, 0); aN.assign(3 * V, 0); aA.assign(3 * V, 0); aC.assign(CS * CS, 0); aL.assign(3 * NL, 0);
  }
  void add(const Grad& g) {
    for (size_t i = 0; i < dX.size(); ++i) {
      dX[i] += g.dX[i]; dN[i] += g.dN[i]; dA[i] += g.dA[i];
      aX[i] += g.aX[i]; aN[i] += g.aN[i]; aA[i] += g.aA[i];
    }
    for (size_t i = 0; i < dC.size(); ++i) { dC[i] += g.dC[i]; aC[i] += g.aC[i]; }
    for (size_t i = 0; i < dL.size(); ++i) { dL[i] += g.dL[i]; aL[i] += g.aL[i]; }
  }
};
inline void acc(std::vector<double>& d, std::vector<double>& a, size_t i, double v) { d[i] += v; a[i] += std::fabs(v); }

// Interior derivative of one camera sample: the exact derivative of the
// per-sample estimator with its samples and decisions held fixed.
constexpr int NI = 34;  // 9 positions, 9 normals, 9 albedos, 4 texels, 3 light channels
typedef Dual<NI> DI;

void interior_sample(const Render& r, const float* o, const float* d, const Hit& h, uint32_t pix, int s,
                     const double* dimg, Grad& g) {
  const int32_t* t = &r.sc->tris[3 * h.f];
  int flip = face_flip(r, h.f, d);
  V3<DI> P[3], N[3], A[3];
  for (int k = 0; k < 3; ++k) {
    V3<double> p = r.v64(t[k]), n = nrm_of(r, t[k]), a = alb_of(r, t[k]);
    P[k] = V3<DI>(DI::var(p.x, 3 * k), DI::var(p.y, 3 * k + 1), DI::var(p.z, 3 * k + 2));
    N[k] = V3<DI>(DI::var(n.x, 9 + 3 * k), DI::var(n.y, 10 + 3 * k), DI::var(n.z, 11 + 3 * k));
    A[k] = V3<DI>(DI::var(a.x, 18 + 3 * k), DI::var(a.y, 19 + 3 * k), DI::var(a.z, 20 + 3 * k));
  }
  Surf<DI> S = surface<DI>(widen(o), widen(d), P, N, A, &r.sc->uv[2 * t[0]], &r.sc->uv[2 * t[1]], &r.sc->uv[2 * t[2]], flip);
  int tex[4]; DI tw[4];
  bilinear<DI>(S.uvu, S.uvv, tex, tw);
  const float* C = r.theta + r.lay.cspec;
  DI cs(0.0);
  for (int k = 0; k < 4; ++k) cs = cs + tw[k] * DI::var(C[tex[k]], 27 + k);
  float x32[3];
  hit_point32(o, d, h.t, x32);
  const double area = (double)r.cfg->light_side * (double)r.cfg->light_side;
  const double inv_spp = 1.0 / r.cfg->spp;
  for (int j = 0; j < r.NL; ++j) {
    U4 q = philox(r.cfg->seed, r.cfg->iter, pix, (uint32_t)s, (uint32_t)(TAG_LIGHT << 8 | j), 0);
    float y32[3];
    light_point32(r.lights[j], r.cfg->light_side, unitf(q.v[0]), unitf(q.v[1]), y32);
    if (!visible(r, x32, y32, h.f, flip)) continue;
    const float* l = r.lightrgb(j);
    V3<DI> lv(DI::var(l[0], 31), DI::var(l[1], 32), DI::var(l[2], 33));
    V3<DI> hv = light_integrand<DI>(S.x, S.ns, S.wo, S.rho, cs, lv, widen(y32), widen(r.lights[j].dl), brdf_of(*r.cfg));
    double w[3] = {dimg[0] * inv_spp * area, dimg[1] * inv_spp * area, dimg[2] * inv_spp * area};
    double gin[NI];
    for (int k = 0; k < NI; ++k) gin[k] = w[0] * hv.x.d[k] + w[1] * hv.y.d[k] + w[2] * hv.z.d[k];
    for (int k = 0; k < 3; ++k)
      for (int c = 0; c < 3; ++c) {
        acc(g.dX, g.aX, 3 * t[k] + c, gin[3 * k + c]);
        acc(g.dN, g.aN, 3 * t[k] + c, gin[9 + 3 * k + c]);
        acc(g.dA, g.aA, 3 * t[k] + c, gin[18 + 3 * k + c]);
      }
    for (int k = 0; k < 4; ++k) acc(g.dC, g.aC, tex[k], gin[27 + k]);
    for (int c = 0; c < 3; ++c) acc(g.dL, g.aL, 3 * j + c, gin[31 + c]);
  }
}

// Screen projection of a posed point (pixel units), FP32 decision form.
inline void project32(const Render& r, const float* p, float* s) {
  float q = r.cfg->d_cam - p[2];
  float X = p[0] / q, Y = p[1] / q;
  s[0] = (X + r.cam_cx) / r.cam_k;
  s[1] = (r.cam_cy - Y) / r.cam_k;
}
template <class T> void project(const Render& r, const V3<T>& p, T* s) {
  T q = T((double)r.cfg->d_cam) - p.z;
  T X = p.x / q, Y = p.y / q;
  s[0] = (X + (double)r.cam_cx) / (double)r.cam_k;
  s[1] = ((double)r.cam_cy - Y) / (double)r.cam_k;
}

// Primary-visibility edge term (Li et al. 2018).  The camera silhouette
// edges in canonical order form one interval [0, nS): edge k covers
// [k, k + 1) with parameter u = z - k along it.  The N = W*H*spp samples of a
// render sample that interval systematically: sample i = pix*spp + s sits at
// z_i = (i + xi0) nS / N with one uniform offset xi0 per render, so that
// (nS / N) sum_i f(z_i) estimates sum_k int_0^1 f(k, u) du without bias.  z_i
// is formed in FP64 (add, multiply, divide in that order).
void primary_edge_sample(const Render& r, uint32_t pix, int s, const double* dimage, Grad& g) {
  const OracleConfig& c = *r.cfg;
  const int nS = (int)r.sil.size();
  if (nS == 0) return;
  U4 q0 = philox(c.seed, c.iter, 0u, 0u, (uint32_t)(TAG_PEDGE_OFFSET << 8), 0);
  const double xi0 = (double)q0.v[0] * (1.0 / 4294967296.0);
  const double i_s = (double)((uint64_t)pix * (uint64_t)c.spp + (uint64_t)s);
  const double n_s = (double)c.W * c.H * c.spp;
  double zt = (i_s + xi0) * (double)nS / n_s;
  int k = (int)std::floor(zt);
  if (k > nS - 1) k = nS - 1;
  float u = (float)(zt - (double)k);
  const Edge& E = r.edges[r.sil[k]];
  float a2[2], b2[2];
  project32(r, r.v32(E.v0), a2);
  project32(r, r.v32(E.v1), b2);
  float ex = b2[0] - a2[0], ey = b2[1] - a2[1];
  float mx = a2[0] + u * ex, my = a2[1] + u * ey;
  float fx = std::floor(mx), fy = std::floor(my);
  if (!(fx >= 0.0f && fx < (float)c.W && fy >= 0.0f && fy < (float)c.H)) return;
  int ipx = (int)fx, ipy = (int)fy;
  const double* dI = dimage + 3 * ((size_t)ipy * c.W + ipx);
  if (dI[0] == 0.0 && dI[1] == 0.0 && dI[2] == 0.0) return;
  float L2 = ex * ex;
  L2 = L2 + ey * ey;
  float L = std::sqrt(L2);
  if (L == 0.0f) return;
  float nx = -ey / L, ny = ex / L;
  float mpx = mx + c.eps_pedge * nx, mpy = my + c.eps_pedge * ny;
  float mmx = mx - c.eps_pedge * nx, mmy = my - c.eps_pedge * ny;
  float dp[3], dm[3];
  camera_dir(r, mpx, mpy, dp);
  camera_dir(r, mmx, mmy, dm);
  V3<double> fp = radiance(r, r.cam_o, dp, TAG_PEDGE_LIGHT, pix, (uint32_t)s, nullptr);
  V3<double> fm = radiance(r, r.cam_o, dm, TAG_PEDGE_LIGHT, pix, (uint32_t)s, nullptr);
  double delta = dI[0] * (fm.x - fp.x) + dI[1] * (fm.y - fp.y) + dI[2] * (fm.z - fp.z);
  if (delta == 0.0) return;
  // the sample is a difference of two estimates: its mass counts both
  double dmass = std::fabs(dI[0]) * (std::fabs(fm.x) + std::fabs(fp.x)) +
                 std::fabs(dI[1]) * (std::fabs(fm.y) + std::fabs(fp.y)) +
                 std::fabs(dI[2]) * (std::fabs(fm.z) + std::fabs(fp.z));
  const double N_es = (double)c.W * c.H * c.spp;
  double w = delta * nS / N_es;
  double wm = dmass * nS / N_es;
  typedef Dual<6> D6;
  V3<double> a = r.v64(E.v0), b = r.v64(E.v1);
  V3<D6> A(D6::var(a.x, 0), D6::var(a.y, 1), D6::var(a.z, 2));
  V3<D6> B(D6::var(b.x, 3), D6::var(b.y, 4), D6::var(b.z, 5));
  D6 sa[2], sb[2];
  project<D6>(r, A, sa);
  project<D6>(r, B, sb);
  double evx = sb[0].v - sa[0].v, evy = sb[1].v - sa[1].v;
  double ud = (double)u;
  for (int i = 0; i < 6; ++i) {
    double mdx = (1.0 - ud) * sa[0].d[i] + ud * sb[0].d[i];
    double mdy = (1.0 - ud) * sa[1].d[i] + ud * sb[1].d[i];
    double vn = -evy * mdx + evx * mdy;          // R90(e) . dm/dtheta
    int v = i < 3 ? E.v0 : E.v1;
    g.dX[3 * v + (i % 3)] += w * vn;
    g.aX[3 * v + (i % 3)] += std::fabs(wm * vn);
  }
}

// Shadow-boundary edge term for one camera sample and one light: pick one
// edge uniformly among the silhouettes (seen from x) whose central projection
// from x crosses the light square, pick a point uniformly in the projected
// edge parameter, difference the integrand across the boundary.
struct Clip { float t0, t1; };

// FP32 candidate test: clip the edge parameter interval to the part in front
// of x (toward the light) whose projection lands in the light square.
bool shadow_clip32(const float* a, const float* b, const float* x, const Light& L, float hs, float kappa, Clip& cl) {
  float xc[3];
  sub3f(x, L.c, xc);
  float al1 = dot3f(xc, L.e1), al2 = dot3f(xc, L.e2);
  float D = -dot3f(xc, L.dl);
  float ca[5], cb[5];
  const float* P[2] = {a, b};
  float* cc[2] = {ca, cb};
  for (int e = 0; e < 2; ++e) {
    float q[3];
    sub3f(P[e], x, q);
    float h = dot3f(q, L.dl), s1 = dot3f(q, L.e1), s2 = dot3f(q, L.e2);
    float n1 = al1 * h + s1 * D;
    float n2 = al2 * h + s2 * D;
    float hh = hs * h;
    cc[e][0] = h - kappa;
    cc[e][1] = hh - n1;
    cc[e][2] = hh + n1;
    cc[e][3] = hh - n2;
    cc[e][4] = hh + n2;
  }
  float t0 = 0.0f, t1 = 1.0f;
  for (int k = 0; k < 5; ++k) {
    float A = ca[k], B = cb[k];
    if (A < 0.0f && B < 0.0f) return false;
    if (A < 0.0f) { float rr = A / (A - B); if (rr > t0) t0 = rr; }
    else if (B < 0.0f) { float rr = A / (A - B); if (rr < t1) t1 = rr; }
  }
  cl.t0 = t0; cl.t1 = t1;
  return t0 < t1;
}

// Central projection from x onto the light plane of the edge point at parameter tau.
inline void edge_proj32(const float* a, const float* b, const float* x, const Light& L, float D, float tau, float* y) {
  float p[3], q[3];
  for (int i = 0; i < 3; ++i) p[i] = a[i] + tau * (b[i] - a[i]);
  sub3f(p, x, q);
  float h = dot3f(q, L.dl);
  float f = D / h;
  for (int i = 0; i < 3; ++i) y[i] = x[i] + f * q[i];
}

bool silhouette_from(const Render& r, const Edge& E, const float* x) {
  float w0[3];
  sub3f(x, r.v32(r.sc->tris[3 * E.f0]), w0);
  float s0 = dot3f(&r.ng32[3 * E.f0], w0);
  if (E.f1 < 0) return s0 != 0.0f;
  float w1[3];
  sub3f(x, r.v32(r.sc->tris[3 * E.f1]), w1);
  float s1 = dot3f(&r.ng32[3 * E.f1], w1);
  return (s0 > 0.0f && s1 < 0.0f) || (s0 < 0.0f && s1 > 0.0f);
}

// Shadow-edge estimate for the camera ray (o, d) hitting face h.f, light j;
// adds  weight . d(estimate)/d(vertex positions)  into g.dX, where `weight`
// is the RGB adjoint of the pixel already divided by spp.
void shadow_edge_sample(const Render& r, const float* o, const float* d, const Hit& h, uint32_t pix, int s, int j,
                        const double* wrgb, Grad& g) {
  const OracleConfig& c = *r.cfg;
  const Light& L = r.lights[j];
  float x32[3];
  hit_point32(o, d, h.t, x32);
  const float hs = 0.5f * c.light_side;
  // enumerate candidates; keep the one with the smallest (hash, index)
  int n = 0, best = -1;
  uint32_t bestkey = 0;
  Clip bestclip{0, 0};
  for (int e = 0; e < (int)r.edges.size(); ++e) {
    const Edge& E = r.edges[e];
    if (E.f0 == h.f || E.f1 == h.f) continue;
    if (!silhouette_from(r, E, x32)) continue;
    Clip cl;
    if (!shadow_clip32(r.v32(E.v0), r.v32(E.v1), x32, L, hs, c.clip_kappa, cl)) continue;
    ++n;
    uint32_t key = philox(c.seed, c.iter, pix, (uint32_t)s, (uint32_t)(TAG_SEDGE_PICK << 8 | j), (uint32_t)e).v[0];
    if (best < 0 || key < bestkey) { best = e; bestkey = key; bestclip = cl; }
  }
  if (n == 0) return;
  const Edge& E = r.edges[best];
  const float* a = r.v32(E.v0);
  const float* b = r.v32(E.v1);
  U4 q = philox(c.seed, c.iter, pix, (uint32_t)s, (uint32_t)(TAG_SEDGE_POINT << 8 | j), 0);
  float u = unitf(q.v[0]);
  float tau = bestclip.t0 + u * (bestclip.t1 - bestclip.t0);
  float xc[3];
  sub3f(x32, L.c, xc);
  float D = -dot3f(xc, L.dl);
  float y[3], y0[3], y1[3], T[3], nv[3];
  edge_proj32(a, b, x32, L, D, tau, y);
  edge_proj32(a, b, x32, L, D, bestclip.t0, y0);
  edge_proj32(a, b, x32, L, D, bestclip.t1, y1);
  sub3f(y1, y0, T);
  cross3f(L.dl, T, nv);
  float nl = std::sqrt(dot3f(nv, nv));
  if (nl == 0.0f) return;
  for (int i = 0; i < 3; ++i) nv[i] = nv[i] / nl;
  float yp[3], ym[3];
  for (int i = 0; i < 3; ++i) { yp[i] = y[i] + c.eps_sedge * nv[i]; ym[i] = y[i] - c.eps_sedge * nv[i]; }
  int flip = face_flip(r, h.f, d);
  bool vp = visible(r, x32, yp, h.f, flip);
  bool vm = visible(r, x32, ym, h.f, flip);
  if (vp == vm) return;  // both sides agree only when another occluder covers the boundary
  Surf<double> S = surface_value(r, h.f, o, d, flip);
  double cs = cspec_value(r, S.u, S.v);
  const float* l = r.lightrgb(j);
  V3<double> lv(l[0], l[1], l[2]);
  V3<double> gp, gm;
  if (vp) gp = light_integrand<double>(S.x, S.ns, S.wo, S.rho, cs, lv, widen(yp), widen(L.dl), brdf_of(c));
  if (vm) gm = light_integrand<double>(S.x, S.ns, S.wo, S.rho, cs, lv, widen(ym), widen(L.dl), brdf_of(c));
  double delta = wrgb[0] * (gm.x - gp.x) + wrgb[1] * (gm.y - gp.y) + wrgb[2] * (gm.z - gp.z);
  if (delta == 0.0) return;
  double dmass = std::fabs(wrgb[0]) * (std::fabs(gm.x) + std::fabs(gp.x)) +
                 std::fabs(wrgb[1]) * (std::fabs(gm.y) + std::fabs(gp.y)) +
                 std::fabs(wrgb[2]) * (std::fabs(gm.z) + std::fabs(gp.z));
  double w = delta * (double)n * ((double)bestclip.t1 - (double)bestclip.t0);
  double wm = dmass * (double)n * ((double)bestclip.t1 - (double)bestclip.t0);
  // y(tau) as a function of the edge endpoints, the hit triangle and tau.
  typedef Dual<16> D16;
  const int32_t* t = &r.sc->tris[3 * h.f];
  V3<double> av = r.v64(E.v0), bv = r.v64(E.v1);
  V3<D16> A(D16::var(av.x, 0), D16::var(av.y, 1), D16::var(av.z, 2));
  V3<D16> B(D16::var(bv.x, 3), D16::var(bv.y, 4), D16::var(bv.z, 5));
  V3<D16> P[3];
  for (int k = 0; k < 3; ++k) {
    V3<double> p = r.v64(t[k]);
    P[k] = V3<D16>(D16::var(p.x, 6 + 3 * k), D16::var(p.y, 7 + 3 * k), D16::var(p.z, 8 + 3 * k));
  }
  D16 tauD = D16::var((double)tau, 15);
  V3<D16> e1 = P[1] - P[0], e2 = P[2] - P[0];
  V3<D16> dd = lift<D16>(widen(d)), so = lift<D16>(widen(o)) - P[0];
  V3<D16> qv = cross(so, e1);
  D16 tt = dot(e2, qv) / dot(e1, cross(dd, e2));
  V3<D16> X = lift<D16>(widen(o)) + dd * tt;
  V3<D16> pp = A + (B - A) * tauD;
  V3<D16> qq = pp - X;
  V3<D16> dlD = lift<D16>(widen(L.dl));
  D16 hq = dot(qq, dlD);
  D16 Dd = dot(lift<D16>(widen(L.c)) - X, dlD);
  V3<D16> Y = X + qq * (Dd / hq);
  V3<double> dYdt(Y.x.d[15], Y.y.d[15], Y.z.d[15]);
  V3<double> Rn = cross(widen(L.dl), dYdt);     // R90 of the tangent within the light plane
  for (int k = 0; k < 15; ++k) {
    double vn = Rn.x * Y.x.d[k] + Rn.y * Y.y.d[k] + Rn.z * Y.z.d[k];
    int v = k < 3 ? E.v0 : (k < 6 ? E.v1 : t[(k - 6) / 3]);
    g.dX[3 * v + (k % 3)] += w * vn;
    g.aX[3 * v + (k % 3)] += std::fabs(wm * vn);
  }
}

// dN (unit vertex normals) -> dX through normalisation and face cross products.
void normals_adjoint(const Render& r, const std::vector<double>& dN, std::vector<double>& dX,
                     const std::vector<double>& aN, std::vector<double>& aX) {
  const int V = r.V;
  std::vector<double> gs(3 * V, 0.0), as(3 * V, 0.0);
  typedef Dual<3> D3;
  for (int v = 0; v < V; ++v) {
    V3<D3> s(D3::var(r.nsum[3 * v], 0), D3::var(r.nsum[3 * v + 1], 1), D3::var(r.nsum[3 * v + 2], 2));
    if (dot(s, s).v == 0.0) continue;
    V3<D3> n = normalize(s);
    for (int k = 0; k < 3; ++k) {
      gs[3 * v + k] = dN[3 * v] * n.x.d[k] + dN[3 * v + 1] * n.y.d[k] + dN[3 * v + 2] * n.z.d[k];
      as[3 * v + k] = aN[3 * v] * std::fabs(n.x.d[k]) + aN[3 * v + 1] * std::fabs(n.y.d[k]) +
                      aN[3 * v + 2] * std::fabs(n.z.d[k]);
    }
  }
  typedef Dual<9> D9;
  for (int f = 0; f < r.F; ++f) {
    const int32_t* t = &r.sc->tris[3 * f];
    V3<D9> P[3];
    for (int k = 0; k < 3; ++k) {
      V3<double> p = r.v64(t[k]);
      P[k] = V3<D9>(D9::var(p.x, 3 * k), D9::var(p.y, 3 * k + 1), D9::var(p.z, 3 * k + 2));
    }
    V3<D9> cr = cross(P[1] - P[0], P[2] - P[0]);
    double gc[3] = {0, 0, 0}, ac[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k)
      for (int cc = 0; cc < 3; ++cc) { gc[cc] += gs[3 * t[k] + cc]; ac[cc] += as[3 * t[k] + cc]; }
    for (int i = 0; i < 9; ++i) {
      dX[3 * t[i / 3] + i % 3] += gc[0] * cr.x.d[i] + gc[1] * cr.y.d[i] + gc[2] * cr.z.d[i];
      aX[3 * t[i / 3] + i % 3] += ac[0] * std::fabs(cr.x.d[i]) + ac[1] * std::fabs(cr.y.d[i]) +
                                  ac[2] * std::fabs(cr.z.d[i]);
    }
  }
}

// dX, dA -> parameter gradient (alpha, beta, delta, pose) ; dC, dL copied.
void geometry_adjoint(const Render& r, const Grad& G, const std::vector<double>& dX, const std::vector<double>& aX,
                      double* out, double* mass) {
  const OracleScene& s = *r.sc;
  const Layout& lay = r.lay;
  const int V = r.V;
  for (int i = 0; i < lay.total; ++i) { out[i] = 0.0; mass[i] = 0.0; }
  // dXm = R^T dX
  std::vector<double> dXm(3 * V), aXm(3 * V);
  for (int v = 0; v < V; ++v)
    for (int c = 0; c < 3; ++c) {
      dXm[3 * v + c] = r.R[c] * dX[3 * v] + r.R[3 + c] * dX[3 * v + 1] + r.R[6 + c] * dX[3 * v + 2];
      aXm[3 * v + c] = std::fabs(r.R[c]) * aX[3 * v] + std::fabs(r.R[3 + c]) * aX[3 * v + 1] +
                       std::fabs(r.R[6 + c]) * aX[3 * v + 2];
    }
  for (int k = 0; k < s.K_id; ++k) {
    double a = 0, m = 0;
    for (int i = 0; i < 3 * V; ++i) {
      double b = s.B_id[(size_t)i * s.K_id + k];
      a += b * dXm[i]; m += std::fabs(b) * aXm[i];
    }
    out[lay.alpha + k] = a; mass[lay.alpha + k] = m;
  }
  for (int k = 0; k < s.K_exp; ++k) {
    double a = 0, m = 0;
    for (int i = 0; i < 3 * V; ++i) {
      double b = s.B_exp[(size_t)i * s.K_exp + k];
      a += b * dXm[i]; m += std::fabs(b) * aXm[i];
    }
    out[lay.beta + k] = a; mass[lay.beta + k] = m;
  }
  for (int k = 0; k < s.K_alb; ++k) {
    double a = 0, m = 0;
    for (int i = 0; i < 3 * V; ++i) {
      double b = s.B_alb[(size_t)i * s.K_alb + k];
      a += b * G.dA[i]; m += std::fabs(b) * G.aA[i];
    }
    out[lay.delta + k] = a; mass[lay.delta + k] = m;
  }
  for (int i = 0; i < CS * CS; ++i) { out[lay.cspec + i] = G.dC[i]; mass[lay.cspec + i] = G.aC[i]; }
  // pose: rotation angles by dual numbers, translation = sum of dX
  typedef Dual<3> D3;
  const float* po = r.theta + lay.pose;
  D3 Rd[9];
  rotation_dual<3>(D3::var(po[0], 0), D3::var(po[1], 1), D3::var(po[2], 2), Rd);
  double dr[3] = {0, 0, 0}, dt[3] = {0, 0, 0}, mr[3] = {0, 0, 0}, mt[3] = {0, 0, 0};
  for (int v = 0; v < V; ++v)
    for (int c = 0; c < 3; ++c) {
      dt[c] += dX[3 * v + c];
      mt[c] += aX[3 * v + c];
      for (int m = 0; m < 3; ++m) {
        double dRx = Rd[3 * c].d[m] * r.Xm[3 * v] + Rd[3 * c + 1].d[m] * r.Xm[3 * v + 1] + Rd[3 * c + 2].d[m] * r.Xm[3 * v + 2];
        dr[m] += dX[3 * v + c] * dRx;
        mr[m] += aX[3 * v + c] * std::fabs(dRx);
      }
    }
  for (int m = 0; m < 3; ++m) {
    out[lay.pose + m] = dr[m]; out[lay.pose + 3 + m] = dt[m];
    mass[lay.pose + m] = mr[m]; mass[lay.pose + 3 + m] = mt[m];
  }
  for (int i = 0; i < 3 * r.NL; ++i) { out[lay.lights + i] = G.dL[i]; mass[lay.lights + i] = G.aL[i]; }
}

}  // namespace

// ---------------------------------------------------------------------------
// C API (ctypes).
extern "C" {

void oracle_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t* out) {
  U4 r = philox(k0, k1, c0, c1, c2, c3);
  for (int i = 0; i < 4; ++i) out[i] = r.v[i];
}

int oracle_n_edges(const OracleConfig* cfg, const OracleScene* sc, const float* theta, int32_t* edges_out) {
  Render r(cfg, sc, theta);
  r.V = sc->V; r.F = sc->F;
  if (build_edges(r)) return -2;
  if (edges_out)
    for (size_t e = 0; e < r.edges.size(); ++e) {
      edges_out[4 * e] = r.edges[e].v0; edges_out[4 * e + 1] = r.edges[e].v1;
      edges_out[4 * e + 2] = r.edges[e].f0; edges_out[4 * e + 3] = r.edges[e].f1;
    }
  return (int)r.edges.size();
}

void oracle_light_stage(int32_t n, float radius, int32_t layout, float* out /*[n*12]: c, e1, e2, dl*/) {
  if (layout == 1 && n != 20) return;
  std::vector<Light> L = light_stage(n, radius, layout);
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < 3; ++i) {
      out[12 * k + i] = L[k].c[i]; out[12 * k + 3 + i] = L[k].e1[i];
      out[12 * k + 6 + i] = L[k].e2[i]; out[12 * k + 9 + i] = L[k].dl[i];
    }
}

// Posed vertices (FP64 and FP32), albedo and unit vertex normals.
int oracle_geometry(const OracleConfig* cfg, const OracleScene* sc, const float* theta,
                    double* X, float* X32, double* albedo, double* normals) {
  Render r(cfg, sc, theta);
  int rc = prepare(r);
  if (rc) return rc;
  size_t n = 3 * (size_t)sc->V;
  if (X) std::memcpy(X, r.X64.data(), n * sizeof(double));
  if (X32) std::memcpy(X32, r.X32.data(), n * sizeof(float));
  if (albedo) std::memcpy(albedo, r.alb.data(), n * sizeof(double));
  if (normals) std::memcpy(normals, r.nrm.data(), n * sizeof(double));
  return (int)r.sil.size();
}

// Forward render.  pix == NULL renders all W*H pixels into image[H*W*3];
// otherwise the n_pix listed pixel indices (py*W+px) into image[n_pix*3].
int oracle_render(const OracleConfig* cfg, const OracleScene* sc, const float* theta,
                  const int32_t* pix, int32_t n_pix, double* image, uint64_t* signature, double* aov) {
  Render r(cfg, sc, theta);
  int rc = prepare(r);
  if (rc) return rc;
  const int npx = pix ? n_pix : cfg->W * cfg->H;
  std::vector<uint64_t> sig(npx, 0);
  parallel_for(npx, nthreads(cfg), [&](int i, int) {
    int p = pix ? pix[i] : i;
    int px = p % cfg->W, py = p / cfg->W;
    V3<double> acc;
    uint64_t sg = 0;
    double f[15] = {0};   // feature sums: n, rho, cs, depth, vis, Y^2, hit, Y
    for (int s = 0; s < cfg->spp; ++s) {
      float d[3];
      uint32_t pp;
      sample_ray(r, px, py, s, d, &pp);
      Aux ax{{0, 0, 0}, {0, 0, 0}, 0, 0, 0, 0};
      V3<double> L = radiance(r, r.cam_o, d, TAG_LIGHT, pp, (uint32_t)s, &sg, aov ? &ax : nullptr);
      acc = acc + L;
      if (aov) {
        double Y = (L.x + L.y + L.z) / 3.0;
        for (int k = 0; k < 3; ++k) { f[3 + k] += ax.n[k]; f[6 + k] += ax.rho[k]; }
        f[9] += ax.cs; f[10] += ax.depth; f[11] += ax.vis; f[12] += Y * Y; f[13] += ax.hit; f[14] += Y;
      }
    }
    acc = acc / (double)cfg->spp;
    image[3 * i] = acc.x; image[3 * i + 1] = acc.y; image[3 * i + 2] = acc.z;
    if (aov) {
      double* o = aov + 14 * (size_t)i;
      o[0] = acc.x; o[1] = acc.y; o[2] = acc.z;
      for (int k = 3; k < 12; ++k) o[k] = f[k] / cfg->spp;
      double mY = f[14] / cfg->spp;
      o[12] = std::max(0.0, f[12] / cfg->spp - mY * mY);
      o[13] = f[13] / cfg->spp;
    }
    sig[i] = sg * 2654435761u + (uint64_t)p;
  });
  if (signature) {
    uint64_t h = 0;
    for (int i = 0; i < npx; ++i) h += sig[i] * (2 * (uint64_t)i + 1);
    *signature = h;
  }
  return 0;
}

// Gradient of <d_image, render(theta)> with respect to theta.  grad[P];
// grad_terms (or NULL) receives the interior, primary-edge and shadow-edge
// parts as three consecutive P-vectors.  cfg->terms selects the terms
// (bitmask 1 | 2 | 4; 0 means all).  Pixels whose adjoint is zero are skipped.
int oracle_render_backward(const OracleConfig* cfg, const OracleScene* sc, const float* theta,
                           const double* d_image, double* grad, double* grad_terms, double* dX_out,
                           double* grad_mass, double* dX_mass) {
  Render r(cfg, sc, theta);
  int rc = prepare(r);
  if (rc) return rc;
  const int nt = nthreads(cfg);
  const int terms = cfg->terms ? cfg->terms : 7;
  const int npx = cfg->W * cfg->H;
  const int P = r.lay.total;
  std::vector<double> total(P, 0.0), tmass(P, 0.0);
  if (grad_terms) std::fill(grad_terms, grad_terms + 3 * P, 0.0);
  std::vector<double> dXtot(3 * r.V, 0.0), aXtot(3 * r.V, 0.0);
  for (int term = 0; term < 3; ++term) {
    int bit = 1 << term;
    if (!(terms & bit)) continue;
    if (cfg->shade_mode == SHADE_FLAT && bit != TERM_PEDGE) continue;
    std::vector<Grad> G(nt);
    for (auto& g : G) g.init(r.V, r.NL);
    parallel_for(npx, nt, [&](int p, int tid) {
      int px = p % cfg->W, py = p / cfg->W;
      const double* dI = d_image + 3 * (size_t)p;
      bool zero = dI[0] == 0.0 && dI[1] == 0.0 && dI[2] == 0.0;
      for (int s = 0; s < cfg->spp; ++s) {
        if (bit == TERM_PEDGE) { primary_edge_sample(r, (uint32_t)p, s, d_image, G[tid]); continue; }
        if (zero) continue;
        float d[3];
        uint32_t pp;
        sample_ray(r, px, py, s, d, &pp);
        Hit h = closest_hit(r, r.cam_o, d);
        if (h.f < 0) continue;
        if (bit == TERM_INTERIOR) {
          interior_sample(r, r.cam_o, d, h, pp, s, dI, G[tid]);
        } else {
          double w[3] = {dI[0] / cfg->spp, dI[1] / cfg->spp, dI[2] / cfg->spp};
          for (int j = 0; j < r.NL; ++j)
            if (r.light_on(j)) shadow_edge_sample(r, r.cam_o, d, h, pp, s, j, w, G[tid]);
        }
      }
    });
    Grad tot;
    tot.init(r.V, r.NL);
    for (auto& gg : G) tot.add(gg);
    std::vector<double> dX = tot.dX, aX = tot.aX;
    normals_adjoint(r, tot.dN, dX, tot.aN, aX);
    for (int i = 0; i < 3 * r.V; ++i) { dXtot[i] += dX[i]; aXtot[i] += aX[i]; }
    std::vector<double> part(P), pmass(P);
    geometry_adjoint(r, tot, dX, aX, part.data(), pmass.data());
    for (int i = 0; i < P; ++i) { total[i] += part[i]; tmass[i] += pmass[i]; }
    if (grad_terms) std::memcpy(grad_terms + term * P, part.data(), P * sizeof(double));
  }
  std::memcpy(grad, total.data(), P * sizeof(double));
  if (dX_out) std::memcpy(dX_out, dXtot.data(), 3 * r.V * sizeof(double));
  if (grad_mass) std::memcpy(grad_mass, tmass.data(), P * sizeof(double));
  if (dX_mass) std::memcpy(dX_mass, aXtot.data(), 3 * r.V * sizeof(double));
  return 0;
}

// E_data + w1 E_prior + w2 E_light (Eq. 1), d_image = dE/d image and the
// regulariser gradients with respect to theta (grad_reg[P], or NULL).
double oracle_loss(const OracleConfig* cfg, const OracleScene* sc, const float* theta,
                   const float* image, const float* target, const uint8_t* mask, const float* m,
                   float w1, float w2, double* d_image, double* grad_reg) {
  Layout lay(*sc, cfg->n_lights);
  const int npx = cfg->W * cfg->H;
  double Ed = 0.0;
  for (int p = 0; p < npx; ++p) {
    bool in = mask ? mask[p] != 0 : true;
    for (int c = 0; c < 3; ++c) {
      double diff = (double)image[3 * p + c] - (double)target[3 * p + c];
      if (in) Ed += diff * diff;
      if (d_image) d_image[3 * p + c] = in ? 2.0 * diff : 0.0;
    }
  }
  double Ep = 0.0;
  for (int i = 0; i < lay.cspec; ++i) Ep += (double)theta[i] * theta[i];
  // E_light = sum_j |l_j - m_j|^2.  The text leaves open what m_j averages;
  // light_prior 0 takes the given m (zero when null) and treats it as a
  // constant, 1 the mean of the N lights in each channel, 2 the mean of
  // light j's three channels.  For 1 and 2, J[i][k] = dm_i/dl_k enters the
  // derivative: dE/dl_k = 2 (l_k - m_k) - sum_i 2 (l_i - m_i) J[i][k].
  const int NV = 3 * cfg->n_lights;
  const float* l = theta + lay.lights;
  std::vector<double> mv(NV, 0.0), J((size_t)NV * NV, 0.0);
  for (int i = 0; i < NV; ++i) {
    const int j = i / 3, c = i % 3;
    if (cfg->light_prior == 1) {
      for (int k = 0; k < cfg->n_lights; ++k) {
        mv[i] += (double)l[3 * k + c];
        J[(size_t)i * NV + 3 * k + c] = 1.0 / cfg->n_lights;
      }
      mv[i] /= cfg->n_lights;
    } else if (cfg->light_prior == 2) {
      for (int c2 = 0; c2 < 3; ++c2) {
        mv[i] += (double)l[3 * j + c2];
        J[(size_t)i * NV + 3 * j + c2] = 1.0 / 3.0;
      }
      mv[i] /= 3.0;
    } else {
      mv[i] = m ? (double)m[i] : 0.0;
    }
  }
  double El = 0.0;
  for (int i = 0; i < NV; ++i) {
    double diff = (double)l[i] - mv[i];
    El += diff * diff;
  }
  if (grad_reg) {
    for (int i = 0; i < lay.total; ++i) grad_reg[i] = 0.0;
    for (int i = 0; i < lay.cspec; ++i) grad_reg[i] = 2.0 * w1 * theta[i];
    for (int k = 0; k < NV; ++k) {
      double g = 2.0 * ((double)l[k] - mv[k]);
      for (int i = 0; i < NV; ++i) g -= 2.0 * ((double)l[i] - mv[i]) * J[(size_t)i * NV + k];
      grad_reg[lay.lights + k] = w2 * g;
    }
  }
  return Ed + (double)w1 * Ep + (double)w2 * El;
}

// --- point-level hooks used by the closed-form pins ---------------------------

// Unshadowed one-light estimate A * h(x, y) at light point (u2, u3) of light j,
// for a surface point with explicit shading frame.
void oracle_light_estimate(const OracleConfig* cfg, const double* x, const double* ns, const double* wo,
                           const double* rho, double cs, const float* lrgb, int32_t j, float u2, float u3,
                           double* out) {
  std::vector<Light> L = light_stage(cfg->n_lights, cfg->light_radius, cfg->light_layout);
  float y[3];
  light_point32(L[j], cfg->light_side, u2, u3, y);
  V3<double> hv = light_integrand<double>(V3<double>(x[0], x[1], x[2]), V3<double>(ns[0], ns[1], ns[2]),
                                          V3<double>(wo[0], wo[1], wo[2]), V3<double>(rho[0], rho[1], rho[2]), cs,
                                          V3<double>(lrgb[0], lrgb[1], lrgb[2]), widen(y), widen(L[j].dl),
                                          brdf_of(*cfg));
  double A = (double)cfg->light_side * cfg->light_side;
  out[0] = hv.x * A; out[1] = hv.y * A; out[2] = hv.z * A;
}

// BRDF value f_r(wi, wo) for a unit normal, used by the energy/reciprocity pins.
void oracle_brdf(const OracleConfig* cfg, const double* n, const double* wi, const double* wo, double rho,
                 double cs, double* out) {
  // light_integrand with y = x + wi (unit distance), cos_y = 1 via dl = wi.
  V3<double> x(0, 0, 0);
  V3<double> hv = light_integrand<double>(x, V3<double>(n[0], n[1], n[2]), V3<double>(wo[0], wo[1], wo[2]),
                                          V3<double>(rho, rho, rho), cs, V3<double>(1, 1, 1),
                                          V3<double>(wi[0], wi[1], wi[2]), V3<double>(wi[0], wi[1], wi[2]),
                                          brdf_of(*cfg));
  double ci = n[0] * wi[0] + n[1] * wi[1] + n[2] * wi[2];
  *out = ci > 0 ? hv.x / ci : 0.0;
}

// Visibility-weighted one-light estimate at the hit of an explicit ray.
int oracle_point_shade(const OracleConfig* cfg, const OracleScene* sc, const float* theta, const float* o,
                       const float* d, int32_t j, float u2, float u3, double* out, int32_t* hit_face) {
  Render r(cfg, sc, theta);
  int rc = prepare(r);
  if (rc) return rc;
  Hit h = closest_hit(r, o, d);
  *hit_face = h.f;
  out[0] = out[1] = out[2] = 0.0;
  if (h.f < 0) return 0;
  int flip = face_flip(r, h.f, d);
  float x32[3], y32[3];
  hit_point32(o, d, h.t, x32);
  light_point32(r.lights[j], cfg->light_side, u2, u3, y32);
  if (!visible(r, x32, y32, h.f, flip)) return 0;
  Surf<double> S = surface_value(r, h.f, o, d, flip);
  double cs = cspec_value(r, S.u, S.v);
  const float* l = r.lightrgb(j);
  V3<double> hv = light_integrand<double>(S.x, S.ns, S.wo, S.rho, cs, V3<double>(l[0], l[1], l[2]), widen(y32),
                                          widen(r.lights[j].dl), brdf_of(*cfg));
  double A = (double)cfg->light_side * cfg->light_side;
  out[0] = hv.x * A; out[1] = hv.y * A; out[2] = hv.z * A;
  return 0;
}

// Shadow-edge estimate for an explicit ray and light, averaged over n_rep
// independent selections (sample index s = 0..n_rep-1): accumulates
// sum_s wrgb . d(estimate_s)/dX into dX[V*3] and returns the number of
// selections that found a candidate edge.
int oracle_shadow_edge_point(const OracleConfig* cfg, const OracleScene* sc, const float* theta, const float* o,
                             const float* d, int32_t j, const double* wrgb, int32_t n_rep, double* dX) {
  Render r(cfg, sc, theta);
  int rc = prepare(r);
  if (rc) return rc;
  Hit h = closest_hit(r, o, d);
  if (h.f < 0) return 0;
  const int nt = nthreads(cfg);
  std::vector<Grad> G(nt);
  for (auto& g : G) g.init(r.V, r.NL);
  parallel_for(n_rep, nt, [&](int s, int tid) { shadow_edge_sample(r, o, d, h, 0u, s, j, wrgb, G[tid]); });
  for (int i = 0; i < 3 * r.V; ++i) {
    double a = 0;
    for (auto& g : G) a += g.dX[i];
    dX[i] = a;
  }
  return 0;
}

}  // extern "C"
