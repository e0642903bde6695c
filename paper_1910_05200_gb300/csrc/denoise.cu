// Per-pixel MLP denoiser for radiance and for the image-space adjoint.
//
// The paper names the sampling rate as its limitation (Results and
// Conclusion: few samples give a noisy render, many samples a slow
// optimisation).  This network maps a pixel's 14 features from a low-spp
// render to its radiance:
//   y = rgb + cov s_out (W4 h3 + b4),  h_l = relu(W_l h_{l-1} + b_l),  h_0 = (t(x) - mu) * is,
// 14 -> 64 -> 64 -> 64 -> 3, FP16 weights and activations, FP32 accumulation.
// t is the identity except for feature 12 (luminance variance), which enters
// as its square root; mu, is and s_out are fixed standardisation constants
// stored with the weights (training leaves them unchanged: their gradient is
// zero); cov is feature 13 (the fraction of samples that hit the face), so
// background pixels pass through unchanged.  The adjoint of the renderer's
// image is J^T d with J = dy/drgb (the other features are treated as
// constants).
//
// Master weights (FP32, packed, nn.Linear layout [out][in]):
//   W1[64][14] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[3][64] b4[3] mu[14] is[14] s_out
#include <cuda_fp16.h>

#include "kernels.cuh"

namespace fr {

namespace {

constexpr int NH = 64, NIN = 14, NOUT = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NH, OFF_W4 = OFF_B3 + NH, OFF_B4 = OFF_W4 + NOUT * NH,
              OFF_MU = OFF_B4 + NOUT, OFF_IS = OFF_MU + NIN, OFF_SOUT = OFF_IS + NIN, NW = OFF_SOUT + 1;

// Shared-memory images of the FP16 weights in the layouts the fragments need
// (B operands are "col": for each output column n, the K values contiguous).
// Rows are padded (16 -> 24, 64 -> 72 halves) so that the 8 rows one
// fragment load touches fall in distinct shared-memory banks.
constexpr int LD16 = 24, LD64 = 72;
struct MlpSmem {
  __half w1[NH][LD16];    // forward L1: n = hidden, k = input (14 padded to 16)
  __half w2[NH][LD64];    // forward L2: [out][in]
  __half w3[NH][LD64];
  __half w4[8][LD64];     // forward L4: 3 outputs padded to 8
  __half w4t[NH][LD16];   // adjoint: d h3 = W4^T dy : n = hidden, k = output (3 padded to 16)
  __half w3t[NH][LD64];   // adjoint: [in][out]
  __half w2t[NH][LD64];
  __half w1t[16][LD64];   // adjoint: n = input (only 0..7 used), k = hidden
  float b1[NH], b2[NH], b3[NH], b4[8];
  float mu[16], is[16], sout;
};

FR_DEV uint32_t pack_h2(float lo, float hi) {
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}

FR_DEV void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragment of an [N][K] FP16 matrix (row n holds K contiguous values):
// b0 = (k = k0+2t, k0+2t+1; n = n0+g), b1 = (k = k0+2t+8, +9; n = n0+g).
FR_DEV void bfrag(const __half* M, int ldk, int n0, int k0, int lane, uint32_t& b0, uint32_t& b1) {
  int g = lane >> 2, t = lane & 3;
  const __half* row = M + (n0 + g) * ldk + k0 + 2 * t;
  b0 = *reinterpret_cast<const uint32_t*>(row);
  b1 = *reinterpret_cast<const uint32_t*>(row + 8);
}

__device__ void load_weights(MlpSmem& S, const float* __restrict__ w) {
  for (int i = threadIdx.x; i < NH * 16; i += blockDim.x) {
    int n = i / 16, k = i % 16;
    S.w1[n][k] = __float2half_rn(k < NIN ? w[OFF_W1 + n * NIN + k] : 0.0f);
    S.w1t[k][n] = S.w1[n][k];
  }
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
    int n = i / NH, k = i % NH;
    __half a = __float2half_rn(w[OFF_W2 + i]), b = __float2half_rn(w[OFF_W3 + i]);
    S.w2[n][k] = a; S.w2t[k][n] = a;
    S.w3[n][k] = b; S.w3t[k][n] = b;
  }
  for (int i = threadIdx.x; i < 8 * NH; i += blockDim.x) {
    int n = i / NH, k = i % NH;
    S.w4[n][k] = __float2half_rn(n < NOUT ? w[OFF_W4 + n * NH + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH * 16; i += blockDim.x) {
    int n = i / 16, k = i % 16;   // n = hidden unit, k = output
    S.w4t[n][k] = __float2half_rn(k < NOUT ? w[OFF_W4 + k * NH + n] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    S.b1[i] = w[OFF_B1 + i]; S.b2[i] = w[OFF_B2 + i]; S.b3[i] = w[OFF_B3 + i];
  }
  for (int i = threadIdx.x; i < 8; i += blockDim.x) S.b4[i] = i < NOUT ? w[OFF_B4 + i] : 0.0f;
  for (int i = threadIdx.x; i < 16; i += blockDim.x) {
    S.mu[i] = i < NIN ? w[OFF_MU + i] : 0.0f;
    S.is[i] = i < NIN ? w[OFF_IS + i] : 0.0f;
  }
  if (threadIdx.x == 0) S.sout = w[OFF_SOUT];
}

FR_DEV float feature(const MlpSmem& S, const float* __restrict__ x, int k) {
  if (k >= NIN) return 0.0f;
  float v = x[k];
  if (k == 12) v = sqrtf(fmaxf(v, 0.0f));
  return (v - S.mu[k]) * S.is[k];
}

// One hidden layer on the tensor cores: C[8 n-tiles] = A[kchunks] x W^T (+ bias),
// ReLU, and repack as FP16 A fragments for the next layer.  mask bit
// (4 * nt + r) records whether accumulator r of n-tile nt was positive.
template <int KCH>
FR_DEV void hidden_layer(const uint32_t (*A)[4], const __half* W, int ldk, const float* bias, int lane,
                         uint32_t (*Aout)[4], uint32_t& mask) {
  float C[8][4];
  int t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float b0 = bias[8 * nt + 2 * t], b1 = bias[8 * nt + 2 * t + 1];
    C[nt][0] = b0; C[nt][1] = b1; C[nt][2] = b0; C[nt][3] = b1;
#pragma unroll
    for (int kc = 0; kc < KCH; ++kc) {
      uint32_t bb0, bb1;
      bfrag(W, ldk, 8 * nt, 16 * kc, lane, bb0, bb1);
      mma16816(C[nt], A[kc], bb0, bb1);
    }
  }
  mask = 0;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (C[nt][r] > 0.0f) mask |= 1u << (4 * nt + r);
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    Aout[kc][0] = pack_h2(fmaxf(C[2 * kc][0], 0.0f), fmaxf(C[2 * kc][1], 0.0f));
    Aout[kc][1] = pack_h2(fmaxf(C[2 * kc][2], 0.0f), fmaxf(C[2 * kc][3], 0.0f));
    Aout[kc][2] = pack_h2(fmaxf(C[2 * kc + 1][0], 0.0f), fmaxf(C[2 * kc + 1][1], 0.0f));
    Aout[kc][3] = pack_h2(fmaxf(C[2 * kc + 1][2], 0.0f), fmaxf(C[2 * kc + 1][3], 0.0f));
  }
}

// Adjoint of a hidden layer: G[8 n-tiles] = A[KCH chunks] x Wt^T, masked by
// the forward ReLU, repacked as FP16 A fragments.
template <int KCH>
FR_DEV void adjoint_layer(const uint32_t (*A)[4], const __half* Wt, int ldk, uint32_t mask, int lane,
                          uint32_t (*Aout)[4]) {
  float C[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    C[nt][0] = C[nt][1] = C[nt][2] = C[nt][3] = 0.0f;
#pragma unroll
    for (int kc = 0; kc < KCH; ++kc) {
      uint32_t bb0, bb1;
      bfrag(Wt, ldk, 8 * nt, 16 * kc, lane, bb0, bb1);
      mma16816(C[nt], A[kc], bb0, bb1);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (!((mask >> (4 * nt + r)) & 1u)) C[nt][r] = 0.0f;
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    Aout[kc][0] = pack_h2(C[2 * kc][0], C[2 * kc][1]);
    Aout[kc][1] = pack_h2(C[2 * kc][2], C[2 * kc][3]);
    Aout[kc][2] = pack_h2(C[2 * kc + 1][0], C[2 * kc + 1][1]);
    Aout[kc][3] = pack_h2(C[2 * kc + 1][2], C[2 * kc + 1][3]);
  }
}

}  // namespace

// Inference and (optionally) the input adjoint.  One warp = 16 pixels
// (rows), 8 warps per block.  aov[n*14] features; out[n*3] = y; with d_out:
// d_rgb[n*3] = J^T d_out, where J = dy/d(rgb features).
__global__ void __launch_bounds__(256) k_mlp_infer(int n_pix, const float* __restrict__ w,
                                                   const float* __restrict__ aov, float* __restrict__ out,
                                                   const float* __restrict__ d_out, float* __restrict__ d_rgb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  load_weights(S, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int row0 = (blockIdx.x * 8 + warp) * 16;
  if (row0 >= n_pix) return;
  const int ra = row0 + g, rb = row0 + g + 8;
  const bool va = ra < n_pix, vb = rb < n_pix;
  // input A fragment (16 features, K = 16)
  uint32_t X[1][4];
  {
    const float* xa = aov + 14 * (size_t)(va ? ra : 0);
    const float* xb = aov + 14 * (size_t)(vb ? rb : 0);
    float a0 = va ? feature(S, xa, 2 * t) : 0.f, a1 = va ? feature(S, xa, 2 * t + 1) : 0.f;
    float b0 = vb ? feature(S, xb, 2 * t) : 0.f, b1 = vb ? feature(S, xb, 2 * t + 1) : 0.f;
    float a2 = va ? feature(S, xa, 2 * t + 8) : 0.f, a3 = va ? feature(S, xa, 2 * t + 9) : 0.f;
    float b2 = vb ? feature(S, xb, 2 * t + 8) : 0.f, b3 = vb ? feature(S, xb, 2 * t + 9) : 0.f;
    X[0][0] = pack_h2(a0, a1); X[0][1] = pack_h2(b0, b1); X[0][2] = pack_h2(a2, a3); X[0][3] = pack_h2(b2, b3);
  }
  uint32_t H1[4][4], H2[4][4], H3[4][4];
  uint32_t m1, m2, m3;
  hidden_layer<1>(X, &S.w1[0][0], LD16, S.b1, lane, H1, m1);
  hidden_layer<4>(H1, &S.w2[0][0], LD64, S.b2, lane, H2, m2);
  hidden_layer<4>(H2, &S.w3[0][0], LD64, S.b3, lane, H3, m3);
  float Y[4];
  Y[0] = S.b4[2 * t]; Y[1] = S.b4[2 * t + 1]; Y[2] = Y[0]; Y[3] = Y[1];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    uint32_t bb0, bb1;
    bfrag(&S.w4[0][0], LD64, 0, 16 * kc, lane, bb0, bb1);
    mma16816(Y, H3[kc], bb0, bb1);
  }
  // lanes with t = 0 hold outputs 0, 1 and t = 1 holds output 2 (rows g, g+8)
  if (t < 2) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int row = r == 0 ? ra : rb;
      bool v = r == 0 ? va : vb;
      if (!v) continue;
      for (int q = 0; q < 2; ++q) {
        int c = 2 * t + q;
        if (c < NOUT) {
          const float* xr = aov + 14 * (size_t)row;
          out[3 * (size_t)row + c] = xr[c] + xr[13] * S.sout * Y[2 * r + q];
        }
      }
    }
  }
  if (!d_out) return;
  // adjoint: scale each pixel's d_out to unit max so FP16 keeps its digits
  float da[3] = {0, 0, 0}, db[3] = {0, 0, 0};
  if (va) for (int c = 0; c < 3; ++c) da[c] = d_out[3 * (size_t)ra + c];
  if (vb) for (int c = 0; c < 3; ++c) db[c] = d_out[3 * (size_t)rb + c];
  float sa = fmaxf(fabsf(da[0]), fmaxf(fabsf(da[1]), fabsf(da[2])));
  float sb = fmaxf(fabsf(db[0]), fmaxf(fabsf(db[1]), fabsf(db[2])));
  float ia = sa > 0.f ? 1.0f / sa : 0.f, ib = sb > 0.f ? 1.0f / sb : 0.f;
  uint32_t D[1][4];
  {
    float a0 = 2 * t < 3 ? da[2 * t] * ia : 0.f, a1 = 2 * t + 1 < 3 ? da[2 * t + 1] * ia : 0.f;
    float b0 = 2 * t < 3 ? db[2 * t] * ib : 0.f, b1 = 2 * t + 1 < 3 ? db[2 * t + 1] * ib : 0.f;
    D[0][0] = pack_h2(a0, a1); D[0][1] = pack_h2(b0, b1); D[0][2] = 0u; D[0][3] = 0u;
  }
  uint32_t G3[4][4], G2[4][4], G1[4][4];
  adjoint_layer<1>(D, &S.w4t[0][0], LD16, m3, lane, G3);
  adjoint_layer<4>(G3, &S.w3t[0][0], LD64, m2, lane, G2);
  adjoint_layer<4>(G2, &S.w2t[0][0], LD64, m1, lane, G1);
  float GX[4] = {0, 0, 0, 0};
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    uint32_t bb0, bb1;
    bfrag(&S.w1t[0][0], LD64, 0, 16 * kc, lane, bb0, bb1);
    mma16816(GX, G1[kc], bb0, bb1);
  }
  if (t < 2) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      int row = r == 0 ? ra : rb;
      bool v = r == 0 ? va : vb;
      if (!v) continue;
      float sc = r == 0 ? sa : sb;
      const float* dd = r == 0 ? da : db;
      for (int q = 0; q < 2; ++q) {
        int c = 2 * t + q;
        // residual + MLP (chain through the output scale and the input standardisation)
        if (c < NOUT)
          d_rgb[3 * (size_t)row + c] = dd[c] + GX[2 * r + q] * sc * S.sout * S.is[c] * aov[14 * (size_t)row + 13];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Training.  Scratch layout per pixel (FP32), written by k_mlp_train_tc and
// reduced by k_mlp_wgrad:
//   h0[16] h1[64] h2[64] h3[64] | g1[64] g2[64] g3[64] g4[8]
// (activations as the FP16 values the layers consumed; gradients with
// respect to each layer's pre-activation).
constexpr int TR_STRIDE = 16 + 3 * NH + 3 * NH + 8;

// One training pass on the tensor cores: one warp = 16 pixels, the forward
// through the fragments of k_mlp_infer, the MSE loss against target, then the MSE gradient
// g4 = 2 e cov s_out / n_pix and its chain through W4^T, W3^T, W2^T with the
// forward ReLU masks.  Each pixel's g4 is scaled to unit maximum before it is
// rounded to FP16 (the gradients are of order 1/n_pix, below FP16's range)
// and scaled back when stored.  Activations and gradients go to the scratch
// for k_mlp_wgrad.
namespace {
// A fragment (packed halves) of 4 k-chunks -> the 64 values of rows g and g+8.
FR_DEV void store_frag_rows(const uint32_t (*A)[4], int t, float* ra, float* rb) {
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __half2 h = *reinterpret_cast<const __half2*>(&A[kc][q]);
      const int col = 16 * kc + 2 * t + ((q & 2) ? 8 : 0);
      float* r = (q & 1) ? rb : ra;
      if (r) { r[col] = __low2float(h); r[col + 1] = __high2float(h); }
    }
  }
}

// adjoint_layer that also stores the FP32 gradients (times the pixel scales
// sa, sb) of rows g and g+8.
template <int KCH>
FR_DEV void adjoint_layer_store(const uint32_t (*A)[4], const __half* Wt, int ldk, uint32_t mask, int lane,
                                uint32_t (*Aout)[4], float* ra, float* rb, float sa, float sb) {
  float C[8][4];
  const int t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    C[nt][0] = C[nt][1] = C[nt][2] = C[nt][3] = 0.0f;
#pragma unroll
    for (int kc = 0; kc < KCH; ++kc) {
      uint32_t bb0, bb1;
      bfrag(Wt, ldk, 8 * nt, 16 * kc, lane, bb0, bb1);
      mma16816(C[nt], A[kc], bb0, bb1);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (!((mask >> (4 * nt + r)) & 1u)) C[nt][r] = 0.0f;
    const int col = 8 * nt + 2 * t;
    if (ra) { ra[col] = C[nt][0] * sa; ra[col + 1] = C[nt][1] * sa; }
    if (rb) { rb[col] = C[nt][2] * sb; rb[col + 1] = C[nt][3] * sb; }
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    Aout[kc][0] = pack_h2(C[2 * kc][0], C[2 * kc][1]);
    Aout[kc][1] = pack_h2(C[2 * kc][2], C[2 * kc][3]);
    Aout[kc][2] = pack_h2(C[2 * kc + 1][0], C[2 * kc + 1][1]);
    Aout[kc][3] = pack_h2(C[2 * kc + 1][2], C[2 * kc + 1][3]);
  }
}
}  // namespace

__global__ void __launch_bounds__(256) k_mlp_train_tc(int n_pix, const float* __restrict__ w,
                                                      const float* __restrict__ aov, const float* __restrict__ target,
                                                      float* __restrict__ scratch, double* __restrict__ loss) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  __shared__ double red[8];
  load_weights(S, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int row0 = (blockIdx.x * 8 + warp) * 16;
  const int ra = row0 + g, rb = row0 + g + 8;
  const bool va = ra < n_pix, vb = rb < n_pix;
  double l = 0.0;
  if (row0 < n_pix) {                        // uniform over the warp
    float* sa_row = va ? scratch + (size_t)ra * TR_STRIDE : nullptr;
    float* sb_row = vb ? scratch + (size_t)rb * TR_STRIDE : nullptr;
    uint32_t X[1][4];
    {
      const float* xa = aov + 14 * (size_t)(va ? ra : 0);
      const float* xb = aov + 14 * (size_t)(vb ? rb : 0);
      float a0 = va ? feature(S, xa, 2 * t) : 0.f, a1 = va ? feature(S, xa, 2 * t + 1) : 0.f;
      float b0 = vb ? feature(S, xb, 2 * t) : 0.f, b1 = vb ? feature(S, xb, 2 * t + 1) : 0.f;
      float a2 = va ? feature(S, xa, 2 * t + 8) : 0.f, a3 = va ? feature(S, xa, 2 * t + 9) : 0.f;
      float b2 = vb ? feature(S, xb, 2 * t + 8) : 0.f, b3 = vb ? feature(S, xb, 2 * t + 9) : 0.f;
      X[0][0] = pack_h2(a0, a1); X[0][1] = pack_h2(b0, b1); X[0][2] = pack_h2(a2, a3); X[0][3] = pack_h2(b2, b3);
      // h0 (the FP16-rounded standardised features), columns 2t, 2t+1, 2t+8, 2t+9
      const uint32_t q[4] = {X[0][0], X[0][1], X[0][2], X[0][3]};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        __half2 h = *reinterpret_cast<const __half2*>(&q[i]);
        float* r = (i & 1) ? sb_row : sa_row;
        const int col = 2 * t + ((i & 2) ? 8 : 0);
        if (r) { r[col] = __low2float(h); r[col + 1] = __high2float(h); }
      }
    }
    uint32_t H1[4][4], H2[4][4], H3[4][4];
    uint32_t m1, m2, m3;
    hidden_layer<1>(X, &S.w1[0][0], LD16, S.b1, lane, H1, m1);
    hidden_layer<4>(H1, &S.w2[0][0], LD64, S.b2, lane, H2, m2);
    hidden_layer<4>(H2, &S.w3[0][0], LD64, S.b3, lane, H3, m3);
    store_frag_rows(H1, t, sa_row ? sa_row + 16 : nullptr, sb_row ? sb_row + 16 : nullptr);
    store_frag_rows(H2, t, sa_row ? sa_row + 16 + NH : nullptr, sb_row ? sb_row + 16 + NH : nullptr);
    store_frag_rows(H3, t, sa_row ? sa_row + 16 + 2 * NH : nullptr, sb_row ? sb_row + 16 + 2 * NH : nullptr);
    float Y[4];
    Y[0] = S.b4[2 * t]; Y[1] = S.b4[2 * t + 1]; Y[2] = Y[0]; Y[3] = Y[1];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      uint32_t bb0, bb1;
      bfrag(&S.w4[0][0], LD64, 0, 16 * kc, lane, bb0, bb1);
      mma16816(Y, H3[kc], bb0, bb1);
    }
    // output gradient of rows g (r = 0) and g + 8 (r = 1), channels 2t, 2t+1
    float g4[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int row = r == 0 ? ra : rb;
      const bool v = r == 0 ? va : vb;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c = 2 * t + q;
        if (!v || c >= NOUT) continue;
        const float* xr = aov + 14 * (size_t)row;
        const float y = xr[c] + xr[13] * S.sout * Y[2 * r + q];
        const float e = y - target[3 * (size_t)row + c];
        l += (double)e * e;
        g4[r][q] = 2.0f * e * xr[13] * S.sout / (float)n_pix;
      }
    }
    // per-pixel scale of g4 (a row's three channels live in lanes t = 0, 1)
    float sa = fmaxf(fabsf(g4[0][0]), fabsf(g4[0][1])), sb = fmaxf(fabsf(g4[1][0]), fabsf(g4[1][1]));
    sa = fmaxf(sa, __shfl_xor_sync(0xffffffffu, sa, 1));
    sb = fmaxf(sb, __shfl_xor_sync(0xffffffffu, sb, 1));
    sa = fmaxf(sa, __shfl_xor_sync(0xffffffffu, sa, 2));
    sb = fmaxf(sb, __shfl_xor_sync(0xffffffffu, sb, 2));
    const float ia = sa > 0.f ? 1.0f / sa : 0.f, ib = sb > 0.f ? 1.0f / sb : 0.f;
    if (t < 2) {
      float* ga = sa_row ? sa_row + 16 + 6 * NH : nullptr;
      float* gb = sb_row ? sb_row + 16 + 6 * NH : nullptr;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (ga) ga[2 * t + q] = g4[0][q];
        if (gb) gb[2 * t + q] = g4[1][q];
      }
      if (t == 1) {
        for (int c = 4; c < 8; ++c) {
          if (ga) ga[c] = 0.f;
          if (gb) gb[c] = 0.f;
        }
      }
    }
    uint32_t D[1][4];
    D[0][0] = pack_h2(g4[0][0] * ia, g4[0][1] * ia);
    D[0][1] = pack_h2(g4[1][0] * ib, g4[1][1] * ib);
    D[0][2] = 0u; D[0][3] = 0u;
    uint32_t G3[4][4], G2[4][4], G1[4][4];
    adjoint_layer_store<1>(D, &S.w4t[0][0], LD16, m3, lane, G3, sa_row ? sa_row + 16 + 5 * NH : nullptr,
                           sb_row ? sb_row + 16 + 5 * NH : nullptr, sa, sb);
    adjoint_layer_store<4>(G3, &S.w3t[0][0], LD64, m2, lane, G2, sa_row ? sa_row + 16 + 4 * NH : nullptr,
                           sb_row ? sb_row + 16 + 4 * NH : nullptr, sa, sb);
    adjoint_layer_store<4>(G2, &S.w2t[0][0], LD64, m1, lane, G1, sa_row ? sa_row + 16 + 3 * NH : nullptr,
                           sb_row ? sb_row + 16 + 3 * NH : nullptr, sa, sb);
    (void)G1;
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if (lane == 0) red[warp] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    atomicAdd(loss, s / (double)n_pix);
  }
}

// Weight gradient of one layer: dW[n][k] = sum_p g[p][n] h[p][k], db[n] = sum_p g[p][n].
// Each block reduces a chunk of pixels; each thread owns some (n, k) entries.
__global__ void k_mlp_wgrad(int n_pix, const float* __restrict__ scratch, int g_off, int h_off, int N, int K,
                            int Kw, float* __restrict__ dW, float* __restrict__ db, int chunk) {
  extern __shared__ float sh[];   // [chunk][N + K]
  int p0 = blockIdx.x * chunk;
  int np = min(chunk, n_pix - p0);
  if (np <= 0) return;
  for (int i = threadIdx.x; i < np * (N + K); i += blockDim.x) {
    int p = i / (N + K), j = i % (N + K);
    const float* sc = scratch + (size_t)(p0 + p) * TR_STRIDE;
    sh[i] = j < N ? sc[g_off + j] : sc[h_off + (j - N)];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * (K + 1); e += blockDim.x) {
    int n = e / (K + 1), k = e % (K + 1);
    float acc = 0.f;
    for (int p = 0; p < np; ++p) {
      const float* row = sh + p * (N + K);
      acc += row[n] * (k < K ? row[N + k] : 1.0f);
    }
    if (k < K) { if (k < Kw) atomicAdd(&dW[n * Kw + k], acc); }
    else atomicAdd(&db[n], acc);
  }
}

// Adam (Kingma & Ba 2015) on the FP32 master weights.
__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

int mlp_n_weights() { return NW; }
size_t mlp_smem_bytes() { return sizeof(MlpSmem); }
int mlp_train_stride() { return TR_STRIDE; }
void mlp_layer_offsets(int* off) {
  off[0] = OFF_W1; off[1] = OFF_B1; off[2] = OFF_W2; off[3] = OFF_B2;
  off[4] = OFF_W3; off[5] = OFF_B3; off[6] = OFF_W4; off[7] = OFF_B4;
}

}  // namespace fr
