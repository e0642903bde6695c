// Adam on the packed parameter vector, for the inverse-rendering loop
// (Optimization paragraph: argmin of Eq. 1 over alpha, beta, delta, c_spec,
// [R t] and the lights, optimised in stages).
#include "kernels.cuh"

namespace fr {

// theta -= lr_i * mhat / (sqrt(vhat) + eps) (Kingma & Ba 2015) with the FP64
// gradient; lr_i = 0 freezes parameter i.  After the step, light intensities
// are kept >= 0 and specular-map texels in [0, 1] (a light cannot emit
// negative radiance; the specular albedo is a reflectance).
__global__ void k_adam_theta(int n, float* __restrict__ theta, const double* __restrict__ grad,
                             float* __restrict__ m, float* __restrict__ v, const float* __restrict__ lr, float c1,
                             float c2, int off_cspec, int n_cspec, int off_lights) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float li = lr[i];
  if (li == 0.0f) return;
  float g = (float)grad[i];
  float mi = 0.9f * m[i] + 0.1f * g;
  float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  float t = theta[i] - li * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  if (i >= off_lights) t = fmaxf(t, 0.0f);
  else if (i >= off_cspec && i < off_cspec + n_cspec) t = fminf(fmaxf(t, 0.0f), 1.0f);
  theta[i] = t;
}

}  // namespace fr
