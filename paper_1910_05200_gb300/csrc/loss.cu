// Eq. 1 of the Optimization paragraph: E_data + w1 E_prior + w2 E_light.
#include "kernels.cuh"

namespace fr {

// E_data over masked pixels and d_image = 2 mask (image - target); FP64
// block reduction, one atomic per block.
__global__ void k_loss_data(int n_pix, const float* __restrict__ image, const float* __restrict__ target,
                            const uint8_t* __restrict__ mask, double* __restrict__ loss, float* __restrict__ d_image) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n_pix; p += gridDim.x * blockDim.x) {
    bool in = mask ? mask[p] != 0 : true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double diff = (double)image[3 * p + c] - (double)target[3 * p + c];
      if (in) acc += diff * diff;
      if (d_image) d_image[3 * p + c] = in ? (float)(2.0 * diff) : 0.0f;
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s);
  }
}

// w1 (|alpha|^2 + |beta|^2 + |delta|^2) + w2 sum_j |l_j - m_j|^2 and their
// gradients (value added to loss, gradient to grad, each when non-null).
// One block.  When m follows
// the lights (prior 1, 2) the gradient through m vanishes: it is minus the
// mean of deviations that sum to zero.
__global__ void k_loss_reg(const float* __restrict__ theta, int n_prior, int off_lights, int n_light_vals,
                           int prior, const float* __restrict__ m, float w1, float w2, double* __restrict__ loss,
                           double* __restrict__ grad) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n_prior; i += blockDim.x) {
    double t = theta[i];
    acc += (double)w1 * t * t;
    if (grad) grad[i] += 2.0 * (double)w1 * t;
  }
  for (int i = threadIdx.x; i < n_light_vals; i += blockDim.x) {
    double d = (double)theta[off_lights + i] - light_prior_mean(theta + off_lights, n_light_vals / 3, prior, m, i);
    acc += (double)w2 * d * d;
    if (grad) grad[off_lights + i] += 2.0 * (double)w2 * d;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    if (loss) atomicAdd(loss, s);
  }
}

}  // namespace fr
