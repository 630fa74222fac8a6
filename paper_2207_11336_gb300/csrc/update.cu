// Image-domain kernels outside the fused FFT epilogue: the plain Haar denoiser
// applied on its own (App. B, one-level orthonormal Haar + positivity), FP64
// norm reductions for the stopping test and the power iteration (App. A), and
// vector scaling.
#include "common.cuh"

namespace pnp {
namespace {

__device__ __forceinline__ float soft_t(float c, float t) {
  const float m = fabsf(c) - t;
  return m > 0.f ? copysignf(m, c) : 0.f;
}

__device__ __forceinline__ void reduce2_atomic(double v0, double v1, double* acc) {
  __shared__ double red[64];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[2 * warp] = v0;
    red[2 * warp + 1] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int w = 0; w < nw; ++w) {
      s0 += red[2 * w];
      s1 += red[2 * w + 1];
    }
    atomicAdd(&acc[0], s0);
    atomicAdd(&acc[1], s1);
  }
}

// out = max(0, Psi S_t Psi^T z) on 2x2 blocks; acc[0] += ||out - x_prev||^2, acc[1] += ||out||^2
__global__ void __launch_bounds__(256) haar_kernel(const float* __restrict__ z, float* __restrict__ out,
                                                   int n, float t, double* acc,
                                                   const float* __restrict__ xp) {
  double s0 = 0.0, s1 = 0.0;
  const int64_t nb = (int64_t)(n / 2) * (n / 2);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nb; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t br = q / (n / 2), bc = q - br * (n / 2);
    const int64_t i00 = 2 * br * n + 2 * bc;
    const float z00 = z[i00], z01 = z[i00 + 1], z10 = z[i00 + n], z11 = z[i00 + n + 1];
    if (!(isfinite(z00) && isfinite(z01) && isfinite(z10) && isfinite(z11)))
      s1 = __longlong_as_double(0x7ff8000000000000LL);  // positivity would hide it otherwise
    const float ha = soft_t(0.5f * (z00 + z01 + z10 + z11), t);
    const float hh = soft_t(0.5f * (z00 - z01 + z10 - z11), t);
    const float hv = soft_t(0.5f * (z00 + z01 - z10 - z11), t);
    const float hd = soft_t(0.5f * (z00 - z01 - z10 + z11), t);
    const float o[4] = {fmaxf(0.f, 0.5f * (ha + hh + hv + hd)), fmaxf(0.f, 0.5f * (ha - hh + hv - hd)),
                        fmaxf(0.f, 0.5f * (ha + hh - hv - hd)), fmaxf(0.f, 0.5f * (ha - hh - hv + hd))};
    const int64_t ix[4] = {i00, i00 + 1, i00 + n, i00 + n + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      out[ix[k]] = o[k];
      s1 += (double)o[k] * o[k];
      if (xp) {
        const double d = (double)o[k] - xp[ix[k]];
        s0 += d * d;
      }
    }
  }
  if (acc) reduce2_atomic(s0, s1, acc);
}

__global__ void __launch_bounds__(256) norm2_kernel(const float* __restrict__ v, int64_t count, double* acc) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)v[i] * v[i];
  reduce2_atomic(s, 0.0, acc);
}

__global__ void scale_kernel(const float* __restrict__ in, float* __restrict__ out, int64_t count,
                             const double* __restrict__ acc, int k) {
  const double nrm = sqrt(acc[k]);
  const float s = nrm > 0 ? (float)(1.0 / nrm) : 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * s;
}

__global__ void fill_kernel(float* out, int64_t count, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

__global__ void mul_kernel(const float* __restrict__ in, float* __restrict__ out, int64_t count, float f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * f;
}

// y_out[m] = d[m] y_in[m] (complex by real, per row)
__global__ void rowscale_kernel(const float2* y_in, const float* __restrict__ d, float2* y_out, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = y_in[i];
    const float s = d[i];
    y_out[i] = make_float2(v.x * s, v.y * s);
  }
}

__global__ void zero_kernel(double* acc, int count) {
  if (threadIdx.x < count) acc[threadIdx.x] = 0.0;
}

int grid_for(int64_t count) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (count + 255) / 256;
  if (b > 4L * sms) b = 4L * sms;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int haar_denoise_dev(cudaStream_t s, const float* z, float* out, int n, float t, double* acc,
                     const float* x_prev) {
  haar_kernel<<<grid_for((int64_t)n * n / 4), 256, 0, s>>>(z, out, n, t, acc, x_prev);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int norm2_dev(cudaStream_t s, const float* v, int64_t count, double* acc) {
  norm2_kernel<<<grid_for(count), 256, 0, s>>>(v, count, acc);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int scale_image(cudaStream_t s, const float* in, float* out, int64_t count, const double* acc, int k) {
  scale_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count, acc, k);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int fill_image(cudaStream_t s, float* out, int64_t count, float v) {
  fill_kernel<<<grid_for(count), 256, 0, s>>>(out, count, v);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int mul_image(cudaStream_t s, const float* in, float* out, int64_t count, float f) {
  mul_kernel<<<grid_for(count), 256, 0, s>>>(in, out, count, f);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int row_scale_c64(cudaStream_t s, const float2* y_in, const float* d, float2* y_out, int64_t count) {
  if (count == 0) return PNP_OK;
  rowscale_kernel<<<grid_for(count), 256, 0, s>>>(y_in, d, y_out, count);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int zero_acc(cudaStream_t s, double* acc, int count) {
  zero_kernel<<<1, 32, 0, s>>>(acc, count);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

}  // namespace pnp
