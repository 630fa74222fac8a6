// Allocation-free entry point: the plain Haar denoiser with the FP64
// stopping-test norms, for callers that must not allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is off limits -- inside a
// region where the host must not allocate (a caller-managed memory pool or a
// fixed memory budget decided up front), or a host runtime that forbids
// allocation after start-up.  Such a caller owns every input and output
// buffer and cannot create a plan, so this call keeps its scratch (one pair of
// FP64 partial sums per pair of image rows) in a file-scope device array that
// lives as long as the library is loaded.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each call writes every partial it later reads, so nothing has to
// be cleared first.  Calls that overlap on the GPU (two streams, or two host
// threads) race on the array and must be serialised by the caller.
#include <cmath>

#include "common.cuh"

namespace pnp {
namespace {

constexpr int NOALLOC_MAX_N = 16384;          // largest image side accepted
constexpr int NOALLOC_ROWS = NOALLOC_MAX_N / 2;

// per pair of image rows: ||x_out - x_prev||^2 and ||x_out||^2 partial sums (128 KiB)
static __device__ __align__(256) double g_noalloc_scratch[2 * NOALLOC_ROWS];

// Device address of the scratch array for the current device (the host-side symbol is only a
// stand-in).  Looked up on every call with the caller's device current: the lookup allocates
// nothing, and a cached address would go stale if the caller recreated the device's primary
// context (cudaDeviceReset), after which the module can load at another address.
int scratch_address(double** out) {
  void* p = nullptr;
  PNP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = static_cast<double*>(p);
  return PNP_OK;
}

// true when the byte ranges [a, a + bytes) and [b, b + bytes) overlap
bool overlaps(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

__device__ __forceinline__ float soft_na(float c, float t) {
  const float m = fabsf(c) - t;
  return m > 0.f ? copysignf(m, c) : 0.f;
}

// One CTA per pair of image rows: Haar soft-threshold + positivity on the row
// pair's 2x2 blocks, then a fixed-order tree reduction of the two norms into
// the scratch slot of this row pair.
__global__ void __launch_bounds__(256) haar_rows_noalloc(const float* __restrict__ z,
                                                         const float* __restrict__ xp,
                                                         float* __restrict__ out, int n, float t,
                                                         double* __restrict__ scratch) {
  __shared__ double red[2 * 256];
  const int pr = blockIdx.x;
  const size_t base = (size_t)2 * pr * n;
  double s0 = 0.0, s1 = 0.0;
  for (int bb = threadIdx.x; bb < n / 2; bb += blockDim.x) {
    const size_t i00 = base + 2 * bb;
    const float z00 = z[i00], z01 = z[i00 + 1], z10 = z[i00 + n], z11 = z[i00 + n + 1];
    const float ha = soft_na(0.5f * (z00 + z01 + z10 + z11), t);
    const float hh = soft_na(0.5f * (z00 - z01 + z10 - z11), t);
    const float hv = soft_na(0.5f * (z00 + z01 - z10 - z11), t);
    const float hd = soft_na(0.5f * (z00 - z01 - z10 + z11), t);
    const float o[4] = {fmaxf(0.f, 0.5f * (ha + hh + hv + hd)), fmaxf(0.f, 0.5f * (ha - hh + hv - hd)),
                        fmaxf(0.f, 0.5f * (ha + hh - hv - hd)), fmaxf(0.f, 0.5f * (ha - hh - hv + hd))};
    const size_t ix[4] = {i00, i00 + 1, i00 + n, i00 + n + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      out[ix[k]] = o[k];
      s1 += (double)o[k] * o[k];
      if (xp) {
        const double d = (double)o[k] - xp[ix[k]];
        s0 += d * d;
      }
    }
    if (!(isfinite(z00) && isfinite(z01) && isfinite(z10) && isfinite(z11)))
      s1 = __longlong_as_double(0x7ff8000000000000LL);
  }
  red[2 * threadIdx.x] = s0;
  red[2 * threadIdx.x + 1] = s1;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[2 * threadIdx.x] += red[2 * (threadIdx.x + s)];
      red[2 * threadIdx.x + 1] += red[2 * (threadIdx.x + s) + 1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scratch[2 * pr] = red[0];
    scratch[2 * pr + 1] = red[1];
  }
}

// Sum the row-pair partials in a fixed order into the caller's two doubles.
__global__ void __launch_bounds__(256) reduce_rows_noalloc(const double* __restrict__ scratch, int rows,
                                                           double* __restrict__ norms) {
  __shared__ double red[2 * 256];
  double s0 = 0.0, s1 = 0.0;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    s0 += scratch[2 * r];
    s1 += scratch[2 * r + 1];
  }
  red[2 * threadIdx.x] = s0;
  red[2 * threadIdx.x + 1] = s1;
  __syncthreads();
  for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[2 * threadIdx.x] += red[2 * (threadIdx.x + s)];
      red[2 * threadIdx.x + 1] += red[2 * (threadIdx.x + s) + 1];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    norms[0] = red[0];
    norms[1] = red[1];
  }
}

}  // namespace
}  // namespace pnp

extern "C" int pnp_haar_denoise_noalloc(const float* z, const float* x_prev, float* x_out, int n,
                                        double t, double* norms, void* stream) {
  using namespace pnp;
  if (!z || !x_out || !norms) return fail(PNP_ERR_INVALID_ARG, "z, x_out and norms must not be NULL");
  if (n < 2 || (n & 1)) return fail(PNP_ERR_INVALID_ARG, "n must be even and >= 2");
  if (n > NOALLOC_MAX_N)
    return fail(PNP_ERR_INVALID_ARG, "n = " + std::to_string(n) + " exceeds the allocation-free limit of " +
                                         std::to_string(NOALLOC_MAX_N) + " pixels per side");
  if (!(t >= 0) || !std::isfinite(t)) return fail(PNP_ERR_INVALID_ARG, "t must be finite and >= 0");
  const size_t bytes = (size_t)n * n * sizeof(float);
  if (overlaps(z, x_out, bytes)) return fail(PNP_ERR_INVALID_ARG, "z and x_out must not overlap");
  if (x_prev && overlaps(x_prev, x_out, bytes))
    return fail(PNP_ERR_INVALID_ARG, "x_prev and x_out must not overlap");
  double* scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  haar_rows_noalloc<<<n / 2, 256, 0, s>>>(z, x_prev, x_out, n, (float)t, scratch);
  PNP_CHECK_LAUNCH();
  reduce_rows_noalloc<<<1, 256, 0, s>>>(scratch, n / 2, norms);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}
