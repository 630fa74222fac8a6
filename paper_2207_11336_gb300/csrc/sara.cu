// uSARA's handcrafted denoiser (App. B): the prox of gamma lambda ||W Psi^T x||_1 + iota_+(x) for
// the SARA dictionary Psi (the Dirac basis and the 2-D Daubechies bases db1..db8, each a multi-level
// separable DWT with periodic extension, divided by 3 so that Psi Psi^T = I), by dual
// forward-backward sub-iterations:
//   x = max(0, z - Psi u),   u <- clip(u + Psi^T x, -t, t),   t = gamma lambda w,
// warm-started from the previous call's u, and the reweighting w = rho / (rho + |Psi^T x|) that
// majorises the log-sum prior at the current image.
//
// Each DWT level is one pass along each axis over the level's m x m block: analysis
// a[j] = sum_k f[k] x[(2 j + k) mod m] (low half, then high half), synthesis as the gather
// x[p] = sum_{k : p - k even} lo[k] a[((p - k) mod m) / 2] + hi[k] d[((p - k) mod m) / 2].
// The Daubechies filters are computed on the host by spectral factorisation (minimum-phase roots
// of z^(N-1) P_N((2 - z - 1/z) / 4), Durand-Kerner iteration with Newton polish).
#include <vector>

#include "common.cuh"
#include "daubechies.h"

namespace pnp {
namespace {

constexpr int SARA_FILTERS = 8, SARA_BASES = 9, MAXTAP = 16;

struct SaraState {
  int n = 0, levels = 0, iters = 0;
  double gl = 0, rho = 0;   // gamma lambda (threshold scale), log-sum floor
  float* filt = nullptr;    // [8][2][16]: low-pass, high-pass (zero padded)
  int len[SARA_FILTERS] = {};
  float *u = nullptr, *w = nullptr;            // 9 n^2: dual variable, weights
  float *A = nullptr, *T = nullptr, *S = nullptr, *X = nullptr;  // n^2 work images
};

// r mod m for 0 <= r < m + L (r - L < m) by subtraction instead of an integer division; a loop, since
// the coarsest levels' blocks can be shorter than a filter
__device__ __forceinline__ int wrap_up(int r, int m) {
  while (r >= m) r -= m;
  return r;
}

// ---- the four passes of a level (analysis and synthesis along each axis of the m x m block, row stride
// n), each shared-memory tiled: a CTA stages the input rows or row segments its outputs need once, so
// each input element is read from memory about once per pass instead of once per tap.
constexpr int DW_TC = 32;          // columns per tile of the axis-0 passes
constexpr int DW_TJ = 32;          // output rows per tile of the axis-0 analysis
constexpr int DW_TP = 64;          // output rows per tile of the axis-0 synthesis
constexpr int DW_TR = 256;         // outputs per CTA of the axis-1 passes
__device__ __forceinline__ int floor_half(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }
__device__ __forceinline__ int wrap_any(int r, int m) {
  while (r >= m) r -= m;
  while (r < 0) r += m;
  return r;
}

// analysis along axis 0: grid (ceil(m / DW_TC), ceil(half / DW_TJ)), 256 threads
__global__ void __launch_bounds__(256) dwt0_tiled(const float* __restrict__ in, float* __restrict__ out, int n, int m,
                                                  const float* __restrict__ f, int L) {
  __shared__ float t[2 * DW_TJ + MAXTAP][DW_TC + 1];
  const int half = m / 2, c0 = blockIdx.x * DW_TC, j0 = blockIdx.y * DW_TJ;
  const int rows = 2 * DW_TJ + L - 1;
  for (int e = threadIdx.x; e < rows * DW_TC; e += blockDim.x) {
    const int rr = e / DW_TC, cc = e % DW_TC, c = c0 + cc;
    t[rr][cc] = c < m ? in[(int64_t)wrap_up(2 * j0 + rr, m) * n + c] : 0.f;
  }
  __syncthreads();
  const int cc = threadIdx.x % DW_TC, c = c0 + cc;
  for (int jj = threadIdx.x / DW_TC; jj < DW_TJ; jj += blockDim.x / DW_TC) {
    const int j = j0 + jj;
    if (j >= half || c >= m) continue;
    float sl = 0.f, sh = 0.f;
    for (int k = 0; k < L; ++k) {
      const float v = t[2 * jj + k][cc];
      sl = fmaf(f[k], v, sl);
      sh = fmaf(f[MAXTAP + k], v, sh);
    }
    out[(int64_t)j * n + c] = sl;
    out[(int64_t)(half + j) * n + c] = sh;
  }
}

// analysis along axis 1: grid (ceil(half / DW_TR), m), DW_TR threads
__global__ void __launch_bounds__(DW_TR) dwt1_tiled(const float* __restrict__ in, float* __restrict__ out, int n, int m,
                                                    const float* __restrict__ f, int L) {
  __shared__ float t[2 * DW_TR + MAXTAP];
  const int half = m / 2, j0 = blockIdx.x * DW_TR, i = blockIdx.y;
  const float* row = in + (int64_t)i * n;
  const int cnt = 2 * DW_TR + L - 1;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) t[e] = row[wrap_up(2 * j0 + e, m)];
  __syncthreads();
  const int j = j0 + threadIdx.x;
  if (j >= half) return;
  float sl = 0.f, sh = 0.f;
  for (int k = 0; k < L; ++k) {
    const float v = t[2 * threadIdx.x + k];
    sl = fmaf(f[k], v, sl);
    sh = fmaf(f[MAXTAP + k], v, sh);
  }
  out[(int64_t)i * n + j] = sl;
  out[(int64_t)i * n + half + j] = sh;
}

// synthesis along axis 1: grid (ceil(m / DW_TR), m), DW_TR threads.  Output p takes the taps k = p mod 2,
// p mod 2 + 2, ... at j = ((p - k) mod m) / 2; the CTA stages j = jb .. of the low and high halves, jb the
// smallest (p - k) / 2 of its outputs (unwrapped), each staged entry wrapped into [0, half).
__global__ void __launch_bounds__(DW_TR) idwt1_tiled(const float* __restrict__ in, float* __restrict__ out, int n,
                                                     int m, const float* __restrict__ f, int L) {
  __shared__ float lo[DW_TR / 2 + MAXTAP / 2 + 2], hi[DW_TR / 2 + MAXTAP / 2 + 2];
  const int half = m / 2, p0 = blockIdx.x * DW_TR, i = blockIdx.y;
  const float* row = in + (int64_t)i * n;
  const int jb = floor_half(p0 - L + 1);
  const int cnt = floor_half(p0 + DW_TR - 1) - jb + 1;
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int j = wrap_any(jb + e, half);
    lo[e] = row[j];
    hi[e] = row[half + j];
  }
  __syncthreads();
  const int p = p0 + threadIdx.x;
  if (p >= m) return;
  float acc = 0.f;
  for (int k = (p & 1); k < L; k += 2) {
    const int e = (p - k) / 2 - jb;  // p - k is even
    acc = fmaf(f[k], lo[e], fmaf(f[MAXTAP + k], hi[e], acc));
  }
  out[(int64_t)i * n + p] = acc;
}

// synthesis along axis 0: grid (ceil(m / DW_TC), ceil(m / DW_TP)), 256 threads
__global__ void __launch_bounds__(256) idwt0_tiled(const float* __restrict__ in, float* __restrict__ out, int n,
                                                   int m, const float* __restrict__ f, int L) {
  __shared__ float lo[DW_TP / 2 + MAXTAP / 2 + 2][DW_TC + 1], hi[DW_TP / 2 + MAXTAP / 2 + 2][DW_TC + 1];
  const int half = m / 2, c0 = blockIdx.x * DW_TC, p0 = blockIdx.y * DW_TP;
  const int jb = floor_half(p0 - L + 1);
  const int cnt = floor_half(p0 + DW_TP - 1) - jb + 1;
  for (int e = threadIdx.x; e < cnt * DW_TC; e += blockDim.x) {
    const int rr = e / DW_TC, cc = e % DW_TC, c = c0 + cc;
    const int j = wrap_any(jb + rr, half);
    lo[rr][cc] = c < m ? in[(int64_t)j * n + c] : 0.f;
    hi[rr][cc] = c < m ? in[(int64_t)(half + j) * n + c] : 0.f;
  }
  __syncthreads();
  const int cc = threadIdx.x % DW_TC, c = c0 + cc;
  for (int pp = threadIdx.x / DW_TC; pp < DW_TP; pp += blockDim.x / DW_TC) {
    const int p = p0 + pp;
    if (p >= m || c >= m) continue;
    float acc = 0.f;
    for (int k = (p & 1); k < L; k += 2) {
      const int e = (p - k) / 2 - jb;
      acc = fmaf(f[k], lo[e][cc], fmaf(f[MAXTAP + k], hi[e][cc], acc));
    }
    out[(int64_t)p * n + c] = acc;
  }
}

// mode 0: s = v / 3;  mode 1: s += v / 3;  mode 2: x = max(0, z - (s + v / 3));  mode 3: x = z - (s + v / 3)
__global__ void sara_accum(const float* __restrict__ v, float* __restrict__ s, const float* __restrict__ z,
                           float* __restrict__ x, int64_t count, int mode) {
  const float third = 1.f / 3.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = v[i] * third;
    if (mode == 0) s[i] = a;
    else if (mode == 1) s[i] += a;
    else if (mode == 2) x[i] = fmaxf(0.f, z[i] - (s[i] + a));
    else x[i] = z[i] - (s[i] + a);
  }
}

__global__ void sara_fill(float* __restrict__ p, int64_t count, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void sara_third(float* __restrict__ c, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    c[i] *= 1.f / 3.f;
}

// u = clip(u + c / 3, -gl w, gl w)  (the dual step; c = B_b x)
__global__ void sara_dual(float* __restrict__ u, const float* __restrict__ c, const float* __restrict__ w, float gl,
                          int64_t count) {
  const float third = 1.f / 3.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float t = gl * w[i];
    u[i] = fminf(t, fmaxf(-t, u[i] + c[i] * third));
  }
}

// w = rho / (rho + |c / 3|)
__global__ void sara_weights(const float* __restrict__ c, float* __restrict__ w, float rho, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = rho / (rho + fabsf(c[i] * (1.f / 3.f)));
}

__global__ void __launch_bounds__(256) sara_norms(const float* __restrict__ x, const float* __restrict__ prev,
                                                  int64_t count, double* acc) {
  __shared__ double r0[256], r1[256];
  double a = 0.0, b = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i], d = v - (prev ? prev[i] : 0.f);
    a += d * d;
    b += v * v;
  }
  r0[threadIdx.x] = a;
  r1[threadIdx.x] = b;
  __syncthreads();
  for (int k = blockDim.x >> 1; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      r0[threadIdx.x] += r0[threadIdx.x + k];
      r1[threadIdx.x] += r1[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&acc[0], r0[0]);
    atomicAdd(&acc[1], r1[0]);
  }
}

int grid1(int64_t count) { return (int)std::min<int64_t>((count + 255) / 256, 4096); }

// c = B_b x for basis b (1..8) of the n x n image x (c may not alias x)
int basis_analysis(SaraState* S, cudaStream_t s, int b, const float* x, float* c) {
  const int n = S->n;
  const float* f = S->filt + (size_t)(b - 1) * 2 * MAXTAP;
  const int L = S->len[b - 1];
  for (int l = 0; l < S->levels; ++l) {  // level 0 reads x; its second pass writes all of c
    const int m = n >> l;
    const int half = m / 2;
    dwt0_tiled<<<dim3((m + DW_TC - 1) / DW_TC, (half + DW_TJ - 1) / DW_TJ), 256, 0, s>>>(l == 0 ? x : c, S->T, n, m,
                                                                                         f, L);
    PNP_CHECK_LAUNCH();
    dwt1_tiled<<<dim3((half + DW_TR - 1) / DW_TR, m), DW_TR, 0, s>>>(S->T, c, n, m, f, L);
    PNP_CHECK_LAUNCH();
  }
  return PNP_OK;
}

// x = B_b^T c (x may not alias c; S->T is scratch)
int basis_synthesis(SaraState* S, cudaStream_t s, int b, const float* c, float* x) {
  const int n = S->n;
  const float* f = S->filt + (size_t)(b - 1) * 2 * MAXTAP;
  const int L = S->len[b - 1];
  PNP_CUDA(cudaMemcpyAsync(x, c, (size_t)n * n * 4, cudaMemcpyDeviceToDevice, s));
  for (int l = S->levels - 1; l >= 0; --l) {
    const int m = n >> l;
    idwt1_tiled<<<dim3((m + DW_TR - 1) / DW_TR, m), DW_TR, 0, s>>>(x, S->T, n, m, f, L);
    PNP_CHECK_LAUNCH();
    idwt0_tiled<<<dim3((m + DW_TC - 1) / DW_TC, (m + DW_TP - 1) / DW_TP), 256, 0, s>>>(S->T, x, n, m, f, L);
    PNP_CHECK_LAUNCH();
  }
  return PNP_OK;
}

// x = max(0, z - Psi u)
int primal(SaraState* S, cudaStream_t s, const float* z, float* x, bool positivity) {
  const int64_t N = (int64_t)S->n * S->n;
  sara_accum<<<grid1(N), 256, 0, s>>>(S->u, S->S, nullptr, nullptr, N, 0);
  PNP_CHECK_LAUNCH();
  for (int b = 1; b < SARA_BASES; ++b) {
    if (int rc = basis_synthesis(S, s, b, S->u + (size_t)b * N, S->A)) return rc;
    sara_accum<<<grid1(N), 256, 0, s>>>(S->A, S->S, z, x, N, b == SARA_BASES - 1 ? (positivity ? 2 : 3) : 1);
    PNP_CHECK_LAUNCH();
  }
  return PNP_OK;
}

}  // namespace

int sara_create(pnp_den* d, int n, int levels, double gl, double rho, int iters) {
  SaraState* S = new SaraState();
  S->n = n;
  S->levels = levels;
  S->iters = iters;
  S->gl = gl;
  S->rho = rho;
  std::vector<float> filt((size_t)SARA_FILTERS * 2 * MAXTAP, 0.f);
  for (int N = 1; N <= SARA_FILTERS; ++N) {
    const std::vector<double> h = daub::daubechies(N);
    const int L = (int)h.size();
    if (L != 2 * N) {  // the factorisation must keep exactly N - 1 roots inside the unit circle
      d->impl = S;
      return fail(PNP_ERR_UNSUPPORTED, "internal: Daubechies factorisation failed for N = " + std::to_string(N));
    }
    S->len[N - 1] = L;
    for (int k = 0; k < L; ++k) {
      filt[(size_t)(N - 1) * 2 * MAXTAP + k] = (float)h[k];
      filt[(size_t)(N - 1) * 2 * MAXTAP + MAXTAP + k] = (float)((k & 1 ? -1.0 : 1.0) * h[L - 1 - k]);
    }
  }
  const size_t N2 = (size_t)n * n;
  bool ok = cudaMalloc(&S->filt, filt.size() * 4) == cudaSuccess &&
            cudaMalloc(&S->u, SARA_BASES * N2 * 4) == cudaSuccess &&
            cudaMalloc(&S->w, SARA_BASES * N2 * 4) == cudaSuccess && cudaMalloc(&S->A, N2 * 4) == cudaSuccess &&
            cudaMalloc(&S->T, N2 * 4) == cudaSuccess && cudaMalloc(&S->S, N2 * 4) == cudaSuccess &&
            cudaMalloc(&S->X, N2 * 4) == cudaSuccess;
  d->impl = S;
  if (!ok) {
    cudaGetLastError();
    return fail(PNP_ERR_OOM, "SARA denoiser allocation failed");
  }
  PNP_CUDA(cudaMemcpy(S->filt, filt.data(), filt.size() * 4, cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemset(S->u, 0, SARA_BASES * N2 * 4));
  sara_fill<<<grid1((int64_t)(SARA_BASES * N2)), 256>>>(S->w, (int64_t)(SARA_BASES * N2), 1.f);  // w = 1
  PNP_CHECK_LAUNCH();
  PNP_CUDA(cudaDeviceSynchronize());
  return PNP_OK;
}

void sara_destroy(pnp_den* d) {
  SaraState* S = static_cast<SaraState*>(d->impl);
  if (!S) return;
  for (float* p : {S->filt, S->u, S->w, S->A, S->T, S->S, S->X}) cudaFree(p);
  delete S;
  d->impl = nullptr;
}

// the prox by S->iters dual-FB iterations from the kept u; out = x; FP64 norms into acc[0..1]
int sara_denoise(pnp_den* d, cudaStream_t s, const float* z, float* out, int n, double* acc, const float* x_prev,
                 bool positivity) {
  SaraState* S = static_cast<SaraState*>(d->impl);
  if (!S || n != S->n) return fail(PNP_ERR_INVALID_ARG, "image side differs from the SARA denoiser's");
  const int64_t N = (int64_t)n * n;
  if (int rc = primal(S, s, z, out, positivity)) return rc;
  for (int it = 0; it < S->iters; ++it) {
    sara_dual<<<grid1(N), 256, 0, s>>>(S->u, out, S->w, (float)S->gl, N);  // the Dirac basis
    PNP_CHECK_LAUNCH();
    for (int b = 1; b < SARA_BASES; ++b) {
      if (int rc = basis_analysis(S, s, b, out, S->A)) return rc;
      sara_dual<<<grid1(N), 256, 0, s>>>(S->u + (size_t)b * N, S->A, S->w + (size_t)b * N, (float)S->gl, N);
      PNP_CHECK_LAUNCH();
    }
    if (int rc = primal(S, s, z, out, positivity)) return rc;
  }
  if (acc) {
    sara_norms<<<grid1(N), 256, 0, s>>>(out, x_prev, N, acc);
    PNP_CHECK_LAUNCH();
  }
  return PNP_OK;
}

int sara_reweight(pnp_den* d, const float* x) {
  SaraState* S = static_cast<SaraState*>(d->impl);
  const int64_t N = (int64_t)S->n * S->n;
  cudaStream_t s = d->stream;
  sara_weights<<<grid1(N), 256, 0, s>>>(x, S->w, (float)S->rho, N);
  PNP_CHECK_LAUNCH();
  for (int b = 1; b < SARA_BASES; ++b) {
    if (int rc = basis_analysis(S, s, b, x, S->A)) return rc;
    sara_weights<<<grid1(N), 256, 0, s>>>(S->A, S->w + (size_t)b * N, (float)S->rho, N);
    PNP_CHECK_LAUNCH();
  }
  return PNP_OK;
}

// direction 1: out (9 n^2) = Psi^T in;  direction -1: out (n^2) = Psi in
int sara_transform(pnp_den* d, const float* in, float* out, int direction) {
  SaraState* S = static_cast<SaraState*>(d->impl);
  const int64_t N = (int64_t)S->n * S->n;
  cudaStream_t s = d->stream;
  if (direction > 0) {
    for (int b = 0; b < SARA_BASES; ++b) {
      float* c = out + (size_t)b * N;
      if (b == 0) PNP_CUDA(cudaMemcpyAsync(c, in, N * 4, cudaMemcpyDeviceToDevice, s));
      else if (int rc = basis_analysis(S, s, b, in, c)) return rc;
      sara_third<<<grid1(N), 256, 0, s>>>(c, N);
      PNP_CHECK_LAUNCH();
    }
  } else {
    sara_accum<<<grid1(N), 256, 0, s>>>(in, out, nullptr, nullptr, N, 0);
    PNP_CHECK_LAUNCH();
    for (int b = 1; b < SARA_BASES; ++b) {
      if (int rc = basis_synthesis(S, s, b, in + (size_t)b * N, S->A)) return rc;
      sara_accum<<<grid1(N), 256, 0, s>>>(S->A, out, nullptr, nullptr, N, 1);
      PNP_CHECK_LAUNCH();
    }
  }
  return PNP_OK;
}

}  // namespace pnp
