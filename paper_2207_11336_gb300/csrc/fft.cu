// Oversampled 2-D DFT F (Eq. 1) fused with zero-padding and grid correction Z,
// and its adjoint F^H fused with Z^H, the real part, the gradient step and the
// plain Haar denoiser (App. A, B).
//
// Layouts.  Image x[a][b] (n x n, float32).  The K x K grid is stored with the
// axis-1 frequency k1 slow and the axis-0 frequency k0 fast: grid[k1*K + k0].
// The forward transform runs in two kernels, each a batch of contiguous
// length-K FFTs in shared memory:
//   P1  rows a of the image: place x[a][b] / (c_a c_b) at (b - n/2) mod K,
//       FFT along axis 1, write the result transposed into T[k1][a] (K x n);
//   P2  rows k1 of T: place T[k1][a] at (a - n/2) mod K, FFT along axis 0,
//       write grid[k1][k0].
// Only n of the K input positions are non-zero in each pass (the zero-padding
// of Z), so both passes read n values per row.  The adjoint runs the mirror:
//   Q1  rows k1 of the gridded data: inverse FFT along axis 0, keep the n
//       image rows, write U[a][k1] (n x K); re-zeroes the grid it consumed;
//   Q2  rows a of U: inverse FFT along axis 1, keep the n image columns,
//       divide by c_a c_b, take the real part, and apply the epilogue
//       (adjoint only / gradient step / gradient step + Haar + positivity /
//       power-iteration norm), two image rows per CTA so the 2 x 2 Haar
//       blocks are local.
//
// Each length-K FFT is a Stockham autosort: radix-16 passes done in registers
// (16 complex values per thread, K/16 threads per row) with the data exchanged
// through padded shared memory between passes, then one radix-2/4/8 pass in
// registers when log2 K is not a multiple of 4.  Twiddles come from a table
// exp(-2 pi i j / K) computed on the host in double precision.
#include "common.cuh"

namespace pnp {
namespace {

constexpr int PAD_SHIFT = 4;
__device__ __forceinline__ int PADI(int i) { return i + (i >> PAD_SHIFT); }

// cos and sin of 2 pi m / 16
__device__ __forceinline__ float2 w16(int m, int dir) {
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, r2 = 0.70710678118654752f;
  float c, s;
  switch (m & 15) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = c1; s = s1; break;
    case 2: c = r2; s = r2; break;
    case 3: c = s1; s = c1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 5: c = -s1; s = c1; break;
    case 6: c = -r2; s = r2; break;
    case 7: c = -c1; s = s1; break;
    case 8: c = -1.f; s = 0.f; break;
    case 9: c = -c1; s = -s1; break;
    case 10: c = -r2; s = -r2; break;
    case 11: c = -s1; s = -c1; break;
    case 12: c = 0.f; s = -1.f; break;
    case 13: c = s1; s = -c1; break;
    case 14: c = r2; s = -r2; break;
    default: c = c1; s = -s1; break;
  }
  // exp(dir * 2 pi i m / 16), dir = -1 forward, +1 inverse
  return make_float2(c, dir < 0 ? -s : s);
}

// multiply by exp(dir * i pi / 2)
template <int DIR>
__device__ __forceinline__ float2 rotq(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// complex add and subtract as one packed FP32x2 instruction each (lane-wise IEEE add, the same
// rounding as two scalar adds)
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&d);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)));
  return *reinterpret_cast<float2*>(&d);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 s02 = padd(x0, x2), d02 = psub(x0, x2);
  float2 s13 = padd(x1, x3), d13 = rotq<DIR>(psub(x1, x3));
  x0 = padd(s02, s13);
  x2 = psub(s02, s13);
  x1 = cadd(d02, d13);   // the quarter-turn swaps lanes: scalar adds take it as operand order
  x3 = csub(d02, d13);
}

// 8-point DFT on u[0..7] (natural order in and out): n = n1 + 4 n2, k = 2 k1 + k2.
template <int DIR>
__device__ __forceinline__ void dft8(float2* u) {
  float2 A[4][2];
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    A[n1][0] = u[n1];
    A[n1][1] = u[n1 + 4];
    dft2<DIR>(A[n1][0], A[n1][1]);
    if (n1) A[n1][1] = cmul(A[n1][1], w16(2 * n1, DIR));
  }
#pragma unroll
  for (int k2 = 0; k2 < 2; ++k2) {
    float2 b0 = A[0][k2], b1 = A[1][k2], b2 = A[2][k2], b3 = A[3][k2];
    dft4<DIR>(b0, b1, b2, b3);
    u[k2] = b0;
    u[2 + k2] = b1;
    u[4 + k2] = b2;
    u[6 + k2] = b3;
  }
}

// 16-point DFT on v[0..15]: n = n1 + 4 n2, k = 4 k1 + k2.
template <int DIR>
__device__ __forceinline__ void dft16(float2* v) {
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) dft4<DIR>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]);
  // now v[n1 + 4 k2] = A[n1][k2]
#pragma unroll
  for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
    for (int k2 = 1; k2 < 4; ++k2) v[n1 + 4 * k2] = cmul(v[n1 + 4 * k2], w16(n1 * k2, DIR));
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) dft4<DIR>(v[4 * k2], v[4 * k2 + 1], v[4 * k2 + 2], v[4 * k2 + 3]);
  // v[k1 + 4 k2] = X[4 k1 + k2]
  float2 t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[(i >> 2) + 4 * (i & 3)];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}

template <int DIR>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int idx) {
  float2 w = __ldg(&tw[idx]);
  if (DIR > 0) w.y = -w.y;
  return w;
}

// Barrier of the threads of one transform: named barrier `id` over `nthr` threads (whole warps), or
// the CTA-wide barrier when id is 0.  Transforms that share a CTA but not data then pass their
// exchanges independently.
__device__ __forceinline__ void group_sync(int id, int nthr) {
  if (id == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthr) : "memory");
}

// Length-K FFT of one row.  On entry v[i] holds element j + i*K/16 of the
// row; on exit v[i] holds output element j + i*K/16 (natural order).
// s is this row's padded shared-memory buffer (K + K/16 float2).
// TWS: stride of the twiddle table tw for the radix-2/4/8 tail pass (the table holds exp(-2 pi i t / L)
// for a length L = TWS 2^LOGK: the plan's length-K table serves the length-K/2 transforms with TWS = 2).
// bid: the barrier of the row's threads (group_sync; 0 = the CTA's).
template <int LOGK, int DIR, int TWS = 1>
__device__ __forceinline__ void fft_row(float2 (&v)[16], float2* s, int j,
                                        const float2* __restrict__ tw, const float2* __restrict__ twp,
                                        int bid = 0) {
  constexpr int K = 1 << LOGK;
  constexpr int Q = LOGK / 4;
  static_assert(Q <= 3, "the pass twiddle tables cover radix-16 passes 1 and 2");
  constexpr int REM = LOGK % 4;
  constexpr int K16 = K / 16;
#pragma unroll
  for (int p = 0; p < Q; ++p) {
    const int Ns = 1 << (4 * p);
    const int k = j & (Ns - 1);
    if (p > 0) {
      // exp(dir 2 pi i r k / 16^(p+1)) from the pass's [r][k] table: consecutive k of a warp read
      // consecutive entries (the full-length table would be read with a stride of r k)
      const float2* tp = twp + (p == 1 ? 0 : 256) + k;
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twiddle<DIR>(tp, r * Ns));
    }
    dft16<DIR>(v);
    if (!(p == Q - 1 && REM == 0)) {
      const int idxD = ((j >> (4 * p)) << (4 * p + 4)) + k;
      group_sync(bid, K16);
#pragma unroll
      for (int r = 0; r < 16; ++r) s[PADI(idxD + r * Ns)] = v[r];
      group_sync(bid, K16);
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = s[PADI(j + r * K16)];
    }
  }
  if constexpr (REM > 0) {
    constexpr int RS = 1 << REM;
    constexpr int G = 16 / RS;
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int jj = j + t * K16;
      float2 u[RS];
#pragma unroll
      for (int r = 0; r < RS; ++r) {
        u[r] = v[t + r * G];
        if (r) u[r] = cmul(u[r], twiddle<DIR>(tw, r * jj * TWS));
      }
      if constexpr (RS == 2) dft2<DIR>(u[0], u[1]);
      if constexpr (RS == 4) dft4<DIR>(u[0], u[1], u[2], u[3]);
      if constexpr (RS == 8) dft8<DIR>(u);
#pragma unroll
      for (int r = 0; r < RS; ++r) v[t + r * G] = u[r];
    }
  }
}

// image column / row index held at padded position e, or -1 when e is padding
__device__ __forceinline__ int unpad_index(int e, int n, int K) {
  const int h = n >> 1;
  return e < h ? e + h : (e >= K - h ? e - (K - h) : -1);
}
__device__ __forceinline__ int pad_position(int a, int n, int K) {
  const int h = n >> 1;
  return a < h ? a + K - h : a - h;
}

struct FftArgs {
  int n;
  const float* x;          // P1 input image / Q2 current iterate
  const float* cinv;       // 1 / c(p)
  const float2* tw;
  const float2* twp;       // radix-16 pass twiddles (TWP_ENTRIES)
  float2* tmp;             // T (K x n) or U (n x K)
  float2* grid;            // P2 output / Q1 input (re-zeroed)
  __nv_bfloat162* grid_lo; // Q1: compensation terms added to the input (re-zeroed), or NULL
  float* out;              // Q2 output image
  double* acc;             // Q1 zeroes acc[0..3]; Q2 accumulates
  float gamma, t;
  int epi;
  const float2* chirp;     // n (w-stack s of several): exp(i pi a_s (a - n/2)^2) per image axis, else NULL
  float* gacc;             // n x n gradient image summed over the w-stacks
  int gacc_mode;           // GACC_*: how the Q2 gradient meets gacc
  const int* rowh;         // K: uv support per grid row k1 (largest centred |k0| of a tap, -1: none)
  int band;                // centred half-width of the band of grid rows k1 that hold taps (-1: none)
};

// Q2 and the sum over w-stacks (Eq. phidagphi): the first stack writes its Re{Z_s^H F^H ...}
// image to gacc, later ones add to it, and the last adds gacc to its own before the epilogue.
enum GaccMode { GACC_NONE = 0, GACC_WRITE = 1, GACC_ADD = 2, GACC_FINAL = 3 };

__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// ---------------------------------------------------------------- P1
// CH: the input is modulated by a w-stack's centre chirp (compiled separately so that the
// plain operator keeps its register allocation)
template <int LOGK, int R, bool CH>
__global__ void __launch_bounds__(R * (1 << LOGK) / 16) fft_p1(const __grid_constant__ FftArgs A) {
  constexpr int K = 1 << LOGK, T = K / 16, SROW = K + K / 16 + 1;
  extern __shared__ float2 smem[];
  const int rr = threadIdx.x / T, j = threadIdx.x % T;
  const int n = A.n;
  const int a = blockIdx.x * R + rr;
  const bool live = a < n;  // the last CTA may hold fewer than R image rows
  float2* s = smem + rr * SROW;
  const float ca = live ? A.cinv[a] : 0.f;
  float2 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int b = unpad_index(j + i * T, n, K);
    v[i] = (live && b >= 0) ? make_float2(A.x[(size_t)a * n + b] * ca * A.cinv[b], 0.f)
                            : make_float2(0.f, 0.f);
  }
  if (CH && live) {  // Z_s of a w-stack: the centre chirp, separable over the two axes
    const float2 cha = A.chirp[a];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int b = unpad_index(j + i * T, n, K);
      if (b >= 0) {
        const float2 c = cmul2(cha, A.chirp[b]);
        v[i] = make_float2(v[i].x * c.x, v[i].x * c.y);
      }
    }
  }
  fft_row<LOGK, -1>(v, s, j, A.tw, A.twp);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16; ++i) s[PADI(j + i * T)] = v[i];
  __syncthreads();
  const int a0 = blockIdx.x * R;
  for (int idx = threadIdx.x; idx < R * K; idx += R * T) {
    const int r = idx % R, k1 = idx / R;
    if (a0 + r < n) A.tmp[(size_t)k1 * n + a0 + r] = smem[r * SROW + PADI(k1)];
  }
}

// ---------------------------------------------------------------- P2
template <int LOGK, int R>
__global__ void __launch_bounds__(R * (1 << LOGK) / 16) fft_p2(const __grid_constant__ FftArgs A) {
  constexpr int K = 1 << LOGK, T = K / 16, SROW = K + K / 16 + 1;
  extern __shared__ float2 smem[];
  const int rr = threadIdx.x / T, j = threadIdx.x % T;
  const int n = A.n;
  const int k1 = blockIdx.x * R + rr;
  float2* s = smem + rr * SROW;
  const float2* row = A.tmp + (size_t)k1 * n;
  float2 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int a = unpad_index(j + i * T, n, K);
    v[i] = a >= 0 ? row[a] : make_float2(0.f, 0.f);
  }
  fft_row<LOGK, -1>(v, s, j, A.tw, A.twp);
  float2* g = A.grid + (size_t)k1 * K;
#pragma unroll
  for (int i = 0; i < 16; ++i) g[j + i * T] = v[i];
}

// ---------------------------------------------------------------- Q1
template <int LOGK, int R>
__global__ void __launch_bounds__(R * (1 << LOGK) / 16) fft_q1(const __grid_constant__ FftArgs A) {
  constexpr int K = 1 << LOGK, T = K / 16, SROW = K + K / 16 + 1;
  extern __shared__ float2 smem[];
  const int rr = threadIdx.x / T, j = threadIdx.x % T;
  const int n = A.n;
  const int k1 = blockIdx.x * R + rr;
  if (blockIdx.x == 0 && threadIdx.x < 4 && A.acc) A.acc[threadIdx.x] = 0.0;
  float2* s = smem + rr * SROW;
  float2* g = A.grid + (size_t)k1 * K;
  float2 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = g[j + i * T];
  if (A.grid_lo) {  // the compensated sums: high part + rounding errors
    __nv_bfloat162* gl = A.grid_lo + (size_t)k1 * K;
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = cadd(v[i], __bfloat1622float2(gl[j + i * T]));
#pragma unroll
    for (int i = 0; i < 16; ++i) gl[j + i * T] = __floats2bfloat162_rn(0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) g[j + i * T] = make_float2(0.f, 0.f);
  fft_row<LOGK, +1>(v, s, j, A.tw, A.twp);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16; ++i) s[PADI(j + i * T)] = v[i];
  __syncthreads();
  const int k10 = blockIdx.x * R;
  for (int idx = threadIdx.x; idx < R * n; idx += R * T) {
    const int r = idx % R, a = idx / R;
    A.tmp[(size_t)a * K + k10 + r] = smem[r * SROW + PADI(pad_position(a, n, K))];
  }
}

__device__ __forceinline__ float soft(float c, float t) {
  const float m = fabsf(c) - t;
  return m > 0.f ? copysignf(m, c) : 0.f;
}

// acc[0] += sum of v0, acc[1] += sum of v1 over the block: warp shuffles, then one pair of
// partial sums per warp in shared memory (red: 2 doubles per warp) summed by thread 0
__device__ __forceinline__ void block_reduce_add(double v0, double v1, double* acc, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (blockDim.x >= 32) {  // whole warps (blocks narrower than a warp keep one value per thread)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v0 += __shfl_xor_sync(0xffffffffu, v0, o);
      v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
  }
  __syncthreads();  // red aliases the FFT buffer
  if (blockDim.x < 32) {
    red[2 * threadIdx.x] = v0;
    red[2 * threadIdx.x + 1] = v1;
  } else if (lane == 0) {
    red[2 * warp] = v0;
    red[2 * warp + 1] = v1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (blockDim.x < 32 ? (int)blockDim.x : (int)(blockDim.x >> 5)); ++w) {
      s0 += red[2 * w];
      s1 += red[2 * w + 1];
    }
    atomicAdd(&acc[0], s0);
    atomicAdd(&acc[1], s1);
  }
}

// ---------------------------------------------------------------- Q2
// Epilogue of the last inverse pass on two image rows a0, a0 + 1 whose gradient values
// Re{Z^H F^H ...} sit in gs (2 x n, shared memory): the w-stack sum, then the adjoint / gradient
// step / gradient step + Haar prox (+ positivity) / power-iteration norm, and the FP64 sums.
template <bool CH>
__device__ __forceinline__ void q2_epilogue(const FftArgs& A, float* gs, int a0, int j, int T) {
  extern __shared__ float2 smem[];
  const int n = A.n;
  if (CH && A.gacc_mode != GACC_NONE) {
    const size_t base = (size_t)a0 * n;
    for (int i = j; i < 2 * n; i += T) {
      float g = gs[i];
      if (A.gacc_mode != GACC_WRITE) g += A.gacc[base + i];
      if (A.gacc_mode == GACC_FINAL) gs[i] = g;
      else A.gacc[base + i] = g;
    }
    if (A.gacc_mode != GACC_FINAL) return;  // uniform over the CTA
    __syncthreads();
  }
  double s0 = 0.0, s1 = 0.0;
  const float gamma = A.gamma;
  const size_t base = (size_t)a0 * n;
  if (A.epi == EPI_ADJ || A.epi == EPI_NORMAL) {
    for (int i = j; i < 2 * n; i += T) {
      const float g = gs[i];
      A.out[base + i] = g;
      s0 += (double)g * g;
    }
  } else if (A.epi == EPI_GRAD) {
    for (int i = j; i < 2 * n; i += T) A.out[base + i] = A.x[base + i] - gamma * gs[i];
  } else {  // EPI_HAAR(_NOPOS): z = x - gamma g on 2x2 blocks, Haar soft-threshold, positivity (or not)
    const float t = A.t;
    const bool pos = A.epi == EPI_HAAR;
    auto proj = [pos](float v) { return pos ? fmaxf(0.f, v) : v; };
    for (int bb = j; bb < n / 2; bb += T) {
      const int b = 2 * bb;
      const float x00 = A.x[base + b], x01 = A.x[base + b + 1];
      const float x10 = A.x[base + n + b], x11 = A.x[base + n + b + 1];
      const float z00 = x00 - gamma * gs[b], z01 = x01 - gamma * gs[b + 1];
      const float z10 = x10 - gamma * gs[n + b], z11 = x11 - gamma * gs[n + b + 1];
      const float ha = soft(0.5f * (z00 + z01 + z10 + z11), t);
      const float hh = soft(0.5f * (z00 - z01 + z10 - z11), t);
      const float hv = soft(0.5f * (z00 + z01 - z10 - z11), t);
      const float hd = soft(0.5f * (z00 - z01 - z10 + z11), t);
      const float o00 = proj(0.5f * (ha + hh + hv + hd));
      const float o01 = proj(0.5f * (ha - hh + hv - hd));
      const float o10 = proj(0.5f * (ha + hh - hv - hd));
      const float o11 = proj(0.5f * (ha - hh - hv + hd));
      A.out[base + b] = o00;
      A.out[base + b + 1] = o01;
      A.out[base + n + b] = o10;
      A.out[base + n + b + 1] = o11;
      const double d00 = (double)o00 - x00, d01 = (double)o01 - x01;
      const double d10 = (double)o10 - x10, d11 = (double)o11 - x11;
      s0 += d00 * d00 + d01 * d01 + d10 * d10 + d11 * d11;
      s1 += (double)o00 * o00 + (double)o01 * o01 + (double)o10 * o10 + (double)o11 * o11;
      // fmaxf(0, NaN) is 0, so positivity would hide a non-finite gradient: poison the norms
      if (!(isfinite(z00) && isfinite(z01) && isfinite(z10) && isfinite(z11))) s1 = __longlong_as_double(0x7ff8000000000000LL);
    }
  }
  if (A.acc && (A.epi == EPI_HAAR || A.epi == EPI_HAAR_NOPOS || A.epi == EPI_NORMAL))
    block_reduce_add(s0, s1, A.acc, reinterpret_cast<double*>(smem));
}

// Two image rows per CTA, processed one after the other through one FFT buffer.
template <int LOGK, bool CH>
__global__ void __launch_bounds__((1 << LOGK) / 16) fft_q2(const __grid_constant__ FftArgs A) {
  constexpr int K = 1 << LOGK, T = K / 16, SROW = K + K / 16 + 1;
  extern __shared__ float2 smem[];
  float* gs = reinterpret_cast<float*>(smem + SROW);  // 2 x n gradient values
  const int j = threadIdx.x;
  const int n = A.n;
  const int a0 = 2 * blockIdx.x;
#pragma unroll 1
  for (int q = 0; q < 2; ++q) {
    const int a = a0 + q;
    const float2* row = A.tmp + (size_t)a * K;
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = row[j + i * T];
    fft_row<LOGK, +1>(v, smem, j, A.tw, A.twp);
    const float ca = A.cinv[a];
    if (CH) {  // Re{conj(chirp) v}: the adjoint of the centre chirp of Z_s
      const float2 cha = A.chirp[a];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int b = unpad_index(j + i * T, n, K);
        if (b >= 0) {
          const float2 c = cmul2(cha, A.chirp[b]);
          gs[q * n + b] = (v[i].x * c.x + v[i].y * c.y) * ca * A.cinv[b];
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int b = unpad_index(j + i * T, n, K);
        if (b >= 0) gs[q * n + b] = v[i].x * ca * A.cinv[b];
      }
    }
  }
  __syncthreads();
  q2_epilogue<CH>(A, gs, a0, j, T);
}

// |centred index| of FFT index k: k for k < K/2, K - k above
__device__ __forceinline__ int centred_abs(int k, int K) { return k < K / 2 ? k : K - k; }

// ---------------------------------------------------------------- split passes (K = 2n)
// With twofold oversampling (K = 2n) each length-K transform of the operator halves into two
// length-n transforms.  Forward, n non-zero inputs at the centred positions p mod K:
//   V[2m] = DFT_n(u)[m],  V[2m + 1] = DFT_n(s w u)[m],
// with u[e] the input at centred offset e (e < n/2) or e - n (e >= n/2), s[e] = +1 (e < n/2) or -1,
// w[e] = exp(-2 pi i e / K).  Inverse, keeping the n centred outputs j in [-n/2, n/2):
//   X[j] = IDFT_n(G[0::2])[j mod n] + exp(+2 pi i j / K) IDFT_n(G[1::2])[j mod n].
// No transform runs over zero padding, and a length-n transform needs one shared-memory exchange
// fewer than a length-2n one.  Layouts and epilogues are those of the general passes above.
//
// The split passes are also pruned to the uv support of G (FftArgs rowh, band): the forward pair
// forms only the rows k1 of the band and writes only the cells of each row that hold taps (the
// degridding reads no other cell; the rest of the forward grid stays zero from the plan's start);
// the adjoint pair reads and re-zeroes only those cells of the gridded data (the gridding writes no
// other), transforms only the band's rows, and Q2 reads U only at the band's columns k1.

// P1 (split): image row a, output parity par (blockIdx.y): the even or odd half of its length-K
// transform along axis 1, written transposed into T[k1 = 2m + par][a].
template <int LOGK, int R, bool CH>
__global__ void __launch_bounds__(R * (1 << LOGK) / 32) fft_p1s(const __grid_constant__ FftArgs A) {
  constexpr int LN = LOGK - 1, N = 1 << LN, T = N / 16, SROW = N + N / 16 + 1, H = N / 2;
  extern __shared__ float2 smem[];
  const int rr = threadIdx.x / T, j = threadIdx.x % T, par = blockIdx.y;
  const int a = blockIdx.x * R + rr;
  const bool live = a < N;
  float2* s = smem + rr * SROW;
  const float ca = live ? A.cinv[a] : 0.f;
  float2 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int e = j + i * T, b = e < H ? e + H : e - H;
    float2 val = make_float2(live ? A.x[(size_t)a * N + b] * ca * A.cinv[b] : 0.f, 0.f);
    if (CH && live) {  // Z_s of a w-stack: the centre chirp, separable over the two axes
      const float2 c = cmul(A.chirp[a], A.chirp[b]);
      val = make_float2(val.x * c.x, val.x * c.y);
    }
    if (par) {
      const float2 w = A.tw[e];
      val = cmul(val, e < H ? w : make_float2(-w.x, -w.y));
    }
    v[i] = val;
  }
  const int bid = T % 32 == 0 && R < 15 ? 1 + rr : 0;  // the row's named barrier (group_sync)
  fft_row<LN, -1, 2>(v, s, j, A.tw, A.twp, bid);
  group_sync(bid, T);
#pragma unroll
  for (int i = 0; i < 16; ++i) s[PADI(j + i * T)] = v[i];
  __syncthreads();
  const int a0 = blockIdx.x * R;
  for (int idx = threadIdx.x; idx < R * N; idx += R * T) {
    const int r = idx % R, m = idx / R;
    if (a0 + r < N && centred_abs(2 * m + par, 2 * N) <= A.band)  // rows k1 outside the band: never read
      A.tmp[(size_t)(2 * m + par) * N + a0 + r] = smem[r * SROW + PADI(m)];
  }
}

// The two length-n transforms of a row run side by side: the CTA's first n/16 threads transform the
// even half in shared-memory buffer A, the next n/16 the odd half in buffer B (each group passes its
// own named barrier until the halves meet), so a thread holds one transform's 16 values (64
// registers) and two CTAs share an SM, one CTA's loads overlapping the other's transforms.
template <int LN>
struct SplitGeom {
  static constexpr int N = 1 << LN, T = N / 16, SROW = N + N / 16 + 1, H = N / 2;
  // named barrier of transform g of the CTA (group_sync), when its threads are whole warps
  static __device__ __forceinline__ int bar(int g) { return T % 32 == 0 && g < 15 ? 1 + g : 0; }
};

// P2 (split): row k1 of T (the n centred inputs along axis 0); both halves, written interleaved
// (one 16-byte store per output pair V[2m], V[2m + 1]).
template <int LOGK>
__global__ void __launch_bounds__((1 << LOGK) / 16, (1 << LOGK) / 16 <= 512 ? 2 : 1) fft_p2s(
    const __grid_constant__ FftArgs A) {
  using Sg = SplitGeom<LOGK - 1>;
  constexpr int N = Sg::N, K = 2 * N, T = Sg::T, H = Sg::H;
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, j = threadIdx.x % T, k1 = blockIdx.x;
  const int h = centred_abs(k1, K) <= A.band ? A.rowh[k1] : -1;  // the row's taps: centred |k0| <= h
  if (h < 0) return;  // a row without taps (uniform over the CTA)
  float2* buf = smem + grp * Sg::SROW;
  const float2* row = A.tmp + (size_t)k1 * N;
  float2 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int e = j + i * T;
    const float2 u = row[e < H ? e + H : e - H];
    if (grp) {
      const float2 t = A.tw[e];
      v[i] = cmul(u, e < H ? t : make_float2(-t.x, -t.y));
    } else {
      v[i] = u;
    }
  }
  fft_row<LOGK - 1, -1, 2>(v, buf, j, A.tw, A.twp, Sg::bar(grp));
  group_sync(Sg::bar(grp), T);
#pragma unroll
  for (int i = 0; i < 16; ++i) buf[PADI(j + i * T)] = v[i];
  __syncthreads();
  float4* g = reinterpret_cast<float4*>(A.grid + (size_t)k1 * K);
  const float2* be = smem;
  const float2* bo = smem + Sg::SROW;
  for (int m = threadIdx.x; m < N; m += 2 * T) {
    if (min(centred_abs(2 * m, K), centred_abs(2 * m + 1, K)) > h) continue;  // no tap in the pair
    const float2 e = be[PADI(m)], o = bo[PADI(m)];
    g[m] = make_float4(e.x, e.y, o.x, o.y);
  }
}

// exp(+2 pi i jo / K) X_o + X_e for the centred output offset jo of transform index q
__device__ __forceinline__ float2 split_combine(float2 xe, float2 xo, int q, int N, const float2* __restrict__ tw) {
  const int jo = q < N / 2 ? q : q - N;
  const float2 t = tw[jo < 0 ? jo + 2 * N : jo];  // exp(-2 pi i jo / K)
  return make_float2(xe.x + xo.x * t.x + xo.y * t.y, xe.y + xo.y * t.x - xo.x * t.y);
}

// Both inverse transforms of a row whose even (grp 0) or odd (grp 1) samples this thread holds in v:
// on return buffer A holds IDFT_n(G[0::2]) and buffer B IDFT_n(G[1::2]) (natural order, padded).
// g: the transform's index in the CTA (its named barrier); the last barrier is the CTA's, since the
// combination reads both buffers.
template <int LN>
__device__ __forceinline__ void split_inverse(float2 (&v)[16], float2* buf, int j,
                                              const float2* __restrict__ tw, const float2* __restrict__ twp, int g) {
  using Sg = SplitGeom<LN>;
  constexpr int T = Sg::T;
  fft_row<LN, +1, 2>(v, buf, j, tw, twp, Sg::bar(g));
  group_sync(Sg::bar(g), T);
#pragma unroll
  for (int i = 0; i < 16; ++i) buf[PADI(j + i * T)] = v[i];
  __syncthreads();
}

// Q1 (split): rows k1, k1 + 1 of the gridded data (for each, the even samples to one thread group,
// the odd to another, plus the compensation grid), inverse transforms, and the n centred outputs of
// both rows written transposed into U[a][k1 .. k1 + 1] (one 16-byte store per image row a); the grid
// (and compensation grid) rows are re-zeroed.
template <int LOGK, int R>
__global__ void __launch_bounds__(R * (1 << LOGK) / 16) fft_q1s(const __grid_constant__ FftArgs A) {
  using Sg = SplitGeom<LOGK - 1>;
  constexpr int N = Sg::N, K = 2 * N, T = Sg::T, H = Sg::H;
  extern __shared__ float2 smem[];
  const int r = threadIdx.x / (2 * T), grp = (threadIdx.x / T) & 1, j = threadIdx.x % T;
  const int k10 = R * blockIdx.x, k1 = k10 + r;
  float2* buf = smem + (2 * r + grp) * Sg::SROW;
  if (blockIdx.x == 0 && threadIdx.x < 4 && A.acc) A.acc[threadIdx.x] = 0.0;
  bool any = false;  // a row of the CTA in the band (else Q2 never reads its columns of U)
#pragma unroll
  for (int q = 0; q < R; ++q) any |= centred_abs(k10 + q, K) <= A.band;
  if (!any) return;
  const int h = centred_abs(k1, K) <= A.band ? A.rowh[k1] : -1;  // cells with centred |k0| <= h
  float2* g = A.grid + (size_t)k1 * K + grp;  // sample 2 m + grp at g[2 m]
  float2 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const bool in = centred_abs(2 * (j + i * T) + grp, K) <= h;
    v[i] = in ? g[2 * (j + i * T)] : make_float2(0.f, 0.f);
  }
  if (A.grid_lo) {  // the compensated sums: high part + rounding errors (BF16 pairs)
    __nv_bfloat162* gl = A.grid_lo + (size_t)k1 * K + grp;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      if (centred_abs(2 * (j + i * T) + grp, K) > h) continue;
      v[i] = cadd(v[i], __bfloat1622float2(gl[2 * (j + i * T)]));
      gl[2 * (j + i * T)] = __floats2bfloat162_rn(0.f, 0.f);
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i)
    if (centred_abs(2 * (j + i * T) + grp, K) <= h) g[2 * (j + i * T)] = make_float2(0.f, 0.f);
  split_inverse<LOGK - 1>(v, buf, j, A.tw, A.twp, 2 * r + grp);
  // transform index q holds image row a = q + n/2 (q < n/2) or q - n/2; combined into the odd
  // buffer: each thread of the row takes pairs (q, q + n/2), both read before either is written
  const float2* be = smem + 2 * r * Sg::SROW;
  float2* bo = smem + (2 * r + 1) * Sg::SROW;
  for (int q = threadIdx.x % (2 * T); q < H; q += 2 * T) {
    const float2 lo = split_combine(be[PADI(q)], bo[PADI(q)], q, N, A.tw);
    const float2 hi = split_combine(be[PADI(q + H)], bo[PADI(q + H)], q + H, N, A.tw);
    bo[PADI(q + H)] = lo;
    bo[PADI(q)] = hi;
  }
  __syncthreads();
  const float2* x0 = smem + Sg::SROW;
  if constexpr (R == 2) {
    const float2* x1 = smem + 3 * Sg::SROW;
    for (int a = threadIdx.x; a < N; a += 4 * T) {
      const float2 u0 = x0[PADI(a)], u1 = x1[PADI(a)];
      *reinterpret_cast<float4*>(A.tmp + (size_t)a * K + k10) = make_float4(u0.x, u0.y, u1.x, u1.y);
    }
  } else {
    for (int a = threadIdx.x; a < N; a += 2 * T) A.tmp[(size_t)a * K + k10] = x0[PADI(a)];
  }
}

// Q2 (split): rows a of U (even samples to one thread group, odd to the other), inverse transforms
// and the centred outputs, then the epilogue of fft_q2 (two image rows per CTA).
template <int LOGK, bool CH>
__global__ void __launch_bounds__((1 << LOGK) / 16, (1 << LOGK) / 16 <= 512 ? 2 : 1) fft_q2s(
    const __grid_constant__ FftArgs A) {
  using Sg = SplitGeom<LOGK - 1>;
  constexpr int N = Sg::N, K = 2 * N, T = Sg::T, H = Sg::H;
  extern __shared__ float2 smem[];
  const int grp = threadIdx.x / T, j = threadIdx.x % T;
  float2* buf = smem + grp * Sg::SROW;
  float* gs = reinterpret_cast<float*>(smem + 2 * Sg::SROW);  // 2 x n gradient values
  const int a0 = 2 * blockIdx.x;
#pragma unroll 1
  for (int q2 = 0; q2 < 2; ++q2) {
    const int a = a0 + q2;
    const float2* row = A.tmp + (size_t)a * K + grp;
    if (q2) __syncthreads();  // the previous row is done with both buffers
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i)  // columns k1 = 2 m + grp outside the band are zero (Q1 skips them)
      v[i] = centred_abs(2 * (j + i * T) + grp, K) <= A.band ? row[2 * (j + i * T)] : make_float2(0.f, 0.f);
    split_inverse<LOGK - 1>(v, buf, j, A.tw, A.twp, grp);
    const float ca = A.cinv[a];
    const float2 cha = CH ? A.chirp[a] : make_float2(1.f, 0.f);
    const float2* be = smem;
    const float2* bo = smem + Sg::SROW;
    for (int q = threadIdx.x; q < N; q += 2 * T) {
      const int b = q < H ? q + H : q - H;
      const float2 x = split_combine(be[PADI(q)], bo[PADI(q)], q, N, A.tw);
      if (CH) {  // Re{conj(chirp) x}: the adjoint of the centre chirp of Z_s
        const float2 c = cmul(cha, A.chirp[b]);
        gs[q2 * N + b] = (x.x * c.x + x.y * c.y) * ca * A.cinv[b];
      } else {
        gs[q2 * N + b] = x.x * ca * A.cinv[b];
      }
    }
  }
  __syncthreads();
  q2_epilogue<CH>(A, gs, a0, threadIdx.x, 2 * T);
}

// ---------------------------------------------------------------- launchers
constexpr int SMEM_BUDGET = 140 * 1024;

template <int LOGK>
constexpr int rows_per_cta() {
  constexpr int K = 1 << LOGK, T = K / 16;
  int r = 16;
  while (r > 1 && (r * T > 1024 || r * (K + K / 16) * 8 > SMEM_BUDGET)) r >>= 1;
  return r;
}

// rows per CTA of the split passes: T = K / 32 threads per row, at most `max_threads` threads and
// `max_rows` rows, the rows' buffers within the shared-memory budget
template <int LOGK>
constexpr int split_rows(int max_threads, int max_rows) {
  constexpr int N = 1 << (LOGK - 1), T = N / 16;
  int r = max_rows;
  while (r > 1 && (r * T > max_threads || r * (N + N / 16 + 1) * 8 > SMEM_BUDGET)) r >>= 1;
  return r;
}

// the split passes when K = 2n (every launch configuration of the general passes otherwise)
template <int LOGK>
int launch_forward_split(pnp_plan* p, const FftArgs& A) {
  using Sg = SplitGeom<LOGK - 1>;
  constexpr int N = Sg::N, T = Sg::T;
  constexpr int R1 = split_rows<LOGK>(1024, 16);
  const int smem1 = R1 * Sg::SROW * 8, smem2 = 2 * Sg::SROW * 8;
  static bool attr = false;
  if (!attr) {
    PNP_CUDA(cudaFuncSetAttribute(fft_p1s<LOGK, R1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    PNP_CUDA(cudaFuncSetAttribute(fft_p1s<LOGK, R1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    PNP_CUDA(cudaFuncSetAttribute(fft_p2s<LOGK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    attr = true;
  }
  const dim3 g1((N + R1 - 1) / R1, 2);
  if (A.chirp)
    fft_p1s<LOGK, R1, true><<<g1, R1 * T, smem1, p->stream>>>(A);
  else
    fft_p1s<LOGK, R1, false><<<g1, R1 * T, smem1, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  fft_p2s<LOGK><<<2 * N, 2 * T, smem2, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

template <int LOGK>
int launch_adjoint_split(pnp_plan* p, const FftArgs& A) {
  using Sg = SplitGeom<LOGK - 1>;
  constexpr int N = Sg::N, T = Sg::T;
  constexpr int RQ = 4 * T <= 1024 ? 2 : 1;  // grid rows per Q1 CTA (two thread groups each)
  const int smem1 = 2 * RQ * Sg::SROW * 8;
  const int smem2 = 2 * Sg::SROW * 8 + 2 * N * 4;
  static bool attr = false;
  if (!attr) {
    PNP_CUDA(cudaFuncSetAttribute(fft_q1s<LOGK, RQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    PNP_CUDA(cudaFuncSetAttribute(fft_q2s<LOGK, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    PNP_CUDA(cudaFuncSetAttribute(fft_q2s<LOGK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    attr = true;
  }
  fft_q1s<LOGK, RQ><<<2 * N / RQ, RQ * 2 * T, smem1, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  if (A.chirp)
    fft_q2s<LOGK, true><<<N / 2, 2 * T, smem2, p->stream>>>(A);
  else
    fft_q2s<LOGK, false><<<N / 2, 2 * T, smem2, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

template <int LOGK>
int launch_forward(pnp_plan* p, const FftArgs& A) {
  if (2 * p->n == (1 << LOGK)) return launch_forward_split<LOGK>(p, A);
  constexpr int K = 1 << LOGK, T = K / 16, R = rows_per_cta<LOGK>(), SROW = K + K / 16 + 1;
  const int smem = R * SROW * 8;
  static bool attr = false;
  if (!attr) {
    PNP_CUDA(cudaFuncSetAttribute(fft_p1<LOGK, R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    PNP_CUDA(cudaFuncSetAttribute(fft_p1<LOGK, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    PNP_CUDA(cudaFuncSetAttribute(fft_p2<LOGK, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = true;
  }
  if (A.chirp)
    fft_p1<LOGK, R, true><<<(p->n + R - 1) / R, R * T, smem, p->stream>>>(A);
  else
    fft_p1<LOGK, R, false><<<(p->n + R - 1) / R, R * T, smem, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  fft_p2<LOGK, R><<<K / R, R * T, smem, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

template <int LOGK>
int launch_adjoint(pnp_plan* p, const FftArgs& A) {
  if (2 * p->n == (1 << LOGK)) return launch_adjoint_split<LOGK>(p, A);
  constexpr int K = 1 << LOGK, T = K / 16, R = rows_per_cta<LOGK>(), SROW = K + K / 16 + 1;
  const int smem1 = R * SROW * 8;
  const int smem2 = SROW * 8 + 2 * p->n * 4;
  static int attr2 = 0;
  static bool attr1 = false;
  if (!attr1) {
    PNP_CUDA(cudaFuncSetAttribute(fft_q1<LOGK, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    attr1 = true;
  }
  if (smem2 > attr2) {
    PNP_CUDA(cudaFuncSetAttribute(fft_q2<LOGK, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    PNP_CUDA(cudaFuncSetAttribute(fft_q2<LOGK, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem2));
    attr2 = smem2;
  }
  fft_q1<LOGK, R><<<K / R, R * T, smem1, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  if (A.chirp)
    fft_q2<LOGK, true><<<p->n / 2, T, smem2, p->stream>>>(A);
  else
    fft_q2<LOGK, false><<<p->n / 2, T, smem2, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

}  // namespace

int fft_forward(pnp_plan* p, const float* x, int s) {
  if (s < 0 || s >= p->nstacks) return fail(PNP_ERR_INVALID_ARG, "internal: stack index out of range");
  FftArgs A{};
  A.chirp = p->nstacks > 1 ? p->d_chirp + (size_t)s * p->n : nullptr;
  A.n = p->n;
  A.x = x;
  A.cinv = p->d_cinv;
  A.tw = p->d_tw;
  A.twp = p->d_twp;
  A.tmp = p->d_tmp;
  A.grid = p->d_gridA;
  A.rowh = p->d_rowh;
  A.band = p->band;
  cudaEvent_t ev;
  if (int rc = stage_begin(p, 0, &ev)) return rc;
  int rc = PNP_OK;
  switch (p->logK) {
    case 6: rc = launch_forward<6>(p, A); break;
    case 7: rc = launch_forward<7>(p, A); break;
    case 8: rc = launch_forward<8>(p, A); break;
    case 9: rc = launch_forward<9>(p, A); break;
    case 10: rc = launch_forward<10>(p, A); break;
    case 11: rc = launch_forward<11>(p, A); break;
    case 12: rc = launch_forward<12>(p, A); break;
    case 13: rc = launch_forward<13>(p, A); break;
    case 14: rc = launch_forward<14>(p, A); break;
    default: rc = fail(PNP_ERR_UNSUPPORTED, "grid side K must be 2^6..2^14");
  }
  if (rc) return rc;
  return stage_end(p, 0, ev);
}

int fft_adjoint(pnp_plan* p, int mode, const float* x, float* out, float gamma, float t, int s) {
  if (s < 0 || s >= p->nstacks) return fail(PNP_ERR_INVALID_ARG, "internal: stack index out of range");
  FftArgs A{};
  if (p->nstacks > 1) {
    A.chirp = p->d_chirp + (size_t)s * p->n;
    A.gacc = p->d_gacc;
    A.gacc_mode = s == 0 ? GACC_WRITE : (s == p->nstacks - 1 ? GACC_FINAL : GACC_ADD);
  }
  A.n = p->n;
  A.x = x;
  A.cinv = p->d_cinv;
  A.tw = p->d_tw;
  A.twp = p->d_twp;
  A.tmp = p->d_tmp;
  A.grid = p->d_gridB;
  A.grid_lo = p->compensated ? p->d_gridB_lo : nullptr;
  A.rowh = p->d_rowh;
  A.band = p->band;
  A.out = out;
  A.acc = p->d_acc;
  A.gamma = gamma;
  A.t = t;
  A.epi = mode;
  cudaEvent_t ev;
  if (int rc = stage_begin(p, 2, &ev)) return rc;
  int rc = PNP_OK;
  switch (p->logK) {
    case 6: rc = launch_adjoint<6>(p, A); break;
    case 7: rc = launch_adjoint<7>(p, A); break;
    case 8: rc = launch_adjoint<8>(p, A); break;
    case 9: rc = launch_adjoint<9>(p, A); break;
    case 10: rc = launch_adjoint<10>(p, A); break;
    case 11: rc = launch_adjoint<11>(p, A); break;
    case 12: rc = launch_adjoint<12>(p, A); break;
    case 13: rc = launch_adjoint<13>(p, A); break;
    case 14: rc = launch_adjoint<14>(p, A); break;
    default: rc = fail(PNP_ERR_UNSUPPORTED, "grid side K must be 2^6..2^14");
  }
  if (rc) return rc;
  return stage_end(p, 2, ev);
}

}  // namespace pnp
