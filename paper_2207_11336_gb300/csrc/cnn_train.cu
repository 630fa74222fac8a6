// Training of the residual CNN denoiser (App. C): l1 loss
//   E || D(u + sigma n) - u ||_1,  D(z) = z - N(z)   (Eq. training_loss, without
// the firm non-expansiveness term), Adam updates, hand-written forward and
// backward kernels.  The Gaussian draws n are inputs.
//
// Precision: weights are kept in FP32 (master copy) and rounded to BF16 for
// every convolution, as in inference; hidden activations and the back-propagated
// pre-activation gradients are BF16 in memory; the loss gradient, weight
// gradients and Adam moments are FP32.
//
// Per step:
//   forward   z = u + sigma n; layer 1 (CUDA cores) -> act1; layers 2..7 on the
//             tensor cores (conv64 forward mode) -> act2..act7; layer 8 and the
//             l1 loss and its gradient g = dL/dN (CUDA cores);
//   backward  dpre7 = (W8^T g) * [act7 > 0];  for k = 6..1: dW_{k+1} from
//             (dpre_{k+1}, act_k) on the tensor cores (mma.sync, the pixels as the
//             contraction) and dpre_k = conv(dpre_{k+1}, flipped W_{k+1}^T)
//             * [act_k > 0] on the tensor cores (conv64 backward-data mode);
//             dW1 from (dpre_1, z) and dW8 on CUDA cores (one channel); bias
//             gradients are pixel sums of dpre;
//   update    Adam on the FP32 master weights, then re-pack the BF16 operands.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace pnp {
namespace {

constexpr int CH = 64;
constexpr int NW1 = CH * 9, NB1 = CH, NWM = CH * CH * 9, NBM = CH, NW8 = CH * 9;
constexpr int64_t OFF_W1 = 0, OFF_B1 = NW1;
constexpr int64_t OFF_MID = NW1 + NB1;  // 6 x (W, b)
constexpr int64_t MID_STRIDE = NWM + NBM;
constexpr int64_t OFF_W8 = OFF_MID + 6 * MID_STRIDE, OFF_B8 = OFF_W8 + NW8;
constexpr int64_t NPARAM = OFF_B8 + 1;
constexpr int WG_CHUNK = 2048;  // pixels per weight-gradient block

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// master FP32 weights -> BF16-rounded first/last layers, biases, packed middle-layer operands
__global__ void prep_weights(const float* __restrict__ w, float* __restrict__ w1r, float* __restrict__ w8r,
                             float* __restrict__ bias, __nv_bfloat16* __restrict__ wf,
                             __nv_bfloat16* __restrict__ wb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < 6 * (int64_t)NWM) {
    const int l = (int)(i / NWM), r = (int)(i % NWM);
    const int co = r / (CH * 9), ci = (r / 9) % CH, t = r % 9;
    const __nv_bfloat16 v = __float2bfloat16_rn(w[OFF_MID + l * MID_STRIDE + r]);
    // forward operand: tap (dy, dx), input ci, output co
    wf[(size_t)l * NWM + conv_wpack_index(t / 3, t % 3, ci, co)] = v;
    // backward-data operand: the flipped tap (2 - dy, 2 - dx) with input and output channels swapped
    wb[(size_t)l * NWM + conv_wpack_index(2 - t / 3, 2 - t % 3, co, ci)] = v;
  }
  if (i < NW1) w1r[i] = bf16r(w[OFF_W1 + i]);
  if (i < NW8) {
    const int ci = (int)(i / 9), t = (int)(i % 9);
    w8r[t * CH + ci] = bf16r(w[OFF_W8 + i]);
  }
  if (i < 8 * CH) {
    const int l = (int)(i / CH), c = (int)(i % CH);
    float b = 0.f;
    if (l == 0) b = w[OFF_B1 + c];
    else if (l < 7) b = w[OFF_MID + (l - 1) * MID_STRIDE + NWM + c];
    else if (c == 0) b = w[OFF_B8];
    bias[i] = b;
  }
}

__global__ void make_z(const float* __restrict__ u, const float* __restrict__ nz, float sigma, float* __restrict__ z,
                       int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = u[i] + sigma * nz[i];
}

struct Dims {
  int B, s, Hc, Wc;
};

__device__ __forceinline__ size_t cidx(const Dims& d, int b, int y, int x, int c) {
  return canvas_index(b, y, x, c, d.Hc, d.Wc);
}

// layer 8 forward, l1 loss and g = dL/dN = -sign(z - N - u) / count
__global__ void __launch_bounds__(256) last_fwd_loss(Dims d, const __nv_bfloat16* __restrict__ act7,
                                                     const float* __restrict__ w8r, const float* __restrict__ bias,
                                                     const float* __restrict__ z, const float* __restrict__ u,
                                                     float* __restrict__ g, double* loss) {
  __shared__ float sw[9 * CH];
  __shared__ double red[256];
  for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[i] = w8r[i];
  __syncthreads();
  const int64_t total = (int64_t)d.B * d.s * d.s;
  const float inv = 1.f / (float)total;
  double s = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / ((int64_t)d.s * d.s)), y = (int)((p / d.s) % d.s), x = (int)(p % d.s);
    float nz = bias[7 * CH];
    for (int t = 0; t < 9; ++t) {
      const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
      if (yy < 0 || yy >= d.s || xx < 0 || xx >= d.s) continue;
#pragma unroll
      for (int cb = 0; cb < 8; ++cb) {
        const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(act7 + cidx(d, b, yy, xx, 8 * cb));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = 4 * cb + k;
          const float2 v = __bfloat1622float2(a[k]);
          nz = fmaf(sw[t * CH + 2 * c], v.x, fmaf(sw[t * CH + 2 * c + 1], v.y, nz));
        }
      }
    }
    const float r = z[p] - nz - u[p];
    s += fabs((double)r);
    g[p] = r > 0.f ? -inv : (r < 0.f ? inv : 0.f);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x >> 1; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * (double)inv);
}

// dpre7[q][ci] = [act7[q][ci] > 0] * sum_t W8[ci][t] g[q - off_t]
__global__ void __launch_bounds__(256) last_bwd(Dims d, const __nv_bfloat16* __restrict__ act7,
                                                const float* __restrict__ w8r, const float* __restrict__ g,
                                                __nv_bfloat16* __restrict__ dpre) {
  __shared__ float sw[9 * CH];
  for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[i] = w8r[i];
  __syncthreads();
  const int64_t total = (int64_t)d.B * d.s * d.s;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / ((int64_t)d.s * d.s)), y = (int)((p / d.s) % d.s), x = (int)(p % d.s);
    float gt[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = y - (t / 3 - 1), xx = x - (t % 3 - 1);
      gt[t] = (yy >= 0 && yy < d.s && xx >= 0 && xx < d.s) ? g[((int64_t)b * d.s + yy) * d.s + xx] : 0.f;
    }
#pragma unroll 4
    for (int c = 0; c < CH / 2; ++c) {
      const size_t at = cidx(d, b, y, x, 2 * c);
      float v0 = 0.f, v1 = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        v0 = fmaf(sw[t * CH + 2 * c], gt[t], v0);
        v1 = fmaf(sw[t * CH + 2 * c + 1], gt[t], v1);
      }
      const float2 av = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(act7 + at));
      *reinterpret_cast<__nv_bfloat162*>(dpre + at) =
          __floats2bfloat162_rn(av.x > 0.f ? v0 : 0.f, av.y > 0.f ? v1 : 0.f);
    }
  }
}

// Gradients of a one-channel layer: thread (t, c) accumulates sum_p s1[p] * s2(p + off_t)[c]
// where one side is a one-channel FP32 image and the other a 64-channel canvas.
//   mode 0 (layer 8): dW8[c][t] += sum_p g[p] act7[p + off_t][c];   db8 += sum_p g[p]
//   mode 1 (layer 1): dW1[c][t] += sum_p dpre1[p][c] z[p + off_t];    db1[c] += sum_p dpre1[p][c]
__global__ void __launch_bounds__(576) wgrad_onechannel(Dims d, int mode, const float* __restrict__ img,
                                                        const __nv_bfloat16* __restrict__ cv, float* __restrict__ dW,
                                                        float* __restrict__ db) {
  const int t = threadIdx.x / CH, c = threadIdx.x % CH;
  const int64_t total = (int64_t)d.B * d.s * d.s;
  const int64_t p0 = (int64_t)blockIdx.x * WG_CHUNK, p1 = min(total, p0 + WG_CHUNK);
  const int dy = t / 3 - 1, dx = t % 3 - 1;
  float acc = 0.f, bacc = 0.f;
  for (int64_t p = p0; p < p1; ++p) {
    const int b = (int)(p / ((int64_t)d.s * d.s)), y = (int)((p / d.s) % d.s), x = (int)(p % d.s);
    const int yy = y + dy, xx = x + dx;
    const bool in = yy >= 0 && yy < d.s && xx >= 0 && xx < d.s;
    if (mode == 0) {
      const float gv = img[p];
      if (in) acc = fmaf(gv, __bfloat162float(cv[cidx(d, b, yy, xx, c)]), acc);
      bacc += gv;
    } else {
      const float dv = __bfloat162float(cv[cidx(d, b, y, x, c)]);
      if (in) acc = fmaf(dv, img[((int64_t)b * d.s + yy) * d.s + xx], acc);
      bacc += dv;
    }
  }
  if (mode == 0) {
    atomicAdd(&dW[c * 9 + t], acc);
    if (threadIdx.x == 0) atomicAdd(&db[0], bacc);
  } else {
    atomicAdd(&dW[c * 9 + t], acc);
    if (t == 4) atomicAdd(&db[c], bacc);
  }
}

// dW[co][ci][t] += sum_p dpre[p][co] act[p + off_t][ci]; db[co] += sum_p dpre[p][co] (t == 4 blocks)
// Weight and bias gradients of a 64 -> 64 layer on the tensor cores (mma.sync m16n8k16, BF16 in, FP32
// accumulate): dW[co][ci][t] = sum_p dpre[p][co] act[p + off_t][ci] is, per tap t, a 64 x 64 GEMM whose
// contraction runs over the pixels.  A CTA walks image rows (b, y) in 64-pixel segments; per segment it
// copies dpre (64 px x 64 ch) and the three activation rows y - 1, y, y + 1 (66 px with the dx halo,
// zero outside the image) into shared memory as [pixel][channel] rows padded to 72 channels (conflict-free
// ldmatrix) with cp.async, double buffered: the next segment's copies are in flight while the current one
// is contracted.  Warp w owns tap w / 2 and output channels 32 (w % 2) .. + 31: 2 x 8 tiles of 16 x 8
// accumulators.  Both operands are stored pixel-major, so the fragments load with ldmatrix.trans.  Bias
// gradients (sums of dpre over the pixels) come from the staged dpre.  One atomic per gradient entry per
// CTA at the end.
constexpr int WGT_PX = 64;                    // pixels per segment (4 K steps of 16)
constexpr int WGT_LD = 72;                    // staged row length (channels + 8 of padding)
constexpr int WGT_WARPS = 18;                 // 9 taps x 2 output-channel halves
constexpr int WGT_THREADS = WGT_WARPS * 32;
constexpr int WGT_CHUNKS = 8 * (WGT_PX + 3 * (WGT_PX + 2));  // 16-byte chunks per segment: 2096
constexpr int WGT_BUF = (WGT_PX + 3 * (WGT_PX + 2)) * WGT_LD;  // staged elements per segment
constexpr int WGT_SMEM = 2 * WGT_BUF * 2;                       // bytes, two buffers

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
// 16-byte asynchronous copy global -> shared; nbytes = 0 fills the destination with zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(
                   __cvta_generic_to_shared(dst))),
               "l"(src), "r"(nbytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// copies of segment sg (image row b * s + y, pixels x0 ..) into the staging buffer buf: chunk e is 16
// bytes of dpre (e < 512, into [px][WGT_LD]) or of activation row y + r - 1 (into [3][66 px][WGT_LD])
__device__ __forceinline__ void wgt_issue(const Dims& d, const __nv_bfloat16* __restrict__ dpre,
                                          const __nv_bfloat16* __restrict__ act, int64_t sg, int segs_per_row,
                                          __nv_bfloat16* buf) {
  const int row = (int)(sg / segs_per_row), x0 = (int)(sg % segs_per_row) * WGT_PX;
  const int b = row / d.s, y = row % d.s;
  for (int e = threadIdx.x; e < WGT_CHUNKS; e += WGT_THREADS) {
    int yy = y, x, kb, slot;
    const __nv_bfloat16* src = dpre;
    if (e < 8 * WGT_PX) {
      x = x0 + (e >> 3);
      kb = e & 7;
      slot = (e >> 3) * WGT_LD + 8 * kb;
    } else {
      const int f = e - 8 * WGT_PX, r = f / (8 * (WGT_PX + 2)), q = f % (8 * (WGT_PX + 2));
      yy = y + r - 1;
      x = x0 - 1 + (q >> 3);
      kb = q & 7;
      slot = WGT_PX * WGT_LD + (r * (WGT_PX + 2) + (q >> 3)) * WGT_LD + 8 * kb;
      src = act;
    }
    const bool in = yy >= 0 && yy < d.s && x >= 0 && x < d.s;
    cp_async16(buf + slot, in ? src + cidx(d, b, yy, x, 8 * kb) : src, in ? 16 : 0);
  }
}

__global__ void __launch_bounds__(WGT_THREADS, 1) wgrad64_tc(Dims d, const __nv_bfloat16* __restrict__ dpre,
                                                             const __nv_bfloat16* __restrict__ act,
                                                             float* __restrict__ dW, float* __restrict__ db) {
  extern __shared__ __align__(16) __nv_bfloat16 wsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = warp >> 1, dy = t / 3, dx = t % 3, co0 = 32 * (warp & 1);
  const int segs_per_row = (d.s + WGT_PX - 1) / WGT_PX;
  const int64_t nseg = (int64_t)d.B * d.s * segs_per_row;
  float acc[2][8][4] = {};
  float bsum = 0.f;
  int cur = 0;
  if ((int64_t)blockIdx.x < nseg) wgt_issue(d, dpre, act, blockIdx.x, segs_per_row, wsm);
  cp_async_commit();
  const int i = lane >> 3, r = lane & 7;
  for (int64_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
    if (sg + gridDim.x < nseg) wgt_issue(d, dpre, act, sg + gridDim.x, segs_per_row, wsm + (1 - cur) * WGT_BUF);
    cp_async_commit();
    cp_async_wait1();  // this thread's copies of the current segment have landed
    __syncthreads();   // and everyone's
    const __nv_bfloat16* sA = wsm + cur * WGT_BUF;
    const __nv_bfloat16* sB = sA + WGT_PX * WGT_LD;
    if (threadIdx.x < CH) {
      float sacc = 0.f;
      for (int p = 0; p < WGT_PX; ++p) sacc += __bfloat162float(sA[p * WGT_LD + threadIdx.x]);
      bsum += sacc;
    }
#pragma unroll
    for (int kk = 0; kk < WGT_PX / 16; ++kk) {
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        ldsm_x4_trans(a[mt], sA + (16 * kk + r + 8 * (i >> 1)) * WGT_LD + co0 + 16 * mt + 8 * (i & 1));
#pragma unroll
      for (int np = 0; np < 4; ++np) {
        uint32_t bq[4];
        ldsm_x4_trans(bq, sB + (dy * (WGT_PX + 2) + 16 * kk + r + 8 * (i & 1) + dx) * WGT_LD + 16 * np + 8 * (i >> 1));
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma16816(acc[mt][2 * np], a[mt], bq[0], bq[1]);
          mma16816(acc[mt][2 * np + 1], a[mt], bq[2], bq[3]);
        }
      }
    }
    __syncthreads();  // the buffer is refilled by the next iteration's copies
    cur = 1 - cur;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  const int g = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int co = co0 + 16 * mt + g + 8 * h, ci = 8 * nt + 2 * tq;
        atomicAdd(&dW[((size_t)co * CH + ci) * 9 + t], acc[mt][nt][2 * h]);
        atomicAdd(&dW[((size_t)co * CH + ci + 1) * 9 + t], acc[mt][nt][2 * h + 1]);
      }
  if (threadIdx.x < CH && db) atomicAdd(&db[threadIdx.x], bsum);
}

int wgrad64_launch(cudaStream_t s, const Dims& d, const __nv_bfloat16* dpre, const __nv_bfloat16* act, float* dW,
                   float* db) {
  static bool attr = false;
  if (!attr) {
    PNP_CUDA(cudaFuncSetAttribute(wgrad64_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, WGT_SMEM));
    attr = true;
  }
  const int64_t nseg = (int64_t)d.B * d.s * ((d.s + WGT_PX - 1) / WGT_PX);
  int dev = 0, sms = 0;
  PNP_CUDA(cudaGetDevice(&dev));
  PNP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nseg, sms));
  wgrad64_tc<<<grid, WGT_THREADS, WGT_SMEM, s>>>(d, dpre, act, dW, db);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

// ---------------------------------------------------------------- Jacobian of Q = 2D - I
// With D(z) = z - N(z), J_Q = I - 2 J_N, and J_N at z is the network with its ReLU masks at z
// frozen and no biases.  Layers 2-7 of J_N v run on the tensor cores (conv64 backward-data mode
// with the forward weights and the masks [act_{k+1} > 0]); J_N^T w is the back-propagation of
// the training step.  These kernels are the one-channel ends of both chains.

// t1[p][c] = [act1[p][c] > 0] * sum_t W1[c][t] v[p + off_t]
__global__ void __launch_bounds__(256) tangent_first(Dims d, const float* __restrict__ v,
                                                     const float* __restrict__ w1r,
                                                     const __nv_bfloat16* __restrict__ act1,
                                                     __nv_bfloat16* __restrict__ t1) {
  __shared__ float sw[9 * CH];
  for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[i] = w1r[i];
  __syncthreads();
  const int64_t total = (int64_t)d.B * d.s * d.s;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / ((int64_t)d.s * d.s)), y = (int)((p / d.s) % d.s), x = (int)(p % d.s);
    float vt[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
      vt[t] = (yy >= 0 && yy < d.s && xx >= 0 && xx < d.s) ? v[((int64_t)b * d.s + yy) * d.s + xx] : 0.f;
    }
#pragma unroll 4
    for (int c = 0; c < CH / 2; ++c) {
      const size_t at = cidx(d, b, y, x, 2 * c);
      float v0 = 0.f, v1 = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        v0 = fmaf(sw[(2 * c) * 9 + t], vt[t], v0);
        v1 = fmaf(sw[(2 * c + 1) * 9 + t], vt[t], v1);
      }
      const float2 av = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(act1 + at));
      *reinterpret_cast<__nv_bfloat162*>(t1 + at) = __floats2bfloat162_rn(av.x > 0.f ? v0 : 0.f, av.y > 0.f ? v1 : 0.f);
    }
  }
}

// w[p] = v[p] - 2 sum_{t, c} W8[c][t] t7[p + off_t][c]   (J_Q v from the layer-7 tangent)
__global__ void __launch_bounds__(256) tangent_last(Dims d, const __nv_bfloat16* __restrict__ t7,
                                                    const float* __restrict__ w8r, const float* __restrict__ v,
                                                    float* __restrict__ w) {
  __shared__ float sw[9 * CH];
  for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[i] = w8r[i];
  __syncthreads();
  const int64_t total = (int64_t)d.B * d.s * d.s;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / ((int64_t)d.s * d.s)), y = (int)((p / d.s) % d.s), x = (int)(p % d.s);
    float jn = 0.f;
    for (int t = 0; t < 9; ++t) {
      const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
      if (yy < 0 || yy >= d.s || xx < 0 || xx >= d.s) continue;
#pragma unroll
      for (int cb = 0; cb < 8; ++cb) {
        const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(t7 + cidx(d, b, yy, xx, 8 * cb));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = 4 * cb + k;
          const float2 tv = __bfloat1622float2(a[k]);
          jn = fmaf(sw[t * CH + 2 * c], tv.x, fmaf(sw[t * CH + 2 * c + 1], tv.y, jn));
        }
      }
    }
    w[p] = v[p] - 2.f * jn;
  }
}

// u[p] = w[p] - 2 sum_{t, c} W1[c][t] dpre1[p - off_t][c]   (J_Q^T w from the layer-1 gradient)
__global__ void __launch_bounds__(256) cotangent_first(Dims d, const __nv_bfloat16* __restrict__ dpre1,
                                                       const float* __restrict__ w1r, const float* __restrict__ w,
                                                       float* __restrict__ u) {
  __shared__ float sw[9 * CH];  // [t][c]
  for (int i = threadIdx.x; i < 9 * CH; i += blockDim.x) sw[(i % 9) * CH + i / 9] = w1r[i];
  __syncthreads();
  const int64_t total = (int64_t)d.B * d.s * d.s;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total; p += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(p / ((int64_t)d.s * d.s)), y = (int)((p / d.s) % d.s), x = (int)(p % d.s);
    float jt = 0.f;
    for (int t = 0; t < 9; ++t) {
      const int yy = y - (t / 3 - 1), xx = x - (t % 3 - 1);
      if (yy < 0 || yy >= d.s || xx < 0 || xx >= d.s) continue;
#pragma unroll
      for (int cb = 0; cb < 8; ++cb) {
        const __nv_bfloat162* a = reinterpret_cast<const __nv_bfloat162*>(dpre1 + cidx(d, b, yy, xx, 8 * cb));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int c = 4 * cb + k;
          const float2 gv = __bfloat1622float2(a[k]);
          jt = fmaf(sw[t * CH + 2 * c], gv.x, fmaf(sw[t * CH + 2 * c + 1], gv.y, jt));
        }
      }
    }
    u[p] = w[p] - 2.f * jt;
  }
}

// n2[b] += sum_p x[b][p]^2 (FP64); grid (blocks per image, B)
__global__ void __launch_bounds__(256) image_norm2(const float* __restrict__ x, int64_t plane, double* n2) {
  __shared__ double red[256];
  const float* xb = x + (int64_t)blockIdx.y * plane;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x)
    s += (double)xb[i] * xb[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x >> 1; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&n2[blockIdx.y], red[0]);
}

// v[b][p] = u[b][p] / sqrt(n2[b]) (a zero image stays zero)
__global__ void __launch_bounds__(256) image_unit(const float* __restrict__ u, const double* __restrict__ n2,
                                                  int64_t plane, int B, float* __restrict__ v) {
  const int64_t total = plane * B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const double n = n2[i / plane];
    v[i] = n > 0.0 ? (float)(u[i] / sqrt(n)) : 0.f;
  }
}

// Cotangent of the soft firm non-expansiveness penalty lam/B sum_b max(||w_b||^2, 1 - eps) with
// w = J_Q v: c[b][p] = -4 lam/B w[b][p] where ||w_b||^2 > 1 - eps, else 0.
__global__ void __launch_bounds__(256) fne_cotangent(const float* __restrict__ w, const double* __restrict__ n2,
                                                     int64_t plane, int B, float scale, double floor_,
                                                     float* __restrict__ c) {
  const int64_t total = plane * B;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    c[i] = n2[i / plane] > floor_ ? -4.f * scale * w[i] : 0.f;
}

// Adam (Kingma & Ba 2015) on the master weights; the gradient is cleared for the next step.
// omb1 = 1 - b1 and omb2 = 1 - b2 come from the host in double precision: formed in FP32 from
// b2 = 0.999f, 1 - b2 would be off by 1.3e-5 relative, and the step m^/sqrt(v^) by half that.
__global__ void adam_step(float* __restrict__ w, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                          int64_t count, float lr, float b1, float b2, float omb1, float omb2, float eps, float c1,
                          float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    g[i] = 0.f;
  }
}

__global__ void zero_f(float* p, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.f;
}

int nblocks(int64_t count, int threads = 256) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (int)std::max<int64_t>(1, std::min<int64_t>((count + threads - 1) / threads, 8L * sms));
}

}  // namespace
}  // namespace pnp

struct pnp_cnn_trainer {
  pnp::Dims d{};
  cudaStream_t stream = nullptr;
  int n_strips = 0, t = 0;
  double lr = 1e-4, b1 = 0.9, b2 = 0.999, eps = 1e-8;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float *w1r = nullptr, *w8r = nullptr, *bias = nullptr;
  __nv_bfloat16 *wf = nullptr, *wb = nullptr;
  __nv_bfloat16* act[8] = {};
  __nv_bfloat16* dp[2] = {};
  float *z = nullptr, *gout = nullptr;
  int4 *facets = nullptr, *strips = nullptr;
  double* loss = nullptr;
  int* status = nullptr;
  float *jv = nullptr, *jw = nullptr, *ju = nullptr;  // Jacobian power iteration images (B x s x s)
  double* jn2 = nullptr;                                // their per-image squared norms [B]
  __nv_bfloat16* tan[8] = {};                           // tangents t_1..t_7 of the penalty's J_N v
  float* junk = nullptr;                                // bias-gradient sink of the tangent network [64]
  alignas(64) unsigned char map_tan[8][256];            // TMA descriptors of tan[1..6]
  alignas(64) unsigned char map_act[8][256];  // TMA descriptors (main, halo) of act[1..7]
  alignas(64) unsigned char map_dp[2][256];   // and of the two gradient canvases
};

using namespace pnp;

namespace {
void trainer_free(pnp_cnn_trainer* T) {
  if (!T) return;
  for (void* p : {(void*)T->w, (void*)T->g, (void*)T->m, (void*)T->v, (void*)T->w1r, (void*)T->w8r, (void*)T->bias,
                  (void*)T->wf, (void*)T->wb, (void*)T->z, (void*)T->gout, (void*)T->facets, (void*)T->strips,
                  (void*)T->loss, (void*)T->status, (void*)T->jv, (void*)T->jw, (void*)T->ju, (void*)T->jn2})
    cudaFree(p);
  for (auto p : T->act) cudaFree(p);
  for (auto p : T->dp) cudaFree(p);
  for (auto p : T->tan) cudaFree(p);
  cudaFree(T->junk);
  delete T;
}

int prep(pnp_cnn_trainer* T) {
  prep_weights<<<nblocks(6 * (int64_t)NWM), 256, 0, T->stream>>>(T->w, T->w1r, T->w8r, T->bias, T->wf, T->wb);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}
}  // namespace

namespace {
// per-image squared norms of x into T->jn2
int image_norms(pnp_cnn_trainer* T, const float* x) {
  const int64_t plane = (int64_t)T->d.s * T->d.s;
  PNP_CUDA(cudaMemsetAsync(T->jn2, 0, T->d.B * sizeof(double), T->stream));
  const int bx = (int)std::min<int64_t>((plane + 255) / 256, 64);
  image_norm2<<<dim3(bx, T->d.B), 256, 0, T->stream>>>(x, plane, T->jn2);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}
}  // namespace

namespace {
// the forward pass at z that fixes the ReLU masks (activations act[1..7])
int primal_forward(pnp_cnn_trainer* T, const float* z) {
  const Dims d = T->d;
  cudaStream_t s = T->stream;
  if (int rc = cnn_first_launch(s, z, d.s, (int64_t)d.s * d.s, T->facets, d.B, d.Hc, d.Wc, T->w1r, T->bias,
                                T->act[1]))
    return rc;
  for (int k = 1; k <= 6; ++k)
    if (int rc = conv64_launch(s, T->map_act[k], T->act[k + 1], T->wf + (size_t)(k - 1) * NWM, T->bias + k * CH,
                               T->strips, T->n_strips, d.Hc, d.Wc, 0, nullptr, T->status))
      return rc;
  return PNP_OK;
}

// Power iteration on J_Q^T J_Q at the current activations from v0 (normalised per image):
// T->jv ends as the last unit iterate; sigma_host (if given) gets ||J_Q v|| of the last step.
int power_iterate(pnp_cnn_trainer* T, const float* v0, int iters, double* sigma_host) {
  const Dims d = T->d;
  const int64_t plane = (int64_t)d.s * d.s, npx = plane * d.B;
  cudaStream_t s = T->stream;
  if (int rc = image_norms(T, v0)) return rc;
  image_unit<<<nblocks(npx), 256, 0, s>>>(v0, T->jn2, plane, d.B, T->jv);
  PNP_CHECK_LAUNCH();
  for (int it = 0; it < iters; ++it) {
    // w = J_Q v: tangents through layers 1..7 (masks [act_k > 0]), then layer 8
    tangent_first<<<nblocks(npx), 256, 0, s>>>(d, T->jv, T->w1r, T->act[1], T->dp[0]);
    PNP_CHECK_LAUNCH();
    int cur = 0;
    for (int k = 1; k <= 6; ++k) {
      if (int rc = conv64_launch(s, T->map_dp[cur], T->dp[1 - cur], T->wf + (size_t)(k - 1) * NWM, nullptr, T->strips,
                                 T->n_strips, d.Hc, d.Wc, 1, T->act[k + 1], T->status))
        return rc;
      cur = 1 - cur;
    }
    tangent_last<<<nblocks(npx), 256, 0, s>>>(d, T->dp[cur], T->w8r, T->jv, T->jw);
    PNP_CHECK_LAUNCH();
    // u = J_Q^T w: the training step's back-propagation with cotangent w
    last_bwd<<<nblocks(npx), 256, 0, s>>>(d, T->act[7], T->w8r, T->jw, T->dp[0]);
    PNP_CHECK_LAUNCH();
    cur = 0;
    for (int k = 6; k >= 1; --k) {
      if (int rc = conv64_launch(s, T->map_dp[cur], T->dp[1 - cur], T->wb + (size_t)(k - 1) * NWM, nullptr, T->strips,
                                 T->n_strips, d.Hc, d.Wc, 1, T->act[k], T->status))
        return rc;
      cur = 1 - cur;
    }
    cotangent_first<<<nblocks(npx), 256, 0, s>>>(d, T->dp[cur], T->w1r, T->jw, T->ju);
    PNP_CHECK_LAUNCH();
    if (sigma_host && it == iters - 1) {  // sigma = ||J_Q v|| for the current unit v
      if (int rc = image_norms(T, T->jw)) return rc;
      PNP_CUDA(cudaMemcpyAsync(sigma_host, T->jn2, d.B * sizeof(double), cudaMemcpyDeviceToHost, s));
      PNP_CUDA(cudaStreamSynchronize(s));
      for (int b = 0; b < d.B; ++b) sigma_host[b] = std::sqrt(sigma_host[b]);
    }
    if (int rc = image_norms(T, T->ju)) return rc;
    image_unit<<<nblocks(npx), 256, 0, s>>>(T->ju, T->jn2, plane, d.B, T->jv);
    PNP_CHECK_LAUNCH();
  }
  return PNP_OK;
}

// Adam on the accumulated gradients, then the BF16 operands are re-packed
int adam_update(pnp_cnn_trainer* T) {
  T->t += 1;
  const float c1 = (float)(1.0 - std::pow(T->b1, T->t)), c2 = (float)(1.0 - std::pow(T->b2, T->t));
  adam_step<<<nblocks(NPARAM), 256, 0, T->stream>>>(T->w, T->g, T->m, T->v, NPARAM, (float)T->lr, (float)T->b1,
                                                    (float)T->b2, (float)(1.0 - T->b1), (float)(1.0 - T->b2),
                                                    (float)T->eps, c1, c2);
  PNP_CHECK_LAUNCH();
  return prep(T);
}
}  // namespace

extern "C" {

int pnp_cnn_trainer_create(pnp_cnn_trainer** out, const float* weights_host, int batch, int size, double lr,
                           void* stream) {
  if (!out || !weights_host || batch < 1 || size < 8 || !(lr > 0)) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  *out = nullptr;
  pnp_cnn_trainer* T = new pnp_cnn_trainer();
  T->stream = reinterpret_cast<cudaStream_t>(stream);
  T->lr = lr;
  T->d = Dims{batch, size, size, (size + 127) / 128 * 128};
  const size_t canvas = (size_t)batch * T->d.Hc * T->d.Wc * CH;
  const int64_t npx = (int64_t)batch * size * size;
  auto al = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  bool ok = al((void**)&T->w, NPARAM * 4) && al((void**)&T->g, NPARAM * 4) && al((void**)&T->m, NPARAM * 4) &&
            al((void**)&T->v, NPARAM * 4) && al((void**)&T->w1r, NW1 * 4) && al((void**)&T->w8r, NW8 * 4) &&
            al((void**)&T->bias, 8 * CH * 4) && al((void**)&T->wf, 6 * (size_t)NWM * 2) &&
            al((void**)&T->wb, 6 * (size_t)NWM * 2) && al((void**)&T->z, npx * 4) && al((void**)&T->gout, npx * 4) &&
            al((void**)&T->facets, batch * sizeof(int4)) && al((void**)&T->loss, sizeof(double)) &&
            al((void**)&T->status, 4 * sizeof(int)) && al((void**)&T->jv, npx * 4) && al((void**)&T->jw, npx * 4) &&
            al((void**)&T->ju, npx * 4) && al((void**)&T->jn2, batch * sizeof(double)) &&
            al((void**)&T->junk, CH * sizeof(float));
  for (int i = 1; ok && i <= 7; ++i) ok = al((void**)&T->act[i], canvas * 2);
  for (int i = 0; ok && i < 2; ++i) ok = al((void**)&T->dp[i], canvas * 2);
  for (int i = 1; ok && i <= 7; ++i) ok = al((void**)&T->tan[i], canvas * 2);
  std::vector<int4> facets(batch, make_int4(0, 0, size, size));
  const std::vector<int> sides(batch, size);
  const std::vector<int4> strips = conv_strips(batch, sides.data(), sides.data());
  T->n_strips = (int)strips.size();
  ok = ok && al((void**)&T->strips, strips.size() * sizeof(int4));
  if (!ok) {
    trainer_free(T);
    return fail(PNP_ERR_OOM, "trainer allocation failed");
  }
  cudaError_t e = cudaMemcpy(T->w, weights_host, NPARAM * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(T->g, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(T->m, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(T->v, 0, NPARAM * 4);
  if (e == cudaSuccess) e = cudaMemset(T->status, 0, 4 * sizeof(int));
  for (int i = 1; e == cudaSuccess && i <= 7; ++i) e = cudaMemset(T->act[i], 0, canvas * 2);
  for (int i = 0; e == cudaSuccess && i < 2; ++i) e = cudaMemset(T->dp[i], 0, canvas * 2);
  for (int i = 1; e == cudaSuccess && i <= 7; ++i) e = cudaMemset(T->tan[i], 0, canvas * 2);
  if (e == cudaSuccess) e = cudaMemcpy(T->facets, facets.data(), batch * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(T->strips, strips.data(), strips.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    trainer_free(T);
    return fail(PNP_ERR_CUDA, std::string("trainer set-up: ") + cudaGetErrorString(e));
  }
  for (int i = 1; i <= 7; ++i)
    if (int rc = canvas_map_create(T->map_act[i], T->act[i], batch, T->d.Hc, T->d.Wc)) {
      trainer_free(T);
      return rc;
    }
  for (int i = 0; i < 2; ++i)
    if (int rc = canvas_map_create(T->map_dp[i], T->dp[i], batch, T->d.Hc, T->d.Wc)) {
      trainer_free(T);
      return rc;
    }
  for (int i = 1; i <= 6; ++i)
    if (int rc = canvas_map_create(T->map_tan[i], T->tan[i], batch, T->d.Hc, T->d.Wc)) {
      trainer_free(T);
      return rc;
    }
  if (int rc = prep(T)) {
    trainer_free(T);
    return rc;
  }
  *out = T;
  return PNP_OK;
}

void pnp_cnn_trainer_destroy(pnp_cnn_trainer* T) {
  if (T) cudaStreamSynchronize(T->stream);
  trainer_free(T);
}

int pnp_cnn_train_step(pnp_cnn_trainer* T, const float* u, const float* noise, double sigma, int update,
                       double* loss_host) {
  if (!T || !u || !noise || !(sigma >= 0)) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  const Dims d = T->d;
  const int64_t npx = (int64_t)d.B * d.s * d.s;
  cudaStream_t s = T->stream;
  // ---------------- forward
  make_z<<<nblocks(npx), 256, 0, s>>>(u, noise, (float)sigma, T->z, npx);
  PNP_CHECK_LAUNCH();
  if (int rc = cnn_first_launch(s, T->z, d.s, (int64_t)d.s * d.s, T->facets, d.B, d.Hc, d.Wc, T->w1r, T->bias,
                                T->act[1]))
    return rc;
  for (int k = 1; k <= 6; ++k)
    if (int rc = conv64_launch(s, T->map_act[k], T->act[k + 1], T->wf + (size_t)(k - 1) * NWM, T->bias + k * CH,
                               T->strips, T->n_strips, d.Hc, d.Wc, 0, nullptr, T->status))
      return rc;
  PNP_CUDA(cudaMemsetAsync(T->loss, 0, sizeof(double), s));
  last_fwd_loss<<<nblocks(npx), 256, 0, s>>>(d, T->act[7], T->w8r, T->bias, T->z, u, T->gout, T->loss);
  PNP_CHECK_LAUNCH();
  // ---------------- backward
  last_bwd<<<nblocks(npx), 256, 0, s>>>(d, T->act[7], T->w8r, T->gout, T->dp[0]);
  PNP_CHECK_LAUNCH();
  const int wgb = (int)((npx + WG_CHUNK - 1) / WG_CHUNK);
  wgrad_onechannel<<<wgb, 576, 0, s>>>(d, 0, T->gout, T->act[7], T->g + OFF_W8, T->g + OFF_B8);
  PNP_CHECK_LAUNCH();
  int cur = 0;
  for (int k = 6; k >= 1; --k) {
    float* gW = T->g + OFF_MID + (k - 1) * MID_STRIDE;
    if (int rc = wgrad64_launch(s, d, T->dp[cur], T->act[k], gW, gW + NWM)) return rc;
    if (int rc = conv64_launch(s, T->map_dp[cur], T->dp[1 - cur], T->wb + (size_t)(k - 1) * NWM, nullptr,
                               T->strips, T->n_strips, d.Hc, d.Wc, 1, T->act[k], T->status))
      return rc;
    cur = 1 - cur;
  }
  wgrad_onechannel<<<wgb, 576, 0, s>>>(d, 1, T->z, T->dp[cur], T->g + OFF_W1, T->g + OFF_B1);
  PNP_CHECK_LAUNCH();
  // ---------------- update
  if (update)
    if (int rc = adam_update(T)) return rc;
  if (loss_host) {
    PNP_CUDA(cudaMemcpyAsync(loss_host, T->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    PNP_CUDA(cudaStreamSynchronize(s));
  }
  return PNP_OK;
}

int pnp_cnn_jacobian_norm(pnp_cnn_trainer* T, const float* z, const float* v0, int iters, double* sigma_host,
                          float* v_out) {
  if (!T || !z || !v0 || iters < 1 || iters > 100000 || !sigma_host) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  const Dims d = T->d;
  const int64_t npx = (int64_t)d.s * d.s * d.B;
  if (int rc = primal_forward(T, z)) return rc;  // fixes the ReLU masks
  if (int rc = power_iterate(T, v0, iters, sigma_host)) return rc;
  if (v_out) PNP_CUDA(cudaMemcpyAsync(v_out, T->jv, npx * sizeof(float), cudaMemcpyDeviceToDevice, T->stream));
  PNP_CUDA(cudaStreamSynchronize(T->stream));
  return PNP_OK;
}

int pnp_cnn_train_step_fne(pnp_cnn_trainer* T, const float* u, const float* noise, double sigma, const float* v0,
                           int iters, double lambda, double eps, int update, double* loss_host,
                           double* penalty_host) {
  if (!T || !u || !noise || !v0 || !(sigma >= 0) || iters < 0 || iters > 100000 || !(lambda >= 0) ||
      !std::isfinite(lambda) || !(eps >= 0) || !(eps <= 1))
    return fail(PNP_ERR_INVALID_ARG, "bad argument");
  const Dims d = T->d;
  const int64_t plane = (int64_t)d.s * d.s, npx = plane * d.B;
  cudaStream_t s = T->stream;
  // the l1 term: forward at z = u + sigma n (activations kept), gradients accumulated, no update
  if (int rc = pnp_cnn_train_step(T, u, noise, sigma, 0, loss_host)) return rc;
  // v: the leading right singular vector of J_Q at z, by power iteration (iters = 0: v0 itself)
  if (iters > 0) {
    if (int rc = power_iterate(T, v0, iters, nullptr)) return rc;
  } else {
    if (int rc = image_norms(T, v0)) return rc;
    image_unit<<<nblocks(npx), 256, 0, s>>>(v0, T->jn2, plane, d.B, T->jv);
    PNP_CHECK_LAUNCH();
  }
  // w = J_Q v with every tangent kept for the weight gradients
  tangent_first<<<nblocks(npx), 256, 0, s>>>(d, T->jv, T->w1r, T->act[1], T->tan[1]);
  PNP_CHECK_LAUNCH();
  for (int k = 1; k <= 6; ++k)
    if (int rc = conv64_launch(s, T->map_tan[k], T->tan[k + 1], T->wf + (size_t)(k - 1) * NWM, nullptr, T->strips,
                               T->n_strips, d.Hc, d.Wc, 1, T->act[k + 1], T->status))
      return rc;
  tangent_last<<<nblocks(npx), 256, 0, s>>>(d, T->tan[7], T->w8r, T->jv, T->jw);
  PNP_CHECK_LAUNCH();
  if (int rc = image_norms(T, T->jw)) return rc;
  fne_cotangent<<<nblocks(npx), 256, 0, s>>>(T->jw, T->jn2, plane, d.B, (float)(lambda / d.B), 1.0 - eps, T->gout);
  PNP_CHECK_LAUNCH();
  // back-propagation of the cotangent through the tangent network (no bias gradients)
  const int wgb = (int)((npx + WG_CHUNK - 1) / WG_CHUNK);
  wgrad_onechannel<<<wgb, 576, 0, s>>>(d, 0, T->gout, T->tan[7], T->g + OFF_W8, T->junk);
  PNP_CHECK_LAUNCH();
  last_bwd<<<nblocks(npx), 256, 0, s>>>(d, T->act[7], T->w8r, T->gout, T->dp[0]);
  PNP_CHECK_LAUNCH();
  int cur = 0;
  for (int k = 6; k >= 1; --k) {
    if (int rc = wgrad64_launch(s, d, T->dp[cur], T->tan[k], T->g + OFF_MID + (k - 1) * MID_STRIDE, T->junk))
      return rc;
    if (int rc = conv64_launch(s, T->map_dp[cur], T->dp[1 - cur], T->wb + (size_t)(k - 1) * NWM, nullptr, T->strips,
                               T->n_strips, d.Hc, d.Wc, 1, T->act[k], T->status))
      return rc;
    cur = 1 - cur;
  }
  wgrad_onechannel<<<wgb, 576, 0, s>>>(d, 1, T->jv, T->dp[cur], T->g + OFF_W1, T->junk);
  PNP_CHECK_LAUNCH();
  if (penalty_host) {
    std::vector<double> n2(d.B);
    PNP_CUDA(cudaMemcpyAsync(n2.data(), T->jn2, d.B * sizeof(double), cudaMemcpyDeviceToHost, s));
    PNP_CUDA(cudaStreamSynchronize(s));
    double P = 0.0;
    for (double q : n2) P += lambda / d.B * std::max(q, 1.0 - eps);
    *penalty_host = P;
  }
  if (update) return adam_update(T);
  return PNP_OK;
}

int pnp_cnn_trainer_read(pnp_cnn_trainer* T, float* weights_host, float* grads_host, int clear_grads) {
  if (!T) return fail(PNP_ERR_INVALID_ARG, "NULL trainer");
  PNP_CUDA(cudaStreamSynchronize(T->stream));
  if (weights_host) PNP_CUDA(cudaMemcpy(weights_host, T->w, NPARAM * 4, cudaMemcpyDeviceToHost));
  if (grads_host) PNP_CUDA(cudaMemcpy(grads_host, T->g, NPARAM * 4, cudaMemcpyDeviceToHost));
  if (clear_grads) {
    zero_f<<<nblocks(NPARAM), 256, 0, T->stream>>>(T->g, NPARAM);
    PNP_CHECK_LAUNCH();
  }
  int st = 0;
  PNP_CUDA(cudaMemcpy(&st, T->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) return fail(PNP_ERR_TIMEOUT, "a bounded wait in the tensor-core convolution gave up");
  return PNP_OK;
}

int pnp_cnn_trainer_apply_update(pnp_cnn_trainer* T) {
  if (!T) return fail(PNP_ERR_INVALID_ARG, "NULL trainer");
  return adam_update(T);
}

int pnp_cnn_trainer_set_lr(pnp_cnn_trainer* T, double lr) {
  if (!T || !(lr > 0)) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  T->lr = lr;
  return PNP_OK;
}

int64_t pnp_cnn_num_params(void) { return NPARAM; }

}  // extern "C"
