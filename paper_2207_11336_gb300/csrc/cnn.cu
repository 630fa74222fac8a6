// Learned residual CNN denoiser (App. C) applied on facets with a halo (App. D).
//
// Network: 8 layers of 3x3 'same' convolutions, 1 -> 64 -> ... -> 64 -> 1,
// bias on every layer, ReLU after all but the last; D(z) = max(0, z - N(z)).
// Weights and hidden activations are BF16, accumulation FP32; the input z, the
// last layer's output and the residual stay FP32.
//
// Facets.  Each facet core is extended by the halo (clipped at the image
// border) and denoised on its own with zero padding at its edges; the cores are
// stitched back.  All facets live in one BF16 activation "canvas" stored in
// planes of 8 channels, [F][Hc][8][Wc][8] (canvas_index), so that one row of an
// 8-channel block is contiguous: the TMA reads whole sectors and the epilogue
// stores whole 512-byte runs per warp.  Cells outside a facet are kept at zero
// so they act as padding.
//
// Kernels per application:
//   cnn_first    z (FP32 image) -> canvas: layer 1 (1 -> 64) on CUDA cores;
//   conv64_rows  canvas -> canvas: one 64 -> 64 layer as an implicit GEMM on the
//                5th-generation tensor cores (tcgen05.mma, FP32 accumulators in
//                tensor memory), one 128-pixel row segment per tile;
//   cnn_last     canvas -> image: layer 8 (64 -> 1) as a tap projection on
//                mma.sync plus a 3 x 3 gather over the facet cores, fused with
//                D(z) = max(0, z - N(z)) and the FP64 stopping-test norms.
//
// conv64_rows layout.  Work is a strip: one 128-pixel column segment (x0 .. x0+127)
// of a run of consecutive output rows of a facet (the strip height is autotuned).
// The strip's input rows (64 channels, pixels x0-1 .. x0+128) stream through a
// ring of shared-memory row slots, staged channel-block-major: [kb][pixel][8 ch]
// with the 130 pixels of a block 16 bytes apart (in a 128-byte aligned 2176-byte
// plane).  That is the canonical no-swizzle K-major operand layout (core matrix
// = 8 pixels x 8 channels, 128 contiguous bytes), and tap (dy, dx) of the 3x3
// stencil is the same matrix with its start address moved by dx pixels (16 B).
// Input row s serves output rows s-2, s-1, s (taps dy = 2, 1, 0): with the
// weights of one (dx, kb) stored as [dy=2 | dy=1 | dy=0] x 64 output channels,
// one MMA of M = 128 pixels, K = 16 channels and N = 192 per (dx, K step) forms
// all three contributions in a fresh accumulator of the row; the epilogue adds
// the three contributions of each output row.  Each staged row is two TMA
// transfers per channel block: the canvas is described as 8-byte elements (2 per
// pixel) so the 128-pixel main box (2 KB) and the 2-pixel halo box (32 B) are
// runs of whole sectors, with zeros outside the canvas.  The rings are pipelined
// with mbarriers; every wait is bounded.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace pnp {
namespace {

constexpr int CH = 64;
constexpr int TILE_PX = 128;                            // output pixels per row segment (the MMA's M)
constexpr int STAGE_PX = TILE_PX + 2;                   // x0-1 .. x0+128
constexpr int KB_BYTES = 136 * 16;                      // one 8-channel block of a staged row: 130 pixels in a
                                                        // 128-byte aligned plane of 136 (2176 bytes)
constexpr int ROW_BYTES = 8 * KB_BYTES;                 // one staged input row, 8 channel blocks (17408)
constexpr int ROW_DATA_BYTES = 8 * STAGE_PX * 16;       // bytes the TMA delivers per staged row (16640)
constexpr int IN_SLOTS = 8;                             // ring of staged input rows
// shared memory of the hidden-layer convolution: the input ring and the layer's weights
constexpr int B_GROUP_BYTES = 3 * CH * 16;              // one (dx, kb) group: [dy=2 | dy=1 | dy=0] x 64 co x 8 ci
constexpr int B_BYTES = 3 * 8 * B_GROUP_BYTES;          // 73728
constexpr int CONV_SMEM = IN_SLOTS * ROW_BYTES + B_BYTES;  // 212992
constexpr int EPI_WARPS = 16;                           // 4 lane quarters x 4 channel quarters
constexpr int MMA_WARP = EPI_WARPS, TMA_WARP = EPI_WARPS + 1;
constexpr int CONV_THREADS = (EPI_WARPS + 2) * 32;
constexpr int FIRST_ROWS = 64;                          // cnn_first: image rows per block
constexpr uint32_t CNN_WAIT_LIMIT = 1u << 26;

struct CnnState {
  int n = 0, F = 0, Hc = 0, Wc = 0, halo = 0;
  std::vector<int> fr0, fr1, fc0, fc1;   // facet cores [r0, r1) x [c0, c1)
  std::vector<int> R0, C0, Hf, Wf;       // extended facets
  int4* d_facets = nullptr;              // per facet: (R0, C0, Hf, Wf)
  int4* d_cores = nullptr;               // per facet: (r0, r1, c0, c1)
  int4* d_strips = nullptr;              // conv64_rows work list (conv_strips)
  int n_strips = 0;
  int4* d_lstrips = nullptr;             // last layer's work list: strips of the facet cores (last_strips)
  int n_lstrips = 0;
  int strip_rows = STRIP_ROWS;           // target output rows per strip of both work lists (autotuned)
  size_t cap_strips = 0, cap_lstrips = 0;  // allocated entries of d_strips, d_lstrips
  uint32_t* d_wfrag = nullptr;           // last layer's weights as mma.sync B fragments [4 k][2 n][32 lanes][2]
  __nv_bfloat16* d_canvas[2] = {nullptr, nullptr};
  float* d_w1 = nullptr;                 // [64][9]  (BF16-rounded values)
  float* d_b = nullptr;                  // [8][64] biases (layer 8 uses entry 0)
  __nv_bfloat16* d_wmid = nullptr;       // 6 x [9][8][64][8] packed for the tensor cores
  float* d_w8 = nullptr;                 // [9][64] (BF16-rounded values)
  int* d_status = nullptr;
  float b8 = 0.f;                        // last layer's bias (host copy)
  CUtensorMap map[2][2];                 // TMA descriptors of the two canvases (main, halo boxes; conv64_rows)
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
  for (uint32_t it = 0; it < CNN_WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\tmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
// 4-D tiled TMA load into shared memory, completion counted on an mbarrier
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(
          su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, BF16 inputs, FP32 accumulate
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on an mbarrier once all previously issued MMAs of this thread completed
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major canonical layout.
//   lbo: byte distance between core matrices adjacent along K
//   sbo: byte distance between 8-row groups along M (or N)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for this architecture
  return d;                // base offset 0, relative LBO mode, no swizzle
}

// Instruction descriptor, kind::f16: FP32 D, BF16 A and B, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TILE_PX >> 4) << 24);
}

struct ConvArgs {
  __nv_bfloat16* out;
  const __nv_bfloat16* w;  // B operand, conv_wpack_index layout
  const float* bias;       // [64] (forward mode)
  const int4* strips;      // conv_strips
  int n_strips, Hc, Wc;
  int* status;
  int mode;                    // 0: forward, out = ReLU(acc + bias); 1: backward data, out = acc * [mask > 0]
  const __nv_bfloat16* mask;   // backward data: activations whose ReLU mask gates the output (same canvas layout)
};

// ------------------------------------------------------------ hidden layers, per-input-row accumulators
// The 64 -> 64 convolution with one fresh accumulator per staged input row: the 12 MMAs of input row s
// (3 dx x 4 K steps of 16 channels, M = 128 pixels, N = 192 = the weights of dy = 2, 1, 0 stacked) write
// D_s = its contributions to output rows s - 2, s - 1, s, in one of two 192-column TMEM buffers, and the
// epilogue sums the three parts of each output row in registers: out(s - 2) = (D_{s-2}[dy 0] +
// D_{s-1}[dy 1]) + D_s[dy 2].  Every MMA has the full N = 192 (no accumulator ring to wrap, no fresh-row
// split), so an input row costs exactly 12 MMAs.  Warp roles: warps 0-15 the epilogue, warp 16 the MMAs
// (one lane), warp 17 the TMA loads (one lane); epilogue warp w reads TMEM lanes 32 (w % 4) .. + 31 and channels 16 (w / 4) .. + 15 of each part.
constexpr int ROW_N = 3 * CH;                 // 192 accumulator columns per staged input row
constexpr int ROW_DBUF = 2;                   // TMEM buffers (2 x 192 of the 512 columns)

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__global__ void __launch_bounds__(CONV_THREADS, 1) conv64_rows(ConvArgs A, const __grid_constant__ CUtensorMap tmain,
                                                               const __grid_constant__ CUtensorMap thalo) {
  extern __shared__ __align__(1024) unsigned char sm[];  // [IN_SLOTS][ROW_BYTES] input ring, then B
  unsigned char* sb = sm + IN_SLOTS * ROW_BYTES;
  __shared__ uint64_t in_full[IN_SLOTS], in_empty[IN_SLOTS], d_full[ROW_DBUF], d_empty[ROW_DBUF];
  __shared__ uint32_t s_tmem;
  __shared__ float s_bias[CH];
  __shared__ volatile int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.w);
    uint4* dst = reinterpret_cast<uint4*>(sb);
    for (int i = threadIdx.x; i < B_BYTES / 16; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x < CH) s_bias[threadIdx.x] = A.bias ? A.bias[threadIdx.x] : 0.f;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < IN_SLOTS; ++i) {
      bar_init(&in_full[i], 1);
      bar_init(&in_empty[i], 1);
    }
    for (int k = 0; k < ROW_DBUF; ++k) {
      bar_init(&d_full[k], 1);
      bar_init(&d_empty[k], EPI_WARPS * 32);  // every epilogue thread reads every buffer
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == MMA_WARP) {
    tmem_alloc(&s_tmem, 512);
    tmem_relinquish();
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const int stride = gridDim.x;

  if (warp == TMA_WARP) {
    // ---------------- TMA producer: input rows ya-1 .. ya+R of each strip, pixels x0-1 .. x0+128; per
    // 8-channel block pixels x0-1 .. x0+126 (2 KB) and x0+127, x0+128 (32 B), each a run of whole sectors
    // of the block's plane (the canvas seen as 8-byte elements, 2 per pixel)
    if (lane == 0) {
      uint32_t L = 0;
      for (int strip = blockIdx.x; strip < A.n_strips && !s_abort; strip += stride) {
        const int4 S = A.strips[strip];
        const int ya = S.z >> 16, R = S.z & 0xFFFF;
        for (int s = 0; s < R + 2; ++s, ++L) {
          const uint32_t slot = L % IN_SLOTS;
          if (L >= IN_SLOTS && !bar_wait(&in_empty[slot], ((L / IN_SLOTS) - 1) & 1)) s_abort = 1;
          if (s_abort) break;
          bar_expect_tx(&in_full[slot], ROW_DATA_BYTES);
          unsigned char* dst = sm + slot * ROW_BYTES;
          const int y = ya - 1 + s;
#pragma unroll 1
          for (int kb = 0; kb < 8; ++kb) {
            tma_load_4d(dst + kb * KB_BYTES, &tmain, 2 * (S.y - 1), kb, y, S.x, &in_full[slot]);
            tma_load_4d(dst + kb * KB_BYTES + TILE_PX * 16, &thalo, 2 * (S.y + TILE_PX - 1), kb, y, S.x, &in_full[slot]);
          }
        }
      }
      for (uint32_t k = (L > IN_SLOTS ? L - IN_SLOTS : 0); k < L; ++k)
        bar_wait(&in_full[k % IN_SLOTS], (k / IN_SLOTS) & 1);
    }
    __syncwarp();
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer: 12 MMAs of N = 192 per staged input row into buffer L % 2
    if (lane == 0) {
      const uint64_t adesc0 = smem_desc(su32(sm), KB_BYTES, 128);
      const uint64_t bdesc0 = smem_desc(su32(sb), B_GROUP_BYTES, 128);
      const uint32_t idesc = idesc_n(ROW_N);
      uint32_t L = 0;
      for (int strip = blockIdx.x; strip < A.n_strips && !s_abort; strip += stride) {
        const int R = A.strips[strip].z & 0xFFFF;
        for (int s = 0; s < R + 2; ++s, ++L) {
          const uint32_t slot = L % IN_SLOTS, buf = L % ROW_DBUF;
          if (!bar_wait(&in_full[slot], (L / IN_SLOTS) & 1)) s_abort = 1;
          if (L >= ROW_DBUF && !bar_wait(&d_empty[buf], ((L / ROW_DBUF) - 1) & 1)) s_abort = 1;
          if (s_abort) break;
          tc_fence_after();
          const uint64_t arow = adesc0 + (uint64_t)((slot * ROW_BYTES) >> 4);
          const uint32_t d = tmem + buf * ROW_N;
#pragma unroll
          for (int dk = 0; dk < 12; ++dk) {
            const int dx = dk >> 2, kk = dk & 3;
            const uint64_t ad = arow + (uint64_t)((2 * kk * KB_BYTES + dx * 16) >> 4);
            const uint64_t bd = bdesc0 + (uint64_t)(((dx * 8 + 2 * kk) * B_GROUP_BYTES) >> 4);
            mma_bf16(d, ad, bd, idesc, dk > 0 ? 1u : 0u);
          }
          mma_commit(&in_empty[slot]);  // the input slot may be refilled
          mma_commit(&d_full[buf]);     // D_s is complete
        }
      }
      // the tensor memory is freed below only after the last MMAs have completed
      if (L > 0) bar_wait(&in_empty[(L - 1) % IN_SLOTS], ((L - 1) / IN_SLOTS) & 1);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: q1 = partial sums of output row s - 1 (its dy = 0 part), q2 = those of
    // row s - 2 (dy = 0 and 1); staged row s completes row s - 2 with its dy = 2 part
    const int lq = warp & 3, cq = warp >> 2;
    const int m = lq * 32 + lane;
    const size_t plane = (size_t)A.Wc * 8;
    uint32_t L = 0;
    bool stop = false;
    for (int strip = blockIdx.x; strip < A.n_strips && !stop; strip += stride) {
      const int4 S = A.strips[strip];
      const int ya = S.z >> 16, R = S.z & 0xFFFF, Hf = S.w >> 16, Wf = S.w & 0xFFFF;
      float q1[16] = {}, q2[16] = {};
      for (int s = 0; s < R + 2; ++s, ++L) {
        const uint32_t buf = L % ROW_DBUF;
        const bool ok = !s_abort && bar_wait(&d_full[buf], (L / ROW_DBUF) & 1);
        if (!ok) s_abort = 1;
        if (!__all_sync(0xffffffffu, ok)) {
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(lq * 32) << 16) + buf * ROW_N + cq * 16;
        uint32_t v2[16];
        tmem_ld16(base, v2);  // dy = 2: output row s - 2 (the other two parts are read after it is stored)
        tmem_wait_ld();
        const int r = s - 2;  // the output row completed by this input row
        if (r >= 0) {
          const int y = ya + r, x = S.y + m;
          if (y < A.Hc && x < A.Wc) {
            const bool live = x < Wf && y < Hf;  // outside the facet the canvas stays zero
            const size_t pix = canvas_index(S.x, y, x, 16 * cq, A.Hc, A.Wc);  // block q at pix + q * plane
            uint4 pk[2];
            uint32_t* pw = reinterpret_cast<uint32_t*>(pk);
            if (A.mode == 0) {
#pragma unroll
              for (int c = 0; c < 16; c += 2) {
                const float a0 = q2[c] + __uint_as_float(v2[c]), a1 = q2[c + 1] + __uint_as_float(v2[c + 1]);
                const float o0 = live ? fmaxf(0.f, a0 + s_bias[16 * cq + c]) : 0.f;
                const float o1 = live ? fmaxf(0.f, a1 + s_bias[16 * cq + c + 1]) : 0.f;
                __nv_bfloat162 h = __floats2bfloat162_rn(o0, o1);
                pw[c / 2] = *reinterpret_cast<uint32_t*>(&h);
              }
            } else {
              uint4 mk[2];
#pragma unroll
              for (int q = 0; q < 2; ++q) mk[q] = *reinterpret_cast<const uint4*>(A.mask + pix + q * plane);
              const __nv_bfloat16* mh = reinterpret_cast<const __nv_bfloat16*>(mk);
#pragma unroll
              for (int c = 0; c < 16; c += 2) {
                const float a0 = q2[c] + __uint_as_float(v2[c]), a1 = q2[c + 1] + __uint_as_float(v2[c + 1]);
                const float o0 = (live && __bfloat162float(mh[c]) > 0.f) ? a0 : 0.f;
                const float o1 = (live && __bfloat162float(mh[c + 1]) > 0.f) ? a1 : 0.f;
                __nv_bfloat162 h = __floats2bfloat162_rn(o0, o1);
                pw[c / 2] = *reinterpret_cast<uint32_t*>(&h);
              }
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) *reinterpret_cast<uint4*>(A.out + pix + q * plane) = pk[q];
          }
        }
        uint32_t v1[16], v0[16];
        tmem_ld16(base + CH, v1);      // dy = 1: output row s - 1
        tmem_ld16(base + 2 * CH, v0);  // dy = 0: output row s
        tmem_wait_ld();
        tc_fence_before();
        bar_arrive(&d_empty[buf]);  // this thread's parts of D_s are in registers
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          q2[c] = q1[c] + __uint_as_float(v1[c]);  // row s - 1: dy = 0 + dy = 1 (not used at s = 0)
          q1[c] = __uint_as_float(v0[c]);          // row s: dy = 0
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && s_abort) atomicOr(A.status, 2);
}

// ------------------------------------------------------------ layer 1 (1 -> 64)
struct FirstArgs {
  const float* z;
  int n;
  int64_t zplane;  // elements between the z planes of consecutive facets (0: one shared image)
  const int4* facets;
  int F, Hc, Wc;
  const float* w1;  // [64][9]
  const float* b1;  // [64]
  __nv_bfloat16* out;
};

// Layer 1 (1 -> 64).  A block covers a 32-pixel column segment of FIRST_ROWS rows of a facet;
// warp w computes the 8 channels of channel block w for the segment's 32 pixels, row after row,
// with that block's 72 weights and 8 biases in registers (each weight is loaded once per block,
// not once per pixel).  The block stages the (FIRST_ROWS + 2) x 34 input window of z (zero
// outside the extended facet: 'same' padding) in shared memory; a warp's store of one row is the
// 32 pixels' 16-byte channel-block vectors, one contiguous 512-byte run of the block's plane.
constexpr int FIRST_PX = 32;

// d = a * b + c on two FP32 lanes at once (packed FMA, one instruction for a channel pair)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*reinterpret_cast<unsigned long long*>(&a)), "l"(*reinterpret_cast<unsigned long long*>(&b)),
        "l"(*reinterpret_cast<unsigned long long*>(&c)));
  return *reinterpret_cast<float2*>(&d);
}

__global__ void __launch_bounds__(256) cnn_first(FirstArgs A) {
  __shared__ float zt[FIRST_ROWS + 2][FIRST_PX + 2];
  const int f = blockIdx.z, ya = blockIdx.y * FIRST_ROWS, x0 = blockIdx.x * FIRST_PX;
  const int4 fc = A.facets[f];  // R0, C0, Hf, Wf
  // canvas cells outside the facet are zero from the canvas's allocation and every layer writes zeros
  // there, so only the facet's own cells are written here
  if (ya >= fc.z || x0 >= fc.w) return;
  const float* zf = A.z + (size_t)f * A.zplane;
  for (int i = threadIdx.x; i < (FIRST_ROWS + 2) * (FIRST_PX + 2); i += blockDim.x) {
    const int r = i / (FIRST_PX + 2), c = i % (FIRST_PX + 2);
    const int yy = ya + r - 1, xx = x0 + c - 1;
    zt[r][c] = (yy >= 0 && yy < fc.z && xx >= 0 && xx < fc.w) ? zf[(size_t)(fc.x + yy) * A.n + fc.y + xx] : 0.f;
  }
  const int cb = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 w[4][9], b[4];  // channel pairs (2 q, 2 q + 1) of the block
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    b[q] = make_float2(A.b1[cb * 8 + 2 * q], A.b1[cb * 8 + 2 * q + 1]);
#pragma unroll
    for (int t = 0; t < 9; ++t) w[q][t] = make_float2(A.w1[(cb * 8 + 2 * q) * 9 + t], A.w1[(cb * 8 + 2 * q + 1) * 9 + t]);
  }
  __syncthreads();
  const int x = x0 + lane;
  if (x >= fc.w) return;
  const int yb = min(ya + FIRST_ROWS, fc.z);
  for (int y = ya; y < yb; ++y) {
    const int r = y - ya;
    float zin[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) zin[t] = zt[r + t / 3][lane + t % 3];
    uint32_t pk[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float2 a = b[q];
#pragma unroll
      for (int t = 0; t < 9; ++t) a = ffma2(w[q][t], make_float2(zin[t], zin[t]), a);
      __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f));
      pk[q] = *reinterpret_cast<uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(A.out + canvas_index(f, y, x, cb * 8, A.Hc, A.Wc)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// ------------------------------------------------------------ last layer (64 -> 1)
// The last layer has one output channel, so as a 3 x 3 convolution it is 1/64 of a hidden layer's
// work; run as the tensor-core convolution above it pays a hidden layer's MMA-issue cost (one
// 4 KB A tile per (dx, K step)).  Here it is split instead into a per-pixel projection onto the
// nine taps, P[y][x][t] = sum_c W8[c][t] h[y][x][c] (a GEMM with M = pixels, K = 64 channels,
// N = 9 taps padded to 16, on the tensor cores with mma.sync: each activation is read once), and
// a 3 x 3 gather N[y][x] = b8 + sum_t P[y + dy - 1][x + dx - 1][t] (t = 3 dy + dx) from a ring of
// three projected rows in shared memory, fused with D(z) = max(0, z - N(z)) and the FP64
// stopping-test sums.  A CTA walks one strip of the last layer's work list (128 core columns x
// about 32 core rows of a facet) row by row; P covers the 144 pixels x0 - 1 .. x0 + 142 of each
// activation row (9 M tiles of 16), so the gather never leaves the CTA.  Each activation row is
// copied into shared memory with cp.async (16-byte pieces, whole runs of each channel block's
// plane, zero-filled outside the facet) one row ahead of its projection, double buffered, and the
// A fragments are read from there with ldmatrix.
constexpr int LAST_PX = 144;   // projected pixels per row: x0 - 1 .. x0 + 142
constexpr int LAST_TS = 9;     // taps kept per pixel in shared memory (row stride: conflict-free gathers)
constexpr int LAST_THREADS = 128;
constexpr int LAST_ROW_BYTES = 8 * LAST_PX * 16;                                  // one staged row: [block][px][8 ch]
constexpr int LAST_SMEM = 2 * LAST_ROW_BYTES + 3 * LAST_PX * LAST_TS * 4;        // two staged rows + the P ring

struct LastArgs {
  const __nv_bfloat16* canvas;  // layer-7 activations (canvas layout)
  const int4* strips;           // last_strips: (f, x0, ya << 16 | rows, Hf << 16 | Wf), facet-local
  int n_strips, Hc, Wc, n;
  const int4* facets;           // (R0, C0, Hf, Wf)
  const int4* cores;            // (r0, r1, c0, c1) in image coordinates
  const uint32_t* wfrag;        // [4 k steps][2 n tiles][32 lanes][2] packed BF16 pairs
  float b8;
  const float* z;
  const float* x_prev;
  float* img;
  double* acc;
  int pos;
};

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(su32(p)));
}
// 16-byte global -> shared copy; nbytes = 0 fills the 16 bytes with zeros (src is not read)
__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, int nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// activation row r of facet f, pixels x0 - 1 .. x0 + 142, into a staged row [block][px][8 ch] (zero outside
// rows [0, Hf) and columns [0, Wf): the 'same' padding at the facet's edges)
__device__ __forceinline__ void last_stage_row(unsigned char* dst, const LastArgs& A, int f, int r, int x0, int Hf,
                                               int Wf) {
  const bool row_ok = r >= 0 && r < Hf;
  for (int c = threadIdx.x; c < 8 * LAST_PX; c += LAST_THREADS) {
    const int b = c / LAST_PX, p = c - b * LAST_PX, x = x0 - 1 + p;
    const bool in = row_ok && x >= 0 && x < Wf;
    const __nv_bfloat16* src = in ? A.canvas + canvas_index(f, r, x, 8 * b, A.Hc, A.Wc) : A.canvas;
    cp_async16_zfill(dst + (size_t)c * 16, src, in ? 16 : 0);
  }
}

__global__ void __launch_bounds__(LAST_THREADS) cnn_last(LastArgs A) {
  extern __shared__ __align__(128) unsigned char lsm[];  // [2][LAST_ROW_BYTES] staged rows, then sP
  float(*sP)[LAST_PX * LAST_TS] = reinterpret_cast<float(*)[LAST_PX * LAST_TS]>(lsm + 2 * LAST_ROW_BYTES);
  __shared__ double red[2][LAST_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  uint32_t bw[4][2][2];  // this lane's B fragments, the whole kernel
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const uint2 v = reinterpret_cast<const uint2*>(A.wfrag)[(ks * 2 + nt) * 32 + lane];
      bw[ks][nt][0] = v.x;
      bw[ks][nt][1] = v.y;
    }
  // ldmatrix row addresses: lane l points at pixel (l % 8) + 8 ((l / 8) % 2) of the tile in channel block
  // 2 ks + l / 16, so the four matrices are the m16n8k16 A fragments a0..a3
  const int lrow = (lane & 7) + 8 * ((lane >> 3) & 1), lblk = lane >> 4;
  double s0 = 0.0, s1 = 0.0;
  for (int si = blockIdx.x; si < A.n_strips; si += gridDim.x) {
    const int4 S = A.strips[si];
    const int f = S.x, x0 = S.y, ya = S.z >> 16, R = S.z & 0xFFFF, Hf = S.w >> 16, Wf = S.w & 0xFFFF;
    const int4 fc = A.facets[f], core = A.cores[f];
    last_stage_row(lsm, A, f, ya - 1, x0, Hf, Wf);
    cp_async_commit_group();
    for (int i = 0; i < R + 2; ++i) {
      const int r = ya - 1 + i;
      if (i + 1 < R + 2) {  // the next row's copies fly while this row is projected
        last_stage_row(lsm + ((i + 1) & 1) * LAST_ROW_BYTES, A, f, r + 1, x0, Hf, Wf);
        cp_async_commit_group();
        cp_async_wait_group<1>();
      } else {
        cp_async_wait_group<0>();
      }
      __syncthreads();  // row r staged by every thread; the gather of the previous row is done with its slot
      // ---- project activation row r onto the taps: warp w takes M tiles w, w + 4, w + 8
      const unsigned char* st = lsm + (i & 1) * LAST_ROW_BYTES;
      float* P = sP[(r - ya + 1) % 3];
#pragma unroll
      for (int ti = 0; ti < 3; ++ti) {
        const int mt = warp + ti * (LAST_THREADS / 32);
        if (mt >= LAST_PX / 16) break;  // warp-uniform
        float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          uint32_t a[4];
          ldmatrix_x4(a, st + ((size_t)(2 * ks + lblk) * LAST_PX + mt * 16 + lrow) * 16);
          mma_bf16_16816(d0, a, bw[ks][0][0], bw[ks][0][1]);
          mma_bf16_16816(d1, a, bw[ks][1][0], bw[ks][1][1]);
        }
        // D fragment: (row g, cols 2 t4, 2 t4 + 1) and (row g + 8, same cols); taps 0..7 in tile 0, 8 in tile 1
        const int pl = mt * 16 + g, ph = pl + 8;
        P[pl * LAST_TS + 2 * t4] = d0[0];
        P[pl * LAST_TS + 2 * t4 + 1] = d0[1];
        P[ph * LAST_TS + 2 * t4] = d0[2];
        P[ph * LAST_TS + 2 * t4 + 1] = d0[3];
        if (t4 == 0) {
          P[pl * LAST_TS + 8] = d1[0];
          P[ph * LAST_TS + 8] = d1[2];
        }
      }
      __syncthreads();
      // ---- output row r - 1: its three projected rows are in the ring
      const int yo = r - 1;
      if (yo >= ya) {
        const float* Pm = sP[(yo - ya) % 3];      // row yo - 1
        const float* P0 = sP[(yo - ya + 1) % 3];  // row yo
        const float* Pp = sP[(yo - ya + 2) % 3];  // row yo + 1
        float nv = A.b8;
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const int q = (tid + dx) * LAST_TS;
          nv += Pm[q + dx] + P0[q + 3 + dx] + Pp[q + 6 + dx];
        }
        const int iy = fc.x + yo, ix = fc.y + x0 + tid;
        if (iy >= core.x && iy < core.y && ix >= core.z && ix < core.w) {
          const size_t pix = (size_t)iy * A.n + ix;
          const float zv = A.z[pix];
          const float res = zv - nv;
          const float o = A.pos ? fmaxf(0.f, res) : res;
          A.img[pix] = o;
          s1 += (double)o * o;
          // fmaxf(0, NaN) is 0, so positivity would hide a non-finite input: poison the norms
          if (!isfinite(zv)) s1 = __longlong_as_double(0x7ff8000000000000LL);
          if (A.x_prev) {
            const double dd = (double)o - A.x_prev[pix];
            s0 += dd * dd;
          }
        }
      }
      // the next iteration's __syncthreads orders this gather before the ring slot of row r - 2 (and the
      // staged row just projected) are overwritten
    }
    __syncthreads();  // the next strip's first copies go to buffer 0 and the ring restarts
  }
  if (A.acc) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
      red[0][warp] = s0;
      red[1][warp] = s1;
    }
    __syncthreads();
    if (tid == 0) {
      double a0 = 0.0, a1 = 0.0;
      for (int w = 0; w < LAST_THREADS / 32; ++w) {
        a0 += red[0][w];
        a1 += red[1][w];
      }
      atomicAdd(&A.acc[0], a0);
      atomicAdd(&A.acc[1], a1);
    }
  }
}

// ------------------------------------------------------------ host helpers
uint16_t to_bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(r >> 16);
}
float bf16_round(float f) {
  const uint32_t u = (uint32_t)to_bf16_bits(f) << 16;
  float o;
  std::memcpy(&o, &u, 4);
  return o;
}

// The two TMA descriptors of a canvas for conv64_rows's row loads (main and halo boxes of one
// channel block's plane row, the canvas seen as 8-byte elements).
int make_canvas_maps(CUtensorMap* maps, const __nv_bfloat16* canvas, int F, int Hc, int Wc) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    PNP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return fail(PNP_ERR_UNSUPPORTED, "cuTensorMapEncodeTiled unavailable");
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // the canvas as 8-byte elements: (2 Wc per 8-channel plane row, 8 channel blocks, Hc rows, F facets)
  const cuuint64_t dims[4] = {2 * (cuuint64_t)Wc, 8, (cuuint64_t)Hc, (cuuint64_t)F};
  const cuuint64_t strides[3] = {(cuuint64_t)Wc * 16, (cuuint64_t)Wc * CH * 2, (cuuint64_t)Hc * Wc * CH * 2};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t box_main[4] = {2 * TILE_PX, 1, 1, 1}, box_halo[4] = {2 * (STAGE_PX - TILE_PX), 1, 1, 1};
  const cuuint32_t* boxes[2] = {box_main, box_halo};
  for (int i = 0; i < 2; ++i) {
    const CUresult r = enc(&maps[i], CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, const_cast<__nv_bfloat16*>(canvas), dims,
                           strides, boxes[i], estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
      return fail(PNP_ERR_UNSUPPORTED, "tensor map encoding failed (" + std::to_string((int)r) + ")");
  }
  return PNP_OK;
}

int sms_of_device() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

}  // namespace

// The two convolution work lists for strips of about `rows` output rows: the hidden layers' strips of
// the extended facets, and the last layer's strips of the facet cores.  Device arrays grow as needed.
static int build_strips(CnnState* S, int rows) {
  const std::vector<int4> strips = conv_strips(S->F, S->Hf.data(), S->Wf.data(), rows);
  std::vector<int4> lstrips;
  for (int f = 0; f < S->F; ++f) {
    const int cr0 = S->fr0[f] - S->R0[f], cr1 = S->fr1[f] - S->R0[f];
    const int cc0 = S->fc0[f] - S->C0[f], cc1 = S->fc1[f] - S->C0[f];
    const int k = std::max(1, (cr1 - cr0 + rows - 1) / rows);
    for (int x0 = cc0; x0 < cc1; x0 += TILE_PX)
      for (int i = 0; i < k; ++i) {
        const int ya = cr0 + (int)((int64_t)(cr1 - cr0) * i / k), yb = cr0 + (int)((int64_t)(cr1 - cr0) * (i + 1) / k);
        if (yb > ya) lstrips.push_back(make_int4(f, x0, (ya << 16) | (yb - ya), (S->Hf[f] << 16) | S->Wf[f]));
      }
  }
  auto fit = [](int4** p, size_t* cap, size_t need) -> int {
    need = std::max<size_t>(1, need);
    if (*p && *cap >= need) return PNP_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(reinterpret_cast<void**>(p), need * sizeof(int4)) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail(PNP_ERR_OOM, "CNN work list allocation failed");
    }
    *cap = need;
    return PNP_OK;
  };
  if (int rc = fit(&S->d_strips, &S->cap_strips, strips.size())) return rc;
  if (int rc = fit(&S->d_lstrips, &S->cap_lstrips, lstrips.size())) return rc;
  if (!strips.empty())
    PNP_CUDA(cudaMemcpy(S->d_strips, strips.data(), strips.size() * sizeof(int4), cudaMemcpyHostToDevice));
  if (!lstrips.empty())
    PNP_CUDA(cudaMemcpy(S->d_lstrips, lstrips.data(), lstrips.size() * sizeof(int4), cudaMemcpyHostToDevice));
  S->n_strips = (int)strips.size();
  S->n_lstrips = (int)lstrips.size();
  S->strip_rows = rows;
  return PNP_OK;
}

int cnn_create(pnp_den* d, const float* W, const int32_t* fr, int nfr, const int32_t* fc, int nfc, int halo,
               int n) {
  CnnState* S = new CnnState();
  d->impl = S;
  S->n = n;
  S->halo = halo;
  std::vector<int> rows = fr && nfr > 0 ? std::vector<int>(fr, fr + nfr) : std::vector<int>{n};
  std::vector<int> cols = fc && nfc > 0 ? std::vector<int>(fc, fc + nfc) : std::vector<int>{n};
  int sr = 0, sc = 0;
  for (int v : rows) {
    if (v <= 0) return fail(PNP_ERR_INVALID_ARG, "facet sizes must be positive");
    sr += v;
  }
  for (int v : cols) {
    if (v <= 0) return fail(PNP_ERR_INVALID_ARG, "facet sizes must be positive");
    sc += v;
  }
  if (sr != n || sc != n) return fail(PNP_ERR_INVALID_ARG, "facet sizes must sum to n along each axis");
  int r = 0;
  for (int a : rows) {
    int c = 0;
    for (int b : cols) {
      S->fr0.push_back(r);
      S->fr1.push_back(r + a);
      S->fc0.push_back(c);
      S->fc1.push_back(c + b);
      const int R0 = std::max(0, r - halo), R1 = std::min(n, r + a + halo);
      const int C0 = std::max(0, c - halo), C1 = std::min(n, c + b + halo);
      S->R0.push_back(R0);
      S->C0.push_back(C0);
      S->Hf.push_back(R1 - R0);
      S->Wf.push_back(C1 - C0);
      c += b;
    }
    r += a;
  }
  S->F = (int)S->R0.size();
  S->Hc = *std::max_element(S->Hf.begin(), S->Hf.end());
  const int wmax = *std::max_element(S->Wf.begin(), S->Wf.end());
  S->Wc = (wmax + TILE_PX - 1) / TILE_PX * TILE_PX;

  std::vector<int4> facets(S->F), cores(S->F);
  for (int f = 0; f < S->F; ++f) {
    facets[f] = make_int4(S->R0[f], S->C0[f], S->Hf[f], S->Wf[f]);
    cores[f] = make_int4(S->fr0[f], S->fr1[f], S->fc0[f], S->fc1[f]);
  }
  // weights: layer shapes 64x1, 6 x 64x64, 1x64, each W[co][ci][3][3] then b[co]
  std::vector<float> w1(CH * 9), w8(9 * CH), bias(8 * CH, 0.f);
  std::vector<uint16_t> wmid((size_t)6 * 9 * CH * CH);
  size_t off = 0;
  for (int co = 0; co < CH; ++co)
    for (int t = 0; t < 9; ++t) w1[co * 9 + t] = bf16_round(W[off + co * 9 + t]);
  off += CH * 9;
  for (int co = 0; co < CH; ++co) bias[co] = W[off + co];
  off += CH;
  for (int l = 0; l < 6; ++l) {
    for (int co = 0; co < CH; ++co)
      for (int ci = 0; ci < CH; ++ci)
        for (int t = 0; t < 9; ++t) {
          wmid[(size_t)l * 9 * CH * CH + conv_wpack_index(t / 3, t % 3, ci, co)] =
              to_bf16_bits(W[off + ((size_t)co * CH + ci) * 9 + t]);
        }
    off += (size_t)CH * CH * 9;
    for (int co = 0; co < CH; ++co) bias[(l + 1) * CH + co] = W[off + co];
    off += CH;
  }
  for (int ci = 0; ci < CH; ++ci)
    for (int t = 0; t < 9; ++t) w8[t * CH + ci] = bf16_round(W[off + ci * 9 + t]);
  // mma.sync B fragments of the tap projection: element (k, n) of K step ks / N tile nt is
  // W8[c = 16 ks + k][tap = 8 nt + n] (zero for taps >= 9); lane l holds k = 2 (l % 4) (+1) in its
  // first register and k + 8 (+9) in its second, n = l / 4, the lower k in the low half
  std::vector<uint32_t> wfrag(4 * 2 * 32 * 2, 0u);
  auto w8bits = [&](int c, int tap) -> uint32_t {
    return tap < 9 ? (uint32_t)to_bf16_bits(W[off + c * 9 + tap]) : 0u;
  };
  for (int ks = 0; ks < 4; ++ks)
    for (int nt = 0; nt < 2; ++nt)
      for (int l = 0; l < 32; ++l) {
        const int tap = 8 * nt + l / 4, k = 16 * ks + 2 * (l % 4);
        uint32_t* o = &wfrag[((ks * 2 + nt) * 32 + l) * 2];
        o[0] = w8bits(k, tap) | (w8bits(k + 1, tap) << 16);
        o[1] = w8bits(k + 8, tap) | (w8bits(k + 9, tap) << 16);
      }
  off += CH * 9;
  bias[7 * CH] = W[off];
  S->b8 = W[off];

  const size_t canvas = (size_t)S->F * S->Hc * S->Wc * CH;
  auto al = [&](void** p, size_t bytes) -> int {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(PNP_ERR_OOM, "CNN buffer allocation failed (" + std::to_string(bytes) + " bytes)");
    }
    return PNP_OK;
  };
  for (int i = 0; i < 2; ++i) {
    if (int rc = al((void**)&S->d_canvas[i], canvas * 2)) return rc;
    PNP_CUDA(cudaMemset(S->d_canvas[i], 0, canvas * 2));
  }
  if (int rc = al((void**)&S->d_facets, S->F * sizeof(int4))) return rc;
  if (int rc = al((void**)&S->d_cores, S->F * sizeof(int4))) return rc;
  if (int rc = al((void**)&S->d_wfrag, wfrag.size() * 4)) return rc;
  if (int rc = al((void**)&S->d_w1, w1.size() * 4)) return rc;
  if (int rc = al((void**)&S->d_w8, w8.size() * 4)) return rc;
  if (int rc = al((void**)&S->d_b, bias.size() * 4)) return rc;
  if (int rc = al((void**)&S->d_wmid, wmid.size() * 2)) return rc;
  if (int rc = al((void**)&S->d_status, 4 * sizeof(int))) return rc;
  PNP_CUDA(cudaMemcpy(S->d_facets, facets.data(), S->F * sizeof(int4), cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemcpy(S->d_cores, cores.data(), S->F * sizeof(int4), cudaMemcpyHostToDevice));
  if (int rc = build_strips(S, S->strip_rows)) return rc;
  PNP_CUDA(cudaMemcpy(S->d_wfrag, wfrag.data(), wfrag.size() * 4, cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemcpy(S->d_w1, w1.data(), w1.size() * 4, cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemcpy(S->d_w8, w8.data(), w8.size() * 4, cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemcpy(S->d_b, bias.data(), bias.size() * 4, cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemcpy(S->d_wmid, wmid.data(), wmid.size() * 2, cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemset(S->d_status, 0, 4 * sizeof(int)));
  for (int i = 0; i < 2; ++i) {
    if (int rc = make_canvas_maps(S->map[i], S->d_canvas[i], S->F, S->Hc, S->Wc)) return rc;
  }
  return PNP_OK;
}

void cnn_destroy(pnp_den* d) {
  CnnState* S = static_cast<CnnState*>(d->impl);
  if (!S) return;
  for (auto p : S->d_canvas) cudaFree(p);
  cudaFree(S->d_facets);
  cudaFree(S->d_cores);
  cudaFree(S->d_strips);
  cudaFree(S->d_lstrips);
  cudaFree(S->d_wfrag);
  cudaFree(S->d_w1);
  cudaFree(S->d_w8);
  cudaFree(S->d_b);
  cudaFree(S->d_wmid);
  cudaFree(S->d_status);
  delete S;
  d->impl = nullptr;
}

int cnn_denoise(pnp_den* d, cudaStream_t s, const float* z, float* out, int n, double* acc, const float* x_prev,
                bool positivity) {
  CnnState* S = static_cast<CnnState*>(d->impl);
  if (!S) return fail(PNP_ERR_INVALID_ARG, "CNN denoiser not initialised");
  if (n != S->n) return fail(PNP_ERR_INVALID_ARG, "image side differs from the one the CNN denoiser was built for");
  const int sms = sms_of_device();
  {
    FirstArgs F{z, n, 0, S->d_facets, S->F, S->Hc, S->Wc, S->d_w1, S->d_b, S->d_canvas[0]};
    cnn_first<<<dim3(S->Wc / FIRST_PX, (S->Hc + FIRST_ROWS - 1) / FIRST_ROWS, S->F), 256, 0, s>>>(F);
    PNP_CHECK_LAUNCH();
  }
  static bool attr = false;
  if (!attr) {
    PNP_CUDA(cudaFuncSetAttribute(conv64_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM));
    PNP_CUDA(cudaFuncSetAttribute(cnn_last, cudaFuncAttributeMaxDynamicSharedMemorySize, LAST_SMEM));
    attr = true;
  }
  int cur = 0;
  for (int l = 0; l < 6; ++l) {
    ConvArgs C{S->d_canvas[1 - cur], S->d_wmid + (size_t)l * 9 * CH * CH, S->d_b + (l + 1) * CH, S->d_strips,
               S->n_strips, S->Hc, S->Wc, S->d_status, 0, nullptr};
    const int grid = std::max(1, std::min(S->n_strips, sms));
    conv64_rows<<<grid, CONV_THREADS, CONV_SMEM, s>>>(C, S->map[cur][0], S->map[cur][1]);
    PNP_CHECK_LAUNCH();
    cur = 1 - cur;
  }
  {
    // layer 8 as a tap projection + 3 x 3 gather, fused with D(z) = max(0, z - N(z)) and the norms
    LastArgs L{S->d_canvas[cur], S->d_lstrips, S->n_lstrips, S->Hc, S->Wc, n, S->d_facets, S->d_cores,
               S->d_wfrag, S->b8, z, x_prev, out, acc, positivity ? 1 : 0};
    cnn_last<<<std::max(1, S->n_lstrips), LAST_THREADS, LAST_SMEM, s>>>(L);
    PNP_CHECK_LAUNCH();
  }
  return PNP_OK;
}

int conv64_launch(cudaStream_t s, const void* in_map, __nv_bfloat16* out, const __nv_bfloat16* w_packed,
                  const float* bias, const int4* strips, int n_strips, int Hc, int Wc, int mode,
                  const __nv_bfloat16* mask, int* status) {
  static bool attr = false;
  if (!attr) {
    PNP_CUDA(cudaFuncSetAttribute(conv64_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, CONV_SMEM));
    attr = true;
  }
  ConvArgs C{out, w_packed, bias, strips, n_strips, Hc, Wc, status, mode, mask};
  const int grid = std::max(1, std::min(n_strips, sms_of_device()));
  const CUtensorMap* maps = static_cast<const CUtensorMap*>(in_map);
  conv64_rows<<<grid, CONV_THREADS, CONV_SMEM, s>>>(C, maps[0], maps[1]);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

std::vector<int4> conv_strips(int F, const int* Hf, const int* Wf, int rows) {
  std::vector<int4> out;
  for (int f = 0; f < F; ++f) {
    const int k = std::max(1, (Hf[f] + rows - 1) / rows);  // strips per column segment
    for (int x0 = 0; x0 < Wf[f]; x0 += TILE_PX)
      for (int i = 0; i < k; ++i) {
        const int ya = (int)((int64_t)Hf[f] * i / k), yb = (int)((int64_t)Hf[f] * (i + 1) / k);
        if (yb > ya) out.push_back(make_int4(f, x0, (ya << 16) | (yb - ya), (Hf[f] << 16) | Wf[f]));
      }
  }
  return out;
}

int cnn_first_launch(cudaStream_t s, const float* z, int n, int64_t zplane, const int4* facets, int F, int Hc,
                     int Wc, const float* w1, const float* b1, __nv_bfloat16* out) {
  FirstArgs A{z, n, zplane, facets, F, Hc, Wc, w1, b1, out};
  cnn_first<<<dim3(Wc / FIRST_PX, (Hc + FIRST_ROWS - 1) / FIRST_ROWS, F), 256, 0, s>>>(A);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int canvas_map_create(void* map_out, const __nv_bfloat16* canvas, int F, int Hc, int Wc) {
  return make_canvas_maps(static_cast<CUtensorMap*>(map_out), canvas, F, Hc, Wc);
}

int cnn_set_strip_rows(pnp_den* d, int rows) {
  CnnState* S = static_cast<CnnState*>(d->impl);
  if (!S) return fail(PNP_ERR_INVALID_ARG, "CNN denoiser not initialised");
  if (rows < 4 || rows > 1024) return fail(PNP_ERR_INVALID_ARG, "strip rows must lie in [4, 1024]");
  PNP_CUDA(cudaDeviceSynchronize());  // launches in flight (on any stream) read the current lists
  return build_strips(S, rows);
}

int cnn_strip_rows(pnp_den* d) {
  const CnnState* S = static_cast<const CnnState*>(d->impl);
  return S ? S->strip_rows : 0;
}

int cnn_status(pnp_den* d, int* flags) {
  CnnState* S = static_cast<CnnState*>(d->impl);
  if (!S) return fail(PNP_ERR_INVALID_ARG, "CNN denoiser not initialised");
  PNP_CUDA(cudaMemcpy(flags, S->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return PNP_OK;
}

}  // namespace pnp
