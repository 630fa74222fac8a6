// De-gridding y = G X (Eq. 1) and gridding G^H r (App. A), separately or fused
// into one pass over G that forms the residual r = G X - y and grids it.
//
// G is CSR with rows sorted by the grid tile holding their first tap (and by
// data block within a tile).  The host cuts the sorted rows into row-aligned
// chunks of at most CHUNK_TAPS taps and groups consecutive chunks of one tile
// into work units.  Each persistent CTA walks its units (round robin) and
// streams their chunks through a ring of NSTAGE shared-memory stages with TMA
// bulk copies (cp.async.bulk, completion counted on one mbarrier per stage):
// the chunk's complex weights, int32 columns, int64 row offsets and (for the
// gridding modes) its visibilities.  One thread issues the copies NSTAGE-1
// chunks ahead -- across unit boundaries -- so HBM latency is hidden by copies
// in flight rather than by resident warps.  Per unit the CTA
//   1. stages the tile plus a (Jmax-1)-cell halo of the input grid X in shared
//      memory (coalesced along k0, wrapped mod K);
//   2. runs warp-per-row SpMV over each chunk from shared memory: lane-strided
//      taps, gathers from the staged grid, warp-shuffle reduction;
//   3. scatters conj(G_mk) r_m into a shared-memory copy of the same region
//      (shared-memory float atomics);
//   4. adds the non-zero cells of that region to the output grid with vector
//      float2 global atomics.
// Grid layout: grid[k1*K + k0]; column index of a tap = k1*K + k0.
#include "common.cuh"

namespace pnp {
namespace {

constexpr uint32_t WAIT_LIMIT = 1u << 26;  // bounded mbarrier waits (seconds, not forever)

struct GArgs {
  int K, logK, T, S, P, ntc;  // grid side, log2 K, tile side, staged region side, region row pitch, tiles per side
  const Unit* units;
  long long u_begin, n_units;  // this launch walks units [u_begin, n_units) (one w-stack)
  const Chunk* chunks;
  const int64_t* rowptr;
  const void* w;
  const uint16_t* cells;  // per tap: cell lr * P + lc of the row's staged region
  const uint8_t* runs;    // per chunk: row offsets where runs of a shared tap window start, then nrows
  const int32_t* perm;
  const float2* y_in;   // sorted order (G_GRID, G_FUSED); NULL in G_FUSED = no data term
  float2* y_out;        // caller order (G_DEGRID)
  const float2* gridA;  // input grid (G_DEGRID, G_FUSED)
  float2* gridB;        // output grid (G_GRID, G_FUSED)
  __nv_bfloat162* gridB_lo;  // compensation grid: the rounding errors of the flushes into gridB, or NULL
  int* status;          // bit 1: pipeline wait timed out; bit 2: inconsistent work list (chunk skipped)
};

// Rounding error of the float sum s = a + b (Knuth's TwoSum): a + b = s + err exactly.  The
// intrinsics keep the compiler from contracting or reassociating the sequence.
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bb = __fsub_rn(s, a);
  return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false when the limit was reached
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <typename WT>
struct WBytes;
template <>
struct WBytes<float2> {
  static constexpr int value = 8;
};
template <>
struct WBytes<__nv_bfloat162> {
  static constexpr int value = 4;
};

template <typename WT>
__device__ __forceinline__ float2 w_at(const unsigned char* base, int i) {
  if constexpr (WBytes<WT>::value == 8) {
    return reinterpret_cast<const float2*>(base)[i];
  } else {
    return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(base)[i]);
  }
}
// Shared-memory stage: [weights | cells | visibilities | run list | chunk descriptor], each
// 128-B aligned.  The producer writes the descriptor with plain stores before its arrive on
// the stage's full barrier (release), so consumers read it from shared memory after their
// wait (acquire) instead of each fetching it from global memory.
// Every row of a chunk has the same support J (rows are sorted by J within a tile), so
// row q of a chunk starts at tap q J^2 and the row offsets need not be read.
template <typename WT>
struct StageLayout {
  static constexpr int al(int b) { return (b + 127) & ~127; }
  static constexpr int W_BYTES = (CHUNK_TAPS + 16) * WBytes<WT>::value;
  static constexpr int C_BYTES = (CHUNK_TAPS + 16) * 2;
  static constexpr int Y_BYTES = (CHUNK_ROWS + 4) * 8;
  static constexpr int R_BYTES = CHUNK_ROWS + 32;
  static constexpr int W_OFF = 0;
  static constexpr int C_OFF = al(W_BYTES);
  static constexpr int Y_OFF = C_OFF + al(C_BYTES);
  static constexpr int R_OFF = Y_OFF + al(Y_BYTES);
  static constexpr int H_OFF = R_OFF + al(R_BYTES);
  static constexpr int SIZE = H_OFF + al((int)sizeof(Chunk));
};

template <int MODE, typename WT>
__device__ __forceinline__ void issue_chunk(const GArgs& A, const Chunk& ch, unsigned char* stage,
                                            uint64_t* bar) {
  using L = StageLayout<WT>;
  constexpr int WB = WBytes<WT>::value;
  // 16-byte aligned copy windows around the chunk, 8 taps (16 B of cells) granular; the arrays
  // are padded at the end
  const long long tb0 = ch.tap_begin & ~7LL, te = (ch.tap_begin + ch.ntaps + 7) & ~7LL;
  const long long rb0 = ch.row_begin & ~1LL, ye = (ch.row_begin + ch.nrows + 1) & ~1LL;
  const uint32_t wbytes = (uint32_t)((te - tb0) * WB), cbytes = (uint32_t)((te - tb0) * 2);
  const uint32_t ybytes = (uint32_t)((ye - rb0) * 8);
  const long long rs0 = ch.run_begin & ~15LL, re = (ch.run_begin + ch.nruns + 1 + 15) & ~15LL;
  const uint32_t rbytes = (uint32_t)(re - rs0);
  const bool need_y = MODE != G_DEGRID && A.y_in != nullptr;
  *reinterpret_cast<Chunk*>(stage + L::H_OFF) = ch;  // published by the arrive below
  mbar_expect_tx(bar, wbytes + cbytes + rbytes + (need_y ? ybytes : 0));
  bulk_g2s(stage + L::W_OFF, reinterpret_cast<const unsigned char*>(A.w) + tb0 * WB, wbytes, bar);
  bulk_g2s(stage + L::C_OFF, A.cells + tb0, cbytes, bar);
  bulk_g2s(stage + L::R_OFF, A.runs + rs0, rbytes, bar);
  if (need_y) bulk_g2s(stage + L::Y_OFF, A.y_in + rb0, ybytes, bar);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// barrier among the consumer warps only (the producer warp never joins it)
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(GPASS_CONSUMERS * 32) : "memory");
}

struct RowCtx {
  float2* sx;     // staged input region (complex), S rows of pitch P cells
  float* sy_re;   // accumulated output region, real plane
  float* sy_im;   // accumulated output region, imaginary plane
  int S, P, r0, c0, logK, Km, lane;
};

// Warp sums of V per-lane values (V a power of two, 2 <= V <= 32).  The first log2 V
// butterfly stages exchange half of the values still held with the partner lane, so each
// stage costs V / 2^(stage+1) shuffles instead of V, and the last stages sum one value; the
// adds follow the same pairing tree as V separate xor butterflies.  On return v[0] of lane l
// holds the sum of value l >> (5 - log2 V).
template <int V>
__device__ __forceinline__ void warp_sum_many(float (&v)[V], int lane) {
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int o = 16 >> st, n = V >> st;
    if (n > 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < n / 2; ++i) {
        const float send = up ? v[i] : v[i + n / 2];
        const float keep = up ? v[i + n / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
  }
}

constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

// Runs k0, k0 + NCW, ... of one J-uniform chunk, SL register slots of 32 taps per lane.
// The rows of a run share their tap window (same first cell, same support): the run's
// cells and staged grid values are loaded once, each row contributes its own residual
// r_m = sum_k G_mk X_k - y_m, and the scatter terms conj(G_mk) r_m are summed in registers
// over the run before one pair of shared atomics per tap.  Lanes without a tap point at
// their own dummy cell S P + lane with weight 0, so the slot loops are branch-free, and
// every cell is clamped into the region.  The residuals of RB rows of a run are formed
// together (independent FMA chains, one multi-value warp sum) before their scatter terms.
template <int MODE, typename WT, int SL, int RB>
__device__ __forceinline__ void process_chunk(const GArgs& A, const Chunk& ch, const unsigned char* stage,
                                              int k0, const RowCtx& C) {
  using L = StageLayout<WT>;
  const unsigned char* sw = stage + L::W_OFF;
  const uint16_t* sc = reinterpret_cast<const uint16_t*>(stage + L::C_OFF);
  const float2* syv = reinterpret_cast<const float2*>(stage + L::Y_OFF);
  const uint8_t* sr = stage + L::R_OFF + (int)(ch.run_begin & 15LL);
  const int toff = (int)(ch.tap_begin & 7LL);
  const int roff = (int)(ch.row_begin & 1LL);
  const int nn = ch.nn;
  const int lane = C.lane;
  const int dummy = C.S * C.P + lane;
  for (int k = k0; k < ch.nruns; k += GPASS_CONSUMERS) {
    const int qe = min((int)sr[k + 1], ch.nrows), qb = min((int)sr[k], qe);
    int idx[SL];
    float2 xv[SL], ar[SL];
#pragma unroll
    for (int s = 0; s < SL; ++s) {
      const int t = lane + 32 * s;
      idx[s] = t < nn ? min((int)sc[toff + qb * nn + t], dummy) : dummy;
      if (MODE != G_GRID) xv[s] = C.sx[idx[s]];
      ar[s] = make_float2(0.f, 0.f);
    }
    if (MODE == G_GRID) {
      for (int q = qb; q < qe; ++q) {
        const int beg = toff + q * nn;
        const float2 r = syv[roff + q];
#pragma unroll
        for (int s = 0; s < SL; ++s) {
          const int t = lane + 32 * s;
          const float2 w = t < nn ? w_at<WT>(sw, beg + t) : make_float2(0.f, 0.f);
          ar[s].x = fmaf(w.x, r.x, fmaf(w.y, r.y, ar[s].x));   // += conj(w) r
          ar[s].y = fmaf(w.x, r.y, fmaf(-w.y, r.x, ar[s].y));
        }
      }
    } else {
      constexpr int SH = 5 - ilog2c(2 * RB);  // value i of the warp sum sits in lane i << SH
      for (int q = qb; q < qe; q += RB) {
        float v[2 * RB];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
          float2 acc = make_float2(0.f, 0.f);
          if (b == 0 || q + b < qe) {  // warp-uniform
            const int beg = toff + (q + b) * nn;
#pragma unroll
            for (int s = 0; s < SL; ++s) {
              const int t = lane + 32 * s;
              const float2 w = t < nn ? w_at<WT>(sw, beg + t) : make_float2(0.f, 0.f);
              acc.x = fmaf(w.x, xv[s].x, fmaf(-w.y, xv[s].y, acc.x));
              acc.y = fmaf(w.x, xv[s].y, fmaf(w.y, xv[s].x, acc.y));
            }
          }
          v[2 * b] = acc.x;
          v[2 * b + 1] = acc.y;
        }
        warp_sum_many<2 * RB>(v, lane);
#pragma unroll
        for (int b = 0; b < RB; ++b) {
          if (b > 0 && q + b >= qe) break;  // warp-uniform
          float2 r = make_float2(__shfl_sync(0xffffffffu, v[0], (2 * b) << SH),
                                 __shfl_sync(0xffffffffu, v[0], (2 * b + 1) << SH));
          if (MODE == G_DEGRID) {
            if (lane == 0) A.y_out[A.perm[ch.row_begin + q + b]] = r;
            continue;
          }
          if (A.y_in) r = csub(r, syv[roff + q + b]);
          const int beg = toff + (q + b) * nn;
#pragma unroll
          for (int s = 0; s < SL; ++s) {
            const int t = lane + 32 * s;
            const float2 w = t < nn ? w_at<WT>(sw, beg + t) : make_float2(0.f, 0.f);
            ar[s].x = fmaf(w.x, r.x, fmaf(w.y, r.y, ar[s].x));   // += conj(w) r
            ar[s].y = fmaf(w.x, r.y, fmaf(-w.y, r.x, ar[s].y));
          }
        }
      }
    }
    if (MODE != G_DEGRID) {
#pragma unroll
      for (int s = 0; s < SL; ++s) {
        if (lane + 32 * s < nn) {  // a predicated pair of atomics, no divergent branch
          atomicAdd(&C.sy_re[idx[s]], ar[s].x);
          atomicAdd(&C.sy_im[idx[s]], ar[s].y);
        }
      }
    }
  }
}


// Compensated flush of a unit's shared-memory partial sums into the output grid: each atomic returns
// the value it added to, so the thread forms the exact rounding error of the (round-to-nearest) sum
// (TwoSum) and adds it to the compensation grid.  A thread issues the atomics of two cells before it
// waits for their results.  Kept out of line so that the registers it needs do not count against the
// main loop of the gridding pass.
__device__ __noinline__ void flush_compensated(const float* sy_re, const float* sy_im, float2* gridB,
                                               __nv_bfloat162* gridB_lo, int S, int P, int r0, int c0,
                                               int logK, int Km, int ctid) {
  constexpr int FB = 2, CT = GPASS_CONSUMERS * 32;
  const int SS = S * S;
  for (int c0f = ctid; c0f < SS; c0f += FB * CT) {
    float2 v[FB], old[FB];
    size_t g[FB];
#pragma unroll
    for (int f = 0; f < FB; ++f) {
      const int c = c0f + f * CT;
      v[f] = make_float2(0.f, 0.f);
      g[f] = 0;
      if (c < SS) {
        const int i = c / S, jj = c - i * S;
        v[f] = make_float2(sy_re[i * P + jj], sy_im[i * P + jj]);
        g[f] = ((size_t)((r0 + i) & Km) << logK) + ((c0 + jj) & Km);
      }
    }
#pragma unroll
    for (int f = 0; f < FB; ++f)
      if (v[f].x != 0.f || v[f].y != 0.f) old[f] = atomicAdd(&gridB[g[f]], v[f]);
#pragma unroll
    for (int f = 0; f < FB; ++f) {
      if (v[f].x != 0.f || v[f].y != 0.f) {
        const float ex = two_sum_err(old[f].x, v[f].x, __fadd_rn(old[f].x, v[f].x));
        const float ey = two_sum_err(old[f].y, v[f].y, __fadd_rn(old[f].y, v[f].y));
        if (ex != 0.f || ey != 0.f) atomicAdd(&gridB_lo[g[f]], __floats2bfloat162_rn(ex, ey));
      }
    }
  }
}

// Warp-specialised CTA: warps 0..GPASS_CONSUMERS-1 consume chunks, the last
// warp produces them.  full[s] completes when stage s has landed (TMA
// transaction count); empty[s] completes when every consumer warp has released
// stage s.  Consumer warps only meet at unit boundaries (tile restage/flush).
template <int MODE, typename WT, int RB, bool COMP>
__global__ void __launch_bounds__(GPASS_THREADS, 1) gpass(GArgs A) {
  using L = StageLayout<WT>;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ uint64_t full[NSTAGE], empty[NSTAGE];
  __shared__ volatile int s_abort;
  const int S = A.S, P = A.P, SS = S * S, SP = S * P, logK = A.logK, Km = A.K - 1;
  const int region_bytes = (((SP + 32) * 8 + 127) & ~127);  // + one dummy cell per lane
  // input region: interleaved complex; output region: separate real and imaginary planes
  // (consecutive cells in consecutive banks); rows of both are P cells apart, P chosen at
  // plan time to spread the lanes of a J x J tap block over the banks (gridding_pitch)
  float2* sx = reinterpret_cast<float2*>(sm);
  float* sy_re = reinterpret_cast<float*>(MODE == G_FUSED ? sm + region_bytes : sm);
  float* sy_im = sy_re + (SP + 32);
  unsigned char* stages = sm + (MODE == G_FUSED ? 2 : 1) * region_bytes;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NCW = GPASS_CONSUMERS;
  constexpr int CT = NCW * 32;

  if (A.u_begin + blockIdx.x >= A.n_units) return;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    fence_barrier_init();
    s_abort = 0;
  }
  __syncthreads();  // the only CTA-wide barrier: roles split below

  if (warp == NCW) {
    // ---------------- producer warp (lane 0 issues every copy)
    if (lane != 0) return;
    // The descriptors of the next chunk are loaded before the current one is issued, so their
    // latency overlaps the wait for a free stage instead of adding to every issue.
    long long u = A.u_begin + blockIdx.x;
    int c = 0;
    Unit U = A.units[u];
    Chunk cur = A.chunks[U.chunk_begin];
    int st = 0;
    uint32_t ph = 0;       // parity of the current use of stage st
    long long j = 0;
    bool more = true;
    while (more) {
      if (j >= NSTAGE && !mbar_wait(&empty[st], ph ^ 1u)) {
        s_abort = 1;
        break;
      }
      if (s_abort) break;
      Chunk nxt = cur;
      if (++c < U.nchunks) {
        nxt = A.chunks[U.chunk_begin + c];
      } else {
        c = 0;
        u += gridDim.x;
        more = u < A.n_units;
        if (more) {
          U = A.units[u];
          nxt = A.chunks[U.chunk_begin];
        }
      }
      fence_proxy_async();
      issue_chunk<MODE, WT>(A, cur, stages + st * L::SIZE, &full[st]);
      ++j;
      if (++st == NSTAGE) {
        st = 0;
        ph ^= 1u;
      }
      cur = nxt;
    }
    // every issued copy must land before the CTA's shared memory can be released
    for (int d = 0; d < NSTAGE && d < j; ++d) {
      if (--st < 0) {
        st = NSTAGE - 1;
        ph ^= 1u;
      }
      mbar_wait(&full[st], ph);
    }
    return;
  }

  // ---------------- consumer warps
  const int ctid = threadIdx.x;  // 0..CT-1
  int st = 0;
  uint32_t ph = 0;
  int rb = 0;  // rows of the stream before the current chunk, modulo NCW
  for (long long u = A.u_begin + blockIdx.x; u < A.n_units; u += gridDim.x) {
    const Unit U = A.units[u];
    const int tr = U.tile / A.ntc, tc = U.tile - tr * A.ntc;
    const int r0 = tr * A.T, c0 = tc * A.T;
    if (MODE != G_GRID)
      for (int c = ctid; c < SS; c += CT) {
        const int i = c / S, jj = c - i * S;
        sx[i * P + jj] = A.gridA[((size_t)((r0 + i) & Km) << logK) + ((c0 + jj) & Km)];
      }
    if (ctid < 32 && MODE != G_GRID) sx[SP + ctid] = make_float2(0.f, 0.f);
    if (MODE != G_DEGRID)
      for (int c = ctid; c < SP + 32; c += CT) {
        sy_re[c] = 0.f;
        sy_im[c] = 0.f;
      }
    consumers_sync();
    const RowCtx C{sx, sy_re, sy_im, S, P, r0, c0, logK, Km, lane};

    for (int ci = 0; ci < U.nchunks; ++ci) {
      bool ok = false;
      if (!s_abort) {
        ok = mbar_wait(&full[st], ph);
        if (!ok) s_abort = 1;
      }
      const unsigned char* stage = stages + st * L::SIZE;
      const Chunk ch = ok ? *reinterpret_cast<const Chunk*>(stage + L::H_OFF) : A.chunks[U.chunk_begin + ci];
      // a warp works on the stage only when all of its lanes saw the copy land
      if (__all_sync(0xffffffffu, ok)) {
        // runs are dealt to warps round robin over the whole stream, so no warp idles per chunk
        const int q0 = warp >= rb ? warp - rb : warp - rb + NCW;
        if (ch.nn * ch.nrows != ch.ntaps || (ch.tap_begin & 7LL) + ch.ntaps > CHUNK_TAPS + 16 ||
            ch.nruns < 1 || ch.nruns > ch.nrows || (ch.run_begin & 15LL) + ch.nruns + 1 > CHUNK_ROWS + 32) {
          if (lane == 0) atomicOr(A.status, 4);  // inconsistent work list: skip the chunk
        } else if (ch.nn <= 64) {
          process_chunk<MODE, WT, 2, RB>(A, ch, stage, q0, C);
        } else if (ch.nn <= 96) {
          process_chunk<MODE, WT, 3, RB>(A, ch, stage, q0, C);
        } else if (ch.nn <= 160) {
          process_chunk<MODE, WT, 5, RB>(A, ch, stage, q0, C);
        } else {
          process_chunk<MODE, WT, 8, RB>(A, ch, stage, q0, C);
        }
      }
      rb = (rb + (ch.nruns > 0 ? ch.nruns : 0)) % NCW;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);  // this warp is done with the stage
      if (++st == NSTAGE) {
        st = 0;
        ph ^= 1u;
      }
    }
    consumers_sync();  // all scatters of this unit are in sy
    if (MODE != G_DEGRID && !s_abort) {
      if (COMP) {
        flush_compensated(sy_re, sy_im, A.gridB, A.gridB_lo, S, P, r0, c0, logK, Km, ctid);
      } else {
        for (int c = ctid; c < SS; c += CT) {
          const int i = c / S, jj = c - i * S;
          const float2 v = make_float2(sy_re[i * P + jj], sy_im[i * P + jj]);
          if (v.x != 0.f || v.y != 0.f) {
            atomicAdd(&A.gridB[((size_t)((r0 + i) & Km) << logK) + ((c0 + jj) & Km)], v);
          }
        }
      }
    }
    consumers_sync();  // the region may be restaged for the next unit
  }
  if (s_abort && ctid == 0) atomicOr(A.status, 2);
}

__global__ void permute_kernel(const float2* __restrict__ y, const int32_t* __restrict__ perm,
                               float2* __restrict__ out, int64_t M, float scale) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = y[perm[i]];
    out[i] = make_float2(v.x * scale, v.y * scale);
  }
}

template <int MODE, typename WT, int RB, bool COMP>
int launch_gpass(pnp_plan* p, const GArgs& A) {
  const int region_bytes = (((A.S * A.P + 32) * 8 + 127) & ~127);
  const int smem = (MODE == G_FUSED ? 2 : 1) * region_bytes + NSTAGE * StageLayout<WT>::SIZE;
  static int attr = 0;
  static int per_sm = 0;
  if (smem > attr) {
    PNP_CUDA(cudaFuncSetAttribute(gpass<MODE, WT, RB, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = smem;
    PNP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gpass<MODE, WT, RB, COMP>, GPASS_THREADS, smem));
  }
  if (per_sm < 1) return fail(PNP_ERR_UNSUPPORTED, "gridding tile does not fit in shared memory");
  long long grid = (long long)per_sm * p->num_sms;
  if (grid > A.n_units - A.u_begin) grid = A.n_units - A.u_begin;
  if (grid < 1) return PNP_OK;
  gpass<MODE, WT, RB, COMP><<<(unsigned)grid, GPASS_THREADS, smem, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

template <int MODE, int RB>
int dispatch_wt(pnp_plan* p, const GArgs& A) {
  if constexpr (MODE == G_DEGRID) {  // no gridding, nothing to compensate
    return p->wdtype == PNP_W_BF16C ? launch_gpass<MODE, __nv_bfloat162, RB, false>(p, A)
                                    : launch_gpass<MODE, float2, RB, false>(p, A);
  } else if (A.gridB_lo) {
    return p->wdtype == PNP_W_BF16C ? launch_gpass<MODE, __nv_bfloat162, RB, true>(p, A)
                                    : launch_gpass<MODE, float2, RB, true>(p, A);
  } else {
    return p->wdtype == PNP_W_BF16C ? launch_gpass<MODE, __nv_bfloat162, RB, false>(p, A)
                                    : launch_gpass<MODE, float2, RB, false>(p, A);
  }
}

// rows whose residuals one warp forms together (G_GRID takes its residuals as input)
template <int MODE>
int dispatch_rb(pnp_plan* p, const GArgs& A) {
  if constexpr (MODE == G_GRID) {
    return dispatch_wt<MODE, 1>(p, A);
  } else {
    switch (p->row_batch) {
      case 1: return dispatch_wt<MODE, 1>(p, A);
      case 4: return dispatch_wt<MODE, 4>(p, A);
      default: return dispatch_wt<MODE, 2>(p, A);
    }
  }
}

// Modelled shared-memory wavefronts of one row of J x J taps on regions of row pitch P: lane t of
// register slot s holds tap 32 s + t at cell (t / J) P + t % J; the residual gathers 8-byte cells
// (two banks each) and the scatter issues one 4-byte atomic per plane.  A wavefront serves each
// bank once, so a warp access costs the largest number of lanes that meet in one bank.
int64_t row_wavefronts(int J, int P) {
  const int nn = J * J;
  int64_t total = 0;
  for (int s = 0; s * 32 < nn; ++s) {
    int g[32] = {}, sc[32] = {};
    const int lanes = std::min(32, nn - 32 * s);
    for (int l = 0; l < lanes; ++l) {
      const int t = 32 * s + l, addr = (t / J) * P + t % J;
      sc[addr & 31]++;
      g[(2 * addr) & 31]++;
      g[(2 * addr + 1) & 31]++;
    }
    int mg = 0, ms = 0;
    for (int b = 0; b < 32; ++b) {
      mg = std::max(mg, g[b]);
      ms = std::max(ms, sc[b]);
    }
    total += std::max(mg, (2 * lanes + 31) / 32) + 2 * ms;
  }
  return total;
}

}  // namespace

int gridding_pitch(pnp_plan* p, const int64_t* rows_per_J) {
  const int S = p->tile + p->Jmax - 1;
  int optin = 0;
  PNP_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
  const int stage = NSTAGE * std::max(StageLayout<float2>::SIZE, StageLayout<__nv_bfloat162>::SIZE);
  if (2 * ((((S * S + 32) * 8 + 127) & ~127)) + stage + 1024 > optin)
    return fail(PNP_ERR_UNSUPPORTED, "gridding tile and pipeline stages do not fit in shared memory");
  int best = S;
  int64_t best_cost = -1;
  for (int P = S; P < S + 32; ++P) {
    const int region_bytes = (((S * P + 32) * 8 + 127) & ~127);
    if (2 * region_bytes + stage + 1024 > optin) break;  // fused pass: two regions + the stages
    int64_t cost = 0;
    for (int J = 1; J <= 16; ++J)
      if (rows_per_J[J]) cost += rows_per_J[J] * row_wavefronts(J, P);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = P;
    }
  }
  p->pitch = best;
  return PNP_OK;
}

int permute_y(pnp_plan* p, const float2* y_user, float scale) {
  if (p->M == 0) return PNP_OK;
  const int threads = 256;
  long long blocks = (p->M + threads - 1) / threads;
  if (blocks > 8L * p->num_sms * 8) blocks = 8L * p->num_sms * 8;
  permute_kernel<<<(unsigned)blocks, threads, 0, p->stream>>>(y_user, p->d_perm, p->d_ysorted, p->M, scale);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

// mode G_DEGRID: y_out (caller order) = G gridA.
// mode G_GRID:   gridB += G^H d_ysorted.
// mode G_FUSED:  gridB += G^H (G gridA - d_ysorted)  (no data term when y_user == NULL).
int gridding_pass(pnp_plan* p, int mode, const float2* y_user, float2* y_out, int s) {
  if (p->M == 0 || p->n_units == 0) return PNP_OK;
  if (s < 0 || s >= p->nstacks) return fail(PNP_ERR_INVALID_ARG, "internal: stack index out of range");
  const long long ub = p->h_stack_units[s], ue = p->h_stack_units[s + 1];
  if (ub >= ue) return PNP_OK;  // a stack without rows grids nothing
  GArgs A{};
  A.K = p->K;
  A.logK = p->logK;
  A.T = p->tile;
  A.S = p->tile + p->Jmax - 1;
  A.P = p->pitch > 0 ? p->pitch : A.S;
  A.ntc = p->ntc;
  A.units = p->d_units;
  A.u_begin = ub;
  A.n_units = ue;
  A.chunks = p->d_chunks;
  A.rowptr = p->d_rowptr;
  A.w = p->d_w;
  A.cells = p->d_cells;
  A.runs = p->d_runs;
  A.perm = p->d_perm;
  A.y_in = (mode == G_DEGRID || y_user == nullptr) ? nullptr : p->d_ysorted;
  A.y_out = y_out;
  A.gridA = p->d_gridA;
  A.gridB = p->d_gridB;
  A.gridB_lo = p->compensated ? p->d_gridB_lo : nullptr;
  A.status = p->d_status;
  cudaEvent_t ev;
  if (int rc = stage_begin(p, 1, &ev)) return rc;
  int rc;
  switch (mode) {
    case G_DEGRID: rc = dispatch_rb<G_DEGRID>(p, A); break;
    case G_GRID: rc = dispatch_rb<G_GRID>(p, A); break;
    default: rc = dispatch_rb<G_FUSED>(p, A); break;
  }
  if (rc) return rc;
  return stage_end(p, 1, ev);
}

}  // namespace pnp
