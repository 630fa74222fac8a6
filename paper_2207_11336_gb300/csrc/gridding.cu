// De-gridding y = G X (Eq. 1) and gridding G^H r (App. A), separately or fused
// into one pass over G that forms the residual r = G X - y and grids it.
//
// G is CSR with rows sorted by the grid tile holding their first tap (and by
// data block within a tile).  A work unit is a run of consecutive rows of one
// tile.  For each unit a CTA
//   1. stages the tile plus a (Jmax-1)-cell halo of the input grid X in shared
//      memory (coalesced along k0, wrapped mod K);
//   2. runs warp-per-row SpMV: the row's taps are read lane-strided (coalesced
//      8-byte weights and 4-byte column indices, streamed past L1/L2), gathered
//      from shared memory and reduced with warp shuffles; RPW rows are in
//      flight per warp so enough loads are outstanding to cover HBM latency;
//   3. scatters conj(G_mk) r_m of every tap into a shared-memory copy of the
//      same tile+halo region (shared-memory float atomics);
//   4. adds the non-zero cells of that region to the output grid with
//      vector float2 global atomics.
// Grid layout: grid[k1*K + k0]; column index of a tap = k1*K + k0.
#include "common.cuh"

namespace pnp {
namespace {

struct GArgs {
  int K, logK, T, S, ntc;
  const Unit* units;
  long long n_units;
  const int64_t* rowptr;
  const void* w;
  const int32_t* cols;
  const int32_t* perm;
  const float2* y_in;   // sorted order (G_GRID, G_FUSED); NULL in G_FUSED = no data term
  float2* y_out;        // caller order (G_DEGRID)
  const float2* gridA;  // input grid (G_DEGRID, G_FUSED)
  float2* gridB;        // output grid (G_GRID, G_FUSED)
  int* status;          // bit 0 set when a tap falls outside the staged region (tap skipped)
};

template <typename WT>
__device__ __forceinline__ float2 load_w(const void* w, int64_t i);
template <>
__device__ __forceinline__ float2 load_w<float2>(const void* w, int64_t i) {
  return __ldcs(reinterpret_cast<const float2*>(w) + i);
}
template <>
__device__ __forceinline__ float2 load_w<__nv_bfloat162>(const void* w, int64_t i) {
  const unsigned int u = __ldcs(reinterpret_cast<const unsigned int*>(w) + i);
  __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&u);
  return __bfloat1622float2(b);
}

template <int MODE, typename WT, int SLOTS, int RPW>
__global__ void __launch_bounds__(256) gpass(GArgs A) {
  extern __shared__ float2 sm[];
  const int S = A.S, SS = S * S, K = A.K, logK = A.logK, Km = K - 1;
  float2* sx = sm;                                     // staged input region
  float2* sy = (MODE == G_FUSED) ? sm + SS : sm;       // accumulated output region
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

  for (long long u = blockIdx.x; u < A.n_units; u += gridDim.x) {
    const Unit U = A.units[u];
    const int tr = U.tile / A.ntc, tc = U.tile - tr * A.ntc;
    const int r0 = tr * A.T, c0 = tc * A.T;
    if (MODE != G_GRID) {
      for (int c = threadIdx.x; c < SS; c += blockDim.x) {
        const int i = c / S, jj = c - i * S;
        sx[c] = A.gridA[((size_t)((r0 + i) & Km) << logK) + ((c0 + jj) & Km)];
      }
    }
    if (MODE != G_DEGRID)
      for (int c = threadIdx.x; c < SS; c += blockDim.x) sy[c] = make_float2(0.f, 0.f);
    __syncthreads();

    for (int q0 = warp * RPW; q0 < U.nrows; q0 += nw * RPW) {
      float2 wv[RPW][SLOTS];
      int idx[RPW][SLOTS];
      long long m[RPW];
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        const bool valid = q0 + q < U.nrows;
        m[q] = U.row_begin + q0 + q;
        const int64_t beg = valid ? A.rowptr[m[q]] : 0;
        const int cnt = valid ? (int)(A.rowptr[m[q] + 1] - beg) : 0;
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
          const int t = lane + 32 * s;
          if (t < cnt) {
            wv[q][s] = load_w<WT>(A.w, beg + t);
            const int col = __ldcs(A.cols + beg + t);
            const int lr = ((col >> logK) - r0) & Km;
            const int lc = ((col & Km) - c0) & Km;
            if (lr < S && lc < S) {
              idx[q][s] = lr * S + lc;
            } else {
              atomicOr(A.status, 1);
              idx[q][s] = -1;
            }
          } else {
            wv[q][s] = make_float2(0.f, 0.f);
            idx[q][s] = -1;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < RPW; ++q) {
        if (q0 + q >= U.nrows) break;
        float2 r = make_float2(0.f, 0.f);
        if (MODE != G_GRID) {
          float2 acc = make_float2(0.f, 0.f);
#pragma unroll
          for (int s = 0; s < SLOTS; ++s)
            if (idx[q][s] >= 0) {
              const float2 xv = sx[idx[q][s]];
              acc.x = fmaf(wv[q][s].x, xv.x, fmaf(-wv[q][s].y, xv.y, acc.x));
              acc.y = fmaf(wv[q][s].x, xv.y, fmaf(wv[q][s].y, xv.x, acc.y));
            }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
          }
          if (MODE == G_DEGRID) {
            if (lane == 0) A.y_out[A.perm[m[q]]] = acc;
            continue;
          }
          r = acc;
          if (A.y_in) r = csub(r, A.y_in[m[q]]);
        } else {
          r = A.y_in[m[q]];
        }
#pragma unroll
        for (int s = 0; s < SLOTS; ++s)
          if (idx[q][s] >= 0) {
            const float2 c = cmulc(wv[q][s], r);
            atomicAdd(&sy[idx[q][s]].x, c.x);
            atomicAdd(&sy[idx[q][s]].y, c.y);
          }
      }
    }
    __syncthreads();
    if (MODE != G_DEGRID) {
      for (int c = threadIdx.x; c < SS; c += blockDim.x) {
        const float2 v = sy[c];
        if (v.x != 0.f || v.y != 0.f) {
          const int i = c / S, jj = c - i * S;
          atomicAdd(&A.gridB[((size_t)((r0 + i) & Km) << logK) + ((c0 + jj) & Km)], v);
        }
      }
      __syncthreads();
    }
  }
}

__global__ void permute_kernel(const float2* __restrict__ y, const int32_t* __restrict__ perm,
                               float2* __restrict__ out, int64_t M) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = y[perm[i]];
}

template <int MODE, typename WT, int SLOTS, int RPW>
int launch_gpass(pnp_plan* p, const GArgs& A) {
  const int smem = (MODE == G_FUSED ? 2 : 1) * A.S * A.S * (int)sizeof(float2);
  static int attr = 0;
  if (smem > attr) {
    PNP_CUDA(cudaFuncSetAttribute(gpass<MODE, WT, SLOTS, RPW>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = smem;
  }
  int per_sm = 0;
  PNP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gpass<MODE, WT, SLOTS, RPW>, 256, smem));
  if (per_sm < 1) return fail(PNP_ERR_UNSUPPORTED, "gridding tile does not fit in shared memory");
  long long grid = (long long)per_sm * p->num_sms;
  if (grid > A.n_units) grid = A.n_units;
  if (grid < 1) return PNP_OK;
  gpass<MODE, WT, SLOTS, RPW><<<(unsigned)grid, 256, smem, p->stream>>>(A);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

template <int MODE, typename WT>
int dispatch_slots(pnp_plan* p, const GArgs& A) {
  const int rpw = p->rpw;
  switch (p->slots) {
    case 2:
      return rpw == 1 ? launch_gpass<MODE, WT, 2, 1>(p, A)
           : rpw == 4 ? launch_gpass<MODE, WT, 2, 4>(p, A) : launch_gpass<MODE, WT, 2, 2>(p, A);
    case 4:
      return rpw == 1 ? launch_gpass<MODE, WT, 4, 1>(p, A)
           : rpw == 4 ? launch_gpass<MODE, WT, 4, 4>(p, A) : launch_gpass<MODE, WT, 4, 2>(p, A);
    default:
      return rpw == 1 ? launch_gpass<MODE, WT, 8, 1>(p, A)
           : rpw == 4 ? launch_gpass<MODE, WT, 8, 4>(p, A) : launch_gpass<MODE, WT, 8, 2>(p, A);
  }
}

template <int MODE>
int dispatch_wt(pnp_plan* p, const GArgs& A) {
  return p->wdtype == PNP_W_BF16C ? dispatch_slots<MODE, __nv_bfloat162>(p, A)
                                  : dispatch_slots<MODE, float2>(p, A);
}

}  // namespace

int permute_y(pnp_plan* p, const float2* y_user) {
  if (p->M == 0) return PNP_OK;
  const int threads = 256;
  long long blocks = (p->M + threads - 1) / threads;
  if (blocks > 8L * p->num_sms * 8) blocks = 8L * p->num_sms * 8;
  permute_kernel<<<(unsigned)blocks, threads, 0, p->stream>>>(y_user, p->d_perm, p->d_ysorted, p->M);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

// mode G_DEGRID: y_out (caller order) = G gridA.
// mode G_GRID:   gridB += G^H d_ysorted.
// mode G_FUSED:  gridB += G^H (G gridA - d_ysorted)  (no data term when y_user == NULL).
int gridding_pass(pnp_plan* p, int mode, const float2* y_user, float2* y_out) {
  if (p->M == 0 || p->n_units == 0) return PNP_OK;
  GArgs A{};
  A.K = p->K;
  A.logK = p->logK;
  A.T = p->tile;
  A.S = p->tile + p->Jmax - 1;
  A.ntc = p->ntc;
  A.units = p->d_units;
  A.n_units = p->n_units;
  A.rowptr = p->d_rowptr;
  A.w = p->d_w;
  A.cols = p->d_cols;
  A.perm = p->d_perm;
  A.y_in = (mode == G_DEGRID || y_user == nullptr) ? nullptr : p->d_ysorted;
  A.y_out = y_out;
  A.gridA = p->d_gridA;
  A.gridB = p->d_gridB;
  A.status = p->d_status;
  cudaEvent_t ev;
  if (int rc = stage_begin(p, 1, &ev)) return rc;
  int rc;
  switch (mode) {
    case G_DEGRID: rc = dispatch_wt<G_DEGRID>(p, A); break;
    case G_GRID: rc = dispatch_wt<G_GRID>(p, A); break;
    default: rc = dispatch_wt<G_FUSED>(p, A); break;
  }
  if (rc) return rc;
  return stage_end(p, 1, ev);
}

}  // namespace pnp
