// Holographic form of the normal operator (App. E, Eq. phidagphi): H = G^H G, so that
// Phi^H Phi = Z^H F^H H F Z and the data-term gradient is Re{Z^H F^H (H F Z x - G^H y)}.
//
// H couples grid cells k, k' only when a row of G touches both, i.e. |k - k'| < Jmax per axis,
// so it is stored as a dense stencil of S x S entries (S = 2 Jmax - 1) per grid cell, laid out
// offset-major: H[delta][k] with delta = (dr + Jmax - 1) S + (dc + Jmax - 1), so that a warp of
// consecutive cells reads one offset's entries contiguously.  It is built once from the plan's
// rows (every pair of taps of a row adds conj(G_mk) G_mk' to H[k' - k][k] with a global atomic)
// and applied as a gather over the S x S neighbourhood with the dirty grid G^H y subtracted in
// the same pass.  Per application it reads S^2 K^2 x 8 B of H instead of the nnz x 10 B of G,
// which pays when the rows per cell are many (M >> K^2), the regime the paper uses it for.
#include "common.cuh"

namespace pnp {
namespace {

constexpr int HB_WARPS = 8;  // rows processed concurrently per block of the build

template <typename WT>
__device__ __forceinline__ float2 hw_at(const void* w, int64_t i) {
  if constexpr (sizeof(WT) == 8) {
    return reinterpret_cast<const float2*>(w)[i];
  } else {
    return __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(w)[i]);
  }
}

struct HBuildArgs {
  const Unit* units;
  int64_t n_units;
  const Chunk* chunks;
  const void* w;
  const uint16_t* cells;
  int T, ntc, P, R, Jmax, S, logK;  // tile side, tiles per side, region pitch and side, stencil side
  float2* H;
  int* status;  // bit 4: a tap pair outside the stencil (skipped)
};

// one block per work unit, one warp per row: the row's taps are staged in shared memory and every
// (i, j) pair adds conj(w_i) w_j to H[cell_j - cell_i][cell_i]
template <typename WT>
__global__ void __launch_bounds__(32 * HB_WARPS) holo_build(HBuildArgs A) {
  __shared__ int s_k[HB_WARPS][256];
  __shared__ short s_r[HB_WARPS][256], s_c[HB_WARPS][256];
  __shared__ float2 s_w[HB_WARPS][256];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int K = 1 << A.logK, Km = K - 1, Jm1 = A.Jmax - 1;
  const int64_t KK = (int64_t)K * K;
  for (int64_t u = blockIdx.x; u < A.n_units; u += gridDim.x) {
    const Unit U = A.units[u];
    const int r0 = (U.tile / A.ntc) * A.T, c0 = (U.tile % A.ntc) * A.T;
    for (int ci = 0; ci < U.nchunks; ++ci) {
      const Chunk ch = A.chunks[U.chunk_begin + ci];
      const int nn = ch.nn;
      if (nn > 256) continue;
      for (int q = wp; q < ch.nrows; q += HB_WARPS) {
        const int64_t base = ch.tap_begin + (int64_t)q * nn;
        for (int t = lane; t < nn; t += 32) {
          const int cell = A.cells[base + t];
          const int lr = cell / A.P, lc = cell - lr * A.P;
          s_r[wp][t] = (short)lr;
          s_c[wp][t] = (short)lc;
          s_k[wp][t] = (((r0 + lr) & Km) << A.logK) + ((c0 + lc) & Km);
          s_w[wp][t] = hw_at<WT>(A.w, base + t);
        }
        __syncwarp();
        for (int i = 0; i < nn; ++i) {
          const float2 wi = s_w[wp][i];
          const int ri = s_r[wp][i], cci = s_c[wp][i], ki = s_k[wp][i];
          for (int j = lane; j < nn; j += 32) {
            const int dr = s_r[wp][j] - ri, dc = s_c[wp][j] - cci;
            if (dr < -Jm1 || dr > Jm1 || dc < -Jm1 || dc > Jm1) {
              atomicOr(A.status, 16);
              continue;
            }
            const int64_t at = (int64_t)((dr + Jm1) * A.S + (dc + Jm1)) * KK + ki;
            atomicAdd(&A.H[at], cmulc(wi, s_w[wp][j]));  // conj(w_i) w_j
          }
        }
        __syncwarp();
      }
    }
  }
}

// out[k] = sum_delta H[delta][k] X[k + delta] - b[k]   (b = NULL: no data term)
__global__ void __launch_bounds__(256) holo_apply(const float2* __restrict__ H, const float2* __restrict__ X,
                                                  const float2* __restrict__ b, float2* __restrict__ out, int logK,
                                                  int Jmax, int S) {
  const int K = 1 << logK, Km = K - 1, Jm1 = Jmax - 1;
  const int64_t KK = (int64_t)K * K;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < KK; k += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(k >> logK), c = (int)(k & Km);
    float2 acc = make_float2(0.f, 0.f);
    for (int dr = -Jm1; dr <= Jm1; ++dr) {
      const float2* xrow = X + ((int64_t)((r + dr) & Km) << logK);
      const float2* hrow = H + (int64_t)(dr + Jm1) * S * KK + k;
      for (int dc = -Jm1; dc <= Jm1; ++dc) {
        const float2 h = hrow[(int64_t)(dc + Jm1) * KK];
        const float2 x = xrow[(c + dc) & Km];
        acc.x = fmaf(h.x, x.x, fmaf(-h.y, x.y, acc.x));
        acc.y = fmaf(h.x, x.y, fmaf(h.y, x.x, acc.y));
      }
    }
    out[k] = b ? csub(acc, b[k]) : acc;
  }
}

}  // namespace

int holo_build_plan(pnp_plan* p) {
  if (p->d_H) return PNP_OK;
  if (p->nstacks != 1) return fail(PNP_ERR_UNSUPPORTED, "the holographic operator is built for one w-stack");
  const int S = 2 * p->Jmax - 1;
  const size_t KK = (size_t)p->K * p->K, bytes = (size_t)S * S * KK * sizeof(float2);
  size_t free_b = 0, total_b = 0;
  PNP_CUDA(cudaMemGetInfo(&free_b, &total_b));
  if (bytes > free_b / 10 * 9) return fail(PNP_ERR_OOM, "H (" + std::to_string(bytes) + " bytes) does not fit");
  float2* H = nullptr;
  if (cudaMalloc(&H, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(PNP_ERR_OOM, "cudaMalloc of H failed");
  }
  float2* dirty = nullptr;
  if (cudaMalloc(&dirty, KK * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(H);
    return fail(PNP_ERR_OOM, "cudaMalloc of the dirty grid failed");
  }
  p->d_H = H;
  p->d_dirty = dirty;
  p->holo_S = S;
  p->device_bytes += (int64_t)(bytes + KK * sizeof(float2));
  PNP_CUDA(cudaMemsetAsync(H, 0, bytes, p->stream));
  if (p->M > 0 && p->n_units > 0) {
    HBuildArgs A{};
    A.units = p->d_units;
    A.n_units = p->n_units;
    A.chunks = p->d_chunks;
    A.w = p->d_w;
    A.cells = p->d_cells;
    A.T = p->tile;
    A.ntc = p->ntc;
    A.R = p->tile + p->Jmax - 1;
    A.P = p->pitch > 0 ? p->pitch : A.R;
    A.Jmax = p->Jmax;
    A.S = S;
    A.logK = p->logK;
    A.H = H;
    A.status = p->d_status;
    const unsigned grid = (unsigned)std::min<int64_t>(p->n_units, (int64_t)p->num_sms * 8);
    if (p->wdtype == PNP_W_BF16C)
      holo_build<__nv_bfloat162><<<grid, 32 * HB_WARPS, 0, p->stream>>>(A);
    else
      holo_build<float2><<<grid, 32 * HB_WARPS, 0, p->stream>>>(A);
    PNP_CHECK_LAUNCH();
  }
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  return PNP_OK;
}

namespace {
// out = hi + lo (lo may be NULL); hi and lo are left zero
__global__ void take_grid(float2* __restrict__ hi, __nv_bfloat162* __restrict__ lo, float2* __restrict__ out,
                          int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    float2 v = hi[i];
    hi[i] = make_float2(0.f, 0.f);
    if (lo) {
      const float2 e = __bfloat1622float2(lo[i]);
      v = make_float2(v.x + e.x, v.y + e.y);
      lo[i] = __floats2bfloat162_rn(0.f, 0.f);
    }
    out[i] = v;
  }
}
}  // namespace

int holo_dirty_grid(pnp_plan* p) {
  // G^H y from the sorted data: the gridding pass accumulates into the (zero) output grid and,
  // compensated, its rounding errors into the compensation grid; dirty = their sum, both re-zeroed
  if (int rc = gridding_pass(p, G_GRID, p->d_ysorted, nullptr, 0)) return rc;
  const int64_t KK = (int64_t)p->K * p->K;
  const unsigned grid = (unsigned)std::min<int64_t>((KK + 255) / 256, (int64_t)p->num_sms * 16);
  take_grid<<<grid, 256, 0, p->stream>>>(p->d_gridB, p->compensated ? p->d_gridB_lo : nullptr, p->d_dirty, KK);
  PNP_CHECK_LAUNCH();
  return PNP_OK;
}

int holo_apply_pass(pnp_plan* p, bool data_term) {
  cudaEvent_t ev;
  if (int rc = stage_begin(p, 1, &ev)) return rc;
  const int64_t KK = (int64_t)p->K * p->K;
  const unsigned grid = (unsigned)std::min<int64_t>((KK + 255) / 256, (int64_t)p->num_sms * 16);
  holo_apply<<<grid, 256, 0, p->stream>>>(p->d_H, p->d_gridA, data_term ? p->d_dirty : nullptr, p->d_gridB,
                                          p->logK, p->Jmax, p->holo_S);
  PNP_CHECK_LAUNCH();
  return stage_end(p, 1, ev);
}

}  // namespace pnp
