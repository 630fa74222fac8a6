// Construction of the measurement operator Phi = G F Z (Eq. 1; App. E).
//
// Host side (once per plan, O(M)): KB shape parameter and grid-correction
// table, FFT twiddles, per-row tap windows, a stable counting sort of the rows
// by (grid tile of the first tap, data block), CSR row offsets and the work
// units of the gridding kernels.
//
// Device side: one warp per row evaluates the row's separable weights
//   g(t) = sum_d w_hat[d] psi(t + d),  psi(t) = I0(beta sqrt(1 - (2t/J)^2)),
// on the J_m taps nearest kappa along each axis, and writes the J_m^2 outer
// products with their column indices.  w_hat is the K-point DFT of the
// paraxial w-chirp exp(i pi a q(p)), a = w dl^2, whose phase profile q equals
// p^2 on the image and is continued smoothly (C^2) to a flat value at |p| = K/2
// (App. E reading: the w-kernel of each row folded into its KB row).  It is
// evaluated from its Taylor series in b = pi a (n/2)^2 about the mid value of
// the normalised profile, using moments mu_j[d] = K^-1 sum_p (qn(p) - c0)^j
// cos(2 pi d p / K) precomputed here in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "common.cuh"

namespace pnp {
namespace {

constexpr int MAX_TERMS = 64;
constexpr int MAX_D = 15;  // |d| <= MAX_D, so 2 MAX_D + 1 <= 32 lanes

struct RowGeom {
  double kap0, kap1, a;  // kappa per axis, chirp rate a = w dl^2
  double d;              // data weight d_m multiplying the row (1 without weighting)
  int s0, s1;            // first tap (unwrapped) per axis
  int J;                 // row support J_m
};

struct BuildArgs {
  int64_t M;
  int K, logK, J;
  double beta, bscale, c0;   // b = bscale * a ; series centre c0
  int nterms, D;
  const double* mu;          // [nterms][2D+1]
  const RowGeom* geom;       // sorted order
  const int64_t* rowptr;
  void* w;
  uint16_t* cells;
  int T, S, P;               // gridding tile side, staged region side and row pitch
  int* err;                  // set when a tap falls outside its row's staged region
  int bf16;
};

__device__ __forceinline__ double kb_psi(double t, int J, double beta) {
  const double z = 1.0 - (2.0 * t / J) * (2.0 * t / J);
  return z >= 0.0 ? cyl_bessel_i0(beta * sqrt(z)) : 0.0;
}

// one warp per row
__global__ void __launch_bounds__(256) build_rows(BuildArgs A) {
  __shared__ double2 s_wh[8][2 * MAX_D + 1];
  __shared__ double s_psi[8][2][32];
  __shared__ double2 s_g[8][2][16];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t row = (int64_t)blockIdx.x * 8 + wl;
  if (row >= A.M) return;
  const RowGeom g = A.geom[row];
  const int Jm = g.J, D = A.D;
  const bool has_w = g.a != 0.0;
  // w-kernel values w_hat[d], d = -D..D
  if (has_w && lane <= 2 * D) {
    const double b = A.bscale * g.a;
    // sum_j (i b)^j / j! mu_j[d]
    double tr = 1.0, ti = 0.0, sr = 0.0, si = 0.0;
    for (int j = 0; j < A.nterms; ++j) {
      const double m = A.mu[j * (2 * D + 1) + lane];
      sr += tr * m;
      si += ti * m;
      const double nr = -ti * b / (j + 1), ni = tr * b / (j + 1);
      tr = nr;
      ti = ni;
    }
    double sn, cs;
    sincos(b * A.c0, &sn, &cs);
    s_wh[wl][lane] = make_double2(sr * cs - si * sn, sr * sn + si * cs);
  }
  // psi(t0 + e) for the integers e with |t0 + e| <= J/2, per axis
  const int ax = lane >> 4, sl = lane & 15;
  const double kap = ax ? g.kap1 : g.kap0;
  const int st = ax ? g.s1 : g.s0;
  const double t0 = kap - st;
  const int emin = (int)ceil(-t0 - 0.5 * A.J);
  s_psi[wl][ax][sl] = kb_psi(t0 + emin + sl, A.J, A.beta);
  __syncwarp();
  if (sl < Jm) {
    double gr = 0.0, gi = 0.0;
    if (has_w) {
      for (int i = 0; i <= A.J; ++i) {
        const double ps = s_psi[wl][ax][i];
        const int d = emin + i + sl;
        if (ps != 0.0 && d >= -D && d <= D) {
          const double2 w = s_wh[wl][d + D];
          gr += w.x * ps;
          gi += w.y * ps;
        }
      }
    } else {
      gr = kb_psi(t0 - sl, A.J, A.beta);
    }
    s_g[wl][ax][sl] = make_double2(gr, gi);
  }
  __syncwarp();
  const int64_t beg = A.rowptr[row];
  const int nn = Jm * Jm, Km = A.K - 1;
  for (int t = lane; t < nn; t += 32) {
    const int i1 = t / Jm, i0 = t - i1 * Jm;  // k1-major, k0-minor
    const double2 a = s_g[wl][0][i0], b = s_g[wl][1][i1];
    const float wr = (float)(g.d * (a.x * b.x - a.y * b.y)), wi = (float)(g.d * (a.x * b.y + a.y * b.x));
    if (A.bf16) {
      __nv_bfloat162 h = __floats2bfloat162_rn(wr, wi);
      reinterpret_cast<__nv_bfloat162*>(A.w)[beg + t] = h;
    } else {
      reinterpret_cast<float2*>(A.w)[beg + t] = make_float2(wr, wi);
    }
    // cell of the tap in the staged region of the row's tile (the tile of its first tap)
    const int r0 = (((g.s1 % A.K) + A.K) % A.K) / A.T * A.T, c0 = (((g.s0 % A.K) + A.K) % A.K) / A.T * A.T;
    const int lr = (g.s1 + i1 - r0) & Km, lc = (g.s0 + i0 - c0) & Km;
    if (lr >= A.S || lc >= A.S) atomicOr(A.err, 1);
    A.cells[beg + t] = (uint16_t)(lr < A.S && lc < A.S ? lr * A.P + lc : 0);
  }
}

// gather rows for export: canonical column order k0*K + k1, float weights.  src_off holds per
// row (first tap, tap count, tile origin r0, tile origin c0); cells are lr * P + lc from the origin.
__global__ void export_rows(const int64_t* __restrict__ src_off, const int64_t* __restrict__ dst_off,
                            int64_t nrows, const void* w, const uint16_t* cells, int P, int bf16, int logK,
                            float2* out_w, int32_t* out_c) {
  const int64_t r = blockIdx.x;
  if (r >= nrows) return;
  const int64_t s = src_off[4 * r], cnt = src_off[4 * r + 1], d = dst_off[r];
  const int r0 = (int)src_off[4 * r + 2], c0 = (int)src_off[4 * r + 3];
  const int Km = (1 << logK) - 1;
  for (int64_t t = threadIdx.x; t < cnt; t += blockDim.x) {
    float2 v;
    if (bf16) v = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(w)[s + t]);
    else v = reinterpret_cast<const float2*>(w)[s + t];
    const int c = cells[s + t], lr = c / P, lc = c - lr * P;
    out_w[d + t] = v;
    out_c[d + t] = (((c0 + lc) & Km) << logK) | ((r0 + lr) & Km);
  }
}

double kb_beta(int J, double sigma) {
  return M_PI * std::sqrt((J / sigma) * (J / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8);
}

double kb_correction(double p, int J, double beta, int K) {
  const double s = M_PI * J * p / K, r2 = beta * beta - s * s;
  if (r2 > 0) {
    const double r = std::sqrt(r2);
    return J * std::sinh(r) / r;
  }
  if (r2 < 0) {
    const double r = std::sqrt(-r2);
    return J * std::sin(r) / r;
  }
  return J;
}

// normalised frozen-chirp phase profile qn(p) = q(p) / (n/2)^2
double chirp_q(double p, int n, int K) {
  const double a = std::fabs(p), h = n / 2.0;
  if (a <= h) return a * a / (h * h);
  const double u = (a - h) / (K / 2.0 - h);
  const double q = h * h + n * (K / 2.0 - h) * (u + u * u / 2.0 - u * u * u * u + 2.0 * std::pow(u, 5) / 5.0);
  return q / (h * h);
}

template <typename T>
int dev_alloc(pnp_plan* p, T** ptr, size_t count) {
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(PNP_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  p->device_bytes += (int64_t)(count * sizeof(T));
  return PNP_OK;
}

}  // namespace

int build_units(pnp_plan* p) {
  ++p->epoch;  // a captured FB graph launches the old work list: it must be captured again
  std::vector<Unit> units;
  std::vector<Chunk> chunks;
  std::vector<uint8_t> runs;
  const int64_t M = p->M;
  auto nnz_of = [&](int64_t i) { return p->h_rowptr[i + 1] - p->h_rowptr[i]; };
  std::vector<int64_t> stack_units(p->nstacks + 1, 0);
  int64_t i = 0;
  while (i < M) {
    const int32_t key = p->h_key[i];
    Unit u;
    u.chunk_begin = (long long)chunks.size();
    u.tile = (int)((key % p->nkeys) / p->nblocks);
    stack_units[key / p->nkeys + 1] = (int64_t)units.size() + 1;  // units of a stack are consecutive
    int64_t unit_taps = 0;
    while (i < M && p->h_key[i] == key && (unit_taps == 0 || unit_taps + nnz_of(i) <= p->unit_nnz)) {
      Chunk ch;
      ch.row_begin = i;
      ch.tap_begin = p->h_rowptr[i];
      int nr = 0;
      int64_t nt = 0;
      const int64_t row_nnz = nnz_of(i);  // every row of a chunk has the same support
      while (i < M && p->h_key[i] == key && nnz_of(i) == row_nnz && nr < CHUNK_ROWS &&
             nt + nnz_of(i) <= CHUNK_TAPS && (unit_taps + nt == 0 || unit_taps + nt + nnz_of(i) <= p->unit_nnz)) {
        nt += nnz_of(i);
        ++nr;
        ++i;
      }
      if (nr == 0) return fail(PNP_ERR_INVALID_ARG, "internal: a row does not fit one gridding chunk");
      ch.nrows = nr;
      ch.ntaps = (int)nt;
      ch.nn = (int)row_nnz;
      // runs: consecutive rows whose first tap is the same cell share their whole tap window
      // (same support), at most run_max rows each
      ch.run_begin = (long long)runs.size();
      int last = 0;
      for (int q = 0; q < nr; ++q)
        if (q == 0 || p->h_start[ch.row_begin + q] != p->h_start[ch.row_begin + q - 1] || q - last == p->run_max) {
          runs.push_back((uint8_t)q);
          last = q;
        }
      ch.nruns = (int)((long long)runs.size() - ch.run_begin);
      runs.push_back((uint8_t)nr);
      chunks.push_back(ch);
      unit_taps += nt;
    }
    u.nchunks = (int)((long long)chunks.size() - u.chunk_begin);
    units.push_back(u);
  }
  if (p->d_units) {
    cudaFree(p->d_units);
    p->device_bytes -= p->n_units * (int64_t)sizeof(Unit);
    p->d_units = nullptr;
  }
  if (p->d_chunks) {
    cudaFree(p->d_chunks);
    p->device_bytes -= p->n_chunks * (int64_t)sizeof(Chunk);
    p->d_chunks = nullptr;
  }
  if (p->d_runs) {
    cudaFree(p->d_runs);
    p->device_bytes -= p->n_runs + 32;
    p->d_runs = nullptr;
  }
  p->n_units = (int64_t)units.size();
  p->n_chunks = (int64_t)chunks.size();
  for (int s = 0; s < p->nstacks; ++s)  // empty stacks start and end where the previous one ends
    stack_units[s + 1] = std::max(stack_units[s + 1], stack_units[s]);
  p->h_stack_units.swap(stack_units);
  if (int rc = dev_alloc(p, &p->d_units, units.size())) return rc;
  if (int rc = dev_alloc(p, &p->d_chunks, chunks.size())) return rc;
  p->n_runs = (int64_t)runs.size();
  runs.resize(runs.size() + 32, 0);  // the stage copies 16-byte windows around each list
  if (int rc = dev_alloc(p, &p->d_runs, runs.size())) return rc;
  PNP_CUDA(cudaMemcpy(p->d_runs, runs.data(), runs.size(), cudaMemcpyHostToDevice));
  if (!units.empty()) {
    PNP_CUDA(cudaMemcpy(p->d_units, units.data(), units.size() * sizeof(Unit), cudaMemcpyHostToDevice));
    PNP_CUDA(cudaMemcpy(p->d_chunks, chunks.data(), chunks.size() * sizeof(Chunk), cudaMemcpyHostToDevice));
  }
  return PNP_OK;
}

int plan_build(pnp_plan* p, const double* uvw, const int8_t* Jrow, const int32_t* block, const int32_t* stack,
               const double* row_scale) {
  const int n = p->n, K = p->K, J = p->J;
  const int64_t M = p->M;
  p->beta = kb_beta(J, (double)K / n);

  // grid correction and twiddles
  std::vector<float> cinv(n);
  for (int a = 0; a < n; ++a) cinv[a] = (float)(1.0 / kb_correction(a - n / 2, J, p->beta, K));
  std::vector<float2> tw(K);
  for (int j = 0; j < K; ++j) {
    const double ang = -2.0 * M_PI * j / K;
    tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }

  // per-row geometry, keys
  const int ntc = (K + p->tile - 1) / p->tile;
  p->ntc = ntc;
  std::vector<RowGeom> geom(M);
  std::vector<int32_t> key(M);
  std::vector<uint16_t> startc(M);  // first tap's cell within its tile
  int Jmax = J;
  double amax = 0.0;
  for (int64_t m = 0; m < M; ++m) {
    RowGeom g;
    g.kap0 = uvw[3 * m] * (K / (2.0 * M_PI));
    g.kap1 = uvw[3 * m + 1] * (K / (2.0 * M_PI));
    if (stack && (stack[m] < 0 || stack[m] >= p->nstacks))
      return fail(PNP_ERR_INVALID_ARG, "stack id out of range at row " + std::to_string(m));
    // w-stacking (App. E): the row kernel carries only the offset from its stack's centre
    const double wres = uvw[3 * m + 2] - (stack ? p->w_centres[stack[m]] : 0.0);
    g.a = p->dl > 0 ? wres * p->dl * p->dl : 0.0;
    g.J = Jrow ? Jrow[m] : J;
    g.d = row_scale ? row_scale[m] : 1.0;
    if (!(g.d > 0.0) || !std::isfinite(g.d))
      return fail(PNP_ERR_INVALID_ARG, "row scale must be finite and > 0 at row " + std::to_string(m));
    if (!(std::isfinite(g.kap0) && std::isfinite(g.kap1) && std::isfinite(g.a)))
      return fail(PNP_ERR_INVALID_ARG, "non-finite uvw at row " + std::to_string(m));
    if (std::fabs(uvw[3 * m]) > 4 * M_PI || std::fabs(uvw[3 * m + 1]) > 4 * M_PI)
      return fail(PNP_ERR_INVALID_ARG, "omega outside [-4 pi, 4 pi] at row " + std::to_string(m));
    if (g.J < J || g.J > 16)
      return fail(PNP_ERR_INVALID_ARG, "J_per_row must lie in [J, 16]; row " + std::to_string(m));
    if (block && (block[m] < 0 || block[m] >= p->nblocks))
      return fail(PNP_ERR_INVALID_ARG, "block id out of range at row " + std::to_string(m));
    g.s0 = (int)std::floor(g.kap0 - 0.5 * g.J) + 1;
    g.s1 = (int)std::floor(g.kap1 - 0.5 * g.J) + 1;
    const int f0 = ((g.s0 % K) + K) % K, f1 = ((g.s1 % K) + K) % K;
    key[m] = ((f1 / p->tile) * ntc + (f0 / p->tile)) * p->nblocks + (block ? block[m] : 0);
    startc[m] = (uint16_t)((f1 % p->tile) * p->tile + (f0 % p->tile));
    Jmax = std::max(Jmax, g.J);
    amax = std::max(amax, std::fabs(g.a));
    geom[m] = g;
  }
  p->Jmax = Jmax;
  p->slots = Jmax * Jmax <= 64 ? 2 : (Jmax * Jmax <= 128 ? 4 : 8);
  {
    std::vector<int64_t> rows_per_J(17, 0);
    for (int64_t m = 0; m < M; ++m) rows_per_J[geom[m].J]++;
    if (int rc = gridding_pitch(p, rows_per_J.data())) return rc;
  }

  // stable LSD counting sort: by the first tap's cell in the tile, then by support J, then by
  // (tile, block) key, so that rows of one tile come out grouped by J (each gridding chunk then
  // holds rows of a single J) and, within that, rows with the same tap window are adjacent
  // (the gridding pass gathers and scatters such a run once)
  std::vector<int32_t> by_j(M);
  {
    const int nc = p->tile * p->tile;
    std::vector<int64_t> cc(nc + 1, 0);
    for (int64_t m = 0; m < M; ++m) cc[startc[m] + 1]++;
    for (int c = 0; c < nc; ++c) cc[c + 1] += cc[c];
    std::vector<int32_t> by_c(M);
    for (int64_t m = 0; m < M; ++m) by_c[cc[startc[m]]++] = (int32_t)m;
    std::vector<int64_t> cj(18, 0);
    for (int64_t m = 0; m < M; ++m) cj[geom[m].J + 1]++;
    for (int j = 0; j < 17; ++j) cj[j + 1] += cj[j];
    for (int64_t i = 0; i < M; ++i) {
      const int32_t m = by_c[i];
      by_j[cj[geom[m].J]++] = m;
    }
  }
  const int64_t nkeys = (int64_t)ntc * ntc * p->nblocks;
  if (nkeys * p->nstacks > INT32_MAX) return fail(PNP_ERR_UNSUPPORTED, "too many (stack, tile, block) keys");
  p->nkeys = nkeys;
  std::vector<int64_t> cnt(nkeys + 1, 0);
  for (int64_t m = 0; m < M; ++m) cnt[key[m] + 1]++;
  for (int64_t k = 0; k < nkeys; ++k) cnt[k + 1] += cnt[k];
  p->h_perm.assign(M, 0);
  p->h_inv.assign(M, 0);
  for (int64_t i = 0; i < M; ++i) {
    const int32_t m = by_j[i];
    p->h_perm[cnt[key[m]]++] = m;
  }
  if (stack && p->nstacks > 1) {  // most significant: the w-stack
    std::vector<int64_t> cs(p->nstacks + 1, 0);
    for (int64_t m = 0; m < M; ++m) cs[stack[m] + 1]++;
    for (int s = 0; s < p->nstacks; ++s) cs[s + 1] += cs[s];
    for (int64_t i = 0; i < M; ++i) {
      const int32_t m = p->h_perm[i];
      by_j[cs[stack[m]]++] = m;
    }
    p->h_perm.swap(by_j);
  }
  for (int64_t i = 0; i < M; ++i) p->h_inv[p->h_perm[i]] = (int32_t)i;
  std::vector<int32_t>().swap(by_j);
  std::vector<RowGeom> sgeom(M);
  p->h_key.assign(M, 0);
  p->h_start.assign(M, 0);
  p->h_rowptr.assign(M + 1, 0);
  for (int64_t i = 0; i < M; ++i) {
    const int64_t m = p->h_perm[i];
    sgeom[i] = geom[m];
    p->h_key[i] = (int32_t)((stack ? (int64_t)stack[m] : 0) * nkeys + key[m]);
    p->h_start[i] = startc[m];
    p->h_rowptr[i + 1] = p->h_rowptr[i] + (int64_t)geom[m].J * geom[m].J;
  }
  p->nnz = p->h_rowptr[M];
  // uv support of G: per grid row k1 the largest centred |k0| of its taps, and the band of rows
  std::vector<int> rowh(K, -1);
  {
    auto centred = [K](int k) {
      k = ((k % K) + K) % K;
      return k < K / 2 ? k : k - K;
    };
    for (int64_t m = 0; m < M; ++m) {
      const RowGeom& g = geom[m];
      const int c0 = centred(g.s0), c0e = c0 + g.J - 1;  // the row's k0 taps, centred (may wrap)
      const int hm = c0e >= K / 2 ? K / 2 : std::max(std::abs(c0), std::abs(c0e));
      for (int t = 0; t < g.J; ++t) {
        int& h = rowh[((g.s1 + t) % K + K) % K];
        h = std::max(h, hm);
      }
    }
    p->band = -1;
    for (int k = 0; k < K; ++k)
      if (rowh[k] >= 0) p->band = std::max(p->band, std::abs(centred(k)));
  }
  std::vector<RowGeom>().swap(geom);

  // w-kernel series: b = bscale * a, qn in [0, qmax], centred at c0 = qmax / 2
  const double h = n / 2.0;
  const double bscale = M_PI * h * h;
  const double qmax = chirp_q(K / 2.0, n, K), c0 = qmax / 2.0;
  const int D = (Jmax + J + 1) / 2 + 1;
  if (D > MAX_D) return fail(PNP_ERR_UNSUPPORTED, "kernel support too large");
  int nterms = 1;
  {
    const double x = bscale * amax * c0;  // largest |b (qn - c0)|
    double term = 1.0;
    while (nterms < MAX_TERMS) {
      term *= x / nterms;
      ++nterms;
      if (term < 1e-18 && nterms > x) break;
    }
    if (nterms >= MAX_TERMS && x > 0)
      return fail(PNP_ERR_UNSUPPORTED, "w-term too large for the w-kernel series (increase K or reduce dl)");
    if (amax == 0.0) nterms = 1;
  }
  std::vector<double> mu((size_t)nterms * (2 * D + 1), 0.0);
  if (amax > 0.0) {
    std::vector<double> qc(K);
    for (int j = 0; j < K; ++j) qc[j] = chirp_q(j - K / 2, n, K) - c0;
    for (int d = -D; d <= D; ++d) {
      std::vector<double> pw(K, 1.0);
      std::vector<double> cs(K);
      for (int j = 0; j < K; ++j) cs[j] = std::cos(2.0 * M_PI * d * (double)(j - K / 2) / K);
      for (int t = 0; t < nterms; ++t) {
        double s = 0.0;
        for (int j = 0; j < K; ++j) {
          s += pw[j] * cs[j];
          pw[j] *= qc[j];
        }
        mu[(size_t)t * (2 * D + 1) + (d + D)] = s / K;
      }
    }
  }

  // device buffers
  const size_t KK = (size_t)K * K;
  if (int rc = dev_alloc(p, &p->d_cinv, n)) return rc;
  if (int rc = dev_alloc(p, &p->d_tw, K)) return rc;
  if (int rc = dev_alloc(p, &p->d_twp, TWP_ENTRIES)) return rc;
  if (int rc = dev_alloc(p, &p->d_gridA, KK)) return rc;
  if (int rc = dev_alloc(p, &p->d_gridB, KK)) return rc;
  if (int rc = dev_alloc(p, &p->d_gridB_lo, KK)) return rc;
  if (int rc = dev_alloc(p, &p->d_tmp, (size_t)K * n)) return rc;
  if (int rc = dev_alloc(p, &p->d_rowh, (size_t)K)) return rc;
  const size_t wbytes = p->wdtype == PNP_W_BF16C ? 4 : 8;
  {
    void* w = nullptr;
    cudaError_t e = cudaMalloc(&w, (p->nnz + TAP_PAD) * wbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PNP_ERR_OOM, "cudaMalloc of G weights (" + std::to_string(p->nnz * wbytes) + " bytes) failed");
    }
    p->d_w = w;
    p->device_bytes += (int64_t)((p->nnz + TAP_PAD) * wbytes);
    PNP_CUDA(cudaMemset(w, 0, (p->nnz + TAP_PAD) * wbytes));
  }
  if (int rc = dev_alloc(p, &p->d_cells, (size_t)p->nnz + TAP_PAD)) return rc;
  if (int rc = dev_alloc(p, &p->d_rowptr, (size_t)M + 1 + ROW_PAD)) return rc;
  if (int rc = dev_alloc(p, &p->d_perm, (size_t)M)) return rc;
  if (int rc = dev_alloc(p, &p->d_ysorted, (size_t)M + ROW_PAD)) return rc;
  PNP_CUDA(cudaMemset(p->d_cells, 0, ((size_t)p->nnz + TAP_PAD) * sizeof(uint16_t)));
  PNP_CUDA(cudaMemset(p->d_ysorted, 0, ((size_t)M + ROW_PAD) * sizeof(float2)));
  if (int rc = dev_alloc(p, &p->d_acc, 8)) return rc;
  if (int rc = dev_alloc(p, &p->d_status, 4)) return rc;
  for (int i = 0; i < 3; ++i)
    if (int rc = dev_alloc(p, &p->d_img[i], (size_t)n * n)) return rc;
  if (p->nstacks > 1) {
    // Z_s of stack s: the paraxial w-modulation of the stack centre, separable per axis
    std::vector<float2> ch((size_t)p->nstacks * n);
    for (int s = 0; s < p->nstacks; ++s) {
      const double as = p->w_centres[s] * p->dl * p->dl;
      for (int a = 0; a < n; ++a) {
        const double q = (double)(a - n / 2), ph = M_PI * as * q * q;
        ch[(size_t)s * n + a] = make_float2((float)std::cos(ph), (float)std::sin(ph));
      }
    }
    if (int rc = dev_alloc(p, &p->d_chirp, ch.size())) return rc;
    if (int rc = dev_alloc(p, &p->d_gacc, (size_t)n * n)) return rc;
    PNP_CUDA(cudaMemcpy(p->d_chirp, ch.data(), ch.size() * sizeof(float2), cudaMemcpyHostToDevice));
  }
  PNP_CUDA(cudaMemcpy(p->d_cinv, cinv.data(), n * sizeof(float), cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemcpy(p->d_tw, tw.data(), K * sizeof(float2), cudaMemcpyHostToDevice));
  {
    std::vector<float2> twp(TWP_ENTRIES);
    for (int q = 1, off = 0; q <= 2; off += 16 * (1 << (4 * q)), ++q) {
      const int Ns = 1 << (4 * q);
      for (int r = 0; r < 16; ++r)
        for (int k = 0; k < Ns; ++k) {
          const double ang = -2.0 * M_PI * (double)(r * k) / (16.0 * Ns);
          twp[off + r * Ns + k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        }
    }
    PNP_CUDA(cudaMemcpy(p->d_twp, twp.data(), TWP_ENTRIES * sizeof(float2), cudaMemcpyHostToDevice));
  }
  // the forward grid outside G's support is never written (the split passes prune it) and reads as 0
  PNP_CUDA(cudaMemset(p->d_gridA, 0, KK * sizeof(float2)));
  PNP_CUDA(cudaMemset(p->d_gridB, 0, KK * sizeof(float2)));
  PNP_CUDA(cudaMemset(p->d_gridB_lo, 0, KK * sizeof(__nv_bfloat162)));
  PNP_CUDA(cudaMemcpy(p->d_rowh, rowh.data(), K * sizeof(int), cudaMemcpyHostToDevice));
  PNP_CUDA(cudaMemset(p->d_acc, 0, 8 * sizeof(double)));
  PNP_CUDA(cudaMemset(p->d_status, 0, 4 * sizeof(int)));
  {
    std::vector<int64_t> rp(p->h_rowptr);
    rp.resize(M + 1 + ROW_PAD, p->nnz);  // padding entries repeat nnz
    PNP_CUDA(cudaMemcpy(p->d_rowptr, rp.data(), rp.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  }
  if (M) PNP_CUDA(cudaMemcpy(p->d_perm, p->h_perm.data(), M * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (M && row_scale) {  // the data weights in the caller's row order, for pnp_plan_scale_data
    std::vector<float> d(M);
    for (int64_t m = 0; m < M; ++m) d[m] = (float)row_scale[m];
    if (int rc = dev_alloc(p, &p->d_rowscale, (size_t)M)) return rc;
    PNP_CUDA(cudaMemcpy(p->d_rowscale, d.data(), M * sizeof(float), cudaMemcpyHostToDevice));
  }

  // build G rows on the GPU
  if (M) {
    RowGeom* d_geom = nullptr;
    double* d_mu = nullptr;
    if (cudaMalloc(&d_geom, M * sizeof(RowGeom)) != cudaSuccess ||
        cudaMalloc(&d_mu, mu.size() * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_geom);
      return fail(PNP_ERR_OOM, "plan build scratch allocation failed");
    }
    PNP_CUDA(cudaMemsetAsync(p->d_status + 3, 0, sizeof(int), p->stream));
    PNP_CUDA(cudaMemcpy(d_geom, sgeom.data(), M * sizeof(RowGeom), cudaMemcpyHostToDevice));
    PNP_CUDA(cudaMemcpy(d_mu, mu.data(), mu.size() * sizeof(double), cudaMemcpyHostToDevice));
    BuildArgs A{};
    A.M = M;
    A.K = K;
    A.logK = p->logK;
    A.J = J;
    A.beta = p->beta;
    A.bscale = bscale;
    A.c0 = c0;
    A.nterms = nterms;
    A.D = D;
    A.mu = d_mu;
    A.geom = d_geom;
    A.rowptr = p->d_rowptr;
    A.w = p->d_w;
    A.cells = p->d_cells;
    A.T = p->tile;
    A.S = p->tile + p->Jmax - 1;
    A.P = p->pitch;
    A.err = p->d_status + 3;
    A.bf16 = p->wdtype == PNP_W_BF16C;
    build_rows<<<(unsigned)((M + 7) / 8), 256, 0, p->stream>>>(A);
    cudaError_t e = cudaGetLastError();
    g_launches.fetch_add(1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    cudaFree(d_geom);
    cudaFree(d_mu);
    if (e != cudaSuccess) return fail(PNP_ERR_CUDA, std::string("build_rows: ") + cudaGetErrorString(e));
    int err = 0;
    PNP_CUDA(cudaMemcpy(&err, p->d_status + 3, sizeof(int), cudaMemcpyDeviceToHost));
    PNP_CUDA(cudaMemset(p->d_status + 3, 0, sizeof(int)));
    if (err) return fail(PNP_ERR_INVALID_ARG, "internal: a tap of G falls outside its row's gridding region");
  }
  return build_units(p);
}

int export_rows_impl(const pnp_plan* p, const int64_t* rows, int64_t nrows, int64_t* offsets,
                     float* weights, int32_t* cols) {
  std::vector<int64_t> src(4 * nrows), dst(nrows);
  offsets[0] = 0;
  for (int64_t i = 0; i < nrows; ++i) {
    if (rows[i] < 0 || rows[i] >= p->M) return fail(PNP_ERR_INVALID_ARG, "export row index out of range");
    const int64_t s = p->h_inv[rows[i]];
    const int tile = (int)((p->h_key[s] % p->nkeys) / p->nblocks);
    src[4 * i] = p->h_rowptr[s];
    src[4 * i + 1] = p->h_rowptr[s + 1] - p->h_rowptr[s];
    src[4 * i + 2] = (int64_t)(tile / p->ntc) * p->tile;
    src[4 * i + 3] = (int64_t)(tile % p->ntc) * p->tile;
    dst[i] = offsets[i];
    offsets[i + 1] = offsets[i] + src[4 * i + 1];
  }
  if (!weights || !cols || nrows == 0) return PNP_OK;
  const int64_t total = offsets[nrows];
  int64_t *d_src = nullptr, *d_dst = nullptr;
  float2* d_w = nullptr;
  int32_t* d_c = nullptr;
  if (cudaMalloc(&d_src, 4 * nrows * sizeof(int64_t)) || cudaMalloc(&d_dst, nrows * sizeof(int64_t)) ||
      cudaMalloc(&d_w, total * sizeof(float2)) || cudaMalloc(&d_c, total * sizeof(int32_t))) {
    cudaGetLastError();
    cudaFree(d_src);
    cudaFree(d_dst);
    cudaFree(d_w);
    return fail(PNP_ERR_OOM, "export scratch allocation failed");
  }
  int rc = PNP_OK;
  cudaError_t e = cudaMemcpy(d_src, src.data(), 4 * nrows * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_dst, dst.data(), nrows * sizeof(int64_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    export_rows<<<(unsigned)nrows, 128, 0, p->stream>>>(d_src, d_dst, nrows, p->d_w, p->d_cells, p->pitch,
                                                         p->wdtype == PNP_W_BF16C, p->logK, d_w, d_c);
    g_launches.fetch_add(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e == cudaSuccess) e = cudaMemcpy(weights, d_w, total * sizeof(float2), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(cols, d_c, total * sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = fail(PNP_ERR_CUDA, std::string("export_rows: ") + cudaGetErrorString(e));
  cudaFree(d_src);
  cudaFree(d_dst);
  cudaFree(d_w);
  cudaFree(d_c);
  return rc;
}

}  // namespace pnp
