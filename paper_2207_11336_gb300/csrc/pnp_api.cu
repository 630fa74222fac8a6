// C ABI entry points (include/pnp.h): plan lifetime, the operator calls of
// Eq. 1 and App. A, power iteration, denoisers and the PnP-FB loop of Eq. fb.
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace pnp {

static thread_local std::string t_err;
std::atomic<int64_t> g_launches{0};
static std::atomic<uint64_t> g_den_serial{0};

void set_error(const std::string& msg) { t_err = msg; }
int fail(int code, const std::string& msg) {
  t_err = msg;
  return code;
}

int export_rows_impl(const pnp_plan* p, const int64_t* rows, int64_t nrows, int64_t* offsets,
                     float* weights, int32_t* cols);
int norm2_dev(cudaStream_t s, const float* v, int64_t count, double* acc);
int fill_image(cudaStream_t s, float* out, int64_t count, float v);

int stage_begin(pnp_plan* p, int stage, cudaEvent_t* a) {
  *a = nullptr;
  if (!p->timing) return PNP_OK;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  PNP_CUDA(cudaStreamIsCapturing(p->stream, &cs));
  if (cs != cudaStreamCaptureStatusNone) return PNP_OK;
  PNP_CUDA(cudaEventCreate(a));
  PNP_CUDA(cudaEventRecord(*a, p->stream));
  (void)stage;
  return PNP_OK;
}

int stage_end(pnp_plan* p, int stage, cudaEvent_t a) {
  if (!a) return PNP_OK;
  cudaEvent_t b;
  PNP_CUDA(cudaEventCreate(&b));
  PNP_CUDA(cudaEventRecord(b, p->stream));
  p->timed.push_back({stage, a, b});
  return PNP_OK;
}

namespace {

void clear_timing(pnp_plan* p) {
  for (auto& t : p->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  p->timed.clear();
}

void free_plan(pnp_plan* p) {
  if (!p) return;
  clear_timing(p);
  cudaFree(p->d_cinv);
  cudaFree(p->d_tw);
  cudaFree(p->d_twp);
  cudaFree(p->d_gridA);
  cudaFree(p->d_gridB);
  cudaFree(p->d_gridB_lo);
  cudaFree(p->d_tmp);
  cudaFree(p->d_w);
  cudaFree(p->d_cells);
  cudaFree(p->d_runs);
  cudaFree(p->d_rowptr);
  cudaFree(p->d_perm);
  cudaFree(p->d_ysorted);
  cudaFree(p->d_units);
  cudaFree(p->d_chunks);
  cudaFree(p->d_acc);
  cudaFree(p->d_status);
  if (p->cstream) cudaStreamDestroy(p->cstream);
  for (auto& e : p->ev_join)
    if (e) cudaEventDestroy(e);
  for (float* im : p->d_img) cudaFree(im);
  cudaFree(p->d_chirp);
  cudaFree(p->d_gacc);
  cudaFree(p->d_H);
  cudaFree(p->d_dirty);
  cudaFree(p->d_rowscale);
  cudaFree(p->d_rowh);
  if (p->graph.exec) cudaGraphExecDestroy(p->graph.exec);
  delete p;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int read_acc(pnp_plan* p, double* h, int count) {
  PNP_CUDA(cudaMemcpyAsync(h, p->d_acc, count * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  return PNP_OK;
}

// Re{Phi^H (Phi xf - y)} (or Re{Phi^H Phi xf} without y) through epilogue `epi`, summed over the
// plan's w-stacks (Eq. phidagphi): per stack the forward FFT with Z_s, the fused gridding pass
// over the stack's rows and the adjoint FFT; all stacks share one pair of grids.
int normal_pass(pnp_plan* p, const float2* y_sorted, const float* xf, int epi, const float* xe, float* out,
                float gamma, float t, bool holo_ok) {
  if (holo_ok && p->holo) {  // App. E, Eq. phidagphi: H F Z x - G^H y without reading G
    if (int rc = fft_forward(p, xf, 0)) return rc;
    if (int rc = holo_apply_pass(p, y_sorted != nullptr)) return rc;
    return fft_adjoint(p, epi, xe, out, gamma, t, 0);
  }
  for (int s = 0; s < p->nstacks; ++s) {
    if (int rc = fft_forward(p, xf, s)) return rc;
    if (int rc = gridding_pass(p, G_FUSED, y_sorted, nullptr, s)) return rc;
    if (int rc = fft_adjoint(p, epi, xe, out, gamma, t, s)) return rc;
  }
  return PNP_OK;
}

// One FB iteration x_next = D(x_cur - gamma grad f(x_cur)); FP64 norms land in acc[0..1].
// pos: the denoiser ends with the positivity projection.
int fb_iteration(pnp_plan* p, pnp_den* d, const float* cur, float* nxt, double gamma, bool pos) {
  const float2* ys = reinterpret_cast<const float2*>(p->d_ysorted);
  if (d->kind == PNP_DEN_HAAR)
    return normal_pass(p, ys, cur, pos ? EPI_HAAR : EPI_HAAR_NOPOS, cur, nxt, (float)gamma, (float)d->t, true);
  if (int rc = normal_pass(p, ys, cur, EPI_GRAD, cur, p->d_img[1], (float)gamma, 0.f, true)) return rc;
  if (d->kind == PNP_DEN_SARA) return sara_denoise(d, p->stream, p->d_img[1], nxt, p->n, p->d_acc, cur, pos);
  return cnn_denoise(d, p->stream, p->d_img[1], nxt, p->n, p->d_acc, cur, pos);
}

// Replays two FB iterations (x -> work -> x) as one CUDA graph on the plan's private stream,
// joined to the caller's stream with events.  The instantiated graph is kept in the plan and
// reused by later pnp_fb_run calls while the denoiser, the iterate buffer, gamma, the
// positivity choice, the holographic switch and the gridding work list are unchanged.
struct GraphRunner {
  pnp_plan* p;
  pnp_den* d;
  float** buf;
  double gamma;
  bool pos;
  GraphRunner(pnp_plan* p_, pnp_den* d_, float** b, double g, bool ps) : p(p_), d(d_), buf(b), gamma(g), pos(ps) {}
  bool cached() const {
    const auto& c = p->graph;
    return c.exec && c.den_serial == d->serial && c.x == buf[0] && c.gamma == gamma && c.epi == (pos ? 1 : 0) &&
           c.holo == p->holo && c.epoch == p->epoch;
  }
  int capture() {
    if (p->graph.exec) {
      cudaGraphExecDestroy(p->graph.exec);
      p->graph.exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    const int64_t before = g_launches.load();
    PNP_CUDA(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    int rc = fb_iteration(p, d, buf[0], buf[1], gamma, pos);
    if (!rc) rc = fb_iteration(p, d, buf[1], buf[0], gamma, pos);
    cudaError_t e = cudaStreamEndCapture(p->stream, &g);
    const int64_t kernels = g_launches.load() - before;
    g_launches.fetch_sub(kernels);
    if (!rc && e != cudaSuccess) {
      cudaGetLastError();
      rc = fail(PNP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    if (!rc) {
      e = cudaGraphInstantiate(&exec, g, 0);
      if (e != cudaSuccess) {
        cudaGetLastError();
        exec = nullptr;
        rc = fail(PNP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
    }
    if (g) cudaGraphDestroy(g);
    if (!rc) {
      auto& c = p->graph;
      c.exec = exec;
      c.kernels = kernels;
      c.den_serial = d->serial;
      c.x = buf[0];
      c.gamma = gamma;
      c.epi = pos ? 1 : 0;
      c.holo = p->holo;
      c.epoch = p->epoch;
    }
    return rc;
  }
  int run_pairs(int pairs) {
    cudaStream_t user = p->stream;
    PNP_CUDA(cudaEventRecord(p->ev_join[0], user));
    PNP_CUDA(cudaStreamWaitEvent(p->cstream, p->ev_join[0], 0));
    p->stream = p->cstream;
    int rc = cached() ? PNP_OK : capture();
    for (int i = 0; i < pairs && rc == PNP_OK; ++i) {
      cudaError_t e = cudaGraphLaunch(p->graph.exec, p->stream);
      if (e != cudaSuccess) {
        cudaGetLastError();
        rc = fail(PNP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
      } else {
        g_launches.fetch_add(p->graph.kernels);
      }
    }
    p->stream = user;
    if (cudaEventRecord(p->ev_join[1], p->cstream) != cudaSuccess ||
        cudaStreamWaitEvent(user, p->ev_join[1], 0) != cudaSuccess) {
      cudaGetLastError();
      if (rc == PNP_OK) rc = fail(PNP_ERR_CUDA, "stream join failed");
    }
    return rc;
  }
};

}  // namespace
}  // namespace pnp

using namespace pnp;

extern "C" {

const char* pnp_last_error(void) { return t_err.c_str(); }

int64_t pnp_kernel_launch_count(void) { return g_launches.load(); }

int pnp_plan_create(pnp_plan** plan, int n, int K, int64_t M, const double* uvw_host, double dl,
                    const int8_t* J_per_row_host, int J, int weight_dtype, const int32_t* block_host,
                    int nblocks, void* stream) {
  return pnp_plan_create_stacked(plan, n, K, M, uvw_host, dl, J_per_row_host, J, weight_dtype, block_host,
                                 nblocks, nullptr, 1, nullptr, stream);
}

int pnp_plan_create_stacked(pnp_plan** plan, int n, int K, int64_t M, const double* uvw_host, double dl,
                            const int8_t* J_per_row_host, int J, int weight_dtype, const int32_t* block_host,
                            int nblocks, const int32_t* stack_host, int nstacks, const double* w_centres_host,
                            void* stream) {
  pnp_plan_desc d{};
  d.n = n;
  d.K = K;
  d.M = M;
  d.uvw_host = uvw_host;
  d.dl = dl;
  d.J_per_row_host = J_per_row_host;
  d.J = J;
  d.weight_dtype = weight_dtype;
  d.block_host = block_host;
  d.nblocks = nblocks;
  d.stack_host = stack_host;
  d.nstacks = nstacks;
  d.w_centres_host = w_centres_host;
  d.stream = stream;
  if (nblocks < 1) return fail(PNP_ERR_INVALID_ARG, "nblocks must be >= 1");
  if (nstacks < 1 || nstacks > 64) return fail(PNP_ERR_INVALID_ARG, "nstacks must lie in [1, 64]");
  return pnp_plan_create_desc(plan, &d);
}

int pnp_plan_create_desc(pnp_plan** plan, const pnp_plan_desc* desc) {
  if (!plan) return fail(PNP_ERR_INVALID_ARG, "plan pointer is NULL");
  *plan = nullptr;
  if (!desc) return fail(PNP_ERR_INVALID_ARG, "plan descriptor is NULL");
  const int n = desc->n, K = desc->K, J = desc->J, weight_dtype = desc->weight_dtype;
  const int64_t M = desc->M;
  const double dl = desc->dl;
  const double* uvw_host = desc->uvw_host;
  const int nblocks = desc->nblocks > 0 ? desc->nblocks : 1;
  const int nstacks = desc->nstacks > 0 ? desc->nstacks : 1;
  const int32_t* stack_host = desc->stack_host;
  const double* w_centres_host = desc->w_centres_host;
  if (n < 8 || (n & 1)) return fail(PNP_ERR_INVALID_ARG, "n must be even and >= 8");
  if (!is_pow2(K) || K < 64 || K > 16384) return fail(PNP_ERR_INVALID_ARG, "K must be a power of two in [64, 16384]");
  if (n > K / 2) return fail(PNP_ERR_INVALID_ARG, "n must be <= K/2 (at least 2x oversampling)");
  if (J < 2 || J > 14) return fail(PNP_ERR_INVALID_ARG, "J must lie in [2, 14]");
  if (M < 0 || M > INT32_MAX) return fail(PNP_ERR_INVALID_ARG, "M must lie in [0, 2^31)");
  if (M > 0 && !uvw_host) return fail(PNP_ERR_INVALID_ARG, "uvw is NULL");
  if (weight_dtype != PNP_W_C64 && weight_dtype != PNP_W_BF16C) return fail(PNP_ERR_INVALID_ARG, "bad weight_dtype");
  if (!(dl >= 0.0) || !std::isfinite(dl)) return fail(PNP_ERR_INVALID_ARG, "dl must be finite and >= 0");
  if (nstacks > 64) return fail(PNP_ERR_INVALID_ARG, "nstacks must lie in [1, 64]");
  if (nstacks > 1 && (!stack_host && M > 0)) return fail(PNP_ERR_INVALID_ARG, "stack ids are NULL");
  if (nstacks > 1 && !w_centres_host) return fail(PNP_ERR_INVALID_ARG, "w_centres is NULL");
  if (nstacks > 1 && dl == 0.0) return fail(PNP_ERR_INVALID_ARG, "w-stacking needs dl > 0");
  for (int s = 0; w_centres_host && s < nstacks; ++s)
    if (!std::isfinite(w_centres_host[s])) return fail(PNP_ERR_INVALID_ARG, "non-finite w centre");
  pnp_plan* p = new pnp_plan();
  p->nstacks = nstacks;
  p->w_centres.assign(nstacks, 0.0);
  if (w_centres_host) p->w_centres.assign(w_centres_host, w_centres_host + nstacks);
  p->n = n;
  p->K = K;
  p->logK = 0;
  while ((1 << p->logK) < K) ++p->logK;
  p->M = M;
  p->J = J;
  p->dl = dl;
  p->wdtype = weight_dtype;
  p->nblocks = nblocks;
  p->stream = reinterpret_cast<cudaStream_t>(desc->stream);
  p->tile = K >= 128 ? 32 : 16;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(PNP_ERR_CUDA, "no CUDA device available");
  }
  if (cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_plan(p);
    return fail(PNP_ERR_CUDA, "stream/event creation failed");
  }
  int rc = plan_build(p, uvw_host, desc->J_per_row_host, desc->block_host, nstacks > 1 ? stack_host : nullptr,
                      desc->row_scale_host);
  if (rc != PNP_OK) {
    std::string keep = t_err;
    free_plan(p);
    t_err = keep;
    return rc;
  }
  *plan = p;
  return PNP_OK;
}

int pnp_plan_scale_data(pnp_plan* p, const float* y_in, float* y_out) {
  if (!p || (p->M > 0 && (!y_in || !y_out))) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  if (p->M == 0) return PNP_OK;
  if (!p->d_rowscale) {
    if (y_in != y_out)
      PNP_CUDA(cudaMemcpyAsync(y_out, y_in, (size_t)p->M * sizeof(float2), cudaMemcpyDeviceToDevice, p->stream));
    return PNP_OK;
  }
  return row_scale_c64(p->stream, reinterpret_cast<const float2*>(y_in), p->d_rowscale,
                       reinterpret_cast<float2*>(y_out), p->M);
}

void pnp_plan_destroy(pnp_plan* plan) {
  if (plan) cudaStreamSynchronize(plan->stream);
  free_plan(plan);
}

int pnp_plan_get_info(const pnp_plan* p, pnp_plan_info* info) {
  if (!p || !info) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  info->n = p->n;
  info->K = p->K;
  info->J = p->J;
  info->weight_dtype = p->wdtype;
  info->tile = p->tile;
  info->nblocks = p->nblocks;
  info->M = p->M;
  info->nnz = p->nnz;
  info->n_units = p->n_units;
  info->beta = p->beta;
  info->dl = p->dl;
  info->device_bytes = p->device_bytes;
  info->region_pitch = p->pitch > 0 ? p->pitch : p->tile + p->Jmax - 1;
  info->run_max = p->run_max;
  info->row_batch = p->row_batch;
  info->nstacks = p->nstacks;
  info->holographic_bytes = p->d_H ? (int64_t)p->holo_S * p->holo_S * p->K * p->K * 8 : 0;
  info->unit_nnz = p->unit_nnz;
  info->compensated = p->compensated ? 1 : 0;
  return PNP_OK;
}

int pnp_plan_set_unit_nnz(pnp_plan* p, int64_t unit_nnz) {
  if (!p || unit_nnz < 0) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  if (unit_nnz == 0) return PNP_OK;
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  p->unit_nnz = unit_nnz;
  return build_units(p);
}

int pnp_plan_set_holographic(pnp_plan* p, int enable) {
  if (!p) return fail(PNP_ERR_INVALID_ARG, "NULL plan");
  if (enable) {
    PNP_CUDA(cudaStreamSynchronize(p->stream));
    if (int rc = holo_build_plan(p)) return rc;
  }
  p->holo = enable != 0;
  return PNP_OK;
}

int pnp_plan_set_compensated(pnp_plan* p, int enable) {
  if (!p || (enable != 0 && enable != 1)) return fail(PNP_ERR_INVALID_ARG, "enable must be 0 or 1");
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  if ((enable == 1) != p->compensated) ++p->epoch;
  p->compensated = enable == 1;
  return PNP_OK;
}

int pnp_plan_set_row_batch(pnp_plan* p, int row_batch) {
  if (!p || (row_batch != 0 && row_batch != 1 && row_batch != 2 && row_batch != 4))
    return fail(PNP_ERR_INVALID_ARG, "row_batch must be 0, 1, 2 or 4");
  if (row_batch == 0) return PNP_OK;
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  if (row_batch != p->row_batch) ++p->epoch;
  p->row_batch = row_batch;
  return PNP_OK;
}

int pnp_plan_autotune(pnp_plan* p, int reps, int* run_max_out, int64_t* unit_nnz_out, double* ms_out) {
  if (!p || reps < 1 || reps > 100) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  const int old_run = p->run_max, old_rb = p->row_batch;
  const int64_t old_unit = p->unit_nnz;
  int best_run = old_run, best_rb = old_rb;
  int64_t best_unit = old_unit;
  float best_ms = -1.f;
  if (p->M > 0 && p->n_units > 0) {
    const int runs[] = {3, 4, 6, 8};
    const int64_t units[] = {int64_t(1) << 16, int64_t(1) << 17, int64_t(1) << 18};
    const int batches[] = {1, 2, 4};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PNP_CUDA(cudaEventCreate(&e0));
    PNP_CUDA(cudaEventCreate(&e1));
    const bool saved_timing = p->timing;
    p->timing = false;
    int rc = PNP_OK;
    for (int r : runs) {
      for (int64_t u : units) {
        p->run_max = r;
        p->unit_nnz = u;
        if ((rc = build_units(p))) break;
        for (int rb : batches) {
          p->row_batch = rb;
          for (int s = 0; s < p->nstacks && !rc; ++s) rc = gridding_pass(p, G_FUSED, nullptr, nullptr, s);  // warm-up
          if (rc) break;
          if (cudaEventRecord(e0, p->stream) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(PNP_ERR_CUDA, "autotune: event record failed");
            break;
          }
          for (int i = 0; i < reps && !rc; ++i)
            for (int s = 0; s < p->nstacks && !rc; ++s) rc = gridding_pass(p, G_FUSED, nullptr, nullptr, s);
          if (rc) break;
          float ms = 0.f;
          if (cudaEventRecord(e1, p->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(PNP_ERR_CUDA, "autotune: timing failed");
            break;
          }
          ms /= reps;
          if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best_run = r;
            best_unit = u;
            best_rb = rb;
          }
        }
        if (rc) break;
      }
      if (rc) break;
    }
    p->timing = saved_timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timed passes accumulated into the output grid: start it from zero again
    if (!rc && (cudaMemsetAsync(p->d_gridB, 0, (size_t)p->K * p->K * sizeof(float2), p->stream) != cudaSuccess ||
                cudaMemsetAsync(p->d_gridB_lo, 0, (size_t)p->K * p->K * sizeof(__nv_bfloat162), p->stream) != cudaSuccess)) {
      cudaGetLastError();
      rc = fail(PNP_ERR_CUDA, "autotune: clearing the grid failed");
    }
    p->run_max = rc ? old_run : best_run;
    p->row_batch = rc ? old_rb : best_rb;
    p->unit_nnz = rc ? old_unit : best_unit;
    if (int rc2 = build_units(p)) return rc2;
    if (rc) return rc;
    PNP_CUDA(cudaStreamSynchronize(p->stream));
  }
  if (run_max_out) *run_max_out = p->run_max;
  if (unit_nnz_out) *unit_nnz_out = p->unit_nnz;
  if (ms_out) *ms_out = best_ms;
  return PNP_OK;
}

int pnp_plan_device_status(pnp_plan* p, int* flags) {
  if (!p || !flags) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  PNP_CUDA(cudaMemcpyAsync(flags, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  return PNP_OK;
}

int pnp_plan_set_timing(pnp_plan* p, int enable) {
  if (!p) return fail(PNP_ERR_INVALID_ARG, "NULL plan");
  p->timing = enable != 0;
  return PNP_OK;
}

int pnp_plan_read_timing(pnp_plan* p, double* ms, int64_t* count) {
  if (!p || !ms || !count) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  PNP_CUDA(cudaStreamSynchronize(p->stream));
  for (int i = 0; i < 3; ++i) {
    ms[i] = 0;
    count[i] = 0;
  }
  for (auto& t : p->timed) {
    float e = 0;
    PNP_CUDA(cudaEventElapsedTime(&e, t.a, t.b));
    if (t.stage >= 0 && t.stage < 3) {
      ms[t.stage] += e;
      count[t.stage] += 1;
    }
  }
  clear_timing(p);
  return PNP_OK;
}

int pnp_plan_export_rows(const pnp_plan* p, const int64_t* rows, int64_t nrows, int64_t* offsets,
                         float* weights, int32_t* cols) {
  if (!p || (nrows > 0 && (!rows || !offsets)) || nrows < 0) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  if (nrows == 0) {
    if (offsets) offsets[0] = 0;
    return PNP_OK;
  }
  return export_rows_impl(p, rows, nrows, offsets, weights, cols);
}

int phi_forward(pnp_plan* p, const float* x, float* y) {
  if (!p || !x || (p->M > 0 && !y)) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  for (int s = 0; s < p->nstacks; ++s) {
    if (int rc = fft_forward(p, x, s)) return rc;
    if (int rc = gridding_pass(p, G_DEGRID, nullptr, reinterpret_cast<float2*>(y), s)) return rc;
  }
  return PNP_OK;
}

int phi_adjoint(pnp_plan* p, const float* y, float* x) {
  if (!p || !x || (p->M > 0 && !y)) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  if (int rc = permute_y(p, reinterpret_cast<const float2*>(y))) return rc;
  for (int s = 0; s < p->nstacks; ++s) {
    if (int rc = gridding_pass(p, G_GRID, reinterpret_cast<const float2*>(y), nullptr, s)) return rc;
    if (int rc = fft_adjoint(p, EPI_ADJ, nullptr, x, 0.f, 0.f, s)) return rc;
  }
  return PNP_OK;
}

int grad_step(pnp_plan* p, const float* x, const float* y, double gamma, float* x_out) {
  if (!p || !x || !x_out || (p->M > 0 && !y)) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  if (x == x_out) return fail(PNP_ERR_INVALID_ARG, "x and x_out must not alias");
  if (!std::isfinite(gamma)) return fail(PNP_ERR_INVALID_ARG, "gamma must be finite");
  if (int rc = permute_y(p, reinterpret_cast<const float2*>(y))) return rc;
  return normal_pass(p, reinterpret_cast<const float2*>(y), x, EPI_GRAD, x, x_out, (float)gamma, 0.f, false);
}

int op_norm(pnp_plan* p, const float* v0, int max_it, double tol, double* L_out, int* iters_out) {
  if (!p || !L_out || max_it < 1 || !(tol >= 0)) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  const int64_t N = (int64_t)p->n * p->n;
  float* v = p->d_img[0];
  float* g = p->d_img[2];
  if (v0) PNP_CUDA(cudaMemcpyAsync(v, v0, N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream));
  else if (int rc = fill_image(p->stream, v, N, 1.f)) return rc;
  if (int rc = zero_acc(p->stream, p->d_acc, 4)) return rc;
  if (int rc = norm2_dev(p->stream, v, N, p->d_acc)) return rc;
  if (int rc = scale_image(p->stream, v, v, N, p->d_acc, 0)) return rc;
  double L = 0.0, h[2];
  int it = 0;
  for (it = 1; it <= max_it; ++it) {
    if (int rc = normal_pass(p, nullptr, v, EPI_NORMAL, nullptr, g, 0.f, 0.f, true)) return rc;
    if (int rc = scale_image(p->stream, g, v, N, p->d_acc, 0)) return rc;
    if (int rc = read_acc(p, h, 1)) return rc;
    const double Ln = std::sqrt(h[0]);
    if (!std::isfinite(Ln)) return fail(PNP_ERR_DIVERGED, "power iteration produced a non-finite norm");
    const bool done = it > 1 && std::fabs(Ln - L) <= tol * Ln;
    L = Ln;
    if (done) break;
  }
  *L_out = L;
  if (iters_out) *iters_out = it > max_it ? max_it : it;
  return PNP_OK;
}

int pnp_den_create_haar(pnp_den** den, double t, void* stream) {
  if (!den || !(t >= 0) || !std::isfinite(t)) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  pnp_den* d = new pnp_den();
  d->kind = PNP_DEN_HAAR;
  d->t = t;
  d->serial = ++g_den_serial;
  d->stream = reinterpret_cast<cudaStream_t>(stream);
  *den = d;
  return PNP_OK;
}

int pnp_den_create_cnn(pnp_den** den, const float* weights_host, const int32_t* facet_rows_host, int nfr,
                       const int32_t* facet_cols_host, int nfc, int halo, int n, void* stream) {
  if (!den || !weights_host || n < 1 || halo < 0) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  *den = nullptr;
  pnp_den* d = new pnp_den();
  d->kind = PNP_DEN_CNN;
  d->serial = ++g_den_serial;
  d->stream = reinterpret_cast<cudaStream_t>(stream);
  int rc = cnn_create(d, weights_host, facet_rows_host, nfr, facet_cols_host, nfc, halo, n);
  if (rc != PNP_OK) {
    std::string keep = t_err;
    cnn_destroy(d);
    delete d;
    t_err = keep;
    return rc;
  }
  *den = d;
  return PNP_OK;
}

int pnp_den_cnn_set_strip_rows(pnp_den* den, int rows) {
  if (!den || den->kind != PNP_DEN_CNN) return fail(PNP_ERR_INVALID_ARG, "not a CNN denoiser");
  if (int rc = cnn_set_strip_rows(den, rows)) return rc;
  den->serial = ++g_den_serial;  // graphs captured with this denoiser hold the old launch sizes
  return PNP_OK;
}

int pnp_den_cnn_autotune(pnp_den* den, const float* z, int n, int reps, int* rows_out, double* ms_out) {
  if (!den || den->kind != PNP_DEN_CNN || !z) return fail(PNP_ERR_INVALID_ARG, "not a CNN denoiser, or NULL input");
  if (reps < 1 || reps > 100) return fail(PNP_ERR_INVALID_ARG, "reps must lie in [1, 100]");
  static const int kRows[] = {16, 24, 32, 48, 64, 96};
  float* out = nullptr;
  if (cudaMalloc(&out, (size_t)n * n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return fail(PNP_ERR_OOM, "autotune scratch image");
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PNP_OK, best = cnn_strip_rows(den);
  double best_ms = -1.0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    rc = fail(PNP_ERR_CUDA, "event creation failed");
  }
  for (int rows : kRows) {
    if (rc) break;
    if ((rc = cnn_set_strip_rows(den, rows))) break;
    if ((rc = cnn_denoise(den, den->stream, z, out, n, nullptr, nullptr))) break;  // warm
    if (cudaEventRecord(e0, den->stream) != cudaSuccess) { rc = fail(PNP_ERR_CUDA, "event record"); break; }
    for (int r = 0; r < reps && !rc; ++r) rc = cnn_denoise(den, den->stream, z, out, n, nullptr, nullptr);
    if (rc) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, den->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(PNP_ERR_CUDA, "event timing failed");
      break;
    }
    const double per = ms / reps;
    if (best_ms < 0 || per < best_ms) {
      best_ms = per;
      best = rows;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (!rc) rc = cnn_set_strip_rows(den, best);
  den->serial = ++g_den_serial;
  if (rc) return rc;
  if (rows_out) *rows_out = best;
  if (ms_out) *ms_out = best_ms;
  return PNP_OK;
}

int pnp_den_create_sara(pnp_den** den, int n, int levels, double gamma_lambda, double rho, int prox_iters,
                        void* stream) {
  if (!den) return fail(PNP_ERR_INVALID_ARG, "NULL denoiser pointer");
  *den = nullptr;
  if (levels < 1 || levels > 8 || n < 2 || n % (1 << levels) != 0)
    return fail(PNP_ERR_INVALID_ARG, "n must be a multiple of 2^levels, levels in [1, 8]");
  if (!(gamma_lambda >= 0) || !std::isfinite(gamma_lambda) || !(rho > 0) || !std::isfinite(rho) || prox_iters < 1)
    return fail(PNP_ERR_INVALID_ARG, "bad SARA parameters");
  pnp_den* d = new pnp_den();
  d->kind = PNP_DEN_SARA;
  d->serial = ++g_den_serial;
  d->t = gamma_lambda;
  d->stream = reinterpret_cast<cudaStream_t>(stream);
  if (int rc = sara_create(d, n, levels, gamma_lambda, rho, prox_iters)) {
    std::string keep = t_err;
    sara_destroy(d);
    delete d;
    t_err = keep;
    return rc;
  }
  *den = d;
  return PNP_OK;
}

int pnp_den_sara_reweight(pnp_den* den, const float* x) {
  if (!den || !x || den->kind != PNP_DEN_SARA) return fail(PNP_ERR_INVALID_ARG, "not a SARA denoiser");
  return sara_reweight(den, x);
}

int pnp_sara_transform(pnp_den* den, const float* in, float* out, int direction) {
  if (!den || !in || !out || den->kind != PNP_DEN_SARA || (direction != 1 && direction != -1))
    return fail(PNP_ERR_INVALID_ARG, "bad argument");
  return sara_transform(den, in, out, direction);
}

void pnp_den_destroy(pnp_den* den) {
  if (!den) return;
  cudaStreamSynchronize(den->stream);
  if (den->kind == PNP_DEN_CNN) cnn_destroy(den);
  if (den->kind == PNP_DEN_SARA) sara_destroy(den);
  delete den;
}

int pnp_den_device_status(pnp_den* d, int* flags) {
  if (!d || !flags) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  *flags = 0;
  if (d->kind != PNP_DEN_CNN) return PNP_OK;
  PNP_CUDA(cudaStreamSynchronize(d->stream));
  return cnn_status(d, flags);
}

int denoise(pnp_den* d, const float* x_in, float* x_out, int n) {
  if (!d || !x_in || !x_out || n < 2 || (n & 1)) return fail(PNP_ERR_INVALID_ARG, "bad argument");
  if (x_in == x_out) return fail(PNP_ERR_INVALID_ARG, "x_in and x_out must not alias");
  if (d->kind == PNP_DEN_HAAR) return haar_denoise_dev(d->stream, x_in, x_out, n, (float)d->t, nullptr, nullptr);
  if (d->kind == PNP_DEN_SARA) return sara_denoise(d, d->stream, x_in, x_out, n, nullptr, nullptr);
  return cnn_denoise(d, d->stream, x_in, x_out, n, nullptr, nullptr);
}

int pnp_fb_run(pnp_plan* p, pnp_den* d, const float* y, const pnp_params* prm, float* x, pnp_stats* st) {
  if (!p || !d || !prm || !x || (p->M > 0 && !y)) return fail(PNP_ERR_INVALID_ARG, "NULL argument");
  if (prm->max_iter < 0) return fail(PNP_ERR_INVALID_ARG, "max_iter must be >= 0");
  if (!std::isfinite(prm->alpha)) return fail(PNP_ERR_INVALID_ARG, "alpha must be finite");
  if (prm->positivity != PNP_POSITIVITY_ON && prm->positivity != PNP_POSITIVITY_OFF)
    return fail(PNP_ERR_INVALID_ARG, "positivity must be PNP_POSITIVITY_ON or PNP_POSITIVITY_OFF");
  if (prm->fallback != 0 && prm->fallback != 1) return fail(PNP_ERR_INVALID_ARG, "fallback must be 0 or 1");
  if (prm->fallback && (!(prm->fallback_t >= 0) || !std::isfinite(prm->fallback_t)))
    return fail(PNP_ERR_INVALID_ARG, "fallback_t must be finite and >= 0");
  if (prm->reweight_every < 0 || (prm->reweight_every > 0 && d->kind != PNP_DEN_SARA))
    return fail(PNP_ERR_INVALID_ARG, "reweight_every must be 0, or > 0 with a SARA denoiser");
  const int rw = prm->reweight_every;
  const double alpha = prm->alpha > 0 ? prm->alpha : 1.0;
  const bool pos = prm->positivity == PNP_POSITIVITY_ON;
  const bool fallback = prm->fallback == 1 && d->kind == PNP_DEN_CNN;
  const int64_t N = (int64_t)p->n * p->n;
  double L = prm->L;
  if (!(L > 0)) {
    if (int rc = op_norm(p, nullptr, 500, 1e-6, &L, nullptr)) return rc;
  }
  const double gamma = prm->gamma > 0 ? prm->gamma : 1.98 / L;
  const int check = prm->check_every > 0 ? prm->check_every : 10;
  const bool graph = prm->use_graph != 0;
  // App. C, Eq. invpb2: iterate on y / alpha from x / alpha
  if (int rc = permute_y(p, reinterpret_cast<const float2*>(y), (float)(1.0 / alpha))) return rc;
  if (p->holo)
    if (int rc = holo_dirty_grid(p)) return rc;  // G^H y once per run (App. E, Eq. phidagphi)
  if (alpha != 1.0)
    if (int rc = mul_image(p->stream, x, x, N, (float)(1.0 / alpha))) return rc;
  float* buf[2] = {x, p->d_img[0]};
  float* keep = p->d_img[2];  // fallback: the last checked finite iterate
  pnp_den plain;              // the fallback's Haar denoiser (no device state)
  plain.kind = PNP_DEN_HAAR;
  plain.t = prm->fallback_t;
  plain.stream = p->stream;
  plain.serial = 0;
  pnp_den* den = d;
  int c = 0, k = 0, rc = PNP_OK, fell = -1, k_keep = 0;
  double h[2] = {0, 0}, rel = 0, xn = 0, xn_min = -1;
  if (fallback) {
    plain.serial = ++g_den_serial;
    if (cudaMemcpyAsync(keep, x, N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(PNP_ERR_CUDA, "saving the start iterate failed");
    }
  }
  while (k < prm->max_iter && rc == PNP_OK) {
    const int bit = 1 << den->kind;
    GraphRunner gr(p, den, buf, gamma, pos);
    int chunk = std::min(check, prm->max_iter - k);
    if (rw > 0) chunk = std::min(chunk, rw - k % rw);  // a chunk ends at every reweighting
    for (int done = 0; done < chunk && rc == PNP_OK;) {
      const int left = chunk - done;
      if (graph && c == 0 && left >= 2 && (p->primed & bit)) {
        rc = gr.run_pairs(left / 2);
        done += 2 * (left / 2);
      } else {
        rc = fb_iteration(p, den, buf[c], buf[1 - c], gamma, pos);
        if (rc == PNP_OK) p->primed |= bit;
        c = 1 - c;
        ++done;
      }
    }
    if (rc) break;
    k += chunk;
    if ((rc = read_acc(p, h, 2))) break;
    xn = std::sqrt(h[1]);
    rel = xn > 0 ? std::sqrt(h[0]) / xn : 0.0;
    std::string why;
    if (!std::isfinite(h[0]) || !std::isfinite(h[1])) why = "iterate became non-finite at iteration " + std::to_string(k);
    else if (prm->diverge_factor > 0 && xn_min > 0 && xn > prm->diverge_factor * xn_min)
      why = "iterate norm grew past the divergence factor at iteration " + std::to_string(k);
    if (!why.empty()) {
      if (fallback && den == d) {
        // App. C: the learned loop falls back to the plain one from the last checked finite iterate
        if (cudaMemcpyAsync(buf[c], keep, N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess) {
          cudaGetLastError();
          rc = fail(PNP_ERR_CUDA, "restoring the last finite iterate failed");
          break;
        }
        den = &plain;
        fell = k_keep;
        k = k_keep;
        xn_min = -1;
        continue;
      }
      rc = fail(PNP_ERR_DIVERGED, why);
      break;
    }
    if (xn > 0 && (xn_min < 0 || xn < xn_min)) xn_min = xn;
    if (fallback && den == d) {
      if (cudaMemcpyAsync(keep, buf[c], N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(PNP_ERR_CUDA, "saving the checked iterate failed");
        break;
      }
      k_keep = k;
    }
    if (prm->tol > 0 && rel < prm->tol) break;
    // uSARA (App. B): the next weighted-l1 surrogate, majorising the log-sum prior at the current iterate
    if (rw > 0 && k % rw == 0) {  // also at the end of the run, so that consecutive calls continue it
      if ((rc = sara_reweight(d, buf[c]))) break;  // on the denoiser's stream: the iterate is ready (read_acc)
      if (d->stream != p->stream && cudaStreamSynchronize(d->stream) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(PNP_ERR_CUDA, "reweighting failed");
        break;
      }
    }
  }
  if (c == 1) {
    cudaError_t e = cudaMemcpyAsync(x, buf[1], (size_t)N * sizeof(float), cudaMemcpyDeviceToDevice, p->stream);
    if (e != cudaSuccess && rc == PNP_OK) {
      cudaGetLastError();
      rc = fail(PNP_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (alpha != 1.0) {  // the solution of the rescaled problem times alpha
    const int rc2 = mul_image(p->stream, x, x, N, (float)alpha);
    if (rc == PNP_OK) rc = rc2;
  }
  if (st) {
    st->iters = k;
    st->L = L;
    st->gamma = gamma;
    st->rel_change = rel;
    st->x_norm = xn;
    st->fallback_iter = fell;
  }
  return rc;
}

}  // extern "C"
