// Shared internals of the PnP-FB library: plan/denoiser structs, error
// plumbing and small device helpers.  Everything here is sm_103a-only.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/pnp.h"

namespace pnp {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
extern std::atomic<int64_t> g_launches;

#define PNP_CUDA(call)                                                           \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      cudaGetLastError(); /* clear a non-sticky error so later checks are clean */ \
      return ::pnp::fail(PNP_ERR_CUDA, std::string(#call) + ": " +              \
                                           cudaGetErrorString(e_));             \
    }                                                                            \
  } while (0)

#define PNP_CHECK_LAUNCH()                                                       \
  do {                                                                           \
    ::pnp::g_launches.fetch_add(1, std::memory_order_relaxed);                   \
    cudaError_t e_ = cudaGetLastError();                                         \
    if (e_ != cudaSuccess)                                                       \
      return ::pnp::fail(PNP_ERR_CUDA, std::string("kernel launch: ") +         \
                                           cudaGetErrorString(e_));             \
  } while (0)

// ------------------------------------------------------------------ complex
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ------------------------------------------------------------------ work units
// Gridding work list.  A chunk is a run of consecutive rows (tile-sorted order)
// with at most CHUNK_TAPS taps and CHUNK_ROWS rows: the unit of one TMA bulk
// transfer.  A unit is a run of consecutive chunks whose rows all have their
// first tap in one grid tile (and one data block).
constexpr int CHUNK_TAPS = 4096;
constexpr int CHUNK_ROWS = 128;
constexpr int NSTAGE = 4;          // shared-memory pipeline depth of the gridding pass
constexpr int GPASS_CONSUMERS = 16; // consumer warps per gridding CTA (plus one producer warp)
constexpr int GPASS_THREADS = 32 * (GPASS_CONSUMERS + 1);
// twiddles of the radix-16 passes 1 and 2 of the FFT: entry off(p) + r 16^p + k holds
// exp(-2 pi i r k / 16^(p+1)), off(1) = 0, off(2) = 256 (independent of the transform length)
constexpr int TWP_ENTRIES = 16 * 16 + 16 * 256;
constexpr int TAP_PAD = 16;        // weights/columns are allocated nnz + TAP_PAD long
constexpr int ROW_PAD = 4;         // row offsets M + 1 + ROW_PAD, sorted y M + ROW_PAD

struct Chunk {
  long long row_begin;
  long long tap_begin;
  long long run_begin;  // first entry of the chunk's run list in the plan's run array
  int nrows;
  int ntaps;
  int nn;     // taps per row (J^2, the same for every row of the chunk)
  int nruns;  // runs of rows sharing one tap window; the list holds nruns + 1 row offsets
};
constexpr int RUN_MAX = 6;         // default cap on rows per run (keeps the consumer warps balanced)

struct Unit {
  long long chunk_begin;
  int nchunks;
  int tile;
};

// Q2 epilogue modes of the last inverse-FFT pass (see fft.cu).
// EPI_HAAR_NOPOS: the Haar prox without the final positivity projection.
enum EpiMode { EPI_ADJ = 0, EPI_GRAD = 1, EPI_HAAR = 2, EPI_Z = 3, EPI_NORMAL = 4, EPI_HAAR_NOPOS = 5 };

// Gridding pass modes (see gridding.cu).
enum GMode { G_DEGRID = 0, G_GRID = 1, G_FUSED = 2 };

}  // namespace pnp

// ------------------------------------------------------------------ plan
struct pnp_plan {
  int n = 0, K = 0, logK = 0, J = 7, Jmax = 7, wdtype = PNP_W_C64, nblocks = 1;
  int tile = 48;       // gridding tile side T (cells)
  int ntc = 0;         // tiles per grid side, ceil(K / tile)
  int slots = 8;       // register slots per lane per row (32*slots >= Jmax^2)
  int pitch = 0;       // row pitch (cells) of the staged gridding regions (0: the region side)
  int run_max = pnp::RUN_MAX;  // rows per run of a shared tap window, at most
  int row_batch = 2;           // rows of a run whose residuals a warp forms together (1, 2, 4)
  int rpw = 2;         // rows per warp in flight
  int64_t M = 0, nnz = 0, unit_nnz = 1 << 17;
  double beta = 0, dl = 0;
  int nstacks = 1;             // w-stacks P (App. E): rows sorted by stack, then tile and block
  int64_t nkeys = 0;           // (tile, block) keys per stack
  std::vector<double> w_centres;       // P stack centres [wavelengths]
  std::vector<int64_t> h_stack_units;  // P+1: the work units of stack s are [s], [s+1])
  cudaStream_t stream = nullptr;   // caller's stream: every launch goes here
  cudaStream_t cstream = nullptr;  // private non-blocking stream for graph capture/replay
  cudaEvent_t ev_join[2] = {nullptr, nullptr};
  int device = 0, num_sms = 0;
  int primed = 0;  // bit k: an eager FB iteration with denoiser kind k has configured every kernel
  uint64_t epoch = 0;  // bumped whenever the gridding work decomposition changes (captured graphs go stale)
  // CUDA graph of two FB iterations kept across pnp_fb_run calls, valid while its key matches
  struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    uint64_t den_serial = 0, epoch = 0;
    const float* x = nullptr;
    double gamma = 0;
    int epi = 0;
    bool holo = false;
  } graph;

  // device buffers
  float* d_cinv = nullptr;     // n: 1 / c(a - n/2)
  float2* d_tw = nullptr;      // K: exp(-2 pi i j / K)
  float2* d_twp = nullptr;     // radix-16 pass twiddles [16 + 256][16]: see fft.cu
  float2* d_gridA = nullptr;   // K*K: F Z x   (layout [k1][k0])
  float2* d_gridB = nullptr;   // K*K: G^H r   (layout [k1][k0]); kept zero between uses
  __nv_bfloat162* d_gridB_lo = nullptr; // K*K: compensation terms of d_gridB's atomic sums (BF16 pairs:
                                         // they are ~2^-24 of the sums); kept zero between uses
  bool compensated = false;    // gridding flushes add their rounding errors to d_gridB_lo (TwoSum)
  float2* d_tmp = nullptr;     // K*n: half-transformed intermediate
  void* d_w = nullptr;         // nnz weights (float2 or bf16x2)
  uint16_t* d_cells = nullptr; // nnz cell indices lr * pitch + lc in the row's staged tile region
  uint8_t* d_runs = nullptr;    // per chunk: row offsets where runs start, then nrows (padded by 16)
  int64_t n_runs = 0;
  int64_t* d_rowptr = nullptr; // M+1 (sorted order)
  int32_t* d_perm = nullptr;   // sorted row -> caller row
  float2* d_ysorted = nullptr; // M scratch: y in sorted order
  pnp::Unit* d_units = nullptr;
  int64_t n_units = 0;
  pnp::Chunk* d_chunks = nullptr;
  int64_t n_chunks = 0;
  double* d_acc = nullptr;     // FP64 accumulators [8]
  int* d_status = nullptr;     // device status flags [4] (bit 0: gridding index out of range)
  float* d_img[3] = {nullptr, nullptr, nullptr};  // n*n work images
  float2* d_chirp = nullptr;   // P*n (P > 1): per stack and image axis exp(i pi a_p (a - n/2)^2)
  float* d_gacc = nullptr;     // n*n (P > 1): gradient image accumulated over the stacks
  float2* d_H = nullptr;       // holographic H = G^H G: [S*S offsets][K*K cells], S = 2 Jmax - 1
  float2* d_dirty = nullptr;   // K*K: G^H y of the current FB run (holographic mode)
  float* d_rowscale = nullptr; // M (caller order): data weights d_m folded into the rows of G, or NULL
  // uv support of G (the grid cells that hold taps, over every row and w-stack): per grid row k1,
  // the largest centred |k0| of a tap in the row (-1: no tap), and the centred half-width of the
  // band of rows k1 that hold taps (-1: none).  The split FFT passes transform and move only what
  // lies in it (the pruned F of Eq. 1: G reads no other cell and writes no other cell).
  int* d_rowh = nullptr;       // K
  int band = -1;
  int holo_S = 0;
  bool holo = false;           // FB loop and op_norm apply H instead of streaming G
  int64_t device_bytes = 0;

  // optional per-stage event timing: (stage, start, stop)
  bool timing = false;
  struct TimedEvent { int stage; cudaEvent_t a, b; };
  std::vector<TimedEvent> timed;

  // host mirrors used by export and work-list rebuilds
  std::vector<int64_t> h_rowptr;   // M+1
  std::vector<int32_t> h_perm;     // sorted -> caller
  std::vector<int32_t> h_inv;      // caller -> sorted
  std::vector<int32_t> h_key;      // sorted: (stack * ntc^2 + tile) * nblocks + block
  std::vector<uint16_t> h_start;   // sorted: first tap's cell in the tile (row * tile + col)
};

struct pnp_den {
  int kind = PNP_DEN_HAAR;
  uint64_t serial = 0;    // unique per denoiser created in this process (keys the plan's graph cache)
  double t = 0;
  cudaStream_t stream = nullptr;
  void* impl = nullptr;   // CNN state (cnn.cu)
};

namespace pnp {
// pnp_api.cu: bracket one stage with events when timing is enabled
int stage_begin(pnp_plan* p, int stage, cudaEvent_t* a);
int stage_end(pnp_plan* p, int stage, cudaEvent_t a);
// fft.cu
// Stack s selects the centre chirp of Z_s (none for a plan with one stack); the adjoint of a
// stack other than the last only accumulates Re{Z_s^H ...} into d_gacc, and the last one adds
// the accumulated sum before its epilogue `mode`.
int fft_forward(pnp_plan* p, const float* x, int s);                       // x -> d_gridA
int fft_adjoint(pnp_plan* p, int mode, const float* x, float* out,         // d_gridB -> out
                float gamma, float t, int s);
// gridding.cu: the work units of stack s
int gridding_pass(pnp_plan* p, int mode, const float2* y_user, float2* y_out, int s);
// choose p->pitch from the plan's number of rows per support J (rows_per_J[0..16])
int gridding_pitch(pnp_plan* p, const int64_t* rows_per_J);
int permute_y(pnp_plan* p, const float2* y_user, float scale = 1.f);  // d_ysorted = scale y_user[perm]
// plan_build.cu
int build_units(pnp_plan* p);
int plan_build(pnp_plan* p, const double* uvw, const int8_t* Jrow, const int32_t* block, const int32_t* stack,
               const double* row_scale);
// holographic.cu: build H (once), the dirty grid of the sorted data, one application of H
int holo_build_plan(pnp_plan* p);
int holo_dirty_grid(pnp_plan* p);
int holo_apply_pass(pnp_plan* p, bool data_term);  // d_gridB = H d_gridA (- d_dirty)
// update.cu
int haar_denoise_dev(cudaStream_t s, const float* z, float* out, int n, float t, double* acc,
                     const float* x_prev);
int scale_image(cudaStream_t s, const float* in, float* out, int64_t count, const double* acc,
                int acc_index);
int zero_acc(cudaStream_t s, double* acc, int count);
int mul_image(cudaStream_t s, const float* in, float* out, int64_t count, float f);  // out = f in
int row_scale_c64(cudaStream_t s, const float2* y_in, const float* d, float2* y_out, int64_t count);
// cnn.cu
int cnn_create(pnp_den* d, const float* weights_host, const int32_t* fr, int nfr,
               const int32_t* fc, int nfc, int halo, int n);
void cnn_destroy(pnp_den* d);
int cnn_status(pnp_den* d, int* flags);
// shared with the CNN trainer (cnn_train.cu)
// B operand of the 64 -> 64 convolution: weight W[co][ci][dy][dx] at
// [dx][ci / 8][2 - dy][co][ci % 8], so that for one (dx, 8-channel block) the three dy taps are
// consecutive 64-row blocks in descending dy (one MMA serves up to three output rows).
__host__ __device__ __forceinline__ size_t conv_wpack_index(int dy, int dx, int ci, int co) {
  return ((((size_t)dx * 8 + (ci >> 3)) * 3 + (2 - dy)) * 64 + co) * 8 + (ci & 7);
}
constexpr int STRIP_ROWS = 32;  // target output rows per convolution work unit
// Work list of the hidden-layer convolution (conv64_rows): per facet, 128-column segments split into strips of about STRIP_ROWS
// output rows; each entry is (facet, x0, ya << 16 | rows, Hf << 16 | Wf).
std::vector<int4> conv_strips(int F, const int* Hf, const int* Wf, int rows = STRIP_ROWS);
// the denoiser's convolution work lists rebuilt for strips of about `rows` output rows (4..1024)
int cnn_set_strip_rows(pnp_den* d, int rows);
int cnn_strip_rows(pnp_den* d);
// the convolution reads its input through the TMA descriptor in_map (canvas_map_create)
int conv64_launch(cudaStream_t s, const void* in_map, __nv_bfloat16* out, const __nv_bfloat16* w_packed,
                  const float* bias, const int4* strips, int n_strips, int Hc, int Wc, int mode,
                  const __nv_bfloat16* mask, int* status);
// Activation canvases of the CNN hold BF16 values in planes of 8 channels:
// [F][Hc][64 / 8][Wc][8], so that a row of one 8-channel block is contiguous (full-sector
// TMA reads, coalesced epilogue stores); element (f, y, x, c) sits at canvas_index(...).
__host__ __device__ __forceinline__ size_t canvas_index(int f, int y, int x, int c, int Hc, int Wc) {
  return ((((size_t)f * Hc + y) * 8 + (c >> 3)) * Wc + x) * 8 + (c & 7);
}
// TMA descriptors of an activation canvas for the convolution's row loads: two 128-byte
// CUtensorMaps written to map_out (the 128-pixel main box and the 2-pixel halo box)
int canvas_map_create(void* map_out, const __nv_bfloat16* canvas, int F, int Hc, int Wc);
int cnn_first_launch(cudaStream_t s, const float* z, int n, int64_t zplane, const int4* facets, int F, int Hc,
                     int Wc, const float* w1, const float* b1, __nv_bfloat16* out);
int cnn_denoise(pnp_den* d, cudaStream_t s, const float* z, float* out, int n, double* acc,
                const float* x_prev, bool positivity = true);
// sara.cu: uSARA's denoiser (App. B)
int sara_create(pnp_den* d, int n, int levels, double gamma_lambda, double rho, int iters);
void sara_destroy(pnp_den* d);
int sara_denoise(pnp_den* d, cudaStream_t s, const float* z, float* out, int n, double* acc, const float* x_prev,
                 bool positivity = true);
int sara_reweight(pnp_den* d, const float* x);
int sara_transform(pnp_den* d, const float* in, float* out, int direction);
}  // namespace pnp
