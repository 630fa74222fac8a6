/*
 * pnp.h - C ABI of the GB300 (sm_103a) plug-and-play forward-backward (PnP-FB)
 * radio-interferometric imaging library (arXiv 2207.11336, Dabbech et al. 2022).
 *
 * The library implements the measurement model of Eq. 1,
 *     y = Phi x + n,   Phi = G F Z,
 * the data-fidelity gradient of App. A,
 *     grad f(x) = Re{Phi^H (Phi x - y)},   L = ||Re{Phi^H Phi}||_S,
 * and the forward-backward iteration of Eq. fb with a plug-in denoiser D:
 *     x^{k+1} = D(x^k - gamma grad f(x^k)).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Image x: n x n float32, row-major x[a*n + b], Jy/pixel.  Pixel (a, b) sits
 *    at the centred offset p = (a - n/2, b - n/2); p = (0, 0) is the phase centre.
 *  - Visibilities y: M complex64 (interleaved re, im) in the caller's row order.
 *    Row m has angular frequencies (omega_0, omega_1) in rad/pixel (omega_0 pairs
 *    with image axis 0) and w in wavelengths.
 *  - Z: zero-padding on a K x K grid plus division by the Kaiser-Bessel (KB)
 *    kernel's continuous Fourier transform c(p0) c(p1).  F: unnormalised 2-D
 *    DFT.  G: sparse rows; row m holds the J_m x J_m taps nearest
 *    kappa = omega K / (2 pi) of the KB kernel (J = 7 by default) convolved
 *    with the row's w-kernel (App. E), stored as complex64 (or bfloat16
 *    complex) weights with int32 column indices and int64 row offsets.
 *  - Device pointers ("dev") are CUDA global-memory addresses owned by the
 *    caller; the library never frees them.  Host pointers ("host") are read
 *    during the call only.
 *  - Every call that takes a plan or denoiser is asynchronous on that handle's
 *    stream unless it says otherwise; results are ready after a stream
 *    synchronisation.
 *  - Return value: PNP_OK (0) or a negative PNP_ERR_* code; pnp_last_error()
 *    gives a message for the calling thread.
 */
#ifndef PNP_H
#define PNP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PNP_OK = 0,
  PNP_ERR_INVALID_ARG = -1, /* a size, pointer or option is out of range      */
  PNP_ERR_OOM = -2,         /* device or host allocation failed               */
  PNP_ERR_CUDA = -3,        /* a CUDA runtime call failed                     */
  PNP_ERR_DIVERGED = -4,    /* NaN/Inf or growing iterate in pnp_fb_run       */
  PNP_ERR_TIMEOUT = -5,     /* a bounded device-side wait gave up             */
  PNP_ERR_UNSUPPORTED = -6  /* valid request outside what this build supports */
};

/* Storage type of G's weights. */
enum { PNP_W_C64 = 0, PNP_W_BF16C = 1 };

/* Denoiser kinds. */
enum { PNP_DEN_HAAR = 0, PNP_DEN_CNN = 1, PNP_DEN_SARA = 2 };

typedef struct pnp_plan pnp_plan;
typedef struct pnp_den pnp_den;

/* Parameters of pnp_fb_run (Eq. fb; App. B, F). */
typedef struct pnp_params {
  double gamma;      /* step size; <= 0 selects 1.98 / L (App. B)                */
  double L;          /* Lipschitz constant; <= 0 runs op_norm first (App. A)    */
  int max_iter;      /* number of FB iterations (>= 0)                           */
  double tol;        /* stop when ||x+ - x|| / ||x+|| < tol (tested only if > 0) */
  int check_every;   /* host reads the FP64 norms every this many iterations    */
  int use_graph;     /* 1: replay iterations as one captured CUDA graph          */
  double diverge_factor; /* > 0: fail with PNP_ERR_DIVERGED if ||x+|| grows past
                            this factor times its smallest checked value        */
  double alpha;      /* rescaling of App. C (Eq. invpb2): the loop solves
                        y / alpha = Phi (x / alpha) + n / alpha, i.e. it starts
                        from x_inout / alpha, iterates on y / alpha and writes
                        alpha x back, so the denoiser (and a Haar threshold)
                        acts on the peak-normalised image; <= 0 means 1       */
  int positivity;    /* PNP_POSITIVITY_ON (0, the default) ends every denoiser
                        with the projection max(0, .) (App. B, C);
                        PNP_POSITIVITY_OFF leaves it out                      */
  int fallback;      /* 1: when the loop with a learned (CNN) denoiser diverges
                        (non-finite iterate or diverge_factor exceeded), restart
                        from the last checked finite iterate with the plain Haar
                        denoiser at threshold fallback_t for the remaining
                        iterations instead of failing (App. C: the plain loop is
                        the learned loop's fallback); 0: fail                 */
  double fallback_t; /* Haar threshold of the fallback, in the rescaled units
                        of alpha (>= 0)                                       */
  int reweight_every; /* uSARA (SARA denoiser only, App. B Eq. B1): > 0 re-forms
                        the weights w = rho / (rho + |Psi^T x|) from the current
                        iterate (the loop's units) after every this many
                        iterations of the run, its last one included (so calls
                        of a multiple of it continue one schedule): the run is
                        a sequence of weighted-l1 surrogates of the log-sum
                        prior; 0 keeps the weights.  Other denoisers: must be
                        0 (PNP_ERR_INVALID_ARG)                               */
} pnp_params;

enum { PNP_POSITIVITY_ON = 0, PNP_POSITIVITY_OFF = 1 };

/* Outputs of pnp_fb_run. */
typedef struct pnp_stats {
  int iters;          /* iterations executed                                     */
  double L;           /* Lipschitz constant used                                 */
  double gamma;       /* step size used                                          */
  double rel_change;  /* ||x^k - x^{k-1}|| / ||x^k|| at the last check (FP64)    */
  double x_norm;      /* ||x^k|| at the last check (FP64), rescaled units        */
  int fallback_iter;  /* iteration from which the plain Haar fallback ran (the
                         last checked finite iterate), or -1 when it did not  */
} pnp_stats;

/* Read-only facts about a plan. */
typedef struct pnp_plan_info {
  int n, K, J, weight_dtype, tile, nblocks;
  int64_t M, nnz, n_units;
  double beta;          /* KB shape parameter                                  */
  double dl;            /* pixel size [rad] used for the w-term (0: none)      */
  int64_t device_bytes; /* device memory held by the plan                      */
  int region_pitch;     /* row pitch (cells) of the gridding pass's shared-memory
                           grid regions, chosen at plan time to limit bank
                           conflicts for the plan's mix of supports J        */
  int run_max;          /* rows at most per run of rows sharing a tap window  */
  int64_t unit_nnz;     /* taps at most per gridding work unit                */
  int row_batch;        /* rows of a run whose residuals one warp forms together */
  int nstacks;          /* w-stacks P of the operator (1: w wholly in G)      */
  int64_t holographic_bytes; /* device bytes of the holographic H (0: not built) */
  int compensated;      /* 1: gridding sums are compensated (pnp_plan_set_compensated) */
} pnp_plan_info;

/* ------------------------------------------------------------------ plans */

/* Build the measurement operator Phi = G F Z of Eq. 1 (w-terms folded into G
 * as in App. E) on the current CUDA device.
 *  n             image side (even, 8 <= n <= K/2)
 *  K             grid side (power of two, 64 <= K <= 16384)
 *  M             number of visibilities (>= 0; 0 gives an empty operator)
 *  uvw_host      host, M x 3 float64 row-major: omega_0, omega_1 [rad/px] in
 *                [-pi, pi), w [wavelengths]
 *  dl            pixel size [rad] for the w-term; 0 disables w (KB rows only)
 *  J_per_row_host host, M int8 supports J_m in [J, 16], or NULL for J_m = J
 *  J             KB kernel support (odd or even, 2 <= J <= 16)
 *  weight_dtype  PNP_W_C64 or PNP_W_BF16C
 *  block_host    host, M int32 data-block ids in [0, nblocks) (App. E data
 *                clustering), or NULL for one block
 *  nblocks       number of data blocks (>= 1)
 *  stream        cudaStream_t for every later call on this plan (NULL: legacy)
 * Rows are reordered internally by grid tile and block; every call takes and
 * returns visibilities in the caller's order.  Errors: INVALID_ARG, OOM, CUDA. */
int pnp_plan_create(pnp_plan** plan, int n, int K, int64_t M, const double* uvw_host,
                    double dl, const int8_t* J_per_row_host, int J, int weight_dtype,
                    const int32_t* block_host, int nblocks, void* stream);

/* The w-stacking hybrid of App. E (Eq. phip): Phi = [Phi_1; ...; Phi_P] with
 * Phi_p = G_p F Z_p.  Arguments as pnp_plan_create, plus
 *  stack_host     host, M int32 stack ids in [0, nstacks) (NULL only when M == 0
 *                 or nstacks == 1)
 *  nstacks        P in [1, 64]
 *  w_centres_host host, P float64 stack centres w_p [wavelengths] (NULL only when
 *                 nstacks == 1, meaning w_1 = 0)
 * Z_p multiplies pixel (a, b) by exp(i pi w_p dl^2 ((a - n/2)^2 + (b - n/2)^2))
 * before the grid correction; row m of stack p is w-folded with w_m - w_p only,
 * so J_per_row may be chosen from that residual.  Every operator call runs the
 * stacks one after the other through the plan's single pair of grids and sums
 * the adjoints (Eq. phidagphi).  dl must be > 0 when nstacks > 1.  Errors as
 * pnp_plan_create; stack ids out of range are PNP_ERR_INVALID_ARG. */
int pnp_plan_create_stacked(pnp_plan** plan, int n, int K, int64_t M, const double* uvw_host,
                            double dl, const int8_t* J_per_row_host, int J, int weight_dtype,
                            const int32_t* block_host, int nblocks, const int32_t* stack_host,
                            int nstacks, const double* w_centres_host, void* stream);

/* Every option of plan creation in one descriptor (zero-initialise it, then set what is
 * needed; a zero stack count or block count means 1).  The fields are those of
 * pnp_plan_create_stacked plus
 *  row_scale_host  host, M float64 data weights d_m > 0 multiplying the rows of G, or NULL
 *                  for none: Phi = D G F Z with D = diag(d).  Sec. 3 images data weighted by
 *                  the Briggs scheme (robust 0); with imaging weights w_m the data fidelity
 *                  1/2 ||D (G F Z x - y)||^2 uses d_m = sqrt(w_m), so that Re{Phi^H Phi} delta
 *                  is the weighted dirty beam and Re{Phi^H y} the weighted dirty image.
 *                  Every call of the plan then takes and returns visibilities of the weighted
 *                  model, y_m = d_m y_raw_m (pnp_plan_scale_data forms them).  Non-finite or
 *                  non-positive entries are PNP_ERR_INVALID_ARG. */
typedef struct pnp_plan_desc {
  int n, K;
  int64_t M;
  const double* uvw_host;
  double dl;
  const int8_t* J_per_row_host;
  int J;
  int weight_dtype;
  const int32_t* block_host;
  int nblocks;
  const int32_t* stack_host;
  int nstacks;
  const double* w_centres_host;
  const double* row_scale_host;
  void* stream;
} pnp_plan_desc;

int pnp_plan_create_desc(pnp_plan** plan, const pnp_plan_desc* desc);

/* y_out = D y_in for the plan's data weights D (the weighted data of the model
 * D y = D G F Z x + D n); a copy when the plan has none.  y_in, y_out: dev M
 * complex64 in the caller's order (may alias). */
int pnp_plan_scale_data(pnp_plan* plan, const float* y_in, float* y_out);

void pnp_plan_destroy(pnp_plan* plan);

int pnp_plan_get_info(const pnp_plan* plan, pnp_plan_info* info);

/* Set the rows per work unit of the gridding kernels (autotuner hook; 0 keeps
 * the current choice).  Rebuilds the work list only; G is unchanged. */
int pnp_plan_set_unit_nnz(pnp_plan* plan, int64_t unit_nnz);

/* Holographic form of the normal operator (App. E, Eq. phidagphi): with enable != 0 the plan
 * builds (once) H = G^H G, stored per grid cell as a (2 Jmax - 1)^2 stencil (device bytes
 * (2 Jmax - 1)^2 K^2 8, reported in pnp_plan_info; PNP_ERR_OOM when that does not fit), and
 * from then on pnp_fb_run forms the dirty grid G^H y once per run and iterates with
 * Re{Z^H F^H (H F Z x - G^H y)}, and op_norm with H, without reading G.  grad_step, phi_forward
 * and phi_adjoint keep using G.  enable == 0 switches back (H is kept).  Plans with several
 * w-stacks: PNP_ERR_UNSUPPORTED.  Synchronous. */
int pnp_plan_set_holographic(pnp_plan* plan, int enable);

/* Compensated summation of the gridding pass's scatter-add (G^H r, App. A; Eq. phidagphi sums
 * many rows into each grid cell).  With enable = 1 every atomic addition of a work
 * unit's partial sums into the output grid is followed by the addition of its exact rounding
 * error (TwoSum, from the value the atomic returns) into a second grid, and the adjoint FFT
 * reads the sum of the two; in dense uv cells, where thousands of rows meet, this removes the
 * error of the FP32 sums over work units.  The errors are ~2^-24 of the sums, so the second grid
 * holds them as BF16 pairs (4 bytes per cell).  enable = 0 uses plain FP32 atomics (faster: no
 * atomic waits for its result and the adjoint FFT reads one grid; at the 4096^2 / M = 2e7
 * workload the compensated flush costs 1.4 ms per iteration for an adjoint error that is at the
 * level of the FP32 FFT either way).  The plan holds the second grid either way.  Default: 0.
 * Synchronises the plan's stream. */
int pnp_plan_set_compensated(pnp_plan* plan, int enable);

/* Set how many rows of a run of rows sharing a tap window one warp of the
 * gridding pass forms the residuals of together (1, 2 or 4; 0 keeps the
 * current choice; anything else is PNP_ERR_INVALID_ARG).  Autotuner hook: a
 * performance setting only, results are unchanged (the warp sums keep their
 * pairing order).  Synchronises the plan's stream. */
int pnp_plan_set_row_batch(pnp_plan* plan, int row_batch);

/* Autotuner of the gridding pass's work decomposition (a performance setting
 * with no counterpart in the paper; results change only in the order of the
 * floating-point sums).  Times `reps` fused gridding passes on the plan's
 * stream for every triple of run cap (rows at most per run of rows sharing a
 * tap window: 3, 4, 6, 8), unit size (2^16, 2^17, 2^18 taps) and row batch
 * (rows of a run whose residuals a warp forms together: 1, 2, 4), keeps the
 * fastest and rebuilds the work list for it (G is unchanged; the chosen row
 * batch is reported by pnp_plan_get_info).  Synchronous; the output
 * grid is left cleared.  Outputs (each may be NULL): the chosen run cap and
 * unit size, and the chosen pass's mean time in ms (-1 for an empty operator).
 * reps must lie in [1, 100]. */
int pnp_plan_autotune(pnp_plan* plan, int reps, int* run_max_out, int64_t* unit_nnz_out, double* ms_out);

/* Device-side status flags of the plan's kernels (synchronous read; the flags
 * stay set for the plan's lifetime).  Each is an internal consistency check
 * that a correct plan never sets:
 *  bit 1 (2)   a wait of the gridding pass's copy pipeline ran out (bounded
 *              wait): the pass stopped early and its output is incomplete;
 *  bit 2 (4)   a chunk of the gridding work list was inconsistent and skipped;
 *  bit 4 (16)  a tap pair outside the holographic stencil was skipped while
 *              building H.
 * Taps outside their staged region are caught when the plan is built
 * (pnp_plan_create fails with PNP_ERR_INVALID_ARG). */
int pnp_plan_device_status(pnp_plan* plan, int* flags_host);

/* Per-stage CUDA-event timing (profiling aid).  While enabled, every
 * forward FFT, gridding pass and adjoint FFT issued eagerly on the plan's stream
 * is bracketed by a pair of CUDA events; launches inside CUDA-graph capture are
 * not timed.  pnp_plan_read_timing synchronises the stream and returns, per
 * stage (0 forward FFT pair, 1 gridding pass, 2 adjoint FFT pair), the summed
 * milliseconds and the number of timed launches, then clears the record. */
int pnp_plan_set_timing(pnp_plan* plan, int enable);
int pnp_plan_read_timing(pnp_plan* plan, double* ms_host /*[3]*/, int64_t* count_host /*[3]*/);

/* Copy rows of G to the host for inspection (synchronous).
 *  rows_host      host, nrows row indices in the caller's order
 *  offsets_host   host, nrows+1 int64: written with exclusive prefix sums of J_m^2
 *  weights_host   host, offsets_host[nrows] complex64 (interleaved)
 *  cols_host      host, offsets_host[nrows] int32 column indices in the
 *                 canonical grid layout (k0 mod K) * K + (k1 mod K)
 * Pass weights_host = cols_host = NULL to query offsets only. */
int pnp_plan_export_rows(const pnp_plan* plan, const int64_t* rows_host, int64_t nrows,
                         int64_t* offsets_host, float* weights_host, int32_t* cols_host);

/* ------------------------------------------------------ operator (Eq. 1) */

/* y = Phi x = G F Z x (Eq. 1).  x: dev n*n float32.  y: dev M complex64. */
int phi_forward(pnp_plan* plan, const float* x, float* y);

/* x = Re{Phi^H y} = Re{Z^H F^H G^H y} (App. A).  y: dev M complex64.  x: dev n*n. */
int phi_adjoint(pnp_plan* plan, const float* y, float* x);

/* x_out = x - gamma Re{Phi^H (Phi x - y)}: the forward (gradient) step of
 * Eq. fb with the gradient of App. A; one pass over G computes the residual
 * and its gridding.  x, x_out: dev n*n (may not alias).  y: dev M complex64. */
int grad_step(pnp_plan* plan, const float* x, const float* y, double gamma, float* x_out);

/* L = ||Re{Phi^H Phi}||_S by power iteration (App. A), FP64 norms.
 *  v0       dev n*n float32 start vector, or NULL for all ones
 *  max_it   iteration cap (>= 1); tol: stop when |L_k - L_{k-1}| <= tol L_k
 *  L_out    host, receives L (synchronous)
 *  iters_out host, receives the iteration count (may be NULL) */
int op_norm(pnp_plan* plan, const float* v0, int max_it, double tol, double* L_out,
            int* iters_out);

/* ------------------------------------------------------------- denoisers */

/* Plain denoiser: one-level orthonormal 2-D Haar on 2x2 blocks, soft-threshold
 * of all four subbands at t, synthesis, then positivity (App. B with the
 * threshold gamma*lambda = tau / sqrt(2L) of Eq. lambda).  t >= 0. */
int pnp_den_create_haar(pnp_den** den, double t, void* stream);

/* Learned denoiser (App. C): residual CNN, 8 layers 3x3, 1->64->...->64->1,
 * ReLU between layers, D(z) = max(0, z - N(z)), applied on facets with a halo
 * (App. D).
 *  weights_host  host float32, the 8 layers' (W, b) concatenated: layer l
 *                stores W[co][ci][3][3] then b[co]; shapes 64x1, 6 x 64x64, 1x64
 *  facet_rows_host / facet_cols_host  host int32 facet core sizes along each
 *                axis (sum n), or NULL for the whole image as one facet
 *  nfr, nfc      number of facet sizes given per axis
 *  halo          facet overlap in pixels (>= 8 makes faceting exact)
 *  n             image side the denoiser will be applied to */
int pnp_den_create_cnn(pnp_den** den, const float* weights_host,
                       const int32_t* facet_rows_host, int nfr,
                       const int32_t* facet_cols_host, int nfc, int halo, int n, void* stream);

/* Work decomposition of a CNN denoiser (a performance setting: the results do not depend on it, bit
 * for bit).  Each convolution layer walks strips of one 128-pixel column segment by about `rows`
 * output rows of a facet (the last layer: of a facet core); a strip stages rows + 2 input rows, so
 * taller strips re-read fewer halo rows and shorter ones balance the SMs better.  Default 32.
 *  rows   in [4, 1024]; PNP_ERR_INVALID_ARG otherwise or for a denoiser that is not a CNN.
 * Synchronises the device (work lists in use by launches in flight are not overwritten). */
int pnp_den_cnn_set_strip_rows(pnp_den* den, int rows);
/* Autotuner of the strip height above: times `reps` denoises (after one warm-up) of the device
 * n x n image z for each of 16, 24, 32, 48, 64 and 96 rows on the denoiser's stream (CUDA events),
 * keeps the fastest and returns it with its time per denoise (rows_out, ms_out may be NULL).
 * Allocates and frees one n x n scratch image.  reps in [1, 100]. */
int pnp_den_cnn_autotune(pnp_den* den, const float* z, int n, int reps, int* rows_out, double* ms_out);

/* uSARA's denoiser (App. B): the prox of gamma_lambda ||W Psi^T x||_1 + iota_+(x) for the SARA
 * dictionary Psi (the Dirac basis and the 2-D Daubechies db1..db8 bases, each a `levels`-level
 * separable DWT with periodic extension, divided by 3 so that Psi Psi^T = I), computed by
 * `prox_iters` dual forward-backward iterations x = max(0, z - Psi u), u <- clip(u + Psi^T x,
 * -gamma_lambda w, gamma_lambda w) warm-started from the previous call's u.  The weights w start
 * at 1; pnp_den_sara_reweight sets w = rho / (rho + |Psi^T x|), the majoriser of the log-sum prior
 * at x (Eq. lambda: gamma_lambda = tau / sqrt(2L), rho = gamma_lambda).
 *  n          image side, a multiple of 2^levels with n / 2^levels >= 1;  levels in [1, 8]
 *  prox_iters >= 1
 * Device memory: 2 x 9 n^2 + 4 n^2 floats.  Used by denoise() and pnp_fb_run like the others. */
int pnp_den_create_sara(pnp_den** den, int n, int levels, double gamma_lambda, double rho, int prox_iters,
                        void* stream);
/* w = rho / (rho + |Psi^T x|) for the device n x n image x (the reweighting step of uSARA). */
int pnp_den_sara_reweight(pnp_den* den, const float* x);
/* The SARA dictionary of a SARA denoiser: direction 1 writes Psi^T in (device, 9 x n x n, basis
 * order Dirac, db1, ..., db8; each DWT's coefficients in one n x n array, the level's approximation
 * in the top-left corner and its details beside and below it); direction -1 writes Psi in
 * (in: 9 x n x n, out: n x n). */
int pnp_sara_transform(pnp_den* den, const float* in, float* out, int direction);

void pnp_den_destroy(pnp_den* den);

/* Device status flags of a denoiser's kernels (synchronous; 0 for the Haar
 * denoiser).  Bit 1: a bounded pipeline wait in the tensor-core convolution
 * gave up (the output of that call is invalid). */
int pnp_den_device_status(pnp_den* den, int* flags_host);

/* x_out = D(x_in) for an n x n image (dev float32; may not alias). */
int denoise(pnp_den* den, const float* x_in, float* x_out, int n);

/* ------------------------------------------------------- CNN training */

/* Trainer of the residual CNN denoiser (App. C): minimises the l1 loss
 * mean |D(u + sigma n) - u|, D(z) = z - N(z), with Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8); the firm non-expansiveness term of Eq. training_loss is not
 * included.  Weights are FP32 master copies rounded to BF16 for every
 * convolution; activations and back-propagated gradients are BF16.
 *  weights_host  FP32 parameters in the layout of pnp_den_create_cnn
 *                (pnp_cnn_num_params() values)
 *  batch, size   images per step and their side (size >= 8)
 *  lr            Adam step size */
typedef struct pnp_cnn_trainer pnp_cnn_trainer;
int pnp_cnn_trainer_create(pnp_cnn_trainer** trainer, const float* weights_host, int batch, int size,
                           double lr, void* stream);
void pnp_cnn_trainer_destroy(pnp_cnn_trainer* trainer);

/* One step: z = u + sigma n, forward, loss, backward; with update != 0 also an
 * Adam update (which clears the gradients).
 *  u, noise   dev, batch x size x size float32: clean images and N(0,1) draws
 *  loss_host  host, receives the mean l1 loss (synchronous), or NULL */
int pnp_cnn_train_step(pnp_cnn_trainer* trainer, const float* u, const float* noise, double sigma, int update,
                       double* loss_host);

/* Copy the FP32 weights and/or accumulated gradients to the host (synchronous;
 * NULL skips one); clear_grads != 0 zeroes the gradients afterwards.  Returns
 * PNP_ERR_TIMEOUT if a bounded device wait gave up during training. */
int pnp_cnn_trainer_read(pnp_cnn_trainer* trainer, float* weights_host, float* grads_host, int clear_grads);

/* One Adam step (the update of pnp_cnn_train_step with update != 0) on the gradients accumulated
 * so far, e.g. by steps with update = 0 whose gradients the caller has read; clears them. */
int pnp_cnn_trainer_apply_update(pnp_cnn_trainer* trainer);

/* Set the Adam step size used by later pnp_cnn_train_step calls (lr > 0); the
 * moment estimates and the step count are kept. */
int pnp_cnn_trainer_set_lr(pnp_cnn_trainer* trainer, double lr);

/* Spectral norm of the Jacobian of Q = 2D - I, D(z) = z - N(z), at each image of a batch: the
 * quantity the firm non-expansiveness constraint of Eq. training_loss (App. C) bounds by 1.
 * Runs `iters` power iterations on J_Q^T J_Q with J_Q = I - 2 J_N, J_N the network with its
 * ReLU masks at z frozen (Jacobian-vector products on the tensor cores, BF16 tangents and
 * gradients as in training), independently per image.
 *  z          device, batch x size x size float32 inputs (the trainer's batch geometry)
 *  v0         device, batch x size x size float32 start vectors (normalised per image)
 *  iters      >= 1
 *  sigma_host host, batch float64: ||J_Q v|| for the last unit iterate v (the estimate)
 *  v_out      device, batch x size x size float32 or NULL: the last iterate, normalised
 * Overwrites the trainer's activations and gradient canvases; synchronous. */
int pnp_cnn_jacobian_norm(pnp_cnn_trainer* trainer, const float* z, const float* v0, int iters,
                          double* sigma_host, float* v_out);

/* One training step with the soft firm non-expansiveness penalty of Eq. training_loss (App. C,
 * the constraint relaxed to a penalty as the paper describes): the l1 loss of
 * pnp_cnn_train_step plus
 *   P = lambda / batch * sum_b max(||J_Q(z_b) v_b||^2, 1 - eps),   z = u + sigma n,
 * with v_b the unit vector after `iters` power iterations on J_Q^T J_Q at z_b from v0 (iters = 0:
 * v0 normalised), held fixed; P's weight gradients come from back-propagating -4 lambda/batch
 * J_Q v through the frozen-mask network (biases get none).  Arguments as pnp_cnn_train_step, plus
 *  v0           device, batch x size x size float32 start vectors
 *  iters        >= 0;  lambda >= 0;  eps in [0, 1]
 *  penalty_host host float64 or NULL: P (synchronous when given) */
int pnp_cnn_train_step_fne(pnp_cnn_trainer* trainer, const float* u, const float* noise, double sigma,
                           const float* v0, int iters, double lambda, double eps, int update,
                           double* loss_host, double* penalty_host);

/* Number of FP32 parameters of the CNN (weights and biases of the 8 layers). */
int64_t pnp_cnn_num_params(void);

/* ------------------------------------------------------------ PnP-FB loop */

/* Run Eq. fb: x^{k+1} = D(x^k - gamma Re{Phi^H (Phi x^k - y)}), starting from
 * x_inout (dev n*n float32, overwritten with the result).  y: dev M complex64.
 * params may leave gamma and L at 0 to derive them (App. B).  stats (host)
 * may be NULL.  Returns PNP_ERR_DIVERGED if the iterate becomes non-finite or
 * grows past params->diverge_factor. */
int pnp_fb_run(pnp_plan* plan, pnp_den* den, const float* y, const pnp_params* params,
               float* x_inout, pnp_stats* stats);

/* Allocation-free plain denoiser with stopping-test norms.  The paper has no
 * counterpart: this call exists for callers that cannot allocate device memory
 * (code running under a fixed, pre-reserved memory budget or a caller-owned
 * pool, or a host runtime that forbids allocation after start-up).  It applies
 * the same Haar soft-threshold + positivity as the Haar denoiser to z (dev
 * n*n float32) and writes x_out (dev n*n), and writes into norms (dev, 2
 * doubles) the FP64 sums ||x_out - x_prev||^2 (0 when x_prev is NULL) and
 * ||x_out||^2, summed in a fixed order.  It calls no cudaMalloc/cudaFree and
 * no allocating library routine: its scratch (two doubles per pair of image
 * rows) is a static device array of 128 KiB that every GPU loading the library
 * holds until exit.  Limit: n even, 2 <= n <= 16384; larger n is rejected with
 * PNP_ERR_INVALID_ARG, and so are z or x_prev overlapping x_out.  Every call
 * looks up the array's device address (cudaGetSymbolAddress, which allocates
 * nothing) with the caller's device current, so the address stays right after
 * the device's context is recreated; the first lookup on a device may load the
 * library's device code, so make the first call on each device before any
 * stream capture.  Every call shares the array: calls that overlap on the GPU
 * race and must be serialised by the caller.  A non-finite z makes
 * norms[1] NaN (the signal the stopping test reads).  Asynchronous on stream
 * (NULL: legacy default stream). */
int pnp_haar_denoise_noalloc(const float* z, const float* x_prev, float* x_out, int n, double t,
                             double* norms, void* stream);

/* Thread-local message of the last failing call ("" if none). */
const char* pnp_last_error(void);

/* Number of this library's kernels launched by the calling process so far. */
int64_t pnp_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* PNP_H */
