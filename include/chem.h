/*
 * libchem -- GB300 (sm_103a) per-cell chemistry step: C ABI.
 *
 * The operation is the paper's chemistry step (Sec. 2.2): each cell's state (T, p, Y_k)
 * is advanced over one flow time step dt by integrating the reaction system of Eq. 1,
 * producing the input -> output map of Eq. 2.  Beside it sit the mixture thermo/transport
 * properties the paper updates on the GPU (Sec. 2.1, "Newton's method and high-order
 * temperature polynomials").
 *
 * Conventions for every entry point
 *   - Array arguments are DEVICE pointers owned by the caller; the library never frees them
 *     and never keeps them after the call returns (the work is enqueued on `stream`).
 *   - States are FP64 structure-of-arrays, species-major: Y[k * ld + i] is species k of cell
 *     i; T[i], p[i] per cell; ld >= n.  Units are SI: K, Pa, kg/m^3, J/kg, W/m/K, Pa s, s.
 *   - Every call is asynchronous on `stream` (NULL = the legacy default stream) and returns
 *     0 on success or a negative CHEM_E* code; chem_last_error() then gives a message
 *     (thread-local).  Kernel-side problems of a single cell never fail the call: they are
 *     reported in the caller's int32 status[] array (codes below).  No kernel traps; every
 *     device loop is bounded.
 *   - Opaque handles are owned by the library and released by their *_free function.
 */
#ifndef CHEM_H
#define CHEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* chem_stream;   /* same object as cudaStream_t */
typedef struct chem_mech_s* chem_mech;

/* return codes */
#define CHEM_OK 0
#define CHEM_E_ARG -1      /* bad argument (null pointer, size, ld < n, ...) */
#define CHEM_E_PARSE -2    /* mechanism file unreadable or malformed */
#define CHEM_E_CUDA -3     /* a CUDA runtime call failed (message says which) */
#define CHEM_E_NOMEM -4    /* device allocation for library-owned tables failed */
#define CHEM_E_WORKSPACE -5 /* workspace missing or smaller than chem_workspace_bytes() */
#define CHEM_E_UNSUPPORTED -6 /* mechanism larger than the compiled kernels support */

/* per-cell status codes written to status[] */
#define CHEM_CELL_OK 0
#define CHEM_CELL_MAX_STEPS 1    /* step budget (opts.max_steps) exhausted */
#define CHEM_CELL_STEP_FAIL 2    /* step size underflow after Newton / error-test failures */
#define CHEM_CELL_NONFINITE 3    /* non-finite input or result; state left unchanged */
#define CHEM_CELL_OUT_OF_RANGE 4 /* input outside the model's validity (T, p, Y) */
#define CHEM_CELL_ANN_FALLBACK 5 /* the learned step flagged the cell; DI result written */

/* Library limits of the compiled kernels. */
#define CHEM_MAX_SPECIES 63      /* n = species + 1 <= 64 unknowns per cell */
#define CHEM_MAX_REACTIONS 1024

/* ---------------------------------------------------------------------------------------- */
/* Mechanism                                                                                */
/* ---------------------------------------------------------------------------------------- */
/* Parse a mechanism file (this project's plain-text SI format: elements, species with
 * molar masses and compositions, two-range NASA-7 coefficients, transport fits
 * ln(mu), ln(lambda) = sum_n b_n (ln T)^n, reactions with Arrhenius A [m,mol,s], b,
 * Ea [J/mol], third-body efficiencies, Troe low-pressure limits and parameters),
 * validate element balance, and upload the device tables to the current device.
 * *out receives a handle owned by the library.  Returns CHEM_E_PARSE on malformed input. */
int chem_load_mech(const char* path, chem_mech* out);
void chem_free_mech(chem_mech mech);
int chem_mech_info(chem_mech mech, int* n_species, int* n_reactions, int* n_elements);

/* ---------------------------------------------------------------------------------------- */
/* Reaction rates (Eq. 1 right-hand side)                                                   */
/* ---------------------------------------------------------------------------------------- */
/* Net molar production rates wdot[k * ld + i] (mol/m^3/s) and, if hrr is not NULL, the heat
 * release rate hrr[i] = -sum_k h_k wdot_k (W/m^3) of n cells at (T[i], p[i], Y[:, i]).
 * Forward rates k = A T^b exp(-Ea/RT) (third-body [M] = sum_k alpha_k C_k; Lindemann falloff
 * with the Troe form), reverse rates from K_c = exp(-sum nu g/RT) (p0/RT)^{sum nu},
 * p0 = 101325 Pa, all in FP64. */
int chem_rates(chem_mech mech, int64_t n, int64_t ld, const double* T, const double* p,
               const double* Y, double* wdot, double* hrr, chem_stream stream);

/* Analytic Jacobian of the constant-pressure reactor right-hand side, z = (Y_1..Y_K, T):
 * jac[i * nn + r * nn_row + c] is d f_r / d z_c of cell i with nn_row = K + 1 and
 * nn = (K + 1)^2 (row-major per cell, cells contiguous).  Exposed for parity testing. */
int chem_jacobian(chem_mech mech, int64_t n, int64_t ld, const double* T, const double* p,
                  const double* Y, double* jac, chem_stream stream);

/* ---------------------------------------------------------------------------------------- */
/* Direct integration (Eq. 2)                                                               */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
  double rtol;       /* relative tolerance (default 1e-9 when <= 0) */
  double atol_Y;     /* absolute tolerance on mass fractions (default 1e-18 when <= 0) */
  double atol_T;     /* absolute tolerance on T in K (default 1e-9 when <= 0) */
  double newton_tol; /* Newton stop: estimated remaining correction in units of the local
                        error test (default 0.2 when <= 0) */
  int max_steps;     /* per-cell step budget (default 20000 when <= 0) */
  int jac_max_age;   /* accepted steps a Jacobian is reused before it is re-evaluated (default
                        100 when <= 0; a Newton failure with a stale Jacobian refreshes it
                        earlier) */
} chem_di_opts;

/* Advance cells over dt by direct integration of the closed, adiabatic, constant-pressure
 * reactor (Eq. 1 with dT/dt = -sum_k h_k wdot_k / (rho c_p)), in place: T[i] and Y[:, i]
 * are overwritten with the state at t + dt; p[i] is constant.  Variable-order (1..5) BDF
 * with a modified Newton iteration (analytic Jacobian, dense LU with partial pivoting, all
 * FP64), one warp per cell.
 *   idx      NULL to integrate cells 0..n-1, else int32 idx[n] lists the cell columns to
 *            integrate (indices into the ld-strided arrays, each < ld).
 *   opts     NULL for defaults.
 *   status   int32 status[n] (per entry of idx, or per cell), CHEM_CELL_* codes; cells whose
 *            status is non-zero keep their input state.
 *   stats    NULL, or int32 stats[4 * n]: steps, RHS evaluations, Jacobian evaluations and
 *            LU factorisations per cell (stats[k * n + i]), for work accounting.
 *   workspace device scratch of at least chem_workspace_bytes(mech, n) bytes (the cell work
 *            queue); it must not be used by another call in flight.
 * Returns CHEM_E_WORKSPACE if the workspace is missing or too small. */
int chem_step_di(chem_mech mech, int64_t n, int64_t ld, double dt, double* T, const double* p,
                 double* Y, const int32_t* idx, const chem_di_opts* opts, int32_t* status,
                 int32_t* stats, void* workspace, size_t ws_bytes, chem_stream stream);

/* Device scratch needed by chem_step_di for n cells (bytes). */
size_t chem_workspace_bytes(chem_mech mech, int64_t n);

/* chem_step_di for callers that cannot allocate device memory (the paper has no
 * counterpart: this is a library convenience).  Such callers include flow solvers in Fortran
 * or C that link this ABI directly after giving all free HBM to their own memory pool, and
 * time-step loops that must avoid cudaMalloc/cudaFree because those calls synchronise the
 * device.  Same arguments and results as chem_step_di, without the workspace: the scratch
 * (the cell work-queue counter) lives in a fixed 256-byte device array inside this library,
 * held by every GPU that loads the library until the process exits.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   - Every call looks up the array's device address (cudaGetSymbolAddress) in the CUDA
 *     context current on the calling thread, so a device reset or another context made
 *     current on the device between calls is followed correctly.
 *   - All calls share the one array: the call clears the counter on `stream` before its
 *     launch, but calls whose work overlaps on the GPU (other streams, other threads) race
 *     on it and must be serialised by the caller.
 *   - The array always holds the call's scratch; n is limited to 2^31 - 1 cells per call by
 *     the 32-bit work-queue counter (CHEM_E_ARG beyond), otherwise the codes of
 *     chem_step_di. */
int chem_step_di_noalloc(chem_mech mech, int64_t n, int64_t ld, double dt, double* T,
                         const double* p, double* Y, const int32_t* idx,
                         const chem_di_opts* opts, int32_t* status, int32_t* stats,
                         chem_stream stream);

/* ---------------------------------------------------------------------------------------- */
/* Learned reaction step (Sec. 2.2: MLP with GELU hidden layers, Box-Cox inputs, Eq. 7,     */
/* lambda = 0.1; loss Eqs. 8-9; Adam) in BF16 on the tensor cores, with DI fallback         */
/* ---------------------------------------------------------------------------------------- */
typedef struct chem_ann_s* chem_ann;

/* Inputs x = [T, p, F(Y_1..Y_K)] (F = Box-Cox), z-scored with the training statistics and
 * stored BF16 [n, 64] (zero padded).  Outputs u_k = (F(Y_k(t+dt)) - F(Y_k(t)) - mu_k)/sigma_k,
 * FP32 [n, n_out_pad] with n_out_pad = 32 (K <= 32) or 64.  Normalisation block (floats):
 * in_mean[n_in], in_std[n_in], in_min[n_in], in_max[n_in], out_mean[K], out_std[K],
 * n_in = K + 2.
 * chem_ann_create: n_hidden GELU layers of hidden[l] units (1..8192 each; widths that are not
 * multiples of 8 are stored rounded up with zero-weight units that stay zero, so chem_ann_info
 * reports the stored widths), weights N(0, 2/fan_in), zero biases, seeded. */
int chem_ann_create(chem_mech mech, const int* hidden, int n_hidden, uint64_t seed, chem_ann* out);
/* One network per species (Sec. 2.2: each species' transformed mass fraction is trained and
 * predicted by its own MLP, hidden widths 1600, 800, 400): K networks of the given hidden
 * widths with one output each, sharing the input x.  Their weights are stored stacked by
 * species (layer l: W [K dims[l+1], dims[l]], species k in rows k dims[l+1] ..), the first
 * layer runs as one GEMM over all species' units and every later layer as one launch of K
 * GEMMs; outputs, normalisation, checks, training options and the rest of the API are those
 * of chem_ann_create's network, and the loss of Eq. 11 sums over the species as for it (with
 * w_mass = w_hrr = 0 training the K networks jointly equals training each one alone).
 * chem_ann_info reports the widths of one species' network (output width 1). */
int chem_ann_create_per_species(chem_mech mech, const int* hidden, int n_hidden, uint64_t seed,
                                chem_ann* out);
/* groups: 1 for chem_ann_create's network, K for per-species networks; n_out_pad: columns of
 * the output rows U (32 or 64). */
int chem_ann_layout(chem_ann ann, int* groups, int* n_out_pad);
void chem_ann_free(chem_ann ann);
int chem_ann_info(chem_ann ann, int* n_in, int* n_out, int* n_layers, int* dims /* [n_layers+1] */,
                  int64_t* n_params);
int chem_ann_set_norm(chem_ann ann, const float* host_norm);
int chem_ann_get_norm(chem_ann ann, float* host_norm);
/* Fit the normalisation (mean, std, min, max of inputs; mean, std of F-increments) on the
 * training states (T, p, Y0) and their DI results Y1 (device, SoA, ld-strided). */
int chem_ann_fit_norm(chem_ann ann, int64_t n, int64_t ld, const double* T, const double* p,
                      const double* Y0, const double* Y1, chem_stream stream);
/* Normalised BF16 features X [n, 64]; if bcty is not NULL also the raw F(Y) as FP32 [n, K]
 * (needed by the mass term of the loss).  If flags is not NULL, flags[i] receives the range
 * flag of the learned step (1 when a raw feature of cell i lies outside [min - m (max - min),
 * max + m (max - min)] of the training set, m = range_margin >= 0; else 0): the first stage
 * of chem_step_ann, exposed so that its stages can be run and checked one by one. */
int chem_ann_features(chem_ann ann, int64_t n, int64_t ld, const double* T, const double* p,
                      const double* Y, void* X, float* bcty, double range_margin, int32_t* flags,
                      chem_stream stream);
/* Normalised FP32 targets U [n, n_out_pad] from the states before (Y0) and after (Y1) DI. */
int chem_ann_targets(chem_ann ann, int64_t n, int64_t ld, const double* Y0, const double* Y1,
                     float* U, chem_stream stream);
/* Raw network output U [n, n_out_pad] for features X [n, 64] (workspace as chem_step_ann). */
int chem_ann_forward(chem_ann ann, const void* X, int64_t n, float* U, void* workspace,
                     size_t ws_bytes, chem_stream stream);

typedef struct {
  float lr, beta1, beta2, eps;   /* Adam */
  float w_data, w_mass;          /* Eq. 11 weights of L_data (Eq. 8) and L_mass (Eq. 9) */
  int apply;                     /* 0: gradients only (chem_ann_get_params(which = 1)) */
  float w_hrr;                   /* Eq. 11 weight of L_HRR (Eq. 10); 0 leaves the term out */
} chem_train_opts;

/* Per-sample coefficients of L_HRR (Eq. 10), read as the step-mean heat release
 * HRR = -(rho / dt) sum_k h_k(T0) (Y_k(t+dt) - Y_k(t)) with mass enthalpies at the initial
 * temperature and rho = p / (R T0 sum_k Y0_k / W_k):  hrr_c [n, K] = -rho (h_k - hbar) /
 * (dt scale), hbar = sum_k Y0_k h_k (a shift that leaves the heat release of mass-conserving
 * changes unchanged and keeps mass-sum errors out of the term), and the DI target
 * hrr_r [n] = sum_k hrr_c (Y1 - Y0), both FP32 in units of `scale` (W/m^3, e.g. the RMS heat
 * release of the training set; pass 1 to obtain raw values). */
int chem_ann_hrr_coeffs(chem_ann ann, int64_t n, int64_t ld, const double* T0, const double* p,
                        const double* Y0, const double* Y1, double dt, double scale, float* hrr_c,
                        float* hrr_r, chem_stream stream);

/* One optimisation step on a minibatch: X [B, 64] BF16, targets Ut [B, n_out_pad] FP32,
 * bcty [B, K] FP32 raw F(Y) (NULL unless w_mass or w_hrr != 0), hrr_c [B, K] and hrr_r [B]
 * from chem_ann_hrr_coeffs (NULL unless w_hrr != 0), B a multiple of 8.  The loss is
 * L = w_data L_data + w_mass L_mass + w_hrr L_HRR with L_HRR = mean_b e_b^2,
 * e_b = sum_k hrr_c (Y*_k - Y_k(t)) - hrr_r.  loss_out (device, nullable) receives
 * {L_tot, L_data, L_mass, L_HRR}.  The library keeps its training buffers. */
int chem_ann_train_step(chem_ann ann, const void* X, const float* Ut, const float* bcty,
                        const float* hrr_c, const float* hrr_r, int64_t B,
                        const chem_train_opts* opts, float* loss_out, chem_stream stream);
/* One training epoch over n_samples rows (X [n, 64] BF16, Ut [n, n_out_pad], bcty [n, K]
 * (NULL unless w_mass or w_hrr != 0), hrr_c [n, K] and hrr_r [n] (NULL unless w_hrr != 0),
 * all device arrays): the rows are visited in a seeded random order -- a permutation of
 * 0..n-1 drawn per (seed, epoch) on the device, no table -- in floor(n / batch) minibatches,
 * each gathered into library-owned buffers and taken through chem_ann_train_step's
 * optimisation step, with the learning rate on a cosine schedule
 *   lr(t) = lr_min + (lr - lr_min) (1 + cos(pi t / (total_steps - 1))) / 2,
 * t = step0 + the step's index in the epoch (clamped to total_steps - 1).  The paper trains
 * its networks with Adam on the loss of Eqs. 8-11 over 1600 epochs (Sec. 2.2, Sec. 4).
 * loss_out (device, nullable) receives the epoch means of {L_tot, L_data, L_mass, L_HRR}.
 * Rows beyond the last full minibatch are not visited in this epoch (they are in others, the
 * order changing per epoch). */
typedef struct {
  chem_train_opts step;   /* Adam and loss weights; step.lr is the schedule's peak */
  int64_t batch;          /* minibatch rows, a multiple of 8 in [8, 2^20], <= n_samples */
  float lr_min;           /* end of the cosine schedule */
  int64_t total_steps;    /* schedule length over all epochs (<= 0: this epoch's steps) */
  int64_t step0;          /* schedule position of this epoch's first step */
  uint64_t seed;          /* minibatch order: one permutation per (seed, epoch) */
  int epoch;
  int reserved;
} chem_train_epoch_opts;
int chem_ann_train_epoch(chem_ann ann, const void* X, const float* Ut, const float* bcty,
                         const float* hrr_c, const float* hrr_r, int64_t n_samples,
                         const chem_train_epoch_opts* opts, float* loss_out, chem_stream stream);

/* Flat FP32 parameters (which = 0) or last gradients (which = 1), per layer W [out, in] then b
 * (per-species networks: W [K out, in] and b [K out], stacked by species). */
int chem_ann_get_params(chem_ann ann, int which, float* host, int64_t count);
int chem_ann_set_params(chem_ann ann, const float* host, int64_t count);
/* Checkpoint (weights, normalisation, Adam step and, if with_moments, the Adam moments; a
 * checkpoint without moments resumes Adam from zero moments) and its reload. */
int chem_ann_save(chem_ann ann, const char* path, int with_moments);
int chem_ann_load(chem_mech mech, const char* path, chem_ann* out);
/* Device error flag of the tensor-core pipelines (non-zero: a wait timed out); reading clears it. */
int chem_ann_error(chem_ann ann, int* host_err);

typedef struct {
  double range_margin;  /* inputs outside [min - m (max-min), max + m (max-min)] fall back (0.05) */
  double elem_tol;      /* max relative change of element moles accepted before the prediction
                           is projected onto exact element conservation (1e-2) */
  double T_min, T_max;  /* accepted new temperature range (250, 3500 K) */
  double dT_max;        /* if > 0, |T_new - T| above it falls back */
  int no_fallback;      /* 1: flagged cells keep their input state (status 5), no DI */
  int reserved;
  chem_di_opts di;      /* options of the fallback direct integration */
} chem_ann_opts;

/* Learned chemistry step for n cells in place (layout and idx as chem_step_di: NULL, or the
 * n cell columns to process; status[] is per entry): features, the MLP
 * on the tensor cores, the new state (inverse Box-Cox, renormalisation, T from enthalpy
 * conservation by Newton's method) and its checks; flagged cells are integrated by DI
 * (status CHEM_CELL_ANN_FALLBACK when DI succeeded, else DI's code).  Workspace:
 * chem_ann_workspace_bytes(ann, n). */
int chem_step_ann(chem_mech mech, chem_ann ann, int64_t n, int64_t ld, double dt, double* T,
                  const double* p, double* Y, const int32_t* idx, const chem_ann_opts* opts,
                  int32_t* status, void* workspace, size_t ws_bytes, chem_stream stream);
size_t chem_ann_workspace_bytes(chem_ann ann, int64_t n);

/* The update stage of chem_step_ann on given network outputs U [n, n_out_pad] (FP32, rows by
 * entry of idx or by cell; from chem_ann_forward), in place on T and Y (layout and idx as
 * chem_step_ann).  The paper defines the output as the change of the Box-Cox transformed
 * species over dt (Sec. 2.2, Eq. 7); T follows from the adiabatic constant-pressure energy
 * balance.  Per cell, in FP32:
 *   1. Y*_k = F^-1(F(Y_k) + sigma_k U_k + mu_k), 0 where the inverse's base is <= 0; a
 *      non-finite argument or a sum of Y* that is not finite and positive sets bit 2 and
 *      ends the cell;
 *   2. Y* /= sum Y*; the largest relative change of element moles over the elements present
 *      in Y above opts->elem_tol sets bit 4;
 *   3. without bit 4, Y* is projected onto exact element conservation (the least-squares
 *      change weighted by 1/Y*_k, clipped at 0);
 *   4. T' solves h(T', Y*) = h(T, Y) by Newton's method; T' non-finite sets bit 2, else T'
 *      outside [T_min, T_max] bit 8, else |T' - T| > dT_max (when dT_max > 0) bit 16.
 * flags (in/out, int32 [n]): on input the range flag (bit 1, e.g. from chem_ann_features;
 * 0 to skip the range check); a cell with a non-zero input flag is left alone.  On output
 * the flag word; status[] = 0 for accepted cells (T, Y overwritten) and
 * CHEM_CELL_ANN_FALLBACK for flagged ones (T, Y unchanged; chem_step_ann then integrates
 * them by DI).  opts NULL selects the defaults (fields as chem_ann_opts; range_margin, di
 * and no_fallback are not used here). */
int chem_ann_update(chem_ann ann, int64_t n, int64_t ld, double* T, const double* p, double* Y,
                    const float* U, const int32_t* idx, const chem_ann_opts* opts, int32_t* flags,
                    int32_t* status, chem_stream stream);

/* ---------------------------------------------------------------------------------------- */
/* Serving loop: continuous batching of chemistry-step requests (the paper keeps fields      */
/* device-resident and bounds GPU memory with a dynamic inference batch, Sec. 2.1)          */
/* ---------------------------------------------------------------------------------------- */
typedef struct chem_server_s* chem_server;

typedef struct {
  size_t hbm_budget_bytes;  /* device memory the server may hold (arenas + workspaces) */
  int n_streams;            /* concurrent batches in flight (1..16) */
  int max_batch_cells;      /* cells per launch and per request (index-list capacity) */
  double starvation_s;      /* > 0: once the oldest waiting request has waited this long,
                               nothing newer is admitted past it, and once an admitted request
                               has waited this long its kind is launched next */
  int di_chunk_cells;       /* cells of one direct-integration request per launch (0: 32768) */
  int reserved;
} chem_server_opts;

typedef struct {
  int64_t submitted, completed, failed, cells, batches;
  double mean_batch_requests;
  double p50_ms, p99_ms, mean_ms, max_ms;   /* latency: submit -> results in host memory */
  double wall_s, cells_per_s, hbm_bytes;
} chem_server_stats;

/* A background host thread admits requests into per-class device arenas (first-fit column
 * ranges within the HBM budget) and, whenever a stream is idle, launches one batch over
 * pieces of the admitted requests of one kind (class, mode, dt) through an index list: the
 * kind of the request with the least work left (or of one past starvation_s), its requests
 * smallest remainder first, a direct-integration request contributing at most
 * di_chunk_cells per launch and a batch at most max_batch_cells.  Each piece's results are
 * copied back when its launch ends; a request completes with its last piece and frees its
 * columns.  Host arrays passed to chem_server_submit must stay valid until the request
 * completes.  Pass pinned (page-locked) host memory: a copy from or to pageable memory blocks
 * the scheduler thread until it ends, which serialises the streams.  Per-cell results do not
 * depend on the batch composition or on the piece a cell runs in. */
int chem_server_create(const chem_server_opts* opts, chem_server* out);
/* Register a class: a mechanism (and optionally a trained ANN for mode 1) with an arena of
 * capacity_cells columns.  Classes are added before the first submit. */
int chem_server_add_class(chem_server server, chem_mech mech, chem_ann ann, int64_t capacity_cells,
                          int* class_id);
/* Queue one request: mode 0 = direct integration, 1 = learned step with fallback; n cells
 * (at most the class arena's capacity) of host SoA state T[n], p[n], Y[K][n] (species-major,
 * ld = n); results to T_out, Y_out, status_out (host).  Non-blocking. */
int chem_server_submit(chem_server server, int class_id, int mode, double dt, int64_t n,
                       const double* T, const double* p, const double* Y, double* T_out,
                       double* Y_out, int32_t* status_out, int64_t* request_id);
/* Block until the request completes or timeout_s passes; *done = 1 if complete, *result =
 * the request's API result (CHEM_OK, or the error code of its launch). */
int chem_server_wait(chem_server server, int64_t request_id, double timeout_s, int* done,
                     int* result);
int chem_server_get_stats(chem_server server, chem_server_stats* stats);
/* Latency of one request (submit -> results on the host) in ms; -1 while it is not done. */
int chem_server_request_latency(chem_server server, int64_t request_id, double* latency_ms);
void chem_server_free(chem_server server);

/* ---------------------------------------------------------------------------------------- */
/* Mixture thermo and transport properties (Sec. 2.1)                                        */
/* ---------------------------------------------------------------------------------------- */
/* Per cell: c_p [J/kg/K] and h [J/kg] (mass-weighted NASA-7), Wilke mixture viscosity mu
 * [Pa s] and the mixture-averaged conductivity kappa = (sum X_k lambda_k + 1/sum X_k/lambda_k)/2
 * [W/m/K], with ln(mu_k), ln(lambda_k) cubic in ln T.  Each output may be NULL.
 * If h_in is not NULL, T is first solved from h(T, Y) = h_in[i] by Newton's method starting
 * at T[i] (|dT| < 1e-9 K, at most 50 iterations, clamped to [200, 6000] K), written to T_out
 * (which may alias T), and the properties are evaluated there.
 * All FP64 when mixed_precision == 0; with mixed_precision == 1 the O(K^2) Wilke and the
 * conductivity sums run in FP32 (relative error below 1e-5) while c_p, h and the Newton
 * solve stay FP64. */
int thermo_props(chem_mech mech, int64_t n, int64_t ld, const double* T, const double* Y,
                 double* cp, double* h, double* mu, double* kappa, const double* h_in,
                 double* T_out, int mixed_precision, chem_stream stream);

/* ---------------------------------------------------------------------------------------- */
/* Random augmentation of training states (the hybrid flamelet/random data method, Sec. 2.2,*/
/* Eqs. 3-6, with the constraints of the same passage)                                       */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
  double alpha, beta, theta;   /* Eqs. 3-6 (0.125, 10, 0.1) */
  double hc[2];                /* accepted molar H/C ([2.65, 4.67]; skipped without carbon) */
  double on[2];                /* accepted molar O/N ([0.254, 0.320]) */
  double phi[2];               /* accepted (2 n_C + n_H / 2) / n_O ([0.20, 1.15]) */
} chem_hfrd_opts;

/* For n base states (T, p, Y; SoA, ld) and uniform draws gamma in [-1, 1] (species-major
 * [3 + K][ld]: rows 0, 1, 2 for T, p and Y_N2, then one row per species, the N2 row unused):
 *   T' = T + alpha gamma_T (T_max - T_min), p' = p + beta gamma_p (p_max - p_min),
 *   Y'_N2 = Y_N2 + alpha gamma_N2 (Y_N2,max - Y_N2,min), Y'_j = Y_j^(1 + theta gamma_j),
 * the ranges taken over the n base states, then Y' divided by its sum.  keep[i] = 1 when
 * T' > 0, p' > 0, Y'_N2 >= 0 and the molar element ratios H/C and O/N and the element-based
 * equivalence ratio lie in the accepted ranges, else 0.  Outputs T_out, p_out [ld], Y_out
 * [K][ld] (written for every state), keep [ld].  opts NULL selects the paper's values.  The
 * mechanism needs a species named N2 and elements H, O and N (CHEM_E_UNSUPPORTED otherwise).
 * workspace: device scratch of chem_hfrd_workspace_bytes() bytes (the ranges). */
int chem_hfrd_augment(chem_mech mech, int64_t n, int64_t ld, const double* T, const double* p,
                      const double* Y, const double* gamma, const chem_hfrd_opts* opts, double* T_out,
                      double* p_out, double* Y_out, int32_t* keep, void* workspace, size_t ws_bytes,
                      chem_stream stream);
size_t chem_hfrd_workspace_bytes(void);

/* ---------------------------------------------------------------------------------------- */
/* PaSR filtered reaction source (the paper's swirl-flame LES closes turbulence-chemistry    */
/* interaction with the partially stirred reactor model and feeds it the chemistry step:    */
/* Sec. 3, "the ANN model only substitutes the direct integration of source terms within    */
/* the PaSR model"; chemical time from the slowest species formation rate, mixing time from  */
/* the Taylor and Kolmogorov scales)                                                         */
/* ---------------------------------------------------------------------------------------- */
/* From the states before (Y0) and after (Y1) one chemistry step of length dt, per cell:
 *   kappa[i]  = tau_c / (tau_c + tau_mix) (1 when both are 0),
 *   tau_mix   = sqrt(sqrt(nu / eps) * k_sgs / eps), or 0 when k_sgs <= 0 or eps <= 0,
 *   tau_c     = max over species with Y1 >= y_min and Y1 - Y0 > r_min Y1 of
 *               dt Y1 / (Y1 - Y0), or 0 when there is none,
 *   omega[k * ld + i] = kappa rho (Y1 - Y0) / dt   (kg/m^3/s).
 * rho (kg/m^3), k_sgs (m^2/s^2), eps (m^2/s^3) and nu (m^2/s) are per-cell arrays [n]; Y0, Y1
 * and omega are species-major [K][ld]; kappa [n] may be NULL.  y_min < 0 and r_min < 0 select
 * the defaults 1e-10 and 1e-9.  tau_mix is formed in FP32 (relative error below 1e-6), the
 * source differences and products in FP64.  Returns CHEM_E_ARG for dt <= 0 or null arrays. */
int chem_pasr_source(chem_mech mech, int64_t n, int64_t ld, double dt, const double* rho,
                     const double* Y0, const double* Y1, const double* k_sgs, const double* eps,
                     const double* nu, double y_min, double r_min, double* omega, double* kappa,
                     chem_stream stream);

/* Testing hook: y[i] = exp(x[i]) by the library's own FP64 exponential (the table-driven
 * method the kernels use), for comparison with CUDA's exp.  Device pointers, n >= 0. */
int chem_selftest_exp(chem_mech mech, int64_t n, const double* x, double* y, chem_stream stream);

/* Testing hook: y[i] = 2^(x[i]/256) = exp(x[i] ln2/256) by the library's FP64 exponential of
 * pre-scaled arguments (the form the chemistry kernels use for rate constants and equilibrium
 * constants, whose exponents are linear in coefficients stored times 256/ln 2), for comparison
 * with an exact-argument exp2.  Device pointers, n >= 0. */
int chem_selftest_exp256(chem_mech mech, int64_t n, const double* x, double* y, chem_stream stream);

/* Testing hook: y[i] = log(x[i]) by the library's own FP64 logarithm (the table-driven method
 * the kernels use for ln T and the falloff logarithms), for comparison with CUDA's log.  Device
 * pointers, n >= 0. */
int chem_selftest_log(chem_mech mech, int64_t n, const double* x, double* y, chem_stream stream);

/* Testing hook: y[i] = 1/x[i] by the library's own FP64 reciprocal (hardware estimate plus one
 * third-order refinement step, used for every reciprocal of the integration and property
 * kernels), for comparison with IEEE division.  Within 1 ulp for normal x whose reciprocal is
 * normal; zero and infinite x give NaN.  Device pointers, n >= 0. */
int chem_selftest_rcp(int64_t n, const double* x, double* y, chem_stream stream);

/* Testing hook: one tensor-core GEMM of the MLP, out = epi(A B^T) with A [M, K] and B [N, K]
 * BF16 row-major (K a multiple of 8, 16-byte aligned), FP32 accumulation.  epi 0: GELU(acc +
 * bias) -> BF16; 1: acc + bias -> FP32; 2: acc * GELU'(z) -> BF16 with z [M, N] BF16;
 * 3: acc -> FP32.  out is [M, N].  *err (device int, zeroed by the caller) receives a
 * non-zero site code if a pipeline wait timed out.  Device pointers. */
int chem_selftest_gemm(int epi, int M, int N, int K, const void* A, const void* B, const float* bias,
                       const void* z, void* out, int* err, chem_stream stream);

/* Testing hook: G GEMMs of the per-species layers in one launch, for g = 0..G-1:
 * out_g = epi(A_g B_g^T) with A_g [M, K] the block of A (row stride lda) starting at row
 * g a_row, column g a_col, B_g [N, K] the block of B (row stride ldb) starting at row g b_row,
 * column g b_col, out_g at out + g out_goff (row stride ldo), bias_g at bias + g bias_goff, z_g
 * at z + g z_goff (row stride ldz); epilogues as chem_selftest_gemm.  A's extent is
 * [M + (G-1) a_row, K + (G-1) a_col], B's [N + (G-1) b_row, K + (G-1) b_col]; entries of A past
 * a group's K inside that extent must be finite (they meet B's zero fill).  Column offsets
 * and strides multiples of 8, pointers 16-byte aligned.  Device pointers. */
int chem_selftest_gemm_grouped(int epi, int G, int M, int N, int K, const void* A, int64_t lda, int a_row,
                               int a_col, const void* B, int64_t ldb, int b_row, int b_col,
                               const float* bias, int bias_goff, const void* z, int64_t ldz,
                               int64_t z_goff, void* out, int64_t ldo, int64_t out_goff, int* err,
                               chem_stream stream);

/* Testing hook: order[i] = the row chem_ann_train_epoch visits at position i of the epoch
 * (seed, epoch) over n rows, a permutation of 0..n-1.  Device pointer, 1 <= n <= 2^31 - 1. */
int chem_selftest_epoch_order(int64_t n, uint64_t seed, int epoch, int32_t* order, chem_stream stream);

/* Thread-local description of the last error returned on this thread. */
const char* chem_last_error(void);

/* Measured FP64 FMA throughput of the current device (GFLOP/s, 2 flops per FMA): a short
 * DFMA kernel over every SM, timed with CUDA events on `stream`.  Used as the denominator of
 * the DI roofline. */
int chem_fp64_peak_gflops(double* gflops, chem_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* CHEM_H */
