/*
 * ft.h -- C ABI of the GB300 (sm_103a) FastTuckerPlus library.
 *
 * The library runs the stochastic epoch of sparse FastTucker decomposition
 * as described in "cuFastTuckerPlus: A Stochastic Parallel Sparse FastTucker
 * Decomposition Using GPU Tensor Cores" (arXiv 2404.10087):
 *
 *   model       xhat = sum_r prod_n c^(n)_r,  c^(n) = a^(n)_{i_n,:} B^(n)
 *               (Sec. 2.3, Eq. "fasttucker"; Kruskal core of
 *               Eq. "fasttucker_core_tensor")
 *   factor phase  for every sampled nonzero, all N rows a^(n)_{i_n,:} move
 *               together: a <- a + gamma_A((x - xhat) d^(n) B^(n)T - lambda_A a)
 *               with d^(n) = prod_{k != n} c^(k)  (Sec. 3.1,
 *               Eq. "Update_FastTuckerPlus_factor", Algorithm 3, Algorithm 4)
 *   core phase  G^(n) = sum_Omega (xhat - x) a^(n)T d^(n);
 *               B^(n) <- B^(n) - gamma_B (G^(n)/|Omega| + lambda_B B^(n))
 *               (Eq. "Update_FastTuckerPlus_core", Algorithm 5)
 *   errors      RMSE and MAE on a test set (Sec. 5.2)
 *
 * Conventions shared by every call:
 *   - Pointers documented as "device" must point to memory of the current
 *     CUDA device; "host" pointers to ordinary host memory.  Arrays of
 *     pointers (idx, A, B, row_step_scale) are host arrays of N device
 *     pointers.
 *   - Coordinates are int32, 0-based, structure-of-arrays: idx[n][m] is the
 *     mode-n index of nonzero m.  The stored order of the nonzeros is the
 *     sampling order of the epoch (the caller shuffles them).
 *   - A^(n) is float32 row-major I_n x J_n; B^(n) is float32 row-major
 *     J_n x R.  Both are caller-owned, borrowed by the context, and updated
 *     in place by the epochs.
 *   - Supported shapes: 1 <= N <= 10, 1 <= J_n <= 32, 1 <= R <= 32, with
 *     N * K <= 160 where K = 16 if max(J_n, R) <= 16, else 32 (so N <= 10 at
 *     K = 16 and N <= 5 at K = 32).  Others return FT_ERR_SHAPE.  nnz < 2^31.
 *   - The library allocates no device memory: all scratch lives in a
 *     caller-provided workspace (ft_workspace_size), 256-byte aligned.
 *     The context itself is the only (host-heap) allocation.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream) unless stated otherwise.
 *   - Errors are status codes; nothing is thrown across the ABI.  A
 *     non-finite residual met inside a kernel is latched in the workspace
 *     and reported by the next synchronising call (ft_rmse, ft_check) as
 *     FT_ERR_NONFINITE.
 */
#ifndef FT_GB300_H
#define FT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FT_MAX_ORDER 10
#define FT_MAX_RANK 32

typedef struct ft_ctx ft_ctx;

typedef enum {
  FT_OK = 0,
  FT_ERR_ARG = -1,        /* null pointer, negative size, bad enum */
  FT_ERR_INDEX = -2,      /* a coordinate outside [0, I_n) */
  FT_ERR_SHAPE = -3,      /* N, J_n or R outside the supported set */
  FT_ERR_CUDA = -4,       /* a CUDA runtime call failed */
  FT_ERR_NONFINITE = -5,  /* a value or residual is NaN or infinite */
  FT_ERR_TIMEOUT = -6,    /* a bounded device wait gave up */
  FT_ERR_WORKSPACE = -7   /* workspace too small or misaligned */
} ft_status;

/* Arithmetic of the two contractions a.B and d.B^T (and of E^T D in the core
 * phase).  Factor and core matrices always stay float32 masters; the
 * accumulators are float32 in every mode (Sec. 4.1 uses FP16 inputs with
 * tensor cores).  FT_FP32 is FP32-accurate: both phases multiply on the
 * tensor cores with three-pass TF32 (each operand split into a TF32 head and
 * tail, x = hi + lo, and the product taken as lo.hi + hi.lo + hi.hi).  FT_TF32 and FT_BF16 round the
 * inputs of every contraction to TF32 or BF16 (tensor cores).  Predictions
 * and test errors are FP32-accurate in every mode.  An FT_BF16 context also
 * keeps BF16 copies of the factor rows in its workspace (sum_n I_n * K * 2
 * bytes), written at the start of every core phase and gathered by the core
 * pass in place of the float32 rows (the same roundings, so the same
 * results). */
enum { FT_FP32 = 0, FT_TF32 = 1, FT_BF16 = 2 };

/* How the factor phase writes rows back.
 * FT_HOGWILD: every warp stores its updated rows directly, as the paper's
 *   kernel does (Algorithm 4); concurrent updates of one row may be lost.
 * FT_DETERMINISTIC: batch-synchronous epoch with batch size det_batch:
 *   every nonzero of a batch reads the factors as they were at the batch
 *   start, the per-nonzero steps of each row are summed in increasing
 *   nonzero order and applied once; results are reproducible bit for bit. */
enum { FT_HOGWILD = 0, FT_DETERMINISTIC = 1 };

typedef struct {
  int precision;       /* FT_FP32 | FT_TF32 | FT_BF16 */
  int scatter;         /* FT_HOGWILD | FT_DETERMINISTIC */
  int64_t det_batch;   /* batch size S of FT_DETERMINISTIC (>= 1) */
  int blocks_per_sm;   /* persistent CTAs per SM; 0 = from the occupancy API */
  /* FT_HOGWILD only: shared-memory write-back cache of the most frequent rows
   * of the tensor (ranked over all modes by their number of training
   * nonzeros).  Each CTA keeps hot_rows rows in shared memory, updates them
   * there, and after every hot_window x 128 of its nonzeros (rounded up to
   * whole CTA tiles: 16 nonzeros per warp, 128 per tcgen05 warpgroup) adds its
   * weighted change of every dirty row (cached row minus the copy it read at
   * the last refresh) to the row in A with float atomics and refreshes its
   * copy: no CTA overwrites another CTA's change, and a CTA sees the others'
   * from its next refresh on.  The weight is 1 for a row that a CTA meets
   * less than once between two write-backs (the CTAs' steps add up, as in
   * Hogwild); a row that every CTA meets many times between two write-backs
   * takes the average of the CTAs' changes (weight 1 / the CTAs expected to
   * change it), since adding them would apply the same move once per CTA.
   * The weights come from the row counts at ft_init.  The workspace holds
   * each CTA's copy (CTAs x hot_rows x K floats).  Only rows with at least
   * hot_min_count training nonzeros are cached.  With the cache on, the
   * warp-tile pass runs one 512-thread CTA per SM where its tile fits 128
   * registers (K = 16 and N <= 3; one cache of twice the rows instead of two
   * CTAs' copies of the same rows), else 256-thread CTAs.  hot_rows: -1 = as
   * many as 96 KB per 256 threads of the CTA hold (3024 rows at K = 16,
   * N <= 3; for the tcgen05 pass with full-width rows, as many of 96 KB as
   * fit beside its 4 x N x 8 KB row stage), 0 = off. */
  int hot_rows;
  int hot_window;      /* 1 .. 2^20; default 256 */
  int hot_min_count;   /* >= 1; default 2 */
  /* Kernel family of the Hogwild factor pass: FT_ENGINE_WARP (default) = one
   * warp per 16-nonzero tile with mma.sync products; FT_ENGINE_TCGEN05 = one
   * warpgroup per 128-nonzero tile, products on tcgen05.mma with TMEM
   * accumulators (FT_BF16, J_n, R <= 16, N <= 4, FT_HOGWILD only; other
   * configurations return FT_ERR_ARG from ft_workspace_size / ft_init). */
  int engine;
  /* How the core phase obtains the rows c^(n) = a^(n) B^(n) (Sec. 5.6,
   * "Replace memory access with calculation"): FT_CORE_CALC (default) forms
   * them for every nonzero from the gathered factor rows (Algorithm 5);
   * FT_CORE_STORE first computes C^(n) = A^(n) B^(n) for every row of every
   * mode (FP32, one dense product per core phase, I_n x K floats of
   * workspace per mode) and gathers its rows instead.  The paper found the
   * storage scheme faster on CUDA cores and calculation faster with tensor
   * cores.  Both give the same gradient up to rounding. */
  int core_scheme;
  /* (A cache hint with no counterpart in the paper.)
   * 1: keep the factor matrices in L2 while other traffic streams through
   * it (for example a host-to-device copy of the next epoch's nonzeros that
   * overlaps this epoch): every launch of the context carries an access-policy
   * window over the address span of A^(0..N-1), marked persisting.  ft_init
   * raises the calling process's persisting-L2 limit (cudaLimitPersistingL2CacheSize
   * of the current device, a per-process setting) to the window size, capped
   * at the device maximum, if it is lower.  Place the factor matrices in one
   * allocation so that the span covers nothing else.  A cache hint only:
   * results are unchanged.  0 (default): off. */
  int l2_persist;
  int reserved[1];     /* must be zero */
} ft_config;

enum { FT_ENGINE_WARP = 0, FT_ENGINE_TCGEN05 = 1 };
enum { FT_CORE_CALC = 0, FT_CORE_STORE = 1 };

/* Fill *cfg with the defaults: FT_FP32, FT_HOGWILD, det_batch 4096, automatic
 * grid, hot_rows -1, hot_window 256, hot_min_count 2, FT_ENGINE_WARP,
 * FT_CORE_CALC, l2_persist 0. */
void ft_config_default(ft_config *cfg);

/* Bytes of device workspace needed by ft_init for this problem (host call;
 * queries the current device).  I, J: host arrays of N entries. */
ft_status ft_workspace_size(int N, const int64_t *I, const int *J, int R, int64_t nnz,
                            const ft_config *cfg, size_t *bytes);

/* Create a context over the training nonzeros.
 *   idx   host array of N device pointers, each nnz int32 coordinates
 *   vals  device, nnz float32 values
 *   A, B  host arrays of N device pointers (row-major float32, see above)
 *   workspace  device, >= ft_workspace_size bytes, 256-byte aligned; owned by
 *         the caller and used by every later call on this context
 * Validates shapes, checks every coordinate and value on the device
 * (FT_ERR_INDEX / FT_ERR_NONFINITE) and, in FT_DETERMINISTIC mode, builds the
 * per-batch row grouping (a host sort over a copy of the coordinates).
 * Synchronises the stream.  On success *out receives the context. */
ft_status ft_init(ft_ctx **out, int N, const int64_t *I, const int *J, int R, int64_t nnz,
                  const int32_t *const *idx, const float *vals, float *const *A,
                  float *const *B, void *workspace, size_t ws_bytes, const ft_config *cfg,
                  void *stream);

/* One factor phase over all nnz training nonzeros in stored order
 * (Algorithm 3 factor loop; Algorithm 4).  Step gamma_A = lr_a, lambda_A =
 * lambda_a.  row_step_scale: NULL, or a host array of N pointers, each NULL
 * or a device array of I_n per-row step multipliers s (the step of row i of
 * mode n becomes lr_a * s[i]). */
ft_status ft_epoch_factors(ft_ctx *ctx, float lr_a, float lambda_a,
                           const float *const *row_step_scale, void *stream);

/* One core phase (Algorithm 5): accumulate G^(n) over all training
 * nonzeros with compensated float32 sums in a fixed order (reproducible bit
 * for bit), then B^(n) <- B^(n) - lr_b (G^(n)/nnz + lambda_b B^(n)). */
ft_status ft_epoch_core(ft_ctx *ctx, float lr_b, float lambda_b, void *stream);

/* Reshuffle the training nonzeros (Algorithm 3 takes the sample sets Psi
 * from Omega at random in every iteration): the context's nonzeros are
 * gathered in the order perm gives into caller-provided arrays,
 *   idx_out[n][m] = idx[n][perm[m]],  vals_out[m] = vals[perm[m]],
 * and the context then borrows idx_out / vals_out (the arrays it used before
 * are no longer read and may be reused, e.g. as the next call's outputs).
 *   perm      device, nnz int32, a permutation of 0..nnz-1 drawn by the
 *             caller (repeated entries are not detected and duplicate
 *             nonzeros)
 *   idx_out   host array of N device pointers, nnz int32 each; vals_out
 *             device, nnz floats; none may alias the current arrays
 *             (FT_ERR_ARG)
 * The hot-row coordinates of the Hogwild pass are rebuilt on the device; in
 * FT_DETERMINISTIC mode the per-batch row grouping is rebuilt on the host
 * (synchronises).  An entry of perm outside [0, nnz) is latched as
 * FT_ERR_INDEX (reported by the next synchronising call) and copies nonzero
 * 0 in its place. */
ft_status ft_permute(ft_ctx *ctx, const int32_t *perm, int32_t *const *idx_out, float *vals_out,
                     void *stream);

/* (A library service with no counterpart in the paper.)  Point the context
 * at another copy of its training nonzeros: the same nnz,
 * in any order, e.g. a buffer that an asynchronous host-to-device copy filled
 * while the previous epoch ran (double buffering).  The arrays are borrowed
 * from then on; the old ones are no longer read once the calls queued before
 * this one have run.  The hot rows chosen at ft_init are kept and their
 * coordinates are rebuilt on the device into the idle one of two copies in
 * the workspace, on `stream`: the passes enqueued since the previous
 * ft_rebind (on any stream) read the other copy, so the rebuild may overlap
 * them on a second stream; passes enqueued later must be ordered after
 * `stream` (the same stream, or an event).  In FT_DETERMINISTIC mode the row grouping is rebuilt on the
 * host (synchronises); otherwise asynchronous.
 * The new coordinates and values are not validated up front: the epoch
 * kernels mask a coordinate outside [0, I_n) and latch FT_ERR_INDEX, and a
 * non-finite value shows as a latched FT_ERR_NONFINITE (both reported by the
 * next synchronising call).
 *   idx   host array of N device pointers, nnz int32 each; vals: device */
ft_status ft_rebind(ft_ctx *ctx, const int32_t *const *idx, const float *vals, void *stream);

/* One core phase in the per-sample-set reading of Algorithm 3, whose core
 * loop applies rule "Update_FastTuckerPlus_core" for every sampled set Psi:
 * the training nonzeros are taken in stored order in consecutive sets of
 * set_size (the last one ragged), and each set makes one step of
 * ft_epoch_core restricted to it, from the core matrices the previous set
 * left: B^(n) <- B^(n) - lr_b (G_Psi^(n) / |Psi| + lambda_b B^(n)).
 * set_size >= nnz is ft_epoch_core.  Each set is one core-gradient pass plus
 * one finalize (and, with FT_CORE_STORE, one C = A B product), in a fixed
 * order: reproducible bit for bit.  set_size < 1: FT_ERR_ARG. */
ft_status ft_epoch_core_sgd(ft_ctx *ctx, float lr_b, float lambda_b, int64_t set_size, void *stream);

/* The core gradient alone, without touching B:
 * G_out (device) receives G^(n) = sum_Omega (xhat - x) a^(n)T d^(n) for
 * n = 0..N-1, each J_n x R row-major, concatenated. */
ft_status ft_core_grad(ft_ctx *ctx, float *G_out, void *stream);

/* The core step of Algorithm 5 from a gradient that the caller supplies:
 *   B^(n) <- B^(n) - lr_b (G^(n) / nnz_total + lambda_b B^(n))
 * for every entry, in the context's B (in place).  With ft_core_grad this
 * splits ft_epoch_core into its two halves, so that the gradient can be
 * summed across processes in between: each process holds a context over its
 * own shard of Omega (Algorithm 5 sums G over all of Omega, so the shards'
 * gradients add), the processes all-reduce their G_out, and each applies the
 * sum with nnz_total = |Omega| (the sum of the shards' nnz), which leaves
 * identical B on every process.  ft_core_grad followed by ft_core_apply with
 * nnz_total = the context's nnz equals ft_epoch_core bit for bit.
 *   G         device, sum_n J_n * R floats in the layout of ft_core_grad's
 *             G_out (mode by mode, each J_n x R row-major); used as given
 *   nnz_total >= 0 (0 applies only the decay term, as an empty Omega would)
 * FT_ERR_ARG for a null pointer, a negative nnz_total or a non-finite step. */
ft_status ft_core_apply(ft_ctx *ctx, const float *G, int64_t nnz_total, float lr_b,
                        float lambda_b, void *stream);

/* The core gradient of ft_core_grad without a context and without any
 * allocation, for callers that cannot call cudaMalloc: for example code whose
 * device memory is owned by another allocator (a framework or service that
 * has reserved the device's memory in its own pool and forbids allocations
 * outside it), or a caller that cannot keep a context and its workspace alive
 * between calls.  The paper has no counterpart; this is a library service.
 *   idx, vals, A, B: as for ft_init (device data; host arrays of N device
 *   pointers); precision: FT_FP32 | FT_TF32 | FT_BF16; G_out (device)
 *   receives G^(n) = sum (xhat - x) a^(n)T d^(n), each J_n x R row-major,
 *   concatenated over n.
 * Scratch: the call needs no workspace.  Its scratch (the per-CTA partial
 * sums of the core pass) lives in one 16 MiB device array compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  Calls that would need more than that (more CTAs times N * K * K
 * partials than fit) return FT_ERR_WORKSPACE; on a GB300 every supported
 * shape fits.  The first call on a device looks up the array's device address
 * with that device current (make that first call before any stream capture)
 * and keeps it for the process: a cudaDeviceReset of that device after the
 * first call is not supported (the kept address would be stale).  Unlike
 * ft_init, the call does not validate its inputs in a separate pass: the
 * kernel masks and reports out-of-range coordinates and non-finite values.
 * Every call shares the array and overwrites it: calls that overlap on the
 * GPU (on different streams or host threads) race and corrupt each other's
 * results, so serialise them.
 * The result equals ft_core_grad's for the same inputs (same grid and fixed
 * summation order).  Synchronises the stream to report bad coordinates
 * (FT_ERR_INDEX) or non-finite residuals (FT_ERR_NONFINITE). */
ft_status ft_core_grad_noalloc(int N, const int64_t *I, const int *J, int R, int64_t nnz,
                               const int32_t *const *idx, const float *vals,
                               const float *const *A, const float *const *B, int precision,
                               float *G_out, void *stream);

/* ---------------------------------------------------------------- batches
 * Many independent tensors trained together (each with its own order N,
 * ranks J_n and R, nonzeros and matrices).  Tensors are grouped by kernel
 * class (N, padded rank K); every class runs one persistent factor kernel and
 * one persistent core kernel over fixed-size units of its tensors' tiles (the
 * units dealt round-robin over the class's tensors), and
 * the whole epoch - the factor pass (Hogwild within each tensor), the core
 * pass and one finalize over all tensors - is captured once as a CUDA graph
 * and replayed by ft_batch_epoch.  The paper treats one tensor at a time
 * (Algorithms 3-5); each tensor of a batch follows exactly those rules.
 */
typedef struct {
  int N;
  const int64_t *I;           /* host, N mode sizes */
  const int *J;               /* host, N factor ranks */
  int R;
  int64_t nnz;
  const int32_t *const *idx;  /* host array of N device pointers (nnz int32 each) */
  const float *vals;          /* device, nnz values */
  float *const *A;            /* host array of N device pointers, I_n x J_n */
  float *const *B;            /* host array of N device pointers, J_n x R */
} ft_tensor_desc;

typedef struct ft_batch ft_batch;

/* Workspace bytes for a batch (host call; queries the current device).
 * cfg: precision as for ft_init; scatter must be FT_HOGWILD; the hot-row
 * cache is not used by batches. */
ft_status ft_batch_workspace_size(int ntensors, const ft_tensor_desc *tensors,
                                  const ft_config *cfg, size_t *bytes);

/* Validate every tensor (as ft_init does), lay out the units with default
 * launch shapes and capture the epoch graph.  The descriptors' host arrays
 * are copied; the device buffers are borrowed.  Synchronises the stream. */
ft_status ft_batch_init(ft_batch **out, int ntensors, const ft_tensor_desc *tensors,
                        const ft_config *cfg, void *workspace, size_t ws_bytes, void *stream);

/* Autotuner: for every kernel class, time the core pass (which changes no
 * factor or core matrix) over candidate launch shapes - tiles per work unit
 * and CTAs per SM - keep the fastest, and recapture the epoch graph.
 * Synchronises the stream. */
ft_status ft_batch_tune(ft_batch *b, void *stream);

/* One epoch of every tensor: factor pass (Algorithm 4), core pass and
 * finalize (Algorithm 5), by one replay of the captured graph. */
ft_status ft_batch_epoch(ft_batch *b, float lr_a, float lambda_a, float lr_b, float lambda_b,
                         void *stream);

/* Test errors of tensor `tensor` of the batch, as ft_rmse. */
ft_status ft_batch_rmse(ft_batch *b, int tensor, int64_t n, const int32_t *const *idx,
                        const float *vals, double *out3, void *stream);

/* Number of kernel classes, and the launch shape of class `cls`:
 * out6 = {N, K, tensors in the class, warp tiles per unit, CTAs per SM,
 * units}. */
int ft_batch_num_classes(const ft_batch *b);
ft_status ft_batch_class_info(const ft_batch *b, int cls, int64_t *out6);

/* Kernels launched by this batch since ft_batch_init (graph nodes included). */
int64_t ft_batch_launch_count(const ft_batch *b);

void ft_batch_destroy(ft_batch *b);

/* Predictions xhat (float32) of n coordinates (idx: host array of N device
 * pointers; out: device, n floats) with the context's current A and B. */
ft_status ft_predict(ft_ctx *ctx, int64_t n, const int32_t *const *idx, float *out,
                     void *stream);

/* Errors on n coordinates with values vals (device): the residuals are
 * float32, their sums are reduced in float64.  out3 (host) receives
 * {RMSE, MAE, sum of squared errors}.  Synchronises the stream; returns
 * FT_ERR_NONFINITE if an earlier kernel latched a non-finite residual. */
ft_status ft_rmse(ft_ctx *ctx, int64_t n, const int32_t *const *idx, const float *vals,
                  double *out3, void *stream);

/* Inputs of the learned per-row step size (an extension: the paper uses
 * one step size, Eq. "Update_FastTuckerPlus_factor").  For every row of every
 * mode (rows concatenated, mode 0 first, sum I_n rows), from the current A, B:
 *   count, mean residual, and the row gradient g = sum_m (-e_m p_m + lambda_a a)
 *   (Eq. "Gradient_low_rank_cp" summed over the row's training nonzeros);
 *   features[3 r .. 3 r + 2] = {log(1 + count), log(1 + ema), mean residual}
 *   with ema <- ema_beta * ema + (1 - ema_beta) |g| / max(count, 1) (ema: device,
 *   rows, in/out; NULL = no history, ema = |g| / count);
 *   labels[r] (NULL = not computed): the exact line-search step along -g of
 *   the row's subproblem sum_m [1/2 (x_m - a.p_m)^2 + 1/2 lambda_a |a|^2],
 *   t* = |g|^2 / (sum_m (p_m.g)^2 + lambda_a count |g|^2), shared among the N
 *   rows that every nonzero moves at once (t* / N: each row's exact step alone
 *   would remove the residual, N of them together N times over), divided by
 *   lr_a, clipped to [1/16, 16], as its natural log (the regression target of
 *   the step-size network; 0 for rows without nonzeros).
 * FP32 with atomic accumulation (the summation order varies between runs). */
ft_status ft_row_stats(ft_ctx *ctx, float lambda_a, float lr_a, float ema_beta, float *ema,
                       float *features, float *labels, void *stream);

/* ------------------------------------------------------- step-size network
 * A small MLP (3 -> 64 -> 64 -> 1, ReLU, linear output u = the predicted
 * log-multiplier; multiplier s = exp(clamp(u, log 1/16, log 16)))
 * that maps the row features of ft_row_stats to per-row step multipliers for
 * ft_epoch_factors (row_step_scale).  Not in the paper.  All state lives in
 * one caller-allocated device buffer of ft_stepnet_bytes() bytes (16-byte
 * aligned): FP32 master parameters, their BF16 copies (used by every kernel,
 * with FP32 accumulation), Adam moments and the last gradient.  Parameter
 * order: W1 [64][3], b1 [64], W2 [64][64], b2 [64], w3 [64], b3. */
size_t ft_stepnet_bytes(void);

/* Initialise the buffer: He-uniform weights from a counter-based hash of
 * (seed, index), zero biases, so u starts near 0 and s near 1. */
ft_status ft_stepnet_init(void *net, uint64_t seed, void *stream);

/* scale[r] = s(features[3 r .. 3 r + 2]) for r < rows (device arrays). */
ft_status ft_stepnet_forward(const void *net, int64_t rows, const float *features, float *scale,
                             void *stream);

/* `steps` full-batch Adam steps (lr, betas 0.9 / 0.999, eps 1e-8) on the mean
 * of 1/2 (u - label)^2 over `rows` samples (labels: log-multipliers, as
 * ft_row_stats writes them; the output is not clamped in the loss, so its
 * gradient does not vanish).  loss_out (host, nullable)
 * receives the loss of the last step's forward pass (synchronises). */
ft_status ft_stepnet_train(void *net, int64_t rows, const float *features, const float *labels,
                           float lr, int steps, double *loss_out, void *stream);

/* Copy 4481 values to host memory: which = 0 FP32 masters, 1 the BF16
 * copies (widened), 2 the gradient of the last training step.  Synchronises. */
ft_status ft_stepnet_get(const void *net, int which, float *out_host, void *stream);

/* Synchronise the stream and report (then clear) the latched device error. */
ft_status ft_check(ft_ctx *ctx, void *stream);

/* Number of kernel launches issued by this context since ft_init. */
int64_t ft_launch_count(const ft_ctx *ctx);

/* Free the context (not the caller's buffers).  NULL is ignored. */
void ft_destroy(ft_ctx *ctx);

/* Static, human-readable name of a status. */
const char *ft_status_str(ft_status s);

#ifdef __cplusplus
}
#endif

#endif /* FT_GB300_H */
