/*
 * rcfar.h -- C ABI of the GB300 radar chain library (librcfar.so).
 *
 * The library computes the data path of Rohman, Andra and Nishimoto,
 * "Optimized 2D CA-CFAR for Drone-Mounted Radar Signal Processing Using
 * Integral Image Algorithm":
 *   Sec. II.A  fast-time DC-shift removal + linear-trend subtraction, slow-time
 *              mean filter + normalisation, slow-time transform restricted to
 *              the 0.3-0.8 Hz respiration band, magnitude  -> band map P
 *   Sec. II.B  summed-area table of P (eq. 3), 2D cell-averaging CFAR whose
 *              reference sum comes from four-corner lookups (eq. 4) of an
 *              outer rectangle minus a guard rectangle, threshold T = alpha*A
 *              (eq. 2) and the H0/H1 decision of eq. 1.
 *
 * Conventions shared by every entry point
 *   - Every function returns rcfar_status and never throws.
 *   - Pointers named x, map, det, thr, view fields and frame fields are DEVICE
 *     pointers owned by the caller, unless stated otherwise; the library owns
 *     only the workspace inside its handle. Arrays are row-major with the
 *     stated leading dimension (in elements).
 *   - A raw frame X is [M][ldx] float32: row m = fast-time sample (range bin),
 *     column n = slow-time sample (trace), N <= ldx. (Sec. II.A, X in R^{MxN}.)
 *   - Work is enqueued on the given stream (a cudaStream_t; NULL = legacy
 *     default stream) and returns before it completes. Asynchronous faults that
 *     kernels detect (a value outside the stated bound, an expired bounded wait)
 *     are recorded in a device status word and reported by rcfar_get_error.
 *   - A handle serves one stream at a time: calls on one handle must not run
 *     concurrently on different streams. Create one handle per stream instead.
 *   - Interpretation choices where the paper is silent (band edges, window
 *     semantics, edge policy, eq. 2's exponent sign, CUT == T) are documented
 *     at the function that applies them.
 */
#ifndef RCFAR_H
#define RCFAR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rcfar_status {
  RCFAR_OK = 0,
  RCFAR_ERR_INVALID_ARG = 1,      /* null pointer, size <= 0, even mean filter, pfa not in (0,1), ... */
  RCFAR_ERR_UNSUPPORTED = 2,      /* size beyond the handle's create-time limits */
  RCFAR_ERR_OUT_OF_WORKSPACE = 3, /* a batch needs more workspace than the handle holds */
  RCFAR_ERR_CUDA = 4,             /* a CUDA runtime call failed */
  RCFAR_ERR_TIMEOUT = 5,          /* a bounded device-side wait expired (results invalid) */
  RCFAR_ERR_BAD_STATE = 6,        /* stale view, wrong handle, destroyed handle */
  RCFAR_ERR_RANGE = 7             /* a map value exceeded the stated bound or was NaN (results invalid) */
} rcfar_status;

typedef struct rcfar_ctx* rcfar_handle;
typedef void* rcfar_stream; /* cudaStream_t */

/* Storage type of a CFAR input map. */
typedef enum rcfar_map_dtype {
  RCFAR_MAP_F32 = 0,
  RCFAR_MAP_F16 = 1 /* IEEE half; value = stored * 2^map_exp2 */
} rcfar_map_dtype;

/* How the summed-area table is stored (paper eq. 3). The map is cut into
 * tiles of 32 rows x 128 columns; band b = tile row, chunk j = tile column.
 * For cell (r, c) of tile (b, j):
 *   S(r, c) = L(r, c) + CC_j(r) + RC_{b-1}(c)
 *   L     : the table of the tile relative to its own origin
 *   CC_j  : col_carry[j][r] = sum of the band's rows <= r left of the tile
 *   RC_b  : row_carry[b][c] = S(last row of band b, c)   (RC_{-1} = 0)
 *  TILE_I64 : L in 64-bit fixed point plus the carries. Exact; 8 B/cell.
 *  TILE_F32 : L in FP32 plus exact 64-bit carries. 4 B/cell; L's rounding
 *             grows with the tile's sum (precision study).
 *  I64      : S itself in 64-bit fixed point (carries folded in). Exact.
 *  NAIVE_F32: S itself in plain FP32 (for contrast only: large maps lose the
 *             reference sums to cancellation).
 * Fixed-point values are round(x * 2^scale_log2) and are added modulo 2^64,
 * so every region sum that fits in 63 bits is exact even where the table
 * itself wraps. */
typedef enum rcfar_sat_mode {
  RCFAR_SAT_TILE_F32 = 0,
  RCFAR_SAT_I64 = 1,
  RCFAR_SAT_NAIVE_F32 = 2,
  RCFAR_SAT_TILE_I64 = 3,
  RCFAR_SAT_FUSED = 4  /* no table in device memory (rcfar_sat_cfar); batch tuning only, not rcfar_sat */
} rcfar_sat_mode;

typedef struct rcfar_config {
  int32_t device;        /* CUDA device ordinal */
  int32_t max_rows;      /* largest M (frame) / map row count */
  int32_t max_cols;      /* largest map column count (band bins incl. halo) */
  int32_t max_n;         /* largest slow-time length N */
  int32_t max_window;    /* largest per-side half-width guard + training */
  int32_t max_frames;    /* largest number of frames in one rcfar_run_batch */
  int64_t batch_bytes;   /* device workspace reserved for rcfar_run_batch (0: none) */
  int32_t cfar_tile_rows; /* SAT-CFAR output tile (0, 0: chosen from the window); */
  int32_t cfar_tile_cols; /* rows in {8,16,32,64}, cols in {16,32,64,128} */
} rcfar_config;

/* Preprocessing parameters (Sec. II.A). */
/* Detector of the band map: the magnitude |DFT| (the paper's "FFT" map) or
 * the square law |DFT|^2, for which eq. 2's alpha is exact on noise. */
typedef enum rcfar_detector { RCFAR_DETECT_MAGNITUDE = 0, RCFAR_DETECT_SQUARE_LAW = 1 } rcfar_detector;
/* "then normalized" (Sec. II.A): divide the frame by its max |y|, or scale
 * each range bin's slow-time series to zero mean and unit standard deviation
 * (z-score; a constant row gives a zero map row). Decisions are invariant to
 * the global scale, not to the per-row one. */
typedef enum rcfar_normalise { RCFAR_NORM_GLOBAL_MAX = 0, RCFAR_NORM_ROW_ZSCORE = 1 } rcfar_normalise;

/* Memory order of a raw frame X (M range bins x N traces). Range-major:
 * X[m][n] at x[m * ldx + n], ldx >= N. Trace-major, the order a radar
 * acquires it in (one trace of M range samples after another, Sec. III):
 * X[m][n] at x[n * ldx + m], ldx >= M; such frames are transposed once into
 * the workspace and then take the range-major path (identical results). */
typedef enum rcfar_x_layout { RCFAR_X_RANGE_MAJOR = 0, RCFAR_X_TRACE_MAJOR = 1 } rcfar_x_layout;

typedef struct rcfar_pre_params {
  double fs_hz;      /* slow-time sampling rate (traces per second) */
  double f_lo_hz;    /* respiration band, inclusive: 0.3 in the paper */
  double f_hi_hz;    /* 0.8 in the paper */
  int32_t mean_len;  /* odd mean-filter length along slow time (e.g. 5) */
  int32_t halo_c;    /* extra bins stored each side of the band (use the CFAR's guard_c + train_c);
                        rcfar_run_batch: -1 = each frame uses its own window's guard_c + train_c */
  int32_t detector;  /* rcfar_detector (0: magnitude) */
  int32_t normalise; /* rcfar_normalise (0: global max) */
  int32_t x_layout;  /* rcfar_x_layout of the raw frames (0: range-major) */
  int32_t pad;
} rcfar_pre_params;

/* Spectral bins of a band map: map column j holds bin k = c0 + j. */
typedef struct rcfar_band {
  int32_t k_lo, k_hi; /* respiration band bins (CUT columns are k_lo-c0 .. k_hi-c0) */
  int32_t c0, c1;     /* first and last stored bin, clipped to [0, N/2] */
  int32_t cols;       /* c1 - c0 + 1 */
  float value_bound;  /* every map value is <= this: N, or N^2 for the square law (for rcfar_sat) */
} rcfar_band;

/* How the reference cells set the threshold.
 * CA: cell averaging (Sec. II.B, eqs. 1-2): T = (alpha / n_ref) S_ref over
 *     the whole training ring, alpha = n_ref (Pfa^(-1/n_ref) - 1).
 * GO / SO (greatest-of / smallest-of; not in the paper, built on the same
 *     eq. 3 table and eq. 4 lookups): the training ring is split along range
 *     into a leading half (rows r - W_r .. r - 1 without the guard rows
 *     r - guard_r .. r - 1) and a lagging half (rows r + 1 .. r + W_r without
 *     r + 1 .. r + guard_r); the training cells in the CUT's own row belong to
 *     neither. Each half has n = W_r (2 W_c + 1) - guard_r (2 guard_c + 1)
 *     cells, and T = t * max (GO) or t * min (SO) of the two half sums, with t
 *     the factor for which iid exponential noise gives false-alarm
 *     probability exactly Pfa (rcfar_threshold_factor).
 * OS (ordered statistic; not in the paper, and not a region sum, so it
 *     cannot use the eq. 3 table): T = alpha_os * X_(k), X_(k) the k-th
 *     smallest of the n_ref training cells (k = os_rank, default
 *     ceil(3 n_ref / 4)), alpha_os such that iid exponential noise gives
 *     false-alarm probability exactly Pfa:
 *     prod_{i<k} (n_ref - i) / (n_ref - i + alpha_os) = Pfa. Run by
 *     rcfar_cfar_direct and by the batched chain (rcfar_run_batch, the
 *     server), n_ref <= 2048; the table-based calls return UNSUPPORTED. */
typedef enum rcfar_cfar_kind {
  RCFAR_CFAR_CA = 0,
  RCFAR_CFAR_GO = 1,
  RCFAR_CFAR_SO = 2,
  RCFAR_CFAR_OS = 3
} rcfar_cfar_kind;

/* CFAR window (Sec. II.B): per-side counts in each dimension. The guard
 * rectangle [r-guard_r, r+guard_r] x [c-guard_c, c+guard_c] contains the CUT;
 * training cells fill the ring out to half-sizes guard+train
 * (W_r = guard_r + train_r, W_c = guard_c + train_c). */
typedef struct rcfar_window {
  int32_t train_r, train_c;
  int32_t guard_r, guard_c;
  double pfa;       /* false-alarm probability, 0 < pfa < 1 */
  int32_t kind;     /* rcfar_cfar_kind (0: cell averaging) */
  int32_t os_rank;  /* OS: rank k (1..n_ref, 0: ceil(3 n_ref / 4)); other kinds: must be 0 */
} rcfar_window;

/* Description of a summed-area table produced by rcfar_sat. The arrays live
 * in the handle's workspace and stay valid until the next rcfar_sat or
 * rcfar_run_batch on the same handle. */
typedef struct rcfar_sat_view {
  int32_t rows, cols;
  int32_t mode;          /* rcfar_sat_mode */
  int32_t tile_h, tile_w;
  int32_t scale_log2;    /* fixed-point scale s (TILE_F32, I64) */
  void* table;           /* TILE_F32/NAIVE_F32: float [rows][ld]; TILE_I64/I64: int64 [rows][ld] */
  int64_t ld;
  int64_t* row_carry;    /* [ceil(rows/tile_h)][ld_carry]: S on each band's last row */
  int64_t* col_carry;    /* [ceil(cols/tile_w)][rows]: band-local sums left of each tile */
  int64_t ld_carry;
  uint64_t generation;   /* handle-side stamp; a stale view is rejected */
} rcfar_sat_view;

/* One frame of a batch: raw frame in, decisions (and optionally the map and
 * thresholds) out. det is [M][ld_det] with band.cols columns. */
typedef struct rcfar_frame_desc {
  const float* x;
  int32_t M, N;
  int64_t ldx;
  rcfar_window window;
  uint8_t* det;
  int64_t ld_det;
  float* thr;      /* optional (NULL): threshold T at CUTs, 0 elsewhere */
  int64_t ld_thr;
  float* map;      /* optional (NULL): normalised band map P */
  int64_t ld_map;
} rcfar_frame_desc;

/* ---- handle ------------------------------------------------------------ */

/* Allocates the workspace for the limits in cfg on cfg->device. */
rcfar_status rcfar_create(const rcfar_config* cfg, rcfar_handle* out);
/* Waits for the handle's device work to finish and frees it. */
rcfar_status rcfar_destroy(rcfar_handle h);

/* ---- host-only helpers (no GPU needed) -------------------------------- */

/* eq. 2 with the exponent's sign corrected (the printed alpha = N(Pfa^{1/N}-1)
 * is negative for Pfa < 1): alpha = n_ref * (pfa^(-1/n_ref) - 1), exact for a
 * cell-averaging CFAR on iid exponential (square-law) noise. */
rcfar_status rcfar_alpha(int32_t n_ref, double pfa, double* alpha_out);
/* n_ref = (2(g_r+t_r)+1)(2(g_c+t_c)+1) - (2g_r+1)(2g_c+1) (Sec. II.B "N"). */
rcfar_status rcfar_n_ref(const rcfar_window* w, int32_t* n_ref_out);
/* The factor the kernels multiply the reference statistic by, computed on the
 * host in FP64: CA: alpha / n_ref (applied to S_ref); GO / SO: t (applied to
 * the larger / smaller half sum), found by bisection on the false-alarm law
 * of the kind (relative accuracy 1e-13). cells_out (may be NULL): n_ref for
 * CA, the cells of one half for GO / SO. OS: alpha_os (applied to the k-th
 * smallest training cell), cells = n_ref. An invalid window (including a GO /
 * SO window with empty halves) is RCFAR_ERR_INVALID_ARG. */
rcfar_status rcfar_threshold_factor(const rcfar_window* w, double* factor_out, int32_t* cells_out);
/* Respiration band of a length-N slow-time transform (Sec. II.A, 0.3-0.8 Hz):
 * k_lo = ceil(f_lo N / fs), k_hi = floor(f_hi N / fs) (inclusive; values
 * within 1e-9 of an integer count as that integer), c0 = max(0, k_lo - halo_c),
 * c1 = min(N/2, k_hi + halo_c). An empty stored range (c1 < c0) is
 * RCFAR_ERR_INVALID_ARG; an empty band with a non-empty halo is valid and
 * has no CUT columns. */
rcfar_status rcfar_band_plan(int32_t N, const rcfar_pre_params* p, rcfar_band* out);
/* Fixed-point scale chosen for a map with |values| <= bound whose largest
 * region sum spans at most max_cells cells. */
rcfar_status rcfar_sat_scale(float bound, int64_t max_cells, int32_t* scale_log2_out);
const char* rcfar_status_string(rcfar_status s);

/* ---- the per-step path ------------------------------------------------- */

/* Sec. II.A: raw frame x (M x N, layout p->x_layout, leading dimension ldx)
 * -> normalised band map [M][ld_map] with band_out->cols columns. Steps, all
 * on the GPU:
 *   x'[m,n] = x[m,n] - a_n - b_n (m - (M-1)/2)      (per-trace LS line over m)
 *   y[m,n]  = mean of x'[m, n-h..n+h] inside [0,N)   (h = (mean_len-1)/2)
 *   y      /= max |y| over the frame                  (unchanged if 0; or a
 *                                                      per-row z-score)
 *   P[m,j]  = | sum_n y[m,n] exp(-2 pi i (c0+j) n / N) |   (or its square)
 * band_out (host pointer, may be NULL) receives the bins used. The first call
 * for a new (N, band) builds its twiddle table (one allocation).
 * Arithmetic: FP32 (each row's mean level removed before the detrend and
 * mean filter); the transform on the tensor cores with FP16 operands: per row
 * and 256-sample block, y scaled by a power of two and split into an 8-bit
 * integer and the FP16 head and tail of the remainder, the twiddles (x 2^9)
 * into a 10-bit integer and the FP16 head and tail of the remainder; the
 * integer x integer product accumulates exactly, the rest in a second FP32
 * accumulator. Each map element is within 1e-4 of FP64 relative to
 * max(|element|, 1e-6 x the map's largest element). Errors: INVALID_ARG for sizes or
 * parameters out of range (M, N <= 0, ldx or ld_map too small, even or too
 * long a mean filter), UNSUPPORTED beyond the handle's maxima, CUDA_ERROR on
 * a failed launch. */
rcfar_status rcfar_preprocess(rcfar_handle h, const float* x, int32_t M, int32_t N, int64_t ldx,
                              const rcfar_pre_params* p, float* map, int64_t ld_map,
                              rcfar_band* band_out, rcfar_stream stream);

/* eq. 3: summed-area table of map [rows][ld] (dtype; F16 values are
 * stored * 2^map_exp2) in the given mode. value_bound > 0 is an upper bound
 * on |value| supplied by the caller (rcfar_preprocess's band.value_bound for
 * its maps); value_bound <= 0 makes the library measure max |value| first
 * (one extra read of the map). Values above the bound, and NaNs, raise
 * RCFAR_ERR_RANGE at rcfar_get_error. view_out (host pointer) describes the
 * table, which lives in the handle's workspace. */
rcfar_status rcfar_sat(rcfar_handle h, const void* map, int32_t dtype, int32_t map_exp2, int32_t rows,
                       int32_t cols, int64_t ld, float value_bound, int32_t mode,
                       rcfar_sat_view* view_out, rcfar_stream stream);

/* eqs. 1, 2, 4: 2D CA-CFAR on a table from rcfar_sat and its map. For an
 * exact table (TILE_I64, I64) the map may be NULL: the CUT value then comes
 * from the table itself as the sum over the 1x1 region. For every
 * interior CUT (outer rectangle inside the map) whose column lies in
 * [cut_c_lo, cut_c_hi]: S_ref = A(outer) - A(guard), each region sum from four
 * table lookups A = L1 + L4 - (L2 + L3); T = alpha * S_ref / n_ref;
 * det = 1 (H1) iff CUT > T (CUT == T decides H0). Every other cell gets
 * det = 0 and thr = 0. det is uint8 [rows][ld_det]; thr (optional, NULL) is
 * float [rows][ld_thr]. Zero interior CUTs is valid (all-zero det).
 * GO / SO windows (w->kind): each half sum is A(rows of the half, outer
 * columns) - A(its guard rows, guard columns), from the same table rows, and
 * T = t * max or min of the two; every table mode supports them. */
rcfar_status rcfar_cfar(rcfar_handle h, const rcfar_sat_view* view, const void* map, int32_t dtype,
                        int32_t map_exp2, int64_t ld_map, const rcfar_window* w, int32_t cut_c_lo,
                        int32_t cut_c_hi, uint8_t* det, int64_t ld_det, float* thr, int64_t ld_thr,
                        rcfar_stream stream);

/* rcfar_sat + rcfar_cfar fused, with no table in device memory: every CTA
 * walks a strip of the map (plus the window halo) down a run of rows,
 * keeping the last rows of the strip's exact 64-bit integral image (eq. 3)
 * in shared memory, and takes the eq. 4 lookups there (float16 maps: one
 * integral image per block of rows instead). The
 * quantisation and fixed-point scale are those rcfar_sat uses for
 * (value_bound > 0, the window), so the decisions and thresholds are
 * bit-identical to rcfar_sat(TILE_I64 or I64) followed by rcfar_cfar with the
 * same CUT source: the map's values when map_cut != 0, else the table's 1 x 1
 * region sums. map: [rows][ld_map] of dtype (F16 values times 2^map_exp2).
 * Float32 maps wider than one strip whose rows start on 16-byte boundaries
 * (map 16-byte aligned, ld_map a multiple of 4) have each stage's rows
 * brought by the tensor memory accelerator, which is faster; the results are
 * the same either way. UNSUPPORTED when the window's halo does not fit shared
 * memory. A value above value_bound (or NaN) is reported by rcfar_get_error
 * as RANGE. */
rcfar_status rcfar_sat_cfar(rcfar_handle h, const void* map, int32_t dtype, int32_t map_exp2, int32_t rows,
                            int32_t cols, int64_t ld_map, float value_bound, const rcfar_window* w, int32_t cut_c_lo,
                            int32_t cut_c_hi, int32_t map_cut, uint8_t* det, int64_t ld_det, float* thr,
                            int64_t ld_thr, rcfar_stream stream);

/* The same decisions with S_ref summed cell by cell over the n_ref training
 * cells (the sliding-window CA-CFAR that the SAT replaces; Sec. III, Table I
 * "CA-CFAR"). map is float32 [rows][ld_map]. Also the OS variant: the k-th
 * smallest training cell of each CUT, selected exactly (a bitwise search
 * over the order-preserving 32-bit keys of the cells). */
rcfar_status rcfar_cfar_direct(rcfar_handle h, const float* map, int32_t rows, int32_t cols,
                               int64_t ld_map, const rcfar_window* w, int32_t cut_c_lo,
                               int32_t cut_c_hi, uint8_t* det, int64_t ld_det, float* thr,
                               int64_t ld_thr, rcfar_stream stream);

/* Writes the table's values S(r, c) as float64 [rows][ld_out] (testing and
 * error studies; S = local + carries * 2^-scale, exact unless the table
 * wrapped modulo 2^64). */
rcfar_status rcfar_sat_materialize(rcfar_handle h, const rcfar_sat_view* view, double* out,
                                   int64_t ld_out, rcfar_stream stream);

/* ---- batched path ------------------------------------------------------ */

/* Whole chain (rcfar_preprocess -> rcfar_sat(TILE_I64) -> rcfar_cfar with the
 * band's CUT columns) for n frames of uneven size and window in a handful of
 * launches over all frames. frames is a HOST array of n descriptors; their
 * pointers are device pointers. Each frame's results are identical whatever
 * the rest of the batch holds. Fails with RCFAR_ERR_OUT_OF_WORKSPACE if the
 * batch needs more than cfg.batch_bytes (see rcfar_batch_bytes). */
rcfar_status rcfar_run_batch(rcfar_handle h, const rcfar_frame_desc* frames, int32_t n,
                             const rcfar_pre_params* p, rcfar_stream stream);
/* Workspace bytes one frame of size M x N with parameters p (and window w,
 * needed when p->halo_c is -1) takes in a batch. */
rcfar_status rcfar_batch_bytes(int32_t M, int32_t N, const rcfar_pre_params* p, const rcfar_window* w,
                               int64_t* bytes_out);
/* Builds the twiddle tables rcfar_run_batch will need for these frames (and
 * rcfar_preprocess for frames of the same N and band) ahead of time, so that
 * those calls can be captured in a CUDA graph (no allocation inside). Only
 * the frames' N and windows are read. */
rcfar_status rcfar_prepare(rcfar_handle h, const rcfar_frame_desc* frames, int32_t n, const rcfar_pre_params* p);

/* ---- batch tuning ------------------------------------------------------- */

/* How rcfar_run_batch lays its work out on the GPU. Every tuning gives the
 * same results (bit for bit): only the schedule changes. */
typedef struct rcfar_batch_tuning {
  int32_t dft_kblocks_per_cta;  /* K blocks (256 samples) per band-DFT CTA; 0 = automatic (about two waves) */
  int32_t sat_mode;             /* RCFAR_SAT_TILE_I64 (tile-local table, register-staged CFAR),
                                   RCFAR_SAT_I64 (table S itself, CFAR streaming it through a
                                   bulk-copy ring) or RCFAR_SAT_FUSED (no table: each CTA builds
                                   its block's integral image in shared memory); a group whose
                                   windows do not fit the chosen kernel uses TILE_I64 */
  int32_t cfar_tile_rows;       /* TILE_I64 CFAR strip: CUT rows per step and columns; 0 = automatic */
  int32_t cfar_tile_cols;
  double best_ms;               /* rcfar_tune_batch: time of one batch with this tuning */
  int32_t candidates;           /* rcfar_tune_batch: tunings timed */
  int32_t dft_operands;         /* band-DFT operand staging: 0 = tensor memory accelerator (default),
                                   1 = cp.async copies (the path taken when a tensor map cannot be
                                   made); both give bit-identical results; the autotuner keeps 0 */
} rcfar_batch_tuning;

/* Autotuner: times rcfar_run_batch on these frames (outputs are written)
 * under candidate tunings -- band-DFT K split {auto, 1, 2, 4, 8, 16}, then the
 * table mode (TILE_I64, I64, FUSED) and CFAR strip shapes with the best split -- with CUDA events
 * on the stream, `reps` batches each after one untimed batch, and keeps the
 * fastest in the handle for later rcfar_run_batch calls (out may be NULL).
 * Synchronises the stream; not usable during stream capture (BAD_STATE). */
rcfar_status rcfar_tune_batch(rcfar_handle h, const rcfar_frame_desc* frames, int32_t n, const rcfar_pre_params* p,
                              int32_t reps, rcfar_batch_tuning* out, rcfar_stream stream);
/* Sets (e.g. a saved tuning) or reads the handle's batch tuning.
 * INVALID_ARG for a negative split, an unknown mode or a bad strip. */
rcfar_status rcfar_set_batch_tuning(rcfar_handle h, const rcfar_batch_tuning* t);
rcfar_status rcfar_get_batch_tuning(rcfar_handle h, rcfar_batch_tuning* out);

/* ---- without allocation ------------------------------------------------ */

/* SAT (exact TILE_I64 table) and SAT CA-CFAR of one float32 map, like
 * rcfar_sat + rcfar_cfar, for callers that cannot allocate device memory:
 * real-time loops whose memory is fixed at start-up (an allocation may
 * synchronise the device and stall the loop), and hosts whose device memory
 * belongs to another memory manager that the library must not bypass. The
 * paper has no counterpart; this is a deployment variant of the same
 * computation.
 * No handle and no allocation: the scratch (table and carries) is one
 * 16 MiB array in the library's device memory, held by every GPU that loads
 * the library until exit. Maps whose table does not fit (about 1.9 million
 * cells, e.g. 1024 x 1800) return RCFAR_ERR_UNSUPPORTED, as do windows whose
 * halo does not fit in shared memory (guard_r + train_r > 1024,
 * guard_c + train_c > 119, or a ring too large for the device). value_bound must be > 0 (an upper
 * bound on |value|). status (optional device int32) is zeroed and then set to
 * a non-zero value if a map value exceeds value_bound or is NaN (results
 * invalid). The first call on a device looks up the array's device address
 * and must come before any stream capture. All calls share the array: calls
 * whose work overlaps on the GPU (other streams, other host threads) race
 * and must be serialised by the caller. */
rcfar_status rcfar_sat_cfar_static(const float* map, int32_t rows, int32_t cols, int64_t ld_map, float value_bound,
                                   const rcfar_window* w, int32_t cut_c_lo, int32_t cut_c_hi, uint8_t* det,
                                   int64_t ld_det, float* thr, int64_t ld_thr, int32_t* status,
                                   rcfar_stream stream);

/* ---- serving: continuous batching of frames from many sources ---------- */

/* A request loop in the library: frames from many sources (drones) are
 * submitted at any time, each from HOST memory or already in DEVICE memory;
 * a scheduler thread admits them, in arrival order, into batches that fit the
 * device-memory budget and runs up to `slots` batches at once, each on its
 * own stream (host frames: copies in, the rcfar_run_batch chain, decisions
 * out; device frames: the chain reads the frame where it lies and writes the
 * decisions to the caller's device buffer), so the work of requests that
 * arrive while others are on the GPU overlaps theirs; a completion thread
 * publishes each frame's completion with timestamps (and copies host
 * frames' decisions to the caller's host buffers). Each frame's decisions are
 * identical to those of the frame run alone (rcfar_run_batch results do not
 * depend on the rest of the batch), whichever memory it came from. The paper
 * processes one frame at a time (Sec. III); this is the deployment form for
 * many radars. Twiddle tables are kept on the device per (N, band) once
 * built. The server's threads call only the library; the server is
 * thread-safe. */
typedef struct rcfar_server_s* rcfar_server;

typedef struct rcfar_server_config {
  int32_t device;
  int64_t budget_bytes;      /* device memory for frames in flight (inputs, decisions, workspaces);
                                split evenly between the slots */
  int32_t slots;             /* batches in flight at once, 1..8 */
  int32_t max_batch_frames;  /* frames per batch, 1..64 */
  int32_t max_rows;          /* largest M accepted */
  int32_t max_n;             /* largest N accepted */
  int32_t max_window;        /* largest guard + training per side accepted */
  rcfar_pre_params params;   /* fs, band, mean filter; halo_c must be -1 (each frame its own window) */
} rcfar_server_config;

/* Where a request's frame and decisions live. */
typedef enum rcfar_memory { RCFAR_MEM_HOST = 0, RCFAR_MEM_DEVICE = 1 } rcfar_memory;

typedef struct rcfar_request {
  const float* x;          /* raw frame, M rows of ldx floats (or N rows of M for trace-major frames).
                              RCFAR_MEM_HOST: host memory (pinned memory: asynchronous copy);
                              RCFAR_MEM_DEVICE: device memory of the server's device, read in place by
                              the chain; the work that wrote it must be complete at submission */
  int32_t M, N;
  int64_t ldx;
  rcfar_window window;
  uint8_t* det;            /* output M x C, C = rcfar_band_plan(N, params with halo_c = the window's
                              guard_c + train_c).cols, in the same memory as x; written before the
                              completion appears (device: by the server's stream, complete when the
                              completion is polled) */
  int64_t ld_det;
  int64_t tag;             /* caller's identifier, returned with the completion */
  int64_t arrival_ns;      /* arrival time on rcfar_server_now_ns's clock; 0 = at submission */
  int32_t memory;          /* rcfar_memory of x and det (0: host) */
  int32_t pad;
} rcfar_request;

typedef struct rcfar_completion {
  int64_t tag;
  int32_t status;          /* rcfar_status of the frame's batch */
  int32_t batch_frames;    /* frames in the batch it ran in */
  int32_t slot;
  int32_t pad;
  int64_t arrival_ns, admit_ns, done_ns;  /* latency = done_ns - arrival_ns */
} rcfar_completion;

typedef struct rcfar_server_stats {
  int64_t submitted, completed, batches;
  int64_t max_batch_frames_seen;
  int64_t max_inflight_frames;    /* largest number of frames admitted at once */
  int64_t device_bytes;           /* device memory held by the server (slots, workspaces, tables) */
} rcfar_server_stats;

/* Creates the server and its threads; allocates all slot memory up front.
 * INVALID_ARG for a bad configuration, CUDA if allocation fails. */
rcfar_status rcfar_server_create(const rcfar_server_config* cfg, rcfar_server* out);
/* Queues one frame (the request is copied; x and det must stay valid until
 * its completion is polled). A device frame takes only its batch workspace
 * from the slot's budget share (no staging copies). UNSUPPORTED if the frame
 * exceeds the configured maxima or could never fit one slot's share of the
 * budget; INVALID_ARG for bad sizes, window or memory kind, or a device
 * pointer that is not memory of the server's device; BAD_STATE after destroy
 * has begun. */
rcfar_status rcfar_server_submit(rcfar_server srv, const rcfar_request* req);
/* Queues reqs[0..n) (a HOST array) in order, under one lock, as if submitted
 * one by one at the same instant (a burst from a front-end). Stops at the
 * first request that rcfar_server_submit would refuse and returns that
 * status; *n_queued (may be NULL) receives how many were queued. */
rcfar_status rcfar_server_submit_many(rcfar_server srv, const rcfar_request* reqs, int32_t n, int32_t* n_queued);
/* Builds, on every slot, the twiddle tables of frames with these slow-time
 * lengths N[i] and windows w[i] (host arrays of n), so that the first frames
 * of each size do not wait for them. Optional. */
rcfar_status rcfar_server_prepare(rcfar_server srv, const int32_t* N, const rcfar_window* w, int32_t n);
/* Returns up to max completions (out: host array); waits up to wait_ms
 * milliseconds for the first one (0: do not wait). */
rcfar_status rcfar_server_poll(rcfar_server srv, rcfar_completion* out, int32_t max, int32_t* n_out,
                               int32_t wait_ms);
rcfar_status rcfar_server_get_stats(rcfar_server srv, rcfar_server_stats* out);
/* Monotonic clock the server stamps requests with (nanoseconds). */
int64_t rcfar_server_now_ns(void);
/* Completes every submitted frame, stops the threads and frees the server. */
rcfar_status rcfar_server_destroy(rcfar_server srv);

/* ---- tracing ----------------------------------------------------------- */

/* Per-kernel device time of the handle's launches (CUDA events around each
 * launch, on the launching stream). Not usable inside CUDA-graph capture. */
typedef struct rcfar_trace_entry {
  char name[32];     /* kernel family: colstats, band_dft, normalise, sat, cfar, cfar_direct, ... */
  int64_t launches;
  double total_ms;
} rcfar_trace_entry;
/* Starts (on != 0) or stops recording; starting clears earlier records. */
rcfar_status rcfar_trace_enable(rcfar_handle h, int32_t on);
/* Waits for the recorded launches and returns one entry per kernel family
 * (out: host array of max_entries; *n_out receives the number written). */
rcfar_status rcfar_trace_read(rcfar_handle h, rcfar_trace_entry* out, int32_t max_entries, int32_t* n_out);

/* ---- errors ------------------------------------------------------------ */

/* Self-test of failure detection: runs one kernel that waits on a barrier
 * nothing completes, giving up after `polls` polls (each suspends at most
 * about a microsecond), the bounded wait every waiting kernel of the library
 * uses; the kernel records the timeout and returns, and the device stays
 * usable. Returns RCFAR_ERR_TIMEOUT when the wait ran out (the expected
 * result), RCFAR_OK if it completed, RCFAR_ERR_INVALID_ARG unless
 * 0 < polls <= 2^20, RCFAR_ERR_CUDA on a CUDA error. Synchronous. */
rcfar_status rcfar_selftest_wait(int32_t device, int32_t polls);

/* Waits for the stream, then returns (and clears) the first asynchronous
 * error the kernels recorded on this handle: RCFAR_ERR_RANGE,
 * RCFAR_ERR_TIMEOUT or RCFAR_OK. */
rcfar_status rcfar_get_error(rcfar_handle h, rcfar_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* RCFAR_H */
