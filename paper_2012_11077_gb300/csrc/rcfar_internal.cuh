// Internal definitions shared by the librcfar translation units.
//
// Device-side descriptors are passed to kernels as __grid_constant__
// parameters (up to 32 KB), so a launch carries its whole batch table and can
// be captured in a CUDA graph without any host->device copy.
#pragma once

#include <cuda.h>
#include <utility>  // CUtensorMap (the type only; the encoder is looked up at run time)
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/rcfar.h"

namespace rcfar {

// Bits of the device status word (sticky until rcfar_get_error).
enum : int { kStatusRange = 1, kStatusTimeout = 2 };

// Bounded waits: iterations of a flag poll (each with a short nanosleep)
// before a kernel gives up, records kStatusTimeout and carries on.
constexpr unsigned kSpinLimit = 1u << 20;

constexpr int kMaxBatch = 64;      // frames / maps per launch
constexpr int kMaxMeanHalf = 16;   // mean filter length <= 33

// ---- summed-area table geometry (TILE_F32 / I64 / NAIVE) ------------------
constexpr int kSatTileH = 32;   // rows per band (one CTA per band)
constexpr int kSatTileW = 128;  // columns per chunk (32 lanes x 4)

// ---- preprocessing ----------------------------------------------------------
constexpr int kStatsStrip = 128;         // columns per column-statistics CTA
constexpr int kStatsRowsPerChunk = 64;   // rows per column-statistics chunk (8 warps x 8)

// Band DFT GEMM on tcgen05: 128 rows (TMEM lanes) x up to kDftMaxBN real
// outputs (TMEM columns) per CTA, K steps of 64 samples (one 128-byte swizzle row of
// FP16 head or tail values).
constexpr int kDftBM = 128;
constexpr int kDftMaxBN = 160;  // real outputs per CTA: two pipeline stages of operands fit shared memory
constexpr int kDftBK = 64;
constexpr int kDftMaxStages = 4;
constexpr int kDftSmemCap = 220 * 1024;
// Operand split of the band DFT. In each K block of 256 samples, y of row m
// is scaled by 2^s(m, block) so that its largest magnitude lies in [64, 128)
// and written as three FP16 planes: Y0 = rint(y 2^s) (an integer, |Y0| <= 128),
// and the FP16 head Rh and tail Rt of the remainder y 2^s - Y0 (|.| <= 1/2).
// The twiddles are scaled by 2^kDftTBits and written as three planes: the
// integer T0 = rint(W 2^9) (|T0| <= 512), the FP16 head T1 of W 2^9 - T0 and
// the FP16 tail T2 of what remains (about 31 bits together).
// Six products per K step go into two accumulators in tensor memory:
//   ACC_A = sum Y0 T0: integers, |.| <= 256 * 128 * 512 = 2^24 per block, so
//           every partial sum is exactly representable in FP32 and the
//           accumulation is exact however the tensor core rounds its adds;
//   ACC_B = sum Y0 T1 + Y0 T2 + Rh T0 + Rh T1 + Rt T0: about 2^-8 of ACC_A's
//           size, so the accumulator's own rounding (toward zero) costs 2^-8
//           of what one FP32 accumulator of the whole product would.
// The drain adds ACC_A + ACC_B once (round to nearest) and scales by
// 2^-s 2^-9 (exact); blocks' partials are added with Kahan compensation.
constexpr int kDftKB = 4;
constexpr int kDftBlock = kDftBK * kDftKB;  // samples per K block
constexpr int kDftYPlanes = 3;              // Y0, Rh, Rt
constexpr int kDftWPlanes = 3;              // T0, T1, T2
constexpr int kDftTBits = 9;                // twiddle scale 2^9: |T0| <= 512
constexpr int kDftThreads = 384;  // warp 0 MMA, warps 1-7 producers, warps 8-11 drain
// y pass: 8 rows (one per warp) x kYCols samples per CTA (two K blocks).
constexpr int kYRows = 8;
constexpr int kYCols = 512;
static_assert(kYCols == 2 * kDftBlock, "a y-pass column block holds two K blocks");

struct PreFrameDev {
  const float* x;
  long long ldx;
  int M, N;
  int c0, C;  // stored bins c0 .. c0 + C - 1
  int h;      // mean filter half length
  float mbar, inv_M, inv_D;
  double inv_D64;    // 1 / sum (m - mbar)^2 in FP64 (the slope's final division)
  const __half* Wt;  // twiddles x 2^kDftTBits, transposed and split: planes T0, T1, T2, each [ldw][npad];
                     // row 2j = cos, 2j+1 = -sin of bin c0+j; zero padded
  long long ldw;     // real output columns incl. padding = ntiles * bn
  __half* yq;        // [kDftYPlanes][M][npad]: Y0, Rh, Rt of (y minus its row mean) x 2^s(m, K block)
                     // (plane stride M * npad); zero for n >= N
  float* yscale;     // [nblocks][M] 2^-s(m, K block) 2^-kDftTBits, by which the drain multiplies each partial
  float* rowmean;    // [M] the row means c_m removed from y
  float* rowsq;      // z-score normalisation: [ycols][M] per-block sums of (y - c_m)^2
  const float* xsrc; // trace-major input [N][ldsrc] transposed into x (nullptr: x is the input)
  long long ldsrc;
  int item_tr, n_tr; // transpose: first CTA and CTA count of this frame
  int detector;      // rcfar_detector
  int normalise;     // rcfar_normalise
  int npad;          // N rounded up to kDftBK
  int bn;            // real output columns per CTA (multiple of 16, <= kDftMaxBN)
  float2* stats;        // [N] (a_n, b_n) of the fast-time line fit
  float4* partial;      // [n_chunks][N] partial sums (sum x, its error, sum (m-mbar) x, its error)
  float* rowpart;       // [n_strips][M] partial row sums sum_j w_j x[m, j]
  float2* strip_ab;     // [n_strips] (sum_j w_j a_j, sum_j w_j b_j) over the strip
  unsigned* strip_cnt;  // [n_strips] arrival counters (self-resetting)
  unsigned* ymax;       // float bits of max |y| over the frame
  float* map;           // [M][ld_map] the normalised band map
  long long ld_map;
  float* kpart;         // K-block partial sums [nblocks][ldk][M], column-major (ldk = ldw)
  int nblocks;          // npad / kDftBlock, rounded up
  long long ldk;
  unsigned* tile_cnt;   // [mtiles * ntiles] arrival counters (self-resetting)
  int chunks_per_cta, n_chunks, n_strips;  // k_colstats: CTAs per frame n_strips x ceil(n_chunks / chunks_per_cta)
  int mtiles, ntiles, splitk, kper;
  int item_stats, item_dft, item_norm, item_y;  // first CTA of this frame in each launch
  int n_norm;                                    // CTAs of this frame in k_dft_reduce
  int ycols;                                     // column blocks of the y pass
};

struct PreBatch {
  int n;
  int dft_smem;  // dynamic shared memory of the k_band_dft launch
  int* status;   // device status word (bounded waits)
  PreFrameDev f[kMaxBatch];
};

// Band DFT fed by the tensor memory accelerator: per frame, the tensor maps
// of the y planes [3][M][npad] (box 64 x 128 x 1) and of the twiddle planes
// [3][ldw][npad] (box 64 x bn x 1), both with the
// 128-byte swizzle the MMA descriptors read. The maps are kernel parameters
// (param space), so a launch needs no copy and is graph-capturable.
struct DftFrameDev {
  float* kpart;         // K-block partials [nblocks][ldk][M], column-major
  const float* yscale;  // [nblocks][M] 2^-s(m, block): the drain writes partials in the units of y
  long long ldk;
  int M, bn, mtiles, ntiles, kper, npad, item_dft, pad;
};
struct DftBatch {
  CUtensorMap ma[kMaxBatch];
  CUtensorMap mb[kMaxBatch];
  DftFrameDev f[kMaxBatch];
  int n;
  int dft_smem;
  int* status;
};
constexpr int kDftTmaThreads = 192;  // warp 0 MMA, warp 1 TMA producer, warps 2-5 drain
static_assert(alignof(CUtensorMap) >= 64 && offsetof(DftBatch, ma) == 0 && offsetof(DftBatch, mb) % 64 == 0,
              "tensor maps must sit 64-byte aligned in the launch parameters");
static_assert(sizeof(DftBatch) <= 32000, "launch parameters are limited to 32 KB");

struct SatMapDev {
  const void* map;
  long long ld;
  int rows, cols;
  float in_scale;        // value = stored * in_scale (F16 maps)
  int scale_log2;        // fixed-point scale; kScaleFromDevice: derive from *bound_dev
  const float* bound_dev;
  float bound;           // |value| bound checked per cell
  long long max_cells;   // largest region (cells) the scale must cover
  void* table;           // float (TILE_F32, NAIVE) or int64 (TILE_I64, I64) [rows][ld_table]
  long long ld_table;
  unsigned long long* col_tot;    // [n_bands][ld_carry]: tile column totals, then each band's row prefix
  unsigned long long* row_tot;    // [n_bands * n_chunks][kSatTileH]: tile row totals
  unsigned long long* row_carry;  // [n_bands][ld_carry]: S(last row of the band, c)
  unsigned long long* col_carry;  // [n_chunks][rows]: band-local sum left of the tile, rows <= r
  long long ld_carry;
  int* scale_out;        // device slot receiving the scale used
  int n_bands, n_chunks;
  int item_tile, item_band, item_vscan;  // first CTA of this map in each launch
};

struct SatBatch {
  int n;
  int* status;
  SatMapDev m[kMaxBatch];
};

constexpr int kScaleFromDevice = -100000;

struct CfarMapDev {
  // table (see rcfar_sat_view)
  const void* table;
  long long ld_table;
  const unsigned long long* row_carry;
  const unsigned long long* col_carry;
  long long ld_carry;
  const int* scale_dev;
  // map with the CUT values
  const void* map;
  long long ld_map;
  float in_scale;
  int rows, cols;
  int wr, wc, gr, gc;  // outer and guard half-sizes
  float kthr;          // CA: alpha / n_ref; GO / SO: the half-sum factor t
  int kind;            // rcfar_cfar_kind
  int os_rank;         // OS: rank k of the order statistic (1-based)
  int n_ref;           // training cells per CUT
  int cut_lo, cut_hi;  // CUT column range (after the interior clip)
  int row_lo, row_hi;  // CUT row range
  unsigned char* det;
  long long ld_det;
  float* thr;
  long long ld_thr;
  int tiles_x;         // CTAs per row of strips
  int item0;
  int bh, bw;          // CUT rows per step, strip width
  int run;             // rows per CTA (a multiple of bh)
  int ring_rows;       // table rows held in shared memory (a power of two; streaming kernel: NS * kRingSR)
  int mode;            // rcfar_sat_mode of the table
  int hcp;             // streaming kernel: u64 per ring row (strip + halo, even); fused kernel: region row pitch
  int sat_scale;       // fused kernel: fixed-point scale s of the quantisation (as the table's)
  float bound;         // fused kernel: |value| bound checked per cell
};

struct CfarBatch {
  int n;
  int* status;  // device status word (bounded waits of the streaming kernel)
  CfarMapDev m[kMaxBatch];
};

// Streaming SAT-CFAR on an exact global table (I64): strips of kRingW
// columns, kRingSR rows per stage (one warp per row), table rows brought
// into a shared-memory ring by the bulk-copy engine.
constexpr int kRingW = 128;
constexpr int kRingSR = 32;
constexpr int kRingThreads = 1024;
constexpr int kRingBarBytes = 128;  // stage mbarriers at the front of shared memory
constexpr int kRingMaxStages = 16;
static_assert(kRingThreads / 32 == kRingSR && kRingW == 128, "one warp per output row and stage, 4 columns per lane");

// Fixed-point scale s such that max_cells * bound * 2^s <= 2^62 (so every
// region sum the CFAR forms fits in 63 bits); clamped to a float-safe range.
__host__ __device__ inline int sat_scale_for(float bound, long long max_cells) {
  if (!(bound > 0.0f)) return 100;
  double v = (double)bound * (double)max_cells;
  int e = 0;
  // v = f * 2^e with 0.5 <= f < 1 -> v < 2^e
  {
    double f = v;
    while (f >= 1.0) { f *= 0.5; ++e; }
    while (f < 0.5) { f *= 2.0; --e; }
  }
  int s = 62 - e;
  if (s > 100) s = 100;
  if (s < -100) s = -100;
  return s;
}

// Locate the descriptor whose first item is the largest <= item.
template <typename T>
__device__ __forceinline__ int find_item(const T* arr, int n, int item, int T::*field) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (arr[mid].*field <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Raise a kernel's dynamic shared-memory limit once per (kernel, device).
cudaError_t ensure_smem(const void* fn, size_t bytes);

// Programmatic dependent launch. A kernel launched by launch_pdl may begin
// while its predecessor on the stream is still running: it calls pdl_trigger()
// first (so that its own successor may launch once all of its CTAs have
// started) and pdl_wait() before its first access to global memory, which
// returns once the predecessor has completed and its writes are visible.
// Since every such kernel waits before touching global memory, each one also
// runs after all earlier kernels on the stream. Both are no-ops for kernels
// launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, std::forward<Args>(args)...);
}

// ---- launchers (implemented in the .cu files) -------------------------------
cudaError_t launch_colstats(const PreBatch& b, int blocks, cudaStream_t s);
// trace-major frames [N][ldsrc] -> range-major copies [M][ldx] (32 x 32 tiles)
cudaError_t launch_transpose(const PreBatch& b, int blocks, cudaStream_t s);
constexpr int kTrTile = 32;
cudaError_t launch_ysplit(const PreBatch& b, int blocks, cudaStream_t s);
cudaError_t launch_band_dft(const PreBatch& b, int blocks, cudaStream_t s);
cudaError_t launch_band_dft_tma(const DftBatch& b, int blocks, cudaStream_t s);
cudaError_t launch_dft_reduce(const PreBatch& b, int blocks, cudaStream_t s);
cudaError_t launch_twiddles(__half* Wt, long long ldw, int npad, int N, int c0, int C, cudaStream_t s);
// bytes of one K step of the band DFT ring: the y planes (128 rows), the twiddle planes (bn rows)
__host__ __device__ inline int dft_stage_bytes(int bn) { return kDftYPlanes * kDftBM * 128 + kDftWPlanes * bn * 128; }
// accumulator buffers of a band-DFT CTA (each holds ACC_A and ACC_B, bn columns apiece): two
// when both fit the 512 tensor-memory columns, so a block's MMAs run while the previous drains
__host__ __device__ inline int dft_acc_buffers(int bn) { return 4 * bn <= 512 ? 2 : 1; }

cudaError_t launch_map_max(const void* map, int dtype, float in_scale, int rows, int cols, long long ld,
                           float* out_bits, cudaStream_t s);
// Summed-area table of every map of the batch: tile pass, carry scans, and
// (global I64 / NAIVE_F32 only) the pass that folds the carries in.
cudaError_t launch_sat(const SatBatch& b, int mode, int dtype, int tiles, int bands, int vscans, cudaStream_t s);
cudaError_t launch_sat_materialize(const SatMapDev& m, int mode, double* out, long long ld_out,
                                   cudaStream_t s);

cudaError_t launch_cfar(const CfarBatch& b, int mode, int dtype, int blocks, size_t smem, int max_hc, cudaStream_t s);
size_t cfar_smem_bytes(int mode, int bh, int bw, int wr, int wc);
int cfar_ring_rows(int bh, int wr);
cudaError_t launch_cfar_direct(const CfarMapDev& m, int blocks, size_t smem, cudaStream_t s);

// Streaming CFAR: ring plan for a window (false if it does not fit), its
// shared memory, the strip/run geometry of one map (returns its CTA count),
// and the launch. map_cut: CUT values from the map (else from the table).
bool cfar_ring_plan(int wr, int wc, size_t smem_cap, int* ring_rows, int* hcp);
size_t cfar_ring_smem(int ring_rows, int hcp);
int cfar_ring_slots(size_t smem);  // resident CTAs of the streaming kernel on this device
int cfar_ring_geometry(CfarMapDev& P, int rows, int cols, int ring_rows, int hcp, int slots);
cudaError_t launch_cfar_ring(const CfarBatch& b, bool map_cut, int dtype, int blocks, size_t smem, cudaStream_t s);

// Threshold factor of a window (host, FP64): alpha / n_ref for cell
// averaging, the half-sum factor t for greatest-of / smallest-of; cells gets
// n_ref or the cells of one half. False for an invalid window.
bool window_factor(const rcfar_window& w, double* factor, int* cells);

// Fused SAT + CFAR without a table in device memory: each CTA builds the
// exact 64-bit integral image of its region (inner run x strip plus the
// window halo) in shared memory and takes the eq. 4 lookups there. Strips
// cover the whole width when it fits (cols + 1 <= kFusedMaxCols), else
// kRingW columns plus halo. Returns false if no run fits shared memory.
constexpr int kFusedMaxCols = 256;
bool cfar_fused_plan(int rows, int cols, int wr, int wc, size_t smem_cap, int* run, int* bw, int* pitch,
                     size_t* smem);
int cfar_fused_geometry(CfarMapDev& P, int rows, int cols, int run, int bw, int pitch);
cudaError_t launch_cfar_fused(const CfarBatch& b, bool map_cut, int dtype, int blocks, size_t smem, cudaStream_t s);

// Streaming fused SAT + CFAR (float32 maps): a CTA walks a strip of columns
// down a run of rows in stages of kStreamKS rows, keeping the last
// kStreamKS + 2 wr + 1 rows of its local integral image in a ring in shared
// memory. Strips are the whole width when cols + 1 <= kFusedMaxCols, else
// kStreamW columns plus halo (then wc <= 63). The plan picks the run that
// minimises waves x stages for `sm_share` SMs; false if the ring does not
// fit smem_cap.
constexpr int kStreamKS = 16;
constexpr int kStreamThreads = 512;  // one warp per row of a stage
constexpr int kStreamW = 128;
static_assert(kStreamThreads / 32 == kStreamKS, "one warp per stage row");
// Row prefix: each lane holds e consecutive region columns (e in {5, 6, 8},
// 32 e >= the region's columns); ring rows are 32 e + 2 wide so that every
// lane's chunk lies inside its row.
int stream_e_of(int rows, int cols, int wc);  // e needed by one map (0 if it cannot stream)
struct StreamPlan {
  int run, bw, pitch, ring_rows, e;
  size_t smem;
  int ctas;
};
// e_min: the e of the launch the map joins (0: its own).
bool cfar_stream_plan(int rows, int cols, int wr, int wc, size_t smem_cap, int sm_share, int e_min,
                      StreamPlan* out);
int cfar_stream_geometry(CfarMapDev& P, int rows, int cols, const StreamPlan& sp);
cudaError_t launch_cfar_stream(const CfarBatch& b, bool map_cut, int e, int blocks, size_t smem, cudaStream_t s);

// The streaming kernel fed by the tensor memory accelerator, for one float32
// map wider than one strip whose rows start on 16-byte boundaries: each
// stage's map rows arrive as one 2-D box (kStreamKS rows x 32 e columns).
// The plan fails (use the kernel above) when the strip plus halo exceeds
// 32 e columns for e = 8 or the ring does not fit smem_cap.
struct CfarTmaParams {
  CUtensorMap tm;  // the map: float32 [rows][ld], box 32 e x kStreamKS, zero fill outside
  CfarMapDev m;
  int* status;
};
bool cfar_stream_tma_plan(int rows, int cols, int wr, int wc, size_t smem_cap, int sm_share, StreamPlan* out);
cudaError_t launch_cfar_stream_tma(const CfarTmaParams& p, bool map_cut, int e, int blocks, size_t smem,
                                   cudaStream_t s);

// Ordered-statistic CFAR on float32 maps: CTAs of kOsRows x 32 CUTs, one warp
// per CUT row; each CUT's k-th smallest training cell is selected exactly.
constexpr int kOsRows = 8;
constexpr int kOsMaxRef = 2048;  // training cells per CUT (64 per lane)
int cfar_os_geometry(CfarMapDev& P, int rows, int cols);  // CTAs of one map
size_t cfar_os_smem(int wr, int wc, int n_ref);
cudaError_t launch_cfar_os(const CfarBatch& b, int max_n_ref, int blocks, size_t smem, cudaStream_t s);
size_t cfar_direct_smem_bytes(int bh, int bw, int wr, int wc);

}  // namespace rcfar

namespace rcfar {
static_assert(2 * (kDftYPlanes * kDftBM * 128 + kDftWPlanes * kDftMaxBN * 128) + 1024 <= kDftSmemCap,
              "two operand stages of the widest band-DFT tile fit the shared memory cap");
static_assert(2 * kDftMaxBN <= 512, "one accumulator buffer (ACC_A, ACC_B) fits tensor memory");
}  // namespace rcfar
