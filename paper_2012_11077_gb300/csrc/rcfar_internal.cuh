// Internal definitions shared by the librcfar translation units.
//
// Device-side descriptors are passed to kernels as __grid_constant__
// parameters (up to 32 KB), so a launch carries its whole batch table and can
// be captured in a CUDA graph without any host->device copy.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
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
constexpr int kStatsStrip = 128;  // columns per column-statistics CTA

// CUDA-core band DFT tile: 128 rows x 64 real outputs (32 bins) x 32 samples.
constexpr int kDftBM = 128;
constexpr int kDftBN = 64;
constexpr int kDftBK = 32;

struct PreFrameDev {
  const float* x;
  long long ldx;
  int M, N;
  int c0, C;  // stored bins c0 .. c0 + C - 1
  int h;      // mean filter half length
  float mbar, inv_M, inv_D;
  const float* W;  // twiddles [N][ldw]: column 2j = cos, 2j+1 = -sin of bin c0+j
  long long ldw;
  float2* stats;        // [N] (a_n, b_n) of the fast-time line fit
  float2* partial;      // [n_chunks][N] partial sums (sum x, sum (m-mbar) x)
  float* rowpart;       // [n_strips][M] partial row sums sum_j w_j x[m, j]
  float2* strip_ab;     // [n_strips] (sum_j w_j a_j, sum_j w_j b_j) over the strip
  unsigned* strip_cnt;  // [n_strips] arrival counters (self-resetting)
  unsigned* ymax;       // float bits of max |y| over the frame
  float* map;           // [M][ld_map] band map (unnormalised until k_normalise)
  long long ld_map;
  float* kpart;         // split-K partial sums [splitk][M][ldk]
  long long ldk;
  unsigned* tile_cnt;   // [mtiles * ntiles] arrival counters (self-resetting)
  int rows_per_chunk, n_chunks, n_strips;
  int mtiles, ntiles, splitk, kper;
  int item_stats, item_dft, item_norm;  // first CTA of this frame in each launch
  int n_norm;                            // CTAs of this frame in k_normalise
};

struct PreBatch {
  int n;
  PreFrameDev f[kMaxBatch];
};

struct SatMapDev {
  const void* map;
  long long ld;
  int rows, cols;
  float in_scale;        // value = stored * in_scale (F16 maps)
  int scale_log2;        // fixed-point scale; kScaleFromDevice: derive from *bound_dev
  const float* bound_dev;
  float bound;           // |value| bound checked per cell
  long long max_cells;   // largest region (cells) the scale must cover
  void* table;           // float (TILE_F32, NAIVE) or int64 (I64) [rows][ld_table]
  long long ld_table;
  // vertical carries: per (band, column) -- band aggregate and inclusive value
  unsigned long long* v_agg;      // [n_bands][ld_carry]
  unsigned long long* row_carry;  // [n_bands][ld_carry] = S(last row of band, c)
  long long ld_carry;
  // horizontal carries: per (tile, band row) -- row totals, aggregate and inclusive
  unsigned long long* h_agg;      // [n_bands * n_chunks][32]
  unsigned long long* h_inc;      // [n_bands * n_chunks][32]
  unsigned long long* col_carry;  // [n_chunks][rows] band-local sums left of the tile
  unsigned* h_flags;     // [n_bands * n_chunks]
  unsigned* v_flags;     // [n_bands * n_chunks]
  int* scale_out;        // device slot receiving the scale used
  int n_bands, n_chunks;
  int item0;             // first tile ticket of this map
};

struct SatBatch {
  int n;
  int total;         // CTAs in the launch (tiles over all maps)
  unsigned* ticket;  // dynamic tile ticket (self-resetting)
  unsigned* done;    // CTAs finished (self-resetting)
  unsigned* gen;     // launch generation tag of the look-back flags
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
  float kthr;          // alpha / n_ref
  int cut_lo, cut_hi;  // CUT column range (after the interior clip)
  int row_lo, row_hi;  // CUT row range
  unsigned char* det;
  long long ld_det;
  float* thr;
  long long ld_thr;
  int tiles_x;         // CTAs per tile row
  int item0;
  int bh, bw;          // output tile
};

struct CfarBatch {
  int n;
  CfarMapDev m[kMaxBatch];
};

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

// ---- launchers (implemented in the .cu files) -------------------------------
cudaError_t launch_colstats(const PreBatch& b, int blocks, cudaStream_t s);
cudaError_t launch_band_dft(const PreBatch& b, int blocks, cudaStream_t s);
cudaError_t launch_normalise(const PreBatch& b, int blocks, cudaStream_t s);
cudaError_t launch_twiddles(float* W, long long ldw, int N, int c0, int C, cudaStream_t s);

cudaError_t launch_map_max(const void* map, int dtype, float in_scale, int rows, int cols, long long ld,
                           float* out_bits, cudaStream_t s);
cudaError_t launch_sat(const SatBatch& b, int mode, int dtype, cudaStream_t s);
cudaError_t launch_sat_materialize(const SatMapDev& m, int mode, double* out, long long ld_out,
                                   cudaStream_t s);

cudaError_t launch_cfar(const CfarBatch& b, int mode, int dtype, int blocks, size_t smem, cudaStream_t s);
size_t cfar_smem_bytes(int mode, int bh, int bw, int wr, int wc);
cudaError_t launch_cfar_direct(const CfarMapDev& m, int blocks, size_t smem, cudaStream_t s);
size_t cfar_direct_smem_bytes(int bh, int bw, int wr, int wc);

}  // namespace rcfar
