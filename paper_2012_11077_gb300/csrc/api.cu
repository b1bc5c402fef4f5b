// C ABI of librcfar (see include/rcfar.h): handle, workspace, plans,
// validation and launch orchestration. All numerical work happens in the
// kernels of pre.cu, sat.cu and cfar.cu.
#include "rcfar_internal.cuh"

#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

using namespace rcfar;

namespace {

constexpr int kStatsRows = kStatsRowsPerChunk;  // rows per column-statistics CTA
// The batched chain stores the exact 64-bit tile-local table: its decisions
// are exact for every window (the FP32 tile-local table loses small windows'
// sums), and it needs no pass to fold the carries in.
constexpr int kBatchSatMode = RCFAR_SAT_TILE_I64;

inline long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }
inline long long round_up(long long a, long long b) { return ceil_div(a, b) * b; }
inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Twiddle {
  __half* Wt = nullptr;
  long long ldw = 0;
  int npad = 0, bn = 0;
  bool has_map = false;
  CUtensorMap mb;  // both planes of Wt for the tensor-memory-accelerator band DFT
};

// cuTensorMapEncodeTiled, looked up once from the driver (no link to libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of nplanes planes [nplanes][rows][npad] FP16 (plane stride rows
// * npad): boxes of kDftBK samples (128 bytes) x box_rows rows x 1 plane,
// 128-byte swizzle, rows past the end read as zeros.
bool make_planes_map(CUtensorMap* out, const __half* base, long long rows, int npad, int box_rows, int nplanes) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (npad % kDftBK) || box_rows < 1 || box_rows > 256)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)npad, (cuuint64_t)rows, (cuuint64_t)nplanes};
  const cuuint64_t strides[2] = {(cuuint64_t)npad * sizeof(__half), (cuuint64_t)rows * npad * sizeof(__half)};
  const cuuint32_t box[3] = {(cuuint32_t)kDftBK, (cuuint32_t)box_rows, 1};
  const cuuint32_t elem[3] = {1, 1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<__half*>(base), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of a float32 matrix [rows][ld] (columns 0 .. cols - 1):
// boxes of box_cols x box_rows, no swizzle, zeros outside the matrix.
bool make_map2d(CUtensorMap* out, const void* base, long long rows, long long cols, long long ld, int box_cols,
                int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || (ld % 4) || box_cols < 4 || box_cols > 256 || (box_cols % 4) ||
      box_rows < 1 || box_rows > 256)
    return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t elem[2] = {1, 1};
  return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Bump allocator over a device region.
struct Carver {
  char* base;
  size_t cap, off = 0;
  Carver(void* b, size_t c) : base((char*)b), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    const size_t bytes = align256(count * sizeof(T));
    if (off + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// Per-frame preprocessing geometry (depends on the frame's own shape only,
// so a frame is computed the same way alone and inside any batch).
struct PreGeom {
  int n_strips, n_chunks;
  int mtiles, ntiles, splitk, kper, bn, nblocks;
  int n_norm;
  int npad, ycols, n_y;
  long long ldk, ldw;
};

// band DFT column tiling: ntiles tiles of bn real outputs (bn a multiple of 16, <= kDftMaxBN)
inline void dft_cols(int C, int* ntiles, int* bn) {
  const long long twoC = 2LL * C;
  *ntiles = (int)ceil_div(twoC, kDftMaxBN);
  *bn = (int)round_up(ceil_div(twoC, *ntiles), 16);
}

// dynamic shared memory of a k_band_dft launch whose widest tile is bn
inline int dft_smem_for(int bn) {
  const int sb = dft_stage_bytes(bn);
  const int stages = std::min(kDftMaxStages, (kDftSmemCap - 1024) / sb);
  return 1024 + stages * sb;
}

// kblocks_per_cta > 0 fixes how many K blocks one CTA of the band DFT takes
// (a batch spreads its total work); 0 = one wave for this frame alone. The
// split never changes results: every K block's partial is reduced in order.
PreGeom pre_geom(int M, int N, int C, int kblocks_per_cta = 0) {
  PreGeom g;
  g.n_strips = (int)ceil_div(N, kStatsStrip);
  g.n_chunks = (int)ceil_div(M, kStatsRows);
  g.npad = (int)round_up(N, kDftBK);
  g.ycols = (int)ceil_div(g.npad, kYCols);
  g.n_y = (int)ceil_div(M, kYRows) * g.ycols;
  g.mtiles = (int)ceil_div(M, kDftBM);
  dft_cols(C, &g.ntiles, &g.bn);
  g.ldw = (long long)g.ntiles * g.bn;
  const int tiles = g.mtiles * g.ntiles;
  // about one CTA per SM for a frame on its own (one wave); splits are whole K blocks
  const int kblk = kDftBlock;
  g.nblocks = (int)ceil_div(g.npad, kblk);
  int sk = kblocks_per_cta > 0 ? (int)ceil_div(g.nblocks, kblocks_per_cta) : std::max(1, 152 / tiles);
  if (sk > g.nblocks) sk = g.nblocks;
  g.kper = (int)round_up(ceil_div(g.npad, sk), kblk);
  g.splitk = (int)ceil_div(g.npad, g.kper);
  g.ldk = g.ldw;
  g.n_norm = (int)ceil_div((long long)M * C, 256);  // k_dft_reduce: one thread per map cell
  return g;
}

struct SatGeom {
  int n_bands, n_chunks;
  long long ld_table, ld_carry;
};

SatGeom sat_geom(int rows, int cols) {
  SatGeom g;
  g.n_bands = (int)ceil_div(rows, kSatTileH);
  g.n_chunks = (int)ceil_div(cols, kSatTileW);
  g.ld_table = round_up(cols, 4);
  g.ld_carry = (long long)g.n_chunks * kSatTileW;
  return g;
}

inline bool exact_table(int mode) { return mode == RCFAR_SAT_I64 || mode == RCFAR_SAT_TILE_I64; }

// bytes of SAT storage: the table (4 or 8 B per cell) and the carry arrays
size_t sat_bytes(int rows, int cols, int mode) {
  SatGeom g = sat_geom(rows, cols);
  size_t b = 0;
  b += align256((size_t)rows * g.ld_table * (exact_table(mode) ? 8 : 4));
  b += 2 * align256((size_t)g.n_bands * g.ld_carry * 8);                 // col_tot + row_carry
  b += align256((size_t)g.n_bands * g.n_chunks * kSatTileH * 8);          // row_tot
  b += align256((size_t)g.n_chunks * rows * 8);                           // col_carry
  return b;
}

// The carry arrays of one table, carved from a region.
struct SatArrays {
  unsigned long long *col_tot, *row_tot, *row_carry, *col_carry;
};
template <typename Carve>
bool carve_sat(Carve& data, int rows, int cols, SatArrays* a) {
  SatGeom g = sat_geom(rows, cols);
  a->col_tot = data.template take<unsigned long long>((size_t)g.n_bands * g.ld_carry);
  a->row_carry = data.template take<unsigned long long>((size_t)g.n_bands * g.ld_carry);
  a->row_tot = data.template take<unsigned long long>((size_t)g.n_bands * g.n_chunks * kSatTileH);
  a->col_carry = data.template take<unsigned long long>((size_t)g.n_chunks * rows);
  return a->col_tot && a->row_carry && a->row_tot && a->col_carry;
}
void set_sat_arrays(SatMapDev& m, const SatArrays& a) {
  m.col_tot = a.col_tot;
  m.row_tot = a.row_tot;
  m.row_carry = a.row_carry;
  m.col_carry = a.col_carry;
}

struct CfarTile {
  int bh, bw;
};

bool cfar_tile_fits(int mode, CfarTile t, int wr, int wc, size_t smem_cap) {
  return t.bh > 0 && t.bh <= 16 && t.bw > 0 && 256 % t.bw == 0 && t.bh * t.bw <= 1024 &&
         cfar_smem_bytes(mode, t.bh, t.bw, wr, wc) <= smem_cap && t.bw + 2 * wc + 1 <= 256;
}

// SAT-CFAR geometry: a strip of bw columns, bh CUT rows per step. The
// configured one if it fits, else the first candidate whose ring of table
// rows fits in shared memory (halo rows at most 256 wide). The choice
// depends only on the window, never on the rest of a batch.
CfarTile pick_cfar_tile(int mode, int wr, int wc, size_t smem_cap, CfarTile pref) {
  if (cfar_tile_fits(mode, pref, wr, wc, smem_cap)) return pref;
  const CfarTile cand[] = {{16, 64}, {16, 32}, {8, 64}, {8, 32}, {8, 16}, {4, 16}};
  for (const CfarTile& t : cand)
    if (cfar_tile_fits(mode, t, wr, wc, smem_cap)) return t;
  return {0, 0};
}

constexpr int kCfarRun = 256;  // rows per SAT-CFAR CTA

// Fills the strip geometry of a CFAR descriptor; returns its CTA count. Runs
// are at most kCfarRun rows, and shorter for small maps so that a map on its
// own still spreads over about two CTAs per SM (the halo rows each run
// re-reads are cheap in L2 at those sizes). Depends only on the map itself.
int set_cfar_geometry(CfarMapDev& P, CfarTile t, int rows, int cols) {
  P.bh = t.bh;
  P.bw = t.bw;
  P.tiles_x = (int)ceil_div(cols, t.bw);
  const long long want = ceil_div((long long)rows * P.tiles_x, 2 * 152);
  P.run = (int)std::min<long long>(kCfarRun, std::max<long long>(t.bh, round_up(want, t.bh)));
  P.ring_rows = cfar_ring_rows(t.bh, P.wr);
  return P.tiles_x * (int)ceil_div(rows, P.run);
}

}  // namespace

static int n_ref_of(const rcfar_window& w) {
  const long long wr = w.guard_r + w.train_r, wc = w.guard_c + w.train_c;
  return (int)((2 * wr + 1) * (2 * wc + 1) - (2LL * w.guard_r + 1) * (2LL * w.guard_c + 1));
}

struct rcfar_ctx {
  rcfar_config cfg{};
  int device = 0;
  size_t smem_optin = 48 * 1024;
  int sms = 152;  // streaming multiprocessors of the device
  void* ws = nullptr;  // one allocation holds everything below
  size_t ws_bytes = 0;
  // control words
  int* status = nullptr;
  int* sat_scale = nullptr;
  float* map_bound = nullptr;
  unsigned* ymax = nullptr;
  // per-step preprocessing
  float2* stats = nullptr;
  float4* partial = nullptr;
  float* rowpart = nullptr;
  float2* strip_ab = nullptr;
  unsigned* strip_cnt = nullptr;
  unsigned* tile_cnt = nullptr;
  float* kpart = nullptr;
  size_t kpart_floats = 0;
  void* kpart_own = nullptr;  // separately allocated K-block partials (grown on demand)
  __half* yq = nullptr;  // the y planes (kDftYPlanes x the largest frame)
  float* yscale = nullptr;
  float* rowmean = nullptr;
  float* rowsq = nullptr;
  float* xt = nullptr;  // range-major copy of a trace-major frame
  // per-step SAT
  void* sat_table = nullptr;
  SatArrays sat{};
  uint64_t sat_generation = 0;
  // batch arena
  void* batch = nullptr;
  size_t batch_bytes = 0;
  // twiddle plans
  std::mutex mu;
  std::map<std::tuple<int, int, int>, Twiddle> plans;
  // tracing
  bool trace_on = false;
  struct TraceRec {
    const char* name;
    cudaEvent_t a, b;
  };
  std::vector<TraceRec> trace_pool;
  size_t trace_used = 0;
  // batch schedule (rcfar_tune_batch / rcfar_set_batch_tuning)
  rcfar_batch_tuning tuning{0, RCFAR_SAT_TILE_I64, 0, 0, 0.0, 0, 0};
};

namespace {
// Brackets one kernel launch with events while tracing is on.
struct TraceScope {
  rcfar_ctx* h;
  rcfar_ctx::TraceRec* rec = nullptr;
  cudaStream_t s;
  TraceScope(rcfar_ctx* hh, const char* name, cudaStream_t st) : h(hh), s(st) {
    if (!h->trace_on) return;
    if (h->trace_used == h->trace_pool.size()) {
      rcfar_ctx::TraceRec r{name, nullptr, nullptr};
      if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
      h->trace_pool.push_back(r);
    }
    rec = &h->trace_pool[h->trace_used++];
    rec->name = name;
    cudaEventRecord(rec->a, s);
  }
  ~TraceScope() {
    if (rec) cudaEventRecord(rec->b, s);
  }
};
}  // namespace

namespace {

rcfar_status cuda_fail(cudaError_t e) { return e == cudaSuccess ? RCFAR_OK : RCFAR_ERR_CUDA; }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

bool valid_window(const rcfar_window* w) {
  if (!w || w->train_r < 0 || w->train_c < 0 || w->guard_r < 0 || w->guard_c < 0 || !(w->pfa > 0.0 && w->pfa < 1.0))
    return false;
  const int nr = n_ref_of(*w);
  if (nr <= 0) return false;
  switch (w->kind) {
    case RCFAR_CFAR_CA: return w->os_rank == 0;
    case RCFAR_CFAR_GO:
    case RCFAR_CFAR_SO:
      return w->os_rank == 0 && (long long)(w->guard_r + w->train_r) * (2LL * (w->guard_c + w->train_c) + 1) -
                                        (long long)w->guard_r * (2LL * w->guard_c + 1) > 0;
    case RCFAR_CFAR_OS: return w->os_rank >= 0 && w->os_rank <= nr;
  }
  return false;
}

}  // namespace

static double alpha_of(int n_ref, double pfa) { return (double)n_ref * (std::pow(pfa, -1.0 / (double)n_ref) - 1.0); }

// Greatest-of / smallest-of false-alarm laws on iid exponential noise. The
// half sums X, Y are Gamma(n, 1) and the CUT Exp(1), so P(CUT > t Z) =
// E[exp(-t Z)] for Z = min(X, Y) or max(X, Y). Writing the Gamma(n, 1)
// distribution function as a Poisson tail and integrating term by term gives
// 2 sum_k u_k with u_k = C(n-1+k, k) (2+t)^-(n+k): the terms k < n make the
// smallest-of law, the terms k >= n the greatest-of law. The terms follow
// u_{k+1} = u_k (n+k) / ((k+1)(2+t)) from u_0 = (2+t)^-n; they are summed
// relative to u_0 with a running rescale (they can span thousands of decades)
// until they shrink below 1e-18 of the tail sum, and the laws are returned
// as natural logarithms.
static void go_so_log_laws(int n, double t, double* log_so, double* log_go) {
  const double q = 2.0 + t;
  double u = 1.0, lo = 0.0, hi = 0.0, shift = -(double)n * std::log(q);
  constexpr double kBig = 1e250, kSmall = 1e-250;
  for (long long k = 0;; ++k) {
    if (k < n) lo += u; else hi += u;
    const double ratio = (double)(n + k) / ((double)(k + 1) * q);
    if (k >= n && ratio < 1.0 && u <= 1e-18 * hi) break;
    u *= ratio;
    if (u > kBig) {
      u *= kSmall;
      lo *= kSmall;
      hi *= kSmall;
      shift -= std::log(kSmall);
    }
  }
  const double l2 = std::log(2.0) + shift;
  *log_so = lo > 0.0 ? std::log(lo) + l2 : -INFINITY;
  *log_go = hi > 0.0 ? std::log(hi) + l2 : -INFINITY;
}

// t with law(t) = pfa by bisection: both laws fall from 1 (t = 0) to 0.
static double go_so_factor_of(int kind, int n, double pfa) {
  const double target = std::log(pfa);
  auto law = [&](double t) {
    double a, b;
    go_so_log_laws(n, t, &a, &b);
    return kind == RCFAR_CFAR_SO ? a : b;
  };
  double lo = 0.0, hi = 1.0;
  while (law(hi) > target && hi < 1e300) hi *= 2.0;
  for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (law(mid) > target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

// Ordered-statistic law on iid exponential noise: the k-th smallest of n
// Exp(1) cells is a sum of independent exponentials with rates n, n-1, ...,
// n-k+1, so P(CUT > a X_(k)) = prod_{i<k} (n-i) / (n-i+a); its logarithm,
// accumulated as a product with a rescale, falls monotonically in a.
static double os_log_law(int n, int k, double a) {
  double prod = 1.0, logacc = 0.0;
  for (int i = 0; i < k; ++i) {
    prod *= (double)(n - i) / ((double)(n - i) + a);
    if (prod < 1e-200) {
      logacc += std::log(prod);
      prod = 1.0;
    }
  }
  return logacc + std::log(prod);
}

static double os_factor_of(int n, int k, double pfa) {
  const double target = std::log(pfa);
  double lo = 0.0, hi = 1.0;
  while (os_log_law(n, k, hi) > target && hi < 1e300) hi *= 2.0;
  for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (os_log_law(n, k, mid) > target) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

static int os_rank_of(const rcfar_window& w) {
  const int nr = n_ref_of(w);
  return w.os_rank > 0 ? w.os_rank : (3 * nr + 3) / 4;
}

static long long half_cells_of(const rcfar_window& w) {
  const long long wr = w.guard_r + w.train_r, wc = w.guard_c + w.train_c;
  return wr * (2 * wc + 1) - (long long)w.guard_r * (2LL * w.guard_c + 1);
}

namespace rcfar {
bool window_factor(const rcfar_window& w, double* factor, int* cells) {
  if (w.train_r < 0 || w.train_c < 0 || w.guard_r < 0 || w.guard_c < 0 || !(w.pfa > 0.0 && w.pfa < 1.0))
    return false;
  const int nr = n_ref_of(w);
  if (nr <= 0) return false;
  if (w.kind != RCFAR_CFAR_OS && w.os_rank != 0) return false;
  if (w.kind == RCFAR_CFAR_CA) {
    *factor = alpha_of(nr, w.pfa) / (double)nr;
    if (cells) *cells = nr;
    return true;
  }
  long long n = 0;
  int k = 0;
  if (w.kind == RCFAR_CFAR_GO || w.kind == RCFAR_CFAR_SO) {
    n = half_cells_of(w);
  } else if (w.kind == RCFAR_CFAR_OS) {
    n = nr;
    k = os_rank_of(w);
    if (w.os_rank < 0 || k > nr) return false;
  } else {
    return false;
  }
  if (n <= 0 || n > (1 << 24)) return false;
  // the bisection costs up to a few hundred microseconds for large windows;
  // batches and servers ask for the same few windows again and again
  struct Entry {
    int kind, n, k;
    double pfa, factor;
  };
  static thread_local Entry cache[8] = {};
  static thread_local int next = 0;
  double f = -1.0;
  for (const Entry& e : cache)
    if (e.n == (int)n && e.kind == w.kind && e.k == k && e.pfa == w.pfa) f = e.factor;
  if (f < 0.0) {
    f = w.kind == RCFAR_CFAR_OS ? os_factor_of((int)n, k, w.pfa) : go_so_factor_of(w.kind, (int)n, w.pfa);
    cache[next] = Entry{w.kind, (int)n, k, w.pfa, f};
    next = (next + 1) % 8;
  }
  *factor = f;
  if (cells) *cells = (int)n;
  return true;
}
}  // namespace rcfar

static bool band_of(int N, const rcfar_pre_params* p, rcfar_band* b) {
  if (!p || N <= 0 || !(p->fs_hz > 0.0) || !(p->f_lo_hz >= 0.0) || !(p->f_hi_hz >= p->f_lo_hz) || p->halo_c < 0)
    return false;
  const double lo = p->f_lo_hz * (double)N / p->fs_hz;
  const double hi = p->f_hi_hz * (double)N / p->fs_hz;
  long long k_lo = (long long)std::ceil(lo - 1e-9);
  long long k_hi = (long long)std::floor(hi + 1e-9);
  const long long nyq = N / 2;
  if (k_lo < 0) k_lo = 0;
  if (k_hi > nyq) k_hi = nyq;
  long long c0 = k_lo - p->halo_c;
  long long c1 = k_hi + p->halo_c;
  if (c0 < 0) c0 = 0;
  if (c1 > nyq) c1 = nyq;
  if (c1 < c0) return false;
  b->k_lo = (int)k_lo;
  b->k_hi = (int)k_hi;
  b->c0 = (int)c0;
  b->c1 = (int)c1;
  b->cols = (int)(c1 - c0 + 1);
  // |sum_n y e^{-i..}| <= sum_n |y| <= N after either normalisation (global
  // max: |y| <= 1; z-score: Cauchy-Schwarz with sum z^2 = N)
  b->value_bound = p->detector == RCFAR_DETECT_SQUARE_LAW ? (float)N * (float)N : (float)N;
  return true;
}

static bool valid_pre(const rcfar_pre_params* p) {
  return p && p->mean_len >= 1 && (p->mean_len & 1) && (p->mean_len - 1) / 2 <= kMaxMeanHalf &&
         (p->detector == RCFAR_DETECT_MAGNITUDE || p->detector == RCFAR_DETECT_SQUARE_LAW) &&
         (p->normalise == RCFAR_NORM_GLOBAL_MAX || p->normalise == RCFAR_NORM_ROW_ZSCORE) &&
         (p->x_layout == RCFAR_X_RANGE_MAJOR || p->x_layout == RCFAR_X_TRACE_MAJOR);
}

// leading dimension a raw frame of M x N needs in the given layout
static bool ldx_ok(const rcfar_pre_params* p, int M, int N, long long ldx) {
  return ldx >= (p->x_layout == RCFAR_X_TRACE_MAJOR ? M : N);
}

// twiddle plan for (N, c0, C); builds it on first use
static rcfar_status get_plan(rcfar_ctx* h, int N, int c0, int C, cudaStream_t s, Twiddle* out) {
  std::lock_guard<std::mutex> lk(h->mu);
  auto key = std::make_tuple(N, c0, C);
  auto it = h->plans.find(key);
  if (it != h->plans.end()) {
    *out = it->second;
    return RCFAR_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return RCFAR_ERR_BAD_STATE;  // plans must exist before capture (rcfar_prepare)
  Twiddle t;
  int ntiles = 0, bn = 0;
  dft_cols(C, &ntiles, &bn);
  t.ldw = (long long)ntiles * bn;
  const int npad = (int)round_up(N, kDftBK);
  const size_t bytes = (size_t)kDftWPlanes * t.ldw * npad * sizeof(__half);  // T0, T1, T2 planes
  if (cudaMalloc(&t.Wt, bytes) != cudaSuccess) return RCFAR_ERR_CUDA;
  cudaError_t e = cudaMemsetAsync(t.Wt, 0, bytes, s);  // padding rows and columns stay zero
  if (e == cudaSuccess) e = launch_twiddles(t.Wt, t.ldw, npad, N, c0, C, s);
  if (e != cudaSuccess) {
    cudaFree(t.Wt);
    return RCFAR_ERR_CUDA;
  }
  t.npad = npad;
  t.bn = bn;
  t.has_map = make_planes_map(&t.mb, t.Wt, t.ldw, npad, bn, kDftWPlanes);
  h->plans[key] = t;
  *out = t;
  return RCFAR_OK;
}

// The band-DFT launch parameters of one frame for the TMA-fed kernel (false
// when a tensor map cannot be made; the cp.async kernel runs instead).
static bool make_dft_frame(DftBatch& db, int k, const PreFrameDev& F, const Twiddle& tw, const PreGeom& g) {
  if (!tw.has_map || tw.bn != g.bn || tw.npad != g.npad) return false;
  if (!make_planes_map(&db.ma[k], F.yq, F.M, g.npad, kDftBM, kDftYPlanes)) return false;
  db.mb[k] = tw.mb;
  DftFrameDev& d = db.f[k];
  d.kpart = F.kpart;
  d.yscale = F.yscale;
  d.ldk = F.ldk;
  d.M = F.M;
  d.bn = g.bn;
  d.mtiles = g.mtiles;
  d.ntiles = g.ntiles;
  d.kper = g.kper;
  d.npad = g.npad;
  d.item_dft = F.item_dft;
  d.pad = 0;
  return true;
}

static PreFrameDev make_pre_frame(const float* x, int M, int N, long long ldx, const rcfar_band& b,
                                  const rcfar_pre_params* p, const Twiddle& tw, const PreGeom& g) {
  const int h = (p->mean_len - 1) / 2;
  PreFrameDev F;
  std::memset(&F, 0, sizeof(F));
  F.detector = p->detector;
  F.normalise = p->normalise;
  F.x = x;
  F.ldx = ldx;
  F.M = M;
  F.N = N;
  F.c0 = b.c0;
  F.C = b.cols;
  F.h = h;
  F.mbar = (float)((M - 1) * 0.5);
  F.inv_M = (float)(1.0 / (double)M);
  const double D = (double)M * ((double)M * M - 1.0) / 12.0;
  F.inv_D = D > 0 ? (float)(1.0 / D) : 0.0f;
  F.inv_D64 = D > 0 ? 1.0 / D : 0.0;
  F.Wt = tw.Wt;
  F.ldw = tw.ldw;
  F.npad = g.npad;
  F.ycols = g.ycols;
  F.bn = g.bn;
  F.chunks_per_cta = 1;
  F.n_chunks = g.n_chunks;
  F.n_strips = g.n_strips;
  F.mtiles = g.mtiles;
  F.ntiles = g.ntiles;
  F.splitk = g.splitk;
  F.kper = g.kper;
  F.ldk = g.ldk;
  F.nblocks = g.nblocks;
  F.n_norm = g.n_norm;
  return F;
}

// workspace of one frame in a batch: data, and control words zeroed per batch
static size_t frame_data_bytes(int M, int N, int C, int x_layout) {
  const PreGeom g = pre_geom(M, N, C);
  size_t t = 0;
  if (x_layout == RCFAR_X_TRACE_MAJOR) t += align256((size_t)M * round_up(N, 4) * sizeof(float));  // xt
  t += align256((size_t)N * sizeof(float2));                       // stats
  t += align256((size_t)g.n_chunks * N * sizeof(float4));          // partial
  t += align256((size_t)g.n_strips * M * sizeof(float));           // rowpart
  t += align256((size_t)g.n_strips * sizeof(float2));              // strip_ab
  t += align256((size_t)g.nblocks * M * g.ldk * 4);              // K-block partials
  t += align256((size_t)kDftYPlanes * M * g.npad * sizeof(__half));  // y planes
  t += align256((size_t)g.nblocks * M * sizeof(float));            // yscale
  t += align256((size_t)M * sizeof(float));                        // rowmean
  t += align256((size_t)g.ycols * M * sizeof(float));              // rowsq
  t += align256((size_t)M * round_up(C, 4) * 4);                   // map
  t += sat_bytes(M, C, kBatchSatMode);
  return t;
}
static size_t frame_ctl_bytes(int M, int N, int C) {
  const PreGeom g = pre_geom(M, N, C);
  return align256((size_t)g.n_strips * 4) + align256((size_t)g.mtiles * g.ntiles * 4) + 256;
}

// -------------------------------------------------------------------------
extern "C" {

const char* rcfar_status_string(rcfar_status s) {
  switch (s) {
    case RCFAR_OK: return "ok";
    case RCFAR_ERR_INVALID_ARG: return "invalid argument";
    case RCFAR_ERR_UNSUPPORTED: return "size beyond the handle's limits";
    case RCFAR_ERR_OUT_OF_WORKSPACE: return "batch needs more workspace than the handle holds";
    case RCFAR_ERR_CUDA: return "CUDA runtime error";
    case RCFAR_ERR_TIMEOUT: return "bounded device wait expired";
    case RCFAR_ERR_BAD_STATE: return "bad state (stale view, capture without plan, ...)";
    case RCFAR_ERR_RANGE: return "map value above its stated bound, or NaN";
  }
  return "unknown status";
}

rcfar_status rcfar_alpha(int32_t n_ref, double pfa, double* alpha_out) {
  if (!alpha_out || n_ref <= 0 || !(pfa > 0.0 && pfa < 1.0)) return RCFAR_ERR_INVALID_ARG;
  *alpha_out = alpha_of(n_ref, pfa);
  return RCFAR_OK;
}

rcfar_status rcfar_n_ref(const rcfar_window* w, int32_t* n_ref_out) {
  if (!w || !n_ref_out || w->train_r < 0 || w->train_c < 0 || w->guard_r < 0 || w->guard_c < 0)
    return RCFAR_ERR_INVALID_ARG;
  *n_ref_out = n_ref_of(*w);
  return RCFAR_OK;
}

rcfar_status rcfar_threshold_factor(const rcfar_window* w, double* factor_out, int32_t* cells_out) {
  if (!w || !factor_out || !valid_window(w)) return RCFAR_ERR_INVALID_ARG;
  int cells = 0;
  if (!window_factor(*w, factor_out, &cells)) return RCFAR_ERR_INVALID_ARG;
  if (cells_out) *cells_out = cells;
  return RCFAR_OK;
}

rcfar_status rcfar_band_plan(int32_t N, const rcfar_pre_params* p, rcfar_band* out) {
  if (!out || !band_of(N, p, out)) return RCFAR_ERR_INVALID_ARG;
  return RCFAR_OK;
}

rcfar_status rcfar_sat_scale(float bound, int64_t max_cells, int32_t* scale_log2_out) {
  if (!scale_log2_out || max_cells <= 0 || !(bound >= 0.0f)) return RCFAR_ERR_INVALID_ARG;
  *scale_log2_out = sat_scale_for(bound, max_cells);
  return RCFAR_OK;
}

rcfar_status rcfar_create(const rcfar_config* cfg, rcfar_handle* out) {
  if (!cfg || !out) return RCFAR_ERR_INVALID_ARG;
  if (cfg->max_rows <= 0 || cfg->max_cols <= 0 || cfg->max_n <= 0 || cfg->max_window < 0 ||
      cfg->max_frames < 0 || cfg->batch_bytes < 0)
    return RCFAR_ERR_INVALID_ARG;
  *out = nullptr;
  rcfar_ctx* h = new (std::nothrow) rcfar_ctx();
  if (!h) return RCFAR_ERR_CUDA;
  h->cfg = *cfg;
  h->device = cfg->device;
  if (cudaSetDevice(cfg->device) != cudaSuccess) {
    delete h;
    return RCFAR_ERR_CUDA;
  }
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cfg->device);
  if (optin > 0) h->smem_optin = (size_t)optin;
  int sm_count = 0;
  cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, cfg->device);
  if (sm_count > 0) h->sms = sm_count;

  const int R = cfg->max_rows, Cm = std::max(cfg->max_cols, 1), Nm = cfg->max_n;
  // per-step preprocessing: largest frame is max_rows x max_n with up to N/2+1 bins
  const int max_tiles = (int)(ceil_div(R, kDftBM) * ceil_div(2LL * Cm, kDftMaxBN));
  const size_t kpart = 0;  // K-block partials are allocated on first use
  const int max_strips = (int)ceil_div(Nm, kStatsStrip);
  const int max_chunks = (int)ceil_div(R, kStatsRows);

  size_t total = 0;
  total += 256;                                   // control words
  total += align256((size_t)Nm * sizeof(float2));  // stats
  total += align256((size_t)max_chunks * Nm * sizeof(float4));  // column-statistics partials
  total += align256((size_t)max_strips * R * sizeof(float));
  total += align256((size_t)max_strips * sizeof(float2));
  total += align256((size_t)max_strips * 4);
  total += align256((size_t)max_tiles * 4);
  total += align256(kpart * 4);
  total += align256((size_t)kDftYPlanes * R * round_up(Nm, kDftBK) * sizeof(__half));  // y planes
  const size_t nblocks_max = (size_t)ceil_div(round_up(Nm, kDftBK), kDftBlock);
  total += align256(nblocks_max * R * sizeof(float));                     // yscale
  total += align256((size_t)R * sizeof(float));                          // rowmean
  const size_t ycols_max = (size_t)ceil_div(round_up(Nm, kDftBK), kYCols);
  total += align256(ycols_max * R * sizeof(float));                      // rowsq
  total += align256((size_t)R * round_up(Nm, 4) * sizeof(float));        // xt
  total += sat_bytes(R, Cm, RCFAR_SAT_I64);
  if (cudaMalloc(&h->ws, total) != cudaSuccess) {
    delete h;
    return RCFAR_ERR_CUDA;
  }
  h->ws_bytes = total;
  cudaMemset(h->ws, 0, total);
  Carver cv(h->ws, total);
  unsigned* ctl = cv.take<unsigned>(64);
  h->status = reinterpret_cast<int*>(ctl + 0);
  h->sat_scale = reinterpret_cast<int*>(ctl + 4);
  h->map_bound = reinterpret_cast<float*>(ctl + 5);
  h->ymax = ctl + 6;
  h->stats = cv.take<float2>(Nm);
  h->partial = cv.take<float4>((size_t)max_chunks * Nm);
  h->rowpart = cv.take<float>((size_t)max_strips * R);
  h->strip_ab = cv.take<float2>(max_strips);
  h->strip_cnt = cv.take<unsigned>(max_strips);
  h->tile_cnt = cv.take<unsigned>(max_tiles);
  h->kpart = cv.take<float>(kpart);
  h->kpart_floats = kpart;
  h->yq = cv.take<__half>((size_t)kDftYPlanes * R * round_up(Nm, kDftBK));
  h->yscale = cv.take<float>(nblocks_max * R);
  h->rowmean = cv.take<float>(R);
  h->rowsq = cv.take<float>(ycols_max * R);
  h->xt = cv.take<float>((size_t)R * round_up(Nm, 4));
  {
    SatGeom g = sat_geom(R, Cm);
    h->sat_table = cv.take<char>((size_t)R * g.ld_table * 8);
    carve_sat(cv, R, Cm, &h->sat);
  }
  if (cfg->batch_bytes > 0) {
    if (cudaMalloc(&h->batch, (size_t)cfg->batch_bytes) != cudaSuccess) {
      cudaFree(h->ws);
      delete h;
      return RCFAR_ERR_CUDA;
    }
    h->batch_bytes = (size_t)cfg->batch_bytes;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(h->ws);
    if (h->batch) cudaFree(h->batch);
    delete h;
    return RCFAR_ERR_CUDA;
  }
  *out = h;
  return RCFAR_OK;
}

rcfar_status rcfar_destroy(rcfar_handle h) {
  if (!h) return RCFAR_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaError_t e = cudaDeviceSynchronize();
  for (auto& kv : h->plans) cudaFree(kv.second.Wt);
  if (h->kpart_own) cudaFree(h->kpart_own);
  for (auto& r : h->trace_pool) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  if (h->ws) cudaFree(h->ws);
  if (h->batch) cudaFree(h->batch);
  delete h;
  return cuda_fail(e);
}

rcfar_status rcfar_trace_enable(rcfar_handle h, int32_t on) {
  if (!h) return RCFAR_ERR_INVALID_ARG;
  if (on) h->trace_used = 0;
  h->trace_on = on != 0;
  return RCFAR_OK;
}

rcfar_status rcfar_trace_read(rcfar_handle h, rcfar_trace_entry* out, int32_t max_entries, int32_t* n_out) {
  if (!h || !n_out || (max_entries > 0 && !out) || max_entries < 0) return RCFAR_ERR_INVALID_ARG;
  DeviceGuard dg(h->device);
  std::vector<rcfar_trace_entry> acc;
  for (size_t i = 0; i < h->trace_used; ++i) {
    const rcfar_ctx::TraceRec& r = h->trace_pool[i];
    if (cudaEventSynchronize(r.b) != cudaSuccess) return RCFAR_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return RCFAR_ERR_CUDA;
    size_t j = 0;
    for (; j < acc.size(); ++j)
      if (std::strncmp(acc[j].name, r.name, sizeof(acc[j].name)) == 0) break;
    if (j == acc.size()) {
      rcfar_trace_entry e;
      std::memset(&e, 0, sizeof(e));
      std::strncpy(e.name, r.name, sizeof(e.name) - 1);
      acc.push_back(e);
    }
    acc[j].launches += 1;
    acc[j].total_ms += ms;
  }
  const int n = (int)std::min<size_t>(acc.size(), (size_t)max_entries);
  for (int i = 0; i < n; ++i) out[i] = acc[i];
  *n_out = n;
  return RCFAR_OK;
}

rcfar_status rcfar_get_error(rcfar_handle h, rcfar_stream stream) {
  if (!h) return RCFAR_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RCFAR_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return RCFAR_ERR_CUDA;
  if (st) {
    // clear the status and any counters a broken launch may have left behind
    cudaMemset(h->status, 0, sizeof(int));
    cudaDeviceSynchronize();
  }
  if (st & kStatusTimeout) return RCFAR_ERR_TIMEOUT;
  if (st & kStatusRange) return RCFAR_ERR_RANGE;
  return RCFAR_OK;
}

rcfar_status rcfar_preprocess(rcfar_handle h, const float* x, int32_t M, int32_t N, int64_t ldx,
                              const rcfar_pre_params* p, float* map, int64_t ld_map, rcfar_band* band_out,
                              rcfar_stream stream) {
  if (!h || !x || !map || M <= 0 || N <= 0 || !valid_pre(p) || !ldx_ok(p, M, N, ldx)) return RCFAR_ERR_INVALID_ARG;
  if (p->mean_len > N) return RCFAR_ERR_INVALID_ARG;
  rcfar_band b;
  if (!band_of(N, p, &b)) return RCFAR_ERR_INVALID_ARG;
  if (ld_map < b.cols) return RCFAR_ERR_INVALID_ARG;
  if (M > h->cfg.max_rows || N > h->cfg.max_n || b.cols > h->cfg.max_cols) return RCFAR_ERR_UNSUPPORTED;
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const PreGeom g = pre_geom(M, N, b.cols);
  {
    // K-block partials: grown on demand (outside stream capture)
    const size_t need = (size_t)g.nblocks * M * g.ldk;
    if (need > h->kpart_floats) {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return RCFAR_ERR_BAD_STATE;
      if (h->kpart_own) {
        cudaStreamSynchronize(s);
        cudaFree(h->kpart_own);
        h->kpart_own = nullptr;
        h->kpart_floats = 0;
      }
      if (cudaMalloc(&h->kpart_own, need * sizeof(float)) != cudaSuccess) return RCFAR_ERR_CUDA;
      h->kpart = static_cast<float*>(h->kpart_own);
      h->kpart_floats = need;
    }
  }
  Twiddle tw;
  rcfar_status st = get_plan(h, N, b.c0, b.cols, s, &tw);
  if (st != RCFAR_OK) return st;

  static thread_local PreBatch pb;
  pb.n = 1;
  pb.status = h->status;
  pb.dft_smem = dft_smem_for(g.bn);
  PreFrameDev& F = pb.f[0];
  F = make_pre_frame(x, M, N, ldx, b, p, tw, g);
  F.stats = h->stats;
  F.partial = h->partial;
  F.rowpart = h->rowpart;
  F.strip_ab = h->strip_ab;
  F.strip_cnt = h->strip_cnt;
  F.ymax = h->ymax;
  F.map = map;
  F.ld_map = ld_map;
  F.kpart = h->kpart;
  F.tile_cnt = h->tile_cnt;
  F.yq = h->yq;  // the planes back to back, plane stride M * npad
  F.yscale = h->yscale;
  F.rowmean = h->rowmean;
  F.rowsq = h->rowsq;
  int n_tr = 0;
  if (p->x_layout == RCFAR_X_TRACE_MAJOR) {
    F.xsrc = x;
    F.ldsrc = ldx;
    F.x = h->xt;
    F.ldx = round_up(N, 4);
    n_tr = (int)(ceil_div(M, kTrTile) * ceil_div(N, kTrTile));
    F.n_tr = n_tr;
  }
  F.item_tr = 0;
  F.item_stats = 0;
  F.item_dft = 0;
  F.item_norm = 0;
  F.item_y = 0;
  cudaError_t e = cudaSuccess;
  if (n_tr > 0) {
    TraceScope t(h, "transpose", s);
    e = launch_transpose(pb, n_tr, s);
  }
  if (e == cudaSuccess) {
    TraceScope t(h, "colstats", s);
    e = launch_colstats(pb, g.n_strips * g.n_chunks, s);
  }
  if (e == cudaSuccess) {
    TraceScope t(h, "ysplit", s);
    e = launch_ysplit(pb, g.n_y, s);
  }
  if (e == cudaSuccess) {
    TraceScope t(h, "band_dft", s);
    static thread_local DftBatch db;
    db.n = 1;
    db.dft_smem = pb.dft_smem;
    db.status = h->status;
    if (make_dft_frame(db, 0, F, tw, g))
      e = launch_band_dft_tma(db, g.mtiles * g.ntiles * g.splitk, s);
    else
      e = launch_band_dft(pb, g.mtiles * g.ntiles * g.splitk, s);
  }
  if (e == cudaSuccess) {
    TraceScope t(h, "dft_reduce", s);
    e = launch_dft_reduce(pb, g.n_norm, s);
  }
  if (e != cudaSuccess) return RCFAR_ERR_CUDA;
  if (band_out) *band_out = b;
  return RCFAR_OK;
}

rcfar_status rcfar_sat(rcfar_handle h, const void* map, int32_t dtype, int32_t map_exp2, int32_t rows, int32_t cols,
                       int64_t ld, float value_bound, int32_t mode, rcfar_sat_view* view_out, rcfar_stream stream) {
  if (!h || !map || !view_out || rows <= 0 || cols <= 0 || ld < cols) return RCFAR_ERR_INVALID_ARG;
  if (dtype != RCFAR_MAP_F32 && dtype != RCFAR_MAP_F16) return RCFAR_ERR_INVALID_ARG;
  if (mode < RCFAR_SAT_TILE_F32 || mode > RCFAR_SAT_TILE_I64) return RCFAR_ERR_INVALID_ARG;
  if (value_bound != value_bound) return RCFAR_ERR_INVALID_ARG;
  if (map_exp2 < -100 || map_exp2 > 100) return RCFAR_ERR_INVALID_ARG;
  if (rows > h->cfg.max_rows || cols > h->cfg.max_cols) return RCFAR_ERR_UNSUPPORTED;
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const SatGeom g = sat_geom(rows, cols);
  const float in_scale = dtype == RCFAR_MAP_F16 ? std::ldexp(1.0f, map_exp2) : 1.0f;
  const long long wmax = h->cfg.max_window;
  const long long max_cells = std::max<long long>((long long)kSatTileH * kSatTileW, (2 * wmax + 1) * (2 * wmax + 1));

  static thread_local SatBatch sb;
  sb.n = 1;
  sb.status = h->status;
  SatMapDev& m = sb.m[0];
  std::memset(&m, 0, sizeof(m));
  m.map = map;
  m.ld = ld;
  m.rows = rows;
  m.cols = cols;
  m.in_scale = in_scale;
  m.max_cells = max_cells;
  if (mode == RCFAR_SAT_NAIVE_F32) {
    m.scale_log2 = 0;  // plain FP32: no fixed point; the check only rejects Inf/NaN without a bound
    m.bound = value_bound > 0.0f ? value_bound : 3.4028235e38f;
  } else if (value_bound > 0.0f) {
    m.bound = value_bound;
    m.scale_log2 = sat_scale_for(value_bound, max_cells);
  } else {
    TraceScope t(h, "map_max", s);
    cudaError_t e = launch_map_max(map, dtype, in_scale, rows, cols, ld, h->map_bound, s);
    if (e != cudaSuccess) return RCFAR_ERR_CUDA;
    m.scale_log2 = kScaleFromDevice;
    m.bound_dev = h->map_bound;
  }
  m.table = h->sat_table;
  m.ld_table = g.ld_table;
  set_sat_arrays(m, h->sat);
  m.ld_carry = g.ld_carry;
  m.scale_out = h->sat_scale;
  m.n_bands = g.n_bands;
  m.n_chunks = g.n_chunks;
  m.item_tile = m.item_band = m.item_vscan = 0;
  cudaError_t e;
  {
    TraceScope t(h, "sat", s);
    e = launch_sat(sb, mode, dtype, g.n_bands * g.n_chunks, g.n_bands, (int)ceil_div(cols, 32), s);
  }
  if (e != cudaSuccess) return RCFAR_ERR_CUDA;

  rcfar_sat_view v;
  std::memset(&v, 0, sizeof(v));
  v.rows = rows;
  v.cols = cols;
  v.mode = mode;
  v.tile_h = kSatTileH;
  v.tile_w = kSatTileW;
  v.scale_log2 = (m.scale_log2 == kScaleFromDevice) ? INT32_MIN : m.scale_log2;
  v.table = h->sat_table;
  v.ld = g.ld_table;
  v.row_carry = reinterpret_cast<int64_t*>(h->sat.row_carry);
  v.col_carry = reinterpret_cast<int64_t*>(h->sat.col_carry);
  v.ld_carry = g.ld_carry;
  v.generation = ++h->sat_generation;
  *view_out = v;
  return RCFAR_OK;
}

static rcfar_status check_view(rcfar_handle h, const rcfar_sat_view* v) {
  if (!v) return RCFAR_ERR_INVALID_ARG;
  if (v->generation != h->sat_generation || v->table != h->sat_table) return RCFAR_ERR_BAD_STATE;
  return RCFAR_OK;
}

static void fill_cfar_window(CfarMapDev& P, const rcfar_window* w, int rows, int cols, int cut_c_lo, int cut_c_hi) {
  P.wr = w->guard_r + w->train_r;
  P.wc = w->guard_c + w->train_c;
  P.gr = w->guard_r;
  P.gc = w->guard_c;
  double k = 0.0;
  window_factor(*w, &k, nullptr);  // the window was validated
  P.kthr = (float)k;
  P.kind = w->kind;
  P.n_ref = n_ref_of(*w);
  P.os_rank = w->kind == RCFAR_CFAR_OS ? os_rank_of(*w) : 0;
  P.row_lo = P.wr;
  P.row_hi = rows - 1 - P.wr;
  P.cut_lo = std::max(P.wc, cut_c_lo);
  P.cut_hi = std::min(cols - 1 - P.wc, cut_c_hi);
}

rcfar_status rcfar_cfar(rcfar_handle h, const rcfar_sat_view* view, const void* map, int32_t dtype, int32_t map_exp2,
                        int64_t ld_map, const rcfar_window* w, int32_t cut_c_lo, int32_t cut_c_hi, uint8_t* det,
                        int64_t ld_det, float* thr, int64_t ld_thr, rcfar_stream stream) {
  if (!h || !view || !det || !valid_window(w)) return RCFAR_ERR_INVALID_ARG;
  if (!map && !exact_table(view->mode)) return RCFAR_ERR_INVALID_ARG;
  if (dtype != RCFAR_MAP_F32 && dtype != RCFAR_MAP_F16) return RCFAR_ERR_INVALID_ARG;
  if ((map && ld_map < view->cols) || ld_det < view->cols || (thr && ld_thr < view->cols))
    return RCFAR_ERR_INVALID_ARG;
  rcfar_status st = check_view(h, view);
  if (st != RCFAR_OK) return st;
  if (w->guard_r + w->train_r > h->cfg.max_window || w->guard_c + w->train_c > h->cfg.max_window ||
      w->kind == RCFAR_CFAR_OS)
    return RCFAR_ERR_UNSUPPORTED;
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  static thread_local CfarBatch cb;
  cb.n = 1;
  CfarMapDev& P = cb.m[0];
  std::memset(&P, 0, sizeof(P));
  P.table = view->table;
  P.ld_table = view->ld;
  P.row_carry = reinterpret_cast<const unsigned long long*>(view->row_carry);
  P.col_carry = reinterpret_cast<const unsigned long long*>(view->col_carry);
  P.ld_carry = view->ld_carry;
  P.scale_dev = h->sat_scale;
  P.map = map;
  P.ld_map = ld_map;
  P.in_scale = dtype == RCFAR_MAP_F16 ? std::ldexp(1.0f, map_exp2) : 1.0f;
  P.rows = view->rows;
  P.cols = view->cols;
  fill_cfar_window(P, w, view->rows, view->cols, cut_c_lo, cut_c_hi);
  P.det = det;
  P.ld_det = ld_det;
  P.thr = thr;
  P.ld_thr = ld_thr;
  P.mode = view->mode;
  P.item0 = 0;
  cb.status = h->status;
  const size_t smem_cap = std::min<size_t>(h->smem_optin, 200 * 1024);
  // exact global table: stream its rows through the bulk-copy ring
  int ring_rows = 0, hcp = 0;
  if (view->mode == RCFAR_SAT_I64 && (view->ld % 2) == 0 && (reinterpret_cast<uintptr_t>(view->table) & 15) == 0 &&
      cfar_ring_plan(P.wr, P.wc, h->smem_optin, &ring_rows, &hcp)) {
    const size_t smem = cfar_ring_smem(ring_rows, hcp);
    const int blocks = cfar_ring_geometry(P, view->rows, view->cols, ring_rows, hcp, cfar_ring_slots(smem));
    TraceScope tr(h, "cfar", s);
    return cuda_fail(launch_cfar_ring(cb, map != nullptr, dtype, blocks, smem, s));
  }
  const CfarTile t = pick_cfar_tile(view->mode, P.wr, P.wc, smem_cap, {h->cfg.cfar_tile_rows, h->cfg.cfar_tile_cols});
  if (t.bh == 0) return RCFAR_ERR_UNSUPPORTED;
  const int blocks = set_cfar_geometry(P, t, view->rows, view->cols);
  TraceScope tr(h, "cfar", s);
  cudaError_t e = launch_cfar(cb, view->mode, dtype, blocks, cfar_smem_bytes(view->mode, t.bh, t.bw, P.wr, P.wc),
                              t.bw + 2 * P.wc + 1, s);
  return cuda_fail(e);
}

rcfar_status rcfar_sat_cfar(rcfar_handle h, const void* map, int32_t dtype, int32_t map_exp2, int32_t rows,
                            int32_t cols, int64_t ld_map, float value_bound, const rcfar_window* w, int32_t cut_c_lo,
                            int32_t cut_c_hi, int32_t map_cut, uint8_t* det, int64_t ld_det, float* thr,
                            int64_t ld_thr, rcfar_stream stream) {
  if (!h || !map || !det || rows <= 0 || cols <= 0 || ld_map < cols || ld_det < cols || !valid_window(w))
    return RCFAR_ERR_INVALID_ARG;
  if ((thr && ld_thr < cols) || (dtype != RCFAR_MAP_F32 && dtype != RCFAR_MAP_F16)) return RCFAR_ERR_INVALID_ARG;
  if (!(value_bound > 0.0f) || !std::isfinite(value_bound)) return RCFAR_ERR_INVALID_ARG;
  if (w->guard_r + w->train_r > h->cfg.max_window || w->guard_c + w->train_c > h->cfg.max_window ||
      w->kind == RCFAR_CFAR_OS)
    return RCFAR_ERR_UNSUPPORTED;
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  static thread_local CfarBatch cb;
  cb.n = 1;
  cb.status = h->status;
  CfarMapDev& P = cb.m[0];
  std::memset(&P, 0, sizeof(P));
  P.map = map;
  P.ld_map = ld_map;
  P.in_scale = dtype == RCFAR_MAP_F16 ? std::ldexp(1.0f, map_exp2) : 1.0f;
  P.rows = rows;
  P.cols = cols;
  fill_cfar_window(P, w, rows, cols, cut_c_lo, cut_c_hi);
  P.det = det;
  P.ld_det = ld_det;
  P.thr = thr;
  P.ld_thr = ld_thr;
  // the scale rcfar_sat takes for this bound and handle
  const long long wmax = h->cfg.max_window;
  const long long max_cells = std::max<long long>((long long)kSatTileH * kSatTileW, (2 * wmax + 1) * (2 * wmax + 1));
  P.sat_scale = sat_scale_for(value_bound, max_cells);
  P.bound = value_bound;
  P.item0 = 0;
  const size_t cap = std::min<size_t>(h->smem_optin, 200 * 1024);
  // float32 maps: the streaming kernel; float16 maps (or windows whose ring
  // does not fit): one integral image per block
  StreamPlan sp;
  // wide float32 maps with 16-byte aligned rows: the stages arrive by tensor-memory-accelerator boxes
  if (dtype == RCFAR_MAP_F32 && cfar_stream_tma_plan(rows, cols, P.wr, P.wc, cap, h->sms, &sp)) {
    static thread_local CfarTmaParams tp;
    if (make_map2d(&tp.tm, map, rows, cols, ld_map, 32 * sp.e, kStreamKS)) {
      tp.m = P;
      tp.status = h->status;
      const int blocks = cfar_stream_geometry(tp.m, rows, cols, sp);
      TraceScope tr(h, "sat_cfar_fused_tma", s);
      return cuda_fail(launch_cfar_stream_tma(tp, map_cut != 0, sp.e, blocks, sp.smem, s));
    }
  }
  if (dtype == RCFAR_MAP_F32 && cfar_stream_plan(rows, cols, P.wr, P.wc, cap, h->sms, 0, &sp)) {
    const int blocks = cfar_stream_geometry(P, rows, cols, sp);
    TraceScope tr(h, "sat_cfar_fused", s);
    return cuda_fail(launch_cfar_stream(cb, map_cut != 0, sp.e, blocks, sp.smem, s));
  }
  int run = 0, bw = 0, pitch = 0;
  size_t smem = 0;
  if (!cfar_fused_plan(rows, cols, P.wr, P.wc, cap, &run, &bw, &pitch, &smem)) return RCFAR_ERR_UNSUPPORTED;
  const int blocks = cfar_fused_geometry(P, rows, cols, run, bw, pitch);
  TraceScope tr(h, "sat_cfar_fused", s);
  return cuda_fail(launch_cfar_fused(cb, map_cut != 0, dtype, blocks, smem, s));
}

rcfar_status rcfar_cfar_direct(rcfar_handle h, const float* map, int32_t rows, int32_t cols, int64_t ld_map,
                               const rcfar_window* w, int32_t cut_c_lo, int32_t cut_c_hi, uint8_t* det,
                               int64_t ld_det, float* thr, int64_t ld_thr, rcfar_stream stream) {
  if (!h || !map || !det || rows <= 0 || cols <= 0 || ld_map < cols || ld_det < cols || !valid_window(w))
    return RCFAR_ERR_INVALID_ARG;
  if (thr && ld_thr < cols) return RCFAR_ERR_INVALID_ARG;
  if (w->guard_r + w->train_r > h->cfg.max_window || w->guard_c + w->train_c > h->cfg.max_window)
    return RCFAR_ERR_UNSUPPORTED;
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  CfarMapDev P;
  std::memset(&P, 0, sizeof(P));
  P.map = map;
  P.ld_map = ld_map;
  P.in_scale = 1.0f;
  P.rows = rows;
  P.cols = cols;
  fill_cfar_window(P, w, rows, cols, cut_c_lo, cut_c_hi);
  P.det = det;
  P.ld_det = ld_det;
  P.thr = thr;
  P.ld_thr = ld_thr;
  if (w->kind == RCFAR_CFAR_OS) {
    const size_t smem = cfar_os_smem(P.wr, P.wc, P.n_ref);
    if (P.n_ref > kOsMaxRef || smem > std::min<size_t>(h->smem_optin, 200 * 1024)) return RCFAR_ERR_UNSUPPORTED;
    static thread_local CfarBatch ob;
    ob.n = 1;
    ob.status = h->status;
    ob.m[0] = P;
    ob.m[0].item0 = 0;
    const int blocks = cfar_os_geometry(ob.m[0], rows, cols);
    TraceScope tr(h, "cfar_os", s);
    return cuda_fail(launch_cfar_os(ob, P.n_ref, blocks, smem, s));
  }
  int bh = 32, bw = 64;
  while (cfar_direct_smem_bytes(bh, bw, P.wr, P.wc) > std::min<size_t>(h->smem_optin, 200 * 1024) && bw > 8) {
    if (bw > bh) bw /= 2; else bh /= 2;
  }
  if (cfar_direct_smem_bytes(bh, bw, P.wr, P.wc) > std::min<size_t>(h->smem_optin, 200 * 1024))
    return RCFAR_ERR_UNSUPPORTED;
  P.bh = bh;
  P.bw = bw;
  P.tiles_x = (int)ceil_div(cols, bw);
  const int blocks = P.tiles_x * (int)ceil_div(rows, bh);
  TraceScope tr(h, "cfar_direct", s);
  return cuda_fail(launch_cfar_direct(P, blocks, cfar_direct_smem_bytes(bh, bw, P.wr, P.wc), s));
}

rcfar_status rcfar_sat_materialize(rcfar_handle h, const rcfar_sat_view* view, double* out, int64_t ld_out,
                                   rcfar_stream stream) {
  if (!h || !view || !out || ld_out < view->cols) return RCFAR_ERR_INVALID_ARG;
  rcfar_status st = check_view(h, view);
  if (st != RCFAR_OK) return st;
  DeviceGuard dg(h->device);
  SatMapDev m;
  std::memset(&m, 0, sizeof(m));
  m.rows = view->rows;
  m.cols = view->cols;
  m.table = view->table;
  m.ld_table = view->ld;
  m.row_carry = reinterpret_cast<unsigned long long*>(view->row_carry);
  m.col_carry = reinterpret_cast<unsigned long long*>(view->col_carry);
  m.ld_carry = view->ld_carry;
  m.scale_out = h->sat_scale;
  return cuda_fail(launch_sat_materialize(m, view->mode, out, ld_out, (cudaStream_t)stream));
}

// ---- batched chain -----------------------------------------------------------

rcfar_status rcfar_batch_bytes(int32_t M, int32_t N, const rcfar_pre_params* p, const rcfar_window* w,
                               int64_t* bytes_out) {
  if (!bytes_out || M <= 0 || N <= 0 || !valid_pre(p)) return RCFAR_ERR_INVALID_ARG;
  rcfar_pre_params pf = *p;
  if (pf.halo_c < 0) {
    if (!w || !valid_window(w)) return RCFAR_ERR_INVALID_ARG;
    pf.halo_c = w->guard_c + w->train_c;
  }
  rcfar_band b;
  if (!band_of(N, &pf, &b)) return RCFAR_ERR_INVALID_ARG;
  *bytes_out = (int64_t)(frame_data_bytes(M, N, b.cols, p->x_layout) + frame_ctl_bytes(M, N, b.cols));
  return RCFAR_OK;
}

rcfar_status rcfar_prepare(rcfar_handle h, const rcfar_frame_desc* frames, int32_t n, const rcfar_pre_params* p) {
  if (!h || (!frames && n > 0) || n < 0 || !valid_pre(p)) return RCFAR_ERR_INVALID_ARG;
  DeviceGuard dg(h->device);
  for (int i = 0; i < n; ++i) {
    rcfar_pre_params pf = *p;
    if (pf.halo_c < 0) pf.halo_c = frames[i].window.guard_c + frames[i].window.train_c;
    rcfar_band b;
    if (!band_of(frames[i].N, &pf, &b)) return RCFAR_ERR_INVALID_ARG;
    Twiddle tw;
    rcfar_status st = get_plan(h, frames[i].N, b.c0, b.cols, 0, &tw);
    if (st != RCFAR_OK) return st;
  }
  return cuda_fail(cudaDeviceSynchronize());
}

rcfar_status rcfar_run_batch(rcfar_handle h, const rcfar_frame_desc* frames, int32_t n, const rcfar_pre_params* p,
                             rcfar_stream stream) {
  if (!h || (!frames && n > 0) || n < 0 || !valid_pre(p)) return RCFAR_ERR_INVALID_ARG;
  if (n == 0) return RCFAR_OK;
  if (n > h->cfg.max_frames) return RCFAR_ERR_UNSUPPORTED;
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  // validate and size
  std::vector<rcfar_band> bands(n);
  size_t need_data = 0, need_ctl = 0;
  for (int i = 0; i < n; ++i) {
    const rcfar_frame_desc& f = frames[i];
    if (!f.x || !f.det || f.M <= 0 || f.N <= 0 || !ldx_ok(p, f.M, f.N, f.ldx) || !valid_window(&f.window) ||
        p->mean_len > f.N)
      return RCFAR_ERR_INVALID_ARG;
    rcfar_pre_params pf = *p;
    if (pf.halo_c < 0) pf.halo_c = f.window.guard_c + f.window.train_c;
    if (!band_of(f.N, &pf, &bands[i])) return RCFAR_ERR_INVALID_ARG;
    const int C = bands[i].cols;
    if (f.ld_det < C || (f.thr && f.ld_thr < C) || (f.map && f.ld_map < C)) return RCFAR_ERR_INVALID_ARG;
    if (f.M > h->cfg.max_rows || f.N > h->cfg.max_n ||
        f.window.guard_r + f.window.train_r > h->cfg.max_window ||
        f.window.guard_c + f.window.train_c > h->cfg.max_window)
      return RCFAR_ERR_UNSUPPORTED;
    if (f.window.kind == RCFAR_CFAR_OS &&
        (n_ref_of(f.window) > kOsMaxRef ||
         cfar_os_smem(f.window.guard_r + f.window.train_r, f.window.guard_c + f.window.train_c, n_ref_of(f.window)) >
             std::min<size_t>(h->smem_optin, 200 * 1024)))
      return RCFAR_ERR_UNSUPPORTED;
    need_ctl += frame_ctl_bytes(f.M, f.N, C);
    need_data += frame_data_bytes(f.M, f.N, C, p->x_layout);
  }
  if (need_ctl + need_data > h->batch_bytes) return RCFAR_ERR_OUT_OF_WORKSPACE;
  // plans
  std::vector<Twiddle> tws(n);
  for (int i = 0; i < n; ++i) {
    rcfar_status st = get_plan(h, frames[i].N, bands[i].c0, bands[i].cols, s, &tws[i]);
    if (st != RCFAR_OK) return st;
  }
  Carver ctl(h->batch, need_ctl);
  Carver data((char*)h->batch + need_ctl, h->batch_bytes - need_ctl);
  if (cudaMemsetAsync(h->batch, 0, need_ctl, s) != cudaSuccess) return RCFAR_ERR_CUDA;

  static thread_local PreBatch pb;
  static thread_local SatBatch sb;
  static thread_local CfarBatch cb;
  for (int base = 0; base < n; base += kMaxBatch) {
    const int cnt = std::min(kMaxBatch, n - base);
    // ordered-statistic frames skip the table: their maps go to the OS kernel
    static thread_local CfarBatch ob;
    int n_sat = 0, n_os = 0;
    for (int k = 0; k < cnt; ++k) (frames[base + k].window.kind == RCFAR_CFAR_OS ? n_os : n_sat) += 1;
    pb.n = cnt;
    pb.status = h->status;
    sb.n = n_sat;
    cb.n = n_sat;
    ob.n = n_os;
    cb.status = h->status;
    sb.status = h->status;
    ob.status = h->status;
    int kb_per_cta = 1;
    {
      int bn_max = 16;
      long long units = 0;  // (output tile, K block) pairs of the band DFT over the group
      for (int k = 0; k < cnt; ++k) {
        const PreGeom g0 = pre_geom(frames[base + k].M, frames[base + k].N, bands[base + k].cols);
        bn_max = std::max(bn_max, g0.bn);
        units += (long long)g0.mtiles * g0.ntiles * g0.nblocks;
      }
      pb.dft_smem = dft_smem_for(bn_max);
      kb_per_cta = h->tuning.dft_kblocks_per_cta > 0
                       ? h->tuning.dft_kblocks_per_cta
                       : (int)std::max<long long>(1, units / (2LL * std::max(1, h->sms)));  // about two waves
    }
    // table mode of this group: the streaming CFAR when tuned so and every
    // frame's window fits its ring
    int sat_mode = RCFAR_SAT_TILE_I64;
    int ring_rows_max = 0, hcp_max = 0;
    size_t fused_smem = 0;
    // fused: every frame's streaming plan, each frame planned for its share
    // of the SMs (by rows)
    std::vector<StreamPlan> splans;
    int stream_e = 0;
    if (h->tuning.sat_mode == RCFAR_SAT_FUSED) {
      sat_mode = RCFAR_SAT_FUSED;
      const size_t cap = std::min<size_t>(h->smem_optin, 200 * 1024);
      long long rows_all = 0;
      for (int k = 0; k < cnt; ++k) rows_all += frames[base + k].M;
      splans.resize(cnt);
      // one row-prefix width (e) for the launch: the widest frame's
      for (int k = 0; k < cnt && sat_mode == RCFAR_SAT_FUSED; ++k) {
        const rcfar_frame_desc& f = frames[base + k];
        if (f.window.kind == RCFAR_CFAR_OS) continue;
        const int e = stream_e_of(f.M, bands[base + k].cols, f.window.guard_c + f.window.train_c);
        if (e == 0) sat_mode = RCFAR_SAT_TILE_I64;
        stream_e = std::max(stream_e, e);
      }
      for (int k = 0; k < cnt && sat_mode == RCFAR_SAT_FUSED; ++k) {
        const rcfar_frame_desc& f = frames[base + k];
        if (f.window.kind == RCFAR_CFAR_OS) continue;
        // the frame's share of the SMs by rows, rounded to nearest (the shares add up to about all SMs)
        const long long ra = std::max<long long>(1, rows_all);
        const int share = (int)std::max<long long>(1, ((long long)h->sms * f.M + ra / 2) / ra);
        if (!cfar_stream_plan(f.M, bands[base + k].cols, f.window.guard_r + f.window.train_r,
                              f.window.guard_c + f.window.train_c, cap, share, stream_e, &splans[k]))
          sat_mode = RCFAR_SAT_TILE_I64;
      }
    }
    if (h->tuning.sat_mode == RCFAR_SAT_I64) {
      sat_mode = RCFAR_SAT_I64;
      for (int k = 0; k < cnt && sat_mode == RCFAR_SAT_I64; ++k) {
        const rcfar_window& w = frames[base + k].window;
        if (w.kind == RCFAR_CFAR_OS) continue;
        int rr = 0, hc = 0;
        if (!cfar_ring_plan(w.guard_r + w.train_r, w.guard_c + w.train_c, h->smem_optin, &rr, &hc))
          sat_mode = RCFAR_SAT_TILE_I64;
      }
    }
    size_t ring_smem = 0;
    static thread_local DftBatch db;
    db.n = cnt;
    db.dft_smem = pb.dft_smem;
    db.status = h->status;
    bool dft_tma_ok = h->tuning.dft_operands == 0;
    // column statistics: several 64-row chunks per CTA when the batch has
    // chunks for more than two waves of CTAs at two chunks each (fewer
    // hand-offs between CTAs; the results do not depend on it)
    int stats_cpc = 1;
    {
      long long chunks = 0;
      for (int k = 0; k < cnt; ++k)
        chunks += ceil_div(frames[base + k].N, kStatsStrip) * ceil_div(frames[base + k].M, kStatsRows);
      const long long wave = 4LL * std::max(1, h->sms);
      while (stats_cpc < 4 && chunks / (2 * stats_cpc) >= 2 * wave) stats_cpc *= 2;
    }
    int it_stats = 0, it_dft = 0, it_norm = 0, it_cfar = 0, it_y = 0, it_tr = 0;
    int it_tile = 0, it_band = 0, it_vscan = 0;
    int i_sat = 0, i_os = 0, it_os = 0, os_nref = 0;  // table items, OS items, OS CTAs
    size_t os_smem = 0;
    int cfar_mode_smem = 0, cfar_max_hc = 0;
    for (int k = 0; k < cnt; ++k) {
      const int i = base + k;
      const rcfar_frame_desc& f = frames[i];
      const rcfar_band& b = bands[i];
      const int C = b.cols;
      const PreGeom g = pre_geom(f.M, f.N, C, kb_per_cta);
      PreFrameDev& F = pb.f[k];
      F = make_pre_frame(f.x, f.M, f.N, f.ldx, b, p, tws[i], g);
      F.item_tr = it_tr;
      if (p->x_layout == RCFAR_X_TRACE_MAJOR) {
        F.xsrc = f.x;
        F.ldsrc = f.ldx;
        F.ldx = round_up(f.N, 4);
        F.x = data.take<float>((size_t)f.M * F.ldx);
        if (!F.x) return RCFAR_ERR_OUT_OF_WORKSPACE;
        F.n_tr = (int)(ceil_div(f.M, kTrTile) * ceil_div(f.N, kTrTile));
        it_tr += F.n_tr;
      }
      F.stats = data.take<float2>(f.N);
      F.partial = data.take<float4>((size_t)g.n_chunks * f.N);
      F.rowpart = data.take<float>((size_t)g.n_strips * f.M);
      F.strip_ab = data.take<float2>(g.n_strips);
      F.kpart = data.take<float>((size_t)g.nblocks * f.M * g.ldk);
      F.yq = data.take<__half>((size_t)kDftYPlanes * f.M * g.npad);  // the y planes back to back
      F.yscale = data.take<float>((size_t)g.nblocks * f.M);
      F.rowmean = data.take<float>(f.M);
      F.rowsq = data.take<float>((size_t)g.ycols * f.M);
      float* map = f.map;
      long long ld_map = f.ld_map;
      if (!map) {
        ld_map = round_up(C, 4);
        map = data.take<float>((size_t)f.M * ld_map);
      }
      F.map = map;
      F.ld_map = ld_map;
      F.strip_cnt = ctl.take<unsigned>(g.n_strips);
      F.tile_cnt = ctl.take<unsigned>((size_t)g.mtiles * g.ntiles);
      unsigned* words = ctl.take<unsigned>(64);
      F.ymax = words;
      F.item_stats = it_stats;
      F.item_dft = it_dft;
      dft_tma_ok = dft_tma_ok && F.yq && F.kpart && make_dft_frame(db, k, F, tws[i], g);
      F.item_norm = it_norm;
      F.item_y = it_y;
      it_y += g.n_y;
      F.chunks_per_cta = stats_cpc;
      it_stats += g.n_strips * (int)ceil_div(g.n_chunks, stats_cpc);
      it_dft += g.mtiles * g.ntiles * g.splitk;
      it_norm += g.n_norm;
      if (!F.stats || !F.partial || !F.rowpart || !F.strip_ab || !F.yq || !F.yscale || !F.rowmean ||
          !F.rowsq || !F.kpart || !map || !F.strip_cnt || !F.tile_cnt || !words)
        return RCFAR_ERR_OUT_OF_WORKSPACE;
      if (f.window.kind == RCFAR_CFAR_OS) {
        CfarMapDev& Q = ob.m[i_os++];
        std::memset(&Q, 0, sizeof(Q));
        Q.map = map;
        Q.ld_map = ld_map;
        Q.in_scale = 1.0f;
        Q.rows = f.M;
        Q.cols = C;
        fill_cfar_window(Q, &f.window, f.M, C, b.k_lo - b.c0, b.k_hi - b.c0);
        Q.det = f.det;
        Q.ld_det = f.ld_det;
        Q.thr = f.thr;
        Q.ld_thr = f.ld_thr;
        Q.item0 = it_os;
        it_os += cfar_os_geometry(Q, f.M, C);
        os_smem = std::max(os_smem, cfar_os_smem(Q.wr, Q.wc, Q.n_ref));
        os_nref = std::max(os_nref, Q.n_ref);
        continue;
      }

      const SatGeom sg = sat_geom(f.M, C);
      SatMapDev& m = sb.m[i_sat];
      std::memset(&m, 0, sizeof(m));
      m.map = map;
      m.ld = ld_map;
      m.rows = f.M;
      m.cols = C;
      m.in_scale = 1.0f;
      const long long wr = f.window.guard_r + f.window.train_r, wc = f.window.guard_c + f.window.train_c;
      m.max_cells = std::max<long long>((long long)kSatTileH * kSatTileW, (2 * wr + 1) * (2 * wc + 1));
      m.bound = b.value_bound;
      m.scale_log2 = sat_scale_for(b.value_bound, m.max_cells);
      m.table = data.take<long long>((size_t)f.M * sg.ld_table);
      m.ld_table = sg.ld_table;
      SatArrays sa;
      const bool sat_ok = carve_sat(data, f.M, C, &sa);
      set_sat_arrays(m, sa);
      m.ld_carry = sg.ld_carry;
      m.scale_out = reinterpret_cast<int*>(words + 1);
      m.n_bands = sg.n_bands;
      m.n_chunks = sg.n_chunks;
      m.item_tile = it_tile;
      m.item_band = it_band;
      m.item_vscan = it_vscan;
      it_tile += sg.n_bands * sg.n_chunks;
      it_band += sg.n_bands;
      it_vscan += (int)ceil_div(C, 32);
      if (!F.stats || !F.partial || !F.rowpart || !F.strip_ab || !F.yq || !F.yscale || !F.rowmean || !F.rowsq ||
          !F.kpart || !map || !m.table ||
          !sat_ok || !F.strip_cnt || !F.tile_cnt || !words)
        return RCFAR_ERR_OUT_OF_WORKSPACE;

      CfarMapDev& P = cb.m[i_sat];
      std::memset(&P, 0, sizeof(P));
      P.table = m.table;
      P.ld_table = m.ld_table;
      P.row_carry = m.row_carry;
      P.col_carry = m.col_carry;
      P.ld_carry = m.ld_carry;
      P.scale_dev = m.scale_out;
      P.map = map;
      P.ld_map = ld_map;
      P.in_scale = 1.0f;
      P.rows = f.M;
      P.cols = C;
      fill_cfar_window(P, &f.window, f.M, C, b.k_lo - b.c0, b.k_hi - b.c0);
      P.det = f.det;
      P.ld_det = f.ld_det;
      P.thr = f.thr;
      P.ld_thr = f.ld_thr;
      P.mode = sat_mode;
      P.item0 = it_cfar;
      if (sat_mode == RCFAR_SAT_FUSED) {
        fused_smem = std::max(fused_smem, splans[k].smem);
        P.sat_scale = m.scale_log2;
        P.bound = m.bound;
        it_cfar += cfar_stream_geometry(P, f.M, C, splans[k]);
      } else if (sat_mode == RCFAR_SAT_I64) {
        int rr = 0, hc = 0;
        cfar_ring_plan(P.wr, P.wc, h->smem_optin, &rr, &hc);
        const size_t sm = cfar_ring_smem(rr, hc);
        ring_smem = std::max(ring_smem, sm);
        ring_rows_max = std::max(ring_rows_max, rr);
        hcp_max = std::max(hcp_max, hc);
        it_cfar += cfar_ring_geometry(P, f.M, C, rr, hc, cfar_ring_slots(sm));
      } else {
        // tile from this frame's own window (batch composition does not matter)
        const CfarTile pref = h->tuning.cfar_tile_rows > 0
                                  ? CfarTile{h->tuning.cfar_tile_rows, h->tuning.cfar_tile_cols}
                                  : CfarTile{h->cfg.cfar_tile_rows, h->cfg.cfar_tile_cols};
        const CfarTile t = pick_cfar_tile(sat_mode, P.wr, P.wc, std::min<size_t>(h->smem_optin, 200 * 1024), pref);
        if (t.bh == 0) return RCFAR_ERR_UNSUPPORTED;
        it_cfar += set_cfar_geometry(P, t, f.M, C);
        cfar_mode_smem = std::max<int>(cfar_mode_smem, (int)cfar_smem_bytes(sat_mode, t.bh, t.bw, P.wr, P.wc));
        cfar_max_hc = std::max(cfar_max_hc, t.bw + 2 * P.wc + 1);
      }
      ++i_sat;
    }
    cudaError_t e = cudaSuccess;
    if (it_tr > 0) {
      TraceScope t(h, "transpose", s);
      e = launch_transpose(pb, it_tr, s);
    }
    if (e == cudaSuccess) {
      TraceScope t(h, "colstats", s);
      e = launch_colstats(pb, it_stats, s);
    }
    if (e == cudaSuccess) {
      TraceScope t(h, "ysplit", s);
      e = launch_ysplit(pb, it_y, s);
    }
    if (e == cudaSuccess) {
      TraceScope t(h, "band_dft", s);
      e = dft_tma_ok ? launch_band_dft_tma(db, it_dft, s) : launch_band_dft(pb, it_dft, s);
    }
    if (e == cudaSuccess) {
      TraceScope t(h, "dft_reduce", s);
      e = launch_dft_reduce(pb, it_norm, s);
    }
    if (e == cudaSuccess) {
      TraceScope t(h, "sat", s);
      if (sat_mode != RCFAR_SAT_FUSED) e = launch_sat(sb, sat_mode, RCFAR_MAP_F32, it_tile, it_band, it_vscan, s);
    }
    if (e == cudaSuccess) {
      TraceScope t(h, "cfar", s);
      e = sat_mode == RCFAR_SAT_FUSED ? launch_cfar_stream(cb, true, stream_e, it_cfar, fused_smem, s)
          : sat_mode == RCFAR_SAT_I64
              ? launch_cfar_ring(cb, true, RCFAR_MAP_F32, it_cfar, ring_smem, s)
              : launch_cfar(cb, sat_mode, RCFAR_MAP_F32, it_cfar, (size_t)cfar_mode_smem, cfar_max_hc, s);
    }
    if (e == cudaSuccess && it_os > 0) {
      TraceScope t(h, "cfar_os", s);
      e = launch_cfar_os(ob, os_nref, it_os, os_smem, s);
    }
    if (e != cudaSuccess) return RCFAR_ERR_CUDA;
  }
  return RCFAR_OK;
}

static bool valid_tuning(const rcfar_batch_tuning* t) {
  return t && t->dft_kblocks_per_cta >= 0 && t->dft_kblocks_per_cta <= 4096 &&
         (t->dft_operands == 0 || t->dft_operands == 1) &&
         (t->sat_mode == RCFAR_SAT_TILE_I64 || t->sat_mode == RCFAR_SAT_I64 || t->sat_mode == RCFAR_SAT_FUSED) &&
         ((t->cfar_tile_rows == 0 && t->cfar_tile_cols == 0) ||
          (t->cfar_tile_rows > 0 && t->cfar_tile_rows <= 16 && t->cfar_tile_cols > 0 && 256 % t->cfar_tile_cols == 0 &&
           t->cfar_tile_rows * t->cfar_tile_cols <= 1024));
}

rcfar_status rcfar_set_batch_tuning(rcfar_handle h, const rcfar_batch_tuning* t) {
  if (!h || !valid_tuning(t)) return RCFAR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  h->tuning = *t;
  return RCFAR_OK;
}

rcfar_status rcfar_get_batch_tuning(rcfar_handle h, rcfar_batch_tuning* out) {
  if (!h || !out) return RCFAR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(h->mu);
  *out = h->tuning;
  return RCFAR_OK;
}

// Times one tuning: one untimed batch, then reps batches between two events.
static rcfar_status time_tuning(rcfar_handle h, const rcfar_frame_desc* frames, int n, const rcfar_pre_params* p,
                                int reps, const rcfar_batch_tuning& t, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                                double* ms) {
  {
    std::lock_guard<std::mutex> lk(h->mu);
    h->tuning = t;
  }
  rcfar_status st = rcfar_run_batch(h, frames, n, p, s);
  if (st != RCFAR_OK) return st;
  if (cudaEventRecord(e0, s) != cudaSuccess) return RCFAR_ERR_CUDA;
  for (int r = 0; r < reps && st == RCFAR_OK; ++r) st = rcfar_run_batch(h, frames, n, p, s);
  if (st != RCFAR_OK) return st;
  float el = 0.f;
  if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&el, e0, e1) != cudaSuccess)
    return RCFAR_ERR_CUDA;
  *ms = (double)el / reps;
  return RCFAR_OK;
}

rcfar_status rcfar_tune_batch(rcfar_handle h, const rcfar_frame_desc* frames, int32_t n, const rcfar_pre_params* p,
                              int32_t reps, rcfar_batch_tuning* out, rcfar_stream stream) {
  if (!h || !frames || n <= 0 || reps <= 0 || reps > 100) return RCFAR_ERR_INVALID_ARG;
  DeviceGuard dg(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return RCFAR_ERR_BAD_STATE;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return RCFAR_ERR_CUDA;
  }
  const rcfar_batch_tuning saved = h->tuning;
  rcfar_batch_tuning best = saved;
  best.best_ms = 1e30;
  int timed = 0;
  rcfar_status st = RCFAR_OK;
  auto consider = [&](rcfar_batch_tuning t) {
    if (st != RCFAR_OK) return;
    double ms = 0.0;
    st = time_tuning(h, frames, n, p, reps, t, s, e0, e1, &ms);
    ++timed;
    if (st == RCFAR_OK && ms < best.best_ms) {
      best = t;
      best.best_ms = ms;
    }
  };
  // stage 1: the band-DFT K split, with the default table and CFAR
  const int splits[] = {0, 1, 2, 4, 8, 16};
  for (int kb : splits) consider(rcfar_batch_tuning{kb, RCFAR_SAT_TILE_I64, 0, 0, 0.0, 0, 0});
  // stage 2: table mode and CFAR strips with the best split
  const int kb = best.dft_kblocks_per_cta;
  consider(rcfar_batch_tuning{kb, RCFAR_SAT_I64, 0, 0, 0.0, 0, 0});
  consider(rcfar_batch_tuning{kb, RCFAR_SAT_FUSED, 0, 0, 0.0, 0, 0});
  const int tiles[][2] = {{16, 64}, {8, 64}, {16, 32}, {8, 128}};
  for (const auto& tl : tiles) consider(rcfar_batch_tuning{kb, RCFAR_SAT_TILE_I64, tl[0], tl[1], 0.0, 0, 0});
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  best.candidates = timed;
  {
    std::lock_guard<std::mutex> lk(h->mu);
    h->tuning = st == RCFAR_OK ? best : saved;
  }
  if (st != RCFAR_OK) return st;
  if (out) *out = best;
  return RCFAR_OK;
}

}  // extern "C"
