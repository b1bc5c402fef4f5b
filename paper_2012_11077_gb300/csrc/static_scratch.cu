// rcfar_sat_cfar_static: the summed-area table and the SAT CA-CFAR of one map
// with no device allocation at all.
//
// Some callers cannot call cudaMalloc (or any allocating routine): real-time
// radar loops whose device memory was fixed at start-up and must not touch
// the allocator (an allocation can synchronise the device and stall the
// loop), and hosts whose device memory is owned by another memory manager
// (a framework's caching pool, an embedded runtime) that the library must
// not bypass. They cannot create a handle, because rcfar_create allocates
// its workspace.
//
// This entry point takes no handle. Its scratch -- the exact 64-bit
// tile-local table, the tile row/column totals and the carries of the table
// -- lives in one file-scope __device__ array of kStaticScratchBytes (16 MiB),
// which every GPU that loads the library holds until the process exits. The
// caller passes the map and the outputs; the kernels are the ones the handle
// path runs (k_sat_tile, k_sat_hscan, k_sat_vscan, k_cfar in TILE_I64 mode).
//
// Host code never dereferences g_static_scratch: in host code the name is a
// stand-in, not a device address. On the first call on each device (that
// device current) the entry point asks the runtime for the array's device
// address with cudaGetSymbolAddress and keeps it; that first call must come
// before any stream capture. Later calls do no set-up.
//
// No device memory is allocated, ever. (On the host, the first call on a
// device records the kernel's shared-memory limit in a small table.)
//
// All calls share the one array, and it keeps the last call's contents:
// every call rewrites all the scratch it reads, so nothing needs clearing,
// but calls whose work overlaps on the GPU (different streams, or several
// host threads) race on the array and must be serialised by the caller.
#include "rcfar_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;  // 16 MiB
constexpr int kMaxDevices = 64;
constexpr long long kMaxStaticHalfRows = 1024;  // guard_r + train_r
constexpr long long kMaxStaticHalfCols = 119;   // guard_c + train_c: 16 + 2 * 119 + 1 <= 256

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }
inline long long rup(long long a, long long b) { return cdiv(a, b) * b; }
inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device (set up once).
rcfar_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RCFAR_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return RCFAR_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return RCFAR_OK;
}

}  // namespace

extern "C" rcfar_status rcfar_sat_cfar_static(const float* map, int32_t rows, int32_t cols, int64_t ld_map,
                                               float value_bound, const rcfar_window* w, int32_t cut_c_lo,
                                               int32_t cut_c_hi, uint8_t* det, int64_t ld_det, float* thr,
                                               int64_t ld_thr, int32_t* status, rcfar_stream stream) {
  using namespace rcfar;
  if (!map || !det || !w || rows <= 0 || cols <= 0 || ld_map < cols || ld_det < cols) return RCFAR_ERR_INVALID_ARG;
  if (thr && ld_thr < cols) return RCFAR_ERR_INVALID_ARG;
  if (!(value_bound > 0.0f) || !std::isfinite(value_bound)) return RCFAR_ERR_INVALID_ARG;
  if (w->train_r < 0 || w->train_c < 0 || w->guard_r < 0 || w->guard_c < 0 || !(w->pfa > 0.0 && w->pfa < 1.0))
    return RCFAR_ERR_INVALID_ARG;
  // half-widths in 64 bits: guard + train of two large int32 counts overflows int;
  // beyond these limits the CFAR's ring of table rows (kMaxStaticHalfRows) or its
  // 256-column strip (kMaxStaticHalfCols) cannot hold the window
  const long long wr64 = (long long)w->guard_r + w->train_r, wc64 = (long long)w->guard_c + w->train_c;
  if (wr64 > kMaxStaticHalfRows || wc64 > kMaxStaticHalfCols) return RCFAR_ERR_UNSUPPORTED;
  const int wr = (int)wr64, wc = (int)wc64;
  const long long n_ref = (2LL * wr + 1) * (2LL * wc + 1) - (2LL * w->guard_r + 1) * (2LL * w->guard_c + 1);
  double kfac = 0.0;
  if (n_ref <= 0 || !window_factor(*w, &kfac, nullptr)) return RCFAR_ERR_INVALID_ARG;
  if (w->kind == RCFAR_CFAR_OS) return RCFAR_ERR_UNSUPPORTED;  // an order statistic is not a region sum

  // scratch layout: control words | table int64 | col_tot | row_carry | row_tot | col_carry
  const int n_bands = (int)cdiv(rows, kSatTileH), n_chunks = (int)cdiv(cols, kSatTileW);
  const long long ld_table = rup(cols, 4), ld_carry = (long long)n_chunks * kSatTileW;
  const size_t b_ctl = 256;
  const size_t b_table = a256((size_t)rows * ld_table * 8);
  const size_t b_vc = a256((size_t)n_bands * ld_carry * 8);
  const size_t b_rt = a256((size_t)n_bands * n_chunks * kSatTileH * 8);
  const size_t b_cc = a256((size_t)n_chunks * rows * 8);
  if (b_ctl + b_table + 2 * b_vc + b_rt + b_cc > kStaticScratchBytes) return RCFAR_ERR_UNSUPPORTED;

  // CFAR strip geometry that fits this window in shared memory
  int optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem_cap = std::min<size_t>(optin > 0 ? (size_t)optin : 48 * 1024, 200 * 1024);
  int bh = 0, bw = 0;
  const int cand[][2] = {{16, 64}, {16, 32}, {8, 64}, {8, 32}, {8, 16}, {4, 16}};
  for (const auto& c : cand) {
    if (cfar_smem_bytes(RCFAR_SAT_TILE_I64, c[0], c[1], wr, wc) <= smem_cap && c[1] + 2 * wc + 1 <= 256) {
      bh = c[0];
      bw = c[1];
      break;
    }
  }
  if (bh == 0) return RCFAR_ERR_UNSUPPORTED;

  void* base = nullptr;
  rcfar_status st = scratch_address(&base);
  if (st != RCFAR_OK) return st;
  char* p = static_cast<char*>(base);
  int* scale_slot = reinterpret_cast<int*>(p);
  long long* table = reinterpret_cast<long long*>(p + b_ctl);
  unsigned long long* col_tot = reinterpret_cast<unsigned long long*>(p + b_ctl + b_table);
  unsigned long long* row_carry = reinterpret_cast<unsigned long long*>(p + b_ctl + b_table + b_vc);
  unsigned long long* row_tot = reinterpret_cast<unsigned long long*>(p + b_ctl + b_table + 2 * b_vc);
  unsigned long long* col_carry = reinterpret_cast<unsigned long long*>(p + b_ctl + b_table + 2 * b_vc + b_rt);

  cudaStream_t s = (cudaStream_t)stream;
  // the status word the kernels OR into must start at zero (caller memory)
  int* status_word = status ? reinterpret_cast<int*>(status) : reinterpret_cast<int*>(p + 64);
  if (cudaMemsetAsync(status_word, 0, sizeof(int), s) != cudaSuccess) return RCFAR_ERR_CUDA;

  const long long box = (2LL * wr + 1) * (2LL * wc + 1);
  const long long max_cells = std::max<long long>((long long)kSatTileH * kSatTileW, box);

  SatBatch sb;  // kernel parameters, on the host stack
  sb.n = 1;
  sb.status = status_word;
  SatMapDev& m = sb.m[0];
  std::memset(&m, 0, sizeof(m));
  m.map = map;
  m.ld = ld_map;
  m.rows = rows;
  m.cols = cols;
  m.in_scale = 1.0f;
  m.bound = value_bound;
  m.scale_log2 = sat_scale_for(value_bound, max_cells);
  m.max_cells = max_cells;
  m.table = table;
  m.ld_table = ld_table;
  m.col_tot = col_tot;
  m.row_tot = row_tot;
  m.row_carry = row_carry;
  m.col_carry = col_carry;
  m.ld_carry = ld_carry;
  m.scale_out = scale_slot;
  m.n_bands = n_bands;
  m.n_chunks = n_chunks;
  cudaError_t e = launch_sat(sb, RCFAR_SAT_TILE_I64, RCFAR_MAP_F32, n_bands * n_chunks, n_bands,
                             (int)cdiv(cols, 32), s);
  if (e != cudaSuccess) return RCFAR_ERR_CUDA;

  CfarBatch cb;
  cb.n = 1;
  cb.status = status_word;
  CfarMapDev& P = cb.m[0];
  std::memset(&P, 0, sizeof(P));
  P.table = table;
  P.ld_table = ld_table;
  P.row_carry = row_carry;
  P.col_carry = col_carry;
  P.ld_carry = ld_carry;
  P.scale_dev = scale_slot;
  P.map = map;
  P.ld_map = ld_map;
  P.in_scale = 1.0f;
  P.rows = rows;
  P.cols = cols;
  P.wr = wr;
  P.wc = wc;
  P.gr = w->guard_r;
  P.gc = w->guard_c;
  P.kthr = (float)kfac;
  P.kind = w->kind;
  P.row_lo = wr;
  P.row_hi = rows - 1 - wr;
  P.cut_lo = std::max(wc, cut_c_lo);
  P.cut_hi = std::min(cols - 1 - wc, cut_c_hi);
  P.det = det;
  P.ld_det = ld_det;
  P.thr = thr;
  P.ld_thr = ld_thr;
  P.mode = RCFAR_SAT_TILE_I64;
  P.bh = bh;
  P.bw = bw;
  P.run = (int)rup(std::min<long long>(256, rup(rows, bh)), bh);
  P.ring_rows = cfar_ring_rows(bh, wr);
  P.tiles_x = (int)cdiv(cols, bw);
  const int blocks = P.tiles_x * (int)cdiv(rows, P.run);
  e = launch_cfar(cb, RCFAR_SAT_TILE_I64, RCFAR_MAP_F32, blocks, cfar_smem_bytes(RCFAR_SAT_TILE_I64, bh, bw, wr, wc),
                  bw + 2 * wc + 1, s);
  return e == cudaSuccess ? RCFAR_OK : RCFAR_ERR_CUDA;
}
