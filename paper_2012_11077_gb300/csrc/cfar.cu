// 2D cell-averaging CFAR kernels (paper Sec. II.B, eqs. 1, 2 and 4).
//
// k_cfar        : SAT CFAR. A CTA owns a bh x bw tile of cells; it rebuilds
//                 the table S over the tile plus its halo in shared memory
//                 (exact 64-bit fixed point: tile-local FP32 value quantised
//                 and added to the band and column carries), then for each
//                 interior CUT takes 8 lookups -- eq. 4 on the outer
//                 rectangle minus eq. 4 on the guard rectangle -- in integer
//                 arithmetic, so the reference sum is exact up to the
//                 quantisation of the map; T = (alpha / n_ref) * S_ref and
//                 det = CUT > T.
// k_cfar_direct : the sliding-window CFAR the SAT replaces: the same
//                 decisions with S_ref summed over the n_ref training cells.
#include "rcfar_internal.cuh"

#include <type_traits>

namespace rcfar {

namespace {

typedef unsigned long long u64;

constexpr int kMaxCutRows = 4;  // CUT rows per thread and step: bh * bw <= 256 * kMaxCutRows


__device__ __forceinline__ float ld_map_val(const float* p, float) { return __ldg(p); }
__device__ __forceinline__ float ld_map_val(const __half* p, float scale) { return __half2float(__ldg(p)) * scale; }

// One table value S(r, c) of the region the CFAR reads (0 outside the map).
template <int MODE>
__device__ __forceinline__ typename std::conditional<MODE == RCFAR_SAT_NAIVE_F32, float, u64>::type
table_value(const CfarMapDev& P, int r, int c, float scalef) {
  if constexpr (MODE == RCFAR_SAT_NAIVE_F32) {
    return __ldg(reinterpret_cast<const float*>(P.table) + (long long)r * P.ld_table + c);
  } else if constexpr (MODE == RCFAR_SAT_I64) {
    return (u64)__ldg(reinterpret_cast<const long long*>(P.table) + (long long)r * P.ld_table + c);
  } else {
    u64 q;
    if constexpr (MODE == RCFAR_SAT_TILE_F32)
      q = (u64)__float2ll_rn(__ldg(reinterpret_cast<const float*>(P.table) + (long long)r * P.ld_table + c) * scalef);
    else
      q = (u64)__ldg(reinterpret_cast<const long long*>(P.table) + (long long)r * P.ld_table + c);
    q += __ldg(P.col_carry + (long long)(c >> 7) * P.rows + r);  // kSatTileW == 128
    const int band = r >> 5;                                       // kSatTileH == 32
    if (band > 0) q += __ldg(P.row_carry + (long long)(band - 1) * P.ld_carry + c);
    return q;
  }
}

// SAT CFAR over a strip of bw columns and a run of rows (P.bh CUT rows per
// step, P.run rows per CTA). The table rows the lookups need live in a ring
// of ring_rows (a power of two >= bh + 2 wr + 1) rows of HC = bw + 2 wc + 1
// columns in shared memory; each step needs only bh new rows, which are
// fetched into registers while the previous step computes (HG groups of 32
// columns per halo row, HC <= 32 HG; bh <= 16 so a warp fetches at most two
// rows per step).
template <int MODE, typename InT, int HG>
__global__ void __launch_bounds__(256) k_cfar(const __grid_constant__ CfarBatch B) {
  typedef typename std::conditional<MODE == RCFAR_SAT_NAIVE_F32, float, u64>::type SV;
  constexpr bool kExact = MODE != RCFAR_SAT_TILE_F32 && MODE != RCFAR_SAT_NAIVE_F32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SV* S = reinterpret_cast<SV*>(smem_raw);

  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &CfarMapDev::item0);
  const CfarMapDev& P = B.m[mi];
  const int local = (int)blockIdx.x - P.item0;
  const int tiles_x = P.tiles_x;
  const int ty = local / tiles_x, tx = local - ty * tiles_x;
  const int bh = P.bh, bw = P.bw;
  const int rows = P.rows, cols = P.cols;
  const int rbeg = ty * P.run, rend = min(rows, rbeg + P.run);
  const int c0 = tx * bw;
  const int wr = P.wr, wc = P.wc, gr = P.gr, gc = P.gc;
  const int HC = bw + 2 * wc + 1;
  const int rmask = P.ring_rows - 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  int s = 0;
  if constexpr (MODE != RCFAR_SAT_NAIVE_F32) s = __ldcg(P.scale_dev);
  const float scalef = ldexpf(1.0f, s);

  // halo row g holds table row gbase + g, in ring slot g & rmask
  const int gbase = rbeg - wr - 1;
  auto fetch_row = [&](int g, SV (&v)[HG]) {
    const int r = gbase + g;
#pragma unroll
    for (int u = 0; u < HG; ++u) {
      const int hc = lane + 32 * u;
      const int cx = c0 - wc - 1 + hc;
      v[u] = (hc < HC && r >= 0 && cx >= 0 && cx < cols) ? table_value<MODE>(P, r, cx, scalef) : SV(0);
    }
  };
  auto store_row = [&](int g, const SV (&v)[HG]) {
    SV* dst = S + (g & rmask) * HC;
#pragma unroll
    for (int u = 0; u < HG; ++u) {
      const int hc = lane + 32 * u;
      if (hc < HC) dst[hc] = v[u];
    }
  };

  // initial fill: every row the first step needs
  int loaded = min(rbeg + bh + wr, rows) - gbase;
  for (int g = warp; g < loaded; g += 8) {
    SV v[HG];
    fetch_row(g, v);
    store_row(g, v);
  }
  __syncthreads();

  const int cc = tid % bw;
  const int rstep = 256 / bw;
  const int c = c0 + cc;
  const bool col_ok = c < cols;
  const bool col_cut = col_ok && c >= P.cut_lo && c <= P.cut_hi;
  const int ca = cc, cb = cc + 2 * wc + 1, cg = cc + wc - gc, cd = cc + wc + gc + 1, cm = cc + wc + 1;
  const float kthr = P.kthr;
  const float kk = kthr * ldexpf(1.0f, -s);
  const float inv_s = ldexpf(1.0f, -s);
  const InT* map = reinterpret_cast<const InT*>(P.map);
  const int row_lo = P.row_lo, row_hi = P.row_hi;

  for (int R = rbeg; R < rend; R += bh) {
    // fetch the rows the next step adds (at most two per warp)
    const int need = (R + bh < rend) ? min(R + 2 * bh + wr, rows) - gbase : loaded;
    SV nxt[2][HG];
    const int g0 = loaded + warp, g1 = loaded + warp + 8;
    if (g0 < need) fetch_row(g0, nxt[0]);
    if (g1 < need) fetch_row(g1, nxt[1]);
    // this step's CUT values from the map (when reading them from it)
    float cutv[kMaxCutRows];
#pragma unroll
    for (int i = 0; i < kMaxCutRows; ++i) {
      const int r = R + tid / bw + i * rstep;
      cutv[i] = 0.f;
      if (map != nullptr && i * rstep < bh && col_cut && r < rend && r >= row_lo && r <= row_hi)
        cutv[i] = ld_map_val(map + (long long)r * P.ld_map + c, P.in_scale);
    }

#pragma unroll
    for (int i = 0; i < kMaxCutRows; ++i) {
      const int rr = tid / bw + i * rstep;
      if (rr >= bh) break;
      const int r = R + rr;
      if (r >= rend || !col_ok) continue;
      unsigned char d = 0;
      float t = 0.f;
      if (col_cut && r >= row_lo && r <= row_hi) {
        const int g = r - gbase;
        const SV* Sa = S + ((g - wr - 1) & rmask) * HC;   // row r - wr - 1
        const SV* Sb = S + ((g + wr) & rmask) * HC;       // row r + wr
        const SV* Sc = S + ((g - gr - 1) & rmask) * HC;   // row r - gr - 1
        const SV* Sd = S + ((g + gr) & rmask) * HC;       // row r + gr
        // eq. 4: A = L1 + L4 - (L2 + L3) for the outer and the guard rectangle
        const SV outer = (Sa[ca] + Sb[cb]) - (Sa[cb] + Sb[ca]);
        const SV guard = (Sc[cg] + Sd[cd]) - (Sc[cd] + Sd[cg]);
        const SV ref = outer - guard;
        if constexpr (kExact) {
          // T = (alpha / n_ref) * S_ref in fixed-point units; the CUT value
          // comes from the map when one is given, else from the exact table
          // (eq. 4 on the 1x1 region)
          const float ts = (float)(long long)ref * kthr;
          t = ts * inv_s;
          if (map != nullptr) {
            d = cutv[i] > t ? 1 : 0;
          } else {
            const SV* S1 = S + (g & rmask) * HC;        // row r
            const SV* S0 = S + ((g - 1) & rmask) * HC;  // row r - 1
            const u64 qc = (S1[cm] + S0[cm - 1]) - (S0[cm] + S1[cm - 1]);
            d = (float)(long long)qc > ts ? 1 : 0;
          }
        } else {
          if constexpr (MODE == RCFAR_SAT_NAIVE_F32) t = ref * kk;
          else t = (float)(long long)ref * kk;
          d = cutv[i] > t ? 1 : 0;
        }
      }
      P.det[(long long)r * P.ld_det + c] = d;
      if (P.thr) P.thr[(long long)r * P.ld_thr + c] = t;
    }
    __syncthreads();  // the rows stored next overwrite ring slots read above
    if (g0 < need) store_row(g0, nxt[0]);
    if (g1 < need) store_row(g1, nxt[1]);
    loaded = need;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_cfar_direct(const __grid_constant__ CfarMapDev P) {
  extern __shared__ __align__(16) float X[];
  const int local = (int)blockIdx.x;
  const int ty = local / P.tiles_x, tx = local % P.tiles_x;
  const int bh = P.bh, bw = P.bw;
  const int r0 = ty * bh, c0 = tx * bw;
  const int wr = P.wr, wc = P.wc, gr = P.gr, gc = P.gc;
  const int HR = bh + 2 * wr, HC = bw + 2 * wc;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* map = reinterpret_cast<const float*>(P.map);
  for (int hr = warp; hr < HR; hr += 8) {
    const int r = r0 - wr + hr;
    for (int hc = lane; hc < HC; hc += 32) {
      const int c = c0 - wc + hc;
      X[hr * HC + hc] = (r >= 0 && r < P.rows && c >= 0 && c < P.cols) ? __ldg(map + (long long)r * P.ld_map + c) : 0.f;
    }
  }
  __syncthreads();
  const int ncell = bh * bw;
  for (int idx = tid; idx < ncell; idx += 256) {
    const int rr = idx / bw, cc = idx - rr * bw;
    const int r = r0 + rr, c = c0 + cc;
    if (r >= P.rows || c >= P.cols) continue;
    unsigned char d = 0;
    float t = 0.f;
    if (r >= P.row_lo && r <= P.row_hi && c >= P.cut_lo && c <= P.cut_hi) {
      float sum = 0.f;
      for (int dr = -wr; dr <= wr; ++dr) {
        const float* row = X + (rr + wr + dr) * HC + cc + wc;
        float rs = 0.f;
        if (dr >= -gr && dr <= gr) {
          for (int dc = -wc; dc < -gc; ++dc) rs += row[dc];
          for (int dc = gc + 1; dc <= wc; ++dc) rs += row[dc];
        } else {
          for (int dc = -wc; dc <= wc; ++dc) rs += row[dc];
        }
        sum += rs;
      }
      t = sum * P.kthr;
      d = X[(rr + wr) * HC + cc + wc] > t ? 1 : 0;
    }
    P.det[(long long)r * P.ld_det + c] = d;
    if (P.thr) P.thr[(long long)r * P.ld_thr + c] = t;
  }
}

}  // namespace

int cfar_ring_rows(int bh, int wr) {
  int n = 1;
  while (n < bh + 2 * wr + 1) n <<= 1;
  return n;
}

size_t cfar_smem_bytes(int mode, int bh, int bw, int wr, int wc) {
  const size_t cell = mode == RCFAR_SAT_NAIVE_F32 ? 4 : 8;
  return (size_t)cfar_ring_rows(bh, wr) * (size_t)(bw + 2 * wc + 1) * cell;
}

size_t cfar_direct_smem_bytes(int bh, int bw, int wr, int wc) {
  return (size_t)(bh + 2 * wr) * (size_t)(bw + 2 * wc) * 4;
}

template <int MODE, typename InT>
static cudaError_t launch_cfar_t(const CfarBatch& b, int blocks, size_t smem, int max_hc, cudaStream_t s) {
  auto fn = max_hc <= 128 ? k_cfar<MODE, InT, 4> : k_cfar<MODE, InT, 8>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  fn<<<blocks, 256, smem, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_cfar(const CfarBatch& b, int mode, int dtype, int blocks, size_t smem, int max_hc, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const bool h = dtype == RCFAR_MAP_F16;
  switch (mode) {
    case RCFAR_SAT_TILE_F32:
      return h ? launch_cfar_t<RCFAR_SAT_TILE_F32, __half>(b, blocks, smem, max_hc, s)
               : launch_cfar_t<RCFAR_SAT_TILE_F32, float>(b, blocks, smem, max_hc, s);
    case RCFAR_SAT_I64:
      return h ? launch_cfar_t<RCFAR_SAT_I64, __half>(b, blocks, smem, max_hc, s)
               : launch_cfar_t<RCFAR_SAT_I64, float>(b, blocks, smem, max_hc, s);
    case RCFAR_SAT_TILE_I64:
      return h ? launch_cfar_t<RCFAR_SAT_TILE_I64, __half>(b, blocks, smem, max_hc, s)
               : launch_cfar_t<RCFAR_SAT_TILE_I64, float>(b, blocks, smem, max_hc, s);
    default:
      return h ? launch_cfar_t<RCFAR_SAT_NAIVE_F32, __half>(b, blocks, smem, max_hc, s)
               : launch_cfar_t<RCFAR_SAT_NAIVE_F32, float>(b, blocks, smem, max_hc, s);
  }
}

cudaError_t launch_cfar_direct(const CfarMapDev& m, int blocks, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(&k_cfar_direct), smem);
  if (e != cudaSuccess) return e;
  k_cfar_direct<<<blocks, 256, smem, s>>>(m);
  return cudaGetLastError();
}

}  // namespace rcfar
