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

constexpr int kHaloGroups = 8;  // halo rows up to 256 columns wide

__device__ __forceinline__ float ld_map_val(const float* p, float) { return __ldg(p); }
__device__ __forceinline__ float ld_map_val(const __half* p, float scale) { return __half2float(__ldg(p)) * scale; }

template <int MODE, typename InT>
__global__ void __launch_bounds__(256) k_cfar(const __grid_constant__ CfarBatch B) {
  typedef typename std::conditional<MODE == RCFAR_SAT_NAIVE_F32, float, u64>::type SV;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SV* S = reinterpret_cast<SV*>(smem_raw);

  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &CfarMapDev::item0);
  const CfarMapDev& P = B.m[mi];
  const int local = (int)blockIdx.x - P.item0;
  const int ty = local / P.tiles_x, tx = local % P.tiles_x;
  const int bh = P.bh, bw = P.bw;
  const int r0 = ty * bh, c0 = tx * bw;
  const int wr = P.wr, wc = P.wc, gr = P.gr, gc = P.gc;
  const int HR = bh + 2 * wr + 1, HC = bw + 2 * wc + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  int s = 0;
  if constexpr (MODE != RCFAR_SAT_NAIVE_F32) s = __ldcg(P.scale_dev);
  const float scalef = ldexpf(1.0f, s);

  // table over rows r0-wr-1 .. r0+bh+wr-1 and cols c0-wc-1 .. c0+bw+wc-1;
  // each lane issues all of its loads of a halo row before storing any
  // (HC <= 32 * kHaloGroups), so a warp keeps several requests in flight
  for (int hr = warp; hr < HR; hr += 8) {
    const int r = r0 - wr - 1 + hr;
    const bool row_ok = r >= 0 && r < P.rows;
    const int band = r >> 5;  // kSatTileH == 32
    SV vals[kHaloGroups];
#pragma unroll
    for (int u = 0; u < kHaloGroups; ++u) {
      const int hc = lane + 32 * u;
      const int c = c0 - wc - 1 + hc;
      SV val = SV(0);
      if (hc < HC && row_ok && c >= 0 && c < P.cols) {
        if constexpr (MODE == RCFAR_SAT_TILE_F32) {
          const float l = __ldg(reinterpret_cast<const float*>(P.table) + (long long)r * P.ld_table + c);
          u64 q = (u64)__float2ll_rn(l * scalef);
          q += __ldg(P.col_carry + (long long)(c >> 7) * P.rows + r);  // kSatTileW == 128
          if (band > 0) q += __ldg(P.row_carry + (long long)(band - 1) * P.ld_carry + c);
          val = q;
        } else if constexpr (MODE == RCFAR_SAT_I64) {
          val = (u64)__ldg(reinterpret_cast<const long long*>(P.table) + (long long)r * P.ld_table + c);
        } else {
          val = __ldg(reinterpret_cast<const float*>(P.table) + (long long)r * P.ld_table + c);
        }
      }
      vals[u] = val;
    }
#pragma unroll
    for (int u = 0; u < kHaloGroups; ++u) {
      const int hc = lane + 32 * u;
      if (hc < HC) S[hr * HC + hc] = vals[u];
    }
  }
  __syncthreads();

  const float kk = P.kthr * ldexpf(1.0f, -s);
  const InT* map = reinterpret_cast<const InT*>(P.map);
  const int ncell = bh * bw;
  for (int idx = tid; idx < ncell; idx += 256) {
    const int rr = idx / bw, cc = idx - rr * bw;
    const int r = r0 + rr, c = c0 + cc;
    if (r >= P.rows || c >= P.cols) continue;
    unsigned char d = 0;
    float t = 0.f;
    if (r >= P.row_lo && r <= P.row_hi && c >= P.cut_lo && c <= P.cut_hi) {
      // halo coordinates of the lookup rows/cols
      const int ra = rr, rb = rr + 2 * wr + 1, rc = rr + wr - gr, rd = rr + wr + gr + 1;
      const int ca = cc, cb = cc + 2 * wc + 1, cg = cc + wc - gc, cd = cc + wc + gc + 1;
      // eq. 4: A = L1 + L4 - (L2 + L3) for the outer and the guard rectangle
      const SV outer = (S[ra * HC + ca] + S[rb * HC + cb]) - (S[ra * HC + cb] + S[rb * HC + ca]);
      const SV guard = (S[rc * HC + cg] + S[rd * HC + cd]) - (S[rc * HC + cd] + S[rd * HC + cg]);
      const SV ref = outer - guard;
      if constexpr (MODE == RCFAR_SAT_I64) {
        // T = (alpha / n_ref) * S_ref in fixed-point units; the CUT value comes
        // from the map when one is given (one coalesced load instead of four
        // table lookups), else from the exact table (eq. 4 on the 1x1 region)
        const float ts = (float)(long long)ref * P.kthr;
        t = ts * ldexpf(1.0f, -s);
        if (map != nullptr) {
          d = ld_map_val(map + (long long)r * P.ld_map + c, P.in_scale) > t ? 1 : 0;
        } else {
          const int r1 = rr + wr + 1, c1 = cc + wc + 1;
          const u64 qc = (S[r1 * HC + c1] + S[(r1 - 1) * HC + c1 - 1]) - (S[(r1 - 1) * HC + c1] + S[r1 * HC + c1 - 1]);
          d = (float)(long long)qc > ts ? 1 : 0;
        }
      } else {
        if constexpr (MODE == RCFAR_SAT_NAIVE_F32) t = ref * kk;
        else t = (float)(long long)ref * kk;
        const float cut = ld_map_val(map + (long long)r * P.ld_map + c, P.in_scale);
        d = cut > t ? 1 : 0;
      }
    }
    P.det[(long long)r * P.ld_det + c] = d;
    if (P.thr) P.thr[(long long)r * P.ld_thr + c] = t;
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

size_t cfar_smem_bytes(int mode, int bh, int bw, int wr, int wc) {
  const size_t cell = mode == RCFAR_SAT_NAIVE_F32 ? 4 : 8;
  return (size_t)(bh + 2 * wr + 1) * (size_t)(bw + 2 * wc + 1) * cell;
}

size_t cfar_direct_smem_bytes(int bh, int bw, int wr, int wc) {
  return (size_t)(bh + 2 * wr) * (size_t)(bw + 2 * wc) * 4;
}

template <int MODE, typename InT>
static cudaError_t launch_cfar_t(const CfarBatch& b, int blocks, size_t smem, cudaStream_t s) {
  auto fn = k_cfar<MODE, InT>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  fn<<<blocks, 256, smem, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_cfar(const CfarBatch& b, int mode, int dtype, int blocks, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const bool h = dtype == RCFAR_MAP_F16;
  switch (mode) {
    case RCFAR_SAT_TILE_F32:
      return h ? launch_cfar_t<RCFAR_SAT_TILE_F32, __half>(b, blocks, smem, s)
               : launch_cfar_t<RCFAR_SAT_TILE_F32, float>(b, blocks, smem, s);
    case RCFAR_SAT_I64:
      return h ? launch_cfar_t<RCFAR_SAT_I64, __half>(b, blocks, smem, s)
               : launch_cfar_t<RCFAR_SAT_I64, float>(b, blocks, smem, s);
    default:
      return h ? launch_cfar_t<RCFAR_SAT_NAIVE_F32, __half>(b, blocks, smem, s)
               : launch_cfar_t<RCFAR_SAT_NAIVE_F32, float>(b, blocks, smem, s);
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
