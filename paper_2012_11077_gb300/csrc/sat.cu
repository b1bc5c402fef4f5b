// Summed-area table of a CFAR input map (paper eq. 3).
//
// The map is cut into tiles of kSatTileH x kSatTileW cells (band b = tile
// row, chunk j = tile column). For cell (r, c) of tile (b, j):
//   S(r, c) = L(r, c) + CC_j(r) + RC_{b-1}(c)
//   L      : table of the tile relative to its own origin (tile-local)
//   CC_j(r): sum over the band's rows <= r and the columns left of the tile
//   RC_b(c): S(last row of band b, c)
// Wait-free passes (no CTA waits for another):
//   k_sat_tile  : (TILE_I64, TILE_F32, NAIVE_F32) one CTA per tile; writes L
//                 and the tile's exact row and column totals (warp-shuffle
//                 row scans, shared-memory column scans across the 8 warps);
//   k_sat_reduce: (I64) the tile totals only, without writing L;
//   k_sat_hscan : one CTA per band; the band's row prefix of the column
//                 totals across the whole width, and CC for every tile;
//   k_sat_vscan : each column's prefix over bands -> RC;
//   k_sat_down  : (I64) the tile prefix plus the carries, written as S;
//   k_sat_finalize (NAIVE_F32) folds the carries into L.
// Carries are 64-bit fixed point q = round(x * 2^s) added modulo 2^64
// (exact; every region sum below 2^63 comes out exact even if S wraps).
#include "rcfar_internal.cuh"
#include "async_copy.cuh"
#include "fixed_point.cuh"

#include <type_traits>

namespace rcfar {

namespace {

typedef unsigned long long u64;

__device__ __forceinline__ float ld_val(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld_val(const __half* p) { return __half2float(__ldg(p)); }

template <typename InT>
__device__ __forceinline__ void load_row4(const InT* row, int c, int cols, bool vec, float scale, float v[4]) {
  if constexpr (std::is_same<InT, float>::value) {
    if (vec && c + 3 < cols) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(row + c));
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      return;
    }
  } else {
    if (vec && c + 3 < cols) {
      const uint2 t = __ldg(reinterpret_cast<const uint2*>(row + c));
      const __half2 h0 = *reinterpret_cast<const __half2*>(&t.x);
      const __half2 h1 = *reinterpret_cast<const __half2*>(&t.y);
      const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
      v[0] = f0.x * scale; v[1] = f0.y * scale; v[2] = f1.x * scale; v[3] = f1.y * scale;
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) v[k] = (c + k < cols) ? ld_val(row + c + k) * scale : 0.0f;
}

template <typename T>
__device__ __forceinline__ T warp_excl_scan(T x, int lane) {
  T incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  return incl - x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// 2D inclusive prefix of a 32 x 128 tile held as x[4][4] per thread
// (warp w: rows 4w..4w+3, lane l: columns 4l..4l+3). wt: 8 x 128 scratch.
template <typename T>
__device__ __forceinline__ void tile_prefix(T x[4][4], T (*wt)[kSatTileW], int w, int lane) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int k = 1; k < 4; ++k) x[i][k] += x[i][k - 1];
    const T e = warp_excl_scan(x[i][3], lane);
#pragma unroll
    for (int k = 0; k < 4; ++k) x[i][k] += e;
  }
#pragma unroll
  for (int i = 1; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) x[i][k] += x[i - 1][k];
#pragma unroll
  for (int k = 0; k < 4; ++k) wt[w][lane * 4 + k] = x[3][k];
  __syncthreads();
  T e[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) e[k] = T(0);
  for (int ww = 0; ww < w; ++ww)
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] += wt[ww][lane * 4 + k];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) x[i][k] += e[k];
}

template <typename Acc>
__device__ __forceinline__ Acc ld_carry(const u64* p) {
  const u64 v = __ldcg(p);
  if constexpr (std::is_same<Acc, float>::value) return __uint_as_float((unsigned)v);
  else return v;
}
template <typename Acc>
__device__ __forceinline__ void st_carry(u64* p, Acc v) {
  if constexpr (std::is_same<Acc, float>::value) __stcg(p, (u64)__float_as_uint(v));
  else __stcg(p, v);
}

template <int MODE>
struct SatTypes {
  // Acc: carry arithmetic (exact fixed point, or FP32 for the naive table)
  typedef typename std::conditional<MODE == RCFAR_SAT_NAIVE_F32, float, u64>::type Acc;
  // Loc: tile-local table arithmetic
  typedef typename std::conditional<MODE == RCFAR_SAT_TILE_I64 || MODE == RCFAR_SAT_I64, u64, float>::type Loc;
};

// Pass 1: one CTA per tile (warp w: rows 4w..4w+3, lane: columns 4l..4l+3).
template <int MODE, typename InT>
__global__ void __launch_bounds__(256) k_sat_tile(const __grid_constant__ SatBatch B) {
  pdl_trigger();
  pdl_wait();
  typedef typename SatTypes<MODE>::Acc Acc;
  typedef typename SatTypes<MODE>::Loc Loc;
  __shared__ Loc s_wt[8][kSatTileW];
  __shared__ Acc s_wc[8][kSatTileW];

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &SatMapDev::item_tile);
  const SatMapDev& Mp = B.m[mi];
  const int tile = (int)blockIdx.x - Mp.item_tile;
  const int nch = Mp.n_chunks;
  const int b = tile / nch, j = tile - b * nch;
  const int r0 = b * kSatTileH;
  const int cbase = j * kSatTileW + lane * 4;
  const int rows = Mp.rows, cols = Mp.cols;
  const InT* map = reinterpret_cast<const InT*>(Mp.map);
  const bool vec = ((Mp.ld & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(map) & (std::is_same<InT, float>::value ? 15 : 7)) == 0);

  int s = Mp.scale_log2;
  float bound = Mp.bound;
  if (s == kScaleFromDevice) {
    bound = __ldcg(Mp.bound_dev);
    s = sat_scale_for(bound, Mp.max_cells);
  }
  if (tile == 0 && tid == 0 && Mp.scale_out) *Mp.scale_out = s;
  const float scalef = ldexpf(1.0f, s);

  float v[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + w * 4 + i;
    if (r < rows) {
      load_row4<InT>(map + (long long)r * Mp.ld, cbase, cols, vec, Mp.in_scale, v[i]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[i][k] = 0.f;
    }
  }
  bool bad = false;
  Acc q[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bad |= !(fabsf(v[i][k]) <= bound);  // NaN fails too
      if constexpr (std::is_same<Acc, float>::value) q[i][k] = v[i][k];
      else q[i][k] = (u64)q_from_f32(v[i][k], scalef);
    }

  // exact row totals -> row_tot[tile][row]
  u64* rt = Mp.row_tot + (long long)tile * kSatTileH;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const Acc t = warp_sum<Acc>(q[i][0] + q[i][1] + q[i][2] + q[i][3]);
    if (lane == i) st_carry<Acc>(rt + w * 4 + i, t);
  }

  Loc L[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (std::is_same<Loc, float>::value) L[i][k] = v[i][k];
      else L[i][k] = q[i][k];
    }
  constexpr bool kExactL = std::is_same<Loc, u64>::value;
  // 4-row column sums of q (before the prefix), when L is not exact
  if constexpr (!kExactL) {
#pragma unroll
    for (int k = 0; k < 4; ++k) s_wc[w][lane * 4 + k] = q[0][k] + q[1][k] + q[2][k] + q[3][k];
  }
  tile_prefix<Loc>(L, s_wt, w, lane);  // contains a __syncthreads

  // column totals -> col_tot[b][c]
  if constexpr (kExactL) {
    // exact L: its last row (warp 7, row 3) is the tile's column prefix, so
    // the column totals are its differences along the row
    if (w == 7) {
      Acc prev = __shfl_up_sync(0xffffffffu, L[3][3], 1);
      if (lane == 0) prev = Acc(0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const Acc t = L[3][k] - prev;
        prev = L[3][k];
        if (cbase + k < cols) st_carry<Acc>(Mp.col_tot + (long long)b * Mp.ld_carry + cbase + k, t);
      }
    }
  } else {
    if (w == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Acc sum = s_wc[0][lane * 4 + k];
#pragma unroll
        for (int ww = 1; ww < 8; ++ww) sum += s_wc[ww][lane * 4 + k];
        if (cbase + k < cols) st_carry<Acc>(Mp.col_tot + (long long)b * Mp.ld_carry + cbase + k, sum);
      }
    }
  }

  // the tile-local table
  if constexpr (std::is_same<Loc, float>::value) {
    float* out = reinterpret_cast<float*>(Mp.table);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + w * 4 + i;
      if (r >= rows) continue;
      float* o = out + (long long)r * Mp.ld_table + cbase;
      if (cbase + 3 < cols) {
        *reinterpret_cast<float4*>(o) = make_float4(L[i][0], L[i][1], L[i][2], L[i][3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cbase + k < cols) o[k] = L[i][k];
      }
    }
  } else {
    long long* out = reinterpret_cast<long long*>(Mp.table);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + w * 4 + i;
      if (r >= rows) continue;
      long long* o = out + (long long)r * Mp.ld_table + cbase;
      if (cbase + 3 < cols) {
        reinterpret_cast<longlong2*>(o)[0] = make_longlong2((long long)L[i][0], (long long)L[i][1]);
        reinterpret_cast<longlong2*>(o)[1] = make_longlong2((long long)L[i][2], (long long)L[i][3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cbase + k < cols) o[k] = (long long)L[i][k];
      }
    }
  }
  if (bad) atomicOr(B.status, kStatusRange);
}

// ---- exact global table (I64): reduce, carry scans, downsweep --------------
// The I64 table stores S itself (eq. 3, 64-bit fixed point), so a reader
// needs no carries. It is built in three wait-free steps: k_sat_reduce reads
// the map once for the tiles' exact row and column totals, the two carry
// scans run on those totals, and k_sat_down reads the map again, forms each
// tile's local prefix and adds the carries as it writes S.

// Totals of four per-lane values across the warp: the total of p[i] ends in
// lanes 8i .. 8i+7. Halving exchanges: 6 64-bit shuffles instead of 20.
__device__ __forceinline__ u64 warp_sum4(const u64 p[4], int lane) {
  const bool h16 = (lane & 16) != 0;
  u64 k0 = h16 ? p[2] : p[0], k1 = h16 ? p[3] : p[1];
  const u64 s0 = h16 ? p[0] : p[2], s1 = h16 ? p[1] : p[3];
  k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
  k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
  const bool h8 = (lane & 8) != 0;
  u64 k = h8 ? k1 : k0;
  k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  k += __shfl_xor_sync(0xffffffffu, k, 4);
  k += __shfl_xor_sync(0xffffffffu, k, 2);
  k += __shfl_xor_sync(0xffffffffu, k, 1);
  return k;
}

template <typename InT>
__device__ __forceinline__ int sat_scale_of(const SatMapDev& Mp, float* bound) {
  int s = Mp.scale_log2;
  *bound = Mp.bound;
  if (s == kScaleFromDevice) {
    *bound = __ldcg(Mp.bound_dev);
    s = sat_scale_for(*bound, Mp.max_cells);
  }
  return s;
}

// I64 step 1: one CTA per tile (warp w: rows 4w..4w+3, lane: columns
// 4l..4l+3); exact row totals -> row_tot, column totals -> col_tot.
template <typename InT>
__global__ void __launch_bounds__(256) k_sat_reduce(const __grid_constant__ SatBatch B) {
  pdl_trigger();
  pdl_wait();
  __shared__ u64 s_col[8][kSatTileW];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &SatMapDev::item_tile);
  const SatMapDev& Mp = B.m[mi];
  const int tile = (int)blockIdx.x - Mp.item_tile;
  const int b = tile / Mp.n_chunks, j = tile - b * Mp.n_chunks;
  const int r0 = b * kSatTileH, cbase = j * kSatTileW + lane * 4;
  const int rows = Mp.rows, cols = Mp.cols;
  const InT* map = reinterpret_cast<const InT*>(Mp.map);
  const bool vec = ((Mp.ld & 3) == 0) &&
                   ((reinterpret_cast<uintptr_t>(map) & (std::is_same<InT, float>::value ? 15 : 7)) == 0);
  float bound;
  const int s = sat_scale_of<InT>(Mp, &bound);
  if (tile == 0 && tid == 0 && Mp.scale_out) *Mp.scale_out = s;
  const float scalef = ldexpf(1.0f, s);

  float v[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + w * 4 + i;
    if (r < rows) {
      load_row4<InT>(map + (long long)r * Mp.ld, cbase, cols, vec, Mp.in_scale, v[i]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[i][k] = 0.f;
    }
  }
  bool bad = false;
  u64 q[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      bad |= !(fabsf(v[i][k]) <= bound);  // NaN fails too
      q[i][k] = (u64)q_from_f32(v[i][k], scalef);
    }
  u64 p[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) p[i] = (q[i][0] + q[i][1]) + (q[i][2] + q[i][3]);
  const u64 rt = warp_sum4(p, lane);
  if ((lane & 7) == 0) __stcg(Mp.row_tot + (long long)tile * kSatTileH + w * 4 + (lane >> 3), rt);
#pragma unroll
  for (int k = 0; k < 4; ++k) s_col[w][lane * 4 + k] = (q[0][k] + q[1][k]) + (q[2][k] + q[3][k]);
  __syncthreads();
  if (tid < kSatTileW) {
    u64 t = 0;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) t += s_col[ww][tid];
    const int c = j * kSatTileW + tid;
    if (c < cols) __stcg(Mp.col_tot + (long long)b * Mp.ld_carry + c, t);
  }
  if (bad) atomicOr(B.status, kStatusRange);
}

// I64 step 3: S = tile-local prefix + CC_j(r) + RC_{b-1}(c), written as the
// table. Grid-stride over tiles; the next tile's map cells are staged into
// shared memory with cp.async while the current tile is scanned (each
// thread stages exactly the cells it later reads, so the staging needs no
// barrier).
template <typename InT>
__global__ void __launch_bounds__(256, 3) k_sat_down(const __grid_constant__ SatBatch B, int total_tiles) {
  pdl_trigger();
  pdl_wait();
  __shared__ __align__(16) InT s_map[2][kSatTileH][kSatTileW];
  __shared__ u64 s_wt[8][kSatTileW];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  constexpr bool kF32 = std::is_same<InT, float>::value;

  auto stage = [&](int t, int buf) {
    const int mi = find_item(B.m, B.n, t, &SatMapDev::item_tile);
    const SatMapDev& Mp = B.m[mi];
    const int tile = t - Mp.item_tile;
    const int b = tile / Mp.n_chunks, j = tile - b * Mp.n_chunks;
    const int cbase = j * kSatTileW + lane * 4;
    const InT* map = reinterpret_cast<const InT*>(Mp.map);
    const bool vec = ((Mp.ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(map) & (kF32 ? 15 : 7)) == 0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int rl = w * 4 + i, r = b * kSatTileH + rl;
      InT* dst = &s_map[buf][rl][lane * 4];
      const InT* src = map + (long long)r * Mp.ld + cbase;
      if (r < Mp.rows && vec && cbase + 3 < Mp.cols) {
        if constexpr (kF32) cp_async16(smem_u32(dst), src, true);
        else cp_async8(smem_u32(dst), src);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) dst[k] = (r < Mp.rows && cbase + k < Mp.cols) ? src[k] : InT(0.0f);
      }
    }
  };

  int t = (int)blockIdx.x;
  if (t < total_tiles) stage(t, 0);
  cp_async_commit();
  for (int buf = 0; t < total_tiles; t += (int)gridDim.x, buf ^= 1) {
    const int tn = t + (int)gridDim.x;
    if (tn < total_tiles) stage(tn, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();

    const int mi = find_item(B.m, B.n, t, &SatMapDev::item_tile);
    const SatMapDev& Mp = B.m[mi];
    const int tile = t - Mp.item_tile;
    const int b = tile / Mp.n_chunks, j = tile - b * Mp.n_chunks;
    const int cbase = j * kSatTileW + lane * 4;
    const int rows = Mp.rows, cols = Mp.cols;
    float bound;
    const float scalef = ldexpf(1.0f, sat_scale_of<InT>(Mp, &bound));

    u64 L[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float v[4];
      if constexpr (kF32) {
        const float4 x = *reinterpret_cast<const float4*>(&s_map[buf][w * 4 + i][lane * 4]);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
      } else {
        const uint2 x = *reinterpret_cast<const uint2*>(&s_map[buf][w * 4 + i][lane * 4]);
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&x.x));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&x.y));
        v[0] = f0.x * Mp.in_scale; v[1] = f0.y * Mp.in_scale; v[2] = f1.x * Mp.in_scale; v[3] = f1.y * Mp.in_scale;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) L[i][k] = (u64)q_from_f32(v[k], scalef);
    }
    tile_prefix<u64>(L, s_wt, w, lane);  // contains a __syncthreads

    u64 rc[4] = {0, 0, 0, 0};
    if (b > 0) {
      const ulonglong2* src = reinterpret_cast<const ulonglong2*>(Mp.row_carry + (long long)(b - 1) * Mp.ld_carry + cbase);
      const ulonglong2 a0 = __ldg(src), a1 = __ldg(src + 1);
      rc[0] = a0.x; rc[1] = a0.y; rc[2] = a1.x; rc[3] = a1.y;
    }
    long long* out = reinterpret_cast<long long*>(Mp.table);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = b * kSatTileH + w * 4 + i;
      if (r >= rows) continue;
      const u64 cc = __ldg(Mp.col_carry + (long long)j * rows + r);
      long long o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) o[k] = (long long)(L[i][k] + rc[k] + cc);
      long long* dst = out + (long long)r * Mp.ld_table + cbase;
      if (cbase + 3 < cols) {
        reinterpret_cast<longlong2*>(dst)[0] = make_longlong2(o[0], o[1]);
        reinterpret_cast<longlong2*>(dst)[1] = make_longlong2(o[2], o[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cbase + k < cols) dst[k] = o[k];
      }
    }
    __syncthreads();  // s_wt is rewritten by the next tile
  }
  cp_async_wait<0>();
}

// Block-wide exclusive scan of one value per thread (256 threads).
template <typename Acc>
__device__ __forceinline__ Acc block_excl_scan(Acc x, Acc* s_warp, Acc* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Acc e = warp_excl_scan(x, lane);
  if (lane == 31) s_warp[w] = e + x;
  __syncthreads();
  Acc base = Acc(0), tot = Acc(0);
#pragma unroll
  for (int ww = 0; ww < 8; ++ww) {
    const Acc t = s_warp[ww];
    if (ww < w) base += t;
    tot += t;
  }
  __syncthreads();
  *total = tot;
  return base + e;
}

// Pass 2: one CTA per band. (a) the band's inclusive row prefix of the
// column totals across the whole width, in place; (b) CC for every tile of
// the band: the 8 warps take consecutive runs of the band's tiles, lane =
// band row. A warp first needs the row sums of all tiles left of its run:
// each warp sums its run's row totals, and a warp starts from the sums of
// the warps before it.
template <typename Acc>
__global__ void __launch_bounds__(256) k_sat_hscan(const __grid_constant__ SatBatch B) {
  pdl_trigger();
  pdl_wait();
  __shared__ Acc s_warp[8];
  __shared__ Acc s_run[8][32];
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &SatMapDev::item_band);
  const SatMapDev& Mp = B.m[mi];
  const int b = (int)blockIdx.x - Mp.item_band;
  const int cols = Mp.cols, rows = Mp.rows;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  u64* row = Mp.col_tot + (long long)b * Mp.ld_carry;
  const int per = (cols + 255) / 256;
  const int c0 = threadIdx.x * per, c1 = min(cols, c0 + per);
  {
    Acc t = Acc(0);
#pragma unroll 4
    for (int c = c0; c < c1; ++c) t += ld_carry<Acc>(row + c);
    Acc tot;
    Acc run = block_excl_scan<Acc>(t, s_warp, &tot);
#pragma unroll 4
    for (int c = c0; c < c1; ++c) {
      run += ld_carry<Acc>(row + c);
      st_carry<Acc>(row + c, run);
    }
  }
  const int nch = Mp.n_chunks;
  const int jper = (nch + 7) / 8;
  const int j0 = w * jper, j1 = min(nch, j0 + jper);
  const int r0 = b * kSatTileH;
  const u64* rt = Mp.row_tot + (long long)b * nch * kSatTileH + lane;
  Acc part = Acc(0);
#pragma unroll 4
  for (int j = j0; j < j1; ++j) part += ld_carry<Acc>(rt + (long long)j * kSatTileH);
  s_run[w][lane] = part;
  __syncthreads();
  Acc hc = Acc(0);
  for (int ww = 0; ww < w; ++ww) hc += s_run[ww][lane];
  for (int j = j0; j < j1; ++j) {
    const Acc t = ld_carry<Acc>(rt + (long long)j * kSatTileH);
    Acc cc = hc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Acc y = __shfl_up_sync(0xffffffffu, cc, o);
      if (lane >= o) cc += y;
    }
    if (r0 + lane < rows) st_carry<Acc>(Mp.col_carry + (long long)j * rows + r0 + lane, cc);
    hc += t;
  }
}

// Pass 3: RC_b(c) = sum over bands <= b of the bands' row prefixes.
// CTA = 32 columns (lane) x 32 groups of consecutive bands (warp).
template <typename Acc>
__global__ void __launch_bounds__(1024) k_sat_vscan(const __grid_constant__ SatBatch B) {
  pdl_trigger();
  pdl_wait();
  __shared__ Acc s_tot[32][32];
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &SatMapDev::item_vscan);
  const SatMapDev& Mp = B.m[mi];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = ((int)blockIdx.x - Mp.item_vscan) * 32 + lane;
  const bool ok = c < Mp.cols;
  const int G = (Mp.n_bands + 31) / 32;
  const int b0 = w * G, b1 = min(Mp.n_bands, b0 + G);
  Acc t = Acc(0);
  if (ok) {
#pragma unroll 4
    for (int b = b0; b < b1; ++b) t += ld_carry<Acc>(Mp.col_tot + (long long)b * Mp.ld_carry + c);
  }
  s_tot[w][lane] = t;
  __syncthreads();
  Acc run = Acc(0);
  for (int ww = 0; ww < w; ++ww) run += s_tot[ww][lane];
  if (ok) {
#pragma unroll 4
    for (int b = b0; b < b1; ++b) {
      run += ld_carry<Acc>(Mp.col_tot + (long long)b * Mp.ld_carry + c);
      st_carry<Acc>(Mp.row_carry + (long long)b * Mp.ld_carry + c, run);
    }
  }
}

// NAIVE_F32: fold the carries into the tile-local table in place.
template <int MODE>
__global__ void __launch_bounds__(256) k_sat_finalize(const __grid_constant__ SatBatch B) {
  pdl_trigger();
  pdl_wait();
  typedef typename SatTypes<MODE>::Acc Acc;
  typedef typename SatTypes<MODE>::Loc Loc;
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &SatMapDev::item_tile);
  const SatMapDev& Mp = B.m[mi];
  const int tile = (int)blockIdx.x - Mp.item_tile;
  const int b = tile / Mp.n_chunks, j = tile - b * Mp.n_chunks;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int cbase = j * kSatTileW + lane * 4;
  Acc rc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    rc[k] = (b > 0 && cbase + k < Mp.cols) ? ld_carry<Acc>(Mp.row_carry + (long long)(b - 1) * Mp.ld_carry + cbase + k)
                                           : Acc(0);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = b * kSatTileH + w * 4 + i;
    if (r >= Mp.rows) continue;
    const Acc cc = ld_carry<Acc>(Mp.col_carry + (long long)j * Mp.rows + r);
    Loc* o = reinterpret_cast<Loc*>(Mp.table) + (long long)r * Mp.ld_table + cbase;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (cbase + k < Mp.cols) o[k] = o[k] + rc[k] + cc;
  }
}

template <typename InT>
__global__ void k_map_max(const InT* map, float scale, int rows, int cols, long long ld, unsigned* out) {
  float m = 0.f;
  const long long total = (long long)rows * cols;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / cols), c = (int)(i % cols);
    const float v = fabsf(ld_val(map + (long long)r * ld + c) * scale);
    m = (v > m || v != v) ? v : m;  // keep NaN so the bound check fails later
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float y = __shfl_xor_sync(0xffffffffu, m, o);
    m = (y > m || y != y) ? y : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

template <int MODE>
__global__ void k_sat_materialize(const __grid_constant__ SatMapDev Mp, double* out, long long ld_out) {
  const long long total = (long long)Mp.rows * Mp.cols;
  const int s = *Mp.scale_out;
  const double inv = ldexp(1.0, -s);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / Mp.cols), c = (int)(i % Mp.cols);
    double v;
    if constexpr (MODE == RCFAR_SAT_TILE_F32 || MODE == RCFAR_SAT_TILE_I64) {
      const int band = r / kSatTileH, chunk = c / kSatTileW;
      u64 carry = Mp.col_carry[(long long)chunk * Mp.rows + r];
      if (band > 0) carry += Mp.row_carry[(long long)(band - 1) * Mp.ld_carry + c];
      if constexpr (MODE == RCFAR_SAT_TILE_F32) {
        const float l = reinterpret_cast<const float*>(Mp.table)[(long long)r * Mp.ld_table + c];
        v = (double)l + (double)(long long)carry * inv;
      } else {
        const u64 l = (u64)reinterpret_cast<const long long*>(Mp.table)[(long long)r * Mp.ld_table + c];
        v = (double)(long long)(l + carry) * inv;
      }
    } else if constexpr (MODE == RCFAR_SAT_I64) {
      v = (double)reinterpret_cast<const long long*>(Mp.table)[(long long)r * Mp.ld_table + c] * inv;
    } else {
      v = (double)reinterpret_cast<const float*>(Mp.table)[(long long)r * Mp.ld_table + c];
    }
    out[(long long)r * ld_out + c] = v;
  }
}

}  // namespace

cudaError_t launch_map_max(const void* map, int dtype, float in_scale, int rows, int cols, long long ld,
                           float* out_bits, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out_bits, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  const long long total = (long long)rows * cols;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  unsigned* o = reinterpret_cast<unsigned*>(out_bits);
  if (dtype == RCFAR_MAP_F16)
    k_map_max<__half><<<blocks, 256, 0, s>>>(reinterpret_cast<const __half*>(map), in_scale, rows, cols, ld, o);
  else
    k_map_max<float><<<blocks, 256, 0, s>>>(reinterpret_cast<const float*>(map), in_scale, rows, cols, ld, o);
  return cudaGetLastError();
}

template <int MODE, typename InT>
static cudaError_t launch_sat_t(const SatBatch& b, int tiles, int bands, int vscans, cudaStream_t s) {
  typedef typename SatTypes<MODE>::Acc Acc;
  cudaError_t e;
  if constexpr (MODE == RCFAR_SAT_I64) {
    if ((e = launch_pdl(k_sat_reduce<InT>, tiles, 256, 0, s, b)) != cudaSuccess) return e;
    if ((e = launch_pdl(k_sat_hscan<Acc>, bands, 256, 0, s, b)) != cudaSuccess) return e;
    if ((e = launch_pdl(k_sat_vscan<Acc>, vscans, 1024, 0, s, b)) != cudaSuccess) return e;
    // grid-stride: about three resident CTAs per SM, each streaming tiles
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = tiles < 3 * sms ? tiles : 3 * sms;
    return launch_pdl(k_sat_down<InT>, grid, 256, 0, s, b, tiles);
  }
  if ((e = launch_pdl(k_sat_tile<MODE, InT>, tiles, 256, 0, s, b)) != cudaSuccess) return e;
  if ((e = launch_pdl(k_sat_hscan<Acc>, bands, 256, 0, s, b)) != cudaSuccess) return e;
  if ((e = launch_pdl(k_sat_vscan<Acc>, vscans, 1024, 0, s, b)) != cudaSuccess) return e;
  if constexpr (MODE == RCFAR_SAT_NAIVE_F32) return launch_pdl(k_sat_finalize<MODE>, tiles, 256, 0, s, b);
  return cudaSuccess;
}

cudaError_t launch_sat(const SatBatch& b, int mode, int dtype, int tiles, int bands, int vscans, cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  const bool h = dtype == RCFAR_MAP_F16;
  switch (mode) {
    case RCFAR_SAT_TILE_F32:
      return h ? launch_sat_t<RCFAR_SAT_TILE_F32, __half>(b, tiles, bands, vscans, s)
               : launch_sat_t<RCFAR_SAT_TILE_F32, float>(b, tiles, bands, vscans, s);
    case RCFAR_SAT_I64:
      return h ? launch_sat_t<RCFAR_SAT_I64, __half>(b, tiles, bands, vscans, s)
               : launch_sat_t<RCFAR_SAT_I64, float>(b, tiles, bands, vscans, s);
    case RCFAR_SAT_TILE_I64:
      return h ? launch_sat_t<RCFAR_SAT_TILE_I64, __half>(b, tiles, bands, vscans, s)
               : launch_sat_t<RCFAR_SAT_TILE_I64, float>(b, tiles, bands, vscans, s);
    default:
      return h ? launch_sat_t<RCFAR_SAT_NAIVE_F32, __half>(b, tiles, bands, vscans, s)
               : launch_sat_t<RCFAR_SAT_NAIVE_F32, float>(b, tiles, bands, vscans, s);
  }
}

cudaError_t launch_sat_materialize(const SatMapDev& m, int mode, double* out, long long ld_out, cudaStream_t s) {
  const long long total = (long long)m.rows * m.cols;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  switch (mode) {
    case RCFAR_SAT_TILE_F32: k_sat_materialize<RCFAR_SAT_TILE_F32><<<blocks, 256, 0, s>>>(m, out, ld_out); break;
    case RCFAR_SAT_I64: k_sat_materialize<RCFAR_SAT_I64><<<blocks, 256, 0, s>>>(m, out, ld_out); break;
    case RCFAR_SAT_TILE_I64: k_sat_materialize<RCFAR_SAT_TILE_I64><<<blocks, 256, 0, s>>>(m, out, ld_out); break;
    default: k_sat_materialize<RCFAR_SAT_NAIVE_F32><<<blocks, 256, 0, s>>>(m, out, ld_out); break;
  }
  return cudaGetLastError();
}

}  // namespace rcfar
