// Summed-area table of a CFAR input map (paper eq. 3), one pass over the map.
//
// The map is cut into tiles of kSatTileH x kSatTileW cells (band b = tile
// row, chunk j = tile column), one CTA per tile, taken in row-major ticket
// order. For cell (r, c) of tile (b, j):
//   S(r, c) = L(r, c) + CC_j(r) + RC_b(c)
//   L      : table of the tile relative to its own origin (tile-local)
//   CC_j(r): sum over band rows <= r and columns left of the tile
//   RC_b(c): S(first row of band b - 1, c), the table on the row above
// Both carries are exclusive scans across tiles, resolved with decoupled
// look-backs: horizontally over the row totals of the tiles to the left
// (vectors of kSatTileH values), then vertically over the column aggregates
// of the tiles above (vectors of kSatTileW values). Each tile publishes its
// aggregate before it looks back, and waits only on tiles with smaller
// tickets, so the chains stay short and every wait ends.
// Carries are 64-bit fixed point q = round(x * 2^s) added modulo 2^64
// (exact; every region sum below 2^63 comes out exact even if S wraps).
//   TILE_F32 : stores L in FP32, RC (as each band's inclusive values) and CC.
//   I64      : stores S itself in fixed point (L exact as well).
//   NAIVE_F32: FP32 everywhere, stores S in FP32.
// Within a tile, row prefixes use warp shuffles (32 lanes x 4 columns) and
// column prefixes a shared-memory exchange between the 8 warps.
#include "rcfar_internal.cuh"

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

__device__ __forceinline__ unsigned ld_flag(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_flag(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Poll a look-back flag until it carries this launch's generation and a
// published state; gives up after kSpinLimit polls, records the timeout and
// returns 0xffffffff.
__device__ __forceinline__ unsigned wait_flag(const unsigned* fp, unsigned gen, int* status) {
  for (unsigned it = 0;; ++it) {
    const unsigned f = ld_flag(fp);
    if ((f >> 2) == gen && (f & 3u) != 0u) return f;
    if (it >= kSpinLimit) {
      atomicOr(status, kStatusTimeout);
      return 0xffffffffu;
    }
    __nanosleep(32);
  }
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

template <int MODE, typename InT>
__global__ void __launch_bounds__(256) k_sat(const __grid_constant__ SatBatch B) {
  // Acc: carry arithmetic (exact fixed point, or FP32 for the naive table)
  typedef typename std::conditional<MODE == RCFAR_SAT_NAIVE_F32, float, u64>::type Acc;
  // Loc: tile-local table arithmetic
  typedef typename std::conditional<MODE == RCFAR_SAT_I64, u64, float>::type Loc;

  __shared__ unsigned s_item, s_gen;
  __shared__ Loc s_wt[8][kSatTileW];
  __shared__ Acc s_wc[8][kSatTileW];
  __shared__ Acc s_rq[kSatTileH];
  __shared__ Acc s_cc[kSatTileH];
  __shared__ Acc s_rc[kSatTileW];

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    s_gen = ld_flag(B.gen);
    s_item = atomicAdd(B.ticket, 1u);
  }
  __syncthreads();
  const int item = (int)s_item;
  const unsigned gen = s_gen & 0x3fffffffu;
  const int mi = find_item(B.m, B.n, item, &SatMapDev::item0);
  const SatMapDev& Mp = B.m[mi];
  const int tile = item - Mp.item0;
  const int b = tile / Mp.n_chunks, j = tile - b * Mp.n_chunks;
  const int r0 = b * kSatTileH;
  const int cbase = j * kSatTileW + lane * 4;
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

  // ---- load and quantise the tile (warp w: rows 4w..4w+3, lane: 4 columns)
  float v[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + w * 4 + i;
    if (r < Mp.rows) {
      load_row4<InT>(map + (long long)r * Mp.ld, cbase, Mp.cols, vec, Mp.in_scale, v[i]);
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
      else q[i][k] = (u64)__float2ll_rn(v[i][k] * scalef);
    }

  // ---- tile-local table
  Loc L[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if constexpr (std::is_same<Loc, float>::value) L[i][k] = v[i][k];
      else L[i][k] = q[i][k];
    }
  tile_prefix<Loc>(L, s_wt, w, lane);

  if constexpr (MODE == RCFAR_SAT_TILE_F32) {
    float* out = reinterpret_cast<float*>(Mp.table);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + w * 4 + i;
      if (r >= Mp.rows) continue;
      float* o = out + (long long)r * Mp.ld_table + cbase;
      if (cbase + 3 < Mp.cols) {
        *reinterpret_cast<float4*>(o) = make_float4(L[i][0], L[i][1], L[i][2], L[i][3]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cbase + k < Mp.cols) o[k] = L[i][k];
      }
    }
  }

  // ---- row totals (exact) and column sums (exact) of the tile
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const Acc t = warp_sum<Acc>(q[i][0] + q[i][1] + q[i][2] + q[i][3]);
    if (lane == i) s_rq[w * 4 + i] = t;
  }
  if constexpr (MODE == RCFAR_SAT_I64) {
    // the exact tile table's last row is the column prefix itself
    if (w == 7) {
#pragma unroll
      for (int k = 0; k < 4; ++k) s_wc[0][lane * 4 + k] = L[3][k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) s_wc[w][lane * 4 + k] = q[0][k] + q[1][k] + q[2][k] + q[3][k];
  }
  __syncthreads();

  const int ntile = b * Mp.n_chunks + j;
  if (w == 0) {
    // ---- horizontal look-back: lane = band row
    const Acc my = s_rq[lane];
    Acc hc = Acc(0);
    if (j == 0) {
      st_carry<Acc>(Mp.h_inc + (long long)ntile * kSatTileH + lane, my);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_flag(Mp.h_flags + ntile, (gen << 2) | 2u);
    } else {
      st_carry<Acc>(Mp.h_agg + (long long)ntile * kSatTileH + lane, my);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_flag(Mp.h_flags + ntile, (gen << 2) | 1u);
      // warp-parallel window: lane l polls the tile l places to the left; the
      // nearest inclusive value ends the walk, aggregates before it are summed
      for (int jj = j - 1; jj >= 0; jj -= 32) {
        const int p = jj - lane;
        unsigned f = 2u;
        if (p >= 0) f = wait_flag(Mp.h_flags + b * Mp.n_chunks + p, gen, B.status);
        if (__any_sync(0xffffffffu, f == 0xffffffffu)) break;  // timed out: status recorded
        const unsigned incm = __ballot_sync(0xffffffffu, p >= 0 && (f & 3u) == 2u);
        const int take = incm ? __ffs(incm) : min(32, jj + 1);
        __threadfence();
        for (int l = 0; l < take; ++l) {
          const long long pt = (long long)b * Mp.n_chunks + (jj - l);
          const u64* src = ((incm >> l) & 1u) ? Mp.h_inc : Mp.h_agg;
          hc += ld_carry<Acc>(src + pt * kSatTileH + lane);
        }
        if (incm) break;
      }
      st_carry<Acc>(Mp.h_inc + (long long)ntile * kSatTileH + lane, hc + my);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_flag(Mp.h_flags + ntile, (gen << 2) | 2u);
    }
    // CC_j(r) = sum over band rows <= r of the horizontal carries
    Acc cc = hc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const Acc y = __shfl_up_sync(0xffffffffu, cc, o);
      if (lane >= o) cc += y;
    }
    s_cc[lane] = cc;
    if constexpr (MODE == RCFAR_SAT_TILE_F32) {
      if (r0 + lane < Mp.rows) st_carry<Acc>(Mp.col_carry + (long long)j * Mp.rows + r0 + lane, cc);
    }
    const Acc base = __shfl_sync(0xffffffffu, cc, 31);

    // ---- column aggregate A(c) = S_band(last row, c); vertical look-back
    Acc a[4];
    if constexpr (MODE == RCFAR_SAT_I64) {
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] = s_wc[0][lane * 4 + k] + base;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        Acc t = s_wc[0][lane * 4 + k];
#pragma unroll
        for (int ww = 1; ww < 8; ++ww) t += s_wc[ww][lane * 4 + k];
        a[k] = t;
      }
#pragma unroll
      for (int k = 1; k < 4; ++k) a[k] += a[k - 1];
      const Acc e = warp_excl_scan(a[3], lane);
#pragma unroll
      for (int k = 0; k < 4; ++k) a[k] += e + base;
    }
    const long long crow = (long long)j * kSatTileW + lane * 4;
    Acc rc[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
    if (b == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) st_carry<Acc>(Mp.row_carry + crow + k, a[k]);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_flag(Mp.v_flags + ntile, (gen << 2) | 2u);
    } else {
      u64* aggp = Mp.v_agg + (long long)b * Mp.ld_carry + crow;
#pragma unroll
      for (int k = 0; k < 4; ++k) st_carry<Acc>(aggp + k, a[k]);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_flag(Mp.v_flags + ntile, (gen << 2) | 1u);
      for (int bb = b - 1; bb >= 0; bb -= 32) {
        const int p = bb - lane;
        unsigned f = 2u;
        if (p >= 0) f = wait_flag(Mp.v_flags + p * Mp.n_chunks + j, gen, B.status);
        if (__any_sync(0xffffffffu, f == 0xffffffffu)) break;  // timed out: status recorded
        const unsigned incm = __ballot_sync(0xffffffffu, p >= 0 && (f & 3u) == 2u);
        const int take = incm ? __ffs(incm) : min(32, bb + 1);
        __threadfence();
        for (int l = 0; l < take; ++l) {
          const u64* src = (((incm >> l) & 1u) ? Mp.row_carry : Mp.v_agg) + (long long)(bb - l) * Mp.ld_carry + crow;
#pragma unroll
          for (int k = 0; k < 4; ++k) rc[k] += ld_carry<Acc>(src + k);
        }
        if (incm) break;
      }
      u64* incp = Mp.row_carry + (long long)b * Mp.ld_carry + crow;
#pragma unroll
      for (int k = 0; k < 4; ++k) st_carry<Acc>(incp + k, rc[k] + a[k]);
      __threadfence();
      __syncwarp();
      if (lane == 0) st_flag(Mp.v_flags + ntile, (gen << 2) | 2u);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) s_rc[lane * 4 + k] = rc[k];
  }

  if constexpr (MODE != RCFAR_SAT_TILE_F32) {
    __syncthreads();
    Acc rcv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) rcv[k] = s_rc[lane * 4 + k];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + w * 4 + i;
      if (r >= Mp.rows) continue;
      const Acc cc = s_cc[w * 4 + i];
      if constexpr (MODE == RCFAR_SAT_I64) {
        long long* o = reinterpret_cast<long long*>(Mp.table) + (long long)r * Mp.ld_table + cbase;
        if (cbase + 3 < Mp.cols) {
          const longlong2 v0 = make_longlong2((long long)(L[i][0] + rcv[0] + cc), (long long)(L[i][1] + rcv[1] + cc));
          const longlong2 v1 = make_longlong2((long long)(L[i][2] + rcv[2] + cc), (long long)(L[i][3] + rcv[3] + cc));
          reinterpret_cast<longlong2*>(o)[0] = v0;
          reinterpret_cast<longlong2*>(o)[1] = v1;
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (cbase + k < Mp.cols) o[k] = (long long)(L[i][k] + rcv[k] + cc);
        }
      } else {
        float* o = reinterpret_cast<float*>(Mp.table) + (long long)r * Mp.ld_table + cbase;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cbase + k < Mp.cols) o[k] = L[i][k] + rcv[k] + cc;
      }
    }
  }

  if (bad) atomicOr(B.status, kStatusRange);
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned d = atomicAdd(B.done, 1u);
    if (d == (unsigned)B.total - 1u) {  // last CTA of the launch: reset for the next one
      *B.ticket = 0u;
      *B.done = 0u;
      __threadfence();
      atomicAdd(B.gen, 1u);
    }
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
    if constexpr (MODE == RCFAR_SAT_TILE_F32) {
      const float l = reinterpret_cast<const float*>(Mp.table)[(long long)r * Mp.ld_table + c];
      const int band = r / kSatTileH, chunk = c / kSatTileW;
      u64 carry = Mp.col_carry[(long long)chunk * Mp.rows + r];
      if (band > 0) carry += Mp.row_carry[(long long)(band - 1) * Mp.ld_carry + c];
      v = (double)l + (double)(long long)carry * inv;
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

cudaError_t launch_sat(const SatBatch& b, int mode, int dtype, cudaStream_t s) {
  if (b.total <= 0) return cudaSuccess;
  const bool h = dtype == RCFAR_MAP_F16;
  switch (mode) {
    case RCFAR_SAT_TILE_F32:
      if (h) k_sat<RCFAR_SAT_TILE_F32, __half><<<b.total, 256, 0, s>>>(b);
      else k_sat<RCFAR_SAT_TILE_F32, float><<<b.total, 256, 0, s>>>(b);
      break;
    case RCFAR_SAT_I64:
      if (h) k_sat<RCFAR_SAT_I64, __half><<<b.total, 256, 0, s>>>(b);
      else k_sat<RCFAR_SAT_I64, float><<<b.total, 256, 0, s>>>(b);
      break;
    default:
      if (h) k_sat<RCFAR_SAT_NAIVE_F32, __half><<<b.total, 256, 0, s>>>(b);
      else k_sat<RCFAR_SAT_NAIVE_F32, float><<<b.total, 256, 0, s>>>(b);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_sat_materialize(const SatMapDev& m, int mode, double* out, long long ld_out, cudaStream_t s) {
  const long long total = (long long)m.rows * m.cols;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  switch (mode) {
    case RCFAR_SAT_TILE_F32: k_sat_materialize<RCFAR_SAT_TILE_F32><<<blocks, 256, 0, s>>>(m, out, ld_out); break;
    case RCFAR_SAT_I64: k_sat_materialize<RCFAR_SAT_I64><<<blocks, 256, 0, s>>>(m, out, ld_out); break;
    default: k_sat_materialize<RCFAR_SAT_NAIVE_F32><<<blocks, 256, 0, s>>>(m, out, ld_out); break;
  }
  return cudaGetLastError();
}

}  // namespace rcfar
