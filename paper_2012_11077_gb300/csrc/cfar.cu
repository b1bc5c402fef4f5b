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
// k_cfar_ring   : the same on the I64 table S itself, whose rows stream
//                 through a shared-memory ring fed by bulk copies.
// k_sat_cfar_fused, k_sat_cfar_stream : SAT and CFAR in one pass, the table
//                 never in device memory (per-block integral images; or a
//                 strip's integral image walked down the rows in a ring).
// k_cfar_direct : the sliding-window CFAR the SAT replaces: the same
//                 decisions with S_ref summed over the n_ref training cells.
// k_cfar_os     : ordered-statistic thresholds (a next-step variant, not a
//                 region sum): the k-th smallest training cell per CUT.
// Greatest-of / smallest-of thresholds take the two half sums of the
// training ring from 16 lookups in every SAT kernel and k_cfar_direct.
#include "rcfar_internal.cuh"
#include "async_copy.cuh"
#include "fixed_point.cuh"

#include <algorithm>
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
      q = (u64)q_from_f32_wide(__ldg(reinterpret_cast<const float*>(P.table) + (long long)r * P.ld_table + c), scalef);
    else
      q = (u64)__ldg(reinterpret_cast<const long long*>(P.table) + (long long)r * P.ld_table + c);
    q += __ldg(P.col_carry + (long long)(c >> 7) * P.rows + r);  // kSatTileW == 128
    const int band = r >> 5;                                       // kSatTileH == 32
    if (band > 0) q += __ldg(P.row_carry + (long long)(band - 1) * P.ld_carry + c);
    return q;
  }
}

// Sum over table rows (top, bot] and the columns within w of the CUT's
// column, by eq. 4; both pointers are at the CUT's column.
template <typename SV>
__device__ __forceinline__ SV box_rows(const SV* top, const SV* bot, int w) {
  return (top[-w - 1] + bot[w]) - (top[w] + bot[-w - 1]);
}
__device__ __forceinline__ bool sv_greater(u64 a, u64 b) { return (long long)a > (long long)b; }
__device__ __forceinline__ bool sv_greater(float a, float b) { return a > b; }

// Greatest-of / smallest-of statistic: the larger (greatest) or smaller of
// the leading half (rows r - wr .. r - 1 minus the guard rows r - gr .. r - 1
// within gc columns) and the lagging half (rows r + 1 .. r + wr minus
// r + 1 .. r + gr). Row pointers at the CUT's column: ra = r - wr - 1,
// r0 = r - 1, rc = r - gr - 1 (leading); r1 = r, rd = r + gr, rb = r + wr
// (lagging). With gr = 0 the guard boxes are empty (rc = r0, rd = r1).
template <typename SV>
__device__ __forceinline__ SV go_so_stat(bool greatest, const SV* ra, const SV* rb, const SV* rc, const SV* rd,
                                         const SV* r1, const SV* r0, int wc, int gc) {
  const SV lead = box_rows(ra, r0, wc) - box_rows(rc, r0, gc);
  const SV lag = box_rows(r1, rb, wc) - box_rows(r1, rd, gc);
  return sv_greater(lead, lag) == greatest ? lead : lag;
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
  pdl_trigger();
  pdl_wait();
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
  const int kind = P.kind;
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
        SV ref;
        if (kind == RCFAR_CFAR_CA) {
          // eq. 4: A = L1 + L4 - (L2 + L3) for the outer and the guard rectangle
          const SV outer = (Sa[ca] + Sb[cb]) - (Sa[cb] + Sb[ca]);
          const SV guard = (Sc[cg] + Sd[cd]) - (Sc[cd] + Sd[cg]);
          ref = outer - guard;
        } else {
          const SV* S1 = S + (g & rmask) * HC + cm;        // row r at the CUT's column
          const SV* S0 = S + ((g - 1) & rmask) * HC + cm;  // row r - 1
          ref = go_so_stat(kind == RCFAR_CFAR_GO, Sa + cm, Sb + cm, Sc + cm, Sd + cm, S1, S0, wc, gc);
        }
        if constexpr (kExact) {
          // T = (alpha / n_ref) * S_ref in fixed-point units; the CUT value
          // comes from the map when one is given, else from the exact table
          // (eq. 4 on the 1x1 region)
          const float ts = f32_from_q((long long)ref) * kthr;
          t = ts * inv_s;
          if (map != nullptr) {
            d = cutv[i] > t ? 1 : 0;
          } else {
            const SV* S1 = S + (g & rmask) * HC;        // row r
            const SV* S0 = S + ((g - 1) & rmask) * HC;  // row r - 1
            const u64 qc = (S1[cm] + S0[cm - 1]) - (S0[cm] + S1[cm - 1]);
            d = f32_from_q((long long)qc) > ts ? 1 : 0;
          }
        } else {
          if constexpr (MODE == RCFAR_SAT_NAIVE_F32) t = ref * kk;
          else t = f32_from_q((long long)ref) * kk;
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


// S_ref by eq. 4 on the outer rectangle minus eq. 4 on the guard rectangle,
// regrouped as (four corners added) - (four corners subtracted). Rows: a =
// r - wr - 1, b = r + wr, c = r - gr - 1, d = r + gr; each pointer is at the
// CUT's column, so [o] is the column offset o from it.
__device__ __forceinline__ u64 ref_sum(const u64* ra, const u64* rb, const u64* rc, const u64* rd, int wc, int gc) {
  const u64 pos = (ra[-wc - 1] + rb[wc]) + (rc[gc] + rd[-gc - 1]);
  const u64 neg = (ra[wc] + rb[-wc - 1]) + (rc[-gc - 1] + rd[gc]);
  return pos - neg;
}


// SAT CFAR streaming an exact global table S (I64 mode: S is eq. 3 itself in
// 64-bit fixed point, so a lookup is one load). A CTA owns a strip of
// kRingW columns and a run of rows; warp w handles row w of each stage of
// kRingSR rows, lane l the columns l, l + 32, l + 64, l + 96 of the strip.
// The table rows the run reads (row -1 .. last CUT row + wr, strip plus
// halo) stream through a ring of ring_rows rows in shared memory, kRingSR rows
// per stage: a stage is kRingSR bulk copies of one table row each, completing
// on the stage's mbarrier, issued up to NS = ring_rows / kRingSR stages ahead. Warps
// never wait for one another: each waits only for the stages it reads, and
// the last warp to finish an output stage (a shared-memory counter per slot)
// issues the copies that refill the slot. Per CUT: S_ref from 8 lookups in
// 64-bit integer arithmetic, T = (alpha / n_ref) S_ref, and det = CUT > T
// with the CUT value from the map (kMapCut) or from the table (eq. 4 on the
// 1 x 1 region). Rows and strips fully inside the CUT range take a path
// without per-cell checks.
template <bool kMapCut, typename InT>
__global__ void __launch_bounds__(kRingThreads, 1) k_cfar_ring(const __grid_constant__ CfarBatch B) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  u64* bars = reinterpret_cast<u64*>(smem_raw);
  u64* ring = reinterpret_cast<u64*>(smem_raw + kRingBarBytes);
  __shared__ int s_fail;
  __shared__ unsigned s_done[kRingMaxStages];  // warps done with the slot's current stage
  constexpr int kWarps = kRingThreads / 32;

  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &CfarMapDev::item0);
  const CfarMapDev& P = B.m[mi];
  const int local = (int)blockIdx.x - P.item0;
  const int ty = local / P.tiles_x, tx = local - ty * P.tiles_x;
  const int rows = P.rows, cols = P.cols;
  const int R0 = ty * P.run, R1 = min(rows, R0 + P.run);
  const int c0 = tx * kRingW;
  const int wr = P.wr, wc = P.wc, gr = P.gr, gc = P.gc;
  const int hs = (c0 - wc - 1) & ~1;  // table column held in ring column 0 (even)
  const int HCP = P.hcp;
  const int RR = P.ring_rows;     // NS stages of kRingSR rows (NS need not be a power of two)
  const int NS = RR / kRingSR;
  const int gbase = R0 - wr - 1;  // ring row index g holds table row gbase + g
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long* T = reinterpret_cast<const long long*>(P.table);
  const long long ldt = P.ld_table;
  // ring slot of row index g: stage g / kRingSR in slot (g / kRingSR) % NS
  auto slot_row = [&](int g) { return ((g / kRingSR) % NS) * kRingSR + (g % kRingSR); };

  // CUTs of this CTA that take lookups
  const int rlo = max(R0, P.row_lo), rhi = min(R1 - 1, P.row_hi);
  const int clo = max(c0, P.cut_lo), chi = min(min(c0 + kRingW, cols) - 1, P.cut_hi);
  const bool work = rlo <= rhi && clo <= chi;
  const bool full_strip = clo == c0 && chi == c0 + kRingW - 1;  // every column is a CUT column
  const int gmax = work ? rhi + wr - gbase : -1;  // last ring row index read
  const int nq = work ? gmax / kRingSR + 1 : 0;   // table stages
  const int QL = (2 * wr + kRingSR) / kRingSR;    // output stage t reads table stages t .. t + QL
  const int nt = (R1 - R0 + kRingSR - 1) / kRingSR;
  // one table row's copy: columns cs .. ce - 1 (even bounds, inside the row's allocation)
  const int cs = max(hs, 0);
  const int ce = (int)min((long long)hs + HCP, ldt);
  const unsigned row_bytes = (unsigned)(ce - cs) * 8u;
  const int dcol = cs - hs;

  if (tid == 0) s_fail = 0;
  if (tid < NS) {
    mbar_init(smem_u32(&bars[tid]), 1);
    s_done[tid] = 0;
  }
  if (work) {
    // columns left of the map read as S(., -1) = 0; so does row -1
    if (hs < 0)
      for (int i = tid; i < RR * (-hs); i += kRingThreads) ring[(i / (-hs)) * HCP + (i % (-hs))] = 0;
    if (gbase <= -1) {
      u64* z = ring + slot_row(-1 - gbase) * HCP;
      for (int i = tid; i < HCP; i += kRingThreads) z[i] = 0;
    }
    fence_proxy_async();
  }
  if (tid == 0) mbar_init_fence();
  __syncthreads();

  auto issue = [&](int q) {  // one whole warp: table stage q into slot q % NS
    const int g0 = q * kRingSR;
    const int glo = max(g0, -gbase);  // rows >= 0 only
    const int ghi = min(g0 + kRingSR, gmax + 1);
    const int n = max(0, ghi - glo);
    const unsigned bar = smem_u32(&bars[q % NS]);
    if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)n * row_bytes);
    __syncwarp();
    if (lane < n) {
      const int g = glo + lane;
      bulk_g2s(smem_u32(ring + slot_row(g) * HCP + dcol), T + (long long)(gbase + g) * ldt + cs, row_bytes, bar);
    }
  };
  if (warp == 0)
    for (int q = 0; q < min(nq, NS); ++q) issue(q);

  const float kthr = P.kthr;
  const int kind = P.kind;
  int s = 0;
  if (work) s = __ldcg(P.scale_dev);
  const float inv_s = ldexpf(1.0f, -s);
  const InT* map = reinterpret_cast<const InT*>(P.map);
  const int cw = c0 + lane;     // this lane's columns: cw + 32 k
  const int x = cw - hs;        // its ring column
  int waited = -1;
  // The rows output row r = R0 + kRingSR t + warp reads have ring index
  // g = kRingSR t + warp + off; each lies in stage t + (warp + off) / kRingSR,
  // row (warp + off) % kRingSR of it. off for rows r - wr - 1, r + wr,
  // r - gr - 1, r + gr, r, r - 1:
  // Relative to the first ring row sb of the slot holding stage t, that row
  // is at sb + warp + off (stages are consecutive slots; wrapped once).
  const int coff[6] = {warp, warp + 2 * wr + 1, warp + wr - gr, warp + wr + gr + 1, warp + wr + 1, warp + wr};
  int sb = 0;  // first ring row of the slot holding stage t

  // CUT values of this warp's row in output stage t (map CUT only)
  auto load_cut = [&](int t, float (&v)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = 0.f;
    if constexpr (kMapCut) {
      const int r = R0 + t * kRingSR + warp;
      if (work && t < nt && r >= rlo && r <= rhi) {
        const InT* mrow = map + (long long)r * P.ld_map + cw;
        if (full_strip) {
#pragma unroll
          for (int k = 0; k < 4; ++k) v[k] = ld_map_val(mrow + 32 * k, P.in_scale);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (cw + 32 * k >= clo && cw + 32 * k <= chi) v[k] = ld_map_val(mrow + 32 * k, P.in_scale);
        }
      }
    }
  };
  float cut[4];
  load_cut(0, cut);

  for (int t = 0; t < nt; ++t) {
    float cut_next[4];
    load_cut(t + 1, cut_next);
    if (work) {
      const int qb = min(t + QL, nq - 1);
      while (waited < qb) {
        ++waited;
        if (!mbar_wait(smem_u32(&bars[waited % NS]), (unsigned)((waited / NS) & 1))) s_fail = 1;
      }
    }
    const int r = R0 + t * kRingSR + warp;
    if (r < R1) {
      unsigned char d[4] = {0, 0, 0, 0};
      float th[4] = {0.f, 0.f, 0.f, 0.f};
      if (work && r >= rlo && r <= rhi) {
        // ring row of each lookup row: slot of stage t, plus the row's stage
        // and row offsets, wrapped once
        auto rrow = [&](int i) {
          int v = sb + coff[i];
          if (v >= RR) v -= RR;
          return ring + v * HCP + x;
        };
        const u64* ra = rrow(0);  // row r - wr - 1 at column cw
        const u64* rb = rrow(1);  // row r + wr
        const u64* rc = rrow(2);  // row r - gr - 1
        const u64* rd = rrow(3);  // row r + gr
        const u64* r1 = rrow(4);  // row r
        const u64* r0 = rrow(5);  // row r - 1
        long long st[4];  // reference statistic in fixed point
        if (kind == RCFAR_CFAR_CA) {
#pragma unroll
          for (int k = 0; k < 4; ++k) st[k] = (long long)ref_sum(ra + 32 * k, rb + 32 * k, rc + 32 * k, rd + 32 * k, wc, gc);
        } else {
          const bool greatest = kind == RCFAR_CFAR_GO;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int o = 32 * k;
            st[k] = (long long)go_so_stat(greatest, ra + o, rb + o, rc + o, rd + o, r1 + o, r0 + o, wc, gc);
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int o = 32 * k;
          const float ts = f32_from_q(st[k]) * kthr;
          th[k] = ts * inv_s;  // T (eq. 2 with A = S_ref / n_ref, or t times a half sum)
          if constexpr (kMapCut) {
            d[k] = cut[k] > th[k];
          } else {
            const u64 qc = (r1[o] + r0[o - 1]) - (r0[o] + r1[o - 1]);
            d[k] = f32_from_q((long long)qc) > ts;
          }
        }
        if (!full_strip) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (cw + 32 * k < clo || cw + 32 * k > chi) {
              d[k] = 0;
              th[k] = 0.f;
            }
        }
      }
      unsigned char* drow = P.det + (long long)r * P.ld_det + cw;
      float* trow = P.thr ? P.thr + (long long)r * P.ld_thr + cw : nullptr;
      if (c0 + kRingW <= cols) {
#pragma unroll
        for (int k = 0; k < 4; ++k) drow[32 * k] = d[k];
        if (trow) {
#pragma unroll
          for (int k = 0; k < 4; ++k) trow[32 * k] = th[k];
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cw + 32 * k < cols) {
            drow[32 * k] = d[k];
            if (trow) trow[32 * k] = th[k];
          }
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) cut[k] = cut_next[k];
    sb += kRingSR;
    if (sb == RR) sb = 0;
    // this warp is done with output stage t (its lookups have returned);
    // the last warp refills slot t % NS with stage t + NS
    if (work && t + NS < nq) {
      __syncwarp();
      unsigned last = 0;
      if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&s_done[t % NS], 1u) == kWarps - 1;
        if (last) {
          s_done[t % NS] = 0;
          __threadfence_block();
        }
      }
      if (__shfl_sync(0xffffffffu, last, 0)) issue(t + NS);
    }
  }
  // every issued stage has completed before the CTA's shared memory is released
  if (work) {
    const int last = min(nq, NS + nt) - 1;
    while (waited < last) {
      ++waited;
      if (!mbar_wait(smem_u32(&bars[waited % NS]), (unsigned)((waited / NS) & 1))) s_fail = 1;
    }
  }
  __syncthreads();
  if (tid == 0 && s_fail && B.status) atomicOr(B.status, kStatusTimeout);
}

// Fused SAT + CFAR (no table in device memory). A CTA owns an inner block of
// rows [R0, R1) x columns [c0, c0 + width) and builds, in shared memory, the
// exact 64-bit fixed-point integral image (eq. 3) of its region: table rows
// R0 - wr - 1 .. R1 - 1 + wr and columns cb - 1 .. cb - 1 + CC - 1, with
// region row 0 and column 0 as the zero origin (cb = c0 - wc, or 0 for a
// strip covering the whole width). A region box sum equals the global
// table's (box sums do not depend on the origin), so S_ref -- 8 lookups,
// eq. 4 on the outer and guard rectangles -- and hence T and the decision are
// bit-identical to the split path's with the same fixed-point scale.
// Steps: quantise the region into shared memory, prefix every row (warp
// scans), prefix every column (one thread per column), then the CUTs.
template <bool kMapCut, typename InT>
__global__ void __launch_bounds__(256) k_sat_cfar_fused(const __grid_constant__ CfarBatch B) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  u64* S = reinterpret_cast<u64*>(smem_raw);
  __shared__ int s_bad;
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &CfarMapDev::item0);
  const CfarMapDev& P = B.m[mi];
  const int local = (int)blockIdx.x - P.item0;
  const int ty = local / P.tiles_x, tx = local - ty * P.tiles_x;
  const int rows = P.rows, cols = P.cols;
  const int R0 = ty * P.run, R1 = min(rows, R0 + P.run);
  const int wr = P.wr, wc = P.wc, gr = P.gr, gc = P.gc;
  const bool full = P.tiles_x == 1 && P.bw >= cols;
  const int c0 = full ? 0 : tx * P.bw;
  const int cw = full ? cols : min(P.bw, cols - c0);  // inner columns
  const int cb = full ? 0 : c0 - wc;                   // table column of region column 1
  const int RR = (R1 - R0) + 2 * wr + 1;
  const int CC = full ? cols + 1 : cw + 2 * wc + 1;
  const int pitch = P.hcp;
  const int rg0 = R0 - wr - 1;  // table row of region row 0 (the origin)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float scalef = ldexpf(1.0f, P.sat_scale);
  const float bound = P.bound;
  const InT* map = reinterpret_cast<const InT*>(P.map);
  if (tid == 0) s_bad = 0;

  // 1. quantised values; the origin row and column and cells outside the map are zero
  bool bad = false;
  for (int idx = tid; idx < RR * CC; idx += 256) {
    const int g = idx / CC, j = idx - g * CC;
    const int r = rg0 + g, c = cb - 1 + j;
    float v = 0.f;
    if (g > 0 && j > 0 && r >= 0 && r < rows && c >= 0 && c < cols) v = ld_map_val(map + (long long)r * P.ld_map + c, P.in_scale);
    bad |= !(fabsf(v) <= bound);
    S[g * pitch + j] = (u64)q_from_f32(v, scalef);
  }
  if (bad) s_bad = 1;
  __syncthreads();
  // 2. row prefixes: a warp per row, 8 consecutive columns per lane (CC <= 256)
  for (int g = warp; g < RR; g += 8) {
    u64* row = S + g * pitch;
    u64 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = 8 * lane + e;
      v[e] = j < CC ? row[j] : 0ull;
    }
#pragma unroll
    for (int e = 1; e < 8; ++e) v[e] += v[e - 1];
    u64 incl = v[7];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const u64 excl = incl - v[7];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = 8 * lane + e;
      if (j < CC) row[j] = v[e] + excl;
    }
  }
  __syncthreads();
  // 3. column prefixes: a thread per column walks down the region
  for (int j = tid; j < CC; j += 256) {
    u64 acc = 0;
#pragma unroll 4
    for (int g = 0; g < RR; ++g) {
      acc += S[g * pitch + j];
      S[g * pitch + j] = acc;
    }
  }
  __syncthreads();
  // 4. the CUTs of the inner block
  int s = P.sat_scale;
  const float inv_s = ldexpf(1.0f, -s);
  const float kthr = P.kthr;
  const int kind = P.kind;
  const int inner = (R1 - R0) * cw;
  for (int idx = tid; idx < inner; idx += 256) {
    const int rr = idx / cw, cc = idx - rr * cw;
    const int r = R0 + rr, c = c0 + cc;
    unsigned char d = 0;
    float th = 0.f;
    if (r >= P.row_lo && r <= P.row_hi && c >= P.cut_lo && c <= P.cut_hi) {
      const int g = r - rg0;       // region row of table row r
      const u64* cutc = S + (c - cb + 1);  // region column of table column c
      const u64* ra = cutc + (g - wr - 1) * pitch;
      const u64* rb = cutc + (g + wr) * pitch;
      const u64* rc = cutc + (g - gr - 1) * pitch;
      const u64* rd = cutc + (g + gr) * pitch;
      const u64* r1 = cutc + g * pitch;
      const u64* r0 = cutc + (g - 1) * pitch;
      const u64 st = kind == RCFAR_CFAR_CA ? ref_sum(ra, rb, rc, rd, wc, gc)
                                           : go_so_stat(kind == RCFAR_CFAR_GO, ra, rb, rc, rd, r1, r0, wc, gc);
      const float ts = f32_from_q((long long)st) * kthr;  // T in fixed-point units
      th = ts * inv_s;
      if constexpr (kMapCut) {
        d = ld_map_val(map + (long long)r * P.ld_map + c, P.in_scale) > th ? 1 : 0;
      } else {
        const u64 qc = (r1[0] + r0[-1]) - (r0[0] + r1[-1]);
        d = f32_from_q((long long)qc) > ts ? 1 : 0;
      }
    }
    P.det[(long long)r * P.ld_det + c] = d;
    if (P.thr) P.thr[(long long)r * P.ld_thr + c] = th;
  }
  __syncthreads();
  if (tid == 0 && s_bad && B.status) atomicOr(B.status, kStatusRange);
}

// One CUT row of the streaming kernel: the lane's columns c = c0 + lane +
// 32 k (k < ncg, c < cend). ra .. r0 point into the ring rows r - wr - 1,
// r + wr, r - gr - 1, r + gr, r, r - 1 at the region column of map column
// c0 + lane. Cell averaging: S_ref from 8 lookups (eq. 4 on the outer
// rectangle minus eq. 4 on the guard rectangle); greatest-of / smallest-of:
// the two half sums from 16. Box sums are taken modulo 2^64 (exact: every
// region sum lies below 2^62).
template <bool kMapCut, bool kHalves, int kCG>
__device__ __forceinline__ void stream_cut_row(const CfarMapDev& P, int ncg, bool all_cut, unsigned cut_mask,
                                               unsigned col_mask, const u64* ra, const u64* rb, const u64* rc,
                                               const u64* rd, const u64* r1, const u64* r0, bool greatest, float kthr,
                                               float inv_s, unsigned char* drow, float* trow, const float* mrow) {
  const int wc = P.wc, gc = P.gc;
  // cut: the CUT's map value (kMapCut; only CUT columns are read, the others may lie past the map's edge)
  auto one = [&](int k, float cut, unsigned char& d, float& th) {
    const int o = 32 * k;
    u64 st;
    if constexpr (!kHalves) {
      const u64 outer = (ra[o - wc - 1] + rb[o + wc]) - (ra[o + wc] + rb[o - wc - 1]);
      const u64 guard = (rc[o - gc - 1] + rd[o + gc]) - (rc[o + gc] + rd[o - gc - 1]);
      st = outer - guard;
    } else {
      // leading half: rows (r - wr - 1, r - 1] minus the guard rows (r - gr - 1, r - 1];
      // lagging half: rows (r, r + wr] minus (r, r + gr]
      const u64 lead = ((ra[o - wc - 1] + r0[o + wc]) - (ra[o + wc] + r0[o - wc - 1])) -
                       ((rc[o - gc - 1] + r0[o + gc]) - (rc[o + gc] + r0[o - gc - 1]));
      const u64 lag = ((r1[o - wc - 1] + rb[o + wc]) - (r1[o + wc] + rb[o - wc - 1])) -
                      ((r1[o - gc - 1] + rd[o + gc]) - (r1[o + gc] + rd[o - gc - 1]));
      st = ((long long)lead > (long long)lag) == greatest ? lead : lag;
    }
    const float ts = f32_from_q((long long)st) * kthr;  // T in fixed-point units
    th = ts * inv_s;
    if constexpr (kMapCut) {
      d = cut > th ? 1 : 0;
    } else {
      const u64 qc = (r1[o] + r0[o - 1]) - (r0[o] + r1[o - 1]);
      d = f32_from_q((long long)qc) > ts ? 1 : 0;
    }
  };
  if (all_cut) {  // every column of the lane is a CUT (uniform over the warp)
    float cutv[kCG];
    if constexpr (kMapCut) {
#pragma unroll
      for (int k = 0; k < kCG; ++k) cutv[k] = __ldg(mrow + 32 * k);
    }
#pragma unroll
    for (int k = 0; k < kCG; ++k) {
      unsigned char d;
      float th;
      one(k, kMapCut ? cutv[k] : 0.f, d, th);
      drow[32 * k] = d;
      if (trow) trow[32 * k] = th;
    }
    return;
  }
#pragma unroll 1
  for (int k = 0; k < ncg; ++k) {
    if (!((col_mask >> k) & 1u)) continue;  // past the strip's last column
    unsigned char d = 0;
    float th = 0.f;
    if ((cut_mask >> k) & 1u) one(k, kMapCut ? __ldg(mrow + 32 * k) : 0.f, d, th);
    drow[32 * k] = d;
    if (trow) trow[32 * k] = th;
  }
}

// Streaming fused SAT + CFAR (float32 maps, no table in device memory). A CTA
// owns the CUT rows [R0, R1) of a strip of columns [c0, c0 + cw) and walks
// the map rows R0 - wr .. R1 - 1 + wr in stages of kStreamKS rows. Its local
// integral image (eq. 3) has its origin (region row 0, region column 0,
// both zero) at table row R0 - wr - 1 and column cb - 1; the last
// kStreamKS + 2 wr + 1 of its rows live in a ring in shared memory (region
// row g in slot g mod RB). Per stage, while cp.async brings the next
// stage's map rows (16-byte copies when the map's rows are 16-byte aligned):
//  (A) warp w quantises row w of the stage and prefixes it across the strip
//      (kE contiguous columns per lane, one warp scan) into the ring; a row
//      whose values all lie below 2^31 in fixed point is quantised with one
//      32-bit conversion per value (the same round-to-nearest-even as the
//      general path);
//  (B) thread j adds each new row's prefix to column j + 1's running sum,
//      which it keeps in a register for the whole run (eq. 3 as
//      S(g, .) = S(g - 1, .) + H(g, .));
//  (C) warp w takes one CUT row whose window is now complete: 8 eq. 4
//      lookups per CUT (16 for greatest-of / smallest-of), T and the
//      decision.
// Box sums do not depend on the origin, and the mod-2^64 wrap of long runs
// cancels in them, so thresholds and decisions are bit-identical to the
// split path's with the same fixed-point scale. kCG: column groups of 32 per
// lane in (C) (4 for strips of kStreamW columns, 8 for whole-width strips).
template <bool kMapCut, int kCG, int kE>
__global__ void __launch_bounds__(kStreamThreads, 2) k_sat_cfar_stream(const __grid_constant__ CfarBatch B) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_bad;
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &CfarMapDev::item0);
  const CfarMapDev& P = B.m[mi];
  const int local = (int)blockIdx.x - P.item0;
  const int ty = local / P.tiles_x, tx = local - ty * P.tiles_x;
  const int rows = P.rows, cols = P.cols;
  const int R0 = ty * P.run, R1 = min(rows, R0 + P.run);
  const int wr = P.wr, wc = P.wc, gr = P.gr;
  const bool full = P.tiles_x == 1 && P.bw >= cols;
  const int c0 = full ? 0 : tx * P.bw;
  const int cw = full ? cols : min(P.bw, cols - c0);
  const int cb = full ? 0 : c0 - wc;          // map column of region column 1
  const int nin = full ? cols : cw + 2 * wc;  // map columns in the region (region columns 1 .. nin)
  const int pitch = P.hcp;                    // u64 per ring row (even, >= nin + 1)
  const int RB = P.ring_rows;                 // >= kStreamKS + 2 wr + 1
  const int ldr = (nin + 6) & ~3;             // floats per staged map row (>= nin + 3, multiple of 4)
  const float* map = reinterpret_cast<const float*>(P.map);
  // 16-byte copies need 16-byte aligned rows; they start at x0 = cb rounded
  // down to a multiple of 4 (so no copy straddles column 0)
  const bool vec = ((reinterpret_cast<uintptr_t>(map) & 15) == 0) && ((P.ld_map & 3) == 0);
  const int xoff = vec ? (cb & 3) : 0;
  const int x0 = cb - xoff;
  u64* ring = reinterpret_cast<u64*>(smem_raw);
  float* raw = reinterpret_cast<float*>(smem_raw + (size_t)RB * pitch * 8);  // 16-byte aligned (pitch even)
  const unsigned raw_a = smem_u32(raw);
  const int ro = R0 - wr - 1;       // table row of region row 0
  const int GT = R1 - R0 + 2 * wr;  // region rows 1 .. GT hold map rows
  const int nst = (GT + kStreamKS - 1) / kStreamKS;
  const int last_cut = R1 - 1 - ro;  // region row of CUT row R1 - 1
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float scalef = ldexpf(1.0f, P.sat_scale);
  const float inv_s = ldexpf(1.0f, -P.sat_scale);
  // |x| below this (as bits) keeps |x 2^s| below 2^31: one 32-bit conversion suffices
  const unsigned fast_bits = __float_as_uint(ldexpf(1.0f, 31 - P.sat_scale));
  const unsigned bound_bits = __float_as_uint(P.bound);  // NaN bit patterns compare above it
  const float kthr = P.kthr;
  const int kind = P.kind;
  const int ncg = (cw + 31) >> 5;
  if (tid == 0) s_bad = 0;
  for (int j = tid; j < pitch; j += kStreamThreads) ring[j] = 0ull;  // region row 0 (slot 0)

  // the lane's CUT columns (fixed for the whole run): which are CUTs, and
  // whether all of them are (then the row's loop has no per-column checks)
  const int cl = c0 + lane;
  unsigned cut_mask = 0, col_mask = 0;  // bit k: column cl + 32 k is a CUT / lies in the strip
  for (int k = 0; k < ncg; ++k) {
    const int c = cl + 32 * k;
    if (c < c0 + cw) col_mask |= 1u << k;
    if (c < c0 + cw && c >= P.cut_lo && c <= P.cut_hi) cut_mask |= 1u << k;
  }
  const bool cols_all = ncg == kCG && cw == 32 * kCG && c0 >= P.cut_lo && c0 + cw - 1 <= P.cut_hi;
  const int jl = c0 - cb + 1 + lane;  // region column of the lane's first CUT column

  // stage t's map rows into raw buffer t & 1: warp w fetches row w
  auto fetch = [&](int t) {
    const int g0 = 1 + t * kStreamKS;
    const int n = min(kStreamKS, GT - g0 + 1);
    if (warp < n) {
      const int r = ro + g0 + warp;
      const bool rok = r >= 0 && r < rows;
      const float* src = map + (long long)(rok ? r : 0) * P.ld_map;
      const unsigned dst = raw_a + (unsigned)(((t & 1) * kStreamKS + warp) * ldr) * 4u;
      if (vec) {
        const int nq = (xoff + nin + 3) >> 2;
        for (int q = lane; q < nq; q += 32) {
          const int cs = x0 + 4 * q;
          const int bytes = (rok && cs >= 0 && cs < cols) ? 4 * min(4, cols - cs) : 0;
          cp_async16_n(dst + 16u * q, bytes ? src + cs : map, bytes);
        }
      } else {
        for (int j = lane; j < nin; j += 32) {
          const int c = cb + j;
          const bool ok = rok && c >= 0 && c < cols;
          cp_async4(dst + 4u * j, ok ? src + c : map, ok);
        }
      }
    }
    cp_async_commit();
  };

  u64 colsum = 0;      // column tid + 1: sum of region rows 1 .. the last built
  unsigned vmax = 0;   // largest |value| (bits) this thread quantised: range check at the end
  int next_cut = wr + 1;  // region row of the next CUT row (row R0)
  int slot0 = 1;          // ring slot of region row g0 (1 + t kStreamKS)
  int cut_slot = (wr + 1) % RB;
  pdl_wait();  // the set-up above overlaps the previous kernel
  fetch(0);
  for (int t = 0; t < nst; ++t) {
    cp_async_wait<0>();
    __syncthreads();  // stage t's rows have landed; the ring rows (A) overwrites are no longer read
    if (t + 1 < nst) fetch(t + 1);
    const int g0 = 1 + t * kStreamKS;
    const int n = min(kStreamKS, GT - g0 + 1);
    // (A) warp w: stage row w quantised and prefixed across the strip (lane l
    // holds region columns 1 + kE l .. kE (l + 1), one warp scan): the row's
    // own prefix H(g, .) goes to the ring (columns past nin are never read)
    if (warp < n) {
      int slot = slot0 + warp;
      if (slot >= RB) slot -= RB;
      u64* hrow = ring + slot * pitch + 1 + kE * lane;
      const float* xr = raw + ((t & 1) * kStreamKS + warp) * ldr + xoff + kE * lane;
      const int lim = nin - kE * lane;  // this lane's columns inside the region
      float x[kE];
      unsigned m = 0;
#pragma unroll
      for (int e = 0; e < kE; ++e) {
        x[e] = e < lim ? xr[e] : 0.f;
        m = max(m, __float_as_uint(x[e]) & 0x7fffffffu);
      }
      vmax = max(vmax, m);
      u64 v[kE];
      if (__all_sync(0xffffffffu, m < fast_bits)) {
#pragma unroll
        for (int e = 0; e < kE; ++e) v[e] = (u64)(long long)__float2int_rn(x[e] * scalef);
      } else {
#pragma unroll
        for (int e = 0; e < kE; ++e) v[e] = (u64)q_from_f32(x[e], scalef);
      }
#pragma unroll
      for (int e = 1; e < kE; ++e) v[e] += v[e - 1];
      u64 incl = v[kE - 1];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const u64 excl = incl - v[kE - 1];
#pragma unroll
      for (int e = 0; e < kE; ++e) hrow[e] = v[e] + excl;
      if (lane == 0) hrow[-1] = 0ull;  // region column 0
    }
    __syncthreads();
    // (B) eq. 3 down the columns: S(g, .) = S(g - 1, .) + H(g, .); thread j
    // keeps column j + 1's running sum in a register for the whole run. The
    // stage's rows occupy slots slot0 .. slot0 + n - 1 (mod RB): every load
    // is issued before the sums are formed.
    if (tid < nin) {
      // the stage's rows are two straight runs of the ring: slots slot0 .. RB - 1,
      // then (after the wrap) 0 ..; row i lies at (i < n1 ? p0 : p1) + i * pitch
      u64* const p0 = ring + slot0 * pitch + 1 + tid;
      u64* const p1 = p0 - RB * pitch;
      const int n1 = RB - slot0;
      u64 hv[kStreamKS];
#pragma unroll
      for (int i = 0; i < kStreamKS; ++i) hv[i] = i < n ? (i < n1 ? p0 : p1)[i * pitch] : 0ull;
#pragma unroll
      for (int i = 0; i < kStreamKS; ++i) {
        colsum += hv[i];
        if (i < n) (i < n1 ? p0 : p1)[i * pitch] = colsum;
      }
    }
    __syncthreads();
    // (C) CUT rows whose windows are complete: region rows next_cut .. hi
    const int hi = min(g0 + n - 1 - wr, last_cut);
    const int cnt = hi - next_cut + 1;  // <= kStreamKS
    if (warp < cnt) {
      int sg = cut_slot + warp;
      if (sg >= RB) sg -= RB;
      // ring rows of region rows g + off at column jl (0 <= sg < RB, |off| <= wr + 1 < RB)
      auto row_at = [&](int off) {
        int x = sg + off;
        if (x < 0) x += RB;
        if (x >= RB) x -= RB;
        return ring + x * pitch + jl;
      };
      const int r = ro + next_cut + warp;
      const bool row_cut = r >= P.row_lo && r <= P.row_hi;
      unsigned char* drow = P.det + (long long)r * P.ld_det + cl;
      float* trow = P.thr ? P.thr + (long long)r * P.ld_thr + cl : nullptr;
      const float* mrow = map + (long long)r * P.ld_map + cl;
      const u64 *ra = row_at(-wr - 1), *rb = row_at(wr), *rc = row_at(-gr - 1), *rd = row_at(gr);
      const u64 *r1 = row_at(0), *r0 = row_at(-1);
      const unsigned mask = row_cut ? cut_mask : 0u;
      const bool all = row_cut && cols_all;
      if (kind == RCFAR_CFAR_CA)
        stream_cut_row<kMapCut, false, kCG>(P, ncg, all, mask, col_mask, ra, rb, rc, rd, r1, r0, false, kthr, inv_s,
                                            drow, trow, mrow);
      else
        stream_cut_row<kMapCut, true, kCG>(P, ncg, all, mask, col_mask, ra, rb, rc, rd, r1, r0,
                                           kind == RCFAR_CFAR_GO, kthr, inv_s, drow, trow, mrow);
    }
    if (cnt > 0) {
      next_cut += cnt;
      cut_slot += cnt;
      if (cut_slot >= RB) cut_slot -= RB;
    }
    slot0 += kStreamKS;
    if (slot0 >= RB) slot0 -= RB;
  }
  if (vmax > bound_bits) s_bad = 1;
  __syncthreads();
  if (tid == 0 && s_bad && B.status) atomicOr(B.status, kStatusRange);
}

// The streaming kernel fed by the tensor memory accelerator (float32 maps
// whose rows start on 16-byte boundaries, strips of kStreamW CUT columns).
// The decomposition is k_sat_cfar_stream's -- per stage of kStreamKS rows:
// (A) warp w quantises and prefixes stage row w, kE contiguous columns per
// lane and one warp scan; (B) thread j adds the new rows' prefixes to column
// j + 1's running sum (eq. 3); (C) warp w takes one complete CUT row, 8 eq.
// 4 lookups per CUT (16 for greatest-of / smallest-of) -- with these
// differences:
//  * one thread brings each stage's map rows as one 2-D box (kStreamKS rows
//    x 32 kE columns from the strip's first halo column rounded down to a
//    multiple of 4), one stage ahead, completing on an mbarrier; rows and
//    columns outside the map arrive as zeros. Region column r >= 1 is map
//    column x0 + r - 1;
//  * ring rows are indexed so that region column r lives at index r + 1:
//    index 1 is the zero column (written once), and every lane's kE
//    columns start on a 16-byte boundary -- the prefix is stored with
//    16-byte stores, which for kE = 6 (lane chunks 48 bytes apart) are free
//    of bank conflicts;
//  * every shared-memory access indexes a typed shared array, and each row
//    offset is formed once per row.
// Thresholds and decisions are bit-identical to k_sat_cfar_stream's and the
// split path's (same quantisation, box sums exact modulo 2^64).
template <bool kMapCut, int kE>
__global__ void __launch_bounds__(kStreamThreads, 2) k_sat_cfar_stream_tma(const __grid_constant__ CfarTmaParams B) {
  constexpr int KS = kStreamKS;
  constexpr int RW = 32 * kE;  // floats per staged row (the box width)
  constexpr int kCG = kStreamW / 32;
  static_assert(kE % 2 == 0, "lanes read and write their columns in pairs");
  pdl_trigger();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar_full[2];
  __shared__ int s_bad, s_fail, s_issued, s_consumed;
  const CfarMapDev& P = B.m;
  const int local = (int)blockIdx.x;
  const int ty = local / P.tiles_x, tx = local - ty * P.tiles_x;
  const int rows = P.rows, cols = P.cols;
  const int R0 = ty * P.run, R1 = min(rows, R0 + P.run);
  const int wr = P.wr, wc = P.wc, gr = P.gr, gc = P.gc;
  const int c0 = tx * P.bw;
  const int cw = min(P.bw, cols - c0);
  const int x0 = (c0 - wc) & ~3;      // map column of region column 1 (16-byte aligned)
  const int xoff = c0 - wc - x0;      // 0 .. 3
  const int nb = cw + 2 * wc + xoff;  // region columns the lookups read: 1 .. nb
  const int pitch = P.hcp;            // u64 per ring row (32 kE + 2)
  const int RB = P.ring_rows;         // >= KS + 2 wr + 1
  u64* const ring = reinterpret_cast<u64*>(smem_raw);
  // staged boxes: 2 x KS x RW floats after the ring, on a 128-byte boundary
  float* const raw = reinterpret_cast<float*>(smem_raw + (((smem_u32(smem_raw) + (unsigned)RB * pitch * 8 + 127u) & ~127u) -
                                                         smem_u32(smem_raw)));
  const int ro = R0 - wr - 1;         // map row of region row 0
  const int GT = R1 - R0 + 2 * wr;    // region rows 1 .. GT hold map rows
  const int nst = (GT + KS - 1) / KS;
  const int last_cut = R1 - 1 - ro;   // region row of CUT row R1 - 1
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float scalef = ldexpf(1.0f, P.sat_scale);
  const float inv_s = ldexpf(1.0f, -P.sat_scale);
  const unsigned fast_bits = __float_as_uint(ldexpf(1.0f, 31 - P.sat_scale));
  const unsigned bound_bits = __float_as_uint(P.bound);
  const float kthr = P.kthr;
  const int kind = P.kind;
  const float* map = reinterpret_cast<const float*>(P.map);
  const unsigned long long tmap = reinterpret_cast<unsigned long long>(&B.tm);
  if (tid == 0) {
    s_bad = 0;
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    mbar_init(smem_u32(&bar_full[0]), 1);
    mbar_init(smem_u32(&bar_full[1]), 1);
    mbar_init_fence();
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
  }
  for (int j = tid; j < pitch; j += kStreamThreads) ring[j] = 0ull;  // region row 0 (slot 0)
  for (int r = 1 + tid; r < RB; r += kStreamThreads) ring[r * pitch + 1] = 0ull;  // region column 0
  const int ncg = (cw + 31) >> 5;
  const int cl = c0 + lane;
  unsigned cut_mask = 0, col_mask = 0;  // bit k: column cl + 32 k is a CUT / lies in the strip
  for (int k = 0; k < ncg; ++k) {
    const int c = cl + 32 * k;
    if (c < c0 + cw) col_mask |= 1u << k;
    if (c < c0 + cw && c >= P.cut_lo && c <= P.cut_hi) cut_mask |= 1u << k;
  }
  const bool cols_all = cw == kStreamW && c0 >= P.cut_lo && c0 + cw - 1 <= P.cut_hi;
  const int jl = c0 - x0 + 2 + lane;  // ring index of the lane's first CUT column
  const unsigned tx_bytes = (unsigned)(KS * RW * 4);
  __syncthreads();  // barriers initialised, ring zeroed

  // stage t's box into raw buffer t & 1 (one thread)
  auto issue = [&](int t) {
    const unsigned bar = smem_u32(&bar_full[t & 1]);
    mbar_arrive_expect_tx(bar, tx_bytes);
    tma_load_2d(smem_u32(raw + (t & 1) * KS * RW), tmap, x0, ro + 1 + t * KS, bar);
    s_issued = t + 1;
  };

  u64 colsum = 0;
  unsigned vmax = 0;
  int next_cut = wr + 1;
  int slot0 = 1;
  int cut_slot = (wr + 1) % RB;
  // (C) state carried from stage to stage: the warp's last CUT row, the ring
  // indices of its rows r - wr - 1, r + wr, r - gr - 1, r + gr, r, r - 1 at
  // the lane's first CUT column, and its output / map row pointers
  int pr = -(1 << 30);
  int ba = 0, bb = 0, bc = 0, bd = 0, b1 = 0, b0 = 0;
  unsigned char* drow = nullptr;
  float* trow = nullptr;
  const float* mrow = nullptr;
  pdl_wait();  // the map may be the previous kernel's output
  if (tid == 0) issue(0);
  for (int t = 0; t < nst; ++t) {
    if (tid == 0 && t + 1 < nst && !s_fail) issue(t + 1);  // its buffer was last read by stage t - 1's (A)
    const int g0 = 1 + t * KS;
    const int n = min(KS, GT - g0 + 1);
    // (A) stage row w: quantise, prefix across the strip, store the row's own prefix H(g, .)
    if (warp < n) {
      // after a failed wait no further boxes are issued, so later stages do not wait
      if (*(volatile int*)&s_fail || !mbar_wait(smem_u32(&bar_full[t & 1]), (unsigned)((t >> 1) & 1)))
        s_fail = 1;
      else if (tid == 0)
        s_consumed = t + 1;
      int slot = slot0 + warp;
      if (slot >= RB) slot -= RB;
      const float2* xr = reinterpret_cast<const float2*>(raw + ((t & 1) * KS + warp) * RW + kE * lane);
      float x[kE];
      unsigned m = 0;
#pragma unroll
      for (int e = 0; e < kE / 2; ++e) {
        const float2 v = xr[e];
        x[2 * e] = v.x;
        x[2 * e + 1] = v.y;
        m = __vimax3_u32(m, __float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu);
      }
      vmax = max(vmax, m);
      u64 v[kE];
      if (__all_sync(0xffffffffu, m < fast_bits)) {
#pragma unroll
        for (int e = 0; e < kE; ++e) v[e] = (u64)(long long)__float2int_rn(x[e] * scalef);
      } else {
#pragma unroll
        for (int e = 0; e < kE; ++e) v[e] = (u64)q_from_f32(x[e], scalef);
      }
#pragma unroll
      for (int e = 1; e < kE; ++e) v[e] += v[e - 1];
      u64 incl = v[kE - 1];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const u64 excl = incl - v[kE - 1];
      ulonglong2* hrow = reinterpret_cast<ulonglong2*>(ring + slot * pitch + 2 + kE * lane);
#pragma unroll
      for (int e = 0; e < kE / 2; ++e) hrow[e] = make_ulonglong2(v[2 * e] + excl, v[2 * e + 1] + excl);
    }
    __syncthreads();
    // (B) S(g, .) = S(g - 1, .) + H(g, .) for region column tid + 1 (ring index tid + 2);
    // the stage's rows are slots slot0 .. RB - 1, then 0 .. after the wrap
    if (tid < nb) {
      const int a0 = slot0 * pitch + 2 + tid;
      const int n1 = RB - slot0;
      const int wrap = RB * pitch;
      if (n == KS) {
        // two batches of KS / 2 rows: each batch's loads are issued before its sums
#pragma unroll
        for (int i0 = 0; i0 < KS; i0 += KS / 2) {
          u64 hv[KS / 2];
#pragma unroll
          for (int i = 0; i < KS / 2; ++i) hv[i] = ring[a0 + (i0 + i) * pitch - (i0 + i >= n1 ? wrap : 0)];
#pragma unroll
          for (int i = 0; i < KS / 2; ++i) {
            colsum += hv[i];
            ring[a0 + (i0 + i) * pitch - (i0 + i >= n1 ? wrap : 0)] = colsum;
          }
        }
      } else {
        for (int i = 0; i < n; ++i) {
          const int a = a0 + i * pitch - (i >= n1 ? wrap : 0);
          colsum += ring[a];
          ring[a] = colsum;
        }
      }
    }
    __syncthreads();
    // (C) CUT rows whose windows are complete: region rows next_cut .. hi
    const int hi = min(g0 + n - 1 - wr, last_cut);
    const int cnt = hi - next_cut + 1;  // <= KS
    if (warp < cnt) {
      const int r = ro + next_cut + warp;
      if (r == pr + KS) {  // the row KS below the last one: every row offset moves KS ring rows on
        const int step = KS * pitch, size = RB * pitch;
        ba += step; ba -= ba >= size ? size : 0;
        bb += step; bb -= bb >= size ? size : 0;
        bc += step; bc -= bc >= size ? size : 0;
        bd += step; bd -= bd >= size ? size : 0;
        b1 += step; b1 -= b1 >= size ? size : 0;
        b0 += step; b0 -= b0 >= size ? size : 0;
        drow += (long long)KS * P.ld_det;
        mrow += (long long)KS * P.ld_map;
        if (trow) trow += (long long)KS * P.ld_thr;
      } else {
        int sg = cut_slot + warp;
        if (sg >= RB) sg -= RB;
        auto rix = [&](int off) {  // ring index of region row (CUT row + off) at the lane's first CUT column
          int x = sg + off;
          if (x < 0) x += RB;
          if (x >= RB) x -= RB;
          return x * pitch + jl;
        };
        ba = rix(-wr - 1);
        bb = rix(wr);
        bc = rix(-gr - 1);
        bd = rix(gr);
        b1 = rix(0);
        b0 = rix(-1);
        drow = P.det + (long long)r * P.ld_det + cl;
        trow = P.thr ? P.thr + (long long)r * P.ld_thr + cl : nullptr;
        mrow = map + (long long)r * P.ld_map + cl;
      }
      pr = r;
      const bool row_cut = r >= P.row_lo && r <= P.row_hi;
      const unsigned mask = row_cut ? cut_mask : 0u;
      const bool all = row_cut && cols_all;
      const bool halves = kind != RCFAR_CFAR_CA;
      const bool greatest = kind == RCFAR_CFAR_GO;
      // the eight corners of eq. 4 (outer and guard rectangles) relative to the lane's CUT column
      const int al = ba - wc - 1, ar = ba + wc, bl = bb - wc - 1, br = bb + wc;
      const int cL = bc - gc - 1, cR = bc + gc, dL = bd - gc - 1, dR = bd + gc;
      // T and the decision of the lane's CUT k (o = 32 k columns along)
      auto one = [&](int o, float cut, unsigned char& d, float& th) {
        u64 st;
        if (!halves) {
          const u64 outer = (ring[al + o] + ring[br + o]) - (ring[ar + o] + ring[bl + o]);
          const u64 guard = (ring[cL + o] + ring[dR + o]) - (ring[cR + o] + ring[dL + o]);
          st = outer - guard;
        } else {
          // leading half: rows (r - wr - 1, r - 1] minus the guard rows (r - gr - 1, r - 1];
          // lagging half: rows (r, r + wr] minus (r, r + gr]
          const u64 lead = ((ring[al + o] + ring[b0 + wc + o]) - (ring[ar + o] + ring[b0 - wc - 1 + o])) -
                           ((ring[cL + o] + ring[b0 + gc + o]) - (ring[cR + o] + ring[b0 - gc - 1 + o]));
          const u64 lag = ((ring[b1 - wc - 1 + o] + ring[br + o]) - (ring[b1 + wc + o] + ring[bl + o])) -
                          ((ring[b1 - gc - 1 + o] + ring[dR + o]) - (ring[b1 + gc + o] + ring[dL + o]));
          st = ((long long)lead > (long long)lag) == greatest ? lead : lag;
        }
        const float ts = f32_from_q((long long)st) * kthr;  // T in fixed-point units
        th = ts * inv_s;
        if constexpr (kMapCut) {
          d = cut > th ? 1 : 0;
        } else {
          const u64 qc = (ring[b1 + o] + ring[b0 - 1 + o]) - (ring[b0 + o] + ring[b1 - 1 + o]);
          d = f32_from_q((long long)qc) > ts ? 1 : 0;
        }
      };
      if (all) {
        float cutv[kCG];
        if constexpr (kMapCut) {
#pragma unroll
          for (int k = 0; k < kCG; ++k) cutv[k] = __ldg(mrow + 32 * k);
        }
#pragma unroll
        for (int k = 0; k < kCG; ++k) {
          unsigned char d;
          float th;
          one(32 * k, kMapCut ? cutv[k] : 0.f, d, th);
          drow[32 * k] = d;
          if (trow) trow[32 * k] = th;
        }
      } else {
#pragma unroll 1
        for (int k = 0; k < ncg; ++k) {
          if (!((col_mask >> k) & 1u)) continue;  // past the strip's last column
          unsigned char d = 0;
          float th = 0.f;
          if ((mask >> k) & 1u) one(32 * k, kMapCut ? __ldg(mrow + 32 * k) : 0.f, d, th);
          drow[32 * k] = d;
          if (trow) trow[32 * k] = th;
        }
      }
    }
    if (cnt > 0) {
      next_cut += cnt;
      cut_slot += cnt;
      if (cut_slot >= RB) cut_slot -= RB;
    }
    slot0 += KS;
    if (slot0 >= RB) slot0 -= RB;
    __syncthreads();  // (C) has read the ring rows the next stage's (A) overwrites
  }
  if (vmax > bound_bits) s_bad = 1;
  // after a failed wait, boxes issued but never waited for land before the shared memory is released
  if (tid == 0)
    for (int t = s_consumed; t < s_issued; ++t) mbar_wait(smem_u32(&bar_full[t & 1]), (unsigned)((t >> 1) & 1));
  __syncthreads();
  if (tid == 0 && B.status) {
    if (s_bad) atomicOr(B.status, kStatusRange);
    if (s_fail) atomicOr(B.status, kStatusTimeout);
  }
}

// Ordered-statistic CFAR. A CTA holds the map tile of kOsRows x 32 CUTs plus
// the window halo in shared memory, and the offsets of the n_ref training
// cells (outer box minus guard box) relative to the CUT. Warp w takes CUT row
// w, one CUT at a time: lane l loads training cells l, l + 32, ... as
// order-preserving 32-bit keys into registers (kNK per lane), and the warp
// finds the k-th smallest key by building it bit by bit from the top: a bit
// is set when fewer than k keys lie below the key with that bit set
// (per-lane counts, one warp reduction per bit; bits above the first one in
// which the window's smallest and largest keys differ are taken from them).
// T = alpha_os X_(k); lane c keeps column c's result and the warp stores
// its row of decisions at the end.
__device__ __forceinline__ unsigned os_key(float v) {
  const unsigned b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float os_value(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

template <int kNK>
__global__ void __launch_bounds__(256, 2) k_cfar_os(const __grid_constant__ CfarBatch B) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int mi = find_item(B.m, B.n, (int)blockIdx.x, &CfarMapDev::item0);
  const CfarMapDev& P = B.m[mi];
  const int local = (int)blockIdx.x - P.item0;
  const int ty = local / P.tiles_x, tx = local - ty * P.tiles_x;
  const int r0 = ty * kOsRows, c0 = tx * 32;
  const int wr = P.wr, wc = P.wc, gr = P.gr, gc = P.gc;
  const int HR = kOsRows + 2 * wr, HC = 32 + 2 * wc;
  const int nref = P.n_ref, kr = P.os_rank;
  float* X = reinterpret_cast<float*>(smem_raw);
  int* offs = reinterpret_cast<int*>(X + HR * HC);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* map = reinterpret_cast<const float*>(P.map);
  for (int i = tid; i < HR * HC; i += 256) {
    const int hr = i / HC, hc = i - hr * HC;
    const int r = r0 - wr + hr, c = c0 - wc + hc;
    X[i] = (r >= 0 && r < P.rows && c >= 0 && c < P.cols) ? __ldg(map + (long long)r * P.ld_map + c) : 0.f;
  }
  // training cell i -> (dr, dc): rows above the guard box (full width), the
  // guard rows (left and right of the guard box), rows below
  {
    const int W = 2 * wc + 1, side = wc - gc;
    const int top = (wr - gr) * W, mid = (2 * gr + 1) * 2 * side;
    for (int i = tid; i < nref; i += 256) {
      int dr, dc;
      if (i < top) {
        dr = -wr + i / W;
        dc = -wc + i % W;
      } else if (i < top + mid) {
        const int j = i - top;
        dr = -gr + j / (2 * side);
        const int q = j % (2 * side);
        dc = q < side ? -wc + q : gc + 1 + (q - side);
      } else {
        const int j = i - top - mid;
        dr = gr + 1 + j / W;
        dc = -wc + j % W;
      }
      offs[i] = dr * HC + dc;
    }
  }
  __syncthreads();
  const int r = r0 + warp;
  unsigned char my_d = 0;
  float my_t = 0.f;
  if (r < P.rows && r >= P.row_lo && r <= P.row_hi) {
    const float alpha = P.kthr;
    for (int cc = 0; cc < 32; ++cc) {
      const int c = c0 + cc;
      if (c < P.cut_lo || c > P.cut_hi || c >= P.cols) continue;  // uniform over the warp
      const float* ctr = X + (warp + wr) * HC + (cc + wc);
      unsigned key[kNK];
      unsigned mn = 0xffffffffu, mx = 0u;
#pragma unroll
      for (int m = 0; m < kNK; ++m) {
        const int i = lane + 32 * m;
        key[m] = i < nref ? os_key(ctr[offs[i]]) : 0xffffffffu;
        if (i < nref) {
          mn = min(mn, key[m]);
          mx = max(mx, key[m]);
        }
      }
      mn = __reduce_min_sync(0xffffffffu, mn);
      mx = __reduce_max_sync(0xffffffffu, mx);
      // bits above the highest differing bit of mn and mx are common to every key
      const unsigned diff = mn ^ mx;
      const int top = diff ? 31 - __clz(diff) : -1;
      unsigned t = top >= 0 ? (mn & ~((2u << top) - 1u)) : mn;
      if (top == 31) t = 0u;
      for (int b = top; b >= 0; --b) {
        const unsigned cand = t | (1u << b);
        int n0 = 0, n1 = 0, n2 = 0, n3 = 0;
#pragma unroll
        for (int m = 0; m < kNK; m += 4) {
          n0 += key[m] < cand;
          if (m + 1 < kNK) n1 += key[m + 1] < cand;
          if (m + 2 < kNK) n2 += key[m + 2] < cand;
          if (m + 3 < kNK) n3 += key[m + 3] < cand;
        }
        const int below = (int)__reduce_add_sync(0xffffffffu, (unsigned)((n0 + n1) + (n2 + n3)));
        if (below < kr) t = cand;
      }
      const float T = alpha * os_value(t);
      if (lane == cc) {
        my_t = T;
        my_d = ctr[0] > T ? 1 : 0;
      }
    }
  }
  const int c = c0 + lane;
  if (r < P.rows && c < P.cols) {
    P.det[(long long)r * P.ld_det + c] = my_d;
    if (P.thr) P.thr[(long long)r * P.ld_thr + c] = my_t;
  }
}

__global__ void __launch_bounds__(256) k_cfar_direct(const __grid_constant__ CfarMapDev P) {
  pdl_trigger();
  pdl_wait();
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
      // cell averaging: every training cell; greatest-of / smallest-of: the
      // rows above the CUT (leading half) and below it (lagging half) apart
      float sum = 0.f, lead = 0.f, lag = 0.f;
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
        if (dr < 0) lead += rs;
        if (dr > 0) lag += rs;
      }
      const float stat = P.kind == RCFAR_CFAR_CA ? sum
                         : P.kind == RCFAR_CFAR_GO ? fmaxf(lead, lag) : fminf(lead, lag);
      t = stat * P.kthr;
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
  return launch_pdl(fn, blocks, 256, smem, s, b);
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


bool cfar_ring_plan(int wr, int wc, size_t smem_cap, int* ring_rows, int* hcp) {
  const int h = kRingW + 2 * wc + 2;  // strip + halo, rounded to an even count
  const int ql = (2 * wr + kRingSR) / kRingSR;
  // ring: as many stages as fit (at most kRingMaxStages, and at most 8
  // beyond the ones an output stage reads); at least one stage in flight
  int ns = (int)((smem_cap - kRingBarBytes) / ((size_t)kRingSR * h * 8));
  ns = std::min(ns, std::min(kRingMaxStages, ql + 1 + 8));
  if (ns < ql + 2) return false;
  *ring_rows = ns * kRingSR;
  *hcp = h;
  return true;
}

size_t cfar_ring_smem(int ring_rows, int hcp) { return (size_t)kRingBarBytes + (size_t)ring_rows * hcp * 8; }

int cfar_ring_slots(size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 152;
  const void* fn = reinterpret_cast<const void*>(k_cfar_ring<true, float>);
  if (ensure_smem(fn, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cfar_ring<true, float>, kRingThreads, smem) != cudaSuccess ||
      per < 1)
    per = 1;
  return sms * per;
}

// Runs per strip chosen to balance the waves of resident CTAs (slots) against
// the 2 wr + 1 halo rows each run streams in before its first output row.
int cfar_ring_geometry(CfarMapDev& P, int rows, int cols, int ring_rows, int hcp, int slots) {
  P.bw = kRingW;
  P.bh = kRingSR;
  P.tiles_x = (cols + kRingW - 1) / kRingW;
  P.ring_rows = ring_rows;
  P.hcp = hcp;
  const int max_runs = std::max(1, (rows + kRingSR - 1) / kRingSR);
  long long best = -1;
  int best_run = kRingSR;
  for (int n = 1; n <= max_runs; ++n) {
    const int run = ((rows + n - 1) / n + kRingSR - 1) / kRingSR * kRingSR;
    const int runs = (rows + run - 1) / run;
    const long long ctas = (long long)P.tiles_x * runs;
    const long long waves = (ctas + slots - 1) / slots;
    const long long cost = waves * (run + 2 * P.wr + 1 + 8);  // 8: per-CTA set-up, in row units
    if (best < 0 || cost < best) {
      best = cost;
      best_run = run;
    }
    if (run == kRingSR) break;
  }
  P.run = best_run;
  return P.tiles_x * ((rows + best_run - 1) / best_run);
}

template <bool kMapCut, typename InT>
static cudaError_t launch_ring_t(const CfarBatch& b, int blocks, size_t smem, cudaStream_t s) {
  auto fn = k_cfar_ring<kMapCut, InT>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(fn, blocks, kRingThreads, smem, s, b);
}

cudaError_t launch_cfar_ring(const CfarBatch& b, bool map_cut, int dtype, int blocks, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (!map_cut) return launch_ring_t<false, float>(b, blocks, smem, s);
  return dtype == RCFAR_MAP_F16 ? launch_ring_t<true, __half>(b, blocks, smem, s)
                                : launch_ring_t<true, float>(b, blocks, smem, s);
}


bool cfar_fused_plan(int rows, int cols, int wr, int wc, size_t smem_cap, int* run, int* bw, int* pitch,
                     size_t* smem) {
  const bool full = cols + 1 <= kFusedMaxCols;
  const int w = full ? cols : kRingW;
  const int cc = full ? cols + 1 : kRingW + 2 * wc + 1;
  if (cc > kFusedMaxCols) return false;
  const int p = (cc + 1) & ~1;
  // runs short enough for about two CTAs per SM (the phases of one CTA run
  // in sequence, so the map's parallelism comes from its CTA count), long
  // enough to amortise the 2 wr + 1 halo rows; multiples of 8, <= 64, and
  // the region must fit
  const long long strips = (cols + w - 1) / w;
  int r = (int)std::min<long long>(64, std::max<long long>(8, ((long long)rows * strips / (2 * 152) + 7) / 8 * 8));
  while (r >= 8 && (size_t)(r + 2 * wr + 1) * p * 8 > smem_cap) r -= 8;
  if (r < 8) return false;
  *run = r;
  *bw = w;
  *pitch = p;
  *smem = (size_t)(r + 2 * wr + 1) * p * 8;
  return true;
}

int cfar_fused_geometry(CfarMapDev& P, int rows, int cols, int run, int bw, int pitch) {
  P.run = run;
  P.bw = bw;
  P.bh = 0;
  P.hcp = pitch;
  P.tiles_x = (cols + bw - 1) / bw;
  return P.tiles_x * ((rows + run - 1) / run);
}

template <bool kMapCut, typename InT>
static cudaError_t launch_fused_t(const CfarBatch& b, int blocks, size_t smem, cudaStream_t s) {
  auto fn = k_sat_cfar_fused<kMapCut, InT>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(fn, blocks, 256, smem, s, b);
}

cudaError_t launch_cfar_fused(const CfarBatch& b, bool map_cut, int dtype, int blocks, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const bool h = dtype == RCFAR_MAP_F16;
  if (map_cut) return h ? launch_fused_t<true, __half>(b, blocks, smem, s) : launch_fused_t<true, float>(b, blocks, smem, s);
  return h ? launch_fused_t<false, __half>(b, blocks, smem, s) : launch_fused_t<false, float>(b, blocks, smem, s);
}

static int stream_nin(int cols, int wc) { return cols + 1 <= kFusedMaxCols ? cols : kStreamW + 2 * wc; }

int stream_e_of(int rows, int cols, int wc) {
  if (rows <= 0 || cols <= 0) return 0;
  const int nin = stream_nin(cols, wc);
  if (nin + 1 > kFusedMaxCols) return 0;
  const int e = (nin + 31) / 32;
  return e <= 5 ? 5 : e == 6 ? 6 : 8;
}

bool cfar_stream_plan(int rows, int cols, int wr, int wc, size_t smem_cap, int sm_share, int e_min,
                      StreamPlan* out) {
  int e = stream_e_of(rows, cols, wc);
  if (e == 0) return false;
  e = std::max(e, e_min);
  if (e != 5 && e != 6 && e != 8) e = 8;
  const bool full = cols + 1 <= kFusedMaxCols;
  const int w = full ? cols : kStreamW;
  const int nin = stream_nin(cols, wc);
  const int pitch = 32 * e + 2;
  const int ldr = (nin + 6) & ~3;
  const int rb = kStreamKS + 2 * wr + 1;
  const size_t smem = (size_t)rb * pitch * 8 + (size_t)2 * kStreamKS * ldr * 4;
  if (smem > smem_cap) return false;
  // two CTAs per SM when their shared memory fits (228 KB per SM, 1 KB reserved per CTA)
  const int per_sm = 2 * (smem + 1024 + 64) <= 228 * 1024 ? 2 : 1;
  const long long slots = (long long)std::max(1, sm_share) * per_sm;
  const long long strips = full ? 1 : (cols + w - 1) / w;
  int best_run = rows;
  long long best = -1;
  // candidate runs: 1..16 and multiples of 8; cost = waves x stages per CTA
  for (int run = 1; run <= rows + 7; run = run < 16 ? run + 1 : run + 8) {
    const int rr = std::min(run, rows);
    const long long ctas = strips * ((rows + rr - 1) / rr);
    const long long waves = (ctas + slots - 1) / slots;
    const long long stages = (rr + 2 * wr + kStreamKS - 1) / kStreamKS;
    const long long cost = waves * stages;
    if (best < 0 || cost < best || (cost == best && rr > best_run)) {
      best = cost;
      best_run = rr;
    }
    if (rr == rows) break;
  }
  out->run = best_run;
  out->bw = w;
  out->pitch = pitch;
  out->ring_rows = rb;
  out->e = e;
  out->smem = smem;
  out->ctas = (int)(strips * ((rows + best_run - 1) / best_run));
  return true;
}

int cfar_stream_geometry(CfarMapDev& P, int rows, int cols, const StreamPlan& sp) {
  P.run = sp.run;
  P.bw = sp.bw;
  P.bh = 0;
  P.hcp = sp.pitch;
  P.ring_rows = sp.ring_rows;
  P.tiles_x = (cols + sp.bw - 1) / sp.bw;
  return P.tiles_x * ((rows + sp.run - 1) / sp.run);
}

template <bool kMapCut, int kCG, int kE>
static cudaError_t launch_stream_t(const CfarBatch& b, int blocks, size_t smem, cudaStream_t s) {
  auto fn = k_sat_cfar_stream<kMapCut, kCG, kE>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(fn, blocks, kStreamThreads, smem, s, b);
}

template <int kCG, int kE>
static cudaError_t launch_stream_ce(const CfarBatch& b, bool map_cut, int blocks, size_t smem, cudaStream_t s) {
  return map_cut ? launch_stream_t<true, kCG, kE>(b, blocks, smem, s) : launch_stream_t<false, kCG, kE>(b, blocks, smem, s);
}

cudaError_t launch_cfar_stream(const CfarBatch& b, bool map_cut, int e, int blocks, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  // 8 column groups per lane only when some item is one whole-width strip wider than 128 columns
  bool wide = false;
  for (int i = 0; i < b.n; ++i) wide = wide || (b.m[i].tiles_x == 1 && b.m[i].cols > kStreamW);
  if (e == 5) return wide ? launch_stream_ce<8, 5>(b, map_cut, blocks, smem, s) : launch_stream_ce<4, 5>(b, map_cut, blocks, smem, s);
  if (e == 6) return wide ? launch_stream_ce<8, 6>(b, map_cut, blocks, smem, s) : launch_stream_ce<4, 6>(b, map_cut, blocks, smem, s);
  return wide ? launch_stream_ce<8, 8>(b, map_cut, blocks, smem, s) : launch_stream_ce<4, 8>(b, map_cut, blocks, smem, s);
}

bool cfar_stream_tma_plan(int rows, int cols, int wr, int wc, size_t smem_cap, int sm_share, StreamPlan* out) {
  if (rows <= 0 || cols + 1 <= kFusedMaxCols) return false;
  const int need = kStreamW + 2 * wc + 3;  // strip, halo and the alignment of its first column
  const int e = need <= 32 * 6 ? 6 : need <= 32 * 8 ? 8 : 0;
  if (e == 0) return false;
  const int pitch = 32 * e + 2;
  const int rb = kStreamKS + 2 * wr + 1;
  const size_t smem = (size_t)rb * pitch * 8 + 128 + (size_t)2 * kStreamKS * 32 * e * 4;  // + alignment of the boxes
  if (smem > smem_cap) return false;
  const int per_sm = 2 * (smem + 1024 + 64) <= 228 * 1024 ? 2 : 1;
  const long long slots = (long long)std::max(1, sm_share) * per_sm;
  const long long strips = (cols + kStreamW - 1) / kStreamW;
  int best_run = rows;
  long long best = -1;
  for (int run = 1; run <= rows + 7; run = run < 16 ? run + 1 : run + 8) {
    const int rr = std::min(run, rows);
    const long long ctas = strips * ((rows + rr - 1) / rr);
    const long long waves = (ctas + slots - 1) / slots;
    const long long stages = (rr + 2 * wr + kStreamKS - 1) / kStreamKS;
    const long long cost = waves * stages;
    if (best < 0 || cost < best || (cost == best && rr > best_run)) {
      best = cost;
      best_run = rr;
    }
    if (rr == rows) break;
  }
  out->run = best_run;
  out->bw = kStreamW;
  out->pitch = pitch;
  out->ring_rows = rb;
  out->e = e;
  out->smem = smem;
  out->ctas = (int)(strips * ((rows + best_run - 1) / best_run));
  return true;
}

template <bool kMapCut, int kE>
static cudaError_t launch_stream_tma_t(const CfarTmaParams& p, int blocks, size_t smem, cudaStream_t s) {
  auto fn = k_sat_cfar_stream_tma<kMapCut, kE>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(fn, blocks, kStreamThreads, smem, s, p);
}

cudaError_t launch_cfar_stream_tma(const CfarTmaParams& p, bool map_cut, int e, int blocks, size_t smem,
                                   cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  if (e == 6) return map_cut ? launch_stream_tma_t<true, 6>(p, blocks, smem, s) : launch_stream_tma_t<false, 6>(p, blocks, smem, s);
  return map_cut ? launch_stream_tma_t<true, 8>(p, blocks, smem, s) : launch_stream_tma_t<false, 8>(p, blocks, smem, s);
}

int cfar_os_geometry(CfarMapDev& P, int rows, int cols) {
  P.tiles_x = (cols + 31) / 32;
  P.bh = kOsRows;
  P.bw = 32;
  return P.tiles_x * ((rows + kOsRows - 1) / kOsRows);
}

size_t cfar_os_smem(int wr, int wc, int n_ref) {
  return (size_t)(kOsRows + 2 * wr) * (32 + 2 * wc) * 4 + (size_t)n_ref * 4;
}

template <int kNK>
static cudaError_t launch_os_t(const CfarBatch& b, int blocks, size_t smem, cudaStream_t s) {
  auto fn = k_cfar_os<kNK>;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(fn), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(fn, blocks, 256, smem, s, b);
}

cudaError_t launch_cfar_os(const CfarBatch& b, int max_n_ref, int blocks, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const int nk = (max_n_ref + 31) / 32;
  if (nk <= 8) return launch_os_t<8>(b, blocks, smem, s);
  if (nk <= 16) return launch_os_t<16>(b, blocks, smem, s);
  if (nk <= 24) return launch_os_t<24>(b, blocks, smem, s);
  if (nk <= 32) return launch_os_t<32>(b, blocks, smem, s);
  if (nk <= 40) return launch_os_t<40>(b, blocks, smem, s);
  if (nk <= 48) return launch_os_t<48>(b, blocks, smem, s);
  if (nk <= 56) return launch_os_t<56>(b, blocks, smem, s);
  if (nk <= 64) return launch_os_t<64>(b, blocks, smem, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_cfar_direct(const CfarMapDev& m, int blocks, size_t smem, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(&k_cfar_direct), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_cfar_direct, blocks, 256, smem, s, m);
}

}  // namespace rcfar
