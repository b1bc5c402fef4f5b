// Preprocessing kernels of the radar chain (paper Sec. II.A).
//
//   k_colstats : per trace n, the least-squares line over fast time m
//                (a_n = mean, b_n = slope about mbar) -- "DC-shift removal and
//                linear trend subtraction" -- from compensated column sums,
//                so that a_n and b_n are correctly rounded; also the pieces
//                of each row's slow-time mean of y (see k_ysplit).
//   k_ysplit   : detrend + slow-time mean filter + max|y|; writes y minus
//                its row mean, scaled per (row, K block) by a power of two
//                and split into an integer plane and the FP16 head and tail
//                of the remainder.
//   k_band_dft : band DFT as a GEMM of y [M x N] with the twiddle matrix
//                [N x 2C] on the tcgen05 tensor cores (six FP16 products
//                per K step into two accumulators in tensor memory, the
//                integer head x head one exact), then the magnitude;
//                split-K for small frames. Each row's
//                mean c_m was removed from y and N c_m is added back to bin
//                0 only: a constant contributes to no other bin, and removing
//                it keeps the FP32 rounding of the large per-range DC offsets
//                out of the small bins.
//   k_dft_reduce: sums the K blocks' partials (fixed order), magnitude.
//   Normalisation ("then normalized") divides the magnitude by max|y|: the
//   DFT is linear, so this equals transforming y / max|y|.
//   k_twiddles : twiddle matrix W[n][2j] = cos(2 pi t/N), W[n][2j+1] = -sin,
//                t = (c0 + j) n mod N, computed once per (N, band) in FP64 and
//                stored x 2^9 as an integer plane and the FP16 head and tail
//                planes of the remainder.
#include "rcfar_internal.cuh"
#include "async_copy.cuh"

#include <mutex>
#include <map>
#include <utility>

namespace rcfar {

cudaError_t ensure_smem(const void* fn, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = done[std::make_pair(fn, dev)];
  if (cur >= bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

namespace {

__device__ __forceinline__ void load4_masked(const float* row, int col, int n, bool vec, float v[4]) {
  if (vec && col + 3 < n) {
    float4 t = __ldg(reinterpret_cast<const float4*>(row + col));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = (col + k < n) ? __ldg(row + col + k) : 0.0f;
  }
}

// Weight of sample j in sum_n y[n] for the truncated centred mean filter:
// w_j = sum over outputs n whose window holds j of 1 / |window(n)| (1 inside).
__device__ __forceinline__ float mean_weight(int j, int N, int h) {
  if (j >= N) return 0.f;
  if (j >= 2 * h && j <= N - 1 - 2 * h) return 1.f;
  float w = 0.f;
  for (int n = max(0, j - h); n <= min(N - 1, j + h); ++n) {
    const int cnt = min(n + h, N - 1) - max(n - h, 0) + 1;
    w += 1.f / (float)cnt;
  }
  return w;
}

// Trace-major frame X[m][n] = xsrc[n * ldsrc + m] -> range-major copy
// x[m * ldx + n]: CTA of 32 x 8 threads per 32 x 32 tile; rows of the source
// are read and rows of the copy written 128 bytes at a time through a padded
// shared tile. Frames given range-major (xsrc == nullptr) have no CTAs.
__global__ void __launch_bounds__(256) k_transpose(const __grid_constant__ PreBatch b) {
  pdl_trigger();
  pdl_wait();
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_tr);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_tr;
  if (local >= F.n_tr || F.xsrc == nullptr) return;
  __shared__ float t[kTrTile][kTrTile + 1];
  const int tiles_m = (F.M + kTrTile - 1) / kTrTile;
  const int tn = local / tiles_m, tm = local - tn * tiles_m;
  const int m0 = tm * kTrTile, n0 = tn * kTrTile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kTrTile; k += 8) {
    const int n = n0 + ty + k, m = m0 + tx;
    t[ty + k][tx] = (n < F.N && m < F.M) ? __ldg(F.xsrc + (long long)n * F.ldsrc + m) : 0.f;
  }
  __syncthreads();
  float* out = const_cast<float*>(F.x);
#pragma unroll
  for (int k = 0; k < kTrTile; k += 8) {
    const int m = m0 + ty + k, n = n0 + tx;
    if (m < F.M && n < F.N) out[(long long)m * F.ldx + n] = t[tx][ty + k];
  }
}

// (value, error) pair += a + b, b the exact error of a: the sum's own FP32
// rounding error is recovered (two_sum, Knuth) and kept in the pair's error.
// The _rn intrinsics keep each operation a single IEEE add (never fused).
__device__ __forceinline__ void acc_pair(float2& acc, float a, float b) {
  const float s = __fadd_rn(acc.x, a);
  const float bb = __fsub_rn(s, acc.x);
  const float e = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(a, bb));
  acc.x = s;
  acc.y = __fadd_rn(acc.y, __fadd_rn(e, b));
}
// Pairs (x, y) and (z, w) of t += those of u.
__device__ __forceinline__ void add_pairs(float4& t, const float4& u) {
  float2 p = make_float2(t.x, t.y), q = make_float2(t.z, t.w);
  acc_pair(p, u.x, u.y);
  acc_pair(q, u.z, u.w);
  t = make_float4(p.x, p.y, q.x, q.y);
}

// grid: for every frame, n_strips x n_groups CTAs of 256 threads; a CTA takes
// chunks_per_cta consecutive chunks of 64 rows (kStatsRowsPerChunk) of one
// 128-column strip, n_groups = ceil(n_chunks / chunks_per_cta). Per chunk,
// thread (g = warp, lane) owns rows g, g+8, ... for 4 columns; all 8 rows
// are loaded before any arithmetic. Every chunk writes its own partial
// column sums, so the results do not depend on chunks_per_cta.
__global__ void __launch_bounds__(256, 4) k_colstats(const __grid_constant__ PreBatch b) {
  pdl_trigger();
  pdl_wait();
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_stats);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_stats;
  const int strip = local % F.n_strips;
  const int group = local / F.n_strips;
  const int ch0 = group * F.chunks_per_cta;
  const int ch1 = min(F.n_chunks, ch0 + F.chunks_per_cta);
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int col0 = strip * kStatsStrip + lane * 4;
  const bool vec = ((F.ldx & 3) == 0) && ((reinterpret_cast<uintptr_t>(F.x) & 15) == 0);
  float wj[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) wj[k] = mean_weight(col0 + k, F.N, F.h);
  __shared__ float4 red[8][kStatsStrip];  // (sum x, its error, sum (m - mbar) x, its error)
  __shared__ bool is_last;

  for (int chunk = ch0; chunk < ch1; ++chunk) {
    const int r0 = chunk * kStatsRowsPerChunk;
    float v[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = r0 + g + 8 * i;
      if (m < F.M) {
        load4_masked(F.x + (long long)m * F.ldx, col0, F.N, vec, v[i]);
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[i][k] = 0.f;
      }
    }
    // column sums carried as unevaluated pairs (value, rounding error), so
    // that a_n and b_n come out correctly rounded: each FP32 add's error is
    // recovered exactly (two_sum) and each product's by one FMA
    float2 sx[4], smx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sx[k] = make_float2(0.f, 0.f);
      smx[k] = make_float2(0.f, 0.f);
    }
    float rs[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float dm = (float)(r0 + g + 8 * i) - F.mbar;
      rs[i] = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        acc_pair(sx[k], v[i][k], 0.f);
        const float p = __fmul_rn(dm, v[i][k]);
        acc_pair(smx[k], p, fmaf(dm, v[i][k], -p));  // the product's exact error
        rs[i] = fmaf(wj[k], v[i][k], rs[i]);
      }
    }
    // row sums over the strip (sum_j w_j x[m, j]): reduce the 8 rows across the warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int i = 0; i < 8; ++i) rs[i] += __shfl_xor_sync(0xffffffffu, rs[i], o);
    if (lane < 8) {
      float mine = rs[0];
#pragma unroll
      for (int i = 1; i < 8; ++i)
        if (lane == i) mine = rs[i];
      const int m = r0 + g + 8 * lane;
      if (m < F.M) F.rowpart[(long long)strip * F.M + m] = mine;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[g][lane * 4 + k] = make_float4(sx[k].x, sx[k].y, smx[k].x, smx[k].y);
    __syncthreads();
    if (threadIdx.x < kStatsStrip) {
      const int c = strip * kStatsStrip + threadIdx.x;
      float4 t = red[0][threadIdx.x];
#pragma unroll
      for (int gg = 1; gg < 8; ++gg) add_pairs(t, red[gg][threadIdx.x]);
      if (c < F.N) F.partial[(long long)chunk * F.N + c] = t;
    }
    __syncthreads();  // red is rewritten by the next chunk
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned nch = (unsigned)(ch1 - ch0);
    const unsigned old = atomicAdd(&F.strip_cnt[strip], nch);
    is_last = (old + nch == (unsigned)F.n_chunks);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    __shared__ float2 ab[kStatsStrip / 32];
    if (threadIdx.x < kStatsStrip) {
      const int c = strip * kStatsStrip + threadIdx.x;
      float2 st = make_float2(0.f, 0.f);
      if (c < F.N) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int cb = 0; cb < F.n_chunks; cb += 8) {  // fixed order: deterministic
          float4 p[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            p[u] = (cb + u < F.n_chunks) ? __ldcg(&F.partial[(long long)(cb + u) * F.N + c])
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < 8; ++u) add_pairs(t, p[u]);
        }
        // a_n = sum x / M, b_n = sum (m - mbar) x / D, each rounded once to FP32
        // (one FP64 division per trace)
        st = make_float2((float)(((double)t.x + (double)t.y) / (double)F.M),
                         (float)(((double)t.z + (double)t.w) * F.inv_D64));
        F.stats[c] = st;
      }
      // (sum_j w_j a_j, sum_j w_j b_j) over the strip: a fixed shuffle tree per warp of 32
      // columns, then the four warps' sums in order
      const float w = mean_weight(c, F.N, F.h);
      float2 t = make_float2(w * st.x, w * st.y);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
        t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
      }
      if (lane == 0) ab[g] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float2 t = ab[0];
#pragma unroll
      for (int i = 1; i < kStatsStrip / 32; ++i) {
        t.x += ab[i].x;
        t.y += ab[i].y;
      }
      F.strip_ab[strip] = t;
      F.strip_cnt[strip] = 0u;
    }
  }
  if (local == 0 && threadIdx.x == 0) *F.ymax = 0u;
}

// Power-of-two shift s of a K block of y: mx 2^s in [64, 128) for the
// block's largest magnitude mx, so that rint(y 2^s) is an integer of at most
// 8 bits (0 for an all-zero or non-finite block; |s| <= 100 keeps 2^s and
// 2^-s normal FP32 numbers).
__device__ __forceinline__ int y_shift(float mx) {
  if (!(mx > 0.f) || !(mx <= 3.0e38f)) return 0;
  int e;
  frexpf(mx, &e);  // mx = f 2^e, 1/2 <= f < 1
  return max(-100, min(100, 7 - e));
}

// v (|v| < 128) as three FP16 values: the integer q = rint(v) (exact in FP16)
// and the FP16 head and tail of the remainder v - q (exact in FP32, |.| <= 1/2):
// about 30 significant bits together.
__device__ __forceinline__ void split_y3(float v, __half* q, __half* rh, __half* rt) {
  const float qf = rintf(v);
  const float r = v - qf;
  const __half h = __float2half_rn(r);
  *q = __float2half_rn(qf);
  *rh = h;
  *rt = __float2half_rn(r - __half2float(h));
}

// y pass: one warp per frame row, kYCols samples per CTA column block.
//   x'[m,n] = x[m,n] - a_n - b_n (m - mbar)       (detrend)
//   y[m,n]  = mean of x'[m, n-h..n+h] in [0, N)    (mean filter)
// evaluated as ((x - rho_m) - a_n) - b_n (m - mbar) with one FMA, rho_m the
// row's mean level, and the mean filter applied to that; y - c_m follows as
// (y - rho_m) - (c_m - rho_m). In exact arithmetic nothing changes; in FP32
// the large per-range offsets no longer pass through the roundings.
// records max |y| and writes y - c_m, where c_m is the row's slow-time mean
// (a constant only reaches bin 0; removing it keeps the FP32 rounding of the
// large per-range offsets out of the other bins), scaled per K block of 256
// samples by a power of two into the FP16 range and split into FP16 head and
// tail for the tensor-core product (the scale is recorded per (row, block)). Samples N..npad-1 are written as 0.
// H: the mean filter's half length when known at compile time (the window
// sum is unrolled), or -1 for any h.
template <int H>
__global__ void __launch_bounds__(256, 4) k_ysplit(const __grid_constant__ PreBatch b) {
  pdl_trigger();
  pdl_wait();
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_y);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_y;
  const int rb = local / F.ycols, cbk = local - rb * F.ycols;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = rb * kYRows + warp;
  const int n0 = cbk * kYCols;
  const int h = H >= 0 ? H : F.h, N = F.N;
  __shared__ float seg[kYRows][kYCols + 2 * kMaxMeanHalf];
  __shared__ float red[kYRows];
  float ymax = 0.f;
  if (m < F.M) {
    const float* xr = F.x + (long long)m * F.ldx;
    // fast layout: the whole block and its halo inside the frame, rows 16-byte
    // aligned, the filter length known at compile time; its samples are
    // loaded first, so their latency overlaps the row mean's
    constexpr int kPad = H >= 0 ? (H + 3) / 4 * 4 : 0;  // halo rounded up to whole float4
    constexpr int kG = (kYCols + 2 * kPad) / 4;         // float4 groups of the fast layout's span
    constexpr int kGL = (kG + 31) / 32;
    const bool vec = ((F.ldx & 3) == 0) && ((reinterpret_cast<uintptr_t>(F.x) & 15) == 0);
    const bool fastv = H >= 0 && vec && n0 - kPad >= 0 && n0 + kYCols + kPad <= N;  // uniform over the CTA
    float4 xq[kGL];
    if (fastv) {
#pragma unroll
      for (int u = 0; u < kGL; ++u) {
        const int g = lane + 32 * u;
        xq[u] = g < kG ? __ldg(reinterpret_cast<const float4*>(xr + n0 - kPad + 4 * g)) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    // row mean c_m = (sum_j w_j x[m,j] - sum_j w_j a_j - (m - mbar) sum_j w_j b_j) / N
    float rs = 0.f, A = 0.f, Bv = 0.f;
    for (int sI = lane; sI < F.n_strips; sI += 32) {
      rs += __ldg(&F.rowpart[(long long)sI * F.M + m]);
      const float2 ab = __ldg(&F.strip_ab[sI]);
      A += ab.x;
      Bv += ab.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rs += __shfl_xor_sync(0xffffffffu, rs, o);
      A += __shfl_xor_sync(0xffffffffu, A, o);
      Bv += __shfl_xor_sync(0xffffffffu, Bv, o);
    }
    const float dm = (float)m - F.mbar;
    // rho: a reference level of the row (its weighted mean of x, near the
    // row's DC offset). x - rho is formed first, so that the detrend and the
    // mean filter add numbers of the signal's size rather than of the offset's;
    // a constant per row only reaches bin 0, where c_m = rho + cmr is added back.
    const float rho = rs / (float)N;
    const float cmr = -fmaf(dm, Bv, A) / (float)N;  // c_m - rho
    const float cmv = rho + cmr;
    if (cbk == 0 && lane == 0) F.rowmean[m] = cmv;
    const long long yplane = (long long)F.M * F.npad;
    __half* y0 = F.yq + (long long)m * F.npad;  // Y0; Rh and Rt one and two planes on
    const float inv_full = 1.0f / (float)(2 * h + 1);
    constexpr int kQ = kYCols / 32;
    // dv[k]: y - c_m of the lane's k-th sample (0 past the frame); k < kQ / 2
    // lie in the block's first K block. Fast layout: sample n0 + 4 lane +
    // 128 (k / 4) + k % 4; general layout: sample n0 + lane + 32 k.
    float dv[kQ];
    float sq = 0.f;  // sum of (y - c_m)^2 over this lane's samples (z-score normalisation)
    if (fastv) {
      // seg[w][i] = x' at column n0 - kPad + i: 16-byte loads of the
      // statistics, 16-byte stores (all loads issued before any store)
      float4 sa[kGL], sb[kGL];
      const float4* st4 = reinterpret_cast<const float4*>(F.stats);  // two (a, b) pairs per float4
#pragma unroll
      for (int u = 0; u < kGL; ++u) {
        const int g = lane + 32 * u;
        if (g < kG) {
          const int c = n0 - kPad + 4 * g;
          sa[u] = __ldg(st4 + c / 2);
          sb[u] = __ldg(st4 + c / 2 + 1);
        }
      }
#pragma unroll
      for (int u = 0; u < kGL; ++u) {
        const int g = lane + 32 * u;
        if (g < kG) {
          float4 o;  // x - rho - a_n - b_n (m - mbar)
          o.x = fmaf(-sa[u].y, dm, (xq[u].x - rho) - sa[u].x);
          o.y = fmaf(-sa[u].w, dm, (xq[u].y - rho) - sa[u].z);
          o.z = fmaf(-sb[u].y, dm, (xq[u].z - rho) - sb[u].x);
          o.w = fmaf(-sb[u].w, dm, (xq[u].w - rho) - sb[u].z);
          *reinterpret_cast<float4*>(&seg[warp][4 * g]) = o;
        }
      }
      __syncwarp();
      // four consecutive outputs per lane and group: their windows from
      // kPad / 2 + 1 aligned 16-byte reads, each summed in the general
      // layout's order
#pragma unroll
      for (int qq = 0; qq < kQ / 4; ++qq) {
        const int base = 4 * lane + 128 * qq;
        float v[2 * kPad + 4];
#pragma unroll
        for (int r = 0; r < (2 * kPad + 4) / 4; ++r) {
          const float4 t = *reinterpret_cast<const float4*>(&seg[warp][base + 4 * r]);
          v[4 * r] = t.x;
          v[4 * r + 1] = t.y;
          v[4 * r + 2] = t.z;
          v[4 * r + 3] = t.w;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float acc = 0.f;
#pragma unroll
          for (int d = 0; d <= 2 * (H >= 0 ? H : 0); ++d) acc += v[kPad - (H >= 0 ? H : 0) + e + d];
          const float y = acc * inv_full;  // y - rho
          ymax = fmaxf(ymax, fabsf(y + rho));
          const float d = y - cmr;
          sq = fmaf(d, d, sq);
          dv[4 * qq + e] = d;
        }
      }
    } else {
      // x' over [n0 - h, n0 + kYCols + h): all loads issued before any store
      constexpr int kSeg = (kYCols + 2 * kMaxMeanHalf) / 32;
      float xv[kSeg];
      float2 sv[kSeg];
#pragma unroll
      for (int u = 0; u < kSeg; ++u) {
        const int i = lane + 32 * u;
        const int n = n0 - h + i;
        const bool ok = i < kYCols + 2 * h && n >= 0 && n < N;
        xv[u] = ok ? __ldg(xr + n) : 0.f;
        sv[u] = ok ? __ldg(&F.stats[n]) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < kSeg; ++u) {
        const int i = lane + 32 * u;
        const int n = n0 - h + i;  // samples outside the frame stay 0 (the truncated windows skip them)
        if (i < kYCols + 2 * h) seg[warp][i] = (n >= 0 && n < N) ? fmaf(-sv[u].y, dm, (xv[u] - rho) - sv[u].x) : 0.f;
      }
      __syncwarp();
      const float* sg = &seg[warp][lane];
      auto window = [&](int q) {
        float acc = 0.f;
        if constexpr (H >= 0) {
#pragma unroll
          for (int d = 0; d <= 2 * H; ++d) acc += sg[32 * q + d];
        } else {
          for (int d = 0; d <= 2 * h; ++d) acc += sg[32 * q + d];
        }
        return acc;
      };
      if (n0 - h >= 0 && n0 + kYCols + h <= N) {
        // every window of this block lies inside the frame
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const float y = window(q) * inv_full;
          ymax = fmaxf(ymax, fabsf(y + rho));
          const float d = y - cmr;
          sq = fmaf(d, d, sq);
          dv[q] = d;
        }
      } else {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          const int n = n0 + lane + 32 * q;
          dv[q] = 0.f;
          if (n < N) {
            const float acc = window(q);
            const int cnt = min(n + h, N - 1) - max(n - h, 0) + 1;
            // a full window multiplies by 1 / (2h + 1); the truncated ones at the ends divide
            const float y = cnt == 2 * h + 1 ? acc * inv_full : acc / (float)cnt;
            ymax = fmaxf(ymax, fabsf(y + rho));
            const float d = y - cmr;
            sq = fmaf(d, d, sq);
            dv[q] = d;
          }
        }
      }
    }
    // the block's two K blocks (q < kQ / 2 and q >= kQ / 2), each scaled by
    // its own power of two so that its largest magnitude lies in [64, 128),
    // then split into the integer Y0 and the FP16 head and tail of the rest
    float mx0 = 0.f, mx1 = 0.f;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      if (q < kQ / 2) mx0 = fmaxf(mx0, fabsf(dv[q]));
      else mx1 = fmaxf(mx1, fabsf(dv[q]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx0 = fmaxf(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
      mx1 = fmaxf(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
    }
    const int s0 = y_shift(mx0), s1 = y_shift(mx1);
    const float f0 = ldexpf(1.0f, s0), f1 = ldexpf(1.0f, s1);
    auto pack = [](const __half* h) {
      return make_uint2((unsigned)__half_as_ushort(h[0]) | ((unsigned)__half_as_ushort(h[1]) << 16),
                        (unsigned)__half_as_ushort(h[2]) | ((unsigned)__half_as_ushort(h[3]) << 16));
    };
    if (fastv) {
      // four consecutive samples per lane and group: one 8-byte store per plane
#pragma unroll
      for (int qq = 0; qq < kQ / 4; ++qq) {
        const int n = n0 + 4 * lane + 128 * qq;
        const float f = qq < kQ / 8 ? f0 : f1;
        __half a[4], b[4], c[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_y3(dv[4 * qq + e] * f, &a[e], &b[e], &c[e]);
        *reinterpret_cast<uint2*>(y0 + n) = pack(a);
        *reinterpret_cast<uint2*>(y0 + yplane + n) = pack(b);
        *reinterpret_cast<uint2*>(y0 + 2 * yplane + n) = pack(c);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kQ; ++q) {
        const int n = n0 + lane + 32 * q;
        if (n < F.npad) split_y3(dv[q] * (q < kQ / 2 ? f0 : f1), &y0[n], &y0[yplane + n], &y0[2 * yplane + n]);
      }
    }
    if (lane == 0) {  // the drain multiplies each partial by 2^-s 2^-kDftTBits (exact)
      const int blk = 2 * cbk;
      if (blk < F.nblocks) F.yscale[(long long)blk * F.M + m] = ldexpf(1.0f, -s0 - kDftTBits);
      if (blk + 1 < F.nblocks) F.yscale[(long long)(blk + 1) * F.M + m] = ldexpf(1.0f, -s1 - kDftTBits);
    }
    if (F.normalise == RCFAR_NORM_ROW_ZSCORE) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
      if (lane == 0) F.rowsq[(long long)cbk * F.M + m] = sq;  // one slot per (block, row): fixed-order sum later
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
  if (lane == 0) red[warp] = ymax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mx = red[0];
    for (int w2 = 1; w2 < kYRows; ++w2) mx = fmaxf(mx, red[w2]);
    atomicMax(F.ymax, __float_as_uint(mx));
  }
}

// Shared-memory matrix descriptor of a K-major operand tile whose rows are
// 128 bytes (64 FP16 values) stored with the 128-byte swizzle: 8-row groups
// 1024 bytes apart (SBO), layout SWIZZLE_128B, descriptor version 1.
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr) {
  return (unsigned long long)((saddr >> 4) & 0x3FFFu) | (1ull << 16) | ((unsigned long long)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void umma_f16(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// The six products of one K step (64 samples: four MMAs of 16 along K
// each): ACC_A += Y0 T0 (integers: exact), ACC_B += Y0 T1 + Y0 T2 + Rh T0 +
// Rh T1 + Rt T0. sa: the stage's Y0 plane (Rh, Rt follow kDftBM * 128 bytes
// apart); sb: its T0 plane (T1, T2 follow bn * 128 bytes apart). first: the
// block's first K step (the accumulators start from zero).
__device__ __forceinline__ void dft_step_mmas(unsigned dA, unsigned dB, unsigned sa, unsigned sb, int bn,
                                              unsigned idesc, bool first) {
  const unsigned pa = kDftBM * 128, pb = (unsigned)bn * 128;
#pragma unroll
  for (int kk = 0; kk < kDftBK / 16; ++kk) {
    const unsigned off = kk * 32;  // 16 FP16 values along K
    const unsigned long long a0 = umma_desc(sa + off), a1 = umma_desc(sa + pa + off), a2 = umma_desc(sa + 2 * pa + off);
    const unsigned long long b0 = umma_desc(sb + off), b1 = umma_desc(sb + pb + off), b2 = umma_desc(sb + 2 * pb + off);
    const unsigned en = (!first || kk > 0) ? 1u : 0u;
    umma_f16(dA, a0, b0, idesc, en);
    umma_f16(dB, a0, b2, idesc, en);
    umma_f16(dB, a0, b1, idesc, 1u);
    umma_f16(dB, a1, b0, idesc, 1u);
    umma_f16(dB, a1, b1, idesc, 1u);
    umma_f16(dB, a2, b0, idesc, 1u);
  }
}

// Drain one accumulator buffer (ACC_A at TMEM column ca, ACC_B at ca + bn)
// for the warp's 32 TMEM lanes (quarter q of the tile) into a block's
// partials, which are column-major: dst[c * cs] = (ACC_A + ACC_B) * f for
// output column c, one rounding (f = 2^-s 2^-9, exact). The lane is the row,
// so each store of a column is 32 consecutive floats across the warp.
// Columns go 32 at a time (16 for a tail; bn is a multiple of 16): both
// accumulators' loads are issued before one wait. Returns once every tensor-
// memory load of the buffer has completed (the stores of the last chunk may
// still be in flight), so the caller can release the buffer.
__device__ __forceinline__ void tmem_ld32(unsigned ta, unsigned* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(ta));
}
__device__ __forceinline__ void tmem_ld16(unsigned ta, unsigned* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
}
__device__ __forceinline__ void dft_drain(unsigned tmem, int q, unsigned ca, int bn, float* dst, long long cs, float f,
                                          bool ok) {
  const unsigned ta = tmem + ((unsigned)(32 * q) << 16) + ca;
  int c = 0;
  for (; c + 32 <= bn; c += 32) {
    unsigned ra[32], rb[32];
    tmem_ld32(ta + (unsigned)c, ra);
    tmem_ld32(ta + (unsigned)(bn + c), rb);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (ok) {
      float* d = dst + (long long)c * cs;
#pragma unroll
      for (int k = 0; k < 32; ++k) d[k * cs] = (__uint_as_float(ra[k]) + __uint_as_float(rb[k])) * f;
    }
  }
  if (c < bn) {  // a tail of 16 columns
    unsigned ra[16], rb[16];
    tmem_ld16(ta + (unsigned)c, ra);
    tmem_ld16(ta + (unsigned)(bn + c), rb);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (ok) {
      float* d = dst + (long long)c * cs;
#pragma unroll
      for (int k = 0; k < 16; ++k) d[k * cs] = (__uint_as_float(ra[k]) + __uint_as_float(rb[k])) * f;
    }
  }
}

// Band DFT as a GEMM on the 5th-generation tensor cores: y [M x npad] (three
// FP16 planes Y0, Rh, Rt) times W^T [npad x ldw] (three planes T0, T1, T2),
// six products per K step into two accumulators (dft_step_mmas; the integer
// head x head product accumulates exactly). One CTA per (128-row tile,
// bn-column tile, K split), 12 warps:
//   warp 0     issues the MMAs (one thread) into tensor memory;
//   warps 1-7  stage K steps of 64 samples with cp.async into a ring of
//              stages in the 128-byte-swizzled K-major layout the MMA reads;
//   warps 8-11 drain the accumulators every kDftKB K steps (a K block of 256
//              samples) into that block's partial sums in global memory.
// When two accumulator buffers fit tensor memory they alternate, so the MMAs
// of block b+1 run while block b is drained. k_dft_reduce adds the blocks'
// partials in a fixed order with Kahan compensation. Every wait is bounded:
// a timeout records kStatusTimeout and the CTA still drains its MMAs, frees
// its tensor memory and returns.
__global__ void __launch_bounds__(kDftThreads, 1) k_band_dft(const __grid_constant__ PreBatch b) {
  pdl_trigger();
  pdl_wait();
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_dft);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_dft;
  const int per_split = F.mtiles * F.ntiles;
  const int ks = local / per_split;
  const int rem = local % per_split;
  const int mt = rem / F.ntiles, nt = rem % F.ntiles;
  const int m0 = mt * kDftBM;
  const int bn = F.bn;
  const int j0 = nt * bn;  // real output column
  const int kbeg = ks * F.kper;  // a multiple of kDftBlock
  const int kend = min(F.npad, kbeg + F.kper);
  const int nk = (kend - kbeg) / kDftBK;
  const int nblk = (nk + kDftKB - 1) / kDftKB;
  const int blk0 = kbeg / (kDftBK * kDftKB);  // global index of this CTA's first K block
  const int stage_bytes = dft_stage_bytes(bn);
  int stages = (b.dft_smem - 1024) / stage_bytes;
  if (stages > kDftMaxStages) stages = kDftMaxStages;

  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) unsigned long long bar_full[kDftMaxStages], bar_empty[kDftMaxStages];
  __shared__ __align__(8) unsigned long long bar_accf[2], bar_acce[2], bar_done;
  __shared__ unsigned tmem_slot;
  __shared__ int s_fail;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nbuf = dft_acc_buffers(bn);  // buffers of (ACC_A, ACC_B), 2 bn columns each
  unsigned tcols = 32;
  while ((int)tcols < 2 * bn * nbuf) tcols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < kDftMaxStages; ++i) {
      mbar_init(smem_u32(&bar_full[i]), 224);
      mbar_init(smem_u32(&bar_empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bar_accf[i]), 1);    // accumulator i holds a finished block
      mbar_init(smem_u32(&bar_acce[i]), 128);  // accumulator i was drained
    }
    mbar_init(smem_u32(&bar_done), 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;

  // instruction descriptor: D FP32 (bits 4-5 = 1), A and B FP16 (bits 7-9, 10-12 = 0),
  // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const unsigned idesc = (1u << 4) | ((unsigned)(bn >> 3) << 17) | ((unsigned)(kDftBM >> 4) << 24);
  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < nk; ++i) {
        const int slot = i % stages;
        const int bi = i / kDftKB, acc = bi % nbuf;
        const bool first = (i % kDftKB) == 0;
        if (first && bi >= nbuf &&
            !mbar_wait(smem_u32(&bar_acce[acc]), (unsigned)(((bi - nbuf) / nbuf) & 1))) {
          s_fail = 1;
          break;
        }
        if (!mbar_wait(smem_u32(&bar_full[slot]), (unsigned)((i / stages) & 1))) {
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned sa = smem_u32(base + slot * stage_bytes);
        const unsigned dA = tmem + (unsigned)(acc * 2 * bn);
        dft_step_mmas(dA, dA + (unsigned)bn, sa, sa + kDftYPlanes * kDftBM * 128, bn, idesc, first);
        umma_commit(smem_u32(&bar_empty[slot]));  // the slot is free once these MMAs finish
        if ((i % kDftKB) == kDftKB - 1 || i == nk - 1) umma_commit(smem_u32(&bar_accf[acc]));  // block done
      }
      umma_commit(smem_u32(&bar_done));  // tracks every MMA issued above
    }
  } else if (warp < 8) {
    // producers: stage i -> ring slot i % stages: Y0 | Rh | Rt | T0 | T1 | T2
    const int ptid = tid - 32;
    const long long plane = F.ldw * F.npad;
    const long long yplane = (long long)F.M * F.npad;
    for (int i = 0; i < nk; ++i) {
      const int slot = i % stages;
      if (i >= stages && !mbar_wait(smem_u32(&bar_empty[slot]), (unsigned)(((i - stages) / stages) & 1))) {
        s_fail = 1;
        break;
      }
      const unsigned sa = smem_u32(base + slot * stage_bytes);
      const unsigned sb0 = sa + kDftYPlanes * kDftBM * 128;
      const int k0 = kbeg + i * kDftBK;
      for (int id = ptid; id < kDftBM * 8; id += 224) {  // y: 128 rows x 8 chunks of 16 bytes, each plane
        const int rr = id >> 3, c = id & 7;
        const int m = m0 + rr;
        const bool ok = m < F.M;
        const long long off = (long long)(ok ? m : 0) * F.npad + k0 + 8 * c;
        const unsigned sw = rr * 128 + ((c ^ (rr & 7)) << 4);
#pragma unroll
        for (int pl = 0; pl < kDftYPlanes; ++pl) cp_async16(sa + pl * kDftBM * 128 + sw, F.yq + pl * yplane + off, ok);
      }
      const __half* wb = F.Wt + (long long)j0 * F.npad + k0;
      for (int id = ptid; id < bn * 8; id += 224) {  // W: bn rows (output columns) x 8 chunks
        const int rr = id >> 3, c = id & 7;
        const __half* src = wb + (long long)rr * F.npad + 8 * c;
        const unsigned sw = rr * 128 + ((c ^ (rr & 7)) << 4);
#pragma unroll
        for (int pl = 0; pl < kDftWPlanes; ++pl) cp_async16(sb0 + pl * bn * 128 + sw, src + pl * plane, true);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (i >= 1) {  // two stages of copies in flight: publish the older one
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
        mbar_arrive(smem_u32(&bar_full[(i - 1) % stages]));
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!s_fail && nk >= 1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&bar_full[(nk - 1) % stages]));
    }
  } else {
    // drain warps: warp -> TMEM lanes 32 (warp & 3) .. (tile rows)
    const int q = warp & 3;
    const int m = m0 + 32 * q + lane;
    for (int bi = 0; bi < nblk; ++bi) {
      const int acc = bi % nbuf;
      if (!mbar_wait(smem_u32(&bar_accf[acc]), (unsigned)((bi / nbuf) & 1))) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* dst = F.kpart + ((long long)(blk0 + bi) * F.ldk + j0) * F.M + (m < F.M ? m : 0);
      // back to the units of y: the block's rows were scaled by 2^s(m, block), the twiddles by 2^9 (exact)
      const float f = m < F.M ? __ldg(F.yscale + (long long)(blk0 + bi) * F.M + m) : 0.f;
      dft_drain(tmem, q, (unsigned)(acc * 2 * bn), bn, dst, F.M, f, m < F.M);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&bar_acce[acc]));
    }
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_u32(&bar_done), 0u) && !s_fail;
  if (!ok && tid == 0) atomicOr(b.status, kStatusTimeout);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// The same GEMM with the operands brought in by the tensor memory
// accelerator: one thread of warp 1 issues, per K step, six box loads
// (the three y planes: 64 samples x 128 rows; the three twiddle planes: 64
// samples x bn columns) that complete on the stage's mbarrier with their byte
// count; rows past the frame arrive as zeros. Warp 0 issues the MMAs,
// warps 2-5 drain the accumulators (warp w reads TMEM lanes 32 (w % 4) ..).
__global__ void __launch_bounds__(kDftTmaThreads, 1) k_band_dft_tma(const __grid_constant__ DftBatch b) {
  pdl_trigger();
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &DftFrameDev::item_dft);
  const DftFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_dft;
  const int per_split = F.mtiles * F.ntiles;
  const int ks = local / per_split;
  const int rem = local % per_split;
  const int mt = rem / F.ntiles, nt = rem % F.ntiles;
  const int m0 = mt * kDftBM;
  const int bn = F.bn;
  const int j0 = nt * bn;
  const int kbeg = ks * F.kper;
  const int kend = min(F.npad, kbeg + F.kper);
  const int nk = (kend - kbeg) / kDftBK;
  const int nblk = (nk + kDftKB - 1) / kDftKB;
  const int blk0 = kbeg / (kDftBK * kDftKB);
  const int stage_bytes = dft_stage_bytes(bn);
  int stages = (b.dft_smem - 1024) / stage_bytes;
  if (stages > kDftMaxStages) stages = kDftMaxStages;

  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) unsigned long long bar_full[kDftMaxStages], bar_empty[kDftMaxStages];
  __shared__ __align__(8) unsigned long long bar_accf[2], bar_acce[2], bar_done;
  __shared__ unsigned tmem_slot;
  __shared__ int s_fail;
  __shared__ int s_issued, s_consumed;  // K steps whose loads were issued / waited for by the MMA thread

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nbuf = dft_acc_buffers(bn);  // buffers of (ACC_A, ACC_B), 2 bn columns each
  unsigned tcols = 32;
  while ((int)tcols < 2 * bn * nbuf) tcols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < kDftMaxStages; ++i) {
      mbar_init(smem_u32(&bar_full[i]), 1);   // the producer's arrive.expect_tx
      mbar_init(smem_u32(&bar_empty[i]), 1);  // the MMAs' commit
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(smem_u32(&bar_accf[i]), 1);
      mbar_init(smem_u32(&bar_acce[i]), 128);
    }
    mbar_init(smem_u32(&bar_done), 1);
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    mbar_init_fence();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  pdl_wait();  // the tensor-memory allocation and barriers above overlap the previous kernel

  // instruction descriptor: D FP32 (bits 4-5 = 1), A and B FP16 (bits 7-9, 10-12 = 0),
  // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const unsigned idesc = (1u << 4) | ((unsigned)(bn >> 3) << 17) | ((unsigned)(kDftBM >> 4) << 24);
  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < nk; ++i) {
        const int slot = i % stages;
        const int bi = i / kDftKB, acc = bi % nbuf;
        const bool first = (i % kDftKB) == 0;
        if (first && bi >= nbuf &&
            !mbar_wait(smem_u32(&bar_acce[acc]), (unsigned)(((bi - nbuf) / nbuf) & 1))) {
          s_fail = 1;
          break;
        }
        if (!mbar_wait(smem_u32(&bar_full[slot]), (unsigned)((i / stages) & 1))) {
          s_fail = 1;
          break;
        }
        s_consumed = i + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned sa = smem_u32(base + slot * stage_bytes);
        const unsigned dA = tmem + (unsigned)(acc * 2 * bn);
        dft_step_mmas(dA, dA + (unsigned)bn, sa, sa + kDftYPlanes * kDftBM * 128, bn, idesc, first);
        umma_commit(smem_u32(&bar_empty[slot]));
        if ((i % kDftKB) == kDftKB - 1 || i == nk - 1) umma_commit(smem_u32(&bar_accf[acc]));
      }
      umma_commit(smem_u32(&bar_done));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const unsigned long long ma = reinterpret_cast<unsigned long long>(&b.ma[fi]);
      const unsigned long long mb = reinterpret_cast<unsigned long long>(&b.mb[fi]);
      asm volatile("prefetch.tensormap [%0];" ::"l"(ma) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(mb) : "memory");
      const unsigned tx = (unsigned)dft_stage_bytes(bn);
      for (int i = 0; i < nk; ++i) {
        const int slot = i % stages;
        if (i >= stages && !mbar_wait(smem_u32(&bar_empty[slot]), (unsigned)(((i - stages) / stages) & 1))) {
          s_fail = 1;
          break;
        }
        const unsigned sa = smem_u32(base + slot * stage_bytes);
        const unsigned sb0 = sa + kDftYPlanes * kDftBM * 128;
        const unsigned bar = smem_u32(&bar_full[slot]);
        const int k0 = kbeg + i * kDftBK;
        mbar_arrive_expect_tx(bar, tx);
#pragma unroll
        for (int pl = 0; pl < kDftYPlanes; ++pl) tma_load_3d(sa + pl * kDftBM * 128, ma, k0, m0, pl, bar);
#pragma unroll
        for (int pl = 0; pl < kDftWPlanes; ++pl) tma_load_3d(sb0 + pl * bn * 128, mb, k0, j0, pl, bar);
        s_issued = i + 1;
      }
    }
  } else {
    const int q = warp & 3;
    const int m = m0 + 32 * q + lane;
    for (int bi = 0; bi < nblk; ++bi) {
      const int acc = bi % nbuf;
      // back to the units of y: the block's rows were scaled by 2^s(m, block), the twiddles by 2^9
      // (exact); loaded before the wait so that its latency overlaps the block's MMAs
      const float f = m < F.M ? __ldg(F.yscale + (long long)(blk0 + bi) * F.M + m) : 0.f;
      if (!mbar_wait(smem_u32(&bar_accf[acc]), (unsigned)((bi / nbuf) & 1))) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* dst = F.kpart + ((long long)(blk0 + bi) * F.ldk + j0) * F.M + (m < F.M ? m : 0);
      dft_drain(tmem, q, (unsigned)(acc * 2 * bn), bn, dst, F.M, f, m < F.M);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&bar_acce[acc]));
    }
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_u32(&bar_done), 0u) && !s_fail;
  if (!ok && tid == 0) atomicOr(b.status, kStatusTimeout);
  // after a failure, the loads issued but never waited for land before the
  // shared memory is released (bounded waits)
  if (tid == 32)
    for (int i = s_consumed; i < s_issued; ++i)
      mbar_wait(smem_u32(&bar_full[i % stages]), (unsigned)((i / stages) & 1));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// Sum of the K blocks' partials in a fixed order with Kahan compensation
// (deterministic, and the same however the K range was split), magnitude,
// bin 0's mean added back, and the normalisation by max |y| ("then
// normalized": the DFT is linear, so this equals transforming y / max|y|).
// Grid: per frame, ceil(M C / 256) CTAs; one thread per map cell, rows
// fastest (the partials are column-major, so a warp's loads are contiguous).
__global__ void __launch_bounds__(256) k_dft_reduce(const __grid_constant__ PreBatch b) {
  pdl_trigger();
  pdl_wait();
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_norm);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_norm;
  // cells in column-major order, 256 per CTA (a CTA may span several bins)
  const long long cell = (long long)local * 256 + threadIdx.x;
  if (cell >= (long long)F.M * F.C) return;
  const int j = (int)(cell / F.M);
  const int m = (int)(cell - (long long)j * F.M);
  float inv;
  if (F.normalise == RCFAR_NORM_ROW_ZSCORE) {
    // z-score: 1 / std of the row's y (population std; 0 for a constant row)
    float ss = 0.f;
    for (int cb = 0; cb < F.ycols; ++cb) ss += __ldg(&F.rowsq[(long long)cb * F.M + m]);
    const float sd = sqrtf(ss / (float)F.N);
    inv = sd > 0.f ? 1.f / sd : 0.f;
  } else {
    const float mx = __uint_as_float(__ldcg(F.ymax));
    inv = mx > 0.f ? 1.f / mx : 1.f;
  }
  // block b's partials: [ldk][M]; bin j's real part in column 2 j, its imaginary part in 2 j + 1
  const long long plane = (long long)F.M * F.ldk;
  const float* src = F.kpart + (long long)(2 * j) * F.M + m;
  float re = 0.f, im = 0.f, cr = 0.f, ci = 0.f;
  for (int b0 = 0; b0 < F.nblocks; b0 += 8) {
    float2 v[8];  // the next 8 blocks' partials, loaded together
#pragma unroll
    for (int u = 0; u < 8; ++u)
      v[u] = (b0 + u < F.nblocks) ? make_float2(__ldcg(src + (b0 + u) * plane), __ldcg(src + (b0 + u) * plane + F.M))
                                  : make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float yr = v[u].x - cr, tr = re + yr;
      cr = __fsub_rn(__fsub_rn(tr, re), yr);
      re = tr;
      const float yi = v[u].y - ci, ti = im + yi;
      ci = __fsub_rn(__fsub_rn(ti, im), yi);
      im = ti;
    }
  }
  // bin 0 gets the mean back (the z-scored series has none)
  if (j == 0 && F.c0 == 0 && F.normalise != RCFAR_NORM_ROW_ZSCORE) re = fmaf((float)F.N, __ldg(&F.rowmean[m]), re);
  // a z-scored series has zero mean: its bin 0 is exactly 0 (only rounding remains in re, im)
  const float p2 = (F.normalise == RCFAR_NORM_ROW_ZSCORE && F.c0 + j == 0) ? 0.f : fmaf(re, re, im * im);
  F.map[(long long)m * F.ld_map + j] = F.detector == RCFAR_DETECT_SQUARE_LAW ? p2 * (inv * inv) : sqrtf(p2) * inv;
}

__global__ void k_twiddles(__half* Wt, long long ldw, int npad, int N, int c0, int C) {
  const long long total = (long long)N * C;
  const long long plane = ldw * npad;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i % N), j = (int)(i / N);
    const long long t = ((long long)(c0 + j) * n) % N;
    double s, c;
    sincospi(2.0 * (double)t / (double)N, &s, &c);
    // scaled by 2^kDftTBits: the integer T0 = rint(.) (exact in FP16, |T0| <= 512), the FP16
    // head T1 of the remainder and the FP16 tail T2 of what is left
    const double sc = (double)(1 << kDftTBits);
    const double v[2] = {c * sc, -s * sc};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const double t0 = rint(v[u]);
      const __half t1 = __double2half(v[u] - t0);
      const long long row = (long long)(2 * j + u) * npad + n;
      Wt[row] = __double2half(t0);
      Wt[plane + row] = t1;
      Wt[2 * plane + row] = __double2half(v[u] - t0 - (double)__half2float(t1));
    }
  }
}

}  // namespace

cudaError_t launch_transpose(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_pdl(k_transpose, blocks, 256, 0, s, b);
}

cudaError_t launch_colstats(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_pdl(k_colstats, blocks, 256, 0, s, b);
}

cudaError_t launch_ysplit(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  // one half length for the whole launch (a batch shares its mean filter)
  switch (b.f[0].h) {
    case 1: return launch_pdl(k_ysplit<1>, blocks, 256, 0, s, b);
    case 2: return launch_pdl(k_ysplit<2>, blocks, 256, 0, s, b);
    case 3: return launch_pdl(k_ysplit<3>, blocks, 256, 0, s, b);
    case 4: return launch_pdl(k_ysplit<4>, blocks, 256, 0, s, b);
    default: return launch_pdl(k_ysplit<-1>, blocks, 256, 0, s, b);
  }
}

cudaError_t launch_band_dft(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = (size_t)b.dft_smem;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(&k_band_dft), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_band_dft, blocks, kDftThreads, smem, s, b);
}

cudaError_t launch_band_dft_tma(const DftBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = (size_t)b.dft_smem;
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(&k_band_dft_tma), smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_band_dft_tma, blocks, kDftTmaThreads, smem, s, b);
}

cudaError_t launch_dft_reduce(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  return launch_pdl(k_dft_reduce, blocks, 256, 0, s, b);
}

cudaError_t launch_twiddles(__half* Wt, long long ldw, int npad, int N, int c0, int C, cudaStream_t s) {
  const long long total = (long long)N * C;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_twiddles<<<blocks, 256, 0, s>>>(Wt, ldw, npad, N, c0, C);
  return cudaGetLastError();
}

}  // namespace rcfar
