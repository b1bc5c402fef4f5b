// Preprocessing kernels of the radar chain (paper Sec. II.A).
//
//   k_colstats : per trace n, the least-squares line over fast time m
//                (a_n = mean, b_n = slope about mbar) -- "DC-shift removal and
//                linear trend subtraction"; also the pieces of each row's
//                slow-time mean of y (see k_band_dft).
//   k_band_dft : fused detrend + slow-time mean filter + max|y| + band DFT
//                (a GEMM of y [M x N] with the twiddle matrix [N x 2C]) +
//                magnitude. CUDA-core FP32 with split-K for small frames.
//                Each row's mean c_m over n is subtracted before the product
//                and N c_m added back to bin 0 only: a constant contributes
//                to no other bin, and removing it keeps the FP32 rounding of
//                the large per-range DC offsets out of the small bins.
//   k_normalise: divide the map by max|y| ("then normalized"); the DFT is
//                linear, so scaling its magnitude equals transforming y/max|y|.
//   k_twiddles : twiddle matrix W[n][2j] = cos(2 pi t/N), W[n][2j+1] = -sin,
//                t = (c0 + j) n mod N, computed once per (N, band) in FP64.
#include "rcfar_internal.cuh"

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

// grid: for every frame, n_strips x n_chunks CTAs of 256 threads.
// Thread (g = warp, lane) sums rows g, g+8, ... of its chunk for 4 columns.
__global__ void __launch_bounds__(256) k_colstats(const __grid_constant__ PreBatch b) {
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_stats);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_stats;
  const int strip = local % F.n_strips;
  const int chunk = local / F.n_strips;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int col0 = strip * kStatsStrip + lane * 4;
  const int r0 = chunk * F.rows_per_chunk;
  const int r1 = min(F.M, r0 + F.rows_per_chunk);
  const bool vec = ((F.ldx & 3) == 0) && ((reinterpret_cast<uintptr_t>(F.x) & 15) == 0);

  float wj[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) wj[k] = mean_weight(col0 + k, F.N, F.h);
  float sx[4] = {0.f, 0.f, 0.f, 0.f}, smx[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m = r0 + g; m < r1; m += 8) {
    float v[4];
    load4_masked(F.x + (long long)m * F.ldx, col0, F.N, vec, v);
    const float dm = (float)m - F.mbar;
    float rs = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sx[k] += v[k];
      smx[k] = fmaf(dm, v[k], smx[k]);
      rs = fmaf(wj[k], v[k], rs);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
    if (lane == 0) F.rowpart[(long long)strip * F.M + m] = rs;
  }
  __shared__ float2 red[8][kStatsStrip];
  __shared__ bool is_last;
#pragma unroll
  for (int k = 0; k < 4; ++k) red[g][lane * 4 + k] = make_float2(sx[k], smx[k]);
  __syncthreads();
  if (threadIdx.x < kStatsStrip) {
    const int c = strip * kStatsStrip + threadIdx.x;
    float2 t = red[0][threadIdx.x];
#pragma unroll
    for (int gg = 1; gg < 8; ++gg) {
      t.x += red[gg][threadIdx.x].x;
      t.y += red[gg][threadIdx.x].y;
    }
    if (c < F.N) F.partial[(long long)chunk * F.N + c] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned old = atomicAdd(&F.strip_cnt[strip], 1u);
    is_last = (old == (unsigned)F.n_chunks - 1u);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    __shared__ float2 ab[kStatsStrip];
    if (threadIdx.x < kStatsStrip) {
      const int c = strip * kStatsStrip + threadIdx.x;
      float2 st = make_float2(0.f, 0.f);
      if (c < F.N) {
        float2 t = make_float2(0.f, 0.f);
        for (int ch = 0; ch < F.n_chunks; ++ch) {  // fixed order: deterministic
          const float2 p = __ldcg(&F.partial[(long long)ch * F.N + c]);
          t.x += p.x;
          t.y += p.y;
        }
        st = make_float2(t.x * F.inv_M, t.y * F.inv_D);
        F.stats[c] = st;
      }
      const float w = mean_weight(c, F.N, F.h);
      ab[threadIdx.x] = make_float2(w * st.x, w * st.y);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float2 t = make_float2(0.f, 0.f);
      for (int i = 0; i < kStatsStrip; ++i) {
        t.x += ab[i].x;
        t.y += ab[i].y;
      }
      F.strip_ab[strip] = t;
      F.strip_cnt[strip] = 0u;
    }
  }
  if (local == 0 && threadIdx.x == 0) *F.ymax = 0u;
}

// Band DFT as a GEMM on CUDA cores. CTA tile: kDftBM rows x kDftBN real
// outputs; each K step stages x' = x - a_n - b_n (m - mbar) for the tile
// rows over samples [n0 - h, n0 + BK + h), forms the mean-filtered y in shared
// memory (transposed), and accumulates y * W.
__global__ void __launch_bounds__(256) k_band_dft(const __grid_constant__ PreBatch b) {
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_dft);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_dft;
  const int per_split = F.mtiles * F.ntiles;
  const int ks = local / per_split;
  const int rem = local % per_split;
  const int mt = rem / F.ntiles, nt = rem % F.ntiles;
  const int m0 = mt * kDftBM;
  const int j0 = nt * kDftBN;  // real output column
  const int twoC = 2 * F.C;
  const int kbeg = ks * F.kper;
  const int kend = min(F.N, kbeg + F.kper);
  const int h = F.h;
  const int XW = kDftBK + 2 * kMaxMeanHalf;  // staged width (>= BK + 2h)

  // dynamic shared memory: As[BK][BM] | Bs[BK][BN] | Xs[BM][BK + 2 kMaxMeanHalf + 1]
  extern __shared__ __align__(16) float dft_smem[];
  float (*As)[kDftBM] = reinterpret_cast<float (*)[kDftBM]>(dft_smem);
  float (*Bs)[kDftBN] = reinterpret_cast<float (*)[kDftBN]>(dft_smem + kDftBK * kDftBM);
  float (*Xs)[kDftBK + 2 * kMaxMeanHalf + 1] =
      reinterpret_cast<float (*)[kDftBK + 2 * kMaxMeanHalf + 1]>(dft_smem + kDftBK * kDftBM + kDftBK * kDftBN);
  __shared__ float red_max[8];
  __shared__ float cm[kDftBM];

  const int tid = threadIdx.x;
  // row means of y: (sum_j w_j x[m,j] - sum_j w_j a_j - (m - mbar) sum_j w_j b_j) / N
  if (tid < kDftBM) {
    const int m = m0 + tid;
    float c = 0.f;
    if (m < F.M) {
      float rsum = 0.f, A = 0.f, Bv = 0.f;
      for (int sI = 0; sI < F.n_strips; ++sI) {  // fixed order: deterministic
        rsum += __ldg(&F.rowpart[(long long)sI * F.M + m]);
        const float2 ab = __ldg(&F.strip_ab[sI]);
        A += ab.x;
        Bv += ab.y;
      }
      c = (rsum - A - ((float)m - F.mbar) * Bv) / (float)F.N;
    }
    cm[tid] = c;
  }
  __syncthreads();
  const int tm = tid >> 4, tn = tid & 15;
  // two-level accumulation: each K step of 32 samples sums into `part`,
  // which is then added into `acc` with a compensation term (Kahan), so the
  // rounding error does not grow with the large oscillating partial sums of
  // strongly modulated rows
  float acc[8][4], comp[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = comp[i][j] = 0.f;
  float ymax = 0.f;

  for (int n0 = kbeg; n0 < kend; n0 += kDftBK) {
    __syncthreads();
    // stage x' for columns n0 - h .. n0 + BK + h - 1
    const int width = kDftBK + 2 * h;
    for (int idx = tid; idx < kDftBM * width; idx += 256) {
      const int r = idx / width, cc = idx % width;
      const int m = m0 + r, n = n0 - h + cc;
      float v = 0.f;
      if (m < F.M && n >= 0 && n < F.N) {
        const float2 st = __ldg(&F.stats[n]);
        const float xv = __ldg(F.x + (long long)m * F.ldx + n);
        v = xv - st.x - st.y * ((float)m - F.mbar);
      }
      Xs[r][cc] = v;
    }
    // twiddle tile
    for (int idx = tid; idx < kDftBK * kDftBN; idx += 256) {
      const int k = idx / kDftBN, j = idx % kDftBN;
      const int n = n0 + k, col = j0 + j;
      Bs[k][j] = (n < kend && col < twoC) ? __ldg(F.W + (long long)n * F.ldw + col) : 0.f;
    }
    __syncthreads();
    // mean filter: thread -> row r = tid / 2, samples half (tid & 1) * 16 .. + 15
    {
      const int r = tid >> 1;
      const int kb = (tid & 1) * (kDftBK / 2);
      const bool row_ok = (m0 + r) < F.M;
      for (int kk = 0; kk < kDftBK / 2; ++kk) {
        const int k = kb + kk;
        const int n = n0 + k;
        float y = 0.f;
        if (row_ok && n < kend) {
          float s = 0.f;
          for (int d = 0; d <= 2 * h; ++d) s += Xs[r][k + d];
          const int lo = max(n - h, 0), hi = min(n + h, F.N - 1);
          y = s / (float)(hi - lo + 1);
          ymax = fmaxf(ymax, fabsf(y));
          y -= cm[r];
        }
        As[k][r] = y;
      }
    }
    __syncthreads();
    float part[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
#pragma unroll 8
    for (int k = 0; k < kDftBK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[k][tm * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[k][tm * 8 + 4]);
      const float4 bb = *reinterpret_cast<const float4*>(&Bs[k][tn * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = fmaf(a[i], bv[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float y = part[i][j] - comp[i][j];
        const float t = acc[i][j] + y;
        comp[i][j] = __fsub_rn(__fsub_rn(t, acc[i][j]), y);
        acc[i][j] = t;
      }
  }
  (void)XW;

  // frame max |y| (only one column of output tiles needs to report it)
  if (nt == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    if ((tid & 31) == 0) red_max[tid >> 5] = ymax;
    __syncthreads();
    if (tid == 0) {
      float m = red_max[0];
      for (int w = 1; w < 8; ++w) m = fmaxf(m, red_max[w]);
      atomicMax(F.ymax, __float_as_uint(m));
    }
  }

  if (F.splitk == 1) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = m0 + tm * 8 + i;
      if (m >= F.M) continue;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int col = j0 + tn * 4 + 2 * p;
        if (col < twoC) {
          float re = acc[i][2 * p];
          const float im = acc[i][2 * p + 1];
          if (col == 0 && F.c0 == 0) re = fmaf((float)F.N, cm[tm * 8 + i], re);  // bin 0 gets the mean back
          F.map[(long long)m * F.ld_map + (col >> 1)] = sqrtf(fmaf(re, re, im * im));
        }
      }
    }
    return;
  }

  // split-K: write partials, the last CTA of this output tile reduces them
  float* part = F.kpart + (long long)ks * F.M * F.ldk;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + tm * 8 + i;
    if (m >= F.M) continue;
    const int col = j0 + tn * 4;
    if (col < twoC) {
      *reinterpret_cast<float4*>(part + (long long)m * F.ldk + col) =
          make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
  }
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned old = atomicAdd(&F.tile_cnt[rem], 1u);
    is_last = (old == (unsigned)F.splitk - 1u);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int idx = tid; idx < kDftBM * (kDftBN / 2); idx += 256) {
    const int r = idx / (kDftBN / 2), p = idx % (kDftBN / 2);
    const int m = m0 + r, col = j0 + 2 * p;
    if (m >= F.M || col >= twoC) continue;
    float re = 0.f, im = 0.f;
    for (int s = 0; s < F.splitk; ++s) {  // fixed order: deterministic
      const float2 v = __ldcg(reinterpret_cast<const float2*>(F.kpart + ((long long)s * F.M + m) * F.ldk + col));
      re += v.x;
      im += v.y;
    }
    if (col == 0 && F.c0 == 0) re = fmaf((float)F.N, cm[r], re);  // bin 0 gets the mean back
    F.map[(long long)m * F.ld_map + (col >> 1)] = sqrtf(fmaf(re, re, im * im));
  }
  if (tid == 0) F.tile_cnt[rem] = 0u;
}

__global__ void __launch_bounds__(256) k_normalise(const __grid_constant__ PreBatch b) {
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_norm);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_norm;
  const float mx = __uint_as_float(__ldcg(F.ymax));
  if (!(mx > 0.f)) return;
  const long long total = (long long)F.M * F.C;
  for (long long i = (long long)local * 256 + threadIdx.x; i < total; i += (long long)F.n_norm * 256) {
    const int m = (int)(i / F.C), j = (int)(i % F.C);
    float* p = F.map + (long long)m * F.ld_map + j;
    *p = *p / mx;
  }
}

__global__ void k_twiddles(float* W, long long ldw, int N, int c0, int C) {
  const long long total = (long long)N * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i / C), j = (int)(i % C);
    const long long t = ((long long)(c0 + j) * n) % N;
    double s, c;
    sincospi(2.0 * (double)t / (double)N, &s, &c);
    W[(long long)n * ldw + 2 * j] = (float)c;
    W[(long long)n * ldw + 2 * j + 1] = (float)(-s);
  }
}

}  // namespace

cudaError_t launch_colstats(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  k_colstats<<<blocks, 256, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_band_dft(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = sizeof(float) * (kDftBK * kDftBM + kDftBK * kDftBN + kDftBM * (kDftBK + 2 * kMaxMeanHalf + 1));
  cudaError_t e = ensure_smem(reinterpret_cast<const void*>(&k_band_dft), smem);
  if (e != cudaSuccess) return e;
  k_band_dft<<<blocks, 256, smem, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_normalise(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  k_normalise<<<blocks, 256, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_twiddles(float* W, long long ldw, int N, int c0, int C, cudaStream_t s) {
  const long long total = (long long)N * C;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_twiddles<<<blocks, 256, 0, s>>>(W, ldw, N, c0, C);
  return cudaGetLastError();
}

}  // namespace rcfar
