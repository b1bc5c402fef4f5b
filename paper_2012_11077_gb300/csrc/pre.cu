// Preprocessing kernels of the radar chain (paper Sec. II.A).
//
//   k_colstats : per trace n, the least-squares line over fast time m
//                (a_n = mean, b_n = slope about mbar) -- "DC-shift removal and
//                linear trend subtraction"; also the pieces of each row's
//                slow-time mean of y (see k_ysplit).
//   k_ysplit   : detrend + slow-time mean filter + max|y|; writes y minus
//                its row mean, split into TF32 head and tail.
//   k_band_dft : band DFT as a GEMM of y [M x N] with the twiddle matrix
//                [N x 2C] on the tensor cores (split TF32, three products),
//                then the magnitude; split-K for small frames. Each row's
//                mean c_m was removed from y and N c_m is added back to bin
//                0 only: a constant contributes to no other bin, and removing
//                it keeps the FP32 rounding of the large per-range DC offsets
//                out of the small bins.
//   k_normalise: divide the map by max|y| ("then normalized"); the DFT is
//                linear, so scaling its magnitude equals transforming y/max|y|.
//   k_twiddles : twiddle matrix W[n][2j] = cos(2 pi t/N), W[n][2j+1] = -sin,
//                t = (c0 + j) n mod N, computed once per (N, band) in FP64 and
//                stored split into TF32 head and tail.
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

__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x as a TF32 head plus a TF32 tail (about 22 significant bits together).
__device__ __forceinline__ float2 split_tf32(float x) {
  const unsigned hi = to_tf32(x);
  const unsigned lo = to_tf32(x - __uint_as_float(hi));
  return make_float2(__uint_as_float(hi), __uint_as_float(lo));
}

// y pass: one warp per frame row, 256 samples per CTA column block.
//   x'[m,n] = x[m,n] - a_n - b_n (m - mbar)       (detrend)
//   y[m,n]  = mean of x'[m, n-h..n+h] in [0, N)    (mean filter)
// records max |y| and writes y - c_m, where c_m is the row's slow-time mean
// (a constant only reaches bin 0; removing it keeps the FP32 rounding of the
// large per-range offsets out of the other bins), split into TF32 head and
// tail for the tensor-core product. Samples N..npad-1 are written as 0.
__global__ void __launch_bounds__(256) k_ysplit(const __grid_constant__ PreBatch b) {
  const int fi = find_item(b.f, b.n, (int)blockIdx.x, &PreFrameDev::item_y);
  const PreFrameDev& F = b.f[fi];
  const int local = (int)blockIdx.x - F.item_y;
  const int rb = local / F.ycols, cbk = local - rb * F.ycols;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = rb * kYRows + warp;
  const int n0 = cbk * kYCols;
  const int h = F.h, N = F.N;
  __shared__ float seg[kYRows][kYCols + 2 * kMaxMeanHalf];
  __shared__ float red[kYRows];
  float ymax = 0.f;
  if (m < F.M) {
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
    const float cmv = (rs - A - dm * Bv) / (float)N;
    if (cbk == 0 && lane == 0) F.rowmean[m] = cmv;
    // x' over [n0 - h, n0 + 256 + h)
    const float* xr = F.x + (long long)m * F.ldx;
    for (int i = lane; i < kYCols + 2 * h; i += 32) {
      const int n = n0 - h + i;
      float v = 0.f;
      if (n >= 0 && n < N) {
        const float2 st = __ldg(&F.stats[n]);
        v = __ldg(xr + n) - st.x - st.y * dm;
      }
      seg[warp][i] = v;
    }
    __syncwarp();
    float2* yr = F.ysplit + (long long)m * F.npad;
#pragma unroll
    for (int q = 0; q < kYCols / 32; ++q) {
      const int i = lane + 32 * q;
      const int n = n0 + i;
      if (n >= F.npad) break;
      float2 out = make_float2(0.f, 0.f);
      if (n < N) {
        float acc = 0.f;
        for (int d = 0; d <= 2 * h; ++d) acc += seg[warp][i + d];
        const int lo = max(n - h, 0), hi = min(n + h, N - 1);
        const float y = acc / (float)(hi - lo + 1);
        ymax = fmaxf(ymax, fabsf(y));
        out = split_tf32(y - cmv);
      }
      yr[n] = out;
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

// D += A * B for one 16x8x8 TF32 tile (FP32 accumulate).
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  const int src_bytes = valid ? 16 : 0;  // 0: the 16 bytes are zero-filled, nothing is read
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory strides (in float2) of the GEMM tiles, padded so that the
// fragment loads of a warp fall on distinct banks.
constexpr int kAS = kDftBK + 4;  // A tile [BM][BK]
constexpr int kBS = kDftBN + 4;  // B tile [BK][BN]

// Band DFT as a GEMM on the tensor cores: ysplit [M x npad] times the
// twiddle plan [npad x 2C], then the magnitude of each (cos, -sin) column
// pair. CTA tile kDftBM rows x kDftBN real outputs; K steps of kDftBK samples
// are staged with cp.async into a two-stage ring. The 8 warps (4 along M x 2
// along N, 32 x 32 each) issue m16n8k8 TF32 MMAs on the split operands:
// head*head + head*tail + tail*head (about 22 bits per product). Each K
// step's partial sum is added to the running sum with Kahan compensation.
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
  const int kend = min(F.npad, kbeg + F.kper);

  extern __shared__ __align__(16) float2 gsm[];
  float2* As = gsm;                          // [2][BM][kAS]
  float2* Bs = gsm + 2 * kDftBM * kAS;       // [2][BK][kBS]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = (warp & 3) * 32, wn = (warp >> 2) * 32;

  // one K step: A 128 x 32 float2 (2048 16-byte chunks), B 32 x 64 float2 (1024 chunks)
  auto stage = [&](int buf, int k0) {
    float2* a = As + buf * kDftBM * kAS;
    float2* bb = Bs + buf * kDftBK * kBS;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int id = tid + 256 * q;
      const int r = id >> 4, c2 = (id & 15) * 2;  // 16 chunks of 2 float2 per row
      const int m = m0 + r;
      const bool ok = m < F.M;
      const float2* src = F.ysplit + (long long)(ok ? m : 0) * F.npad + k0 + c2;
      cp_async16(a + r * kAS + c2, src, ok);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int id = tid + 256 * q;
      const int k = id >> 5, c2 = (id & 31) * 2;  // 32 chunks of 2 float2 per row
      const float2* src = F.W2 + (long long)(k0 + k) * F.ldw + j0 + c2;
      cp_async16(bb + k * kBS + c2, src, true);
    }
    cp_async_commit();
  };

  float acc[2][4][4], comp[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = comp[i][j][e] = 0.f;

  stage(0, kbeg);
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += kDftBK, buf ^= 1) {
    if (k0 + kDftBK < kend) {
      stage(buf ^ 1, k0 + kDftBK);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float2* a = As + buf * kDftBM * kAS;
    const float2* bb = Bs + buf * kDftBK * kBS;
    float part[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) part[i][j][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < kDftBK; kk += 8) {
      unsigned ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int mr = wm + i * 16 + g;
        const float2 v0 = a[mr * kAS + kk + t], v1 = a[(mr + 8) * kAS + kk + t];
        const float2 v2 = a[mr * kAS + kk + t + 4], v3 = a[(mr + 8) * kAS + kk + t + 4];
        ah[i][0] = __float_as_uint(v0.x); al[i][0] = __float_as_uint(v0.y);
        ah[i][1] = __float_as_uint(v1.x); al[i][1] = __float_as_uint(v1.y);
        ah[i][2] = __float_as_uint(v2.x); al[i][2] = __float_as_uint(v2.y);
        ah[i][3] = __float_as_uint(v3.x); al[i][3] = __float_as_uint(v3.y);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int nc = wn + j * 8 + g;
        const float2 u0 = bb[(kk + t) * kBS + nc], u1 = bb[(kk + t + 4) * kBS + nc];
        bh[j][0] = __float_as_uint(u0.x); bl[j][0] = __float_as_uint(u0.y);
        bh[j][1] = __float_as_uint(u1.x); bl[j][1] = __float_as_uint(u1.y);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          mma_tf32(part[i][j], al[i], bh[j]);
          mma_tf32(part[i][j], ah[i], bl[j]);
          mma_tf32(part[i][j], ah[i], bh[j]);
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float y = part[i][j][e] - comp[i][j][e];
          const float s2 = acc[i][j][e] + y;
          comp[i][j][e] = __fsub_rn(__fsub_rn(s2, acc[i][j][e]), y);
          acc[i][j][e] = s2;
        }
    __syncthreads();  // the next stage() overwrites this buffer
  }

  // fragment (i, j): rows wm + 16 i + g (+8), real columns wn + 8 j + 2 t (+1)
  if (F.splitk == 1) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int hlf = 0; hlf < 2; ++hlf) {
          const int m = m0 + wm + i * 16 + g + 8 * hlf;
          const int col = j0 + wn + j * 8 + 2 * t;
          if (m >= F.M || col >= twoC) continue;
          float re = acc[i][j][2 * hlf];
          const float im = acc[i][j][2 * hlf + 1];
          if (col == 0 && F.c0 == 0) re = fmaf((float)F.N, __ldg(&F.rowmean[m]), re);  // bin 0 gets the mean back
          F.map[(long long)m * F.ld_map + (col >> 1)] = sqrtf(fmaf(re, re, im * im));
        }
    return;
  }

  // split-K: write partials, the last CTA of this output tile reduces them
  float* part_out = F.kpart + (long long)ks * F.M * F.ldk;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int hlf = 0; hlf < 2; ++hlf) {
        const int m = m0 + wm + i * 16 + g + 8 * hlf;
        const int col = j0 + wn + j * 8 + 2 * t;
        if (m >= F.M || col >= twoC) continue;
        *reinterpret_cast<float2*>(part_out + (long long)m * F.ldk + col) =
            make_float2(acc[i][j][2 * hlf], acc[i][j][2 * hlf + 1]);
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
    for (int sp = 0; sp < F.splitk; ++sp) {  // fixed order: deterministic
      const float2 v = __ldcg(reinterpret_cast<const float2*>(F.kpart + ((long long)sp * F.M + m) * F.ldk + col));
      re += v.x;
      im += v.y;
    }
    if (col == 0 && F.c0 == 0) re = fmaf((float)F.N, __ldg(&F.rowmean[m]), re);  // bin 0 gets the mean back
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

__global__ void k_twiddles(float2* W2, long long ldw, int N, int c0, int C) {
  const long long total = (long long)N * C;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int n = (int)(i / C), j = (int)(i % C);
    const long long t = ((long long)(c0 + j) * n) % N;
    double s, c;
    sincospi(2.0 * (double)t / (double)N, &s, &c);
    W2[(long long)n * ldw + 2 * j] = split_tf32((float)c);
    W2[(long long)n * ldw + 2 * j + 1] = split_tf32((float)(-s));
  }
}

}  // namespace

cudaError_t launch_colstats(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  k_colstats<<<blocks, 256, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_ysplit(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  k_ysplit<<<blocks, 256, 0, s>>>(b);
  return cudaGetLastError();
}

cudaError_t launch_band_dft(const PreBatch& b, int blocks, cudaStream_t s) {
  if (blocks <= 0) return cudaSuccess;
  const size_t smem = sizeof(float2) * (2 * kDftBM * kAS + 2 * kDftBK * kBS);
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

cudaError_t launch_twiddles(float2* W2, long long ldw, int N, int c0, int C, cudaStream_t s) {
  const long long total = (long long)N * C;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_twiddles<<<blocks, 256, 0, s>>>(W2, ldw, N, c0, C);
  return cudaGetLastError();
}

}  // namespace rcfar
