// Self-test of the bounded device waits (failure detection without a fault).
//
// Every kernel of the library that waits (on an mbarrier phase: copies,
// tensor-core work) gives up after a bounded number of polls, records
// kStatusTimeout in the handle's status word and finishes normally, so a
// lost completion shows up as RCFAR_ERR_TIMEOUT from rcfar_get_error and the
// context stays usable. rcfar_selftest_wait runs that path on purpose: one
// warp waits on an mbarrier whose phase nothing completes.
#include "rcfar_internal.cuh"
#include "async_copy.cuh"

namespace {

__global__ void k_wait_selftest(unsigned polls, int* status) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    rcfar::mbar_init(rcfar::smem_u32(&bar), 1);  // expects one arrival; none comes
    rcfar::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !rcfar::mbar_wait_bounded(rcfar::smem_u32(&bar), 0u, polls))
    atomicOr(status, rcfar::kStatusTimeout);
}

}  // namespace

extern "C" rcfar_status rcfar_selftest_wait(int32_t device, int32_t polls) {
  if (polls <= 0 || polls > (1 << 20)) return RCFAR_ERR_INVALID_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return RCFAR_ERR_CUDA;
  int* st = nullptr;
  int host = 0;
  rcfar_status out = RCFAR_ERR_CUDA;
  if (cudaMalloc(&st, sizeof(int)) == cudaSuccess && cudaMemset(st, 0, sizeof(int)) == cudaSuccess) {
    k_wait_selftest<<<1, 32>>>((unsigned)polls, st);
    if (cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(&host, st, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
      out = (host & rcfar::kStatusTimeout) ? RCFAR_ERR_TIMEOUT : RCFAR_OK;
  }
  if (st) cudaFree(st);
  cudaSetDevice(prev);
  return out;
}
