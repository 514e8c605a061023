// k_selftest.cu — self-test of the bounded device-side waits: one CTA waits on
// an mbarrier phase that nothing completes, with the same time-bounded wait the
// tensor-core and cluster kernels use, gives up after limit_ns, records the
// timeout in an error word and returns; the context stays usable.
#include "lcf_internal.cuh"
#include "tc_util.cuh"

namespace lcf {

__global__ void selftest_wait_kernel(unsigned long long limit_ns, int* err, unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) tc::mbar_init(&bar, 1);   // expects one arrival; none comes
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint64_t t0 = tc::globaltimer_ns();
    const bool ok = tc::mbar_wait(&bar, 0, limit_ns);
    *waited_ns = tc::globaltimer_ns() - t0;
    if (!ok) atomicOr(err, 1);
  }
}

}  // namespace lcf

extern "C" lcf_status lcf_selftest_wait_timeout(int device, unsigned long long limit_ns, double* waited_s) {
  if (limit_ns == 0 || limit_ns > 2000000000ull) return LCF_EINVAL;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return LCF_EINVAL;
  int* d_err = nullptr;
  unsigned long long* d_ns = nullptr;
  lcf_status s = LCF_OK;
  if (cudaMalloc((void**)&d_err, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&d_ns, sizeof(unsigned long long)) != cudaSuccess) {
    s = LCF_ENOMEM;
  } else {
    int err = 0;
    unsigned long long ns = 0;
    cudaMemset(d_err, 0, sizeof(int));
    lcf::selftest_wait_kernel<<<1, 32>>>(limit_ns, d_err, d_ns);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&ns, d_ns, sizeof(ns), cudaMemcpyDeviceToHost) != cudaSuccess) {
      s = LCF_ECUDA;
    } else {
      if (waited_s) *waited_s = ns * 1e-9;
      s = err ? LCF_ETIMEOUT : LCF_OK;
    }
  }
  if (d_err) cudaFree(d_err);
  if (d_ns) cudaFree(d_ns);
  cudaSetDevice(prev);
  return s;
}
