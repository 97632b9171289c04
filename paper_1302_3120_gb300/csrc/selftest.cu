// selftest.cu — self-test of the bounded device-side wait.
//
// The only waits in the library's kernels are the mbarrier waits of the column-pass
// cluster exchanges (col_pass.cuh), each limited in time so that a peer CTA that never
// signals cannot hang the GPU: the kernel latches a timeout and returns.  This entry
// point runs that wait on an mbarrier that nothing arrives at, so the limit runs out, and
// reports what the kernel saw.
#include "col_pass.cuh"

namespace csar {

__global__ void k_wait_selftest(uint32_t* out, unsigned long long limit_ns) {
  __shared__ uint64_t mb;
  if (threadIdx.x == 0) mbar_init(smem_addr(&mb), 1u);
  __syncthreads();
  // nothing arrives: phase 0 never completes
  const bool done = mbar_wait_for(smem_addr(&mb), 0u, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0) out[0] = done ? 0u : 1u;
}

}  // namespace csar

using namespace csar;

extern "C" csar_status csar_selftest_wait_timeout(int32_t limit_ms) {
  if (limit_ms <= 0 || limit_ms > 10000)
    return set_error(CSAR_E_INVALID, "csar_selftest_wait_timeout: limit_ms must be in 1..10000");
  uint32_t* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(uint32_t));
  if (e != cudaSuccess) return set_error(CSAR_E_OOM, cudaGetErrorString(e));
  uint32_t h = 0;
  e = cudaMemset(d, 0, sizeof(uint32_t));
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 64>>>(d, (unsigned long long)limit_ms * 1000000ull);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return set_error(CSAR_E_CUDA, cudaGetErrorString(e));
  if (h) return set_error(CSAR_E_TIMEOUT, "bounded wait ran out (expected: nothing arrived)");
  return set_error(CSAR_E_INTERNAL, "the wait completed although nothing arrived");
}
