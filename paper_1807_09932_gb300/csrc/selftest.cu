// Self-test of the bounded device wait that every pipeline wait of the library uses.
//
// One thread initialises an mbarrier that expects one arrival, then waits on it with the same
// helper the evaluator uses for its TMA stages (mbar_wait_bounded, bounded by %globaltimer).
// Nothing ever arrives, so the wait expires after `timeout_ns`; the kernel records the expiry in
// a device word and returns normally. This exercises the timeout path end to end without any
// fault, trap or unbounded spin, and leaves the context usable.
#include <string>

#include "device_common.cuh"
#include "ebic.h"
#include "ebic_internal.h"

namespace ebic {
namespace {

__global__ void wait_timeout_kernel(uint64_t timeout_ns, uint32_t* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  dev::mbar_init(&bar, 1);
  dev::fence_barrier_init();
  const bool done = dev::mbar_wait_bounded(&bar, 0, timeout_ns);
  *out = done ? 0u : kErrTimeout;
}

}  // namespace
}  // namespace ebic

using namespace ebic;

extern "C" int ebic_selftest_wait_timeout(uint64_t timeout_ns, void* stream) {
  if (timeout_ns == 0 || timeout_ns > 100000000ull)
    return set_last_error(EBIC_ERR_INVALID_ARG, "timeout_ns must be in (0, 1e8]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* d = nullptr;
  uint32_t h = 0;
  cudaError_t e = cudaMallocAsync(&d, sizeof(uint32_t), s);
  if (e == cudaSuccess) {
    count_launch();
    wait_timeout_kernel<<<1, 32, 0, s>>>(timeout_ns, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, s);
    cudaError_t f = cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = f;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return set_last_error(EBIC_ERR_CUDA, (std::string("selftest: ") + cudaGetErrorString(e)).c_str());
  }
  if (h & kErrTimeout)
    return set_last_error(EBIC_ERR_DEVICE_TIMEOUT, "bounded device wait expired (as intended)");
  return EBIC_OK;
}
