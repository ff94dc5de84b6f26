// Self-test of the bounded device waits used by the level sweeps: every block
// of a small cooperative launch waits at a level barrier whose count can never
// reach the number of blocks (nothing arrives).  Each wait gives up after
// max_spin polls, records ERRBIT_TIMEOUT and returns, so the launch ends and
// the context stays usable; the host reads the error word.
#include "sweepsync.cuh"

namespace ggp {
namespace {

__global__ void barrier_timeout_kernel(LevelBarrier lb, uint32_t* reached) {
  __shared__ int s_flag;
  // nobody arrives at level 0, so gridDim.x + 1 arrivals never happen
  if (lb.wait(0, gridDim.x + 1, &s_flag)) return;
  if (threadIdx.x == 0) atomicAdd(reached, 1u);  // not reached while the bound works
}

}  // namespace
}  // namespace ggp

using namespace ggp;

extern "C" int graphgp_selftest_wait_timeout(int64_t max_spin, void* stream) {
  if (max_spin < 1 || max_spin > ((int64_t)1 << 30)) return GRAPHGP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch sc(s);
  uint32_t* words = nullptr;  // [0] count, [1] error word, [2] reached
  GGP_TRY(sc.alloc(&words, 4));
  GGP_CUDA(cudaMemsetAsync(words, 0, 4 * sizeof(uint32_t), s));
  LevelBarrier lb{words, words + 1, max_spin};
  uint32_t* reached = words + 2;
  void* args[] = {(void*)&lb, (void*)&reached};
  GGP_CUDA(cudaLaunchCooperativeKernel((const void*)barrier_timeout_kernel, dim3(2), dim3(64), args,
                                       0, s));
  uint32_t h[4] = {0, 0, 0, 0};
  GGP_CUDA(cudaMemcpyAsync(h, words, sizeof(h), cudaMemcpyDeviceToHost, s));
  GGP_CUDA(cudaStreamSynchronize(s));
  if (h[2] != 0) return GRAPHGP_ERR_INVALID;  // a wait passed without arrivals
  return (h[1] & ERRBIT_TIMEOUT) ? GRAPHGP_ERR_TIMEOUT : GRAPHGP_OK;
}

// Target of the device code actually loaded: binaryVersion of one of the
// library's kernels (major * 10 + minor, 103 for sm_103a).
extern "C" int graphgp_binary_version(int* version) {
  if (!version) return GRAPHGP_ERR_INVALID;
  cudaFuncAttributes a;
  GGP_CUDA(cudaFuncGetAttributes(&a, (const void*)barrier_timeout_kernel));
  *version = a.binaryVersion;
  return GRAPHGP_OK;
}
