// q2_expectation_noalloc: the energy of q2_expectation without device allocation.
//
// The scratch that q2_expectation takes from stream-ordered temporary memory
// (per-CTA partial sums and the two result slots) and the Hamiltonian's
// device tables (group and block descriptors, LUT) live here in one
// file-scope static device array of Q2_NOALLOC_SCRATCH_BYTES.  Host code
// only ever uses the array's device address, looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/q2.h"
#include "kernels.h"
#include "q2_internal.h"

namespace q2 {
q2_status ham_host_plan(const q2_ham *h, q2_dtype d, const HamPlan **plan, int *chunk);
int ham_qubits(const q2_ham *h);
q2_status set_error(q2_status s, const char *msg);
}  // namespace q2

using namespace q2;

static __device__ __align__(256) unsigned char q2_noalloc_scratch[Q2_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
q2_status scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(Q2_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(Q2_ERR_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, q2_noalloc_scratch);
    if (e != cudaSuccess || !p) return set_error(Q2_ERR_CUDA, "cudaGetSymbolAddress failed for the no-allocation scratch");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return Q2_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename R>
cudaError_t run(const R *psi, int n, const HamPlan &h, const GroupDesc *groups, const BlockDesc *blocks,
                const void *lut, double *partial, int grid, double *out, cudaStream_t st) {
  for (size_t i = 0; i < h.passes.size(); ++i) {
    cudaError_t e = launch_expect<R>(psi, n, h.passes[i], groups, blocks, lut, partial, grid, i == 0, st);
    if (e != cudaSuccess) return e;
  }
  return launch_reduce_pairs(partial, grid, out, st);
}

}  // namespace

extern "C" q2_status q2_expectation_noalloc(const void *psi_dev, int n, q2_dtype dtype, const q2_ham *ham,
                                            double *energy_out, double *norm_out, void *stream) {
  if (dtype != Q2_C64 && dtype != Q2_C128) return set_error(Q2_ERR_INVALID, "unknown dtype");
  if (n < 1 || n > (dtype == Q2_C64 ? 34 : 33)) return set_error(Q2_ERR_INVALID, "qubit count out of range");
  if (!ham || !energy_out) return set_error(Q2_ERR_INVALID, "NULL argument");
  if (ham_qubits(ham) != n) return set_error(Q2_ERR_INVALID, "Hamiltonian qubit count differs from n");
  if (!psi_dev || ((uintptr_t)psi_dev % 16) != 0)
    return set_error(Q2_ERR_INVALID, "psi must be a 16-byte aligned device pointer");
  const HamPlan *hp = nullptr;
  int chunk = 0;
  q2_status s = ham_host_plan(ham, dtype, &hp, &chunk);
  if (s != Q2_OK) return s;
  const int amp = dtype == Q2_C64 ? 8 : 16;
  const int C = std::min(chunk, hp->T);
  const int grid = dtype == Q2_C64 ? expect_grid<float>(n, hp->T, C) : expect_grid<double>(n, hp->T, C);
  // scratch layout: [out 2][partials 2*grid][groups][blocks][lut]
  const size_t o_part = 256;
  const size_t o_groups = o_part + up256(sizeof(double) * 2 * (size_t)grid);
  const size_t o_blocks = o_groups + up256(sizeof(GroupDesc) * hp->groups.size());
  const size_t o_lut = o_blocks + up256(sizeof(BlockDesc) * hp->blocks.size());
  const size_t total = o_lut + up256((size_t)amp * (size_t)hp->lut_entries);
  if (total > Q2_NOALLOC_SCRATCH_BYTES) {
    const std::string msg = "Hamiltonian tables and partial sums need " + std::to_string(total) +
                            " bytes; the no-allocation scratch holds " + std::to_string(Q2_NOALLOC_SCRATCH_BYTES);
    return set_error(Q2_ERR_INVALID, msg.c_str());
  }
  void *base_v = nullptr;
  if ((s = scratch_address(&base_v)) != Q2_OK) return s;
  unsigned char *base = static_cast<unsigned char *>(base_v);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  std::vector<float> lutf;
  const void *lut_src = hp->lut2.data();
  if (dtype == Q2_C64) {
    lutf.resize(hp->lut2.size());
    for (size_t i = 0; i < lutf.size(); ++i) lutf[i] = (float)hp->lut2[i];
    lut_src = lutf.data();
  }
  cudaError_t e = cudaMemcpyAsync(base + o_groups, hp->groups.data(), sizeof(GroupDesc) * hp->groups.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !hp->blocks.empty())
    e = cudaMemcpyAsync(base + o_blocks, hp->blocks.data(), sizeof(BlockDesc) * hp->blocks.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && hp->lut_entries > 0)
    e = cudaMemcpyAsync(base + o_lut, lut_src, (size_t)amp * (size_t)hp->lut_entries, cudaMemcpyHostToDevice, st);
  double *out = reinterpret_cast<double *>(base);
  double *partial = reinterpret_cast<double *>(base + o_part);
  const GroupDesc *groups = reinterpret_cast<const GroupDesc *>(base + o_groups);
  const BlockDesc *blocks = reinterpret_cast<const BlockDesc *>(base + o_blocks);
  if (e == cudaSuccess)
    e = dtype == Q2_C64
            ? run<float>(static_cast<const float *>(psi_dev), n, *hp, groups, blocks, base + o_lut, partial, grid, out, st)
            : run<double>(static_cast<const double *>(psi_dev), n, *hp, groups, blocks, base + o_lut, partial, grid, out,
                          st);
  double host_out[2] = {0.0, 0.0};
  unsigned waits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, out, sizeof(host_out), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = read_wait_timeouts_async(&waits, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return set_error(Q2_ERR_CUDA, cudaGetErrorString(e));
  if (waits) {
    clear_wait_timeouts(st);
    return set_error(Q2_ERR_TIMEOUT, "a device wait for a tile copy timed out");
  }
  *energy_out = host_out[0] / host_out[1];
  if (norm_out) *norm_out = host_out[1];
  return Q2_OK;
}
