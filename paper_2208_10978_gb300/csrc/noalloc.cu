// q2_expectation_noalloc: the energy of q2_expectation without device allocation.
//
// The scratch that q2_expectation takes from stream-ordered temporary memory
// (per-CTA partial sums, the two result slots and the call's fault word) and
// the Hamiltonian's device tables (group and block descriptors, LUT) live
// here in one file-scope static device array of Q2_NOALLOC_SCRATCH_BYTES.
// Host code only ever uses the array's device address, which
// cudaGetSymbolAddress gives for the current device; it is looked up once per
// CUDA context (the first call on each device, and again if that device's
// context is destroyed and created anew, since the module and its array are
// then loaded at a new address).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
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
bool lean_expect_enabled();
}  // namespace q2

using namespace q2;

static __device__ __align__(256) unsigned char q2_noalloc_scratch[Q2_NOALLOC_SCRATCH_BYTES];

namespace {

// Driver calls that name the calling thread's current context, reached through
// the runtime so that the library needs no link against the driver library.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

std::mutex g_mu;
std::map<unsigned long long, void *> g_addr;   // context id -> device address of the scratch
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_ctx_fns_tried = false;

// Unique id of the current context (ids are never reused within a process); false if unknown.
bool current_context_id(unsigned long long *id) {
  if (!g_ctx_fns_tried) {
    g_ctx_fns_tried = true;
    cudaDriverEntryPointQueryResult q1, q2r;
    void *f1 = nullptr, *f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2r) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2r == cudaDriverEntryPointSuccess) {
      g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
  }
  if (!g_ctx_current || !g_ctx_id) return false;
  void *ctx = nullptr;
  if (g_ctx_current(&ctx) != 0 || !ctx) return false;
  return g_ctx_id(ctx, id) == 0;
}

// Device address of the scratch array in the current context.
q2_status scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaSetDevice(dev);   // makes the device's primary context current
  if (e != cudaSuccess) return set_error(Q2_ERR_CUDA, cudaGetErrorString(e));
  std::lock_guard<std::mutex> g(g_mu);
  unsigned long long id = 0;
  const bool keyed = current_context_id(&id);
  if (keyed) {
    auto it = g_addr.find(id);
    if (it != g_addr.end()) {
      *out = it->second;
      return Q2_OK;
    }
  }
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, q2_noalloc_scratch);
  if (e != cudaSuccess || !p) return set_error(Q2_ERR_CUDA, "cudaGetSymbolAddress failed for the no-allocation scratch");
  if (keyed) g_addr[id] = p;   // without a context id the address is looked up on every call
  *out = p;
  return Q2_OK;
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename R>
cudaError_t run(const R *psi, int n, const HamPlan &h, const GroupDesc *groups, const BlockDesc *blocks,
                const void *lut, double *partial, int grid, double *out, unsigned *fault, cudaStream_t st) {
  if (h.passes.empty()) {   // no terms (or a shard without passes): energy 0, norm by a dot product
    const int dg = dot_grid<R>(n);
    cudaError_t e = launch_dot<R>(psi, psi, n, partial, dg, st);
    if (e == cudaSuccess) e = launch_reduce_pairs(partial, dg, out, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(double), st);
    return e;
  }
  for (size_t i = 0; i < h.passes.size(); ++i) {
    const bool lean = lean_expect_enabled() && i < h.pass_lean.size() && h.pass_lean[i];
    cudaError_t e =
        launch_expect<R>(psi, n, h.passes[i], groups, blocks, lut, partial, grid, i == 0, fault, lean, st);
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
  const int slots = std::max(grid, dtype == Q2_C64 ? dot_grid<float>(n) : dot_grid<double>(n));
  // scratch layout: [out 2][fault word][partials 2*slots][groups][blocks][lut]
  const size_t o_part = 256;
  const size_t o_groups = o_part + up256(sizeof(double) * 2 * (size_t)slots);
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
  if (dtype == Q2_C64) {   // (R, R) for REAL and DIAG groups, as the handle's own device LUT
    lutf = hp->lut_f32();
    lut_src = lutf.data();
  }
  double *out = reinterpret_cast<double *>(base);
  unsigned *fault = reinterpret_cast<unsigned *>(base + 2 * sizeof(double));
  cudaError_t e = cudaMemsetAsync(base, 0, 2 * sizeof(double) + sizeof(unsigned), st);   // sums and fault word
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + o_groups, hp->groups.data(), sizeof(GroupDesc) * hp->groups.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !hp->blocks.empty())
    e = cudaMemcpyAsync(base + o_blocks, hp->blocks.data(), sizeof(BlockDesc) * hp->blocks.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && hp->lut_entries > 0)
    e = cudaMemcpyAsync(base + o_lut, lut_src, (size_t)amp * (size_t)hp->lut_entries, cudaMemcpyHostToDevice, st);
  double *partial = reinterpret_cast<double *>(base + o_part);
  const GroupDesc *groups = reinterpret_cast<const GroupDesc *>(base + o_groups);
  const BlockDesc *blocks = reinterpret_cast<const BlockDesc *>(base + o_blocks);
  if (e == cudaSuccess)
    e = dtype == Q2_C64
            ? run<float>(static_cast<const float *>(psi_dev), n, *hp, groups, blocks, base + o_lut, partial, grid, out,
                         fault, st)
            : run<double>(static_cast<const double *>(psi_dev), n, *hp, groups, blocks, base + o_lut, partial, grid, out,
                          fault, st);
  double host_out[2] = {0.0, 0.0};
  unsigned waits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, out, sizeof(host_out), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&waits, fault, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  const cudaError_t es = cudaStreamSynchronize(st);   // always: the host buffers above must outlive the copies
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return set_error(Q2_ERR_CUDA, cudaGetErrorString(e));
  if (waits) return set_error(Q2_ERR_TIMEOUT, "a device wait for a tile copy timed out");
  *energy_out = host_out[0] / host_out[1];
  if (norm_out) *norm_out = host_out[1];
  return Q2_OK;
}
