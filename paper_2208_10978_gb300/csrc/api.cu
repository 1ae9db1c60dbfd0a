// C ABI (include/q2.h): argument checks, handles, schedules and launch order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/q2.h"
#include "kernels.h"
#include "q2_internal.h"
#include "small.h"

using namespace q2;

namespace {

thread_local std::string g_err;

// Per-thread phase timing of q2_vqe_energy_grad (enabled by q2_debug_enable_timing).
struct PhaseTiming {
  bool enabled = false;
  bool valid = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int device = -1;
  double counts[4] = {0, 0, 0, 0};   // sweep, expect/happly, reverse launches, state bytes
  double total_launches = 0;
  bool has_reverse = false;
  ~PhaseTiming() {}
  cudaError_t ensure() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (ev[0] && device == dev) return cudaSuccess;
    for (int i = 0; i < 4; ++i) {
      if ((e = cudaEventCreate(&ev[i])) != cudaSuccess) return e;
    }
    device = dev;
    return cudaSuccess;
  }
};
thread_local PhaseTiming g_timing;

q2_status fail(q2_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

q2_status cuda_fail(cudaError_t e, const char *where) {
  return fail(e == cudaErrorMemoryAllocation ? Q2_ERR_OOM : Q2_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define Q2_CUDA(call, where)                     \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

int g_tile[2] = {12, 11};       // tile qubits per dtype
bool g_canon4_enabled = true;   // canonical 4-dimensional sweep blocks take the fast path
bool g_lean_expect_enabled = true;   // REAL/DIAG expectation passes take the lean path
const int g_chunk[2] = {4, 3};  // minimum contiguous low qubits per dtype (128-byte chunks)
std::mutex g_cfg_mu;

int amp_bytes(q2_dtype d) { return d == Q2_C64 ? 8 : 16; }
int max_qubits(q2_dtype d) { return d == Q2_C64 ? 34 : 33; }

bool valid_dtype(int d) { return d == Q2_C64 || d == Q2_C128; }

q2_status check_n(int n, q2_dtype d) {
  if (!valid_dtype(d)) return fail(Q2_ERR_INVALID, "unknown dtype");
  if (n < 1 || n > max_qubits(d))
    return fail(Q2_ERR_INVALID, "qubit count " + std::to_string(n) + " out of range");
  return Q2_OK;
}

q2_status check_masks(int n, int64_t cnt, const uint64_t *x, const uint64_t *z, const char *what) {
  if (cnt < 0) return fail(Q2_ERR_INVALID, std::string(what) + ": negative count");
  if (cnt > 0 && (!x || !z)) return fail(Q2_ERR_INVALID, std::string(what) + ": NULL mask array");
  const uint64_t bad = n >= 64 ? 0 : ~((1ull << n) - 1);
  for (int64_t k = 0; k < cnt; ++k)
    if ((x[k] | z[k]) & bad)
      return fail(Q2_ERR_INVALID, std::string(what) + ": mask bit >= n at entry " + std::to_string(k));
  return Q2_OK;
}

q2_status check_finite(int64_t cnt, const double *v, const char *what) {
  if (cnt > 0 && !v) return fail(Q2_ERR_INVALID, std::string(what) + ": NULL array");
  for (int64_t k = 0; k < cnt; ++k)
    if (!std::isfinite(v[k]))
      return fail(Q2_ERR_INVALID, std::string(what) + ": non-finite value at " + std::to_string(k));
  return Q2_OK;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

int tile_bits(q2_dtype d) {
  std::lock_guard<std::mutex> g(g_cfg_mu);
  return g_tile[d];
}

// Hamiltonian passes use one more tile qubit than rotation passes (more groups
// per pass; measured faster), within the shared-memory limit of H apply's two tiles.
int ham_tile_bits(q2_dtype d) { return std::min(tile_bits(d) + 1, d == Q2_C64 ? T_LIMIT : T_LIMIT - 1); }

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Device copies of a plan's groups (and optionally a LUT), owned by a handle.
struct DevTables {
  bool ready = false;
  int device = -1;
  int T = 0;
  GroupDesc *groups = nullptr;
  BlockDesc *blocks = nullptr;
  void *lut = nullptr;          // Hamiltonian LUT in the dtype's precision
  uint64_t *signmask = nullptr; // rotation sign masks
  void *wlut = nullptr;         // gradient weights of one-parameter rotation groups (dtype precision)
  void release() {
    if (groups) cudaFree(groups);
    if (blocks) cudaFree(blocks);
    if (lut) cudaFree(lut);
    if (signmask) cudaFree(signmask);
    if (wlut) cudaFree(wlut);
    groups = nullptr;
    blocks = nullptr;
    lut = nullptr;
    signmask = nullptr;
    wlut = nullptr;
    ready = false;
  }
};

// Convert an interleaved double LUT to the dtype's precision.
std::vector<unsigned char> lut_bytes(const std::vector<double> &lut2, q2_dtype d) {
  std::vector<unsigned char> out(lut2.size() * (d == Q2_C64 ? sizeof(float) : sizeof(double)));
  if (d == Q2_C64) {
    float *f = reinterpret_cast<float *>(out.data());
    for (size_t i = 0; i < lut2.size(); ++i) f[i] = (float)lut2[i];
  } else {
    std::memcpy(out.data(), lut2.data(), lut2.size() * sizeof(double));
  }
  return out;
}

}  // namespace

struct q2_ham {
  int n = 0;
  std::vector<uint64_t> x, z;
  std::vector<double> c;
  int64_t n_groups = 0;
  int shard = 0, n_shards = 1;   // a shard evaluates only its share of the passes of the full plan
  HamPlan plan[2];
  bool planned[2] = {false, false};
  DevTables dev[2];
  // single-tile plan (identity local basis) for the batched small-state path
  HamPlan splan;
  bool splanned = false;
  DevTables sdev[2];
  std::mutex mu;
};

namespace q2 {
q2_status ham_host_plan(const q2_ham *hc, q2_dtype d, const HamPlan **plan, int *chunk);
}

struct q2_ansatz {
  int n = 0, n_elec = 0;
  int32_t n_params = 0;
  std::vector<uint64_t> x, z;
  std::vector<int32_t> param;
  std::vector<double> coef;
  RotPlan plan[2];
  bool planned[2] = {false, false};
  DevTables dev[2];
  RotPlan splan;
  bool splanned = false;
  DevTables sdev;
  int32_t *sgrot = nullptr;     // device: first rotation of each group of splan
  std::mutex mu;
};

namespace {

// Host schedule of a Hamiltonian for a dtype (the caller holds h->mu); a shard keeps
// only its passes of the full schedule.
q2_status plan_ham_locked(q2_ham *h, q2_dtype d) {
  if (h->planned[d]) return Q2_OK;
  try {
    h->plan[d] = build_ham_plan(h->n, (int64_t)h->c.size(), h->x.data(), h->z.data(), h->c.data(),
                                ham_tile_bits(d), g_chunk[d], d == Q2_C64 ? LUT_STAGE_HAM_C64 : LUT_STAGE);
    restrict_to_shard(h->plan[d], h->shard, h->n_shards);
  } catch (const std::exception &e) {
    return fail(Q2_ERR_INVALID, std::string("Hamiltonian schedule: ") + e.what());
  }
  h->planned[d] = true;
  return Q2_OK;
}

q2_status ham_tables(const q2_ham *hc, q2_dtype d, const HamPlan **plan, const DevTables **dev) {
  q2_ham *h = const_cast<q2_ham *>(hc);
  std::lock_guard<std::mutex> g(h->mu);
  q2_status ps = plan_ham_locked(h, d);
  if (ps != Q2_OK) return ps;
  DevTables &t = h->dev[d];
  int device = 0;
  Q2_CUDA(cudaGetDevice(&device), "cudaGetDevice");
  if (t.ready && t.device != device) return fail(Q2_ERR_INVALID, "Hamiltonian handle used on another device");
  if (!t.ready) {
    const HamPlan &p = h->plan[d];
    const size_t gb = sizeof(GroupDesc) * std::max<size_t>(1, p.groups.size());
    std::vector<unsigned char> lb = lut_bytes(p.lut2, d);
    if (d == Q2_C64 && !p.lut2.empty()) {   // (R, R) for REAL and DIAG groups: the lean path reads both halves
      const std::vector<float> f = p.lut_f32();
      std::memcpy(lb.data(), f.data(), sizeof(float) * f.size());
    }
    const size_t bb = sizeof(BlockDesc) * std::max<size_t>(1, p.blocks.size());
    Q2_CUDA(cudaMalloc(&t.groups, gb), "cudaMalloc(groups)");
    if (cudaMalloc(&t.lut, std::max<size_t>(16, lb.size())) != cudaSuccess ||
        cudaMalloc(&t.blocks, bb) != cudaSuccess) {
      t.release();
      return fail(Q2_ERR_OOM, "cudaMalloc(Hamiltonian tables)");
    }
    if (!p.groups.empty())
      Q2_CUDA(cudaMemcpy(t.groups, p.groups.data(), sizeof(GroupDesc) * p.groups.size(),
                         cudaMemcpyHostToDevice), "upload groups");
    if (!p.blocks.empty())
      Q2_CUDA(cudaMemcpy(t.blocks, p.blocks.data(), sizeof(BlockDesc) * p.blocks.size(),
                         cudaMemcpyHostToDevice), "upload blocks");
    if (!lb.empty()) Q2_CUDA(cudaMemcpy(t.lut, lb.data(), lb.size(), cudaMemcpyHostToDevice), "upload LUT");
    t.device = device;
    t.T = p.T;
    t.ready = true;
  }
  *plan = &h->plan[d];
  *dev = &t;
  return Q2_OK;
}

q2_status ansatz_tables(const q2_ansatz *ac, q2_dtype d, const RotPlan **plan, const DevTables **dev) {
  q2_ansatz *a = const_cast<q2_ansatz *>(ac);
  std::lock_guard<std::mutex> g(a->mu);
  if (!a->planned[d]) {
    try {
      a->plan[d] = build_rot_plan(a->n, (int64_t)a->x.size(), a->x.data(), a->z.data(), tile_bits(d),
                                  g_chunk[d]);
      set_param_weights(a->plan[d], a->param.data(), a->coef.data());
    } catch (const std::exception &e) {
      return fail(Q2_ERR_INVALID, std::string("rotation schedule: ") + e.what());
    }
    a->planned[d] = true;
  }
  if (!dev) {
    *plan = &a->plan[d];
    return Q2_OK;
  }
  DevTables &t = a->dev[d];
  int device = 0;
  Q2_CUDA(cudaGetDevice(&device), "cudaGetDevice");
  if (t.ready && t.device != device) return fail(Q2_ERR_INVALID, "ansatz handle used on another device");
  if (!t.ready) {
    const RotPlan &p = a->plan[d];
    const size_t gb = sizeof(GroupDesc) * std::max<size_t>(1, p.groups.size());
    const size_t sb = sizeof(uint64_t) * std::max<size_t>(1, p.signmask.size());
    const size_t bb = sizeof(BlockDesc) * std::max<size_t>(1, p.blocks.size());
    Q2_CUDA(cudaMalloc(&t.groups, gb), "cudaMalloc(groups)");
    if (cudaMalloc(&t.signmask, sb) != cudaSuccess || cudaMalloc(&t.blocks, bb) != cudaSuccess) {
      t.release();
      return fail(Q2_ERR_OOM, "cudaMalloc(rotation tables)");
    }
    if (!p.groups.empty())
      Q2_CUDA(cudaMemcpy(t.groups, p.groups.data(), sizeof(GroupDesc) * p.groups.size(),
                         cudaMemcpyHostToDevice), "upload groups");
    if (!p.blocks.empty())
      Q2_CUDA(cudaMemcpy(t.blocks, p.blocks.data(), sizeof(BlockDesc) * p.blocks.size(),
                         cudaMemcpyHostToDevice), "upload blocks");
    if (!p.signmask.empty())
      Q2_CUDA(cudaMemcpy(t.signmask, p.signmask.data(), sizeof(uint64_t) * p.signmask.size(),
                         cudaMemcpyHostToDevice), "upload sign masks");
    const std::vector<unsigned char> wb = lut_bytes(p.wlut.empty() ? std::vector<double>(1, 0.0) : p.wlut, d);
    if (cudaMalloc(&t.wlut, wb.size()) != cudaSuccess) {
      t.release();
      return fail(Q2_ERR_OOM, "cudaMalloc(gradient weights)");
    }
    Q2_CUDA(cudaMemcpy(t.wlut, wb.data(), wb.size(), cudaMemcpyHostToDevice), "upload gradient weights");
    t.device = device;
    t.T = p.T;
    t.ready = true;
  }
  *plan = &a->plan[d];
  *dev = &t;
  return Q2_OK;
}

template <typename R>
cudaError_t run_sweep(R *psi, int n, const RotPlan &p, const GroupDesc *dgroups, const BlockDesc *dblocks,
                      const void *dlut, unsigned *fault, cudaStream_t st) {
  for (size_t i = 0; i < p.passes.size(); ++i) {
    const PassDesc &pd = p.passes[i];
    const bool c4 = i < p.pass_canon4.size() && p.pass_canon4[i] && g_canon4_enabled;
    cudaError_t e = launch_sweep<R>(psi, n, pd, dgroups, dblocks, dlut, fault, c4, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t run_expect(const R *psi, int n, const HamPlan &h, const DevTables &t, double *partial,
                       int grid, double *out2, unsigned *fault, cudaStream_t st) {
  if (h.passes.empty()) {   // no terms (or a shard without passes): energy 0, norm by a dot product
    const int dg = dot_grid<R>(n);
    cudaError_t e = launch_dot<R>(psi, psi, n, partial, dg, st);
    if (e == cudaSuccess) e = launch_reduce_pairs(partial, dg, out2, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(out2, 0, sizeof(double), st);
    return e;
  }
  for (size_t i = 0; i < h.passes.size(); ++i) {
    const bool lean = g_lean_expect_enabled && i < h.pass_lean.size() && h.pass_lean[i];
    cudaError_t e =
        launch_expect<R>(psi, n, h.passes[i], t.groups, t.blocks, t.lut, partial, grid, i == 0, fault, lean, st);
    if (e != cudaSuccess) return e;
  }
  return launch_reduce_pairs(partial, grid, out2, st);
}

template <typename R>
cudaError_t run_happly(const R *psi, R *lam, int n, const HamPlan &h, const DevTables &t, unsigned *fault,
                       cudaStream_t st) {
  if (h.passes.empty()) return cudaMemsetAsync(lam, 0, (2 * sizeof(R)) << n, st);   // H = 0 here
  for (size_t i = 0; i < h.passes.size(); ++i) {
    cudaError_t e = launch_happly<R>(psi, lam, n, h.passes[i], t.groups, t.blocks, t.lut, i == 0, fault, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int partial_doubles(int grad) {
  const int blocks = max_grid_blocks(8, 12);
  return grad ? blocks * RP_MAX : blocks * 2;
}

// Workspace of q2_vqe_energy_grad / q2_pool_gradients: psi, lambda, the
// per-call angle LUT, dE/dphi, CTA partials and a 32-byte result block
// (out[0] <psi|H|psi>, out[1] <psi|psi>, then the call's fault word).
struct WsLayout {
  size_t psi, lam, lut, gphi, partial, out, total;
};

// The fault word of a 4-double result block (after the two sums).
unsigned *fault_word(double *out4) { return reinterpret_cast<unsigned *>(out4 + 2); }
unsigned fault_of(const double *host4) {
  unsigned f;
  std::memcpy(&f, host4 + 2, sizeof f);
  return f;
}

WsLayout ws_layout(int n, q2_dtype d, int grad, int64_t lut_entries, int64_t n_rot) {
  WsLayout L;
  const size_t vec = (size_t)amp_bytes(d) << n;
  size_t o = 0;
  L.psi = o;
  o = align_up(o + vec, 256);
  L.lam = o;
  if (grad) o = align_up(o + vec, 256);
  L.lut = o;
  o = align_up(o + (size_t)std::max<int64_t>(1, lut_entries) * amp_bytes(d), 256);
  L.gphi = o;
  if (grad) o = align_up(o + sizeof(double) * (size_t)std::max<int64_t>(1, n_rot), 256);
  L.partial = o;
  o = align_up(o + sizeof(double) * (size_t)partial_doubles(grad), 256);
  L.out = o;
  o = align_up(o + sizeof(double) * 4, 256);
  L.total = o;
  return L;
}

template <typename R>
q2_status vqe_impl(const q2_ansatz *a, const q2_ham *h, const double *theta, q2_dtype d, int want_grad,
                   double *energy_out, double *grad_out, void *ws, size_t ws_bytes, cudaStream_t st) {
  const RotPlan *rp;
  const DevTables *rt;
  q2_status s = ansatz_tables(a, d, &rp, &rt);
  if (s != Q2_OK) return s;
  const HamPlan *hp;
  const DevTables *ht;
  if ((s = ham_tables(h, d, &hp, &ht)) != Q2_OK) return s;
  const int n = a->n;
  const WsLayout L = ws_layout(n, d, want_grad, rp->lut_entries, (int64_t)a->x.size());
  if (ws_bytes < L.total) return fail(Q2_ERR_INVALID, "workspace too small");
  unsigned char *base = static_cast<unsigned char *>(ws);
  R *psi = reinterpret_cast<R *>(base + L.psi);
  R *lam = reinterpret_cast<R *>(base + L.lam);
  double *gphi = reinterpret_cast<double *>(base + L.gphi);
  double *partial = reinterpret_cast<double *>(base + L.partial);
  double *out = reinterpret_cast<double *>(base + L.out);

  // angles and the per-call LUT (host, double precision)
  const size_t nrot = a->x.size();
  std::vector<double> phi(nrot);
  for (size_t k = 0; k < nrot; ++k) phi[k] = a->coef[k] * theta[a->param[k]];
  std::vector<double> lut2(2 * (size_t)std::max<int64_t>(1, rp->lut_entries));
  rp->build_lut(phi.data(), lut2.data());
  std::vector<unsigned char> lb = lut_bytes(lut2, d);
  Q2_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 4, st), "clear results");
  Q2_CUDA(cudaMemcpyAsync(base + L.lut, lb.data(), lb.size(), cudaMemcpyHostToDevice, st), "upload LUT");
  unsigned *fault = fault_word(out);

  const bool timing = g_timing.enabled;
  g_timing.valid = false;
  if (timing) Q2_CUDA(g_timing.ensure(), "timing events");
  Q2_CUDA(launch_init_hf<R>(psi, n, a->n_elec, st), "init_hf");
  if (timing) Q2_CUDA(cudaEventRecord(g_timing.ev[0], st), "event");
  Q2_CUDA(run_sweep<R>(psi, n, *rp, rt->groups, rt->blocks, base + L.lut, fault, st), "sweep");
  if (timing) Q2_CUDA(cudaEventRecord(g_timing.ev[1], st), "event");
  double host_out[4] = {0, 0, 0, 0};
  g_timing.counts[0] = (double)rp->passes.size();
  g_timing.counts[3] = (double)((size_t)amp_bytes(d) << n);
  if (!want_grad) {
    const int grid = expect_grid<R>(n, hp->T, std::min(g_chunk[d], hp->T));
    Q2_CUDA(run_expect<R>(psi, n, *hp, *ht, partial, grid, out, fault, st), "expectation");
    if (timing) Q2_CUDA(cudaEventRecord(g_timing.ev[2], st), "event");
    Q2_CUDA(cudaMemcpyAsync(host_out, out, sizeof(host_out), cudaMemcpyDeviceToHost, st), "D2H");
    Q2_CUDA(cudaStreamSynchronize(st), "sync");
    if (fault_of(host_out)) return fail(Q2_ERR_TIMEOUT, "a device wait for a tile copy timed out");
    *energy_out = host_out[0] / host_out[1];
    if (timing) {
      g_timing.counts[1] = (double)hp->passes.size() + 1;
      g_timing.counts[2] = 0;
      g_timing.total_launches = 1 + g_timing.counts[0] + g_timing.counts[1];
      g_timing.has_reverse = false;
      g_timing.valid = true;
    }
    return Q2_OK;
  }
  Q2_CUDA(run_happly<R>(psi, lam, n, *hp, *ht, fault, st), "H apply");
  const int dgrid = dot_grid<R>(n);
  Q2_CUDA(launch_dot<R>(psi, lam, n, partial, dgrid, st), "dot");
  Q2_CUDA(launch_reduce_pairs(partial, dgrid, out, st), "reduce");
  if (timing) Q2_CUDA(cudaEventRecord(g_timing.ev[2], st), "event");
  for (size_t i = rp->passes.size(); i-- > 0;) {
    Q2_CUDA(launch_reverse<R>(psi, lam, n, rp->passes[i], rt->groups, rt->blocks, rp->pass_one_param[i] != 0,
                              base + L.lut, rt->signmask, static_cast<const R *>(rt->wlut), partial, gphi, fault,
                              st),
            "reverse sweep");
  }
  if (timing) Q2_CUDA(cudaEventRecord(g_timing.ev[3], st), "event");
  if (timing) {
    g_timing.counts[1] = (double)hp->passes.size() + 2;
    g_timing.counts[2] = 2.0 * (double)rp->passes.size();
    g_timing.total_launches = 1 + g_timing.counts[0] + g_timing.counts[1] + g_timing.counts[2];
    g_timing.has_reverse = true;
    g_timing.valid = true;
  }
  std::vector<double> g(nrot);
  Q2_CUDA(cudaMemcpyAsync(host_out, out, sizeof(host_out), cudaMemcpyDeviceToHost, st), "D2H");
  if (nrot) Q2_CUDA(cudaMemcpyAsync(g.data(), gphi, sizeof(double) * nrot, cudaMemcpyDeviceToHost, st), "D2H");
  Q2_CUDA(cudaStreamSynchronize(st), "sync");
  if (fault_of(host_out)) return fail(Q2_ERR_TIMEOUT, "a device wait for a tile copy timed out");
  *energy_out = host_out[0] / host_out[1];
  for (int p = 0; p < a->n_params; ++p) grad_out[p] = 0.0;
  for (size_t k = 0; k < nrot; ++k) grad_out[a->param[k]] += rp->fold[k] * g[k];
  return Q2_OK;
}

// ---- batched small-state path: single-tile plans (identity local basis)

struct BatchSlot {
  size_t lut_off, out_off, stage_end;
};

const RotPlan &small_rot_plan(const q2_ansatz *ac) {
  q2_ansatz *a = const_cast<q2_ansatz *>(ac);
  std::lock_guard<std::mutex> g(a->mu);
  if (!a->splanned) {
    a->splan = build_rot_plan(a->n, (int64_t)a->x.size(), a->x.data(), a->z.data(), a->n, a->n);
    a->splanned = true;
  }
  return a->splan;
}

q2_status small_ansatz_tables(const q2_ansatz *ac, const DevTables **dev, const int32_t **grot) {
  const RotPlan &p = small_rot_plan(ac);
  q2_ansatz *a = const_cast<q2_ansatz *>(ac);
  std::lock_guard<std::mutex> g(a->mu);
  DevTables &t = a->sdev;
  int device = 0;
  Q2_CUDA(cudaGetDevice(&device), "cudaGetDevice");
  if (t.ready && t.device != device) return fail(Q2_ERR_INVALID, "ansatz handle used on another device");
  if (!t.ready) {
    const size_t gb = sizeof(GroupDesc) * std::max<size_t>(1, p.groups.size());
    const size_t sb = sizeof(uint64_t) * std::max<size_t>(1, p.signmask.size());
    const size_t rb = sizeof(int32_t) * std::max<size_t>(1, p.grp_rot_begin.size());
    if (cudaMalloc(&t.groups, gb) != cudaSuccess || cudaMalloc(&t.signmask, sb) != cudaSuccess ||
        cudaMalloc(&a->sgrot, rb) != cudaSuccess) {
      t.release();
      return fail(Q2_ERR_OOM, "cudaMalloc(small rotation tables)");
    }
    std::vector<int32_t> gr(p.grp_rot_begin.begin(), p.grp_rot_begin.end());
    if (!p.groups.empty())
      Q2_CUDA(cudaMemcpy(t.groups, p.groups.data(), sizeof(GroupDesc) * p.groups.size(), cudaMemcpyHostToDevice),
              "upload groups");
    if (!p.signmask.empty())
      Q2_CUDA(cudaMemcpy(t.signmask, p.signmask.data(), sizeof(uint64_t) * p.signmask.size(),
                         cudaMemcpyHostToDevice), "upload sign masks");
    if (!gr.empty())
      Q2_CUDA(cudaMemcpy(a->sgrot, gr.data(), sizeof(int32_t) * gr.size(), cudaMemcpyHostToDevice),
              "upload group rotations");
    t.device = device;
    t.T = p.T;
    t.ready = true;
  }
  *dev = &t;
  *grot = a->sgrot;
  return Q2_OK;
}

q2_status small_ham_tables(const q2_ham *hc, q2_dtype d, const HamPlan **plan, const DevTables **dev) {
  q2_ham *h = const_cast<q2_ham *>(hc);
  std::lock_guard<std::mutex> g(h->mu);
  if (!h->splanned) {
    try {
      h->splan = build_ham_plan(h->n, (int64_t)h->c.size(), h->x.data(), h->z.data(), h->c.data(), h->n, h->n);
    } catch (const std::exception &e) {
      return fail(Q2_ERR_INVALID, std::string("Hamiltonian schedule: ") + e.what());
    }
    h->splanned = true;
  }
  DevTables &t = h->sdev[d];
  int device = 0;
  Q2_CUDA(cudaGetDevice(&device), "cudaGetDevice");
  if (t.ready && t.device != device) return fail(Q2_ERR_INVALID, "Hamiltonian handle used on another device");
  if (!t.ready) {
    const HamPlan &p = h->splan;
    const size_t gb = sizeof(GroupDesc) * std::max<size_t>(1, p.groups.size());
    std::vector<unsigned char> lb = lut_bytes(p.lut2, d);
    if (cudaMalloc(&t.groups, gb) != cudaSuccess || cudaMalloc(&t.lut, std::max<size_t>(16, lb.size())) != cudaSuccess) {
      t.release();
      return fail(Q2_ERR_OOM, "cudaMalloc(small Hamiltonian tables)");
    }
    if (!p.groups.empty())
      Q2_CUDA(cudaMemcpy(t.groups, p.groups.data(), sizeof(GroupDesc) * p.groups.size(), cudaMemcpyHostToDevice),
              "upload groups");
    if (!lb.empty()) Q2_CUDA(cudaMemcpy(t.lut, lb.data(), lb.size(), cudaMemcpyHostToDevice), "upload LUT");
    t.device = device;
    t.T = p.T;
    t.ready = true;
  }
  *plan = &h->splan;
  *dev = &t;
  return Q2_OK;
}

// Workspace of a batch: [items][per-request rotation LUTs][per-request outputs]; the
// staging image uploaded per call covers items and LUTs.
q2_status batch_layout(int nreq, const q2_ansatz *const *ansatz, q2_dtype d, std::vector<BatchSlot> *slots,
                       size_t *total) {
  const size_t lut_b = d == Q2_C64 ? 2 * sizeof(float) : 2 * sizeof(double);
  size_t o = align_up(sizeof(BatchItem) * (size_t)std::max(1, nreq), 256);
  std::vector<BatchSlot> sl(nreq);
  for (int b = 0; b < nreq; ++b) {
    if (!ansatz[b]) return fail(Q2_ERR_INVALID, "NULL ansatz");
    if (ansatz[b]->n > SMALL_MAX_QUBITS) return fail(Q2_ERR_INVALID, "batched requests need n <= 12");
    const RotPlan &p = small_rot_plan(ansatz[b]);
    sl[b].lut_off = o;
    o = align_up(o + lut_b * (size_t)std::max<int64_t>(1, p.lut_entries), 256);
  }
  const size_t stage_end = o;
  for (int b = 0; b < nreq; ++b) {
    sl[b].out_off = o;
    sl[b].stage_end = stage_end;
    o = align_up(o + sizeof(double) * (2 + ansatz[b]->x.size()), 256);
  }
  if (slots) *slots = sl;
  *total = o;
  return Q2_OK;
}

}  // namespace

extern "C" {

int q2_version(void) { return 100; }

const char *q2_last_error(void) { return g_err.c_str(); }

q2_status q2_set_tile_qubits(q2_dtype dtype, int tile_qubits) {
  if (!valid_dtype(dtype)) return fail(Q2_ERR_INVALID, "unknown dtype");
  // the reverse sweep holds two tiles: 2 * 2^T * 16 bytes must stay within shared memory
  const int tmax = dtype == Q2_C64 ? T_LIMIT : T_LIMIT - 1;
  if (tile_qubits < T_MIN || tile_qubits > tmax) return fail(Q2_ERR_INVALID, "tile qubits out of range");
  std::lock_guard<std::mutex> g(g_cfg_mu);
  g_tile[dtype] = tile_qubits;
  return Q2_OK;
}

q2_status q2_state_init_hf(void *psi_dev, int n, int n_elec, q2_dtype dtype, void *stream) {
  q2_status s = check_n(n, dtype);
  if (s != Q2_OK) return s;
  if (n_elec < 0 || n_elec > n) return fail(Q2_ERR_INVALID, "n_elec out of range");
  if (!psi_dev || !aligned(psi_dev, 16)) return fail(Q2_ERR_INVALID, "psi must be a 16-byte aligned device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = dtype == Q2_C64 ? launch_init_hf<float>(static_cast<float *>(psi_dev), n, n_elec, st)
                                  : launch_init_hf<double>(static_cast<double *>(psi_dev), n, n_elec, st);
  if (e != cudaSuccess) return cuda_fail(e, "init_hf");
  return Q2_OK;
}

q2_status q2_apply_pauli_rotations(void *psi_dev, int n, q2_dtype dtype, const uint64_t *xmask,
                                   const uint64_t *zmask, const double *angles, int64_t n_rot,
                                   void *stream) {
  q2_status s = check_n(n, dtype);
  if (s != Q2_OK) return s;
  if (!psi_dev || !aligned(psi_dev, 16)) return fail(Q2_ERR_INVALID, "psi must be a 16-byte aligned device pointer");
  if ((s = check_masks(n, n_rot, xmask, zmask, "rotations")) != Q2_OK) return s;
  if ((s = check_finite(n_rot, angles, "angles")) != Q2_OK) return s;
  if (n_rot == 0) return Q2_OK;
  RotPlan p;
  try {
    p = build_rot_plan(n, n_rot, xmask, zmask, tile_bits(dtype), g_chunk[dtype]);
  } catch (const std::exception &e) {
    return fail(Q2_ERR_INVALID, std::string("rotation schedule: ") + e.what());
  }
  std::vector<double> lut2(2 * (size_t)std::max<int64_t>(1, p.lut_entries));
  p.build_lut(angles, lut2.data());
  std::vector<unsigned char> lb = lut_bytes(lut2, dtype);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t gb = align_up(sizeof(GroupDesc) * p.groups.size(), 256);
  const size_t bb = align_up(sizeof(BlockDesc) * p.blocks.size(), 256);
  unsigned char *tmp = nullptr;
  Q2_CUDA(cudaMallocAsync((void **)&tmp, gb + bb + lb.size(), st), "cudaMallocAsync(schedule)");
  cudaError_t e = cudaMemcpyAsync(tmp, p.groups.data(), sizeof(GroupDesc) * p.groups.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tmp + gb, p.blocks.data(), sizeof(BlockDesc) * p.blocks.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tmp + gb + bb, lb.data(), lb.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const GroupDesc *dg = reinterpret_cast<const GroupDesc *>(tmp);
    const BlockDesc *db = reinterpret_cast<const BlockDesc *>(tmp + gb);
    e = dtype == Q2_C64
            ? run_sweep<float>(static_cast<float *>(psi_dev), n, p, dg, db, tmp + gb + bb, nullptr, st)
            : run_sweep<double>(static_cast<double *>(psi_dev), n, p, dg, db, tmp + gb + bb, nullptr, st);
  }
  cudaFreeAsync(tmp, st);
  if (e != cudaSuccess) return cuda_fail(e, "apply_pauli_rotations");
  return Q2_OK;
}

q2_status q2_ham_create(int n, const uint64_t *x, const uint64_t *z, const double *coef, int64_t n_terms,
                        q2_ham **out) {
  if (!out) return fail(Q2_ERR_INVALID, "NULL output handle");
  *out = nullptr;
  if (n < 1 || n > 34) return fail(Q2_ERR_INVALID, "qubit count out of range");
  q2_status s = check_masks(n, n_terms, x, z, "Hamiltonian");
  if (s != Q2_OK) return s;
  if ((s = check_finite(n_terms, coef, "coefficients")) != Q2_OK) return s;
  q2_ham *h = new (std::nothrow) q2_ham;
  if (!h) return fail(Q2_ERR_OOM, "host allocation");
  h->n = n;
  h->x.assign(x, x + n_terms);
  h->z.assign(z, z + n_terms);
  h->c.assign(coef, coef + n_terms);
  h->n_groups = count_x_groups(n_terms, x);
  *out = h;
  return Q2_OK;
}

q2_status q2_ham_destroy(q2_ham *ham) {
  if (!ham) return Q2_OK;
  ham->dev[0].release();
  ham->dev[1].release();
  ham->sdev[0].release();
  ham->sdev[1].release();
  delete ham;
  return Q2_OK;
}

q2_status q2_async_status(void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned host = 0;
  Q2_CUDA(take_async_faults(&host, st), "read asynchronous fault count");
  Q2_CUDA(cudaStreamSynchronize(st), "sync");
  if (host) return fail(Q2_ERR_TIMEOUT, "a device wait for a tile copy of an asynchronous call timed out");
  return Q2_OK;
}

q2_status q2_ham_shard(const q2_ham *ham, int shard, int n_shards, q2_ham **out) {
  if (!ham || !out) return fail(Q2_ERR_INVALID, "NULL argument");
  *out = nullptr;
  if (ham->n_shards != 1) return fail(Q2_ERR_INVALID, "a shard cannot be sharded again");
  if (n_shards < 1 || shard < 0 || shard >= n_shards) return fail(Q2_ERR_INVALID, "shard index out of range");
  q2_ham *h = new (std::nothrow) q2_ham;
  if (!h) return fail(Q2_ERR_OOM, "host allocation");
  h->n = ham->n;
  h->x = ham->x;
  h->z = ham->z;
  h->c = ham->c;
  h->n_groups = ham->n_groups;
  h->shard = shard;
  h->n_shards = n_shards;
  *out = h;
  return Q2_OK;
}

q2_status q2_ham_shard_terms(const q2_ham *ham, q2_dtype dtype, int64_t *idx_out, int64_t *count) {
  if (!ham || !count) return fail(Q2_ERR_INVALID, "NULL argument");
  if (!valid_dtype(dtype)) return fail(Q2_ERR_INVALID, "unknown dtype");
  const HamPlan *hp;
  int chunk = 0;
  q2_status s = ham_host_plan(ham, dtype, &hp, &chunk);
  if (s != Q2_OK) return s;
  std::vector<int64_t> idx;
  for (const PassDesc &pd : hp->passes)
    for (int g = pd.g_begin; g < pd.g_end; ++g)
      idx.insert(idx.end(), hp->term_idx.begin() + hp->term_begin[g], hp->term_idx.begin() + hp->term_begin[g + 1]);
  std::sort(idx.begin(), idx.end());
  if (idx_out) {
    if (*count < (int64_t)idx.size()) return fail(Q2_ERR_INVALID, "term index buffer too small");
    std::copy(idx.begin(), idx.end(), idx_out);
  }
  *count = (int64_t)idx.size();
  return Q2_OK;
}

q2_status q2_ham_info(const q2_ham *ham, int64_t *n_terms, int64_t *n_groups) {
  if (!ham) return fail(Q2_ERR_INVALID, "NULL handle");
  if (n_terms) *n_terms = (int64_t)ham->c.size();
  if (n_groups) *n_groups = ham->n_groups;
  return Q2_OK;
}

q2_status q2_expectation(const void *psi_dev, int n, q2_dtype dtype, const q2_ham *ham, double *energy_out,
                         double *norm_out, void *stream) {
  q2_status s = check_n(n, dtype);
  if (s != Q2_OK) return s;
  if (!ham || !energy_out) return fail(Q2_ERR_INVALID, "NULL argument");
  if (ham->n != n) return fail(Q2_ERR_INVALID, "Hamiltonian qubit count differs from n");
  if (!psi_dev || !aligned(psi_dev, 16)) return fail(Q2_ERR_INVALID, "psi must be a 16-byte aligned device pointer");
  const HamPlan *hp;
  const DevTables *ht;
  if ((s = ham_tables(ham, dtype, &hp, &ht)) != Q2_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int C = std::min(g_chunk[dtype], hp->T);
  const int grid = dtype == Q2_C64 ? expect_grid<float>(n, hp->T, C) : expect_grid<double>(n, hp->T, C);
  const int slots = std::max(grid, dtype == Q2_C64 ? dot_grid<float>(n) : dot_grid<double>(n));
  // [partials 2 * slots][result block of 4 doubles: sums, fault word]
  double *tmp = nullptr;
  Q2_CUDA(cudaMallocAsync((void **)&tmp, sizeof(double) * (2 * (size_t)slots + 4), st), "cudaMallocAsync(partials)");
  double *out4 = tmp + 2 * slots;
  double host_out[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemsetAsync(out4, 0, sizeof(double) * 4, st);
  if (e == cudaSuccess)
    e = dtype == Q2_C64 ? run_expect<float>(static_cast<const float *>(psi_dev), n, *hp, *ht, tmp, grid, out4,
                                            fault_word(out4), st)
                        : run_expect<double>(static_cast<const double *>(psi_dev), n, *hp, *ht, tmp, grid, out4,
                                             fault_word(out4), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, out4, sizeof(host_out), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(tmp, st);
  const cudaError_t es = cudaStreamSynchronize(st);   // always: nothing may still use tmp or host_out
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(e, "expectation");
  if (fault_of(host_out)) return fail(Q2_ERR_TIMEOUT, "a device wait for a tile copy timed out");
  *energy_out = host_out[0] / host_out[1];
  if (norm_out) *norm_out = host_out[1];
  return Q2_OK;
}

q2_status q2_apply_hamiltonian(const void *psi_dev, void *lam_dev, int n, q2_dtype dtype, const q2_ham *ham,
                               void *stream) {
  q2_status s = check_n(n, dtype);
  if (s != Q2_OK) return s;
  if (!ham) return fail(Q2_ERR_INVALID, "NULL Hamiltonian");
  if (ham->n != n) return fail(Q2_ERR_INVALID, "Hamiltonian qubit count differs from n");
  if (!psi_dev || !lam_dev || !aligned(psi_dev, 16) || !aligned(lam_dev, 16))
    return fail(Q2_ERR_INVALID, "psi and lambda must be 16-byte aligned device pointers");
  if (psi_dev == lam_dev) return fail(Q2_ERR_INVALID, "psi and lambda must be distinct buffers");
  const HamPlan *hp;
  const DevTables *ht;
  if ((s = ham_tables(ham, dtype, &hp, &ht)) != Q2_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = dtype == Q2_C64
                      ? run_happly<float>(static_cast<const float *>(psi_dev), static_cast<float *>(lam_dev), n, *hp,
                                          *ht, nullptr, st)
                      : run_happly<double>(static_cast<const double *>(psi_dev), static_cast<double *>(lam_dev), n,
                                           *hp, *ht, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "apply_hamiltonian");
  return Q2_OK;
}

q2_status q2_ansatz_create(int n, int n_elec, int64_t n_rot, const uint64_t *x, const uint64_t *z,
                           const int32_t *param_idx, const double *coef, int32_t n_params, q2_ansatz **out) {
  if (!out) return fail(Q2_ERR_INVALID, "NULL output handle");
  *out = nullptr;
  if (n < 1 || n > 34) return fail(Q2_ERR_INVALID, "qubit count out of range");
  if (n_elec < 0 || n_elec > n) return fail(Q2_ERR_INVALID, "n_elec out of range");
  if (n_params < 0) return fail(Q2_ERR_INVALID, "negative parameter count");
  q2_status s = check_masks(n, n_rot, x, z, "ansatz");
  if (s != Q2_OK) return s;
  if ((s = check_finite(n_rot, coef, "ansatz coefficients")) != Q2_OK) return s;
  if (n_rot > 0 && !param_idx) return fail(Q2_ERR_INVALID, "NULL parameter index array");
  for (int64_t k = 0; k < n_rot; ++k)
    if (param_idx[k] < 0 || param_idx[k] >= n_params)
      return fail(Q2_ERR_INVALID, "parameter index out of range at " + std::to_string(k));
  q2_ansatz *a = new (std::nothrow) q2_ansatz;
  if (!a) return fail(Q2_ERR_OOM, "host allocation");
  a->n = n;
  a->n_elec = n_elec;
  a->n_params = n_params;
  a->x.assign(x, x + n_rot);
  a->z.assign(z, z + n_rot);
  a->param.assign(param_idx, param_idx + n_rot);
  a->coef.assign(coef, coef + n_rot);
  *out = a;
  return Q2_OK;
}

q2_status q2_ansatz_destroy(q2_ansatz *ansatz) {
  if (!ansatz) return Q2_OK;
  ansatz->dev[0].release();
  ansatz->dev[1].release();
  ansatz->sdev.release();
  if (ansatz->sgrot) cudaFree(ansatz->sgrot);
  delete ansatz;
  return Q2_OK;
}

q2_status q2_ansatz_info(const q2_ansatz *ansatz, q2_dtype dtype, int64_t *n_passes, int64_t *n_groups) {
  if (!ansatz) return fail(Q2_ERR_INVALID, "NULL handle");
  if (!valid_dtype(dtype)) return fail(Q2_ERR_INVALID, "unknown dtype");
  const RotPlan *rp;
  q2_status s = ansatz_tables(ansatz, dtype, &rp, nullptr);
  if (s != Q2_OK) return s;
  if (n_passes) *n_passes = (int64_t)rp->passes.size();
  if (n_groups) *n_groups = (int64_t)rp->groups.size();
  return Q2_OK;
}

q2_status q2_ham_table_bytes(const q2_ham *ham, q2_dtype dtype, size_t *device_bytes) {
  if (!ham || !device_bytes) return fail(Q2_ERR_INVALID, "NULL argument");
  if (!valid_dtype(dtype)) return fail(Q2_ERR_INVALID, "unknown dtype");
  const HamPlan *hp;
  int chunk = 0;
  q2_status s = ham_host_plan(ham, dtype, &hp, &chunk);
  if (s != Q2_OK) return s;
  *device_bytes = sizeof(GroupDesc) * std::max<size_t>(1, hp->groups.size()) +
                  sizeof(BlockDesc) * std::max<size_t>(1, hp->blocks.size()) +
                  std::max<size_t>(16, hp->lut2.size() * (size_t)(amp_bytes(dtype) / 2));
  return Q2_OK;
}

q2_status q2_ansatz_table_bytes(const q2_ansatz *ansatz, q2_dtype dtype, size_t *device_bytes,
                                size_t *per_call_bytes) {
  if (!ansatz || !device_bytes) return fail(Q2_ERR_INVALID, "NULL argument");
  if (!valid_dtype(dtype)) return fail(Q2_ERR_INVALID, "unknown dtype");
  const RotPlan *rp;
  q2_status s = ansatz_tables(ansatz, dtype, &rp, nullptr);
  if (s != Q2_OK) return s;
  const size_t real = (size_t)amp_bytes(dtype) / 2;
  *device_bytes = sizeof(GroupDesc) * std::max<size_t>(1, rp->groups.size()) +
                  sizeof(BlockDesc) * std::max<size_t>(1, rp->blocks.size()) +
                  sizeof(uint64_t) * std::max<size_t>(1, rp->signmask.size()) +
                  real * std::max<size_t>(1, rp->wlut.size());
  if (per_call_bytes) *per_call_bytes = (size_t)amp_bytes(dtype) * (size_t)std::max<int64_t>(1, rp->lut_entries);
  return Q2_OK;
}

size_t q2_vqe_workspace_bytes(const q2_ansatz *ansatz, q2_dtype dtype, int want_grad) {
  if (!ansatz || !valid_dtype(dtype)) return 0;
  const RotPlan *rp;
  if (ansatz_tables(ansatz, dtype, &rp, nullptr) != Q2_OK) return 0;
  return ws_layout(ansatz->n, dtype, want_grad ? 1 : 0, rp->lut_entries, (int64_t)ansatz->x.size()).total;
}

q2_status q2_vqe_energy_grad(const q2_ansatz *ansatz, const q2_ham *ham, const double *theta, q2_dtype dtype,
                             int want_grad, double *energy_out, double *grad_out, void *workspace_dev,
                             size_t workspace_bytes, void *stream) {
  if (!ansatz || !ham || !energy_out) return fail(Q2_ERR_INVALID, "NULL argument");
  q2_status s = check_n(ansatz->n, dtype);
  if (s != Q2_OK) return s;
  if (ham->n != ansatz->n) return fail(Q2_ERR_INVALID, "Hamiltonian and ansatz qubit counts differ");
  if ((s = check_finite(ansatz->n_params, theta, "theta")) != Q2_OK) return s;
  if (want_grad && !grad_out) return fail(Q2_ERR_INVALID, "NULL gradient output");
  if (!workspace_dev || !aligned(workspace_dev, 256))
    return fail(Q2_ERR_INVALID, "workspace must be a 256-byte aligned device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return dtype == Q2_C64 ? vqe_impl<float>(ansatz, ham, theta, dtype, want_grad ? 1 : 0, energy_out, grad_out,
                                           workspace_dev, workspace_bytes, st)
                         : vqe_impl<double>(ansatz, ham, theta, dtype, want_grad ? 1 : 0, energy_out, grad_out,
                                            workspace_dev, workspace_bytes, st);
}

}  // extern "C"

namespace {

// ---- operator-pool gradients: Im<lambda|P_k|psi> for a list of Pauli strings at the final state

template <typename R>
q2_status pool_impl(const q2_ansatz *a, const q2_ham *h, const double *theta, q2_dtype d, int64_t n_pool,
                    const uint64_t *px, const uint64_t *pz, double *energy_out, double *pool_out, void *ws,
                    size_t ws_bytes, cudaStream_t st) {
  const RotPlan *rp;
  const DevTables *rt;
  q2_status s = ansatz_tables(a, d, &rp, &rt);
  if (s != Q2_OK) return s;
  const HamPlan *hp;
  const DevTables *ht;
  if ((s = ham_tables(h, d, &hp, &ht)) != Q2_OK) return s;
  const int n = a->n;
  const WsLayout L = ws_layout(n, d, 1, rp->lut_entries, (int64_t)a->x.size());
  if (ws_bytes < L.total) return fail(Q2_ERR_INVALID, "workspace too small");
  RotPlan pp;
  try {
    pp = build_rot_plan(n, n_pool, px, pz, tile_bits(d), g_chunk[d]);
  } catch (const std::exception &e) {
    return fail(Q2_ERR_INVALID, std::string("pool schedule: ") + e.what());
  }
  unsigned char *base = static_cast<unsigned char *>(ws);
  R *psi = reinterpret_cast<R *>(base + L.psi);
  R *lam = reinterpret_cast<R *>(base + L.lam);
  double *partial = reinterpret_cast<double *>(base + L.partial);
  double *out = reinterpret_cast<double *>(base + L.out);
  // forward: psi = U(theta)|HF>, lambda = H psi, E
  const size_t nrot = a->x.size();
  std::vector<double> phi(nrot);
  for (size_t k = 0; k < nrot; ++k) phi[k] = a->coef[k] * theta[a->param[k]];
  std::vector<double> lut2(2 * (size_t)std::max<int64_t>(1, rp->lut_entries));
  rp->build_lut(phi.data(), lut2.data());
  std::vector<unsigned char> lb = lut_bytes(lut2, d);
  Q2_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * 4, st), "clear results");
  unsigned *fault = fault_word(out);
  Q2_CUDA(cudaMemcpyAsync(base + L.lut, lb.data(), lb.size(), cudaMemcpyHostToDevice, st), "upload LUT");
  Q2_CUDA(launch_init_hf<R>(psi, n, a->n_elec, st), "init_hf");
  Q2_CUDA(run_sweep<R>(psi, n, *rp, rt->groups, rt->blocks, base + L.lut, fault, st), "sweep");
  Q2_CUDA(run_happly<R>(psi, lam, n, *hp, *ht, fault, st), "H apply");
  const int dgrid = dot_grid<R>(n);
  Q2_CUDA(launch_dot<R>(psi, lam, n, partial, dgrid, st), "dot");
  Q2_CUDA(launch_reduce_pairs(partial, dgrid, out, st), "reduce");
  // pool strings as rotations of angle 0 (cos = 1, sin = 0): the reverse sweep reads
  // Im<lambda|P_k|psi> for each and leaves psi and lambda unchanged
  std::vector<double> zero(std::max<int64_t>(1, n_pool), 0.0);
  std::vector<double> plut(2 * (size_t)std::max<int64_t>(1, pp.lut_entries));
  pp.build_lut(zero.data(), plut.data());
  std::vector<unsigned char> plb = lut_bytes(plut, d);
  const size_t o_groups = 0;
  const size_t o_sm = align_up(o_groups + sizeof(GroupDesc) * std::max<size_t>(1, pp.groups.size()), 256);
  const size_t o_lut = align_up(o_sm + sizeof(uint64_t) * std::max<size_t>(1, pp.signmask.size()), 256);
  const size_t o_g = align_up(o_lut + plb.size(), 256);
  const size_t total = o_g + sizeof(double) * (size_t)std::max<int64_t>(1, n_pool);
  unsigned char *tmp = nullptr;
  Q2_CUDA(cudaMallocAsync((void **)&tmp, total, st), "cudaMallocAsync(pool tables)");
  cudaError_t e = cudaSuccess;
  if (!pp.groups.empty())
    e = cudaMemcpyAsync(tmp + o_groups, pp.groups.data(), sizeof(GroupDesc) * pp.groups.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !pp.signmask.empty())
    e = cudaMemcpyAsync(tmp + o_sm, pp.signmask.data(), sizeof(uint64_t) * pp.signmask.size(),
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tmp + o_lut, plb.data(), plb.size(), cudaMemcpyHostToDevice, st);
  double *gpool = reinterpret_cast<double *>(tmp + o_g);
  for (size_t i = pp.passes.size(); e == cudaSuccess && i-- > 0;)
    e = launch_reverse<R>(psi, lam, n, pp.passes[i], reinterpret_cast<const GroupDesc *>(tmp + o_groups), nullptr,
                          false, tmp + o_lut, reinterpret_cast<const uint64_t *>(tmp + o_sm),
                          static_cast<const R *>(rt->wlut), partial, gpool, fault, st);
  double host_out[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, out, sizeof(host_out), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && n_pool)
    e = cudaMemcpyAsync(pool_out, gpool, sizeof(double) * (size_t)n_pool, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(tmp, st);
  const cudaError_t es = cudaStreamSynchronize(st);   // always: nothing may still use tmp or the outputs
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(e, "pool gradients");
  if (fault_of(host_out)) return fail(Q2_ERR_TIMEOUT, "a device wait for a tile copy timed out");
  *energy_out = host_out[0] / host_out[1];
  return Q2_OK;
}

}  // namespace

extern "C" {

q2_status q2_pool_gradients(const q2_ansatz *ansatz, const q2_ham *ham, const double *theta, q2_dtype dtype,
                            int64_t n_pool, const uint64_t *pool_x, const uint64_t *pool_z, double *energy_out,
                            double *grad_out, void *workspace_dev, size_t workspace_bytes, void *stream) {
  if (!ansatz || !ham || !energy_out || (n_pool > 0 && (!pool_x || !pool_z || !grad_out)))
    return fail(Q2_ERR_INVALID, "NULL argument");
  if (n_pool < 0) return fail(Q2_ERR_INVALID, "negative pool size");
  q2_status s = check_n(ansatz->n, dtype);
  if (s != Q2_OK) return s;
  if (ham->n != ansatz->n) return fail(Q2_ERR_INVALID, "Hamiltonian and ansatz qubit counts differ");
  if ((s = check_finite(ansatz->n_params, theta, "theta")) != Q2_OK) return s;
  if ((s = check_masks(ansatz->n, n_pool, pool_x, pool_z, "pool")) != Q2_OK) return s;
  if (!workspace_dev || !aligned(workspace_dev, 256))
    return fail(Q2_ERR_INVALID, "workspace must be a 256-byte aligned device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return dtype == Q2_C64 ? pool_impl<float>(ansatz, ham, theta, dtype, n_pool, pool_x, pool_z, energy_out,
                                            grad_out, workspace_dev, workspace_bytes, st)
                         : pool_impl<double>(ansatz, ham, theta, dtype, n_pool, pool_x, pool_z, energy_out,
                                             grad_out, workspace_dev, workspace_bytes, st);
}

size_t q2_batch_workspace_bytes(int n_requests, const q2_ansatz *const *ansatz, const q2_ham *const *ham,
                                q2_dtype dtype) {
  if (n_requests < 0 || (n_requests > 0 && (!ansatz || !ham)) || !valid_dtype(dtype)) return 0;
  size_t total = 0;
  if (batch_layout(n_requests, ansatz, dtype, nullptr, &total) != Q2_OK) return 0;
  return total;
}

q2_status q2_batch_energy_grad(int n_requests, const q2_ansatz *const *ansatz, const q2_ham *const *ham,
                               const double *const *theta, const int *want_grad, q2_dtype dtype,
                               double *energy_out, double *const *grad_out, void *workspace_dev,
                               size_t workspace_bytes, void *stream) {
  if (n_requests < 0) return fail(Q2_ERR_INVALID, "negative request count");
  if (n_requests == 0) return Q2_OK;
  if (!ansatz || !ham || !theta || !want_grad || !energy_out) return fail(Q2_ERR_INVALID, "NULL argument");
  if (!valid_dtype(dtype)) return fail(Q2_ERR_INVALID, "unknown dtype");
  if (!workspace_dev || !aligned(workspace_dev, 256))
    return fail(Q2_ERR_INVALID, "workspace must be a 256-byte aligned device pointer");
  for (int b = 0; b < n_requests; ++b) {
    if (!ansatz[b] || !ham[b] || !theta[b]) return fail(Q2_ERR_INVALID, "NULL request entry");
    if (ansatz[b]->n > SMALL_MAX_QUBITS) return fail(Q2_ERR_INVALID, "batched requests need n <= 12");
    if (ham[b]->n != ansatz[b]->n) return fail(Q2_ERR_INVALID, "Hamiltonian and ansatz qubit counts differ");
    if (ham[b]->n_shards != 1) return fail(Q2_ERR_UNSUPPORTED, "the batched path takes whole Hamiltonians, not shards");
    q2_status s = check_finite(ansatz[b]->n_params, theta[b], "theta");
    if (s != Q2_OK) return s;
    if (want_grad[b] && (!grad_out || !grad_out[b])) return fail(Q2_ERR_INVALID, "NULL gradient output");
  }
  std::vector<BatchSlot> slots;
  size_t total = 0;
  q2_status s = batch_layout(n_requests, ansatz, dtype, &slots, &total);
  if (s != Q2_OK) return s;
  if (workspace_bytes < total) return fail(Q2_ERR_INVALID, "workspace too small");
  unsigned char *ws = static_cast<unsigned char *>(workspace_dev);
  const size_t lut_b = dtype == Q2_C64 ? sizeof(float) : sizeof(double);
  std::vector<unsigned char> stage(slots.empty() ? 0 : slots.back().stage_end, 0);
  int max_n = 1, any_grad = 0;
  for (int b = 0; b < n_requests; ++b) {
    const q2_ansatz *a = ansatz[b];
    const DevTables *at;
    const int32_t *grot;
    const DevTables *ht;
    const HamPlan *hp;
    if ((s = small_ansatz_tables(a, &at, &grot)) != Q2_OK) return s;
    if ((s = small_ham_tables(ham[b], dtype, &hp, &ht)) != Q2_OK) return s;
    const RotPlan &rp = a->splan;
    std::vector<double> phi(a->x.size());
    for (size_t k = 0; k < phi.size(); ++k) phi[k] = a->coef[k] * theta[b][a->param[k]];
    std::vector<double> lut2(2 * (size_t)std::max<int64_t>(1, rp.lut_entries));
    rp.build_lut(phi.data(), lut2.data());
    unsigned char *dst = stage.data() + slots[b].lut_off;
    if (dtype == Q2_C64) {
      float *f = reinterpret_cast<float *>(dst);
      for (size_t i = 0; i < lut2.size(); ++i) f[i] = (float)lut2[i];
    } else {
      std::memcpy(dst, lut2.data(), lut2.size() * sizeof(double));
    }
    BatchItem it;
    std::memset(&it, 0, sizeof(it));
    it.rg = at->groups;
    it.grot = grot;
    it.sm = at->signmask;
    it.rlut = ws + slots[b].lut_off;
    it.hg = ht->groups;
    it.hlut = ht->lut;
    it.out = reinterpret_cast<double *>(ws + slots[b].out_off);
    it.nrg = (int32_t)rp.groups.size();
    it.nhg = (int32_t)hp->groups.size();
    it.n = a->n;
    it.n_elec = a->n_elec;
    it.want_grad = want_grad[b] ? 1 : 0;
    it.n_rot = (int32_t)a->x.size();
    std::memcpy(stage.data() + sizeof(BatchItem) * (size_t)b, &it, sizeof(it));
    max_n = std::max(max_n, a->n);
    any_grad |= it.want_grad;
    (void)lut_b;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Q2_CUDA(cudaMemcpyAsync(ws, stage.data(), stage.size(), cudaMemcpyHostToDevice, st), "upload batch");
  cudaError_t e = dtype == Q2_C64
                      ? launch_batch<float>(reinterpret_cast<const BatchItem *>(ws), n_requests, max_n, any_grad, st)
                      : launch_batch<double>(reinterpret_cast<const BatchItem *>(ws), n_requests, max_n, any_grad, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel");
  const size_t out_begin = slots[0].out_off;
  const size_t out_bytes = total - out_begin;
  std::vector<double> outs(out_bytes / sizeof(double));
  // The kernel is queued: synchronise before any return, so the workspace is never handed back in use.
  const cudaError_t ce = cudaMemcpyAsync(outs.data(), ws + out_begin, out_bytes, cudaMemcpyDeviceToHost, st);
  const cudaError_t se = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return cuda_fail(ce, "read batch");
  if (se != cudaSuccess) return cuda_fail(se, "sync");
  for (int b = 0; b < n_requests; ++b) {
    const double *o = outs.data() + (slots[b].out_off - out_begin) / sizeof(double);
    energy_out[b] = o[0] / o[1];
    if (want_grad[b]) {
      const q2_ansatz *a = ansatz[b];
      double *g = grad_out[b];
      for (int p = 0; p < a->n_params; ++p) g[p] = 0.0;
      for (size_t k = 0; k < a->x.size(); ++k) g[a->param[k]] += a->coef[k] * o[2 + k];
    }
  }
  return Q2_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ schedule introspection

#include "../../include/q2_debug.h"

static_assert(sizeof(PassDesc) == 152, "q2_pass layout");

extern "C" {

q2_status q2_debug_rot_plan(int n, int64_t n_rot, const uint64_t *x, const uint64_t *z, const double *angles,
                            int tile_qubits, int chunk_qubits, int64_t *counts, void *passes, void *groups,
                            void *blocks, double *lut2, uint64_t *signmask) {
  if (n < 1 || n > 34 || !counts) return fail(Q2_ERR_INVALID, "bad arguments");
  if (tile_qubits < 1 || tile_qubits > T_LIMIT || chunk_qubits < 1) return fail(Q2_ERR_INVALID, "bad tile shape");
  q2_status s = check_masks(n, n_rot, x, z, "rotations");
  if (s != Q2_OK) return s;
  RotPlan p;
  try {
    p = build_rot_plan(n, n_rot, x, z, tile_qubits, chunk_qubits);
  } catch (const std::exception &e) {
    return fail(Q2_ERR_INVALID, e.what());
  }
  counts[0] = (int64_t)p.passes.size();
  counts[1] = (int64_t)p.groups.size();
  counts[2] = p.lut_entries;
  counts[3] = (int64_t)p.blocks.size();
  if (passes) std::memcpy(passes, p.passes.data(), sizeof(PassDesc) * p.passes.size());
  if (groups) std::memcpy(groups, p.groups.data(), sizeof(GroupDesc) * p.groups.size());
  if (blocks) std::memcpy(blocks, p.blocks.data(), sizeof(BlockDesc) * p.blocks.size());
  if (lut2) {
    if ((s = check_finite(n_rot, angles, "angles")) != Q2_OK) return s;
    p.build_lut(angles, lut2);
  }
  if (signmask) std::memcpy(signmask, p.signmask.data(), sizeof(uint64_t) * p.signmask.size());
  return Q2_OK;
}

q2_status q2_debug_rot_weights(int n, int64_t n_rot, const uint64_t *x, const uint64_t *z, const int32_t *param,
                               const double *coef, int tile_qubits, int chunk_qubits, int64_t *n_weights,
                               void *groups, double *wlut, double *fold) {
  if (n < 1 || n > 34 || !n_weights || (n_rot > 0 && (!param || !coef))) return fail(Q2_ERR_INVALID, "bad arguments");
  if (tile_qubits < 1 || tile_qubits > T_LIMIT || chunk_qubits < 1) return fail(Q2_ERR_INVALID, "bad tile shape");
  q2_status s = check_masks(n, n_rot, x, z, "rotations");
  if (s != Q2_OK) return s;
  RotPlan p;
  try {
    p = build_rot_plan(n, n_rot, x, z, tile_qubits, chunk_qubits);
    set_param_weights(p, param, coef);
  } catch (const std::exception &e) {
    return fail(Q2_ERR_INVALID, e.what());
  }
  *n_weights = (int64_t)p.wlut.size();
  if (groups) std::memcpy(groups, p.groups.data(), sizeof(GroupDesc) * p.groups.size());
  if (wlut) std::memcpy(wlut, p.wlut.data(), sizeof(double) * p.wlut.size());
  if (fold) std::memcpy(fold, p.fold.data(), sizeof(double) * p.fold.size());
  return Q2_OK;
}

q2_status q2_debug_ham_plan(int n, int64_t n_terms, const uint64_t *x, const uint64_t *z, const double *coef,
                            int tile_qubits, int chunk_qubits, int64_t *counts, void *passes, void *groups,
                            void *blocks, double *lut2) {
  if (n < 1 || n > 34 || !counts) return fail(Q2_ERR_INVALID, "bad arguments");
  if (tile_qubits < 1 || tile_qubits > T_LIMIT || chunk_qubits < 1) return fail(Q2_ERR_INVALID, "bad tile shape");
  q2_status s = check_masks(n, n_terms, x, z, "Hamiltonian");
  if (s != Q2_OK) return s;
  if ((s = check_finite(n_terms, coef, "coefficients")) != Q2_OK) return s;
  HamPlan p;
  try {
    p = build_ham_plan(n, n_terms, x, z, coef, tile_qubits, chunk_qubits);
  } catch (const std::exception &e) {
    return fail(Q2_ERR_INVALID, e.what());
  }
  counts[0] = (int64_t)p.passes.size();
  counts[1] = (int64_t)p.groups.size();
  counts[2] = p.lut_entries;
  counts[3] = (int64_t)p.blocks.size();
  if (passes) std::memcpy(passes, p.passes.data(), sizeof(PassDesc) * p.passes.size());
  if (groups) std::memcpy(groups, p.groups.data(), sizeof(GroupDesc) * p.groups.size());
  if (blocks) std::memcpy(blocks, p.blocks.data(), sizeof(BlockDesc) * p.blocks.size());
  if (lut2) std::memcpy(lut2, p.lut2.data(), sizeof(double) * p.lut2.size());
  return Q2_OK;
}

int q2_debug_threads_per_cta(void) { return NT; }

q2_status q2_debug_sweep_fast_path(int enable) {
  g_canon4_enabled = enable != 0;
  return Q2_OK;
}

q2_status q2_debug_expect_fast_path(int enable) {
  g_lean_expect_enabled = enable != 0;
  return Q2_OK;
}

q2_status q2_debug_enable_timing(int enable) {
  g_timing.enabled = enable != 0;
  g_timing.valid = false;
  return Q2_OK;
}

q2_status q2_debug_wait_probe(unsigned polls, void *stream) {
  if (polls == 0 || polls > (1u << 22)) return fail(Q2_ERR_INVALID, "polls must be in 1..2^22");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned *fault = nullptr;
  Q2_CUDA(cudaMallocAsync((void **)&fault, sizeof(unsigned), st), "cudaMallocAsync(fault word)");
  unsigned host = 0;
  cudaError_t e = cudaMemsetAsync(fault, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = launch_wait_probe(polls, fault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, fault, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(fault, st);
  const cudaError_t es = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = es;
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  if (host) return fail(Q2_ERR_TIMEOUT, "a device wait for a tile copy timed out");
  return Q2_OK;
}

q2_status q2_debug_fp64_rate(double *flops_per_s, void *stream) {
  if (!flops_per_s) return fail(Q2_ERR_INVALID, "NULL output");
  Q2_CUDA(measure_fp64_rate(flops_per_s, static_cast<cudaStream_t>(stream)), "FP64 rate probe");
  return Q2_OK;
}

q2_status q2_debug_last_timing(double *out8) {
  if (!out8) return fail(Q2_ERR_INVALID, "NULL output");
  if (!g_timing.valid) return fail(Q2_ERR_INVALID, "no timed call on this thread");
  float ms[3] = {0, 0, 0};
  Q2_CUDA(cudaEventElapsedTime(&ms[0], g_timing.ev[0], g_timing.ev[1]), "elapsed");
  Q2_CUDA(cudaEventElapsedTime(&ms[1], g_timing.ev[1], g_timing.ev[2]), "elapsed");
  if (g_timing.has_reverse) Q2_CUDA(cudaEventElapsedTime(&ms[2], g_timing.ev[2], g_timing.ev[3]), "elapsed");
  out8[0] = ms[0];
  out8[1] = ms[1];
  out8[2] = ms[2];
  out8[3] = g_timing.counts[0];
  out8[4] = g_timing.counts[1];
  out8[5] = g_timing.counts[2];
  out8[6] = g_timing.total_launches;
  out8[7] = g_timing.counts[3];
  return Q2_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ helpers for noalloc.cu

namespace q2 {

// Host schedule of a Hamiltonian for a dtype, built and cached in the handle
// without any device work; *chunk receives the dtype's low contiguous qubits.
q2_status ham_host_plan(const q2_ham *hc, q2_dtype d, const HamPlan **plan, int *chunk) {
  q2_ham *h = const_cast<q2_ham *>(hc);
  std::lock_guard<std::mutex> g(h->mu);
  q2_status s = plan_ham_locked(h, d);
  if (s != Q2_OK) return s;
  *plan = &h->plan[d];
  *chunk = g_chunk[d];
  return Q2_OK;
}

int ham_qubits(const q2_ham *h) { return h->n; }

bool lean_expect_enabled() { return g_lean_expect_enabled; }

q2_status set_error(q2_status s, const char *msg) { return fail(s, msg); }

}  // namespace q2
