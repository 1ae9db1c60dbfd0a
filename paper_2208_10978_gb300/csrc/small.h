// Batched small-state evaluation (serving path): one CTA per request, whole
// state (and lambda) in shared memory.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "q2_internal.h"

namespace q2 {

constexpr int SMALL_MAX_QUBITS = 12;

// One request of a batch, as the kernel reads it (device pointers).
struct alignas(16) BatchItem {
  const GroupDesc *rg;      // rotation groups (single-tile plan, identity local basis)
  const int32_t *grot;      // first rotation of each rotation group
  const uint64_t *sm;       // per-rotation sign masks
  const void *rlut;         // rotation LUT for this request's angles (dtype precision)
  const GroupDesc *hg;      // Hamiltonian groups (single-tile plan)
  const void *hlut;         // Hamiltonian LUT (dtype precision)
  double *out;              // [0] <psi|H|psi>, [1] <psi|psi>, [2 + k] dE/dphi_k
  int32_t nrg, nhg, n, n_elec, want_grad, n_rot;
  int32_t pad[2];
};

template <typename R>
cudaError_t launch_batch(const BatchItem *items, int n_items, int max_qubits, int any_grad, cudaStream_t st);

}  // namespace q2
