// Launchers of the tile kernels (kernels.cu); R = float (complex64) or double (complex128).
#pragma once

#include <cuda_runtime.h>

#include "q2_internal.h"

namespace q2 {

size_t tile_smem_bytes(int amp_bytes, int T, int C, int vectors);
size_t reverse_smem_bytes(int amp_bytes, int T, int C);
int max_grid_blocks(int amp_bytes, int T);
cudaError_t launch_reduce_pairs(const double *partial, int nblocks, double *out, cudaStream_t st);
// Bounded device waits that gave up (bulk tile copies), counted since the last clear.
cudaError_t read_wait_timeouts_async(unsigned *host, cudaStream_t st);
cudaError_t clear_wait_timeouts(cudaStream_t st);
cudaError_t launch_wait_probe(uint32_t polls, cudaStream_t st);

template <typename R> cudaError_t launch_init_hf(R *psi, int n, int n_elec, cudaStream_t st);
template <typename R>
cudaError_t launch_sweep(R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                         const BlockDesc *blocks, const void *lut, cudaStream_t st);
template <typename R> int expect_grid(int n, int T, int C);
template <typename R>
cudaError_t launch_expect(const R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                          const BlockDesc *blocks, const void *lut, double *partial, int grid, bool first,
                          cudaStream_t st);
template <typename R>
cudaError_t launch_happly(const R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                          const BlockDesc *blocks, const void *lut, bool first, cudaStream_t st);
template <typename R> int dot_grid(int n);
template <typename R>
cudaError_t launch_dot(const R *psi, const R *lam, int n, double *partial, int grid, cudaStream_t st);
template <typename R>
cudaError_t launch_reverse(R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                           const BlockDesc *blocks, bool one_param, const void *lut, const uint64_t *signmask,
                           const R *wlut, double *partial, double *gphi, cudaStream_t st);

}  // namespace q2
