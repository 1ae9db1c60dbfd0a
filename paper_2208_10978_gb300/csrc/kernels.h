// Launchers of the tile kernels (kernels.cu); R = float (complex64) or double (complex128).
#pragma once

#include <cuda_runtime.h>

#include "q2_internal.h"

namespace q2 {

size_t tile_smem_bytes(int amp_bytes, int T, int C, int vectors);
size_t reverse_smem_bytes(int amp_bytes, int T, int C);
int max_grid_blocks(int amp_bytes, int T);
cudaError_t launch_reduce_pairs(const double *partial, int nblocks, double *out, cudaStream_t st);
// Bounded device waits for bulk tile copies.  Every tile kernel takes a fault
// word (device, zeroed by the calling API function before its first launch)
// to which a wait that gives up adds one; with fault == nullptr the give-up is
// counted in a per-device word for the asynchronous calls, read and cleared
// by take_async_faults.
cudaError_t take_async_faults(unsigned *host, cudaStream_t st);
cudaError_t launch_wait_probe(uint32_t polls, unsigned *fault, cudaStream_t st);
// Measured FP64 FMA throughput of the device (flop/s), timed with events on st.
cudaError_t measure_fp64_rate(double *flops_per_s, cudaStream_t st);

template <typename R> cudaError_t launch_init_hf(R *psi, int n, int n_elec, cudaStream_t st);
template <typename R>
cudaError_t launch_sweep(R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                         const BlockDesc *blocks, const void *lut, unsigned *fault, bool canon4, cudaStream_t st);
template <typename R> int expect_grid(int n, int T, int C);
template <typename R>
cudaError_t launch_expect(const R *psi, int n, const PassDesc &pd, const GroupDesc *groups,
                          const BlockDesc *blocks, const void *lut, double *partial, int grid, bool first,
                          unsigned *fault, bool lean, cudaStream_t st);
template <typename R>
cudaError_t launch_happly(const R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                          const BlockDesc *blocks, const void *lut, bool first, unsigned *fault,
                          cudaStream_t st);
template <typename R> int dot_grid(int n);
template <typename R>
cudaError_t launch_dot(const R *psi, const R *lam, int n, double *partial, int grid, cudaStream_t st);
template <typename R>
cudaError_t launch_reverse(R *psi, R *lam, int n, const PassDesc &pd, const GroupDesc *groups,
                           const BlockDesc *blocks, bool one_param, const void *lut, const uint64_t *signmask,
                           const R *wlut, double *partial, double *gphi, unsigned *fault, cudaStream_t st);

}  // namespace q2
