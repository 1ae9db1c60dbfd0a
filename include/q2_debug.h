/*
 * q2_debug.h -- introspection of the host schedules behind include/q2.h.
 *
 * These calls run on the host only (no device work) and expose the pass and
 * group tables that q2_apply_pauli_rotations / q2_ansatz_create and
 * q2_ham_create build, so that the schedule can be checked without a GPU.
 * The paper has no counterpart: they describe this library's tiling of the
 * state vector, not the method.
 *
 * Layouts (little endian, packed as below; see the library's q2_internal.h):
 *   q2_pass  (152 bytes): uint64 w[13] local basis; uint64 umask; int32 T, C,
 *            g_begin, g_end, rot_begin, rot_end, lut_begin, lut_count,
 *            b_begin, b_end.
 *   q2_group (272 bytes): uint64 bp[8] code basis in packed-index space;
 *            uint32 xl, lut, rot0; uint8 kind, r, m, a; uint8 bjcode[16],
 *            bccode[16], blane[32], bwarp[8] (register-block enumeration);
 *            uint8 pivot, one_param, pad[2]; uint32 wlut; uint8 pjcode[32],
 *            plane[32], pwarp[8]; uint16 pu[16] (pair enumeration); uint8 pad[8].
 *            one_param/wlut are set only for ansatz handles (gradient weights).
 *   q2_block (80 bytes): uint16 comb[16], uj[16]; uint8 d, piv[4], canon, pad[2];
 *            uint16 g_begin, g_end; uint8 pad[4].
 * counts[0..3] = number of passes, groups, LUT entries, register blocks.
 * Output arrays may be NULL (sizes only); otherwise they must hold counts[]
 * entries.  lut2 holds two doubles per entry: (cos, sin) of the combined
 * angle for rotation plans, (R, Q) combined coefficients for Hamiltonian
 * plans.  signmask (rotation plans, n_rot entries): bit c set iff rotation k
 * enters its group's angle with a minus sign at code c.
 * Errors: Q2_ERR_INVALID for bad sizes or masks (see q2.h).
 */
#ifndef Q2_DEBUG_H
#define Q2_DEBUG_H

#include "q2.h"

#ifdef __cplusplus
extern "C" {
#endif

q2_status q2_debug_rot_plan(int n, int64_t n_rot, const uint64_t *x, const uint64_t *z,
                            const double *angles, int tile_qubits, int chunk_qubits,
                            int64_t *counts, void *passes, void *groups, void *blocks,
                            double *lut2, uint64_t *signmask);

q2_status q2_debug_ham_plan(int n, int64_t n_terms, const uint64_t *x, const uint64_t *z,
                            const double *coef, int tile_qubits, int chunk_qubits,
                            int64_t *counts, void *passes, void *groups, void *blocks,
                            double *lut2);

/*
 * Gradient tables of an ansatz's rotation schedule (the ones q2_vqe_energy_grad
 * uses): the groups of q2_debug_rot_plan with one_param and wlut set, the
 * weights w_g(code) = sum_k coef_k sign_k(code) of every one-parameter group
 * (*n_weights doubles in total, group g's at its wlut offset) and per
 * rotation the factor that folds its reverse-sweep sum into dE/dtheta
 * (n_rot doubles).  Output arrays may be NULL (sizes only).
 */
q2_status q2_debug_rot_weights(int n, int64_t n_rot, const uint64_t *x, const uint64_t *z, const int32_t *param,
                               const double *coef, int tile_qubits, int chunk_qubits, int64_t *n_weights,
                               void *groups, double *wlut, double *fold);

/* Threads per CTA of the tile kernels (the per-thread offsets of q2_group.jcode use it). */
int q2_debug_threads_per_cta(void);

/*
 * Per-phase device timing of q2_vqe_energy_grad, for benchmarks.  When
 * enabled (per calling thread), the call records CUDA events on its own
 * stream around each phase; q2_debug_last_timing then fills out[0..7] with
 * the last call's: sweep ms, expectation ms (energy-only) or H-apply + dot ms
 * (gradient), reverse-sweep ms, number of sweep kernels, number of
 * expectation / H-apply kernels, number of reverse kernels, total kernels
 * launched, and the state bytes (2^n * amplitude size).  Returns
 * Q2_ERR_INVALID if timing was off for the last call.
 */
q2_status q2_debug_enable_timing(int enable);
q2_status q2_debug_last_timing(double *out8);

/*
 * Failure-path check of the bounded device waits: launches one CTA that
 * waits, with `polls` polls (1..2^22), on an mbarrier that nothing completes
 * -- the situation of a tile copy that never lands.  The wait gives up,
 * the kernel returns, and the call reports it exactly as the compute calls
 * do: Q2_ERR_TIMEOUT, counted in a fault word of this call's own (so
 * concurrent calls on other streams are not affected).  Q2_OK would mean the
 * give-up path is broken.  Synchronizes the stream.
 */
q2_status q2_debug_wait_probe(unsigned polls, void *stream);

/*
 * Measured FP64 fused multiply-add throughput of the current device in flop/s
 * (one launch of independent FMA chains on every SM, timed with CUDA events on
 * `stream`): the denominator of the complex128 sweep's FP64-ALU roofline.
 */
q2_status q2_debug_fp64_rate(double *flops_per_s, void *stream);

/*
 * Tests only: enable (default) or disable the fast path of the rotation sweep
 * for passes made of canonical 4-dimensional register blocks, so that both the
 * fast path and the general block path can be checked against the oracle.
 * Affects calls made afterwards, on every thread.
 */
q2_status q2_debug_sweep_fast_path(int enable);

/*
 * Tests only: enable (default) or disable the lean path of the expectation
 * (complex64 passes of REAL and DIAG groups in blocks of at most 3 dimensions),
 * so that both it and the general path can be checked against the oracle.
 * Affects calls made afterwards, on every thread.
 */
q2_status q2_debug_expect_fast_path(int enable);

#ifdef __cplusplus
}
#endif

#endif /* Q2_DEBUG_H */
