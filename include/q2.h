/*
 * q2.h -- C ABI of the GB300 state-vector engine for JW-mapped UCCSD-VQE.
 *
 * The operations are those of arXiv 2208.10978 (Q^2Chemistry):
 *   - the state vector of Eq. sv: 2^n complex amplitudes, qubit q = bit q of
 *     the amplitude index (little endian);
 *   - the Hartree-Fock determinant of Eq. jw-wfn-map;
 *   - the single-Trotter-step UCC circuit: a product of Pauli-string
 *     exponentials (the product formula following Eq. ucc);
 *   - the energy of a qubit Hamiltonian H = sum_i c_i P_i (Eq. qubit-ham,
 *     Eq. qubit-ham-detail);
 *   - reverse-mode differentiation (Algorithm 1).
 *
 * Pauli strings are two uint64 masks (x, z) meaning P = i^{popcount(x&z)} X^x Z^z,
 * so qubit q carries I, X, Z, Y for (x_q, z_q) = (0,0), (1,0), (0,1), (1,1).
 * A rotation (x, z, phi) is exp(-i phi/2 P); the paper's exp(i theta P) is
 * phi = -2 theta.
 *
 * Device memory layout: amplitudes interleaved (re, im): Q2_C64 = two float
 * (8 bytes per amplitude), Q2_C128 = two double (16 bytes).  Device buffers
 * must be 16-byte aligned.
 *
 * Ownership: device buffers (states, workspaces) belong to the caller; host
 * arrays are borrowed for the duration of the call; handles (q2_ham,
 * q2_ansatz) belong to the library until their destroy call.  A handle's
 * device tables are created on the device that is current at its first use
 * and must be used on that device only.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Calls returning results to host memory synchronize that stream.
 *
 * Errors: every call returns a q2_status; nothing throws across the ABI.
 * q2_last_error() gives a thread-local message for the last failure.
 * Q2_ERR_INVALID is returned, before any device work, for: n < 1,
 * n > 34 (Q2_C64) or n > 33 (Q2_C128), n_elec outside [0, n], a mask bit
 * >= n, a non-finite angle, coefficient or theta, a NULL pointer that is not
 * documented as optional, a misaligned device pointer, or a workspace that
 * is too small.  Q2_ERR_CUDA wraps launch and driver errors, Q2_ERR_OOM a
 * failed device allocation.  Q2_ERR_TIMEOUT: a bounded device-side wait for
 * a tile copy gave up (the kernel stops instead of spinning) and the results
 * of that call are not valid.  Each call that reads results back
 * (q2_expectation, q2_expectation_noalloc, q2_vqe_energy_grad,
 * q2_pool_gradients) counts its own give-ups in a fault word of its own
 * (in its workspace or temporary memory), so calls running concurrently on
 * other streams or threads never see each other's timeouts.  The
 * asynchronous calls (q2_apply_pauli_rotations, q2_apply_hamiltonian) count
 * give-ups in one per-device word that q2_async_status reads and clears.
 */
#ifndef Q2_H
#define Q2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    Q2_OK = 0,
    Q2_ERR_INVALID = 1,
    Q2_ERR_OOM = 2,
    Q2_ERR_CUDA = 3,
    Q2_ERR_TIMEOUT = 4,
    Q2_ERR_UNSUPPORTED = 5
} q2_status;

typedef enum { Q2_C64 = 0, Q2_C128 = 1 } q2_dtype;

typedef struct q2_ham q2_ham;
typedef struct q2_ansatz q2_ansatz;

/* Library version as major*10000 + minor*100 + patch. */
int q2_version(void);

/* Thread-local text of the last error (empty string if none). */
const char *q2_last_error(void);

/*
 * HF determinant (Eq. jw-wfn-map): psi = |1...1 0...0>, i.e. amplitude 1 at
 * index 2^n_elec - 1 and 0 elsewhere.  psi_dev: 2^n amplitudes of `dtype`.
 * Asynchronous on `stream`.
 */
q2_status q2_state_init_hf(void *psi_dev, int n, int n_elec, q2_dtype dtype, void *stream);

/*
 * psi <- U_{n_rot-1} ... U_1 U_0 psi with U_k = exp(-i angles[k]/2 P(xmask[k], zmask[k]))
 * (product formula after Eq. ucc; k ascending is the circuit order).
 * psi_dev: device, 2^n amplitudes, updated in place.  xmask, zmask, angles:
 * host arrays of n_rot entries (angles in radians, double).  n_rot = 0 is a
 * no-op.  The host builds a pass schedule (runs of rotations whose xmasks fit
 * one on-chip tile), uploads it to stream-ordered temporary device memory and
 * launches one tile kernel per pass; the call returns once the work is queued.
 */
q2_status q2_apply_pauli_rotations(void *psi_dev, int n, q2_dtype dtype, const uint64_t *xmask,
                                   const uint64_t *zmask, const double *angles, int64_t n_rot,
                                   void *stream);

/*
 * Qubit Hamiltonian H = sum_t coef[t] P(x[t], z[t]) (Eq. qubit-ham) on n
 * qubits.  Host arrays of n_terms entries, copied.  Terms are grouped by
 * xmask (the grouping keeps the sum exact; repeated strings are allowed and
 * add).  Coefficients are real: H is Hermitian.  *out receives the handle.
 */
q2_status q2_ham_create(int n, const uint64_t *x, const uint64_t *z, const double *coef,
                        int64_t n_terms, q2_ham **out);
q2_status q2_ham_destroy(q2_ham *ham);

/*
 * Timeouts of the asynchronous calls: synchronizes `stream`, then reads and
 * clears the count of bounded device waits that gave up in kernels of
 * q2_apply_pauli_rotations and q2_apply_hamiltonian on the current device
 * (all streams and host threads share this one count).  Returns
 * Q2_ERR_TIMEOUT if any did since the last check (the states those calls
 * wrote are then not valid), Q2_OK otherwise.
 */
q2_status q2_async_status(void *stream);

/*
 * Term-group parallelism (Sec. "Parallel evaluation of an expectation value",
 * Fig. 4: the Pauli strings are split over processes and the partial
 * energies are summed).  q2_ham_shard creates a handle for shard `shard` of
 * `n_shards` of `ham`: it holds a copy of all terms but evaluates only its
 * share of the xmask-group passes of ham's full schedule (for each dtype the
 * schedule is built as for ham, and its passes are dealt to the shards
 * largest first -- work = pair evaluations per amplitude plus one state
 * read -- each to the least loaded shard).  The shards of one Hamiltonian
 * partition its terms, so with the same psi (or ansatz and theta) the
 * energies of q2_expectation / q2_vqe_energy_grad on the shards, and their
 * gradients, sum to those of ham (each shard's energy is its share of
 * <psi|H|psi> divided by the full <psi|psi>); the gradient of a shard is that
 * of its share of <psi|H|psi>.  A shard may get no pass (more shards than
 * passes): its energy and gradient are then 0.  A shard cannot be sharded
 * again and is not accepted by q2_batch_energy_grad (Q2_ERR_UNSUPPORTED).
 * `n_shards` >= 1, 0 <= shard < n_shards.  *out is owned by the caller
 * (q2_ham_destroy).
 */
q2_status q2_ham_shard(const q2_ham *ham, int shard, int n_shards, q2_ham **out);

/*
 * Indices (into the term arrays given to q2_ham_create, ascending) of the
 * terms a handle evaluates for `dtype`: all terms for a whole Hamiltonian,
 * the shard's terms for a shard.  With idx_out = NULL only *count is set;
 * otherwise *count must hold idx_out's capacity on entry and receives the
 * number written.  Host only.
 */
q2_status q2_ham_shard_terms(const q2_ham *ham, q2_dtype dtype, int64_t *idx_out, int64_t *count);

/* Number of terms and of distinct xmask groups of a Hamiltonian handle. */
q2_status q2_ham_info(const q2_ham *ham, int64_t *n_terms, int64_t *n_groups);

/*
 * Energy (Eq. qubit-ham-detail) of psi: *energy_out = <psi|H|psi> / <psi|psi>,
 * *norm_out = <psi|psi> (norm_out may be NULL).  Both sums are accumulated in
 * double precision whatever the state dtype.  psi_dev is not modified.
 * Uses stream-ordered temporary device memory for block partial sums;
 * synchronizes `stream` before returning.
 */
q2_status q2_expectation(const void *psi_dev, int n, q2_dtype dtype, const q2_ham *ham,
                         double *energy_out, double *norm_out, void *stream);

/*
 * The energy of q2_expectation, computed without allocating device memory.
 * The paper has no counterpart: this is a calling convention of this library.
 *
 * For callers that may not allocate device memory while they run: code whose
 * device memory belongs to a framework's own pool, which forbids direct
 * driver allocations, or a latency-critical loop in which an allocation, and
 * the device-wide synchronization a free can imply, is not acceptable.
 * Where q2_expectation takes temporary device memory, this call uses one
 * fixed library buffer of Q2_NOALLOC_SCRATCH_BYTES (4 MiB): a static device
 * array that every GPU which loads the library holds until the process
 * exits.  It receives the per-CTA partial sums, the two result slots, the
 * call's fault word and a copy of the Hamiltonian's group, block and LUT
 * tables (uploaded on every call, so the handle's own device tables are not
 * needed).
 * Arguments and results are those of q2_expectation.  Extra error:
 * Q2_ERR_INVALID if the tables and partial sums do not fit the buffer (the
 * message gives the bytes needed); nothing is launched then.  The first call
 * in each CUDA context (that is, the first call on each device, and again
 * after that device's context has been destroyed and created anew) looks up
 * the buffer's device address with cudaGetSymbolAddress, with that device
 * current; make that first call before any stream capture.  Every call
 * shares the buffer, which keeps the last call's contents; a call clears the
 * parts that must start at zero (result slots and fault word) itself, on its
 * stream.  Calls that can overlap on the GPU (other streams, other host
 * threads on the same device) race, and the caller must serialize them.
 * Synchronizes `stream`.
 */
#define Q2_NOALLOC_SCRATCH_BYTES (4u << 20)
q2_status q2_expectation_noalloc(const void *psi_dev, int n, q2_dtype dtype, const q2_ham *ham,
                                 double *energy_out, double *norm_out, void *stream);

/*
 * lambda = H psi (the first step of Algorithm 1's backward pass).  psi_dev,
 * lam_dev: device, 2^n amplitudes each, distinct buffers; lam is overwritten.
 * Asynchronous on `stream`.
 */
q2_status q2_apply_hamiltonian(const void *psi_dev, void *lam_dev, int n, q2_dtype dtype,
                               const q2_ham *ham, void *stream);

/*
 * UCC ansatz as a rotation list: rotation j is exp(-i phi_j/2 P(x[j], z[j]))
 * with phi_j = coef[j] * theta[param_idx[j]], applied in order j = 0..n_rot-1
 * to |HF> with n_elec electrons (Eq. ucc after the JW mapping and the
 * first-order Trotter product).  Host arrays of n_rot entries, copied;
 * param_idx values in [0, n_params).  The pass schedule, the gradient
 * weights and the device tables are built once per dtype, at first use.
 */
q2_status q2_ansatz_create(int n, int n_elec, int64_t n_rot, const uint64_t *x, const uint64_t *z,
                           const int32_t *param_idx, const double *coef, int32_t n_params,
                           q2_ansatz **out);
q2_status q2_ansatz_destroy(q2_ansatz *ansatz);

/* Number of HBM passes and of rotation groups of the ansatz's schedule for a dtype. */
q2_status q2_ansatz_info(const q2_ansatz *ansatz, q2_dtype dtype, int64_t *n_passes,
                         int64_t *n_groups);

/*
 * Device bytes of the resident tables a handle uploads for `dtype` at its
 * first use by the tile kernels (the host schedule is built if needed):
 * group and register-block descriptors and the LUT of combined coefficients
 * for a Hamiltonian; group and block descriptors, sign masks and gradient
 * weights for an ansatz.  *per_call_bytes (may be NULL) receives the bytes of
 * the angle LUT that every q2_vqe_energy_grad call uploads.  Used for memory
 * accounting (the request loop charges resident tables to its budget) and to
 * count host-to-device traffic.
 */
q2_status q2_ham_table_bytes(const q2_ham *ham, q2_dtype dtype, size_t *device_bytes);
q2_status q2_ansatz_table_bytes(const q2_ansatz *ansatz, q2_dtype dtype, size_t *device_bytes,
                                size_t *per_call_bytes);

/*
 * Bytes of device workspace q2_vqe_energy_grad needs for this ansatz.  It takes
 * the ansatz rather than (n, dtype, want_grad) because the workspace also
 * holds the per-call angle LUT, whose size depends on the ansatz's schedule.
 */
size_t q2_vqe_workspace_bytes(const q2_ansatz *ansatz, q2_dtype dtype, int want_grad);

/*
 * One VQE evaluation: psi = U(theta)|HF>, *energy_out = <psi|H|psi>/<psi|psi>
 * and, if want_grad, grad_out[p] = dE/dtheta_p for p < n_params by the
 * reverse-mode sweep of Algorithm 1 (lambda = H psi, then psi and lambda are
 * un-rotated together and dE/dphi_j = Im <lambda|P_j|psi> is read before
 * rotation j is undone; dE/dtheta_p = sum_{j: param_j = p} coef_j dE/dphi_j).
 * The gradient is that of the unnormalised <psi|H|psi> (the state stays
 * normalised up to rounding).
 * theta: host, n_params doubles.  grad_out: host, n_params doubles, or NULL
 * when want_grad = 0.  workspace_dev: device buffer of at least
 * q2_vqe_workspace_bytes(ansatz, dtype, want_grad) bytes, 256-byte aligned.
 * On return its first 2^n amplitudes hold psi(theta) when want_grad = 0; with
 * want_grad they hold the state after the reverse sweep (|HF> up to rounding).
 * `ham` must act on the same n as the ansatz.  Synchronizes `stream`.
 */
q2_status q2_vqe_energy_grad(const q2_ansatz *ansatz, const q2_ham *ham, const double *theta,
                             q2_dtype dtype, int want_grad, double *energy_out, double *grad_out,
                             void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * Operator-pool gradients at U(theta)|HF>: grad_out[k] = Im <lambda|P_k|psi>
 * with psi = U(theta)|HF> and lambda = H psi, for the Pauli strings
 * P_k = (pool_x[k], pool_z[k]), k < n_pool.  This is dE/dphi of a rotation
 * exp(-i phi/2 P_k) appended to the circuit, at phi = 0: the screening step
 * of adaptive ansatz growth (the operator pools of Sec. "Variational quantum
 * circuit ansatz"), computed with the reverse-mode machinery of Algorithm 1
 * (the pool strings are grouped by xmask and read in one pass per group
 * span, without changing psi or lambda).  *energy_out = <psi|H|psi>/<psi|psi>.
 * theta: host, n_params doubles; pool_x, pool_z: host, n_pool masks (bits < n);
 * grad_out: host, n_pool doubles.  workspace_dev: at least
 * q2_vqe_workspace_bytes(ansatz, dtype, 1) bytes, 256-byte aligned.  The
 * pool's tables are built and freed on `stream` by the call.  Synchronizes
 * the stream.
 */
q2_status q2_pool_gradients(const q2_ansatz *ansatz, const q2_ham *ham, const double *theta, q2_dtype dtype,
                            int64_t n_pool, const uint64_t *pool_x, const uint64_t *pool_z, double *energy_out,
                            double *grad_out, void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * Batched evaluation of many small problems in one launch (the serving
 * path): request b uses ansatz[b], ham[b], theta[b] (host pointer to
 * n_params doubles) and want_grad[b]; every ansatz must have n <= 12.
 * One CTA keeps a whole state (and lambda) in shared memory and runs the
 * sweep, the energy and the reverse sweep without touching HBM except for
 * its tables.  energy_out[b] and, where want_grad[b], grad_out[b][0..n_params)
 * are written on the host.  workspace_dev must hold
 * q2_batch_workspace_bytes(...) bytes.  Synchronizes `stream`.
 */
size_t q2_batch_workspace_bytes(int n_requests, const q2_ansatz *const *ansatz,
                                const q2_ham *const *ham, q2_dtype dtype);
q2_status q2_batch_energy_grad(int n_requests, const q2_ansatz *const *ansatz,
                               const q2_ham *const *ham, const double *const *theta,
                               const int *want_grad, q2_dtype dtype, double *energy_out,
                               double *const *grad_out, void *workspace_dev,
                               size_t workspace_bytes, void *stream);

/*
 * Tile size tuning: number of qubits held on chip per tile of the rotation
 * passes for a dtype (default 12 for Q2_C64, 11 for Q2_C128; allowed 8..13
 * for Q2_C64 and 8..12 for Q2_C128).  Hamiltonian passes use one qubit more
 * (at most 13 for Q2_C64, 12 for Q2_C128).  Affects handles
 * and calls made afterwards.
 */
q2_status q2_set_tile_qubits(q2_dtype dtype, int tile_qubits);

#ifdef __cplusplus
}
#endif

#endif /* Q2_H */
