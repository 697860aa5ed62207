/*
 * qf.h -- C ABI of libqf, a GB300 (sm_103a) state-vector engine for products of
 * Pauli-string exponentials and Pauli-sum expectation values, after the
 * state-vector simulator of QForte (Stair & Evangelista, arXiv:2108.04413).
 *
 * Conventions shared by every call
 * --------------------------------
 * Basis (Sec. "The QubitBasis class", Eq. 3): amplitude index b = sum_i q_i 2^i,
 *   bit i of b is qubit q_i.  A state of n qubits is 2^n complex amplitudes,
 *   stored interleaved (re, im): 16 bytes each for QF_C128 (two doubles),
 *   8 bytes each for QF_C64 (two floats), amplitude b at byte offset b*size.
 * Pauli string (Eq. 10): a pair of bit masks (x, z); qubit i carries X if only
 *   x_i is set, Z if only z_i is set, Y if both are set.  It is the Hermitian
 *   operator P with P|b> = i^{popc(x&z)} (-1)^{popc(z&b)} |b xor x>.
 * Rotation (Eq. 9 with the factor -i*theta of the worked example Eq. 11-13):
 *   exp(-i theta P) = cos(theta) I - i sin(theta) P.
 * Circuits are applied in list order: element 0 acts first on the state.
 *
 * Streams, ownership, errors
 * --------------------------
 * Every call that touches a state runs on the CUDA stream given at creation and
 * returns once its work is queued, except calls that return host values
 * (qf_expectation, qf_energy_grad, qf_state_copy_to_host), which synchronise
 * that stream.  Input arrays are read (and planned) before a call returns, so
 * the caller may free them afterwards.  Handles are owned by the library and
 * released with qf_state_destroy; a handle must not be used by two host
 * threads at once (distinct handles on distinct streams may run concurrently).
 * Every call returns a qf_status; on failure the state is unchanged unless the
 * status is QF_ECUDA, and qf_last_error() gives a thread-local message.
 * Invalid arguments (null pointers, n outside 1..QF_MAX_QUBITS, a mask with a
 * bit at or above n, a parameter index outside the parameter array, a size
 * that does not match the state) give QF_EINVAL before any GPU work.
 */
#ifndef QF_H
#define QF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QF_MAX_QUBITS 34

typedef enum { QF_OK = 0, QF_EINVAL = 1, QF_ENOMEM = 2, QF_ECUDA = 3, QF_ETIMEOUT = 4 } qf_status;
typedef enum { QF_C128 = 0, QF_C64 = 1 } qf_dtype;

/* One rotation exp(-i theta P(x, z)). */
typedef struct { uint64_t x, z; double theta; } qf_rot;
/* One Hamiltonian term coeff * P(x, z); real coeff, so the sum is Hermitian (Eq. 2). */
typedef struct { uint64_t x, z; double coeff; } qf_term;
/* One ansatz rotation exp(-i theta P(x, z)) with theta = coeff * t[param]. */
typedef struct { uint64_t x, z; double coeff; int32_t param; int32_t reserved; } qf_arot;

typedef struct qf_state qf_state;

/* Create a state of n qubits (the "Computer" of Eq. 4 / Lst. 1), initialised to
 * |0...0>.  stream: a cudaStream_t (NULL = legacy default stream).
 * dev_buf: NULL to let the library allocate the 2^n amplitudes, or caller-owned
 * device memory of dev_buf_bytes >= 2^n * size bytes, 256-byte aligned, which must
 * outlive the handle.  Work buffers (reduction partials, and the second state
 * used by qf_energy_grad) are allocated by the library.  QF_ENOMEM if an
 * allocation fails. */
qf_status qf_state_create(int n, qf_dtype dtype, void* stream, void* dev_buf, size_t dev_buf_bytes,
                          qf_state** out);
qf_status qf_state_destroy(qf_state* st);

/* Set the state to the basis determinant |det> (Eq. 17's reference |Phi_0>). */
qf_status qf_set_basis(qf_state* st, uint64_t det);

/* Apply exp(-i theta P(x, z)) (Eq. 9, Lst. 4). */
qf_status qf_apply_pauli_exp(qf_state* st, uint64_t x, uint64_t z, double theta);

/* Apply the product of n_rot rotations in list order (a Circuit, Sec. "The
 * Circuit class"; the dUCC product of Eq. 19 once each theta is known).  The
 * library fuses runs of rotations internally; the result equals applying them
 * one by one up to rounding. */
qf_status qf_apply_circuit(qf_state* st, const qf_rot* rots, size_t n_rot);

/* Exact operator averaging <psi|H|psi> for H = sum_l coeff_l P_l (Eq. 18, Lst. 5).
 * Terms may repeat.  *re receives the value; *im receives 0 (the coefficients
 * are real, so the value is real; the kernel sums each amplitude pair's two
 * Hermitian-conjugate contributions together).  Synchronises the stream. */
qf_status qf_expectation(qf_state* st, const qf_term* terms, size_t n_terms, double* re, double* im);

/* (Calls that run a persistent kernel with grid barriers -- qf_apply_circuit
 * and qf_trotter on sector states -- return QF_ETIMEOUT if a barrier wait
 * exceeds 2 s.) */

/* Energy and gradient of E(t) = <Phi|U(t)^+ H U(t)|Phi> (Eq. 17-18) with
 * |Phi> = |det> and U(t) the ansatz rotations in list order, theta_k = coeff_k *
 * t[param_k].  The gradient comes from a reverse (adjoint) sweep:
 * dE/dtheta_k = 2 Im <lambda_k|P_k|psi_k>, dE/dt_p = sum_{k: param_k = p} coeff_k
 * dE/dtheta_k.  U(t)|Phi> has unit norm; the returned energy and gradient are
 * divided by the computed <psi|psi> (FP64), which removes the rounding drift of
 * the stored norm (it matters for QF_C64 states).  grad has n_par entries.  The
 * reverse sweep undoes the circuit, so on return the state holds |det> again
 * up to rounding (call qf_apply_circuit to rebuild U(t)|Phi>); when every
 * block keeps the reference's alpha and beta occupation counts it holds |det>
 * exactly.  Device memory kept with the handle after the first call that needs
 * it: a second state-sized buffer (lambda = H psi) for the general path; on that
 * sector path instead a compact copy of the sector (2 * members amplitudes),
 * the run plan's tables, and a forward log of one amplitude pair per (member
 * pair, excitation) item -- 2.05 GB for a 24-qubit dUCCSD in complex128, at
 * most 16 GB (past that, or if it cannot be allocated, the reverse sweep
 * recomputes psi instead).  qf_state_destroy frees it.
 * Synchronises the stream. */
qf_status qf_energy_grad(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                         size_t n_par, const qf_term* terms, size_t n_terms, double* energy, double* grad);

/* Energy and gradient for n_req parameter vectors of one system (the paper has
 * no counterpart: a serving path for many small requests).  t holds n_req rows
 * of n_par parameters; energies[q] and, when grads is not NULL, grads[q * n_par ..]
 * are those qf_energy_grad gives for row q (equal within rounding: the
 * summation order differs).  Once the handle has planned this ansatz and
 * Hamiltonian for this sector (a qf_energy_grad call does; the first call here
 * runs its first row through qf_energy_grad to do so), and when every block is
 * a real two-row sector block, H has direct sector tables and the sector's
 * psi and lambda fit in one CTA's shared memory (about 6000 members in
 * QF_C128, 12000 in QF_C64: up to 16 qubits at half filling), all rows run in
 * ONE kernel launch, one CTA per row, each holding its state in shared memory
 * through the forward blocks, H|psi> and the reverse blocks.  Otherwise the rows
 * run one after another through qf_energy_grad.  Errors as qf_energy_grad.
 * Synchronises the stream; leaves the state holding |det>. */
qf_status qf_energy_grad_multi(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                               size_t n_par, size_t n_req, const qf_term* terms, size_t n_terms, double* energies,
                               double* grads);

/* PQE residuals (Sec. PQE, Eq. 23): for each of the n_dets basis determinants b,
 * res[2k] + i res[2k+1] = <b| U(t)^+ H U(t) |det> / |U(t) det|, with the energy
 * and, when grad is not NULL, the gradient of qf_energy_grad (same arguments,
 * same pass).  The residual of an excited determinant tau_mu|det> is its
 * fermionic sign times the value at tau_mu's basis index (the host prep module
 * gives both).  res holds 2 * n_dets doubles.  The value is read from
 * lambda = U^+ H U |det> at the end of the reverse sweep.  When every b shares
 * the reference's alpha and beta occupation counts the compact sector path
 * computes it; otherwise the call takes the general path, since H may connect
 * sectors.  A bit of b at or above n gives QF_EINVAL.  Synchronises the stream;
 * leaves the state as qf_energy_grad does. */
qf_status qf_residuals(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                       size_t n_par, const qf_term* terms, size_t n_terms, const uint64_t* dets, size_t n_dets,
                       double* energy, double* grad, double* res);

/* Operator-pool gradients of ADAPT (Sec. ADAPT, Eq. 21): for the state
 * psi = U(t)|det>, pool_grad[p] = <psi|[H, kappa_p]|psi> for each pool operator p,
 * where the pool is a rotation list like an ansatz (pool[k].param in [0, n_pool)
 * names its operator, exp(s_p kappa_p) = prod_{k in p} exp(-i s_p coeff_k P_k)).
 * Equivalently, the derivative at s = 0 of the energy with the operator
 * appended to the ansatz.  Also returns the energy.  On the compact sector path
 * (every ansatz and pool block a sector block, real H) one overlap pass on the
 * final (psi, H psi) gives every pool gradient and no reverse sweep is run.
 * Otherwise the pool is appended to the ansatz at zero angle and differentiated
 * with qf_energy_grad's general path.  The pool's block structure is planned
 * once per handle.  Synchronises the stream. */
qf_status qf_pool_gradients(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                            size_t n_par, const qf_term* terms, size_t n_terms, const qf_arot* pool, size_t n_pool_rot,
                            size_t n_pool, double* energy, double* pool_grad);

/* Trotterized time evolution (Eq. 39, used by the quantum Krylov methods): apply
 * (prod_l exp(-i time coeff_l P_l / steps))^steps, the terms in list order
 * within each step, through the fused rotation path of qf_apply_circuit.
 * steps < 1 or a non-finite time gives QF_EINVAL. */
qf_status qf_trotter(qf_state* st, const qf_term* terms, size_t n_terms, double time, int steps);

/* Copy the state to / from host memory (bytes must equal 2^n * size).  The
 * copy to host folds the internal scale into the amplitudes first. */
qf_status qf_state_copy_to_host(qf_state* st, void* host, size_t bytes);
qf_status qf_state_copy_from_host(qf_state* st, const void* host, size_t bytes);

/* The library may keep a state as scale * stored amplitudes (a rotation then
 * costs two fused multiply-adds per amplitude instead of four).  This folds the
 * scale into the stored amplitudes so that device memory holds the state
 * itself.  Queued on the stream. */
qf_status qf_state_fold_scale(qf_state* st);

/* Query a state: qubit count, dtype, device pointer of the amplitudes and the
 * current scale (amplitudes = scale * stored values).  Any pointer may be NULL. */
qf_status qf_state_info(const qf_state* st, int* n, qf_dtype* dtype, void** dev_ptr, double* scale);

/* Arithmetic of qf_energy_grad's H|psi> for QF_C128 states that are exactly
 * real with a Hamiltonian whose strings all have an even number of Y letters
 * (every dUCC state of a real Hamiltonian).  GB300 runs FP64 multiply-adds at
 * 1/58 of its FP32 rate, and this step needs one per (X group, amplitude).
 * QF_HPSI_FP64: FP64 multiply-adds.  QF_HPSI_DS (default): double-single
 * multiply-adds on the FP32 pipe -- values and tables split into (hi, lo) float
 * pairs (~48 bits), products formed exactly in their leading part, error-free
 * TwoSum accumulation, FP64 for the energy, norm and overlaps; relative error
 * per operation ~2^-46.  Other states always use FP64. */
#define QF_HPSI_FP64 0
#define QF_HPSI_DS 1
qf_status qf_state_set_hpsi_mode(qf_state* st, int mode);

/* Drop the Pauli-sum plans (X-mask groups and their tables) cached in the
 * handle, so the next qf_expectation / qf_energy_grad groups and uploads its
 * terms again. */
qf_status qf_state_clear_plans(qf_state* st);

/* Number of kernels this thread's calls have launched since the last reset
 * (reset = 1 clears the counter after reading). */
uint64_t qf_kernel_launches(int reset);

/* Bytes this thread's calls have copied host-to-device (state uploads, plan
 * tables, block descriptors) and device-to-host (results, state downloads)
 * since the last reset (reset = 1 clears after reading).  Either pointer may be
 * NULL. */
void qf_transfer_bytes(int reset, uint64_t* h2d_bytes, uint64_t* d2h_bytes);

/* Kernel kinds for the timing calls below. */
#define QF_K_SET 1u          /* basis preparation, scale folding */
#define QF_K_ROT 2u          /* unfused rotation (one pair sweep) */
#define QF_K_TILE 4u         /* fused rotations in shared-memory tiles */
#define QF_K_SPARSE 8u       /* sparse composite block */
#define QF_K_EXPECT 16u      /* grouped expectation value */
#define QF_K_HPSI 32u        /* H|psi> with <psi|H|psi> and <psi|psi> */
#define QF_K_ADJ_ROT 64u     /* adjoint step of one rotation */
#define QF_K_ADJ_SPARSE 128u /* adjoint step of a sparse block */

/* Kernel timing for this host thread: after qf_profile_begin(mask), every launch
 * of a kind in mask is bracketed by two CUDA events recorded on its stream.
 * qf_profile_read waits for the recorded events and returns, for the kinds in
 * mask, the number of launches and their summed device time in milliseconds.
 * qf_profile_end stops recording and drops the records. */
qf_status qf_profile_begin(unsigned kind_mask);
qf_status qf_profile_read(unsigned kind_mask, uint64_t* launches, double* total_ms);
qf_status qf_profile_end(void);

/* Plan introspection for measurement (the paper has no counterpart).  For the
 * last qf_energy_grad / qf_residuals call on st that ran its sweeps as
 * part-local runs of the compact sector layout (one kernel launch per run and
 * sweep): the number of runs into *n_runs and, for the first min(cap, runs)
 * runs in plan order, the (sector member pair, excitation) items one sweep
 * processes in that run into items (host array of cap entries; may be NULL when
 * cap = 0).  The forward sweep launches the runs in plan order, the reverse
 * sweep last to first.  The items of all runs sum to the forward log's pair
 * count.  QF_EINVAL when no such sweep has run on st. */
qf_status qf_sweep_run_items(const qf_state* st, uint64_t* items, size_t cap, size_t* n_runs);

/* Allocation-free expectation value.  The paper has no counterpart: this call
 * exists for callers that cannot allocate device memory -- for instance when
 * all of the GPU's memory is already reserved by another allocator (a
 * framework's caching pool, a serving process with a fixed memory budget), or
 * in a latency-critical loop that must not take cudaMalloc's implicit device
 * synchronisation.  qf_expectation needs a qf_state, whose creation allocates;
 * this call computes the same <psi|H|psi> (same kernel, same precision) from
 * amplitudes the caller owns.
 *   amplitudes: device pointer to 2^n amplitudes in the layout above (the state
 *     itself, no separate scale), 16-byte aligned; not modified.
 *   stream: cudaStream_t the work is queued on (NULL = legacy default stream);
 *     the call synchronises it before returning *re (and *im = 0).
 *   terms: host array of n_terms <= QF_NOALLOC_MAX_TERMS terms (more gives
 *     QF_EINVAL before any GPU work).
 * It calls no cudaMalloc / cudaFree: its scratch (reduction partials, counter,
 * result and grouped term tables) is one static device array of
 * QF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress), so make the first call on each device before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents (the counter is cleared at each call's start).  Two calls whose GPU
 * work overlapped would race on it; to prevent that, a call holds a
 * process-wide lock from uploading its tables until its stream has
 * synchronised, so calls from several host threads (on any streams) run one
 * after another. */
#define QF_NOALLOC_MAX_TERMS 2048
#define QF_NOALLOC_SCRATCH_BYTES (1u << 20)
qf_status qf_expectation_noalloc(const void* amplitudes, int n, qf_dtype dtype, void* stream,
                                 const qf_term* terms, size_t n_terms, double* re, double* im);

/* Measured FP64 arithmetic peaks of the current device (the paper has no
 * counterpart: a measurement helper for roofline denominators; GB300 runs FP64 at
 * a small fraction of its FP32 rate, so these bound the complex128 kernels).
 *   fma_flops: FP64 fused multiply-add throughput of the CUDA cores;
 *   dmma_flops: FP64 matrix multiply-accumulate throughput (mma.sync m8n8k4);
 * both in flop/s (one multiply-add = 2 flop), from kernels of independent
 * operations on every SM, each timed with CUDA events on `stream` after a
 * warm-up launch.  Either pointer may be NULL.  Allocates a few KB of scratch,
 * takes tens of milliseconds and synchronises the stream. */
qf_status qf_probe_fp64_peaks(void* stream, double* fma_flops, double* dmma_flops);

/* Self-test of the bounded device wait used by the grid barriers of the
 * persistent kernels: one thread waits up to limit_s seconds (0 < limit_s <= 10)
 * on a word that nothing changes.  Returns QF_ETIMEOUT when the wait gave up as
 * designed (the context stays usable), QF_ECUDA otherwise. */
qf_status qf_selftest_bounded_wait(void* stream, double limit_s);

/* Thread-local message describing the last failure. */
const char* qf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QF_H */
