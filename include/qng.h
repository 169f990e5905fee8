/*
 * qng.h - C ABI of libqng, a GB300 (sm_103a) library for the quantum natural gradient of a
 * P-parameter unitary ansatz, after T. Jones, "Efficient classical calculation of the Quantum
 * Natural Gradient" (arXiv:2011.02991).
 *
 * What the library computes, for a circuit U(theta) = W U_P(theta_P) ... U_1(theta_1) acting on
 * |in> = |0...0> and a Hamiltonian H = sum_k c_k sigma_k of Pauli strings:
 *   - the Fubini-Study metric g = Re G, G_ij = <d_i psi|d_j psi> - <d_i psi|psi><psi|d_j psi>
 *     (Eq. 4), evaluated through the paper's recurrences: T_i = <psi_i|dU_i|psi_{i-1}>
 *     (Eq. t_recurrent_def), L_ij = prod[dU_i psi_{i-1}, phi_{i+1,j}] (Eq. L_recurrent_def),
 *     L_ii = 1/4 a priori (Eq. L_diag_when_single_pauli) and G_ij = L_ij - T_i^* T_j
 *     (Eq. g_t_L_def), organised as Algorithm 1 (Sec. 3);
 *   - the energy <E> = <psi|H|psi> and its gradient d<E>/d theta_i (Eq. 2);
 *   - the natural-gradient step dtheta solving (g + lambda I) dtheta = -dt grad<E> (Eq. 3 with a
 *     Tikhonov term lambda added to every diagonal entry).
 *
 * Conventions
 *   - Parametric gates are R_sigma(theta) = exp(-i theta sigma / 2), sigma in {X, Y, Z}; the k-th
 *     parametric gate of a circuit must carry param == k (one unique parameter per gate, Sec. 2).
 *   - Fixed gates between parametric gates k-1 and k belong to U_k = R_k F_k; fixed gates after
 *     the last parametric gate form W (part of psi, so of <E>, but cancelling in G).
 *   - Qubit q is bit q of an amplitude index (q = 0 is the least significant bit).
 *   - All theta and result arrays are float64. Unless a name ends in _host, pointers are DEVICE
 *     pointers, read and written asynchronously on the context's CUDA stream: results are valid
 *     once that stream has reached the end of the call (qng_sync waits for it).
 *   - Batched contexts concatenate instance b's parameters at param_offset[b] (theta, grad,
 *     dtheta) and its P_b x P_b row-major metric at metric_offset[b]; energies are one per instance.
 *   - Memory: the caller owns every device buffer. The library never calls cudaMalloc: it works in
 *     a caller-provided workspace of qng_workspace_size() bytes (qng_set_workspace). The context
 *     itself holds only host copies of the descriptions passed to qng_create*.
 *   - Errors: every call returns a qng_status. Argument errors are found on the host and returned
 *     before anything is launched. Errors found on the device (a non-positive pivot in the solve)
 *     are recorded in a status word in the workspace and returned by the next qng_sync.
 *   - Thread safety: a context may be used by one host thread at a time; calls on one context
 *     are ordered by its stream. Distinct contexts are independent.
 */
#ifndef QNG_H
#define QNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qng_ctx qng_ctx;

typedef enum {
    QNG_OK = 0,
    QNG_ERR_ARG = 1,         /* invalid argument (qubit range, parameter numbering, sizes, NaN theta ...) */
    QNG_ERR_OOM = 2,         /* host allocation failed */
    QNG_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    QNG_ERR_TIMEOUT = 4,     /* a bounded device wait gave up */
    QNG_ERR_NOT_SPD = 5,     /* g + lambda I had a non-positive pivot in the Cholesky factorisation */
    QNG_ERR_WORKSPACE = 6,   /* no workspace set, or the one set is too small or misaligned */
    QNG_ERR_UNSUPPORTED = 7  /* a valid request this build does not handle (e.g. too many qubits) */
} qng_status;

/* gate kinds (qng_gate.kind) */
enum {
    QNG_GATE_RX = 0,   /* exp(-i theta X / 2) on q0                     */
    QNG_GATE_RY = 1,   /* exp(-i theta Y / 2) on q0                     */
    QNG_GATE_RZ = 2,   /* exp(-i theta Z / 2) on q0                     */
    QNG_GATE_CZ = 3,   /* controlled-Z on (q0, q1)                      */
    QNG_GATE_CNOT = 4, /* controlled-X, control q0, target q1           */
    QNG_GATE_X = 5,    /* Pauli X on q0                                 */
    QNG_GATE_Y = 6,    /* Pauli Y on q0                                 */
    QNG_GATE_Z = 7,    /* Pauli Z on q0                                 */
    QNG_GATE_H = 8     /* Hadamard on q0                                */
};

/* amplitude precisions */
enum {
    QNG_C64 = 0,  /* complex64 amplitudes; float64 accumulation of inner products, assembly and solve */
    QNG_C128 = 1  /* complex128 amplitudes, float64 arithmetic throughout                            */
};

/* One gate: param is the index of its angle in theta for RX/RY/RZ and -1 for fixed gates;
 * q1 is -1 for one-qubit gates. */
typedef struct {
    int32_t kind;
    int32_t q0;
    int32_t q1;
    int32_t param;
} qng_gate;

/* One Pauli string c * sigma: bit q of xmask / zmask set means an X / Z factor on qubit q, both
 * set means Y (sigma |k> = i^{#Y} (-1)^{popcount(k & zmask)} |k ^ xmask>), neither means identity. */
typedef struct {
    double coeff;
    uint64_t xmask;
    uint64_t zmask;
} qng_pauli;

/* Create a single-instance context. gates[0..n_gates-1] and terms[0..n_terms-1] are host arrays,
 * copied. n_qubits in 1..30; precision QNG_C64 or QNG_C128. On success *out owns the copies.
 * Instances of more than 16 qubits run on the streaming path (state vectors in HBM). */
qng_status qng_create(int n_qubits, const qng_gate *gates, int n_gates, const qng_pauli *terms, int n_terms,
                      int precision, qng_ctx **out);

/* Create a context of `count` independent instances (the batched form). Instance b has n_qubits[b]
 * qubits, the n_gates[b] gates that follow those of instances 0..b-1 in `gates`, and likewise
 * n_terms[b] terms of `terms`. Each instance is validated as in qng_create. Batched contexts take
 * instances of at most 16 qubits. */
qng_status qng_create_batch(int count, const int32_t *n_qubits, const qng_gate *gates, const int32_t *n_gates,
                            const qng_pauli *terms, const int32_t *n_terms, int precision, qng_ctx **out);

/* Sizes of a context: number of instances, sum of P_b, sum of P_b^2. Any pointer may be NULL. */
qng_status qng_get_sizes(const qng_ctx *ctx, int32_t *count, int64_t *total_params, int64_t *total_metric);

/* Host arrays of count+1 offsets: param_offset[b] = sum_{c<b} P_c, metric_offset[b] = sum_{c<b} P_c^2.
 * Either pointer may be NULL. */
qng_status qng_get_offsets(const qng_ctx *ctx, int64_t *param_offset, int64_t *metric_offset);

/* Bytes of device workspace the context needs (a multiple of 256). */
qng_status qng_workspace_size(const qng_ctx *ctx, size_t *bytes);

/* Hand the context a device workspace (256-byte aligned, >= qng_workspace_size bytes, owned by
 * the caller and kept alive while the context uses it) and the CUDA stream (cudaStream_t, may be
 * NULL for the legacy default stream) every later call is ordered on. Uploads the circuit tables
 * into the workspace with asynchronous copies on that stream. */
qng_status qng_set_workspace(qng_ctx *ctx, void *workspace, size_t bytes, void *stream);

/* Change the stream later calls are ordered on (the workspace stays). */
qng_status qng_set_stream(qng_ctx *ctx, void *stream);

/* Metric only (Algorithm 1 and Eq. g_t_L_def): g (device, sum P_b^2 float64, row-major per
 * instance) = Re G. sigma_opt (device, sum P_b, may be NULL) receives <psi_k|sigma_k|psi_k>, the
 * Pauli expectation right after rotation k, so T_k = -(i/2) sigma_opt[k]. */
qng_status qng_metric(qng_ctx *ctx, const double *theta, double *g, double *sigma_opt);

/* The whole quantum geometric tensor G = g + i g_im of Eq. 4 (Sec. 1). The same recurrence takes the
 * imaginary part of each inner product as well. T_i^* T_j is real (T_k = -(i/2) sigma_k), so
 * g_im = Im L: antisymmetric, zero diagonal. The imaginary-time coefficient matrix Re<d_i psi|d_j psi>
 * (G without its phase terms, Sec. 1) is g + sigma_i sigma_j / 4. g and g_im are device arrays in
 * qng_metric's layout; sigma_opt is as there. Both paths: the streaming path runs a second metric
 * schedule whose steps keep both parts. QNG_ERR_UNSUPPORTED when the on-chip column kernel's extra
 * shared memory (P+1 float64 per warp) does not fit. */
qng_status qng_metric_complex(qng_ctx *ctx, const double *theta, double *g, double *g_im, double *sigma_opt);

/* Energy <E> (device, one float64 per instance) and gradient d<E>/d theta (device, sum P_b). */
qng_status qng_gradient(qng_ctx *ctx, const double *theta, double *grad, double *energy);

/* Energy only. */
qng_status qng_energy(qng_ctx *ctx, const double *theta, double *energy);

/* Reverse-mode backward of <E>(theta): grad_theta = grad_out * d<E>/d theta, with grad_out a
 * DEVICE pointer to one float64 per instance (the upstream gradient). Adjoint (reverse) sweep. */
qng_status qng_energy_backward(qng_ctx *ctx, const double *theta, const double *grad_out, double *grad_theta);

/* One natural-gradient step: dtheta (device, sum P_b) solves (g + lambda I) dtheta = -dt grad<E>
 * (Eq. 3) by a float64 Cholesky factorisation: one kernel per instance when the rows fit in the
 * shared memory of a cluster (P up to about 330), else, for a single instance, one launch per
 * 16-column block with the factor in global memory (P up to about 1300), else one CTA. g_opt, grad_opt, energy_opt (device, may be NULL)
 * also receive the metric, the gradient and the energy. lambda >= 0; a non-positive pivot sets
 * QNG_ERR_NOT_SPD, reported by qng_sync. */
/* The natural-gradient descent loop (Eq. 3, Sec. 1): iters times, one qng_step at theta followed by
 * theta <- theta + dtheta, all on the context's stream. theta (device, sum P_b float64) is read and
 * updated in place; energies (device, iters * count float64, may be NULL) receives <E> of every
 * instance at the start of each iteration (row t = iteration t). A device-side error (e.g.
 * QNG_ERR_NOT_SPD) freezes theta at its last good value and is reported by qng_sync. */
qng_status qng_optimize(qng_ctx *ctx, double *theta, double dt, double lambda, int iters, double *energies);

qng_status qng_step(qng_ctx *ctx, const double *theta, double dt, double lambda, double *dtheta, double *g_opt,
                    double *grad_opt, double *energy_opt);

/* qng_step with HOST buffers: copies theta_host in, runs the step, copies the results out and
 * waits for the stream. Pageable or pinned host memory; g_host, grad_host, energy_host may be NULL. */
qng_status qng_step_host(qng_ctx *ctx, const double *theta_host, double dt, double lambda, double *dtheta_host,
                         double *g_host, double *grad_host, double *energy_host);

/* Capture one qng_step with these arguments (device pointers that must stay valid) into a CUDA
 * graph owned by the context, on the context's stream (which must not be the legacy default
 * stream). qng_graph_launch replays it on that stream. A new capture replaces the old one; the
 * graph is freed by qng_destroy. Re-capture after qng_set_workspace, qng_set_path or tuning. */
qng_status qng_graph_capture(qng_ctx *ctx, const double *theta, double dt, double lambda, double *dtheta,
                             double *g_opt, double *grad_opt, double *energy_opt);
qng_status qng_graph_launch(qng_ctx *ctx);

/* Autotuner of the on-chip path: for every qubit count present in the context, times qng_step
 * (reps repetitions after one warm-up, CUDA events) for every cluster size (1..8 CTAs) and CTA size
 * (64, 128, 256 threads) that fits, and keeps the fastest; theta is a device array of the context's
 * parameters. report (may be NULL) receives the number of shapes timed. Shapes needing more
 * workspace than the one set are skipped. Drops a captured graph. */
qng_status qng_autotune(qng_ctx *ctx, const double *theta, int reps, int64_t *report);

/* Launch shape used for instances of n_qubits qubits (after defaults, autotuning and qng_set_shape):
 * cluster_log2 = log2 of CTAs per state, threads = CTA size of the column kernel (64..256),
 * forward_threads = CTA size of the checkpoint sweep (64..512); any output pointer may be NULL.
 * qng_set_shape is the manual override (cluster_log2 -1, threads 0 and forward_threads 0 restore
 * the defaults); QNG_ERR_ARG for values out of range, QNG_ERR_WORKSPACE (old shape kept) when the
 * new shape needs more workspace than the one set. */
qng_status qng_get_tuning(const qng_ctx *ctx, int n_qubits, int *cluster_log2, int *threads, int *forward_threads);
qng_status qng_set_shape(qng_ctx *ctx, int n_qubits, int cluster_log2, int threads, int forward_threads);

/* Wait for the context's stream, then return (and clear) the device-side status word. */
qng_status qng_sync(qng_ctx *ctx);

/* Launch-shape controls (used by the autotuner; 0 leaves a value on automatic):
 * cluster_log2 = log2 of CTAs per state (0..3), threads = CTA size (64..256, a multiple of 32).
 * For batched contexts the settings apply to the instances with n_qubits >= min_qubits. */
qng_status qng_set_tuning(qng_ctx *ctx, int min_qubits, int cluster_log2, int threads);

/* Execution path: 0 automatic (on-chip for n <= 16 qubits, streaming above), 1 on-chip (every
 * state of an instance in the shared memory of one thread-block cluster, O(P) checkpoints in HBM),
 * 2 streaming (single instance only: O(1) registers of 2^n amplitudes in HBM, tiled passes). A
 * change re-plans the context; if the workspace already set is then too small the call returns
 * QNG_ERR_WORKSPACE and keeps the old path (query qng_workspace_size before setting a workspace). */
qng_status qng_set_path(qng_ctx *ctx, int path);

/* Streaming path only: HBM bytes one qng_step moves through the pass schedule (registers loaded
 * and stored by every pass), split into the metric columns and the rest (forward, energy, adjoint),
 * and the number of inner-product steps (elements) of the metric. Zeros on the on-chip path. */
qng_status qng_stream_traffic(const qng_ctx *ctx, int64_t *metric_bytes, int64_t *other_bytes, int64_t *metric_passes);

/* Kernel timing with CUDA events recorded on the context's stream around every launch.
 * qng_profile(ctx, 1) starts recording, qng_profile(ctx, 0) stops. qng_profile_read waits for the
 * stream, then returns per kernel class (0 coefficients, 1 checkpoints/forward, 2 recurrence
 * columns, 3 assembly and solve) the summed milliseconds and the launch counts since the last read. */
#define QNG_KERNEL_CLASSES 4
qng_status qng_profile(qng_ctx *ctx, int enable);
qng_status qng_profile_read(qng_ctx *ctx, double *ms, int64_t *launches);

/* Number of kernel launches the last compute call issued (for accounting). */
qng_status qng_last_launch_count(const qng_ctx *ctx, int64_t *launches);

/* Metric without any allocation, for callers that cannot allocate device memory: programs whose
 * GPU memory is owned by a host application's own pool (plugins, embedded solvers) or that must
 * not pay cudaMalloc's implicit synchronisation, and callers that cannot keep a workspace alive
 * between calls. The paper has no counterpart; this is a packaging of qng_metric.
 *   Inputs and outputs are as in qng_metric for ONE instance (n_qubits <= 16, at most 1024 gates
 *   and 320 parameters): theta (device, P float64), g (device, P*P float64), stream (cudaStream_t
 *   or NULL). Every other buffer lives in one static device array of QNG_NOALLOC_SCRATCH_BYTES
 *   bytes that each GPU loading the library holds until the process exits.
 *   Returns QNG_ERR_WORKSPACE when the instance needs more than that array (for example 12 qubits
 *   at complex128 fit with P <= 240), QNG_ERR_ARG for an invalid circuit, QNG_ERR_CUDA for a
 *   failed CUDA call. Device-side conditions (a non-finite theta) are not reported.
 *   All calls on a device share the array, which keeps the last call's contents: calls whose work
 *   overlaps on the GPU race and must be ordered by the caller. The first call on each device
 *   looks up the array's address (with that device current); make it before any stream capture.
 *   No cudaMalloc, cudaFree or other allocating routine is called. */
#define QNG_NOALLOC_SCRATCH_BYTES (16u << 20)
qng_status qng_metric_noalloc(int n_qubits, const qng_gate *gates, int n_gates, int precision, const double *theta,
                              double *g, void *stream);

void qng_destroy(qng_ctx *ctx);

const char *qng_status_string(qng_status s);

#ifdef __cplusplus
}
#endif

#endif /* QNG_H */
