/*
 * sv_gb300.h -- C ABI of the GB300 fused-gate state-vector library (libsvgb300.so).
 *
 * The library applies a stream of fused k-qubit gates (k = 1..6) to a 2^n complex64 state vector
 * on one GPU (paper section II-A, Eq. 3: every group of 2^k amplitudes whose indices differ only
 * in the target bits is multiplied by the 2^k x 2^k gate matrix).  Gates are fused on the host
 * (section IV-D: vertical fusion = matrix product, horizontal fusion = tensor product, Eq. 4).
 *
 * Conventions used by every call:
 *   - amplitude index bit q <-> qubit q (qubit 0 is the least-significant bit);
 *   - a gate matrix is 2^k x 2^k, row-major, complex128 interleaved (re, im), and local index
 *     bit j <-> targets[j];
 *   - a control qubit means "apply only where that bit is 1" (the sentence after Eq. 3);
 *   - every call returns SV_OK (0) or a negative SV_E* code; sv_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread);
 *   - pointers passed in are borrowed for the duration of the call only (except the state
 *     buffer handed to sv_alloc, which must outlive the sv_state); the library never frees
 *     caller memory;
 *   - device work is enqueued on the stream given to sv_alloc; calls returning results to the
 *     host (sv_norm, sv_sample, sv_store to host) synchronise that stream before returning.
 *
 * Device layout of the state (section IV-A's in-place layout adjustment, re-designed for
 * 128-byte GPU transactions): amplitudes are stored in blocks of 32; block b holds the 32 real
 * parts of amplitudes 32b..32b+31 followed by their 32 imaginary parts (256 bytes per block).
 * sv_load / sv_store convert from / to the standard interleaved complex64 order.
 */
#ifndef SV_GB300_H
#define SV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SV_API __attribute__((visibility("default")))
#else
#define SV_API
#endif

#define SV_MAX_QUBITS 35
#define SV_MAX_K 6
#define SV_MAX_CONTROLS 33

enum sv_status {
    SV_OK = 0,
    SV_EINVAL = -1,     /* bad argument (qubit index, k, null pointer, size) */
    SV_ENOMEM = -2,     /* device or host memory too small / allocation failed */
    SV_ECUDA = -3,      /* a CUDA runtime call failed (message has the CUDA error string) */
    SV_ETIMEOUT = -4,   /* a bounded device-side wait gave up (persistent batch kernel) */
    SV_EUNITARY = -5,   /* a gate matrix is not unitary within 1e-8 (checked by sv_fuse_circuit) */
    SV_ESTATE = -6      /* object used in the wrong state (e.g. fused circuit for another n) */
};

/* Kernel path of one fused gate.  LOW: every target < 5 (inside one 32-amplitude block);
 * HIGH: every target >= 5; MIXED: both.  TC_*: tensor-core contraction (fused gates of 4-6 qubits). */
enum sv_path {
    SV_PATH_AUTO = 0,
    SV_PATH_LOW = 1,
    SV_PATH_HIGH = 2,
    SV_PATH_MIXED = 3,
    SV_PATH_TC_TF32 = 4,
    SV_PATH_TC_BF16X3 = 5,
    SV_PATH_CONTROLLED = 6,  /* a gate kept with its controls: only amplitudes whose control bits
                                are all 1 are read and written (Section IV, ApplyControlledGate) */
    SV_PATH_SWAPS = 7,       /* a swap network (SV_FUSE_PHASES): disjoint qubit swaps applied in one
                                in-place pass; k = 0 and no matrix (sv_fused_get_swaps) */
    SV_PATH_POST_PHASES = 256 /* not a path: a flag or-ed into the tensor-core path passed to a
                                 caller's cost function (sv_fuse_opts.cost_us) for a gate that
                                 carries post-phases (SV_FUSE_PHASES) */
};

enum sv_precision {
    SV_PREC_FP32 = 0,     /* CUDA-core fp32 for every k */
    SV_PREC_TF32 = 1,     /* fused gates with k >= tc_min_k on tensor cores, tf32 inputs */
    SV_PREC_BF16X3 = 2    /* same, 3-term bf16 split products (hi*hi + hi*lo + lo*hi) */
};

enum sv_fuse_mode {
    SV_FUSE_GREEDY = 0,   /* greedy fusion up to max_k qubits */
    SV_FUSE_LEARNED = 1,  /* partition chosen by a cost model (the learned sv_mlp, or a caller's cost
                             function): candidates are greedy partitions at every max size 2..max_k
                             under three rules for which blocks a gate closes, each improved by
                             cost-guided merging (two blocks merge when their union has <= max_k
                             qubits, one commutes past the blocks between them, and the merged gate
                             is predicted 2% faster than the two); with tensor-core precision,
                             max_k 6, no start_qubits and a circuit holding diagonal two-qubit
                             gates, the SV_FUSE_PHASES partition is a candidate too (its gates with
                             post-phases scored as such); the candidate with the least predicted
                             time wins, each fused gate on its cheapest predicted path */
    SV_FUSE_NONE = 2,     /* no fusion: every input gate becomes its own dense gate (timing, baselines) */
    SV_FUSE_PHASES = 3    /* greedy fusion into gates of up to max_k = 6 qubits (one open gate at a
                             time) for the tensor cores (precision TF32 or BF16X3), where a diagonal
                             gate with one qubit in a full fused gate and one outside it does not
                             end the gate: its phase on the two qubits' common 1s is applied to the
                             fused gate's outputs in the same pass (a post-phase; the linear parts
                             go into the matrix or wait for the outside qubit's next gate).  A
                             controlled-phase ladder (a QFT) then costs one pass per six qubits.
                             Gates that cannot carry post-phases (fewer than six qubits, or three or
                             more targets below qubit 5) get them as diagonal fused gates after
                             them.  On states of 10 or more qubits, three or more consecutive SWAP
                             gates on disjoint qubits become one swap network (SV_PATH_SWAPS: one
                             in-place permutation pass).  Not with start_qubits. */
};

typedef struct sv_state sv_state;   /* opaque; owns no state memory, only small workspaces */
typedef struct sv_fused sv_fused;   /* opaque fused circuit (host matrices + lazily made device copies) */
typedef struct sv_mlp sv_mlp;       /* opaque learned cost model */


/* One input gate.  mat: 2^k x 2^k complex128 row-major interleaved (re, im), local bit j <->
 * targets[j]; the gate acts only where every control qubit is 1.  The fuser folds the controls
 * into a dense (k + n_controls)-qubit matrix when k + n_controls <= the fusion size (max_k; 6 in
 * SV_FUSE_NONE mode), so the gate can fuse with its neighbours.  Otherwise, for k <= 3, it keeps
 * the gate controlled (SV_PATH_CONTROLLED: one pass over the 2^(n - n_controls) amplitudes whose
 * control bits are 1; a fusion barrier for every qubit it names); a larger k is folded if
 * k + n_controls <= 6 and rejected (SV_EINVAL) if not. */
typedef struct sv_gate {
    int k;
    int targets[SV_MAX_K];
    int n_controls;
    int controls[SV_MAX_CONTROLS];
    const double *mat;
} sv_gate;

typedef struct sv_fuse_opts {
    int max_k;          /* largest fused gate, 1..6 (greedy mode); 0 = 4 */
    int mode;           /* enum sv_fuse_mode */
    int precision;      /* enum sv_precision */
    int tc_min_k;       /* smallest k sent to tensor cores when precision != FP32; 0 = 5 */
    int force_path;     /* enum sv_path; SV_PATH_AUTO lets the library choose (testing knob) */
    const sv_mlp *model;/* learned mode: trained cost model; NULL, untrained or a validation error
                           above 25% => greedy fusion at max_k (model's fallback k when present) */
    int start_qubits;   /* 0 (default): fuse the circuit as one.  m in 1..28: the circuit will start
                           from a basis state through sv_init_apply, so the gates of its light cone
                           on m qubits (min(m, n - 1)) are fused apart and placed first: in circuit
                           order, a qubit set S grows with each gate's qubits (targets and controls)
                           while it has at most m; a gate joins the first part when no earlier gate
                           left out shares a qubit with it and its qubits lie in S.  sv_init_apply
                           then runs that part on its small state; applied with
                           sv_apply_fused_gates the result is the same state, but may take more
                           passes than fusing without the split.  Greedy and learned modes; the
                           learned mode also scores light cones of m - 1 .. m - 4 qubits (their gates
                           costed on the smaller start state) and keeps the cheapest. */
    /* Learned mode with a caller's cost model instead of `model` (used when non-NULL): predicted
     * microseconds of one fused gate of k qubits (targets ascending) run on kernel path `path` in an
     * n-qubit state.  Called on the calling thread during sv_fuse_circuit, once per candidate fused
     * gate and path (a gate that carries post-phases: path = its tensor-core path |
     * SV_PATH_POST_PHASES); it must not call back into the library.  A negative or non-finite result makes
     * sv_fuse_circuit fail with SV_EINVAL.  cost_ctx is passed through. */
    double (*cost_us)(int k, const int *targets, int path, int n_qubits, void *cost_ctx);
    void *cost_ctx;
} sv_fuse_opts;

/* Post-phases of fused gate i (SV_FUSE_PHASES): after the gate's matrix, an amplitude whose bits
 * targets[target[t]] and qubit[t] are both 1 is multiplied by exp(i angle[t]), for every term t.
 * Writes up to max_terms terms (any output may be NULL) and returns the number of terms, or a
 * negative SV_E* code. */
SV_API int sv_fused_get_post_phases(const sv_fused *f, int i, int max_terms, int *target, int *qubit, double *angle);

/* Swap network of fused gate i (path SV_PATH_SWAPS): the qubit pairs (qubit_a[t], qubit_b[t]) whose
 * amplitudes it exchanges, all disjoint.  Writes up to max_pairs pairs (outputs may be NULL) and
 * returns the number of pairs (0 for any other gate), or a negative SV_E* code. */
SV_API int sv_fused_get_swaps(const sv_fused *f, int i, int max_pairs, int *qubit_a, int *qubit_b);

/* Facts about one fused gate (introspection). */
typedef struct sv_fused_info {
    int k;
    int targets[SV_MAX_K];   /* ascending; the fused matrix uses local bit j <-> targets[j] */
    int path;                /* enum sv_path chosen for it */
    int n_source_gates;      /* how many input gates it absorbed */
    uint64_t control_mask;   /* SV_PATH_CONTROLLED: bit q set <-> qubit q is a control; else 0 */
} sv_fused_info;

/* One timing record, written by sv_apply_fused_gates when asked (CUDA events around each launch). */
typedef struct sv_timing {
    float us;                /* device time of this fused gate's kernel, microseconds */
    int k;
    int path;                /* the kernel path; SV_PATH_AUTO for a gate sv_init_apply ran on its small state */
    int flags;               /* SV_TIMING_* bits */
    uint64_t target_mask;    /* bit q set <-> qubit q is a target */
} sv_timing;

/* sv_timing.flags: the gate read its inputs from sv_init_apply's small start state (the first
 * full-state gate after a lazy start, when it runs on a direct tensor-core kernel): it wrote the
 * whole state but read only the small state's 2^a amplitudes, so its time is not that of a full
 * pass and is no sample of the kernel's usual cost. */
#define SV_TIMING_SMALL_SOURCE 1

/* ---------------------------------------------------------------------------------------------
 * State
 * ------------------------------------------------------------------------------------------- */

/* Bytes a state buffer of n qubits needs: max(8 * 2^n, 256) (8 bytes per complex64 amplitude;
 * the artifact appendix states 2^(n+3) bytes for an n-qubit run). */
SV_API size_t sv_required_bytes(int n_qubits);

/* Wrap a caller-owned device buffer of `bytes` bytes (>= sv_required_bytes(n), 256-byte aligned)
 * as an n-qubit state; 1 <= n <= SV_MAX_QUBITS.  `cuda_stream` is a cudaStream_t (NULL = legacy
 * default stream) on which every later call enqueues work.  Allocates a small reduction workspace
 * on the current device.  The buffer's contents are undefined until sv_init / sv_load. */
SV_API int sv_alloc(int n_qubits, void *dev_ptr, size_t bytes, void *cuda_stream, sv_state **out);

/* Release the handle and its workspace (not the caller's buffer).  Synchronises the stream. */
SV_API void sv_free(sv_state *st);

/* Set the state to the basis state |basis_index> (basis_index < 2^n), in the blocked layout. */
SV_API int sv_init(sv_state *st, uint64_t basis_index);

/* Import 2^n complex64 amplitudes in standard interleaved order from `src` (host memory when
 * src_on_host != 0, else device memory not overlapping the state) and convert to the blocked
 * layout in place. */
SV_API int sv_load(sv_state *st, const void *src, int src_on_host);

/* Export the state as 2^n complex64 interleaved amplitudes to `dst` (host when dst_on_host != 0,
 * else a device buffer of 8 * 2^n bytes not overlapping the state).  For a host destination the
 * state is converted in place, copied, and converted back; the stream is synchronised. */
SV_API int sv_store(const sv_state *st, void *dst, int dst_on_host);

/* ---------------------------------------------------------------------------------------------
 * Fusion (host) and application (device)
 * ------------------------------------------------------------------------------------------- */

/* Fuse `n_gates` gates of an n-qubit circuit into a sequence of dense fused gates of at most
 * opts->max_k qubits (section IV-D).  Products are formed in fp64; each fused matrix is rounded
 * to fp32 once.  Every input matrix is checked for unitarity (SV_EUNITARY).  Host only: no device
 * memory is touched here.  opts may be NULL (greedy, max_k = 4, fp32). */
SV_API int sv_fuse_circuit(const sv_gate *gates, int n_gates, int n_qubits, const sv_fuse_opts *opts,
                    sv_fused **out);

/* Frees a fused circuit.  If its device images exist, waits first for the last launch of every
 * stream that applied it (sv_apply_fused_gates / sv_init_apply on a state's stream); work on other
 * streams is not waited for. */
SV_API void sv_fused_free(sv_fused *f);

SV_API int sv_fused_count(const sv_fused *f);
SV_API int sv_fused_get_info(const sv_fused *f, int i, sv_fused_info *info);
/* Copy fused gate i's fp64 matrix (2^k x 2^k complex, interleaved, row-major) into `out`. */
SV_API int sv_fused_get_matrix(const sv_fused *f, int i, double *out);

/* Apply every fused gate, in order, to the state (Eq. 3 per fused gate).  The first call with a
 * given fused circuit uploads the matrices that do not travel as kernel arguments (k = 6 and the
 * tensor-core operands) with cudaMalloc/cudaMemcpy.  With `timings` non-NULL (one record per
 * fused gate) each launch is bracketed by CUDA events and the call synchronises. */
SV_API int sv_apply_fused_gates(sv_state *st, const sv_fused *f, sv_timing *timings);

/* ---------------------------------------------------------------------------------------------
 * Learned fusion cost model (no counterpart in the paper's code: the paper tunes its fusion size
 * per machine with a synthetic benchmark, section VI-C; here the simulator learns a cost model
 * from timings of its own kernels).  A 16 -> 64 -> 64 -> 64 -> 1 fp32 MLP with ReLU predicts
 * y = ln(t / 1 us) - n ln 2 (standardised), the log device time per amplitude of one fused gate.
 * Forward, backward and Adam run as CUDA kernels on the device current at creation, on the given
 * stream.  sv_fuse_circuit in SV_FUSE_LEARNED mode uses it to choose the fusion partition, the
 * largest fused size and each fused gate's kernel path.
 * ------------------------------------------------------------------------------------------- */

typedef struct sv_mlp_train_opts {
    int epochs;         /* passes over the training rows */
    int batch;          /* rows per Adam step, 1..1024 */
    float lr;           /* Adam learning rate (beta1 0.9, beta2 0.999, eps 1e-8) */
    uint64_t seed;      /* shuffling and the train / validation split */
    float val_frac;     /* fraction held out to measure the prediction error, [0, 0.9) */
    int fallback_k;     /* greedy max size used when the model is not trusted */
} sv_mlp_train_opts;

typedef struct sv_mlp_stats {
    float train_loss;   /* mean squared error (standardised) over the last epoch */
    float val_mape;     /* mean |predicted - measured| / measured time on the held-out rows */
    long long n_train, n_val, steps;
    int trained;
    float y_mean, y_std;
    int fallback_k;
} sv_mlp_stats;

/* Number of parameters (9473).  Flat order: W1 (64x16 row-major), b1, W2 (64x64), b2, W3, b3,
 * W4 (1x64), b4. */
SV_API int sv_mlp_num_params(void);
/* New model with He-normal weights drawn from `seed` (SplitMix64 + Box-Muller), zero biases. */
SV_API int sv_mlp_create(uint64_t seed, void *cuda_stream, sv_mlp **out);
SV_API void sv_mlp_free(sv_mlp *m);
SV_API int sv_mlp_get_params(const sv_mlp *m, float *out);     /* host buffer of sv_mlp_num_params() */
SV_API int sv_mlp_set_params(sv_mlp *m, const float *in);
/* Feature vector (16 floats) of a fused gate with k targets (any order), kernel path (enum sv_path)
 * and n qubits, carrying post-phases (SV_FUSE_PHASES) or not (post_phases 1 or 0):
 * [k/6, sorted targets / n (6, padded with -1), one-hot path LOW..TC_BF16X3 (5), n/34,
 * (#targets < 5)/5, max target / n, post_phases]. */
SV_API int sv_mlp_features(int k, const int *targets, int path, int n_qubits, int post_phases, float *out);
/* Loss and gradient of the mean squared error for B rows (X: B x 16, t: B standardised targets,
 * both host), at the current parameters; grads: host buffer of sv_mlp_num_params().  B <= 1024. */
SV_API int sv_mlp_gradients(sv_mlp *m, const float *X, const float *t, int B, float *loss, float *grads);
/* One Adam update with the gradient left by the last sv_mlp_gradients call. */
SV_API int sv_mlp_adam_step(sv_mlp *m, float lr);
/* Train on N rows of features X (N x 16, host) and measured times us (N, microseconds, host).
 * opts may be NULL (200 epochs, batch 256, lr 1e-3, seed 1, 10% validation, fallback k 4). */
SV_API int sv_mlp_train(sv_mlp *m, const float *X, const float *us, long long N, const sv_mlp_train_opts *opts,
                        sv_mlp_stats *stats);
/* Predicted microseconds for `rows` feature rows (host in, host out).  Needs a trained model. */
SV_API int sv_mlp_predict(sv_mlp *m, const float *X, int rows, double *out_us);
SV_API int sv_mlp_get_stats(const sv_mlp *m, sv_mlp_stats *stats);
/* Binary file: 8-byte magic, parameter count, trained flag, fallback k, y mean, y deviation,
 * validation error, parameters (little-endian fp32). */
SV_API int sv_mlp_save(const sv_mlp *m, const char *path);
SV_API int sv_mlp_load(const char *path, void *cuda_stream, sv_mlp **out);

/* ---------------------------------------------------------------------------------------------
 * Reductions
 * ------------------------------------------------------------------------------------------- */

/* *out = sum_i |c_i|^2, accumulated in fp64 (normalisation condition under Eq. 1).  Synchronises. */
SV_API int sv_norm(const sv_state *st, double *out);

/* For each of the n_samples uniforms u (host array, values in [0, 1)), out[s] (host array) =
 * the smallest index i with |c_0|^2 + ... + |c_i|^2 > u_s * sum_j |c_j|^2 (fp64 prefix sums;
 * Eq. 1: |c_i|^2 is the probability of observing basis state i).  Grows a workspace on the
 * state's device when n_samples exceeds the previous maximum.  Synchronises. */
SV_API int sv_sample(const sv_state *st, const double *uniforms, int n_samples, uint64_t *out);
/* sv_sample and sv_norm from one read pass: the sampling's fp64 prefix sums end in the total
 * probability, which is returned in *norm_out (the same fp64 sum as sv_norm up to summation order).
 * n_samples may be 0 (norm only).  Synchronises. */
SV_API int sv_sample_norm(const sv_state *st, const double *uniforms, int n_samples, uint64_t *out, double *norm_out);

/* ---------------------------------------------------------------------------------------------
 * Complex128 states (no counterpart in the paper's single-precision runs).  The same operations
 * in fp64: amplitudes are complex128 (16 bytes), stored in 512-byte blocks of 32 real then 32
 * imaginary parts, and fused gates are applied with their fp64 matrices in fp64 arithmetic, so the
 * result matches the complex128 definition up to summation order.  fp64 arithmetic bounds these
 * kernels (about 1.2 TFLOP/s of fp64 FMA on GB300, 1/58 of fp32); small fusion sizes (2-3) are
 * the cheapest.  On a complex128 state sv_init, sv_load / sv_store (interleaved complex128),
 * sv_apply_fused_gates (every path, including kept controls, runs the fp64 kernel; the tensor-core
 * and precision options are ignored), sv_norm and sv_sample work as documented above;
 * sv_expval_pauli returns SV_EINVAL.
 * ------------------------------------------------------------------------------------------- */
/* Bytes of a complex128 n-qubit state: 16 * 2^n (at least one 512-byte block); 0 if n is out of range. */
SV_API size_t sv_required_bytes_c128(int n_qubits);
/* Like sv_alloc for a complex128 state: bytes >= sv_required_bytes_c128(n_qubits), 256-byte aligned. */
SV_API int sv_alloc_c128(int n_qubits, void *dev_ptr, size_t bytes, void *cuda_stream, sv_state **out);

/* Expectation values of Pauli strings (Section IV: the ExpectationValue routine runs the
 * ApplyGate group loop and reduces instead of storing).  String p is
 *     P_p = tensor product over qubits q of sigma_q,
 *     sigma_q = X if bit q is set in x_masks[p] only, Z if in z_masks[p] only, Y if in both, else I,
 * and out[p] (host array of count doubles) = <psi|P_p|psi>, real because P_p is Hermitian; the
 * state is not normalised first (divide by sv_norm for a state that is not unit-norm).  Each
 * amplitude's term is formed in fp32 and accumulated in float-float per thread, fp64 across
 * threads, in a fixed order (deterministic).  Strings sharing an x mask share read passes, up to 8
 * strings per pass over the 8 * 2^n bytes.  SV_EINVAL if a mask has a bit >= n.  Grows a small
 * workspace on the state's device when count exceeds the previous maximum.  Synchronises. */
SV_API int sv_expval_pauli(const sv_state *st, const uint64_t *x_masks, const uint64_t *z_masks, int count, double *out);

/* ---------------------------------------------------------------------------------------------
 * Batched circuits (no counterpart in the paper's code, which runs one circuit at a time): many
 * independent circuits of uneven size, each already fused (k <= 4, n <= 24), run from |0...0> in
 * ONE persistent kernel launch.  CTAs take work items from a device queue in an order the host
 * fixes: circuits of at most smem_max_n qubits are simulated whole in one CTA's shared memory and
 * stored once; circuits of at least split_min_n qubits are cut into tiles of 2^tile_log2 groups
 * per fused gate that any CTA may take (a tile waits, bounded, for the previous gate's tiles of
 * its circuit); the rest run whole in one CTA on their global buffer.  If a wait gives up, the
 * launch ends early and sv_device_status reports SV_ETIMEOUT.  The launch is captured once in a
 * CUDA graph (per option set) and replayed.
 * ------------------------------------------------------------------------------------------- */
typedef struct sv_batch sv_batch;

typedef struct sv_batch_opts {
    int threads;        /* threads per CTA, multiple of 32 in [32, 512] (default 256) */
    int smem_max_n;     /* largest circuit kept in shared memory, 0..14 (default 12) */
    int ctas;           /* persistent CTAs (default 2 x SM count) */
    int use_graph;      /* nonzero: capture once, replay (default 1) */
    int split_min_n;    /* circuits of at least this many qubits are split into tiles of each
                           step that all CTAs share; 0 = never (default 15) */
    int tile_log2;      /* groups per tile of a split circuit's step: 2^tile_log2, 5..16 (default 12) */
    int wave_mb;        /* split circuits run in waves of at most this many MB of state, one wave
                           after another, so a wave's states stay in L2; 0 = one wave (default 0) */
    int stage_log2;     /* 0 (default): a split circuit runs one fused gate per step over global
                           memory.  8..14: a split circuit of at least 8 qubits runs in stages
                           instead; a stage is a run of gates (a gate moves ahead only past gates on
                           other qubits) whose qubits lie in one set of stage_log2 qubits that
                           includes qubits 0-2, and each of its 2^(n - stage_log2) tiles (the
                           amplitudes that agree on the other qubits) is loaded into shared memory
                           once, gets every gate of the stage there and is stored once */
    int stage_k;        /* staged circuits: each stage's gates are fused again (greedy, fp64
                           products) into gates of at most stage_k qubits, 1..4; 0 = kept as given
                           (default 0) */
    int stage_layers;   /* staged circuits with tiles of 10 or more qubits: nonzero = a run of
                           one-qubit gates in a stage (between two gates on more qubits) is one
                           layer -- each qubit's 2x2 product -- and the layers and the +-1 sign
                           runs between them are applied in register phases: windows of five
                           local qubits held in registers, one shared-memory round trip per
                           phase, instead of stage_k-qubit gates (default 0) */
    int ctas_per_sm;    /* 0 or 1 (default 1): one CTA per SM; 2: two CTAs share each SM (CTAs of at most 256 threads,
                           128 registers a thread), so that one CTA's memory traffic, waits and
                           barriers overlap the other's arithmetic; SV_EINVAL unless two CTAs'
                           shared memory (matrix area, descriptors and the larger of the
                           smem_max_n state and the stage tile) fits on one SM */
} sv_batch_opts;

/* Bytes of the state arena for these circuit sizes: each state in the blocked layout, 256-byte
 * aligned, in the given order.  0 if a size is outside 1..24. */
SV_API size_t sv_batch_arena_bytes(const int *n_qubits, int count);
/* Describe a batch over `circuits` (borrowed: they must outlive the batch) with states in the
 * caller's device `arena` (>= sv_batch_arena_bytes, 256-byte aligned).  Uploads the fused
 * matrices (cudaMalloc); work is enqueued on `cuda_stream`. */
SV_API int sv_batch_create(const sv_fused *const *circuits, int count, void *arena, size_t arena_bytes, void *cuda_stream,
                           sv_batch **out);
SV_API void sv_batch_free(sv_batch *b);
/* Options take effect at the next sv_batch_run (which rebuilds the work list, synchronously, when
 * smem_max_n, split_min_n, tile_log2, wave_mb, stage_log2, stage_k or stage_layers changed).  SV_EINVAL for a
 * value out of range. */
SV_API int sv_batch_set_opts(sv_batch *b, const sv_batch_opts *opts);
SV_API int sv_batch_get_opts(const sv_batch *b, sv_batch_opts *opts);
/* Run every circuit from |0...0> into its state buffer: one persistent launch (asynchronous). */
SV_API int sv_batch_run(sv_batch *b);
/* The same work as one launch per fused gate, circuit after circuit (comparison baseline). */
SV_API int sv_batch_run_loop(sv_batch *b);
/* What the work list for the current options holds (built here if sv_batch_run has not built it
 * yet, which needs the device).  traffic_bytes: the bytes the list moves to and from the state
 * buffers in global memory if nothing stays in cache -- per whole circuit in shared memory one
 * store of its state; per circuit run gate by gate (one CTA, or split into tiles) a write of the
 * initial state and a read and a write per fused gate; per staged circuit a read and a write per
 * stage, less the first stage's read. */
typedef struct sv_batch_info {
    int items;              /* work items */
    int whole;              /* circuits held in shared memory */
    int single;             /* circuits run by one CTA in global memory */
    int split;              /* circuits split into tiles of each fused gate */
    int staged;             /* circuits run in stages */
    int stages;             /* stages of all staged circuits */
    int stage_gates;        /* gates of all stages (after stage_k re-fusion) */
    double traffic_bytes;
} sv_batch_info;
SV_API int sv_batch_get_info(sv_batch *b, sv_batch_info *out);
/* Byte offset of circuit i's state inside the arena. */
SV_API int sv_batch_state_offset(const sv_batch *b, int i, size_t *offset_bytes);
/* The stages a batch cuts fused circuit f into at tiles of stage_log2 qubits (8..14; a circuit of
 * fewer qubits uses all of them) -- host only, no GPU.  The circuit's n must be 8..24 and its gates
 * uncontrolled.  Returns the number of stages S (or a negative SV_E* code) and writes, for the
 * first min(S, max_stages) stages s:
 *   gates[s]              the number of fused gates the stage applies;
 *   lam[s]                its local qubits (bit q: circuit qubit q), 2^popcount amplitudes a tile;
 *   load_pos[32 s + q]    the bit of a global index where qubit q sits when the stage loads its
 *                         tiles (the layout the previous stage stored in; for the first stage, the
 *                         layout it stores in);
 *   store_pos[32 s + q]   and where it sits when the stage stores them (the last stage: q itself),
 * and order[0 .. count(f)) = the fused gates' indices in the order the stages apply them (a
 * reordering that moves gates only past gates on other qubits).  Any output may be NULL. */
SV_API int sv_batch_plan_stages(const sv_fused *f, int stage_log2, int max_stages, int *gates, unsigned *lam, int *load_pos,
                                int *store_pos, int *order);
/* Test hook for the bounded waits.  on != 0: from the next sv_batch_run the first split circuit's
 * initialisation step (its first stage, when staged) counts one tile more than exists, so the
 * tiles of the next step wait on a counter that never fills; each gives up after about a second,
 * the launch ends early without a fault, the states are left incomplete and sv_device_status
 * returns SV_ETIMEOUT.  on = 0 undoes it.  No effect when no circuit is split, or when the first
 * split circuit is staged in a single stage. */
SV_API int sv_batch_inject_stall(sv_batch *b, int on);

/* sv_init(st, basis_index) then sv_apply_fused_gates(st, f, timings), with the same result up to
 * rounding order, computed with less memory traffic.  One pass over the fused gates picks those
 * that share no qubit with an earlier gate left out (so they commute past it) while the qubits they
 * name, targets and controls, number at most L and fewer than n (L: the qubits the light-cone part
 * names when f was fused with start_qubits, else 26); every other qubit still holds its
 * bit of basis_index, so the picked gates run first, in order, on the small state of the named
 * qubits (in a library-owned buffer of up to 2 GiB grown on first use; tensor-core gates stay on
 * the tensor cores when the small state has at least k + 5 qubits, the others run on CUDA cores), which
 * one kernel then writes into the zeroed full state; the rest run, in order, as in
 * sv_apply_fused_gates.  Timing records stay in circuit order.  Complex128 states take the plain
 * route.  Asynchronous unless timings are requested. */
SV_API int sv_init_apply(sv_state *st, uint64_t basis_index, const sv_fused *f, sv_timing *timings);

/* SV_OK if no kernel on the current device has given up a bounded wait since the last call, else
 * SV_ETIMEOUT (the error is cleared by the call).  Synchronises the device. */
SV_API int sv_device_status(void);

/* Sampling for callers that cannot allocate device memory.  No counterpart in the paper.
 *
 * Same result as sv_sample, bit for bit, but it needs no sv_state and calls no cudaMalloc,
 * cudaFree or allocating library routine: every intermediate lives in one fixed array compiled
 * into the library (about 1.1 MB per GPU, held until process exit).  The array is placed on a GPU
 * when the library's module is loaded there; CUDA loads modules lazily by default, i.e. at the
 * first launch of one of the library's kernels on that GPU (at the latest, the first call of this
 * function), so a caller that lets its own pool claim the GPU afterwards should make one warm-up
 * call (any size) first.  This is
 * for callers that own all device memory up front and must not let a library grow it (a serving
 * process whose pool already claims the GPU, where cudaMalloc would fail or fragment), and for
 * callers that cannot afford the device-wide synchronisation cudaMalloc/cudaFree may cause.
 *
 * dev_state: the blocked-layout state of an n-qubit register (as sv_alloc would wrap), read only.
 * n_qubits <= 30 and n_samples <= 4096 (the fixed array's limits; larger requests return
 * SV_EINVAL with a message).  uniforms / out: host arrays as in sv_sample.  Work is enqueued on
 * cuda_stream on the current device, and the call synchronises that stream before returning.
 * The first call on a device looks up the array's device address with that device current; make
 * that first call before capturing work on the device into a graph.  Every call on a device uses
 * the same array, and calls whose GPU work overlaps race on it: serialise them. */
SV_API int sv_sample_noalloc(const void *dev_state, int n_qubits, void *cuda_stream, const double *uniforms,
                             int n_samples, uint64_t *out);

SV_API const char *sv_last_error(void);
SV_API const char *sv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SV_GB300_H */
