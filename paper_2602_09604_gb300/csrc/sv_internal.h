// Internal declarations shared by the library's translation units (not installed).
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <functional>
#include <mutex>
#include <utility>
#include <string>
#include <vector>

#include "../../include/sv_gb300.h"

struct sv_fused;
struct sv_mlp;

namespace svg {

void set_error(const char *fmt, ...);
// fn(i) for every i in [0, n) on up to `threads` host threads (the caller's included; fewer when
// the machine has fewer or no more can start), indices handed out through a shared counter.
// Rethrows the first exception a worker raised, after every worker has finished.
void host_parallel_for(size_t n, size_t threads, const std::function<void(size_t)> &fn);
void clear_error();

#define SV_CUDA_TRY(call)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            ::svg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                             __LINE__);                                                       \
            return SV_ECUDA;                                                                  \
        }                                                                                     \
    } while (0)

#define SV_TRY(expr)            \
    do {                        \
        int rc_ = (expr);       \
        if (rc_ != SV_OK)       \
            return rc_;         \
    } while (0)

using cplx = std::complex<double>;

// One fused gate: dense matrix over ascending targets (local bit j <-> targets[j]).
struct FusedGate {
    int k = 0;
    int targets[SV_MAX_K] = {0, 0, 0, 0, 0, 0};
    uint32_t mask_lo = 0;   // bits of targets below 32
    uint64_t mask = 0;      // bit q set <-> qubit q is a target
    int path = SV_PATH_AUTO;
    int n_src = 0;
    uint64_t cmask = 0;     // SV_PATH_CONTROLLED: control qubits (all must be 1); else 0
    std::vector<cplx> mat;  // 2^k x 2^k row-major, fp64
    std::vector<float> ur, ui;  // fp32 rounded once from mat
    // post-phases (SV_FUSE_PHASES): after the matrix, amplitude i is multiplied by
    // exp(i * sum of theta over the terms with bit targets[j] and bit q of i both set)
    struct PostTerm {
        int j;        // target index
        int q;        // a qubit that is not a target
        double theta;
    };
    std::vector<PostTerm> post;
    // SV_PATH_SWAPS: the gate is these disjoint qubit swaps (k = 0, no matrix; mask = their qubits)
    std::vector<std::pair<int, int>> swaps;
};

// Shared-memory tile geometry of a fused gate (used by the CUDA-core tile kernel and the
// tensor-core kernel).  A tile is 2^f blocks of 32 amplitudes: the blocks obtained by varying the
// block bits in F = {target block bits} + {lowest non-target block bits}.  Inside a tile the
// amplitude index has 5 + f bits (in-block position, then the F bits in ascending order).
constexpr int kMaxTileF = 8;   // tiles of up to 2^8 blocks (64 KB)

struct TileMap {
    long long fblk[1 << kMaxTileF];   // block offset of tile block phi (deposit of phi into the F bits)
    int fpos[kMaxTileF];              // ascending block-bit positions of F
    int loff[64];             // tile-local amplitude offset of local index j
    int loffo[64];            // the same in the blocked layout's float offsets: a group's member j sits at
                              // float offset (group base's offset, swizzled) ^ loffo[j] (disjoint bits)
    int ltpos[6];             // ascending tile-local target positions
    int f;                    // a tile is 2^f blocks
    int lsh;                  // 5 - (number of targets below 5)
    int lmask;                // 2^(number of targets below 5) - 1
    int gather;               // F is not {0 .. f-1}
    long long n_tiles;        // 2^(n - 5 - f)
    unsigned char swz[1 << kMaxTileF];   // in-block position XOR of tile block phi (bank-conflict swizzle)
    unsigned char gswz[32];   // the same XOR, indexed by (group >> lsh) & lmask
};
// Requires kMaxTileF >= f, max(0, n - 5) >= f >= (number of targets >= 5); returns SV_EINVAL
// (and fills nothing usable) otherwise.
int make_tile_map(const FusedGate &g, int n, int f, TileMap *m);

// Tensor-core operand images of one fused gate (built on the host, uploaded once).
struct TcOperands {
    size_t offset_bytes = 0;  // into sv_fused::d_tc
    size_t bytes = 0;
};

// Classify the kernel path of a fused gate from its targets and the requested precision.
int classify_path(const FusedGate &g, int n, int precision, int tc_min_k, int force_path);
// Greedy fusion (the rules of SV_FUSE_GREEDY, horizontal pass included) of uncontrolled fused
// gates, each taken as one input gate, into gates of at most max_k qubits (a larger input stays
// whole); products in fp64, rounded once to fp32; global qubit numbers; path SV_PATH_AUTO.
// Throws std::bad_alloc when host memory runs out.
std::vector<FusedGate> refuse_gates(const std::vector<const FusedGate *> &in, int n_qubits, int max_k);

// Device copy bookkeeping for fused circuits; defined in sv_apply.cu.
struct DeviceMats;

// Launch the kernel for one fused gate on `stream`; `dmat` is the device fp32 matrix image
// (ur then ui, 2 * 4^k floats) for paths that read the matrix from memory (may be null for k<=5
// CUDA-core paths, which take it as a kernel argument).  Returns SV_OK or SV_ECUDA/SV_EINVAL.
int launch_fused_gate(float *sv, int n, const FusedGate &g, const float *dmat, const void *dtc,
                      cudaStream_t stream, int num_sms);

int device_sm_count(int device);

// Swap networks (sv_swap.cu): one in-place pass applying g.swaps (10 <= n qubits).
int launch_swaps(float *sv, int n, const FusedGate &g, cudaStream_t stream, int num_sms);

// Tensor-core path (sv_tc.cu): host-side operand images and the launcher.
// Tensor-core operand images of f's tensor-core gates: plan_tc_operands sets f->tc_offset (byte
// offsets, 128-byte aligned) and the total size; write_tc_operands writes every image at
// dst + offset (the gaps between images are left as they are).
int plan_tc_operands(sv_fused *f, size_t *bytes);
int write_tc_operands(const sv_fused *f, unsigned char *dst);
// A pinned host staging buffer of at least `bytes` (library-owned, grown on demand), held with
// its lock: the caller fills it and copies from it while holding `lock`.
int pinned_staging(size_t bytes, unsigned char **out, std::unique_lock<std::mutex> &lock);
// Device buffers for fused-circuit images, reused across fused circuits: dev_buffer_get hands out
// a cached buffer of this device that fits (at most 4x the request) or allocates one;
// dev_buffer_put takes one back (the caller has waited for every launch that reads it)
// and frees what the cache does not keep (at most 8 buffers, 256 MB per device).
int dev_buffer_get(int device, size_t bytes, void **out, size_t *got_bytes);
void dev_buffer_put(int device, void *p, size_t bytes);
// A gate's inputs read from another buffer: input amplitude i is src[offset(i) - off] when
// (i & mask) == rest and 0 otherwise (offset = the blocked-layout float offset); the outputs still
// cover the whole state.  Used for the first full-state gate after a lazy start: src is the small
// state of qubits 0 .. a-1, mask the bits from a up, rest the basis bits there.
struct TcSource {
    const float *src;
    unsigned long long mask, rest;
    long long off;
};
int launch_tc_gate(float *sv, int n, const FusedGate &g, const void *dtc, cudaStream_t stream, int num_sms,
                   const TcSource *vs = nullptr);
// The gate runs on a direct tensor-core kernel (at most two targets below qubit 5), the kernels
// that take a TcSource.
bool tc_gate_is_direct(const FusedGate &g);
// Cost model (sv_mlp.cu): feature vector, batched prediction in microseconds, trust test.
void mlp_features(int k, const int *targets_sorted, int path, int n, int post, float *f);
int mlp_predict_us(sv_mlp *m, const float *X, int rows, double *out_us);
bool mlp_usable(const sv_mlp *m, double max_mape);
int mlp_fallback_k(const sv_mlp *m);

// The current device's error word (allocated on first use); kernels that give up a bounded wait
// write a nonzero code there.
int device_err_word(int **out);
// Complex128 states (sv_c128.cu): the same operations in fp64 on a 16-byte-per-amplitude layout.
int c128_init(sv_state *st, uint64_t basis_index);
int c128_load(sv_state *st, const void *src, int src_on_host);
int c128_store(const sv_state *st, void *dst, int dst_on_host);
int c128_norm(const sv_state *st, double *out);
int c128_sample(sv_state *st, int n_samples);   // uniforms already in st->d_uniforms; results to st->d_samples
int c128_apply_gate(sv_state *st, const FusedGate &g, const double *umem);
// Reads and clears the current device's error word written by kernels whose bounded waits timed
// out (0 = none).  Synchronous.
int read_device_errors(int *code);

}  // namespace svg

struct sv_state {
    int n = 0;
    int c128 = 0;                   // nonzero: complex128 amplitudes (d points to doubles)
    float *d = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    // reduction workspace (library-owned)
    double *d_partials = nullptr;   // per-CTA partial sums
    unsigned *d_counter = nullptr;  // last-block-done counter (kept at 0 between calls)
    double *d_result = nullptr;     // scalar result
    int max_partials = 0;
    // sampling workspace (library-owned, grown on demand)
    double *d_chunk = nullptr;      // chunk sums, then exclusive prefix (2 * n_chunks doubles)
    double *d_uniforms = nullptr;
    unsigned long long *d_samples = nullptr;
    int sample_capacity = 0;
    long long n_chunks = 0;
    // expectation-value workspace (library-owned, grown on demand): per-CTA partials, results, counter
    double *d_ev = nullptr;
    int ev_capacity = 0;
    // small state for sv_init_apply's lazy start (library-owned, grown on demand)
    float *d_compact = nullptr;
    size_t compact_bytes = 0;
};

struct sv_fused {
    int n = 0;
    int precision = SV_PREC_FP32;
    int lazy_limit = 0;             // fused with a light-cone split: the qubits its light-cone part
                                    // names (sv_init_apply's small-state limit); 0 = the default
    std::vector<svg::FusedGate> gates;
    // device images (lazily uploaded on the first apply)
    int device = -1;
    float *d_mats = nullptr;        // fp32 (ur, ui) images of gates whose path reads memory
    std::vector<size_t> mat_offset; // per gate offset in floats into d_mats, or SIZE_MAX
    void *d_tc = nullptr;           // tensor-core operand images
    std::vector<size_t> tc_offset;  // per gate byte offset into d_tc, or SIZE_MAX
    void *d_buf = nullptr;          // one device buffer holding d_mats and d_tc
    size_t d_buf_bytes = 0;
    bool c64_ready = false;         // the complex64 images above are uploaded
    double *d_mats64 = nullptr;     // fp64 (re, im) images of k >= 5 gates, for complex128 states
    size_t d_mats64_bytes = 0;
    std::vector<size_t> mat64_offset;
    // one event per stream that has applied this circuit, recorded after its last launch there:
    // sv_fused_free waits for these (not for the whole device) before the images are reused
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> use_events;
};
