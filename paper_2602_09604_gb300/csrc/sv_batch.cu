// Batched simulation of many independent, uneven circuits in one persistent kernel launch.
//
// The paper simulates one circuit at a time (threads share the groups of one gate, section IV);
// with many small circuits that leaves a GPU idle between launches.  Here one launch covers the
// batch: persistent CTAs take work items from a device queue, a list the host orders once:
//   * a whole small circuit (at most `smem_max_n` qubits): the CTA writes |0...0> into shared
//     memory, applies every fused gate with a __syncthreads between gates, stores the state once;
//   * a whole mid-size circuit, by one CTA in the circuit's global buffer;
//   * a tile of one step of a large circuit (at least `split_min_n` qubits): step 0 writes
//     |0...0>, step s applies fused gate s-1 to 2^tile_log2 groups, in the global buffer.  A tile
//     of step s waits (bounded spin) until every tile of step s-1 of its circuit has finished.
//     Items are dequeued in list order and a dequeued item is held by a running CTA, so the tiles
//     waited on were taken earlier and finish (by induction on list position): no deadlock.  The
//     list interleaves the large circuits step by step, so a wait overlaps other circuits' work,
//     optionally in waves of at most `wave_mb` MB of state so that a wave stays in L2.
// States use the library's blocked layout (32 reals then 32 imaginaries per 256-byte block).
// The launch can be captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sv_internal.h"

using namespace svg;

namespace {

constexpr int kBatchMaxK = 4;
constexpr int kBatchMaxN = 24;   // states up to 2^25 floats: 32-bit offsets

struct BGate {
    int k;
    int targets[SV_MAX_K];   // ascending
    int mat_off;             // in float2 units into the matrix table
};

struct BCirc {
    long long state_off;     // in floats into the arena
    int n;
    int gate_begin;
    int gate_count;
    int done_off;            // large circuits: first completion counter (one per step)
};

// Work item kinds.  A circuit runs as one of them:
//   kWhole  - circuit c entirely in one CTA's shared memory;
//   kSingle - circuit c by one CTA in its global buffer, gate after gate;
//   kTile   - tile `tile` of step `step` of circuit c, in its global buffer (step 0 writes |0...0>,
//             step s >= 1 applies fused gate s-1 to 2^tile_log2 groups).
enum : int { kWhole = 0, kSingle = 1, kTile = 2 };

struct BItem {
    int kind;
    int c;
    int step;
    int tile;
};

template <int V, bool L2ONLY>
__device__ __forceinline__ void ld_v(const float *p, float (&v)[V])
{
    if constexpr (V == 4) {
        const float4 t = L2ONLY ? __ldcg(reinterpret_cast<const float4 *>(p)) : *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (V == 2) {
        const float2 t = L2ONLY ? __ldcg(reinterpret_cast<const float2 *>(p)) : *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = L2ONLY ? __ldcg(p) : *p;
    }
}

template <int V>
__device__ __forceinline__ void st_v(float *p, const float (&v)[V])
{
    if constexpr (V == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else if constexpr (V == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else *p = v[0];
}

// Apply one fused gate of K qubits to groups [g_begin, g_end) of the state S (shared or global)
// of n <= 24 qubits with all threads of the CTA; U (float2, row-major 2^K x 2^K) is in shared
// memory.  A thread takes V consecutive groups at a time: with no target below log2(V) their
// amplitudes are V consecutive positions of a block, moved with one V-wide access (and each
// matrix element read once serves V groups).  Offsets are 32-bit and recomputed for the stores.
template <int K, int V, bool L2ONLY>
__device__ void apply_in_cta(float *S, const BGate &g, const float2 *__restrict__ U, unsigned g_begin, unsigned g_end)
{
    constexpr int D = 1 << K;
    unsigned bit[K];
#pragma unroll
    for (int b = 0; b < K; ++b) bit[b] = 1u << g.targets[b];
    for (unsigned it = g_begin / V + threadIdx.x; it < g_end / V; it += blockDim.x) {
        // the matrix pointer goes through an opaque move each iteration: otherwise the 4^K
        // loop-invariant matrix loads are hoisted out of this loop into registers
        const float2 *Ui;
        {
            unsigned long long v = reinterpret_cast<unsigned long long>(U);
            asm volatile("mov.b64 %0, %0;" : "+l"(v));
            Ui = reinterpret_cast<const float2 *>(v);
        }
        unsigned base = it * V;
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const unsigned low = base & (bit[b] - 1u);
            base = ((base - low) << 1) | low;
        }
        float xr[D][V], xi[D][V];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            unsigned i = base;
#pragma unroll
            for (int b = 0; b < K; ++b)
                if ((j >> b) & 1) i |= bit[b];
            const unsigned o = ((i >> 5) << 6) | (i & 31u);
            // L2ONLY: other CTAs wrote these, so read through L2 rather than a stale L1 line
            ld_v<V, L2ONLY>(S + o, xr[j]);
            ld_v<V, L2ONLY>(S + o + 32, xi[j]);
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float yr[V], yi[V];
#pragma unroll
            for (int v = 0; v < V; ++v) yr[v] = yi[v] = 0.f;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float2 u = Ui[r * D + j];
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    yr[v] = fmaf(u.x, xr[j][v], yr[v]);
                    yr[v] = fmaf(u.y, -xi[j][v], yr[v]);
                    yi[v] = fmaf(u.x, xi[j][v], yi[v]);
                    yi[v] = fmaf(u.y, xr[j][v], yi[v]);
                }
            }
            unsigned i = base;
#pragma unroll
            for (int b = 0; b < K; ++b)
                if ((r >> b) & 1) i |= bit[b];
            const unsigned o = ((i >> 5) << 6) | (i & 31u);
            st_v<V>(S + o, yr);
            st_v<V>(S + o + 32, yi);
        }
    }
}

// V: 4 when no target is below qubit 2, 2 when none is qubit 0, else 1; never more than the
// 2^(n-K) groups.  WIDE (CTAs of at most 256 threads, up to 255 registers a thread) allows K = 4
// with V > 1; with 512-thread CTAs (128 registers) K = 4 keeps V = 1, whose 2^5 inputs per group
// already fill the budget.
template <bool L2ONLY, bool WIDE>
__device__ void apply_gate_cta(float *S, int n, const BGate &g, const float2 *U, unsigned g_begin, unsigned g_end)
{
    const int t0 = g.targets[0];   // ascending
    int v = t0 >= 2 ? 4 : (t0 == 1 ? 2 : 1);
    if (g.k == 4 && !WIDE) v = 1;
    while (v > 1 && (1 << (n - g.k)) < v) v >>= 1;
#define SV_BATCH_CASE(KK)                                                         \
    case KK:                                                                      \
        if (v == 4) apply_in_cta<KK, 4, L2ONLY>(S, g, U, g_begin, g_end);         \
        else if (v == 2) apply_in_cta<KK, 2, L2ONLY>(S, g, U, g_begin, g_end);    \
        else apply_in_cta<KK, 1, L2ONLY>(S, g, U, g_begin, g_end);                \
        break;
    switch (g.k) {
    SV_BATCH_CASE(1)
    SV_BATCH_CASE(2)
    SV_BATCH_CASE(3)
    default:
        if constexpr (WIDE) {
            if (v == 4) apply_in_cta<4, 4, L2ONLY>(S, g, U, g_begin, g_end);
            else if (v == 2) apply_in_cta<4, 2, L2ONLY>(S, g, U, g_begin, g_end);
            else apply_in_cta<4, 1, L2ONLY>(S, g, U, g_begin, g_end);
        } else {
            apply_in_cta<4, 1, L2ONLY>(S, g, U, g_begin, g_end);
        }
        break;
    }
#undef SV_BATCH_CASE
}

// blocked-layout float count of an n-qubit state (at least one 64-float block)
__device__ __host__ __forceinline__ long long state_floats(int n) { return n >= 5 ? (2ll << n) : 64ll; }

constexpr long long kSpinLimit = 1ll << 22;   // bounded wait on a step counter (about a second)
constexpr int kBatchErrCode = 0xBA7C;          // written to the device error word when a wait gives up

struct BatchArgs {
    float *arena;
    const BCirc *circ;
    const BItem *items;
    int n_items;
    const BGate *gates;
    const float2 *mats;
    int *sync;         // [0] queue head, [1] abort flag, [2 + i] completion counter i
    const int *need;   // tiles of each counted step
    int *err;          // library-wide device error word
    int tile_log2;
};

__device__ __forceinline__ void stage_matrix(float2 *sU, const float2 *mats, const BGate &g)
{
    const int dd = 1 << (2 * g.k);
    for (int i = threadIdx.x; i < dd; i += blockDim.x) sU[i] = mats[g.mat_off + i];
}

__device__ __forceinline__ void zero_floats(float *S, long long f0, long long f1)
{
    for (long long i = f0 / 4 + threadIdx.x; i < f1 / 4; i += blockDim.x)
        reinterpret_cast<float4 *>(S)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int MAXT>
__global__ void __launch_bounds__(MAXT, 1) batch_kernel(BatchArgs A)
{
    extern __shared__ __align__(16) float smem[];
    float2 *sU = reinterpret_cast<float2 *>(smem);                  // (1 << 2*kBatchMaxK) complex
    float *sS = smem + 2 * (1 << (2 * kBatchMaxK));                   // state of a shared-memory circuit
    __shared__ int cur;
    __shared__ int ok;
    for (;;) {
        if (threadIdx.x == 0) cur = (int)atomicAdd(reinterpret_cast<unsigned *>(A.sync), 1u);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= A.n_items) break;
        const BItem W = A.items[it];
        const BCirc C = A.circ[W.c];
        float *G = A.arena + C.state_off;
        const long long nf = state_floats(C.n);
        if (W.kind != kTile) {
            // whole circuit in one CTA: shared memory or the global buffer
            float *S = W.kind == kWhole ? sS : G;
            zero_floats(S, 0, nf);
            __syncthreads();
            if (threadIdx.x == 0) S[0] = 1.f;
            for (int gi = 0; gi < C.gate_count; ++gi) {
                const BGate g = A.gates[C.gate_begin + gi];
                stage_matrix(sU, A.mats, g);
                __syncthreads();   // matrix staged; previous gate's writes visible
                apply_gate_cta<false, (MAXT <= 256)>(S, C.n, g, sU, 0u, 1u << (C.n - g.k));
                __syncthreads();
            }
            if (W.kind == kWhole) {
                float4 *dst = reinterpret_cast<float4 *>(G);
                for (long long i = threadIdx.x; i < nf / 4; i += blockDim.x) dst[i] = reinterpret_cast<const float4 *>(S)[i];
                __syncthreads();
            }
            continue;
        }
        // one tile of one step of a large circuit
        int *done = A.sync + 2 + C.done_off;
        if (threadIdx.x == 0) {
            ok = 1;
            if (W.step > 0) {
                const volatile int *d = done + W.step - 1;
                const int want = A.need[C.done_off + W.step - 1];
                long long spin = 0;
                while (*d < want) {
                    if (*(volatile int *)(A.sync + 1) || ++spin > kSpinLimit) {
                        ok = 0;
                        atomicExch(A.sync + 1, 1);
                        atomicCAS(A.err, 0, kBatchErrCode);
                        break;
                    }
                    __nanosleep(128);
                }
                __threadfence();   // acquire: the previous step's writes before this step's reads
            }
        }
        __syncthreads();
        if (!ok) break;
        if (W.step == 0) {
            const long long span = 2ll << (A.tile_log2 + 3);   // floats zeroed per tile
            const long long f0 = (long long)W.tile * span;
            zero_floats(G, f0, f0 + span < nf ? f0 + span : nf);
            __syncthreads();
            if (W.tile == 0 && threadIdx.x == 0) G[0] = 1.f;
        } else {
            const BGate g = A.gates[C.gate_begin + W.step - 1];
            stage_matrix(sU, A.mats, g);
            __syncthreads();
            const unsigned groups = 1u << (C.n - g.k);
            const unsigned g0 = (unsigned)W.tile << A.tile_log2;
            const unsigned g1 = g0 + (1u << A.tile_log2) < groups ? g0 + (1u << A.tile_log2) : groups;
            apply_gate_cta<true, (MAXT <= 256)>(G, C.n, g, sU, g0, g1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();   // release: this tile's writes before the count
            atomicAdd(done + W.step, 1);
        }
    }
}

__global__ void set_one_kernel(float *p) { p[0] = 1.f; }

}  // namespace

struct sv_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *arena = nullptr;          // caller's buffer
    size_t arena_bytes = 0;
    int count = 0;
    std::vector<int> n;              // per circuit (caller order)
    std::vector<long long> off;      // per circuit, floats (caller order)
    std::vector<const sv_fused *> fused;
    std::vector<BCirc> hc;           // per circuit, largest first (device order)
    std::vector<BGate> hg;
    BCirc *d_circ = nullptr;
    BGate *d_gates = nullptr;
    float2 *d_mats = nullptr;
    // work list for the options it was built for
    BItem *d_items = nullptr;
    int *d_need = nullptr;
    int *d_sync = nullptr;
    int *d_err = nullptr;            // library's device error word (not owned)
    int n_items = 0;
    int n_counters = 0;
    int list_cfg[4] = {-1, -1, -1, -1};   // smem_max_n, split_min_n, tile_log2, wave_mb
    bool stall = false;              // test hook: first split step counts one tile too many
    bool list_stall = false;
    sv_batch_opts opts{};
    cudaGraphExec_t graph = nullptr;
    int graph_cfg[6] = {0, 0, 0, 0, 0, 0};
};

namespace {

size_t state_bytes(int n) { return sizeof(float) * (size_t)state_floats(n); }

size_t smem_bytes(const sv_batch_opts &o)
{
    return sizeof(float) * 2 * (1 << (2 * kBatchMaxK)) + (o.smem_max_n > 0 ? state_bytes(o.smem_max_n) : 0);
}

// Work list: single-CTA circuits in global memory first (largest first: the rigid chains start
// early), then the tiles of the split circuits step by step across circuits, then the circuits
// held in shared memory (short; they fill the tail).
int build_work_list(sv_batch *b)
{
    const int cfg[4] = {b->opts.smem_max_n, b->opts.split_min_n, b->opts.tile_log2, b->opts.wave_mb};
    if (b->d_items && std::memcmp(cfg, b->list_cfg, sizeof(cfg)) == 0 && b->list_stall == b->stall) return SV_OK;
    std::vector<BItem> items;
    std::vector<int> need;
    std::vector<BCirc> hc = b->hc;
    std::vector<int> split;
    for (int c = 0; c < (int)hc.size(); ++c) {
        const int n = hc[(size_t)c].n;
        hc[(size_t)c].done_off = 0;
        if (n <= b->opts.smem_max_n) continue;
        if (b->opts.split_min_n > 0 && n >= b->opts.split_min_n) {
            hc[(size_t)c].done_off = (int)need.size();
            const long long span = 2ll << (b->opts.tile_log2 + 3);
            need.push_back((int)((state_floats(n) + span - 1) / span));
            for (int gi = 0; gi < hc[(size_t)c].gate_count; ++gi) {
                const BGate &g = b->hg[(size_t)(hc[(size_t)c].gate_begin + gi)];
                const long long groups = 1ll << (n - g.k);
                need.push_back((int)((groups + (1ll << b->opts.tile_log2) - 1) >> b->opts.tile_log2));
            }
            split.push_back(c);
        } else {
            items.push_back(BItem{kSingle, c, 0, 0});
        }
    }
    // split circuits in waves of at most wave_mb MB of state (0: one wave), so a wave's states can
    // stay in L2 while its steps run; inside a wave the circuits' steps interleave level by level
    std::vector<std::vector<int>> waves;
    {
        const size_t cap = (size_t)b->opts.wave_mb << 20;
        size_t acc = 0;
        for (int c : split) {
            const size_t bytes = sizeof(float) * (size_t)state_floats(hc[(size_t)c].n);
            if (waves.empty() || (cap > 0 && acc + bytes > cap && acc > 0)) {
                waves.emplace_back();
                acc = 0;
            }
            waves.back().push_back(c);
            acc += bytes;
        }
    }
    for (const std::vector<int> &wave : waves)
        for (int s = 0;; ++s) {
            bool any = false;
            for (int c : wave) {
                if (s > hc[(size_t)c].gate_count) continue;
                any = true;
                const int t = need[(size_t)(hc[(size_t)c].done_off + s)];
                for (int i = 0; i < t; ++i) items.push_back(BItem{kTile, c, s, i});
            }
            if (!any) break;
        }
    for (int c = 0; c < (int)hc.size(); ++c)
        if (hc[(size_t)c].n <= b->opts.smem_max_n) items.push_back(BItem{kWhole, c, 0, 0});
    if (b->stall && !need.empty()) need[0] += 1;   // nothing completes the extra tile: its waiters give up
    cudaFree(b->d_items);
    cudaFree(b->d_need);
    cudaFree(b->d_sync);
    b->d_items = nullptr;
    b->d_need = nullptr;
    b->d_sync = nullptr;
    b->n_items = (int)items.size();
    b->n_counters = (int)need.size();
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(BItem) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_need, sizeof(int) * std::max<size_t>(need.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sync, sizeof(int) * (2 + need.size()));
    if (e == cudaSuccess && !items.empty()) e = cudaMemcpy(b->d_items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !need.empty()) e = cudaMemcpy(b->d_need, need.data(), sizeof(int) * need.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_circ, hc.data(), sizeof(BCirc) * hc.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        b->list_cfg[0] = -1;
        set_error("sv_batch: work list upload: %s", cudaGetErrorString(e));
        return SV_ECUDA;
    }
    std::memcpy(b->list_cfg, cfg, sizeof(cfg));
    b->list_stall = b->stall;
    return SV_OK;
}

int launch_batch(sv_batch *b)
{
    BatchArgs a;
    a.arena = b->arena;
    a.circ = b->d_circ;
    a.items = b->d_items;
    a.n_items = b->n_items;
    a.gates = b->d_gates;
    a.mats = b->d_mats;
    a.sync = b->d_sync;
    a.need = b->d_need;
    a.err = b->d_err;
    a.tile_log2 = b->opts.tile_log2;
    SV_CUDA_TRY(cudaMemsetAsync(b->d_sync, 0, sizeof(int) * (2 + (size_t)b->n_counters), b->stream));
    if (b->opts.threads <= 256)
        batch_kernel<256><<<(unsigned)b->opts.ctas, (unsigned)b->opts.threads, smem_bytes(b->opts), b->stream>>>(a);
    else
        batch_kernel<512><<<(unsigned)b->opts.ctas, (unsigned)b->opts.threads, smem_bytes(b->opts), b->stream>>>(a);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

int check_opts(const sv_batch_opts &o)
{
    if (o.threads < 32 || o.threads > 512 || (o.threads & 31)) { set_error("sv_batch: threads must be a multiple of 32 in [32, 512]"); return SV_EINVAL; }
    if (o.smem_max_n < 0 || o.smem_max_n > 14) { set_error("sv_batch: smem_max_n must be in [0, 14]"); return SV_EINVAL; }
    if (o.ctas < 1) { set_error("sv_batch: ctas must be >= 1"); return SV_EINVAL; }
    if (o.split_min_n < 0 || o.split_min_n > kBatchMaxN) { set_error("sv_batch: split_min_n must be in [0, %d]", kBatchMaxN); return SV_EINVAL; }
    if (o.tile_log2 < 5 || o.tile_log2 > 16) { set_error("sv_batch: tile_log2 must be in [5, 16]"); return SV_EINVAL; }
    if (o.wave_mb < 0 || o.wave_mb > (1 << 20)) { set_error("sv_batch: wave_mb must be in [0, 2^20]"); return SV_EINVAL; }
    return SV_OK;
}

}  // namespace

extern "C" size_t sv_batch_arena_bytes(const int *n_qubits, int count)
{
    if (!n_qubits || count < 0) return 0;
    size_t t = 0;
    for (int i = 0; i < count; ++i) {
        if (n_qubits[i] < 1 || n_qubits[i] > kBatchMaxN) return 0;
        t += (state_bytes(n_qubits[i]) + 255) & ~size_t(255);
    }
    return t;
}

extern "C" int sv_batch_create(const sv_fused *const *circuits, int count, void *arena, size_t arena_bytes, void *cuda_stream,
                               sv_batch **out)
{
    clear_error();
    if (!out || count < 1 || !circuits || !arena) { set_error("sv_batch_create: bad argument"); return SV_EINVAL; }
    *out = nullptr;
    std::vector<int> ns((size_t)count);
    for (int i = 0; i < count; ++i) {
        if (!circuits[i]) { set_error("sv_batch_create: circuit %d is NULL", i); return SV_EINVAL; }
        ns[(size_t)i] = circuits[i]->n;
        for (const FusedGate &g : circuits[i]->gates) {
            if (g.k > kBatchMaxK) { set_error("sv_batch_create: circuit %d has a %d-qubit fused gate (batch kernel takes k <= %d)", i, g.k, kBatchMaxK); return SV_EINVAL; }
            if (g.cmask) { set_error("sv_batch_create: circuit %d keeps a controlled gate (fuse with max_k >= its qubit count)", i); return SV_EINVAL; }
        }
    }
    const size_t need = sv_batch_arena_bytes(ns.data(), count);
    if (need == 0) { set_error("sv_batch_create: circuits must have 1..%d qubits", kBatchMaxN); return SV_EINVAL; }
    if (arena_bytes < need) { set_error("sv_batch_create: arena of %zu bytes is smaller than the %zu needed", arena_bytes, need); return SV_ENOMEM; }
    if ((reinterpret_cast<uintptr_t>(arena) & 255u) != 0) { set_error("sv_batch_create: arena must be 256-byte aligned"); return SV_EINVAL; }
    sv_batch *b = new (std::nothrow) sv_batch();
    if (!b) { set_error("sv_batch_create: out of host memory"); return SV_ENOMEM; }
    cudaGetDevice(&b->device);
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->arena = static_cast<float *>(arena);
    b->arena_bytes = arena_bytes;
    b->count = count;
    b->n = ns;
    b->fused.assign(circuits, circuits + count);
    size_t o = 0;
    for (int i = 0; i < count; ++i) {
        b->off.push_back((long long)(o / sizeof(float)));
        o += (state_bytes(ns[(size_t)i]) + 255) & ~size_t(255);
    }
    // device circuit order: largest first
    std::vector<int> order((size_t)count);
    for (int i = 0; i < count; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ns[(size_t)x] > ns[(size_t)y]; });
    std::vector<BCirc> hc;
    std::vector<BGate> hg;
    std::vector<float2> hm;
    for (int i : order) {
        BCirc c{};
        c.state_off = b->off[(size_t)i];
        c.n = ns[(size_t)i];
        c.gate_begin = (int)hg.size();
        for (const FusedGate &g : circuits[i]->gates) {
            BGate bg{};
            bg.k = g.k;
            for (int j = 0; j < g.k; ++j) bg.targets[j] = g.targets[j];
            bg.mat_off = (int)hm.size();
            for (size_t e = 0; e < g.ur.size(); ++e) hm.push_back(make_float2(g.ur[e], g.ui[e]));
            hg.push_back(bg);
        }
        c.gate_count = (int)hg.size() - c.gate_begin;
        hc.push_back(c);
    }
    cudaError_t e = cudaMalloc(&b->d_circ, sizeof(BCirc) * hc.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_gates, sizeof(BGate) * std::max<size_t>(hg.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_mats, sizeof(float2) * std::max<size_t>(hm.size(), 1));
    if (e == cudaSuccess && !hg.empty()) e = cudaMemcpy(b->d_gates, hg.data(), sizeof(BGate) * hg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hm.empty()) e = cudaMemcpy(b->d_mats, hm.data(), sizeof(float2) * hm.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("sv_batch_create: %s", cudaGetErrorString(e));
        sv_batch_free(b);
        return SV_ECUDA;
    }
    b->hc = std::move(hc);
    b->hg = std::move(hg);
    // the error word is allocated here, outside any later stream capture
    if (device_err_word(&b->d_err) != SV_OK) {
        sv_batch_free(b);
        return SV_ECUDA;
    }
    const int sms = device_sm_count(b->device);
    b->opts.threads = 256;
    b->opts.smem_max_n = 12;
    b->opts.ctas = sms * 2;
    b->opts.use_graph = 1;
    b->opts.split_min_n = 15;
    b->opts.tile_log2 = 12;
    b->opts.wave_mb = 0;
    *out = b;
    return SV_OK;
}

extern "C" void sv_batch_free(sv_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaFree(b->d_circ);
    cudaFree(b->d_gates);
    cudaFree(b->d_mats);
    cudaFree(b->d_items);
    cudaFree(b->d_need);
    cudaFree(b->d_sync);
    delete b;
}

extern "C" int sv_batch_set_opts(sv_batch *b, const sv_batch_opts *o)
{
    clear_error();
    if (!b || !o) { set_error("sv_batch_set_opts: NULL argument"); return SV_EINVAL; }
    SV_TRY(check_opts(*o));
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(*o)));
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(*o)));
    b->opts = *o;
    return SV_OK;
}

extern "C" int sv_batch_get_opts(const sv_batch *b, sv_batch_opts *o)
{
    clear_error();
    if (!b || !o) { set_error("sv_batch_get_opts: NULL argument"); return SV_EINVAL; }
    *o = b->opts;
    return SV_OK;
}

extern "C" int sv_batch_run(sv_batch *b)
{
    clear_error();
    if (!b) { set_error("sv_batch_run: NULL batch"); return SV_EINVAL; }
    SV_TRY(check_opts(b->opts));
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(b->opts)));
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(b->opts)));
    const bool relist = !b->d_items || b->list_cfg[0] != b->opts.smem_max_n || b->list_cfg[1] != b->opts.split_min_n ||
                        b->list_cfg[2] != b->opts.tile_log2 || b->list_cfg[3] != b->opts.wave_mb || b->list_stall != b->stall;
    if (relist) {
        // the captured graph holds the old list's pointers
        SV_CUDA_TRY(cudaStreamSynchronize(b->stream));
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        SV_TRY(build_work_list(b));
    }
    if (!b->opts.use_graph) return launch_batch(b);
    const int cfg[6] = {b->opts.threads, b->opts.smem_max_n, b->opts.ctas, b->opts.split_min_n, b->opts.tile_log2, b->opts.wave_mb};
    if (b->graph && std::memcmp(cfg, b->graph_cfg, sizeof(cfg)) != 0) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (!b->graph) {
        // capture the counter reset and the persistent launch once; replays reuse them
        cudaStream_t cs = nullptr;
        SV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaStream_t saved = b->stream;
        b->stream = cs;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int rc = e == cudaSuccess ? launch_batch(b) : SV_ECUDA;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        b->stream = saved;
        cudaStreamDestroy(cs);
        if (e != cudaSuccess || e2 != cudaSuccess || rc != SV_OK) {
            if (g) cudaGraphDestroy(g);
            set_error("sv_batch_run: graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
            return SV_ECUDA;
        }
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { set_error("sv_batch_run: graph instantiate failed: %s", cudaGetErrorString(e)); return SV_ECUDA; }
        std::memcpy(b->graph_cfg, cfg, sizeof(cfg));
    }
    SV_CUDA_TRY(cudaGraphLaunch(b->graph, b->stream));
    return SV_OK;
}

// Baseline: the same circuits one after another with the single-circuit kernels: per circuit a
// state reset and one launch per fused gate (what a caller looping over sv_apply_fused_gates runs).
extern "C" int sv_batch_run_loop(sv_batch *b)
{
    clear_error();
    if (!b) { set_error("sv_batch_run_loop: NULL batch"); return SV_EINVAL; }
    const int sms = device_sm_count(b->device);
    for (int i = 0; i < b->count; ++i) {
        float *p = b->arena + b->off[(size_t)i];
        const int n = b->n[(size_t)i];
        SV_CUDA_TRY(cudaMemsetAsync(p, 0, state_bytes(n), b->stream));
        set_one_kernel<<<1, 1, 0, b->stream>>>(p);
        SV_CUDA_TRY(cudaGetLastError());
        for (const FusedGate &g : b->fused[(size_t)i]->gates)
            SV_TRY(launch_fused_gate(p, n, g, nullptr, nullptr, b->stream, sms));
    }
    return SV_OK;
}

extern "C" int sv_batch_inject_stall(sv_batch *b, int on)
{
    clear_error();
    if (!b) { set_error("sv_batch_inject_stall: NULL batch"); return SV_EINVAL; }
    b->stall = on != 0;
    return SV_OK;
}

extern "C" int sv_batch_state_offset(const sv_batch *b, int i, size_t *offset_bytes)
{
    clear_error();
    if (!b || !offset_bytes || i < 0 || i >= b->count) { set_error("sv_batch_state_offset: bad argument"); return SV_EINVAL; }
    *offset_bytes = sizeof(float) * (size_t)b->off[(size_t)i];
    return SV_OK;
}
