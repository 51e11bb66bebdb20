// Batched simulation of many independent, uneven circuits in one persistent kernel launch.
//
// The paper simulates one circuit at a time (threads share the groups of one gate, section IV);
// with many small circuits that leaves a GPU idle between launches.  Here every CTA takes whole
// circuits from a device work queue (largest first) and runs all of a circuit's fused gates
// itself, so one launch covers the batch:
//   * circuits of at most `smem_max_n` qubits live in shared memory: the CTA writes |0...0> there,
//     applies every fused gate with a __syncthreads between gates, and stores the state once;
//   * larger circuits are initialised and updated in their global state buffer (L2-resident for
//     the sizes this serves) by the same CTA, gate after gate.
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
    int pad;
};

__device__ __forceinline__ unsigned long long bins0(unsigned long long x, int p)
{
    const unsigned long long low = x & ((1ull << p) - 1ull);
    return ((x >> p) << (p + 1)) | low;
}

__device__ __forceinline__ long long boff(unsigned long long i) { return (long long)(((i >> 5) << 6) | (i & 31ull)); }

// Apply one fused gate of K qubits to the state S (shared or global) of n <= 24 qubits with all
// threads of the CTA; U (float2, row-major 2^K x 2^K) is in shared memory.  Offsets are 32-bit
// and recomputed for the stores, so a thread holds only its group's 2^(K+1) values.
template <int K>
__device__ void apply_in_cta(float *S, int n, const BGate &g, const float2 *__restrict__ U)
{
    constexpr int D = 1 << K;
    unsigned bit[K];
#pragma unroll
    for (int b = 0; b < K; ++b) bit[b] = 1u << g.targets[b];
    const unsigned groups = 1u << (n - K);
    for (unsigned grp = threadIdx.x; grp < groups; grp += blockDim.x) {
        // the matrix pointer goes through an opaque move each iteration: otherwise the 4^K
        // loop-invariant matrix loads are hoisted out of this loop into registers
        const float2 *Ui;
        {
            unsigned long long v = reinterpret_cast<unsigned long long>(U);
            asm volatile("mov.b64 %0, %0;" : "+l"(v));
            Ui = reinterpret_cast<const float2 *>(v);
        }
        unsigned base = grp;
#pragma unroll
        for (int b = 0; b < K; ++b) {
            const unsigned low = base & (bit[b] - 1u);
            base = ((base - low) << 1) | low;
        }
        float xr[D], xi[D];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            unsigned i = base;
#pragma unroll
            for (int b = 0; b < K; ++b)
                if ((j >> b) & 1) i |= bit[b];
            const unsigned o = ((i >> 5) << 6) | (i & 31u);
            xr[j] = S[o];
            xi[j] = S[o + 32];
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float yr = 0.f, yi = 0.f;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const float2 u = Ui[r * D + j];
                yr = fmaf(u.x, xr[j], yr);
                yr = fmaf(u.y, -xi[j], yr);
                yi = fmaf(u.x, xi[j], yi);
                yi = fmaf(u.y, xr[j], yi);
            }
            unsigned i = base;
#pragma unroll
            for (int b = 0; b < K; ++b)
                if ((r >> b) & 1) i |= bit[b];
            const unsigned o = ((i >> 5) << 6) | (i & 31u);
            S[o] = yr;
            S[o + 32] = yi;
        }
    }
}

__device__ void apply_gate_cta(float *S, int n, const BGate &g, const float2 *U)
{
    switch (g.k) {
    case 1: apply_in_cta<1>(S, n, g, U); break;
    case 2: apply_in_cta<2>(S, n, g, U); break;
    case 3: apply_in_cta<3>(S, n, g, U); break;
    default: apply_in_cta<4>(S, n, g, U); break;
    }
}

// blocked-layout float count of an n-qubit state (at least one 64-float block)
__device__ __host__ __forceinline__ long long state_floats(int n) { return n >= 5 ? (2ll << n) : 64ll; }

__global__ void __launch_bounds__(512, 1) batch_kernel(float *__restrict__ arena, const BCirc *__restrict__ circ, int n_circ,
                             const BGate *__restrict__ gates, const float2 *__restrict__ mats,
                             unsigned *__restrict__ queue, int smem_max_n)
{
    extern __shared__ __align__(16) float smem[];
    float2 *sU = reinterpret_cast<float2 *>(smem);                  // (1 << 2*kBatchMaxK) complex
    float *sS = smem + 2 * (1 << (2 * kBatchMaxK));                   // state of a shared-memory circuit
    __shared__ int cur;
    for (;;) {
        if (threadIdx.x == 0) cur = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int c = cur;
        __syncthreads();
        if (c >= n_circ) break;
        const BCirc C = circ[c];
        const bool in_smem = C.n <= smem_max_n;
        float *S = in_smem ? sS : arena + C.state_off;
        const long long nf = state_floats(C.n);
        // |0...0>
        for (long long i = threadIdx.x; i < nf / 4; i += blockDim.x)
            reinterpret_cast<float4 *>(S)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        if (threadIdx.x == 0) S[0] = 1.f;
        for (int gi = 0; gi < C.gate_count; ++gi) {
            const BGate g = gates[C.gate_begin + gi];
            const int dd = 1 << (2 * g.k);
            for (int i = threadIdx.x; i < dd; i += blockDim.x) sU[i] = mats[g.mat_off + i];
            __syncthreads();   // matrix staged; previous gate's writes visible
            apply_gate_cta(S, C.n, g, sU);
            __syncthreads();
        }
        if (in_smem) {
            float4 *dst = reinterpret_cast<float4 *>(arena + C.state_off);
            for (long long i = threadIdx.x; i < nf / 4; i += blockDim.x) dst[i] = reinterpret_cast<const float4 *>(S)[i];
            __syncthreads();
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
    BCirc *d_circ = nullptr;
    BGate *d_gates = nullptr;
    float2 *d_mats = nullptr;
    unsigned *d_queue = nullptr;
    int n_gates = 0;
    sv_batch_opts opts{};
    cudaGraphExec_t graph = nullptr;
    int graph_cfg[3] = {0, 0, 0};
};

namespace {

size_t state_bytes(int n) { return sizeof(float) * (size_t)state_floats(n); }

int launch_batch(sv_batch *b)
{
    const int smem_n = b->opts.smem_max_n;
    const size_t smem = sizeof(float) * 2 * (1 << (2 * kBatchMaxK)) + (smem_n > 0 ? state_bytes(smem_n) : 0);
    SV_CUDA_TRY(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned), b->stream));
    batch_kernel<<<(unsigned)b->opts.ctas, (unsigned)b->opts.threads, smem, b->stream>>>(b->arena, b->d_circ, b->count, b->d_gates,
                                                                                       b->d_mats, b->d_queue, smem_n);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

int check_opts(const sv_batch_opts &o, int num_sms)
{
    (void)num_sms;
    if (o.threads < 32 || o.threads > 1024 || (o.threads & 31)) { set_error("sv_batch: threads must be a multiple of 32 in [32, 1024]"); return SV_EINVAL; }
    if (o.smem_max_n < 0 || o.smem_max_n > 14) { set_error("sv_batch: smem_max_n must be in [0, 14]"); return SV_EINVAL; }
    if (o.ctas < 1) { set_error("sv_batch: ctas must be >= 1"); return SV_EINVAL; }
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
        for (const FusedGate &g : circuits[i]->gates)
            if (g.k > kBatchMaxK) { set_error("sv_batch_create: circuit %d has a %d-qubit fused gate (batch kernel takes k <= %d)", i, g.k, kBatchMaxK); return SV_EINVAL; }
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
    // work queue order: largest circuits first (the long poles start early)
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
    b->n_gates = (int)hg.size();
    cudaError_t e = cudaMalloc(&b->d_circ, sizeof(BCirc) * hc.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_gates, sizeof(BGate) * std::max<size_t>(hg.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_mats, sizeof(float2) * std::max<size_t>(hm.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_circ, hc.data(), sizeof(BCirc) * hc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hg.empty()) e = cudaMemcpy(b->d_gates, hg.data(), sizeof(BGate) * hg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hm.empty()) e = cudaMemcpy(b->d_mats, hm.data(), sizeof(float2) * hm.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        set_error("sv_batch_create: %s", cudaGetErrorString(e));
        sv_batch_free(b);
        return SV_ECUDA;
    }
    const int sms = device_sm_count(b->device);
    b->opts.threads = 256;
    b->opts.smem_max_n = 13;
    b->opts.ctas = sms * 2;
    b->opts.use_graph = 1;
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
    cudaFree(b->d_queue);
    delete b;
}

extern "C" int sv_batch_set_opts(sv_batch *b, const sv_batch_opts *o)
{
    clear_error();
    if (!b || !o) { set_error("sv_batch_set_opts: NULL argument"); return SV_EINVAL; }
    SV_TRY(check_opts(*o, device_sm_count(b->device)));
    const size_t smem = sizeof(float) * 2 * (1 << (2 * kBatchMaxK)) + (o->smem_max_n > 0 ? state_bytes(o->smem_max_n) : 0);
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
    SV_TRY(check_opts(b->opts, 0));
    {
        const size_t smem = sizeof(float) * 2 * (1 << (2 * kBatchMaxK)) + (b->opts.smem_max_n > 0 ? state_bytes(b->opts.smem_max_n) : 0);
        SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (!b->opts.use_graph) return launch_batch(b);
    const int cfg[3] = {b->opts.threads, b->opts.smem_max_n, b->opts.ctas};
    if (b->graph && std::memcmp(cfg, b->graph_cfg, sizeof(cfg)) != 0) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (!b->graph) {
        // capture the queue reset and the persistent launch once; replays reuse them
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

extern "C" int sv_batch_state_offset(const sv_batch *b, int i, size_t *offset_bytes)
{
    clear_error();
    if (!b || !offset_bytes || i < 0 || i >= b->count) { set_error("sv_batch_state_offset: bad argument"); return SV_EINVAL; }
    *offset_bytes = sizeof(float) * (size_t)b->off[(size_t)i];
    return SV_OK;
}
