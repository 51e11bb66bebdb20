// CUDA-core kernels that apply one fused k-qubit gate (Eq. 3) to the blocked complex64 state.
//
// Three target classes get separate kernels (section IV-C distinguishes "regular" loops, whose
// target bits lie above the vector width, from "irregular" ones below it; here the width is the
// 32-amplitude block of the layout):
//   HIGH  -- every target >= 5.  A group's 2^k amplitudes sit at the same position of 2^k different
//            blocks, so each thread loads its group straight into registers with 128-bit loads;
//            a warp's loads cover whole 128-byte lines.  No shared memory.
//   LOW   -- every target < 5, or more generally a tile whose blocks are contiguous.  A warp copies
//            a tile of 2^f consecutive blocks into shared memory through registers (16-byte loads,
//            XOR-swizzled stores), applies the gate to every group of the tile from shared memory,
//            and writes the tile back with 16-byte stores.
//   MIXED -- low and high targets.  Same as LOW, but the tile's 2^f blocks are gathered over the
//            high target bits (plus the lowest free block bits, so copies stay >= 512 bytes).
// Section IV-B's load buffering is kept: a thread reads its whole group into registers first and
// then writes each output row as soon as it is formed, so rows never overwrite pending inputs.
//
// The fp32 gate matrix of a k <= 5 gate travels by value in the kernel's parameter block
// (__grid_constant__, constant bank): with the mat-vec fully unrolled every matrix element is an
// immediate constant-bank operand of its FFMA, so the inner loop issues no loads for the matrix.
// k = 6 (32 KB of matrix, beyond the 32,764-byte parameter limit) stages the matrix in shared
// memory once per CTA instead.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "sv_internal.h"

namespace svg {
namespace {

constexpr int kHighThreads = 256;
constexpr int kTileThreads = 128;
constexpr int kTileWarps = kTileThreads / 32;

// fp32 matrix image passed by value: (re, im) pairs, ordered the way the kernel walks them so
// consecutive FFMAs read neighbouring constant-bank words (HIGH: row-major; tile: column-major).
template <int K>
struct MatArg {
    float u[2 << (2 * K)];
};
struct NoMat {};

template <int K>
using MatOf = typename std::conditional<(K <= 5), MatArg<K>, NoMat>::type;

template <int K>
struct HighArgs {
    MatOf<K> m;
    long long boff[1 << K];   // float offset of local index j relative to the group's first block
    int tpos[K];              // ascending block-bit positions (target - 5)
    long long n_items;        // block-groups * threads per block-group
};

template <int K>
struct TileArgs {
    MatOf<K> m;
    TileMap t;
};

// Controlled gate kept whole (Section IV, ApplyControlledGate): only the groups whose control
// bits are all 1 exist, so the group index enumerates the free bits (neither target nor control).
template <int K>
struct CtrlArgs {
    MatArg<K> m;
    long long foff[1 << K];                 // float offset of local index j from the group base
    int pos[SV_MAX_K + SV_MAX_CONTROLS];    // ascending target and control qubits
    int npos;
    unsigned long long cmask;               // control bits, set in every group base
    long long n_groups;                     // 2^(n - k - n_controls)
};

template <int K>
__host__ __device__ constexpr int high_vec() { return K <= 2 ? 4 : (K <= 4 ? 2 : 1); }

// Minimum resident CTAs per SM handed to __launch_bounds__: caps registers per thread so the
// unrolled mat-vec cannot trade occupancy (memory parallelism) for scheduling freedom.
template <int K>
__host__ __device__ constexpr int high_min_blocks() { return K <= 3 ? 4 : (K <= 5 ? 2 : 1); }
template <int K>
__host__ __device__ constexpr int tile_min_blocks() { return K <= 3 ? 8 : (K == 4 ? 6 : (K == 5 ? 4 : 1)); }

// Returns x unchanged through an opaque move, so address arithmetic recomputed from it for the
// output phase is not merged with (and kept alive from) the input phase.
template <typename T>
__device__ __forceinline__ T opaque(T x)
{
    if constexpr (sizeof(T) == 8) {
        unsigned long long v = reinterpret_cast<unsigned long long &>(x);
        asm volatile("mov.b64 %0, %0;" : "+l"(v));
        return reinterpret_cast<T &>(v);
    } else {
        unsigned v = reinterpret_cast<unsigned &>(x);
        asm volatile("mov.b32 %0, %0;" : "+r"(v));
        return reinterpret_cast<T &>(v);
    }
}

__device__ __forceinline__ unsigned long long insert_zero(unsigned long long x, int p)
{
    const unsigned long long low = x & ((1ull << p) - 1ull);
    return ((x >> p) << (p + 1)) | low;
}

template <int V>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[V])
{
    if constexpr (V == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (V == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = *p;
    }
}

template <int V>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[V])
{
    if constexpr (V == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

// y_r = sum_j U[r][j] x_j for one complex row; U from the parameter block (K <= 5).
template <int K, int V>
__device__ __forceinline__ void row_param(const MatArg<K> &m, int r, const float (&xr)[1 << K][V],
                                          const float (&xi)[1 << K][V], float (&yr)[V], float (&yi)[V])
{
    constexpr int D = 1 << K;
#pragma unroll
    for (int v = 0; v < V; ++v) { yr[v] = 0.f; yi[v] = 0.f; }
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float ar = m.u[2 * (r * D + j)], ai = m.u[2 * (r * D + j) + 1];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            yr[v] = fmaf(ar, xr[j][v], yr[v]);
            yr[v] = fmaf(ai, -xi[j][v], yr[v]);
            yi[v] = fmaf(ar, xi[j][v], yi[v]);
            yi[v] = fmaf(ai, xr[j][v], yi[v]);
        }
    }
}

// Same with U as interleaved (re, im) pairs in shared memory (K = 6).
template <int K, int V>
__device__ __forceinline__ void row_smem(const float2 *__restrict__ su, int r, const float (&xr)[1 << K][V],
                                         const float (&xi)[1 << K][V], float (&yr)[V], float (&yi)[V])
{
    constexpr int D = 1 << K;
#pragma unroll
    for (int v = 0; v < V; ++v) { yr[v] = 0.f; yi[v] = 0.f; }
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float2 a = su[r * D + j];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            yr[v] = fmaf(a.x, xr[j][v], yr[v]);
            yr[v] = fmaf(a.y, -xi[j][v], yr[v]);
            yi[v] = fmaf(a.x, xi[j][v], yi[v]);
            yi[v] = fmaf(a.y, xr[j][v], yi[v]);
        }
    }
}

// ------------------------------------------------------------------------------------ HIGH
// One work item per thread and no loop around it: a loop would let the compiler hoist the
// 2 * 4^k loop-invariant matrix loads into registers instead of folding them into the FFMAs.
template <int K>
__global__ void __launch_bounds__(kHighThreads, high_min_blocks<K>()) apply_high_kernel(float *__restrict__ sv, const __grid_constant__ HighArgs<K> a,
                                                                   const float2 *__restrict__ umem)
{
    constexpr int V = high_vec<K>();
    constexpr int TPB = 32 / V;
    constexpr int D = 1 << K;
    extern __shared__ float2 s_u[];
    if constexpr (K == 6) {
        for (int i = threadIdx.x; i < D * D; i += blockDim.x) s_u[i] = umem[i];
        __syncthreads();
    }
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= a.n_items) return;
    unsigned long long blk = (unsigned long long)w / TPB;
    const int pos = int(w % TPB) * V;
#pragma unroll
    for (int b = 0; b < K; ++b) blk = insert_zero(blk, a.tpos[b]);
    float *base = sv + (long long)(blk << 6) + pos;
    float xr[D][V], xi[D][V];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        ld_vec<V>(base + a.boff[j], xr[j]);
        ld_vec<V>(base + a.boff[j] + 32, xi[j]);
    }
    float *obase = opaque(base);
    if constexpr (K <= 5) {
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float yr[V], yi[V];
            row_param<K, V>(a.m, r, xr, xi, yr, yi);
            float *p = opaque(obase) + a.boff[r];
            st_vec<V>(p, yr);
            st_vec<V>(p + 32, yi);
        }
    } else {
#pragma unroll 1
        for (int r = 0; r < D; ++r) {
            float yr[V], yi[V];
            row_smem<K, V>(s_u, r, xr, xi, yr, yi);
            st_vec<V>(obase + a.boff[r], yr);
            st_vec<V>(obase + a.boff[r] + 32, yi);
        }
    }
}

// ------------------------------------------------------------------------------ LOW / MIXED

// Tile size in blocks (log2) for the fixed-size tile kernel: 2^F blocks = 32 * 2^F amplitudes,
// so every lane of the warp owns 2^(F-K) >= 1 groups.
template <int K>
__host__ __device__ constexpr int tile_f() { return K < 3 ? 3 : K; }

// XOR permutation of the four floats of one 16-byte chunk (s & 1 swaps neighbours, s & 2 swaps
// pairs); it is its own inverse.
__device__ __forceinline__ float4 xor_perm4(float4 v, unsigned s)
{
    if (s & 1u) { float t = v.x; v.x = v.y; v.y = t; t = v.z; v.z = v.w; v.w = t; }
    if (s & 2u) { float t = v.x; v.x = v.z; v.z = t; t = v.y; v.y = v.w; v.w = t; }
    return v;
}

// One tile per warp.  FIXED: f = tile_f<K>() known at compile time (states with at least 2^f
// blocks) -- straight-line code, matrix elements stay constant-bank operands.  !FIXED: small
// states with fewer blocks than that; f is a runtime value and the group loop is a real loop.
//
// Bank conflicts: the L targets below 5 leave only 2^(5-L) distinct in-block positions per input
// index, so lanes whose groups sit in different blocks would hit the same banks 2^L times.  Each
// tile block phi is therefore stored with its in-block positions XOR-ed by swz[phi], which puts
// distinct values on the low target bits of the 2^L blocks one warp instruction touches.  Groups
// keep their members in blocks with the same swizzle (members differ only in target bits), so a
// lane applies one XOR, gswz, to all of its addresses.  The copies move 16-byte chunks through
// registers: the XOR's bits 2-4 pick the chunk, bits 0-1 permute inside it.
template <int K, bool GATHER, bool FIXED>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<K>()) apply_tile_kernel(float *__restrict__ sv, const __grid_constant__ TileArgs<K> a,
                                                                   const float2 *__restrict__ umem)
{
    constexpr int D = 1 << K;
    extern __shared__ __align__(16) float smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int f = FIXED ? tile_f<K>() : a.t.f;
    const int tile_floats = 64 << f;
    float2 *s_u = reinterpret_cast<float2 *>(smem);
    float *buf = smem + (K == 6 ? 2 * D * D : 0) + warp * tile_floats;
    if constexpr (K == 6) {
        for (int i = threadIdx.x; i < D * D; i += blockDim.x) s_u[i] = umem[i];
        __syncthreads();
    }
    const long long t = (long long)blockIdx.x * kTileWarps + warp;
    if (t >= a.t.n_tiles) return;
    unsigned long long b0 = (unsigned long long)t;
    if constexpr (GATHER) {
        for (int i = 0; i < f; ++i) b0 = insert_zero(b0, a.t.fpos[i]);
    } else {
        b0 <<= f;
    }
    // chunk c of the tile: block phi = c >> 4, half (re / im) = (c >> 3) & 1, chunk q = c & 7
    auto gaddr = [&](int c) -> float * {
        const int phi = c >> 4;
        const unsigned long long blk = GATHER ? b0 + (unsigned long long)a.t.fblk[phi] : b0 + (unsigned long long)phi;
        return sv + (long long)(blk << 6) + (c & 15) * 4;
    };
    auto saddr = [&](int c, unsigned &sw) -> float * {
        const int phi = c >> 4;
        sw = a.t.swz[phi];
        return buf + phi * 64 + (c & 8) * 4 + (((c & 7) ^ (int)(sw >> 2)) << 2);
    };
    if constexpr (FIXED) {
        constexpr int CPL = (16 << tile_f<K>()) / 32;   // chunks per lane
        float4 v[CPL];
#pragma unroll
        for (int i = 0; i < CPL; ++i) v[i] = *reinterpret_cast<const float4 *>(gaddr(lane + 32 * i));
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            unsigned sw;
            float *d = saddr(lane + 32 * i, sw);
            *reinterpret_cast<float4 *>(d) = xor_perm4(v[i], sw);
        }
    } else {
        for (int c = lane; c < (16 << f); c += 32) {
            const float4 v = *reinterpret_cast<const float4 *>(gaddr(c));
            unsigned sw;
            float *d = saddr(c, sw);
            *reinterpret_cast<float4 *>(d) = xor_perm4(v, sw);
        }
    }
    __syncwarp();

    // k <= 5: column order -- all 2^k outputs accumulate in registers while the inputs stream
    // from shared memory one at a time (2^(k+1) accumulators, and every input step offers 2^(k+2)
    // independent FFMAs).  The group's inputs are all read before any output is written back.
    // k = 6: row order with the inputs held in registers and the matrix read from shared memory.
    auto do_group = [&](int g) {
        unsigned base = (unsigned)g;
#pragma unroll
        for (int b = 0; b < K; ++b) base = (unsigned)insert_zero(base, a.t.ltpos[b]);
        const unsigned sg = a.t.gswz[(g >> a.t.lsh) & a.t.lmask];
        // member j's float offset: the layout map moves index bits and the swizzle XORs in-block
        // bits, both bitwise, and the base has zeros at the targets, so one XOR per member
        const unsigned ob = ((base >> 5) << 6) | ((base & 31u) ^ sg);
        if constexpr (K <= 5) {
            float yr[D], yi[D];
#pragma unroll
            for (int r = 0; r < D; ++r) { yr[r] = 0.f; yi[r] = 0.f; }
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const unsigned o = ob ^ (unsigned)a.t.loffo[j];
                const float xr = buf[o], xi = buf[o + 32];
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    const float ar = a.m.u[2 * (j * D + r)], ai = a.m.u[2 * (j * D + r) + 1];
                    yr[r] = fmaf(ar, xr, yr[r]);
                    yr[r] = fmaf(ai, -xi, yr[r]);
                    yi[r] = fmaf(ar, xi, yi[r]);
                    yi[r] = fmaf(ai, xr, yi[r]);
                }
            }
            // Groups of different lanes are disjoint, so no lane synchronisation is needed here.
#pragma unroll
            for (int r = 0; r < D; ++r) {
                const unsigned o = ob ^ (unsigned)a.t.loffo[r];
                buf[o] = yr[r];
                buf[o + 32] = yi[r];
            }
        } else {
            float xr[D][1], xi[D][1];
#pragma unroll
            for (int j = 0; j < D; ++j) {
                const unsigned o = ob ^ (unsigned)a.t.loffo[j];
                xr[j][0] = buf[o];
                xi[j][0] = buf[o + 32];
            }
            const unsigned obo = opaque(ob);
#pragma unroll 1
            for (int r = 0; r < D; ++r) {
                float yr[1], yi[1];
                row_smem<K, 1>(s_u, r, xr, xi, yr, yi);
                const unsigned o = obo ^ (unsigned)a.t.loffo[r];
                buf[o] = yr[0];
                buf[o + 32] = yi[0];
            }
        }
    };
    if constexpr (FIXED) {
        constexpr int per_lane = 1 << (tile_f<K>() - K);
#pragma unroll
        for (int m = 0; m < per_lane; ++m) do_group(lane + 32 * m);
    } else {
        const int groups = 1 << (5 + f - K);
        for (int g = lane; g < groups; g += 32) do_group(g);
    }
    __syncwarp();
    for (int c = lane; c < (16 << f); c += 32) {
        unsigned sw;
        const float *s_ = saddr(c, sw);
        *reinterpret_cast<float4 *>(gaddr(c)) = xor_perm4(*reinterpret_cast<const float4 *>(s_), sw);
    }
}

// ------------------------------------------------------------------------------ host side
template <typename T>
void fill_mat(T &m, const FusedGate &g, bool column_major)
{
    if constexpr (!std::is_same<T, NoMat>::value) {
        const int D = 1 << g.k;
        for (int r = 0; r < D; ++r)
            for (int j = 0; j < D; ++j) {
                const int e = column_major ? j * D + r : r * D + j;
                m.u[2 * e] = g.ur[size_t(r) * D + j];
                m.u[2 * e + 1] = g.ui[size_t(r) * D + j];
            }
    } else {
        (void)m;
        (void)g;
        (void)column_major;
    }
}

// Kernel attributes already set, as a bit per device (function attributes are per device).
struct Occ {
    uint64_t high[7] = {0};
    uint64_t tile[7][4] = {};   // [K][gather + 2 * fixed]
};
Occ g_occ;
std::mutex g_occ_mu;

uint64_t current_device_bit()
{
    int dev = 0;
    cudaGetDevice(&dev);
    return dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
}

// One group per thread: the base index has a zero inserted at every target and control position
// (ascending) and the control bits then set; the 2^K amplitudes are gathered, multiplied by U
// (constant-bank operands) and written back in place.
template <int K>
__global__ void __launch_bounds__(kHighThreads) apply_ctrl_kernel(float *__restrict__ sv, const __grid_constant__ CtrlArgs<K> a)
{
    constexpr int D = 1 << K;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_groups) return;
    unsigned long long b = (unsigned long long)g;
    for (int i = 0; i < a.npos; ++i) b = insert_zero(b, a.pos[i]);
    b |= a.cmask;
    float *base = sv + (long long)(((b >> 5) << 6) | (b & 31ull));
    float xr[D][1], xi[D][1];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        xr[j][0] = base[a.foff[j]];
        xi[j][0] = base[a.foff[j] + 32];
    }
    float *obase = opaque(base);
#pragma unroll
    for (int r = 0; r < D; ++r) {
        float yr[1], yi[1];
        row_param<K, 1>(a.m, r, xr, xi, yr, yi);
        obase[a.foff[r]] = yr[0];
        obase[a.foff[r] + 32] = yi[0];
    }
}

template <int K>
int launch_ctrl(float *sv, int n, const FusedGate &g, const float2 *, cudaStream_t stream, int)
{
    CtrlArgs<K> a;
    std::memset(&a, 0, sizeof(a));
    fill_mat(a.m, g, false);
    for (int j = 0; j < (1 << K); ++j) {
        unsigned long long o = 0;
        for (int t = 0; t < K; ++t)
            if ((j >> t) & 1) o |= 1ull << g.targets[t];
        a.foff[j] = (long long)(((o >> 5) << 6) | (o & 31ull));
    }
    const unsigned long long all = g.mask | g.cmask;
    int np = 0;
    for (int q = 0; q < n; ++q)
        if ((all >> q) & 1) a.pos[np++] = q;
    if (np != K + __builtin_popcountll(g.cmask) || (g.mask & g.cmask) || (all >> n)) {
        set_error("launch: controlled gate names a qubit twice or outside the state");
        return SV_EINVAL;
    }
    a.npos = np;
    a.cmask = g.cmask;
    a.n_groups = 1ll << (n - np);
    const long long grid = (a.n_groups + kHighThreads - 1) / kHighThreads;
    apply_ctrl_kernel<K><<<(unsigned)grid, kHighThreads, 0, stream>>>(sv, a);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

template <int K>
int launch_high(float *sv, int n, const FusedGate &g, const float2 *umem, cudaStream_t stream, int num_sms)
{
    HighArgs<K> a;
    std::memset(&a, 0, sizeof(a));
    fill_mat(a.m, g, false);
    for (int b = 0; b < K; ++b) a.tpos[b] = g.targets[b] - 5;
    for (int j = 0; j < (1 << K); ++j) {
        long long o = 0;
        for (int b = 0; b < K; ++b)
            if ((j >> b) & 1) o |= 1ll << a.tpos[b];
        a.boff[j] = o << 6;
    }
    constexpr int V = high_vec<K>();
    a.n_items = (1ll << (n - 5 - K)) * (32 / V);
    const size_t smem = K == 6 ? sizeof(float2) * 64 * 64 : 0;
    auto kern = apply_high_kernel<K>;
    {
        const uint64_t bit = current_device_bit();
        std::lock_guard<std::mutex> lk(g_occ_mu);
        if (!(g_occ.high[K] & bit) || !bit) {
            if (smem > 48 * 1024) SV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            g_occ.high[K] |= bit;
        }
    }
    (void)num_sms;
    const long long grid = (a.n_items + kHighThreads - 1) / kHighThreads;
    kern<<<(unsigned)grid, kHighThreads, smem, stream>>>(sv, a, umem);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

template <int K>
int launch_tile(float *sv, int n, const FusedGate &g, const float2 *umem, cudaStream_t stream, int num_sms)
{
    TileArgs<K> a;
    std::memset(&a, 0, sizeof(a));
    fill_mat(a.m, g, true);
    const int nb = n > 5 ? n - 5 : 0;
    const bool fixed = nb >= tile_f<K>();
    const int f = fixed ? tile_f<K>() : nb;   // (targets >= 5) <= K <= tile_f<K>(), and <= nb always
    SV_TRY(make_tile_map(g, n, f, &a.t));
    const bool gather = a.t.gather != 0;
    const size_t smem = size_t(kTileWarps) * (64u << f) * sizeof(float) + (K == 6 ? sizeof(float2) * 64 * 64 : 0);
    auto kern = fixed ? (gather ? apply_tile_kernel<K, true, true> : apply_tile_kernel<K, false, true>)
                      : (gather ? apply_tile_kernel<K, true, false> : apply_tile_kernel<K, false, false>);
    {
        const uint64_t bit = current_device_bit();
        std::lock_guard<std::mutex> lk(g_occ_mu);
        uint64_t &slot = g_occ.tile[K][(gather ? 1 : 0) + (fixed ? 2 : 0)];
        if (!(slot & bit) || !bit) {
            if (smem > 48 * 1024 || K == 6)
                SV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)(kTileWarps * (64u << 6) * sizeof(float) + sizeof(float2) * 64 * 64)));
            slot |= bit;
        }
    }
    (void)num_sms;
    const long long grid = (a.t.n_tiles + kTileWarps - 1) / kTileWarps;
    kern<<<(unsigned)grid, kTileThreads, smem, stream>>>(sv, a, umem);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

using LaunchFn = int (*)(float *, int, const FusedGate &, const float2 *, cudaStream_t, int);
const LaunchFn kHigh[7] = {nullptr, launch_high<1>, launch_high<2>, launch_high<3>, launch_high<4>, launch_high<5>, launch_high<6>};
const LaunchFn kTile[7] = {nullptr, launch_tile<1>, launch_tile<2>, launch_tile<3>, launch_tile<4>, launch_tile<5>, launch_tile<6>};
const LaunchFn kCtrl[4] = {nullptr, launch_ctrl<1>, launch_ctrl<2>, launch_ctrl<3>};

}  // namespace

int make_tile_map(const FusedGate &g, int n, int f, TileMap *m)
{
    std::memset(m, 0, sizeof(*m));
    const int K = g.k;
    const int nb = n > 5 ? n - 5 : 0;
    int high = 0;
    for (int b = 0; b < K; ++b) high += g.targets[b] >= 5;
    if (f < 0 || f > kMaxTileF || f > nb || f < high || K < 1 || K > SV_MAX_K) {
        set_error("tile map: tile of 2^%d blocks does not fit (n=%d, k=%d, %d high targets)", f, n, K, high);
        return SV_EINVAL;
    }
    uint64_t fm = 0;   // F = high target block bits + lowest free block bits
    for (int b = 0; b < K; ++b)
        if (g.targets[b] >= 5) fm |= 1ull << (g.targets[b] - 5);
    for (int p = 0; __builtin_popcountll(fm) < f && p < nb; ++p) fm |= 1ull << p;
    int cnt = 0;
    for (int p = 0; p < nb; ++p)
        if ((fm >> p) & 1) m->fpos[cnt++] = p;
    m->f = f;
    for (int phi = 0; phi < (1 << f); ++phi) {
        long long o = 0;
        for (int i = 0; i < f; ++i)
            if ((phi >> i) & 1) o |= 1ll << m->fpos[i];
        m->fblk[phi] = o;
    }
    m->gather = fm != ((1ull << f) - 1ull);
    for (int b = 0; b < K; ++b) {
        const int t = g.targets[b];
        if (t < 5) {
            m->ltpos[b] = t;
        } else {
            int r = 0;
            while (m->fpos[r] != t - 5) ++r;
            m->ltpos[b] = 5 + r;
        }
    }
    for (int j = 0; j < (1 << K); ++j) {
        int o = 0;
        for (int b = 0; b < K; ++b)
            if ((j >> b) & 1) o |= 1 << m->ltpos[b];
        m->loff[j] = o;
        m->loffo[j] = ((o >> 5) << 6) | (o & 31);
    }
    // swizzle: deposit the lowest L non-target tile-block bits onto the L low target positions
    int lowt[5], L = 0;
    for (int b = 0; b < K; ++b)
        if (g.targets[b] < 5) lowt[L++] = g.targets[b];
    int nont[kMaxTileF], nn = 0;
    for (int r = 0; r < f; ++r) {
        bool is_t = false;
        for (int b = 0; b < K; ++b)
            if (m->ltpos[b] == 5 + r) is_t = true;
        if (!is_t) nont[nn++] = r;
    }
    auto deposit_low = [&](int v) {
        int o = 0;
        for (int i = 0; i < L; ++i)
            if ((v >> i) & 1) o |= 1 << lowt[i];
        return o;
    };
    for (int phi = 0; phi < (1 << f); ++phi) {
        int c = 0;
        for (int i = 0; i < nn; ++i)
            if ((phi >> nont[i]) & 1) c |= 1 << i;
        m->swz[phi] = (unsigned char)deposit_low(c & ((1 << L) - 1));
    }
    for (int v = 0; v < (1 << L); ++v) m->gswz[v] = (unsigned char)deposit_low(v);
    m->lsh = 5 - L;
    m->lmask = (1 << L) - 1;
    m->n_tiles = 1ll << (nb - f);
    return SV_OK;
}

int launch_fused_gate(float *sv, int n, const FusedGate &g, const float *dmat, const void *dtc, cudaStream_t stream, int num_sms)
{
    if (g.path == SV_PATH_SWAPS) return launch_swaps(sv, n, g, stream, num_sms);
    if (g.k < 1 || g.k > SV_MAX_K) { set_error("launch: bad k=%d", g.k); return SV_EINVAL; }
    const float2 *umem = reinterpret_cast<const float2 *>(dmat);
    if (g.k == 6 && !umem && g.path != SV_PATH_TC_TF32 && g.path != SV_PATH_TC_BF16X3) {
        set_error("launch: k=6 gate has no device matrix");
        return SV_EINVAL;
    }
    switch (g.path) {
    case SV_PATH_HIGH:
        for (int b = 0; b < g.k; ++b)
            if (g.targets[b] < 5 || n < 5 + g.k) { set_error("launch: HIGH path needs every target >= 5"); return SV_EINVAL; }
        return kHigh[g.k](sv, n, g, umem, stream, num_sms);
    case SV_PATH_LOW:
    case SV_PATH_MIXED:
        return kTile[g.k](sv, n, g, umem, stream, num_sms);
    case SV_PATH_TC_TF32:
    case SV_PATH_TC_BF16X3:
        return launch_tc_gate(sv, n, g, dtc, stream, num_sms);
    case SV_PATH_CONTROLLED:
        if (g.k > 3 || !g.cmask) { set_error("launch: a controlled gate has 1..3 targets and a control"); return SV_EINVAL; }
        return kCtrl[g.k](sv, n, g, umem, stream, num_sms);
    default:
        set_error("launch: unknown path %d", g.path);
        return SV_EINVAL;
    }
}

}  // namespace svg

using namespace svg;

namespace {

int upload_fused(sv_fused *f, int device)
{
    if (f->device == device && f->c64_ready) return SV_OK;
    if (f->device >= 0 && f->device != device) { set_error("sv_apply_fused_gates: fused circuit was uploaded to another device"); return SV_ESTATE; }
    // k = 6 CUDA-core kernels read an interleaved fp32 matrix image from device memory (made for
    // every k = 6 gate: sv_init_apply may run a tensor-core gate on CUDA cores on a small state)
    // one device buffer (from the library's cache) for both image kinds: fp32 (ur, ui) images
    // of the k = 6 gates, then the tensor-core images at a 256-byte aligned offset; built in a
    // pinned staging buffer and copied once
    f->mat_offset.assign(f->gates.size(), SIZE_MAX);
    size_t mat_floats = 0;
    for (size_t i = 0; i < f->gates.size(); ++i)
        if (f->gates[i].k == 6) {
            f->mat_offset[i] = mat_floats;
            mat_floats += 2 * f->gates[i].ur.size();
        }
    size_t tc_bytes = 0;
    SV_TRY(plan_tc_operands(f, &tc_bytes));
    const size_t mat_bytes = mat_floats * sizeof(float);
    const size_t tc_off = (mat_bytes + 255) & ~size_t(255);
    const size_t total = tc_off + tc_bytes;
    if (total > 0) {
        void *buf = nullptr;
        size_t got = 0;
        SV_TRY(dev_buffer_get(device, total, &buf, &got));
        std::unique_lock<std::mutex> lk;
        unsigned char *img = nullptr;
        int rc = pinned_staging(total, &img, lk);
        if (rc == SV_OK) {
            // every byte is written: the fp32 images, the gap to tc_off, the tensor-core images
            // (whole multiples of 128 bytes, so contiguous)
            std::memset(img + mat_bytes, 0, tc_off - mat_bytes);
            float *m = reinterpret_cast<float *>(img);
            for (size_t i = 0; i < f->gates.size(); ++i) {
                if (f->mat_offset[i] == SIZE_MAX) continue;
                const FusedGate &g = f->gates[i];
                float *d = m + f->mat_offset[i];
                for (size_t e = 0; e < g.ur.size(); ++e) {
                    d[2 * e] = g.ur[e];
                    d[2 * e + 1] = g.ui[e];
                }
            }
            if (tc_bytes) rc = write_tc_operands(f, img + tc_off);
        }
        if (rc == SV_OK) {
            const cudaError_t e = cudaMemcpy(buf, img, total, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                set_error("sv_apply_fused_gates: image upload: %s", cudaGetErrorString(e));
                rc = SV_ECUDA;
            }
        }
        if (rc != SV_OK) {
            dev_buffer_put(device, buf, got);
            return rc;
        }
        f->d_buf = buf;
        f->d_buf_bytes = got;
        f->d_mats = mat_bytes ? static_cast<float *>(buf) : nullptr;
        f->d_tc = tc_bytes ? static_cast<unsigned char *>(buf) + tc_off : nullptr;
    }
    f->device = device;
    f->c64_ready = true;
    return SV_OK;
}

// complex128 states read k >= 5 matrices from device memory in fp64 (built on first use)
int upload_fused_c128(sv_fused *f, int device)
{
    if (f->device >= 0 && f->device != device) { set_error("sv_apply_fused_gates: fused circuit was uploaded to another device"); return SV_ESTATE; }
    if (f->d_mats64 || !f->mat64_offset.empty()) return SV_OK;
    std::vector<double> host;
    f->mat64_offset.assign(f->gates.size(), SIZE_MAX);
    for (size_t i = 0; i < f->gates.size(); ++i) {
        const FusedGate &g = f->gates[i];
        if (g.k < 5) continue;
        f->mat64_offset[i] = host.size();
        for (const cplx &c : g.mat) {
            host.push_back(c.real());
            host.push_back(c.imag());
        }
    }
    if (!host.empty()) {
        void *buf = nullptr;
        size_t got = 0;
        SV_TRY(dev_buffer_get(device, host.size() * sizeof(double), &buf, &got));
        const cudaError_t e = cudaMemcpy(buf, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            dev_buffer_put(device, buf, got);
            set_error("sv_apply_fused_gates: fp64 image upload: %s", cudaGetErrorString(e));
            return SV_ECUDA;
        }
        f->d_mats64 = static_cast<double *>(buf);
        f->d_mats64_bytes = got;
    }
    f->device = device;
    return SV_OK;
}

}  // namespace

namespace svg {
namespace {

// Lazy start from a basis state (sv_init_apply): while the gates so far name at most
// kCompactMaxQubits qubits A, every other qubit still holds its bit of x, so the state is
// |x on the rest> (x) |small state on A>; those gates run on the 2^|A| small state, which one
// kernel then writes into the zeroed full state.
constexpr int kCompactMaxQubits = 28;   // a 2 GiB small state
constexpr int kDefaultLazyQubits = 26;  // circuits fused without a light-cone split: a 512 MB small state

struct ExpandArgs {
    int pos[kCompactMaxQubits];   // ascending qubits of A: small-state bit b -> full-state bit pos[b]
    int a;
    int l0;                       // pos[b] == b for b < l0 (A's lowest qubits are 0 .. l0 - 1)
    unsigned long long rest;      // x on the qubits outside A
    long long n_small;
};

__global__ void put_one_kernel(float *s, long long off) { s[off] = 1.0f; }

// Small-state amplitude c goes to full index rest | (bit b of c placed at pos[b]).  When A's
// lowest qubits are 0 .. l0 - 1 (l0 >= 2), the low l0 bits of c stay in place: a thread moves four
// amplitudes at a time (16-byte loads and stores of real and imaginary parts) and deposits only
// the bits above l0; otherwise one amplitude at a time with every bit deposited.
__global__ void expand_compact_kernel(float *__restrict__ full, const float *__restrict__ small, const __grid_constant__ ExpandArgs e)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (e.l0 >= 2) {
        const unsigned long long lowmask = (1ull << e.l0) - 1ull;
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (e.n_small >> 2); t += stride) {
            const unsigned long long c = (unsigned long long)t << 2;
            unsigned long long i = e.rest | (c & lowmask);
            for (int b = e.l0; b < e.a; ++b)
                if ((c >> b) & 1) i |= 1ull << e.pos[b];
            const long long fo = (long long)(((i >> 5) << 6) | (i & 31ull));
            const long long so = (long long)(((c >> 5) << 6) | (c & 31ull));
            *reinterpret_cast<float4 *>(full + fo) = *reinterpret_cast<const float4 *>(small + so);
            *reinterpret_cast<float4 *>(full + fo + 32) = *reinterpret_cast<const float4 *>(small + so + 32);
        }
        return;
    }
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < e.n_small; c += stride) {
        unsigned long long i = e.rest;
        for (int b = 0; b < e.a; ++b)
            if ((c >> b) & 1) i |= 1ull << e.pos[b];
        const long long fo = (long long)(((i >> 5) << 6) | (i & 31ull));
        const long long so = (long long)((((unsigned long long)c >> 5) << 6) | ((unsigned long long)c & 31ull));
        full[fo] = small[so];
        full[fo + 32] = small[so + 32];
    }
}

}  // namespace
}  // namespace svg

namespace {

int rank_in(uint64_t A, int q) { return __builtin_popcountll(A & ((1ull << q) - 1ull)); }

// Records that `stream` has launched kernels reading f's device images (one reusable event per
// stream), so that sv_fused_free can wait for exactly that work.
int note_fused_use(sv_fused *f, cudaStream_t stream)
{
    for (auto &u : f->use_events)
        if (u.first == stream) {
            SV_CUDA_TRY(cudaEventRecord(u.second, stream));
            return SV_OK;
        }
    cudaEvent_t e = nullptr;
    SV_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    f->use_events.emplace_back(stream, e);
    SV_CUDA_TRY(cudaEventRecord(e, stream));
    return SV_OK;
}

// gate g re-expressed on the small state of the qubits in A (ascending order is kept, so the
// matrix, its local index order and its tensor-core operand image are unchanged): a tensor-core
// gate stays on the tensor cores when the small state is large enough for them (a >= k + 5),
// every other gate takes the CUDA-core path its new targets call for
FusedGate remap_gate(const FusedGate &g, uint64_t A, int a)
{
    FusedGate r;
    r.k = g.k;
    r.n_src = g.n_src;
    for (int j = 0; j < g.k; ++j) {
        r.targets[j] = rank_in(A, g.targets[j]);
        r.mask |= 1ull << r.targets[j];
        if (r.targets[j] < 32) r.mask_lo |= 1u << r.targets[j];
    }
    for (int q = 0; q < 64; ++q)
        if ((g.cmask >> q) & 1) r.cmask |= 1ull << rank_in(A, q);
    r.mat = g.mat;
    r.ur = g.ur;
    r.ui = g.ui;
    const bool tc = (g.path == SV_PATH_TC_TF32 || g.path == SV_PATH_TC_BF16X3) && a >= g.k + 5;
    r.path = tc ? g.path : classify_path(r, a, SV_PREC_FP32, SV_MAX_K + 1, SV_PATH_AUTO);
    return r;
}

// Applies every fused gate of f to st.  With `lazy` (one flag per gate, a set closed under the
// gates' order: no flagged gate shares a qubit with an earlier unflagged one) the flagged gates run
// first, in order, on the small state of the qubits in A started from basis x (see above), which
// then replaces the whole state; the others follow in order.  Moving a flagged gate ahead of
// earlier unflagged ones is exact: they share no qubit, so they commute.
int apply_core(sv_state *st, sv_fused *f, sv_timing *timings, const std::vector<char> *lazy, uint64_t A, uint64_t x, const char *who)
{
    if (st->c128)
        for (const FusedGate &g : f->gates)
            if (!g.post.empty() || !g.swaps.empty()) {
                set_error("%s: post-phases and swap networks (SV_FUSE_PHASES) are for complex64 states", who);
                return SV_EINVAL;
            }
    if (st->c128) SV_TRY(upload_fused_c128(f, st->device));
    else SV_TRY(upload_fused(f, st->device));
    const size_t ng = f->gates.size();
    const int a = __builtin_popcountll(A);
    size_t m = 0;   // gates run on the small state
    if (lazy)
        for (char c : *lazy) m += c != 0;
    float *small = nullptr;
    if (m > 0) {
        const size_t bytes = sv_required_bytes(a);
        if (bytes > st->compact_bytes) {
            cudaStreamSynchronize(st->stream);
            cudaFree(st->d_compact);
            st->d_compact = nullptr;
            st->compact_bytes = 0;
            SV_CUDA_TRY(cudaMalloc(&st->d_compact, bytes));
            st->compact_bytes = bytes;
        }
        small = st->d_compact;
        uint64_t cx = 0;   // x restricted to A, packed
        for (int q = 0, b = 0; q < 64; ++q)
            if ((A >> q) & 1) cx |= ((x >> q) & 1ull) << b++;
        SV_CUDA_TRY(cudaMemsetAsync(small, 0, bytes, st->stream));
        put_one_kernel<<<1, 1, 0, st->stream>>>(small, (long long)(((cx >> 5) << 6) | (cx & 31ull)));
        SV_CUDA_TRY(cudaGetLastError());
    }
    auto expand = [&]() -> int {
        ExpandArgs e;
        std::memset(&e, 0, sizeof(e));
        for (int q = 0, b = 0; q < 64; ++q)
            if ((A >> q) & 1) e.pos[b++] = q;
        e.a = a;
        e.l0 = 0;
        while (e.l0 < a && e.pos[e.l0] == e.l0) ++e.l0;
        if (a < 2) e.l0 = 0;   // fewer than four amplitudes: one at a time
        e.rest = x & ~A;
        e.n_small = 1ll << a;
        SV_CUDA_TRY(cudaMemsetAsync(st->d, 0, sv_required_bytes(st->n), st->stream));
        const long long grid = std::min<long long>((e.n_small + 255) / 256, (long long)st->num_sms * 8);
        expand_compact_kernel<<<(unsigned)grid, 256, 0, st->stream>>>(st->d, small, e);
        SV_CUDA_TRY(cudaGetLastError());
        return SV_OK;
    };
    std::vector<cudaEvent_t> ev;
    if (timings && ng) {
        ev.resize(2 * ng);
        for (auto &e : ev) SV_CUDA_TRY(cudaEventCreate(&e));
    }
    // execution order: the small-state gates, then the rest (each in their original order)
    std::vector<size_t> order;
    order.reserve(ng);
    for (size_t i = 0; i < ng; ++i)
        if (m > 0 && (*lazy)[i]) order.push_back(i);
    for (size_t i = 0; i < ng; ++i)
        if (!(m > 0 && (*lazy)[i])) order.push_back(i);
    // The first full-state gate after the small ones can read the small state itself (amplitudes
    // outside it read as zero) and write every amplitude, which saves the zeroing pass and the
    // copy: when it runs on a direct tensor-core kernel and A is qubits 0 .. a - 1 (a >= 5, so the
    // basis bits outside A lie above the block bits and offsets split cleanly).
    const uint64_t amask = a >= 64 ? ~0ull : ((1ull << a) - 1ull);
    const uint64_t nmask = st->n >= 64 ? ~0ull : ((1ull << st->n) - 1ull);
    bool first_reads_small = false;
    if (m > 0 && m < ng && !st->c128 && A == amask && a >= 5) {
        const size_t i0 = order[m];
        const FusedGate &g0 = f->gates[i0];
        first_reads_small = tc_gate_is_direct(g0) && f->d_tc && i0 < f->tc_offset.size() && f->tc_offset[i0] != SIZE_MAX &&
                            st->n >= g0.k + 5 && g0.post.empty();
    }
    int rc = SV_OK;
    for (size_t oi = 0; oi < ng && rc == SV_OK; ++oi) {
        if (m > 0 && oi == m && !first_reads_small) rc = expand();
        if (rc != SV_OK) break;
        const size_t i = order[oi];
        const bool on_small = oi < m;
        const FusedGate &g = f->gates[i];
        const float *dm = (i < f->mat_offset.size() && f->mat_offset[i] != SIZE_MAX) ? f->d_mats + f->mat_offset[i] : nullptr;
        const void *dt = (f->d_tc && i < f->tc_offset.size() && f->tc_offset[i] != SIZE_MAX)
                             ? static_cast<const char *>(f->d_tc) + f->tc_offset[i] : nullptr;
        if (timings) cudaEventRecord(ev[2 * i], st->stream);
        if (on_small) {
            const FusedGate rg = remap_gate(g, A, a);
            const bool tc = rg.path == SV_PATH_TC_TF32 || rg.path == SV_PATH_TC_BF16X3;
            rc = launch_fused_gate(small, a, rg, dm, tc ? dt : nullptr, st->stream, st->num_sms);
        } else if (st->c128) {
            const double *um = (f->d_mats64 && f->mat64_offset[i] != SIZE_MAX) ? f->d_mats64 + f->mat64_offset[i] : nullptr;
            rc = c128_apply_gate(st, g, um);
        } else if (first_reads_small && oi == m) {
            const uint64_t rest = x & ~A & nmask;
            const TcSource vs{small, nmask & ~amask, rest, (long long)((rest >> 5) << 6)};
            rc = launch_tc_gate(st->d, st->n, g, dt, st->stream, st->num_sms, &vs);
        } else {
            rc = launch_fused_gate(st->d, st->n, g, dm, dt, st->stream, st->num_sms);
        }
        if (timings) cudaEventRecord(ev[2 * i + 1], st->stream);
    }
    if (rc == SV_OK && m > 0 && m == ng) rc = expand();
    if (timings && ng) {
        cudaError_t e = cudaStreamSynchronize(st->stream);
        for (size_t i = 0; i < ng; ++i) {
            float ms = 0.f;
            if (e == cudaSuccess && rc == SV_OK) cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
            const FusedGate &g = f->gates[i];
            timings[i].us = ms * 1000.f;
            timings[i].k = g.k;
            timings[i].path = (m > 0 && (*lazy)[i]) ? SV_PATH_AUTO : g.path;   // AUTO: ran on the small state
            timings[i].flags = (first_reads_small && m < ng && i == order[m]) ? SV_TIMING_SMALL_SOURCE : 0;
            timings[i].target_mask = g.mask;
        }
        for (auto &xv : ev) cudaEventDestroy(xv);
        if (e != cudaSuccess && rc == SV_OK) { set_error("%s: %s", who, cudaGetErrorString(e)); rc = SV_ECUDA; }
        int code = 0;
        if (rc == SV_OK && read_device_errors(&code) == SV_OK && code) {
            set_error("%s: a kernel gave up a bounded wait (device code 0x%x)", who, code);
            rc = SV_ETIMEOUT;
        }
    }
    const int urc = note_fused_use(f, st->stream);   // even after an error: launches may be queued
    return rc != SV_OK ? rc : urc;
}

}  // namespace

extern "C" int sv_apply_fused_gates(sv_state *st, const sv_fused *fc, sv_timing *timings)
{
    clear_error();
    if (!st || !fc) { set_error("sv_apply_fused_gates: NULL argument"); return SV_EINVAL; }
    sv_fused *f = const_cast<sv_fused *>(fc);
    if (f->n != st->n) { set_error("sv_apply_fused_gates: circuit is for %d qubits, state has %d", f->n, st->n); return SV_ESTATE; }
    return apply_core(st, f, timings, nullptr, 0, 0, "sv_apply_fused_gates");
}

extern "C" int sv_init_apply(sv_state *st, uint64_t basis_index, const sv_fused *fc, sv_timing *timings)
{
    clear_error();
    if (!st || !fc) { set_error("sv_init_apply: NULL argument"); return SV_EINVAL; }
    sv_fused *f = const_cast<sv_fused *>(fc);
    if (f->n != st->n) { set_error("sv_init_apply: circuit is for %d qubits, state has %d", f->n, st->n); return SV_ESTATE; }
    if (basis_index >> st->n) { set_error("sv_init_apply: basis index out of range for %d qubits", st->n); return SV_EINVAL; }
    // gates for the small state, in one pass over the circuit: a gate qualifies if no earlier gate
    // left out shares a qubit with it (so it commutes past those) and the qubits named so far, its
    // own included, stay within the limit
    // the light-cone part the fuser placed first (its qubit count), else the default
    const int limit = std::min(f->lazy_limit > 0 ? std::min(f->lazy_limit, kCompactMaxQubits) : kDefaultLazyQubits, st->n - 1);
    std::vector<char> lazy(f->gates.size(), 0);
    uint64_t A = 0, blocked = 0;
    size_t m = 0;
    if (!st->c128)
        for (size_t i = 0; i < f->gates.size(); ++i) {
            const FusedGate &g = f->gates[i];
            // a gate with post-phases runs on the full state, and its phases name qubits outside
            // it: a later gate on those cannot move ahead of it either; so does a swap network
            uint64_t q = g.mask | g.cmask;
            for (const FusedGate::PostTerm &t : g.post) q |= uint64_t(1) << t.q;
            if (!(q & blocked) && __builtin_popcountll(A | q) <= limit && g.post.empty() && g.swaps.empty()) {
                A |= q;
                lazy[i] = 1;
                ++m;
            } else {
                blocked |= q;
            }
        }
    if (m == 0) {
        SV_TRY(sv_init(st, basis_index));
        return apply_core(st, f, timings, nullptr, 0, 0, "sv_init_apply");
    }
    return apply_core(st, f, timings, &lazy, A, basis_index, "sv_init_apply");
}

extern "C" int sv_device_status(void)
{
    clear_error();
    SV_CUDA_TRY(cudaDeviceSynchronize());
    int code = 0;
    SV_TRY(read_device_errors(&code));
    if (code) {
        set_error("a kernel gave up a bounded wait (device code 0x%x)", code);
        return SV_ETIMEOUT;
    }
    return SV_OK;
}

extern "C" void sv_fused_free(sv_fused *f)
{
    if (!f) return;
    if (f->d_buf || f->d_mats64 || !f->use_events.empty()) {
        // only the streams that applied this circuit can still read its images: wait for each
        // one's last launch (its event), then return the buffers to the library's cache
        int cur = -1;
        cudaGetDevice(&cur);
        if (f->device >= 0 && cur != f->device) cudaSetDevice(f->device);
        for (auto &u : f->use_events) {
            cudaEventSynchronize(u.second);
            cudaEventDestroy(u.second);
        }
        f->use_events.clear();
        dev_buffer_put(f->device, f->d_buf, f->d_buf_bytes);
        dev_buffer_put(f->device, f->d_mats64, f->d_mats64_bytes);
        if (f->device >= 0 && cur >= 0 && cur != f->device) cudaSetDevice(cur);
    }
    delete f;
}
