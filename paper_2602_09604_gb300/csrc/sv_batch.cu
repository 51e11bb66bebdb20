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
//     optionally in waves of at most `wave_mb` MB of state so that a wave stays in L2;
//   * or, with `stage_log2` = L set, a tile of one stage of a large circuit: the host cuts the
//     circuit into stages, each a set of gates whose qubits all lie in one set S of L qubits
//     (gates move ahead only past gates on other qubits, so the order of the circuit is kept).
//     The tiles of a stage are the 2^(n-L) sets of amplitudes that agree on the qubits outside
//     S; a CTA loads its tile into shared memory once, applies every gate of the stage there
//     (targets renumbered inside S) and stores it once, so the state crosses memory once per
//     stage instead of once per gate.  S always holds qubits 0-2, so every tile moves in whole
//     32-byte runs.  The first stage writes |0...0> instead of loading.  A tile waits (bounded)
//     for every tile of the previous stage, as the steps above do.
// States use the library's blocked layout (32 reals then 32 imaginaries per 256-byte block).
// The launch can be captured once in a CUDA graph and replayed.
#include <algorithm>
#include <cstdlib>
#include <stdexcept>
#include <array>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sv_internal.h"

using namespace svg;

namespace {

constexpr int kBatchMaxK = 4;
constexpr int kBatchMaxN = 24;   // states up to 2^25 floats: 32-bit offsets

// A fused gate of the batch.  Stage gates may carry a sign run: diagonal gates with entries +-1 on
// one or two qubits (CZ, Z, ...) that come right before the gate and are applied to its inputs:
// amplitude i is negated when gsign + popc(i & zmask) + sum_d popc(i & (i >> dist[d]) & dmask[d])
// is odd (any +-1 diagonal on at most two qubits is such a quadratic form over GF(2)).  k = 0 is a
// sign-only sweep (a run with no gate after it in its stage, or before a 4-qubit gate); k = -2 is
// a register phase and k = -3, -4 are its records (see run_phase).
constexpr int kSignDist = 4;   // distinct qubit distances of the pair terms of one run

struct alignas(16) BGate {
    int k;
    int targets[SV_MAX_K];   // ascending
    int mat_off;             // in float2 units into the matrix table
    int nd;                  // pair-term distances in use
    unsigned gsign;          // 0 or 1
    unsigned zmask;          // single-qubit terms
    unsigned dmask[kSignDist];   // pair terms (a, a + dist[d]): bit a
    int dist[kSignDist];
    unsigned lmask;          // k = -4 (a phase's sign run): the run's form on the window bits alone
};

static_assert(sizeof(BGate) % 16 == 0, "stage gate descriptors are copied 16 bytes at a time");

struct BCirc {
    long long state_off;     // in floats into the arena
    int n;
    int gate_begin;
    int gate_count;
    int done_off;            // large circuits: first completion counter (one per step or stage)
    int stage_begin;         // staged circuits: first stage in the stage table
    int n_stages;
};

// One stage of a staged circuit: its tiles hold the qubits of `lmask` (local qubit i = the i-th
// set bit); its gates (in the stage gate table, naming local qubits) come in chunks whose
// descriptors and matrices fit the shared-memory areas reserved for them.
struct BStage {
    unsigned lmask;          // physical qubits of the tile as it is loaded (as stored, for a first stage)
    int chunk_begin;
    int chunk_count;
    unsigned frame;          // local qubits whose bits the tile holds flipped when its gates end
    int map;                 // store map (the next stage's qubit layout), -1: stored as loaded
};

// A stage tile stored in another qubit layout than it was loaded in (the next stage's): store-local
// index bit j (the order of the store layout, its physical qubits 0-2 first) is load-local bit
// src[j]; the store layout's physical local qubits are lmask; bit j of the tile index lands on
// physical qubit tbit[j].
struct alignas(16) BStoreMap {
    unsigned lmask;
    unsigned char src[16];
    unsigned char tbit[16];
    unsigned pad[3];
};
static_assert(sizeof(BStoreMap) == 48, "store maps are read 16 bytes at a time");

struct BChunk {
    int gate_begin;          // in the stage gate table
    int gate_count;
    int mat_begin;           // the chunk's matrices: one contiguous range of the stage matrix table
    int mat_count;           // (float2 units)
};

constexpr int kStageMatCap = 4096;   // float2 of matrices per chunk (32 KB): 31 three-qubit gates (U and U')
constexpr int kStageGateCap = 64;    // gate descriptors per chunk

// Work item kinds.  A circuit runs as one of them:
//   kWhole  - circuit c entirely in one CTA's shared memory;
//   kSingle - circuit c by one CTA in its global buffer, gate after gate;
//   kTile   - tile `tile` of step `step` of circuit c, in its global buffer (step 0 writes |0...0>,
//             step s >= 1 applies fused gate s-1 to 2^tile_log2 groups);
//   kStage  - tile `tile` of stage `step` of circuit c, through shared memory.
enum : int { kWhole = 0, kSingle = 1, kTile = 2, kStage = 3 };

struct alignas(16) BItem {   // 80 bytes
    int kind;
    int c;
    int step;
    int tile;
    // kStage: what the item needs, copied here so that one 80-byte read starts it (instead of a
    // chain of dependent reads through the circuit, stage and chunk tables)
    int n;
    int done_off;            // the circuit's first completion counter
    int need_prev;           // tiles of the previous stage (the wait's target)
    unsigned lmask;          // the stage's local qubits
    long long state_off;
    int chunk_begin;
    int chunk_count;
    BChunk ch0;              // the stage's first chunk (empty when it has none)
    unsigned frame;          // the stage's frame (see BStage): the tile stores local index l ^ frame
    int map;                 // the stage's store map, -1: stored as loaded
    int pad[2];
};
static_assert(sizeof(BItem) == 80, "work items are read 16 bytes at a time");

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

// 16-byte asynchronous copy global -> shared (cached in L2 only), and the wait for all of them
__device__ __forceinline__ void cp_async16(float *dst_smem, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// x's bits deposited, lowest first, into the set bits of mask
__device__ __host__ __forceinline__ unsigned deposit_bits(unsigned x, unsigned mask)
{
    unsigned r = 0u;
    for (unsigned m = mask; m != 0u; m &= m - 1u) {
        if (x & 1u) r |= m & (0u - m);
        x >>= 1;
    }
    return r;
}

// The sign run of g at local index i: true when the amplitude is negated.
__device__ __forceinline__ bool sign_odd(const BGate &g, unsigned i)
{
    unsigned p = g.gsign + (unsigned)__popc(i & g.zmask);
#pragma unroll
    for (int d = 0; d < kSignDist; ++d)
        if (d < g.nd) p += (unsigned)__popc(i & (i >> g.dist[d]) & g.dmask[d]);
    return (p & 1u) != 0u;
}

// A sign-only sweep over a 2^n-amplitude state in shared memory (four amplitudes per thread).
__device__ void sign_sweep(float *S, int n, const BGate &g)
{
    const unsigned count = n >= 2 ? (1u << n) >> 2 : 1u;
    for (unsigned q = threadIdx.x; q < count; q += blockDim.x) {
        const unsigned i0 = q << 2;
        const unsigned o = ((i0 >> 5) << 6) | (i0 & 31u);
        float4 re = *reinterpret_cast<float4 *>(S + o), im = *reinterpret_cast<float4 *>(S + o + 32);
        float *r = &re.x, *m = &im.x;
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if ((n >= 2 || (unsigned)v < (1u << n)) && sign_odd(g, i0 + (unsigned)v)) {
                r[v] = -r[v];
                m[v] = -m[v];
            }
        *reinterpret_cast<float4 *>(S + o) = re;
        *reinterpret_cast<float4 *>(S + o + 32) = im;
    }
}

// Register phases.  A phase record (k = -2; targets[0] = Q0, targets[1] = the number of records
// that follow it) applies its records, in order, to a 2^L-amplitude tile in shared memory, every
// thread holding in registers the 32 amplitudes that differ only in the window of local qubits
// Q0..Q0+4 (slot m: window bits m):
//   k = -3: a 2x2 matrix on window qubit targets[0] (U at mat_off, row-major, then X U X);
//   k = -5: a real 2x2 matrix on window qubit targets[0] (R, then X R X: four floats each);
//   k = -8: T(t_r) = (1, -t_r; t_r, 1) on all five window qubits (pairs t_r, -t_r), one
//           straight-line pass with no branch per gate: two multiply-adds per pair and component;
//   k = -6: a diagonal over the tile's qubits that factors over them: amplitude i times
//           C * prod_{q : i_q = 1} w_q, from tables at mat_off: 32 entries over the window bits,
//           32 over the thread's first five non-window bits (times C), 16 over its next four;
//   k = -4: a sign run (the fields of a sign run; lmask = the run's form on the window bits alone,
//           targets[r] = the pair partners of window qubit r) -- the amplitudes it negates.
// One shared-memory round trip then serves every gate and sign run of the phase, in registers whose
// indices are compile-time constants.  Q0 >= 5: the lanes of a warp take consecutive in-block
// positions, scalar accesses without bank conflicts.  Q0 = 0: a thread holds one block and reads it
// as eight 16-byte chunks in the order j ^ k (k = its block index mod 8, so the eight threads of a
// shared-memory access phase meet eight different chunks); slot m then holds window position
// m ^ 4k, i.e. local index bp ^ m with bp = base | 4k, and a gate on a window qubit whose bit is
// set in 4k runs with its two rows and columns exchanged (X U X).
//
// Sign runs in registers: the run's quadratic form q over GF(2) splits as
// q(bp ^ y) = q(bp) ^ q0(y) ^ sum_r y_r * parity(bp & N_r) for y in the window (q0: q without the
// constant), so a thread forms the 32 slot signs as one mask: the host's table of q0 on the window,
// flipped as a whole by q(bp) and on the slots with bit r set by the parity of bp's partners of r.
__host__ __device__ constexpr unsigned slot_bit(int r)   // slots m with bit r set
{
    return r == 0 ? 0xAAAAAAAAu : r == 1 ? 0xCCCCCCCCu : r == 2 ? 0xF0F0F0F0u : r == 3 ? 0xFF00FF00u : 0xFFFF0000u;
}
constexpr int kPhaseMaxRecords = 48;   // records of one phase (a chunk holds it whole)

template <int R>
__device__ __forceinline__ void slot_gate(float (&xr)[32], float (&xi)[32], const float4 p, const float4 q)
{
    // p = (u00, u01), q = (u10, u11) as (re, im) pairs
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        if ((m >> R) & 1) continue;
        const int m1 = m | (1 << R);
        const float ar = xr[m], ai = xi[m], br = xr[m1], bi = xi[m1];
        xr[m] = fmaf(p.x, ar, fmaf(-p.y, ai, fmaf(p.z, br, -p.w * bi)));
        xi[m] = fmaf(p.x, ai, fmaf(p.y, ar, fmaf(p.z, bi, p.w * br)));
        xr[m1] = fmaf(q.x, ar, fmaf(-q.y, ai, fmaf(q.z, br, -q.w * bi)));
        xi[m1] = fmaf(q.x, ai, fmaf(q.y, ar, fmaf(q.z, bi, q.w * br)));
    }
}

template <int R>
__device__ __forceinline__ void slot_tan(float (&xr)[32], float (&xi)[32], const float t)
{
    // (a, b) -> (a - t b, t a + b): two multiply-adds per component
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        if ((m >> R) & 1) continue;
        const int m1 = m | (1 << R);
        const float ar = xr[m], ai = xi[m], br = xr[m1], bi = xi[m1];
        xr[m] = fmaf(-t, br, ar);
        xi[m] = fmaf(-t, bi, ai);
        xr[m1] = fmaf(t, ar, br);
        xi[m1] = fmaf(t, ai, bi);
    }
}

template <int R>
__device__ __forceinline__ void slot_rot(float (&xr)[32], float (&xi)[32], const float4 u)
{
    // u = (a00, a01, a10, a11), real
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        if ((m >> R) & 1) continue;
        const int m1 = m | (1 << R);
        const float ar = xr[m], ai = xi[m], br = xr[m1], bi = xi[m1];
        xr[m] = fmaf(u.x, ar, u.y * br);
        xi[m] = fmaf(u.x, ai, u.y * bi);
        xr[m1] = fmaf(u.z, ar, u.w * br);
        xi[m1] = fmaf(u.z, ai, u.w * bi);
    }
}

template <int Q0>
__device__ void run_phase(float *S, int L, const BGate *ops, int nops, const float2 *U, int mb)
{
    static_assert(Q0 == 0 || Q0 >= 5, "windows start at qubit 0 or above the block");
    const unsigned nb = 1u << (L - 5);
    for (unsigned it = threadIdx.x; it < nb; it += blockDim.x) {
        unsigned base, f = 0u;
        if constexpr (Q0 == 0) {
            base = it << 5;
            f = (it & 7u) << 2;
        } else {
            base = (it & ((1u << Q0) - 1u)) | ((it >> Q0) << (Q0 + 5));
        }
        const unsigned bp = base | f;
        const unsigned ob = ((base >> 5) << 6) | (base & 31u);
        float xr[32], xi[32];
        if constexpr (Q0 == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const unsigned o = ob + ((unsigned)(4 * j) ^ f);
                const float4 re = *reinterpret_cast<const float4 *>(S + o), im = *reinterpret_cast<const float4 *>(S + o + 32);
                xr[4 * j] = re.x; xr[4 * j + 1] = re.y; xr[4 * j + 2] = re.z; xr[4 * j + 3] = re.w;
                xi[4 * j] = im.x; xi[4 * j + 1] = im.y; xi[4 * j + 2] = im.z; xi[4 * j + 3] = im.w;
            }
        } else {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                xr[m] = S[ob + ((unsigned)m << (Q0 + 1))];
                xi[m] = S[ob + 32 + ((unsigned)m << (Q0 + 1))];
            }
        }
        for (int t = 0; t < nops; ++t) {
            const BGate &g = ops[t];
            if (g.k == -8) {
                // T(t_r) = (1, -t_r; t_r, 1) on all five window bits, straight-line (t = 0 where the
                // layer has none): the pairs (t_r, -t_r) at mat_off, the second for a flipped bit
                const float *tp = reinterpret_cast<const float *>(U + (g.mat_off - mb));
                slot_tan<0>(xr, xi, tp[0]);
                slot_tan<1>(xr, xi, tp[2]);
                slot_tan<2>(xr, xi, tp[4 + (int)((f >> 2) & 1u)]);
                slot_tan<3>(xr, xi, tp[6 + (int)((f >> 3) & 1u)]);
                slot_tan<4>(xr, xi, tp[8 + (int)((f >> 4) & 1u)]);
            } else if (g.k == -5) {
                const int r = g.targets[0];
                const unsigned flip = Q0 == 0 ? (f >> r) & 1u : 0u;
                const float4 u = *reinterpret_cast<const float4 *>(U + (g.mat_off - mb) + 2 * (int)flip);
                switch (r) {
                case 0: slot_rot<0>(xr, xi, u); break;
                case 1: slot_rot<1>(xr, xi, u); break;
                case 2: slot_rot<2>(xr, xi, u); break;
                case 3: slot_rot<3>(xr, xi, u); break;
                default: slot_rot<4>(xr, xi, u); break;
                }
            } else if (g.k == -6) {
                // diagonal: the thread's factor (its non-window bits are it) times the slot's
                const float2 *T = U + (g.mat_off - mb);
                const float2 ta = T[32 + (it & 31u)], tb = T[64 + (it >> 5)];
                const float tr = ta.x * tb.x - ta.y * tb.y, ti = ta.x * tb.y + ta.y * tb.x;
#pragma unroll
                for (int m = 0; m < 32; m += 2) {
                    // entries m ^ f and (m + 1) ^ f are adjacent (f is a multiple of 4): one 16-byte read
                    const float4 sl = *reinterpret_cast<const float4 *>(T + ((unsigned)m ^ f));
                    asm volatile("" ::: "memory");   // one table read at a time: no hoisting into registers
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float sx = h ? sl.z : sl.x, sy = h ? sl.w : sl.y;
                        const float fr = tr * sx - ti * sy, fi = tr * sy + ti * sx;
                        const float ar = xr[m + h], ai = xi[m + h];
                        xr[m + h] = ar * fr - ai * fi;
                        xi[m + h] = ar * fi + ai * fr;
                    }
                }
            } else if (g.k == -3) {
                const int r = g.targets[0];
                const unsigned flip = Q0 == 0 ? (f >> r) & 1u : 0u;
                const float4 *u = reinterpret_cast<const float4 *>(U + (g.mat_off - mb) + 4 * (int)flip);
                const float4 p = u[0], q = u[1];
                switch (r) {
                case 0: slot_gate<0>(xr, xi, p, q); break;
                case 1: slot_gate<1>(xr, xi, p, q); break;
                case 2: slot_gate<2>(xr, xi, p, q); break;
                case 3: slot_gate<3>(xr, xi, p, q); break;
                default: slot_gate<4>(xr, xi, p, q); break;
                }
            } else {
                unsigned par = g.gsign + (unsigned)__popc(bp & g.zmask);
                for (int d = 0; d < g.nd; ++d) par += (unsigned)__popc(bp & (bp >> g.dist[d]) & g.dmask[d]);
                unsigned sm = g.lmask ^ (0u - (par & 1u));
#pragma unroll
                for (int r = 0; r < 5; ++r) sm ^= (0u - ((unsigned)__popc(bp & (unsigned)g.targets[r]) & 1u)) & slot_bit(r);
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    const unsigned sb = (sm << (31 - m)) & 0x80000000u;
                    xr[m] = __uint_as_float(__float_as_uint(xr[m]) ^ sb);
                    xi[m] = __uint_as_float(__float_as_uint(xi[m]) ^ sb);
                }
            }
        }
        if constexpr (Q0 == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const unsigned o = ob + ((unsigned)(4 * j) ^ f);
                *reinterpret_cast<float4 *>(S + o) = make_float4(xr[4 * j], xr[4 * j + 1], xr[4 * j + 2], xr[4 * j + 3]);
                *reinterpret_cast<float4 *>(S + o + 32) = make_float4(xi[4 * j], xi[4 * j + 1], xi[4 * j + 2], xi[4 * j + 3]);
            }
        } else {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                S[ob + ((unsigned)m << (Q0 + 1))] = xr[m];
                S[ob + 32 + ((unsigned)m << (Q0 + 1))] = xi[m];
            }
        }
    }
}

// The records ops[0, nops) of a phase whose window starts at local qubit q0 (0, 5 or L - 5 for
// tiles of L = 10..14 qubits: the start picks the compiled form); U holds the chunk's matrices,
// the first at offset mb of the stage matrix table.  Not inlined: the phase's 64 amplitude
// registers get the register file to themselves, the caller's state is saved once per call.
__device__ __noinline__ void apply_phase(float *S, int L, int q0, const BGate *ops, int nops, const float2 *U, int mb)
{
    switch (q0) {
    case 0: run_phase<0>(S, L, ops, nops, U, mb); break;
    case 5: run_phase<5>(S, L, ops, nops, U, mb); break;
    case 6: run_phase<6>(S, L, ops, nops, U, mb); break;
    case 7: run_phase<7>(S, L, ops, nops, U, mb); break;
    case 8: run_phase<8>(S, L, ops, nops, U, mb); break;
    default: run_phase<9>(S, L, ops, nops, U, mb); break;
    }
}

// Apply one fused gate of K qubits to groups [g_begin, g_end) of the state S (shared or global)
// of n <= 24 qubits with all threads of the CTA; U (float2, row-major 2^K x 2^K) is in shared
// memory.  A thread takes V consecutive groups at a time: with no target below log2(V) their
// amplitudes are V consecutive positions of a block, moved with one V-wide access (and each
// matrix element read once serves V groups).  Offsets are 32-bit and recomputed for the stores.
//
// XS (S in shared memory): with m targets below qubit 5, the 32 consecutive groups of one
// shared-memory access phase lie in 2^m blocks, and for a fixed local index j all of them sit at
// positions with the same low-target bits, so two blocks' halves would meet in the same banks.
// Each thread therefore takes its amplitudes in the order j ^ s, s = the index of its block among
// the 2^m: it holds x'[j] = x[j ^ s], forms y'[r] = sum_j U[r ^ s][j ^ s] x'[j] = y[r ^ s] and
// stores it at the place of r ^ s.  The result is the same; the phase's accesses cover every bank
// once.
template <int K, int V, bool L2ONLY, bool XS, bool SG>
__device__ void apply_in_cta(float *S, const BGate &g, const float2 *__restrict__ U, unsigned g_begin, unsigned g_end)
{
    constexpr int D = 1 << K;
    unsigned bit[K], obit[K];   // target bit of the index, and of the blocked-layout float offset
    int nlow = 0;
#pragma unroll
    for (int b = 0; b < K; ++b) {
        bit[b] = 1u << g.targets[b];
        obit[b] = g.targets[b] < 5 ? bit[b] : bit[b] << 1;
        nlow += g.targets[b] < 5;
    }
    const unsigned fshift = 5u - (unsigned)nlow, smask = (1u << nlow) - 1u;
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
        unsigned s = 0u;   // XS: this thread's local-index offset (bits of the low targets)
        if constexpr (XS) {
            s = ((it * V) >> fshift) & smask;
#pragma unroll
            for (int b = 0; b < K; ++b) base |= ((s >> b) & 1u) ? bit[b] : 0u;   // base of index s
        }
        // the float offset ((i >> 5) << 6) | (i & 31) moves index bits without mixing them, so
        // the offset of index j ^ s is the base's offset with the targets' offset bits flipped
        const unsigned obase = ((base >> 5) << 6) | (base & 31u);
        float xr[D][V], xi[D][V];
#pragma unroll
        for (int j = 0; j < D; ++j) {
            unsigned o = obase;
#pragma unroll
            for (int b = 0; b < K; ++b)
                if ((j >> b) & 1) o ^= obit[b];   // index j ^ s (plain j when s = 0)
            // L2ONLY: other CTAs wrote these, so read through L2 rather than a stale L1 line
            ld_v<V, L2ONLY>(S + o, xr[j]);
            ld_v<V, L2ONLY>(S + o + 32, xi[j]);
            if constexpr (SG && K <= 3) {   // stage gates: the sign run before this gate, on its inputs
                if (g.nd | g.zmask | g.gsign) {
                    unsigned ij = base;   // index of member j (j ^ s in the XS order) of group v = 0
#pragma unroll
                    for (int b = 0; b < K; ++b)
                        if ((j >> b) & 1) ij ^= bit[b];
#pragma unroll
                    for (int v = 0; v < V; ++v)
                        if (sign_odd(g, ij + (unsigned)v)) {
                            xr[j][v] = -xr[j][v];
                            xi[j][v] = -xi[j][v];
                        }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
            float yr[V], yi[V];
#pragma unroll
            for (int v = 0; v < V; ++v) yr[v] = yi[v] = 0.f;
            // row r ^ s, two entries per 16-byte read: entries (j ^ s, (j + 1) ^ s) for even j are
            // the pair at (j ^ s) & ~1 of U when s is even, and of the pair-swapped copy U' (stored
            // right after U) when s is odd
            const float4 *Ur = reinterpret_cast<const float4 *>(Ui + ((s & 1u) ? D * D : 0) + ((unsigned)r ^ s) * D);
#pragma unroll
            for (int jp = 0; jp < D / 2; ++jp) {
                const float4 q = Ur[(unsigned)jp ^ (s >> 1)];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 2 * jp + h;
                    const float ux = h ? q.z : q.x, uy = h ? q.w : q.y;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        yr[v] = fmaf(ux, xr[j][v], yr[v]);
                        yr[v] = fmaf(uy, -xi[j][v], yr[v]);
                        yi[v] = fmaf(ux, xi[j][v], yi[v]);
                        yi[v] = fmaf(uy, xr[j][v], yi[v]);
                    }
                }
            }
            unsigned o = obase;
#pragma unroll
            for (int b = 0; b < K; ++b)
                if ((r >> b) & 1) o ^= obit[b];
            st_v<V>(S + o, yr);
            st_v<V>(S + o + 32, yi);
        }
    }
}

// V: 4 when no target is below qubit 2, 2 when none is qubit 0, else 1; never more than the
// 2^(n-K) groups.  WIDE (CTAs of at most 256 threads, up to 255 registers a thread) allows K = 4
// with V > 1; with 512-thread CTAs (128 registers) K = 4 keeps V = 1, whose 2^5 inputs per group
// already fill the budget.
template <bool L2ONLY, bool WIDE, bool XS, bool SG>
__device__ void apply_gate_cta(float *S, int n, const BGate &g, const float2 *U, unsigned g_begin, unsigned g_end)
{
    const int t0 = g.targets[0];   // ascending
    int v = t0 >= 2 ? 4 : (t0 == 1 ? 2 : 1);
    if (g.k == 4 && !WIDE) v = 1;
    while (v > 1 && (1 << (n - g.k)) < v) v >>= 1;
#define SV_BATCH_CASE(KK)                                                             \
    case KK:                                                                          \
        if (v == 4) apply_in_cta<KK, 4, L2ONLY, XS, SG>(S, g, U, g_begin, g_end);         \
        else if (v == 2) apply_in_cta<KK, 2, L2ONLY, XS, SG>(S, g, U, g_begin, g_end);    \
        else apply_in_cta<KK, 1, L2ONLY, XS, SG>(S, g, U, g_begin, g_end);                \
        break;
    switch (g.k) {
    SV_BATCH_CASE(1)
    SV_BATCH_CASE(2)
    SV_BATCH_CASE(3)
    default:
        if constexpr (WIDE) {
            if (v == 4) apply_in_cta<4, 4, L2ONLY, XS, SG>(S, g, U, g_begin, g_end);
            else if (v == 2) apply_in_cta<4, 2, L2ONLY, XS, SG>(S, g, U, g_begin, g_end);
            else apply_in_cta<4, 1, L2ONLY, XS, SG>(S, g, U, g_begin, g_end);
        } else {
            apply_in_cta<4, 1, L2ONLY, XS, SG>(S, g, U, g_begin, g_end);
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
    const BStage *stages;    // staged circuits: stage table
    const BChunk *chunks;    // their gate chunks
    const BGate *sgates;     // stage gates (local targets)
    const float2 *smats;     // their matrices
    const BStoreMap *smaps;  // stage tiles stored in another layout
    int mat_cap;             // float2 of the shared-memory matrix area (>= 4^kBatchMaxK)
    int gate_cap;            // gate descriptors of the shared-memory descriptor area
    int *sync;         // [0] queue head, [1] abort flag, [2 + i] completion counter i
    const int *need;   // tiles of each counted step or stage
    int *err;          // library-wide device error word
    int tile_log2;
    int stage_log2;
};


// Bounded wait (thread 0) until counter d reaches want; false when it gave up or another CTA
// already did (the abort flag), after raising the abort flag and the error word.
__device__ bool wait_count(const BatchArgs &A, const int *d, int want)
{
    long long spin = 0;
    while (*(const volatile int *)d < want) {
        if (*(volatile int *)(A.sync + 1) || ++spin > kSpinLimit) {
            atomicExch(A.sync + 1, 1);
            atomicCAS(A.err, 0, kBatchErrCode);
            return false;
        }
        __nanosleep(128);
    }
    __threadfence();   // acquire: the counted tiles' writes before this tile's reads
    return true;
}

// U (row-major) into sU[0, 4^k) and its pair-swapped copy U'[r][j] = U[r][j ^ 1] into
// sU[4^k, 2 * 4^k) (read by threads whose XOR order s is odd)
__device__ __forceinline__ void stage_matrix(float2 *sU, const float2 *mats, const BGate &g)
{
    const int dd = 1 << (2 * g.k);
    for (int i = threadIdx.x; i < dd; i += blockDim.x) {
        const float2 u = mats[g.mat_off + i];
        sU[i] = u;
        sU[dd + (i ^ 1)] = u;
    }
}

__device__ __forceinline__ void zero_floats(float *S, long long f0, long long f1)
{
    for (long long i = f0 / 4 + threadIdx.x; i < f1 / 4; i += blockDim.x)
        reinterpret_cast<float4 *>(S)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Three compiled forms: <256, 1> CTAs of at most 256 threads with up to 255 registers a thread
// (WIDE: 4-qubit gates may move several groups per access), <512, 1> and <256, 2> (two CTAs on an
// SM: 128 registers a thread, so that one CTA's loads, waits and barriers overlap the other's
// arithmetic).
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) batch_kernel(BatchArgs A)
{
    extern __shared__ __align__(16) float smem[];
    float2 *sU = reinterpret_cast<float2 *>(smem);                  // matrix area: A.mat_cap complex
    BGate *sG = reinterpret_cast<BGate *>(smem + 2 * A.mat_cap);     // staged: a chunk's descriptors
    float *sS = smem + 2 * A.mat_cap + A.gate_cap * (int)(sizeof(BGate) / 4);   // circuit state or tile
    __shared__ int ok;
    __shared__ int sIt[2];        // item index of each slot
    __shared__ BItem sWb[2];      // the current item and the next one (fetched ahead); fields are
                                  // read where used (no long-lived registers)
    __shared__ unsigned sT[96];   // staged tiles: deposits of local index bits 3-8 ([0, 64)) and 9-13
    __shared__ BStoreMap sMap;    // a stage tile stored in another layout: its map
    __shared__ unsigned short sP[256];   // and store-local -> load-local index, bits 0-6 ([0, 128)) and 7-13
    // a stage chunk's gate descriptors and matrices into shared memory by asynchronous 16-byte copies
    auto load_chunk = [&](const BChunk &c) {
        const float *src = reinterpret_cast<const float *>(A.sgates + c.gate_begin);
        float *dst = reinterpret_cast<float *>(sG);
        const int nv = c.gate_count * (int)(sizeof(BGate) / 16);
        for (int i = threadIdx.x; i < nv; i += blockDim.x) cp_async16(dst + 4 * i, src + 4 * i);
        const float *ms = reinterpret_cast<const float *>(A.smats + c.mat_begin);
        float *md = reinterpret_cast<float *>(sU);
        for (int i = threadIdx.x; i < (c.mat_count + 1) / 2; i += blockDim.x) cp_async16(md + 4 * i, ms + 4 * i);
    };
    // (thread 0) the next item from the queue into slot s: its index, and its record by asynchronous
    // copies.  Taking an item ahead keeps the list order's guarantee: the earliest unfinished item
    // is never one held ahead (the item its CTA works on is earlier and unfinished), so it runs and
    // waits only on finished items.
    auto fetch = [&](int s) {
        const int nx = (int)atomicAdd(reinterpret_cast<unsigned *>(A.sync), 1u);
        sIt[s] = nx;
        if (nx < A.n_items)
            for (int v = 0; v < (int)(sizeof(BItem) / 16); ++v)
                cp_async16(reinterpret_cast<float *>(&sWb[s]) + 4 * v, reinterpret_cast<const float *>(A.items + nx) + 4 * v);
    };
    int slot = 0;
    if (threadIdx.x == 0) {
        fetch(0);
        cp_async_wait_all();
    }
    __syncthreads();
    for (;;) {
        if (sIt[slot] >= A.n_items) break;
        const BItem &W = sWb[slot];
        if (W.kind == kStage) {
            // (the tile's pointers and bits are formed again from the item where they are used, so
            // that nothing of them stays live in registers across the phases)
            const int L = W.n < A.stage_log2 ? W.n : A.stage_log2;   // tile qubits (>= 8)
            auto tile_bits = [&]() { return deposit_bits((unsigned)W.tile, ((1u << W.n) - 1u) & ~W.lmask); };
            // the first chunk's copy overlaps the wait
            BChunk ch = W.ch0;
            if (W.chunk_count > 0) load_chunk(ch);
            if (W.map >= 0 && threadIdx.x < (int)(sizeof(BStoreMap) / 16))
                cp_async16(reinterpret_cast<float *>(&sMap) + 4 * threadIdx.x,
                           reinterpret_cast<const float *>(A.smaps + W.map) + 4 * threadIdx.x);
            if (threadIdx.x == 0) ok = W.step == 0 || wait_count(A, A.sync + 2 + W.done_off + W.step - 1, W.need_prev);
            for (unsigned i = threadIdx.x; i < 96u; i += blockDim.x)
                sT[i] = i < 64u ? deposit_bits(i << 3, W.lmask) : deposit_bits((i - 64u) << 9, W.lmask);
            cp_async_wait_all();
            __syncthreads();
            if (!ok) break;
            // local index l -> global index: bits 0-2 stay (S holds qubits 0-2), the rest deposit
            // into S's higher qubits, the tile's bits fill the others.  A thread moves four
            // amplitudes (16 bytes of real and of imaginary parts) at a time; eight consecutive
            // local indices are one 32-byte run in global memory.  The tile loads by asynchronous
            // copies straight into shared memory (through L2: other CTAs wrote it in the previous
            // stage), all of a thread's copies in flight at once, and the next item is taken
            // from the queue meanwhile.
            const int nq = 1 << (L - 2);
            auto gofs = [&](unsigned l, unsigned tb) -> unsigned {
                const unsigned gi = (l & 7u) | sT[(l >> 3) & 63u] | sT[64 + (l >> 9)] | tb;
                return ((gi >> 5) << 6) | (gi & 31u);
            };
            if (W.step == 0) {
                zero_floats(sS, 0, 2ll << L);
                __syncthreads();
                if (W.tile == 0 && threadIdx.x == 0) sS[0] = 1.f;
            } else {
                const float *G = A.arena + W.state_off;
                const unsigned tb = tile_bits();
                for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                    const unsigned l = (unsigned)q << 2, lo = ((l >> 5) << 6) | (l & 31u);
                    const unsigned go = gofs(l, tb);
                    cp_async16(sS + lo, G + go);
                    cp_async16(sS + lo + 32, G + go + 32);
                }
            }
            if (threadIdx.x == 0) fetch(slot ^ 1);
            cp_async_wait_all();
            __syncthreads();
            for (int ci = 0; ci < W.chunk_count; ++ci) {
                if (ci > 0) {   // the previous chunk's last gate ended with a barrier
                    ch = A.chunks[W.chunk_begin + ci];
                    load_chunk(ch);
                    cp_async_wait_all();
                    __syncthreads();
                }
                for (int gi = 0; gi < ch.gate_count; ++gi) {
                    const BGate &g = sG[gi];   // read in place: the sign fields stay in shared memory
                    if (g.k < 0) {   // a phase and its records
                        const int q0 = g.targets[0];
                        apply_phase(sS, L, q0, sG + gi + 1, g.targets[1], sU, ch.mat_begin);
                        gi += g.targets[1];
                        // windows at 0 and 5: a warp holds the same 1024 amplitudes (local bits 0-9)
                        // in both, so when the next record of this chunk is such a phase too, the
                        // warp reads only what it wrote itself
                        if (q0 <= 5 && gi + 1 < ch.gate_count && sG[gi + 1].k == -2 && sG[gi + 1].targets[0] <= 5) {
                            __syncwarp();
                            continue;
                        }
                    } else if (g.k == 0) sign_sweep(sS, L, g);
                    else apply_gate_cta<false, (MAXT <= 256 && MINB == 1), true, true>(sS, L, g, sU + (g.mat_off - ch.mat_begin), 0u, 1u << (L - g.k));
                    __syncthreads();   // this gate's writes before the next gate's reads
                }
            }
            if (W.map >= 0) {
                // stored in the next stage's layout: store-local index s (that layout's physical
                // qubits 0-2 first) is load-local index P(s), held at P(s) ^ frame; four amplitudes
                // consecutive in the store layout are gathered one by one and written as a float4
                for (int i = threadIdx.x; i < 256; i += blockDim.x) {
                    unsigned v = 0u;
                    for (int j = 0; j < 7; ++j) {
                        const int sj = (i >> 7) * 7 + j;
                        if (sj < L && ((i >> j) & 1)) v |= 1u << sMap.src[sj];
                    }
                    sP[i] = (unsigned short)v;
                }
                for (unsigned i = threadIdx.x; i < 96u; i += blockDim.x)
                    sT[i] = i < 64u ? deposit_bits(i << 3, sMap.lmask) : deposit_bits((i - 64u) << 9, sMap.lmask);
                __syncthreads();
                float *G = A.arena + W.state_off;
                unsigned tb = 0u;
                for (int j = 0; j < W.n - L; ++j) tb |= (((unsigned)W.tile >> j) & 1u) << sMap.tbit[j];
                const unsigned fr = W.frame, c1 = 1u << sMap.src[0], c2 = 1u << sMap.src[1];
                for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                    const unsigned s0 = (unsigned)q << 2;
                    const unsigned lb = ((unsigned)sP[s0 & 127u] | (unsigned)sP[128 + (s0 >> 7)]) ^ fr;
                    float re[4], im[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const unsigned l = lb ^ ((j & 1) ? c1 : 0u) ^ ((j & 2) ? c2 : 0u);
                        const unsigned o = ((l >> 5) << 6) | (l & 31u);
                        re[j] = sS[o];
                        im[j] = sS[o + 32];
                    }
                    const unsigned go = gofs(s0, tb);
                    *reinterpret_cast<float4 *>(G + go) = make_float4(re[0], re[1], re[2], re[3]);
                    *reinterpret_cast<float4 *>(G + go + 32) = make_float4(im[0], im[1], im[2], im[3]);
                }
            } else {
                // the tile holds amplitude l at l ^ frame: its four amplitudes l..l+3 are the float4
                // at (l ^ frame) & ~3, permuted by the frame's two low bits
                float *G = A.arena + W.state_off;
                const unsigned tb = tile_bits(), fr = W.frame;
                auto perm = [fr](const float4 v) {
                    switch (fr & 3u) {
                    case 0: return v;
                    case 1: return make_float4(v.y, v.x, v.w, v.z);
                    case 2: return make_float4(v.z, v.w, v.x, v.y);
                    default: return make_float4(v.w, v.z, v.y, v.x);
                    }
                };
                for (int q = threadIdx.x; q < nq; q += blockDim.x) {
                    const unsigned l = (unsigned)q << 2, ls = l ^ (fr & ~3u), lo = ((ls >> 5) << 6) | (ls & 31u);
                    const unsigned go = gofs(l, tb);
                    *reinterpret_cast<float4 *>(G + go) = perm(*reinterpret_cast<const float4 *>(sS + lo));
                    *reinterpret_cast<float4 *>(G + go + 32) = perm(*reinterpret_cast<const float4 *>(sS + lo + 32));
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();   // release: this tile's writes before the count
                atomicAdd(A.sync + 2 + W.done_off + W.step, 1);
            }
            slot ^= 1;
            continue;
        }
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
                if (W.kind == kWhole) apply_gate_cta<false, (MAXT <= 256 && MINB == 1), true, false>(S, C.n, g, sU, 0u, 1u << (C.n - g.k));
                else apply_gate_cta<false, (MAXT <= 256 && MINB == 1), false, false>(S, C.n, g, sU, 0u, 1u << (C.n - g.k));
                __syncthreads();
            }
            if (W.kind == kWhole) {
                float4 *dst = reinterpret_cast<float4 *>(G);
                for (long long i = threadIdx.x; i < nf / 4; i += blockDim.x) dst[i] = reinterpret_cast<const float4 *>(S)[i];
                __syncthreads();
            }
        } else {
            // one tile of one step of a large circuit
            int *done = A.sync + 2 + C.done_off;
            if (threadIdx.x == 0) ok = W.step == 0 || wait_count(A, done + W.step - 1, A.need[C.done_off + W.step - 1]);
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
                apply_gate_cta<true, (MAXT <= 256 && MINB == 1), false, false>(G, C.n, g, sU, g0, g1);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();   // release: this tile's writes before the count
                atomicAdd(done + W.step, 1);
            }
        }
        // the next item (the other kinds take it here, after their work)
        if (threadIdx.x == 0) {
            fetch(slot ^ 1);
            cp_async_wait_all();
        }
        __syncthreads();
        slot ^= 1;
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
    std::vector<const FusedGate *> src;   // per entry of hg: the fused gate it came from
    BCirc *d_circ = nullptr;
    BGate *d_gates = nullptr;
    float2 *d_mats = nullptr;
    // work list for the options it was built for
    BItem *d_items = nullptr;
    int *d_need = nullptr;
    int *d_sync = nullptr;
    BStage *d_stages = nullptr;      // staged circuits (stage_log2 > 0): stages, chunks, gates, matrices
    BChunk *d_chunks = nullptr;
    BGate *d_sgates = nullptr;
    float2 *d_smats = nullptr;
    BStoreMap *d_smaps = nullptr;
    int *d_err = nullptr;            // library's device error word (not owned)
    int n_items = 0;
    int n_counters = 0;
    sv_batch_info info{};            // what the current list holds
    int list_cfg[7] = {-1, -1, -1, -1, -1, -1, -1};   // smem_max_n, split_min_n, tile_log2, wave_mb, stage_log2, stage_k, stage_layers
    bool stall = false;              // test hook: first split step counts one tile too many
    bool list_stall = false;
    sv_batch_opts opts{};
    cudaGraphExec_t graph = nullptr;
    int graph_cfg[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
};

namespace {

size_t state_bytes(int n) { return sizeof(float) * (size_t)state_floats(n); }

// shared-memory areas: matrices, gate descriptors, then the state of a whole circuit or a tile
int mat_cap(const sv_batch_opts &o) { return o.stage_log2 > 0 ? kStageMatCap : 2 << (2 * kBatchMaxK); }
int gate_cap(const sv_batch_opts &o) { return o.stage_log2 > 0 ? kStageGateCap : 0; }

size_t smem_bytes(const sv_batch_opts &o)
{
    const size_t whole = o.smem_max_n > 0 ? state_bytes(o.smem_max_n) : 0;
    const size_t tile = o.stage_log2 > 0 ? state_bytes(o.stage_log2) : 0;
    return sizeof(float2) * (size_t)mat_cap(o) + sizeof(BGate) * (size_t)gate_cap(o) + std::max(whole, tile);
}

constexpr int kStageMinN = 8;         // staged circuits have at least this many qubits

// A diagonal gate with entries +-1 on one or two qubits, as its signs bit[x] (1 = -1) over the
// local index x; false for any other gate.
bool sign_pattern(const FusedGate &g, int (&bits)[4])
{
    if (g.cmask || g.k < 1 || g.k > 2) return false;
    const int D = 1 << g.k;
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            const cplx u = g.mat[(size_t)(r * D + c)];
            if (r != c) {
                if (std::abs(u) > 1e-12) return false;
            } else if (std::abs(u - 1.0) <= 1e-12) {
                bits[r] = 0;
            } else if (std::abs(u + 1.0) <= 1e-12) {
                bits[r] = 1;
            } else {
                return false;
            }
        }
    return true;
}

// Product of sign gates as a quadratic form over GF(2) in the local index bits (see BGate).
struct SignRun {
    unsigned gsign = 0, zmask = 0;
    std::vector<std::pair<int, unsigned>> pairs;   // (distance, mask of the lower qubits)
    bool empty() const
    {
        if (gsign || zmask) return false;
        for (const auto &p : pairs)
            if (p.second) return false;
        return true;
    }
    template <typename Local>
    bool fits(const FusedGate &g, Local local) const
    {
        if (g.k < 2) return true;
        const int d = std::abs(local(g.targets[1]) - local(g.targets[0]));
        for (const auto &p : pairs)
            if (p.first == d) return true;
        return pairs.size() < (size_t)kSignDist;
    }
    // s(x) = s00 + (s00 ^ s10) x_a + (s00 ^ s01) x_b + (s00 ^ s10 ^ s01 ^ s11) x_a x_b over GF(2)
    template <typename Local>
    void add(const FusedGate &g, const int (&s_in)[4], Local local)
    {
        // the gate's two qubits in local order (a below b); s over (bit of a) + 2 (bit of b)
        int a = local(g.targets[0]);
        int s[4] = {s_in[0], s_in[1], s_in[2], s_in[3]};
        if (g.k >= 2 && local(g.targets[1]) < a) {
            a = local(g.targets[1]);
            std::swap(s[1], s[2]);
        }
        gsign ^= (unsigned)s[0];
        if (s[0] ^ s[1]) zmask ^= 1u << a;
        if (g.k < 2) return;
        const int b = std::max(local(g.targets[0]), local(g.targets[1]));
        if (s[0] ^ s[2]) zmask ^= 1u << b;
        if (s[0] ^ s[1] ^ s[2] ^ s[3]) {
            for (auto &p : pairs)
                if (p.first == b - a) {
                    p.second ^= 1u << a;
                    return;
                }
            pairs.push_back({b - a, 1u << a});
        }
    }
    // the same signs over the index with the bits of F flipped: x_a -> x_a ^ f_a turns a linear term
    // into itself plus a constant and a pair term into itself plus linear terms and a constant
    SignRun flipped(unsigned F) const
    {
        SignRun r = *this;
        r.gsign ^= (unsigned)__builtin_popcount(zmask & F) & 1u;
        for (const auto &p : pairs)
            for (unsigned m = p.second; m; m &= m - 1u) {
                const int a = __builtin_ctz(m), b = a + p.first;
                const unsigned fa = (F >> a) & 1u, fb = (F >> b) & 1u;
                if (fb) r.zmask ^= 1u << a;
                if (fa) r.zmask ^= 1u << b;
                r.gsign ^= fa & fb;
            }
        return r;
    }
    void fill(BGate &b) const
    {
        b.gsign = gsign;
        b.zmask = zmask;
        b.nd = 0;
        for (const auto &p : pairs)
            if (p.second) {
                b.dist[b.nd] = p.first;
                b.dmask[b.nd] = p.second;
                ++b.nd;
            }
    }
};
// A 2x2 unitary as U = P R Q: P = diag(p0, p1), R = (c, -s; s, c) real with c = |u00| and s = |u10|,
// Q = diag(1, q1).  With U = e^(i phi) (x, -conj(y); y, conj(x)): p0 = u00 / |u00|, p1 = u10 / |u10|,
// q1 = -u01 / (|u01| p0) (a zero column entry takes the other entry of its row's phase).  False when
// the factors do not give back U to 1e-9 (a matrix that is not unitary).
bool factor_prq(const std::array<cplx, 4> &U, cplx &p0, cplx &p1, double &c, double &s, cplx &q1)
{
    const double a = std::abs(U[0]), b = std::abs(U[1]), cc = std::abs(U[2]), d = std::abs(U[3]);
    constexpr double kTiny = 1e-12;
    auto unit = [](const cplx &z) { return z / std::abs(z); };
    c = a;
    s = cc;
    if (cc <= kTiny && b <= kTiny) {   // diagonal
        if (a <= kTiny || d <= kTiny) return false;
        p0 = unit(U[0]);
        p1 = unit(U[3]);
        q1 = 1.0;
        s = 0.0;
        c = 1.0;
    } else if (a <= kTiny && d <= kTiny) {   // anti-diagonal
        p0 = -unit(U[1]);
        p1 = unit(U[2]);
        q1 = 1.0;
        c = 0.0;
        s = 1.0;
    } else {
        if (a <= kTiny || cc <= kTiny || b <= kTiny) return false;
        p0 = unit(U[0]);
        p1 = unit(U[2]);
        q1 = -unit(U[1]) / p0;
    }
    const cplx r[4] = {p0 * c, -p0 * s * q1, p1 * s, p1 * c * q1};
    for (int e = 0; e < 4; ++e)
        if (std::abs(r[e] - U[(size_t)e]) > 1e-9) return false;
    return true;
}

constexpr unsigned kStageBase = 7u;   // qubits 0-2: in every stage's local set

// A stage of a staged circuit: its gates, its local qubits and their order in the tile, and how the
// tile moves between global memory and shared memory.
struct StagePlan {
    std::vector<const FusedGate *> gates;   // in circuit order
    unsigned lam = 0u;                      // its local (logical) qubits
    int local_of[32];                       // logical qubit -> local bit, -1 outside the tile
    unsigned lmask = 0u;                    // physical local qubits of the load (of the store, first stage)
    bool mapped = false;                    // stored in another layout than loaded
    BStoreMap map{};
    int load_pos[32];                       // logical qubit -> physical position, as loaded (as stored, first stage)
    int store_pos[32];                      // and as stored
};

// Cut circuit gates gs (n qubits) into stages of at most L local qubits.
//
// Greedy: scanning the gates not yet placed in circuit order, a gate joins the stage when no
// earlier unplaced gate shares a qubit with it (it commutes past every gate it overtakes) and the
// stage's qubits with its own still number at most L; otherwise its qubits are closed for the
// rest of the scan.
//
// A tile moves in 32-byte runs, so physical qubits 0-2 must be local at its load and at its store.
// Between stages the state is relabelled: the layout a stage loads in puts three qubits that are
// local in it and in the stage before at physical 0-2 (swapped there from the next layout), and
// the stage before stores its tile in that layout.  The last stage stores in the circuit's own
// order, so qubits 0-2 are local in it; the first builds its tile and stores it in the second's
// layout.  Where the last stage has no room for qubits 0-2, or two neighbouring stages cannot
// share three local qubits, a stage without gates goes in between (one pass that only relabels).
// Any room left is filled with the qubits at the lowest physical positions (longer contiguous
// runs per tile).
std::vector<StagePlan> plan_stages(const std::vector<const FusedGate *> &gs, int n, int L)
{
    struct Stg {
        std::vector<const FusedGate *> gates;
        unsigned lam = 0u;    // local qubits so far
        int B[3] = {0, 1, 2}; // the qubits its load layout puts at physical 0-2
    };
    const unsigned all = n >= 32 ? ~0u : (1u << n) - 1u;
    std::vector<Stg> sv;
    {
        std::vector<const FusedGate *> rest = gs, left;
        while (sv.empty() || !rest.empty()) {
            Stg t;
            unsigned blocked = 0u;
            left.clear();
            for (const FusedGate *g : rest) {
                const unsigned q = (unsigned)g->mask;
                if (!(q & blocked) && __builtin_popcount(t.lam | q) <= L) {
                    t.lam |= q;
                    t.gates.push_back(g);
                } else {
                    blocked |= q;
                    left.push_back(g);
                }
            }
            sv.push_back(std::move(t));
            rest.swap(left);
        }
    }
    // qubits 0-2 local in the last stage (it stores in the circuit's order)
    if (__builtin_popcount(sv.back().lam | 7u) <= L) {
        sv.back().lam |= 7u;
    } else {
        Stg t;
        t.lam = 7u;
        sv.push_back(t);
    }
    // boundaries from the last: three qubits local in both neighbours, preferring the qubits at
    // physical 0-2 of the layout after the later one (the later one then stores as it loads),
    // then shared qubits, then qubits that fit in one side's spare room
    for (int k = (int)sv.size() - 2; k >= 0; --k) {
        Stg &nx = sv[(size_t)k + 1];
        int pref[3] = {0, 1, 2};
        if (k + 2 < (int)sv.size()) std::copy(sv[(size_t)k + 2].B, sv[(size_t)k + 2].B + 3, pref);
        auto pick = [&](Stg &cur) {
            int B[3], nb = 0;
            unsigned lam_r = cur.lam, lam_n = nx.lam;
            auto try_add = [&](int x) {
                if (nb == 3) return;
                for (int j = 0; j < nb; ++j)
                    if (B[j] == x) return;
                const unsigned bit = 1u << x;
                const bool in_r = lam_r & bit, in_n = lam_n & bit;
                if ((!in_r && __builtin_popcount(lam_r) >= L) || (!in_n && __builtin_popcount(lam_n) >= L)) return;
                lam_r |= bit;
                lam_n |= bit;
                B[nb++] = x;
            };
            for (int j = 0; j < 3; ++j) try_add(pref[j]);
            if (nb < 3) {   // not all three: start over with shared qubits, then spare room
                nb = 0;
                lam_r = cur.lam;
                lam_n = nx.lam;
                for (int x = 0; x < n; ++x)
                    if ((cur.lam & nx.lam) >> x & 1u) try_add(x);
                for (int x = 0; x < n; ++x)
                    if ((cur.lam | nx.lam) >> x & 1u) try_add(x);
                for (int x = 0; x < n; ++x) try_add(x);
            }
            if (nb < 3) return false;
            std::copy(B, B + 3, nx.B);
            nx.lam = lam_n;
            cur.lam = lam_r;
            return true;
        };
        if (pick(sv[(size_t)k])) continue;
        // a relabelling stage between them: three local qubits of each side
        Stg t;
        for (int x = 0, c = 0; x < n && c < 3; ++x)
            if ((nx.lam >> x) & 1u) {
                t.lam |= 1u << x;
                ++c;
            }
        for (int x = 0, c = 0; x < n && c < 3; ++x)
            if ((sv[(size_t)k].lam >> x) & 1u) {
                t.lam |= 1u << x;
                ++c;
            }
        sv.insert(sv.begin() + k + 1, t);
        k += 2;   // next: the boundary (new stage, next), then (k, new stage); both share three qubits
    }
    // layouts, last stage first: the last stores in the circuit's order; stage k loads in layout
    // pi[k] (= pi[k + 1] with B[k] swapped to physical 0-2), which stage k - 1 stores in
    const int K = (int)sv.size();
    std::vector<std::array<int, 32>> pi((size_t)K + 1);
    for (int x = 0; x < 32; ++x) pi[(size_t)K][(size_t)x] = x;
    for (int k = K - 1; k >= 1; --k) {
        std::array<int, 32> p = pi[(size_t)k + 1];
        const Stg &r = sv[(size_t)k];
        for (int i = 0; i < 3; ++i) {
            const int b = r.B[i];
            int y = 0;
            for (int x = 0; x < n; ++x)
                if (p[(size_t)x] == i) y = x;
            std::swap(p[(size_t)b], p[(size_t)y]);
        }
        pi[(size_t)k] = p;
    }
    pi[0] = pi[1];   // (the first stage loads nothing)
    std::vector<StagePlan> out((size_t)K);
    for (int k = 0; k < K; ++k) {
        const Stg &r = sv[(size_t)k];
        StagePlan &P = out[(size_t)k];
        P.gates = r.gates;
        const std::array<int, 32> &lay = k == 0 ? pi[1] : pi[(size_t)k];   // the first stage's order is its store's
        const std::array<int, 32> &sto = pi[(size_t)k + 1];
        unsigned lam = r.lam;
        // the load layout's physical 0-2 are local (the last stage's are qubits 0-2)
        for (int x = 0; x < n; ++x)
            if (lay[(size_t)x] < 3) lam |= 1u << x;
        // fill: lowest physical positions first
        for (int pos = 0; pos < n && __builtin_popcount(lam) < L; ++pos)
            for (int x = 0; x < n; ++x)
                if (lay[(size_t)x] == pos) lam |= 1u << x;
        P.lam = lam & all;
        // local order: by physical position in the load layout (physical 0-2 first)
        int order[32], no = 0;
        for (int pos = 0; pos < n; ++pos)
            for (int x = 0; x < n; ++x)
                if (lay[(size_t)x] == pos && ((lam >> x) & 1u)) order[no++] = x;
        for (int x = 0; x < 32; ++x) P.local_of[x] = -1;
        P.lmask = 0u;
        for (int i = 0; i < no; ++i) {
            P.local_of[order[i]] = i;
            P.lmask |= 1u << lay[(size_t)order[i]];
        }
        for (int x = 0; x < 32; ++x) {
            P.load_pos[x] = lay[(size_t)x];
            P.store_pos[x] = sto[(size_t)x];
        }
        P.mapped = k > 0 && lay != sto;
        if (P.mapped) {
            int so[32], ns = 0;
            for (int pos = 0; pos < n; ++pos)
                for (int x = 0; x < n; ++x)
                    if (sto[(size_t)x] == pos && ((lam >> x) & 1u)) so[ns++] = x;
            P.map.lmask = 0u;
            for (int j = 0; j < ns; ++j) {
                P.map.src[j] = (unsigned char)P.local_of[so[j]];
                P.map.lmask |= 1u << sto[(size_t)so[j]];
            }
            int t = 0;   // tile index bit t: the t-th non-local physical position of the load layout
            for (int pos = 0; pos < n; ++pos)
                if (!((P.lmask >> pos) & 1u)) {
                    int x = 0;
                    for (int y = 0; y < n; ++y)
                        if (lay[(size_t)y] == pos) x = y;
                    P.map.tbit[t++] = (unsigned char)sto[(size_t)x];
                }
        }
    }
    return out;
}

// Append the stages of circuit gates gs (global targets, n qubits; see plan_stages) to the stage
// tables: stage gates are re-fused to at most stage_k qubits (0: kept as they are) and renumbered to
// local qubits.
void build_stages(const std::vector<const FusedGate *> &gs, int n, int L, int stage_k, bool phase_opt, std::vector<BStage> &st,
                  std::vector<BChunk> &chunks, std::vector<BGate> &sg, std::vector<float2> &sm, std::vector<BStoreMap> &maps)
{
    for (const StagePlan &plan : plan_stages(gs, n, L)) {
        const std::vector<const FusedGate *> &taken = plan.gates;
        BStage bs{};
        bs.lmask = plan.lmask;
        bs.chunk_begin = (int)chunks.size();
        bs.map = -1;
        if (plan.mapped) {
            bs.map = (int)maps.size();
            maps.push_back(plan.map);
        }
        auto local = [&](int q) { return plan.local_of[q]; };
        // a chunk's matrices start at an even offset of the table (16-byte copies)
        auto new_chunk = [&]() {
            if (sm.size() & 1) sm.push_back(make_float2(0.f, 0.f));
            chunks.push_back(BChunk{(int)sg.size(), 0, (int)sm.size(), 0});
        };
        const bool phases = phase_opt && L >= 10;
        // per gate: U then its pair-swapped copy U' (U'[r][j] = U[r][j ^ 1]), starting at an even
        // offset of the chunk (16-byte aligned in shared memory); a sign run rides on the gate
        // (k = 0: a sign-only sweep)
        // the tile's frame: local qubits whose bits it holds flipped (X applied, so that a rotation by
        // more than 45 degrees costs what a small one does; see add_layer).  Everything emitted acts
        // on the flipped tile: matrices conjugated by the flips, sign runs over the flipped index;
        // the store puts amplitude l back at l ^ frame.
        unsigned frame = 0u;
        auto emit = [&](const FusedGate *g, const SignRun &run_true) {
            const int dd = g ? (int)g->ur.size() : 0;
            const SignRun run = run_true.flipped(frame);
            // the kernel takes a gate's local targets ascending: perm[j] = the position in g's
            // targets of its j-th lowest local target (the matrix index bits follow); fm = the
            // flips on g's targets, as bits of its matrix index
            int perm[SV_MAX_K] = {0, 1, 2, 3, 4, 5};
            unsigned fm = 0u;
            if (g) {
                std::sort(perm, perm + g->k, [&](int x, int y) { return local(g->targets[x]) < local(g->targets[y]); });
                for (int j = 0; j < g->k; ++j)
                    if ((frame >> local(g->targets[j])) & 1u) fm |= 1u << j;
            }
            if (chunks.size() == (size_t)bs.chunk_begin || chunks.back().gate_count == kStageGateCap ||
                chunks.back().mat_count + 1 + 2 * dd > kStageMatCap)
                new_chunk();
            if (chunks.back().mat_count & 1) {
                sm.push_back(make_float2(0.f, 0.f));
                chunks.back().mat_count += 1;
            }
            BGate b{};
            run.fill(b);
            b.mat_off = (int)sm.size();
            if (g) {
                b.k = g->k;
                for (int j = 0; j < g->k; ++j) b.targets[j] = local(g->targets[perm[j]]);
                // X^f U X^f with the index bits reordered: entry (r, c) from (old(r) ^ f, old(c) ^ f)
                const int D = 1 << g->k;
                auto old_index = [&](int x) {
                    int y = 0;
                    for (int j = 0; j < g->k; ++j)
                        if ((x >> j) & 1) y |= 1 << perm[j];
                    return y;
                };
                auto src = [&](int e) { return ((old_index(e / D) ^ (int)fm) * D) + (old_index(e % D) ^ (int)fm); };
                for (int e = 0; e < dd; ++e) sm.push_back(make_float2(g->ur[(size_t)src(e)], g->ui[(size_t)src(e)]));
                for (int e = 0; e < dd; ++e) sm.push_back(make_float2(g->ur[(size_t)src(e ^ 1)], g->ui[(size_t)src(e ^ 1)]));
            }
            sg.push_back(b);
            chunks.back().gate_count += 1;
            chunks.back().mat_count += 2 * dd;
        };
        // The stage's gates in order: dense gates collect in a run that is re-fused (stage_k) when
        // it ends; diagonal +-1 gates on at most two qubits collect in a sign run that is applied to
        // the inputs of the first gate emitted after it.  A sign gate that shares a qubit with the
        // dense run ends that run first (the sign run so far, which precedes the dense run, rides on
        // the run's first gate); one that does not commutes past the dense run into the sign run.
        SignRun run;
        std::vector<const FusedGate *> dense_run;
        uint64_t dense_q = 0;
        auto flush = [&]() {
            if (!dense_run.empty()) {
                std::vector<FusedGate> fused;
                if (stage_k > 0) fused = refuse_gates(dense_run, n, stage_k);
                for (size_t i = 0; i < (stage_k > 0 ? fused.size() : dense_run.size()); ++i) {
                    const FusedGate *g = stage_k > 0 ? &fused[i] : dense_run[i];
                    // the kernel applies a run on the inputs of gates of up to three qubits (a
                    // 4-qubit gate's 16 inputs leave no registers for it): else a sweep of its own
                    if (i == 0 && g->k > 3 && !run.empty()) emit(nullptr, run);
                    emit(g, i == 0 && g->k <= 3 ? run : SignRun{});
                }
            } else if (!run.empty()) {
                emit(nullptr, run);
            }
            run = SignRun{};
            dense_run.clear();
            dense_q = 0;
        };
        // Register phases (tiles of at least 10 qubits).  A run of one-qubit gates is a layer: per
        // qubit the product of its gates, in order; the layers and the sign runs between them go
        // into phases over windows of five local qubits starting at 0, 5 and L - 5.  A layer's
        // gates all commute, so its windows may run in any order: it starts with the open phase's
        // window when it has gates there (the sign run before it and its first window's gates join
        // that phase) and ends on the far side, where the next layer starts.  A sign run joins the
        // open phase (or waits for the next one).
        //
        // Each qubit's 2x2 unitary is factored U = P R Q (P, Q diagonal, R a real rotation; see
        // factor_prq): the layer runs as real rotations, 4 multiply-adds per amplitude instead of
        // 8, and one layer's P's with the next layer's Q's -- all diagonal, all commuting with the
        // sign run between the layers -- become one diagonal over the tile's qubits, applied
        // right before the next layer's first rotation (a complex factor per amplitude).
        const int nwin = L > 10 ? 3 : 2;
        const int q0s[3] = {0, 5, L - 5};
        enum : int { kSubGate = 0, kSubSign = 1, kSubRot = 2, kSubDiag = 3, kSubTan5 = 4 };
        using Diag = std::array<std::array<cplx, 2>, 32>;   // per local qubit: its diagonal (d0, d1)
        struct Sub {
            int kind;
            int r;
            std::array<cplx, 4> U;      // kSubGate: the matrix; kSubRot: (c, -s, s, c) in the real parts
            SignRun s;
            Diag D;
            std::array<std::array<double, 4>, 5> R5;   // kSubTan5: window bit r's t in R5[r][0]
        };
        auto unit_diag = []() {
            Diag d;
            for (auto &e : d) e = {cplx(1.0), cplx(1.0)};
            return d;
        };
        int open_w = -1;
        std::vector<Sub> open_subs;
        std::vector<SignRun> pending;
        Diag pend_p = unit_diag();   // the last layer's P's, not yet applied
        bool pend_p_set = false;
        auto emit_phase = [&]() {
            if (open_w < 0) return;
            int nm = 0;   // float2 of matrices
            for (const Sub &u : open_subs)
                nm += u.kind == kSubGate ? 8 : u.kind == kSubRot ? 4 : u.kind == kSubDiag ? 80 : u.kind == kSubTan5 ? 6 : 0;
            const int recs = 1 + (int)open_subs.size();
            if (chunks.size() == (size_t)bs.chunk_begin || chunks.back().gate_count + recs > kStageGateCap ||
                chunks.back().mat_count + 1 + nm > kStageMatCap)
                new_chunk();
            if (chunks.back().mat_count & 1) {
                sm.push_back(make_float2(0.f, 0.f));
                chunks.back().mat_count += 1;
            }
            const int q0 = q0s[open_w];
            BGate h{};
            h.k = -2;
            h.targets[0] = q0;
            h.targets[1] = recs - 1;
            sg.push_back(h);
            auto f2 = [](const cplx &c) { return make_float2((float)c.real(), (float)c.imag()); };
            for (const Sub &u : open_subs) {
                BGate b{};
                if (u.kind == kSubGate) {
                    b.k = -3;
                    b.targets[0] = u.r;
                    b.mat_off = (int)sm.size();
                    for (int e = 0; e < 4; ++e) sm.push_back(f2(u.U[(size_t)e]));
                    for (int e = 0; e < 4; ++e) sm.push_back(f2(u.U[(size_t)(3 - e)]));   // X U X
                } else if (u.kind == kSubRot) {
                    b.k = -5;
                    b.targets[0] = u.r;
                    b.mat_off = (int)sm.size();
                    const float a00 = (float)u.U[0].real(), a01 = (float)u.U[1].real(), a10 = (float)u.U[2].real(),
                                a11 = (float)u.U[3].real();
                    sm.push_back(make_float2(a00, a01));
                    sm.push_back(make_float2(a10, a11));
                    sm.push_back(make_float2(a11, a10));   // X R X
                    sm.push_back(make_float2(a01, a00));
                } else if (u.kind == kSubTan5) {
                    b.k = -8;
                    b.mat_off = (int)sm.size();
                    for (int r = 0; r < 5; ++r) sm.push_back(make_float2((float)u.R5[(size_t)r][0], -(float)u.R5[(size_t)r][0]));
                    sm.push_back(make_float2(0.f, 0.f));
                } else if (u.kind == kSubDiag) {
                    // amplitude i gets C * prod over set bits q of i of w_q (w_q = d1 / d0, C = prod
                    // of the d0): tables over the window's 5 bits (slot), the thread's first 5
                    // non-window bits (with C) and its next 4 -- a thread's non-window bits are its
                    // phase index it, bit j of it being the j-th non-window qubit, ascending
                    b.k = -6;
                    b.mat_off = (int)sm.size();
                    cplx C(1.0);
                    std::array<cplx, 32> w;
                    for (int q = 0; q < 32; ++q) {
                        C *= u.D[(size_t)q][0];
                        w[(size_t)q] = u.D[(size_t)q][1] / u.D[(size_t)q][0];
                    }
                    int nw[9], nn = 0;
                    for (int q = 0; q < L && nn < 9; ++q)
                        if (q < q0 || q >= q0 + 5) nw[nn++] = q;
                    for (int x = 0; x < 32; ++x) {
                        cplx t(1.0);
                        for (int r = 0; r < 5; ++r)
                            if ((x >> r) & 1) t *= w[(size_t)(q0 + r)];
                        sm.push_back(f2(t));
                    }
                    for (int x = 0; x < 32; ++x) {
                        cplx t = C;
                        for (int j = 0; j < 5 && j < nn; ++j)
                            if ((x >> j) & 1) t *= w[(size_t)nw[j]];
                        sm.push_back(f2(t));
                    }
                    for (int x = 0; x < 16; ++x) {
                        cplx t(1.0);
                        for (int j = 0; j < 4 && 5 + j < nn; ++j)
                            if ((x >> j) & 1) t *= w[(size_t)nw[5 + j]];
                        sm.push_back(f2(t));
                    }
                } else {
                    u.s.fill(b);
                    b.k = -4;
                    unsigned qw = 0u;   // the form on the window bits alone, per slot
                    for (unsigned m = 0; m < 32u; ++m) {
                        const unsigned y = m << q0;
                        unsigned par = (unsigned)__builtin_popcount(y & u.s.zmask);
                        for (const auto &pr : u.s.pairs) par += (unsigned)__builtin_popcount(y & (y >> pr.first) & pr.second);
                        qw |= (par & 1u) << m;
                    }
                    b.lmask = qw;
                    for (int r = 0; r < 5; ++r) {   // pair partners of window qubit r
                        const int c = q0 + r;
                        unsigned nb = 0u;
                        for (const auto &pr : u.s.pairs) {
                            if (c >= pr.first && ((pr.second >> (c - pr.first)) & 1u)) nb |= 1u << (c - pr.first);
                            if ((pr.second >> c) & 1u) nb |= 1u << (c + pr.first);
                        }
                        b.targets[r] = (int)nb;
                    }
                }
                sg.push_back(b);
            }
            chunks.back().gate_count += recs;
            chunks.back().mat_count += nm;
            open_w = -1;
            open_subs.clear();
        };
        auto open_phase = [&](int w) {
            emit_phase();
            open_w = w;
            for (const SignRun &r : pending) open_subs.push_back(Sub{kSubSign, 0, {}, r.flipped(frame), {}, {}});
            pending.clear();
        };
        auto add_sub = [&](Sub u) {
            if ((int)open_subs.size() + 2 > kPhaseMaxRecords) open_phase(open_w);
            open_subs.push_back(std::move(u));
        };
        auto add_signs = [&](const SignRun &r) {   // r over the true index (pending runs stay so)
            if (r.empty()) return;
            if (open_w >= 0) add_sub(Sub{kSubSign, 0, {}, r.flipped(frame), {}, {}});
            else pending.push_back(r);
        };
        // the diagonal as it acts on the flipped tile: entries exchanged on the frame's qubits
        auto diag_phys = [&](Diag d) {
            for (int q = 0; q < 32; ++q)
                if ((frame >> q) & 1u) std::swap(d[(size_t)q][0], d[(size_t)q][1]);
            return d;
        };
        auto conj_phys = [&](std::array<cplx, 4> u, int q) {   // X U X on a flipped qubit
            if ((frame >> q) & 1u) u = {u[3], u[2], u[1], u[0]};
            return u;
        };
        // A rotation R = (c, -s; s, c) with 0 <= s, c runs as a multiple of T(t) = (1, -t; t, 1), two
        // multiply-adds per pair of amplitudes: R = c T(s/c) when s <= c; otherwise R = s X T(c/s) Z
        // (Z = diag(1, -1) before it, X after), and the X goes into the frame instead of being
        // applied.  So |t| <= 1, and every scale (at least 1/sqrt 2) and Z joins the layer's
        // leading diagonal.
        auto add_layer = [&]() {
            std::array<std::array<cplx, 4>, 32> U{};
            unsigned lm = 0u;
            for (const FusedGate *g : dense_run) {
                const int q = local(g->targets[0]);
                const cplx *G = g->mat.data();
                std::array<cplx, 4> &P = U[(size_t)q];
                if (!((lm >> q) & 1u)) {
                    P = {G[0], G[1], G[2], G[3]};
                    lm |= 1u << q;
                } else {
                    P = {G[0] * P[0] + G[1] * P[2], G[0] * P[1] + G[1] * P[3], G[2] * P[0] + G[3] * P[2], G[2] * P[1] + G[3] * P[3]};
                }
            }
            // windows: qubits 0-4 in the first, 10 and up in the last; L - 5..9 in either
            unsigned need[3] = {0u, 0u, 0u}, flex = 0u;
            for (int q = 0; q < L; ++q) {
                if (!((lm >> q) & 1u)) continue;
                if (q < 5) need[0] |= 1u << q;
                else if (nwin == 3 && q >= 10) need[2] |= 1u << q;
                else if (nwin == 3 && q >= L - 5) flex |= 1u << q;
                else need[1] |= 1u << q;
            }
            if (flex) {
                const int w = need[2] ? 2 : need[1] ? 1 : open_w == 2 ? 2 : 1;
                need[w] |= flex;
            }
            int order[3], no = 0;
            const bool open_in = open_w >= 0 && need[open_w] != 0u;
            if (open_in) {
                order[no++] = open_w;
                if (open_w == nwin - 1) {
                    for (int w = nwin - 2; w >= 0; --w)
                        if (need[w]) order[no++] = w;
                } else {
                    for (int w = 0; w < nwin; ++w)
                        if (w != open_w && need[w]) order[no++] = w;
                }
            } else {
                for (int w = 0; w < nwin; ++w)
                    if (need[w]) order[no++] = w;
            }
            // factors: the diagonal before the rotations (pending P's times this layer's Q's) and
            // the P's left pending; a matrix that does not factor stays a complex gate.  Windows
            // with three or more rotations run them as one straight-line record in T form.
            Diag E = pend_p;
            bool e_set = pend_p_set;
            pend_p = unit_diag();
            pend_p_set = false;
            std::array<bool, 32> rot{};
            std::array<double, 32> tq{};
            unsigned tan_q = 0u, z_q = 0u;
            double scale = 1.0;
            for (int q = 0; q < L; ++q) {
                if (!((lm >> q) & 1u)) continue;
                cplx p0, p1, q1;
                double c, sn;
                if (factor_prq(U[(size_t)q], p0, p1, c, sn, q1)) {
                    rot[(size_t)q] = true;
                    U[(size_t)q] = {cplx(c), cplx(-sn), cplx(sn), cplx(c)};
                    E[(size_t)q][1] *= q1;
                    pend_p[(size_t)q] = {p0, p1};
                    e_set = true;
                    pend_p_set = true;
                    tq[(size_t)q] = sn <= c ? sn / c : c / sn;
                }
            }
            for (int w = 0; w < nwin; ++w) {
                unsigned rm = 0u;
                for (unsigned m = need[w]; m; m &= m - 1u)
                    if (rot[(size_t)__builtin_ctz(m)]) rm |= m & (0u - m);
                if (__builtin_popcount(rm) >= 3) tan_q |= rm;
            }
            for (unsigned m = tan_q; m; m &= m - 1u) {
                const int q = __builtin_ctz(m);
                const double c = U[(size_t)q][0].real(), sn = U[(size_t)q][2].real();
                if (sn <= c) {
                    scale *= c;
                } else {
                    scale *= sn;
                    z_q |= 1u << q;
                    E[(size_t)q][1] = -E[(size_t)q][1];
                }
            }
            if (tan_q) {
                E[0][0] *= scale;
                E[0][1] *= scale;
                e_set = true;
            }
            for (int i = 0; i < no; ++i) {
                const int w = order[i];
                if (!(i == 0 && open_in)) open_phase(w);
                if (i == 0 && e_set) add_sub(Sub{kSubDiag, 0, {}, SignRun{}, diag_phys(E), {}});
                const unsigned tw = tan_q & need[w];
                if (tw) {
                    Sub f5{kSubTan5, 0, {}, SignRun{}, {}, {}};
                    for (int r = 0; r < 5; ++r) {
                        const int q = q0s[w] + r;
                        const double t = ((tw >> q) & 1u) ? tq[(size_t)q] : 0.0;
                        f5.R5[(size_t)r][0] = ((frame >> q) & 1u) ? -t : t;   // X T(t) X = T(-t)
                    }
                    add_sub(f5);
                    frame ^= z_q & tw;   // the X after each rotation that went the long way
                }
                for (unsigned m = need[w] & ~tw; m; m &= m - 1u) {
                    const int q = __builtin_ctz(m);
                    add_sub(Sub{rot[(size_t)q] ? kSubRot : kSubGate, q - q0s[w], conj_phys(U[(size_t)q], q), SignRun{}, {}, {}});
                }
            }
        };
        auto flush_phases = [&]() {   // before a gate outside the phases, and at the stage's end
            if (pend_p_set && open_w >= 0) add_sub(Sub{kSubDiag, 0, {}, SignRun{}, diag_phys(pend_p), {}});
            pend_p = unit_diag();
            pend_p_set = false;
            emit_phase();
            for (const SignRun &r : pending) emit(nullptr, r);
            pending.clear();
        };
        // with phases: a run of one-qubit gates is a layer; other dense runs end the phases
        auto flush_all = [&]() {
            bool one_qubit = phases && !dense_run.empty();
            for (const FusedGate *g : dense_run) one_qubit = one_qubit && g->k == 1;
            if (one_qubit) {
                add_signs(run);
                add_layer();
                run = SignRun{};
                dense_run.clear();
                dense_q = 0;
            } else if (phases && dense_run.empty()) {
                add_signs(run);
                run = SignRun{};
            } else {
                if (phases) flush_phases();
                flush();
            }
        };
        for (const FusedGate *g : taken) {
            int sg_bits[4];
            if (sign_pattern(*g, sg_bits)) {
                if ((g->mask & dense_q) || !run.fits(*g, local)) flush_all();
                run.add(*g, sg_bits, local);
            } else {
                dense_run.push_back(g);
                dense_q |= g->mask;
            }
        }
        flush_all();
        if (phases) flush_phases();
        bs.chunk_count = (int)chunks.size() - bs.chunk_begin;
        bs.frame = frame;
        st.push_back(bs);
    }
}

// Work list: single-CTA circuits in global memory first (largest first: the rigid chains start
// early), then the tiles of the split circuits step by step across circuits, then the circuits
// held in shared memory (short; they fill the tail).
int build_work_list(sv_batch *b)
{
    const int cfg[7] = {b->opts.smem_max_n, b->opts.split_min_n, b->opts.tile_log2, b->opts.wave_mb, b->opts.stage_log2,
                        b->opts.stage_k, b->opts.stage_layers};
    if (b->d_items && std::memcmp(cfg, b->list_cfg, sizeof(cfg)) == 0 && b->list_stall == b->stall) return SV_OK;
    std::vector<BItem> items;
    std::vector<int> need;
    std::vector<BCirc> hc = b->hc;
    std::vector<int> split;
    std::vector<BStage> hst;
    std::vector<BChunk> hch;
    std::vector<BGate> hsg;
    std::vector<float2> hsm;
    std::vector<BStoreMap> hmap;
    for (int c = 0; c < (int)hc.size(); ++c) {
        const int n = hc[(size_t)c].n;
        hc[(size_t)c].done_off = 0;
        hc[(size_t)c].stage_begin = 0;
        hc[(size_t)c].n_stages = 0;
        if (n <= b->opts.smem_max_n) continue;
        if (b->opts.split_min_n > 0 && n >= b->opts.split_min_n && b->opts.stage_log2 > 0 && n >= kStageMinN) {
            // staged: one counter per stage, 2^(n - L) tiles each
            const int L = std::min(n, b->opts.stage_log2);
            std::vector<const FusedGate *> gs;
            for (int gi = 0; gi < hc[(size_t)c].gate_count; ++gi) gs.push_back(b->src[(size_t)(hc[(size_t)c].gate_begin + gi)]);
            hc[(size_t)c].stage_begin = (int)hst.size();
            try {
                build_stages(gs, n, L, b->opts.stage_k, b->opts.stage_layers != 0, hst, hch, hsg, hsm, hmap);
            } catch (const std::bad_alloc &) {
                set_error("sv_batch: out of host memory building stages");
                return SV_ENOMEM;
            }
            hc[(size_t)c].n_stages = (int)hst.size() - hc[(size_t)c].stage_begin;
            hc[(size_t)c].done_off = (int)need.size();
            for (int s = 0; s < hc[(size_t)c].n_stages; ++s) need.push_back(1 << (n - L));
            split.push_back(c);
        } else if (b->opts.split_min_n > 0 && n >= b->opts.split_min_n) {
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
            items.push_back(BItem{kSingle, c, 0, 0, 0, 0, 0, 0u, 0, 0, 0, BChunk{}, 0u, -1, {0, 0}});
        }
    }
    if (hsm.size() & 1) hsm.push_back(make_float2(0.f, 0.f));   // the last chunk's 16-byte copy stays inside
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
                const bool staged = hc[(size_t)c].n_stages > 0;
                if (s >= (staged ? hc[(size_t)c].n_stages : hc[(size_t)c].gate_count + 1)) continue;
                any = true;
                const int t = need[(size_t)(hc[(size_t)c].done_off + s)];
                BItem it{staged ? kStage : kTile, c, s, 0, 0, 0, 0, 0u, 0, 0, 0, BChunk{}, 0u, -1, {0, 0}};
                if (staged) {
                    const BCirc &C = hc[(size_t)c];
                    const BStage &St = hst[(size_t)(C.stage_begin + s)];
                    it.n = C.n;
                    it.done_off = C.done_off;
                    it.need_prev = s > 0 ? need[(size_t)(C.done_off + s - 1)] : 0;
                    it.lmask = St.lmask;
                    it.state_off = C.state_off;
                    it.chunk_begin = St.chunk_begin;
                    it.chunk_count = St.chunk_count;
                    if (St.chunk_count > 0) it.ch0 = hch[(size_t)St.chunk_begin];
                    it.frame = St.frame;
                    it.map = St.map;
                }
                for (int i = 0; i < t; ++i) {
                    it.tile = i;
                    items.push_back(it);
                }
            }
            if (!any) break;
        }
    for (int c = 0; c < (int)hc.size(); ++c)
        if (hc[(size_t)c].n <= b->opts.smem_max_n) items.push_back(BItem{kWhole, c, 0, 0, 0, 0, 0, 0u, 0, 0, 0, BChunk{}, 0u, -1, {0, 0}});
    if (b->stall && !need.empty()) {   // nothing completes the extra tile: its waiters give up
        need[0] += 1;
        for (BItem &w : items)
            if (w.kind == kStage && w.done_off == 0 && w.step == 1) w.need_prev += 1;
    }
    cudaFree(b->d_items);
    cudaFree(b->d_need);
    cudaFree(b->d_sync);
    cudaFree(b->d_stages);
    cudaFree(b->d_chunks);
    cudaFree(b->d_sgates);
    cudaFree(b->d_smats);
    cudaFree(b->d_smaps);
    b->d_smaps = nullptr;
    b->d_items = nullptr;
    b->d_need = nullptr;
    b->d_sync = nullptr;
    b->d_stages = nullptr;
    b->d_chunks = nullptr;
    b->d_sgates = nullptr;
    b->d_smats = nullptr;
    b->n_items = (int)items.size();
    b->n_counters = (int)need.size();
    {
        sv_batch_info in{};
        in.items = (int)items.size();
        in.stages = (int)hst.size();
        in.stage_gates = (int)hsg.size();
        for (const BCirc &c : hc) {
            const double sb = (double)state_bytes(c.n);
            if (c.n <= b->opts.smem_max_n) {
                ++in.whole;
                in.traffic_bytes += sb;
            } else if (c.n_stages > 0) {
                ++in.staged;
                in.traffic_bytes += sb * (2.0 * c.n_stages - 1.0);
            } else {
                ++(b->opts.split_min_n > 0 && c.n >= b->opts.split_min_n ? in.split : in.single);
                in.traffic_bytes += sb * (1.0 + 2.0 * c.gate_count);
            }
        }
        b->info = in;
    }
    cudaError_t e = cudaMalloc(&b->d_items, sizeof(BItem) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_need, sizeof(int) * std::max<size_t>(need.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sync, sizeof(int) * (2 + need.size()));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_stages, sizeof(BStage) * std::max<size_t>(hst.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_chunks, sizeof(BChunk) * std::max<size_t>(hch.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sgates, sizeof(BGate) * std::max<size_t>(hsg.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_smats, sizeof(float2) * std::max<size_t>(hsm.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_smaps, sizeof(BStoreMap) * std::max<size_t>(hmap.size(), 1));
    if (e == cudaSuccess && !hmap.empty())
        e = cudaMemcpy(b->d_smaps, hmap.data(), sizeof(BStoreMap) * hmap.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !items.empty()) e = cudaMemcpy(b->d_items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !need.empty()) e = cudaMemcpy(b->d_need, need.data(), sizeof(int) * need.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hst.empty()) e = cudaMemcpy(b->d_stages, hst.data(), sizeof(BStage) * hst.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hch.empty()) e = cudaMemcpy(b->d_chunks, hch.data(), sizeof(BChunk) * hch.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hsg.empty()) e = cudaMemcpy(b->d_sgates, hsg.data(), sizeof(BGate) * hsg.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !hsm.empty()) e = cudaMemcpy(b->d_smats, hsm.data(), sizeof(float2) * hsm.size(), cudaMemcpyHostToDevice);
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
    a.stages = b->d_stages;
    a.chunks = b->d_chunks;
    a.mat_cap = mat_cap(b->opts);
    a.gate_cap = gate_cap(b->opts);
    a.sgates = b->d_sgates;
    a.smats = b->d_smats;
    a.smaps = b->d_smaps;
    a.sync = b->d_sync;
    a.need = b->d_need;
    a.err = b->d_err;
    a.tile_log2 = b->opts.tile_log2;
    a.stage_log2 = b->opts.stage_log2;
    SV_CUDA_TRY(cudaMemsetAsync(b->d_sync, 0, sizeof(int) * (2 + (size_t)b->n_counters), b->stream));
    const dim3 grid((unsigned)b->opts.ctas), block((unsigned)b->opts.threads);
    if (b->opts.ctas_per_sm == 2)
        batch_kernel<256, 2><<<grid, block, smem_bytes(b->opts), b->stream>>>(a);
    else if (b->opts.threads <= 256)
        batch_kernel<256, 1><<<grid, block, smem_bytes(b->opts), b->stream>>>(a);
    else
        batch_kernel<512, 1><<<grid, block, smem_bytes(b->opts), b->stream>>>(a);
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
    if (o.stage_log2 != 0 && (o.stage_log2 < kStageMinN || o.stage_log2 > 14)) { set_error("sv_batch: stage_log2 must be 0 or in [%d, 14]", kStageMinN); return SV_EINVAL; }
    if (o.stage_k < 0 || o.stage_k > kBatchMaxK) { set_error("sv_batch: stage_k must be in [0, %d]", kBatchMaxK); return SV_EINVAL; }
    if (o.stage_layers != 0 && o.stage_layers != 1) { set_error("sv_batch: stage_layers must be 0 or 1"); return SV_EINVAL; }
    if (o.ctas_per_sm < 0 || o.ctas_per_sm > 2) { set_error("sv_batch: ctas_per_sm must be 0, 1 or 2"); return SV_EINVAL; }
    if (o.ctas_per_sm == 2) {
        if (o.threads > 256) { set_error("sv_batch: ctas_per_sm = 2 takes CTAs of at most 256 threads"); return SV_EINVAL; }
        int dev = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
            set_error("sv_batch: device query failed");
            return SV_ECUDA;
        }
        // each CTA also holds its static shared memory (under 3 KB) and the 1 KB the system reserves
        if (2 * (smem_bytes(o) + 4096) > (size_t)per_sm) {
            set_error("sv_batch: ctas_per_sm = 2 needs two CTAs' shared memory (%zu bytes each) on one SM", smem_bytes(o));
            return SV_EINVAL;
        }
    }
    return SV_OK;
}

int set_smem_attrs(const sv_batch_opts &o)
{
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(o)));
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<512, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(o)));
    SV_CUDA_TRY(cudaFuncSetAttribute(batch_kernel<256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(o)));
    return SV_OK;
}

}  // namespace

extern "C" int sv_batch_plan_stages(const sv_fused *f, int stage_log2, int max_stages, int *gates, unsigned *lam, int *load_pos,
                                    int *store_pos, int *order)
{
    clear_error();
    if (!f || max_stages < 0) { set_error("sv_batch_plan_stages: bad argument"); return SV_EINVAL; }
    if (f->n < kStageMinN || f->n > kBatchMaxN) { set_error("sv_batch_plan_stages: n must be in [%d, %d]", kStageMinN, kBatchMaxN); return SV_EINVAL; }
    if (stage_log2 < kStageMinN || stage_log2 > 14) { set_error("sv_batch_plan_stages: stage_log2 must be in [%d, 14]", kStageMinN); return SV_EINVAL; }
    std::vector<const FusedGate *> gs;
    for (const FusedGate &g : f->gates) {
        if (g.cmask) { set_error("sv_batch_plan_stages: a gate keeps controls"); return SV_EINVAL; }
        if (!g.post.empty() || !g.swaps.empty() || g.k < 1) { set_error("sv_batch_plan_stages: post-phases and swap networks are not staged"); return SV_EINVAL; }
        gs.push_back(&g);
    }
    std::vector<StagePlan> plan;
    try {
        plan = plan_stages(gs, f->n, std::min(f->n, stage_log2));
    } catch (const std::bad_alloc &) {
        set_error("sv_batch_plan_stages: out of host memory");
        return SV_ENOMEM;
    }
    int at = 0;
    for (int s = 0; s < (int)plan.size(); ++s) {
        const StagePlan &P = plan[(size_t)s];
        if (order)
            for (const FusedGate *g : P.gates) order[at++] = (int)(g - f->gates.data());
        if (s >= max_stages) continue;
        if (gates) gates[s] = (int)P.gates.size();
        if (lam) lam[s] = P.lam;
        for (int q = 0; q < 32; ++q) {
            if (load_pos) load_pos[32 * s + q] = q < f->n ? P.load_pos[q] : q;
            if (store_pos) store_pos[32 * s + q] = q < f->n ? P.store_pos[q] : q;
        }
    }
    return (int)plan.size();
}

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
            if (!g.post.empty() || !g.swaps.empty()) { set_error("sv_batch_create: circuit %d has post-phases or a swap network (SV_FUSE_PHASES is for single states)", i); return SV_EINVAL; }
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
    std::vector<const FusedGate *> src;
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
            src.push_back(&g);
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
    b->src = std::move(src);
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
    b->opts.stage_log2 = 0;
    b->opts.stage_k = 0;
    b->opts.stage_layers = 0;
    b->opts.ctas_per_sm = 1;
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
    cudaFree(b->d_stages);
    cudaFree(b->d_chunks);
    cudaFree(b->d_sgates);
    cudaFree(b->d_smats);
    cudaFree(b->d_smaps);
    delete b;
}

extern "C" int sv_batch_set_opts(sv_batch *b, const sv_batch_opts *o)
{
    clear_error();
    if (!b || !o) { set_error("sv_batch_set_opts: NULL argument"); return SV_EINVAL; }
    SV_TRY(check_opts(*o));
    SV_TRY(set_smem_attrs(*o));
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
    SV_TRY(set_smem_attrs(b->opts));
    const int lcfg[7] = {b->opts.smem_max_n, b->opts.split_min_n, b->opts.tile_log2, b->opts.wave_mb, b->opts.stage_log2,
                         b->opts.stage_k, b->opts.stage_layers};
    const bool relist = !b->d_items || std::memcmp(lcfg, b->list_cfg, sizeof(lcfg)) != 0 || b->list_stall != b->stall;
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
    const int cfg[10] = {b->opts.threads, b->opts.smem_max_n, b->opts.ctas, b->opts.split_min_n, b->opts.tile_log2, b->opts.wave_mb,
                         b->opts.stage_log2, b->opts.stage_k, b->opts.stage_layers, b->opts.ctas_per_sm};
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

extern "C" int sv_batch_get_info(sv_batch *b, sv_batch_info *out)
{
    clear_error();
    if (!b || !out) { set_error("sv_batch_get_info: NULL argument"); return SV_EINVAL; }
    SV_TRY(check_opts(b->opts));
    const int lcfg[7] = {b->opts.smem_max_n, b->opts.split_min_n, b->opts.tile_log2, b->opts.wave_mb, b->opts.stage_log2,
                         b->opts.stage_k, b->opts.stage_layers};
    if (!b->d_items || std::memcmp(lcfg, b->list_cfg, sizeof(lcfg)) != 0 || b->list_stall != b->stall) {
        SV_CUDA_TRY(cudaStreamSynchronize(b->stream));   // a captured graph may still run on the old list
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        SV_TRY(build_work_list(b));
    }
    *out = b->info;
    return SV_OK;
}

extern "C" int sv_batch_state_offset(const sv_batch *b, int i, size_t *offset_bytes)
{
    clear_error();
    if (!b || !offset_bytes || i < 0 || i >= b->count) { set_error("sv_batch_state_offset: bad argument"); return SV_EINVAL; }
    *offset_bytes = sizeof(float) * (size_t)b->off[(size_t)i];
    return SV_OK;
}
