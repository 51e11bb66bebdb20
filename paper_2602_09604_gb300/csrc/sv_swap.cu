// Swap networks (SV_PATH_SWAPS): a fused gate made of disjoint two-qubit SWAP gates, applied in one
// in-place pass.  A SWAP of qubits a and b exchanges the amplitudes whose bits a and b differ
// (Eq. 3 with the SWAP matrix: c'_i = c_{P(i)}, P exchanging bits a and b of the index); a set of
// disjoint swaps is one bit permutation P of the index with P(P(i)) = i, so the pass reads every
// amplitude once and writes it once, whatever the number of swaps.
//
// Layout: blocks of 32 amplitudes (index bits 0-4 inside the block, 32 real parts then 32
// imaginary parts), block index = the bits from 5 up.  Pairs are of three kinds: both qubits
// below 5 (the amplitude moves inside its block), both at or above 5 (whole blocks move), one of
// each (the amplitude crosses blocks and in-block positions: a transpose).  A tile is the 2^tb
// blocks obtained by varying its local block bits: the block bits paired with in-block bits, then
// the lowest block bits that no swap touches or whose pair partner joins too (both bits of a
// block-bit pair), as room allows.  P maps a tile onto the tile whose base has the remaining
// block-bit pairs exchanged (its partner, perhaps itself), and each local amplitude to the same
// local position in every tile.  A CTA moves a tile and its partner through shared memory (all
// reads land before any write, so the pass is in place), with the reads of the next tiles in
// flight (cp.async, a ring of stages) while it writes the current one.
#include <algorithm>
#include <cstring>

#include "sv_internal.h"

namespace svg {
namespace {

constexpr int kSwapThreads = 512;
constexpr int kSwapStages = 6;
constexpr int kSwapStageBlocks = 64;   // 16 KB per stage: a tile pair of 2 x 32 blocks or one tile of 64
constexpr int kSwapCtasPerSm = 2;      // 2 x 5 stages of 16 KB in flight per SM
constexpr int kSwapMaxPairs = (SV_MAX_QUBITS + 1) / 2;
constexpr int kSwapChunksPerThread = kSwapStageBlocks * 16 / kSwapThreads;   // 16-byte chunks of a stage
constexpr int kSwapRowsPerWarp = kSwapStageBlocks * 2 / (kSwapThreads / 32);  // 128-byte rows of a stage

struct SwapArgs {
    int tb;                              // tile-local block bits
    int tpos[6];                         // block-index bit of local block bit c
    int n_loc;                           // pairs inside the tile, as local-index bits
    int loc_a[kSwapMaxPairs], loc_b[kSwapMaxPairs];   //   (0..4 in-block, 5 + c local block bit c)
    int n_x;                             // local block bits paired with in-block bits (bank swizzle)
    int x_c[5], x_l[5];
    int n_out;                           // block-bit pairs outside the tile
    int out_a[kSwapMaxPairs], out_b[kSwapMaxPairs];
    int n_o;                             // block-index bits outside the tile, ascending
    int opos[SV_MAX_QUBITS];
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(kSwapThreads, kSwapCtasPerSm) swap_kernel(float *__restrict__ sv, const __grid_constant__ SwapArgs a)
{
    extern __shared__ __align__(16) float smem[];
    const int nb = 1 << a.tb;   // blocks per tile
    float *stage = smem;        // kSwapStages x kSwapStageBlocks x 64 floats
    long long *toff = reinterpret_cast<long long *>(smem + kSwapStages * kSwapStageBlocks * 64);   // nb
    long long *meta = toff + nb;   // (kSwapStages + 1) x (base, partner): the tiles of the coming stages
    unsigned short *tab = reinterpret_cast<unsigned short *>(meta + 2 * (kSwapStages + 1) + 2 * a.n_o);   // nb * 32
    unsigned char *fsw = reinterpret_cast<unsigned char *>(tab + nb * 32);                     // nb
    // float offset of tile block t from the tile's base block, and its bank swizzle: the 16-byte
    // chunk j of block t's real (imaginary) half is stored at chunk j ^ fsw[t], fsw[t] = t's bits
    // paired with in-block bits 2..4 placed at those bits less 2.  The gather (a warp writes one
    // output block, its sources spread over blocks) then meets at most 2^(pairs on in-block bits
    // 0 and 1) lanes per bank.
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        long long o = 0;
        for (int i = 0; i < a.tb; ++i) o |= (long long)((t >> i) & 1) << a.tpos[i];
        toff[t] = o * 64;
        int g = 0;
        for (int i = 0; i < a.n_x; ++i)
            if (a.x_l[i] >= 2) g |= ((t >> a.x_c[i]) & 1) << (a.x_l[i] - 2);
        fsw[t] = (unsigned char)g;
    }
    __syncthreads();
    // source of output (t, p) in the source tile: its shared-memory float offset (without the half)
    for (int e = threadIdx.x; e < nb * 32; e += blockDim.x) {
        int x = e;   // local index: p in bits 0..4, t above
        for (int i = 0; i < a.n_loc; ++i)
            if (((x >> a.loc_a[i]) ^ (x >> a.loc_b[i])) & 1) x ^= (1 << a.loc_a[i]) | (1 << a.loc_b[i]);
        const int ts = x >> 5, ps = x & 31;
        tab[e] = (unsigned short)(ts * 64 + 4 * ((ps >> 2) ^ fsw[ts]) + (ps & 3));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int nw = kSwapThreads / 32;
    // thread 0 walks this CTA's contiguous range of tile ids and fills the stage table one stage
    // ahead of its copies.  base(u) deposits u's bits at opos; the partner is base ^ L(base), L
    // linear over GF(2) (each outside pair (x, y) adds x ^ y at both bits), so stepping u -> u + 1
    // (bits opos[0..k] toggle, k = the trailing ones of u) updates base and L(base) by two table
    // entries.
    long long *flip = meta + 2 * (kSwapStages + 1);   // n_o entries: toggled block bits
    long long *flipl = flip + a.n_o;                    // n_o entries: L of those
    const long long n_tiles = 1ll << a.n_o;
    const long long per = (n_tiles + gridDim.x - 1) / gridDim.x;
    long long u = (long long)blockIdx.x * per, u_end = u + per < n_tiles ? u + per : n_tiles;
    long long wb = 0, wl = 0;   // base(u) and L(base(u)), thread 0 only
    if (threadIdx.x == 0) {
        long long m = 0, l = 0;
        for (int i = 0; i < a.n_o; ++i) {
            const long long bit = 1ll << a.opos[i];
            long long lbit = 0;
            for (int j = 0; j < a.n_out; ++j)
                if (a.opos[i] == a.out_a[j] || a.opos[i] == a.out_b[j]) lbit = (1ll << a.out_a[j]) | (1ll << a.out_b[j]);
            m |= bit;
            l ^= lbit;
            flip[i] = m;
            flipl[i] = l;
            if ((u >> i) & 1) {
                wb |= bit;
                wl ^= lbit;
            }
        }
    }
    auto plan = [&](int j) {   // tile of stage j (a pair is moved from its smaller base)
        long long b = -1, p = -1;
        while (u < u_end) {
            const long long pp = wb ^ wl;
            const bool ok = pp >= wb;
            if (ok) {
                b = wb;
                p = pp;
            }
            const int k = __ffsll(~u) - 1;   // u -> u + 1 toggles opos[0..k]
            ++u;
            if (k < a.n_o) {
                wb ^= flip[k];
                wl ^= flipl[k];
            }
            if (ok) break;
        }
        meta[2 * (j % (kSwapStages + 1))] = b;
        meta[2 * (j % (kSwapStages + 1)) + 1] = p;
    };
    __syncthreads();   // tables ready
    // this thread's share of every stage is the same up to the tile bases: its copies (chunk q =
    // (tile s, block t, 16-byte chunk c16 of 16: real 0..7, imaginary 8..15)) and its output rows
    // (row r = (tile s, block t, half c); the warp's rows all have c = warp & 1), with offsets
    // taken once from the tables
    // (block offsets are kept as 32-bit block counts: a state has at most 2^30 blocks)
    const int c16 = threadIdx.x & 15;      // the same in every chunk of this thread
    uint32_t cdst[kSwapChunksPerThread];   // byte offset in the stage
    uint32_t cblk[kSwapChunksPerThread];   // block offset from the tile's base
#pragma unroll
    for (int j = 0; j < kSwapChunksPerThread; ++j) {
        const int q = threadIdx.x + kSwapThreads * j;
        const int sq = q >> (a.tb + 4), t = (q >> 4) & (nb - 1);
        cdst[j] = 16u * (uint32_t)((sq * nb + t) * 16 + (c16 ^ fsw[t]));
        cblk[j] = (uint32_t)(toff[t] >> 6);
    }
    const int cl = (warp & 1) * 32 + lane;   // the rows' half and lane: the same in every row
    uint32_t rsrc[kSwapRowsPerWarp];         // source float offset in the stage's tile
    uint32_t rblk[kSwapRowsPerWarp];         // block offset from the output tile's base
#pragma unroll
    for (int k = 0; k < kSwapRowsPerWarp; ++k) {
        const int r = warp + nw * k;
        const int t = (r >> 1) & (nb - 1);
        rsrc[k] = (uint32_t)(tab[t * 32 + lane] + (r & 1) * 32);
        rblk[k] = (uint32_t)(toff[t] >> 6);
    }
    // 16-byte copies of stage j's tile (and partner) into its slot
    auto issue = [&](int j) {
        const long long base = meta[2 * (j % (kSwapStages + 1))], part = meta[2 * (j % (kSwapStages + 1)) + 1];
        if (base >= 0) {
            const int chunks = (part == base ? 16 : 32) * nb;
            const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(stage + (j % kSwapStages) * kSwapStageBlocks * 64);
            const float *gb = sv + base * 64 + 4 * c16, *gp = sv + part * 64 + 4 * c16;
#pragma unroll
            for (int i = 0; i < kSwapChunksPerThread; ++i) {
                const int q = threadIdx.x + kSwapThreads * i;
                if (q < chunks) cp_async16(s0 + cdst[i], ((q >> (a.tb + 4)) ? gp : gb) + (size_t)cblk[i] * 64);
            }
        }
        cp_async_commit();   // one group per stage, empty or not
    };
    if (threadIdx.x == 0)
        for (int j = 0; j < kSwapStages; ++j) plan(j);
    __syncthreads();   // the first stages' tiles ready
#pragma unroll 1
    for (int j = 0; j < kSwapStages - 1; ++j) issue(j);
#pragma unroll 1
    for (int i = 0;; ++i) {
        cp_async_wait<kSwapStages - 2>();   // this thread's copies of stage i have landed
        __syncthreads();                    // everyone's have; stage i - 1 is no longer read
        const long long base = meta[2 * (i % (kSwapStages + 1))], part = meta[2 * (i % (kSwapStages + 1)) + 1];
        if (base < 0) break;   // no tile left (the same in every thread)
        issue(i + kSwapStages - 1);
        if (threadIdx.x == 0) plan(i + kSwapStages);
        // output tile s takes its amplitudes from the other tile (from itself when it is its own
        // partner)
        const float *buf = stage + (i % kSwapStages) * kSwapStageBlocks * 64;
        const int rows = (part == base ? 2 : 4) * nb;
        float *ob = sv + base * 64 + cl, *op = sv + part * 64 + cl;
        const float *other = part == base ? buf : buf + nb * 64;   // the source of the base tile's rows
#pragma unroll
        for (int k = 0; k < kSwapRowsPerWarp; ++k) {
            const int r = warp + nw * k;
            if (r < rows) {
                const bool s = (r >> (a.tb + 1)) != 0;
                (s ? op : ob)[(size_t)rblk[k] * 64] = (s ? buf : other)[rsrc[k]];
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace

int launch_swaps(float *sv, int n, const FusedGate &g, cudaStream_t stream, int num_sms)
{
    if (g.swaps.empty() || (int)g.swaps.size() > kSwapMaxPairs || n < 10 || n > SV_MAX_QUBITS) {
        set_error("launch: a swap network needs 1..%d pairs on a state of 10..%d qubits", kSwapMaxPairs, SV_MAX_QUBITS);
        return SV_EINVAL;
    }
    SwapArgs a;
    std::memset(&a, 0, sizeof(a));
    const int nbits = n - 5;   // block-index bits
    uint64_t used = 0;         // qubits named so far (the pairs must be disjoint)
    int partner[SV_MAX_QUBITS];
    for (int q = 0; q < SV_MAX_QUBITS; ++q) partner[q] = -1;
    for (const auto &pr : g.swaps) {
        const int x = std::min(pr.first, pr.second), y = std::max(pr.first, pr.second);
        if (x < 0 || y >= n || x == y || ((used >> x) & 1) || ((used >> y) & 1)) {
            set_error("launch: swap pairs must name distinct qubits below %d", n);
            return SV_EINVAL;
        }
        used |= (1ull << x) | (1ull << y);
        partner[x] = y;
        partner[y] = x;
    }
    // local block bits: the partners of in-block bits first, then the lowest block bits that no
    // swap touches or whose partner fits too; a tile and its partner fill one stage (a tile with
    // no block-bit pair left outside is its own partner and may fill it alone)
    int local_of[SV_MAX_QUBITS];   // qubit -> local index bit, or -1
    for (int q = 0; q < SV_MAX_QUBITS; ++q) local_of[q] = q < 5 ? q : -1;
    a.tb = 0;
    for (int q = 0; q < 5; ++q)
        if (partner[q] >= 5) {
            a.x_c[a.n_x] = a.tb;
            a.x_l[a.n_x] = q;
            ++a.n_x;
            local_of[partner[q]] = 5 + a.tb;
            a.tpos[a.tb++] = partner[q] - 5;
        }
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0 sizes the tile for pairs of tiles; pass 1 grows it by one bit when no block-bit
        // pair is left outside (the tile is its own partner)
        int out_left = 0;
        for (int q = 5; q < n; ++q) out_left += partner[q] > q && local_of[q] < 0;
        const int limit = (pass == 0 || out_left > 0) ? 5 : 6;
        for (int q = 5; q < n && a.tb < limit; ++q) {
            if (local_of[q] >= 0) continue;
            if (partner[q] < 0) {
                local_of[q] = 5 + a.tb;
                a.tpos[a.tb++] = q - 5;
            } else if (partner[q] > q && a.tb + 2 <= limit) {
                local_of[q] = 5 + a.tb;
                a.tpos[a.tb++] = q - 5;
                local_of[partner[q]] = 5 + a.tb;
                a.tpos[a.tb++] = partner[q] - 5;
            }
        }
    }
    for (int q = 0; q < n; ++q)
        if (partner[q] > q) {
            if (local_of[q] >= 0 && local_of[partner[q]] >= 0) {
                a.loc_a[a.n_loc] = local_of[q];
                a.loc_b[a.n_loc] = local_of[partner[q]];
                ++a.n_loc;
            } else {
                a.out_a[a.n_out] = q - 5;
                a.out_b[a.n_out] = partner[q] - 5;
                ++a.n_out;
            }
        }
    for (int b = 0; b < nbits; ++b)
        if (local_of[b + 5] < 0) a.opos[a.n_o++] = b;
    const int nb = 1 << a.tb;
    if ((a.n_out > 0 ? 2 : 1) * nb > kSwapStageBlocks) {
        set_error("launch: swap tile larger than a stage");
        return SV_EINVAL;
    }
    const size_t smem = (size_t)kSwapStages * kSwapStageBlocks * 64 * sizeof(float) + (size_t)nb * sizeof(long long) +
                        (size_t)(2 * (kSwapStages + 1) + 2 * a.n_o) * sizeof(long long) + (size_t)nb * 32 * sizeof(unsigned short) +
                        (size_t)nb;
    // the shared-memory limit is a per-device function attribute: set once per device
    static std::mutex mu;
    static uint64_t attr_set = 0;
    int dev = 0;
    SV_CUDA_TRY(cudaGetDevice(&dev));
    {
        const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
        std::lock_guard<std::mutex> lk(mu);
        if (!(attr_set & bit) || !bit) {
            SV_CUDA_TRY(cudaFuncSetAttribute(swap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((size_t)kSwapStages * kSwapStageBlocks * 64 * sizeof(float) + 8192)));
            attr_set |= bit;
        }
    }
    const long long n_tiles = 1ll << a.n_o;
    const long long grid = std::min<long long>(n_tiles, (long long)num_sms * kSwapCtasPerSm);
    swap_kernel<<<(unsigned)grid, kSwapThreads, smem, stream>>>(sv, a);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

}  // namespace svg
