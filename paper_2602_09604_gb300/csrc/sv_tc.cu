// Tensor-core path: a fused k-qubit gate (k = 4..6) as a real GEMM on the 5th-generation tensor
// cores (tcgen05, accumulators in tensor memory).
//
// Eq. 3 for all groups at once is the complex product Y = U X with X = [x_g] (2^k x 2^(n-k)).
// Written over the reals with the groups as rows:
//     Y^T[g, (c', r)] = sum_(c, j) X^T[g, (c, j)] * B[(c, j), (c', r)]
// where (c, j) indexes (real/imaginary part, amplitude j of the group) and
//     B[(0,j),(0,r)] = Re U[r][j]   B[(1,j),(0,r)] = -Im U[r][j]
//     B[(0,j),(1,r)] = Im U[r][j]   B[(1,j),(1,r)] =  Re U[r][j].
// One MMA tile is M = 128 groups, N = K = 2^(k+1).  Precision modes:
//   TF32   -- inputs rounded to tf32 (cvt.rna), one product, fp32 accumulation;
//   BF16X3 -- each operand split into bf16 hi + lo (lo = the rounded remainder), three products
//             hi*hi + hi*lo + lo*hi accumulated in fp32; the dropped lo*lo term and the split
//             remainders are ~2^-16 relative.
//
// Kernel forms (all persistent; B -- the gate's real block matrix, pre-split and pre-laid-out on the
// host in the tcgen05 K-major no-swizzle core-matrix layout -- is copied once per CTA into shared
// memory with a bulk asynchronous copy (TMA engine) completing on an mbarrier):
//   * two-warpgroup kernels (k = 4..6): each warpgroup is a pipeline over every other MMA tile of
//     the CTA: its threads load a tile's groups (direct: lane m owns group 128 t + m; staged:
//     through per-warp shared-memory tiles), write the A operand into tensor memory, one thread
//     issues the tcgen05.mma chain and commits it to an mbarrier, and the threads read the
//     accumulator back (tcgen05.ld) and store the outputs in place;
//   * the warp-specialised kernel (k = 6 with at most two targets below qubit 5): loader warps,
//     one MMA thread and epilogue warps connected by mbarriers, with A in a two-stage
//     shared-memory ring and four accumulators in tensor memory (see that kernel).
// Every mbarrier wait is bounded: on time-out the kernel records an error code in a device word,
// frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <exception>
#include <mutex>
#include <type_traits>

#include "sv_internal.h"

namespace svg {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;
constexpr long long kWaitIters = 4000000;   // ~0.3 s with the backoff below

enum : int { kModeTF32 = 0, kModeBF16X3 = 1 };

struct TcArgs {
    TileMap t;                 // per-warp tile geometry (f = k: 32 groups per warp tile), staged variant
    long long foff[64];        // direct variant: float offset of local amplitude j from the group base
    int tpos[SV_MAX_K];        // direct variant: ascending target qubits
    long long n_groups;        // 2^(n-k)
    long long n_mma_tiles;     // MMA tiles of 128 groups
    const void *bimg;          // device B image(s)
    unsigned bbytes;           // bytes of the B image(s)
    int *err;                  // device error word (bounded-wait time-outs)
    const float *ph;           // post-phases: angle tables [target][index byte][256]
    int ph_nb;                 // index bytes the tables cover
};

// Virtual source (direct kernels with VS): input amplitude i is src[offset(i) - off] when
// (i & mask) == rest and 0 otherwise; the outputs go to sv as usual.
struct VsArgs {
    const float *src;
    unsigned long long mask, rest;
    long long off;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false on time-out.
__device__ __noinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (long long i = 0; i < kWaitIters; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start >> 4 in bits 0-13, leading-dimension byte
// offset >> 4 in bits 16-29, stride-dimension byte offset >> 4 in bits 32-45, the fixed
// descriptor version 1 in bits 46-47, no base offset, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum)
{
    if constexpr (MODE == kModeTF32) {
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                     : "memory");
    } else {
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                     : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}


// 16 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t f32_to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// pack (x0 low, x1 high) to bf16x2 with round-to-nearest-even
__device__ __forceinline__ uint32_t pack_bf16x2(float x0, float x1)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ unsigned opaque_u32(unsigned v)
{
    asm volatile("mov.b32 %0, %0;" : "+r"(v));
    return v;
}

__device__ __forceinline__ unsigned long long ins0(unsigned long long x, int p)
{
    const unsigned long long low = x & ((1ull << p) - 1ull);
    return ((x >> p) << (p + 1)) | low;
}

template <int K, int MODE>
struct TcShape {
    static constexpr int D = 1 << K;             // amplitudes per group
    static constexpr int KD = 2 * D;             // GEMM K = N
    static constexpr int ESZ = MODE == kModeTF32 ? 4 : 2;
    static constexpr int NIMG = MODE == kModeTF32 ? 1 : 2;            // operand images (hi, lo)
    static constexpr int ROW_BYTES = KD * ESZ;                         // one B row
    static constexpr int EPC = 16 / ESZ;                               // elements per 16-byte core row
    static constexpr int B_IMG = KD * ROW_BYTES;                       // N = KD rows
    static constexpr int B_BYTES = NIMG * B_IMG;
    static constexpr int LBO_B = (KD / 8) * 128;                       // next 16-byte K chunk
    static constexpr int WTILE_FLOATS = 64 << K;                       // one warp tile: 2^k blocks
    // shared memory: B image(s), the eight warp tiles (staged variant only), barriers and status
    static constexpr int WBUF_BYTES_STAGED = 8 * WTILE_FLOATS * 4;
    static constexpr int SMEM_STAGED = B_BYTES + WBUF_BYTES_STAGED + 256;
    static constexpr int SMEM_DIRECT = B_BYTES + 256;   // the rest of the SM's 256 KB stays L1 cache
    static constexpr int CPL = (16 << K) / 32;                         // 16-byte chunks per lane
    static constexpr int A_COLS = KD * ESZ / 4;                        // TMEM columns of one A image
    static constexpr int WG_COLS = NIMG * A_COLS + KD;                 // A image(s) + accumulator
    static constexpr int TMEM_COLS = 2 * WG_COLS < 32 ? 32 : 2 * WG_COLS;   // two warpgroups
    static constexpr int KSTEP = MODE == kModeTF32 ? 8 : 16;           // K per instruction
    // warp-specialised kernel: A image(s) of one M = 128 tile in shared memory, K-major no-swizzle
    // core-matrix layout
    static constexpr int A_IMG_SMEM = kTcM * KD * ESZ;
    static constexpr int A_SMEM = NIMG * A_IMG_SMEM;
    static constexpr int LBO_A = (kTcM / 8) * 128;                     // next 16-byte K chunk of A
    // CTAs per SM the registers allow: the direct variant gains from more concurrent warpgroup
    // pipelines; the staged one needs more registers (its shared-memory traffic) and spills if capped
    static constexpr int MIN_BLOCKS_DIRECT = K == 6 ? 1 : (K == 5 ? 2 : 3);
    static constexpr int MIN_BLOCKS_STAGED = K == 6 ? 1 : (K == 5 ? 1 : 2);
};

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
        "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
        "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

template <int MODE>
__device__ __forceinline__ void mma_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t idesc, uint32_t accum)
{
    if constexpr (MODE == kModeTF32) {
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
                     "r"(tmem_a), "l"(bd), "r"(idesc), "r"(accum)
                     : "memory");
    } else {
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
                     "r"(tmem_a), "l"(bd), "r"(idesc), "r"(accum)
                     : "memory");
    }
}

__device__ __forceinline__ void wg_sync(int wg) { asm volatile("bar.sync %0, 128;" ::"r"(wg + 1) : "memory"); }

__device__ __forceinline__ float4 xor_perm4(float4 v, unsigned sw)
{
    if (sw & 1u) { float t = v.x; v.x = v.y; v.y = t; t = v.z; v.z = v.w; v.w = t; }
    if (sw & 2u) { float t = v.x; v.x = v.z; v.z = t; t = v.y; v.y = v.w; v.w = t; }
    return v;
}

// Two warpgroups per CTA, each an independent pipeline over every other MMA tile of the CTA,
// sharing the B operand in shared memory.
//
// DIRECT variant (at most two targets below qubit 5): row m of MMA tile t is group 128 t + m and
// each lane loads its group straight into registers (the next tile's loads are issued before the
// current tile's epilogue) and stores its outputs straight back.  With no low target a warp's 32
// groups are the 32 positions of one block, so every warp access is a whole 128-byte line; with
// one or two, an access spans two or four lines whose other parts the neighbouring amplitudes'
// accesses take (from L1 for loads; merged in L2 for stores).
//
// STAGED variant (three or more targets below qubit 5): an MMA tile is four warp tiles; a warp tile is the
// 2^k blocks holding 32 groups (the tile geometry of the CUDA-core tile kernel with f = k), so
// global memory is still read and written in whole 128-byte lines.
// Per warp and tile:
//   1. the next warp tile's 16-byte chunks are loaded into registers before the current tile's
//      epilogue (2 x 128 threads x 2^(k+1) floats in flight per CTA);
//   2. the epilogue reads the accumulator (tcgen05.ld) into the group's places of the warp's
//      shared-memory tile, which then goes back to global memory with 16-byte stores;
//   3. the prefetched chunks are stored XOR-swizzled into the warp's tile (bank-conflict-free
//      group reads), and each lane streams its A row, 32 tensor-memory columns at a time, into
//      the warpgroup's A region (tcgen05.st);
//   4. one thread per warpgroup issues the MMAs (A from tensor memory, B from shared memory).
// VS (direct variant only): inputs from the virtual source v instead of sv.  The body is inlined
// into two entry points so the kernels without a virtual source keep their own parameter block.
template <int K, int MODE, bool STAGED, bool VS>
__device__ __forceinline__ void tc_kernel_body(float *__restrict__ sv, const TcArgs &a, const VsArgs &v)
{
    using S = TcShape<K, MODE>;
    constexpr int D = S::D;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sB = smem;
    const int tid = threadIdx.x;
    const int wg = tid >> 7;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    float *wbuf = reinterpret_cast<float *>(smem + S::B_BYTES) + warp * S::WTILE_FLOATS;   // staged only
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + S::B_BYTES + (STAGED ? S::WBUF_BYTES_STAGED : 0));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 4);
    volatile int *status = reinterpret_cast<volatile int *>(tslot + 1);   // [0], [1]: per warpgroup
    const uint32_t bar_b = smem_u32(&bars[0]);
    const uint32_t bar_mma = smem_u32(&bars[1 + wg]);

    if (tid == 0) {
        mbar_init(bar_b, 1);
        mbar_init(smem_u32(&bars[1]), 1);
        mbar_init(smem_u32(&bars[2]), 1);
        status[0] = 0;
        status[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"((uint32_t)S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t t_wg = tmem + (uint32_t)(wg * S::WG_COLS);        // this warpgroup's columns
    const uint32_t t_lane = ((uint32_t)((warp & 3) * 32)) << 16;     // this warp's lane quarter
    const uint32_t tA = t_wg;                                         // A image(s)
    const uint32_t tD = t_wg + (uint32_t)(S::NIMG * S::A_COLS);      // accumulator

    if (tid == 0) {   // B image: bulk copies of up to 32 KB, all completing on bar_b
        mbar_arrive_expect_tx(bar_b, a.bbytes);
        for (unsigned off = 0; off < a.bbytes; off += 32768u) {
            const unsigned sz = a.bbytes - off < 32768u ? a.bbytes - off : 32768u;
            bulk_g2s(smem_u32(sB + off), static_cast<const unsigned char *>(a.bimg) + off, sz, bar_b);
        }
    }

    const uint32_t idesc = (1u << 4) | ((MODE == kModeTF32 ? 2u : 1u) << 7) | ((MODE == kModeTF32 ? 2u : 1u) << 10) |
                           ((uint32_t)(S::KD >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

    // this lane's group inside the warp tile (fixed for every tile)
    unsigned gbase = (unsigned)lane;
#pragma unroll
    for (int b = 0; b < K; ++b) gbase = (unsigned)ins0(gbase, a.t.ltpos[b]);
    const unsigned gsw = a.t.gswz[(lane >> a.t.lsh) & a.t.lmask];
    // shared-memory float offset of the group's real part j (gb: gbase through an opaque move,
    // so the offsets are recomputed per use rather than held in registers across the tile loop)
    auto spos = [&](unsigned gb, int j) -> unsigned {   // bitwise maps on disjoint bits: one XOR
        return (((gb >> 5) << 6) | ((gb & 31u) ^ gsw)) ^ (unsigned)a.t.loffo[j];
    };
    auto tile_block0 = [&](long long wt) -> unsigned long long {
        unsigned long long b0 = (unsigned long long)wt;
#pragma unroll
        for (int i = 0; i < K; ++i) b0 = ins0(b0, a.t.fpos[i]);
        return b0;
    };
    auto gchunk = [&](unsigned long long b0, int c) -> float * {
        return sv + (long long)((b0 + (unsigned long long)a.t.fblk[c >> 4]) << 6) + (c & 15) * 4;
    };
    auto schunk = [&](int c, unsigned &sw) -> float * {
        sw = a.t.swz[c >> 4];
        return wbuf + (c >> 4) * 64 + (c & 8) * 4 + (((c & 7) ^ (int)(sw >> 2)) << 2);
    };

    // ---- direct variant: the lane's group in registers
    float xd[STAGED ? 1 : 2 * D];
    long long fb_next = 0, fb_cur = 0;
    bool v_next = false, v_cur = false;
    auto load_direct = [&](long long tile) {
        if constexpr (!STAGED) {
            const long long g = tile * kTcM + (tid & 127);
            v_next = g < a.n_groups;
            fb_next = 0;
            if (v_next) {
                unsigned long long b = (unsigned long long)g;
#pragma unroll
                for (int i = 0; i < K; ++i) b = ins0(b, a.tpos[i]);
                fb_next = (long long)(((b >> 5) << 6) | (b & 31ull));
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    if constexpr (VS) {
                        unsigned long long ij = b;   // index of local amplitude j
#pragma unroll
                        for (int i = 0; i < K; ++i)
                            if ((j >> i) & 1) ij |= 1ull << a.tpos[i];
                        const bool in = (ij & v.mask) == v.rest;
                        xd[j] = in ? v.src[fb_next + a.foff[j] - v.off] : 0.f;
                        xd[D + j] = in ? v.src[fb_next + a.foff[j] + 32 - v.off] : 0.f;
                    } else {
                        xd[j] = sv[fb_next + a.foff[j]];
                        xd[D + j] = sv[fb_next + a.foff[j] + 32];
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 2 * D; ++j) xd[j] = 0.f;
            }
        }
    };
    float4 pre[STAGED ? S::CPL : 1];
    auto prefetch = [&](long long wt) {
        if constexpr (!STAGED) {
            (void)wt;
        } else if (wt < a.t.n_tiles) {
            const unsigned long long b0 = tile_block0(wt);
            const int ln = (int)opaque_u32((unsigned)lane);
#pragma unroll
            for (int i = 0; i < S::CPL; ++i) pre[i] = *reinterpret_cast<const float4 *>(gchunk(b0, ln + 32 * i));
        } else {
#pragma unroll
            for (int i = 0; i < S::CPL; ++i) pre[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto fetch = [&](long long tile) {   // next MMA tile's inputs, either variant
        if constexpr (STAGED) prefetch(4 * tile + (warp & 3));
        else load_direct(tile);
    };
    // prefetched chunks -> swizzled warp tile -> this lane's A row in tensor memory
    auto stage_and_write_a = [&]() {
        if constexpr (STAGED) {
            const int ln = (int)opaque_u32((unsigned)lane);
#pragma unroll
            for (int i = 0; i < S::CPL; ++i) {
                unsigned sw;
                float *d = schunk(ln + 32 * i, sw);
                *reinterpret_cast<float4 *>(d) = xor_perm4(pre[i], sw);
            }
            __syncwarp();
        }
        const unsigned gb = opaque_u32(gbase);
        // A row element kk = (c, j): kk < D real part of amplitude kk, else imaginary part of kk - D
        auto elem = [&](int kk) -> float {
            if constexpr (STAGED) return wbuf[spos(gb, kk % D) + (kk >= D ? 32 : 0)];
            else return xd[kk];
        };
        if constexpr (MODE == kModeTF32) {
#pragma unroll
            for (int cb = 0; cb < S::KD / 32; ++cb) {
                uint32_t r[32];
#pragma unroll
                for (int i = 0; i < 32; ++i) r[i] = f32_to_tf32(elem(cb * 32 + i));
                tmem_st32(tA + t_lane + cb * 32, r);
            }
        } else {
            // a 32-bit column holds two bf16 elements: element 2c in the low half of column c
            constexpr int NC = 16;   // columns per chunk (32 elements): keeps the live set small
#pragma unroll
            for (int cb = 0; cb < S::KD / (2 * NC); ++cb) {
                float xs[2 * NC];
#pragma unroll
                for (int e = 0; e < 2 * NC; ++e) xs[e] = elem(cb * 2 * NC + e);
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    uint32_t r[32];
#pragma unroll
                    for (int c = 0; c < 32; ++c) {
                        if (c < NC) {
                            const float x0 = xs[2 * c], x1 = xs[2 * c + 1];
                            const uint32_t hi = pack_bf16x2(x0, x1);
                            if (part == 0) {
                                r[c] = hi;
                            } else {
                                const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xffff0000u);
                                r[c] = pack_bf16x2(x0 - h0, x1 - h1);
                            }
                        } else {
                            r[c] = 0u;
                        }
                    }
                    tmem_st16(tA + t_lane + (uint32_t)(part * S::A_COLS + cb * NC), r);
                }
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    };
    auto issue_mma = [&]() {   // one thread per warpgroup
        const uint32_t b0 = smem_u32(sB);
        constexpr int NSTEP = S::KD / S::KSTEP;
        constexpr int ACOL = S::KSTEP * S::ESZ / 4;     // TMEM columns per instruction (8)
        constexpr int CH = S::KSTEP / S::EPC;           // 16-byte chunks of B per instruction (2)
        if constexpr (MODE == kModeTF32) {
#pragma unroll
            for (int st = 0; st < NSTEP; ++st)
                mma_ta<MODE>(tD, tA + st * ACOL, sdesc(b0 + st * CH * S::LBO_B, S::LBO_B, 128), idesc, st > 0);
        } else {
            const uint32_t a_img[3] = {tA, tA, tA + (uint32_t)S::A_COLS};   // hi, hi, lo
            const uint32_t b_img[3] = {b0, b0 + (uint32_t)S::B_IMG, b0};     // hi, lo, hi
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int st = 0; st < NSTEP; ++st)
                    mma_ta<MODE>(tD, a_img[p] + st * ACOL, sdesc(b_img[p] + st * CH * S::LBO_B, S::LBO_B, 128), idesc,
                                 (p > 0 || st > 0));
        }
        mma_commit(bar_mma);
    };
    // accumulator -> the group's places in the warp tile -> global memory (16-byte stores)
    auto epilogue_direct = [&]() {
#pragma unroll
        for (int cb = 0; cb < S::KD / 16; ++cb) {
            float v[16];
            tmem_ld16(tD + t_lane + cb * 16, v);
            if (v_cur) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int col = cb * 16 + i;           // column (c', r): c' = col / D, r = col % D
                    sv[fb_cur + a.foff[col % D] + (col >= D ? 32 : 0)] = v[i];
                }
            }
        }
    };
    auto epilogue = [&](long long wt) {
#pragma unroll
        for (int cb = 0; cb < S::KD / 16; ++cb) {
            float v[16];
            tmem_ld16(tD + t_lane + cb * 16, v);
            const unsigned gb = opaque_u32(gbase);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int col = cb * 16 + i;           // column (c', r): c' = col / D, r = col % D
                wbuf[spos(gb, col % D) + (col >= D ? 32 : 0)] = v[i];
            }
        }
        __syncwarp();
        if (wt < a.t.n_tiles) {
            const unsigned long long b0 = tile_block0(wt);
            const int ln = (int)opaque_u32((unsigned)lane);
            // ordered batches of four shared loads then four global stores (volatile asm keeps
            // the order), so at most 16 registers of copy data are live
#pragma unroll
            for (int i0 = 0; i0 < S::CPL; i0 += 4) {
                float4 v[4];
                unsigned sw[4];
#pragma unroll
                for (int q = 0; q < 4 && i0 + q < S::CPL; ++q) {
                    const float *src = schunk(ln + 32 * (i0 + q), sw[q]);
                    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                                 : "=f"(v[q].x), "=f"(v[q].y), "=f"(v[q].z), "=f"(v[q].w)
                                 : "r"(smem_u32(src)));
                }
#pragma unroll
                for (int q = 0; q < 4 && i0 + q < S::CPL; ++q) {
                    const float4 w = xor_perm4(v[q], sw[q]);
                    asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(gchunk(b0, ln + 32 * (i0 + q))), "f"(w.x),
                                 "f"(w.y), "f"(w.z), "f"(w.w)
                                 : "memory");
                }
            }
        }
        __syncwarp();
    };

    // MMA tiles of this warpgroup: blockIdx.x + (2 i + wg) * gridDim.x; warp tile = 4 * tile + (warp & 3)
    const long long tstride = 2ll * gridDim.x;
    long long tile = blockIdx.x + (long long)wg * gridDim.x;
    uint32_t phase = 0u;
    bool ok = true;
    const bool lead = (tid & 127) == 0;
    if (tile < a.n_mma_tiles) {
        fetch(tile);
        fb_cur = fb_next;
        v_cur = v_next;
        stage_and_write_a();
        tc_fence_before();
        wg_sync(wg);
        if (lead) {
            tc_fence_after();
            if (!mbar_wait_bounded(bar_b, 0)) status[wg] = 1;
            else issue_mma();
        }
        wg_sync(wg);
        ok = status[wg] == 0;
    }
    while (ok && tile < a.n_mma_tiles) {
        const long long nt = tile + tstride;
        if (nt < a.n_mma_tiles) fetch(nt);                    // in flight during the wait + epilogue
        if (lead && !mbar_wait_bounded(bar_mma, phase)) status[wg] = 2;
        wg_sync(wg);
        if (status[wg] != 0) { ok = false; break; }
        phase ^= 1u;
        tc_fence_after();
        if constexpr (STAGED) epilogue(4 * tile + (warp & 3));   // reads D; MMA(nt) writes D after the sync
        else epilogue_direct();
        fb_cur = fb_next;
        v_cur = v_next;
        if (nt < a.n_mma_tiles) stage_and_write_a();          // A region is free: MMA(tile) completed
        tc_fence_before();
        wg_sync(wg);
        if (nt < a.n_mma_tiles && lead) {
            tc_fence_after();
            issue_mma();
        }
        tile = nt;
    }
    if (!ok && lead) atomicOr(a.err, status[wg] == 1 ? 0x10 : 0x20);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::TMEM_COLS) : "memory");
    }
}

template <int K, int MODE, bool STAGED>
__global__ void __launch_bounds__(2 * kTcThreads, STAGED ? TcShape<K, MODE>::MIN_BLOCKS_STAGED : TcShape<K, MODE>::MIN_BLOCKS_DIRECT)
    apply_tc_kernel(float *__restrict__ sv, const __grid_constant__ TcArgs a)
{
    tc_kernel_body<K, MODE, STAGED, false>(sv, a, VsArgs{});
}

template <int K, int MODE>
__global__ void __launch_bounds__(2 * kTcThreads, TcShape<K, MODE>::MIN_BLOCKS_DIRECT)
    apply_tc_kernel_vs(float *__restrict__ sv, const __grid_constant__ TcArgs a, const __grid_constant__ VsArgs v)
{
    tc_kernel_body<K, MODE, false, true>(sv, a, v);
}

// ------------------------------------------------------------------------ warp-specialised kernel
// k = 6 gates on the direct (lane-per-group) access pattern, with the work split by role so that
// loads are always in flight.  One persistent CTA per SM walks its MMA tiles i = 0, 1, ...
// (tile blockIdx.x + i * gridDim.x, 128 groups each):
//   * LW loader warps: warp w owns rows 32 (w % 4) .. +31 of every tile and a slice of each row's
//     amplitudes; per tile it converts its registers (bf16 hi/lo split, or tf32) into the A image of
//     shared-memory stage i % 2 (K-major core-matrix layout) and, chunk by chunk, reloads them with
//     the next tile's amplitudes, so the next tile's loads are in flight while this one converts
//     and while the warp waits for a free stage;
//   * one MMA thread: per tile it waits for the stage and for a free accumulator (four in tensor
//     memory, 128 columns each), issues the products and commits them to the stage's "empty" and
//     the accumulator's "full" barriers;
//   * EW epilogue warps (warp index % 4 = the tensor-memory lane quarter they may read): per tile
//     they read the accumulator (tcgen05.ld) and store the outputs in place, then free it.
// A tile depends only on earlier tiles' barrier phases, so the pipeline cannot deadlock.  Every
// wait is bounded; a role that gives up sets a shared abort flag (the others stop at their next
// wait) and the device error word; the MMA thread then waits (bounded) for its products to
// complete before tensor memory is freed.
constexpr int kWsStages = 2;   // A stages in shared memory (64 KB each)
constexpr int kWsAcc = 4;      // accumulators in tensor memory (4 x 128 columns: all 512)

template <int MODE>
struct WsShape {
    using S = TcShape<6, MODE>;
    static constexpr int A_STAGE = S::A_SMEM;
    static constexpr int OFF_A = S::B_BYTES;
    static constexpr int OFF_BAR = S::B_BYTES + kWsStages * A_STAGE;
    static constexpr int N_BAR = 1 + 2 * kWsStages + 2 * kWsAcc + 1;   // b, a full/empty, acc full/empty, drain
    static constexpr int SMEM = OFF_BAR + N_BAR * 8 + 16;
    static constexpr int TMEM_COLS = kWsAcc * S::KD;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane.
// two loads of 16 columns each (a, b), one wait for both
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float (&va)[16], float (&vb)[16])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        va[i] = __uint_as_float(r[i]);
        vb[i] = __uint_as_float(r[16 + i]);
    }
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int MODE, bool VS, int LW, int EW, int WIN, bool V4, bool PH = false>
__device__ __forceinline__ void tc_ws_body(float *__restrict__ sv, const TcArgs &a, const VsArgs &v)
{
    using S = TcShape<6, MODE>;
    using W = WsShape<MODE>;
    constexpr int K = 6, D = 64;
    constexpr int MMA_WARP = LW + EW;
    static_assert(LW % 4 == 0 && (D / (LW / 4)) % 8 == 0, "loader warps: whole row quarters, 8-amplitude chunks");
    static_assert(EW == 4 || EW == 8, "epilogue warps: one or two per lane quarter");
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + W::OFF_BAR);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + W::N_BAR);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const uint32_t bar_b = smem_u32(&bars[0]);
    const uint32_t bar_afull = smem_u32(&bars[1]);                            // + 8 s
    const uint32_t bar_aempty = smem_u32(&bars[1 + kWsStages]);               // + 8 s
    const uint32_t bar_accfull = smem_u32(&bars[1 + 2 * kWsStages]);          // + 8 c
    const uint32_t bar_accempty = smem_u32(&bars[1 + 2 * kWsStages + kWsAcc]);   // + 8 c
    const uint32_t bar_drain = smem_u32(&bars[W::N_BAR - 1]);
    const uint32_t sA0 = smem_u32(smem + W::OFF_A);

    if (threadIdx.x == 0) {
        mbar_init(bar_b, 1);
        for (int s = 0; s < kWsStages; ++s) {
            mbar_init(bar_afull + 8 * s, LW * 32);
            mbar_init(bar_aempty + 8 * s, 1);
        }
        for (int c = 0; c < kWsAcc; ++c) {
            mbar_init(bar_accfull + 8 * c, 1);
            mbar_init(bar_accempty + 8 * c, EW * 32);
        }
        mbar_init(bar_drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"((uint32_t)W::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const long long ntile = a.n_mma_tiles;
    const long long cnt = (long long)blockIdx.x < ntile ? (ntile - 1 - (long long)blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](long long i) -> long long { return (long long)blockIdx.x + i * (long long)gridDim.x; };
    // bounded wait; gives up early once another role has given up
    auto wait = [&](uint32_t bar, uint32_t parity, int code) -> bool {
        for (long long it = 0; it < kWaitIters; ++it) {
            if (mbar_try_wait(bar, parity)) return true;
            if (*abort_flag) return false;
            if (it > 32) __nanosleep(64);
        }
        *abort_flag = 1;
        atomicOr(a.err, code);
        return false;
    };
    // group 128 * tile + m: index with zeros at the targets (b) and its float offset (fb)
    auto group_base = [&](long long tile, int m, unsigned long long &b, long long &fb) -> bool {
        const long long g = tile * kTcM + m;
        b = (unsigned long long)g;
#pragma unroll
        for (int i = 0; i < K; ++i) b = ins0(b, a.tpos[i]);
        fb = (long long)(((b >> 5) << 6) | (b & 31ull));
        return g < a.n_groups;
    };

    if (warp < LW) {
        // ------------------------------------------------------------------ loaders
        constexpr int AMPS = D / (LW / 4);   // amplitudes of a row this lane converts
        constexpr int CH = AMPS / 8;         // chunks of 8 amplitudes (16 floats in registers each)
        const int m = 32 * (warp & 3) + lane;
        const int j_lo = (warp >> 2) * AMPS;
        const uint32_t row_off = (uint32_t)((m >> 3) * 128 + (m & 7) * 16);
        float xr[WIN][CH][16];   // WIN tiles' slices in flight
        auto load_chunk = [&](float (&x)[CH][16], bool valid, unsigned long long b, long long fb, int c) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = j_lo + 8 * c + e;
                if constexpr (VS) {
                    const long long fo = a.foff[j];
                    const unsigned long long ij = b | ((unsigned long long)(fo >> 6) << 5) | (unsigned long long)(fo & 31);
                    const bool in = valid && (ij & v.mask) == v.rest;
                    x[c][e] = in ? v.src[fb + fo - v.off] : 0.f;
                    x[c][8 + e] = in ? v.src[fb + fo + 32 - v.off] : 0.f;
                } else if constexpr (V4) {
                    // targets 0 and 1: members j .. j + 3 are four consecutive floats (16-byte aligned)
                    if (e % 4 == 0) {
                        float4 re = make_float4(0.f, 0.f, 0.f, 0.f), im = re;
                        if (valid) {
                            re = *reinterpret_cast<const float4 *>(sv + fb + a.foff[j]);
                            im = *reinterpret_cast<const float4 *>(sv + fb + a.foff[j] + 32);
                        }
                        x[c][e] = re.x; x[c][e + 1] = re.y; x[c][e + 2] = re.z; x[c][e + 3] = re.w;
                        x[c][8 + e] = im.x; x[c][9 + e] = im.y; x[c][10 + e] = im.z; x[c][11 + e] = im.w;
                    }
                } else {
                    x[c][e] = valid ? sv[fb + a.foff[j]] : 0.f;
                    x[c][8 + e] = valid ? sv[fb + a.foff[j] + 32] : 0.f;
                }
            }
        };
        auto st16 = [](uint32_t addr, uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3) {
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(w0), "r"(w1), "r"(w2), "r"(w3) : "memory");
        };
        // chunk c of this lane's row into the A image(s) at stage base sa: element kk of the row is
        // the real part of amplitude kk (kk < 64) or the imaginary part of amplitude kk - 64
        auto convert_chunk = [&](const float (&x)[CH][16], int c, uint32_t sa) {
            const int j0 = j_lo + 8 * c;
#pragma unroll
            for (int part = 0; part < 2; ++part) {   // real, imaginary
                if constexpr (MODE == kModeTF32) {
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        const int kc = (64 * part + j0 + 4 * hf) / 4;
                        const float *xx = &x[c][8 * part + 4 * hf];
                        st16(sa + (uint32_t)(kc * S::LBO_A) + row_off, f32_to_tf32(xx[0]), f32_to_tf32(xx[1]),
                             f32_to_tf32(xx[2]), f32_to_tf32(xx[3]));
                    }
                } else {
                    uint32_t hi[4], lo[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float x0 = x[c][8 * part + 2 * q], x1 = x[c][8 * part + 2 * q + 1];
                        hi[q] = pack_bf16x2(x0, x1);   // element 2q in the low half
                        const float h0 = __uint_as_float(hi[q] << 16), h1 = __uint_as_float(hi[q] & 0xffff0000u);
                        lo[q] = pack_bf16x2(x0 - h0, x1 - h1);
                    }
                    const uint32_t o = (uint32_t)(((64 * part + j0) / 8) * S::LBO_A) + row_off;
                    st16(sa + o, hi[0], hi[1], hi[2], hi[3]);
                    st16(sa + (uint32_t)S::A_IMG_SMEM + o, lo[0], lo[1], lo[2], lo[3]);
                }
            }
        };
        unsigned long long b_n = 0;
        long long fb_n = 0;
        bool v_n = false;
#pragma unroll
        for (int w = 0; w < WIN; ++w)   // the first WIN tiles' loads
            if (w < cnt) {
                v_n = group_base(tile_of(w), m, b_n, fb_n);
#pragma unroll
                for (int c = 0; c < CH; ++c) load_chunk(xr[w], v_n, b_n, fb_n, c);
            }
        bool go = true;
        for (long long i0 = 0; go && i0 < cnt; i0 += WIN) {
#pragma unroll
            for (int w = 0; w < WIN; ++w) {
                const long long i = i0 + w;
                if (!go || i >= cnt) break;
                const int s = (int)(i % kWsStages);
                const bool more = i + WIN < cnt;
                if (more) v_n = group_base(tile_of(i + WIN), m, b_n, fb_n);
                if (i >= kWsStages && !wait(bar_aempty + 8 * s, (uint32_t)((i / kWsStages - 1) & 1), 0x40)) {
                    go = false;
                    break;
                }
                const uint32_t sa = sA0 + (uint32_t)(s * W::A_STAGE);
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    convert_chunk(xr[w], c, sa);
                    if (more) load_chunk(xr[w], v_n, b_n, fb_n, c);   // tile i + WIN's chunk, in flight from here
                }
                fence_proxy_async();   // generic-proxy stores -> read by the tensor core (async proxy)
                mbar_arrive(bar_afull + 8 * s);
            }
        }
    } else if (warp < MMA_WARP) {
        // ------------------------------------------------------------------ epilogue
        const int quarter = warp & 3;
        const int part = (warp - LW) >> 2;   // EW = 8: which half of the columns
        const int m = 32 * quarter + lane;
        const uint32_t t_lane = ((uint32_t)(quarter * 32)) << 16;
        for (long long i = 0; i < cnt; ++i) {
            const int c = (int)(i % kWsAcc);
            unsigned long long b;
            long long fb;
            const bool valid = group_base(tile_of(i), m, b, fb);
            // post-phases: output member r of group b times exp(i sum_{t: r_t = 1} phi_t(b)), with
            // phi_t(b) = the sum of target t's table entries over b's index bytes (b has zeros at the
            // targets): every table read in flight at once, before the wait for the accumulator
            float er[PH ? K : 1], ei[PH ? K : 1];
            if constexpr (PH) {
                constexpr int kMaxBytes = 5;   // indices of up to 40 bits
                float tab[K][kMaxBytes];
#pragma unroll
                for (int t = 0; t < K; ++t)
#pragma unroll
                    for (int cbyte = 0; cbyte < kMaxBytes; ++cbyte)
                        tab[t][cbyte] = (valid && cbyte < a.ph_nb)
                                             ? __ldg(a.ph + (t * a.ph_nb + cbyte) * 256 + (int)((b >> (8 * cbyte)) & 255ull))
                                             : 0.f;
#pragma unroll
                for (int t = 0; t < K; ++t) {
                    const float phi = ((tab[t][0] + tab[t][1]) + (tab[t][2] + tab[t][3])) + tab[t][4];
                    // |phi| <= 5 pi: less the nearest multiple of 2 pi (2 pi split into a float
                    // and its remainder, so r keeps the rounding of phi), then the hardware
                    // sine and cosine, whose absolute error on [-pi, pi] is below 1e-6, scaled
                    // back to unit modulus (the phases keep the state's norm)
                    const float k = rintf(phi * 0.15915494309189535f);
                    const float r = fmaf(-k, -1.7484555e-07f, fmaf(-k, 6.28318548f, phi));
                    float sn, cs;
                    __sincosf(r, &sn, &cs);
                    const float inv = rsqrtf(fmaf(cs, cs, sn * sn));
                    er[t] = cs * inv;
                    ei[t] = sn * inv;
                }
            }
            if (!wait(bar_accfull + 8 * c, (uint32_t)((i / kWsAcc) & 1), 0x20)) break;
            tc_fence_after();
            const uint32_t td = tmem + (uint32_t)(c * S::KD) + t_lane;
            if constexpr (PH) {
                // members in Gray-code order, one complex product each; chunk qc = members
                // 16 qc .. 16 qc + 15 (columns: real, then + 64 imaginary), a compile-time index
                // so that the member offsets are immediate operands and e_t stays in registers
                auto chunk = [&](auto qc_c) {
                    constexpr int qc = decltype(qc_c)::value;
                    float ore[16], oim[16];
                    tmem_ld16x2(td + (uint32_t)(16 * qc), td + (uint32_t)(64 + 16 * qc), ore, oim);
                    if (valid) {
                        // the chunk's members share bits 4 and 5 (= qc)
                        float fr = 1.f, fi = 0.f;
                        if constexpr ((qc & 1) != 0) {
                            fr = er[4];
                            fi = ei[4];
                        }
                        if constexpr ((qc & 2) != 0) {
                            const float nr = fr * er[5] - fi * ei[5], ni = fr * ei[5] + fi * er[5];
                            fr = nr;
                            fi = ni;
                        }
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int x = i ^ (i >> 1);
                            if (i > 0) {   // bit t of the member changed: times e_t or its conjugate
                                const int t = (i & 1) ? 0 : (i & 2) ? 1 : (i & 4) ? 2 : 3;
                                const float si = ((x >> t) & 1) ? ei[t] : -ei[t];
                                const float nr = fr * er[t] - fi * si, ni = fr * si + fi * er[t];
                                fr = nr;
                                fi = ni;
                            }
                            const float yr = ore[x] * fr - oim[x] * fi, yi = ore[x] * fi + oim[x] * fr;
                            sv[fb + a.foff[16 * qc + x]] = yr;
                            sv[fb + a.foff[16 * qc + x] + 32] = yi;
                        }
                    }
                };
                if constexpr (EW == 8) {   // two warps per lane quarter, each with half of the members
                    if (part == 0) {
                        chunk(std::integral_constant<int, 0>{});
                        chunk(std::integral_constant<int, 1>{});
                    } else {
                        chunk(std::integral_constant<int, 2>{});
                        chunk(std::integral_constant<int, 3>{});
                    }
                } else {
                    chunk(std::integral_constant<int, 0>{});
                    chunk(std::integral_constant<int, 1>{});
                    chunk(std::integral_constant<int, 2>{});
                    chunk(std::integral_constant<int, 3>{});
                }
            } else {
            constexpr int NB = EW == 4 ? 4 : 2;   // 32-column blocks this warp reads
#pragma unroll
            for (int cb = 0; cb < NB; ++cb) {
                // EW = 4: blocks 0..3 (columns 0..127); EW = 8: real block `part`, imaginary block 2 + part
                const int blk = EW == 4 ? cb : (cb == 0 ? part : 2 + part);
                float o[32];
                tmem_ld32(td + (uint32_t)(32 * blk), o);
                if (valid) {
#pragma unroll
                    for (int x = 0; x < 32; ++x) {
                        const int col = 32 * blk + x;   // (c', r): c' = col / 64, r = col % 64
                        sv[fb + a.foff[col % D] + (col >= D ? 32 : 0)] = o[x];
                    }
                }
            }
            }
            tc_fence_before();
            mbar_arrive(bar_accempty + 8 * c);
        }
    } else if (lane == 0) {
        // ------------------------------------------------------------------ MMA issue
        const uint32_t idesc = (1u << 4) | ((MODE == kModeTF32 ? 2u : 1u) << 7) | ((MODE == kModeTF32 ? 2u : 1u) << 10) |
                               ((uint32_t)(S::KD >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
        const uint32_t b0 = smem_u32(smem);
        bool b_done = false;
        if (cnt > 0) {   // B image: bulk copies of up to 32 KB, all completing on bar_b
            mbar_arrive_expect_tx(bar_b, a.bbytes);
            for (unsigned off = 0; off < a.bbytes; off += 32768u) {
                const unsigned sz = a.bbytes - off < 32768u ? a.bbytes - off : 32768u;
                bulk_g2s(b0 + off, static_cast<const unsigned char *>(a.bimg) + off, sz, bar_b);
            }
            b_done = wait(bar_b, 0, 0x10);
        }
        for (long long i = 0; b_done && i < cnt; ++i) {
            const int s = (int)(i % kWsStages), c = (int)(i % kWsAcc);
            if (!wait(bar_afull + 8 * s, (uint32_t)((i / kWsStages) & 1), 0x20)) break;
            if (i >= kWsAcc && !wait(bar_accempty + 8 * c, (uint32_t)((i / kWsAcc - 1) & 1), 0x20)) break;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(c * S::KD);
            const uint32_t sa = sA0 + (uint32_t)(s * W::A_STAGE);
            constexpr int NSTEP = S::KD / S::KSTEP;
            constexpr int CHS = S::KSTEP / S::EPC;   // 16-byte chunks per instruction (2)
            if constexpr (MODE == kModeTF32) {
#pragma unroll
                for (int st = 0; st < NSTEP; ++st)
                    mma<MODE>(d, sdesc(sa + st * CHS * S::LBO_A, S::LBO_A, 128), sdesc(b0 + st * CHS * S::LBO_B, S::LBO_B, 128),
                              idesc, st > 0);
            } else {
                const uint32_t a_img[3] = {sa, sa, sa + (uint32_t)S::A_IMG_SMEM};   // hi, hi, lo
                const uint32_t b_img[3] = {b0, b0 + (uint32_t)S::B_IMG, b0};        // hi, lo, hi
#pragma unroll
                for (int p = 0; p < 3; ++p)
#pragma unroll
                    for (int st = 0; st < NSTEP; ++st)
                        mma<MODE>(d, sdesc(a_img[p] + st * CHS * S::LBO_A, S::LBO_A, 128),
                                  sdesc(b_img[p] + st * CHS * S::LBO_B, S::LBO_B, 128), idesc, (p > 0 || st > 0));
            }
            mma_commit(bar_aempty + 8 * s);   // the stage may be overwritten once these products are done
            mma_commit(bar_accfull + 8 * c);
        }
        // every product issued above completes before tensor memory is freed, and the B copy
        // before its shared memory is released (bounded: the error word records a give-up)
        mma_commit(bar_drain);
        if (!mbar_wait_bounded(bar_drain, 0)) atomicOr(a.err, 0x80);
        if (cnt > 0 && !b_done && !mbar_wait_bounded(bar_b, 0)) atomicOr(a.err, 0x80);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)W::TMEM_COLS) : "memory");
    }
}

constexpr int kWsLoadWarps = 16;
constexpr int kWsEpiWarps = 4;
constexpr int kWsWindow = 1;   // tiles whose loads each loader lane keeps in flight
constexpr int kWsThreads = (kWsLoadWarps + kWsEpiWarps + 1) * 32;

// V4: the gate's two lowest targets are qubits 0 and 1, so the loaders move four members of a group
// with one 16-byte access (a warp's accesses are then whole lines)
template <int MODE, bool V4>
__global__ void __launch_bounds__(kWsThreads, 1) apply_tc_ws_kernel(float *__restrict__ sv, const __grid_constant__ TcArgs a)
{
    tc_ws_body<MODE, false, kWsLoadWarps, kWsEpiWarps, kWsWindow, V4>(sv, a, VsArgs{});
}

template <int MODE>
__global__ void __launch_bounds__(kWsThreads, 1)
    apply_tc_ws_kernel_vs(float *__restrict__ sv, const __grid_constant__ TcArgs a, const __grid_constant__ VsArgs v)
{
    tc_ws_body<MODE, true, kWsLoadWarps, kWsEpiWarps, kWsWindow, false>(sv, a, v);
}

// k = 6, at most two targets below qubit 5 (not both 0 and 1), with post-phases in the epilogue:
// one epilogue warp per tensor-memory lane quarter, as without them (two per quarter, 800 threads
// at 72 registers, gave the loaders fewer registers and ran 2% slower)
constexpr int kWsPhEpiWarps = 4;
constexpr int kWsPhThreads = (kWsLoadWarps + kWsPhEpiWarps + 1) * 32;
template <int MODE>
__global__ void __launch_bounds__(kWsPhThreads, 1) apply_tc_ws_kernel_ph(float *__restrict__ sv, const __grid_constant__ TcArgs a)
{
    tc_ws_body<MODE, false, kWsLoadWarps, kWsPhEpiWarps, kWsWindow, false, true>(sv, a, VsArgs{});
}

// ---------------------------------------------------------------------------------------- host
uint16_t bf16_rn(double v)
{
    // round an fp64 value to bf16 (nearest, ties to even) through fp32: exact enough for |v| <= 1
    // matrix entries (double rounding only matters within 2^-29 of a tie).
    float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}
double bf16_to_d(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}
uint32_t tf32_rna(double v)
{
    float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    return u;
}

template <int ESZ>
uint32_t host_core_off(int row, int kk, int rows)
{
    constexpr int EPC = 16 / ESZ;
    const int kc = kk / EPC, e = kk % EPC;
    return (uint32_t)((kc * (rows / 8) + (row >> 3)) * 128 + (row & 7) * 16 + e * ESZ);
}

// Bytes of the B image(s) of a k-qubit gate in `mode` (a multiple of 128 for k >= 4).
size_t b_image_bytes(int k, int mode)
{
    const size_t KD = size_t(2) << k;
    return mode == kModeTF32 ? KD * KD * 4 : 2 * KD * KD * 2;
}

// Post-phase tables after a gate's B image (16-byte aligned): for target t and index byte c,
// entry v = the sum of the angles of the terms on target t whose qubit is bit (q - 8c) of v,
// reduced to (-pi, pi] in fp64 before rounding.
size_t ph_table_offset(int k, int mode) { return (b_image_bytes(k, mode) + 15) & ~size_t(15); }
size_t ph_table_bytes(int k, int n) { return sizeof(float) * (size_t)k * (size_t)((n + 7) / 8) * 256; }

void write_ph_tables(const FusedGate &g, int n, float *out)
{
    const int nb = (n + 7) / 8;
    for (int t = 0; t < g.k; ++t)
        for (int c = 0; c < nb; ++c)
            for (int v = 0; v < 256; ++v) {
                double s = 0.0;
                for (const FusedGate::PostTerm &pt : g.post)
                    if (pt.j == t && pt.q >= 8 * c && pt.q < 8 * c + 8 && ((v >> (pt.q - 8 * c)) & 1)) s += pt.theta;
                s = std::remainder(s, 2.0 * M_PI);
                out[(t * nb + c) * 256 + v] = (float)s;
            }
}


// B image(s) of one gate in the tcgen05 K-major no-swizzle layout (rows = output columns (c', r),
// K = input columns (c, j)), written to img (b_image_bytes(g.k, mode) bytes, every byte set).
void write_b_image(const FusedGate &g, int mode, unsigned char *img)
{
    const int D = 1 << g.k, KD = 2 * D;
    auto B = [&](int kk, int nn) -> double {
        const int c = kk / D, j = kk % D, cp = nn / D, r = nn % D;
        const cplx u = g.mat[size_t(r) * D + j];
        if (c == 0 && cp == 0) return u.real();
        if (c == 1 && cp == 0) return -u.imag();
        if (c == 0 && cp == 1) return u.imag();
        return u.real();
    };
    if (mode == kModeTF32) {
        for (int nn = 0; nn < KD; ++nn)
            for (int kk = 0; kk < KD; ++kk) {
                const uint32_t v = tf32_rna(B(kk, nn));
                std::memcpy(&img[host_core_off<4>(nn, kk, KD)], &v, 4);
            }
        return;
    }
    const size_t one = size_t(KD) * KD * 2;
    for (int nn = 0; nn < KD; ++nn)
        for (int kk = 0; kk < KD; ++kk) {
            const double v = B(kk, nn);
            const uint16_t hi = bf16_rn(v);
            const uint16_t lo = bf16_rn(v - bf16_to_d(hi));
            const uint32_t o = host_core_off<2>(nn, kk, KD);
            std::memcpy(&img[o], &hi, 2);
            std::memcpy(&img[one + o], &lo, 2);
        }
}

int *g_err_word[64] = {};
std::mutex g_tc_mu;

}  // namespace

int device_err_word(int **out)
{
    int dev = 0;
    SV_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tc_mu);
    if (dev < 0 || dev >= 64) { set_error("tc: device id out of range"); return SV_EINVAL; }
    if (!g_err_word[dev]) {
        SV_CUDA_TRY(cudaMalloc(&g_err_word[dev], sizeof(int)));
        SV_CUDA_TRY(cudaMemset(g_err_word[dev], 0, sizeof(int)));
    }
    *out = g_err_word[dev];
    return SV_OK;
}

namespace {

// Kernel form of a tensor-core gate, decided by its targets below qubit 5 (they lie inside a
// 32-amplitude block).  One function decides for the launcher and for tc_gate_is_direct.
//   1 (staged): three or more such targets -- lane-per-group accesses would span >= 8 lines, so
//     data moves through the per-warp shared-memory tiles (measured at n = 30, k = 6: staged 4.47
//     TB/s, warp-specialised 2.66, two-warpgroup direct 2.3-3.9);
//   2 (warp-specialised, k = 6): at most two such targets (k = 6 at n = 30: no low target
//     6.54-6.75 TB/s against 5.83-6.15 for the two-warpgroup kernel with A in shared memory; one
//     at qubit 0: 6.51 vs 5.54; two: 6.00 vs 5.35);
//   0 (two-warpgroup direct, A in tensor memory): k = 4 and 5 with at most two such targets
//     (6.4-6.6 TB/s: four warpgroup pipelines per SM already hide the latency there).
int tc_variant(const FusedGate &g)
{
    int nlow = 0;
    for (int b = 0; b < g.k; ++b) nlow += g.targets[b] < 5;
    if (nlow >= 3) return 1;
    return g.k == 6 ? 2 : 0;
}

template <int K, int MODE>
int launch_tc_t(float *sv, int n, const FusedGate &g, const void *dtc, cudaStream_t stream, int num_sms, const TcSource *vs)
{
    using S = TcShape<K, MODE>;
    if (n < K + 5) { set_error("tensor-core path needs n >= k + 5 (n=%d, k=%d)", n, K); return SV_EINVAL; }
    const int variant = tc_variant(g);
    const bool staged = variant == 1;
    TcArgs a;
    std::memset(&a, 0, sizeof(a));
    SV_TRY(make_tile_map(g, n, K, &a.t));
    for (int b = 0; b < K; ++b) a.tpos[b] = g.targets[b];
    for (int j = 0; j < (1 << K); ++j) {
        unsigned long long o = 0;
        for (int b = 0; b < K; ++b)
            if ((j >> b) & 1) o |= 1ull << g.targets[b];
        a.foff[j] = (long long)(((o >> 5) << 6) | (o & 31ull));
    }
    a.n_groups = 1ll << (n - K);
    a.n_mma_tiles = staged ? (a.t.n_tiles + 3) / 4 : (a.n_groups + kTcM - 1) / kTcM;
    a.bimg = dtc;
    a.bbytes = (unsigned)S::B_BYTES;
    SV_TRY(device_err_word(&a.err));
    if (vs && staged) { set_error("tensor-core gate: a virtual source needs a direct variant"); return SV_EINVAL; }
    const bool ph = !g.post.empty();
    if (ph) {
        if (K != 6 || variant != 2 || vs || (g.targets[0] == 0 && g.targets[1] == 1)) {
            set_error("tensor-core gate: post-phases need a k = 6 gate on the warp-specialised kernel");
            return SV_EINVAL;
        }
        a.ph = reinterpret_cast<const float *>(static_cast<const unsigned char *>(dtc) + ph_table_offset(K, MODE));
        a.ph_nb = (n + 7) / 8;
    }
    VsArgs v{};
    if (vs) v = VsArgs{vs->src, vs->mask, vs->rest, vs->off};
    void (*kern)(float *, const TcArgs) = staged ? apply_tc_kernel<K, MODE, true> : apply_tc_kernel<K, MODE, false>;
    void (*kern_vs)(float *, const TcArgs, const VsArgs) = apply_tc_kernel_vs<K, MODE>;
    int smem = staged ? S::SMEM_STAGED : S::SMEM_DIRECT;
    int tmem_cols = S::TMEM_COLS;
    int threads = 2 * kTcThreads;
    int per_sm_regs = staged ? S::MIN_BLOCKS_STAGED : S::MIN_BLOCKS_DIRECT;
    if constexpr (K == 6) {   // the warp-specialised kernel exists for k = 6 only
        if (variant == 2) {
            const bool v4 = g.targets[0] == 0 && g.targets[1] == 1;
            kern = ph ? apply_tc_ws_kernel_ph<MODE> : v4 ? apply_tc_ws_kernel<MODE, true> : apply_tc_ws_kernel<MODE, false>;
            kern_vs = apply_tc_ws_kernel_vs<MODE>;
            smem = WsShape<MODE>::SMEM;
            tmem_cols = WsShape<MODE>::TMEM_COLS;
            threads = ph ? kWsPhThreads : kWsThreads;
            per_sm_regs = 1;
        }
    }
    // function-attribute slot: variant, virtual source, 16-byte loaders, post-phases
    const int akey = ph ? 9 : variant + (vs ? 3 : 0) + (variant == 2 && !vs && g.targets[0] == 0 && g.targets[1] == 1 ? 6 : 0);
    static uint64_t attr_set[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};   // per kernel form, a bit per device (attributes are per device)
    {
        int dev = 0;
        SV_CUDA_TRY(cudaGetDevice(&dev));
        const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
        std::lock_guard<std::mutex> lk(g_tc_mu);
        if (!(attr_set[akey] & bit) || !bit) {
            if (vs) SV_CUDA_TRY(cudaFuncSetAttribute(kern_vs, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            else SV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            attr_set[akey] |= bit;
        }
    }
    // CTAs per SM bounded by registers, shared memory and tensor memory (512 columns)
    const int by_tmem = std::max(1, 512 / tmem_cols);
    const int by_smem = std::max(1, (227 * 1024) / (smem + 1024));
    const int per_sm = std::min(per_sm_regs, std::min(by_tmem, by_smem));
    // the two-warpgroup kernels take two MMA tiles per CTA round, the warp-specialised one one
    const long long tiles_per_cta = variant == 2 ? 1 : 2;
    const long long grid = std::min<long long>((a.n_mma_tiles + tiles_per_cta - 1) / tiles_per_cta, (long long)num_sms * per_sm);
    if (vs) kern_vs<<<(unsigned)grid, threads, smem, stream>>>(sv, a, v);
    else kern<<<(unsigned)grid, threads, smem, stream>>>(sv, a);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

}  // namespace

int plan_tc_operands(sv_fused *f, size_t *bytes)
{
    f->tc_offset.assign(f->gates.size(), SIZE_MAX);
    size_t total = 0;   // each tensor-core gate's images at a 128-byte aligned offset
    for (size_t i = 0; i < f->gates.size(); ++i) {
        const FusedGate &g = f->gates[i];
        if (g.path != SV_PATH_TC_TF32 && g.path != SV_PATH_TC_BF16X3) continue;
        if (g.k < 4 || g.k > 6) {
            set_error("tensor-core path handles fused gates of 4 to 6 qubits (gate %zu has %d)", i, g.k);
            return SV_EINVAL;
        }
        f->tc_offset[i] = (total + 127) & ~size_t(127);
        const int mode = g.path == SV_PATH_TC_TF32 ? kModeTF32 : kModeBF16X3;
        total = f->tc_offset[i] + b_image_bytes(g.k, mode);
        if (!g.post.empty()) total = f->tc_offset[i] + ph_table_offset(g.k, mode) + ph_table_bytes(g.k, f->n);
    }
    *bytes = total;
    return SV_OK;
}

int write_tc_operands(const sv_fused *f, unsigned char *dst)
{
    std::vector<size_t> tc;
    for (size_t i = 0; i < f->gates.size(); ++i)
        if (f->tc_offset[i] != SIZE_MAX) tc.push_back(i);
    try {
        // the gates' images are independent: built on host threads (a k = 6 image is 32 K elements)
        host_parallel_for(tc.size(), (tc.size() + 3) / 4, [&](size_t t) {
            const FusedGate &g = f->gates[tc[t]];
            const int mode = g.path == SV_PATH_TC_TF32 ? kModeTF32 : kModeBF16X3;
            write_b_image(g, mode, dst + f->tc_offset[tc[t]]);
            if (!g.post.empty()) write_ph_tables(g, f->n, reinterpret_cast<float *>(dst + f->tc_offset[tc[t]] + ph_table_offset(g.k, mode)));
        });
    } catch (const std::exception &e) {
        set_error("tensor-core operand images: %s", e.what());
        return SV_ENOMEM;
    }
    return SV_OK;
}

bool tc_gate_is_direct(const FusedGate &g)
{
    return (g.path == SV_PATH_TC_TF32 || g.path == SV_PATH_TC_BF16X3) && g.k >= 4 && g.k <= 6 && tc_variant(g) != 1;
}

int launch_tc_gate(float *sv, int n, const FusedGate &g, const void *dtc, cudaStream_t stream, int num_sms, const TcSource *vs)
{
    if (!dtc) { set_error("tensor-core gate has no device operand image"); return SV_EINVAL; }
    const bool tf = g.path == SV_PATH_TC_TF32;
    switch (g.k) {
    case 4: return tf ? launch_tc_t<4, kModeTF32>(sv, n, g, dtc, stream, num_sms, vs) : launch_tc_t<4, kModeBF16X3>(sv, n, g, dtc, stream, num_sms, vs);
    case 5: return tf ? launch_tc_t<5, kModeTF32>(sv, n, g, dtc, stream, num_sms, vs) : launch_tc_t<5, kModeBF16X3>(sv, n, g, dtc, stream, num_sms, vs);
    case 6: return tf ? launch_tc_t<6, kModeTF32>(sv, n, g, dtc, stream, num_sms, vs) : launch_tc_t<6, kModeBF16X3>(sv, n, g, dtc, stream, num_sms, vs);
    default: set_error("tensor-core path handles k = 4..6, got %d", g.k); return SV_EINVAL;
    }
}

int read_device_errors(int *code)
{
    *code = 0;
    int dev = 0;
    SV_CUDA_TRY(cudaGetDevice(&dev));
    int *w = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_tc_mu);
        if (dev >= 0 && dev < 64) w = g_err_word[dev];
    }
    if (!w) return SV_OK;
    SV_CUDA_TRY(cudaMemcpy(code, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (*code) SV_CUDA_TRY(cudaMemset(w, 0, sizeof(int)));
    return SV_OK;
}

}  // namespace svg
