// Expectation values of Pauli strings, <psi|P|psi>, as a read-only reduction over the state.
//
// Section IV runs ExpectationValue with the same group loop as ApplyGate but reduces the result
// instead of storing it back.  For a Pauli string the "matrix-vector product" of a group is a
// signed, phased permutation, so the reduction needs no matrix at all.  Write the string as two
// bit masks over the qubits: x (X or Y on that qubit) and z (Z or Y).  With Y = i X Z,
//     P |j> = i^popc(x & z) (-1)^popc(j & z) |j ^ x>,
//     <psi|P|psi> = i^popc(x & z) * S,   S = sum_j (-1)^popc(j & z) conj(c_(j^x)) c_j.
// P is Hermitian, so the value is real: Re S, -Im S, -Re S or Im S for popc(x & z) = 0, 1, 2, 3
// (mod 4); each string accumulates only the component it needs.
//
// Strings with the same x read the same pairs of amplitudes, so up to kEvMaxStrings of them are
// evaluated in one pass: each amplitude is read once, its term conj(c_(j^x)) c_j is formed once in
// fp32, and every string adds it with its own sign into a float-float accumulator (two-sum); the
// per-thread results are combined in fp64, per CTA and then by the last CTA in a fixed order
// (strided per-thread sums, then a fixed-shape tree), so results are deterministic.
//
// Work unit = one block (x has no bit >= 5) or one pair of blocks b, b ^ (x >> 5) with bit
// `pair_bit` of b clear (otherwise); a warp reads each block's 32 real and 32 imaginary parts with
// coalesced loads, and the partner amplitude j ^ x inside the paired block comes from lane
// (lane ^ (x & 31)) through a shuffle.  A warp takes 32 consecutive units and handles them in
// batches of 8 (eight blocks or pairs of loads in flight per warp).  Signs are bit lookups: for
// unit u of a range starting at u0 (a multiple of 32), parity(b & zb) = parity(u0 & zu) ^ bit
// (u - u0) of a 32-bit parity table of zu's low five bits, where zu is zb with the pair bit
// deleted (b is u with a zero inserted there); these bits are the same in every lane.  The lane
// part parity(lane & zl) is fixed per thread and applied once at the end.  Each string sums a
// batch's signed terms in fp32 (with four or more strings, through one 8-point Walsh-Hadamard
// transform of the batch that serves every string), then adds the batch sum to its float-float
// accumulator.
#include <algorithm>
#include <cstring>
#include <vector>

#include "sv_internal.h"

namespace svg {
namespace {

constexpr int kEvThreads = 256;
constexpr int kEvMaxStrings = 8;

struct EvArgs {
    long long n_units;        // blocks, or block pairs
    unsigned long long xb;    // x >> 5
    int xl;                   // x & 31
    int pair_bit;             // bit of the block index inserted as 0 to enumerate pairs; -1: no pairing
    unsigned long long zu[kEvMaxStrings];   // z >> 5 with the pair bit deleted (unit-index parity mask)
    unsigned ztab[kEvMaxStrings];           // bit i = parity(i & zu & 31), i < 32
    unsigned zc[kEvMaxStrings];             // zu & 7: the Walsh-Hadamard entry of a batch of 8 units
    unsigned zl[kEvMaxStrings];             // z & 31
    unsigned pairpar[kEvMaxStrings];        // parity((x >> 5) & (z >> 5)): sign change to the paired block
    int comp[kEvMaxStrings];  // 0: accumulate the real part of the term, 1: the imaginary part
    int m;                    // strings in this pass (<= the kernel's M; the rest are padding)
};

struct FF2 {
    float hi, lo;
};

__device__ __forceinline__ void ff_add(FF2 &a, float x)
{
    const float s = a.hi + x;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (x - bp);
    a.hi = s;
    a.lo += e;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long ins_zero(unsigned long long v, int p)
{
    const unsigned long long low = v & ((1ull << p) - 1ull);
    return ((v >> p) << (p + 1)) | low;
}

constexpr int kEvBatch = 8;     // units per batch

// in place: w[c] <- sum_i (-1)^popc(i & c) w[i]
__device__ __forceinline__ void wht8(float (&w)[8])
{
#pragma unroll
    for (int h = 1; h < 8; h <<= 1)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (!(i & h)) {
                const float x = w[i], y = w[i + h];
                w[i] = x + y;
                w[i + h] = x - y;
            }
}

// w[c] for a warp-uniform c < 8 without indexing a register array (three levels of selects)
__device__ __forceinline__ float sel8(const float (&w)[8], unsigned c)
{
    const float a0 = (c & 1u) ? w[1] : w[0], a1 = (c & 1u) ? w[3] : w[2];
    const float a2 = (c & 1u) ? w[5] : w[4], a3 = (c & 1u) ? w[7] : w[6];
    const float b0 = (c & 2u) ? a1 : a0, b1 = (c & 2u) ? a3 : a2;
    return (c & 4u) ? b1 : b0;
}
constexpr int kEvRange = 32;    // units per warp range (one parity table)

template <int M, bool PAIRED>
__global__ void __launch_bounds__(kEvThreads, M >= 4 ? 3 : 4) expval_kernel(const float *__restrict__ sv, const __grid_constant__ EvArgs a,
                                                           double *__restrict__ partials, unsigned *__restrict__ counter,
                                                           double *__restrict__ result)
{
    FF2 acc[M];
#pragma unroll
    for (int p = 0; p < M; ++p) acc[p] = FF2{0.f, 0.f};
    const unsigned lane = threadIdx.x & 31u;
    const unsigned plane = lane ^ (unsigned)a.xl;
    const long long n_ranges = (a.n_units + kEvRange - 1) / kEvRange;
    const long long wstride = (long long)gridDim.x * (kEvThreads / 32);
    for (long long r = (long long)blockIdx.x * (kEvThreads / 32) + (threadIdx.x >> 5); r < n_ranges; r += wstride) {
        const long long u0 = r * kEvRange;
        unsigned sgn0[M];   // block-parity sign bit of the range base, per string (warp-uniform)
#pragma unroll
        for (int p = 0; p < M; ++p) sgn0[p] = (unsigned)(__popcll((unsigned long long)u0 & a.zu[p]) & 1) << 31;
#pragma unroll 1
        for (int bt = 0; bt < kEvRange / kEvBatch; ++bt) {
            float ur[kEvBatch], ui[kEvBatch], vr[kEvBatch], vi[kEvBatch];
#pragma unroll
            for (int i = 0; i < kEvBatch; ++i) {
                const long long u = u0 + bt * kEvBatch + i;
                ur[i] = ui[i] = vr[i] = vi[i] = 0.f;
                if (u < a.n_units) {
                    const unsigned long long b = PAIRED ? ins_zero((unsigned long long)u, a.pair_bit) : (unsigned long long)u;
                    ur[i] = __ldcs(sv + b * 64 + lane);
                    ui[i] = __ldcs(sv + b * 64 + 32 + lane);
                    if constexpr (PAIRED) {
                        const unsigned long long b2 = b ^ a.xb;
                        vr[i] = __ldcs(sv + b2 * 64 + lane);
                        vi[i] = __ldcs(sv + b2 * 64 + 32 + lane);
                    }
                }
            }
            float tr[kEvBatch], ti[kEvBatch], sr[kEvBatch], si[kEvBatch];
#pragma unroll
            for (int i = 0; i < kEvBatch; ++i) {
                if constexpr (PAIRED) {
                    const float vpr = __shfl_sync(0xffffffffu, vr[i], plane), vpi = __shfl_sync(0xffffffffu, vi[i], plane);
                    const float upr = __shfl_sync(0xffffffffu, ur[i], plane), upi = __shfl_sync(0xffffffffu, ui[i], plane);
                    // j in block b (partner in b2) and j' in block b2 (partner in b)
                    tr[i] = fmaf(vpr, ur[i], vpi * ui[i]);
                    ti[i] = fmaf(vpr, ui[i], -(vpi * ur[i]));
                    sr[i] = fmaf(upr, vr[i], upi * vi[i]);
                    si[i] = fmaf(upr, vi[i], -(upi * vr[i]));
                } else {
                    const float pr = __shfl_sync(0xffffffffu, ur[i], plane), pi = __shfl_sync(0xffffffffu, ui[i], plane);
                    tr[i] = fmaf(pr, ur[i], pi * ui[i]);
                    ti[i] = fmaf(pr, ui[i], -(pi * ur[i]));
                }
            }
            if constexpr (M >= 4) {
                // many strings: an 8-point Walsh-Hadamard transform of the batch's terms gives,
                // for every mask c of the batch's unit bits, the sum of the terms signed by
                // parity(i & c); string p then takes entry zu & 7, signed by the batch's base parity
                wht8(tr);
                wht8(ti);
                if constexpr (PAIRED) {
                    wht8(sr);
                    wht8(si);
                }
#pragma unroll
                for (int p = 0; p < M; ++p) {
                    const unsigned c = a.zc[p];
                    const unsigned sg = sgn0[p] ^ (((a.ztab[p] >> (bt * kEvBatch)) & 1u) << 31);
                    float v = a.comp[p] ? sel8(ti, c) : sel8(tr, c);
                    if constexpr (PAIRED) {
                        const float w = a.comp[p] ? sel8(si, c) : sel8(sr, c);
                        v += __uint_as_float(__float_as_uint(w) ^ (a.pairpar[p] << 31));
                    }
                    ff_add(acc[p], __uint_as_float(__float_as_uint(v) ^ sg));
                }
            } else {
#pragma unroll
                for (int p = 0; p < M; ++p) {
                    // block-parity sign bits of the batch's units: warp-uniform; the lane's own
                    // parity (lane & zl) is applied once at the end
                    const unsigned tab = a.ztab[p] >> (bt * kEvBatch);
                    float sum = 0.f;
                    if (a.comp[p] == 0) {
#pragma unroll
                        for (int i = 0; i < kEvBatch; ++i) {
                            const unsigned sg = sgn0[p] ^ (((tab >> i) & 1u) << 31);
                            sum += __uint_as_float(__float_as_uint(tr[i]) ^ sg);
                            if constexpr (PAIRED) sum += __uint_as_float(__float_as_uint(sr[i]) ^ sg ^ (a.pairpar[p] << 31));
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < kEvBatch; ++i) {
                            const unsigned sg = sgn0[p] ^ (((tab >> i) & 1u) << 31);
                            sum += __uint_as_float(__float_as_uint(ti[i]) ^ sg);
                            if constexpr (PAIRED) sum += __uint_as_float(__float_as_uint(si[i]) ^ sg ^ (a.pairpar[p] << 31));
                        }
                    }
                    ff_add(acc[p], sum);
                }
            }
        }
    }
    // the lane's parity(lane & zl) sign, common to every term this thread added
#pragma unroll
    for (int p = 0; p < M; ++p)
        if (__popc(lane & a.zl[p]) & 1) {
            acc[p].hi = -acc[p].hi;
            acc[p].lo = -acc[p].lo;
        }
    __shared__ double ws[kEvThreads / 32][M];
    __shared__ bool last;
#pragma unroll
    for (int p = 0; p < M; ++p) {
        const double v = warp_sum((double)acc[p].hi + (double)acc[p].lo);
        if (lane == 0) ws[threadIdx.x >> 5][p] = v;
    }
    __syncthreads();
    if (threadIdx.x < M) {
        double s = 0.0;
        for (int w = 0; w < kEvThreads / 32; ++w) s += ws[w][threadIdx.x];
        partials[(size_t)blockIdx.x * M + threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(counter, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // last CTA: every thread sums a fixed strided subset of the partials, then a fixed-shape tree
    __threadfence();
    __shared__ double red[kEvThreads][M];
    {
        const volatile double *pp = partials;
        double s[M];
#pragma unroll
        for (int p = 0; p < M; ++p) s[p] = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += kEvThreads)
#pragma unroll
            for (int p = 0; p < M; ++p) s[p] += pp[(size_t)i * M + p];
#pragma unroll
        for (int p = 0; p < M; ++p) red[threadIdx.x][p] = s[p];
    }
    __syncthreads();
    for (int w = kEvThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int p = 0; p < M; ++p) red[threadIdx.x][p] += red[threadIdx.x + w][p];
        __syncthreads();
    }
    if ((int)threadIdx.x < a.m) result[threadIdx.x] = red[0][threadIdx.x];
    if (threadIdx.x == 0) *counter = 0u;   // ready for the next launch
}

// The grid is one wave of resident CTAs (occupancy x SMs), capped by the work and by max_grid:
// every CTA then loops over an equal share of the ranges with no second, partly filled wave.
template <int M>
int launch_ev(const float *sv, const EvArgs &a, double *partials, unsigned *counter, double *result, long long work_ctas,
              int num_sms, int max_grid, cudaStream_t s)
{
    auto kern = a.pair_bit >= 0 ? expval_kernel<M, true> : expval_kernel<M, false>;
    int per_sm = 1;
    SV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kEvThreads, 0));
    long long g = (long long)num_sms * (per_sm > 0 ? per_sm : 1);
    if (g > max_grid) g = max_grid;
    if (g > work_ctas) g = work_ctas;
    if (g < 1) g = 1;
    kern<<<(unsigned)g, kEvThreads, 0, s>>>(sv, a, partials, counter, result);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

int highest_bit(unsigned long long v)
{
    int h = -1;
    while (v) {
        ++h;
        v >>= 1;
    }
    return h;
}

}  // namespace
}  // namespace svg

using namespace svg;

extern "C" int sv_expval_pauli(const sv_state *st_c, const uint64_t *x_masks, const uint64_t *z_masks, int count, double *out)
{
    clear_error();
    sv_state *st = const_cast<sv_state *>(st_c);
    if (!st || count < 0 || (count > 0 && (!x_masks || !z_masks || !out))) { set_error("sv_expval_pauli: bad argument"); return SV_EINVAL; }
    if (st->c128) { set_error("sv_expval_pauli: expectation values need a complex64 state"); return SV_EINVAL; }
    if (count == 0) return SV_OK;
    const int n = st->n;
    const uint64_t valid = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
    for (int i = 0; i < count; ++i)
        if ((x_masks[i] | z_masks[i]) & ~valid) {
            set_error("sv_expval_pauli: string %d acts on a qubit >= n = %d", i, n);
            return SV_EINVAL;
        }
    // workspace: per-CTA partials for one launch, a counter, and one result per string
    const int max_grid = st->num_sms * 8;
    if (count > st->ev_capacity) {
        cudaStreamSynchronize(st->stream);
        cudaFree(st->d_ev);
        st->d_ev = nullptr;
        st->ev_capacity = 0;
        const size_t doubles = (size_t)max_grid * kEvMaxStrings + (size_t)count + 1;
        cudaError_t e = cudaMalloc(&st->d_ev, sizeof(double) * doubles);
        if (e == cudaSuccess) e = cudaMemsetAsync(st->d_ev, 0, sizeof(double) * doubles, st->stream);
        if (e != cudaSuccess) { set_error("sv_expval_pauli: workspace allocation failed: %s", cudaGetErrorString(e)); return SV_ENOMEM; }
        st->ev_capacity = count;
    }
    double *partials = st->d_ev;
    double *results = partials + (size_t)max_grid * kEvMaxStrings;
    unsigned *counter = reinterpret_cast<unsigned *>(results + st->ev_capacity);

    // strings grouped by x mask (first-appearance order), at most kEvMaxStrings per pass
    std::vector<int> order((size_t)count);
    for (int i = 0; i < count; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return x_masks[p] < x_masks[q]; });
    const long long nb = n >= 5 ? (1ll << (n - 5)) : 1ll;
    std::vector<int> slot_of((size_t)count);
    int pos = 0;
    while (pos < count) {
        const uint64_t x = x_masks[order[(size_t)pos]];
        int m = 0;
        while (pos + m < count && m < kEvMaxStrings && x_masks[order[(size_t)(pos + m)]] == x) ++m;
        EvArgs a;
        std::memset(&a, 0, sizeof(a));
        a.xb = x >> 5;
        a.xl = (int)(x & 31u);
        a.pair_bit = a.xb ? highest_bit(a.xb) : -1;
        a.n_units = a.xb ? nb / 2 : nb;
        a.m = m;
        for (int p = 0; p < m; ++p) {
            const int s = order[(size_t)(pos + p)];
            const unsigned long long zb = z_masks[s] >> 5;
            unsigned long long zu = zb;
            if (a.pair_bit >= 0) {   // delete the pair bit: b = u with a zero inserted there
                const unsigned long long low = zb & ((1ull << a.pair_bit) - 1ull);
                zu = ((zb >> (a.pair_bit + 1)) << a.pair_bit) | low;
            }
            a.zu[p] = zu;
            unsigned tab = 0;
            for (unsigned i = 0; i < 32; ++i) tab |= (unsigned)(__builtin_popcountll(i & zu & 31ull) & 1) << i;
            a.ztab[p] = tab;
            a.zc[p] = (unsigned)(zu & 7ull);
            a.zl[p] = (unsigned)(z_masks[s] & 31u);
            a.pairpar[p] = (unsigned)(__builtin_popcountll(a.xb & zb) & 1);
            a.comp[p] = __builtin_popcountll(x & z_masks[s]) & 1;
            slot_of[(size_t)s] = pos + p;
        }
        const long long ranges = (a.n_units + kEvRange - 1) / kEvRange;
        const long long work = (ranges * 32 + kEvThreads - 1) / kEvThreads;   // CTAs with a range per warp
        const float *sv = st->d;
        double *res = results + pos;
        int rc;
        if (m == 1) rc = launch_ev<1>(sv, a, partials, counter, res, work, st->num_sms, max_grid, st->stream);
        else if (m == 2) rc = launch_ev<2>(sv, a, partials, counter, res, work, st->num_sms, max_grid, st->stream);
        else if (m <= 4) rc = launch_ev<4>(sv, a, partials, counter, res, work, st->num_sms, max_grid, st->stream);
        else rc = launch_ev<8>(sv, a, partials, counter, res, work, st->num_sms, max_grid, st->stream);
        if (rc != SV_OK) return rc;
        pos += m;
    }
    std::vector<double> host((size_t)count + kEvMaxStrings);
    SV_CUDA_TRY(cudaMemcpyAsync(host.data(), results, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, st->stream));
    SV_CUDA_TRY(cudaStreamSynchronize(st->stream));
    for (int i = 0; i < count; ++i) {
        const double s = host[(size_t)slot_of[(size_t)i]];
        // <psi|P|psi> = i^popc(x & z) * S; the accumulated component is Re S (even) or Im S (odd)
        switch (__builtin_popcountll(x_masks[i] & z_masks[i]) & 3) {
        case 0: out[i] = s; break;
        case 1: out[i] = -s; break;
        case 2: out[i] = -s; break;
        default: out[i] = s; break;
        }
    }
    return SV_OK;
}
