// Complex128 states: the same method (Eq. 3 per fused gate, Eq. 1 norm and sampling) in fp64.
//
// Layout: as for complex64, amplitude i lives in block i >> 5, now 64 doubles (512 bytes): the 32
// real parts then the 32 imaginary parts, converted from / to interleaved complex128 in place.
// Arithmetic is native fp64 with the fused matrices in fp64 (no fp32 rounding anywhere), so the
// result agrees with the complex128 oracle up to summation order.  GB300 executes fp64 FMAs at
// about 1/58 of the fp32 rate, so these kernels are bound by fp64 arithmetic, not HBM: a fused
// gate of k qubits costs 8 * 2^k flops per amplitude, and small k (2-3) minimises the total.
//
// Kernels: one group per thread; the group base inserts a zero at every target (and control)
// position and sets the control bits, the 2^k amplitudes are gathered, multiplied by U (k <= 4:
// a kernel parameter, read as constant-bank operands; k >= 5: device memory) and written back.
#include <cstring>
#include <vector>

#include "sv_internal.h"

namespace svg {
namespace {

constexpr int kC128Threads = 256;
constexpr int kC128ChunkLog2 = 14;

__host__ __device__ inline long long c128_off(unsigned long long i) { return (long long)(((i >> 5) << 6) | (i & 31ull)); }

int grid_c(long long items, int threads, int num_sms, int per_sm)
{
    long long g = (items + threads - 1) / threads;
    const long long cap = (long long)num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

long long n_blocks_c(int n) { return n >= 5 ? (1ll << (n - 5)) : 1ll; }

// in-place conversion of one 512-byte block per warp
__global__ void c128_block_layout_kernel(double *__restrict__ sv, long long n_blocks, int to_blocked)
{
    const int lane = threadIdx.x & 31;
    long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
    for (; w < n_blocks; w += stride) {
        double *b = sv + w * 64;
        double re, im;
        if (to_blocked) {
            const double2 v = reinterpret_cast<const double2 *>(b)[lane];
            re = v.x;
            im = v.y;
        } else {
            re = b[lane];
            im = b[32 + lane];
        }
        __syncwarp();
        if (to_blocked) {
            b[lane] = re;
            b[32 + lane] = im;
        } else {
            reinterpret_cast<double2 *>(b)[lane] = make_double2(re, im);
        }
        __syncwarp();
    }
}

__global__ void c128_copy_layout_kernel(double *__restrict__ dst, const double *__restrict__ src, long long n_amps, int to_blocked)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n_amps; i += stride) {
        const long long b = c128_off((unsigned long long)i);
        if (to_blocked) {
            const double2 v = reinterpret_cast<const double2 *>(src)[i];
            dst[b] = v.x;
            dst[b + 32] = v.y;
        } else {
            reinterpret_cast<double2 *>(dst)[i] = make_double2(src[b], src[b + 32]);
        }
    }
}

__global__ void c128_set_basis_kernel(double *sv, long long off) { sv[off] = 1.0; }

__device__ __forceinline__ double warp_sum_c(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum of |c_i|^2 in fp64; last CTA: strided per-thread sums, then a fixed-shape tree
__global__ void __launch_bounds__(kC128Threads) c128_norm_kernel(const double *__restrict__ sv, long long n_blocks,
                                                                  double *__restrict__ partials, unsigned *__restrict__ counter,
                                                                  double *__restrict__ result)
{
    double acc = 0.0;
    const long long items = n_blocks * 32;   // (block, lane)
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items; it += (long long)gridDim.x * blockDim.x) {
        const long long b = it >> 5;
        const int l = int(it & 31);
        const double re = sv[b * 64 + l], im = sv[b * 64 + 32 + l];
        acc = fma(re, re, acc);
        acc = fma(im, im, acc);
    }
    __shared__ double ws[kC128Threads / 32];
    __shared__ bool last;
    const double v = warp_sum_c(acc);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kC128Threads / 32; ++i) s += ws[i];
        partials[blockIdx.x] = s;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double red[kC128Threads];
    {
        const volatile double *p = partials;
        double s = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += kC128Threads) s += p[i];
        red[threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = kC128Threads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *result = red[0];
        *counter = 0u;
    }
}

// sampling: per-chunk sums of |c_i|^2, a single-CTA exclusive scan, one warp per sample
__global__ void c128_chunk_sum_kernel(const double *__restrict__ sv, long long n_chunks, int chunk_blocks_log2,
                                      double *__restrict__ chunk_sum)
{
    const int lane = threadIdx.x & 31;
    long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
    const long long cb = 1ll << chunk_blocks_log2;
    for (; w < n_chunks; w += stride) {
        double acc = 0.0;
        const double *base = sv + (w << chunk_blocks_log2) * 64;
        for (long long b = 0; b < cb; ++b) {
            const double re = base[b * 64 + lane], im = base[b * 64 + 32 + lane];
            acc = fma(re, re, acc);
            acc = fma(im, im, acc);
        }
        const double v = warp_sum_c(acc);
        if (lane == 0) chunk_sum[w] = v;
    }
}

__global__ void __launch_bounds__(1024) c128_chunk_scan_kernel(const double *__restrict__ sums, double *__restrict__ prefix, long long n)
{
    __shared__ double seg[1024];
    const long long per = (n + 1023) / 1024;
    const long long lo = threadIdx.x * per;
    const long long hi = lo + per < n ? lo + per : n;
    double s = 0.0;
    for (long long i = lo; i < hi; ++i) s += sums[i];
    seg[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = 0.0;
        for (int t = 0; t < 1024; ++t) {
            const double v = seg[t];
            seg[t] = run;
            run += v;
        }
        prefix[n] = run;
    }
    __syncthreads();
    double run = seg[threadIdx.x];
    for (long long i = lo; i < hi; ++i) {
        prefix[i] = run;
        run += sums[i];
    }
}

__global__ void c128_sample_search_kernel(const double *__restrict__ sv, int n, long long n_chunks, int chunk_log2,
                                          const double *__restrict__ prefix, const double *__restrict__ uniforms, int n_samples,
                                          unsigned long long *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (s >= n_samples) return;
    const double total = prefix[n_chunks];
    const double target = uniforms[s] * total;
    long long lo = 0, hi = n_chunks - 1;
    while (lo < hi) {   // largest chunk c with prefix[c] <= target
        const long long mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= target) lo = mid;
        else hi = mid - 1;
    }
    const unsigned long long N = 1ull << n;
    unsigned long long answer = N - 1;
    double run = prefix[lo];
    bool found = false;
    for (unsigned long long base = (unsigned long long)lo << chunk_log2; base < N && !found; base += 32) {
        const unsigned long long i = base + lane;
        double p = 0.0;
        if (i < N) {
            const long long o = c128_off(i);
            const double re = sv[o], im = sv[o + 32];
            p = fma(re, re, im * im);
        }
        double incl = p;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const bool hit = i < N && run + incl > target;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) {
            answer = base + (unsigned long long)__ffs(m) - 1;
            found = true;
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) out[s] = answer;
}

// ----------------------------------------------------------------------------------- gates
template <int K>
struct C128Mat {
    double u[(K <= 4) ? (2 << (2 * K)) : 2];   // row-major (re, im); K >= 5 reads device memory
};

template <int K>
struct C128Args {
    C128Mat<K> m;
    long long foff[1 << K];                 // offset (doubles) of local index j from the group base
    int pos[SV_MAX_K + SV_MAX_CONTROLS];    // ascending target and control qubits
    int npos;
    unsigned long long cmask;
    long long n_groups;
    const double *umem;                     // K >= 5: row-major (re, im) matrix in device memory
};

template <int K>
__global__ void __launch_bounds__(kC128Threads) apply_c128_kernel(double *__restrict__ sv, const __grid_constant__ C128Args<K> a)
{
    constexpr int D = 1 << K;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_groups) return;
    unsigned long long b = (unsigned long long)g;
    for (int i = 0; i < a.npos; ++i) {
        const unsigned long long low = b & ((1ull << a.pos[i]) - 1ull);
        b = ((b >> a.pos[i]) << (a.pos[i] + 1)) | low;
    }
    b |= a.cmask;
    double *base = sv + c128_off(b);
    double xr[D], xi[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        xr[j] = base[a.foff[j]];
        xi[j] = base[a.foff[j] + 32];
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
        double yr = 0.0, yi = 0.0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double ur, ui;
            if constexpr (K <= 4) {
                ur = a.m.u[2 * (r * D + j)];
                ui = a.m.u[2 * (r * D + j) + 1];
            } else {
                ur = a.umem[2 * (r * D + j)];
                ui = a.umem[2 * (r * D + j) + 1];
            }
            yr = fma(ur, xr[j], yr);
            yr = fma(-ui, xi[j], yr);
            yi = fma(ur, xi[j], yi);
            yi = fma(ui, xr[j], yi);
        }
        base[a.foff[r]] = yr;
        base[a.foff[r] + 32] = yi;
    }
}

template <int K>
int launch_c128_t(double *sv, int n, const FusedGate &g, const double *umem, cudaStream_t stream)
{
    C128Args<K> a;
    std::memset(&a, 0, sizeof(a));
    constexpr int D = 1 << K;
    if constexpr (K <= 4) {
        for (int e = 0; e < D * D; ++e) {
            a.m.u[2 * e] = g.mat[(size_t)e].real();
            a.m.u[2 * e + 1] = g.mat[(size_t)e].imag();
        }
    } else {
        if (!umem) { set_error("complex128 apply: k=%d gate has no device matrix", K); return SV_EINVAL; }
    }
    a.umem = umem;
    for (int j = 0; j < D; ++j) {
        unsigned long long o = 0;
        for (int t = 0; t < K; ++t)
            if ((j >> t) & 1) o |= 1ull << g.targets[t];
        a.foff[j] = c128_off(o);
    }
    const unsigned long long all = g.mask | g.cmask;
    int np = 0;
    for (int q = 0; q < n; ++q)
        if ((all >> q) & 1) a.pos[np++] = q;
    if (np != K + __builtin_popcountll(g.cmask) || (g.mask & g.cmask) || (n < 64 && (all >> n))) {
        set_error("complex128 apply: gate names a qubit twice or outside the state");
        return SV_EINVAL;
    }
    a.npos = np;
    a.cmask = g.cmask;
    a.n_groups = 1ll << (n - np);
    const long long grid = (a.n_groups + kC128Threads - 1) / kC128Threads;
    apply_c128_kernel<K><<<(unsigned)grid, kC128Threads, 0, stream>>>(sv, a);
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

}  // namespace

int c128_init(sv_state *st, uint64_t basis_index)
{
    SV_CUDA_TRY(cudaMemsetAsync(st->d, 0, sv_required_bytes_c128(st->n), st->stream));
    c128_set_basis_kernel<<<1, 1, 0, st->stream>>>(reinterpret_cast<double *>(st->d), c128_off(basis_index));
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

int c128_load(sv_state *st, const void *src, int src_on_host)
{
    double *d = reinterpret_cast<double *>(st->d);
    const size_t payload = size_t(16) << st->n;
    const long long nb = n_blocks_c(st->n);
    if (payload < 512) SV_CUDA_TRY(cudaMemsetAsync(d, 0, 512, st->stream));
    if (src_on_host) {
        SV_CUDA_TRY(cudaMemcpyAsync(d, src, payload, cudaMemcpyHostToDevice, st->stream));
        c128_block_layout_kernel<<<grid_c(nb * 32, 256, st->num_sms, 8), 256, 0, st->stream>>>(d, nb, 1);
    } else {
        const char *s = static_cast<const char *>(src);
        const char *dd = reinterpret_cast<const char *>(d);
        if (s < dd + sv_required_bytes_c128(st->n) && dd < s + payload) { set_error("sv_load: source overlaps the state"); return SV_EINVAL; }
        const long long na = 1ll << st->n;
        c128_copy_layout_kernel<<<grid_c(na, 256, st->num_sms, 8), 256, 0, st->stream>>>(d, static_cast<const double *>(src), na, 1);
    }
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

int c128_store(const sv_state *st, void *dst, int dst_on_host)
{
    double *d = reinterpret_cast<double *>(st->d);
    const size_t payload = size_t(16) << st->n;
    const long long nb = n_blocks_c(st->n);
    const int g = grid_c(nb * 32, 256, st->num_sms, 8);
    if (dst_on_host) {
        c128_block_layout_kernel<<<g, 256, 0, st->stream>>>(d, nb, 0);
        SV_CUDA_TRY(cudaGetLastError());
        SV_CUDA_TRY(cudaMemcpyAsync(dst, d, payload, cudaMemcpyDeviceToHost, st->stream));
        c128_block_layout_kernel<<<g, 256, 0, st->stream>>>(d, nb, 1);
        SV_CUDA_TRY(cudaGetLastError());
        SV_CUDA_TRY(cudaStreamSynchronize(st->stream));
    } else {
        const char *s = reinterpret_cast<const char *>(d);
        const char *dd = static_cast<const char *>(dst);
        if (s < dd + payload && dd < s + sv_required_bytes_c128(st->n)) { set_error("sv_store: destination overlaps the state"); return SV_EINVAL; }
        const long long na = 1ll << st->n;
        c128_copy_layout_kernel<<<grid_c(na, 256, st->num_sms, 8), 256, 0, st->stream>>>(static_cast<double *>(dst), d, na, 0);
        SV_CUDA_TRY(cudaGetLastError());
    }
    return SV_OK;
}

int c128_norm(const sv_state *st, double *out)
{
    const long long nb = n_blocks_c(st->n);
    const int g = grid_c(nb * 32, kC128Threads, st->num_sms, 4);
    if (g > st->max_partials) { set_error("sv_norm: internal grid too large"); return SV_EINVAL; }
    c128_norm_kernel<<<g, kC128Threads, 0, st->stream>>>(reinterpret_cast<const double *>(st->d), nb, st->d_partials, st->d_counter,
                                                         st->d_result);
    SV_CUDA_TRY(cudaGetLastError());
    SV_CUDA_TRY(cudaMemcpyAsync(out, st->d_result, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    SV_CUDA_TRY(cudaStreamSynchronize(st->stream));
    return SV_OK;
}

// chunk sums and their prefix (the total is the norm), then the samples if n_samples > 0; the
// uniforms are already in st->d_uniforms and the samples go to st->d_samples
int c128_sample(sv_state *st, int n_samples)
{
    const int n = st->n;
    const int chunk_log2 = n > kC128ChunkLog2 ? kC128ChunkLog2 : (n >= 5 ? n : 5);
    const long long nc = st->n_chunks;
    double *sums = st->d_chunk;
    double *prefix = st->d_chunk + nc;
    const double *sv = reinterpret_cast<const double *>(st->d);
    c128_chunk_sum_kernel<<<grid_c(nc * 32, 256, st->num_sms, 8), 256, 0, st->stream>>>(sv, nc, chunk_log2 - 5, sums);
    SV_CUDA_TRY(cudaGetLastError());
    c128_chunk_scan_kernel<<<1, 1024, 0, st->stream>>>(sums, prefix, nc);
    SV_CUDA_TRY(cudaGetLastError());
    if (n_samples > 0) {
        const int wpb = 8;
        c128_sample_search_kernel<<<(n_samples + wpb - 1) / wpb, 32 * wpb, 0, st->stream>>>(sv, n, nc, chunk_log2, prefix, st->d_uniforms,
                                                                                          n_samples, st->d_samples);
        SV_CUDA_TRY(cudaGetLastError());
    }
    return SV_OK;
}

int c128_apply_gate(sv_state *st, const FusedGate &g, const double *umem)
{
    double *sv = reinterpret_cast<double *>(st->d);
    switch (g.k) {
    case 1: return launch_c128_t<1>(sv, st->n, g, umem, st->stream);
    case 2: return launch_c128_t<2>(sv, st->n, g, umem, st->stream);
    case 3: return launch_c128_t<3>(sv, st->n, g, umem, st->stream);
    case 4: return launch_c128_t<4>(sv, st->n, g, umem, st->stream);
    case 5: return launch_c128_t<5>(sv, st->n, g, umem, st->stream);
    case 6: return launch_c128_t<6>(sv, st->n, g, umem, st->stream);
    default: set_error("complex128 apply: bad k=%d", g.k); return SV_EINVAL;
    }
}

}  // namespace svg

using namespace svg;

extern "C" size_t sv_required_bytes_c128(int n_qubits)
{
    if (n_qubits < 1 || n_qubits > SV_MAX_QUBITS) return 0;
    const size_t b = size_t(16) << n_qubits;
    return b < 512 ? 512 : b;
}
