// State handle, blocked layout conversion, norm and sampling kernels.
//
// Layout (paper section IV-A adjusts the layout in place so vector loads see contiguous reals and
// imaginaries; here the block is sized for 128-byte GPU transactions): amplitude i lives in block
// i >> 5; a block is 64 floats, the 32 real parts followed by the 32 imaginary parts.  Converting
// between this layout and interleaved complex64 only permutes floats inside one 256-byte block,
// so it runs in place with one read and one write of the state.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sv_internal.h"

using namespace svg;

namespace {

constexpr int kRedThreads = 256;
constexpr int kChunkLog2 = 14;   // sampling chunk: 2^14 amplitudes

__host__ __device__ inline long long re_off(unsigned long long i) { return (long long)(((i >> 5) << 6) | (i & 31ull)); }

// ---------------------------------------------------------------------------------------------
// in-place layout conversion, one warp per 256-byte block
__global__ void block_layout_kernel(float *__restrict__ sv, long long n_blocks, int to_blocked)
{
    const int lane = threadIdx.x & 31;
    long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
    for (; w < n_blocks; w += stride) {
        float *b = sv + w * 64;
        float re, im;
        if (to_blocked) {
            float2 v = reinterpret_cast<const float2 *>(b)[lane];
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
            reinterpret_cast<float2 *>(b)[lane] = make_float2(re, im);
        }
        __syncwarp();
    }
}

// out-of-place conversion: blocked `src` -> interleaved `dst` (to_blocked = 0) or back
__global__ void copy_layout_kernel(float *__restrict__ dst, const float *__restrict__ src, long long n_amps, int to_blocked)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; i < n_amps; i += stride) {
        const long long b = re_off((unsigned long long)i);
        if (to_blocked) {
            float2 v = reinterpret_cast<const float2 *>(src)[i];
            dst[b] = v.x;
            dst[b + 32] = v.y;
        } else {
            reinterpret_cast<float2 *>(dst)[i] = make_float2(src[b], src[b + 32]);
        }
    }
}

__global__ void set_basis_kernel(float *sv, long long off) { sv[off] = 1.0f; }

// ---------------------------------------------------------------------------------------------
// fp64-accurate sum of |c|^2.  Each thread keeps a float-float accumulator (hi, lo): squares are
// split exactly with fma (re*re = p + ep), sums use Knuth's two-sum, so the per-thread result
// carries ~48 significant bits; threads then combine in fp64.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ void ff_add(FF &a, float x)
{
    float s = a.hi + x;
    float bp = s - a.hi;
    float e = (a.hi - (s - bp)) + (x - bp);
    a.hi = s;
    a.lo += e;
}

__device__ __forceinline__ void ff_add_sq(FF &a, float v)
{
    float p = v * v;
    float ep = fmaf(v, v, -p);
    ff_add(a, p);
    a.lo += ep;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block b covers floats [b*64, b*64+64).  Work item = (block, quarter): 8 re + 8 im floats.
__global__ void __launch_bounds__(kRedThreads) norm_kernel(const float *__restrict__ sv, long long n_blocks,
                                                            double *__restrict__ partials, unsigned *__restrict__ counter,
                                                            double *__restrict__ result)
{
    FF acc{0.f, 0.f};
    const long long items = n_blocks * 8;   // 8 float4 pairs per block
    long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (; it < items; it += stride) {
        const long long b = it >> 3;
        const int q = int(it & 7);
        const float4 r = __ldcs(reinterpret_cast<const float4 *>(sv + b * 64) + q);
        const float4 m = __ldcs(reinterpret_cast<const float4 *>(sv + b * 64 + 32) + q);
        ff_add_sq(acc, r.x); ff_add_sq(acc, r.y); ff_add_sq(acc, r.z); ff_add_sq(acc, r.w);
        ff_add_sq(acc, m.x); ff_add_sq(acc, m.y); ff_add_sq(acc, m.z); ff_add_sq(acc, m.w);
    }
    double v = warp_sum_d((double)acc.hi + (double)acc.lo);
    __shared__ double ws[kRedThreads / 32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kRedThreads / 32; ++i) s += ws[i];
        partials[blockIdx.x] = s;
        __threadfence();
        unsigned done = atomicAdd(counter, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // last CTA: strided per-thread sums of the partials, then a fixed-shape tree (deterministic)
    __threadfence();
    __shared__ double red[kRedThreads];
    {
        const volatile double *p = partials;
        double s = 0.0;
        for (unsigned i = threadIdx.x; i < gridDim.x; i += kRedThreads) s += p[i];
        red[threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *result = red[0];
        *counter = 0u;   // ready for the next call
    }
}

// ---------------------------------------------------------------------------------------------
// sampling: chunk sums (fp64 via float-float per lane), exclusive prefix, then one warp per sample
__global__ void chunk_sum_kernel(const float *__restrict__ sv, long long n_chunks, int chunk_blocks_log2,
                                 double *__restrict__ chunk_sum)
{
    const int lane = threadIdx.x & 31;
    long long w = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
    const long long cb = 1ll << chunk_blocks_log2;
    for (; w < n_chunks; w += stride) {
        FF acc{0.f, 0.f};
        const float *base = sv + (w << chunk_blocks_log2) * 64;
        for (long long b = 0; b < cb; ++b) {
            ff_add_sq(acc, base[b * 64 + lane]);
            ff_add_sq(acc, base[b * 64 + 32 + lane]);
        }
        double v = warp_sum_d((double)acc.hi + (double)acc.lo);
        if (lane == 0) chunk_sum[w] = v;
    }
}

// single CTA exclusive scan of n chunk sums (in: sums, out: prefix), total at prefix[n]
__global__ void __launch_bounds__(1024) chunk_scan_kernel(const double *__restrict__ sums, double *__restrict__ prefix, long long n)
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
            double v = seg[t];
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

// One CTA of kSearchWarps warps per sample; p_i = re^2 + im^2 in fp64 (products of widened
// floats are exact).  After the chunk holding the sample is found (binary search on the chunk
// prefix sums), each warp sums p over its own part of the chunk with independent loads; thread 0
// picks the part where the running total passes the target; one warp then walks that part 32
// amplitudes at a time (warp scan) to the first index whose running total exceeds it, going on
// into the next part if the walk's rounding leaves the target just past this part's end.
constexpr int kSearchWarps = 8;

__global__ void __launch_bounds__(32 * kSearchWarps) sample_search_kernel(const float *__restrict__ sv, int n, long long n_chunks,
                                                                          int chunk_log2, const double *__restrict__ prefix,
                                                                          const double *__restrict__ uniforms, int n_samples,
                                                                          unsigned long long *__restrict__ out)
{
    __shared__ double part[kSearchWarps];
    __shared__ int s_part;
    __shared__ double s_run;
    const int s = blockIdx.x;
    if (s >= n_samples) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const double total = prefix[n_chunks];
    const double target = uniforms[s] * total;
    // largest chunk c with prefix[c] <= target
    long long lo = 0, hi = n_chunks - 1;
    while (lo < hi) {
        long long mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= target) lo = mid; else hi = mid - 1;
    }
    const unsigned long long N = 1ull << n;
    const unsigned long long i0 = (unsigned long long)lo << chunk_log2;
    const unsigned long long part_amps = (1ull << chunk_log2) / kSearchWarps;
    double acc = 0.0;
    for (unsigned long long k = lane; k < part_amps; k += 32) {
        const unsigned long long i = i0 + (unsigned long long)warp * part_amps + k;
        if (i < N) {
            const long long o = re_off(i);
            const double re = (double)sv[o], im = (double)sv[o + 32];
            acc += re * re + im * im;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double run = prefix[lo];
        int p = 0;
        while (p < kSearchWarps - 1 && run + part[p] <= target) run += part[p++];
        s_part = p;
        s_run = run;
    }
    __syncthreads();
    if (warp != 0) return;
    double run = s_run;
    unsigned long long answer = N - 1;
    bool found = false;
    for (unsigned long long base = i0 + (unsigned long long)s_part * part_amps; base < N && !found; base += 32) {
        const unsigned long long i = base + lane;
        double p = 0.0;
        if (i < N) {
            const long long o = re_off(i);
            const double re = (double)sv[o], im = (double)sv[o + 32];
            p = re * re + im * im;
        }
        // inclusive warp scan
        double incl = p;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            double t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, (i < N) && (run + incl > target));
        if (hit) {
            answer = base + (unsigned long long)(__ffs(hit) - 1);
            found = true;
        }
        run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) out[s] = answer;
}

int grid_for(long long items, int threads, int num_sms, int per_sm)
{
    long long g = (items + threads - 1) / threads;
    long long cap = (long long)num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

long long n_blocks_of(int n) { return n >= 5 ? (1ll << (n - 5)) : 1ll; }

}  // namespace

// ================================================================================== C ABI
extern "C" size_t sv_required_bytes(int n_qubits)
{
    if (n_qubits < 1 || n_qubits > SV_MAX_QUBITS) return 0;
    size_t b = size_t(8) << n_qubits;
    return b < 256 ? 256 : b;
}

namespace {

int alloc_state(int n_qubits, void *dev_ptr, size_t bytes, void *cuda_stream, sv_state **out, int c128)
{
    clear_error();
    if (!out) { set_error("sv_alloc: out is NULL"); return SV_EINVAL; }
    *out = nullptr;
    if (n_qubits < 1 || n_qubits > SV_MAX_QUBITS) { set_error("sv_alloc: n_qubits=%d outside [1, %d]", n_qubits, SV_MAX_QUBITS); return SV_EINVAL; }
    if (!dev_ptr) { set_error("sv_alloc: dev_ptr is NULL"); return SV_EINVAL; }
    if ((reinterpret_cast<uintptr_t>(dev_ptr) & 255u) != 0) { set_error("sv_alloc: dev_ptr must be 256-byte aligned"); return SV_EINVAL; }
    const size_t need = c128 ? sv_required_bytes_c128(n_qubits) : sv_required_bytes(n_qubits);
    if (bytes < need) {
        set_error("sv_alloc: buffer of %zu bytes is smaller than the %zu an %d-qubit state needs", bytes, need, n_qubits);
        return SV_ENOMEM;
    }
    cudaPointerAttributes attr{};
    SV_CUDA_TRY(cudaPointerGetAttributes(&attr, dev_ptr));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
        set_error("sv_alloc: dev_ptr is not device memory");
        return SV_EINVAL;
    }
    sv_state *st = new (std::nothrow) sv_state();
    if (!st) { set_error("sv_alloc: out of host memory"); return SV_ENOMEM; }
    st->n = n_qubits;
    st->c128 = c128;
    st->d = static_cast<float *>(dev_ptr);
    st->bytes = bytes;
    st->stream = static_cast<cudaStream_t>(cuda_stream);
    st->device = attr.device;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != st->device) { delete st; set_error("sv_alloc: buffer lives on device %d but device %d is current", attr.device, cur); return SV_EINVAL; }
    st->num_sms = device_sm_count(st->device);
    st->max_partials = st->num_sms * 8;
    const long long nb = n_blocks_of(n_qubits);
    st->n_chunks = n_qubits > kChunkLog2 ? (1ll << (n_qubits - kChunkLog2)) : 1ll;
    (void)nb;
    cudaError_t e = cudaMalloc(&st->d_partials, sizeof(double) * (size_t(st->max_partials) + 1) + sizeof(unsigned) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&st->d_chunk, sizeof(double) * (2 * size_t(st->n_chunks) + 1));
    if (e != cudaSuccess) {
        cudaFree(st->d_partials);
        delete st;
        set_error("sv_alloc: workspace allocation failed: %s", cudaGetErrorString(e));
        return SV_ENOMEM;
    }
    st->d_result = st->d_partials + st->max_partials;
    st->d_counter = reinterpret_cast<unsigned *>(st->d_result + 1);
    e = cudaMemsetAsync(st->d_counter, 0, sizeof(unsigned) * 4, st->stream);
    if (e != cudaSuccess) { sv_free(st); set_error("sv_alloc: %s", cudaGetErrorString(e)); return SV_ECUDA; }
    *out = st;
    return SV_OK;
}

}  // namespace

extern "C" int sv_alloc(int n_qubits, void *dev_ptr, size_t bytes, void *cuda_stream, sv_state **out)
{
    return alloc_state(n_qubits, dev_ptr, bytes, cuda_stream, out, 0);
}

extern "C" int sv_alloc_c128(int n_qubits, void *dev_ptr, size_t bytes, void *cuda_stream, sv_state **out)
{
    return alloc_state(n_qubits, dev_ptr, bytes, cuda_stream, out, 1);
}

extern "C" void sv_free(sv_state *st)
{
    if (!st) return;
    cudaStreamSynchronize(st->stream);
    cudaFree(st->d_partials);
    cudaFree(st->d_chunk);
    cudaFree(st->d_uniforms);
    cudaFree(st->d_samples);
    cudaFree(st->d_ev);
    cudaFree(st->d_compact);
    delete st;
}

extern "C" int sv_init(sv_state *st, uint64_t basis_index)
{
    clear_error();
    if (!st) { set_error("sv_init: state is NULL"); return SV_EINVAL; }
    if (basis_index >> st->n) { set_error("sv_init: basis index out of range for %d qubits", st->n); return SV_EINVAL; }
    if (st->c128) return c128_init(st, basis_index);
    const size_t used = sv_required_bytes(st->n);
    SV_CUDA_TRY(cudaMemsetAsync(st->d, 0, used, st->stream));
    set_basis_kernel<<<1, 1, 0, st->stream>>>(st->d, re_off(basis_index));
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

extern "C" int sv_load(sv_state *st, const void *src, int src_on_host)
{
    clear_error();
    if (!st || !src) { set_error("sv_load: NULL argument"); return SV_EINVAL; }
    if (st->c128) return c128_load(st, src, src_on_host);
    const size_t payload = size_t(8) << st->n;
    const long long nb = n_blocks_of(st->n);
    if (src_on_host) {
        if (payload < 256) SV_CUDA_TRY(cudaMemsetAsync(st->d, 0, 256, st->stream));
        SV_CUDA_TRY(cudaMemcpyAsync(st->d, src, payload, cudaMemcpyHostToDevice, st->stream));
        block_layout_kernel<<<grid_for(nb * 32, 256, st->num_sms, 8), 256, 0, st->stream>>>(st->d, nb, 1);
    } else {
        const char *s = static_cast<const char *>(src);
        const char *d = reinterpret_cast<const char *>(st->d);
        if (s < d + sv_required_bytes(st->n) && d < s + payload) { set_error("sv_load: source overlaps the state"); return SV_EINVAL; }
        if (payload < 256) SV_CUDA_TRY(cudaMemsetAsync(st->d, 0, 256, st->stream));
        const long long na = 1ll << st->n;
        copy_layout_kernel<<<grid_for(na, 256, st->num_sms, 8), 256, 0, st->stream>>>(st->d, static_cast<const float *>(src), na, 1);
    }
    SV_CUDA_TRY(cudaGetLastError());
    return SV_OK;
}

extern "C" int sv_store(const sv_state *st, void *dst, int dst_on_host)
{
    clear_error();
    if (!st || !dst) { set_error("sv_store: NULL argument"); return SV_EINVAL; }
    if (st->c128) return c128_store(st, dst, dst_on_host);
    const size_t payload = size_t(8) << st->n;
    const long long nb = n_blocks_of(st->n);
    const int g = grid_for(nb * 32, 256, st->num_sms, 8);
    if (dst_on_host) {
        block_layout_kernel<<<g, 256, 0, st->stream>>>(st->d, nb, 0);
        SV_CUDA_TRY(cudaGetLastError());
        SV_CUDA_TRY(cudaMemcpyAsync(dst, st->d, payload, cudaMemcpyDeviceToHost, st->stream));
        block_layout_kernel<<<g, 256, 0, st->stream>>>(st->d, nb, 1);
        SV_CUDA_TRY(cudaGetLastError());
        SV_CUDA_TRY(cudaStreamSynchronize(st->stream));
    } else {
        const char *s = reinterpret_cast<const char *>(st->d);
        const char *d = static_cast<const char *>(dst);
        if (s < d + payload && d < s + sv_required_bytes(st->n)) { set_error("sv_store: destination overlaps the state"); return SV_EINVAL; }
        const long long na = 1ll << st->n;
        copy_layout_kernel<<<grid_for(na, 256, st->num_sms, 8), 256, 0, st->stream>>>(static_cast<float *>(dst), st->d, na, 0);
        SV_CUDA_TRY(cudaGetLastError());
    }
    return SV_OK;
}

extern "C" int sv_norm(const sv_state *st, double *out)
{
    clear_error();
    if (!st || !out) { set_error("sv_norm: NULL argument"); return SV_EINVAL; }
    if (st->c128) return c128_norm(st, out);
    const long long nb = n_blocks_of(st->n);
    const int g = grid_for(nb * 8, kRedThreads, st->num_sms, 4);
    if (g > st->max_partials) { set_error("sv_norm: internal grid too large"); return SV_EINVAL; }
    norm_kernel<<<g, kRedThreads, 0, st->stream>>>(st->d, nb, st->d_partials, st->d_counter, st->d_result);
    SV_CUDA_TRY(cudaGetLastError());
    SV_CUDA_TRY(cudaMemcpyAsync(out, st->d_result, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    SV_CUDA_TRY(cudaStreamSynchronize(st->stream));
    return SV_OK;
}

namespace {

// Chunk sums of |c_i|^2 (fp64), their exclusive prefix (whose last entry is the total, i.e. the
// norm), then one warp per sample; norm_out (optional) receives that total.
int sample_impl(sv_state *st, const double *uniforms, int n_samples, uint64_t *out, double *norm_out, const char *who)
{
    if (!st || n_samples < 0 || (n_samples > 0 && (!uniforms || !out))) { set_error("%s: bad argument", who); return SV_EINVAL; }
    if (n_samples == 0 && !norm_out) return SV_OK;
    for (int s = 0; s < n_samples; ++s)
        if (!(uniforms[s] >= 0.0 && uniforms[s] < 1.0)) { set_error("%s: uniform %d = %g is not in [0, 1)", who, s, uniforms[s]); return SV_EINVAL; }
    if (n_samples > st->sample_capacity) {
        cudaStreamSynchronize(st->stream);
        cudaFree(st->d_uniforms);
        cudaFree(st->d_samples);
        st->d_uniforms = nullptr;
        st->d_samples = nullptr;
        st->sample_capacity = 0;
        cudaError_t e = cudaMalloc(&st->d_uniforms, sizeof(double) * size_t(n_samples));
        if (e == cudaSuccess) e = cudaMalloc(&st->d_samples, sizeof(unsigned long long) * size_t(n_samples));
        if (e != cudaSuccess) { set_error("%s: workspace allocation failed: %s", who, cudaGetErrorString(e)); return SV_ENOMEM; }
        st->sample_capacity = n_samples;
    }
    const int n = st->n;
    const int chunk_log2 = n > kChunkLog2 ? kChunkLog2 : (n >= 5 ? n : 5);
    const int chunk_blocks_log2 = chunk_log2 - 5;
    const long long nc = st->n_chunks;
    double *sums = st->d_chunk;
    double *prefix = st->d_chunk + nc;
    if (n_samples > 0)
        SV_CUDA_TRY(cudaMemcpyAsync(st->d_uniforms, uniforms, sizeof(double) * size_t(n_samples), cudaMemcpyHostToDevice, st->stream));
    if (st->c128) {
        SV_TRY(c128_sample(st, n_samples));
    } else {
        chunk_sum_kernel<<<grid_for(nc * 32, 256, st->num_sms, 8), 256, 0, st->stream>>>(st->d, nc, chunk_blocks_log2, sums);
        SV_CUDA_TRY(cudaGetLastError());
        chunk_scan_kernel<<<1, 1024, 0, st->stream>>>(sums, prefix, nc);
        SV_CUDA_TRY(cudaGetLastError());
        if (n_samples > 0) {
            sample_search_kernel<<<n_samples, 32 * kSearchWarps, 0, st->stream>>>(st->d, n, nc, chunk_log2, prefix, st->d_uniforms,
                                                                                 n_samples, st->d_samples);
            SV_CUDA_TRY(cudaGetLastError());
        }
    }
    if (n_samples > 0)
        SV_CUDA_TRY(cudaMemcpyAsync(out, st->d_samples, sizeof(unsigned long long) * size_t(n_samples), cudaMemcpyDeviceToHost, st->stream));
    if (norm_out) SV_CUDA_TRY(cudaMemcpyAsync(norm_out, prefix + nc, sizeof(double), cudaMemcpyDeviceToHost, st->stream));
    SV_CUDA_TRY(cudaStreamSynchronize(st->stream));
    return SV_OK;
}

}  // namespace

extern "C" int sv_sample(const sv_state *st, const double *uniforms, int n_samples, uint64_t *out)
{
    clear_error();
    return sample_impl(const_cast<sv_state *>(st), uniforms, n_samples, out, nullptr, "sv_sample");
}

extern "C" int sv_sample_norm(const sv_state *st, const double *uniforms, int n_samples, uint64_t *out, double *norm_out)
{
    clear_error();
    if (!norm_out) { set_error("sv_sample_norm: norm_out is NULL"); return SV_EINVAL; }
    return sample_impl(const_cast<sv_state *>(st), uniforms, n_samples, out, norm_out, "sv_sample_norm");
}

// ================================================================== sampling without allocation
// sv_sample_noalloc: the same three sampling kernels as sv_sample, but every intermediate buffer
// lives in one file-scope device array instead of memory from cudaMalloc.  Each GPU that loads
// the library holds this array (about 1.1 MB) until the process exits; all calls on a GPU share
// it, so calls whose GPU work overlaps (different streams, or threads) race on it.
namespace {

constexpr int kNoAllocMaxQubits = 30;
constexpr long long kNoAllocMaxChunks = 1ll << (kNoAllocMaxQubits - kChunkLog2);
constexpr int kNoAllocMaxSamples = 4096;
constexpr size_t kNoAllocDoubles = size_t(kNoAllocMaxChunks) * 2 + 1 + size_t(kNoAllocMaxSamples) * 2;

static __device__ __align__(256) double g_sample_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

// Host code must not pass the array's name to a kernel (on the host it names a stand-in, not
// device memory); the device address is looked up once per device, with that device current.
int noalloc_scratch(int device, double **out)
{
    if (device < 0 || device >= kMaxDevices) { set_error("sv_sample_noalloc: device %d out of range", device); return SV_EINVAL; }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_sample_scratch);
        if (e != cudaSuccess || !p) {
            set_error("sv_sample_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return SV_ECUDA;
        }
        g_noalloc_ptr[device] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[device];
    return SV_OK;
}

}  // namespace

extern "C" int sv_sample_noalloc(const void *dev_state, int n_qubits, void *cuda_stream, const double *uniforms,
                                 int n_samples, uint64_t *out)
{
    clear_error();
    if (!dev_state || n_samples < 0 || (n_samples > 0 && (!uniforms || !out))) { set_error("sv_sample_noalloc: bad argument"); return SV_EINVAL; }
    if (n_qubits < 1 || n_qubits > kNoAllocMaxQubits) {
        set_error("sv_sample_noalloc: n_qubits=%d outside [1, %d], the most its fixed scratch holds", n_qubits, kNoAllocMaxQubits);
        return SV_EINVAL;
    }
    if (n_samples > kNoAllocMaxSamples) {
        set_error("sv_sample_noalloc: n_samples=%d exceeds the %d its fixed scratch holds", n_samples, kNoAllocMaxSamples);
        return SV_EINVAL;
    }
    if (n_samples == 0) return SV_OK;
    for (int s = 0; s < n_samples; ++s)
        if (!(uniforms[s] >= 0.0 && uniforms[s] < 1.0)) { set_error("sv_sample_noalloc: uniform %d = %g is not in [0, 1)", s, uniforms[s]); return SV_EINVAL; }
    int device = 0;
    SV_CUDA_TRY(cudaGetDevice(&device));
    double *scratch = nullptr;
    SV_TRY(noalloc_scratch(device, &scratch));
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const int num_sms = device_sm_count(device);
    const int n = n_qubits;
    const int chunk_log2 = n > kChunkLog2 ? kChunkLog2 : (n >= 5 ? n : 5);
    const long long nc = n > kChunkLog2 ? (1ll << (n - kChunkLog2)) : 1ll;
    double *sums = scratch;
    double *prefix = scratch + kNoAllocMaxChunks;
    double *d_u = scratch + 2 * kNoAllocMaxChunks + 1;
    unsigned long long *d_out = reinterpret_cast<unsigned long long *>(d_u + kNoAllocMaxSamples);
    const float *sv = static_cast<const float *>(dev_state);
    SV_CUDA_TRY(cudaMemcpyAsync(d_u, uniforms, sizeof(double) * size_t(n_samples), cudaMemcpyHostToDevice, stream));
    chunk_sum_kernel<<<grid_for(nc * 32, 256, num_sms, 8), 256, 0, stream>>>(sv, nc, chunk_log2 - 5, sums);
    SV_CUDA_TRY(cudaGetLastError());
    chunk_scan_kernel<<<1, 1024, 0, stream>>>(sums, prefix, nc);
    SV_CUDA_TRY(cudaGetLastError());
    sample_search_kernel<<<n_samples, 32 * kSearchWarps, 0, stream>>>(sv, n, nc, chunk_log2, prefix, d_u, n_samples, d_out);
    SV_CUDA_TRY(cudaGetLastError());
    SV_CUDA_TRY(cudaMemcpyAsync(out, d_out, sizeof(unsigned long long) * size_t(n_samples), cudaMemcpyDeviceToHost, stream));
    SV_CUDA_TRY(cudaStreamSynchronize(stream));
    return SV_OK;
}
