/*
 * sv_oracle.c -- plain, slow, complex128 reference for the fused-gate state-vector path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this file;
 * only the test-suite, the smoke check and the CPU-baseline leg of the benchmark do.
 *
 * What it computes (paper section II-A, Eq. 1-3):
 *   - the state |psi> is 2^n complex amplitudes c_i, index bit q <-> qubit q (qubit 0 = LSB);
 *   - a k-qubit gate U (2^k x 2^k) on targets t_0..t_{k-1} is applied, for every one of the
 *     2^(n-k) groups, as a mat-vec over the 2^k amplitudes whose indices differ only in the
 *     target bits (Eq. 3).  Local matrix index bit j <-> qubit t_j.
 *   - with control qubits, the group is updated only when every control bit is 1 (Eq. 3
 *     and the sentence after it); otherwise it is left alone.
 *   - norm: sum_i |c_i|^2 (the normalisation condition under Eq. 1), in fp64.
 *   - sample: for uniforms u in [0,1), the smallest index i whose running sum of |c_j|^2
 *     (j <= i) exceeds u * total.  The uniforms are inputs; nothing random happens here.
 *
 * Gates are applied one at a time, unfused, in circuit order.  No blocking, no reordering:
 * the loop below is the definition written out.  An optional OpenMP "parallel for" over the
 * groups only splits the independent iterations of that same loop across host cores (used to
 * time the CPU baseline); results do not depend on it.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Insert a zero bit at each position of `pos` (sorted ascending) into g. */
static uint64_t insert_zero_bits(uint64_t g, const int *pos_sorted, int m)
{
    for (int b = 0; b < m; ++b) {
        int p = pos_sorted[b];
        uint64_t low = g & ((1ull << p) - 1ull);
        g = ((g >> p) << (p + 1)) | low;
    }
    return g;
}

static void sort_ints(int *a, int m)
{
    for (int i = 1; i < m; ++i) {
        int v = a[i], j = i - 1;
        while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
        a[j + 1] = v;
    }
}

/* Returns 0 on success, -1 on bad arguments. */
int oracle_apply_gate(cplx *psi, int n, int k, const int *targets, int n_controls,
                      const int *controls, const cplx *U, int n_threads)
{
    if (n < 1 || n > 40 || k < 1 || k > 10 || k > n || n_controls < 0 || n_controls + k > n)
        return -1;
    int sorted_t[16];
    uint64_t used = 0, cmask = 0;
    for (int j = 0; j < k; ++j) {
        if (targets[j] < 0 || targets[j] >= n || (used >> targets[j] & 1ull)) return -1;
        used |= 1ull << targets[j];
        sorted_t[j] = targets[j];
    }
    for (int c = 0; c < n_controls; ++c) {
        if (controls[c] < 0 || controls[c] >= n || (used >> controls[c] & 1ull)) return -1;
        used |= 1ull << controls[c];
        cmask |= 1ull << controls[c];
    }
    sort_ints(sorted_t, k);

    const int64_t dim = (int64_t)1 << k;
    const int64_t n_groups = (int64_t)1 << (n - k);
    /* offset of local index j: bit b of j goes to qubit targets[b] */
    uint64_t *off = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)dim);
    if (!off) return -1;
    for (int64_t j = 0; j < dim; ++j) {
        uint64_t o = 0;
        for (int b = 0; b < k; ++b)
            if ((j >> b) & 1) o |= 1ull << targets[b];
        off[j] = o;
    }

#ifdef _OPENMP
    if (n_threads < 1) n_threads = 1;
#pragma omp parallel num_threads(n_threads)
#endif
    {
        cplx x[1 << 10];
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t g = 0; g < n_groups; ++g) {
            uint64_t base = insert_zero_bits((uint64_t)g, sorted_t, k);
            if ((base & cmask) != cmask) continue;          /* a control bit is 0: untouched */
            for (int64_t j = 0; j < dim; ++j) x[j] = psi[base | off[j]];
            for (int64_t r = 0; r < dim; ++r) {
                cplx acc = 0.0;
                for (int64_t j = 0; j < dim; ++j) acc += U[r * dim + j] * x[j];
                psi[base | off[r]] = acc;
            }
        }
    }
    (void)n_threads;
    free(off);
    return 0;
}

double oracle_norm(const cplx *psi, int n)
{
    const int64_t N = (int64_t)1 << n;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double re = creal(psi[i]), im = cimag(psi[i]);
        s += re * re + im * im;
    }
    return s;
}

/* Same sum over a complex64 state read as fp64 (each float widened exactly). */
double oracle_norm_c64(const float *psi_interleaved, int n)
{
    const int64_t N = (int64_t)1 << n;
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double re = (double)psi_interleaved[2 * i], im = (double)psi_interleaved[2 * i + 1];
        s += re * re + im * im;
    }
    return s;
}

/* probabilities p_i = |c_i|^2 (fp64) are taken as given; out[s] = smallest i with
 * p_0 + ... + p_i > u_s * (p_0 + ... + p_{N-1}).  Sample order of `u` is kept. */
typedef struct { double u; int64_t s; } upair;
static int cmp_upair(const void *a, const void *b)
{
    double x = ((const upair *)a)->u, y = ((const upair *)b)->u;
    return (x > y) - (x < y);
}

int oracle_sample_probs(const double *p, int64_t N, const double *u, int64_t S, uint64_t *out)
{
    double total = 0.0;
    for (int64_t i = 0; i < N; ++i) total += p[i];
    upair *q = (upair *)malloc(sizeof(upair) * (size_t)(S > 0 ? S : 1));
    if (!q) return -1;
    for (int64_t s = 0; s < S; ++s) { q[s].u = u[s]; q[s].s = s; }
    qsort(q, (size_t)S, sizeof(upair), cmp_upair);
    double run = 0.0;
    int64_t i = 0;
    for (int64_t r = 0; r < S; ++r) {
        double target = q[r].u * total;
        while (i < N - 1 && !(run + p[i] > target)) { run += p[i]; ++i; }
        out[q[r].s] = (uint64_t)i;
    }
    free(q);
    return 0;
}
