/*
 * FP64 index-loop oracle for generalized qudit gates (plain C).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/ and by the CPU-baseline legs of
 * bench.py through ctypes; nothing on the product path links or calls it, and
 * it shares no code with the CUDA library.
 *
 * What it computes (QuDiet, arXiv 2211.07918): psi <- U_full psi for one gate,
 * where U_full is the gate matrix over its acting qudits padded with
 * identities (Sec. 3.5-3.6).  The register is mixed-radix with qudit 0 the
 * least significant digit (Sec. 3.2), s_q = prod_{p<q} d_p.  A controlled gate
 * is identity except on basis states whose control digits equal the control
 * levels (Sec. 2.1.2, C_{X,d} and C^n_{X,d}).
 *
 * Method, in the plainest form: for every basis index i, extract the digits of
 * the acting qudits by division and remainder; if every target digit is 0 and
 * every control digit equals its level, i is the base of one group; gather the
 * D amplitudes of the group (local index j, first target most significant),
 * multiply by the D x D matrix in FP64, scatter them back.
 *
 * Layout: psi and g are interleaved (re, im) doubles; g is row-major D x D.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QO_MAXQ 64
#define QO_MAXD 4096

/* Returns 0 on success, -1 on bad arguments. */
int qo_apply(double *psi, int32_t n, const int32_t *dims, const double *g, int32_t k,
             const int32_t *targets, int32_t nc, const int32_t *controls,
             const int32_t *levels, int32_t nthreads)
{
    if (n < 1 || n > QO_MAXQ || k < 1 || nc < 0) return -1;
    int64_t s[QO_MAXQ];
    int64_t N = 1;
    for (int q = 0; q < n; ++q) {
        if (dims[q] < 2) return -1;
        s[q] = N;
        N *= dims[q];
    }
    int64_t D = 1;
    for (int m = 0; m < k; ++m) {
        if (targets[m] < 0 || targets[m] >= n) return -1;
        D *= dims[targets[m]];
    }
    for (int c = 0; c < nc; ++c)
        if (controls[c] < 0 || controls[c] >= n || levels[c] < 0 || levels[c] >= dims[controls[c]])
            return -1;
    if (D > QO_MAXD) return -1;

    /* offset of local index j: digits of j in the target radices, the first
     * target most significant */
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)D);
    if (!off) return -1;
    for (int64_t j = 0; j < D; ++j) {
        int64_t rem = j, o = 0;
        for (int m = k - 1; m >= 0; --m) {
            int t = targets[m];
            o += (rem % dims[t]) * s[t];
            rem /= dims[t];
        }
        off[j] = o;
    }

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double *v = (double *)malloc(sizeof(double) * 2 * (size_t)D);
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t i = 0; i < N; ++i) {
            int is_base = 1;
            for (int m = 0; m < k && is_base; ++m)
                if ((i / s[targets[m]]) % dims[targets[m]] != 0) is_base = 0;
            for (int c = 0; c < nc && is_base; ++c)
                if ((i / s[controls[c]]) % dims[controls[c]] != levels[c]) is_base = 0;
            if (!is_base) continue;
            for (int64_t j = 0; j < D; ++j) {
                v[2 * j] = psi[2 * (i + off[j])];
                v[2 * j + 1] = psi[2 * (i + off[j]) + 1];
            }
            for (int64_t r = 0; r < D; ++r) {
                double re = 0.0, im = 0.0;
                const double *row = g + 2 * r * D;
                for (int64_t c = 0; c < D; ++c) {
                    re += row[2 * c] * v[2 * c] - row[2 * c + 1] * v[2 * c + 1];
                    im += row[2 * c] * v[2 * c + 1] + row[2 * c + 1] * v[2 * c];
                }
                psi[2 * (i + off[r])] = re;
                psi[2 * (i + off[r]) + 1] = im;
            }
        }
        free(v);
    }
    free(off);
    return 0;
}

/* sum_i |psi_i|^2, left to right, FP64. */
double qo_norm2(const double *psi, int64_t N)
{
    double acc = 0.0;
    for (int64_t i = 0; i < N; ++i) acc += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    return acc;
}

int qo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
