/*
 * Oracle state-vector kernel in complex128 -- TEST INFRASTRUCTURE ONLY.
 *
 * Applies one k-qubit gate matrix to a 2^n complex128 state, the literal
 * definition of gate application in the paper's Sec. 2.1 (a unitary acting on
 * the amplitudes) and Sec. 3.2.2 (state viewed with qubit q as bit n-1-q,
 * "reshape (2^k, 2, 2^(n-k-1))", App. A).  For every assignment of the other
 * n-k bits it gathers the 2^k amplitudes that differ only in the gate's bits,
 * multiplies them by the matrix and scatters them back.  No fusion, no
 * tables, no special cases.
 *
 * Only tests/, __graft_entry__.smoke() and the bench's CPU-baseline legs load
 * this library.  It shares no code with the CUDA path.
 */
#include <complex.h>
#include <stdint.h>

#define ORC_MAX_K 6

/* Apply the 2^k x 2^k row-major matrix U to wires qubits[0..k-1] (qubits[0] is
 * the most significant bit of the matrix index).  Returns 0, or -1 on a bad
 * argument. */
int orc_apply(int n, double complex *psi, int k, const int *qubits, const double complex *U)
{
    if (n < 1 || n > 40 || k < 1 || k > ORC_MAX_K || k > n)
        return -1;
    int pos[ORC_MAX_K];
    for (int m = 0; m < k; ++m) {
        if (qubits[m] < 0 || qubits[m] >= n)
            return -1;
        pos[m] = n - 1 - qubits[m];
        for (int j = 0; j < m; ++j)
            if (pos[j] == pos[m])
                return -1;
    }
    int sorted[ORC_MAX_K];
    for (int m = 0; m < k; ++m)
        sorted[m] = pos[m];
    for (int a = 0; a < k; ++a)          /* insertion sort, ascending */
        for (int b = a + 1; b < k; ++b)
            if (sorted[b] < sorted[a]) {
                int t = sorted[a];
                sorted[a] = sorted[b];
                sorted[b] = t;
            }
    const int K = 1 << k;
    const int64_t nbase = ((int64_t)1) << (n - k);

#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < nbase; ++r) {
        int64_t base = r;
        for (int m = 0; m < k; ++m) {    /* open a zero bit at each gate position */
            int64_t p = sorted[m];
            int64_t lowmask = (((int64_t)1) << p) - 1;
            base = ((base & ~lowmask) << 1) | (base & lowmask);
        }
        int64_t idx[1 << ORC_MAX_K];
        double complex a[1 << ORC_MAX_K];
        for (int j = 0; j < K; ++j) {
            int64_t x = base;
            for (int m = 0; m < k; ++m)
                if ((j >> (k - 1 - m)) & 1)
                    x |= ((int64_t)1) << pos[m];
            idx[j] = x;
            a[j] = psi[x];
        }
        for (int i = 0; i < K; ++i) {
            double complex s = 0.0;
            for (int j = 0; j < K; ++j)
                s += U[i * K + j] * a[j];
            psi[idx[i]] = s;
        }
    }
    return 0;
}

/* <a|b> = sum conj(a_x) b_x, accumulated in complex128. */
void orc_vdot(int64_t dim, const double complex *a, const double complex *b, double *out_re, double *out_im)
{
    double re = 0.0, im = 0.0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (int64_t x = 0; x < dim; ++x) {
        double complex v = conj(a[x]) * b[x];
        re += creal(v);
        im += cimag(v);
    }
    *out_re = re;
    *out_im = im;
}

/* Thread count of the parallel loops above (timing only; results do not
 * depend on it beyond the order of the vdot reduction). */
void orc_set_threads(int t)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (t > 0)
        omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
