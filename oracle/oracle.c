/*
 * FP64 CPU oracle for mixed-radix (qubit-qudit) state-vector simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg load it.  It shares no code with the CUDA
 * path.
 *
 * What it computes is the plain definition of applying one gate to a state
 * vector, written index by index, not the block decomposition that the
 * paper (and the CUDA path) uses to reach the same result faster:
 *
 *   * Basis index j of a system with wire dimensions d_0..d_{n-1} reads as
 *     mixed-radix digits with q_0 least significant (section "Proposed
 *     Methodology").  The digit of wire w is
 *         x_w(j) = floor(j / b_w) mod d_w,   b_w = d_0 * ... * d_{w-1},
 *     the control-condition formula of section "Controlled and
 *     Multi-Controlled Gates".
 *   * A gate is a P x P complex matrix U on target wires w_0..w_{k-1}
 *     (first-listed least significant in the local index, P = prod d_{w_m})
 *     plus control wires c_m with values v_m.  As an operator on the whole
 *     space it is  Pi (x) U + (1 - Pi) (x) 1, with Pi the projector on basis
 *     states whose control digits all match.  Element by element:
 *         out[j] = psi[j]                                   if a control fails
 *         out[j] = sum_c U[r(j)][c] * psi[j + sum_m (c_m - r_m) b_{w_m}]
 *                                                            otherwise,
 *     where r(j) is the local row index of j and c_m the digits of column c.
 *
 * All arithmetic is IEEE binary64, built with -ffp-contract=off so that no
 * multiply-add is fused; sums run in a fixed order.  Readouts use
 * Neumaier's compensated summation (Neumaier, ZAMM 54, 1974).
 *
 * Amplitudes are interleaved (re, im) doubles.  Functions return 0 on
 * success and a negative code on invalid arguments.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAX_WIRES 64
#define OR_MAX_P 4096

static int64_t or_strides(int32_t n, const int32_t* dims, int64_t* b)
{
    int64_t D = 1;
    for (int32_t i = 0; i < n; ++i) {
        if (dims[i] < 2) return -1;
        b[i] = D;
        if (D > (int64_t)1 << 40) return -1;
        D *= dims[i];
    }
    b[n] = D;
    return D;
}

int64_t or_dim(int32_t n, const int32_t* dims)
{
    int64_t b[OR_MAX_WIRES + 1];
    if (n < 1 || n > OR_MAX_WIRES) return -1;
    return or_strides(n, dims, b);
}

/* Digit of wire w in basis index j: floor(j / b_w) mod d_w. */
static inline int64_t digit(int64_t j, int64_t bw, int64_t dw)
{
    return (j / bw) % dw;
}

/*
 * Apply one gate out of place: out = G psi.  psi and out hold 2*D doubles
 * and must not overlap.  nthreads <= 0 means one thread.
 */
int or_apply(int32_t n, const int32_t* dims, const double* psi, double* out,
             int32_t k, const int32_t* wires, const double* U,
             int32_t m, const int32_t* cw, const int32_t* cv, int32_t nthreads)
{
    int64_t b[OR_MAX_WIRES + 1];
    if (n < 1 || n > OR_MAX_WIRES || k < 1 || k > n || m < 0 || m > n) return -1;
    const int64_t D = or_strides(n, dims, b);
    if (D < 0) return -1;
    int64_t P = 1;
    for (int32_t a = 0; a < k; ++a) {
        if (wires[a] < 0 || wires[a] >= n) return -2;
        for (int32_t a2 = 0; a2 < a; ++a2)
            if (wires[a2] == wires[a]) return -2;
        P *= dims[wires[a]];
    }
    if (P > OR_MAX_P) return -3;
    for (int32_t a = 0; a < m; ++a) {
        if (cw[a] < 0 || cw[a] >= n) return -4;
        if (cv[a] < 0 || cv[a] >= dims[cw[a]]) return -4;
        for (int32_t a2 = 0; a2 < k; ++a2)
            if (wires[a2] == cw[a]) return -4;
        for (int32_t a2 = 0; a2 < a; ++a2)
            if (cw[a2] == cw[a]) return -4;
    }
    if (nthreads < 1) nthreads = 1;

    #pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t j = 0; j < D; ++j) {
        int ok = 1;
        for (int32_t a = 0; a < m; ++a)
            if (digit(j, b[cw[a]], dims[cw[a]]) != cv[a]) { ok = 0; break; }
        if (!ok) {
            out[2 * j] = psi[2 * j];
            out[2 * j + 1] = psi[2 * j + 1];
            continue;
        }
        /* local row index r(j) and the base index with every gate digit 0 */
        int64_t r = 0, place = 1, base = j;
        for (int32_t a = 0; a < k; ++a) {
            const int64_t x = digit(j, b[wires[a]], dims[wires[a]]);
            r += x * place;
            place *= dims[wires[a]];
            base -= x * b[wires[a]];
        }
        double re = 0.0, im = 0.0;
        for (int64_t c = 0; c < P; ++c) {
            /* index of the column-c member: base + sum_m c_m * b_{w_m} */
            int64_t jc = base, rem = c;
            for (int32_t a = 0; a < k; ++a) {
                const int64_t dw = dims[wires[a]];
                jc += (rem % dw) * b[wires[a]];
                rem /= dw;
            }
            const double ur = U[2 * (r * P + c)], ui = U[2 * (r * P + c) + 1];
            const double xr = psi[2 * jc], xi = psi[2 * jc + 1];
            re += ur * xr - ui * xi;
            im += ur * xi + ui * xr;
        }
        out[2 * j] = re;
        out[2 * j + 1] = im;
    }
    return 0;
}

/* Neumaier's compensated sum step. */
static inline void neumaier_add(double* s, double* c, double x)
{
    const double t = *s + x;
    if ((*s >= 0 ? *s : -*s) >= (x >= 0 ? x : -x))
        *c += (*s - t) + x;
    else
        *c += (x - t) + *s;
    *s = t;
}

/* Squared norm sum_j |psi_j|^2 (compensated, sequential order). */
double or_norm(int64_t D, const double* psi)
{
    double s = 0.0, c = 0.0;
    for (int64_t j = 0; j < D; ++j) {
        const double p = psi[2 * j] * psi[2 * j] + psi[2 * j + 1] * psi[2 * j + 1];
        neumaier_add(&s, &c, p);
    }
    return s + c;
}

/* Born probabilities |psi_j|^2. */
void or_probabilities(int64_t D, const double* psi, double* out)
{
    for (int64_t j = 0; j < D; ++j)
        out[j] = psi[2 * j] * psi[2 * j] + psi[2 * j + 1] * psi[2 * j + 1];
}

/* Marginal distribution of one wire: p(x) = sum_{j : x_w(j) = x} |psi_j|^2. */
int or_marginal(int32_t n, const int32_t* dims, const double* psi, int32_t w, double* out)
{
    int64_t b[OR_MAX_WIRES + 1];
    if (n < 1 || n > OR_MAX_WIRES || w < 0 || w >= n) return -1;
    const int64_t D = or_strides(n, dims, b);
    if (D < 0) return -1;
    const int32_t dw = dims[w];
    double* s = (double*)calloc((size_t)dw * 2, sizeof(double));
    if (!s) return -5;
    for (int64_t j = 0; j < D; ++j) {
        const int64_t x = digit(j, b[w], dw);
        const double p = psi[2 * j] * psi[2 * j] + psi[2 * j + 1] * psi[2 * j + 1];
        neumaier_add(&s[2 * x], &s[2 * x + 1], p);
    }
    for (int32_t x = 0; x < dw; ++x) out[x] = s[2 * x] + s[2 * x + 1];
    free(s);
    return 0;
}

/* Number of OpenMP threads available (1 without OpenMP). */
int32_t or_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
