/*
 * sl_oracle.c -- plain, slow, FP64 CPU oracle for the element-local
 * semi-Lagrangian Monte-Carlo step of Natarajan, Popov & Jacobs,
 * "A high-order semi-Lagrangian method for the consistent Monte-Carlo solution
 * of stochastic Lagrangian drift-diffusion models coupled with Eulerian
 * discontinuous spectral element method" (arXiv:2009.07340), Section 5.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library never
 * links, includes or calls it, and it never calls the CUDA library; the two
 * share no code, header, table or constant generator.
 *
 * Every function follows the paper's definition as literally as possible:
 * no blocking, no fusion, no algebraic shortcuts beyond what the cited
 * equation states.  Where the paper is silent the reading adopted is stated
 * at the point of use:
 *   - Gauss nodes use (i+1/2)pi/N (Eq. gaussquad has N+1, which is neither
 *     symmetric nor interleaved with the Lobatto nodes as Section 3 states).
 *   - The constrained least-squares remap is the stacked, unweighted system
 *     min |V q - phi*|^2 + |B q - g|^2 (Section 5.3 defers the details to the
 *     authors' earlier deterministic paper).
 *   - The Wiener increment is drawn from Philox4x32-10 with a Box-Muller
 *     transform built on the own ln / sincospi below (the paper names no RNG).
 *   - Nodal drift and diffusion (the field solver's values at the Gauss
 *     nodes, Section 5.2): interface values given, else the mean of the two
 *     neighbouring elements' traces (the inside trace at a Dirichlet
 *     boundary, a derived D clipped at 0).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -pthread sl_oracle.c -lm
 * (contraction off: fma() is used only where written explicitly).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Ten rounds; round r uses the key bumped r times */
/* by the Weyl constants.                                                     */
/* ------------------------------------------------------------------------ */
#define PHILOX_M4x32_0 0xD2511F53u
#define PHILOX_M4x32_1 0xCD9E8D57u
#define PHILOX_W32_0 0x9E3779B9u
#define PHILOX_W32_1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W32_0;
            k1 += PHILOX_W32_1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M4x32_0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M4x32_1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    out[0] = c[0];
    out[1] = c[1];
    out[2] = c[2];
    out[3] = c[3];
}

/* ------------------------------------------------------------------------ */
/* Natural logarithm for x in (0, 1], written out so that the CPU and GPU    */
/* sides can reproduce it bit for bit.  x = m 2^k with m in [sqrt(1/2),     */
/* sqrt(2)) (exact split), ln m = 2 atanh(t), t = (m-1)/(m+1), by its Taylor */
/* series in t^2 (Horner, explicit fma), and k ln 2 with a two-part ln 2     */
/* (Cody & Waite) so that k*ln2_hi is exact.                                 */
/* ------------------------------------------------------------------------ */
static const double ORC_LN2_HI = 0.693146705627441406250;       /* ln 2 to 21 bits      */
static const double ORC_LN2_LO = 4.7493250390316726e-07;        /* ln 2 - ORC_LN2_HI    */
static const double ORC_SQRT_HALF = 0.70710678118654752440084436; /* sqrt(1/2)         */

double orc_log(double x)
{
    int e;
    double m = frexp(x, &e); /* x = m 2^e, m in [1/2, 1), exact */
    if (m < ORC_SQRT_HALF) {
        m = m * 2.0; /* exact */
        e = e - 1;
    }
    double t = (m - 1.0) / (m + 1.0);
    double s = t * t;
    /* atanh(t)/t = sum_{k>=0} s^k / (2k+1); |t| <= 0.1716, 12 terms */
    double p = 1.0 / 23.0;
    p = fma(p, s, 1.0 / 21.0);
    p = fma(p, s, 1.0 / 19.0);
    p = fma(p, s, 1.0 / 17.0);
    p = fma(p, s, 1.0 / 15.0);
    p = fma(p, s, 1.0 / 13.0);
    p = fma(p, s, 1.0 / 11.0);
    p = fma(p, s, 1.0 / 9.0);
    p = fma(p, s, 1.0 / 7.0);
    p = fma(p, s, 1.0 / 5.0);
    p = fma(p, s, 1.0 / 3.0);
    p = fma(p, s, 1.0);
    double lnm = (t * p) * 2.0;
    double k = (double)e;
    double hi = k * ORC_LN2_HI; /* exact: |k| < 2^11 and ORC_LN2_HI has 21 bits */
    double lo = k * ORC_LN2_LO + lnm;
    return hi + lo;
}

/* sin(pi r), cos(pi r) for |r| <= 1/4 by their Taylor series, coefficients  */
/* (-1)^k pi^(2k+1)/(2k+1)! and (-1)^k pi^(2k)/(2k)! rounded to double.      */
static const double ORC_SINPI_C[10] = {
    3.141592653589793238462643,     -5.167712780049970029246053,
    2.550164039877345443856178,     -0.5992645293207920768877394,
    0.08214588661112822879880237,   -0.00737043094571435077725909,
    0.0004663028057676125644206289, -0.00002191535344783021582738465,
    0.0000007952054001475512784783207, -2.294842899726987311020387e-8};
static const double ORC_COSPI_C[10] = {
    1.0,                            -4.934802200544679309417245,
    4.058712126416768218185014,     -1.335262768854589495875305,
    0.2353306303588932045418794,    -0.02580689139001406001259829,
    0.001929574309403923047903346,  -0.0001046381049248457071180167,
    0.000004303069587032947007297824, -0.0000001387895246221377211446809};

/* sin(pi y), cos(pi y) for y in [0, 2]: y = j/2 + r, |r| <= 1/4 (exact),   */
/* then the quadrant identities.                                             */
void orc_sincospi(double y, double *sp, double *cp)
{
    double j = rint(y * 2.0); /* exact scaling; quadrant index 0..4 */
    double r = y - j * 0.5;   /* exact */
    double r2 = r * r;
    double ps = ORC_SINPI_C[9];
    for (int k = 8; k >= 0; --k) ps = fma(ps, r2, ORC_SINPI_C[k]);
    double s = ps * r;
    double pc = ORC_COSPI_C[9];
    for (int k = 8; k >= 0; --k) pc = fma(pc, r2, ORC_COSPI_C[k]);
    double c = pc;
    int q = ((int)j) & 3;
    if (q == 0) {
        *sp = s;
        *cp = c;
    } else if (q == 1) {
        *sp = c;
        *cp = -s;
    } else if (q == 2) {
        *sp = -s;
        *cp = -c;
    } else {
        *sp = -c;
        *cp = s;
    }
}

/* Two standard normals for (seed, step, sample, tag): Philox words          */
/* c0..c3 -> two 52-bit integers -> uniforms (2x+1) 2^-53 in (0,1) -> Box-  */
/* Muller z1 = r cos(2 pi u2), z2 = r sin(2 pi u2), r = sqrt(-2 ln u1).      */
void orc_normals(unsigned long long seed, uint32_t step, uint32_t sample, uint32_t tag,
                 double z[2])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {step, sample, tag, 0u};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    uint64_t x1 = (((uint64_t)w[0] << 32) | (uint64_t)w[1]) >> 12;
    uint64_t x2 = (((uint64_t)w[2] << 32) | (uint64_t)w[3]) >> 12;
    double u1 = (double)(2 * x1 + 1) * 0x1p-53;
    double u2 = (double)(2 * x2 + 1) * 0x1p-53;
    double r = sqrt(-2.0 * orc_log(u1));
    double s, c;
    orc_sincospi(2.0 * u2, &s, &c);
    z[0] = r * c;
    z[1] = r * s;
}

/* Wiener increments dW = sqrt(dt) z for steps [step0, step0+nsteps), all M  */
/* samples, d dimensions: out[step][sample][dim].  One increment per sample  */
/* per step per dimension, shared by every node of every element (Section    */
/* 5.2, Eq. def_dx and the paragraph after it).                              */
void orc_wiener(unsigned long long seed, int dim, int M, long step0, int nsteps, double dt,
                double *out)
{
    double sdt = sqrt(dt);
    for (int n = 0; n < nsteps; ++n)
        for (int s = 0; s < M; ++s) {
            double z[2];
            orc_normals(seed, (uint32_t)(step0 + n), (uint32_t)s, 0u, z);
            for (int d = 0; d < dim; ++d) out[((long)n * M + s) * dim + d] = sdt * z[d];
        }
}

/* ------------------------------------------------------------------------ */
/* Reference element (Section 3).                                            */
/* ------------------------------------------------------------------------ */

/* Chebyshev-Gauss solution nodes on [0,1], Eq. (gaussquad) with (i+1/2)/N. */
void orc_nodes(int N, double *xi)
{
    for (int i = 0; i < N; ++i) xi[i] = 0.5 * (1.0 - cos((i + 0.5) * M_PI / N));
}

/* Lagrange polynomial h_j through the points base[m] + off[m] (m < N),      */
/* evaluated at xb + xo, by the product formula of Eq. (3.5) / Eq. (h_star).  */
/* Points are passed as a base position plus an offset and every difference  */
/* is formed as (base difference) + (offset difference): a particle position */
/* x* = x + dx (Eq. def_dx) is never rounded as a whole, so a displacement    */
/* much smaller than x keeps its full relative precision.                    */
double orc_lagrange_split(int N, const double *base, const double *off, int j, double xb, double xo)
{
    double v = 1.0;
    for (int m = 0; m < N; ++m)
        if (m != j)
            v *= ((xb - base[m]) + (xo - off[m])) / ((base[j] - base[m]) + (off[j] - off[m]));
    return v;
}

static const double ORC_ZEROS[256] = {0.0}; /* offsets of unmoved points (n <= 256) */

/* Lagrange polynomial h_j through pts[0..N-1] at x (Eq. 3.5). */
double orc_lagrange(int N, const double *pts, int j, double x)
{
    return orc_lagrange_split(N, pts, ORC_ZEROS, j, x, 0.0);
}

/* Derivative of h_j at x: sum over the dropped factor (product rule). */
double orc_lagrange_deriv(int N, const double *pts, int j, double x)
{
    double sum = 0.0;
    for (int k = 0; k < N; ++k) {
        if (k == j) continue;
        double v = 1.0 / (pts[j] - pts[k]);
        for (int m = 0; m < N; ++m)
            if (m != j && m != k) v *= (x - pts[m]) / (pts[j] - pts[m]);
        sum += v;
    }
    return sum;
}

/* Fejer first-rule weights on the Chebyshev-Gauss nodes, scaled to [0,1]   */
/* (Fejer 1933; Waldvogel 2006).  Exact for polynomials of degree <= N-1.   */
void orc_quad_weights(int N, double *w)
{
    for (int k = 0; k < N; ++k) {
        double th = (k + 0.5) * M_PI / N;
        double s = 0.0;
        for (int j = 1; j <= N / 2; ++j) s += cos(2.0 * j * th) / (4.0 * j * j - 1.0);
        w[k] = 0.5 * (2.0 / N) * (1.0 - 2.0 * s);
    }
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra (textbook; Golub & Van Loan).                        */
/* ------------------------------------------------------------------------ */

/* Solve A x = b, A n-by-n row-major, by LU with partial pivoting.  A and b  */
/* are copied.  Returns 0, or -1 on a zero or non-finite pivot.             */
int orc_lu_solve(int n, const double *Ain, const double *bin, double *x)
{
    double *A = (double *)malloc(sizeof(double) * n * n);
    double *b = (double *)malloc(sizeof(double) * n);
    memcpy(A, Ain, sizeof(double) * n * n);
    memcpy(b, bin, sizeof(double) * n);
    int rc = 0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[piv * n + k])) piv = i;
        if (!(fabs(A[piv * n + k]) > 0.0) || !isfinite(A[piv * n + k])) {
            rc = -1;
            goto done;
        }
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j];
                A[k * n + j] = A[piv * n + j];
                A[piv * n + j] = t;
            }
            double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
            b[i] -= l * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
        x[i] = s / A[i * n + i];
    }
done:
    free(A);
    free(b);
    return rc;
}

/* Least squares min |A x - b|_2, A m-by-n row-major (m >= n), by           */
/* Householder QR and back substitution.  Returns 0, or -1 if R is singular. */
int orc_lstsq(int m, int n, const double *Ain, const double *bin, double *x)
{
    double *A = (double *)malloc(sizeof(double) * m * n);
    double *b = (double *)malloc(sizeof(double) * m);
    double *v = (double *)malloc(sizeof(double) * m);
    memcpy(A, Ain, sizeof(double) * m * n);
    memcpy(b, bin, sizeof(double) * m);
    int rc = 0;
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += A[i * n + k] * A[i * n + k];
        nrm = sqrt(nrm);
        if (!(nrm > 0.0) || !isfinite(nrm)) {
            rc = -1;
            goto done;
        }
        double alpha = A[k * n + k] > 0.0 ? -nrm : nrm;
        for (int i = k; i < m; ++i) v[i] = A[i * n + k];
        v[k] -= alpha;
        double vv = 0.0;
        for (int i = k; i < m; ++i) vv += v[i] * v[i];
        if (vv > 0.0) {
            for (int j = k; j < n; ++j) {
                double d = 0.0;
                for (int i = k; i < m; ++i) d += v[i] * A[i * n + j];
                double f = 2.0 * d / vv;
                for (int i = k; i < m; ++i) A[i * n + j] -= f * v[i];
            }
            double d = 0.0;
            for (int i = k; i < m; ++i) d += v[i] * b[i];
            double f = 2.0 * d / vv;
            for (int i = k; i < m; ++i) b[i] -= f * v[i];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
        if (!(fabs(A[i * n + i]) > 0.0)) {
            rc = -1;
            goto done;
        }
        x[i] = s / A[i * n + i];
    }
done:
    free(A);
    free(b);
    free(v);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* One element: interpolation of the advected polynomial and the            */
/* constrained least-squares remap (Section 5.3).                            */
/* ------------------------------------------------------------------------ */

/* 1D: values of the advected interpolant (Eq. phi_stardef) at the element  */
/* faces xi = 0 and xi = 1 (Eq. remap_bnd), using the Lagrange basis on the  */
/* advected points xi_j + d_j (Eq. h_star).                                  */
void orc_faces_1d_split(int N, const double *xi, const double *d, const double *phs, double *e0,
                        double *e1)
{
    double a = 0.0, b = 0.0;
    for (int j = 0; j < N; ++j) {
        a += phs[j] * orc_lagrange_split(N, xi, d, j, 0.0, 0.0);
        b += phs[j] * orc_lagrange_split(N, xi, d, j, 1.0, 0.0);
    }
    *e0 = a;
    *e1 = b;
}

/* 1D remap: q = argmin |V q - phi*|^2 + w^2 |B q - g|^2 where V[p][i] =     */
/* h_i(xi_p + d_p) (Gauss-node basis at the advected particles) and B holds  */
/* the rows h_i(0), h_i(1) with the upwinded face values g = (gL, gR)        */
/* (Section 5.3 with the boundary rows weighted by w).  w = INFINITY is the  */
/* hard-constrained problem min |V q - phi*|^2 subject to B q = g, solved    */
/* through its Lagrange (KKT) conditions V^T V q + B^T lambda = V^T phi*,    */
/* B q = g, by LU.                                                           */
int orc_remap_1d_split_w(int N, const double *xi, const double *d, const double *phs, double gL,
                         double gR, double w, double *q)
{
    int m = N + 2;
    double *A = (double *)malloc(sizeof(double) * m * N);
    double *rhs = (double *)malloc(sizeof(double) * m);
    for (int p = 0; p < N; ++p) {
        for (int i = 0; i < N; ++i) A[p * N + i] = orc_lagrange_split(N, xi, ORC_ZEROS, i, xi[p], d[p]);
        rhs[p] = phs[p];
    }
    for (int i = 0; i < N; ++i) {
        A[N * N + i] = orc_lagrange(N, xi, i, 0.0);
        A[(N + 1) * N + i] = orc_lagrange(N, xi, i, 1.0);
    }
    rhs[N] = gL;
    rhs[N + 1] = gR;
    int rc;
    if (isinf(w)) {
        int k = N + 2;
        double *KKT = (double *)calloc((size_t)k * k, sizeof(double));
        double *b = (double *)calloc((size_t)k, sizeof(double));
        double *sol = (double *)malloc(sizeof(double) * k);
        for (int i = 0; i < N; ++i) {
            for (int j = 0; j < N; ++j) {
                double s = 0.0;
                for (int p = 0; p < N; ++p) s += A[p * N + i] * A[p * N + j];
                KKT[i * k + j] = s;
            }
            double s = 0.0;
            for (int p = 0; p < N; ++p) s += A[p * N + i] * phs[p];
            b[i] = s;
            KKT[i * k + N] = A[N * N + i];
            KKT[i * k + N + 1] = A[(N + 1) * N + i];
            KKT[N * k + i] = A[N * N + i];
            KKT[(N + 1) * k + i] = A[(N + 1) * N + i];
        }
        b[N] = gL;
        b[N + 1] = gR;
        rc = orc_lu_solve(k, KKT, b, sol);
        for (int i = 0; i < N; ++i) q[i] = sol[i];
        free(KKT);
        free(b);
        free(sol);
    } else {
        for (int r = N; r < m; ++r) {
            for (int i = 0; i < N; ++i) A[r * N + i] *= w;
            rhs[r] *= w;
        }
        rc = orc_lstsq(m, N, A, rhs, q);
    }
    free(A);
    free(rhs);
    return rc;
}

/* The unweighted remap (w = 1).                                             */
int orc_remap_1d_split(int N, const double *xi, const double *d, const double *phs, double gL,
                       double gR, double *q)
{
    return orc_remap_1d_split_w(N, xi, d, phs, gL, gR, 1.0, q);
}

/* The same with the advected particles given as absolute positions xs.      */
void orc_faces_1d(int N, const double *xs, const double *phs, double *e0, double *e1)
{
    orc_faces_1d_split(N, xs, ORC_ZEROS, phs, e0, e1);
}

int orc_remap_1d(int N, const double *xi, const double *xs, const double *phs, double gL, double gR,
                 double *q)
{
    /* xs_p = xi_p + (xs_p - xi_p) would round; use the positions as bases */
    int m = N + 2;
    double *A = (double *)malloc(sizeof(double) * m * N);
    double *rhs = (double *)malloc(sizeof(double) * m);
    for (int p = 0; p < N; ++p) {
        for (int i = 0; i < N; ++i) A[p * N + i] = orc_lagrange(N, xi, i, xs[p]);
        rhs[p] = phs[p];
    }
    for (int i = 0; i < N; ++i) {
        A[N * N + i] = orc_lagrange(N, xi, i, 0.0);
        A[(N + 1) * N + i] = orc_lagrange(N, xi, i, 1.0);
    }
    rhs[N] = gL;
    rhs[N + 1] = gR;
    int rc = orc_lstsq(m, N, A, rhs, q);
    free(A);
    free(rhs);
    return rc;
}

/* 2D tensor-product element, nodes p = j*N + i (x index i fastest).         */
/* V[p][(i',j')] = h_i'(x*_p) h_j'(y*_p) on the scattered advected particles, */
/* particle p at (bx_p + ox_p, by_p + oy_p) (base plus offset, see           */
/* orc_lagrange_split).                                                      */
static void orc_build_V2(int N, const double *xi, const double *bx, const double *ox, const double *by,
                         const double *oy, double *V)
{
    int n = N * N;
    for (int p = 0; p < n; ++p)
        for (int jj = 0; jj < N; ++jj)
            for (int ii = 0; ii < N; ++ii)
                V[p * n + jj * N + ii] = orc_lagrange_split(N, xi, ORC_ZEROS, ii, bx[p], ox[p]) *
                                         orc_lagrange_split(N, xi, ORC_ZEROS, jj, by[p], oy[p]);
}

/* 2D face values of the advected interpolant: alpha = V^{-1} phi* are its  */
/* nodal values (Eq. phi_star in tensor form); then at the N Gauss-node      */
/* positions of each face: left (xi=0), right (xi=1), bottom (eta=0), top.   */
/* faces[0..N) left, [N..2N) right, [2N..3N) bottom, [3N..4N) top.           */
static int orc_faces_2d_core(int N, const double *xi, const double *bx, const double *ox,
                             const double *by, const double *oy, const double *phs, double *faces)
{
    int n = N * N;
    double *V = (double *)malloc(sizeof(double) * n * n);
    double *alpha = (double *)malloc(sizeof(double) * n);
    orc_build_V2(N, xi, bx, ox, by, oy, V);
    int rc = orc_lu_solve(n, V, phs, alpha);
    if (rc == 0) {
        for (int j = 0; j < N; ++j) {
            double l = 0.0, r = 0.0;
            for (int ii = 0; ii < N; ++ii) {
                l += alpha[j * N + ii] * orc_lagrange(N, xi, ii, 0.0);
                r += alpha[j * N + ii] * orc_lagrange(N, xi, ii, 1.0);
            }
            faces[j] = l;
            faces[N + j] = r;
        }
        for (int i = 0; i < N; ++i) {
            double bo = 0.0, to = 0.0;
            for (int jj = 0; jj < N; ++jj) {
                bo += alpha[jj * N + i] * orc_lagrange(N, xi, jj, 0.0);
                to += alpha[jj * N + i] * orc_lagrange(N, xi, jj, 1.0);
            }
            faces[2 * N + i] = bo;
            faces[3 * N + i] = to;
        }
    }
    free(V);
    free(alpha);
    return rc;
}

/* 2D remap: min |V q - phi*|^2 + w^2 |B q - g|^2, B = the 4N face rows at  */
/* the Gauss-node positions along each face, g ordered as in the face values */
/* (w finite).                                                               */
static int orc_remap_2d_core(int N, const double *xi, const double *bx, const double *ox,
                             const double *by, const double *oy, const double *phs, const double *g,
                             double w, double *q)
{
    int n = N * N, m = n + 4 * N;
    double *A = (double *)calloc((size_t)m * n, sizeof(double));
    double *rhs = (double *)malloc(sizeof(double) * m);
    orc_build_V2(N, xi, bx, ox, by, oy, A);
    for (int p = 0; p < n; ++p) rhs[p] = phs[p];
    for (int j = 0; j < N; ++j)
        for (int ii = 0; ii < N; ++ii) {
            A[(n + j) * n + j * N + ii] = orc_lagrange(N, xi, ii, 0.0);
            A[(n + N + j) * n + j * N + ii] = orc_lagrange(N, xi, ii, 1.0);
        }
    for (int i = 0; i < N; ++i)
        for (int jj = 0; jj < N; ++jj) {
            A[(n + 2 * N + i) * n + jj * N + i] = orc_lagrange(N, xi, jj, 0.0);
            A[(n + 3 * N + i) * n + jj * N + i] = orc_lagrange(N, xi, jj, 1.0);
        }
    for (int f = 0; f < 4 * N; ++f) rhs[n + f] = g[f];
    for (int r = n; r < m; ++r) {
        for (int i = 0; i < n; ++i) A[r * n + i] *= w;
        rhs[r] *= w;
    }
    int rc = orc_lstsq(m, n, A, rhs, q);
    free(A);
    free(rhs);
    return rc;
}

/* Absolute particle positions xs, ys. */
int orc_faces_2d(int N, const double *xi, const double *xs, const double *ys, const double *phs,
                 double *faces)
{
    return orc_faces_2d_core(N, xi, xs, ORC_ZEROS, ys, ORC_ZEROS, phs, faces);
}

int orc_remap_2d(int N, const double *xi, const double *xs, const double *ys, const double *phs,
                 const double *g, double *q)
{
    return orc_remap_2d_core(N, xi, xs, ORC_ZEROS, ys, ORC_ZEROS, phs, g, 1.0, q);
}

/* Particles at the Gauss nodes plus displacements dx, dy (element units). */
int orc_faces_2d_split(int N, const double *xi, const double *dx, const double *dy,
                       const double *phs, double *faces)
{
    int n = N * N;
    double *bx = (double *)malloc(sizeof(double) * n), *by = (double *)malloc(sizeof(double) * n);
    for (int p = 0; p < n; ++p) {
        bx[p] = xi[p % N];
        by[p] = xi[p / N];
    }
    int rc = orc_faces_2d_core(N, xi, bx, dx, by, dy, phs, faces);
    free(bx);
    free(by);
    return rc;
}

int orc_remap_2d_split_w(int N, const double *xi, const double *dx, const double *dy,
                         const double *phs, const double *g, double w, double *q)
{
    int n = N * N;
    double *bx = (double *)malloc(sizeof(double) * n), *by = (double *)malloc(sizeof(double) * n);
    for (int p = 0; p < n; ++p) {
        bx[p] = xi[p % N];
        by[p] = xi[p / N];
    }
    int rc = orc_remap_2d_core(N, xi, bx, dx, by, dy, phs, g, w, q);
    free(bx);
    free(by);
    return rc;
}

int orc_remap_2d_split(int N, const double *xi, const double *dx, const double *dy,
                       const double *phs, const double *g, double *q)
{
    return orc_remap_2d_split_w(N, xi, dx, dy, phs, g, 1.0, q);
}

/* ------------------------------------------------------------------------ */
/* Problem description and prescribed fields.                               */
/* ------------------------------------------------------------------------ */
enum { ORC_U_CONST = 0, ORC_U_SIN = 1, ORC_U_ROTATION = 2, ORC_U_NODAL = 3 };
enum { ORC_D_CONST = 0, ORC_D_COS = 1, ORC_D_SINSIN = 2, ORC_D_NODAL = 3 };
enum { ORC_PHI_GAUSS = 0, ORC_PHI_FOURIER = 1, ORC_PHI_SINE = 2, ORC_PHI_SINSIN = 3 };

typedef struct {
    int dim;
    int K[2];
    double lo[2], hi[2];
    int N;
    int drift_kind;
    double drift_p[8];
    int diff_kind;
    double diff_p[8];
    int phi0_kind;
    double phi0_p[40];
    unsigned long long seed;
    double dt;
    double omega; /* weight of the boundary rows of the remap; <= 0 means 1; INFINITY: hard (1D) */
    int periodic;     /* 1: periodic; 0: Dirichlet ghost values at x = lo, hi (1D)         */
    int reseed_every; /* > 0: every sample set to the sample mean after each step n with    */
                      /* (n + 1) % reseed_every == 0 (Eq. re-seed); 0: never                */
    /* Nodal fields, the form a field solver hands over (Section 5.2 takes    */
    /* du/dx from the DSEM solver).  Nodes: [dim][E][n] drift components,     */
    /* [E][n] D.  Interface points (optional, NULL: derived): the normal      */
    /* drift component or D, 1D [K+1] at x = lo + f h; 2D the vertical        */
    /* interfaces [Ky][Kx+1][N] then the horizontal ones [Ky+1][Kx][N].       */
    const double *drift_nodal, *drift_face;
    const double *diff_nodal, *diff_face;
} orc_problem;

/* Drift u(x) (1D: u[0]; 2D: u[0], u[1]).                                    */
/*  CONST:    u = (p0, p1)                                                   */
/*  SIN:      u = p0 + p1 sin(p2 pi x)                       (1D)            */
/*  ROTATION: u = p0 (-(y - p2), x - p1)   solid body about (p1, p2)  (2D)   */
static void orc_drift(const orc_problem *pb, double x, double y, double *u)
{
    const double *p = pb->drift_p;
    if (pb->drift_kind == ORC_U_CONST) {
        u[0] = p[0];
        u[1] = p[1];
    } else if (pb->drift_kind == ORC_U_SIN) {
        u[0] = p[0] + p[1] * sin(p[2] * M_PI * x);
        u[1] = 0.0;
    } else {
        u[0] = -p[0] * (y - p[2]);
        u[1] = p[0] * (x - p[1]);
    }
}

/* Diffusion coefficient D(x) >= 0.                                          */
/*  CONST:  p0;  COS: p0 (1 + p1 cos(p2 pi x));                              */
/*  SINSIN: p0 (1 + p1 sin(p2 pi x) sin(p3 pi y))                           */
static double orc_diffusion(const orc_problem *pb, double x, double y)
{
    const double *p = pb->diff_p;
    if (pb->diff_kind == ORC_D_CONST) return p[0];
    if (pb->diff_kind == ORC_D_COS) return p[0] * (1.0 + p[1] * cos(p[2] * M_PI * x));
    return p[0] * (1.0 + p[1] * sin(p[2] * M_PI * x) * sin(p[3] * M_PI * y));
}

/* Initial condition phi0(x).                                                */
/*  GAUSS:   p0 exp(-|x - c|^2 / (2 p1^2)), c = (p2, p3), summed over the     */
/*           nearest periodic images in every periodic direction             */
/*  FOURIER: p0 + sum_{k=1}^{p2} (p[3+2(k-1)] cos(k p1 pi x)                 */
/*                              + p[4+2(k-1)] sin(k p1 pi x))      (1D)      */
/*  SINE:    p0 + p1 sin(2 pi p2 x)                                  (1D)    */
/*  SINSIN:  p0 + p1 sin(2 pi p2 x) sin(2 pi p2 y)                   (2D)    */
static double orc_phi0(const orc_problem *pb, double x, double y)
{
    const double *p = pb->phi0_p;
    if (pb->phi0_kind == ORC_PHI_GAUSS) {
        double Lx = pb->hi[0] - pb->lo[0], Ly = pb->hi[1] - pb->lo[1];
        double v = 0.0;
        int ny = pb->dim == 2 ? 1 : 0;
        for (int ix = -1; ix <= 1; ++ix)
            for (int iy = -ny; iy <= ny; ++iy) {
                double dx = x - p[2] + ix * Lx;
                double r2 = dx * dx;
                if (pb->dim == 2) {
                    double dy = y - p[3] + iy * Ly;
                    r2 += dy * dy;
                }
                v += exp(-r2 / (2.0 * p[1] * p[1]));
            }
        return p[0] * v;
    }
    if (pb->phi0_kind == ORC_PHI_FOURIER) {
        double v = p[0];
        int nk = (int)p[2];
        for (int k = 1; k <= nk; ++k)
            v += p[3 + 2 * (k - 1)] * cos(k * p[1] * M_PI * x) +
                 p[4 + 2 * (k - 1)] * sin(k * p[1] * M_PI * x);
        return v;
    }
    if (pb->phi0_kind == ORC_PHI_SINE) return p[0] + p[1] * sin(2.0 * M_PI * p[2] * x);
    return p[0] + p[1] * sin(2.0 * M_PI * p[2] * x) * sin(2.0 * M_PI * p[2] * y);
}

/* Per-node and per-face coefficients of one problem (shared by samples).    */
typedef struct {
    int dim, N, n, E, Kx, Ky;
    double hx, hy;
    double *xi;          /* [N] reference nodes                               */
    double *ax, *ay;     /* [E][n] u_x dt, u_y dt at the nodes                */
    double *b;           /* [E][n] sqrt(2 D) at the nodes                     */
    double *c;           /* [E][n] 1 - dt div u (Eq. advection_phi)           */
    double *div;         /* [E][n] du_j/dx_j at the nodes                     */
    double *afx, *bfx;   /* [Ky][Kx][N(2D) or 1] vertical faces: u_x dt, sqrt(2D) */
    double *afy, *bfy;   /* [Ky][Kx][N] horizontal faces (2D)                 */
    double omega;        /* boundary-row weight of the remap                  */
    int periodic;        /* 0: Dirichlet boundaries                           */
    double afx_hi, bfx_hi; /* 1D: u dt and sqrt(2D) at the right boundary x = hi */
    double *afx_hi2, *bfx_hi2; /* 2D: [Ky][N] u_x dt, sqrt(2D) on the face x = hi */
    double *afy_hi2, *bfy_hi2; /* 2D: [Kx][N] u_y dt, sqrt(2D) on the face y = hi */
} orc_coeffs;

static void orc_coeffs_free(orc_coeffs *cf)
{
    free(cf->xi);
    free(cf->ax);
    free(cf->ay);
    free(cf->b);
    free(cf->c);
    free(cf->div);
    free(cf->afx);
    free(cf->bfx);
    free(cf->afy);
    free(cf->bfy);
    free(cf->afx_hi2);
    free(cf->bfx_hi2);
    free(cf->afy_hi2);
    free(cf->bfy_hi2);
}

/* Node (x, y) of node p in element e. */
static void orc_node_xy(const orc_problem *pb, const orc_coeffs *cf, int e, int p, double *x,
                        double *y)
{
    int kx = e % cf->Kx, ky = e / cf->Kx;
    int i = p % cf->N, j = p / cf->N;
    *x = pb->lo[0] + (kx + cf->xi[i]) * cf->hx;
    *y = cf->dim == 2 ? pb->lo[1] + (ky + cf->xi[j]) * cf->hy : 0.0;
}

/* Element index of the element at position k along direction dir on grid  */
/* line `line` (the row ky for dir 0, the column kx for dir 1).              */
static int orc_elem_on_line(const orc_coeffs *cf, int dir, int line, int k)
{
    return dir == 0 ? line * cf->Kx + k : k * cf->Kx + line;
}

/* Trace of element e's nodal interpolant of `vals` ([E][n]) on its face     */
/* xi_dir = side (0 or 1), at the face's Gauss point pt (2D; 0 in 1D): the   */
/* Lagrange expansion of the element's nodal values (Section 3) evaluated at */
/* the face.                                                                 */
static double orc_trace(const orc_coeffs *cf, const double *vals, int e, int dir, int side, int pt)
{
    int N = cf->N;
    double s = 0.0;
    for (int l = 0; l < N; ++l) {
        int node = cf->dim == 1 ? l : (dir == 0 ? pt * N + l : l * N + pt);
        s += orc_lagrange(N, cf->xi, l, (double)side) * vals[(size_t)e * cf->n + node];
    }
    return s;
}

/* A nodal field at interface point pt of interface idx (0..K along dir) on  */
/* grid line `line`: the caller's interface table if given, else the mean of */
/* the traces of the elements on both sides (the one inside trace at a       */
/* Dirichlet boundary).  On a periodic mesh interface K is interface 0.      */
/* Reading: Section 5.2 takes the fields from the DSEM solver and the upwind */
/* rule (Eq. bnd_update) needs them at the interface points; the paper does  */
/* not say how, and the mean of the two traces is the central value of a     */
/* discontinuous spectral element method.                                    */
static double orc_iface_nodal(const orc_problem *pb, const orc_coeffs *cf, const double *vals,
                              const double *face, int dir, int line, int idx, int pt)
{
    int K = dir == 0 ? cf->Kx : cf->Ky;
    if (pb->periodic && idx == K) idx = 0;
    if (face) {
        if (cf->dim == 1) return face[idx];
        if (dir == 0) return face[((size_t)line * (cf->Kx + 1) + idx) * cf->N + pt];
        return face[(size_t)cf->Ky * (cf->Kx + 1) * cf->N + ((size_t)idx * cf->Kx + line) * cf->N + pt];
    }
    double left = 0.0, right = 0.0;
    int have_left = idx > 0 || pb->periodic, have_right = idx < K;
    if (have_left)
        left = orc_trace(cf, vals, orc_elem_on_line(cf, dir, line, (idx - 1 + K) % K), dir, 1, pt);
    if (have_right) right = orc_trace(cf, vals, orc_elem_on_line(cf, dir, line, idx), dir, 0, pt);
    if (have_left && have_right) return 0.5 * (left + right);
    return have_left ? left : right;
}

/* Normal drift u_dir and D at an interface point, the quantities of the     */
/* upwind test sigma = u dt + sqrt(2 D) dW (Eq. bnd_update).  Analytic kinds */
/* are evaluated at (x, y); nodal ones by orc_iface_nodal, D clipped at 0    */
/* where a derived trace undershoots (D >= 0 on the nodes does not bound the */
/* interpolant between them).  Returns -1 for a negative given value.        */
static int orc_face_fields(const orc_problem *pb, const orc_coeffs *cf, int dir, int line, int idx,
                           int pt, double x, double y, double *un, double *D)
{
    if (pb->drift_kind == ORC_U_NODAL) {
        *un = orc_iface_nodal(pb, cf, pb->drift_nodal + (size_t)dir * cf->E * cf->n, pb->drift_face,
                              dir, line, idx, pt);
    } else {
        double u[2];
        orc_drift(pb, x, y, u);
        *un = u[dir];
    }
    if (pb->diff_kind == ORC_D_NODAL) {
        *D = orc_iface_nodal(pb, cf, pb->diff_nodal, pb->diff_face, dir, line, idx, pt);
        if (pb->diff_face) {
            if (!(*D >= 0.0)) return -1;
        } else if (*D < 0.0) {
            *D = 0.0;
        }
    } else {
        *D = orc_diffusion(pb, x, y);
    }
    return 0;
}

/* Coefficients of Section 5.2: a = u dt, b = sqrt(2 D) at the Gauss nodes   */
/* (Eq. def_dx, explicit in time), c = 1 - dt du_j/dx_j (Eq. advection_phi) */
/* with the divergence by spectral differentiation of the nodal drift within */
/* the element (the paper takes it from the DSEM field solver).              */
static int orc_build_coeffs(const orc_problem *pb, orc_coeffs *cf)
{
    memset(cf, 0, sizeof(*cf));
    int N = pb->N, d = pb->dim;
    cf->dim = d;
    cf->N = N;
    cf->n = d == 2 ? N * N : N;
    cf->Kx = pb->K[0];
    cf->Ky = d == 2 ? pb->K[1] : 1;
    cf->E = cf->Kx * cf->Ky;
    cf->hx = (pb->hi[0] - pb->lo[0]) / cf->Kx;
    cf->hy = d == 2 ? (pb->hi[1] - pb->lo[1]) / cf->Ky : 1.0;
    cf->omega = pb->omega > 0.0 ? pb->omega : 1.0;
    cf->periodic = pb->periodic;
    int E = cf->E, n = cf->n;
    cf->xi = (double *)malloc(sizeof(double) * N);
    orc_nodes(N, cf->xi);
    cf->ax = (double *)calloc((size_t)E * n, sizeof(double));
    cf->ay = (double *)calloc((size_t)E * n, sizeof(double));
    cf->b = (double *)calloc((size_t)E * n, sizeof(double));
    cf->c = (double *)calloc((size_t)E * n, sizeof(double));
    cf->div = (double *)calloc((size_t)E * n, sizeof(double));
    int nf = d == 2 ? N : 1;
    cf->afx = (double *)calloc((size_t)E * nf, sizeof(double));
    cf->bfx = (double *)calloc((size_t)E * nf, sizeof(double));
    cf->afy = (double *)calloc((size_t)E * nf, sizeof(double));
    cf->bfy = (double *)calloc((size_t)E * nf, sizeof(double));
    int rc = 0;
    double *ux = (double *)malloc(sizeof(double) * n), *uy = (double *)malloc(sizeof(double) * n);
    for (int e = 0; e < E; ++e) {
        for (int p = 0; p < n; ++p) {
            double x, y, u[2], D;
            orc_node_xy(pb, cf, e, p, &x, &y);
            if (pb->drift_kind == ORC_U_NODAL) {
                u[0] = pb->drift_nodal[(size_t)e * n + p];
                u[1] = d == 2 ? pb->drift_nodal[(size_t)E * n + (size_t)e * n + p] : 0.0;
            } else {
                orc_drift(pb, x, y, u);
            }
            D = pb->diff_kind == ORC_D_NODAL ? pb->diff_nodal[(size_t)e * n + p] : orc_diffusion(pb, x, y);
            if (!(D >= 0.0)) { rc = -1; goto done; }
            ux[p] = u[0];
            uy[p] = u[1];
            cf->ax[e * n + p] = u[0] * pb->dt;
            cf->ay[e * n + p] = u[1] * pb->dt;
            cf->b[e * n + p] = sqrt(2.0 * D);
        }
        for (int p = 0; p < n; ++p) {
            int i = p % N, j = p / N;
            double div = 0.0;
            if (d == 1) {
                for (int m = 0; m < N; ++m)
                    div += orc_lagrange_deriv(N, cf->xi, m, cf->xi[i]) * ux[m];
                div /= cf->hx;
            } else {
                double dx = 0.0, dy = 0.0;
                for (int m = 0; m < N; ++m) {
                    dx += orc_lagrange_deriv(N, cf->xi, m, cf->xi[i]) * ux[j * N + m];
                    dy += orc_lagrange_deriv(N, cf->xi, m, cf->xi[j]) * uy[m * N + i];
                }
                div = dx / cf->hx + dy / cf->hy;
            }
            cf->div[e * n + p] = div;
            cf->c[e * n + p] = 1.0 - pb->dt * div;
        }
        /* faces at the low side of element e: vertical face x = x_kx, and   */
        /* (2D) horizontal face y = y_ky, at the Gauss-node positions.       */
        int kx = e % cf->Kx, ky = e / cf->Kx;
        for (int f = 0; f < nf; ++f) {
            double un, D;
            double xf = pb->lo[0] + kx * cf->hx;
            double yf = d == 2 ? pb->lo[1] + (ky + cf->xi[f]) * cf->hy : 0.0;
            if (orc_face_fields(pb, cf, 0, ky, kx, d == 2 ? f : 0, xf, yf, &un, &D) != 0) { rc = -1; goto done; }
            cf->afx[e * nf + f] = un * pb->dt;
            cf->bfx[e * nf + f] = sqrt(2.0 * D);
            if (d == 2) {
                double xh = pb->lo[0] + (kx + cf->xi[f]) * cf->hx;
                double yh = pb->lo[1] + ky * cf->hy;
                if (orc_face_fields(pb, cf, 1, kx, ky, f, xh, yh, &un, &D) != 0) { rc = -1; goto done; }
                cf->afy[e * nf + f] = un * pb->dt;
                cf->bfy[e * nf + f] = sqrt(2.0 * D);
            }
        }
    }
    if (d == 1) {
        double un, D;
        if (orc_face_fields(pb, cf, 0, 0, cf->Kx, 0, pb->hi[0], 0.0, &un, &D) != 0) { rc = -1; goto done; }
        cf->afx_hi = un * pb->dt;
        cf->bfx_hi = sqrt(2.0 * D);
    } else {
        cf->afx_hi2 = (double *)calloc((size_t)cf->Ky * N, sizeof(double));
        cf->bfx_hi2 = (double *)calloc((size_t)cf->Ky * N, sizeof(double));
        cf->afy_hi2 = (double *)calloc((size_t)cf->Kx * N, sizeof(double));
        cf->bfy_hi2 = (double *)calloc((size_t)cf->Kx * N, sizeof(double));
        for (int ky = 0; ky < cf->Ky; ++ky)
            for (int f = 0; f < N; ++f) { /* x = hi at the Gauss nodes of row ky */
                double un, D, yf = pb->lo[1] + (ky + cf->xi[f]) * cf->hy;
                if (orc_face_fields(pb, cf, 0, ky, cf->Kx, f, pb->hi[0], yf, &un, &D) != 0) { rc = -1; goto done; }
                cf->afx_hi2[ky * N + f] = un * pb->dt;
                cf->bfx_hi2[ky * N + f] = sqrt(2.0 * D);
            }
        for (int kx = 0; kx < cf->Kx; ++kx)
            for (int f = 0; f < N; ++f) { /* y = hi at the Gauss nodes of column kx */
                double un, D, xf = pb->lo[0] + (kx + cf->xi[f]) * cf->hx;
                if (orc_face_fields(pb, cf, 1, kx, cf->Ky, f, xf, pb->hi[1], &un, &D) != 0) { rc = -1; goto done; }
                cf->afy_hi2[kx * N + f] = un * pb->dt;
                cf->bfy_hi2[kx * N + f] = sqrt(2.0 * D);
            }
    }
done:
    free(ux);
    free(uy);
    return rc;
}

/* Initial nodal state phi0 at the Gauss nodes, [E][n] (Eq. soln_init; every */
/* sample starts from the same phi0).                                        */
int orc_init_state(const orc_problem *pb, double *out)
{
    orc_coeffs cf;
    if (orc_build_coeffs(pb, &cf) != 0) {
        orc_coeffs_free(&cf);
        return -1;
    }
    for (int e = 0; e < cf.E; ++e)
        for (int p = 0; p < cf.n; ++p) {
            double x, y;
            orc_node_xy(pb, &cf, e, p, &x, &y);
            out[e * cf.n + p] = orc_phi0(pb, x, y);
        }
    orc_coeffs_free(&cf);
    return 0;
}

/* Node coefficients for inspection: a (x part), b, c, each [E][n]. */
int orc_get_coeffs(const orc_problem *pb, double *ax, double *ay, double *b, double *c)
{
    orc_coeffs cf;
    if (orc_build_coeffs(pb, &cf) != 0) {
        orc_coeffs_free(&cf);
        return -1;
    }
    size_t sz = sizeof(double) * cf.E * cf.n;
    memcpy(ax, cf.ax, sz);
    memcpy(ay, cf.ay, sz);
    memcpy(b, cf.b, sz);
    memcpy(c, cf.c, sz);
    orc_coeffs_free(&cf);
    return 0;
}

/* Interface coefficients for inspection, in the interface layout of the    */
/* nodal fields: a = u_normal dt and b = sqrt(2 D); 1D [K+1], 2D the         */
/* vertical interfaces [Ky][Kx+1][N] then the horizontal [Ky+1][Kx][N].      */
/* On a periodic mesh the last interface of a line repeats the first.        */
int orc_get_face_coeffs(const orc_problem *pb, double *a, double *b)
{
    orc_coeffs cf;
    if (orc_build_coeffs(pb, &cf) != 0) {
        orc_coeffs_free(&cf);
        return -1;
    }
    int N = cf.N, Kx = cf.Kx, Ky = cf.Ky;
    if (cf.dim == 1) {
        for (int f = 0; f <= Kx; ++f) {
            a[f] = f < Kx ? cf.afx[f] : (cf.periodic ? cf.afx[0] : cf.afx_hi);
            b[f] = f < Kx ? cf.bfx[f] : (cf.periodic ? cf.bfx[0] : cf.bfx_hi);
        }
    } else {
        size_t o = 0;
        for (int ky = 0; ky < Ky; ++ky)
            for (int f = 0; f <= Kx; ++f)
                for (int j = 0; j < N; ++j, ++o) {
                    if (f < Kx || cf.periodic) {
                        int e = ky * Kx + (f < Kx ? f : 0);
                        a[o] = cf.afx[e * N + j];
                        b[o] = cf.bfx[e * N + j];
                    } else {
                        a[o] = cf.afx_hi2[ky * N + j];
                        b[o] = cf.bfx_hi2[ky * N + j];
                    }
                }
        for (int g = 0; g <= Ky; ++g)
            for (int kx = 0; kx < Kx; ++kx)
                for (int i = 0; i < N; ++i, ++o) {
                    if (g < Ky || cf.periodic) {
                        int e = (g < Ky ? g : 0) * Kx + kx;
                        a[o] = cf.afy[e * N + i];
                        b[o] = cf.bfy[e * N + i];
                    } else {
                        a[o] = cf.afy_hi2[kx * N + i];
                        b[o] = cf.bfy_hi2[kx * N + i];
                    }
                }
    }
    orc_coeffs_free(&cf);
    return 0;
}

/* One SL step of one sample (Sections 5.2-5.3), state Q [E][n] in place.    */
/* One SL step of one 1D sample.  ghost (Dirichlet only): the boundary values */
/* at x = lo and x = hi at the end of the step, the ghost solution that takes */
/* the place of the missing neighbour in the upwind rule.                     */
static int orc_step_1d(const orc_coeffs *cf, double dt, double dW, const double *ghost, double *Q)
{
    int N = cf->N, K = cf->Kx;
    double *d = (double *)malloc(sizeof(double) * K * N);
    double *phs = (double *)malloc(sizeof(double) * K * N);
    double *e0 = (double *)malloc(sizeof(double) * K);
    double *e1 = (double *)malloc(sizeof(double) * K);
    double *g = (double *)malloc(sizeof(double) * (K + 1)); /* interface values, g[K]: x = hi */
    int rc = 0;
    /* advance (Eq. def_dx): particle p moves from xi_p by d_p = (u dt +      */
    /* sqrt(2D) dW) / h in element units; compositional update              */
    /* (Eq. advection_phi): phi* = phi + dt (-phi du/dx)                     */
    for (int k = 0; k < K; ++k)
        for (int p = 0; p < N; ++p) {
            d[k * N + p] = (cf->ax[k * N + p] + cf->b[k * N + p] * dW) / cf->hx;
            phs[k * N + p] = Q[k * N + p] + dt * (-Q[k * N + p] * cf->div[k * N + p]);
        }
    for (int k = 0; k < K; ++k) orc_faces_1d_split(N, cf->xi, d + k * N, phs + k * N, &e0[k], &e1[k]);
    /* upwinding (Eq. bnd_update): interface f sits between elements f-1 and */
    /* f (periodic); take the left element's value when u dt + sqrt(2D) dW > 0 */
    for (int f = 0; f < K; ++f) {
        double sigma = cf->afx[f] + cf->bfx[f] * dW;
        double left = (f == 0 && !cf->periodic) ? ghost[0] : e1[(f - 1 + K) % K];
        g[f] = sigma > 0.0 ? left : e0[f];
    }
    if (cf->periodic)
        g[K] = g[0];
    else {
        double sigma = cf->afx_hi + cf->bfx_hi * dW;
        g[K] = sigma > 0.0 ? e1[K - 1] : ghost[1];
    }
    for (int k = 0; k < K && rc == 0; ++k)
        rc = orc_remap_1d_split_w(N, cf->xi, d + k * N, phs + k * N, g[k], g[k + 1], cf->omega, Q + k * N);
    free(d);
    free(phs);
    free(e0);
    free(e1);
    free(g);
    return rc;
}

/* One SL step of one 2D sample.  ghost (Dirichlet only): boundary values at */
/* the face points after the step, [left Ky][N] (x = lo), [right Ky][N]       */
/* (x = hi), [bottom Kx][N] (y = lo), [top Kx][N] (y = hi), each at the Gauss */
/* nodes along the face; they take the place of the missing neighbour in the */
/* upwind rule.                                                              */
static int orc_step_2d(const orc_coeffs *cf, double dt, const double dW[2], const double *ghost, double *Q)
{
    int N = cf->N, n = cf->n, Kx = cf->Kx, Ky = cf->Ky, E = cf->E;
    double *dx = (double *)malloc(sizeof(double) * E * n);
    double *dy = (double *)malloc(sizeof(double) * E * n);
    double *phs = (double *)malloc(sizeof(double) * E * n);
    double *faces = (double *)malloc(sizeof(double) * E * 4 * N);
    double *gv = (double *)malloc(sizeof(double) * E * N); /* vertical face at low x of e */
    double *gh = (double *)malloc(sizeof(double) * E * N); /* horizontal face at low y of e */
    double *g = (double *)malloc(sizeof(double) * 4 * N);
    double *gvR = (double *)malloc(sizeof(double) * Ky * N); /* x = hi interface (Dirichlet) */
    double *ghT = (double *)malloc(sizeof(double) * Kx * N); /* y = hi interface (Dirichlet) */
    const int dir = !cf->periodic;
    const double *gL = dir ? ghost : NULL, *gR = dir ? ghost + Ky * N : NULL;
    const double *gB = dir ? ghost + 2 * Ky * N : NULL, *gT = dir ? ghost + 2 * Ky * N + Kx * N : NULL;
    int rc = 0;
    for (int e = 0; e < E; ++e)
        for (int p = 0; p < n; ++p) {
            dx[e * n + p] = (cf->ax[e * n + p] + cf->b[e * n + p] * dW[0]) / cf->hx;
            dy[e * n + p] = (cf->ay[e * n + p] + cf->b[e * n + p] * dW[1]) / cf->hy;
            phs[e * n + p] = Q[e * n + p] + dt * (-Q[e * n + p] * cf->div[e * n + p]);
        }
    for (int e = 0; e < E && rc == 0; ++e)
        rc = orc_faces_2d_split(N, cf->xi, dx + e * n, dy + e * n, phs + e * n, faces + e * 4 * N);
    for (int ky = 0; ky < Ky && rc == 0; ++ky)
        for (int kx = 0; kx < Kx; ++kx) {
            int e = ky * Kx + kx;
            int eL = ky * Kx + (kx - 1 + Kx) % Kx;   /* left neighbour  */
            int eB = ((ky - 1 + Ky) % Ky) * Kx + kx; /* lower neighbour */
            for (int f = 0; f < N; ++f) {
                double sx = cf->afx[e * N + f] + cf->bfx[e * N + f] * dW[0];
                double left = (dir && kx == 0) ? gL[ky * N + f] : faces[eL * 4 * N + N + f];
                gv[e * N + f] = sx > 0.0 ? left : faces[e * 4 * N + f];
                double sy = cf->afy[e * N + f] + cf->bfy[e * N + f] * dW[1];
                double below = (dir && ky == 0) ? gB[kx * N + f] : faces[eB * 4 * N + 3 * N + f];
                gh[e * N + f] = sy > 0.0 ? below : faces[e * 4 * N + 2 * N + f];
            }
        }
    if (dir) {
        for (int ky = 0; ky < Ky; ++ky)
            for (int f = 0; f < N; ++f) {
                int e = ky * Kx + Kx - 1;
                double sx = cf->afx_hi2[ky * N + f] + cf->bfx_hi2[ky * N + f] * dW[0];
                gvR[ky * N + f] = sx > 0.0 ? faces[e * 4 * N + N + f] : gR[ky * N + f];
            }
        for (int kx = 0; kx < Kx; ++kx)
            for (int f = 0; f < N; ++f) {
                int e = (Ky - 1) * Kx + kx;
                double sy = cf->afy_hi2[kx * N + f] + cf->bfy_hi2[kx * N + f] * dW[1];
                ghT[kx * N + f] = sy > 0.0 ? faces[e * 4 * N + 3 * N + f] : gT[kx * N + f];
            }
    }
    for (int ky = 0; ky < Ky && rc == 0; ++ky)
        for (int kx = 0; kx < Kx && rc == 0; ++kx) {
            int e = ky * Kx + kx;
            int eR = ky * Kx + (kx + 1) % Kx;
            int eT = ((ky + 1) % Ky) * Kx + kx;
            for (int f = 0; f < N; ++f) {
                g[f] = gv[e * N + f];
                g[N + f] = (dir && kx == Kx - 1) ? gvR[ky * N + f] : gv[eR * N + f];
                g[2 * N + f] = gh[e * N + f];
                g[3 * N + f] = (dir && ky == Ky - 1) ? ghT[kx * N + f] : gh[eT * N + f];
            }
            rc = orc_remap_2d_split_w(N, cf->xi, dx + e * n, dy + e * n, phs + e * n, g, cf->omega, Q + e * n);
        }
    free(dx);
    free(dy);
    free(phs);
    free(faces);
    free(gv);
    free(gh);
    free(g);
    free(gvR);
    free(ghT);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Driver: samples [s0, s0+ns) through steps [step0, step0+nsteps).          */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_problem *pb;
    const orc_coeffs *cf;
    long step0;
    int nsteps, s_begin, s_end, s0;
    const double *state_in;
    const double *phi0; /* [E][n] initial state when state_in is NULL */
    double *state_out;
    double *sum, *sumsq; /* this thread's partial sums [E][n] */
    const double *ghost; /* [nsteps][2] Dirichlet values (1D, non-periodic), else NULL */
    int rc;
} orc_job;

/* Boundary values per step: 2 in 1D (x = lo, hi), 2 (Kx + Ky) N in 2D.    */
static int orc_ghost_width(const orc_coeffs *cf) { return cf->dim == 1 ? 2 : 2 * (cf->Kx + cf->Ky) * cf->N; }

static void *orc_worker(void *arg)
{
    orc_job *jb = (orc_job *)arg;
    const orc_coeffs *cf = jb->cf;
    size_t sz = (size_t)cf->E * cf->n;
    double *Q = (double *)malloc(sizeof(double) * sz);
    double sdt = sqrt(jb->pb->dt);
    jb->rc = 0;
    for (int s = jb->s_begin; s < jb->s_end && jb->rc == 0; ++s) {
        if (jb->state_in)
            memcpy(Q, jb->state_in + (size_t)(s - jb->s0) * sz, sizeof(double) * sz);
        else
            memcpy(Q, jb->phi0, sizeof(double) * sz);
        for (int t = 0; t < jb->nsteps && jb->rc == 0; ++t) {
            double z[2], dW[2];
            orc_normals(jb->pb->seed, (uint32_t)(jb->step0 + t), (uint32_t)s, 0u, z);
            dW[0] = sdt * z[0];
            dW[1] = sdt * z[1];
            const double *gt = jb->ghost ? jb->ghost + (size_t)orc_ghost_width(cf) * t : NULL;
            jb->rc = cf->dim == 1 ? orc_step_1d(cf, jb->pb->dt, dW[0], gt, Q) : orc_step_2d(cf, jb->pb->dt, dW, gt, Q);
        }
        if (jb->state_out) memcpy(jb->state_out + (size_t)(s - jb->s0) * sz, Q, sizeof(double) * sz);
        if (jb->sum)
            for (size_t i = 0; i < sz; ++i) {
                jb->sum[i] += Q[i];
                jb->sumsq[i] += Q[i] * Q[i];
            }
    }
    free(Q);
    return NULL;
}

/* Samples [s0, s0+ns) through steps [step0, step0+nsteps) without          */
/* reseeding: the samples are independent and run on `nthreads` threads.    */
static int orc_run_segment(const orc_problem *pb, const orc_coeffs *cf, const double *phi0, long step0,
                           int nsteps, int s0, int ns, int nthreads, const double *ghost,
                           const double *state_in, double *state_out, double *sum, double *sumsq)
{
    size_t sz = (size_t)cf->E * cf->n;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > ns && ns > 0) nthreads = ns;
    orc_job *jobs = (orc_job *)calloc(nthreads, sizeof(orc_job));
    pthread_t *th = (pthread_t *)calloc(nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].pb = pb;
        jobs[t].cf = cf;
        jobs[t].step0 = step0;
        jobs[t].nsteps = nsteps;
        jobs[t].s0 = s0;
        jobs[t].s_begin = s0 + (int)((long)ns * t / nthreads);
        jobs[t].s_end = s0 + (int)((long)ns * (t + 1) / nthreads);
        jobs[t].state_in = state_in;
        jobs[t].phi0 = phi0;
        jobs[t].state_out = state_out;
        jobs[t].ghost = ghost;
        if (sum) {
            jobs[t].sum = (double *)calloc(sz, sizeof(double));
            jobs[t].sumsq = (double *)calloc(sz, sizeof(double));
        }
    }
    if (nthreads == 1)
        orc_worker(&jobs[0]);
    else {
        for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_worker, &jobs[t]);
        for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    int rc = 0;
    if (sum) {
        for (size_t i = 0; i < sz; ++i) {
            sum[i] = 0.0;
            sumsq[i] = 0.0;
        }
        for (int t = 0; t < nthreads; ++t)
            for (size_t i = 0; i < sz; ++i) {
                sum[i] += jobs[t].sum[i];
                sumsq[i] += jobs[t].sumsq[i];
            }
    }
    for (int t = 0; t < nthreads; ++t) {
        if (jobs[t].rc != 0) rc = -1;
        free(jobs[t].sum);
        free(jobs[t].sumsq);
    }
    free(jobs);
    free(th);
    return rc;
}

/* Runs samples [s0, s0+ns).  state_in ([ns][E][n]) or NULL for phi0;       */
/* state_out ([ns][E][n]) may be NULL; sum and sumsq ([E][n]) may be NULL and */
/* receive sum_s Q and sum_s Q^2, threads' partials added in thread order,  */
/* each thread in ascending sample order.  ghost: [nsteps][width] boundary  */
/* values after each step (Dirichlet; NULL when periodic): 1D x = lo, hi;    */
/* 2D left, right, bottom, top faces (see orc_step_2d).                      */
/* With reseed_every > 0 the run stops after each step n with               */
/* (n + 1) % reseed_every == 0 and sets every sample to the mean of the ns  */
/* samples (summed in ascending sample order), Eq. re-seed.  Returns 0/-1.  */
int orc_run(const orc_problem *pb, long step0, int nsteps, int s0, int ns, int nthreads,
            const double *ghost, const double *state_in, double *state_out, double *sum, double *sumsq)
{
    if (pb->dim < 1 || pb->dim > 2 || pb->N < 2 || ns < 0 || nsteps < 0 || pb->dt < 0.0) return -1;
    if (pb->dim == 2 && isinf(pb->omega)) return -1; /* hard constraints: 1D only */
    if (!pb->periodic && !ghost) return -1; /* Dirichlet: boundary values needed */
    if (pb->reseed_every < 0) return -1;
    orc_coeffs cf;
    if (orc_build_coeffs(pb, &cf) != 0) {
        orc_coeffs_free(&cf);
        return -1;
    }
    size_t sz = (size_t)cf.E * cf.n;
    double *phi0 = (double *)malloc(sizeof(double) * sz);
    orc_init_state(pb, phi0);
    int rc = 0;
    if (pb->reseed_every == 0 || nsteps == 0) {
        rc = orc_run_segment(pb, &cf, phi0, step0, nsteps, s0, ns, nthreads, pb->periodic ? NULL : ghost,
                             state_in, state_out, sum, sumsq);
    } else {
        const long R = pb->reseed_every;
        double *cur = (double *)malloc(sizeof(double) * sz * (size_t)(ns > 0 ? ns : 1));
        double *nxt = (double *)malloc(sizeof(double) * sz * (size_t)(ns > 0 ? ns : 1));
        for (int s = 0; s < ns; ++s) memcpy(cur + (size_t)s * sz, state_in ? state_in + (size_t)s * sz : phi0, sizeof(double) * sz);
        long t = 0;
        while (t < nsteps && rc == 0) {
            long seg = R - (step0 + t) % R; /* steps up to and including the next reseed step */
            if (seg > nsteps - t) seg = nsteps - t;
            rc = orc_run_segment(pb, &cf, phi0, step0 + t, (int)seg, s0, ns, nthreads,
                                 pb->periodic ? NULL : ghost + (size_t)orc_ghost_width(&cf) * t, cur, nxt, NULL, NULL);
            double *tmp = cur;
            cur = nxt;
            nxt = tmp;
            t += seg;
            if ((step0 + t) % R == 0 && ns > 0) { /* Eq. re-seed */
                for (size_t i = 0; i < sz; ++i) {
                    double m = 0.0;
                    for (int s = 0; s < ns; ++s) m += cur[(size_t)s * sz + i];
                    nxt[i] = m / ns;
                }
                for (int s = 0; s < ns; ++s) memcpy(cur + (size_t)s * sz, nxt, sizeof(double) * sz);
            }
        }
        if (state_out) memcpy(state_out, cur, sizeof(double) * sz * (size_t)ns);
        if (sum)
            for (size_t i = 0; i < sz; ++i) {
                sum[i] = 0.0;
                sumsq[i] = 0.0;
                for (int s = 0; s < ns; ++s) {
                    double q = cur[(size_t)s * sz + i];
                    sum[i] += q;
                    sumsq[i] += q * q;
                }
            }
        free(cur);
        free(nxt);
    }
    free(phi0);
    orc_coeffs_free(&cf);
    return rc;
}

/* Largest dt with |u|max dt + sqrt(2 Dmax dt) <= dx_min in every direction */
/* (Eq. 1d_timestep; Eq. 1d_difftimestep when u = 0), dx_min being the       */
/* smallest node-to-node gap times h, maxima over the nodes.                 */
static double orc_dt_bound(const orc_problem *pb, int edge)
{
    orc_problem q = *pb;
    q.dt = 1.0;
    orc_coeffs cf;
    if (orc_build_coeffs(&q, &cf) != 0) {
        orc_coeffs_free(&cf);
        return -1.0;
    }
    double gap = 1.0;
    for (int i = 0; i + 1 < cf.N; ++i)
        if (cf.xi[i + 1] - cf.xi[i] < gap) gap = cf.xi[i + 1] - cf.xi[i];
    if (edge) gap = cf.xi[0]; /* distance of the first node to the element face */
    double best = INFINITY;
    for (int d = 0; d < cf.dim; ++d) {
        double umax = 0.0, bmax = 0.0;
        const double *a = d == 0 ? cf.ax : cf.ay;
        for (int i = 0; i < cf.E * cf.n; ++i) {
            if (fabs(a[i]) > umax) umax = fabs(a[i]);
            if (cf.b[i] > bmax) bmax = cf.b[i];
        }
        double dx = gap * (d == 0 ? cf.hx : cf.hy);
        double dt;
        /* |u| s^2 + sqrt(2D) s - dx = 0 with s = sqrt(dt) */
        if (umax == 0.0)
            dt = bmax > 0.0 ? dx * dx / (bmax * bmax) : INFINITY;
        else {
            double s = (-bmax + sqrt(bmax * bmax + 4.0 * umax * dx)) / (2.0 * umax);
            dt = s * s;
        }
        if (dt < best) best = dt;
    }
    orc_coeffs_free(&cf);
    return best;
}

double orc_dt_max(const orc_problem *pb) { return orc_dt_bound(pb, 0); }

/* The same bound with dx_min = the first node's distance to the element     */
/* face: a particle moved by u dt plus one standard deviation of the        */
/* diffusion stays inside its element (the paper restricts dt so that      */
/* particles do not leave the subdomain, Section 5.2).                       */
double orc_dt_edge(const orc_problem *pb) { return orc_dt_bound(pb, 1); }
