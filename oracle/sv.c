/*
 * FP64 dense state-vector simulator: ORACLE, test infrastructure only.
 * Only the tests, the smoke check and the timed CPU baseline of the benchmark
 * may load this file; the library's compute path never does.
 *
 * What it computes (Section 2.2): the amplitude <x|U|psi0> of a circuit U
 * acting on a product state psi0 of n qudits of dimension d.  The state is a
 * d^n vector with qudit 0 the most significant digit; gates are applied one at
 * a time in circuit order, in place.  A 1-qudit gate is a d x d matrix
 * U[out][in]; a 2-qudit gate on (q1, q2) is a d^2 x d^2 matrix
 * U[(o1 o2)][(i1 i2)], q1 the more significant digit of the pair.
 *
 * oracle_sv_env computes, for every gate k, the environment
 *     env_k[o][i] = d/dU_k[o][i] ( lam^T . U_L ... U_1 psi0 )
 * where lam is a given bra vector (a weighted sum of basis bras).  It runs the
 * textbook adjoint sweep: lam_{k-1} = U_k^T lam_k backwards, with the forward
 * states psi_{k-1} rebuilt from checkpoints (no inverse gates are applied, so
 * non-unitary gates are handled exactly).
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static int64_t ipow(int64_t b, int e) { int64_t r = 1; while (e-- > 0) r *= b; return r; }

void oracle_sv_product(int n, int d, const double *init, double *psi_out)
{
    /* psi[x] = prod_q init_q[x_q]; init holds n vectors of d complex values */
    const cplx *v = (const cplx *)init;
    cplx *psi = (cplx *)psi_out;
    int64_t N = ipow(d, n);
    #pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        cplx a = 1.0;
        int64_t r = x;
        for (int q = n - 1; q >= 0; --q) { a *= v[q * d + (r % d)]; r /= d; }
        psi[x] = a;
    }
}

/* Apply one gate (k = 1 or 2 qudits) in place.  transpose != 0 applies U^T. */
void oracle_sv_apply(int n, int d, double *psi_io, int k, const int *qudits,
                     const double *mat, int transpose)
{
    cplx *psi = (cplx *)psi_io;
    const cplx *U = (const cplx *)mat;
    int64_t N = ipow(d, n);
    int m = (k == 1) ? d : d * d;
    if (k == 1) {
        int64_t s = ipow(d, n - 1 - qudits[0]);
        int64_t nblk = N / (s * d);
        #pragma omp parallel for collapse(2) schedule(static)
        for (int64_t h = 0; h < nblk; ++h)
            for (int64_t l = 0; l < s; ++l) {
                cplx v[16], w[16];
                int64_t base = h * s * d + l;
                for (int j = 0; j < d; ++j) v[j] = psi[base + j * s];
                for (int i = 0; i < d; ++i) {
                    cplx acc = 0;
                    for (int j = 0; j < d; ++j)
                        acc += (transpose ? U[j * m + i] : U[i * m + j]) * v[j];
                    w[i] = acc;
                }
                for (int i = 0; i < d; ++i) psi[base + i * s] = w[i];
            }
    } else {
        int64_t s1 = ipow(d, n - 1 - qudits[0]);
        int64_t s2 = ipow(d, n - 1 - qudits[1]);
        int64_t sb = s1 > s2 ? s1 : s2, ss = s1 > s2 ? s2 : s1;
        int64_t nh = N / (sb * d), nm = sb / (ss * d);
        #pragma omp parallel for collapse(3) schedule(static)
        for (int64_t h = 0; h < nh; ++h)
            for (int64_t mm = 0; mm < nm; ++mm)
                for (int64_t l = 0; l < ss; ++l) {
                    cplx v[256], w[256];
                    int64_t base = h * sb * d + mm * ss * d + l;
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b)
                            v[a * d + b] = psi[base + a * s1 + b * s2];
                    for (int i = 0; i < m; ++i) {
                        cplx acc = 0;
                        for (int j = 0; j < m; ++j)
                            acc += (transpose ? U[j * m + i] : U[i * m + j]) * v[j];
                        w[i] = acc;
                    }
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b)
                            psi[base + a * s1 + b * s2] = w[a * d + b];
                }
    }
}

/* Gate list layout: gate g acts on gate_k[g] qudits gate_q[2g], gate_q[2g+1];
 * its matrix starts at complex offset mat_off[g] of mats. */
static void apply_range(int n, int d, cplx *psi, int g0, int g1, const int *gate_k,
                        const int *gate_q, const double *mats, const int64_t *mat_off)
{
    for (int g = g0; g < g1; ++g)
        oracle_sv_apply(n, d, (double *)psi, gate_k[g], gate_q + 2 * g,
                        mats + 2 * mat_off[g], 0);
}

void oracle_sv_run(int n, int d, const double *init, int n_gates, const int *gate_k,
                   const int *gate_q, const double *mats, const int64_t *mat_off,
                   double *psi_out)
{
    oracle_sv_product(n, d, init, psi_out);
    apply_range(n, d, (cplx *)psi_out, 0, n_gates, gate_k, gate_q, mats, mat_off);
}

/* env_k[o][i] = sum_y lam_k[y with digits(q)=o] psi_{k-1}[y with digits(q)=i] */
static void gate_env(int n, int d, const cplx *lam, const cplx *psi, int k,
                     const int *qudits, cplx *env)
{
    int64_t N = ipow(d, n);
    int m = (k == 1) ? d : d * d;
    for (int e = 0; e < m * m; ++e) env[e] = 0;
    if (k == 1) {
        int64_t s = ipow(d, n - 1 - qudits[0]);
        int64_t nblk = N / (s * d);
        for (int o = 0; o < d; ++o)
            for (int i = 0; i < d; ++i) {
                cplx acc = 0;
                #pragma omp parallel for collapse(2) reduction(+:acc) schedule(static)
                for (int64_t h = 0; h < nblk; ++h)
                    for (int64_t l = 0; l < s; ++l) {
                        int64_t base = h * s * d + l;
                        acc += lam[base + o * s] * psi[base + i * s];
                    }
                env[o * m + i] = acc;
            }
    } else {
        int64_t s1 = ipow(d, n - 1 - qudits[0]);
        int64_t s2 = ipow(d, n - 1 - qudits[1]);
        int64_t sb = s1 > s2 ? s1 : s2, ss = s1 > s2 ? s2 : s1;
        int64_t nh = N / (sb * d), nm = sb / (ss * d);
        for (int o = 0; o < m; ++o)
            for (int i = 0; i < m; ++i) {
                int64_t oo = (o / d) * s1 + (o % d) * s2, ii = (i / d) * s1 + (i % d) * s2;
                cplx acc = 0;
                #pragma omp parallel for collapse(3) reduction(+:acc) schedule(static)
                for (int64_t h = 0; h < nh; ++h)
                    for (int64_t mm = 0; mm < nm; ++mm)
                        for (int64_t l = 0; l < ss; ++l) {
                            int64_t base = h * sb * d + mm * ss * d + l;
                            acc += lam[base + oo] * psi[base + ii];
                        }
                env[o * m + i] = acc;
            }
    }
}

/* Returns 0 on success, -1 on allocation failure.  env_out holds, for gate g,
 * (d^k)^2 complex values at complex offset mat_off[g] (the same layout as mats). */
int oracle_sv_env(int n, int d, const double *init, int n_gates, const int *gate_k,
                  const int *gate_q, const double *mats, const int64_t *mat_off,
                  const double *lam_in, double *env_out)
{
    int64_t N = ipow(d, n);
    int S = 1;
    while ((int64_t)S * S < n_gates) ++S;             /* segment length ~ sqrt(#gates) */
    int n_seg = (n_gates + S - 1) / S;
    size_t bytes = (size_t)N * sizeof(cplx);
    cplx *ckpt = malloc(bytes * (size_t)(n_seg > 0 ? n_seg : 1));
    cplx *seg = malloc(bytes * (size_t)S);
    cplx *lam = malloc(bytes);
    if (!ckpt || !seg || !lam) { free(ckpt); free(seg); free(lam); return -1; }
    /* forward: checkpoint c holds the state before gate c*S */
    oracle_sv_product(n, d, init, (double *)ckpt);
    for (int c = 1; c < n_seg; ++c) {
        memcpy(ckpt + (size_t)c * N, ckpt + (size_t)(c - 1) * N, bytes);
        apply_range(n, d, ckpt + (size_t)c * N, (c - 1) * S, c * S, gate_k, gate_q, mats, mat_off);
    }
    memcpy(lam, lam_in, bytes);
    for (int c = n_seg - 1; c >= 0; --c) {
        int g0 = c * S, g1 = g0 + S < n_gates ? g0 + S : n_gates;
        memcpy(seg, ckpt + (size_t)c * N, bytes);
        for (int g = g0 + 1; g < g1; ++g) {           /* seg[j] = state before gate g0+j */
            memcpy(seg + (size_t)(g - g0) * N, seg + (size_t)(g - g0 - 1) * N, bytes);
            apply_range(n, d, seg + (size_t)(g - g0) * N, g - 1, g, gate_k, gate_q, mats, mat_off);
        }
        for (int g = g1 - 1; g >= g0; --g) {
            gate_env(n, d, lam, seg + (size_t)(g - g0) * N, gate_k[g], gate_q + 2 * g,
                     (cplx *)env_out + mat_off[g]);
            oracle_sv_apply(n, d, (double *)lam, gate_k[g], gate_q + 2 * g,
                            mats + 2 * mat_off[g], 1);
        }
    }
    free(ckpt); free(seg); free(lam);
    return 0;
}
