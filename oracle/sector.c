/*
 * FP64 photon-number-sector state vector: ORACLE, test infrastructure only.
 * Only the tests, the smoke check and the timed CPU baseline of the benchmark
 * may load this file; the library's compute path never does.
 *
 * What it computes (Section 2.2, for the bosonic qudit networks of Section 4
 * and Algorithm 1): the amplitude <p|U|psi0> of a product initial state psi0
 * of n modes with Fock cutoff d under a sequence of gates that conserve the
 * total photon number.  A two-mode gate on (q1, q2) is a d^2 x d^2 matrix
 * U[(o1 o2)][(i1 i2)] that must vanish unless o1 + o2 = i1 + i2 (a
 * beamsplitter); a one-mode gate must be diagonal.  Such gates never mix
 * states of different total photon number N, so the amplitude of a pattern p
 * with total N only needs the sector-N part of psi0, evolved inside the
 * sector.  The sector holds the compositions of N into n parts in [0, d), far
 * fewer than d^n for small or large N, which is what lets a 16-mode, d = 4
 * network (4^16 amplitudes, 64 GiB in FP64) be checked on a host.
 *
 * Sector states are numbered in lexicographic order, mode 0 most significant
 * (the same digit order as the dense state vector of sv.c), through the
 * counting table cnt[k][s] = number of ways modes k..n-1 sum to s.  A gate
 * is applied block by block: the states that agree outside (q1, q2) and have
 * the same n_q1 + n_q2 form one block, handled by the member with the
 * smallest n_q1, which gathers the block, multiplies it by the gate's
 * sub-matrix and scatters it into the output vector, so every state is
 * written exactly once.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define SEC_MAXN 64
#define SEC_MAXD 16

typedef struct {
    int n, d, N;
    int64_t *cnt;   /* (n + 1) x (n (d - 1) + 1) */
    int smax;
} Sector;

static int64_t cnt_at(const Sector *S, int k, int s)
{
    if (s < 0 || s > S->smax) return 0;
    return S->cnt[(int64_t)k * (S->smax + 1) + s];
}

static int sector_init(Sector *S, int n, int d, int N)
{
    S->n = n;
    S->d = d;
    S->N = N;
    S->smax = n * (d - 1);
    S->cnt = (int64_t *)calloc((size_t)(n + 1) * (S->smax + 1), sizeof(int64_t));
    if (!S->cnt) return 1;
    S->cnt[(int64_t)n * (S->smax + 1) + 0] = 1;
    for (int k = n - 1; k >= 0; --k)
        for (int s = 0; s <= S->smax; ++s) {
            int64_t c = 0;
            for (int v = 0; v < d && v <= s; ++v) c += cnt_at(S, k + 1, s - v);
            S->cnt[(int64_t)k * (S->smax + 1) + s] = c;
        }
    return 0;
}

static int64_t sector_dim(const Sector *S) { return cnt_at(S, 0, S->N); }

/* rank of a composition x (sum N) among the sector's states */
static int64_t sector_rank(const Sector *S, const int *x)
{
    int64_t r = 0;
    int p = 0;
    for (int k = 0; k < S->n; ++k) {
        for (int v = 0; v < x[k]; ++v) r += cnt_at(S, k + 1, S->N - p - v);
        p += x[k];
    }
    return r;
}

static void sector_unrank(const Sector *S, int64_t r, int *x)
{
    int p = 0;
    for (int k = 0; k < S->n; ++k) {
        int v = 0;
        for (; v < S->d; ++v) {
            int64_t c = cnt_at(S, k + 1, S->N - p - v);
            if (r < c) break;
            r -= c;
        }
        x[k] = v;
        p += v;
    }
}

/* lexicographic successor with the same sum; returns 0 after the last state */
static int sector_next(const Sector *S, int *x)
{
    int rest = 0;
    for (int i = S->n - 1; i >= 0; --i) {
        if (x[i] < S->d - 1 && rest >= 1) {
            x[i] += 1;
            rest -= 1;
            for (int j = S->n - 1; j > i; --j) {
                x[j] = rest < S->d - 1 ? rest : S->d - 1;
                rest -= x[j];
            }
            return 1;
        }
        rest += x[i];
    }
    return 0;
}

#define SEC_CHUNK 4096

/* Check that a gate conserves the total photon number (exact zeros). */
static int conserves(int d, int k, const cplx *U)
{
    if (k == 1) {
        for (int o = 0; o < d; ++o)
            for (int i = 0; i < d; ++i)
                if (o != i && U[o * d + i] != 0) return 0;
        return 1;
    }
    for (int o = 0; o < d * d; ++o)
        for (int i = 0; i < d * d; ++i)
            if ((o / d + o % d) != (i / d + i % d) && U[(int64_t)o * d * d + i] != 0) return 0;
    return 1;
}

static void apply_gate(const Sector *S, const cplx *psi, cplx *phi, int64_t dim, int k, const int *q,
                       const cplx *U)
{
    const int d = S->d;
    const int64_t n_chunks = (dim + SEC_CHUNK - 1) / SEC_CHUNK;
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < n_chunks; ++c) {
        int x[SEC_MAXN];
        int64_t r0 = c * SEC_CHUNK, r1 = r0 + SEC_CHUNK < dim ? r0 + SEC_CHUNK : dim;
        sector_unrank(S, r0, x);
        for (int64_t r = r0; r < r1; ++r) {
            if (k == 1) {
                phi[r] = U[x[q[0]] * d + x[q[0]]] * psi[r];
            } else {
                const int a = q[0], b = q[1];
                const int s = x[a] + x[b];
                const int lo = s - (d - 1) > 0 ? s - (d - 1) : 0, hi = s < d - 1 ? s : d - 1;
                if (x[a] == lo) {   /* block leader */
                    int64_t idx[SEC_MAXD];
                    cplx v[SEC_MAXD];
                    int y[SEC_MAXN];
                    memcpy(y, x, sizeof(int) * S->n);
                    for (int m = lo; m <= hi; ++m) {
                        y[a] = m;
                        y[b] = s - m;
                        idx[m - lo] = (m == x[a]) ? r : sector_rank(S, y);
                        v[m - lo] = psi[idx[m - lo]];
                    }
                    for (int o = lo; o <= hi; ++o) {
                        cplx w = 0;
                        const int64_t row = (int64_t)(o * d + (s - o)) * d * d;
                        for (int i = lo; i <= hi; ++i) w += U[row + i * d + (s - i)] * v[i - lo];
                        phi[idx[o - lo]] = w;
                    }
                }
            }
            if (r + 1 < r1) sector_next(S, x);
        }
    }
}

/*
 * amps_out[j] = <patterns[j] | U_{G-1} ... U_0 | psi0>, complex128.
 * init: n vectors of d complex values (psi0 = their tensor product); gates as
 * in sv.c (gate_k[g] qudits at qudits[2g..], matrix at mats + 2 * mat_off[g]
 * doubles).  Sectors larger than max_dim states are refused.
 * Returns 0; 1 if a gate does not conserve the photon number; 2 on allocation
 * failure; 3 if a needed sector exceeds max_dim; 4 on bad sizes.
 */
int oracle_sector_amplitudes(int n, int d, const double *init, int n_gates, const int *gate_k,
                             const int *qudits, const double *mats, const int64_t *mat_off, int n_pat,
                             const int *patterns, double *amps_out, int64_t max_dim)
{
    if (n < 1 || n > SEC_MAXN || d < 1 || d > SEC_MAXD) return 4;
    const cplx *iv = (const cplx *)init;
    cplx *amps = (cplx *)amps_out;
    for (int g = 0; g < n_gates; ++g)
        if (!conserves(d, gate_k[g], (const cplx *)mats + mat_off[g])) return 1;
    int *done = (int *)calloc((size_t)n_pat, sizeof(int));
    if (!done) return 2;
    int rc = 0;
    for (int j0 = 0; j0 < n_pat && rc == 0; ++j0) {
        if (done[j0]) continue;
        int N = 0;
        for (int k = 0; k < n; ++k) N += patterns[(int64_t)j0 * n + k];
        Sector S;
        if (sector_init(&S, n, d, N)) { rc = 2; break; }
        const int64_t dim = sector_dim(&S);
        if (dim > max_dim) { free(S.cnt); rc = 3; break; }
        cplx *psi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
        cplx *phi = (cplx *)malloc(sizeof(cplx) * (size_t)dim);
        if (!psi || !phi) { free(psi); free(phi); free(S.cnt); rc = 2; break; }
        /* sector-N part of the product state */
        const int64_t n_chunks = (dim + SEC_CHUNK - 1) / SEC_CHUNK;
        #pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < n_chunks; ++c) {
            int x[SEC_MAXN];
            int64_t r0 = c * SEC_CHUNK, r1 = r0 + SEC_CHUNK < dim ? r0 + SEC_CHUNK : dim;
            sector_unrank(&S, r0, x);
            for (int64_t r = r0; r < r1; ++r) {
                cplx a = 1.0;
                for (int k = 0; k < n; ++k) a *= iv[k * d + x[k]];
                psi[r] = a;
                if (r + 1 < r1) sector_next(&S, x);
            }
        }
        for (int g = 0; g < n_gates; ++g) {
            apply_gate(&S, psi, phi, dim, gate_k[g], qudits + 2 * g, (const cplx *)mats + mat_off[g]);
            cplx *t = psi;
            psi = phi;
            phi = t;
        }
        for (int j = j0; j < n_pat; ++j) {
            int Nj = 0;
            for (int k = 0; k < n; ++k) Nj += patterns[(int64_t)j * n + k];
            if (Nj != N) continue;
            amps[j] = psi[sector_rank(&S, patterns + (int64_t)j * n)];
            done[j] = 1;
        }
        free(psi);
        free(phi);
        free(S.cnt);
    }
    free(done);
    return rc;
}

/* Number of states in the total-photon sector N (the oracle's cost driver). */
int64_t oracle_sector_dim(int n, int d, int N)
{
    Sector S;
    if (n < 1 || n > SEC_MAXN || d < 1 || sector_init(&S, n, d, N)) return -1;
    const int64_t dim = sector_dim(&S);
    free(S.cnt);
    return dim;
}
