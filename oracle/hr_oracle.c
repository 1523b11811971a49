/*
 * hr_oracle.c -- plain FP64 CPU oracle for the Wilson-Dirac hot path of
 * HiRep v2 (arXiv 2503.06721).  TEST INFRASTRUCTURE ONLY: loaded by the test
 * suite, the smoke check and the benchmark's CPU-baseline leg; never by the
 * GPU library, which shares no code with it.
 *
 * Every routine writes out a definition from the paper as directly as
 * possible (loops over sites, directions, spins and colours with no blocking
 * or fusion).  OpenMP is used only to parallelise independent output sites so
 * the CPU baseline can be timed on all host cores; it does not change the
 * order of any floating-point sum.
 */
#include "hr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* largest representation dimension handled (SU(4) adjoint is 15) */
#define OR_MAXD 16

/* ------------------------------------------------------------------ */
/* small dense matrix helpers (row-major n x n)                         */
/* ------------------------------------------------------------------ */
static void mat_mul(int n, const orc *A, const orc *B, orc *C)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            orc s = 0;
            for (int k = 0; k < n; k++) s += A[i * n + k] * B[k * n + j];
            C[i * n + j] = s;
        }
}

static void mat_dag(int n, const orc *A, orc *B)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) B[i * n + j] = conj(A[j * n + i]);
}

static void mat_transpose(int n, const orc *A, orc *B)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) B[i * n + j] = A[j * n + i];
}

static orc mat_trace(int n, const orc *A)
{
    orc s = 0;
    for (int i = 0; i < n; i++) s += A[i * n + i];
    return s;
}

/* ------------------------------------------------------------------ */
/* Table 1: dimensions of the supported representations                 */
/* ------------------------------------------------------------------ */
int or_rep_dim(int N, int rep)
{
    switch (rep) {
    case OR_FUND: return N;
    case OR_ADJ:  return N * N - 1;
    case OR_SYM:  return N * (N + 1) / 2;
    case OR_ASYM: return N * (N - 1) / 2;
    case OR_ASYM_REAL: return N == 4 ? 6 : -1;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.2: gamma_mu = [[0, e_mu], [e_mu^dag, 0]],                      */
/* e_0 = -1, e_i = -i sigma_i; gamma5 = gamma0 gamma1 gamma2 gamma3      */
/* ------------------------------------------------------------------ */
static void pauli(int i, orc s[4])
{
    memset(s, 0, 4 * sizeof(orc));
    if (i == 1) { s[1] = 1; s[2] = 1; }
    if (i == 2) { s[1] = -I; s[2] = I; }
    if (i == 3) { s[0] = 1; s[3] = -1; }
}

void or_gamma(int mu, orc *g)
{
    if (mu == 4) {
        orc a[16], b[16], c[16], d[16], t1[16], t2[16];
        or_gamma(0, a); or_gamma(1, b); or_gamma(2, c); or_gamma(3, d);
        mat_mul(4, a, b, t1);
        mat_mul(4, t1, c, t2);
        mat_mul(4, t2, d, g);
        return;
    }
    orc e[4];
    if (mu == 0) {
        e[0] = -1; e[1] = 0; e[2] = 0; e[3] = -1;
    } else {
        orc s[4];
        pauli(mu, s);
        for (int k = 0; k < 4; k++) e[k] = -I * s[k];
    }
    memset(g, 0, 16 * sizeof(orc));
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            g[i * 4 + (j + 2)] = e[i * 2 + j];            /* upper-right e   */
            g[(i + 2) * 4 + j] = conj(e[j * 2 + i]);      /* lower-left e^dag */
        }
}

/* ------------------------------------------------------------------ */
/* generators of SU(N): generalised Gell-Mann matrices / 2               */
/* order: for each pair j<k, (E_jk+E_kj)/2 then -i(E_jk-E_kj)/2; then the */
/* diagonal ones diag(1,..,1,-l,0,..)/sqrt(2l(l+1)), l = 1..N-1          */
/* ------------------------------------------------------------------ */
void or_generators(int N, orc *T)
{
    int ng = N * N - 1, a = 0;
    memset(T, 0, (size_t)ng * N * N * sizeof(orc));
    for (int j = 0; j < N; j++)
        for (int k = j + 1; k < N; k++) {
            orc *S = T + (size_t)a * N * N;
            S[j * N + k] = 0.5; S[k * N + j] = 0.5;
            a++;
            orc *A = T + (size_t)a * N * N;
            A[j * N + k] = -0.5 * I; A[k * N + j] = 0.5 * I;
            a++;
        }
    for (int l = 1; l < N; l++) {
        orc *D = T + (size_t)a * N * N;
        double nrm = 1.0 / sqrt(2.0 * l * (l + 1));
        for (int i = 0; i < l; i++) D[i * N + i] = nrm;
        D[l * N + l] = -l * nrm;
        a++;
    }
}

int or_rep_basis(int N, int rep, orc *E)
{
    if (rep == OR_ADJ) {
        or_generators(N, E);
        return N * N - 1;
    }
    if (rep == OR_FUND) return 0;
    if (rep == OR_ASYM_REAL) {
        if (N != 4) return 0;
        /* pairs P with complement Q and the sign s of the permutation (P, Q) */
        static const int P[3][2] = {{0, 1}, {0, 2}, {0, 3}}, Q[3][2] = {{2, 3}, {1, 3}, {1, 2}};
        static const double sg[3] = {1.0, -1.0, 1.0};
        for (int k = 0; k < 3; k++)
            for (int im = 0; im < 2; im++) {
                orc *B = E + (size_t)(2 * k + im) * 16;
                memset(B, 0, 16 * sizeof(orc));
                orc c = im ? 0.5 * I : 0.5;          /* 1/sqrt2 of f times 1/sqrt2 of e */
                double q = im ? -sg[k] : sg[k];
                B[P[k][0] * 4 + P[k][1]] += c;
                B[P[k][1] * 4 + P[k][0]] -= c;
                B[Q[k][0] * 4 + Q[k][1]] += q * c;
                B[Q[k][1] * 4 + Q[k][0]] -= q * c;
            }
        return 6;
    }
    int n = 0;
    double r2 = 1.0 / sqrt(2.0);
    for (int i = 0; i < N; i++)
        for (int j = i; j < N; j++) {
            if (rep == OR_ASYM && i == j) continue;
            orc *B = E + (size_t)n * N * N;
            memset(B, 0, (size_t)N * N * sizeof(orc));
            if (i == j) {
                B[i * N + i] = 1.0;
            } else if (rep == OR_SYM) {
                B[i * N + j] = r2; B[j * N + i] = r2;
            } else {
                B[i * N + j] = r2; B[j * N + i] = -r2;
            }
            n++;
        }
    return n;
}

/* R(U):  FUND  R = U
 *        ADJ   R_ab = 2 Tr(T_a U T_b U^dag)
 *        SYM/ASYM  R_nm = Tr(e_n^dag U e_m U^T)                         */
int or_represent_link(int N, int rep, const orc *U, orc *R)
{
    int D = or_rep_dim(N, rep);
    if (rep == OR_FUND) {
        memcpy(R, U, (size_t)N * N * sizeof(orc));
        return D;
    }
    int nn = N * N;
    orc *E = malloc((size_t)D * nn * sizeof(orc));
    orc *Ud = malloc((size_t)nn * sizeof(orc));
    orc *Ut = malloc((size_t)nn * sizeof(orc));
    orc *t1 = malloc((size_t)nn * sizeof(orc));
    orc *t2 = malloc((size_t)nn * sizeof(orc));
    orc *t3 = malloc((size_t)nn * sizeof(orc));
    orc *Ed = malloc((size_t)nn * sizeof(orc));
    or_rep_basis(N, rep, E);
    mat_dag(N, U, Ud);
    mat_transpose(N, U, Ut);
    for (int m = 0; m < D; m++) {
        /* t2 = U e_m U^dag (ADJ) or U e_m U^T (SYM/ASYM) */
        mat_mul(N, U, E + (size_t)m * nn, t1);
        mat_mul(N, t1, rep == OR_ADJ ? Ud : Ut, t2);
        for (int n = 0; n < D; n++) {
            if (rep == OR_ADJ) {
                mat_mul(N, E + (size_t)n * nn, t2, t3);
                R[n * D + m] = 2.0 * mat_trace(N, t3);
            } else {
                mat_dag(N, E + (size_t)n * nn, Ed);
                mat_mul(N, Ed, t2, t3);
                R[n * D + m] = mat_trace(N, t3);
            }
        }
    }
    free(E); free(Ud); free(Ut); free(t1); free(t2); free(t3); free(Ed);
    return D;
}

/* T_R^a = -i d/de R(exp(i e T^a)) at e = 0:
 *   FUND  T^a
 *   ADJ   (T_R^a)_bc = 2 Tr(T_b [T_a, T_c])
 *   SYM/ASYM  (T_R^a)_nm = Tr(e_n^dag (T_a e_m + e_m T_a^T))            */
void or_rep_generators(int N, int rep, orc *TR)
{
    int ng = N * N - 1, nn = N * N, D = or_rep_dim(N, rep);
    orc *T = malloc((size_t)ng * nn * sizeof(orc));
    or_generators(N, T);
    if (rep == OR_FUND) {
        memcpy(TR, T, (size_t)ng * nn * sizeof(orc));
        free(T);
        return;
    }
    orc *E = malloc((size_t)D * nn * sizeof(orc));
    orc *t1 = malloc((size_t)nn * sizeof(orc));
    orc *t2 = malloc((size_t)nn * sizeof(orc));
    orc *t3 = malloc((size_t)nn * sizeof(orc));
    orc *Ta_t = malloc((size_t)nn * sizeof(orc));
    orc *Ed = malloc((size_t)nn * sizeof(orc));
    or_rep_basis(N, rep, E);
    for (int a = 0; a < ng; a++) {
        const orc *Ta = T + (size_t)a * nn;
        mat_transpose(N, Ta, Ta_t);
        for (int m = 0; m < D; m++) {
            const orc *Em = E + (size_t)m * nn;
            /* t3 = [T_a, E_m] (ADJ) or T_a E_m + E_m T_a^T (SYM/ASYM) */
            mat_mul(N, Ta, Em, t1);
            mat_mul(N, Em, rep == OR_ADJ ? Ta : Ta_t, t2);
            for (int k = 0; k < nn; k++)
                t3[k] = rep == OR_ADJ ? t1[k] - t2[k] : t1[k] + t2[k];
            for (int n = 0; n < D; n++) {
                const orc *En = E + (size_t)n * nn;
                if (rep == OR_ADJ) {
                    mat_mul(N, En, t3, t1);
                    TR[((size_t)a * D + n) * D + m] = 2.0 * mat_trace(N, t1);
                } else {
                    mat_dag(N, En, Ed);
                    mat_mul(N, Ed, t3, t1);
                    TR[((size_t)a * D + n) * D + m] = mat_trace(N, t1);
                }
            }
        }
    }
    free(T); free(E); free(t1); free(t2); free(t3); free(Ta_t); free(Ed);
}

/* ------------------------------------------------------------------ */
/* lattice geometry (Sec. 2.1)                                           */
/* ------------------------------------------------------------------ */
long or_volume(const or_lat *L)
{
    return (long)L->dims[0] * L->dims[1] * L->dims[2] * L->dims[3];
}

void or_coords(const or_lat *L, long lex, int c[4])
{
    for (int mu = 3; mu >= 0; mu--) {
        c[mu] = (int)(lex % L->dims[mu]);
        lex /= L->dims[mu];
    }
}

long or_lex(const or_lat *L, const int c[4])
{
    long lex = 0;
    for (int mu = 0; mu < 4; mu++) lex = lex * L->dims[mu] + c[mu];
    return lex;
}

long or_neighbour(const or_lat *L, long lex, int mu, int dir)
{
    int c[4];
    or_coords(L, lex, c);
    c[mu] = (c[mu] + dir + L->dims[mu]) % L->dims[mu];
    return or_lex(L, c);
}

int or_parity(const or_lat *L, long lex)
{
    int c[4];
    or_coords(L, lex, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

void or_represent_field(const or_lat *L, const orc *UF, orc *UR)
{
    long V = or_volume(L);
    int N = L->N, D = or_rep_dim(L->N, L->rep);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        int c[4];
        or_coords(L, x, c);
        for (int mu = 0; mu < 4; mu++) {
            orc *R = UR + ((size_t)x * 4 + mu) * D * D;
            or_represent_link(N, L->rep, UF + ((size_t)x * 4 + mu) * N * N, R);
            if (L->bc[mu] == -1 && c[mu] == L->dims[mu] - 1)
                for (int k = 0; k < D * D; k++) R[k] = -R[k];
        }
    }
}

/* ------------------------------------------------------------------ */
/* Wilson-Dirac operator, Eq. (D_m^R):                                   */
/* D_m psi(x) = (4+m) psi(x) - 1/2 sum_mu [ (1-g_mu) U(x,mu) psi(x+mu)   */
/*                               + (1+g_mu) U(x-mu,mu)^dag psi(x-mu) ]   */
/* ------------------------------------------------------------------ */

/* acc[s][r] += -1/2 * sum_mu [...] at site x; sg = +1 (D) or -1 (D^dag) */
static void hop_site(const or_lat *L, const orc *UR, const orc *in, long x,
                     double sg, orc *acc, const orc gam[4][16])
{
    int D = or_rep_dim(L->N, L->rep);
    orc chi[4 * OR_MAXD];
    for (int mu = 0; mu < 4; mu++) {
        for (int dir = +1; dir >= -1; dir -= 2) {
            long y = or_neighbour(L, x, mu, dir);
            /* forward: U(x,mu) psi(x+mu); backward: U(x-mu,mu)^dag psi(x-mu) */
            const orc *U = UR + ((size_t)(dir > 0 ? x : y) * 4 + mu) * D * D;
            const orc *psi = in + (size_t)y * 4 * D;
            for (int s = 0; s < 4; s++)
                for (int r = 0; r < D; r++) {
                    orc v = 0;
                    for (int cc = 0; cc < D; cc++)
                        v += (dir > 0 ? U[r * D + cc] : conj(U[cc * D + r])) *
                             psi[s * D + cc];
                    chi[s * D + r] = v;
                }
            /* projector (1 - dir*sg*gamma_mu) */
            double pm = -(double)dir * sg;
            for (int s = 0; s < 4; s++)
                for (int r = 0; r < D; r++) {
                    orc v = chi[s * D + r];
                    for (int t = 0; t < 4; t++)
                        v += pm * gam[mu][s * 4 + t] * chi[t * D + r];
                    acc[s * D + r] += -0.5 * v;
                }
        }
    }
}

static void load_gammas(orc gam[4][16])
{
    for (int mu = 0; mu < 4; mu++) or_gamma(mu, gam[mu]);
}

void or_dirac_full(const or_lat *L, const orc *UR, const orc *in, orc *out,
                   int dagger)
{
    long V = or_volume(L);
    int D = or_rep_dim(L->N, L->rep);
    orc gam[4][16];
    load_gammas(gam);
    double sg = dagger ? -1.0 : 1.0;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        orc acc[4 * OR_MAXD];
        for (int k = 0; k < 4 * D; k++)
            acc[k] = (4.0 + L->m0) * in[(size_t)x * 4 * D + k];
        hop_site(L, UR, in, x, sg, acc, gam);
        for (int k = 0; k < 4 * D; k++) out[(size_t)x * 4 * D + k] = acc[k];
    }
}

void or_split_parity(const or_lat *L, const orc *full, orc *even, orc *odd)
{
    long V = or_volume(L);
    int D = or_rep_dim(L->N, L->rep);
    for (long x = 0; x < V; x++) {
        orc *dst = or_parity(L, x) == 0 ? even : odd;
        if (!dst) continue;
        memcpy(dst + (size_t)(x / 2) * 4 * D, full + (size_t)x * 4 * D,
               4 * D * sizeof(orc));
    }
}

void or_merge_parity(const or_lat *L, const orc *even, const orc *odd,
                     orc *full)
{
    long V = or_volume(L);
    int D = or_rep_dim(L->N, L->rep);
    for (long x = 0; x < V; x++) {
        const orc *src = or_parity(L, x) == 0 ? even : odd;
        if (src)
            memcpy(full + (size_t)x * 4 * D, src + (size_t)(x / 2) * 4 * D,
                   4 * D * sizeof(orc));
        else
            memset(full + (size_t)x * 4 * D, 0, 4 * D * sizeof(orc));
    }
}

void or_hop_parity(const or_lat *L, const orc *UR, int out_parity,
                   const orc *in_half, orc *out_half, int dagger)
{
    long V = or_volume(L);
    int D = or_rep_dim(L->N, L->rep);
    orc *full = malloc((size_t)V * 4 * D * sizeof(orc));
    if (out_parity == 0)
        or_merge_parity(L, NULL, in_half, full);
    else
        or_merge_parity(L, in_half, NULL, full);
    orc gam[4][16];
    load_gammas(gam);
    double sg = dagger ? -1.0 : 1.0;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        if (or_parity(L, x) != out_parity) continue;
        orc acc[4 * OR_MAXD];
        for (int k = 0; k < 4 * D; k++) acc[k] = 0;
        hop_site(L, UR, full, x, sg, acc, gam);
        memcpy(out_half + (size_t)(x / 2) * 4 * D, acc, 4 * D * sizeof(orc));
    }
    free(full);
}

void or_dhat(const or_lat *L, const orc *UR, const orc *in_e, orc *out_e,
             int dagger)
{
    long Vh = or_volume(L) / 2;
    int D = or_rep_dim(L->N, L->rep);
    size_t n = (size_t)Vh * 4 * D;
    orc *tmp_o = malloc(n * sizeof(orc));
    orc *tmp_e = malloc(n * sizeof(orc));
    or_hop_parity(L, UR, 1, in_e, tmp_o, dagger);   /* D_oe in_e        */
    or_hop_parity(L, UR, 0, tmp_o, tmp_e, dagger);  /* D_eo D_oe in_e   */
    double m4 = 4.0 + L->m0;
    for (size_t k = 0; k < n; k++) out_e[k] = m4 * m4 * in_e[k] - tmp_e[k];
    free(tmp_o);
    free(tmp_e);
}

void or_hop_sites(const or_lat *L, const orc *UF, int out_parity,
                  const orc *in_half, const long *sites, long nsites,
                  orc *out, int dagger)
{
    int N = L->N, D = or_rep_dim(L->N, L->rep);
    long V = or_volume(L);
    orc gam[4][16];
    load_gammas(gam);
    double sg = dagger ? -1.0 : 1.0;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < nsites; k++) {
        /* the site of parity out_parity with half index sites[k] */
        long x = -1;
        for (long cand = 2 * sites[k]; cand <= 2 * sites[k] + 1 && cand < V; cand++)
            if (or_parity(L, cand) == out_parity) x = cand;
        orc acc[4 * OR_MAXD], R[OR_MAXD * OR_MAXD], chi[4 * OR_MAXD];
        for (int q = 0; q < 4 * D; q++) acc[q] = 0;
        int c[4];
        or_coords(L, x, c);
        for (int mu = 0; mu < 4; mu++)
            for (int dir = +1; dir >= -1; dir -= 2) {
                long y = or_neighbour(L, x, mu, dir);
                long owner = dir > 0 ? x : y;   /* the link U(owner, mu) */
                or_represent_link(N, L->rep, UF + ((size_t)owner * 4 + mu) * N * N, R);
                int cown = dir > 0 ? c[mu] : (c[mu] - 1 + L->dims[mu]) % L->dims[mu];
                double sign = (L->bc[mu] == -1 && cown == L->dims[mu] - 1) ? -1.0 : 1.0;
                const orc *psi = in_half + (size_t)(y / 2) * 4 * D;
                for (int s = 0; s < 4; s++)
                    for (int r = 0; r < D; r++) {
                        orc v = 0;
                        for (int cc = 0; cc < D; cc++)
                            v += (dir > 0 ? R[r * D + cc] : conj(R[cc * D + r])) * psi[s * D + cc];
                        chi[s * D + r] = sign * v;
                    }
                double pm = -(double)dir * sg;
                for (int s = 0; s < 4; s++)
                    for (int r = 0; r < D; r++) {
                        orc v = chi[s * D + r];
                        for (int t = 0; t < 4; t++) v += pm * gam[mu][s * 4 + t] * chi[t * D + r];
                        acc[s * D + r] += -0.5 * v;
                    }
            }
        for (int q = 0; q < 4 * D; q++) out[(size_t)k * 4 * D + q] = acc[q];
    }
}

void or_hop_local_rep(const or_lat *L, const int c[4], const orc *Rlinks,
                      const orc *psi, orc *out, int dagger)
{
    int D = or_rep_dim(L->N, L->rep);
    orc gam[4][16];
    load_gammas(gam);
    double sg = dagger ? -1.0 : 1.0;
    orc chi[4 * OR_MAXD];
    for (int q = 0; q < 4 * D; q++) out[q] = 0;
    for (int k = 0; k < 8; k++) {
        int mu = k & 3, dir = k < 4 ? +1 : -1;
        const orc *R = Rlinks + (size_t)k * D * D;
        int cown = dir > 0 ? c[mu] : (c[mu] - 1 + L->dims[mu]) % L->dims[mu];
        double sign = (L->bc[mu] == -1 && cown == L->dims[mu] - 1) ? -1.0 : 1.0;
        const orc *p = psi + (size_t)k * 4 * D;
        for (int s = 0; s < 4; s++)
            for (int r = 0; r < D; r++) {
                orc v = 0;
                for (int cc = 0; cc < D; cc++)
                    v += (dir > 0 ? R[r * D + cc] : conj(R[cc * D + r])) * p[s * D + cc];
                chi[s * D + r] = sign * v;
            }
        double pm = -(double)dir * sg;
        for (int s = 0; s < 4; s++)
            for (int r = 0; r < D; r++) {
                orc v = chi[s * D + r];
                for (int t = 0; t < 4; t++) v += pm * gam[mu][s * 4 + t] * chi[t * D + r];
                out[s * D + r] += -0.5 * v;
            }
    }
}

void or_hop_local(const or_lat *L, const int c[4], const orc *Ulinks,
                  const orc *psi, orc *out, int dagger)
{
    int N = L->N, D = or_rep_dim(L->N, L->rep);
    orc R[8 * OR_MAXD * OR_MAXD];
    for (int k = 0; k < 8; k++)
        or_represent_link(N, L->rep, Ulinks + (size_t)k * N * N, R + (size_t)k * D * D);
    or_hop_local_rep(L, c, R, psi, out, dagger);
}

void or_represent_links(int N, int rep, long n, const orc *U, orc *R)
{
    int D = or_rep_dim(N, rep);
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; k++)
        or_represent_link(N, rep, U + (size_t)k * N * N, R + (size_t)k * D * D);
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1.1: compensated summation                                     */
/* ------------------------------------------------------------------ */
void or_fast_two_sum(double a, double b, double *s, double *c)
{
    volatile double sv = a + b;   /* volatile: keep the compensation */
    double ss = sv;
    if (fabs(a) >= fabs(b)) {
        volatile double t = ss - a;
        *c = b - t;
    } else {
        volatile double t = ss - b;
        *c = a - t;
    }
    *s = ss;
}

double or_sum_naive(const double *a, long n)
{
    double s = 0;
    for (long i = 0; i < n; i++) s += a[i];
    return s;
}

double or_sum_neumaier(const double *a, long n)
{
    double s = 0, c = 0, e;
    for (long i = 0; i < n; i++) {
        or_fast_two_sum(s, a[i], &s, &e);
        c += e;
    }
    return s + c;
}

double or_sum_neumaier2(const double *a, long n)
{
    double s = 0, c = 0, c2 = 0, e;
    for (long i = 0; i < n; i++) {
        or_fast_two_sum(s, a[i], &s, &e);
        or_fast_two_sum(c, e, &c, &e);
        c2 += e;
    }
    return s + (c + c2);
}

double or_sum_double_double(const double *a, long n)
{
    double s = 0, c = 0, e;
    for (long i = 0; i < n; i++) {
        or_fast_two_sum(s, a[i], &s, &e);
        or_fast_two_sum(s, c + e, &s, &c);
    }
    return s;
}

orc or_dot(const orc *u, const orc *v, long n)
{
    double sr = 0, cr = 0, si = 0, ci = 0, e;
    for (long i = 0; i < n; i++) {
        orc p = conj(u[i]) * v[i];
        or_fast_two_sum(sr, creal(p), &sr, &e);
        cr += e;
        or_fast_two_sum(si, cimag(p), &si, &e);
        ci += e;
    }
    return (sr + cr) + I * (si + ci);
}

double or_norm2(const orc *u, long n)
{
    double s = 0, c = 0, e;
    for (long i = 0; i < n; i++) {
        double p = creal(u[i]) * creal(u[i]) + cimag(u[i]) * cimag(u[i]);
        or_fast_two_sum(s, p, &s, &e);
        c += e;
    }
    return s + c;
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1.2: conjugate gradient on the normal equations                */
/* ------------------------------------------------------------------ */
/* out = (A + sigma) in with A = D^dag D (sys 0) or Dhat^dag Dhat (sys 1) */
static void apply_normal(const or_lat *L, const orc *UR, int sys, double sigma,
                         const orc *in, orc *out, orc *tmp)
{
    long V = or_volume(L);
    long n = (sys == 0 ? V : V / 2) * 4L * or_rep_dim(L->N, L->rep);
    if (sys == 0) {
        or_dirac_full(L, UR, in, tmp, 0);
        or_dirac_full(L, UR, tmp, out, 1);
    } else {
        or_dhat(L, UR, in, tmp, 0);
        or_dhat(L, UR, tmp, out, 1);
    }
    if (sigma != 0)
        for (long i = 0; i < n; i++) out[i] += sigma * in[i];
}

int or_cg(const or_lat *L, const orc *UR, int sys, const orc *b, orc *x,
          double tol, int max_iter, int *iters, double *true_rel_res)
{
    return or_cg_shifted(L, UR, sys, 0.0, b, x, tol, max_iter, iters,
                         true_rel_res);
}

int or_cg_shifted(const or_lat *L, const orc *UR, int sys, double sigma,
                  const orc *b, orc *x, double tol, int max_iter, int *iters,
                  double *true_rel_res)
{
    long V = or_volume(L);
    int D = or_rep_dim(L->N, L->rep);
    long n = (sys == 0 ? V : V / 2) * 4L * D;
    orc *r = malloc(n * sizeof(orc)), *p = malloc(n * sizeof(orc));
    orc *Ap = malloc(n * sizeof(orc)), *tmp = malloc(n * sizeof(orc));
    double bnorm = sqrt(or_norm2(b, n));
    int k = 0, done = 0;
    double rel = 0;
    if (bnorm == 0) {
        memset(x, 0, n * sizeof(orc));
        *iters = 0;
        *true_rel_res = 0;
        free(r); free(p); free(Ap); free(tmp);
        return 0;
    }
    while (!done) {
        /* (re)start from the true residual r = b - A x */
        apply_normal(L, UR, sys, sigma, x, Ap, tmp);
        for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
        rel = sqrt(or_norm2(r, n)) / bnorm;
        if (rel <= tol || k >= max_iter) break;
        memcpy(p, r, n * sizeof(orc));
        double rr = or_norm2(r, n);
        while (k < max_iter) {
            apply_normal(L, UR, sys, sigma, p, Ap, tmp);
            double pAp = creal(or_dot(p, Ap, n));
            double alpha = rr / pAp;
            for (long i = 0; i < n; i++) {
                x[i] += alpha * p[i];
                r[i] -= alpha * Ap[i];
            }
            double rr_new = or_norm2(r, n);
            k++;
            if (sqrt(rr_new) / bnorm <= tol) break;
            double beta = rr_new / rr;
            for (long i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
            rr = rr_new;
        }
        if (k >= max_iter) {
            apply_normal(L, UR, sys, sigma, x, Ap, tmp);
            for (long i = 0; i < n; i++) r[i] = b[i] - Ap[i];
            rel = sqrt(or_norm2(r, n)) / bnorm;
            done = 1;
        }
    }
    *iters = k;
    *true_rel_res = rel;
    free(r); free(p); free(Ap); free(tmp);
    return rel <= tol ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* fermion force (Sec. 2.5)                                              */
/* ------------------------------------------------------------------ */
void or_force(const or_lat *L, const orc *UR, const orc *X, const orc *Y,
              double *F)
{
    long V = or_volume(L);
    int N = L->N, D = or_rep_dim(L->N, L->rep), ng = N * N - 1;
    orc *TR = malloc((size_t)ng * D * D * sizeof(orc));
    or_rep_generators(N, L->rep, TR);
    orc gam[4][16];
    load_gammas(gam);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        orc PX[4 * OR_MAXD], PY[4 * OR_MAXD], A[OR_MAXD * OR_MAXD], B[OR_MAXD * OR_MAXD];
        orc M[OR_MAXD * OR_MAXD], Ud[OR_MAXD * OR_MAXD], t1[OR_MAXD * OR_MAXD],
            t2[OR_MAXD * OR_MAXD];
        for (int mu = 0; mu < 4; mu++) {
            long y = or_neighbour(L, x, mu, +1);
            const orc *Xy = X + (size_t)y * 4 * D, *Yy = Y + (size_t)y * 4 * D;
            const orc *Xx = X + (size_t)x * 4 * D, *Yx = Y + (size_t)x * 4 * D;
            /* PX = (1 - g_mu) X(x+mu),  PY = (1 + g_mu) Y(x+mu) */
            for (int s = 0; s < 4; s++)
                for (int c = 0; c < D; c++) {
                    orc vx = Xy[s * D + c], vy = Yy[s * D + c];
                    for (int t = 0; t < 4; t++) {
                        vx -= gam[mu][s * 4 + t] * Xy[t * D + c];
                        vy += gam[mu][s * 4 + t] * Yy[t * D + c];
                    }
                    PX[s * D + c] = vx;
                    PY[s * D + c] = vy;
                }
            for (int i = 0; i < D; i++)
                for (int j = 0; j < D; j++) {
                    orc a = 0, bb = 0;
                    for (int s = 0; s < 4; s++) {
                        a += PX[s * D + i] * conj(Yx[s * D + j]);
                        bb += Xx[s * D + i] * conj(PY[s * D + j]);
                    }
                    A[i * D + j] = a;
                    B[i * D + j] = bb;
                }
            const orc *U = UR + ((size_t)x * 4 + mu) * D * D;
            mat_dag(D, U, Ud);
            mat_mul(D, U, A, t1);
            mat_mul(D, B, Ud, t2);
            for (int k = 0; k < D * D; k++) M[k] = t1[k] - t2[k];
            for (int a = 0; a < ng; a++) {
                mat_mul(D, TR + (size_t)a * D * D, M, t1);
                orc tr = mat_trace(D, t1);
                F[((size_t)x * 4 + mu) * ng + a] = creal(I * tr);
            }
        }
    }
    free(TR);
}

/* ------------------------------------------------------------------ */
/* Wilson gauge action and its force (Sec. 2.4 Eq. plaquette, Sec. 2.5)  */
/* ------------------------------------------------------------------ */
/* P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag.  The gauge
 * field is periodic in every direction (the fermion boundary signs live in
 * the represented links only). */
static void plaquette(const or_lat *L, const orc *UF, long x, int mu, int nu,
                      orc *P)
{
    int N = L->N;
    long xm = or_neighbour(L, x, mu, +1), xn = or_neighbour(L, x, nu, +1);
    const orc *U1 = UF + ((size_t)x * 4 + mu) * N * N;
    const orc *U2 = UF + ((size_t)xm * 4 + nu) * N * N;
    const orc *U3 = UF + ((size_t)xn * 4 + mu) * N * N;
    const orc *U4 = UF + ((size_t)x * 4 + nu) * N * N;
    orc a[OR_MAXD * OR_MAXD], b[OR_MAXD * OR_MAXD], d[OR_MAXD * OR_MAXD];
    mat_mul(N, U1, U2, a);
    mat_dag(N, U3, d);
    mat_mul(N, a, d, b);
    mat_dag(N, U4, d);
    mat_mul(N, b, d, P);
}

double or_plaquette_action(const or_lat *L, const orc *UF, double beta)
{
    long V = or_volume(L);
    int N = L->N;
    double *site = malloc(V * sizeof(double));
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        orc P[OR_MAXD * OR_MAXD];
        double s = 0;
        for (int mu = 0; mu < 4; mu++)
            for (int nu = mu + 1; nu < 4; nu++) {
                plaquette(L, UF, x, mu, nu, P);
                s += 1.0 - creal(mat_trace(N, P)) / N;
            }
        site[x] = s;
    }
    double S = beta * or_sum_neumaier(site, V);
    free(site);
    return S;
}

/* F[x][mu][a] = d/de S_g(U_mu(x) -> exp(i e T^a) U_mu(x)) at e = 0.  The
 * plaquettes that hold U_mu(x) give Re tr(U_mu(x) W) with the staple sum
 *   W = sum_{nu != mu} [ U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
 *                      + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) ],
 * so  F^a = -(beta/N) Re tr(i T^a U_mu(x) W). */
void or_gauge_force(const or_lat *L, const orc *UF, double beta, double *F)
{
    long V = or_volume(L);
    int N = L->N, ng = N * N - 1;
    orc *T = malloc((size_t)ng * N * N * sizeof(orc));
    or_generators(N, T);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; x++) {
        orc W[OR_MAXD * OR_MAXD], a[OR_MAXD * OR_MAXD], b[OR_MAXD * OR_MAXD],
            d[OR_MAXD * OR_MAXD], M[OR_MAXD * OR_MAXD];
        for (int mu = 0; mu < 4; mu++) {
            for (int k = 0; k < N * N; k++) W[k] = 0;
            long xm = or_neighbour(L, x, mu, +1);
            for (int nu = 0; nu < 4; nu++) {
                if (nu == mu) continue;
                long xn = or_neighbour(L, x, nu, +1);
                long xdn = or_neighbour(L, x, nu, -1);
                long xmdn = or_neighbour(L, xm, nu, -1);
                /* upper staple */
                mat_dag(N, UF + ((size_t)xn * 4 + mu) * N * N, d);
                mat_mul(N, UF + ((size_t)xm * 4 + nu) * N * N, d, a);
                mat_dag(N, UF + ((size_t)x * 4 + nu) * N * N, d);
                mat_mul(N, a, d, b);
                for (int k = 0; k < N * N; k++) W[k] += b[k];
                /* lower staple */
                mat_dag(N, UF + ((size_t)xmdn * 4 + nu) * N * N, a);
                mat_dag(N, UF + ((size_t)xdn * 4 + mu) * N * N, d);
                mat_mul(N, a, d, b);
                mat_mul(N, b, UF + ((size_t)xdn * 4 + nu) * N * N, a);
                for (int k = 0; k < N * N; k++) W[k] += a[k];
            }
            mat_mul(N, UF + ((size_t)x * 4 + mu) * N * N, W, M);
            for (int g = 0; g < ng; g++) {
                mat_mul(N, T + (size_t)g * N * N, M, a);
                F[((size_t)x * 4 + mu) * ng + g] =
                    -(beta / N) * creal(I * mat_trace(N, a));
            }
        }
    }
    free(T);
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
