/*
 * hr_oracle.h -- plain FP64 CPU oracle for the Wilson-Dirac hot path of
 * "High-Performance Simulations of Higher Representations of Wilson Fermions"
 * (HiRep v2, arXiv 2503.06721).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * restatement of the paper's definitions that the GPU library is checked
 * against.  Only tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Conventions (all FP64, complex numbers are C99 double _Complex):
 *   lattice dims[4] = {T, X, Y, Z}, mu = 0 is time (Sec. 2.1).
 *   lexicographic site index  lex = ((t*X + x)*Y + y)*Z + z.
 *   even sites: (t+x+y+z) mod 2 == 0 (Sec. 4.3.3, even-odd preconditioning).
 *   half (parity) fields are indexed by lex/2 inside their parity (Z even).
 *   spinor field  psi[lex][spin 0..3][colour 0..D-1]
 *   gauge field   U[lex][mu 0..3][row][col]  (links in the + directions,
 *                 Sec. 3.1.3 "Field Types").
 *   force field   F[lex][mu][a], a = 0..N^2-2 (Lie-algebra components).
 */
#ifndef HR_ORACLE_H
#define HR_ORACLE_H

#include <complex.h>

typedef double _Complex orc;

/* OR_ASYM_REAL: the two-index antisymmetric representation of SU(4) (the 6,
 * a real representation, Table 1) written in a basis in which R(U) is real
 * orthogonal; only N = 4 */
enum { OR_FUND = 0, OR_ADJ = 1, OR_SYM = 2, OR_ASYM = 3, OR_ASYM_REAL = 4 };

typedef struct {
    int N;        /* gauge group SU(N) */
    int rep;      /* OR_FUND / OR_ADJ / OR_SYM / OR_ASYM / OR_ASYM_REAL (Table 1) */
    int dims[4];  /* T, X, Y, Z */
    int bc[4];    /* +1 periodic, -1 antiperiodic (Sec. 5.3.1) */
    double m0;    /* bare mass m in D_m = D + m (Eq. D_m) */
} or_lat;

/* ---- representation data (Sec. 2.3, Table 1) ---- */
int  or_rep_dim(int N, int rep);
/* gamma matrices of Sec. 2.2 (mu = 0..3) and gamma5 = g0 g1 g2 g3 (mu = 4),
 * row-major 4x4 */
void or_gamma(int mu, orc *g);
/* generators T^a of SU(N), Tr T^a T^b = delta/2, [(N^2-1)][N][N] */
void or_generators(int N, orc *T);
/* orthonormal basis of the representation space: for ADJ the T^a (with the
 * coordinate map v_a = 2 Tr(T^a X)); for SYM/ASYM the matrices e_n with
 * Tr(e_n^dag e_m) = delta; for ASYM_REAL (N = 4) the antisymmetric matrices
 *   f = (e_P + s e_Q)/sqrt2,  f' = i (e_P - s e_Q)/sqrt2
 * for the index pairs (P, Q; s) = ((01),(23);+1), ((02),(13);-1),
 * ((03),(12);+1), each pair P with its complement Q, s the sign of the
 * permutation (P, Q): every such f is fixed by A -> *conj(A) with
 * (*A)_ij = 1/2 eps_ijkl A_kl, a map that commutes with A -> U A U^T for
 * det U = 1, so R(U) is real in this basis.  Returns the number of basis
 * matrices */
int  or_rep_basis(int N, int rep, orc *E);
/* represented link R(U) (D x D, row-major).  returns D */
int  or_represent_link(int N, int rep, const orc *U, orc *R);
/* T_R^a = -i d/de R(exp(i e T^a)) at e = 0, [(N^2-1)][D][D] */
void or_rep_generators(int N, int rep, orc *TR);

/* ---- fields ---- */
long or_volume(const or_lat *L);
void or_coords(const or_lat *L, long lex, int c[4]);
long or_lex(const or_lat *L, const int c[4]);
long or_neighbour(const or_lat *L, long lex, int mu, int dir /* +1 / -1 */);
int  or_parity(const or_lat *L, long lex);

/* U_R(x,mu) = R(U_F(x,mu)), times -1 on links with x_mu = L_mu - 1 in every
 * antiperiodic direction (Sec. 5.3.1: a minus sign on one slice of the
 * represented field). UR is [V][4][D][D]. */
void or_represent_field(const or_lat *L, const orc *UF, orc *UR);

/* ---- Wilson-Dirac operator, Eq. (D_m^R) ---- */
/* out = D_m in (dagger = 0) or D_m^dag in (dagger = 1), full lexicographic
 * fields.  D^dag is D with gamma_mu -> -gamma_mu (gamma_mu Hermitian). */
void or_dirac_full(const or_lat *L, const orc *UR, const orc *in, orc *out,
                   int dagger);
/* hopping block D_{p,1-p} = P_p (D_m - (4+m)) P_{1-p}, half fields:
 * out_half (parity p) = D_{p,1-p} in_half (parity 1-p).  Sec. 4.3.3 Eq. (dmeo) */
void or_hop_parity(const or_lat *L, const orc *UR, int out_parity,
                   const orc *in_half, orc *out_half, int dagger);
/* even-odd preconditioned operator of Sec. 4.3.3 for plain Wilson fermions:
 *   Dhat = (4+m)^2 - D_eo D_oe, on even half fields.
 * dagger = 1 gives Dhat^dag = (4+m)^2 - (D^dag)_eo (D^dag)_oe. */
void or_dhat(const or_lat *L, const orc *UR, const orc *in_e, orc *out_e,
             int dagger);

/* The same hopping block at a list of output sites only, for checking large
 * lattices one site at a time: out[k] = (D_{p,1-p} in_half)(site k) where the
 * sites are given as half indices of parity p.  Links are taken from the
 * FUNDAMENTAL field UF and represented on the fly (or_represent_link, with the
 * boundary signs of or_represent_field).  out is [nsites][4][D]. */
void or_hop_sites(const or_lat *L, const orc *UF, int out_parity,
                  const orc *in_half, const long *sites, long nsites,
                  orc *out, int dagger);

/* One output site from gathered data, for lattices too large to hold on the
 * host: c = coordinates (t,x,y,z) of the output site x; Ulinks[8][N][N] the
 * FUNDAMENTAL links U(x, mu) (k = mu < 4) and U(x - mu, mu) (k = 4 + mu);
 * psi[8][4][D] the neighbour spinors psi(x + mu) (k < 4), psi(x - mu) (k >= 4).
 * out[4][D] = -1/2 sum_mu [ (1 -+ g_mu) U_R(x,mu) psi(x+mu)
 *                         + (1 +- g_mu) U_R(x-mu,mu)^dag psi(x-mu) ]
 * with the boundary signs of or_represent_field; lower signs for dagger. */
void or_hop_local(const or_lat *L, const int c[4], const orc *Ulinks,
                  const orc *psi, orc *out, int dagger);
/* The same from represented links: Rlinks[8][D][D] = R(U) of the 8 links
 * above (without boundary signs; the sign is applied from the coordinates,
 * as in or_hop_local), e.g. rounded copies of the stored links. */
void or_hop_local_rep(const or_lat *L, const int c[4], const orc *Rlinks,
                      const orc *psi, orc *out, int dagger);
/* R[k] = or_represent_link(U[k]) for k < n. */
void or_represent_links(int N, int rep, long n, const orc *U, orc *R);

/* ---- reductions (Sec. 4.1.1, Algorithms FastTwoSum .. DoubleDoubleSum) ---- */
void   or_fast_two_sum(double a, double b, double *s, double *c);
double or_sum_naive(const double *a, long n);
double or_sum_neumaier(const double *a, long n);
double or_sum_neumaier2(const double *a, long n);
double or_sum_double_double(const double *a, long n);
/* <u, v> = sum conj(u_i) v_i, real and imaginary parts each Neumaier-summed */
orc    or_dot(const orc *u, const orc *v, long n);
double or_norm2(const orc *u, long n);

/* ---- CG on the normal equations (Sec. 4.1.2) ----
 * sys = 0: A = D_m^dag D_m on full lexicographic fields (n = V*4*D)
 * sys = 1: A = Dhat^dag Dhat on even half fields      (n = V/2*4*D)
 * Textbook Hestenes-Stiefel CG from x (x is the initial guess on entry),
 * stopping when the recomputed true residual |b - A x| / |b| <= tol.
 * Returns 0 on convergence, 1 otherwise. */
int or_cg(const or_lat *L, const orc *UR, int sys, const orc *b, orc *x,
          double tol, int max_iter, int *iters, double *true_rel_res);
/* The same textbook CG on the shifted system (A + sigma) x = b, sigma >= 0.
 * The multi-shift inversion of the RHMC (Sec. 4.3.2) solves
 * (Q^2 + beta_k) x_k = phi for every pole beta_k of the rational
 * approximation; its definition is one such solve per shift, which is what
 * this function provides (sigma = 0 is or_cg). */
int or_cg_shifted(const or_lat *L, const orc *UR, int sys, double sigma,
                  const orc *b, orc *x, double tol, int max_iter, int *iters,
                  double *true_rel_res);

/* ---- fermion force (Sec. 2.5, HMC) ----
 * F[x][mu][a] = d/de  S(U_F(x,mu) -> exp(i e T^a) U_F(x,mu)) at e = 0 for
 * S = -2 Re <Y, D_m X> with X, Y held fixed.  When X = (D^dag D)^{-1} phi and
 * Y = D X this is the derivative of S_f = phi^dag (D^dag D)^{-1} phi.
 *   F^a = Re tr[ i T_R^a (U_R A - B U_R^dag) ],
 *   A = sum_s [(1 - g_mu) X(x+mu)]_s Y_s(x)^dag,
 *   B = sum_s X_s(x) [(1 + g_mu) Y(x+mu)]_s^dag.
 * UR must carry the boundary signs (as from or_represent_field). */
void or_force(const or_lat *L, const orc *UR, const orc *X, const orc *Y,
              double *F);

/* ---- Wilson gauge action (Sec. 2.4, Eq. plaquette) and its force ----
 * S_g = beta sum_{x, mu<nu} (1 - Re tr P_{mu nu}(x) / N), the gauge field
 * periodic in every direction.  F[x][mu][a] = d/de S_g(U_mu(x) ->
 * exp(i e T^a) U_mu(x)) at e = 0 = -(beta/N) Re tr(i T^a U_mu(x) W_mu(x)),
 * W the sum of the six staples (Sec. 2.5 writes this, divided by -T_F, as
 * the gauge force F_G). */
double or_plaquette_action(const or_lat *L, const orc *UF, double beta);
void or_gauge_force(const or_lat *L, const orc *UF, double beta, double *F);

/* ---- helpers ---- */
void or_split_parity(const or_lat *L, const orc *full, orc *even, orc *odd);
void or_merge_parity(const or_lat *L, const orc *even, const orc *odd,
                     orc *full);
int  or_num_threads(void);

#endif
