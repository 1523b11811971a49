// hr_rep.cuh -- representation maps of SU(N) written as sparse compile-time
// structure (Sec. 2.3, Table 1).
//
// Generators T^a: generalised Gell-Mann matrices / 2 (Tr T^a T^b = delta/2),
// ordered: for each pair j<k (lexicographic) the symmetric one
// (E_jk+E_kj)/2 then the antisymmetric one -i(E_jk-E_kj)/2; then the
// diagonal ones diag(1,..,1,-l,0,..)/sqrt(2l(l+1)), l = 1..N-1.
// ADJ coordinates: v_a = 2 Tr(T^a X) for X = sum_a v_a T^a, action X -> U X U^dag.
// SYM/ASYM basis: e_(ii) = E_ii, e_(ij) = (E_ij +- E_ji)/sqrt(2) (i<j, lex),
// coordinates v_n = Tr(e_n^dag X), action X -> U X U^T.
// Hence R(U)_ab = 2 Tr(T^a U T^b U^dag) (ADJ), R(U)_nm = Tr(e_n^dag U e_m U^T).
#pragma once

#include <type_traits>

#include "hr_internal.cuh"

namespace hr {

__host__ __device__ constexpr int ngen(int N) { return N * N - 1; }
__host__ __device__ constexpr int noff(int N) { return N * (N - 1); }

// --- generator T^a: number of nonzero entries, their (row, col, value) ---
__host__ __device__ constexpr int gen_nent(int N, int a) { return a < noff(N) ? 2 : a - noff(N) + 2; }
__host__ __device__ constexpr int gen_row(int N, int a, int e)
{
    return a < noff(N) ? (e == 0 ? pair_j(N, a / 2) : pair_k(N, a / 2)) : e;
}
__host__ __device__ constexpr int gen_col(int N, int a, int e)
{
    return a < noff(N) ? (e == 0 ? pair_k(N, a / 2) : pair_j(N, a / 2)) : e;
}
__host__ __device__ inline double diag_norm(int l)
{
    // 1 / sqrt(2 l (l+1))
    return l == 1 ? 0.5 : l == 2 ? 0.28867513459481288225 : l == 3 ? 0.20412414523193150818
                                                                    : 1.0 / sqrt(2.0 * l * (l + 1));
}
template <class R>
__host__ __device__ inline cx<R> gen_val(int N, int a, int e)
{
    if (a < noff(N)) {
        if ((a & 1) == 0) return {(R)0.5, (R)0};
        return e == 0 ? cx<R>{(R)0, (R)-0.5} : cx<R>{(R)0, (R)0.5};
    }
    int l = a - noff(N) + 1;
    double n = diag_norm(l);
    return {(R)(e < l ? n : -l * n), (R)0};
}

// --- SYM / ASYM basis element n ---
#define HR_RSQRT2 0.70710678118654752440
#define HR_SQRT2 1.41421356237309504880
__host__ __device__ constexpr int sb_i(int N, int rep, int n) { return sympair_i(N, n, rep == HR_ASYM); }
__host__ __device__ constexpr int sb_j(int N, int rep, int n) { return sympair_j(N, n, rep == HR_ASYM); }
__host__ __device__ constexpr int sb_nent(int N, int rep, int n) { return sb_i(N, rep, n) == sb_j(N, rep, n) ? 1 : 2; }
__host__ __device__ constexpr int sb_row(int N, int rep, int n, int e) { return e == 0 ? sb_i(N, rep, n) : sb_j(N, rep, n); }
__host__ __device__ constexpr int sb_col(int N, int rep, int n, int e) { return e == 0 ? sb_j(N, rep, n) : sb_i(N, rep, n); }
__host__ __device__ inline double sb_val(int N, int rep, int n, int e)
{
    if (sb_nent(N, rep, n) == 1) return 1.0;
    return (rep == HR_ASYM && e == 1) ? -HR_RSQRT2 : HR_RSQRT2;
}

// --- the real basis of the SU(4) 2AS (HR_ASYM_REAL): f_n = c_n S_n with
// c_n = 1 (n even) or i (n odd) and S_n real antisymmetric, entries +-1/2 at
// (P0,P1), (P1,P0), (Q0,Q1), (Q1,Q0) for the k-th pair P with complement Q:
//   f_2k = (e_P + s_k e_Q)/sqrt2,  f_2k+1 = i (e_P - s_k e_Q)/sqrt2,
//   (P, Q, s) = ((0,1),(2,3),+1), ((0,2),(1,3),-1), ((0,3),(1,2),+1).
// Each f_n is fixed by A -> *conj(A), (*A)_ij = eps_ijkl A_kl / 2, which
// commutes with A -> U A U^T when det U = 1, so R(U) is real in this basis.
__host__ __device__ constexpr int rb_p(int k, int j) { return j == 0 ? 0 : k + 1; }
__host__ __device__ constexpr int rb_q(int k, int j) { return k == 0 ? 2 + j : k == 1 ? 1 + 2 * j : 1 + j; }
__host__ __device__ constexpr int rb_row(int n, int e)
{
    return e == 0 ? rb_p(n / 2, 0) : e == 1 ? rb_p(n / 2, 1) : e == 2 ? rb_q(n / 2, 0) : rb_q(n / 2, 1);
}
__host__ __device__ constexpr int rb_col(int n, int e)
{
    return e == 0 ? rb_p(n / 2, 1) : e == 1 ? rb_p(n / 2, 0) : e == 2 ? rb_q(n / 2, 1) : rb_q(n / 2, 0);
}
// entry e of S_n
__host__ __device__ constexpr double rb_val(int n, int e)
{
    return (e & 1 ? -0.5 : 0.5) * (e < 2 ? 1.0 : ((n & 1) ? -1.0 : 1.0) * (n / 2 == 1 ? -1.0 : 1.0));
}
// c_n v for the coordinate v of f_n (i v for odd n), and conj(c_n) v
template <class R>
__host__ __device__ __forceinline__ cx<R> rb_c(int n, cx<R> v) { return (n & 1) ? cx<R>{-v.im, v.re} : v; }
template <class R>
__host__ __device__ __forceinline__ cx<R> rb_cc(int n, cx<R> v) { return (n & 1) ? cx<R>{v.im, -v.re} : v; }

// --- R(U) as a dense D x D matrix (FP64), U given as N x N: the plain sums
// over the basis elements, the definition that the folded per-entry and
// per-row formulas below are checked against (tests/host/host_checks.cu) ---
template <int N, int REP>
__host__ __device__ inline void represent(const cx<double> (&U)[N][N], cx<double> (&Rm)[rep_dim(N, REP)][rep_dim(N, REP)])
{
    constexpr int D = rep_dim(N, REP);
    if constexpr (REP == HR_FUND) {
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) Rm[i][j] = U[i][j];
    } else if constexpr (REP == HR_ADJ) {
        // R_ab = 2 Re sum_{(i,j,al) in T_a} sum_{(k,l,be) in T_b} al be U_jk conj(U_il)
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++) {
                cx<double> s = {0, 0};
                for (int e1 = 0; e1 < gen_nent(N, a); e1++) {
                    int i = gen_row(N, a, e1), j = gen_col(N, a, e1);
                    cx<double> al = gen_val<double>(N, a, e1);
                    for (int e2 = 0; e2 < gen_nent(N, b); e2++) {
                        int k = gen_row(N, b, e2), l = gen_col(N, b, e2);
                        cx<double> be = gen_val<double>(N, b, e2);
                        s = s + (al * be) * (U[j][k] * conj(U[i][l]));
                    }
                }
                Rm[a][b] = {2.0 * s.re, 0.0};
            }
    } else if constexpr (REP == HR_ASYM_REAL) {
        // R_nm = Tr(f_n^dag U f_m U^T) = conj(c_n) c_m sum_{S_n} sum_{S_m} w v U_ik U_jl
        for (int n = 0; n < D; n++)
            for (int m = 0; m < D; m++) {
                cx<double> s = {0, 0};
                for (int e1 = 0; e1 < 4; e1++) {
                    const int i = rb_row(n, e1), j = rb_col(n, e1);
                    const double w = rb_val(n, e1);
                    for (int e2 = 0; e2 < 4; e2++) {
                        const int k = rb_row(m, e2), l = rb_col(m, e2);
                        s = s + (w * rb_val(m, e2)) * (U[i][k] * U[j][l]);
                    }
                }
                Rm[n][m] = rb_cc(n, rb_c(m, s));
            }
    } else {
        // R_nm = sum_{(i,j,w) in e_n} sum_{(k,l,v) in e_m} w v U_ik U_jl
        for (int n = 0; n < D; n++)
            for (int m = 0; m < D; m++) {
                cx<double> s = {0, 0};
                for (int e1 = 0; e1 < sb_nent(N, REP, n); e1++) {
                    int i = sb_row(N, REP, n, e1), j = sb_col(N, REP, n, e1);
                    double w = sb_val(N, REP, n, e1);
                    for (int e2 = 0; e2 < sb_nent(N, REP, m); e2++) {
                        int k = sb_row(N, REP, m, e2), l = sb_col(N, REP, m, e2);
                        double v = sb_val(N, REP, m, e2);
                        s = s + (w * v) * (U[i][k] * U[j][l]);
                    }
                }
                Rm[n][m] = s;
            }
    }
}

// compile-time loop: f(std::integral_constant<int, I>) for I = B..E-1
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// a b + sgn c d as one fma chain per part
__host__ __device__ __forceinline__ cx<double> cx_pair(cx<double> a, cx<double> b, double sgn, cx<double> c, cx<double> d)
{
    const cx<double> sc = {sgn * c.re, sgn * c.im};
    return {fma(a.re, b.re, fma(-a.im, b.im, fma(sc.re, d.re, -sc.im * d.im))),
            fma(a.re, b.im, fma(a.im, b.re, fma(sc.re, d.im, sc.im * d.re)))};
}

// the 2 x 2 minor of U on rows (a, b) and columns (c, d): U_ac U_bd - U_ad U_bc
template <int N, int a, int b, int c, int d>
__host__ __device__ __forceinline__ cx<double> minor2(const cx<double> (&U)[N][N])
{
    return cx_pair(U[a][c], U[b][d], -1.0, U[a][d], U[b][c]);
}

// --- one entry R(U)_AB with every basis index a compile-time constant, so
// that a kernel can form and store the entries one at a time with U alone in
// registers.  The sums of represent() are folded where basis elements pair
// up (the compiler merges the products shared by several entries):
//   SYM:  R_(ii),(kk) = U_ik^2,  R_(ii),(kl) = sqrt2 U_ik U_il,
//         R_(ij),(kk) = sqrt2 U_ik U_jk,  R_(ij),(kl) = U_ik U_jl + U_il U_jk;
//   ASYM: R_(ij),(kl) = U_ik U_jl - U_il U_jk, a 2 x 2 minor of U;
//   real-basis 2AS: with f_n = c_n S_n, S_n = (E_P - E_P^T + s_n (E_Q - E_Q^T))/2
//         on the oriented pairs P, Q of n, sum w v U_ik U_jl =
//         (M(P_n;P_m) + s_m M(P_n;Q_m) + s_n M(Q_n;P_m) + s_n s_m M(Q_n;Q_m)) / 2,
//         M the minors of U;
//   ADJ:  the generators on one index pair share two products U_jk conj(U_il)
//         among the four entries of their block. ---
template <int N, int REP, int A, int B>
__host__ __device__ __forceinline__ cx<double> rep_entry(const cx<double> (&U)[N][N])
{
    if constexpr (REP == HR_FUND) {
        return U[A][B];
    } else if constexpr (REP == HR_ADJ) {
        constexpr int NO = noff(N);
        if constexpr (A < NO && B < NO) {
            // T_a, T_b on the pairs (p, q), (r, s): with z1 = U_qr conj(U_ps),
            // z2 = U_qs conj(U_pr) the four (symmetric, antisymmetric) entries are
            // Re z1 + Re z2, Im z1 - Im z2, Im z1 + Im z2, Re z2 - Re z1
            constexpr int p = pair_j(N, A / 2), q = pair_k(N, A / 2), r = pair_j(N, B / 2), t = pair_k(N, B / 2);
            const cx<double> z1 = U[q][r] * conj(U[p][t]), z2 = U[q][t] * conj(U[p][r]);
            if constexpr (!(A & 1) && !(B & 1)) return {z1.re + z2.re, 0.0};
            if constexpr (!(A & 1) && (B & 1)) return {z1.im - z2.im, 0.0};
            if constexpr ((A & 1) && !(B & 1)) return {z1.im + z2.im, 0.0};
            return {z2.re - z1.re, 0.0};
        } else if constexpr (A < NO) {
            // T_a on (p, q), T_b = diag(b_f): 2 sum_f b_f (Re or Im) U_qf conj(U_pf)
            constexpr int p = pair_j(N, A / 2), q = pair_k(N, A / 2), l = B - NO + 1;
            double acc = 0.0;
            static_for<0, l + 1>([&](auto FF) {
                constexpr int f = decltype(FF)::value;
                const double bf = gen_val<double>(N, B, f).re;
                const cx<double> y = U[q][f] * conj(U[p][f]);
                acc = fma(bf, (A & 1) ? y.im : y.re, acc);
            });
            return {2.0 * acc, 0.0};
        } else if constexpr (B < NO) {
            // T_a = diag(a_e), T_b on (r, s): 2 sum_e a_e (Re or Im) U_er conj(U_es)
            constexpr int r = pair_j(N, B / 2), t = pair_k(N, B / 2), l = A - NO + 1;
            double acc = 0.0;
            static_for<0, l + 1>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                const double ae = gen_val<double>(N, A, e).re;
                const cx<double> x = U[e][r] * conj(U[e][t]);
                acc = fma(ae, (B & 1) ? x.im : x.re, acc);
            });
            return {2.0 * acc, 0.0};
        } else {
            // both diagonal: 2 sum_e sum_f a_e b_f |U_ef|^2
            constexpr int la = A - NO + 1, lb = B - NO + 1;
            double acc = 0.0;
            static_for<0, la + 1>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                double row = 0.0;
                static_for<0, lb + 1>([&](auto FF) {
                    constexpr int f = decltype(FF)::value;
                    const double n2 = fma(U[e][f].re, U[e][f].re, U[e][f].im * U[e][f].im);
                    row = fma(gen_val<double>(N, B, f).re, n2, row);
                });
                acc = fma(gen_val<double>(N, A, e).re, row, acc);
            });
            return {2.0 * acc, 0.0};
        }
    } else if constexpr (REP == HR_ASYM_REAL) {
        constexpr int kn = A / 2, km = B / 2;
        constexpr double sn = rb_val(A, 2) * 2.0, sm = rb_val(B, 2) * 2.0;
        constexpr int p0 = rb_p(kn, 0), p1 = rb_p(kn, 1), q0 = rb_q(kn, 0), q1 = rb_q(kn, 1);
        constexpr int r0 = rb_p(km, 0), r1 = rb_p(km, 1), t0 = rb_q(km, 0), t1 = rb_q(km, 1);
        const cx<double> m1 = minor2<N, p0, p1, r0, r1>(U), m2 = minor2<N, p0, p1, t0, t1>(U);
        const cx<double> m3 = minor2<N, q0, q1, r0, r1>(U), m4 = minor2<N, q0, q1, t0, t1>(U);
        const cx<double> s = {0.5 * ((m1.re + sm * m2.re) + sn * (m3.re + sm * m4.re)),
                              0.5 * ((m1.im + sm * m2.im) + sn * (m3.im + sm * m4.im))};
        return rb_cc(A, rb_c(B, s));
    } else {
        constexpr bool asym = REP == HR_ASYM;
        constexpr int i = sb_i(N, REP, A), j = sb_j(N, REP, A), k = sb_i(N, REP, B), l = sb_j(N, REP, B);
        if constexpr (asym) {
            return minor2<N, i, j, k, l>(U);
        } else if constexpr (i == j && k == l) {
            return U[i][k] * U[i][k];
        } else if constexpr (i == j || k == l) {
            // one index pair is diagonal: sqrt2 U_ik U_jl (the other product is the same)
            const cx<double> pr = U[i][k] * U[j][l];
            return {HR_SQRT2 * pr.re, HR_SQRT2 * pr.im};
        } else {
            return cx_pair(U[i][k], U[j][l], 1.0, U[i][l], U[j][k]);
        }
    }
}

// --- row n of R(U), n known only at run time (the represent kernel's rolled
// row loop, whose body stays small enough for the instruction caches); the
// column indices are compile-time constants and ld(i, k) returns U_ik.  The
// sums are those of rep_entry.  For ADJ only the rows of the off-diagonal
// generators (n < N(N-1)) are formed here; rep_entry gives the diagonal ones. ---
template <int N, int REP, class LD>
__host__ __device__ __forceinline__ void rep_row(int n, LD &&ld, cx<double> (&e)[rep_dim(N, REP)])
{
    constexpr int D = rep_dim(N, REP);
    if constexpr (REP == HR_FUND) {
        static_for<0, N>([&](auto K) { e[decltype(K)::value] = ld(n, decltype(K)::value); });
    } else if constexpr (REP == HR_SYM || REP == HR_ASYM) {
        const int i = sb_i(N, REP, n), j = sb_j(N, REP, n);
        cx<double> ui[N], uj[N];
        static_for<0, N>([&](auto K) {
            constexpr int k = decltype(K)::value;
            ui[k] = ld(i, k);
            uj[k] = ld(j, k);
        });
        if (REP == HR_SYM && i == j) {
            static_for<0, D>([&](auto M) {
                constexpr int m = decltype(M)::value, k = sb_i(N, REP, m), l = sb_j(N, REP, m);
                if constexpr (k == l) {
                    e[m] = ui[k] * ui[k];
                } else {
                    const cx<double> pr = ui[k] * ui[l];
                    e[m] = {HR_SQRT2 * pr.re, HR_SQRT2 * pr.im};
                }
            });
        } else {
            static_for<0, D>([&](auto M) {
                constexpr int m = decltype(M)::value, k = sb_i(N, REP, m), l = sb_j(N, REP, m);
                if constexpr (REP == HR_ASYM) {
                    e[m] = cx_pair(ui[k], uj[l], -1.0, ui[l], uj[k]);
                } else if constexpr (k == l) {
                    const cx<double> pr = ui[k] * uj[k];
                    e[m] = {HR_SQRT2 * pr.re, HR_SQRT2 * pr.im};
                } else {
                    e[m] = cx_pair(ui[k], uj[l], 1.0, ui[l], uj[k]);
                }
            });
        }
    } else if constexpr (REP == HR_ASYM_REAL) {
        const int kn = n >> 1;
        const double sn = ((n & 1) ? -1.0 : 1.0) * (kn == 1 ? -1.0 : 1.0);
        cx<double> up0[N], up1[N], uq0[N], uq1[N];
        const int p0 = rb_p(kn, 0), p1 = rb_p(kn, 1), q0 = rb_q(kn, 0), q1 = rb_q(kn, 1);
        static_for<0, N>([&](auto K) {
            constexpr int k = decltype(K)::value;
            up0[k] = ld(p0, k);
            up1[k] = ld(p1, k);
            uq0[k] = ld(q0, k);
            uq1[k] = ld(q1, k);
        });
        static_for<0, D>([&](auto M) {
            constexpr int m = decltype(M)::value, km = m / 2;
            constexpr double sm = rb_val(m, 2) * 2.0;
            constexpr int r0 = rb_p(km, 0), r1 = rb_p(km, 1), t0 = rb_q(km, 0), t1 = rb_q(km, 1);
            const cx<double> m1 = cx_pair(up0[r0], up1[r1], -1.0, up0[r1], up1[r0]);
            const cx<double> m2 = cx_pair(up0[t0], up1[t1], -1.0, up0[t1], up1[t0]);
            const cx<double> m3 = cx_pair(uq0[r0], uq1[r1], -1.0, uq0[r1], uq1[r0]);
            const cx<double> m4 = cx_pair(uq0[t0], uq1[t1], -1.0, uq0[t1], uq1[t0]);
            const cx<double> sv = {0.5 * ((m1.re + sm * m2.re) + sn * (m3.re + sm * m4.re)),
                                   0.5 * ((m1.im + sm * m2.im) + sn * (m3.im + sm * m4.im))};
            e[m] = rb_cc(n, rb_c(m, sv));
        });
    } else {
        // ADJ, off-diagonal generator on the pair (p, q), symmetric or antisymmetric
        const int p = pair_j(N, n >> 1), q = pair_k(N, n >> 1);
        const bool anti = n & 1;
        cx<double> up[N], uq[N];
        static_for<0, N>([&](auto K) {
            constexpr int k = decltype(K)::value;
            up[k] = ld(p, k);
            uq[k] = ld(q, k);
        });
        constexpr int NO = noff(N);
        static_for<0, D>([&](auto B) {
            constexpr int b = decltype(B)::value;
            if constexpr (b < NO) {
                constexpr int r = pair_j(N, b / 2), t = pair_k(N, b / 2);
                const cx<double> z1 = uq[r] * conj(up[t]), z2 = uq[t] * conj(up[r]);
                double v;
                if constexpr (!(b & 1))
                    v = anti ? z1.im + z2.im : z1.re + z2.re;
                else
                    v = anti ? z2.re - z1.re : z1.im - z2.im;
                e[b] = {v, 0.0};
            } else {
                constexpr int l = b - NO + 1;
                double are = 0.0, aim = 0.0;
                static_for<0, l + 1>([&](auto FF) {
                    constexpr int f = decltype(FF)::value;
                    const double bf = gen_val<double>(N, b, f).re;
                    const cx<double> y = uq[f] * conj(up[f]);
                    are = fma(bf, y.re, are);
                    aim = fma(bf, y.im, aim);
                });
                e[b] = {2.0 * (anti ? aim : are), 0.0};
            }
        });
    }
}

// --- action of R(F) on a colour vector without forming R(F) (in-kernel
// rebuild): vector -> matrix, conjugate by F, matrix -> vector.  All basis
// indices are compile-time constants (static_for), so X, Z stay in registers.
template <int N, int REP, class R>
__device__ __forceinline__ void rep_act(const cx<R> (&F)[N][N], const cx<R> (&v)[rep_dim(N, REP)],
                                        cx<R> (&out)[rep_dim(N, REP)])
{
    constexpr int D = rep_dim(N, REP);
    if constexpr (REP == HR_FUND) {
#pragma unroll
        for (int i = 0; i < N; i++) {
            cx<R> s = {0, 0};
#pragma unroll
            for (int j = 0; j < N; j++) cmac(s, F[i][j], v[j]);
            out[i] = s;
        }
    } else {
        cx<R> X[N][N];
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) X[i][j] = {0, 0};
        if constexpr (REP == HR_ADJ) {
            static_for<0, D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                static_for<0, gen_nent(N, a)>([&](auto EE) {
                    constexpr int e = decltype(EE)::value;
                    cmac(X[gen_row(N, a, e)][gen_col(N, a, e)], gen_val<R>(N, a, e), v[a]);
                });
            });
        } else if constexpr (REP == HR_ASYM_REAL) {
            static_for<0, D>([&](auto NN) {
                constexpr int n = decltype(NN)::value;
                const cx<R> cv = rb_c(n, v[n]);
                static_for<0, 4>([&](auto EE) {
                    constexpr int e = decltype(EE)::value;
                    rmac(X[rb_row(n, e)][rb_col(n, e)], (R)rb_val(n, e), cv);
                });
            });
        } else {
            static_for<0, D>([&](auto NN) {
                constexpr int n = decltype(NN)::value;
                static_for<0, sb_nent(N, REP, n)>([&](auto EE) {
                    constexpr int e = decltype(EE)::value;
                    rmac(X[sb_row(N, REP, n, e)][sb_col(N, REP, n, e)], (R)sb_val(N, REP, n, e), v[n]);
                });
            });
        }
        // Z = F X
        cx<R> Z[N][N];
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) {
                cx<R> s = {0, 0};
#pragma unroll
                for (int k = 0; k < N; k++) cmac(s, F[i][k], X[k][j]);
                Z[i][j] = s;
            }
        if constexpr (REP == HR_ADJ) {
            // v'_a = 2 sum_{(i,j,al) in T_a} al Y_ji,  Y = Z F^dag: Y_ji = sum_k Z_jk conj(F_ik)
            static_for<0, D>([&](auto A) {
                constexpr int a = decltype(A)::value;
                cx<R> s = {0, 0};
                static_for<0, gen_nent(N, a)>([&](auto EE) {
                    constexpr int e = decltype(EE)::value;
                    constexpr int i = gen_row(N, a, e), j = gen_col(N, a, e);
                    cx<R> y = {0, 0};
#pragma unroll
                    for (int k = 0; k < N; k++) cmac_cj(y, F[i][k], Z[j][k]);
                    cmac(s, gen_val<R>(N, a, e), y);
                });
                out[a] = (R)2 * s;
            });
        } else if constexpr (REP == HR_ASYM_REAL) {
            // v'_n = Tr(f_n^dag Y) = conj(c_n) sum_{(i,j,w) in S_n} w Y_ij,  Y = Z F^T
            static_for<0, D>([&](auto NN) {
                constexpr int n = decltype(NN)::value;
                cx<R> s = {0, 0};
                static_for<0, 4>([&](auto EE) {
                    constexpr int e = decltype(EE)::value;
                    constexpr int i = rb_row(n, e), j = rb_col(n, e);
                    cx<R> y = {0, 0};
#pragma unroll
                    for (int k = 0; k < N; k++) cmac(y, Z[i][k], F[j][k]);
                    rmac(s, (R)rb_val(n, e), y);
                });
                out[n] = rb_cc(n, s);
            });
        } else {
            // v'_n = sum_{(i,j,w) in e_n} w Y_ij with Y = Z F^T = F X F^T, which is
            // symmetric (SYM) or antisymmetric (2AS) like X: the two entries of an
            // off-diagonal e_n contribute alike, v'_n = sqrt2 Y_ij (i < j), and
            // only Y_ij = sum_k Z_ik F_jk of the upper triangle is formed
            static_for<0, D>([&](auto NN) {
                constexpr int n = decltype(NN)::value;
                constexpr int i = sb_i(N, REP, n), j = sb_j(N, REP, n);
                cx<R> y = {0, 0};
#pragma unroll
                for (int k = 0; k < N; k++) cmac(y, Z[i][k], F[j][k]);
                out[n] = i == j ? y : cx<R>{(R)HR_SQRT2 * y.re, (R)HR_SQRT2 * y.im};
            });
        }
    }
}

}  // namespace hr
