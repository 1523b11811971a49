// hr_gauge_inst.cu -- represent kernel (U_F -> U_R with boundary signs,
// Sec. 2.3 and Sec. 5.3.1) and fermion-force kernel (Sec. 2.5) for one
// (N, representation) pair; compiled once per pair like hr_dslash_inst.cu.
#include "hr_gauge.cuh"

namespace hr {

// one link entry in precision P (real: the real part only)
__device__ inline void store_entry(int P, bool real, char *dst, cx<double> v)
{
    if (P == HR_DF64) {
        const df re(v.re), im(v.im);
        if (real)
            *reinterpret_cast<float2 *>(dst) = make_float2(re.hi, re.lo);
        else
            *reinterpret_cast<float4 *>(dst) = make_float4(re.hi, re.lo, im.hi, im.lo);
        return;
    }
    if (real) {
        if (P == HR_F64) *reinterpret_cast<double *>(dst) = v.re;
        if (P == HR_F32) *reinterpret_cast<float *>(dst) = (float)v.re;
        if (P == HR_F16) *reinterpret_cast<__half *>(dst) = __double2half(v.re);
        if (P == HR_BF16) *reinterpret_cast<__nv_bfloat16 *>(dst) = __double2bfloat16(v.re);
    } else {
        if (P == HR_F64) *reinterpret_cast<double2 *>(dst) = make_double2(v.re, v.im);
        if (P == HR_F32) *reinterpret_cast<float2 *>(dst) = make_float2((float)v.re, (float)v.im);
        if (P == HR_F16) *reinterpret_cast<__half2 *>(dst) = __halves2half2(__double2half(v.re), __double2half(v.im));
        if (P == HR_BF16)
            *reinterpret_cast<__nv_bfloat162 *>(dst) = __halves2bfloat162(__double2bfloat16(v.re), __double2bfloat16(v.im));
    }
}

// ---------------------------------------------------------------------------
// represent: one thread per link (x, mu), x of parity p with half index
// tile*32 + lane, so every link is represented exactly once (in FP64) and
// written twice, both writes coalesced:
//   slot mu   of x's record (parity p):        U_R(x, mu)
//   slot 4+mu of (x+mu)'s record (parity 1-p): U_R(x, mu)^dag = R(U(x, mu)^dag)
// with -1 on both if bc_mu = -1 and x_mu = L_mu - 1 (Sec. 5.3.1).  The
// fundamental records get U and U^dag (the in-kernel rebuild applies the
// sign itself).
// ---------------------------------------------------------------------------
template <int N, int REP>
__global__ void __launch_bounds__(128) represent_kernel(const double2 *__restrict__ UF, const Geom g, const RepOut o0,
                                                        const RepOut o1)
{
    constexpr int D = rep_dim(N, REP);
    constexpr bool REAL = rep_real(REP);
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(t & 31);
    long rest = t >> 5;
    const int mu = (int)(rest & 3);
    rest >>= 2;
    const long tile = rest % g.ntiles;
    const int parity = (int)(rest / g.ntiles);
    if (parity > 1) return;
    const long i = tile * HR_TILE + lane;
    if (i >= g.vh) return;
    const Site s = site_of(g, i, parity);
    const long ib = neighbour(g, s, mu, +1);   // half index of x + mu in parity 1 - p
    const long tb = ib / HR_TILE;
    const int lb = (int)(ib % HR_TILE);
    const RepOut &of = parity == 0 ? o0 : o1;   // records of x's parity
    const RepOut &ob = parity == 0 ? o1 : o0;   // records of (x+mu)'s parity
    const int L[4] = {g.T, g.X, g.Y, g.Z};
    const long lex = lex_of(g, s);
    const double2 *u = UF + ((size_t)lex * 4 + mu) * N * N;
    cx<double> U[N][N];
    for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++) {
            const double2 v = u[a * N + b];
            U[a][b] = {v.x, v.y};
        }
    const bool neg = g.bc[mu] == -1 && s.c[mu] == L[mu] - 1;
    bool any_rep = false;
    for (int p = 0; p < HR_NPREC; p++) any_rep |= of.rep[p] != nullptr;
    if (any_rep) {
        cx<double> Rm[D][D];
        represent<N, REP>(U, Rm);
        const double sg = neg ? -1.0 : 1.0;
        for (int r = 0; r < D; r++)
            for (int q = 0; q < D; q++) {
                const cx<double> v = sg * Rm[r][q];
                for (int P = 0; P < HR_NPREC; P++) {
                    if (!of.rep[P]) continue;
                    const int RS = link_row_stride(N, REP, P);
                    store_entry(P, REAL, reinterpret_cast<char *>(of.rep[P]) + link_offset(P, REAL, D * RS, tile, mu, lane, r * RS + q), v);
                    // the dagger: entry (q, r) of the backward slot
                    store_entry(P, REAL, reinterpret_cast<char *>(ob.rep[P]) + link_offset(P, REAL, D * RS, tb, 4 + mu, lb, q * RS + r), conj(v));
                }
            }
    }
    for (int r = 0; r < N; r++)
        for (int q = 0; q < N; q++)
            for (int P = 0; P < HR_NPREC; P++) {
                if (!of.fund[P]) continue;
                store_entry(P, false, reinterpret_cast<char *>(of.fund[P]) + link_offset(P, false, N * N, tile, mu, lane, r * N + q), U[r][q]);
                store_entry(P, false, reinterpret_cast<char *>(ob.fund[P]) + link_offset(P, false, N * N, tb, 4 + mu, lb, q * N + r), conj(U[r][q]));
            }
}

template <int N, int REP>
hr_status represent_launch(const hr_gauge &gg, const double2 *UF, cudaStream_t stream)
{
    const Geom &g = gg.geom;
    RepOut o[2];
    for (int parity = 0; parity < 2; parity++)
        for (int p = 0; p < HR_NPREC; p++) {
            o[parity].rep[p] = gg.rep[p][parity];
            o[parity].fund[p] = gg.fund[p][parity];
        }
    const long threads = 2 * g.ntiles * 4 * HR_TILE;
    represent_kernel<N, REP><<<(unsigned)((threads + 127) / 128), 128, 0, stream>>>(UF, g, o[0], o[1]);
    HR_LAUNCH_CHECK("represent_kernel");
    return HR_OK;
}

// ---------------------------------------------------------------------------
// fermion force (Sec. 2.5): for the link U(x, mu) owned by site x,
//   A = sum_s [(1 - g_mu) X(x+mu)]_s Y_s(x)^dag,
//   B = sum_s X_s(x) [(1 + g_mu) Y(x+mu)]_s^dag,
//   F^a += coeff * Re tr(i T_R^a (U_R A - B U_R^dag)).
// The projectors leave two independent spin components, so
//   A = sum_{r=0,1} hX_r z_r^dag,  B = sum_r w_r hY_r^dag   with
//   hX = upper[(1 - g_mu) X(x+mu)],  z = upper[(1 - g_mu) Y(x)],
//   hY = upper[(1 + g_mu) Y(x+mu)],  w = upper[(1 + g_mu) X(x)],
// and U A - B U^dag = K = sum_r (U hX_r) z_r^dag - w_r (U hY_r)^dag needs four
// matrix-vector products.  tr(T_R^a K) is pulled back to the fundamental,
// tr(T_R^a K) = tr(T^a P) (below), so only the N x N matrix P meets the
// generators.
// One thread per (site of `parity`, mu); FP64 throughout.
// ---------------------------------------------------------------------------
// The pullback tr(T_R^a K) = tr(T^a P) for K = x y^dag (x, y in the space of
// R), written with the N x N matrices of the representation-space vectors:
//   SYM/2AS: X = sum_n x_n e_n (e_n the orthonormal basis of symmetric /
//     antisymmetric matrices, R(U) X = U X U^T, T_R^a X = T X + X T^T), so
//     y^dag T_R^a x = tr(Y^dag (T X + X T^T)) = tr(T^a (X Y^dag + (Y^dag X)^T))
//     and with X^T = s X, Y^T = s Y (s = +1 SYM, -1 2AS) this is
//     P = 2 s X conj(Y);
//   ADJ: X = sum_a x_a T^a (R(U) X = U X U^dag, T_R^a X = [T^a, X], and
//     x_a = 2 tr(T^a X)), so y^dag T_R^a x = 2 tr(Y^dag [T^a, X]) and
//     P = 2 [X, Y^dag] with Y^dag = sum_a conj(y_a) T^a;
//   FUND: P = K.
// Each costs N^3 (SYM/2AS) or 2 N^3 (ADJ) complex products instead of the
// D_R^2 products of K itself.

// M = sum_n x_n e_n (SYM/2AS) or sum_a x_a T^a (ADJ); conj_x: use conj(x_n)
// (for the complex real-basis matrices f_n of the SU(4) 2AS: conj(sum x_n f_n))
template <int N, int REP, bool CONJ_X>
__device__ __forceinline__ void rep_matrix(const cx<double> (&x)[rep_dim(N, REP)], cx<double> (&M)[N][N])
{
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) M[i][j] = {0, 0};
    if constexpr (REP == HR_ADJ) {
        static_for<0, N * N - 1>([&](auto AA) {
            constexpr int a = decltype(AA)::value;
            const cx<double> xa = CONJ_X ? conj(x[a]) : x[a];
            static_for<0, gen_nent(N, a)>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                cx<double> &m = M[gen_row(N, a, e)][gen_col(N, a, e)];
                cmac(m, gen_val<double>(N, a, e), xa);
            });
        });
    } else if constexpr (REP == HR_ASYM_REAL) {
        // sum_n x_n f_n, f_n = c_n S_n; with CONJ_X its complex conjugate
        static_for<0, rep_dim(N, REP)>([&](auto NN) {
            constexpr int n = decltype(NN)::value;
            const cx<double> t = rb_c(n, x[n]);
            const cx<double> xn = CONJ_X ? conj(t) : t;
            static_for<0, 4>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                rmac(M[rb_row(n, e)][rb_col(n, e)], rb_val(n, e), xn);
            });
        });
    } else {
        static_for<0, rep_dim(N, REP)>([&](auto NN) {
            constexpr int n = decltype(NN)::value;
            const cx<double> xn = CONJ_X ? conj(x[n]) : x[n];
            static_for<0, sb_nent(N, REP, n)>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                cx<double> &m = M[sb_row(N, REP, n, e)][sb_col(N, REP, n, e)];
                rmac(m, sb_val(N, REP, n, e), xn);
            });
        });
    }
}

// P += f (A B)
template <int N>
__device__ __forceinline__ void mat_mac(cx<double> (&P)[N][N], double f, const cx<double> (&A)[N][N],
                                        const cx<double> (&B)[N][N])
{
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) {
            cx<double> s = {0, 0};
#pragma unroll
            for (int k = 0; k < N; k++) cmac(s, A[i][k], B[k][j]);
            rmac(P[i][j], f, s);
        }
}

// P += sgn * (pullback of x y^dag)
template <int N, int REP>
__device__ __forceinline__ void pullback_add(cx<double> (&P)[N][N], double sgn, const cx<double> (&x)[rep_dim(N, REP)],
                                             const cx<double> (&y)[rep_dim(N, REP)])
{
    if constexpr (REP == HR_FUND) {
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) rmac(P[i][j], sgn, x[i] * conj(y[j]));
    } else if constexpr (REP == HR_ADJ) {
        cx<double> X[N][N], Yd[N][N];
        rep_matrix<N, REP, false>(x, X);
        rep_matrix<N, REP, true>(y, Yd);   // Y^dag (T^a Hermitian)
        mat_mac<N>(P, 2.0 * sgn, X, Yd);
        mat_mac<N>(P, -2.0 * sgn, Yd, X);
    } else {
        cx<double> X[N][N], Yc[N][N];
        rep_matrix<N, REP, false>(x, X);
        rep_matrix<N, REP, true>(y, Yc);   // conj(Y)
        mat_mac<N>(P, (REP == HR_SYM ? 2.0 : -2.0) * sgn, X, Yc);
    }
}

template <int N, int REP>
__global__ void __launch_bounds__(128) force_kernel(const ForceParams fp)
{
    constexpr int D = rep_dim(N, REP);
    constexpr int NG = N * N - 1;
    constexpr bool REAL = rep_real(REP);
    using SIO = SpinorIO<HR_F64, D>;
    constexpr int RS = link_row_stride(N, REP, HR_F64);
    using LIO = LinkIO<HR_F64, REAL, D * RS>;
    const Geom &g = fp.g;
    // two threads per link (adjacent lanes): spin component r = 0, 1 of the projections
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = (int)(t & 1);
    const long link = t >> 1;
    const long i = link >> 2;
    const int mu = (int)(link & 3);
    const bool active = i < g.vh;   // both lanes of a pair agree
    cx<double> P[N][N];
    if (active) {
        Site s = site_of(g, i, fp.parity);
        const long nb = neighbour(g, s, mu, +1);
        const int q = 2 + eperm(mu, r), ph = ephase(mu, r);
        auto ld = [&](const FieldView &f, long site, int sp, int c) {
            const uint4 v = __ldg(SIO::site_ptr(f, 0, site) + (sp * D + c));
            return cx<double>{__hiloint2double((int)v.y, (int)v.x), __hiloint2double((int)v.w, (int)v.z)};
        };
        // upper component r of (1 -+ g_mu) psi: psi_r -+ i^{ph} psi_q
        cx<double> hX[D], hY[D], z[D], w[D];
        for (int c = 0; c < D; c++) {
            hX[c] = ld(fp.X_nb, nb, r, c) + (-1.0) * ipow(ph, ld(fp.X_nb, nb, q, c));
            hY[c] = ld(fp.Y_nb, nb, r, c) + ipow(ph, ld(fp.Y_nb, nb, q, c));
            z[c] = ld(fp.Y_here, i, r, c) + (-1.0) * ipow(ph, ld(fp.Y_here, i, q, c));
            w[c] = ld(fp.X_here, i, r, c) + ipow(ph, ld(fp.X_here, i, q, c));
        }
        // u = U hX, v = U hY with U_R(x, mu) (slot mu, boundary sign included), row by row
        const long tile = i / HR_TILE;
        const int lane = (int)(i % HR_TILE);
        const uint4 *lp = LIO::slot_ptr(fp.links, tile, mu, lane);
        cx<double> u[D], v[D];
        for (int a = 0; a < D; a++) {
            cx<double> su = {0, 0}, sv = {0, 0};
            for (int b = 0; b < D; b++) {
                const int cc = a * RS + b;
                const uint4 ch = __ldg(lp + (size_t)(cc / LIO::VPC) * HR_TILE);
                cx<double> uab;
                if constexpr (REAL)
                    uab = {LIO::runpack(ch, cc % LIO::VPC), 0.0};
                else
                    uab = LIO::cunpack(ch, 0);
                cmac(su, uab, hX[b]);
                cmac(sv, uab, hY[b]);
            }
            u[a] = su;
            v[a] = sv;
        }
        // K_r = u z^dag - w v^dag, pulled back to the fundamental
#pragma unroll
        for (int a = 0; a < N; a++)
#pragma unroll
            for (int b = 0; b < N; b++) P[a][b] = {0, 0};
        pullback_add<N, REP>(P, 1.0, u, z);
        pullback_add<N, REP>(P, -1.0, w, v);
    } else {
#pragma unroll
        for (int a = 0; a < N; a++)
#pragma unroll
            for (int b = 0; b < N; b++) P[a][b] = {0, 0};
    }
    // combine the two spin components of the link
#pragma unroll
    for (int a = 0; a < N; a++)
#pragma unroll
        for (int b = 0; b < N; b++) {
            P[a][b].re += __shfl_xor_sync(0xffffffffu, P[a][b].re, 1);
            P[a][b].im += __shfl_xor_sync(0xffffffffu, P[a][b].im, 1);
        }
    if (!active || r != 0) return;
    const long lex = lex_of(g, site_of(g, i, fp.parity));
    double *Fo = fp.F + ((size_t)lex * 4 + mu) * NG;
    // F^a += -coeff Im tr(T^a P) = -coeff Im sum_{(i,j,al) in T^a} al P_ji
    static_for<0, NG>([&](auto AA) {
        constexpr int a = decltype(AA)::value;
        cx<double> tr = {0, 0};
        static_for<0, gen_nent(N, a)>([&](auto EE) {
            constexpr int e = decltype(EE)::value;
            cmac(tr, gen_val<double>(N, a, e), P[gen_col(N, a, e)][gen_row(N, a, e)]);
        });
        Fo[a] += -fp.coeff * tr.im;
    });
}

template <int N, int REP>
hr_status force_launch(const ForceParams &fp, cudaStream_t stream)
{
    const long threads = fp.g.vh * 8;   // two threads per link
    force_kernel<N, REP><<<(unsigned)((threads + 127) / 128), 128, 0, stream>>>(fp);
    HR_LAUNCH_CHECK("force_kernel");
    return HR_OK;
}

template hr_status represent_launch<HR_INST_N, HR_INST_REP>(const hr_gauge &, const double2 *, cudaStream_t);
template hr_status force_launch<HR_INST_N, HR_INST_REP>(const ForceParams &, cudaStream_t);

}  // namespace hr
