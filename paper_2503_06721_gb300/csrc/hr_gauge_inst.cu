// hr_gauge_inst.cu -- represent kernel (U_F -> U_R with boundary signs,
// Sec. 2.3 and Sec. 5.3.1) and fermion-force kernel (Sec. 2.5) for one
// (N, representation) pair; compiled once per pair like hr_dslash_inst.cu.
#include "hr_gauge.cuh"

namespace hr {

// one link entry v in precision P at fw and its conjugate at bw (real: the
// real part only); each part is rounded once and the conjugate's imaginary
// part is the exact negation of the rounded one
template <int P, bool REAL>
__device__ __forceinline__ void store_pair(char *fw, char *bw, cx<double> v)
{
    if constexpr (P == HR_DF64) {
        const df re(v.re);
        if constexpr (REAL) {
            *reinterpret_cast<float2 *>(fw) = make_float2(re.hi, re.lo);
            *reinterpret_cast<float2 *>(bw) = make_float2(re.hi, re.lo);
        } else {
            const df im(v.im);
            *reinterpret_cast<float4 *>(fw) = make_float4(re.hi, re.lo, im.hi, im.lo);
            *reinterpret_cast<float4 *>(bw) = make_float4(re.hi, re.lo, -im.hi, -im.lo);
        }
    } else if constexpr (REAL) {
        if constexpr (P == HR_F64) {
            *reinterpret_cast<double *>(fw) = v.re;
            *reinterpret_cast<double *>(bw) = v.re;
        } else if constexpr (P == HR_F32) {
            const float r = f32_rn(v.re);
            *reinterpret_cast<float *>(fw) = r;
            *reinterpret_cast<float *>(bw) = r;
        } else if constexpr (P == HR_F16) {
            const __half r = __double2half(v.re);
            *reinterpret_cast<__half *>(fw) = r;
            *reinterpret_cast<__half *>(bw) = r;
        } else {
            const __nv_bfloat16 r = __double2bfloat16(v.re);
            *reinterpret_cast<__nv_bfloat16 *>(fw) = r;
            *reinterpret_cast<__nv_bfloat16 *>(bw) = r;
        }
    } else {
        if constexpr (P == HR_F64) {
            *reinterpret_cast<double2 *>(fw) = make_double2(v.re, v.im);
            *reinterpret_cast<double2 *>(bw) = make_double2(v.re, -v.im);
        } else if constexpr (P == HR_F32) {
            const float r = f32_rn(v.re), i = f32_rn(v.im);
            *reinterpret_cast<float2 *>(fw) = make_float2(r, i);
            *reinterpret_cast<float2 *>(bw) = make_float2(r, -i);
        } else if constexpr (P == HR_F16) {
            const __half r = __double2half(v.re), i = __double2half(v.im);
            *reinterpret_cast<__half2 *>(fw) = __halves2half2(r, i);
            *reinterpret_cast<__half2 *>(bw) = __halves2half2(r, __hneg(i));
        } else {
            const __nv_bfloat16 r = __double2bfloat16(v.re), i = __double2bfloat16(v.im);
            *reinterpret_cast<__nv_bfloat162 *>(fw) = __halves2bfloat162(r, i);
            *reinterpret_cast<__nv_bfloat162 *>(bw) = __halves2bfloat162(r, __hneg(i));
        }
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
    const long lex = lex_of(g, s);
    const double2 *u = UF + ((size_t)lex * 4 + mu) * N * N;
    auto uld = [&](int a, int b) {
        const double2 v = __ldg(u + a * N + b);
        return cx<double>{v.x, v.y};
    };
    // the fundamental entries are copied one at a time (an 8 x 8 link would
    // not fit in registers); a higher representation needs all of U at once
    constexpr int NU = REP == HR_FUND ? 1 : N;
    cx<double> U[NU][NU];
    if constexpr (REP != HR_FUND) {
#pragma unroll
        for (int a = 0; a < N; a++)
#pragma unroll
            for (int b = 0; b < N; b++) U[a][b] = uld(a, b);
    }
    const int Lmu = mu == 0 ? g.T : mu == 1 ? g.X : mu == 2 ? g.Y : g.Z;
    const int xmu = mu == 0 ? s.c[0] : mu == 1 ? s.c[1] : mu == 2 ? s.c[2] : s.c[3];
    const int bmu = mu == 0 ? g.bc[0] : mu == 1 ? g.bc[1] : mu == 2 ? g.bc[2] : g.bc[3];
    // the boundary sign as a flip of the sign bits (no FP64 multiply)
    const unsigned long long sgn = bmu == -1 && xmu == Lmu - 1 ? 0x8000000000000000ull : 0ull;
    auto sg = [&](cx<double> e) {
        return cx<double>{__longlong_as_double(__double_as_longlong(e.re) ^ (long long)sgn),
                          __longlong_as_double(__double_as_longlong(e.im) ^ (long long)sgn)};
    };
    bool any_rep = false;
    static_for<0, HR_NPREC>([&](auto PP) { any_rep |= of.rep[decltype(PP)::value] != nullptr; });
    // every entry is formed once, in FP64, a row at a time, and the row is
    // written to the forward and backward records of each precision present.
    // The loop over rows is rolled: its body (one row, the stores of all
    // precisions) fits the instruction caches, which the fully unrolled D x D
    // entries with every precision's stores interleaved did not.
    auto put_row = [&](int r, const cx<double> (&e)[D]) {
        static_for<0, HR_NPREC>([&](auto PP) {
            constexpr int P = decltype(PP)::value;
            if (!of.rep[P]) return;
            constexpr int RS = link_row_stride(N, REP, P);
            char *fw = reinterpret_cast<char *>(of.rep[P]);
            char *bw = reinterpret_cast<char *>(ob.rep[P]);
            static_for<0, D>([&](auto QQ) {
                constexpr int q = decltype(QQ)::value;
                // the dagger: entry (q, r) of the backward slot
                store_pair<P, REAL>(fw + link_offset(P, REAL, D * RS, tile, mu, lane, r * RS + q),
                                    bw + link_offset(P, REAL, D * RS, tb, 4 + mu, lb, q * RS + r), sg(e[q]));
            });
        });
    };
    if (any_rep) {
        constexpr int NROLL = REP == HR_ADJ ? noff(N) : D;
#pragma unroll 1
        for (int r = 0; r < NROLL; r++) {
            cx<double> e[D];
            rep_row<N, REP>(r, uld, e);
            put_row(r, e);
        }
        if constexpr (REP == HR_ADJ)
            static_for<noff(N), D>([&](auto RR) {
                constexpr int r = decltype(RR)::value;
                cx<double> e[D];
                static_for<0, D>([&](auto QQ) { e[decltype(QQ)::value] = rep_entry<N, REP, r, decltype(QQ)::value>(U); });
                put_row(r, e);
            });
    }
    static_for<0, HR_NPREC>([&](auto PP) {
        constexpr int P = decltype(PP)::value;
        if (!of.fund[P]) return;
#pragma unroll
        for (int r = 0; r < N; r++)
#pragma unroll
            for (int q = 0; q < N; q++) {
                cx<double> w;
                if constexpr (REP == HR_FUND)
                    w = uld(r, q);
                else
                    w = U[r][q];
                store_pair<P, false>(reinterpret_cast<char *>(of.fund[P]) +
                                         link_offset(P, false, N * N, tile, mu, lane, r * N + q),
                                     reinterpret_cast<char *>(ob.fund[P]) +
                                         link_offset(P, false, N * N, tb, 4 + mu, lb, q * N + r), w);
            }
    });
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
// One thread per (site of `parity`, mu); FP64 throughout, or float-float.
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
// (for the complex real-basis matrices f_n of the SU(4) 2AS: conj(sum x_n f_n)).
// R = double, or df for the float-float force.
template <int N, int REP, bool CONJ_X, class R>
__device__ __forceinline__ void rep_matrix(const cx<R> (&x)[rep_dim(N, REP)], cx<R> (&M)[N][N])
{
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) M[i][j] = {R(0), R(0)};
    if constexpr (REP == HR_ADJ) {
        static_for<0, N * N - 1>([&](auto AA) {
            constexpr int a = decltype(AA)::value;
            const cx<R> xa = CONJ_X ? conj(x[a]) : x[a];
            static_for<0, gen_nent(N, a)>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                cx<R> &m = M[gen_row(N, a, e)][gen_col(N, a, e)];
                cmac(m, gen_val<R>(N, a, e), xa);
            });
        });
    } else if constexpr (REP == HR_ASYM_REAL) {
        // sum_n x_n f_n, f_n = c_n S_n; with CONJ_X its complex conjugate
        static_for<0, rep_dim(N, REP)>([&](auto NN) {
            constexpr int n = decltype(NN)::value;
            const cx<R> t = rb_c(n, x[n]);
            const cx<R> xn = CONJ_X ? conj(t) : t;
            static_for<0, 4>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                rmac(M[rb_row(n, e)][rb_col(n, e)], R(rb_val(n, e)), xn);
            });
        });
    } else {
        static_for<0, rep_dim(N, REP)>([&](auto NN) {
            constexpr int n = decltype(NN)::value;
            const cx<R> xn = CONJ_X ? conj(x[n]) : x[n];
            static_for<0, sb_nent(N, REP, n)>([&](auto EE) {
                constexpr int e = decltype(EE)::value;
                cx<R> &m = M[sb_row(N, REP, n, e)][sb_col(N, REP, n, e)];
                rmac(m, R(sb_val(N, REP, n, e)), xn);
            });
        });
    }
}

// P += f (A B)
template <int N, class R>
__device__ __forceinline__ void mat_mac(cx<R> (&P)[N][N], R f, const cx<R> (&A)[N][N], const cx<R> (&B)[N][N])
{
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j < N; j++) {
            cx<R> s = {R(0), R(0)};
#pragma unroll
            for (int k = 0; k < N; k++) cmac(s, A[i][k], B[k][j]);
            rmac(P[i][j], f, s);
        }
}

// P += sgn * (pullback of x y^dag)
template <int N, int REP, class R>
__device__ __forceinline__ void pullback_add(cx<R> (&P)[N][N], double sgn, const cx<R> (&x)[rep_dim(N, REP)],
                                             const cx<R> (&y)[rep_dim(N, REP)])
{
    if constexpr (REP == HR_FUND) {
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
            for (int j = 0; j < N; j++) rmac(P[i][j], R(sgn), x[i] * conj(y[j]));
    } else if constexpr (REP == HR_ADJ) {
        cx<R> X[N][N], Yd[N][N];
        rep_matrix<N, REP, false>(x, X);
        rep_matrix<N, REP, true>(y, Yd);   // Y^dag (T^a Hermitian)
        mat_mac<N>(P, R(2.0 * sgn), X, Yd);
        mat_mac<N>(P, R(-2.0 * sgn), Yd, X);
    } else {
        cx<R> X[N][N], Yc[N][N];
        rep_matrix<N, REP, false>(x, X);
        rep_matrix<N, REP, true>(y, Yc);   // conj(Y)
        mat_mac<N>(P, R((REP == HR_SYM ? 2.0 : -2.0) * sgn), X, Yc);
    }
}

// the sum of a value over the two lanes of a pair
__device__ __forceinline__ double pair_sum(double v) { return v + __shfl_xor_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ df pair_sum(df v)
{
    return v + df(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
}
// ... and over the two pairs of a group of four lanes
__device__ __forceinline__ df quad_sum(df v)
{
    return v + df(__shfl_xor_sync(0xffffffffu, v.hi, 2), __shfl_xor_sync(0xffffffffu, v.lo, 2));
}
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(df v) { return (double)v; }

// FP64 arithmetic on the FP64 links, two threads per link
template <int N, int REP>
__global__ void __launch_bounds__(128) force_kernel(const ForceParams fp)
{
    constexpr int LP = HR_F64;
    constexpr int D = rep_dim(N, REP);
    constexpr int NG = N * N - 1;
    constexpr bool REAL = rep_real(REP);
    using R = typename St<LP>::R;
    using SIO = SpinorIO<HR_F64, D>;
    constexpr int RS = link_row_stride(N, REP, LP);
    using LIO = LinkIO<LP, REAL, D * RS>;
    const Geom &g = fp.g;
    // two threads per link (adjacent lanes): spin component r = 0, 1 of the projections
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = (int)(t & 1);
    const long link = t >> 1;
    const long i = link >> 2;
    const int mu = (int)(link & 3);
    const bool active = i < g.vh;   // both lanes of a pair agree
    cx<R> P[N][N];
#pragma unroll
    for (int a = 0; a < N; a++)
#pragma unroll
        for (int b = 0; b < N; b++) P[a][b] = {R(0), R(0)};
    if (active) {
        Site s = site_of(g, i, fp.parity);
        const long nb = neighbour(g, s, mu, +1);
        const int q = 2 + eperm(mu, r), ph = ephase(mu, r);
        auto ld = [&](const FieldView &f, long site, int sp, int c) {
            const uint4 v = __ldg(SIO::site_ptr(f, 0, site) + (sp * D + c));
            return cx<double>{__hiloint2double((int)v.y, (int)v.x), __hiloint2double((int)v.w, (int)v.z)};
        };
        auto cv = [](cx<double> v) { return cx<R>{R(v.re), R(v.im)}; };
        // upper component r of (1 -+ g_mu) psi: psi_r -+ i^{ph} psi_q
        cx<R> hX[D], hY[D], z[D], w[D];
#pragma unroll
        for (int c = 0; c < D; c++) {
            hX[c] = cv(ld(fp.X_nb, nb, r, c) + (-1.0) * ipow(ph, ld(fp.X_nb, nb, q, c)));
            hY[c] = cv(ld(fp.Y_nb, nb, r, c) + ipow(ph, ld(fp.Y_nb, nb, q, c)));
            z[c] = cv(ld(fp.Y_here, i, r, c) + (-1.0) * ipow(ph, ld(fp.Y_here, i, q, c)));
            w[c] = cv(ld(fp.X_here, i, r, c) + ipow(ph, ld(fp.X_here, i, q, c)));
        }
        // u = U hX, v = U hY with U_R(x, mu) (slot mu, boundary sign included), row by row
        const long tile = i / HR_TILE;
        const int lane = (int)(i % HR_TILE);
        const uint4 *lp = LIO::slot_ptr(fp.links, tile, mu, lane);
        auto link = [&](int a, int b) {
            const int cc = a * RS + b;
            const uint4 ch = __ldg(lp + (size_t)(cc / LIO::VPC) * HR_TILE);
            if constexpr (REAL)
                return cx<R>{LIO::runpack(ch, cc % LIO::VPC), R(0)};
            else
                return LIO::cunpack(ch, 0);
        };
        cx<R> u[D], v[D];
#pragma unroll
        for (int a = 0; a < D; a++) {
            cx<R> su = {R(0), R(0)}, sv = {R(0), R(0)};
#pragma unroll
            for (int b = 0; b < D; b++) {
                const cx<R> uab = link(a, b);
                cmac(su, uab, hX[b]);
                cmac(sv, uab, hY[b]);
            }
            u[a] = su;
            v[a] = sv;
        }
        // K_r = u z^dag - w v^dag, pulled back to the fundamental
        pullback_add<N, REP>(P, 1.0, u, z);
        pullback_add<N, REP>(P, -1.0, w, v);
    }
    // combine the two spin components of the link
#pragma unroll
    for (int a = 0; a < N; a++)
#pragma unroll
        for (int b = 0; b < N; b++) {
            P[a][b].re = pair_sum(P[a][b].re);
            P[a][b].im = pair_sum(P[a][b].im);
        }
    if (!active || r != 0) return;
    const long lex = lex_of(g, site_of(g, i, fp.parity));
    double *Fo = fp.F + ((size_t)lex * 4 + mu) * NG;
    // F^a += -coeff Im tr(T^a P) = -coeff Im sum_{(i,j,al) in T^a} al P_ji
    static_for<0, NG>([&](auto AA) {
        constexpr int a = decltype(AA)::value;
        cx<R> tr = {R(0), R(0)};
        static_for<0, gen_nent(N, a)>([&](auto EE) {
            constexpr int e = decltype(EE)::value;
            cmac(tr, gen_val<R>(N, a, e), P[gen_col(N, a, e)][gen_row(N, a, e)]);
        });
        Fo[a] += -fp.coeff * to_double(tr.im);
    });
}

// Float-float arithmetic on the DF64 links, four threads per link: thread
// (r, k) forms one term of K_r -- k = 0: +(U hX_r) z_r^dag, k = 1: -w_r (U
// hY_r)^dag -- so that a thread runs one matrix-vector product and one
// pullback (float-float code is about three times the FP64 code; with both
// terms in one thread the warps waited on instruction fetch).  The FP64
// spinors are projected in FP64 and split into float-float pairs; the four
// partial P are summed with shuffles.
template <int N, int REP>
__global__ void __launch_bounds__(128) force_df64_kernel(const ForceParams fp)
{
    constexpr int D = rep_dim(N, REP);
    constexpr int NG = N * N - 1;
    constexpr bool REAL = rep_real(REP);
    using R = df;
    using SIO = SpinorIO<HR_F64, D>;
    constexpr int RS = link_row_stride(N, REP, HR_DF64);
    using LIO = LinkIO<HR_DF64, REAL, D * RS>;
    const Geom &g = fp.g;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = (int)(t & 1), r = (int)((t >> 1) & 1);
    const long link = t >> 2;
    const long i = link >> 2;
    const int mu = (int)(link & 3);
    const bool active = i < g.vh;   // the four lanes of a link agree
    cx<R> P[N][N];
#pragma unroll
    for (int a = 0; a < N; a++)
#pragma unroll
        for (int b = 0; b < N; b++) P[a][b] = {R(0), R(0)};
    if (active) {
        Site s = site_of(g, i, fp.parity);
        const long nb = neighbour(g, s, mu, +1);
        const int q = 2 + eperm(mu, r), ph = ephase(mu, r);
        // k = 0: h = hX = upper[(1 - g) X(x+mu)], o = z = upper[(1 - g) Y(x)]
        // k = 1: h = hY = upper[(1 + g) Y(x+mu)], o = w = upper[(1 + g) X(x)]
        const FieldView &fh = k ? fp.Y_nb : fp.X_nb;
        const FieldView &fo = k ? fp.X_here : fp.Y_here;
        // the sign -1 (k = 0) as a flip of the sign bits of i^ph psi_q
        const unsigned flip = k ? 0u : 0x80000000u;
        auto ld = [&](const FieldView &f, long site, int sp, int c, unsigned fl) {
            const uint4 v = __ldg(SIO::site_ptr(f, 0, site) + (sp * D + c));
            return cx<double>{__hiloint2double((int)(v.y ^ fl), (int)v.x), __hiloint2double((int)(v.w ^ fl), (int)v.z)};
        };
        auto cv = [](cx<double> v) { return cx<R>{R(v.re), R(v.im)}; };
        cx<R> h[D], o[D];
#pragma unroll
        for (int c = 0; c < D; c++) {
            h[c] = cv(ld(fh, nb, r, c, 0u) + ipow(ph, ld(fh, nb, q, c, flip)));
            o[c] = cv(ld(fo, i, r, c, 0u) + ipow(ph, ld(fo, i, q, c, flip)));
        }
        const long tile = i / HR_TILE;
        const int lane = (int)(i % HR_TILE);
        const uint4 *lp = LIO::slot_ptr(fp.links, tile, mu, lane);
        cx<R> m[D];
#pragma unroll
        for (int a = 0; a < D; a++) {
            cx<R> sm = {R(0), R(0)};
#pragma unroll
            for (int b = 0; b < D; b++) {
                const int cc = a * RS + b;
                const uint4 ch = __ldg(lp + (size_t)(cc / LIO::VPC) * HR_TILE);
                cx<R> uab;
                if constexpr (REAL)
                    uab = {LIO::runpack(ch, cc % LIO::VPC), R(0)};
                else
                    uab = LIO::cunpack(ch, 0);
                cmac(sm, uab, h[b]);
            }
            m[a] = sm;
        }
        if (k == 0)
            pullback_add<N, REP>(P, 1.0, m, o);
        else
            pullback_add<N, REP>(P, -1.0, o, m);
    }
#pragma unroll
    for (int a = 0; a < N; a++)
#pragma unroll
        for (int b = 0; b < N; b++) {
            P[a][b].re = pair_sum(P[a][b].re);
            P[a][b].im = pair_sum(P[a][b].im);
            P[a][b].re = quad_sum(P[a][b].re);
            P[a][b].im = quad_sum(P[a][b].im);
        }
    if (!active || (t & 3) != 0) return;
    const long lex = lex_of(g, site_of(g, i, fp.parity));
    double *Fo = fp.F + ((size_t)lex * 4 + mu) * NG;
    static_for<0, NG>([&](auto AA) {
        constexpr int a = decltype(AA)::value;
        cx<R> tr = {R(0), R(0)};
        static_for<0, gen_nent(N, a)>([&](auto EE) {
            constexpr int e = decltype(EE)::value;
            cmac(tr, gen_val<R>(N, a, e), P[gen_col(N, a, e)][gen_row(N, a, e)]);
        });
        Fo[a] += -fp.coeff * to_double(tr.im);
    });
}

template <int N, int REP>
hr_status force_launch(const ForceParams &fp, cudaStream_t stream)
{
    if (fp.arith == HR_DF64) {
        const long threads = fp.g.vh * 16;   // four threads per link
        force_df64_kernel<N, REP><<<(unsigned)((threads + 127) / 128), 128, 0, stream>>>(fp);
        HR_LAUNCH_CHECK("force_df64_kernel");
    } else {
        const long threads = fp.g.vh * 8;    // two threads per link
        force_kernel<N, REP><<<(unsigned)((threads + 127) / 128), 128, 0, stream>>>(fp);
        HR_LAUNCH_CHECK("force_kernel");
    }
    return HR_OK;
}

template hr_status represent_launch<HR_INST_N, HR_INST_REP>(const hr_gauge &, const double2 *, cudaStream_t);
template hr_status force_launch<HR_INST_N, HR_INST_REP>(const ForceParams &, cudaStream_t);

}  // namespace hr
