// hr_gauge_inst.cu -- represent kernel (U_F -> U_R with boundary signs,
// Sec. 2.3 and Sec. 5.3.1) and fermion-force kernel (Sec. 2.5) for one
// (N, representation) pair; compiled once per pair like hr_dslash_inst.cu.
#include "hr_gauge.cuh"

namespace hr {

// one link entry in precision P (real: the real part only)
__device__ inline void store_entry(int P, bool real, char *dst, cx<double> v)
{
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
// represent: one thread per (tile, slot, lane) so the record writes coalesce.
// slot k < 4 : U_R(x, mu)        with -1 if bc_mu = -1 and x_mu = L_mu - 1
// slot k >= 4: U_R(x - mu, mu)^dag = R(U_F(x - mu, mu)^dag), -1 if x_mu = 0
// ---------------------------------------------------------------------------
template <int N, int REP>
__global__ void __launch_bounds__(128) represent_kernel(const double2 *__restrict__ UF, const Geom g, int parity,
                                                        const RepOut o)
{
    constexpr int D = rep_dim(N, REP);
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = (int)(t & 31);
    const long rest = t >> 5;
    const int slot = (int)(rest & 7);
    const long tile = rest >> 3;
    if (tile >= g.ntiles) return;
    const long i = tile * HR_TILE + lane;
    if (i >= g.vh) return;
    Site s = site_of(g, i, parity);
    const int mu = slot & 3;
    const bool fwd = slot < 4;
    int c[4] = {s.c[0], s.c[1], s.c[2], s.c[3]};
    const int L[4] = {g.T, g.X, g.Y, g.Z};
    if (!fwd) c[mu] = (c[mu] - 1 + L[mu]) % L[mu];
    const long lex = (((long)c[0] * g.X + c[1]) * g.Y + c[2]) * g.Z + c[3];
    const double2 *u = UF + ((size_t)lex * 4 + mu) * N * N;
    cx<double> U[N][N];
    for (int a = 0; a < N; a++)
        for (int b = 0; b < N; b++) {
            double2 v = u[a * N + b];
            if (fwd)
                U[a][b] = {v.x, v.y};
            else
                U[b][a] = {v.x, -v.y};   // dagger
        }
    const bool neg = g.bc[mu] == -1 && (fwd ? s.c[mu] == L[mu] - 1 : s.c[mu] == 0);
    bool any_rep = false;
    for (int p = 0; p < 4; p++) any_rep |= o.rep[p] != nullptr;
    constexpr bool REAL = rep_real(REP);
    if (any_rep) {
        cx<double> Rm[D][D];
        represent<N, REP>(U, Rm);
        const double sg = neg ? -1.0 : 1.0;
        for (int r = 0; r < D; r++)
            for (int q = 0; q < D; q++) {
                const int c = r * D + q;
                const cx<double> v = sg * Rm[r][q];
                for (int P = 0; P < 4; P++) {
                    if (!o.rep[P]) continue;
                    char *dst = reinterpret_cast<char *>(o.rep[P]) + link_offset(P, REAL, D * D, tile, slot, lane, c);
                    store_entry(P, REAL, dst, v);
                }
            }
    }
    for (int r = 0; r < N; r++)
        for (int q = 0; q < N; q++) {
            const int c = r * N + q;
            for (int P = 0; P < 4; P++) {
                if (!o.fund[P]) continue;
                char *dst = reinterpret_cast<char *>(o.fund[P]) + link_offset(P, false, N * N, tile, slot, lane, c);
                store_entry(P, false, dst, U[r][q]);
            }
        }
}

template <int N, int REP>
hr_status represent_launch(const hr_gauge &gg, const double2 *UF, cudaStream_t stream)
{
    const Geom &g = gg.geom;
    for (int parity = 0; parity < 2; parity++) {
        RepOut o;
        for (int p = 0; p < 4; p++) {
            o.rep[p] = gg.rep[p][parity];
            o.fund[p] = gg.fund[p][parity];
        }
        const long threads = g.ntiles * 8 * HR_TILE;
        represent_kernel<N, REP><<<(unsigned)((threads + 127) / 128), 128, 0, stream>>>(UF, g, parity, o);
        HR_LAUNCH_CHECK("represent_kernel");
    }
    return HR_OK;
}

// ---------------------------------------------------------------------------
// fermion force (Sec. 2.5): for the link U(x, mu) owned by site x,
//   A = sum_s [(1 - g_mu) X(x+mu)]_s Y_s(x)^dag,
//   B = sum_s X_s(x) [(1 + g_mu) Y(x+mu)]_s^dag,
//   M = U_R A - B U_R^dag,   F^a += coeff * Re tr(i T_R^a M) = -coeff Im tr(T_R^a M).
// One thread per (site of `parity`, mu); X, Y read in FP64.
// ---------------------------------------------------------------------------
template <int N, int REP>
__global__ void __launch_bounds__(128) force_kernel(const ForceParams fp)
{
    constexpr int D = rep_dim(N, REP);
    constexpr int NG = N * N - 1;
    constexpr bool REAL = rep_real(REP);
    using SIO = SpinorIO<HR_F64, D>;
    using LIO = LinkIO<HR_F64, REAL, D * D>;
    const Geom &g = fp.g;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long i = t >> 2;
    const int mu = (int)(t & 3);
    if (i >= g.vh) return;
    Site s = site_of(g, i, fp.parity);
    const long nb = neighbour(g, s, mu, +1);
    cx<double> Xn[4][D], Yn[4][D], Xh[4][D], Yh[4][D];
    SIO::load(fp.X_nb, 0, nb, Xn);
    SIO::load(fp.Y_nb, 0, nb, Yn);
    SIO::load(fp.X_here, 0, i, Xh);
    SIO::load(fp.Y_here, 0, i, Yh);
    // PX = (1 - g_mu) X(x+mu), PY = (1 + g_mu) Y(x+mu) via the e_mu structure:
    // (1 + sp g) psi = [up + sp e dn ; dn + sp e^dag up]
    cx<double> PX[4][D], PY[4][D];
    for (int c = 0; c < D; c++) {
        for (int r = 0; r < 2; r++) {
            const int q = eperm(mu, r), ph = ephase(mu, r);
            PX[r][c] = Xn[r][c] + (-1.0) * ipow(ph, Xn[2 + q][c]);
            PY[r][c] = Yn[r][c] + ipow(ph, Yn[2 + q][c]);
            // lower row q gets conj(e_{r q}) times the upper component r
            PX[2 + q][c] = Xn[2 + q][c] + (-1.0) * ipow(4 - ph, Xn[r][c]);
            PY[2 + q][c] = Yn[2 + q][c] + ipow(4 - ph, Yn[r][c]);
        }
    }
    cx<double> A[D][D], B[D][D];
    for (int a = 0; a < D; a++)
        for (int b = 0; b < D; b++) {
            cx<double> sa = {0, 0}, sb = {0, 0};
            for (int sp = 0; sp < 4; sp++) {
                cmac(sa, PX[sp][a], conj(Yh[sp][b]));
                cmac(sb, Xh[sp][a], conj(PY[sp][b]));
            }
            A[a][b] = sa;
            B[a][b] = sb;
        }
    // U_R(x, mu): slot mu of this site's record (carries the boundary sign)
    const long tile = i / HR_TILE;
    const int lane = (int)(i % HR_TILE);
    const uint4 *lp = LIO::slot_ptr(fp.links, tile, mu, lane);
    cx<double> U[D][D];
    if constexpr (REAL) {
        double W[D * D];
        LIO::load(lp, W);
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++) U[a][b] = {W[a * D + b], 0.0};
    } else {
        cx<double> W[D * D];
        LIO::load(lp, W);
        for (int a = 0; a < D; a++)
            for (int b = 0; b < D; b++) U[a][b] = W[a * D + b];
    }
    // M = U A - B U^dag
    cx<double> M[D][D];
    for (int a = 0; a < D; a++)
        for (int b = 0; b < D; b++) {
            cx<double> m = {0, 0};
            for (int k = 0; k < D; k++) {
                cmac(m, U[a][k], A[k][b]);
                cmac(m, (-1.0) * B[a][k], conj(U[b][k]));
            }
            M[a][b] = m;
        }
    const long lex = lex_of(g, s);
    double *Fo = fp.F + ((size_t)lex * 4 + mu) * NG;
    for (int a = 0; a < NG; a++) {
        const double2 *T = reinterpret_cast<const double2 *>(fp.TR) + (size_t)a * D * D;
        double im = 0;
        for (int p = 0; p < D; p++)
            for (int q = 0; q < D; q++) {
                const double2 tv = __ldg(&T[p * D + q]);
                const cx<double> mv = M[q][p];
                im += tv.x * mv.im + tv.y * mv.re;
            }
        Fo[a] += -fp.coeff * im;
    }
}

template <int N, int REP>
hr_status force_launch(const ForceParams &fp, cudaStream_t stream)
{
    const long threads = fp.g.vh * 4;
    force_kernel<N, REP><<<(unsigned)((threads + 127) / 128), 128, 0, stream>>>(fp);
    HR_LAUNCH_CHECK("force_kernel");
    return HR_OK;
}

template hr_status represent_launch<HR_INST_N, HR_INST_REP>(const hr_gauge &, const double2 *, cudaStream_t);
template hr_status force_launch<HR_INST_N, HR_INST_REP>(const ForceParams &, cudaStream_t);

}  // namespace hr
