// hr_dslash_split.cuh -- the hopping kernel with two threads per output site
// (each owning half of the colour rows), for stored links.
//
// The paper's "D_R-site-parallel" observation (Sec. 6.2): splitting the
// colour matrix-vector products of a site over several threads lowers the
// registers a thread needs, which matters once D_R grows.  Here a pair of
// adjacent lanes shares a site: both load the neighbour spinor (the same
// address in the same instruction, so one request) and form the full
// half-spinor, and each multiplies it by its D/2 rows of the link (its own
// 16-byte chunks of the slot record) and accumulates its D/2 rows of the
// four output spin components.  The arithmetic per hop equals hr_dslash.cuh.
#pragma once

#include "hr_dslash.cuh"

namespace hr {

template <int N, int REP, int P>
struct SplitShape {
    static constexpr int D = rep_dim(N, REP);
    static constexpr bool REAL = rep_real(REP);
    static constexpr int DR = D / 2;
    static constexpr int VPC = link_vpc(P, REAL);
    static constexpr bool OK = (D % 2 == 0) && ((DR * D) % VPC == 0);
    static constexpr int NCH = (DR * D) / VPC;   // chunks per half slot
};

template <int N, int REP, int P, int EPI>
__global__ void __launch_bounds__(128) hop_split_kernel(const HopParams prm)
{
    using Sh = SplitShape<N, REP, P>;
    static_assert(Sh::OK, "split kernel needs an even D and whole chunks per half slot");
    using S = St<P>;
    using R = typename S::R;
    constexpr int D = Sh::D, DR = Sh::DR;
    constexpr bool REAL = Sh::REAL;
    using SIO = SpinorIO<P, D>;
    using LIO = LinkIO<P, REAL, D * D>;

    const Geom &g = prm.g;
    const int rhs = blockIdx.y;
    if (prm.state && cg_idle(prm.state[rhs])) return;
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long i = t >> 1;
    const int part = (int)(t & 1);
    const bool active = i < g.vh;
    const R sg = prm.dagger ? (R)-1 : (R)1;

    cx<R> acc[4][DR];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < DR; c++) acc[s][c] = {0, 0};

    if (active) {
        const Site st = site_of(g, i, prm.out_parity);
        const long tile = i / HR_TILE;
        const int lane = (int)(i % HR_TILE);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int mu = k & 3;
            const bool fwd = k < 4;
            const long nb = neighbour(g, st, mu, fwd ? +1 : -1);
            const R sp = fwd ? -sg : sg;
            cx<R> psi[4][D];
            SIO::load(prm.in, rhs, nb, psi);
            cx<R> h[2][D];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < D; c++)
                    h[r][c] = psi[r][c] + sp * ipow(ephase(mu, r), psi[2 + eperm(mu, r)][c]);
            // this thread's rows part*DR .. part*DR+DR-1 of the slot
            const uint4 *lp = LIO::slot_ptr(prm.links, tile, k, lane) + (size_t)part * Sh::NCH * HR_TILE;
#pragma unroll
            for (int j = 0; j < Sh::NCH; j++) {
                const uint4 v = __ldcs(lp + (size_t)j * HR_TILE);
#pragma unroll
                for (int q = 0; q < Sh::VPC; q++) {
                    const int cc = j * Sh::VPC + q;   // component inside the half slot
                    const int row = cc / D, col = cc % D;
                    cx<R> w;
                    if constexpr (REAL)
                        w = {LIO::runpack(v, q), (R)0};
                    else
                        w = LIO::cunpack(v, q);
                    // accumulate straight into the reconstruction
                    cx<R> s0 = {0, 0}, s1 = {0, 0};
                    if constexpr (REAL) {
                        rmac(s0, w.re, h[0][col]);
                        rmac(s1, w.re, h[1][col]);
                    } else {
                        cmac(s0, w, h[0][col]);
                        cmac(s1, w, h[1][col]);
                    }
                    acc[0][row] = acc[0][row] + s0;
                    acc[1][row] = acc[1][row] + s1;
                    acc[2 + eperm(mu, 0)][row] = acc[2 + eperm(mu, 0)][row] + sp * ipow(4 - ephase(mu, 0), s0);
                    acc[2 + eperm(mu, 1)][row] = acc[2 + eperm(mu, 1)][row] + sp * ipow(4 - ephase(mu, 1), s1);
                }
            }
        }
        const R a = (R)prm.a, b = (R)prm.b;
        const R dsc = (R)SIO::ld_scale(prm.diag.data ? prm.diag : prm.in, rhs, i);
#pragma unroll
        for (int s = 0; s < 4; s++) {
            if (prm.diag.data) {
                cx<R> d[D];
                SIO::load_spin(prm.diag, rhs, i, s, dsc, d);
#pragma unroll
                for (int c = 0; c < DR; c++) acc[s][c] = a * acc[s][c] + b * d[part * DR + c];
            } else {
#pragma unroll
                for (int c = 0; c < DR; c++) acc[s][c] = a * acc[s][c];
            }
        }
    }

    double red = 0;
    if constexpr (EPI == EPI_STORE || EPI == EPI_STORE_NORM) {
        // the site scale (F16/BF16) is the max over both halves of the site
        R m = 0;
        if constexpr (S::scaled) {
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < DR; c++) m = fmaxf(m, fmaxf(fabsf(acc[s][c].re), fabsf(acc[s][c].im)));
            m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        }
        if (active) {
            char *base = prm.out.data + (size_t)rhs * prm.out.rhs_stride + (size_t)i * SIO::BYTES;
            const R inv = (S::scaled && m > 0) ? (R)1 / m : (R)1;
            if constexpr (S::scaled)
                if (part == 0) *(reinterpret_cast<float *>(prm.out.scale + (size_t)rhs * prm.out.rhs_stride) + i) = m;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < DR; c++) {
                    char *e = base + (size_t)(s * D + part * DR + c) * prec_cbytes(P);
                    if constexpr (P == HR_F64)
                        *reinterpret_cast<double2 *>(e) = make_double2(acc[s][c].re, acc[s][c].im);
                    else if constexpr (P == HR_F32)
                        *reinterpret_cast<float2 *>(e) = make_float2(acc[s][c].re, acc[s][c].im);
                    else
                        *reinterpret_cast<typename S::C *>(e) = S::st(inv * acc[s][c]);
                    red += (double)(acc[s][c].re * acc[s][c].re + acc[s][c].im * acc[s][c].im);
                }
        }
        if constexpr (EPI == EPI_STORE) return;
    } else {
        if (active) {
            using CIO = SpinorIO<(P == HR_F64 ? HR_F64 : HR_F32), D>;
            const R alpha = (R)prm.state[rhs].alpha;
            const R psc = (R)SIO::ld_scale(prm.p, rhs, i);
#pragma unroll
            for (int s = 0; s < 4; s++) {
                cx<R> rr[D], xx[D], pp[D];
                CIO::load_spin(prm.r, rhs, i, s, (R)1, rr);
                CIO::load_spin(prm.x, rhs, i, s, (R)1, xx);
                SIO::load_spin(prm.p, rhs, i, s, psc, pp);
#pragma unroll
                for (int c = 0; c < DR; c++) {
                    const int cc = part * DR + c;
                    rr[cc] = rr[cc] - alpha * acc[s][c];
                    xx[cc] = xx[cc] + alpha * pp[cc];
                    red += (double)(rr[cc].re * rr[cc].re + rr[cc].im * rr[cc].im);
                    char *er = prm.r.data + (size_t)rhs * prm.r.rhs_stride + (size_t)i * CIO::BYTES +
                               (size_t)(s * D + cc) * prec_cbytes(P == HR_F64 ? HR_F64 : HR_F32);
                    char *ex = prm.x.data + (size_t)rhs * prm.x.rhs_stride + (size_t)i * CIO::BYTES +
                               (size_t)(s * D + cc) * prec_cbytes(P == HR_F64 ? HR_F64 : HR_F32);
                    if constexpr (P == HR_F64) {
                        *reinterpret_cast<double2 *>(er) = make_double2(rr[cc].re, rr[cc].im);
                        *reinterpret_cast<double2 *>(ex) = make_double2(xx[cc].re, xx[cc].im);
                    } else {
                        *reinterpret_cast<float2 *>(er) = make_float2(rr[cc].re, rr[cc].im);
                        *reinterpret_cast<float2 *>(ex) = make_float2(xx[cc].re, xx[cc].im);
                    }
                }
            }
        }
    }
    double v[1] = {red};
    double tot[1];
    if (grid_reduce<1>(v, prm.partials + (size_t)rhs * gridDim.x, prm.counters + rhs, gridDim.x, blockIdx.x, tot))
        hop_finalize(prm, rhs, tot[0]);
}

}  // namespace hr
