// hr_dslash_colour.cuh -- the colour-parallel ("D_R-site-parallel") hopping
// kernel for large representations.
//
// Sec. 8.2 (single-GPU efficiency) reports that a kernel holding a whole site per
// thread spills registers once the representation grows (large N, or a large
// D_R), and that a kernel in which each thread computes one colour
// component of one output site keeps the per-thread state small: the local
// work becomes D_R-length dot products of a link row with the projected
// neighbour spinor instead of D_R x D_R matrix-vector products.  It serves
// the fundamental of SU(5), SU(6), SU(8) and the SU(4) adjoint (D_R = 15, real
// links) and symmetric (D_R = 10) representations.
//
// Here a thread block is one 32-site tile times D_R colour rows.  For the
// link rows the threads are (row a, site j), site fastest, so every link-row
// load of a warp reads 32 consecutive lanes of the AoSoA link record; for
// the site-major spinors they are (site, colour), colour fastest, so that
// consecutive threads read and write consecutive numbers of one record.  Per
// hop each thread issues the loads of its neighbour-spinor colour and of the
// 16-byte chunks of its link row one hop ahead of their use (software
// pipelining), forms its component of the two projected half-spinors
// h_r = (1 -+ gamma_mu) psi in shared memory, and after a barrier forms
// chi_r[a] = sum_b U[a][b] h_r[b] of its own row and reconstructs its four
// spin components; the results return through shared memory to the spinor
// mapping for the stores.  Stored links only (the boundary
// signs are in the records), FP64 and FP32, epilogues store and
// store + |out|^2.
#pragma once

#include "hr_dslash.cuh"

namespace hr {

// resident blocks per SM asked of the register allocator in FP32: the
// largest count whose register cap does not make ptxas spill (D = 5: 5
// blocks of 160 threads at 72 registers; D = 6: 4 of 192; D = 8: 3 of 256,
// <= 80 registers; D = 10: 2 of 320), except D = 15: 2 blocks of 480 at 64
// registers with a small spill; FP64 unconstrained.  ncu on SU(5) at 4
// blocks: 20 warps per SM, stalled on the gathers (long scoreboard)
template <int D, int P>
constexpr int colour_minb() { return P == HR_F64 ? 1 : (D <= 5 ? 5 : D <= 6 ? 4 : D <= 8 ? 3 : 2); }

template <int N, int REP, int P, int EPI>
__global__ void __launch_bounds__(32 * rep_dim(N, REP), colour_minb<rep_dim(N, REP), P>())
    hop_colour_kernel(const HopParams prm)
{
    using R = typename St<P>::R;
    using C2 = typename std::conditional<P == HR_F64, double2, float2>::type;
    constexpr int D = rep_dim(N, REP);
    constexpr bool REAL = rep_real(REP);
    constexpr int RS = link_row_stride(N, REP, P);   // padded to whole chunks
    using LIO = LinkIO<P, REAL, D * RS>;
    const Geom &g = prm.g;
    const int rhs = blockIdx.y;
    if (prm.state && cg_idle(prm.state[rhs])) return;   // uniform per block
    const long tile = blockIdx.x;
    // link mapping (site fastest): thread = (row a, site j)
    const int j = threadIdx.x & 31;
    const int a = threadIdx.x >> 5;
    // spinor mapping (colour fastest): thread = (site jA, colour aA), so that
    // consecutive threads read and write consecutive numbers of one record
    const int jA = threadIdx.x / D;
    const int aA = threadIdx.x % D;
    const bool active = tile * HR_TILE + j < g.vh;
    const long iA = tile * HR_TILE + jA;
    const bool activeA = iA < g.vh;
    const R sg = prm.dagger ? (R)-1 : (R)1;
    constexpr int NC = 4 * D;                                 // complex numbers per spinor record
    constexpr int MAXC = (D + LIO::VPC - 1) / LIO::VPC;       // chunks a row takes
    // one padding column: the colour-fastest accesses of a warp (same site,
    // consecutive colours) then fall in different banks
    // the two half-spinor planes of the hop loop live in the first two planes
    // of the output buffer, which is only written after the loop's last barrier
    __shared__ cx<R> os[4][D][HR_TILE + 1];
    auto &hs = os;

    cx<R> acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    Site stA;
    if (activeA) stA = site_of(g, iA, prm.out_parity);
    const char *in = prm.in.data + (size_t)rhs * prm.in.rhs_stride;
    auto comp = [&](const char *base, long site, int s) -> cx<R> {
        const C2 v = *reinterpret_cast<const C2 *>(base + ((size_t)site * NC + (size_t)s * D + aA) * sizeof(C2));
        return {(R)v.x, (R)v.y};
    };
    // the row's elements e = a RS .. a RS + D - 1 lie in chunks c0 .. c0 + nch - 1
    // (RS a multiple of the chunk size: the row starts a chunk)
    const int e0 = a * RS, c0 = e0 / LIO::VPC, nch = (e0 + D - 1) / LIO::VPC - c0 + 1;
    // the loads of hop k: colour aA of site jA's neighbour, link row a of site j
    auto fetch = [&](int k, cx<R> (&psi)[4], uint4 (&lv)[MAXC]) {
        if (activeA) {
            const long nb = neighbour(g, stA, k & 3, k < 4 ? +1 : -1);
#pragma unroll
            for (int s = 0; s < 4; s++) psi[s] = comp(in, nb, s);
        }
        if (active) {
            const uint4 *lp = LIO::slot_ptr(prm.links, tile, k, j) + (size_t)c0 * HR_TILE;
#pragma unroll
            for (int cc = 0; cc < MAXC; cc++)
                if (cc < nch) lv[cc] = __ldg(lp + (size_t)cc * HR_TILE);
        }
    };
    cx<R> psi[2][4];
    uint4 lv[2][MAXC];
    fetch(0, psi[0], lv[0]);
    // software pipeline: the loads of hop k + 1 are in flight while hop k is formed
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int cur = k & 1;
        const int mu = k & 3;
        const bool fwd = k < 4;
        const R sp = fwd ? -sg : sg;
        if (activeA) {
#pragma unroll
            for (int r = 0; r < 2; r++)
                hs[r][aA][jA] = psi[cur][r] + sp * ipow(ephase(mu, r), psi[cur][2 + eperm(mu, r)]);
        }
        if (k + 1 < 8) fetch(k + 1, psi[cur ^ 1], lv[cur ^ 1]);
        __syncthreads();
        if (active) {
            cx<R> chi[2] = {{0, 0}, {0, 0}};
#pragma unroll
            for (int cc = 0; cc < MAXC; cc++) {
                if (cc >= nch) break;
#pragma unroll
                for (int q = 0; q < LIO::VPC; q++) {
                    const int b = (c0 + cc) * LIO::VPC + q - e0;
                    if (b < 0 || b >= D) continue;
                    if constexpr (REAL) {
                        const R u = LIO::runpack(lv[cur][cc], q);
                        rmac(chi[0], u, hs[0][b][j]);
                        rmac(chi[1], u, hs[1][b][j]);
                    } else {
                        const cx<R> u = LIO::cunpack(lv[cur][cc], q);
                        cmac(chi[0], u, hs[0][b][j]);
                        cmac(chi[1], u, hs[1][b][j]);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 2; r++) {
                acc[r] = acc[r] + chi[r];
                acc[2 + eperm(mu, r)] = acc[2 + eperm(mu, r)] + sp * ipow(4 - ephase(mu, r), chi[r]);
            }
        }
        __syncthreads();
    }
    // back to the spinor mapping for the epilogue and the coalesced stores
    if (active)
#pragma unroll
        for (int s = 0; s < 4; s++) os[s][a][j] = acc[s];
    __syncthreads();
    const R ca = (R)prm.a, cb = (R)prm.b;
    R n2 = 0;
    if (activeA) {
        cx<R> o[4];
#pragma unroll
        for (int s = 0; s < 4; s++) o[s] = os[s][aA][jA];
        if (prm.diag.data) {
            const char *dg = prm.diag.data + (size_t)rhs * prm.diag.rhs_stride;
#pragma unroll
            for (int s = 0; s < 4; s++) o[s] = axpby(ca, o[s], cb, comp(dg, iA, s));
        } else {
#pragma unroll
            for (int s = 0; s < 4; s++) o[s] = ca * o[s];
        }
        char *out = prm.out.data + (size_t)rhs * prm.out.rhs_stride;
#pragma unroll
        for (int s = 0; s < 4; s++) {
            C2 v;
            v.x = o[s].re;
            v.y = o[s].im;
            *reinterpret_cast<C2 *>(out + ((size_t)iA * NC + (size_t)s * D + aA) * sizeof(C2)) = v;
            norm_acc(n2, o[s]);
        }
    }
    if constexpr (EPI == EPI_STORE_NORM) {
        double v[1] = {(double)n2};
        double tot[1];
        if (grid_reduce<1>(v, prm.partials + (size_t)rhs * gridDim.x, prm.counters + rhs, gridDim.x, blockIdx.x, tot))
            hop_finalize(prm, rhs, tot[0]);
    }
}

template <int N, int REP, int P>
hr_status launch_colour(const HopParams &prm, int epi, cudaStream_t stream)
{
    constexpr int D = rep_dim(N, REP);
    const dim3 grid((unsigned)prm.g.ntiles, (unsigned)prm.nrhs);
    switch (epi) {
    case EPI_STORE: hop_colour_kernel<N, REP, P, EPI_STORE><<<grid, 32 * D, 0, stream>>>(prm); break;
    case EPI_STORE_NORM: hop_colour_kernel<N, REP, P, EPI_STORE_NORM><<<grid, 32 * D, 0, stream>>>(prm); break;
    default:
        set_error("the colour-parallel hopping kernel has no fused CG-update epilogue");
        return HR_ERR_UNSUPPORTED;
    }
    HR_LAUNCH_CHECK("hop_colour_kernel");
    return HR_OK;
}

}  // namespace hr
