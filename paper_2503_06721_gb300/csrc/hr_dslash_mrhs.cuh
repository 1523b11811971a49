// hr_dslash_mrhs.cuh -- the hopping kernel for a block of right-hand sides
// sharing each loaded link record.
//
// One block of 4 warps serves one 32-site tile for 4 right-hand sides: warp
// w computes right-hand side 4g + w of the tile's sites.  The tile's link
// records of hop k+1 (one contiguous block per slot in the AoSoA layout) are
// copied once into shared memory by all 128 threads while hop k is computed,
// and all four warps read them there, so the links cross L2 and HBM once per
// 4 right-hand sides instead of once per right-hand side.  The neighbour
// spinors and the output / CG-update records of each warp move through
// shared memory as in hop_staged_kernel, but through one buffer per warp:
// as soon as hop k's half-spinors are in registers the buffer takes the
// gather of hop k+1, which then overlaps hop k's link products.  With one
// spinor buffer a block takes 45 KB of shared memory (complex 2AS, FP32),
// so 4 blocks (16 warps) fit an SM and the register budget is 128; with two
// buffers 3 blocks did (ncu: 12 warps per SM, issue- and latency-bound).  Consecutive blocks are the
// right-hand-side groups of one tile, so the other groups find the tile's
// links in L2.  The arithmetic per site equals hop_kernel, bit for bit.
//
// Fused reductions are per right-hand side: each warp adds its tile's
// partial, and the last warp to arrive for a right-hand side (atomic ticket,
// no spin-wait) sums the tile partials in a fixed order in double-double.
#pragma once

#include "hr_dslash_staged.cuh"

namespace hr {

constexpr int MRHS_WARPS = 4;   // right-hand sides per block

template <int P, int D, int EPI, int LCH>
struct MrhsShape {
    using SS = StageShape<P, D, EPI>;
    static constexpr int SU = SS::SU;
    static constexpr int BUF = SS::BUF;            // chunks per warp spinor buffer
    static constexpr int LBUF = LCH * 32;          // chunks per block link buffer
    static constexpr size_t SMEM = ((size_t)MRHS_WARPS * BUF + 2 * LBUF) * 16;
};

// warp-level grid reduction of one value per right-hand side over `nparts`
// contributions; returns true in lane 0 of the last warp to arrive, with the
// total in tot.  partials: [nparts] for this right-hand side; counter: one
// unsigned, reset to 0 by the last warp.
__device__ inline bool warp_grid_reduce(double v, double *partials, unsigned *counter, long nparts, long part,
                                        double &tot)
{
    const int lane = threadIdx.x & 31;
    double vv[1] = {v};
    warp_sum<1>(vv);
    unsigned last = 0;
    if (lane == 0) {
        partials[part] = vv[0];
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        last = prev == (unsigned)(nparts - 1);
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return false;
    __threadfence();
    double hi = 0, lo = 0;
    for (long p = lane; p < nparts; p += 32) {
        double s, e;
        two_sum(hi, __ldcg(&partials[p]), s, e);
        hi = s;
        lo += e;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double h2 = __shfl_down_sync(0xffffffffu, hi, off);
        const double l2 = __shfl_down_sync(0xffffffffu, lo, off);
        double s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo += l2 + e;
    }
    if (lane == 0) {
        tot = hi + lo;
        *counter = 0;
    }
    return lane == 0;
}

template <int N, int REP, int P, bool REBUILD, int EPI, int MINB = 1>
__global__ void __launch_bounds__(128, MINB) hop_mrhs_kernel(const HopParams prm)
{
    using S = St<P>;
    using R = typename S::R;
    constexpr int D = rep_dim(N, REP);
    constexpr bool REAL = rep_real(REP) && !REBUILD;
    constexpr int NCOMP = REBUILD ? N * N : D * D;
    using SIO = SpinorIO<P, D>;
    using LIO = LinkIO<P, REAL, NCOMP>;
    using Sh = MrhsShape<P, D, EPI, LIO::NCHUNK>;
    constexpr int NC = SpinorIO<P, D>::NV, SU = Sh::SU;

    extern __shared__ uint4 mrhs_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint4 *const buf = mrhs_smem + (size_t)warp * Sh::BUF;   // the warp's record buffer
    uint4 *const own = buf + lane * SU;                        // this lane's record in it
    uint4 *const lbase = mrhs_smem + (size_t)MRHS_WARPS * Sh::BUF;
    auto lbuf = [&](int g) { return lbase + (g % 2) * Sh::LBUF; };

    const Geom &g = prm.g;
    const int ngroups = (prm.nrhs + MRHS_WARPS - 1) / MRHS_WARPS;
    const long tile = blockIdx.x / ngroups;
    const int rhs_raw = (int)(blockIdx.x % ngroups) * MRHS_WARPS + warp;
    // warps past the last right-hand side, or whose right-hand side has
    // converged, still copy links and meet every barrier, but compute nothing
    const int rhs = rhs_raw < prm.nrhs ? rhs_raw : prm.nrhs - 1;
    const bool work = rhs_raw < prm.nrhs && !(prm.state && cg_idle(prm.state[rhs]));
    const long i = tile * HR_TILE + lane;
    const long wfirst = tile * HR_TILE;
    const bool active = i < g.vh;
    const long ie = active ? i : g.vh - 1;
    const R sg = prm.dagger ? (R)-1 : (R)1;
    const char *in_base = prm.in.data + (size_t)rhs * prm.in.rhs_stride;
    const Site st = site_of(g, ie, prm.out_parity);
    const uint64_t lpol = policy_evict_first();

    // the tile's records of slot kk, by all threads of the block; the last
    // right-hand-side group of the tile reads them for the last time
    const bool last_group = (int)(blockIdx.x % ngroups) == ngroups - 1;
    auto copy_links = [&](int kk) {
        const uint4 *src = LIO::slot_ptr(prm.links, tile, kk, 0);
        uint4 *dst = lbuf(kk);
        for (int c = threadIdx.x; c < Sh::LBUF; c += blockDim.x) {
            if (last_group)
                cp_async16_hint(dst + c, src + c, lpol);
            else
                cp_async16(dst + c, src + c);
        }
    };
    auto gather_site = [&](int kk) {
        return kk < 8 ? (int)neighbour(g, st, kk & 3, kk < 4 ? +1 : -1) : (int)ie;
    };
    const char *diag_base = prm.diag.data ? prm.diag.data + (size_t)rhs * prm.diag.rhs_stride : nullptr;

    cx<R> acc[4][D];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < D; c++) acc[s][c] = {0, 0};

    // cp.async groups, per thread, in the order issued: [links 0 + gather 0],
    // then per hop k: [links k+1] at the top, [gather k+1 (or the diagonal)]
    // once hop k's half-spinors are in registers.  At the top of hop k the
    // wait for all but the newest group therefore means: gather k and links k
    // have landed.
    R scale_cur;
    {
        const int site = gather_site(0);
        scale_cur = (R)SIO::ld_scale(prm.in, rhs, site);
        if (work) warp_gather<NC, SU>(buf, in_base, site, lane);
        copy_links(0);
        cp_async_commit();
    }
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int mu = k & 3;
        const bool fwd = k < 4;
        if (k + 1 < 8) copy_links(k + 1);   // into the buffer hop k-1 used (all warps are past it)
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();   // hop k's links (copied by all warps) and spinors have landed
        const R sc = scale_cur;
        const R sp = fwd ? -sg : sg;
        cx<R> h[2][D];
        if (work) {
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < D; c++) {
                    // F16/BF16: codes as stored; the scale sc enters in the accumulation
                    const cx<R> up = rec_comp<P>(own, r * D + c);
                    const cx<R> dn = rec_comp<P>(own, (2 + eperm(mu, r)) * D + c);
                    h[r][c] = up + sp * ipow(ephase(mu, r), dn);
                }
        }
        __syncwarp();   // every lane has its half-spinors: the buffer takes the next gather
        {
            const int q = k + 1;
            if (q < 8) {
                const int site = gather_site(q);
                scale_cur = (R)SIO::ld_scale(prm.in, rhs, site);
                if (work) warp_gather<NC, SU>(buf, in_base, site, lane);
            } else if (diag_base && work) {
                warp_gather<NC, SU>(buf, diag_base, (int)ie, lane);
            }
            cp_async_commit();
        }
        if (work) {
            cx<R> chi[2][D];
            const uint4 *lp = lbuf(k) + lane;
            if constexpr (REBUILD) {
                cx<R> Wf[N * N];
                LIO::load_shared(lp, Wf);
                cx<R> F[N][N];
#pragma unroll
                for (int a = 0; a < N; a++)
#pragma unroll
                    for (int b = 0; b < N; b++) F[a][b] = Wf[a * N + b];
                rep_act<N, REP, R>(F, h[0], chi[0]);
                rep_act<N, REP, R>(F, h[1], chi[1]);
                const int xc = st.c[mu];
                const int L = mu == 0 ? g.T : mu == 1 ? g.X : mu == 2 ? g.Y : g.Z;
                if (g.bc[mu] == -1 && (fwd ? xc == L - 1 : xc == 0)) {
#pragma unroll
                    for (int r = 0; r < 2; r++)
#pragma unroll
                        for (int c = 0; c < D; c++) chi[r][c] = (R)-1 * chi[r][c];
                }
            } else {
#pragma unroll
                for (int row = 0; row < D; row++) {
                    cx<R> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
                    for (int col = 0; col < D; col++) {
                        const int cc = row * D + col;
                        const uint4 v = lp[(cc / LIO::VPC) * HR_TILE];
                        if constexpr (REAL) {
                            const R w = LIO::runpack(v, cc % LIO::VPC);
                            rmac(s0, w, h[0][col]);
                            rmac(s1, w, h[1][col]);
                        } else {
                            const cx<R> w = LIO::cunpack(v, cc % LIO::VPC);
                            cmac(s0, w, h[0][col]);
                            cmac(s1, w, h[1][col]);
                        }
                    }
                    chi[0][row] = s0;
                    chi[1][row] = s1;
                    asm volatile("" ::: "memory");
                }
            }
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < D; c++) {
                    if constexpr (S::scaled) {
                        acc_scaled(acc[r][c], sc, chi[r][c]);
                        acc_scaled(acc[2 + eperm(mu, r)][c], sc, sp * ipow(4 - ephase(mu, r), chi[r][c]));
                    } else {
                        acc[r][c] = acc[r][c] + chi[r][c];
                        acc[2 + eperm(mu, r)][c] = acc[2 + eperm(mu, r)][c] + sp * ipow(4 - ephase(mu, r), chi[r][c]);
                    }
                }
        }
        __syncthreads();   // every warp is done with hop k's links before hop k+2's refill them
    }
    cp_async_wait<0>();
    __syncwarp();
    if (!work) return;   // no barriers past this point

    const R a = (R)prm.a, b = (R)prm.b;
    if (prm.diag.data) {
        const R dsc = (R)SIO::ld_scale(prm.diag, rhs, ie);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) {
                cx<R> d = rec_comp<P>(own, s * D + c);
                if constexpr (S::scaled) d = scale_rn(dsc, d);
                acc[s][c] = axpby(a, acc[s][c], b, d);
            }
    } else {
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) acc[s][c] = a * acc[s][c];
    }
    __syncwarp();

    double *part = prm.partials + (size_t)rhs * g.ntiles;
    if constexpr (EPI == EPI_STORE || EPI == EPI_STORE_NORM) {
        R inv = 1;
        if constexpr (S::scaled) {
            R m = 0;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) m = fmaxf(m, fmaxf(fabsf(acc[s][c].re), fabsf(acc[s][c].im)));
            if (active) *(reinterpret_cast<float *>(prm.out.scale + (size_t)rhs * prm.out.rhs_stride) + i) = m;
            inv = m > 0 ? (R)1 / m : (R)0;
        }
        __syncwarp();   // every lane has read its diagonal record from the buffer
        rec_store<P, D>(own, acc, inv);
        __syncwarp();
        warp_scatter<NC, SU>(buf, prm.out.data + (size_t)rhs * prm.out.rhs_stride, wfirst, g.vh, lane);
        if constexpr (EPI == EPI_STORE) return;
        R n2 = 0;
        if (active) {
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) norm_acc(n2, acc[s][c]);
        }
        double tot;
        if (warp_grid_reduce((double)n2, part, prm.counters + rhs, g.ntiles, tile, tot)) hop_finalize(prm, rhs, tot);
    } else {
        constexpr int PC = StageShape<P, D, EPI>::PC;
        constexpr int NCC = StageShape<P, D, EPI>::NCC;
        using RC = typename St<PC>::R;
        constexpr int CPC = 16 / (int)prec_cbytes(PC);
        char *r_base = prm.r.data + (size_t)rhs * prm.r.rhs_stride;
        char *x_base = prm.x.data + (size_t)rhs * prm.x.rhs_stride;
        // r, then p, then x through the warp's one buffer
        warp_gather<NCC, SU>(buf, r_base, (int)ie, lane);
        cp_async_commit();
        const R alpha = (R)prm.state[rhs].alpha;
        R n2 = 0;
        cp_async_wait<0>();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NCC; j++) {
            uint4 v = own[j];
#pragma unroll
            for (int q = 0; q < CPC; q++) {
                const int n = j * CPC + q;
                cx<RC> rr = rec_comp<PC>(&v, q);
                rmac(rr, -alpha, acc[n / D][n % D]);
                norm_acc(n2, rr);
                if constexpr (PC == HR_F64) {
                    v = make_uint4((unsigned)__double2loint(rr.re), (unsigned)__double2hiint(rr.re),
                                   (unsigned)__double2loint(rr.im), (unsigned)__double2hiint(rr.im));
                } else if (q == 0) {
                    v.x = __float_as_uint(rr.re);
                    v.y = __float_as_uint(rr.im);
                } else {
                    v.z = __float_as_uint(rr.re);
                    v.w = __float_as_uint(rr.im);
                }
            }
            own[j] = v;
        }
        __syncwarp();
        warp_scatter<NCC, SU>(buf, r_base, wfirst, g.vh, lane);
        __syncwarp();
        warp_gather<NC, SU>(buf, prm.p.data + (size_t)rhs * prm.p.rhs_stride, (int)ie, lane);
        cp_async_commit();
        const R psc = (R)SIO::ld_scale(prm.p, rhs, ie);
        cp_async_wait<0>();
        __syncwarp();
        cx<R> pp[4 * D];
#pragma unroll
        for (int n = 0; n < 4 * D; n++) {
            pp[n] = rec_comp<P>(own, n);
            if constexpr (S::scaled) pp[n] = scale_rn(psc, pp[n]);
        }
        __syncwarp();
        warp_gather<NCC, SU>(buf, x_base, (int)ie, lane);
        cp_async_commit();
        cp_async_wait<0>();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NCC; j++) {
            uint4 v = own[j];
#pragma unroll
            for (int q = 0; q < CPC; q++) {
                const int n = j * CPC + q;
                cx<RC> xx = rec_comp<PC>(&v, q);
                rmac(xx, alpha, pp[n]);
                if constexpr (PC == HR_F64) {
                    v = make_uint4((unsigned)__double2loint(xx.re), (unsigned)__double2hiint(xx.re),
                                   (unsigned)__double2loint(xx.im), (unsigned)__double2hiint(xx.im));
                } else if (q == 0) {
                    v.x = __float_as_uint(xx.re);
                    v.y = __float_as_uint(xx.im);
                } else {
                    v.z = __float_as_uint(xx.re);
                    v.w = __float_as_uint(xx.im);
                }
            }
            own[j] = v;
        }
        __syncwarp();
        warp_scatter<NCC, SU>(buf, x_base, wfirst, g.vh, lane);
        double tot;
        if (warp_grid_reduce(active ? (double)n2 : 0.0, part, prm.counters + rhs, g.ntiles, tile, tot))
            hop_finalize(prm, rhs, tot);
    }
}

}  // namespace hr
