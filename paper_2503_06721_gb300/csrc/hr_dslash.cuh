// hr_dslash.cuh -- the Wilson hopping kernel (Eq. D_m^R, Sec. 2.3):
//
//   H psi(x) = sum_mu [ (1 - s g_mu) U_R(x,mu) psi(x+mu)
//                     + (1 + s g_mu) U_R(x-mu,mu)^dag psi(x-mu) ],
//   s = +1 for D, s = -1 for D^dag (gamma_mu Hermitian),
//
// evaluated for all sites of one output parity.  One thread owns one output
// site (and one right-hand side).  For each of the 8 hops it loads the
// neighbour spinor (16-byte vector loads, read-only path), projects it to the
// two-component half spinor h = up + s' e_mu dn, multiplies both components by
// the link (streamed from the AoSoA link record with evict-first loads, or
// rebuilt from the fundamental link in registers) and reconstructs the lower
// spin components as s' e_mu^dag (U h).  The epilogue forms
//   out = a * H(in) + b * diag
// and, depending on EPI, stores it, reduces |out|^2, or performs the fused CG
// update r -= alpha * out, x += alpha * p, |r|^2 without storing out.
#pragma once

#include "hr_fields.cuh"
#include "hr_rep.cuh"

namespace hr {

enum { EPI_STORE = 0, EPI_STORE_NORM = 1, EPI_CG_UPDATE = 2 };
enum { FIN_WRITE = 0, FIN_CG_ALPHA = 1, FIN_CG_BETA = 2 };

struct HopParams {
    Geom g;
    int out_parity;
    int dagger;
    const void *links;        // link records of the output parity
    FieldView in;             // opposite parity
    FieldView out;            // output parity (EPI_STORE*)
    FieldView diag;           // output parity, may have data == nullptr
    double a, b;
    int nrhs;
    // reductions
    double *partials;         // [nrhs][nblocks][1]
    unsigned *counters;       // [nrhs]
    double *red_out;          // [nrhs]   (FIN_WRITE)
    const double *carry;      // [nrhs] added to the total before finalising, or nullptr
    int fin;                  // FIN_WRITE / FIN_CG_ALPHA / FIN_CG_BETA
    CgState *state;           // [nrhs]   (CG epilogues; skip converged rhs)
    // right-hand-side-fastest block order: block b serves rhs b % nrhs and
    // site block b / nrhs, so the blocks of one site range run back to back
    // and every rhs after the first finds the links in L2
    int rhs_inner;
    int nblk;                 // site blocks per rhs
    // fused CG update (compute-type arrays, same layout as the fields)
    FieldView r, x, p;
};

// what the last block does with the grid total of a fused reduction
__device__ __forceinline__ void hop_finalize(const HopParams &prm, int rhs, double tot)
{
    if (prm.carry) tot += prm.carry[rhs];
    if (prm.fin == FIN_WRITE) {
        prm.red_out[rhs] = tot;
    } else if (prm.fin == FIN_CG_ALPHA) {
        CgState &cs = prm.state[rhs];
        cs.pAp = tot;
        cs.alpha = cs.rr / tot;
        if (!isfinite(cs.alpha) || tot <= 0.0) {
            cs.nonfinite = isfinite(tot) ? 0 : 1;
            cs.converged = 1;   // breakdown: stop this rhs, the host inspects it
            cs.alpha = 0;
        }
    } else {
        CgState &cs = prm.state[rhs];
        cs.iter += 1;
        if (!isfinite(tot)) {
            cs.nonfinite = 1;
            cs.converged = 1;
        } else {
            cs.beta = tot / cs.rr;
            cs.rr = tot;
            if (tot <= cs.stop2) cs.converged = 1;
        }
    }
}

template <int N, int REP, int P, bool REBUILD, int EPI, int MINB = 1>
__global__ void __launch_bounds__(128, MINB) hop_kernel(const HopParams prm)
{
    using S = St<P>;
    using R = typename S::R;
    constexpr int D = rep_dim(N, REP);
    constexpr bool REAL = rep_real(REP) && !REBUILD;
    constexpr int NCOMP = REBUILD ? N * N : D * D;
    using SIO = SpinorIO<P, D>;
    using LIO = LinkIO<P, REAL, NCOMP>;

    const Geom &g = prm.g;
    const int rhs = prm.rhs_inner ? (int)(blockIdx.x % prm.nrhs) : (int)blockIdx.y;
    const int bx = prm.rhs_inner ? (int)(blockIdx.x / prm.nrhs) : (int)blockIdx.x;
    const int nblk = prm.rhs_inner ? prm.nblk : (int)gridDim.x;
    if (prm.state && cg_idle(prm.state[rhs])) return;   // uniform per block
    const long i = (long)bx * blockDim.x + threadIdx.x;
    const bool active = i < g.vh;
    const R sg = prm.dagger ? (R)-1 : (R)1;

    cx<R> acc[4][D];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < D; c++) acc[s][c] = {0, 0};

    Site st;
    if (active) {
        st = site_of(g, i, prm.out_parity);
        const long tile = i / HR_TILE;
        const int lane = (int)(i % HR_TILE);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int mu = k & 3;
            const bool fwd = k < 4;
            const long nb = neighbour(g, st, mu, fwd ? +1 : -1);
            // projector (1 + sp gamma_mu): sp = -s forward, +s backward
            const R sp = fwd ? -sg : sg;
            // F16/BF16: the codes are projected and multiplied as stored; the
            // site scale sc enters once, in the accumulation below
            cx<R> psi[4][D];
            R sc = 1;
            if constexpr (S::scaled) {
                SIO::load_codes(prm.in, rhs, nb, psi);
                sc = (R)SIO::ld_scale(prm.in, rhs, nb);
            } else {
                SIO::load(prm.in, rhs, nb, psi);
            }
            cx<R> h[2][D];
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < D; c++)
                    h[r][c] = psi[r][c] + sp * ipow(ephase(mu, r), psi[2 + eperm(mu, r)][c]);
            cx<R> chi[2][D];
            const uint4 *lp = LIO::slot_ptr(prm.links, tile, k, lane);
            const bool keep = prm.rhs_inner;   // other rhs re-read these links from L2
            if constexpr (REBUILD) {
                cx<R> Wf[N * N];
                LIO::load(lp, Wf, keep);
                cx<R> F[N][N];
#pragma unroll
                for (int a = 0; a < N; a++)
#pragma unroll
                    for (int b = 0; b < N; b++) F[a][b] = Wf[a * N + b];
                rep_act<N, REP, R>(F, h[0], chi[0]);
                rep_act<N, REP, R>(F, h[1], chi[1]);
                // fermion boundary sign on the t = T-1 <-> 0 (etc.) hop
                const int xc = st.c[mu];
                const int L = mu == 0 ? g.T : mu == 1 ? g.X : mu == 2 ? g.Y : g.Z;
                if (g.bc[mu] == -1 && (fwd ? xc == L - 1 : xc == 0)) {
#pragma unroll
                    for (int r = 0; r < 2; r++)
#pragma unroll
                        for (int c = 0; c < D; c++) chi[r][c] = (R)-1 * chi[r][c];
                }
            } else if constexpr (REAL) {
                R W[D * D];
                LIO::load(lp, W, keep);
#pragma unroll
                for (int row = 0; row < D; row++) {
                    cx<R> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
                    for (int col = 0; col < D; col++) {
                        rmac(s0, W[row * D + col], h[0][col]);
                        rmac(s1, W[row * D + col], h[1][col]);
                    }
                    chi[0][row] = s0;
                    chi[1][row] = s1;
                }
            } else {
                cx<R> W[D * D];
                LIO::load(lp, W, keep);
#pragma unroll
                for (int row = 0; row < D; row++) {
                    cx<R> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
                    for (int col = 0; col < D; col++) {
                        cmac(s0, W[row * D + col], h[0][col]);
                        cmac(s1, W[row * D + col], h[1][col]);
                    }
                    chi[0][row] = s0;
                    chi[1][row] = s1;
                }
            }
            // reconstruct: upper += chi, lower_{eperm(r)} += sp i^{-ephase(r)} chi_r
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
        // epilogue: out = a * H + b * diag
        const R a = (R)prm.a, b = (R)prm.b;
        if (prm.diag.data) {
            cx<R> d[4][D];
            SIO::load(prm.diag, rhs, i, d);
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) acc[s][c] = axpby(a, acc[s][c], b, d[s][c]);
        } else {
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) acc[s][c] = a * acc[s][c];
        }
    }

    if constexpr (EPI == EPI_STORE) {
        if (active) SIO::store(prm.out, rhs, i, acc);
        return;
    } else if constexpr (EPI == EPI_STORE_NORM) {
        double v[1] = {0.0};
        if (active) {
            SIO::store(prm.out, rhs, i, acc);
            R n2 = 0;
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) norm_acc(n2, acc[s][c]);
            v[0] = (double)n2;
        }
        double tot[1];
        if (grid_reduce<1>(v, prm.partials + (size_t)rhs * nblk, prm.counters + rhs, nblk, bx, tot))
            hop_finalize(prm, rhs, tot[0]);
    } else {
        // fused CG update with out = A p:  x += alpha p;  r -= alpha A p;  |r|^2
        double v[1] = {0.0};
        if (active) {
            using CIO = SpinorIO<(P == HR_F64 ? HR_F64 : HR_F32), D>;
            const R alpha = (R)prm.state[rhs].alpha;
            const R psc = (R)SIO::ld_scale(prm.p, rhs, i);
            R n2 = 0;
            // one spin component at a time keeps r, x, p out of the register budget
#pragma unroll
            for (int s = 0; s < 4; s++) {
                cx<R> rr[D], xx[D], pp[D];
                CIO::load_spin(prm.r, rhs, i, s, (R)1, rr);
                CIO::load_spin(prm.x, rhs, i, s, (R)1, xx);
                SIO::load_spin(prm.p, rhs, i, s, psc, pp);
#pragma unroll
                for (int c = 0; c < D; c++) {
                    rmac(rr[c], -alpha, acc[s][c]);
                    rmac(xx[c], alpha, pp[c]);
                    norm_acc(n2, rr[c]);
                }
                CIO::store_spin(prm.r, rhs, i, s, rr);
                CIO::store_spin(prm.x, rhs, i, s, xx);
            }
            v[0] = (double)n2;
        }
        double tot[1];
        if (grid_reduce<1>(v, prm.partials + (size_t)rhs * nblk, prm.counters + rhs, nblk, bx, tot))
            hop_finalize(prm, rhs, tot[0]);
    }
}

// The float-float (DF64) hop, for stored links and a plain store.  Each df
// product-sum takes about 15 FP32 instructions, so with the 8 hops unrolled
// as in hop_kernel the code no longer fits the instruction caches (ncu: most
// issue slots stall on "no instruction").  Here the hop loop stays rolled:
// one hop body serves all 8 directions, with the direction-dependent spin
// permutation and phases chosen at run time (uniform across the warp).
template <int N, int REP>
__global__ void __launch_bounds__(128) hop_df64_kernel(const HopParams prm)
{
    using S = St<HR_DF64>;
    using R = typename S::R;
    constexpr int D = rep_dim(N, REP);
    constexpr bool REAL = rep_real(REP);
    using SIO = SpinorIO<HR_DF64, D>;
    using LIO = LinkIO<HR_DF64, REAL, D * D>;

    const Geom &g = prm.g;
    const int rhs = prm.rhs_inner ? (int)(blockIdx.x % prm.nrhs) : (int)blockIdx.y;
    const int bx = prm.rhs_inner ? (int)(blockIdx.x / prm.nrhs) : (int)blockIdx.x;
    const long i = (long)bx * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const R sg = prm.dagger ? (R)-1 : (R)1;
    cx<R> acc[4][D];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < D; c++) acc[s][c] = {0, 0};
    const Site st = site_of(g, i, prm.out_parity);
    const long tile = i / HR_TILE;
    const int lane = (int)(i % HR_TILE);
#pragma unroll 1
    for (int k = 0; k < 8; k++) {
        const int mu = k & 3;
        const bool fwd = k < 4;
        const long nb = neighbour(g, st, mu, fwd ? +1 : -1);
        const R sp = fwd ? -sg : sg;
        // lower spin component paired with upper r: 2 + r, or 3 - r for mu = 1, 2
        const bool swap = mu == 1 || mu == 2;
        const int ph0 = ephase(mu, 0), ph1 = ephase(mu, 1);
        cx<R> psi[4][D];
        SIO::load(prm.in, rhs, nb, psi);
        cx<R> h[2][D];
#pragma unroll
        for (int c = 0; c < D; c++) {
            const cx<R> dn0 = swap ? psi[3][c] : psi[2][c];
            const cx<R> dn1 = swap ? psi[2][c] : psi[3][c];
            h[0][c] = psi[0][c] + sp * ipow(ph0, dn0);
            h[1][c] = psi[1][c] + sp * ipow(ph1, dn1);
        }
        const uint4 *lp = LIO::slot_ptr(prm.links, tile, k, lane);
        cx<R> chi[2][D];
        if constexpr (REAL) {
            R W[D * D];
            LIO::load(lp, W);
#pragma unroll
            for (int row = 0; row < D; row++) {
                cx<R> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
                for (int col = 0; col < D; col++) {
                    rmac(s0, W[row * D + col], h[0][col]);
                    rmac(s1, W[row * D + col], h[1][col]);
                }
                chi[0][row] = s0;
                chi[1][row] = s1;
            }
        } else {
            cx<R> W[D * D];
            LIO::load(lp, W);
#pragma unroll
            for (int row = 0; row < D; row++) {
                cx<R> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
                for (int col = 0; col < D; col++) {
                    cmac(s0, W[row * D + col], h[0][col]);
                    cmac(s1, W[row * D + col], h[1][col]);
                }
                chi[0][row] = s0;
                chi[1][row] = s1;
            }
        }
#pragma unroll
        for (int c = 0; c < D; c++) {
            acc[0][c] = acc[0][c] + chi[0][c];
            acc[1][c] = acc[1][c] + chi[1][c];
            const cx<R> t0 = sp * ipow(4 - ph0, chi[0][c]);
            const cx<R> t1 = sp * ipow(4 - ph1, chi[1][c]);
            if (swap) {
                acc[3][c] = acc[3][c] + t0;
                acc[2][c] = acc[2][c] + t1;
            } else {
                acc[2][c] = acc[2][c] + t0;
                acc[3][c] = acc[3][c] + t1;
            }
        }
    }
    const R a = (R)prm.a, b = (R)prm.b;
    if (prm.diag.data) {
        cx<R> d[4][D];
        SIO::load(prm.diag, rhs, i, d);
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) acc[s][c] = axpby(a, acc[s][c], b, d[s][c]);
    } else {
#pragma unroll
        for (int s = 0; s < 4; s++)
#pragma unroll
            for (int c = 0; c < D; c++) acc[s][c] = a * acc[s][c];
    }
    SIO::store(prm.out, rhs, i, acc);
}

// Kernel variants of one hopping launch.  Every variant computes the same
// bits; which one is fastest depends on N, R, precision, link mode, epilogue,
// lattice and right-hand-side count, and the autotuner picks among them.
//   HOP_DIRECT        hop_kernel: each lane loads its own neighbour records
//   HOP_STAGED        hop_staged_kernel: warp-cooperative spinor gathers
//                     through shared memory, register budget for 2 (D_R > 4)
//                     or 3 (D_R <= 4) blocks of 128 threads per SM
//   HOP_STAGED_TIGHT  the same held to 3 blocks per SM (D_R > 4 only)
//   HOP_STAGED_LINKS  the staged kernel with the link records staged too
//   HOP_MRHS          hop_mrhs_kernel: a block of 4 right-hand sides shares
//                     each tile's link records (nrhs >= 2 only)
// FP64 and DF64 have the direct kernel only: they are bound by FP64 (or
// float-float) arithmetic, not by the memory system.
enum { HOP_DIRECT = 0, HOP_STAGED = 1, HOP_STAGED_TIGHT = 2, HOP_STAGED_LINKS = 3, HOP_MRHS = 4, HOP_NVARIANTS = 5 };
// bit v set: variant v is compiled for (N, REP, P)
__host__ __device__ constexpr unsigned hop_variant_mask(int N, int REP, int P)
{
    return (P == HR_F64 || P == HR_DF64) ? 0x1u : rep_dim(N, REP) <= 4 ? 0x1Bu : 0x1Fu;
}
// whether variant v can serve a launch of nrhs right-hand sides
__host__ __device__ constexpr bool hop_variant_fits(int v, int nrhs) { return v != HOP_MRHS || nrhs >= 2; }

// host-side launchers, instantiated per (N, REP, P) in hr_dslash_inst.cu
template <int N, int REP, int P>
hr_status launch_hop(const HopParams &prm, bool rebuild, int epi, int variant, cudaStream_t stream);


}  // namespace hr
