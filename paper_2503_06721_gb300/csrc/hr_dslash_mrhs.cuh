// hr_dslash_mrhs.cuh -- the hopping kernel for a block of right-hand sides
// that share one gauge field: every link is read from HBM once per
// application and reused by all right-hand sides.
//
// A CTA has one warp per right-hand side (lane = site of a 32-site tile) and
// walks a strided sequence of tiles.  For each (tile, slot) item, one thread
// brings the slot's link record (all 32 sites, 16-byte chunks) into a shared
// memory stage with a 1-D TMA bulk copy (evict-first L2 policy) that
// completes on the stage's "full" mbarrier; every warp reads the link from
// shared memory, gathers its own neighbour spinor from global memory, and
// arrives on the stage's "empty" mbarrier when done.  STAGES items are in
// flight.  All waits are bounded: a wait that exceeds the limit sets the
// error flag, drains, and the warp leaves.
// Per-rhs reductions are warp-level, with one ticket per (rhs, block) and the
// last warp for each rhs combining the per-block partials in a fixed order.
#pragma once

#include "hr_dslash.cuh"
#include "hr_tma.cuh"

namespace hr {

// right-hand sides per launch (one warp each): 8 in FP64, 12 otherwise, so
// the block's register budget covers the kernel without spills
constexpr int MRHS_STAGES = 4;
__host__ __device__ constexpr int mrhs_max(int P) { return P == HR_F64 ? 8 : 12; }

// warp-level grid reduction for one rhs: lane 0 of the last warp to arrive
// (over all blocks) returns true with the double-double total in tot
__device__ inline bool warp_grid_reduce(double v, double *partials, unsigned *counter, int nblocks, int block,
                                        double &tot)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31;
    unsigned last = 0;
    if (lane == 0) {
        partials[block] = v;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nblocks - 1;
    }
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return false;
    __threadfence();
    double hi = 0, lo = 0;
    for (int b = lane; b < nblocks; b += 32) {
        double s, e;
        two_sum(hi, __ldcg(&partials[b]), s, e);
        hi = s;
        lo += e;
    }
    // fixed-order combination of the 32 lane sums
    double H = 0, L = 0;
    for (int l = 0; l < 32; l++) {
        const double h = __shfl_sync(0xffffffffu, hi, l), q = __shfl_sync(0xffffffffu, lo, l);
        double s, e;
        two_sum(H, h, s, e);
        H = s;
        L += e + q;
    }
    if (lane == 0) {
        tot = H + L;
        *counter = 0;
    }
    return lane == 0;
}

template <int N, int REP, int P>
struct MrhsShape {
    static constexpr int D = rep_dim(N, REP);
    static constexpr bool REAL = rep_real(REP);
    static constexpr int NCHUNK = link_nchunk(P, REAL, D * D);
    static constexpr int STAGE_BYTES = NCHUNK * HR_TILE * 16;
    static constexpr size_t SMEM = (size_t)MRHS_STAGES * STAGE_BYTES;
};

template <int N, int REP, int P, int EPI>
__global__ void __launch_bounds__(mrhs_max(P) * 32) hop_mrhs_kernel(const HopParams prm, int *err)
{
    using Sh = MrhsShape<N, REP, P>;
    using S = St<P>;
    using R = typename S::R;
    constexpr int D = Sh::D;
    constexpr bool REAL = Sh::REAL;
    using SIO = SpinorIO<P, D>;
    using LIO = LinkIO<P, REAL, D * D>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t full[MRHS_STAGES], empty[MRHS_STAGES];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;   // right-hand sides in this launch
    const int rhs = warp;
    const Geom &g = prm.g;
    const bool idle = prm.state && cg_idle(prm.state[rhs]);   // per warp, fixed for the launch
    const long ntiles_mine = blockIdx.x < g.ntiles ? (g.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long nitems = ntiles_mine * 8;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MRHS_STAGES; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], nw);
        }
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t pol = policy_evict_first();
    bool ok = true;

    auto issue = [&](long j) {   // thread 0 only
        const int s = (int)(j % MRHS_STAGES);
        if (j >= MRHS_STAGES) {
            // the stage was used by item j - STAGES: wait until every warp released it
            if (!mbar_wait(&empty[s], (uint32_t)(((j / MRHS_STAGES) - 1) & 1))) return false;
        }
        const long tile = blockIdx.x + (j >> 3) * gridDim.x;
        const int slot = (int)(j & 7);
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[s], Sh::STAGE_BYTES);
        bulk_g2s(smem + (size_t)s * Sh::STAGE_BYTES,
                 reinterpret_cast<const uint4 *>(prm.links) + ((size_t)tile * 8 + slot) * Sh::NCHUNK * HR_TILE,
                 Sh::STAGE_BYTES, &full[s], pol);
        return true;
    };
    if (threadIdx.x == 0)
        for (long j = 0; j < MRHS_STAGES && j < nitems; j++)
            if (!issue(j)) { atomicExch(err, 1); ok = false; }

    const R sg = prm.dagger ? (R)-1 : (R)1;
    const R a = (R)prm.a, bcoef = (R)prm.b;
    double red = 0;
    cx<R> acc[4][D];
    Site st;
    for (long j = 0; j < nitems; j++) {
        const int s = (int)(j % MRHS_STAGES);
        const int slot = (int)(j & 7);
        const long tile = blockIdx.x + (j >> 3) * gridDim.x;
        const long i = tile * HR_TILE + lane;
        const bool active = i < g.vh && !idle;
        if (slot == 0) {
#pragma unroll
            for (int q = 0; q < 4; q++)
#pragma unroll
                for (int c = 0; c < D; c++) acc[q][c] = {0, 0};
            if (i < g.vh) st = site_of(g, i, prm.out_parity);
        }
        // neighbour spinor first (its latency overlaps the link wait)
        uint4 raw[SIO::NV];
        R sc = 1;
        if (active) {
            const long nb = neighbour(g, st, slot & 3, slot < 4 ? +1 : -1);
            const uint4 *pp = SIO::site_ptr(prm.in, rhs, nb);
#pragma unroll
            for (int q = 0; q < SIO::NV; q++) raw[q] = __ldg(pp + q);
            if constexpr (S::scaled) sc = (R)SIO::ld_scale(prm.in, rhs, nb);
        }
        if (!mbar_wait(&full[s], (uint32_t)((j / MRHS_STAGES) & 1))) {
            if (lane == 0) atomicExch(err, 1);
            ok = false;
        }
        if (active && ok) {
            const uint4 *Wp = reinterpret_cast<const uint4 *>(smem + (size_t)s * Sh::STAGE_BYTES) + lane;
            static_for<0, 8>([&](auto KK) {
                constexpr int k = decltype(KK)::value;
                if (slot != k) return;
                constexpr int mu = k & 3;
                const R sp_ = (k < 4) ? -sg : sg;
                cx<R> h[2][D];
#pragma unroll
                for (int r = 0; r < 2; r++)
#pragma unroll
                    for (int c = 0; c < D; c++) {
                        cx<R> up = SIO::comp(raw, r * D + c), dn = SIO::comp(raw, (2 + eperm(mu, r)) * D + c);
                        if constexpr (S::scaled) {
                            up = sc * up;
                            dn = sc * dn;
                        }
                        h[r][c] = up + sp_ * ipow(ephase(mu, r), dn);
                    }
#pragma unroll
                for (int row = 0; row < D; row++) {
                    cx<R> s0 = {0, 0}, s1 = {0, 0};
#pragma unroll
                    for (int col = 0; col < D; col++) {
                        const int cc = row * D + col;
                        const uint4 w = Wp[(cc / LIO::VPC) * HR_TILE];
                        if constexpr (REAL) {
                            const R wr = LIO::runpack(w, cc % LIO::VPC);
                            rmac(s0, wr, h[0][col]);
                            rmac(s1, wr, h[1][col]);
                        } else {
                            const cx<R> wc = LIO::cunpack(w, cc % LIO::VPC);
                            cmac(s0, wc, h[0][col]);
                            cmac(s1, wc, h[1][col]);
                        }
                    }
                    acc[0][row] = acc[0][row] + s0;
                    acc[1][row] = acc[1][row] + s1;
                    acc[2 + eperm(mu, 0)][row] = acc[2 + eperm(mu, 0)][row] + sp_ * ipow(4 - ephase(mu, 0), s0);
                    acc[2 + eperm(mu, 1)][row] = acc[2 + eperm(mu, 1)][row] + sp_ * ipow(4 - ephase(mu, 1), s1);
                }
            });
        }
        // release the stage, then thread 0 refills it with item j + STAGES
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (threadIdx.x == 0 && ok && j + MRHS_STAGES < nitems)
            if (!issue(j + MRHS_STAGES)) { atomicExch(err, 1); ok = false; }
        if (!__all_sync(0xffffffffu, ok)) ok = false;
        if (!ok) break;
        if (slot == 7 && active) {
            if (prm.diag.data) {
                cx<R> d[4][D];
                SIO::load(prm.diag, rhs, i, d);
#pragma unroll
                for (int q = 0; q < 4; q++)
#pragma unroll
                    for (int c = 0; c < D; c++) acc[q][c] = a * acc[q][c] + bcoef * d[q][c];
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++)
#pragma unroll
                    for (int c = 0; c < D; c++) acc[q][c] = a * acc[q][c];
            }
            if constexpr (EPI == EPI_STORE || EPI == EPI_STORE_NORM) {
                SIO::store(prm.out, rhs, i, acc);
                if constexpr (EPI == EPI_STORE_NORM) {
                    R n2 = 0;
#pragma unroll
                    for (int q = 0; q < 4; q++)
#pragma unroll
                        for (int c = 0; c < D; c++) n2 += acc[q][c].re * acc[q][c].re + acc[q][c].im * acc[q][c].im;
                    red += (double)n2;
                }
            } else {
                using CIO = SpinorIO<(P == HR_F64 ? HR_F64 : HR_F32), D>;
                const R alpha = (R)prm.state[rhs].alpha;
                const R psc = (R)SIO::ld_scale(prm.p, rhs, i);
                R n2 = 0;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    cx<R> rr[D], xx[D], pp[D];
                    CIO::load_spin(prm.r, rhs, i, q, (R)1, rr);
                    CIO::load_spin(prm.x, rhs, i, q, (R)1, xx);
                    SIO::load_spin(prm.p, rhs, i, q, psc, pp);
#pragma unroll
                    for (int c = 0; c < D; c++) {
                        rr[c] = rr[c] - alpha * acc[q][c];
                        xx[c] = xx[c] + alpha * pp[c];
                        n2 += rr[c].re * rr[c].re + rr[c].im * rr[c].im;
                    }
                    CIO::store_spin(prm.r, rhs, i, q, rr);
                    CIO::store_spin(prm.x, rhs, i, q, xx);
                }
                red += (double)n2;
            }
        }
    }
    if (!ok) {
        // drain: wait (bounded) for the copies this CTA may still have in flight
        if (threadIdx.x == 0)
            for (int s = 0; s < MRHS_STAGES; s++) mbar_wait(&full[s], 0), mbar_wait(&full[s], 1);
        return;
    }
    if constexpr (EPI != EPI_STORE) {
        if (!idle) {
            double tot;
            if (warp_grid_reduce(red, prm.partials + (size_t)rhs * gridDim.x, prm.counters + rhs, gridDim.x,
                                 blockIdx.x, tot))
                hop_finalize(prm, rhs, tot);
        }
    }
}

}  // namespace hr
