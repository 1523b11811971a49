// hr_dslash_tma.cuh -- the hopping kernel with an asynchronous shared-memory
// pipeline (stored links).
//
// Persistent: each warp owns a strided sequence of 32-site tiles and walks
// the (tile, slot) items in order.  For every item two transfers land in a
// per-warp stage buffer, STAGES - 1 items ahead of the compute:
//   * the slot's link record (NCOMP x 32 entries, one contiguous block) by a
//     1-D TMA bulk copy (cp.async.bulk) with an evict-first L2 policy,
//     completing on the stage's mbarrier;
//   * each lane's neighbour spinor by 16-byte cp.async gathers.
// Compute reads both from shared memory (conflict-free strides), so neither
// the link stream nor the spinor gather latency occupies registers.
// The arithmetic per hop is identical to hr_dslash.cuh.
#pragma once

#include "hr_dslash.cuh"
#include "hr_tma.cuh"

namespace hr {

template <int N, int REP, int P>
struct TmaShape {
    using S = St<P>;
    static constexpr int D = rep_dim(N, REP);
    static constexpr bool REAL = rep_real(REP);
    static constexpr int NCOMP = D * D;
    static constexpr int NCHUNK = link_nchunk(P, REAL, NCOMP);
    static constexpr int LINK_BYTES = NCHUNK * HR_TILE * 16;                     // one slot record
    static constexpr int SPIN_BYTES = 4 * D * (int)prec_cbytes(P);               // one site
    // per-lane stride: a multiple of 16 bytes that is an odd multiple of 16,
    // so 16-byte reads of eight consecutive lanes hit distinct banks
    static constexpr int LANE_STRIDE = ((SPIN_BYTES / 16) % 2 == 0) ? SPIN_BYTES + 16 : SPIN_BYTES;
    static constexpr int STAGE_BYTES = LINK_BYTES + HR_TILE * LANE_STRIDE;
};

template <int N, int REP, int P, int WARPS, int STAGES, int EPI>
__global__ void __launch_bounds__(WARPS * 32, 1) hop_tma_kernel(const HopParams prm, int *err)
{
    using Sh = TmaShape<N, REP, P>;
    using S = St<P>;
    using R = typename S::R;
    constexpr int D = Sh::D;
    constexpr bool REAL = Sh::REAL;
    using SIO = SpinorIO<P, D>;
    using LIO = LinkIO<P, REAL, D * D>;

    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem + (size_t)warp * STAGES * Sh::STAGE_BYTES;
    __shared__ uint64_t bars[WARPS][STAGES];

    const Geom &g = prm.g;
    const int rhs = blockIdx.y;
    if (prm.state && cg_idle(prm.state[rhs])) return;

    const long first = (long)blockIdx.x * WARPS + warp;
    const long step = (long)gridDim.x * WARPS;
    const long ntiles_mine = first < g.ntiles ? (g.ntiles - 1 - first) / step + 1 : 0;
    const long nitems = ntiles_mine * 8;

    if (lane == 0) {
        for (int s = 0; s < STAGES; s++) mbar_init(&bars[warp][s], 1);
        fence_mbar_init();
    }
    __syncwarp();
    const uint64_t pol = policy_evict_first();
    const char *in_base = prm.in.data + (size_t)rhs * prm.in.rhs_stride;

    auto issue = [&](long j) {
        const int s = (int)(j % STAGES);
        const long tile = first + (j >> 3) * step;
        const int slot = (int)(j & 7);
        unsigned char *sb = wbase + (size_t)s * Sh::STAGE_BYTES;
        if (lane == 0) {
            fence_proxy_async();
            mbar_arrive_expect_tx(&bars[warp][s], Sh::LINK_BYTES);
            const uint4 *src = reinterpret_cast<const uint4 *>(prm.links) + ((size_t)tile * 8 + slot) * Sh::NCHUNK * HR_TILE;
            bulk_g2s(sb, src, Sh::LINK_BYTES, &bars[warp][s], pol);
        }
        const long i = tile * HR_TILE + lane;
        if (i < g.vh) {
            Site st = site_of(g, i, prm.out_parity);
            const int mu = slot & 3;
            const long nb = neighbour(g, st, mu, slot < 4 ? +1 : -1);
            const char *src = in_base + (size_t)nb * Sh::SPIN_BYTES;
            unsigned char *dst = sb + Sh::LINK_BYTES + lane * Sh::LANE_STRIDE;
#pragma unroll
            for (int q = 0; q < Sh::SPIN_BYTES / 16; q++) cp_async16(dst + 16 * q, src + 16 * q);
        }
        cp_async_commit();
    };

    // prologue
    for (long j = 0; j < STAGES - 1; j++) {
        if (j < nitems)
            issue(j);
        else
            cp_async_commit();
    }

    const R sg = prm.dagger ? (R)-1 : (R)1;
    const R a = (R)prm.a, bcoef = (R)prm.b;
    double red = 0.0;
    bool ok = true;
    cx<R> acc[4][D];

    for (long j = 0; j < nitems && ok; j++) {
        if (j + STAGES - 1 < nitems)
            issue(j + STAGES - 1);
        else
            cp_async_commit();
        const int s = (int)(j % STAGES);
        const int slot = (int)(j & 7);
        const long tile = first + (j >> 3) * step;
        const long i = tile * HR_TILE + lane;
        const bool active = i < g.vh;
        cp_async_wait<STAGES - 1>();
        if (!mbar_wait(&bars[warp][s], (uint32_t)((j / STAGES) & 1))) {
            ok = false;
            if (lane == 0) atomicExch(err, 1);
            break;
        }
        if (slot == 0) {
#pragma unroll
            for (int q = 0; q < 4; q++)
#pragma unroll
                for (int c = 0; c < D; c++) acc[q][c] = {0, 0};
        }
        const unsigned char *sb = wbase + (size_t)s * Sh::STAGE_BYTES;
        if (active) {
            // neighbour spinor from this lane's slot
            const uint4 *sp = reinterpret_cast<const uint4 *>(sb + Sh::LINK_BYTES + lane * Sh::LANE_STRIDE);
            uint4 raw[SIO::NV];
#pragma unroll
            for (int q = 0; q < SIO::NV; q++) raw[q] = sp[q];
            R sc = 1;
            if constexpr (S::scaled) {
                Site st = site_of(g, i, prm.out_parity);
                const long nb = neighbour(g, st, slot & 3, slot < 4 ? +1 : -1);
                sc = (R)SIO::ld_scale(prm.in, rhs, nb);
            }
            const uint4 *Wp = reinterpret_cast<const uint4 *>(sb) + lane;
            // unrolled over the 8 slot values so mu and the projector are constants
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
        __syncwarp();
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
        // drain this warp's outstanding copies (bounded) before leaving
        cp_async_wait<0>();
        if (lane == 0)
            for (int s = 0; s < STAGES; s++) mbar_wait(&bars[warp][s], 0), mbar_wait(&bars[warp][s], 1);
        __syncwarp();
    }
    if constexpr (EPI != EPI_STORE) {
        double v[1] = {red};
        double tot[1];
        if (grid_reduce<1>(v, prm.partials + (size_t)rhs * gridDim.x, prm.counters + rhs, gridDim.x, blockIdx.x,
                           tot))
            hop_finalize(prm, rhs, tot[0]);
    }
}

template <int N, int REP, int P, int WARPS, int STAGES>
constexpr size_t tma_smem_bytes()
{
    return (size_t)WARPS * STAGES * TmaShape<N, REP, P>::STAGE_BYTES;
}

}  // namespace hr
