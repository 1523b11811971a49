// hr_dslash_staged.cuh -- the hopping kernel of hr_dslash.cuh with every
// site-record access of a warp staged through shared memory.
//
// Spinor records are site-major ([site][spin][colour], 32*D bytes per site in
// FP32), so when each lane reads its own neighbour's record a warp load
// instruction touches 32 different cache lines: the L1 data pipe, not DRAM,
// becomes the limit (ncu: l1tex__data_pipe_lsu_wavefronts near 90 % of peak
// for the adjoint at 55 % of DRAM peak).  Here the warp moves the 32 records
// it needs cooperatively: lane l copies 16-byte chunk (l + 32 j) of the
// concatenated records, so consecutive lanes read consecutive bytes of one
// record and a warp instruction touches 4-5 lines instead of 32.  The copies
// are cp.async (global -> shared without registers), double-buffered: the
// records of hop k+1 are in flight while hop k is computed from shared
// memory.  Records sit in shared memory at an odd multiple of 16 bytes apart,
// so each lane's 16-byte reads of its own record are free of bank conflicts.
// The output records (and, in the fused CG update, r, x and p, which are
// read and written at the warp's own 32 consecutive sites) take the same
// route in the other direction: lanes write their record to shared memory,
// and the warp stores the contiguous block of 32 records with coalesced
// 16-byte stores.  Link records are already lane-interleaved (a warp reads
// 512 contiguous bytes per instruction) and are loaded directly.
//
// The arithmetic per site is that of hop_kernel (same projection, products,
// reconstruction and epilogues), so results agree with it bit for bit.
#pragma once

#include "hr_dslash.cuh"
#include "hr_async.cuh"

namespace hr {

// shared-memory geometry of the staged kernel for (P, D, epilogue, pipeline
// depth, 16-byte chunks per link record when the links are staged too, else 0)
template <int P, int D, int EPI, int NST = 2, int LCH = 0>
struct StageShape {
    static constexpr int PC = (P == HR_F64 || P == HR_DF64) ? P : HR_F32;  // r, x precision (CG update)
    static constexpr int NC = SpinorIO<P, D>::NV;                          // 16-byte chunks per record
    static constexpr int NCC = SpinorIO<PC, D>::NV;
    static constexpr int NMAX = (EPI == EPI_CG_UPDATE && NCC > NC) ? NCC : NC;
    static constexpr int SU = (NMAX % 2) ? NMAX : NMAX + 1;   // record stride in chunks (odd)
    static constexpr int BUF = 32 * SU;                       // chunks per warp buffer
    static constexpr int LBUF = LCH * 32;                     // chunks per warp link buffer
    static constexpr int WARPS = 4;
    static constexpr size_t SMEM = (size_t)WARPS * NST * (BUF + LBUF) * 16;
};

// the records of the sites held by the 32 lanes (lane s holds site `site`)
// -> buf, record s at buf + s*SU; NCR chunks per record, record bytes 16*NCR
template <int NCR, int SU>
__device__ __forceinline__ void warp_gather(uint4 *buf, const char *base, int site, int lane)
{
#pragma unroll
    for (int j = 0; j < NCR; j++) {
        const int f = j * 32 + lane;
        const int s = f / NCR, c = f - s * NCR;
        const int src = __shfl_sync(0xffffffffu, site, s);
        cp_async16(buf + s * SU + c, base + ((size_t)src * NCR + c) * 16);
    }
}

// buf (record s at buf + s*SU) -> the contiguous records of sites
// first .. first+31, skipping sites >= limit
template <int NCR, int SU>
__device__ __forceinline__ void warp_scatter(const uint4 *buf, char *base, long first, long limit, int lane)
{
#pragma unroll
    for (int j = 0; j < NCR; j++) {
        const int f = j * 32 + lane;
        const int s = f / NCR, c = f - s * NCR;
        if (first + s < limit) reinterpret_cast<uint4 *>(base)[(first + s) * NCR + c] = buf[s * SU + c];
    }
}

// complex n of a record in precision P held as 16-byte chunks
template <int P>
__device__ __forceinline__ cx<typename St<P>::R> rec_comp(const uint4 *rec, int n)
{
    using S = St<P>;
    using R = typename S::R;
    if constexpr (P == HR_F64) {
        const uint4 v = rec[n];
        return {__hiloint2double((int)v.y, (int)v.x), __hiloint2double((int)v.w, (int)v.z)};
    } else if constexpr (P == HR_DF64) {
        const uint4 v = rec[n];
        return {df(__uint_as_float(v.x), __uint_as_float(v.y)), df(__uint_as_float(v.z), __uint_as_float(v.w))};
    } else if constexpr (P == HR_F32) {
        const uint4 v = rec[n >> 1];
        return (n & 1) ? cx<R>{__uint_as_float(v.z), __uint_as_float(v.w)}
                       : cx<R>{__uint_as_float(v.x), __uint_as_float(v.y)};
    } else {
        const uint4 v = rec[n >> 2];
        const unsigned w = (n & 3) == 0 ? v.x : (n & 3) == 1 ? v.y : (n & 3) == 2 ? v.z : v.w;
        typename S::C h;
        memcpy(&h, &w, 4);
        return S::ld(h);
    }
}

// acc (already multiplied by inv for scaled precisions) -> the lane's record
template <int P, int D>
__device__ __forceinline__ void rec_store(uint4 *rec, const cx<typename St<P>::R> (&acc)[4][D], typename St<P>::R inv)
{
    using S = St<P>;
    constexpr int NV = SpinorIO<P, D>::NV;
    uint4 raw[NV];
#pragma unroll
    for (int n = 0; n < 4 * D; n++) {
        const auto v = acc[n / D][n % D];
        if constexpr (P == HR_F64) {
            raw[n] = make_uint4((unsigned)__double2loint(v.re), (unsigned)__double2hiint(v.re),
                                (unsigned)__double2loint(v.im), (unsigned)__double2hiint(v.im));
        } else if constexpr (P == HR_DF64) {
            raw[n] = make_uint4(__float_as_uint(v.re.hi), __float_as_uint(v.re.lo), __float_as_uint(v.im.hi),
                                __float_as_uint(v.im.lo));
        } else if constexpr (P == HR_F32) {
            if (n & 1) {
                raw[n >> 1].z = __float_as_uint(v.re);
                raw[n >> 1].w = __float_as_uint(v.im);
            } else {
                raw[n >> 1].x = __float_as_uint(v.re);
                raw[n >> 1].y = __float_as_uint(v.im);
            }
        } else {
            typename S::C h = S::st(inv * v);
            unsigned w;
            memcpy(&w, &h, 4);
            if ((n & 3) == 0) raw[n >> 2].x = w;
            if ((n & 3) == 1) raw[n >> 2].y = w;
            if ((n & 3) == 2) raw[n >> 2].z = w;
            if ((n & 3) == 3) raw[n >> 2].w = w;
        }
    }
#pragma unroll
    for (int j = 0; j < NV; j++) rec[j] = raw[j];
}

// LST: the warp's link records of hop k+1 are copied to shared memory with
// the spinors (one contiguous 512-byte-per-chunk block per slot in the AoSoA
// layout), so both are in flight while hop k is computed and the links do not
// occupy registers until they are used.
template <int N, int REP, int P, bool REBUILD, int EPI, int MINB = 1, int NST = 2, bool LST = false>
__global__ void __launch_bounds__(128, MINB) hop_staged_kernel(const HopParams prm)
{
    using S = St<P>;
    using R = typename S::R;
    constexpr int D = rep_dim(N, REP);
    constexpr bool REAL = rep_real(REP) && !REBUILD;
    constexpr int NCOMP = REBUILD ? N * N : D * D;
    using SIO = SpinorIO<P, D>;
    using LIO = LinkIO<P, REAL, NCOMP>;
    using Sh = StageShape<P, D, EPI, NST, LST ? LIO::NCHUNK : 0>;
    static_assert(NST >= 2 && NST <= 4, "pipeline depth");
    constexpr int NC = Sh::NC, SU = Sh::SU;

    extern __shared__ uint4 stage_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // NST record buffers per warp; gather g (hops 0..7, then the diagonal
    // term's records as gather 8) lands in buffer g % NST
    uint4 *const wbuf = stage_smem + (size_t)warp * NST * (Sh::BUF + Sh::LBUF);
    auto buf = [&](int g) { return wbuf + (g % NST) * Sh::BUF; };
    auto own = [&](int g) { return wbuf + (g % NST) * Sh::BUF + lane * SU; };
    // link buffers after the spinor buffers; chunk j of lane l at [j * 32 + l]
    auto lbuf = [&](int g) { return wbuf + NST * Sh::BUF + (g % NST) * Sh::LBUF; };

    const Geom &g = prm.g;
    const int rhs = prm.rhs_inner ? (int)(blockIdx.x % prm.nrhs) : (int)blockIdx.y;
    const int bx = prm.rhs_inner ? (int)(blockIdx.x / prm.nrhs) : (int)blockIdx.x;
    const int nblk = prm.rhs_inner ? prm.nblk : (int)gridDim.x;
    if (prm.state && cg_idle(prm.state[rhs])) return;   // uniform per block
    const long i = (long)bx * blockDim.x + threadIdx.x;
    const long wfirst = i - lane;                        // first site of this warp
    const bool active = i < g.vh;
    // lanes past the end work on the last site (all loads stay in bounds) and store nothing
    const long ie = active ? i : g.vh - 1;
    const R sg = prm.dagger ? (R)-1 : (R)1;
    const char *in_base = prm.in.data + (size_t)rhs * prm.in.rhs_stride;

    const Site st = site_of(g, ie, prm.out_parity);
    const long tile = ie / HR_TILE;
    const int llane = (int)(ie % HR_TILE);
    // the warp's own tile (a block of 128 threads covers 4 whole tiles); a warp
    // entirely past the end copies the last tile's records and stores nothing
    const long wtile = min(wfirst / HR_TILE, g.ntiles - 1);
    const bool keep = prm.rhs_inner;   // other rhs re-read these links from L2
    uint64_t lpol = 0;
    if constexpr (LST) lpol = policy_evict_first();
    auto copy_links = [&](int kk) {
        if constexpr (LST) {
            const uint4 *src = LIO::slot_ptr(prm.links, wtile, kk, 0);
            uint4 *dst = lbuf(kk);
#pragma unroll
            for (int j = 0; j < LIO::NCHUNK; j++) {
                if (keep)
                    cp_async16(dst + j * 32 + lane, src + (size_t)j * HR_TILE + lane);
                else
                    cp_async16_hint(dst + j * 32 + lane, src + (size_t)j * HR_TILE + lane, lpol);
            }
        }
    };

    cx<R> acc[4][D];
#pragma unroll
    for (int s = 0; s < 4; s++)
#pragma unroll
        for (int c = 0; c < D; c++) acc[s][c] = {0, 0};

    // the neighbour of hop k (k < 8), or the own site for the diagonal records (k = 8)
    auto gather_site = [&](int kk) {
        return kk < 8 ? (int)neighbour(g, st, kk & 3, kk < 4 ? +1 : -1) : (int)ie;
    };
    const char *diag_base = prm.diag.data ? prm.diag.data + (size_t)rhs * prm.diag.rhs_stride : nullptr;
    if constexpr (EPI == EPI_CG_UPDATE) {
        // the fused update reads the warp's own r, x and p records only after
        // the eight hops: start bringing them into L2 now (the warp's 32
        // sites are contiguous records), so that the epilogue's gathers do not
        // wait on DRAM
        if (lane == 0 && wfirst < g.vh) {
            const long nw = min((long)HR_TILE, g.vh - wfirst);
            constexpr uint32_t RC = 16u * Sh::NCC, RP = 16u * NC;
            prefetch_l2_bulk(prm.r.data + (size_t)rhs * prm.r.rhs_stride + (size_t)wfirst * RC, (uint32_t)nw * RC);
            prefetch_l2_bulk(prm.x.data + (size_t)rhs * prm.x.rhs_stride + (size_t)wfirst * RC, (uint32_t)nw * RC);
            prefetch_l2_bulk(prm.p.data + (size_t)rhs * prm.p.rhs_stride + (size_t)wfirst * RP, (uint32_t)nw * RP);
        }
    }
    // gathers 0 .. NST-2 in flight before the first hop
    R scale_q[NST];
#pragma unroll
    for (int q = 0; q < NST - 1; q++) {
        const int site = gather_site(q);
        scale_q[q] = (R)SIO::ld_scale(prm.in, rhs, site);
        warp_gather<NC, SU>(buf(q), in_base, site, lane);
        copy_links(q);
        cp_async_commit();
    }

#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int mu = k & 3;
        const bool fwd = k < 4;
        {
            // keep NST-1 gathers ahead: issue gather k+NST-1 (one group per
            // iteration, empty past the end, so the wait below always means
            // "gather k has landed")
            const int q = k + NST - 1;
            if (q < 8) {
                const int site = gather_site(q);
                scale_q[q % NST] = (R)SIO::ld_scale(prm.in, rhs, site);
                warp_gather<NC, SU>(buf(q), in_base, site, lane);
                copy_links(q);
            } else if (q == 8 && diag_base) {
                warp_gather<NC, SU>(buf(8), diag_base, (int)ie, lane);
            }
            cp_async_commit();
            cp_async_wait<NST - 1>();
        }
        const R sc = scale_q[k % NST];
        __syncwarp();
        const R sp = fwd ? -sg : sg;
        cx<R> h[2][D];
        {
            const uint4 *rec = own(k);
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int c = 0; c < D; c++) {
                    // F16/BF16: codes as stored; the scale sc enters in the accumulation
                    const cx<R> up = rec_comp<P>(rec, r * D + c);
                    const cx<R> dn = rec_comp<P>(rec, (2 + eperm(mu, r)) * D + c);
                    h[r][c] = up + sp * ipow(ephase(mu, r), dn);
                }
        }
        cx<R> chi[2][D];
        const uint4 *lp = LST ? lbuf(k) + lane : LIO::slot_ptr(prm.links, tile, k, llane);
        auto load_links = [&](auto &W) {
            if constexpr (LST)
                LIO::load_shared(lp, W);
            else
                LIO::load(lp, W, keep);
        };
        if constexpr (REBUILD) {
            cx<R> Wf[N * N];
            load_links(Wf);
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
        } else if constexpr (LST) {
            // links from shared memory one row at a time (the compiler barrier
            // keeps the rows from being hoisted into one register-hungry block)
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
        } else if constexpr (REAL) {
            R W[D * D];
            load_links(W);
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
            load_links(W);
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
        __syncwarp();   // this hop's buffers are refilled by gather k+NST
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

    // epilogue: out = a * H + b * diag   (diagonal records in buffer 8 % NST)
    {
        const R a = (R)prm.a, b = (R)prm.b;
        if (prm.diag.data) {
            cp_async_wait<0>();
            __syncwarp();
            const R dsc = (R)SIO::ld_scale(prm.diag, rhs, ie);
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) {
                    cx<R> d = rec_comp<P>(own(8), s * D + c);
                    if constexpr (S::scaled) d = scale_rn(dsc, d);
                    acc[s][c] = axpby(a, acc[s][c], b, d);
                }
        } else {
#pragma unroll
            for (int s = 0; s < 4; s++)
#pragma unroll
                for (int c = 0; c < D; c++) acc[s][c] = a * acc[s][c];
        }
    }
    __syncwarp();

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
        rec_store<P, D>(own(7), acc, inv);
        __syncwarp();
        warp_scatter<NC, SU>(buf(7), prm.out.data + (size_t)rhs * prm.out.rhs_stride, wfirst, g.vh, lane);
        if constexpr (EPI == EPI_STORE) return;
        double v[1] = {0.0};
        if (active) {
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
        // fused CG update with out = A p:  r -= alpha A p, |r|^2;  x += alpha p
        constexpr int PC = Sh::PC;
        constexpr int NCC = Sh::NCC;
        using RC = typename St<PC>::R;
        constexpr int CPC = 16 / (int)prec_cbytes(PC);   // complex numbers per chunk of r, x
        char *r_base = prm.r.data + (size_t)rhs * prm.r.rhs_stride;
        char *x_base = prm.x.data + (size_t)rhs * prm.x.rhs_stride;
        // r in buffer 8 % NST (free once the diagonal term is consumed), x in 7 % NST
        warp_gather<NCC, SU>(buf(8), r_base, (int)ie, lane);
        cp_async_commit();
        warp_gather<NCC, SU>(buf(7), x_base, (int)ie, lane);
        cp_async_commit();
        const R alpha = (R)prm.state[rhs].alpha;
        R n2 = 0;
        cp_async_wait<1>();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NCC; j++) {
            uint4 v = own(8)[j];
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
            own(8)[j] = v;
        }
        __syncwarp();
        warp_scatter<NCC, SU>(buf(8), r_base, wfirst, g.vh, lane);
        __syncwarp();   // the scatter reads the buffer before p lands in it
        warp_gather<NC, SU>(buf(8), prm.p.data + (size_t)rhs * prm.p.rhs_stride, (int)ie, lane);
        cp_async_commit();
        const R psc = (R)SIO::ld_scale(prm.p, rhs, ie);
        cp_async_wait<0>();
        __syncwarp();
#pragma unroll
        for (int j = 0; j < NCC; j++) {
            uint4 v = own(7)[j];
#pragma unroll
            for (int q = 0; q < CPC; q++) {
                const int n = j * CPC + q;
                cx<RC> xx = rec_comp<PC>(&v, q);
                cx<R> pp = rec_comp<P>(own(8), n);
                if constexpr (S::scaled) pp = scale_rn(psc, pp);
                rmac(xx, alpha, pp);
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
            own(7)[j] = v;
        }
        __syncwarp();
        warp_scatter<NCC, SU>(buf(7), x_base, wfirst, g.vh, lane);
        double v[1] = {active ? (double)n2 : 0.0};
        double tot[1];
        if (grid_reduce<1>(v, prm.partials + (size_t)rhs * nblk, prm.counters + rhs, nblk, bx, tot))
            hop_finalize(prm, rhs, tot[0]);
    }
}

}  // namespace hr
