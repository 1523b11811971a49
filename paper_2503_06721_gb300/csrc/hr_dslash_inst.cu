// hr_dslash_inst.cu -- launcher and explicit instantiation of the hopping
// kernel for one (N, representation, precision).  The build compiles this
// file once per combination with -DHR_INST_N=<N> -DHR_INST_REP=<rep>
// -DHR_INST_P=<prec> so the instantiations compile in parallel.
#include "hr_dslash_mrhs.cuh"

namespace hr {

// register budget of the direct variant: F16/BF16 launches with D_R <= 4
// are held to 4 blocks of 128 threads per SM (128 registers, which they fit
// without spilling; ncu showed the unconstrained kernel at 168 registers and
// 12 warps per SM, stalled on its gathers); larger D_R spill at that cap and
// stay unconstrained, as do the other precisions
template <int N, int REP, int P>
constexpr int direct_minb() { return St<P>::scaled && rep_dim(N, REP) <= 4 ? 4 : 1; }

// register budget (resident blocks of 128 threads per SM) of a staged variant
template <int N, int REP>
constexpr int staged_minb(int variant)
{
    return rep_dim(N, REP) <= 4 ? 3 : (variant == HOP_STAGED ? 1 : 3);
}

// the staged kernel with staged links: as many blocks per SM as its shared
// memory allows (at most 4)
template <int N, int REP, int P, bool RB, int EPI>
constexpr int links_minb()
{
    constexpr int NCH = link_nchunk(P, rep_real(REP) && !RB, RB ? N * N : rep_dim(N, REP) * rep_dim(N, REP));
    constexpr size_t smem = StageShape<P, rep_dim(N, REP), EPI, 2, NCH>::SMEM + 8192;
    constexpr int b = (int)((size_t)227 * 1024 / smem);
    return b < 1 ? 1 : b > 4 ? 4 : b;
}

template <int N, int REP, int P, bool RB, int EPI, int MINB, bool LST = false>
static hr_status launch_staged(const HopParams &prm, dim3 grid, cudaStream_t stream)
{
    constexpr int NCH = link_nchunk(P, rep_real(REP) && !RB, RB ? N * N : rep_dim(N, REP) * rep_dim(N, REP));
    constexpr size_t smem = StageShape<P, rep_dim(N, REP), EPI, 2, LST ? NCH : 0>::SMEM;
    auto kern = hop_staged_kernel<N, REP, P, RB, EPI, MINB, 2, LST>;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return cuda_fail(attr, "cudaFuncSetAttribute(hop_staged_kernel)");
    kern<<<grid, 128, smem, stream>>>(prm);
    HR_LAUNCH_CHECK("hop_staged_kernel");
    return HR_OK;
}

template <int N, int REP, int P, bool RB, int MINB>
static hr_status launch_staged_epi(const HopParams &prm, int epi, dim3 grid, cudaStream_t stream)
{
    switch (epi) {
    case EPI_STORE: return launch_staged<N, REP, P, RB, EPI_STORE, MINB>(prm, grid, stream);
    case EPI_STORE_NORM: return launch_staged<N, REP, P, RB, EPI_STORE_NORM, MINB>(prm, grid, stream);
    case EPI_CG_UPDATE: return launch_staged<N, REP, P, RB, EPI_CG_UPDATE, MINB>(prm, grid, stream);
    default: set_error("bad epilogue %d", epi); return HR_ERR_INVALID;
    }
}

template <int N, int REP, int P, bool RB>
static hr_status launch_links_epi(const HopParams &prm, int epi, dim3 grid, cudaStream_t stream)
{
    switch (epi) {
    case EPI_STORE:
        return launch_staged<N, REP, P, RB, EPI_STORE, links_minb<N, REP, P, RB, EPI_STORE>(), true>(prm, grid, stream);
    case EPI_STORE_NORM:
        return launch_staged<N, REP, P, RB, EPI_STORE_NORM, links_minb<N, REP, P, RB, EPI_STORE_NORM>(), true>(
            prm, grid, stream);
    case EPI_CG_UPDATE:
        return launch_staged<N, REP, P, RB, EPI_CG_UPDATE, links_minb<N, REP, P, RB, EPI_CG_UPDATE>(), true>(
            prm, grid, stream);
    default: set_error("bad epilogue %d", epi); return HR_ERR_INVALID;
    }
}

template <int N, int REP, int P, bool RB, int EPI>
static hr_status launch_mrhs(const HopParams &prm, cudaStream_t stream)
{
    constexpr int NCH = link_nchunk(P, rep_real(REP) && !RB, RB ? N * N : rep_dim(N, REP) * rep_dim(N, REP));
    constexpr size_t smem = MrhsShape<P, rep_dim(N, REP), EPI, NCH>::SMEM;
    constexpr int b = (int)((size_t)227 * 1024 / (smem + 8192));
    // as many blocks as the shared memory allows (at most 4: 128 registers,
    // small spills with stored links); the in-kernel rebuild needs more
    // registers and keeps a budget of 2 blocks
    constexpr int bm = RB ? 2 : 4;
    constexpr int MINB = b < 1 ? 1 : b > bm ? bm : b;
    auto kern = hop_mrhs_kernel<N, REP, P, RB, EPI, MINB>;
    static const cudaError_t attr =
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (attr != cudaSuccess) return cuda_fail(attr, "cudaFuncSetAttribute(hop_mrhs_kernel)");
    const unsigned groups = (unsigned)((prm.nrhs + MRHS_WARPS - 1) / MRHS_WARPS);
    kern<<<(unsigned)prm.g.ntiles * groups, 32 * MRHS_WARPS, smem, stream>>>(prm);
    HR_LAUNCH_CHECK("hop_mrhs_kernel");
    return HR_OK;
}

template <int N, int REP, int P, bool RB>
static hr_status launch_epi(const HopParams &prm, int epi, int variant, cudaStream_t stream)
{
    if constexpr (P == HR_DF64) {
        // float-float is compiled for stored links and plain stores only (the
        // solver uses it for its FP64-class true residuals)
        if (RB || epi != EPI_STORE) {
            set_error("DF64 is available for stored links and plain applications only");
            return HR_ERR_UNSUPPORTED;
        }
    }
    constexpr unsigned mask = hop_variant_mask(N, REP, P);
    if (variant < 0 || variant >= HOP_NVARIANTS || !(mask & (1u << variant))) {
        set_error("hop kernel variant %d not compiled for this precision", variant);
        return HR_ERR_INVALID;
    }
    dim3 block(128);
    const unsigned nb = (unsigned)((prm.g.vh + 127) / 128);
    dim3 grid = prm.rhs_inner ? dim3(nb * (unsigned)prm.nrhs) : dim3(nb, (unsigned)prm.nrhs);
    if constexpr ((mask >> HOP_STAGED) & 1u) {
        if (variant == HOP_STAGED)
            return launch_staged_epi<N, REP, P, RB, staged_minb<N, REP>(HOP_STAGED)>(prm, epi, grid, stream);
    }
    if constexpr ((mask >> HOP_STAGED_TIGHT) & 1u) {
        if (variant == HOP_STAGED_TIGHT)
            return launch_staged_epi<N, REP, P, RB, staged_minb<N, REP>(HOP_STAGED_TIGHT)>(prm, epi, grid, stream);
    }
    if constexpr ((mask >> HOP_STAGED_LINKS) & 1u) {
        if (variant == HOP_STAGED_LINKS) return launch_links_epi<N, REP, P, RB>(prm, epi, grid, stream);
    }
    if constexpr ((mask >> HOP_MRHS) & 1u) {
        if (variant == HOP_MRHS) {
            if (prm.nrhs < 2) {
                set_error("the multi-RHS hop variant needs nrhs >= 2");
                return HR_ERR_INVALID;
            }
            switch (epi) {
            case EPI_STORE: return launch_mrhs<N, REP, P, RB, EPI_STORE>(prm, stream);
            case EPI_STORE_NORM: return launch_mrhs<N, REP, P, RB, EPI_STORE_NORM>(prm, stream);
            case EPI_CG_UPDATE: return launch_mrhs<N, REP, P, RB, EPI_CG_UPDATE>(prm, stream);
            default: set_error("bad epilogue %d", epi); return HR_ERR_INVALID;
            }
        }
    }
    if constexpr (P == HR_DF64) {
        if constexpr (!RB) hop_df64_kernel<N, REP><<<grid, block, 0, stream>>>(prm);
    } else {
        switch (epi) {
        case EPI_STORE: hop_kernel<N, REP, P, RB, EPI_STORE, direct_minb<N, REP, P>()><<<grid, block, 0, stream>>>(prm); break;
        case EPI_STORE_NORM:
            hop_kernel<N, REP, P, RB, EPI_STORE_NORM, direct_minb<N, REP, P>()><<<grid, block, 0, stream>>>(prm);
            break;
        case EPI_CG_UPDATE:
            hop_kernel<N, REP, P, RB, EPI_CG_UPDATE, direct_minb<N, REP, P>()><<<grid, block, 0, stream>>>(prm);
            break;
        default: set_error("bad epilogue %d", epi); return HR_ERR_INVALID;
        }
    }
    HR_LAUNCH_CHECK(P == HR_DF64 ? "hop_df64_kernel" : "hop_kernel");
    return HR_OK;
}

template <int N, int REP, int P>
hr_status launch_hop(const HopParams &prm, bool rebuild, int epi, int variant, cudaStream_t stream)
{
    return rebuild ? launch_epi<N, REP, P, true>(prm, epi, variant, stream)
                   : launch_epi<N, REP, P, false>(prm, epi, variant, stream);
}

template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_INST_P>(const HopParams &, bool, int, int, cudaStream_t);

}  // namespace hr
