// hr_dslash_inst.cu -- launcher and explicit instantiation of the hopping
// kernel for one (N, representation) pair.  The build compiles this file once
// per pair with -DHR_INST_N=<N> -DHR_INST_REP=<rep> so the instantiations
// compile in parallel.
#include "hr_dslash_mrhs.cuh"

namespace hr {

template <int N, int REP, int P, bool RB>
static hr_status launch_epi(const HopParams &prm, int epi, cudaStream_t stream)
{
    dim3 block(128);
    dim3 grid((unsigned)((prm.g.vh + 127) / 128), (unsigned)prm.nrhs);
    switch (epi) {
    case EPI_STORE: hop_kernel<N, REP, P, RB, EPI_STORE><<<grid, block, 0, stream>>>(prm); break;
    case EPI_STORE_NORM: hop_kernel<N, REP, P, RB, EPI_STORE_NORM><<<grid, block, 0, stream>>>(prm); break;
    case EPI_CG_UPDATE: hop_kernel<N, REP, P, RB, EPI_CG_UPDATE><<<grid, block, 0, stream>>>(prm); break;
    default: set_error("bad epilogue %d", epi); return HR_ERR_INVALID;
    }
    HR_LAUNCH_CHECK("hop_kernel");
    return HR_OK;
}

template <int N, int REP, int P>
hr_status launch_hop(const HopParams &prm, bool rebuild, int epi, cudaStream_t stream)
{
    return rebuild ? launch_epi<N, REP, P, true>(prm, epi, stream) : launch_epi<N, REP, P, false>(prm, epi, stream);
}

// multi-right-hand-side kernel: one CTA per group of tiles, one warp per rhs
template <int N, int REP, int P>
hr_status launch_hop_mrhs(const HopParams &prm, int epi, int *err, cudaStream_t stream)
{
    using Sh = MrhsShape<N, REP, P>;
    static int blocks_per_sm[3] = {0, 0, 0};   // per epilogue, for the largest block size
    auto kern = epi == EPI_STORE ? hop_mrhs_kernel<N, REP, P, EPI_STORE>
                : epi == EPI_STORE_NORM ? hop_mrhs_kernel<N, REP, P, EPI_STORE_NORM>
                                        : hop_mrhs_kernel<N, REP, P, EPI_CG_UPDATE>;
    if (blocks_per_sm[epi] == 0) {
        HR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM));
        int per = 0;
        HR_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, mrhs_max(P) * 32, Sh::SMEM));
        blocks_per_sm[epi] = per > 0 ? per : 1;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    long grid = (long)nsm * blocks_per_sm[epi];
    if (grid > prm.g.ntiles) grid = prm.g.ntiles;
    kern<<<(unsigned)grid, prm.nrhs * 32, Sh::SMEM, stream>>>(prm, err);
    HR_LAUNCH_CHECK("hop_mrhs_kernel");
    return HR_OK;
}

template hr_status launch_hop_mrhs<HR_INST_N, HR_INST_REP, HR_F64>(const HopParams &, int, int *, cudaStream_t);
template hr_status launch_hop_mrhs<HR_INST_N, HR_INST_REP, HR_F32>(const HopParams &, int, int *, cudaStream_t);
template hr_status launch_hop_mrhs<HR_INST_N, HR_INST_REP, HR_F16>(const HopParams &, int, int *, cudaStream_t);
template hr_status launch_hop_mrhs<HR_INST_N, HR_INST_REP, HR_BF16>(const HopParams &, int, int *, cudaStream_t);

template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_F64>(const HopParams &, bool, int, cudaStream_t);
template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_F32>(const HopParams &, bool, int, cudaStream_t);
template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_F16>(const HopParams &, bool, int, cudaStream_t);
template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_BF16>(const HopParams &, bool, int, cudaStream_t);

}  // namespace hr
