// hr_dslash_inst.cu -- launcher and explicit instantiation of the hopping
// kernel for one (N, representation) pair.  The build compiles this file once
// per pair with -DHR_INST_N=<N> -DHR_INST_REP=<rep> so the instantiations
// compile in parallel.
#include "hr_dslash.cuh"

namespace hr {

template <int N, int REP, int P, bool RB>
static hr_status launch_epi(const HopParams &prm, int epi, cudaStream_t stream)
{
    dim3 block(128);
    const unsigned nb = (unsigned)((prm.g.vh + 127) / 128);
    dim3 grid = prm.rhs_inner ? dim3(nb * (unsigned)prm.nrhs) : dim3(nb, (unsigned)prm.nrhs);
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

template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_F64>(const HopParams &, bool, int, cudaStream_t);
template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_F32>(const HopParams &, bool, int, cudaStream_t);
template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_F16>(const HopParams &, bool, int, cudaStream_t);
template hr_status launch_hop<HR_INST_N, HR_INST_REP, HR_BF16>(const HopParams &, bool, int, cudaStream_t);

}  // namespace hr
