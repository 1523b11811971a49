// hr_dslash_colour.cu -- explicit instantiation of the colour-parallel
// hopping kernel for one (N, representation, precision) of the pairs it
// serves.  The build compiles this file once per combination with
// -DHR_INST_N=<N> -DHR_INST_REP=<rep> -DHR_INST_P=<prec>.
#include "hr_dslash_colour.cuh"

namespace hr {

template hr_status launch_colour<HR_INST_N, HR_INST_REP, HR_INST_P>(const HopParams &, int, cudaStream_t);

}  // namespace hr
