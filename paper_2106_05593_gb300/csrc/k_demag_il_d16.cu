// Interleaved 2D demag kernels, configuration CfgD16 (FP64, radix 16).
#include "k_demag_il.cuh"

namespace mmc {

template void launch_il<CfgD16>(const Launch &L, const DemagLaunch &P, DemagArgs<double> A);
template cudaError_t il_set_smem<CfgD16>(int bytes);

}  // namespace mmc
