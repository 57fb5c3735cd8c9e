// Interleaved 2D demag kernels, configuration CfgF16 (FP32, radix 16, 768 threads).
#include "k_demag_il.cuh"

namespace mmc {

template void launch_il<CfgF16>(const Launch &L, const DemagLaunch &P, DemagArgs<float> A);
template cudaError_t il_set_smem<CfgF16>(int bytes);

}  // namespace mmc
