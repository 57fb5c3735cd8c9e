// Interleaved 2D demag kernels, configuration CfgF32 (FP32, radix 32, 384 threads).
#include "k_demag_il.cuh"

namespace mmc {

template void launch_il<CfgF32>(const Launch &L, const DemagLaunch &P, DemagArgs<float> A);
template cudaError_t il_set_smem<CfgF32>(int bytes);

}  // namespace mmc
