// Interleaved 2D demag kernels, configuration CfgF16h (FP32, radix 16, 384 threads, two blocks per SM).
#include "k_demag_il.cuh"

namespace mmc {

template void launch_il<CfgF16h>(const Launch &L, const DemagLaunch &P, DemagArgs<float> A);
template cudaError_t il_set_smem<CfgF16h>(int bytes);

}  // namespace mmc
