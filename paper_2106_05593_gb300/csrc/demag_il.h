// Configurations and entry points of the interleaved 2D demag kernels
// (Sec. III, Eq. 14); the kernels themselves are in k_demag_il.cuh, compiled
// once per configuration in its own translation unit.
#pragma once

#include "demag_args.cuh"

namespace mmc {

// 2D fast path (Pz == 1): interleaved radix-16 transforms, E complex elements
// per block, V per thread (E / V threads).  The spectrum buffer is tiled by
// column groups of CC = E / (3 Py) columns: element (comp, y, kx) at
// ((comp * NG + kx / CC) * ny + y) * CC + kx % CC, NG = Sx / CC, so a row kernel
// block (2 E / (3 Px) consecutive rows) writes runs of rows * CC elements and a
// column kernel block reads and writes contiguous ny * CC runs.

// kernel configurations: E elements per block, V values per thread (E / V
// threads), MINB blocks per SM for the register budget.  The three FP32
// configurations (radix 16 with 768 threads; radix 32 with 384 threads; radix
// 16 with 384 threads, two blocks per SM) are timed against each other on the
// actual batch at create; FP64 uses radix 16 with 384 threads.
struct CfgF16 { using R = float; static constexpr int E = 12288, V = 16, MINB = 1; };
struct CfgF32 { using R = float; static constexpr int E = 12288, V = 32, MINB = 1; };
struct CfgD16 { using R = double; static constexpr int E = 6144, V = 16, MINB = 1; };
struct CfgF16h { using R = float; static constexpr int E = 6144, V = 16, MINB = 2; };

template <typename CFG>
void launch_il(const Launch &L, const DemagLaunch &P, DemagArgs<typename CFG::R> A);
template <typename CFG>
cudaError_t il_set_smem(int bytes);

}  // namespace mmc
