// Launcher of the angular-deviation histogram (k_angles.cu).
#pragma once

#include "mmc_internal.h"

namespace mmc {

void launch_angle_hist(const Launch &L, const ChainDev *chains, int c, long long slots, const float4 *m,
                       const double n[3], double lo, double hi, int bins, unsigned long long *hist);

}  // namespace mmc
