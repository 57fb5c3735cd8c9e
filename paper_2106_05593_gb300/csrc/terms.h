// Launcher of the per-term size of the trial moves (k_terms.cu).
#pragma once

#include "mmc_internal.h"

namespace mmc {

// blocks (and 6-double partials) the launch uses for a chain of `slots` slots per colour
int trial_terms_blocks(long long slots);

// sums over the cells of chain c of |dF_term| / kT (ex, dmi, an, zee, long, demag)
// into out[6]; part holds trial_terms_blocks(slots) x 6 doubles
void launch_trial_terms(const Launch &L, const ChainDev *chains, const ChainState *st, int c, long long slots,
                        bool percell, const float4 *m, const float4 *heff, const float4 *tab, unsigned sweep,
                        unsigned key0, unsigned key1, float omc_override, double *part, double *out);

}  // namespace mmc
