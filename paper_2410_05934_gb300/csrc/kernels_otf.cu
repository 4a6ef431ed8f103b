// Explicit instantiation of the on-the-fly-twiddle configurations
// (NTT_OTF_CONFIGS), in their own translation unit so they compile in
// parallel with the schedule slices.
#include "ntt_kernels.cuh"
#include "ntt_schedules.h"

namespace nttgb {
NTT_OTF_CONFIGS(NTT_INST_S1, NTT_INST_S2)
}  // namespace nttgb
