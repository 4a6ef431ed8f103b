// Explicit instantiation of the NTT_SCHEDULES_HUGE slice of the schedule
// list (kept in its own translation unit so slices compile in parallel).
#include "ntt_kernels.cuh"
#include "ntt_schedules.h"

namespace nttgb {
NTT_SCHEDULES_HUGE(NTT_INST_S1, NTT_INST_S2)
}  // namespace nttgb
