// Instantiation unit: heat with a Kahan-compensated binary32 update, binary32 storage (single
// grid; one translation unit per update, as each is built for several tile sides).
#include "launch.cuh"

namespace swept {
const OpTable *optable_heat_kahan_f32() { return Launch<HeatKahanOp<float>>::table(); }
}  // namespace swept
