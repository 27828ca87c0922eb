// Instantiation unit: heat with a Kahan-compensated binary32 update, bfloat16 storage (single
// grid; one translation unit per update, as each is built for several tile sides).
#include "launch.cuh"

namespace swept {
const OpTable *optable_heat_kahan_bf16() { return Launch<HeatKahanOp<__nv_bfloat16>>::table(); }
}  // namespace swept
