// Instantiation unit: heat and the Euler system with binary32 arithmetic and
// Kahan-compensated time accumulation, state stored in binary32 or bfloat16.
#include "launch.cuh"

namespace swept {
const OpTable *optable_heat_kahan_f32() { return Launch<HeatKahanOp<float>>::table(); }
const OpTable *optable_heat_kahan_bf16() { return Launch<HeatKahanOp<__nv_bfloat16>>::table(); }
const OpTable *optable_euler_kahan_f32() { return Launch<EulerKahanOp<float>>::table(); }
const OpTable *optable_euler_kahan_bf16() { return Launch<EulerKahanOp<__nv_bfloat16>>::table(); }
}  // namespace swept
