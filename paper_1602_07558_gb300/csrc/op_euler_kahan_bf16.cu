// Instantiation unit: the Euler system in binary32 with a Kahan-compensated update, bfloat16
// storage (single grid; one translation unit per update, as each is built for several tile
// sides).
#include "launch.cuh"

namespace swept {
const OpTable *optable_euler_kahan_bf16() { return Launch<EulerKahanOp<__nv_bfloat16>>::table(); }
}  // namespace swept
