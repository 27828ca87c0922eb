// Instantiation unit: the Euler system in binary32 with a Kahan-compensated update, binary32
// storage (single grid; one translation unit per update, as each is built for several tile
// sides).
#include "launch.cuh"

namespace swept {
const OpTable *optable_euler_kahan_f32() { return Launch<EulerKahanOp<float>>::table(); }
}  // namespace swept
