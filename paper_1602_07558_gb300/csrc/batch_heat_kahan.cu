// Instantiation unit: the batched kernels of heat with a Kahan-compensated
// binary32 update, in binary32 and in bfloat16 storage.
#include "batch.cuh"

namespace swept {
const BatchTable *batchtable_heat_kahan_f32() { return BatchLaunch<HeatKahanOp<float>>::table(); }
const BatchTable *batchtable_heat_kahan_bf16() {
    return BatchLaunch<HeatKahanOp<__nv_bfloat16>>::table();
}
}  // namespace swept
