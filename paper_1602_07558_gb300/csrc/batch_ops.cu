// Instantiation unit: the batched kernels for the point updates that support
// batches (heat FP64, heat with compensated binary32 update in binary32 or
// bfloat16 storage, and the hash test update).
#include "batch.cuh"

namespace swept {
const BatchTable *batchtable_heat() { return BatchLaunch<HeatOp>::table(); }
const BatchTable *batchtable_heat_kahan_f32() { return BatchLaunch<HeatKahanOp<float>>::table(); }
const BatchTable *batchtable_heat_kahan_bf16() {
    return BatchLaunch<HeatKahanOp<__nv_bfloat16>>::table();
}
const BatchTable *batchtable_hash() { return BatchLaunch<HashOp>::table(); }
}  // namespace swept
