// Instantiation unit: the batched kernels of the Euler system in binary32 with a
// Kahan-compensated update, in binary32 and in bfloat16 storage.
#include "batch.cuh"

namespace swept {
const BatchTable *batchtable_euler_kahan_f32() {
    return BatchLaunch<EulerKahanOp<float>>::table();
}
const BatchTable *batchtable_euler_kahan_bf16() {
    return BatchLaunch<EulerKahanOp<__nv_bfloat16>>::table();
}
}  // namespace swept
