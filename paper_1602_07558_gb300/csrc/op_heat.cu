// Instantiation unit: forward-Euler 5-point heat update.
#include "launch.cuh"

namespace swept {
const OpTable *optable_heat() { return Launch<HeatOp>::table(); }
}  // namespace swept
