// Instantiation unit: the Section 3.1 increment example and the test updates
// (hash, level tag, eq. (complex_step) as two sub-steps), and the leapfrog
// wave equation of Section 6.
#include "launch.cuh"

namespace swept {
const OpTable *optable_increment() { return Launch<IncrementOp>::table(); }
const OpTable *optable_hash() { return Launch<HashOp>::table(); }
const OpTable *optable_leveltag() { return Launch<LevelTagOp>::table(); }
const OpTable *optable_wide2() { return Launch<Wide2Op>::table(); }
const OpTable *optable_wave() { return Launch<WaveOp>::table(); }
}  // namespace swept
