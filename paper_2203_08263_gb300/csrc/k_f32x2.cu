// Plain FP32 force sum, packed f32x2 arithmetic.
#include "force_inst.cuh"

namespace nb {
static const ForceEntry kTable[] = {
    NB_ENTRY(AccelF32x2, 128, 1), NB_ENTRY(AccelF32x2, 128, 2), NB_ENTRY(AccelF32x2, 128, 4),
    NB_ENTRY(AccelF32x2, 128, 8), NB_ENTRY(AccelF32x2, 256, 2), NB_ENTRY(AccelF32x2, 256, 4),
    NB_ENTRY(AccelF32x2, 256, 8),
};
const ForceEntry *table_f32x2(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace nb
