// Plain FP32 force sum, scalar arithmetic (comparison shape for the tuner).
#include "force_inst.cuh"

namespace nb {
static const ForceEntry kTable[] = {
    NB_ENTRY(AccelScalar, 128, 4), NB_ENTRY(AccelScalar, 256, 4), NB_ENTRY(AccelScalar, 256, 8),
};
const ForceEntry *table_scalar(int *count) {
    *count = (int)(sizeof(kTable) / sizeof(kTable[0]));
    return kTable;
}
}  // namespace nb
