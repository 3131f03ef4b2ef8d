// Compensated FP32 force sum (FP64 state) and the softened potential.
#include "force_inst.cuh"

namespace nb {
static const ForceEntry kComp[] = {
    NB_ENTRY(AccelComp, 128, 2), NB_ENTRY(AccelComp, 128, 4), NB_ENTRY(AccelComp, 256, 2),
    NB_ENTRY(AccelComp, 256, 4), NB_ENTRY(AccelComp, 256, 8),
};
static const ForceEntry kPot[] = {
    NB_ENTRY(Potential, 128, 2), NB_ENTRY(Potential, 256, 4),
};
const ForceEntry *table_comp(int *count) {
    *count = (int)(sizeof(kComp) / sizeof(kComp[0]));
    return kComp;
}
const ForceEntry *table_pot(int *count) {
    *count = (int)(sizeof(kPot) / sizeof(kPot[0]));
    return kPot;
}
}  // namespace nb
