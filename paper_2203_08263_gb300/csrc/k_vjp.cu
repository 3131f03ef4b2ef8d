// Adjoint VJP of the force sum (plain FP32 and precision form).
#include "force_inst.cuh"

namespace nb {
// Shapes whose registers fit the 128-register cap without spilling.
static const ForceEntry kVjp[] = {
    NB_ENTRY(VjpF32x2, 128, 1), NB_ENTRY(VjpF32x2, 128, 2), NB_ENTRY(VjpF32x2, 256, 1),
    NB_ENTRY(VjpF32x2, 256, 2),
};
static const ForceEntry kVjpComp[] = {
    NB_ENTRY(VjpComp, 128, 1), NB_ENTRY(VjpComp, 256, 1),
};
const ForceEntry *table_vjp(int *count) {
    *count = (int)(sizeof(kVjp) / sizeof(kVjp[0]));
    return kVjp;
}
const ForceEntry *table_vjp_comp(int *count) {
    *count = (int)(sizeof(kVjpComp) / sizeof(kVjpComp[0]));
    return kVjpComp;
}
}  // namespace nb
