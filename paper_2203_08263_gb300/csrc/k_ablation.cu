// Math-operation ablation of the force sum (sqrt + divide, powf).
#include "force_inst.cuh"

namespace nb {
static const ForceEntry kDiv[] = {
    NB_ENTRY(AccelMath<1>, 128, 4), NB_ENTRY(AccelMath<1>, 256, 4),
};
static const ForceEntry kPow[] = {
    NB_ENTRY(AccelMath<2>, 128, 4), NB_ENTRY(AccelMath<2>, 256, 4),
};
const ForceEntry *table_div(int *count) {
    *count = (int)(sizeof(kDiv) / sizeof(kDiv[0]));
    return kDiv;
}
const ForceEntry *table_pow(int *count) {
    *count = (int)(sizeof(kPow) / sizeof(kPow[0]));
    return kPow;
}
}  // namespace nb
