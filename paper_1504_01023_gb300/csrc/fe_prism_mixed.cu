// Prism kernels, mixed form (float arithmetic, double Jacobian fix-up).
#include "fe_inst.cuh"
namespace fe {
const void *kernel_prism_mixed(int kind, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_prism_mixed_idx(kind, cpq, outl);
    FE_ALL16(FE_ELEM_CASE, PRISM, MIXED, Q_PRISM6) FE_PK8(FE_ELEM_CASE, PRISM, MIXED, Q_PRISM6) FE_FN2(FE_ELEM_CASE, 0, PRISM, MIXED, Q_PRISM6) FE_FN2(FE_ELEM_CASE, 1, PRISM, MIXED, Q_PRISM6)
    return nullptr;
}
const void *kernel_fixup_prism(int kind, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_fixup_prism_idx(kind, cpq, outl);
    FE_ALL16(FE_FIX_CASE, PRISM, MIXED, Q_PRISM6) FE_PK8(FE_FIX_CASE, PRISM, MIXED, Q_PRISM6) FE_FN2(FE_FIX_CASE, 0, PRISM, MIXED, Q_PRISM6) FE_FN2(FE_FIX_CASE, 1, PRISM, MIXED, Q_PRISM6)
    return nullptr;
}
}  // namespace fe
