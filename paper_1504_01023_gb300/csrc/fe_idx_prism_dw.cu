// Prism kernels with INDEXED geometry (node table), double-word form.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_prism_dw_idx(int kind, int cpq, int outl) {
    const int inl = INDEXED;
    FE_IDX8(FE_ELEM_CASE, PRISM, DWORD, Q_PRISM6)
    return nullptr;
}
const void *kernel_fixup_prism_dw_idx(int kind, int cpq, int outl) {
    const int inl = INDEXED;
    FE_IDX8(FE_FIX_CASE, PRISM, DWORD, Q_PRISM6)
    return nullptr;
}
}  // namespace fe
