// Prism kernels, double-word form, Laplace kind with packed (upper-triangle) output.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_prism_dw_packed(int kind, int cpq, int inl, int outl) {
    FE_PK8(FE_ELEM_CASE, PRISM, DWORD, Q_PRISM6)
    return nullptr;
}
const void *kernel_fixup_prism_dw_packed(int kind, int cpq, int inl, int outl) {
    FE_PK8(FE_FIX_CASE, PRISM, DWORD, Q_PRISM6)
    return nullptr;
}
}  // namespace fe
