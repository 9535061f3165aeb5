// Prism kernels, double-word form, generic (convection-diffusion-reaction) kind.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_prism_dw_generic(int kind, int cpq, int inl, int outl) {
    FE_ALL8(FE_ELEM_CASE, 1, PRISM, DWORD, Q_PRISM6) FE_FN2(FE_ELEM_CASE, 1, PRISM, DWORD, Q_PRISM6)
    return nullptr;
}
const void *kernel_fixup_prism_dw_generic(int kind, int cpq, int inl, int outl) {
    FE_ALL8(FE_FIX_CASE, 1, PRISM, DWORD, Q_PRISM6) FE_FN2(FE_FIX_CASE, 1, PRISM, DWORD, Q_PRISM6)
    return nullptr;
}
}  // namespace fe
