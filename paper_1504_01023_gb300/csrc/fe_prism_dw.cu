// Prism kernels, double-word form (double-accuracy results from float pipes;
// flagged elements redone in double): Laplace kind here (its packed outputs in
// fe_prism_dw_packed.cu), generic kind in fe_prism_dw_generic.cu (the units
// compile in parallel).
#include "fe_inst.cuh"
namespace fe {
const void *kernel_prism_dw_generic(int kind, int cpq, int inl, int outl);
const void *kernel_fixup_prism_dw_generic(int kind, int cpq, int inl, int outl);
const void *kernel_prism_dw_packed(int kind, int cpq, int inl, int outl);
const void *kernel_fixup_prism_dw_packed(int kind, int cpq, int inl, int outl);

const void *kernel_prism_dw(int kind, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_prism_dw_idx(kind, cpq, outl);
    if (out_packed(outl)) return kernel_prism_dw_packed(kind, cpq, inl, outl);
    FE_ALL8(FE_ELEM_CASE, 0, PRISM, DWORD, Q_PRISM6) FE_FN2(FE_ELEM_CASE, 0, PRISM, DWORD, Q_PRISM6)
    return kernel_prism_dw_generic(kind, cpq, inl, outl);
}
const void *kernel_fixup_prism_dw(int kind, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_fixup_prism_dw_idx(kind, cpq, outl);
    if (out_packed(outl)) return kernel_fixup_prism_dw_packed(kind, cpq, inl, outl);
    FE_ALL8(FE_FIX_CASE, 0, PRISM, DWORD, Q_PRISM6) FE_FN2(FE_FIX_CASE, 0, PRISM, DWORD, Q_PRISM6)
    return kernel_fixup_prism_dw_generic(kind, cpq, inl, outl);
}
}  // namespace fe
