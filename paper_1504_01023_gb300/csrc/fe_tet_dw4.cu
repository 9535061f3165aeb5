// Tetrahedron kernels, double-word form, four-point rule.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_tet_dw4(int kind, int cpq, int inl, int outl) {
    FE_ALL16(FE_DWT_CASE, TET, DWORD, Q_TET4) FE_PK8(FE_DWT_CASE, TET, DWORD, Q_TET4) FE_FN2(FE_ELEM_CASE, 0, TET, DWORD, Q_TET4) FE_FN2(FE_ELEM_CASE, 1, TET, DWORD, Q_TET4)
    return nullptr;
}
const void *kernel_fixup_tet_dw4(int kind, int cpq, int inl, int outl) {
    FE_ALL16(FE_FIX_CASE, TET, DWORD, Q_TET4) FE_PK8(FE_FIX_CASE, TET, DWORD, Q_TET4) FE_FN2(FE_FIX_CASE, 0, TET, DWORD, Q_TET4) FE_FN2(FE_FIX_CASE, 1, TET, DWORD, Q_TET4)
    return nullptr;
}
}  // namespace fe
