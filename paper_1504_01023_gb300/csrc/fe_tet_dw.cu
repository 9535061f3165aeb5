// Tetrahedron kernels, double-word form (double-accuracy results from float
// pipes; flagged elements redone in double): the one-point rule here, the
// four-point rule in fe_tet_dw4.cu (two units compile in parallel).
#include "fe_inst.cuh"
namespace fe {
const void *kernel_tet_dw4(int kind, int cpq, int inl, int outl);
const void *kernel_fixup_tet_dw4(int kind, int cpq, int inl, int outl);

const void *kernel_tet_dw(int kind, int quad, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_tet_dw_idx(kind, quad, cpq, outl);
    if (quad == Q_TET4) return kernel_tet_dw4(kind, cpq, inl, outl);
    if (quad == Q_TET1) { FE_ALL16(FE_DWT_CASE, TET, DWORD, Q_TET1) FE_PK8(FE_DWT_CASE, TET, DWORD, Q_TET1) FE_FN2(FE_ELEM_CASE, 0, TET, DWORD, Q_TET1) FE_FN2(FE_ELEM_CASE, 1, TET, DWORD, Q_TET1) }
    return nullptr;
}
const void *kernel_fixup_tet_dw(int kind, int quad, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_fixup_tet_dw_idx(kind, quad, cpq, outl);
    if (quad == Q_TET4) return kernel_fixup_tet_dw4(kind, cpq, inl, outl);
    if (quad == Q_TET1) { FE_ALL16(FE_FIX_CASE, TET, DWORD, Q_TET1) FE_PK8(FE_FIX_CASE, TET, DWORD, Q_TET1) FE_FN2(FE_FIX_CASE, 0, TET, DWORD, Q_TET1) FE_FN2(FE_FIX_CASE, 1, TET, DWORD, Q_TET1) }
    return nullptr;
}
}  // namespace fe
