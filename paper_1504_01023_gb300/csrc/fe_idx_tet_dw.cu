// Tetrahedron kernels with INDEXED geometry (node table), double-word form.
// Unstaged (gather_kernel): measured 32.5 vs 28.1 Gelem/s staged for the generic
// mixed tetrahedron.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_tet_dw_idx(int kind, int quad, int cpq, int outl) {
    const int inl = INDEXED;
    if (quad == Q_TET1) { FE_IDX8(FE_GATHER_CASE, TET, DWORD, Q_TET1) FE_IDXA4(FE_GATHER_CASE, TET, DWORD, Q_TET1) }
    if (quad == Q_TET4) { FE_IDX8(FE_GATHER_CASE, TET, DWORD, Q_TET4) FE_IDXA4(FE_GATHER_CASE, TET, DWORD, Q_TET4) }
    return nullptr;
}
const void *kernel_fixup_tet_dw_idx(int kind, int quad, int cpq, int outl) {
    const int inl = INDEXED;
    if (quad == Q_TET1) { FE_IDX8(FE_FIX_CASE, TET, DWORD, Q_TET1) FE_IDXA4(FE_FIX_CASE, TET, DWORD, Q_TET1) }
    if (quad == Q_TET4) { FE_IDX8(FE_FIX_CASE, TET, DWORD, Q_TET4) FE_IDXA4(FE_FIX_CASE, TET, DWORD, Q_TET4) }
    return nullptr;
}
}  // namespace fe
