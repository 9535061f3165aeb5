// Tetrahedron kernels, mixed form (float arithmetic, double Jacobian fix-up).
#include "fe_inst.cuh"
namespace fe {
const void *kernel_tet_mixed(int kind, int quad, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_tet_mixed_idx(kind, quad, cpq, outl);
    if (quad == Q_TET1) { FE_ALL16(FE_ELEM_CASE, TET, MIXED, Q_TET1) FE_PK8(FE_ELEM_CASE, TET, MIXED, Q_TET1) FE_FN2(FE_ELEM_CASE, 0, TET, MIXED, Q_TET1) FE_FN2(FE_ELEM_CASE, 1, TET, MIXED, Q_TET1) }
    if (quad == Q_TET4) { FE_ALL16(FE_ELEM_CASE, TET, MIXED, Q_TET4) FE_PK8(FE_ELEM_CASE, TET, MIXED, Q_TET4) FE_FN2(FE_ELEM_CASE, 0, TET, MIXED, Q_TET4) FE_FN2(FE_ELEM_CASE, 1, TET, MIXED, Q_TET4) }
    return nullptr;
}
const void *kernel_fixup_tet(int kind, int quad, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_fixup_tet_idx(kind, quad, cpq, outl);
    if (quad == Q_TET1) { FE_ALL16(FE_FIX_CASE, TET, MIXED, Q_TET1) FE_PK8(FE_FIX_CASE, TET, MIXED, Q_TET1) FE_FN2(FE_FIX_CASE, 0, TET, MIXED, Q_TET1) FE_FN2(FE_FIX_CASE, 1, TET, MIXED, Q_TET1) }
    if (quad == Q_TET4) { FE_ALL16(FE_FIX_CASE, TET, MIXED, Q_TET4) FE_PK8(FE_FIX_CASE, TET, MIXED, Q_TET4) FE_FN2(FE_FIX_CASE, 0, TET, MIXED, Q_TET4) FE_FN2(FE_FIX_CASE, 1, TET, MIXED, Q_TET4) }
    return nullptr;
}
}  // namespace fe
