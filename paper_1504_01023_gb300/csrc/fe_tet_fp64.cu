// Tetrahedron kernels, FP64 form.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_tet_fp64(int kind, int quad, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_tet_fp64_idx(kind, quad, cpq, outl);
    if (quad == Q_TET1) { FE_ALL16(FE_F64T_CASE, TET, FP64, Q_TET1) FE_PK8(FE_F64T_CASE, TET, FP64, Q_TET1) FE_FN2(FE_F64T_CASE, 0, TET, FP64, Q_TET1) FE_FN2(FE_F64T_CASE, 1, TET, FP64, Q_TET1) }
    if (quad == Q_TET4) { FE_ALL16(FE_F64T_CASE, TET, FP64, Q_TET4) FE_PK8(FE_F64T_CASE, TET, FP64, Q_TET4) FE_FN2(FE_F64T_CASE, 0, TET, FP64, Q_TET4) FE_FN2(FE_F64T_CASE, 1, TET, FP64, Q_TET4) }
    return nullptr;
}
}  // namespace fe
