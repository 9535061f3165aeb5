// Tetrahedron kernels with four threads per element (one row of A^e each; the
// Jacobian terms formed once per element and shared by shuffles), element-
// contiguous input and output, every precision form, kind, tetrahedral rule and
// coefficient mode with coefficient arrays.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_group_tet(int kind, int prec, int quad, int cpq) {
#define FE_GRP(KD, PR, QD, CP)                                                 \
    if (kind == KD && prec == PR && quad == QD && cpq == CP)                   \
        return reinterpret_cast<const void *>(&group_kernel<TET, KD, PR, QD, CP>);
#define FE_GRP4(PR, QD) FE_GRP(POISSON, PR, QD, 0) FE_GRP(POISSON, PR, QD, 1) FE_GRP(GENERIC, PR, QD, 0) FE_GRP(GENERIC, PR, QD, 1)
    FE_GRP4(FP64, Q_TET1) FE_GRP4(FP64, Q_TET4) FE_GRP4(MIXED, Q_TET1) FE_GRP4(MIXED, Q_TET4)
    FE_GRP4(DWORD, Q_TET1) FE_GRP4(DWORD, Q_TET4)
#undef FE_GRP4
#undef FE_GRP
    return nullptr;
}
}  // namespace fe
