// Tetrahedron kernels with sixteen threads per element (one entry of A^e each;
// the Jacobian terms formed once per element and shared by shuffles), element-
// contiguous input and output, every precision form, kind, tetrahedral rule and
// coefficient mode with coefficient arrays.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_entry_tet(int kind, int prec, int quad, int cpq) {
#define FE_ENT(KD, PR, QD, CP)                                                 \
    if (kind == KD && prec == PR && quad == QD && cpq == CP)                   \
        return reinterpret_cast<const void *>(&entry_kernel<KD, PR, QD, CP>);
#define FE_ENT4(PR, QD) FE_ENT(POISSON, PR, QD, 0) FE_ENT(POISSON, PR, QD, 1) FE_ENT(GENERIC, PR, QD, 0) FE_ENT(GENERIC, PR, QD, 1)
    FE_ENT4(FP64, Q_TET1) FE_ENT4(FP64, Q_TET4) FE_ENT4(MIXED, Q_TET1) FE_ENT4(MIXED, Q_TET4)
    FE_ENT4(DWORD, Q_TET1) FE_ENT4(DWORD, Q_TET4)
#undef FE_ENT4
#undef FE_ENT
    return nullptr;
}
}  // namespace fe
