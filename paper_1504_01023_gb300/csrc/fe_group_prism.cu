// Prism kernels with six threads per element (lane q forms the Jacobian terms at
// point q and owns row q of A^e; the points' terms are shared by shuffles),
// element-contiguous input and output, every precision form, kind and
// coefficient mode with coefficient arrays.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_group_prism(int kind, int prec, int cpq) {
#define FE_GRP(KD, PR, CP)                                                     \
    if (kind == KD && prec == PR && cpq == CP)                                 \
        return reinterpret_cast<const void *>(&group_kernel<PRISM, KD, PR, Q_PRISM6, CP>);
    FE_GRP(POISSON, FP64, 0) FE_GRP(POISSON, FP64, 1) FE_GRP(GENERIC, FP64, 0) FE_GRP(GENERIC, FP64, 1)
    FE_GRP(POISSON, MIXED, 0) FE_GRP(POISSON, MIXED, 1) FE_GRP(GENERIC, MIXED, 0) FE_GRP(GENERIC, MIXED, 1)
    FE_GRP(POISSON, DWORD, 0) FE_GRP(POISSON, DWORD, 1) FE_GRP(GENERIC, DWORD, 0) FE_GRP(GENERIC, DWORD, 1)
#undef FE_GRP
    return nullptr;
}
}  // namespace fe
