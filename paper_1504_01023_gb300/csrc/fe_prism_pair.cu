// Prism kernels with two threads per element (one zeta level each), element-
// contiguous input and output, every precision form and coefficient mode with
// coefficient arrays.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_prism_pair(int kind, int prec, int cpq) {
#define FE_PAIR(KD, PR, CP) \
    if (kind == KD && prec == PR && cpq == CP) return reinterpret_cast<const void *>(&pair_kernel<KD, PR, CP>);
    FE_PAIR(POISSON, FP64, 0) FE_PAIR(POISSON, FP64, 1) FE_PAIR(GENERIC, FP64, 0) FE_PAIR(GENERIC, FP64, 1)
    FE_PAIR(POISSON, MIXED, 0) FE_PAIR(POISSON, MIXED, 1) FE_PAIR(GENERIC, MIXED, 0) FE_PAIR(GENERIC, MIXED, 1)
    FE_PAIR(POISSON, DWORD, 0) FE_PAIR(POISSON, DWORD, 1) FE_PAIR(GENERIC, DWORD, 0) FE_PAIR(GENERIC, DWORD, 1)
#undef FE_PAIR
    return nullptr;
}
}  // namespace fe
