// Prism kernels, FP64 form.
#include "fe_inst.cuh"
namespace fe {
const void *kernel_prism_fp64(int kind, int cpq, int inl, int outl) {
    if (inl == INDEXED) return kernel_prism_fp64_idx(kind, cpq, outl);
    FE_ALL16(FE_ELEM_CASE, PRISM, FP64, Q_PRISM6) FE_PK8(FE_ELEM_CASE, PRISM, FP64, Q_PRISM6) FE_FN2(FE_ELEM_CASE, 0, PRISM, FP64, Q_PRISM6) FE_FN2(FE_ELEM_CASE, 1, PRISM, FP64, Q_PRISM6)
    return nullptr;
}
}  // namespace fe
