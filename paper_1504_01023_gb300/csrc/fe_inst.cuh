// Explicit kernel tables: every (kind, coefficient mode, input layout, output
// layout) combination of one element type, precision and rule.
#pragma once
#include "fe_kernels.cuh"

#define FE_ELEM_CASE(ET, PREC, QUAD, KD, CP, IL, OL)                                  \
    if (kind == KD && cpq == CP && inl == IL && outl == OL)                          \
        return reinterpret_cast<const void *>(&fe::elem_kernel<ET, KD, PREC, QUAD, CP, IL, OL>);
// FP64 tetrahedra: the register-capped variant of the main kernel.
#define FE_F64T_CASE(ET, PREC, QUAD, KD, CP, IL, OL)                                  \
    if (kind == KD && cpq == CP && inl == IL && outl == OL)                          \
        return reinterpret_cast<const void *>(&fe::elem_kernel_f64t<KD, QUAD, CP, IL, OL>);
// Double-word tetrahedra: the register-capped variant of the main kernel for
// per-element coefficients (dw_tet_kernel).
#define FE_DWT_CASE(ET, PREC, QUAD, KD, CP, IL, OL)                                   \
    if (kind == KD && cpq == CP && inl == IL && outl == OL) return fe::dw_tet_kernel<KD, QUAD, CP, IL, OL>();
#define FE_FIX_CASE(ET, PREC, QUAD, KD, CP, IL, OL)                                   \
    if (kind == KD && cpq == CP && inl == IL && outl == OL)                          \
        return reinterpret_cast<const void *>(&fe::fixup_kernel<ET, KD, PREC, QUAD, CP, IL, OL>);

#define FE_ALL16(M, ...)                                                              \
    M(__VA_ARGS__, 0, 0, 0, 0) M(__VA_ARGS__, 0, 0, 0, 1) M(__VA_ARGS__, 0, 0, 1, 0)  \
    M(__VA_ARGS__, 0, 0, 1, 1) M(__VA_ARGS__, 0, 1, 0, 0) M(__VA_ARGS__, 0, 1, 0, 1)  \
    M(__VA_ARGS__, 0, 1, 1, 0) M(__VA_ARGS__, 0, 1, 1, 1) M(__VA_ARGS__, 1, 0, 0, 0)  \
    M(__VA_ARGS__, 1, 0, 0, 1) M(__VA_ARGS__, 1, 0, 1, 0) M(__VA_ARGS__, 1, 0, 1, 1)  \
    M(__VA_ARGS__, 1, 1, 0, 0) M(__VA_ARGS__, 1, 1, 0, 1) M(__VA_ARGS__, 1, 1, 1, 0)  \
    M(__VA_ARGS__, 1, 1, 1, 1)

// The eight (coefficient mode, input layout, output layout) combinations of one kind.
#define FE_ALL8(M, KD, ...)                                                           \
    M(__VA_ARGS__, KD, 0, 0, 0) M(__VA_ARGS__, KD, 0, 0, 1) M(__VA_ARGS__, KD, 0, 1, 0) \
    M(__VA_ARGS__, KD, 0, 1, 1) M(__VA_ARGS__, KD, 1, 0, 0) M(__VA_ARGS__, KD, 1, 0, 1) \
    M(__VA_ARGS__, KD, 1, 1, 0) M(__VA_ARGS__, KD, 1, 1, 1)

// The eight (kind, coefficient mode, output layout) combinations with INDEXED
// geometry (inputs fixed: node table, element-contiguous coefficients).
#define FE_IDX8(M, ...)                                                               \
    M(__VA_ARGS__, 0, 0, 2, 0) M(__VA_ARGS__, 0, 0, 2, 1) M(__VA_ARGS__, 0, 1, 2, 0)  \
    M(__VA_ARGS__, 0, 1, 2, 1) M(__VA_ARGS__, 1, 0, 2, 0) M(__VA_ARGS__, 1, 0, 2, 1)  \
    M(__VA_ARGS__, 1, 1, 2, 0) M(__VA_ARGS__, 1, 1, 2, 1)

// INDEXED geometry: the kernel that reads straight from global memory.
#define FE_GATHER_CASE(ET, PREC, QUAD, KD, CP, IL, OL)                                \
    if (kind == KD && cpq == CP && inl == IL && outl == OL)                          \
        return reinterpret_cast<const void *>(&fe::gather_kernel<ET, KD, PREC, QUAD, CP, OL>);

// The four (kind, coefficient mode) combinations of the matrix-free output
// (INDEXED geometry, OUTL == APPLY).
#define FE_IDXA4(M, ...)                                                              \
    M(__VA_ARGS__, 0, 0, 2, 2) M(__VA_ARGS__, 0, 1, 2, 2) M(__VA_ARGS__, 1, 0, 2, 2)  \
    M(__VA_ARGS__, 1, 1, 2, 2)

// Packed (upper-triangle) outputs, Laplace kind only: coefficient mode x input
// layout (SOA, AOS) x output (SOA_PACKED, AOS_PACKED).
#define FE_PK8(M, ...)                                                                \
    M(__VA_ARGS__, 0, 0, 0, 3) M(__VA_ARGS__, 0, 0, 0, 4) M(__VA_ARGS__, 0, 0, 1, 3)  \
    M(__VA_ARGS__, 0, 0, 1, 4) M(__VA_ARGS__, 0, 1, 0, 3) M(__VA_ARGS__, 0, 1, 0, 4)  \
    M(__VA_ARGS__, 0, 1, 1, 3) M(__VA_ARGS__, 0, 1, 1, 4)

// The coefficient function of a nodal field (CPQ == 2): element-contiguous input,
// full output in either layout, one kind.
#define FE_FN2(M, KD, ...) M(__VA_ARGS__, KD, 2, 1, 0) M(__VA_ARGS__, KD, 2, 1, 1)
