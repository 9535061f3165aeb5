// Internal interface between the runtime (fe_runtime.cu) and the kernel
// translation units. Plain C++ types only; no CUDA headers needed by users.
#pragma once
#include <cstdint>

namespace fe {

enum ElemType { TET = 0, PRISM = 1 };
enum Kind { POISSON = 0, GENERIC = 1 };
enum Prec { FP64 = 0, MIXED = 1, DWORD = 2, MIXED_SQS = 3, MIXED_SSQ = 4 };
// The mixed form with the loop orderings of Algorithms 4-7 (SQS, SSQ), for the
// ordering study: float arithmetic, shape test and double-Jacobian fix-up as MIXED.
constexpr bool float_form(int prec) { return prec == MIXED || prec == MIXED_SQS || prec == MIXED_SSQ; }
enum Quad { Q_TET1 = 0, Q_TET4 = 1, Q_PRISM6 = 2 };
enum Layout { SOA = 0, AOS = 1, INDEXED = 2, APPLY = 2 };  // APPLY: output mode of fe_apply_*
// Output modes beyond the layouts: the upper triangle of a symmetric A^e.
constexpr int SOA_PACKED = 3, AOS_PACKED = 4;
constexpr bool out_soa(int o) { return o == SOA || o == SOA_PACKED; }
constexpr bool out_packed(int o) { return o == SOA_PACKED || o == AOS_PACKED; }
// Index of entry (r, s), s >= r, of a packed upper triangle of an NS x NS matrix.
constexpr int packed_index(int ns, int r, int s) { return r * ns - r * (r - 1) / 2 + (s - r); }

// Bits of the device status word (one per context, read at sync).
enum StatusBits : int {
    ST_TMA_TIMEOUT = 1,       // a bounded wait on a bulk copy ran out
    ST_FIXUP_OVERFLOW = 2,    // the fix-up list was too short (never with capacity = n)
    ST_BAD_TILE = 4,          // a batch tile descriptor was out of range
    ST_SKIPPED_TILES = 8      // injected fault: tiles were skipped, outputs incomplete
};

// One homogeneous element set as the kernels see it (device pointers).
struct ElemParams {
    int64_t n;                     // elements
    const double *X;               // coordinates
    int64_t xs;                    // SOA plane stride (elements)
    const void *C;                 // coefficients (double or float)
    int64_t cs;                    // SOA plane stride
    void *A;                       // outputs (double or float)
    void *B;
    int64_t os;                    // SOA plane stride of A and B
    uint8_t *flags;                // may be null
    unsigned long long *fix_list;  // mixed precision: flagged elements (item << 40 | element)
    unsigned int *fix_count;
    unsigned int fix_cap;
    unsigned int item;             // batch item id (0 for a plain call)
    int *status;                   // device status word
    int tma_in, tma_out;           // SOA tiles moved by 2-D tensor copies (maps in TmaMaps)
    const int *conn;               // INDEXED: [n][NS] node indices into X (nodes [n_nodes][3])
    long long n_nodes;
    const void *xv;                // APPLY: nodal input vector; A is y, B is f (may be null)
    long long skip_mod;            // injected fault (fe_ctx_inject_fault): > 0 skips every
                                   // tile whose index is a multiple of it; 0 in normal use
};

// Parameters of the coefficient function (FE_COEF_FUNCTION_U), passed by value
// as a kernel parameter: c_j(u) = p[0][j] + p[1][j] u + p[2][j] u^2, in double and
// in float (the mixed form reads the float copy).
struct CoefFn {
    double pd[3][20];
    float pf[3][20];
};

// Tensor-copy descriptors (CUtensorMap, 128 bytes each) of the plane-major
// inputs and outputs of one launch: coordinates, coefficients, A, b.
struct alignas(64) TmaMaps {
    unsigned char x[128], c[128], a[128], b[128];
};

// Compile-time configuration of one element kernel.
struct KernelKey {
    int type, kind, prec, quad, cpq, in_layout, out_layout;
};

// Kernel pointer for a key, or nullptr if that combination is not built.
// Implemented in the instantiation units.
const void *kernel_tet_fp64(int kind, int quad, int cpq, int inl, int outl);
const void *kernel_tet_mixed(int kind, int quad, int cpq, int inl, int outl);
const void *kernel_prism_fp64(int kind, int cpq, int inl, int outl);
const void *kernel_prism_mixed(int kind, int cpq, int inl, int outl);
const void *kernel_tet_dw(int kind, int quad, int cpq, int inl, int outl);
const void *kernel_prism_dw(int kind, int cpq, int inl, int outl);
// prisms, two threads per element (element-contiguous input and output)
const void *kernel_prism_pair(int kind, int prec, int cpq);
// One group of NS lanes per element (4 for tetrahedra, 6 for prisms), one row each.
const void *kernel_group_tet(int kind, int prec, int quad, int cpq);
// Sixteen threads per tetrahedron (one entry of A^e each): entry_kernel.
const void *kernel_entry_tet(int kind, int prec, int quad, int cpq);
const void *kernel_group_prism(int kind, int prec, int cpq);

// Fix-up kernels (flagged elements of the mixed and double-word forms, redone
// with the Jacobian terms in double); they read the list written by the main kernel.
const void *kernel_fixup_tet(int kind, int quad, int cpq, int inl, int outl);
const void *kernel_fixup_prism(int kind, int cpq, int inl, int outl);
const void *kernel_fixup_tet_dw(int kind, int quad, int cpq, int inl, int outl);
const void *kernel_fixup_prism_dw(int kind, int cpq, int inl, int outl);

// Ordering study (fe_study.cu): mixed form, element-contiguous in and out,
// order 1 = SQS, 2 = SSQ.
const void *kernel_study(int type, int kind, int quad, int cpq, int order);
const void *kernel_fixup_study(int type, int kind, int quad, int cpq, int order);

// INDEXED geometry (node table): the same tables, in their own translation units.
const void *kernel_tet_fp64_idx(int kind, int quad, int cpq, int outl);
const void *kernel_tet_mixed_idx(int kind, int quad, int cpq, int outl);
const void *kernel_tet_dw_idx(int kind, int quad, int cpq, int outl);
const void *kernel_prism_fp64_idx(int kind, int cpq, int outl);
const void *kernel_prism_mixed_idx(int kind, int cpq, int outl);
const void *kernel_prism_dw_idx(int kind, int cpq, int outl);
const void *kernel_fixup_tet_idx(int kind, int quad, int cpq, int outl);
const void *kernel_fixup_tet_dw_idx(int kind, int quad, int cpq, int outl);
const void *kernel_fixup_prism_idx(int kind, int cpq, int outl);
const void *kernel_fixup_prism_dw_idx(int kind, int cpq, int outl);

// Batched persistent kernel (fe_batch.cu): one descriptor per element set and
// one per tile of consecutive elements of a set.
struct BatchItemDev {
    ElemParams p;             // element-contiguous inputs and outputs, mixed precision
    int combo;                // (type, kind, rule, coefficient mode), see batch_combo()
    int pad;
};
// The tiles of one combination are implicit: its items, largest first, each with
// the index of its first tile within the combination (a prefix sum of
// ceil(n / B)). A block maps a tile index to its item by binary search.
struct BatchSeg {
    unsigned int item;        // index into the item table
    unsigned int first_tile;  // tiles of earlier items of this combination
    long long n;              // elements of the item
};
// Dense index of the 12 (type, kind, rule, coefficient mode) combinations of the
// batched kernel with one thread per element, or -1.
inline int batch_combo(int type, int kind, int quad, int cpq) {
    if (type == TET && (quad == Q_TET1 || quad == Q_TET4)) return ((kind * 2 + (quad == Q_TET4)) * 2 + cpq);
    if (type == PRISM && quad == Q_PRISM6) return 8 + kind * 2 + cpq;
    return -1;
}
// Combinations 12..15: the prism combinations 8..11 with two threads per element.
constexpr int kCombos = 16;
inline int batch_tpe(int combo) { return combo >= 12 ? 2 : 1; }
inline int batch_pair_combo(int combo) { return combo >= 8 && combo < 12 ? combo + 4 : combo; }
const void *kernel_batch(int combo);   // persistent kernel of one combination
const void *kernel_batch_fixup();
const void *kernel_selftest_wait();
// Dynamic shared memory of one block of the batched kernel for a combination.
long long batch_smem_bytes(int combo, int block);

}  // namespace fe
