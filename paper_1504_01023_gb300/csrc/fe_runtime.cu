// C ABI of the integration library: context, argument validation, launch shapes
// and the autotuner, profiling, and the chunked host-buffer pipeline.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>

#include <cudaTypedefs.h>

#include "fe_runtime.h"

namespace fe {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string t_last_error;

fe_status set_error(fe_ctx *ctx, fe_status st, const std::string &msg) {
    t_last_error = msg;
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->last_error = msg;
    }
    return st;
}

fe_status cuda_check(fe_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return FE_OK;
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return set_error(ctx, e == cudaErrorMemoryAllocation ? FE_ERR_OOM : FE_ERR_CUDA, msg);
}

bool take_alloc_fault(fe_ctx *ctx) {
    if (!ctx) return false;
    int64_t left = ctx->fail_allocs.load();
    while (left > 0)
        if (ctx->fail_allocs.compare_exchange_weak(left, left - 1)) return true;
    return false;
}

fe_status ctx_malloc(fe_ctx *ctx, void **p, size_t bytes, const char *what) {
    if (take_alloc_fault(ctx)) {
        *p = nullptr;
        return set_error(ctx, FE_ERR_OOM, std::string(what) + ": injected allocation failure");
    }
    return cuda_check(ctx, cudaMalloc(p, bytes), what);
}

int ns_of(fe_elem_type t) { return t == FE_TET ? 4 : 6; }
int nq_of(fe_quad q) { return q == FE_QUAD_TET1 ? 1 : (q == FE_QUAD_TET4 ? 4 : 6); }
int nc_of(fe_elem_type type, const fe_elem_args *a) {
    if (a->coef_mode == FE_COEF_FUNCTION_U) return ns_of(type);  // nodal values of the field
    return (a->kind == FE_POISSON ? 1 : 20) * (a->coef_mode == FE_COEF_PER_QPOINT ? nq_of(a->quad) : 1);
}
static int csize(fe_precision p) { return p == FE_FP32_MIXED ? 4 : 8; }

fe_status ensure_scratch(fe_ctx *ctx, Scratch &s, uint64_t n) {
    if (!s.fix_count) {
        fe_status st = ctx_malloc(ctx, reinterpret_cast<void **>(&s.fix_count), 64, "cudaMalloc(fix_count)");
        if (st != FE_OK) return st;
        st = ctx_malloc(ctx, reinterpret_cast<void **>(&s.status), 64, "cudaMalloc(status)");
        if (st != FE_OK) return st;
        cudaMemset(s.fix_count, 0, 64);
        cudaMemset(s.status, 0, 64);
    }
    if (n > 0xFFFFFFFFull) return set_error(ctx, FE_ERR_INVALID_ARG, "more than 2^32-1 elements in one call");
    if (n > s.fix_cap) {
        if (s.fix_list) cudaFree(s.fix_list);
        s.fix_list = nullptr;
        s.fix_cap = 0;
        uint64_t cap = std::max<uint64_t>(n, 1024);
        fe_status st = ctx_malloc(ctx, reinterpret_cast<void **>(&s.fix_list), cap * sizeof(unsigned long long),
                                  "cudaMalloc(fix_list)");
        if (st != FE_OK) return st;
        s.fix_cap = static_cast<unsigned>(cap);
    }
    return FE_OK;
}

void free_scratch(Scratch &s) {
    if (s.fix_list) cudaFree(s.fix_list);
    if (s.fix_count) cudaFree(s.fix_count);
    if (s.status) cudaFree(s.status);
    s = Scratch{};
}

// Kernel template value of the coefficient mode: 0 per element, 1 per point,
// 2 the function of a nodal field.
static int cpq_of(const fe_elem_args *a) { return a->coef_mode == FE_COEF_FUNCTION_U ? 2 : a->coef_mode == FE_COEF_PER_QPOINT; }

// Two threads per element: prisms with element-contiguous coordinates, full
// element-contiguous outputs, coefficient arrays and the QSS order.
static bool pair_ok(fe_elem_type type, const fe_elem_args *a, int outl) {
    return type == FE_PRISM && a->coords_layout == FE_LAYOUT_AOS && outl == AOS && !a->ordering && cpq_of(a) < 2;
}

// Several threads per element of any type (one row each): the same inputs and
// outputs as two threads per prism.
static bool group_ok(fe_elem_type type, const fe_elem_args *a, int outl) {
    return a->coords_layout == FE_LAYOUT_AOS && outl == AOS && !a->ordering && cpq_of(a) < 2 && (type == FE_TET || type == FE_PRISM);
}

// Threads per element a key may use: 1; 2 (prisms), NS (4 for tetrahedra, 6 for
// prisms) and 16 (tetrahedra) with element-contiguous inputs and outputs,
// coefficient arrays, QSS.
static bool tpe_ok(fe_elem_type type, const fe_elem_args *a, int outl, int tpe) {
    if (tpe == 1) return true;
    if (tpe == 2) return pair_ok(type, a, outl);
    if (tpe == 16) return type == FE_TET && group_ok(type, a, outl);
    return tpe == ns_of(type) && group_ok(type, a, outl);
}

static const void *main_kernel(fe_elem_type type, const fe_elem_args *a, int outl, int tpe = 1) {
    const int cpq = cpq_of(a);
    if (tpe == 2) return pair_ok(type, a, outl) ? kernel_prism_pair(a->kind, a->prec, cpq) : nullptr;
    if (tpe > 2) {
        if (!tpe_ok(type, a, outl, tpe)) return nullptr;
        if (tpe == 16) return kernel_entry_tet(a->kind, a->prec, a->quad, cpq);
        return type == FE_TET ? kernel_group_tet(a->kind, a->prec, a->quad, cpq) : kernel_group_prism(a->kind, a->prec, cpq);
    }
    if (tpe != 1) return nullptr;
    if (a->ordering) return kernel_study(type, a->kind, a->quad, cpq, a->ordering);
    const int il = a->coords_layout;
    if (type == FE_TET) {
        switch (a->prec) {
            case FE_FP64: return kernel_tet_fp64(a->kind, a->quad, cpq, il, outl);
            case FE_FP32_MIXED: return kernel_tet_mixed(a->kind, a->quad, cpq, il, outl);
            case FE_FP64_DW: return kernel_tet_dw(a->kind, a->quad, cpq, il, outl);
        }
        return nullptr;
    }
    switch (a->prec) {
        case FE_FP64: return kernel_prism_fp64(a->kind, cpq, il, outl);
        case FE_FP32_MIXED: return kernel_prism_mixed(a->kind, cpq, il, outl);
        case FE_FP64_DW: return kernel_prism_dw(a->kind, cpq, il, outl);
    }
    return nullptr;
}

static const void *fix_kernel(fe_elem_type type, const fe_elem_args *a, int outl) {
    const int cpq = cpq_of(a);
    if (a->ordering) return kernel_fixup_study(type, a->kind, a->quad, cpq, a->ordering);
    const int il = a->coords_layout;
    if (a->prec == FE_FP64_DW)
        return type == FE_TET ? kernel_fixup_tet_dw(a->kind, a->quad, cpq, il, outl)
                              : kernel_fixup_prism_dw(a->kind, cpq, il, outl);
    return type == FE_TET ? kernel_fixup_tet(a->kind, a->quad, cpq, il, outl) : kernel_fixup_prism(a->kind, cpq, il, outl);
}

// Dynamic shared memory of one block: the tile's inputs and outputs, each region
// rounded to 16 bytes exactly as BlockSmem in fe_kernels.cuh lays them out.
// Output mode of fe_apply_* (matrix-free), passed where an fe_layout goes.
static constexpr int kOutApply = 2;

// Kernel output mode of an fe_out: its layout, or the packed upper triangle.
static int out_mode(const fe_out *o) {
    if (o->layout == kOutApply) return kOutApply;
    return o->packed ? (o->layout == FE_LAYOUT_SOA ? SOA_PACKED : AOS_PACKED) : int(o->layout);
}
// A^e entries written per element.
static int na_out(fe_elem_type type, int outl) {
    const int ns = ns_of(type);
    return out_packed(outl) ? ns * (ns + 1) / 2 : ns * ns;
}

static int64_t smem_bytes(fe_elem_type type, const fe_elem_args *a, int outl, int B) {
    // tetrahedra with a node table read straight from global memory (gather_kernel)
    if (a->coords_layout == FE_LAYOUT_INDEXED && type == FE_TET) return 0;
    const int ns = ns_of(type), nc = nc_of(type, a), cs = csize(a->prec);
    auto r16 = [](int64_t v) { return (v + 15) / 16 * 16; };
    const int64_t geo = a->coords_layout == FE_LAYOUT_INDEXED ? r16(int64_t(B) * ns * 4) : int64_t(B) * 3 * ns * 8;
    const int64_t in = geo + r16(int64_t(B) * nc * cs),
                  out = r16(int64_t(B) * na_out(type, outl) * cs) + r16(int64_t(B) * ns * cs);
    if (outl == kOutApply) return in;  // matrix-free: results leave from registers
    return in > out ? in : out;
}

// Static shared memory of the kernels (the mbarrier), kept out of the dynamic budget.
static constexpr int64_t kStaticSmem = 1024;

fe_status set_smem_attr(fe_ctx *ctx, const void *k, int64_t smem) {
    static std::mutex mu;
    static std::map<const void *, int64_t> done;
    std::lock_guard<std::mutex> lk(mu);
    auto it = done.find(k);
    if (it != done.end() && it->second >= smem) return FE_OK;
    fe_status e = cuda_check(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                             "cudaFuncSetAttribute");
    if (e == FE_OK) done[k] = smem;
    return e;
}

static std::string shape_key(fe_elem_type type, const fe_elem_args *a, const fe_out *o) {
    int bucket = 0;
    for (int64_t n = a->n_elem; n > 1; n >>= 2) ++bucket;  // size class: floor(log4 n)
    std::ostringstream k;
    k << "t" << type << "k" << a->kind << "p" << a->prec << "q" << a->quad << "c" << a->coef_mode << "i"
      << a->coords_layout << "o" << out_mode(o) << "r" << a->ordering << "n" << bucket;
    return k.str();
}

Shape default_shape(fe_elem_type type) { return Shape{type == FE_TET ? 256 : 128, 0}; }

// Largest block of a kernel (its launch bounds): 512 for float and double
// tetrahedra, 256 for prisms and double-word tetrahedra.
static int max_block(fe_elem_type type, fe_precision prec) {
    return type == FE_TET && prec != FE_FP64_DW ? 512 : 256;
}

// Threads of a block of `block` elements with `tpe` threads each: groups of tpe
// lanes fill a warp 32 / tpe at a time (6 lanes per prism: 5 groups per warp, two
// lanes idle). 0 if `block` is not a whole number of warps' groups.
static int shape_threads(int block, int tpe) {
    const int epw = 32 / tpe;
    if (block < 1 || block % epw) return 0;
    return block / epw * 32;
}

static cudaEvent_t pool_event(fe_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// ---------------------------------------------------------------------------
// Tensor-copy descriptors for plane-major (SOA) tiles.
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

// Planes of `n` elements (`planes` of them, `pitch` bytes apart) as a 2-D tensor
// with box (box_n elements, all planes). False if the layout does not meet the
// tensor-copy rules (16-byte aligned base and pitch, box rows of 16-byte multiples,
// at most 256 elements and 256 planes per box, coordinates within 31 bits).
static bool encode_planes(void *out, bool dbl, const void *base, uint64_t n, uint64_t planes, uint64_t pitch,
                          uint32_t box_n) {
    auto enc = tensor_map_encoder();
    const uint32_t elt = dbl ? 8 : 4;
    if (!enc || !base || n == 0 || n >= (1ull << 31) || planes == 0 || planes > 256 || box_n > 256 ||
        (uint64_t(box_n) * elt) % 16 || reinterpret_cast<uintptr_t>(base) % 16)
        return false;
    if (planes == 1) pitch = (n * elt + 15) / 16 * 16;
    if (pitch % 16 || pitch < n * elt) return false;
    const cuuint64_t dims[2] = {n, planes};
    const cuuint64_t strides[1] = {pitch};
    const cuuint32_t box[2] = {box_n, uint32_t(planes)};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap *>(out), dbl ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                     2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

fe_status launch_set(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *a, const fe_out *o, Scratch &s, cudaStream_t st,
                     const Shape *force, const void *x) {
    if (a->n_elem == 0) return FE_OK;
    const int outl = out_mode(o);
    Shape sh = default_shape(type);
    if (force) {
        sh = *force;
    } else {
        auto it = ctx->shapes.find(shape_key(type, a, o));
        if (it != ctx->shapes.end()) sh = it->second;
    }
    const void *k = main_kernel(type, a, outl, sh.tpe);
    if (!k) return set_error(ctx, FE_ERR_UNSUPPORTED, "no kernel for this combination");
    const int threads = shape_threads(sh.block, sh.tpe);
    if (!threads) return set_error(ctx, FE_ERR_INVALID_ARG, "bad launch shape");
    const int64_t smem = smem_bytes(type, a, outl, sh.block);
    if (smem + kStaticSmem > ctx->max_smem_optin)
        return set_error(ctx, FE_ERR_UNSUPPORTED, "shared memory of this launch shape too large");
    {
        fe_status e = set_smem_attr(ctx, k, smem);
        if (e != FE_OK) return e;
    }
    const int64_t ntiles = (a->n_elem + sh.block - 1) / sh.block;
    int64_t grid = ntiles;
    if (sh.persistent) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, size_t(smem));
        grid = std::min<int64_t>(ntiles, int64_t(std::max(per_sm, 1)) * ctx->sms);
    }
    grid = std::min<int64_t>(grid, 0x7FFFFFFF);

    ElemParams p{};
    p.n = a->n_elem;
    p.X = a->coords;
    p.xs = a->coords_stride ? a->coords_stride : a->n_elem;
    p.C = a->coefs;
    p.cs = a->coefs_stride ? a->coefs_stride : a->n_elem;
    p.A = o->A;
    p.B = o->b;
    p.os = o->stride ? o->stride : a->n_elem;
    p.flags = o->flags;
    p.item = 0;
    p.conn = a->coords_layout == FE_LAYOUT_INDEXED ? a->conn : nullptr;
    p.n_nodes = a->coords_layout == FE_LAYOUT_INDEXED ? a->n_nodes : 0;
    p.xv = x;
    if (ctx->skip_launches.load() > 0 && !force) {   // injected fault: this launch skips tiles
        if (ctx->skip_launches.fetch_sub(1) > 0) p.skip_mod = ctx->skip_mod;
    }
    const bool fixup = a->prec != FE_FP64;   // mixed and double-word forms flag elements
    if (fixup) {
        fe_status e = ensure_scratch(ctx, s, uint64_t(a->n_elem));
        if (e != FE_OK) return e;
        p.fix_list = s.fix_list;
        p.fix_count = s.fix_count;
        p.fix_cap = s.fix_cap;
        cudaError_t ce = cudaMemsetAsync(s.fix_count, 0, sizeof(unsigned), st);
        if (ce != cudaSuccess) return cuda_check(ctx, ce, "cudaMemsetAsync");
    } else if (!s.status) {
        fe_status e = ensure_scratch(ctx, s, 0);
        if (e != FE_OK) return e;
    }
    p.status = s.status;

    // plane-major tiles of up to 256 elements move as 2-D tensor copies
    TmaMaps tm;
    memset(&tm, 0, sizeof tm);
    if (sh.block <= 256) {
        const int ns = ns_of(type), nc = nc_of(type, a);
        const bool dbl = a->prec != FE_FP32_MIXED;
        const uint64_t cs = dbl ? 8 : 4;
        if (a->coords_layout == FE_LAYOUT_SOA)
            p.tma_in = encode_planes(tm.x, true, a->coords, uint64_t(a->n_elem), 3 * ns, uint64_t(p.xs) * 8, sh.block) &&
                       encode_planes(tm.c, dbl, a->coefs, uint64_t(a->n_elem), nc, uint64_t(p.cs) * cs, sh.block);
        if (o->layout == FE_LAYOUT_SOA)
            p.tma_out = encode_planes(tm.a, dbl, o->A, uint64_t(a->n_elem), na_out(type, outl), uint64_t(p.os) * cs,
                                      sh.block) &&
                        encode_planes(tm.b, dbl, o->b, uint64_t(a->n_elem), ns, uint64_t(p.os) * cs, sh.block);
    }

    CoefFn fn;
    memset(&fn, 0, sizeof fn);
    if (a->coef_mode == FE_COEF_FUNCTION_U)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 20; ++j) {
                fn.pd[i][j] = a->coef_fn->p[i][j];
                fn.pf[i][j] = float(a->coef_fn->p[i][j]);
            }
    void *args[] = {&p, &tm, &fn};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const bool profile = ctx->profiling && !force;
    if (profile) {
        ev0 = pool_event(ctx);
        ev1 = pool_event(ctx);
        cudaEventRecord(ev0, st);
    }
    cudaError_t ce = cudaLaunchKernel(k, dim3(unsigned(grid)), dim3(unsigned(threads)), args, size_t(smem), st);
    if (ce != cudaSuccess) {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, k);
        std::ostringstream m;
        m << "cudaLaunchKernel(elem) grid " << grid << " block " << threads << " smem " << smem
          << " (func: max threads " << fa.maxThreadsPerBlock << ", max dyn smem " << fa.maxDynamicSharedSizeBytes
          << ", static smem " << fa.sharedSizeBytes << ", regs " << fa.numRegs << ")";
        return cuda_check(ctx, ce, m.str().c_str());
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (profile) {
        cudaEventRecord(ev1, st);
        ctx->prof_events.emplace_back(ev0, ev1);
    }
    if (fixup) {
        const void *fk = fix_kernel(type, a, outl);
        const int64_t fgrid = std::min<int64_t>((a->n_elem + 255) / 256, int64_t(ctx->sms) * 4);
        void *fargs[] = {&p, &fn};
        ce = cudaLaunchKernel(fk, dim3(unsigned(std::max<int64_t>(fgrid, 1))), dim3(256), fargs, 0, st);
        if (ce != cudaSuccess) return cuda_check(ctx, ce, "cudaLaunchKernel(fixup)");
        g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    return FE_OK;
}

// Chunked pipeline for host buffers: copy-in, kernels and copy-out of
// consecutive chunks overlap on three streams (double-buffered staging).
static fe_status ensure_stage(fe_ctx *ctx, int slot, int idx, uint64_t bytes) {
    if (ctx->stage[slot][idx] && ctx->stage_bytes[slot][idx] >= bytes) return FE_OK;
    if (ctx->stage[slot][idx]) cudaFree(ctx->stage[slot][idx]);
    ctx->stage[slot][idx] = nullptr;
    ctx->stage_bytes[slot][idx] = 0;
    bytes = std::max<uint64_t>(bytes, 256);
    fe_status st = ctx_malloc(ctx, &ctx->stage[slot][idx], bytes, "cudaMalloc(stage)");
    if (st == FE_OK) ctx->stage_bytes[slot][idx] = bytes;
    return st;
}

static fe_status host_pipeline(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *a, const fe_out *o, cudaStream_t user) {
    const int64_t n = a->n_elem;
    const int ns = ns_of(type), nc = nc_of(type, a), cs = csize(a->prec);
    const int nx = 3 * ns, na = na_out(type, out_mode(o));
    const int64_t K = std::min<int64_t>(n, int64_t(1) << 20);
    const bool in_host = a->memory == FE_MEM_HOST, out_host = o->memory == FE_MEM_HOST;
    const uint64_t need[5] = {uint64_t(K) * nx * 8, uint64_t(K) * nc * cs, uint64_t(K) * na * cs, uint64_t(K) * ns * cs,
                              uint64_t(K)};
    for (int slot = 0; slot < 2; ++slot)
        for (int i = 0; i < 5; ++i) {
            if ((i < 2 && !in_host) || (i >= 2 && !out_host)) continue;
            fe_status st = ensure_stage(ctx, slot, i, need[i]);
            if (st != FE_OK) return st;
        }
    if (!ctx->s_in) {
        cudaStreamCreateWithFlags(&ctx->s_in, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&ctx->s_out, cudaStreamNonBlocking);
    }
    cudaEvent_t start, in_done[2], comp_done[2], out_done[2];
    cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    for (int i = 0; i < 2; ++i) {
        cudaEventCreateWithFlags(&in_done[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&comp_done[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&out_done[i], cudaEventDisableTiming);
    }
    cudaEventRecord(start, user);
    cudaStreamWaitEvent(ctx->s_in, start, 0);
    cudaStreamWaitEvent(ctx->s_comp, start, 0);
    cudaStreamWaitEvent(ctx->s_out, start, 0);
    const int64_t xs = a->coords_stride ? a->coords_stride : n;
    const int64_t cst = a->coefs_stride ? a->coefs_stride : n;
    const int64_t os = o->stride ? o->stride : n;
    const char *X = reinterpret_cast<const char *>(a->coords);
    const char *C = static_cast<const char *>(a->coefs);
    char *A = static_cast<char *>(o->A);
    char *B = static_cast<char *>(o->b);
    fe_status result = FE_OK;
    int64_t chunk = 0;
    for (int64_t c0 = 0; c0 < n && result == FE_OK; c0 += K, ++chunk) {
        const int slot = int(chunk & 1);
        const int64_t m = std::min(K, n - c0);
        if (chunk >= 2) {
            cudaStreamWaitEvent(ctx->s_in, out_done[slot], 0);
            cudaStreamWaitEvent(ctx->s_comp, out_done[slot], 0);
        }
        fe_elem_args ca = *a;
        fe_out co = *o;
        ca.n_elem = m;
        ca.memory = FE_MEM_DEVICE;
        co.memory = FE_MEM_DEVICE;
        // inputs
        if (in_host) {
            char *dX = static_cast<char *>(ctx->stage[slot][0]);
            char *dC = static_cast<char *>(ctx->stage[slot][1]);
            if (a->coords_layout == FE_LAYOUT_SOA) {
                cudaMemcpy2DAsync(dX, size_t(K) * 8, X + c0 * 8, size_t(xs) * 8, size_t(m) * 8, nx, cudaMemcpyHostToDevice,
                                  ctx->s_in);
                cudaMemcpy2DAsync(dC, size_t(K) * cs, C + c0 * cs, size_t(cst) * cs, size_t(m) * cs, nc,
                                  cudaMemcpyHostToDevice, ctx->s_in);
                ca.coords_stride = K;
                ca.coefs_stride = K;
            } else {
                cudaMemcpyAsync(dX, X + c0 * nx * 8, size_t(m) * nx * 8, cudaMemcpyHostToDevice, ctx->s_in);
                cudaMemcpyAsync(dC, C + c0 * nc * cs, size_t(m) * nc * cs, cudaMemcpyHostToDevice, ctx->s_in);
            }
            ca.coords = reinterpret_cast<const double *>(dX);
            ca.coefs = dC;
            cudaEventRecord(in_done[slot], ctx->s_in);
            cudaStreamWaitEvent(ctx->s_comp, in_done[slot], 0);
        } else {
            if (a->coords_layout == FE_LAYOUT_SOA) {
                ca.coords = reinterpret_cast<const double *>(X + c0 * 8);
                ca.coefs = C + c0 * cs;
                ca.coords_stride = xs;
                ca.coefs_stride = cst;
            } else {
                ca.coords = reinterpret_cast<const double *>(X + c0 * nx * 8);
                ca.coefs = C + c0 * nc * cs;
            }
        }
        // outputs
        if (out_host) {
            co.A = ctx->stage[slot][2];
            co.b = ctx->stage[slot][3];
            co.flags = o->flags ? static_cast<uint8_t *>(ctx->stage[slot][4]) : nullptr;
            co.stride = K;
        } else {
            if (o->layout == FE_LAYOUT_SOA) {
                co.A = A + c0 * cs;
                co.b = B + c0 * cs;
                co.stride = os;
            } else {
                co.A = A + c0 * na * cs;
                co.b = B + c0 * ns * cs;
            }
            co.flags = o->flags ? o->flags + c0 : nullptr;
        }
        if (co.layout == FE_LAYOUT_SOA && out_host) co.stride = K;
        result = launch_set(ctx, type, &ca, &co, ctx->scratch, ctx->s_comp);
        cudaEventRecord(comp_done[slot], ctx->s_comp);
        if (out_host) {
            cudaStreamWaitEvent(ctx->s_out, comp_done[slot], 0);
            if (o->layout == FE_LAYOUT_SOA) {
                cudaMemcpy2DAsync(A + c0 * cs, size_t(os) * cs, co.A, size_t(K) * cs, size_t(m) * cs, na,
                                  cudaMemcpyDeviceToHost, ctx->s_out);
                cudaMemcpy2DAsync(B + c0 * cs, size_t(os) * cs, co.b, size_t(K) * cs, size_t(m) * cs, ns,
                                  cudaMemcpyDeviceToHost, ctx->s_out);
            } else {
                cudaMemcpyAsync(A + c0 * na * cs, co.A, size_t(m) * na * cs, cudaMemcpyDeviceToHost, ctx->s_out);
                cudaMemcpyAsync(B + c0 * ns * cs, co.b, size_t(m) * ns * cs, cudaMemcpyDeviceToHost, ctx->s_out);
            }
            if (o->flags) cudaMemcpyAsync(o->flags + c0, co.flags, size_t(m), cudaMemcpyDeviceToHost, ctx->s_out);
            cudaEventRecord(out_done[slot], ctx->s_out);
        } else {
            cudaEventRecord(out_done[slot], ctx->s_comp);
        }
    }
    cudaError_t e1 = cudaStreamSynchronize(ctx->s_in);
    cudaError_t e2 = cudaStreamSynchronize(ctx->s_comp);
    cudaError_t e3 = cudaStreamSynchronize(ctx->s_out);
    cudaEventDestroy(start);
    for (int i = 0; i < 2; ++i) {
        cudaEventDestroy(in_done[i]);
        cudaEventDestroy(comp_done[i]);
        cudaEventDestroy(out_done[i]);
    }
    if (result != FE_OK) return result;
    fe_status st = cuda_check(ctx, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3), "host pipeline");
    return st;
}

// Device address of pinned (page-locked, mapped) host memory, or null for
// pageable memory. Through NVLink-C2C (or PCIe) the kernels can then read and
// write the host buffers directly, with no staging copies.
static const void *mapped_host(const void *p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Host buffers that are all pinned: one launch on the mapped addresses, then wait.
static bool zero_copy(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *a, const fe_out *o, cudaStream_t s,
                      fe_status &st) {
    fe_elem_args da = *a;
    fe_out dout = *o;
    if (a->memory == FE_MEM_HOST) {
        da.coords = static_cast<const double *>(mapped_host(a->coords));
        da.coefs = mapped_host(a->coefs);
        if (!da.coords || !da.coefs) return false;
        da.memory = FE_MEM_DEVICE;
    }
    if (o->memory == FE_MEM_HOST) {
        dout.A = const_cast<void *>(mapped_host(o->A));
        dout.b = const_cast<void *>(mapped_host(o->b));
        dout.flags = o->flags ? static_cast<uint8_t *>(const_cast<void *>(mapped_host(o->flags))) : nullptr;
        if (!dout.A || !dout.b || (o->flags && !dout.flags)) return false;
        dout.memory = FE_MEM_DEVICE;
    }
    st = launch_set(ctx, type, &da, &dout, ctx->scratch, s);
    if (st == FE_OK) st = cuda_check(ctx, cudaStreamSynchronize(s), "zero-copy integration");
    return true;
}

static fe_status integrate(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *a, const fe_out *o, void *stream) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    fe_status st = fe_check_args(type, a, o);
    if (st != FE_OK) {
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->last_error = t_last_error;
        return st;
    }
    if (a->n_elem == 0) return FE_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (a->memory == FE_MEM_HOST || o->memory == FE_MEM_HOST) {
        fe_status zst = FE_OK;
        if (zero_copy(ctx, type, a, o, s, zst)) return zst;
        return host_pipeline(ctx, type, a, o, s);   // pageable memory: chunked, staged copies
    }
    if (ctx->autotune && !ctx->shapes.count(shape_key(type, a, o))) {
        st = fe_tune(ctx, type, a, o, stream);
        if (st != FE_OK) return st;
    }
    return launch_set(ctx, type, a, o, ctx->scratch, s);
}

static void load_tuning_cache(fe_ctx *ctx) {
    if (ctx->tuning_cache_path.empty()) return;
    std::ifstream f(ctx->tuning_cache_path);
    std::string line;
    while (std::getline(f, line)) {
        // device key elements persistent [threads-per-element]
        std::istringstream ls(line);
        std::string dev, key;
        int block = 0, pers = 0, tpe = 1;
        if (!(ls >> dev >> key >> block >> pers)) continue;
        if (!(ls >> tpe)) tpe = 1;
        if (dev == ctx->device_name && block > 0 && (tpe == 1 || tpe == 2 || tpe == 4 || tpe == 6 || tpe == 16) &&
            shape_threads(block, tpe))
            ctx->shapes[key] = Shape{block, pers, tpe};
    }
}

static void save_tuning_cache(fe_ctx *ctx) {
    if (ctx->tuning_cache_path.empty()) return;
    std::ofstream f(ctx->tuning_cache_path, std::ios::trunc);
    for (auto &kv : ctx->shapes)
        f << ctx->device_name << " " << kv.first << " " << kv.second.block << " " << kv.second.persistent << " "
          << kv.second.tpe << "\n";
}

}  // namespace fe

using namespace fe;

extern "C" {

fe_status fe_check_args(fe_elem_type type, const fe_elem_args *a, const fe_out *o) {
    if (type != FE_TET && type != FE_PRISM) return set_error(nullptr, FE_ERR_INVALID_ARG, "bad element type");
    if (!a || !o) return set_error(nullptr, FE_ERR_INVALID_ARG, "null args or out");
    if (a->n_elem < 0) return set_error(nullptr, FE_ERR_INVALID_ARG, "n_elem < 0");
    if (a->kind != FE_POISSON && a->kind != FE_GENERIC) return set_error(nullptr, FE_ERR_INVALID_ARG, "bad problem kind");
    if (a->prec != FE_FP64 && a->prec != FE_FP32_MIXED && a->prec != FE_FP64_DW)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "bad precision");
    if (a->coef_mode != FE_COEF_PER_ELEMENT && a->coef_mode != FE_COEF_PER_QPOINT && a->coef_mode != FE_COEF_FUNCTION_U)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "bad coefficient mode");
    if (a->coef_mode == FE_COEF_FUNCTION_U) {
        if (!a->coef_fn) return set_error(nullptr, FE_ERR_INVALID_ARG, "FE_COEF_FUNCTION_U without coef_fn");
        if (a->coords_layout != FE_LAYOUT_AOS || o->packed || a->ordering)
            return set_error(nullptr, FE_ERR_UNSUPPORTED,
                             "the coefficient function takes element-contiguous coordinates, full outputs, ordering 0");
    }
    if (type == FE_TET && a->quad != FE_QUAD_TET1 && a->quad != FE_QUAD_TET4)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "tetrahedra take FE_QUAD_TET1 or FE_QUAD_TET4");
    if (type == FE_PRISM && a->quad != FE_QUAD_PRISM6)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "prisms take FE_QUAD_PRISM6");
    if ((a->coords_layout != FE_LAYOUT_SOA && a->coords_layout != FE_LAYOUT_AOS && a->coords_layout != FE_LAYOUT_INDEXED) ||
        (o->layout != FE_LAYOUT_SOA && o->layout != FE_LAYOUT_AOS))
        return set_error(nullptr, FE_ERR_INVALID_ARG, "bad layout");
    const bool indexed = a->coords_layout == FE_LAYOUT_INDEXED;
    if (o->packed != 0 && o->packed != 1) return set_error(nullptr, FE_ERR_INVALID_ARG, "packed must be 0 or 1");
    if (a->ordering < 0 || a->ordering > 2) return set_error(nullptr, FE_ERR_INVALID_ARG, "ordering must be 0, 1 or 2");
    if (a->ordering && (a->prec != FE_FP32_MIXED || a->coords_layout != FE_LAYOUT_AOS || o->layout != FE_LAYOUT_AOS ||
                        o->packed))
        return set_error(nullptr, FE_ERR_UNSUPPORTED,
                         "the SQS and SSQ orderings take FE_FP32_MIXED with element-contiguous inputs and outputs");
    if (o->packed && a->kind != FE_POISSON)
        return set_error(nullptr, FE_ERR_UNSUPPORTED, "packed output needs a symmetric A^e (FE_POISSON)");
    if (o->packed && indexed)
        return set_error(nullptr, FE_ERR_UNSUPPORTED, "packed output is not available with a node table");
    if (indexed ? a->coefs_layout != FE_LAYOUT_AOS : a->coefs_layout != a->coords_layout)
        return set_error(nullptr, FE_ERR_UNSUPPORTED,
                         "coefficients must use the layout of the coordinates (element-contiguous with a node table)");
    if ((a->memory != FE_MEM_DEVICE && a->memory != FE_MEM_HOST) || (o->memory != FE_MEM_DEVICE && o->memory != FE_MEM_HOST))
        return set_error(nullptr, FE_ERR_INVALID_ARG, "bad memory kind");
    if (indexed && (a->memory != FE_MEM_DEVICE || o->memory != FE_MEM_DEVICE))
        return set_error(nullptr, FE_ERR_UNSUPPORTED, "a node table needs device memory");
    if (a->n_elem == 0) return FE_OK;
    if (!a->coords || !a->coefs || !o->A || !o->b) return set_error(nullptr, FE_ERR_INVALID_ARG, "null data pointer");
    if (indexed) {
        if (!a->conn || a->n_nodes <= 0 || a->n_nodes >= (int64_t(1) << 31))
            return set_error(nullptr, FE_ERR_INVALID_ARG, "node table: null conn or n_nodes outside [1, 2^31)");
        if (reinterpret_cast<uintptr_t>(a->conn) & 3) return set_error(nullptr, FE_ERR_INVALID_ARG, "misaligned conn");
    }
    const int64_t n = a->n_elem;
    // plane strides up to 2^40 elements: every plane offset (at most 120 planes)
    // stays far inside 64-bit addressing
    constexpr int64_t kMaxStride = int64_t(1) << 40;
    if (a->coords_layout == FE_LAYOUT_SOA) {
        if ((a->coords_stride != 0 && a->coords_stride < n) || (a->coefs_stride != 0 && a->coefs_stride < n))
            return set_error(nullptr, FE_ERR_INVALID_ARG, "SOA input stride smaller than n_elem");
        if (a->coords_stride > kMaxStride || a->coefs_stride > kMaxStride)
            return set_error(nullptr, FE_ERR_INVALID_ARG, "SOA input stride above 2^40");
    }
    if (o->layout == FE_LAYOUT_SOA && o->stride != 0 && o->stride < n)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "SOA output stride smaller than n_elem");
    if (o->layout == FE_LAYOUT_SOA && o->stride > kMaxStride)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "SOA output stride above 2^40");
    const unsigned cs = unsigned(csize(a->prec));
    if ((reinterpret_cast<uintptr_t>(a->coords) & 7) || (reinterpret_cast<uintptr_t>(a->coefs) & (cs - 1)) ||
        (reinterpret_cast<uintptr_t>(o->A) & (cs - 1)) || (reinterpret_cast<uintptr_t>(o->b) & (cs - 1)))
        return set_error(nullptr, FE_ERR_INVALID_ARG, "misaligned data pointer");
    if (n > 0xFFFFFFFFLL) return set_error(nullptr, FE_ERR_INVALID_ARG, "more than 2^32-1 elements in one call");
    return FE_OK;
}

int64_t fe_bytes_per_element(fe_elem_type type, fe_problem kind, fe_quad quad, fe_coef_mode mode, fe_precision prec) {
    if (type != FE_TET && type != FE_PRISM) return -1;
    if (kind != FE_POISSON && kind != FE_GENERIC) return -1;
    if (prec != FE_FP64 && prec != FE_FP32_MIXED && prec != FE_FP64_DW) return -1;
    if (type == FE_TET && quad != FE_QUAD_TET1 && quad != FE_QUAD_TET4) return -1;
    if (type == FE_PRISM && quad != FE_QUAD_PRISM6) return -1;
    if (mode != FE_COEF_PER_ELEMENT && mode != FE_COEF_PER_QPOINT && mode != FE_COEF_FUNCTION_U) return -1;
    fe_elem_args a{};
    a.kind = kind;
    a.quad = quad;
    a.coef_mode = mode;
    const int ns = ns_of(type), cs = csize(prec);
    return int64_t(3 * ns) * 8 + int64_t(nc_of(type, &a)) * cs + int64_t(ns * ns + ns) * cs;
}

fe_status fe_ctx_create(const fe_ctx_config *cfg, fe_ctx **out) {
    if (!out) return set_error(nullptr, FE_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    fe_ctx_config c{};
    if (cfg) c = *cfg;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return set_error(nullptr, FE_ERR_CUDA, "no CUDA device available");
    if (c.device < 0 || c.device >= ndev) return set_error(nullptr, FE_ERR_INVALID_ARG, "bad device ordinal");
    e = cudaSetDevice(c.device);
    if (e != cudaSuccess) return cuda_check(nullptr, e, "cudaSetDevice");
    fe_ctx *ctx = new fe_ctx();
    ctx->device = c.device;
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, c.device);
    ctx->sms = prop.multiProcessorCount;
    ctx->max_smem_optin = int(prop.sharedMemPerBlockOptin);
    ctx->device_name = prop.name;
    for (auto &ch : ctx->device_name)
        if (ch == ' ') ch = '_';
    ctx->autotune = c.autotune;
    ctx->hbm_budget = c.hbm_budget_bytes ? c.hbm_budget_bytes : 120000000000ull;
    ctx->serve_slots = c.serve_slots > 0 ? std::min(c.serve_slots, 64) : 4;
    if (c.tuning_cache_path) ctx->tuning_cache_path = c.tuning_cache_path;
    load_tuning_cache(ctx);
    fe_status st = ensure_scratch(ctx, ctx->scratch, 0);
    if (st != FE_OK) {
        delete ctx;
        return st;
    }
    cudaMallocHost(&ctx->h_status, sizeof(int));
    *out = ctx;
    return FE_OK;
}

fe_status fe_ctx_destroy(fe_ctx *ctx) {
    if (!ctx) return FE_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    serve_destroy(ctx);
    batch_destroy(ctx);
    cudaDeviceSynchronize();
    free_scratch(ctx->scratch);
    for (auto &kv : ctx->meshes) cudaFree(kv.second.coords);
    for (int s = 0; s < 2; ++s)
        for (int i = 0; i < 5; ++i)
            if (ctx->stage[s][i]) cudaFree(ctx->stage[s][i]);
    if (ctx->s_in) {
        cudaStreamDestroy(ctx->s_in);
        cudaStreamDestroy(ctx->s_comp);
        cudaStreamDestroy(ctx->s_out);
    }
    for (auto &pr : ctx->prof_events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto ev : ctx->event_pool) cudaEventDestroy(ev);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    delete ctx;
    return FE_OK;
}

fe_status fe_ctx_sync(fe_ctx *ctx) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_check(ctx, e, "device synchronize");
    if (ctx->scratch.status) {
        cudaMemcpy(ctx->h_status, ctx->scratch.status, sizeof(int), cudaMemcpyDeviceToHost);
        const int s = *ctx->h_status;
        if (s) {
            cudaMemset(ctx->scratch.status, 0, sizeof(int));
            if (s & ST_TMA_TIMEOUT) return set_error(ctx, FE_ERR_TIMEOUT, "a bulk copy wait ran out");
            if (s & ST_SKIPPED_TILES)
                return set_error(ctx, FE_ERR_PARTIAL, "tiles were skipped (injected fault): outputs incomplete");
            return set_error(ctx, FE_ERR_CUDA, "device status word " + std::to_string(s));
        }
    }
    if (ctx->async_error != FE_OK) {
        fe_status st = ctx->async_error;
        ctx->async_error = FE_OK;
        return st;
    }
    return FE_OK;
}

const char *fe_last_error(fe_ctx *ctx) {
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        t_last_error = ctx->last_error;
    }
    return t_last_error.c_str();
}

fe_status fe_integrate_tet(fe_ctx *ctx, const fe_elem_args *args, const fe_out *out, void *stream) {
    TraceRange tr("fe_integrate_tet");
    return integrate(ctx, FE_TET, args, out, stream);
}

fe_status fe_integrate_prism(fe_ctx *ctx, const fe_elem_args *args, const fe_out *out, void *stream) {
    TraceRange tr("fe_integrate_prism");
    return integrate(ctx, FE_PRISM, args, out, stream);
}

// Matrix-free application: the element kernels with the APPLY output mode.
static fe_status apply(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *a, const void *x, void *y, void *f,
                       uint8_t *flags, void *stream) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    fe_out o{};
    o.A = y;
    o.b = y;          // validation only: f may be null
    o.layout = FE_LAYOUT_AOS;
    o.flags = flags;
    o.memory = FE_MEM_DEVICE;
    fe_status st = fe_check_args(type, a, &o);
    if (st == FE_OK && a && a->coords_layout != FE_LAYOUT_INDEXED)
        st = set_error(nullptr, FE_ERR_UNSUPPORTED, "matrix-free application needs a node table (FE_LAYOUT_INDEXED)");
    const unsigned cs = a ? unsigned(csize(a->prec)) : 8;
    if (st == FE_OK && a->n_elem > 0 &&
        (!x || !y || (reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(f)) & (cs - 1)))
        st = set_error(nullptr, FE_ERR_INVALID_ARG, "null or misaligned x or y (or misaligned f)");
    if (st != FE_OK) {
        std::lock_guard<std::mutex> lk(ctx->err_mu);
        ctx->last_error = t_last_error;
        return st;
    }
    if (a->n_elem == 0) return FE_OK;
    cudaSetDevice(ctx->device);
    o.b = f;
    o.layout = static_cast<fe_layout>(kOutApply);
    // launch shape: the tuner cannot time this call (it accumulates into y), so a
    // key of its own gets the shape measured best for the unstaged node-table
    // kernels unless fe_set_shape chose one
    const std::string key = shape_key(type, a, &o);
    if (!ctx->shapes.count(key)) ctx->shapes[key] = Shape{64, 1};
    return launch_set(ctx, type, a, &o, ctx->scratch, static_cast<cudaStream_t>(stream), nullptr, x);
}

fe_status fe_apply_tet(fe_ctx *ctx, const fe_elem_args *args, const void *x, void *y, void *f, uint8_t *flags,
                       void *stream) {
    TraceRange tr("fe_apply_tet");
    return apply(ctx, FE_TET, args, x, y, f, flags, stream);
}

fe_status fe_apply_prism(fe_ctx *ctx, const fe_elem_args *args, const void *x, void *y, void *f, uint8_t *flags,
                         void *stream) {
    TraceRange tr("fe_apply_prism");
    return apply(ctx, FE_PRISM, args, x, y, f, flags, stream);
}

uint64_t fe_launch_count(void) { return g_launches.load(); }

fe_status fe_ctx_inject_fault(fe_ctx *ctx, fe_fault kind, int64_t count, int64_t param) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    if (count < 0) return set_error(ctx, FE_ERR_INVALID_ARG, "negative fault count");
    switch (kind) {
        case FE_FAULT_NONE:
            ctx->fail_allocs = 0;
            ctx->skip_launches = 0;
            ctx->skip_mod = 0;
            return FE_OK;
        case FE_FAULT_ALLOC:
            ctx->fail_allocs = count;
            return FE_OK;
        case FE_FAULT_SKIP_TILES:
            if (param < 1) return set_error(ctx, FE_ERR_INVALID_ARG, "tile period must be >= 1");
            ctx->skip_mod = param;
            ctx->skip_launches = count;
            return FE_OK;
    }
    return set_error(ctx, FE_ERR_INVALID_ARG, "unknown fault kind");
}

fe_status fe_selftest_bounded_wait(fe_ctx *ctx, unsigned polls, void *stream) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    if (polls == 0 || polls > (1u << 22)) return set_error(ctx, FE_ERR_INVALID_ARG, "polls must be in [1, 2^22]");
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *status = ctx->scratch.status;
    void *args[] = {&polls, &status};
    cudaError_t e = cudaLaunchKernel(kernel_selftest_wait(), dim3(1), dim3(32), args, 0, s);
    if (e != cudaSuccess) return cuda_check(ctx, e, "cudaLaunchKernel(selftest)");
    g_launches.fetch_add(1);
    return fe_ctx_sync(ctx);
}

fe_status fe_ctx_set_profiling(fe_ctx *ctx, int on) {
    if (!ctx) return FE_ERR_INVALID_ARG;
    ctx->profiling = on != 0;
    return FE_OK;
}

fe_status fe_ctx_kernel_time(fe_ctx *ctx, double *ms, int64_t *launches, int reset) {
    if (!ctx || !ms || !launches) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    cudaSetDevice(ctx->device);
    double total = 0.0;
    for (auto &pr : ctx->prof_events) {
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e != cudaSuccess) return cuda_check(ctx, e, "cudaEventSynchronize");
        float t = 0.0f;
        cudaEventElapsedTime(&t, pr.first, pr.second);
        total += t;
    }
    *ms = total;
    *launches = int64_t(ctx->prof_events.size());
    if (reset) {
        for (auto &pr : ctx->prof_events) {
            ctx->event_pool.push_back(pr.first);
            ctx->event_pool.push_back(pr.second);
        }
        ctx->prof_events.clear();
    }
    return FE_OK;
}

fe_status fe_get_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out, int *block_threads,
                       int *persistent) {
    if (!ctx || !block_threads || !persistent) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    fe_status st = fe_check_args(type, args, out);
    if (st != FE_OK) return st;
    Shape sh = default_shape(type);
    auto it = ctx->shapes.find(shape_key(type, args, out));
    if (it != ctx->shapes.end()) sh = it->second;
    *block_threads = shape_threads(sh.block, sh.tpe);
    *persistent = sh.persistent;
    return FE_OK;
}

fe_status fe_get_launch_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out,
                              fe_launch_shape *shape) {
    if (!ctx || !shape) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    fe_status st = fe_check_args(type, args, out);
    if (st != FE_OK) return st;
    Shape sh = default_shape(type);
    auto it = ctx->shapes.find(shape_key(type, args, out));
    if (it != ctx->shapes.end()) sh = it->second;
    shape->elems_per_block = sh.block;
    shape->threads_per_elem = sh.tpe;
    shape->persistent = sh.persistent;
    return FE_OK;
}

fe_status fe_set_launch_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out,
                              const fe_launch_shape *shape) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    if (!shape) return set_error(ctx, FE_ERR_INVALID_ARG, "null argument");
    fe_status st = fe_check_args(type, args, out);
    if (st != FE_OK) return st;
    const int B = shape->elems_per_block, t = shape->threads_per_elem;
    const int threads = (t == 1 || t == 2 || t == 4 || t == 6 || t == 16) ? shape_threads(B, t) : 0;
    if (!threads || threads > (t == 1 ? max_block(type, args->prec) : 256) ||
        (shape->persistent != 0 && shape->persistent != 1))
        return set_error(ctx, FE_ERR_INVALID_ARG, "bad launch shape");
    if (!tpe_ok(type, args, out_mode(out), t))
        return set_error(ctx, FE_ERR_UNSUPPORTED, "several threads per element: 2 for prisms, 4 or 16 for tetrahedra, "
                                                  "6 for prisms, with element-contiguous coordinates and outputs, "
                                                  "coefficient arrays and the QSS order only");
    if (smem_bytes(type, args, out_mode(out), B) + kStaticSmem > ctx->max_smem_optin)
        return set_error(ctx, FE_ERR_UNSUPPORTED, "shared memory of this launch shape too large");
    ctx->shapes[shape_key(type, args, out)] = Shape{B, shape->persistent, t};
    save_tuning_cache(ctx);
    return FE_OK;
}

fe_status fe_set_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out, int block_threads,
                       int persistent) {
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    fe_status st = fe_check_args(type, args, out);
    if (st != FE_OK) return st;
    if (block_threads < 32 || block_threads > max_block(type, args->prec) || block_threads % 32 || (persistent != 0 && persistent != 1))
        return set_error(ctx, FE_ERR_INVALID_ARG, "bad launch shape");
    if (smem_bytes(type, args, out_mode(out), block_threads) + kStaticSmem > ctx->max_smem_optin)
        return set_error(ctx, FE_ERR_UNSUPPORTED, "shared memory of this launch shape too large");
    ctx->shapes[shape_key(type, args, out)] = Shape{block_threads, persistent};
    save_tuning_cache(ctx);
    return FE_OK;
}

fe_status fe_tune(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *a, const fe_out *o, void *stream) {
    TraceRange tr("fe_tune");
    if (!ctx) return set_error(nullptr, FE_ERR_INVALID_ARG, "null context");
    fe_status st = fe_check_args(type, a, o);
    if (st != FE_OK) return st;
    if (a->memory != FE_MEM_DEVICE || o->memory != FE_MEM_DEVICE)
        return set_error(ctx, FE_ERR_INVALID_ARG, "tuning needs device buffers");
    if (a->n_elem == 0) return FE_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool was_prof = ctx->profiling;
    ctx->profiling = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Shape best_shape = default_shape(type);
    // candidates: elements per tile x grid kind, and with element-contiguous data
    // also several threads per element (2 or 6 per prism, 4 or 16 per
    // tetrahedron): blocks of 64 up to the kernel's limit of threads
    std::vector<Shape> cands;
    for (int tpe : {1, 2, 4, 6, 16}) {
        if (!tpe_ok(type, a, out_mode(o), tpe)) continue;
        const int lim = tpe == 1 ? max_block(type, a->prec) : 256, epw = 32 / tpe;
        for (int warps = 2; warps * 32 <= lim; warps *= 2)
            for (int pers = 0; pers < 2; ++pers) cands.push_back(Shape{warps * epw, pers, tpe});
    }
    for (const Shape &sh : cands) {
        if (smem_bytes(type, a, out_mode(o), sh.block) + kStaticSmem > ctx->max_smem_optin) continue;
        st = launch_set(ctx, type, a, o, ctx->scratch, s, &sh);  // warm-up
        if (st != FE_OK) break;
        cudaEventRecord(e0, s);
        const int reps = 3;
        for (int r = 0; r < reps && st == FE_OK; ++r) st = launch_set(ctx, type, a, o, ctx->scratch, s, &sh);
        cudaEventRecord(e1, s);
        if (st != FE_OK) break;
        cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) {
            st = cuda_check(ctx, ce, "tuning");
            break;
        }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) {
            best = t;
            best_shape = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->profiling = was_prof;
    if (st != FE_OK) return st;
    ctx->shapes[shape_key(type, a, o)] = best_shape;
    save_tuning_cache(ctx);
    return FE_OK;
}

}  // extern "C"
