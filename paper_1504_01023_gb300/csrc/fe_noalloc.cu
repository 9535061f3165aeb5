// Mixed-precision tetrahedron integration for callers that must not allocate.
//
// Some callers cannot call cudaMalloc: code running inside a memory arena that
// a host application owns (e.g. a solver that reserves all device memory up
// front and hands out slices), real-time loops that forbid allocator calls
// because they can block or fragment, and plugins that are not allowed to
// create a context. They still need the mixed-precision path, whose
// double-Jacobian fix-up pass uses scratch memory (a list of flagged elements,
// its counter and a status word). This file gives them one entry point whose
// scratch is a fixed, file-scope device array instead of an allocation.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (kScratchBytes) until the process exits. All calls share it
// and it keeps the last call's contents; each call clears the counter and the
// status word before its kernels run. Calls that overlap on the GPU (different
// streams or threads at the same time) race on the array and must not be made.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "fe_runtime.h"

namespace {

constexpr size_t kScratchBytes = size_t(4) << 20;             // 4 MiB per device
constexpr size_t kHeaderWords = 32;                             // counter, status (256 bytes)
constexpr uint64_t kListCap = kScratchBytes / 8 - kHeaderWords;  // flagged-element entries = max elements per call

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchBytes / 8];

struct DeviceSetup {
    bool done = false;
    unsigned long long *scratch = nullptr;
    int sms = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[256];

// Host code cannot pass the array's name to a kernel: it is a host-side stand-in.
// The device address comes from cudaGetSymbolAddress, once per device, with that
// device current. It is kept for the life of the process: a device reset by the
// host application unloads the module, and calls after one are not supported.
fe_status setup_device(int dev, DeviceSetup *&out) {
    if (dev < 0 || dev >= 256) return fe::set_error(nullptr, FE_ERR_INVALID_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return fe::cuda_check(nullptr, e, "cudaGetSymbolAddress(no-alloc scratch)");
        e = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fe::cuda_check(nullptr, e, "cudaDeviceGetAttribute");
        s.scratch = static_cast<unsigned long long *>(ptr);
        s.done = true;
    }
    out = &s;
    return FE_OK;
}

}  // namespace

extern "C" fe_status fe_integrate_tet_noalloc(const fe_elem_args *args, const fe_out *out, void *stream) {
    using namespace fe;
    fe_status st = fe_check_args(FE_TET, args, out);
    if (st != FE_OK) return st;
    if (args->prec != FE_FP32_MIXED)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "fe_integrate_tet_noalloc takes FE_FP32_MIXED only");
    if (args->memory != FE_MEM_DEVICE || out->memory != FE_MEM_DEVICE)
        return set_error(nullptr, FE_ERR_INVALID_ARG, "fe_integrate_tet_noalloc takes device buffers only");
    if (args->coords_layout == FE_LAYOUT_INDEXED || out->packed || args->coef_mode == FE_COEF_FUNCTION_U ||
        args->ordering != 0)
        return set_error(nullptr, FE_ERR_UNSUPPORTED,
                         "fe_integrate_tet_noalloc takes no node table, packed output, coefficient function or "
                         "loop ordering other than QSS");
    if (uint64_t(args->n_elem) > kListCap)
        return set_error(nullptr, FE_ERR_INVALID_ARG,
                         "n_elem exceeds the " + std::to_string(kListCap) +
                             "-element capacity of the static scratch of fe_integrate_tet_noalloc");
    if (args->n_elem == 0) return FE_OK;

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_check(nullptr, ce, "cudaGetDevice");
    DeviceSetup *s = nullptr;
    st = setup_device(dev, s);
    if (st != FE_OK) return st;

    const int cpq = args->coef_mode == FE_COEF_PER_QPOINT;
    const void *k = kernel_tet_mixed(args->kind, args->quad, cpq, args->coords_layout, out->layout);
    const void *fk = kernel_fixup_tet(args->kind, args->quad, cpq, args->coords_layout, out->layout);
    if (!k || !fk) return set_error(nullptr, FE_ERR_UNSUPPORTED, "no kernel for this combination");

    // 128 elements per block; shared memory = the tile's input and output records
    const int B = 128;
    const int nc = nc_of(FE_TET, args);
    auto r16 = [](int64_t v) { return (v + 15) / 16 * 16; };
    const int64_t smem_in = int64_t(B) * 12 * 8 + r16(int64_t(B) * nc * 4), smem_out = r16(int64_t(B) * 16 * 4) + r16(int64_t(B) * 4 * 4);
    const int64_t smem = smem_in > smem_out ? smem_in : smem_out;
    // raise the kernel's dynamic shared-memory limit if needed, never lower it,
    // through the same record as the other entry points that launch this kernel
    st = set_smem_attr(nullptr, k, smem);
    if (st != FE_OK) return st;

    cudaStream_t strm = static_cast<cudaStream_t>(stream);
    unsigned int *count = reinterpret_cast<unsigned int *>(s->scratch);
    int *status = reinterpret_cast<int *>(s->scratch + 1);
    ce = cudaMemsetAsync(s->scratch, 0, kHeaderWords * 8, strm);   // counter and status start at zero
    if (ce != cudaSuccess) return cuda_check(nullptr, ce, "cudaMemsetAsync(no-alloc scratch)");

    ElemParams p{};
    p.n = args->n_elem;
    p.X = args->coords;
    p.xs = args->coords_stride ? args->coords_stride : args->n_elem;
    p.C = args->coefs;
    p.cs = args->coefs_stride ? args->coefs_stride : args->n_elem;
    p.A = out->A;
    p.B = out->b;
    p.os = out->stride ? out->stride : args->n_elem;
    p.flags = out->flags;
    p.fix_list = s->scratch + kHeaderWords;
    p.fix_count = count;
    p.fix_cap = static_cast<unsigned>(kListCap);
    p.item = 0;
    p.status = status;
    TmaMaps no_maps;                                  // plane copies stay per-plane bulk copies here
    memset(&no_maps, 0, sizeof no_maps);
    CoefFn no_fn;                                     // coefficient arrays only here
    memset(&no_fn, 0, sizeof no_fn);
    void *kargs[] = {&p, &no_maps, &no_fn};
    const int64_t grid = (args->n_elem + B - 1) / B;
    ce = cudaLaunchKernel(k, dim3(unsigned(grid)), dim3(B), kargs, size_t(smem), strm);
    if (ce != cudaSuccess) return cuda_check(nullptr, ce, "cudaLaunchKernel(elem, no-alloc)");
    g_launches.fetch_add(1, std::memory_order_relaxed);
    int64_t fgrid = std::min<int64_t>((args->n_elem + 255) / 256, int64_t(s->sms) * 4);
    void *fargs[] = {&p, &no_fn};
    ce = cudaLaunchKernel(fk, dim3(unsigned(fgrid < 1 ? 1 : fgrid)), dim3(256), fargs, 0, strm);
    if (ce != cudaSuccess) return cuda_check(nullptr, ce, "cudaLaunchKernel(fixup, no-alloc)");
    g_launches.fetch_add(1, std::memory_order_relaxed);

    // The call returns when its kernels are done, so that it can report their
    // device status without any other entry point.
    ce = cudaStreamSynchronize(strm);
    if (ce != cudaSuccess) return cuda_check(nullptr, ce, "cudaStreamSynchronize");
    int h_status = 0;
    ce = cudaMemcpy(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_check(nullptr, ce, "cudaMemcpy(status)");
    if (h_status & ST_TMA_TIMEOUT) return set_error(nullptr, FE_ERR_TIMEOUT, "a bulk copy wait ran out");
    if (h_status) return set_error(nullptr, FE_ERR_CUDA, "device status word " + std::to_string(h_status));
    return FE_OK;
}
