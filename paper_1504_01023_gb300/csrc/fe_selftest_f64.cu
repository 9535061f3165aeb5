// Self-test of the integer-instruction double multiplication and addition
// (fe_f64int.cuh) against the double-precision instructions, per operation and
// through the FP64 tetrahedron arithmetic that uses them.
#include <cuda_runtime.h>

#include "fe_kernels.cuh"
#include "fe_runtime.h"

namespace fe {

__global__ void selftest_ops_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                    double *__restrict__ out_int, double *__restrict__ out_hw) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double a = x[i], b = y[i];
        out_int[i] = i64_dmul(a, b);
        out_hw[i] = __dmul_rn(a, b);
        out_int[n + i] = i64_dadd(a, b);
        out_hw[n + i] = __dadd_rn(a, b);
    }
}

// The products of i64_dmul_nz, completed by the DMUL instruction where it reports
// a special case.
__global__ void selftest_mul_nz_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                       double *__restrict__ out_int, double *__restrict__ out_hw) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double a = x[i], b = y[i];
        bool special = false;
        const double r = i64_dmul_nz(a, b, special);
        out_int[i] = special ? __dmul_rn(a, b) : r;
        out_hw[i] = __dmul_rn(a, b);
    }
}

// The sums of i64_dadd_nz, completed by the DADD instruction where it reports a
// special case.
__global__ void selftest_add_nz_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                       double *__restrict__ out_int, double *__restrict__ out_hw) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const double a = x[i], b = y[i];
        bool special = false;
        const double r = i64_dadd_nz(a, b, special);
        out_int[i] = special ? __dadd_rn(a, b) : r;
        out_hw[i] = __dadd_rn(a, b);
    }
}

// The FP64 tetrahedron arithmetic both ways: KIND 1 generic with TET4 and
// per-element coefficients (y: 20 per element), KIND 0 Laplace with TET1 (y: d^0
// per element); out: A^e (16) then b^e (4) per element, zeros for degenerate ones.
template <int KIND>
__global__ void selftest_tet_kernel(const double *__restrict__ x, const double *__restrict__ y, int64_t n,
                                    double *__restrict__ out_int, double *__restrict__ out_hw) {
    constexpr int NC = KIND ? 20 : 1;
    constexpr int QUAD = KIND ? Q_TET4 : Q_TET1;
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const Src<AOS, double> xs{x + e * 12, 0};
        const Src<AOS, double> cs{y + e * NC, 0};
        double *oi = out_int + e * 20, *oh = out_hw + e * 20;
        // returns true when an integer multiplication left a special case
        auto one = [&](auto tf, double *o) {
            using TF = decltype(tf);
            double a[3][3], det, A[16], b[4];
            bool sp = false;
            if (!TF::geometry(xs, a, det, sp)) {
                for (int k = 0; k < 20; ++k) o[k] = 0.0;
                return sp;
            }
            if constexpr (KIND)
                TF::template generic<QUAD>(a, det, cs, A, b, sp);
            else
                TF::template poisson<QUAD, 0>(a, det, cs, A, b, sp);
            for (int k = 0; k < 16; ++k) o[k] = A[k];
            for (int k = 0; k < 4; ++k) o[16 + k] = b[k];
            return sp;
        };
        using TH = TetF64<F64<false>, F64<false>, F64<false>, F64<false>>;
        // integer instructions throughout, redone on the double pipe on a special
        // case (as the kernels do), against the double pipe throughout
        if (one(TetF64<F64<true>, F64<true>, F64<true>, F64<true>>{}, oi)) one(TH{}, oi);
        one(TH{}, oh);
    }
}

}  // namespace fe

using namespace fe;

extern "C" fe_status fe_selftest_f64_int(int what, const double *x, const double *y, int64_t n, double *out_int,
                                         double *out_hw, void *stream) {
    if (what < 0 || what > 4 || n < 0 || (n > 0 && (!x || !y || !out_int || !out_hw)))
        return set_error(nullptr, FE_ERR_INVALID_ARG, "fe_selftest_f64_int: bad arguments");
    if (n == 0) return FE_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    if (what == 0)
        selftest_ops_kernel<<<unsigned(blocks), 256, 0, s>>>(x, y, n, out_int, out_hw);
    else if (what == 3)
        selftest_mul_nz_kernel<<<unsigned(blocks), 256, 0, s>>>(x, y, n, out_int, out_hw);
    else if (what == 4)
        selftest_add_nz_kernel<<<unsigned(blocks), 256, 0, s>>>(x, y, n, out_int, out_hw);
    else if (what == 1)
        selftest_tet_kernel<1><<<unsigned(blocks), 256, 0, s>>>(x, y, n, out_int, out_hw);
    else
        selftest_tet_kernel<0><<<unsigned(blocks), 256, 0, s>>>(x, y, n, out_int, out_hw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(nullptr, e, "fe_selftest_f64_int launch");
    g_launches.fetch_add(1);
    e = cudaStreamSynchronize(s);
    return cuda_check(nullptr, e, "fe_selftest_f64_int");
}
