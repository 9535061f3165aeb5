// Device-side building blocks of the integration kernels: reference rules,
// memory helpers, exact-enough edge vectors from double coordinates, and the
// per-element arithmetic of Sec. 2.2-2.3 (Eqs. sm_local, lv_local,
// change_of_variables, quadrature; Algorithms 2 and 3).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "fe_dword.cuh"
#include "fe_f64int.cuh"
#include "fe_internal.h"

namespace fe {

// ---------------------------------------------------------------------------
// Reference rules (Eq. quadrature). The paper only says "Gaussian"; the point
// sets are the readings documented in include/fe.h.
// ---------------------------------------------------------------------------
constexpr double kTet4A = 0.13819660112501051517954131656343618822796908201942;  // (5 - sqrt 5) / 20
constexpr double kTet4B = 0.58541019662496845446137605030969143531609275394172;  // (5 + 3 sqrt 5) / 20
constexpr double kInvSqrt3 = 0.57735026918962576450914878050195745564760175127013;

template <int QUAD> struct Rule;

template <> struct Rule<Q_TET1> {
    static constexpr int NQ = 1;
    __host__ __device__ static constexpr double w(int) { return 1.0 / 6.0; }
    // shape value phi_r at point q (shape functions = barycentric coordinates)
    __host__ __device__ static constexpr double phi(int, int) { return 0.25; }
};

template <> struct Rule<Q_TET4> {
    static constexpr int NQ = 4;
    __host__ __device__ static constexpr double w(int) { return 1.0 / 24.0; }
    // point q: barycentric weight B on vertex q, A on the other three
    __host__ __device__ static constexpr double phi(int q, int r) { return q == r ? kTet4B : kTet4A; }
};

template <> struct Rule<Q_PRISM6> {
    static constexpr int NQ = 6;  // q = 3*l + t: zeta level l, triangle point t
    __host__ __device__ static constexpr double w(int) { return 1.0 / 6.0; }
    // triangle point t: barycentric 2/3 on vertex t, 1/6 on the others
    __host__ __device__ static constexpr double lam(int t, int k) { return t == k ? 2.0 / 3.0 : 1.0 / 6.0; }
    // zeta = -1/sqrt3 (l = 0) or +1/sqrt3 (l = 1); zb = (1 - zeta)/2, zt = (1 + zeta)/2
    __host__ __device__ static constexpr double zb(int l) { return 0.5 * (1.0 + (l ? -kInvSqrt3 : kInvSqrt3)); }
    __host__ __device__ static constexpr double zt(int l) { return 0.5 * (1.0 + (l ? kInvSqrt3 : -kInvSqrt3)); }
    __host__ __device__ static constexpr double phi(int q, int r) {
        return r < 3 ? lam(q % 3, r) * zb(q / 3) : lam(q % 3, r - 3) * zt(q / 3);
    }
};

// Quadrature sums that do not depend on the element (Sec. 4.4 counts loop-invariant
// motion of such terms): W = sum w_q, m_r = sum w_q phi_r(q), M2_rs = sum w_q phi_r phi_s.
struct TetSums {
    double W, m[4], M2[4][4];
};
template <int QUAD> __host__ __device__ constexpr TetSums tet_sums() {
    TetSums s{};
    for (int q = 0; q < Rule<QUAD>::NQ; ++q) {
        s.W += Rule<QUAD>::w(q);
        for (int r = 0; r < 4; ++r) {
            s.m[r] += Rule<QUAD>::w(q) * Rule<QUAD>::phi(q, r);
            for (int c = 0; c < 4; ++c) s.M2[r][c] += Rule<QUAD>::w(q) * Rule<QUAD>::phi(q, r) * Rule<QUAD>::phi(q, c);
        }
    }
    return s;
}

// Mean-ratio shape test constants. q = 3 |det T|^{2/3} / ||T||_F^2 with T = J S^{-1},
// S the reference-to-ideal map; q < 0.1 <=> K det_J^2 / f^3 < 1e-3 with f = ||T||_F^2
// and K = 27 det(S^{-1})^2: tetrahedron det S^{-1} = sqrt 2 (K = 54), prism
// det S^{-1} = 4/sqrt 3 (K = 144).
constexpr float kQualityQ3 = 1.0e-3f;  // 0.1^3
constexpr float kTetQK = 54.0f;
constexpr float kPrismQK = 144.0f;

// ---------------------------------------------------------------------------
// Small vectors
// ---------------------------------------------------------------------------
template <class T> struct V3 {
    T x, y, z;
};
template <class T> __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> __device__ __forceinline__ V3<T> operator*(T s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T> __device__ __forceinline__ V3<T> operator-(V3<T> a) { return {-a.x, -a.y, -a.z}; }
template <class T> __device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
// Double-word dot and cross products: one fused accumulation per result.
__device__ __forceinline__ DW dot(V3<DW> a, V3<DW> b) {
    const DW x[3] = {a.x, a.y, a.z}, y[3] = {b.x, b.y, b.z};
    return dw_dot<3>(x, y);
}
__device__ __forceinline__ V3<DW> cross(V3<DW> a, V3<DW> b) {
    return {dw_diff_prod(a.y, b.z, a.z, b.y), dw_diff_prod(a.z, b.x, a.x, b.z), dw_diff_prod(a.x, b.y, a.y, b.x)};
}

// ---------------------------------------------------------------------------
// Memory helpers
// ---------------------------------------------------------------------------
template <class T> __device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }
template <class T> __device__ __forceinline__ void st_stream(T *p, T v) { __stcs(p, v); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// mbarrier + bulk copy (cp.async.bulk, the 1-D TMA path) for staging element
// blocks of the "natural" element-contiguous layout through shared memory
// (Sec. 4.2, Fig. 1 a: coalesced reading through shared memory).
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}
// 2-D tensor copies (plane-major tiles): box = (tile elements, planes), written
// to / read from shared memory as [planes][elements]. Loads fill elements past
// the array end with zeros, stores clip them.
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const void *tmap, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap), "r"(x), "r"(y),
                 "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait on an mbarrier phase. Returns false (and sets the status bit) if
// the copy has not landed after ~2^22 polls with back-off (seconds); callers
// then skip their work for this block instead of spinning forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase, int *status,
                                                  unsigned polls = 1u << 22) {
    for (unsigned it = 0; it < polls; ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if (it > 64) __nanosleep(256);
    }
    if (status) atomicOr(status, ST_TMA_TIMEOUT);
    return false;
}

// ---------------------------------------------------------------------------
// Double -> (hi, lo) float pair with integer operations only. The product needs
// edge vectors x_k - x_0 with float relative accuracy although x_k are absolute
// coordinates in double; rounding each coordinate to float first would lose
// ~|x|/h ulps. hi = x truncated to 24 significant bits, lo = x - hi (exact up to
// the last 6 of 53 bits). The double pipe of this GPU runs at 1/64 of the float
// rate, so no double instruction is used. Coordinates with |x| outside
// [2^-74, 2^128) (other than 0) give NaN, which fails the shape test and sends
// the element down the double-precision path.
// ---------------------------------------------------------------------------
struct HiLo {
    float hi, lo;
};
__device__ __forceinline__ HiLo split_double(double x) {
    const uint32_t h = static_cast<uint32_t>(__double2hiint(x));
    const uint32_t l = static_cast<uint32_t>(__double2loint(x));
    const uint32_t sign = h & 0x80000000u;
    const uint32_t e = (h >> 20) & 0x7FFu;                       // biased double exponent
    const uint32_t frac23 = ((h & 0xFFFFFu) << 3) | (l >> 29);    // top 23 fraction bits
    const uint32_t ehi = (e - 896u) << 23;                        // float exponent field of hi
    const uint32_t elo = (e - 919u) << 23;                        // float exponent of 2^(E-23)
    const float p = __uint_as_float(elo);
    // 2^(E-23) * (1 + next23 / 2^23) - 2^(E-23): exact by Sterbenz
    const float lo_mag = __uint_as_float(elo | ((l >> 6) & 0x7FFFFFu)) - p;
    const bool in_range = (e - 949u) <= (1150u - 949u);
    const bool zero = ((h & 0x7FFFFFFFu) | l) == 0u;
    HiLo r;
    r.hi = in_range ? __uint_as_float(sign | ehi | frac23) : (zero ? 0.0f : __uint_as_float(0x7FC00000u));
    r.lo = in_range ? __uint_as_float(__float_as_uint(lo_mag) | sign) : 0.0f;
    return r;
}
__device__ __forceinline__ float diff_hilo(HiLo a, HiLo b) { return (a.hi - b.hi) + (a.lo - b.lo); }

// ---------------------------------------------------------------------------
// Accessors for the per-element inputs. SOA: global planes (coalesced across
// the warp). AOS: the element's contiguous record staged in shared memory.
// ---------------------------------------------------------------------------
template <int LAYOUT, class T> struct Src {
    const T *base;   // SOA: global array; AOS: this element's record in shared memory
    int64_t stride;  // SOA plane stride
    __device__ __forceinline__ T operator()(int j) const {
        if (LAYOUT == SOA) return ld_stream(base + j * stride);
        return base[j];
    }
};

// ---------------------------------------------------------------------------
// Tetrahedron (Algorithm 3, QSS_geo_linear): Jacobian terms once per element.
// J = [e1 e2 e3] (columns x_k - x_0). Rows of J^{-1} are a_m / det with
// a_1 = e2 x e3, a_2 = e3 x e1, a_3 = e1 x e2, det = e1 . a_1; the global
// gradient of phi_m (m = 1..3) is row m of J^{-1} and grad phi_0 = -sum.
// ---------------------------------------------------------------------------
template <class T> struct TetGeo {
    V3<T> a[3];
    T det;
};
template <class T> __device__ __forceinline__ TetGeo<T> tet_geometry(V3<T> e1, V3<T> e2, V3<T> e3) {
    TetGeo<T> g;
    g.a[0] = cross(e2, e3);
    g.a[1] = cross(e3, e1);
    g.a[2] = cross(e1, e2);
    g.det = dot(e1, g.a[0]);
    return g;
}

// Shape test on float edges: true if the mean ratio is below 0.1 (or not finite).
// ||T||_F^2 = |e1|^2 + |2 e2 - e1|^2 / 3 + |3 e3 - e1 - e2|^2 / 6 for the
// equilateral ideal; q^3 = 54 det^2 / f^3.
__device__ __forceinline__ bool tet_poor(V3<float> e1, V3<float> e2, V3<float> e3, float det) {
    const V3<float> t1 = 2.0f * e2 - e1;
    const V3<float> t2 = 3.0f * e3 - e1 - e2;
    const float f = dot(e1, e1) + dot(t1, t1) * (1.0f / 3.0f) + dot(t2, t2) * (1.0f / 6.0f);
    const float r = rsqrtf(f);
    const float x = det * r * r * r;
    return !(kTetQK * x * x >= kQualityQ3);
}

// Coefficient products and accumulation for a tetrahedron, given the global
// gradients g[0..3] and V = |det J|. Per-element coefficients fold the Q loop
// into the reference sums W, m, M2 (loop-invariant motion, Sec. 3.3 end); per-point
// coefficients accumulate their weighted sums over Q first.
//   A_rs = V ( g_r . Cbar g_s + P_s . g_r + R_r . g_s + M_rs )
//   b_r  = V ( dbar . g_r + e_r )
// with Cbar = sum_q w c^{ij}, P_s = sum_q w phi_s c^{i0}, R_r = sum_q w phi_r c^{0i},
// M_rs = sum_q w c^{00} phi_r phi_s, dbar = sum_q w d^i, e_r = sum_q w d^0 phi_r.
template <class T, int QUAD, int CPQ, class CS>
__device__ __forceinline__ void tet_generic_products(const V3<T> g[4], T V, const CS &c, T A[16], T b[4]) {
    constexpr TetSums S = tet_sums<QUAD>();
    constexpr int NQ = Rule<QUAD>::NQ;
    V3<T> Cg[4];                 // Cbar g_s
    T conv[4][4];                // P_s . g_r + R_r . g_s
    T M[4][4];
    V3<T> db;
    T eb[4];
    if (!CPQ) {
        // P_s = m_s c^{i;0}, R_r = m_r c^{0;i}: conv_rs = m_s (c^{i0} . g_r) + m_r (c^{0i} . g_s)
        const V3<T> ci0 = {c(4), c(8), c(12)};
        const V3<T> c0i = {c(1), c(2), c(3)};
        T cr[4], cs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cr[k] = dot(ci0, g[k]);
            cs[k] = dot(c0i, g[k]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) conv[r][s] = T(S.m[s]) * cr[r] + T(S.m[r]) * cs[s];
        const T Wt = T(S.W);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            Cg[s].x = Wt * (c(5) * g[s].x + c(6) * g[s].y + c(7) * g[s].z);
            Cg[s].y = Wt * (c(9) * g[s].x + c(10) * g[s].y + c(11) * g[s].z);
            Cg[s].z = Wt * (c(13) * g[s].x + c(14) * g[s].y + c(15) * g[s].z);
        }
        const T c00 = c(0);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) M[r][s] = c00 * T(S.M2[r][s]);
        db = {Wt * c(17), Wt * c(18), Wt * c(19)};
        const T d0 = c(16);
#pragma unroll
        for (int r = 0; r < 4; ++r) eb[r] = d0 * T(S.m[r]);
    } else {
        T Cb[3][3];
        V3<T> P[4], R[4];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Cb[i][j] = T(0);
        db = {T(0), T(0), T(0)};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            eb[r] = T(0);
            P[r] = R[r] = {T(0), T(0), T(0)};
#pragma unroll
            for (int s = 0; s < 4; ++s) M[r][s] = T(0);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int o = 20 * q;
            const T w = T(Rule<QUAD>::w(q));
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Cb[i][j] += w * c(o + 4 * (i + 1) + (j + 1));
            const V3<T> ci0 = {w * c(o + 4), w * c(o + 8), w * c(o + 12)};
            const V3<T> c0i = {w * c(o + 1), w * c(o + 2), w * c(o + 3)};
            db = db + w * V3<T>{c(o + 17), c(o + 18), c(o + 19)};
            const T c00 = w * c(o);
            const T d0 = w * c(o + 16);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const T ph = T(Rule<QUAD>::phi(q, r));
                P[r] = P[r] + ph * ci0;
                R[r] = R[r] + ph * c0i;
                eb[r] += ph * d0;
#pragma unroll
                for (int s = 0; s < 4; ++s) M[r][s] += c00 * T(Rule<QUAD>::phi(q, r) * Rule<QUAD>::phi(q, s));
            }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            Cg[s].x = Cb[0][0] * g[s].x + Cb[0][1] * g[s].y + Cb[0][2] * g[s].z;
            Cg[s].y = Cb[1][0] * g[s].x + Cb[1][1] * g[s].y + Cb[1][2] * g[s].z;
            Cg[s].z = Cb[2][0] * g[s].x + Cb[2][1] * g[s].y + Cb[2][2] * g[s].z;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int s = 0; s < 4; ++s) conv[r][s] = dot(P[s], g[r]) + dot(R[r], g[s]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int s = 0; s < 4; ++s) A[4 * r + s] = V * (dot(g[r], Cg[s]) + conv[r][s] + M[r][s]);
        b[r] = V * (dot(db, g[r]) + eb[r]);
    }
}

// The same products for per-element coefficients with fewer operations (used
// where arithmetic, not memory, bounds the kernel). With g_0 = -(g_1 + g_2 + g_3):
//   K_rs = g_r . (V W C) g_s for r, s = 1..3; row and column 0 of K from the
//   vanishing sums;
//   convection m_r (c^{i0} . g_r) pairs with m_s: as m_r = W/4 for both rules,
//   V (P_s . g_r + R_r . g_s) = V W/4 (cr_r + cs_s);
//   mass V c^{00} M2_rs with M2 one value off the diagonal and one on it;
//   b_r = V W (d^i . g_r) + V d^0 W/4.
template <class T, int QUAD, class CS>
__device__ __forceinline__ void tet_generic_products_pe(const V3<T> g[3], T V, const CS &c, T A[16], T b[4]) {
    constexpr TetSums S = tet_sums<QUAD>();
    const T VW = V * T(S.W);
    V3<T> Crow[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) Crow[i] = {VW * c(4 * i + 5), VW * c(4 * i + 6), VW * c(4 * i + 7)};
    V3<T> CG[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) CG[s] = {dot(Crow[0], g[s]), dot(Crow[1], g[s]), dot(Crow[2], g[s])};
    T K[4][4];
#pragma unroll
    for (int r = 1; r < 4; ++r)
#pragma unroll
        for (int s = 1; s < 4; ++s) K[r][s] = dot(g[r - 1], CG[s - 1]);
#pragma unroll
    for (int s = 1; s < 4; ++s) K[0][s] = -(K[1][s] + K[2][s] + K[3][s]);
#pragma unroll
    for (int r = 1; r < 4; ++r) K[r][0] = -(K[r][1] + K[r][2] + K[r][3]);
    K[0][0] = -(K[0][1] + K[0][2] + K[0][3]);
    const V3<T> ci0 = {c(4), c(8), c(12)}, c0i = {c(1), c(2), c(3)};
    T cr[4], cs[4];
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        cr[k] = dot(ci0, g[k - 1]);
        cs[k] = dot(c0i, g[k - 1]);
    }
    cr[0] = -(cr[1] + cr[2] + cr[3]);
    cs[0] = -(cs[1] + cs[2] + cs[3]);
    const T Vm = V * T(S.W / 4);
    const T Vc00 = V * c(0);
    const T mo = Vc00 * T(S.M2[0][1]);
    T rho[4], sig[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        rho[k] = Vm * cr[k] + mo;
        sig[k] = Vm * cs[k];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) A[4 * r + s] = K[r][s] + rho[r] + sig[s];
    if constexpr (S.M2[0][0] != S.M2[0][1]) {
        const T dl = Vc00 * T(S.M2[0][0] - S.M2[0][1]);
#pragma unroll
        for (int r = 0; r < 4; ++r) A[5 * r] += dl;
    }
    const V3<T> dv = {c(17), c(18), c(19)};
    T t[4];
#pragma unroll
    for (int k = 1; k < 4; ++k) t[k] = dot(dv, g[k - 1]);
    t[0] = -(t[1] + t[2] + t[3]);
    const T e = Vm * c(16);
#pragma unroll
    for (int r = 0; r < 4; ++r) b[r] = VW * t[r] + e;
}

// z + x . y and 4 q - (p1 + p2 + p3): double with fused multiply-adds, double-word
// with one compensated accumulation each.
__device__ __forceinline__ double dot3_add(const double x[3], const double y[3], double z) {
    return fma(x[2], y[2], fma(x[1], y[1], fma(x[0], y[0], z)));
}
__device__ __forceinline__ DW dot3_add(const DW x[3], const DW y[3], DW z) { return dw_dot_add<3>(x, y, z); }
__device__ __forceinline__ float dot3_add(const float x[3], const float y[3], float z) {
    return fmaf(x[2], y[2], fmaf(x[1], y[1], fmaf(x[0], y[0], z)));
}
__device__ __forceinline__ float lin4(float p1, float p2, float p3, float q) { return fmaf(4.0f, q, -((p1 + p2) + p3)); }
__device__ __forceinline__ double lin4(double p1, double p2, double p3, double q) {
    return fma(4.0, q, -((p1 + p2) + p3));
}
__device__ __forceinline__ DW lin4(DW p1, DW p2, DW p3, DW q) { return dw_lin4(p1, p2, p3, q); }

// w / v in double for v in [2^-1022, 2^1021] (v > 0). The float reciprocal of v's
// leading 24 bits scaled by v's exponent (integer operations) gives y0 with a
// relative error below 2^-22; one step of the third-order Newton iteration
// (Householder) y = y0 (1 + e + e^2), e = 1 - v y0, leaves e^3 < 2^-66, so w y is
// within about an ulp of w / v: four double operations instead of a correctly
// rounded division (a few times as many on this GPU's double pipe).
__device__ __forceinline__ double recip_scaled(double v, double w) {
    const uint32_t hw = static_cast<uint32_t>(__double2hiint(v));
    const uint32_t lw = static_cast<uint32_t>(__double2loint(v));
    const uint32_t ev = (hw >> 20) & 0x7FFu;
    const float m = __uint_as_float(0x3F800000u | ((hw & 0xFFFFFu) << 3) | (lw >> 29));   // in [1, 2)
    const uint32_t rb = __float_as_uint(__frcp_rn(m));                                      // in (1/2, 1]
    const uint32_t er = (rb >> 23) & 0xFFu;
    // r 2^(1023 - ev): double exponent field er - 127 + 1023 - (ev - 1023)
    const uint32_t yh = ((er + 1919u - ev) << 20) | ((rb & 0x7FFFFFu) >> 3);
    const double y0 = __hiloint2double(static_cast<int>(yh), static_cast<int>(rb << 29));
    const double wy0 = w * y0;
    const double e = fma(-v, y0, 1.0);
    return fma(wy0, fma(e, e, e), wy0);
}

// Sign and degeneracy tests on the bit pattern (integer operations; the double
// comparisons issue on the double pipe): det < 0, and !(|det| > 1e-300) with NaN
// counted as degenerate (non-negative doubles order like their bit patterns).
__device__ __forceinline__ bool is_neg(double v) { return __double2hiint(v) < 0; }
__device__ __forceinline__ bool is_neg(float v) { return v < 0.0f; }
__device__ __forceinline__ bool is_neg(DW v) { return v.h < 0.0f; }
__device__ __forceinline__ bool degenerate_det(double det) {
    const long long vb = __double_as_longlong(det) & 0x7FFFFFFFFFFFFFFFll;
    return !(vb > __double_as_longlong(1e-300) && vb <= 0x7FF0000000000000ll);
}

// Generic tetrahedron with per-element coefficients as one bilinear form (FP64
// and double-word forms, whose arithmetic bounds the kernel). With the cofactor
// rows a_m = det J grad phi_m (m = 1..3), a_0 = -(a_1 + a_2 + a_3), the augmented
// rows at_r = (a_r, 1) and
//   M = [ f C      sm c^{i0} ]      f = W / |det J|, sm = sign(det J) W / 4,
//       [ sm c^{0j}   mu     ]      mu = |det J| c^{00} M2_01,
// every entry of A^e is at_r M at_s^T, plus (M2_00 - M2_01) |det J| c^{00} on
// the diagonal: the diffusion V W grad phi_r C grad phi_s, the convection
// V m (c^{i0} . grad phi_r) + V m (c^{0i} . grad phi_s) (m_r = W/4 for both rules)
// and the mass V c^{00} M2_rs of tet_generic_products_pe, regrouped (the same
// quadrature, another rounding order). Row and column 0 follow from
// at_0 = -(at_1 + at_2 + at_3) + (0, 0, 0, 4). Likewise b_r = at_r . (sW d, e)
// with sW = sign(det J) W, e = |det J| d^0 W / 4.
template <class T, int QUAD, class CS>
__device__ __forceinline__ void tet_generic_aug(const V3<T> a3[3], T f, T sm, T sW, T V, const CS &c, T A[16],
                                                T b[4]) {
    constexpr TetSums S = tet_sums<QUAD>();
    const T a[3][3] = {{a3[0].x, a3[0].y, a3[0].z}, {a3[1].x, a3[1].y, a3[1].z}, {a3[2].x, a3[2].y, a3[2].z}};
    T M[3][4], M3[4];          // rows i = 0..2 of M (columns 0..3), then row 3
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) M[i][j] = f * c(4 * (i + 1) + (j + 1));
        M[i][3] = sm * c(4 * (i + 1));
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) M3[j] = sm * c(j + 1);
    const T mu = (V * c(0)) * T(S.M2[0][1]);
    M3[3] = mu;
    // P_r = at_r M, r = 1..3, then P_0
    T P[4][4];
#pragma unroll
    for (int r = 1; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T col[3] = {M[0][k], M[1][k], M[2][k]};
            P[r][k] = dot3_add(a[r - 1], col, M3[k]);
        }
#pragma unroll
    for (int k = 0; k < 4; ++k) P[0][k] = lin4(P[1][k], P[2][k], P[3][k], M3[k]);
    // A_rs = P_r . at_s
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const T pr[3] = {P[r][0], P[r][1], P[r][2]};
#pragma unroll
        for (int s = 1; s < 4; ++s) A[4 * r + s] = dot3_add(pr, a[s - 1], P[r][3]);
        A[4 * r] = lin4(A[4 * r + 1], A[4 * r + 2], A[4 * r + 3], P[r][3]);
    }
    if constexpr (S.M2[0][0] != S.M2[0][1]) {
        // the diagonal of the mass term: M2_00 - M2_01 = M2_01 for TET4
        constexpr double ratio = (S.M2[0][0] - S.M2[0][1]) / S.M2[0][1];
        const T dl = ratio == 1.0 ? mu : mu * T(ratio);
#pragma unroll
        for (int r = 0; r < 4; ++r) A[5 * r] += dl;
    }
    const T d[3] = {sW * c(17), sW * c(18), sW * c(19)};
    const T e = (V * c(16)) * T(S.W / 4);
#pragma unroll
    for (int r = 1; r < 4; ++r) b[r] = dot3_add(a[r - 1], d, e);
    b[0] = lin4(b[1], b[2], b[3], e);
}

// ---------------------------------------------------------------------------
// Plain FP64 tetrahedra with explicit double operations. Each group of
// multiplications and additions runs on the double pipe (F64<false>) or in
// integer instructions (F64<true>): OE the edge vectors, OX the products of the
// cofactors and det J, OM the scalings of the coefficients and of det J, OS the
// sums of rows and columns; the fused multiply-adds always on the double pipe.
// Every choice gives the same bits (the same IEEE operations in the same order).
// An integer multiplication that meets an operand or a product outside the
// normal range (zero aside) sets `sp`; the caller then redoes the element with
// the double pipe, as TetF64 with F64<false> throughout.
// The arithmetic is that of tet_geometry, recip_scaled and tet_generic_aug /
// tet_poisson_products, written out with explicit operations.
// ---------------------------------------------------------------------------
template <class OE, class OX, class OM, class OS> struct TetF64 {
    using O = F64<false>;   // fused multiply-adds
    // a = u x v, component i = u_j v_k - u_k v_j as fma(u_j, v_k, -(u_k v_j))
    __device__ __forceinline__ static void cross(const double u[3], const double v[3], double w[3], bool &sp) {
        w[0] = O::fma(u[1], v[2], -OX::mul(u[2], v[1], sp));
        w[1] = O::fma(u[2], v[0], -OX::mul(u[0], v[2], sp));
        w[2] = O::fma(u[0], v[1], -OX::mul(u[1], v[0], sp));
    }
    template <class OP = OX>
    __device__ __forceinline__ static double dot3(const double u[3], const double v[3], bool &sp) {
        return O::fma(u[2], v[2], O::fma(u[1], v[1], OP::mul(u[0], v[0], sp)));
    }
    __device__ __forceinline__ static double dot3_add(const double u[3], const double v[3], double z) {
        return O::fma(u[2], v[2], O::fma(u[1], v[1], O::fma(u[0], v[0], z)));
    }
    // 4 q - (p1 + p2 + p3)
    __device__ __forceinline__ static double lin4(double p1, double p2, double p3, double q, bool &sp) {
        return O::fma(4.0, q, -OS::add(OS::add(p1, p2, sp), p3, sp));
    }
    // w / v as recip_scaled
    __device__ __forceinline__ static double recip_w(double v, double w, bool &sp) {
        const uint32_t hw = static_cast<uint32_t>(__double2hiint(v));
        const uint32_t lw = static_cast<uint32_t>(__double2loint(v));
        const uint32_t ev = (hw >> 20) & 0x7FFu;
        const float m = __uint_as_float(0x3F800000u | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
        const uint32_t rb = __float_as_uint(__frcp_rn(m));
        const uint32_t er = (rb >> 23) & 0xFFu;
        const uint32_t yh = ((er + 1919u - ev) << 20) | ((rb & 0x7FFFFFu) >> 3);
        const double y0 = __hiloint2double(static_cast<int>(yh), static_cast<int>(rb << 29));
        const double wy0 = OM::mul(w, y0, sp);
        const double e = O::fma(-v, y0, 1.0);
        return O::fma(wy0, O::fma(e, e, e), wy0);
    }
    // Edge vectors, cofactor rows a_1..a_3 and det J of the element; false if
    // degenerate (!(|det J| > 1e-300), NaN included).
    template <class XS>
    __device__ __forceinline__ static bool geometry(const XS &x, double a[3][3], double &det, bool &sp) {
        double e[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int i = 0; i < 3; ++i) e[k][i] = OE::add(x(3 * (k + 1) + i), -x(i), sp);
        cross(e[1], e[2], a[0], sp);
        cross(e[2], e[0], a[1], sp);
        cross(e[0], e[1], a[2], sp);
        det = dot3(e[0], a[0], sp);
        return !degenerate_det(det);
    }
    // tet_generic_aug with explicit operations
    template <int QUAD, class CS>
    __device__ __forceinline__ static void generic(const double a[3][3], double det, const CS &c, double A[16],
                                                   double b[4], bool &sp) {
        constexpr TetSums S = tet_sums<QUAD>();
        const bool neg = is_neg(det);
        const double V = fabs(det);
        const double f = recip_w(V, S.W, sp);
        const double sm = neg ? -S.W / 4 : S.W / 4, sW = neg ? -S.W : S.W;
        double M[3][4], M3[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
#pragma unroll
            for (int j = 0; j < 3; ++j) M[i][j] = OM::mul(f, c(4 * (i + 1) + (j + 1)), sp);
            M[i][3] = OM::mul(sm, c(4 * (i + 1)), sp);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) M3[j] = OM::mul(sm, c(j + 1), sp);
        const double mu = OM::mul(OM::mul(V, c(0), sp), S.M2[0][1], sp);
        M3[3] = mu;
        double P[4][4];
#pragma unroll
        for (int r = 1; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double col[3] = {M[0][k], M[1][k], M[2][k]};
                P[r][k] = dot3_add(a[r - 1], col, M3[k]);
            }
#pragma unroll
        for (int k = 0; k < 4; ++k) P[0][k] = lin4(P[1][k], P[2][k], P[3][k], M3[k], sp);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const double pr[3] = {P[r][0], P[r][1], P[r][2]};
#pragma unroll
            for (int s = 1; s < 4; ++s) A[4 * r + s] = dot3_add(pr, a[s - 1], P[r][3]);
            A[4 * r] = lin4(A[4 * r + 1], A[4 * r + 2], A[4 * r + 3], P[r][3], sp);
        }
        if constexpr (S.M2[0][0] != S.M2[0][1]) {
            constexpr double ratio = (S.M2[0][0] - S.M2[0][1]) / S.M2[0][1];
            const double dl = ratio == 1.0 ? mu : OM::mul(mu, ratio, sp);
#pragma unroll
            for (int r = 0; r < 4; ++r) A[5 * r] = OS::add(A[5 * r], dl, sp);
        }
        const double d[3] = {OM::mul(sW, c(17), sp), OM::mul(sW, c(18), sp), OM::mul(sW, c(19), sp)};
        const double e = OM::mul(OM::mul(V, c(16), sp), S.W / 4, sp);
#pragma unroll
        for (int r = 1; r < 4; ++r) b[r] = dot3_add(a[r - 1], d, e);
        b[0] = lin4(b[1], b[2], b[3], e, sp);
    }
    // tet_poisson_products with explicit operations: A_rs = W / |det| a_r . a_s
    // (r, s = 1..3), row and column 0 from the vanishing sums; b as tet_poisson_b.
    template <int QUAD, int CPQ, class CS>
    __device__ __forceinline__ static void poisson(const double a[3][3], double det, const CS &c, double A[16],
                                                   double b[4], bool &sp) {
        constexpr TetSums S = tet_sums<QUAD>();
        const double V = fabs(det);
        const double k = recip_w(V, S.W, sp);
        double G[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = r; s < 3; ++s) G[r][s] = G[s][r] = OM::mul(k, dot3<OM>(a[r], a[s], sp), sp);
        double row0[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) row0[s] = -OS::add(OS::add(G[0][s], G[1][s], sp), G[2][s], sp);
        A[0] = -OS::add(OS::add(row0[0], row0[1], sp), row0[2], sp);
#pragma unroll
        for (int s = 0; s < 3; ++s) A[1 + s] = A[4 * (1 + s)] = row0[s];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = 0; s < 3; ++s) A[4 * (r + 1) + (s + 1)] = G[r][s];
        if constexpr (!CPQ || Rule<QUAD>::NQ == 1) {
            // d^0 per element or a one-point rule: b_r = V d0 m_r, m_r = W / 4
            const double vd = OM::mul(OM::mul(V, c(0), sp), S.m[0], sp);   // m_r = W / 4 for both rules
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] = vd;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] = 0.0;
#pragma unroll
            for (int q = 0; q < Rule<QUAD>::NQ; ++q) {
                const double wd = OM::mul(Rule<QUAD>::w(q), c(q), sp);
#pragma unroll
                for (int r = 0; r < 4; ++r) b[r] = O::fma(wd, Rule<QUAD>::phi(q, r), b[r]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] = OM::mul(b[r], V, sp);
        }
    }
};

// Laplace load vector: b_r = V sum_q w_q d0_q phi_r(q) (d0 per element: V d0 m_r).
template <class T, int QUAD, int CPQ, class CS> __device__ __forceinline__ void tet_poisson_b(T V, const CS &c, T b[4]) {
    constexpr TetSums S = tet_sums<QUAD>();
    if (!CPQ) {
        const T vd = V * c(0);
#pragma unroll
        for (int r = 0; r < 4; ++r) b[r] = vd * T(S.m[r]);
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) b[r] = T(0);
#pragma unroll
        for (int q = 0; q < Rule<QUAD>::NQ; ++q) {
            const T wd = T(Rule<QUAD>::w(q)) * c(q);
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] += wd * T(Rule<QUAD>::phi(q, r));
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) b[r] *= V;
    }
}

// Poisson tetrahedron: A_rs = W / |det| (a_r . a_s) for r,s = 1..3; row and column 0
// from the vanishing row sums (sum_k grad phi_k = 0); b_r = |det| sum_q w d0_q phi_r(q).
template <class T, int QUAD, int CPQ, class CS>
__device__ __forceinline__ void tet_poisson_products(const TetGeo<T> &geo, T invabs, T V, const CS &c, T A[16], T b[4]) {
    constexpr TetSums S = tet_sums<QUAD>();
    const T k = T(S.W) * invabs;
    T G[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = r; s < 3; ++s) {
            G[r][s] = k * dot(geo.a[r], geo.a[s]);
            G[s][r] = G[r][s];
        }
    T row0[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) row0[s] = -(G[0][s] + G[1][s] + G[2][s]);
    const T a00 = -(row0[0] + row0[1] + row0[2]);
    A[0] = a00;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        A[1 + s] = row0[s];
        A[4 * (1 + s)] = row0[s];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) A[4 * (r + 1) + (s + 1)] = G[r][s];
    tet_poisson_b<T, QUAD, CPQ>(V, c, b);
}

// Poisson tetrahedron from gradients (used by the double-Jacobian fix-up).
template <class T, int QUAD, int CPQ, class CS>
__device__ __forceinline__ void tet_poisson_from_grads(const V3<T> g[4], T V, const CS &c, T A[16], T b[4]) {
    constexpr TetSums S = tet_sums<QUAD>();
    const T k = T(S.W) * V;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = r; s < 4; ++s) {
            const T v = k * dot(g[r], g[s]);
            A[4 * r + s] = v;
            A[4 * s + r] = v;
        }
    if (!CPQ) {
        const T vd = V * c(0);
#pragma unroll
        for (int r = 0; r < 4; ++r) b[r] = vd * T(S.m[r]);
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) b[r] = T(0);
#pragma unroll
        for (int q = 0; q < Rule<QUAD>::NQ; ++q) {
            const T wd = T(Rule<QUAD>::w(q)) * c(q);
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] += wd * T(Rule<QUAD>::phi(q, r));
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) b[r] *= V;
    }
}

// ---------------------------------------------------------------------------
// Prism (Algorithm 2, QSS_geo_generic): Jacobian terms at every point.
// With r_k = x_k - x_0, the columns of J at (xi, eta, zeta) are
//   d x / d xi   = zb (r1 - r0) + zt (r4 - r3)
//   d x / d eta  = zb (r2 - r0) + zt (r5 - r3)
//   d x / d zeta = 1/2 sum_k lambda_k (r_{k+3} - r_k)
// (the derivatives of phi_k = lambda_k zb, phi_{k+3} = lambda_k zt). Rows of
// J^{-1}: rho_1 = (cy x cz)/det, rho_2 = (cz x cx)/det, rho_3 = (cx x cy)/det.
// grad phi_k = zb P_k - lambda_k/2 rho_3, grad phi_{k+3} = zt P_k + lambda_k/2 rho_3
// with P_0 = -(rho_1 + rho_2), P_1 = rho_1, P_2 = rho_2.
// ---------------------------------------------------------------------------
template <class T> struct PrismFrame {
    V3<T> ub, ut, vb, vt, w0, w1, w2;
};
template <class T> __device__ __forceinline__ PrismFrame<T> prism_frame(const V3<T> r[6]) {
    PrismFrame<T> f;
    f.ub = r[1] - r[0];
    f.ut = r[4] - r[3];
    f.vb = r[2] - r[0];
    f.vt = r[5] - r[3];
    f.w0 = r[3] - r[0];
    f.w1 = r[4] - r[1];
    f.w2 = r[5] - r[2];
    return f;
}

// 1/v: in double the scaled float reciprocal and one third-order Newton step
// (recip_scaled, within about an ulp; v's sign copied with integer operations);
// in float the hardware reciprocal (within 2 ulp), ample for the float form's
// tolerance; both far cheaper than a correctly rounded division.
__device__ __forceinline__ double recip_fast(double v) {
    const double r = recip_scaled(fabs(v), 1.0);
    return __hiloint2double(__double2hiint(r) | (__double2hiint(v) & int(0x80000000u)), __double2loint(r));
}
__device__ __forceinline__ float recip_fast(float v) { return __fdividef(1.0f, v); }
__device__ __forceinline__ DW recip_fast(DW v) { return dw_recip(v); }

// Global gradients at point (l, t) of PRISM6. Returns det J.
template <class T>
__device__ __forceinline__ T prism_point(const PrismFrame<T> &f, V3<T> cx, V3<T> cy, V3<T> a3, int l, int t, V3<T> g[6],
                                         V3<T> &cz_out) {
    using R = Rule<Q_PRISM6>;
    // lambda_k / 2 at triangle point t (t may be a run-time index): 1/3 or 1/12
    const T h0 = t == 0 ? T(1.0 / 3.0) : T(1.0 / 12.0), h1 = t == 1 ? T(1.0 / 3.0) : T(1.0 / 12.0),
            h2 = t == 2 ? T(1.0 / 3.0) : T(1.0 / 12.0);
    const V3<T> cz = h0 * f.w0 + h1 * f.w1 + h2 * f.w2;
    const V3<T> a1 = cross(cy, cz);
    const V3<T> a2 = cross(cz, cx);
    const T det = dot(cx, a1);
    const T inv = recip_fast(det);
    const V3<T> r1 = inv * a1, r2 = inv * a2, r3 = inv * a3;
    const V3<T> P[3] = {-(r1 + r2), r1, r2};
    const T zb = l ? T(R::zb(1)) : T(R::zb(0)), zt = l ? T(R::zt(1)) : T(R::zt(0));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T hl = k == 0 ? h0 : (k == 1 ? h1 : h2);
        g[k] = zb * P[k] - hl * r3;
        g[k + 3] = zt * P[k] + hl * r3;
    }
    cz_out = cz;
    return det;
}

// Shape test at a prism point: ideal = unit-edge equilateral triangle x unit height;
// ||T||_F^2 = |cx|^2 + |2 cy - cx|^2 / 3 + 4 |cz|^2; q^3 = 144 det^2 / f^3.
__device__ __forceinline__ bool prism_poor(float fxy, V3<float> cz, float det) {
    const float f = fxy + 4.0f * dot(cz, cz);
    const float r = rsqrtf(f);
    const float x = det * r * r * r;
    return !(kPrismQK * x * x >= kQualityQ3);
}

// Generic coefficient products at one prism point (the S x S x (N_D+1)^2 update of
// Algorithm 2): T_as = sum_b vol c_ab Phi_bs, A_rs += sum_a Phi_ar T_as;
// b_r += sum_a vol d_a Phi_ar. Phi_0s = phi_s(q), Phi_is = (grad phi_s)_i.
template <class T, int Q, class CS>
__device__ __forceinline__ void prism_generic_update(const V3<T> g[6], T vol, const CS &c, int o, T A[36], T b[6]) {
    T C[4][4], d[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) C[a][bb] = vol * c(o + 4 * a + bb);
        d[a] = vol * c(o + 16 + a);
    }
    T Tm[4][6];
#pragma unroll
    for (int s = 0; s < 6; ++s) {
        const T ph = T(Rule<Q_PRISM6>::phi(Q, s));
#pragma unroll
        for (int a = 0; a < 4; ++a) Tm[a][s] = C[a][0] * ph + C[a][1] * g[s].x + C[a][2] * g[s].y + C[a][3] * g[s].z;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const T ph = T(Rule<Q_PRISM6>::phi(Q, r));
#pragma unroll
        for (int s = 0; s < 6; ++s)
            A[6 * r + s] += ph * Tm[0][s] + g[r].x * Tm[1][s] + g[r].y * Tm[2][s] + g[r].z * Tm[3][s];
        b[r] += d[0] * ph + d[1] * g[r].x + d[2] * g[r].y + d[3] * g[r].z;
    }
}

// A^e and b^e of the generic prism, accumulated as unnormalised double-word
// pairs by its level expansion (level_expand), made double-words again (no-op
// for the other types).
template <class T> __device__ __forceinline__ void prism_dw_normalise(T A[36], T b[6]) {
    if constexpr (std::is_same<T, DW>::value) {
#pragma unroll
        for (int k = 0; k < 36; ++k) A[k] = dw_acc_norm(A[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) b[k] = dw_acc_norm(b[k]);
    }
}

// Poisson products at one prism point: A_rs += vol grad phi_r . grad phi_s,
// b_r += vol d0_q phi_r(q) (upper triangle accumulated; mirrored at the end).
template <class T, int Q>
__device__ __forceinline__ void prism_poisson_update(const V3<T> g[6], T vol, T d0, T A[36], T b[6]) {
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const V3<T> gr = vol * g[r];
#pragma unroll
        for (int s = r; s < 6; ++s) A[6 * r + s] += dot(gr, g[s]);
        b[r] += (vol * d0) * T(Rule<Q_PRISM6>::phi(Q, r));
    }
}

// Laplace matrix of a prism from the Gram terms of J^{-1} (the sum over the six
// points of vol grad phi_m . grad phi_n, regrouped; the same quadrature as
// Algorithm 2, different rounding order).
//
// At a point (l, t), with rho_i the rows of J^{-1} and h_a = lambda_a(t)/2,
//   grad phi_m = z_m P_a + sigma_m h_a rho_3     (a = m mod 3),
// where z_m = zb(l), sigma_m = -1 for the bottom nodes, z_m = zt(l), sigma_m = +1
// for the top ones, and P_0 = -(rho_1 + rho_2), P_1 = rho_1, P_2 = rho_2. Every
// product vol grad phi_m . grad phi_n is then a combination, with coefficients
// fixed by the rule, of the six terms gamma_ij = vol rho_i . rho_j =
// (w / |det J|) a_i . a_j (a_i = det J rho_i, the cross products of the columns
// of J):
//   z_m z_n Pi_ab + sigma_n z_m h_b pi_a + sigma_m z_n h_a pi_b + sigma_m sigma_n h_a h_b gamma_33,
// Pi_ab = vol P_a . P_b (linear in gamma_11, gamma_12, gamma_22) and
// pi_a = vol P_a . rho_3 (linear in gamma_13, gamma_23). Summed over the points,
// each coefficient factors into a level part and a triangle-point part, so the
// point loop keeps only
//   L[l]    = sum over the points t of level l of (gamma_11, gamma_12, gamma_22),
//   v[l][t] = (gamma_13, gamma_23) at every point,
//   c3[t]   = sum over the two levels of gamma_33 at triangle point t,
// and this function forms the 21 distinct entries from them (upper triangle of
// A, row-major 6 x 6; the lower triangle is left alone).
template <class T>
__device__ __forceinline__ void prism_laplace_assemble(const T L[2][3], const T v[2][3][2], const T c3[3], T A[36]) {
    using R = Rule<Q_PRISM6>;
    constexpr double zb0 = R::zb(0), zb1 = R::zb(1), zt0 = R::zt(0), zt1 = R::zt(1);
    // z_m z_n summed over the levels: bottom-bottom, top-top, bottom-top
    T Pi[3][3][3];   // [pair kind][a][b]
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double w0 = k == 0 ? zb0 * zb0 : (k == 1 ? zt0 * zt0 : zb0 * zt0);
        const double w1 = k == 0 ? zb1 * zb1 : (k == 1 ? zt1 * zt1 : zb1 * zt1);
        T g[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) g[j] = T(w0) * L[0][j] + T(w1) * L[1][j];
        Pi[k][1][1] = g[0];
        Pi[k][2][2] = g[2];
        Pi[k][1][2] = Pi[k][2][1] = g[1];
        Pi[k][0][1] = Pi[k][1][0] = -(g[0] + g[1]);
        Pi[k][0][2] = Pi[k][2][0] = -(g[1] + g[2]);
        Pi[k][0][0] = (g[0] + g[2]) + T(2.0) * g[1];
    }
    // nu[side][b] = sum_l z_side(l) sum_t h_b(t) v[l][t], h_b(t) = 1/12 + delta_bt / 4;
    // then pi[side][a][b] = pi_a(nu[side][b])
    T pi[2][3][3];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const double z0 = side ? zt0 : zb0, z1 = side ? zt1 : zb1;
        T V[2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
            V[i] = T(z0 / 12.0) * ((v[0][0][i] + v[0][1][i]) + v[0][2][i]) +
                   T(z1 / 12.0) * ((v[1][0][i] + v[1][1][i]) + v[1][2][i]);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            const T n0 = V[0] + (T(z0 / 4.0) * v[0][bb][0] + T(z1 / 4.0) * v[1][bb][0]);
            const T n1 = V[1] + (T(z0 / 4.0) * v[0][bb][1] + T(z1 / 4.0) * v[1][bb][1]);
            pi[side][1][bb] = n0;
            pi[side][2][bb] = n1;
            pi[side][0][bb] = -(n0 + n1);
        }
    }
    // H_ab = sum_t h_a(t) h_b(t) c3[t]
    const T C = T(1.0 / 144.0) * ((c3[0] + c3[1]) + c3[2]);
    T H[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        H[a][a] = C + T(15.0 / 144.0) * c3[a];
#pragma unroll
        for (int bb = a + 1; bb < 3; ++bb) H[a][bb] = H[bb][a] = C + T(3.0 / 144.0) * (c3[a] + c3[bb]);
    }
#pragma unroll
    for (int m = 0; m < 6; ++m) {
#pragma unroll
        for (int n = m; n < 6; ++n) {
            const int a = m % 3, bb = n % 3;
            const bool tm = m >= 3, tn = n >= 3;
            const T p = Pi[tm == tn ? (tm ? 1 : 0) : 2][a][bb];
            const T x = pi[tm ? 1 : 0][a][bb];   // z_m h_b pi_a, sign sigma_n
            const T y = pi[tn ? 1 : 0][bb][a];   // z_n h_a pi_b, sign sigma_m
            const T cross_terms = (tn ? x : -x) + (tm ? y : -y);
            A[6 * m + n] = p + cross_terms + (tm == tn ? H[a][bb] : -H[a][bb]);
        }
    }
}

// Partner exchange of two threads per element (lanes 2j and 2j+1 of a warp;
// `mask` holds every lane that takes part, both lanes of each pair).
__device__ __forceinline__ float pair_other(float v, unsigned mask) { return __shfl_xor_sync(mask, v, 1); }
__device__ __forceinline__ double pair_other(double v, unsigned mask) { return __shfl_xor_sync(mask, v, 1); }
__device__ __forceinline__ DW pair_other(DW v, unsigned mask) {
    return DW(__shfl_xor_sync(mask, v.h, 1), __shfl_xor_sync(mask, v.l, 1));
}
__device__ __forceinline__ bool pair_any(bool v, unsigned mask) {
    return (__shfl_xor_sync(mask, int(v), 1) | int(v)) != 0;
}
// Both lanes get the same sum (addition of the two partials commutes).
template <class T> __device__ __forceinline__ T pair_sum(T v, unsigned mask) { return v + pair_other(v, mask); }

// Groups of n lanes per element (lanes base .. base + n - 1 of a warp; `mask`
// holds every lane that takes part): the value of lane `src` to every lane.
__device__ __forceinline__ float grp_get(float v, unsigned mask, int src) { return __shfl_sync(mask, v, src); }
__device__ __forceinline__ double grp_get(double v, unsigned mask, int src) { return __shfl_sync(mask, v, src); }
__device__ __forceinline__ DW grp_get(DW v, unsigned mask, int src) {
    return DW(__shfl_sync(mask, v.h, src), __shfl_sync(mask, v.l, src));
}
template <class T> __device__ __forceinline__ V3<T> grp_get(V3<T> v, unsigned mask, int src) {
    return {grp_get(v.x, mask, src), grp_get(v.y, mask, src), grp_get(v.z, mask, src)};
}
// OR of a flag, and sum of a float, over the group (every lane gets the result).
__device__ __forceinline__ bool grp_any(bool v, unsigned mask, int base, int n) {
    return ((__ballot_sync(mask, v) >> base) & ((1u << n) - 1u)) != 0u;
}
__device__ __forceinline__ float grp_sum(float v, unsigned mask, int base, int n) {
    float s = 0.0f;
    for (int k = 0; k < n; ++k) s = __fadd_rn(s, __shfl_sync(mask, v, base + k));
    return s;
}

}  // namespace fe
