// Integration kernels: one element per thread (the element-loop parallelisation
// of Sec. 3.2), QSS loop order (Algorithms 2 and 3), inputs in "coalesced"
// plane order or in the "natural" element-contiguous order staged through shared
// memory by bulk copies (Sec. 4.2, Fig. 1), outputs in either order (Fig. 2).
#pragma once
#include <type_traits>

#include "fe_device.cuh"

namespace fe {

template <int ET, int KIND, int PREC, int QUAD, int CPQ> struct ElemCfg {
    static constexpr int NS = ET == TET ? 4 : 6;
    static constexpr int NX = 3 * NS;
    static constexpr int NA = NS * NS;
    static constexpr int NQ = Rule<QUAD>::NQ;
    // coefficients per element; CPQ == 2: the nodal values of the field u of the
    // coefficient function
    static constexpr int NC = CPQ == 2 ? NS : (KIND == POISSON ? 1 : 20) * (CPQ ? NQ : 1);
    using CT = typename std::conditional<float_form(PREC), float, double>::type;
};

__device__ __forceinline__ V3<float> to_f(V3<double> v) {
    return {static_cast<float>(v.x), static_cast<float>(v.y), static_cast<float>(v.z)};
}

// Float view of a value for the shape test (the high word of a double-word).
__device__ __forceinline__ float hi_f(float v) { return v; }
__device__ __forceinline__ float hi_f(double v) { return static_cast<float>(v); }
__device__ __forceinline__ float hi_f(DW v) { return v.h; }
template <class T> __device__ __forceinline__ V3<float> hi_f(V3<T> v) { return {hi_f(v.x), hi_f(v.y), hi_f(v.z)}; }

// Coefficients of the double-word form: double in memory, split on read.
template <class CS> struct DwCoef {
    const CS &c;
    __device__ __forceinline__ DW operator()(int j) const { return dw_coef(c(j)); }
};

// Edge vector x_k - x_0 of the double-word form: difference in double (one DADD
// per component, exact to 2^-53), then split.
template <class XS> __device__ __forceinline__ V3<DW> dw_edge_vec(const XS &x, int k) {
    return {dw_edge(x(3 * k) - x(0)), dw_edge(x(3 * k + 1) - x(1)), dw_edge(x(3 * k + 2) - x(2))};
}

// ---------------------------------------------------------------------------
// One element: inputs through accessors, outputs into registers.
// Returns the flag byte; `poor` is set when the mixed-precision shape test fails.
// ---------------------------------------------------------------------------
template <int ET, int KIND, int PREC, int QUAD, int CPQ> struct ElemMath;

// Tetrahedron, FP64 (Algorithm 3 in double). The Laplace kind and the generic
// kind with per-element coefficients run the scalings of the coefficients and of
// det J and the products of the cofactors (TetF64's OM and OX groups) in integer
// instructions that report special cases (the same IEEE results): they relieve
// the double pipe (6M generic tetrahedra 3.94 -> 4.04 Gelem/s with the cofactor
// products, Laplace 9.26 -> 9.65). Integer edges or row sums lengthen the chain
// of dependent additions and measured slower even in the reporting form (generic:
// sums 0.83x, edges and sums 0.76x; Laplace 0.84x, 0.71x). Per-point
// coefficients take the general products.
template <int KIND, int QUAD, int CPQ> struct ElemMath<TET, KIND, FP64, QUAD, CPQ> {
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, double A[16], double b[4], bool &poor) {
        poor = false;
        if constexpr (KIND == GENERIC && CPQ) {
            const V3<double> x0 = {x(0), x(1), x(2)};
            const V3<double> e1 = V3<double>{x(3), x(4), x(5)} - x0;
            const V3<double> e2 = V3<double>{x(6), x(7), x(8)} - x0;
            const V3<double> e3 = V3<double>{x(9), x(10), x(11)} - x0;
            const TetGeo<double> geo = tet_geometry(e1, e2, e3);
            if (degenerate_det(geo.det)) return zero(A, b);
            const double V = fabs(geo.det);
            const double inv = recip_fast(geo.det);
            V3<double> g[4];
            g[1] = inv * geo.a[0];
            g[2] = inv * geo.a[1];
            g[3] = inv * geo.a[2];
            g[0] = -1.0 * (g[1] + g[2] + g[3]);
            tet_generic_products<double, QUAD, CPQ>(g, V, c, A, b);
            return is_neg(geo.det) ? 2 : 0;
        } else {
            // scalings in integer instructions; an element that meets a special
            // operand or product there is redone on the double pipe (one branch
            // per element, never taken on ordinary data)
            using TF = TetF64<F64<false>, F64<true>, F64<true>, F64<false>>;
            using TH = TetF64<F64<false>, F64<false>, F64<false>, F64<false>>;
            double a[3][3], det;
            bool sp = false;
            if (!TF::geometry(x, a, det, sp)) return zero(A, b);
            if constexpr (KIND == POISSON)
                TF::template poisson<QUAD, CPQ>(a, det, c, A, b, sp);
            else
                TF::template generic<QUAD>(a, det, c, A, b, sp);
            if (sp) {
                // from the inputs again (the compiler barrier keeps the first pass's
                // values from being held for this path)
                asm volatile("" ::: "memory");
                double a2[3][3], det2;
                TH::geometry(x, a2, det2, sp);
                if constexpr (KIND == POISSON)
                    TH::template poisson<QUAD, CPQ>(a2, det2, c, A, b, sp);
                else
                    TH::template generic<QUAD>(a2, det2, c, A, b, sp);
            }
            return is_neg(det) ? 2 : 0;
        }
    }
    __device__ __forceinline__ static uint8_t zero(double A[16], double b[4]) {
#pragma unroll
        for (int k = 0; k < 16; ++k) A[k] = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) b[k] = 0.0;
        return 4;
    }
};

// Tetrahedron, mixed: float arithmetic from hi/lo edge vectors; shape test.
template <int KIND, int QUAD, int CPQ> struct ElemMath<TET, KIND, MIXED, QUAD, CPQ> {
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, float A[16], float b[4], bool &poor) {
        HiLo h[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) h[j] = split_double(x(j));
        V3<float> e[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            e[k] = {diff_hilo(h[3 * (k + 1)], h[0]), diff_hilo(h[3 * (k + 1) + 1], h[1]), diff_hilo(h[3 * (k + 1) + 2], h[2])};
        const TetGeo<float> geo = tet_geometry(e[0], e[1], e[2]);
        poor = tet_poor(e[0], e[1], e[2], geo.det);
        const float V = fabsf(geo.det);
        const float inv = 1.0f / geo.det;
        if (KIND == POISSON) {
            tet_poisson_products<float, QUAD, CPQ>(geo, fabsf(inv), V, c, A, b);
        } else {
            V3<float> g[4];
            g[1] = inv * geo.a[0];
            g[2] = inv * geo.a[1];
            g[3] = inv * geo.a[2];
            g[0] = -1.0f * (g[1] + g[2] + g[3]);
            tet_generic_products<float, QUAD, CPQ>(g, V, c, A, b);
        }
        return geo.det < 0.0f ? 2 : 0;
    }
    // Double-precision Jacobian for a flagged element: det, inverse and gradients
    // in double, narrowed to float, the rest in float.
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t fixup(const XS &x, const CS &c, float A[16], float b[4]) {
        const V3<double> x0 = {x(0), x(1), x(2)};
        const V3<double> e1 = V3<double>{x(3), x(4), x(5)} - x0;
        const V3<double> e2 = V3<double>{x(6), x(7), x(8)} - x0;
        const V3<double> e3 = V3<double>{x(9), x(10), x(11)} - x0;
        const TetGeo<double> geo = tet_geometry(e1, e2, e3);
        if (!(fabs(geo.det) > 1e-300)) {
#pragma unroll
            for (int k = 0; k < 16; ++k) A[k] = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) b[k] = 0.0f;
            return 1 | 4;
        }
        const double inv = 1.0 / geo.det;
        V3<double> gd[4];
        gd[1] = inv * geo.a[0];
        gd[2] = inv * geo.a[1];
        gd[3] = inv * geo.a[2];
        gd[0] = -1.0 * (gd[1] + gd[2] + gd[3]);
        V3<float> g[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) g[k] = to_f(gd[k]);
        const float V = static_cast<float>(fabs(geo.det));
        if (KIND == POISSON)
            tet_poisson_from_grads<float, QUAD, CPQ>(g, V, c, A, b);
        else
            tet_generic_products<float, QUAD, CPQ>(g, V, c, A, b);
        return 1 | (geo.det < 0.0 ? 2 : 0);
    }
};

// Tetrahedron, double-word: Algorithm 3 in double-word arithmetic from double
// edge vectors. An element that fails the shape test, whose |det J| or results
// leave the double-word window, or whose inputs do, is flagged and redone in
// double by the fix-up kernel.
template <int KIND, int QUAD, int CPQ> struct ElemMath<TET, KIND, DWORD, QUAD, CPQ> {
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, double A[16], double b[4], bool &poor) {
        const V3<DW> e1 = dw_edge_vec(x, 1), e2 = dw_edge_vec(x, 2), e3 = dw_edge_vec(x, 3);
        const TetGeo<DW> geo = tet_geometry(e1, e2, e3);
        poor = tet_poor(hi_f(e1), hi_f(e2), hi_f(e3), geo.det.h) || !dw_det_ok(geo.det.h);
        const DwCoef<CS> cd{c};
        const DW V = dw_abs(geo.det);
        const DW inv = dw_recip(geo.det);
        if constexpr (KIND == POISSON) {
            poisson(geo, dw_abs(inv), V, cd, A, b, poor);
        } else {
            DW Ad[16], bd[4];
            if constexpr (!CPQ) {
                constexpr TetSums S = tet_sums<QUAD>();
                const bool neg = geo.det.h < 0.0f;
                const DW f = DW(S.W) * dw_recip(V);
                tet_generic_aug<DW, QUAD>(geo.a, f, neg ? DW(-S.W / 4) : DW(S.W / 4), neg ? DW(-S.W) : DW(S.W), V, cd,
                                          Ad, bd);
            } else {
                V3<DW> g[4];
                g[1] = inv * geo.a[0];
                g[2] = inv * geo.a[1];
                g[3] = inv * geo.a[2];
                g[0] = -(g[1] + g[2] + g[3]);
                tet_generic_products<DW, QUAD, CPQ>(g, V, cd, Ad, bd);
            }
            poor = poor || !dw_group_ok<16>(Ad) || !dw_group_ok<4>(bd);
#pragma unroll
            for (int k = 0; k < 16; ++k) A[k] = dw_to_double(Ad[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) b[k] = dw_to_double(bd[k]);
        }
        return geo.det.h < 0.0f ? 2 : 0;
    }
    // Laplace products (as tet_poisson_products): the ten distinct entries of the
    // symmetric A^e are computed and converted once each; b^e is uniform for
    // per-element coefficients or a one-point rule (m_r = |T|/4 for both rules).
    // The six entries of G convert with integer operations, the rest with one DADD
    // each, which balances the double and integer pipes of this kernel (measured:
    // 6 + 5 beats 11 + 0 and 0 + 11).
    template <class CS>
    __device__ __forceinline__ static void poisson(const TetGeo<DW> &geo, DW invabs, DW V, const CS &c, double A[16],
                                                   double b[4], bool &poor) {
        constexpr TetSums S = tet_sums<QUAD>();
        const DW k = DW(S.W) * invabs;
        DW G[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = r; s < 3; ++s) G[r][s] = G[s][r] = k * dot(geo.a[r], geo.a[s]);
        DW row0[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) row0[s] = -(G[0][s] + G[1][s] + G[2][s]);
        const DW a00 = -(row0[0] + row0[1] + row0[2]);
        DW bd[4];
        tet_poisson_b<DW, QUAD, CPQ>(V, c, bd);
        constexpr bool uniform_b = !CPQ || Rule<QUAD>::NQ == 1;
        // window check over all 16 (4) entries, repeated ones counted twice (four times)
        float sa = fabsf(a00.h) + fabsf(G[0][0].h) + fabsf(G[1][1].h) + fabsf(G[2][2].h);
        float so = fabsf(G[0][1].h) + fabsf(G[0][2].h) + fabsf(G[1][2].h) + fabsf(row0[0].h) + fabsf(row0[1].h) +
                   fabsf(row0[2].h);
        sa = __fmaf_rn(2.0f, so, sa);
        float sb = uniform_b ? 4.0f * fabsf(bd[0].h)
                             : fabsf(bd[0].h) + fabsf(bd[1].h) + fabsf(bd[2].h) + fabsf(bd[3].h);
        poor = poor || !(sa == 0.0f || (sa >= 0x1p-80f && sa <= 0x1p100f)) ||
               !(sb == 0.0f || (sb >= 0x1p-80f && sb <= 0x1p100f));
        A[0] = dw_to_double(a00);
#pragma unroll
        for (int s = 0; s < 3; ++s) A[1 + s] = A[4 * (1 + s)] = dw_to_double(row0[s]);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int s = r; s < 3; ++s) A[4 * (r + 1) + (s + 1)] = A[4 * (s + 1) + (r + 1)] = dw_to_double_int(G[r][s]);
        if (uniform_b) {
            const double v = dw_to_double(bd[0]);
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] = v;
        } else {
#pragma unroll
            for (int r = 0; r < 4; ++r) b[r] = dw_to_double(bd[r]);
        }
    }
    // Flagged element: the whole element in double.
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t fixup(const XS &x, const CS &c, double A[16], double b[4]) {
        bool unused;
        return 1 | ElemMath<TET, KIND, FP64, QUAD, CPQ>::run(x, c, A, b, unused);
    }
};

// Prism (Algorithm 2): T = double, float or double-word arithmetic after the
// edge vectors.
// The half of a prism's A^e and b^e that lane `part` of a pair writes: entry
// pair_entry(j, part) of A^e (row-major) in Ah[j], entry pair_b_entry(j, part) of
// b^e in bh[j]. Laplace: entries 2j + part, picked from the whole A^e and b^e that
// both lanes hold. Generic: lane 0 the diagonal blocks (bottom-bottom, top-top) of
// A^e and b_0..2, lane 1 the off-diagonal blocks and b_3..5, as pair_blocks leaves
// them in A[0..17] and b[0..2].
template <int KIND> __device__ __forceinline__ int pair_entry(int j, int part) {
    if constexpr (KIND == GENERIC) {
        const int blk = j / 9, k = (j % 9) / 3, kk = j % 3;
        return 6 * (k + 3 * blk) + kk + 3 * (blk ^ part);
    } else {
        return 2 * j + part;
    }
}
template <int KIND> __device__ __forceinline__ int pair_b_entry(int j, int part) {
    return KIND == GENERIC ? 3 * part + j : 2 * j + part;
}
template <int KIND, class T>
__device__ __forceinline__ void pick_half(const T A[36], const T b[6], T Ah[18], T bh[3], int part) {
    if constexpr (KIND == GENERIC) {
#pragma unroll
        for (int j = 0; j < 18; ++j) Ah[j] = A[j];
#pragma unroll
        for (int j = 0; j < 3; ++j) bh[j] = b[j];
    } else {
#pragma unroll
        for (int j = 0; j < 18; ++j) Ah[j] = part ? A[2 * j + 1] : A[2 * j];
#pragma unroll
        for (int j = 0; j < 3; ++j) bh[j] = part ? b[2 * j + 1] : b[2 * j];
    }
}

template <int KIND, int PREC, int CPQ> struct PrismMath {
    using T = typename std::conditional<PREC == FP64, double,
                                        typename std::conditional<PREC == MIXED, float, DW>::type>::type;

    // Q loop on relative coordinates r[0..5] (r[0] = 0). Returns bit1/bit2 flags.
    // Generic coefficients: the three points of a zeta level run in a rolled loop
    // (which keeps the body in the instruction cache) and gather per-level sums of
    // the reference-space coefficient matrix (level_sums); A^e is expanded from
    // them once per level (level_expand). Laplace: the points only gather Gram
    // terms of J^{-1} (prism_laplace_assemble forms A^e from them once).
    //
    // TPE == 2 (two threads per element): the lane of parity `part` takes the three
    // points of zeta level `part` and the pair combines its partial results
    // through shuffles within `mask`. Laplace: both lanes end with the whole A^e
    // and b^e. Generic: each lane ends with its half (pair_blocks).
    //
    // FP64: the products off the critical path run in integer instructions, and
    // sp is set when one of them meets an operand or a product outside the normal
    // range (zero aside; with TPE == 2 for both lanes of the pair); the caller then
    // redoes the element with HW = true (those products on the double pipe).
    template <int TPE = 1, bool HW = false, class CS>
    __device__ __forceinline__ static uint8_t qloop(const V3<T> r[6], const CS &c, T A[36], T b[6], bool &poor,
                                                    bool &sp, int part = 0, unsigned mask = 0xFFFFFFFFu) {
        const PrismFrame<T> f = prism_frame(r);
#pragma unroll
        for (int k = 0; k < 6; ++k) b[k] = T(0);
        bool neg = false, degenerate = false;
        poor = false;
        if constexpr (KIND == POISSON) {
            T L[2][3], v[2][3][2], c3[3];
            if constexpr (TPE == 1) {
                T c3l[2][3];
#pragma unroll
                for (int l = 0; l < 2; ++l)
                    level_laplace<HW>(f, l, c, L[l], v[l], c3l[l], b, poor, neg, degenerate, sp);
#pragma unroll
                for (int t = 0; t < 3; ++t) c3[t] = c3l[0][t] + c3l[1][t];
            } else {
                T Lm[3], vm[3][2], c3m[3];
                level_laplace<HW>(f, part, c, Lm, vm, c3m, b, poor, neg, degenerate, sp);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const T o = pair_other(Lm[j], mask);
                    L[0][j] = part ? o : Lm[j];
                    L[1][j] = part ? Lm[j] : o;
                    c3[j] = pair_sum(c3m[j], mask);
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const T w = pair_other(vm[j][i], mask);
                        v[0][j][i] = part ? w : vm[j][i];
                        v[1][j][i] = part ? vm[j][i] : w;
                    }
                }
            }
            prism_laplace_assemble<T>(L, v, c3, A);
            mirror(A);
        } else {
#pragma unroll
            for (int k = 0; k < 36; ++k) A[k] = T(0);
            const T r12 = T(1.0 / 12.0);
            const V3<T> wm = r12 * ((f.w0 + f.w1) + f.w2);
            if constexpr (TPE == 1) {
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    LevelSums S;
                    level_sums<HW>(f, wm, l, c, S, poor, neg, degenerate, sp);
                    level_expand(S, l, A, b);
                }
                prism_dw_normalise<T>(A, b);
            } else {
                LevelSums S;
                level_sums<HW>(f, wm, part, c, S, poor, neg, degenerate, sp);
                pair_blocks(S, part, mask, A, b);
            }
        }
        if constexpr (TPE == 2) {
            if constexpr (KIND == POISSON) {
#pragma unroll
                for (int k = 0; k < 6; ++k) b[k] = pair_sum(b[k], mask);
            }
            poor = pair_any(poor, mask);
            if constexpr (PREC == FP64 && !HW) sp = pair_any(sp, mask);
            neg = pair_any(neg, mask);
            degenerate = pair_any(degenerate, mask);
        }
        if (degenerate) {
#pragma unroll
            for (int k = 0; k < 36; ++k) A[k] = T(0);
#pragma unroll
            for (int k = 0; k < 6; ++k) b[k] = T(0);
            return 4;
        }
        return neg ? 2 : 0;
    }

    // Laplace: the three points of zeta level l (a constant after unrolling, or a
    // run-time lane parity): per-level sum of (gamma_11, gamma_12, gamma_22), the
    // points' (gamma_13, gamma_23) and gamma_33, and the load vector terms.
    // HW: the FP64 products on the double pipe (the redo after a special case).
    template <bool HW = false, class CS>
    __device__ __forceinline__ static void level_laplace(const PrismFrame<T> &f, int l, const CS &c, T Ll[3],
                                                         T vl[3][2], T c3l[3], T b[6], bool &poor, bool &neg,
                                                         bool &degenerate, bool &sp) {
        using R = Rule<Q_PRISM6>;
        const T zb = l ? T(R::zb(1)) : T(R::zb(0)), zt = l ? T(R::zt(1)) : T(R::zt(0));
        const V3<T> cx = zb * f.ub + zt * f.ut;
        const V3<T> cy = zb * f.vb + zt * f.vt;
        const V3<T> a3 = cross(cx, cy);
        const T a33 = dot(a3, a3);
        float fxy = 0.0f;
        if constexpr (PREC != FP64) {
            const V3<float> cxf = hi_f(cx), t1 = 2.0f * hi_f(cy) - cxf;
            fxy = dot(cxf, cxf) + dot(t1, t1) * (1.0f / 3.0f);
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int q = 3 * l + t;
            // lambda_k / 2 at triangle point t
            const T h0 = T(t == 0 ? 1.0 / 3.0 : 1.0 / 12.0), h1 = T(t == 1 ? 1.0 / 3.0 : 1.0 / 12.0),
                    h2 = T(t == 2 ? 1.0 / 3.0 : 1.0 / 12.0);
            const V3<T> cz = h0 * f.w0 + h1 * f.w1 + h2 * f.w2;
            const V3<T> a1 = cross(cy, cz), a2 = cross(cz, cx);
            const T det = dot(cx, a1);
            if constexpr (PREC != FP64) poor |= prism_poor(fxy, hi_f(cz), hi_f(det));
            if constexpr (PREC == DWORD) poor |= !dw_det_ok(det.h);
            if constexpr (PREC == FP64) degenerate |= degenerate_det(det);
            neg |= is_neg(det);
            const T adet = abs_t(det);
            const T sw = recip_w(adet, T(R::w(0)));          // vol / det^2 (equal weights)
            const T g11 = mul_off<HW>(sw, dot(a1, a1), sp), g12 = mul_off<HW>(sw, dot(a1, a2), sp),
                    g22 = mul_off<HW>(sw, dot(a2, a2), sp);
            if (t == 0) {
                Ll[0] = g11;
                Ll[1] = g12;
                Ll[2] = g22;
            } else {
                Ll[0] += g11;
                Ll[1] += g12;
                Ll[2] += g22;
            }
            vl[t][0] = mul_off<HW>(sw, dot(a1, a3), sp);
            vl[t][1] = mul_off<HW>(sw, dot(a2, a3), sp);
            c3l[t] = mul_off<HW>(sw, a33, sp);
            const T vd = mul_off<HW>(mul_off<HW>(adet, T(R::w(0)), sp), c(CPQ ? q : 0), sp);
#pragma unroll
            for (int k = 0; k < 6; ++k) b[k] += vd * (l ? T(R::phi(3 + t, k)) : T(R::phi(t, k)));
        }
    }

    // Generic coefficients at zeta level l, contracted in reference space (the
    // same PRISM6 sum as Algorithm 2's per-point update, regrouped). With the
    // cofactor rows a_i of J (J^{-1} has rows a_i / det) and vol = w |det J|, each
    // point forms the reference-space coefficient matrix
    //   Gamma = vol B^T C B,  B = diag(1, J^{-T}):
    //   Gamma_00 = vol c00, Gamma_0j = w sgn(det) c0. a_j, Gamma_i0 = w sgn(det) a_i . c.0,
    //   Gamma_ij = (w / |det|) a_i^T C3 a_j  (i, j = 1..3).
    // The reference derivatives (phi, d/dxi, d/deta, d/dzeta) of shape function
    // (k, m) (k the triangle vertex, m = 0 bottom, 1 top) are
    //   psi_(k,m) = z_m u_k + s_m h_k e_3,  u_k = (2 h_k, D_k1, D_k2, 0),
    // with z_m the level's (1 -+ zeta)/2, s_m = -1 / +1, h_k = lambda_k(t) / 2 and
    // D = d lambda / d(xi, eta) = ((-1, -1), (1, 0), (0, 1)). A point adds
    // psi_r^T Gamma psi_s to A_rs; only h_k and Gamma change between the three
    // points of a level, so the points accumulate the sums
    //   SF_kk' = sum_t u_k^T Gamma[0..2][0..2] u_k',  SP_kk' = sum_t h_k' u_k . Gamma[0..2][3],
    //   SQ_kk' = sum_t h_k Gamma[3][0..2] . u_k',      SG_kk' = sum_t h_k h_k' Gamma_33,
    // and the 6 x 6 expansion runs once per level:
    //   A_(k,m),(k',m') += z_m z_m' SF + z_m s_m' SP + s_m z_m' SQ + s_m s_m' SG.
    // Likewise b_(k,m) += z_m BU_k + s_m BR_k with BU_k = sum_t (2 h_k vol d0 +
    // sum_i D_ki w sgn(det) d. a_i) and BR_k = sum_t h_k w sgn(det) d. a_3.
    // wm = (w_0 + w_1 + w_2) / 12, so that d x / d zeta at point t is wm + w_t / 4.
    // HW as for level_laplace.
    struct LevelSums {
        T SF[9], SP[9], SQ[9], SG[6], BU[3], BR[3];
    };
    template <bool HW = false, class CS>
    __device__ __forceinline__ static void level_sums(const PrismFrame<T> &f, const V3<T> &wm, int l, const CS &c,
                                                      LevelSums &Sl, bool &poor, bool &neg, bool &degenerate,
                                                      bool &sp) {
        using R = Rule<Q_PRISM6>;
        const T zb = l ? T(R::zb(1)) : T(R::zb(0)), zt = l ? T(R::zt(1)) : T(R::zt(0));
        const V3<T> cx = zb * f.ub + zt * f.ut;
        const V3<T> cy = zb * f.vb + zt * f.vt;
        const V3<T> a3 = cross(cx, cy);
        float fxy = 0.0f;
        if constexpr (PREC != FP64) {
            const V3<float> cxf = hi_f(cx), t1 = 2.0f * hi_f(cy) - cxf;
            fxy = dot(cxf, cxf) + dot(t1, t1) * (1.0f / 3.0f);
        }
        T SF[9], SP[9], SQ[9], SG[6], S4[4], BU[3], BR[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) SF[k] = SP[k] = SQ[k] = T(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) SG[k] = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) S4[k] = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k) BU[k] = BR[k] = T(0);
#pragma unroll 1
        for (int t = 0; t < 3; ++t) {
            const int o = CPQ ? 20 * (3 * l + t) : 0;
            const V3<T> wt = t == 0 ? f.w0 : (t == 1 ? f.w1 : f.w2);
            const V3<T> cz = {madd(T(0.25), wt.x, wm.x), madd(T(0.25), wt.y, wm.y), madd(T(0.25), wt.z, wm.z)};
            const V3<T> a1 = cross(cy, cz), a2 = cross(cz, cx);
            const T det = dot(cx, a1);
            if constexpr (PREC != FP64) poor |= prism_poor(fxy, hi_f(cz), hi_f(det));
            if constexpr (PREC == DWORD) poor |= !dw_det_ok(det.h);
            if constexpr (PREC == FP64) degenerate |= degenerate_det(det);
            const bool ng = is_neg(det);
            neg |= ng;
            const T adet = abs_t(det);
            const T s2 = recip_w(adet, T(R::w(0)));              // w / |det|
            const T s1 = ng ? T(-R::w(0)) : T(R::w(0));          // w sgn(det)
            const T s0 = mul_off<HW>(adet, T(R::w(0)), sp);      // vol
            const V3<T> av[3] = {a1, a2, a3};
            const V3<T> c0 = {mul_off<HW>(s1, c(o + 1), sp), mul_off<HW>(s1, c(o + 2), sp),
                              mul_off<HW>(s1, c(o + 3), sp)};
            const V3<T> ci0 = {mul_off<HW>(s1, c(o + 4), sp), mul_off<HW>(s1, c(o + 8), sp),
                               mul_off<HW>(s1, c(o + 12), sp)};
            V3<T> C3[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                C3[i] = {mul_off<HW>(s2, c(o + 4 * i + 5), sp), mul_off<HW>(s2, c(o + 4 * i + 6), sp),
                         mul_off<HW>(s2, c(o + 4 * i + 7), sp)};
            T G[4][4];
            G[0][0] = mul_off<HW>(s0, c(o), sp);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const V3<T> Ca = {dot(C3[0], av[j]), dot(C3[1], av[j]), dot(C3[2], av[j])};
                G[0][j + 1] = dot(c0, av[j]);
                G[j + 1][0] = dot(av[j], ci0);
#pragma unroll
                for (int i = 0; i < 3; ++i) G[i + 1][j + 1] = dot(av[i], Ca);
            }
            // h_k = lambda_k(t) / 2 and 2 h_k
            T h[3], h2[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                h[k] = t == k ? T(1.0 / 3.0) : T(1.0 / 12.0);
                h2[k] = t == k ? T(2.0 / 3.0) : T(1.0 / 6.0);
            }
            // SF: 4 h_k h_k' G00 + 2 h_k x_k' + 2 h_k' y_k (the D-block of G summed apart in S4)
            const T xs[3] = {-(G[0][1] + G[0][2]), G[0][1], G[0][2]};
            const T ys[3] = {-(G[1][0] + G[2][0]), G[1][0], G[2][0]};
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const T e = madd(h2[kk], G[0][0], xs[kk]);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    acc(SF[3 * k + kk], h2[k], e);
                    acc(SF[3 * k + kk], h2[kk], ys[k]);
                }
            }
            acc1(S4[0], G[1][1]);
            acc1(S4[1], G[1][2]);
            acc1(S4[2], G[2][1]);
            acc1(S4[3], G[2][2]);
            const T p[3] = {madd(h2[0], G[0][3], -(G[1][3] + G[2][3])), madd(h2[1], G[0][3], G[1][3]),
                            madd(h2[2], G[0][3], G[2][3])};
            const T qv[3] = {madd(h2[0], G[3][0], -(G[3][1] + G[3][2])), madd(h2[1], G[3][0], G[3][1]),
                             madd(h2[2], G[3][0], G[3][2])};
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int kk = 0; kk < 3; ++kk) {
                    acc(SP[3 * k + kk], h[kk], p[k]);
                    acc(SQ[3 * k + kk], h[k], qv[kk]);
                }
#pragma unroll
            for (int k = 0; k < 3; ++k) acc(SG[k], t == k ? T(1.0 / 9.0) : T(1.0 / 144.0), G[3][3]);
            acc(SG[3], t == 2 ? T(1.0 / 144.0) : T(1.0 / 36.0), G[3][3]);   // (0, 1)
            acc(SG[4], t == 1 ? T(1.0 / 144.0) : T(1.0 / 36.0), G[3][3]);   // (0, 2)
            acc(SG[5], t == 0 ? T(1.0 / 144.0) : T(1.0 / 36.0), G[3][3]);   // (1, 2)
            // load vector
            const T d0 = mul_off<HW>(s0, c(o + 16), sp);
            const V3<T> dv = {mul_off<HW>(s1, c(o + 17), sp), mul_off<HW>(s1, c(o + 18), sp),
                              mul_off<HW>(s1, c(o + 19), sp)};
            const T dl1 = dot(dv, a1), dl2 = dot(dv, a2), dl3 = dot(dv, a3);
            const T dd[3] = {-(dl1 + dl2), dl1, dl2};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                acc(BU[k], h2[k], d0);
                acc1(BU[k], dd[k]);
                acc(BR[k], h[k], dl3);
            }
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            SF[k] = acc_norm(SF[k]);
            SP[k] = acc_norm(SP[k]);
            SQ[k] = acc_norm(SQ[k]);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) SG[k] = acc_norm(SG[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) S4[k] = acc_norm(S4[k]);
        // SF += D S4 D^T
        SF[4] = SF[4] + S4[0];
        SF[5] = SF[5] + S4[1];
        SF[7] = SF[7] + S4[2];
        SF[8] = SF[8] + S4[3];
        SF[3] = SF[3] - (S4[0] + S4[1]);
        SF[6] = SF[6] - (S4[2] + S4[3]);
        SF[1] = SF[1] - (S4[0] + S4[2]);
        SF[2] = SF[2] - (S4[1] + S4[3]);
        SF[0] = SF[0] + ((S4[0] + S4[1]) + (S4[2] + S4[3]));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            Sl.SF[k] = SF[k];
            Sl.SP[k] = SP[k];
            Sl.SQ[k] = SQ[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) Sl.SG[k] = SG[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Sl.BU[k] = acc_norm(BU[k]);
            Sl.BR[k] = acc_norm(BR[k]);
        }
    }

    // One thread per element: the level's share of A and b, accumulated into them
    // (unnormalised double-word pairs until prism_dw_normalise).
    __device__ __forceinline__ static void level_expand(const LevelSums &S, int l, T A[36], T b[6]) {
        using R = Rule<Q_PRISM6>;
        const T zb = l ? T(R::zb(1)) : T(R::zb(0)), zt = l ? T(R::zt(1)) : T(R::zt(0));
        const T *SF = S.SF, *SP = S.SP, *SQ = S.SQ, *SG = S.SG;
        // the level's share of A and b
        const T zbb = l ? T(R::zb(1) * R::zb(1)) : T(R::zb(0) * R::zb(0));
        const T ztt = l ? T(R::zt(1) * R::zt(1)) : T(R::zt(0) * R::zt(0));
        const T zbt = l ? T(R::zb(1) * R::zt(1)) : T(R::zb(0) * R::zt(0));
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const T sf = SF[3 * k + kk], sp = SP[3 * k + kk], sq = SQ[3 * k + kk];
                const T sg = SG[k == kk ? k : k + kk + 2];
                T &a00 = A[6 * k + kk], &a01 = A[6 * k + kk + 3], &a10 = A[6 * (k + 3) + kk],
                  &a11 = A[6 * (k + 3) + kk + 3];
                acc(a00, zbb, sf);
                acc(a00, -zb, sp);
                acc(a00, -zb, sq);
                acc1(a00, sg);
                acc(a01, zbt, sf);
                acc(a01, zb, sp);
                acc(a01, -zt, sq);
                acc1(a01, -sg);
                acc(a10, zbt, sf);
                acc(a10, -zt, sp);
                acc(a10, zb, sq);
                acc1(a10, -sg);
                acc(a11, ztt, sf);
                acc(a11, zt, sp);
                acc(a11, zt, sq);
                acc1(a11, sg);
            }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T bu = S.BU[k], br = S.BR[k];
            acc(b[k], zb, bu);
            acc1(b[k], -br);
            acc(b[k + 3], zt, bu);
            acc1(b[k + 3], br);
        }
    }

    // Two threads per element, lane `part` holding the sums of zeta level `part`.
    // With zb = 1/2 + s c and zt = 1/2 - s c on the level (c = 1/(2 sqrt 3), s = +1
    // on level 0 and -1 on level 1), zb^2 = 1/3 + s c, zt^2 = 1/3 - s c and
    // zb zt = 1/6, so the level's share of the four 3 x 3 blocks of A^e is
    //   A_00 = X + Y, A_11 = X - Y, A_01 = U + V, A_10 = U - V,
    //   X = SF/3 + SG - s c (SP + SQ),  U = SF/2 - X,  Y = s c SF - (SP + SQ)/2,
    //   V = (SP - SQ)/2,
    // and of b^e: b_k = Bx + By, b_(k+3) = Bx - By with Bx = BU/2, By = s c BU - BR.
    // Lane 0 keeps X and Y (blocks 00 and 11) and b_0..2, lane 1 U and V (blocks 01
    // and 10) and b_3..5; each sends the other the two sums that the other keeps,
    // so that no lane forms all 36 entries. On return A[j] (j < 18) holds the
    // lane's entries in the order of pair_entry and b[0..2] its entries of b^e.
    __device__ __forceinline__ static void pair_blocks(const LevelSums &S, int part, unsigned mask, T A[36],
                                                       T b[6]) {
        const T c = T(0.5 * kInvSqrt3);
        const T sc = part ? -c : c, nsc = part ? c : -c;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const int i = 3 * k + kk;
                const T sg = S.SG[k == kk ? k : k + kk + 2];
                const T spq = S.SP[i] + S.SQ[i], smq = S.SP[i] - S.SQ[i];
                const T X = madd(nsc, spq, madd(T(1.0 / 3.0), S.SF[i], sg));
                const T U = half(S.SF[i]) - X;
                const T Y = madd(sc, S.SF[i], -half(spq));
                const T V = half(smq);
                const T P = (part ? U : X) + pair_other(part ? X : U, mask);
                const T Q = (part ? V : Y) + pair_other(part ? Y : V, mask);
                A[i] = P + Q;
                A[9 + i] = P - Q;
            }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T bx = half(S.BU[k]), by = madd(sc, S.BU[k], -S.BR[k]);
            const T Bx = bx + pair_other(bx, mask), By = by + pair_other(by, mask);
            b[k] = part ? Bx - By : Bx + By;
        }
    }

    // a b + c; s += a b and s += a (in double-word s stays an unnormalised pair
    // until acc_norm); plain fused multiply-adds in the other forms
    __device__ __forceinline__ static T madd(T a, T b, T c) {
        if constexpr (PREC == DWORD)
            return dw_dot_add<1>(&a, &b, c);
        else
            return a * b + c;
    }
    // x / 2 (exact)
    __device__ __forceinline__ static T half(T x) {
        if constexpr (PREC == DWORD)
            return DW(0.5f * x.h, 0.5f * x.l);
        else
            return T(0.5) * x;
    }
    __device__ __forceinline__ static void acc(T &s, T a, T b) {
        if constexpr (PREC == DWORD)
            dw_acc(s, a, b);
        else
            s = a * b + s;
    }
    __device__ __forceinline__ static void acc1(T &s, T a) {
        if constexpr (PREC == DWORD)
            dw_acc_add(s, a);
        else
            s = s + a;
    }
    __device__ __forceinline__ static T acc_norm(T s) {
        if constexpr (PREC == DWORD)
            return dw_acc_norm(s);
        else
            return s;
    }
    __device__ __forceinline__ static T abs_t(T v) {
        if constexpr (PREC == FP64)   // the sign bit cleared (an integer operation)
            return __longlong_as_double(__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFll);
        else
            return v < T(0) ? -v : v;
    }
    // a b for the products off the critical path: in FP64 in integer instructions
    // (the same IEEE product, off the double pipe; a special case sets sp, see
    // TetF64), or on the double pipe with HW. The Laplace kind keeps the
    // hardware instruction beside each product instead (i64_dmul): with the
    // element-level redo its kernel spilled and ran 1% slower (measured).
    template <bool HW>
    __device__ __forceinline__ static T mul_off(T a, T b, bool &sp) {
        if constexpr (PREC == FP64 && !HW && KIND == POISSON)
            return i64_dmul(a, b);
        else if constexpr (PREC == FP64 && !HW)
            return i64_dmul_nz(a, b, sp);
        else if constexpr (PREC == FP64)
            return __dmul_rn(a, b);
        else
            return a * b;
    }
    // w / v for v > 0
    __device__ __forceinline__ static T recip_w(T v, T w) {
        if constexpr (PREC == FP64)
            return recip_scaled(v, w);
        else
            return w * recip_fast(v);
    }
    __device__ __forceinline__ static void mirror(T A[36]) {
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int s = 0; s < r; ++s) A[6 * r + s] = A[6 * s + r];
    }

    template <class CS>
    __device__ __forceinline__ static void update_point(int q, const V3<T> g[6], T vol, const CS &c, T A[36], T b[6]) {
        // q is a compile-time constant after unrolling; dispatch to the templated update
        switch (q) {
            case 0: upd<0>(g, vol, c, A, b); break;
            case 1: upd<1>(g, vol, c, A, b); break;
            case 2: upd<2>(g, vol, c, A, b); break;
            case 3: upd<3>(g, vol, c, A, b); break;
            case 4: upd<4>(g, vol, c, A, b); break;
            default: upd<5>(g, vol, c, A, b); break;
        }
    }
    template <int Q, class CS>
    __device__ __forceinline__ static void upd(const V3<T> g[6], T vol, const CS &c, T A[36], T b[6]) {
        if (KIND == POISSON)
            prism_poisson_update<T, Q>(g, vol, c(CPQ ? Q : 0), A, b);
        else
            prism_generic_update<T, Q>(g, vol, c, CPQ ? 20 * Q : 0, A, b);
    }
};

template <int KIND, int CPQ> struct ElemMath<PRISM, KIND, FP64, Q_PRISM6, CPQ> {
    template <class XS> __device__ __forceinline__ static void rel(const XS &x, V3<double> r[6]) {
        const V3<double> x0 = {x(0), x(1), x(2)};
        r[0] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 1; k < 6; ++k) r[k] = V3<double>{x(3 * k), x(3 * k + 1), x(3 * k + 2)} - x0;
    }
    // An element whose integer-instruction products met a special case is redone
    // from its inputs with those products on the double pipe (one branch per
    // element, never taken on ordinary data; the compiler barrier keeps the first
    // pass's values from being held for it).
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, double A[36], double b[6], bool &poor) {
        V3<double> r[6];
        rel(x, r);
        bool sp = false;
        uint8_t fl = PrismMath<KIND, FP64, CPQ>::qloop(r, c, A, b, poor, sp);
        if (sp) {
            asm volatile("" ::: "memory");
            rel(x, r);
            fl = PrismMath<KIND, FP64, CPQ>::template qloop<1, true>(r, c, A, b, poor, sp);
        }
        return fl;
    }
    // Two threads per element: this lane's zeta level; the lane's half out (pick_half).
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run_pair(const XS &x, const CS &c, double Ah[18], double bh[3], bool &poor,
                                                       int part, unsigned mask) {
        V3<double> r[6];
        rel(x, r);
        double A[36], b[6];
        bool sp = false;
        uint8_t fl = PrismMath<KIND, FP64, CPQ>::template qloop<2>(r, c, A, b, poor, sp, part, mask);
        if (sp) {   // both lanes of the pair: their shuffles within the pair alone
            asm volatile("" ::: "memory");
            rel(x, r);
            const unsigned pm = 3u << ((threadIdx.x & 31u) & ~1u);
            fl = PrismMath<KIND, FP64, CPQ>::template qloop<2, true>(r, c, A, b, poor, sp, part, pm);
        }
        pick_half<KIND>(A, b, Ah, bh, part);
        return fl;
    }
};

template <int KIND, int CPQ> struct ElemMath<PRISM, KIND, MIXED, Q_PRISM6, CPQ> {
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, float A[36], float b[6], bool &poor) {
        HiLo h[18];
#pragma unroll
        for (int j = 0; j < 18; ++j) h[j] = split_double(x(j));
        V3<float> r[6];
        r[0] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int k = 1; k < 6; ++k)
            r[k] = {diff_hilo(h[3 * k], h[0]), diff_hilo(h[3 * k + 1], h[1]), diff_hilo(h[3 * k + 2], h[2])};
        bool sp;   // set by the FP64 form only
        return PrismMath<KIND, MIXED, CPQ>::qloop(r, c, A, b, poor, sp);
    }
    // Two threads per element: this lane's zeta level; the lane's half out (pick_half).
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run_pair(const XS &x, const CS &c, float Ah[18], float bh[3], bool &poor,
                                                       int part, unsigned mask) {
        HiLo h[18];
#pragma unroll
        for (int j = 0; j < 18; ++j) h[j] = split_double(x(j));
        V3<float> r[6];
        r[0] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int k = 1; k < 6; ++k)
            r[k] = {diff_hilo(h[3 * k], h[0]), diff_hilo(h[3 * k + 1], h[1]), diff_hilo(h[3 * k + 2], h[2])};
        float A[36], b[6];
        bool sp;   // set by the FP64 form only
        const uint8_t fl = PrismMath<KIND, MIXED, CPQ>::template qloop<2>(r, c, A, b, poor, sp, part, mask);
        pick_half<KIND>(A, b, Ah, bh, part);
        return fl;
    }
    // Flagged element: Jacobian terms in double at every point, narrowed to float.
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t fixup(const XS &x, const CS &c, float A[36], float b[6]) {
        V3<double> r[6];
        const V3<double> x0 = {x(0), x(1), x(2)};
        r[0] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 1; k < 6; ++k) r[k] = V3<double>{x(3 * k), x(3 * k + 1), x(3 * k + 2)} - x0;
        const PrismFrame<double> f = prism_frame(r);
#pragma unroll
        for (int k = 0; k < 36; ++k) A[k] = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) b[k] = 0.0f;
        bool neg = false, degenerate = false;
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const double zb = Rule<Q_PRISM6>::zb(l), zt = Rule<Q_PRISM6>::zt(l);
            const V3<double> cx = zb * f.ub + zt * f.ut;
            const V3<double> cy = zb * f.vb + zt * f.vt;
            const V3<double> a3 = cross(cx, cy);
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                V3<double> gd[6], cz;
                const double det = prism_point(f, cx, cy, a3, l, t, gd, cz);
                degenerate |= !(fabs(det) > 1e-300);
                neg |= det < 0.0;
                V3<float> g[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) g[k] = to_f(gd[k]);
                const float vol = static_cast<float>(fabs(det) * Rule<Q_PRISM6>::w(3 * l + t));
                PrismMath<KIND, MIXED, CPQ>::update_point(3 * l + t, g, vol, c, A, b);
            }
        }
        if (KIND == POISSON) PrismMath<KIND, MIXED, CPQ>::mirror(A);
        if (degenerate) {
#pragma unroll
            for (int k = 0; k < 36; ++k) A[k] = 0.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k) b[k] = 0.0f;
            return 1 | 4;
        }
        return 1 | (neg ? 2 : 0);
    }
};

template <int KIND, int CPQ> struct ElemMath<PRISM, KIND, DWORD, Q_PRISM6, CPQ> {
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, double A[36], double b[6], bool &poor) {
        V3<DW> r[6];
        r[0] = {DW(0), DW(0), DW(0)};
#pragma unroll
        for (int k = 1; k < 6; ++k) r[k] = dw_edge_vec(x, k);
        const DwCoef<CS> cd{c};
        DW Ad[36], bd[6];
        bool sp;   // set by the FP64 form only
        const uint8_t fl = PrismMath<KIND, DWORD, CPQ>::qloop(r, cd, Ad, bd, poor, sp);
        poor = poor || !dw_group_ok<36>(Ad) || !dw_group_ok<6>(bd);
#pragma unroll
        for (int k = 0; k < 36; ++k) A[k] = dw_to_double(Ad[k]);
#pragma unroll
        for (int k = 0; k < 6; ++k) b[k] = dw_to_double(bd[k]);
        return fl;
    }
    // Two threads per element: this lane's zeta level; the lane's half out
    // (pick_half; each lane converts its own half).
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run_pair(const XS &x, const CS &c, double Ah[18], double bh[3], bool &poor,
                                                       int part, unsigned mask) {
        V3<DW> r[6];
        r[0] = {DW(0), DW(0), DW(0)};
#pragma unroll
        for (int k = 1; k < 6; ++k) r[k] = dw_edge_vec(x, k);
        const DwCoef<CS> cd{c};
        DW Ad[36], bd[6];
        bool sp;   // set by the FP64 form only
        const uint8_t fl = PrismMath<KIND, DWORD, CPQ>::template qloop<2>(r, cd, Ad, bd, poor, sp, part, mask);
        DW Adh[18], bdh[3];
        pick_half<KIND>(Ad, bd, Adh, bdh, part);
        // the group tests on the sums over both halves (the same on both lanes); the
        // shuffles run on every lane of `mask`, whatever the lane's flags
        const float sa = dw_abs_sum<18>(Adh), sb = dw_abs_sum<3>(bdh);
        const float ta = __fadd_rn(sa, pair_other(sa, mask)), tb = __fadd_rn(sb, pair_other(sb, mask));
        poor = poor || !dw_sum_ok(ta) || !dw_sum_ok(tb);
#pragma unroll
        for (int j = 0; j < 18; ++j) Ah[j] = dw_to_double(Adh[j]);
#pragma unroll
        for (int j = 0; j < 3; ++j) bh[j] = dw_to_double(bdh[j]);
        return fl;
    }
    // Flagged element: the whole element in double.
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t fixup(const XS &x, const CS &c, double A[36], double b[6]) {
        bool unused;
        return 1 | ElemMath<PRISM, KIND, FP64, Q_PRISM6, CPQ>::run(x, c, A, b, unused);
    }
};

// ---------------------------------------------------------------------------
// Several threads per element, one row each (the intra-element parallelism of
// the paper's SQS ordering, Algorithms 4 and 5, with the QSS loop order kept):
// a group of NS lanes per element, lane r owns row r of A^e and entry r of b^e.
// The Jacobian terms are formed once per element (tetrahedra) or once per point
// (prisms, lane q at point q) and passed to the group by shuffles, not recomputed
// per row as Algorithm 4 does.
// ---------------------------------------------------------------------------
template <int PREC> struct Form;
template <> struct Form<FP64> { using T = double; };
template <> struct Form<MIXED> { using T = float; };
template <> struct Form<DWORD> { using T = DW; };

// Edge vector x_k - x_0 in the arithmetic of a form (as ElemMath forms it).
template <int PREC, class XS> __device__ __forceinline__ V3<typename Form<PREC>::T> form_edge(const XS &x, int k) {
    if constexpr (PREC == FP64) {
        return V3<double>{x(3 * k), x(3 * k + 1), x(3 * k + 2)} - V3<double>{x(0), x(1), x(2)};
    } else if constexpr (PREC == DWORD) {
        return dw_edge_vec(x, k);
    } else {
        return {diff_hilo(split_double(x(3 * k)), split_double(x(0))),
                diff_hilo(split_double(x(3 * k + 1)), split_double(x(1))),
                diff_hilo(split_double(x(3 * k + 2)), split_double(x(2)))};
    }
}
__device__ __forceinline__ double form_abs(double v) { return fabs(v); }
__device__ __forceinline__ float form_abs(float v) { return fabsf(v); }
__device__ __forceinline__ DW form_abs(DW v) { return dw_abs(v); }
// w / v for v > 0
__device__ __forceinline__ double form_recip_w(double v, double w) { return recip_scaled(v, w); }
__device__ __forceinline__ float form_recip_w(float v, float w) { return w * recip_fast(v); }
__device__ __forceinline__ DW form_recip_w(DW v, DW w) { return w * dw_recip(v); }
template <class T> __device__ __forceinline__ T sel4(int r, T v0, T v1, T v2, T v3) {
    return r == 0 ? v0 : (r == 1 ? v1 : (r == 2 ? v2 : v3));
}
template <class T> __device__ __forceinline__ T sel3(int r, T v0, T v1, T v2) { return r == 0 ? v0 : (r == 1 ? v1 : v2); }
// Double-word results of a row: the group's windows (as dw_group_ok over the whole
// A^e and b^e, from the sums of the rows' magnitudes), then conversion.
template <int N>
__device__ __forceinline__ bool dw_rows_out(const DW *A, DW b, double *Ar, double &br, unsigned mask, int base,
                                            int lanes = N) {
    float sa = 0.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) sa = __fadd_rn(sa, fabsf(A[k].h));
    sa = grp_sum(sa, mask, base, lanes);
    const float sb = grp_sum(fabsf(b.h), mask, base, lanes);
#pragma unroll
    for (int k = 0; k < N; ++k) Ar[k] = dw_to_double(A[k]);
    br = dw_to_double(b);
    return (sa == 0.0f || (sa >= 0x1p-80f && sa <= 0x1p100f)) && (sb == 0.0f || (sb >= 0x1p-80f && sb <= 0x1p100f));
}

template <int KIND, int PREC, int QUAD, int CPQ> struct TetRows {
    using T = typename Form<PREC>::T;
    using CT = typename std::conditional<PREC == MIXED, float, double>::type;

    // Lane r of the group (lanes base .. base + 3): row r of A^e in Ar, b^e_r in br.
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, CT Ar[4], CT &br, bool &poor, int r,
                                                  unsigned mask, int base) {
        // edge e_r on lanes 1..3, then every edge on every lane
        const V3<T> er = form_edge<PREC>(x, r > 0 ? r : 1);
        V3<T> e[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) e[k] = grp_get(er, mask, base + 1 + k);
        // cofactor row a_r on lane r (a_1 = e2 x e3, a_2 = e3 x e1, a_3 = e1 x e2), det = e1 . a_1 on lane 1
        const V3<T> u = sel3(r % 3, e[0], e[1], e[2]), v = sel3((r + 1) % 3, e[0], e[1], e[2]);
        const V3<T> ar = cross(u, v);
        const T det_r = dot(e[0], ar);
        V3<T> a[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] = grp_get(ar, mask, base + 1 + k);
        const T det = grp_get(det_r, mask, base + 1);
        const bool neg = is_neg(det);
        poor = false;
        if constexpr (PREC != FP64) poor = tet_poor(hi_f(e[0]), hi_f(e[1]), hi_f(e[2]), hi_f(det));
        if constexpr (PREC == DWORD) poor = poor || !dw_det_ok(det.h);
        if constexpr (PREC == FP64) {
            if (degenerate_det(det)) {
#pragma unroll
                for (int s = 0; s < 4; ++s) Ar[s] = 0.0;
                br = 0.0;
                return 4;
            }
        }
        if constexpr (PREC == DWORD) {
            const DwCoef<CS> cd{c};
            DW A[4], b;
            products(a, det, neg, cd, r, A, b);
            poor = !dw_rows_out<4>(A, b, Ar, br, mask, base) || poor;
        } else {
            products(a, det, neg, c, r, Ar, br);
        }
        return neg ? 2 : 0;
    }

    // Row r of A^e and b^e_r from the cofactor rows a_1..a_3 and det J.
    template <class CS>
    __device__ __forceinline__ static void products(const V3<T> a[3], T det, bool neg, const CS &c, int r, T A[4],
                                                    T &b) {
        constexpr TetSums S = tet_sums<QUAD>();
        const T V = form_abs(det);
        const V3<T> a0 = -(a[0] + a[1] + a[2]);
        const V3<T> arow = sel4(r, a0, a[0], a[1], a[2]);
        if constexpr (KIND == POISSON) {
            // A_rs = W / |det| a_r . a_s
            const T k = form_recip_w(V, T(S.W));
            const V3<T> kr = k * arow;
            A[0] = dot(kr, a0);
#pragma unroll
            for (int s = 1; s < 4; ++s) A[s] = dot(kr, a[s - 1]);
            T bb[4];
            tet_poisson_b<T, QUAD, CPQ>(V, c, bb);
            b = sel4(r, bb[0], bb[1], bb[2], bb[3]);
        } else if constexpr (!CPQ) {
            // row r of the augmented bilinear form of tet_generic_aug
            const T f = form_recip_w(V, T(S.W));
            const T sm = neg ? T(-S.W / 4) : T(S.W / 4), sW = neg ? T(-S.W) : T(S.W);
            T M[3][4], M3[4];
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
            const T at[3] = {arow.x, arow.y, arow.z};
            T P[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const T col[3] = {M[0][k], M[1][k], M[2][k]};
                P[k] = dot3_add(at, col, M3[k]);
            }
            const T pr[3] = {P[0], P[1], P[2]};
#pragma unroll
            for (int s = 1; s < 4; ++s) {
                const T as[3] = {a[s - 1].x, a[s - 1].y, a[s - 1].z};
                A[s] = dot3_add(pr, as, P[3]);
            }
            A[0] = lin4(A[1], A[2], A[3], P[3]);
            if constexpr (S.M2[0][0] != S.M2[0][1]) {
                constexpr double ratio = (S.M2[0][0] - S.M2[0][1]) / S.M2[0][1];
                const T dl = ratio == 1.0 ? mu : mu * T(ratio);
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    if (s == r) A[s] += dl;
            }
            const T d[3] = {sW * c(17), sW * c(18), sW * c(19)};
            b = dot3_add(at, d, (V * c(16)) * T(S.W / 4));
        } else {
            // per-point coefficients: the weighted sums of tet_generic_products, row r
            const T inv = recip_fast(det);
            V3<T> g[4];
#pragma unroll
            for (int k = 1; k < 4; ++k) g[k] = inv * a[k - 1];
            g[0] = -(g[1] + g[2] + g[3]);
            const V3<T> gr = inv * arow;
            T Cb[3][3];
            V3<T> db = {T(0), T(0), T(0)}, Rr = {T(0), T(0), T(0)}, Ps[4];
            T Mr[4], er = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) Cb[i][j] = T(0);
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                Ps[s] = {T(0), T(0), T(0)};
                Mr[s] = T(0);
            }
#pragma unroll
            for (int q = 0; q < Rule<QUAD>::NQ; ++q) {
                const int o = 20 * q;
                const T w = T(Rule<QUAD>::w(q));
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) Cb[i][j] += w * c(o + 4 * (i + 1) + (j + 1));
                const V3<T> ci0 = {w * c(o + 4), w * c(o + 8), w * c(o + 12)};
                const V3<T> c0i = {w * c(o + 1), w * c(o + 2), w * c(o + 3)};
                db = db + w * V3<T>{c(o + 17), c(o + 18), c(o + 19)};
                const T phr = sel4(r, T(Rule<QUAD>::phi(q, 0)), T(Rule<QUAD>::phi(q, 1)), T(Rule<QUAD>::phi(q, 2)),
                                   T(Rule<QUAD>::phi(q, 3)));
                Rr = Rr + phr * c0i;
                er += (phr * w) * c(o + 16);
                const T c00 = (w * c(o)) * phr;
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    Ps[s] = Ps[s] + T(Rule<QUAD>::phi(q, s)) * ci0;
                    Mr[s] += c00 * T(Rule<QUAD>::phi(q, s));
                }
            }
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const V3<T> Cg = {Cb[0][0] * g[s].x + Cb[0][1] * g[s].y + Cb[0][2] * g[s].z,
                                  Cb[1][0] * g[s].x + Cb[1][1] * g[s].y + Cb[1][2] * g[s].z,
                                  Cb[2][0] * g[s].x + Cb[2][1] * g[s].y + Cb[2][2] * g[s].z};
                A[s] = V * (dot(gr, Cg) + dot(Ps[s], gr) + dot(Rr, g[s]) + Mr[s]);
            }
            b = V * (dot(db, gr) + er);
        }
    }
};

// Sixteen threads per tetrahedron (the entry-per-work-item mapping of the
// paper's entry-outer orderings, Sec. 3.3, Algorithm 7): lane sub = 4 r + s of the
// group (lanes base .. base + 15) delivers entry (r, s) of A^e, and lanes with
// s == 0 also b^e_r. Lanes 1..3 form edge k and cofactor row a_k (det J on lane
// 1) as TetRows does, shared by shuffles; every lane then forms row r of the
// QSS products (TetRows::products, so the four lanes of a row repeat it, as each
// entry's loop does in Algorithm 7) and keeps entry s.
template <int KIND, int PREC, int QUAD, int CPQ> struct TetEntries {
    using TR = TetRows<KIND, PREC, QUAD, CPQ>;
    using T = typename TR::T;
    using CT = typename TR::CT;

    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, CT &Ars, CT &br, bool &poor, int sub,
                                                  unsigned mask, int base) {
        const int r = sub >> 2, s = sub & 3;
        const int k = (sub >= 1 && sub <= 3) ? sub : 1;
        const V3<T> ek = form_edge<PREC>(x, k);
        V3<T> e[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) e[j] = grp_get(ek, mask, base + 1 + j);
        const V3<T> u = sel3(k % 3, e[0], e[1], e[2]), v = sel3((k + 1) % 3, e[0], e[1], e[2]);
        const V3<T> ak = cross(u, v);
        const T det_k = dot(e[0], ak);
        V3<T> a[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) a[j] = grp_get(ak, mask, base + 1 + j);
        const T det = grp_get(det_k, mask, base + 1);
        const bool neg = is_neg(det);
        poor = false;
        if constexpr (PREC != FP64) poor = tet_poor(hi_f(e[0]), hi_f(e[1]), hi_f(e[2]), hi_f(det));
        if constexpr (PREC == DWORD) poor = poor || !dw_det_ok(det.h);
        if constexpr (PREC == FP64) {
            if (degenerate_det(det)) {
                Ars = 0.0;
                br = 0.0;
                return 4;
            }
        }
        T Arow[4], b;
        if constexpr (PREC == DWORD) {
            const DwCoef<CS> cd{c};
            TR::products(a, det, neg, cd, r, Arow, b);
            // the windows of the double-word form on the group's sums of magnitudes
            const DW ars = sel4(s, Arow[0], Arow[1], Arow[2], Arow[3]);
            const DW bs = s == 0 ? b : DW(0.0f, 0.0f);
            double A1[1], b1;
            const bool ok = dw_rows_out<1>(&ars, bs, A1, b1, mask, base, 16);
            Ars = A1[0];
            br = b1;
            poor = !ok || poor;
        } else {
            TR::products(a, det, neg, c, r, Arow, b);
            Ars = sel4(s, Arow[0], Arow[1], Arow[2], Arow[3]);
            br = b;
        }
        return neg ? 2 : 0;
    }
};

template <int KIND, int PREC, int CPQ> struct PrismRows {
    using T = typename Form<PREC>::T;
    using CT = typename std::conditional<PREC == MIXED, float, double>::type;

    // Lane k of the group (lanes base .. base + 5): the Jacobian terms at point
    // q = k, then row k of A^e in Ar and b^e_k in br over all six points.
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, CT Ar[6], CT &br, bool &poor, int k,
                                                  unsigned mask, int base) {
        using R = Rule<Q_PRISM6>;
        const V3<T> ek = form_edge<PREC>(x, k > 0 ? k : 1);
        V3<T> rv[6];
        rv[0] = {T(0), T(0), T(0)};
#pragma unroll
        for (int j = 1; j < 6; ++j) rv[j] = grp_get(ek, mask, base + j);
        const PrismFrame<T> f = prism_frame(rv);
        // this lane's point: level l, triangle point t
        const int l = k >= 3, t = k - 3 * l;
        const T zb = l ? T(R::zb(1)) : T(R::zb(0)), zt = l ? T(R::zt(1)) : T(R::zt(0));
        const T h0 = t == 0 ? T(1.0 / 3.0) : T(1.0 / 12.0), h1 = t == 1 ? T(1.0 / 3.0) : T(1.0 / 12.0),
                h2 = t == 2 ? T(1.0 / 3.0) : T(1.0 / 12.0);
        const V3<T> cx = zb * f.ub + zt * f.ut;
        const V3<T> cy = zb * f.vb + zt * f.vt;
        const V3<T> cz = h0 * f.w0 + h1 * f.w1 + h2 * f.w2;
        const V3<T> a1 = cross(cy, cz), a2 = cross(cz, cx), a3 = cross(cx, cy);
        const T det = dot(cx, a1);
        bool bad = false, degenerate = false;
        if constexpr (PREC != FP64) {
            const V3<float> cxf = hi_f(cx), t1 = 2.0f * hi_f(cy) - cxf;
            bad = prism_poor(dot(cxf, cxf) + dot(t1, t1) * (1.0f / 3.0f), hi_f(cz), hi_f(det));
        }
        if constexpr (PREC == DWORD) bad = bad || !dw_det_ok(det.h);
        if constexpr (PREC == FP64) degenerate = degenerate_det(det);
        poor = grp_any(bad, mask, base, 6);
        const bool neg = grp_any(is_neg(det), mask, base, 6);
        degenerate = grp_any(degenerate, mask, base, 6);
        const T inv = recip_fast(det);
        const V3<T> rho1 = inv * a1, rho2 = inv * a2, rho3 = inv * a3;
        const T vol = form_abs(det) * T(R::w(0));
        if constexpr (PREC == DWORD) {
            const DwCoef<CS> cd{c};
            DW A[6], b;
            accumulate(rho1, rho2, rho3, vol, cd, k, mask, base, A, b);
            poor = !dw_rows_out<6>(A, b, Ar, br, mask, base) || poor;
        } else {
            accumulate(rho1, rho2, rho3, vol, c, k, mask, base, Ar, br);
        }
        if (degenerate) {
#pragma unroll
            for (int s = 0; s < 6; ++s) Ar[s] = CT(0);
            br = CT(0);
            return 4;
        }
        return neg ? 2 : 0;
    }

    // Row k over the six points: the point's rows of J^{-1} and vol from lane q.
    // With Phi_0s = phi_s, Phi_is = (grad phi_s)_i and u_b = vol sum_a Phi_ak c_ab,
    // A_ks += sum_b u_b Phi_bs = u_0 phi_s + z_s (u . P_{s mod 3}) + sigma_s h_{s mod 3} (u . rho_3),
    // grad phi_s = z_s P_a + sigma_s h_a rho_3 (P_0 = -(rho_1 + rho_2), P_1 = rho_1,
    // P_2 = rho_2; z = zb, sigma = -1 for the bottom nodes, z = zt, sigma = +1 for
    // the top ones; h_a = lambda_a / 2 at the triangle point).
    template <class CS>
    __device__ __forceinline__ static void accumulate(V3<T> rho1, V3<T> rho2, V3<T> rho3, T vol, const CS &c, int k,
                                                      unsigned mask, int base, T A[6], T &b) {
        using R = Rule<Q_PRISM6>;
        const int ak = k - 3 * (k >= 3);
#pragma unroll
        for (int s = 0; s < 6; ++s) A[s] = T(0);
        b = T(0);
#pragma unroll 1
        for (int q = 0; q < 6; ++q) {
            const V3<T> p1 = grp_get(rho1, mask, base + q), p2 = grp_get(rho2, mask, base + q),
                        p3 = grp_get(rho3, mask, base + q);
            const T vq = grp_get(vol, mask, base + q);
            const int lq = q >= 3, tq = q - 3 * lq;
            const T zb = lq ? T(R::zb(1)) : T(R::zb(0)), zt = lq ? T(R::zt(1)) : T(R::zt(0));
            T hq[3], lam[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                hq[a] = a == tq ? T(1.0 / 3.0) : T(1.0 / 12.0);
                lam[a] = a == tq ? T(2.0 / 3.0) : T(1.0 / 6.0);
            }
            const V3<T> P0 = -(p1 + p2);
            // this lane's shape function at q: value and gradient
            const T zk = k < 3 ? zb : zt;
            const T hk = sel3(ak, hq[0], hq[1], hq[2]);
            const V3<T> gk = zk * sel3(ak, P0, p1, p2) + (k < 3 ? -hk : hk) * p3;
            const T phk = sel3(ak, lam[0], lam[1], lam[2]) * zk;
            T u0 = T(0);
            V3<T> u;
            if constexpr (KIND == GENERIC) {
                const int o = CPQ ? 20 * q : 0;
                T ub[4];
#pragma unroll
                for (int bb = 0; bb < 4; ++bb)
                    ub[bb] = vq * (phk * c(o + bb) + gk.x * c(o + 4 + bb) + gk.y * c(o + 8 + bb) + gk.z * c(o + 12 + bb));
                u0 = ub[0];
                u = {ub[1], ub[2], ub[3]};
                b += vq * (c(o + 16) * phk + c(o + 17) * gk.x + c(o + 18) * gk.y + c(o + 19) * gk.z);
            } else {
                u = vq * gk;
                b += (vq * c(CPQ ? q : 0)) * phk;
            }
            const T w1 = dot(u, p1), w2 = dot(u, p2), w3 = dot(u, p3);
            const T uP[3] = {-(w1 + w2), w1, w2};
#pragma unroll
            for (int s = 0; s < 6; ++s) {
                const int as = s % 3;
                const T zs = s < 3 ? zb : zt;
                T v = zs * uP[as] + (s < 3 ? -hq[as] : hq[as]) * w3;
                if constexpr (KIND == GENERIC) v = v + u0 * (lam[as] * zs);
                A[s] += v;
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Shared-memory layout of one block: inputs and outputs of the tile's elements.
// AOS regions hold element records back to back; SOA regions hold one row of B
// scalars per plane. Every region starts on a 16-byte boundary.
// ---------------------------------------------------------------------------
template <int ET, int KIND, int PREC, int QUAD, int CPQ, int INL = AOS, int OUTL = AOS> struct BlockSmem {
    using CF = ElemCfg<ET, KIND, PREC, QUAD, CPQ>;
    using CT = typename CF::CT;
    // A^e entries written per element (upper triangle when packed)
    static constexpr int NAO = out_packed(OUTL) ? CF::NS * (CF::NS + 1) / 2 : CF::NA;
    __host__ __device__ static constexpr int64_t r16(int64_t v) { return (v + 15) / 16 * 16; }
    // geometry of the tile: coordinates, or node indices for INDEXED
    __host__ __device__ static constexpr int64_t x_bytes(int B) {
        return INL == INDEXED ? r16(int64_t(B) * CF::NS * 4) : int64_t(B) * CF::NX * 8;
    }
    __host__ __device__ static constexpr int64_t c_bytes(int B) { return r16(int64_t(B) * CF::NC * int64_t(sizeof(CT))); }
    __host__ __device__ static constexpr int64_t a_bytes(int B) { return r16(int64_t(B) * NAO * int64_t(sizeof(CT))); }
    __host__ __device__ static constexpr int64_t b_bytes(int B) { return r16(int64_t(B) * CF::NS * int64_t(sizeof(CT))); }
    __host__ __device__ static constexpr int64_t in_bytes(int B) { return x_bytes(B) + c_bytes(B); }
    __host__ __device__ static constexpr int64_t out_bytes(int B) { return a_bytes(B) + b_bytes(B); }
    __host__ __device__ static constexpr int64_t total(int B) { return in_bytes(B) > out_bytes(B) ? in_bytes(B) : out_bytes(B); }
};

__device__ __forceinline__ bool aligned16(const void *p, uint64_t bytes) {
    return ((reinterpret_cast<uintptr_t>(p) | bytes) & 15u) == 0;
}

// Shared-memory accessor: element record (stride 1) or plane rows (stride B).
template <class T> struct SmemSrc {
    const T *base;
    int stride;
    __device__ __forceinline__ T operator()(int j) const { return base[j * stride]; }
};

// Register accessor (coordinates gathered through the node table).
template <class T> struct RegSrc {
    const T *v;
    __device__ __forceinline__ T operator()(int j) const { return v[j]; }
};

// Coefficients from the function of a nodal field (CPQ == 2): u at every point
// of the rule (u_Q = sum_k phi_k(Q) u_k), then coefficient j of point q as the
// per-point layout indexes it (generic j = 20 q + k, Laplace j = q with d^0 in
// slot 16): p0 + u_Q (p1 + u_Q p2).
template <class CT, int ET, int KIND, int QUAD> struct FnSrc {
    static constexpr int NS = ET == TET ? 4 : 6;
    static constexpr int NQ = Rule<QUAD>::NQ;
    CT uq[NQ];
    const CoefFn *fn;
    template <class US> __device__ __forceinline__ FnSrc(const US &u, const CoefFn *f) : fn(f) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            CT s = CT(0);
#pragma unroll
            for (int k = 0; k < NS; ++k) s += CT(Rule<QUAD>::phi(q, k)) * u(k);
            uq[q] = s;
        }
    }
    __device__ __forceinline__ CT operator()(int j) const {
        const int q = KIND == POISSON ? j : j / 20;
        const int k = KIND == POISSON ? 16 : j - 20 * q;
        const CT u = uq[q];
        if constexpr (sizeof(CT) == 4)
            return fn->pf[0][k] + u * (fn->pf[1][k] + u * fn->pf[2][k]);
        else
            return fn->pd[0][k] + u * (fn->pd[1][k] + u * fn->pd[2][k]);
    }
};

// Coordinates of an element of an INDEXED set: vertex v is node idx[v] of the
// node array X ([n_nodes][3]). An index outside [0, n_nodes) is not followed
// (node 0 is read instead) and the result is false.
template <int NS>
__device__ __forceinline__ bool gather_nodes(const double *__restrict__ X, long long n_nodes, const int *idx,
                                             double x[3 * NS]) {
    bool ok = true;
#pragma unroll
    for (int v = 0; v < NS; ++v) {
        const long long i = idx[v];
        const bool in = static_cast<unsigned long long>(i) < static_cast<unsigned long long>(n_nodes);
        ok &= in;
        const double *q = X + 3 * (in ? i : 0);
#pragma unroll
        for (int d = 0; d < 3; ++d) x[3 * v + d] = __ldg(q + d);
    }
    return ok;
}

// Matrix-free output (OUTL == APPLY): y[idx[r]] += sum_s A_rs x[idx[s]] and
// f[idx[r]] += b_r (f may be null), by atomic additions.
template <class CT, int NS>
__device__ __forceinline__ void scatter_apply(const ElemParams &p, const int idx[NS], const CT A[NS * NS],
                                              const CT b[NS]) {
    const CT *x = static_cast<const CT *>(p.xv);
    CT *y = static_cast<CT *>(p.A);
    CT *f = static_cast<CT *>(p.B);
    CT xs[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) xs[s] = __ldg(x + idx[s]);
#pragma unroll
    for (int r = 0; r < NS; ++r) {
        CT yr = A[NS * r] * xs[0];
#pragma unroll
        for (int s = 1; s < NS; ++s) yr += A[NS * r + s] * xs[s];
        atomicAdd(y + idx[r], yr);
    }
    if (f) {
#pragma unroll
        for (int r = 0; r < NS; ++r) atomicAdd(f + idx[r], b[r]);
    }
}

// Append flagged elements of this warp to the fix-up list (one atomic per warp).
__device__ __forceinline__ void append_fixup(const ElemParams &p, bool poor, int64_t e) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, poor);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(p.fix_count, static_cast<unsigned>(__popc(m)));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (poor) {
        const unsigned slot = base + __popc(m & ((1u << lane) - 1u));
        if (slot < p.fix_cap)
            p.fix_list[slot] = (static_cast<unsigned long long>(p.item) << 40) | static_cast<unsigned long long>(e);
        else
            atomicOr(p.status, ST_FIXUP_OVERFLOW);
    }
}

// Copy `rows` rows of `bytes` from global rows (pitch gpitch elements) into
// shared rows (pitch spitch elements). Bulk copies issued by the lanes of warp 0
// when `bulk`; otherwise every thread of the block copies element by element.
template <class T>
__device__ __forceinline__ void stage_rows_in(T *s, int64_t spitch, const T *g, int64_t gpitch, int rows, int count,
                                              bool bulk, uint64_t *bar) {
    if (bulk) {
        if (threadIdx.x < 32)
            for (int r = threadIdx.x; r < rows; r += 32)
                bulk_g2s(s + r * spitch, g + r * gpitch, static_cast<unsigned>(count * sizeof(T)), bar);
    } else {
        for (int r = 0; r < rows; ++r)
            for (int i = threadIdx.x; i < count; i += blockDim.x) s[r * spitch + i] = g[r * gpitch + i];
    }
}

template <class T>
__device__ __forceinline__ void stage_rows_out(T *g, int64_t gpitch, const T *s, int64_t spitch, int rows, int count,
                                               bool bulk) {
    if (bulk) {
        if (threadIdx.x < 32) {
            for (int r = threadIdx.x; r < rows; r += 32)
                bulk_s2g(g + r * gpitch, s + r * spitch, static_cast<unsigned>(count * sizeof(T)));
        }
    } else {
        for (int r = 0; r < rows; ++r)
            for (int i = threadIdx.x; i < count; i += blockDim.x) st_stream(g + r * gpitch + i, s[r * spitch + i]);
    }
}

// ---------------------------------------------------------------------------
// One tile of nb <= blockDim.x elements starting at e0, for every thread of the
// block: inputs staged into shared memory by bulk copies (cp.async.bulk,
// completion on the block's mbarrier), computed one element per thread, written
// back by bulk copies from shared memory. Returns false (for the whole block) if
// a bounded wait on a copy ran out; the caller must then stop.
// ---------------------------------------------------------------------------
// One element through ElemMath, the coefficients read as given or, for the
// coefficient function (CPQ == 2), evaluated from the nodal field.
template <int ET, int KIND, int PREC, int QUAD, int CPQ, class XS, class CS, class CT>
__device__ __forceinline__ uint8_t run_elem(const XS &x, const CS &c, const CoefFn *fn, CT *A, CT *b, bool &poor) {
    if constexpr (CPQ == 2) {
        const FnSrc<CT, ET, KIND, QUAD> cf(c, fn);
        return ElemMath<ET, KIND, PREC, QUAD, CPQ>::run(x, cf, A, b, poor);
    } else {
        return ElemMath<ET, KIND, PREC, QUAD, CPQ>::run(x, c, A, b, poor);
    }
}
// Float values of a double accessor (the fix-up's coefficient function).
template <class S> struct NarrowSrc {
    const S &s;
    __device__ __forceinline__ float operator()(int j) const { return static_cast<float>(s(j)); }
};
// Double values of a float accessor (the nodal field of the mixed form).
template <class S> struct WidenSrc {
    const S &s;
    __device__ __forceinline__ double operator()(int j) const { return static_cast<double>(s(j)); }
};

template <int ET, int KIND, int PREC, int QUAD, int CPQ, class XS, class CS, class CT>
__device__ __forceinline__ uint8_t fix_elem(const XS &x, const CS &c, const CoefFn *fn, CT *A, CT *b) {
    if constexpr (CPQ == 2) {
        // a flagged element evaluates the coefficient function in double (u_Q and
        // c(u_Q)), so that coefficients near a root of their polynomial keep their
        // relative accuracy where poorly shaped elements amplify it
        const WidenSrc<CS> cw{c};
        const FnSrc<double, ET, KIND, QUAD> cfd(cw, fn);
        if constexpr (sizeof(CT) == 4) {
            const NarrowSrc<FnSrc<double, ET, KIND, QUAD>> cf{cfd};
            return ElemMath<ET, KIND, PREC, QUAD, CPQ>::fixup(x, cf, A, b);
        } else {
            return ElemMath<ET, KIND, PREC, QUAD, CPQ>::fixup(x, cfd, A, b);
        }
    } else {
        return ElemMath<ET, KIND, PREC, QUAD, CPQ>::fixup(x, c, A, b);
    }
}

//
// TPE > 1 (element-contiguous input and output, coefficient arrays, QSS):
// a group of TPE lanes of one warp per element, 32 / TPE groups per warp (for
// TPE = 6 five groups, lanes 30 and 31 idle); the block holds
// (blockDim.x / 32) x (32 / TPE) elements.
//   TPE == 2 (prisms): lanes 2j and 2j + 1, one zeta level of the point loop
//     each; each lane writes every other entry of its element.
//   TPE == NS (4 for tetrahedra, 6 for prisms): one row of A^e and one entry of
//     b^e per lane (TetRows, PrismRows).
template <int ET, int KIND, int PREC, int QUAD, int CPQ, int INL, int OUTL, int TPE = 1>
__device__ __forceinline__ bool process_tile(const ElemParams &p, int64_t e0, int nb, unsigned char *smem, uint64_t *bar,
                                             unsigned &phase, const TmaMaps *tm = nullptr,
                                             const CoefFn *fn = nullptr) {
    using CF = ElemCfg<ET, KIND, PREC, QUAD, CPQ>;
    using CT = typename CF::CT;
    using SM = BlockSmem<ET, KIND, PREC, QUAD, CPQ, INL, OUTL>;
    constexpr int NAO = SM::NAO;
    constexpr int NS = CF::NS, NX = CF::NX, NA = CF::NA, NC = CF::NC;
    static_assert(TPE == 1 || (INL == AOS && OUTL == AOS && CPQ < 2 &&
                               (TPE == NS || (TPE == 2 && ET == PRISM) || (TPE == 16 && ET == TET))),
                  "several threads per element: element-contiguous, coefficient arrays; 2 (prisms), NS or 16 (tets)");
    constexpr int EPW = 32 / TPE;            // elements (groups) per warp
    const int lane = threadIdx.x & 31;
    const int B = (blockDim.x >> 5) * EPW;   // elements per tile
    const int tid = (threadIdx.x >> 5) * EPW + lane / TPE;  // this thread's element in the tile
    const int sub = lane % TPE;              // its lane within the element's group
    double *sX = reinterpret_cast<double *>(smem);
    int *sN = reinterpret_cast<int *>(smem);  // INDEXED: the tile's node indices
    CT *sC = reinterpret_cast<CT *>(smem + SM::x_bytes(B));
    CT *sA = reinterpret_cast<CT *>(smem);
    CT *sB = reinterpret_cast<CT *>(smem + SM::a_bytes(B));
    const double *X = p.X;
    const CT *C = static_cast<const CT *>(p.C);
    CT *Aout = static_cast<CT *>(p.A);
    CT *Bout = static_cast<CT *>(p.B);
    const int64_t e = e0 + tid;
    const bool active = lane < EPW * TPE && tid < nb;

    // ---- stage inputs ----
    if (INL == SOA && tm && p.tma_in) {
        // two tensor copies: coordinate planes and coefficient planes of the tile
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            mbar_expect_tx(bar, unsigned(B) * NX * 8u + unsigned(B) * NC * unsigned(sizeof(CT)));
            tma_load_2d(sX, tm->x, int(e0), 0, bar);
            tma_load_2d(sC, tm->c, int(e0), 0, bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase, p.status);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            mbar_wait_bounded(bar, phase ^ 1u, nullptr);
            return false;
        }
    } else {
        // alignment of bases and SOA plane pitches, then of this tile's byte counts
        // (INDEXED: the node-index records of the tile, element-contiguous)
        const bool x_ok = INL == INDEXED ? aligned16(p.conn + e0 * NS, 0) : aligned16(X, INL == SOA ? uint64_t(p.xs) * 8 : 0);
        const bool c_ok = aligned16(C, INL == SOA ? uint64_t(p.cs) * sizeof(CT) : 0);
        constexpr unsigned kXe = INL == INDEXED ? NS * 4u : NX * 8u;  // geometry bytes per element
        const bool tX = x_ok && ((uint64_t(nb) * (INL == SOA ? 8 : kXe)) % 16 == 0);
        const bool tC = c_ok && ((uint64_t(nb) * (INL == SOA ? 1 : NC) * sizeof(CT)) % 16 == 0);
        const unsigned tx = (tX ? unsigned(nb) * kXe : 0u) + (tC ? unsigned(nb) * NC * unsigned(sizeof(CT)) : 0u);
        if (threadIdx.x == 0 && tx) {
            fence_proxy_async_smem();
            mbar_expect_tx(bar, tx);
        }
        if (tx) __syncwarp();
        if (INL == SOA) {
            stage_rows_in(sX, B, X + e0, p.xs, NX, nb, tX, bar);
            stage_rows_in(sC, B, C + e0, p.cs, NC, nb, tC, bar);
        } else if (INL == INDEXED) {
            stage_rows_in(sN, 0, p.conn + e0 * NS, 0, 1, nb * NS, tX, bar);
            stage_rows_in(sC, 0, C + e0 * NC, 0, 1, nb * NC, tC, bar);
        } else {
            stage_rows_in(sX, 0, X + e0 * NX, 0, 1, nb * NX, tX, bar);
            stage_rows_in(sC, 0, C + e0 * NC, 0, 1, nb * NC, tC, bar);
        }
        bool ok = true;
        if (tx) {
            ok = mbar_wait_bounded(bar, phase, p.status);
            phase ^= 1u;
        }
        if (__syncthreads_or(!ok)) {
            // a copy did not land: wait once more (bounded) so nothing is in flight
            if (tx) mbar_wait_bounded(bar, phase ^ 1u, nullptr);
            return false;
        }
    }

    // ---- compute ----
    CT A[NA], b[NS];   // TPE == 2: this lane's half (pair_entry) in A[j], b[j]; TPE == NS: row sub in A[0..NS), b[0]
    bool poor = false;
    bool idx_ok = true;  // INDEXED: every node index of this element is in range
    // lanes that take part in the pairs' exchanges (both lanes of an element)
    const unsigned pmask = TPE > 1 ? __ballot_sync(0xFFFFFFFFu, active) : 0xFFFFFFFFu;
    if (active) {
        const SmemSrc<CT> cs{INL == SOA ? sC + tid : sC + tid * NC, INL == SOA ? B : 1};
        uint8_t fl;
        if constexpr (INL == INDEXED) {
            double xr[NX];
            idx_ok = gather_nodes<NS>(X, p.n_nodes, sN + tid * NS, xr);
            fl = run_elem<ET, KIND, PREC, QUAD, CPQ>(RegSrc<double>{xr}, cs, fn, A, b, poor);
            if (!idx_ok) {
#pragma unroll
                for (int k = 0; k < NA; ++k) A[k] = CT(0);
#pragma unroll
                for (int k = 0; k < NS; ++k) b[k] = CT(0);
                fl = 8;
                poor = false;
            }
        } else {
            const SmemSrc<double> xs{INL == SOA ? sX + tid : sX + tid * NX, INL == SOA ? B : 1};
            if constexpr (TPE == 1)
                fl = run_elem<ET, KIND, PREC, QUAD, CPQ>(xs, cs, fn, A, b, poor);
            else if constexpr (TPE == 2)
                fl = ElemMath<ET, KIND, PREC, QUAD, CPQ>::run_pair(xs, cs, A, b, poor, sub, pmask);
            else if constexpr (ET == TET && TPE == 16)
                fl = TetEntries<KIND, PREC, QUAD, CPQ>::run(xs, cs, A[0], b[0], poor, sub, pmask, lane - sub);
            else if constexpr (ET == TET)
                fl = TetRows<KIND, PREC, QUAD, CPQ>::run(xs, cs, A, b[0], poor, sub, pmask, lane - sub);
            else
                fl = PrismRows<KIND, PREC, CPQ>::run(xs, cs, A, b[0], poor, sub, pmask, lane - sub);
        }
        if (PREC != FP64 && poor) fl |= 1;
        if (p.flags && sub == 0) p.flags[e] = fl;
    }
    if constexpr (OUTL == APPLY) {
        // matrix-free: scatter from registers (indices still in shared memory)
        if (active && idx_ok && !(PREC != FP64 && poor)) scatter_apply<CT, NS>(p, sN + tid * NS, A, b);
        if (PREC != FP64) append_fixup(p, active && poor, e);
        __syncthreads();   // the next tile's copies overwrite the indices
        return true;
    }
    __syncthreads();   // every input read: the output records reuse the same shared memory
    if (TPE == 2 && active) {
#pragma unroll
        for (int j = 0; j < NA / TPE; ++j) sA[tid * NAO + pair_entry<KIND>(j, sub)] = A[j];
#pragma unroll
        for (int j = 0; j < NS / TPE; ++j) sB[tid * NS + pair_b_entry<KIND>(j, sub)] = b[j];
    }
    if (TPE == NS && TPE > 2 && active) {
#pragma unroll
        for (int j = 0; j < NS; ++j) sA[tid * NAO + NS * sub + j] = A[j];
        sB[tid * NS + sub] = b[0];
    }
    if (TPE == 16 && active) {
        sA[tid * NAO + sub] = A[0];
        if ((sub & 3) == 0) sB[tid * NS + (sub >> 2)] = b[0];
    }
    if (TPE == 1 && active) {
        // entry k_out of the written A^e: (r, s) row-major, or its upper triangle
#pragma unroll
        for (int r = 0; r < NS; ++r)
#pragma unroll
            for (int s = out_packed(OUTL) ? r : 0; s < NS; ++s) {
                const int ko = out_packed(OUTL) ? packed_index(NS, r, s) : r * NS + s;
                if (out_soa(OUTL))
                    sA[ko * B + tid] = A[r * NS + s];
                else
                    sA[tid * NAO + ko] = A[r * NS + s];
            }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (out_soa(OUTL))
                sB[k * B + tid] = b[k];
            else
                sB[tid * NS + k] = b[k];
        }
    }
    if (PREC != FP64) append_fixup(p, active && poor && sub == 0, e);

    // ---- store outputs ----
    fence_proxy_async_smem();
    __syncthreads();
    if (out_soa(OUTL) && tm && p.tma_out) {
        if (threadIdx.x == 0) {
            tma_store_2d(tm->a, int(e0), 0, sA);
            tma_store_2d(tm->b, int(e0), 0, sB);
            bulk_commit();
            bulk_wait_read0();
        }
    } else {
        const bool a_ok = aligned16(Aout, out_soa(OUTL) ? uint64_t(p.os) * sizeof(CT) : 0);
        const bool b_ok = aligned16(Bout, out_soa(OUTL) ? uint64_t(p.os) * sizeof(CT) : 0);
        const bool tA = a_ok && ((uint64_t(nb) * (out_soa(OUTL) ? 1 : NAO) * sizeof(CT)) % 16 == 0);
        const bool tB = b_ok && ((uint64_t(nb) * (out_soa(OUTL) ? 1 : NS) * sizeof(CT)) % 16 == 0);
        if (out_soa(OUTL)) {
            stage_rows_out(Aout + e0, p.os, sA, B, NAO, nb, tA);
            stage_rows_out(Bout + e0, p.os, sB, B, NS, nb, tB);
        } else {
            stage_rows_out(Aout + e0 * NAO, 0, sA, 0, 1, nb * NAO, tA);
            stage_rows_out(Bout + e0 * NS, 0, sB, 0, 1, nb * NS, tB);
        }
        if ((tA || tB) && threadIdx.x < 32) {
            bulk_commit();
            bulk_wait_read0();
        }
    }
    __syncthreads();
    return true;
}

// ---------------------------------------------------------------------------
// Main kernel: tiles of blockDim.x elements, grid-stride over tiles.
// ---------------------------------------------------------------------------
template <int ET, int KIND, int PREC, int QUAD, int CPQ, int INL, int OUTL>
__device__ __forceinline__ void elem_tiles(const ElemParams &p, const TmaMaps *tm, const CoefFn *fn) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase = 0;
    const int B = blockDim.x;
    const int64_t ntiles = (p.n + B - 1) / B;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (p.skip_mod > 0 && tile % p.skip_mod == 0) {   // injected fault: no load, no store
            if (threadIdx.x == 0) atomicOr(p.status, ST_SKIPPED_TILES);
            continue;
        }
        const int64_t e0 = tile * B;
        const int nb = static_cast<int>(p.n - e0 < B ? p.n - e0 : B);
        if (!process_tile<ET, KIND, PREC, QUAD, CPQ, INL, OUTL>(p, e0, nb, smem, &bar, phase, tm, fn)) return;
    }
    if (threadIdx.x < 32) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <int ET, int KIND, int PREC, int QUAD, int CPQ, int INL, int OUTL>
// Launch bounds: 512 threads for float and double tetrahedra, 256 otherwise; the
// double-word Laplace prism is held to two resident 256-thread blocks per SM
// (128 registers: 2.77 -> 3.15 Gelem/s measured against 144 registers).
__global__ void __launch_bounds__(ET == TET && PREC != DWORD ? 512 : 256,
                                  (ET == PRISM && PREC == DWORD && KIND == POISSON) ? 2 : 0)
    elem_kernel(const ElemParams p, const __grid_constant__ TmaMaps tm, const __grid_constant__ CoefFn fn) {
    elem_tiles<ET, KIND, PREC, QUAD, CPQ, INL, OUTL>(p, &tm, &fn);
}

// The same kernel for FP64 tetrahedra with fewer registers per thread. Generic
// kind 104 (6M tetrahedra 4.10 -> 4.18 Gelem/s against 128 registers; 96 and 80
// spilled more and measured 4.14 and 4.04): still four warps per SM
// sub-partition, but the allocation under the bound keeps the double pipe busier
// (ncu 87.3% -> 89.7%). Laplace kind 80 (6M TET1 9.77 -> 10.58 Gelem/s against
// 100; 88 and 72 measured 10.29 and 10.52): six warps per sub-partition instead
// of five to cover the chains of the integer-instruction products. ptxas gets
// both the block bound (.maxntid 512) and the register bound (.maxnreg); with the
// register bound alone it allocates differently (the generic element-contiguous
// kernel spilled 360 bytes instead of 20).
template <int KIND, int QUAD, int CPQ, int INL, int OUTL>
__global__ void __launch_bounds__(512) __maxnreg__(KIND == POISSON ? 80 : 104)
    elem_kernel_f64t(const ElemParams p, const __grid_constant__ TmaMaps tm, const __grid_constant__ CoefFn fn) {
    elem_tiles<TET, KIND, FP64, QUAD, CPQ, INL, OUTL>(p, &tm, &fn);
}

// The same kernel for double-word tetrahedra with per-element coefficients and
// fewer registers per thread: generic kind 72 (6M tetrahedra 7.83 -> 8.46 Gelem/s
// against 88 registers; 80 and 64 measured 8.28 and 7.62), Laplace kind 48 (6M
// TET1 16.99 -> 19.44 Gelem/s against 60; 56 and 40 measured 18.37 and 17.28):
// more resident warps cover the chains of dependent double-word operations. Both
// bounds reach ptxas as for elem_kernel_f64t. Per-point coefficients keep
// elem_kernel (at 72 registers the generic kind spilled 3.5 KB).
template <int KIND, int QUAD, int CPQ, int INL, int OUTL>
__global__ void __launch_bounds__(256) __maxnreg__(KIND == POISSON ? 48 : 72)
    elem_kernel_dwt(const ElemParams p, const __grid_constant__ TmaMaps tm, const __grid_constant__ CoefFn fn) {
    elem_tiles<TET, KIND, DWORD, QUAD, CPQ, INL, OUTL>(p, &tm, &fn);
}
template <int KIND, int QUAD, int CPQ, int INL, int OUTL> const void *dw_tet_kernel() {
    if constexpr (CPQ == 0)
        return reinterpret_cast<const void *>(&elem_kernel_dwt<KIND, QUAD, CPQ, INL, OUTL>);
    else
        return reinterpret_cast<const void *>(&elem_kernel<TET, KIND, DWORD, QUAD, CPQ, INL, OUTL>);
}

// ---------------------------------------------------------------------------
// Prisms with two threads per element (element-contiguous input and output):
// tiles of blockDim.x / 2 elements, grid-stride over tiles.
// ---------------------------------------------------------------------------
template <int KIND, int PREC, int CPQ>
__global__ void __launch_bounds__(256)
    pair_kernel(const ElemParams p, const __grid_constant__ TmaMaps tm, const __grid_constant__ CoefFn fn) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase = 0;
    const int B = blockDim.x / 2;
    const int64_t ntiles = (p.n + B - 1) / B;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (p.skip_mod > 0 && tile % p.skip_mod == 0) {   // injected fault: no load, no store
            if (threadIdx.x == 0) atomicOr(p.status, ST_SKIPPED_TILES);
            continue;
        }
        const int64_t e0 = tile * B;
        const int nb = static_cast<int>(p.n - e0 < B ? p.n - e0 : B);
        if (!process_tile<PRISM, KIND, PREC, Q_PRISM6, CPQ, AOS, AOS, 2>(p, e0, nb, smem, &bar, phase, &tm, &fn))
            return;
    }
    if (threadIdx.x < 32) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// One group of NS lanes per element (TetRows, PrismRows), element-contiguous
// input and output: tiles of (blockDim.x / 32) x (32 / NS) elements, grid-stride
// over tiles.
// ---------------------------------------------------------------------------
template <int ET, int KIND, int PREC, int QUAD, int CPQ>
__global__ void __launch_bounds__(256)
    group_kernel(const ElemParams p, const __grid_constant__ TmaMaps tm, const __grid_constant__ CoefFn fn) {
    constexpr int TPE = ET == TET ? 4 : 6;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase = 0;
    const int B = (blockDim.x >> 5) * (32 / TPE);
    const int64_t ntiles = (p.n + B - 1) / B;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (p.skip_mod > 0 && tile % p.skip_mod == 0) {   // injected fault: no load, no store
            if (threadIdx.x == 0) atomicOr(p.status, ST_SKIPPED_TILES);
            continue;
        }
        const int64_t e0 = tile * B;
        const int nb = static_cast<int>(p.n - e0 < B ? p.n - e0 : B);
        if (!process_tile<ET, KIND, PREC, QUAD, CPQ, AOS, AOS, TPE>(p, e0, nb, smem, &bar, phase, &tm, &fn)) return;
    }
    if (threadIdx.x < 32) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Sixteen lanes per tetrahedron (TetEntries), element-contiguous input and
// output: tiles of (blockDim.x / 32) x 2 elements, grid-stride over tiles.
// ---------------------------------------------------------------------------
template <int KIND, int PREC, int QUAD, int CPQ>
__global__ void __launch_bounds__(256)
    entry_kernel(const ElemParams p, const __grid_constant__ TmaMaps tm, const __grid_constant__ CoefFn fn) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned phase = 0;
    const int B = (blockDim.x >> 5) * 2;
    const int64_t ntiles = (p.n + B - 1) / B;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (p.skip_mod > 0 && tile % p.skip_mod == 0) {   // injected fault: no load, no store
            if (threadIdx.x == 0) atomicOr(p.status, ST_SKIPPED_TILES);
            continue;
        }
        const int64_t e0 = tile * B;
        const int nb = static_cast<int>(p.n - e0 < B ? p.n - e0 : B);
        if (!process_tile<TET, KIND, PREC, QUAD, CPQ, AOS, AOS, 16>(p, e0, nb, smem, &bar, phase, &tm, &fn)) return;
    }
    if (threadIdx.x < 32) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// INDEXED geometry without staging: each thread reads its node-index record,
// gathers its nodes (the node array is small enough to stay in L2), reads its
// coefficient record and writes its results with vector accesses straight from
// and to global memory. No shared memory and no block barrier per tile, so many
// independent loads stay in flight per thread.
// ---------------------------------------------------------------------------
template <class T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int K = 4;
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int K = 2;
};
template <> struct Vec16<int> {
    using type = int4;
    static constexpr int K = 4;
};

// N values from src: 16-byte loads through the read-only path when the record is
// a whole number of 16-byte vectors and vec16 (the base is 16-byte aligned).
template <class T, int N> __device__ __forceinline__ void ld_record(const T *src, T v[N], bool vec16) {
    if constexpr ((N * sizeof(T)) % 16 == 0) {
        if (vec16) {
            using V = typename Vec16<T>::type;
            constexpr int K = Vec16<T>::K;
            const V *s = reinterpret_cast<const V *>(src);
#pragma unroll
            for (int i = 0; i < N / K; ++i) {
                const V q = __ldg(s + i);
                if constexpr (K == 4) {
                    v[4 * i] = q.x;
                    v[4 * i + 1] = q.y;
                    v[4 * i + 2] = q.z;
                    v[4 * i + 3] = q.w;
                } else {
                    v[2 * i] = q.x;
                    v[2 * i + 1] = q.y;
                }
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = __ldg(src + i);
}
// N values to dst with streaming stores, 16-byte vectors when possible.
template <class T, int N> __device__ __forceinline__ void st_record(T *dst, const T v[N], bool vec16) {
    if constexpr ((N * sizeof(T)) % 16 == 0) {
        if (vec16) {
            using V = typename Vec16<T>::type;
            constexpr int K = Vec16<T>::K;
            V *d = reinterpret_cast<V *>(dst);
#pragma unroll
            for (int i = 0; i < N / K; ++i) {
                V q;
                if constexpr (K == 4) {
                    q.x = v[4 * i];
                    q.y = v[4 * i + 1];
                    q.z = v[4 * i + 2];
                    q.w = v[4 * i + 3];
                } else {
                    q.x = v[2 * i];
                    q.y = v[2 * i + 1];
                }
                __stcs(d + i, q);
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) __stcs(dst + i, v[i]);
}

template <int ET, int KIND, int PREC, int QUAD, int CPQ, int OUTL>
__global__ void __launch_bounds__(ET == TET && PREC != DWORD ? 512 : 256)
    gather_kernel(const ElemParams p, const __grid_constant__ TmaMaps, const __grid_constant__ CoefFn) {
    using CF = ElemCfg<ET, KIND, PREC, QUAD, CPQ>;
    using CT = typename CF::CT;
    constexpr int NS = CF::NS, NX = CF::NX, NA = CF::NA, NC = CF::NC;
    // coefficient records up to 160 bytes are read whole into registers; longer
    // (per-point generic prisms) are read value by value where they are used
    constexpr bool kCoefRegs = NC * sizeof(CT) <= 160;
    const CT *C = static_cast<const CT *>(p.C);
    CT *Aout = static_cast<CT *>(p.A);
    CT *Bout = static_cast<CT *>(p.B);
    const bool n16 = aligned16(p.conn, 0), c16 = aligned16(C, 0);
    const bool o16 = OUTL == AOS && aligned16(Aout, 0) && aligned16(Bout, 0);
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    // whole blocks iterate together (the fix-up append is warp-collective)
    for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < p.n; base += stride) {
        const int64_t e = base + threadIdx.x;
        const bool active = e < p.n;
        bool poor = false;
        if (active) {
            int idx[NS];
            ld_record<int, NS>(p.conn + e * NS, idx, n16);
            double xr[NX];
            const bool ok = gather_nodes<NS>(p.X, p.n_nodes, idx, xr);
            CT A[NA], b[NS];
            uint8_t fl;
            if constexpr (kCoefRegs) {
                CT cv[NC];
                ld_record<CT, NC>(C + e * NC, cv, c16);
                fl = ElemMath<ET, KIND, PREC, QUAD, CPQ>::run(RegSrc<double>{xr}, RegSrc<CT>{cv}, A, b, poor);
            } else {
                const Src<AOS, CT> cs{C + e * NC, 0};
                fl = ElemMath<ET, KIND, PREC, QUAD, CPQ>::run(RegSrc<double>{xr}, cs, A, b, poor);
            }
            if (!ok) {
#pragma unroll
                for (int k = 0; k < NA; ++k) A[k] = CT(0);
#pragma unroll
                for (int k = 0; k < NS; ++k) b[k] = CT(0);
                fl = 8;
                poor = false;
            }
            if (PREC != FP64 && poor) fl |= 1;
            if (p.flags) p.flags[e] = fl;
            if constexpr (OUTL == APPLY) {
                if (ok && !(PREC != FP64 && poor)) scatter_apply<CT, NS>(p, idx, A, b);  // flagged: the fix-up adds
            } else if (OUTL == SOA) {
#pragma unroll
                for (int k = 0; k < NA; ++k) st_stream(Aout + k * p.os + e, A[k]);
#pragma unroll
                for (int k = 0; k < NS; ++k) st_stream(Bout + k * p.os + e, b[k]);
            } else {
                st_record<CT, NA>(Aout + e * NA, A, o16);
                st_record<CT, NS>(Bout + e * NS, b, o16);
            }
        }
        if (PREC != FP64) append_fixup(p, active && poor, e);
    }
}

// ---------------------------------------------------------------------------
// Fix-up of one flagged element (mixed and double-word forms): read straight
// from global memory, Jacobian terms in double, results overwrite the main
// kernel's.
// ---------------------------------------------------------------------------
template <int ET, int KIND, int PREC, int QUAD, int CPQ, int INL, int OUTL>
__device__ __forceinline__ void fixup_element(const ElemParams &p, int64_t e, const CoefFn *fn = nullptr) {
    using CF = ElemCfg<ET, KIND, PREC, QUAD, CPQ>;
    using CT = typename CF::CT;
    constexpr int NS = CF::NS, NX = CF::NX, NA = CF::NA, NC = CF::NC;
    const CT *C = static_cast<const CT *>(p.C);
    CT *Aout = static_cast<CT *>(p.A);
    CT *Bout = static_cast<CT *>(p.B);
    CT A[NA], b[NS];
    uint8_t fl;
    if (INL == SOA) {
        const Src<SOA, double> xs{p.X + e, p.xs};
        const Src<SOA, CT> cs{C + e, p.cs};
        fl = fix_elem<ET, KIND, PREC, QUAD, CPQ>(xs, cs, fn, A, b);
    } else if (INL == INDEXED) {
        double xr[NX];
        gather_nodes<NS>(p.X, p.n_nodes, p.conn + e * NS, xr);  // flagged elements have valid indices
        const Src<AOS, CT> cs{C + e * NC, 0};
        fl = fix_elem<ET, KIND, PREC, QUAD, CPQ>(RegSrc<double>{xr}, cs, fn, A, b);
    } else {
        const Src<AOS, double> xs{p.X + e * NX, 0};
        const Src<AOS, CT> cs{C + e * NC, 0};
        fl = fix_elem<ET, KIND, PREC, QUAD, CPQ>(xs, cs, fn, A, b);
    }
    if constexpr (OUTL == APPLY) {
        if (INL == INDEXED) scatter_apply<CT, NS>(p, p.conn + e * NS, A, b);
    } else {
        constexpr int NAO = out_packed(OUTL) ? NS * (NS + 1) / 2 : NA;
#pragma unroll
        for (int r = 0; r < NS; ++r)
#pragma unroll
            for (int s = out_packed(OUTL) ? r : 0; s < NS; ++s) {
                const int ko = out_packed(OUTL) ? packed_index(NS, r, s) : r * NS + s;
                if (out_soa(OUTL))
                    Aout[ko * p.os + e] = A[r * NS + s];
                else
                    Aout[e * NAO + ko] = A[r * NS + s];
            }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
            if (out_soa(OUTL))
                Bout[k * p.os + e] = b[k];
            else
                Bout[e * NS + k] = b[k];
        }
    }
    if (p.flags) p.flags[e] = fl;
}

// Fix-up kernel of one call: grid-stride over the list written by the main kernel.
template <int ET, int KIND, int PREC, int QUAD, int CPQ, int INL, int OUTL>
__global__ void __launch_bounds__(256) fixup_kernel(const ElemParams p, const __grid_constant__ CoefFn fn) {
    const unsigned cnt = *p.fix_count;
    const unsigned n = cnt < p.fix_cap ? cnt : p.fix_cap;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t e = static_cast<int64_t>(p.fix_list[i] & ((1ull << 40) - 1));
        if (e >= p.n) {
            atomicOr(p.status, ST_BAD_TILE);
            continue;
        }
        fixup_element<ET, KIND, PREC, QUAD, CPQ, INL, OUTL>(p, e, &fn);
    }
}

}  // namespace fe
