// Loop-ordering study (Sec. 3.3): the SQS and SSQ orderings of Algorithms 4-7 in
// the mixed form, beside the QSS kernels of the library, for a counterpart of the
// paper's Table 7. Geometrically linear tetrahedra compute the Jacobian once
// (Algorithms 5, 7); prisms recompute it at every point for every row (SQS,
// Algorithm 4) or for every entry (SSQ, Algorithm 6). The loops over rows,
// entries and points are rolled, as the algorithms are written; the element
// matrix then lives in local memory. Edge vectors, the shape test and the
// double-Jacobian fix-up are those of the mixed form.
#include "fe_inst.cuh"

namespace fe {

// Phi_{a,k} at one point: a = 0 the shape value, a = 1..3 the gradient.
struct Col {
    float v[4];
};
__device__ __forceinline__ Col col(float phi, V3<float> g) { return {{phi, g.x, g.y, g.z}}; }

// sum_{a,b} c^{a;b} Phi_{a,i} Phi_{b,j} (Laplace: the gradient block, c = identity)
template <int KIND, class CS> __device__ __forceinline__ float a_term(const CS &c, int o, const Col &pi, const Col &pj) {
    if (KIND == POISSON) return pi.v[1] * pj.v[1] + pi.v[2] * pj.v[2] + pi.v[3] * pj.v[3];
    float s = 0.0f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        float t = 0.0f;
#pragma unroll
        for (int bb = 0; bb < 4; ++bb) t += c(o + 4 * a + bb) * pj.v[bb];
        s += pi.v[a] * t;
    }
    return s;
}
// sum_a d^a Phi_{a,i} (Laplace: d^0 phi_i)
template <int KIND, class CS> __device__ __forceinline__ float b_term(const CS &c, int o, int oq, const Col &pi) {
    if (KIND == POISSON) return c(oq) * pi.v[0];
    return c(o + 16) * pi.v[0] + c(o + 17) * pi.v[1] + c(o + 18) * pi.v[2] + c(o + 19) * pi.v[3];
}

template <class T> __device__ __forceinline__ T pick6(int k, T a0, T a1, T a2, T a3, T a4, T a5) {
    return k == 0 ? a0 : k == 1 ? a1 : k == 2 ? a2 : k == 3 ? a3 : k == 4 ? a4 : a5;
}

// Tetrahedron (geometrically linear): Jacobian and gradients once, then rows
// (SQS: i, q, j) or entries (SSQ: i, j, q).
template <int KIND, int ORD, int QUAD, int CPQ> struct StudyTet {
    template <class XS, class CS>
    __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, float A[16], float b[4], bool &poor) {
        using R = Rule<QUAD>;
        HiLo h[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) h[j] = split_double(x(j));
        V3<float> e[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            e[k] = {diff_hilo(h[3 * (k + 1)], h[0]), diff_hilo(h[3 * (k + 1) + 1], h[1]), diff_hilo(h[3 * (k + 1) + 2], h[2])};
        const TetGeo<float> geo = tet_geometry(e[0], e[1], e[2]);
        poor = tet_poor(e[0], e[1], e[2], geo.det);
        const float V = fabsf(geo.det), inv = 1.0f / geo.det;
        V3<float> g[4];
        g[1] = inv * geo.a[0];
        g[2] = inv * geo.a[1];
        g[3] = inv * geo.a[2];
        g[0] = -1.0f * (g[1] + g[2] + g[3]);
        float Al[16];
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            if (ORD == MIXED_SQS) {
                float row[4] = {0.0f, 0.0f, 0.0f, 0.0f}, bi = 0.0f;
#pragma unroll 1
                for (int q = 0; q < R::NQ; ++q) {
                    const float vol = V * float(R::w(q));
                    const int o = CPQ ? 20 * q : 0, oq = CPQ ? q : 0;
                    const Col pi = col(phi_at<QUAD>(q, i), g[i]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) row[j] += vol * a_term<KIND>(c, o, pi, col(phi_at<QUAD>(q, j), g[j]));
                    bi += vol * b_term<KIND>(c, o, oq, pi);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) Al[4 * i + j] = row[j];
                b[i] = bi;
            } else {
                float bi = 0.0f;
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    float aij = 0.0f;
#pragma unroll 1
                    for (int q = 0; q < R::NQ; ++q) {
                        const float vol = V * float(R::w(q));
                        const int o = CPQ ? 20 * q : 0, oq = CPQ ? q : 0;
                        const Col pi = col(phi_at<QUAD>(q, i), g[i]);
                        aij += vol * a_term<KIND>(c, o, pi, col(phi_at<QUAD>(q, j), g[j]));
                        if (i == j) bi += vol * b_term<KIND>(c, o, oq, pi);
                    }
                    Al[4 * i + j] = aij;
                }
                b[i] = bi;
            }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) A[k] = Al[k];
        return geo.det < 0.0f ? 2 : 0;
    }
    // shape value phi_k at point q of the rule (q, k run-time)
    template <int Q> __device__ __forceinline__ static float phi_at(int q, int k) {
        return Q == Q_TET1 ? 0.25f : (q == k ? float(kTet4B) : float(kTet4A));
    }
};

// Prism (geometrically multilinear): the Jacobian at point q is recomputed for
// every row (SQS) or every entry (SSQ).
template <int KIND, int ORD, int CPQ> struct StudyPrism {
    // gradients and volume at point q = 3 l + t
    __device__ __forceinline__ static float point(const PrismFrame<float> &f, int q, V3<float> g[6], float &fxy,
                                                  V3<float> &cz) {
        using R = Rule<Q_PRISM6>;
        const int l = q / 3, t = q - 3 * l;
        const float zb = l ? float(R::zb(1)) : float(R::zb(0)), zt = l ? float(R::zt(1)) : float(R::zt(0));
        const V3<float> cx = zb * f.ub + zt * f.ut;
        const V3<float> cy = zb * f.vb + zt * f.vt;
        const V3<float> t1 = 2.0f * cy - cx;
        fxy = dot(cx, cx) + dot(t1, t1) * (1.0f / 3.0f);
        return prism_point(f, cx, cy, cross(cx, cy), l, t, g, cz);
    }
    __device__ __forceinline__ static float phi(int q, int k) {
        using R = Rule<Q_PRISM6>;
        const int l = q / 3, t = q - 3 * l, kk = k < 3 ? k : k - 3;
        const float lam = t == kk ? float(2.0 / 3.0) : float(1.0 / 6.0);
        const float z = k < 3 ? (l ? float(R::zb(1)) : float(R::zb(0))) : (l ? float(R::zt(1)) : float(R::zt(0)));
        return lam * z;
    }
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
        const PrismFrame<float> f = prism_frame(r);
        const float w = float(Rule<Q_PRISM6>::w(0));
        bool neg = false;
        poor = false;
        float Al[36];
#pragma unroll 1
        for (int i = 0; i < 6; ++i) {
            float bi = 0.0f;
            if (ORD == MIXED_SQS) {
                float row[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 1
                for (int q = 0; q < 6; ++q) {
                    V3<float> g[6], cz;
                    float fxy;
                    const float det = point(f, q, g, fxy, cz);
                    if (i == 0) {
                        poor |= prism_poor(fxy, cz, det);
                        neg |= det < 0.0f;
                    }
                    const float vol = fabsf(det) * w;
                    const int o = CPQ ? 20 * q : 0, oq = CPQ ? q : 0;
                    const Col pi = col(phi(q, i), pick6(i, g[0], g[1], g[2], g[3], g[4], g[5]));
#pragma unroll
                    for (int j = 0; j < 6; ++j) row[j] += vol * a_term<KIND>(c, o, pi, col(phi(q, j), g[j]));
                    bi += vol * b_term<KIND>(c, o, oq, pi);
                }
#pragma unroll
                for (int j = 0; j < 6; ++j) Al[6 * i + j] = row[j];
            } else {
#pragma unroll 1
                for (int j = 0; j < 6; ++j) {
                    float aij = 0.0f;
#pragma unroll 1
                    for (int q = 0; q < 6; ++q) {
                        V3<float> g[6], cz;
                        float fxy;
                        const float det = point(f, q, g, fxy, cz);
                        if (i == 0 && j == 0) {
                            poor |= prism_poor(fxy, cz, det);
                            neg |= det < 0.0f;
                        }
                        const float vol = fabsf(det) * w;
                        const int o = CPQ ? 20 * q : 0, oq = CPQ ? q : 0;
                        const Col pi = col(phi(q, i), pick6(i, g[0], g[1], g[2], g[3], g[4], g[5]));
                        const Col pj = col(phi(q, j), pick6(j, g[0], g[1], g[2], g[3], g[4], g[5]));
                        aij += vol * a_term<KIND>(c, o, pi, pj);
                        if (i == j) bi += vol * b_term<KIND>(c, o, oq, pi);
                    }
                    Al[6 * i + j] = aij;
                }
            }
            b[i] = bi;
        }
#pragma unroll
        for (int k = 0; k < 36; ++k) A[k] = Al[k];
        return neg ? 2 : 0;
    }
};

#define FE_STUDY_TET(ORD)                                                                                      \
    template <int KIND, int QUAD, int CPQ> struct ElemMath<TET, KIND, ORD, QUAD, CPQ> {                         \
        template <class XS, class CS>                                                                          \
        __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, float A[16], float b[4], bool &poor) { \
            return StudyTet<KIND, ORD, QUAD, CPQ>::run(x, c, A, b, poor);                                      \
        }                                                                                                      \
        template <class XS, class CS>                                                                          \
        __device__ __forceinline__ static uint8_t fixup(const XS &x, const CS &c, float A[16], float b[4]) {   \
            return ElemMath<TET, KIND, MIXED, QUAD, CPQ>::fixup(x, c, A, b);                                   \
        }                                                                                                      \
    };
#define FE_STUDY_PRISM(ORD)                                                                                    \
    template <int KIND, int CPQ> struct ElemMath<PRISM, KIND, ORD, Q_PRISM6, CPQ> {                             \
        template <class XS, class CS>                                                                          \
        __device__ __forceinline__ static uint8_t run(const XS &x, const CS &c, float A[36], float b[6], bool &poor) { \
            return StudyPrism<KIND, ORD, CPQ>::run(x, c, A, b, poor);                                          \
        }                                                                                                      \
        template <class XS, class CS>                                                                          \
        __device__ __forceinline__ static uint8_t fixup(const XS &x, const CS &c, float A[36], float b[6]) {   \
            return ElemMath<PRISM, KIND, MIXED, Q_PRISM6, CPQ>::fixup(x, c, A, b);                             \
        }                                                                                                      \
    };
FE_STUDY_TET(MIXED_SQS)
FE_STUDY_TET(MIXED_SSQ)
FE_STUDY_PRISM(MIXED_SQS)
FE_STUDY_PRISM(MIXED_SSQ)
#undef FE_STUDY_TET
#undef FE_STUDY_PRISM

#define FE_STUDY_CASE(ET, ORD, QUAD, KD, CP)                                                       \
    if (type == ET && order == (ORD == MIXED_SQS ? 1 : 2) && quad == QUAD && kind == KD && cpq == CP) \
        return reinterpret_cast<const void *>(&elem_kernel<ET, KD, ORD, QUAD, CP, AOS, AOS>);
#define FE_STUDY_FIX(ET, ORD, QUAD, KD, CP)                                                        \
    if (type == ET && order == (ORD == MIXED_SQS ? 1 : 2) && quad == QUAD && kind == KD && cpq == CP) \
        return reinterpret_cast<const void *>(&fixup_kernel<ET, KD, ORD, QUAD, CP, AOS, AOS>);
#define FE_STUDY_ALL(M)                                                                            \
    M(TET, MIXED_SQS, Q_TET1, 0, 0) M(TET, MIXED_SQS, Q_TET1, 0, 1) M(TET, MIXED_SQS, Q_TET1, 1, 0)    \
    M(TET, MIXED_SQS, Q_TET1, 1, 1) M(TET, MIXED_SQS, Q_TET4, 0, 0) M(TET, MIXED_SQS, Q_TET4, 0, 1)    \
    M(TET, MIXED_SQS, Q_TET4, 1, 0) M(TET, MIXED_SQS, Q_TET4, 1, 1) M(TET, MIXED_SSQ, Q_TET1, 0, 0)    \
    M(TET, MIXED_SSQ, Q_TET1, 0, 1) M(TET, MIXED_SSQ, Q_TET1, 1, 0) M(TET, MIXED_SSQ, Q_TET1, 1, 1)    \
    M(TET, MIXED_SSQ, Q_TET4, 0, 0) M(TET, MIXED_SSQ, Q_TET4, 0, 1) M(TET, MIXED_SSQ, Q_TET4, 1, 0)    \
    M(TET, MIXED_SSQ, Q_TET4, 1, 1) M(PRISM, MIXED_SQS, Q_PRISM6, 0, 0)                                \
    M(PRISM, MIXED_SQS, Q_PRISM6, 0, 1) M(PRISM, MIXED_SQS, Q_PRISM6, 1, 0)                            \
    M(PRISM, MIXED_SQS, Q_PRISM6, 1, 1) M(PRISM, MIXED_SSQ, Q_PRISM6, 0, 0)                            \
    M(PRISM, MIXED_SSQ, Q_PRISM6, 0, 1) M(PRISM, MIXED_SSQ, Q_PRISM6, 1, 0)                            \
    M(PRISM, MIXED_SSQ, Q_PRISM6, 1, 1)

const void *kernel_study(int type, int kind, int quad, int cpq, int order) {
    FE_STUDY_ALL(FE_STUDY_CASE)
    return nullptr;
}
const void *kernel_fixup_study(int type, int kind, int quad, int cpq, int order) {
    FE_STUDY_ALL(FE_STUDY_FIX)
    return nullptr;
}

}  // namespace fe
