// The kernels' quadrature tables, read back on the host (fe_rule_table): the same
// compile-time constants the kernels use, so that a test can compare them with an
// independent statement of the rules.
#include "fe_device.cuh"
#include "fe_runtime.h"

namespace {

template <int QUAD> int rule_table(int ns, int max_points, double *weights, double *shape_values) {
    using R = fe::Rule<QUAD>;
    if (max_points < R::NQ) return -1;
    for (int q = 0; q < R::NQ; ++q) {
        if (weights) weights[q] = R::w(q);
        if (shape_values)
            for (int r = 0; r < ns; ++r) shape_values[q * ns + r] = R::phi(q, r);
    }
    return R::NQ;
}

}  // namespace

extern "C" fe_status fe_rule_table(fe_quad quad, int max_points, int *n_points, double *weights,
                                   double *shape_values) {
    using namespace fe;
    if (!n_points) return set_error(nullptr, FE_ERR_INVALID_ARG, "null argument");
    int n = -1;
    switch (quad) {
        case FE_QUAD_TET1: n = rule_table<Q_TET1>(4, max_points, weights, shape_values); break;
        case FE_QUAD_TET4: n = rule_table<Q_TET4>(4, max_points, weights, shape_values); break;
        case FE_QUAD_PRISM6: n = rule_table<Q_PRISM6>(6, max_points, weights, shape_values); break;
        default: return set_error(nullptr, FE_ERR_INVALID_ARG, "unknown rule");
    }
    if (n < 0) return set_error(nullptr, FE_ERR_INVALID_ARG, "max_points smaller than the rule");
    *n_points = n;
    return FE_OK;
}
