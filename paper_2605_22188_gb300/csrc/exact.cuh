// Shared by the certificate kernels: the layout of the exact-splitting product
// of X^T zeta (the digit slices and the per-job partial products) and the
// FP64 combine of one entry with its error bound.
#pragma once

#include "engine.h"

namespace kglm {

// Entry (b, j) of X^T zeta from the job partials P_t (slice t at Qs + t * stride,
// row b at b * p): tau_b sigma_j sum_t w_t P_t[b][j], summed in job order.  err:
// tau_b sigma_j n E, a bound on the distance to the exact product.
__device__ __forceinline__ double exact_q(const float* Qs, int nq, size_t stride, const double* w, size_t idx,
                                          double scale, double ebound, double* err) {
    double acc = 0.0;
    for (int t = 0; t < nq; ++t) acc += w[t] * (double)__ldg(Qs + (size_t)t * stride + idx);
    *err = scale * ebound;
    return acc * scale;
}

}  // namespace kglm
