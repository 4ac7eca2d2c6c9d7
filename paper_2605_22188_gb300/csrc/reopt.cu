// Re-optimization on the rounded support of each node (§4.3): projected
// FISTA (the prox is the projection onto [-M, M]) for
//   v(S) = min { F(X_S b) + lambda2 ||b||^2 : ||b||_inf <= M },
// one CTA per node, FP64, warm-started from the node's relaxed beta on S.
// Least squares runs on the k x k Gram block (X^T X)_SS and (X^T y)_S; the
// logistic loss needs the gather-and-reduce passes over the n samples of
// §4.3 (s_i = sum_r X_{i,S_r} b_r and grad_r = sum_i X_{i,S_r} R_i).  The step
// is 1/L with L from the Gershgorin bound of the Gram block (an upper bound
// of the largest eigenvalue).  The objective v(S) is recomputed exactly in a
// final pass over the samples.
#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;

struct ReoptShared {
    int S[kMaxK];
    double A[kMaxK * kMaxK];
    double c[kMaxK];
    double bcur[kMaxK], bold[kMaxK], v[kMaxK], grad[kMaxK], bnew[kMaxK];
    double part[NW][kMaxK];
    double red[4 * NW];
    double L;
    int ks;
};

// grad = gradient of F(X_S b) + lambda2 ||b||^2 at sh.v (in sh.grad)
__device__ void gradient(const ReoptArgs& a, ReoptShared& sh, const double* vec) {
    const int ks = sh.ks;
    if (a.kind == kLSQ) {
        // 2 (A b - c) with A = G_SS + lambda2 I
        for (int r = threadIdx.x; r < ks; r += NT) {
            double s = 0.0;
            for (int t = 0; t < ks; ++t) s += sh.A[r * kMaxK + t] * vec[t];
            sh.grad[r] = 2.0 * (s - sh.c[r]);
        }
        __syncthreads();
        return;
    }
    double acc[kMaxK];
    for (int r = 0; r < ks; ++r) acc[r] = 0.0;
    for (int i = threadIdx.x; i < a.n; i += NT) {
        double s = 0.0;
        for (int r = 0; r < ks; ++r) s += a.Xt[(size_t)sh.S[r] * a.n + i] * vec[r];
        const double d = dloss(s, a.y[i], a.kind);
        for (int r = 0; r < ks; ++r) acc[r] += a.Xt[(size_t)sh.S[r] * a.n + i] * d;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int r = 0; r < ks; ++r) {
        const double x = warp_sum(acc[r]);
        if (l == 0) sh.part[w][r] = x;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < ks; r += NT) {
        double s = 0.0;
        for (int q = 0; q < NW; ++q) s += sh.part[q][r];
        sh.grad[r] = s + 2.0 * a.lam2 * vec[r];
    }
    __syncthreads();
}

__global__ __launch_bounds__(NT) void k_reopt(ReoptArgs a) {
    __shared__ ReoptShared sh;
    const int b = blockIdx.x, k = a.k, p = a.p;
    if (threadIdx.x == 0) {
        int ks = 0;
        for (int r = 0; r < k; ++r) {
            const int j = a.support[(size_t)b * k + r];
            if (j >= 0) sh.S[ks++] = j;
        }
        sh.ks = ks;
    }
    __syncthreads();
    const int ks = sh.ks;
    const double M = a.M;
    for (int t = threadIdx.x; t < ks * ks; t += NT) {
        const int r = t / ks, q = t % ks;
        double g = a.gram[(size_t)sh.S[r] * p + sh.S[q]];
        if (a.kind == kLSQ && r == q) g += a.lam2;
        sh.A[r * kMaxK + q] = g;
    }
    for (int r = threadIdx.x; r < ks; r += NT) {
        sh.c[r] = a.Xty[sh.S[r]];
        const size_t bj = (size_t)b * p + sh.S[r];
        const double w = a.b_is_f64 ? static_cast<const double*>(a.B)[bj] : (double)static_cast<const float*>(a.B)[bj];
        sh.bcur[r] = sh.bold[r] = fmin(M, fmax(-M, w));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double gmax = 0.0;                             // Gershgorin bound of the Gram block
        for (int r = 0; r < ks; ++r) {
            double s = 0.0;
            for (int q = 0; q < ks; ++q) s += fabs(sh.A[r * kMaxK + q]);
            gmax = fmax(gmax, s);
        }
        sh.L = a.kind == kLSQ ? 2.0 * gmax : 0.25 * gmax + 2.0 * a.lam2;
        if (!(sh.L > 0.0)) sh.L = 1.0;
    }
    __syncthreads();
    const double L = sh.L;
    if (ks > 0) {
        gradient(a, sh, sh.bcur);
        double g0 = 0.0;
        for (int r = 0; r < ks; ++r) g0 += sh.grad[r] * sh.grad[r];
        const double stop = a.tol * fmax(1.0, sqrt(g0));
        double t = 1.0;
        for (int it = 0; it < a.max_iter; ++it) {
            const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            const double coef = (t - 1.0) / tn;
            for (int r = threadIdx.x; r < ks; r += NT) sh.v[r] = sh.bcur[r] + coef * (sh.bcur[r] - sh.bold[r]);
            __syncthreads();
            gradient(a, sh, sh.v);
            for (int r = threadIdx.x; r < ks; r += NT) sh.bnew[r] = fmin(M, fmax(-M, sh.v[r] - sh.grad[r] / L));
            __syncthreads();
            double dot = 0.0;
            for (int r = 0; r < ks; ++r) dot += (sh.v[r] - sh.bnew[r]) * (sh.bnew[r] - sh.bcur[r]);
            t = dot > 0.0 ? 1.0 : tn;
            __syncthreads();
            for (int r = threadIdx.x; r < ks; r += NT) { sh.bold[r] = sh.bcur[r]; sh.bcur[r] = sh.bnew[r]; }
            __syncthreads();
            if ((it & 7) == 7) {                        // gradient-mapping test
                gradient(a, sh, sh.bcur);
                double gm = 0.0;
                for (int r = 0; r < ks; ++r) {
                    const double d = sh.bcur[r] - fmin(M, fmax(-M, sh.bcur[r] - sh.grad[r] / L));
                    gm += d * d;
                }
                __syncthreads();
                if (L * sqrt(gm) <= stop) break;
            }
        }
    }
    // exact objective: sum_i l((X_S b)_i, y_i) + lambda2 ||b||^2
    double acc[1] = {0.0};
    for (int i = threadIdx.x; i < a.n; i += NT) {
        double s = 0.0;
        for (int r = 0; r < ks; ++r) s += a.Xt[(size_t)sh.S[r] * a.n + i] * sh.bcur[r];
        acc[0] += loss64(s, a.y[i], a.kind);
    }
    block_sum<NT, 1, double>(acc, sh.red);
    if (threadIdx.x == 0) {
        double rid = 0.0;
        for (int r = 0; r < ks; ++r) rid += sh.bcur[r] * sh.bcur[r];
        a.ub[b] = acc[0] + a.lam2 * rid;
    }
    for (int r = threadIdx.x; r < k; r += NT) a.beta_re[(size_t)b * k + r] = r < ks ? sh.bcur[r] : 0.0;
}

}  // namespace

void reopt_launch(cudaStream_t s, const ReoptArgs& a) {
    if (a.m <= 0) return;
    k_reopt<<<a.m, NT, 0, s>>>(a);
}

}  // namespace kglm
