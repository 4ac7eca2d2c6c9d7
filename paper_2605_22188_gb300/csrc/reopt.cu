// Re-optimization on the rounded support of each node (§4.3):
//   v(S) = min { F(X_S b) + lambda2 ||b||^2 : ||b||_inf <= M },
// one CTA per node, FP64, warm-started from the node's relaxed beta on S.
//
// §4.3 allows any proximal-gradient method whose prox is the projection onto
// [-M, M]; the problem has at most k variables, so this kernel takes
// projected Newton steps instead (Bertsekas, "Projected Newton methods for
// optimization problems with simple constraints", SIAM J. Control Optim.
// 1982): coordinates at a bound whose gradient points outward (within
// eps = min(eps0, ||b - P(b - g)||)) are held, the Newton system is solved on
// the others by Cholesky, and the step is backtracked along the projection
// arc P(b + alpha d) until the Armijo condition holds.  It stops when the
// projected gradient ||b - P(b - g)|| <= tol * max(1, ||g(b_0)||), the same
// optimum the FISTA re-optimization reaches.  In the reduced-precision modes
// the logistic steps run in FP32 (tolerance 2e-5): v(S) is flat at its
// minimizer, so the FP64 objective at an FP32-accurate minimizer is within
// O(tol^2) of the minimum.
//
// Least squares uses the Gram block (X^T X)_SS and (X^T y)_S; the logistic
// gradient and Hessian are the gather-and-reduce passes of §4.3 over the n
// samples (chunks of CH samples of X_S staged in shared memory).  The
// returned v(S) is recomputed exactly in a final pass over the samples.
#include "common.cuh"
#include "engine.h"

namespace kglm {

// Samples per staged chunk: as many as fit 24 KB of X_S, a multiple of 32, at most one per thread.
__host__ __device__ inline int reopt_chunk(int k) {
    int ch = (24576 / (8 * (k > 0 ? k : 1))) / 32 * 32;
    return ch < 32 ? 32 : (ch > 256 ? 256 : ch);
}
// Row stride of the staged X_S chunk: CH + 1 keeps the rows of a pair loop in different banks.
__host__ __device__ inline int reopt_stride(int k) { return reopt_chunk(k) + 1; }

namespace {

constexpr int NT = 256;
constexpr int MAXOWN = (kMaxK * (kMaxK + 1) / 2 + kMaxK + NT - 1) / NT;

struct RS {
    int S[kMaxK];
    double b[kMaxK], bn[kMaxK], g[kMaxK], d[kMaxK], c[kMaxK];
    int fr[kMaxK];
    double red[NT / 32];
    double f, fn, alpha, gnorm0;
    int ks, done, accept;
};

// Dynamic shared memory: H[k*k], Lc[k*k], Xs[k*ch], dv[ch], wv[ch] (ch samples per staged chunk).
struct Dyn {
    double *H, *Lc, *Xs, *dv, *wv;
    int ch;
};

__device__ double block_total(double v, double* red) {
    double a[1] = {v};
    block_sum<NT, 1, double>(a, red);
    return a[0];
}

__device__ __forceinline__ float softplusf(float t) { return t > 0.f ? t + log1pf(expf(-t)) : log1pf(expf(t)); }
__device__ __forceinline__ float softplus_t(float t) { return softplusf(t); }
__device__ __forceinline__ double softplus_t(double t) { return softplus(t); }
__device__ __forceinline__ float exp_t(float t) { return expf(t); }
__device__ __forceinline__ double exp_t(double t) { return exp(t); }

// f at vec (up to the constant y^T y for least squares); with `full`, also g and H at vec.
// The logistic passes run in TI (float in the reduced-precision modes, using
// the FP32 copy of X^T; double in the FP64 mode).
template <typename TI>
__device__ void evaluate(const ReoptArgs& a, RS& sh, Dyn& dy, const double* vec, bool full) {
    const int ks = sh.ks, k = a.k, tid = threadIdx.x;
    if (a.kind == kLSQ) {
        // f = b^T (G + lambda2 I) b - 2 c^T b ; g = 2 ((G + lambda2 I) b - c) ; H = 2 (G + lambda2 I)
        double part = 0.0;
        for (int r = tid; r < ks; r += NT) {
            double s = 0.0;
            for (int q = 0; q < ks; ++q) s += a.gram[(size_t)sh.S[r] * a.p + sh.S[q]] * vec[q];
            s += a.lam2 * vec[r];
            part += vec[r] * s - 2.0 * sh.c[r] * vec[r];
            if (full) sh.g[r] = 2.0 * (s - sh.c[r]);
        }
        if (full)
            for (int t = tid; t < ks * ks; t += NT) {
                const int r = t / ks, q = t % ks;
                dy.H[r * k + q] = 2.0 * (a.gram[(size_t)sh.S[r] * a.p + sh.S[q]] + (r == q ? a.lam2 : 0.0));
            }
        const double f = block_total(part, sh.red);
        if (tid == 0) { if (full) sh.f = f; else sh.fn = f; }
        __syncthreads();
        return;
    }
    const int npairs = ks * (ks + 1) / 2;
    const TI* Xt = static_cast<const TI*>(sizeof(TI) == 8 ? (const void*)a.Xt : (const void*)a.Xt32);
    const TI* yv = static_cast<const TI*>(sizeof(TI) == 8 ? (const void*)a.y : (const void*)a.y32);
    TI* Xs = reinterpret_cast<TI*>(dy.Xs);
    TI* dv = reinterpret_cast<TI*>(dy.dv);
    TI* wv = reinterpret_cast<TI*>(dy.wv);
    TI acc[MAXOWN];
#pragma unroll
    for (int o = 0; o < MAXOWN; ++o) acc[o] = TI(0);
    TI floss = TI(0);
    const int CH = dy.ch, XS = CH + 1;
    for (int i0 = 0; i0 < a.n; i0 += CH) {
        if (tid < CH) {
            const int i = i0 + tid;
            TI s = TI(0);
            if (i < a.n) {
                for (int r = 0; r < ks; ++r) {
                    const TI x = Xt[(size_t)sh.S[r] * a.n + i];
                    Xs[r * XS + tid] = x;
                    s += x * TI(vec[r]);
                }
                const TI yi = yv[i];
                floss += softplus_t(-yi * s);
                const TI sg = TI(1) / (TI(1) + exp_t(yi * s));   // sigma(-y s)
                dv[tid] = -yi * sg;
                wv[tid] = sg * (TI(1) - sg);
            } else {
                for (int r = 0; r < ks; ++r) Xs[r * XS + tid] = TI(0);
                dv[tid] = wv[tid] = TI(0);
            }
        }
        __syncthreads();
        if (full) {
#pragma unroll
            for (int o = 0; o < MAXOWN; ++o) {
                const int P = tid + o * NT;
                if (P < ks) {
                    TI s = TI(0);
                    for (int t = 0; t < CH; ++t) s += Xs[P * XS + t] * dv[t];
                    acc[o] += s;
                } else if (P < ks + npairs) {
                    int q = P - ks, r = 0;
                    while (q > r) { q -= r + 1; ++r; }          // pair (r, q), q <= r
                    TI s = TI(0);
                    for (int t = 0; t < CH; ++t) s += Xs[r * XS + t] * Xs[q * XS + t] * wv[t];
                    acc[o] += s;
                }
            }
        }
        __syncthreads();
    }
    double ridge = 0.0;
    for (int r = 0; r < ks; ++r) ridge += vec[r] * vec[r];
    const double f = block_total((double)floss, sh.red) + a.lam2 * ridge;
    if (full) {
#pragma unroll
        for (int o = 0; o < MAXOWN; ++o) {
            const int P = tid + o * NT;
            if (P < ks) {
                sh.g[P] = (double)acc[o] + 2.0 * a.lam2 * vec[P];
            } else if (P < ks + npairs) {
                int q = P - ks, r = 0;
                while (q > r) { q -= r + 1; ++r; }
                const double h = (double)acc[o] + (r == q ? 2.0 * a.lam2 : 0.0);
                dy.H[r * k + q] = h;
                dy.H[q * k + r] = h;
            }
        }
    }
    if (tid == 0) { if (full) sh.f = f; else sh.fn = f; }
    __syncthreads();
}

template <typename TI>
__global__ __launch_bounds__(NT) void k_reopt(ReoptArgs a) {
    // stopping levels of the working precision: projected-gradient tolerance,
    // and the predicted decrease below which f cannot check Armijo
    const double tol = sizeof(TI) == 8 ? a.tol : fmax(a.tol, 2e-5);
    const double tiny_rel = sizeof(TI) == 8 ? 1e-14 : 3e-7;
    __shared__ RS sh;
    extern __shared__ __align__(16) double dyn[];
    const int k = a.k, p = a.p, b = blockIdx.x, tid = threadIdx.x;
    const int CH = reopt_chunk(k), XS = reopt_stride(k);
    Dyn dy{dyn, dyn + k * k, dyn + 2 * k * k, dyn + 2 * k * k + k * XS, dyn + 2 * k * k + k * XS + CH, CH};
    const double M = a.M;
    if (tid == 0) {
        int ks = 0;
        for (int r = 0; r < k; ++r) {
            const int j = a.support[(size_t)b * k + r];
            if (j >= 0) sh.S[ks++] = j;
        }
        sh.ks = ks;
        sh.done = 0;
    }
    __syncthreads();
    const int ks = sh.ks;
    for (int r = tid; r < ks; r += NT) {
        sh.c[r] = a.Xty[sh.S[r]];
        const size_t bj = (size_t)b * p + sh.S[r];
        const double w = a.b_is_f64 ? static_cast<const double*>(a.B)[bj] : (double)static_cast<const float*>(a.B)[bj];
        sh.b[r] = fmin(M, fmax(-M, w));
    }
    __syncthreads();
    if (ks > 0) {
        evaluate<TI>(a, sh, dy, sh.b, true);
        if (tid == 0) {
            double g2 = 0.0;
            for (int r = 0; r < ks; ++r) g2 += sh.g[r] * sh.g[r];
            sh.gnorm0 = fmax(1.0, sqrt(g2));
        }
        __syncthreads();
        for (int it = 0; it < a.max_iter; ++it) {
            if (tid == 0) {
                double pg = 0.0;
                for (int r = 0; r < ks; ++r) {
                    const double t = sh.b[r] - fmin(M, fmax(-M, sh.b[r] - sh.g[r]));
                    pg += t * t;
                }
                pg = sqrt(pg);
                if (pg <= tol * sh.gnorm0) {
                    sh.done = 1;
                } else {
                    const double eps = fmin(1e-3 * M, pg);
                    int nf = 0;
                    for (int r = 0; r < ks; ++r) {
                        const bool held = (sh.b[r] <= -M + eps && sh.g[r] > 0.0) || (sh.b[r] >= M - eps && sh.g[r] < 0.0);
                        sh.fr[r] = held ? -1 : nf++;
                        sh.d[r] = 0.0;
                    }
                    // Cholesky of H_FF, then d_F = -H_FF^{-1} g_F
                    double* L = dy.Lc;
                    for (int r = 0, ir = 0; r < ks; ++r) {
                        if (sh.fr[r] < 0) continue;
                        for (int q = 0, iq = 0; q < ks; ++q) {
                            if (sh.fr[q] < 0) continue;
                            L[ir * k + iq] = dy.H[r * k + q];
                            ++iq;
                        }
                        ++ir;
                    }
                    for (int j = 0; j < nf; ++j) {
                        double s = L[j * k + j];
                        for (int t = 0; t < j; ++t) s -= L[j * k + t] * L[j * k + t];
                        s = s > 1e-300 ? sqrt(s) : 1e-150;
                        L[j * k + j] = s;
                        for (int i = j + 1; i < nf; ++i) {
                            double v = L[i * k + j];
                            for (int t = 0; t < j; ++t) v -= L[i * k + t] * L[j * k + t];
                            L[i * k + j] = v / s;
                        }
                    }
                    double z[kMaxK];
                    for (int r = 0, ir = 0; r < ks; ++r) {
                        if (sh.fr[r] < 0) continue;
                        double v = -sh.g[r];
                        for (int t = 0; t < ir; ++t) v -= L[ir * k + t] * z[t];
                        z[ir] = v / L[ir * k + ir];
                        ++ir;
                    }
                    for (int ir = nf - 1; ir >= 0; --ir) {
                        double v = z[ir];
                        for (int t = ir + 1; t < nf; ++t) v -= L[t * k + ir] * z[t];
                        z[ir] = v / L[ir * k + ir];
                    }
                    for (int r = 0; r < ks; ++r)
                        if (sh.fr[r] >= 0) sh.d[r] = z[sh.fr[r]];
                    sh.alpha = 1.0;
                }
            }
            __syncthreads();
            if (sh.done) break;
            // Armijo backtracking along the projection arc
            bool moved = false;
            for (int ls = 0; ls < 40; ++ls) {
                for (int r = tid; r < ks; r += NT) sh.bn[r] = fmin(M, fmax(-M, sh.b[r] + sh.alpha * sh.d[r]));
                __syncthreads();
                evaluate<TI>(a, sh, dy, sh.bn, false);
                if (tid == 0) {
                    double dec = 0.0, step = 0.0;
                    for (int r = 0; r < ks; ++r) {
                        dec += sh.g[r] * (sh.bn[r] - sh.b[r]);
                        step = fmax(step, fabs(sh.bn[r] - sh.b[r]));
                    }
                    // a predicted decrease below the rounding level of f cannot be checked:
                    // take the step (Newton is then in its quadratic region)
                    const bool tiny = fabs(dec) <= tiny_rel * (1.0 + fabs(sh.f));
                    sh.accept = (sh.fn <= sh.f + 1e-4 * dec || tiny) ? 1 : (step <= 1e-16 * M ? 2 : 0);
                    if (sh.accept == 1 && step <= 1e-15 * M) sh.done = 1;   // converged to FP64 resolution
                    if (!sh.accept) sh.alpha *= 0.5;
                }
                __syncthreads();
                if (sh.accept) { moved = (sh.accept == 1); break; }
            }
            if (!moved) break;                                   // no progress possible in FP64
            for (int r = tid; r < ks; r += NT) sh.b[r] = sh.bn[r];
            __syncthreads();
            if (sh.done) break;
            evaluate<TI>(a, sh, dy, sh.b, true);
        }
    }
    // objective of the returned coefficients b: sum_i l((X_S b)_i, y_i) + lambda2 ||b||^2,
    // the predictor in FP64; the logistic loss in the reduced-precision modes
    // as an FP32 evaluation plus a margin that makes the sum an upper bound:
    // t = y s rounded to FP32 moves the 1-Lipschitz loss by <= 2^-24 |t|;
    // expf (2 ulp) and log1pf (1 ulp, documented maxima) give <= 2^-21 relative
    // on log1p(e^-|t|) [d/dE log1p(E) * E <= log1p(E)], one more rounding for
    // the sum: margin 2^-23 |t| + 2^-20 l~ + 2^-125 per sample.
    double part = 0.0;
    const bool fast = sizeof(TI) == 4 && a.kind == kLOGISTIC;
    for (int i = tid; i < a.n; i += NT) {
        double s = 0.0;
        for (int r = 0; r < ks; ++r) s += a.Xt[(size_t)sh.S[r] * a.n + i] * sh.b[r];
        if (fast) {
            const double t = a.y[i] * s;
            const float tf = (float)t;
            const float l = fmaxf(-tf, 0.f) + log1pf(expf(-fabsf(tf)));
            part += (double)l + (ldexp(fabs(t), -23) + ldexp((double)l, -20) + 0x1p-125);
        } else {
            part += loss64(s, a.y[i], a.kind);
        }
    }
    const double tot = block_total(part, sh.red);
    if (tid == 0) {
        double rid = 0.0;
        for (int r = 0; r < ks; ++r) rid += sh.b[r] * sh.b[r];
        a.ub[b] = tot + a.lam2 * rid;
    }
    for (int r = tid; r < k; r += NT) a.beta_re[(size_t)b * k + r] = r < ks ? sh.b[r] : 0.0;
}

// FP64 objective F(X_S b) + lambda2 ||b||^2 of one coefficient vector (one CTA).
__global__ __launch_bounds__(NT) void k_objective64(const double* Xt, const double* y, int n, int kind,
                                                    double lam2, const int* S, const double* b, int ks,
                                                    double* out) {
    __shared__ double red[NT / 32];
    double part = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) {
        double s = 0.0;
        for (int r = 0; r < ks; ++r) s += Xt[(size_t)S[r] * n + i] * b[r];
        part += loss64(s, y[i], kind);
    }
    const double tot = block_total(part, red);
    if (threadIdx.x == 0) {
        double rid = 0.0;
        for (int r = 0; r < ks; ++r) rid += b[r] * b[r];
        *out = tot + lam2 * rid;
    }
}

}  // namespace

void objective64_launch(cudaStream_t s, const double* Xt, const double* y, int n, int kind, double lam2,
                        const int* S, const double* b, int ks, double* out) {
    k_objective64<<<1, NT, 0, s>>>(Xt, y, n, kind, lam2, S, b, ks, out);
}

size_t reopt_smem_bytes(int k) {
    const int ch = reopt_chunk(k);
    return sizeof(double) * (size_t)(2 * k * k + k * reopt_stride(k) + 2 * ch);
}

int reopt_launch(cudaStream_t s, const ReoptArgs& a) {
    if (a.m <= 0) return 0;
    const size_t smem = reopt_smem_bytes(a.k);
    const bool f32 = a.kind == kLOGISTIC && a.Xt32 != nullptr && a.y32 != nullptr;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(f32 ? k_reopt<float> : k_reopt<double>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return -1;
    }
    if (f32) k_reopt<float><<<a.m, NT, smem, s>>>(a);
    else k_reopt<double><<<a.m, NT, smem, s>>>(a);
    return 0;
}

}  // namespace kglm
