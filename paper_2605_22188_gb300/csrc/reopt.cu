// Re-optimization on the rounded support of each node (§4.3):
//   v(S) = min { F(X_S b) + lambda2 ||b||^2 : ||b||_inf <= M },
// warm-started from the node's relaxed beta on S: for the logistic loss one
// CTA per node; for least squares one warp per node on the Gram block
// (k_reopt_lsq_warp below).
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
// optimum the FISTA re-optimization reaches, or once an accepted Newton step
// predicts a decrease below the working precision's resolution of f (for a
// Newton step the predicted decrease g.d is twice the model's f - f*).  In
// the reduced-precision modes the logistic steps run in FP32: v(S) is flat at
// its minimizer, so the FP64 objective at an FP32-accurate minimizer is within
// O(eps32) relative of the minimum.
//
// Least squares uses the Gram block (X^T X)_SS and (X^T y)_S.  The logistic
// loss, gradient and Hessian are the gather-and-reduce passes of §4.3 over the
// n samples: chunks of X_S are staged in shared memory (one sample per
// thread), and H = X_S^T diag(w) X_S is accumulated in 4 x 4 register blocks
// on and above the diagonal, each block's samples split over a power-of-two
// group of lanes that is summed by shuffles.  Every line-search trial is a
// full evaluation (f, g, H), so an accepted step needs no further pass.  The
// returned v(S) is recomputed in a final pass over the samples: FP64 in the
// FP64 mode; in the others an FP64 predictor with the logistic loss and its
// rigorous rounding margin in FP32 (rounded upward), an upper bound of v(S).
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "engine.h"

namespace kglm {

namespace {

constexpr int NT = 256;

// Hessian block map: nb = ceil(ks / 4) block rows, nbp = nb (nb + 1) / 2 blocks
// on and above the diagonal, ss lanes (a power of two <= 32) per block.
struct PairMap {
    int nb, nbp, ss;
};
__host__ __device__ inline PairMap pair_map(int ks) {
    PairMap pm;
    pm.nb = (ks + 3) / 4;
    pm.nbp = pm.nb * (pm.nb + 1) / 2;
    pm.ss = 1;
    while (pm.ss < 32 && 2 * pm.ss * pm.nbp <= NT) pm.ss *= 2;   // largest power of two with ss * nbp <= NT
    return pm;
}

// Row stride (elements) of the staged sample-major X_S chunk: 4 nb columns
// plus padding that makes the number of 16-byte segments per row odd, so that
// eight consecutive rows read through 16-byte loads fall in distinct banks.
__host__ __device__ inline int xs_stride(int k, int esize) {
    const int nb = (k + 3) / 4;
    if (esize == 4) return nb % 2 ? 4 * nb : 4 * nb + 4;
    return 4 * nb + 2;
}
// Samples per staged chunk: about 40 KB of X_S, a multiple of 32 in [32, 1024].
__host__ __device__ inline int xs_chunk(int k, int esize) {
    int ch = 40960 / (xs_stride(k, esize) * esize) / 32 * 32;
    return ch < 32 ? 32 : (ch > 1024 ? 1024 : ch);
}

struct RS {
    int S[kMaxK];
    int fidx[kMaxK];
    double b[kMaxK], bn[kMaxK], d[kMaxK], c[kMaxK];
    double g[2][kMaxK];
    double vt[kMaxK];        // evaluation point in the working precision
    double red[NT / 32];
    double f[2], alpha, gnorm0;
    int ks, done, accept, cur;
};

// Dynamic shared memory: H[2][k*k] (FP64), the Cholesky factor L[k*k] and
// right-hand side z[k] (working precision), the X_S chunk Xs[ch * stride] and
// (w, d) per staged sample.
template <typename TI>
struct Dyn {
    double* H[2];
    TI* L;
    TI* z;
    TI* Xs;
    TI* wd;
    int ch, xs;
};

// (least squares never touches the X_S chunk: with_xs = false leaves it out)
template <typename TI>
__host__ __device__ inline size_t dyn_bytes(int k, bool with_xs) {
    const int es = (int)sizeof(TI);
    const int ch = xs_chunk(k, es), xs = xs_stride(k, es);
    size_t b = sizeof(double) * 2 * (size_t)k * k;
    b += (size_t)es * ((size_t)k * k + k);
    b = (b + 15) / 16 * 16;
    if (with_xs) b += (size_t)es * ((size_t)ch * xs + 2 * (size_t)ch);
    return b;
}

template <typename TI>
__device__ Dyn<TI> carve(unsigned char* base, int k) {
    const int es = (int)sizeof(TI);
    Dyn<TI> d;
    d.ch = xs_chunk(k, es);
    d.xs = xs_stride(k, es);
    d.H[0] = reinterpret_cast<double*>(base);
    d.H[1] = d.H[0] + (size_t)k * k;
    d.L = reinterpret_cast<TI*>(d.H[1] + (size_t)k * k);
    d.z = d.L + (size_t)k * k;
    size_t off = sizeof(double) * 2 * (size_t)k * k + (size_t)es * ((size_t)k * k + k);
    off = (off + 15) / 16 * 16;
    d.Xs = reinterpret_cast<TI*>(base + off);
    d.wd = d.Xs + (size_t)d.ch * d.xs;
    return d;
}

// Sum over the CTA, returned in thread 0 (the only reader); the other threads
// skip the final FP64 additions.  Same order as block_sum.
__device__ double block_total(double v, double* red) {
    constexpr int NW = NT / 32;
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NW; ++w) s += red[w];
    return s;
}

__device__ __forceinline__ float softplus_t(float t) { return t > 0.f ? t + log1pf(expf(-t)) : log1pf(expf(t)); }
__device__ __forceinline__ double softplus_t(double t) { return softplus(t); }
__device__ __forceinline__ float exp_t(float t) { return expf(t); }
__device__ __forceinline__ double exp_t(double t) { return exp(t); }
__device__ __forceinline__ float sqrt_t(float t) { return sqrtf(t); }
__device__ __forceinline__ double sqrt_t(double t) { return sqrt(t); }

// 4 consecutive elements from / to 16-byte aligned shared memory.
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
    const double2 q0 = *reinterpret_cast<const double2*>(p);
    const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
    v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}
__device__ __forceinline__ void st4(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&v)[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ld2(const float* p, float& a, float& b) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    a = q.x; b = q.y;
}
__device__ __forceinline__ void ld2(const double* p, double& a, double& b) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    a = q.x; b = q.y;
}
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }
__device__ __forceinline__ void st2(double* p, double a, double b) { *reinterpret_cast<double2*>(p) = make_double2(a, b); }

// Full evaluation at vec: f into sh.f[buf], g into sh.g[buf], H into dy.H[buf]
// (least squares: f up to the constant y^T y).
template <typename TI>
__device__ void evaluate(const ReoptArgs& a, RS& sh, const Dyn<TI>& dy, const double* vec, int buf) {
    const int ks = sh.ks, k = a.k, tid = threadIdx.x;
    double* H = dy.H[buf];
    double* g = sh.g[buf];
    if (a.kind == kLSQ) {
        // f = b^T (G + lambda2 I) b - 2 c^T b ; g = 2 ((G + lambda2 I) b - c) ; H = 2 (G + lambda2 I)
        double part = 0.0;
        for (int r = tid; r < ks; r += NT) {
            double s = 0.0;
            for (int q = 0; q < ks; ++q) s += a.gram[(size_t)sh.S[r] * a.p + sh.S[q]] * vec[q];
            s += a.lam2 * vec[r];
            part += vec[r] * s - 2.0 * sh.c[r] * vec[r];
            g[r] = 2.0 * (s - sh.c[r]);
        }
        for (int t = tid; t < ks * ks; t += NT) {
            const int r = t / ks, q = t % ks;
            H[r * k + q] = 2.0 * (a.gram[(size_t)sh.S[r] * a.p + sh.S[q]] + (r == q ? a.lam2 : 0.0));
        }
        const double f = block_total(part, sh.red);
        if (tid == 0) sh.f[buf] = f;
        __syncthreads();
        return;
    }
    const TI* Xt = static_cast<const TI*>(sizeof(TI) == 8 ? (const void*)a.Xt : (const void*)a.Xt32);
    const TI* yv = static_cast<const TI*>(sizeof(TI) == 8 ? (const void*)a.y : (const void*)a.y32);
    TI* vt = reinterpret_cast<TI*>(sh.vt);
    for (int r = tid; r < 4 * ((ks + 3) / 4); r += NT) vt[r] = r < ks ? (TI)vec[r] : TI(0);
    __syncthreads();
    const PairMap pm = pair_map(ks);
    const int bp = tid / pm.ss, sl = tid % pm.ss;
    int R = 0, Q = 0;
    if (bp < pm.nbp) {                       // block (R, Q), R <= Q, row-major over the upper triangle
        int t = bp;
        while (t >= pm.nb - R) { t -= pm.nb - R; ++R; }
        Q = R + t;
    }
    TI acc[16], gacc[4];
#pragma unroll
    for (int o = 0; o < 16; ++o) acc[o] = TI(0);
#pragma unroll
    for (int o = 0; o < 4; ++o) gacc[o] = TI(0);
    TI floss = TI(0);
    const int CH = dy.ch, XS = dy.xs;
    for (int i0 = 0; i0 < a.n; i0 += CH) {
        const int cn = min(CH, a.n - i0);
        // stage: one sample per thread; s = x_S . vec, loss, w = sigma (1 - sigma), d = dl/ds
        for (int t = tid; t < cn; t += NT) {
            const int i = i0 + t;
            TI s = TI(0);
            for (int r4 = 0; r4 < pm.nb; ++r4) {
                TI x[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int r = 4 * r4 + e;
                    x[e] = r < ks ? Xt[(size_t)sh.S[r] * a.n + i] : TI(0);
                    s += x[e] * vt[r];
                }
                st4(dy.Xs + (size_t)t * XS + 4 * r4, x);
            }
            const TI yi = yv[i];
            floss += softplus_t(-yi * s);
            const TI sg = TI(1) / (TI(1) + exp_t(yi * s));   // sigma(-y s)
            st2(dy.wd + 2 * t, sg * (TI(1) - sg), -yi * sg);
        }
        __syncthreads();
        if (bp < pm.nbp) {
            const TI* xr_base = dy.Xs + 4 * R;
            const TI* xq_base = dy.Xs + 4 * Q;
            if (R == Q) {
                for (int t = sl; t < cn; t += pm.ss) {
                    TI xr[4], w, dd;
                    ld4(xr_base + (size_t)t * XS, xr);
                    ld2(dy.wd + 2 * t, w, dd);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const TI xw = xr[e] * w;
                        gacc[e] += xr[e] * dd;
#pragma unroll
                        for (int f = 0; f < 4; ++f) acc[e * 4 + f] += xw * xr[f];
                    }
                }
            } else {
                for (int t = sl; t < cn; t += pm.ss) {
                    TI xr[4], xq[4], w, dd;
                    ld4(xr_base + (size_t)t * XS, xr);
                    ld4(xq_base + (size_t)t * XS, xq);
                    ld2(dy.wd + 2 * t, w, dd);
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const TI xw = xr[e] * w;
#pragma unroll
                        for (int f = 0; f < 4; ++f) acc[e * 4 + f] += xw * xq[f];
                    }
                }
            }
        }
        __syncthreads();
    }
    // sum each block over its ss lanes (aligned power-of-two lane groups)
    for (int o = pm.ss / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
#pragma unroll
        for (int e = 0; e < 4; ++e) gacc[e] += __shfl_xor_sync(0xffffffffu, gacc[e], o);
    }
    if (bp < pm.nbp && sl == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = 4 * R + e;
            if (r >= ks) continue;
            if (R == Q) g[r] = (double)gacc[e] + 2.0 * a.lam2 * vec[r];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const int q = 4 * Q + f;
                if (q >= ks || (R == Q && f < e)) continue;
                const double h = (double)acc[e * 4 + f] + (r == q ? 2.0 * a.lam2 : 0.0);
                H[r * k + q] = h;
                H[q * k + r] = h;
            }
        }
    }
    const double fl = block_total((double)floss, sh.red);
    if (tid == 0) {                // the ridge term once (FP64 is the slow pipe), same sum as before
        double ridge = 0.0;
        for (int r = 0; r < ks; ++r) ridge += vec[r] * vec[r];
        sh.f[buf] = fl + a.lam2 * ridge;
    }
    __syncthreads();
}

// Newton direction on the free set (warp 0): the projected-gradient test,
// the held set, then d_F = -H_FF^{-1} g_F by a right-looking Cholesky
// factorization in the working precision, lane l owning the factor rows
// l, l + 32.  Sets sh.done when the projected gradient is below tolerance.
template <typename TI>
__device__ void newton_direction(RS& sh, const Dyn<TI>& dy, int k, double M, double tol) {
    const int lane = threadIdx.x & 31, ks = sh.ks, cur = sh.cur;
    const double* H = dy.H[cur];
    const double* g = sh.g[cur];
    double pg = 0.0;
    for (int r = lane; r < ks; r += 32) {
        const double t = sh.b[r] - fmin(M, fmax(-M, sh.b[r] - g[r]));
        pg += t * t;
    }
    pg = sqrt(warp_sum(pg));
    if (pg <= tol * sh.gnorm0) {
        if (lane == 0) sh.done = 1;
        return;
    }
    const double eps = fmin(1e-3 * M, pg);
    int nf = 0;
    for (int base = 0; base < ks; base += 32) {
        const int r = base + lane;
        bool fr = false;
        if (r < ks) {
            const bool held = (sh.b[r] <= -M + eps && g[r] > 0.0) || (sh.b[r] >= M - eps && g[r] < 0.0);
            fr = !held;
            sh.d[r] = 0.0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, fr);
        if (fr) sh.fidx[nf + __popc(bal & ((1u << lane) - 1u))] = r;
        nf += __popc(bal);
    }
    __syncwarp();
    TI* L = dy.L;
    TI* z = dy.z;
    for (int i = lane; i < nf; i += 32) {
        const int ri = sh.fidx[i];
        for (int j = 0; j <= i; ++j) L[i * k + j] = (TI)H[ri * k + sh.fidx[j]];
        z[i] = -(TI)g[ri];
    }
    __syncwarp();
    for (int j = 0; j < nf; ++j) {
        // H_FF is positive definite (>= 2 lambda2 I); a pivot lost to rounding is floored
        const TI floor_j = TI(1e-7) * (TI)H[sh.fidx[j] * k + sh.fidx[j]];
        const TI piv = L[j * k + j];
        const TI dj = sqrt_t(piv > floor_j ? piv : floor_j);
        __syncwarp();
        for (int i = lane; i < nf; i += 32) {
            if (i == j) L[j * k + j] = dj;
            else if (i > j) L[i * k + j] /= dj;
        }
        __syncwarp();
        for (int i = lane; i < nf; i += 32) {
            if (i <= j) continue;
            const TI lij = L[i * k + j];
            for (int q = j + 1; q <= i; ++q) L[i * k + q] -= lij * L[q * k + j];
        }
        __syncwarp();
    }
    for (int j = 0; j < nf; ++j) {            // L y = -g_F
        if (lane == (j & 31)) z[j] /= L[j * k + j];
        __syncwarp();
        const TI zj = z[j];
        for (int i = lane; i < nf; i += 32)
            if (i > j) z[i] -= L[i * k + j] * zj;
        __syncwarp();
    }
    for (int j = nf - 1; j >= 0; --j) {       // L^T d = y
        if (lane == (j & 31)) z[j] /= L[j * k + j];
        __syncwarp();
        const TI zj = z[j];
        for (int i = lane; i < nf; i += 32)
            if (i < j) z[i] -= L[j * k + i] * zj;
        __syncwarp();
    }
    for (int i = lane; i < nf; i += 32) sh.d[sh.fidx[i]] = (double)z[i];
    if (lane == 0) sh.alpha = 1.0;
}

template <typename TI>
__global__ __launch_bounds__(NT, sizeof(TI) == 4 ? 4 : 1) void k_reopt(ReoptArgs a) {
    // stopping level of the working precision: the predicted decrease below
    // which f can neither check Armijo nor improve
    const double tol = a.tol;
    const double tiny_rel = sizeof(TI) == 8 ? 1e-14 : 3e-7;
    __shared__ RS sh;
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    const int k = a.k, p = a.p, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const Dyn<TI> dy = carve<TI>(dyn_raw, k);
    const double M = a.M;
    if (tid == 0) {
        int ks = 0;
        for (int r = 0; r < k; ++r) {
            const int j = a.support[(size_t)b * k + r];
            if (j >= 0 && kglm_check(j < a.p, a.chk, kChkReopt)) sh.S[ks++] = j;
        }
        sh.ks = ks;
        sh.done = 0;
        sh.cur = 0;
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
        evaluate<TI>(a, sh, dy, sh.b, 0);
        if (tid < 32) {
            double g2 = 0.0;
            for (int r = lane; r < ks; r += 32) g2 += sh.g[0][r] * sh.g[0][r];
            g2 = warp_sum(g2);
            if (lane == 0) sh.gnorm0 = fmax(1.0, sqrt(g2));
        }
        __syncthreads();
        for (int it = 0; it < a.max_iter; ++it) {
            if (tid < 32) newton_direction<TI>(sh, dy, k, M, tol);
            __syncthreads();
            if (sh.done) break;
            const int cur = sh.cur, nxt = 1 - cur;
            // Armijo backtracking along the projection arc; every trial is a full evaluation,
            // except a first trial whose predicted decrease is below the working precision's
            // resolution of f: it is accepted and ends the solve whatever f there is (the
            // test below), so its evaluation (f, g and H over the samples) is skipped
            bool moved = false;
            for (int ls = 0; ls < 40; ++ls) {
                for (int r = tid; r < ks; r += NT) sh.bn[r] = fmin(M, fmax(-M, sh.b[r] + sh.alpha * sh.d[r]));
                __syncthreads();
                if (ls == 0) {
                    if (tid < 32) {
                        double dec = 0.0;
                        for (int r = lane; r < ks; r += 32) dec += sh.g[cur][r] * (sh.bn[r] - sh.b[r]);
                        dec = warp_sum(dec);
                        if (lane == 0) {
                            const bool tiny = fabs(dec) <= tiny_rel * (1.0 + fabs(sh.f[cur]));
                            sh.accept = tiny ? 1 : 0;
                            if (tiny) sh.done = 1;
                        }
                    }
                    __syncthreads();
                    if (sh.done) { moved = true; break; }
                }
                evaluate<TI>(a, sh, dy, sh.bn, nxt);
                if (tid < 32) {
                    double dec = 0.0, step = 0.0;
                    for (int r = lane; r < ks; r += 32) {
                        dec += sh.g[cur][r] * (sh.bn[r] - sh.b[r]);
                        step = fmax(step, fabs(sh.bn[r] - sh.b[r]));
                    }
                    dec = warp_sum(dec);
                    step = warp_max(step);
                    if (lane == 0) {
                        // a predicted decrease below the rounding level of f cannot be checked:
                        // take the step (Newton is then in its quadratic region)
                        const bool tiny = fabs(dec) <= tiny_rel * (1.0 + fabs(sh.f[cur]));
                        sh.accept = (sh.f[nxt] <= sh.f[cur] + 1e-4 * dec || tiny) ? 1 : (step <= 1e-16 * M ? 2 : 0);
                        // converged: the full step's predicted decrease is below resolution
                        if (sh.accept == 1 && ((tiny && ls == 0) || step <= 1e-15 * M)) sh.done = 1;
                        if (!sh.accept) sh.alpha *= 0.5;
                    }
                }
                __syncthreads();
                if (sh.accept) { moved = (sh.accept == 1); break; }
            }
            if (!moved) break;                                   // no progress possible
            for (int r = tid; r < ks; r += NT) sh.b[r] = sh.bn[r];
            __syncthreads();
            if (tid == 0) sh.cur = nxt;
            __syncthreads();
            if (sh.done) break;
        }
    }
    // objective of the returned coefficients b: sum_i l((X_S b)_i, y_i) + lambda2 ||b||^2,
    // the predictor in FP64; the logistic loss in the reduced-precision modes
    // as an FP32 evaluation plus a margin that makes the sum an upper bound.
    // (i) t = y s rounded to FP32 moves t by <= 2^-24 |t| (< 1 for |t| < 2^24),
    // and |l'(xi)| = 1 / (1 + e^xi) <= min(1, e^(1 - tf)) on that interval:
    // margin 2^-23 |t| min(1, e^(1 - tf) (1 + 2^-20)) (expf within 2 ulp).
    // (ii) expf (2 ulp) and log1pf (1 ulp), documented maxima, and the final
    // addition give l~ within 2^-22 + 2^-23 + 2^-24 < 2^-21 relative of l(tf)
    // [the relative error of E passes to log1p(E) damped, since
    // d log1p(E)/dE * E <= log1p(E)]: margin 2^-21 l~ + 2^-125 per sample.
    // The margin and l~ + margin are formed in FP32 rounded upward (|t| <=
    // |tf| / (1 - 2^-24), so 2^-23 |t| <= 2^-23 |tf| (1 + 2^-22)); only the
    // predictor and the running sum take FP64 operations, the slow pipe here.
    double part = 0.0;
    const bool fast = sizeof(TI) == 4 && a.kind == kLOGISTIC;
    for (int i = tid; i < a.n; i += NT) {
        double s = 0.0;
        for (int r = 0; r < ks; ++r) s += a.Xt[(size_t)sh.S[r] * a.n + i] * sh.b[r];
        if (fast) {
            const double t = a.y[i] * s;
            const float tf = (float)t;
            const float l = fmaxf(-tf, 0.f) + log1pf(expf(-fabsf(tf)));
            const float slope = tf > 1.f ? fminf(1.f, __fmul_ru(expf(1.f - tf), 1.f + 0x1p-20f)) : 1.f;
            const float m1 = __fmul_ru(__fmul_ru(fabsf(tf), 0x1p-23f * (1.f + 0x1p-22f)), slope);
            const float mg = __fadd_ru(__fadd_ru(m1, l * 0x1p-21f), 0x1p-125f);
            part += (double)__fadd_ru(l, mg);
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

// Least squares, one warp per node.  The whole problem lives on the Gram block:
//   f(b) = b^T (G_SS + lambda2 I) b - 2 c^T b,  c = (X^T y)_S,  g = 2 ((G_SS + lambda2 I) b - c),
// and v(S) = y^T y + f(b*), so no pass over the n samples is needed; the
// projected Newton iteration of k_reopt (held set, Newton step on the free set
// by Cholesky, Armijo backtracking along the projection arc, the same stopping
// tests) runs in FP64 inside one warp, without CTA barriers, several nodes per
// CTA.  Per-warp shared memory: A = G_SS + lambda2 I and the factor L (k x k
// FP64 each) and a few k-vectors.
struct WarpLsq {
    double c[kMaxK], b[kMaxK], bn[kMaxK], d[kMaxK], g[2][kMaxK];
    int S[kMaxK], fidx[kMaxK];
};
__host__ __device__ inline size_t lsq_warp_bytes(int k) {
    return (sizeof(WarpLsq) + 2 * sizeof(double) * (size_t)k * k + 15) / 16 * 16;
}

// f and g at vec (k-vector in shared memory): rows r = lane, lane + 32.
__device__ __forceinline__ double lsq_eval(const double* A, const WarpLsq& w, int k, int ks, const double* vec,
                                           double* g, int lane) {
    double part = 0.0;
    for (int r = lane; r < ks; r += 32) {
        double s = 0.0;
        for (int q = 0; q < ks; ++q) s += A[r * k + q] * vec[q];
        part += vec[r] * s - 2.0 * w.c[r] * vec[r];
        g[r] = 2.0 * (s - w.c[r]);
    }
    __syncwarp();
    return warp_sum(part);
}

__global__ __launch_bounds__(256) void k_reopt_lsq_warp(ReoptArgs a) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    const int b = blockIdx.x * wpc + warp;
    if (b >= a.m) return;
    const int k = a.k, p = a.p;
    const double M = a.M;
    unsigned char* base = dyn_raw + (size_t)warp * lsq_warp_bytes(k);
    WarpLsq& w = *reinterpret_cast<WarpLsq*>(base);
    double* A = reinterpret_cast<double*>(base + sizeof(WarpLsq));
    double* L = A + (size_t)k * k;
    // the support (ascending, -1 padded) and the warm start clipped to the box
    int ks = 0;
    for (int r0 = 0; r0 < k; r0 += 32) {
        const int r = r0 + lane;
        const int j0 = r < k ? a.support[(size_t)b * k + r] : -1;
        const int j = (j0 < 0 || kglm_check(j0 < a.p, a.chk, kChkReopt)) ? j0 : -1;
        const unsigned bal = __ballot_sync(0xffffffffu, j >= 0);
        if (j >= 0) w.S[ks + __popc(bal & ((1u << lane) - 1u))] = j;
        ks += __popc(bal);
    }
    __syncwarp();
    for (int r = lane; r < ks; r += 32) {
        const int j = w.S[r];
        w.c[r] = a.Xty[j];
        const size_t bj = (size_t)b * p + j;
        const double v = a.b_is_f64 ? static_cast<const double*>(a.B)[bj] : (double)static_cast<const float*>(a.B)[bj];
        w.b[r] = fmin(M, fmax(-M, v));
    }
    __syncwarp();
    for (int t = lane; t < ks * ks; t += 32) {
        const int r = t / ks, q = t % ks;
        A[r * k + q] = a.gram[(size_t)w.S[r] * p + w.S[q]] + (r == q ? a.lam2 : 0.0);
    }
    __syncwarp();
    double fcur = 0.0;
    int cur = 0;
    if (ks > 0) {
        fcur = lsq_eval(A, w, k, ks, w.b, w.g[0], lane);
        double g2 = 0.0;
        for (int r = lane; r < ks; r += 32) g2 += w.g[0][r] * w.g[0][r];
        const double gnorm0 = fmax(1.0, sqrt(warp_sum(g2)));
        for (int it = 0; it < a.max_iter; ++it) {
            const double* g = w.g[cur];
            double pg = 0.0;
            for (int r = lane; r < ks; r += 32) {
                const double t = w.b[r] - fmin(M, fmax(-M, w.b[r] - g[r]));
                pg += t * t;
            }
            pg = sqrt(warp_sum(pg));
            if (pg <= a.tol * gnorm0) break;
            // held set (bound reached, gradient outward), Newton step on the rest
            const double eps = fmin(1e-3 * M, pg);
            int nf = 0;
            for (int r0 = 0; r0 < ks; r0 += 32) {
                const int r = r0 + lane;
                bool fr = false;
                if (r < ks) {
                    const bool held = (w.b[r] <= -M + eps && g[r] > 0.0) || (w.b[r] >= M - eps && g[r] < 0.0);
                    fr = !held;
                    w.d[r] = 0.0;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, fr);
                if (fr) w.fidx[nf + __popc(bal & ((1u << lane) - 1u))] = r;
                nf += __popc(bal);
            }
            __syncwarp();
            // L L^T = 2 A_FF (lower triangle), then 2 A_FF d_F = -g_F
            for (int i = lane; i < nf; i += 32) {
                const int ri = w.fidx[i];
                for (int j = 0; j <= i; ++j) L[i * k + j] = 2.0 * A[ri * k + w.fidx[j]];
                w.bn[i] = -g[ri];               // right-hand side, then the solution
            }
            __syncwarp();
            for (int j = 0; j < nf; ++j) {
                // A_FF is positive definite (>= lambda2 I); a pivot lost to rounding is floored
                const double floor_j = 1e-14 * 2.0 * A[w.fidx[j] * k + w.fidx[j]];
                const double piv = L[j * k + j];
                const double dj = sqrt(piv > floor_j ? piv : floor_j);
                __syncwarp();
                for (int i = lane; i < nf; i += 32) {
                    if (i == j) L[j * k + j] = dj;
                    else if (i > j) L[i * k + j] /= dj;
                }
                __syncwarp();
                for (int i = lane; i < nf; i += 32) {
                    if (i <= j) continue;
                    const double lij = L[i * k + j];
                    for (int q = j + 1; q <= i; ++q) L[i * k + q] -= lij * L[q * k + j];
                }
                __syncwarp();
            }
            for (int j = 0; j < nf; ++j) {                // L y = -g_F
                if (lane == (j & 31)) w.bn[j] /= L[j * k + j];
                __syncwarp();
                const double zj = w.bn[j];
                for (int i = lane; i < nf; i += 32)
                    if (i > j) w.bn[i] -= L[i * k + j] * zj;
                __syncwarp();
            }
            for (int j = nf - 1; j >= 0; --j) {           // L^T d = y
                if (lane == (j & 31)) w.bn[j] /= L[j * k + j];
                __syncwarp();
                const double zj = w.bn[j];
                for (int i = lane; i < nf; i += 32)
                    if (i < j) w.bn[i] -= L[j * k + i] * zj;
                __syncwarp();
            }
            for (int i = lane; i < nf; i += 32) w.d[w.fidx[i]] = w.bn[i];
            __syncwarp();
            // Armijo backtracking along the projection arc (every trial evaluates f and g)
            const int nxt = 1 - cur;
            double alpha = 1.0, fn = 0.0;
            int accept = 0;
            bool done = false;
            for (int ls = 0; ls < 40 && !accept; ++ls) {
                for (int r = lane; r < ks; r += 32) w.bn[r] = fmin(M, fmax(-M, w.b[r] + alpha * w.d[r]));
                __syncwarp();
                fn = lsq_eval(A, w, k, ks, w.bn, w.g[nxt], lane);
                double dec = 0.0, step = 0.0;
                for (int r = lane; r < ks; r += 32) {
                    dec += g[r] * (w.bn[r] - w.b[r]);
                    step = fmax(step, fabs(w.bn[r] - w.b[r]));
                }
                dec = warp_sum(dec);
                step = warp_max(step);
                // a predicted decrease below the rounding level of f cannot be checked:
                // take the step (Newton is then in its quadratic region)
                const bool tiny = fabs(dec) <= 1e-14 * (1.0 + fabs(fcur));
                accept = (fn <= fcur + 1e-4 * dec || tiny) ? 1 : (step <= 1e-16 * M ? 2 : 0);
                if (accept == 1 && ((tiny && ls == 0) || step <= 1e-15 * M)) done = true;
                if (!accept) alpha *= 0.5;
            }
            if (accept != 1) break;                       // no progress possible
            for (int r = lane; r < ks; r += 32) w.b[r] = w.bn[r];
            __syncwarp();
            fcur = fn;
            cur = nxt;
            if (done) break;
        }
    }
    if (lane == 0) a.ub[b] = a.yty + fcur;
    for (int r = lane; r < k; r += 32) a.beta_re[(size_t)b * k + r] = r < ks ? w.b[r] : 0.0;
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
    const size_t a = dyn_bytes<double>(k, true), b = dyn_bytes<float>(k, true);
    return a > b ? a : b;
}

// The dynamic shared memory opt-in of k_reopt<TI> is set to each launch's need
// and the launch is issued under the same lock.  (Without the lock, a
// concurrent context with a smaller k could lower the opt-in between another
// context's setting and its launch, which then failed with "too many resources
// requested".)
static std::mutex g_reopt_launch_mu;

int reopt_launch(cudaStream_t s, const ReoptArgs& a) {
    if (a.m <= 0) return 0;
    if (a.kind == kLSQ) {
        const size_t per = lsq_warp_bytes(a.k);
        const int wpc = (int)std::max<size_t>(1, std::min<size_t>(8, (96u << 10) / per));
        {
            static std::mutex mu;
            static bool opted = false;
            std::lock_guard<std::mutex> lock(mu);
            if (!opted) {
                if (cudaFuncSetAttribute(k_reopt_lsq_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         96 << 10) != cudaSuccess)
                    return -1;
                opted = true;
            }
        }
        k_reopt_lsq_warp<<<(a.m + wpc - 1) / wpc, 32 * wpc, wpc * per, s>>>(a);
        return 0;
    }
    const bool f32 = a.kind == kLOGISTIC && a.Xt32 != nullptr && a.y32 != nullptr;
    const size_t smem = f32 ? dyn_bytes<float>(a.k, true) : dyn_bytes<double>(a.k, a.kind == kLOGISTIC);
    // the opt-in covers static + dynamic shared memory above the 48 KB default
    std::lock_guard<std::mutex> lock(g_reopt_launch_mu);
    if (cudaFuncSetAttribute(f32 ? k_reopt<float> : k_reopt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return -1;
    if (f32) k_reopt<float><<<a.m, NT, smem, s>>>(a);
    else k_reopt<double><<<a.m, NT, smem, s>>>(a);
    return 0;
}

}  // namespace kglm
