// The certificate product X^T zeta (§4.4 Eq. (batched_dual_candidate_matrix_form))
// of the reduced-precision modes, on the BF16 tensor cores by error-free
// splitting (Ozaki, Ogita, Oishi and Rump, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012; on tensor cores: Mukunoki,
// Ozaki, Ogita and Imamura, ICCS 2020).
//
// Column j of X is scaled by sigma_j = 2^e > max_i |X_ij| and the dual point
// of node b by tau_b = 2^f > max_i |zeta_ib| (exact).  A scaled value v in
// (-1, 1) is rounded to the fixed-point integer V = rint(v 2^62) (error at
// most 2^-63) and cut into s signed digits of beta bits from the top,
//   d_a = round(V / 2^(62 - beta a)),  V <- V - d_a 2^(62 - beta a),
// so v = sum_a d_a 2^(-beta a) + r with |d_1| <= 2^beta, |d_a| <= 2^(beta-1)
// (a >= 2) and |r| <= 2^(-beta s - 1) + 2^-63.  The digits are integers of at
// most 7 bits: exact in BF16, their products exact in FP32.  The digit pairs
// (a, c) of one level l = a + c share the weight 2^(-beta l), so each level
// is one product with its pairs concatenated along K:
//   P_l[b][j] = sum_{a + c = l} sum_i dz_c(i, b) dx_a(i, j).
// X's digits are stored a = 1 .. s along K and zeta's in reverse, so level l
// reads a prefix of X's row and a window of zeta's.  K is cut into jobs
// whose sum of |digit products| is at most 2^24: every FP32 accumulation
// of a job is an integer of at most 24 bits, exact whatever the order or
// rounding of the accumulator.  Levels 2 .. s + 1 are formed, and
//   Q~_bj = sigma_j tau_b sum_jobs 2^(-beta l) P_job[b][j]       (FP64)
// satisfies |Q~_bj - (X^T zeta)_jb| <= sigma_j tau_b n E with
//   E = 2 (2^(-beta s - 1) + 2^-63) + (2^(-beta s - 1) + 2^-63)^2
//       + sum_{l = s+2}^{2s} (2s - l + 1) 2^(2 beta - 2) 2^(-beta l)   (levels left out)
//       + 2^-44                                                      (FP64 combine)
// per unit of sigma_j tau_b and per sample.  The certificate then uses
// |Q~| + sigma tau n E, an entrywise upper bound of |X^T zeta|; H_M and the
// TopSum are increasing in |q|, so the bound remains a valid lower bound.
#include <math.h>

#include "common.cuh"
#include "engine.h"
#include "exact.cuh"

namespace kglm {
namespace {

constexpr int NT = 256;

// One CTA per row r of V (rows x n, row stride ldv): scale[r] = 2^e > max |V_r| (0 for a zero row),
// digits of V_r / 2^e into D row r (s segments of npad BF16 values, zero
// past n); segment a - 1 holds digit a, or segment s - a when reversed.
__global__ __launch_bounds__(NT) void k_digits(const double* V, int n, size_t ldv, int npad, int s, int beta,
                                               int reversed, __nv_bfloat16* D, double* scale) {
    __shared__ double red[NT / 32];
    const int r = blockIdx.x;
    const double* v = V + (size_t)r * ldv;
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += NT) mx = fmax(mx, fabs(v[i]));
    mx = block_max<NT, double>(mx, red);
    const int e = mx > 0.0 ? ilogb(mx) + 1 : 0;            // 2^e > mx
    if (threadIdx.x == 0) scale[r] = mx > 0.0 ? ldexp(1.0, e) : 0.0;   // a zero row is exact: no bound
    __nv_bfloat16* d = D + (size_t)r * s * npad;
    for (int i = threadIdx.x; i < npad; i += NT) {
        long long z = i < n ? llrint(ldexp(v[i], 62 - e)) : 0ll;     // |z| < 2^62
        for (int a = 1; a <= s; ++a) {
            const int sh = 62 - beta * a;
            const long long dg = (z + (1ll << (sh - 1))) >> sh;      // nearest, halves up
            z -= dg << sh;
            d[(size_t)(reversed ? s - a : a - 1) * npad + i] = __int2bfloat16_rn((int)dg);
        }
    }
}

struct Weights {
    double w[kTcMaxJobs];
};

// Q[b][j] and its bound from the job partials (kglm_xtz).
__global__ void k_exact_combine(int m, int p, const float* Qs, int nq, size_t stride,
                                const __grid_constant__ Weights W, const double* sigma, const double* tau,
                                double ebound, double* Q, double* E) {
    const size_t total = (size_t)m * p;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(idx / p), j = (int)(idx % p);
        double err;
        Q[idx] = exact_q(Qs, nq, stride, W.w, idx, sigma[j] * tau[b], ebound, &err);
        if (E) E[idx] = err;
    }
}

}  // namespace

void exact_digits(cudaStream_t s, const double* V, int rows, int n, size_t ldv, int npad, int nd, int beta,
                  int reversed, __nv_bfloat16* D, double* scale) {
    if (rows <= 0) return;
    k_digits<<<rows, NT, 0, s>>>(V, n, ldv, npad, nd, beta, reversed, D, scale);
}

void exact_combine(cudaStream_t s, int m, int p, const float* Qs, int nq, size_t stride, const double* w,
                   const double* sigma, const double* tau, double ebound, double* Q, double* E) {
    if (m <= 0 || nq > kTcMaxJobs) return;
    Weights W{};
    for (int t = 0; t < nq; ++t) W.w[t] = w[t];
    k_exact_combine<<<2 * 152, 256, 0, s>>>(m, p, Qs, nq, stride, W, sigma, tau, ebound, Q, E);
}

bool exact_plan(int n, int beta, int nd, ExactPlan* pl) {
    if (beta < 2 || beta > 7 || nd < 1 || beta * nd > 60) return false;
    pl->beta = beta;
    pl->nd = nd;
    pl->npad = (n + 63) / 64 * 64;
    pl->kbs = pl->npad / 64;
    pl->njobs = 0;
    const double lim = 16777216.0;                          // 2^24
    auto dmax = [&](int a) { return a == 1 ? ldexp(1.0, beta) : ldexp(1.0, beta - 1); };
    for (int l = 2; l <= nd + 1; ++l) {
        const int nkb = (l - 1) * pl->kbs;
        int u0 = 0;
        double acc = 0.0;
        for (int u = 0; u <= nkb; ++u) {
            double add = 0.0;
            if (u < nkb) {
                const int a = u / pl->kbs + 1, c = l - a;      // X digit a against zeta digit c
                add = 64.0 * dmax(a) * dmax(c);
                if (add > lim) return false;
            }
            if (u == nkb || acc + add > lim) {
                if (pl->njobs >= kTcMaxJobs) return false;
                TcJob& jb = pl->jobs[pl->njobs];
                jb.ka = (nd - l + 1) * pl->kbs + u0;          // zeta's window starts at digit l - 1
                jb.kb = u0;
                jb.nkb = u - u0;
                jb.slice = pl->njobs;
                pl->w[pl->njobs] = ldexp(1.0, -beta * l);
                ++pl->njobs;
                u0 = u;
                acc = 0.0;
            }
            acc += add;
        }
    }
    const double r = ldexp(1.0, -beta * nd - 1) + ldexp(1.0, -63);
    double E = 2.0 * r + r * r + ldexp(1.0, -44);
    for (int l = nd + 2; l <= 2 * nd; ++l) E += (2 * nd - l + 1) * ldexp(1.0, 2 * beta - 2 - beta * l);
    pl->ebound = (double)n * E * (1.0 + 1e-12);
    return true;
}

void exact_plan_widen(ExactPlan* pl, int tiles, size_t max_slices) {
    while ((size_t)tiles * pl->njobs < 2 * 152 && 2 * pl->njobs <= kTcMaxJobs && (size_t)2 * pl->njobs <= max_slices) {
        bool any = false;
        ExactPlan q = *pl;
        q.njobs = 0;
        for (int t = 0; t < pl->njobs; ++t) {
            const TcJob jb = pl->jobs[t];
            if (jb.nkb >= 8) {
                const int h = jb.nkb / 2;
                q.jobs[q.njobs] = {jb.ka, jb.kb, h, q.njobs};
                q.w[q.njobs++] = pl->w[t];
                q.jobs[q.njobs] = {jb.ka + h, jb.kb + h, jb.nkb - h, q.njobs};
                q.w[q.njobs++] = pl->w[t];
                any = true;
            } else {
                q.jobs[q.njobs] = {jb.ka, jb.kb, jb.nkb, q.njobs};
                q.w[q.njobs++] = pl->w[t];
            }
        }
        if (!any) break;
        *pl = q;
    }
}

}  // namespace kglm
