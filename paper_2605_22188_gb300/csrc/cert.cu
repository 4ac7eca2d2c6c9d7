// The safe lower bound of §3 "Safe Lower Bound and Pruning", batched as in §4.4:
//   zeta_b = -dl(X beta_b, y)                       (Eq. (dual_candidate_vector_form))
//   q_b    = X^T zeta_b / (2 lambda2)               (Eq. (batched_dual_candidate_matrix_form))
//   LB_b   = -sum_i l*(-zeta_ib, y_i) - 2 lambda2 [ sum_{J1} H_M(q_j) + TopSum_kbar {H_M(q_j)}_{Jf} ]
//                                                   (Eq. (batched_dual_value_component))
// for every node whatever precision the iterations used: by weak duality it
// is a valid bound for any zeta.  X^T zeta, the Huber/TopSum terms and all
// sums are FP64; in the reduced-precision modes the conjugate terms are FP32
// evaluations with explicit rounding margins (k_dual_point_f32), so the
// returned value is a rigorous lower estimate of Psi(zeta).  The same per-node pass
// evaluates Phi_b = sum l + 2 lambda2 g(beta_b) with g from Theorem 4.1, the
// rounded support J1 cup top-kbar |beta| and the branching index
// argmax_{Jf} |beta_j| of §4.3 (ties to the smaller index).
#include <float.h>

#include <algorithm>

#include "common.cuh"
#include "engine.h"
#include "exact.cuh"

namespace kglm {
namespace {

constexpr double kFeasRtol = 1e-12;

// Reduced-precision modes: the dual point is built in FP32 and the conjugate
// sum is an upper bound with an explicit rounding margin, so that the bound
// stays below Psi(zeta) for the zeta actually used (the FP32 value, exact in
// FP64).  Least squares: zeta = -2 r with r = fl(s - fl(y)) (any zeta is
// admissible), l*(-zeta) = w y + w^2/4 with w = 2 r and the data y:
//   w y + w^2/4 = 2 r y + r^2 = 2 r y32 + 2 r ylo + r^2,   y32 + ylo = y to ~2^-48,
// where 2 r y32 and r^2 are formed exactly as FP32 pairs (product and its
// FMA residual) and 2 r ylo (below 2^-24 of 2 r y) in FP32.  Logistic:
// a = sigma(-y s) in FP32, zeta = y a (exact), and
//   l*(-zeta) = a ln a + (1-a) ln(1-a)
// with logf / log1pf, whose maximum errors in the CUDA C Programming Guide's
// accuracy table are 1 and 2 ulp (taken as 2^-23 and 2^-22 relative).  With
// one rounding per product and 1-a exact for a >= 1/2 (one rounding below):
//   |t1 - a ln a| <= (2^-23 + 2^-24)|a ln a|             <= 2^-22 |t1|,
//   |t2 - (1-a) ln(1-a)| <= (2^-22 + 2 * 2^-24)|...|     <= 2^-21 |t2|,
// so each term carries the margin 2^-22|t1| + 2^-21|t2| + 2^-125 (the last
// for denormal products); a term plus its margin is formed in FP32 rounded
// upward (never below the exact sum of the same parts).
// The running sums of a thread are FP32 pairs (hi, lo) updated by the exact
// two-sum of Knuth (hi + a = s + err exactly in round-to-nearest), about 2^-44
// relative per term, far below the logistic margins and of the order of the
// FP64 rounding of the least-squares terms; they reach FP64 once per thread,
// so that the GPU's slow FP64 pipe carries only the FP64 copy of zeta.
// (The _rn intrinsics keep the compiler from contracting a product into the
// two-sum's first addition, which would break its exactness.)
struct FPair {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float s = __fadd_rn(hi, v);
        const float bb = __fsub_rn(s, hi);
        lo += __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
        hi = s;
    }
    // the exact product a b as its rounded value plus the FMA residual
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float pr = __fmul_rn(a, b);
        add(pr);
        lo += fmaf(a, b, -pr);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// zeta of one sample in the reduced-precision modes (the value the certificate uses).
__device__ __forceinline__ float dual_z(float s, float yi, int kind) {
    if (kind == kLSQ) return -2.0f * (s - yi);
    const float t = yi * s;
    const float e = __expf(-fabsf(t));
    return yi * (t >= 0.f ? e / (1.0f + e) : 1.0f / (1.0f + e));   // y sigma(-t)
}

// Digits of v = z / 2^e (|v| < 1) as in k_digits of cert_exact.cu, from the FP32
// value alone: V = rint(v 2^62) by integer shifts of z's significand (nearest,
// halves away from zero: |V - v 2^62| <= 1/2 as the error bound assumes), then
// the same signed digits from the top, segment nd - a for digit a (reversed).
__device__ __forceinline__ void dz_digits(float z, int e, int nd, int beta, __nv_bfloat16* d, size_t npad,
                                          size_t i) {
    long long V = 0;
    const uint32_t u = __float_as_uint(z);
    const int ex = (int)((u >> 23) & 0xffu);
    if (ex != 255 && (ex != 0 || (u & 0x7fffffu) != 0)) {       // a non-finite z has no digits
        const long long mnt = ex ? (long long)((u & 0x7fffffu) | 0x800000u) : (long long)(u & 0x7fffffu);
        const int sh = (ex ? ex : 1) - 150 + 62 - e;              // z = mnt 2^(ex - 150), v 2^62 = mnt 2^sh
        long long mag = 0;
        if (sh >= 0) mag = sh < 63 ? mnt << sh : 0;                // |v| < 1: below 2^62, so sh < 62
        else if (sh > -26) mag = (mnt + (1ll << (-sh - 1))) >> (-sh);
        V = (u >> 31) ? -mag : mag;
    }
    for (int a = 1; a <= nd; ++a) {
        const int sh = 62 - beta * a;
        const long long dg = (V + (1ll << (sh - 1))) >> sh;        // nearest, halves up
        V -= dg << sh;
        d[(size_t)(nd - a) * npad + i] = __int2bfloat16_rn((int)dg);
    }
}

template <int NT>
__global__ __launch_bounds__(NT) void k_dual_point_f32(CertArgs a) {
    __shared__ double red[2 * (NT / 32)];
    __shared__ float redf[NT / 32];
    const int b = blockIdx.x;
    const size_t base = (size_t)b * a.n;
    FPair sl, sc;
    float zmax = 0.f;
    const float* S = static_cast<const float*>(a.S);
    for (int i = threadIdx.x; i < a.n; i += NT) {
        const float s = S[base + i];
        const float yi = a.y32[i];
        const float z = dual_z(s, yi, a.kind);
        zmax = fmaxf(zmax, fabsf(z));
        if (a.kind == kLSQ) {
            const float r = s - yi;
            a.zeta[base + i] = (double)z;
            sl.add(__fmul_rn(r, r));                         // the loss term as the iterations form it
            const float r2 = 2.0f * r;                        // w = -zeta, exact
            sc.add_prod(r2, yi);                              // 2 r y32, exact as a pair
            sc.add_prod(r, r);                                // r^2 = w^2 / 4, exact as a pair
            sc.lo += r2 * a.ylo[i];                           // 2 r ylo
        } else {
            const float t = yi * s;
            const float e = __expf(-fabsf(t));
            const float sg = t >= 0.f ? e / (1.0f + e) : 1.0f / (1.0f + e);     // sigma(-t)
            a.zeta[base + i] = (double)z;
            sl.add(fmaxf(-t, 0.f) + log1pf(e));
            float t1 = 0.f, t2 = 0.f;
            if (sg > 0.f) t1 = sg * logf(sg);
            if (sg < 1.f) t2 = (1.0f - sg) * log1pf(-sg);
            // margin and term in FP32 rounded upward (an upper bound of the exact term)
            const float mg = __fadd_ru(__fadd_ru(fabsf(t1) * 0x1p-22f, fabsf(t2) * 0x1p-21f), 0x1p-125f);
            sc.add(__fadd_ru(__fadd_ru(t1, t2), mg));
        }
    }
    double acc[2] = {sl.value(), sc.value()};
    block_sum<NT, 2, double>(acc, red);
    if (threadIdx.x == 0) {
        a.sum_loss[b] = acc[0];
        a.sum_conj[b] = acc[1];
    }
    if (a.DZ == nullptr) return;
    // the digits of zeta for the exact-splitting X^T zeta: the row's scale from the
    // first pass, then zeta again (the same FP32 operations) and its digits
    zmax = warp_max(zmax);
    if ((threadIdx.x & 31) == 0) redf[threadIdx.x >> 5] = zmax;
    __syncthreads();
    float mx = 0.f;
    for (int w = 0; w < NT / 32; ++w) mx = fmaxf(mx, redf[w]);
    const int e = mx > 0.f ? ilogbf(mx) + 1 : 0;                   // 2^e > mx
    if (threadIdx.x == 0) a.ztau[b] = mx > 0.f ? ldexp(1.0, e) : 0.0;   // a zero row is exact
    __nv_bfloat16* d = a.DZ + (size_t)b * a.dz_nd * a.dz_npad;
    for (int i = threadIdx.x; i < a.dz_npad; i += NT) {
        const float z = i < a.n ? dual_z(S[base + i], a.y32[i], a.kind) : 0.f;
        dz_digits(z, e, a.dz_nd, a.dz_beta, d, (size_t)a.dz_npad, (size_t)i);
    }
}

template <int NT>
__global__ __launch_bounds__(NT) void k_dual_point(CertArgs a) {
    __shared__ double red[2 * (NT / 32)];
    const int b = blockIdx.x;
    const size_t base = (size_t)b * a.n;
    double acc[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < a.n; i += NT) {
        const double s = a.s_is_f64 ? static_cast<const double*>(a.S)[base + i]
                                    : (double)static_cast<const float*>(a.S)[base + i];
        const double yi = a.y[i];
        const double d = dloss(s, yi, a.kind);       // zeta = -d
        a.zeta[base + i] = -d;
        acc[0] += loss64(s, yi, a.kind);
        acc[1] += loss_conj64(d, yi, a.kind);        // l*(-zeta) = l*(d)
    }
    block_sum<NT, 2, double>(acc, red);
    if (threadIdx.x == 0) {
        a.sum_loss[b] = acc[0];
        a.sum_conj[b] = acc[1];
    }
}

struct CertShared {
    SelectShared sel;
    double red[6 * 32];
    int ired[32];
    int cnt;
    double topv[kMaxK];
    int topi[kMaxK];
    double sv[kMaxK];
    int si[kMaxK];
    int sup[kMaxK];
    int sups[kMaxK];
    double gfree;
};

template <int NT, int E>
__global__ __launch_bounds__(NT) void k_cert_bound(const __grid_constant__ CertArgs a) {
    using K = unsigned long long;
    __shared__ CertShared sh;
    const int b = blockIdx.x, p = a.p;
    const size_t base = (size_t)b * p;
    const double M = a.M, inv2l = 1.0 / (2.0 * a.lam2);
    const uint32_t* im = a.in_mask + (size_t)b * a.W;
    const uint32_t* om = a.out_mask + (size_t)b * a.W;
    double q[E], be[E];
    uint32_t valid = 0, fin = 0, fout = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int j = threadIdx.x + e * NT;
        q[e] = be[e] = 0.0;
        if (j < p) {
            valid |= 1u << e;
            if (a.Qs) {
                // |X^T zeta| bounded from above: |Q~| + its distance bound (H_M, TopSum increase in |q|)
                double err;
                const double qv = exact_q(a.Qs, a.nqs, a.qs_stride, a.qs_w, base + j, a.xsig[j] * a.ztau[b], a.ebound, &err);
                q[e] = (fabs(qv) + err) * inv2l;
            } else {
                q[e] = a.Q[base + j] * inv2l;
            }
            be[e] = a.b_is_f64 ? static_cast<const double*>(a.B)[base + j]
                               : (double)static_cast<const float*>(a.B)[base + j];
            if ((im[j >> 5] >> (j & 31)) & 1u) fin |= 1u << e;
            else if ((om[j >> 5] >> (j & 31)) & 1u) fout |= 1u << e;
        }
    }
    const uint32_t ffree = valid & ~fin & ~fout;
    const int kb = a.kbar[b], pf = a.pf[b];

    // ---- TopSum_kbar of H_M(q) over Jf (H_M is increasing in |q|)
    double hthr = 0.0;
    int need = 0;
    K thr = 0;
    const bool topsum_sel = (kb > 0 && pf > kb);
    if (topsum_sel) {
        K key[E];
#pragma unroll
        for (int e = 0; e < E; ++e) key[e] = mag_key(fabs(q[e]));
        block_kth_largest<NT, E, K>(key, ffree, kb, sh.sel, thr, need);
        hthr = huber64(__longlong_as_double((long long)thr), M);
    }
    // sums: [J1 Huber, J1 beta^2, free |beta|, free nnz, free beta^2, infeasible, topsum part]
    double acc[6] = {0, 0, 0, 0, 0, 0};
    double ts[1] = {0.0};
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (!((valid >> e) & 1u)) continue;
        const double ab = fabs(be[e]);
        if ((fin >> e) & 1u) {
            acc[0] += huber64(q[e], M);
            acc[1] += be[e] * be[e];
            if (ab > M * (1.0 + kFeasRtol)) acc[5] += 1.0;
        } else if ((fout >> e) & 1u) {
            if (be[e] != 0.0) acc[5] += 1.0;
        } else {
            acc[2] += ab;
            acc[3] += ab > 0.0 ? 1.0 : 0.0;
            acc[4] += ab * ab;
            if (ab > M * (1.0 + kFeasRtol)) acc[5] += 1.0;
            if (kb > 0) {
                if (!topsum_sel) ts[0] += huber64(q[e], M);
                else if (mag_key(fabs(q[e])) > thr) ts[0] += huber64(q[e], M);
            }
        }
    }
    block_sum<NT, 6, double>(acc, sh.red);
    block_sum<NT, 1, double>(ts, sh.red);
    const double topsum = ts[0] + (topsum_sel ? need * hthr : 0.0);
    const double gconj = acc[0] + topsum;
    const double lb = -a.sum_conj[b] - 2.0 * a.lam2 * gconj;

    // ---- top-kbar |beta| over Jf (ties to the smaller index): rounding, j*, Theorem 4.1
    if (threadIdx.x == 0) sh.cnt = 0;
    __syncthreads();
    const bool leaf = (kb == 0 || pf <= kb);
    uint32_t sel = 0;
    if (!leaf) {
        K key[E];
#pragma unroll
        for (int e = 0; e < E; ++e) key[e] = mag_key(fabs(be[e]));
        sel = block_topk_select<NT, E, K>(key, ffree, kb, sh.sel, sh.ired);
#pragma unroll
        for (int e = 0; e < E; ++e)
            if ((sel >> e) & 1u) {
                const int s = atomicAdd(&sh.cnt, 1);
                sh.topv[s] = fabs(be[e]);
                sh.topi[s] = threadIdx.x + e * NT;
            }
        __syncthreads();
        warp_rank_sort_desc<double>(sh.topv, sh.topi, kb, sh.sv, sh.si);
    } else if (kb > 0) {
        sel = ffree;                                   // every free coordinate fits the budget
    }
    __syncthreads();
    // support = J1 cup selected free, ascending
    if (threadIdx.x == 0) sh.cnt = 0;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e)
        if ((((fin | sel) >> e) & 1u)) {
            const int c = atomicAdd(&sh.cnt, 1);
            if (kglm_check(c < kMaxK, a.chk, kChkCert)) sh.sup[c] = threadIdx.x + e * NT;
        }
    __syncthreads();
    const int ns = sh.cnt;
    if (threadIdx.x < 32) {
        for (int i = threadIdx.x; i < ns; i += 32) {
            const int v = sh.sup[i];
            int r = 0;
            for (int j = 0; j < ns; ++j) r += sh.sup[j] < v;
            sh.sups[r] = v;
        }
    }
    // Theorem 4.1 on the free part (thread 0)
    if (threadIdx.x == 0) {
        const double total = acc[2], nnz = acc[3], sumsq = acc[4];
        double gf;
        if (acc[5] > 0.0) gf = INFINITY;
        else if (kb == 0) gf = total > 0.0 ? INFINITY : 0.0;
        else if (total / M > kb * (1.0 + kFeasRtol)) gf = INFINITY;
        else if (nnz <= kb) gf = 0.5 * sumsq;
        else {
            // s = the smallest index with tau_s >= |beta|_(s+1); then |beta|_(s) > tau_s
            // too, as Theorem 4.1 requires.  s = kbar - 1 qualifies in exact
            // arithmetic; it is also taken if rounding in total - pre says otherwise.
            double pre = 0.0, presq = 0.0;
            int s = 0;
            for (; s < kb - 1; ++s) {
                if ((total - pre) / (kb - s) >= sh.sv[s]) break;
                pre += sh.sv[s];
                presq += sh.sv[s] * sh.sv[s];
            }
            const double tail = total - pre;
            gf = 0.5 * (presq + tail / (kb - s) * tail);
        }
        sh.gfree = gf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.lb[b] = lb;
        const double g = 0.5 * acc[1] + sh.gfree;
        a.primal[b] = isinf(g) ? INFINITY : a.sum_loss[b] + 2.0 * a.lam2 * g;
        a.jstar[b] = leaf ? -1 : sh.si[0];
    }
    for (int i = threadIdx.x; i < a.k; i += NT) a.support[(size_t)b * a.k + i] = i < ns ? sh.sups[i] : -1;
}

// ---- the same bound, primal, support and branching index with a warp per node,
// for FP32 beta with X^T zeta as exact-splitting partials (BF16/TF32 modes).
// The CTA kernel above spends its time in FP64 arithmetic on every coordinate
// (the slice combine, H_M, the sums) and in the barriers of two block-wide
// radix selections.  Here FP64 work is confined to the few coordinates whose
// values are summed:
// * one pass over the free coordinates combines the slices in FP32 with a
//   rigorous error bound and keeps in shared memory an upper bound u_j, and in
//   registers the lane's two largest lower bounds l_j, of the value
//   v_j = (|q~_j| + err_j) / (2 lambda2) that the FP64 combine gives
//   (l_j <= v_j <= u_j); the beta sums of Theorem 4.1 run in compensated FP32;
// * TopSum: the kbar-th largest of the 64 lane samples, t, is at most the
//   kbar-th largest l, hence at most the kbar-th largest v, so every coordinate
//   of the top kbar has u_j >= t; those (normally a few more than kbar) get
//   their exact FP64 v_j (the combine of the CTA kernel) and are ranked; when
//   more than kCertCap qualify (near-ties), they are streamed through an exact
//   top-kbar list instead;
// * top-kbar |beta| over Jf (ties to the smaller index): lane samples of the
//   beta keys, a gather of the candidates and their ranks; zeros tie-break by
//   index directly (the smallest free indices with beta = 0).
constexpr int kCertCap = 128;
constexpr int kCertMaxWarps = 16;

struct CertWarp {
    int cand[kCertCap];
    union {
        double cval[kCertCap];                 // exact v of the TopSum candidates
        unsigned long long bkey[kCertCap];     // (|beta| key, ~j) of the beta candidates
    };
    double tv[kMaxK];
    float sv[kMaxK];
    int si[kMaxK];
    int sup[2 * kMaxK];
    int ncand, nsup;
};

__host__ __device__ inline size_t cert_row(int p) { return ((size_t)p + 3) / 4 * 4; }
__host__ __device__ inline size_t cert_hdr() { return (sizeof(CertWarp) + 15) / 16 * 16; }
__host__ __device__ inline size_t cert_warp_bytes(int p) { return cert_hdr() + cert_row(p) * sizeof(uint32_t); }
__host__ __device__ inline size_t cert_cta_bytes(int p, int wpc) {
    return (kTcMaxJobs + cert_row(p)) * sizeof(float) + wpc * cert_warp_bytes(p);
}

// compensated FP32 accumulation (Knuth's two-sum; the product error by an FMA)
__device__ __forceinline__ void acc2(float& hi, float& lo, float x) {
    const float s = hi + x, bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}
__device__ __forceinline__ void acc2_sq(float& hi, float& lo, float x) {
    const float pr = x * x;
    acc2(hi, lo, pr);
    lo += fmaf(x, x, -pr);
}

__device__ __forceinline__ double cert_exact_v(const CertArgs& a, size_t base, int j, int b, double inv2l) {
    double err;
    const double qv = exact_q(a.Qs, a.nqs, a.qs_stride, a.qs_w, base + j, a.xsig[j] * a.ztau[b], a.ebound, &err);
    return (fabs(qv) + err) * inv2l;
}

__global__ __launch_bounds__(32 * kCertMaxWarps) void k_cert_bound_warp(const __grid_constant__ CertArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    const int p = a.p, nq = a.nqs;
    float* wf = reinterpret_cast<float*>(smem);                 // slice weights (powers of two) in FP32
    float* xs = wf + kTcMaxJobs;                                // sigma_j in FP32 (shared by the CTA)
    unsigned char* wb = smem + (kTcMaxJobs + cert_row(p)) * sizeof(float) + (size_t)warp * cert_warp_bytes(p);
    CertWarp& h = *reinterpret_cast<CertWarp*>(wb);
    uint32_t* su = reinterpret_cast<uint32_t*>(wb + cert_hdr());
    for (int j = threadIdx.x; j < p; j += blockDim.x) xs[j] = (float)a.xsig[j];
    for (int t = threadIdx.x; t < nq; t += blockDim.x) wf[t] = (float)a.qs_w[t];
    __syncthreads();
    const double M = a.M, inv2l = 1.0 / (2.0 * a.lam2);
    const double mth = M * (1.0 + kFeasRtol);
    const float mth_f = __double2float_rd(mth);                // |b| > mth  <=>  |b| > mth_f for FP32 b
    const float ebf = (float)a.ebound;
    const float gam = (float)(nq + 2) * 0x1p-23f;               // |acc_f - acc| <= gam * sum |w P|, with margin
    const float rlo = 1.0f - 0x1p-19f, rhi = 1.0f + 0x1p-19f;   // covers the FP32 roundings below
    // node b to CTA b mod grid: the CTAs (and SMs) hold equal shares of the nodes
    for (int b = warp * gridDim.x + blockIdx.x; b < a.m; b += gridDim.x * wpc) {
        const size_t base = (size_t)b * p;
        const uint32_t* im = a.in_mask + (size_t)b * a.W;
        const uint32_t* om = a.out_mask + (size_t)b * a.W;
        const int kb = a.kbar[b], pf = a.pf[b];
        const float* B = static_cast<const float*>(a.B) + base;
        const float zf = (float)(a.ztau[b] * inv2l);
        if (lane == 0) { h.ncand = 0; h.nsup = 0; }
        // ---- pass over the coordinates: u_j to shared memory, lane samples, free beta sums
        float s1h = 0.f, s1l = 0.f, s2h = 0.f, s2l = 0.f;       // free sum |beta|, sum beta^2
        int nnz = 0, infeas = 0;
        uint32_t l1 = 0, l2 = 0, b1 = 0, b2 = 0;                 // two largest l keys, beta keys
        for (int j = lane; j < p; j += 32) {
            const uint32_t w = j >> 5, bit = 1u << (j & 31);
            const bool in = (im[w] & bit) != 0, out = !in && (om[w] & bit) != 0;
            uint32_t ukey = 0;
            if (!in && !out) {
                const float* qp = a.Qs + base + j;
                float accf = 0.f, absf = 0.f;
                // all the slices' loads of a coordinate in flight at once (up to 32)
                for (int t0 = 0; t0 < nq; t0 += 32) {
                    float v[32];
#pragma unroll
                    for (int t = 0; t < 32; ++t) v[t] = (t0 + t < nq) ? __ldg(qp + (size_t)(t0 + t) * a.qs_stride) : 0.f;
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        if (t0 + t < nq) {
                            const float wt = wf[t0 + t];
                            accf = fmaf(wt, v[t], accf);
                            absf = fmaf(wt, fabsf(v[t]), absf);
                        }
                    }
                }
                const float cf = xs[j] * zf, d = gam * absf, aa = fabsf(accf);
                float vl = cf * ((aa - d) + ebf) * rlo - 4.0f * FLT_MIN;
                float vu = cf * ((aa + d) + ebf) * rhi + 4.0f * FLT_MIN;
                vl = fminf(fmaxf(vl, 0.f), 0.5f * FLT_MAX);          // an overflowed l: v is larger still
                if (!(vu >= 0.f) || !(cf >= FLT_MIN)) {              // NaN, or sigma tau / 2 lambda2 below
                    vu = INFINITY;                                   // the normal range: no bound, always
                    vl = 0.f;                                        // a candidate
                }
                ukey = __float_as_uint(vu) + 1u;
                const uint32_t lkey = __float_as_uint(vl) + 1u;
                if (lkey > l1) { l2 = l1; l1 = lkey; } else if (lkey > l2) { l2 = lkey; }
                const float bv = B[j], ab = fabsf(bv);
                acc2(s1h, s1l, ab);
                acc2_sq(s2h, s2l, ab);
                nnz += ab > 0.f;
                infeas += ab > mth_f;
                const uint32_t bk = __float_as_uint(ab) + 1u;
                if (bk > b1) { b2 = b1; b1 = bk; } else if (bk > b2) { b2 = bk; }
            } else if (out) {
                infeas += B[j] != 0.f;
            }
            su[j] = ukey;
        }
        const double total = warp_sum((double)s1h + (double)s1l);
        const double sumsq = warp_sum((double)s2h + (double)s2l);
        nnz = warp_sum(nnz);
        // ---- J1: exact v, beta^2 and feasibility (at most k coordinates)
        for (int w = lane; w < a.W; w += 32) {
            uint32_t bits = im[w];
            while (bits) {
                const int j = 32 * w + __ffs(bits) - 1;
                bits &= bits - 1;
                const int c = atomicAdd(&h.nsup, 1);
                if (kglm_check(c < kMaxK, a.chk, kChkCert) && c < kMaxK) h.sup[c] = j;   // |J1| <= k <= kMaxK when validated
            }
        }
        __syncwarp();
        const int n1 = min(h.nsup, kMaxK);
        double hj1 = 0.0, bj1 = 0.0;
        for (int i = lane; i < n1; i += 32) {
            const int j = h.sup[i];
            hj1 += huber64(cert_exact_v(a, base, j, b, inv2l), M);
            const double bv = (double)B[j];
            bj1 += bv * bv;
            infeas += fabs(bv) > mth;
        }
        hj1 = warp_sum(hj1);
        bj1 = warp_sum(bj1);
        infeas = warp_sum(infeas);
        const bool leaf = kb == 0 || pf <= kb;
        // ---- TopSum_kbar {H_M(v_j)}_{j in Jf}
        double part = 0.0;
        if (!leaf) {
            uint32_t k0 = l1, k1 = l2;
            sort64(k0, k1, lane);
            const int pos = 64 - kb;
            const uint32_t ta = __shfl_sync(0xffffffffu, k0, pos >> 1), tb = __shfl_sync(0xffffffffu, k1, pos >> 1);
            const uint32_t tau = max((pos & 1) ? tb : ta, 1u);
            for (int j = lane; j < p; j += 32)
                if (su[j] >= tau) {
                    const int c = atomicAdd(&h.ncand, 1);
                    if (c < kCertCap) h.cand[c] = j;
                }
            __syncwarp();
            const int total_c = h.ncand;
            if (total_c <= kCertCap) {
                for (int i = lane; i < total_c; i += 32) h.cval[i] = cert_exact_v(a, base, h.cand[i], b, inv2l);
                __syncwarp();
                for (int i = lane; i < total_c; i += 32) {
                    const double ci = h.cval[i];
                    int r = 0;
                    for (int t = 0; t < total_c; ++t) r += h.cval[t] > ci || (h.cval[t] == ci && t < i);
                    if (r < kb) part += huber64(ci, M);
                }
            } else {
                // near-ties: every qualifying coordinate through an exact top-kbar list (descending)
                int nt = 0;
                double vmin = -1.0;
                for (int j0 = 0; j0 < p; j0 += 32) {
                    const int j = j0 + lane;
                    double v = -1.0;
                    if (j < p && su[j] >= tau) v = cert_exact_v(a, base, j, b, inv2l);
                    uint32_t bal = __ballot_sync(0xffffffffu, v > vmin);
                    while (bal) {
                        const int src = __ffs(bal) - 1;
                        bal &= bal - 1;
                        const double x = __shfl_sync(0xffffffffu, v, src);
                        if (nt == kb && !(x > vmin)) continue;
                        if (lane == 0) {
                            int i = nt < kb ? nt : kb - 1;
                            while (i > 0 && h.tv[i - 1] < x) { h.tv[i] = h.tv[i - 1]; --i; }
                            h.tv[i] = x;
                        }
                        __syncwarp();
                        nt = min(nt + 1, kb);
                        vmin = nt == kb ? h.tv[kb - 1] : -1.0;
                    }
                }
                for (int i = lane; i < nt; i += 32) part += huber64(h.tv[i], M);
            }
            __syncwarp();
            if (lane == 0) h.ncand = 0;
        } else if (kb > 0) {
            // every free coordinate fits the budget (pf <= kbar <= kMaxK): all join the sum and the support
            for (int j = lane; j < p; j += 32)
                if (su[j] != 0u) {
                    part += huber64(cert_exact_v(a, base, j, b, inv2l), M);
                    const int c = atomicAdd(&h.nsup, 1);
                    if (kglm_check(c < 2 * kMaxK, a.chk, kChkCert) && c < 2 * kMaxK) h.sup[c] = j;
                }
        }
        const double topsum = warp_sum(part);
        const double lb = -a.sum_conj[b] - 2.0 * a.lam2 * (hj1 + topsum);
        __syncwarp();
        // ---- top-kbar |beta| over Jf, ties to the smaller index
        if (!leaf) {
            uint32_t k0 = b1, k1 = b2;
            sort64(k0, k1, lane);
            const int pos = 64 - kb;
            const uint32_t ta = __shfl_sync(0xffffffffu, k0, pos >> 1), tb = __shfl_sync(0xffffffffu, k1, pos >> 1);
            const uint32_t tau = max((pos & 1) ? tb : ta, 2u);     // nonzero |beta| only; zeros below
            for (int j = lane; j < p; j += 32) {
                if (su[j] == 0u) continue;
                const uint32_t key = __float_as_uint(fabsf(B[j])) + 1u;
                if (key >= tau) {
                    const int c = atomicAdd(&h.ncand, 1);
                    if (c < kCertCap) h.bkey[c] = ((unsigned long long)key << 32) | (0xffffffffu - (uint32_t)j);
                }
            }
            __syncwarp();
            const int total_c = h.ncand;
            int got = 0;
            if (total_c <= kCertCap) {
                for (int i = lane; i < total_c; i += 32) {
                    const unsigned long long ci = h.bkey[i];
                    int r = 0;
                    for (int t = 0; t < total_c; ++t) r += h.bkey[t] > ci;
                    if (r < kb) {
                        h.sv[r] = __uint_as_float((uint32_t)(ci >> 32) - 1u);
                        h.si[r] = (int)(0xffffffffu - (uint32_t)ci);
                    }
                }
                got = min(total_c, kb);
            } else {
                unsigned long long last = ~0ull;                    // kb rounds of a warp argmax
                for (int r = 0; r < kb; ++r) {
                    unsigned long long best = 0ull;
                    for (int j = lane; j < p; j += 32) {
                        if (su[j] == 0u) continue;
                        const uint32_t key = __float_as_uint(fabsf(B[j])) + 1u;
                        const unsigned long long pk = ((unsigned long long)key << 32) | (0xffffffffu - (uint32_t)j);
                        if (key >= 2u && pk < last && pk > best) best = pk;
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
                        best = x > best ? x : best;
                    }
                    if (best == 0ull) break;
                    last = best;
                    if (lane == 0) {
                        h.sv[r] = __uint_as_float((uint32_t)(best >> 32) - 1u);
                        h.si[r] = (int)(0xffffffffu - (uint32_t)best);
                    }
                    ++got;
                }
            }
            __syncwarp();
            // fewer than kbar nonzero: the free zeros of smallest index fill the rest
            for (int j0 = 0; j0 < p && got < kb; j0 += 32) {
                const int j = j0 + lane;
                const bool z = j < p && su[j] != 0u && B[j] == 0.f;
                uint32_t bal = __ballot_sync(0xffffffffu, z);
                const int before = __popc(bal & ((1u << lane) - 1u));
                if (z && got + before < kb && kglm_check(got + before < kMaxK, a.chk, kChkCert)) {
                    h.sv[got + before] = 0.f;
                    h.si[got + before] = j;
                }
                got = min(kb, got + __popc(bal));
            }
            __syncwarp();
            for (int i = lane; i < kb; i += 32) h.sup[n1 + i] = h.si[i];
            __syncwarp();
            if (lane == 0) h.nsup = n1 + kb;
        }
        __syncwarp();
        // ---- support ascending (the warp); Theorem 4.1 and the outputs (lane 0)
        const int ns = min(h.nsup, kMaxK);
        int srt[2] = {-1, -1};
        for (int i = lane, t = 0; i < ns && t < 2; i += 32, ++t) {
            const int v = h.sup[i];
            int r = 0;
            for (int q = 0; q < ns; ++q) r += h.sup[q] < v;
            srt[t] = r;
        }
        const int vals[2] = {lane < ns ? h.sup[lane] : -1, lane + 32 < ns ? h.sup[lane + 32] : -1};
        __syncwarp();
        for (int t = 0; t < 2; ++t)
            if (srt[t] >= 0) h.sup[srt[t]] = vals[t];
        __syncwarp();
        for (int i = lane; i < a.k; i += 32) a.support[(size_t)b * a.k + i] = i < ns ? h.sup[i] : -1;
        if (lane == 0) {
            double gf;
            if (infeas > 0) gf = INFINITY;
            else if (kb == 0) gf = total > 0.0 ? INFINITY : 0.0;
            else if (total / M > kb * (1.0 + kFeasRtol)) gf = INFINITY;
            else if (nnz <= kb) gf = 0.5 * sumsq;
            else {
                // s = the smallest index with tau_s >= |beta|_(s+1) (Theorem 4.1), s = kbar - 1
                // taken also if rounding in total - pre says otherwise
                double pre = 0.0, presq = 0.0;
                int s = 0;
                for (; s < kb - 1; ++s) {
                    const double v = (double)h.sv[s];
                    if ((total - pre) / (kb - s) >= v) break;
                    pre += v;
                    presq += v * v;
                }
                const double tail = total - pre;
                gf = 0.5 * (presq + tail / (kb - s) * tail);
            }
            const double g = 0.5 * bj1 + gf;
            a.lb[b] = lb;
            a.primal[b] = isinf(g) ? INFINITY : a.sum_loss[b] + 2.0 * a.lam2 * g;
            a.jstar[b] = leaf ? -1 : h.si[0];
        }
        __syncwarp();
    }
}

}  // namespace

void cert_dual_point(cudaStream_t s, const CertArgs& a) {
    if (a.m <= 0) return;
    if (a.s_is_f64) k_dual_point<256><<<a.m, 256, 0, s>>>(a);
    else k_dual_point_f32<256><<<a.m, 256, 0, s>>>(a);
}

// The warp kernel's FP32 combine needs weights that are powers of two (products
// with the FP32 slices exact) within FP32's normal range.
static bool cert_warp_ok(const CertArgs& a) {
    if (a.nqs < 1 || a.nqs > kTcMaxJobs) return false;
    for (int t = 0; t < a.nqs; ++t) {
        int e = 0;
        if (frexp(a.qs_w[t], &e) != 0.5 || e < -90 || e > 40) return false;
    }
    return true;
}

int cert_bound(cudaStream_t s, const CertArgs& a) {
    const int p = a.p, m = a.m;
    if (m <= 0) return 0;
    if (!a.b_is_f64 && a.Qs && p > 512 && p <= 16384 && cert_warp_ok(a)) {
        // a warp per node (as many as fit in shared memory, at most 16 per CTA)
        static const int opted = [] {
            return cudaFuncSetAttribute(k_cert_bound_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024) ==
                   cudaSuccess;
        }();
        int wpc = kCertMaxWarps;
        while (wpc > 1 && cert_cta_bytes(p, wpc) > (227u << 10)) --wpc;
        if (opted && cert_cta_bytes(p, wpc) <= (227u << 10)) {
            const int per_sm = std::max(1, (int)((228u << 10) / (cert_cta_bytes(p, wpc) + 1024)));
            const int grid = std::max(1, std::min(152 * per_sm, m));
            k_cert_bound_warp<<<grid, 32 * wpc, cert_cta_bytes(p, wpc), s>>>(a);
            return 0;
        }
    }
#define KGLM_CERT(NT_, E_) k_cert_bound<NT_, E_><<<m, NT_, 0, s>>>(a)
    if (p <= 64) KGLM_CERT(32, 2);
    else if (p <= 128) KGLM_CERT(64, 2);
    else if (p <= 256) KGLM_CERT(64, 4);
    else if (p <= 512) KGLM_CERT(128, 4);
    else if (p <= 1024) KGLM_CERT(128, 8);
    else if (p <= 2048) KGLM_CERT(256, 8);
    else if (p <= 4096) KGLM_CERT(512, 8);
    else if (p <= 8192) KGLM_CERT(512, 16);
    else return -1;
#undef KGLM_CERT
    return 0;
}

}  // namespace kglm
