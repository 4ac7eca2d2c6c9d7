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

#include "common.cuh"
#include "engine.h"
#include "exact.cuh"

namespace kglm {
namespace {

constexpr double kFeasRtol = 1e-12;

// Reduced-precision modes: the dual point is built in FP32 and the conjugate
// sum is an upper bound with an explicit rounding margin, so that the bound
// stays below Psi(zeta) for the zeta actually used (the FP32 value, exact in
// FP64).  Least squares: zeta = -2(s - y) in FP32 (any zeta is admissible),
// l*(-zeta) = -zeta*y + zeta^2/4 in FP64 with the FP64 data y (exact up to
// FP64 rounding, no transcendental).  Logistic:
// a = sigma(-y s) in FP32, zeta = y a (exact), and
//   l*(-zeta) = a ln a + (1-a) ln(1-a)
// with logf / log1pf, whose maximum errors in the CUDA C Programming Guide's
// accuracy table are 1 and 2 ulp (taken as 2^-23 and 2^-22 relative).  With
// one rounding per product and 1-a exact for a >= 1/2 (one rounding below):
//   |t1 - a ln a| <= (2^-23 + 2^-24)|a ln a|             <= 2^-22 |t1|,
//   |t2 - (1-a) ln(1-a)| <= (2^-22 + 2 * 2^-24)|...|     <= 2^-21 |t2|,
// so each term carries the margin 2^-22|t1| + 2^-21|t2| + 2^-125 (the last
// for denormal products); a term plus its margin is formed in FP32 rounded
// upward (never below the exact sum of the same parts) and the terms are
// summed in FP64.
template <int NT>
__global__ __launch_bounds__(NT) void k_dual_point_f32(CertArgs a) {
    __shared__ double red[2 * (NT / 32)];
    const int b = blockIdx.x;
    const size_t base = (size_t)b * a.n;
    double acc[2] = {0.0, 0.0};
    const float* S = static_cast<const float*>(a.S);
    for (int i = threadIdx.x; i < a.n; i += NT) {
        const float s = S[base + i];
        const float yi = (float)a.y[i];
        if (a.kind == kLSQ) {
            const float z = -2.0f * (s - yi);
            a.zeta[base + i] = (double)z;
            const float r = s - yi;
            acc[0] += (double)(r * r);
            const double w = -(double)z;
            acc[1] += w * a.y[i] + 0.25 * w * w;          // the exact FP64 y: l* is of the data
        } else {
            const float t = yi * s;
            const float e = __expf(-fabsf(t));
            const float sg = t >= 0.f ? e / (1.0f + e) : 1.0f / (1.0f + e);     // sigma(-t)
            a.zeta[base + i] = (double)(yi * sg);
            acc[0] += (double)(fmaxf(-t, 0.f) + log1pf(e));
            float t1 = 0.f, t2 = 0.f;
            if (sg > 0.f) t1 = sg * logf(sg);
            if (sg < 1.f) t2 = (1.0f - sg) * log1pf(-sg);
            // margin and sum in FP32 rounded upward (an upper bound, as the FP64 sum of the
            // same terms was), so that only the running sum uses the slow FP64 pipe
            const float mg = __fadd_ru(__fadd_ru(fabsf(t1) * 0x1p-22f, fabsf(t2) * 0x1p-21f), 0x1p-125f);
            acc[1] += (double)__fadd_ru(__fadd_ru(t1, t2), mg);
        }
    }
    block_sum<NT, 2, double>(acc, red);
    if (threadIdx.x == 0) {
        a.sum_loss[b] = acc[0];
        a.sum_conj[b] = acc[1];
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
        if ((((fin | sel) >> e) & 1u)) sh.sup[atomicAdd(&sh.cnt, 1)] = threadIdx.x + e * NT;
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

}  // namespace

void cert_dual_point(cudaStream_t s, const CertArgs& a) {
    if (a.m <= 0) return;
    if (a.s_is_f64) k_dual_point<256><<<a.m, 256, 0, s>>>(a);
    else k_dual_point_f32<256><<<a.m, 256, 0, s>>>(a);
}

int cert_bound(cudaStream_t s, const CertArgs& a) {
    const int p = a.p, m = a.m;
    if (m <= 0) return 0;
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
