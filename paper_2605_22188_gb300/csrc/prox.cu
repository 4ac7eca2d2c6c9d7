// Masked proximal step of §3 Eq. (pgd_step_vector_form) for a batch of nodes,
// fused with the FISTA extrapolation and gradient restart.  One warp per node
// up to 512 coordinates (four nodes per CTA; a tuned option up to 2048), one
// CTA per node above.  In FP32 with 512 < p <= 4096 the default is the
// persistent kernel of prox_stream.cu (the kernels here remain tuned options).
//
// For node N with step eta, c = 2*eta*lambda2 = 1/rho and u = v - eta*G:
//   J0:  beta_j = 0
//   J1:  beta_j = sign(u_j) min(|u_j|/(1+c), M)          (Huber prox, weight rho)
//   Jf:  beta_j = u_j - rho^{-1} [prox_{rho g*}(rho u)]_j with prox_{rho g*} by
//        Algorithm 1 (App. B) on the free coordinates, budget kbar.
// Algorithm 1 sorts |rho u|, shrinks the kbar largest by the Huber prox and
// pools adjacent violators.  Violations can only start at the kbar / kbar+1
// boundary (App. B), so the pooled result has one block with common value
// theta (here in the scale of u, theta' = theta/rho):
//   top (the kbar largest |u|):  v_j = max(p(|u_j|), theta'),
//   tail (the others):           v_j = min(|u_j|, theta'),
// p(a) = prox_{rho H_M}(rho a)/rho.  theta' is the root of the block's
// optimality condition
//   f(x) = sum_tail (|u_j| - x)^+ - sum_top (h(x) - |u_j|)^+ = 0,
//   h(x) = x + min(x/c, M),
// a strictly decreasing function.  Instead of the padded column sort of §4.2
// (Fig. 2) the kernel selects the kbar largest free magnitudes (a CTA by radix
// select, a warp by candidates above the kbar-th largest lane maximum),
// sorts only those, finds the piece of f between consecutive top entry points
// p(|u_j|) that holds the root (binary search), and solves the piece by Newton
// steps from its left end: f is convex there, so the steps never pass the
// root, and a step that crosses no tail value lands on it exactly.
// beta_j = sign(u_j)(|u_j| - v_j) then gives
//   top:  sign(u_j) min(|u_j|/(1+c), M, |u_j| - theta'),  tail: sign(u_j)(|u_j| - theta')^+.
#include <float.h>

#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

template <typename T> struct KeyOf;
template <> struct KeyOf<float> { using type = uint32_t; };
template <> struct KeyOf<double> { using type = unsigned long long; };

template <typename T, int NW>
struct ProxShared {
    SelectShared sel;
    T red[2 * 32];
    T fred[kMaxK * NW];   // CTA groups: per-warp tail sums at every breakpoint of the piece search
    int fpos[kMaxK];      // and f > 0 at each breakpoint
    int ired[32];
    int topcnt;
    T topv[kMaxK];
    int topi[kMaxK];
    T sv[kMaxK];      // top magnitudes, descending
    int si[kMaxK];
    T ep[kMaxK];      // their entry points p(sv[i]), descending
    T coef;           // FISTA momentum coefficient of this step
    int r;
};

// p(a) in the scale of u: the Huber prox of weight rho at rho*a, divided by rho.
template <typename T>
__device__ __forceinline__ T entry_point(T a, T c, T M) {
    return a <= (T(1) + c) * M ? a * c / (T(1) + c) : a - M;
}

// Root of n_t (x + min(x/c, M)) - S_t = S_l - n_l x  (the merged block's
// value: Algorithm 1's prox_{rho_bar H_M}(xi_bar) written in the scale of u).
template <typename T>
__device__ __forceinline__ T model_root(T nt, T St, T nl, T Sl, T c, T M) {
    const T xa = c * (St + Sl) / (nt * (T(1) + c) + c * nl);
    if (xa <= c * M) return xa;
    return (St + Sl - nt * M) / (nt + nl);
}

// One node per group (a CTA of NT threads, or a warp with GPC groups per CTA).
template <typename T, typename Grp, int E, int GPC>
__device__ __forceinline__ void prox_node(const ProxArgs& a) {
    using G = Grp;
    using K = typename KeyOf<T>::type;
    constexpr int NT = G::N;
    constexpr int NWG = NT / 32;
    __shared__ ProxShared<T, NWG> shared_all[GPC];
    const int grp = GPC == 1 ? 0 : (int)(threadIdx.x / 32);
    ProxShared<T, NWG>& sh = shared_all[grp];
    const int b = blockIdx.x * GPC + grp;
    // programmatic dependent launch (no-ops without the launch attribute): let the
    // next kernel start its prologue, then wait for the gradient's producer
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (b >= a.m) return;
    if (a.active != nullptr && a.active[b] == 0) return;
    const int p = a.p;
    const size_t base = (size_t)b * p;
    const T* __restrict__ Gm = static_cast<const T*>(a.G);
    T* __restrict__ V = static_cast<T*>(a.V);
    T* __restrict__ Bm = static_cast<T*>(a.B);
    const T eta = T(a.eta), c = T(a.c), M = T(a.M);
    const uint32_t* im = a.in_mask + (size_t)b * a.W;
    const uint32_t* om = a.out_mask + (size_t)b * a.W;

    using Mk = ElemMask<E>;
    // up to 16 elements per thread keep v and beta in registers; more re-read
    // them (the same addresses, from L1/L2) when they are needed again
    constexpr bool HOLD = E <= 16;
    T u[E], vv[HOLD ? E : 1], bo[HOLD ? E : 1];
    Mk valid = 0, fin = 0, fout = 0;
    // A warp per node loads its momentum t, V, beta and fixing bits before the
    // gradient, so that these loads overlap the gradient's (a CTA per node loads
    // them after it: holding them across the gradient loads costs registers, and
    // registers bound how many node CTAs an SM holds).
    constexpr bool EARLY = std::is_same<Grp, WarpGroup>::value;
    const double tprev = (EARLY && G::rank() == 0) ? a.tmom[b] : 0.0;
    auto load_node = [&](int e) {
        const int j = G::rank() + e * NT;
        if constexpr (HOLD) vv[e] = bo[e] = T(0);
        if (j < p) {
            valid |= Mk(1) << e;
            if constexpr (HOLD) {
                vv[e] = V[base + j];
                bo[e] = Bm[base + j];
            }
            if ((im[j >> 5] >> (j & 31)) & 1u) fin |= Mk(1) << e;
            else if ((om[j >> 5] >> (j & 31)) & 1u) fout |= Mk(1) << e;
        }
    };
    if constexpr (EARLY) {
#pragma unroll
        for (int e = 0; e < E; ++e) load_node(e);
    }
    // gradient: G, or the sum of its split slices (slice-outer so that the E
    // loads of a slice are in flight together; order of the sum fixed)
    T gsum[E];
#pragma unroll
    for (int e = 0; e < E; ++e) gsum[e] = T(0);
    if (a.gsplits > 0) {
        // QB slices' loads in flight together; the sum keeps the slice order
        constexpr int QB = E <= 8 ? (EARLY ? 8 : 4) : (E <= 16 ? 2 : 1);   // a warp per node: more slices in flight
        int q = 0;
        for (; q + QB <= a.gsplits; q += QB) {
            float t[QB][E];
#pragma unroll
            for (int qq = 0; qq < QB; ++qq) {
                const float* gp = a.Gpart + (size_t)(q + qq) * a.gstride + base;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int j = G::rank() + e * NT;
                    t[qq][e] = j < p ? gp[j] : 0.f;
                }
            }
#pragma unroll
            for (int qq = 0; qq < QB; ++qq)
#pragma unroll
                for (int e = 0; e < E; ++e) gsum[e] += T(t[qq][e]);
        }
        for (; q < a.gsplits; ++q) {
            const float* gp = a.Gpart + (size_t)q * a.gstride + base;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = G::rank() + e * NT;
                if (j < p) gsum[e] += T(gp[j]);
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = G::rank() + e * NT;
            if (j < p) gsum[e] = Gm[base + j];
        }
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if constexpr (!EARLY) load_node(e);
        u[e] = T(0);
        if (bit(valid, e)) {
            T v;
            if constexpr (HOLD) v = vv[e];
            else v = V[base + G::rank() + e * NT];
            u[e] = v - eta * gsum[e];
        }
    }
    const Mk ffree = valid & ~fin & ~fout;
    // FISTA t update (FP64; tmom holds t_k of the iterate x_k this step makes,
    // t_1 = 1): without a restart t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2 and
    // v_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1}); a restart starts over
    // from x_k (v_{k+1} = x_k, t_{k+1} = 1, so the next coefficient is 0 too).
    // The test picks one at the end; a warp per node computes the candidates
    // here, off the end of its critical path.
    double t_keep = 0.0, c_keep = 0.0;
    auto t_candidates = [&](double tp) {
        t_keep = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tp * tp));
        c_keep = (tp - 1.0) / t_keep;
    };
    if (EARLY && G::rank() == 0) t_candidates(tprev);
    const int kb = a.kbar[b], pf = a.pf[b];

    T theta = T(0);
    Mk top = 0;
    if (kb > 0 && pf > kb) {
        T amax;
        if constexpr (NT == 32) {
            // one warp per node: selection by candidates (FP32) or tournament, already sorted
            if constexpr (sizeof(T) == 4) top = warp_topk_candidates<E, Mk>(u, ffree, kb, sh.sv, sh.si, sh.sel.ckey);
            else top = warp_topk_tournament<E, T, Mk>(u, ffree, kb, sh.sv, sh.si);
            T tmax = T(0);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (bit(ffree & ~top, e)) tmax = max(tmax, abs(u[e]));
            amax = G::max(tmax, sh.red);
        } else {
            static_assert(E <= 32, "the CTA selection takes 32-bit element masks");
            K key[E];
#pragma unroll
            for (int e = 0; e < E; ++e) key[e] = mag_key(abs(u[e]));
            top = group_topk_select<G, E, K>(key, (uint32_t)ffree, kb, sh.sel, sh.ired);
            if (G::rank() == 0) sh.topcnt = 0;
            G::sync();
            T tmax = T(0);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (bit(top, e)) {
                    const int s = atomicAdd(&sh.topcnt, 1);
                    sh.topv[s] = abs(u[e]);
                    sh.topi[s] = G::rank() + e * NT;
                } else if (bit(ffree, e)) {
                    tmax = max(tmax, abs(u[e]));
                }
            }
            amax = G::max(tmax, sh.red);   // also publishes topv (via its barriers)
            G::sync();
            warp_rank_sort_desc<T, G>(sh.topv, sh.topi, kb, sh.sv, sh.si);
        }
        G::sync();
        // entry points p(sv[i]) of the top values, one per group member
        for (int i = G::rank(); i < kb; i += NT) sh.ep[i] = entry_point(sh.sv[i], c, M);
        G::sync();
        if (amax > T(0)) {
            // entry points in ascending order: e_(i) = ep[kb - i], i = 1..kb
            const T emin = sh.ep[kb - 1];
            if (emin >= amax) {
                theta = amax;                      // no violation: nothing pools
            } else {
                int r = 0;                         // entry points below amax (from shared memory)
                for (int i = 0; i < kb; ++i) r += sh.ep[i] < amax;
                auto xval = [&](int i) -> T { return i == 0 ? T(0) : (i <= r ? sh.ep[kb - i] : amax); };
                int lo = 0, hi = r + 1;
                if constexpr (NT == 32) {
                    // one warp: binary search, each probe a shuffle reduction
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        const T x = xval(mid);
                        const T h = x + min(x / c, M);
                        // f(x) = sum_tail (|u| - x)^+ - sum_{top, p(t) < x} (h(x) - t)
                        T part[1] = {T(0)};
#pragma unroll
                        for (int e = 0; e < E; ++e)
                            if (bit(ffree & ~top, e)) part[0] += max(abs(u[e]) - x, T(0));
                        for (int i = G::rank(); i < kb; i += NT)
                            if (sh.ep[i] < x) part[0] -= max(h - sh.sv[i], T(0));
                        G::template sum<1, T>(part, sh.red);
                        if (part[0] > T(0)) lo = mid; else hi = mid;
                    }
                } else {
                    // a CTA: f at every breakpoint x_1..x_r in one pass (per-warp tail
                    // sums, then one thread per breakpoint), f decreasing: lo = #{f > 0}
                    const int w = (int)(threadIdx.x >> 5), ln = (int)(threadIdx.x & 31);
                    for (int i = 1; i <= r; ++i) {
                        const T x = xval(i);
                        T part = T(0);
#pragma unroll
                        for (int e = 0; e < E; ++e)
                            if (bit(ffree & ~top, e)) part += max(abs(u[e]) - x, T(0));
                        part = warp_sum(part);
                        if (ln == 0) sh.fred[(i - 1) * NWG + w] = part;
                    }
                    G::sync();
                    for (int i = G::rank() + 1; i <= r; i += NT) {
                        const T x = xval(i);
                        const T h = x + min(x / c, M);
                        T f = T(0);
                        for (int q = 0; q < NWG; ++q) f += sh.fred[(i - 1) * NWG + q];
                        for (int j = 0; j < kb; ++j)
                            if (sh.ep[j] < x) f -= max(h - sh.sv[j], T(0));
                        sh.fpos[i - 1] = f > T(0);
                    }
                    G::sync();
                    for (int i = 0; i < r; ++i) lo += sh.fpos[i];
                    hi = lo + 1;
                }
                const T xlo = xval(lo), xhi = xval(hi);
                // the block's top part: entries whose entry point is at most xlo (from shared memory)
                T nt = T(0), St = T(0);
                for (int i = 0; i < kb; ++i)
                    if (sh.ep[i] <= xlo) { nt += T(1); St += sh.sv[i]; }
                T th = xlo;
                T q[2] = {T(0), T(0)};
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (bit(ffree & ~top, e) && abs(u[e]) > th) { q[0] += T(1); q[1] += abs(u[e]); }
                G::template sum<2, T>(q, sh.red);
                T nl = q[0], Sl = q[1];
                for (int it = 0; it < 4 * kMaxK + 64; ++it) {
                    T tn = model_root(nt, St, nl, Sl, c, M);
                    tn = min(max(tn, th), xhi);
                    q[0] = q[1] = T(0);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (bit(ffree & ~top, e) && abs(u[e]) > tn) { q[0] += T(1); q[1] += abs(u[e]); }
                    G::template sum<2, T>(q, sh.red);
                    const bool done = (q[0] == nl);
                    th = tn;
                    nl = q[0];
                    Sl = q[1];
                    if (done) break;
                }
                theta = th;
            }
        }
    }

    // the new beta_j; with more than 16 elements per thread it is recomputed in
    // the store loop instead of held (registers bound the nodes in flight)
    auto beta_new = [&](int e) -> T {
        const T au = abs(u[e]);
        T mag = T(0);
        if (bit(fout, e)) {
            mag = T(0);
        } else if (bit(fin, e)) {
            mag = min(au / (T(1) + c), M);
        } else if (kb == 0) {
            mag = T(0);
        } else if (pf <= kb) {
            mag = min(au / (T(1) + c), M);
        } else if (bit(top, e)) {
            mag = max(min(min(au / (T(1) + c), M), au - theta), T(0));
        } else {
            mag = max(au - theta, T(0));
        }
        return u[e] < T(0) ? -mag : mag;
    };
    constexpr bool KEEP = E <= 16;
    T bn[KEEP ? E : 1];
    T dot[1] = {T(0)};
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if constexpr (KEEP) bn[e] = T(0);
        if (!bit(valid, e)) continue;
        const T bv = beta_new(e);
        if constexpr (KEEP) bn[e] = bv;
        T ve, be;
        if constexpr (HOLD) { ve = vv[e]; be = bo[e]; }
        else { const int j = G::rank() + e * NT; ve = V[base + j]; be = Bm[base + j]; }
        dot[0] += (ve - bv) * (bv - be);
    }
    G::template sum<1, T>(dot, sh.red);
    if (G::rank() == 0) {                  // FISTA t update, once per node, in FP64
        if constexpr (!EARLY) t_candidates(a.tmom[b]);
        const bool rs = a.restart && dot[0] > T(0);
        sh.coef = rs ? T(0) : T(c_keep);
        a.tmom[b] = rs ? 1.0 : t_keep;      // restart: start over from this iterate, t = 1
    }
    G::sync();
    const T coef = sh.coef;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int j = G::rank() + e * NT;
        if (bit(valid, e)) {
            T be;
            if constexpr (HOLD) be = bo[e];
            else be = Bm[base + j];         // read before this thread overwrites it
            T bv;
            if constexpr (KEEP) bv = bn[e];
            else bv = beta_new(e);
            const T vn = bv + coef * (bv - be);
            Bm[base + j] = bv;
            V[base + j] = vn;
            if (a.Vop != nullptr) store_operand2(a.Vop, a.Vop_lo, (size_t)b * a.op_ld + j, (float)vn, a.op_bf16);
        }
    }
}

template <typename T, typename Grp, int E, int GPC>
__global__ __launch_bounds__(Grp::N * GPC) void k_prox_fista(ProxArgs a) { prox_node<T, Grp, E, GPC>(a); }

// A warp per node with 32 or more elements per lane, capped at 128 registers
// (four 128-thread CTAs per SM): its nodes are independent, so nodes in flight
// per SM is what hides their latency.
template <typename T, int E>
__global__ __launch_bounds__(128, 4) void k_prox_fista_wide(ProxArgs a) { prox_node<T, WarpGroup, E, 4>(a); }

template <typename T, typename Grp, int E, int GPC>
void launch(cudaStream_t s, const ProxArgs& a, int grid, int block) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.pdl ? 1 : 0;
    // errors surface at the caller's check
    if constexpr (std::is_same<Grp, WarpGroup>::value && E >= 32) cudaLaunchKernelEx(&cfg, k_prox_fista_wide<T, E>, a);
    else cudaLaunchKernelEx(&cfg, k_prox_fista<T, Grp, E, GPC>, a);
}

// Threads per node for the CTA kernels: the default splits a node's
// coordinates 8 per thread; a.threads (FP32, tuned) trades threads for more
// coordinates per thread so that more nodes are in flight per SM.
template <typename T>
int dispatch(cudaStream_t s, const ProxArgs& a) {
    const int p = a.p, m = a.m;
    if (m <= 0) return 0;
#define KGLM_PROX(NT_, E_) launch<T, CtaGroup<NT_>, E_, 1>(s, a, m, NT_)
#define KGLM_PROX_WARP(E_) launch<T, WarpGroup, E_, 4>(s, a, (m + 3) / 4, 128)
    // up to 512 coordinates: one warp per node, four nodes per CTA
    if (p <= 32) KGLM_PROX_WARP(1);
    else if (p <= 64) KGLM_PROX_WARP(2);
    else if (p <= 128) KGLM_PROX_WARP(4);
    else if (p <= 256) KGLM_PROX_WARP(8);
    else if (p <= 512) KGLM_PROX_WARP(16);
    else if constexpr (sizeof(T) == 4) {
        const int t = a.threads;
        if (t == 0 && p <= kStreamMaxP) {           // persistent, a warp streams nodes
            const int rc = prox_stream_f32(s, a);
            if (rc <= 0) return rc;                 // 1: too few warps fit; the kernels below
        }
        if (p <= 1024) {
            if (t == 64) KGLM_PROX(64, 16);
            else if (t == 32) KGLM_PROX_WARP(32);
            else KGLM_PROX(128, 8);
        } else if (p <= 2048) {
            if (t == 128) KGLM_PROX(128, 16);
            else if (t == 64) KGLM_PROX(64, 32);
            else if (t == 32) KGLM_PROX_WARP(64);
            else KGLM_PROX(256, 8);
        } else if (p <= 4096) {
            if (t == 256) KGLM_PROX(256, 16);
            else if (t == 128) KGLM_PROX(128, 32);
            else KGLM_PROX(512, 8);
        } else if (p <= 8192) {
            if (t == 256) KGLM_PROX(256, 32);
            else KGLM_PROX(512, 16);
        } else {
            return -1;
        }
    } else {
        if (p <= 1024) KGLM_PROX(128, 8);
        else if (p <= 2048) KGLM_PROX(256, 8);
        else if (p <= 4096) KGLM_PROX(512, 8);
        else return -1;
    }
#undef KGLM_PROX
#undef KGLM_PROX_WARP
    return 0;
}

}  // namespace

int prox_fista_f64(cudaStream_t s, const ProxArgs& a) { return dispatch<double>(s, a); }
int prox_thread_options(int p, int* out) {
    int n = 0;
    out[n++] = 0;
    if (p > 512 && p <= 1024) { out[n++] = 64; out[n++] = 32; }
    else if (p > 1024 && p <= 2048) { out[n++] = 128; out[n++] = 64; out[n++] = 32; }
    else if (p > 2048 && p <= 4096) { out[n++] = 256; out[n++] = 128; }
    else if (p > 4096 && p <= 8192) { out[n++] = 256; }
    return n;
}
int prox_fista_f32(cudaStream_t s, const ProxArgs& a) { return dispatch<float>(s, a); }

}  // namespace kglm
