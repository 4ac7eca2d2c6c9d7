// Masked proximal step of §3 Eq. (pgd_step_vector_form) with the FISTA
// extrapolation and gradient restart, for FP32 batches with 512 < p <= 4096:
// a persistent kernel in which every warp streams nodes, one at a time, through
// its own slice of shared memory.
//
// The step is the one of prox.cu (Algorithm 1 of App. B as top-kbar selection
// plus one pooled block with threshold theta, in the scale of u):
//   J0: beta = 0;  J1: beta = sign(u) min(|u|/(1+c), M);
//   top (kbar largest free |u|): sign(u) max(min(|u|/(1+c), M, |u| - theta), 0);
//   tail (other free):           sign(u) max(|u| - theta, 0);
//   theta = the root of f(x) = sum_tail (|u|-x)^+ - sum_top (h(x)-|u|)^+,
//   h(x) = x + min(x/c, M), or max tail |u| when no entry point lies below it.
// What differs is the schedule.  The CTA-per-node kernel holds a node's
// coordinates in registers and spends most of its time in barrier-separated
// phases with three nodes per SM, so HBM idles.  Here a warp copies the node's
// rows of G (or its first split slice) and V into shared memory with
// asynchronous 16-byte copies (one round trip per node, no registers held),
// and every later pass runs on shared memory with warp shuffles only, so that
// an SM keeps a dozen nodes in flight and their copies overlap the others'
// passes.  beta_old is read once, by the write pass.  Global memory sees each
// input once and each output once.
//
// Per node (one warp):
//  A. copy G, V and the two fixing-mask rows; u = v - eta G replaces G
//     (J0 and J1 entries set to 0, so that every later pass sees only free
//     coordinates: 0 never exceeds a non-negative threshold, and the passes
//     need neither masks nor branches); J1 entries go to a short list
//     (index, u); each lane keeps its two largest free |u|.
//  B. the free |u| above a threshold tau are gathered (at most kCandCap) as
//     keys (|u| bits, complemented index) and ranked: the kbar best are the top
//     set (ties to the smaller index), the next one is the largest tail value.
//     tau comes from the node's previous step (7/8 of its kbar-th largest |u|;
//     the gathering then happens in pass A) when that gathers more than kbar
//     and at most kCandCap entries; else tau = the kbar-th largest of the 64
//     lane top-two values (at least kbar free |u| reach it) and one more pass
//     gathers.  If more than kCandCap qualify, kbar rounds of a warp argmax
//     over shared memory select the top set instead.
//  C. the top coordinates are set to 0 too; theta on the piece of f between
//     top entry points that holds the root, then Newton steps on it (f is
//     convex there), each a pass over the tail in shared memory.  The first
//     pass tests 0.97 times the node's previous threshold: if f > 0 there, the
//     root lies above it on the last piece and Newton starts there.  Else the
//     last piece is tested at its left end (with small c every entry point is
//     tiny and the root lies above all of them), else a binary search finds
//     the piece and Newton starts at its left end.  Every start is left of
//     the root, so the steps converge to it from below.
//  D. beta in shared memory (tail formula, 0 for the other entries, then the
//     top and J1 lists scattered in); one pass writes beta and
//     v' = beta + ((t-1)/t')(beta - beta_old) (and the tensor-core operand
//     copy of v') while summing the restart test <v - beta, beta - beta_old>;
//     if the test fires, v' = beta is written again (rare).
#include <float.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

constexpr int kCandCap = 128;
constexpr int kSMs = 152;
constexpr int kStreamMaxWarps = 16;
constexpr int kStreamMinWarps = 6;      // below this the CTA-per-node kernel is used
constexpr size_t kSmemPerSM = 227 * 1024;
// Hints carried from the previous step of the same node: the candidates are
// gathered during the first pass above this fraction of the last kbar-th
// largest free |u|, and Newton starts at this fraction of the last threshold
// (each only after a check that it is usable; otherwise the full search runs).
constexpr float kTauHint = 0.875f;
constexpr float kThetaHint = 0.97f;

struct WarpHdr {
    unsigned long long cand[kCandCap];
    float sv[kMaxK];     // top magnitudes, descending
    float tu[kMaxK];     // their u (signed)
    int si[kMaxK];       // their coordinates (-1: an empty slot)
    float ep[kMaxK];     // entry points p(sv[i]), descending
    float j1u[kMaxK];
    int j1i[kMaxK];
    int ncand, nj1;
    float amax;
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
// a row of p floats padded to a multiple of 4 (the padding stays 0)
__host__ __device__ inline size_t row_bytes(int p) { return align16((size_t)p * sizeof(float)); }
__host__ __device__ inline size_t mask_bytes(int W) { return align16((size_t)W * sizeof(uint32_t)); }
// per warp: a header, then the rows of its node: two mask rows and the u (G) and
// v rows (beta_old is read from global memory by the write pass, its only use).
// A second row set, for the next node's rows to arrive during the current
// node's passes, halves the warps per SM at p = 2000 and slowed the kernel
// 2.3x: a node's passes are a chain of dependent shared-memory steps that
// other warps must cover.
__host__ __device__ inline size_t warp_bytes(int p, int W) {
    return align16(sizeof(WarpHdr)) + 2 * mask_bytes(W) + 2 * row_bytes(p);
}

__device__ __forceinline__ float entry_pt(float a, float c, float M) {
    return a <= (1.f + c) * M ? a * c / (1.f + c) : a - M;
}
__device__ __forceinline__ float model_root_f(float nt, float St, float nl, float Sl, float c, float M) {
    const float xa = c * (St + Sl) / (nt * (1.f + c) + c * nl);
    if (xa <= c * M) return xa;
    return (St + Sl - nt * M) / (nt + nl);
}
__device__ __forceinline__ float sgn_mag(float u, float mag) { return u < 0.f ? -mag : mag; }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Tensor-core operand copy of 4 consecutive values of v' (index i, a multiple of 4).
__device__ __forceinline__ void store_operand4(void* base, float* lo, size_t i, float4 v, int bf16) {
    if (bf16) {
        __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&h0);
        w.y = *reinterpret_cast<uint32_t*>(&h1);
        *reinterpret_cast<uint2*>(static_cast<__nv_bfloat16*>(base) + i) = w;
    } else {
        const float4 hi = make_float4(to_tf32(v.x), to_tf32(v.y), to_tf32(v.z), to_tf32(v.w));
        *reinterpret_cast<float4*>(static_cast<float*>(base) + i) = hi;
        if (lo)
            *reinterpret_cast<float4*>(lo + i) =
                make_float4(to_tf32(v.x - hi.x), to_tf32(v.y - hi.y), to_tf32(v.z - hi.z), to_tf32(v.w - hi.w));
    }
}

// Sum over the tail of (|u| - x)^+, four independent partial sums per lane.
__device__ __forceinline__ float tail_excess(const float4* su4, int p4, int lane, float x) {
    float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
    for (int q = lane; q < p4; q += 32) {
        const float4 s = su4[q];
        f0 += fmaxf(fabsf(s.x) - x, 0.f);
        f1 += fmaxf(fabsf(s.y) - x, 0.f);
        f2 += fmaxf(fabsf(s.z) - x, 0.f);
        f3 += fmaxf(fabsf(s.w) - x, 0.f);
    }
    return (f0 + f1) + (f2 + f3);
}

// Count and sum of the tail above x (entries at 0 never count for x >= 0).
__device__ __forceinline__ void tail_above(const float4* su4, int p4, int lane, float x, float& cnt, float& sum) {
    float n0 = 0.f, n1 = 0.f, s0 = 0.f, s1 = 0.f;
    for (int q = lane; q < p4; q += 32) {
        const float4 s = su4[q];
        const float a0 = fabsf(s.x), a1 = fabsf(s.y), a2 = fabsf(s.z), a3 = fabsf(s.w);
        n0 += (a0 > x ? 1.f : 0.f) + (a2 > x ? 1.f : 0.f);
        n1 += (a1 > x ? 1.f : 0.f) + (a3 > x ? 1.f : 0.f);
        s0 += (a0 > x ? a0 : 0.f) + (a2 > x ? a2 : 0.f);
        s1 += (a1 > x ? a1 : 0.f) + (a3 > x ? a3 : 0.f);
    }
    cnt = warp_sum(n0 + n1);
    sum = warp_sum(s0 + s1);
}

// VEC = 4: 16-byte copies and stores (p a multiple of 4, 16-byte aligned rows);
// VEC = 1: 4-byte ones.  Shared-memory passes use 16-byte accesses either way
// (the padded rows).
// Zero padding of a row set's rows past p (the passes read whole float4s).
__device__ __forceinline__ void stream_pad(unsigned char* rows, int p, int W, int lane) {
    float* su = reinterpret_cast<float*>(rows + 2 * mask_bytes(W));
    float* sv = su + row_bytes(p) / sizeof(float);
    const int p4 = (p + 3) >> 2;
    for (int j = p + lane; j < 4 * p4; j += 32) su[j] = sv[j] = 0.f;
    __syncwarp();
}

// A. node b's masks, G and V rows into the row set `rows` (asynchronous copies,
// one commit group).
template <int VEC>
__device__ __forceinline__ void stream_issue(const ProxArgs& a, int b, int lane, unsigned char* rows) {
    const int p = a.p, W = a.W, nq = p / VEC;
    uint32_t* smi = reinterpret_cast<uint32_t*>(rows);
    uint32_t* smo = reinterpret_cast<uint32_t*>(rows + mask_bytes(W));
    float* su = reinterpret_cast<float*>(rows + 2 * mask_bytes(W));
    float* sv = su + row_bytes(p) / sizeof(float);
    const size_t base = (size_t)b * p;
    const float* V = static_cast<const float*>(a.V) + base;
    const float* G0 = a.gsplits == 0 ? static_cast<const float*>(a.G) + base : a.Gpart + base;
    for (int q = lane; q < W; q += 32) {
        cp_async4(smi + q, a.in_mask + (size_t)b * W + q);
        cp_async4(smo + q, a.out_mask + (size_t)b * W + q);
    }
    for (int q = lane; q < nq; q += 32) {
        if constexpr (VEC == 4) {
            cp_async16(su + 4 * q, G0 + 4 * q);
            cp_async16(sv + 4 * q, V + 4 * q);
        } else {
            cp_async4(su + q, G0 + q);
            cp_async4(sv + q, V + q);
        }
    }
    cp_async_commit();
}

// B-E. node b of problem a by one warp: header h, its rows requested by
// stream_issue (the node's scalars are read while they arrive), laid out for
// a.p and a.W with the padding zeroed.
template <int VEC>
__device__ __forceinline__ void stream_node(const ProxArgs& a, int b, int lane, WarpHdr& h, unsigned char* rows) {
    const int p = a.p, p4 = (p + 3) >> 2, W = a.W;
    uint32_t* smi = reinterpret_cast<uint32_t*>(rows);
    uint32_t* smo = reinterpret_cast<uint32_t*>(rows + mask_bytes(W));
    float* su = reinterpret_cast<float*>(rows + 2 * mask_bytes(W));
    float* sv = su + row_bytes(p) / sizeof(float);
    float4* su4 = reinterpret_cast<float4*>(su);
    const float eta = (float)a.eta, c = (float)a.c, M = (float)a.M, c1 = 1.f + c;
    const int nq = p / VEC;
    {
        const size_t base = (size_t)b * p;
        float* __restrict__ V = static_cast<float*>(a.V) + base;
        float* __restrict__ Bm = static_cast<float*>(a.B) + base;
        const int kb = a.kbar[b], pf = a.pf[b];
        const double tprev = lane == 0 ? a.tmom[b] : 0.0;
        const bool sel = kb > 0 && pf > kb;         // a top set to select and a block to pool
        float tau_h = 0.f, th_h = 0.f;
        if (a.hint != nullptr && sel) { tau_h = a.hint[2 * b]; th_h = a.hint[2 * b + 1]; }
        const float tg = tau_h > 0.f ? tau_h * kTauHint : __builtin_huge_valf();

        if (lane == 0) { h.nj1 = 0; h.ncand = 0; }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        // u = v - eta G (split slices after the first are added from global memory, in
        // order); J0 entries become 0 now, J1 entries once they are listed below.
        // Two running top-two pairs (even and odd positions) keep the chains short.
        float t1 = 0.f, t2 = 0.f, t1b = 0.f, t2b = 0.f;
        for (int q = lane; q < p4; q += 32) {
            float4 g = su4[q];
            const float4 v = reinterpret_cast<const float4*>(sv)[q];
            const int j0 = 4 * q;
            for (int s = 1; s < a.gsplits; ++s) {
                const float* gs = a.Gpart + (size_t)s * a.gstride + base;
                g.x += gs[j0];
                if (j0 + 1 < p) g.y += gs[j0 + 1];
                if (j0 + 2 < p) g.z += gs[j0 + 2];
                if (j0 + 3 < p) g.w += gs[j0 + 3];
            }
            const uint32_t wi = smi[j0 >> 5] >> (j0 & 31), wo = smo[j0 >> 5] >> (j0 & 31);
            const float uu[4] = {v.x - eta * g.x, v.y - eta * g.y, v.z - eta * g.z, v.w - eta * g.w};
            float o[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool inb = j0 + t < p, out = (wo >> t) & 1u, fr = inb && !(((wi | wo) >> t) & 1u);
                const float au = fr ? fabsf(uu[t]) : 0.f;
                if (t & 1) { t2b = fmaxf(t2b, fminf(t1b, au)); t1b = fmaxf(t1b, au); }
                else { t2 = fmaxf(t2, fminf(t1, au)); t1 = fmaxf(t1, au); }
                if (au >= tg) {                        // candidate above the hinted threshold
                    const int qq = atomicAdd(&h.ncand, 1);
                    if (qq < kCandCap)
                        h.cand[qq] = ((unsigned long long)__float_as_uint(au) << 32) | (0xffffffffu - (uint32_t)(j0 + t));
                }
                o[t] = inb && !out ? uu[t] : 0.f;
            }
            su4[q] = make_float4(o[0], o[1], o[2], o[3]);
        }
        t2 = fmaxf(fminf(t1, t1b), fmaxf(t2, t2b));     // the lane's two largest
        t1 = fmaxf(t1, t1b);
        __syncwarp();
        // J1 (at most k entries): listed from the mask words, then set to 0
        for (int q = lane; q < W; q += 32) {
            uint32_t bits = smi[q];
            while (bits) {
                const int j = 32 * q + __ffs(bits) - 1;
                bits &= bits - 1;
                const int qq = atomicAdd(&h.nj1, 1);
                if (kglm_check(qq < kMaxK, a.chk, kChkProx)) {
                    const bool ok = kglm_check(j < p, a.chk, kChkProx);
                    h.j1i[qq] = ok ? j : -1;
                    h.j1u[qq] = ok ? su[j] : 0.f;
                    if (ok) su[j] = 0.f;
                }
            }
        }
        __syncwarp();

        // ---- B. top-kbar selection over the free coordinates
        float theta = 0.f;
        int ntop = 0;
        if (sel) {
            ntop = kb;
            // a top slot stays empty (si -1, value 0) only if fewer than kbar free
            // |u| are positive; an empty slot stands for a zero entry
            for (int i = lane; i < kb; i += 32) { h.si[i] = -1; h.sv[i] = 0.f; }
            __syncwarp();
            int total = h.ncand;
            float amax_lo = 0.f;
            if (!(tau_h > 0.f && total >= kb + 1 && total <= kCandCap)) {
            // no usable hint: tau from the lane top-two values, then a gathering pass
            if (lane == 0) h.ncand = 0;
            __syncwarp();
            uint32_t k0 = __float_as_uint(t1), k1 = __float_as_uint(t2);
            sort64(k0, k1, lane);
            const int pos = 64 - kb;                           // kb-th largest of 64 (kb <= kMaxK = 64)
            const uint32_t ka = __shfl_sync(0xffffffffu, k0, pos >> 1), kbk = __shfl_sync(0xffffffffu, k1, pos >> 1);
            const uint32_t tau = max((pos & 1) ? kbk : ka, 1u);
            float lo_max = 0.f;
            for (int q = lane; q < p4; q += 32) {
                const float4 s4 = su4[q];
                const float e[4] = {fabsf(s4.x), fabsf(s4.y), fabsf(s4.z), fabsf(s4.w)};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint32_t key = __float_as_uint(e[t]);
                    if (key >= tau) {
                        const int qq = atomicAdd(&h.ncand, 1);
                        if (qq < kCandCap)
                            h.cand[qq] = ((unsigned long long)key << 32) | (0xffffffffu - (uint32_t)(4 * q + t));
                    } else {
                        lo_max = fmaxf(lo_max, e[t]);
                    }
                }
            }
            __syncwarp();
            total = h.ncand;
            amax_lo = warp_max(lo_max);
            }
            if (total <= kCandCap) {
                for (int i = lane; i < total; i += 32) {
                    const unsigned long long ci = h.cand[i];
                    int r = 0;
                    for (int t = 0; t < total; ++t) r += h.cand[t] > ci;
                    const float val = __uint_as_float((uint32_t)(ci >> 32));
                    if (r < kb) {
                        h.sv[r] = val;
                        h.si[r] = (int)(0xffffffffu - (uint32_t)ci);
                    } else if (r == kb) {
                        h.amax = val;
                    }
                }
                __syncwarp();
                if (lane == 0 && total <= kb) h.amax = amax_lo;
            } else {
                // too many ties near tau: kb rounds of a warp argmax below the last winner
                unsigned long long last = ~0ull;
                for (int r = 0; r <= kb; ++r) {
                    unsigned long long best = 0ull;
                    for (int q = lane; q < p4; q += 32) {
                        const float4 s4 = su4[q];
                        const float e[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const unsigned long long pk = ((unsigned long long)__float_as_uint(fabsf(e[t])) << 32) |
                                                          (0xffffffffu - (uint32_t)(4 * q + t));
                            if (pk < last && pk > best) best = pk;
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
                        best = x > best ? x : best;
                    }
                    last = best;
                    if (lane == 0) {
                        const int j = (int)(0xffffffffu - (uint32_t)best);
                        if (r < kb) {
                            if (best != 0ull && j < p) {
                                h.sv[r] = __uint_as_float((uint32_t)(best >> 32));
                                h.si[r] = j;
                            }
                        } else {
                            h.amax = best ? __uint_as_float((uint32_t)(best >> 32)) : 0.f;
                        }
                    }
                }
                __syncwarp();
            }
            // ---- C. the top set leaves the tail (set to 0), then the pooled block's threshold
            for (int i = lane; i < kb; i += 32) {
                const int j = h.si[i];
                h.tu[i] = (unsigned)j < (unsigned)p ? su[j] : 0.f;
                h.ep[i] = entry_pt(h.sv[i], c, M);
            }
            __syncwarp();
            for (int i = lane; i < kb; i += 32)
                if ((unsigned)h.si[i] < (unsigned)p) su[h.si[i]] = 0.f;
            __syncwarp();
            const float amax = h.amax;
            if (amax > 0.f) {
                const float emin = h.ep[kb - 1];
                if (emin >= amax) {
                    theta = amax;                          // nothing pools
                } else {
                    int r = 0;
                    for (int i = 0; i < kb; ++i) r += h.ep[i] < amax;
                    auto xval = [&](int i) -> float { return i == 0 ? 0.f : (i <= r ? h.ep[kb - i] : amax); };
                    auto f_at = [&](int i) -> float {   // f at breakpoint i (one pass)
                        const float x = xval(i);
                        const float hx = x + fminf(x / c, M);
                        float f = tail_excess(su4, p4, lane, x);
                        if (lane < kb && h.ep[lane] < x) f -= fmaxf(hx - h.sv[lane], 0.f);
                        if (lane + 32 < kb && h.ep[lane + 32] < x) f -= fmaxf(hx - h.sv[lane + 32], 0.f);
                        return warp_sum(f);
                    };
                    // top part of f on the last piece (every entry point below amax counts)
                    auto top_last = [&](float x) -> float {
                        const float hx = x + fminf(x / c, M);
                        float f = 0.f;
                        if (lane < kb && h.ep[lane] < amax) f += fmaxf(hx - h.sv[lane], 0.f);
                        if (lane + 32 < kb && h.ep[lane + 32] < amax) f += fmaxf(hx - h.sv[lane + 32], 0.f);
                        return warp_sum(f);
                    };
                    const float xr = r > 0 ? h.ep[kb - r] : 0.f;   // the largest entry point below amax
                    int lo = 0, hi = r + 1;
                    float th = 0.f, nl = 0.f, Sl = 0.f;
                    bool started = false;
                    const float start = th_h * kThetaHint;
                    if (start > xr && start < amax) {
                        // the last step's threshold, lowered: if f > 0 there, the root is
                        // above it on the last piece and Newton can start there
                        tail_above(su4, p4, lane, start, nl, Sl);
                        if (Sl - start * nl - top_last(start) > 0.f) { lo = r; th = start; started = true; }
                    }
                    if (!started && r > 0) {
                        // f at the largest entry point below amax (one pass, also Newton's first)
                        tail_above(su4, p4, lane, xr, nl, Sl);
                        const float hx = xr + fminf(xr / c, M);
                        float tp = 0.f;
                        if (lane < kb && h.ep[lane] < xr) tp += fmaxf(hx - h.sv[lane], 0.f);
                        if (lane + 32 < kb && h.ep[lane + 32] < xr) tp += fmaxf(hx - h.sv[lane + 32], 0.f);
                        if (Sl - xr * nl - warp_sum(tp) > 0.f) { lo = r; th = xr; started = true; }
                        else hi = r;
                    }
                    if (!started) {
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (f_at(mid) > 0.f) lo = mid; else hi = mid;
                        }
                        th = xval(lo);
                        tail_above(su4, p4, lane, th, nl, Sl);
                    }
                    const float xlo = xval(lo), xhi = xval(hi);
                    float nt = 0.f, St = 0.f;
                    for (int i = 0; i < kb; ++i)
                        if (h.ep[i] <= xlo) { nt += 1.f; St += h.sv[i]; }
                    for (int it = 0; it < 4 * kMaxK + 64; ++it) {
                        float tn = model_root_f(nt, St, nl, Sl, c, M);
                        tn = fminf(fmaxf(tn, th), xhi);
                        float q0, q1;
                        tail_above(su4, p4, lane, tn, q0, q1);
                        const bool done = q0 == nl;
                        th = tn;
                        nl = q0;
                        Sl = q1;
                        if (done) break;
                    }
                    theta = th;
                }
            }
        }

        // ---- D. beta in shared memory, then the fused write / restart pass
        const bool ridge = kb > 0 && pf <= kb;      // every free coordinate fits the budget
        for (int q = lane; q < p4; q += 32) {
            const float4 s4 = su4[q];
            auto bf = [&](float u) -> float {
                const float au = fabsf(u);
                const float mag = kb == 0 ? 0.f : (ridge ? fminf(au / c1, M) : fmaxf(au - theta, 0.f));
                return sgn_mag(u, mag);
            };
            su4[q] = make_float4(bf(s4.x), bf(s4.y), bf(s4.z), bf(s4.w));
        }
        __syncwarp();
        for (int i = lane; i < ntop; i += 32) {       // top first: a J1 entry never loses to an empty slot
            const int j = h.si[i];
            if ((unsigned)j >= (unsigned)p) continue;
            const float u = h.tu[i], au = fabsf(u);
            su[j] = sgn_mag(u, fmaxf(fminf(fminf(au / c1, M), au - theta), 0.f));
        }
        __syncwarp();
        const int nj1 = min(h.nj1, kMaxK);
        for (int i = lane; i < nj1; i += 32) {
            const float u = h.j1u[i];
            const int j = h.j1i[i];
            if (kglm_check((unsigned)j < (unsigned)p, a.chk, kChkProx)) su[j] = sgn_mag(u, fminf(fabsf(u) / c1, M));
        }
        __syncwarp();
        double t_keep = 0.0, c_keep = 0.0;
        if (lane == 0) {
            t_keep = 0.5 * (1.0 + sqrt(1.0 + 4.0 * tprev * tprev));
            c_keep = (tprev - 1.0) / t_keep;
        }
        const float coef = (float)__shfl_sync(0xffffffffu, c_keep, 0);
        float d0 = 0.f, d1 = 0.f;
        const size_t ob = (size_t)b * a.op_ld;
        constexpr int UN = VEC == 4 ? 4 : 8;          // beta_old loads in flight per lane
        using VT = typename std::conditional<VEC == 4, float4, float>::type;
        for (int q0 = lane; q0 < nq; q0 += 32 * UN) {
            VT bo[UN];
#pragma unroll
            for (int r = 0; r < UN; ++r)
                if (q0 + 32 * r < nq) bo[r] = reinterpret_cast<const VT*>(Bm)[q0 + 32 * r];
#pragma unroll
            for (int r = 0; r < UN; ++r) {
                const int q = q0 + 32 * r;
                if (q >= nq) break;
                if constexpr (VEC == 4) {
                    const float4 v = reinterpret_cast<const float4*>(sv)[q];
                    const float4 bn = su4[q];
                    d0 += (v.x - bn.x) * (bn.x - bo[r].x) + (v.z - bn.z) * (bn.z - bo[r].z);
                    d1 += (v.y - bn.y) * (bn.y - bo[r].y) + (v.w - bn.w) * (bn.w - bo[r].w);
                    const float4 vn = make_float4(bn.x + coef * (bn.x - bo[r].x), bn.y + coef * (bn.y - bo[r].y),
                                                  bn.z + coef * (bn.z - bo[r].z), bn.w + coef * (bn.w - bo[r].w));
                    reinterpret_cast<float4*>(Bm)[q] = bn;
                    reinterpret_cast<float4*>(V)[q] = vn;
                    if (a.Vop != nullptr) store_operand4(a.Vop, a.Vop_lo, ob + 4 * q, vn, a.op_bf16);
                } else {
                    const float v = sv[q], bn = su[q];
                    d0 += (v - bn) * (bn - bo[r]);
                    const float vn = bn + coef * (bn - bo[r]);
                    Bm[q] = bn;
                    V[q] = vn;
                    if (a.Vop != nullptr) store_operand2(a.Vop, a.Vop_lo, ob + q, vn, a.op_bf16);
                }
            }
        }
        const float dot = warp_sum(d0 + d1);
        const bool rs = a.restart && dot > 0.f;
        if (lane == 0) {
            a.tmom[b] = rs ? 1.0 : t_keep;   // restart: start over from beta, t = 1
            if (a.hint != nullptr) {
                a.hint[2 * b] = sel ? h.sv[kb - 1] : 0.f;
                a.hint[2 * b + 1] = sel ? theta : 0.f;
            }
        }
        if (rs) {
            // momentum off: v' = beta
            for (int j = lane; j < p; j += 32) {
                const float bn = su[j];
                V[j] = bn;
                if (a.Vop != nullptr) store_operand2(a.Vop, a.Vop_lo, ob + j, bn, a.op_bf16);
            }
        }
        __syncwarp();
    }
}

template <int VEC>
__global__ void __launch_bounds__(32 * kStreamMaxWarps, 1) k_prox_stream(ProxArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    unsigned char* wbase = smem + (size_t)warp * warp_bytes(a.p, a.W);
    WarpHdr& h = *reinterpret_cast<WarpHdr*>(wbase);
    unsigned char* rows = wbase + align16(sizeof(WarpHdr));
    stream_pad(rows, a.p, a.W, lane);
    // nodes go round the CTAs first (node b to CTA b mod grid), so that every SM
    // holds the same number of nodes and a last partial round is spread over all
    // SMs rather than packed onto the first few
    for (int b = warp * gridDim.x + blockIdx.x; b < a.m; b += gridDim.x * wpc) {
        if (a.active != nullptr && a.active[b] == 0) continue;
        stream_issue<VEC>(a, b, lane, rows);
        stream_node<VEC>(a, b, lane, h, rows);
    }
}

// The nodes of several problems (instances of the serving loop) in one launch:
// node t < total belongs to the problem pi with nbase[pi] <= t < nbase[pi + 1];
// every warp's region is sized for the largest p and W and laid out anew (its
// padding zeroed) when the warp moves to another problem.
template <int VEC>
__global__ void __launch_bounds__(32 * kStreamMaxWarps, 1) k_prox_stream_group(const __grid_constant__ ProxGroup g) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpc = blockDim.x >> 5;
    unsigned char* wbase = smem + (size_t)warp * warp_bytes(g.pmax, g.Wmax);
    WarpHdr& h = *reinterpret_cast<WarpHdr*>(wbase);
    unsigned char* rows = wbase + align16(sizeof(WarpHdr));
    int last = -1;
    for (int t = warp * gridDim.x + blockIdx.x; t < g.nbase[g.np]; t += gridDim.x * wpc) {
        int pi = 0;
        while (pi + 1 < g.np && t >= g.nbase[pi + 1]) ++pi;
        const ProxArgs& a = g.a[pi];
        const int b = t - g.nbase[pi];
        if (a.active != nullptr && a.active[b] == 0) continue;
        if (pi != last) {
            stream_pad(rows, a.p, a.W, lane);
            last = pi;
        }
        stream_issue<VEC>(a, b, lane, rows);
        stream_node<VEC>(a, b, lane, h, rows);
    }
}

template <int VEC>
int launch_stream(cudaStream_t s, const ProxArgs& a, int wpc) {
    const size_t smem = (size_t)wpc * warp_bytes(a.p, a.W);
    auto kern = k_prox_stream<VEC>;
    {
        // set once per kernel to the SM's whole shared memory, so that no launch
        // ever finds the opt-in below its need
        static std::mutex mu;
        static bool opted = false;
        std::lock_guard<std::mutex> lock(mu);
        if (!opted) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemPerSM) != cudaSuccess)
                return -1;
            opted = true;
        }
    }
    // a CTA per SM (its shared memory is the SM's); fewer nodes than SMs take one
    // SM each
    const int grid = std::max(1, std::min(kSMs, a.m));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(32 * wpc);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kern, a);   // errors surface at the caller's check
    return 0;
}

}  // namespace

int prox_stream_warps(int p, int W) {
    return (int)std::min<size_t>(kStreamMaxWarps, kSmemPerSM / warp_bytes(p, W));
}

namespace {
bool stream_vec_ok(const ProxArgs& a) {
    return (a.p % 4 == 0) && ((uintptr_t)a.V % 16 == 0) && ((uintptr_t)a.B % 16 == 0) &&
           (a.Vop == nullptr || (a.op_ld % 4 == 0 && (uintptr_t)a.Vop % 16 == 0 &&
                                 (a.Vop_lo == nullptr || (uintptr_t)a.Vop_lo % 16 == 0))) &&
           (a.gsplits == 0 ? ((uintptr_t)a.G % 16 == 0) : ((uintptr_t)a.Gpart % 16 == 0 && a.gstride % 4 == 0));
}

template <int VEC>
int launch_stream_group(cudaStream_t s, const ProxGroup& g, int wpc) {
    auto kern = k_prox_stream_group<VEC>;
    {
        static std::mutex mu;
        static bool opted = false;
        std::lock_guard<std::mutex> lock(mu);
        if (!opted) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemPerSM) != cudaSuccess)
                return -1;
            opted = true;
        }
    }
    const int total = g.nbase[g.np];
    const int grid = std::max(1, std::min(kSMs, total));
    kern<<<grid, 32 * wpc, (size_t)wpc * warp_bytes(g.pmax, g.Wmax), s>>>(g);
    return 0;
}
}  // namespace

int prox_stream_group(cudaStream_t s, ProxGroup& g) {
    if (g.np <= 0 || g.np > kGroupMax) return 1;
    g.pmax = 0;
    g.Wmax = 0;
    bool vec = true;
    g.nbase[0] = 0;
    for (int i = 0; i < g.np; ++i) {
        const ProxArgs& a = g.a[i];
        if (a.p > kStreamMaxP) return 1;
        g.pmax = std::max(g.pmax, a.p);
        g.Wmax = std::max(g.Wmax, a.W);
        vec = vec && stream_vec_ok(a);
        g.nbase[i + 1] = g.nbase[i] + std::max(0, a.m);
    }
    if (g.nbase[g.np] == 0) return 0;
    const int wpc = prox_stream_warps(g.pmax, g.Wmax);
    if (wpc < kStreamMinWarps) return 1;
    return vec ? launch_stream_group<4>(s, g, wpc) : launch_stream_group<1>(s, g, wpc);
}

int prox_stream_f32(cudaStream_t s, const ProxArgs& a) {
    if (a.m <= 0) return 0;
    const int wpc = prox_stream_warps(a.p, a.W);
    if (a.p > kStreamMaxP || wpc < kStreamMinWarps) return 1;     // not this kernel's range
    const bool vec = (a.p % 4 == 0) && ((uintptr_t)a.V % 16 == 0) && ((uintptr_t)a.B % 16 == 0) &&
                     (a.Vop == nullptr || (a.op_ld % 4 == 0 && (uintptr_t)a.Vop % 16 == 0 &&
                                           (a.Vop_lo == nullptr || (uintptr_t)a.Vop_lo % 16 == 0))) &&
                     (a.gsplits == 0 ? ((uintptr_t)a.G % 16 == 0)
                                     : ((uintptr_t)a.Gpart % 16 == 0 && a.gstride % 4 == 0));
    return vec ? launch_stream<4>(s, a, wpc) : launch_stream<1>(s, a, wpc);
}

}  // namespace kglm
