// Device helpers of the node-bound engine: GLM loss functions, CTA-wide
// reductions and the CTA top-k selection that replaces the padded column sort
// of §4.2 (Fig. 2): a radix select of the k-th largest key among a node's free
// coordinates, ties broken by the smaller coordinate index.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

namespace kglm {

constexpr int kLSQ = 0;
constexpr int kLOGISTIC = 1;
constexpr int kMaxK = 64;

// ------------------------------------------------------------------ bounds-checked build
// Compiled with KGLM_CHECKS=1 (libkglm_checks.so), the kernels check the indices
// they write or gather with (J1 and top-set lists, supports) before using them: a
// failed check sets its kernel's bit in the context's error word and the access is
// skipped, and the evaluation that launched the kernel returns KGLM_EINVAL.  In the
// normal build the condition is taken as true (the inputs are validated on the
// host or by the push's device checks) and the guard compiles to nothing.
#ifndef KGLM_CHECKS
#define KGLM_CHECKS 0
#endif
constexpr int kChkProx = 1 << 16, kChkCert = 1 << 17, kChkReopt = 1 << 18, kChkSelf = 1 << 19;
constexpr int kChkAll = kChkProx | kChkCert | kChkReopt | kChkSelf;
__device__ __forceinline__ bool kglm_check(bool cond, int* word, int bit) {
#if KGLM_CHECKS
    if (!cond) {
        if (word) atomicOr(word, bit);
        return false;
    }
#else
    (void)cond; (void)word; (void)bit;
#endif
    return true;
}

// ------------------------------------------------------------------ losses
// l(s, y) = (s - y)^2 or log(1 + exp(-y s)); dl/ds; l*(w, y)   (§4.2, §4.4)

__device__ __forceinline__ float dloss(float s, float y, int kind) {
    return kind == kLSQ ? 2.0f * (s - y) : -y / (1.0f + expf(y * s));
}
__device__ __forceinline__ double dloss(double s, double y, int kind) {
    return kind == kLSQ ? 2.0 * (s - y) : -y / (1.0 + exp(y * s));
}

__device__ __forceinline__ double softplus(double t) {   // log(1 + e^t), no overflow
    return t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t));
}

__device__ __forceinline__ double loss64(double s, double y, int kind) {
    if (kind == kLSQ) { double r = s - y; return r * r; }
    return softplus(-y * s);
}

__device__ __forceinline__ double xlogx(double a) { return a > 0.0 ? a * log(a) : 0.0; }

// l*(w, y): least squares w*y + w^2/4; logistic a ln a + (1-a) ln(1-a), a = -w*y
// clamped into [0, 1] (the dual point is built inside the domain).
__device__ __forceinline__ double loss_conj64(double w, double y, int kind) {
    if (kind == kLSQ) return w * y + 0.25 * w * w;
    double a = fmin(1.0, fmax(0.0, -w * y));
    return xlogx(a) + xlogx(1.0 - a);
}

// Huber H_M (§3 Eq. (prelim_node_conjugate)).
__device__ __forceinline__ double huber64(double q, double M) {
    double a = fabs(q);
    return a <= M ? 0.5 * a * a : M * a - 0.5 * M * M;
}

// Bitonic sort (ascending) of 64 keys held two per lane (element 2*lane + s).
template <typename T>
__device__ __forceinline__ void sort64(T& k0, T& k1, int lane) {
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 1) {
                const int g = 2 * lane;                  // pair (g, g+1) in this lane
                const bool asc = (g & k) == 0;
                const T lo = k0 < k1 ? k0 : k1, hi = k0 < k1 ? k1 : k0;
                k0 = asc ? lo : hi;
                k1 = asc ? hi : lo;
            } else {
                const int lj = j >> 1;                   // partner lane
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    T& x = s ? k1 : k0;
                    const T o = __shfl_xor_sync(0xffffffffu, x, lj);
                    const int g = 2 * lane + s;
                    const bool asc = (g & k) == 0, lower = (g & j) == 0;
                    x = (asc == lower) ? (x < o ? x : o) : (x < o ? o : x);
                }
            }
        }
    }
}

// FP32 rounded to the nearest TF32 value (low 13 mantissa bits cleared).
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Store of a tensor-core operand: BF16 or TF32 (in an FP32 word).
__device__ __forceinline__ void store_operand(void* base, size_t i, float v, int bf16) {
    if (bf16) static_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16(v);
    else static_cast<float*>(base)[i] = to_tf32(v);
}
// Operand copy of v for the tensor-core products; with lo != NULL (TF32 only)
// also the TF32 low part v - hi, so that hi + lo carries v to ~22 bits.
__device__ __forceinline__ void store_operand2(void* base, float* lo, size_t i, float v, int bf16) {
    if (bf16) {
        static_cast<__nv_bfloat16*>(base)[i] = __float2bfloat16(v);
    } else {
        const float h = to_tf32(v);
        static_cast<float*>(base)[i] = h;
        if (lo) lo[i] = to_tf32(v - h);
    }
}

// ------------------------------------------------------------------ reductions

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum of NV values over the CTA; every thread gets the totals, summed in a
// fixed order (deterministic).  red: shared scratch of NV * (NT/32) entries.
template <int NT, int NV, typename T>
__device__ __forceinline__ void block_sum(T (&v)[NV], T* red) {
    constexpr int NW = NT / 32;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) red[q * NW + (threadIdx.x >> 5)] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        T s = T(0);
#pragma unroll
        for (int w = 0; w < NW; ++w) s += red[q * NW + w];
        v[q] = s;
    }
}

template <int NT, typename T>
__device__ __forceinline__ T block_max(T v, T* red) {
    constexpr int NW = NT / 32;
    v = warp_max(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = red[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) s = max(s, red[w]);
    return s;
}

template <int NT>
__device__ __forceinline__ int block_count(int v, int* red) {
    int a[1] = {v};
    block_sum<NT, 1, int>(a, red);
    return a[0];
}

// ------------------------------------------------------------------ groups
// A per-node kernel is written once over a group policy: a CTA of NT threads
// (one node per CTA) or one warp (one node per warp).  Reductions give every
// member the total, summed in a fixed order.

template <int NT>
struct CtaGroup {
    static constexpr int N = NT;
    __device__ static int rank() { return threadIdx.x; }
    __device__ static void sync() { __syncthreads(); }
    __device__ static bool first_warp() { return threadIdx.x < 32; }
    template <int NV, typename T>
    __device__ static void sum(T (&v)[NV], T* red) { block_sum<NT, NV, T>(v, red); }
    template <typename T>
    __device__ static T max(T v, T* red) { return block_max<NT, T>(v, red); }
    __device__ static int count(int v, int* red) { return block_count<NT>(v, red); }
};

struct WarpGroup {
    static constexpr int N = 32;
    __device__ static int rank() { return threadIdx.x & 31; }
    __device__ static void sync() { __syncwarp(); }
    __device__ static bool first_warp() { return true; }
    template <int NV, typename T>
    __device__ static void sum(T (&v)[NV], T*) {
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    }
    template <typename T>
    __device__ static T max(T v, T*) { return warp_max(v); }
    __device__ static int count(int v, int*) { return warp_sum(v); }
};

// ------------------------------------------------------------------ selection

// Order-preserving unsigned key of a non-negative float / double magnitude.
__device__ __forceinline__ uint32_t mag_key(float a) { return __float_as_uint(a); }
__device__ __forceinline__ unsigned long long mag_key(double a) {
    return (unsigned long long)__double_as_longlong(a);
}

struct SelectShared {
    unsigned hist[256];
    int digit;
    unsigned above;
    unsigned bincnt;                  // elements in the chosen bin
    int ncand;                        // early exit: candidates gathered
    int need;
    unsigned long long thr;
    unsigned long long ckey[64];
};

// Radix select over the CTA: the kth (1-based) largest key among the elements
// whose bit is set in `valid`.  Returns the key and `need`, the number of
// elements equal to it that belong to the kth largest.  Requires 1 <= kth <=
// number of valid elements.  Once the bin holding the kth key has at most 64
// elements, they are gathered to shared memory and ranked there by one warp
// (the remaining 8-bit passes would only split that bin further).
template <typename G, int E, typename K>
__device__ void group_kth_largest(const K (&key)[E], uint32_t valid, int kth, SelectShared& sh,
                                  K& thr, int& need) {
    constexpr int BITS = int(sizeof(K)) * 8;
    K prefix = 0, pmask = 0;
    int rem = kth;
#pragma unroll 1
    for (int shift = BITS - 8; shift >= 0; shift -= 8) {
        G::sync();
        for (int i = G::rank(); i < 256; i += G::N) sh.hist[i] = 0u;
        G::sync();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            // warp-aggregated: lanes hitting the same bin add once (magnitudes
            // mostly share their exponent byte, so the first passes collide)
            const bool in = ((valid >> e) & 1u) && (key[e] & pmask) == prefix;
            const unsigned bin = in ? ((unsigned)(key[e] >> shift) & 255u) : 256u;
            const unsigned same = __match_any_sync(0xffffffffu, bin);
            if (in && (threadIdx.x & 31) == (unsigned)(__ffs(same) - 1)) atomicAdd(&sh.hist[bin], (unsigned)__popc(same));
        }
        G::sync();
        if (G::rank() < 32) {
            const int l = G::rank();
            unsigned c[8], tot = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) { c[q] = sh.hist[l * 8 + q]; tot += c[q]; }
            unsigned incl = tot;   // sum over lanes >= l (higher digits)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned x = __shfl_down_sync(0xffffffffu, incl, o);
                if (l + o < 32) incl += x;
            }
            unsigned above = incl - tot;
            if (above < (unsigned)rem && (unsigned)rem <= incl) {
                unsigned acc = above;
#pragma unroll
                for (int q = 7; q >= 0; --q) {
                    if (acc + c[q] >= (unsigned)rem) {
                        sh.digit = l * 8 + q;
                        sh.above = acc;
                        sh.bincnt = c[q];
                        break;
                    }
                    acc += c[q];
                }
            }
            if (l == 0) sh.ncand = 0;
        }
        G::sync();
        rem -= (int)sh.above;
        prefix |= K(sh.digit) << shift;
        pmask |= K(255) << shift;
        if (shift > 0 && sh.bincnt <= 64u) {
            // gather the bin's elements, then rank them in one warp
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (((valid >> e) & 1u) && (key[e] & pmask) == prefix) sh.ckey[atomicAdd(&sh.ncand, 1)] = key[e];
            G::sync();
            if (G::rank() < 32) {
                const int nc = sh.ncand, l = G::rank();
                for (int i = l; i < nc; i += 32) {
                    const unsigned long long ki = sh.ckey[i];
                    int gt = 0, eq = 0;
                    for (int j = 0; j < nc; ++j) {
                        gt += sh.ckey[j] > ki;
                        eq += sh.ckey[j] == ki;
                    }
                    if (gt <= rem - 1 && rem - 1 < gt + eq) {   // ki is the rem-th largest
                        sh.thr = ki;
                        sh.need = rem - gt;
                    }
                }
            }
            G::sync();
            thr = K(sh.thr);
            need = sh.need;
            return;
        }
    }
    G::sync();
    thr = prefix;
    need = rem;
}

template <int NT, int E, typename K>
__device__ void block_kth_largest(const K (&key)[E], uint32_t valid, int kth, SelectShared& sh,
                                  K& thr, int& need) {
    group_kth_largest<CtaGroup<NT>, E, K>(key, valid, kth, sh, thr, need);
}

// Selection of the kth largest keys with ties to the smaller index.  Element
// e of thread t is coordinate j = t + e*NT.  On return sel has bit e set for
// the selected elements (exactly kth of them).
template <typename G, int E, typename K>
__device__ uint32_t group_topk_select(const K (&key)[E], uint32_t valid, int kth, SelectShared& sh,
                                      int* ired) {
    K thr;
    int need;
    group_kth_largest<G, E, K>(key, valid, kth, sh, thr, need);
    uint32_t gt = 0, eq = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if ((valid >> e) & 1u) {
            if (key[e] > thr) gt |= 1u << e;
            else if (key[e] == thr) eq |= 1u << e;
        }
    }
    int n_eq = G::count(__popc(eq), ired);
    if (n_eq == need) return gt | eq;
    // ties straddle the threshold: take the `need` smallest indices among them
    uint32_t ikey[E];
#pragma unroll
    for (int e = 0; e < E; ++e) ikey[e] = ~(uint32_t)(G::rank() + e * G::N);
    uint32_t ithr;
    int ineed;
    group_kth_largest<G, E, uint32_t>(ikey, eq, need, sh, ithr, ineed);
    uint32_t take = 0;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (((eq >> e) & 1u) && ikey[e] >= ithr) take |= 1u << e;
    return gt | take;
}

// Bit e of a per-thread element mask (E <= 64 elements per thread).
template <int E>
using ElemMask = typename std::conditional<(E > 32), unsigned long long, uint32_t>::type;
template <typename Mk>
__device__ __forceinline__ bool bit(Mk m, int e) { return (m >> e) & Mk(1); }

// Warp tournament: the kth largest of |val| over the valid elements of the
// warp, ties to the smaller index (element e of lane l is index l + 32e), in
// kth rounds of a warp-wide argmax over each lane's best untaken element.
// Writes the selection sorted (magnitude descending) to sv/si (lane 0) and
// returns the lane's mask of selected elements.
template <int E, typename T, typename Mk>
__device__ Mk warp_topk_tournament(const T (&val)[E], Mk valid, int kth, T* sv, int* si) {
    const int lane = threadIdx.x & 31;
    Mk taken = 0;
    if constexpr (sizeof(T) == 4) {
        // FP32: the bits of a non-negative float order like the value, so a round is
        // two warp reductions (redux.sync): the largest magnitude, then the smallest
        // index holding it.  A lane with nothing left offers key 0 with an index
        // above every coordinate, so it never wins against a valid element.
        for (int r = 0; r < kth; ++r) {
            unsigned bkey = 0u, bidx = 0x7fffffffu;
            int be = -1;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (bit(valid & ~taken, e)) {
                    const unsigned k = __float_as_uint(fabsf(val[e]));
                    if (be < 0 || k > bkey) { bkey = k; bidx = (unsigned)(lane + 32 * e); be = e; }
                }
            const unsigned wk = __reduce_max_sync(0xffffffffu, bkey);
            const unsigned wi = __reduce_min_sync(0xffffffffu, bkey == wk ? bidx : 0x7fffffffu);
            if (be >= 0 && bidx == wi) taken |= Mk(1) << be;
            if (lane == 0) { sv[r] = __uint_as_float(wk); si[r] = (int)wi; }
        }
        __syncwarp();
        return taken;
    }
    for (int r = 0; r < kth; ++r) {
        T best = T(-1);
        int bidx = 0x7fffffff, be = -1;
#pragma unroll
        for (int e = 0; e < E; ++e)
            if (bit(valid & ~taken, e)) {
                const int idx = lane + 32 * e;
                const T x = abs(val[e]);
                if (x > best || (x == best && idx < bidx)) { best = x; bidx = idx; be = e; }
            }
        T wv = best;
        int wi = bidx;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(0xffffffffu, wv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, wi, o);
            if (ov > wv || (ov == wv && oi < wi)) { wv = ov; wi = oi; }
        }
        if (be >= 0 && bidx == wi) taken |= Mk(1) << be;
        if (lane == 0) { sv[r] = wv; si[r] = wi; }
    }
    __syncwarp();
    return taken;
}

// FP32 warp selection by candidates: tau = the kth largest of the 32 lane
// maxima (kth lanes each hold an element >= tau, so at least kth elements
// qualify); when at most 64 elements are >= tau they are ranked in shared
// memory (cbuf, 64 entries: key above, complemented index below, so that the
// order of the packed words is magnitude descending, index ascending),
// otherwise the tournament runs.  Same result, order and tie rule as the
// tournament; writes sv/si (kth entries) and returns the lane's mask.
template <int E, typename Mk>
__device__ Mk warp_topk_candidates(const float (&val)[E], Mk valid, int kth, float* sv, int* si,
                                   unsigned long long* cbuf) {
    const int lane = threadIdx.x & 31;
    if (kth > 32) return warp_topk_tournament<E, float, Mk>(val, valid, kth, sv, si);
    // keys are recomputed where needed (one instruction) rather than held
    auto key = [&](int e) { return __float_as_uint(fabsf(val[e])); };
    unsigned lm = 0u;   // an empty lane offers 0, at or below every valid key
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (bit(valid, e)) lm = max(lm, key(e));
    // bitonic sort of the lane maxima, ascending over the lanes
    unsigned x = lm;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned o = __shfl_xor_sync(0xffffffffu, x, j);
            x = (((lane & j) == 0) == ((lane & k) == 0)) ? min(x, o) : max(x, o);
        }
    const unsigned tau = __shfl_sync(0xffffffffu, x, 32 - kth);
    int cnt = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) cnt += (bit(valid, e) && key(e) >= tau) ? 1 : 0;
    const int total = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
    if (total > 64) return warp_topk_tournament<E, float, Mk>(val, valid, kth, sv, si);
    int incl = cnt;   // inclusive prefix over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    int pos = incl - cnt;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (bit(valid, e) && key(e) >= tau)
            cbuf[pos++] = ((unsigned long long)key(e) << 32) | (unsigned long long)(0xffffffffu - (unsigned)(lane + 32 * e));
    __syncwarp();
    for (int i = lane; i < total; i += 32) {
        const unsigned long long ci = cbuf[i];
        int r = 0;
        for (int t = 0; t < total; ++t) r += cbuf[t] > ci;
        if (r < kth) {
            sv[r] = __uint_as_float((unsigned)(ci >> 32));
            si[r] = (int)(0xffffffffu - (unsigned)ci);
        }
    }
    __syncwarp();
    const unsigned thk = __float_as_uint(sv[kth - 1]);
    const int thi = si[kth - 1];
    Mk sel = 0;
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (bit(valid, e) && (key(e) > thk || (key(e) == thk && lane + 32 * e <= thi))) sel |= Mk(1) << e;
    __syncwarp();
    return sel;
}

template <int NT, int E, typename K>
__device__ uint32_t block_topk_select(const K (&key)[E], uint32_t valid, int kth, SelectShared& sh,
                                      int* ired) {
    return group_topk_select<CtaGroup<NT>, E, K>(key, valid, kth, sh, ired);
}

// Sort up to kMaxK (value, index) pairs held in shared memory by value
// descending, index ascending; done by the group's first warp (the warp
// itself for a warp group).  out arrays must not alias in.
template <typename T, typename G = CtaGroup<64>>
__device__ void warp_rank_sort_desc(const T* val, const int* idx, int cnt, T* oval, int* oidx) {
    if (!G::first_warp()) return;
    for (int i = (threadIdx.x & 31); i < cnt; i += 32) {
        T v = val[i];
        int ix = idx[i];
        int r = 0;
        for (int j = 0; j < cnt; ++j) {
            T w = val[j];
            int jx = idx[j];
            r += (w > v) || (w == v && jx < ix);
        }
        oval[r] = v;
        oidx[r] = ix;
    }
}

}  // namespace kglm
