// Device-resident open-node queue for the hybrid loop of Fig. 1.
//
// The open nodes of a search live in device memory as a pool sorted by the
// key (parent bound, id): each entry holds its fixing masks (J1 then J0, W
// words each), the bound inherited from its parent, an id and the warm-start
// slot its parent's final beta was stored in (-1: cold start).  One round:
//   select  the first min(batch, N) entries are the best-bound batch (every
//           entry left in the pool is below the pruning threshold, so no test
//           is needed); their masks become the batch layout directly;
//   (the batch is evaluated by the engine)
//   update  the incumbent becomes the minimum of the batch's re-optimized
//           objectives (ties to the earlier node); slots of the evaluated
//           nodes are released; a node is closed when its bound reaches
//           UB - delta, it is a leaf (j* < 0) or its gap is within delta,
//           otherwise it branches on j* into (J0 + j*) and (J1 + j*) with ids
//           in batch order (the J0 child first) and both children warm-start
//           from one new slot holding the node's beta (while slots last);
//           the children are ranked by key and merged with the rest of the
//           pool into the other pool buffer, and entries at or above the
//           threshold are dropped (their slots released): the sorted pool
//           makes pruning a truncation.
// Keys are unique (ids are), so every merge position is taken exactly once.
// The order of evaluation, the incumbent updates and the children are those
// of the host queue (best bound, ties to the smaller id); a bound that is NaN
// is replaced by the parent's (never pruned on it).  Slot identities differ
// from the host loop's, slot availability does not: frees precede
// allocations in each round and both are counted in batch order.
#include <math.h>

#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

__device__ __forceinline__ bool key_less(double la, long long ia, double lb, long long ib) {
    return la < lb || (la == lb && ia < ib);
}

__device__ __forceinline__ double delta_dev(double ub, double gap_tol) {
    return isfinite(ub) ? gap_tol * fmax(1.0, fabs(ub)) : 0.0;
}

__device__ __forceinline__ void release_slot(int s, int nslots, int* sref, int* sfree, int* nfree) {
    if (s >= 0 && s < nslots && atomicSub(&sref[s], 1) == 1) sfree[atomicAdd(nfree, 1)] = s;
}

// entries [lo, hi) of the pool whose key is below (l, i)
__device__ __forceinline__ int pool_count_less(const double* lb, const long long* id, int lo, int hi, double l,
                                               long long i) {
    int a = lo, b = hi;
    while (a < b) {
        const int mid = (a + b) >> 1;
        if (key_less(lb[mid], id[mid], l, i)) a = mid + 1;
        else b = mid;
    }
    return a - lo;
}

// children (in key order through perm) whose key is below (l, i)
__device__ __forceinline__ int child_count_less(const double* clb, const long long* cid, const int* perm, int C,
                                                double l, long long i) {
    int a = 0, b = C;
    while (a < b) {
        const int mid = (a + b) >> 1;
        const int c = perm[mid];
        if (key_less(clb[c], cid[c], l, i)) a = mid + 1;
        else b = mid;
    }
    return a;
}

__global__ void k_dq_init(DqState* st, int nslots, int W, int k, double* lb, long long* id, int* slot,
                          uint32_t* mask, int* sref, int* sfree, int* best_sup, double* best_coef) {
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        sref[i] = 0;
        sfree[i] = nslots - 1 - i;                // slot 0 is handed out first
    }
    for (int w = threadIdx.x; w < 2 * W; w += blockDim.x) mask[w] = 0u;
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
        best_sup[r] = -1;
        best_coef[r] = 0.0;
    }
    if (threadIdx.x == 0) {
        lb[0] = -INFINITY;                        // the root
        id[0] = 0;
        slot[0] = -1;
        st->next_id = 1;
        st->id_base = 0;
        st->ub = INFINITY;
        st->sum_out = 0;
        st->N = 1;
        st->m = 0;
        st->nbranch = 0;
        st->nfree = nslots;
        st->nkeep = 1;
        st->overflow = 0;
    }
}

// the batch: the first min(batch, N) entries below the pruning threshold
__global__ void k_dq_select(DqState* st, int batch, const double* lb, double gap_tol) {
    if (threadIdx.x != 0) return;
    const double thr = st->ub - delta_dev(st->ub, gap_tol);
    int a = 0, b = st->N;
    while (a < b) {
        const int mid = (a + b) >> 1;
        if (lb[mid] < thr) a = mid + 1;
        else b = mid;
    }
    st->m = min(batch, a);
    st->sum_out = 0;
}

// batch row b = pool entry b: masks, kbar, pf, parent bound and slot
__global__ void k_dq_layout(DqState* st, int W, int p, int k, const double* lb, const int* slot,
                            const uint32_t* mask, uint32_t* in_mask, uint32_t* out_mask, int* kbar, int* pf,
                            double* lbp, int* bslot) {
    const int b = blockIdx.x;
    if (b >= st->m) return;
    __shared__ int red[2][32];
    int n1 = 0, n0 = 0;
    const uint32_t* src = mask + (size_t)b * 2 * W;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const uint32_t in = src[w], out = src[W + w];
        in_mask[(size_t)b * W + w] = in;
        out_mask[(size_t)b * W + w] = out;
        n1 += __popc(in);
        n0 += __popc(out);
    }
    n1 = warp_sum(n1);
    n0 = warp_sum(n0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { red[0][warp] = n1; red[1][warp] = n0; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s1 = 0, s0 = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { s1 += red[0][q]; s0 += red[1][q]; }
        kbar[b] = k - s1;
        pf[b] = p - s1 - s0;
        lbp[b] = lb[b];
        bslot[b] = slot[b];
        atomicAdd(reinterpret_cast<unsigned long long*>(&st->sum_out), (unsigned long long)s0);
    }
}

// incumbent: the smallest re-optimized objective of the batch, ties to the earlier node
__global__ void k_dq_incumbent(DqState* st, const double* ubc, const int* support, const double* beta_re, int k,
                               int* best_sup, double* best_coef) {
    __shared__ double sv[32];
    __shared__ int sb[32];
    __shared__ int win;
    const int m = st->m;
    double v = INFINITY;
    int bi = 0x7fffffff;
    for (int b = threadIdx.x; b < m; b += blockDim.x)
        if (ubc[b] < v) { v = ubc[b]; bi = b; }      // ascending b per thread: the first minimum
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double xv = __shfl_xor_sync(0xffffffffu, v, o);
        const int xb = __shfl_xor_sync(0xffffffffu, bi, o);
        if (xv < v || (xv == v && xb < bi)) { v = xv; bi = xb; }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { sv[warp] = v; sb[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            if (sv[q] < sv[0] || (sv[q] == sv[0] && sb[q] < sb[0])) { sv[0] = sv[q]; sb[0] = sb[q]; }
        win = -1;
        if (sv[0] < st->ub) {
            st->ub = sv[0];
            win = sb[0];
        }
    }
    __syncthreads();
    if (win >= 0)
        for (int r = threadIdx.x; r < k; r += blockDim.x) {
            best_sup[r] = support[(size_t)win * k + r];
            best_coef[r] = beta_re[(size_t)win * k + r];
        }
}

// close or branch every batch node (one CTA): slots of the batch released, then
// the branching nodes ranked in batch order and given new slots while they last
__global__ void k_dq_branch(DqState* st, const double* lb_best, double* lbp, const int* jstar, const double* ubc,
                            const int* bslot, int* sref, int* sfree, int nslots, double gap_tol, int* brank,
                            int* cslot_b) {
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int m = st->m;
    for (int b = threadIdx.x; b < m; b += blockDim.x) release_slot(bslot[b], nslots, sref, sfree, &st->nfree);
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    const double ub = st->ub, d = delta_dev(ub, gap_tol);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < m; base += blockDim.x) {
        const int b = base + threadIdx.x;
        bool f = false;
        if (b < m) {
            double lbb = lb_best[b] < lbp[b] ? lbp[b] : lb_best[b];
            if (isnan(lbb)) lbb = lbp[b];
            lbp[b] = lbb;                                    // the children's bound
            f = !(lbb >= ub - d || jstar[b] < 0 || ubc[b] - lbb <= d);
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        int before = carry_s;
        for (int q = 0; q < warp; ++q) before += wsum[q];
        before += __popc(bal & ((1u << lane) - 1u));
        if (b < m) brank[b] = f ? before : -1;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int q = 0; q < nw; ++q) t += wsum[q];
            carry_s += t;
        }
        __syncthreads();
    }
    // the count was moved by atomics above: read it at L2, past any stale L1 copy of the state's line
    const int T = carry_s, nf = atomicAdd(&st->nfree, 0);
    for (int b = threadIdx.x; b < m; b += blockDim.x) {
        const int r = brank[b];
        if (r < 0) continue;
        const int s = r < nf ? sfree[nf - 1 - r] : -1;
        if (s >= 0) sref[s] = 2;
        cslot_b[b] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->nfree = nf - min(T, nf);
        st->nbranch = T;
        st->id_base = st->next_id;
        st->next_id += 2LL * T;
    }
}

// the two children of a branching batch node b (J0 + j* first), and its beta into their slot
template <typename T>
__global__ void k_dq_children(const DqState* st, int W, int p, const uint32_t* in_mask, const uint32_t* out_mask,
                              const int* jstar, const int* brank, const double* lbb, const int* cslot_b, const T* B,
                              T* pool, double* clb, long long* cid, int* cslot, uint32_t* cmask) {
    const int b = blockIdx.x;
    if (b >= st->m) return;
    const int r = brank[b];
    if (r < 0) return;
    const int j = jstar[b], s = cslot_b[b];
    const int jw = j >> 5;
    const uint32_t bit = 1u << (j & 31);
    uint32_t* c0 = cmask + (size_t)(2 * r) * 2 * W;
    uint32_t* c1 = c0 + 2 * W;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const uint32_t in = in_mask[(size_t)b * W + w], out = out_mask[(size_t)b * W + w];
        c0[w] = in;
        c0[W + w] = out | (w == jw ? bit : 0u);
        c1[w] = in | (w == jw ? bit : 0u);
        c1[W + w] = out;
    }
    if (threadIdx.x == 0) {
        const long long id0 = st->id_base + 2LL * r;
        clb[2 * r] = lbb[b];
        clb[2 * r + 1] = lbb[b];
        cid[2 * r] = id0;
        cid[2 * r + 1] = id0 + 1;
        cslot[2 * r] = s;
        cslot[2 * r + 1] = s;
    }
    if (s >= 0)
        for (int q = threadIdx.x; q < p; q += blockDim.x) pool[(size_t)s * p + q] = B[(size_t)b * p + q];
}

// children in key order: perm[rank] = child
__global__ void k_dq_rank(const DqState* st, const double* clb, const long long* cid, int* perm) {
    __shared__ double tl[256];
    __shared__ long long ti[256];
    const int C = 2 * st->nbranch;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool mine = i < C;
    const double l = mine ? clb[i] : 0.0;
    const long long id = mine ? cid[i] : 0;
    int rank = 0;
    for (int t0 = 0; t0 < C; t0 += 256) {
        __syncthreads();
        if (t0 + (int)threadIdx.x < C) {
            tl[threadIdx.x] = clb[t0 + threadIdx.x];
            ti[threadIdx.x] = cid[t0 + threadIdx.x];
        }
        __syncthreads();
        const int n = min(256, C - t0);
        if (mine)
            for (int q = 0; q < n; ++q) rank += key_less(tl[q], ti[q], l, id);
    }
    if (mine) perm[rank] = i;
}

// how many entries of the merged pool stay: keys below the pruning threshold
__global__ void k_dq_keep(DqState* st, const double* lb, const double* clb, const int* perm, int cap,
                          double gap_tol) {
    if (threadIdx.x != 0) return;
    const double thr = st->ub - delta_dev(st->ub, gap_tol);
    int a = st->m, b = st->N;
    while (a < b) {
        const int mid = (a + b) >> 1;
        if (lb[mid] < thr) a = mid + 1;
        else b = mid;
    }
    const int kr = a - st->m;
    const int C = 2 * st->nbranch;
    int u = 0, v = C;
    while (u < v) {
        const int mid = (u + v) >> 1;
        if (clb[perm[mid]] < thr) u = mid + 1;
        else v = mid;
    }
    st->nkeep = kr + u;
    st->overflow = kr + u > cap ? 1 : 0;
}

// the merge of the rest of the pool [m, N) and the sorted children into the
// other pool buffer (a warp per entry); entries past the kept count release
// their slots
__global__ void k_dq_merge(DqState* st, int W, int cap, int nslots, const double* lb, const long long* id,
                           const int* slot, const uint32_t* mask, const double* clb, const long long* cid,
                           const int* cslot, const uint32_t* cmask, const int* perm, double* lb2, long long* id2,
                           int* slot2, uint32_t* mask2, int* sref, int* sfree) {
    const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int m = st->m, N = st->N, C = 2 * st->nbranch, NR = N - m;
    if (e >= NR + C) return;
    double l;
    long long key_id;
    int s, pos;
    const uint32_t* src;
    if (e < NR) {
        const int i = m + e;
        l = lb[i];
        key_id = id[i];
        s = slot[i];
        src = mask + (size_t)i * 2 * W;
        pos = e + child_count_less(clb, cid, perm, C, l, key_id);
    } else {
        const int r = e - NR, c = perm[r];
        l = clb[c];
        key_id = cid[c];
        s = cslot[c];
        src = cmask + (size_t)c * 2 * W;
        pos = r + pool_count_less(lb, id, m, N, l, key_id);
    }
    const int lim = min(st->nkeep, cap);
    if (pos < lim) {
        uint32_t* dst = mask2 + (size_t)pos * 2 * W;
        for (int w = lane; w < 2 * W; w += 32) dst[w] = src[w];
        if (lane == 0) {
            lb2[pos] = l;
            id2[pos] = key_id;
            slot2[pos] = s;
        }
    } else if (lane == 0) {
        release_slot(s, nslots, sref, sfree, &st->nfree);
    }
}

__global__ void k_dq_finish(DqState* st, int cap) {
    if (threadIdx.x == 0) st->N = min(st->nkeep, cap);
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

void dq_init(cudaStream_t s, DevQueue& q) {
    q.cur = 0;
    k_dq_init<<<1, 256, 0, s>>>(q.st, q.nslots, q.W, q.k, q.lb[0], q.id[0], q.slot[0], q.mask[0], q.sref, q.sfree,
                                q.best_sup, q.best_coef);
}

void dq_select(cudaStream_t s, DevQueue& q, int batch, double gap_tol, uint32_t* in_mask, uint32_t* out_mask,
               int* kbar, int* pf) {
    const int c = q.cur;
    k_dq_select<<<1, 32, 0, s>>>(q.st, batch, q.lb[c], gap_tol);
    k_dq_layout<<<batch, 64, 0, s>>>(q.st, q.W, q.p, q.k, q.lb[c], q.slot[c], q.mask[c], in_mask, out_mask, kbar, pf,
                                    q.lbp, q.bslot);
}

void dq_update(cudaStream_t s, DevQueue& q, int m, int N, double gap_tol, const double* lb_best, const double* ubc,
               const int* jstar, const int* support, const double* beta_re, const uint32_t* in_mask,
               const uint32_t* out_mask, const void* B, int is_f64, void* pool) {
    const int c = q.cur, o = c ^ 1;
    k_dq_incumbent<<<1, 1024, 0, s>>>(q.st, ubc, support, beta_re, q.k, q.best_sup, q.best_coef);
    k_dq_branch<<<1, 1024, 0, s>>>(q.st, lb_best, q.lbp, jstar, ubc, q.bslot, q.sref, q.sfree, q.nslots, gap_tol,
                                   q.brank, q.cslot_b);
    if (is_f64)
        k_dq_children<double><<<m, 128, 0, s>>>(q.st, q.W, q.p, in_mask, out_mask, jstar, q.brank, q.lbp, q.cslot_b,
                                                static_cast<const double*>(B), static_cast<double*>(pool), q.clb,
                                                q.cid, q.cslot, q.cmask);
    else
        k_dq_children<float><<<m, 128, 0, s>>>(q.st, q.W, q.p, in_mask, out_mask, jstar, q.brank, q.lbp, q.cslot_b,
                                               static_cast<const float*>(B), static_cast<float*>(pool), q.clb, q.cid,
                                               q.cslot, q.cmask);
    k_dq_rank<<<nblk(2 * (size_t)m, 256), 256, 0, s>>>(q.st, q.clb, q.cid, q.cperm);
    k_dq_keep<<<1, 32, 0, s>>>(q.st, q.lb[c], q.clb, q.cperm, q.cap, gap_tol);
    const size_t E = (size_t)(N - m) + 2 * (size_t)m;   // at most: the rest of the pool and two children per node
    if (E > 0)
        k_dq_merge<<<nblk(E * 32, 256), 256, 0, s>>>(q.st, q.W, q.cap, q.nslots, q.lb[c], q.id[c], q.slot[c],
                                                     q.mask[c], q.clb, q.cid, q.cslot, q.cmask, q.cperm, q.lb[o],
                                                     q.id[o], q.slot[o], q.mask[o], q.sref, q.sfree);
    k_dq_finish<<<1, 32, 0, s>>>(q.st, q.cap);
    q.cur = o;
}

}  // namespace kglm
