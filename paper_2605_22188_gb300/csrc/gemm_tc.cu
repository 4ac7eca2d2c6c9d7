// Tensor-core products of the BF16 and TF32 modes: S = X V (with the
// loss/link fused) and G = X^T R of §4.2 Eq. (gradient_matrix_form), and the
// digit products of the exact certificate, on the fifth-generation tensor
// cores of sm_103a.
//
// C[r][c] = sum_k A[r][k] B[c][k] with both operands K-contiguous.  The
// output is cut into 128 x BN tiles (BN <= 256, a multiple of 16) and,
// optionally, into K ranges (split-K slices or the jobs of the certificate):
// one work unit is one (tile, K range).  The kernel is persistent: one CTA per
// SM walks the units u = blockIdx.x, blockIdx.x + gridDim.x, ... with
//   warps 0 and 10,  TMA producers: 128-byte-swizzled K slices of A and B
//   lane 0           (cp.async.bulk.tensor.2d) into a ring of stages, warp 0
//                    filling the even stages and warp 10 the odd ones (one
//                    issuing thread takes a few hundred cycles per stage,
//                    small or large, and would leave the tensor pipe waiting);
//   warp 1, lane 0   MMA issuer: tcgen05.mma.cta_group::1 (kind::f16 with BF16
//                    operands, or kind::tf32) into one of two FP32
//                    accumulators in tensor memory (512 columns), so that the
//                    next unit's products run while the epilogue drains the
//                    last one; tcgen05.commit frees a stage / publishes an
//                    accumulator;
//   warps 2-9        epilogue: tcgen05.ld of the accumulator (warp w reads
//                    TMEM lanes 32(w%4).., the tile's rows, and every other
//                    16-column chunk, so two warps share each sub-partition),
//                    a 32 x 16 transpose through shared memory, then
//                    row-contiguous stores of the link, the plain product, a
//                    split-K partial or a slice of the partial products.
// Units run row tiles fastest when B is the larger operand (its panel is
// then reused by consecutive CTAs while A stays in L2) and column tiles
// fastest otherwise.
// The B operand can be given as two parts (hi + lo, both multiplied into the
// same accumulator): the engine does this for X in S = X V, so that X enters
// one of the two products of an iteration with ~16 (BF16) or ~22 (TF32) bits.
// Were X rounded in both products, the fixed point would solve the normal
// equations of X~ = X + E, whose Gram matrix carries the positive diagonal
// E^T E ~ n u^2 E[x^2]: a ridge shift comparable to lambda2 at n in the
// thousands.  FP32 operands reach kind::tf32 rounded to nearest (the tensor
// core would otherwise truncate them, a bias toward zero).
// With A also given as hi + lo (NA = 2, TF32 only) a K slice takes three
// products, A_hi B_hi + A_hi B_lo + A_lo B_hi: each FP32 operand is carried to
// ~22 bits and the dropped A_lo B_lo term is below 2^-22 of the product, so
// the result has the accuracy of an FP32 product (the FP32-accurate mode);
// its link epilogue writes R as the same hi + lo pair.
// Split-K with the plain or link epilogue: partial tiles go to scratch and
// the last epilogue warp to finish a 32-row slab and column half of a tile
// (an arrival counter for each) sums its partials in fixed order; no warp
// waits on another.
// CTA pairs (BF16, single operands): a cluster of two CTAs computes a 256-row
// tile with tcgen05.mma.cta_group::2 (M = 256) issued by the even CTA.  Each
// CTA copies its own 128 rows of A and half of the B tile's rows into its own
// ring, so that an SM takes in 32 KB instead of 48 KB per 128 x 256 x 64
// slice of products; a pair's stage holds two K slices (fewer, larger stages:
// the copies are bound by their round trip per stage); both CTAs' copies
// complete on the even CTA's stage barrier, and each CTA's epilogue drains its
// 128 rows of the accumulator from its own tensor memory.
// Every mbarrier wait is bounded; a wait that runs out sets an error flag,
// the roles stop, the MMA issuer drains its products and the producer its
// copies before the tensor memory is freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

constexpr int BM = 128;                 // rows per tile (one UMMA M = 128)
constexpr int ROWB = 128;               // bytes of K per stage and row (one swizzle row)
constexpr int MAXBN = 256;
constexpr int NT = 352;                 // eleven warps: producer, MMA, eight epilogue warps, second producer
constexpr int EPI_WARPS = 8;
constexpr int PROD2_WARP = 2 + EPI_WARPS;   // fills the odd ring stages (warp 0 the even ones)
constexpr uint32_t STAGE_A = BM * ROWB;
constexpr uint32_t TMEM_COLS = 512;     // two accumulators of up to 256 columns
constexpr int TPAD = 20;                // transpose buffer row: 16 + 4 (16-byte rows, no 128-bit bank conflicts on write)
constexpr int SMS = 152;
// A stage holds one K slice of every operand part: A (and A2 when NA = 2,
// the FP32-accurate split A_hi B_hi + A_hi B_lo + A_lo B_hi), B (and B2 when
// NB = 2, hi + lo).  The ring has as many stages as fit next to the epilogue
// buffer for the launch's tile width (at most kMaxStages).
constexpr int kMaxStages = 8;
constexpr size_t kEpiBytes = EPI_WARPS * 32 * TPAD * sizeof(float);
constexpr size_t kSmemMax = 224 * 1024;                    // dynamic shared memory per CTA (static 1 KB on top)
constexpr size_t kSmemFixed = 1024 + kEpiBytes + 256;      // alignment slack, epilogue, barriers
__host__ __device__ constexpr uint32_t stage_stride(int na, int nb, int bn) {
    return (uint32_t)na * STAGE_A + (uint32_t)nb * (uint32_t)bn * ROWB;   // a multiple of 2048
}
inline int ring_stages(int na, int nb, int bn) {
    const size_t n = (kSmemMax - kSmemFixed) / stage_stride(na, nb, bn);
    return (int)std::min<size_t>(n, kMaxStages);
}
inline size_t smem_for(int na, int nb, int bn) {
    return kSmemFixed + (size_t)ring_stages(na, nb, bn) * stage_stride(na, nb, bn);
}
constexpr uint32_t WAIT_LIMIT = 1u << 22;   // try_wait rounds before a wait gives up

// ------------------------------------------------------------------ arguments and epilogues

struct TcArgs {
    int M, N;                 // output rows (A rows) and columns (B rows)
    int arow0;                // first A row (a sub-batch of the A operand's rows)
    int bn;                   // columns per tile, multiple of 16, <= MAXBN
    int mt, nt, nz;           // row tiles, column tiles, K ranges (splits or jobs)
    int m_fast;               // units walk row tiles fastest
    int nkb, kb_per_split;    // K in 128-byte slices, slices per split
    uint32_t idesc;           // instruction descriptor
    int epi;                  // TC_EPI_*
    int stages;               // ring stages (<= kMaxStages)
    int ks;                   // K slices per stage (each with its own A and B parts)
    int round_tf32;           // round FP32 link outputs to TF32 (nearest) for the next product
    float* pout;              // TC_EPI_PARTIAL: slice z at pout + z * pstride, row stride pld
    size_t pstride;
    int pld;
    void* out;
    float* out_lo;            // TC_EPI_LINK_F32: TF32 low part of each output (NULL: none)
    int ldo;
    const float* y;
    int loss;
    float* part;              // split-K partial tiles (nz > 1, epi != PARTIAL)
    int* counters;
    int* err;
    int njobs;                // > 0: K range z is job z (its own K offsets in A and B, and slice)
    TcJob jobs[kTcMaxJobs];
};

// One problem of a grouped launch (BF16, single operands, no split-K link):
// its operand maps, shape, tiling and outputs; the fields the kernel reads per
// unit carry the names of TcArgs.
struct TcProb {
    CUtensorMap tmA, tmB;
    int M, N, arow0, mt, nt, nz, nkb, kb_per_split, m_fast;
    void* out;
    float* out_lo;
    int ldo;
    const float* y;
    int loss;
    float* pout;
    size_t pstride;
    int pld;
    float* part;
    int* counters;
};
// A grouped launch: the shared parameters (tile width, ring, instruction
// descriptor, epilogue kind, error flag) in a, and up to kTcGroupMax problems
// whose units are numbered consecutively (problem pi owns units ubase[pi] ..).
constexpr int kTcGroupMax = 8;
struct TcGroupArgs {
    TcArgs a;
    int np;
    int ubase[kTcGroupMax + 1];
    TcProb prob[kTcGroupMax];
};

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Loss derivative for operands that are rounded to BF16/TF32 (or split into
// TF32 hi + lo) next: fast exponential and approximate division, a few ulp of
// FP32, below the 2^-22 of the split.  Both are branch-free, so the 32 values
// of a chunk are evaluated interleaved (a correctly rounded reciprocal
// serialises them).  1 + e^{ys} = inf gives -0, the limit.
__device__ __forceinline__ float dloss_fast(float s, float y, int kind) {
    return kind == kLSQ ? 2.0f * (s - y) : __fdividef(-y, 1.0f + __expf(y * s));
}

// One output value v at (r, c) of problem q (r < M, c < N checked by the caller).
template <class Q>
__device__ __forceinline__ void tc_store(const TcArgs& a, const Q& q, int r, int c, float v, float yc, int zs) {
    if (a.epi == TC_EPI_PARTIAL) {
        q.pout[(size_t)zs * q.pstride + (size_t)r * q.pld + c] = v;
    } else if (a.epi == TC_EPI_STORE_F32) {
        static_cast<float*>(q.out)[(size_t)r * q.ldo + c] = v;
    } else if (a.epi == TC_EPI_LINK_F32) {
        const float d = dloss_fast(v, yc, q.loss);
        const float h = a.round_tf32 ? tf32_rn(d) : d;
        static_cast<float*>(q.out)[(size_t)r * q.ldo + c] = h;
        if (q.out_lo) q.out_lo[(size_t)r * q.ldo + c] = tf32_rn(d - h);
    } else {
        static_cast<__nv_bfloat16*>(q.out)[(size_t)r * q.ldo + c] = __float2bfloat16(dloss_fast(v, yc, q.loss));
    }
}

// The unit's tile and K range.
struct Unit {
    int mtile, ntile, z, ka, kb, nloc, slice, pi;   // pi: the problem (grouped launches), else 0
};
__device__ __forceinline__ Unit unit_of(const TcArgs& a, int u) {
    Unit w;
    w.pi = 0;
    const int tiles = a.mt * a.nt;
    w.z = u / tiles;
    const int t = u - w.z * tiles;
    if (a.m_fast) { w.mtile = t % a.mt; w.ntile = t / a.mt; }
    else          { w.ntile = t % a.nt; w.mtile = t / a.nt; }
    if (a.njobs > 0) {
        const TcJob& jb = a.jobs[w.z];
        w.ka = jb.ka; w.kb = jb.kb; w.nloc = jb.nkb; w.slice = jb.slice;
    } else {
        w.ka = w.kb = w.z * a.kb_per_split;
        w.nloc = max(0, min(a.nkb, w.ka + a.kb_per_split) - w.ka);
        w.slice = w.z;
    }
    return w;
}

// The unit of a CTA pair (CL = 2): pair units run over (row-tile pair, column
// tile, K range); the CTA of cluster rank r takes row tile 2 mp + r and columns
// [n0 + r bn/2, n0 + (r + 1) bn/2) of the B tile, so both CTAs of a pair share the
// column tile and K range.  A row tile past the last one (odd row-tile count)
// reads rows past M (or zeros) and stores nothing.
__device__ __forceinline__ Unit unit_of_pair(const TcArgs& a, int u, int crank) {
    Unit w;
    w.pi = 0;
    const int mtp = (a.mt + 1) >> 1;
    const int tiles = mtp * a.nt;
    w.z = u / tiles;
    const int t = u - w.z * tiles;
    int mp;
    if (a.m_fast) { mp = t % mtp; w.ntile = t / mtp; }
    else          { w.ntile = t % a.nt; mp = t / a.nt; }
    w.mtile = 2 * mp + crank;
    if (a.njobs > 0) {
        const TcJob& jb = a.jobs[w.z];
        w.ka = jb.ka; w.kb = jb.kb; w.nloc = jb.nkb; w.slice = jb.slice;
    } else {
        w.ka = w.kb = w.z * a.kb_per_split;
        w.nloc = max(0, min(a.nkb, w.ka + a.kb_per_split) - w.ka);
        w.slice = w.z;
    }
    return w;
}

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and the error flag) when it runs out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
#pragma unroll 1
    for (uint32_t i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicOr(err, 8);
    return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// A copy of this CTA's part of a pair's stage (cta_group::2): the bytes land in
// this CTA's shared memory at dst and complete on the mbarrier at the cluster
// address bar, the even CTA's stage barrier.
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// The cluster address of the shared-memory word at this CTA's offset addr in the CTA of rank r.
__device__ __forceinline__ uint32_t mapa_rank(uint32_t addr, uint32_t r) {
    uint32_t out;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(addr), "r"(r));
    return out;
}

// One arrival on an mbarrier given by its cluster address (this CTA's or the peer's).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Every thread of both CTAs of the cluster.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// CG = 2: one warp of each CTA of the pair takes part (the same columns in both).
template <int CG>
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    if constexpr (CG == 2) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

template <int CG>
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    if constexpr (CG == 2)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND == 0) {
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
            "}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    } else {
        asm volatile(
            "{\n"
            ".reg .pred p;\n"
            "setp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
            "}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc)
            : "memory");
    }
}

// The pair's product (BF16, M = 256): issued by the even CTA; A and B descriptors
// name the same offsets in both CTAs, the accumulator the same columns.
__device__ __forceinline__ void umma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive on the mbarrier at this offset in both CTAs of the pair once the pair's issued products finish.
__device__ __forceinline__ void umma_commit_pair_mc(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(bar), "h"((uint16_t)3)
                 : "memory");
}

// Arrive on this CTA's mbarrier once the pair's issued products finish.
__device__ __forceinline__ void umma_commit_pair(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes
// apart (stride byte offset), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused by swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                  // version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// ------------------------------------------------------------------ the kernel

// Programmatic dependent launch: let the next kernel in the stream be scheduled
// (its prologue overlaps this grid), and wait for the previous grid to have
// completed with its memory visible.  Both are no-ops without the launch attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The kernel body over a source of units and problems: SrcOne (the launch's
// operand maps and TcArgs) or SrcGroup (a table of problems).
template <int KIND, int NB, int NA, int CL, class S>
__device__ __forceinline__ void tc_body(const TcArgs& a, const S& src) {
    static_assert(CL == 1 || (KIND == 0 && NA == 1 && NB == 1), "CTA pairs: BF16 single operands");
    const int STAGES = a.stages;
    // B rows per CTA: a pair's CTAs hold half of the tile's columns each
    const int bnl = CL == 2 ? a.bn / 2 : a.bn;
    // a stage holds KS consecutive K slices (one barrier, one release for all)
    const int KS = a.ks;
    const uint32_t SLSTR = stage_stride(NA, NB, bnl);
    const uint32_t SSTR = (uint32_t)KS * SLSTR;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    // stage s at smem + s SSTR: A, A2 (NA = 2), B, B2 (NB = 2); every part 1024-byte aligned
    const uint32_t offB = (uint32_t)NA * STAGE_A, offB2 = offB + (uint32_t)bnl * ROWB;
    float* sT = reinterpret_cast<float*>(smem + (size_t)STAGES * SSTR);            // 4 x 32 x TPAD
    uint64_t* bars = reinterpret_cast<uint64_t*>(sT + EPI_WARPS * 32 * TPAD);
    // bars: full[S], empty[S], tfull[2], tempty[2], drain
    uint64_t* full = bars;
    uint64_t* empty = bars + kMaxStages;
    uint64_t* tfull = bars + 2 * kMaxStages;
    uint64_t* tempty = bars + 2 * kMaxStages + 2;
    uint64_t* drain = bars + 2 * kMaxStages + 4;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kMaxStages + 5);
    __shared__ int s_consumed;       // stage fills the MMA issuer consumed (producer drain at exit)
    __shared__ int s_issued[2];      // per producer: one past the last stage fill it issued

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KE = KIND == 0 ? 64 : 32;          // elements per 128-byte row
    const uint32_t stage_bytes = (uint32_t)NA * STAGE_A + (uint32_t)NB * bnl * ROWB;
    // CL = 2: CTA pairs (clusters of two) walk pair units; the even CTA (the
    // leader) waits for both CTAs' copies on its stage barriers, issues the pair's
    // products and frees each stage, and publishes each accumulator, in both
    // CTAs; both epilogues release an accumulator on the leader's barrier
    const int crank = CL == 2 ? (int)cluster_ctarank() : 0;
    const bool leader = crank == 0;
    const int units = src.units(CL);
    const int ucta = blockIdx.x / CL, ustride = gridDim.x / CL;
    auto unit = [&](int u) { return src.unit(u, CL, crank); };

    pdl_trigger();
    if (threadIdx.x == 32) {
        // descriptors of the operand maps into the TMA unit's cache before the first copy
        src.prefetch(NB, NA);
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < STAGES; ++q) { mbar_init(smem_u32(&full[q]), 1); mbar_init(smem_u32(&empty[q]), 1); }
        // accumulator releases: every epilogue thread of this CTA, or one per
        // epilogue warp of both CTAs of a pair
        for (int q = 0; q < 2; ++q) {
            mbar_init(smem_u32(&tfull[q]), 1);
            mbar_init(smem_u32(&tempty[q]), CL == 2 ? 2 * EPI_WARPS : 32 * EPI_WARPS);
        }
        mbar_init(smem_u32(drain), 1);
        s_consumed = 0;
        s_issued[0] = s_issued[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc<CL>(smem_u32(tmem_slot), TMEM_COLS);
    tc_fence_before();
    __syncwarp();                    // whole warps at the CTA barrier (lane 0 of warp 0 ran the setup)
    __syncthreads();
    if constexpr (CL == 2) cluster_sync();   // both CTAs' barriers initialised before any remote arrival
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    pdl_wait();                      // operands and outputs belong to the previous grid until it completes
    // Two producers, lane 0 of warp 0 (even ring stages) and of warp PROD2_WARP (odd
    // ones): a thread that issues TMA copies takes a few hundred cycles per stage
    // whatever its size, so one thread alone cannot keep the tensor pipe fed.
    // The producers split the ring by stage, stage s to producer s % 2, so that every
    // stage has one producer, which fills it in order and so waits on its empty
    // barrier at most one phase ahead (were fills g and g + STAGES of a stage issued
    // by different producers, one of them could test the barrier two phases ahead,
    // where the parity cannot tell the phases apart).  A one-stage ring has one.
    const int nprod = STAGES >= 2 ? 2 : 1;
    if (warp == 0 || warp == PROD2_WARP) {
      // lanes 1-31 of both producer warps wait at the exit barrier
      if (lane == 0 && (warp == 0 || nprod == 2)) {
        const int pidx = warp == 0 ? 0 : 1;
        int g = 0, mine = 0;
        bool ok = true;
        for (int u = ucta; u < units && ok; u += ustride) {
            const Unit w = unit(u);
            const auto& pq = src.q(w.pi);
            const int m0 = w.mtile * BM, n0 = w.ntile * a.bn;
            const int nst = (w.nloc + KS - 1) / KS;     // stages of this unit
            for (int i = 0; i < nst; ++i, ++g) {
                if ((g % STAGES) % nprod != pidx) continue;
                const int s = g % STAGES;
                const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u, a.err)) { ok = false; break; }
                const uint32_t fb = smem_u32(&full[s]);
                const int nsl = min(KS, w.nloc - i * KS);   // K slices in this stage
                if constexpr (CL == 2) {
                    if (leader) mbar_expect_tx(fb, 2 * stage_bytes * (uint32_t)nsl);
                } else {
                    mbar_expect_tx(fb, stage_bytes * (uint32_t)nsl);
                }
                for (int t = 0; t < nsl; ++t) {
                    const int kxa = (w.ka + i * KS + t) * KE, kxb = (w.kb + i * KS + t) * KE;
                    uint8_t* sp = smem + (size_t)s * SSTR + (size_t)t * SLSTR;
                    if constexpr (CL == 2) {
                        // this CTA's rows of A and half of B, completing on the leader's barrier
                        const uint32_t lb = mapa_rank(fb, 0);
                        tma_load_2d_pair(smem_u32(sp), src.mapA(w.pi), kxa, pq.arow0 + m0, lb);
                        tma_load_2d_pair(smem_u32(sp + offB), src.mapB(w.pi), kxb, n0 + crank * bnl, lb);
                    } else {
                        tma_load_2d(smem_u32(sp), src.mapA(w.pi), kxa, pq.arow0 + m0, fb);
                        if (NA == 2) tma_load_2d(smem_u32(sp + STAGE_A), src.mapA2(w.pi), kxa, pq.arow0 + m0, fb);
                        tma_load_2d(smem_u32(sp + offB), src.mapB(w.pi), kxb, n0, fb);
                        if (NB == 2) tma_load_2d(smem_u32(sp + offB2), src.mapB2(w.pi), kxb, n0, fb);
                    }
                }
                mine = g + 1;
            }
        }
        s_issued[pidx] = mine;
      }
    } else if (warp == 1) {
        if (CL == 2 && !leader) {
            // the odd CTA of a pair issues no products
        } else if (lane == 0) {
            // MMA issuer
            int g = 0, li = 0;
            bool ok = true;
            for (int u = ucta; u < units && ok; u += ustride, ++li) {
                const Unit w = unit(u);
                const int b = li & 1;
                const uint32_t use = (uint32_t)(li >> 1) & 1u;
                if (!mbar_wait(smem_u32(&tempty[b]), use ^ 1u, a.err)) break;
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * MAXBN);
                const int nst = (w.nloc + KS - 1) / KS;
                for (int i = 0; i < nst; ++i, ++g) {
                    const int s = g % STAGES;
                    const uint32_t ph = (uint32_t)(g / STAGES) & 1u;
                    if (!mbar_wait(smem_u32(&full[s]), ph, a.err)) { ok = false; break; }
                    tc_fence_after();
                    const int nsl = min(KS, w.nloc - i * KS);
                    for (int t = 0; t < nsl; ++t) {
                        const uint32_t aa = smem_u32(smem + (size_t)s * SSTR + (size_t)t * SLSTR), bb = aa + offB;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {   // four MMAs of 32 bytes of K each (per B part)
                            const uint32_t accf = (i > 0 || t > 0 || kk > 0) ? 1u : 0u;
                            if constexpr (CL == 2) {
                                umma_pair(acc, smem_desc(aa + kk * 32), smem_desc(bb + kk * 32), a.idesc, accf);
                            } else {
                                umma<KIND>(acc, smem_desc(aa + kk * 32), smem_desc(bb + kk * 32), a.idesc, accf);
                                if (NB == 2)
                                    umma<KIND>(acc, smem_desc(aa + kk * 32), smem_desc(aa + offB2 + kk * 32), a.idesc, 1u);
                                if (NA == 2)
                                    umma<KIND>(acc, smem_desc(aa + STAGE_A + kk * 32), smem_desc(bb + kk * 32), a.idesc, 1u);
                            }
                        }
                    }
                    if constexpr (CL == 2) umma_commit_pair_mc(smem_u32(&empty[s]));   // in both CTAs
                    else umma_commit(smem_u32(&empty[s]));   // stage s is free once these MMAs finish
                    s_consumed = g + 1;
                }
                // the accumulator is complete (or abandoned)
                if constexpr (CL == 2) umma_commit_pair_mc(smem_u32(&tfull[b]));
                else umma_commit(smem_u32(&tfull[b]));
            }
            // every product issued so far has finished once this commit arrives
            if constexpr (CL == 2) umma_commit_pair(smem_u32(drain));
            else umma_commit(smem_u32(drain));
            mbar_wait(smem_u32(drain), 0u, a.err);
        }
    } else if (warp < 2 + EPI_WARPS) {
        // epilogue: warps 2..9; warp w reads the TMEM lane quadrant w % 4 (the
        // tile's rows 32 (w % 4) ..) and every other 16-column chunk of the tile,
        // starting at chunk h = (w - 2) / 4, so that two warps per SM
        // sub-partition overlap one's link arithmetic with the other's stores
        const int quad = warp & 3;
        const int h = (warp - 2) >> 2;
        float* tb = sT + (warp - 2) * 32 * TPAD;
        int li = 0;
        for (int u = ucta; u < units; u += ustride, ++li) {
            const Unit w = unit(u);
            const auto& pq = src.q(w.pi);
            const int b = li & 1;
            const uint32_t use = (uint32_t)(li >> 1) & 1u;
            // the link's y of this warp's columns (lane l < 16 holds column c + l of
            // its chunk q at c = 16 h + 32 q), loaded before the wait so that the
            // epilogue does not wait on them per chunk
            float ypre[MAXBN / 32];
            const bool linky = pq.y != nullptr && pq.nz == 1 && (a.epi == TC_EPI_LINK_F32 || a.epi == TC_EPI_LINK_BF16);
#pragma unroll
            for (int q = 0; q < MAXBN / 32; ++q) {
                const int cc = 16 * h + 32 * q + (lane & 15);
                const int col = w.ntile * a.bn + cc;
                ypre[q] = (linky && cc < a.bn && col < pq.N) ? __ldg(pq.y + col) : 0.f;
            }
            const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&tfull[b]), use, a.err));
            if (!ok) break;
            tc_fence_after();
            const int m0 = w.mtile * BM, n0 = w.ntile * a.bn;
            const int rbase = m0 + quad * 32;             // this warp's 32 rows
            const bool split = pq.nz > 1 && a.epi != TC_EPI_PARTIAL;
            const int tile = w.mtile * pq.nt + w.ntile;
            const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * MAXBN);
#pragma unroll 1
            for (int c = 16 * h, q = 0; c < a.bn; c += 32, ++q) {
                float v[16];
                if (w.nloc > 0) {
                    tmem_ld16(tl + (uint32_t)c, v);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = 0.f;
                }
                const int c0 = n0 + c;
                if (!split && (a.epi == TC_EPI_LINK_F32 || a.epi == TC_EPI_LINK_BF16)) {
                    // link on the row-per-lane values; y of column c0 + j from lane j
                    float yl = 0.f;
#pragma unroll
                    for (int t = 0; t < MAXBN / 32; ++t)
                        if (t == q) yl = ypre[t];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = dloss_fast(v[j], __shfl_sync(0xffffffffu, yl, j), pq.loss);
                }
#pragma unroll
                for (int j = 0; j < 16; j += 4)                         // row lane, columns j..j+3
                    *reinterpret_cast<float4*>(tb + lane * TPAD + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                __syncwarp();
                if (split) {
                    // 8 rows x 64 bytes per instruction
                    float* pt = pq.part + (((size_t)w.z * (pq.mt * pq.nt) + tile) * BM + quad * 32) * MAXBN + c;
                    const int qq = lane & 3, r0 = lane >> 2;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = r0 + 8 * i;
                        *reinterpret_cast<float4*>(pt + (size_t)r * MAXBN + 4 * qq) =
                            *reinterpret_cast<const float4*>(tb + r * TPAD + 4 * qq);
                    }
                } else if (a.epi == TC_EPI_LINK_BF16) {
                    // 16 rows x 32 bytes per instruction (8 BF16 per lane)
                    __nv_bfloat16* o = static_cast<__nv_bfloat16*>(pq.out);
                    const int qq = lane & 1, r0 = lane >> 1;
                    const bool vec = (pq.ldo % 8) == 0 && c0 + 8 * qq + 8 <= pq.N;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int r = r0 + 16 * i, row = rbase + r;
                        if (row >= pq.M) continue;
                        const float4 x0 = *reinterpret_cast<const float4*>(tb + r * TPAD + 8 * qq);
                        const float4 x1 = *reinterpret_cast<const float4*>(tb + r * TPAD + 8 * qq + 4);
                        __nv_bfloat16* dst = o + (size_t)row * pq.ldo + c0 + 8 * qq;
                        if (vec) {
                            __nv_bfloat162 hh[4] = {__floats2bfloat162_rn(x0.x, x0.y), __floats2bfloat162_rn(x0.z, x0.w),
                                                    __floats2bfloat162_rn(x1.x, x1.y), __floats2bfloat162_rn(x1.z, x1.w)};
                            *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(hh);
                        } else {
                            const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                            for (int t = 0; t < 8; ++t)
                                if (c0 + 8 * qq + t < pq.N) dst[t] = __float2bfloat16(xs[t]);
                        }
                    }
                } else {
                    // FP32 outputs (product, link, partial slice): 8 rows x 64 bytes per instruction
                    float* o;
                    size_t ld;
                    if (a.epi == TC_EPI_PARTIAL) { o = pq.pout + (size_t)w.slice * pq.pstride; ld = (size_t)pq.pld; }
                    else { o = static_cast<float*>(pq.out); ld = (size_t)pq.ldo; }
                    const bool link = a.epi == TC_EPI_LINK_F32;
                    const bool rnd = link && a.round_tf32;
                    float* ol = link ? pq.out_lo : nullptr;
                    const int qq = lane & 3, r0 = lane >> 2;
                    const bool vec = (ld % 4) == 0 && (reinterpret_cast<uintptr_t>(o) % 16) == 0 &&
                                     (ol == nullptr || (reinterpret_cast<uintptr_t>(ol) % 16) == 0) && c0 + 4 * qq + 4 <= pq.N;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = r0 + 8 * i, row = rbase + r;
                        if (row >= pq.M) continue;
                        const float4 x = *reinterpret_cast<const float4*>(tb + r * TPAD + 4 * qq);
                        float xs[4] = {x.x, x.y, x.z, x.w}, ls[4] = {0.f, 0.f, 0.f, 0.f};
                        if (rnd) {
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const float hi = tf32_rn(xs[t]);
                                ls[t] = tf32_rn(xs[t] - hi);
                                xs[t] = hi;
                            }
                        }
                        float* dst = o + (size_t)row * ld + c0 + 4 * qq;
                        float* dlo = ol ? ol + (size_t)row * ld + c0 + 4 * qq : nullptr;
                        if (vec) {
                            *reinterpret_cast<float4*>(dst) = make_float4(xs[0], xs[1], xs[2], xs[3]);
                            if (dlo) *reinterpret_cast<float4*>(dlo) = make_float4(ls[0], ls[1], ls[2], ls[3]);
                        } else {
#pragma unroll
                            for (int t = 0; t < 4; ++t)
                                if (c0 + 4 * qq + t < pq.N) {
                                    dst[t] = xs[t];
                                    if (dlo) dlo[t] = ls[t];
                                }
                        }
                    }
                }
                __syncwarp();
            }
            // the accumulator may be overwritten by the unit after next
            tc_fence_before();
            if constexpr (CL == 2) {
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(mapa_rank(smem_u32(&tempty[b]), 0));
            } else {
                mbar_arrive(smem_u32(&tempty[b]));
            }
            if (split) {
                // per-warp arrival: the last of the nz units of this tile to finish
                // this warp's 32 rows and chunks sums their partials (no warp waits
                // on another)
                __threadfence();
                __syncwarp();
                const int slab = (tile * 4 + quad) * 2 + h;
                int last = 0;
                if (lane == 0) last = atomicAdd(&pq.counters[slab], 1) == pq.nz - 1;
                last = __shfl_sync(0xffffffffu, last, 0);
                if (last) {
                    __threadfence();
                    // lanes 0-15 take chunk c, lanes 16-31 chunk c + 32 (this warp's next)
                    // eight rows at a time, so that their partial loads are in flight
                    // together (each sum still runs over z = 0.. in order)
                    for (int c = 16 * h; c < a.bn; c += 64) {
                        const int cc = c + (lane < 16 ? lane : 16 + lane);
                        const int col = n0 + cc;
                        const bool in = cc < a.bn && col < pq.N;
                        const float yc = (in && pq.y != nullptr) ? __ldg(pq.y + col) : 0.f;
                        for (int r0 = 0; r0 < 32; r0 += 8) {
                            float acc[8];
#pragma unroll
                            for (int rr = 0; rr < 8; ++rr) acc[rr] = 0.f;
                            if (in)
                                for (int z = 0; z < pq.nz; ++z) {
                                    const float* pz = pq.part + (((size_t)z * (pq.mt * pq.nt) + tile) * BM + quad * 32 + r0) * MAXBN + cc;
#pragma unroll
                                    for (int rr = 0; rr < 8; ++rr) acc[rr] += __ldcg(pz + (size_t)rr * MAXBN);
                                }
#pragma unroll
                            for (int rr = 0; rr < 8; ++rr)
                                if (in && rbase + r0 + rr < pq.M) tc_store(a, pq, rbase + r0 + rr, col, acc[rr], yc, 0);
                        }
                    }
                    if (lane == 0) pq.counters[slab] = 0;
                }
            }
        }
    }
    // reconverge the role warps (one lane each ran the producer / MMA loop) so
    // that the barrier holds every thread until the epilogue warps are done
    __syncwarp();
    __syncthreads();
    if (warp == 0 && lane == 0) {
        const int issued = max(s_issued[0], s_issued[1]);
        // copies still in flight (a wait that ran out) land before the CTA exits
        // (a pair's copies all complete on the leader's barriers)
        if (leader)
            for (int g = s_consumed; g < issued; ++g)
                mbar_wait(smem_u32(&full[g % STAGES]), (uint32_t)(g / STAGES) & 1u, a.err);
        if constexpr (CL == 2) {
            // the leader's releases of this CTA's last stage fills (commits that
            // arrive here from the other SM) land before the CTA frees or leaves
            if (a.err == nullptr || *reinterpret_cast<volatile int*>(a.err) == 0)
                for (int g = max(0, issued - STAGES); g < issued; ++g)
                    if (!mbar_wait(smem_u32(&empty[g % STAGES]), (uint32_t)(g / STAGES) & 1u, a.err)) break;
        }
    }
    // a pair: the leader's products (which read both CTAs' shared memory and write
    // both CTAs' tensor memory) and both epilogues are done before either CTA
    // frees its tensor memory or leaves
    if constexpr (CL == 2) {
        __syncwarp();
        cluster_sync();
    }
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc<CL>(tmem, TMEM_COLS);
    }
}

struct SrcOne {
    const CUtensorMap *A, *B, *B2, *A2;
    const TcArgs& a;
    __device__ int units(int CL) const { return (CL == 2 ? (a.mt + 1) / 2 : a.mt) * a.nt * a.nz; }
    __device__ Unit unit(int u, int CL, int crank) const { return CL == 2 ? unit_of_pair(a, u, crank) : unit_of(a, u); }
    __device__ const TcArgs& q(int) const { return a; }
    __device__ const CUtensorMap* mapA(int) const { return A; }
    __device__ const CUtensorMap* mapB(int) const { return B; }
    __device__ const CUtensorMap* mapB2(int) const { return B2; }
    __device__ const CUtensorMap* mapA2(int) const { return A2; }
    __device__ void prefetch(int nb, int na) const {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(A)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(B)) : "memory");
        if (nb == 2) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(B2)) : "memory");
        if (na == 2) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(A2)) : "memory");
    }
};

// The units of problem pi: its tiles (row tiles fastest if m_fast) times its K ranges.
__device__ __forceinline__ Unit unit_of_prob(const TcProb& q, int u) {
    Unit w;
    const int tiles = q.mt * q.nt;
    w.z = u / tiles;
    const int t = u - w.z * tiles;
    if (q.m_fast) { w.mtile = t % q.mt; w.ntile = t / q.mt; }
    else          { w.ntile = t % q.nt; w.mtile = t / q.nt; }
    w.ka = w.kb = w.z * q.kb_per_split;
    w.nloc = max(0, min(q.nkb, w.ka + q.kb_per_split) - w.ka);
    w.slice = w.z;
    return w;
}

struct SrcGroup {
    const TcGroupArgs& g;
    __device__ int units(int) const { return g.ubase[g.np]; }
    __device__ Unit unit(int u, int, int) const {
        int pi = 0;
        while (pi + 1 < g.np && u >= g.ubase[pi + 1]) ++pi;
        Unit w = unit_of_prob(g.prob[pi], u - g.ubase[pi]);
        w.pi = pi;
        return w;
    }
    __device__ const TcProb& q(int pi) const { return g.prob[pi]; }
    __device__ const CUtensorMap* mapA(int pi) const { return &g.prob[pi].tmA; }
    __device__ const CUtensorMap* mapB(int pi) const { return &g.prob[pi].tmB; }
    __device__ const CUtensorMap* mapB2(int pi) const { return &g.prob[pi].tmB; }
    __device__ const CUtensorMap* mapA2(int pi) const { return &g.prob[pi].tmA; }
    __device__ void prefetch(int, int) const {
        for (int i = 0; i < g.np; ++i) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&g.prob[i].tmA)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&g.prob[i].tmB)) : "memory");
        }
    }
};

template <int KIND, int NB, int NA, int CL>
__global__ void __launch_bounds__(NT, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB,
                                                   const __grid_constant__ CUtensorMap tmB2,
                                                   const __grid_constant__ CUtensorMap tmA2,
                                                   const __grid_constant__ TcArgs a) {
    const SrcOne src{&tmA, &tmB, &tmB2, &tmA2, a};
    tc_body<KIND, NB, NA, CL>(a, src);
}

// Several problems (the instances of the serving loop) in one persistent launch.
__global__ void __launch_bounds__(NT, 1) k_tc_gemm_group(const __grid_constant__ TcGroupArgs g) {
    const SrcGroup src{g};
    tc_body<0, 1, 1, 1>(g.a, src);
}

// A wait that nothing ends: one thread waits on an mbarrier no thread arrives
// on, for `rounds` try_wait rounds, then reports the timeout through the same
// flag as the products' waits (bit 8).  Checks the timeout path end to end.
__global__ void k_wait_probe(uint32_t rounds, int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = false;
        for (uint32_t i = 0; i < rounds && !ok; ++i) ok = mbar_try_wait(smem_u32(&bar), 0u);
        if (!ok) atomicOr(err, 8);
    }
}

// ------------------------------------------------------------------ host side

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

template <int KIND, int NB, int NA, int CL = 1>
int set_smem_attr() {
    // once per process (thread-safe static initialisation: serving contexts launch from several threads)
    static const int rc = cudaFuncSetAttribute(k_tc_gemm<KIND, NB, NA, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmemMax) == cudaSuccess ? 0 : -1;
    return rc;
}

// Clusters of two of k_tc_gemm<0, 1, 1, 2> that can be resident at once (once per process).
int pair_clusters() {
    static const int n = [] {
        if (set_smem_attr<0, 1, 1, 2>() != 0) return 0;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(2 * SMS);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = kSmemMax;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int c = 0;
        if (cudaOccupancyMaxActiveClusters(&c, k_tc_gemm<0, 1, 1, 2>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            c = 0;
        }
        return c;
    }();
    return n;
}

}  // namespace

void wait_probe(cudaStream_t s, uint32_t rounds, int* err) { k_wait_probe<<<1, 32, 0, s>>>(rounds, err); }

int tc_prepare() {
    return set_smem_attr<0, 1, 1>() | set_smem_attr<0, 2, 1>() | set_smem_attr<1, 1, 1>() | set_smem_attr<1, 2, 1>() |
           set_smem_attr<1, 2, 2>() | set_smem_attr<0, 1, 1, 2>() | (pair_clusters() > 0 ? 0 : 0);
}

int tc_make_map(TcMap* out, const void* base, int is_bf16, int rows, int cols, int ld, int box_rows) {
    static_assert(sizeof(TcMap) >= sizeof(CUtensorMap), "TcMap too small");
    auto fn = encode_fn();
    if (!fn) return -1;
    const int esz = is_bf16 ? 2 : 4;
    if (((uintptr_t)base % 16) != 0 || ((size_t)ld * esz) % 16 != 0 || box_rows < 1 || box_rows > 256) return -2;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(ROWB / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const auto dt = is_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(out->bytes), dt, 2, const_cast<void*>(base), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -3;
    out->has_half = 0;
    if (box_rows % 16 == 0) {
        // half the box rows: each CTA of a pair copies half of a B tile
        box[1] = (cuuint32_t)(box_rows / 2);
        r = fn(reinterpret_cast<CUtensorMap*>(out->half), dt, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return -3;
        out->has_half = 1;
    }
    return 0;
}

int tc_tile_cols(int N) { return N >= MAXBN ? MAXBN : ((N + 15) / 16) * 16; }
int tc_split_cap(int M, int N) {
    const int tiles = ((M + BM - 1) / BM) * ((N + tc_tile_cols(N) - 1) / tc_tile_cols(N));
    return std::max(1, std::min(16, (SMS + tiles - 1) / tiles));
}
int tc_tile_cols_wide(int N) { return N > MAXBN ? 128 : tc_tile_cols(N); }

size_t tc_scratch_bytes() { return (size_t)3 * SMS * BM * MAXBN * sizeof(float); }
int tc_scratch_counters() { return 8 * SMS; }   // one per 32-row slab and column half of a tile

// Persistent grid: one CTA per SM (at most one per unit).
static int grid_of(int units) { return std::max(1, std::min(units, SMS)); }

int tc_gemm(cudaStream_t s, const TcMap& A, const TcMap& B, const TcMap* B2, const TcGemm& g,
            const GemmScratch* scr) {
    if (g.M <= 0 || g.N <= 0) return 0;
    if (g.bn < 16 || g.bn > MAXBN || g.bn % 16 != 0) return -4;
    const int nb = B2 ? 2 : 1, na = g.A2 ? 2 : 1;
    if (na == 2 && (g.kind != 1 || nb != 2)) return -6;     // the split is TF32 hi/lo on both sides
    const int rc = na == 2 ? set_smem_attr<1, 2, 2>()
                 : g.kind == 0 ? (nb == 1 ? set_smem_attr<0, 1, 1>() : set_smem_attr<0, 2, 1>())
                               : (nb == 1 ? set_smem_attr<1, 1, 1>() : set_smem_attr<1, 2, 1>());
    if (rc) return -5;
    const int KE = g.kind == 0 ? 64 : 32;
    TcArgs a{};
    a.M = g.M; a.N = g.N; a.bn = g.bn;
    a.arow0 = g.arow0;
    a.nkb = (g.K + KE - 1) / KE;
    a.mt = (g.M + BM - 1) / BM;
    a.nt = (g.N + g.bn - 1) / g.bn;
    const int tiles = a.mt * a.nt;
    // split-K: at least 4 slices of K per unit, until the units fill the SMs
    int splits = 1;
    if (g.epi == TC_EPI_PARTIAL) {
        splits = std::max(1, std::min(g.max_splits, std::min((a.nkb + 3) / 4, std::max(1, SMS / tiles))));
    } else if (tiles < SMS && scr && scr->part && scr->counters && scr->n_counters >= 8 * tiles) {
        splits = std::min((a.nkb + 3) / 4, std::max(1, SMS / tiles));
        const size_t need = (size_t)splits * tiles * BM * MAXBN * sizeof(float);
        if (need > scr->part_bytes) splits = (int)std::max<size_t>(1, scr->part_bytes / ((size_t)tiles * BM * MAXBN * sizeof(float)));
    }
    a.kb_per_split = (a.nkb + splits - 1) / splits;
    splits = (a.nkb + a.kb_per_split - 1) / a.kb_per_split;
    a.nz = splits;
    if (g.splits_used) *g.splits_used = splits;
    // reuse the larger operand's panels on consecutive units
    a.m_fast = (size_t)g.N * (size_t)nb >= (size_t)g.M;
    a.pout = g.pout; a.pstride = g.pstride; a.pld = g.pld;
    // instruction descriptor: D F32 (bits 4-5 = 1), A/B format (bits 7-9, 10-12:
    // BF16 = 1 for kind::f16, TF32 = 2 for kind::tf32), K-major A and B, N>>3 at
    // bit 17, M>>4 at bit 24
    const uint32_t ab = g.kind == 0 ? 1u : 2u;
    a.idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(g.bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    a.epi = g.epi; a.out = g.out; a.out_lo = g.out_lo; a.ldo = g.ldo; a.y = g.y; a.loss = g.loss;
    a.round_tf32 = g.kind == 1;
    a.part = splits > 1 ? static_cast<float*>(scr->part) : nullptr;
    a.counters = splits > 1 ? scr->counters : nullptr;
    a.err = g.err;
    const CUtensorMap& ma = *reinterpret_cast<const CUtensorMap*>(A.bytes);
    const CUtensorMap& mb = *reinterpret_cast<const CUtensorMap*>(B.bytes);
    const CUtensorMap& mb2 = *reinterpret_cast<const CUtensorMap*>((B2 ? B2 : &B)->bytes);
    const CUtensorMap& ma2 = *reinterpret_cast<const CUtensorMap*>((g.A2 ? g.A2 : &A)->bytes);
    // CTA pairs: BF16 single operands, at least two row tiles, no split-K link epilogue
    // (its partial tiles and arrival counters are indexed per tile), a B map with a
    // half box
    const bool pair = g.pair && g.kind == 0 && nb == 1 && na == 1 && a.mt >= 2 &&
                      (splits == 1 || g.epi == TC_EPI_PARTIAL) && a.njobs == 0 && B.has_half &&
                      pair_clusters() > 0;
    // a pair's ring holds this CTA's half of each B slice, two K slices per stage:
    // its copies are bound by their round trip, so fewer and larger stages
    // (three of 64 KB at 256 columns) keep more bytes in flight per stage than six
    // of 32 KB; its products have M = 256
    a.ks = pair ? 2 : 1;
    {
        const size_t sl = pair ? stage_stride(1, 1, g.bn / 2) : stage_stride(na, nb, g.bn);
        a.stages = (int)std::min<size_t>((kSmemMax - kSmemFixed) / ((size_t)a.ks * sl), kMaxStages);
    }
    const size_t smem = kSmemFixed + (size_t)a.stages * a.ks *
                                         (pair ? stage_stride(1, 1, g.bn / 2) : stage_stride(na, nb, g.bn));
    if (pair) a.idesc = (a.idesc & ~(0x1Fu << 24)) | ((uint32_t)((2 * BM) >> 4) << 24);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(pair ? 2 * std::max(1, std::min(((a.mt + 1) / 2) * a.nt * splits, pair_clusters()))
                            : grid_of(tiles * splits));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    int na_ = 0;
    if (g.pdl) {
        attr[na_].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na_].val.programmaticStreamSerializationAllowed = 1;
        ++na_;
    }
    if (pair) {
        attr[na_].id = cudaLaunchAttributeClusterDimension;
        attr[na_].val.clusterDim.x = 2;
        attr[na_].val.clusterDim.y = 1;
        attr[na_].val.clusterDim.z = 1;
        ++na_;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na_;
    cudaError_t e;
    const CUtensorMap& mbh = *reinterpret_cast<const CUtensorMap*>(B.half);
    if (pair) e = cudaLaunchKernelEx(&cfg, k_tc_gemm<0, 1, 1, 2>, ma, mbh, mbh, ma, a);
    else if (na == 2) e = cudaLaunchKernelEx(&cfg, k_tc_gemm<1, 2, 2, 1>, ma, mb, mb2, ma2, a);
    else if (g.kind == 0) e = nb == 1 ? cudaLaunchKernelEx(&cfg, k_tc_gemm<0, 1, 1, 1>, ma, mb, mb2, ma, a)
                                      : cudaLaunchKernelEx(&cfg, k_tc_gemm<0, 2, 1, 1>, ma, mb, mb2, ma, a);
    else e = nb == 1 ? cudaLaunchKernelEx(&cfg, k_tc_gemm<1, 1, 1, 1>, ma, mb, mb2, ma, a)
                     : cudaLaunchKernelEx(&cfg, k_tc_gemm<1, 2, 1, 1>, ma, mb, mb2, ma, a);
    return e == cudaSuccess ? 0 : -7;
}

int tc_gemm_group(cudaStream_t s, const TcGroupItem* items, int np, int bn, int epi, int* err) {
    static_assert(sizeof(TcGroupArgs) <= 32764, "kernel parameters of a grouped launch");
    if (np <= 0) return 0;
    if (np > kTcGroupMax || bn < 16 || bn > MAXBN || bn % 16 != 0) return -4;
    if (epi != TC_EPI_LINK_BF16 && epi != TC_EPI_PARTIAL) return -4;
    static const int rc = cudaFuncSetAttribute(k_tc_gemm_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)kSmemMax) == cudaSuccess ? 0 : -1;
    if (rc) return -5;
    TcGroupArgs g{};
    g.a.bn = bn;
    g.a.epi = epi;
    g.a.stages = ring_stages(1, 1, bn);
    g.a.ks = 1;
    g.a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    g.a.round_tf32 = 0;
    g.a.err = err;
    g.np = np;
    int units = 0;
    for (int i = 0; i < np; ++i) {
        const TcGroupItem& it = items[i];
        TcProb& q = g.prob[i];
        memcpy(&q.tmA, it.A->bytes, sizeof(CUtensorMap));
        memcpy(&q.tmB, it.B->bytes, sizeof(CUtensorMap));
        q.M = std::max(0, it.M);
        q.N = it.N;
        q.arow0 = it.arow0;
        q.nkb = (it.K + 63) / 64;
        q.mt = (q.M + BM - 1) / BM;
        q.nt = (it.N + bn - 1) / bn;
        // split-K of a partial product from the problem alone: its tile count at its
        // own width, so that its slices do not depend on the other problems
        int splits = 1;
        if (epi == TC_EPI_PARTIAL && q.M > 0) {
            const int tiles_alone = q.mt * ((it.N + it.splits_bn - 1) / it.splits_bn);
            splits = std::max(1, std::min(it.max_splits, std::min((q.nkb + 3) / 4, std::max(1, SMS / tiles_alone))));
        }
        q.kb_per_split = (q.nkb + splits - 1) / splits;
        splits = std::max(1, (q.nkb + q.kb_per_split - 1) / q.kb_per_split);
        q.nz = splits;
        if (it.splits_used) *it.splits_used = splits;
        q.m_fast = it.N >= q.M;
        q.out = it.out;
        q.out_lo = nullptr;
        q.ldo = it.ldo;
        q.y = it.y;
        q.loss = it.loss;
        q.pout = it.pout;
        q.pstride = it.pstride;
        q.pld = it.pld;
        q.part = nullptr;
        q.counters = nullptr;
        g.ubase[i] = units;
        units += q.M > 0 ? q.mt * q.nt * q.nz : 0;
    }
    g.ubase[np] = units;
    if (units == 0) return 0;
    k_tc_gemm_group<<<grid_of(units), NT, smem_for(1, 1, bn), s>>>(g);
    return 0;
}

int tc_gemm_jobs(cudaStream_t s, const TcMap& A, const TcMap& B, int M, int N, int bn, const TcJob* jobs,
                 int njobs, float* pout, size_t pstride, int pld, int* err, int pair_on) {
    if (M <= 0 || N <= 0 || njobs <= 0) return 0;
    if (bn < 16 || bn > MAXBN || bn % 16 != 0 || njobs > kTcMaxJobs) return -4;
    if (set_smem_attr<0, 1, 1>()) return -5;
    TcArgs a{};
    a.M = M; a.N = N; a.bn = bn;
    a.mt = (M + BM - 1) / BM;
    a.nt = (N + bn - 1) / bn;
    a.nz = njobs;
    a.m_fast = N >= M;
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    a.epi = TC_EPI_PARTIAL;
    a.stages = ring_stages(1, 1, bn);
    a.ks = 1;
    a.pout = pout; a.pstride = pstride; a.pld = pld;
    a.err = err;
    a.njobs = njobs;
    for (int j = 0; j < njobs; ++j) a.jobs[j] = jobs[j];
    const CUtensorMap& ma = *reinterpret_cast<const CUtensorMap*>(A.bytes);
    const CUtensorMap& mb = *reinterpret_cast<const CUtensorMap*>(B.bytes);
    // CTA pairs as in tc_gemm: 256-row tiles, half of B per CTA, two K slices per stage
    const bool pair = pair_on && a.mt >= 2 && B.has_half && pair_clusters() > 0;
    if (!pair) {
        const dim3 grid(grid_of(a.mt * a.nt * njobs));
        k_tc_gemm<0, 1, 1, 1><<<grid, NT, smem_for(1, 1, bn), s>>>(ma, mb, mb, ma, a);
        return 0;
    }
    a.ks = 2;
    const size_t sl = stage_stride(1, 1, bn / 2);
    a.stages = (int)std::min<size_t>((kSmemMax - kSmemFixed) / (2 * sl), kMaxStages);
    a.idesc = (a.idesc & ~(0x1Fu << 24)) | ((uint32_t)((2 * BM) >> 4) << 24);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(2 * std::max(1, std::min(((a.mt + 1) / 2) * a.nt * njobs, pair_clusters())));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = kSmemFixed + (size_t)a.stages * 2 * sl;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const CUtensorMap& mbh = *reinterpret_cast<const CUtensorMap*>(B.half);
    return cudaLaunchKernelEx(&cfg, k_tc_gemm<0, 1, 1, 2>, ma, mbh, mbh, ma, a) == cudaSuccess ? 0 : -7;
}

}  // namespace kglm
