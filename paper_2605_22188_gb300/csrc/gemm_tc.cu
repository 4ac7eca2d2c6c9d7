// Tensor-core products of the BF16 and TF32 modes: S = X V (with the
// loss/link fused) and G = X^T R of §4.2 Eq. (gradient_matrix_form), on the
// fifth-generation tensor cores of sm_103a.
//
// C[r][c] = sum_k A[r][k] B[c][k] with both operands K-contiguous.  One CTA
// computes a 128 x BN tile (BN <= 256, a multiple of 16) of one K range:
//   warp 0, lane 0   TMA producer: 128-byte-swizzled K slices of A and B
//                    (cp.async.bulk.tensor.2d) into a 4-stage ring;
//   warp 1, lane 0   MMA issuer: tcgen05.mma.cta_group::1 (kind::f16 with BF16
//                    operands, or kind::tf32), FP32 accumulator in tensor
//                    memory; tcgen05.commit frees a stage / signals the tile;
//   warps 0-7        epilogue: tcgen05.ld of the accumulator (warp w reads
//                    TMEM lanes 32(w%4).. , i.e. tile rows, and every other
//                    32-column chunk), then the link, a plain store or a
//                    split-K partial.
// The B operand can be given as two parts (hi + lo, both multiplied into the
// same accumulator): the engine does this for X in S = X V, so that X enters
// one of the two products of an iteration with ~16 (BF16) or ~22 (TF32) bits.
// Were X rounded in both products, the fixed point would solve the normal
// equations of X~ = X + E, whose Gram matrix carries the positive diagonal
// E^T E ~ n u^2 E[x^2]: a ridge shift comparable to lambda2 at n in the
// thousands.  FP32 operands reach kind::tf32 rounded to nearest (the tensor
// core would otherwise truncate them, a bias toward zero).
// Split-K uses the scheme of the CUDA-core GEMM: partial tiles in scratch,
// the last CTA of a tile (arrival counter) sums them in fixed order.
// Every mbarrier wait is bounded; a wait that runs out sets an error flag,
// the CTA still drains its MMAs and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

constexpr int BM = 128;                 // rows per tile (one UMMA M = 128)
constexpr int ROWB = 128;               // bytes of K per stage and row (one swizzle row)
constexpr int MAXBN = 256;
constexpr int NT = 256;                 // eight warps
constexpr uint32_t STAGE_A = BM * ROWB;
constexpr uint32_t STAGE_B = MAXBN * ROWB;
constexpr uint32_t TMEM_COLS = 256;
// NB = 1: one B operand, four stages; NB = 2: B given as hi + lo parts
// (both multiplied into the same accumulator), two stages.
template <int NB> constexpr int stages() { return NB == 1 ? 4 : 2; }
template <int NB> constexpr size_t smem_bytes() { return 1024 + stages<NB>() * (STAGE_A + NB * STAGE_B) + 256; }
constexpr uint32_t WAIT_LIMIT = 1u << 22;   // try_wait rounds before a wait gives up

// ------------------------------------------------------------------ arguments and epilogues

struct TcArgs {
    int M, N;                 // output rows (A rows) and columns (B rows)
    int bn;                   // columns per tile, multiple of 16, <= MAXBN
    int nkb, kb_per_split;    // K in 128-byte slices, slices per CTA
    uint32_t idesc;           // instruction descriptor
    int epi;                  // TC_EPI_*
    int round_tf32;           // round FP32 link outputs to TF32 (nearest) for the next product
    float* pout;              // TC_EPI_PARTIAL: slice z at pout + z * pstride, row stride pld
    size_t pstride;
    int pld;
    void* out;
    int ldo;
    const float* y;
    int loss;
    float* part;
    int* counters;
    int* err;
    int njobs;                // > 0: job z = blockIdx.z takes its own K ranges and slice
    TcJob jobs[kTcMaxJobs];
};

__device__ __forceinline__ float tf32_rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Loss derivative for operands that are rounded to BF16/TF32 next: fast
// exponential and reciprocal (relative error far below the operand rounding).
__device__ __forceinline__ float dloss_fast(float s, float y, int kind) {
    return kind == kLSQ ? 2.0f * (s - y) : -y * __frcp_rn(1.0f + __expf(y * s));
}

// Writes columns c0 .. c0+31 of output row r (columns >= N are skipped); ys:
// the tile's y values staged in shared memory (index c0 - n0 + j); zs: the
// slice of a partial product.
__device__ __forceinline__ void tc_epilogue(const TcArgs& a, int r, int c0, const float (&v)[32], const float* ys,
                                            int zs) {
    if (r >= a.M) return;
    if (a.epi == TC_EPI_PARTIAL) {
        float* o = a.pout + (size_t)zs * a.pstride + (size_t)r * a.pld;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (c0 + j < a.N) o[c0 + j] = v[j];
    } else if (a.epi == TC_EPI_STORE_F32) {
        float* o = static_cast<float*>(a.out) + (size_t)r * a.ldo;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (c0 + j < a.N) o[c0 + j] = v[j];
    } else if (a.epi == TC_EPI_LINK_F32) {
        float* o = static_cast<float*>(a.out) + (size_t)r * a.ldo;
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (c0 + j < a.N) {
                const float d = dloss_fast(v[j], ys[j], a.loss);
                o[c0 + j] = a.round_tf32 ? tf32_rn(d) : d;
            }
    } else {
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(a.out) + (size_t)r * a.ldo;
        if (c0 + 32 <= a.N && (a.ldo % 8) == 0) {
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
                __nv_bfloat162 h[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    h[q] = __floats2bfloat162_rn(dloss_fast(v[j + 2 * q], ys[j + 2 * q], a.loss),
                                                 dloss_fast(v[j + 2 * q + 1], ys[j + 2 * q + 1], a.loss));
                *reinterpret_cast<uint4*>(o + c0 + j) = *reinterpret_cast<const uint4*>(h);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (c0 + j < a.N) o[c0 + j] = __float2bfloat16(dloss_fast(v[j], ys[j], a.loss));
        }
    }
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

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
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

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
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

template <int KIND, int NB>
__global__ void __launch_bounds__(NT, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB,
                                                   const __grid_constant__ CUtensorMap tmB2,
                                                   const __grid_constant__ TcArgs a) {
    constexpr int STAGES = stages<NB>();
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + STAGES * STAGE_A;                    // stage s: B at s, B2 (NB = 2) at STAGES + s
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + NB * STAGES * STAGE_B);   // full[S], empty[S], accum
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    __shared__ int s_last;
    __shared__ float ys[MAXBN + 32];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * a.bn;
    // K slices of this CTA: a split of [0, nkb), or the job's own ranges of A and B
    int ka0, kbb0, nloc, zs;
    if (a.njobs > 0) {
        const TcJob& jb = a.jobs[blockIdx.z];
        ka0 = jb.ka; kbb0 = jb.kb; nloc = jb.nkb; zs = jb.slice;
    } else {
        ka0 = kbb0 = blockIdx.z * a.kb_per_split;
        nloc = min(a.nkb, ka0 + a.kb_per_split) - ka0;
        zs = blockIdx.z;
    }
    constexpr int KE = KIND == 0 ? 64 : 32;          // elements per 128-byte row
    const uint32_t stage_bytes = STAGE_A + (uint32_t)NB * a.bn * ROWB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * STAGES + 1; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer
        for (int i = 0; i < nloc; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(smem_u32(&bars[STAGES + s]), ph ^ 1u, a.err)) break;
            const uint32_t full = smem_u32(&bars[s]);
            mbar_expect_tx(full, stage_bytes);
            const int kxa = (ka0 + i) * KE, kxb = (kbb0 + i) * KE;
            tma_load_2d(smem_u32(sA + s * STAGE_A), &tmA, kxa, m0, full);
            tma_load_2d(smem_u32(sB + s * STAGE_B), &tmB, kxb, n0, full);
            if (NB == 2) tma_load_2d(smem_u32(sB + (STAGES + s) * STAGE_B), &tmB2, kxb, n0, full);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int i = 0; i < nloc; ++i) {
            const int s = i % STAGES;
            const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
            if (!mbar_wait(smem_u32(&bars[s]), ph, a.err)) break;
            tc_fence_after();
            const uint32_t aa = smem_u32(sA + s * STAGE_A), bb = smem_u32(sB + s * STAGE_B);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {   // four MMAs of 32 bytes of K each (per B part)
                umma<KIND>(tmem, smem_desc(aa + kk * 32), smem_desc(bb + kk * 32), a.idesc, (i > 0 || kk > 0) ? 1u : 0u);
                if (NB == 2) {
                    const uint32_t b2 = smem_u32(sB + (STAGES + s) * STAGE_B);
                    umma<KIND>(tmem, smem_desc(aa + kk * 32), smem_desc(b2 + kk * 32), a.idesc, 1u);
                }
            }
            umma_commit(smem_u32(&bars[STAGES + s]));   // stage s is free once these MMAs finish
        }
        umma_commit(smem_u32(&bars[2 * STAGES]));       // the accumulator is complete (or drained)
    }
    __syncwarp();

    // epilogue: all eight warps; warp w reads TMEM lanes 32*(w%4).. (tile rows)
    // and the 32-column chunks of parity w/4
    if (a.y != nullptr)
        for (int c = threadIdx.x; c < a.bn + 32; c += NT) ys[c] = (n0 + c < a.N) ? a.y[n0 + c] : 0.f;
    __syncthreads();
    // warp-uniform: tcgen05.ld below is .sync.aligned
    const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bars[2 * STAGES]), 0u, a.err) && nloc > 0);
    tc_fence_after();
    const int quad = warp & 3, half = warp >> 2;
    const int row = m0 + quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16);
    // split-K with the last-CTA reduction (TC_EPI_PARTIAL keeps every slice instead)
    const bool split = gridDim.z > 1 && a.epi != TC_EPI_PARTIAL;
    const int ntile = gridDim.x * gridDim.y;
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    if (ok) {
        for (int c = half * 32; c < a.bn; c += 64) {
            float v[32];
            tmem_ld32(tl + (uint32_t)c, v);
            if (!split) {
                tc_epilogue(a, row, n0 + c, v, ys + c, zs);
            } else {
                float* my = a.part + (((size_t)blockIdx.z * ntile + tile) * BM + quad * 32 + lane) * MAXBN + c;
#pragma unroll
                for (int q = 0; q < 32; q += 4) *reinterpret_cast<float4*>(my + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
            }
        }
    }
    tc_fence_before();
    if (split) {
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(&a.counters[tile], 1) == (int)gridDim.z - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int c = half * 32; c < a.bn; c += 64) {
                float v[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = 0.f;
                for (int s = 0; s < (int)gridDim.z; ++s) {
                    const float* ps = a.part + (((size_t)s * ntile + tile) * BM + quad * 32 + lane) * MAXBN + c;
#pragma unroll
                    for (int q = 0; q < 32; q += 4) {
                        const float4 x = __ldcg(reinterpret_cast<const float4*>(ps + q));
                        v[q] += x.x; v[q + 1] += x.y; v[q + 2] += x.z; v[q + 3] += x.w;
                    }
                }
                tc_epilogue(a, row, n0 + c, v, ys + c, 0);
            }
            if (threadIdx.x == 0) a.counters[tile] = 0;
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
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

template <int KIND, int NB>
int set_smem_attr() {
    static int done = 0;
    if (!done) {
        if (cudaFuncSetAttribute(k_tc_gemm<KIND, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes<NB>()) != cudaSuccess)
            return -1;
        done = 1;
    }
    return 0;
}

}  // namespace

int tc_prepare() {
    return set_smem_attr<0, 1>() | set_smem_attr<0, 2>() | set_smem_attr<1, 1>() | set_smem_attr<1, 2>();
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
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(out->bytes), is_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

int tc_tile_cols(int N) { return N >= MAXBN ? MAXBN : ((N + 15) / 16) * 16; }
int tc_tile_cols_wide(int N) { return N > MAXBN ? 128 : tc_tile_cols(N); }

size_t tc_scratch_bytes() { return (size_t)3 * 152 * BM * MAXBN * sizeof(float); }
int tc_scratch_counters() { return 3 * 152; }

int tc_gemm(cudaStream_t s, const TcMap& A, const TcMap& B, const TcMap* B2, const TcGemm& g,
            const GemmScratch* scr) {
    if (g.M <= 0 || g.N <= 0) return 0;
    if (g.bn < 16 || g.bn > MAXBN || g.bn % 16 != 0) return -4;
    const int nb = B2 ? 2 : 1;
    const int rc = g.kind == 0 ? (nb == 1 ? set_smem_attr<0, 1>() : set_smem_attr<0, 2>())
                               : (nb == 1 ? set_smem_attr<1, 1>() : set_smem_attr<1, 2>());
    if (rc) return -5;
    const int KE = g.kind == 0 ? 64 : 32;
    TcArgs a{};
    a.M = g.M; a.N = g.N; a.bn = g.bn;
    a.nkb = (g.K + KE - 1) / KE;
    const int gx = (g.N + g.bn - 1) / g.bn, gy = (g.M + BM - 1) / BM;
    const int tiles = gx * gy;
    // split-K: at least 4 slices of K per CTA, at most one wave of CTAs
    int splits = 1;
    if (g.epi == TC_EPI_PARTIAL) {
        splits = std::max(1, std::min(g.max_splits, std::min((a.nkb + 3) / 4, std::max(1, 152 / tiles))));
    } else if (tiles < 152 && scr && scr->part && scr->counters && scr->n_counters >= tiles) {
        splits = std::min((a.nkb + 3) / 4, std::max(1, 152 / tiles));
        const size_t need = (size_t)splits * tiles * BM * MAXBN * sizeof(float);
        if (need > scr->part_bytes) splits = (int)std::max<size_t>(1, scr->part_bytes / ((size_t)tiles * BM * MAXBN * sizeof(float)));
    }
    a.kb_per_split = (a.nkb + splits - 1) / splits;
    splits = (a.nkb + a.kb_per_split - 1) / a.kb_per_split;
    if (g.splits_used) *g.splits_used = splits;
    a.pout = g.pout; a.pstride = g.pstride; a.pld = g.pld;
    // instruction descriptor: D F32 (bits 4-5 = 1), A/B format (bits 7-9, 10-12:
    // BF16 = 1 for kind::f16, TF32 = 2 for kind::tf32), K-major A and B, N>>3 at
    // bit 17, M>>4 at bit 24
    const uint32_t ab = g.kind == 0 ? 1u : 2u;
    a.idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(g.bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    a.epi = g.epi; a.out = g.out; a.ldo = g.ldo; a.y = g.y; a.loss = g.loss;
    a.round_tf32 = g.kind == 1;
    a.part = splits > 1 ? static_cast<float*>(scr->part) : nullptr;
    a.counters = splits > 1 ? scr->counters : nullptr;
    a.err = g.err;
    const CUtensorMap& ma = *reinterpret_cast<const CUtensorMap*>(A.bytes);
    const CUtensorMap& mb = *reinterpret_cast<const CUtensorMap*>(B.bytes);
    const CUtensorMap& mb2 = *reinterpret_cast<const CUtensorMap*>((B2 ? B2 : &B)->bytes);
    dim3 grid(gx, gy, splits);
    if (g.kind == 0) {
        if (nb == 1) k_tc_gemm<0, 1><<<grid, NT, smem_bytes<1>(), s>>>(ma, mb, mb2, a);
        else k_tc_gemm<0, 2><<<grid, NT, smem_bytes<2>(), s>>>(ma, mb, mb2, a);
    } else {
        if (nb == 1) k_tc_gemm<1, 1><<<grid, NT, smem_bytes<1>(), s>>>(ma, mb, mb2, a);
        else k_tc_gemm<1, 2><<<grid, NT, smem_bytes<2>(), s>>>(ma, mb, mb2, a);
    }
    return 0;
}

int tc_gemm_jobs(cudaStream_t s, const TcMap& A, const TcMap& B, int M, int N, int bn, const TcJob* jobs,
                 int njobs, float* pout, size_t pstride, int pld, int* err) {
    if (M <= 0 || N <= 0 || njobs <= 0) return 0;
    if (bn < 16 || bn > MAXBN || bn % 16 != 0 || njobs > kTcMaxJobs) return -4;
    if (set_smem_attr<0, 1>()) return -5;
    TcArgs a{};
    a.M = M; a.N = N; a.bn = bn;
    a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
    a.epi = TC_EPI_PARTIAL;
    a.pout = pout; a.pstride = pstride; a.pld = pld;
    a.err = err;
    a.njobs = njobs;
    for (int j = 0; j < njobs; ++j) a.jobs[j] = jobs[j];
    const CUtensorMap& ma = *reinterpret_cast<const CUtensorMap*>(A.bytes);
    const CUtensorMap& mb = *reinterpret_cast<const CUtensorMap*>(B.bytes);
    dim3 grid((N + bn - 1) / bn, (M + BM - 1) / BM, njobs);
    k_tc_gemm<0, 1><<<grid, NT, smem_bytes<1>(), s>>>(ma, mb, mb, a);
    return 0;
}

}  // namespace kglm
