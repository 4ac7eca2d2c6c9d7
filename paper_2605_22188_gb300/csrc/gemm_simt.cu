// CUDA-core GEMMs of the FP64 and FP32 paths: S = X B and G = X^T R of §4.2
// Eq. (gradient_matrix_form) in the node-major layout, with the loss/link of
// §4.2 fused into the epilogue of S (R = dl(S, y) is written, S is not).
//
// C[r][c] = sum_k A[r][k] B[c][k]: both operands are K-contiguous (node rows
// of V or R against rows of X or X^T).  Each CTA computes a BM x BN tile with
// TM x TN contiguous outputs per thread; the next K slice is prefetched into
// registers while the current one is multiplied from shared memory.
//
// Split-K: when the output has too few tiles to fill the GPU (X^T R is only
// m x p while K = n), the K range is cut into `splits` chunks (grid z).  Each
// CTA stores its partial tile in a scratch buffer, fences, and increments the
// tile's arrival counter; the CTA that arrives last sums the partials in the
// fixed order s = 0..splits-1 (so the result does not depend on arrival
// order), applies the epilogue and sets the counter back to 0.  No CTA waits
// for another.
#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

template <typename T>
struct EpiStore {
    T* out;
    int ldo;
    __device__ __forceinline__ void operator()(int r, int c, T v) const { out[(size_t)r * ldo + c] = v; }
};

template <typename T>
struct EpiLink {
    T* out;
    int ldo;
    const T* y;
    int kind;
    __device__ __forceinline__ void operator()(int r, int c, T v) const {
        out[(size_t)r * ldo + c] = dloss(v, y[c], kind);
    }
};

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double2; };   // 16-byte vector

template <typename T, int BM, int BN, int BK, int TM, int TN, bool VEC, typename Epi>
__global__ __launch_bounds__((BM / TM) * (BN / TN)) void k_gemm_nt(int R, int C, int K, const T* __restrict__ A,
                                                                   int lda, const T* __restrict__ B, int ldb,
                                                                   Epi epi, int kchunk, T* __restrict__ part,
                                                                   int* __restrict__ counters) {
    constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
    constexpr int VW = 16 / sizeof(T);                 // elements per 16-byte vector
    constexpr int PAD = VW;
    constexpr int AV = BM * BK / VW, BV = BN * BK / VW; // vectors per tile
    constexpr int AL = (AV + NT - 1) / NT, BL = (BV + NT - 1) / NT;
    static_assert(BK % VW == 0, "BK must be a multiple of the vector width");
    __shared__ __align__(16) T As[BK][BM + PAD];
    __shared__ __align__(16) T Bs[BK][BN + PAD];
    __shared__ int s_last;

    const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);

    T ra[AL][VW], rb[BL][VW];
    auto load = [&](int k0) {
#pragma unroll
        for (int l = 0; l < AL; ++l) {
            const int v = tid + l * NT;
            const int row = v / (BK / VW), kk = (v % (BK / VW)) * VW;
            const int gr = r0 + row, gk = k0 + kk;
            if (v < AV) {
                if (VEC && gr < R && gk + VW <= kend) {
                    const auto x = *reinterpret_cast<const typename Vec4<T>::type*>(A + (size_t)gr * lda + gk);
                    const T* px = reinterpret_cast<const T*>(&x);
#pragma unroll
                    for (int q = 0; q < VW; ++q) ra[l][q] = px[q];
                } else {
#pragma unroll
                    for (int q = 0; q < VW; ++q)
                        ra[l][q] = (gr < R && gk + q < kend) ? A[(size_t)gr * lda + gk + q] : T(0);
                }
            }
        }
#pragma unroll
        for (int l = 0; l < BL; ++l) {
            const int v = tid + l * NT;
            const int col = v / (BK / VW), kk = (v % (BK / VW)) * VW;
            const int gc = c0 + col, gk = k0 + kk;
            if (v < BV) {
                if (VEC && gc < C && gk + VW <= kend) {
                    const auto x = *reinterpret_cast<const typename Vec4<T>::type*>(B + (size_t)gc * ldb + gk);
                    const T* px = reinterpret_cast<const T*>(&x);
#pragma unroll
                    for (int q = 0; q < VW; ++q) rb[l][q] = px[q];
                } else {
#pragma unroll
                    for (int q = 0; q < VW; ++q)
                        rb[l][q] = (gc < C && gk + q < kend) ? B[(size_t)gc * ldb + gk + q] : T(0);
                }
            }
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int l = 0; l < AL; ++l) {
            const int v = tid + l * NT;
            if (v < AV) {
                const int row = v / (BK / VW), kk = (v % (BK / VW)) * VW;
#pragma unroll
                for (int q = 0; q < VW; ++q) As[kk + q][row] = ra[l][q];
            }
        }
#pragma unroll
        for (int l = 0; l < BL; ++l) {
            const int v = tid + l * NT;
            if (v < BV) {
                const int col = v / (BK / VW), kk = (v % (BK / VW)) * VW;
#pragma unroll
                for (int q = 0; q < VW; ++q) Bs[kk + q][col] = rb[l][q];
            }
        }
    };

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    if (kbeg < kend) load(kbeg);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        store();
        __syncthreads();
        if (k0 + BK < kend) load(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; i += VW) {
                const auto x = *reinterpret_cast<const typename Vec4<T>::type*>(&As[kk][ty * TM + i]);
                const T* px = reinterpret_cast<const T*>(&x);
#pragma unroll
                for (int q = 0; q < VW; ++q) a[i + q] = px[q];
            }
#pragma unroll
            for (int j = 0; j < TN; j += VW) {
                const auto x = *reinterpret_cast<const typename Vec4<T>::type*>(&Bs[kk][tx * TN + j]);
                const T* px = reinterpret_cast<const T*>(&x);
#pragma unroll
                for (int q = 0; q < VW; ++q) b[j + q] = px[q];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    if (gridDim.z == 1) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int r = r0 + ty * TM + i, c = c0 + tx * TN + j;
                if (r < R && c < C) epi(r, c, acc[i][j]);
            }
        return;
    }
    // split-K: publish the partial tile, the last arriving CTA reduces it
    const int tile = blockIdx.y * gridDim.x + blockIdx.x;
    const int ntile = gridDim.x * gridDim.y;
    T* my = part + ((size_t)blockIdx.z * ntile + tile) * (BM * BN);
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) my[(ty * TM + i) * BN + tx * TN + j] = acc[i][j];
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&counters[tile], 1) == (int)gridDim.z - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int s = 0; s < (int)gridDim.z; ++s) {
        const T* ps = part + ((size_t)s * ntile + tile) * (BM * BN);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] += __ldcg(ps + (ty * TM + i) * BN + tx * TN + j);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int r = r0 + ty * TM + i, c = c0 + tx * TN + j;
            if (r < R && c < C) epi(r, c, acc[i][j]);
        }
    if (tid == 0) counters[tile] = 0;
}

constexpr int kSMs = 152;

template <typename T>
struct Tile;
template <> struct Tile<float> { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };
template <> struct Tile<double> { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };

// Resident CTAs per SM of the tile configuration (2 for the FP32 tile, 128
// registers x 256 threads; queried once from the runtime, with that default).
template <typename T>
int ctas_per_sm();

// Split-K factor: the one whose CTA count best fills whole waves of
// (SMs x resident CTAs), with a small penalty per split for the partial-tile
// traffic; each CTA keeps at least 64 of the K range and the grid stays
// within about two waves (so splits x tiles < 3 x SMs x resident CTAs).
inline int choose_splits(int tiles, int K, int BK, int per_sm) {
    const int slots = kSMs * per_sm;
    if (tiles >= slots) return 1;
    // at least 64 of K per CTA, and at most about two waves of CTAs
    const int max_split = max(1, min(min(64, K / 64), (2 * slots + tiles - 1) / tiles));
    int best = 1;
    double best_score = -1.0;
    for (int s = 1; s <= max_split; ++s) {
        const long ctas = (long)tiles * s;
        const long waves = (ctas + slots - 1) / slots;
        const double eff = (double)ctas / (double)(waves * slots);
        const double score = eff - 0.01 * s;
        if (score > best_score + 1e-12) { best_score = score; best = s; }
    }
    return best;
}

template <typename T>
GemmPlan plan_for(int R, int C, int K) {
    using TL = Tile<T>;
    GemmPlan g{};
    g.gx = (C + TL::BN - 1) / TL::BN;
    g.gy = (R + TL::BM - 1) / TL::BM;
    const int tiles = g.gx * g.gy;
    int splits = choose_splits(tiles, K, TL::BK, ctas_per_sm<T>());
    int kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + TL::BK - 1) / TL::BK * TL::BK;                 // keep vector alignment per chunk
    splits = (K + kchunk - 1) / kchunk;
    g.splits = max(1, splits);
    g.kchunk = kchunk;
    g.part_elems = g.splits > 1 ? (size_t)g.splits * tiles * TL::BM * TL::BN : 0;
    g.tiles = tiles;
    return g;
}

template <typename T, typename Epi>
void launch(cudaStream_t s, int R, int C, int K, const T* A, int lda, const T* B, int ldb, Epi epi,
            const GemmScratch* scr) {
    if (R <= 0 || C <= 0) return;
    using TL = Tile<T>;
    GemmPlan g = plan_for<T>(R, C, K);
    T* part = nullptr;
    int* cnt = nullptr;
    if (g.splits > 1) {
        if (scr == nullptr || scr->part == nullptr || scr->part_bytes < g.part_elems * sizeof(T) ||
            scr->counters == nullptr || scr->n_counters < g.tiles) {
            g.splits = 1;                                               // no scratch: one pass over K
            g.kchunk = K;
        } else {
            part = static_cast<T*>(scr->part);
            cnt = scr->counters;
        }
    }
    if (K <= 0) g.kchunk = 1;
    constexpr int VW = 16 / sizeof(T);
    const bool vec = (lda % VW == 0) && (ldb % VW == 0) && ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0);
    dim3 grid(g.gx, g.gy, g.splits);
    constexpr int NT = (TL::BM / TL::TM) * (TL::BN / TL::TN);
    if (vec)
        k_gemm_nt<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, true, Epi><<<grid, NT, 0, s>>>(
            R, C, K, A, lda, B, ldb, epi, g.kchunk, part, cnt);
    else
        k_gemm_nt<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, false, Epi><<<grid, NT, 0, s>>>(
            R, C, K, A, lda, B, ldb, epi, g.kchunk, part, cnt);
}

// Like launch(), but when the scratch cannot hold the planned partials the
// split factor is lowered to what it holds instead of dropping to one pass.
template <typename T, typename Epi>
void launch_clamped(cudaStream_t s, int R, int C, int K, const T* A, int lda, const T* B, int ldb, Epi epi,
                    const GemmScratch& scr) {
    if (R <= 0 || C <= 0) return;
    using TL = Tile<T>;
    GemmPlan g = plan_for<T>(R, C, K);
    const size_t tile_bytes = (size_t)TL::BM * TL::BN * sizeof(T);
    if (g.splits > 1) {
        const size_t fit = (g.tiles > scr.n_counters || scr.part == nullptr) ? 1
                         : scr.part_bytes / ((size_t)g.tiles * tile_bytes);
        if ((size_t)g.splits > fit) {
            const int splits = (int)(fit < 1 ? 1 : fit);
            int kchunk = (K + splits - 1) / splits;
            kchunk = (kchunk + TL::BK - 1) / TL::BK * TL::BK;
            g.kchunk = kchunk;
            g.splits = (K + kchunk - 1) / kchunk;
        }
    }
    if (g.splits <= 1) {
        g.splits = 1;
        g.kchunk = K > 0 ? K : 1;
    }
    constexpr int VW = 16 / sizeof(T);
    const bool vec = (lda % VW == 0) && (ldb % VW == 0) && ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0);
    dim3 grid(g.gx, g.gy, g.splits);
    constexpr int NT = (TL::BM / TL::TM) * (TL::BN / TL::TN);
    T* part = g.splits > 1 ? static_cast<T*>(scr.part) : nullptr;
    int* cnt = g.splits > 1 ? scr.counters : nullptr;
    if (vec)
        k_gemm_nt<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, true, Epi><<<grid, NT, 0, s>>>(
            R, C, K, A, lda, B, ldb, epi, g.kchunk, part, cnt);
    else
        k_gemm_nt<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, false, Epi><<<grid, NT, 0, s>>>(
            R, C, K, A, lda, B, ldb, epi, g.kchunk, part, cnt);
}

template <typename T>
int ctas_per_sm() {
    // computed once per process (a function-local static initialiser is
    // thread-safe; calls may come from several host threads at once)
    static const int cached = [] {
        using TL = Tile<T>;
        constexpr int NT = (TL::BM / TL::TM) * (TL::BN / TL::TN);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &n, k_gemm_nt<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, true, EpiStore<T>>, NT, 0) != cudaSuccess ||
            n <= 0) {
            cudaGetLastError();
            n = 2;
        }
        return n;
    }();
    return cached;
}

}  // namespace

size_t gemm_scratch_bytes(int is_f64) {
    // splits x tiles < 3 x (SMs x resident CTAs), each partial tile BM x BN
    if (is_f64) return (size_t)3 * kSMs * ctas_per_sm<double>() * Tile<double>::BM * Tile<double>::BN * sizeof(double);
    return (size_t)3 * kSMs * ctas_per_sm<float>() * Tile<float>::BM * Tile<float>::BN * sizeof(float);
}
int gemm_scratch_counters(int is_f64) { return 3 * kSMs * (is_f64 ? ctas_per_sm<double>() : ctas_per_sm<float>()); }

GemmPlan gemm_plan(int R, int C, int K, int is_f64) {
    return is_f64 ? plan_for<double>(R, C, K) : plan_for<float>(R, C, K);
}

void gemm_nt_f64(cudaStream_t s, int R, int C, int K, const double* A, int lda, const double* B, int ldb,
                 double* out, int ldo, const GemmScratch* scr) {
    launch<double>(s, R, C, K, A, lda, B, ldb, EpiStore<double>{out, ldo}, scr);
}
void gemm_nt_f32(cudaStream_t s, int R, int C, int K, const float* A, int lda, const float* B, int ldb,
                 float* out, int ldo, const GemmScratch* scr) {
    launch<float>(s, R, C, K, A, lda, B, ldb, EpiStore<float>{out, ldo}, scr);
}
void gemm_nt_f32_clamped(cudaStream_t s, int R, int C, int K, const float* A, int lda, const float* B, int ldb,
                         float* out, int ldo, const GemmScratch& scr) {
    launch_clamped<float>(s, R, C, K, A, lda, B, ldb, EpiStore<float>{out, ldo}, scr);
}
int gemm_tile_rows_f32() { return Tile<float>::BM; }
int gemm_tile_cols_f32() { return Tile<float>::BN; }
void gemm_link_f64(cudaStream_t s, int m, int n, int p, const double* V, const double* X, const double* y,
                   int kind, double* out, const GemmScratch* scr) {
    launch<double>(s, m, n, p, V, p, X, p, EpiLink<double>{out, n, y, kind}, scr);
}
void gemm_link_f32(cudaStream_t s, int m, int n, int p, const float* V, const float* X, const float* y,
                   int kind, float* out, const GemmScratch* scr) {
    launch<float>(s, m, n, p, V, p, X, p, EpiLink<float>{out, n, y, kind}, scr);
}

}  // namespace kglm
