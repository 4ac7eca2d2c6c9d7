// CUDA-core GEMMs of the FP64 and FP32 paths: S = X B and G = X^T R of §4.2
// Eq. (gradient_matrix_form) in the node-major layout, with the loss/link of
// §4.2 fused into the epilogue of S (R = dl(S, y) is written, S is not).
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

// C[r][c] = sum_k A[r][k] B[c][k]; tile BM x BN per CTA, TM x TN per thread.
template <typename T, int BM, int BN, int BK, int TM, int TN, typename Epi>
__global__ __launch_bounds__((BM / TM) * (BN / TN)) void k_gemm_nt(int R, int C, int K,
                                                                   const T* __restrict__ A, int lda,
                                                                   const T* __restrict__ B, int ldb,
                                                                   Epi epi) {
    constexpr int NTX = BN / TN, NTY = BM / TM, NT = NTX * NTY;
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid % NTX, ty = tid / NTX;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        for (int e = tid; e < BM * BK; e += NT) {
            const int rr = e / BK, kk = e % BK, gr = r0 + rr, gk = k0 + kk;
            As[kk][rr] = (gr < R && gk < K) ? A[(size_t)gr * lda + gk] : T(0);
        }
        for (int e = tid; e < BN * BK; e += NT) {
            const int cc = e / BK, kk = e % BK, gc = c0 + cc, gk = k0 + kk;
            Bs[kk][cc] = (gc < C && gk < K) ? B[(size_t)gc * ldb + gk] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[TM], b[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * NTY];
#pragma unroll
            for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * NTX];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int r = r0 + ty + i * NTY, c = c0 + tx + j * NTX;
            if (r < R && c < C) epi(r, c, acc[i][j]);
        }
}

template <typename T, typename Epi>
void launch(cudaStream_t s, int R, int C, int K, const T* A, int lda, const T* B, int ldb, Epi epi) {
    if (R <= 0 || C <= 0) return;
    if constexpr (sizeof(T) == 8) {
        constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
        dim3 grid((C + BN - 1) / BN, (R + BM - 1) / BM);
        k_gemm_nt<T, BM, BN, BK, TM, TN, Epi><<<grid, (BM / TM) * (BN / TN), 0, s>>>(R, C, K, A, lda, B, ldb, epi);
    } else {
        constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
        dim3 grid((C + BN - 1) / BN, (R + BM - 1) / BM);
        k_gemm_nt<T, BM, BN, BK, TM, TN, Epi><<<grid, (BM / TM) * (BN / TN), 0, s>>>(R, C, K, A, lda, B, ldb, epi);
    }
}

}  // namespace

void gemm_nt_f64(cudaStream_t s, int R, int C, int K, const double* A, int lda, const double* B, int ldb,
                 double* out, int ldo) {
    launch<double>(s, R, C, K, A, lda, B, ldb, EpiStore<double>{out, ldo});
}
void gemm_nt_f32(cudaStream_t s, int R, int C, int K, const float* A, int lda, const float* B, int ldb,
                 float* out, int ldo) {
    launch<float>(s, R, C, K, A, lda, B, ldb, EpiStore<float>{out, ldo});
}
void gemm_link_f64(cudaStream_t s, int m, int n, int p, const double* V, const double* X, const double* y,
                   int kind, double* out) {
    launch<double>(s, m, n, p, V, p, X, p, EpiLink<double>{out, n, y, kind});
}
void gemm_link_f32(cudaStream_t s, int m, int n, int p, const float* V, const float* X, const float* y,
                   int kind, float* out) {
    launch<float>(s, m, n, p, V, p, X, p, EpiLink<float>{out, n, y, kind});
}

}  // namespace kglm
