// Node-batch layout (§4.2, Fig. 2 "padding"): the CSR fixing lists of a batch
// become two bit masks per node (J1 and J0, ceil(p/32) words each), the
// reduced budget kbar = k - |J1| and the free count pf = p - |J0| - |J1|.
// Coordinates outside Jf are the padded entries of Fig. 2: the prox and
// certificate kernels skip them instead of sorting sentinel keys.  Also: warm
// starts from the device pool, pool stores, the pruning test of §3 and the
// per-node bookkeeping of the periodic certificate.
#include "common.cuh"
#include "engine.h"

namespace kglm {
namespace {

__global__ void k_set_bits(int nnz, const int* __restrict__ ptr, int m, const int* __restrict__ idx, int W,
                           int p, uint32_t* __restrict__ mask, int* err) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    if (idx[t] < 0 || idx[t] >= p) {                  // out of range: flag and skip
        if (err) atomicOr(err, 1);
        return;
    }
    // node of entry t: largest b with ptr[b] <= t (binary search over m+1 offsets)
    int lo = 0, hi = m;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ptr[mid] <= t) lo = mid; else hi = mid;
    }
    const int j = idx[t];
    atomicOr(&mask[(size_t)lo * W + (j >> 5)], 1u << (j & 31));
}

// Device-side checks of a pushed batch (CSR offsets, |J1| <= k, no repeats,
// J0 and J1 disjoint) after the masks are built: a repeat collapses a bit, so
// it shows up as a popcount below the list length.
__global__ void k_validate(int m, int k, int W, int nnz_in, int nnz_out, const int* in_ptr, const int* out_ptr,
                           const uint32_t* in_mask, const uint32_t* out_mask, int* err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    int bad = 0;
    const int n1 = in_ptr[b + 1] - in_ptr[b], n0 = out_ptr[b + 1] - out_ptr[b];
    if (b == 0 && (in_ptr[0] != 0 || out_ptr[0] != 0)) bad = 1;
    if (b == m - 1 && (in_ptr[m] != nnz_in || out_ptr[m] != nnz_out)) bad = 1;
    if (n1 < 0 || n0 < 0 || n1 > k) bad = 1;
    int c1 = 0, c0 = 0;
    for (int w = 0; w < W; ++w) {
        const uint32_t a = in_mask[(size_t)b * W + w], o = out_mask[(size_t)b * W + w];
        if (a & o) bad = 1;
        c1 += __popc(a);
        c0 += __popc(o);
    }
    if (c1 != n1 || c0 != n0) bad = 1;
    if (bad) atomicOr(err, 2);
}

#if KGLM_CHECKS
// The bounds-checked build's self-test: a write one past the end of buf (len
// entries) through the checked path; the check catches it and skips the write.
// Compiled only into that build: elsewhere the guard does not check.
__global__ void k_check_probe(int* buf, int len, int* word) {
    const int idx = len + (int)threadIdx.x;
    if (kglm_check(idx < len, word, kChkSelf)) buf[idx] = 0;
}
#endif

__global__ void k_check_slots(int m, const int* slot, int nslots, int* err) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < m && (slot[b] < -1 || slot[b] >= nslots)) atomicOr(err, 4);
}

__global__ void k_counts(int m, int p, int k, const int* in_ptr, const int* out_ptr, int* kbar, int* pf) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    const int n1 = in_ptr[b + 1] - in_ptr[b], n0 = out_ptr[b + 1] - out_ptr[b];
    kbar[b] = k - n1;
    pf[b] = p - n1 - n0;
}

template <typename T>
__global__ void k_warm(int m, int p, int W, const int* slot, int nslots, const T* pool, const double* warmB,
                       const uint32_t* out_mask, T* B, T* V, void* Vop, float* Vop_lo, int op_ld, int op_bf16) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)m * p) return;
    const int b = (int)(t / p), j = (int)(t % p);
    T w = T(0);
    const int s = slot ? slot[b] : -1;
    if (s >= 0 && s < nslots) w = pool[(size_t)s * p + j];
    else if (warmB) w = T(warmB[t]);
    if ((out_mask[(size_t)b * W + (j >> 5)] >> (j & 31)) & 1u) w = T(0);
    B[t] = w;
    V[t] = w;
    if (Vop) store_operand2(Vop, Vop_lo, (size_t)b * op_ld + j, (float)w, op_bf16);
}

// hi = operand(x), lo = operand(x - hi) (x - hi is exact in FP64)
__global__ void k_convert_pad(const double* in, int rows, int cols, int ld_in, void* out, int ld_out, int to_bf16,
                              void* lo) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)rows * ld_out) return;
    const int r = (int)(t / ld_out), c = (int)(t % ld_out);
    const double v = c < cols ? in[(size_t)r * ld_in + c] : 0.0;
    double hi;
    if (to_bf16) {
        const __nv_bfloat16 h = __double2bfloat16(v);
        static_cast<__nv_bfloat16*>(out)[t] = h;
        hi = (double)__bfloat162float(h);
    } else {
        const float h = to_tf32((float)v);
        static_cast<float*>(out)[t] = h;
        hi = (double)h;
    }
    if (lo) {
        const double d = v - hi;
        if (to_bf16) static_cast<__nv_bfloat16*>(lo)[t] = __double2bfloat16(d);
        else static_cast<float*>(lo)[t] = to_tf32((float)d);
    }
}

__global__ void k_convert_pad_f32(const float* in, int rows, int cols, void* out, int ld_out, int to_bf16,
                                  float* lo) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)rows * ld_out) return;
    const int r = (int)(t / ld_out), c = (int)(t % ld_out);
    store_operand2(out, lo, t, c < cols ? in[(size_t)r * cols + c] : 0.f, to_bf16);
}

__global__ void k_node_init(int m, double t0, double* tmom, int* active, float* hint) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    tmom[b] = t0;
    active[b] = 1;
    if (hint) hint[2 * b] = hint[2 * b + 1] = 0.f;
}

template <typename T>
__global__ void k_pool_store(int count, int p, const int* rows, const int* slots, const T* B, T* pool) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)count * p) return;
    const int c = (int)(t / p), j = (int)(t % p);
    pool[(size_t)slots[c] * p + j] = B[(size_t)rows[c] * p + j];
}

__global__ void k_prune(int m, const double* lb, double thr, uint8_t* pruned) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m) return;
    pruned[b] = lb[b] >= thr ? 1 : 0;
}

// At a certificate check: keep the best bound; freeze nodes that are pruned
// (LB >= UB - delta) or whose relative gap is below gap_rtol.
__global__ void k_check(int m, const double* lb_now, const double* primal_now, double* lb_best,
                        double* primal_last, int* active, int* iters_done, int it, double ub_thr,
                        double gap_rtol) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= m || !active[b]) return;
    const double lb = fmax(lb_best[b], lb_now[b]);
    lb_best[b] = lb;
    primal_last[b] = primal_now[b];
    const double ph = primal_now[b];
    if (lb >= ub_thr || ph - lb <= gap_rtol * fmax(1.0, fabs(ph))) {
        active[b] = 0;
        iters_done[b] = it;
    }
}

__global__ void k_f64_to_f32(const double* in, float* out, size_t n) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (float)in[t];
}
// out (cols x rows) = in (rows x cols)^T, both row-major: 32 x 32 tiles through shared
// memory (one padded column against bank conflicts), 32 x 8 threads.
__global__ void k_transpose_f64(const double* in, double* out, size_t rows, size_t cols) {
    __shared__ double t[32][33];
    const size_t r0 = (size_t)blockIdx.x * 32, c0 = (size_t)blockIdx.y * 32;   // rows on x (up to 2^31 tiles)
    for (int k = threadIdx.y; k < 32; k += 8) {
        const size_t r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[k][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const size_t c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[c * rows + r] = t[threadIdx.x][k];
    }
}
__global__ void k_f32_to_f64(const float* in, double* out, size_t n) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = (double)in[t];
}

inline unsigned blocks(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int layout_masks(cudaStream_t s, int m, int p, int W, int k, const int* in_ptr, const int* in_idx,
                 const int* out_ptr, const int* out_idx, uint32_t* in_mask, uint32_t* out_mask,
                 int* kbar, int* pf, int nnz_in, int nnz_out, int* err) {
    int launches = 1;
    cudaMemsetAsync(in_mask, 0, sizeof(uint32_t) * (size_t)m * W, s);
    cudaMemsetAsync(out_mask, 0, sizeof(uint32_t) * (size_t)m * W, s);
    if (nnz_in > 0) {
        k_set_bits<<<blocks(nnz_in, 256), 256, 0, s>>>(nnz_in, in_ptr, m, in_idx, W, p, in_mask, err);
        ++launches;
    }
    if (nnz_out > 0) {
        k_set_bits<<<blocks(nnz_out, 256), 256, 0, s>>>(nnz_out, out_ptr, m, out_idx, W, p, out_mask, err);
        ++launches;
    }
    k_counts<<<blocks(m, 256), 256, 0, s>>>(m, p, k, in_ptr, out_ptr, kbar, pf);
    return launches;
}

int layout_validate(cudaStream_t s, int m, int k, int W, int nnz_in, int nnz_out, const int* in_ptr,
                    const int* out_ptr, const uint32_t* in_mask, const uint32_t* out_mask, const int* slot,
                    int nslots, int* err) {
    k_validate<<<blocks(m, 128), 128, 0, s>>>(m, k, W, nnz_in, nnz_out, in_ptr, out_ptr, in_mask, out_mask, err);
    if (slot) k_check_slots<<<blocks(m, 256), 256, 0, s>>>(m, slot, nslots, err);
    return slot ? 2 : 1;
}

int layout_warm(cudaStream_t s, int m, int p, int W, int is_f64, const int* slot, int nslots, const void* pool,
                const double* warmB, const uint32_t* out_mask, void* B, void* V, void* Vop, float* Vop_lo, int op_ld,
                int op_bf16, double* tmom, int* active, float* hint) {
    const size_t n = (size_t)m * p;
    if (is_f64)
        k_warm<double><<<blocks(n, 256), 256, 0, s>>>(m, p, W, slot, nslots, (const double*)pool, warmB, out_mask,
                                                      (double*)B, (double*)V, Vop, Vop_lo, op_ld, op_bf16);
    else
        k_warm<float><<<blocks(n, 256), 256, 0, s>>>(m, p, W, slot, nslots, (const float*)pool, warmB, out_mask,
                                                     (float*)B, (float*)V, Vop, Vop_lo, op_ld, op_bf16);
    // t_1 = 1 (Beck and Teboulle): the first extrapolation, after x_1, takes no momentum
    k_node_init<<<blocks(m, 256), 256, 0, s>>>(m, 1.0, tmom, active, hint);
    return 2;
}

void convert_pad(cudaStream_t s, const double* in, int rows, int cols, int ld_in, void* out, int ld_out, int to_bf16,
                 void* lo) {
    const size_t n = (size_t)rows * ld_out;
    if (n) k_convert_pad<<<blocks(n, 256), 256, 0, s>>>(in, rows, cols, ld_in, out, ld_out, to_bf16, lo);
}

void convert_pad_f32(cudaStream_t s, const float* in, int rows, int cols, void* out, int ld_out, int to_bf16,
                     float* lo) {
    const size_t n = (size_t)rows * ld_out;
    if (n) k_convert_pad_f32<<<blocks(n, 256), 256, 0, s>>>(in, rows, cols, out, ld_out, to_bf16, lo);
}

void pool_store(cudaStream_t s, int count, int p, int is_f64, const int* rows, const int* slots, const void* B,
                void* pool) {
    const size_t n = (size_t)count * p;
    if (n == 0) return;
    if (is_f64)
        k_pool_store<double><<<blocks(n, 256), 256, 0, s>>>(count, p, rows, slots, (const double*)B, (double*)pool);
    else
        k_pool_store<float><<<blocks(n, 256), 256, 0, s>>>(count, p, rows, slots, (const float*)B, (float*)pool);
}

void prune_launch(cudaStream_t s, int m, const double* lb, double thr, uint8_t* pruned) {
    if (m > 0) k_prune<<<blocks(m, 256), 256, 0, s>>>(m, lb, thr, pruned);
}

void check_update(cudaStream_t s, int m, const double* lb_now, const double* primal_now, double* lb_best,
                  double* primal_last, int* active, int* iters_done, int it, double ub_thr, double gap_rtol) {
    if (m > 0)
        k_check<<<blocks(m, 256), 256, 0, s>>>(m, lb_now, primal_now, lb_best, primal_last, active, iters_done, it,
                                               ub_thr, gap_rtol);
}

#if KGLM_CHECKS
void check_probe(cudaStream_t s, int* buf, int len, int* word) { k_check_probe<<<1, 1, 0, s>>>(buf, len, word); }
#endif

void convert_f64_to_f32(cudaStream_t s, const double* in, float* out, size_t count) {
    if (count) k_f64_to_f32<<<blocks(count, 256), 256, 0, s>>>(in, out, count);
}

void transpose_f64(cudaStream_t s, const double* in, double* out, size_t rows, size_t cols) {
    if (rows == 0 || cols == 0) return;
    const dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
    k_transpose_f64<<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols);
}

void convert_to_f64(cudaStream_t s, const void* in, int is_f64, double* out, size_t count) {
    if (!count) return;
    if (is_f64) cudaMemcpyAsync(out, in, count * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else k_f32_to_f64<<<blocks(count, 256), 256, 0, s>>>((const float*)in, out, count);
}

}  // namespace kglm
