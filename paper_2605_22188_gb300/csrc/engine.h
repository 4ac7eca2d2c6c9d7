// Internal launchers of the node-bound engine (host side).  All matrices are
// row-major; node-major batch buffers hold one node per row (B[b*p + j]).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "kglm.h"

namespace kglm {

// Split-K scratch of the CUDA-core GEMMs: partial tiles and per-tile arrival
// counters (zero between launches; the reducing CTA resets them).
struct GemmScratch {
    void* part;
    size_t part_bytes;
    int* counters;
    int n_counters;
};
struct GemmPlan {
    int gx, gy, splits, kchunk, tiles;
    size_t part_elems;
};
// Bytes of scratch the launch plan needs are part_elems * sizeof(T).
GemmPlan gemm_plan(int R, int C, int K, int is_f64);
// Scratch that covers every plan (partial bytes and tile counters).
size_t gemm_scratch_bytes(int is_f64);
int gemm_scratch_counters(int is_f64);

// C[r][c] = sum_k A[r*lda + k] * B[c*ldb + k]  (both operands K-contiguous).
// scr may be NULL (then no split-K).
void gemm_nt_f64(cudaStream_t s, int R, int C, int K, const double* A, int lda,
                 const double* B, int ldb, double* out, int ldo, const GemmScratch* scr);
void gemm_nt_f32(cudaStream_t s, int R, int C, int K, const float* A, int lda,
                 const float* B, int ldb, float* out, int ldo, const GemmScratch* scr);
// FP32 product with a fixed scratch: split-K is lowered to what scr holds.
void gemm_nt_f32_clamped(cudaStream_t s, int R, int C, int K, const float* A, int lda,
                         const float* B, int ldb, float* out, int ldo, const GemmScratch& scr);
int gemm_tile_rows_f32();
int gemm_tile_cols_f32();
// S = V X^T fused with the link: out[b][i] = dl(S[b][i], y[i])   (§4.2 Eq. (gradient_matrix_form))
void gemm_link_f64(cudaStream_t s, int m, int n, int p, const double* V, const double* X,
                   const double* y, int kind, double* out, const GemmScratch* scr);
void gemm_link_f32(cudaStream_t s, int m, int n, int p, const float* V, const float* X,
                   const float* y, int kind, float* out, const GemmScratch* scr);

// ---- tensor-core products (tcgen05, TMA); see gemm_tc.cu
struct TcMap {
    alignas(64) unsigned char bytes[128];   // a CUtensorMap
    // the same tensor with half the box rows: the B operand of a CTA pair, whose
    // CTAs each hold half of the tile's columns (made when the box rows are a
    // multiple of 16)
    alignas(64) unsigned char half[128];
    int has_half;
};
// TC_EPI_PARTIAL: split z writes its partial product to pout + z*pstride (row
// stride pld); the consumer sums the slices (no reduction in the kernel).
enum { TC_EPI_STORE_F32 = 0, TC_EPI_LINK_F32 = 1, TC_EPI_LINK_BF16 = 2, TC_EPI_PARTIAL = 3 };
struct TcGemm {
    int kind;        // 0: BF16 operands (kind::f16), 1: FP32 operands read as TF32 (kind::tf32)
    int M, N, K;     // out[r][c] = sum_k A[r][k] B[c][k], r < M, c < N, k < K
    int bn;          // tile columns (tc_tile_cols(N)); the B map's box rows
    int epi;         // TC_EPI_*
    void* out;
    int ldo;
    const float* y;  // link: y per output column
    int loss;
    int* err;        // device flag for a wait that ran out (may be NULL)
    float* pout;     // TC_EPI_PARTIAL destination, slice stride and row stride
    size_t pstride;
    int pld;
    int max_splits;  // TC_EPI_PARTIAL: upper bound on the number of slices
    int* splits_used;
    const TcMap* A2; // TF32 low part of A (out = (A + A2)(B + B2)^T less A2 B2^T); needs kind 1 and B2
    float* out_lo;   // TC_EPI_LINK_F32: TF32 low part of each output (NULL: none)
    int pdl;         // launch with programmatic stream serialization (prologue overlaps the previous kernel)
    int arow0;       // first row of A used (rows arow0 .. arow0 + M); outputs are indexed from row 0
    int pair;        // 1: CTA pairs (clusters of two) computing 256-row tiles with one
                     // cta_group::2 MMA, each CTA holding its 128 rows of A and half of
                     // the B tile, where supported (BF16, single operands, no split-K
                     // link, a B map with a half box); 0: one CTA per 128-row tile
};
// TMA map of a row-major rows x cols matrix (row stride ld elements) with
// 128-byte boxes along cols and box_rows rows.  0 on success.
int tc_make_map(TcMap* out, const void* base, int is_bf16, int rows, int cols, int ld, int box_rows);
// Sets the kernels' shared-memory attributes (call before any stream capture).
int tc_prepare();
// A bounded wait on an mbarrier nothing arrives on (rounds try_wait rounds); sets bit 8 of *err.
void wait_probe(cudaStream_t s, uint32_t rounds, int* err);
int tc_tile_cols(int N);
// Split-K slices of a TC_EPI_PARTIAL product with M x N output: enough units
// to fill the SMs, at most 16.
int tc_split_cap(int M, int N);
int tc_tile_cols_wide(int N);   // 128-column tiles for N > 256 (more CTAs for a wide output)
size_t tc_scratch_bytes();
int tc_scratch_counters();
// B2: optional low part of B (out = A (B + B2)^T); NULL for a single B.
// One job of a grouped BF16 product: K slices [ka, ka + nkb) of A against
// [kb, kb + nkb) of B (128-byte slices), written as partial slice `slice`.
constexpr int kTcMaxJobs = 64;
struct TcJob {
    int ka, kb, nkb, slice;
};
// out slice jobs[z].slice (at pout + slice * pstride, row stride pld) =
// A[:, K range of job z] . B[:, K range of job z]^T for every job, in one launch.
// pair_on: as CTA pairs (256-row tiles) where the B map has a half box.
int tc_gemm_jobs(cudaStream_t s, const TcMap& A, const TcMap& B, int M, int N, int bn, const TcJob* jobs,
                 int njobs, float* pout, size_t pstride, int pld, int* err, int pair_on);
// Exact-splitting certificate product (cert_exact.cu): jobs of the level
// products, their weights 2^(-beta l) and the bound n E per unit sigma tau.
struct ExactPlan {
    int beta, nd, npad, kbs;     // digit bits, digits per value, K padded to 64, 64-wide K slices per digit
    int njobs;
    TcJob jobs[kTcMaxJobs];
    double w[kTcMaxJobs];
    double ebound;
};
// Jobs whose FP32 accumulations are exact; false if they do not fit kTcMaxJobs.
bool exact_plan(int n, int beta, int nd, ExactPlan* pl);
// Halves jobs while fewer than two waves of CTAs would run (tiles per job) and
// the slices fit max_slices.
void exact_plan_widen(ExactPlan* pl, int tiles, size_t max_slices);
// Digits of the rows of V (rows x n, row stride ldv) into D (rows x nd*npad BF16)
// and the row scales 2^e > max |V_r|.
void exact_digits(cudaStream_t s, const double* V, int rows, int n, size_t ldv, int npad, int nd, int beta,
                  int reversed, __nv_bfloat16* D, double* scale);
// Q (m x p) and its entrywise bound E (nullable) from the job partials; w: the
// jobs' weights (host array of nq values).
void exact_combine(cudaStream_t s, int m, int p, const float* Qs, int nq, size_t stride, const double* w,
                   const double* sigma, const double* tau, double ebound, double* Q, double* E);
int tc_gemm(cudaStream_t s, const TcMap& A, const TcMap& B, const TcMap* B2, const TcGemm& g,
            const GemmScratch* scr);
// One problem of a grouped BF16 product (single operands): out[r][c] = sum_k A[arow0 + r][k] B[c][k],
// r < M, c < N, k < K; the link epilogue (BF16 R, y, loss) or partial slices (pout, pstride, pld)
// with split-K set from the problem alone (its tile count at width splits_bn, at most max_splits).
struct TcGroupItem {
    const TcMap* A;      // box rows 128
    const TcMap* B;      // box rows = the launch's bn
    int M, N, K, arow0;
    void* out;
    int ldo;
    const float* y;
    int loss;
    float* pout;
    size_t pstride;
    int pld;
    int max_splits;
    int splits_bn;
    int* splits_used;
};
// Up to 8 problems in one persistent launch of tile width bn, epi TC_EPI_LINK_BF16 or TC_EPI_PARTIAL.
int tc_gemm_group(cudaStream_t s, const TcGroupItem* items, int np, int bn, int epi, int* err);

struct ProxArgs {
    int m, p, W;
    const void* G;        // gradient X^T R, node-major m x p (working type)
    const float* Gpart;   // or: gsplits FP32 slices of it, slice s at Gpart + s*gstride (summed in order)
    int gsplits;
    size_t gstride;
    void* V;              // extrapolated point v (in: v_k, out: v_{k+1})
    void* B;              // iterate beta (in: beta_k, out: beta_{k+1})
    void* Vop;            // optional copy of V for the tensor-core products (row stride op_ld)
    float* Vop_lo;        // its TF32 low part (FP32-accurate mode), or NULL
    int op_ld;
    int op_bf16;          // 1: BF16, 0: FP32 rounded to TF32 (nearest)
    const uint32_t* in_mask;
    const uint32_t* out_mask;
    const int* kbar;
    const int* pf;
    double* tmom;         // FISTA t' per node
    const int* active;    // 1 = iterate this node
    double eta, c, M;     // step, c = 2 eta lambda2 = 1/rho, box
    int restart;
    int pdl;              // launch with programmatic stream serialization
    int threads;          // FP32, p > 512: threads per node (0: 8 coordinates per thread)
    float* hint;          // per node (2 floats): the last step's kbar-th largest free |u| and
                          // block threshold, for the streaming FP32 prox (0: none; NULL: unused)
    int* chk;             // bounds-checked build: the context's error word (kglm_check)
};
// One FISTA step per node: u = v - eta*G, beta' = prox(u), restart, next v.
int prox_fista_f64(cudaStream_t s, const ProxArgs& a);
int prox_fista_f32(cudaStream_t s, const ProxArgs& a);
// Candidate threads-per-node values of the FP32 prox for p (0 = default first,
// 32 = one warp per node); returns the count written to out (at most 4).
int prox_thread_options(int p, int* out);
// The FP32 prox as a persistent kernel, a warp streaming nodes through shared
// memory (prox_stream.cu); the default for 512 < p <= kStreamMaxP where at
// least six warps' rows fit in an SM's shared memory.  Returns 0 when
// launched, 1 when p is outside its range (no launch), -1 on a CUDA error.
constexpr int kStreamMaxP = 4096;
int prox_stream_f32(cudaStream_t s, const ProxArgs& a);
// The streaming prox over the nodes of up to kGroupMax problems in one launch
// (fills nbase, pmax, Wmax); 0 launched, 1 not this kernel's range (p above
// the streaming limit or too few warps per SM), -1 attribute refused.
constexpr int kGroupMax = 8;
struct ProxGroup {
    int np;
    int nbase[kGroupMax + 1];
    int pmax, Wmax;
    ProxArgs a[kGroupMax];
};
int prox_stream_group(cudaStream_t s, ProxGroup& g);

struct CertArgs {
    int m, n, p, W, k, kind;
    double lam2, M;
    const void* S;        // S = X beta (m x n), working type or FP64 (s_is_f64)
    int s_is_f64;
    const double* y;
    const float* y32;     // reduced-precision modes: y as FP32 high part y32 = fl(y) and low
    const float* ylo;     // part ylo = fl(y - y32), for the compensated least-squares sums
    double* zeta;         // out: m x n FP64 dual points
    // reduced-precision modes with the exact-splitting certificate: the dual point
    // pass also writes zeta's digits (the layout of exact_digits, reversed) and
    // its row scales 2^e > max |zeta_b| (DZ NULL: not done there)
    __nv_bfloat16* DZ;
    int dz_npad, dz_nd, dz_beta;
    double* sum_loss;     // out: m
    double* sum_conj;     // out: m
    const double* Q;      // X^T zeta (m x p) FP64
    const void* B;        // beta (m x p) working type
    int b_is_f64;
    const uint32_t* in_mask;
    const uint32_t* out_mask;
    const int* kbar;
    const int* pf;
    double* lb;           // out
    double* primal;       // out
    int* support;         // out m x k
    int* jstar;           // out
    // reduced-precision modes: X^T zeta from the exact-splitting partials
    // (Qs != NULL) with the entrywise bound xsig_j ztau_b ebound, instead of Q
    const float* Qs;
    int nqs;
    size_t qs_stride;
    double qs_w[kTcMaxJobs];
    const double* xsig;
    double* ztau;
    double ebound;
    int* chk;             // bounds-checked build: the context's error word (kglm_check)
};
// zeta = -dl(S), row sums of l and l*(-zeta)   (§4.4 Eq. (batched_dual_candidate_matrix_form))
void cert_dual_point(cudaStream_t s, const CertArgs& a);
// LB = -sum l* - 2 lambda2 g*(Q/(2 lambda2)), Phi, support, j*   (§4.4, §4.3)
int cert_bound(cudaStream_t s, const CertArgs& a);

struct ReoptArgs {
    int m, n, p, k, kind, max_iter;
    double lam2, M, tol;
    const double* Xt;      // p x n FP64
    const double* y;       // n
    const float* Xt32;     // p x n FP32 copy (NULL in the FP64 mode)
    const float* y32;
    const double* gram;    // p x p FP64 X^T X
    const double* Xty;     // p FP64
    const int* support;    // m x k
    const void* B;         // warm start beta (m x p)
    int b_is_f64;
    double* ub;            // out: v(S_b)
    double* beta_re;       // out: m x k
    double yty;            // y^T y (least squares: v(S) = y^T y + b^T (G_SS + lambda2 I) b - 2 c^T b)
    int* chk;              // bounds-checked build: the context's error word (kglm_check)
};
// returns 0, or -1 if the dynamic shared memory for k cannot be granted
int reopt_launch(cudaStream_t s, const ReoptArgs& a);
size_t reopt_smem_bytes(int k);
// FP64 objective F(X_S b) + lambda2 ||b||^2 of one support (device S[ks], b[ks]) into *out.
void objective64_launch(cudaStream_t s, const double* Xt, const double* y, int n, int kind, double lam2,
                        const int* S, const double* b, int ks, double* out);

// node-batch layout (a2): CSR fixing lists -> masks, kbar, pf; warm starts
// (layout launchers return the number of kernels they launched)
int layout_masks(cudaStream_t s, int m, int p, int W, int k, const int* in_ptr, const int* in_idx,
                 const int* out_ptr, const int* out_idx, uint32_t* in_mask, uint32_t* out_mask,
                 int* kbar, int* pf, int nnz_in, int nnz_out, int* err);
int layout_validate(cudaStream_t s, int m, int k, int W, int nnz_in, int nnz_out, const int* in_ptr,
                    const int* out_ptr, const uint32_t* in_mask, const uint32_t* out_mask, const int* slot,
                    int nslots, int* err);
int layout_warm(cudaStream_t s, int m, int p, int W, int is_f64, const int* slot, int nslots, const void* pool,
                const double* warmB, const uint32_t* out_mask, void* B, void* V, void* Vop, float* Vop_lo, int op_ld,
                int op_bf16, double* tmom, int* active, float* hint);
// rows x cols FP64 (row stride ld_in) -> BF16 or TF32-in-FP32 with row stride ld_out, zero padded;
// with lo != NULL also the low part bf16/tf32(x - hi) into lo.
void convert_pad(cudaStream_t s, const double* in, int rows, int cols, int ld_in, void* out, int ld_out, int to_bf16,
                 void* lo = nullptr);
// rows x cols FP32 (stride cols) -> BF16 or TF32-in-FP32 with row stride ld_out
// (with lo != NULL, TF32 only: also the low parts)
void convert_pad_f32(cudaStream_t s, const float* in, int rows, int cols, void* out, int ld_out, int to_bf16,
                     float* lo = nullptr);
void pool_store(cudaStream_t s, int count, int p, int is_f64, const int* rows, const int* slots,
                const void* B, void* pool);
// a8: pruned[b] = lb[b] >= thr ; alive[b] &= !pruned
void prune_launch(cudaStream_t s, int m, const double* lb, double thr, uint8_t* pruned);
// early-stop bookkeeping at a check: best LB, freeze nodes
void check_update(cudaStream_t s, int m, const double* lb_now, const double* primal_now, double* lb_best,
                  double* primal_last, int* active, int* iters_done, int it, double ub_thr, double gap_rtol);
// bounds-checked build only: one checked write one past the end of buf (len entries)
void check_probe(cudaStream_t s, int* buf, int len, int* word);
void convert_f64_to_f32(cudaStream_t s, const double* in, float* out, size_t count);
// out (cols x rows) = in^T for a row-major rows x cols FP64 matrix (device buffers)
void transpose_f64(cudaStream_t s, const double* in, double* out, size_t rows, size_t cols);
void convert_to_f64(cudaStream_t s, const void* in, int is_f64, double* out, size_t count);

// ---- host side shared by the C ABI and the serving loop (api.cu)
// Device bytes kglm_create allocates for desc (see kglm_estimate_bytes).
size_t device_footprint(const kglm_desc& d);
// Device-resident open-node queue of the hybrid loop (queue.cu).
struct DqState {
    long long next_id;   // the next node id
    long long id_base;   // first id of this round's children
    double ub;           // incumbent objective
    long long sum_out;   // sum of |J0| over the selected batch
    int N;               // open nodes in the pool
    int m;               // nodes of the selected batch
    int nbranch;         // branching nodes of the last batch
    int nfree;           // free warm-start slots
    int nkeep;           // pool entries kept by the last merge
    int overflow;        // the last merge had more entries than the capacity
};
struct DevQueue {
    int cap = 0, W = 0, p = 0, k = 0, nslots = 0, cur = 0;
    double* lb[2] = {nullptr, nullptr};      // pool buffers: parent bound, id, slot, masks (J1 then J0, 2W words)
    long long* id[2] = {nullptr, nullptr};
    int* slot[2] = {nullptr, nullptr};
    uint32_t* mask[2] = {nullptr, nullptr};
    double* clb = nullptr;                   // children of a batch (2 per node)
    long long* cid = nullptr;
    int* cslot = nullptr;
    uint32_t* cmask = nullptr;
    int* cperm = nullptr;                    // children in key order
    double* lbp = nullptr;                   // batch: parent bound (then the children's bound)
    int* bslot = nullptr;                    // batch: warm-start slot
    int* brank = nullptr;                    // batch: rank among the branching nodes, -1 if closed
    int* cslot_b = nullptr;                  // batch: the new slot of a branching node
    int* sref = nullptr;                     // slot reference counts
    int* sfree = nullptr;                    // stack of free slots
    int* best_sup = nullptr;                 // incumbent support and coefficients
    double* best_coef = nullptr;
    DqState* st = nullptr;
};
void dq_init(cudaStream_t s, DevQueue& q);
// k_dq_select + layout of the first min(batch, N) pool entries into the batch arrays
void dq_select(cudaStream_t s, DevQueue& q, int batch, double gap_tol, uint32_t* in_mask, uint32_t* out_mask,
               int* kbar, int* pf);
// incumbent, close/branch, children, merge (m, N: the host's copies of the state)
void dq_update(cudaStream_t s, DevQueue& q, int m, int N, double gap_tol, const double* lb_best, const double* ubc,
               const int* jstar, const int* support, const double* beta_re, const uint32_t* in_mask,
               const uint32_t* out_mask, const void* B, int is_f64, void* pool);

struct SolveResult {
    double opt = 0, gap = 0;
    std::vector<int> support;
    int64_t nodes = 0, batches = 0;
    bool cancelled = false;
};
// The serving loop's steps on contexts with a device queue (open_cap > 0):
// serve_begin starts a search, serve_select puts its next batch in place
// (*m = 0: nothing open), serve_evaluate evaluates the selected batches of
// several contexts that share one stream with the iterations in shared
// launches (*shared: the launches that carried more than one), serve_update closes, branches and merges, serve_finish reports
// (and frees the state; serve_free frees it without a report).
struct ServeSolve;
kglm_status serve_begin(kglm_ctx* c, int batch, ServeSolve** out);
kglm_status serve_select(ServeSolve* s, int* m);
kglm_status serve_evaluate(kglm_ctx* const* cs, int count, int iters, int check_every, int64_t* shared);
kglm_status serve_update(ServeSolve* s);
kglm_status serve_finish(ServeSolve* s, bool stopped, SolveResult* r);
void serve_free(ServeSolve* s);
// kglm_solve that also stops (between batches) once *cancel is non-zero.
kglm_status solve_cancellable(kglm_ctx* ctx, int batch, int iters, int check_every, double time_limit_s,
                              const std::atomic<int>* cancel, SolveResult* r);

}  // namespace kglm
