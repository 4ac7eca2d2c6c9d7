/*
 * kglm.h -- C ABI of the GB300 batched node-bound engine for certified
 * k-sparse GLM branch and bound (Liu & Lodi, "From Sequential Nodes to GPU
 * Batches: Parallel Branch and Bound for Optimal k-Sparse GLMs").
 *
 * Problem (§1, problem (intro_sparse_glm)):
 *     min_beta  f(X beta, y) + lambda2 ||beta||_2^2
 *     s.t.      ||beta||_0 <= k,  ||beta||_inf <= M
 * with f(s, y) = sum_i l(s_i, y_i), l(s, y) = (s - y)^2 (least squares) or
 * log(1 + exp(-y s)) with y in {-1, +1} (logistic).
 *
 * A BnB node N fixes z_j = 0 on J0(N) and z_j = 1 on J1(N); the other
 * coordinates are free (§3, definition of g_N).  The engine evaluates a batch
 * of m nodes at once (§4.2): FISTA iterations on the perspective relaxation
 * Phi_N = F(X beta) + 2 lambda2 g_N(beta) (§3 Eq. (node_composite)), each
 * iteration two dense products S = X B and G = X^T R (§4.2 Eq.
 * (gradient_matrix_form)) and the column-wise proximal step of §3 Eq.
 * (pgd_step_vector_form); then the Fenchel-dual certificate
 * Psi_N(zeta) = -F*(-zeta) - G_N*(X^T zeta) (§3 Eq. (prelim_fenchel_dual),
 * §4.4 Eq. (batched_dual_value_component)) evaluated in FP64, the rounding,
 * re-optimization and branching index of §4.3, and the pruning test of §3.
 *
 * Conventions for every call:
 *  - host arrays are read before the call returns and never kept; outputs go
 *    to caller-owned host buffers (any output pointer may be NULL to skip it);
 *  - the context owns all device memory; one context is used by one host
 *    thread at a time and runs its work on the stream given at creation;
 *  - no C++ exception crosses this ABI; every call returns a kglm_status and
 *    kglm_last_error() gives a message;
 *  - an argument error returns KGLM_EINVAL and leaves the context unchanged;
 *  - indices are 0-based int32; matrices are row-major as stated per call.
 */
#ifndef KGLM_H
#define KGLM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kglm_ctx kglm_ctx;

typedef enum {
    KGLM_OK = 0,
    KGLM_EINVAL = -1,   /* bad argument (sizes, indices, overlapping fixings, y not +-1, ...) */
    KGLM_ENOMEM = -2,   /* device or host allocation failed, or over the HBM budget */
    KGLM_ECUDA = -3,    /* a CUDA call failed; the message names it */
    KGLM_ETIMEOUT = -4, /* a bounded device wait ran out */
    KGLM_ESTATE = -5,   /* call out of order (e.g. evaluate before push) */
    KGLM_ENUMERIC = -6  /* non-finite X or y */
} kglm_status;

typedef enum { KGLM_LSQ = 0, KGLM_LOGISTIC = 1 } kglm_loss;

/* Arithmetic of the FISTA iterations.  The certificate is valid in every
 * mode: the bound of §3 holds for any dual point zeta, and the engine returns
 * Psi_N(zeta) evaluated with FP64 X^T zeta and FP64 sums (KGLM_FP64), or a
 * rigorous lower estimate of it whose conjugate terms are FP32 evaluations
 * plus explicit rounding margins (the other modes; looser by ~1e-7
 * relative). */
typedef enum {
    KGLM_FP64 = 0,  /* FP64 products and prox */
    KGLM_FP32 = 1,  /* FP32 products (CUDA cores) and prox */
    KGLM_BF16 = 2,  /* BF16 tensor-core products, FP32 accumulate and prox */
    KGLM_TF32 = 3,  /* TF32 tensor-core products, FP32 accumulate and prox */
    KGLM_TF32X3 = 4 /* FP32-accurate tensor-core products: every FP32 operand split into
                       TF32 hi + lo, hi*hi + hi*lo + lo*hi, FP32 accumulate; FP32 prox */
} kglm_prec;

typedef struct {
    int64_t n;            /* samples (rows of X), > 0 */
    int64_t p;            /* features (columns of X), > 0 */
    int32_t k;            /* sparsity budget, 1 <= k <= KGLM_MAX_K and k <= p */
    int32_t loss;         /* kglm_loss */
    int32_t prec;         /* kglm_prec */
    int32_t restart;      /* 1: FISTA with gradient restart; 0: plain FISTA */
    double lambda2;       /* ridge coefficient, > 0 */
    double M;             /* box ||beta||_inf <= M, > 0 */
    double lipschitz;     /* L of grad F; 0: the engine computes 2||X||^2 or ||X||^2/4 */
    double gap_tol;       /* pruning slack delta = gap_tol*max(1,|UB|); 0 selects 1e-6 */
    int32_t max_batch;    /* node-batch capacity m_max, >= 1 */
    int32_t pool_slots;   /* warm-start slots kept on the device (0: 4*max_batch) */
    int64_t hbm_budget;   /* bytes the context may hold on the device; 0: no limit */
    int64_t open_cap;     /* open nodes the device-resident queue holds (kglm_solve_device);
                             0: no device queue */
} kglm_desc;

#define KGLM_MAX_K 64

/* Create an instance (§1 problem (intro_sparse_glm)).
 * X: host, n x p row-major FP64; y: host, n FP64 (logistic: every y_i is
 * -1 or +1).  Both are copied to the device (FP64, plus the working copies of
 * the chosen precision).  stream: a cudaStream_t to run on, or NULL for a
 * stream the context creates.  On success *out owns the instance. */
kglm_status kglm_create(const kglm_desc* desc, const double* X, const double* y,
                        void* stream, kglm_ctx** out);

/* Define the next node batch (§4.2, Fig. 1 "assemble a batch of open nodes").
 * m nodes, 1 <= m <= max_batch.  Node b fixes J1(b) = in_idx[in_ptr[b] ..
 * in_ptr[b+1]) and J0(b) = out_idx[out_ptr[b] .. out_ptr[b+1]) (CSR, m+1
 * offsets each; indices in [0, p), no repeats, J0 and J1 disjoint,
 * |J1| <= k).  Warm start of node b, first that applies:
 *   warm_slot[b] >= 0: the beta stored in that pool slot (kglm_save_warm);
 *   warm_B != NULL:    row b of warm_B (host, m x p row-major FP64);
 *   otherwise beta = 0.
 * J0 entries of the warm start are set to 0.  warm_slot may be NULL. */
kglm_status kglm_push_nodes(kglm_ctx* ctx, int32_t m,
                            const int32_t* in_ptr, const int32_t* in_idx,
                            const int32_t* out_ptr, const int32_t* out_idx,
                            const int32_t* warm_slot, const double* warm_B);

/* Evaluate the pushed batch: `iters` FISTA iterations (§3 Eq.
 * (pgd_step_vector_form) with acceleration and gradient restart), then the
 * safe bound LB_b = Psi_{N_b}(zeta_b), zeta_b = -grad F(X beta_b) (§3 Eq.
 * (dual_candidate_vector_form)), the primal value Phi_b with g by Theorem 4.1,
 * the rounded support S_b = J1 cup top-kbar |beta| over Jf and its
 * re-optimized objective v(S_b) (§4.3), and the branching index
 * j*_b = argmax_{Jf} |beta_j| (§4.3; -1 for a leaf: kbar = 0 or
 * |J1| + |Jf| <= k).  With check_every > 0 the certificate is also taken
 * every check_every iterations; a node stops iterating once its bound
 * reaches ub - delta (the incumbent of kglm_set_incumbent) or its relative
 * gap falls below 1e-9, and lb is the best certificate seen.
 * Outputs (host, m entries each unless stated):
 *   lb       FP64 safe lower bounds;   primal  FP64 Phi_b at the last iterate;
 *   ub_cand  FP64 v(S_b);              support m x k int32, S_b ascending, -1 padded;
 *   beta_re  m x k FP64 coefficients of the re-optimized model on S_b;
 *   branch_j int32 j*_b;               iters_done int32 iterations run per node. */
kglm_status kglm_evaluate(kglm_ctx* ctx, int32_t iters, int32_t check_every,
                          double* lb, double* primal, double* ub_cand,
                          int32_t* support, double* beta_re,
                          int32_t* branch_j, int32_t* iters_done);

/* Read back the batch's final iterates B (host, m x p row-major FP64) and the
 * dual points zeta used by the last certificate (host, m x n row-major FP64).
 * Either pointer may be NULL. */
kglm_status kglm_read_batch(kglm_ctx* ctx, double* beta, double* zeta);

/* Store the final beta of batch rows rows[0..count) in pool slots
 * slots[0..count) (warm starts for children, Fig. 1 "warm starts"). */
kglm_status kglm_save_warm(kglm_ctx* ctx, int32_t count, const int32_t* rows, const int32_t* slots);

/* Record the incumbent objective UB (§3): used by kglm_prune and by the early
 * stop of kglm_evaluate. */
kglm_status kglm_set_incumbent(kglm_ctx* ctx, double ub);

/* Prune the evaluated batch against ub (§3 "Safe Lower Bound and Pruning"):
 * pruned[b] = 1 iff lb_b >= ub - delta, delta = gap_tol * max(1, |ub|).
 * *n_survivors counts the others.  pruned: host, m uint8 (may be NULL). */
kglm_status kglm_prune(kglm_ctx* ctx, double ub, uint8_t* pruned, int32_t* n_survivors);

/* Children of the surviving, non-leaf nodes of the evaluated batch whose own
 * rounding is not within delta of their bound (§4.3 branching, App. A):
 * child 2c is (batch row parent[c], fix z_j = 0 on j = branch_j), child 2c+1
 * fixes z_j = 1.  parent: host, capacity m int32; *n_parents receives the
 * number of branched rows. */
kglm_status kglm_branch(kglm_ctx* ctx, double ub, int32_t* parent, int32_t* branch_j,
                        int32_t* n_parents);

/* Certify the instance with the built-in hybrid BnB loop of Fig. 1: best-bound
 * node queue on the host, batches of up to `batch` nodes (0: the autotuned
 * batch, see kglm_autotune) evaluated with
 * `iters` iterations (certificate every `check_every`), incumbent from the
 * batched rounding and re-optimization, pruning and branching on j*.
 * time_limit_s <= 0 means none.  Outputs: *opt the certified objective,
 * opt_support (k int32, ascending, -1 padded), opt_beta (p FP64), *gap the
 * final relative gap (0 when certified), *nodes the evaluated node count,
 * *batches the number of batches. */
kglm_status kglm_solve(kglm_ctx* ctx, int32_t batch, int32_t iters, int32_t check_every,
                       double time_limit_s, double* opt, int32_t* opt_support,
                       double* opt_beta, double* gap, int64_t* nodes, int64_t* batches);

/* kglm_solve with the open-node queue on the device (the context must be
 * created with desc.open_cap > 0): the open nodes (fixing masks, parent bound,
 * warm-start slot) stay in a device pool sorted by (bound, id), and each round
 * selects the first `batch` nodes, evaluates them, updates the incumbent and
 * merges the children into the pool on the device; pruning is a truncation of
 * the sorted pool.  The host reads a few scalars per round.  Nodes are
 * evaluated in the order of kglm_solve (best bound, ties to the older node)
 * and the certified optimum is the same.  Outputs as kglm_solve; a search
 * whose open nodes would exceed open_cap stops with *gap > 0.  No checkpoint
 * is kept (kglm_solve_checkpoint returns KGLM_ESTATE after it). */
kglm_status kglm_solve_device(kglm_ctx* ctx, int32_t batch, int32_t iters, int32_t check_every,
                              double time_limit_s, double* opt, int32_t* opt_support,
                              double* opt_beta, double* gap, int64_t* nodes, int64_t* batches);

/* Stop kglm_solve after max_batches node batches (0: no limit), counted per
 * call; the open queue it leaves can be checkpointed.  (A deployment aid for
 * long searches; the paper's loop runs to completion or a time limit.) */
kglm_status kglm_set_solve_limit(kglm_ctx* ctx, int64_t max_batches);

/* Checkpoint of an unfinished certified solve (Fig. 1's loop stopped by its
 * time limit, its batch limit or cancellation): writes to `path` the open node
 * queue (each node's J0, J1, parent bound and warm start beta) and the
 * incumbent (objective, support, coefficients) with the node and batch counts,
 * and a signature of the instance (n, p, k, loss, lambda2, M and the sum of X
 * and y).  KGLM_ESTATE if the last kglm_solve on ctx completed (nothing is
 * left open); KGLM_EINVAL if the file cannot be written. */
kglm_status kglm_solve_checkpoint(kglm_ctx* ctx, const char* path);

/* Continue a checkpointed solve on a context of the same instance (any
 * precision or batch size): the search restarts from the stored open nodes,
 * warm starts and incumbent, and the outputs are those of kglm_solve for the
 * whole search (node and batch counts include the checkpointed part).
 * KGLM_EINVAL if the file is unreadable, malformed or written for another
 * instance. */
kglm_status kglm_solve_resume(kglm_ctx* ctx, const char* path, int32_t batch, int32_t iters, int32_t check_every,
                              double time_limit_s, double* opt, int32_t* opt_support, double* opt_beta,
                              double* gap, int64_t* nodes, int64_t* batches);

/* kglm_push_nodes with the CSR arrays (and warm_slot, if not NULL) already
 * in device memory: in_ptr/out_ptr hold m+1 offsets, nnz_in = in_ptr[m] and
 * nnz_out = out_ptr[m] are passed by value.  The arrays are read on the
 * device before the call returns; the same checks as kglm_push_nodes run
 * there and a failure returns KGLM_EINVAL (the batch is then undefined and
 * must be pushed again).  No warm_B variant: use pool slots. */
kglm_status kglm_push_nodes_dev(kglm_ctx* ctx, int32_t m, const int32_t* in_ptr, const int32_t* in_idx,
                                const int32_t* out_ptr, const int32_t* out_idx, int32_t nnz_in,
                                int32_t nnz_out, const int32_t* warm_slot);

/* The batched product G = R X of §4.2 Eq. (gradient_matrix_form) for the
 * instance's X: G[b][j] = sum_i R[b][i] X[i][j], i.e. column b of X^T R.
 * R: device, m x n row-major; G: device, m x p row-major; both in the
 * context's working type (double in KGLM_FP64, float otherwise).  In the
 * BF16 and TF32 modes the product runs on the tensor cores (R is first
 * rounded to the operand type).  1 <= m <= max_batch.  Runs on the context's
 * stream with the context's split-K scratch and returns when G is written;
 * KGLM_ETIMEOUT if a tensor-core pipeline wait ran out. */
kglm_status kglm_xtr(kglm_ctx* ctx, int32_t m, const void* R, void* G);

/* The certificate product of the context: Q[b][j] = sum_i Z[b][i] X[i][j]
 * (X^T zeta of §4.4 Eq. (batched_dual_candidate_matrix_form), one dual point
 * per row of Z) with an entrywise bound Qerr[b][j] >= |Q[b][j] - exact|.
 *   Z: host, m x n row-major FP64; Q, Qerr: host, m x p row-major FP64
 *   outputs (Qerr may be NULL); 1 <= m <= max_batch.
 * The FP64 mode computes Q by an FP64 GEMM and writes Qerr = 0 (FP64
 * rounding only).  The reduced-precision modes use the engine's
 * exact-splitting product on the BF16 tensor cores (6-bit digits of X and
 * Z, integer-exact FP32 accumulation, FP64 combine) with its rigorous bound
 * in Qerr; where that product is not set up (job count or HBM budget) they
 * fall back to the FP64 GEMM with Qerr = 0.  Uses the batch buffers: call
 * it between evaluations, not between a push and its evaluation (the pushed
 * batch's dual points are overwritten).  KGLM_ETIMEOUT if a tensor-core
 * pipeline wait ran out. */
kglm_status kglm_xtz(kglm_ctx* ctx, int32_t m, const double* Z, double* Q, double* Qerr);

/* kglm_xtr for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment aid.  Callers that run inside CUDA graph
 * capture, draw every byte from a host application's own pool, or must not
 * grow their footprint once serving cannot call cudaMalloc (directly or
 * through a context); this call computes G[b][j] = sum_i R[b][i] Xt[j][i]
 * with no allocation of any kind, keeping its split-K partial tiles and tile
 * counters in a file-scope device array of KGLM_XTR_NOALLOC_SCRATCH_FLOATS
 * floats and KGLM_XTR_NOALLOC_MAX_TILES ints that every GPU loading the
 * library holds until the process exits.
 *   R: device, m x n row-major FP32; Xt: device, p x n row-major FP32 (X^T);
 *   G: device, m x p row-major FP32 output; stream: cudaStream_t or NULL.
 * The output grid of 128 x 128 tiles, ceil(m/128) * ceil(p/128), may not
 * exceed KGLM_XTR_NOALLOC_MAX_TILES (KGLM_EINVAL otherwise); n is free.
 * The call only enqueues work on `stream` (G is ready when the stream
 * reaches it).  The first call on a device, with that device current, looks
 * up the array's device address and clears the counters; make that first
 * call before any stream capture (a first call on a capturing stream returns
 * KGLM_EINVAL and changes nothing).  All calls share the one array, which
 * keeps the last call's partial tiles (the counters return to 0 after each
 * call): calls that overlap on the GPU, on any streams, race.  Errors:
 * KGLM_EINVAL for bad sizes or pointers, KGLM_ECUDA for a failed CUDA call,
 * and also, without launching, when an error from earlier work on the calling
 * thread is still pending (it is left for its owner to read); no message is
 * recorded (there is no context). */
#define KGLM_XTR_NOALLOC_SCRATCH_FLOATS (4u << 20)
#define KGLM_XTR_NOALLOC_MAX_TILES 256
kglm_status kglm_xtr_noalloc_f32(int32_t m, int32_t n, int32_t p, const float* R, const float* Xt,
                                 float* G, void* stream);

/* Per-phase device timers: a tracing aid in the spirit of the paper's
 * per-component runtime breakdown (App. F).  While enabled, every kernel the context
 * launches is bracketed by CUDA events on the context's stream; kglm_stats_read
 * returns, per phase, the summed device milliseconds (0 while disabled), the
 * kernel launch count (always counted) and the algorithmic work (FLOPs for
 * products, bytes for the others; 0 when not defined).  Any output pointer may
 * be NULL; arrays hold KGLM_NPHASE entries.  Phases: see kglm_phase_name.
 * kglm_stats_enable resets the counters. */
#define KGLM_NPHASE 11
kglm_status kglm_stats_enable(kglm_ctx* ctx, int32_t enable);
kglm_status kglm_stats_read(kglm_ctx* ctx, double* ms, int64_t* launches, double* work);
const char* kglm_phase_name(int32_t phase);

/* Autotuner (project-written; the paper picks the batch by memory, App. E.4,
 * and shows throughput flattening with the batch size, Fig. 3).  Times node
 * evaluations (iters FISTA iterations, certificate, re-optimization) of random
 * fixing patterns (|J1| ~ U{0..k}, |J0| ~ U{0..p/2}; `seed`) on the context:
 * in the tensor-core modes first the column tile of S = X V (64/128/256), then
 * the column tile and split-K cap of G = X^T R, at the full batch; then every
 * power-of-two batch size up to max_batch; programmatic dependent launch of
 * the iteration kernels (each kernel's prologue overlapping the previous
 * kernel) is timed on and off at the chosen tiles, then 1, 2 or 4 sub-batches
 * (node ranges iterated side by side on forked streams, tensor-core modes),
 * in the BF16 mode CTA pairs for the products on and off, and for p > 512 in
 * the FP32-type modes the prox's threads per node.  The context keeps the
 * fastest configuration; the batch chosen is the smallest within 5% of the best node rate
 * (kglm_solve with batch 0 uses it, tuning first with min(iters, 20) if
 * needed).  Discards the pushed batch (push again before kglm_evaluate). */
typedef struct {
    int32_t batch;            /* chosen node-batch size */
    int32_t link_tile_cols;   /* column tile of S = X V (tensor-core modes; 0 otherwise) */
    int32_t grad_tile_cols;   /* column tile of G = X^T R (tensor-core modes; 0 otherwise) */
    int32_t grad_split_cap;   /* split-K cap of G (tensor-core modes; 0 otherwise) */
    int32_t timed;            /* configurations timed */
    int32_t pdl;              /* 1: iteration kernels use programmatic dependent launch */
    int32_t sub_batches;      /* iteration loop split into this many node ranges on parallel streams */
    int32_t prox_threads;     /* threads per node of the prox for p > 512 in the FP32-type modes (0: default;
                                 32: one warp per node, p <= 2048) */
    int32_t pair;             /* BF16: the iteration products as CTA pairs (clusters of two), each pair
                                 computing a 256-row tile with one cta_group::2 product and each CTA
                                 holding half of the B tile: 1 on, -1 off (kglm_configure: 0 keeps) */
    double nodes_per_s;       /* node evaluations per second at the chosen batch */
    double best_nodes_per_s;  /* the best rate over all batch sizes */
} kglm_tune;
kglm_status kglm_autotune(kglm_ctx* ctx, int32_t iters, uint64_t seed, kglm_tune* out);

/* Set the tuning choices by hand (the fields of kglm_tune; a 0 tile, split cap
 * batch or sub_batches keeps the current value; `timed` and the rates are
 * ignored).  The
 * split cap may not exceed the slices allocated at creation.  pdl 0 launches
 * the iteration kernels without programmatic dependent launch. */
kglm_status kglm_configure(kglm_ctx* ctx, const kglm_tune* cfg);

/* Device bytes kglm_create allocates for *desc (App. E.4 sizes the batch from
 * the memory per node; admission control needs the whole footprint before
 * any allocation).  Host-only arithmetic, no CUDA call.  Not included: one
 * max_batch x p FP64 buffer that kglm_push_nodes with warm_B, and one that
 * kglm_xtz, allocate on first use.  KGLM_EINVAL for a desc kglm_create would
 * reject on its sizes, ranges or enums. */
kglm_status kglm_estimate_bytes(const kglm_desc* desc, int64_t* bytes);

/* Device bytes the context holds (what kglm_estimate_bytes predicted, plus
 * the first-use buffers above once allocated). */
kglm_status kglm_device_bytes(const kglm_ctx* ctx, int64_t* bytes);

/* Automatic batch size of App. E.4: the largest power of two m <= cap such
 * that the instance with max_batch = m (and desc's other fields; pool_slots 0
 * scales with m) fits in `budget` device bytes.  KGLM_ENOMEM if even m = 1
 * does not fit; KGLM_EINVAL for bad arguments. */
kglm_status kglm_suggest_batch(const kglm_desc* desc, int64_t budget, int32_t cap, int32_t* batch);

/* ---- Rashomon-set collection (§4.5, App. G).
 * The support-level Rashomon set is R = {S : |S| <= k, v(S) <= (1 + eps) Phi*}
 * with v(S) the optimal objective on support S and Phi* the optimum of the
 * problem.  The BnB loop of kglm_solve collects it by changing the pruning
 * threshold: a node is pruned only when its bound exceeds
 * tau = min((1 + eps) UB, v_(N)) (v_(N): the N-th best stored objective when
 * max_models = N > 0), every re-optimized support with objective <= tau is
 * stored, and nodes are branched until they hold one support (kbar = 0 or no
 * free coordinate).  At completion UB = Phi* and the pool is the certified set
 * (or its N best members). */

/* Pool of supports in the layout of App. G: a trie whose non-root nodes carry
 * one feature index (node 0 is the root; node v > 0 has parent[v] and
 * label[v]); record m is a trie leaf whose root-to-leaf labels are its support
 * in insertion order, its objective, and its coefficients c[o[m] .. o[m+1])
 * in the order of those labels (o[0] = 0).  Host memory; one pool per
 * collection. */
typedef struct kglm_pool kglm_pool;
kglm_status kglm_pool_create(int32_t p, kglm_pool** out);
/* Adds a record (seq: len distinct indices in [0, p), insertion order; coef:
 * len coefficients in the same order).  A support already held (as a set) is
 * not added again: *record = -1 then. */
kglm_status kglm_pool_insert(kglm_pool* pool, int32_t len, const int32_t* seq, const double* coef,
                             double objective, int64_t* record);
kglm_status kglm_pool_size(const kglm_pool* pool, int64_t* records, int64_t* trie_nodes, int64_t* coef_len);
/* Copies the layout out (any pointer may be NULL): offsets records+1, coef
 * coef_len, objective records, leaf records, parent and label trie_nodes. */
kglm_status kglm_pool_read(const kglm_pool* pool, int64_t* offsets, double* coef, double* objective,
                           int32_t* leaf, int32_t* parent, int32_t* label);
/* Root-to-leaf labels of a record (at most k entries). */
kglm_status kglm_pool_support(const kglm_pool* pool, int64_t record, int32_t* labels, int32_t* len);
/* Keeps the records with objective <= threshold and, if keep_best > 0, the
 * keep_best best of them (ties to the earlier record), in their order. */
kglm_status kglm_pool_filter(kglm_pool* pool, double threshold, int64_t keep_best);
void kglm_pool_destroy(kglm_pool* pool);

/* Collect the Rashomon set of the instance into `pool` (cleared first; created
 * with this instance's p).  batch, iters, check_every, time_limit_s as for
 * kglm_solve; eps >= 0; max_models 0 for no cap.  In the reduced-precision
 * modes the stored objectives are replaced by FP64 evaluations of the stored
 * coefficients at the end and the pool is filtered at the final threshold.
 * Outputs: *opt = Phi* (the incumbent), *nodes evaluated, *complete = 1 when
 * the search finished (0 when the time limit stopped it). */
kglm_status kglm_rashomon(kglm_ctx* ctx, double eps, int64_t max_models, int32_t batch, int32_t iters,
                          int32_t check_every, double time_limit_s, kglm_pool* pool, double* opt, int64_t* nodes,
                          int32_t* complete);

/* ---- Serving loop: certified solves of many instances, admitted as they
 * arrive (continuous batching at node-batch granularity).  Each admitted
 * request keeps X and its open-node queue on the device (kglm_solve_device's
 * queue) on a context that runs on the server's stream.  One scheduler
 * thread runs rounds: every running request's next node batch (up to its
 * max_batch nodes, best bound first) is selected on the device, the selected
 * batches are evaluated together -- the FISTA iterations of the BF16
 * requests as shared launches (per iteration one grouped S = X V + link, one
 * grouped G = X^T R and one prox launch over all their nodes, up to 8
 * requests per launch), the other precisions with their own launches on the
 * same stream -- and each batch is then closed, branched and merged into
 * its request's queue on the device.  Admission is FIFO at round
 * boundaries: the request at the head of the queue starts once a slot is
 * free (max_active) and its device footprint (kglm_estimate_bytes, queue
 * included) fits in the budget the running requests leave; a request's
 * memory returns to the budget when it finishes.  A request's nodes see the
 * same arithmetic whatever shares the launches, so its result (objective,
 * support, node count) does not depend on the other requests. */
typedef struct kglm_server kglm_server;

typedef struct {
    int64_t hbm_budget;   /* device bytes all admitted requests may hold; 0: 80% of the free memory at creation */
    int32_t max_active;   /* requests solved at once (worker threads and streams), 1..256 */
    int32_t batch_cap;    /* cap of the automatic batch size (requests with max_batch 0); 0: 4096 */
    int32_t iters;        /* FISTA iterations per node evaluation (kglm_solve's iters), >= 1 */
    int32_t check_every;  /* certificate every check_every iterations (kglm_solve's), >= 0 */
    double time_limit_s;  /* per request, counted from admission; <= 0: none */
    int64_t open_cap;     /* open nodes each request's device queue holds; 0: what a quarter of
                             budget / max_active holds (at most 1 GiB or 2^22 nodes, at least
                             64 max_batch) */
} kglm_server_desc;

enum { KGLM_REQ_QUEUED = 0, KGLM_REQ_RUNNING = 1, KGLM_REQ_DONE = 2, KGLM_REQ_FAILED = 3, KGLM_REQ_CANCELLED = 4 };

typedef struct {
    int32_t state;                  /* KGLM_REQ_* */
    int32_t status;                 /* kglm_status of the request (KGLM_OK unless FAILED) */
    double opt;                     /* best objective found (certified when gap <= gap_tol) */
    double gap;                     /* final relative gap; > 0 if the time limit stopped the search */
    int32_t support[KGLM_MAX_K];    /* support of opt, ascending, -1 padded */
    int64_t nodes, batches;         /* nodes evaluated, batches launched */
    int64_t device_bytes;           /* admitted footprint */
    int32_t batch;                  /* node-batch size used */
    int32_t reserved;
    double t_submit, t_admit, t_done;   /* seconds since server creation; -1 until reached */
    char message[128];              /* FAILED: the failing call's message (kglm_last_error) */
} kglm_request_info;

typedef struct {
    int64_t submitted, finished, queued;
    int32_t active, peak_active;
    int64_t bytes_in_use, peak_bytes, budget;
    double elapsed_s;
    int64_t rounds;           /* scheduler rounds with at least one batch evaluated */
    int64_t round_batches;    /* node batches evaluated in those rounds */
    int64_t shared_launches;  /* iteration launches that carried the nodes of more than one request */
} kglm_server_stats_t;

/* Start a server on the current CUDA device (its scheduler thread and stream). */
kglm_status kglm_server_create(const kglm_server_desc* desc, kglm_server** out);

/* Queue an instance (the arguments of kglm_create; desc->hbm_budget is
 * ignored, desc->max_batch 0 selects the App. E.4 batch for an even share of
 * the budget, capped at batch_cap).  X and y are copied before the call
 * returns.  *id identifies the request.  KGLM_ENOMEM if the instance needs
 * more than the server's whole budget; KGLM_EINVAL for a desc kglm_create
 * would reject on its sizes (data checks happen at admission and end the
 * request as FAILED with the status of kglm_create). */
kglm_status kglm_server_submit(kglm_server* s, const kglm_desc* desc, const double* X, const double* y,
                               int64_t* id);

/* Snapshot of a request (any state). */
kglm_status kglm_server_info(kglm_server* s, int64_t id, kglm_request_info* info);

/* Block until the request has finished (DONE, FAILED or CANCELLED), at most
 * timeout_s seconds (<= 0: no limit; KGLM_ETIMEOUT when it runs out). */
kglm_status kglm_server_wait(kglm_server* s, int64_t id, double timeout_s, kglm_request_info* info);

/* Block until every submitted request has finished (timeout as above). */
kglm_status kglm_server_drain(kglm_server* s, double timeout_s);

kglm_status kglm_server_stats(kglm_server* s, kglm_server_stats_t* out);

/* Message of the last rejected submission (valid until the next call on s). */
const char* kglm_server_last_error(kglm_server* s);

/* Stop the server: running requests stop at their next batch boundary
 * (CANCELLED), queued ones are dropped; joins the workers and frees all. */
void kglm_server_destroy(kglm_server* s);

/* Self-test of the device-wait timeout path (failure detection without a GPU
 * fault; the paper has no counterpart).  Every wait in the engine's kernels
 * (the tensor-core pipelines' mbarriers) is bounded: when it runs out the
 * kernel sets an error flag, drains its own work and returns, and the call
 * that launched it returns KGLM_ETIMEOUT with the context still usable.  This
 * call launches one kernel whose wait is on an mbarrier nothing arrives on,
 * bounded by `rounds` try_wait rounds, and returns KGLM_ETIMEOUT when the
 * timeout was detected and reported (KGLM_ECUDA if it was not). */
kglm_status kglm_selftest_timeout(kglm_ctx* ctx, int32_t rounds);

/* Bounds-checked build (no counterpart in the paper; a debugging aid, since no
 * device sanitizer runs where this library is tested).  The library built with
 * KGLM_CHECKS=1 (libkglm_checks.so) checks, on the device, the indices its prox,
 * certificate and re-optimization kernels write or gather with; a failed check
 * records which kernel failed and skips the access, and the evaluation returns
 * KGLM_EINVAL naming the kernel.  kglm_checks_enabled returns 1 for that build
 * and 0 for the normal one (no device needed). */
int32_t kglm_checks_enabled(void);

/* Self-test of the bounds-checked build: launches one kernel that attempts a
 * write one past the end of a context buffer through the checked path; the
 * check catches it, the write does not happen, and the call returns KGLM_EINVAL
 * with the context still usable.  In the normal build it launches nothing and
 * returns KGLM_ESTATE. */
kglm_status kglm_selftest_checks(kglm_ctx* ctx);

/* Message of the last failed call on ctx (never NULL). */
const char* kglm_last_error(const kglm_ctx* ctx);

/* Free the context and all its device memory.  NULL is ignored. */
void kglm_destroy(kglm_ctx* ctx);

/* Engine build string, e.g. "kglm sm_103a". */
const char* kglm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KGLM_H */
