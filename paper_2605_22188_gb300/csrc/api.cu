// C ABI of the node-bound engine (include/kglm.h): instance setup, node-batch
// push, the batched evaluation pipeline, pruning/branching, and the hybrid
// CPU-GPU branch-and-bound loop of §4.1 (Fig. 1).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <exception>
#include <map>
#include <queue>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "engine.h"
#include "kglm.h"
#include "pool.h"

using namespace kglm;

// An unfinished certified solve (the open node queue and the incumbent), kept
// when kglm_solve stops before the queue is empty, for kglm_solve_checkpoint.
struct SavedNode {
    double lb;                    // the parent's bound
    int64_t id;
    std::vector<int> J0, J1;
    std::vector<double> wb;       // warm start (p values; empty: start at 0)
};
struct SavedSolve {
    bool valid = false;
    std::vector<SavedNode> open;
    double ub = INFINITY;
    std::vector<int> sup;
    std::vector<double> coef;
    int64_t nodes = 0, batches = 0, next_id = 0;
};

struct kglm_ctx {
    kglm_desc d{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::string err;
    int n = 0, p = 0, k = 0, W = 0, kind = 0, prec = 0;
    bool f64 = true;
    double lam2 = 0, M = 0, L = 0, eta = 0, c = 0, gap_tol = 1e-6;
    double data_sum = 0;          // sum of X and y (instance signature of checkpoints)
    int64_t solve_max_batches = 0;   // kglm_solve stops after this many node batches (0: no limit)
    SavedSolve saved;
    size_t bytes = 0;
    std::vector<void*> allocs;
    // instance (device)
    double *X64 = nullptr, *Xt64 = nullptr, *y64 = nullptr, *gram = nullptr, *Xty = nullptr;
    double yty = 0.0;             // y^T y (host, FP64)
    float *X32 = nullptr, *Xt32 = nullptr, *y32 = nullptr;
    float* ylo32 = nullptr;       // fl(y - y32): with y32, y to ~48 bits in FP32 pairs
    std::vector<float> ylo_host;  // its host source (kept until the context goes)
    // node batch (device), capacity mcap
    int mcap = 0, m = 0;
    bool pushed = false, evaluated = false;
    uint32_t *in_mask = nullptr, *out_mask = nullptr;
    int *kbar = nullptr, *pf = nullptr;
    void *B = nullptr, *V = nullptr, *G = nullptr, *R = nullptr;
    double *tmom = nullptr, *zeta = nullptr, *Q = nullptr;
    float* phint = nullptr;       // per node: the streaming prox's selection and threshold hints
    int *active = nullptr, *iters_done = nullptr, *support = nullptr, *jstar = nullptr;
    double *sum_loss = nullptr, *sum_conj = nullptr, *lb_now = nullptr, *primal_now = nullptr;
    double *lb_best = nullptr, *primal_last = nullptr, *ub = nullptr, *beta_re = nullptr;
    uint8_t* pruned = nullptr;
    int *d_in_ptr = nullptr, *d_out_ptr = nullptr, *d_slot = nullptr, *d_rows = nullptr, *d_slots = nullptr;
    int *d_in_idx = nullptr, *d_out_idx = nullptr;   // CSR index staging: mcap*k and mcap*p entries
    double* d_warmB = nullptr;
    void* pool = nullptr;
    int pool_slots = 0;
    DevQueue dq;                  // device-resident open-node queue (desc.open_cap > 0)
    bool dq_on = false;
    double ub_inc = INFINITY;
    int* d_err = nullptr;
    GemmScratch gs32{}, gs64{};   // split-K scratch of the CUDA-core GEMMs
    // tensor-core products (BF16 / TF32 modes): padded operand copies and TMA maps
    bool tc = false;
    int tc_kind = 0;              // 0: BF16 operands, 1: TF32
    bool x3 = false;              // FP32-accurate split: TF32 hi + lo of every operand
    // X as hi + lo in S = X V (TF32 modes).  In the BF16 mode X is rounded once:
    // there V and R are rounded to BF16 as well, and their rounding sets the
    // bound's accuracy (the bound after 50 or 300 iterations moves by the same
    // ~1e-3 relative with or without X's low part), so the low part would only
    // double the product's tensor work.
    bool xlo = false;
    int pK = 0, nK = 0;           // operand row strides (multiples of 8 elements)
    void *Xop = nullptr, *Xop_lo = nullptr, *Xtop = nullptr, *Vop = nullptr, *Rop = nullptr;
    float *Xtop_lo = nullptr, *Vop_lo = nullptr, *Rop_lo = nullptr;   // low parts (FP32-accurate mode)
    TcMap mA1{}, mB1{}, mB1lo{}, mA2{}, mB2{}, mA1lo{}, mA2lo{}, mB2lo{};
    TcMap gB1{}, gB2{};            // X and X^T maps at the bucketed tile widths of grouped launches
    int gbn1 = 0, gbn2 = 0;
    // FP32-accurate mode: beta as a TF32 hi + lo operand for the certificate's X beta
    float *Bop = nullptr, *Bop_lo = nullptr;
    TcMap mAb{}, mAblo{};
    // BF16 mode: X as TF32 hi + lo for the certificate's X beta on the tensor
    // cores (FP32-accurate, as in the FP32-accurate mode; the iterations keep BF16)
    float *Xc = nullptr, *Xc_lo = nullptr;
    TcMap mXc{}, mXclo{};
    int bnc = 0;
    bool tc_check_pending = false;   // the tensor-core error flag is on its way to the pinned staging
    int bn1 = 0, bn2 = 0;
    int tuned_batch = 0;          // kglm_autotune's choice (0: not tuned)
    bool pdl = false;             // programmatic dependent launch inside the iteration graph (tuned)
    bool pair = false;            // BF16 iteration products as CTA pairs with 256-row tiles (tuned)
    // sub-batches of the iteration loop on forked streams (tensor-core modes, tuned)
    static constexpr int kMaxSub = 4;
    int nsub = 1;
    int prox_threads = 0;         // FP32 CTA prox: threads per node (0: default; tuned)
    cudaStream_t sub_st[kMaxSub] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxSub] = {};
    GemmScratch gtc{};
    int* d_tcerr = nullptr;
    float* Gpart = nullptr;       // split slices of X^T R (summed by the prox kernel)
    // exact-splitting certificate product (reduced-precision modes): digits of
    // X (features x K) and of the batch's dual points (nodes x K), job partials
    bool cexact = false;
    ExactPlan xplan{};
    __nv_bfloat16 *DX = nullptr, *DZ = nullptr;
    double *xsig = nullptr, *ztau = nullptr, *Qerr = nullptr;
    float* Qs = nullptr;
    size_t qs_slices = 0;         // partial slices of mcap x p
    TcMap mAz{}, mBx{};
    int bnx = 0;
    int gsplit_max = 4;
    // host mirror of the evaluated batch
    std::vector<int> h_kbar, h_pf, h_jstar;
    std::vector<double> h_lb, h_ub;
    // pinned staging of the per-batch results read back to the host (asynchronous
    // copies; pageable destinations would stage and serialise each one)
    unsigned char* pin = nullptr;
    size_t pin_m = 0;   // max_batch rounded up to 8
    template <typename T>
    T* pinned(size_t off) { return reinterpret_cast<T*>(pin + off); }
    size_t off_lb() const { return 0; }
    size_t off_ub() const { return 8 * pin_m; }
    size_t off_primal() const { return 16 * pin_m; }
    size_t off_beta() const { return 24 * pin_m; }
    size_t off_jstar() const { return 24 * pin_m + 8 * pin_m * (size_t)k; }
    size_t off_iters() const { return off_jstar() + 4 * pin_m; }
    size_t off_support() const { return off_iters() + 4 * pin_m; }
    size_t off_err() const { return off_support() + 4 * pin_m * (size_t)k; }
    size_t off_tcerr() const { return off_err() + 8; }
    size_t off_kbar() const { return off_err() + 16; }
    size_t off_pf() const { return off_kbar() + 4 * pin_m; }
    size_t off_dq() const { return off_pf() + 4 * pin_m; }
    size_t pin_bytes() const { return off_dq() + 128; }
    double sum_pa = 0.0;   // sum over the batch of p - |J0(b)|
    // per-phase device timers and launch counters
    struct Rec {
        int ph;
        cudaEvent_t a, b;
    };
    bool stats_on = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<Rec> pending;
    double st_ms[KGLM_NPHASE] = {};
    double st_work[KGLM_NPHASE] = {};
    int64_t st_n[KGLM_NPHASE] = {};
    // CUDA graphs of the iteration loop, one per (batch size, iterations, timing on/off)
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        std::vector<Rec> recs;           // event pairs inside the graph (timing on)
        double work[KGLM_NPHASE] = {};
        int64_t launches[KGLM_NPHASE] = {};
    };
    std::map<std::tuple<int, int, int, int>, Graph> graphs;
    bool capturing = false;
    Graph* cap = nullptr;
};

namespace {

struct Fail {
    kglm_status st;
    std::string msg;
};

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) throw Fail{KGLM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define REQ(cond, msg)                                      \
    do {                                                    \
        if (!(cond)) throw Fail{KGLM_EINVAL, (msg)};        \
    } while (0)

template <typename F>
kglm_status guarded(kglm_ctx* ctx, F&& f) {
    try {
        f();
        return KGLM_OK;
    } catch (const Fail& e) {
        if (ctx) ctx->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->err = "host allocation failed";
        return KGLM_ENOMEM;
    } catch (const std::exception& e) {
        if (ctx) ctx->err = e.what();
        return KGLM_EINVAL;
    }
}

void* dalloc(kglm_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->d.hbm_budget > 0 && (int64_t)(c->bytes + bytes) > c->d.hbm_budget)
        throw Fail{KGLM_ENOMEM, "over the HBM budget of the context"};
    void* p = nullptr;
    // stream-ordered: no device-wide synchronization when contexts come and go
    // while others run (the serving loop)
    cudaError_t e = cudaMallocAsync(&p, bytes, c->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{KGLM_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e)};
    }
    c->allocs.push_back(p);
    c->bytes += bytes;
    return p;
}

template <typename T>
T* dalloc_t(kglm_ctx* c, size_t count) {
    return static_cast<T*>(dalloc(c, count * sizeof(T)));
}

void check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Fail{KGLM_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e)};
}

void sync(kglm_ctx* c) { CK(cudaStreamSynchronize(c->st)); }

enum Phase {
    PH_LAYOUT = 0, PH_GEMM_LINK, PH_GEMM_GRAD, PH_PROX, PH_CERT_XB, PH_CERT_DUAL, PH_CERT_Q, PH_CERT_BOUND,
    PH_REOPT, PH_SMALL, PH_COPY
};
const char* const kPhaseNames[KGLM_NPHASE] = {
    "layout", "gemm_xv_link", "gemm_xtr", "prox_fista", "cert_xb", "cert_dual_point", "cert_xtzeta",
    "cert_bound", "reopt", "prune_check", "copies"};

cudaEvent_t take_event(kglm_ctx* c) {
    if (c->ev_free.empty()) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        return e;
    }
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
}

// Brackets the launches of one phase with events on the context's stream
// (only while timing is enabled) and adds the phase's algorithmic work.
// NVTX range on the host thread (header-only NVTX v3: a no-op unless a tool such as
// Nsight Systems or ncu --nvtx is attached), so that a profile shows the phases
// of a node batch and the calls of the C ABI.
struct Nvtx {
    explicit Nvtx(const char* name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
};

struct Scope {
    kglm_ctx* c;
    int ph;
    cudaEvent_t a = nullptr;
    bool ranged = false;
    Scope(kglm_ctx* c_, int ph_, int launches, double work) : c(c_), ph(ph_) {
        if (!c->capturing) {
            nvtxRangePushA(kPhaseNames[ph]);
            ranged = true;
        }
        if (c->capturing) {                        // counted per graph launch instead
            c->cap->launches[ph] += launches;
            c->cap->work[ph] += work;
            // an external record becomes a graph node (a plain record would only order the capture)
            if (c->stats_on && cudaEventCreate(&a) == cudaSuccess)
                cudaEventRecordWithFlags(a, c->st, cudaEventRecordExternal);
            return;
        }
        c->st_n[ph] += launches;
        c->st_work[ph] += work;
        if (c->stats_on) {
            a = take_event(c);
            cudaEventRecord(a, c->st);
        }
    }
    ~Scope() {
        if (ranged) nvtxRangePop();
        if (!a) return;
        cudaEvent_t b = nullptr;
        if (c->capturing) {
            if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
            cudaEventRecordWithFlags(b, c->st, cudaEventRecordExternal);
            c->cap->recs.push_back({ph, a, b});
            return;
        }
        if (c->ev_free.empty()) {
            if (cudaEventCreate(&b) != cudaSuccess) { c->ev_free.push_back(a); return; }
        } else {
            b = c->ev_free.back();
            c->ev_free.pop_back();
        }
        cudaEventRecord(b, c->st);
        c->pending.push_back({ph, a, b});
    }
};

void harvest(kglm_ctx* c) {
    for (auto& r : c->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
            c->st_ms[r.ph] += ms;
        c->ev_free.push_back(r.a);
        c->ev_free.push_back(r.b);
    }
    c->pending.clear();
    cudaGetLastError();
}

void check_tc_error(kglm_ctx* c);

double delta_of(const kglm_ctx* c, double ub) { return isfinite(ub) ? c->gap_tol * fmax(1.0, fabs(ub)) : 0.0; }

// Largest eigenvalue of the FP64 Gram matrix by power iteration (the
// Lipschitz constant of grad F is 2||X||^2 or ||X||^2/4).
double gram_lambda_max(kglm_ctx* c) {
    const int p = c->p;
    double* v = dalloc_t<double>(c, p);
    double* w = dalloc_t<double>(c, p);
    std::vector<double> h(p, 1.0 / sqrt((double)p));
    double lam = 0.0;
    for (int it = 0; it < 500; ++it) {
        CK(cudaMemcpyAsync(v, h.data(), sizeof(double) * p, cudaMemcpyHostToDevice, c->st));
        gemm_nt_f64(c->st, p, 1, p, c->gram, p, v, p, w, 1, &c->gs64);
        check_launch();
        CK(cudaMemcpyAsync(h.data(), w, sizeof(double) * p, cudaMemcpyDeviceToHost, c->st));
        sync(c);
        double nrm = 0.0;
        for (double x : h) nrm += x * x;
        nrm = sqrt(nrm);
        if (!(nrm > 0.0)) break;
        const double lam_new = nrm;   // ||G v|| with ||v|| = 1
        for (double& x : h) x /= nrm;
        if (it > 20 && fabs(lam_new - lam) <= 1e-13 * lam_new) { lam = lam_new; break; }
        lam = lam_new;
    }
    return lam;
}

// X^T zeta of the batch's dual points (c->zeta, m x n): FP64 GEMM into c->Q,
// or in the reduced-precision modes the exact-splitting product on the
// tensor cores, whose partials and bound are recorded in the certificate's
// arguments.
void xtzeta(kglm_ctx* c, int m, CertArgs& a) {
    const int n = c->n, p = c->p;
    a.Qs = nullptr;
    if (!c->cexact) {
        gemm_nt_f64(c->st, m, p, n, c->zeta, n, c->Xt64, n, c->Q, p, &c->gs64);
        return;
    }
    const ExactPlan& x = c->xplan;
    // the batch's certificate makes zeta's digits in its dual point pass
    if (a.DZ == nullptr) exact_digits(c->st, c->zeta, m, n, (size_t)n, x.npad, x.nd, x.beta, 1, c->DZ, c->ztau);
    ExactPlan pl = x;
    const int tiles = ((p + c->bnx - 1) / c->bnx) * ((m + 127) / 128);
    exact_plan_widen(&pl, tiles, c->qs_slices * (size_t)c->mcap / (size_t)m);
    if (tc_gemm_jobs(c->st, c->mAz, c->mBx, m, p, c->bnx, pl.jobs, pl.njobs, c->Qs, (size_t)m * p, p, c->d_tcerr,
                     c->pair) != 0)
        throw Fail{KGLM_ECUDA, "tensor-core certificate product setup failed"};
    a.Qs = c->Qs;
    a.nqs = pl.njobs;
    a.qs_stride = (size_t)m * p;
    for (int t = 0; t < pl.njobs; ++t) a.qs_w[t] = pl.w[t];
    a.xsig = c->xsig;
    a.ztau = c->ztau;
    a.ebound = pl.ebound;
}

void certify(kglm_ctx* c) {
    Nvtx range("certificate");
    const int m = c->m, n = c->n, p = c->p;
    CertArgs a{};
    a.m = m; a.n = n; a.p = p; a.W = c->W; a.k = c->k; a.kind = c->kind;
    a.lam2 = c->lam2; a.M = c->M;
    a.S = c->R;                                         // the m x n buffer is free here
    a.s_is_f64 = c->f64;
    a.y = c->y64; a.y32 = c->y32; a.ylo = c->ylo32;
    a.chk = c->d_err;
    a.zeta = c->zeta; a.sum_loss = c->sum_loss; a.sum_conj = c->sum_conj;
    a.Q = c->Q; a.B = c->B; a.b_is_f64 = c->f64;
    a.in_mask = c->in_mask; a.out_mask = c->out_mask; a.kbar = c->kbar; a.pf = c->pf;
    a.lb = c->lb_now; a.primal = c->primal_now; a.support = c->support; a.jstar = c->jstar;
    if (c->cexact && !c->f64) {
        // zeta's digits for the exact-splitting X^T zeta, made by the dual point pass
        a.DZ = c->DZ; a.ztau = c->ztau;
        a.dz_npad = c->xplan.npad; a.dz_nd = c->xplan.nd; a.dz_beta = c->xplan.beta;
    }
    const double ws = c->f64 ? 8.0 : 4.0;
    {
        Scope sc(c, PH_CERT_XB, 1, 2.0 * n * c->sum_pa);
        if (c->f64) {
            gemm_nt_f64(c->st, m, n, p, (const double*)c->B, p, c->X64, p, (double*)c->R, n, &c->gs64);
        } else if (c->tc) {
            // tensor-core modes: X beta as the TF32 hi + lo split (hi hi + hi lo + lo hi,
            // FP32 accumulate; FP32-accurate), with the TF32 modes' own X hi + lo operands
            // and, in the BF16 mode, the TF32 copies of X kept for this product
            convert_pad_f32(c->st, (const float*)c->B, m, p, c->Bop, c->pK, 0, c->Bop_lo);
            check_launch();
            const bool own = c->tc_kind == 0;
            TcGemm g{};
            g.kind = 1; g.M = m; g.N = n; g.K = p; g.bn = own ? c->bnc : c->bn1;
            g.epi = TC_EPI_STORE_F32; g.out = c->R; g.ldo = n; g.err = c->d_tcerr;
            g.A2 = &c->mAblo;
            if (tc_gemm(c->st, c->mAb, own ? c->mXc : c->mB1, own ? &c->mXclo : &c->mB1lo, g, &c->gtc) != 0)
                throw Fail{KGLM_ECUDA, "tensor-core launch failed (certificate X beta)"};
        } else {
            gemm_nt_f32(c->st, m, n, p, (const float*)c->B, p, c->X32, p, (float*)c->R, n, &c->gs32);
        }
        check_launch();
    }
    {
        Scope sc(c, PH_CERT_DUAL, 1, (ws + 8.0) * (double)m * n);
        cert_dual_point(c->st, a);
        check_launch();
    }
    {
        Scope sc(c, PH_CERT_Q, c->cexact ? 2 : 1, 2.0 * n * c->sum_pa);
        xtzeta(c, m, a);
        check_launch();
    }
    {
        Scope sc(c, PH_CERT_BOUND, 1, (8.0 + ws) * c->sum_pa);
        if (cert_bound(c->st, a) != 0) throw Fail{KGLM_EINVAL, "p too large for the certificate kernel"};
        check_launch();
    }
}

__global__ void k_fold(int m, const double* lb_now, double* lb_best) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < m) lb_best[b] = fmax(lb_best[b], lb_now[b]);
}
__global__ void k_fill(int m, double* x, double v) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < m) x[b] = v;
}
__global__ void k_filli(int m, int* x, int v) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < m) x[b] = v;
}

// The prox of batch rows [row0, row0 + mr) after a tensor-core iteration's
// products (G as `splits` partial slices).
ProxArgs prox_args_rows(kglm_ctx* c, int row0, int mr, int splits, bool pdl) {
    const int p = c->p;
    const size_t es = c->tc_kind == 0 ? 2 : 4;
    ProxArgs a{};
    a.m = mr; a.p = p; a.W = c->W;
    a.G = nullptr;
    a.V = static_cast<float*>(c->V) + (size_t)row0 * p;
    a.B = static_cast<float*>(c->B) + (size_t)row0 * p;
    a.Gpart = c->Gpart + (size_t)row0 * p;
    a.gsplits = splits;
    a.gstride = (size_t)c->mcap * p;
    a.Vop = static_cast<char*>(c->Vop) + (size_t)row0 * c->pK * es;
    a.Vop_lo = c->Vop_lo ? c->Vop_lo + (size_t)row0 * c->pK : nullptr;
    a.op_ld = c->pK; a.op_bf16 = c->tc_kind == 0;
    a.in_mask = c->in_mask + (size_t)row0 * c->W; a.out_mask = c->out_mask + (size_t)row0 * c->W;
    a.kbar = c->kbar + row0; a.pf = c->pf + row0;
    a.tmom = c->tmom + row0; a.active = c->active + row0;
    a.hint = c->phint + 2 * (size_t)row0;
    a.eta = c->eta; a.c = c->c; a.M = c->M; a.restart = c->d.restart;
    a.pdl = pdl ? 1 : 0;
    a.threads = c->prox_threads;
    a.chk = c->d_err;
    return a;
}

// One FISTA iteration of batch rows [row0, row0 + mr) on stream st (tensor-core
// modes): S = X V with the link, G = X^T R as split slices, the prox.  Rows of
// different calls touch disjoint rows of every buffer, and the link product
// takes no split-K scratch while sub-batches run side by side.
void iterate_rows(kglm_ctx* c, cudaStream_t st, int row0, int mr, bool sub) {
    const int n = c->n, p = c->p;
    const double share = c->m > 0 ? (double)mr / c->m : 1.0;
    const double flops = 2.0 * n * c->sum_pa * share;
    const size_t es = c->tc_kind == 0 ? 2 : 4;
    const bool pdl = c->pdl && c->capturing && !c->stats_on;   // inside the iteration graph
    {
        Scope sc(c, PH_GEMM_LINK, 1, flops);
        TcGemm g{};
        g.kind = c->tc_kind; g.M = mr; g.N = n; g.K = p; g.bn = c->bn1;
        g.arow0 = row0;
        g.epi = c->tc_kind == 0 ? TC_EPI_LINK_BF16 : TC_EPI_LINK_F32;
        g.out = static_cast<char*>(c->Rop) + (size_t)row0 * c->nK * es;
        g.ldo = c->nK; g.y = c->y32; g.loss = c->kind; g.err = c->d_tcerr;
        if (c->x3) { g.A2 = &c->mA1lo; g.out_lo = c->Rop_lo + (size_t)row0 * c->nK; }
        g.pdl = pdl;
        g.pair = c->pair;
        if (tc_gemm(st, c->mA1, c->mB1, c->xlo ? &c->mB1lo : nullptr, g, sub ? nullptr : &c->gtc) != 0)
            throw Fail{KGLM_ECUDA, "tensor-core product setup failed"};
        check_launch();
    }
    int splits = 0;
    {
        Scope sc(c, PH_GEMM_GRAD, 1, flops);
        TcGemm g{};
        g.kind = c->tc_kind; g.M = mr; g.N = p; g.K = n; g.bn = c->bn2;
        g.arow0 = row0;
        g.epi = TC_EPI_PARTIAL; g.err = c->d_tcerr;
        g.pout = c->Gpart + (size_t)row0 * p; g.pstride = (size_t)c->mcap * p; g.pld = p;
        g.max_splits = c->gsplit_max; g.splits_used = &splits;
        if (c->x3) g.A2 = &c->mA2lo;
        g.pdl = pdl;
        g.pair = c->pair;
        if (tc_gemm(st, c->mA2, c->mB2, c->x3 ? &c->mB2lo : nullptr, g, &c->gtc) != 0)
            throw Fail{KGLM_ECUDA, "tensor-core product setup failed"};
        check_launch();
    }
    const ProxArgs a = prox_args_rows(c, row0, mr, splits, pdl);
    Scope sc(c, PH_PROX, 1, 4.0 * 5.0 * c->sum_pa * share);
    if (prox_fista_f32(st, a) != 0) throw Fail{KGLM_EINVAL, "p too large for the prox kernel"};
    check_launch();
}

void iterate(kglm_ctx* c) {
    const int m = c->m, n = c->n, p = c->p;
    const double flops = 2.0 * n * c->sum_pa;
    if (c->tc) {
        iterate_rows(c, c->st, 0, m, false);
        return;
    }
    {
        Scope sc(c, PH_GEMM_LINK, 1, flops);
        if (c->f64) gemm_link_f64(c->st, m, n, p, (const double*)c->V, c->X64, c->y64, c->kind, (double*)c->R, &c->gs64);
        else gemm_link_f32(c->st, m, n, p, (const float*)c->V, c->X32, c->y32, c->kind, (float*)c->R, &c->gs32);
        check_launch();
    }
    {
        Scope sc(c, PH_GEMM_GRAD, 1, flops);
        if (c->f64) gemm_nt_f64(c->st, m, p, n, (const double*)c->R, n, c->Xt64, n, (double*)c->G, p, &c->gs64);
        else gemm_nt_f32(c->st, m, p, n, (const float*)c->R, n, c->Xt32, n, (float*)c->G, p, &c->gs32);
        check_launch();
    }
    ProxArgs a{};
    a.m = m; a.p = p; a.W = c->W;
    a.G = c->G; a.V = c->V; a.B = c->B;
    a.in_mask = c->in_mask; a.out_mask = c->out_mask; a.kbar = c->kbar; a.pf = c->pf;
    a.tmom = c->tmom; a.active = c->active;
    a.hint = c->phint;
    a.eta = c->eta; a.c = c->c; a.M = c->M; a.restart = c->d.restart;
    a.threads = c->prox_threads;
    a.chk = c->d_err;
    Scope sc(c, PH_PROX, 1, (c->f64 ? 8.0 : 4.0) * 5.0 * c->sum_pa);
    const int rc = c->f64 ? prox_fista_f64(c->st, a) : prox_fista_f32(c->st, a);
    if (rc != 0) throw Fail{KGLM_EINVAL, "p too large for the prox kernel"};
    check_launch();
}

// Sub-batches of the current batch: rows split into nsub parts (multiples of
// 128 rows but the last), at most one per 128 rows.
int sub_count(const kglm_ctx* c) {
    if (!c->tc || c->stats_on || c->nsub <= 1) return 1;
    return std::max(1, std::min(c->nsub, c->m / 128));
}

// `count` iterations; with sub-batches, forked onto the sub-streams and joined
// back onto the context's stream (inside a graph capture this is one graph
// with parallel branches).
void iterate_many(kglm_ctx* c, int count) {
    const int ns = sub_count(c);
    if (ns == 1) {
        for (int i = 0; i < count; ++i) iterate(c);
        return;
    }
    const int per = ((c->m + ns - 1) / ns + 127) / 128 * 128;
    CK(cudaEventRecord(c->ev_fork, c->st));
    for (int q = 0; q < ns; ++q) CK(cudaStreamWaitEvent(c->sub_st[q], c->ev_fork, 0));
    for (int i = 0; i < count; ++i)
        for (int q = 0; q < ns; ++q) {
            const int r0 = q * per, mr = std::min(c->m, r0 + per) - r0;
            if (mr > 0) iterate_rows(c, c->sub_st[q], r0, mr, true);
        }
    for (int q = 0; q < ns; ++q) {
        CK(cudaEventRecord(c->ev_join[q], c->sub_st[q]));
        CK(cudaStreamWaitEvent(c->st, c->ev_join[q], 0));
    }
}

void destroy_graphs(kglm_ctx* c) {
    for (auto& kv : c->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        for (auto& r : kv.second.recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    }
    c->graphs.clear();
}

// `count` FISTA iterations of the pushed batch, replayed from a CUDA graph
// captured on first use (kernel arguments depend only on the batch size).
void run_iters(kglm_ctx* c, int count) {
    if (count <= 0) return;
    if (c->st == nullptr || c->st == cudaStreamLegacy || c->st == cudaStreamPerThread) {
        for (int i = 0; i < count; ++i) iterate(c);   // the legacy streams cannot be captured
        return;
    }
    const auto key = std::make_tuple(c->m, count, c->stats_on ? 1 : 0, sub_count(c));
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        if (c->graphs.size() >= 16) destroy_graphs(c);
        kglm_ctx::Graph& g = c->graphs[key];
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        c->cap = &g;
        try {
            iterate_many(c, count);
        } catch (...) {
            c->capturing = false;
            cudaStreamEndCapture(c->st, &graph);
            if (graph) cudaGraphDestroy(graph);
            c->graphs.erase(key);
            throw;
        }
        c->capturing = false;
        c->cap = nullptr;
        CK(cudaStreamEndCapture(c->st, &graph));
        const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            c->graphs.erase(key);
            throw Fail{KGLM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)};
        }
        it = c->graphs.find(key);
    }
    kglm_ctx::Graph& g = it->second;
    CK(cudaGraphLaunch(g.exec, c->st));
    for (int ph = 0; ph < KGLM_NPHASE; ++ph) {
        c->st_n[ph] += g.launches[ph];
        c->st_work[ph] += g.work[ph];
    }
    if (!g.recs.empty()) {                          // timing on: read the graph's events
        sync(c);
        for (auto& r : g.recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) c->st_ms[r.ph] += ms;
        }
        cudaGetLastError();
    }
}

// The steps of one batch evaluation: the bound and iteration counters reset,
// a certificate check after `it` iterations (bounds kept, finished nodes frozen,
// the active flags copied to h asynchronously: the caller synchronises), and the
// final certificate, bound fold and re-optimization.
void evaluate_begin(kglm_ctx* c, int iters) {
    const int m = c->m;
    const unsigned gb = (unsigned)((m + 255) / 256);
    Scope sc(c, PH_SMALL, 2, 0.0);
    k_fill<<<gb, 256, 0, c->st>>>(m, c->lb_best, -INFINITY);
    k_filli<<<gb, 256, 0, c->st>>>(m, c->iters_done, iters);
    check_launch();
}

void evaluate_check(kglm_ctx* c, int it, std::vector<int>& h) {
    const int m = c->m;
    const double thr = c->ub_inc - delta_of(c, c->ub_inc);
    certify(c);
    {
        Scope sc(c, PH_SMALL, 1, 0.0);
        check_update(c->st, m, c->lb_now, c->primal_now, c->lb_best, c->primal_last, c->active, c->iters_done, it, thr,
                     1e-9);
        check_launch();
    }
    h.resize(m);
    Scope sc(c, PH_COPY, 0, 4.0 * m);
    CK(cudaMemcpyAsync(h.data(), c->active, sizeof(int) * m, cudaMemcpyDeviceToHost, c->st));
}

void evaluate_end(kglm_ctx* c) {
    const int m = c->m;
    const unsigned gb = (unsigned)((m + 255) / 256);
    certify(c);
    {
        Scope sc(c, PH_SMALL, 1, 0.0);
        k_fold<<<gb, 256, 0, c->st>>>(m, c->lb_now, c->lb_best);
        check_launch();
    }
    ReoptArgs r{};
    r.m = m; r.n = c->n; r.p = c->p; r.k = c->k; r.kind = c->kind;
    r.max_iter = 100;                                   // projected Newton steps
    r.lam2 = c->lam2; r.M = c->M; r.tol = 1e-12;
    r.Xt = c->Xt64; r.y = c->y64; r.gram = c->gram; r.Xty = c->Xty;
    r.Xt32 = c->f64 ? nullptr : c->Xt32;
    r.y32 = c->f64 ? nullptr : c->y32;
    r.support = c->support; r.B = c->B; r.b_is_f64 = c->f64;
    r.ub = c->ub; r.beta_re = c->beta_re;
    r.yty = c->yty;
    r.chk = c->d_err;
    {
        Scope sc(c, PH_REOPT, 1, 0.0);
        if (reopt_launch(c->st, r) != 0) throw Fail{KGLM_ECUDA, "re-optimization kernel: shared memory for k refused"};
        check_launch();
    }
    if (c->tc || c->cexact) {
        // read back with the results (one synchronisation), checked by finish_tc_check
        CK(cudaMemcpyAsync(c->pinned<int>(c->off_tcerr()), c->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        c->tc_check_pending = true;
    }
}

void evaluate_impl(kglm_ctx* c, int iters, int check_every) {
    Nvtx range("kglm evaluate: iterations, certificate, rounding, re-optimization");
    evaluate_begin(c, iters);
    std::vector<int> h_active;
    for (int it = 0; it < iters;) {
        const int seg = check_every > 0 ? std::min(check_every, iters - it) : iters - it;
        run_iters(c, seg);
        it += seg;
        if (check_every > 0 && it % check_every == 0 && it < iters) {
            evaluate_check(c, it, h_active);
            sync(c);
            bool any = false;
            for (int v : h_active) any |= (v != 0);
            if (!any) break;
        }
    }
    evaluate_end(c);
}

// ---- several contexts' batches in shared launches (the serving loop)
// BF16 contexts with single operands and p in the streaming prox's range take
// part: per FISTA iteration one launch of S = X V + link and one of G = X^T R
// for every (tile width, up to 8 contexts), and one streaming prox launch for
// up to 8 contexts' nodes.  Each context keeps its own split-K (set from its
// own shape) and node-level work, so its results do not depend on the others;
// the tile width is bucketed from its own n and p.  Other contexts run their
// iterations with their own launches in the same round.
bool groupable(const kglm_ctx* c) {
    return c->tc && c->tc_kind == 0 && !c->x3 && !c->xlo && c->p <= kStreamMaxP && c->m > 0;
}

int bucket_bn(int N) { return N >= 256 ? 256 : (N >= 128 ? 128 : 64); }

void group_maps(kglm_ctx* c) {
    const int b1 = bucket_bn(c->n), b2 = bucket_bn(c->p);
    if (c->gbn1 == b1 && c->gbn2 == b2) return;
    if (tc_make_map(&c->gB1, c->Xop, 1, c->n, c->p, c->pK, b1) ||
        tc_make_map(&c->gB2, c->Xtop, 1, c->p, c->n, c->nK, b2))
        throw Fail{KGLM_ECUDA, "cuTensorMapEncodeTiled failed for a grouped product"};
    c->gbn1 = b1;
    c->gbn2 = b2;
}

void iterate_group(const std::vector<kglm_ctx*>& A, int64_t* shared) {
    std::vector<kglm_ctx*> g;
    for (kglm_ctx* c : A) {
        if (groupable(c)) {
            group_maps(c);
            g.push_back(c);
        } else {
            iterate(c);
        }
    }
    if (g.empty()) return;
    cudaStream_t st = g[0]->st;
    std::vector<int> splits(g.size(), 1);
    for (int grad = 0; grad < 2; ++grad) {
        std::vector<char> done(g.size(), 0);
        for (size_t i = 0; i < g.size(); ++i) {
            if (done[i]) continue;
            const int bn = grad ? g[i]->gbn2 : g[i]->gbn1;
            std::vector<TcGroupItem> items;
            for (size_t j = i; j < g.size() && (int)items.size() < kGroupMax; ++j) {
                if (done[j] || (grad ? g[j]->gbn2 : g[j]->gbn1) != bn) continue;
                done[j] = 1;
                kglm_ctx* c = g[j];
                TcGroupItem it{};
                it.M = c->m;
                if (!grad) {
                    it.A = &c->mA1; it.B = &c->gB1; it.N = c->n; it.K = c->p;
                    it.out = c->Rop; it.ldo = c->nK; it.y = c->y32; it.loss = c->kind;
                } else {
                    it.A = &c->mA2; it.B = &c->gB2; it.N = c->p; it.K = c->n;
                    it.pout = c->Gpart; it.pstride = (size_t)c->mcap * c->p; it.pld = c->p;
                    it.max_splits = c->gsplit_max; it.splits_bn = c->bn2; it.splits_used = &splits[j];
                }
                items.push_back(it);
            }
            Scope sc(g[i], grad ? PH_GEMM_GRAD : PH_GEMM_LINK, 1, 0.0);
            if (tc_gemm_group(st, items.data(), (int)items.size(), bn, grad ? TC_EPI_PARTIAL : TC_EPI_LINK_BF16,
                              g[i]->d_tcerr) != 0)
                throw Fail{KGLM_ECUDA, "grouped tensor-core product setup failed"};
            check_launch();
            if (shared && items.size() > 1) ++*shared;
        }
    }
    for (size_t i0 = 0; i0 < g.size(); i0 += kGroupMax) {
        ProxGroup pg{};
        pg.np = (int)std::min<size_t>(kGroupMax, g.size() - i0);
        for (int t = 0; t < pg.np; ++t) pg.a[t] = prox_args_rows(g[i0 + t], 0, g[i0 + t]->m, splits[i0 + t], false);
        Scope sc(g[i0], PH_PROX, 1, 0.0);
        const int rc = prox_stream_group(st, pg);
        if (rc < 0) throw Fail{KGLM_ECUDA, "prox kernel: shared memory attribute refused"};
        if (rc == 1)
            for (int t = 0; t < pg.np; ++t)
                if (prox_fista_f32(st, pg.a[t]) != 0) throw Fail{KGLM_EINVAL, "p too large for the prox kernel"};
        check_launch();
        if (shared && rc == 0 && pg.np > 1) ++*shared;
    }
}

// evaluate_impl of every context (all on one stream), their iterations in shared
// launches (*shared counts the launches that carried more than one context)
void evaluate_group(const std::vector<kglm_ctx*>& cs, int iters, int check_every, int64_t* shared) {
    Nvtx range("kglm evaluate (grouped contexts)");
    for (kglm_ctx* c : cs) {
        REQ(c->pushed, "evaluate before push");
        REQ(c->st == cs[0]->st, "grouped contexts must share one stream");
    }
    for (kglm_ctx* c : cs) evaluate_begin(c, iters);
    std::vector<kglm_ctx*> A(cs);
    std::vector<std::vector<int>> h;
    for (int it = 0; it < iters && !A.empty();) {
        const int seg = check_every > 0 ? std::min(check_every, iters - it) : iters - it;
        for (int i = 0; i < seg; ++i) iterate_group(A, shared);
        it += seg;
        if (check_every > 0 && it % check_every == 0 && it < iters) {
            h.resize(A.size());
            for (size_t i = 0; i < A.size(); ++i) evaluate_check(A[i], it, h[i]);
            sync(A[0]);
            std::vector<kglm_ctx*> keep;
            for (size_t i = 0; i < A.size(); ++i) {
                bool any = false;
                for (int v : h[i]) any |= (v != 0);
                if (any) keep.push_back(A[i]);
            }
            A.swap(keep);
        }
    }
    for (kglm_ctx* c : cs) evaluate_end(c);
}

// After a synchronisation that follows evaluate_impl: the tensor-core error flag
// it sent to the pinned staging.
void finish_tc_check(kglm_ctx* c) {
#if KGLM_CHECKS
    {
        // the bounds-checked build: which kernel's device check failed, if any
        int h = 0;
        CK(cudaMemcpyAsync(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        sync(c);
        if (h & kChkAll) {
            CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
            sync(c);
            throw Fail{KGLM_EINVAL, std::string("device bounds check failed in") + ((h & kChkProx) ? " the prox" : "") +
                                        ((h & kChkCert) ? " the certificate" : "") +
                                        ((h & kChkReopt) ? " the re-optimization" : "")};
        }
    }
#endif
    if (!c->tc_check_pending) return;
    c->tc_check_pending = false;
    if (*c->pinned<int>(c->off_tcerr())) {
        CK(cudaMemsetAsync(c->d_tcerr, 0, sizeof(int), c->st));
        throw Fail{KGLM_ETIMEOUT, "a tensor-core product's pipeline wait ran out"};
    }
}

// A tensor-core product whose mbarrier wait ran out leaves a flag (the kernel
// drained its work and freed its tensor memory before returning).
void check_tc_error(kglm_ctx* c) {
    int h = 0;
    CK(cudaMemcpyAsync(&h, c->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    sync(c);
    if (h) {
        CK(cudaMemsetAsync(c->d_tcerr, 0, sizeof(int), c->st));
        throw Fail{KGLM_ETIMEOUT, "a tensor-core product's pipeline wait ran out"};
    }
}

void validate_nodes(const kglm_ctx* c, int m, const int32_t* in_ptr, const int32_t* in_idx,
                    const int32_t* out_ptr, const int32_t* out_idx, const int32_t* warm_slot) {
    REQ(m >= 1 && m <= c->mcap, "m must be in [1, max_batch]");
    REQ(in_ptr && out_ptr, "in_ptr and out_ptr are required");
    REQ(in_ptr[0] == 0 && out_ptr[0] == 0, "CSR offsets must start at 0");
    std::vector<int> stamp(c->p, -1);
    for (int b = 0; b < m; ++b) {
        REQ(in_ptr[b + 1] >= in_ptr[b] && out_ptr[b + 1] >= out_ptr[b], "CSR offsets must be non-decreasing");
        REQ(in_ptr[b + 1] - in_ptr[b] <= c->k, "|J1| > k");
        for (int t = in_ptr[b]; t < in_ptr[b + 1]; ++t) {
            const int j = in_idx[t];
            REQ(j >= 0 && j < c->p, "J1 index out of range");
            REQ(stamp[j] != 2 * b, "repeated J1 index");
            stamp[j] = 2 * b;
        }
        for (int t = out_ptr[b]; t < out_ptr[b + 1]; ++t) {
            const int j = out_idx[t];
            REQ(j >= 0 && j < c->p, "J0 index out of range");
            REQ(stamp[j] != 2 * b, "J0 and J1 overlap");
            REQ(stamp[j] != 2 * b + 1, "repeated J0 index");
            stamp[j] = 2 * b + 1;
        }
        if (warm_slot) REQ(warm_slot[b] >= -1 && warm_slot[b] < c->pool_slots, "warm slot out of range");
    }
}

void push_impl(kglm_ctx* c, int m, const int32_t* in_ptr, const int32_t* in_idx, const int32_t* out_ptr,
               const int32_t* out_idx, const int32_t* warm_slot, const double* warm_B) {
    validate_nodes(c, m, in_ptr, in_idx, out_ptr, out_idx, warm_slot);
    const size_t nnz_in = in_ptr[m], nnz_out = out_ptr[m];   // <= m k and <= m p (validated)
    if (!c->d_warmB && warm_B) c->d_warmB = dalloc_t<double>(c, (size_t)c->mcap * c->p);
    const int* slot = warm_slot ? c->d_slot : nullptr;
    const double* wb = warm_B ? c->d_warmB : nullptr;
    {
        Scope sc(c, PH_COPY, 0, 4.0 * (2.0 * (m + 1) + nnz_in + nnz_out + (warm_slot ? m : 0)) +
                                    (warm_B ? 8.0 * m * c->p : 0.0));
        CK(cudaMemcpyAsync(c->d_in_ptr, in_ptr, sizeof(int) * (m + 1), cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(c->d_out_ptr, out_ptr, sizeof(int) * (m + 1), cudaMemcpyHostToDevice, c->st));
        if (nnz_in) CK(cudaMemcpyAsync(c->d_in_idx, in_idx, sizeof(int) * nnz_in, cudaMemcpyHostToDevice, c->st));
        if (nnz_out) CK(cudaMemcpyAsync(c->d_out_idx, out_idx, sizeof(int) * nnz_out, cudaMemcpyHostToDevice, c->st));
        if (warm_slot) CK(cudaMemcpyAsync(c->d_slot, warm_slot, sizeof(int) * m, cudaMemcpyHostToDevice, c->st));
        if (warm_B)
            CK(cudaMemcpyAsync(c->d_warmB, warm_B, sizeof(double) * (size_t)m * c->p, cudaMemcpyHostToDevice, c->st));
    }
    c->h_kbar.resize(m);
    c->h_pf.resize(m);
    c->sum_pa = 0.0;
    for (int b = 0; b < m; ++b) {
        const int n1 = in_ptr[b + 1] - in_ptr[b], n0 = out_ptr[b + 1] - out_ptr[b];
        c->h_kbar[b] = c->k - n1;
        c->h_pf[b] = c->p - n1 - n0;
        c->sum_pa += c->p - n0;
    }
    {
        Scope sc(c, PH_LAYOUT, 0, (c->f64 ? 16.0 : 8.0) * m * c->p);
        c->st_n[PH_LAYOUT] += layout_masks(c->st, m, c->p, c->W, c->k, c->d_in_ptr, c->d_in_idx, c->d_out_ptr,
                                           c->d_out_idx, c->in_mask, c->out_mask, c->kbar, c->pf, (int)nnz_in,
                                           (int)nnz_out, nullptr);
        check_launch();
        c->st_n[PH_LAYOUT] += layout_warm(c->st, m, c->p, c->W, c->f64, slot, c->pool_slots, c->pool, wb,
                                          c->out_mask, c->B, c->V, c->Vop, c->Vop_lo, c->pK, c->tc_kind == 0, c->tmom, c->active, c->phint);
        check_launch();
    }
    sync(c);   // host arrays may be pageable and reused by the caller
    c->m = m;
    c->pushed = true;
    c->evaluated = false;
}

void push_dev_impl(kglm_ctx* c, int m, const int32_t* in_ptr, const int32_t* in_idx, const int32_t* out_ptr,
                   const int32_t* out_idx, int nnz_in, int nnz_out, const int32_t* warm_slot) {
    REQ(m >= 1 && m <= c->mcap, "m must be in [1, max_batch]");
    REQ(in_ptr && out_ptr, "in_ptr and out_ptr are required");
    REQ(nnz_in >= 0 && nnz_out >= 0, "nnz must be >= 0");
    REQ((nnz_in == 0 || in_idx) && (nnz_out == 0 || out_idx), "index arrays are required");
    c->pushed = false;
    c->evaluated = false;
    std::vector<int> hk(m), hp(m);
    int herr = 0;
    {
        Scope sc(c, PH_LAYOUT, 0, (c->f64 ? 16.0 : 8.0) * m * c->p);
        CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->st));
        c->st_n[PH_LAYOUT] += layout_masks(c->st, m, c->p, c->W, c->k, in_ptr, in_idx, out_ptr, out_idx, c->in_mask,
                                           c->out_mask, c->kbar, c->pf, nnz_in, nnz_out, c->d_err);
        check_launch();
        c->st_n[PH_LAYOUT] += layout_validate(c->st, m, c->k, c->W, nnz_in, nnz_out, in_ptr, out_ptr, c->in_mask,
                                              c->out_mask, warm_slot, c->pool_slots, c->d_err);
        check_launch();
        c->st_n[PH_LAYOUT] += layout_warm(c->st, m, c->p, c->W, c->f64, warm_slot, c->pool_slots, c->pool, nullptr,
                                          c->out_mask, c->B, c->V, c->Vop, c->Vop_lo, c->pK, c->tc_kind == 0, c->tmom, c->active, c->phint);
        check_launch();
    }
    {
        Scope sc(c, PH_COPY, 0, 4.0 + 8.0 * m);
        CK(cudaMemcpyAsync(c->pinned<int>(c->off_err()), c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(c->pinned<int>(c->off_kbar()), c->kbar, sizeof(int) * m, cudaMemcpyDeviceToHost, c->st));
        CK(cudaMemcpyAsync(c->pinned<int>(c->off_pf()), c->pf, sizeof(int) * m, cudaMemcpyDeviceToHost, c->st));
    }
    sync(c);
    herr = *c->pinned<int>(c->off_err());
    memcpy(hk.data(), c->pinned<int>(c->off_kbar()), sizeof(int) * m);
    memcpy(hp.data(), c->pinned<int>(c->off_pf()), sizeof(int) * m);
    if (herr) throw Fail{KGLM_EINVAL, std::string("device checks of the pushed batch failed (") +
                                          ((herr & 1) ? "index out of range " : "") +
                                          ((herr & 2) ? "bad offsets, |J1| > k, repeat or J0/J1 overlap " : "") +
                                          ((herr & 4) ? "warm slot out of range" : "") + ")"};
    c->h_kbar = hk;
    c->h_pf = hp;
    c->sum_pa = 0.0;
    for (int b = 0; b < m; ++b) c->sum_pa += hp[b] + (c->k - hk[b]);
    c->m = m;
    c->pushed = true;
}

void evaluate_outputs(kglm_ctx* c, double* lb, double* primal, double* ub_cand, int32_t* support,
                      double* beta_re, int32_t* branch_j, int32_t* iters_done) {
    const int m = c->m;
    c->h_lb.resize(m);
    c->h_ub.resize(m);
    c->h_jstar.resize(m);
    Scope sc(c, PH_COPY, 0, (double)m * (20.0 + (primal ? 8 : 0) + (support ? 4.0 * c->k : 0) +
                                         (beta_re ? 8.0 * c->k : 0) + (iters_done ? 4 : 0)));
    const size_t mk = (size_t)m * c->k;
    CK(cudaMemcpyAsync(c->pinned<double>(c->off_lb()), c->lb_best, sizeof(double) * m, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(c->pinned<double>(c->off_ub()), c->ub, sizeof(double) * m, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(c->pinned<int>(c->off_jstar()), c->jstar, sizeof(int) * m, cudaMemcpyDeviceToHost, c->st));
    if (primal)
        CK(cudaMemcpyAsync(c->pinned<double>(c->off_primal()), c->primal_now, sizeof(double) * m, cudaMemcpyDeviceToHost, c->st));
    if (support)
        CK(cudaMemcpyAsync(c->pinned<int>(c->off_support()), c->support, sizeof(int) * mk, cudaMemcpyDeviceToHost, c->st));
    if (beta_re)
        CK(cudaMemcpyAsync(c->pinned<double>(c->off_beta()), c->beta_re, sizeof(double) * mk, cudaMemcpyDeviceToHost, c->st));
    if (iters_done)
        CK(cudaMemcpyAsync(c->pinned<int>(c->off_iters()), c->iters_done, sizeof(int) * m, cudaMemcpyDeviceToHost, c->st));
    sync(c);
    finish_tc_check(c);
    memcpy(c->h_lb.data(), c->pinned<double>(c->off_lb()), sizeof(double) * m);
    memcpy(c->h_ub.data(), c->pinned<double>(c->off_ub()), sizeof(double) * m);
    memcpy(c->h_jstar.data(), c->pinned<int>(c->off_jstar()), sizeof(int) * m);
    if (primal) memcpy(primal, c->pinned<double>(c->off_primal()), sizeof(double) * m);
    if (support) memcpy(support, c->pinned<int>(c->off_support()), sizeof(int) * mk);
    if (beta_re) memcpy(beta_re, c->pinned<double>(c->off_beta()), sizeof(double) * mk);
    if (iters_done) memcpy(iters_done, c->pinned<int>(c->off_iters()), sizeof(int) * m);
    harvest(c);
    if (lb) memcpy(lb, c->h_lb.data(), sizeof(double) * m);
    if (ub_cand) memcpy(ub_cand, c->h_ub.data(), sizeof(double) * m);
    if (branch_j) memcpy(branch_j, c->h_jstar.data(), sizeof(int) * m);
}

// Device bytes kglm_create allocates for desc: the same allocations, in the
// same order (the exact-splitting digits are skipped when they would pass the
// budget), so that admission control can decide before any allocation.
// Excluded: the buffers that kglm_push_nodes with warm_B and kglm_xtz
// allocate on first use (one max_batch x p FP64 array each).
size_t footprint(const kglm_desc& d) {
    size_t est = 0;
    auto add = [&](size_t b) { est += b == 0 ? 16 : b; };
    const size_t n = (size_t)d.n, p = (size_t)d.p, mc = (size_t)d.max_batch, k = (size_t)d.k;
    const bool f64 = d.prec == KGLM_FP64, tc = d.prec == KGLM_BF16 || d.prec == KGLM_TF32 || d.prec == KGLM_TF32X3;
    const bool x3 = d.prec == KGLM_TF32X3;
    const size_t ws = f64 ? 8 : 4, W = (p + 31) / 32;
    add(8 * n * p); add(8 * n * p); add(8 * n);
    if (!f64) { add(4 * n * p); add(4 * n * p); add(4 * n); add(4 * n); }
    add(gemm_scratch_bytes(1)); add(4 * (size_t)gemm_scratch_counters(1));
    if (!f64) { add(gemm_scratch_bytes(0)); add(4 * (size_t)gemm_scratch_counters(0)); }
    bool tcerr = false;
    if (tc) {
        const size_t es = d.prec == KGLM_BF16 ? 2 : 4;
        const size_t pK = (p + 7) / 8 * 8, nK = (n + 7) / 8 * 8;
        add(n * pK * es); if (d.prec != KGLM_BF16) add(n * pK * es); add(p * nK * es);
        if (x3) add(4 * p * nK);
        add(mc * pK * es); add(mc * nK * es);
        if (x3) { add(4 * mc * pK); add(4 * mc * nK); }
        add(4 * mc * pK); add(4 * mc * pK);                              // beta hi + lo (certificate)
        if (d.prec == KGLM_BF16) { add(4 * n * pK); add(4 * n * pK); }  // X as TF32 hi + lo (certificate)
        add(tc_scratch_bytes()); add(4 * (size_t)tc_scratch_counters());
        add(4 * (size_t)tc_split_cap((int)mc, (int)p) * mc * p);   // split slices of X^T R
        add(4);
        tcerr = true;
    }
    add(8 * p * p); add(8 * p);
    if (!(d.lipschitz > 0)) { add(8 * p); add(8 * p); }
    add(4 * mc * W); add(4 * mc * W); add(4 * mc); add(4 * mc);
    add(mc * p * ws); add(mc * p * ws); add(mc * p * ws);
    add(mc * n * std::max(ws, (size_t)4));
    add(8 * mc); add(4 * mc); add(8 * mc); add(4 * mc);
    add(8 * mc * n); add(8 * mc * p);
    for (int t = 0; t < 7; ++t) add(8 * mc);
    add(8 * mc * k); add(4 * mc * k); add(4 * mc); add(mc);
    add(4 * (mc + 1)); add(4 * (mc + 1)); add(4 * mc); add(4 * std::max(mc, k)); add(4 * mc); add(4);
    const size_t slots = d.pool_slots > 0 ? (size_t)d.pool_slots : 4 * mc;
    add(slots * p * ws);
    add(4 * mc * k); add(4 * mc * p);
    if (d.open_cap > 0) {
        const size_t cap = (size_t)d.open_cap, W2 = 2 * W, m2 = 2 * mc;
        for (int b = 0; b < 2; ++b) { add(8 * cap); add(8 * cap); add(4 * cap); add(4 * cap * W2); }
        add(8 * m2); add(8 * m2); add(4 * m2); add(4 * m2 * W2); add(4 * m2);
        add(8 * mc); add(4 * mc); add(4 * mc); add(4 * mc);
        add(4 * slots); add(4 * slots); add(4 * k); add(8 * k);
        add(sizeof(DqState));
    }
    ExactPlan x{};
    if (!f64 && exact_plan((int)n, 6, 7, &x)) {
        const size_t K2 = (size_t)x.nd * x.npad;
        const size_t need = 2 * K2 * (p + mc) + 8 * (p + mc) + 4 * (size_t)x.njobs * mc * p + 64;
        if (d.hbm_budget <= 0 || (int64_t)(est + need) <= d.hbm_budget) {
            add(2 * p * K2); add(8 * p); add(2 * mc * K2); add(8 * mc); add(4 * (size_t)x.njobs * mc * p);
            if (!tcerr) add(4);
        }
    }
    return est;
}

// The hybrid CPU-GPU loop of Fig. 1 on one context: best-bound host queue,
// batches of up to `batch` open nodes evaluated on the device, incumbent from
// the batched rounding and re-optimization, pruning and branching on j*.
// Stops when the queue is empty, the time limit passes or *cancel is set
// (checked between batches).
struct SolveOut {
    double opt = INFINITY, gap = INFINITY;
    std::vector<int> support;
    std::vector<double> beta;
    int64_t nodes = 0, batches = 0;
    bool cancelled = false;
    bool complete = false;       // the open queue was emptied
};

// Rashomon-set collection (§4.5): prune a node only when its bound exceeds
// tau = min((1 + eps) UB, the cap-th best stored objective), keep every
// re-optimized support whose objective is at most tau, and branch until a
// node holds a single support (kbar = 0 or no free coordinate).
struct RashomonOpts {
    double eps = 0.0;
    int64_t cap = 0;
    kglm_pool* pool = nullptr;
};

// FP64 objective F(X_S b) + lambda2 ||b||^2 of a support (k entries, -1 padded)
// with its coefficients; `fallback` when the support is empty.
double exact_objective(kglm_ctx* ctx, const std::vector<int>& sup, const std::vector<double>& coef,
                       double fallback) {
    std::vector<int> Sv;
    std::vector<double> bv;
    for (int r = 0; r < ctx->k; ++r)
        if (sup[r] >= 0) { Sv.push_back(sup[r]); bv.push_back(coef[r]); }
    const int ks = (int)Sv.size();
    if (ks == 0) return fallback;
    CK(cudaMemcpyAsync(ctx->d_rows, Sv.data(), sizeof(int) * ks, cudaMemcpyHostToDevice, ctx->st));
    CK(cudaMemcpyAsync(ctx->beta_re, bv.data(), sizeof(double) * ks, cudaMemcpyHostToDevice, ctx->st));
    objective64_launch(ctx->st, ctx->Xt64, ctx->y64, ctx->n, ctx->kind, ctx->lam2, ctx->d_rows, ctx->beta_re, ks,
                       ctx->ub);
    check_launch();
    double exact = fallback;
    CK(cudaMemcpyAsync(&exact, ctx->ub, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
    sync(ctx);
    return exact;
}

// The hybrid loop of Fig. 1 with the open-node queue on the device (queue.cu),
// in steps so that a scheduler can interleave the batches of several
// contexts: begin(); per round select() (0: nothing open), the batch's
// evaluation, update(); finish().  The host reads the queue's state (a few
// scalars) once after each step; node data never leaves the device.
struct DevSolve {
    kglm_ctx* c = nullptr;
    int batch = 0;
    DqState hs{};
    int64_t nodes = 0, batches = 0;
    bool overflow = false;

    void read_state() {
        CK(cudaMemcpyAsync(c->pinned<DqState>(c->off_dq()), c->dq.st, sizeof(DqState), cudaMemcpyDeviceToHost, c->st));
        sync(c);
        hs = *c->pinned<DqState>(c->off_dq());
    }
    void begin() {
        c->saved = SavedSolve{};                       // a device-queue search leaves no host checkpoint
        dq_init(c->st, c->dq);
        check_launch();
        read_state();
    }
    // the next batch into the batch arrays; its size
    int select() {
        if (hs.N == 0 || overflow) return 0;
        {
            Scope sc(c, PH_LAYOUT, 2, 8.0 * c->W * batch);
            dq_select(c->st, c->dq, batch, c->gap_tol, c->in_mask, c->out_mask, c->kbar, c->pf);
            check_launch();
        }
        read_state();
        const int m = hs.m;
        if (m == 0) return 0;
        {
            Scope sc(c, PH_LAYOUT, 0, (c->f64 ? 16.0 : 8.0) * m * c->p);
            c->st_n[PH_LAYOUT] += layout_warm(c->st, m, c->p, c->W, c->f64, c->dq.bslot, c->pool_slots, c->pool,
                                              nullptr, c->out_mask, c->B, c->V, c->Vop, c->Vop_lo, c->pK,
                                              c->tc_kind == 0, c->tmom, c->active, c->phint);
            check_launch();
        }
        c->m = m;
        c->pushed = true;
        c->evaluated = false;
        c->sum_pa = (double)m * c->p - (double)hs.sum_out;
        c->ub_inc = hs.ub;
        return m;
    }
    // incumbent, closing and branching, children and the merged pool
    void update() {
        {
            Scope sc(c, PH_SMALL, 7, 0.0);
            dq_update(c->st, c->dq, c->m, hs.N, c->gap_tol, c->lb_best, c->ub, c->jstar, c->support, c->beta_re,
                      c->in_mask, c->out_mask, c->B, c->f64, c->pool);
            check_launch();
        }
        read_state();
        finish_tc_check(c);
        harvest(c);
        c->evaluated = true;
        nodes += c->m;
        ++batches;
        overflow = hs.overflow != 0;
    }
    void finish(SolveOut& out, bool stopped) {
        const int k = c->k;
        std::vector<int> sup(k);
        std::vector<double> coef(k);
        double open_lb = INFINITY;
        CK(cudaMemcpyAsync(c->pinned<int>(c->off_support()), c->dq.best_sup, sizeof(int) * k, cudaMemcpyDeviceToHost,
                           c->st));
        CK(cudaMemcpyAsync(c->pinned<double>(c->off_beta()), c->dq.best_coef, sizeof(double) * k,
                           cudaMemcpyDeviceToHost, c->st));
        if (hs.N > 0)                                   // the pool is sorted: its first bound is the least
            CK(cudaMemcpyAsync(c->pinned<double>(c->off_lb()), c->dq.lb[c->dq.cur], sizeof(double),
                               cudaMemcpyDeviceToHost, c->st));
        sync(c);
        memcpy(sup.data(), c->pinned<int>(c->off_support()), sizeof(int) * k);
        memcpy(coef.data(), c->pinned<double>(c->off_beta()), sizeof(double) * k);
        if (hs.N > 0) open_lb = *c->pinned<double>(c->off_lb());
        double ub = hs.ub;
        if (!c->f64 && isfinite(ub)) ub = exact_objective(c, sup, coef, ub);
        out.complete = hs.N == 0 && !overflow && !stopped;
        const double glb = std::min(open_lb, ub);
        out.opt = ub;
        out.gap = isfinite(ub) ? (ub - glb) / fmax(1.0, fabs(ub)) : INFINITY;
        out.nodes = nodes;
        out.batches = batches;
        out.support = sup;
        out.beta.assign(c->p, 0.0);
        for (int r = 0; r < k; ++r)
            if (sup[r] >= 0) out.beta[sup[r]] = coef[r];
    }
};

void solve_dev_impl(kglm_ctx* ctx, int batch, int iters, int check_every, double time_limit_s,
                    const std::atomic<int>* cancel, SolveOut& out) {
    REQ(ctx->dq_on, "the context has no device queue (created with open_cap = 0)");
    REQ(batch >= 1 && batch <= ctx->mcap, "batch must be in [1, max_batch]");
    REQ(iters >= 1, "iters must be >= 1");
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&] { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    DevSolve d;
    d.c = ctx;
    d.batch = batch;
    d.begin();
    bool stopped = false;
    for (;;) {
        if ((time_limit_s > 0 && elapsed() > time_limit_s) ||
            (ctx->solve_max_batches > 0 && d.batches >= ctx->solve_max_batches)) {
            stopped = true;
            break;
        }
        if (cancel && cancel->load(std::memory_order_relaxed)) {
            out.cancelled = true;
            stopped = true;
            break;
        }
        Nvtx range("bnb batch (device queue)");
        if (d.select() == 0) break;
        evaluate_impl(ctx, iters, check_every);
        d.update();
    }
    d.finish(out, stopped);
}

void solve_impl(kglm_ctx* ctx, int batch, int iters, int check_every, double time_limit_s,
                const std::atomic<int>* cancel, SolveOut& out, const RashomonOpts* rs = nullptr,
                const SavedSolve* resume = nullptr) {
    REQ(batch >= 1 && batch <= ctx->mcap, "batch must be in [1, max_batch]");
    REQ(iters >= 1, "iters must be >= 1");
    struct Open {
        double lb;
        int64_t id;
        std::vector<int> J0, J1;
        int slot;
        std::vector<double> wb;   // host warm start (resumed nodes), used when slot < 0
    };
    struct Cmp {
        bool operator()(const Open* a, const Open* b) const {
            return a->lb > b->lb || (a->lb == b->lb && a->id > b->id);
        }
    };
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&] {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    std::priority_queue<Open*, std::vector<Open*>, Cmp> open;
    std::vector<int> slot_ref(ctx->pool_slots, 0), free_slots;
    for (int s = ctx->pool_slots - 1; s >= 0; --s) free_slots.push_back(s);
    auto release = [&](int s) {
        if (s >= 0 && --slot_ref[s] == 0) free_slots.push_back(s);
    };
    int64_t next_id = 0, n_nodes = 0, n_batches = 0;
    double ub = INFINITY;
    std::vector<int> best_sup(ctx->k, -1);
    std::vector<double> best_coef(ctx->k, 0.0);
    const int k = ctx->k;
    if (resume) {
        // continue a checkpointed search: its open nodes (with their warm starts), incumbent and counts
        ub = resume->ub;
        best_sup = resume->sup;
        best_coef = resume->coef;
        n_nodes = resume->nodes;
        n_batches = resume->batches;
        next_id = resume->next_id;
        for (const SavedNode& sn : resume->open) open.push(new Open{sn.lb, sn.id, sn.J0, sn.J1, -1, sn.wb});
    } else {
        open.push(new Open{-INFINITY, next_id++, {}, {}, -1, {}});
    }
    const int64_t batch0 = n_batches;
    ctx->saved = SavedSolve{};
    std::vector<double> warm_host;
    std::vector<int> in_ptr, in_idx, out_ptr, out_idx, wslot;
    std::vector<double> lb(batch), ubc(batch), bre((size_t)batch * k);
    std::vector<int> sup((size_t)batch * k), bj(batch);
    std::vector<Open*> cur;
    // the pruning threshold: the incumbent, or the Rashomon threshold tau
    auto tau = [&]() {
        double t = isfinite(ub) ? (1.0 + rs->eps) * ub : INFINITY;
        if (rs->cap > 0) t = std::min(t, rs->pool->nth_best(rs->cap));
        return t;
    };
    auto pruned = [&](double lbv) {
        if (!rs) return lbv >= ub - delta_of(ctx, ub);
        const double t = tau();
        return lbv > t + delta_of(ctx, t);
    };
    try {
        while (!open.empty()) {
            if (time_limit_s > 0 && elapsed() > time_limit_s) break;
            if (ctx->solve_max_batches > 0 && n_batches - batch0 >= ctx->solve_max_batches) break;
            if (cancel && cancel->load(std::memory_order_relaxed)) {
                out.cancelled = true;
                break;
            }
            cur.clear();
            Nvtx range("bnb batch");
            const double dl = delta_of(ctx, ub);
            while (!open.empty() && (int)cur.size() < batch) {
                Open* o = open.top();
                open.pop();
                if (pruned(o->lb)) {
                    release(o->slot);
                    delete o;
                    continue;
                }
                cur.push_back(o);
            }
            if (cur.empty()) break;
            const int m = (int)cur.size();
            in_ptr.assign(1, 0);
            out_ptr.assign(1, 0);
            in_idx.clear();
            out_idx.clear();
            wslot.resize(m);
            bool host_warm = false;
            for (int b = 0; b < m; ++b) {
                in_idx.insert(in_idx.end(), cur[b]->J1.begin(), cur[b]->J1.end());
                out_idx.insert(out_idx.end(), cur[b]->J0.begin(), cur[b]->J0.end());
                in_ptr.push_back((int)in_idx.size());
                out_ptr.push_back((int)out_idx.size());
                wslot[b] = cur[b]->slot;
                host_warm |= cur[b]->slot < 0 && !cur[b]->wb.empty();
            }
            if (host_warm) {                    // resumed nodes: warm starts from the checkpoint
                warm_host.assign((size_t)m * ctx->p, 0.0);
                for (int b = 0; b < m; ++b)
                    if (cur[b]->slot < 0 && !cur[b]->wb.empty())
                        std::copy(cur[b]->wb.begin(), cur[b]->wb.end(), warm_host.begin() + (size_t)b * ctx->p);
            }
            push_impl(ctx, m, in_ptr.data(), in_idx.data(), out_ptr.data(), out_idx.data(), wslot.data(),
                      host_warm ? warm_host.data() : nullptr);
            if (rs) {
                const double t = tau();
                ctx->ub_inc = t + 2.0 * delta_of(ctx, t);   // stop iterating once the bound passes tau
            } else {
                ctx->ub_inc = ub;
            }
            evaluate_impl(ctx, iters, check_every);
            evaluate_outputs(ctx, lb.data(), nullptr, ubc.data(), sup.data(), bre.data(), bj.data(), nullptr);
            ctx->evaluated = true;
            n_nodes += m;
            ++n_batches;
            for (int b = 0; b < m; ++b) {
                release(cur[b]->slot);
                if (ubc[b] < ub) {
                    ub = ubc[b];
                    std::copy(sup.begin() + (size_t)b * k, sup.begin() + (size_t)(b + 1) * k, best_sup.begin());
                    std::copy(bre.begin() + (size_t)b * k, bre.begin() + (size_t)(b + 1) * k, best_coef.begin());
                }
            }
            if (rs) {
                // store the supports at or below tau: the node's own fixed-in features in
                // branching order, then the rest of its rounded support ascending
                const double t = tau();
                for (int b = 0; b < m; ++b) {
                    if (!(ubc[b] <= t)) continue;
                    std::vector<int> seq(cur[b]->J1);
                    std::vector<double> cf;
                    for (int j : seq) {
                        for (int r = 0; r < k; ++r)
                            if (sup[(size_t)b * k + r] == j) cf.push_back(bre[(size_t)b * k + r]);
                    }
                    for (int r = 0; r < k; ++r) {
                        const int j = sup[(size_t)b * k + r];
                        if (j < 0 || std::find(cur[b]->J1.begin(), cur[b]->J1.end(), j) != cur[b]->J1.end()) continue;
                        seq.push_back(j);
                        cf.push_back(bre[(size_t)b * k + r]);
                    }
                    rs->pool->insert(seq, cf, ubc[b]);
                }
                rs->pool->filter(tau(), rs->cap);
            }
            const double dl2 = delta_of(ctx, ub);
            std::vector<int> rows, slots;
            for (int b = 0; b < m; ++b) {
                Open* o = cur[b];
                const double lbb = std::max(lb[b], o->lb);
                int j = bj[b];
                if (rs) {
                    const int kb = k - (int)o->J1.size(), pf = ctx->p - (int)o->J0.size() - (int)o->J1.size();
                    if (pruned(lbb) || kb == 0 || pf == 0) {
                        delete o;
                        continue;
                    }
                    if (j < 0) {   // every free coordinate fits: branch on the smallest
                        std::vector<char> fixed(ctx->p, 0);
                        for (int q : o->J0) fixed[q] = 1;
                        for (int q : o->J1) fixed[q] = 1;
                        j = 0;
                        while (fixed[j]) ++j;
                    }
                } else if (lbb >= ub - dl2 || bj[b] < 0 || ubc[b] - lbb <= dl2) {
                    delete o;
                    continue;
                }
                int s = -1;
                if (!free_slots.empty()) {
                    s = free_slots.back();
                    free_slots.pop_back();
                    slot_ref[s] = 2;
                    rows.push_back(b);
                    slots.push_back(s);
                }
                Open* c0 = new Open{lbb, next_id++, o->J0, o->J1, s};
                c0->J0.push_back(j);
                Open* c1 = new Open{lbb, next_id++, o->J0, o->J1, s};
                c1->J1.push_back(j);
                open.push(c0);
                open.push(c1);
                delete o;
            }
            if (!rows.empty()) {
                CK(cudaMemcpyAsync(ctx->d_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice, ctx->st));
                CK(cudaMemcpyAsync(ctx->d_slots, slots.data(), sizeof(int) * slots.size(), cudaMemcpyHostToDevice, ctx->st));
                {
                    Scope sc(ctx, PH_SMALL, 1, 2.0 * (ctx->f64 ? 8 : 4) * (double)rows.size() * ctx->p);
                    pool_store(ctx->st, (int)rows.size(), ctx->p, ctx->f64, ctx->d_rows, ctx->d_slots, ctx->B,
                               ctx->pool);
                    check_launch();
                }
                sync(ctx);
            }
        }
    } catch (...) {
        while (!open.empty()) { delete open.top(); open.pop(); }
        throw;
    }
    // the reduced-precision modes keep an upper bound of each incumbent's
    // objective during the search; report the exact FP64 objective
    if (!ctx->f64 && isfinite(ub)) ub = exact_objective(ctx, best_sup, best_coef, ub);
    if (rs && !ctx->f64 && !rs->pool->leaf.empty()) {
        // the reduced modes store upper estimates of v(S): replace them by the FP64
        // objective of each record's coefficients, then filter at the final tau
        kglm_pool& q = *rs->pool;
        std::vector<double> ex(q.leaf.size());
        for (size_t r = 0; r < q.leaf.size(); ++r) {
            const std::vector<int> Sv = q.path(q.leaf[r]);
            const int ks = (int)Sv.size();
            ex[r] = q.obj[r];
            if (ks == 0) continue;
            CK(cudaMemcpyAsync(ctx->d_rows, Sv.data(), sizeof(int) * ks, cudaMemcpyHostToDevice, ctx->st));
            CK(cudaMemcpyAsync(ctx->beta_re, q.coef.data() + q.off[r], sizeof(double) * ks, cudaMemcpyHostToDevice,
                               ctx->st));
            objective64_launch(ctx->st, ctx->Xt64, ctx->y64, ctx->n, ctx->kind, ctx->lam2, ctx->d_rows,
                               ctx->beta_re, ks, ctx->ub);
            check_launch();
            CK(cudaMemcpyAsync(&ex[r], ctx->ub, sizeof(double), cudaMemcpyDeviceToHost, ctx->st));
            sync(ctx);
        }
        q.obj = ex;
        q.filter(tau(), rs->cap);
    }
    out.complete = open.empty() && !out.cancelled;
    if (!open.empty() && !rs) {
        // stopped early: keep the open queue and the incumbent for kglm_solve_checkpoint
        SavedSolve& sv = ctx->saved;
        sv.valid = true;
        sv.ub = ub;
        sv.sup = best_sup;
        sv.coef = best_coef;
        sv.nodes = n_nodes;
        sv.batches = n_batches;
        sv.next_id = next_id;
        std::vector<Open*> rest;
        while (!open.empty()) { rest.push_back(open.top()); open.pop(); }
        const size_t ws = ctx->f64 ? 8 : 4, pp = (size_t)ctx->p;
        std::vector<unsigned char> row(pp * ws);
        for (Open* o : rest) {
            SavedNode sn{o->lb, o->id, o->J0, o->J1, o->wb};
            if (o->slot >= 0) {
                CK(cudaMemcpyAsync(row.data(), static_cast<const unsigned char*>(ctx->pool) + (size_t)o->slot * pp * ws,
                                   pp * ws, cudaMemcpyDeviceToHost, ctx->st));
                sync(ctx);
                sn.wb.resize(pp);
                for (size_t j = 0; j < pp; ++j)
                    sn.wb[j] = ctx->f64 ? reinterpret_cast<const double*>(row.data())[j]
                                        : (double)reinterpret_cast<const float*>(row.data())[j];
            }
            sv.open.push_back(std::move(sn));
            open.push(o);
        }
    }
    double open_lb = INFINITY;
    while (!open.empty()) {
        open_lb = std::min(open_lb, open.top()->lb);
        delete open.top();
        open.pop();
    }
    const double glb = std::min(open_lb, ub);
    out.opt = ub;
    out.gap = isfinite(ub) ? (ub - glb) / fmax(1.0, fabs(ub)) : INFINITY;
    out.nodes = n_nodes;
    out.batches = n_batches;
    out.support = best_sup;
    out.beta.assign(ctx->p, 0.0);
    for (int r = 0; r < k; ++r)
        if (best_sup[r] >= 0) out.beta[best_sup[r]] = best_coef[r];
}

// ---- autotuner: tile shapes of the tensor-core products and the batch size

// Column tiles of the products: rebuild the B operands' maps (box rows = tile).
void set_tiles(kglm_ctx* c, int bn1, int bn2) {
    const int ob = c->tc_kind == 0;
    if (tc_make_map(&c->mB1, c->Xop, ob, c->n, c->p, c->pK, bn1) ||
        (c->xlo && tc_make_map(&c->mB1lo, c->Xop_lo, ob, c->n, c->p, c->pK, bn1)) ||
        tc_make_map(&c->mB2, c->Xtop, ob, c->p, c->n, c->nK, bn2) ||
        (c->x3 && tc_make_map(&c->mB2lo, c->Xtop_lo, 0, c->p, c->n, c->nK, bn2)))
        throw Fail{KGLM_ECUDA, "cuTensorMapEncodeTiled failed while tuning the tiles"};
    c->bn1 = bn1;
    c->bn2 = bn2;
    destroy_graphs(c);                     // captured launches hold the old maps
}

// Random fixing patterns for timing (|J1| ~ U{0..k}, |J0| ~ U{0..p/2}), from a
// 64-bit linear congruential generator seeded by the caller.
struct TuneNodes {
    std::vector<int> in_ptr{0}, in_idx, out_ptr{0}, out_idx;
};
TuneNodes tune_nodes(int m, int p, int k, uint64_t seed) {
    TuneNodes t;
    uint64_t x = seed * 6364136223846793005ull + 1442695040888963407ull;
    auto next = [&](uint32_t bound) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        return (uint32_t)((x >> 33) % bound);
    };
    std::vector<int> perm(p);
    for (int b = 0; b < m; ++b) {
        for (int j = 0; j < p; ++j) perm[j] = j;
        const int n1 = (int)next((uint32_t)k + 1);
        const int n0 = std::min((int)next((uint32_t)(p / 2) + 1), p - n1);
        for (int i = 0; i < n1 + n0; ++i) std::swap(perm[i], perm[i + (int)next((uint32_t)(p - i))]);
        std::sort(perm.begin(), perm.begin() + n1);
        std::sort(perm.begin() + n1, perm.begin() + n1 + n0);
        t.in_idx.insert(t.in_idx.end(), perm.begin(), perm.begin() + n1);
        t.out_idx.insert(t.out_idx.end(), perm.begin() + n1, perm.begin() + n1 + n0);
        t.in_ptr.push_back((int)t.in_idx.size());
        t.out_ptr.push_back((int)t.out_idx.size());
    }
    return t;
}

// Device milliseconds of one node evaluation (iters iterations, certificate,
// re-optimization) of the first m tuning nodes: best of `reps` runs after one
// untimed run (graph capture).
double time_eval(kglm_ctx* c, const TuneNodes& t, int m, int iters, int reps) {
    std::vector<int> ip(t.in_ptr.begin(), t.in_ptr.begin() + m + 1), op(t.out_ptr.begin(), t.out_ptr.begin() + m + 1);
    push_impl(c, m, ip.data(), t.in_idx.data(), op.data(), t.out_idx.data(), nullptr, nullptr);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = INFINITY;
    try {
        for (int r = 0; r <= reps; ++r) {
            c->ub_inc = INFINITY;
            CK(cudaEventRecord(e0, c->st));
            evaluate_impl(c, iters, 0);
            CK(cudaEventRecord(e1, c->st));
            CK(cudaEventSynchronize(e1));
            finish_tc_check(c);
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) best = std::min(best, (double)ms);
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

void autotune_impl(kglm_ctx* c, int iters, uint64_t seed, kglm_tune* out) {
    REQ(iters >= 1, "iters must be >= 1");
    const int mc = c->mcap;
    const TuneNodes t = tune_nodes(mc, c->p, c->k, seed);
    int timed = 0;
    kglm_tune r{};
    if (c->tc) {
        // coordinate descent at the full batch: the link product's column tile,
        // then the gradient product's column tile and split cap
        const int cap = c->gsplit_max;
        // link tile: every width from 32 columns (multiples of 16) up to the sample count
        std::vector<int> t1;
        for (int bn = 32; bn <= tc_tile_cols(c->n); bn += 16) t1.push_back(bn);
        if (t1.empty()) t1.push_back(tc_tile_cols(c->n));
        std::vector<int> t2{tc_tile_cols(c->p)};
        if (c->p > 128) t2.push_back(128);
        if (c->p > 64) t2.push_back(64);
        double best = INFINITY;
        int b1 = c->bn1, b2 = c->bn2, bs = cap;
        // BF16: CTA pairs on or off at the starting tiles first, so that the tiles
        // are tuned for the kind of launch that will run them (checked again below)
        if (c->tc_kind == 0 && !c->x3) {
            double tp[2] = {INFINITY, INFINITY};
            for (int on = 0; on <= 1; ++on) {
                c->pair = on != 0;
                destroy_graphs(c);
                tp[on] = time_eval(c, t, mc, iters, 3);
                ++timed;
            }
            c->pair = tp[1] < tp[0];
            destroy_graphs(c);
        }
        for (int bn : t1) {
            set_tiles(c, bn, b2);
            const double ms = time_eval(c, t, mc, iters, 3);
            ++timed;
            if (ms < best) { best = ms; b1 = bn; }
        }
        for (int bn : t2)
            for (int sc = 1; sc <= cap; sc *= 2) {
                set_tiles(c, b1, bn);
                c->gsplit_max = sc;
                const double ms = time_eval(c, t, mc, iters, 3);
                ++timed;
                if (ms < best) { best = ms; b2 = bn; bs = sc; }
            }
        // the other gradient widths (multiples of 16 from 64) at the best split cap
        for (int bn = 64; bn <= tc_tile_cols(c->p); bn += 16) {
            if (std::find(t2.begin(), t2.end(), bn) != t2.end()) continue;
            set_tiles(c, b1, bn);
            c->gsplit_max = bs;
            const double ms = time_eval(c, t, mc, iters, 3);
            ++timed;
            if (ms < best) { best = ms; b2 = bn; }
        }
        set_tiles(c, b1, b2);
        c->gsplit_max = bs;
        // programmatic dependent launch on or off at the chosen tiles
        bool bp = c->pdl;
        for (int on = 0; on <= 1; ++on) {
            if ((bool)on == c->pdl) continue;
            const bool keep = c->pdl;
            c->pdl = on != 0;
            destroy_graphs(c);
            const double ms = time_eval(c, t, mc, iters, 3);
            ++timed;
            if (ms < best) { best = ms; bp = c->pdl; }
            c->pdl = keep;
        }
        c->pdl = bp;
        destroy_graphs(c);
        // BF16: the products as CTA pairs (256-row tiles, half of B in each CTA), or one CTA per tile
        if (c->tc_kind == 0 && !c->x3) {
            bool bpair = c->pair;
            const bool keep = c->pair;
            c->pair = !keep;
            destroy_graphs(c);
            const double ms = time_eval(c, t, mc, iters, 3);
            ++timed;
            if (ms < best) { best = ms; bpair = c->pair; }
            c->pair = bpair;
            destroy_graphs(c);
        }
        // sub-batches of the iteration loop side by side on forked streams
        int bsub = c->nsub;
        for (int ns : {1, 2, 4}) {
            if (ns == c->nsub || mc < 128 * ns) continue;
            const int keep = c->nsub;
            c->nsub = ns;
            const double ms = time_eval(c, t, mc, iters, 3);
            ++timed;
            if (ms < best) { best = ms; bsub = ns; }
            c->nsub = keep;
        }
        c->nsub = bsub;
        r.link_tile_cols = b1;
        r.grad_tile_cols = b2;
        r.grad_split_cap = bs;
    }
    r.pdl = c->pdl ? 1 : 0;
    r.pair = c->pair ? 1 : -1;
    r.sub_batches = c->nsub;
    // threads per node of the prox (FP32 working type, p > 512)
    if (!c->f64) {
        int opts[4];
        const int no = prox_thread_options(c->p, opts);
        if (no > 1) {
            double best = INFINITY;
            int bt = c->prox_threads;
            for (int q = 0; q < no; ++q) {
                c->prox_threads = opts[q];
                destroy_graphs(c);
                const double ms = time_eval(c, t, mc, iters, 3);
                ++timed;
                if (ms < best) { best = ms; bt = opts[q]; }
            }
            c->prox_threads = bt;
            destroy_graphs(c);
        }
    }
    r.prox_threads = c->prox_threads;
    // batch size: node bounds per second at each power of two; the smallest
    // within 5% of the best (larger batches evaluate nodes the search may
    // never need, Fig. 3's plateau)
    std::vector<std::pair<int, double>> rates;
    for (int m = std::min(64, mc); m <= mc; m *= 2) {
        const double ms = time_eval(c, t, m, iters, 1);
        ++timed;
        rates.push_back({m, m / (ms * 1e-3)});
        if (m == mc) break;
        if (m * 2 > mc && m != mc) {
            const double ms2 = time_eval(c, t, mc, iters, 1);
            ++timed;
            rates.push_back({mc, mc / (ms2 * 1e-3)});
            break;
        }
    }
    double top = 0.0;
    for (auto& q : rates) top = std::max(top, q.second);
    for (auto& q : rates)
        if (q.second >= 0.95 * top) { r.batch = q.first; r.nodes_per_s = q.second; break; }
    r.best_nodes_per_s = top;
    r.timed = timed;
    c->tuned_batch = r.batch;
    c->pushed = c->evaluated = false;
    if (out) *out = r;
}

}  // namespace

namespace kglm {

size_t device_footprint(const kglm_desc& d) { return footprint(d); }

struct ServeSolve {
    DevSolve d;
};

kglm_status serve_begin(kglm_ctx* c, int batch, ServeSolve** out) {
    if (!c || !out) return KGLM_EINVAL;
    *out = nullptr;
    return guarded(c, [&] {
        REQ(c->dq_on, "the context has no device queue (created with open_cap = 0)");
        REQ(batch >= 1 && batch <= c->mcap, "batch must be in [1, max_batch]");
        ServeSolve* s = new ServeSolve();
        s->d.c = c;
        s->d.batch = batch;
        try {
            s->d.begin();
        } catch (...) {
            delete s;
            throw;
        }
        *out = s;
    });
}

kglm_status serve_select(ServeSolve* s, int* m) {
    *m = 0;
    return guarded(s->d.c, [&] { *m = s->d.select(); });
}

kglm_status serve_evaluate(kglm_ctx* const* cs, int count, int iters, int check_every, int64_t* shared) {
    if (count <= 0) return KGLM_OK;
    return guarded(cs[0], [&] {
        REQ(iters >= 1 && check_every >= 0, "iters must be >= 1 and check_every >= 0");
        evaluate_group(std::vector<kglm_ctx*>(cs, cs + count), iters, check_every, shared);
    });
}

kglm_status serve_update(ServeSolve* s) { return guarded(s->d.c, [&] { s->d.update(); }); }

kglm_status serve_finish(ServeSolve* s, bool stopped, SolveResult* r) {
    SolveOut o;
    const kglm_status st = guarded(s->d.c, [&] { s->d.finish(o, stopped); });
    r->opt = o.opt;
    r->gap = o.gap;
    r->support = o.support;
    r->nodes = o.nodes;
    r->batches = o.batches;
    r->cancelled = stopped;
    delete s;
    return st;
}

void serve_free(ServeSolve* s) { delete s; }

kglm_status solve_cancellable(kglm_ctx* ctx, int batch, int iters, int check_every, double time_limit_s,
                              const std::atomic<int>* cancel, SolveResult* r) {
    if (!ctx || !r) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        SolveOut o;
        solve_impl(ctx, batch, iters, check_every, time_limit_s, cancel, o);
        r->opt = o.opt;
        r->gap = o.gap;
        r->support = o.support;
        r->nodes = o.nodes;
        r->batches = o.batches;
        r->cancelled = o.cancelled;
    });
}

}  // namespace kglm

extern "C" {

const char* kglm_version(void) { return "kglm 0.1 sm_103a"; }

// Message of a failed kglm_create (the context does not survive it).
static thread_local std::string g_create_err = "no error";

const char* kglm_last_error(const kglm_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

void kglm_destroy(kglm_ctx* ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    destroy_graphs(ctx);
    for (auto& r : ctx->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
    for (void* p : ctx->allocs) cudaFreeAsync(p, ctx->st);
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    cudaGetLastError();
    for (int q = 0; q < kglm_ctx::kMaxSub; ++q) {
        if (ctx->sub_st[q]) cudaStreamDestroy(ctx->sub_st[q]);
        if (ctx->ev_join[q]) cudaEventDestroy(ctx->ev_join[q]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->own_stream && ctx->st) cudaStreamDestroy(ctx->st);
    delete ctx;
}

kglm_status kglm_create(const kglm_desc* desc, const double* X, const double* y, void* stream, kglm_ctx** out) {
    if (!out) return KGLM_EINVAL;
    *out = nullptr;
    if (!desc || !X || !y) return KGLM_EINVAL;
    kglm_ctx* c = new (std::nothrow) kglm_ctx();
    if (!c) return KGLM_ENOMEM;
    kglm_status st = guarded(c, [&] {
        const kglm_desc& d = *desc;
        REQ(d.n > 0 && d.p > 0 && d.n < (1LL << 31) && d.p < (1LL << 31), "n and p must be positive");
        REQ(d.k >= 1 && d.k <= KGLM_MAX_K && d.k <= d.p, "k must be in [1, min(p, KGLM_MAX_K)]");
        REQ(d.lambda2 > 0 && isfinite(d.lambda2), "lambda2 must be positive");
        REQ(d.M > 0 && isfinite(d.M), "M must be positive");
        REQ(d.loss == KGLM_LSQ || d.loss == KGLM_LOGISTIC, "unknown loss");
        REQ(d.prec == KGLM_FP64 || d.prec == KGLM_FP32 || d.prec == KGLM_BF16 || d.prec == KGLM_TF32 ||
                d.prec == KGLM_TF32X3,
            "unknown precision");
        REQ(d.max_batch >= 1, "max_batch must be >= 1");
        REQ(d.open_cap >= 0 && d.open_cap <= (int64_t)1 << 28, "open_cap must be in [0, 2^28]");
        REQ(d.p <= (d.prec == KGLM_FP64 ? 4096 : 8192), "p above the prox kernel limit for this precision");
        c->d = d;
        c->n = (int)d.n; c->p = (int)d.p; c->k = d.k; c->kind = d.loss; c->prec = d.prec;
        c->f64 = d.prec == KGLM_FP64;
        c->tc = d.prec == KGLM_BF16 || d.prec == KGLM_TF32 || d.prec == KGLM_TF32X3;
        c->tc_kind = d.prec == KGLM_BF16 ? 0 : 1;
        c->x3 = d.prec == KGLM_TF32X3;
        c->xlo = d.prec == KGLM_TF32 || d.prec == KGLM_TF32X3;
        c->W = (c->p + 31) / 32;
        c->lam2 = d.lambda2; c->M = d.M;
        c->gap_tol = d.gap_tol > 0 ? d.gap_tol : 1e-6;
        const size_t n = c->n, p = c->p;
        for (size_t t = 0; t < n * p; ++t) {
            if (!isfinite(X[t])) throw Fail{KGLM_ENUMERIC, "X has a non-finite entry"};
            c->data_sum += X[t];
        }
        for (size_t i = 0; i < n; ++i) c->data_sum += y[i];
        for (size_t i = 0; i < n; ++i) {
            if (!isfinite(y[i])) throw Fail{KGLM_ENUMERIC, "y has a non-finite entry"};
            if (d.loss == KGLM_LOGISTIC) REQ(y[i] == 1.0 || y[i] == -1.0, "logistic labels must be -1 or +1");
        }
        if (stream) {
            c->st = (cudaStream_t)stream;
        } else {
            CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        // instance: FP64 X, X^T, y (+ FP32 working copies), Gram and X^T y for re-optimization
        c->X64 = dalloc_t<double>(c, n * p);
        c->Xt64 = dalloc_t<double>(c, n * p);
        c->y64 = dalloc_t<double>(c, n);
        CK(cudaMemcpyAsync(c->X64, X, sizeof(double) * n * p, cudaMemcpyHostToDevice, c->st));
        transpose_f64(c->st, c->X64, c->Xt64, n, p);        // X^T on the device (one host copy of X)
        check_launch();
        CK(cudaMemcpyAsync(c->y64, y, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
        c->yty = 0.0;
        for (size_t i = 0; i < (size_t)n; ++i) c->yty += y[i] * y[i];
        if (!c->f64) {
            c->X32 = dalloc_t<float>(c, n * p);
            c->Xt32 = dalloc_t<float>(c, n * p);
            c->y32 = dalloc_t<float>(c, n);
            c->ylo32 = dalloc_t<float>(c, n);
            convert_f64_to_f32(c->st, c->X64, c->X32, n * p);
            convert_f64_to_f32(c->st, c->Xt64, c->Xt32, n * p);
            convert_f64_to_f32(c->st, c->y64, c->y32, n);
            check_launch();
            // the low part on the host (y is host data here; fl(y) is the same rounding as on the device)
            c->ylo_host.resize(n);
            for (size_t i = 0; i < (size_t)n; ++i) c->ylo_host[i] = (float)(y[i] - (double)(float)y[i]);
            CK(cudaMemcpyAsync(c->ylo32, c->ylo_host.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->st));
        }
        // split-K scratch: a plan splits only when its tiles do not fill the GPU,
        // so (splits x tiles) stays below two waves plus one wave of tiles
        auto scratch = [&](GemmScratch& g, int is_f64) {
            g.part_bytes = gemm_scratch_bytes(is_f64);
            g.part = dalloc(c, g.part_bytes);
            g.n_counters = gemm_scratch_counters(is_f64);
            g.counters = dalloc_t<int>(c, g.n_counters);
            CK(cudaMemsetAsync(g.counters, 0, sizeof(int) * g.n_counters, c->st));
        };
        scratch(c->gs64, 1);
        if (!c->f64) scratch(c->gs32, 0);
        if (c->tc) {
            // padded operand copies (TMA rows must be 16-byte multiples), their
            // maps, the split-K scratch of the tensor-core products
            const int ob = c->tc_kind == 0;
            const size_t es = ob ? 2 : 4;
            c->pK = (int)((p + 7) / 8 * 8);
            c->nK = (int)((n + 7) / 8 * 8);
            c->Xop = dalloc(c, n * c->pK * es);
            if (c->xlo) c->Xop_lo = dalloc(c, n * c->pK * es);
            c->Xtop = dalloc(c, p * c->nK * es);
            if (c->x3) c->Xtop_lo = dalloc_t<float>(c, p * c->nK);
            convert_pad(c->st, c->X64, (int)n, (int)p, (int)p, c->Xop, c->pK, ob, c->Xop_lo);
            convert_pad(c->st, c->Xt64, (int)p, (int)n, (int)n, c->Xtop, c->nK, ob, c->Xtop_lo);
            check_launch();
            const size_t mc = (size_t)d.max_batch;
            c->Vop = dalloc(c, mc * c->pK * es);
            c->Rop = dalloc(c, mc * c->nK * es);
            CK(cudaMemsetAsync(c->Vop, 0, mc * c->pK * es, c->st));
            CK(cudaMemsetAsync(c->Rop, 0, mc * c->nK * es, c->st));
            if (c->x3) {
                c->Vop_lo = dalloc_t<float>(c, mc * c->pK);
                c->Rop_lo = dalloc_t<float>(c, mc * c->nK);
                CK(cudaMemsetAsync(c->Vop_lo, 0, mc * c->pK * 4, c->st));
                CK(cudaMemsetAsync(c->Rop_lo, 0, mc * c->nK * 4, c->st));
            }
            c->Bop = dalloc_t<float>(c, mc * c->pK);
            c->Bop_lo = dalloc_t<float>(c, mc * c->pK);
            if (c->tc_kind == 0) {
                c->Xc = dalloc_t<float>(c, n * c->pK);
                c->Xc_lo = dalloc_t<float>(c, n * c->pK);
                convert_pad(c->st, c->X64, (int)n, (int)p, (int)p, c->Xc, c->pK, 0, c->Xc_lo);
                check_launch();
                c->bnc = tc_tile_cols_wide((int)n);
                if (tc_make_map(&c->mXc, c->Xc, 0, (int)n, (int)p, c->pK, c->bnc) ||
                    tc_make_map(&c->mXclo, c->Xc_lo, 0, (int)n, (int)p, c->pK, c->bnc))
                    throw Fail{KGLM_ECUDA, "cuTensorMapEncodeTiled failed for the certificate's X"};
            }
            if (tc_make_map(&c->mAb, c->Bop, 0, (int)mc, (int)p, c->pK, 128) ||
                tc_make_map(&c->mAblo, c->Bop_lo, 0, (int)mc, (int)p, c->pK, 128))
                throw Fail{KGLM_ECUDA, "cuTensorMapEncodeTiled failed for the certificate's beta"};
            c->bn1 = tc_tile_cols_wide((int)n);
            c->bn2 = tc_tile_cols((int)p);
            if (tc_make_map(&c->mA1, c->Vop, ob, (int)mc, (int)p, c->pK, 128) ||
                tc_make_map(&c->mB1, c->Xop, ob, (int)n, (int)p, c->pK, c->bn1) ||
                (c->xlo && tc_make_map(&c->mB1lo, c->Xop_lo, ob, (int)n, (int)p, c->pK, c->bn1)) ||
                tc_make_map(&c->mA2, c->Rop, ob, (int)mc, (int)n, c->nK, 128) ||
                tc_make_map(&c->mB2, c->Xtop, ob, (int)p, (int)n, c->nK, c->bn2))
                throw Fail{KGLM_ECUDA, "cuTensorMapEncodeTiled failed for an operand"};
            if (c->x3 && (tc_make_map(&c->mA1lo, c->Vop_lo, 0, (int)mc, (int)p, c->pK, 128) ||
                          tc_make_map(&c->mA2lo, c->Rop_lo, 0, (int)mc, (int)n, c->nK, 128) ||
                          tc_make_map(&c->mB2lo, c->Xtop_lo, 0, (int)p, (int)n, c->nK, c->bn2)))
                throw Fail{KGLM_ECUDA, "cuTensorMapEncodeTiled failed for a low-part operand"};
            if (tc_prepare() != 0) throw Fail{KGLM_ECUDA, "tensor-core kernels: shared memory attribute refused"};
            c->gtc.part_bytes = tc_scratch_bytes();
            c->gtc.part = dalloc(c, c->gtc.part_bytes);
            c->gtc.n_counters = tc_scratch_counters();
            c->gtc.counters = dalloc_t<int>(c, c->gtc.n_counters);
            CK(cudaMemsetAsync(c->gtc.counters, 0, sizeof(int) * c->gtc.n_counters, c->st));
            c->gsplit_max = tc_split_cap((int)mc, (int)p);
            c->Gpart = dalloc_t<float>(c, (size_t)c->gsplit_max * mc * p);
            c->d_tcerr = dalloc_t<int>(c, 1);
            CK(cudaMemsetAsync(c->d_tcerr, 0, sizeof(int), c->st));
            for (int q = 0; q < kglm_ctx::kMaxSub; ++q) {
                CK(cudaStreamCreateWithFlags(&c->sub_st[q], cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&c->ev_join[q], cudaEventDisableTiming));
            }
            CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        }
        c->gram = dalloc_t<double>(c, p * p);
        c->Xty = dalloc_t<double>(c, p);
        gemm_nt_f64(c->st, (int)p, (int)p, (int)n, c->Xt64, (int)n, c->Xt64, (int)n, c->gram, (int)p, &c->gs64);
        gemm_nt_f64(c->st, (int)p, 1, (int)n, c->Xt64, (int)n, c->y64, (int)n, c->Xty, 1, &c->gs64);
        check_launch();
        if (d.lipschitz > 0) {
            c->L = d.lipschitz;
        } else {
            const double lam = gram_lambda_max(c) * (1.0 + 1e-6);
            c->L = d.loss == KGLM_LSQ ? 2.0 * lam : 0.25 * lam;
        }
        c->eta = 1.0 / c->L;
        c->c = 2.0 * c->eta * c->lam2;
        // node batch
        const size_t mc = (size_t)d.max_batch;
        c->mcap = d.max_batch;
        c->pin_m = (mc + 7) / 8 * 8;
        if (cudaHostAlloc((void**)&c->pin, c->pin_bytes(), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            c->pin = nullptr;
            throw Fail{KGLM_ENOMEM, "pinned host staging of the batch results refused"};
        }
        const size_t ws = c->f64 ? sizeof(double) : sizeof(float);
        c->in_mask = dalloc_t<uint32_t>(c, mc * c->W);
        c->out_mask = dalloc_t<uint32_t>(c, mc * c->W);
        c->kbar = dalloc_t<int>(c, mc);
        c->pf = dalloc_t<int>(c, mc);
        c->B = dalloc(c, mc * p * ws);
        c->V = dalloc(c, mc * p * ws);
        c->G = dalloc(c, mc * p * ws);
        c->R = dalloc(c, mc * n * std::max(ws, sizeof(float)));
        c->tmom = dalloc_t<double>(c, mc);
        c->active = dalloc_t<int>(c, mc);
        c->phint = dalloc_t<float>(c, 2 * mc);
        c->iters_done = dalloc_t<int>(c, mc);
        c->zeta = dalloc_t<double>(c, mc * n);
        c->Q = dalloc_t<double>(c, mc * p);
        c->sum_loss = dalloc_t<double>(c, mc);
        c->sum_conj = dalloc_t<double>(c, mc);
        c->lb_now = dalloc_t<double>(c, mc);
        c->primal_now = dalloc_t<double>(c, mc);
        c->lb_best = dalloc_t<double>(c, mc);
        c->primal_last = dalloc_t<double>(c, mc);
        c->ub = dalloc_t<double>(c, mc);
        c->beta_re = dalloc_t<double>(c, mc * c->k);
        c->support = dalloc_t<int>(c, mc * c->k);
        c->jstar = dalloc_t<int>(c, mc);
        c->pruned = dalloc_t<uint8_t>(c, mc);
        c->d_in_ptr = dalloc_t<int>(c, mc + 1);
        c->d_out_ptr = dalloc_t<int>(c, mc + 1);
        c->d_slot = dalloc_t<int>(c, mc);
        c->d_rows = dalloc_t<int>(c, std::max(mc, (size_t)c->k));   // also a support's indices
        c->d_slots = dalloc_t<int>(c, mc);
        c->d_err = dalloc_t<int>(c, 1);
        c->pool_slots = d.pool_slots > 0 ? d.pool_slots : 4 * d.max_batch;
        c->pool = dalloc(c, (size_t)c->pool_slots * p * ws);
        c->d_in_idx = dalloc_t<int>(c, mc * c->k);
        c->d_out_idx = dalloc_t<int>(c, mc * p);
        if (d.open_cap > 0) {
            // the device-resident open-node queue: two pool buffers, the children of a
            // batch, per-batch bookkeeping, slot counts, the incumbent and the state
            DevQueue& q = c->dq;
            q.cap = (int)d.open_cap; q.W = c->W; q.p = c->p; q.k = c->k; q.nslots = c->pool_slots;
            const size_t cap = (size_t)d.open_cap, W2 = 2 * (size_t)c->W, m2 = 2 * mc;
            for (int b = 0; b < 2; ++b) {
                q.lb[b] = dalloc_t<double>(c, cap);
                q.id[b] = dalloc_t<long long>(c, cap);
                q.slot[b] = dalloc_t<int>(c, cap);
                q.mask[b] = dalloc_t<uint32_t>(c, cap * W2);
            }
            q.clb = dalloc_t<double>(c, m2);
            q.cid = dalloc_t<long long>(c, m2);
            q.cslot = dalloc_t<int>(c, m2);
            q.cmask = dalloc_t<uint32_t>(c, m2 * W2);
            q.cperm = dalloc_t<int>(c, m2);
            q.lbp = dalloc_t<double>(c, mc);
            q.bslot = dalloc_t<int>(c, mc);
            q.brank = dalloc_t<int>(c, mc);
            q.cslot_b = dalloc_t<int>(c, mc);
            q.sref = dalloc_t<int>(c, (size_t)c->pool_slots);
            q.sfree = dalloc_t<int>(c, (size_t)c->pool_slots);
            q.best_sup = dalloc_t<int>(c, (size_t)c->k);
            q.best_coef = dalloc_t<double>(c, (size_t)c->k);
            q.st = static_cast<DqState*>(dalloc(c, sizeof(DqState)));
            c->dq_on = true;
        }
        // reduced-precision modes: digits of X for the exact certificate product
        // (6-bit digits, 7 per value), when the jobs and the HBM budget allow
        if (!c->f64 && exact_plan((int)n, 6, 7, &c->xplan)) {
            const ExactPlan& x = c->xplan;
            const size_t K2 = (size_t)x.nd * x.npad;
            const size_t need = 2 * K2 * (p + mc) + 8 * (p + mc) + 4 * (size_t)x.njobs * mc * p + 64;
            if (c->d.hbm_budget <= 0 || (int64_t)(c->bytes + need) <= c->d.hbm_budget) {
                c->DX = dalloc_t<__nv_bfloat16>(c, p * K2);
                c->xsig = dalloc_t<double>(c, p);
                exact_digits(c->st, c->Xt64, (int)p, (int)n, n, x.npad, x.nd, x.beta, 0, c->DX, c->xsig);
                check_launch();
                c->DZ = dalloc_t<__nv_bfloat16>(c, mc * K2);
                CK(cudaMemsetAsync(c->DZ, 0, sizeof(__nv_bfloat16) * mc * K2, c->st));
                c->ztau = dalloc_t<double>(c, mc);
                c->qs_slices = (size_t)x.njobs;
                c->Qs = dalloc_t<float>(c, c->qs_slices * mc * p);
                c->bnx = tc_tile_cols((int)p);
                if (tc_make_map(&c->mBx, c->DX, 1, (int)p, (int)K2, (int)K2, c->bnx) ||
                    tc_make_map(&c->mAz, c->DZ, 1, (int)mc, (int)K2, (int)K2, 128))
                    throw Fail{KGLM_ECUDA, "cuTensorMapEncodeTiled failed for the certificate digits"};
                if (tc_prepare() != 0) throw Fail{KGLM_ECUDA, "tensor-core kernels: shared memory attribute refused"};
                if (!c->d_tcerr) {
                    c->d_tcerr = dalloc_t<int>(c, 1);
                    CK(cudaMemsetAsync(c->d_tcerr, 0, sizeof(int), c->st));
                }
                c->cexact = true;
            }
        }
        sync(c);
    });
    if (st != KGLM_OK) {
        g_create_err = c->err;                         // kglm_last_error(NULL) returns it
        kglm_destroy(c);
        return st;
    }
    *out = c;
    return KGLM_OK;
}

kglm_status kglm_push_nodes(kglm_ctx* ctx, int32_t m, const int32_t* in_ptr, const int32_t* in_idx,
                            const int32_t* out_ptr, const int32_t* out_idx, const int32_t* warm_slot,
                            const double* warm_B) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] { push_impl(ctx, m, in_ptr, in_idx, out_ptr, out_idx, warm_slot, warm_B); });
}

kglm_status kglm_push_nodes_dev(kglm_ctx* ctx, int32_t m, const int32_t* in_ptr, const int32_t* in_idx,
                                const int32_t* out_ptr, const int32_t* out_idx, int32_t nnz_in, int32_t nnz_out,
                                const int32_t* warm_slot) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] { push_dev_impl(ctx, m, in_ptr, in_idx, out_ptr, out_idx, nnz_in, nnz_out, warm_slot); });
}

kglm_status kglm_xtr(kglm_ctx* ctx, int32_t m, const void* R, void* G) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(m >= 1 && m <= ctx->mcap, "m must be in [1, max_batch]");
        REQ(R && G, "R and G are required");
        Scope sc(ctx, PH_GEMM_GRAD, 1, 2.0 * ctx->n * (double)m * ctx->p);
        if (ctx->tc) {
            convert_pad_f32(ctx->st, (const float*)R, m, ctx->n, ctx->Rop, ctx->nK, ctx->tc_kind == 0, ctx->Rop_lo);
            check_launch();
            TcGemm g{};
            g.kind = ctx->tc_kind; g.M = m; g.N = ctx->p; g.K = ctx->n; g.bn = ctx->bn2;
            g.epi = TC_EPI_STORE_F32; g.out = G; g.ldo = ctx->p; g.err = ctx->d_tcerr;
            if (ctx->x3) g.A2 = &ctx->mA2lo;
            if (tc_gemm(ctx->st, ctx->mA2, ctx->mB2, ctx->x3 ? &ctx->mB2lo : nullptr, g, &ctx->gtc) != 0)
                throw Fail{KGLM_ECUDA, "tensor-core product setup failed"};
            check_launch();
            sync(ctx);
            check_tc_error(ctx);
            return;
        }
        if (ctx->f64)
            gemm_nt_f64(ctx->st, m, ctx->p, ctx->n, (const double*)R, ctx->n, ctx->Xt64, ctx->n, (double*)G, ctx->p,
                        &ctx->gs64);
        else
            gemm_nt_f32(ctx->st, m, ctx->p, ctx->n, (const float*)R, ctx->n, ctx->Xt32, ctx->n, (float*)G, ctx->p,
                        &ctx->gs32);
        check_launch();
        sync(ctx);
    });
}

kglm_status kglm_xtz(kglm_ctx* ctx, int32_t m, const double* Z, double* Q, double* Qerr) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(m >= 1 && m <= ctx->mcap, "m must be in [1, max_batch]");
        REQ(Z && Q, "Z and Q are required");
        kglm_ctx* c = ctx;
        const size_t mp = (size_t)m * c->p;
        CK(cudaMemcpyAsync(c->zeta, Z, sizeof(double) * m * (size_t)c->n, cudaMemcpyHostToDevice, c->st));
        CertArgs a{};
        {
            Scope sc(c, PH_CERT_Q, c->cexact ? 2 : 1, 2.0 * c->n * (double)mp);
            xtzeta(c, m, a);
            check_launch();
        }
        if (!c->Qerr) c->Qerr = dalloc_t<double>(c, (size_t)c->mcap * c->p);
        if (a.Qs) {
            exact_combine(c->st, m, c->p, a.Qs, a.nqs, a.qs_stride, a.qs_w, c->xsig, c->ztau, a.ebound, c->Q,
                          c->Qerr);
            check_launch();
        } else {
            CK(cudaMemsetAsync(c->Qerr, 0, sizeof(double) * mp, c->st));
        }
        CK(cudaMemcpyAsync(Q, c->Q, sizeof(double) * mp, cudaMemcpyDeviceToHost, c->st));
        if (Qerr) CK(cudaMemcpyAsync(Qerr, c->Qerr, sizeof(double) * mp, cudaMemcpyDeviceToHost, c->st));
        sync(c);
        if (c->cexact) check_tc_error(c);
    });
}

kglm_status kglm_stats_enable(kglm_ctx* ctx, int32_t enable) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        sync(ctx);
        harvest(ctx);
        for (int i = 0; i < KGLM_NPHASE; ++i) ctx->st_ms[i] = ctx->st_work[i] = 0.0, ctx->st_n[i] = 0;
        ctx->stats_on = enable != 0;
    });
}

kglm_status kglm_stats_read(kglm_ctx* ctx, double* ms, int64_t* launches, double* work) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        sync(ctx);
        harvest(ctx);
        for (int i = 0; i < KGLM_NPHASE; ++i) {
            if (ms) ms[i] = ctx->st_ms[i];
            if (launches) launches[i] = ctx->st_n[i];
            if (work) work[i] = ctx->st_work[i];
        }
    });
}

const char* kglm_phase_name(int32_t phase) {
    return (phase >= 0 && phase < KGLM_NPHASE) ? kPhaseNames[phase] : "unknown";
}

kglm_status kglm_evaluate(kglm_ctx* ctx, int32_t iters, int32_t check_every, double* lb, double* primal,
                          double* ub_cand, int32_t* support, double* beta_re, int32_t* branch_j,
                          int32_t* iters_done) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (!ctx->pushed) throw Fail{KGLM_ESTATE, "no node batch pushed"};
        REQ(iters >= 0 && check_every >= 0, "iters and check_every must be >= 0");
        evaluate_impl(ctx, iters, check_every);
        evaluate_outputs(ctx, lb, primal, ub_cand, support, beta_re, branch_j, iters_done);
        ctx->evaluated = true;
    });
}

kglm_status kglm_read_batch(kglm_ctx* ctx, double* beta, double* zeta) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (!ctx->evaluated) throw Fail{KGLM_ESTATE, "batch not evaluated"};
        const size_t mp = (size_t)ctx->m * ctx->p, mn = (size_t)ctx->m * ctx->n;
        if (beta) {
            if (ctx->f64) {
                CK(cudaMemcpyAsync(beta, ctx->B, sizeof(double) * mp, cudaMemcpyDeviceToHost, ctx->st));
                sync(ctx);
            } else {
                std::vector<float> h(mp);
                CK(cudaMemcpyAsync(h.data(), ctx->B, sizeof(float) * mp, cudaMemcpyDeviceToHost, ctx->st));
                sync(ctx);
                for (size_t t = 0; t < mp; ++t) beta[t] = h[t];
            }
        }
        if (zeta) {
            CK(cudaMemcpyAsync(zeta, ctx->zeta, sizeof(double) * mn, cudaMemcpyDeviceToHost, ctx->st));
            sync(ctx);
        }
    });
}

kglm_status kglm_save_warm(kglm_ctx* ctx, int32_t count, const int32_t* rows, const int32_t* slots) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (!ctx->evaluated) throw Fail{KGLM_ESTATE, "batch not evaluated"};
        REQ(count >= 0 && count <= ctx->m, "count out of range");
        if (count == 0) return;
        REQ(rows && slots, "rows and slots are required");
        for (int t = 0; t < count; ++t) {
            REQ(rows[t] >= 0 && rows[t] < ctx->m, "row out of range");
            REQ(slots[t] >= 0 && slots[t] < ctx->pool_slots, "slot out of range");
        }
        CK(cudaMemcpyAsync(ctx->d_rows, rows, sizeof(int) * count, cudaMemcpyHostToDevice, ctx->st));
        CK(cudaMemcpyAsync(ctx->d_slots, slots, sizeof(int) * count, cudaMemcpyHostToDevice, ctx->st));
        {
            Scope sc(ctx, PH_SMALL, 1, 2.0 * (ctx->f64 ? 8 : 4) * (double)count * ctx->p);
            pool_store(ctx->st, count, ctx->p, ctx->f64, ctx->d_rows, ctx->d_slots, ctx->B, ctx->pool);
            check_launch();
        }
        sync(ctx);
    });
}

kglm_status kglm_set_incumbent(kglm_ctx* ctx, double ub) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(!isnan(ub), "ub is NaN");
        ctx->ub_inc = ub;
    });
}

kglm_status kglm_prune(kglm_ctx* ctx, double ub, uint8_t* pruned, int32_t* n_survivors) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (!ctx->evaluated) throw Fail{KGLM_ESTATE, "batch not evaluated"};
        REQ(!isnan(ub), "ub is NaN");
        const int m = ctx->m;
        const double thr = ub - delta_of(ctx, ub);
        {
            Scope sc(ctx, PH_SMALL, 1, 9.0 * m);
            prune_launch(ctx->st, m, ctx->lb_best, thr, ctx->pruned);
            check_launch();
        }
        std::vector<uint8_t> h(m);
        CK(cudaMemcpyAsync(h.data(), ctx->pruned, m, cudaMemcpyDeviceToHost, ctx->st));
        sync(ctx);
        int surv = 0;
        for (uint8_t v : h) surv += v ? 0 : 1;
        if (pruned) memcpy(pruned, h.data(), m);
        if (n_survivors) *n_survivors = surv;
    });
}

kglm_status kglm_branch(kglm_ctx* ctx, double ub, int32_t* parent, int32_t* branch_j, int32_t* n_parents) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (!ctx->evaluated) throw Fail{KGLM_ESTATE, "batch not evaluated"};
        REQ(!isnan(ub), "ub is NaN");
        const double dl = delta_of(ctx, ub);
        int cnt = 0;
        for (int b = 0; b < ctx->m; ++b) {
            const double lb = ctx->h_lb[b];
            if (lb >= ub - dl) continue;                   // pruned
            if (ctx->h_jstar[b] < 0) continue;             // leaf
            if (ctx->h_ub[b] - lb <= dl) continue;         // fathomed by its own rounding
            if (parent) parent[cnt] = b;
            if (branch_j) branch_j[cnt] = ctx->h_jstar[b];
            ++cnt;
        }
        if (n_parents) *n_parents = cnt;
    });
}

kglm_status kglm_solve(kglm_ctx* ctx, int32_t batch, int32_t iters, int32_t check_every, double time_limit_s,
                       double* opt, int32_t* opt_support, double* opt_beta, double* gap, int64_t* nodes,
                       int64_t* batches) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (batch == 0) {
            if (ctx->tuned_batch == 0) autotune_impl(ctx, std::min(iters, 20), 1, nullptr);
            batch = ctx->tuned_batch;
        }
        SolveOut o;
        solve_impl(ctx, batch, iters, check_every, time_limit_s, nullptr, o);
        if (opt) *opt = o.opt;
        if (gap) *gap = o.gap;
        if (nodes) *nodes = o.nodes;
        if (batches) *batches = o.batches;
        if (opt_support) std::copy(o.support.begin(), o.support.end(), opt_support);
        if (opt_beta) std::copy(o.beta.begin(), o.beta.end(), opt_beta);
    });
}


kglm_status kglm_solve_device(kglm_ctx* ctx, int32_t batch, int32_t iters, int32_t check_every, double time_limit_s,
                              double* opt, int32_t* opt_support, double* opt_beta, double* gap, int64_t* nodes,
                              int64_t* batches) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (batch == 0) {
            if (ctx->tuned_batch == 0) autotune_impl(ctx, std::min(iters, 20), 1, nullptr);
            batch = ctx->tuned_batch;
        }
        SolveOut o;
        solve_dev_impl(ctx, batch, iters, check_every, time_limit_s, nullptr, o);
        if (opt) *opt = o.opt;
        if (gap) *gap = o.gap;
        if (nodes) *nodes = o.nodes;
        if (batches) *batches = o.batches;
        if (opt_support) std::copy(o.support.begin(), o.support.end(), opt_support);
        if (opt_beta) std::copy(o.beta.begin(), o.beta.end(), opt_beta);
    });
}

// ---- checkpoint and resume of an unfinished certified solve
// File: magic "KGLMCKP1", then int64 n, p; int32 k, loss; double lambda2, M, data_sum
// (the instance signature); double ub; int32 sup[k]; double coef[k]; int64 nodes,
// batches, next_id, count; then per open node: double lb; int64 id; int32 n0, n1,
// has_warm; int32 J0[n0], J1[n1]; double warm[p] if has_warm.  Native byte order.
namespace {
constexpr char kCkpMagic[8] = {'K', 'G', 'L', 'M', 'C', 'K', 'P', '1'};

struct File {
    FILE* f = nullptr;
    ~File() { if (f) fclose(f); }
};
void put_raw(FILE* f, const void* v, size_t size, size_t n) {
    if (n && fwrite(v, size, n, f) != n) throw Fail{KGLM_EINVAL, "checkpoint: write failed"};
}
void get_raw(FILE* f, void* v, size_t size, size_t n) {
    if (n && fread(v, size, n, f) != n) throw Fail{KGLM_EINVAL, "checkpoint: truncated or unreadable file"};
}
}  // namespace
#define put(f, v, n) put_raw((f), (v), sizeof(*(v)), (n))
#define get(f, v, n) get_raw((f), (v), sizeof(*(v)), (n))

extern "C" kglm_status kglm_set_solve_limit(kglm_ctx* ctx, int64_t max_batches) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(max_batches >= 0, "max_batches must be >= 0");
        ctx->solve_max_batches = max_batches;
    });
}

extern "C" kglm_status kglm_solve_checkpoint(kglm_ctx* ctx, const char* path) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(path != nullptr, "path is required");
        const SavedSolve& sv = ctx->saved;
        if (!sv.valid) throw Fail{KGLM_ESTATE, "no unfinished solve to checkpoint (the last kglm_solve completed)"};
        File fl;
        fl.f = fopen(path, "wb");
        if (!fl.f) throw Fail{KGLM_EINVAL, std::string("checkpoint: cannot open ") + path + " for writing"};
        FILE* f = fl.f;
        const int64_t np[2] = {ctx->n, ctx->p};
        const int32_t kl[2] = {ctx->k, ctx->kind};
        const double sig[3] = {ctx->lam2, ctx->M, ctx->data_sum};
        put(f, kCkpMagic, 8);
        put(f, np, 2);
        put(f, kl, 2);
        put(f, sig, 3);
        put(f, &sv.ub, 1);
        std::vector<int32_t> sup(sv.sup.begin(), sv.sup.end());
        put(f, sup.data(), sup.size());
        put(f, sv.coef.data(), sv.coef.size());
        const int64_t cnt[4] = {sv.nodes, sv.batches, sv.next_id, (int64_t)sv.open.size()};
        put(f, cnt, 4);
        for (const SavedNode& sn : sv.open) {
            const int32_t hdr[3] = {(int32_t)sn.J0.size(), (int32_t)sn.J1.size(), sn.wb.empty() ? 0 : 1};
            put(f, &sn.lb, 1);
            put(f, &sn.id, 1);
            put(f, hdr, 3);
            std::vector<int32_t> j0(sn.J0.begin(), sn.J0.end()), j1(sn.J1.begin(), sn.J1.end());
            put(f, j0.data(), j0.size());
            put(f, j1.data(), j1.size());
            put(f, sn.wb.data(), sn.wb.size());
        }
        if (fflush(f) != 0) throw Fail{KGLM_EINVAL, "checkpoint: write failed"};
    });
}

extern "C" kglm_status kglm_solve_resume(kglm_ctx* ctx, const char* path, int32_t batch, int32_t iters,
                                         int32_t check_every, double time_limit_s, double* opt,
                                         int32_t* opt_support, double* opt_beta, double* gap, int64_t* nodes,
                                         int64_t* batches) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(path != nullptr, "path is required");
        File fl;
        fl.f = fopen(path, "rb");
        if (!fl.f) throw Fail{KGLM_EINVAL, std::string("checkpoint: cannot open ") + path};
        FILE* f = fl.f;
        char magic[8];
        int64_t np[2];
        int32_t kl[2];
        double sig[3];
        get(f, magic, 8);
        REQ(memcmp(magic, kCkpMagic, 8) == 0, "checkpoint: not a checkpoint file");
        get(f, np, 2);
        get(f, kl, 2);
        get(f, sig, 3);
        REQ(np[0] == ctx->n && np[1] == ctx->p && kl[0] == ctx->k && kl[1] == ctx->kind && sig[0] == ctx->lam2 &&
                sig[1] == ctx->M && sig[2] == ctx->data_sum,
            "checkpoint: written for another instance (n, p, k, loss, lambda2, M or data differ)");
        SavedSolve sv;
        sv.valid = true;
        get(f, &sv.ub, 1);
        std::vector<int32_t> sup(ctx->k);
        get(f, sup.data(), sup.size());
        sv.sup.assign(sup.begin(), sup.end());
        sv.coef.resize(ctx->k);
        get(f, sv.coef.data(), sv.coef.size());
        int64_t cnt[4];
        get(f, cnt, 4);
        REQ(cnt[0] >= 0 && cnt[1] >= 0 && cnt[2] >= 0 && cnt[3] >= 0 && cnt[3] < (int64_t(1) << 40),
            "checkpoint: bad counts");
        sv.nodes = cnt[0];
        sv.batches = cnt[1];
        sv.next_id = cnt[2];
        for (int64_t q = 0; q < cnt[3]; ++q) {
            SavedNode sn;
            int32_t hdr[3];
            get(f, &sn.lb, 1);
            get(f, &sn.id, 1);
            get(f, hdr, 3);
            REQ(hdr[0] >= 0 && hdr[0] <= ctx->p && hdr[1] >= 0 && hdr[1] <= ctx->k && hdr[2] >= 0 && hdr[2] <= 1,
                "checkpoint: bad node record");
            std::vector<int32_t> j0(hdr[0]), j1(hdr[1]);
            get(f, j0.data(), j0.size());
            get(f, j1.data(), j1.size());
            std::vector<char> seen(ctx->p, 0);
            for (int32_t j : j0) { REQ(j >= 0 && j < ctx->p && !seen[j], "checkpoint: bad fixing index"); seen[j] = 1; }
            for (int32_t j : j1) { REQ(j >= 0 && j < ctx->p && !seen[j], "checkpoint: bad fixing index"); seen[j] = 1; }
            sn.J0.assign(j0.begin(), j0.end());
            sn.J1.assign(j1.begin(), j1.end());
            if (hdr[2]) {
                sn.wb.resize(ctx->p);
                get(f, sn.wb.data(), sn.wb.size());
            }
            sv.open.push_back(std::move(sn));
        }
        if (batch == 0) {
            if (ctx->tuned_batch == 0) autotune_impl(ctx, std::min(iters, 20), 1, nullptr);
            batch = ctx->tuned_batch;
        }
        SolveOut o;
        solve_impl(ctx, batch, iters, check_every, time_limit_s, nullptr, o, nullptr, &sv);
        if (opt) *opt = o.opt;
        if (gap) *gap = o.gap;
        if (nodes) *nodes = o.nodes;
        if (batches) *batches = o.batches;
        if (opt_support) std::copy(o.support.begin(), o.support.end(), opt_support);
        if (opt_beta) std::copy(o.beta.begin(), o.beta.end(), opt_beta);
    });
}
#undef put
#undef get

// Checks of kglm_create that need no data (sizes, ranges, enums).
static kglm_status check_desc(const kglm_desc* d) {
    if (!d) return KGLM_EINVAL;
    if (!(d->n > 0 && d->p > 0 && d->n < (1LL << 31) && d->p < (1LL << 31))) return KGLM_EINVAL;
    if (!(d->k >= 1 && d->k <= KGLM_MAX_K && d->k <= d->p)) return KGLM_EINVAL;
    if (!(d->lambda2 > 0 && d->M > 0)) return KGLM_EINVAL;
    if (d->loss != KGLM_LSQ && d->loss != KGLM_LOGISTIC) return KGLM_EINVAL;
    if (d->prec < KGLM_FP64 || d->prec > KGLM_TF32X3) return KGLM_EINVAL;
    if (d->max_batch < 1) return KGLM_EINVAL;
    if (d->p > (d->prec == KGLM_FP64 ? 4096 : 8192)) return KGLM_EINVAL;
    return KGLM_OK;
}

kglm_status kglm_estimate_bytes(const kglm_desc* desc, int64_t* bytes) {
    if (!bytes) return KGLM_EINVAL;
    const kglm_status st = check_desc(desc);
    if (st != KGLM_OK) return st;
    *bytes = (int64_t)footprint(*desc);
    return KGLM_OK;
}

kglm_status kglm_device_bytes(const kglm_ctx* ctx, int64_t* bytes) {
    if (!ctx || !bytes) return KGLM_EINVAL;
    *bytes = (int64_t)ctx->bytes;
    return KGLM_OK;
}

kglm_status kglm_suggest_batch(const kglm_desc* desc, int64_t budget, int32_t cap, int32_t* batch) {
    if (!batch || budget <= 0 || cap < 1) return KGLM_EINVAL;
    kglm_desc d = *desc;
    d.max_batch = 1;
    const kglm_status st = check_desc(&d);
    if (st != KGLM_OK) return st;
    if ((int64_t)footprint(d) > budget) return KGLM_ENOMEM;
    int32_t best = 1;
    for (int64_t m = 2; m <= cap && m <= (1 << 20); m *= 2) {
        d.max_batch = (int32_t)m;
        if ((int64_t)footprint(d) > budget) break;
        best = (int32_t)m;
    }
    *batch = best;
    return KGLM_OK;
}

kglm_status kglm_autotune(kglm_ctx* ctx, int32_t iters, uint64_t seed, kglm_tune* out) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] { autotune_impl(ctx, iters, seed, out); });
}

kglm_status kglm_configure(kglm_ctx* ctx, const kglm_tune* cfg) {
    if (!ctx || !cfg) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        if (cfg->batch != 0) {
            REQ(cfg->batch >= 1 && cfg->batch <= ctx->mcap, "batch must be in [1, max_batch]");
            ctx->tuned_batch = cfg->batch;
        }
        ctx->pdl = cfg->pdl != 0;
        if (cfg->pair != 0) {
            REQ(cfg->pair == 1 || cfg->pair == -1, "pair must be 1 (on), -1 (off) or 0 (keep)");
            if (ctx->pair != (cfg->pair == 1)) destroy_graphs(ctx);
            ctx->pair = cfg->pair == 1;
        }
        if (cfg->prox_threads != 0) {
            int opts[4];
            const int no = prox_thread_options(ctx->p, opts);
            bool ok = false;
            for (int q = 0; q < no; ++q) ok |= opts[q] == cfg->prox_threads;
            REQ(ok && !ctx->f64, "prox_threads is not an option for this p and precision");
            ctx->prox_threads = cfg->prox_threads;
        }
        if (cfg->sub_batches != 0) {
            REQ(cfg->sub_batches >= 1 && cfg->sub_batches <= kglm_ctx::kMaxSub, "sub_batches must be in [1, 4]");
            ctx->nsub = cfg->sub_batches;
        }
        if (ctx->tc) {
            const int b1 = cfg->link_tile_cols ? cfg->link_tile_cols : ctx->bn1;
            const int b2 = cfg->grad_tile_cols ? cfg->grad_tile_cols : ctx->bn2;
            REQ(b1 >= 16 && b1 <= 256 && b1 % 16 == 0 && b2 >= 16 && b2 <= 256 && b2 % 16 == 0,
                "tile columns must be multiples of 16 in [16, 256]");
            if (cfg->grad_split_cap != 0) {
                REQ(cfg->grad_split_cap >= 1 && cfg->grad_split_cap <= tc_split_cap(ctx->mcap, ctx->p),
                    "split cap must be in [1, the allocated slices]");
                ctx->gsplit_max = cfg->grad_split_cap;
            }
            set_tiles(ctx, b1, b2);
        }
        destroy_graphs(ctx);
    });
}

kglm_status kglm_rashomon(kglm_ctx* ctx, double eps, int64_t max_models, int32_t batch, int32_t iters,
                          int32_t check_every, double time_limit_s, kglm_pool* pool, double* opt, int64_t* nodes,
                          int32_t* complete) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(pool != nullptr && pool->p == ctx->p, "pool must be created for this instance's p");
        REQ(eps >= 0.0 && isfinite(eps), "eps must be finite and >= 0");
        REQ(max_models >= 0, "max_models must be >= 0");
        if (batch == 0) {
            if (ctx->tuned_batch == 0) autotune_impl(ctx, std::min(iters, 20), 1, nullptr);
            batch = ctx->tuned_batch;
        }
        *pool = kglm_pool();
        pool->p = ctx->p;
        RashomonOpts rs;
        rs.eps = eps;
        rs.cap = max_models;
        rs.pool = pool;
        SolveOut o;
        solve_impl(ctx, batch, iters, check_every, time_limit_s, nullptr, o, &rs);
        if (opt) *opt = o.opt;
        if (nodes) *nodes = o.nodes;
        if (complete) *complete = o.complete ? 1 : 0;
    });
}

kglm_status kglm_selftest_timeout(kglm_ctx* ctx, int32_t rounds) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
        REQ(rounds >= 1, "rounds must be >= 1");
        int* flag = ctx->d_tcerr ? ctx->d_tcerr : ctx->d_err;
        CK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->st));
        wait_probe(ctx->st, (uint32_t)rounds, flag);
        check_launch();
        int h = 0;
        CK(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        sync(ctx);
        CK(cudaMemsetAsync(flag, 0, sizeof(int), ctx->st));
        sync(ctx);
        if (h & 8) throw Fail{KGLM_ETIMEOUT, "self-test: the bounded device wait ran out and reported it"};
        throw Fail{KGLM_ECUDA, "self-test: the bounded device wait did not report its timeout"};
    });
}

int32_t kglm_checks_enabled(void) { return KGLM_CHECKS ? 1 : 0; }

kglm_status kglm_selftest_checks(kglm_ctx* ctx) {
    if (!ctx) return KGLM_EINVAL;
    return guarded(ctx, [&] {
#if KGLM_CHECKS
        CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->st));
        check_probe(ctx->st, ctx->kbar, ctx->mcap, ctx->d_err);
        check_launch();
        int h = 0;
        CK(cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        sync(ctx);
        CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->st));
        sync(ctx);
        if (h & kChkSelf) throw Fail{KGLM_EINVAL, "self-test: the checked write one past the end was caught and skipped"};
        throw Fail{KGLM_ECUDA, "self-test: the checked write one past the end was not caught"};
#else
        throw Fail{KGLM_ESTATE, "not the bounds-checked build (build with checks=True, load with KGLM_CHECKS=1)"};
#endif
    });
}

}  // extern "C"
