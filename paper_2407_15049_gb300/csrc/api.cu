// C ABI of the LoRADS GB300 library (include/lorads.h): input validation and
// upload, the standalone hot-path entry points, and the device-resident solve
// loop (one captured CUDA graph per L-BFGS iteration + ALM outer step, gated
// by a device control block; the host only polls a status copy).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lorads.h"
#include "admm.h"
#include "common.cuh"
#include "control.h"
#include "kernels.cuh"
#include "launch_decl.h"
#include "prob_host.h"

using namespace lorads;

namespace {

thread_local std::string g_create_error;

enum { PART_DIR = 0, PART_LS, PART_CONS_LS, PART_UPD, PART_CONS, PART_OBJ, PART_YTIL, PART_MISC, NPART };
constexpr int kPartStride = 32;         // doubles per block per region (>= every NQ)

struct SolverState {
    int prec = -1;
    int r = 0, ld = 0;
    Shape sh{1, 1};
    Shape sh_ls{1, 1};                  // lane shape of the line-search SpMM (kernel_variant bit 5)
    size_t esR = 0, esD = 0, esDir = 0;  // element bytes of R, of C D and G, of D and the history
    int rtype = 0;                      // storage of R: 0 double, 1 double-float, 2 float
    void* R = nullptr;
    void* CR = nullptr;
    void* D = nullptr;
    void* CD = nullptr;
    void* G = nullptr;
    void* W = nullptr;
    void* hist = nullptr;
    int64_t slot_stride = 0;
    double* y = nullptr;
    double* ytil = nullptr;
    void* zrow = nullptr;               // A(RR^T)_k - b_k of the diagonal constraint of each row
                                        // (double on the FP64 path, float otherwise)
    dfloat* ydf = nullptr;              // double-float mirror of y (FP32-unit paths), else null
    double* zk = nullptr;               // same for the off-diagonal constraints (by constraint)
    cudaGraphExec_t exec = nullptr;
    bool have_solution = false;
};

// Work arrays of the splitting (ADMM) stage: block iterates U, V (type of R),
// CG vectors r, p, Q (work type), the m-vector w = y - rho (A(X V^T) - b) and
// the stage's device control block; one captured graph per ADMM iteration.
struct AdmmState {
    int rtype = -1, wtype = -1, ld = 0;
    bool borrowed = false;              // U, V, r, p, Q, w live in the solver state's arrays
    size_t esR = 0, esW = 0;
    void* U = nullptr;
    void* V = nullptr;
    void* r = nullptr;
    void* p = nullptr;
    void* Q = nullptr;
    void* om = nullptr;
    AdmmCtrl* ac = nullptr;
    AdmmCtrl* h_ac = nullptr;           // pinned
    cudaGraphExec_t exec = nullptr;
    int64_t graph_nodes = 0;
};

// Per-kernel-family CUDA-event timing of the host-stepped (verbose >= 2) solve.
enum { FAM_DIR = 0, FAM_SPMM_LS, FAM_CONS_LS, FAM_ROOT, FAM_STEP, FAM_CONS_YTIL, FAM_SPMM_A, FAM_UPDATE, FAM_HIST,
       FAM_CONS_YUPD, FAM_SPMM_CR, FAM_OUTER, FAM_GRAD, FAM_MISC, NFAM };
const char* const kFamNames[NFAM] = {"k_dir", "k_spmm_c(CD,ls)", "k_cons(ls)", "k_ctrl_root", "k_step",
                                     "k_cons(ytil)", "k_spmm_a", "k_update(step)", "k_ctrl_hist",
                                     "k_cons(yupd)", "k_spmm_c(CR,obj)", "k_ctrl_outer", "k_update(grad)",
                                     "setup"};
struct Prof {
    static constexpr int kPool = 64;
    cudaEvent_t ev[kPool][2];
    int fam[kPool];
    int used = 0;
    double total_ms[NFAM] = {0};
    int64_t count[NFAM] = {0};
};

}  // namespace

struct lorads_ctx {
    int64_t n = 0, m = 0, nnz_c = 0, m_diag = 0, m_off = 0, nnz_aoff = 0;
    cudaStream_t stream = nullptr;       // caller's stream (entry points)
    cudaStream_t solve_stream = nullptr; // owned, capture-capable
    cudaEvent_t ev_sync = nullptr;
    cudaEvent_t ev_poll[2] = {nullptr, nullptr};
    int device = 0, num_sms = 0, max_blocks = 0;
    lorads_params prm{};
    std::string err;
    double bnorm_inf = 0, bnorm1 = 0, cnorm1 = 0, mean_abs_c = 1;
    // device problem arrays
    int64_t* c_rowptr = nullptr;
    int32_t* c_col = nullptr;
    double* c_val = nullptr;
    double* c_val0 = nullptr;           // C as uploaded, kept once re-opt scales c_val
    float* c_val32 = nullptr;
    dfloat* c_valdf = nullptr;
    int32_t* dk = nullptr;
    double* da = nullptr;
    float* da32 = nullptr;
    dfloat* da_df = nullptr;
    dfloat* b_df = nullptr;
    int64_t* a_rowptr = nullptr;
    int32_t* a_col = nullptr;
    int32_t* a_k = nullptr;
    double* a_a = nullptr;
    int32_t* k_row = nullptr;
    int32_t* k_col = nullptr;
    double* k_a = nullptr;
    int32_t* k_id = nullptr;
    int64_t* k_ptr = nullptr;           // general form: triplet range of each list position
    double* b = nullptr;
    dfloat* k_adf = nullptr;
    dfloat* a_adf = nullptr;
    ProbDev pd{};
    // scratch
    double* part = nullptr;
    double* small = nullptr;            // 64 doubles of scratch results
    double* h_small = nullptr;          // pinned mirror
    Ctrl* ctrl = nullptr;
    Ctrl* h_ctrl = nullptr;             // pinned, 2 slots
    SolverState st;
    AdmmState admm;
    Prof* prof = nullptr;
    bool prof_valid = false;
    bool prof_active = false;
    int64_t launches = 0;          // kernels launched by the current solve
    int64_t iter_limit = 0;        // cap on the total L-BFGS iterations of a solve (0: none)
    int64_t graph_nodes = 0;       // kernel nodes of the captured iteration graph
};

// ============================================================== helpers
namespace {

bool set_err(lorads_ctx* c, const std::string& msg) {
    if (c) c->err = msg;
    return false;
}

#define CK(call)                                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return LORADS_ERR_CUDA;                                                        \
        }                                                                                  \
    } while (0)

template <typename T>
lorads_status dalloc(lorads_ctx* ctx, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return LORADS_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes: " +
                   cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? LORADS_ERR_OOM : LORADS_ERR_CUDA;
    }
    return LORADS_OK;
}

template <typename T>
lorads_status upload(lorads_ctx* ctx, T** p, const T* host, size_t count) {
    lorads_status s = dalloc(ctx, p, count);
    if (s != LORADS_OK || count == 0) return s;
    CK(cudaMemcpy(*p, host, count * sizeof(T), cudaMemcpyHostToDevice));
    return LORADS_OK;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

int row_blocks(const lorads_ctx* c, int64_t rows, int L) {
    const int64_t per_block = kThreads / L;
    int64_t b = (rows + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, c->max_blocks);
}

int flat_blocks(const lorads_ctx* c, int64_t items) {
    int64_t b = (items + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    return (int)std::min<int64_t>(b, c->max_blocks);
}

double* part_of(const lorads_ctx* c, int region) {
    return c->part + (size_t)region * c->max_blocks * kPartStride;
}

lorads_status check_launch(lorads_ctx* ctx, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
        return LORADS_ERR_CUDA;
    }
    return LORADS_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

size_t elem_size(int prec) {
    switch (prec) {
        case LORADS_FP64: return 8;
        case LORADS_FP32: return 4;
        case LORADS_BF16: return 2;
        default: return 0;
    }
}

lorads_status check_factor_args(lorads_ctx* ctx, int32_t r, int32_t ld, int prec, Shape* sh) {
    if (elem_size(prec) == 0) return set_err(ctx, "prec must be LORADS_FP64, LORADS_FP32 or LORADS_BF16"), LORADS_ERR_INVALID_ARG;
    if (r < 1 || ld < r) return set_err(ctx, "need 1 <= r <= ld"), LORADS_ERR_INVALID_ARG;
    if (!shape_for_ld(ld, sh))
        return set_err(ctx, "ld=" + std::to_string(ld) + " is not a supported row width (a multiple of 4, at most " +
                                std::to_string(kMaxLd) + ")"),
               LORADS_ERR_INVALID_ARG;
    return LORADS_OK;
}

}  // namespace

// ============================================================== params
extern "C" void lorads_default_params(lorads_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->tol = 1e-5;
    p->time_limit = 1e4;
    p->lbfgs_mem = 4;
    p->max_inner = 500;
    p->max_outer = 200;
    p->rank_update_threshold = 3;
    p->rho0 = 0.0;
    p->rho_growth = 2.0;
    p->rho_max = 1e12;
    p->infeas_decrease = 0.25;
    p->inner_rel = 1.0;
    p->inner_progress = 0.1;
    p->prec = LORADS_FP64;
    p->check_every = 16;
    p->seed = 0;
    p->compute_err2 = 0;
    p->lanczos_steps = 200;
    p->verbose = 0;
    p->lbfgs_scaling = 1;
    p->rho_policy = 2;
    p->inner_scale = 2;
    p->kernel_variant = 2 | 8 | 128 | 256;
    p->admm_switch = 0.0;
    p->cg_rel = 1e-2;
    p->cg_max = 50;
    p->admm_max_iter = 20000;
    p->reopt_level = 0;
    p->max_reopt = 5;
    p->reopt_factor = 0.1;
}

extern "C" const char* lorads_create_error(void) { return g_create_error.c_str(); }

extern "C" const char* lorads_last_error(const lorads_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ============================================================== destroy
namespace {
void free_state(SolverState& st) {
    if (st.exec) cudaGraphExecDestroy(st.exec);
    dfree(st.R); dfree(st.CR); dfree(st.D); dfree(st.CD); dfree(st.G); dfree(st.W); dfree(st.hist);
    dfree(st.y); dfree(st.ytil); dfree(st.zrow); dfree(st.zk); dfree(st.ydf);
    st = SolverState();
}
// Frees what the ADMM state owns; arrays lent by the solver state stay.
void release_admm_arrays(AdmmState& a) {
    if (!a.borrowed) {
        dfree(a.U); dfree(a.V); dfree(a.r); dfree(a.p); dfree(a.Q); dfree(a.om);
    }
    a.U = a.V = a.r = a.p = a.Q = a.om = nullptr;
    a.borrowed = false;
    a.rtype = a.wtype = -1;
    a.ld = 0;
}
void free_admm(AdmmState& a) {
    if (a.exec) cudaGraphExecDestroy(a.exec);
    release_admm_arrays(a);
    dfree(a.ac);
    if (a.h_ac) cudaFreeHost(a.h_ac);
    a = AdmmState();
}
}  // namespace

extern "C" void lorads_destroy(lorads_ctx* ctx) {
    if (!ctx) return;
    if (ctx->solve_stream) cudaStreamSynchronize(ctx->solve_stream);
    free_state(ctx->st);
    free_admm(ctx->admm);
    dfree(ctx->c_rowptr); dfree(ctx->c_col); dfree(ctx->c_val); dfree(ctx->c_val0); dfree(ctx->c_val32); dfree(ctx->c_valdf);
    dfree(ctx->dk); dfree(ctx->da); dfree(ctx->da32); dfree(ctx->da_df); dfree(ctx->b_df);
    dfree(ctx->a_rowptr); dfree(ctx->a_col); dfree(ctx->a_k); dfree(ctx->a_a);
    dfree(ctx->k_row); dfree(ctx->k_col); dfree(ctx->k_a); dfree(ctx->k_id); dfree(ctx->k_ptr); dfree(ctx->b);
    dfree(ctx->k_adf); dfree(ctx->a_adf);
    dfree(ctx->part); dfree(ctx->small); dfree(ctx->ctrl);
    if (ctx->h_small) cudaFreeHost(ctx->h_small);
    if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
    if (ctx->ev_sync) cudaEventDestroy(ctx->ev_sync);
    for (auto& e : ctx->ev_poll) if (e) cudaEventDestroy(e);
    if (ctx->prof) {
        for (int q = 0; q < Prof::kPool; ++q)
            for (int e = 0; e < 2; ++e)
                if (ctx->prof->ev[q][e]) cudaEventDestroy(ctx->prof->ev[q][e]);
        delete ctx->prof;
    }
    if (ctx->solve_stream) cudaStreamDestroy(ctx->solve_stream);
    delete ctx;
}

// ============================================================== create
namespace {

lorads_status validate_and_build(lorads_ctx* ctx, int64_t n, const int64_t* rp, const int32_t* ci,
                                 const double* cv, int64_t m, int64_t nnz_a, const int32_t* acon,
                                 const int32_t* arow, const int32_t* acol, const double* aval,
                                 const double* b) {
    HostProb hp;
    const lorads_status hs = build_host_prob(&hp, &ctx->err, n, rp, ci, cv, m, nnz_a, acon, arow, acol, aval, b);
    if (hs != LORADS_OK) return hs;
    ctx->cnorm1 = hp.cnorm1;
    ctx->mean_abs_c = hp.mean_abs_c;
    ctx->bnorm_inf = hp.bnorm_inf;
    ctx->bnorm1 = hp.bnorm1;
    ctx->nnz_aoff = hp.nnz_aoff;
    ctx->n = n; ctx->m = m; ctx->nnz_c = hp.nnz_c; ctx->m_diag = hp.m_diag; ctx->m_off = hp.m_off;
    const int64_t nnz = hp.nnz_c, m_diag = hp.m_diag, m_off = hp.m_off;
    // device (queried only once the host-side checks have passed)
    cudaError_t ce = cudaGetDevice(&ctx->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        ctx->err = std::string("CUDA device query: ") + cudaGetErrorString(ce);
        return LORADS_ERR_CUDA;
    }
    ctx->max_blocks = ctx->num_sms * 8;
    // upload
    lorads_status s;
    if ((s = upload(ctx, &ctx->c_rowptr, rp, n + 1))) return s;
    if ((s = upload(ctx, &ctx->c_col, ci, nnz))) return s;
    if ((s = upload(ctx, &ctx->c_val, cv, nnz))) return s;
    if ((s = upload(ctx, &ctx->c_val32, hp.cv32.data(), nnz))) return s;
    if ((s = upload(ctx, &ctx->c_valdf, hp.cvdf.data(), nnz))) return s;
    if (m_diag > 0) {
        if ((s = upload(ctx, &ctx->dk, hp.dk.data(), n))) return s;
        if ((s = upload(ctx, &ctx->da, hp.da.data(), n))) return s;
        if ((s = upload(ctx, &ctx->da32, hp.da32.data(), n))) return s;
        if ((s = upload(ctx, &ctx->da_df, hp.dadf.data(), n))) return s;
    }
    if ((s = upload(ctx, &ctx->b_df, hp.bdf.data(), m))) return s;
    if (m_off > 0) {
        if ((s = upload(ctx, &ctx->a_rowptr, hp.a_rp.data(), n + 1))) return s;
        if ((s = upload(ctx, &ctx->a_col, hp.a_col.data(), hp.a_col.size()))) return s;
        if ((s = upload(ctx, &ctx->a_k, hp.a_k.data(), hp.a_k.size()))) return s;
        if ((s = upload(ctx, &ctx->a_a, hp.a_a.data(), hp.a_a.size()))) return s;
    }
    const size_t n_trip = hp.k_row.size();       // m, or the triplet count of the general form
    if ((s = upload(ctx, &ctx->k_row, hp.k_row.data(), n_trip))) return s;
    if ((s = upload(ctx, &ctx->k_col, hp.k_col.data(), n_trip))) return s;
    if ((s = upload(ctx, &ctx->k_a, hp.k_a.data(), n_trip))) return s;
    if ((s = upload(ctx, &ctx->k_id, hp.k_id.data(), m))) return s;
    if (!hp.k_ptr.empty() && (s = upload(ctx, &ctx->k_ptr, hp.k_ptr.data(), m + 1))) return s;
    if ((s = upload(ctx, &ctx->b, b, m))) return s;
    if ((s = upload(ctx, &ctx->k_adf, hp.k_adf.data(), n_trip))) return s;
    if (m_off > 0 && (s = upload(ctx, &ctx->a_adf, hp.a_adf.data(), hp.a_adf.size()))) return s;
    ProbDev& p = ctx->pd;
    p.n = n; p.m = m;
    p.c_rowptr = ctx->c_rowptr; p.c_col = ctx->c_col; p.c_val = ctx->c_val; p.c_val32 = ctx->c_val32;
    p.c_valdf = ctx->c_valdf;
    p.dk = ctx->dk; p.da = ctx->da; p.da32 = ctx->da32; p.da_df = ctx->da_df; p.b_df = ctx->b_df;
    p.a_rowptr = ctx->a_rowptr; p.a_col = ctx->a_col; p.a_k = ctx->a_k; p.a_a = ctx->a_a;
    p.k_row = ctx->k_row; p.k_col = ctx->k_col; p.k_a = ctx->k_a; p.k_id = ctx->k_id; p.k_ptr = ctx->k_ptr;
    p.m_diag = m_diag; p.m_off = m_off;
    p.b = ctx->b;
    p.k_adf = ctx->k_adf;
    p.a_adf = ctx->a_adf;
    return LORADS_OK;
}

}  // namespace

extern "C" lorads_status lorads_create(lorads_ctx** out, int64_t n, const int64_t* c_rowptr,
                                       const int32_t* c_colind, const double* c_val, int64_t m, int64_t nnz_a,
                                       const int32_t* a_con, const int32_t* a_row, const int32_t* a_col,
                                       const double* a_val, const double* b, const lorads_params* p,
                                       void* cuda_stream) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return LORADS_ERR_INVALID_ARG;
    }
    *out = nullptr;
    lorads_ctx* ctx = new (std::nothrow) lorads_ctx();
    if (!ctx) {
        g_create_error = "host allocation failed";
        return LORADS_ERR_OOM;
    }
    lorads_default_params(&ctx->prm);
    if (p) ctx->prm = *p;
    const std::string perr = solver_params_error(ctx->prm);
    if (!perr.empty()) {
        g_create_error = perr;
        delete ctx;
        return LORADS_ERR_INVALID_ARG;
    }
    if (ctx->prm.check_every < 1) ctx->prm.check_every = 1;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    lorads_status s = validate_and_build(ctx, n, c_rowptr, c_colind, c_val, m, nnz_a, a_con, a_row, a_col, a_val, b);
    if (s == LORADS_OK) s = dalloc(ctx, &ctx->part, (size_t)NPART * ctx->max_blocks * kPartStride);
    if (s == LORADS_OK) s = dalloc(ctx, &ctx->small, 64);
    if (s == LORADS_OK) s = dalloc(ctx, &ctx->ctrl, 1);
    if (s == LORADS_OK) {
        if (cudaMallocHost(&ctx->h_small, 64 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&ctx->h_ctrl, 2 * sizeof(Ctrl)) != cudaSuccess ||
            cudaStreamCreateWithFlags(&ctx->solve_stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_sync, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_poll[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_poll[1], cudaEventDisableTiming) != cudaSuccess) {
            ctx->err = "pinned memory / stream / event creation failed";
            s = LORADS_ERR_CUDA;
        }
    }
    if (s != LORADS_OK) {
        g_create_error = ctx->err;
        if (s == LORADS_ERR_INVALID_ARG || s == LORADS_ERR_NOT_SYMMETRIC || s == LORADS_ERR_UNSUPPORTED) {
            delete ctx;          // nothing was allocated on the device
        } else {
            lorads_destroy(ctx);
        }
        return s;
    }
    *out = ctx;
    return LORADS_OK;
}

extern "C" lorads_status lorads_problem_info(const lorads_ctx* ctx, int64_t* n, int64_t* m, int64_t* nnz_c,
                                             int64_t* m_diag, int64_t* m_offdiag) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    if (n) *n = ctx->n;
    if (m) *m = ctx->m;
    if (nnz_c) *nnz_c = ctx->nnz_c;
    if (m_diag) *m_diag = ctx->m_diag;
    if (m_offdiag) *m_offdiag = ctx->m_off;
    return LORADS_OK;
}

// ============================================================== standalone entry points
extern "C" lorads_status lorads_spmm(lorads_ctx* ctx, const void* R, int32_t r, int32_t ld, const double* v,
                                     void* out, int32_t prec) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    Shape sh;
    lorads_status s = check_factor_args(ctx, r, ld, prec, &sh);
    if (s) return s;
    if (!R || !out || !aligned16(R) || !aligned16(out)) return set_err(ctx, "R and out must be 16-byte aligned device pointers"), LORADS_ERR_INVALID_ARG;
    if (R == out) return set_err(ctx, "out must not alias R"), LORADS_ERR_INVALID_ARG;
    const int nb = row_blocks(ctx, ctx->n, sh.L);
    SpmmCArgs a{ctx->pd, R, out, ld, sh, v, 1, EPI_NONE, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0, nullptr,
                nb, nullptr, PH_ALWAYS, ctx->stream};
    SpmmAArgs aa{ctx->pd, R, out, ld, sh, v, -1.0, 1, nb, nullptr, PH_ALWAYS, ctx->stream};
    switch (prec) {
        case LORADS_FP64:
            launch_spmm_c<double, double, double>(a);
            if (v && ctx->m_off) launch_spmm_a<double, double>(aa);
            break;
        case LORADS_FP32:
            launch_spmm_c<float, float, float>(a);
            if (v && ctx->m_off) launch_spmm_a<float, float>(aa);
            break;
        default:
            launch_spmm_c<bf16, float, bf16>(a);
            if (v && ctx->m_off) launch_spmm_a<bf16, float>(aa);
            break;
    }
    return check_launch(ctx, "lorads_spmm launch");
}

extern "C" lorads_status lorads_constraint_eval(lorads_ctx* ctx, const void* U, const void* V, int32_t r,
                                                int32_t ld, double* out, int32_t prec) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    Shape sh;
    lorads_status s = check_factor_args(ctx, r, ld, prec, &sh);
    if (s) return s;
    if (!U || !V || !out || !aligned16(U) || !aligned16(V))
        return set_err(ctx, "U, V must be 16-byte aligned device pointers and out non-NULL"), LORADS_ERR_INVALID_ARG;
    ConsArgs a{ctx->pd, CONS_EVAL, 0, ctx->m, U, V, ld, sh, nullptr, out, nullptr, nullptr, nullptr, 0.0, nullptr,
               row_blocks(ctx, ctx->m, sh.L), nullptr, PH_ALWAYS, ctx->stream};
    switch (prec) {
        case LORADS_FP64: launch_cons<double, double>(a); break;
        case LORADS_FP32: launch_cons<float, float>(a); break;
        default: launch_cons<bf16, bf16>(a); break;
    }
    return check_launch(ctx, "lorads_constraint_eval launch");
}

extern "C" lorads_status lorads_linesearch_coeffs(lorads_ctx* ctx, const void* R, const void* D, int32_t r,
                                                  int32_t ld, const double* y, double rho, double* a_out,
                                                  double* tau_out, int32_t prec) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    Shape sh;
    lorads_status s = check_factor_args(ctx, r, ld, prec, &sh);
    if (s) return s;
    if (!R || !D || !y || !a_out || !aligned16(R) || !aligned16(D))
        return set_err(ctx, "R, D, y must be device pointers (R, D 16-byte aligned) and a_out non-NULL"),
               LORADS_ERR_INVALID_ARG;
    if (!std::isfinite(rho) || rho < 0) return set_err(ctx, "rho must be finite and >= 0"), LORADS_ERR_INVALID_ARG;
    const int nb = row_blocks(ctx, ctx->n, sh.L);
    const int nbc = row_blocks(ctx, std::max<int64_t>(ctx->m_off, 1), sh.L);
    double* pl = part_of(ctx, PART_LS);
    double* pc = part_of(ctx, PART_CONS_LS);
    SpmmCArgs a{ctx->pd, D, nullptr, ld, sh, nullptr, 0, EPI_LS, R, y, nullptr, nullptr, nullptr, rho, pl,
                nb, nullptr, PH_ALWAYS, ctx->stream};
    ConsArgs ca{ctx->pd, CONS_LS, ctx->m_diag, ctx->m, R, D, ld, sh, const_cast<double*>(y), nullptr, nullptr, nullptr, nullptr, rho,
                pc, nbc, nullptr, PH_ALWAYS, ctx->stream};
    switch (prec) {
        case LORADS_FP64:
            launch_spmm_c<double, double, double>(a);
            launch_cons<double, double>(ca);
            break;
        case LORADS_FP32:
            launch_spmm_c<float, float, float>(a);
            launch_cons<float, float>(ca);
            break;
        default:
            launch_spmm_c<bf16, float, bf16>(a);
            launch_cons<bf16, bf16>(ca);
            break;
    }
    ls_finish(ctx->stream, pl, nb, ctx->m_off ? pc : nullptr, nbc, rho, ctx->small);
    if ((s = check_launch(ctx, "lorads_linesearch_coeffs launch"))) return s;
    CK(cudaMemcpyAsync(ctx->h_small, ctx->small, 5 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < 4; ++q) a_out[q] = ctx->h_small[q];
    if (tau_out) *tau_out = ctx->h_small[4];
    return LORADS_OK;
}

// ============================================================== solver
namespace {

lorads_status run_lanczos(lorads_ctx* ctx, const double* ydev, int k, uint64_t seed, double* sigma_out);

template <typename TR, typename TD, typename TDIR = TD>
struct Driver {
    // y~ of the off-diagonal constraints is double-float on every path but FP64
    static constexpr int kYtilDf = std::is_same<TR, double>::value ? 0 : 1;
    lorads_ctx* c;
    SolverState& st;
    cudaStream_t s;
    int nb_rows, nb_ls, nb_flat, nb_off, nb_all;
    int64_t nunits;

    Driver(lorads_ctx* ctx) : c(ctx), st(ctx->st), s(ctx->solve_stream) { refresh(); }

    void refresh() {
        nb_rows = row_blocks(c, c->n, st.sh.L);
        nb_ls = row_blocks(c, c->n, st.sh_ls.L);
        nunits = c->n * (int64_t)st.ld / 4;
        nb_flat = flat_blocks(c, nunits);
        nb_off = row_blocks(c, std::max<int64_t>(c->m_off, 1), st.sh.L);
        nb_all = row_blocks(c, c->m, st.sh.L);
    }

    const ProbDev& p() const { return c->pd; }

    // Launch with an event pair around it when profiling.
    template <class F>
    void timed(int fam, F&& launch) {
        c->launches += 1;
        Prof* pf = c->prof;
        if (pf && pf->used < Prof::kPool) {
            const int q = pf->used++;
            pf->fam[q] = fam;
            cudaEventRecord(pf->ev[q][0], s);
            launch();
            cudaEventRecord(pf->ev[q][1], s);
        } else {
            launch();
        }
    }

    // G = grad L at the current R (outer tail and start): [y~, W], update, reset
    void outer_gradient(int ph) {
        if (c->m_off) {
            ConsArgs yt{p(), CONS_YTIL, c->m_diag, c->m, st.R, st.R, st.ld, st.sh, st.y, st.ytil, st.zk, st.ydf, c->ctrl, 0.0,
                        part_of(c, PART_YTIL), nb_off, c->ctrl, ph, s};
            timed(FAM_CONS_YTIL, [&] { launch_cons<TR, TR>(yt); });
            SpmmAArgs w{p(), st.R, st.W, st.ld, st.sh, st.ytil, 1.0, 0, nb_rows, c->ctrl, ph, s, kYtilDf};
            timed(FAM_SPMM_A, [&] { launch_spmm_a<TR, TD>(w); });
        }
        UpdateArgs u{p(), false, false, st.R, st.CR, st.D, st.CD, st.G, c->m_off ? st.W : nullptr, st.hist,
                     st.slot_stride, st.ld, st.sh, st.y, st.ydf, st.zrow, c->ctrl, part_of(c, PART_UPD), nb_rows, c->ctrl, ph, s};
        timed(FAM_GRAD, [&] { launch_update<TR, TD, TDIR>(u); });
        timed(FAM_HIST, [&] {
            ctrl_hist(s, c->ctrl, HIST_RESET, part_of(c, PART_UPD), nb_rows,
                      c->m_off ? part_of(c, PART_YTIL) : nullptr, nb_off);
        });
    }

    void spmm_CR(int ph) {
        SpmmCArgs a{p(), st.R, st.CR, st.ld, st.sh, nullptr, 1, EPI_OBJ, st.R, st.y, nullptr, nullptr, c->ctrl, 0.0,
                    part_of(c, PART_OBJ), nb_rows, c->ctrl, ph, s};
        timed(FAM_SPMM_CR, [&] { launch_spmm_c<TR, TR, TR>(a); });
    }

    void enqueue_init() {
        spmm_CR(PH_ALWAYS);
        ConsArgs zz{p(), CONS_ZZ, 0, c->m, st.R, st.R, st.ld, st.sh, st.y, nullptr, nullptr, nullptr, c->ctrl, 0.0,
                    part_of(c, PART_CONS), nb_all, c->ctrl, PH_ALWAYS, s};
        timed(FAM_MISC, [&] { launch_cons<TR, TR>(zz); });
        timed(FAM_MISC, [&] { ctrl_init(s, c->ctrl, part_of(c, PART_CONS), nb_all, part_of(c, PART_OBJ), nb_rows); });
        outer_gradient(PH_OUTER);
    }

    void enqueue_resume() {
        timed(FAM_MISC, [&] { ctrl_resume(s, c->ctrl); });
        spmm_CR(PH_OUTER);
        outer_gradient(PH_OUTER);
    }

    void enqueue_inner() {
        DirArgs d{nunits, st.G, st.D, st.hist, st.slot_stride, c->ctrl, part_of(c, PART_DIR), nb_flat, c->ctrl,
                  PH_INNER, s};
        timed(FAM_DIR, [&] { launch_dir<TD, TDIR>(d); });
        SpmmCArgs ls{p(), st.D, st.CD, st.ld, st.sh_ls, nullptr, 1, EPI_LS, st.R, st.y, st.zrow, st.ydf, c->ctrl, 0.0,
                     part_of(c, PART_LS), nb_ls, c->ctrl, PH_INNER, s,
                     (c->prm.kernel_variant & 8) ? ((c->prm.kernel_variant & 64) ? 2 : 1) : 0,
                     (c->prm.kernel_variant & 256) ? 1 : 0};
        timed(FAM_SPMM_LS, [&] { launch_spmm_c<TDIR, TD, TR>(ls); });
        if (c->m_off) {
            ConsArgs cl{p(), CONS_LS, c->m_diag, c->m, st.R, st.D, st.ld, st.sh, st.y, nullptr, st.zk, st.ydf, c->ctrl, 0.0,
                        part_of(c, PART_CONS_LS), nb_off, c->ctrl, PH_INNER, s};
            timed(FAM_CONS_LS, [&] { launch_cons<TR, TDIR>(cl); });
        }
        timed(FAM_ROOT, [&] {
            ctrl_root(s, c->ctrl, part_of(c, PART_DIR), nb_flat, part_of(c, PART_LS), nb_ls,
                      c->m_off ? part_of(c, PART_CONS_LS) : nullptr, nb_off);
        });
        if (c->m_off) {
            StepArgs sa{nunits, st.R, st.CR, st.D, st.CD, c->ctrl, nb_flat, c->ctrl, PH_STEP, s};
            timed(FAM_STEP, [&] { launch_step<TR, TD, TDIR>(sa); });
            ConsArgs yt{p(), CONS_YTIL, c->m_diag, c->m, st.R, st.R, st.ld, st.sh, st.y, st.ytil, st.zk, st.ydf, c->ctrl, 0.0,
                        part_of(c, PART_YTIL), nb_off, c->ctrl, PH_STEP, s};
            timed(FAM_CONS_YTIL, [&] { launch_cons<TR, TR>(yt); });
            SpmmAArgs w{p(), st.R, st.W, st.ld, st.sh, st.ytil, 1.0, 0, nb_rows, c->ctrl, PH_STEP, s, kYtilDf};
            timed(FAM_SPMM_A, [&] { launch_spmm_a<TR, TD>(w); });
        }
        UpdateArgs u{p(), c->m_off == 0, true, st.R, st.CR, st.D, st.CD, st.G, c->m_off ? st.W : nullptr, st.hist,
                     st.slot_stride, st.ld, st.sh, st.y, st.ydf, st.zrow, c->ctrl, part_of(c, PART_UPD), nb_rows, c->ctrl, PH_STEP, s,
                     (c->prm.kernel_variant & 4) ? 2 : ((c->prm.kernel_variant & 2) ? 1 : 0),
                     (c->prm.kernel_variant & 16) ? 1 : 0, (c->prm.kernel_variant & 128) ? 1 : 0,
                     c->prm.lbfgs_mem - 1};
        timed(FAM_UPDATE, [&] { launch_update<TR, TD, TDIR>(u); });
        timed(FAM_HIST, [&] {
            ctrl_hist(s, c->ctrl, HIST_STEP, part_of(c, PART_UPD), nb_rows,
                      c->m_off ? part_of(c, PART_YTIL) : nullptr, nb_off);
        });
    }

    // ALM outer step (Sec. 2.1) once the inner loop has finished
    void enqueue_outer() {
        ConsArgs yu{p(), CONS_YUPD, 0, c->m, st.R, st.R, st.ld, st.sh, st.y, nullptr, nullptr, st.ydf, c->ctrl, 0.0,
                    part_of(c, PART_CONS), nb_all, c->ctrl, PH_OUTER, s};
        timed(FAM_CONS_YUPD, [&] { launch_cons<TR, TR>(yu); });
        spmm_CR(PH_OUTER);
        timed(FAM_OUTER, [&] {
            ctrl_outer(s, c->ctrl, part_of(c, PART_CONS), nb_all, part_of(c, PART_OBJ), nb_rows);
        });
        outer_gradient(PH_OUTER);
    }

    void enqueue_iteration() {
        enqueue_inner();
        enqueue_outer();
    }
};

template <typename TR, typename TD, typename TDIR = TD>
lorads_status alloc_state(lorads_ctx* ctx, int prec, int r) {
    SolverState& st = ctx->st;
    const int ld = padded_ld(r);
    Shape sh;
    if (!shape_for_ld(ld, &sh))
        return set_err(ctx, "rank " + std::to_string(r) + " exceeds the supported row width"), LORADS_ERR_UNSUPPORTED;
    if (st.prec == prec && st.ld == ld && st.R) {
        st.r = r;
        return LORADS_OK;
    }
    free_state(st);
    st.prec = prec;
    st.r = r;
    st.ld = ld;
    st.sh = sh;
    st.sh_ls = sh;
    if (ctx->prm.kernel_variant & 32) shape_narrow(ld, &st.sh_ls);
    st.esR = sizeof(TR);
    st.esD = sizeof(TD);
    st.esDir = sizeof(TDIR);
    st.rtype = std::is_same<TR, double>::value ? 0 : (std::is_same<TR, dfloat>::value ? 1 : 2);
    const size_t nl = (size_t)ctx->n * ld;
    lorads_status s;
    const int T = ctx->prm.lbfgs_mem;
    if ((s = dalloc(ctx, reinterpret_cast<TR**>(&st.R), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TR**>(&st.CR), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TDIR**>(&st.D), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TD**>(&st.CD), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TD**>(&st.G), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TDIR**>(&st.hist), nl * 2 * T))) return s;
    st.slot_stride = (int64_t)nl;
    if (ctx->m_off) {
        if ((s = dalloc(ctx, reinterpret_cast<TD**>(&st.W), nl))) return s;
        if ((s = dalloc(ctx, &st.ytil, ctx->m))) return s;
    }
    if ((s = dalloc(ctx, &st.y, ctx->m))) return s;
    const bool fp64_path = std::is_same<TR, double>::value && std::is_same<TD, double>::value;
    // z cache: double (FP64), double-float (DF64) or float (mixed, FP32): 8 bytes covers all
    if ((s = dalloc(ctx, reinterpret_cast<double**>(&st.zrow), ctx->n))) return s;
    if (!fp64_path && (s = dalloc(ctx, &st.ydf, ctx->m))) return s;
    if ((s = dalloc(ctx, &st.zk, ctx->m))) return s;
    CK(cudaMemset(st.R, 0, nl * sizeof(TR)));
    CK(cudaMemset(st.CR, 0, nl * sizeof(TR)));
    CK(cudaMemset(st.D, 0, nl * sizeof(TDIR)));
    CK(cudaMemset(st.CD, 0, nl * sizeof(TD)));
    CK(cudaMemset(st.G, 0, nl * sizeof(TD)));
    CK(cudaMemset(st.hist, 0, nl * 2 * T * sizeof(TDIR)));
    if (st.W) CK(cudaMemset(st.W, 0, nl * sizeof(TD)));
    return LORADS_OK;
}

template <typename TR, typename TD, typename TDIR = TD>
lorads_status capture(lorads_ctx* ctx) {
    SolverState& st = ctx->st;
    if (st.exec) {
        cudaGraphExecDestroy(st.exec);
        st.exec = nullptr;
    }
    Driver<TR, TD, TDIR> drv(ctx);
    cudaGraph_t g = nullptr;
    const int64_t before = ctx->launches;
    CK(cudaStreamBeginCapture(ctx->solve_stream, cudaStreamCaptureModeThreadLocal));
    drv.enqueue_iteration();
    ctx->graph_nodes = ctx->launches - before;
    ctx->launches = before;
    cudaError_t e = cudaStreamEndCapture(ctx->solve_stream, &g);
    if (e != cudaSuccess) {
        ctx->err = std::string("graph capture: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return LORADS_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&st.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->err = std::string("graph instantiate: ") + cudaGetErrorString(e);
        return LORADS_ERR_CUDA;
    }
    return LORADS_OK;
}

// Grows the rank (App. A.1): new columns N(0, (1e-3 ||R||_F / sqrt(n r))^2).
template <typename TR, typename TD, typename TDIR = TD>
lorads_status grow_rank(lorads_ctx* ctx, int prec, int outer_done) {
    SolverState& st = ctx->st;
    const int r_old = st.r;
    const int r_cap = (int)std::ceil(std::sqrt(2.0 * (double)ctx->m));
    // App. A.1's rule, also bounded by the widest row the kernels support
    const int r_new = std::min(std::min((int)std::ceil(1.5 * r_old), r_cap), kMaxLd);
    if (r_new <= r_old) return LORADS_OK;
    cudaStream_t s = ctx->solve_stream;
    // ||R||_F^2
    double* pm = part_of(ctx, PART_MISC);
    const int nb = flat_blocks(ctx, ctx->n * (int64_t)r_old);
    sumsq<TR>(s, ctx->n, st.ld, r_old, st.R, pm, nb);
    fold_to(s, pm, nb, 1, ctx->small);
    CK(cudaMemcpyAsync(ctx->h_small, ctx->small, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double scale = 1e-3 * std::sqrt(ctx->h_small[0]) / std::sqrt((double)ctx->n * r_old);
    // keep R and y, rebuild everything else at the new width
    const int ld_old = st.ld;
    TR* R_old = nullptr;
    lorads_status rs;
    if ((rs = dalloc(ctx, &R_old, (size_t)ctx->n * ld_old))) return rs;
    CK(cudaMemcpyAsync(R_old, st.R, (size_t)ctx->n * ld_old * sizeof(TR), cudaMemcpyDeviceToDevice, s));
    double* y_keep = nullptr;
    if ((rs = dalloc(ctx, &y_keep, ctx->m))) return rs;
    CK(cudaMemcpyAsync(y_keep, st.y, ctx->m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    st.prec = -1;                                   // force reallocation
    if ((rs = alloc_state<TR, TD, TDIR>(ctx, prec, r_new))) return rs;
    convert<TR, TR>(s, ctx->n, ld_old, st.ld, r_old, R_old, st.R, flat_blocks(ctx, ctx->n * (int64_t)st.ld));
    rank_columns<TR>(s, ctx->n, st.ld, r_old, r_new, scale, ctx->prm.seed, (uint64_t)(outer_done - 1), st.R,
                     flat_blocks(ctx, ctx->n * (int64_t)(r_new - r_old)));
    ctx->launches += 4;                     // sumsq, fold, convert, columns
    CK(cudaMemcpyAsync(st.y, y_keep, ctx->m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (st.ydf) convert<double, dfloat>(s, ctx->m, 1, 1, 1, st.y, st.ydf, flat_blocks(ctx, ctx->m));
    CK(cudaStreamSynchronize(s));
    cudaFree(R_old);
    cudaFree(y_keep);
    return check_launch(ctx, "rank update");
}

lorads_status fill_result(lorads_ctx* ctx, std::chrono::steady_clock::time_point t0, bool timed_out,
                          lorads_result* res) {
    Ctrl hc;
    CK(cudaStreamSynchronize(ctx->solve_stream));
    CK(cudaMemcpy(&hc, ctx->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    ctx->st.have_solution = true;
    const lorads_status final_status =
        timed_out && !hc.solve_done ? LORADS_ERR_TIMEOUT : (lorads_status)hc.status;
    if (res) {
        res->primal_obj = hc.primal_obj;
        res->dual_obj = hc.dual_obj;
        res->err1 = hc.err1;
        res->err2 = -1.0;
        res->err3 = hc.err3;
        res->sigma_min = 0.0;
        res->rho = hc.rho;
        res->rank = ctx->st.r;
        res->outer_iters = hc.outer;
        res->inner_iters = hc.total_inner;
        res->status = final_status;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        res->kernel_launches = ctx->launches;
        res->reopt_scale = 1.0;
    }
    return final_status;
}

// Host-stepped solve with a CUDA-event pair around every launch (verbose >= 2):
// same kernels and decisions as the graph path, one host sync per iteration.
template <typename TR, typename TD, typename TDIR = TD>
lorads_status run_profiled(lorads_ctx* ctx, int prec, std::chrono::steady_clock::time_point t0,
                           lorads_result* res) {
    lorads_status s;
    if (!ctx->prof) {
        ctx->prof = new (std::nothrow) Prof();
        if (!ctx->prof) return set_err(ctx, "host allocation failed"), LORADS_ERR_OOM;
        for (int q = 0; q < Prof::kPool; ++q)
            for (int e = 0; e < 2; ++e) CK(cudaEventCreate(&ctx->prof->ev[q][e]));
    }
    Prof* pf = ctx->prof;
    for (int f = 0; f < NFAM; ++f) { pf->total_ms[f] = 0; pf->count[f] = 0; }
    cudaStream_t ss = ctx->solve_stream;
    bool timed_out = false;
    for (;;) {
        Ctrl hc;
        CK(cudaMemcpyAsync(&ctx->h_ctrl[0], ctx->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, ss));
        CK(cudaStreamSynchronize(ss));
        hc = ctx->h_ctrl[0];
        if (hc.solve_done) break;
        Driver<TR, TD, TDIR> drv(ctx);
        if (hc.pause) {
            if ((s = grow_rank<TR, TD, TDIR>(ctx, prec, hc.outer))) return s;
            Driver<TR, TD, TDIR> d2(ctx);
            d2.enqueue_resume();
            continue;
        }
        pf->used = 0;
        if (hc.phase == PHASE_INNER) drv.enqueue_inner();
        else drv.enqueue_outer();
        if ((s = check_launch(ctx, "profiled iteration"))) return s;
        CK(cudaStreamSynchronize(ss));
        for (int q = 0; q < pf->used; ++q) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, pf->ev[q][0], pf->ev[q][1]));
            pf->total_ms[pf->fam[q]] += ms;
            pf->count[pf->fam[q]] += 1;
        }
        pf->used = 0;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > ctx->prm.time_limit) { timed_out = true; break; }
    }
    ctx->prof_valid = true;
    ctx->prof_active = false;
    return fill_result(ctx, t0, timed_out, res);
}

// Allocates the solver state for the starting rank and loads R <- R0 (or the
// device random start) and y <- y0 (or 0), with the double-float mirror of y.
template <typename TR, typename TD, typename TDIR = TD>
lorads_status start_state(lorads_ctx* ctx, int prec, const double* R0, int32_t r0, int32_t r0_on_device,
                          const double* y0) {
    const lorads_params& P = ctx->prm;
    lorads_status s;
    int r = r0;
    if (r <= 0) r = std::max(1, (int)std::ceil(std::log2((double)std::max<int64_t>(ctx->m, 2))));
    if ((s = alloc_state<TR, TD, TDIR>(ctx, prec, r))) return s;
    SolverState& st = ctx->st;
    cudaStream_t ss = ctx->solve_stream;
    CK(cudaEventRecord(ctx->ev_sync, ctx->stream));
    CK(cudaStreamWaitEvent(ss, ctx->ev_sync, 0));
    const size_t nl = (size_t)ctx->n * st.ld;
    // R <- R0 (padded to ld, converted to TR)
    if (R0) {
        double* tmp = nullptr;
        if ((s = dalloc(ctx, &tmp, (size_t)ctx->n * r))) return s;
        CK(cudaMemcpyAsync(tmp, R0, (size_t)ctx->n * r * sizeof(double),
                           r0_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ss));
        convert<double, TR>(ss, ctx->n, r, st.ld, r, tmp, st.R, flat_blocks(ctx, (int64_t)nl));
        ctx->launches += 1;
        CK(cudaStreamSynchronize(ss));
        cudaFree(tmp);
    } else {
        CK(cudaMemsetAsync(st.R, 0, nl * sizeof(TR), ss));
        const double scale = std::sqrt(std::max(0.5 * ctx->bnorm1, 1.0) / ((double)ctx->n * r));
        random_start<TR>(ss, ctx->n, st.ld, r, P.seed, ctx->m_diag == ctx->m ? 1 : 0, scale, st.R,
                         flat_blocks(ctx, ctx->n));
        ctx->launches += 1;
    }
    if (y0) CK(cudaMemcpyAsync(st.y, y0, ctx->m * sizeof(double), cudaMemcpyHostToDevice, ss));
    else CK(cudaMemsetAsync(st.y, 0, ctx->m * sizeof(double), ss));
    if (st.ydf) {
        convert<double, dfloat>(ss, ctx->m, 1, 1, 1, st.y, st.ydf, flat_blocks(ctx, ctx->m));
        ctx->launches += 1;
    }
    return check_launch(ctx, "start");
}

// ---------------------------------------------------------------- ADMM stage (Sec. 2.2)
template <typename T>
constexpr int type_code() {
    return std::is_same<T, double>::value ? 0 : (std::is_same<T, dfloat>::value ? 1 : 2);
}

lorads_status admm_ctrl_alloc(lorads_ctx* ctx) {
    AdmmState& a = ctx->admm;
    lorads_status s;
    if (!a.ac && (s = dalloc(ctx, &a.ac, 1))) return s;
    if (!a.h_ac && cudaMallocHost(&a.h_ac, sizeof(AdmmCtrl)) != cudaSuccess) {
        cudaGetLastError();
        a.h_ac = nullptr;
        return set_err(ctx, "pinned allocation failed"), LORADS_ERR_OOM;
    }
    return LORADS_OK;
}

// Work arrays of the stage for row width ld, owned by the context (kept for later calls).
template <typename TR, typename TW>
lorads_status admm_alloc(lorads_ctx* ctx, int ld) {
    AdmmState& a = ctx->admm;
    if (a.U && !a.borrowed && a.rtype == type_code<TR>() && a.wtype == type_code<TW>() && a.ld == ld)
        return LORADS_OK;
    release_admm_arrays(a);
    const size_t nl = (size_t)ctx->n * ld;
    lorads_status s;
    if ((s = admm_ctrl_alloc(ctx))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TR**>(&a.U), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TR**>(&a.V), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TW**>(&a.r), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TW**>(&a.p), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<TW**>(&a.Q), nl))) return s;
    if ((s = dalloc(ctx, reinterpret_cast<double**>(&a.om), ctx->m))) return s;
    CK(cudaMemset(a.r, 0, nl * sizeof(TW)));
    CK(cudaMemset(a.p, 0, nl * sizeof(TW)));
    CK(cudaMemset(a.Q, 0, nl * sizeof(TW)));
    a.rtype = type_code<TR>();
    a.wtype = type_code<TW>();
    a.ld = ld;
    a.esR = sizeof(TR);
    a.esW = sizeof(TW);
    return LORADS_OK;
}

// The stage after an ALM solve: its arrays are lent by the solver state, whose
// L-BFGS history, gradient, direction and C D are not needed any more: r = G,
// p = C D, Q = D (or the first history bytes when D is stored narrower), U and V
// in the history slots, w in the z cache of the constraints (m doubles).  With
// two stored pairs of float history and double-float R the history holds U and V
// exactly.  When it is too small, owned arrays are used instead.
template <typename TR, typename TW>
lorads_status admm_bind(lorads_ctx* ctx) {
    AdmmState& a = ctx->admm;
    SolverState& st = ctx->st;
    const size_t nl = (size_t)ctx->n * st.ld;     // a multiple of 4: every offset below is 16-byte aligned
    const bool q_in_d = st.esDir == sizeof(TW);
    const size_t q_bytes = q_in_d ? 0 : nl * sizeof(TW);
    const size_t need = q_bytes + 2 * nl * sizeof(TR);
    const size_t have = nl * st.esDir * 2 * (size_t)ctx->prm.lbfgs_mem;
    if (need > have || st.esD != sizeof(TW)) return admm_alloc<TR, TW>(ctx, st.ld);
    lorads_status s;
    release_admm_arrays(a);
    if ((s = admm_ctrl_alloc(ctx))) return s;
    char* h = static_cast<char*>(st.hist);
    a.r = st.G;
    a.p = st.CD;
    a.Q = q_in_d ? st.D : static_cast<void*>(h);
    a.U = h + q_bytes;
    a.V = h + q_bytes + nl * sizeof(TR);
    a.om = st.zk;
    a.borrowed = true;
    a.rtype = type_code<TR>();
    a.wtype = type_code<TW>();
    a.ld = st.ld;
    a.esR = sizeof(TR);
    a.esW = sizeof(TW);
    return LORADS_OK;
}

AdmmRows admm_rows(const lorads_ctx* ctx, int ld, const Shape& sh, cudaStream_t s) {
    AdmmRows r;
    r.p = &ctx->pd;
    r.ld = ld;
    r.sh = sh;
    r.nb_rows = row_blocks(ctx, ctx->n, sh.L);
    r.nb_cons = row_blocks(ctx, ctx->m, sh.L);
    r.nb_flat = flat_blocks(ctx, ctx->n * (int64_t)ld / 4);
    r.stream = s;
    return r;
}

// One block step of Eq. (2.2): X <- the CG solution of frakA_Vf(X) = frakb_Vf(y)
// (Algorithm 2 from the current X, at most cg_max steps).  Returns kernels enqueued.
template <typename TR, typename TW>
int64_t admm_enqueue_block(lorads_ctx* ctx, const AdmmRows& rows, void* X, const void* Vf, double* y,
                           dfloat* ydf, int cg_max) {
    AdmmState& a = ctx->admm;
    cudaStream_t s = rows.stream;
    double* pr = part_of(ctx, PART_LS);
    double* pq = part_of(ctx, PART_DIR);
    double* pu = part_of(ctx, PART_UPD);
    admm_omega<TR>(rows, X, Vf, y, ydf, a.om, a.ac);
    admm_resid<TR, TW>(rows, X, Vf, a.om, a.r, a.p, a.ac, pr);
    admm_cg_init(s, a.ac, pr, rows.nb_rows);
    // general form: w of the listed constraints reuses the m-vector of the start
    // residual (read only by admm_resid, before the first CG step)
    const bool general = ctx->pd.k_ptr != nullptr && ctx->m_off > 0;
    double* pw = general ? part_of(ctx, PART_CONS_LS) : nullptr;
    for (int k = 0; k < cg_max; ++k) {
        admm_op<TR, TW>(rows, Vf, a.r, a.p, a.Q, a.ac, 0.0, 1, pq, a.om, pw);
        admm_alpha(s, a.ac, pq, rows.nb_rows, pw, rows.nb_cons);
        admm_upd<TR, TW>(rows, X, a.p, a.r, a.Q, a.ac, pu);
        admm_beta(s, a.ac, pu, rows.nb_flat);
    }
    return 3 + (int64_t)cg_max * (general ? 6 : (ctx->m_off ? 5 : 4));
}

// Multiplier step and the errors of Sec. 4.2 at R = (U + V)/2.
template <typename TR>
int64_t admm_enqueue_outer(lorads_ctx* ctx, const AdmmRows& rows) {
    AdmmState& a = ctx->admm;
    SolverState& st = ctx->st;
    cudaStream_t s = rows.stream;
    admm_yupd<TR>(rows, a.U, a.V, st.y, st.ydf, a.ac, part_of(ctx, PART_YTIL));
    admm_avg<TR>(rows, a.U, a.V, st.R);
    SpmmCArgs o{ctx->pd, st.R, st.CR, rows.ld, rows.sh, nullptr, 1, EPI_OBJ, st.R, st.y, nullptr, nullptr, nullptr,
                0.0, part_of(ctx, PART_OBJ), rows.nb_rows, nullptr, PH_ALWAYS, s};
    launch_spmm_c<TR, TR, TR>(o);
    ConsArgs z{ctx->pd, CONS_ZZ, 0, ctx->m, st.R, st.R, rows.ld, rows.sh, nullptr, nullptr, nullptr, nullptr,
               nullptr, 0.0, part_of(ctx, PART_CONS), rows.nb_cons, nullptr, PH_ALWAYS, s};
    launch_cons<TR, TR>(z);
    admm_outer(s, a.ac, part_of(ctx, PART_YTIL), rows.nb_cons, part_of(ctx, PART_CONS), rows.nb_cons,
               part_of(ctx, PART_OBJ), rows.nb_rows);
    return 5;
}

// The ADMM stage from U = V = R (the solver state), multiplier y of the state,
// penalty rho (fixed): one captured graph per ADMM iteration (U step, V step,
// multiplier step and errors), launched until the device control block says done.
template <typename TR, typename TW>
lorads_status run_admm(lorads_ctx* ctx, double rho, std::chrono::steady_clock::time_point t0, lorads_result* res) {
    SolverState& st = ctx->st;
    const lorads_params& P = ctx->prm;
    lorads_status s;
    if ((s = admm_bind<TR, TW>(ctx))) return s;
    AdmmState& a = ctx->admm;
    cudaStream_t ss = ctx->solve_stream;
    const size_t bytes = (size_t)ctx->n * st.ld * sizeof(TR);
    CK(cudaMemcpyAsync(a.U, st.R, bytes, cudaMemcpyDeviceToDevice, ss));
    CK(cudaMemcpyAsync(a.V, st.R, bytes, cudaMemcpyDeviceToDevice, ss));
    AdmmCtrl h{};
    h.rho = rho;
    h.cg_rel = P.cg_rel;
    h.tol = P.tol;
    h.bnorm_inf = ctx->bnorm_inf;
    h.cg_max = P.cg_max;
    h.max_iter = P.admm_max_iter;
    h.status = LORADS_ERR_MAXITER;
    CK(cudaMemcpyAsync(a.ac, &h, sizeof(AdmmCtrl), cudaMemcpyHostToDevice, ss));
    *a.h_ac = h;
    bool timed_out = false;
    if (P.admm_max_iter > 0) {
        if (a.exec) {
            cudaGraphExecDestroy(a.exec);
            a.exec = nullptr;
        }
        const AdmmRows rows = admm_rows(ctx, st.ld, st.sh, ss);
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ss, cudaStreamCaptureModeThreadLocal));
        int64_t nodes = admm_enqueue_block<TR, TW>(ctx, rows, a.U, a.V, st.y, st.ydf, P.cg_max);
        nodes += admm_enqueue_block<TR, TW>(ctx, rows, a.V, a.U, st.y, st.ydf, P.cg_max);
        nodes += admm_enqueue_outer<TR>(ctx, rows);
        cudaError_t e = cudaStreamEndCapture(ss, &g);
        if (e != cudaSuccess) {
            ctx->err = std::string("ADMM graph capture: ") + cudaGetErrorString(e);
            cudaGetLastError();
            return LORADS_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&a.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->err = std::string("ADMM graph instantiate: ") + cudaGetErrorString(e);
            return LORADS_ERR_CUDA;
        }
        a.graph_nodes = nodes;
        for (;;) {
            CK(cudaGraphLaunch(a.exec, ss));
            ctx->launches += a.graph_nodes;
            CK(cudaMemcpyAsync(a.h_ac, a.ac, sizeof(AdmmCtrl), cudaMemcpyDeviceToHost, ss));
            CK(cudaStreamSynchronize(ss));
            const AdmmCtrl& hc = *a.h_ac;
            if (P.verbose == 1)
                std::fprintf(stderr, "[lorads] admm %d cg %d err1 %.3e err3 %.3e obj %.10g t %.3fs\n", hc.iters,
                             hc.cg_total, hc.err1, hc.err3, hc.primal_obj,
                             std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
            if (hc.done) break;
            if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > P.time_limit) {
                timed_out = true;
                break;
            }
        }
    }
    st.have_solution = true;
    const AdmmCtrl& hc = *a.h_ac;
    const lorads_status fs = timed_out ? LORADS_ERR_TIMEOUT : (lorads_status)hc.status;
    if (res) {
        if (hc.iters > 0) {
            res->primal_obj = hc.primal_obj;
            res->dual_obj = hc.dual_obj;
            res->err1 = hc.err1;
            res->err3 = hc.err3;
        }
        res->rho = rho;
        res->rank = st.r;
        res->admm_iters = hc.iters;
        res->cg_steps = hc.cg_total;
        res->status = fs;
        res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        res->kernel_launches = ctx->launches;
    }
    return fs;
}

template <typename TR, typename TD, typename TDIR>
lorads_status run_graph(lorads_ctx* ctx, int prec, std::chrono::steady_clock::time_point t0, lorads_result* res);

// Uploads a fresh control block (penalty rho, stop tolerance and rule) and
// enqueues the start of an ALM solve from the state's R and y.
template <typename TR, typename TD, typename TDIR>
lorads_status start_alm(lorads_ctx* ctx, double rho, double tol, int stop_rule) {
    const lorads_params& P = ctx->prm;
    Ctrl h{};
    h.rho = rho;
    h.lbfgs_mem = P.lbfgs_mem;
    h.total_limit = ctx->iter_limit > 0 ? (int)std::min<int64_t>(ctx->iter_limit, INT32_MAX) : 0;
    h.max_inner = P.max_inner;
    h.max_outer = P.max_outer;
    h.rank_threshold = std::max(1, P.rank_update_threshold);
    h.lbfgs_scaling = P.lbfgs_scaling;
    h.rho_policy = P.rho_policy;
    h.inner_scale = P.inner_scale;
    h.stop_rule = stop_rule;
    h.tol = tol;
    h.inner_rel = P.inner_rel;
    h.inner_progress = P.inner_progress;
    h.bnorm1 = ctx->bnorm1;
    h.bnorm_inf = ctx->bnorm_inf;
    h.rho_growth = P.rho_growth;
    h.rho_max = P.rho_max;
    h.infeas_decrease = P.infeas_decrease;
    h.status = LORADS_ERR_MAXITER;
    for (int q = 0; q < kMaxMem; ++q) h.order[q] = q;
    CK(cudaMemcpyAsync(ctx->ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, ctx->solve_stream));
    Driver<TR, TD, TDIR> drv(ctx);
    drv.enqueue_init();
    return check_launch(ctx, "solve init");
}

template <typename TR, typename TD, typename TDIR>
lorads_status run_alm(lorads_ctx* ctx, int prec, std::chrono::steady_clock::time_point t0, lorads_result* res) {
    if (ctx->prm.verbose >= 2) return run_profiled<TR, TD, TDIR>(ctx, prec, t0, res);
    return run_graph<TR, TD, TDIR>(ctx, prec, t0, res);
}

// Re-opt (Sec. 4.1) after an ALM solve that stopped on primal feasibility
// alone: while the final criteria of the chosen level (Sec. 4.2; level 1: err1
// with 1 + ||b||_1 and |err3|; level 2: also err2) fail on the original
// problem, scale C by reopt_factor (compounding), keep R and rho, scale y with
// C, and solve the scaled problem again with the same stop.  At the end y and C
// are those of the original problem again.
template <typename TR, typename TD, typename TDIR>
lorads_status run_reopt(lorads_ctx* ctx, int prec, std::chrono::steady_clock::time_point t0, lorads_result* res) {
    const lorads_params& P = ctx->prm;
    SolverState& st = ctx->st;
    cudaStream_t ss = ctx->solve_stream;
    const int nbc = flat_blocks(ctx, ctx->nnz_c), nbm = flat_blocks(ctx, ctx->m);
    double scale = 1.0;
    int rounds = 0;
    int64_t inner = res->inner_iters, outer = res->outer_iters;
    lorads_status s = LORADS_OK;
    bool met = false;
    double obj = 0, by = 0, err3 = 0;
    for (;;) {
        // errors of the original problem: <C, X> = <sC, X>/s, b^T y = b^T (s y)/s
        obj = res->primal_obj / scale;
        by = res->dual_obj / scale;
        err3 = (obj - by) / (1.0 + std::fabs(obj) + std::fabs(by));
        const double err1_l1 = res->err1 * (1.0 + ctx->bnorm_inf) / (1.0 + ctx->bnorm1);
        met = err1_l1 <= P.tol && std::fabs(err3) <= P.tol;
        if (met && P.reopt_level >= 2) {
            double sig = 0.0;           // sigma_min(sC - A*(s y)) = s sigma_min(C - A*(y))
            if ((s = run_lanczos(ctx, st.y, P.lanczos_steps, P.seed, &sig))) break;
            met = std::max(0.0, -sig / scale) / (1.0 + ctx->cnorm1) <= P.tol;
        }
        if (met || rounds >= P.max_reopt) break;
        if (!ctx->c_val0) {
            if ((s = dalloc(ctx, &ctx->c_val0, (size_t)ctx->nnz_c))) break;
            CK(cudaMemcpyAsync(ctx->c_val0, ctx->c_val, (size_t)ctx->nnz_c * sizeof(double),
                               cudaMemcpyDeviceToDevice, ss));
        }
        const double s_new = scale * P.reopt_factor;
        scale_c(ss, ctx->nnz_c, ctx->c_val0, s_new, ctx->c_val, ctx->c_val32, ctx->c_valdf, nbc);
        rescale_y(ss, ctx->m, st.y, st.ydf, scale, s_new, nbm);
        ctx->launches += 2;
        scale = s_new;
        rounds += 1;
        if ((s = start_alm<TR, TD, TDIR>(ctx, res->rho, P.tol, 1))) break;
        lorads_result r2{};
        s = run_alm<TR, TD, TDIR>(ctx, prec, t0, &r2);
        inner += r2.inner_iters;
        outer += r2.outer_iters;
        *res = r2;
        if (s != LORADS_OK) break;
    }
    if (scale != 1.0) {
        rescale_y(ss, ctx->m, st.y, st.ydf, scale, 1.0, nbm);
        scale_c(ss, ctx->nnz_c, ctx->c_val0, 1.0, ctx->c_val, ctx->c_val32, ctx->c_valdf, nbc);
        ctx->launches += 2;
        CK(cudaStreamSynchronize(ss));
        if (s == LORADS_OK) {
            obj = res->primal_obj / scale;
            by = res->dual_obj / scale;
            err3 = (obj - by) / (1.0 + std::fabs(obj) + std::fabs(by));
        }
    }
    res->primal_obj = obj;
    res->dual_obj = by;
    res->err3 = err3;
    res->inner_iters = (int32_t)std::min<int64_t>(inner, INT32_MAX);
    res->outer_iters = (int32_t)std::min<int64_t>(outer, INT32_MAX);
    res->reopt_rounds = rounds;
    res->reopt_scale = scale;
    res->kernel_launches = ctx->launches;
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (s == LORADS_OK && !met) s = LORADS_ERR_MAXITER;
    res->status = s;
    return s;
}

template <typename TR, typename TD, typename TDIR = TD>
lorads_status run_solve(lorads_ctx* ctx, int prec, const double* R0, int32_t r0, int32_t r0_on_device,
                        const double* y0, lorads_result* res) {
    const auto t0 = std::chrono::steady_clock::now();
    const lorads_params& P = ctx->prm;
    ctx->launches = 0;
    lorads_status s;
    if ((s = start_state<TR, TD, TDIR>(ctx, prec, R0, r0, r0_on_device, y0))) return s;
    // two-stage solve: the ALM stage stops at the switch tolerance; re-opt: the
    // first solve stops on primal feasibility alone
    const bool two_stage = P.admm_switch > 0 && P.reopt_level <= 0;
    const double alm_tol = two_stage ? std::max(P.admm_switch, P.tol) : P.tol;
    const double rho0 = P.rho0 > 0 ? P.rho0 : 1.0 / ctx->mean_abs_c;
    if ((s = start_alm<TR, TD, TDIR>(ctx, rho0, alm_tol, P.reopt_level > 0 ? 1 : 0))) return s;
    lorads_result alm{};
    lorads_status fs = run_alm<TR, TD, TDIR>(ctx, prec, t0, &alm);
    if (fs == LORADS_OK && P.reopt_level > 0)
        fs = run_reopt<TR, TD, TDIR>(ctx, prec, t0, &alm);
    else if (fs == LORADS_OK && two_stage && !(alm.err1 <= P.tol && std::fabs(alm.err3) <= P.tol))
        fs = run_admm<TR, TD>(ctx, alm.rho, t0, &alm);
    if (res) *res = alm;
    return fs;
}

// The ALM stage on the captured iteration graph: launch it in batches, poll the
// status of the previous batch, grow the rank when the device asks.
template <typename TR, typename TD, typename TDIR>
lorads_status run_graph(lorads_ctx* ctx, int prec, std::chrono::steady_clock::time_point t0, lorads_result* res) {
    const lorads_params& P = ctx->prm;
    SolverState& st = ctx->st;
    cudaStream_t ss = ctx->solve_stream;
    lorads_status s;
    if ((s = capture<TR, TD, TDIR>(ctx))) return s;
    // ---- iterate: launch the graph in batches, poll the status of the previous batch
    int slot = 0;
    bool pending = false;
    int last_outer_printed = -1;
    bool timed_out = false;
    for (;;) {
        for (int k = 0; k < P.check_every; ++k) CK(cudaGraphLaunch(st.exec, ss));
        ctx->launches += (int64_t)P.check_every * ctx->graph_nodes;
        CK(cudaMemcpyAsync(&ctx->h_ctrl[slot], ctx->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, ss));
        CK(cudaEventRecord(ctx->ev_poll[slot], ss));
        if (pending) {
            CK(cudaEventSynchronize(ctx->ev_poll[slot ^ 1]));
            const Ctrl& hc = ctx->h_ctrl[slot ^ 1];
            if (P.verbose == 1 && hc.outer != last_outer_printed) {
                last_outer_printed = hc.outer;
                std::fprintf(stderr, "[lorads] outer %d inner %d rho %.3g err1 %.3e err3 %.3e obj %.10g r %d t %.3fs\n",
                             hc.outer, hc.total_inner, hc.last_iter_rho, hc.err1, hc.err3, hc.primal_obj, st.r,
                             std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
            }
            if (hc.solve_done || hc.pause) {
                CK(cudaStreamSynchronize(ss));
                const Ctrl& now = ctx->h_ctrl[slot];
                if (now.solve_done) break;
                // pause: grow the rank, then continue with the outer tail
                if ((s = grow_rank<TR, TD, TDIR>(ctx, prec, now.outer))) return s;
                Driver<TR, TD, TDIR> drv(ctx);
                drv.enqueue_resume();
                if ((s = check_launch(ctx, "resume"))) return s;
                if ((s = capture<TR, TD, TDIR>(ctx))) return s;
                pending = false;
                slot = 0;
                continue;
            }
        }
        pending = true;
        slot ^= 1;
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > P.time_limit) {
            CK(cudaStreamSynchronize(ss));
            timed_out = true;
            break;
        }
    }
    return fill_result(ctx, t0, timed_out, res);
}

}  // namespace

namespace {
lorads_status run_lanczos(lorads_ctx* ctx, const double* ydev, int k, uint64_t seed, double* sigma_out);
lorads_status finish_err2(lorads_ctx* ctx, lorads_status s, lorads_result* res);
}  // namespace

extern "C" lorads_status lorads_solve(lorads_ctx* ctx, const double* R0, int32_t r0, int32_t r0_on_device,
                                      const double* y0, lorads_result* res) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    if (res) std::memset(res, 0, sizeof(*res));
    if (R0 && r0 < 1) return set_err(ctx, "r0 must be >= 1 when R0 is given"), LORADS_ERR_INVALID_ARG;
    const int prec = ctx->prm.prec;
    lorads_status s;
    switch (prec) {
        case LORADS_FP64: s = run_solve<double, double>(ctx, prec, R0, r0, r0_on_device, y0, res); break;
        case LORADS_MIXED: s = run_solve<dfloat, float>(ctx, prec, R0, r0, r0_on_device, y0, res); break;
        case LORADS_DF64: s = run_solve<dfloat, dfloat>(ctx, prec, R0, r0, r0_on_device, y0, res); break;
        case LORADS_FP32: s = run_solve<float, float>(ctx, prec, R0, r0, r0_on_device, y0, res); break;
        case LORADS_MIXED_BF16:
            s = run_solve<dfloat, float, __nv_bfloat16>(ctx, prec, R0, r0, r0_on_device, y0, res);
            break;
        default:
            return set_err(ctx, "params.prec must be FP64, MIXED, DF64, FP32 or MIXED_BF16 for lorads_solve"),
                   LORADS_ERR_INVALID_ARG;
    }
    return finish_err2(ctx, s, res);
}

namespace {

// err2 of Sec. 4.2 at the returned multiplier: sigma_min(C - A*(y)) by Lanczos.
lorads_status finish_err2(lorads_ctx* ctx, lorads_status s, lorads_result* res) {
    if (res && res->status == 0 && s != LORADS_OK) res->status = s;
    if (ctx->prm.compute_err2 && ctx->st.have_solution && (s == LORADS_OK || s == LORADS_ERR_MAXITER)) {
        double sig = 0.0;
        const lorads_status ls = run_lanczos(ctx, ctx->st.y, ctx->prm.lanczos_steps, ctx->prm.seed, &sig);
        if (ls != LORADS_OK) return ls;
        if (res) {
            res->sigma_min = sig;
            res->err2 = std::max(0.0, -sig) / (1.0 + ctx->cnorm1);
            res->kernel_launches = ctx->launches;
        }
    }
    return s;
}

template <typename TR, typename TD, typename TDIR = TD>
lorads_status run_stage(lorads_ctx* ctx, int prec, const double* R0, int32_t r0, int32_t r0_on_device,
                        const double* y0, double rho, lorads_result* res) {
    const auto t0 = std::chrono::steady_clock::now();
    ctx->launches = 0;
    lorads_status s;
    if ((s = start_state<TR, TD, TDIR>(ctx, prec, R0, r0, r0_on_device, y0))) return s;
    lorads_result out{};
    s = run_admm<TR, TD>(ctx, rho, t0, &out);
    if (res) *res = out;
    return s;
}

template <typename TR, typename TW>
lorads_status run_admm_cg(lorads_ctx* ctx, const void* V, void* X, const double* y, double rho, int ld,
                          const Shape& sh, double cg_rel, int cg_max, int32_t* steps_out) {
    lorads_status s;
    if ((s = admm_alloc<TR, TW>(ctx, ld))) return s;
    AdmmState& a = ctx->admm;
    AdmmCtrl h{};
    h.rho = rho;
    h.cg_rel = cg_rel;
    h.cg_max = cg_max;
    h.tol = ctx->prm.tol;
    h.bnorm_inf = ctx->bnorm_inf;
    h.max_iter = 1;
    h.status = LORADS_OK;
    CK(cudaMemcpyAsync(a.ac, &h, sizeof(AdmmCtrl), cudaMemcpyHostToDevice, ctx->stream));
    const AdmmRows rows = admm_rows(ctx, ld, sh, ctx->stream);
    admm_enqueue_block<TR, TW>(ctx, rows, X, V, const_cast<double*>(y), nullptr, cg_max);
    if ((s = check_launch(ctx, "lorads_admm_cg launch"))) return s;
    CK(cudaMemcpyAsync(a.h_ac, a.ac, sizeof(AdmmCtrl), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (steps_out) *steps_out = a.h_ac->cg_k;
    if (a.h_ac->status == LORADS_ERR_NUMERIC) return set_err(ctx, "non-finite CG residual"), LORADS_ERR_NUMERIC;
    return LORADS_OK;
}

lorads_status check_admm_factors(lorads_ctx* ctx, int32_t r, int32_t ld, int32_t prec, double rho, Shape* sh) {
    lorads_status s = check_factor_args(ctx, r, ld, prec, sh);
    if (s) return s;
    if (prec != LORADS_FP64 && prec != LORADS_FP32)
        return set_err(ctx, "prec must be LORADS_FP64 or LORADS_FP32"), LORADS_ERR_INVALID_ARG;
    if (!(rho > 0.0) || !std::isfinite(rho)) return set_err(ctx, "rho must be finite and > 0"), LORADS_ERR_INVALID_ARG;
    return LORADS_OK;
}

}  // namespace

extern "C" lorads_status lorads_admm_operator(lorads_ctx* ctx, const void* V, const void* X, int32_t r, int32_t ld,
                                              double rho, void* out, int32_t prec) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    Shape sh;
    lorads_status s = check_admm_factors(ctx, r, ld, prec, rho, &sh);
    if (s) return s;
    if (!V || !X || !out || !aligned16(V) || !aligned16(X) || !aligned16(out))
        return set_err(ctx, "V, X and out must be 16-byte aligned device pointers"), LORADS_ERR_INVALID_ARG;
    if (out == V || out == X) return set_err(ctx, "out must alias neither V nor X"), LORADS_ERR_INVALID_ARG;
    if (ctx->pd.k_ptr != nullptr)
        return set_err(ctx, "the ADMM operator takes constraints of one triplet each"), LORADS_ERR_UNSUPPORTED;
    const AdmmRows rows = admm_rows(ctx, ld, sh, ctx->stream);
    if (prec == LORADS_FP64)
        admm_op<double, double>(rows, V, nullptr, const_cast<void*>(X), out, nullptr, rho, 0, part_of(ctx, PART_MISC),
                                nullptr, nullptr);
    else
        admm_op<float, float>(rows, V, nullptr, const_cast<void*>(X), out, nullptr, rho, 0, part_of(ctx, PART_MISC),
                              nullptr, nullptr);
    return check_launch(ctx, "lorads_admm_operator launch");
}

extern "C" lorads_status lorads_admm_cg(lorads_ctx* ctx, const void* V, void* X, const double* y, double rho,
                                        int32_t r, int32_t ld, double cg_rel, int32_t cg_max, int32_t* steps_out,
                                        int32_t prec) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    Shape sh;
    lorads_status s = check_admm_factors(ctx, r, ld, prec, rho, &sh);
    if (s) return s;
    if (!V || !X || !y || !aligned16(V) || !aligned16(X))
        return set_err(ctx, "V, X (16-byte aligned) and y must be device pointers"), LORADS_ERR_INVALID_ARG;
    if (V == X) return set_err(ctx, "X must not alias V"), LORADS_ERR_INVALID_ARG;
    if (!(cg_rel > 0.0 && cg_rel < 1.0) || cg_max < 1)
        return set_err(ctx, "need 0 < cg_rel < 1 and cg_max >= 1"), LORADS_ERR_INVALID_ARG;
    if (prec == LORADS_FP64) return run_admm_cg<double, double>(ctx, V, X, y, rho, ld, sh, cg_rel, cg_max, steps_out);
    return run_admm_cg<float, float>(ctx, V, X, y, rho, ld, sh, cg_rel, cg_max, steps_out);
}

extern "C" lorads_status lorads_admm_stage(lorads_ctx* ctx, const double* R0, int32_t r0, int32_t r0_on_device,
                                           const double* y0, double rho, lorads_result* res) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    if (res) std::memset(res, 0, sizeof(*res));
    if (R0 && r0 < 1) return set_err(ctx, "r0 must be >= 1 when R0 is given"), LORADS_ERR_INVALID_ARG;
    if (!(rho > 0.0) || !std::isfinite(rho)) return set_err(ctx, "rho must be finite and > 0"), LORADS_ERR_INVALID_ARG;
    const int prec = ctx->prm.prec;
    lorads_status s;
    switch (prec) {
        case LORADS_FP64: s = run_stage<double, double>(ctx, prec, R0, r0, r0_on_device, y0, rho, res); break;
        case LORADS_MIXED: s = run_stage<dfloat, float>(ctx, prec, R0, r0, r0_on_device, y0, rho, res); break;
        case LORADS_DF64: s = run_stage<dfloat, dfloat>(ctx, prec, R0, r0, r0_on_device, y0, rho, res); break;
        case LORADS_FP32: s = run_stage<float, float>(ctx, prec, R0, r0, r0_on_device, y0, rho, res); break;
        case LORADS_MIXED_BF16:
            s = run_stage<dfloat, float, __nv_bfloat16>(ctx, prec, R0, r0, r0_on_device, y0, rho, res);
            break;
        default:
            return set_err(ctx, "params.prec must be FP64, MIXED, DF64, FP32 or MIXED_BF16"), LORADS_ERR_INVALID_ARG;
    }
    return finish_err2(ctx, s, res);
}

extern "C" lorads_status lorads_get_solution(lorads_ctx* ctx, double* R_host, int64_t R_capacity, int32_t* rank_out,
                                             double* y_host) {
    if (!ctx) return LORADS_ERR_INVALID_ARG;
    SolverState& st = ctx->st;
    if (!st.have_solution) return set_err(ctx, "no solution: call lorads_solve first"), LORADS_ERR_INVALID_ARG;
    if (rank_out) *rank_out = st.r;
    cudaStream_t s = ctx->solve_stream;
    if (R_host) {
        if (R_capacity < ctx->n * (int64_t)st.r) return set_err(ctx, "R_host too small"), LORADS_ERR_INVALID_ARG;
        double* tmp = nullptr;
        lorads_status rs;
        if ((rs = dalloc(ctx, &tmp, (size_t)ctx->n * st.r))) return rs;
        const int nbk = flat_blocks(ctx, ctx->n * (int64_t)st.r);
        if (st.rtype == 0) convert<double, double>(s, ctx->n, st.ld, st.r, st.r, st.R, tmp, nbk);
        else if (st.rtype == 1) convert<dfloat, double>(s, ctx->n, st.ld, st.r, st.r, st.R, tmp, nbk);
        else convert<float, double>(s, ctx->n, st.ld, st.r, st.r, st.R, tmp, nbk);
        CK(cudaMemcpyAsync(R_host, tmp, (size_t)ctx->n * st.r * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        cudaFree(tmp);
    }
    if (y_host) {
        CK(cudaMemcpyAsync(y_host, st.y, ctx->m * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return LORADS_OK;
}

// ============================================================== dual slack eigenvalue
namespace {

// sigma_min(C - A*(y)) by a k-step Lanczos run (no reorthogonalisation: the
// smallest Ritz value converges first and bounds sigma_min from above).
lorads_status run_lanczos(lorads_ctx* ctx, const double* ydev, int k, uint64_t seed, double* sigma_out) {
    const int64_t n = ctx->n;
    k = (int)std::max<int64_t>(1, std::min<int64_t>(k, n));
    cudaStream_t s = ctx->solve_stream;
    double *buf = nullptr, *lz = nullptr;
    lorads_status rs;
    if ((rs = dalloc(ctx, &buf, (size_t)3 * n * 4))) return rs;
    if ((rs = dalloc(ctx, &lz, (size_t)2 * k + 8))) { cudaFree(buf); return rs; }
    double* v = buf;
    double* vp = buf + (size_t)n * 4;
    double* w = buf + (size_t)2 * n * 4;
    CK(cudaMemsetAsync(buf, 0, (size_t)3 * n * 4 * sizeof(double), s));
    CK(cudaMemsetAsync(lz, 0, ((size_t)2 * k + 8) * sizeof(double), s));
    const int beta_off = k, sc = 2 * k + 2;
    Shape sh;
    shape_for_ld(4, &sh);
    const int nbf = flat_blocks(ctx, n), nbr = row_blocks(ctx, n, sh.L);
    double* part = part_of(ctx, PART_MISC);
    lz_random(s, n, seed, v, part, nbf);
    lz_scalar(s, part, nbf, lz, sc, 1);
    lz_scale(s, n, v, lz, sc, nbf);
    for (int j = 0; j < k; ++j) {
        SpmmCArgs a{ctx->pd, v, w, 4, sh, ydev, 1, EPI_NONE, nullptr, nullptr, nullptr, nullptr, nullptr, 0.0,
                    nullptr, nbr, nullptr, PH_ALWAYS, s};
        launch_spmm_c<double, double, double>(a);
        if (ctx->m_off) {
            SpmmAArgs aa{ctx->pd, v, w, 4, sh, ydev, -1.0, 1, nbr, nullptr, PH_ALWAYS, s};
            launch_spmm_a<double, double>(aa);
        }
        lz_dot(s, n, w, v, part, nbf);
        lz_scalar(s, part, nbf, lz, j, 0);                                  // alpha_j
        lz_orth(s, n, w, v, vp, lz, j, j > 0 ? beta_off + j : -1, part, nbf);
        lz_scalar(s, part, nbf, lz, beta_off + j + 1, 1);                   // beta_{j+1}
        if (j + 1 < k) {
            lz_scale(s, n, w, lz, beta_off + j + 1, nbf);
            double* t = vp;
            vp = v;
            v = w;
            w = t;
        }
    }
    lz_tridiag_min(s, lz, k, beta_off, lz + sc + 1);
    ctx->launches += 4 + (int64_t)k * (ctx->m_off ? 6 : 5) + (k - 1);
    lorads_status cs = check_launch(ctx, "lanczos");
    if (cs == LORADS_OK) {
        cudaError_t e = cudaMemcpyAsync(sigma_out, lz + sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            ctx->err = std::string("lanczos: ") + cudaGetErrorString(e);
            cs = LORADS_ERR_CUDA;
        }
    }
    cudaFree(buf);
    cudaFree(lz);
    return cs;
}

}  // namespace

extern "C" lorads_status lorads_dual_min_eig(lorads_ctx* ctx, const double* y, int32_t steps, uint64_t seed,
                                             double* sigma_out) {
    if (!ctx || !sigma_out || steps < 1) return LORADS_ERR_INVALID_ARG;
    const double* ydev = y;
    if (!ydev) {
        if (!ctx->st.have_solution) return set_err(ctx, "y is NULL and no solution is stored"), LORADS_ERR_INVALID_ARG;
        ydev = ctx->st.y;
    }
    CK(cudaEventRecord(ctx->ev_sync, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->solve_stream, ctx->ev_sync, 0));
    return run_lanczos(ctx, ydev, steps, seed, sigma_out);
}

extern "C" lorads_status lorads_set_iteration_limit(lorads_ctx* ctx, int64_t max_total_inner) {
    if (!ctx || max_total_inner < 0) return LORADS_ERR_INVALID_ARG;
    ctx->iter_limit = max_total_inner;
    return LORADS_OK;
}

extern "C" int32_t lorads_kernel_times(const lorads_ctx* ctx, const char** names, double* ms, int32_t cap) {
    if (!ctx || !ctx->prof || !ctx->prof_valid) return 0;
    int32_t k = 0;
    for (int f = 0; f < NFAM && k < cap; ++f) {
        if (ctx->prof->count[f] == 0) continue;
        if (names) names[k] = kFamNames[f];
        if (ms) ms[k] = ctx->prof->total_ms[f] / (double)ctx->prof->count[f];
        ++k;
    }
    return k;
}

extern "C" int32_t lorads_kernel_counts(const lorads_ctx* ctx, const char** names, int64_t* counts, int32_t cap) {
    if (!ctx || !ctx->prof || !ctx->prof_valid) return 0;
    int32_t k = 0;
    for (int f = 0; f < NFAM && k < cap; ++f) {
        if (ctx->prof->count[f] == 0) continue;
        if (names) names[k] = kFamNames[f];
        if (counts) counts[k] = ctx->prof->count[f];
        ++k;
    }
    return k;
}
