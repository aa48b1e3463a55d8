// Batched persistent solve: many independent SDP instances (Eq. (1.1)) in one
// kernel launch.  Each block of the launch takes the next instance from a
// device work queue and runs the complete solve on it -- the ALM outer loop of
// Sec. 2.1, the L-BFGS inner loop of Algorithm 1 with the exact line search of
// App. A.2 and the rank rule of App. A.1 -- with the same kernel bodies and the
// same scalar decisions (control_dev.cuh) as the single-instance solve, run by
// one block with block-wide reductions instead of one launch per step.  Its
// control block lives in shared memory for the whole solve.
//
// Layout: all problem arrays of all instances in one device pool, all iterates
// in a second pool; each instance owns n x ld_cap slots per factor array
// (ld_cap: the width after two rank updates), so a rank update re-lays the
// rows in place without allocating.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lorads.h"
#include "batch_kernel.cuh"
#include "prob_host.h"

using namespace lorads;
using namespace lorads::batch;

namespace {

// ------------------------------------------------------------------ host side
size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

int ceil_log2(int64_t m) {
    int r = 0;
    while (((int64_t)1 << r) < m) ++r;
    return std::max(r, 1);
}

}  // namespace

struct lorads_batch {
    int count = 0;
    lorads_params prm{};
    int prec = LORADS_FP64;
    size_t esR = 8, esD = 8;
    cudaStream_t stream = nullptr;          // caller's
    cudaStream_t solve_stream = nullptr;    // owned, capture-capable
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int device = 0, num_sms = 0;
    std::string err;
    char* prob_pool = nullptr;
    char* state_pool = nullptr;
    BInst* d_inst = nullptr;
    Ctrl* d_ctrl0 = nullptr;
    BOut* d_out = nullptr;
    int* d_order = nullptr;                 // [2][count]: input order, largest first
    int* d_queue = nullptr;
    std::vector<BInst> h_inst;
    std::vector<BOut> h_out;
    std::vector<int64_t> n, m;
    std::vector<double> cnorm1;
    lorads_batch_shape shape{2, 8, 1, 256, 1, 0};
    int64_t iter_limit = 0;
    cudaGraphExec_t exec = nullptr;
    lorads_batch_shape exec_shape{0, 0, 0, 0};
    int64_t exec_limit = -1;
    bool have_solution = false;
};

namespace {

#define BCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return LORADS_ERR_CUDA;                                                        \
        }                                                                                  \
    } while (0)

void* kernel_for(int prec) {
    switch (prec) {
        case LORADS_FP64: return kernel_fp64();
        case LORADS_MIXED: return kernel_mixed();
        default: return kernel_fp32();
    }
}

// Writes the per-instance control blocks of a fresh solve (as lorads_solve does).
void fill_ctrl0(const lorads_params& P, const HostProb& hp, int64_t iter_limit, Ctrl* h) {
    std::memset(h, 0, sizeof(Ctrl));
    h->rho = P.rho0 > 0 ? P.rho0 : 1.0 / hp.mean_abs_c;
    h->lbfgs_mem = P.lbfgs_mem;
    h->total_limit = iter_limit > 0 ? (int)std::min<int64_t>(iter_limit, INT32_MAX) : 0;
    h->max_inner = P.max_inner;
    h->max_outer = P.max_outer;
    h->rank_threshold = std::max(1, P.rank_update_threshold);
    h->lbfgs_scaling = P.lbfgs_scaling;
    h->rho_policy = P.rho_policy;
    h->inner_scale = P.inner_scale;
    // two-stage solve: the ALM stage stops at the switch tolerance
    h->tol = P.admm_switch > 0 ? std::max(P.admm_switch, P.tol) : P.tol;
    h->inner_rel = P.inner_rel;
    h->inner_progress = P.inner_progress;
    h->bnorm1 = hp.bnorm1;
    h->bnorm_inf = hp.bnorm_inf;
    h->rho_growth = P.rho_growth;
    h->rho_max = P.rho_max;
    h->infeas_decrease = P.infeas_decrease;
    h->status = LORADS_ERR_MAXITER;
    for (int q = 0; q < kMaxMem; ++q) h->order[q] = q;
}

int threads_of(const lorads_batch_shape& s) { return s.threads == 512 ? 512 : 256; }
int cluster_of(const lorads_batch_shape& s) { return s.cluster > 1 ? s.cluster : 1; }

// Grid of the launch: SMs x blocks per SM without clusters; with clusters, as
// many whole clusters as can be resident at once (a persistent kernel needs all
// its blocks resident: blocks of a cluster wait for one another).
lorads_status launch_grid(lorads_batch* b, const lorads_batch_shape& sh, int* grid, int* n_team) {
    const int cs = cluster_of(sh);
    if (cs == 1) {
        *grid = std::max(1, std::min(b->count, b->num_sms * sh.ctas_per_sm));
        *n_team = 0;
        return LORADS_OK;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs * 64);
    cfg.blockDim = dim3(threads_of(sh));
    cfg.dynamicSmemBytes = 0;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, kernel_for(b->prec), &cfg);
    if (e != cudaSuccess || nclusters < 1) {
        cudaGetLastError();
        b->err = std::string("cluster size ") + std::to_string(cs) + " cannot be resident: " +
                 (e != cudaSuccess ? cudaGetErrorString(e) : "no cluster fits");
        return LORADS_ERR_UNSUPPORTED;
    }
    // ctas_per_sm bounds the clusters as it bounds plain blocks
    nclusters = std::min(nclusters, std::max(1, b->num_sms * sh.ctas_per_sm / cs));
    *grid = nclusters * cs;
    *n_team = std::min(b->count, std::max(0, sh.team_count));
    return LORADS_OK;
}

lorads_status capture_batch(lorads_batch* b) {
    if (b->exec && std::memcmp(&b->exec_shape, &b->shape, sizeof(lorads_batch_shape)) == 0 &&
        b->exec_limit == b->iter_limit)
        return LORADS_OK;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    int grid = 0, n_team = 0;
    lorads_status gs = launch_grid(b, b->shape, &grid, &n_team);
    if (gs != LORADS_OK) return gs;
    const int* order = b->d_order + (b->shape.order ? b->count : 0);
    const long long tl = b->prm.time_limit > 0 ? (long long)std::min(b->prm.time_limit * 1e9, 9.0e18) : 0;
    const BInst* insts = b->d_inst;
    const Ctrl* ctrl0 = b->d_ctrl0;
    BOut* out = b->d_out;
    int count = b->count;
    int* queues = b->d_queue;
    int rpw = b->shape.rows_per_warp;
    void* args[] = {(void*)&insts, (void*)&ctrl0, (void*)&out, (void*)&order, (void*)&count, (void*)&n_team,
                    (void*)&queues, (void*)&rpw, (void*)const_cast<long long*>(&tl)};
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->solve_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(int), b->solve_stream);
    cudaError_t e2;
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(threads_of(b->shape));
        cfg.dynamicSmemBytes = 0;
        cfg.stream = b->solve_stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster_of(b->shape);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e2 = cudaLaunchKernelExC(&cfg, kernel_for(b->prec), args);
    }
    cudaError_t e3 = cudaStreamEndCapture(b->solve_stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        b->err = std::string("batch capture: ") +
                 cudaGetErrorString(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3));
        return LORADS_ERR_CUDA;
    }
    cudaError_t e4 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e4 != cudaSuccess) {
        b->exec = nullptr;
        b->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e4);
        return LORADS_ERR_CUDA;
    }
    b->exec_shape = b->shape;
    b->exec_limit = b->iter_limit;
    return LORADS_OK;
}

int max_ctas_per_sm(int prec, int threads) {
    int nb = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_for(prec), threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, std::min(nb, 4));
}

lorads_status set_iter_limit(lorads_batch* b, int64_t lim) {
    if (lim == b->iter_limit) return LORADS_OK;
    b->iter_limit = lim;
    const int L = lim > 0 ? (int)std::min<int64_t>(lim, INT32_MAX) : 0;
    std::vector<Ctrl> h(b->count);
    BCK(cudaMemcpy(h.data(), b->d_ctrl0, sizeof(Ctrl) * b->count, cudaMemcpyDeviceToHost));
    for (auto& c : h) c.total_limit = L;
    BCK(cudaMemcpy(b->d_ctrl0, h.data(), sizeof(Ctrl) * b->count, cudaMemcpyHostToDevice));
    return LORADS_OK;
}

lorads_status run_batch(lorads_batch* b, lorads_result* results, lorads_batch_stats* stats) {
    lorads_status s = capture_batch(b);
    if (s != LORADS_OK) return s;
    BCK(cudaEventRecord(b->ev0, b->solve_stream));
    BCK(cudaGraphLaunch(b->exec, b->solve_stream));
    BCK(cudaEventRecord(b->ev1, b->solve_stream));
    BCK(cudaStreamSynchronize(b->solve_stream));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    BCK(cudaMemcpy(b->h_out.data(), b->d_out, sizeof(BOut) * b->count, cudaMemcpyDeviceToHost));
    b->have_solution = true;
    long long t0 = 0;
    bool first = true;
    for (const BOut& o : b->h_out)
        if (first || o.t_begin < t0) { t0 = o.t_begin; first = false; }
    std::vector<double> lat(b->count);
    int64_t inner = 0;
    int solved = 0;
    for (int i = 0; i < b->count; ++i) {
        const BOut& o = b->h_out[i];
        const Ctrl& c = o.ctrl;
        lat[i] = (double)(o.t_end - t0) * 1e-6;
        inner += c.total_inner;
        solved += c.status == LORADS_OK;
        if (results) {
            lorads_result& r = results[i];
            std::memset(&r, 0, sizeof(r));
            r.primal_obj = c.primal_obj;
            r.dual_obj = c.dual_obj;
            r.err1 = c.err1;
            r.err2 = -1.0;
            r.err3 = c.err3;
            r.rho = c.rho;
            r.seconds = (double)(o.t_end - o.t_begin) * 1e-9;
            r.rank = o.r;
            r.outer_iters = c.outer;
            r.inner_iters = c.total_inner;
            r.status = c.status;
            r.kernel_launches = 1;
            r.admm_iters = o.admm_iters;
            r.cg_steps = o.cg_steps;
            r.reopt_scale = 1.0;
        }
    }
    if (stats) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double q) {
            const size_t k = (size_t)std::min<double>(lat.size() - 1, std::ceil(q * lat.size()) - 1);
            return lat[k];
        };
        stats->seconds = ms * 1e-3;
        stats->instances_per_s = ms > 0 ? b->count / (ms * 1e-3) : 0.0;
        stats->latency_p50_ms = pct(0.50);
        stats->latency_p99_ms = pct(0.99);
        stats->latency_max_ms = lat.back();
        stats->inner_iters = inner;
        stats->solved = solved;
        int grid = 0, n_team = 0;
        launch_grid(b, b->shape, &grid, &n_team);
        stats->grid = grid;
        stats->shape = b->shape;
    }
    return LORADS_OK;
}

bool valid_shape(const lorads_batch_shape& s) {
    const int r = s.rows_per_warp;
    const int c = s.cluster;
    return s.ctas_per_sm >= 1 && s.ctas_per_sm <= 4 && (r == 1 || r == 2 || r == 4 || r == 8) &&
           (s.order == 0 || s.order == 1) && (s.threads == 0 || s.threads == 256 || s.threads == 512) &&
           (c == 0 || c == 1 || c == 2 || c == 4 || c == 8) && s.team_count >= 0;
}

void free_batch(lorads_batch* b) {
    if (b->solve_stream) cudaStreamSynchronize(b->solve_stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->prob_pool) cudaFree(b->prob_pool);
    if (b->state_pool) cudaFree(b->state_pool);
    if (b->d_inst) cudaFree(b->d_inst);
    if (b->d_ctrl0) cudaFree(b->d_ctrl0);
    if (b->d_out) cudaFree(b->d_out);
    if (b->d_order) cudaFree(b->d_order);
    if (b->d_queue) cudaFree(b->d_queue);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->solve_stream) cudaStreamDestroy(b->solve_stream);
    delete b;
}

thread_local std::string g_batch_create_error;

}  // namespace

extern "C" const char* lorads_batch_last_error(const lorads_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" void lorads_batch_destroy(lorads_batch* b) {
    if (b) free_batch(b);
}

extern "C" lorads_status lorads_batch_create(lorads_batch** out, int32_t count, const int64_t* n_in,
                                             const int64_t* m_in, const int64_t* c_rowptr, const int32_t* c_colind,
                                             const double* c_val, const int32_t* a_con, const int32_t* a_row,
                                             const int32_t* a_col, const double* a_val, const double* b_in,
                                             const int32_t* r0_in, const double* R0, const lorads_params* p,
                                             void* cuda_stream) {
    if (!out) return LORADS_ERR_INVALID_ARG;
    *out = nullptr;
    auto fail = [&](lorads_status s, const std::string& msg) {
        g_batch_create_error = msg;
        return s;
    };
    if (count < 1) return fail(LORADS_ERR_INVALID_ARG, "count must be >= 1");
    if (!n_in || !m_in || !c_rowptr || !c_colind || !c_val || !a_con || !a_row || !a_col || !a_val || !b_in)
        return fail(LORADS_ERR_INVALID_ARG, "null input pointer");
    lorads_params P;
    if (p) P = *p;
    else lorads_default_params(&P);
    if (P.prec != LORADS_FP64 && P.prec != LORADS_MIXED && P.prec != LORADS_FP32)
        return fail(LORADS_ERR_INVALID_ARG, "batch prec must be LORADS_FP64, LORADS_MIXED or LORADS_FP32");
    {
        const std::string perr = solver_params_error(P);
        if (!perr.empty()) return fail(LORADS_ERR_INVALID_ARG, perr);
    }
    const size_t esR = P.prec == LORADS_FP64 ? 8 : (P.prec == LORADS_MIXED ? 8 : 4);
    const size_t esD = P.prec == LORADS_FP64 ? 8 : 4;
    const bool fp64 = P.prec == LORADS_FP64;
    // ---- validate every instance and lay out the two pools
    std::vector<HostProb> hp(count);
    std::vector<int> r0(count), ldcap(count), rcap(count);
    std::vector<size_t> prob_off(count + 1, 0), state_off(count + 1, 0);
    int64_t rp_at = 0, nnz_at = 0, k_at = 0, r0_at = 0;
    std::vector<int64_t> rp_start(count), nnz_start(count), k_start(count), r0_start(count);
    for (int i = 0; i < count; ++i) {
        const int64_t n = n_in[i], m = m_in[i];
        if (n < 1 || m < 1) return fail(LORADS_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": n, m must be >= 1");
        rp_start[i] = rp_at;
        nnz_start[i] = nnz_at;
        k_start[i] = k_at;
        const int64_t* rp = c_rowptr + rp_at;
        const int64_t nnz = rp[n];
        if (nnz < 0) return fail(LORADS_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": bad row pointers");
        std::string e;
        lorads_status s = build_host_prob(&hp[i], &e, n, rp, c_colind + nnz_at, c_val + nnz_at, m, m, a_con + k_at,
                                          a_row + k_at, a_col + k_at, a_val + k_at, b_in + k_at);
        if (s != LORADS_OK) return fail(s, "instance " + std::to_string(i) + ": " + e);
        if (!hp[i].k_ptr.empty())
            return fail(LORADS_ERR_UNSUPPORTED, "instance " + std::to_string(i) + ": several constraints on one "
                        "entry (the general form) is solved by lorads_solve, not by the batched solve");
        rp_at += n + 1;
        nnz_at += nnz;
        k_at += m;
        r0[i] = r0_in ? r0_in[i] : ceil_log2(m);
        rcap[i] = (int)std::ceil(std::sqrt(2.0 * (double)m));
        if (r0[i] < 1 || r0[i] > kBatchLdMax)
            return fail(LORADS_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": r0 must be in [1, 128]");
        r0_start[i] = r0_at;
        if (R0) r0_at += n * r0[i];
        int rc = std::max(r0[i], std::min(rcap[i], (int)std::ceil(1.5 * std::ceil(1.5 * r0[i]))));
        ldcap[i] = std::min(kBatchLdMax, (rc + 3) / 4 * 4);
        rcap[i] = std::max(rcap[i], r0[i]);
        // problem pool
        const HostProb& h = hp[i];
        size_t ps = 0;
        ps += align_up((n + 1) * 8) + align_up(nnz * 4) + align_up(nnz * 8) + align_up(nnz * 4) + align_up(nnz * 8);
        if (h.m_diag) ps += align_up(n * 4) + align_up(n * 8) + align_up(n * 4) + align_up(n * 8);
        ps += align_up(m * 8);                                             // b_df
        if (h.m_off) ps += align_up((n + 1) * 8) + 2 * align_up(h.a_col.size() * 4) + align_up(h.a_a.size() * 8);
        ps += 3 * align_up(m * 4) + align_up(m * 8) + align_up(m * 8);    // k_row/col/id, k_a, b
        ps += align_up(m * 8);                                             // k_a double-float mirror
        if (h.m_off) ps += align_up(h.a_a.size() * 8);                     // a_a double-float mirror
        if (R0) ps += align_up(n * r0[i] * 8);
        prob_off[i + 1] = prob_off[i] + ps;
        // state pool
        const size_t nl = (size_t)n * ldcap[i];
        size_t ss = 2 * align_up(nl * esR) + 3 * align_up(nl * esD) + align_up(nl * esD * 2 * P.lbfgs_mem);
        if (h.m_off) ss += align_up(nl * esD) + 2 * align_up(m * 8);
        ss += align_up(m * 8) + align_up(n * 8);                           // y, zrow
        if (!fp64) ss += align_up(m * 8);                                  // ydf
        if (P.admm_switch > 0) ss += 2 * align_up(nl * esR) + align_up(m * 8);   // U, V, w (ADMM stage)
        state_off[i + 1] = state_off[i] + ss;
    }
    lorads_batch* b = new (std::nothrow) lorads_batch();
    if (!b) return fail(LORADS_ERR_OOM, "host allocation");
    b->count = count;
    b->prm = P;
    b->prec = P.prec;
    b->esR = esR;
    b->esD = esD;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    auto bail = [&](lorads_status s) {
        g_batch_create_error = b->err;
        free_batch(b);
        return s;
    };
#define BCREATE(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
            return bail(e_ == cudaErrorMemoryAllocation ? LORADS_ERR_OOM : LORADS_ERR_CUDA); \
        }                                                                                  \
    } while (0)
    BCREATE(cudaGetDevice(&b->device));
    BCREATE(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
    BCREATE(cudaStreamCreateWithFlags(&b->solve_stream, cudaStreamNonBlocking));
    BCREATE(cudaEventCreate(&b->ev0));
    BCREATE(cudaEventCreate(&b->ev1));
    BCREATE(cudaMalloc(&b->prob_pool, std::max<size_t>(prob_off[count], 256)));
    BCREATE(cudaMalloc(&b->state_pool, std::max<size_t>(state_off[count], 256)));
    BCREATE(cudaMemset(b->state_pool, 0, std::max<size_t>(state_off[count], 256)));
    // ---- stage the problem pool on the host, upload once
    std::vector<char> stage(prob_off[count]);
    b->h_inst.resize(count);
    b->h_out.resize(count);
    b->n.resize(count);
    b->m.resize(count);
    b->cnorm1.resize(count);
    std::vector<Ctrl> ctrl0(count);
    std::vector<double> work(count);
    for (int i = 0; i < count; ++i) {
        const HostProb& h = hp[i];
        const int64_t n = h.n, m = h.m, nnz = h.nnz_c;
        size_t at = prob_off[i];
        auto put = [&](const void* src, size_t bytes) -> void* {
            if (bytes) std::memcpy(stage.data() + at, src, bytes);
            void* dev = b->prob_pool + at;
            at += align_up(bytes);
            return dev;
        };
        ProbDev pd{};
        pd.n = n;
        pd.m = m;
        pd.c_rowptr = static_cast<const int64_t*>(put(h.rp, (n + 1) * 8));
        pd.c_col = static_cast<const int32_t*>(put(h.ci, nnz * 4));
        pd.c_val = static_cast<const double*>(put(h.cv, nnz * 8));
        pd.c_val32 = static_cast<const float*>(put(h.cv32.data(), nnz * 4));
        pd.c_valdf = static_cast<const dfloat*>(put(h.cvdf.data(), nnz * 8));
        if (h.m_diag) {
            pd.dk = static_cast<const int32_t*>(put(h.dk.data(), n * 4));
            pd.da = static_cast<const double*>(put(h.da.data(), n * 8));
            pd.da32 = static_cast<const float*>(put(h.da32.data(), n * 4));
            pd.da_df = static_cast<const dfloat*>(put(h.dadf.data(), n * 8));
        }
        pd.b_df = static_cast<const dfloat*>(put(h.bdf.data(), m * 8));
        if (h.m_off) {
            pd.a_rowptr = static_cast<const int64_t*>(put(h.a_rp.data(), (n + 1) * 8));
            pd.a_col = static_cast<const int32_t*>(put(h.a_col.data(), h.a_col.size() * 4));
            pd.a_k = static_cast<const int32_t*>(put(h.a_k.data(), h.a_k.size() * 4));
            pd.a_a = static_cast<const double*>(put(h.a_a.data(), h.a_a.size() * 8));
        }
        pd.k_row = static_cast<const int32_t*>(put(h.k_row.data(), m * 4));
        pd.k_col = static_cast<const int32_t*>(put(h.k_col.data(), m * 4));
        pd.k_id = static_cast<const int32_t*>(put(h.k_id.data(), m * 4));
        pd.k_a = static_cast<const double*>(put(h.k_a.data(), m * 8));
        pd.b = static_cast<const double*>(put(h.b, m * 8));
        pd.k_adf = static_cast<const dfloat*>(put(h.k_adf.data(), m * 8));
        if (h.m_off) pd.a_adf = static_cast<const dfloat*>(put(h.a_adf.data(), h.a_adf.size() * 8));
        pd.m_diag = h.m_diag;
        pd.m_off = h.m_off;
        BInst& I = b->h_inst[i];
        std::memset(&I, 0, sizeof(I));
        I.p = pd;
        I.R0 = R0 ? static_cast<const double*>(put(R0 + r0_start[i], n * r0[i] * 8)) : nullptr;
        // iterate
        char* sa = b->state_pool + state_off[i];
        const size_t nl = (size_t)n * ldcap[i];
        auto take = [&](size_t bytes) -> void* {
            void* d = sa;
            sa += align_up(bytes);
            return d;
        };
        I.R = take(nl * esR);
        I.CR = take(nl * esR);
        I.D = take(nl * esD);
        I.CD = take(nl * esD);
        I.G = take(nl * esD);
        I.hist = take(nl * esD * 2 * P.lbfgs_mem);
        if (h.m_off) {
            I.W = take(nl * esD);
            I.ytil = static_cast<double*>(take(m * 8));
            I.zk = static_cast<double*>(take(m * 8));
        }
        I.y = static_cast<double*>(take(m * 8));
        I.zrow = take(n * 8);
        if (!fp64) I.ydf = static_cast<dfloat*>(take(m * 8));
        if (P.admm_switch > 0) {
            I.U = take(nl * esR);
            I.V = take(nl * esR);
            I.om = take(m * 8);
            I.admm_on = 1;
            I.admm_tol = P.tol;
            I.cg_rel = P.cg_rel;
            I.cg_max = P.cg_max;
            I.admm_max_iter = P.admm_max_iter;
        }
        I.slot_stride = (int64_t)nl;
        I.r0 = r0[i];
        I.ld_cap = ldcap[i];
        I.r_cap = rcap[i];
        I.unit_rows = h.m_diag == h.m ? 1 : 0;
        I.start_scale = std::sqrt(std::max(0.5 * h.bnorm1, 1.0) / ((double)n * r0[i]));
        I.seed = P.seed;
        b->n[i] = n;
        b->m[i] = m;
        b->cnorm1[i] = h.cnorm1;
        fill_ctrl0(P, h, 0, &ctrl0[i]);
        const int ld0 = (r0[i] + 3) / 4 * 4;
        work[i] = (double)(nnz + 2 * h.m_off + n) * ld0 + (double)n * ld0 * (2 * P.lbfgs_mem + 12);
    }
    BCREATE(cudaMemcpy(b->prob_pool, stage.data(), stage.size(), cudaMemcpyHostToDevice));
    BCREATE(cudaMalloc(&b->d_inst, sizeof(BInst) * count));
    BCREATE(cudaMemcpy(b->d_inst, b->h_inst.data(), sizeof(BInst) * count, cudaMemcpyHostToDevice));
    BCREATE(cudaMalloc(&b->d_ctrl0, sizeof(Ctrl) * count));
    BCREATE(cudaMemcpy(b->d_ctrl0, ctrl0.data(), sizeof(Ctrl) * count, cudaMemcpyHostToDevice));
    BCREATE(cudaMalloc(&b->d_out, sizeof(BOut) * count));
    BCREATE(cudaMemset(b->d_out, 0, sizeof(BOut) * count));
    std::vector<int> ord(2 * count);
    std::iota(ord.begin(), ord.begin() + count, 0);
    std::iota(ord.begin() + count, ord.end(), 0);
    std::stable_sort(ord.begin() + count, ord.end(), [&](int x, int y) { return work[x] > work[y]; });
    BCREATE(cudaMalloc(&b->d_order, sizeof(int) * 2 * count));
    BCREATE(cudaMemcpy(b->d_order, ord.data(), sizeof(int) * 2 * count, cudaMemcpyHostToDevice));
    BCREATE(cudaMalloc(&b->d_queue, 2 * sizeof(int)));
    b->shape.ctas_per_sm = std::min(2, max_ctas_per_sm(b->prec, 256));
#undef BCREATE
    *out = b;
    return LORADS_OK;
}

extern "C" lorads_status lorads_batch_solve(lorads_batch* b, lorads_result* results, lorads_batch_stats* stats) {
    if (!b) return LORADS_ERR_INVALID_ARG;
    if (b->stream) {
        // order after the caller's stream (inputs written there)
        cudaEvent_t e;
        BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        BCK(cudaEventRecord(e, b->stream));
        BCK(cudaStreamWaitEvent(b->solve_stream, e, 0));
        cudaEventDestroy(e);
    }
    return run_batch(b, results, stats);
}

extern "C" lorads_status lorads_batch_set_shape(lorads_batch* b, const lorads_batch_shape* shape) {
    if (!b || !shape) return LORADS_ERR_INVALID_ARG;
    if (!valid_shape(*shape)) {
        b->err = "shape: ctas_per_sm in [1,4], rows_per_warp in {1,2,4,8}, order 0 or 1, threads 256 or 512, "
                 "cluster 1, 2, 4 or 8, team_count >= 0";
        return LORADS_ERR_INVALID_ARG;
    }
    lorads_batch_shape sh = *shape;
    sh.threads = threads_of(sh);
    sh.cluster = cluster_of(sh);
    if (sh.cluster == 1) sh.team_count = 0;
    if (sh.ctas_per_sm > max_ctas_per_sm(b->prec, sh.threads)) {
        b->err = "shape: more blocks per SM than the kernel's occupancy allows";
        return LORADS_ERR_INVALID_ARG;
    }
    int grid = 0, n_team = 0;
    lorads_status gs = launch_grid(b, sh, &grid, &n_team);
    if (gs != LORADS_OK) return gs;
    b->shape = sh;
    return LORADS_OK;
}

extern "C" lorads_status lorads_batch_set_iteration_limit(lorads_batch* b, int64_t max_total_inner) {
    if (!b || max_total_inner < 0) return LORADS_ERR_INVALID_ARG;
    return set_iter_limit(b, max_total_inner);
}

extern "C" lorads_status lorads_batch_tune(lorads_batch* b, int32_t probe_iters, lorads_batch_shape* best) {
    if (!b || probe_iters < 1) return LORADS_ERR_INVALID_ARG;
    const int64_t keep_limit = b->iter_limit;
    const lorads_batch_shape keep = b->shape;
    lorads_status s = set_iter_limit(b, probe_iters);
    if (s != LORADS_OK) return s;
    double best_t = 1e300;
    lorads_batch_shape best_s = keep;
    auto probe = [&](const lorads_batch_shape& sh) -> lorads_status {
        int grid = 0, n_team = 0;
        if (launch_grid(b, sh, &grid, &n_team) != LORADS_OK) {
            cudaGetLastError();
            return LORADS_OK;                    // shape not launchable here: skip it
        }
        b->shape = sh;
        lorads_batch_stats st{};
        lorads_status rs = run_batch(b, nullptr, &st);
        if (rs != LORADS_OK) return rs;
        if (st.seconds < 0.97 * best_t) {        // a later candidate must win by 3% (timing noise)
            best_t = st.seconds;
            best_s = sh;
        }
        return LORADS_OK;
    };
    // one block per instance: threads x blocks per SM x rows per warp x order
    for (int threads : {256, 512})
        for (int order = 1; order >= 0; --order)
            for (int ctas = 1; ctas <= max_ctas_per_sm(b->prec, threads); ++ctas)
                for (int rpw : {8, 4, 2, 1})
                    if ((s = probe(lorads_batch_shape{ctas, rpw, order, threads, 1, 0})) != LORADS_OK) break;
    // clusters for the largest instances (largest first), on top of the best plain shape
    const lorads_batch_shape base = best_s;
    for (int cs : {2, 4, 8}) {
        if (s != LORADS_OK) break;
        const int nclusters = std::max(1, b->num_sms * base.ctas_per_sm / cs);
        for (int mult : {1, 2, 4}) {
            lorads_batch_shape sh = base;
            sh.order = 1;
            sh.cluster = cs;
            sh.team_count = std::min(b->count, nclusters * mult);
            if ((s = probe(sh)) != LORADS_OK) break;
        }
    }
    if (s != LORADS_OK) {
        b->shape = keep;
        set_iter_limit(b, keep_limit);
        return s;
    }
    b->shape = best_s;
    if (best) *best = best_s;
    b->have_solution = false;           // the probes' iterates are not solutions
    return set_iter_limit(b, keep_limit);
}

extern "C" lorads_status lorads_batch_get_solution(lorads_batch* b, int32_t i, double* R_host, int64_t R_capacity,
                                                   int32_t* rank_out, double* y_host) {
    if (!b || i < 0 || i >= b->count) return LORADS_ERR_INVALID_ARG;
    if (!b->have_solution) {
        b->err = "no solution: call lorads_batch_solve first";
        return LORADS_ERR_INVALID_ARG;
    }
    const BOut& o = b->h_out[i];
    const BInst& I = b->h_inst[i];
    const int64_t n = b->n[i], m = b->m[i];
    if (rank_out) *rank_out = o.r;
    if (R_host) {
        if (R_capacity < n * (int64_t)o.r) {
            b->err = "R_host too small";
            return LORADS_ERR_INVALID_ARG;
        }
        std::vector<char> raw((size_t)n * o.ld * b->esR);
        BCK(cudaMemcpy(raw.data(), I.R, raw.size(), cudaMemcpyDeviceToHost));
        for (int64_t r = 0; r < n; ++r)
            for (int c = 0; c < o.r; ++c) {
                const size_t e = (size_t)r * o.ld + c;
                double v;
                if (b->prec == LORADS_FP64) {
                    std::memcpy(&v, raw.data() + e * 8, 8);
                } else if (b->prec == LORADS_MIXED) {
                    float hl[2];
                    std::memcpy(hl, raw.data() + e * 8, 8);
                    v = (double)hl[0] + (double)hl[1];
                } else {
                    float f;
                    std::memcpy(&f, raw.data() + e * 4, 4);
                    v = f;
                }
                R_host[r * o.r + c] = v;
            }
    }
    if (y_host) BCK(cudaMemcpy(y_host, I.y, m * sizeof(double), cudaMemcpyDeviceToHost));
    return LORADS_OK;
}

extern "C" const char* lorads_batch_create_error(void) { return g_batch_create_error.c_str(); }

extern "C" int32_t lorads_batch_phase_times(const lorads_batch* b, int32_t i, const char** names, double* ms,
                                            int32_t cap) {
    static const char* const kNames[BP_N] = {"init", "direction", "spmm_ls", "cons_ls", "root", "step", "ytil",
                                             "spmm_a", "update", "hist", "outer", "outer_gradient", "rank_update",
                                             "admm"};
    if (!b || !b->have_solution || i < -1 || i >= b->count || cap < 1) return 0;
    const int k = std::min<int>(cap, BP_N);
    for (int q = 0; q < k; ++q) {
        double t = 0.0;
        for (int j = (i < 0 ? 0 : i); j < (i < 0 ? b->count : i + 1); ++j) t += (double)b->h_out[j].phase_ns[q];
        if (names) names[q] = kNames[q];
        if (ms) ms[q] = t * 1e-6;
    }
    return k;
}
