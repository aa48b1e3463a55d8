// Device side of the batched persistent solve (see batch.cu): the instance
// descriptor, the per-instance solve run by one block or one thread-block
// cluster, and the persistent kernel.  Included by one translation unit per
// precision so that the three instantiations compile in parallel.
#pragma once

#include <cooperative_groups.h>

#include "../../include/lorads.h"
#include "admm.cuh"
#include "common.cuh"
#include "control_dev.cuh"
#include "kernels.cuh"

namespace lorads {
namespace batch {

namespace cg = cooperative_groups;


// Device descriptor of one instance.
struct BInst {
    ProbDev p;
    void* R;
    void* CR;
    void* D;
    void* CD;
    void* G;
    void* W;                  // A*_off(y~) R (off-diagonal constraints only)
    void* hist;               // 2T slots of n x ld_cap: S_u, Y_u
    void* zrow;               // z of the diagonal constraint of each row
    double* y;
    double* ytil;             // y~ of the off-diagonal constraints
    double* zk;               // z of the off-diagonal constraints
    dfloat* ydf;              // double-float mirror of y (FP32-unit precisions)
    const double* R0;         // FP64 starting factor (n x r0) or null
    int64_t slot_stride;      // n * ld_cap
    int r0, ld_cap, r_cap, unit_rows;
    double start_scale;
    uint64_t seed;
    // splitting ADMM stage (Sec. 2.2) after the ALM stage (admm_on): block iterates
    // U, V (n x ld_cap, type of R), the m-vector w, the final tolerance and CG limits
    void* U;
    void* V;
    void* om;
    int admm_on, cg_max, admm_max_iter;
    double admm_tol, cg_rel;
};

// Per-instance result written by the kernel.
// phases of the per-instance solve timed by the persistent kernel
enum { BP_INIT = 0, BP_DIR, BP_LS, BP_CONS_LS, BP_ROOT, BP_STEP, BP_YTIL, BP_SPMM_A, BP_UPDATE, BP_HIST, BP_OUTER,
       BP_GRAD, BP_RANK, BP_ADMM, BP_N };

struct BOut {
    Ctrl ctrl;
    int r, ld;
    int admm_iters, cg_steps;
    long long t_begin, t_end;     // %globaltimer (ns)
    long long phase_ns[BP_N];     // time of each phase (thread 0 of the block, after its barrier)
};

// shared-memory slots of the reduced sums (one block: the partial is the sum)
// (SP_CONS, SP_OBJ, SP_TIME are adjacent: the outer step reduces them together)
enum { SP_DIR = 0, SP_LS = 2, SP_CLS = 9, SP_UPD = 16, SP_CONS = 30, SP_OBJ = 32, SP_TIME = 33, SP_YT = 34,
       SP_ZERO = 40, SP_MISC = 48, SP_N = 56 };
static_assert(SP_LS - SP_DIR >= PD_N && SP_CLS - SP_LS >= PL_N && SP_UPD - SP_CLS >= PL_N &&
                  SP_CONS - SP_UPD >= PU_N && SP_OBJ - SP_CONS == PC_N && SP_TIME - SP_OBJ == PO_N &&
                  SP_YT - SP_TIME >= 1 && SP_ZERO - SP_YT >= PC_N && SP_MISC - SP_ZERO >= PL_N,
              "partial-sum slots overlap");

constexpr int kBatchLdMax = 128;          // one 16-byte unit per lane (CPL = 1)
constexpr int kBatchMaxThreads = 512;     // threads per block: 256 or 512 (register budget 128 each)

__device__ __forceinline__ long long globaltimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int batch_lanes(int Q, int rows_per_warp) {
    int L = 1;
    while (L < Q) L <<= 1;
    const int Lr = 32 / rows_per_warp;
    return L > Lr ? L : Lr;
}

template <typename T>
__device__ __forceinline__ double as_double(T v) {
    return static_cast<double>(v);
}

// Starting factor: the given R0, else rows of SplitMix64 normals as the
// single-instance solve draws them (unit rows for diagonal constraints).
// The blocks that solve one instance: one block (size 1), or the blocks of a
// thread-block cluster that split the rows and constraints of one large
// instance, reduce their partial sums through distributed shared memory and
// each keep an identical copy of the control block.
struct Team {
    int rank, size;
    __device__ __forceinline__ void sync() const {
        if (size > 1) cg::this_cluster().sync();
        else __syncthreads();
    }
    __device__ __forceinline__ int64_t tid() const { return (int64_t)rank * blockDim.x + threadIdx.x; }
    __device__ __forceinline__ int64_t nthreads() const { return (int64_t)size * blockDim.x; }
};

// Starting factor: the given R0, else rows of SplitMix64 normals as the
// single-instance solve draws them (unit rows for diagonal constraints).
template <typename TR>
__device__ void batch_start(const BInst& I, TR* R, int r, int ld, const Team& tm) {
    const int64_t n = I.p.n;
    if (I.R0 != nullptr) {
        for (int64_t e = tm.tid(); e < n * ld; e += tm.nthreads()) {
            const int64_t i = e / ld;
            const int c = (int)(e - i * ld);
            R[e] = c < r ? TR(I.R0[i * r + c]) : TR(0.0);
        }
        return;
    }
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    const uint64_t base = I.seed ^ (~0ull * golden);
    for (int64_t i = tm.tid(); i < n; i += tm.nthreads()) {
        double nrm = 0.0;
        for (int c = 0; c < r; ++c) {
            const double g = normal_at(base, i * r + c);
            nrm += g * g;
        }
        for (int c = 0; c < ld; ++c) {
            double v = 0.0;
            if (c < r) {
                const double g = normal_at(base, i * r + c);
                v = I.unit_rows ? g / sqrt(nrm) : I.start_scale * g;
            }
            R[i * ld + c] = TR(v);
        }
    }
}

// sp: this block's partial sums; tot: the team's sums (== sp for one block)
template <typename TR, typename TD>
__device__ void batch_solve_one(const BInst& I, const Ctrl& c0, BOut& o, Ctrl* c, AdmmCtrl* ac, double* sp,
                                double* tot, int rows_per_warp, long long time_limit_ns, long long* ph,
                                const Team tm) {
    using ZS = zrow_t<TD, TR>;
    // y~ and the cached z of the off-diagonal constraints: double-float unless FP64
    constexpr bool kYtilDf = !std::is_same<TR, double>::value;
    const VGrid vg{tm.rank, tm.size, 0};
    const int tid = threadIdx.x;
    const long long t_begin = globaltimer_ns();
    long long t_last = t_begin;
    if (tid < BP_N) ph[tid] = 0;
    // time since the previous tick goes to phase q (thread 0, right after a barrier)
    auto tick = [&](int q) {
        if (tid == 0) {
            const long long now = globaltimer_ns();
            ph[q] += now - t_last;
            t_last = now;
        }
    };
    // after a body that wrote its partials to sp[off, off+nq): the team's sums in
    // tot (fixed rank order: every block gets bit-identical sums)
    auto reduce = [&](int off, int nq) {
        tm.sync();
        if (tm.size > 1) {
            cg::cluster_group cl = cg::this_cluster();
            for (int q = tid; q < nq; q += blockDim.x) {
                double acc = 0.0;
                for (int rk = 0; rk < tm.size; ++rk) acc += cl.map_shared_rank(sp, rk)[off + q];
                tot[off + q] = acc;
            }
            __syncthreads();
        }
    };
    {
        const int* src = reinterpret_cast<const int*>(&c0);
        int* dst = reinterpret_cast<int*>(c);
        for (int w = tid; w < (int)(sizeof(Ctrl) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        if (tid < SP_N - SP_ZERO) {
            sp[SP_ZERO + tid] = 0.0;
            tot[SP_ZERO + tid] = 0.0;
        }
    }
    const ProbDev p = I.p;
    TR* R = static_cast<TR*>(I.R);
    TR* CR = static_cast<TR*>(I.CR);
    TD* D = static_cast<TD*>(I.D);
    TD* CD = static_cast<TD*>(I.CD);
    TD* G = static_cast<TD*>(I.G);
    TD* W = static_cast<TD*>(I.W);
    TD* hist = static_cast<TD*>(I.hist);
    ZS* zrow = static_cast<ZS*>(I.zrow);
    double* y = I.y;
    double* ytil = I.ytil;
    double* zk = I.zk;
    dfloat* ydf = I.ydf;
    const int64_t sstride = I.slot_stride;
    int r = I.r0;
    int ld = (r + 3) / 4 * 4;
    int Q = ld / 4;
    int L = batch_lanes(Q, rows_per_warp);
    int64_t nunits = p.n * (int64_t)ld / 4;

    batch_start<TR>(I, R, r, ld, tm);
    for (int64_t k = tm.tid(); k < p.m; k += tm.nthreads()) {
        y[k] = 0.0;
        if (ydf) ydf[k] = dfloat(0.0f, 0.0f);
    }
    tm.sync();

    auto spmm_cr = [&]() {
        k_spmm_c_body<TR, TR, TR, 1, EPI_OBJ>(p, R, CR, ld, L, Q, nullptr, 1, R, y, nullptr, nullptr, c, 0.0,
                                               sp + SP_OBJ, vg);
    };
    // G = grad L at the current R, then a fresh inner loop (memory empty)
    auto outer_gradient = [&]() {
        if (p.m_off) {
            k_cons_body<TR, TR, 1, CONS_YTIL>(p, p.m_diag, p.m, R, R, ld, L, Q, y, ytil, zk, ydf, c, 0.0,
                                              sp + SP_YT, vg);
            tm.sync();
            k_spmm_a_body<TR, TD, 1, kYtilDf>(p, R, W, ld, L, Q, ytil, 1.0, 0, vg);
            tm.sync();
        }
        k_update_body<TR, TD, 1, false, false>(p, R, CR, D, CD, G, p.m_off ? W : nullptr, hist, sstride, ld, L, Q,
                                               y, ydf, zrow, c, sp + SP_UPD, vg);
        reduce(SP_UPD, PU_N);
        if (p.m_off) reduce(SP_YT, PC_N);
        if (tid == 0) ctrl_hist_apply(c, true, true, tot + SP_UPD, p.m_off ? tot + SP_YT : tot + SP_ZERO);
        tm.sync();
        tick(BP_GRAD);
    };

    // ---- start: err1 at R0, objective, first gradient
    spmm_cr();
    tm.sync();
    k_cons_body<TR, TR, 1, CONS_ZZ>(p, 0, p.m, R, R, ld, L, Q, y, nullptr, nullptr, nullptr, c, 0.0, sp + SP_CONS,
                                    vg);
    reduce(SP_CONS, PC_N + PO_N);
    if (tid == 0) ctrl_init_apply(c, tot + SP_CONS, tot + SP_OBJ);
    tm.sync();
    tick(BP_INIT);
    outer_gradient();

    while (!c->solve_done) {
        if (c->pause) {
            // ---- rank update (App. A.1) within the instance's allocation
            const int r_old = r;
            int r_new = (int)ceil(1.5 * r_old);
            r_new = min(r_new, min(I.r_cap, I.ld_cap));
            if (r_new > r_old) {
                double acc[1] = {0.0};
                for (int64_t e = tm.tid(); e < p.n * ld; e += tm.nthreads()) {
                    const double v = as_double(R[e]);
                    acc[0] += v * v;
                }
                block_partials<1>(acc, sp + SP_MISC, 0);
                reduce(SP_MISC, 1);
                const double scale = 1e-3 * sqrt(tot[SP_MISC]) / sqrt((double)p.n * r_old);
                for (int64_t e = tm.tid(); e < p.n * ld; e += tm.nthreads()) CR[e] = R[e];     // old rows
                tm.sync();
                const int ld_new = (r_new + 3) / 4 * 4;
                const int k = r_new - r_old;
                const uint64_t golden = 0x9E3779B97F4A7C15ull;
                const uint64_t base = I.seed ^ ((uint64_t)(c->outer - 1) * golden);
                for (int64_t e = tm.tid(); e < p.n * ld_new; e += tm.nthreads()) {
                    const int64_t i = e / ld_new;
                    const int cc = (int)(e - i * ld_new);
                    TR v = TR(0.0);
                    if (cc < r_old) v = CR[i * ld + cc];
                    else if (cc < r_new) v = TR(scale * normal_at(base, i * k + (cc - r_old)));
                    R[e] = v;
                }
                tm.sync();
                r = r_new;
                ld = ld_new;
                Q = ld / 4;
                L = batch_lanes(Q, rows_per_warp);
                nunits = p.n * (int64_t)ld / 4;
            }
            if (tid == 0) {
                c->pause = 0;
                c->phase = PHASE_OUTER;
            }
            spmm_cr();
            tm.sync();
            tick(BP_RANK);
            outer_gradient();
            continue;
        }
        if (c->phase == PHASE_INNER) {
            // ---- one iteration of Algorithm 1: direction, exact line search, step
            k_dir_body<TD>(nunits, G, D, hist, sstride, c, sp + SP_DIR, vg);
            tm.sync();
            tick(BP_DIR);
            k_spmm_c_body<TD, TD, TR, 1, EPI_LS>(p, D, CD, ld, L, Q, nullptr, 1, R, y, zrow, ydf, c, 0.0,
                                                 sp + SP_LS, vg);
            tm.sync();
            tick(BP_LS);
            if (p.m_off) {
                k_cons_body<TR, TD, 1, CONS_LS>(p, p.m_diag, p.m, R, D, ld, L, Q, y, nullptr, zk, ydf, c, 0.0,
                                                sp + SP_CLS, vg);
                tm.sync();
                tick(BP_CONS_LS);
            }
            reduce(SP_DIR, SP_UPD - SP_DIR);          // direction, C pass and constraint pass sums
            if (tid == 0) ctrl_root_apply(c, tot + SP_DIR, tot + SP_LS, p.m_off ? tot + SP_CLS : tot + SP_ZERO);
            tm.sync();
            tick(BP_ROOT);
            if (c->solve_done) break;
            if (c->step_ok) {
                if (p.m_off) {
                    k_step_body<TR, TD>(nunits, R, CR, D, CD, c, vg);
                    tm.sync();
                    tick(BP_STEP);
                    k_cons_body<TR, TR, 1, CONS_YTIL>(p, p.m_diag, p.m, R, R, ld, L, Q, y, ytil, zk, ydf, c, 0.0,
                                                      sp + SP_YT, vg);
                    tm.sync();
                    tick(BP_YTIL);
                    k_spmm_a_body<TR, TD, 1, kYtilDf>(p, R, W, ld, L, Q, ytil, 1.0, 0, vg);
                    tm.sync();
                    tick(BP_SPMM_A);
                    k_update_body<TR, TD, 1, false, true>(p, R, CR, D, CD, G, W, hist, sstride, ld, L, Q, y, ydf,
                                                          zrow, c, sp + SP_UPD, vg);
                    reduce(SP_UPD, PU_N);
                    reduce(SP_YT, PC_N);
                } else {
                    k_update_body<TR, TD, 1, true, true>(p, R, CR, D, CD, G, nullptr, hist, sstride, ld, L, Q, y,
                                                         ydf, zrow, c, sp + SP_UPD, vg);
                    reduce(SP_UPD, PU_N);
                }
                tick(BP_UPDATE);
            }
            if (tid == 0 && !c->solve_done && !c->pause && c->phase == PHASE_INNER)
                ctrl_hist_apply(c, false, c->step_ok != 0, tot + SP_UPD, p.m_off ? tot + SP_YT : tot + SP_ZERO);
            tm.sync();
            tick(BP_HIST);
        }
        if (!c->solve_done && !c->pause && c->phase == PHASE_OUTER) {
            // ---- multiplier step of Sec. 2.1 and the outer tests
            k_cons_body<TR, TR, 1, CONS_YUPD>(p, 0, p.m, R, R, ld, L, Q, y, nullptr, nullptr, ydf, c, 0.0,
                                              sp + SP_CONS, vg);
            tm.sync();
            spmm_cr();
            // the time limit: rank 0's clock, summed with the partials so that
            // every block of a team takes the same decision
            if (tid == 0) sp[SP_TIME] = tm.rank == 0 ? (double)(globaltimer_ns() - t_begin) : 0.0;
            reduce(SP_CONS, PC_N + PO_N + 1);
            if (tid == 0) {
                ctrl_outer_apply(c, tot + SP_CONS, tot + SP_OBJ);
                if (!c->solve_done && time_limit_ns > 0 && tot[SP_TIME] > (double)time_limit_ns) {
                    c->status = LORADS_ERR_TIMEOUT;
                    c->solve_done = 1;
                }
            }
            tm.sync();
            tick(BP_OUTER);
            if (!c->solve_done && !c->pause) outer_gradient();
        }
    }
    tm.sync();
    // ---- the splitting ADMM stage (Sec. 2.2) when the ALM stage stopped at the switch
    // tolerance: U = V = R, the ALM stage's y and rho (fixed); Algorithm 2's CG for each
    // block step as a device loop; the direction, C D and gradient arrays hold r, p, Q.
    int admm_iters = 0, cg_steps = 0;
    if (I.admm_on && c->status == LORADS_OK && !(c->err1 <= I.admm_tol && fabs(c->err3) <= I.admm_tol)) {
        enum { SA_R = SP_DIR, SA_Q = SP_LS };
        TR* U = static_cast<TR*>(I.U);
        TR* V = static_cast<TR*>(I.V);
        TD* rv = D;
        TD* pv = CD;
        TD* Qv = G;
        for (int64_t e = tm.tid(); e < p.n * ld; e += tm.nthreads()) {
            U[e] = R[e];
            V[e] = R[e];
        }
        if (tid == 0) {
            *ac = AdmmCtrl{};
            ac->rho = c->rho;
            ac->cg_rel = I.cg_rel;
            ac->cg_max = I.cg_max;
            ac->tol = I.admm_tol;
            ac->bnorm_inf = c->bnorm_inf;
            ac->max_iter = I.admm_max_iter;
            ac->status = LORADS_ERR_MAXITER;
        }
        tm.sync();
        while (!ac->done) {
            for (int half = 0; half < 2 && !ac->done; ++half) {
                TR* X = half == 0 ? U : V;
                const TR* Vf = half == 0 ? V : U;
                k_admm_cons_body<TR, 1, 0>(p, X, Vf, ld, L, Q, y, ydf, I.om, ac, nullptr, vg);
                tm.sync();
                k_admm_resid_body<TR, TD, 1>(p, X, Vf, ld, L, Q, I.om, rv, pv, ac, sp + SA_R, vg);
                reduce(SA_R, 1);
                if (tid == 0) admm_cg_init_apply(ac, tot[SA_R]);
                tm.sync();
                while (ac->cg_active) {
                    if (p.m_off > 0) {
                        k_admm_pupd_body<TD>(nunits, rv, pv, ac, vg);
                        tm.sync();
                        k_admm_op_body<TR, TD, 1, false>(p, Vf, ld, L, Q, rv, pv, Qv, ac, 0.0, sp + SA_Q, vg);
                    } else {
                        k_admm_op_body<TR, TD, 1, true>(p, Vf, ld, L, Q, rv, pv, Qv, ac, 0.0, sp + SA_Q, vg);
                    }
                    reduce(SA_Q, PQ_N);
                    if (tid == 0) admm_alpha_apply(ac, tot[SA_Q + PQ_PP], tot[SA_Q + PQ_WW]);
                    tm.sync();
                    if (!ac->cg_active) break;
                    k_admm_upd_body<TR, TD>(nunits, X, pv, rv, Qv, ac, sp + SA_R, vg);
                    reduce(SA_R, 1);
                    if (tid == 0) admm_beta_apply(ac, tot[SA_R]);
                    tm.sync();
                }
            }
            if (ac->done) break;
            // multiplier step, R = (U + V)/2, <C R, R> and ||A(RR^T) - b|| (Sec. 4.2 at R)
            k_admm_cons_body<TR, 1, 1>(p, U, V, ld, L, Q, y, ydf, nullptr, ac, sp + SP_YT, vg);
            tm.sync();
            k_admm_avg_body<TR>(nunits, U, V, R, vg);
            tm.sync();
            spmm_cr();
            tm.sync();
            k_cons_body<TR, TR, 1, CONS_ZZ>(p, 0, p.m, R, R, ld, L, Q, y, nullptr, nullptr, nullptr, c, 0.0,
                                            sp + SP_CONS, vg);
            if (tid == 0) sp[SP_TIME] = tm.rank == 0 ? (double)(globaltimer_ns() - t_begin) : 0.0;
            reduce(SP_CONS, PC_N + PO_N + 1);
            reduce(SP_YT, PY_N);
            if (tid == 0) {
                admm_outer_apply(ac, tot[SP_CONS + PC_ZZ], tot[SP_YT + PY_BY], tot[SP_OBJ + PO_CRR]);
                if (!ac->done && time_limit_ns > 0 && tot[SP_TIME] > (double)time_limit_ns) {
                    ac->status = LORADS_ERR_TIMEOUT;
                    ac->done = 1;
                }
            }
            tm.sync();
            tick(BP_ADMM);
        }
        if (tid == 0) {
            if (ac->iters > 0) {
                c->primal_obj = ac->primal_obj;
                c->dual_obj = ac->dual_obj;
                c->err1 = ac->err1;
                c->err3 = ac->err3;
            }
            c->status = ac->status;
        }
        admm_iters = ac->iters;
        cg_steps = ac->cg_total;
        tm.sync();
    }
    if (tm.rank == 0) {
        const int* src = reinterpret_cast<const int*>(c);
        int* dst = reinterpret_cast<int*>(&o.ctrl);
        for (int w = tid; w < (int)(sizeof(Ctrl) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
        if (tid == 0) {
            o.r = r;
            o.ld = ld;
            o.admm_iters = admm_iters;
            o.cg_steps = cg_steps;
            o.t_begin = t_begin;
            o.t_end = globaltimer_ns();
            for (int q = 0; q < BP_N; ++q) o.phase_ns[q] = ph[q];
        }
    }
}

// The persistent kernel.  With clusters of size > 1, each cluster first takes
// the large instances (order[0, n_team)) from one queue and solves each with
// all its blocks; once that queue is empty its blocks take the remaining
// instances one block each from a second queue.  Without clusters every block
// takes instances from the second queue starting at order[0].
template <typename TR, typename TD>
__global__ void __launch_bounds__(kBatchMaxThreads, 1)
k_batch_solve(const BInst* __restrict__ insts, const Ctrl* __restrict__ ctrl0, BOut* out,
              const int* __restrict__ order, int count, int n_team, int* queues, int rows_per_warp,
              long long time_limit_ns) {
    __shared__ Ctrl c;
    __shared__ AdmmCtrl ac;
    __shared__ double sp[SP_N];
    __shared__ double tot[SP_N];
    __shared__ long long s_ph[BP_N];
    __shared__ int s_item;
    __shared__ int s_team_item;
    cg::cluster_group cl = cg::this_cluster();
    const int csize = (int)cl.num_blocks();
    bool team_phase = csize > 1;
    for (;;) {
        int it;
        Team tm{0, 1};
        if (team_phase) {
            if (cl.block_rank() == 0 && threadIdx.x == 0) s_team_item = atomicAdd(queues, 1);
            cl.sync();
            it = *cl.map_shared_rank(&s_team_item, 0);
            cl.sync();                      // every block has read rank 0's slot
            if (it >= n_team) {
                team_phase = false;         // the same decision in every block of the cluster
                continue;
            }
            tm = Team{(int)cl.block_rank(), csize};
        } else {
            __syncthreads();
            if (threadIdx.x == 0) s_item = (csize > 1 ? n_team : 0) + atomicAdd(queues + 1, 1);
            __syncthreads();
            it = s_item;
            if (it >= count) return;
        }
        const int k = order[it];
        batch_solve_one<TR, TD>(insts[k], ctrl0[k], out[k], &c, &ac, sp, tm.size > 1 ? tot : sp, rows_per_warp,
                                time_limit_ns, s_ph, tm);
    }
}

// Address of the persistent kernel for storage types (TR, TD); one
// instantiation per precision translation unit.
void* kernel_fp64();
void* kernel_mixed();
void* kernel_fp32();

}  // namespace batch
}  // namespace lorads
