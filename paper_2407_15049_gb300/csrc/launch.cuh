// Host launchers of the streaming kernels.  Declared for every precision in
// launch_decl.h and explicitly instantiated per precision in kern_*.cu, so the
// template-heavy device code compiles in parallel translation units.
#pragma once

#include "kernels.cuh"
#include "launch_decl.h"

namespace lorads {

#define LORADS_CPL_SWITCH(cpl, ...)                                   \
    switch (cpl) {                                                      \
        case 1: { constexpr int CPL = 1; __VA_ARGS__; } break;         \
        case 2: { constexpr int CPL = 2; __VA_ARGS__; } break;         \
        case 3: { constexpr int CPL = 3; __VA_ARGS__; } break;         \
        case 4: { constexpr int CPL = 4; __VA_ARGS__; } break;         \
        default: break;                                                 \
    }

template <typename TX, typename TO, typename TR, int CPL, int EPI, bool DENSE, int PF>
void launch_spmm_c_one(const SpmmCArgs& a, int L) {
    k_spmm_c<TX, TO, TR, CPL, EPI, DENSE, PF><<<a.blocks, kThreads, 0, a.stream>>>(
        a.p, static_cast<const TX*>(a.X), static_cast<TO*>(a.out), a.ld, L, a.sh.Q, a.v, a.write_out,
        static_cast<const TR*>(a.R), a.y, a.zrow, a.ydf, a.ctrl, a.rho, a.part, a.gate, a.ph);
}

// The line-search form takes the prefetch depth (and packed groups) as template
// arguments; the other epilogues run without prefetch.
template <typename TX, typename TO, typename TR>
void launch_spmm_c(const SpmmCArgs& a) {
    if (a.epi == EPI_LS && a.dense && packed_rows_gain(a.sh)) {
        if (a.prefetch == 2) launch_spmm_c_one<TX, TO, TR, 1, EPI_LS, true, 2>(a, a.sh.Q);
        else if (a.prefetch == 1) launch_spmm_c_one<TX, TO, TR, 1, EPI_LS, true, 1>(a, a.sh.Q);
        else launch_spmm_c_one<TX, TO, TR, 1, EPI_LS, true, 0>(a, a.sh.Q);
        return;
    }
    LORADS_CPL_SWITCH(a.sh.CPL, {
        if (a.epi == EPI_LS) {
            if (a.prefetch == 2) launch_spmm_c_one<TX, TO, TR, CPL, EPI_LS, false, 2>(a, a.sh.L);
            else if (a.prefetch == 1) launch_spmm_c_one<TX, TO, TR, CPL, EPI_LS, false, 1>(a, a.sh.L);
            else launch_spmm_c_one<TX, TO, TR, CPL, EPI_LS, false, 0>(a, a.sh.L);
        } else if (a.epi == EPI_OBJ) {
            launch_spmm_c_one<TX, TO, TR, CPL, EPI_OBJ, false, 0>(a, a.sh.L);
        } else {
            launch_spmm_c_one<TX, TO, TR, CPL, EPI_NONE, false, 0>(a, a.sh.L);
        }
    })
}

template <typename TX, typename TO>
void launch_spmm_a(const SpmmAArgs& a) {
    const TX* X = static_cast<const TX*>(a.X);
    TO* out = static_cast<TO*>(a.out);
    if constexpr (!std::is_same_v<arith_t<TO>, double>) {
        if (a.v_df) {
            LORADS_CPL_SWITCH(a.sh.CPL, {
                k_spmm_a<TX, TO, CPL, true><<<a.blocks, kThreads, 0, a.stream>>>(
                    a.p, X, out, a.ld, a.sh.L, a.sh.Q, a.v, a.alpha, a.accumulate, a.gate, a.ph);
            })
            return;
        }
    }
    LORADS_CPL_SWITCH(a.sh.CPL, {
        k_spmm_a<TX, TO, CPL, false><<<a.blocks, kThreads, 0, a.stream>>>(
            a.p, X, out, a.ld, a.sh.L, a.sh.Q, a.v, a.alpha, a.accumulate, a.gate, a.ph);
    })
}

template <typename TU, typename TV>
void launch_cons(const ConsArgs& a) {
    const TU* U = static_cast<const TU*>(a.U);
    const TV* V = static_cast<const TV*>(a.V);
    if (a.k1 <= a.k0) return;
    LORADS_CPL_SWITCH(a.sh.CPL, {
        switch (a.mode) {
            case CONS_EVAL:
                k_cons<TU, TV, CPL, CONS_EVAL><<<a.blocks, kThreads, 0, a.stream>>>(
                    a.p, a.k0, a.k1, U, V, a.ld, a.sh.L, a.sh.Q, a.y, a.out, a.zk, a.ydf, a.ctrl, a.rho, a.part, a.gate, a.ph);
                break;
            case CONS_LS:
                k_cons<TU, TV, CPL, CONS_LS><<<a.blocks, kThreads, 0, a.stream>>>(
                    a.p, a.k0, a.k1, U, V, a.ld, a.sh.L, a.sh.Q, a.y, a.out, a.zk, a.ydf, a.ctrl, a.rho, a.part, a.gate, a.ph);
                break;
            case CONS_YTIL:
                k_cons<TU, TV, CPL, CONS_YTIL><<<a.blocks, kThreads, 0, a.stream>>>(
                    a.p, a.k0, a.k1, U, V, a.ld, a.sh.L, a.sh.Q, a.y, a.out, a.zk, a.ydf, a.ctrl, a.rho, a.part, a.gate, a.ph);
                break;
            case CONS_YUPD:
                k_cons<TU, TV, CPL, CONS_YUPD><<<a.blocks, kThreads, 0, a.stream>>>(
                    a.p, a.k0, a.k1, U, V, a.ld, a.sh.L, a.sh.Q, a.y, a.out, a.zk, a.ydf, a.ctrl, a.rho, a.part, a.gate, a.ph);
                break;
            case CONS_ZZ:
                k_cons<TU, TV, CPL, CONS_ZZ><<<a.blocks, kThreads, 0, a.stream>>>(
                    a.p, a.k0, a.k1, U, V, a.ld, a.sh.L, a.sh.Q, a.y, a.out, a.zk, a.ydf, a.ctrl, a.rho, a.part, a.gate, a.ph);
                break;
            default: break;
        }
    })
}

template <typename TD, typename TDIR>
void launch_dir(const DirArgs& a) {
    k_dir<TD, TDIR><<<a.blocks, kThreads, 0, a.stream>>>(
        a.nunits, static_cast<const TD*>(a.G), static_cast<TDIR*>(a.D), static_cast<const TDIR*>(a.hist),
        a.slot_stride, a.ctrl, a.part, a.gate, a.ph);
}

template <typename TR, typename TD, typename TDIR>
void launch_step(const StepArgs& a) {
    k_step<TR, TD, TDIR><<<a.blocks, kThreads, 0, a.stream>>>(
        a.nunits, static_cast<TR*>(a.R), static_cast<TR*>(a.CR), static_cast<const TDIR*>(a.D),
        static_cast<const TD*>(a.CD), a.ctrl, a.gate, a.ph);
}

template <typename TR, typename TD, typename TDIR, int CPL, int EXTRA, bool DENSE, int MAXOLD>
void launch_update_occ(const UpdateArgs& a, int L) {
    k_update_step_occ<TR, TD, CPL, EXTRA, TDIR, DENSE, MAXOLD><<<a.blocks, kThreads, 0, a.stream>>>(
        a.p, static_cast<TR*>(a.R), static_cast<TR*>(a.CR), static_cast<const TDIR*>(a.D),
        static_cast<const TD*>(a.CD), static_cast<TD*>(a.G), static_cast<const TD*>(a.W), static_cast<TDIR*>(a.hist),
        a.slot_stride, a.ld, L, a.sh.Q, a.y, a.ydf, a.zrow, a.ctrl, a.part, a.gate, a.ph, a.prefetch);
}

// The step update with more resident blocks: one instantiation per lane shape and
// per bound on the stored pairs (T <= 2, or up to 4).
template <typename TR, typename TD, typename TDIR, int CPL, int EXTRA>
void launch_update_occ_shape(const UpdateArgs& a) {
    const bool dense = CPL == 1 && a.dense && packed_rows_gain(a.sh);
    if (dense) {
        if (a.max_old <= 1) launch_update_occ<TR, TD, TDIR, 1, EXTRA, true, 1>(a, a.sh.Q);
        else launch_update_occ<TR, TD, TDIR, 1, EXTRA, true, kMaxMem - 1>(a, a.sh.Q);
    } else {
        if (a.max_old <= 1) launch_update_occ<TR, TD, TDIR, CPL, EXTRA, false, 1>(a, a.sh.L);
        else launch_update_occ<TR, TD, TDIR, CPL, EXTRA, false, kMaxMem - 1>(a, a.sh.L);
    }
}

template <typename TR, typename TD, typename TDIR>
void launch_update(const UpdateArgs& a) {
    TR* R = static_cast<TR*>(a.R);
    TR* CR = static_cast<TR*>(a.CR);
    const TDIR* D = static_cast<const TDIR*>(a.D);
    const TD* CD = static_cast<const TD*>(a.CD);
    TD* G = static_cast<TD*>(a.G);
    const TD* W = static_cast<const TD*>(a.W);
    TDIR* H = static_cast<TDIR*>(a.hist);          // pairs stored in the direction's type
    LORADS_CPL_SWITCH(a.sh.CPL, {
        if (a.step && a.hist_on && a.extra_blocks == 1)
            launch_update_occ_shape<TR, TD, TDIR, CPL, 1>(a);
        else if (a.step && a.hist_on && a.extra_blocks == 2)
            launch_update_occ_shape<TR, TD, TDIR, CPL, 2>(a);
        else if (a.step && a.hist_on)
            k_update<TR, TD, CPL, true, true, TDIR><<<a.blocks, kThreads, 0, a.stream>>>(
                a.p, R, CR, D, CD, G, W, H, a.slot_stride, a.ld, a.sh.L, a.sh.Q, a.y, a.ydf, a.zrow, a.ctrl, a.part, a.gate, a.ph);
        else if (!a.step && a.hist_on)
            k_update<TR, TD, CPL, false, true, TDIR><<<a.blocks, kThreads, 0, a.stream>>>(
                a.p, R, CR, D, CD, G, W, H, a.slot_stride, a.ld, a.sh.L, a.sh.Q, a.y, a.ydf, a.zrow, a.ctrl, a.part, a.gate, a.ph);
        else
            k_update<TR, TD, CPL, false, false, TDIR><<<a.blocks, kThreads, 0, a.stream>>>(
                a.p, R, CR, D, CD, G, W, H, a.slot_stride, a.ld, a.sh.L, a.sh.Q, a.y, a.ydf, a.zrow, a.ctrl, a.part, a.gate, a.ph);
    })
}

#define LORADS_INSTANTIATE_SPMM_C(TX, TO, TR) template void launch_spmm_c<TX, TO, TR>(const SpmmCArgs&);
#define LORADS_INSTANTIATE_SPMM_A(TX, TO) template void launch_spmm_a<TX, TO>(const SpmmAArgs&);
#define LORADS_INSTANTIATE_CONS(TU, TV) template void launch_cons<TU, TV>(const ConsArgs&);
#define LORADS_INSTANTIATE_DIR(TD) template void launch_dir<TD, TD>(const DirArgs&);
#define LORADS_INSTANTIATE_DIR2(TD, TDIR) template void launch_dir<TD, TDIR>(const DirArgs&);
#define LORADS_INSTANTIATE_STEP(TR, TD) template void launch_step<TR, TD, TD>(const StepArgs&);
#define LORADS_INSTANTIATE_STEP2(TR, TD, TDIR) template void launch_step<TR, TD, TDIR>(const StepArgs&);
#define LORADS_INSTANTIATE_UPDATE(TR, TD) template void launch_update<TR, TD, TD>(const UpdateArgs&);
#define LORADS_INSTANTIATE_UPDATE2(TR, TD, TDIR) template void launch_update<TR, TD, TDIR>(const UpdateArgs&);

}  // namespace lorads
