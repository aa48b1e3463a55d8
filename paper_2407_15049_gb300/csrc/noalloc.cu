// lorads_linesearch_coeffs_noalloc: the exact line-search coefficients without
// a context and without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// step: frameworks whose caching allocator owns the device memory (a cudaMalloc
// beside it can fail or fragment what the framework holds), and latency-critical
// loops that cannot afford the device-wide synchronisation cudaMalloc and
// cudaFree may imply.  This entry point takes every input as caller-owned device
// memory and keeps its only scratch (the per-block partial sums of its two
// reductions) in one file-scope device array of fixed size: 2 x 1024 blocks x 7
// doubles, 114,688 bytes.  Launch grids are capped at 1024 blocks, so the
// scratch never grows with the problem.
//
// That array is a single region shared by every call on a device: calls that
// overlap on the GPU (different streams or threads without ordering) race on
// it and must be serialised by the caller.  It keeps the last call's contents;
// every call overwrites all the partial slots it later reads, so nothing needs
// clearing.  Every GPU that loads this library holds the array until the
// process exits.
//
// The address of the array on each device is looked up once, on the first
// call with that device current, and cached per device ordinal.  A
// cudaDeviceReset (or any teardown of the device's primary context) unloads
// the module; the cached address is then stale, so a process that resets a
// device must not call this entry point on that device afterwards.
#include <mutex>
#include <string>

#include "../../include/lorads.h"
#include "common.cuh"
#include "control.h"
#include "kernels.cuh"
#include "launch_decl.h"

using namespace lorads;

namespace {

constexpr int kNoallocBlocks = 1024;        // grid cap of each reduction launch
constexpr int kNoallocParts = kNoallocBlocks * PL_N;
constexpr int kNoallocWords = 2 * kNoallocParts;       // two partial regions

// The scratch.  In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocWords];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};
thread_local std::string g_noalloc_err;

// Device address of the scratch for the current device (looked up once per device).
lorads_status scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return LORADS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        g_noalloc_err = "device ordinal beyond the supported 64";
        return LORADS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            g_noalloc_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return LORADS_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return LORADS_OK;
}

int capped_blocks(int64_t items, int L) {
    const int64_t per_block = kThreads / L;
    int64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    return (int)(b < kNoallocBlocks ? b : kNoallocBlocks);
}

}  // namespace

extern "C" const char* lorads_noalloc_error(void) { return g_noalloc_err.c_str(); }

extern "C" lorads_status lorads_linesearch_coeffs_noalloc(
    int64_t n, const int64_t* c_rowptr, const int32_t* c_colind, const double* c_val, int64_t m,
    const int32_t* a_con, const int32_t* a_row, const int32_t* a_col, const double* a_val, const double* b,
    const double* R, const double* D, int32_t r, int32_t ld, const double* y, double rho, double* out,
    void* cuda_stream) {
    g_noalloc_err.clear();
    if (n < 1 || n > INT32_MAX || m < 1 || m > INT32_MAX) {
        g_noalloc_err = "n and m must be in [1, 2^31)";
        return LORADS_ERR_INVALID_ARG;
    }
    Shape sh;
    if (r < 1 || ld < r || !shape_for_ld(ld, &sh)) {
        g_noalloc_err = "need 1 <= r <= ld, ld a multiple of 4 and at most " + std::to_string(kMaxLd);
        return LORADS_ERR_INVALID_ARG;
    }
    if (!c_rowptr || !c_colind || !c_val || !a_con || !a_row || !a_col || !a_val || !b || !R || !D || !y || !out) {
        g_noalloc_err = "null device pointer";
        return LORADS_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(R) | reinterpret_cast<uintptr_t>(D)) & 15u) {
        g_noalloc_err = "R and D must be 16-byte aligned";
        return LORADS_ERR_INVALID_ARG;
    }
    if (!(rho >= 0.0) || rho != rho || rho > 1e300) {
        g_noalloc_err = "rho must be finite and >= 0";
        return LORADS_ERR_INVALID_ARG;
    }
    double* scratch = nullptr;
    lorads_status s = scratch_for_current_device(&scratch);
    if (s != LORADS_OK) return s;
    double* part_ls = scratch;
    double* part_cons = scratch + kNoallocParts;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // Each triplet is passed to the constraint pass as its own constraint, so the
    // per-constraint products q1_k q2_k, q1_k^2, q2_k^2 of App. A.2 are formed per
    // triplet.  That equals the per-constraint sums only when every constraint has
    // exactly one triplet (the input lorads_create accepts); several triplets of
    // one constraint would give wrong coefficients, not an error.
    ProbDev p{};
    p.n = n;
    p.m = m;
    p.c_rowptr = c_rowptr;
    p.c_col = c_colind;
    p.c_val = c_val;
    p.k_row = a_row;                   // constraint k = triplet k: every constraint goes
    p.k_col = a_col;                   // through the constraint pass (no row fusion)
    p.k_a = a_val;
    p.k_id = a_con;
    p.b = b;
    p.m_diag = 0;
    p.m_off = m;
    const int nb_rows = capped_blocks(n, sh.L);
    const int nb_cons = capped_blocks(m, sh.L);
    // p1 = 2<CD, R>, p2 = <CD, D> over C; then the constraint terms; then a1..a4, tau
    SpmmCArgs a{p, D, nullptr, ld, sh, nullptr, 0, EPI_LS, R, y, nullptr, nullptr, nullptr, rho, part_ls,
                nb_rows, nullptr, PH_ALWAYS, stream};
    launch_spmm_c<double, double, double>(a);
    ConsArgs ca{p, CONS_LS, 0, m, R, D, ld, sh, const_cast<double*>(y), nullptr, nullptr, nullptr, nullptr, rho,
                part_cons, nb_cons, nullptr, PH_ALWAYS, stream};
    launch_cons<double, double>(ca);
    ls_finish(stream, part_ls, nb_rows, part_cons, nb_cons, rho, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_noalloc_err = std::string("launch: ") + cudaGetErrorString(e);
        return LORADS_ERR_CUDA;
    }
    return LORADS_OK;
}
