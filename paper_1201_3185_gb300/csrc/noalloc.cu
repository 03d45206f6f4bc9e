// A QUMOND solve that allocates nothing: qumond_solve_mond_noalloc.
//
// Some callers cannot allocate device memory at the time they need a solve:
// code running inside a memory pool or arena that owns the whole device
// budget, a host thread that must not take the allocator's locks, or a
// caller that has already reserved every byte for its own buffers.  For
// them this entry point keeps all of its scratch (the multigrid levels and
// the norm reduction buffers) in one file-scope device array of fixed size,
// so a call makes no cudaMalloc, cudaFree or other allocating call.  The
// caller still provides the right-hand side, the parent potential and the
// output, as for qumond_solve_mond.
//
// The array is created when the library's module is loaded on a device and
// stays allocated on every device that loaded it until the process exits.
// Only the device-side address is usable by kernels: in host code the array's
// name is a host stand-in, so the first call on each device looks the address
// up with cudaGetSymbolAddress (with that device current) and caches it; a
// device reset (cudaDeviceReset) in the same process is not supported, since
// the cached address would then be stale.  All
// calls on a device share the array and it keeps the previous call's
// contents, so every call clears it first; two calls whose work overlaps on
// the GPU (different streams, or different host threads) race on it.
#include "qumond.h"
#include "qumond_internal.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

using namespace qumond;

namespace {

// Size of one level's two colour-split arrays (iterate and right-hand side)
// in FP32, matching make_view().
constexpr long long level_cs(int n)
{
    return ((long long)((((n / 2 + 1) + 3) & ~3)) * (n + 1) * (n + 1) + 63) & ~63LL;
}
constexpr size_t level_bytes(int n) { return (size_t)(2 * 2 * level_cs(n)) * sizeof(float); }
constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr long long residual_blocks(int n) { return (long long)((n - 1 + 127) / 128) * (n - 1) * (n - 1); }

constexpr int kMaxN = QUMOND_NOALLOC_MAX_N;
constexpr size_t kLevelsBytes = round256(level_bytes(64)) + round256(level_bytes(32)) + round256(level_bytes(16));
constexpr size_t kPartialBytes = round256(sizeof(double) * 2 * (size_t)(residual_blocks(kMaxN) + 1));
constexpr size_t kScratchBytes = kLevelsBytes + kPartialBytes + 256;
static_assert(kMaxN == 64, "the scratch layout above is sized for n <= 64");
static_assert(kScratchBytes <= (size_t)QUMOND_NOALLOC_SCRATCH_BYTES, "header constant too small");

static __device__ __align__(256) unsigned char g_scratch[QUMOND_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Set-up of the current device, once per device: the device address of
// g_scratch, and the kernel attributes the solve needs (the coarse-grid
// kernel takes more than the default 48 KB of dynamic shared memory for
// n >= 16).  Neither step allocates.  qumond_create sets the same attributes,
// but a caller of this entry point may never create a context.
cudaError_t scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        e = prepare_kernels();
        if (e != cudaSuccess) return e;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return cudaSuccess;
}

struct NLevel {
    LevelView v;
    float* e = nullptr;
    float* f = nullptr;
};

struct Solver {
    const qumond_params* p;
    int L = 0, lc = 0;
    NLevel lev[8];
    double* partials = nullptr;
    double* norms = nullptr;
    double h = 0.0;  // finest spacing
    cudaStream_t s = nullptr;

    double level_h(int l) const { return h * (double)(1 << (L - l)); }

    cudaError_t vcycle(int l, bool zero_guess)
    {
        const double hl = level_h(l);
        if (l <= lc)
            return launch_coarse<float>(0, lev[l].e, lev[l].f, lev[l].v, hl, nullptr, 0, p->ncycle, p->npre, p->npost, s);
        for (int q = 0; q < p->npre; ++q) {
            launch_rb_half<float>(lev[l].e, lev[l].f, lev[l].v, 0, zero_guess && q == 0, hl, s);
            launch_rb_half<float>(lev[l].e, lev[l].f, lev[l].v, 1, false, hl, s);
        }
        launch_restrict_resid_red<float>(lev[l].e, lev[l].f, lev[l].v, lev[l - 1].f, lev[l - 1].v, hl, s);
        cudaError_t err = vcycle(l - 1, true);
        if (err != cudaSuccess) return err;
        launch_prolong_black<float>(lev[l - 1].e, lev[l - 1].v, lev[l].e, lev[l].v, true, s);
        for (int q = 0; q < p->npost; ++q) {
            launch_rb_half<float>(lev[l].e, lev[l].f, lev[l].v, 0, false, hl, s);
            launch_rb_half<float>(lev[l].e, lev[l].f, lev[l].v, 1, false, hl, s);
        }
        return cudaSuccess;
    }

    cudaError_t fmg(const double* u64)
    {
        for (int l = L - 1; l >= lc; --l) launch_restrict_full<float>(lev[l + 1].f, lev[l + 1].v, lev[l].f, lev[l].v, s);
        cudaError_t err = launch_coarse<float>(1, lev[lc].e, lev[lc].f, lev[lc].v, level_h(lc), u64, p->n, p->ncycle,
                                               p->npre, p->npost, s);
        if (err != cudaSuccess) return err;
        for (int l = lc + 1; l <= L; ++l) {
            launch_set_boundary<float>(lev[l].e, lev[l].v, u64, p->n, s);
            launch_prolong_black<float>(lev[l - 1].e, lev[l - 1].v, lev[l].e, lev[l].v, false, s);
            launch_set_boundary<float>(lev[l - 1].e, lev[l - 1].v, nullptr, p->n, s);
            for (int q = 0; q < p->ncycle; ++q) {
                err = vcycle(l, false);
                if (err != cudaSuccess) return err;
            }
        }
        return cudaSuccess;
    }

    cudaError_t norms_of(const double* u, const double* rhs, double* rr, double* ff)
    {
        const int nb = launch_residual_outer<float>(u, rhs, 1.0, p->n, h, lev[L].f, lev[L].v, partials, s);
        launch_reduce_norms(partials, nb, norms, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double host[2] = {0.0, 0.0};
        e = cudaMemcpyAsync(host, norms, sizeof(host), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(s);
        *rr = host[0];
        *ff = host[1];
        return e;
    }
};

bool is_device_ptr(const void* ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

qumond_status set_err(char* err, size_t len, qumond_status st, const char* msg)
{
    if (err && len) snprintf(err, len, "%s", msg);
    return st;
}

}  // namespace

extern "C" qumond_status qumond_solve_mond_noalloc(const qumond_params* p, int box, const double* src,
                                                   const double* phi_parent, double* phi, qumond_stats* stats,
                                                   void* stream, char* err, size_t err_len)
{
    char msg[256];
    if (err && err_len) err[0] = '\0';
    if (!p) return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "params is NULL");
    const int n = p->n;
    if (n < 2 || n > kMaxN || (n & (n - 1))) {
        snprintf(msg, sizeof(msg), "n=%d: this entry point takes a power of two n <= %d (its fixed scratch of %zu bytes"
                 " holds no larger grid); use qumond_solve_mond for bigger grids", n, kMaxN,
                 (size_t)QUMOND_NOALLOC_SCRATCH_BYTES);
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, msg);
    }
    if (p->precision != QUMOND_PREC_MIXED)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "only QUMOND_PREC_MIXED is supported without allocation");
    if (p->nboxes < 1 || p->nboxes > kMaxBoxes || box < 0 || box >= p->nboxes)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "box or nboxes out of range");
    if (!(p->L0 > 0.0) || !std::isfinite(p->L0))
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "L0 must be positive and finite");
    if (p->npre < 1 || p->npost < 1 || p->npre > 16 || p->npost > 16 || p->ncycle < 1 || p->ncycle > 128)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "npre, npost in [1,16] and ncycle in [1,128] required");
    if (!(p->rel_tol >= 0.0) || p->max_vcycles < 0 || p->max_vcycles > 10000)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "rel_tol >= 0 and max_vcycles in [0,10000] required");
    if (p->dc_vcycles < 1 || p->dc_vcycles > 8)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "dc_vcycles must be in [1, 8]");
    if (p->bc_mode != QUMOND_BC_ZERO && p->bc_mode != QUMOND_BC_GIVEN)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "unknown bc_mode");
    if (p->warm_start != 0 && p->warm_start != 1)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "warm_start must be 0 or 1");
    if (box > 0 && p->box_ratio != 2 && p->box_ratio != 4 && p->box_ratio != 8)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "box_ratio must be 2, 4 or 8");
    if (box > 0 && n < 2 * p->box_ratio)
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "n too small for nested boxes of this ratio");
    if (!is_device_ptr(src) || !is_device_ptr(phi))
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "src and phi must be device pointers");
    if (box > 0 && !is_device_ptr(phi_parent))
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "box >= 1 needs the parent potential (device pointer)");
    if (src == phi || (box > 0 && phi_parent == phi))
        return set_err(err, err_len, QUMOND_ERR_INVALID_ARG, "phi must not alias its inputs");

    void* base = nullptr;
    cudaError_t ce = scratch_address(&base);
    if (ce != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(msg, sizeof(msg), "scratch address lookup: %s", cudaGetErrorString(ce));
        return set_err(err, err_len, QUMOND_ERR_CUDA, msg);
    }

    Solver S;
    S.p = p;
    S.s = reinterpret_cast<cudaStream_t>(stream);
    while ((2 << S.L) < n) ++S.L;
    while ((2 << S.lc) < kCoarseN && S.lc < S.L) ++S.lc;
    int ratio_log = 0;
    while ((1 << ratio_log) < p->box_ratio) ++ratio_log;
    S.h = std::ldexp(p->L0, -box * ratio_log) / (double)n;
    unsigned char* cur = static_cast<unsigned char*>(base);
    for (int l = 0; l <= S.L; ++l) {
        S.lev[l].v = make_view(2 << l);
        if (l < S.lc) continue;
        const size_t half = (size_t)(2 * S.lev[l].v.cs) * sizeof(float);
        S.lev[l].e = reinterpret_cast<float*>(cur);
        S.lev[l].f = reinterpret_cast<float*>(cur + half);
        cur += round256(2 * half);
    }
    S.partials = reinterpret_cast<double*>(cur);
    cur += round256(sizeof(double) * 2 * (size_t)(residual_blocks(n > 2 ? n : 2) + 1));
    S.norms = reinterpret_cast<double*>(cur);
    cur += 256;
    const size_t used = (size_t)(cur - static_cast<unsigned char*>(base));

    // the previous call's contents must not leak into this one
    ce = cudaMemsetAsync(base, 0, used, S.s);
    if (ce == cudaSuccess) {
        if (box > 0) launch_boundary_from_parent(phi_parent, phi, n, p->box_ratio, S.s);
        else if (p->bc_mode == QUMOND_BC_ZERO) launch_boundary_zero(phi, n, S.s);
        if (!p->warm_start) {
            launch_convert_rhs<float>(src, 1.0, n, S.lev[S.L].f, S.lev[S.L].v, S.s);
            ce = S.fmg(phi);
            if (ce == cudaSuccess) {
                launch_assign_outer<float>(phi, n, S.lev[S.L].e, S.lev[S.L].v, false, S.s);
                launch_set_boundary<float>(S.lev[S.L].e, S.lev[S.L].v, nullptr, n, S.s);
            }
        }
        if (ce == cudaSuccess) ce = cudaGetLastError();
    }
    if (ce != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(msg, sizeof(msg), "launch: %s", cudaGetErrorString(ce));
        return set_err(err, err_len, QUMOND_ERR_CUDA, msg);
    }
    const bool refine = p->rel_tol > 0.0 && p->max_vcycles > 0;
    if (!refine && !stats) return QUMOND_OK;
    double rr = 0.0, ff = 0.0;
    ce = S.norms_of(phi, src, &rr, &ff);
    const double denom = ff > 0.0 ? std::sqrt(ff) : 1.0;
    double rel = std::sqrt(rr) / denom;
    const double rel0 = rel;
    int made = 0;
    while (ce == cudaSuccess && refine && rel > p->rel_tol && made < p->max_vcycles && std::isfinite(rel)) {
        for (int q = 0; q < p->dc_vcycles && ce == cudaSuccess; ++q) ce = S.vcycle(S.L, q == 0);
        if (ce != cudaSuccess) break;
        launch_assign_outer<float>(phi, n, S.lev[S.L].e, S.lev[S.L].v, true, S.s);
        made += p->dc_vcycles;
        ce = S.norms_of(phi, src, &rr, &ff);
        rel = std::sqrt(rr) / denom;
    }
    if (ce != cudaSuccess) {
        (void)cudaGetLastError();
        snprintf(msg, sizeof(msg), "solve: %s", cudaGetErrorString(ce));
        return set_err(err, err_len, QUMOND_ERR_CUDA, msg);
    }
    const bool ok = std::isfinite(rel) && (!refine || rel <= p->rel_tol);
    if (stats) {
        stats->vcycles = made;
        stats->converged = ok ? 1 : 0;
        stats->rel_residual_fmg = rel0;
        stats->rel_residual = rel;
    }
    if (!ok) {
        snprintf(msg, sizeof(msg), "relative residual %.3e after %d V-cycles (tol %.3e)", rel, made, p->rel_tol);
        return set_err(err, err_len, QUMOND_ERR_NOT_CONVERGED, msg);
    }
    return QUMOND_OK;
}
