// C ABI of the QUMOND path (include/qumond.h): argument checks, the
// context's multigrid scratch, and the host-side schedule of the full
// multigrid solves (Section 2).
#include "qumond.h"
#include "qumond_internal.h"

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace qumond;

namespace {

struct Level {
    LevelView v;
    void* e = nullptr;  // iterate / correction, 2 colours
    void* f = nullptr;  // right-hand side, 2 colours
    RbMaps maps;        // TMA descriptors of e (FP32 levels with n >= 64)
};

// Kernel classes of the tracer.
enum Kind {
    K_DEPOSIT, K_FIXED_TO_RHO, K_BOUNDARY, K_CONVERT_RHS, K_RESTRICT_FULL, K_COARSE, K_RB_FINEST, K_RB_COARSER,
    K_RESTRICT_RESID, K_PROLONG, K_SET_BOUNDARY, K_ASSIGN_OUTER, K_RESIDUAL_OUTER, K_REDUCE, K_SOURCE, K_FORCES,
    K_ROTATION_CURVE, K_FIXED_SETUP, K_FIXED_OUTPUT, K_CHI2, K_PROFILE, K_VSUB, K_FAR_FIELD, K_COUNT
};
const char* const kKindNames[K_COUNT] = {
    "cic_deposit", "fixed_to_rho", "boundary_fill", "convert_rhs", "restrict_full", "coarse_solver",
    "rb_half_finest", "rb_half_coarser", "restrict_resid_red", "prolong_black", "set_boundary", "update_outer",
    "residual_outer", "reduce_norms", "qumond_source", "forces", "rotation_curve", "fixed_setup", "fixed_output", "chi2", "profile", "vcycle_small_levels",
    "far_field",
};
constexpr int kMaxTimed = 32768;

// Launch counts of a sequence of kernels (a captured graph phase).
struct Phase {
    long long launches[K_COUNT] = {};
    double bytes[K_COUNT] = {};
    long long cell_updates = 0;
};

struct Tracer {
    bool on = false;
    std::vector<cudaEvent_t> ev;  // 2 per timed launch
    std::vector<int> kind_of;     // per timed launch
    long long launches[K_COUNT] = {};
    double bytes[K_COUNT] = {};
    double ms[K_COUNT] = {};
    long long timed[K_COUNT] = {};
    double timed_bytes[K_COUNT] = {};
    std::vector<double> kind_bytes;  // per timed launch (one-by-one mode)
    long long cell_updates = 0;
    int only = -1;          // timing on: -1 every class (launches one by one), else this class only
    Phase* sink = nullptr;  // while capturing: counts go here
    // while capturing a preamble with timing on: event pairs recorded into the graph
    std::vector<cudaEvent_t>* cap_events = nullptr;
    std::vector<int>* cap_kinds = nullptr;  // per event pair: number of launches it brackets
    std::vector<double>* cap_bytes = nullptr;  // per event pair: algorithmic bytes it brackets
    bool run_open = false;
    int run_count = 0;
    double run_bytes = 0.0;

    // a phase run `times` times; its bytes and cell updates count `work` times
    // (with several sets, the sets whose correction stopped skip later runs)
    void add(const Phase& ph, long long times, double work)
    {
        for (int k = 0; k < K_COUNT; ++k) {
            launches[k] += ph.launches[k] * times;
            bytes[k] += ph.bytes[k] * work;
        }
        cell_updates += (long long)((double)ph.cell_updates * work);
    }
};

// One captured solve: the preamble (boundary values, FMG, first residual
// check) and, in tolerance mode, a WHILE node whose body is one V-cycle of
// the defect correction plus its residual check.
struct SolveGraph {
    int kind = -1;  // 0 Newton, 1 QUMOND
    int box = -1;
    const double* rhs = nullptr;
    const double* parent = nullptr;
    double* u = nullptr;
    bool norms = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Phase pre, body;
    unsigned long long last_use = 0;
    int timed_class = -1;             // class bracketed by event nodes in the preamble, or -1
    std::vector<cudaEvent_t> events;  // 2 per bracketed run of timed_class launches
    std::vector<int> event_kinds;     // launches in each run
    std::vector<double> event_bytes;  // algorithmic bytes of each run
};
constexpr size_t kMaxGraphs = 64;

}  // namespace

struct qumond_ctx {
    qumond_params p;
    int L = 0;   // finest level index: n = 2 << L
    int lc = 0;  // level handed to the coarse-grid kernel
    size_t elt = 4;
    std::vector<Level> lev;  // index l = 0..L; only l >= lc allocated
    double* partials = nullptr;
    int max_partials = 0;
    double* d_norms = nullptr;
    double* h_norms = nullptr;  // pinned
    SolveState* d_state = nullptr;
    SolveState* h_state = nullptr;  // pinned
    int64_t* Ufix = nullptr;        // fixed-point master iterate (QUMOND_PREC_MIXED_FIXED), buffer 0
    int64_t* Ufix2 = nullptr;       // its second buffer (the iterate alternates: current = buffer it & 1)
    FixedMaps fmaps{};              // TMA descriptors of the fixed-point arrays (n >= 128)
    int nsets = 1;                  // independent problems of this shape (every array holds nsets of them)
    long long pstride = 0;          // doubles between two sets' partial norms
    bool in_body = false;           // enqueueing a defect-correction V-cycle (sets that stopped are skipped)
    int vtop = -1;                  // top level of the cooperative small-level V-cycle kernel, -1: not used
    int vgrid = 0;                  // its CTAs (one per SM)
    int vcs = 0;                    // persistent_vcycle = 2 or 3: CTAs of the cluster that runs it (per set)
    unsigned* vbar = nullptr;       // its grid-barrier counter
    long long barrier_polls = 1LL << 26;  // polls before one of its grid barriers gives up
    int64_t* Ffix = nullptr;        // fixed-point right-hand side
    unsigned* maxbits = nullptr;
    int* fault = nullptr;           // set by kernels whose bounded waits ran out
    double* ff = nullptr;           // far-field reductions (QUMOND_BC_MULTIPOLE)
    cudaStream_t cap_stream = nullptr;
    std::vector<SolveGraph> graphs;
    unsigned long long use_clock = 0;
    Tracer tr;
    std::string err;
};

namespace {

qumond_status fail(qumond_ctx* c, qumond_status st, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

qumond_status cuda_fail(qumond_ctx* c, cudaError_t e, const char* where)
{
    (void)cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? QUMOND_ERR_OUT_OF_MEMORY : QUMOND_ERR_CUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

#define CUDA_TRY(ctx, expr, where)                                                                                     \
    do {                                                                                                               \
        cudaError_t _e = (expr);                                                                                       \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, where);                                                       \
    } while (0)

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Device (or managed) memory check: a host pointer handed to a kernel would
// fault, so it is refused before anything is launched.
bool device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

qumond_status check_params(qumond_ctx* c, const qumond_params* p)
{
    if (!p) return fail(c, QUMOND_ERR_INVALID_ARG, "params is NULL");
    if (!is_pow2(p->n) || p->n < 2 || p->n > 1024) return fail(c, QUMOND_ERR_INVALID_ARG, "n=%d: need a power of two in [2, 1024]", p->n);
    if (p->nboxes < 1 || p->nboxes > kMaxBoxes) return fail(c, QUMOND_ERR_INVALID_ARG, "nboxes=%d: need 1..%d", p->nboxes, kMaxBoxes);
    if (!(p->L0 > 0.0) || !std::isfinite(p->L0)) return fail(c, QUMOND_ERR_INVALID_ARG, "L0 must be positive and finite");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->center[a])) return fail(c, QUMOND_ERR_INVALID_ARG, "center must be finite");
    if (!(p->G > 0.0) || !std::isfinite(p->G)) return fail(c, QUMOND_ERR_INVALID_ARG, "G must be positive");
    if (!(p->a0 >= 0.0) || !std::isfinite(p->a0)) return fail(c, QUMOND_ERR_INVALID_ARG, "a0 must be >= 0");
    if (p->npre < 1 || p->npost < 1 || p->npre > 16 || p->npost > 16)
        return fail(c, QUMOND_ERR_INVALID_ARG, "npre, npost must be in [1, 16]");
    if (p->ncycle < 1 || p->ncycle > 128) return fail(c, QUMOND_ERR_INVALID_ARG, "ncycle must be in [1, 128]");
    if (!(p->rel_tol >= 0.0)) return fail(c, QUMOND_ERR_INVALID_ARG, "rel_tol must be >= 0");
    if (p->max_vcycles < 0 || p->max_vcycles > 10000) return fail(c, QUMOND_ERR_INVALID_ARG, "max_vcycles must be in [0, 10000]");
    if (p->precision != QUMOND_PREC_FP64 && p->precision != QUMOND_PREC_MIXED && p->precision != QUMOND_PREC_MIXED_FIXED)
        return fail(c, QUMOND_ERR_INVALID_ARG, "unknown precision %d", p->precision);
    if (p->bc_mode != QUMOND_BC_ZERO && p->bc_mode != QUMOND_BC_GIVEN && p->bc_mode != QUMOND_BC_MULTIPOLE)
        return fail(c, QUMOND_ERR_INVALID_ARG, "unknown bc_mode %d", p->bc_mode);
    if (p->warm_start != 0 && p->warm_start != 1) return fail(c, QUMOND_ERR_INVALID_ARG, "warm_start must be 0 or 1");
    if (p->deposit_shift < 0 || p->deposit_shift > 40) return fail(c, QUMOND_ERR_INVALID_ARG, "deposit_shift must be in [0, 40]");
    if (!(p->rc_box_frac > 0.0) || !(p->rc_box_frac <= 0.5)) return fail(c, QUMOND_ERR_INVALID_ARG, "rc_box_frac must be in (0, 0.5]");
    if (p->box_ratio != 2 && p->box_ratio != 4 && p->box_ratio != 8)
        return fail(c, QUMOND_ERR_INVALID_ARG, "box_ratio must be 2, 4 or 8");
    if (p->use_graphs != 0 && p->use_graphs != 1) return fail(c, QUMOND_ERR_INVALID_ARG, "use_graphs must be 0 or 1");
    if (p->persistent_vcycle < 0 || p->persistent_vcycle > 3)
        return fail(c, QUMOND_ERR_INVALID_ARG, "persistent_vcycle must be 0, 1, 2 or 3");
    if (p->small_cluster != 0 && p->small_cluster != 4 && p->small_cluster != 8 && p->small_cluster != 16)
        return fail(c, QUMOND_ERR_INVALID_ARG, "small_cluster must be 0, 4, 8 or 16");
    if (p->dc_vcycles < 1 || p->dc_vcycles > 8) return fail(c, QUMOND_ERR_INVALID_ARG, "dc_vcycles must be in [1, 8]");
    if (p->nboxes > 1 && p->n < 2 * p->box_ratio)
        return fail(c, QUMOND_ERR_INVALID_ARG, "n=%d too small for nested boxes of ratio %d", p->n, p->box_ratio);
    if (p->nsets < 1 || p->nsets > 1024 || (long long)p->nsets * (p->n + 1) > 65535)
        return fail(c, QUMOND_ERR_INVALID_ARG, "nsets=%d: need 1 <= nsets <= 1024 and nsets * (n + 1) <= 65535",
                    p->nsets);
    if (p->tile_small < 0 || p->tile_small > 2) return fail(c, QUMOND_ERR_INVALID_ARG, "tile_small must be 0, 1 or 2");
    if (p->nsets > 1 && p->persistent_vcycle == 1)
        return fail(c, QUMOND_ERR_INVALID_ARG, "persistent_vcycle = 1 needs nsets = 1");
    return QUMOND_OK;
}

inline int log2i(int v) { int r = 0; while ((1 << r) < v) ++r; return r; }
inline double box_side(const qumond_ctx* c, int box) { return std::ldexp(c->p.L0, -box * log2i(c->p.box_ratio)); }
inline double box_h(const qumond_ctx* c, int box) { return box_side(c, box) / (double)c->p.n; }
inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// --- the solver schedule ----------------------------------------------------
template <typename T>
T* E(qumond_ctx* c, int l) { return static_cast<T*>(c->lev[l].e); }
template <typename T>
T* F(qumond_ctx* c, int l) { return static_cast<T*>(c->lev[l].f); }

inline double level_h(const qumond_ctx* c, int box, int l) { return box_h(c, box) * (double)(1 << (c->L - l)); }

inline double cube(int n) { return (double)(n + 1) * (double)(n + 1) * (double)(n + 1); }

inline void close_run(Tracer& t, cudaStream_t s)
{
    cudaEvent_t e1 = nullptr;
    if (cudaEventCreate(&e1) == cudaSuccess) {
        cudaEventRecordWithFlags(e1, s, cudaEventRecordExternal);
        t.cap_events->push_back(e1);
        t.cap_kinds->push_back(t.run_count);
        t.cap_bytes->push_back(t.run_bytes);
    } else {
        t.cap_events->pop_back();
    }
    t.run_open = false;
}

// Every launch goes through here: counted, and bracketed by events while
// timing is on.
template <class Launch>
void run(qumond_ctx* c, int kind, double bytes, cudaStream_t s, Launch&& launch)
{
    Tracer& t = c->tr;
    bytes *= c->nsets;  // every launch covers all sets
    if (t.sink) {
        // timing one class inside a captured graph: one event pair per run of
        // consecutive launches of that class (event-record nodes cost several
        // microseconds each, so they bracket runs rather than single launches)
        if (t.cap_events) {
            if (kind == t.only && !t.run_open) {
                cudaEvent_t e0 = nullptr;
                if (cudaEventCreate(&e0) == cudaSuccess) {
                    cudaEventRecordWithFlags(e0, s, cudaEventRecordExternal);  // becomes an event-record node
                    t.cap_events->push_back(e0);
                    t.run_open = true;
                    t.run_count = 0;
                    t.run_bytes = 0.0;
                }
            } else if (kind != t.only && t.run_open) {
                close_run(t, s);
            }
        }
        launch();
        if (t.run_open && kind == t.only) {
            t.run_count += 1;
            t.run_bytes += bytes;
        }
        t.sink->launches[kind] += 1;
        t.sink->bytes[kind] += bytes;
        return;
    }
    const size_t slot = t.kind_of.size();
    const bool rec = t.on && (t.only < 0 || kind == t.only) && slot < (size_t)kMaxTimed;
    if (rec) cudaEventRecord(t.ev[2 * slot], s);
    launch();
    if (rec) {
        cudaEventRecord(t.ev[2 * slot + 1], s);
        t.kind_of.push_back(kind);
        t.kind_bytes.push_back(bytes);
    }
    t.launches[kind] += 1;
    t.bytes[kind] += bytes;
}

inline Sets sets_of(const qumond_ctx* c)
{
    Sets st;
    st.n = c->nsets;
    st.act = (c->in_body && c->nsets > 1) ? c->d_state : nullptr;
    st.pstride = c->pstride;
    st.tile_small = c->p.tile_small;
    return st;
}

inline void count_cells(qumond_ctx* c, long long n)
{
    n *= c->nsets;
    if (c->tr.sink) c->tr.sink->cell_updates += n;
    else c->tr.cell_updates += n;
}

template <typename T>
void rb(qumond_ctx* c, int l, int colour, bool zero, double h, cudaStream_t s)
{
    const int n = c->lev[l].v.n;
    const double nodes = cube(n);
    count_cells(c, ((long long)(n - 1) * (n - 1) * (n - 1) + (colour == 0 ? 1 : 0)) / 2);
    run(c, l == c->L ? K_RB_FINEST : K_RB_COARSER, (zero ? 1.0 : 1.5) * nodes * sizeof(T), s, [&] {
        if (sizeof(T) == sizeof(float) && !zero && c->lev[l].maps.ok)
            launch_rb_half_tma(reinterpret_cast<float*>(E<T>(c, l)), reinterpret_cast<const float*>(F<T>(c, l)),
                               c->lev[l].v, colour, c->lev[l].maps, h, c->fault, s, sets_of(c));
        else
            launch_rb_half<T>(E<T>(c, l), F<T>(c, l), c->lev[l].v, colour, zero, h, s, sets_of(c));
    });
}

// The first pre-smoothing sweep of a correction that starts from zero, both
// half-sweeps in one launch, on the FP32 levels whose black half-sweep has no
// TMA form (the same bits as rb() for colour 0 from zero, then colour 1).
// Returns false where it does not apply.
template <typename T>
bool rb_first(qumond_ctx* c, int l, double h, cudaStream_t s)
{
    if (sizeof(T) != sizeof(float) || c->lev[l].v.n < 8 || c->lev[l].maps.ok) return false;
    const int n = c->lev[l].v.n;
    const long long inner = (long long)(n - 1) * (n - 1) * (n - 1);
    count_cells(c, (inner + 1) / 2 + inner / 2);
    run(c, l == c->L ? K_RB_FINEST : K_RB_COARSER, 2.0 * cube(n) * sizeof(T), s, [&] {
        launch_rb_first(reinterpret_cast<float*>(E<T>(c, l)), reinterpret_cast<const float*>(F<T>(c, l)),
                        c->lev[l].v, h, s, sets_of(c));
    });
    return true;
}

template <typename T>
void prolong(qumond_ctx* c, int l, bool add, cudaStream_t s)
{
    const double nodes = cube(c->lev[l].v.n);
    run(c, K_PROLONG, ((add ? 1.0 : 0.5) + 0.125) * nodes * sizeof(T), s,
        [&] {
            if (sizeof(T) == sizeof(float) && add && c->lev[l].maps.pok)
                launch_prolong_tma(reinterpret_cast<float*>(E<T>(c, l)), c->lev[l].v, c->lev[l].maps, c->fault, s,
                                   sets_of(c));
            else
                launch_prolong_black<T>(E<T>(c, l - 1), c->lev[l - 1].v, E<T>(c, l), c->lev[l].v, add, s, sets_of(c));
        });
}

template <typename T>
void set_bnd(qumond_ctx* c, int l, const double* u64, cudaStream_t s)
{
    const double nb = 6.0 * (c->lev[l].v.n + 1) * (double)(c->lev[l].v.n + 1);
    run(c, K_SET_BOUNDARY, nb * (sizeof(T) + (u64 ? 8.0 : 0.0)), s,
        [&] { launch_set_boundary<T>(E<T>(c, l), c->lev[l].v, u64, c->p.n, s, sets_of(c)); });
}

template <typename T>
cudaError_t coarse(qumond_ctx* c, int box, int fmg_mode, const double* u64, cudaStream_t s)
{
    const int l = c->lc;
    const int n = c->lev[l].v.n;
    long long upd = 0;  // red-black updates inside the kernel (approximate count of its sweeps)
    for (int m = 4; m <= n; m *= 2) upd += (long long)(c->p.npre + c->p.npost) * (m - 1) * (m - 1) * (m - 1);
    count_cells(c, fmg_mode ? upd * c->p.ncycle : upd);
    cudaError_t err = cudaSuccess;
    run(c, K_COARSE, 2.0 * cube(n) * sizeof(T), s, [&] {
        err = launch_coarse<T>(fmg_mode, E<T>(c, l), F<T>(c, l), c->lev[l].v, level_h(c, box, l), u64, c->p.n,
                               c->p.ncycle, c->p.npre, c->p.npost, s, sets_of(c));
    });
    return err;
}

// The V-cycle from level vtop down, as one cooperative kernel.
template <typename T>
cudaError_t vsub(qumond_ctx* c, int box, bool zero_top, cudaStream_t s)
{
    const qumond_params& p = c->p;
    T* e[8];
    T* f[8];
    LevelView v[8];
    double h[8];
    double bytes = 2.0 * cube(c->lev[c->lc].v.n) * sizeof(T);
    long long upd = 0;
    for (int m = 4; m <= c->lev[c->lc].v.n; m *= 2) upd += (long long)(p.npre + p.npost) * (m - 1) * (m - 1) * (m - 1);
    const int nlev = c->vtop - c->lc + 1;
    for (int q = 0; q < nlev; ++q) {
        const int l = c->lc + q;
        e[q] = E<T>(c, l);
        f[q] = F<T>(c, l);
        v[q] = c->lev[l].v;
        h[q] = level_h(c, box, l);
        if (q > 0) {
            const double nodes = cube(v[q].n);
            bytes += ((3.0 * (p.npre + p.npost) - 0.5) + 1.625 + 1.125) * nodes * sizeof(T);
            upd += (long long)(p.npre + p.npost) * (v[q].n - 1) * (v[q].n - 1) * (v[q].n - 1);
        }
    }
    count_cells(c, upd);
    cudaError_t err = cudaSuccess;
    run(c, K_VSUB, bytes, s, [&] {
        if constexpr (sizeof(T) == sizeof(float)) {
            if (p.persistent_vcycle == 3) {
                err = launch_vslab(reinterpret_cast<float*>(e[1]), reinterpret_cast<const float*>(f[1]), v[1], h[1],
                                   h[0], zero_top ? 1 : 0, p.npre, p.npost, c->vcs, s, sets_of(c));
                return;
            }
        }
        if (p.persistent_vcycle == 2)
            err = launch_vcluster<T>(e, f, v, h, nlev, zero_top ? 1 : 0, p.npre, p.npost, c->vcs, s, sets_of(c));
        else
            err = launch_vsub<T>(e, f, v, h, nlev, zero_top ? 1 : 0, p.npre, p.npost, c->vbar, c->fault,
                                 c->barrier_polls, c->vgrid, s);
    });
    return err;
}

// One V-cycle at level l on the correction problem held in lev[l] (for l <
// L the initial guess is zero; at l = L the caller says so).
template <typename T>
cudaError_t vcycle(qumond_ctx* c, int box, int l, bool zero_guess, cudaStream_t s)
{
    const qumond_params& p = c->p;
    const double h = level_h(c, box, l);
    if (l <= c->lc) return coarse<T>(c, box, 0, nullptr, s);
    if (l == c->vtop) return vsub<T>(c, box, zero_guess, s);
    for (int q = 0; q < p.npre; ++q) {
        if (zero_guess && q == 0 && rb_first<T>(c, l, h, s)) continue;
        rb<T>(c, l, 0, zero_guess && q == 0, h, s);
        rb<T>(c, l, 1, false, h, s);
    }
    const double nodes = cube(c->lev[l].v.n);
    run(c, K_RESTRICT_RESID, (1.5 + 0.125) * nodes * sizeof(T), s, [&] {
        if (sizeof(T) == sizeof(float) && c->lev[l].maps.ok)
            launch_restrict_tma(reinterpret_cast<float*>(F<T>(c, l - 1)), c->lev[l].v, c->lev[l - 1].v, c->lev[l].maps,
                                h, c->fault, s, sets_of(c));
        else
            launch_restrict_resid_red<T>(E<T>(c, l), F<T>(c, l), c->lev[l].v, F<T>(c, l - 1), c->lev[l - 1].v, h, s,
                                         sets_of(c));
    });
    cudaError_t err = vcycle<T>(c, box, l - 1, true, s);
    if (err != cudaSuccess) return err;
    prolong<T>(c, l, true, s);
    for (int q = 0; q < p.npost; ++q) {
        rb<T>(c, l, 0, false, h, s);
        rb<T>(c, l, 1, false, h, s);
    }
    return cudaSuccess;
}

// Full multigrid (Section 2) on lev[L].f with the boundary values of u64:
// the right-hand side is restricted level by level, the coarse-grid kernel
// solves up to level lc, and each finer level is interpolated and given
// ncycle V-cycles.  Coarser levels take the finest boundary values at the
// same positions; a level becomes a zero-boundary correction level once the
// next finer level has been interpolated from it.
template <typename T>
cudaError_t fmg(qumond_ctx* c, int box, const double* u64, cudaStream_t s)
{
    const qumond_params& p = c->p;
    for (int l = c->L - 1; l >= c->lc; --l) {
        const double nodes = cube(c->lev[l + 1].v.n);
        run(c, K_RESTRICT_FULL, 1.125 * nodes * sizeof(T), s, [&] {
            launch_restrict_full<T>(F<T>(c, l + 1), c->lev[l + 1].v, F<T>(c, l), c->lev[l].v, s, sets_of(c));
        });
    }
    cudaError_t err = coarse<T>(c, box, 1, u64, s);
    if (err != cudaSuccess) return err;
    for (int l = c->lc + 1; l <= c->L; ++l) {
        set_bnd<T>(c, l, u64, s);
        prolong<T>(c, l, false, s);
        set_bnd<T>(c, l - 1, nullptr, s);
        for (int q = 0; q < p.ncycle; ++q) {
            err = vcycle<T>(c, box, l, false, s);
            if (err != cudaSuccess) return err;
        }
    }
    return cudaSuccess;
}

// Residual r = coef*rhs - L u into the finest level and the decision whether
// to continue (device-side; drives the graph's WHILE node when capturing).
inline bool fixed_mode(const qumond_ctx* c) { return c->p.precision == QUMOND_PREC_MIXED_FIXED; }

// defect-correction steps allowed by max_vcycles (dc_vcycles V-cycles each, the last one may go past it)
inline int dc_steps(const qumond_params& p) { return (p.max_vcycles + p.dc_vcycles - 1) / p.dc_vcycles; }

template <typename T>
void check(qumond_ctx* c, int box, const double* rhs, double coef, const double* u, bool first,
           const cudaGraphConditionalHandle* handle, cudaStream_t s)
{
    const qumond_params& p = c->p;
    int nb = residual_rows_blocks(p.n);
    if (fixed_mode(c)) {
        nb = fixed_residual_blocks(p.n);
        run(c, K_RESIDUAL_OUTER, cube(p.n) * 20.0, s, [&] {
            launch_fixed_residual(c->Ufix, c->Ffix, p.n, box_h(c, box), c->d_state, first,
                                  reinterpret_cast<float*>(F<T>(c, c->L)), c->lev[c->L].v, c->partials, s,
                                  sets_of(c));
        });
    } else {
        run(c, K_RESIDUAL_OUTER, cube(p.n) * (16.0 + sizeof(T)), s, [&] {
            launch_residual_rows<T>(u, rhs, coef, p.n, box_h(c, box), F<T>(c, c->L), c->lev[c->L].v, c->partials, s,
                                    sets_of(c));
        });
    }
    run(c, K_REDUCE, 16.0 * nb, s, [&] {
        launch_decide(c->partials, nb, c->d_state, p.rel_tol, dc_steps(p), first, p.rel_tol > 0.0 && p.max_vcycles > 0,
                      handle, c->fault, s, sets_of(c));
    });
}

// --- the solve, as a sequence of launches ------------------------------------
// Preamble: boundary values (from the parent box, or zero for box 0 in the
// paper's setup), FMG, and (when norms are wanted) the first residual check.
template <typename T>
cudaError_t enqueue_preamble(qumond_ctx* c, int box, const double* rhs, double coef, const double* parent, double* u,
                             bool norms, const cudaGraphConditionalHandle* handle, cudaStream_t s)
{
    const qumond_params& p = c->p;
    const int n = p.n;
    const double nodes = cube(n);
    const double nbnd = 6.0 * (n + 1) * (double)(n + 1);
    if (box > 0)
        run(c, K_BOUNDARY, nbnd * 16.0, s,
            [&] { launch_boundary_from_parent(parent, u, n, p.box_ratio, s, c->nsets); });
    else if (p.bc_mode == QUMOND_BC_ZERO)
        run(c, K_BOUNDARY, nbnd * 8.0, s, [&] { launch_boundary_zero(u, n, s, c->nsets); });
    const bool fixed = fixed_mode(c) && norms;
    if (!p.warm_start) {
        run(c, K_CONVERT_RHS, nodes * (8.0 + sizeof(T)), s,
            [&] { launch_convert_rhs<T>(rhs, coef, n, F<T>(c, c->L), c->lev[c->L].v, s, sets_of(c)); });
        cudaError_t err = fmg<T>(c, box, u, s);
        if (err != cudaSuccess) return err;
        if (!fixed)
            run(c, K_ASSIGN_OUTER, nodes * (8.0 + sizeof(T)), s,
                [&] { launch_assign_outer<T>(u, n, E<T>(c, c->L), c->lev[c->L].v, false, s, sets_of(c)); });
    }
    if (fixed) {
        const float* eL = reinterpret_cast<const float*>(E<T>(c, c->L));
        run(c, K_FIXED_SETUP, nodes * 32.0, s, [&] {
            launch_fixed_scale(eL, c->lev[c->L].v, u, n, p.warm_start != 0, c->maxbits, c->d_state, s, sets_of(c));
            launch_fixed_init(eL, c->lev[c->L].v, u, rhs, coef, box_h(c, box), n, p.warm_start != 0, c->d_state,
                              c->Ufix, c->Ufix2, c->Ffix, s, sets_of(c));
        });
    }
    if (!p.warm_start) set_bnd<T>(c, c->L, nullptr, s);
    if (norms) check<T>(c, box, rhs, coef, u, true, handle, s);
    return cudaGetLastError();
}

// After the defect correction (fixed-point mode): u = U 2^-S.
template <typename T>
cudaError_t enqueue_post(qumond_ctx* c, double* u, cudaStream_t s)
{
    if (!fixed_mode(c)) return cudaSuccess;
    run(c, K_FIXED_OUTPUT, cube(c->p.n) * 16.0, s,
        [&] { launch_fixed_output(c->Ufix, c->Ufix2, u, c->p.n, c->d_state, s, sets_of(c)); });
    return cudaGetLastError();
}

// Body of the defect correction: one V-cycle on L e = r from e = 0, u += e,
// and the residual check that decides whether to go on.
template <typename T>
cudaError_t enqueue_body(qumond_ctx* c, int box, const double* rhs, double coef, double* u,
                         const cudaGraphConditionalHandle* handle, cudaStream_t s)
{
    const int n = c->p.n;
    struct BodyFlag {  // kernels of this V-cycle skip the sets that have stopped
        qumond_ctx* c;
        explicit BodyFlag(qumond_ctx* cc) : c(cc) { c->in_body = true; }
        ~BodyFlag() { c->in_body = false; }
    } body_flag(c);
    for (int q = 0; q < c->p.dc_vcycles; ++q) {  // the first from e = 0, the others continue it
        cudaError_t err = vcycle<T>(c, box, c->L, q == 0, s);
        if (err != cudaSuccess) return err;
    }
    if (fixed_mode(c)) {
        // update and residual in one pass (U' into the other buffer), then the decision
        int nb = 0;
        run(c, K_RESIDUAL_OUTER, cube(n) * 32.0, s, [&] {
            if (c->fmaps.ok)
                nb = launch_fixed_update_residual_tma(c->Ufix, c->Ufix2, c->fmaps, n, box_h(c, box), c->d_state,
                                                      reinterpret_cast<float*>(F<T>(c, c->L)), c->lev[c->L].v,
                                                      c->partials, c->fault, s, sets_of(c));
            else
                nb = launch_fixed_update_residual(c->Ufix, c->Ufix2, c->Ffix,
                                                  reinterpret_cast<const float*>(E<T>(c, c->L)), n, box_h(c, box),
                                                  c->d_state, reinterpret_cast<float*>(F<T>(c, c->L)), c->lev[c->L].v,
                                                  c->partials, s, sets_of(c));
        });
        const qumond_params& p = c->p;
        run(c, K_REDUCE, 16.0 * nb, s, [&] {
            launch_decide(c->partials, nb, c->d_state, p.rel_tol, dc_steps(p), false,
                          p.rel_tol > 0.0 && p.max_vcycles > 0, handle, c->fault, s, sets_of(c));
        });
        return cudaGetLastError();
    }
    run(c, K_ASSIGN_OUTER, cube(n) * (16.0 + sizeof(T)), s,
        [&] { launch_assign_outer<T>(u, n, E<T>(c, c->L), c->lev[c->L].v, true, s, sets_of(c)); });
    check<T>(c, box, rhs, coef, u, false, handle, s);
    return cudaGetLastError();
}

SolveGraph* find_graph(qumond_ctx* c, int kind, int box, const double* rhs, const double* parent, double* u,
                       bool norms)
{
    const int timed_class = c->tr.on ? c->tr.only : -1;
    for (auto& g : c->graphs)
        if (g.kind == kind && g.box == box && g.rhs == rhs && g.parent == parent && g.u == u && g.norms == norms &&
            g.timed_class == timed_class)
            return &g;
    return nullptr;
}

void destroy_graph(SolveGraph& g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    for (cudaEvent_t e : g.events) cudaEventDestroy(e);
    g.events.clear();
    g.event_kinds.clear();
    g.event_bytes.clear();
    g.exec = nullptr;
    g.graph = nullptr;
}

// Captures the solve into a graph on the context's private stream.  The
// WHILE node's condition is set on the device by the residual check, so a
// launch runs FMG and every V-cycle the tolerance needs without the host.
template <typename T>
qumond_status capture(qumond_ctx* c, int kind, int box, const double* rhs, double coef, const double* parent,
                      double* u, bool norms, bool refine, SolveGraph* out)
{
    cudaStream_t cs = c->cap_stream;
    SolveGraph g;
    g.kind = kind;
    g.box = box;
    g.rhs = rhs;
    g.parent = parent;
    g.u = u;
    g.norms = norms;
    CUDA_TRY(c, cudaGraphCreate(&g.graph, 0), "graph create");
    cudaGraphConditionalHandle handle = 0;
    cudaError_t err = cudaSuccess;
    if (refine) err = cudaGraphConditionalHandleCreate(&handle, g.graph, 0, cudaGraphCondAssignDefault);
    std::vector<cudaGraphNode_t> tail;
    if (err == cudaSuccess) err = cudaStreamBeginCaptureToGraph(cs, g.graph, nullptr, nullptr, 0,
                                                                cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
        c->tr.sink = &g.pre;
        g.timed_class = c->tr.on ? c->tr.only : -1;
        if (g.timed_class >= 0) {
            c->tr.cap_events = &g.events;
            c->tr.cap_kinds = &g.event_kinds;
            c->tr.cap_bytes = &g.event_bytes;
        }
        cudaError_t e1 = enqueue_preamble<T>(c, box, rhs, coef, parent, u, norms, refine ? &handle : nullptr, cs);
        if (e1 == cudaSuccess && !refine && norms) e1 = enqueue_post<T>(c, u, cs);
        if (c->tr.run_open) close_run(c->tr, cs);
        c->tr.sink = nullptr;
        c->tr.cap_events = nullptr;
        c->tr.cap_kinds = nullptr;
        c->tr.cap_bytes = nullptr;
        if (refine && e1 == cudaSuccess) {
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            e1 = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
            if (e1 == cudaSuccess) tail.assign(deps, deps + nd);
        }
        cudaGraph_t captured = g.graph;
        cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
        err = e1 != cudaSuccess ? e1 : e2;
    }
    cudaGraphNode_t wnode = nullptr;
    if (err == cudaSuccess && refine) {
        // cudaGraphNodeParams has no usable default constructor: zeroed storage
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        memset(raw, 0, sizeof(raw));
        cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
        cp->type = cudaGraphNodeTypeConditional;
        cp->conditional.handle = handle;
        cp->conditional.type = cudaGraphCondTypeWhile;
        cp->conditional.size = 1;
        err = cudaGraphAddNode(&wnode, g.graph, tail.data(), nullptr, tail.size(), cp);
        if (err == cudaSuccess) {
            cudaGraph_t body = cp->conditional.phGraph_out[0];
            err = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                c->tr.sink = &g.body;
                cudaError_t e1 = enqueue_body<T>(c, box, rhs, coef, u, &handle, cs);
                c->tr.sink = nullptr;
                cudaGraph_t captured = body;
                cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
                err = e1 != cudaSuccess ? e1 : e2;
            }
        }
        if (err == cudaSuccess) {  // after the loop
            err = cudaStreamBeginCaptureToGraph(cs, g.graph, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                c->tr.sink = &g.pre;
                cudaError_t e1 = enqueue_post<T>(c, u, cs);
                c->tr.sink = nullptr;
                cudaGraph_t captured = g.graph;
                cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
                err = e1 != cudaSuccess ? e1 : e2;
            }
        }
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (err != cudaSuccess) {
        destroy_graph(g);
        return cuda_fail(c, err, "graph capture");
    }
    *out = g;
    return QUMOND_OK;
}

// Steps 2 and 4: boundary values, FMG, then defect correction to rel_tol.
//   r = coef*rhs - L u   (FP64, caller's arrays)
//   V-cycle on L e = r   (precision T, zero initial guess, zero boundary)
//   u += e               (FP64)
// Launched as one cached CUDA graph per (solve, box, arrays); with kernel
// timing on, the same launches are issued one by one and the host reads the
// residual after each V-cycle instead.
template <typename T>
qumond_status solve_t(qumond_ctx* c, int kind, int box, const double* rhs, double coef, const double* parent,
                      double* u, qumond_stats* st, cudaStream_t s)
{
    const qumond_params& p = c->p;
    const bool refine = p.rel_tol > 0.0 && p.max_vcycles > 0;
    const bool norms = refine || st != nullptr;
    const int ns = c->nsets;
    if (p.use_graphs && !(c->tr.on && c->tr.only < 0)) {
        SolveGraph* g = find_graph(c, kind, box, rhs, parent, u, norms);
        if (!g) {
            if (c->graphs.size() >= kMaxGraphs) {
                size_t oldest = 0;
                for (size_t q = 1; q < c->graphs.size(); ++q)
                    if (c->graphs[q].last_use < c->graphs[oldest].last_use) oldest = q;
                CUDA_TRY(c, cudaDeviceSynchronize(), "graph eviction");
                destroy_graph(c->graphs[oldest]);
                c->graphs.erase(c->graphs.begin() + oldest);
            }
            SolveGraph ng;
            qumond_status cs = capture<T>(c, kind, box, rhs, coef, parent, u, norms, refine, &ng);
            if (cs != QUMOND_OK) return cs;
            c->graphs.push_back(ng);
            g = &c->graphs.back();
        }
        g->last_use = ++c->use_clock;
        CUDA_TRY(c, cudaGraphLaunch(g->exec, s), "graph launch");
        c->tr.add(g->pre, 1, 1.0);
        if (!norms) return QUMOND_OK;
        CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, ns * sizeof(SolveState), cudaMemcpyDeviceToHost, s),
                 "state copy");
        CUDA_TRY(c, cudaStreamSynchronize(s), "solve");
        int most = 0;
        double all = 0.0;
        for (int q = 0; q < ns; ++q) {
            most = c->h_state[q].it > most ? c->h_state[q].it : most;
            all += c->h_state[q].it;
        }
        c->tr.add(g->body, most, all / ns);
        for (size_t q = 0; q < g->event_kinds.size(); ++q) {  // one pair per run of g->timed_class launches
            float ms = 0.0f;
            CUDA_TRY(c, cudaEventElapsedTime(&ms, g->events[2 * q], g->events[2 * q + 1]), "trace: elapsed");
            c->tr.ms[g->timed_class] += ms;
            c->tr.timed[g->timed_class] += g->event_kinds[q];
            c->tr.timed_bytes[g->timed_class] += g->event_bytes[q];
        }
    } else {
        CUDA_TRY(c, enqueue_preamble<T>(c, box, rhs, coef, parent, u, norms, nullptr, s), "solve launch");
        if (!norms) return QUMOND_OK;
        for (;;) {
            CUDA_TRY(c, cudaMemcpyAsync(c->h_state, c->d_state, ns * sizeof(SolveState), cudaMemcpyDeviceToHost, s),
                     "state copy");
            CUDA_TRY(c, cudaStreamSynchronize(s), "solve");
            bool any = false;
            for (int q = 0; q < ns; ++q) any = any || c->h_state[q].cont;
            if (!any) break;
            CUDA_TRY(c, enqueue_body<T>(c, box, rhs, coef, u, nullptr, s), "vcycle launch");
        }
        CUDA_TRY(c, enqueue_post<T>(c, u, s), "output launch");
    }
    for (int q = 0; q < ns; ++q)
        if (c->h_state[q].fault)
            return fail(c, QUMOND_ERR_TIMEOUT, "box %d: a kernel gave up waiting for its shared-memory pipeline", box);
    if (st)
        for (int q = 0; q < ns; ++q) {
            const SolveState& r = c->h_state[q];
            st[q].vcycles = r.it * p.dc_vcycles;
            st[q].converged = r.converged;
            st[q].rel_residual_fmg = r.rel0;
            st[q].rel_residual = r.rel;
        }
    for (int q = 0; q < ns; ++q) {
        const SolveState& r = c->h_state[q];
        if (!r.converged) {
            if (ns == 1)
                return fail(c, QUMOND_ERR_NOT_CONVERGED, "box %d: relative residual %.3e after %d V-cycles (tol %.3e)",
                            box, r.rel, r.it * p.dc_vcycles, p.rel_tol);
            return fail(c, QUMOND_ERR_NOT_CONVERGED,
                        "set %d, box %d: relative residual %.3e after %d V-cycles (tol %.3e)", q, box, r.rel,
                        r.it * p.dc_vcycles, p.rel_tol);
        }
    }
    return QUMOND_OK;
}

qumond_status solve(qumond_ctx* c, int box, const double* rhs, double coef, const double* parent, double* u,
                    qumond_stats* st, void* stream, const char* what)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    if (box < 0 || box >= c->p.nboxes) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: box %d out of range", what, box);
    if (!device_ptr(rhs) || !device_ptr(u)) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: rhs and phi must be device pointers", what);
    if (box > 0 && !device_ptr(parent)) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: box %d needs the parent potential (device)", what, box);
    if (rhs == u || (box > 0 && parent == u)) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: phi must not alias its inputs", what);
    const int kind = coef == 1.0 ? 1 : 0;
    if (c->p.precision == QUMOND_PREC_FP64) return solve_t<double>(c, kind, box, rhs, coef, parent, u, st, S(stream));
    return solve_t<float>(c, kind, box, rhs, coef, parent, u, st, S(stream));
}

BoxSet box_set(const qumond_ctx* c, const double* const* phis)
{
    BoxSet bs;
    memset(&bs, 0, sizeof(bs));
    bs.nboxes = c->p.nboxes;
    bs.n = c->p.n;
    for (int b = 0; b < c->p.nboxes; ++b) {
        const double L = box_side(c, b);
        bs.b[b].phi = phis[b];
        bs.b[b].L = L;
        bs.b[b].h = L / (double)c->p.n;
        bs.b[b].inv_h = (double)c->p.n / L;
        bs.b[b].xlo = c->p.center[0] - 0.5 * L;
        bs.b[b].ylo = c->p.center[1] - 0.5 * L;
        bs.b[b].zlo = c->p.center[2] - 0.5 * L;
    }
    return bs;
}

qumond_status check_phis(qumond_ctx* c, const double* const* phis, const char* what)
{
    if (!phis) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: phi_boxes is NULL", what);
    for (int b = 0; b < c->p.nboxes; ++b)
        if (!device_ptr(phis[b])) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: phi_boxes[%d] is not a device pointer", what, b);
    return QUMOND_OK;
}

}  // namespace

extern "C" {

void qumond_default_params(qumond_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->n = 256;
    p->nboxes = 1;
    p->L0 = 120000.0;
    p->G = 4.30e-3;
    p->a0 = 3.6;
    p->npre = 2;
    p->npost = 2;
    p->ncycle = 6;
    p->rel_tol = 0.0;
    p->max_vcycles = 50;
    p->precision = QUMOND_PREC_MIXED;
    p->bc_mode = QUMOND_BC_ZERO;
    p->warm_start = 0;
    p->deposit_shift = 24;
    p->rc_box_frac = 0.2;
    p->box_ratio = 2;
    p->use_graphs = 1;
    p->persistent_vcycle = 3;
    p->nsets = 1;
    p->tile_small = 0;
    p->small_cluster = 0;
    p->dc_vcycles = 2;
}

qumond_status qumond_create(const qumond_params* p, qumond_ctx** out)
{
    if (!out) return QUMOND_ERR_INVALID_ARG;
    *out = nullptr;
    qumond_ctx* c = new qumond_ctx();
    qumond_status st = check_params(c, p);
    if (st != QUMOND_OK) {
        delete c;
        return st;
    }
    c->p = *p;
    c->nsets = p->nsets;
    const size_t ns = (size_t)p->nsets;
    c->elt = p->precision == QUMOND_PREC_FP64 ? sizeof(double) : sizeof(float);  // FIXED smooths in FP32
    int L = 0;
    while ((2 << L) < p->n) ++L;
    c->L = L;
    int lc = 0;
    while ((2 << lc) < kCoarseN && lc < L) ++lc;
    c->lc = lc;
    c->lev.resize(L + 1);
    bool ok = true;
    for (int l = 0; l <= L; ++l) {
        c->lev[l].v = make_view(2 << l);
        if (l < lc) continue;
        const size_t bytes = (size_t)(2 * c->lev[l].v.cs) * c->elt * ns;
        if (cudaMalloc(&c->lev[l].e, bytes) != cudaSuccess || cudaMalloc(&c->lev[l].f, bytes) != cudaSuccess) {
            ok = false;
            break;
        }
        if (cudaMemset(c->lev[l].e, 0, bytes) != cudaSuccess || cudaMemset(c->lev[l].f, 0, bytes) != cudaSuccess) {
            ok = false;
            break;
        }
    }
    if (ok) {
        const int nrows = residual_rows_blocks(p->n > 2 ? p->n : 2);
        const int nouter = residual_outer_blocks(p->n > 2 ? p->n : 2);
        c->max_partials = nrows > nouter ? nrows : nouter;
        c->pstride = 2 * (long long)(c->max_partials + 1);
        ok = cudaMalloc(&c->partials, sizeof(double) * (size_t)c->pstride * ns) == cudaSuccess &&
             cudaMalloc(&c->d_norms, sizeof(double) * 2) == cudaSuccess &&
             cudaMallocHost(&c->h_norms, sizeof(double) * 2) == cudaSuccess &&
             cudaMalloc(&c->d_state, sizeof(SolveState) * ns) == cudaSuccess &&
             cudaMallocHost(&c->h_state, sizeof(SolveState) * ns) == cudaSuccess &&
             cudaMemset(c->d_state, 0, sizeof(SolveState) * ns) == cudaSuccess &&
             cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
             cudaMalloc(&c->fault, sizeof(int)) == cudaSuccess && cudaMemset(c->fault, 0, sizeof(int)) == cudaSuccess &&
             (p->bc_mode != QUMOND_BC_MULTIPOLE ||
              cudaMalloc(&c->ff, sizeof(double) * far_field_scratch_doubles(p->nsets)) == cudaSuccess) &&
             prepare_kernels() == cudaSuccess;
        if (ok && c->elt == sizeof(float))
            for (int l = lc; l <= L; ++l) {
                make_rb_maps(static_cast<float*>(c->lev[l].e), static_cast<float*>(c->lev[l].f), c->lev[l].v,
                             &c->lev[l].maps, (int)ns);
                if (l > 0)
                    make_prolong_maps(static_cast<float*>(c->lev[l - 1].e), c->lev[l - 1].v,
                                      static_cast<float*>(c->lev[l].e), c->lev[l].v, &c->lev[l].maps, (int)ns);
            }
        if (ok && p->precision == QUMOND_PREC_MIXED_FIXED) {
            const size_t nn = fixed_elems(p->n) * ns;
            const int nfix = fixed_residual_blocks(p->n > 2 ? p->n : 2);
            if (nfix > c->max_partials) ok = false;  // partial buffer sized above covers it
            ok = ok && cudaMalloc(&c->Ufix, nn * sizeof(int64_t)) == cudaSuccess &&
                 cudaMalloc(&c->Ufix2, nn * sizeof(int64_t)) == cudaSuccess &&
                 cudaMalloc(&c->Ffix, nn * sizeof(int64_t)) == cudaSuccess &&
                 cudaMemset(c->Ufix, 0, nn * sizeof(int64_t)) == cudaSuccess &&
                 cudaMemset(c->Ufix2, 0, nn * sizeof(int64_t)) == cudaSuccess &&
                 cudaMemset(c->Ffix, 0, nn * sizeof(int64_t)) == cudaSuccess &&
                 cudaMalloc(&c->maxbits, sizeof(unsigned) * ns) == cudaSuccess &&
                 cudaMemset(c->maxbits, 0, sizeof(unsigned) * ns) == cudaSuccess;
            if (ok && c->elt == sizeof(float)) {
                const int n = p->n;
                const long long items = (long long)((n - 1 + 31) / 32) * ((n - 1 + 7) / 8) * ((n - 1 + 15) / 16);
                if (items <= c->max_partials)
                    make_fixed_maps(c->Ufix, c->Ufix2, c->Ffix, static_cast<float*>(c->lev[L].e), c->lev[L].v,
                                    &c->fmaps, (int)ns);
            }
        }
    }
    if (ok && p->persistent_vcycle == 2) {
        // levels lc+1 .. vtop (n <= 64, below the finest) as one thread-block cluster per set
        int top = -1;
        for (int l = c->lc + 1; l < L; ++l)
            if (c->lev[l].v.n <= 64) top = l;
        const int cs = vcluster_size(p->precision == QUMOND_PREC_FP64);
        if (cs >= 2 && top > c->lc && top - c->lc + 1 <= 6) {
            c->vtop = top;
            c->vcs = cs;
        }
    }
    if (ok && p->persistent_vcycle == 3 && c->elt == sizeof(float) && lc + 1 < L && c->lev[lc + 1].v.n == 32) {
        // the 32-interval level (below the finest) and the levels under it in one cluster's shared memory
        const int cs = vslab_size(p->small_cluster ? p->small_cluster : 8);
        if (cs > 0) {
            c->vtop = lc + 1;
            c->vcs = cs;
        }
    }
    if (ok && p->persistent_vcycle == 1) {
        // levels lc+1 .. vtop (n <= 64, below the finest) in one cooperative kernel
        int dev = 0, coop = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int top = -1;
        for (int l = c->lc + 1; l < L; ++l)
            if (c->lev[l].v.n <= 64) top = l;
        if (coop && sms > 0 && top > c->lc && top - c->lc + 1 <= 6) {
            ok = cudaMalloc(&c->vbar, sizeof(unsigned)) == cudaSuccess;
            if (ok) {
                c->vtop = top;
                c->vgrid = vsub_grid(sms);
            }
        }
    }
    if (!ok) {
        (void)cudaGetLastError();
        qumond_destroy(c);
        return QUMOND_ERR_OUT_OF_MEMORY;
    }
    *out = c;
    return QUMOND_OK;
}

void qumond_destroy(qumond_ctx* c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    for (auto& l : c->lev) {
        if (l.e) cudaFree(l.e);
        if (l.f) cudaFree(l.f);
    }
    if (c->partials) cudaFree(c->partials);
    if (c->d_norms) cudaFree(c->d_norms);
    if (c->h_norms) cudaFreeHost(c->h_norms);
    if (c->d_state) cudaFree(c->d_state);
    if (c->fault) cudaFree(c->fault);
    if (c->ff) cudaFree(c->ff);
    if (c->Ufix) cudaFree(c->Ufix);
    if (c->Ufix2) cudaFree(c->Ufix2);
    if (c->vbar) cudaFree(c->vbar);
    if (c->Ffix) cudaFree(c->Ffix);
    if (c->maxbits) cudaFree(c->maxbits);
    if (c->h_state) cudaFreeHost(c->h_state);
    for (auto& g : c->graphs) destroy_graph(g);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaEvent_t e : c->tr.ev) cudaEventDestroy(e);
    (void)cudaGetLastError();
    delete c;
}

const char* qumond_last_error(const qumond_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

qumond_status qumond_deposit(qumond_ctx* c, int box, const double* x, const double* y, const double* z,
                             const double* mass, int64_t np, int64_t* rho_fixed, double* rho, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    if (box < 0 || box >= c->p.nboxes) return fail(c, QUMOND_ERR_INVALID_ARG, "deposit: box %d out of range", box);
    if (np < 0) return fail(c, QUMOND_ERR_INVALID_ARG, "deposit: np < 0");
    if (np > 0 && (!device_ptr(x) || !device_ptr(y) || !device_ptr(z) || !device_ptr(mass)))
        return fail(c, QUMOND_ERR_INVALID_ARG, "deposit: x, y, z, mass must be device pointers");
    if (!device_ptr(rho_fixed)) return fail(c, QUMOND_ERR_INVALID_ARG, "deposit: rho_fixed must be a device pointer");
    if (rho && !device_ptr(rho)) return fail(c, QUMOND_ERR_INVALID_ARG, "deposit: rho must be a device pointer or NULL");
    const int n = c->p.n;
    const long long count = (long long)(n + 1) * (n + 1) * (n + 1);
    const double L = box_side(c, box);
    const double inv_h = (double)n / L;
    cudaStream_t s = S(stream);
    CUDA_TRY(c, cudaMemsetAsync(rho_fixed, 0, sizeof(int64_t) * count * c->nsets, s), "deposit: clear");
    run(c, K_DEPOSIT, 32.0 * (double)np, s, [&] {
        launch_cic_deposit(x, y, z, mass, np, n, c->p.center[0] - 0.5 * L, c->p.center[1] - 0.5 * L,
                           c->p.center[2] - 0.5 * L, inv_h, std::ldexp(1.0, c->p.deposit_shift), rho_fixed, s,
                           c->nsets);
    });
    if (rho) {
        const double scale = std::ldexp(1.0, -c->p.deposit_shift) * (inv_h * inv_h * inv_h);
        run(c, K_FIXED_TO_RHO, 16.0 * (double)count, s,
            [&] { launch_fixed_to_rho(rho_fixed, rho, count * c->nsets, scale, s); });
    }
    CUDA_TRY(c, cudaGetLastError(), "deposit launch");
    return QUMOND_OK;
}

qumond_status qumond_solve_newton(qumond_ctx* c, int box, const double* rho, const double* phiN_parent, double* phiN,
                                  qumond_stats* stats, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    return solve(c, box, rho, 4.0 * M_PI * c->p.G, phiN_parent, phiN, stats, stream, "solve_newton");
}

qumond_status qumond_solve_mond(qumond_ctx* c, int box, const double* src, const double* phi_parent, double* phi,
                                qumond_stats* stats, void* stream)
{
    return solve(c, box, src, 1.0, phi_parent, phi, stats, stream, "solve_mond");
}

qumond_status qumond_source(qumond_ctx* c, int box, const double* phiN, double* src, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    if (box < 0 || box >= c->p.nboxes) return fail(c, QUMOND_ERR_INVALID_ARG, "source: box %d out of range", box);
    if (!device_ptr(phiN) || !device_ptr(src)) return fail(c, QUMOND_ERR_INVALID_ARG, "source: phiN and src must be device pointers");
    if (phiN == src) return fail(c, QUMOND_ERR_INVALID_ARG, "source: src must not alias phiN");
    run(c, K_SOURCE, 16.0 * cube(c->p.n), S(stream),
        [&] { launch_source(phiN, src, c->p.n, box_h(c, box), c->p.a0, S(stream), c->nsets); });
    CUDA_TRY(c, cudaGetLastError(), "source launch");
    return QUMOND_OK;
}

qumond_status qumond_forces(qumond_ctx* c, const double* const* phi_boxes, const double* qx, const double* qy,
                            const double* qz, int64_t nq, double* gx, double* gy, double* gz, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    qumond_status st = check_phis(c, phi_boxes, "forces");
    if (st != QUMOND_OK) return st;
    if (nq < 0) return fail(c, QUMOND_ERR_INVALID_ARG, "forces: nq < 0");
    if (nq == 0) return QUMOND_OK;
    if (!device_ptr(qx) || !device_ptr(qy) || !device_ptr(qz) || !device_ptr(gx) || !device_ptr(gy) || !device_ptr(gz))
        return fail(c, QUMOND_ERR_INVALID_ARG, "forces: point and force arrays must be device pointers");
    run(c, K_FORCES, 48.0 * (double)nq, S(stream),
        [&] { launch_forces(box_set(c, phi_boxes), qx, qy, qz, nq, gx, gy, gz, S(stream), c->nsets); });
    CUDA_TRY(c, cudaGetLastError(), "forces launch");
    return QUMOND_OK;
}

qumond_status qumond_rotation_curve(qumond_ctx* c, const double* const* phi_boxes, int nbins, double rmax, int nphi,
                                    double* r_out, double* vc_out, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    qumond_status st = check_phis(c, phi_boxes, "rotation_curve");
    if (st != QUMOND_OK) return st;
    if (nbins < 1 || nbins > 65535) return fail(c, QUMOND_ERR_INVALID_ARG, "rotation_curve: nbins must be in [1, 65535]");
    if (nphi < 1 || nphi > 1024) return fail(c, QUMOND_ERR_INVALID_ARG, "rotation_curve: nphi must be in [1, 1024]");
    if (!(rmax > 0.0) || !std::isfinite(rmax)) return fail(c, QUMOND_ERR_INVALID_ARG, "rotation_curve: rmax must be positive");
    if (!device_ptr(r_out) || !device_ptr(vc_out)) return fail(c, QUMOND_ERR_INVALID_ARG, "rotation_curve: outputs must be device pointers");
    run(c, K_ROTATION_CURVE, 16.0 * nbins, S(stream), [&] {
        launch_rotation_curve(box_set(c, phi_boxes), c->p.center[0], c->p.center[1], c->p.center[2], nbins, rmax,
                              nullptr, nphi, c->p.rc_box_frac, r_out, vc_out, S(stream), c->nsets);
    });
    CUDA_TRY(c, cudaGetLastError(), "rotation_curve launch");
    return QUMOND_OK;
}

qumond_status qumond_rotation_curve_sets(qumond_ctx* c, const double* const* phi_boxes, int nbins, const double* rmax,
                                         int nphi, double* r_out, double* vc_out, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    qumond_status st = check_phis(c, phi_boxes, "rotation_curve_sets");
    if (st != QUMOND_OK) return st;
    if (nbins < 1 || nbins > 65535) return fail(c, QUMOND_ERR_INVALID_ARG, "rotation_curve_sets: nbins must be in [1, 65535]");
    if (nphi < 1 || nphi > 1024) return fail(c, QUMOND_ERR_INVALID_ARG, "rotation_curve_sets: nphi must be in [1, 1024]");
    if (!device_ptr(rmax) || !device_ptr(r_out) || !device_ptr(vc_out))
        return fail(c, QUMOND_ERR_INVALID_ARG, "rotation_curve_sets: rmax and the outputs must be device pointers");
    run(c, K_ROTATION_CURVE, 16.0 * nbins, S(stream), [&] {
        launch_rotation_curve(box_set(c, phi_boxes), c->p.center[0], c->p.center[1], c->p.center[2], nbins, 0.0, rmax,
                              nphi, c->p.rc_box_frac, r_out, vc_out, S(stream), c->nsets);
    });
    CUDA_TRY(c, cudaGetLastError(), "rotation_curve_sets launch");
    return QUMOND_OK;
}

namespace {
qumond_status profile(qumond_ctx* c, const double* const* phi_boxes, int nbins, double rmax, int nphi, int mode,
                      double z_eval, double h, double* r_out, double* out, void* stream, const char* what)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    qumond_status st = check_phis(c, phi_boxes, what);
    if (st != QUMOND_OK) return st;
    if (nbins < 1 || nbins > 65535) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: nbins must be in [1, 65535]", what);
    if (nphi < 1 || nphi > 1024) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: nphi must be in [1, 1024]", what);
    if (!(rmax > 0.0) || !std::isfinite(rmax)) return fail(c, QUMOND_ERR_INVALID_ARG, "%s: rmax must be positive", what);
    if (mode == 1 && (!(z_eval > 0.0) || !(h > 0.0) || !std::isfinite(z_eval) || !std::isfinite(h)))
        return fail(c, QUMOND_ERR_INVALID_ARG, "%s: z_eval and h must be positive", what);
    if (!device_ptr(r_out) || !device_ptr(out))
        return fail(c, QUMOND_ERR_INVALID_ARG, "%s: outputs must be device pointers", what);
    run(c, K_PROFILE, 16.0 * nbins, S(stream), [&] {
        launch_profile(box_set(c, phi_boxes), c->p.center[0], c->p.center[1], c->p.center[2], nbins, rmax, nphi,
                       c->p.rc_box_frac, mode, c->p.a0, z_eval, h, r_out, out, S(stream), c->nsets);
    });
    CUDA_TRY(c, cudaGetLastError(), what);
    return QUMOND_OK;
}
}  // namespace

qumond_status qumond_rotation_curve_algebraic(qumond_ctx* c, const double* const* phiN_boxes, int nbins, double rmax,
                                              int nphi, double* r_out, double* vc_out, void* stream)
{
    return profile(c, phiN_boxes, nbins, rmax, nphi, 0, 0.0, 1.0, r_out, vc_out, stream, "rotation_curve_algebraic");
}

qumond_status qumond_sigma_z(qumond_ctx* c, const double* const* phi_boxes, int nbins, double rmax, int nphi,
                             double z_eval, double h, double* r_out, double* sigma_out, void* stream)
{
    return profile(c, phi_boxes, nbins, rmax, nphi, 1, z_eval, h, r_out, sigma_out, stream, "sigma_z");
}

qumond_status qumond_chi2(qumond_ctx* c, const double* vc, const double* v_obs, const double* sigma, int nbins,
                          int nsets, double* chi2, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    if (nbins < 1 || nsets < 0) return fail(c, QUMOND_ERR_INVALID_ARG, "chi2: need nbins >= 1 and nsets >= 0");
    if (nsets == 0) return QUMOND_OK;
    if (!device_ptr(vc) || !device_ptr(v_obs) || !device_ptr(sigma) || !device_ptr(chi2))
        return fail(c, QUMOND_ERR_INVALID_ARG, "chi2: every array must be a device pointer");
    run(c, K_CHI2, 8.0 * ((double)nbins * (nsets + 2) + nsets), S(stream),
        [&] { launch_chi2(vc, v_obs, sigma, nbins, nsets, chi2, S(stream)); });
    CUDA_TRY(c, cudaGetLastError(), "chi2 launch");
    return QUMOND_OK;
}

qumond_status qumond_set_barrier_poll_limit(qumond_ctx* c, int64_t polls)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    if (polls < 1) return fail(c, QUMOND_ERR_INVALID_ARG, "barrier poll limit must be >= 1");
    if (polls == c->barrier_polls) return QUMOND_OK;
    // the limit is an argument of the captured kernels: drop the cached graphs
    CUDA_TRY(c, cudaDeviceSynchronize(), "barrier poll limit");
    for (auto& g : c->graphs) destroy_graph(g);
    c->graphs.clear();
    c->barrier_polls = polls;
    return QUMOND_OK;
}

qumond_status qumond_far_field(qumond_ctx* c, const double* rho, double* phiN, double* phi, void* stream)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    if (c->p.bc_mode != QUMOND_BC_MULTIPOLE)
        return fail(c, QUMOND_ERR_INVALID_ARG, "far_field: the context's bc_mode is not QUMOND_BC_MULTIPOLE");
    if (!device_ptr(rho) || !device_ptr(phiN) || !device_ptr(phi))
        return fail(c, QUMOND_ERR_INVALID_ARG, "far_field: rho, phiN and phi must be device pointers");
    if (phiN == phi || rho == phiN || rho == phi)
        return fail(c, QUMOND_ERR_INVALID_ARG, "far_field: rho, phiN and phi must be distinct arrays");
    const double nodes = cube(c->p.n);
    const double nbnd = 6.0 * (c->p.n + 1) * (double)(c->p.n + 1);
    run(c, K_FAR_FIELD, 2.0 * 8.0 * nodes + 2.0 * 8.0 * nbnd, S(stream), [&] {
        launch_far_field(rho, c->p.n, box_side(c, 0), c->p.center[0], c->p.center[1], c->p.center[2], c->p.G,
                         c->p.a0, phiN, phi, c->ff, c->nsets, S(stream));
    });
    CUDA_TRY(c, cudaGetLastError(), "far_field launch");
    return QUMOND_OK;
}

int qumond_trace_classes(void) { return K_COUNT; }

qumond_status qumond_trace_timing(qumond_ctx* c, int on, int only_class)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    if (only_class < -1 || only_class >= K_COUNT) return fail(c, QUMOND_ERR_INVALID_ARG, "trace: no class %d", only_class);
    Tracer& t = c->tr;
    t.only = only_class;
    if (on) {
        if (t.ev.empty()) {
            t.ev.resize(2 * (size_t)kMaxTimed);
            for (auto& e : t.ev) CUDA_TRY(c, cudaEventCreate(&e), "trace: event create");
            t.kind_of.reserve(kMaxTimed);
        }
        CUDA_TRY(c, cudaDeviceSynchronize(), "trace: start");
        t.kind_of.clear();
        t.kind_bytes.clear();
        for (int k = 0; k < K_COUNT; ++k) {
            t.ms[k] = 0.0;
            t.timed[k] = 0;
            t.timed_bytes[k] = 0.0;
        }
    }
    t.on = on != 0;
    return QUMOND_OK;
}

qumond_status qumond_trace_read(qumond_ctx* c, qumond_kernel_stat* out, int cap, qumond_counters* totals, int reset)
{
    if (!c) return QUMOND_ERR_INVALID_ARG;
    c->err.clear();
    Tracer& t = c->tr;
    if (!t.kind_of.empty()) {
        CUDA_TRY(c, cudaEventSynchronize(t.ev[2 * (t.kind_of.size() - 1) + 1]), "trace: sync");
        for (size_t q = 0; q < t.kind_of.size(); ++q) {
            float ms = 0.0f;
            CUDA_TRY(c, cudaEventElapsedTime(&ms, t.ev[2 * q], t.ev[2 * q + 1]), "trace: elapsed");
            t.ms[t.kind_of[q]] += ms;
            t.timed[t.kind_of[q]] += 1;
            t.timed_bytes[t.kind_of[q]] += t.kind_bytes[q];
        }
        t.kind_of.clear();
        t.kind_bytes.clear();
    }
    long long total = 0;
    for (int k = 0; k < K_COUNT; ++k) total += t.launches[k];
    if (out)
        for (int k = 0; k < K_COUNT && k < cap; ++k) {
            out[k].name = kKindNames[k];
            out[k].launches = t.launches[k];
            out[k].bytes = t.bytes[k];
            out[k].ms = t.ms[k];
            out[k].timed = t.timed[k];
            out[k].timed_bytes = t.timed_bytes[k];
        }
    if (totals) {
        totals->launches = total;
        totals->cell_updates = t.cell_updates;
    }
    if (reset) {
        for (int k = 0; k < K_COUNT; ++k) {
            t.launches[k] = 0;
            t.bytes[k] = 0.0;
            t.ms[k] = 0.0;
            t.timed[k] = 0;
            t.timed_bytes[k] = 0.0;
        }
        t.cell_updates = 0;
    }
    return QUMOND_OK;
}

}  // extern "C"
