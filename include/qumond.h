/*
 * qumond.h -- C ABI of the GB300 QUMOND particle-mesh hot path.
 *
 * Angus et al., "A QUMOND galactic N-body code I: Poisson solver and rotation
 * curve fitting" (arXiv:1201.3185).  One evaluation of the method (Section 2)
 * is, for every nested box b = 0 (outermost) .. nboxes-1:
 *   qumond_deposit       step 1, cloud-in-cell density
 *   qumond_solve_newton  step 2, full multigrid for  lap Phi_N = 4 pi G rho  (Eq. 1)
 *   qumond_source        step 3, the QUMOND source  div[nu(|grad Phi_N|/a0) grad Phi_N]  (Eq. 2)
 *   qumond_solve_mond    step 4, full multigrid for  lap Phi = source  (Eq. 2)
 * and then, over all boxes,
 *   qumond_forces          gravity -grad Phi interpolated to points with CIC weights
 *   qumond_rotation_curve  v_c^2 = R dPhi/dR at z = 0  (Eq. 4)
 *
 * Conventions (every entry point):
 * - Grids are vertex grids of n intervals per side, (n+1)^3 nodes, x fastest:
 *   node (i,j,k) is element i + (n+1)*(j + (n+1)*k).  Box b has side
 *   L_b = L0 / box_ratio^b (box_ratio = 2 in the paper), is centred on
 *   params.center, and has spacing h_b = L_b / n;
 *   node i sits at center - L_b/2 + i*h_b.  Units: pc, Msun, km/s.
 * - Every array argument is a DEVICE pointer to memory the caller owns and
 *   keeps alive until the work queued on `stream` has finished.  Host
 *   pointers are rejected with QUMOND_ERR_INVALID_ARG.  The context owns only
 *   its scratch (multigrid levels, reduction buffers).
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Work is queued asynchronously; argument errors are reported
 *   synchronously before anything is queued.  The solves read residual norms
 *   back to the host (they synchronise `stream`) when a tolerance is set or
 *   when `stats` is non-NULL.
 * - A context is not thread safe: one host thread per context.  Its calls
 *   may be issued on any stream but must not overlap on the GPU (the
 *   multigrid scratch is shared by all calls of a context).  With use_graphs,
 *   each solve is captured once per (box, arrays) into a CUDA graph on the
 *   context's own stream and relaunched on `stream`; the caller's stream must
 *   not itself be capturing.
 * - On error the status is returned and qumond_last_error(ctx) describes it.
 *   QUMOND_ERR_NOT_CONVERGED still leaves the best iterate in the output.
 * - Sets: a context created with params.nsets = S > 1 holds S independent
 *   problems of the same shape (same n, boxes and parameters; different
 *   particles, densities, potentials), e.g. the parameter sets of a fit
 *   sweep.  Every grid argument is then S consecutive grids of (n+1)^3
 *   elements (set s at s*(n+1)^3), per-particle or per-point arrays hold S
 *   consecutive runs of np (or nq) entries, rotation-curve outputs S runs of
 *   nbins, and `stats` points to S structs.  Each step is one launch per
 *   kernel for all sets.  With a tolerance, V-cycles go on until every set
 *   has converged; a set that has converged is skipped by the later V-cycles,
 *   so each set's result is the same as a solve of that set alone.
 *   NOT_CONVERGED and TIMEOUT are returned when any set fails (the message
 *   names the set).
 */
#ifndef QUMOND_H
#define QUMOND_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QUMOND_API __attribute__((visibility("default")))
#else
#define QUMOND_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int qumond_status;
enum {
    QUMOND_OK = 0,
    QUMOND_ERR_INVALID_ARG = 1,
    QUMOND_ERR_CUDA = 2,
    QUMOND_ERR_NOT_CONVERGED = 3,
    QUMOND_ERR_TIMEOUT = 4,
    QUMOND_ERR_OUT_OF_MEMORY = 5
};

/* Arithmetic of the multigrid solves. */
enum {
    /* FP64 everywhere: the plain full-multigrid baseline. */
    QUMOND_PREC_FP64 = 0,
    /* FP32 smoothing, residual restriction and prolongation; FP64 residual,
       defect correction (iterative refinement) and master iterate; FP64 for
       the coarsest grid of the FP64 steps and for all boundary values. */
    QUMOND_PREC_MIXED = 1,
    /* As QUMOND_PREC_MIXED, but the defect correction carries its master
       iterate u and right-hand side in 64-bit fixed point (u * 2^S, S chosen
       per solve so that max|u| * 2^S ~ 2^56): the 7-point residual is then an
       exact integer sum, rounded once to FP32 for the V-cycle.  Resolution
       ~2^-56 max|u| (FP64: 2^-53 |u|); the FP64 pipe, slow on this GPU, is
       used only to convert the FP64 inputs and output once per solve. */
    QUMOND_PREC_MIXED_FIXED = 2
};

/* Boundary values of box 0 (boxes b >= 1 always interpolate theirs from box
   b-1, Section 2). */
enum {
    QUMOND_BC_ZERO = 0,     /* Phi = 0 on the outermost box, as in the paper */
    QUMOND_BC_GIVEN = 1,    /* the caller stores them in the boundary nodes of phi */
    QUMOND_BC_MULTIPOLE = 2 /* from the mass inside box 0: qumond_far_field writes them into
                               the boundary nodes of phiN and phi, and the solves of box 0
                               keep them (as with QUMOND_BC_GIVEN) */
};

typedef struct {
    int n;              /* intervals per side: a power of two, 2 <= n <= 1024 */
    int nboxes;         /* nested boxes, 1 <= nboxes <= 16 */
    double L0;          /* side of box 0, pc */
    double center[3];   /* common centre of all boxes, pc */
    double G;           /* gravitational constant, pc (km/s)^2 / Msun (4.30e-3) */
    double a0;          /* MOND acceleration, (km/s)^2 / pc (3.6, Section 2) */
    int npre, npost;    /* red-black Gauss-Seidel sweeps around the coarse-grid
                           correction, each >= 1 (paper: 2 and 2, Section 2) */
    int ncycle;         /* V-cycles per full-multigrid level, >= 1 (paper: 6) */
    double rel_tol;     /* > 0: after FMG, V-cycles until ||f - L u||_2 <= rel_tol ||f||_2
                           over interior nodes (absolute when f == 0); 0: paper mode */
    int max_vcycles;    /* cap on those V-cycles; reaching it gives NOT_CONVERGED */
    int precision;      /* QUMOND_PREC_* */
    int bc_mode;        /* QUMOND_BC_* */
    int warm_start;     /* 1: skip FMG and refine the interior values the caller
                           left in phi (an initial guess); 0: FMG from scratch */
    int deposit_shift;  /* fixed-point scale of the deposit: 2^shift units per Msun */
    double rc_box_frac; /* rotation curve: radius R uses the finest box with
                           R < rc_box_frac * L_b (0.2 gives Section 3.1's rule) */
    int box_ratio;      /* side ratio of consecutive boxes: 2 (Section 2, each
                           refinement halves the box), 4 or 8 */
    int use_graphs;     /* 1: each solve runs as one cached CUDA graph (FMG and
                           the whole tolerance loop, decided on the device);
                           0: kernels are launched one by one */
    int persistent_vcycle; /* the part of each V-cycle on the small levels
                           below the finest: 0: one launch per step; 1: the
                           levels n <= 64 as one cooperative
                           kernel over all SMs with grid barriers (when the
                           device supports cooperative launches; nsets = 1
                           only); 2: the levels n <= 64 as one thread-block
                           cluster per set (16 CTAs where the device can
                           place them, else 8, 4 or 2) meeting at the
                           cluster's hardware barrier, data in global memory;
                           3 (default): the level n = 32 and those under it
                           as one cluster of small_cluster CTAs per set
                           holding the level in distributed shared memory
                           (FP32 smoothing and finest n >= 64 only;
                           otherwise, or where the cluster cannot be placed,
                           mode 0).  The results
                           are the same bits in every mode.  On GB300 the
                           cooperative form is not faster (a grid barrier
                           costs about what a graph launch does, and it
                           serialises concurrent solves). */
    int nsets;          /* independent problems of this shape held by the
                           context (the parameter sets of a rotation-curve fit,
                           Section 3.5), 1 <= nsets <= 1024 with
                           nsets * (n + 1) <= 65535; default 1.  See "Sets"
                           above.  nsets > 1 excludes persistent_vcycle = 1. */
    int tile_small;     /* block shape of the FP32 half-sweeps and prolongations
                           on the levels with n <= 64: 0 (default) = 8 x 16
                           threads (32 row entries x 16 rows per block),
                           1 = 4 x 32, 2 = 2 x 64.  The same bits for every
                           shape; only the speed differs (picked by timing,
                           e.g. by the fit sweep's autotuner). */
    int small_cluster;  /* CTAs per cluster of persistent_vcycle = 3: 4, 8 or
                           16 (16 is a non-portable cluster size), 0 = 8. */
    int dc_vcycles;     /* tolerance mode: V-cycles on the correction
                           equation per defect-correction step, 1 <= dc_vcycles
                           <= 8 (default 2).  Each step then solves L e = r
                           more closely before u += e and the next residual,
                           so fewer residual checks (each a full pass over u
                           and the right-hand side) are needed.  max_vcycles
                           and the reported vcycles count V-cycles; the
                           residual is checked after every dc_vcycles of
                           them (so the cap is max_vcycles rounded up to a
                           multiple of dc_vcycles). */
} qumond_params;

/* Per-solve report (host struct). */
typedef struct {
    int vcycles;               /* V-cycles made after FMG */
    int converged;             /* 1 if rel_tol was met (always 1 in paper mode) */
    double rel_residual_fmg;   /* ||f - L u|| / ||f|| after FMG (or of the warm start) */
    double rel_residual;       /* the same at return */
} qumond_stats;

typedef struct qumond_ctx qumond_ctx;

/* Paper defaults: n = 256, one box of 120 kpc, G = 4.30e-3, a0 = 3.6,
   npre = npost = 2, ncycle = 6, rel_tol = 0 (paper mode), max_vcycles = 50,
   QUMOND_PREC_MIXED, QUMOND_BC_ZERO, warm_start = 0, deposit_shift = 24,
   rc_box_frac = 0.2, box_ratio = 2, use_graphs = 1, persistent_vcycle = 3,
   nsets = 1, tile_small = 0, small_cluster = 0, dc_vcycles = 2. */
QUMOND_API void qumond_default_params(qumond_params* p);

/* Validates p and allocates the context's device scratch on the current
   device (about 10 (n+1)^3 bytes per set in QUMOND_PREC_MIXED, 20 in FP64,
   34 in QUMOND_PREC_MIXED_FIXED).
   Returns INVALID_ARG, OUT_OF_MEMORY or CUDA_ERROR on failure (*out = NULL). */
QUMOND_API qumond_status qumond_create(const qumond_params* p, qumond_ctx** out);

/* Frees the scratch (synchronises the device first).  NULL is a no-op. */
QUMOND_API void qumond_destroy(qumond_ctx* ctx);

/* Message of the last error on ctx ("" if none).  Valid until the next call. */
QUMOND_API const char* qumond_last_error(const qumond_ctx* ctx);

/* Step 1 (Section 2): cloud-in-cell deposit of np particles into box `box`.
   x, y, z, mass: np doubles each (positions in pc, mass in Msun; the stars
   and the gas carry their own particle mass, Section 3.4).  A particle in
   cell (i,j,k) (0 <= i,j,k < n, half open; others are skipped) adds
   llrint(((mass*2^shift * w_x) * w_y) * w_z) to each of the 8 corner nodes,
   w = 1-d or d, d the offset inside the cell: exact FP64 products, round half
   to even, so the int64 grid does not depend on order.
   rho_fixed: (n+1)^3 int64, overwritten (required).
   rho: (n+1)^3 doubles = rho_fixed * 2^-shift / h^3 in Msun/pc^3, or NULL.
   With several sets, np is the count per set: set s's particles are
   entries s*np .. s*np+np-1 (a set with fewer particles pads with
   particles outside the box, which are skipped). */
QUMOND_API qumond_status qumond_deposit(qumond_ctx* ctx, int box, const double* x, const double* y, const double* z,
                             const double* mass, int64_t np, int64_t* rho_fixed, double* rho, void* stream);

/* Step 2 (Section 2, Eq. 1): Phi_N of box `box` by full multigrid with
   red-black Gauss-Seidel V-cycles (then refinement when rel_tol > 0).
   rho: (n+1)^3 doubles (the deposit of this box), read at interior nodes.
   phiN_parent: Phi_N of box-1 (required when box >= 1, ignored for box 0).
   phiN: (n+1)^3 doubles, overwritten: its boundary nodes are set from the
   parent (or by bc_mode for box 0), its interior by the solve.
   stats: host struct (nsets structs with several sets) or NULL. */
QUMOND_API qumond_status qumond_solve_newton(qumond_ctx* ctx, int box, const double* rho, const double* phiN_parent,
                                  double* phiN, qumond_stats* stats, void* stream);

/* Step 3 (Section 2, Eq. 2): src = div[nu(|grad Phi_N|/a0) grad Phi_N] on
   interior nodes by the face-flux difference
     src(c) = h^-2 * sum over the 6 faces f of c: nu_f * (Phi_N(nbr) - Phi_N(c)),
   nu(y) = 1/2 + 1/2 sqrt(1 + 4/y), y = |g_f|/a0, g_f the gradient at the face
   (normal: the one-sided difference; transverse: mean of the central
   differences at the face's two nodes); a face with g_f = 0 carries no flux.
   Boundary nodes of src are set to 0.  phiN, src: (n+1)^3 doubles. */
QUMOND_API qumond_status qumond_source(qumond_ctx* ctx, int box, const double* phiN, double* src, void* stream);

/* Step 4 (Section 2, Eq. 2): Phi of box `box`; as qumond_solve_newton with
   right-hand side src (no 4 pi G factor) and boundary values from phi_parent. */
QUMOND_API qumond_status qumond_solve_mond(qumond_ctx* ctx, int box, const double* src, const double* phi_parent,
                                double* phi, qumond_stats* stats, void* stream);

/* Forces (Section 2): g = -grad Phi by central differences at the nodes,
   interpolated to nq points with trilinear (CIC) weights.  A point uses the
   finest box whose containing cell has all 8 corners at interior nodes;
   a point in no such cell gets g = 0.
   phi_boxes: HOST array of ctx->nboxes DEVICE pointers (box 0 first).
   qx, qy, qz, gx, gy, gz: nq doubles each. */
QUMOND_API qumond_status qumond_forces(qumond_ctx* ctx, const double* const* phi_boxes, const double* qx, const double* qy,
                            const double* qz, int64_t nq, double* gx, double* gy, double* gz, void* stream);

/* Rotation curve (Section 2, Eq. 4; box rule of Section 3.1): for nbins
   radii R_k = (k + 1/2) rmax / nbins, the mean of dPhi/dR = -(g_x cos t +
   g_y sin t) over nphi azimuths t_m = 2 pi m / nphi at z = center[2], taken
   in index order; v_c = sign(s) sqrt(|s|), s = R_k * mean.  The forces come
   from the finest box with R_k < rc_box_frac * L_b (box 0 if none),
   falling back to coarser boxes where a cell is not interior.
   r_out, vc_out: nbins doubles (device). */
QUMOND_API qumond_status qumond_rotation_curve(qumond_ctx* ctx, const double* const* phi_boxes, int nbins, double rmax,
                                    int nphi, double* r_out, double* vc_out, void* stream);

/* The rotation curve of every set of a context with several sets, each with
   its own outermost radius: set s uses rmax[s] (a fit sweep scales the radii
   of its observed points with the set's distance, Section 3.5) and writes
   its nbins radii and speeds at s * nbins of r_out and vc_out.  rmax: nsets
   doubles (device, > 0).  Otherwise as qumond_rotation_curve. */
QUMOND_API qumond_status qumond_rotation_curve_sets(qumond_ctx* ctx, const double* const* phi_boxes, int nbins,
                                                    const double* rmax, int nphi, double* r_out, double* vc_out,
                                                    void* stream);

/* Algebraic MOND rotation curve (Eq. 3, compared with the QUMOND curve in
   Section 3.3): the tracers and box rule of qumond_rotation_curve, applied
   to the NEWTONIAN potentials, with the field at each tracer taken as
   nu(|g_N|/a0) g_N, nu(y) = 1/2 + 1/2 sqrt(1 + 4/y) (a tracer with g_N = 0
   adds 0); v_c = sign(s) sqrt(|s|), s = R_k * mean of -(g . R^).
   phiN_boxes: HOST array of ctx->nboxes DEVICE pointers; r_out, vc_out:
   nbins doubles (device).  Errors as qumond_rotation_curve. */
QUMOND_API qumond_status qumond_rotation_curve_algebraic(qumond_ctx* ctx, const double* const* phiN_boxes, int nbins,
                                                         double rmax, int nphi, double* r_out, double* vc_out,
                                                         void* stream);

/* Vertical velocity dispersion of an isothermal stellar layer (Section 5.6):
   sigma_z^2 = -dPhi/dz * rho_s / (d rho_s/dz).  For the sech^2(z/h) layers of
   the realisations, rho_s / (d rho_s/dz) = -h / (2 tanh(z/h)); with tracers
   at height z_eval above the plane (radii, azimuths and box rule of
   qumond_rotation_curve), sigma_out[k] = sign(s) sqrt(|s|),
   s = (mean of dPhi/dz) * h / (2 tanh(z_eval/h)).  z_eval, h > 0 (pc).
   r_out, sigma_out: nbins doubles (device). */
QUMOND_API qumond_status qumond_sigma_z(qumond_ctx* ctx, const double* const* phi_boxes, int nbins, double rmax,
                                        int nphi, double z_eval, double h, double* r_out, double* sigma_out,
                                        void* stream);

/* Quality of a rotation-curve fit (Section 3.5): for each of nsets curves,
     chi2[s] = (1/nbins) * sum_i ((vc[s*nbins + i] - v_obs[i]) / sigma[i])^2
   (the reduced chi^2 the paper minimises over distance, M/L and scale
   heights).  vc: nsets x nbins doubles, row-major; v_obs, sigma: nbins
   doubles; chi2: nsets doubles; all device pointers, owned by the caller.
   sigma must be non-zero (a zero gives inf or nan).  nsets = 0 does nothing.
   Errors: QUMOND_ERR_INVALID_ARG for nbins < 1, nsets < 0 or a host pointer. */
QUMOND_API qumond_status qumond_chi2(qumond_ctx* ctx, const double* vc, const double* v_obs, const double* sigma,
                                     int nbins, int nsets, double* chi2, void* stream);

/* Boundary values of box 0 from the mass inside it (QUMOND_BC_MULTIPOLE).
   Section 2 sets Phi = 0 on a box 2^10 times the galaxy and refines inwards;
   with fewer boxes the outer boundary lies near the mass, and this computes
   the values the far field of that mass takes there:
   - phiN: the exterior multipole expansion, to degree 8, of the node masses
     m_k = rho_k h_0^3 (every node of box 0) about their centre of mass c,
       Phi_N(x) = -G sum_k m_k sum_{l<=8} |x_k - c|^l / |x - c|^(l+1) P_l(cos g_k),
     g_k the angle between x_k - c and x - c (evaluated through the moments
     of the solid harmonics, FP64, fixed-order sums);
   - phi: the QUMOND potential of the total mass M as a point at c,
       F(r) = -A/(2r) + 1/2 [-sqrt(A^2 + C r^2)/r + sqrt(C) asinh(sqrt(C) r/A)],
     A = G M, C = 4 a0 A, r = |x - c|: F'(r) = nu(G M/(a0 r^2)) G M/r^2, the
     field of a point mass under Eq. 2.
   rho: box 0's density ((n+1)^3 doubles, device, e.g. from qumond_deposit);
   phiN, phi: (n+1)^3 doubles (device): only their boundary nodes are
   written.  With M = 0 both are set to 0.  Requires bc_mode =
   QUMOND_BC_MULTIPOLE (else QUMOND_ERR_INVALID_ARG); enqueue it before the
   solves of box 0.  With several sets, each set's own mass. */
QUMOND_API qumond_status qumond_far_field(qumond_ctx* ctx, const double* rho, double* phiN, double* phi,
                                          void* stream);

/* Bound on the polls of one grid barrier of the cooperative small-level
   V-cycle kernel (persistent_vcycle = 1) before the barrier gives up; the
   solve then stops its V-cycles and returns QUMOND_ERR_TIMEOUT (the output
   holds no usable solution).  Default 2^26 polls (far beyond any barrier of
   a healthy solve).  Not part of the method: it exists so that the timeout
   path can be exercised (a limit of 1 makes the barriers give up).  Drops
   the context's cached solve graphs (synchronises the device) when the
   limit changes.  polls >= 1, else QUMOND_ERR_INVALID_ARG. */
QUMOND_API qumond_status qumond_set_barrier_poll_limit(qumond_ctx* ctx, int64_t polls);

/* --- tracing (not part of the method: instrumentation of the kernels) ------ */

/* Per-kernel-class counters of a context since it was created or last reset. */
typedef struct {
    const char* name;     /* kernel class, e.g. "rb_half_finest" (static storage) */
    int64_t launches;     /* kernels of this class launched */
    double bytes;         /* algorithmic HBM bytes of those launches (the minimum
                             each kernel must read and write) */
    double ms;            /* summed CUDA-event time of the launches that were
                             bracketed while timing was on (0 otherwise) */
    int64_t timed;        /* how many launches were bracketed */
    double timed_bytes;   /* algorithmic bytes of the bracketed launches */
} qumond_kernel_stat;

typedef struct {
    int64_t launches;      /* all kernels launched by this context */
    int64_t cell_updates;  /* red-black node updates, all levels */
} qumond_counters;

/* Number of kernel classes (size of the array qumond_trace_read fills). */
QUMOND_API int qumond_trace_classes(void);

/* Start (on != 0) or stop timing kernels with CUDA events on their stream.
   only_class = -1: every launch is bracketed and the solves launch their
   kernels one by one (graphs off); at most 32768 launches per start are
   timed, later ones are only counted.
   only_class = k (an index into qumond_trace_read's array): only launches of
   class k are timed, and the solves keep running as CUDA graphs: their
   graphs are captured with one pair of event-record nodes around each run of
   consecutive class-k launches in the preamble (boundary values, FMG, first
   residual check; a conditional loop body cannot hold event nodes), and each
   solve with residual checks adds those intervals and the launches they
   cover after its final synchronisation.
   Starting discards earlier timings.  Counters are always kept. */
QUMOND_API qumond_status qumond_trace_timing(qumond_ctx* ctx, int on, int only_class);

/* Copies the per-class statistics into out[0 .. min(cap, classes)-1] and the
   totals into *totals (either may be NULL).  Synchronises the device when
   timed launches are pending.  reset != 0 then zeroes every counter. */
QUMOND_API qumond_status qumond_trace_read(qumond_ctx* ctx, qumond_kernel_stat* out, int cap,
                                           qumond_counters* totals, int reset);

/* --- a solve that allocates nothing ------------------------------------------
   The paper has no counterpart: this is a service to callers that cannot
   allocate device memory when they need a solve (a caller whose memory pool
   or arena already owns the whole device budget, or a thread that must not
   enter the allocator).  qumond_create allocates the multigrid scratch; this
   entry point instead keeps it in one fixed device array inside the library,
   QUMOND_NOALLOC_SCRATCH_BYTES long, which exists on every device that loads
   the library until the process exits.  That bounds the grid: n must be a
   power of two <= QUMOND_NOALLOC_MAX_N; larger n is rejected with
   QUMOND_ERR_INVALID_ARG and a message.  Only QUMOND_PREC_MIXED is offered.

   Arguments and result: as qumond_solve_mond (the parameters are passed
   directly since there is no context; they are checked as qumond_create
   checks them).  err (may be NULL): receives a message of at most err_len
   bytes on failure.

   The call makes no cudaMalloc, cudaFree or other allocating call.  The first
   call on each device does a one-time set-up with that device current: it
   looks up the array's device address and caches it, and sets the kernel
   attributes the solve needs (neither allocates).  The cached address
   assumes the device is not reset: calling cudaDeviceReset in the same
   process and then this entry point again is not supported.  When a
   tolerance is set (rel_tol > 0 and max_vcycles > 0) or stats is non-NULL,
   the call copies residual norms to a host buffer and synchronises `stream`
   after each residual check.
   All calls on a device share the array, which keeps the previous call's
   contents (each call clears it before use): calls whose GPU work overlaps,
   on different streams or host threads, race and give wrong results. */
#define QUMOND_NOALLOC_MAX_N 64
#define QUMOND_NOALLOC_SCRATCH_BYTES 2903552
QUMOND_API qumond_status qumond_solve_mond_noalloc(const qumond_params* p, int box, const double* src,
                                                   const double* phi_parent, double* phi, qumond_stats* stats,
                                                   void* stream, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* QUMOND_H */
