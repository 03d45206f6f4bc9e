// Internal declarations shared by the CUDA translation units of libqumond.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qumond {

// Colour-split storage of one multigrid level (n intervals, (n+1)^3 nodes).
// Node (i,j,k) has colour c = (i+j+k) & 1 (0 = red, updated first).  Each
// colour is its own array of rows: row (j,k) of colour c holds that colour's
// nodes of the row, node i at position i >> 1.  Rows are M entries long
// (M >= n/2 + 1, a multiple of 4 so rows start on 16-byte boundaries) and the
// two colour arrays sit cs elements apart.
//
// With this layout a red-black half-sweep streams only the colour it writes
// and the colour it reads: the six neighbours of node (2m+p, j, k) of colour
// c are, in colour 1-c, entries m-1+p and m+p of the same row (x), entry m of
// rows j-1 and j+1 (y) and entry m of planes k-1 and k+1 (z), where
// p = (c + j + k) & 1 is the parity of i in that row.
struct LevelView {
    int n;
    int M;
    long long cs;
};

__host__ __device__ inline long long row_off(const LevelView& v, int c, int j, int k)
{
    return (long long)c * v.cs + ((long long)k * (v.n + 1) + j) * (long long)v.M;
}

__host__ __device__ inline long long node_off(const LevelView& v, int i, int j, int k)
{
    return row_off(v, (i + j + k) & 1, j, k) + (i >> 1);
}

inline LevelView make_view(int n)
{
    LevelView v;
    v.n = n;
    v.M = ((n / 2 + 1) + 3) & ~3;
    long long plane = (long long)v.M * (n + 1) * (n + 1);
    v.cs = (plane + 63) & ~63LL;
    return v;
}

// Largest level handled entirely by the single-CTA coarse-grid kernel.
constexpr int kCoarseN = 16;

// Device-side state of a defect-correction loop.
struct SolveState {
    double denom;  // ||coef*rhs||_2 (1 when zero)
    double rel0;   // relative residual after FMG / of the warm start
    double rel;    // latest relative residual
    int it;        // V-cycles made after FMG
    int cont;      // 1: another V-cycle is needed
    int converged; // 1: rel <= tol (or no tolerance) and finite
    int scale_exp; // fixed-point outer loop: U = u * 2^scale_exp
    int fault;     // 1: a kernel gave up waiting (bounded spin) since the last check
    int nonfinite; // fixed-point mode: the start (FMG result, boundary or warm-start values, right-hand
                   // side) holds a NaN or an infinity, so no integer iterate represents it
};
// Independent problems of one shape held by one context ("sets", e.g. the
// parameter sets of a rotation-curve fit sweep).  Every array of such a
// context holds the sets one after another -- set s of a level array at
// s * 2 cs elements, of a natural (n+1)^3 grid at s (n+1)^3, of a fixed-point
// array at s * fixed_elems(n), of the partial norms at s * pstride -- and one
// launch covers all sets: the kernels take the set index from a grid
// dimension.  act, when non-null, makes the kernels of a defect-correction
// V-cycle skip the sets whose correction has stopped (act[s].cont == 0), so
// each set gets exactly the iterations a solve of it alone would get.
struct Sets {
    int n = 1;
    const SolveState* act = nullptr;
    long long pstride = 0;  // doubles between two sets' partial norms
    int tile_small = 0;     // block shape of the row-vector kernels on levels n <= 64 (qumond_params.tile_small)
};
__host__ __device__ inline long long nat_elems(int n) { return (long long)(n + 1) * (n + 1) * (n + 1); }

// --- multigrid kernels (mg_kernels.cu), T = float or double ---------------
template <typename T> void launch_rb_half(T* e, const T* f, const LevelView& v, int colour, bool zero_guess,
                                          double h, cudaStream_t s, const Sets& sets = Sets());
// Both half-sweeps of the first sweep from zero in one launch (FP32, n >= 8):
// the same bits as launch_rb_half(colour 0, zero) then launch_rb_half(colour 1).
void launch_rb_first(float* e, const float* f, const LevelView& v, double h, cudaStream_t s, const Sets& sets);
template <typename T> void launch_restrict_resid_red(const T* ef, const T* ff, const LevelView& vf, T* fc,
                                                     const LevelView& vc, double hf, cudaStream_t s,
                                                     const Sets& sets = Sets());
template <typename T> void launch_restrict_full(const T* ff, const LevelView& vf, T* fc, const LevelView& vc,
                                                cudaStream_t s, const Sets& sets = Sets());
template <typename T> void launch_prolong_black(const T* ec, const LevelView& vc, T* ef, const LevelView& vf,
                                                bool add, cudaStream_t s, const Sets& sets = Sets());
template <typename T> void launch_set_boundary(T* e, const LevelView& v, const double* u64, int nfine,
                                               cudaStream_t s, const Sets& sets = Sets());
// the V-cycle on levels 0 .. nlev-1 (level 0 = the coarse-grid level) as one cooperative kernel
template <typename T> cudaError_t launch_vsub(T* const* e, T* const* f, const LevelView* v, const double* h, int nlev,
                                              int zero_top, int npre, int npost, unsigned* bar, int* fault,
                                              long long polls, int grid, cudaStream_t s);
int vsub_grid(int sms);
// the same V-cycle as one thread-block cluster of csize CTAs per set (no grid-wide barrier)
template <typename T> cudaError_t launch_vcluster(T* const* e, T* const* f, const LevelView* v, const double* h,
                                                  int nlev, int zero_top, int npre, int npost, int csize,
                                                  cudaStream_t s, const Sets& sets = Sets());
// largest cluster size (16, 8, 4 or 2) the device can schedule for it, 0 if none
int vcluster_size(bool fp64);
// The V-cycle from the 32-interval level down in the shared memory of one
// thread-block cluster of csize (4, 8 or 16) CTAs per set (FP32 levels; v is
// the 32-interval level, h its spacing, hc that of the 16-interval level).
cudaError_t launch_vslab(float* e, const float* f, const LevelView& v, double h, double hc, int zero_top, int npre,
                         int npost, int csize, cudaStream_t s, const Sets& sets);
int vslab_size(int want);
template <typename T> cudaError_t launch_coarse(int fmg, T* e, const T* f, const LevelView& v, double h,
                                                const double* u64, int nfine, int ncycle, int npre, int npost,
                                                cudaStream_t s, const Sets& sets = Sets());
// FP64 outer steps on the caller's natural-layout arrays.
template <typename T> void launch_convert_rhs(const double* rhs, double coef, int n, T* f, const LevelView& v,
                                              cudaStream_t s, const Sets& sets = Sets());
template <typename T> void launch_assign_outer(double* u, int n, const T* e, const LevelView& v, bool add,
                                               cudaStream_t s, const Sets& sets = Sets());
template <typename T> int launch_residual_outer(const double* u, const double* rhs, double coef, int n, double h,
                                                T* r, const LevelView& v, double* partials, cudaStream_t s);
void launch_reduce_norms(const double* partials, int nblocks, double* out, cudaStream_t s);
int residual_outer_blocks(int n);

// Residual with a fixed number of blocks (residual_rows_blocks(n) partial sums).
template <typename T> int launch_residual_rows(const double* u, const double* rhs, double coef, int n, double h, T* r,
                                               const LevelView& v, double* partials, cudaStream_t s,
                                               const Sets& sets = Sets());
int residual_rows_blocks(int n);

// Reduces the partial norms and decides whether to continue; with a
// non-null handle it also sets the graph's WHILE condition.
// With several sets, one block per set decides for its set (a set whose
// correction has stopped keeps its state) and one more kernel takes over the
// fault flag and sets the WHILE condition when any set goes on.
void launch_decide(const double* partials, int nblocks, SolveState* st, double tol, int max_it, bool first,
                   bool refine, const cudaGraphConditionalHandle* handle, int* fault, cudaStream_t s,
                   const Sets& sets = Sets());

// --- TMA-staged half-sweep for FP32 levels with n >= 64 (rb_tma.cu) ----------
struct RbMaps {
    CUtensorMap map[2];   // colour c of the iterate as a 3-D tensor (m, j, k), tile + halo boxes
    CUtensorMap fmap[2];  // colour c of the right-hand side, tile boxes
    CUtensorMap rmap_black, rmap_red, rmap_f;  // the restriction's boxes (black with halo, red, red f)
    CUtensorMap pmap_fine, pmap_c[2];  // the prolongation's boxes: this level's black tile, the coarser level's colours
    bool ok = false;
    bool pok = false;  // the prolongation maps are set
};
// 4-D maps (m, j, k, set) over the nsets sets of a level
bool make_rb_maps(float* e, float* f, const LevelView& v, RbMaps* out, int nsets = 1);
void launch_rb_half_tma(float* e, const float* f, const LevelView& v, int colour, const RbMaps& maps, double h,
                        int* fault, cudaStream_t s, const Sets& sets = Sets());
// Full weighting of the red residuals of the fine level whose maps are given (right after a black half-sweep)
// into the coarse right-hand side fc, the fine planes staged by the TMA unit.
void launch_restrict_tma(float* fc, const LevelView& vf, const LevelView& vc, const RbMaps& maps, double hf,
                         int* fault, cudaStream_t s, const Sets& sets = Sets());
// The coarse-grid correction of this level's black nodes from the next coarser level (ec, vc), planes staged by
// the TMA unit; make_prolong_maps adds the boxes to this level's maps (after make_rb_maps).
bool make_prolong_maps(float* ec, const LevelView& vc, float* ef, const LevelView& vf, RbMaps* out, int nsets = 1);
void launch_prolong_tma(float* ef, const LevelView& vf, const RbMaps& maps, int* fault, cudaStream_t s,
                        const Sets& sets = Sets());
// Sets kernel attributes (shared memory of the coarse-grid kernel); call
// before any stream capture.
cudaError_t prepare_kernels();

// --- fixed-point defect correction (fixed_outer.cu) ---------------------------
void launch_fixed_scale(const float* e, const LevelView& v, const double* u64, int n, bool from_u64, unsigned* maxbits,
                        SolveState* st, cudaStream_t s, const Sets& sets = Sets());
void launch_fixed_init(const float* e, const LevelView& v, const double* u64, const double* rhs, double coef, double h,
                       int n, bool from_u64, SolveState* st, int64_t* U, int64_t* U2, int64_t* F, cudaStream_t s,
                       const Sets& sets = Sets());
int fixed_residual_blocks(int n);
int launch_fixed_residual(const int64_t* U, const int64_t* F, int n, double h, const SolveState* st, bool want_f,
                          float* r, const LevelView& v, double* partials, cudaStream_t s, const Sets& sets = Sets());
void launch_fixed_output(const int64_t* U, const int64_t* U2, double* u, int n, const SolveState* st, cudaStream_t s,
                         const Sets& sets = Sets());
// U' = U + round(e 2^S) into the other buffer and the residual of U' (one pass); returns the blocks written
// elements of a fixed-point array (rows padded to n + 2 entries)
size_t fixed_elems(int n);
// TMA descriptors of the fixed-point arrays (both buffers of U, F) and of the finest level's e (two colours)
struct FixedMaps {
    CUtensorMap u[2];
    CUtensorMap f;
    CUtensorMap e[2];
    bool ok;
};
// 4-D maps (i, j, k, set) over the nsets sets
bool make_fixed_maps(int64_t* U, int64_t* U2, int64_t* F, float* e, const LevelView& v, FixedMaps* out,
                     int nsets = 1);
// the fused update + residual with TMA-staged planes (n >= 128); returns the blocks written
int launch_fixed_update_residual_tma(int64_t* U, int64_t* U2, const FixedMaps& maps, int n, double h,
                                     const SolveState* st, float* r, const LevelView& v, double* partials, int* fault,
                                     cudaStream_t s, const Sets& sets = Sets());
int launch_fixed_update_residual(int64_t* U, int64_t* U2, const int64_t* F, const float* e, int n, double h,
                                 const SolveState* st, float* r, const LevelView& v, double* partials, cudaStream_t s,
                                 const Sets& sets = Sets());

// --- grid kernels (grid_kernels.cu) ------------------------------------------
// np particles per set (set s's at s * np in x, y, z, m)
void launch_cic_deposit(const double* x, const double* y, const double* z, const double* m, long long np, int n,
                        double xlo, double ylo, double zlo, double inv_h, double two_shift, int64_t* q,
                        cudaStream_t s, int nsets = 1);
void launch_fixed_to_rho(const int64_t* q, double* rho, long long count, double scale, cudaStream_t s);
void launch_boundary_zero(double* u, int n, cudaStream_t s, int nsets = 1);
void launch_boundary_from_parent(const double* parent, double* u, int n, int ratio, cudaStream_t s, int nsets = 1);
void launch_source(const double* phi, double* src, int n, double h, double a0, cudaStream_t s, int nsets = 1);

struct BoxGeom {
    const double* phi;
    double xlo, ylo, zlo;
    double inv_h;
    double h;
    double L;
};
constexpr int kMaxBoxes = 16;
struct BoxSet {
    BoxGeom b[kMaxBoxes];
    int nboxes;
    int n;
};
// nq points per set; with several sets, set s's points, forces, radii and
// curves follow set s-1's, and its potentials sit at s (n+1)^3 in every box
void launch_forces(const BoxSet& boxes, const double* qx, const double* qy, const double* qz, long long nq,
                   double* gx, double* gy, double* gz, cudaStream_t s, int nsets = 1);
// rmax_sets: nsets device values (each set's outermost radius), or NULL for rmax
void launch_rotation_curve(const BoxSet& boxes, double cx, double cy, double cz, int nbins, double rmax,
                           const double* rmax_sets, int nphi, double frac, double* r_out, double* vc_out,
                           cudaStream_t s, int nsets = 1);
void launch_chi2(const double* vc, const double* v_obs, const double* sigma, int nbins, int nsets, double* chi2,
                 cudaStream_t s);

// --- far-field boundary values of box 0 (farfield.cu) ------------------------
// scratch: far_field_scratch_doubles(nsets) doubles of device memory
size_t far_field_scratch_doubles(int nsets);
void launch_far_field(const double* rho, int n, double L, double cx, double cy, double cz, double G, double a0,
                      double* phiN, double* phi, double* scratch, int nsets, cudaStream_t s);
void launch_profile(const BoxSet& boxes, double cx, double cy, double cz, int nbins, double rmax, int nphi, double frac,
                    int mode, double a0, double z_eval, double h, double* r_out, double* out, cudaStream_t s,
                    int nsets = 1);

}  // namespace qumond
