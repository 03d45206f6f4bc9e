/*
 * QUMOND particle-mesh oracle: plain, slow, FP64 CPU reference.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke() check in
 * __graft_entry__.py and the cpu_baseline / reference legs of bench.py may
 * load this library.  The CUDA path never calls it and shares no code with it.
 *
 * Paper: Angus et al., "A QUMOND galactic N-body code I: Poisson solver and
 * rotation curve fitting" (arXiv:1201.3185).  Section numbers and equations
 * below refer to that paper.
 *
 * Grids are vertex grids with n intervals per side (n a power of two), i.e.
 * (n+1)^3 nodes, x fastest: index i + (n+1)*(j + (n+1)*k).  A box of side L
 * centred on c has spacing h = L/n and node i at c - L/2 + i*h.
 * Units: pc, Msun, km/s.
 *
 * Every loop below is a direct transcription of a definition: no blocking,
 * fusion or reordering.  Loops over independent nodes may run under OpenMP;
 * that never changes a result, and every reduction is summed in a fixed
 * serial order so results do not depend on the thread count.
 *
 * Compiled with -ffp-contract=off so that no multiply-add is fused: the
 * fixed-point CIC deposit must be reproducible bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(n, i, j, k) ((size_t)(i) + (size_t)((n) + 1) * ((size_t)(j) + (size_t)((n) + 1) * (size_t)(k)))

static size_t nodes(int n) { return (size_t)(n + 1) * (size_t)(n + 1) * (size_t)(n + 1); }

/* ------------------------------------------------------------------------ */
/* Step 1 (Section 2): cloud-in-cell assignment of particle mass to the grid.
 * The stars and the gas each carry their own particle mass (Section 2, and
 * Section 3.4: half of the particles per component, weighted by the
 * component's total mass), so the mass is passed per particle.
 *
 * Reading of the paper (cloud in cell on a vertex grid): a particle in cell
 * (i,j,k) -- the cube whose lowest node is (i,j,k) -- gives each of the 8
 * corner nodes the fraction w_x*w_y*w_z of its mass, with w = 1-d for the lower
 * node and d for the upper one, d the fractional offset inside the cell.  A
 * particle is kept iff 0 <= i,j,k < n (a half-open box).
 *
 * The deposit is accumulated in 64-bit fixed point: each corner contribution
 * is q = llrint(((m*2^shift * w_x) * w_y) * w_z), rounded half to even, so
 * the integer grid does not depend on summation order.  inv_h = n / L.
 * Returns the number of particles kept. */
int64_t ora_cic_deposit(int n, double L, double cx, double cy, double cz, int shift,
                        const double* x, const double* y, const double* z, const double* m,
                        int64_t np, int64_t* q)
{
    const double inv_h = (double)n / L;
    const double xlo = cx - 0.5 * L, ylo = cy - 0.5 * L, zlo = cz - 0.5 * L;
    int64_t kept = 0;
    for (int64_t p = 0; p < np; ++p) {
        double tx = (x[p] - xlo) * inv_h;
        double ty = (y[p] - ylo) * inv_h;
        double tz = (z[p] - zlo) * inv_h;
        if (!(tx >= 0.0 && tx < (double)n && ty >= 0.0 && ty < (double)n && tz >= 0.0 && tz < (double)n))
            continue;
        double fx = floor(tx), fy = floor(ty), fz = floor(tz);
        int i = (int)fx, j = (int)fy, k = (int)fz;
        if (i >= n || j >= n || k >= n) continue; /* tx just below n can round up */
        double dx = tx - fx, dy = ty - fy, dz = tz - fz;
        double wx[2] = {1.0 - dx, dx};
        double wy[2] = {1.0 - dy, dy};
        double wz[2] = {1.0 - dz, dz};
        double ms = ldexp(m[p], shift);
        for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    double w = ((ms * wx[a]) * wy[b]) * wz[c];
                    q[IDX(n, i + a, j + b, k + c)] += (int64_t)llrint(w);
                }
        ++kept;
    }
    return kept;
}

/* Density from the fixed-point grid: rho = q * 2^-shift / h^3. */
void ora_rho_from_fixed(int n, double L, int shift, const int64_t* q, double* rho)
{
    const double inv_h = (double)n / L;
    const double scale = ldexp(1.0, -shift) * (inv_h * inv_h * inv_h);
    size_t nn = nodes(n);
    for (size_t t = 0; t < nn; ++t) rho[t] = (double)q[t] * scale;
}

/* ------------------------------------------------------------------------ */
/* Steps 2 and 4 (Section 2): full multigrid with red-black Gauss-Seidel,
 * after the textbook FMG the paper cites, extended to 3D.
 *
 * Discrete problem: for every interior node,
 *   (u[i+1]+u[i-1]+u[j+1]+u[j-1]+u[k+1]+u[k-1] - 6 u) / h^2 = f,
 * with Dirichlet values held in the boundary nodes of u.
 */

/* One red-black Gauss-Seidel sweep: every red node (i+j+k even), then every
 * black node, each set to the value that zeroes its own residual. */
void ora_relax_rbgs(int n, double h, double* u, const double* f)
{
    const double h2 = h * h;
    for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for schedule(static)
        for (int k = 1; k < n; ++k)
            for (int j = 1; j < n; ++j)
                for (int i = 1; i < n; ++i) {
                    if (((i + j + k) & 1) != colour) continue;
                    double s = u[IDX(n, i + 1, j, k)] + u[IDX(n, i - 1, j, k)]
                             + u[IDX(n, i, j + 1, k)] + u[IDX(n, i, j - 1, k)]
                             + u[IDX(n, i, j, k + 1)] + u[IDX(n, i, j, k - 1)];
                    u[IDX(n, i, j, k)] = (s - h2 * f[IDX(n, i, j, k)]) / 6.0;
                }
    }
}

/* Residual r = f - L u on interior nodes; r = 0 on the boundary. */
void ora_residual(int n, double h, const double* u, const double* f, double* r)
{
    const double ih2 = 1.0 / (h * h);
    memset(r, 0, nodes(n) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 1; k < n; ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                double lap = (u[IDX(n, i + 1, j, k)] + u[IDX(n, i - 1, j, k)]
                            + u[IDX(n, i, j + 1, k)] + u[IDX(n, i, j - 1, k)]
                            + u[IDX(n, i, j, k + 1)] + u[IDX(n, i, j, k - 1)]
                            - 6.0 * u[IDX(n, i, j, k)]) * ih2;
                r[IDX(n, i, j, k)] = f[IDX(n, i, j, k)] - lap;
            }
}

/* Sum of squares over interior nodes, in a fixed serial order. */
double ora_interior_sumsq(int n, const double* a)
{
    double s = 0.0;
    for (int k = 1; k < n; ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                double v = a[IDX(n, i, j, k)];
                s += v * v;
            }
    return s;
}

/* Restriction to the grid with nf/2 intervals.  The paper says "bilinear";
 * in 3D we take full weighting, the transpose of trilinear prolongation
 * (scaled): weight (1/2 or 1/4 per axis for offset 0 or +-1).  Coarse
 * boundary nodes are set to 0. */
void ora_restrict_fw(int nf, const double* fine, double* coarse)
{
    const int nc = nf / 2;
    memset(coarse, 0, nodes(nc) * sizeof(double));
    static const double w[3] = {0.25, 0.5, 0.25};
#pragma omp parallel for schedule(static)
    for (int K = 1; K < nc; ++K)
        for (int J = 1; J < nc; ++J)
            for (int I = 1; I < nc; ++I) {
                double s = 0.0;
                for (int c = -1; c <= 1; ++c)
                    for (int b = -1; b <= 1; ++b)
                        for (int a = -1; a <= 1; ++a)
                            s += w[a + 1] * w[b + 1] * w[c + 1]
                               * fine[IDX(nf, 2 * I + a, 2 * J + b, 2 * K + c)];
                coarse[IDX(nc, I, J, K)] = s;
            }
}

/* Trilinear ("bilinear" in the paper) prolongation from the grid with nc
 * intervals to the one with 2*nc, on the interior fine nodes only:
 * add == 0: fine = P coarse; add != 0: fine += P coarse. */
void ora_prolong(int nc, const double* coarse, double* fine, int add)
{
    const int nf = 2 * nc;
#pragma omp parallel for schedule(static)
    for (int k = 1; k < nf; ++k)
        for (int j = 1; j < nf; ++j)
            for (int i = 1; i < nf; ++i) {
                int i0 = i / 2, j0 = j / 2, k0 = k / 2;
                int i1 = (i + 1) / 2, j1 = (j + 1) / 2, k1 = (k + 1) / 2;
                double v = 0.125 * (coarse[IDX(nc, i0, j0, k0)] + coarse[IDX(nc, i1, j0, k0)]
                                  + coarse[IDX(nc, i0, j1, k0)] + coarse[IDX(nc, i1, j1, k0)]
                                  + coarse[IDX(nc, i0, j0, k1)] + coarse[IDX(nc, i1, j0, k1)]
                                  + coarse[IDX(nc, i0, j1, k1)] + coarse[IDX(nc, i1, j1, k1)]);
                if (add) fine[IDX(nf, i, j, k)] += v;
                else fine[IDX(nf, i, j, k)] = v;
            }
}

/* Exact solve on the coarsest grid, 3x3x3 (Section 2): one unknown, the
 * centre node, u = (sum of its 6 neighbours - h^2 f) / 6.  With zero
 * boundary values this is proportional to the centre density. */
void ora_coarsest(double h, double* u, const double* f)
{
    double s = u[IDX(2, 2, 1, 1)] + u[IDX(2, 0, 1, 1)] + u[IDX(2, 1, 2, 1)]
             + u[IDX(2, 1, 0, 1)] + u[IDX(2, 1, 1, 2)] + u[IDX(2, 1, 1, 0)];
    u[IDX(2, 1, 1, 1)] = (s - h * h * f[IDX(2, 1, 1, 1)]) / 6.0;
}

/* One V-cycle (Section 2: finest to coarsest and back, npre and npost
 * red-black sweeps before and after the coarse-grid correction).  u holds
 * its own boundary values; the coarse-grid corrections have zero boundary
 * values and start from zero. */
void ora_vcycle(int n, double h, double* u, const double* f, int npre, int npost)
{
    if (n == 2) { ora_coarsest(h, u, f); return; }
    for (int s = 0; s < npre; ++s) ora_relax_rbgs(n, h, u, f);
    double* r = (double*)malloc(nodes(n) * sizeof(double));
    ora_residual(n, h, u, f, r);
    int nc = n / 2;
    double* fc = (double*)malloc(nodes(nc) * sizeof(double));
    double* ec = (double*)calloc(nodes(nc), sizeof(double));
    ora_restrict_fw(n, r, fc);
    free(r);
    ora_vcycle(nc, 2.0 * h, ec, fc, npre, npost);
    ora_prolong(nc, ec, u, 1);
    free(fc);
    free(ec);
    for (int s = 0; s < npost; ++s) ora_relax_rbgs(n, h, u, f);
}

/* Copy the boundary nodes of the finest grid (n intervals) onto the boundary
 * of a coarser grid with nc intervals by injection (coarse node I sits on
 * fine node I*n/nc). */
static void inject_boundary(int n, const double* fine, int nc, double* coarse)
{
    int s = n / nc;
    for (int K = 0; K <= nc; ++K)
        for (int J = 0; J <= nc; ++J)
            for (int I = 0; I <= nc; ++I) {
                if (I != 0 && I != nc && J != 0 && J != nc && K != 0 && K != nc) continue;
                coarse[IDX(nc, I, J, K)] = fine[IDX(n, I * s, J * s, K * s)];
            }
}

/* Full multigrid (Section 2): the right-hand side is restricted down to the
 * 3x3x3 grid, solved there exactly, interpolated to each finer grid in turn,
 * and at every grid ncycle V-cycles are made.  Boundary values on the coarser
 * FMG grids are the finest boundary values at the same positions.  On return
 * u (finest) holds the FMG result; its boundary values are untouched. */
void ora_fmg(int n, double h, double* u, const double* f, int ncycle, int npre, int npost)
{
    int nlev = 0;
    for (int m = n; m >= 2; m /= 2) ++nlev; /* levels with n = 2, 4, ..., n */
    double** fl = (double**)malloc(sizeof(double*) * nlev);
    double** ul = (double**)malloc(sizeof(double*) * nlev);
    /* level index L = nlev-1 is the finest */
    fl[nlev - 1] = (double*)f;
    ul[nlev - 1] = u;
    for (int l = nlev - 2; l >= 0; --l) {
        int nl = 2 << l;
        fl[l] = (double*)malloc(nodes(nl) * sizeof(double));
        ul[l] = (double*)calloc(nodes(nl), sizeof(double));
        ora_restrict_fw(2 * nl, fl[l + 1], fl[l]);
    }
    /* coarsest exact solve with the injected boundary values */
    if (nlev > 1) inject_boundary(n, u, 2, ul[0]);
    ora_coarsest(h * (double)(n / 2), ul[0], fl[0]);
    for (int l = 1; l < nlev; ++l) {
        int nl = 2 << l;
        double hl = h * (double)(n / nl);
        if (l < nlev - 1) inject_boundary(n, u, nl, ul[l]);
        ora_prolong(nl / 2, ul[l - 1], ul[l], 0);
        for (int c = 0; c < ncycle; ++c) ora_vcycle(nl, hl, ul[l], fl[l], npre, npost);
    }
    for (int l = 0; l < nlev - 1; ++l) { free(fl[l]); free(ul[l]); }
    free(fl);
    free(ul);
}

/* A complete solve.  u: boundary nodes hold the Dirichlet values; the
 * interior is the initial guess when fmg == 0, else it is overwritten by FMG.
 * After FMG (paper mode, Section 3.2: six V-cycles per level) further
 * V-cycles are made until ||f - L u||_2 <= tol ||f||_2 over interior nodes
 * (tol alone when f == 0), at most max_vcycles of them (tol <= 0 or max_vcycles == 0: none).
 * hist[0..] receives the relative residual after FMG and after each further
 * V-cycle.  Returns the number of further V-cycles made, or -1 if the
 * tolerance was not met. */
int ora_solve(int n, double h, double* u, const double* f, int fmg, int ncycle, int npre, int npost,
              double tol, int max_vcycles, double* hist, int hist_cap)
{
    if (fmg) ora_fmg(n, h, u, f, ncycle, npre, npost);
    double* r = (double*)malloc(nodes(n) * sizeof(double));
    double fn = sqrt(ora_interior_sumsq(n, f));
    double denom = fn > 0.0 ? fn : 1.0; /* f == 0: absolute residual */
    ora_residual(n, h, u, f, r);
    double rel = sqrt(ora_interior_sumsq(n, r)) / denom;
    int nh = 0;
    if (hist && nh < hist_cap) hist[nh++] = rel;
    int made = 0;
    while (tol > 0.0 && rel > tol && made < max_vcycles) {
        ora_vcycle(n, h, u, f, npre, npost);
        ++made;
        ora_residual(n, h, u, f, r);
        rel = sqrt(ora_interior_sumsq(n, r)) / denom;
        if (hist && nh < hist_cap) hist[nh++] = rel;
    }
    free(r);
    if (tol > 0.0 && rel > tol) return -1;
    return made;
}

/* ------------------------------------------------------------------------ */
/* Step 3 (Section 2, Eq. 2): the QUMOND source div[nu(|grad Phi_N|/a0)
 * grad Phi_N] by finite differences, nu(y) = 1/2 + 1/2 sqrt(1 + 4/y).
 *
 * Reading of the paper: a face-flux form.  For interior node c,
 *   src(c) = (1/h^2) * sum over its 6 faces of nu_f * (Phi(nbr) - Phi(c)),
 * where at the face between nodes P and Q = P + e_a the gradient has normal
 * component (Phi(Q) - Phi(P))/h and each transverse component b is the mean
 * of the central differences at P and Q:
 *   ((Phi(P+e_b) - Phi(P-e_b)) + (Phi(Q+e_b) - Phi(Q-e_b))) / (4h).
 * nu_f = nu(|g_f| / a0) = 0.5 * (1 + sqrt(1 + 4 a0 / |g_f|)); a face with
 * |g_f| = 0 carries no flux.  Boundary nodes get src = 0. */
static double face_flux(int n, double h, double a0, const double* p, int pi, int pj, int pk, int axis)
{
    int qi = pi + (axis == 0), qj = pj + (axis == 1), qk = pk + (axis == 2);
    double gsq = 0.0;
    double dn = p[IDX(n, qi, qj, qk)] - p[IDX(n, pi, pj, pk)];
    double gn = dn / h;
    gsq += gn * gn;
    for (int b = 0; b < 3; ++b) {
        if (b == axis) continue;
        int ei = (b == 0), ej = (b == 1), ek = (b == 2);
        double cp = p[IDX(n, pi + ei, pj + ej, pk + ek)] - p[IDX(n, pi - ei, pj - ej, pk - ek)];
        double cq = p[IDX(n, qi + ei, qj + ej, qk + ek)] - p[IDX(n, qi - ei, qj - ej, qk - ek)];
        double gt = (cp + cq) / (4.0 * h);
        gsq += gt * gt;
    }
    double g = sqrt(gsq);
    if (g == 0.0) return 0.0;
    double nu = 0.5 * (1.0 + sqrt(1.0 + 4.0 * a0 / g));
    return nu * dn; /* flux through the face, times h */
}

void ora_source(int n, double h, double a0, const double* phiN, double* src)
{
    const double ih2 = 1.0 / (h * h);
    memset(src, 0, nodes(n) * sizeof(double));
#pragma omp parallel for schedule(static)
    for (int k = 1; k < n; ++k)
        for (int j = 1; j < n; ++j)
            for (int i = 1; i < n; ++i) {
                /* outward faces: +x, +y, +z from c; inward: from c-e_a to c */
                double s = face_flux(n, h, a0, phiN, i, j, k, 0)
                         - face_flux(n, h, a0, phiN, i - 1, j, k, 0)
                         + face_flux(n, h, a0, phiN, i, j, k, 1)
                         - face_flux(n, h, a0, phiN, i, j - 1, k, 1)
                         + face_flux(n, h, a0, phiN, i, j, k, 2)
                         - face_flux(n, h, a0, phiN, i, j, k - 1, 2);
                src[IDX(n, i, j, k)] = s * ih2;
            }
}

/* ------------------------------------------------------------------------ */
/* Nested-box boundary values (Section 2): a refined box, half the size of its
 * parent, takes its boundary values by interpolating through the parent's
 * solution.  Trilinear interpolation at each boundary node's position. */
static double trilinear(int n, double L, double cx, double cy, double cz, const double* a,
                        double x, double y, double z)
{
    const double h = L / (double)n;
    double t[3] = {(x - (cx - 0.5 * L)) / h, (y - (cy - 0.5 * L)) / h, (z - (cz - 0.5 * L)) / h};
    int i0[3];
    double d[3];
    for (int a3 = 0; a3 < 3; ++a3) {
        double fl = floor(t[a3]);
        int ii = (int)fl;
        if (ii < 0) ii = 0;
        if (ii > n - 1) ii = n - 1;
        i0[a3] = ii;
        d[a3] = t[a3] - (double)ii;
    }
    double v = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a3 = 0; a3 < 2; ++a3) {
                double w = (a3 ? d[0] : 1.0 - d[0]) * (b ? d[1] : 1.0 - d[1]) * (c ? d[2] : 1.0 - d[2]);
                v += w * a[IDX(n, i0[0] + a3, i0[1] + b, i0[2] + c)];
            }
    return v;
}

void ora_boundary_fill(int n, double Lp, double cpx, double cpy, double cpz, const double* up,
                       double L, double cx, double cy, double cz, double* u)
{
    const double h = L / (double)n;
    for (int k = 0; k <= n; ++k)
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n; ++i) {
                if (i != 0 && i != n && j != 0 && j != n && k != 0 && k != n) continue;
                double x = cx - 0.5 * L + i * h, y = cy - 0.5 * L + j * h, z = cz - 0.5 * L + k * h;
                u[IDX(n, i, j, k)] = trilinear(n, Lp, cpx, cpy, cpz, up, x, y, z);
            }
}

/* ------------------------------------------------------------------------ */
/* Forces (Section 2): the gravity -grad Phi by central differences at the
 * nodes, interpolated to a point with the cloud-in-cell (trilinear) weights.
 * Boxes b = 0..nboxes-1 have side L0/ratio^b (ratio 2 in the paper: each
 * refinement halves the box), all centred on c.  A point uses the
 * finest box whose containing cell has all 8 corners at interior nodes
 * (where the central difference exists).  Points in no such cell get 0.
 * Returns the number of points that found no box. */
static int find_cell(int n, double L, double cx, double cy, double cz, double x, double y, double z,
                     int* ijk, double* d)
{
    const double inv_h = (double)n / L;
    double t[3] = {(x - (cx - 0.5 * L)) * inv_h, (y - (cy - 0.5 * L)) * inv_h, (z - (cz - 0.5 * L)) * inv_h};
    for (int a = 0; a < 3; ++a) {
        if (!(t[a] >= 1.0 && t[a] < (double)(n - 1))) return 0;
        double fl = floor(t[a]);
        ijk[a] = (int)fl;
        d[a] = t[a] - fl;
        if (ijk[a] < 1 || ijk[a] > n - 2) return 0;
    }
    return 1;
}

static void grad_at(int n, double L, const double* phi, const int* ijk, const double* d, double* g)
{
    const double h = L / (double)n;
    g[0] = g[1] = g[2] = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                int i = ijk[0] + a, j = ijk[1] + b, k = ijk[2] + c;
                double w = (a ? d[0] : 1.0 - d[0]) * (b ? d[1] : 1.0 - d[1]) * (c ? d[2] : 1.0 - d[2]);
                double gx = -(phi[IDX(n, i + 1, j, k)] - phi[IDX(n, i - 1, j, k)]) / (2.0 * h);
                double gy = -(phi[IDX(n, i, j + 1, k)] - phi[IDX(n, i, j - 1, k)]) / (2.0 * h);
                double gz = -(phi[IDX(n, i, j, k + 1)] - phi[IDX(n, i, j, k - 1)]) / (2.0 * h);
                g[0] += w * gx;
                g[1] += w * gy;
                g[2] += w * gz;
            }
}

int64_t ora_forces(int nboxes, int n, double L0, int ratio, double cx, double cy, double cz, const double* const* phi,
                   const double* qx, const double* qy, const double* qz, int64_t nq,
                   double* gx, double* gy, double* gz)
{
    int64_t missed = 0;
    for (int64_t p = 0; p < nq; ++p) {
        double g[3] = {0.0, 0.0, 0.0};
        int found = 0;
        for (int b = nboxes - 1; b >= 0 && !found; --b) {
            double L = L0 / pow((double)ratio, (double)b);
            int ijk[3];
            double d[3];
            if (find_cell(n, L, cx, cy, cz, qx[p], qy[p], qz[p], ijk, d)) {
                grad_at(n, L, phi[b], ijk, d, g);
                found = 1;
            }
        }
        if (!found) ++missed;
        gx[p] = g[0];
        gy[p] = g[1];
        gz[p] = g[2];
    }
    return missed;
}

/* Rotation curve (Section 2, Eq. 4): v_c^2 = R dPhi/dR at z = 0.
 * Reading of the paper: nbins radii R_k = (k + 1/2) rmax / nbins, and at
 * each radius nphi tracer points at azimuths 2 pi m / nphi in the plane z = c_z.
 * dPhi/dR = -(g_x cos phi + g_y sin phi) with g from the box rule of
 * Section 3.1: the finest box with R < frac * L_b (frac = 0.2 reproduces
 * 0.8 kpc for the 4 kpc box), falling back to coarser boxes whose cell is
 * interior.  The azimuthal mean is summed in index order.
 * vc_out = sign(v_c^2) sqrt(|v_c^2|). */
void ora_rotation_curve(int nboxes, int n, double L0, int ratio, double cx, double cy, double cz,
                        const double* const* phi, int nbins, double rmax, int nphi, double frac,
                        double* r_out, double* vc_out)
{
    const double twopi = 6.283185307179586476925286766559;
    for (int kb = 0; kb < nbins; ++kb) {
        double R = ((double)kb + 0.5) * rmax / (double)nbins;
        int b0 = 0;
        for (int b = nboxes - 1; b >= 0; --b)
            if (R < frac * (L0 / pow((double)ratio, (double)b))) { b0 = b; break; }
        double sum = 0.0;
        for (int m = 0; m < nphi; ++m) {
            double ph = twopi * (double)m / (double)nphi;
            double c = cos(ph), s = sin(ph);
            double x = cx + R * c, y = cy + R * s, z = cz;
            double g[3] = {0.0, 0.0, 0.0};
            for (int b = b0; b >= 0; --b) {
                double L = L0 / pow((double)ratio, (double)b);
                int ijk[3];
                double d[3];
                if (find_cell(n, L, cx, cy, cz, x, y, z, ijk, d)) {
                    grad_at(n, L, phi[b], ijk, d, g);
                    break;
                }
            }
            sum += -(g[0] * c + g[1] * s);
        }
        double v2 = R * (sum / (double)nphi);
        r_out[kb] = R;
        vc_out[kb] = v2 >= 0.0 ? sqrt(v2) : -sqrt(-v2);
    }
}

/* ------------------------------------------------------------------------ */
/* Quality of a fit (Section 3.5): chi^2/n = (1/n) sum_i (V_fit(R_i) - V_obs(R_i))^2 / sigma_obs(R_i)^2,
 * for nsets rotation curves of nbins points each (vc row-major [set][bin]). */
void ora_chi2(const double* vc, const double* v_obs, const double* sigma, int nbins, int nsets, double* chi2)
{
    for (int s = 0; s < nsets; ++s) {
        double acc = 0.0;
        for (int i = 0; i < nbins; ++i) {
            double d = (vc[(size_t)s * nbins + i] - v_obs[i]) / sigma[i];
            acc += d * d;
        }
        chi2[s] = acc / (double)nbins;
    }
}

/* ------------------------------------------------------------------------ */
/* Science extras on a solved set of boxes (tracers and box rule as
 * ora_rotation_curve).
 *
 * Algebraic MOND rotation curve (Eq. 3, compared with QUMOND in Section 3.3):
 * the field at a tracer is taken as nu(|g_N|/a0) g_N, g_N = -grad Phi_N
 * interpolated as for the forces, nu(y) = 1/2 + 1/2 sqrt(1 + 4/y); a tracer
 * with |g_N| = 0 contributes 0.  v_c^2 = R * mean over azimuths of -(g . R^). */
void ora_rotation_curve_algebraic(int nboxes, int n, double L0, int ratio, double cx, double cy, double cz,
                                  const double* const* phiN, int nbins, double rmax, int nphi, double frac,
                                  double a0, double* r_out, double* vc_out)
{
    const double twopi = 6.283185307179586476925286766559;
    for (int kb = 0; kb < nbins; ++kb) {
        double R = ((double)kb + 0.5) * rmax / (double)nbins;
        int b0 = 0;
        for (int b = nboxes - 1; b >= 0; --b)
            if (R < frac * (L0 / pow((double)ratio, (double)b))) { b0 = b; break; }
        double sum = 0.0;
        for (int m = 0; m < nphi; ++m) {
            double ph = twopi * (double)m / (double)nphi;
            double c = cos(ph), s = sin(ph);
            double g[3] = {0.0, 0.0, 0.0};
            for (int b = b0; b >= 0; --b) {
                double L = L0 / pow((double)ratio, (double)b);
                int ijk[3];
                double d[3];
                if (find_cell(n, L, cx, cy, cz, cx + R * c, cy + R * s, cz, ijk, d)) {
                    grad_at(n, L, phiN[b], ijk, d, g);
                    break;
                }
            }
            double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            double nu = gm > 0.0 ? 0.5 + 0.5 * sqrt(1.0 + 4.0 * a0 / gm) : 0.0;
            sum += -nu * (g[0] * c + g[1] * s);
        }
        double v2 = R * (sum / (double)nphi);
        r_out[kb] = R;
        vc_out[kb] = v2 >= 0.0 ? sqrt(v2) : -sqrt(-v2);
    }
}

/* Vertical velocity dispersion of an isothermal stellar layer (Section 5.6):
 * sigma_z^2 = -dPhi/dz * rho_s / (d rho_s/dz), rho_s the stellar density.  For
 * rho_s ~ sech^2(z/h), rho_s / (d rho_s/dz) = -h / (2 tanh(z/h)), so at height z_eval above the plane
 * sigma_z^2(R) = <dPhi/dz>(R, z_eval) * h / (2 tanh(z_eval/h)), the mean of
 * dPhi/dz = -g_z over the nphi azimuths.  sig_out = sign(s) sqrt(|s|). */
void ora_sigma_z(int nboxes, int n, double L0, int ratio, double cx, double cy, double cz, const double* const* phi,
                 int nbins, double rmax, int nphi, double frac, double z_eval, double h, double* r_out,
                 double* sig_out)
{
    const double twopi = 6.283185307179586476925286766559;
    for (int kb = 0; kb < nbins; ++kb) {
        double R = ((double)kb + 0.5) * rmax / (double)nbins;
        int b0 = 0;
        for (int b = nboxes - 1; b >= 0; --b)
            if (R < frac * (L0 / pow((double)ratio, (double)b))) { b0 = b; break; }
        double sum = 0.0;
        for (int m = 0; m < nphi; ++m) {
            double ph = twopi * (double)m / (double)nphi;
            double c = cos(ph), s = sin(ph);
            double g[3] = {0.0, 0.0, 0.0};
            for (int b = b0; b >= 0; --b) {
                double L = L0 / pow((double)ratio, (double)b);
                int ijk[3];
                double d[3];
                if (find_cell(n, L, cx, cy, cz, cx + R * c, cy + R * s, cz + z_eval, ijk, d)) {
                    grad_at(n, L, phi[b], ijk, d, g);
                    break;
                }
            }
            sum += -g[2];
        }
        double s2 = (sum / (double)nphi) * h / (2.0 * tanh(z_eval / h));
        r_out[kb] = R;
        sig_out[kb] = s2 >= 0.0 ? sqrt(s2) : -sqrt(-s2);
    }
}

/* ------------------------------------------------------------------------ */
/* Far-field boundary values of the outermost box.  Section 2 puts Phi = 0 on
 * a box 2^10 times larger than the galaxy and refines inwards; with fewer
 * boxes the outermost boundary lies close to the mass, and the boundary values
 * come from the mass inside the box instead:
 *
 *  - Phi_N: the exterior multipole expansion of the node masses m_k = rho_k h^3
 *    (all nodes) about their centre of mass c, truncated at degree lmax:
 *      Phi_N(x) = -G sum_k m_k sum_{l=0}^{lmax} |x_k - c|^l / |x - c|^{l+1} P_l(cos g_k),
 *    g_k the angle between x_k - c and x - c.  Written with the addition
 *    theorem of Legendre polynomials, P_l(cos g) = sum_{m=0}^{l} (2 - [m=0])
 *    (l-m)!/(l+m)! P_l^m(cos t) P_l^m(cos t') cos(m (f - f')), and with the
 *    solid harmonics T_lm(d) = |d|^l P_l^m(cos t) e^{i m f} of d = (dx, dy, dz)
 *    (polynomials in dx, dy, dz), the expansion is
 *      Phi_N(x) = -G sum_l sum_m w_lm [Re T_lm(d) A_lm + Im T_lm(d) B_lm] / |d|^{2l+1},
 *    w_lm = (2 - [m=0]) (l-m)!/(l+m)!, A_lm + i B_lm = sum_k m_k T_lm(x_k - c), d = x - c.
 *  - Phi: the QUMOND potential of the whole mass M = sum_k m_k taken as a
 *    point at c, F(|x - c|) with F'(r) = nu(G M/(a0 r^2)) G M/r^2 and
 *    nu(y) = 1/2 + 1/2 sqrt(1 + 4/y) (Section 2, Eq. 2 for a spherical mass):
 *      F(r) = -A/(2r) + (1/2) [ -sqrt(A^2 + C r^2)/r + sqrt(C) asinh(sqrt(C) r / A) ],
 *    A = G M, C = 4 a0 A.  Far from the galaxy the QUMOND field is that of
 *    its total mass; only the monopole is kept.
 *
 * T_lm follows from P_l^m (taken without the (-1)^m phase, which cancels in
 * the products): T_mm = (2m-1)!! (dx + i dy)^m, T_{m+1,m} = (2m+1) dz T_mm,
 * (l-m) T_lm = (2l-1) dz T_{l-1,m} - (l+m-1) |d|^2 T_{l-2,m}.
 * Writes the boundary nodes of phiN and phi (interior untouched); with M = 0
 * both are set to 0.  lmax <= 16.  Returns M. */
#define ORA_LMAX 16
static void solid_harmonics(int lmax, double dx, double dy, double dz, double re[ORA_LMAX + 1][ORA_LMAX + 1],
                            double im[ORA_LMAX + 1][ORA_LMAX + 1])
{
    const double r2 = dx * dx + dy * dy + dz * dz;
    double pr = 1.0, pi = 0.0; /* (dx + i dy)^m */
    double dfact = 1.0;        /* (2m-1)!! */
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) {
            double nr = pr * dx - pi * dy, ni = pr * dy + pi * dx;
            pr = nr;
            pi = ni;
            dfact *= (double)(2 * m - 1);
        }
        re[m][m] = dfact * pr;
        im[m][m] = dfact * pi;
        if (m + 1 <= lmax) {
            re[m + 1][m] = (double)(2 * m + 1) * dz * re[m][m];
            im[m + 1][m] = (double)(2 * m + 1) * dz * im[m][m];
        }
        for (int l = m + 2; l <= lmax; ++l) {
            re[l][m] = ((double)(2 * l - 1) * dz * re[l - 1][m] - (double)(l + m - 1) * r2 * re[l - 2][m]) / (double)(l - m);
            im[l][m] = ((double)(2 * l - 1) * dz * im[l - 1][m] - (double)(l + m - 1) * r2 * im[l - 2][m]) / (double)(l - m);
        }
    }
}

double ora_far_field(int n, double L, double cx, double cy, double cz, const double* rho, double G, double a0,
                     int lmax, double* phiN, double* phi)
{
    if (lmax < 0) lmax = 0;
    if (lmax > ORA_LMAX) lmax = ORA_LMAX;
    const double h = L / (double)n, h3 = h * h * h;
    const double x0 = cx - 0.5 * L, y0 = cy - 0.5 * L, z0 = cz - 0.5 * L;
    /* total mass and centre of mass */
    double M = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int k = 0; k <= n; ++k)
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n; ++i) {
                double m = rho[IDX(n, i, j, k)] * h3;
                M += m;
                mx += m * (x0 + i * h);
                my += m * (y0 + j * h);
                mz += m * (z0 + k * h);
            }
    if (M == 0.0) {
        for (int k = 0; k <= n; ++k)
            for (int j = 0; j <= n; ++j)
                for (int i = 0; i <= n; ++i)
                    if (i == 0 || i == n || j == 0 || j == n || k == 0 || k == n)
                        phiN[IDX(n, i, j, k)] = phi[IDX(n, i, j, k)] = 0.0;
        return 0.0;
    }
    const double comx = mx / M, comy = my / M, comz = mz / M;
    /* moments A_lm + i B_lm */
    double A[ORA_LMAX + 1][ORA_LMAX + 1], B[ORA_LMAX + 1][ORA_LMAX + 1];
    double re[ORA_LMAX + 1][ORA_LMAX + 1], im[ORA_LMAX + 1][ORA_LMAX + 1];
    memset(A, 0, sizeof(A));
    memset(B, 0, sizeof(B));
    for (int k = 0; k <= n; ++k)
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n; ++i) {
                double m = rho[IDX(n, i, j, k)] * h3;
                if (m == 0.0) continue;
                solid_harmonics(lmax, x0 + i * h - comx, y0 + j * h - comy, z0 + k * h - comz, re, im);
                for (int l = 0; l <= lmax; ++l)
                    for (int mm = 0; mm <= l; ++mm) {
                        A[l][mm] += m * re[l][mm];
                        B[l][mm] += m * im[l][mm];
                    }
            }
    /* w_lm = (2 - [m=0]) (l-m)!/(l+m)! */
    double w[ORA_LMAX + 1][ORA_LMAX + 1];
    for (int l = 0; l <= lmax; ++l)
        for (int mm = 0; mm <= l; ++mm) {
            double r = 1.0;
            for (int t = l - mm + 1; t <= l + mm; ++t) r /= (double)t;
            w[l][mm] = (mm == 0 ? 1.0 : 2.0) * r;
        }
    const double Am = G * M, C = 4.0 * a0 * Am;
    for (int k = 0; k <= n; ++k)
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n; ++i) {
                if (i != 0 && i != n && j != 0 && j != n && k != 0 && k != n) continue;
                double dx = x0 + i * h - comx, dy = y0 + j * h - comy, dz = z0 + k * h - comz;
                double r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
                solid_harmonics(lmax, dx, dy, dz, re, im);
                double sum = 0.0, rpow = r; /* |d|^{2l+1} */
                for (int l = 0; l <= lmax; ++l) {
                    double sl = 0.0;
                    for (int mm = 0; mm <= l; ++mm) sl += w[l][mm] * (re[l][mm] * A[l][mm] + im[l][mm] * B[l][mm]);
                    sum += sl / rpow;
                    rpow *= r2;
                }
                phiN[IDX(n, i, j, k)] = -G * sum;
                phi[IDX(n, i, j, k)] = -Am / (2.0 * r) +
                                       0.5 * (-sqrt(Am * Am + C * r2) / r + sqrt(C) * asinh(sqrt(C) * r / Am));
            }
    return M;
}
