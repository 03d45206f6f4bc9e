// Multigrid kernels of the QUMOND solves (Section 2, steps 2 and 4): red-black
// Gauss-Seidel half-sweeps, residual restriction, prolongation, boundary
// injection, the single-CTA coarse-grid solver, and the FP64 outer steps of
// the defect correction.  T is the smoothing precision (float or double).
//
// Level arrays use the colour-split layout of qumond_internal.h.  Two facts
// of red-black Gauss-Seidel are used to skip dead work (both exact in exact
// arithmetic, so the iterates are those of the textbook V-cycle):
//  * a node's update does not read its own old value, so after a coarse-grid
//    correction only the black nodes need the prolonged correction before the
//    next red half-sweep, and an FMG interpolation only has to fill black
//    nodes;
//  * right after a black half-sweep the black residuals are zero, so the
//    residual to restrict is nonzero only at red nodes.
#include "qumond_internal.h"

#include <cstdio>

namespace qumond {

namespace {

constexpr int kBX = 32;
constexpr int kBY = 8;

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// One half-sweep: every interior node of `colour` is set to
//   (sum of its 6 neighbours - h^2 f) / 6,
// its neighbours all being of the other colour.  ZERO: the neighbours are
// known to be zero (first sweep of a correction that starts from zero).
template <typename T, bool ZERO>
__device__ __forceinline__ void rb_node(T* __restrict__ own, const T* __restrict__ other, const T* __restrict__ f,
                                        const LevelView& v, int colour, T h2, T sixth, int m, int j, int k)
{
    const int p = (colour + j + k) & 1;  // parity of i in this row
    if (p == 0 && m == 0) return;        // i = 0 is a boundary node
    const long long row = ((long long)k * (v.n + 1) + j) * v.M;
    T s = T(0);
    if (!ZERO) {
        const T* o = other + row;
        const long long P = v.M, Q = (long long)v.M * (v.n + 1);
        s = (o[m - 1 + p] + o[m + p]) + (o[m - P] + o[m + P]) + (o[m - Q] + o[m + Q]);
    }
    own[row + m] = (s - h2 * f[row + m]) * sixth;
}

// The set index of a context with several sets, folded into blockIdx.z
// (per planes per set): returns it and the plane index within the set.
__device__ __forceinline__ int set_of(int per, int& within)
{
    if ((int)gridDim.z == per) {  // one set: no division
        within = (int)blockIdx.z;
        return 0;
    }
    const int s = (int)blockIdx.z / per;
    within = (int)blockIdx.z - s * per;
    return s;
}

template <typename T, bool ZERO>
__global__ void __launch_bounds__(kBX * kBY)
rb_half_kernel(T* __restrict__ own, const T* __restrict__ other, const T* __restrict__ f, LevelView v, int colour,
               T h2, T sixth, const SolveState* __restrict__ act)
{
    int kz;
    const int set = set_of(v.n - 1, kz);
    if (act && !act[set].cont) return;
    const long long so = (long long)set * 2 * v.cs;
    const int half = v.n >> 1;
    const int m = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y + 1;
    const int k = kz + 1;
    if (m >= half || j >= v.n) return;
    rb_node<T, ZERO>(own + so, other + so, f + so, v, colour, h2, sixth, m, j, k);
}

// The same half-sweep on FP32 levels with four consecutive entries of a row
// per thread (the parity of i is the same along a row): 16-byte loads of the
// row, its four neighbour rows and f, two scalars for the x-neighbours past
// the ends, one 16-byte store; the node arithmetic is rb_node's, in the same
// order.  half = n/2 is a multiple of 4, so a group lies wholly inside or
// outside the row's entries; the scalar before entry 0 (read from the padding
// at the end of the previous row) only feeds the boundary node i = 0, which
// is not written.
// Block shapes: VX threads along a row (4 VX entries) x 128/VX rows.  The
// default 8 x 16 suits large levels; the small levels (n/2 = 8 .. 32 entries
// per row) leave most of an 8-wide block idle, so a context can pick 4 x 32 or
// 2 x 64 for levels n <= 64 (params.tile_small).  Every shape gives the same
// bits: each thread's entries are updated by the same arithmetic.
constexpr int kVX = 8;  // default: 32 entries x 16 rows per block
constexpr int kVThreads = 128;
constexpr int kVBlocksPerSM = 16;  // full occupancy (<= 32 registers): the small levels are latency-bound
constexpr int kTileSmallN = 64;  // the alternative shapes apply to levels with n <= this

template <bool ZERO, int VX = kVX>
__global__ void __launch_bounds__(kVThreads, kVBlocksPerSM)
rb_half4_kernel(float* __restrict__ own, const float* __restrict__ other, const float* __restrict__ f, LevelView v,
                int colour, float h2, float sixth, const SolveState* __restrict__ act)
{
    int kz;
    const int set = set_of(v.n - 1, kz);
    if (act && !act[set].cont) return;
    {
        const long long so = (long long)set * 2 * v.cs;
        own += so, other += so, f += so;
    }
    const int half = v.n >> 1;
    const int mA = 4 * (blockIdx.x * VX + threadIdx.x);
    const int j = blockIdx.y * (kVThreads / VX) + threadIdx.y + 1;
    const int k = kz + 1;
    if (mA >= half || j >= v.n) return;
    const int p = (colour + j + k) & 1;
    const long long row = ((long long)k * (v.n + 1) + j) * v.M;
    float sum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (!ZERO) {
        const float* o = other + row + mA;
        const long long P = v.M, Q = (long long)v.M * (v.n + 1);
        const float4 V = *reinterpret_cast<const float4*>(o);
        const float x[6] = {o[-1], V.x, V.y, V.z, V.w, o[4]};  // entries mA-1 .. mA+4
        const float4 Y0 = *reinterpret_cast<const float4*>(o - P), Y1 = *reinterpret_cast<const float4*>(o + P);
        const float4 Z0 = *reinterpret_cast<const float4*>(o - Q), Z1 = *reinterpret_cast<const float4*>(o + Q);
        const float y0[4] = {Y0.x, Y0.y, Y0.z, Y0.w}, y1[4] = {Y1.x, Y1.y, Y1.z, Y1.w};
        const float z0[4] = {Z0.x, Z0.y, Z0.z, Z0.w}, z1[4] = {Z1.x, Z1.y, Z1.z, Z1.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float lo = p ? x[e + 1] : x[e];
            const float hi = p ? x[e + 2] : x[e + 1];
            sum[e] = (lo + hi) + (y0[e] + y1[e]) + (z0[e] + z1[e]);
        }
    }
    const float4 F = *reinterpret_cast<const float4*>(f + row + mA);
    const float fv[4] = {F.x, F.y, F.z, F.w};
    float r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) r[e] = (sum[e] - h2 * fv[e]) * sixth;
    if (p == 0 && mA == 0) {  // i = 0 is a boundary node
        own[row + 1] = r[1], own[row + 2] = r[2], own[row + 3] = r[3];
    } else {
        *reinterpret_cast<float4*>(own + row + mA) = make_float4(r[0], r[1], r[2], r[3]);
    }
}

// The first sweep of a correction that starts from zero, both half-sweeps in
// one pass (FP32 levels, four entries per thread as in rb_half4_kernel).  The
// red half-sweep from zero sets each interior red node to (0 - h^2 f)/6, a
// function of its own f alone, so the black half-sweep after it can form its
// red neighbours from f instead of reading them back: each thread writes the
// four red entries of its row that rb_half4_kernel<true> would write and
// updates the four black entries of the row with rb_half4_kernel<false>'s
// sums in their order, so the results are the same bits as the two launches.
// Red neighbours on the boundary (i, j or k = 0 or n) are not written by the
// red half-sweep; they are read from e, as the black half-sweep reads them.
constexpr int kFirstBlocksPerSM = 10;  // <= 48 registers: the fused sweep holds both colours' values
template <int VX = kVX>
__global__ void __launch_bounds__(kVThreads, kFirstBlocksPerSM)
rb_first4_kernel(float* __restrict__ e, const float* __restrict__ f, LevelView v, float h2, float sixth,
                 const SolveState* __restrict__ act)
{
    int kz;
    const int set = set_of(v.n - 1, kz);
    if (act && !act[set].cont) return;
    {
        const long long so = (long long)set * 2 * v.cs;
        e += so, f += so;
    }
    float* red = e;
    float* black = e + v.cs;
    const float* fr = f;
    const float* fb = f + v.cs;
    const int n = v.n, half = n >> 1;
    const int mA = 4 * (blockIdx.x * VX + threadIdx.x);
    const int j = blockIdx.y * (kVThreads / VX) + threadIdx.y + 1;
    const int k = kz + 1;
    if (mA >= half || j >= n) return;
    const int pr = (j + k) & 1;  // parity of i along this row: red entries
    const int pb = pr ^ 1;       // black entries
    const long long row = ((long long)k * (n + 1) + j) * v.M;
    const long long P = v.M, Q = (long long)v.M * (n + 1);
    const float zero = 0.0f;
    // red entries mA-1 .. mA+4 of this row after the half-sweep from zero
    const float* fo = fr + row + mA;
    const float4 FV = *reinterpret_cast<const float4*>(fo);
    const float fv[4] = {FV.x, FV.y, FV.z, FV.w};
    float rr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) rr[q] = (zero - h2 * fv[q]) * sixth;
    float x[6] = {(zero - h2 * fo[-1]) * sixth, rr[0], rr[1], rr[2], rr[3], (zero - h2 * fo[4]) * sixth};
    if (pr == 0) {  // red boundary nodes of the row: i = 0 (entry 0) and i = n (entry half)
        if (mA == 0) x[1] = red[row];
        if (mA + 4 == half) x[5] = red[row + half];
    }
    // red entries mA .. mA+3 of the neighbouring rows (boundary rows as stored)
    float y0[4], y1[4], z0[4], z1[4];
    auto nbr = [&](long long off, bool bnd, float* out) {
        if (bnd) {
            const float4 E = *reinterpret_cast<const float4*>(red + row + mA + off);
            out[0] = E.x, out[1] = E.y, out[2] = E.z, out[3] = E.w;
        } else {
            const float4 F = *reinterpret_cast<const float4*>(fr + row + mA + off);
            out[0] = (zero - h2 * F.x) * sixth, out[1] = (zero - h2 * F.y) * sixth;
            out[2] = (zero - h2 * F.z) * sixth, out[3] = (zero - h2 * F.w) * sixth;
        }
    };
    nbr(-P, j == 1, y0);
    nbr(P, j + 1 == n, y1);
    nbr(-Q, k == 1, z0);
    nbr(Q, k + 1 == n, z1);
    const float4 FB = *reinterpret_cast<const float4*>(fb + row + mA);
    const float fbv[4] = {FB.x, FB.y, FB.z, FB.w};
    float rb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float lo = pb ? x[q + 1] : x[q];
        const float hi = pb ? x[q + 2] : x[q + 1];
        const float sum = (lo + hi) + (y0[q] + y1[q]) + (z0[q] + z1[q]);
        rb[q] = (sum - h2 * fbv[q]) * sixth;
    }
    if (pr == 0 && mA == 0) {  // i = 0 is a boundary node
        red[row + 1] = rr[1], red[row + 2] = rr[2], red[row + 3] = rr[3];
    } else {
        *reinterpret_cast<float4*>(red + row + mA) = make_float4(rr[0], rr[1], rr[2], rr[3]);
    }
    if (pb == 0 && mA == 0) {
        black[row + 1] = rb[1], black[row + 2] = rb[2], black[row + 3] = rb[3];
    } else {
        *reinterpret_cast<float4*>(black + row + mA) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    }
}

// Residual f - L u at the red node (i, j, k) of a level.
template <typename T>
__device__ __forceinline__ T red_residual(const T* __restrict__ e, const T* __restrict__ f, const LevelView& v, int i,
                                          int j, int k, T ih2)
{
    const int p = (j + k) & 1;
    const int m = i >> 1;
    const long long row = ((long long)k * (v.n + 1) + j) * v.M;
    const T* eb = e + v.cs + row;
    const long long P = v.M, Q = (long long)v.M * (v.n + 1);
    const T s = (eb[m - 1 + p] + eb[m + p]) + (eb[m - P] + eb[m + P]) + (eb[m - Q] + eb[m + Q]);
    return f[row + m] - (s - T(6) * e[row + m]) * ih2;
}

// Full weighting of the residual onto the coarse interior node (I, J, K):
// weight 1/8 at the coinciding fine node and 1/32 at its 12 edge neighbours
// (the other 14 fine nodes of the stencil are black, residual zero).
template <typename T>
__device__ __forceinline__ void restrict_node(const T* __restrict__ ef, const T* __restrict__ ff, const LevelView& vf,
                                              T* __restrict__ fc, const LevelView& vc, T ih2, int I, int J, int K)
{
    const int i = 2 * I, j = 2 * J, k = 2 * K;
    T edge = (red_residual(ef, ff, vf, i + 1, j + 1, k, ih2) + red_residual(ef, ff, vf, i - 1, j + 1, k, ih2))
           + (red_residual(ef, ff, vf, i + 1, j - 1, k, ih2) + red_residual(ef, ff, vf, i - 1, j - 1, k, ih2));
    edge += (red_residual(ef, ff, vf, i + 1, j, k + 1, ih2) + red_residual(ef, ff, vf, i - 1, j, k + 1, ih2))
          + (red_residual(ef, ff, vf, i + 1, j, k - 1, ih2) + red_residual(ef, ff, vf, i - 1, j, k - 1, ih2));
    edge += (red_residual(ef, ff, vf, i, j + 1, k + 1, ih2) + red_residual(ef, ff, vf, i, j - 1, k + 1, ih2))
          + (red_residual(ef, ff, vf, i, j + 1, k - 1, ih2) + red_residual(ef, ff, vf, i, j - 1, k - 1, ih2));
    const T centre = red_residual(ef, ff, vf, i, j, k, ih2);
    fc[node_off(vc, I, J, K)] = T(0.125) * centre + T(0.03125) * edge;
}

template <typename T>
__global__ void __launch_bounds__(kBX * kBY)
restrict_resid_red_kernel(const T* __restrict__ ef, const T* __restrict__ ff, LevelView vf, T* __restrict__ fc,
                          LevelView vc, T ih2, const SolveState* __restrict__ act)
{
    int kz;
    const int set = set_of(vc.n - 1, kz);
    if (act && !act[set].cont) return;
    const long long sf = (long long)set * 2 * vf.cs, sc = (long long)set * 2 * vc.cs;
    const int I = blockIdx.x * kBX + threadIdx.x + 1;
    const int J = blockIdx.y * kBY + threadIdx.y + 1;
    const int K = kz + 1;
    if (I >= vc.n || J >= vc.n) return;
    restrict_node<T>(ef + sf, ff + sf, vf, fc + sc, vc, ih2, I, J, K);
}

// The same restriction on FP32 levels without recomputation: a CTA owns a
// tile of 32 x 8 coarse (I, J) columns and rk coarse planes (up to 8, fewer
// when the level has too few tiles to fill the GPU), and marches over
// the fine planes 2K0-1 .. 2K1-1.  For each fine plane it computes the red
// residuals of the rows 2J0-1 .. 2J0+15 and entries I0-1 .. I0+34 once (four
// consecutive entries per thread, 16-byte loads, red_residual's arithmetic in
// its order) into a three-plane shared ring; after each odd plane 2K+1 it
// full-weights coarse plane K from the ring with restrict_node's sums in their
// order.  A red residual is evaluated once per CTA instead of by each of the
// up to four coarse nodes that weight it, and the loads of fine plane k+1 are
// issued before the barriers of plane k.
constexpr int kRI = 32, kRJ = 8, kRK = 8;  // coarse tile and the most planes per CTA
constexpr int kRG = 9;                     // groups of four red entries per fine row (36 entries)
constexpr int kRR = 2 * kRJ + 1;           // fine rows per tile
static_assert(kRR * kRG <= kRI * kRJ, "one thread per residual group");

__global__ void __launch_bounds__(kRI * kRJ)
restrict_resid4_kernel(const float* __restrict__ ef, const float* __restrict__ ff, LevelView vf,
                       float* __restrict__ fc, LevelView vc, float ih2, int rk, int zper,
                       const SolveState* __restrict__ act)
{
    __shared__ __align__(16) float ring[3][kRR][kRG * 4];
    int kz;
    const int set = set_of(zper, kz);
    if (act && !act[set].cont) return;
    {
        const long long sf = (long long)set * 2 * vf.cs;
        ef += sf, ff += sf, fc += (long long)set * 2 * vc.cs;
    }
    const int n = vf.n, nc = vc.n;
    const int I0 = 1 + blockIdx.x * kRI, J0 = 1 + blockIdx.y * kRJ, K0 = 1 + kz * rk;
    const int K1 = min(K0 + rk, nc);  // coarse planes K0 .. K1-1
    const int t = threadIdx.x;
    const int mbase = I0 - 1;          // a multiple of 32: the groups start on 16-byte boundaries
    // residual phase: row rr, group rg of the fine tile
    const int rr = t / kRG, rg = t % kRG;
    const int jf = 2 * J0 - 1 + rr;
    const int m0 = mbase + 4 * rg;
    const bool ract = t < kRR * kRG && jf >= 1 && jf <= n - 1 && m0 < vf.M;
    // coarse phase: node (I, J)
    const int cI = t % kRI, cJ = t / kRI;
    const int I = I0 + cI, J = J0 + cJ;
    const bool cact = I <= nc - 1 && J <= nc - 1;
    const long long P = vf.M, Q = (long long)vf.M * (n + 1);
    // the inputs of one fine plane: the black row with its two outer neighbours, the black rows j-1, j+1
    // and planes k-1, k+1, the red values and f
    struct In {
        float4 V, Y0, Y1, Z0, Z1, E, F;
        float xl, xr;
    };
    auto load = [&](int k, In& d) {
        const long long row = ((long long)k * (n + 1) + jf) * vf.M + m0;
        const float* eb = ef + vf.cs + row;
        d.V = *reinterpret_cast<const float4*>(eb);
        d.xl = eb[-1], d.xr = eb[4];
        d.Y0 = *reinterpret_cast<const float4*>(eb - P), d.Y1 = *reinterpret_cast<const float4*>(eb + P);
        d.Z0 = *reinterpret_cast<const float4*>(eb - Q), d.Z1 = *reinterpret_cast<const float4*>(eb + Q);
        d.E = *reinterpret_cast<const float4*>(ef + row);
        d.F = *reinterpret_cast<const float4*>(ff + row);
    };
    In cur;
    if (ract) load(2 * K0 - 1, cur);
    for (int k = 2 * K0 - 1; k <= 2 * K1 - 1; ++k) {
        if (ract) {
            const int p = (jf + k) & 1;
            const float x[6] = {cur.xl, cur.V.x, cur.V.y, cur.V.z, cur.V.w, cur.xr};
            const float y0[4] = {cur.Y0.x, cur.Y0.y, cur.Y0.z, cur.Y0.w}, y1[4] = {cur.Y1.x, cur.Y1.y, cur.Y1.z, cur.Y1.w};
            const float z0[4] = {cur.Z0.x, cur.Z0.y, cur.Z0.z, cur.Z0.w}, z1[4] = {cur.Z1.x, cur.Z1.y, cur.Z1.z, cur.Z1.w};
            const float ev[4] = {cur.E.x, cur.E.y, cur.E.z, cur.E.w}, fv[4] = {cur.F.x, cur.F.y, cur.F.z, cur.F.w};
            float r[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float lo = p ? x[e + 1] : x[e];
                const float hi = p ? x[e + 2] : x[e + 1];
                const float sum = (lo + hi) + (y0[e] + y1[e]) + (z0[e] + z1[e]);
                r[e] = fv[e] - (sum - 6.0f * ev[e]) * ih2;
            }
            *reinterpret_cast<float4*>(&ring[k % 3][rr][4 * rg]) = make_float4(r[0], r[1], r[2], r[3]);
            // the next plane's loads are in flight across the barriers and the coarse plane below
            if (k < 2 * K1 - 1) load(k + 1, cur);
        }
        __syncthreads();
        if ((k & 1) && k >= 2 * K0 + 1 && cact) {
            const int K = (k - 1) >> 1;
            const float(*pm)[kRG * 4] = ring[(k + 1) % 3];  // fine plane 2K-1
            const float(*p0)[kRG * 4] = ring[(k + 2) % 3];  // 2K
            const float(*pp)[kRG * 4] = ring[k % 3];        // 2K+1
            // fine node (i, j) = (2I, 2J): row 2cJ+1 of the tile; entries I-1 (i-1) and I (i, i+1)
            const int a = 2 * cJ + 1, lo = cI, hi = cI + 1;
            float edge = (p0[a + 1][hi] + p0[a + 1][lo]) + (p0[a - 1][hi] + p0[a - 1][lo]);
            edge += (pp[a][hi] + pp[a][lo]) + (pm[a][hi] + pm[a][lo]);
            edge += (pp[a + 1][hi] + pp[a - 1][hi]) + (pm[a + 1][hi] + pm[a - 1][hi]);
            const float centre = p0[a][hi];
            fc[node_off(vc, I, J, K)] = 0.125f * centre + 0.03125f * edge;
        }
        __syncthreads();
    }
}

// The coarse-grid correction / FMG interpolation on FP32 levels with four
// consecutive black entries of a fine row per thread.  For a coarse row
// (J', K') the nodes I = mA .. mA+4 alternate between the two colour arrays
// (entries mA/2 .. mA/2+2 and mA/2 .. mA/2+1), read with 8-byte loads; the
// sums are prolong_node's, in its order, and the fine row is read and
// written with 16-byte accesses.
template <bool ADD, int VX = kVX>
__global__ void __launch_bounds__(kVThreads, kVBlocksPerSM)
prolong_black4_kernel(const float* __restrict__ ec, LevelView vc, float* __restrict__ ef, LevelView vf,
                      const SolveState* __restrict__ act)
{
    int kz;
    const int set = set_of(vf.n - 1, kz);
    if (act && !act[set].cont) return;
    ec += (long long)set * 2 * vc.cs;
    ef += (long long)set * 2 * vf.cs;
    const int half = vf.n >> 1;
    const int mA = 4 * (blockIdx.x * VX + threadIdx.x);
    const int j = blockIdx.y * (kVThreads / VX) + threadIdx.y + 1;
    const int k = kz + 1;
    if (mA >= half || j >= vf.n) return;
    const int p = (1 + j + k) & 1;  // parity of i of the black nodes in this row
    const int J0 = j >> 1, J1 = (j + 1) >> 1, K0 = k >> 1, K1 = (k + 1) >> 1;
    // coarse nodes I = mA + d (d = 0..4) of row (Jr, Kr)
    auto row5 = [&](int Jr, int Kr, float* c) {
        const int ca = (mA + Jr + Kr) & 1;  // colour of the even d
        const long long base = ((long long)Kr * (vc.n + 1) + Jr) * vc.M + (mA >> 1);
        const float* A = ec + (long long)ca * vc.cs + base;
        const float* B = ec + (long long)(ca ^ 1) * vc.cs + base;
        const float2 a2 = *reinterpret_cast<const float2*>(A);
        const float2 b2 = *reinterpret_cast<const float2*>(B);
        c[0] = a2.x, c[1] = b2.x, c[2] = a2.y, c[3] = b2.y, c[4] = A[2];
    };
    float c00[5], c10[5], c01[5], c11[5];  // (J0, K0), (J1, K0), (J0, K1), (J1, K1)
    row5(J0, K0, c00);
    row5(J1, K0, c10);
    row5(J0, K1, c01);
    row5(J1, K1, c11);
    const long long o = vf.cs + ((long long)k * (vf.n + 1) + j) * vf.M + mA;
    float4 cur = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (ADD) cur = *reinterpret_cast<const float4*>(ef + o);
    const float cv[4] = {cur.x, cur.y, cur.z, cur.w};
    float r[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        // I0 = mA + e, I1 = mA + e + p
        const float a0 = c00[e], a1 = p ? c00[e + 1] : c00[e];
        const float b0 = c10[e], b1 = p ? c10[e + 1] : c10[e];
        const float d0 = c01[e], d1 = p ? c01[e + 1] : c01[e];
        const float g0 = c11[e], g1 = p ? c11[e + 1] : c11[e];
        float sv = (a0 + a1) + (b0 + b1);
        sv += (d0 + d1) + (g0 + g1);
        sv *= 0.125f;
        r[e] = ADD ? cv[e] + sv : sv;
    }
    if (p == 0 && mA == 0) {  // i = 0 is a boundary node
        ef[o + 1] = r[1], ef[o + 2] = r[2], ef[o + 3] = r[3];
    } else {
        *reinterpret_cast<float4*>(ef + o) = make_float4(r[0], r[1], r[2], r[3]);
    }
}

// Full weighting of a right-hand side (both colours) onto coarse interior nodes.
template <typename T>
__global__ void __launch_bounds__(kBX * kBY)
restrict_full_kernel(const T* __restrict__ ff, LevelView vf, T* __restrict__ fc, LevelView vc)
{
    int kz;
    const int set = set_of(vc.n - 1, kz);
    ff += (long long)set * 2 * vf.cs;
    fc += (long long)set * 2 * vc.cs;
    const int I = blockIdx.x * kBX + threadIdx.x + 1;
    const int J = blockIdx.y * kBY + threadIdx.y + 1;
    const int K = kz + 1;
    if (I >= vc.n || J >= vc.n) return;
    const T w[3] = {T(0.25), T(0.5), T(0.25)};
    T acc = T(0);
    for (int c = -1; c <= 1; ++c)
        for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a)
                acc += (w[a + 1] * w[b + 1] * w[c + 1]) * ff[node_off(vf, 2 * I + a, 2 * J + b, 2 * K + c)];
    fc[node_off(vc, I, J, K)] = acc;
}

// Trilinear prolongation of a coarse array to the black interior nodes of the
// next finer level: assign (FMG interpolation) or add (coarse-grid correction).
template <typename T, bool ADD>
__device__ __forceinline__ void prolong_node(const T* __restrict__ ec, const LevelView& vc, T* __restrict__ ef,
                                             const LevelView& vf, int m, int j, int k)
{
    const int p = (1 + j + k) & 1;
    const int i = 2 * m + p;
    if (i < 1) return;
    const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1, K0 = k >> 1, K1 = (k + 1) >> 1;
    T s = (ec[node_off(vc, I0, J0, K0)] + ec[node_off(vc, I1, J0, K0)])
        + (ec[node_off(vc, I0, J1, K0)] + ec[node_off(vc, I1, J1, K0)]);
    s += (ec[node_off(vc, I0, J0, K1)] + ec[node_off(vc, I1, J0, K1)])
       + (ec[node_off(vc, I0, J1, K1)] + ec[node_off(vc, I1, J1, K1)]);
    s *= T(0.125);
    const long long o = vf.cs + ((long long)k * (vf.n + 1) + j) * vf.M + m;
    ef[o] = ADD ? ef[o] + s : s;
}

template <typename T, bool ADD>
__global__ void __launch_bounds__(kBX * kBY)
prolong_black_kernel(const T* __restrict__ ec, LevelView vc, T* __restrict__ ef, LevelView vf,
                     const SolveState* __restrict__ act)
{
    int kz;
    const int set = set_of(vf.n - 1, kz);
    if (act && !act[set].cont) return;
    const int half = vf.n >> 1;
    const int m = blockIdx.x * kBX + threadIdx.x;
    const int j = blockIdx.y * kBY + threadIdx.y + 1;
    const int k = kz + 1;
    if (m >= half || j >= vf.n) return;
    prolong_node<T, ADD>(ec + (long long)set * 2 * vc.cs, vc, ef + (long long)set * 2 * vf.cs, vf, m, j, k);
}

// Boundary nodes of a level <- the finest boundary values at the same
// positions (u64: finest natural-layout array with nfine intervals), or 0.
__device__ __forceinline__ void face_node(int face, int a, int b, int n, int& i, int& j, int& k)
{
    switch (face) {
    case 0: i = 0; j = a; k = b; break;
    case 1: i = n; j = a; k = b; break;
    case 2: i = a; j = 0; k = b; break;
    case 3: i = a; j = n; k = b; break;
    case 4: i = a; j = b; k = 0; break;
    default: i = a; j = b; k = n; break;
    }
}

template <typename T>
__global__ void set_boundary_kernel(T* __restrict__ e, LevelView v, const double* __restrict__ u64, int nfine)
{
    int face;
    const int set = set_of(6, face);
    e += (long long)set * 2 * v.cs;
    if (u64) u64 += set * nat_elems(nfine);
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (a > v.n) return;
    int i, j, k;
    face_node(face, a, b, v.n, i, j, k);
    T val = T(0);
    if (u64) {
        const int s = nfine / v.n;
        const long long P = nfine + 1;
        val = (T)u64[(long long)i * s + P * ((long long)j * s + P * (long long)k * s)];
    }
    e[node_off(v, i, j, k)] = val;
}

// ---------------------------------------------------------------------------
// Coarse-grid solver: one CTA runs every level with n <= kCoarseN in shared
// memory (natural layout), so the small levels cost one launch instead of
// dozens.  Level l has n_l = 2 << l intervals; `top` is the level it is
// given (its right-hand side f comes from global memory).
//  fmg = 1: full multigrid from 3^3 up to `top` (boundary values injected
//           from u64, or zero), ncycle V-cycles per level;
//  fmg = 0: one V-cycle from a zero initial guess with zero boundary values.
// The result (all nodes, boundary included) is written to e.
// The shared-memory routines below stride over their nodes by the block's
// size: the coarse-grid kernel runs them with kCoarseThreads, the cooperative
// and cluster V-cycle kernels with kVsubThreads.  (1024 threads for the
// coarse-grid kernel measured no faster than 512.)
constexpr int kCoarseThreads = 512;
constexpr int kVsubThreads = 512;
constexpr int kMaxCoarseLevels = 4;  // n = 2, 4, 8, 16

__host__ __device__ inline int cube(int n) { return (n + 1) * (n + 1) * (n + 1); }

template <typename T>
struct CoarseSmem {
    T* u[kMaxCoarseLevels];
    T* f[kMaxCoarseLevels];
    T* r[kMaxCoarseLevels];
};

// Every level size is a compile-time constant (N = 2 << L), so the index
// arithmetic below is shifts and multiplications.  Each routine is run either
// by the whole block (W = false: stride blockDim.x, a multiple of 8, and a
// block barrier at the end) or by warp 0 alone (W = true: the levels n <= 4,
// at most 27 nodes a phase, stride 32 and a warp barrier), which spares the
// smallest levels a block-wide barrier per phase; the arithmetic of every
// node is the same either way.
template <bool W>
__device__ __forceinline__ int sm_stride()
{
    return W ? 32 : (int)blockDim.x;
}

template <bool W>
__device__ __forceinline__ void sm_sync()
{
    if (W)
        __syncwarp();
    else
        __syncthreads();
}

// One colour of the interior of an N-level: row (j, k) holds that colour's
// nodes at i = first, first + 2, ... (first = 1 or 2), N/2 slots per row.
// The stride is a multiple of N/2, so a thread keeps its slot and steps its
// row (j, k) without divisions (the residual and the prolongation below do
// the same with N lanes per row, the last one idle).
template <typename T, int N, bool W = false>
__device__ void sm_relax(T* u, const T* f, T h2, int colour)
{
    constexpr int M = N - 1, P = N + 1, H = N / 2, ROWS = M * M;
    const int dr = sm_stride<W>() / H;  // rows advanced per pass
    const int dj = dr % M, dk = dr / M;
    const int sl = (int)threadIdx.x % H;
    int row = (int)threadIdx.x / H;
    int j = row % M + 1, k = row / M + 1;
    for (; row < ROWS; row += dr) {
        const int i = 1 + (((1 + j + k) & 1) != colour ? 1 : 0) + 2 * sl;
        if (i <= M) {
            const int o = i + P * (j + P * k);
            const T sum = (u[o + 1] + u[o - 1]) + (u[o + P] + u[o - P]) + (u[o + P * P] + u[o - P * P]);
            u[o] = (sum - h2 * f[o]) * (T(1) / T(6));
        }
        j += dj;
        k += dk;
        if (j > M) {
            j -= M;
            ++k;
        }
    }
    sm_sync<W>();
}

template <typename T, int N, bool W = false>
__device__ void sm_residual(const T* u, const T* f, T* r, T ih2)
{
    constexpr int M = N - 1, P = N + 1, ROWS = M * M;
    const int dr = sm_stride<W>() / N;  // rows advanced per pass: a row is N lanes, the last one idle
    const int dj = dr % M, dk = dr / M;
    const int i = (int)threadIdx.x % N + 1;
    int row = (int)threadIdx.x / N;
    int j = row % M + 1, k = row / M + 1;
    for (; row < ROWS; row += dr) {
        if (i <= M) {
            const int o = i + P * (j + P * k);
            const T sum = (u[o + 1] + u[o - 1]) + (u[o + P] + u[o - P]) + (u[o + P * P] + u[o - P * P]);
            r[o] = f[o] - (sum - T(6) * u[o]) * ih2;
        }
        j += dj;
        k += dk;
        if (j > M) {
            j -= M;
            ++k;
        }
    }
    sm_sync<W>();
}

template <typename T, int NF, bool W = false>
__device__ void sm_restrict(const T* fine, T* coarse)
{
    constexpr int NC = NF / 2, MC = NC - 1, PF = NF + 1, PC = NC + 1, TOT = MC * MC * MC;
    for (int t = threadIdx.x; t < TOT; t += sm_stride<W>()) {
        const int I = t % MC + 1, J = (t / MC) % MC + 1, K = t / (MC * MC) + 1;
        T acc = T(0);
#pragma unroll
        for (int c = -1; c <= 1; ++c)
#pragma unroll
            for (int b = -1; b <= 1; ++b)
#pragma unroll
                for (int a = -1; a <= 1; ++a) {
                    const T w = T(0.125) * T(a == 0 ? 2 : 1) * T(b == 0 ? 2 : 1) * T(c == 0 ? 2 : 1) * T(0.125);
                    acc += w * fine[(2 * I + a) + PF * ((2 * J + b) + PF * (2 * K + c))];
                }
        coarse[I + PC * (J + PC * K)] = acc;
    }
    sm_sync<W>();
}

template <typename T, int NC, bool W = false>
__device__ void sm_prolong(const T* coarse, T* fine, bool add)
{
    constexpr int NF = 2 * NC, M = NF - 1, PF = NF + 1, PC = NC + 1, ROWS = M * M;
    const int dr = sm_stride<W>() / NF;  // rows advanced per pass: a row is NF lanes, the last one idle
    const int dj = dr % M, dk = dr / M;
    const int i = (int)threadIdx.x % NF + 1;
    int row = (int)threadIdx.x / NF;
    int j = row % M + 1, k = row / M + 1;
    for (; row < ROWS; row += dr) {
        if (i <= M) {
            const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1, K0 = k >> 1, K1 = (k + 1) >> 1;
            T sum = (coarse[I0 + PC * (J0 + PC * K0)] + coarse[I1 + PC * (J0 + PC * K0)])
                  + (coarse[I0 + PC * (J1 + PC * K0)] + coarse[I1 + PC * (J1 + PC * K0)]);
            sum += (coarse[I0 + PC * (J0 + PC * K1)] + coarse[I1 + PC * (J0 + PC * K1)])
                 + (coarse[I0 + PC * (J1 + PC * K1)] + coarse[I1 + PC * (J1 + PC * K1)]);
            sum *= T(0.125);
            const int o = i + PF * (j + PF * k);
            fine[o] = add ? fine[o] + sum : sum;
        }
        j += dj;
        k += dk;
        if (j > M) {
            j -= M;
            ++k;
        }
    }
    sm_sync<W>();
}

template <typename T, int N, bool W = false>
__device__ void sm_fill(T* a, T val)
{
    constexpr int TOT = (N + 1) * (N + 1) * (N + 1);
    for (int t = threadIdx.x; t < TOT; t += sm_stride<W>()) a[t] = val;
    sm_sync<W>();
}

// The single unknown of the 3^3 grid (Section 2): u = (sum of 6 nbrs - h^2 f)/6.
template <typename T, bool W = false>
__device__ void sm_coarsest(T* u, const T* f, T h)
{
    if (threadIdx.x == 0) {
        const T sum = (u[14] + u[12]) + (u[16] + u[10]) + (u[22] + u[4]);
        u[13] = (sum - h * h * f[13]) * (T(1) / T(6));
    }
    sm_sync<W>();
}

// V(npre, npost) cycle from level L down to the 3^3 grid; the coarser levels
// start from zero (zero boundary values), level L from what u[L] holds.  The
// levels n <= 4 are run by warp 0 while the rest of the block waits.
template <typename T, int L, bool W = false>
__device__ void sm_vcycle(CoarseSmem<T>& S, T h, int npre, int npost)
{
    constexpr int N = 2 << L;
    if constexpr (!W && L <= 1) {
        if (threadIdx.x < 32) sm_vcycle<T, L, true>(S, h, npre, npost);
        __syncthreads();
    } else if constexpr (L == 0) {
        sm_coarsest<T, W>(S.u[0], S.f[0], h);
    } else {
        for (int q = 0; q < npre; ++q) {
            sm_relax<T, N, W>(S.u[L], S.f[L], h * h, 0);
            sm_relax<T, N, W>(S.u[L], S.f[L], h * h, 1);
        }
        sm_residual<T, N, W>(S.u[L], S.f[L], S.r[L], T(1) / (h * h));
        sm_restrict<T, N, W>(S.r[L], S.f[L - 1]);
        sm_fill<T, N / 2, W>(S.u[L - 1], T(0));
        sm_vcycle<T, L - 1, W>(S, h * T(2), npre, npost);
        sm_prolong<T, N / 2, W>(S.u[L - 1], S.u[L], true);
        for (int q = 0; q < npost; ++q) {
            sm_relax<T, N, W>(S.u[L], S.f[L], h * h, 0);
            sm_relax<T, N, W>(S.u[L], S.f[L], h * h, 1);
        }
    }
}

// f restricted from level L down to level 0
template <typename T, int L>
__device__ void sm_restrict_down(CoarseSmem<T>& S)
{
    if constexpr (L > 0) {
        sm_restrict<T, (2 << L)>(S.f[L], S.f[L - 1]);
        sm_restrict_down<T, L - 1>(S);
    }
}

// boundary values of level L (and below): injected from the finest grid (nfine intervals), or zero
template <typename T, int L>
__device__ void sm_inject(CoarseSmem<T>& S, const double* __restrict__ u64, int nfine)
{
    constexpr int N = 2 << L, P = N + 1, TOT = P * P * P;
    const int st = u64 ? nfine / N : 0;
    const long long PF = nfine + 1;
    for (int t = threadIdx.x; t < TOT; t += (int)blockDim.x) {
        const int i = t % P, j = (t / P) % P, k = t / (P * P);
        const bool inner = i > 0 && i < N && j > 0 && j < N && k > 0 && k < N;
        T val = T(0);
        if (!inner && u64) val = (T)u64[(long long)i * st + PF * ((long long)j * st + PF * (long long)k * st)];
        S.u[L][t] = val;
    }
    if constexpr (L > 0) sm_inject<T, L - 1>(S, u64, nfine);
}

// FMG from the 3^3 grid up to level L: prolong, then ncycle V-cycles per level
template <typename T, int L>
__device__ void sm_fmg_up(CoarseSmem<T>& S, T h0, int ncycle, int npre, int npost)
{
    if constexpr (L == 0) {
        sm_coarsest(S.u[0], S.f[0], h0);
    } else {
        sm_fmg_up<T, L - 1>(S, h0, ncycle, npre, npost);
        const T h = h0 / T(1 << L);
        sm_prolong<T, (2 << (L - 1))>(S.u[L - 1], S.u[L], false);
        for (int c = 0; c < ncycle; ++c) sm_vcycle<T, L>(S, h, npre, npost);
    }
}

template <typename T, int TOP>
__device__ void coarse_run(unsigned char* smem_raw, int fmg, T* __restrict__ e, const T* __restrict__ f, LevelView v,
                           T htop, const double* __restrict__ u64, int nfine, int ncycle, int npre, int npost)
{
    T* base = reinterpret_cast<T*>(smem_raw);
    CoarseSmem<T> S;
#pragma unroll
    for (int l = 0; l <= TOP; ++l) {
        const int c = cube(2 << l);
        S.u[l] = base;
        S.f[l] = base + c;
        S.r[l] = base + 2 * c;
        base += 3 * c;
    }
    constexpr int N = 2 << TOP, P = N + 1, TOT = P * P * P;
    // right-hand side of the top level (interior), zero elsewhere
#pragma unroll 5
    for (int t = threadIdx.x; t < TOT; t += (int)blockDim.x) {
        const int i = t % P, j = (t / P) % P, k = t / (P * P);
        const bool inner = i > 0 && i < N && j > 0 && j < N && k > 0 && k < N;
        S.f[TOP][t] = inner ? f[node_off(v, i, j, k)] : T(0);
    }
    if (fmg) {
        __syncthreads();
        sm_restrict_down<T, TOP>(S);
        sm_inject<T, TOP>(S, u64, nfine);
        __syncthreads();
        sm_fmg_up<T, TOP>(S, htop * T(1 << TOP), ncycle, npre, npost);
    } else {
        for (int t = threadIdx.x; t < TOT; t += (int)blockDim.x) S.u[TOP][t] = T(0);
        __syncthreads();
        sm_vcycle<T, TOP>(S, htop, npre, npost);
    }
#pragma unroll 5
    for (int t = threadIdx.x; t < TOT; t += (int)blockDim.x) {
        const int i = t % P, j = (t / P) % P, k = t / (P * P);
        e[node_off(v, i, j, k)] = S.u[TOP][t];
    }
}

template <typename T, int TOP>
__global__ void __launch_bounds__(kCoarseThreads)
coarse_kernel(int fmg, T* __restrict__ e, const T* __restrict__ f, LevelView v, T htop, const double* __restrict__ u64,
              int nfine, int ncycle, int npre, int npost, const SolveState* __restrict__ act)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int set = blockIdx.x;  // one CTA per set
    if (act && !act[set].cont) return;
    const long long so = (long long)set * 2 * v.cs;
    coarse_run<T, TOP>(smem_raw, fmg, e + so, f + so, v, htop, u64 ? u64 + set * nat_elems(nfine) : nullptr, nfine,
                       ncycle, npre, npost);
}

// ---------------------------------------------------------------------------
// The V-cycle below a level, as one cooperative kernel: the levels top .. 1 of
// a.lev (level 0 = the coarse-grid level) are smoothed, restricted and
// corrected phase by phase, every CTA taking a grid-stride share of each
// phase, with a grid barrier between phases; CTA 0 runs the coarse-grid solver
// in shared memory.  Each node's arithmetic is that of the one-launch-per-step
// kernels (rb_node, restrict_node, prolong_node, coarse_run), and nodes within
// a phase are independent, so the result is the same bits.  The barrier
// counter is zeroed before each launch; a barrier that waits too long records
// a fault (reported by the solve as a timeout) and the kernel gives up.
template <typename T>
struct VsubLevel {
    T* e;
    T* f;
    LevelView v;
    T h;
};

constexpr int kVsubMaxLevels = 6;

template <typename T>
struct VsubArgs {
    VsubLevel<T> lev[kVsubMaxLevels];
    int top;        // index of the top level in lev
    int zero_top;   // the top level's correction starts from zero
    int npre, npost;
    unsigned* bar;  // barrier counter (zeroed before the launch)
    int* fault;
    long long polls;  // a barrier gives up after this many polls of the counter
    const SolveState* act;  // cluster form with several sets: skip the sets that have stopped
};

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& gen, int* fault, long long polls)
{
    __syncthreads();
    __shared__ int give_up;
    if (threadIdx.x == 0) {
        give_up = 0;
        gen += gridDim.x;
        __threadfence();
        atomicAdd(bar, 1u);
        long long spins = 0;
        while (*(volatile unsigned*)bar < gen) {
            if (++spins > polls) {
                atomicExch(fault, 4);
                give_up = 1;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return give_up == 0;
}

// Phase work is dealt to `nblk` CTAs, this one being `rank`.
template <typename T>
__device__ void vsub_rb(const VsubLevel<T>& L, int colour, bool zero, int rank, int nblk)
{
    const LevelView& v = L.v;
    const int half = v.n >> 1, rows = v.n - 1;
    const long long W = (long long)half * rows * rows;
    const T h2 = L.h * L.h, sixth = T(1) / T(6);
    T* own = L.e + (long long)colour * v.cs;
    const T* other = L.e + (long long)(colour ^ 1) * v.cs;
    const T* f = L.f + (long long)colour * v.cs;
    for (long long w = rank * (long long)blockDim.x + threadIdx.x; w < W; w += (long long)nblk * blockDim.x) {
        const int m = (int)(w % half);
        const long long r = w / half;
        const int j = (int)(r % rows) + 1, k = (int)(r / rows) + 1;
        if (zero)
            rb_node<T, true>(own, other, f, v, colour, h2, sixth, m, j, k);
        else
            rb_node<T, false>(own, other, f, v, colour, h2, sixth, m, j, k);
    }
}

// The V-cycle on lev[top] .. lev[0] with `nblk` CTAs sharing each phase and
// `sync()` between phases (false: a barrier gave up, stop); CTA rank 0 runs
// the coarse-grid level in its shared memory.
template <typename T, class Sync>
__device__ void vsub_body(const VsubArgs<T>& a, const VsubLevel<T>* lev, int rank, int nblk, unsigned char* smem_raw,
                          Sync&& sync)
{
    bool ok = true;
    // down: smooth, restrict
    for (int l = a.top; l >= 1 && ok; --l) {
        const VsubLevel<T>& L = lev[l];
        for (int q = 0; q < a.npre && ok; ++q) {
            vsub_rb(L, 0, q == 0 && (l < a.top || a.zero_top), rank, nblk);
            ok = sync();
            if (!ok) break;
            vsub_rb(L, 1, false, rank, nblk);
            ok = sync();
        }
        if (!ok) break;
        const VsubLevel<T>& C = lev[l - 1];
        const int mc = C.v.n - 1;
        const long long W = (long long)mc * mc * mc;
        const T ih2 = T(1) / (L.h * L.h);
        for (long long w = rank * (long long)blockDim.x + threadIdx.x; w < W; w += (long long)nblk * blockDim.x) {
            const int I = (int)(w % mc) + 1, J = (int)((w / mc) % mc) + 1, K = (int)(w / ((long long)mc * mc)) + 1;
            restrict_node<T>(L.e, L.f, L.v, C.f, C.v, ih2, I, J, K);
        }
        ok = sync();
    }
    if (!ok) return;
    // the coarse-grid level: one V-cycle from zero in CTA 0's shared memory
    if (rank == 0) {
        const VsubLevel<T>& C = lev[0];
        switch (C.v.n) {
        case 2: coarse_run<T, 0>(smem_raw, 0, C.e, C.f, C.v, C.h, nullptr, 0, 0, a.npre, a.npost); break;
        case 4: coarse_run<T, 1>(smem_raw, 0, C.e, C.f, C.v, C.h, nullptr, 0, 0, a.npre, a.npost); break;
        case 8: coarse_run<T, 2>(smem_raw, 0, C.e, C.f, C.v, C.h, nullptr, 0, 0, a.npre, a.npost); break;
        default: coarse_run<T, 3>(smem_raw, 0, C.e, C.f, C.v, C.h, nullptr, 0, 0, a.npre, a.npost); break;
        }
    }
    ok = sync();
    // up: correct, smooth
    for (int l = 1; l <= a.top && ok; ++l) {
        const VsubLevel<T>& L = lev[l];
        const VsubLevel<T>& C = lev[l - 1];
        const int half = L.v.n >> 1, rows = L.v.n - 1;
        const long long W = (long long)half * rows * rows;
        for (long long w = rank * (long long)blockDim.x + threadIdx.x; w < W; w += (long long)nblk * blockDim.x) {
            const int m = (int)(w % half);
            const long long r = w / half;
            prolong_node<T, true>(C.e, C.v, L.e, L.v, m, (int)(r % rows) + 1, (int)(r / rows) + 1);
        }
        ok = sync();
        for (int q = 0; q < a.npost && ok; ++q) {
            vsub_rb(L, 0, false, rank, nblk);
            ok = sync();
            if (!ok) break;
            vsub_rb(L, 1, false, rank, nblk);
            if (l < a.top || q + 1 < a.npost) ok = sync();
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kVsubThreads) vsub_kernel(VsubArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned gen = 0;
    vsub_body(a, a.lev, (int)blockIdx.x, (int)gridDim.x, smem_raw,
              [&]() { return grid_barrier(a.bar, gen, a.fault, a.polls); });
}

// The same V-cycle as one thread-block cluster per set (csize CTAs; cluster
// s takes set s).  The phases meet at the cluster's hardware barrier with
// release / acquire semantics, so every global write of a phase is visible to
// the whole cluster in the next.  The hardware schedules a cluster's CTAs
// together and every CTA of it passes the same barriers (a set whose
// correction has stopped returns in all of them before the first), so no
// wait is left open.  No grid-wide synchronisation: concurrent solves and
// the sets of a context run side by side.
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename T>
__global__ void __launch_bounds__(kVsubThreads) vcluster_kernel(VsubArgs<T> a, int csize)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int set = (int)blockIdx.x / csize, rank = (int)blockIdx.x - set * csize;
    if (a.act && !a.act[set].cont) return;
    VsubLevel<T> lev[kVsubMaxLevels];
#pragma unroll
    for (int l = 0; l < kVsubMaxLevels; ++l) {
        lev[l] = a.lev[l];
        if (l <= a.top) {
            lev[l].e += (long long)set * 2 * lev[l].v.cs;
            lev[l].f += (long long)set * 2 * lev[l].v.cs;
        }
    }
    vsub_body(a, lev, rank, csize, smem_raw, []() {
        cluster_sync_all();
        return true;
    });
}

// ---------------------------------------------------------------------------
// The V-cycle from the 32-interval level down, in shared memory: one
// thread-block cluster of C CTAs per set.  CTA r keeps the planes
// k0 .. k1-1 of that level's e and f (both colours, each plane's rows laid
// out as in global memory); CTA 0 also keeps the boundary plane 0 and CTA
// C-1 the boundary plane 32.  A node on the first or last plane of a slab
// reads the plane beyond it from the adjacent CTA's shared memory
// (distributed shared memory, through a table of per-plane addresses).
// Phases, separated by the cluster's hardware barrier (release / acquire):
//   npre (red, black) half-sweeps;
//   full weighting of the red residuals, written straight into CTA 0's
//   arrays of the 16-interval level;
//   one V-cycle of the levels 16 .. 2 in CTA 0 (sm_vcycle, as coarse_run);
//   the trilinear correction of the black nodes, read from CTA 0;
//   npost (red, black) half-sweeps;
// then each CTA writes its interior nodes back.  The arithmetic of every
// node is that of the per-step kernels (rb_half4_kernel, restrict_node,
// coarse_run, prolong_node) in the same order, with the same constants, so
// the result is the same bits; the 32-interval level costs one launch and
// no global traffic between its phases.
constexpr int kSlabN = 32;
constexpr int kSlabP = kSlabN + 1;
constexpr int kSlabM = ((kSlabN / 2 + 1) + 3) & ~3;  // row length of the colour-split layout (make_view)
constexpr int kSlabColour = kSlabP * kSlabM;         // floats of one colour of one plane
constexpr int kSlabPlane = 2 * kSlabColour;          // floats of one plane, both colours
constexpr int kSlabThreads = 512;
constexpr int kSlabCoarseP = kSlabN / 2 + 1;  // 17: natural layout of CTA 0's 16-interval arrays

__host__ __device__ inline int slab_depth(int csize) { return (kSlabN - 1 + csize - 1) / csize; }

struct SlabArgs {
    float* e;  // the 32-interval level (set 0; set s at + 2 s cs)
    const float* f;
    long long cs;
    float h2, sixth, ih2;  // that level's h^2, 1/6 and 1/h^2 as the per-step kernels take them
    float hc;              // h of the 16-interval level
    int zero_top, npre, npost, csize;
    const SolveState* act;
};

__device__ __forceinline__ float* cluster_map(float* p, int rank)
{
    unsigned long long out;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(reinterpret_cast<unsigned long long>(p)), "r"(rank));
    return reinterpret_cast<float*>(out);
}

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// One half-sweep of `colour` over the slab's planes (per-node arithmetic of
// rb_half4_kernel: (x pair) + (y pair) + (z pair), then (sum - h2 f) / 6).
template <bool ZERO>
__device__ __forceinline__ void slab_rb(float* const* pe, const float* const* pf, int k0, int k1, int colour,
                                        float h2, float sixth)
{
    const int tot = (k1 - k0) * (kSlabN - 1) * (kSlabN / 2);
    for (int t = threadIdx.x; t < tot; t += kSlabThreads) {
        const int m = t & (kSlabN / 2 - 1);
        const int r = t >> 4;
        const int j = r % (kSlabN - 1) + 1, k = k0 + r / (kSlabN - 1);
        const int p = (colour + j + k) & 1;
        if (p == 0 && m == 0) continue;  // i = 0 is a boundary node
        const int row = j * kSlabM;
        float sum = 0.0f;
        if (!ZERO) {
            const int oc = (colour ^ 1) * kSlabColour + row;
            const float* o = pe[k] + oc;
            const float lo = o[m - 1 + p], hi = o[m + p];
            const float y0 = o[m - kSlabM], y1 = o[m + kSlabM];
            const float z0 = pe[k - 1][oc + m], z1 = pe[k + 1][oc + m];
            sum = (lo + hi) + (y0 + y1) + (z0 + z1);
        }
        const float fv = pf[k][colour * kSlabColour + row + m];
        pe[k][colour * kSlabColour + row + m] = (sum - h2 * fv) * sixth;
    }
}

// red_residual on the slab tables
__device__ __forceinline__ float slab_red_residual(float* const* pe, const float* const* pf, int i, int j, int k,
                                                   float ih2)
{
    const int p = (j + k) & 1;
    const int m = i >> 1;
    const int row = j * kSlabM;
    const float* eb = pe[k] + kSlabColour + row;
    const float s = (eb[m - 1 + p] + eb[m + p]) + (eb[m - kSlabM] + eb[m + kSlabM]) +
                    (pe[k - 1][kSlabColour + row + m] + pe[k + 1][kSlabColour + row + m]);
    return pf[k][row + m] - (s - 6.0f * pe[k][row + m]) * ih2;
}

__global__ void __launch_bounds__(kSlabThreads) vslab_kernel(SlabArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = a.csize;
    const int set = (int)blockIdx.x / C;
    const int rank = (int)cluster_rank();
    if (a.act && !a.act[set].cont) return;  // the whole cluster reads the same flag
    const int q = slab_depth(C);
    const int k0 = 1 + rank * q;
    const int k1 = min(kSlabN, k0 + q);
    float* se = reinterpret_cast<float*>(smem_raw);  // slot s holds plane k0 - 1 + s
    float* sf = se + (size_t)(q + 2) * kSlabPlane;   // slot s holds plane k0 + s
    float** pe = reinterpret_cast<float**>(sf + (size_t)q * kSlabPlane);
    float** pf = pe + 40;
    unsigned char* coarse_raw = reinterpret_cast<unsigned char*>(pf + 40);
    CoarseSmem<float> S;
    {
        float* base = reinterpret_cast<float*>(coarse_raw);
        for (int l = 0; l <= 3; ++l) {
            const int c = cube(2 << l);
            S.u[l] = base;
            S.f[l] = base + c;
            S.r[l] = base + 2 * c;
            base += 3 * c;
        }
    }
    float* const e = a.e + (long long)set * 2 * a.cs;
    const float* const f = a.f + (long long)set * 2 * a.cs;
    constexpr int kC3 = kSlabCoarseP * kSlabCoarseP * kSlabCoarseP;

    // plane tables: plane k of e lives in the CTA that owns it (plane 0 in CTA 0, plane 32 in CTA C-1)
    if (threadIdx.x <= kSlabN) {
        const int k = threadIdx.x;
        const int owner = k == 0 ? 0 : (k == kSlabN ? C - 1 : (k - 1) / q);
        const int slot = k - (1 + owner * q) + 1;
        float* local = se + (size_t)slot * kSlabPlane;
        pe[k] = owner == rank ? local : cluster_map(local, owner);
        if (k >= 1 && k < kSlabN) {
            float* lf = sf + (size_t)(k - (1 + owner * q)) * kSlabPlane;
            pf[k] = owner == rank ? lf : cluster_map(lf, owner);
        }
    }
    // own planes of f (and of e unless the correction starts from zero), and the boundary planes held here
    {
        const int kb = (rank == 0) ? 0 : k0;
        const int ke = (rank == C - 1) ? kSlabN + 1 : k1;
        const int n4 = kSlabColour / 4;  // float4 per colour-plane
        for (int t = threadIdx.x; t < (k1 - k0) * 2 * n4; t += kSlabThreads) {
            const int kk = t / (2 * n4), c = (t / n4) & 1, x = t % n4;
            const float4* src = reinterpret_cast<const float4*>(f + (long long)c * a.cs +
                                                                (long long)(k0 + kk) * kSlabColour);
            reinterpret_cast<float4*>(sf + (size_t)kk * kSlabPlane + c * kSlabColour)[x] = src[x];
        }
        for (int t = threadIdx.x; t < (ke - kb) * 2 * n4; t += kSlabThreads) {
            const int kk = t / (2 * n4), c = (t / n4) & 1, x = t % n4;
            const int k = kb + kk;
            float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (!a.zero_top)
                v = reinterpret_cast<const float4*>(e + (long long)c * a.cs + (long long)k * kSlabColour)[x];
            reinterpret_cast<float4*>(se + (size_t)(k - k0 + 1) * kSlabPlane + c * kSlabColour)[x] = v;
        }
        if (rank == 0)  // coarse_run with a zero start: u = 0, f = 0 off the interior
            for (int t = threadIdx.x; t < kC3; t += kSlabThreads) {
                S.u[3][t] = 0.0f;
                S.f[3][t] = 0.0f;
            }
    }
    __syncthreads();
    cluster_sync_all();

    // pre-smoothing
    for (int qq = 0; qq < a.npre; ++qq) {
        if (qq == 0 && a.zero_top)
            slab_rb<true>(pe, pf, k0, k1, 0, a.h2, a.sixth);
        else
            slab_rb<false>(pe, pf, k0, k1, 0, a.h2, a.sixth);
        cluster_sync_all();
        slab_rb<false>(pe, pf, k0, k1, 1, a.h2, a.sixth);
        cluster_sync_all();
    }
    // restriction of the red residuals onto the coarse planes K with 2K in this slab
    {
        float* fc = rank == 0 ? S.f[3] : cluster_map(S.f[3], 0);
        const int K0 = (k0 + 1) >> 1, K1 = (k1 + 1) >> 1;  // 2K in [k0, k1)
        constexpr int MC = kSlabN / 2 - 1;
        const int tot = (K1 - K0) * MC * MC;
        for (int t = threadIdx.x; t < tot; t += kSlabThreads) {
            const int I = t % MC + 1, J = (t / MC) % MC + 1, K = K0 + t / (MC * MC);
            const int i = 2 * I, j = 2 * J, k = 2 * K;
            const float ih2 = a.ih2;
            float edge = (slab_red_residual(pe, pf, i + 1, j + 1, k, ih2) + slab_red_residual(pe, pf, i - 1, j + 1, k, ih2))
                       + (slab_red_residual(pe, pf, i + 1, j - 1, k, ih2) + slab_red_residual(pe, pf, i - 1, j - 1, k, ih2));
            edge += (slab_red_residual(pe, pf, i + 1, j, k + 1, ih2) + slab_red_residual(pe, pf, i - 1, j, k + 1, ih2))
                  + (slab_red_residual(pe, pf, i + 1, j, k - 1, ih2) + slab_red_residual(pe, pf, i - 1, j, k - 1, ih2));
            edge += (slab_red_residual(pe, pf, i, j + 1, k + 1, ih2) + slab_red_residual(pe, pf, i, j - 1, k + 1, ih2))
                  + (slab_red_residual(pe, pf, i, j + 1, k - 1, ih2) + slab_red_residual(pe, pf, i, j - 1, k - 1, ih2));
            const float centre = slab_red_residual(pe, pf, i, j, k, ih2);
            fc[I + kSlabCoarseP * (J + kSlabCoarseP * K)] = 0.125f * centre + 0.03125f * edge;
        }
    }
    cluster_sync_all();
    if (rank == 0) sm_vcycle<float, 3>(S, a.hc, a.npre, a.npost);
    cluster_sync_all();
    // coarse-grid correction of the black nodes (prolong_node's sums in its order); the coarse planes
    // k0/2 .. k1/2 that this slab interpolates from are first copied from CTA 0 into the same place of
    // this CTA's (otherwise unused) coarse arrays, so that CTA 0's shared memory is read once per value
    {
        if (rank != 0) {
            const float* src = cluster_map(S.u[3], 0);
            const int lo = (k0 >> 1) * kSlabCoarseP * kSlabCoarseP;
            const int hi = ((k1 >> 1) + 1) * kSlabCoarseP * kSlabCoarseP;
            for (int t = lo + threadIdx.x; t < hi; t += 4 * kSlabThreads) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (t + u * kSlabThreads < hi) v[u] = src[t + u * kSlabThreads];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (t + u * kSlabThreads < hi) S.u[3][t + u * kSlabThreads] = v[u];
            }
            __syncthreads();
        }
        const float* ec = S.u[3];
        const int tot = (k1 - k0) * (kSlabN - 1) * (kSlabN / 2);
        for (int t = threadIdx.x; t < tot; t += kSlabThreads) {
            const int m = t & (kSlabN / 2 - 1);
            const int r = t >> 4;
            const int j = r % (kSlabN - 1) + 1, k = k0 + r / (kSlabN - 1);
            const int p = (1 + j + k) & 1;
            const int i = 2 * m + p;
            if (i < 1) continue;
            const int I0 = i >> 1, I1 = (i + 1) >> 1, J0 = j >> 1, J1 = (j + 1) >> 1, K0 = k >> 1, K1 = (k + 1) >> 1;
            constexpr int PC = kSlabCoarseP;
            float s = (ec[I0 + PC * (J0 + PC * K0)] + ec[I1 + PC * (J0 + PC * K0)])
                    + (ec[I0 + PC * (J1 + PC * K0)] + ec[I1 + PC * (J1 + PC * K0)]);
            s += (ec[I0 + PC * (J0 + PC * K1)] + ec[I1 + PC * (J0 + PC * K1)])
               + (ec[I0 + PC * (J1 + PC * K1)] + ec[I1 + PC * (J1 + PC * K1)]);
            s *= 0.125f;
            float* o = pe[k] + kSlabColour + j * kSlabM + m;
            *o = *o + s;
        }
    }
    cluster_sync_all();
    // post-smoothing
    for (int qq = 0; qq < a.npost; ++qq) {
        slab_rb<false>(pe, pf, k0, k1, 0, a.h2, a.sixth);
        cluster_sync_all();
        slab_rb<false>(pe, pf, k0, k1, 1, a.h2, a.sixth);
        cluster_sync_all();  // also: no CTA leaves while a neighbour still reads its planes
    }
    // the interior nodes of this slab back to global memory
    {
        const int tot = (k1 - k0) * 2 * (kSlabN - 1) * (kSlabN / 2);
        for (int t = threadIdx.x; t < tot; t += kSlabThreads) {
            const int m = t & (kSlabN / 2 - 1);
            const int r = t >> 4;
            const int j = r % (kSlabN - 1) + 1;
            const int r2 = r / (kSlabN - 1);
            const int c = r2 & 1, k = k0 + (r2 >> 1);
            const int p = (c + j + k) & 1;
            if (p == 0 && m == 0) continue;
            const int o = c * kSlabColour + j * kSlabM + m;
            e[(long long)c * a.cs + (long long)k * kSlabColour + j * kSlabM + m] = se[(size_t)(k - k0 + 1) * kSlabPlane + o];
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 outer steps on the caller's natural-layout arrays (n intervals).
__device__ __forceinline__ long long nat(int n, int i, int j, int k)
{
    const long long P = n + 1;
    return (long long)i + P * ((long long)j + P * (long long)k);
}

// f = coef rhs on interior nodes, a pair of consecutive nodes (2m, 2m+1) per
// thread: one red and one black entry with the same index m, so the stores of
// a warp are contiguous in each colour array.
template <typename T>
__global__ void convert_rhs_kernel(const double* __restrict__ rhs, double coef, int n, T* __restrict__ f, LevelView v)
{
    int kz;
    const int set = set_of(n - 1, kz);
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y + 1, k = kz + 1;
    if (m >= n / 2) return;
    const double* src = rhs + set * nat_elems(n) + nat(n, 2 * m, j, k);
    T* row = f + set * 2 * v.cs + ((long long)k * (v.n + 1) + j) * v.M + m;
    const int c = (2 * m + j + k) & 1;  // colour of node 2m; node 2m+1 has the other one
    if (m > 0) row[(long long)c * v.cs] = (T)(coef * src[0]);  // node 0 is a boundary node
    row[(long long)(c ^ 1) * v.cs] = (T)(coef * src[1]);
}

template <typename T, bool ADD>
__global__ void assign_outer_kernel(double* __restrict__ u, int n, const T* __restrict__ e, LevelView v,
                                    const SolveState* __restrict__ act)
{
    int kz;
    const int set = set_of(n - 1, kz);
    if (act && !act[set].cont) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y + 1, k = kz + 1;
    if (i >= n) return;
    const long long o = set * nat_elems(n) + nat(n, i, j, k);
    const double d = (double)e[set * 2 * v.cs + node_off(v, i, j, k)];
    u[o] = ADD ? u[o] + d : d;
}

constexpr int kOuterThreads = 128;

// r = coef*rhs - L u in FP64 on interior nodes, stored in precision T; each
// block writes its partial sums of r^2 and (coef*rhs)^2 (fixed-order
// reductions, so the norms are reproducible run to run).
template <typename T>
__global__ void __launch_bounds__(kOuterThreads)
residual_outer_kernel(const double* __restrict__ u, const double* __restrict__ rhs, double coef, int n, double ih2,
                      T* __restrict__ r, LevelView v, double* __restrict__ partials)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y + 1, k = blockIdx.z + 1;
    double rr = 0.0, ff = 0.0;
    if (i < n) {
        const long long P = n + 1, Q = P * P;
        const long long o = nat(n, i, j, k);
        const double s = (u[o + 1] + u[o - 1]) + (u[o + P] + u[o - P]) + (u[o + Q] + u[o - Q]);
        const double fv = coef * rhs[o];
        const double res = fv - (s - 6.0 * u[o]) * ih2;
        r[node_off(v, i, j, k)] = (T)res;
        rr = res * res;
        ff = fv * fv;
    }
    for (int off = 16; off > 0; off >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, off);
        ff += __shfl_down_sync(0xffffffffu, ff, off);
    }
    __shared__ double sr[kOuterThreads / 32], sf[kOuterThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sr[w] = rr;
        sf[w] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kOuterThreads / 32; ++q) {
            a += sr[q];
            b += sf[q];
        }
        const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        partials[2 * bid] = a;
        partials[2 * bid + 1] = b;
    }
}

// The same residual, with rows of the grid dealt to a fixed number of blocks
// (so only a few thousand partial sums need reducing).
constexpr int kResidBlocksPerSM = 16;
constexpr int kResidMaxBlocks = 152 * kResidBlocksPerSM;
constexpr int kRowThreads = 128;

template <typename T>
__global__ void __launch_bounds__(kRowThreads)
residual_rows_kernel(const double* __restrict__ u, const double* __restrict__ rhs, double coef, int n, double ih2,
                     T* __restrict__ r, LevelView v, double* __restrict__ partials, long long pstride,
                     const SolveState* __restrict__ act)
{
    const int set = blockIdx.y;  // one row of blocks per set
    if (act && !act[set].cont) return;
    u += set * nat_elems(n);
    rhs += set * nat_elems(n);
    r += set * 2 * v.cs;
    partials += set * pstride;
    const long long P = n + 1, Q = P * P;
    const int rows = (n - 1) * (n - 1);
    double rr = 0.0, ff = 0.0;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = row % (n - 1) + 1, k = row / (n - 1) + 1;
        for (int i = threadIdx.x + 1; i < n; i += kRowThreads) {
            const long long o = nat(n, i, j, k);
            const double s = (u[o + 1] + u[o - 1]) + (u[o + P] + u[o - P]) + (u[o + Q] + u[o - Q]);
            const double fv = coef * rhs[o];
            const double res = fv - (s - 6.0 * u[o]) * ih2;
            r[node_off(v, i, j, k)] = (T)res;
            rr = fma(res, res, rr);
            ff = fma(fv, fv, ff);
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, off);
        ff += __shfl_down_sync(0xffffffffu, ff, off);
    }
    __shared__ double sr[kRowThreads / 32], sf[kRowThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sr[w] = rr;
        sf[w] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kRowThreads / 32; ++q) {
            a += sr[q];
            b += sf[q];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = b;
    }
}

constexpr int kReduceThreads = 1024;

__global__ void __launch_bounds__(kReduceThreads) reduce_norms_kernel(const double* __restrict__ partials, int nblocks,
                                                                      double* __restrict__ out)
{
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nblocks; t += kReduceThreads) {
        a += partials[2 * t];
        b += partials[2 * t + 1];
    }
    __shared__ double sa[kReduceThreads], sb[kReduceThreads];
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int s = kReduceThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sa[0];
        out[1] = sb[0];
    }
}

// Sums the partial norms in a fixed order and decides whether the defect
// correction goes on: continue = refine && rel > tol && it < max_it && rel
// finite.  first: this is the residual after FMG (sets the denominator
// ||coef*rhs||, or 1 when it is 0, and it = 0).  Inside a graph the decision
// drives the WHILE node through `handle`.
//
// Several sets (fault == NULL): block s decides for set s; a set whose
// correction has already stopped keeps its state; decide_any_kernel then
// takes over the fault flag and drives the WHILE node.
template <bool GRAPH>
__global__ void __launch_bounds__(kReduceThreads)
decide_kernel(const double* __restrict__ partials, int nblocks, SolveState* __restrict__ st, double tol, int max_it,
              int first, int refine, cudaGraphConditionalHandle handle, int* __restrict__ fault, long long pstride)
{
    const int set = blockIdx.x;
    partials += set * pstride;
    st += set;
    if (!fault && !first && st->cont == 0) return;
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nblocks; t += kReduceThreads) {
        a += partials[2 * t];
        b += partials[2 * t + 1];
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __shared__ double sa[kReduceThreads / 32], sb[kReduceThreads / 32];
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        a = sa[threadIdx.x];
        b = sb[threadIdx.x];
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, off);
            b += __shfl_down_sync(0xffffffffu, b, off);
        }
        if (threadIdx.x == 0) {
            sa[0] = a;
            sb[0] = b;
        }
    }
    if (threadIdx.x == 0) {
        if (first) {
            st->denom = sb[0] > 0.0 ? sqrt(sb[0]) : 1.0;
            st->it = 0;
        } else {
            st->it += 1;
        }
        const double rel = sqrt(sa[0]) / st->denom;
        if (first) st->rel0 = rel;
        st->rel = rel;
        const bool finite = isfinite(rel) && !st->nonfinite;
        const int faulted = (fault && *fault) ? 1 : 0;
        if (first) st->fault = 0;
        if (faulted) {
            st->fault = 1;
            *fault = 0;
        }
        st->converged = (finite && !st->fault && (!refine || rel <= tol)) ? 1 : 0;
        const int cont = (refine && finite && !st->fault && rel > tol && st->it < max_it) ? 1 : 0;
        st->cont = cont;
        if (GRAPH && fault) cudaGraphSetConditional(handle, (unsigned)cont);
    }
}

// After the per-set decisions: a fault recorded since the last check stops
// every set; the loop goes on while any set goes on.
template <bool GRAPH>
__global__ void decide_any_kernel(SolveState* __restrict__ st, int nsets, int first, cudaGraphConditionalHandle handle,
                                  int* __restrict__ fault)
{
    if (threadIdx.x != 0) return;
    const int faulted = *fault;
    if (faulted) *fault = 0;
    unsigned any = 0;
    for (int q = 0; q < nsets; ++q) {
        if (faulted) {
            st[q].fault = 1;
            st[q].converged = 0;
            st[q].cont = 0;
        }
        any |= (unsigned)st[q].cont;
    }
    if (GRAPH) cudaGraphSetConditional(handle, any);
}

inline dim3 half_grid(int n) { return dim3(cdiv(n / 2, kBX), cdiv(n - 1, kBY), (unsigned)(n - 1)); }
inline dim3 inner_grid(int n) { return dim3(cdiv(n - 1, kBX), cdiv(n - 1, kBY), (unsigned)(n - 1)); }
inline dim3 outer_grid(int n) { return dim3(cdiv(n - 1, kOuterThreads), (unsigned)(n - 1), (unsigned)(n - 1)); }

template <typename T>
size_t coarse_smem_bytes(int n)
{
    size_t tot = 0;
    for (int m = 2; m <= n; m *= 2) tot += 3 * (size_t)cube(m);
    return tot * sizeof(T);
}

// shared memory of the slab V-cycle kernel: e planes (slab + 2), f planes
// (slab), the two plane tables, and CTA 0's arrays of the levels 16 .. 2
inline size_t slab_smem_bytes(int csize)
{
    const int q = slab_depth(csize);
    return sizeof(float) * (size_t)kSlabPlane * (size_t)(2 * q + 2) + 2 * 40 * sizeof(float*) +
           coarse_smem_bytes<float>(kSlabN / 2);
}

}  // namespace

// --- launchers ------------------------------------------------------------
// With several sets every grid's z extent (or, for the per-set kernels, its x
// or y extent) is multiplied by the number of sets; the qumond_create checks
// keep the products within the launch limits.
inline dim3 per_sets(dim3 g, const Sets& sets) { return dim3(g.x, g.y, g.z * (unsigned)sets.n); }

// threads along a row of the row-vector kernels on a level of n intervals
inline int vx_of(int n, const Sets& sets)
{
    if (n > kTileSmallN) return kVX;
    return sets.tile_small == 1 ? 4 : (sets.tile_small == 2 ? 2 : kVX);
}

template <typename T>
void launch_rb_half(T* e, const T* f, const LevelView& v, int colour, bool zero_guess, double h, cudaStream_t s,
                    const Sets& sets)
{
    T* own = e + (long long)colour * v.cs;
    const T* other = e + (long long)(colour ^ 1) * v.cs;
    const T* fc = f + (long long)colour * v.cs;
    const dim3 blk(kBX, kBY);
    if (sizeof(T) == sizeof(float) && v.n >= 8) {
        float* o4 = reinterpret_cast<float*>(own);
        const float* x4 = reinterpret_cast<const float*>(other);
        const float* f4 = reinterpret_cast<const float*>(fc);
        const int vx = vx_of(v.n, sets);
        const dim3 grid(cdiv(v.n / 2, 4 * vx), cdiv(v.n - 1, kVThreads / vx), (unsigned)(v.n - 1) * (unsigned)sets.n);
        const dim3 blk(vx, kVThreads / vx);
        const float h2 = (float)(h * h), sixth = 1.0f / 6.0f;
        switch ((zero_guess ? 8 : 0) + vx) {
        case 8 + 8: rb_half4_kernel<true, 8><<<grid, blk, 0, s>>>(o4, x4, f4, v, colour, h2, sixth, sets.act); break;
        case 8 + 4: rb_half4_kernel<true, 4><<<grid, blk, 0, s>>>(o4, x4, f4, v, colour, h2, sixth, sets.act); break;
        case 8 + 2: rb_half4_kernel<true, 2><<<grid, blk, 0, s>>>(o4, x4, f4, v, colour, h2, sixth, sets.act); break;
        case 8: rb_half4_kernel<false, 8><<<grid, blk, 0, s>>>(o4, x4, f4, v, colour, h2, sixth, sets.act); break;
        case 4: rb_half4_kernel<false, 4><<<grid, blk, 0, s>>>(o4, x4, f4, v, colour, h2, sixth, sets.act); break;
        default: rb_half4_kernel<false, 2><<<grid, blk, 0, s>>>(o4, x4, f4, v, colour, h2, sixth, sets.act); break;
        }
        return;
    }
    if (zero_guess)
        rb_half_kernel<T, true><<<per_sets(half_grid(v.n), sets), blk, 0, s>>>(own, other, fc, v, colour, (T)(h * h),
                                                                                T(1) / T(6), sets.act);
    else
        rb_half_kernel<T, false><<<per_sets(half_grid(v.n), sets), blk, 0, s>>>(own, other, fc, v, colour, (T)(h * h),
                                                                                 T(1) / T(6), sets.act);
}

void launch_rb_first(float* e, const float* f, const LevelView& v, double h, cudaStream_t s, const Sets& sets)
{
    const int vx = vx_of(v.n, sets);
    const dim3 grid(cdiv(v.n / 2, 4 * vx), cdiv(v.n - 1, kVThreads / vx), (unsigned)(v.n - 1) * (unsigned)sets.n);
    const dim3 blk(vx, kVThreads / vx);
    const float h2 = (float)(h * h), sixth = 1.0f / 6.0f;
    switch (vx) {
    case 8: rb_first4_kernel<8><<<grid, blk, 0, s>>>(e, f, v, h2, sixth, sets.act); break;
    case 4: rb_first4_kernel<4><<<grid, blk, 0, s>>>(e, f, v, h2, sixth, sets.act); break;
    default: rb_first4_kernel<2><<<grid, blk, 0, s>>>(e, f, v, h2, sixth, sets.act); break;
    }
}

template <typename T>
void launch_restrict_resid_red(const T* ef, const T* ff, const LevelView& vf, T* fc, const LevelView& vc, double hf,
                               cudaStream_t s, const Sets& sets)
{
    if (sizeof(T) == sizeof(float) && vf.n >= 128) {
        // planes per CTA: as many as keep about two CTAs per multiprocessor busy
        static int sms = 0;
        if (sms <= 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
        }
        const int tiles = (int)(cdiv(vc.n - 1, kRI) * cdiv(vc.n - 1, kRJ)) * sets.n;
        int rk = kRK;
        while (rk > 1 && tiles * (int)cdiv(vc.n - 1, rk) < 2 * sms) --rk;
        const int zper = (int)cdiv(vc.n - 1, rk);
        const dim3 grid(cdiv(vc.n - 1, kRI), cdiv(vc.n - 1, kRJ), (unsigned)(zper * sets.n));
        restrict_resid4_kernel<<<grid, kRI * kRJ, 0, s>>>(reinterpret_cast<const float*>(ef),
                                                           reinterpret_cast<const float*>(ff), vf,
                                                           reinterpret_cast<float*>(fc), vc, (float)(1.0 / (hf * hf)),
                                                           rk, zper, sets.act);
        return;
    }
    restrict_resid_red_kernel<T><<<per_sets(inner_grid(vc.n), sets), dim3(kBX, kBY), 0, s>>>(
        ef, ff, vf, fc, vc, (T)(1.0 / (hf * hf)), sets.act);
}

template <typename T>
void launch_restrict_full(const T* ff, const LevelView& vf, T* fc, const LevelView& vc, cudaStream_t s,
                          const Sets& sets)
{
    restrict_full_kernel<T><<<per_sets(inner_grid(vc.n), sets), dim3(kBX, kBY), 0, s>>>(ff, vf, fc, vc);
}

template <typename T>
void launch_prolong_black(const T* ec, const LevelView& vc, T* ef, const LevelView& vf, bool add, cudaStream_t s,
                          const Sets& sets)
{
    if (sizeof(T) == sizeof(float) && vf.n >= 8) {
        const float* c4 = reinterpret_cast<const float*>(ec);
        float* f4 = reinterpret_cast<float*>(ef);
        const int vx = vx_of(vf.n, sets);
        const dim3 grid(cdiv(vf.n / 2, 4 * vx), cdiv(vf.n - 1, kVThreads / vx), (unsigned)(vf.n - 1) * (unsigned)sets.n);
        const dim3 blk(vx, kVThreads / vx);
        switch ((add ? 8 : 0) + vx) {
        case 8 + 8: prolong_black4_kernel<true, 8><<<grid, blk, 0, s>>>(c4, vc, f4, vf, sets.act); break;
        case 8 + 4: prolong_black4_kernel<true, 4><<<grid, blk, 0, s>>>(c4, vc, f4, vf, sets.act); break;
        case 8 + 2: prolong_black4_kernel<true, 2><<<grid, blk, 0, s>>>(c4, vc, f4, vf, sets.act); break;
        case 8: prolong_black4_kernel<false, 8><<<grid, blk, 0, s>>>(c4, vc, f4, vf, sets.act); break;
        case 4: prolong_black4_kernel<false, 4><<<grid, blk, 0, s>>>(c4, vc, f4, vf, sets.act); break;
        default: prolong_black4_kernel<false, 2><<<grid, blk, 0, s>>>(c4, vc, f4, vf, sets.act); break;
        }
        return;
    }
    if (add)
        prolong_black_kernel<T, true><<<per_sets(half_grid(vf.n), sets), dim3(kBX, kBY), 0, s>>>(ec, vc, ef, vf,
                                                                                                  sets.act);
    else
        prolong_black_kernel<T, false><<<per_sets(half_grid(vf.n), sets), dim3(kBX, kBY), 0, s>>>(ec, vc, ef, vf,
                                                                                                   sets.act);
}

template <typename T>
void launch_set_boundary(T* e, const LevelView& v, const double* u64, int nfine, cudaStream_t s, const Sets& sets)
{
    set_boundary_kernel<T><<<dim3(cdiv(v.n + 1, 128), (unsigned)(v.n + 1), 6 * (unsigned)sets.n), 128, 0, s>>>(
        e, v, u64, nfine);
}

template <typename T>
cudaError_t launch_coarse(int fmg, T* e, const T* f, const LevelView& v, double h, const double* u64, int nfine,
                          int ncycle, int npre, int npost, cudaStream_t s, const Sets& sets)
{
    const size_t bytes = coarse_smem_bytes<T>(v.n);
    const unsigned g = (unsigned)sets.n;  // one CTA per set
    const SolveState* act = sets.act;
    switch (v.n) {
    case 2: coarse_kernel<T, 0><<<g, kCoarseThreads, bytes, s>>>(fmg, e, f, v, (T)h, u64, nfine, ncycle, npre, npost, act); break;
    case 4: coarse_kernel<T, 1><<<g, kCoarseThreads, bytes, s>>>(fmg, e, f, v, (T)h, u64, nfine, ncycle, npre, npost, act); break;
    case 8: coarse_kernel<T, 2><<<g, kCoarseThreads, bytes, s>>>(fmg, e, f, v, (T)h, u64, nfine, ncycle, npre, npost, act); break;
    case 16: coarse_kernel<T, 3><<<g, kCoarseThreads, bytes, s>>>(fmg, e, f, v, (T)h, u64, nfine, ncycle, npre, npost, act); break;
    default: return cudaErrorInvalidValue;  // the coarse solver covers the levels n = 2 .. 16
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_vsub(T* const* e, T* const* f, const LevelView* v, const double* h, int nlev, int zero_top, int npre,
                        int npost, unsigned* bar, int* fault, long long polls, int grid, cudaStream_t s)
{
    if (nlev < 2 || nlev > kVsubMaxLevels || v[0].n > kCoarseN) return cudaErrorInvalidValue;
    VsubArgs<T> a{};
    for (int l = 0; l < nlev; ++l) a.lev[l] = VsubLevel<T>{e[l], f[l], v[l], (T)h[l]};
    a.top = nlev - 1;
    a.zero_top = zero_top;
    a.npre = npre;
    a.npost = npost;
    a.bar = bar;
    a.fault = fault;
    a.polls = polls;
    cudaError_t err = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kVsubThreads);
    cfg.dynamicSmemBytes = coarse_smem_bytes<T>(v[0].n);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, vsub_kernel<T>, a);
}

template <typename T>
cudaError_t launch_vcluster(T* const* e, T* const* f, const LevelView* v, const double* h, int nlev, int zero_top,
                            int npre, int npost, int csize, cudaStream_t s, const Sets& sets)
{
    if (nlev < 2 || nlev > kVsubMaxLevels || v[0].n > kCoarseN || csize < 1) return cudaErrorInvalidValue;
    VsubArgs<T> a{};
    for (int l = 0; l < nlev; ++l) a.lev[l] = VsubLevel<T>{e[l], f[l], v[l], (T)h[l]};
    a.top = nlev - 1;
    a.zero_top = zero_top;
    a.npre = npre;
    a.npost = npost;
    a.act = sets.act;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(csize * sets.n));
    cfg.blockDim = dim3(kVsubThreads);
    cfg.dynamicSmemBytes = coarse_smem_bytes<T>(v[0].n);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, vcluster_kernel<T>, a, csize);
}

int vcluster_size(bool fp64)
{
    // the largest cluster (16 needs the non-portable size) of which at least one fits on the device
    for (int cs = 16; cs >= 2; cs /= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)cs);
        cfg.blockDim = dim3(kVsubThreads);
        cfg.dynamicSmemBytes = fp64 ? coarse_smem_bytes<double>(kCoarseN) : coarse_smem_bytes<float>(kCoarseN);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        const cudaError_t e = fp64 ? cudaOccupancyMaxActiveClusters(&n, vcluster_kernel<double>, &cfg)
                                   : cudaOccupancyMaxActiveClusters(&n, vcluster_kernel<float>, &cfg);
        if (e == cudaSuccess && n >= 1) return cs;
        (void)cudaGetLastError();
    }
    return 0;
}

cudaError_t launch_vslab(float* e, const float* f, const LevelView& v, double h, double hc, int zero_top, int npre,
                         int npost, int csize, cudaStream_t s, const Sets& sets)
{
    if (v.n != kSlabN || v.M != kSlabM || (v.cs & 3) != 0 || (reinterpret_cast<uintptr_t>(e) & 15) != 0 ||
        (reinterpret_cast<uintptr_t>(f) & 15) != 0 || !(csize == 4 || csize == 8 || csize == 16))
        return cudaErrorInvalidValue;
    SlabArgs a{};
    a.e = e;
    a.f = f;
    a.cs = v.cs;
    a.h2 = (float)(h * h);
    a.sixth = 1.0f / 6.0f;
    a.ih2 = (float)(1.0 / (h * h));
    a.hc = (float)hc;
    a.zero_top = zero_top;
    a.npre = npre;
    a.npost = npost;
    a.csize = csize;
    a.act = sets.act;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(csize * sets.n));
    cfg.blockDim = dim3(kSlabThreads);
    cfg.dynamicSmemBytes = slab_smem_bytes(csize);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)csize;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, vslab_kernel, a);
}

int vslab_size(int want)
{
    // `want` CTAs per cluster (4, 8 or 16) if at least one such cluster fits on the device, else 0
    if (!(want == 4 || want == 8 || want == 16)) return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)want);
    cfg.blockDim = dim3(kSlabThreads);
    cfg.dynamicSmemBytes = slab_smem_bytes(want);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)want;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, vslab_kernel, &cfg) == cudaSuccess && n >= 1) return want;
    (void)cudaGetLastError();
    return 0;
}

int vsub_grid(int sms)
{
    // one CTA per SM: the kernel's shared memory (the coarse solver's) allows one or more per SM
    return sms;
}

template <typename T>
void launch_convert_rhs(const double* rhs, double coef, int n, T* f, const LevelView& v, cudaStream_t s,
                        const Sets& sets)
{
    const dim3 g(cdiv(n / 2, kOuterThreads), (unsigned)(n - 1), (unsigned)(n - 1));
    convert_rhs_kernel<T><<<per_sets(g, sets), kOuterThreads, 0, s>>>(rhs, coef, n, f, v);
}

template <typename T>
void launch_assign_outer(double* u, int n, const T* e, const LevelView& v, bool add, cudaStream_t s, const Sets& sets)
{
    if (add)
        assign_outer_kernel<T, true><<<per_sets(outer_grid(n), sets), kOuterThreads, 0, s>>>(u, n, e, v, sets.act);
    else
        assign_outer_kernel<T, false><<<per_sets(outer_grid(n), sets), kOuterThreads, 0, s>>>(u, n, e, v, sets.act);
}

int residual_outer_blocks(int n)
{
    const dim3 g = outer_grid(n);
    return (int)(g.x * g.y * g.z);
}

template <typename T>
int launch_residual_outer(const double* u, const double* rhs, double coef, int n, double h, T* r, const LevelView& v,
                          double* partials, cudaStream_t s)
{
    residual_outer_kernel<T><<<outer_grid(n), kOuterThreads, 0, s>>>(u, rhs, coef, n, 1.0 / (h * h), r, v, partials);
    return residual_outer_blocks(n);
}

int residual_rows_blocks(int n)
{
    const int rows = (n - 1) * (n - 1);
    return rows < kResidMaxBlocks ? rows : kResidMaxBlocks;
}

template <typename T>
int launch_residual_rows(const double* u, const double* rhs, double coef, int n, double h, T* r, const LevelView& v,
                         double* partials, cudaStream_t s, const Sets& sets)
{
    const int nb = residual_rows_blocks(n);
    residual_rows_kernel<T><<<dim3(nb, sets.n), kRowThreads, 0, s>>>(u, rhs, coef, n, 1.0 / (h * h), r, v, partials,
                                                                     sets.pstride, sets.act);
    return nb;
}

void launch_decide(const double* partials, int nblocks, SolveState* st, double tol, int max_it, bool first,
                   bool refine, const cudaGraphConditionalHandle* handle, int* fault, cudaStream_t s, const Sets& sets)
{
    if (sets.n == 1) {
        if (handle)
            decide_kernel<true><<<1, kReduceThreads, 0, s>>>(partials, nblocks, st, tol, max_it, first, refine,
                                                             *handle, fault, 0);
        else
            decide_kernel<false><<<1, kReduceThreads, 0, s>>>(partials, nblocks, st, tol, max_it, first, refine, 0,
                                                              fault, 0);
        return;
    }
    decide_kernel<false><<<sets.n, kReduceThreads, 0, s>>>(partials, nblocks, st, tol, max_it, first, refine, 0,
                                                           nullptr, sets.pstride);
    if (handle)
        decide_any_kernel<true><<<1, 32, 0, s>>>(st, sets.n, first, *handle, fault);
    else
        decide_any_kernel<false><<<1, 32, 0, s>>>(st, sets.n, first, 0, fault);
}

cudaError_t prepare_kernels()
{
    if (cudaFuncSetAttribute(vsub_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)coarse_smem_bytes<float>(kCoarseN)) != cudaSuccess ||
        cudaFuncSetAttribute(vsub_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)coarse_smem_bytes<double>(kCoarseN)) != cudaSuccess ||
        cudaFuncSetAttribute(vcluster_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)coarse_smem_bytes<float>(kCoarseN)) != cudaSuccess ||
        cudaFuncSetAttribute(vcluster_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)coarse_smem_bytes<double>(kCoarseN)) != cudaSuccess ||
        cudaFuncSetAttribute(vcluster_kernel<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess ||
        cudaFuncSetAttribute(vcluster_kernel<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
        return cudaGetLastError();
    if (cudaFuncSetAttribute(vslab_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)slab_smem_bytes(4)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(vslab_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return cudaGetLastError();
    cudaError_t e = cudaFuncSetAttribute(coarse_kernel<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)coarse_smem_bytes<float>(kCoarseN));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(coarse_kernel<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)coarse_smem_bytes<double>(kCoarseN));
}

void launch_reduce_norms(const double* partials, int nblocks, double* out, cudaStream_t s)
{
    reduce_norms_kernel<<<1, kReduceThreads, 0, s>>>(partials, nblocks, out);
}

#define QUMOND_INSTANTIATE(T)                                                                                          \
    template void launch_rb_half<T>(T*, const T*, const LevelView&, int, bool, double, cudaStream_t, const Sets&);    \
    template void launch_restrict_resid_red<T>(const T*, const T*, const LevelView&, T*, const LevelView&, double,    \
                                               cudaStream_t, const Sets&);                                             \
    template void launch_restrict_full<T>(const T*, const LevelView&, T*, const LevelView&, cudaStream_t,             \
                                          const Sets&);                                                                \
    template void launch_prolong_black<T>(const T*, const LevelView&, T*, const LevelView&, bool, cudaStream_t,       \
                                          const Sets&);                                                                \
    template void launch_set_boundary<T>(T*, const LevelView&, const double*, int, cudaStream_t, const Sets&);        \
    template cudaError_t launch_vsub<T>(T* const*, T* const*, const LevelView*, const double*, int, int, int, int,     \
                                        unsigned*, int*, long long, int, cudaStream_t);                               \
    template cudaError_t launch_vcluster<T>(T* const*, T* const*, const LevelView*, const double*, int, int, int, int, \
                                            int, cudaStream_t, const Sets&);                                           \
    template cudaError_t launch_coarse<T>(int, T*, const T*, const LevelView&, double, const double*, int, int, int,  \
                                          int, cudaStream_t, const Sets&);                                             \
    template void launch_convert_rhs<T>(const double*, double, int, T*, const LevelView&, cudaStream_t, const Sets&); \
    template void launch_assign_outer<T>(double*, int, const T*, const LevelView&, bool, cudaStream_t, const Sets&);  \
    template int launch_residual_outer<T>(const double*, const double*, double, int, double, T*, const LevelView&,    \
                                          double*, cudaStream_t);                                                      \
    template int launch_residual_rows<T>(const double*, const double*, double, int, double, T*, const LevelView&,     \
                                         double*, cudaStream_t, const Sets&);

QUMOND_INSTANTIATE(float)
QUMOND_INSTANTIATE(double)

}  // namespace qumond
