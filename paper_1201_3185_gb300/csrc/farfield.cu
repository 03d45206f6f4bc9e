// Far-field boundary values of the outermost box (QUMOND_BC_MULTIPOLE).
//
// Section 2 sets Phi = 0 on a box 2^10 times larger than the galaxy and
// refines inwards.  With a few boxes the outermost boundary lies close to the
// mass, so its values come from the mass inside the box instead:
//  * Phi_N: the exterior multipole expansion, to degree kFFL = 8, of the node
//    masses m_k = rho_k h^3 about their centre of mass c:
//      Phi_N(x) = -G sum_{l<=8} sum_{m<=l} w_lm [Re T_lm(d) A_lm + Im T_lm(d) B_lm] / |d|^(2l+1),
//    d = x - c, T_lm(d) = |d|^l P_l^m(cos theta) e^{i m phi} (the solid harmonics, polynomials in
//    d), A_lm + i B_lm = sum_k m_k T_lm(x_k - c), w_lm = (2 - [m = 0]) (l-m)!/(l+m)!  -- the
//    Legendre series of -G sum_k m_k / |x - x_k| regrouped by the addition theorem;
//  * Phi: the QUMOND potential of the total mass M as a point at c,
//      F(r) = -A/(2r) + (1/2) [-sqrt(A^2 + C r^2)/r + sqrt(C) asinh(sqrt(C) r / A)],
//    A = G M, C = 4 a0 A, whose gradient is nu(G M/(a0 r^2)) G M / r^2 (Eq. 2 for a sphere).
// T_lm: T_mm = (2m-1)!! (dx + i dy)^m, T_{m+1,m} = (2m+1) dz T_mm,
// (l-m) T_lm = (2l-1) dz T_{l-1,m} - (l+m-1) |d|^2 T_{l-2,m} (P_l^m without the (-1)^m phase,
// which cancels in the products).
//
// All in FP64; the sums over nodes are per-block partial sums added in a
// fixed order, so the values are the same on every run.  Every grid of a
// context with several sets is handled in the same launches (blockIdx.y or the
// face index carries the set).
#include "qumond_internal.h"

namespace qumond {

namespace {

constexpr int kFFL = 8;
constexpr int kFFTerms = (kFFL + 1) * (kFFL + 2) / 2;  // (l, m), 0 <= m <= l <= 8: 45
constexpr int kFFThreads = 128;
constexpr int kFFBlocks = 2 * 152;  // blocks per set of the two reductions over nodes

__host__ __device__ constexpr int term(int l, int m) { return l * (l + 1) / 2 + m; }

// T_lm(d) for l <= 8 into re[term(l, m)], im[term(l, m)]
__device__ __forceinline__ void solid(double dx, double dy, double dz, double* re, double* im)
{
    const double r2 = dx * dx + dy * dy + dz * dz;
    double pr = 1.0, pi = 0.0, df = 1.0;  // (dx + i dy)^m, (2m-1)!!
#pragma unroll
    for (int m = 0; m <= kFFL; ++m) {
        if (m > 0) {
            const double a = pr * dx - pi * dy, b = pr * dy + pi * dx;
            pr = a;
            pi = b;
            df *= (double)(2 * m - 1);
        }
        re[term(m, m)] = df * pr;
        im[term(m, m)] = df * pi;
        if (m + 1 <= kFFL) {
            re[term(m + 1, m)] = (double)(2 * m + 1) * dz * re[term(m, m)];
            im[term(m + 1, m)] = (double)(2 * m + 1) * dz * im[term(m, m)];
        }
#pragma unroll
        for (int l = m + 2; l <= kFFL; ++l) {
            const double inv = 1.0 / (double)(l - m);
            re[term(l, m)] = ((double)(2 * l - 1) * dz * re[term(l - 1, m)] - (double)(l + m - 1) * r2 * re[term(l - 2, m)]) * inv;
            im[term(l, m)] = ((double)(2 * l - 1) * dz * im[term(l - 1, m)] - (double)(l + m - 1) * r2 * im[term(l - 2, m)]) * inv;
        }
    }
}

// Sum of v over the block in a fixed order (warp trees, then the warps in order); valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kFFThreads / 32; ++w) s += sh[w];
    return s;
}

struct Geo {
    int n;
    double x0, y0, z0, h, h3;
};

__device__ __forceinline__ void node_pos(const Geo& g, long long t, double& x, double& y, double& z)
{
    const long long P = g.n + 1;
    const int i = (int)(t % P), j = (int)((t / P) % P), k = (int)(t / (P * P));
    x = g.x0 + i * g.h;
    y = g.y0 + j * g.h;
    z = g.z0 + k * g.h;
}

// The node loops stream the whole density once per kernel with few threads
// (the reductions keep one partial per block), so each thread loads kFFILP
// values before using any: enough bytes in flight to approach the memory
// bandwidth.  Nodes are visited in the same order for any unrolling.
constexpr int kFFILP = 8;

// per-block sums of m, m x, m y, m z
__global__ void __launch_bounds__(kFFThreads) ff_mass_kernel(const double* __restrict__ rho, Geo g,
                                                              double* __restrict__ part)
{
    __shared__ double sh[kFFThreads / 32];
    const int set = blockIdx.y;
    const long long N = nat_elems(g.n);
    rho += set * N;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * kFFThreads;
    for (long long t0 = blockIdx.x * (long long)kFFThreads + threadIdx.x; t0 < N; t0 += kFFILP * stride) {
        double r[kFFILP];
#pragma unroll
        for (int q = 0; q < kFFILP; ++q) r[q] = t0 + q * stride < N ? rho[t0 + q * stride] : 0.0;
#pragma unroll
        for (int q = 0; q < kFFILP; ++q) {
            const double m = r[q] * g.h3;
            if (m == 0.0) continue;
            double x, y, z;
            node_pos(g, t0 + q * stride, x, y, z);
            a[0] += m;
            a[1] += m * x;
            a[2] += m * y;
            a[3] += m * z;
        }
    }
    double* out = part + ((long long)set * gridDim.x + blockIdx.x) * 4;
    for (int q = 0; q < 4; ++q) {
        const double s = block_sum(a[q], sh);
        if (threadIdx.x == 0) out[q] = s;
    }
}

// M and the centre of mass of each set: the block sums added in block order
__global__ void ff_com_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ com)
{
    const int set = blockIdx.x;
    if (threadIdx.x != 0) return;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nblocks; ++b)
        for (int q = 0; q < 4; ++q) a[q] += part[((long long)set * nblocks + b) * 4 + q];
    double* c = com + 4 * set;
    c[0] = a[0];
    c[1] = a[0] != 0.0 ? a[1] / a[0] : 0.0;
    c[2] = a[0] != 0.0 ? a[2] / a[0] : 0.0;
    c[3] = a[0] != 0.0 ? a[3] / a[0] : 0.0;
}

// per-block sums of m T_lm(x - c)
__global__ void __launch_bounds__(kFFThreads) ff_moments_kernel(const double* __restrict__ rho, Geo g,
                                                                 const double* __restrict__ com,
                                                                 double* __restrict__ part)
{
    __shared__ double sh[kFFThreads / 32];
    const int set = blockIdx.y;
    const long long N = nat_elems(g.n);
    rho += set * N;
    const double cx = com[4 * set + 1], cy = com[4 * set + 2], cz = com[4 * set + 3];
    double A[kFFTerms], B[kFFTerms];
#pragma unroll
    for (int q = 0; q < kFFTerms; ++q) A[q] = B[q] = 0.0;
    const long long stride = (long long)gridDim.x * kFFThreads;
    for (long long t0 = blockIdx.x * (long long)kFFThreads + threadIdx.x; t0 < N; t0 += kFFILP * stride) {
        double r[kFFILP];
#pragma unroll
        for (int q = 0; q < kFFILP; ++q) r[q] = t0 + q * stride < N ? rho[t0 + q * stride] : 0.0;
#pragma unroll 1
        for (int q = 0; q < kFFILP; ++q) {
            const double m = r[q] * g.h3;
            if (m == 0.0) continue;
            double x, y, z;
            node_pos(g, t0 + q * stride, x, y, z);
            double re[kFFTerms], im[kFFTerms];
            solid(x - cx, y - cy, z - cz, re, im);
#pragma unroll
            for (int p = 0; p < kFFTerms; ++p) {
                A[p] += m * re[p];
                B[p] += m * im[p];
            }
        }
    }
    double* out = part + ((long long)set * gridDim.x + blockIdx.x) * (2 * kFFTerms);
#pragma unroll 1
    for (int q = 0; q < kFFTerms; ++q) {
        const double sa = block_sum(A[q], sh);
        const double sb = block_sum(B[q], sh);
        if (threadIdx.x == 0) {
            out[q] = sa;
            out[kFFTerms + q] = sb;
        }
    }
}

// the moments of each set: the block sums added in block order, then weighted by w_lm
__global__ void ff_moments_reduce_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ mom)
{
    const int set = blockIdx.x, q = threadIdx.x;
    if (q >= 2 * kFFTerms) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[((long long)set * nblocks + b) * (2 * kFFTerms) + q];
    const int t = q % kFFTerms;
    int l = 0;
    while (term(l + 1, 0) <= t) ++l;
    const int m = t - term(l, 0);
    double w = m == 0 ? 1.0 : 2.0;  // (2 - [m = 0]) (l-m)!/(l+m)!
    for (int k = l - m + 1; k <= l + m; ++k) w /= (double)k;
    mom[(long long)set * 2 * kFFTerms + q] = w * s;
}

// boundary nodes of both potentials; blockIdx.z = 6 * set + face
__global__ void __launch_bounds__(kFFThreads) ff_boundary_kernel(Geo g, const double* __restrict__ com,
                                                                  const double* __restrict__ mom, double G, double a0,
                                                                  double* __restrict__ phiN, double* __restrict__ phi)
{
    const int set = blockIdx.z / 6, face = blockIdx.z - 6 * set;
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    const int n = g.n;
    if (a > n) return;
    int i, j, k;
    switch (face) {
    case 0: i = 0; j = a; k = b; break;
    case 1: i = n; j = a; k = b; break;
    case 2: i = a; j = 0; k = b; break;
    case 3: i = a; j = n; k = b; break;
    case 4: i = a; j = b; k = 0; break;
    default: i = a; j = b; k = n; break;
    }
    const long long o = set * nat_elems(n) + i + (long long)(n + 1) * (j + (long long)(n + 1) * k);
    const double M = com[4 * set];
    if (M == 0.0) {
        phiN[o] = 0.0;
        phi[o] = 0.0;
        return;
    }
    const double dx = g.x0 + i * g.h - com[4 * set + 1];
    const double dy = g.y0 + j * g.h - com[4 * set + 2];
    const double dz = g.z0 + k * g.h - com[4 * set + 3];
    const double r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
    double re[kFFTerms], im[kFFTerms];
    solid(dx, dy, dz, re, im);
    const double* A = mom + (long long)set * 2 * kFFTerms;
    const double* B = A + kFFTerms;
    const double ir = 1.0 / r, ir2 = ir * ir;
    double sum = 0.0, ip = ir;  // |d|^-(2l+1)
#pragma unroll
    for (int l = 0; l <= kFFL; ++l) {
        double sl = 0.0;
#pragma unroll
        for (int m = 0; m <= l; ++m) sl += re[term(l, m)] * A[term(l, m)] + im[term(l, m)] * B[term(l, m)];
        sum += sl * ip;
        ip *= ir2;
    }
    phiN[o] = -G * sum;
    const double Am = G * M, C = 4.0 * a0 * Am;
    phi[o] = -Am / (2.0 * r) + 0.5 * (-sqrt(Am * Am + C * r2) / r + sqrt(C) * asinh(sqrt(C) * r / Am));
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

size_t far_field_scratch_doubles(int nsets)
{
    return (size_t)nsets * ((size_t)kFFBlocks * (4 + 2 * kFFTerms) + 4 + 2 * kFFTerms);
}

void launch_far_field(const double* rho, int n, double L, double cx, double cy, double cz, double G, double a0,
                      double* phiN, double* phi, double* scratch, int nsets, cudaStream_t s)
{
    Geo g;
    g.n = n;
    g.h = L / (double)n;
    g.h3 = g.h * g.h * g.h;
    g.x0 = cx - 0.5 * L;
    g.y0 = cy - 0.5 * L;
    g.z0 = cz - 0.5 * L;
    double* mass_part = scratch;
    double* mom_part = mass_part + (size_t)nsets * kFFBlocks * 4;
    double* com = mom_part + (size_t)nsets * kFFBlocks * 2 * kFFTerms;
    double* mom = com + (size_t)nsets * 4;
    ff_mass_kernel<<<dim3(kFFBlocks, nsets), kFFThreads, 0, s>>>(rho, g, mass_part);
    ff_com_kernel<<<nsets, 32, 0, s>>>(mass_part, kFFBlocks, com);
    ff_moments_kernel<<<dim3(kFFBlocks, nsets), kFFThreads, 0, s>>>(rho, g, com, mom_part);
    ff_moments_reduce_kernel<<<nsets, 2 * kFFTerms, 0, s>>>(mom_part, kFFBlocks, mom);
    ff_boundary_kernel<<<dim3(cdiv(n + 1, kFFThreads), (unsigned)(n + 1), 6 * (unsigned)nsets), kFFThreads, 0, s>>>(
        g, com, mom, G, a0, phiN, phi);
}

}  // namespace qumond
