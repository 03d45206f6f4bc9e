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
// Precision: the moments and the terms of degree l <= 2 (monopole, dipole,
// quadrupole: all but ~1e-3 of Phi_N for a galaxy inside its box) are FP64;
// the terms of degree 3..8 are evaluated in FP32 on the unit vector d/|d| with
// moments scaled by s^-l (s the half side of the box), which keeps their
// values in range and their rounding (~1e-6 of a term) far below 1e-9 of
// Phi_N; F(r) is FP64.  The FP64 pipe of this GPU is slow, and these boundary
// nodes (6 (n+1)^2) dominate the cost.  The sums over nodes are per-block
// partial sums added in a fixed order, so the values are the same on every
// run.  Every grid of a context with several sets is handled in the same
// launches (blockIdx.y, or the face index, carries the set).
#include "qumond_internal.h"

namespace qumond {

namespace {

constexpr int kFFL = 8;
constexpr int kFFTerms = (kFFL + 1) * (kFFL + 2) / 2;  // (l, m), 0 <= m <= l <= 8: 45
constexpr int kFFThreads = 128;
constexpr int kFFBlocks = 2 * 152;  // blocks per set of the two reductions over nodes

__host__ __device__ constexpr int term(int l, int m) { return l * (l + 1) / 2 + m; }

// mass T_lm(d) added to A[term(l, m)] + i B[term(l, m)] for l <= 8: the
// recurrence runs along l for each m with the two previous values only, so no
// table of T is kept (A and B stay in registers).
__device__ __forceinline__ void add_moments(double mass, double dx, double dy, double dz, double* A, double* B)
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
        double r0 = df * pr, i0 = df * pi;  // T_mm
        A[term(m, m)] += mass * r0;
        B[term(m, m)] += mass * i0;
        if (m + 1 <= kFFL) {
            double r1 = (double)(2 * m + 1) * dz * r0, i1 = (double)(2 * m + 1) * dz * i0;  // T_{m+1,m}
            A[term(m + 1, m)] += mass * r1;
            B[term(m + 1, m)] += mass * i1;
#pragma unroll
            for (int l = m + 2; l <= kFFL; ++l) {
                const double inv = 1.0 / (double)(l - m);
                const double rl = ((double)(2 * l - 1) * dz * r1 - (double)(l + m - 1) * r2 * r0) * inv;
                const double il = ((double)(2 * l - 1) * dz * i1 - (double)(l + m - 1) * r2 * i0) * inv;
                A[term(l, m)] += mass * rl;
                B[term(l, m)] += mass * il;
                r0 = r1, i0 = i1, r1 = rl, i1 = il;
            }
        }
    }
}

// T_lm(u) for 3 <= l <= 8 in FP32 (the same recurrence), u a unit vector
__device__ __forceinline__ void solid_high_f32(float ux, float uy, float uz, float* re, float* im)
{
    float pr = 1.0f, pi = 0.0f, df = 1.0f;
#pragma unroll
    for (int m = 0; m <= kFFL; ++m) {
        if (m > 0) {
            const float a = pr * ux - pi * uy, b = pr * uy + pi * ux;
            pr = a;
            pi = b;
            df *= (float)(2 * m - 1);
        }
        float r0 = df * pr, i0 = df * pi;
        if (m >= 3) re[term(m, m)] = r0, im[term(m, m)] = i0;
        if (m + 1 <= kFFL) {
            float r1 = (float)(2 * m + 1) * uz * r0, i1 = (float)(2 * m + 1) * uz * i0;
            if (m + 1 >= 3) re[term(m + 1, m)] = r1, im[term(m + 1, m)] = i1;
#pragma unroll
            for (int l = m + 2; l <= kFFL; ++l) {
                const float inv = 1.0f / (float)(l - m);
                const float rl = ((float)(2 * l - 1) * uz * r1 - (float)(l + m - 1) * r0) * inv;  // |u| = 1
                const float il = ((float)(2 * l - 1) * uz * i1 - (float)(l + m - 1) * i0) * inv;
                if (l >= 3) re[term(l, m)] = rl, im[term(l, m)] = il;
                r0 = r1, i0 = i1, r1 = rl, i1 = il;
            }
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

// Sum over the block's threads of one value each, in a fixed order; valid in thread 0.
__device__ __forceinline__ double block_total(double v, double* sh)
{
    return block_sum(v, sh);
}

struct Geo {
    int n;
    double x0, y0, z0, h, h3;
    double s;  // half side of the box: the scale of the FP32 high-degree terms
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

// M and the centre of mass of each set from the block sums (thread t adds
// blocks t, t + 128, ...; then the fixed-order block sum)
__global__ void __launch_bounds__(kFFThreads) ff_com_kernel(const double* __restrict__ part, int nblocks,
                                                             double* __restrict__ com)
{
    __shared__ double sh[kFFThreads / 32];
    const int set = blockIdx.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kFFThreads)
        for (int q = 0; q < 4; ++q) a[q] += part[((long long)set * nblocks + b) * 4 + q];
    double t[4];
    for (int q = 0; q < 4; ++q) t[q] = block_total(a[q], sh);
    if (threadIdx.x == 0) {
        double* c = com + 4 * set;
        c[0] = t[0];
        c[1] = t[0] != 0.0 ? t[1] / t[0] : 0.0;
        c[2] = t[0] != 0.0 ? t[2] / t[0] : 0.0;
        c[3] = t[0] != 0.0 ? t[3] / t[0] : 0.0;
    }
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
    for (int q = 0; q < kFFTerms; ++q) A[q] = B[q] = 0.0;  // in registers: every index is a constant
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
            add_moments(m, x - cx, y - cy, z - cz, A, B);
        }
    }
    double* out = part + ((long long)set * gridDim.x + blockIdx.x) * (2 * kFFTerms);
#pragma unroll  // constant indices keep A and B in registers
    for (int q = 0; q < kFFTerms; ++q) {
        const double sa = block_sum(A[q], sh);
        const double sb = block_sum(B[q], sh);
        if (threadIdx.x == 0) {
            out[q] = sa;
            out[kFFTerms + q] = sb;
        }
    }
}

// the moments of each set: the block sums (one block per moment and set:
// thread t adds blocks t, t + 128, ..., then the fixed-order block sum),
// weighted by w_lm = (2 - [m = 0]) (l-m)!/(l+m)!; FP64 for all degrees and,
// for degrees >= 3, an FP32 copy scaled by s^-l
__global__ void __launch_bounds__(kFFThreads) ff_moments_reduce_kernel(const double* __restrict__ part, int nblocks,
                                                                        double s, double* __restrict__ mom,
                                                                        float* __restrict__ momf)
{
    __shared__ double sh[kFFThreads / 32];
    const int q = blockIdx.x, set = blockIdx.y;  // q < 2 kFFTerms: A_lm, then B_lm
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kFFThreads) v += part[((long long)set * nblocks + b) * (2 * kFFTerms) + q];
    const double tot = block_total(v, sh);
    if (threadIdx.x != 0) return;
    const int t = q % kFFTerms;
    int l = 0;
    while (term(l + 1, 0) <= t) ++l;
    const int m = t - term(l, 0);
    double w = m == 0 ? 1.0 : 2.0;
    for (int k = l - m + 1; k <= l + m; ++k) w /= (double)k;
    mom[(long long)set * 2 * kFFTerms + q] = w * tot;
    momf[(long long)set * 2 * kFFTerms + q] = (float)(w * tot / pow(s, (double)l));
}

// boundary nodes of both potentials; blockIdx.z = 6 * set + face
__global__ void __launch_bounds__(kFFThreads) ff_boundary_kernel(Geo g, const double* __restrict__ com,
                                                                  const double* __restrict__ mom,
                                                                  const float* __restrict__ momf, double G, double a0,
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
    const double ir = 1.0 / r, ir2 = ir * ir;
    const double* A = mom + (long long)set * 2 * kFFTerms;
    const double* B = A + kFFTerms;
    // degrees 0..2 in FP64: T_00 = 1, T_10 = dz, T_11 = dx + i dy, T_20 = (3 dz^2 - |d|^2)/2,
    // T_21 = 3 dz (dx + i dy), T_22 = 3 (dx + i dy)^2 (the recurrence written out)
    const double t20 = 0.5 * (3.0 * dz * dz - r2), t22r = 3.0 * (dx * dx - dy * dy), t22i = 6.0 * dx * dy;
    const double s0 = A[term(0, 0)];
    const double s1 = A[term(1, 0)] * dz + (A[term(1, 1)] * dx + B[term(1, 1)] * dy);
    const double s2 = A[term(2, 0)] * t20 + (A[term(2, 1)] * (3.0 * dz * dx) + B[term(2, 1)] * (3.0 * dz * dy)) +
                      (A[term(2, 2)] * t22r + B[term(2, 2)] * t22i);
    const double low = (s0 + (s1 + s2 * ir2) * ir2) * ir;
    // degrees 3..8 in FP32 on the unit vector, moments scaled by s^-l: T_lm(d) / |d|^(2l+1) = T_lm(u) (s/r)^l / (s^l r)
    const float ux = (float)(dx * ir), uy = (float)(dy * ir), uz = (float)(dz * ir);
    float re[kFFTerms], im[kFFTerms];
    solid_high_f32(ux, uy, uz, re, im);
    const float* Af = momf + (long long)set * 2 * kFFTerms;
    const float* Bf = Af + kFFTerms;
    const float q = (float)(g.s * ir);
    float high = 0.0f, qp = q * q * q;
#pragma unroll
    for (int l = 3; l <= kFFL; ++l) {
        float sl = 0.0f;
#pragma unroll
        for (int m = 0; m <= l; ++m) sl += re[term(l, m)] * Af[term(l, m)] + im[term(l, m)] * Bf[term(l, m)];
        high += sl * qp;
        qp *= q;
    }
    phiN[o] = -G * (low + (double)high * ir);
    const double Am = G * M, C = 4.0 * a0 * Am;
    phi[o] = -Am / (2.0 * r) + 0.5 * (-sqrt(Am * Am + C * r2) / r + sqrt(C) * asinh(sqrt(C) * r / Am));
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

size_t far_field_scratch_doubles(int nsets)
{
    return (size_t)nsets * ((size_t)kFFBlocks * (4 + 2 * kFFTerms) + 4 + 2 * kFFTerms + kFFTerms);  // + FP32 copy
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
    g.s = 0.5 * L;
    double* mass_part = scratch;
    double* mom_part = mass_part + (size_t)nsets * kFFBlocks * 4;
    double* com = mom_part + (size_t)nsets * kFFBlocks * 2 * kFFTerms;
    double* mom = com + (size_t)nsets * 4;
    float* momf = reinterpret_cast<float*>(mom + (size_t)nsets * 2 * kFFTerms);
    ff_mass_kernel<<<dim3(kFFBlocks, nsets), kFFThreads, 0, s>>>(rho, g, mass_part);
    ff_com_kernel<<<nsets, kFFThreads, 0, s>>>(mass_part, kFFBlocks, com);
    ff_moments_kernel<<<dim3(kFFBlocks, nsets), kFFThreads, 0, s>>>(rho, g, com, mom_part);
    ff_moments_reduce_kernel<<<dim3(2 * kFFTerms, nsets), kFFThreads, 0, s>>>(mom_part, kFFBlocks, g.s, mom, momf);
    ff_boundary_kernel<<<dim3(cdiv(n + 1, kFFThreads), (unsigned)(n + 1), 6 * (unsigned)nsets), kFFThreads, 0, s>>>(
        g, com, mom, momf, G, a0, phiN, phi);
}

}  // namespace qumond
