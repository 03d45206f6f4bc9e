// Grid kernels of the QUMOND path on natural-layout FP64 arrays: the
// fixed-point CIC deposit (Section 2 step 1), nested-box boundary values
// (Section 2), the QUMOND source (Section 2 step 3, Eq. 2), forces and the
// rotation curve (Section 2, Eq. 4; box rule of Section 3.1).
#include "qumond_internal.h"

namespace qumond {

namespace {

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ long long nat(int n, int i, int j, int k)
{
    const long long P = n + 1;
    return (long long)i + P * ((long long)j + P * (long long)k);
}

// ---------------------------------------------------------------------------
// Cloud-in-cell deposit in 64-bit fixed point.  Every product is an
// individually rounded FP64 operation (no fused multiply-add), and the
// conversion rounds half to even, so each corner's integer share is the same
// on any machine and the grid does not depend on the order of the atomics.
__global__ void cic_deposit_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                   const double* __restrict__ z, const double* __restrict__ m, long long np, int n,
                                   double xlo, double ylo, double zlo, double inv_h, double two_shift,
                                   unsigned long long* __restrict__ q)
{
    {
        const int set = blockIdx.y;  // one row of blocks per set: np particles each
        const long long po = set * np;
        x += po, y += po, z += po, m += po;
        q += set * nat_elems(n);
    }
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double tx = __dmul_rn(__dsub_rn(x[p], xlo), inv_h);
    const double ty = __dmul_rn(__dsub_rn(y[p], ylo), inv_h);
    const double tz = __dmul_rn(__dsub_rn(z[p], zlo), inv_h);
    const double dn = (double)n;
    if (!(tx >= 0.0 && tx < dn && ty >= 0.0 && ty < dn && tz >= 0.0 && tz < dn)) return;
    const double fx = floor(tx), fy = floor(ty), fz = floor(tz);
    const int i = (int)fx, j = (int)fy, k = (int)fz;
    if (i >= n || j >= n || k >= n) return;
    const double dx = __dsub_rn(tx, fx), dy = __dsub_rn(ty, fy), dz = __dsub_rn(tz, fz);
    const double wx[2] = {__dsub_rn(1.0, dx), dx};
    const double wy[2] = {__dsub_rn(1.0, dy), dy};
    const double wz[2] = {__dsub_rn(1.0, dz), dz};
    const double ms = __dmul_rn(m[p], two_shift);
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const double mbc = ms;  // ((ms * wx) * wy) * wz, left to right
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const double w = __dmul_rn(__dmul_rn(__dmul_rn(mbc, wx[a]), wy[b]), wz[c]);
                const long long qv = __double2ll_rn(w);
                atomicAdd(q + nat(n, i + a, j + b, k + c), (unsigned long long)qv);
            }
        }
}

__global__ void fixed_to_rho_kernel(const long long* __restrict__ q, double* __restrict__ rho, long long count,
                                    double scale)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < count) rho[t] = __ll2double_rn(q[t]) * scale;
}

// ---------------------------------------------------------------------------
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

// blockIdx.z = 6 * set + face
__global__ void boundary_zero_kernel(double* __restrict__ u, int n)
{
    const int set = blockIdx.z / 6, face = blockIdx.z - 6 * set;
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a > n) return;
    int i, j, k;
    face_node(face, a, b, n, i, j, k);
    u[set * nat_elems(n) + nat(n, i, j, k)] = 0.0;
}

// Trilinear interpolation of a natural-layout grid at index coordinates t.
__device__ __forceinline__ double trilinear_idx(const double* __restrict__ a, int n, double tx, double ty, double tz)
{
    const double t[3] = {tx, ty, tz};
    int i0[3];
    double d[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        int ii = (int)floor(t[q]);
        ii = ii < 0 ? 0 : (ii > n - 1 ? n - 1 : ii);
        i0[q] = ii;
        d[q] = t[q] - (double)ii;
    }
    double v = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a3 = 0; a3 < 2; ++a3) {
                const double w = (a3 ? d[0] : 1.0 - d[0]) * (b ? d[1] : 1.0 - d[1]) * (c ? d[2] : 1.0 - d[2]);
                v += w * a[nat(n, i0[0] + a3, i0[1] + b, i0[2] + c)];
            }
    return v;
}

// Boundary of a box from its parent (box_ratio times the side, same centre,
// same n): child node i sits at parent index n (r-1)/(2r) + i/r along each
// axis (Section 2: the parent solution is interpolated onto the child's
// boundary).
__global__ void boundary_from_parent_kernel(const double* __restrict__ parent, double* __restrict__ u, int n, int ratio)
{
    const int set = blockIdx.z / 6, face = blockIdx.z - 6 * set;  // blockIdx.z = 6 * set + face
    parent += set * nat_elems(n);
    u += set * nat_elems(n);
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a > n) return;
    int i, j, k;
    face_node(face, a, b, n, i, j, k);
    const double inv_r = 1.0 / (double)ratio;
    const double q = 0.5 * (double)n * (1.0 - inv_r);
    u[nat(n, i, j, k)] = trilinear_idx(parent, n, q + inv_r * i, q + inv_r * j, q + inv_r * k);
}

// ---------------------------------------------------------------------------
// QUMOND source by the face-flux difference (Section 2 step 3, Eq. 2).
//
// Precision: the differences of the potential carry the information and are
// taken to ~48 bits; the gradient magnitude, nu and the fluxes are FP32
// (which perturbs the solved potential by ~1e-8 relative).  FP64 arithmetic
// and 64-bit conversions are ~60x slower than FP32 on this GPU, so each FP64
// value is split once, with integer instructions, into an exact pair of FP32
// numbers hi + lo (hi: the top 24 significant bits, lo: the next 24), and a
// difference is (hi_a - hi_b) + (lo_a - lo_b).
//
// Layout: a CTA owns a 32 x 8 tile of (i, j) and walks k through a chunk of
// planes.  Three consecutive planes of the tile plus a one-node halo sit in
// shared memory as hi/lo pairs; every node computes the fluxes through its
// +x, +y and +z faces once, and its source is the difference of its own
// fluxes and those of its -x, -y, -z neighbours (the -z one carried over from
// the previous plane).
constexpr int kSrcTX = 32, kSrcTY = 8, kSrcKC = 16;
constexpr int kSrcPX = kSrcTX + 2, kSrcPY = kSrcTY + 2;

// x = hi + lo exactly up to the 48th significant bit, both FP32, integer ops
// only.  |x| < 2^-126 gives (0, 0); lo is dropped below |x| < 2^-74.
__device__ __forceinline__ void split_hi_lo(double x, float& hi, float& lo)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const int E = (int)((b >> 52) & 0x7ffu);
    if (E < 897) {
        hi = 0.0f;
        lo = 0.0f;
        return;
    }
    if (E > 1150) {  // beyond FP32 range (or inf/nan): no split
        hi = __double2float_rn(x);
        lo = 0.0f;
        return;
    }
    const unsigned long long M = b & 0xFFFFFFFFFFFFFull;
    hi = __uint_as_float(sign | ((unsigned)(E - 896) << 23) | (unsigned)(M >> 29));
    if (E < 949) {
        lo = 0.0f;
        return;
    }
    const float r = __uint2float_rn((unsigned)(M & 0x1FFFFFFFull));  // < 2^29
    lo = __uint_as_float(sign | __float_as_uint(r * __uint_as_float((unsigned)(E - 948) << 23)));
}

// Exact FP32 -> FP64 with integer ops (subnormals flushed to zero).
__device__ __forceinline__ double f32_to_f64(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0) return __longlong_as_double((long long)sign);
    const unsigned long long ed = e == 255 ? 2047ull : (unsigned long long)(e + 896);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

struct SrcPlanes {
    float hi[3][kSrcPY][kSrcPX];
    float lo[3][kSrcPY][kSrcPX];
};

// Phi(a) - Phi(b) for smem positions (plane, y, x).
#define SRC_D(pa, ya, xa, pb, yb, xb)                                                                                  \
    ((S.hi[pa][ya][xa] - S.hi[pb][yb][xb]) + (S.lo[pa][ya][xa] - S.lo[pb][yb][xb]))

// Flux (times h) through the face from node P to node P + e_axis:
// nu(|g|/a0) * (Phi(Q) - Phi(P)); |g| from the normal difference and the
// means of the two nodes' transverse central differences.
__device__ __forceinline__ float face_flux(float dn, float ta, float tb, float inv_h, float four_a0)
{
    const float gn = dn * inv_h;
    const float q = 0.25f * inv_h;
    const float g2 = gn * gn + (ta * q) * (ta * q) + (tb * q) * (tb * q);
    if (!(g2 > 0.0f)) return 0.0f;
    const float nu = 0.5f * (1.0f + sqrtf(1.0f + four_a0 * rsqrtf(g2)));
    return nu * dn;
}

// Face fluxes with P at smem position (plane p, y, x).  pm/pp: planes below/above p.
__device__ __forceinline__ float flux_x(const SrcPlanes& S, int pm, int p, int pp, int y, int x, float ih, float fa)
{
    const float dn = SRC_D(p, y, x + 1, p, y, x);
    const float ty = SRC_D(p, y + 1, x, p, y - 1, x) + SRC_D(p, y + 1, x + 1, p, y - 1, x + 1);
    const float tz = SRC_D(pp, y, x, pm, y, x) + SRC_D(pp, y, x + 1, pm, y, x + 1);
    return face_flux(dn, ty, tz, ih, fa);
}
__device__ __forceinline__ float flux_y(const SrcPlanes& S, int pm, int p, int pp, int y, int x, float ih, float fa)
{
    const float dn = SRC_D(p, y + 1, x, p, y, x);
    const float tx = SRC_D(p, y, x + 1, p, y, x - 1) + SRC_D(p, y + 1, x + 1, p, y + 1, x - 1);
    const float tz = SRC_D(pp, y, x, pm, y, x) + SRC_D(pp, y + 1, x, pm, y + 1, x);
    return face_flux(dn, tx, tz, ih, fa);
}
// face between plane p (P) and plane pp (Q = P + e_z)
__device__ __forceinline__ float flux_z(const SrcPlanes& S, int p, int pp, int y, int x, float ih, float fa)
{
    const float dn = SRC_D(pp, y, x, p, y, x);
    const float tx = SRC_D(p, y, x + 1, p, y, x - 1) + SRC_D(pp, y, x + 1, pp, y, x - 1);
    const float ty = SRC_D(p, y + 1, x, p, y - 1, x) + SRC_D(pp, y + 1, x, pp, y - 1, x);
    return face_flux(dn, tx, ty, ih, fa);
}

__global__ void __launch_bounds__(kSrcTX * kSrcTY)
source_kernel(const double* __restrict__ phi, double* __restrict__ src, int n, float inv_h, float four_a0,
              float inv_h2, int zper)
{
    __shared__ SrcPlanes S;
    __shared__ float Fx[kSrcTY][kSrcTX + 1];  // Fx[y][x + 1]: face (x, x+1), x = -1 .. 31
    __shared__ float Fy[kSrcTY + 1][kSrcTX];  // Fy[y + 1][x]: face (y, y+1), y = -1 .. 7
    const int set = (int)gridDim.z == zper ? 0 : blockIdx.z / zper;  // blockIdx.z = zper * set + chunk
    const int kc = blockIdx.z - set * zper;
    phi += set * nat_elems(n);
    src += set * nat_elems(n);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kSrcTX + tx;
    const int i0 = blockIdx.x * kSrcTX, j0 = blockIdx.y * kSrcTY;
    const int k0 = kc * kSrcKC;
    const int k1 = min(k0 + kSrcKC, n + 1);
    const long long P = n + 1;

    // plane k of the tile (with halo) into slot `slot`; outside the grid -> 0
    auto load_plane = [&](int k, int slot) {
        for (int t = tid; t < kSrcPX * kSrcPY; t += kSrcTX * kSrcTY) {
            const int lx = t % kSrcPX, ly = t / kSrcPX;
            const int gi = i0 - 1 + lx, gj = j0 - 1 + ly;
            float h = 0.0f, l = 0.0f;
            if (k >= 0 && k <= n && gi >= 0 && gi <= n && gj >= 0 && gj <= n)
                split_hi_lo(phi[gi + P * (gj + P * (long long)k)], h, l);
            S.hi[slot][ly][lx] = h;
            S.lo[slot][ly][lx] = l;
        }
    };

    const int x = tx + 1, y = ty + 1;
    const int i = i0 + tx, j = j0 + ty;
    load_plane(k0 - 1, 0);
    load_plane(k0, 1);
    // the next plane's values are fetched into registers one plane ahead, so their loads are in flight
    // while the current plane's fluxes are computed
    constexpr int kEnt = (kSrcPX * kSrcPY + kSrcTX * kSrcTY - 1) / (kSrcTX * kSrcTY);  // 2
    double pre[kEnt];
    auto fetch = [&](int k) {
#pragma unroll
        for (int q = 0; q < kEnt; ++q) {
            const int t = tid + q * kSrcTX * kSrcTY;
            const int lx = t % kSrcPX, ly = t / kSrcPX;
            const int gi = i0 - 1 + lx, gj = j0 - 1 + ly;
            pre[q] = (t < kSrcPX * kSrcPY && k >= 0 && k <= n && gi >= 0 && gi <= n && gj >= 0 && gj <= n)
                         ? phi[gi + P * (gj + P * (long long)k)]
                         : 0.0;
        }
    };
    auto store = [&](int slot) {  // the fetched plane into a slot, split into hi/lo
#pragma unroll
        for (int q = 0; q < kEnt; ++q) {
            const int t = tid + q * kSrcTX * kSrcTY;
            if (t >= kSrcPX * kSrcPY) continue;
            const int lx = t % kSrcPX, ly = t / kSrcPX;
            float h = 0.0f, l = 0.0f;
            split_hi_lo(pre[q], h, l);  // zero -> (0, 0), as for nodes outside the grid
            S.hi[slot][ly][lx] = h;
            S.lo[slot][ly][lx] = l;
        }
    };
    fetch(k0 + 1);
    __syncthreads();
    // flux through the -z face of plane k0 (between k0-1 and k0)
    float fz_prev = flux_z(S, 0, 1, y, x, inv_h, four_a0);
    int pm = 0, pc = 1, pp = 2;  // slots of planes k-1, k, k+1
    for (int k = k0; k < k1; ++k) {
        __syncthreads();  // everyone is done with the slot about to be overwritten
        store(pp);        // plane k + 1
        if (k + 1 < k1) fetch(k + 2);
        __syncthreads();
        Fx[ty][tx + 1] = flux_x(S, pm, pc, pp, y, x, inv_h, four_a0);
        if (tx == 0) Fx[ty][0] = flux_x(S, pm, pc, pp, y, x - 1, inv_h, four_a0);
        Fy[ty + 1][tx] = flux_y(S, pm, pc, pp, y, x, inv_h, four_a0);
        if (ty == 0) Fy[0][tx] = flux_y(S, pm, pc, pp, y - 1, x, inv_h, four_a0);
        const float fz = flux_z(S, pc, pp, y, x, inv_h, four_a0);
        __syncthreads();
        if (i <= n && j <= n) {
            const bool inner = i > 0 && i < n && j > 0 && j < n && k > 0 && k < n;
            const float v = inner ? ((Fx[ty][tx + 1] - Fx[ty][tx]) + (Fy[ty + 1][tx] - Fy[ty][tx]) + (fz - fz_prev)) * inv_h2
                                  : 0.0f;
            src[i + P * (j + P * (long long)k)] = f32_to_f64(v);
        }
        fz_prev = fz;
        const int t = pm;
        pm = pc;
        pc = pp;
        pp = t;
    }
}
#undef SRC_D

// ---------------------------------------------------------------------------
// Forces at points: finest box whose containing cell has 8 interior corners.
__device__ __forceinline__ bool find_cell(const BoxGeom& g, int n, double x, double y, double z, int* ijk, double* d)
{
    const double t[3] = {(x - g.xlo) * g.inv_h, (y - g.ylo) * g.inv_h, (z - g.zlo) * g.inv_h};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!(t[a] >= 1.0 && t[a] < (double)(n - 1))) return false;
        const double fl = floor(t[a]);
        ijk[a] = (int)fl;
        d[a] = t[a] - fl;
        if (ijk[a] < 1 || ijk[a] > n - 2) return false;
    }
    return true;
}

// set: which of the context's sets (its potentials sit at set (n+1)^3 in every box)
__device__ __forceinline__ void grad_at(const BoxGeom& g, int n, const int* ijk, const double* d, double* out,
                                        int set = 0)
{
    const double* phi = g.phi + set * nat_elems(n);
    const double s = -0.5 / g.h;
    const long long P = n + 1, Q = P * P;
    double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const long long o = nat(n, ijk[0] + a, ijk[1] + b, ijk[2] + c);
                const double w = (a ? d[0] : 1.0 - d[0]) * (b ? d[1] : 1.0 - d[1]) * (c ? d[2] : 1.0 - d[2]);
                gx += w * ((phi[o + 1] - phi[o - 1]) * s);
                gy += w * ((phi[o + P] - phi[o - P]) * s);
                gz += w * ((phi[o + Q] - phi[o - Q]) * s);
            }
    out[0] = gx;
    out[1] = gy;
    out[2] = gz;
}

__global__ void forces_kernel(BoxSet boxes, const double* __restrict__ qx, const double* __restrict__ qy,
                              const double* __restrict__ qz, long long nq, double* __restrict__ gx,
                              double* __restrict__ gy, double* __restrict__ gz)
{
    const int set = blockIdx.y;  // one row of blocks per set: nq points each
    {
        const long long po = set * nq;
        qx += po, qy += po, qz += po, gx += po, gy += po, gz += po;
    }
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= nq) return;
    const double x = qx[p], y = qy[p], z = qz[p];
    double g[3] = {0.0, 0.0, 0.0};
    for (int b = boxes.nboxes - 1; b >= 0; --b) {
        int ijk[3];
        double d[3];
        if (find_cell(boxes.b[b], boxes.n, x, y, z, ijk, d)) {
            grad_at(boxes.b[b], boxes.n, ijk, d, g, set);
            break;
        }
    }
    gx[p] = g[0];
    gy[p] = g[1];
    gz[p] = g[2];
}

// One CTA per radius bin, one thread per azimuth; the azimuthal mean is
// summed in index order by thread 0, so the result is reproducible.
constexpr int kMaxPhi = 1024;

// With several sets: blockIdx.y = set, its outermost radius rmax_sets[set]
// when given, its bins at set * nbins of the outputs.
__global__ void rotation_curve_kernel(BoxSet boxes, double cx, double cy, double cz, int nbins, double rmax,
                                      const double* __restrict__ rmax_sets, int nphi, double frac,
                                      double* __restrict__ r_out, double* __restrict__ vc_out)
{
    __shared__ double dphidr[kMaxPhi];
    const int set = blockIdx.y;
    if (rmax_sets) rmax = rmax_sets[set];
    r_out += set * (long long)nbins;
    vc_out += set * (long long)nbins;
    const int kb = blockIdx.x;
    const double R = ((double)kb + 0.5) * rmax / (double)nbins;
    int b0 = 0;
    for (int b = boxes.nboxes - 1; b >= 0; --b)
        if (R < frac * boxes.b[b].L) {
            b0 = b;
            break;
        }
    for (int m = threadIdx.x; m < nphi; m += blockDim.x) {
        const double ph = 6.283185307179586476925286766559 * (double)m / (double)nphi;
        double s, c;
        sincos(ph, &s, &c);
        const double x = cx + R * c, y = cy + R * s, z = cz;
        double g[3] = {0.0, 0.0, 0.0};
        for (int b = b0; b >= 0; --b) {
            int ijk[3];
            double d[3];
            if (find_cell(boxes.b[b], boxes.n, x, y, z, ijk, d)) {
                grad_at(boxes.b[b], boxes.n, ijk, d, g, set);
                break;
            }
        }
        dphidr[m] = -(g[0] * c + g[1] * s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int m = 0; m < nphi; ++m) sum += dphidr[m];
        const double v2 = R * (sum / (double)nphi);
        r_out[kb] = R;
        vc_out[kb] = v2 >= 0.0 ? sqrt(v2) : -sqrt(-v2);
    }
}

// Science extras on the same tracers and box rule as the rotation curve.
// mode 0 (Eq. 3, algebraic MOND): the field at a tracer is nu(|g_N|/a0) g_N
//   from the Newtonian potentials (a tracer with g_N = 0 adds 0), out = sign(s) sqrt(|s|),
//   s = R * mean of -(g . R^);
// mode 1 (Section 5.6, isothermal sech^2(z/h) stellar layer): tracers at height z_eval,
//   s = mean of dPhi/dz * h / (2 tanh(z_eval / h)), out = sign(s) sqrt(|s|) = sigma_z.
__global__ void profile_kernel(BoxSet boxes, double cx, double cy, double cz, int nbins, double rmax, int nphi,
                               double frac, int mode, double a0, double z_eval, double h, double* __restrict__ r_out,
                               double* __restrict__ out)
{
    __shared__ double val[kMaxPhi];
    const int set = blockIdx.y;  // one row of blocks per set
    r_out += set * (long long)nbins;
    out += set * (long long)nbins;
    const int kb = blockIdx.x;
    const double R = ((double)kb + 0.5) * rmax / (double)nbins;
    int b0 = 0;
    for (int b = boxes.nboxes - 1; b >= 0; --b)
        if (R < frac * boxes.b[b].L) {
            b0 = b;
            break;
        }
    const double zt = mode == 1 ? cz + z_eval : cz;
    for (int m = threadIdx.x; m < nphi; m += blockDim.x) {
        const double ph = 6.283185307179586476925286766559 * (double)m / (double)nphi;
        double s, c;
        sincos(ph, &s, &c);
        double g[3] = {0.0, 0.0, 0.0};
        for (int b = b0; b >= 0; --b) {
            int ijk[3];
            double d[3];
            if (find_cell(boxes.b[b], boxes.n, cx + R * c, cy + R * s, zt, ijk, d)) {
                grad_at(boxes.b[b], boxes.n, ijk, d, g, set);
                break;
            }
        }
        if (mode == 0) {
            const double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            const double nu = gm > 0.0 ? 0.5 + 0.5 * sqrt(1.0 + 4.0 * a0 / gm) : 0.0;
            val[m] = -nu * (g[0] * c + g[1] * s);
        } else {
            val[m] = -g[2];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int m = 0; m < nphi; ++m) sum += val[m];
        const double mean = sum / (double)nphi;
        const double v2 = mode == 0 ? R * mean : mean * h / (2.0 * tanh(z_eval / h));
        r_out[kb] = R;
        out[kb] = v2 >= 0.0 ? sqrt(v2) : -sqrt(-v2);
    }
}

}  // namespace

// --- launchers ----------------------------------------------------------------
void launch_cic_deposit(const double* x, const double* y, const double* z, const double* m, long long np, int n,
                        double xlo, double ylo, double zlo, double inv_h, double two_shift, int64_t* q,
                        cudaStream_t s, int nsets)
{
    if (np <= 0) return;
    cic_deposit_kernel<<<dim3(cdiv(np, 256), (unsigned)nsets), 256, 0, s>>>(
        x, y, z, m, np, n, xlo, ylo, zlo, inv_h, two_shift, reinterpret_cast<unsigned long long*>(q));
}

void launch_fixed_to_rho(const int64_t* q, double* rho, long long count, double scale, cudaStream_t s)
{
    fixed_to_rho_kernel<<<cdiv(count, 256), 256, 0, s>>>(reinterpret_cast<const long long*>(q), rho, count, scale);
}

void launch_boundary_zero(double* u, int n, cudaStream_t s, int nsets)
{
    boundary_zero_kernel<<<dim3(cdiv(n + 1, 128), (unsigned)(n + 1), 6 * (unsigned)nsets), 128, 0, s>>>(u, n);
}

void launch_boundary_from_parent(const double* parent, double* u, int n, int ratio, cudaStream_t s, int nsets)
{
    boundary_from_parent_kernel<<<dim3(cdiv(n + 1, 128), (unsigned)(n + 1), 6 * (unsigned)nsets), 128, 0, s>>>(
        parent, u, n, ratio);
}

void launch_source(const double* phi, double* src, int n, double h, double a0, cudaStream_t s, int nsets)
{
    const unsigned zper = cdiv(n + 1, kSrcKC);
    const dim3 grid(cdiv(n + 1, kSrcTX), cdiv(n + 1, kSrcTY), zper * (unsigned)nsets);
    source_kernel<<<grid, dim3(kSrcTX, kSrcTY), 0, s>>>(phi, src, n, (float)(1.0 / h), (float)(4.0 * a0),
                                                        (float)(1.0 / (h * h)), (int)zper);
}

void launch_forces(const BoxSet& boxes, const double* qx, const double* qy, const double* qz, long long nq,
                   double* gx, double* gy, double* gz, cudaStream_t s, int nsets)
{
    if (nq <= 0) return;
    forces_kernel<<<dim3(cdiv(nq, 128), (unsigned)nsets), 128, 0, s>>>(boxes, qx, qy, qz, nq, gx, gy, gz);
}

void launch_rotation_curve(const BoxSet& boxes, double cx, double cy, double cz, int nbins, double rmax,
                           const double* rmax_sets, int nphi, double frac, double* r_out, double* vc_out,
                           cudaStream_t s, int nsets)
{
    rotation_curve_kernel<<<dim3(nbins, nsets), 128, 0, s>>>(boxes, cx, cy, cz, nbins, rmax, rmax_sets, nphi, frac,
                                                             r_out, vc_out);
}

void launch_profile(const BoxSet& boxes, double cx, double cy, double cz, int nbins, double rmax, int nphi, double frac,
                    int mode, double a0, double z_eval, double h, double* r_out, double* out, cudaStream_t s,
                    int nsets)
{
    profile_kernel<<<dim3(nbins, nsets), 128, 0, s>>>(boxes, cx, cy, cz, nbins, rmax, nphi, frac, mode, a0, z_eval, h,
                                                      r_out, out);
}

// Quality of fit (Section 3.5): chi2[s] = (1/nbins) sum_i ((vc[s][i] - v_obs[i]) / sigma[i])^2.
// One warp per parameter set; lane l sums bins l, l+32, ... and the warp adds
// the 32 partial sums by a fixed shuffle tree, so the result does not depend
// on scheduling.
__global__ void chi2_kernel(const double* __restrict__ vc, const double* __restrict__ v_obs,
                            const double* __restrict__ sigma, int nbins, int nsets, double* __restrict__ chi2)
{
    const int set = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (set >= nsets) return;
    const double* row = vc + (long long)set * nbins;
    double acc = 0.0;
    for (int i = lane; i < nbins; i += 32) {
        const double d = (row[i] - v_obs[i]) / sigma[i];
        acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) chi2[set] = acc / (double)nbins;
}

void launch_chi2(const double* vc, const double* v_obs, const double* sigma, int nbins, int nsets, double* chi2,
                 cudaStream_t s)
{
    const int warps = 4;
    chi2_kernel<<<(nsets + warps - 1) / warps, 32 * warps, 0, s>>>(vc, v_obs, sigma, nbins, nsets, chi2);
}

}  // namespace qumond
