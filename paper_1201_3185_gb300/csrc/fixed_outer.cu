// Defect correction with a 64-bit fixed-point master iterate
// (QUMOND_PREC_MIXED_FIXED).
//
// The outer loop of the mixed-precision solve needs a residual r = f - L u
// accurate well beyond FP32.  On this GPU FP64 arithmetic and every 64-bit
// float conversion run at ~2 operations per clock per SM (FP32: ~110), so a
// 7-point FP64 residual is bound by the FP64 pipe at ~4x its memory time.
// Here the iterate is held as integers U = u * 2^S and the right-hand side as
// F = coef * rhs * h^2 * 2^S, both int64.  Then
//   R = F - (sum of the 6 neighbours of U - 6 U)
// is exact integer arithmetic, and r = R * 2^-S / h^2 is rounded once, to
// FP32, for the V-cycle.  S is chosen per solve so that max|u| * 2^S is about
// 2^56 (the FMG result bounds max|u| to ~1%); the resolution 2^-S is then
// ~2^-56 max|u|, finer than FP64's 2^-53 relative spacing near max|u|, and
// |F| <= 12 max|U| < 2^60 cannot overflow for a solution of the problem.
//
// Only the once-per-solve scaling of the FP64 right-hand side uses the FP64
// pipe (one multiply per node); the conversions between FP64 and int64 are
// done on the integer pipe (fixed_conv.h), and the per-V-cycle kernels use
// integer and FP32 instructions only.
#include "qumond_internal.h"
#include "fixed_conv.h"

namespace qumond {

namespace {

__device__ __forceinline__ long long nat(int n, int i, int j, int k)
{
    const long long P = n + 1;
    return (long long)i + P * ((long long)j + P * (long long)k);
}

// The fixed-point arrays (U, its second buffer, F) have rows of n + 2 entries
// (one unused), so that a row is a multiple of 16 bytes and the arrays can be
// described to the tensor-memory accelerator.
__device__ __forceinline__ long long fix(int n, int i, int j, int k)
{
    return (long long)i + (long long)(n + 2) * ((long long)j + (long long)(n + 1) * (long long)k);
}

// int64 -> FP32 through its two 32-bit halves (within one FP32 rounding of
// the exact value); integer and FP32 pipes only.
__device__ __forceinline__ float i64_to_f32(long long x)
{
    const float hi = (float)(int)(x >> 32);
    const float lo = (float)(unsigned)(x & 0xffffffffLL);
    return fmaf(hi, 4294967296.0f, lo);
}

// FP32 -> int64, round to nearest: exact when |v| >= 2^23 (v is then an
// integer), __float2int_rn below that.
__device__ __forceinline__ long long f32_to_i64(float v)
{
    if (fabsf(v) < 8388608.0f) return (long long)__float2int_rn(v);
    const unsigned bits = __float_as_uint(v);
    const int ex = (int)((bits >> 23) & 0xffu) - 150;
    if (ex > 38) return (bits >> 31) ? -(1LL << 62) : (1LL << 62);  // saturate (only a diverging solve gets here)
    const long long m = (long long)((bits & 0x7fffffu) | 0x800000u) << ex;
    return (bits >> 31) ? -m : m;
}

// 2^e as FP32 / FP64 from an integer exponent.
__device__ __forceinline__ float pow2f(int e) { return ldexpf(1.0f, e); }
__device__ __forceinline__ double pow2d(int e) { return ldexp(1.0, e); }

constexpr int kThreads = 128;
constexpr int kMaxBlocks = 152 * 16;

// --- choice of the scale S ---------------------------------------------------
// Largest |u| over the FMG result (FP32, both colours, interior) or, for a
// warm start, over the caller's interior values, and over the boundary values.
__global__ void __launch_bounds__(kThreads)
scan_max_kernel(const float* __restrict__ e, LevelView v, const double* __restrict__ u64, int n, int from_u64,
                unsigned* __restrict__ out)
{
    const int set = blockIdx.y;  // one row of blocks per set
    e += set * 2 * v.cs;
    u64 += set * nat_elems(n);
    out += set;
    unsigned local = 0u;
    const int rows = (n + 1) * (n + 1);
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = row % (n + 1), k = row / (n + 1);
        const bool brow = j == 0 || j == n || k == 0 || k == n;
        for (int i = threadIdx.x; i <= n; i += kThreads) {
            const bool bnd = brow || i == 0 || i == n;
            float val;
            if (bnd || from_u64) val = (float)u64[nat(n, i, j, k)];
            else val = e[node_off(v, i, j, k)];
            const unsigned b = __float_as_uint(fabsf(val));
            local = b > local ? b : local;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned o = __shfl_down_sync(0xffffffffu, local, off);
        local = o > local ? o : local;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, local);
}

// The same maximum after FMG (not a warm start), as one flat pass over the
// finest FP32 level with 16-byte loads: its boundary entries hold the FP32
// values of the boundary data (set before FMG interpolates into the level),
// and the entries that are no node (beyond i = n, row padding) hold zero.
__global__ void __launch_bounds__(256) scan_max_level_kernel(const float4* __restrict__ e, long long n4,
                                                             unsigned* __restrict__ out)
{
    const int set = blockIdx.y;  // one row of blocks per set; n4 float4 per set
    e += set * n4;
    out += set;
    unsigned local = 0u;
    for (long long q = blockIdx.x * 256LL + threadIdx.x; q < n4; q += (long long)gridDim.x * 256) {
        const float4 x = e[q];
        const unsigned a = __float_as_uint(fabsf(x.x)), b = __float_as_uint(fabsf(x.y));
        const unsigned c = __float_as_uint(fabsf(x.z)), d = __float_as_uint(fabsf(x.w));
        const unsigned m1 = a > b ? a : b, m2 = c > d ? c : d;
        const unsigned m = m1 > m2 ? m1 : m2;
        local = m > local ? m : local;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned o = __shfl_down_sync(0xffffffffu, local, off);
        local = o > local ? o : local;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(out, local);
}

// S = 56 - ceil(log2(max|u|)), kept in [-60, 100] so that 2^S and 2^-S stay
// normal FP32 numbers; also clears the max for the next solve.
__global__ void choose_scale_kernel(unsigned* __restrict__ maxbits, SolveState* __restrict__ st)
{
    maxbits += blockIdx.x;  // one block per set
    st += blockIdx.x;
    const float m = __uint_as_float(*maxbits);
    int S = 0;
    if (m > 0.0f && isfinite(m)) {
        int ex;
        frexpf(m, &ex);  // m = f * 2^ex, 0.5 <= f < 1, so m < 2^ex
        S = 56 - ex;
        S = S < -60 ? -60 : (S > 100 ? 100 : S);
    }
    st->scale_exp = S;
    st->nonfinite = isfinite(m) ? 0 : 1;  // a NaN or infinity in the start: no integer iterate holds it
    *maxbits = 0u;
}

// The binary64 exponent field is all ones: an infinity or a NaN (integer pipe only).
__device__ __forceinline__ bool f64_nonfinite(double x) { return ((f64_bits(x) >> 52) & 0x7ff) == 0x7ff; }

// U = round(u * 2^S) on every node (interior from the FP32 FMG result or the
// caller's warm start, boundary from the boundary data), F = round(coef h^2 f
// 2^S) on the interior (0 on the boundary); the boundary of the second buffer
// too.  One thread per pair of nodes (i = 2a, 2a+1) of a row over a flat
// grid; the pair is one 16-byte store in U and F (their rows start on 16-byte
// boundaries), and the entry i = n+1 of a row (padding) is written as zero.
__global__ void __launch_bounds__(256)
fixed_init_pairs_kernel(const float* __restrict__ e, LevelView v, const double* __restrict__ u64,
                        const double* __restrict__ rhs, double coef_h2, int n, int from_u64,
                        SolveState* __restrict__ st, long long* __restrict__ U, long long* __restrict__ U2,
                        long long* __restrict__ F)
{
    {
        const int set = blockIdx.y;  // one row of blocks per set
        e += set * 2 * v.cs;
        u64 += set * nat_elems(n);
        rhs += set * nat_elems(n);
        st += set;
        const long long fs = set * (long long)(n + 2) * (n + 1) * (n + 1);
        U += fs, U2 += fs, F += fs;
    }
    const int pairs = n / 2 + 1;
    const long long idx = blockIdx.x * 256LL + threadIdx.x;
    if (idx >= (long long)pairs * (n + 1) * (n + 1)) return;
    const int row = (int)(idx / pairs), a = (int)(idx - (long long)row * pairs);
    const int j = row % (n + 1), k = row / (n + 1);
    const int S = st->scale_exp;
    const double sc = pow2d(S);
    const float scf = pow2f(S);
    const double kf = coef_h2 * sc;
    const bool brow = j == 0 || j == n || k == 0 || k == n;
    const int i0 = 2 * a;
    const bool has1 = i0 + 1 <= n;
    const bool b0 = brow || i0 == 0 || i0 == n, b1 = brow || i0 + 1 == n;
    const long long o = nat(n, i0, j, k), of = fix(n, i0, j, k);
    const int c0 = (i0 + j + k) & 1;
    const long long er = ((long long)k * (n + 1) + j) * v.M + a;  // entry of both nodes in their colour rows
    // FP64 -> int64 on the integer pipe (round to nearest even, as the FP64 conversion instruction)
    const long long v0 = (b0 || from_u64) ? f64_to_i64_rn(u64[o] * sc) : f32_to_i64(e[(long long)c0 * v.cs + er] * scf);
    long long v1 = 0, f1 = 0;
    if (has1) {
        v1 = (b1 || from_u64) ? f64_to_i64_rn(u64[o + 1] * sc) : f32_to_i64(e[(long long)(c0 ^ 1) * v.cs + er] * scf);
        f1 = b1 ? 0LL : f64_to_i64_rn(rhs[o + 1] * kf);
    }
    const long long f0 = b0 ? 0LL : f64_to_i64_rn(rhs[o] * kf);
    if ((!b0 && f64_nonfinite(rhs[o])) || (has1 && !b1 && f64_nonfinite(rhs[o + 1]))) st->nonfinite = 1;
    *reinterpret_cast<longlong2*>(U + of) = make_longlong2(v0, v1);
    *reinterpret_cast<longlong2*>(F + of) = make_longlong2(f0, f1);
    // the second buffer's interior is written before it is read
    if (b0) U2[of] = v0;
    if (has1 && b1) U2[of + 1] = v1;
}

// R = F - (sum of 6 neighbours - 6 U), exact; r = R 2^-S / h^2 in FP32 into
// the finest level; per-block partial sums of r^2 (and, on the first check,
// of f^2 with f = F 2^-S / h^2).  The squares are summed as (R 2^-30)^2 in
// FP32 (|R| <= 2^60, so they lie in [2^-60, 2^60]: no overflow or
// underflow) and scaled back per block in FP64.  A thread takes a pair of
// consecutive nodes (i even, i+1; rows of n+2 entries, so the pair starts on
// a 16-byte boundary): 16-byte loads of the pair and of its four neighbour
// pairs, two scalars for the x-neighbours past the ends; the two nodes are
// one red and one black entry with the same index, so the stores of a warp
// are contiguous in each colour array.
__global__ void __launch_bounds__(kThreads)
fixed_residual_kernel(const long long* __restrict__ U, const long long* __restrict__ F, int n, float ih2,
                      const SolveState* __restrict__ st, int want_f, float* __restrict__ r, LevelView v,
                      double* __restrict__ partials, long long pstride)
{
    {
        const int set = blockIdx.y;  // one row of blocks per set
        const long long fs = set * (long long)(n + 2) * (n + 1) * (n + 1);
        U += fs, F += fs;
        st += set;
        r += set * 2 * v.cs;
        partials += set * pstride;
    }
    const long long P = n + 2, Q = P * (n + 1);
    const float k = pow2f(-st->scale_exp) * ih2;
    const int half = n / 2;
    const long long items = (long long)(n - 1) * (n - 1) * half;  // (row, pair)
    float rr = 0.0f, ff = 0.0f;
    constexpr float kDown = 9.313225746154785e-10f;  // 2^-30
    for (long long it = blockIdx.x * (long long)kThreads + threadIdx.x; it < items;
         it += (long long)gridDim.x * kThreads) {
        const int m = (int)(it % half);
        const long long row = it / half;
        const int j = (int)(row % (n - 1)) + 1, kk = (int)(row / (n - 1)) + 1;
        const int i = 2 * m;  // nodes i (i = 0 is a boundary node) and i + 1 (<= n - 1)
        const long long o = fix(n, i, j, kk);
        const longlong2 c = *reinterpret_cast<const longlong2*>(U + o);
        const long long left = U[o - 1], right = U[o + 2];
        const longlong2 yp = *reinterpret_cast<const longlong2*>(U + o + P);
        const longlong2 ym = *reinterpret_cast<const longlong2*>(U + o - P);
        const longlong2 zp = *reinterpret_cast<const longlong2*>(U + o + Q);
        const longlong2 zm = *reinterpret_cast<const longlong2*>(U + o - Q);
        const longlong2 fv = *reinterpret_cast<const longlong2*>(F + o);
        // the same integer sums as one node per thread (exact, so their order does not matter)
        const long long s0 = (c.y + left) + (yp.x + ym.x) + (zp.x + zm.x) - 6 * c.x;
        const long long s1 = (right + c.x) + (yp.y + ym.y) + (zp.y + zm.y) - 6 * c.y;
        const long long rowb = ((long long)kk * (v.n + 1) + j) * v.M + m;
        const int c0 = (i + j + kk) & 1;  // colour of node i; node i + 1 has the other one
        if (i >= 1) {
            const float R0 = i64_to_f32(fv.x - s0);
            r[(long long)c0 * v.cs + rowb] = R0 * k;
            const float Rs = R0 * kDown;
            rr = fmaf(Rs, Rs, rr);
            if (want_f) {
                const float Fs = i64_to_f32(fv.x) * kDown;
                ff = fmaf(Fs, Fs, ff);
            }
        }
        {
            const float R1 = i64_to_f32(fv.y - s1);
            r[(long long)(c0 ^ 1) * v.cs + rowb] = R1 * k;
            const float Rs = R1 * kDown;
            rr = fmaf(Rs, Rs, rr);
            if (want_f) {
                const float Fs = i64_to_f32(fv.y) * kDown;
                ff = fmaf(Fs, Fs, ff);
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, off);
        ff += __shfl_down_sync(0xffffffffu, ff, off);
    }
    __shared__ double sr[kThreads / 32], sf[kThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sr[w] = rr;
        sf[w] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < kThreads / 32; ++q) {
            a += sr[q];
            b += sf[q];
        }
        const double up = ldexp((double)k, 30);  // back to r = R k
        partials[2 * blockIdx.x] = a * up * up;
        partials[2 * blockIdx.x + 1] = b * up * up;
    }
}

// One defect-correction iteration after its V-cycle, in one pass:
//   U' = U + round(e 2^S) on interior nodes (U' = U on the boundary),
//   R = F - (sum of the 6 neighbours of U' - 6 U'),  r = R 2^-S / h^2,
// the same integers as updating every interior node and then running
// fixed_residual_kernel.
// A CTA owns a 32 x 8 tile of (i, j) columns and a chunk of k-planes; it forms
// U' on each plane of the tile and its one-node halo in shared memory (a ring
// of three planes) and writes U' for its own nodes.  Since a CTA reads the
// old values of its halo while the neighbouring CTA writes their new ones,
// the iterate alternates between two buffers: the current one is buffer
// (it & 1), it = V-cycles made so far (advanced by the decide kernel after).
constexpr int kFTI = 32, kFTJ = 8, kFKC = 16;
constexpr int kFW = kFTI + 2, kFH = kFTJ + 2;

__global__ void __launch_bounds__(kFTI * kFTJ)
fixed_update_residual_kernel(long long* Ua, long long* Ub, const long long* __restrict__ F,
                             const float* __restrict__ e, int n, float ih2, const SolveState* __restrict__ st,
                             float* __restrict__ r, LevelView v, double* __restrict__ partials, long long pstride,
                             int skip_stopped)
{
    __shared__ long long pl[3][kFH][kFW];
    {
        const int set = blockIdx.y;  // one row of blocks per set
        st += set;
        if (skip_stopped && !st->cont) return;
        const long long fs = set * (long long)(n + 2) * (n + 1) * (n + 1);
        Ua += fs, Ub += fs, F += fs;
        e += set * 2 * v.cs;
        r += set * 2 * v.cs;
        partials += set * pstride;
    }
    const bool odd = (st->it & 1) != 0;
    const long long* __restrict__ cur = odd ? Ub : Ua;
    long long* __restrict__ nxt = odd ? Ua : Ub;
    const int S = st->scale_exp;
    const float scf = pow2f(S);
    const float k = pow2f(-S) * ih2;
    constexpr float kDown = 9.313225746154785e-10f;  // 2^-30
    const long long P = n + 2, Q = P * (n + 1);          // padded rows of the fixed-point arrays
    const long long plane_e = (long long)(n + 1) * v.M;  // one plane of one colour array of the level
    const int ni = (n - 1 + kFTI - 1) / kFTI, nj = (n - 1 + kFTJ - 1) / kFTJ, nk = (n - 1 + kFKC - 1) / kFKC;
    const int items = ni * nj * nk;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kFTI + tx;
    constexpr int kEnt = 2;  // halo entries per thread per plane: tid and tid + 256 (34 x 10 = 340 entries)
    float rr = 0.0f;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int i0 = 1 + (item % ni) * kFTI, j0 = 1 + ((item / ni) % nj) * kFTJ, kb = 1 + (item / (ni * nj)) * kFKC;
        const int ke = kb + kFKC < n ? kb + kFKC : n;  // residual planes kb .. ke-1; planes kb-1 .. ke are formed
        // per entry: position, validity, and the parts of its offsets that do not depend on the plane
        int hi[kEnt], hj[kEnt], ii[kEnt];
        bool valid[kEnt], inner[kEnt], own[kEnt];
        long long ob[kEnt], eb[kEnt];
#pragma unroll
        for (int q = 0; q < kEnt; ++q) {
            const int t = tid + q * kFTI * kFTJ;
            hi[q] = t % kFW;
            hj[q] = t / kFW;
            const int i = i0 - 1 + hi[q], j = j0 - 1 + hj[q];  // >= 0 since i0, j0 >= 1
            ii[q] = i + j;
            valid[q] = t < kFW * kFH && i <= n && j <= n;
            inner[q] = valid[q] && i >= 1 && i < n && j >= 1 && j < n;
            own[q] = inner[q] && hi[q] >= 1 && hi[q] <= kFTI && hj[q] >= 1 && hj[q] <= kFTJ;
            ob[q] = (long long)i + P * (long long)j;
            eb[q] = (long long)j * v.M + (i >> 1);
        }
        const int ri = i0 + tx, rj = j0 + ty;
        const bool rok = ri < n && rj < n;
        const long long rb = (long long)ri + P * (long long)rj;
        long long ru[kEnt];
        float re[kEnt];
        auto fetch = [&](int q) {  // raw U and e of plane q for this thread's entries
            const bool qin = q >= 1 && q < n;
#pragma unroll
            for (int m = 0; m < kEnt; ++m) {
                ru[m] = valid[m] ? cur[ob[m] + Q * q] : 0LL;
                re[m] = (inner[m] && qin) ? e[(long long)((ii[m] + q) & 1) * v.cs + q * plane_e + eb[m]] : 0.0f;
            }
        };
        fetch(kb - 1);
        long long fcur = 0;
        for (int q = kb - 1; q <= ke; ++q) {
            const bool qin = q >= 1 && q < n, qown = q >= kb && q < ke;
            long long(*dst)[kFW] = pl[q % 3];
#pragma unroll
            for (int m = 0; m < kEnt; ++m) {
                if (tid + m * kFTI * kFTJ < kFW * kFH) {
                    long long val = ru[m];
                    if (inner[m] && qin) {
                        val += f32_to_i64(re[m] * scf);
                        if (own[m] && qown) nxt[ob[m] + Q * q] = val;
                    }
                    dst[hj[m]][hi[m]] = val;
                }
            }
            // loads for the next plane and the right-hand side of the next residual plane, in flight
            // across the barrier and this plane's residual
            if (q + 1 <= ke) fetch(q + 1);
            const long long fnext = (rok && qown) ? F[rb + Q * q] : 0LL;
            __syncthreads();
            const int kk = q - 1;
            if (kk >= kb && rok) {
                const long long(*pm)[kFW] = pl[(kk - 1) % 3];
                const long long(*p0)[kFW] = pl[kk % 3];
                const long long(*pp)[kFW] = pl[(kk + 1) % 3];
                const int hx = tx + 1, hy = ty + 1;
                const long long sum = (p0[hy][hx + 1] + p0[hy][hx - 1]) + (p0[hy + 1][hx] + p0[hy - 1][hx]) +
                                      (pp[hy][hx] + pm[hy][hx]) - 6 * p0[hy][hx];
                const float R = i64_to_f32(fcur - sum);
                r[node_off(v, ri, rj, kk)] = R * k;
                const float Rs = R * kDown;
                rr = fmaf(Rs, Rs, rr);
            }
            fcur = fnext;
            __syncthreads();
        }
    }
    for (int off = 16; off > 0; off >>= 1) rr += __shfl_down_sync(0xffffffffu, rr, off);
    __shared__ double sr[kFTI * kFTJ / 32];
    if ((tid & 31) == 0) sr[tid >> 5] = rr;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int q = 0; q < kFTI * kFTJ / 32; ++q) a += sr[q];
        const double up = ldexp((double)k, 30);
        partials[2 * blockIdx.x] = a * up * up;
        partials[2 * blockIdx.x + 1] = 0.0;
    }
}

__global__ void __launch_bounds__(kThreads)
fixed_output_kernel(const long long* Ua, const long long* Ub, double* __restrict__ u, int n,
                    const SolveState* __restrict__ st)
{
    {
        const int set = blockIdx.y;  // one row of blocks per set
        const long long fs = set * (long long)(n + 2) * (n + 1) * (n + 1);
        Ua += fs, Ub += fs;
        u += set * nat_elems(n);
        st += set;
    }
    const long long* __restrict__ U = (st->it & 1) ? Ub : Ua;
    const int S = st->scale_exp;
    const int rows = (n - 1) * (n - 1);
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = row % (n - 1) + 1, k = row / (n - 1) + 1;
        // U 2^-S: int64 -> FP64 on the integer pipe (round to nearest even, then an exact power-of-two scale)
        for (int i = threadIdx.x + 1; i < n; i += kThreads) u[nat(n, i, j, k)] = i64_to_f64_rn_scaled(U[fix(n, i, j, k)], -S);
    }
}

inline int blocks_for_rows(long long rows) { return (int)(rows < kMaxBlocks ? rows : kMaxBlocks); }

}  // namespace

void launch_fixed_scale(const float* e, const LevelView& v, const double* u64, int n, bool from_u64, unsigned* maxbits,
                        SolveState* st, cudaStream_t s, const Sets& sets)
{
    const unsigned ns = (unsigned)sets.n;
    if (from_u64)
        scan_max_kernel<<<dim3(blocks_for_rows((long long)(n + 1) * (n + 1)), ns), kThreads, 0, s>>>(e, v, u64, n, 1,
                                                                                                  maxbits);
    else
        scan_max_level_kernel<<<dim3(kMaxBlocks, ns), 256, 0, s>>>(reinterpret_cast<const float4*>(e), 2 * v.cs / 4,
                                                                   maxbits);
    choose_scale_kernel<<<ns, 1, 0, s>>>(maxbits, st);
}

void launch_fixed_init(const float* e, const LevelView& v, const double* u64, const double* rhs, double coef, double h,
                       int n, bool from_u64, SolveState* st, int64_t* U, int64_t* U2, int64_t* F, cudaStream_t s,
                       const Sets& sets)
{
    const long long threads = (long long)(n / 2 + 1) * (n + 1) * (n + 1);
    fixed_init_pairs_kernel<<<dim3((unsigned)((threads + 255) / 256), (unsigned)sets.n), 256, 0, s>>>(
        e, v, u64, rhs, coef * h * h, n, from_u64 ? 1 : 0, st, reinterpret_cast<long long*>(U),
        reinterpret_cast<long long*>(U2), reinterpret_cast<long long*>(F));
}

int launch_fixed_update_residual(int64_t* U, int64_t* U2, const int64_t* F, const float* e, int n, double h,
                                 const SolveState* st, float* r, const LevelView& v, double* partials, cudaStream_t s,
                                 const Sets& sets)
{
    const long long items = (long long)((n - 1 + kFTI - 1) / kFTI) * ((n - 1 + kFTJ - 1) / kFTJ) *
                            ((n - 1 + kFKC - 1) / kFKC);
    const int cap = fixed_residual_blocks(n);
    const int nb = (int)(items < cap ? items : cap);
    fixed_update_residual_kernel<<<dim3(nb, sets.n), dim3(kFTI, kFTJ), 0, s>>>(
        reinterpret_cast<long long*>(U), reinterpret_cast<long long*>(U2), reinterpret_cast<const long long*>(F), e, n,
        (float)(1.0 / (h * h)), st, r, v, partials, sets.pstride, sets.act ? 1 : 0);
    return nb;
}

int fixed_residual_blocks(int n) { return blocks_for_rows((long long)(n - 1) * (n - 1)); }

size_t fixed_elems(int n) { return (size_t)(n + 2) * (n + 1) * (n + 1); }

int launch_fixed_residual(const int64_t* U, const int64_t* F, int n, double h, const SolveState* st, bool want_f,
                          float* r, const LevelView& v, double* partials, cudaStream_t s, const Sets& sets)
{
    const int nb = fixed_residual_blocks(n);
    fixed_residual_kernel<<<dim3(nb, sets.n), kThreads, 0, s>>>(reinterpret_cast<const long long*>(U),
                                                                reinterpret_cast<const long long*>(F), n,
                                                                (float)(1.0 / (h * h)), st, want_f ? 1 : 0, r, v,
                                                                partials, sets.pstride);
    return nb;
}

void launch_fixed_output(const int64_t* U, const int64_t* U2, double* u, int n, const SolveState* st, cudaStream_t s,
                         const Sets& sets)
{
    fixed_output_kernel<<<dim3(fixed_residual_blocks(n), sets.n), kThreads, 0, s>>>(
        reinterpret_cast<const long long*>(U), reinterpret_cast<const long long*>(U2), u, n, st);
}

}  // namespace qumond
