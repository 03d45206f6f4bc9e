// One defect-correction iteration (update of the fixed-point iterate and the
// residual of the updated iterate, QUMOND_PREC_MIXED_FIXED) with its planes
// staged by the tensor-memory accelerator, for finest levels of n >= 128.
//
// The arithmetic is that of fixed_update_residual_kernel (fixed_outer.cu):
//   U' = U + round(e 2^S) on interior nodes, U' = U on the boundary,
//   R = F - (sum of the 6 neighbours of U' - 6 U'),  r = R 2^-S / h^2,
// U' written to the iterate's other buffer.  A CTA owns a 32 x 8 tile of
// (i, j) columns and 16 k-planes; for every plane it needs, one thread issues
// three 3-D boxes (U with a one-node halo, the two colour rows of e covering
// the same nodes, F of the tile) into a four-slot shared-memory ring
// completed by mbarriers, so each input byte crosses HBM once and the loads of
// three planes are in flight while a plane is processed.  Waits are bounded:
// after kSpinLimit polls a CTA records a fault (reported by the solve as a
// timeout) and finishes without waiting further.
#include "qumond_internal.h"

namespace qumond {

namespace {

constexpr int kTI = 32, kTJ = 8, kKC = 16;
constexpr int kW = kTI + 2, kH = kTJ + 2;            // U box: 34 x 10 nodes (int64)
constexpr int kEW = 20;                              // e box: 20 row entries (17 used) x 10 rows (FP32)
constexpr unsigned kUBytes = kW * kH * 8;            // 2720
constexpr unsigned kEBytes = kEW * kH * 4;           // 800
constexpr unsigned kFBytes = kW * kTJ * 8;           // 2176
constexpr unsigned kOffE0 = 2816, kOffE1 = 3712, kOffF = 4608, kSlotBytes = 6784;  // 128-byte aligned parts
constexpr int kSlots = 4;
constexpr long long kSpinLimit = 1LL << 24;
constexpr int kMinN = 128;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float i64_to_f32(long long x)
{
    const float hi = (float)(int)(x >> 32);
    const float lo = (float)(unsigned)(x & 0xffffffffLL);
    return fmaf(hi, 4294967296.0f, lo);
}

__device__ __forceinline__ long long f32_to_i64(float v)
{
    if (fabsf(v) < 8388608.0f) return (long long)__float2int_rn(v);
    const unsigned bits = __float_as_uint(v);
    const int ex = (int)((bits >> 23) & 0xffu) - 150;
    if (ex > 38) return (bits >> 31) ? -(1LL << 62) : (1LL << 62);
    const long long m = (long long)((bits & 0x7fffffu) | 0x800000u) << ex;
    return (bits >> 31) ? -m : m;
}

__global__ void __launch_bounds__(kTI * kTJ)
fixed_update_residual_tma_kernel(const __grid_constant__ CUtensorMap map_u0, const __grid_constant__ CUtensorMap map_u1,
                                 const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_e0,
                                 const __grid_constant__ CUtensorMap map_e1, long long* Ua, long long* Ub, int n,
                                 float ih2, const SolveState* __restrict__ st, float* __restrict__ r, LevelView v,
                                 double* __restrict__ partials, int* __restrict__ fault)
{
    __shared__ __align__(128) unsigned char slot[kSlots][kSlotBytes];
    __shared__ long long pl[3][kH][kW];
    __shared__ __align__(8) unsigned long long bar[kSlots];
    __shared__ int abort_flag;
    __shared__ double sr[kTI * kTJ / 32];
    const bool odd = (st->it & 1) != 0;
    const CUtensorMap* mu = odd ? &map_u1 : &map_u0;
    long long* __restrict__ nxt = odd ? Ua : Ub;
    const int S = st->scale_exp;
    const float scf = ldexpf(1.0f, S);
    const float k = ldexpf(1.0f, -S) * ih2;
    constexpr float kDown = 9.313225746154785e-10f;  // 2^-30
    const long long P = n + 2, Q = P * (n + 1);
    const int ni = (n - 1 + kTI - 1) / kTI, nj = (n - 1 + kTJ - 1) / kTJ;
    const int item = blockIdx.x;
    const int ti = item % ni;
    const int i0 = 1 + ti * kTI, j0 = 1 + ((item / ni) % nj) * kTJ, kb = 1 + (item / (ni * nj)) * kKC;
    const int ke = kb + kKC < n ? kb + kKC : n;  // residual planes kb .. ke-1; planes kb-1 .. ke are staged
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTI + tx;
    const bool leader = tid == 0;
    if (leader) {
        abort_flag = 0;
        for (int q = 0; q < kSlots; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int q) {  // plane q into its slot (leader only)
        const int u = q - (kb - 1);
        unsigned char* base = &slot[u % kSlots][0];
        if ((smem_u32(base) & 127u) != 0u) {  // never issue a copy the TMA unit would reject
            atomicExch(fault, 2);
            atomicExch(&abort_flag, 1);
            return;
        }
        unsigned long long* b = &bar[u % kSlots];
        mbar_expect_tx(b, kUBytes + 2 * kEBytes + kFBytes);
        tma_load_3d(base, mu, i0 - 1, j0 - 1, q, b);
        tma_load_3d(base + kOffE0, &map_e0, (i0 - 1) >> 1, j0 - 1, q, b);
        tma_load_3d(base + kOffE1, &map_e1, (i0 - 1) >> 1, j0 - 1, q, b);
        tma_load_3d(base + kOffF, &map_f, i0 - 1, j0, q, b);
    };
    if (leader)
        for (int q = kb - 1; q < kb - 1 + kSlots && q <= ke; ++q) issue(q);
    bool ok = true;
    auto wait = [&](int q) {  // lane 0 of each warp polls; __syncwarp passes the completed phase to the warp
        if ((tid & 31) == 0) {
            const int u = q - (kb - 1);
            long long spins = 0;
            while (ok && !mbar_try_wait(&bar[u % kSlots], (unsigned)((u / kSlots) & 1))) {
                if (++spins > kSpinLimit || *(volatile int*)&abort_flag) {
                    ok = false;
                    atomicExch(fault, 1);
                }
            }
        }
        __syncwarp();
    };
    // this thread's (up to) two halo entries of a plane
    constexpr int kEnt = 2;
    int hi[kEnt], hj[kEnt], isum[kEnt], em[kEnt];
    bool inner[kEnt], own[kEnt], used[kEnt];
    long long ob[kEnt];
#pragma unroll
    for (int m = 0; m < kEnt; ++m) {
        const int t = tid + m * kTI * kTJ;
        used[m] = t < kW * kH;
        hi[m] = t % kW;
        hj[m] = t / kW;
        const int i = i0 - 1 + hi[m], j = j0 - 1 + hj[m];
        inner[m] = used[m] && i >= 1 && i < n && j >= 1 && j < n;
        own[m] = inner[m] && hi[m] >= 1 && hi[m] <= kTI && hj[m] >= 1 && hj[m] <= kTJ;
        isum[m] = i + j;
        em[m] = (i >> 1) - ((i0 - 1) >> 1);  // entry of the node in its colour row of the e box
        ob[m] = (long long)i + P * (long long)j;
    }
    const int ri = i0 + tx, rj = j0 + ty;
    const bool rok = ri < n && rj < n;
    float rr = 0.0f;
    for (int q = kb - 1; q <= ke; ++q) {
        const int u = q - (kb - 1);
        wait(q);
        const unsigned char* base = &slot[u % kSlots][0];
        const long long(*ub)[kW] = reinterpret_cast<const long long(*)[kW]>(base);
        const float(*e0)[kEW] = reinterpret_cast<const float(*)[kEW]>(base + kOffE0);
        const float(*e1)[kEW] = reinterpret_cast<const float(*)[kEW]>(base + kOffE1);
        const bool qin = q >= 1 && q < n, qown = q >= kb && q < ke;
        long long(*dst)[kW] = pl[q % 3];
#pragma unroll
        for (int m = 0; m < kEnt; ++m) {
            if (!used[m]) continue;
            long long val = ub[hj[m]][hi[m]];  // zero beyond the array (TMA fill), as for i or j > n
            if (inner[m] && qin) {
                const float ev = ((isum[m] + q) & 1) ? e1[hj[m]][em[m]] : e0[hj[m]][em[m]];
                val += f32_to_i64(ev * scf);
                if (own[m] && qown) nxt[ob[m] + Q * q] = val;
            }
            dst[hj[m]][hi[m]] = val;
        }
        __syncthreads();
        const int kk = q - 1;
        if (kk >= kb && rok && ok) {
            const long long(*fb)[kW] =
                reinterpret_cast<const long long(*)[kW]>(&slot[(u - 1) % kSlots][0] + kOffF);
            const long long(*pm)[kW] = pl[(kk - 1) % 3];
            const long long(*p0)[kW] = pl[kk % 3];
            const long long(*pp)[kW] = pl[(kk + 1) % 3];
            const int hx = tx + 1, hy = ty + 1;
            const long long sum = (p0[hy][hx + 1] + p0[hy][hx - 1]) + (p0[hy + 1][hx] + p0[hy - 1][hx]) +
                                  (pp[hy][hx] + pm[hy][hx]) - 6 * p0[hy][hx];
            const float R = i64_to_f32(fb[ty][tx + 1] - sum);
            r[node_off(v, ri, rj, kk)] = R * k;
            const float Rs = R * kDown;
            rr = fmaf(Rs, Rs, rr);
        }
        __syncthreads();  // slot of plane q-1 is free
        if (leader && q >= kb && q + kSlots - 1 <= ke) issue(q + kSlots - 1);
    }
    for (int off = 16; off > 0; off >>= 1) rr += __shfl_down_sync(0xffffffffu, rr, off);
    if ((tid & 31) == 0) sr[tid >> 5] = rr;
    __syncthreads();
    if (leader) {
        double a = 0.0;
        for (int q = 0; q < kTI * kTJ / 32; ++q) a += sr[q];
        const double up = ldexp((double)k, 30);
        partials[2 * blockIdx.x] = a * up * up;
        partials[2 * blockIdx.x + 1] = 0.0;
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            (void)cudaGetLastError();
    }
    return fn;
}

bool encode3(EncodeTiledFn enc, CUtensorMap* m, CUtensorMapDataType t, void* base, cuuint64_t d0, cuuint64_t d1,
             cuuint64_t d2, cuuint64_t s1, cuuint64_t s2, cuuint32_t b0, cuuint32_t b1)
{
    const cuuint64_t dims[3] = {d0, d1, d2};
    const cuuint64_t strides[2] = {s1, s2};
    const cuuint32_t box[3] = {b0, b1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, t, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool make_fixed_maps(int64_t* U, int64_t* U2, int64_t* F, float* e, const LevelView& v, FixedMaps* out)
{
    out->ok = false;
    const int n = v.n;
    if (n < kMinN) return false;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t rowb = (cuuint64_t)(n + 2) * 8, planeb = rowb * (n + 1);
    const cuuint64_t erow = (cuuint64_t)v.M * 4, eplane = erow * (n + 1);
    bool ok = encode3(enc, &out->u[0], CU_TENSOR_MAP_DATA_TYPE_INT64, U, n + 2, n + 1, n + 1, rowb, planeb, kW, kH) &&
              encode3(enc, &out->u[1], CU_TENSOR_MAP_DATA_TYPE_INT64, U2, n + 2, n + 1, n + 1, rowb, planeb, kW, kH) &&
              encode3(enc, &out->f, CU_TENSOR_MAP_DATA_TYPE_INT64, F, n + 2, n + 1, n + 1, rowb, planeb, kW, kTJ);
    for (int c = 0; ok && c < 2; ++c)
        ok = encode3(enc, &out->e[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, e + (long long)c * v.cs, v.M, n + 1, n + 1, erow,
                     eplane, kEW, kH);
    out->ok = ok;
    return ok;
}

int launch_fixed_update_residual_tma(int64_t* U, int64_t* U2, const FixedMaps& maps, int n, double h,
                                     const SolveState* st, float* r, const LevelView& v, double* partials, int* fault,
                                     cudaStream_t s)
{
    const int items = ((n - 1 + kTI - 1) / kTI) * ((n - 1 + kTJ - 1) / kTJ) * ((n - 1 + kKC - 1) / kKC);
    fixed_update_residual_tma_kernel<<<items, dim3(kTI, kTJ), 0, s>>>(
        maps.u[0], maps.u[1], maps.f, maps.e[0], maps.e[1], reinterpret_cast<long long*>(U),
        reinterpret_cast<long long*>(U2), n, (float)(1.0 / (h * h)), st, r, v, partials, fault);
    return items;
}

}  // namespace qumond
