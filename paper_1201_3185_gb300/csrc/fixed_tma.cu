// One defect-correction iteration (update of the fixed-point iterate and the
// residual of the updated iterate, QUMOND_PREC_MIXED_FIXED) with its planes
// staged by the tensor-memory accelerator, for finest levels of n >= 128.
//
// The arithmetic is that of fixed_update_residual_kernel (fixed_outer.cu):
//   U' = U + round(e 2^S) on interior nodes, U' = U on the boundary,
//   R = F - (sum of the 6 neighbours of U' - 6 U'),  r = R 2^-S / h^2,
// U' written to the iterate's other buffer.  A CTA owns a 32 x 8 tile of
// (i, j) columns, i from a multiple of 32, and 16 k-planes; for every plane it
// needs, one thread issues four 3-D boxes (U over i0-2 .. i0+33 and a one-row
// halo, the two colour rows of e covering the same nodes, F of the tile) into
// a three-slot shared-memory ring completed by mbarriers, so each input byte
// crosses HBM once and the loads of the next plane are in flight while a
// plane is processed (three slots rather than four leave room for seven CTAs
// per multiprocessor instead of six, which measured faster).  A thread works on a pair of consecutive nodes (i even, i+1):
// the pairs start on 16-byte boundaries in every staged array, so the update
// and the stencil use 16-byte shared-memory loads and stores.  Waits are bounded:
// after kSpinLimit polls a CTA records a fault (reported by the solve as a
// timeout), issues no further copies, waits (bounded) for the copies already
// in flight, and finishes.
#include "qumond_internal.h"

namespace qumond {

namespace {

constexpr int kTI = 32, kTJ = 8, kKC = 16;
constexpr int kPX = kTI / 2;                         // threads along i: one pair of nodes each
constexpr int kW = kTI + 4, kH = kTJ + 2;            // U box: i0-2 .. i0+33 x j0-1 .. j0+8 (int64)
constexpr int kEW = 24;                              // e box: entries i0/2-4 .. i0/2+19 (FP32)
constexpr unsigned kUBytes = kW * kH * 8;            // 2880
constexpr unsigned kEBytes = kEW * kH * 4;           // 960
constexpr unsigned kFBytes = kTI * kTJ * 8;          // 2048
constexpr unsigned kOffE0 = 2944, kOffE1 = 3968, kOffF = 4992, kSlotBytes = 7040;  // 128-byte aligned parts
static_assert(kOffE0 >= kUBytes && kOffE1 >= kOffE0 + kEBytes && kOffF >= kOffE1 + kEBytes &&
                  kSlotBytes >= kOffF + kFBytes && kOffE0 % 128 == 0 && kOffE1 % 128 == 0 && kOffF % 128 == 0 &&
                  kSlotBytes % 128 == 0,
              "slot parts are disjoint and 128-byte aligned");
constexpr int kSlots = 3;
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

// One box of a 4-D tensor (i, j, k, set); the 4th coordinate selects the set (0 for one set).
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
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

__global__ void __launch_bounds__(kPX * kTJ)
fixed_update_residual_tma_kernel(const __grid_constant__ CUtensorMap map_u0, const __grid_constant__ CUtensorMap map_u1,
                                 const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_e0,
                                 const __grid_constant__ CUtensorMap map_e1, long long* Ua, long long* Ub, int n,
                                 float ih2, const SolveState* __restrict__ st, float* __restrict__ r, LevelView v,
                                 double* __restrict__ partials, int* __restrict__ fault, long long pstride,
                                 int skip_stopped)
{
    const int set = blockIdx.y;  // one row of blocks per set
    st += set;
    if (skip_stopped && !st->cont) return;  // this set's correction has stopped (whole CTA, before any barrier)
    {
        const long long fs = set * (long long)(n + 2) * (n + 1) * (n + 1);
        Ua += fs, Ub += fs;
        r += set * 2 * v.cs;
        partials += set * pstride;
    }
    __shared__ __align__(128) unsigned char slot[kSlots][kSlotBytes];
    __shared__ __align__(16) long long pl[3][kH][kW];
    __shared__ __align__(8) unsigned long long bar[kSlots];
    __shared__ int abort_flag;
    __shared__ double sr[kPX * kTJ / 32];
    const bool odd = (st->it & 1) != 0;
    const CUtensorMap* mu = odd ? &map_u1 : &map_u0;
    long long* __restrict__ nxt = odd ? Ua : Ub;
    const int S = st->scale_exp;
    const float scf = ldexpf(1.0f, S);
    const float k = ldexpf(1.0f, -S) * ih2;
    constexpr float kDown = 9.313225746154785e-10f;  // 2^-30
    const long long P = n + 2, Q = P * (n + 1);
    const int ni = n / kTI, nj = (n - 1 + kTJ - 1) / kTJ;
    const int item = blockIdx.x;
    const int i0 = (item % ni) * kTI, j0 = 1 + ((item / ni) % nj) * kTJ, kb = 1 + (item / (ni * nj)) * kKC;
    const int ke = kb + kKC < n ? kb + kKC : n;  // residual planes kb .. ke-1; planes kb-1 .. ke are staged
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPX + tx;
    const bool leader = tid == 0;
    if (leader) {
        abort_flag = 0;
        for (int q = 0; q < kSlots; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // leader: planes kb-1 .. issued-1 have been issued; lane 0 of a warp: planes
    // before `landed` have been seen complete
    int issued = kb - 1, landed = kb - 1;
    auto issue = [&](int q) {  // plane q into its slot (leader only); nothing more once a wait gave up
        if (*(volatile int*)&abort_flag) return;
        const int u = q - (kb - 1);
        unsigned char* base = &slot[u % kSlots][0];
        if ((smem_u32(base) & 127u) != 0u) {  // never issue a copy the TMA unit would reject
            atomicExch(fault, 2);
            atomicExch(&abort_flag, 1);
            return;
        }
        unsigned long long* b = &bar[u % kSlots];
        mbar_expect_tx(b, kUBytes + 2 * kEBytes + kFBytes);
        tma_load_4d(base, mu, i0 - 2, j0 - 1, q, set, b);  // x: even int64 index, a 16-byte boundary
        tma_load_4d(base + kOffE0, &map_e0, i0 / 2 - 4, j0 - 1, q, set, b);  // x: a multiple of 4 floats
        tma_load_4d(base + kOffE1, &map_e1, i0 / 2 - 4, j0 - 1, q, set, b);
        tma_load_4d(base + kOffF, &map_f, i0, j0, q, set, b);
        issued = q + 1;
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
                    *(volatile int*)&abort_flag = 1;  // the leader stops issuing copies
                }
            }
            if (ok) landed = q + 1;
        }
        __syncwarp();
    };
    // this thread's (up to) two halo pairs of a plane: nodes (a, a+1), a = i0-2 + 2 hp, row j0-1 + hj
    constexpr int kPairs = kW / 2 * kH;  // 180
    constexpr int kEnt = (kPairs + kPX * kTJ - 1) / (kPX * kTJ);
    int hp[kEnt], hj[kEnt], em[kEnt], ipar[kEnt];
    bool used[kEnt], inner0[kEnt], inner1[kEnt], own[kEnt];
    long long ob[kEnt];
#pragma unroll
    for (int m = 0; m < kEnt; ++m) {
        const int t = tid + m * kPX * kTJ;
        used[m] = t < kPairs;
        hp[m] = t % (kW / 2);
        hj[m] = t / (kW / 2);
        const int a = i0 - 2 + 2 * hp[m], j = j0 - 1 + hj[m];
        const bool jin = used[m] && j >= 1 && j < n;
        inner0[m] = jin && a >= 1 && a < n;
        inner1[m] = jin && a + 1 >= 1 && a + 1 < n;
        // the pair is stored when both nodes lie in the tile (a >= i0, rows of the tile); a boundary node
        // (i = 0) is stored with its unchanged value, which the other buffer already holds
        own[m] = jin && a >= i0 && a < i0 + kTI && hj[m] >= 1 && hj[m] <= kTJ;
        ipar[m] = (a + j) & 1;                 // colour of node a in plane 0
        em[m] = (a >> 1) - (i0 / 2 - 4);       // entry of both nodes in their colour rows of the e box
        ob[m] = (long long)a + P * (long long)j;
    }
    // the residual pair: nodes ri, ri+1 of row rj; ri = 0 is a boundary node
    const int ri = i0 + 2 * tx, rj = j0 + ty;
    const bool rok = rj < n;
    const int hx = 2 * tx + 2, hy = ty + 1;
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
            const longlong2 uv = *reinterpret_cast<const longlong2*>(&ub[hj[m]][2 * hp[m]]);
            long long v0 = uv.x, v1 = uv.y;  // zero beyond the array (TMA fill), as for i or j > n
            if (qin && (inner0[m] || inner1[m])) {
                // node a has colour (a + j + q) & 1, node a+1 the other one
                const bool c0 = ((ipar[m] + q) & 1) != 0;
                const float ea = c0 ? e1[hj[m]][em[m]] : e0[hj[m]][em[m]];
                const float eb = c0 ? e0[hj[m]][em[m]] : e1[hj[m]][em[m]];
                if (inner0[m]) v0 += f32_to_i64(ea * scf);
                if (inner1[m]) v1 += f32_to_i64(eb * scf);
                if (own[m] && qown) *reinterpret_cast<longlong2*>(nxt + ob[m] + Q * q) = make_longlong2(v0, v1);
            }
            *reinterpret_cast<longlong2*>(&dst[hj[m]][2 * hp[m]]) = make_longlong2(v0, v1);
        }
        __syncthreads();
        const int kk = q - 1;
        if (kk >= kb && rok && ok) {
            const long long(*fb)[kTI] = reinterpret_cast<const long long(*)[kTI]>(&slot[(u - 1) % kSlots][0] + kOffF);
            const long long(*pm)[kW] = pl[(kk - 1) % 3];
            const long long(*p0)[kW] = pl[kk % 3];
            const long long(*pp)[kW] = pl[(kk + 1) % 3];
            const longlong2 w0 = *reinterpret_cast<const longlong2*>(&p0[hy][hx - 2]);
            const longlong2 w1 = *reinterpret_cast<const longlong2*>(&p0[hy][hx]);
            const longlong2 w2 = *reinterpret_cast<const longlong2*>(&p0[hy][hx + 2]);
            const longlong2 yn = *reinterpret_cast<const longlong2*>(&p0[hy - 1][hx]);
            const longlong2 ys = *reinterpret_cast<const longlong2*>(&p0[hy + 1][hx]);
            const longlong2 zm = *reinterpret_cast<const longlong2*>(&pm[hy][hx]);
            const longlong2 zp = *reinterpret_cast<const longlong2*>(&pp[hy][hx]);
            const longlong2 fv = *reinterpret_cast<const longlong2*>(&fb[ty][2 * tx]);
            // the same sums, in the same order, as the single-node form
            const long long s0 = (w1.y + w0.y) + (ys.x + yn.x) + (zp.x + zm.x) - 6 * w1.x;
            const long long s1 = (w2.x + w1.x) + (ys.y + yn.y) + (zp.y + zm.y) - 6 * w1.y;
            const long long rowb = ((long long)kk * (v.n + 1) + rj) * v.M + (ri >> 1);
            const int c = (ri + rj + kk) & 1;  // colour of node ri; ri + 1 has the other one
            if (ri >= 1) {
                const float R0 = i64_to_f32(fv.x - s0);
                r[(long long)c * v.cs + rowb] = R0 * k;
                const float Rs = R0 * kDown;
                rr = fmaf(Rs, Rs, rr);
            }
            {
                const float R1 = i64_to_f32(fv.y - s1);
                r[(long long)(c ^ 1) * v.cs + rowb] = R1 * k;
                const float Rs = R1 * kDown;
                rr = fmaf(Rs, Rs, rr);
            }
        }
        __syncthreads();  // slot of plane q-1 is free
        if (leader && q >= kb && q + kSlots - 1 <= ke) issue(q + kSlots - 1);
    }
    for (int off = 16; off > 0; off >>= 1) rr += __shfl_down_sync(0xffffffffu, rr, off);
    if ((tid & 31) == 0) sr[tid >> 5] = rr;
    __syncthreads();
    if (leader && *(volatile int*)&abort_flag) {
        // a wait gave up: copies issued earlier may still be landing in this CTA's shared memory, so wait
        // for every plane in [landed, issued) before exiting (bounded again; the fault is recorded)
        for (int q = landed; q < issued; ++q) {
            const int u = q - (kb - 1);
            long long spins = 0;
            while (!mbar_try_wait(&bar[u % kSlots], (unsigned)((u / kSlots) & 1)) && ++spins <= kSpinLimit) {
            }
        }
    }
    if (leader) {
        double a = 0.0;
        for (int q = 0; q < kPX * kTJ / 32; ++q) a += sr[q];
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

// rows of d0 elements, planes of d1 rows, d2 planes, d3 sets (strides s1, s2, s3 bytes); boxes b0 x b1 x 1 x 1
bool encode4(EncodeTiledFn enc, CUtensorMap* m, CUtensorMapDataType t, void* base, cuuint64_t d0, cuuint64_t d1,
             cuuint64_t d2, cuuint64_t d3, cuuint64_t s1, cuuint64_t s2, cuuint64_t s3, cuuint32_t b0, cuuint32_t b1)
{
    const cuuint64_t dims[4] = {d0, d1, d2, d3};
    const cuuint64_t strides[3] = {s1, s2, s3};
    const cuuint32_t box[4] = {b0, b1, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(m, t, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool make_fixed_maps(int64_t* U, int64_t* U2, int64_t* F, float* e, const LevelView& v, FixedMaps* out, int nsets)
{
    out->ok = false;
    const int n = v.n;
    if (n < kMinN) return false;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t rowb = (cuuint64_t)(n + 2) * 8, planeb = rowb * (n + 1), setb = planeb * (n + 1);
    const cuuint64_t erow = (cuuint64_t)v.M * 4, eplane = erow * (n + 1), eset = (cuuint64_t)(2 * v.cs) * 4;
    const cuuint64_t ns = (cuuint64_t)nsets;
    bool ok = encode4(enc, &out->u[0], CU_TENSOR_MAP_DATA_TYPE_INT64, U, n + 2, n + 1, n + 1, ns, rowb, planeb, setb,
                      kW, kH) &&
              encode4(enc, &out->u[1], CU_TENSOR_MAP_DATA_TYPE_INT64, U2, n + 2, n + 1, n + 1, ns, rowb, planeb, setb,
                      kW, kH) &&
              encode4(enc, &out->f, CU_TENSOR_MAP_DATA_TYPE_INT64, F, n + 2, n + 1, n + 1, ns, rowb, planeb, setb, kTI,
                      kTJ);
    for (int c = 0; ok && c < 2; ++c)
        ok = encode4(enc, &out->e[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, e + (long long)c * v.cs, v.M, n + 1, n + 1, ns,
                     erow, eplane, eset, kEW, kH);
    out->ok = ok;
    return ok;
}

int launch_fixed_update_residual_tma(int64_t* U, int64_t* U2, const FixedMaps& maps, int n, double h,
                                     const SolveState* st, float* r, const LevelView& v, double* partials, int* fault,
                                     cudaStream_t s, const Sets& sets)
{
    const int items = (n / kTI) * ((n - 1 + kTJ - 1) / kTJ) * ((n - 1 + kKC - 1) / kKC);
    fixed_update_residual_tma_kernel<<<dim3(items, sets.n), dim3(kPX, kTJ), 0, s>>>(
        maps.u[0], maps.u[1], maps.f, maps.e[0], maps.e[1], reinterpret_cast<long long*>(U),
        reinterpret_cast<long long*>(U2), n, (float)(1.0 / (h * h)), st, r, v, partials, fault, sets.pstride,
        sets.act ? 1 : 0);
    return items;
}

}  // namespace qumond
