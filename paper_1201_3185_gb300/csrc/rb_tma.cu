// Red-black half-sweep with TMA-staged neighbour planes (FP32 levels, n >= 64).
//
// Same update as rb_half_kernel -- every interior node of `colour` becomes
// (sum of its 6 other-colour neighbours - h^2 f) / 6 -- but organised for the
// memory system: a CTA owns a tile of 64 row entries (m) x 8 rows (j) of the
// colour-split level and walks a chunk of k-planes.  The other colour's
// planes k-1, k, k+1 (tile plus a one-row halo in j and the x-neighbours in m)
// are brought into shared memory by the tensor-memory accelerator, one 3-D box
// per plane, into a ring of four slots completed through mbarriers, so each
// other-colour value crosses HBM once and the six neighbour reads hit shared
// memory; f comes through the TMA unit with the same planes (both boxes
// complete one mbarrier) and the result is written straight to global memory.
// A thread updates four consecutive entries of a row (the parity of i is the
// same along a row): 16-byte shared-memory loads of the row and of its four
// neighbour rows, two scalars for the x-neighbours past the ends, and one
// 16-byte store, which keeps the kernel bound by memory rather than by
// instruction issue.
//
// The box starts at m0 - 4 so that its innermost coordinate is a multiple of
// 16 bytes; entries before row start (m0 = 0) are filled with zeros by the
// TMA unit and are never used by an interior node.  Waits are bounded: after
// kSpinLimit failed polls a CTA records a fault (reported by the solve as a
// timeout), issues no further copies, waits (bounded) for the copies already
// in flight, and finishes instead of hanging.
#include "qumond_internal.h"

namespace qumond {

namespace {

constexpr int kTM = 64;          // four consecutive row entries per thread: m0 + 4 tx .. m0 + 4 tx + 3
constexpr int kTJ = 8;
constexpr int kThreadsX = kTM / 4;
constexpr int kBoxX = kTM + 8;  // m0-4 .. m0+67
constexpr int kBoxY = kTJ + 2;  // j0-1 .. j0+8
constexpr int kSlots = 6;
constexpr int kKC = 16;  // planes per CTA
constexpr unsigned kPlaneBytes = kBoxX * kBoxY * sizeof(float);  // other colour, tile + halo
constexpr unsigned kFBytes = kTM * kTJ * sizeof(float);           // own right-hand side, tile
// TMA writes a box densely at a 128-byte aligned shared-memory address: pad each part.
constexpr int kPlaneFloats = ((kPlaneBytes + 127) / 128) * 128 / sizeof(float);
constexpr int kSlotFloats = kPlaneFloats + kFBytes / sizeof(float);
constexpr long long kSpinLimit = 1LL << 24;
// Levels below this size have too few planes per CTA column for the ring to pay off.
constexpr int kTmaMinN = 256;
constexpr int kTmaMinNSets = 128;  // with four or more sets in one launch

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

// One box of a 4-D tensor (m, j, k, set) into shared memory; the 4th
// coordinate selects the set of a context with several sets (0 for one set).
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// After a wait gave up, copies the leader issued may still be landing in this
// CTA's shared memory: before the CTA exits, the leader waits for every plane
// in [landed, issued) (bounded again; the fault is already recorded).  Only
// the leader issues, so its own progress bounds what is in flight.
__device__ __forceinline__ void drain_after_abort(bool leader, int* abort_flag, unsigned long long* bar, int first,
                                                  int landed, int issued)
{
    __syncthreads();
    if (!leader || !*(volatile int*)abort_flag) return;
    for (int q = landed; q < issued; ++q) {
        const int u = q - first;
        long long spins = 0;
        while (!mbar_try_wait(&bar[u % kSlots], (unsigned)((u / kSlots) & 1)) && ++spins <= kSpinLimit) {
        }
    }
}

__global__ void __launch_bounds__(kThreadsX * kTJ)
rb_tma_kernel(const __grid_constant__ CUtensorMap other_map, const __grid_constant__ CUtensorMap f_map,
              float* __restrict__ own, LevelView v, int colour, float h2, float sixth, int* __restrict__ fault,
              int zper, const SolveState* __restrict__ act)
{
    __shared__ __align__(128) float plane[kSlots][kSlotFloats];
    __shared__ __align__(8) unsigned long long bar[kSlots];
    __shared__ int abort_flag;
    // blockIdx.z = zper * set + chunk of planes
    const int set = (int)gridDim.z == zper ? 0 : (int)blockIdx.z / zper;
    if (act && !act[set].cont) return;  // this set's correction has stopped (whole CTA, before any barrier)
    own += (long long)set * 2 * v.cs;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m0 = blockIdx.x * kTM, j0 = 1 + blockIdx.y * kTJ;
    const int kb = 1 + ((int)blockIdx.z - set * zper) * kKC;
    const int ke = min(kb + kKC, v.n);  // output planes kb .. ke-1; planes kb-1 .. ke are read
    const bool leader = tx == 0 && ty == 0;
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
        float* dst = &plane[u % kSlots][0];
        float* fdst = dst + kPlaneFloats;
        if (((smem_u32(dst) | smem_u32(fdst)) & 127u) != 0u) {  // never issue a copy the TMA unit would reject
            atomicExch(fault, 2);
            atomicExch(&abort_flag, 1);
            return;
        }
        mbar_expect_tx(&bar[u % kSlots], kPlaneBytes + kFBytes);
        tma_load_4d(dst, &other_map, m0 - 4, j0 - 1, q, set, &bar[u % kSlots]);
        tma_load_4d(fdst, &f_map, m0, j0, q, set, &bar[u % kSlots]);
        issued = q + 1;
    };
    if (leader)
        for (int q = kb - 1; q < kb + kSlots - 1 && q <= ke; ++q) issue(q);
    bool ok = true;
    // lane 0 of each warp polls; __syncwarp passes the completed phase on to the warp
    const bool lane0 = ((tx + ty * kThreadsX) & 31) == 0;
    auto wait = [&](int q) {
        if (lane0) {
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
    const int j = j0 + ty;
    const int half = v.n >> 1;
    const long long plane_stride = (long long)(v.n + 1) * v.M;
    // per-thread constants: smem offsets of the four entries (box column 4 + 4 tx) and of their f, the
    // first entry, validity of each entry apart from the parity rule at m = 0
    const int c = (ty + 1) * kBoxX + 4 + 4 * tx;
    const int fo = kPlaneFloats + ty * kTM + 4 * tx;
    const int mA = m0 + 4 * tx;
    const bool rowok = j < v.n;
    bool ok4[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) ok4[e] = rowok && mA + e < half;
    long long row = ((long long)kb * (v.n + 1) + j) * v.M;
    int p = (colour + j + kb) & 1;
    int sm = 0, s0 = 1, sp = 2;  // slots of planes k-1, k, k+1
    for (int k = kb; k < ke; ++k) {
        if (k == kb) {
            wait(k - 1);
            wait(k);
        }
        wait(k + 1);
        const float* pm = &plane[sm][0];
        const float* p0 = &plane[s0][0];
        const float* pp = &plane[sp][0];
        if (rowok && mA < half) {
            const float4 V = *reinterpret_cast<const float4*>(p0 + c);
            const float x[6] = {p0[c - 1], V.x, V.y, V.z, V.w, p0[c + 4]};  // entries mA-1 .. mA+4
            const float4 Y0 = *reinterpret_cast<const float4*>(p0 + c - kBoxX);
            const float4 Y1 = *reinterpret_cast<const float4*>(p0 + c + kBoxX);
            const float4 Zm = *reinterpret_cast<const float4*>(pm + c);
            const float4 Zp = *reinterpret_cast<const float4*>(pp + c);
            const float4 F = *reinterpret_cast<const float4*>(p0 + fo);
            const float y0[4] = {Y0.x, Y0.y, Y0.z, Y0.w}, y1[4] = {Y1.x, Y1.y, Y1.z, Y1.w};
            const float zm[4] = {Zm.x, Zm.y, Zm.z, Zm.w}, zp[4] = {Zp.x, Zp.y, Zp.z, Zp.w};
            const float fv[4] = {F.x, F.y, F.z, F.w};
            float r[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                // x-neighbours: entries m-1+p and m+p
                const float lo = p ? x[e + 1] : x[e];
                const float hi = p ? x[e + 2] : x[e + 1];
                const float sum = (lo + hi) + (y0[e] + y1[e]) + (zm[e] + zp[e]);
                r[e] = (sum - h2 * fv[e]) * sixth;
            }
            // i = 2m + p must lie in 1 .. n-1: only the row's first entry (m = 0, p = 0) is a boundary node
            const bool first = p == 0 && mA == 0;
            if (!first && ok4[3])
                *reinterpret_cast<float4*>(own + row + mA) = make_float4(r[0], r[1], r[2], r[3]);
            else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (ok4[e] && !(first && e == 0)) own[row + mA + e] = r[e];
            }
        }
        __syncthreads();  // slot of plane k-1 is free
        if (leader && k + kSlots - 1 <= ke) issue(k + kSlots - 1);
        row += plane_stride;
        p ^= 1;
        const int t = sm;
        sm = s0;
        s0 = sp;
        sp = t + 3 < kSlots ? t + 3 : t + 3 - kSlots;  // slot of plane k+2 = (slot of k-1) + 3
    }
    drain_after_abort(leader, &abort_flag, bar, kb - 1, landed, issued);
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

}  // namespace

bool make_rb_maps(float* e, float* f, const LevelView& v, RbMaps* out, int nsets)
{
    out->ok = false;
    // one set: only levels with enough planes per CTA column to fill the GPU; several sets fill it together
    if (v.n < (nsets >= 4 ? kTmaMinNSets : kTmaMinN)) return false;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)v.M, (cuuint64_t)(v.n + 1), (cuuint64_t)(v.n + 1), (cuuint64_t)nsets};
    const cuuint64_t strides[3] = {(cuuint64_t)v.M * sizeof(float), (cuuint64_t)v.M * (v.n + 1) * sizeof(float),
                                   (cuuint64_t)(2 * v.cs) * sizeof(float)};
    const cuuint32_t box[4] = {kBoxX, kBoxY, 1, 1};
    const cuuint32_t fbox[4] = {kTM, kTJ, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int c = 0; c < 2; ++c) {
        if (enc(&out->map[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, e + (long long)c * v.cs, dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
        if (enc(&out->fmap[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, f + (long long)c * v.cs, dims, strides, fbox, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    out->ok = true;
    return true;
}

void launch_rb_half_tma(float* e, const float* f, const LevelView& v, int colour, const RbMaps& maps, double h,
                        int* fault, cudaStream_t s, const Sets& sets)
{
    const int zper = (v.n - 1 + kKC - 1) / kKC;
    const dim3 grid((unsigned)((v.n / 2 + kTM - 1) / kTM), (unsigned)((v.n - 1 + kTJ - 1) / kTJ),
                    (unsigned)(zper * sets.n));
    (void)f;
    rb_tma_kernel<<<grid, dim3(kThreadsX, kTJ), 0, s>>>(maps.map[colour ^ 1], maps.fmap[colour], e + (long long)colour * v.cs,
                                                  v, colour, (float)(h * h), 1.0f / 6.0f, fault, zper, sets.act);
}

}  // namespace qumond
