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

// ---------------------------------------------------------------------------
// Restriction of the red residuals (after a black half-sweep the black
// residuals vanish) onto the coarse level, with the fine planes staged by the
// TMA unit.  A CTA owns a tile of 32 x 8 coarse (I, J) columns and up to 8
// coarse planes K0 .. K1-1, and walks the fine planes 2K0-2 .. 2K1: for each,
// three boxes land in a five-slot ring completed by one mbarrier -- the black
// entries mbase-4 .. mbase+39 of the fine rows 2J0-2 .. 2J0+16 (mbase = I0-1,
// a multiple of 32), and the red entries and f of the red rows 2J0-1 ..
// 2J0+15, entries mbase .. mbase+35.  The red residuals of fine plane k are
// computed from the black planes k-1, k, k+1 of the ring (four consecutive
// entries per thread, red_residual's arithmetic in its order) into a
// three-plane residual ring; after each odd plane 2K+1 the coarse plane K is
// full-weighted from it with restrict_node's sums in their order.  Each fine
// value crosses HBM once and the loads of three planes are in flight while
// one is processed.  Boxes outside the level read zeros; they only feed
// residuals that no coarse interior node uses.  Waits are bounded as in the
// half-sweep.
constexpr int kRTI = 32, kRTJ = 8, kRTK = 8;  // coarse tile, the most coarse planes per CTA
constexpr int kRBX = 44, kRBY = 2 * kRTJ + 3;  // black box: 44 entries x 19 rows
constexpr int kRRX = 36, kRRY = 2 * kRTJ + 1;  // red and f boxes: 36 entries x 17 rows
constexpr int kRG = kRRX / 4;                  // groups of four red entries per fine row
constexpr int kRBlackFloats = ((kRBX * kRBY * 4 + 127) / 128) * 128 / 4;
constexpr int kRRedFloats = ((kRRX * kRRY * 4 + 127) / 128) * 128 / 4;
constexpr int kRSlotFloats = kRBlackFloats + 2 * kRRedFloats;
constexpr int kRSlots = 5;
constexpr unsigned kRPlaneBytes = (kRBX * kRBY + 2 * kRRX * kRRY) * 4;
constexpr size_t kRSmemBytes = sizeof(float) * ((size_t)kRSlots * kRSlotFloats + 3 * kRRY * kRRX);
static_assert(kRRY * kRG <= kRTI * kRTJ, "one thread per residual group");
static_assert((kRBX * 4) % 16 == 0 && (kRRX * 4) % 16 == 0, "box rows are whole 16-byte units");

__device__ __forceinline__ void restrict_drain(bool leader, int* abort_flag, unsigned long long* bar, int first,
                                               int landed, int issued)
{
    __syncthreads();
    if (!leader || !*(volatile int*)abort_flag) return;
    for (int q = landed; q < issued; ++q) {
        const int u = q - first;
        long long spins = 0;
        while (!mbar_try_wait(&bar[u % kRSlots], (unsigned)((u / kRSlots) & 1)) && ++spins <= kSpinLimit) {
        }
    }
}

__global__ void __launch_bounds__(kRTI * kRTJ)
restrict_tma_kernel(const __grid_constant__ CUtensorMap black_map, const __grid_constant__ CUtensorMap red_map,
                    const __grid_constant__ CUtensorMap f_map, float* __restrict__ fc, LevelView vf, LevelView vc,
                    float ih2, int* __restrict__ fault, int zper, const SolveState* __restrict__ act)
{
    extern __shared__ __align__(128) float rsm[];
    float(*ring)[kRRY][kRRX] = reinterpret_cast<float(*)[kRRY][kRRX]>(rsm + kRSlots * kRSlotFloats);
    __shared__ __align__(8) unsigned long long bar[kRSlots];
    __shared__ int abort_flag;
    const int set = (int)gridDim.z == zper ? 0 : (int)blockIdx.z / zper;
    if (act && !act[set].cont) return;  // this set's correction has stopped (whole CTA, before any barrier)
    fc += (long long)set * 2 * vc.cs;
    const int n = vf.n, nc = vc.n;
    const int I0 = 1 + blockIdx.x * kRTI, J0 = 1 + blockIdx.y * kRTJ;
    const int K0 = 1 + ((int)blockIdx.z - set * zper) * kRTK;
    const int K1 = min(K0 + kRTK, nc);  // coarse planes K0 .. K1-1
    const int mbase = I0 - 1;           // a multiple of 32
    const int jb = 2 * J0 - 2;          // first black row of the box; the red rows start at jb + 1
    const int first = 2 * K0 - 2, last = 2 * K1;  // fine planes staged
    const int t = threadIdx.x;
    const bool leader = t == 0;
    if (leader) {
        abort_flag = 0;
        for (int q = 0; q < kRSlots; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int issued = first, landed = first;
    auto slot_of = [&](int q) { return rsm + ((q - first) % kRSlots) * kRSlotFloats; };
    auto issue = [&](int q) {  // plane q into its slot (leader only); nothing more once a wait gave up
        if (*(volatile int*)&abort_flag) return;
        const int u = q - first;
        float* base = rsm + (u % kRSlots) * kRSlotFloats;
        if (((smem_u32(base) | smem_u32(base + kRBlackFloats) | smem_u32(base + kRBlackFloats + kRRedFloats)) &
             127u) != 0u) {  // never issue a copy the TMA unit would reject
            atomicExch(fault, 2);
            atomicExch(&abort_flag, 1);
            return;
        }
        unsigned long long* b = &bar[u % kRSlots];
        mbar_expect_tx(b, kRPlaneBytes);
        tma_load_4d(base, &black_map, mbase - 4, jb, q, set, b);  // x: a multiple of 4 floats
        tma_load_4d(base + kRBlackFloats, &red_map, mbase, jb + 1, q, set, b);
        tma_load_4d(base + kRBlackFloats + kRRedFloats, &f_map, mbase, jb + 1, q, set, b);
        issued = q + 1;
    };
    if (leader)
        for (int q = first; q < first + kRSlots && q <= last; ++q) issue(q);
    bool ok = true;
    const bool lane0 = (t & 31) == 0;
    auto wait = [&](int q) {
        if (lane0) {
            const int u = q - first;
            long long spins = 0;
            while (ok && !mbar_try_wait(&bar[u % kRSlots], (unsigned)((u / kRSlots) & 1))) {
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
    // residual phase: red row rr (fine row jb + 1 + rr), group rg (entries mbase + 4 rg .. + 3)
    const int rr = t / kRG, rg = t % kRG;
    const int jf = jb + 1 + rr;
    const bool ract = t < kRRY * kRG && jf >= 1 && jf <= n - 1 && mbase + 4 * rg < vf.M;
    const int cb = (rr + 1) * kRBX + 4 + 4 * rg;  // black box index of entry mbase + 4 rg in the same row
    const int cr = rr * kRRX + 4 * rg;            // red / f box index
    // coarse phase: node (I, J)
    const int cI = t % kRTI, cJ = t / kRTI;
    const int I = I0 + cI, J = J0 + cJ;
    const bool cact = I <= nc - 1 && J <= nc - 1;
    for (int k = first + 1; k <= last - 1; ++k) {
        if (k == first + 1) {
            wait(first);
            wait(first + 1);
        }
        wait(k + 1);
        if (ract) {
            const float* bm = slot_of(k - 1);
            const float* b0 = slot_of(k);
            const float* bp = slot_of(k + 1);
            const float* red = b0 + kRBlackFloats;
            const float* fr = red + kRRedFloats;
            const int p = (jf + k) & 1;
            const float4 V = *reinterpret_cast<const float4*>(b0 + cb);
            const float x[6] = {b0[cb - 1], V.x, V.y, V.z, V.w, b0[cb + 4]};
            const float4 Y0 = *reinterpret_cast<const float4*>(b0 + cb - kRBX);
            const float4 Y1 = *reinterpret_cast<const float4*>(b0 + cb + kRBX);
            const float4 Z0 = *reinterpret_cast<const float4*>(bm + cb);
            const float4 Z1 = *reinterpret_cast<const float4*>(bp + cb);
            const float4 E = *reinterpret_cast<const float4*>(red + cr);
            const float4 F = *reinterpret_cast<const float4*>(fr + cr);
            const float y0[4] = {Y0.x, Y0.y, Y0.z, Y0.w}, y1[4] = {Y1.x, Y1.y, Y1.z, Y1.w};
            const float z0[4] = {Z0.x, Z0.y, Z0.z, Z0.w}, z1[4] = {Z1.x, Z1.y, Z1.z, Z1.w};
            const float ev[4] = {E.x, E.y, E.z, E.w}, fv[4] = {F.x, F.y, F.z, F.w};
            float r[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float lo = p ? x[e + 1] : x[e];
                const float hi = p ? x[e + 2] : x[e + 1];
                const float sum = (lo + hi) + (y0[e] + y1[e]) + (z0[e] + z1[e]);
                r[e] = fv[e] - (sum - 6.0f * ev[e]) * ih2;
            }
            *reinterpret_cast<float4*>(&ring[k % 3][rr][4 * rg]) = make_float4(r[0], r[1], r[2], r[3]);
        }
        __syncthreads();
        if ((k & 1) && k >= 2 * K0 + 1 && cact && ok) {
            const int K = (k - 1) >> 1;
            const float(*pm)[kRRX] = ring[(k + 1) % 3];  // fine plane 2K-1
            const float(*p0)[kRRX] = ring[(k + 2) % 3];  // 2K
            const float(*pp)[kRRX] = ring[k % 3];        // 2K+1
            // fine node (i, j) = (2I, 2J): row 2cJ+1 of the tile; entries I-1 (i-1) and I (i, i+1)
            const int a = 2 * cJ + 1, lo = cI, hi = cI + 1;
            float edge = (p0[a + 1][hi] + p0[a + 1][lo]) + (p0[a - 1][hi] + p0[a - 1][lo]);
            edge += (pp[a][hi] + pp[a][lo]) + (pm[a][hi] + pm[a][lo]);
            edge += (pp[a + 1][hi] + pp[a - 1][hi]) + (pm[a + 1][hi] + pm[a - 1][hi]);
            const float centre = p0[a][hi];
            fc[node_off(vc, I, J, K)] = 0.125f * centre + 0.03125f * edge;
        }
        __syncthreads();  // the slot of plane k-1 is free
        if (leader && k + kRSlots - 1 <= last) issue(k + kRSlots - 1);
    }
    restrict_drain(leader, &abort_flag, bar, first, landed, issued);
}

// ---------------------------------------------------------------------------
// The coarse-grid correction of the black nodes of a fine level with TMA maps
// (prolong_black4_kernel's arithmetic, add), the planes staged by the TMA
// unit.  A CTA owns 64 black entries x 8 rows of the fine level (four entries
// per thread, 16 x 8 threads) and walks a chunk of 16 fine planes.  The slot
// of fine plane q holds the CTA's black tile of plane q and both colours of the
// coarse plane (q+1)/2 (entries m0/2 .. m0/2+35 of the coarse rows j0/2 ..
// j0/2+4); fine plane k interpolates from coarse planes k/2 and (k+1)/2, held
// by the slots of planes k-1 and k, so the ring starts one plane early.  The
// black values are read once through the TMA unit and written back with
// 16-byte stores; waits are bounded as in the half-sweep.
constexpr int kPTM = 64, kPTJ = 8, kPKC = 16;  // fine tile (black entries x rows), planes per CTA
constexpr int kPCX = 36, kPCY = kPTJ / 2 + 1;  // coarse box per colour: 36 entries x 5 rows
constexpr int kPFineFloats = kPTM * kPTJ;      // 512 floats = 2048 bytes
constexpr int kPCoarseFloats = ((kPCX * kPCY * 4 + 127) / 128) * 128 / 4;
constexpr int kPSlotFloats = kPFineFloats + 2 * kPCoarseFloats;
constexpr int kPSlots = 4;
constexpr unsigned kPPlaneBytes = (kPTM * kPTJ + 2 * kPCX * kPCY) * 4;
static_assert((kPFineFloats * 4) % 128 == 0 && (kPCoarseFloats * 4) % 128 == 0, "slot parts 128-byte aligned");

__global__ void __launch_bounds__((kPTM / 4) * kPTJ)
prolong_tma_kernel(const __grid_constant__ CUtensorMap fine_map, const __grid_constant__ CUtensorMap c0_map,
                   const __grid_constant__ CUtensorMap c1_map, float* __restrict__ ef, LevelView vf, int* __restrict__ fault,
                   int zper, const SolveState* __restrict__ act)
{
    __shared__ __align__(128) float slotm[kPSlots][kPSlotFloats];
    __shared__ __align__(8) unsigned long long bar[kPSlots];
    __shared__ int abort_flag;
    const int set = (int)gridDim.z == zper ? 0 : (int)blockIdx.z / zper;
    if (act && !act[set].cont) return;  // this set's correction has stopped (whole CTA, before any barrier)
    ef += (long long)set * 2 * vf.cs;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m0 = blockIdx.x * kPTM, j0 = 1 + blockIdx.y * kPTJ;
    const int kb = 1 + ((int)blockIdx.z - set * zper) * kPKC;
    const int ke = min(kb + kPKC, vf.n);  // fine planes kb .. ke-1; planes kb-1 .. ke-1 are staged
    const int first = kb - 1;
    const int Jb = j0 >> 1, cx0 = m0 >> 1;
    const bool leader = tx == 0 && ty == 0;
    if (leader) {
        abort_flag = 0;
        for (int q = 0; q < kPSlots; ++q) mbar_init(&bar[q], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int issued = first, landed = first;
    auto issue = [&](int q) {  // plane q into its slot (leader only); nothing more once a wait gave up
        if (*(volatile int*)&abort_flag) return;
        const int u = q - first;
        float* base = &slotm[u % kPSlots][0];
        if (((smem_u32(base) | smem_u32(base + kPFineFloats) | smem_u32(base + kPFineFloats + kPCoarseFloats)) &
             127u) != 0u) {  // never issue a copy the TMA unit would reject
            atomicExch(fault, 2);
            atomicExch(&abort_flag, 1);
            return;
        }
        unsigned long long* b = &bar[u % kPSlots];
        mbar_expect_tx(b, kPPlaneBytes);
        tma_load_4d(base, &fine_map, m0, j0, q, set, b);  // x: a multiple of 64 floats
        tma_load_4d(base + kPFineFloats, &c0_map, cx0, Jb, (q + 1) >> 1, set, b);  // x: a multiple of 32 floats
        tma_load_4d(base + kPFineFloats + kPCoarseFloats, &c1_map, cx0, Jb, (q + 1) >> 1, set, b);
        issued = q + 1;
    };
    if (leader)
        for (int q = first; q < first + kPSlots && q <= ke - 1; ++q) issue(q);
    bool ok = true;
    const bool lane0 = ((tx + ty * (kPTM / 4)) & 31) == 0;
    auto wait = [&](int q) {
        if (lane0) {
            const int u = q - first;
            long long spins = 0;
            while (ok && !mbar_try_wait(&bar[u % kPSlots], (unsigned)((u / kPSlots) & 1))) {
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
    const int half = vf.n >> 1;
    const int j = j0 + ty;
    const int mA = m0 + 4 * tx;
    const bool act4 = j < vf.n && mA < half;
    const int J0 = j >> 1, J1 = (j + 1) >> 1;
    for (int k = kb; k < ke; ++k) {
        if (k == kb) wait(k - 1);
        wait(k);
        if (act4) {
            const int p = (1 + j + k) & 1;  // parity of i of the black nodes in this row
            const int K0 = k >> 1, K1 = (k + 1) >> 1;
            // coarse plane K is carried by the slot of fine plane 2K-1 or 2K: K1 by plane k, K0 by plane k-1
            const float* s1 = &slotm[(k - first) % kPSlots][0];
            const float* s0 = K0 == K1 ? s1 : &slotm[(k - 1 - first) % kPSlots][0];
            auto row5 = [&](int Jr, const float* sl, int Kr, float* cc) {
                const int ca = (mA + Jr + Kr) & 1;  // colour of the even d
                const int base = (Jr - Jb) * kPCX + ((mA >> 1) - cx0);
                const float* A = sl + kPFineFloats + ca * kPCoarseFloats + base;
                const float* B = sl + kPFineFloats + (ca ^ 1) * kPCoarseFloats + base;
                const float2 a2 = *reinterpret_cast<const float2*>(A);
                const float2 b2 = *reinterpret_cast<const float2*>(B);
                cc[0] = a2.x, cc[1] = b2.x, cc[2] = a2.y, cc[3] = b2.y, cc[4] = A[2];
            };
            float c00[5], c10[5], c01[5], c11[5];  // (J0, K0), (J1, K0), (J0, K1), (J1, K1)
            row5(J0, s0, K0, c00);
            row5(J1, s0, K0, c10);
            row5(J0, s1, K1, c01);
            row5(J1, s1, K1, c11);
            const float4 cur = *reinterpret_cast<const float4*>(s1 + ty * kPTM + 4 * tx);
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
                r[e] = cv[e] + sv;
            }
            float* o = ef + vf.cs + ((long long)k * (vf.n + 1) + j) * vf.M + mA;
            if (p == 0 && mA == 0) {  // i = 0 is a boundary node
                o[1] = r[1], o[2] = r[2], o[3] = r[3];
            } else {
                *reinterpret_cast<float4*>(o) = make_float4(r[0], r[1], r[2], r[3]);
            }
        }
        __syncthreads();  // the slot of plane k-1 is free
        if (leader && k - 1 + kPSlots <= ke - 1) issue(k - 1 + kPSlots);
    }
    // drain after a fault, as in the half-sweep
    __syncthreads();
    if (leader && *(volatile int*)&abort_flag)
        for (int q = landed; q < issued; ++q) {
            const int u = q - first;
            long long spins = 0;
            while (!mbar_try_wait(&bar[u % kPSlots], (unsigned)((u / kPSlots) & 1)) && ++spins <= kSpinLimit) {
            }
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
    const cuuint32_t bbox[4] = {kRBX, kRBY, 1, 1};
    const cuuint32_t rbox[4] = {kRRX, kRRY, 1, 1};
    auto enc1 = [&](CUtensorMap* m, float* base, const cuuint32_t* bx) {
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, bx, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    // the restriction's boxes: black iterate with halo, red iterate, red right-hand side
    if (!enc1(&out->rmap_black, e + v.cs, bbox) || !enc1(&out->rmap_red, e, rbox) || !enc1(&out->rmap_f, f, rbox))
        return false;
    if (cudaFuncSetAttribute(restrict_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRSmemBytes) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
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

bool make_prolong_maps(float* ec, const LevelView& vc, float* ef, const LevelView& vf, RbMaps* out, int nsets)
{
    out->pok = false;
    if (!out->ok || vf.n != 2 * vc.n || (vc.M & 3) != 0) return false;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    auto enc1 = [&](CUtensorMap* m, float* base, const LevelView& v, cuuint32_t bx, cuuint32_t by) {
        const cuuint64_t dims[4] = {(cuuint64_t)v.M, (cuuint64_t)(v.n + 1), (cuuint64_t)(v.n + 1), (cuuint64_t)nsets};
        const cuuint64_t strides[3] = {(cuuint64_t)v.M * sizeof(float), (cuuint64_t)v.M * (v.n + 1) * sizeof(float),
                                       (cuuint64_t)(2 * v.cs) * sizeof(float)};
        const cuuint32_t box[4] = {bx, by, 1, 1};
        return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    if (!enc1(&out->pmap_fine, ef + vf.cs, vf, kPTM, kPTJ) || !enc1(&out->pmap_c[0], ec, vc, kPCX, kPCY) ||
        !enc1(&out->pmap_c[1], ec + vc.cs, vc, kPCX, kPCY))
        return false;
    out->pok = true;
    return true;
}

void launch_prolong_tma(float* ef, const LevelView& vf, const RbMaps& maps, int* fault, cudaStream_t s,
                        const Sets& sets)
{
    const int zper = (vf.n - 1 + kPKC - 1) / kPKC;
    const dim3 grid((unsigned)((vf.n / 2 + kPTM - 1) / kPTM), (unsigned)((vf.n - 1 + kPTJ - 1) / kPTJ),
                    (unsigned)(zper * sets.n));
    prolong_tma_kernel<<<grid, dim3(kPTM / 4, kPTJ), 0, s>>>(maps.pmap_fine, maps.pmap_c[0], maps.pmap_c[1], ef, vf,
                                                             fault, zper, sets.act);
}

void launch_restrict_tma(float* fc, const LevelView& vf, const LevelView& vc, const RbMaps& maps, double hf,
                         int* fault, cudaStream_t s, const Sets& sets)
{
    const int zper = (vc.n - 1 + kRTK - 1) / kRTK;
    const dim3 grid((unsigned)((vc.n - 1 + kRTI - 1) / kRTI), (unsigned)((vc.n - 1 + kRTJ - 1) / kRTJ),
                    (unsigned)(zper * sets.n));
    restrict_tma_kernel<<<grid, kRTI * kRTJ, kRSmemBytes, s>>>(maps.rmap_black, maps.rmap_red, maps.rmap_f, fc, vf, vc,
                                                              (float)(1.0 / (hf * hf)), fault, zper, sets.act);
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
