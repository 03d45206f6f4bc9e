// The U-Net's 3^3 convolution on the fifth-generation tensor cores
// (tcgen05): an implicit GEMM with M = 128 output voxels, N = up to 64 output
// channels, K = 27 taps x 16 input channels per chunk, accumulated in tensor
// memory (TMEM) and read back by the four warps for the epilogue.
//
// Layout trick: the input brick of a CTA is 1 x 16 x 8 voxels (z, y, x) and
// its halo 3 x 18 x 10; the halo of a 16-channel chunk is kept in shared
// memory as two planes (channels 0-7 and 8-15), 16 bytes per voxel.  Eight
// consecutive voxels of an x-row are then one 8 x 16-byte core matrix of the
// canonical K-major layout, the sixteen y-rows are core matrices a constant
// 160 bytes apart, and the two channel halves a plane apart, so the A operand
// of every tap is a shared-memory descriptor into the same halo (no im2col
// copy).  The weights of the chunk are stored per tap as [channel half]
// [output channel][8 channels].  One thread issues the 27 MMAs of a chunk and
// commits them to an mbarrier; the CTA waits (bounded) before it overwrites
// the chunk's shared memory.
//
// The shared-memory descriptors follow the PTX ISA's canonical K-major layout
// without swizzling: core matrices of 8 rows x 16 bytes, the leading-dimension
// byte offset (bits 16-29) the distance between core matrices adjacent along
// K, the stride-dimension byte offset (bits 32-45) the distance between
// 8-row groups along M (or N).  tc_selftest checks one MMA with that encoding
// against a CPU product (a unit test; the product path does not call it).
#include "unet_internal.h"

#include <cstdio>
#include <cstring>
#include <vector>

namespace qumond {
namespace unet {

namespace {

constexpr int kHX = 10, kHY = 18, kHZ = 3;  // halo of a 1 x 16 x 8 brick
constexpr int kHV = kHX * kHY * kHZ;        // 540 halo voxels
constexpr unsigned kPlaneBytes = kHV * 16;  // one channel half of the halo
constexpr long long kSpinLimit = 1LL << 24;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major, no swizzle: start address >> 4 in
// bits 0-13; leading-dimension byte offset >> 4 (between core matrices along
// K) in bits 16-29; stride-dimension byte offset >> 4 (between 8-row groups
// along M or N) in bits 32-45; the descriptor version (1) at bit 46; base
// offset 0, swizzle mode 0 (bits 61-63).
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned kstride, unsigned mnstride)
{
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((kstride >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((mnstride >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, N and M
__host__ __device__ constexpr unsigned idesc_bf16(int N, int M)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
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

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// bounded wait on an mbarrier phase: gives up after kSpinLimit polls or about a second, whichever comes first;
// false (and *fault = 3) when it gave up
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* fault)
{
    long long spins = 0;
    unsigned long long t0 = 0;
    while (!mbar_try_wait(bar, parity)) {
        ++spins;
        if ((spins & 1023) == 0) {
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            else if (now - t0 > 1000000000ull) spins = kSpinLimit + 1;
        }
        if (spins > kSpinLimit) {
            if (fault) atomicExch(fault, 3);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc, int acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void commit(unsigned long long* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float* v)
{
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// ---------------------------------------------------------------------------
// Self-test: D (128 x 16) = A (128 x 16) B^T (16 x 16) for small integer
// operands, A and B in a compact canonical layout (core matrix (g, h) of rows
// 8g.. and K-columns 8h.. at g*256 + h*128 bytes), read back from TMEM.  Every
// address the descriptors form lies inside A or B.
__global__ void __launch_bounds__(128) tc_selftest_kernel(float* out, int* fault)
{
    __shared__ __align__(128) __nv_bfloat16 A[128 * 16];
    __shared__ __align__(128) __nv_bfloat16 B[16 * 16];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int e = tid; e < 128 * 16; e += 128) {
        const int m = e / 16, k = e % 16;
        A[(m / 8) * 128 + (k / 8) * 64 + (m % 8) * 8 + (k % 8)] = __float2bfloat16_rn((float)((m + 3 * k) % 7 - 3));
    }
    for (int e = tid; e < 16 * 16; e += 128) {
        const int n = e / 16, k = e % 16;
        B[(n / 8) * 128 + (k / 8) * 64 + (n % 8) * 8 + (k % 8)] = __float2bfloat16_rn((float)((2 * n + k) % 5 - 2));
    }
    if (warp == 0) tmem_alloc(&slot, 32);
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_proxy();
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned taddr = slot;
    if (tid == 0) {
        mma(taddr, sdesc(smem_u32(A), 128, 256), sdesc(smem_u32(B), 128, 256), idesc_bf16(16, 128), 0);
        commit(&bar);
    }
    const bool ok = mbar_wait(&bar, 0, fault);
    fence_after();
    float v[16];
    tmem_ld16(taddr + ((unsigned)(warp * 32) << 16), v);
    for (int q = 0; q < 16; ++q) out[(warp * 32 + lane) * 16 + q] = ok ? v[q] : __int_as_float(0x7fc00000);
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, 32);
}

}  // namespace

// ---------------------------------------------------------------------------
template <int NT>
__global__ void __launch_bounds__(128) conv3_tc_kernel(ConvArgs a)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(smem_raw);                     // 2 planes x kHV x 8
    __nv_bfloat16* wts = reinterpret_cast<__nv_bfloat16*>(smem_raw + 2 * kPlaneBytes);     // 27 x 2 x NT x 8
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned slot;
    constexpr unsigned kCols = NT <= 32 ? 32 : 64;
    constexpr unsigned kIdesc = idesc_bf16(NT, 128);

    const int S = a.S;
    const int nbx = S / 8, nby = S / 16;
    const int brick = blockIdx.x;
    const int x0 = (brick % nbx) * 8, y0 = ((brick / nbx) % nby) * 16, z0 = brick / (nbx * nby);
    const int co0 = blockIdx.y * NT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) tmem_alloc(&slot, kCols);
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned taddr = slot;
    const unsigned hbase = smem_u32(halo), wbase = smem_u32(wts);
    bool ok = true;
    const int nchunks = a.cin / 16;
    for (int c = 0; c < nchunks; ++c) {
        const int ci0 = c * 16;
        // the chunk's halo: voxel hv -> planes 0 and 1 (channels ci0..ci0+7, ci0+8..ci0+15)
        for (int q = tid; q < kHV * 2; q += 128) {
            const int hv = q >> 1, part = q & 1;
            const int ix = hv % kHX, iy = (hv / kHX) % kHY, iz = hv / (kHX * kHY);
            const int gx = x0 + ix - 1, gy = y0 + iy - 1, gz = z0 + iz - 1;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (gx >= 0 && gx < S && gy >= 0 && gy < S && gz >= 0 && gz < S) {
                const long long v = ((long long)gz * S + gy) * S + gx;
                val = *reinterpret_cast<const uint4*>(a.in + v * a.ld_in + a.in_off + ci0 + part * 8);
            }
            *reinterpret_cast<uint4*>(halo + ((size_t)part * kHV + hv) * 8) = val;
        }
        // the chunk's weights: W[co0 + n][t][ci0 + 8 part ..] -> wts[(t * 2 + part) * NT + n]
        for (int q = tid; q < 27 * 2 * NT; q += 128) {
            const int n = q % NT, part = (q / NT) & 1, t = q / (2 * NT);
            const uint4 val =
                *reinterpret_cast<const uint4*>(a.w + ((long long)(co0 + n) * 27 + t) * a.cin + ci0 + part * 8);
            *reinterpret_cast<uint4*>(wts + ((size_t)(t * 2 + part) * NT + n) * 8) = val;
        }
        fence_proxy();
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0 && ok) {
#pragma unroll 1
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;  // halo offsets 0..2 of the tap
                const unsigned aoff = (unsigned)(((dz * kHY + dy) * kHX + dx) * 16);
                const unsigned long long ad = sdesc(hbase + aoff, kPlaneBytes, kHX * 16);
                const unsigned long long bd = sdesc(wbase + (unsigned)(t * 2 * NT * 16), NT * 16, 128);
                mma(taddr, ad, bd, kIdesc, (c > 0 || t > 0) ? 1 : 0);
            }
            commit(&bar);
        }
        // the MMAs have read this chunk's shared memory once the commit arrives
        if (ok) ok = mbar_wait(&bar, (unsigned)(c & 1), a.fault);
        fence_after();
    }
    // epilogue: warp w holds TMEM lanes 32w..32w+31 = brick voxels 32w + lane
    const int m = warp * 32 + lane;
    const int ly = m / 8, lx = m % 8;
    const long long v = ((long long)z0 * S + (y0 + ly)) * S + (x0 + lx);
#pragma unroll
    for (int c0 = 0; c0 < NT; c0 += 16) {
        float r[16];
        tmem_ld16(taddr + ((unsigned)(warp * 32) << 16) + (unsigned)c0, r);
        if (!ok) continue;
        const int co = co0 + c0;
        __nv_bfloat16 h[16];
        __nv_bfloat16 mk[16];
        if (a.mask) {
            const uint4* mp = reinterpret_cast<const uint4*>(a.mask + v * a.ld_mask + a.mask_off + co);
            *reinterpret_cast<uint4*>(&mk[0]) = mp[0];
            *reinterpret_cast<uint4*>(&mk[8]) = mp[1];
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float x = r[q];
            if (a.bias) x += a.bias[co + q];
            if (a.relu) x = fmaxf(x, 0.0f);
            if (a.mask && !(__bfloat162float(mk[q]) > 0.0f)) x = 0.0f;
            h[q] = __float2bfloat16_rn(x);
        }
        uint4* dst = reinterpret_cast<uint4*>(a.out + v * a.ld_out + a.out_off + co);
        dst[0] = *reinterpret_cast<uint4*>(&h[0]);
        dst[1] = *reinterpret_cast<uint4*>(&h[8]);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, kCols);
}

size_t conv3_tc_smem_bytes(int nt) { return (size_t)2 * kPlaneBytes + (size_t)27 * 2 * nt * 16; }

bool conv3_tc_applies(const ConvArgs& a)
{
    // 16 <= S (the 1 x 16 x 8 brick), channel counts in 16-channel chunks, row strides and offsets in
    // 16-byte units (8 channels) for the vector loads and stores
    return a.use_tc && a.S >= 16 && a.S % 16 == 0 && a.cin % 16 == 0 && a.cout % 16 == 0 &&
           a.ld_in % 8 == 0 && a.in_off % 8 == 0 && a.ld_out % 8 == 0 && a.out_off % 8 == 0 &&
           (!a.mask || (a.ld_mask % 8 == 0 && a.mask_off % 8 == 0));
}

void prepare_conv3_tc()
{
    cudaFuncSetAttribute(conv3_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv3_tc_smem_bytes(16));
    cudaFuncSetAttribute(conv3_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv3_tc_smem_bytes(32));
    cudaFuncSetAttribute(conv3_tc_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv3_tc_smem_bytes(48));
    cudaFuncSetAttribute(conv3_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)conv3_tc_smem_bytes(64));
}

void launch_conv3_tc(const ConvArgs& a, cudaStream_t s)
{
    const int nt = conv3_tile(a.cout);
    const dim3 grid((unsigned)((a.S / 8) * (a.S / 16) * a.S), (unsigned)(a.cout / nt));
    const size_t smem = conv3_tc_smem_bytes(nt);
    switch (nt) {
    case 64: conv3_tc_kernel<64><<<grid, 128, smem, s>>>(a); break;
    case 48: conv3_tc_kernel<48><<<grid, 128, smem, s>>>(a); break;
    case 32: conv3_tc_kernel<32><<<grid, 128, smem, s>>>(a); break;
    default: conv3_tc_kernel<16><<<grid, 128, smem, s>>>(a); break;
    }
}

// One MMA with the library's descriptor encoding against the CPU product of
// the same small integer operands: 1 if every element matches, 0 if not, -1
// on a CUDA error.  A unit test of the encoding; the product path does not run it.
int tc_selftest()
{
    float* d_out = nullptr;
    int* d_fault = nullptr;
    if (cudaMalloc(&d_out, 128 * 16 * sizeof(float)) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    if (cudaMalloc(&d_fault, sizeof(int)) != cudaSuccess || cudaMemset(d_fault, 0, sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(d_out);
        return -1;
    }
    std::vector<float> want(128 * 16), got(128 * 16);
    for (int m = 0; m < 128; ++m)
        for (int n = 0; n < 16; ++n) {
            float s = 0.0f;
            for (int k = 0; k < 16; ++k) s += (float)((m + 3 * k) % 7 - 3) * (float)((2 * n + k) % 5 - 2);
            want[m * 16 + n] = s;
        }
    int result = -1;
    tc_selftest_kernel<<<1, 128>>>(d_out, d_fault);
    int fault = 0;
    if (cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(got.data(), d_out, got.size() * sizeof(float), cudaMemcpyDeviceToHost) == cudaSuccess &&
        cudaMemcpy(&fault, d_fault, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
        result = (fault == 0 && std::memcmp(got.data(), want.data(), got.size() * sizeof(float)) == 0) ? 1 : 0;
    else
        (void)cudaGetLastError();
    cudaFree(d_out);
    cudaFree(d_fault);
    return result;
}

}  // namespace unet
}  // namespace qumond
