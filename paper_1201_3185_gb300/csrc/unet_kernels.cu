// Kernels of the learned initial guess: a 3-D U-Net (3^3 convolutions, BF16
// activations and weights, FP32 accumulation) that maps (rho, Phi_N) of a box
// to Phi - Phi_N, the starting point of the QUMOND solve (Eq. 2) in place of
// FMG.  Activations are channels-last: voxel v = (z*S + y)*S + x of an S^3
// level holds its channels contiguously, with a row stride `ld` (>= the
// channel count) so that a layer can write into a slice of a concatenation.
//
// The 3^3 convolutions are implicit GEMMs on the tensor cores: M = output
// voxels (a CTA owns a brick of up to 128 voxels), N = output channels, K =
// 27 taps x input channels, in chunks of 16 channels.  A chunk's input brick
// with its one-voxel halo and the chunk's weights are staged in shared memory;
// each warp owns 16 voxels and issues m16n8k16 BF16 MMAs with FP32
// accumulators.  The weight gradient is the same contraction with K = voxels
// (both operands staged transposed), reduced over CTAs in a fixed order.
#include "unet_internal.h"

#include <cuda_bf16.h>

namespace qumond {
namespace unet {

namespace {

constexpr int kHaloMax = 432;     // (2+2) x (4+2) x (16+2) voxels: the largest brick halo
constexpr int kHaloStride = 24;   // bf16 per halo voxel: 16 channels + 8 padding (conflict-free A fragments)
constexpr int kWRow = 440;        // bf16 per output channel of a weight chunk: 27 x 16 + 8 padding

__device__ __forceinline__ unsigned lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const unsigned*>(p); }

__device__ __forceinline__ void mma16816(float* d, const unsigned* a, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned*>(&v);
}

__device__ __forceinline__ void brick_coords(const Brick& b, int l, int& lz, int& ly, int& lx)
{
    lx = l % b.bx;
    ly = (l / b.bx) % b.by;
    lz = l / (b.bx * b.by);
}

}  // namespace

// ---------------------------------------------------------------------------
// y[v, co] = act( bias[co] + sum_{tap, ci} x[v + off(tap), ci] W[co][tap][ci] ) * (mask[v, co] > 0)
// with zero padding outside the S^3 level; tap = (dz+1)*9 + (dy+1)*3 + (dx+1).
// NTILES = output channels per CTA / 8.  grid = (bricks, Cout / (8 NTILES)).
template <int NTILES>
__global__ void __launch_bounds__(256) conv3_kernel(ConvArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16* halo = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    __nv_bfloat16* wsm = halo + kHaloMax * kHaloStride;
    constexpr int NT = NTILES * 8;

    const Brick b = a.brick;
    const int S = a.S;
    const int nbx = S / b.bx, nby = S / b.by;
    const int brick = blockIdx.x;
    const int x0 = (brick % nbx) * b.bx, y0 = ((brick / nbx) % nby) * b.by, z0 = (brick / (nbx * nby)) * b.bz;
    const int co0 = blockIdx.y * NT;
    const int hx = b.bx + 2, hy = b.by + 2, hz = b.bz + 2;
    const int hv_count = hx * hy * hz;
    const int nvox = b.bx * b.by * b.bz;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    const bool warp_on = warp * 16 < nvox;
    // the two rows (voxels) of this thread in the warp's m16 tile
    const int l0 = warp * 16 + g, l1 = l0 + 8;
    const bool v0ok = l0 < nvox, v1ok = l1 < nvox;
    int hc0 = 0, hc1 = 0;  // halo index of the voxel itself (tap 13)
    {
        int lz, ly, lx;
        brick_coords(b, v0ok ? l0 : 0, lz, ly, lx);
        hc0 = ((lz + 1) * hy + (ly + 1)) * hx + (lx + 1);
        brick_coords(b, v1ok ? l1 : 0, lz, ly, lx);
        hc1 = ((lz + 1) * hy + (ly + 1)) * hx + (lx + 1);
    }

    float acc[NTILES][4];
#pragma unroll
    for (int j = 0; j < NTILES; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;

    for (int ci0 = 0; ci0 < a.cin; ci0 += 16) {
        // stage the input brick + halo, 16 channels (two 16-byte pieces per voxel)
        for (int q = threadIdx.x; q < hv_count * 2; q += blockDim.x) {
            const int hv = q >> 1, part = q & 1;
            const int ix = hv % hx, iy = (hv / hx) % hy, iz = hv / (hx * hy);
            const int gx = x0 + ix - 1, gy = y0 + iy - 1, gz = z0 + iz - 1;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (gx >= 0 && gx < S && gy >= 0 && gy < S && gz >= 0 && gz < S) {
                const long long v = ((long long)gz * S + gy) * S + gx;
                val = *reinterpret_cast<const uint4*>(a.in + v * a.ld_in + a.in_off + ci0 + part * 8);
            }
            *reinterpret_cast<uint4*>(halo + hv * kHaloStride + part * 8) = val;
        }
        // stage the weight chunk: W[co0 + n][tap][ci0 .. ci0+15]
        for (int q = threadIdx.x; q < NT * 27 * 2; q += blockDim.x) {
            const int part = q & 1, t = (q >> 1) % 27, n = (q >> 1) / 27;
            const uint4 val =
                *reinterpret_cast<const uint4*>(a.w + ((long long)(co0 + n) * 27 + t) * a.cin + ci0 + part * 8);
            *reinterpret_cast<uint4*>(wsm + n * kWRow + t * 16 + part * 8) = val;
        }
        __syncthreads();
        if (warp_on) {
#pragma unroll 1
            for (int t = 0; t < 27; ++t) {
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                const int off = (dz * hy + dy) * hx + dx;
                const __nv_bfloat16* r0 = halo + (hc0 + off) * kHaloStride + tig * 2;
                const __nv_bfloat16* r1 = halo + (hc1 + off) * kHaloStride + tig * 2;
                unsigned af[4];
                af[0] = lds32(r0);
                af[1] = lds32(r1);
                af[2] = lds32(r0 + 8);
                af[3] = lds32(r1 + 8);
#pragma unroll
                for (int j = 0; j < NTILES; ++j) {
                    const __nv_bfloat16* wp = wsm + (j * 8 + g) * kWRow + t * 16 + tig * 2;
                    mma16816(acc[j], af, lds32(wp), lds32(wp + 8));
                }
            }
        }
        __syncthreads();
    }
    if (!warp_on) return;
    // epilogue: bias, ReLU, mask, BF16 store
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int l = half ? l1 : l0;
        if (l >= nvox) continue;
        int lz, ly, lx;
        brick_coords(b, l, lz, ly, lx);
        const long long v = ((long long)(z0 + lz) * S + (y0 + ly)) * S + (x0 + lx);
#pragma unroll
        for (int j = 0; j < NTILES; ++j) {
            const int co = co0 + j * 8 + tig * 2;
            float r0 = acc[j][half * 2], r1 = acc[j][half * 2 + 1];
            if (a.bias) {
                r0 += a.bias[co];
                r1 += a.bias[co + 1];
            }
            if (a.relu) {
                r0 = fmaxf(r0, 0.0f);
                r1 = fmaxf(r1, 0.0f);
            }
            if (a.mask) {
                const __nv_bfloat16* mp = a.mask + v * a.ld_mask + a.mask_off + co;
                if (!(__bfloat162float(mp[0]) > 0.0f)) r0 = 0.0f;
                if (!(__bfloat162float(mp[1]) > 0.0f)) r1 = 0.0f;
            }
            *reinterpret_cast<unsigned*>(a.out + v * a.ld_out + a.out_off + co) = pack_bf16(r0, r1);
        }
    }
}

Brick brick_for(int S)
{
    // 128 voxels where the level allows (two planes of 4 rows of 16), else the whole level
    Brick b;
    if (S >= 16) {
        b.bz = 2, b.by = 4, b.bx = 16;
    } else if (S == 8) {
        b.bz = 2, b.by = 8, b.bx = 8;
    } else {
        b.bz = S, b.by = S, b.bx = S;  // S = 4: 64 voxels; S = 2: 8
    }
    return b;
}

size_t conv3_smem_bytes(int cout_tile)
{
    return (size_t)kHaloMax * kHaloStride * 2 + (size_t)cout_tile * kWRow * 2;
}

int conv3_tile(int cout)
{
    if (cout % 64 == 0) return 64;
    if (cout % 48 == 0) return 48;
    if (cout % 32 == 0) return 32;
    return 16;
}

template <int NTILES>
static void launch_conv3_t(const ConvArgs& a, int bricks, cudaStream_t s)
{
    const size_t smem = conv3_smem_bytes(NTILES * 8);
    conv3_kernel<NTILES><<<dim3(bricks, a.cout / (NTILES * 8)), 256, smem, s>>>(a);
}

void prepare_conv3()
{
    const int tiles[4] = {16, 32, 48, 64};
    for (int t : tiles) {
        const int smem = (int)conv3_smem_bytes(t);
        if (t == 16) cudaFuncSetAttribute(conv3_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (t == 32) cudaFuncSetAttribute(conv3_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (t == 48) cudaFuncSetAttribute(conv3_kernel<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (t == 64) cudaFuncSetAttribute(conv3_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
}

void launch_conv3(ConvArgs a, cudaStream_t s)
{
    if (conv3_tc_applies(a)) {
        launch_conv3_tc(a, s);
        return;
    }
    a.brick = brick_for(a.S);
    const int bricks = (a.S / a.brick.bx) * (a.S / a.brick.by) * (a.S / a.brick.bz);
    switch (conv3_tile(a.cout)) {
    case 64: launch_conv3_t<8>(a, bricks, s); break;
    case 48: launch_conv3_t<6>(a, bricks, s); break;
    case 32: launch_conv3_t<4>(a, bricks, s); break;
    default: launch_conv3_t<2>(a, bricks, s); break;
    }
}

// ---------------------------------------------------------------------------
// Weight gradient: part[blk][co][tap][ci] = sum over the CTA's voxels of
// g[v, co0+co] x[v + off(tap), ci0+ci], for a tile of 16 MT output channels
// and 16 input channels; grid = (vblocks, cout/(16 MT), cin/16).  Warp w takes
// taps w, w+8, w+16, w+24.  The k-dimension (voxels) must be contiguous in
// pairs for the MMA fragments, so both operands are staged transposed: g as
// [co][voxel], x as three copies [dx][ci][halo row][x] each shifted by its dx.
template <int MT>
__global__ void __launch_bounds__(256) wgrad_kernel(WgradArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Brick b = a.brick;
    const int S = a.S;
    const int nvox = b.bx * b.by * b.bz;
    const int gstride = 128 + 8;                           // bf16 per channel row of gT
    const int hrows = (b.by + 2) * (b.bz + 2);
    const int xstride = hrows * b.bx + 8;                  // bf16 per channel row of xT
    __nv_bfloat16* gT = reinterpret_cast<__nv_bfloat16*>(smem_raw);
    __nv_bfloat16* xT = gT + 16 * MT * gstride;            // [3][16][xstride]

    const int nbx = S / b.bx, nby = S / b.by;
    const int nbricks = nbx * nby * (S / b.bz);
    const int co0 = blockIdx.y * 16 * MT, ci0 = blockIdx.z * 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tig = lane & 3;
    const int ntap = warp < 3 ? 4 : 3;  // taps warp, warp+8, warp+16 (, warp+24)

    float acc[4][MT][2][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int j = 0; j < 2; ++j) acc[q][m][j][0] = acc[q][m][j][1] = acc[q][m][j][2] = acc[q][m][j][3] = 0.0f;

    for (int brick = blockIdx.x; brick < nbricks; brick += gridDim.x) {
        const int x0 = (brick % nbx) * b.bx, y0 = ((brick / nbx) % nby) * b.by, z0 = (brick / (nbx * nby)) * b.bz;
        // g^T: 16 MT channels x nvox voxels (voxels past nvox are zero)
        for (int q = threadIdx.x; q < 128 * 2 * MT; q += blockDim.x) {
            const int l = q % 128, part = q / 128;  // part: 8 channels
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (l < nvox) {
                int lz, ly, lx;
                brick_coords(b, l, lz, ly, lx);
                const long long v = ((long long)(z0 + lz) * S + (y0 + ly)) * S + (x0 + lx);
                val = *reinterpret_cast<const uint4*>(a.g + v * a.ld_g + a.g_off + co0 + part * 8);
            }
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&val);
#pragma unroll
            for (int c = 0; c < 8; ++c) gT[(part * 8 + c) * gstride + l] = e[c];
        }
        // x^T: halo rows of the brick, three copies shifted by dx
        const int hx = b.bx + 2;
        for (int q = threadIdx.x; q < hrows * hx * 2; q += blockDim.x) {
            const int part = q & 1, hv = q >> 1;
            const int ix = hv % hx, row = hv / hx;
            const int iy = row % (b.by + 2), iz = row / (b.by + 2);
            const int gx = x0 + ix - 1, gy = y0 + iy - 1, gz = z0 + iz - 1;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (gx >= 0 && gx < S && gy >= 0 && gy < S && gz >= 0 && gz < S) {
                const long long v = ((long long)gz * S + gy) * S + gx;
                val = *reinterpret_cast<const uint4*>(a.x + v * a.ld_x + a.x_off + ci0 + part * 8);
            }
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&val);
#pragma unroll
            for (int d = 0; d < 3; ++d) {  // copy d holds dx = d - 1: xT[d][ci][row][lx] = x(lx + dx)
                const int lx = ix - d;     // ix = lx + dx + 1
                if (lx >= 0 && lx < b.bx) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) xT[(d * 16 + part * 8 + c) * xstride + row * b.bx + lx] = e[c];
                }
            }
        }
        __syncthreads();
        for (int s = 0; s * 16 < nvox; ++s) {
            // A fragments (co x voxel), shared by the warp's taps
            unsigned af[MT][4];
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const __nv_bfloat16* p0 = gT + (m * 16 + g) * gstride + s * 16 + tig * 2;
                const __nv_bfloat16* p1 = p0 + 8 * gstride;
                af[m][0] = lds32(p0);
                af[m][1] = lds32(p1);
                af[m][2] = lds32(p0 + 8);
                af[m][3] = lds32(p1 + 8);
            }
            // this thread's two k-pairs: voxels s*16 + tig*2 (+1) and + 8
            int rowk[2], lxk[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int l = s * 16 + tig * 2 + h * 8;
                int lz, ly, lx;
                brick_coords(b, l < nvox ? l : 0, lz, ly, lx);
                rowk[h] = (lz + 1) * (b.by + 2) + (ly + 1);
                lxk[h] = lx;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q < ntap) {
                    const int t = warp + 8 * q;
                    const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                    const int roff = dz * (b.by + 2) + dy;
                    const __nv_bfloat16* base = xT + ((dx + 1) * 16) * xstride;
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const __nv_bfloat16* cb = base + (j * 8 + g) * xstride;
                        const unsigned b0 = lds32(cb + (rowk[0] + roff) * b.bx + lxk[0]);
                        const unsigned b1 = lds32(cb + (rowk[1] + roff) * b.bx + lxk[1]);
#pragma unroll
                        for (int m = 0; m < MT; ++m) mma16816(acc[q][m][j], af[m], b0, b1);
                    }
                }
            }
        }
        __syncthreads();
    }
    // partials: part[blk][co (16 MT)][27][16]
    const long long blk = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    float* out = a.part + blk * (16 * MT * 27 * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (q >= ntap) continue;
        const int t = warp + 8 * q;
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int co = m * 16 + g, ci = j * 8 + tig * 2;
                out[((long long)co * 27 + t) * 16 + ci] = acc[q][m][j][0];
                out[((long long)co * 27 + t) * 16 + ci + 1] = acc[q][m][j][1];
                out[((long long)(co + 8) * 27 + t) * 16 + ci] = acc[q][m][j][2];
                out[((long long)(co + 8) * 27 + t) * 16 + ci + 1] = acc[q][m][j][3];
            }
    }
}

// dW[co][tap][ci] (+)= sum over the vblocks, in order, of the partials
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int vblocks, int mt, int cout, int cin,
                                    float* __restrict__ dw, int accumulate)
{
    const long long total = (long long)cout * 27 * cin;
    const int tile_co = 16 * mt;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(e % cin);
        const int t = (int)((e / cin) % 27);
        const int co = (int)(e / (27LL * cin));
        const int cot = co / tile_co, cil = ci / 16;
        const long long blk0 = ((long long)cil * (cout / tile_co) + cot) * vblocks;
        const long long inner = ((long long)(co % tile_co) * 27 + t) * 16 + (ci % 16);
        float s = 0.0f;
        for (int vb = 0; vb < vblocks; ++vb) s += part[(blk0 + vb) * (tile_co * 27 * 16) + inner];
        dw[e] = accumulate ? dw[e] + s : s;
    }
}

int wgrad_mt(int cout) { return cout % 32 == 0 ? 2 : 1; }

size_t wgrad_smem_bytes(int mt, const Brick& b)
{
    const int hrows = (b.by + 2) * (b.bz + 2);
    return (size_t)2 * (16 * mt * (128 + 8) + 3 * 16 * (hrows * b.bx + 8));
}

int wgrad_vblocks(int S, int cout, int cin, int sms)
{
    const Brick b = brick_for(S);
    const int nbricks = (S / b.bx) * (S / b.by) * (S / b.bz);
    const int tiles = (cout / (16 * wgrad_mt(cout))) * (cin / 16);
    int vb = (2 * sms + tiles - 1) / tiles;
    if (vb > nbricks) vb = nbricks;
    return vb < 1 ? 1 : vb;
}

void prepare_wgrad()
{
    const Brick b = brick_for(128);
    cudaFuncSetAttribute(wgrad_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem_bytes(1, b));
    cudaFuncSetAttribute(wgrad_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_smem_bytes(2, b));
}

void launch_wgrad(WgradArgs a, int vblocks, float* dw, int accumulate, cudaStream_t s)
{
    a.brick = brick_for(a.S);
    const int mt = wgrad_mt(a.cout);
    const dim3 grid(vblocks, a.cout / (16 * mt), a.cin / 16);
    const size_t smem = wgrad_smem_bytes(mt, a.brick);
    if (mt == 2)
        wgrad_kernel<2><<<grid, 256, smem, s>>>(a);
    else
        wgrad_kernel<1><<<grid, 256, smem, s>>>(a);
    const long long total = (long long)a.cout * 27 * a.cin;
    const int blocks = (int)((total + 255) / 256 < 2048 ? (total + 255) / 256 : 2048);
    wgrad_reduce_kernel<<<blocks, 256, 0, s>>>(a.part, vblocks, mt, a.cout, a.cin, dw, accumulate);
}

// ---------------------------------------------------------------------------
// Bias gradient: db[c] (+)= sum_v g[v, c], per-block partial sums in voxel
// order, then the blocks in order.
__global__ void colsum_kernel(const __nv_bfloat16* __restrict__ g, int ld, int off, int C, long long nvox,
                              float* __restrict__ part)
{
    // block: 256 threads = C columns x (256 / C) row lanes (C divides 256)
    const int c = threadIdx.x % C, lane = threadIdx.x / C, lanes = blockDim.x / C;
    const long long chunk = (nvox + gridDim.x - 1) / gridDim.x;
    const long long v0 = blockIdx.x * chunk, v1 = v0 + chunk < nvox ? v0 + chunk : nvox;
    float s = 0.0f;
    for (long long v = v0 + lane; v < v1; v += lanes) s += __bfloat162float(g[v * ld + off + c]);
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    if (lane == 0) {
        float t = 0.0f;
        for (int r = 0; r < lanes; ++r) t += red[r * C + c];
        part[(long long)blockIdx.x * C + c] = t;
    }
}

__global__ void colsum_reduce_kernel(const float* __restrict__ part, int nb, int C, float* __restrict__ out,
                                     int accumulate)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.0f;
    for (int b = 0; b < nb; ++b) s += part[(long long)b * C + c];
    out[c] = accumulate ? out[c] + s : s;
}

void launch_bias_grad(const __nv_bfloat16* g, int ld, int off, int C, long long nvox, float* part, int nb, float* db,
                      int accumulate, cudaStream_t s)
{
    // C <= 256 and a power of two times 16 or 48 ... the layer widths are 16, 32, 64, 128
    colsum_kernel<<<nb, 256, 0, s>>>(g, ld, off, C, nvox, part);
    colsum_reduce_kernel<<<(C + 127) / 128, 128, 0, s>>>(part, nb, C, db, accumulate);
}

// ---------------------------------------------------------------------------
// 2x2x2 average pooling (S -> S/2) and its adjoint with the skip gradient and the ReLU mask
__global__ void pool_kernel(const __nv_bfloat16* __restrict__ x, int ld_x, int off_x, int C, int S,
                            __nv_bfloat16* __restrict__ y)
{
    const int Sh = S / 2;
    const long long total = (long long)Sh * Sh * Sh * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long p = e / C;
        const int px = (int)(p % Sh), py = (int)((p / Sh) % Sh), pz = (int)(p / ((long long)Sh * Sh));
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long long v = ((long long)(2 * pz + (q >> 2)) * S + (2 * py + ((q >> 1) & 1))) * S + 2 * px + (q & 1);
            s += __bfloat162float(x[v * ld_x + off_x + c]);
        }
        y[e] = __float2bfloat16_rn(0.125f * s);
    }
}

// gx[v, c] = (gp[parent(v), c] / 8 + gskip[v, off_s + c]) * (mask[v, off_m + c] > 0)
__global__ void pool_back_kernel(const __nv_bfloat16* __restrict__ gp, const __nv_bfloat16* __restrict__ gskip,
                                 int ld_s, int off_s, const __nv_bfloat16* __restrict__ mask, int ld_m, int off_m,
                                 int C, int S, __nv_bfloat16* __restrict__ gx)
{
    const int Sh = S / 2;
    const long long total = (long long)S * S * S * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long v = e / C;
        const int x = (int)(v % S), y = (int)((v / S) % S), z = (int)(v / ((long long)S * S));
        const long long p = ((long long)(z / 2) * Sh + y / 2) * Sh + x / 2;
        float r = 0.125f * __bfloat162float(gp[p * C + c]);
        if (gskip) r += __bfloat162float(gskip[v * ld_s + off_s + c]);
        if (!(__bfloat162float(mask[v * ld_m + off_m + c]) > 0.0f)) r = 0.0f;
        gx[e] = __float2bfloat16_rn(r);
    }
}

// nearest-neighbour upsampling S/2 -> S into channels [0, C) of a concatenation (row stride ld_y)
__global__ void up_kernel(const __nv_bfloat16* __restrict__ x, int C, int S, __nv_bfloat16* __restrict__ y, int ld_y)
{
    const int Sh = S / 2;
    const long long total = (long long)S * S * S * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long v = e / C;
        const int px = (int)(v % S) / 2, py = (int)((v / S) % S) / 2, pz = (int)(v / ((long long)S * S)) / 2;
        y[v * ld_y + c] = x[(((long long)pz * Sh + py) * Sh + px) * C + c];
    }
}

// gx[p, c] = (sum of gy over the 8 children, channels [0, C) of row stride ld_y) * (mask[p, c] > 0)
__global__ void up_back_kernel(const __nv_bfloat16* __restrict__ gy, int ld_y, const __nv_bfloat16* __restrict__ mask,
                               int C, int S, __nv_bfloat16* __restrict__ gx)
{
    const int Sh = S / 2;
    const long long total = (long long)Sh * Sh * Sh * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        const long long p = e / C;
        const int px = (int)(p % Sh), py = (int)((p / Sh) % Sh), pz = (int)(p / ((long long)Sh * Sh));
        float s = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const long long v = ((long long)(2 * pz + (q >> 2)) * S + (2 * py + ((q >> 1) & 1))) * S + 2 * px + (q & 1);
            s += __bfloat162float(gy[v * ld_y + c]);
        }
        if (!(__bfloat162float(mask[p * C + c]) > 0.0f)) s = 0.0f;
        gx[e] = __float2bfloat16_rn(s);
    }
}

static int ew_blocks(long long total)
{
    long long b = (total + 255) / 256;
    return (int)(b < 152 * 16 ? b : 152 * 16);
}

void launch_pool(const __nv_bfloat16* x, int ld_x, int off_x, int C, int S, __nv_bfloat16* y, cudaStream_t s)
{
    pool_kernel<<<ew_blocks((long long)(S / 2) * (S / 2) * (S / 2) * C), 256, 0, s>>>(x, ld_x, off_x, C, S, y);
}

void launch_pool_back(const __nv_bfloat16* gp, const __nv_bfloat16* gskip, int ld_s, int off_s,
                      const __nv_bfloat16* mask, int ld_m, int off_m, int C, int S, __nv_bfloat16* gx, cudaStream_t s)
{
    pool_back_kernel<<<ew_blocks((long long)S * S * S * C), 256, 0, s>>>(gp, gskip, ld_s, off_s, mask, ld_m, off_m, C,
                                                                         S, gx);
}

void launch_up(const __nv_bfloat16* x, int C, int S, __nv_bfloat16* y, int ld_y, cudaStream_t s)
{
    up_kernel<<<ew_blocks((long long)S * S * S * C), 256, 0, s>>>(x, C, S, y, ld_y);
}

void launch_up_back(const __nv_bfloat16* gy, int ld_y, const __nv_bfloat16* mask, int C, int S, __nv_bfloat16* gx,
                    cudaStream_t s)
{
    up_back_kernel<<<ew_blocks((long long)(S / 2) * (S / 2) * (S / 2) * C), 256, 0, s>>>(gy, ld_y, mask, C, S, gx);
}

// ---------------------------------------------------------------------------
// Network input.  Voxel (x, y, z) of the S^3 input is node (x, y, z) of the
// box's (S+1)^3 grid: channel 0 = rho_scale * rho, channel 1 = Phi_N / phi_scale,
// channel 2 = the box flag, channels 3..15 = 0.
__global__ void input_from_grids_kernel(const double* __restrict__ rho, const double* __restrict__ phiN, int S,
                                        double rho_scale, double inv_phi, float flag, __nv_bfloat16* __restrict__ x0)
{
    const long long total = (long long)S * S * S;
    const int n1 = S + 1;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % S), y = (int)((v / S) % S), z = (int)(v / ((long long)S * S));
        const long long node = ((long long)z * n1 + y) * n1 + x;
        __nv_bfloat16 row[16];
        row[0] = __float2bfloat16_rn((float)(rho[node] * rho_scale));
        row[1] = __float2bfloat16_rn((float)(phiN[node] * inv_phi));
        row[2] = __float2bfloat16_rn(flag);
#pragma unroll
        for (int c = 3; c < 16; ++c) row[c] = __float2bfloat16_rn(0.0f);
        uint4* dst = reinterpret_cast<uint4*>(x0 + v * 16);
        dst[0] = *reinterpret_cast<uint4*>(&row[0]);
        dst[1] = *reinterpret_cast<uint4*>(&row[8]);
    }
}

// training sample: [0] rho channel, [1] Phi_N channel, [2] target (Phi - Phi_N) / phi_scale, each S^3 BF16
__global__ void make_sample_kernel(const double* __restrict__ rho, const double* __restrict__ phiN,
                                   const double* __restrict__ phi, int S, double rho_scale, double inv_phi,
                                   __nv_bfloat16* __restrict__ sample)
{
    const long long total = (long long)S * S * S;
    const int n1 = S + 1;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(v % S), y = (int)((v / S) % S), z = (int)(v / ((long long)S * S));
        const long long node = ((long long)z * n1 + y) * n1 + x;
        sample[v] = __float2bfloat16_rn((float)(rho[node] * rho_scale));
        sample[total + v] = __float2bfloat16_rn((float)(phiN[node] * inv_phi));
        sample[2 * total + v] = __float2bfloat16_rn((float)((phi[node] - phiN[node]) * inv_phi));
    }
}

__global__ void input_from_sample_kernel(const __nv_bfloat16* __restrict__ sample, int S, float flag,
                                         __nv_bfloat16* __restrict__ x0)
{
    const long long total = (long long)S * S * S;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total;
         v += (long long)gridDim.x * blockDim.x) {
        __nv_bfloat16 row[16];
        row[0] = sample[v];
        row[1] = sample[total + v];
        row[2] = __float2bfloat16_rn(flag);
#pragma unroll
        for (int c = 3; c < 16; ++c) row[c] = __float2bfloat16_rn(0.0f);
        uint4* dst = reinterpret_cast<uint4*>(x0 + v * 16);
        dst[0] = *reinterpret_cast<uint4*>(&row[0]);
        dst[1] = *reinterpret_cast<uint4*>(&row[8]);
    }
}

void launch_input_from_grids(const double* rho, const double* phiN, int S, double rho_scale, double inv_phi,
                             float flag, __nv_bfloat16* x0, cudaStream_t s)
{
    input_from_grids_kernel<<<ew_blocks((long long)S * S * S), 256, 0, s>>>(rho, phiN, S, rho_scale, inv_phi, flag, x0);
}

void launch_make_sample(const double* rho, const double* phiN, const double* phi, int S, double rho_scale,
                        double inv_phi, __nv_bfloat16* sample, cudaStream_t s)
{
    make_sample_kernel<<<ew_blocks((long long)S * S * S), 256, 0, s>>>(rho, phiN, phi, S, rho_scale, inv_phi, sample);
}

void launch_input_from_sample(const __nv_bfloat16* sample, int S, float flag, __nv_bfloat16* x0, cudaStream_t s)
{
    input_from_sample_kernel<<<ew_blocks((long long)S * S * S), 256, 0, s>>>(sample, S, flag, x0);
}

// ---------------------------------------------------------------------------
// Head: yhat[v] = b + sum_c w[c] a[v, c]  (1x1x1 convolution, FP32 output).
// Training form: with target t and scale k = 2 / (S^3 nbatch):
//   loss partial += (yhat - t)^2, dy = k (yhat - t),
//   ga[v, c] = dy w[c] (a[v, c] > 0), head-gradient partials sum dy a[v, c] and sum dy.
__global__ void head_kernel(const __nv_bfloat16* __restrict__ a, const float* __restrict__ wb, long long nvox,
                            float* __restrict__ yhat)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        float s = wb[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) s += wb[c] * __bfloat162float(a[v * 16 + c]);
        yhat[v] = s;
    }
}

__global__ void head_train_kernel(const __nv_bfloat16* __restrict__ a, const float* __restrict__ wb,
                                  const __nv_bfloat16* __restrict__ target, long long nvox, float k,
                                  __nv_bfloat16* __restrict__ ga, float* __restrict__ part)
{
    // part[block][0..15] = sum dy a[:, c], [16] = sum dy, [17] = sum (yhat - t)^2
    float pw[18];
#pragma unroll
    for (int c = 0; c < 18; ++c) pw[c] = 0.0f;
    float w[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) w[c] = wb[c];
    const long long chunk = (nvox + gridDim.x - 1) / gridDim.x;
    const long long v0 = blockIdx.x * chunk, v1 = v0 + chunk < nvox ? v0 + chunk : nvox;
    for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        float av[16];
        float s = wb[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            av[c] = __bfloat162float(a[v * 16 + c]);
            s += w[c] * av[c];
        }
        const float d = s - __bfloat162float(target[v]);
        const float dy = k * d;
        __nv_bfloat16 row[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            pw[c] += dy * av[c];
            row[c] = __float2bfloat16_rn(av[c] > 0.0f ? dy * w[c] : 0.0f);
        }
        pw[16] += dy;
        pw[17] += d * d;
        uint4* dst = reinterpret_cast<uint4*>(ga + v * 16);
        dst[0] = *reinterpret_cast<uint4*>(&row[0]);
        dst[1] = *reinterpret_cast<uint4*>(&row[8]);
    }
    __shared__ float red[18][256];
#pragma unroll
    for (int c = 0; c < 18; ++c) red[c][threadIdx.x] = pw[c];
    __syncthreads();
    if (threadIdx.x < 18) {
        float t = 0.0f;
        for (int r = 0; r < (int)blockDim.x; ++r) t += red[threadIdx.x][r];
        part[(long long)blockIdx.x * 18 + threadIdx.x] = t;
    }
}

// out[0..16] (+)= head gradients, loss_out (+)= sum of squares * loss_scale
__global__ void head_reduce_kernel(const float* __restrict__ part, int nb, float* __restrict__ dwb, int accumulate,
                                   float* __restrict__ loss, float loss_scale)
{
    const int c = threadIdx.x;
    if (c >= 18) return;
    float s = 0.0f;
    for (int b = 0; b < nb; ++b) s += part[(long long)b * 18 + c];
    if (c < 17)
        dwb[c] = accumulate ? dwb[c] + s : s;
    else if (loss)
        *loss = (accumulate ? *loss : 0.0f) + s * loss_scale;
}

void launch_head(const __nv_bfloat16* a, const float* wb, long long nvox, float* yhat, cudaStream_t s)
{
    head_kernel<<<ew_blocks(nvox), 256, 0, s>>>(a, wb, nvox, yhat);
}

void launch_head_train(const __nv_bfloat16* a, const float* wb, const __nv_bfloat16* target, long long nvox, float k,
                       __nv_bfloat16* ga, float* part, int nb, float* dwb, int accumulate, float* loss,
                       float loss_scale, cudaStream_t s)
{
    head_train_kernel<<<nb, 256, 0, s>>>(a, wb, target, nvox, k, ga, part);
    head_reduce_kernel<<<1, 32, 0, s>>>(part, nb, dwb, accumulate, loss, loss_scale);
}

// phi[node] = phiN[node] + phi_scale * yhat[v] on the interior nodes 1..S-1 of each axis
__global__ void apply_guess_kernel(const double* __restrict__ phiN, const float* __restrict__ yhat, int S,
                                   double phi_scale, double* __restrict__ phi)
{
    const long long total = (long long)(S - 1) * (S - 1) * (S - 1);
    const int n1 = S + 1;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = 1 + (int)(e % (S - 1)), y = 1 + (int)((e / (S - 1)) % (S - 1)),
                  z = 1 + (int)(e / ((long long)(S - 1) * (S - 1)));
        const long long node = ((long long)z * n1 + y) * n1 + x;
        const long long v = ((long long)z * S + y) * S + x;
        phi[node] = phiN[node] + phi_scale * (double)yhat[v];
    }
}

void launch_apply_guess(const double* phiN, const float* yhat, int S, double phi_scale, double* phi, cudaStream_t s)
{
    apply_guess_kernel<<<ew_blocks((long long)(S - 1) * (S - 1) * (S - 1)), 256, 0, s>>>(phiN, yhat, S, phi_scale, phi);
}

// ---------------------------------------------------------------------------
// Adam on the FP32 master parameters (gradients already averaged over the
// batch), then the BF16 copies in the two layouts the convolutions read:
// forward W[co][tap][ci] and data-gradient Wd[ci][26 - tap][co].
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

__global__ void weights_bf16_kernel(const float* __restrict__ w, int cout, int cin, __nv_bfloat16* __restrict__ wf,
                                    __nv_bfloat16* __restrict__ wd)
{
    const long long total = (long long)cout * 27 * cin;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(e % cin), t = (int)((e / cin) % 27), co = (int)(e / (27LL * cin));
        const __nv_bfloat16 h = __float2bfloat16_rn(w[e]);
        wf[e] = h;
        if (wd) wd[((long long)ci * 27 + (26 - t)) * cout + co] = h;
    }
}

void launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t s)
{
    adam_kernel<<<ew_blocks(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
}

void launch_weights_bf16(const float* w, int cout, int cin, __nv_bfloat16* wf, __nv_bfloat16* wd, cudaStream_t s)
{
    weights_bf16_kernel<<<ew_blocks((long long)cout * 27 * cin), 256, 0, s>>>(w, cout, cin, wf, wd);
}

__global__ void scale_kernel(float* __restrict__ x, long long n, float k)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= k;
}

void launch_scale(float* x, long long n, float k, cudaStream_t s) { scale_kernel<<<ew_blocks(n), 256, 0, s>>>(x, n, k); }

}  // namespace unet
}  // namespace qumond
