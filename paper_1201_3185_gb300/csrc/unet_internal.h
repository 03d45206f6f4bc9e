// Internal interface of the learned-initial-guess kernels (unet_kernels.cu)
// and the network built from them (unet_api.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

namespace qumond {
namespace unet {

struct Brick {
    int bz, by, bx;  // voxels of a CTA's output brick along z, y, x (product <= 128)
};

// A 3^3 convolution (zero padding, stride 1) on an S^3 level, channels last.
struct ConvArgs {
    const __nv_bfloat16* in;  // input, row stride ld_in, channels [in_off, in_off + cin)
    int ld_in, in_off, cin;
    const __nv_bfloat16* w;   // weights [cout][27][cin]
    const float* bias;        // cout, or null
    __nv_bfloat16* out;       // output, row stride ld_out, channels [out_off, out_off + cout)
    int ld_out, out_off, cout;
    const __nv_bfloat16* mask;  // multiply output channel co by (mask[v, mask_off + co] > 0), or null
    int ld_mask, mask_off;
    int relu;
    int S;
    Brick brick;  // set by the launcher
    int use_tc;   // 1: the convolution may run on the tcgen05 path (where conv3_tc_applies); 0: mma.sync
    int* fault;   // set to 3 when a bounded wait of the tcgen05 path gave up
};

// Weight gradient of a 3^3 convolution: dW[co][tap][ci] = sum_v g[v, co] x[v + off(tap), ci].
struct WgradArgs {
    const __nv_bfloat16* x;  // layer input, row stride ld_x, channels [x_off, x_off + cin)
    int ld_x, x_off, cin;
    const __nv_bfloat16* g;  // gradient at the layer output (after the ReLU mask), row stride ld_g
    int ld_g, g_off, cout;
    float* part;             // partial sums, (cout/16MT) x (cin/16) x vblocks x (16MT x 27 x 16) floats
    int S;
    Brick brick;
};

Brick brick_for(int S);
size_t conv3_smem_bytes(int cout_tile);
int conv3_tile(int cout);
void prepare_conv3();
void launch_conv3(ConvArgs a, cudaStream_t s);

// tcgen05 path (unet_tc.cu)
int tc_selftest();
bool conv3_tc_applies(const ConvArgs& a);
size_t conv3_tc_smem_bytes(int nt);
void prepare_conv3_tc();
void launch_conv3_tc(const ConvArgs& a, cudaStream_t s);

int wgrad_mt(int cout);
size_t wgrad_smem_bytes(int mt, const Brick& b);
int wgrad_vblocks(int S, int cout, int cin, int sms);
void prepare_wgrad();
void launch_wgrad(WgradArgs a, int vblocks, float* dw, int accumulate, cudaStream_t s);

void launch_bias_grad(const __nv_bfloat16* g, int ld, int off, int C, long long nvox, float* part, int nb, float* db,
                      int accumulate, cudaStream_t s);
void launch_pool(const __nv_bfloat16* x, int ld_x, int off_x, int C, int S, __nv_bfloat16* y, cudaStream_t s);
void launch_pool_back(const __nv_bfloat16* gp, const __nv_bfloat16* gskip, int ld_s, int off_s,
                      const __nv_bfloat16* mask, int ld_m, int off_m, int C, int S, __nv_bfloat16* gx, cudaStream_t s);
void launch_up(const __nv_bfloat16* x, int C, int S, __nv_bfloat16* y, int ld_y, cudaStream_t s);
void launch_up_back(const __nv_bfloat16* gy, int ld_y, const __nv_bfloat16* mask, int C, int S, __nv_bfloat16* gx,
                    cudaStream_t s);
void launch_input_from_grids(const double* rho, const double* phiN, int S, double rho_scale, double inv_phi,
                             float flag, __nv_bfloat16* x0, cudaStream_t s);
void launch_make_sample(const double* rho, const double* phiN, const double* phi, int S, double rho_scale,
                        double inv_phi, __nv_bfloat16* sample, cudaStream_t s);
void launch_input_from_sample(const __nv_bfloat16* sample, int S, float flag, __nv_bfloat16* x0, cudaStream_t s);
void launch_head(const __nv_bfloat16* a, const float* wb, long long nvox, float* yhat, cudaStream_t s);
void launch_head_train(const __nv_bfloat16* a, const float* wb, const __nv_bfloat16* target, long long nvox, float k,
                       __nv_bfloat16* ga, float* part, int nb, float* dwb, int accumulate, float* loss,
                       float loss_scale, cudaStream_t s);
void launch_apply_guess(const double* phiN, const float* yhat, int S, double phi_scale, double* phi, cudaStream_t s);
void launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2, float eps,
                 float c1, float c2, cudaStream_t s);
void launch_weights_bf16(const float* w, int cout, int cin, __nv_bfloat16* wf, __nv_bfloat16* wd, cudaStream_t s);
void launch_scale(float* x, long long n, float k, cudaStream_t s);

}  // namespace unet
}  // namespace qumond
