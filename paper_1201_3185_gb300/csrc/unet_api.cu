// The learned initial guess behind the C ABI of include/qumond_guess.h: the
// U-Net's layer table, its buffers, and the order of the kernels of
// unet_kernels.cu for inference, gradients and an Adam step.
#include "qumond_guess.h"
#include "unet_internal.h"

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

using namespace qumond::unet;

namespace {

struct LayerDef {
    int cin, cout, level;
};
// encoder 0..7 (two per level), decoder 8..13 (two per level, first reads the concatenation)
constexpr LayerDef kLayers[14] = {{16, 16, 0},   {16, 16, 0}, {16, 32, 1}, {32, 32, 1}, {32, 64, 2},
                                  {64, 64, 2},   {64, 128, 3}, {128, 128, 3}, {192, 64, 2}, {64, 64, 2},
                                  {96, 32, 1},   {32, 32, 1}, {48, 16, 0}, {16, 16, 0}};
constexpr int kNumLayers = 14;

long long layer_weights(int l) { return 27LL * kLayers[l].cin * kLayers[l].cout; }

long long param_count()
{
    long long n = 17;  // head
    for (int l = 0; l < kNumLayers; ++l) n += layer_weights(l) + kLayers[l].cout;
    return n;
}

}  // namespace

struct qumond_guess {
    int S = 0;
    double phi_scale = 1.0;
    int sms = 152;
    long long nparams = 0;
    std::string err;
    int step = 0;
    // parameters (FP32 master), gradients, Adam moments; per-layer offsets into them
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    long long woff[kNumLayers] = {}, boff[kNumLayers] = {}, head_off = 0;
    // BF16 weights: forward layout and data-gradient layout, per layer
    __nv_bfloat16* wf[kNumLayers] = {};
    __nv_bfloat16* wd[kNumLayers] = {};
    // activations
    __nv_bfloat16 *X0 = nullptr, *A[kNumLayers] = {}, *D[3] = {}, *P[3] = {};
    float* yhat = nullptr;
    // gradients of the activations
    __nv_bfloat16 *G[kNumLayers] = {}, *GD[3] = {}, *GP[3] = {};
    // reduction scratch
    float* wpart = nullptr;
    float* cpart = nullptr;
    float* hpart = nullptr;
    int cblocks = 0, hblocks = 0;
    int tc_ok = 0;        // the device runs tcgen05 (compute capability 10.3, the architecture this library is built for)
    int use_tc = 0;       // 1: tcgen05 convolutions where they apply, 0: mma.sync everywhere
    int* fault = nullptr; // bounded waits of the tcgen05 path
    long long launches = 0;  // kernels enqueued by the API calls (each launch_* helper's count at its call site)
    std::vector<void*> allocs;
};

namespace {

qumond_status fail(qumond_guess* g, qumond_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (g) g->err = buf;
    return st;
}

#define GTRY(g, expr, where)                                                                       \
    do {                                                                                           \
        cudaError_t _e = (expr);                                                                   \
        if (_e != cudaSuccess) return fail(g, QUMOND_ERR_CUDA, "%s: %s", where, cudaGetErrorString(_e)); \
    } while (0)

bool dev_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaStream_t S_(void* s) { return reinterpret_cast<cudaStream_t>(s); }

template <typename T>
bool alloc(qumond_guess* g, T** p, size_t count)
{
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    g->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

long long vox(const qumond_guess* g, int level)
{
    const long long s = g->S >> level;
    return s * s * s;
}

// channels of the concatenation at a decoder level: upsampled part first, then the skip
int cat_channels(int level) { return level == 0 ? 48 : level == 1 ? 96 : 192; }
int up_channels(int level) { return level == 0 ? 32 : level == 1 ? 64 : 128; }

// Where layer l reads its input and writes its output.
struct Where {
    const __nv_bfloat16* in;
    int ld_in, in_off;
    __nv_bfloat16* out;
    int ld_out, out_off;
};

Where where(qumond_guess* g, int l)
{
    Where w{};
    const int lev = kLayers[l].level;
    // input
    if (l == 0) {
        w.in = g->X0, w.ld_in = 16, w.in_off = 0;
    } else if (l == 2 || l == 4 || l == 6) {
        w.in = g->P[lev - 1], w.ld_in = kLayers[l].cin, w.in_off = 0;
    } else if (l == 8 || l == 10 || l == 12) {
        w.in = g->D[lev], w.ld_in = cat_channels(lev), w.in_off = 0;
    } else {
        w.in = g->A[l - 1], w.ld_in = kLayers[l].cin, w.in_off = 0;
    }
    // output: the second encoder layer of levels 0..2 writes the skip slice of the concatenation
    if (l == 1 || l == 3 || l == 5) {
        w.out = g->D[lev], w.ld_out = cat_channels(lev), w.out_off = up_channels(lev);
    } else {
        w.out = g->A[l], w.ld_out = kLayers[l].cout, w.out_off = 0;
    }
    return w;
}

// the layer's output as a read-only view (for masks and the next layer)
void out_view(qumond_guess* g, int l, const __nv_bfloat16** p, int* ld, int* off)
{
    const Where w = where(g, l);
    *p = w.out, *ld = w.ld_out, *off = w.out_off;
}

void conv(qumond_guess* g, int l, cudaStream_t s)
{
    const Where w = where(g, l);
    ConvArgs a{};
    a.in = w.in, a.ld_in = w.ld_in, a.in_off = w.in_off, a.cin = kLayers[l].cin;
    a.w = g->wf[l], a.bias = g->params + g->boff[l];
    a.out = w.out, a.ld_out = w.ld_out, a.out_off = w.out_off, a.cout = kLayers[l].cout;
    a.relu = 1;
    a.S = g->S >> kLayers[l].level;
    a.use_tc = g->use_tc;
    a.fault = g->fault;
    launch_conv3(a, s);
    g->launches += 1;
}

void forward(qumond_guess* g, cudaStream_t s)
{
    for (int l = 0; l < kNumLayers; ++l) {
        const int lev = kLayers[l].level;
        const int S = g->S >> lev;
        if (l == 2 || l == 4 || l == 6) {  // pool the previous level's skip output
            const int C = kLayers[l].cin;
            launch_pool(g->D[lev - 1], cat_channels(lev - 1), up_channels(lev - 1), C, S * 2, g->P[lev - 1], s);
            g->launches += 1;
        }
        if (l == 8 || l == 10 || l == 12) {  // upsample the level below into the concatenation
            launch_up(g->A[l - 1], up_channels(lev), S, g->D[lev], cat_channels(lev), s);
            g->launches += 1;
        }
        conv(g, l, s);
    }
}

// gradient of the whole network for one sample, accumulated into g->grads (accumulate = 0: overwrite)
void backward(qumond_guess* g, const __nv_bfloat16* target, float k, float loss_scale, float* loss, int accumulate,
              cudaStream_t s)
{
    const long long n0 = vox(g, 0);
    g->launches += 2;  // head + its reduction
    launch_head_train(g->A[13], g->params + g->head_off, target, n0, k, g->G[13], g->hpart, g->hblocks,
                      g->grads + g->head_off, accumulate, loss, loss_scale, s);
    for (int l = kNumLayers - 1; l >= 0; --l) {
        const int lev = kLayers[l].level;
        const int S = g->S >> lev;
        const int cin = kLayers[l].cin, cout = kLayers[l].cout;
        const Where w = where(g, l);
        // weight and bias gradients
        WgradArgs wa{};
        wa.x = w.in, wa.ld_x = w.ld_in, wa.x_off = w.in_off, wa.cin = cin;
        wa.g = g->G[l], wa.ld_g = cout, wa.g_off = 0, wa.cout = cout;
        wa.part = g->wpart;
        wa.S = S;
        launch_wgrad(wa, wgrad_vblocks(S, cout, cin, g->sms), g->grads + g->woff[l], accumulate, s);
        g->launches += 4;  // weight gradient + reduction, bias gradient + reduction
        launch_bias_grad(g->G[l], cout, 0, cout, vox(g, lev), g->cpart, g->cblocks, g->grads + g->boff[l], accumulate,
                         s);
        if (l == 0) break;
        // data gradient: d(input) = conv(G[l], Wd[l]); masked when the input is a ReLU output
        ConvArgs a{};
        a.in = g->G[l], a.ld_in = cout, a.in_off = 0, a.cin = cout;
        a.w = g->wd[l], a.bias = nullptr, a.relu = 0, a.cout = cin, a.S = S;
        a.use_tc = g->use_tc;
        a.fault = g->fault;
        const bool from_pool = (l == 2 || l == 4 || l == 6);
        const bool from_cat = (l == 8 || l == 10 || l == 12);
        if (from_pool) {
            a.out = g->GP[lev - 1], a.ld_out = cin, a.out_off = 0;
        } else if (from_cat) {
            a.out = g->GD[lev], a.ld_out = cat_channels(lev), a.out_off = 0;
        } else {
            // the input is layer l-1's output (ReLU): mask by it
            const __nv_bfloat16* mp;
            int ld, off;
            out_view(g, l - 1, &mp, &ld, &off);
            a.out = g->G[l - 1], a.ld_out = cin, a.out_off = 0;
            a.mask = mp, a.ld_mask = ld, a.mask_off = off;
        }
        launch_conv3(a, s);
        g->launches += 1;
        if (from_pool) {
            // layer l-1 (second encoder layer of the level above) gets the pooled gradient plus the skip gradient
            const int up = lev - 1;
            const int C = cin;
            g->launches += 1;
            launch_pool_back(g->GP[up], g->GD[up], cat_channels(up), up_channels(up), g->D[up], cat_channels(up),
                             up_channels(up), C, S * 2, g->G[l - 1], s);
        } else if (from_cat) {
            // layer l-1 (the level below) gets the sum over the 8 children of the upsampled slice
            launch_up_back(g->GD[lev], cat_channels(lev), g->A[l - 1], up_channels(lev), S, g->G[l - 1], s);
            g->launches += 1;
        }
    }
}

void refresh_bf16(qumond_guess* g, cudaStream_t s)
{
    for (int l = 0; l < kNumLayers; ++l)
        launch_weights_bf16(g->params + g->woff[l], kLayers[l].cout, kLayers[l].cin, g->wf[l], g->wd[l], s);
    g->launches += kNumLayers;
}

qumond_status check_samples(qumond_guess* g, const uint16_t* const* samples, const float* flags, int nbatch)
{
    if (!samples || !flags || nbatch < 1) return fail(g, QUMOND_ERR_INVALID_ARG, "need nbatch >= 1 samples and flags");
    for (int i = 0; i < nbatch; ++i)
        if (!dev_ptr(samples[i])) return fail(g, QUMOND_ERR_INVALID_ARG, "sample %d is not a device pointer", i);
    return QUMOND_OK;
}

qumond_status batch_gradients(qumond_guess* g, const uint16_t* const* samples, const float* flags, int nbatch,
                              float* loss, cudaStream_t s)
{
    const long long n0 = vox(g, 0);
    const float k = 2.0f / (float)((double)n0 * nbatch);
    const float ls = 1.0f / (float)((double)n0 * nbatch);
    for (int i = 0; i < nbatch; ++i) {
        const __nv_bfloat16* smp = reinterpret_cast<const __nv_bfloat16*>(samples[i]);
        launch_input_from_sample(smp, g->S, flags[i], g->X0, s);
        g->launches += 1;
        forward(g, s);
        backward(g, smp + 2 * n0, k, ls, loss, i > 0, s);
    }
    GTRY(g, cudaGetLastError(), "gradient launch");
    return QUMOND_OK;
}

}  // namespace

extern "C" {

int64_t qumond_guess_num_params(void) { return param_count(); }

const char* qumond_guess_last_error(qumond_guess* g) { return g ? g->err.c_str() : "null network"; }

qumond_status qumond_guess_create(int S, double phi_scale, qumond_guess** out)
{
    if (!out) return QUMOND_ERR_INVALID_ARG;
    *out = nullptr;
    if (S < 16 || S > 512 || S % 16 != 0) return QUMOND_ERR_INVALID_ARG;
    if (!(phi_scale > 0.0)) return QUMOND_ERR_INVALID_ARG;
    qumond_guess* g = new qumond_guess();
    g->S = S;
    g->phi_scale = phi_scale;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
    g->nparams = param_count();
    long long off = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        g->woff[l] = off;
        off += layer_weights(l);
        g->boff[l] = off;
        off += kLayers[l].cout;
    }
    g->head_off = off;
    bool ok = alloc(g, &g->params, g->nparams) && alloc(g, &g->grads, g->nparams) &&
              alloc(g, &g->adam_m, g->nparams) && alloc(g, &g->adam_v, g->nparams);
    for (int l = 0; ok && l < kNumLayers; ++l)
        ok = alloc(g, &g->wf[l], layer_weights(l)) && alloc(g, &g->wd[l], layer_weights(l));
    ok = ok && alloc(g, &g->X0, vox(g, 0) * 16) && alloc(g, &g->yhat, vox(g, 0));
    for (int lev = 0; ok && lev < 3; ++lev)
        ok = alloc(g, &g->D[lev], vox(g, lev) * cat_channels(lev)) && alloc(g, &g->GD[lev], vox(g, lev) * cat_channels(lev)) &&
             alloc(g, &g->P[lev], vox(g, lev + 1) * kLayers[2 * lev + 2].cin) &&
             alloc(g, &g->GP[lev], vox(g, lev + 1) * kLayers[2 * lev + 2].cin);
    for (int l = 0; ok && l < kNumLayers; ++l) {
        const long long nv = vox(g, kLayers[l].level) * kLayers[l].cout;
        if (!(l == 1 || l == 3 || l == 5)) ok = alloc(g, &g->A[l], nv);
        ok = ok && alloc(g, &g->G[l], nv);
    }
    // weight-gradient partials: the largest layer
    long long wp = 0;
    for (int l = 0; l < kNumLayers; ++l) {
        const int S_l = S >> kLayers[l].level;
        const int mt = wgrad_mt(kLayers[l].cout);
        const long long tiles = (kLayers[l].cout / (16 * mt)) * (kLayers[l].cin / 16);
        const long long need = tiles * wgrad_vblocks(S_l, kLayers[l].cout, kLayers[l].cin, g->sms) * (16LL * mt * 27 * 16);
        if (need > wp) wp = need;
    }
    g->cblocks = 2 * g->sms;
    g->hblocks = 2 * g->sms;
    ok = ok && alloc(g, &g->wpart, wp) && alloc(g, &g->cpart, (size_t)g->cblocks * 128) &&
         alloc(g, &g->hpart, (size_t)g->hblocks * 18) && alloc(g, &g->fault, 1) &&
         cudaMemset(g->fault, 0, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMemset(g->params, 0, g->nparams * sizeof(float)) == cudaSuccess &&
         cudaMemset(g->adam_m, 0, g->nparams * sizeof(float)) == cudaSuccess &&
         cudaMemset(g->adam_v, 0, g->nparams * sizeof(float)) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        qumond_guess_destroy(g);
        return QUMOND_ERR_CUDA;
    }
    prepare_conv3();
    prepare_wgrad();
    prepare_conv3_tc();
    {
        int dev = 0, major = 0, minor = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        g->tc_ok = (major == 10 && minor == 3) ? 1 : 0;
        g->use_tc = g->tc_ok;
    }
    refresh_bf16(g, nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        (void)cudaGetLastError();
        qumond_guess_destroy(g);
        return QUMOND_ERR_CUDA;
    }
    *out = g;
    return QUMOND_OK;
}

void qumond_guess_destroy(qumond_guess* g)
{
    if (!g) return;
    cudaDeviceSynchronize();
    for (void* p : g->allocs) cudaFree(p);
    delete g;
}

qumond_status qumond_guess_tensor_path(qumond_guess* g, int mode)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    if (mode != 0 && mode != 1) return fail(g, QUMOND_ERR_INVALID_ARG, "tensor_path: mode must be 0 or 1");
    if (mode == 1 && !g->tc_ok)
        return fail(g, QUMOND_ERR_INVALID_ARG, "tensor_path: this device has no tcgen05 tensor cores");
    g->use_tc = mode;
    return QUMOND_OK;
}

int qumond_guess_tensor_path_available(qumond_guess* g) { return g && g->tc_ok ? 1 : 0; }

int qumond_guess_tc_selftest(void) { return tc_selftest(); }

int64_t qumond_guess_launches(qumond_guess* g) { return g ? g->launches : 0; }

qumond_status qumond_guess_status(qumond_guess* g, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    int f = 0;
    GTRY(g, cudaMemcpyAsync(&f, g->fault, sizeof(int), cudaMemcpyDeviceToHost, S_(stream)), "status");
    GTRY(g, cudaStreamSynchronize(S_(stream)), "status");
    if (f) {
        GTRY(g, cudaMemset(g->fault, 0, sizeof(int)), "status");
        return fail(g, QUMOND_ERR_TIMEOUT, "a tensor-core convolution gave up waiting for its MMAs");
    }
    return QUMOND_OK;
}

qumond_status qumond_guess_set_params(qumond_guess* g, const float* params, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    if (!dev_ptr(params)) return fail(g, QUMOND_ERR_INVALID_ARG, "set_params: params must be a device pointer");
    cudaStream_t s = S_(stream);
    GTRY(g, cudaMemcpyAsync(g->params, params, g->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s), "set_params");
    GTRY(g, cudaMemsetAsync(g->adam_m, 0, g->nparams * sizeof(float), s), "set_params");
    GTRY(g, cudaMemsetAsync(g->adam_v, 0, g->nparams * sizeof(float), s), "set_params");
    g->step = 0;
    refresh_bf16(g, s);
    GTRY(g, cudaGetLastError(), "set_params");
    return QUMOND_OK;
}

qumond_status qumond_guess_get_params(qumond_guess* g, float* params, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    if (!dev_ptr(params)) return fail(g, QUMOND_ERR_INVALID_ARG, "get_params: params must be a device pointer");
    GTRY(g, cudaMemcpyAsync(params, g->params, g->nparams * sizeof(float), cudaMemcpyDeviceToDevice, S_(stream)),
         "get_params");
    return QUMOND_OK;
}

qumond_status qumond_guess_make_sample(qumond_guess* g, double rho_scale, const double* rho, const double* phiN,
                                       const double* phi, uint16_t* sample, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    if (!dev_ptr(rho) || !dev_ptr(phiN) || !dev_ptr(phi) || !dev_ptr(sample))
        return fail(g, QUMOND_ERR_INVALID_ARG, "make_sample: every array must be a device pointer");
    g->launches += 1;
    launch_make_sample(rho, phiN, phi, g->S, rho_scale, 1.0 / g->phi_scale, reinterpret_cast<__nv_bfloat16*>(sample),
                       S_(stream));
    GTRY(g, cudaGetLastError(), "make_sample");
    return QUMOND_OK;
}

qumond_status qumond_guess_forward(qumond_guess* g, const uint16_t* sample, float box_flag, float* y, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    if (!dev_ptr(sample) || !dev_ptr(y)) return fail(g, QUMOND_ERR_INVALID_ARG, "forward: device pointers required");
    cudaStream_t s = S_(stream);
    launch_input_from_sample(reinterpret_cast<const __nv_bfloat16*>(sample), g->S, box_flag, g->X0, s);
    forward(g, s);
    launch_head(g->A[13], g->params + g->head_off, vox(g, 0), y, s);
    g->launches += 2;
    GTRY(g, cudaGetLastError(), "forward");
    return QUMOND_OK;
}

qumond_status qumond_guess_gradients(qumond_guess* g, const uint16_t* const* samples, const float* box_flags,
                                     int nbatch, float* grads, float* loss, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    qumond_status st = check_samples(g, samples, box_flags, nbatch);
    if (st != QUMOND_OK) return st;
    if (!dev_ptr(grads) || (loss && !dev_ptr(loss)))
        return fail(g, QUMOND_ERR_INVALID_ARG, "gradients: grads (and loss) must be device pointers");
    cudaStream_t s = S_(stream);
    st = batch_gradients(g, samples, box_flags, nbatch, loss, s);
    if (st != QUMOND_OK) return st;
    GTRY(g, cudaMemcpyAsync(grads, g->grads, g->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s), "gradients");
    return QUMOND_OK;
}

qumond_status qumond_guess_train_step(qumond_guess* g, const uint16_t* const* samples, const float* box_flags,
                                      int nbatch, float lr, float* loss, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    qumond_status st = check_samples(g, samples, box_flags, nbatch);
    if (st != QUMOND_OK) return st;
    if (loss && !dev_ptr(loss)) return fail(g, QUMOND_ERR_INVALID_ARG, "train_step: loss must be a device pointer");
    if (!(lr > 0.0f)) return fail(g, QUMOND_ERR_INVALID_ARG, "train_step: lr must be positive");
    cudaStream_t s = S_(stream);
    st = batch_gradients(g, samples, box_flags, nbatch, loss, s);
    if (st != QUMOND_OK) return st;
    g->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    double p1 = 1.0, p2 = 1.0;
    for (int i = 0; i < g->step; ++i) p1 *= b1, p2 *= b2;
    g->launches += 1;
    launch_adam(g->params, g->grads, g->adam_m, g->adam_v, g->nparams, lr, b1, b2, 1e-8f, (float)(1.0 / (1.0 - p1)),
                (float)(1.0 / (1.0 - p2)), s);
    refresh_bf16(g, s);
    GTRY(g, cudaGetLastError(), "train_step");
    return QUMOND_OK;
}

qumond_status qumond_guess_apply(qumond_guess* g, double rho_scale, float box_flag, const double* rho,
                                 const double* phiN, double* phi, void* stream)
{
    if (!g) return QUMOND_ERR_INVALID_ARG;
    g->err.clear();
    if (!dev_ptr(rho) || !dev_ptr(phiN) || !dev_ptr(phi))
        return fail(g, QUMOND_ERR_INVALID_ARG, "apply: every array must be a device pointer");
    cudaStream_t s = S_(stream);
    launch_input_from_grids(rho, phiN, g->S, rho_scale, 1.0 / g->phi_scale, box_flag, g->X0, s);
    forward(g, s);
    launch_head(g->A[13], g->params + g->head_off, vox(g, 0), g->yhat, s);
    launch_apply_guess(phiN, g->yhat, g->S, g->phi_scale, phi, s);
    g->launches += 3;
    GTRY(g, cudaGetLastError(), "apply");
    return QUMOND_OK;
}

}  // extern "C"
