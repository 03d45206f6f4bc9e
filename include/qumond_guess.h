/*
 * qumond_guess.h -- C ABI of the learned initial guess for the QUMOND solve.
 *
 * The paper starts every solve from FMG (Section 2) and remarks that a good
 * initial guess shortens the iteration; it has no learned component.  This
 * part adds one: a small 3-D U-Net that maps the density and Newtonian
 * potential of a box to Phi - Phi_N, the QUMOND correction (Eq. 2), so that
 * the second solve of the box can start from Phi_N + (network output) and run
 * V-cycles to the tolerance instead of FMG (qumond_params.warm_start = 1).
 * FMG stays the default and the fallback; the network is measured by the
 * residual it starts from and the V-cycles it saves.
 *
 * Network (fixed): input S^3 voxels x 16 channels, voxel (x,y,z) = node
 * (x,y,z) of the box's (S+1)^3 grid (S = n, a multiple of 16, >= 16):
 *   channel 0 = rho_scale * rho, channel 1 = Phi_N / phi_scale,
 *   channel 2 = box flag (0 outermost box, 1 inner boxes), channels 3..15 = 0.
 * Four levels S, S/2, S/4, S/8 with 16, 32, 64, 128 channels; every
 * convolution 3x3x3 (zero padding) + bias + ReLU; two per level on the way
 * down (2x2x2 average pooling between levels) and two per level on the way
 * up (nearest-neighbour upsampling, then concatenation [upsampled, skip]);
 * a 1x1x1 head (16 -> 1, bias, no ReLU) gives y = (Phi - Phi_N) / phi_scale.
 * Layers, in order (cin -> cout): 16->16, 16->16 | 16->32, 32->32 |
 * 32->64, 64->64 | 64->128, 128->128 | 192->64, 64->64 | 96->32, 32->32 |
 * 48->16, 16->16 | head 16->1.
 * Parameters: one FP32 array, per layer W[cout][27][cin] (tap = (dz+1)*9 +
 * (dy+1)*3 + (dx+1), input voxel v + (dx,dy,dz)) then b[cout]; then the
 * head's w[16], b.  Arithmetic: BF16 weights and activations, FP32
 * accumulation, FP32 head output.
 *
 * Training samples: one BF16 array (uint16 bit patterns) of 3 S^3 values,
 * [0] the rho channel, [1] the Phi_N channel, [2] the target
 * (Phi - Phi_N) / phi_scale, written by qumond_guess_make_sample.  The loss
 * of a batch is the mean over samples of the mean over voxels of
 * (y - target)^2; the optimiser is Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 *
 * Conventions: as qumond.h (device pointers owned by the caller, stream as
 * void*, argument errors before anything is queued, one host thread per
 * object, calls of one object must not overlap on the GPU).  On error
 * qumond_guess_last_error(g) describes it.
 */
#ifndef QUMOND_GUESS_H
#define QUMOND_GUESS_H

#include "qumond.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qumond_guess qumond_guess;

/* Number of FP32 parameters of the network (1,466,065). */
QUMOND_API int64_t qumond_guess_num_params(void);

/* Creates a network for inputs of S^3 voxels (S a multiple of 16, 16..512)
   on the current device: parameters, Adam state, BF16 weight copies and
   every activation and gradient buffer of one sample.  The parameters start
   at zero: set them before use. */
QUMOND_API qumond_status qumond_guess_create(int S, double phi_scale, qumond_guess** out);
QUMOND_API void qumond_guess_destroy(qumond_guess* g);
QUMOND_API const char* qumond_guess_last_error(qumond_guess* g);

/* Convolution path: mode 1 (the default when available) runs the 3x3x3
   convolutions of levels with S >= 16 on the tcgen05 tensor cores with TMEM
   accumulators; mode 0 runs every convolution with mma.sync.  The tcgen05
   path is available on devices of compute capability 10.3 (the architecture
   the library is built for); mode 1 is rejected (QUMOND_ERR_INVALID_ARG)
   otherwise.  Both give FP32-accumulated BF16 results. */
QUMOND_API qumond_status qumond_guess_tensor_path(qumond_guess* g, int mode);
QUMOND_API int qumond_guess_tensor_path_available(qumond_guess* g);

/* A unit test of the tcgen05 path's shared-memory descriptors (the PTX ISA's
   canonical K-major layout without swizzling): one 128 x 16 x 16 BF16 MMA
   from descriptors built as the convolution builds them, read back from
   tensor memory and compared with the CPU product of the same small
   integers.  Returns 1 if every element matches, 0 if not, -1 on a CUDA
   error.  Uses the current device; not called by any other entry point. */
QUMOND_API int qumond_guess_tc_selftest(void);

/* Kernels this object has enqueued since it was created: every call above
   and below adds the kernels it launched (0 for a null object). */
QUMOND_API int64_t qumond_guess_launches(qumond_guess* g);

/* Synchronises `stream` and reports QUMOND_ERR_TIMEOUT (and clears the flag)
   if a tensor-core convolution gave up a bounded wait since the last call;
   the outputs of such calls are undefined. */
QUMOND_API qumond_status qumond_guess_status(qumond_guess* g, void* stream);

/* Copies num_params FP32 values from / to a device array; setting also
   resets the Adam state. */
QUMOND_API qumond_status qumond_guess_set_params(qumond_guess* g, const float* params, void* stream);
QUMOND_API qumond_status qumond_guess_get_params(qumond_guess* g, float* params, void* stream);

/* A training sample from one solved box: rho, phiN, phi are the box's
   (S+1)^3 FP64 grids; sample receives 3 S^3 BF16 values (see above). */
QUMOND_API qumond_status qumond_guess_make_sample(qumond_guess* g, double rho_scale, const double* rho,
                                                  const double* phiN, const double* phi, uint16_t* sample,
                                                  void* stream);

/* Network output y (S^3 FP32, voxel order) for the inputs of a sample. */
QUMOND_API qumond_status qumond_guess_forward(qumond_guess* g, const uint16_t* sample, float box_flag, float* y,
                                              void* stream);

/* Loss of a batch and its gradient with respect to every parameter (FP32,
   num_params values, the parameter layout above), without an update.
   samples, box_flags: HOST arrays of nbatch entries (device sample pointers,
   flags).  loss: device float, or NULL. */
QUMOND_API qumond_status qumond_guess_gradients(qumond_guess* g, const uint16_t* const* samples,
                                                const float* box_flags, int nbatch, float* grads, float* loss,
                                                void* stream);

/* One Adam step on a batch (gradients as qumond_guess_gradients), learning
   rate lr.  loss: device float receiving the batch loss before the step, or NULL. */
QUMOND_API qumond_status qumond_guess_train_step(qumond_guess* g, const uint16_t* const* samples,
                                                 const float* box_flags, int nbatch, float lr, float* loss,
                                                 void* stream);

/* Inference: phi = phiN + phi_scale * y on the interior nodes (1..S-1 on
   each axis) of the box, from the box's rho and phiN ((S+1)^3 FP64 grids);
   the boundary nodes of phi are left as they are (the solve sets them). */
QUMOND_API qumond_status qumond_guess_apply(qumond_guess* g, double rho_scale, float box_flag, const double* rho,
                                            const double* phiN, double* phi, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* QUMOND_GUESS_H */
