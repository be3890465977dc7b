/*
 * pns_unet.h -- C ABI of the learned Newton initial guess of libpns: a 3D U-Net that maps the solid
 * mask, the Stokes solution and the Reynolds number of an image to a correction of the Stokes
 * solution towards the Navier-Stokes solution (single GPU, NVIDIA GB300, sm_103a).
 *
 * The paper has no such network: it only notes that the initial iterate is Newton's weak point
 * (Sec. 9.4) and starts Newton from the Stokes solution or a nearby converged state (Sec. 4, Sec. 8).
 * The architecture and encodings below are this library's:
 *
 *   levels L (1..5) with channels c_0..c_{L-1} (each a multiple of 8, at most 128);
 *   encoder level l: two 3x3x3 convolutions (zero padding 1, bias), each followed by ReLU; a 2x2x2
 *     max-pool between levels (ties go to the first element in (dz, dy, dx) order);
 *   decoder level l < L-1: nearest 2x upsampling of level l+1's output, concatenated (upsampled channels
 *     first, then the encoder output of level l), two 3x3x3 convolutions with ReLU;
 *   head: a 1x1x1 convolution to the output channels, no activation.
 *
 * Parameters (FP32 master copy, flat, in this order): for each convolution enc0.0, enc0.1, ...,
 * enc{L-1}.1, dec{L-2}.0, dec{L-2}.1, ..., dec0.1, head: its weight w[o][c][kz][ky][kx] then its bias b[o].
 * Activations are BF16 (channels-last inside the library), every product accumulates in FP32 on the
 * tensor cores (tcgen05.mma kind::f16), and the optimiser (Adam) updates the FP32 master weights.
 *
 * Tensors at this boundary are DEVICE pointers to FP32 arrays in (N, C, D, H, W) order, C order,
 * caller-owned.  D, H, W must be multiples of 2^(L-1).  Every call enqueues on the stream given at
 * creation and returns without synchronising unless stated.  Errors: PNS_OK (0) or a negative
 * PNS_ERR_* code of pns.h; the message is kept (pns_unet_last_error).
 */
#ifndef PNS_UNET_H
#define PNS_UNET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pns_unet pns_unet;

/* Create a network and the device buffers for inputs of shape (batch, in_ch, nz, ny, nx); later calls
 * may use any batch <= `batch` and any dimensions whose voxel count does not exceed nz*ny*nx and that
 * are multiples of 2^(levels-1).  Parameters start as He-normal weights (seeded), zero biases and a zero head
 * (so that the untrained network proposes no correction).
 * channels: `levels` entries.  stream: a cudaStream_t (NULL = legacy default).  Synchronises. */
int pns_unet_create(pns_unet** out, int levels, const int* channels, int in_ch, int out_ch, int batch, int nz,
                    int ny, int nx, uint64_t seed, void* stream);

/* Free everything the network holds.  NULL is accepted. */
void pns_unet_destroy(pns_unet* net);

/* Message of the last error ("" if none). */
const char* pns_unet_last_error(const pns_unet* net);

/* Number of parameters (FP32 entries of the flat parameter vector). */
long long pns_unet_num_params(const pns_unet* net);

/* Copy the flat FP32 parameters from / to a HOST array of pns_unet_num_params entries; set also resets
 * the optimiser state.  Synchronises. */
int pns_unet_set_params(pns_unet* net, const float* params);
int pns_unet_get_params(const pns_unet* net, float* params);

/* Copy the gradients of the last pns_unet_backward (flat, the parameter order) to a HOST array.
 * Synchronises. */
int pns_unet_get_grads(const pns_unet* net, float* grads);

/* out (batch, out_ch, nz, ny, nx) = network(x), x (batch, in_ch, nz, ny, nx).  Keeps the activations
 * for a following pns_unet_backward. */
int pns_unet_forward(pns_unet* net, const float* x, int batch, int nz, int ny, int nx, float* out);

/* Gradients of a scalar loss with respect to every parameter, given gout = dL/d(out) of the last
 * forward (batch, out_ch, nz, ny, nx).  Overwrites the gradient buffer. */
int pns_unet_backward(pns_unet* net, const float* gout);

/* Masked mean-squared error of the last forward's output against target (same shape), weighted by
 * weight (batch, 1, nz, ny, nx): L = sum(w (out - t)^2) / sum(w) over every channel (weight is
 * broadcast over channels).  Writes gout = dL/d(out) (device, may be NULL) and *loss (HOST).
 * Synchronises. */
int pns_unet_mse(pns_unet* net, const float* out, const float* target, const float* weight, int batch, int nz,
                 int ny, int nx, float* gout, double* loss);

/* One Adam step (Kingma & Ba 2015, bias-corrected moments) on the FP32 master parameters with the
 * gradients of the last backward: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
 * theta <- theta - lr m_hat / (sqrt(v_hat) + eps); refreshes the BF16 working weights. */
int pns_unet_adam(pns_unet* net, float lr, float b1, float b2, float eps);

/* forward + masked MSE + backward + Adam in one call; *loss (HOST) is the loss before the update.
 * Synchronises (to read the loss). */
int pns_unet_train_step(pns_unet* net, const float* x, const float* target, const float* weight, int batch, int nz,
                        int ny, int nx, float lr, double* loss);

/* Input encoding of one 3D image (batch entry `b` of x, shape (., in_ch = 6, nz, ny, nx)):
 *   channel 0 the void mask; 1..3 the Stokes velocities u_x, u_y, u_z (the face arrays of the low-face
 *   convention of pns.h, image-shaped) divided by U = max |u|; 4 the Stokes pressure divided by
 *   P = max |p| (1 when zero); 5 log10(re) everywhere.
 * mask: DEVICE uint8 (nz*ny*nx); x_stokes: DEVICE FP64 full layout of pns.h (4 * nz*ny*nx).
 * scales (HOST, may be NULL) receives {U, P}.  Synchronises. */
int pns_unet_features(pns_unet* net, const uint8_t* mask, const double* x_stokes, double re, int nz, int ny, int nx,
                      float* x, int b, double* scales);

/* Target encoding: t[b] (4, nz, ny, nx) = (x_ns - x_stokes) / (U, U, U, P), and the loss weight
 * w[b] (1, nz, ny, nx) = the void mask.  x_ns, x_stokes: DEVICE FP64 full layout. */
int pns_unet_targets(pns_unet* net, const uint8_t* mask, const double* x_ns, const double* x_stokes, double u_scale,
                     double p_scale, int nz, int ny, int nx, float* t, float* w, int b);

/* Decoding: x_out (DEVICE FP64 full layout) = x_stokes + (out[b] channels scaled back by U, U, U, P), entries
 * that are not unknowns are set by the caller's next pns_residual (the library ignores them). */
int pns_unet_proposal(pns_unet* net, const float* out, int b, const double* x_stokes, double u_scale, double p_scale,
                      int nz, int ny, int nx, double* x_out);

#ifdef __cplusplus
}
#endif

#endif /* PNS_UNET_H */
