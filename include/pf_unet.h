/*
 * pf_unet.h -- C ABI of the warm-start network of the displacement solve.
 *
 * The mechanics step of the model solves the equilibrium of Sec. 2.4
 * (div sigma = 0 with the transformation eigenstrain of Sec. 2.2) by PCG.
 * This network predicts that solve's displacement from per-cell inputs, so
 * that the PCG starts near the answer; the PCG's residual test still decides
 * every step, so results never depend on the network's accuracy.
 *
 * Network: periodic U-Net on a 2D or 3D grid.  Level l = 0..levels-1 has
 * channels[l] channels; each level's encoder is two 3^D convolutions with
 * ReLU, levels are linked by 2^D average pooling, each decoder level
 * concatenates the encoder output (skip) with the nearest-neighbour upsampled
 * coarser decoder output and applies two 3^D convolutions with ReLU; a 1x1
 * convolution maps channels[0] to ndim outputs.  Every convolution has a
 * bias and wraps periodically.
 *
 * Parameters: one flat FP32 vector; for each convolution, in the order
 * enc_0a, enc_0b, ..., enc_{L-1}b, dec_{L-2}a, dec_{L-2}b, ..., dec_0a,
 * dec_0b, out, the weights W[c_out][c_in][taps] (taps row-major over
 * (dz,) dy, dx, tap offset = index - 1) followed by the bias b[c_out].
 *
 * Arithmetic: BF16 activations and weights on the tensor cores with FP32
 * accumulation; FP32 master weights, gradients and Adam moments.
 *
 * Arrays: inputs (cin channels) and outputs/targets (ndim channels) are FP32
 * device arrays, channels last: a[((b * cells) + p) * C + c], p the x-fastest
 * cell index of sample b.  Grid sizes: nx % 2^(levels-1) * 16 == 0 and, in 2D,
 * ny % 2^(levels-1) * 8 == 0; in 3D ny % 2^(levels-1) * 4 == 0 and
 * nz % 2^(levels-1) * 2 == 0 (PF_EINVAL otherwise).
 *
 * Errors: int status codes of pf.h; pf_unet_last_error(net) gives a text
 * (pf_unet_last_error(NULL): the last failed pf_unet_create).
 */
#ifndef PF_UNET_H
#define PF_UNET_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int ndim;          /* 2 or 3                                              */
    int cin;           /* input channels, 1..16                                */
    int levels;        /* 1..5                                                 */
    int channels[5];   /* per level, each a multiple of 16, at most 64         */
} pf_unet_config;

typedef struct pf_unet pf_unet;

int pf_unet_create(const pf_unet_config *cfg, pf_unet **out);
long long pf_unet_param_count(const pf_unet *net);
/* Copy the flat FP32 parameter vector in / out (host arrays of
 * pf_unet_param_count floats).  Setting resets the Adam state. */
int pf_unet_set_params(pf_unet *net, const float *host);
int pf_unet_get_params(pf_unet *net, float *host);

/* out = net(in) for nb samples of nx * ny * nz cells (device arrays). */
int pf_unet_forward(pf_unet *net, const float *in, float *out, int nb, int nx, int ny, int nz, void *cudaStream);

/* Training loss (e = net(in) - target, n = cells * ndim over the batch):
 *   PF_UNET_LOSS_MSE  (default)  (1/n) sum |e|^2
 *   PF_UNET_LOSS_GRAD            (1/n) sum_p w_p sum_d |e(p + e_d) - e(p)|^2,
 *     periodic forward differences, w_p = floor + (1 - floor)(1 - in[p, weight_channel])
 *     (with the gas weight as channel: the error of the displacement
 *     gradient where the material is stiff, a stand-in for the energy norm
 *     the PCG reduces; blind to rigid translations).
 * PF_EINVAL for an unknown kind, a channel outside 0..cin-1 or floor
 * outside [0, 1]. */
enum { PF_UNET_LOSS_MSE = 0, PF_UNET_LOSS_GRAD = 1 };
int pf_unet_set_loss(pf_unet *net, int kind, int weight_channel, double floor);

/* The training loss of net(in) against target and its gradient with
 * respect to the parameters, kept for pf_unet_adam_step; *loss (host)
 * receives the loss, grad_host (nullable) a copy of the gradient. */
int pf_unet_loss_grad(pf_unet *net, const float *in, const float *target, int nb, int nx, int ny, int nz,
                      double *loss, float *grad_host, void *cudaStream);

/* One Adam step (Kingma & Ba 2015) with the gradient of the last
 * pf_unet_loss_grad; beta1 = 0.9, beta2 = 0.999, eps = 1e-8. */
int pf_unet_adam_step(pf_unet *net, double lr, void *cudaStream);

const char *pf_unet_last_error(const pf_unet *net);
void pf_unet_destroy(pf_unet *net);

#ifdef __cplusplus
}
#endif
#endif
