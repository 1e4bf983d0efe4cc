/*
 * lbm_nn.h -- C ABI of the kernels of the learned warm start.
 *
 * The paper has no counterpart: its method starts every run from the
 * initial phase field and relaxes it with the lattice Boltzmann step.  These
 * entry points train and run a small convolutional encoder-decoder that maps
 * (solid indicator phi0, initial phi1, cos theta) to a phase field near
 * equilibrium; the lattice Boltzmann step of lbm.h then relaxes that field,
 * so the method's own steps still decide the final state.
 *
 * Conventions.  Every tensor pointer is a device pointer owned by the
 * caller; nothing here allocates.  Activations are float32 NHWC (pixel
 * p = (n h + y) w + x, channel innermost).  Convolution weights are a BF16
 * copy [tap][cout][cin] (tap = 3 ky + kx) of float32 master weights; 3x3
 * convolutions use zero padding, stride 1, BF16 operands (activations are
 * rounded to BF16 as they enter) and FP32 accumulation on the tensor cores.
 * Work is enqueued on `stream` (a cudaStream_t, may be NULL).  Each call
 * returns 0, -1 for an invalid argument (nothing enqueued) or -3 when the
 * launch failed.
 */
#ifndef LBM_NN_H_
#define LBM_NN_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* y[p][co] = act(bias[co] + sum_{tap, ci} x[p + shift(tap)][ci] wt[tap][co][ci]),
 * act = ReLU when relu != 0.  cin a multiple of 16, cout of 32; bias may be NULL.
 * Runs on the tcgen05 tensor cores (FP32 accumulator in tensor memory); a
 * CTA whose bounded wait for its matrix products gives up writes nothing and
 * raises the flag that lbm_nn_check reports. */
int lbm_nn_conv3x3(const float* x, const void* wt_bf16, const float* bias, float* y, int n, int h, int w,
                   int cin, int cout, int relu, void* stream);

/* 0, or -5 when a convolution since the last call gave up waiting for the
 * tensor cores (its output is incomplete); clears the flag.  Synchronous with
 * respect to the device (reads a device flag), -3 on a CUDA error. */
int lbm_nn_check(void);

/* Floats of workspace lbm_nn_conv3x3_wgrad needs for this shape. */
long long lbm_nn_wgrad_workspace(int n, int h, int w, int cin, int cout);

/* Weight and bias gradients of lbm_nn_conv3x3 (before its activation):
 * dw[tap][co][ci] = sum_p dy[p][co] x[p + shift(tap)][ci] and db[co] = sum_p dy[p][co]
 * (db may be NULL), both overwritten; x and dy are rounded to BF16 as for the
 * forward pass (db sums dy unrounded).  Deterministic: per-chunk partial sums
 * in `work` (work_len floats) are added in a fixed order.  cin a multiple of
 * 16, cout of 16. */
int lbm_nn_conv3x3_wgrad(const float* x, const float* dy, float* dw, float* db, float* work, long long work_len,
                         int n, int h, int w, int cin, int cout, void* stream);

/* wf[tap][ci][co] = wt[8 - tap][co][ci]: with it, lbm_nn_conv3x3(dy, wf, NULL, dx,
 * ..., cin = cout, cout = cin, 0) gives the data gradient of the convolution. */
int lbm_nn_flip_transpose(const void* wt_bf16, void* wf_bf16, int cin, int cout, void* stream);

/* dx[i] = dy[i] where y[i] > 0, else 0: the gradient through a ReLU whose
 * output is y.  dx may be dy. */
int lbm_nn_relu_bwd(const float* dy, const float* y, float* dx, long long n, void* stream);

/* 2x2 average pooling of an (n, h, w, c) tensor into (n, h/2, w/2, c); with
 * backward != 0 its adjoint: x = gradient of the pooled tensor, y = gradient of
 * the (n, h, w, c) input.  h and w even. */
int lbm_nn_pool2(const float* x, float* y, int n, int h, int w, int c, int backward, void* stream);

/* Nearest 2x upsampling of an (n, h, w, c) tensor into (n, 2h, 2w, c); with
 * backward != 0 its adjoint (sum of each 2x2 block), h and w the coarse size. */
int lbm_nn_up2(const float* x, float* y, int n, int h, int w, int c, int backward, void* stream);

/* z[i] = x[i] + a y[i]; z may be x or y. */
int lbm_nn_add(float* z, const float* x, const float* y, float a, long long n, void* stream);

/* Network input x[p][16] = (phi0, phi1, cos theta of the image, 0, ..., 0);
 * costh holds n values. */
int lbm_nn_pack_input(const float* phi0, const float* phi1, const float* costh, float* x, int n, int h, int w,
                      void* stream);

/* Residual prediction pred[p] = base[p] + out[p][0] (out has cpad channels);
 * *loss = sum_p (pred - target)^2 in float64 (work: at least ceil(P / 128)
 * doubles); dout[p][0] = 2 (pred - target) / P, other channels 0. */
int lbm_nn_mse_residual(const float* out, int cpad, const float* base, const float* target, float* dout,
                        double* work, long long work_len, double* loss, long long P, void* stream);

/* Adam step t >= 1 with bias correction on float32 master weights w (moments
 * m, v); writes the BF16 copy w_bf16 when it is not NULL. */
int lbm_nn_adam(float* w, float* m, float* v, const float* grad, void* w_bf16, long long n, float lr, float b1,
                float b2, float eps, int t, void* stream);

/* b = BF16(a), round to nearest even. */
int lbm_nn_to_bf16(const float* a, void* b, long long n, void* stream);

/* Warm-start field from the network output: per pixel the prediction is
 * phi1[p] + out[p][0] (out has cpad channels), clamped to [0, hi], hi =
 * max(1 - phi0, 0).  Then three correction passes per image: field +=
 * lambda b(field) with the bump b(q) = q (hi - q) / hi (0 where hi = 0) and
 * lambda = clamp((sum phi1 - sum field) / sum b, -1, 1), which restores the
 * phase mass of the initial field (sum phi1) while every value stays in
 * [0, hi] (for |lambda| <= 1 the correction is monotone with fixed points 0
 * and hi).  work: at least 192 n doubles. */
int lbm_nn_project(const float* out, int cpad, const float* phi0, const float* phi1, float* field, double* work,
                   long long work_len, int n, int h, int w, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NN_H_ */
