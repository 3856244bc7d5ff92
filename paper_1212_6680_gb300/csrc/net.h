// net.h -- the learned post-correction of the (1,0) SMG cycle inside flexible PCG (not part of
// arXiv:1212.6680; eq. (2) is what lets the preconditioner be nonlinear).
//
// Network: 3x3x3 convolutions 1 -> 16 -> 16 -> 1 channels, zero padding, no bias, ReLU after the
// first two; the input residual is divided by its RMS and the output multiplied back.  Weights
// (7776, FP32 master copy on the device) are in the layer order and [out][in][tap] layout of the
// C ABI, tap t = (dz+1)*9 + (dy+1)*3 + (dx+1).  Activations are channel-last, [point][16], in
// BF16 (the product path) or FP32 (the reference-accuracy path of the gradient checks); the
// backward pass keeps its gradient tensors in FP32 on both; every sum accumulates in FP32.
#pragma once

#include <cuda_runtime.h>

#include "smg_internal.h"

namespace smg {

constexpr int kNetC = 16;
constexpr int kNetW1 = 0;                               // [16][1][27]
constexpr int kNetW2 = kNetC * 27;                      // [16][16][27]
constexpr int kNetW3 = kNetW2 + kNetC * kNetC * 27;     // [1][16][27]
constexpr int kNetWeights = kNetW3 + kNetC * 27;        // 7776

// Device scalars of one forward / training step.
struct NetScal {
    double rr;          // sum rho^2 (the judge's "before")
    double rms, inv_rms;
    double num, den;    // (e - delta)^T A (e - delta), e^T A e
    double loss, gscale;  // num / den, -2 rms / den
    double after;       // sum (rho - A delta)^2
    double loss_sum;    // sum of the losses since the last reset
    long long calls, accepts;
    int accepted;
    int pad;
};

// Buffers for one grid size.  act: 0 BF16 activations, 1 FP32.
struct NetWork {
    long long n = 0;
    int act = 0;
    bool training = false;
    void *a1 = nullptr, *a2 = nullptr;   // forward activations [n][16]
    float *g1 = nullptr, *g2 = nullptr;  // masked gradients [n][16], FP32 (training)
    float *rho = nullptr;                // input residual [n]
    float *delta = nullptr;              // correction [n]
    float *e = nullptr;                  // training target [n]
    float *ad = nullptr;                 // A (e - delta) [n] (training)
    double *part = nullptr;              // reduction partials
    NetScal *sc = nullptr;
    float *w = nullptr;                  // master weights [7776]
    void *w2b = nullptr;                 // layer 2 weights as the tensor-core operand
    float *grad = nullptr, *m = nullptr, *v = nullptr;  // training
    float *wpart = nullptr;              // per-block weight-gradient partials
    int wpart_blocks = 0;
    long long launches = 0;
};

cudaError_t net_alloc(NetWork &nw, long long n, int act, bool training);
void net_free(NetWork &nw);

// delta = rms(rho) Net(rho / rms(rho)) from nw.rho (FP32) into nw.delta; keeps a1, a2.
cudaError_t net_forward(NetWork &nw, int nx, int ny, int nz, cudaStream_t st);
// One training step on (nw.rho, nw.e): forward, loss, backward into nw.grad (FP32, 7776).
cudaError_t net_loss_grad(NetWork &nw, int nx, int ny, int nz, cudaStream_t st);
// Adam update of nw.w with nw.grad (step >= 1).
cudaError_t net_adam(NetWork &nw, int step, float lr, cudaStream_t st);

// Inference inside the preconditioner: rho = r - A s (s in storage precision), delta = Net
// correction, judge ||rho - A delta|| < ||rho||, s += delta if accepted -- all on the device.
cudaError_t net_learned_correct(NetWork &nw, Prec storage, int nx, int ny, int nz, const double *r, void *s,
                                cudaStream_t st);

// Training pairs along a flexible PCG run: rho = r - A s, e = xstar - x - s (FP32 outputs).
cudaError_t net_capture(Prec storage, int nx, int ny, int nz, const double *r, const void *s, const double *x,
                        const double *xstar, float *rho_out, float *e_out, cudaStream_t st);

// FP64 -> FP32 conversion of n values (rounding to nearest).
cudaError_t net_to_f32(long long n, const double *src, float *dst, cudaStream_t st);
cudaError_t net_to_f64(long long n, const float *src, double *dst, cudaStream_t st);

// The 16 -> 16 channel layer with ReLU on the tcgen05 tensor cores (BF16 in and out, FP32
// accumulation): conv_tc.cu.  Used for the BF16 layer 2 while net_tensor_cores() is on.
cudaError_t conv16_tc(int nx, int ny, int nz, const void *in, void *out, const void *wb, cudaStream_t st);
// wb (27 * 512 bytes) = the layer's weights w ([16 out][16 in][27] FP32) as conv16_tc's BF16 operand.
cudaError_t conv16_tc_prep(const float *w, void *wb, cudaStream_t st);
constexpr size_t kConv16TcWeightBytes = 27 * 512;
// 1 if a CTA of conv16_tc gave up waiting for its accumulators since the last call (then cleared).
cudaError_t conv16_tc_status(int *err);
bool &net_tensor_cores();

}  // namespace smg
