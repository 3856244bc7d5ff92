// net_api.cpp -- C ABI of the learned post-correction that needs no SMG handle: one forward
// pass, one loss + gradient evaluation, and the training loop (Adam over recorded pairs).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <utility>
#include <string>
#include <vector>

#include "../../include/smg.h"
#include "net.h"
#include "smg_internal.h"

using namespace smg;

namespace {

int nfail(int code, const std::string &msg) {
    set_last_error(msg);
    return code;
}

#define NET_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            net_free(nw);                                                                       \
            return nfail(SMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
        }                                                                                       \
    } while (0)

int check_grid(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1 || nx > kMaxNx || ny > kMaxNy || nz > kMaxNz)
        return nfail(SMG_ERR_ARG, "need 1 <= nx <= 512, 1 <= ny <= 512, 1 <= nz <= 4096");
    return SMG_OK;
}

int act_of(int prec, int *act) {
    if (prec == SMG_BF16) *act = 0;
    else if (prec == SMG_FP32) *act = 1;
    else return nfail(SMG_ERR_ARG, "activation precision must be SMG_BF16 or SMG_FP32");
    return SMG_OK;
}

// SplitMix64 (Steele, Lea, Flood 2014): the shuffle order of the training pairs.
uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" int smg_net_forward(int nx, int ny, int nz, int act_prec, const float *w, const double *rho, double *delta,
                               void *stream) {
    if (int rc = check_grid(nx, ny, nz)) return rc;
    int act = 0;
    if (int rc = act_of(act_prec, &act)) return rc;
    if (!w || !rho || !delta) return nfail(SMG_ERR_ARG, "null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = static_cast<long long>(nx) * ny * nz;
    NetWork nw;
    NET_CUDA(net_alloc(nw, n, act, false));
    NET_CUDA(cudaMemcpyAsync(nw.w, w, kNetWeights * sizeof(float), cudaMemcpyHostToDevice, st));
    NET_CUDA(net_to_f32(n, rho, nw.rho, st));
    NET_CUDA(net_forward(nw, nx, ny, nz, st));
    NET_CUDA(net_to_f64(n, nw.delta, delta, st));
    NET_CUDA(cudaStreamSynchronize(st));
    net_free(nw);
    return SMG_OK;
}

extern "C" int smg_net_loss_grad(int nx, int ny, int nz, int act_prec, const float *w, const double *rho,
                                 const double *e, double *loss, float *grad, void *stream) {
    if (int rc = check_grid(nx, ny, nz)) return rc;
    int act = 0;
    if (int rc = act_of(act_prec, &act)) return rc;
    if (!w || !rho || !e || !loss || !grad) return nfail(SMG_ERR_ARG, "null pointer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = static_cast<long long>(nx) * ny * nz;
    NetWork nw;
    NET_CUDA(net_alloc(nw, n, act, true));
    NET_CUDA(cudaMemcpyAsync(nw.w, w, kNetWeights * sizeof(float), cudaMemcpyHostToDevice, st));
    NET_CUDA(net_to_f32(n, rho, nw.rho, st));
    NET_CUDA(net_to_f32(n, e, nw.e, st));
    NET_CUDA(net_loss_grad(nw, nx, ny, nz, st));
    NetScal sc;
    NET_CUDA(cudaMemcpyAsync(&sc, nw.sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
    NET_CUDA(cudaMemcpyAsync(grad, nw.grad, kNetWeights * sizeof(float), cudaMemcpyDeviceToHost, st));
    NET_CUDA(cudaStreamSynchronize(st));
    *loss = sc.loss;
    net_free(nw);
    return SMG_OK;
}

extern "C" int smg_net_train(int npairs, const int *dims, const float *const *rho, const float *const *e, int epochs,
                             double lr, unsigned long long seed, int act_prec, float *w, double *loss_hist,
                             void *stream) {
    if (npairs < 1 || !dims || !rho || !e || !w || !loss_hist) return nfail(SMG_ERR_ARG, "null pointer or npairs < 1");
    if (epochs < 1 || !(lr > 0.0) || !std::isfinite(lr)) return nfail(SMG_ERR_ARG, "epochs >= 1 and lr > 0 required");
    int act = 0;
    if (int rc = act_of(act_prec, &act)) return rc;
    long long nmax = 0;
    for (int i = 0; i < npairs; ++i) {
        if (int rc = check_grid(dims[3 * i], dims[3 * i + 1], dims[3 * i + 2])) return rc;
        if (!rho[i] || !e[i]) return nfail(SMG_ERR_ARG, "null pair pointer");
        nmax = std::max<long long>(nmax, static_cast<long long>(dims[3 * i]) * dims[3 * i + 1] * dims[3 * i + 2]);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    NetWork nw;
    NET_CUDA(net_alloc(nw, nmax, act, true));
    NET_CUDA(cudaMemcpyAsync(nw.w, w, kNetWeights * sizeof(float), cudaMemcpyHostToDevice, st));
    // the pairs are read in place: the work buffers' own input / target arrays are set aside
    float *own_rho = nw.rho, *own_e = nw.e;
    std::vector<int> order(npairs);
    uint64_t rs = seed;
    int step = 0;
    cudaError_t err = cudaSuccess;
    for (int ep = 0; ep < epochs && err == cudaSuccess; ++ep) {
        for (int i = 0; i < npairs; ++i) order[i] = i;
        for (int i = npairs - 1; i > 0; --i) {  // Fisher-Yates
            const int j = static_cast<int>(splitmix64(rs) % static_cast<uint64_t>(i + 1));
            std::swap(order[i], order[j]);
        }
        err = cudaMemsetAsync(&nw.sc->loss_sum, 0, sizeof(double), st);
        for (int k = 0; k < npairs && err == cudaSuccess; ++k) {
            const int i = order[k];
            nw.rho = const_cast<float *>(rho[i]);
            nw.e = const_cast<float *>(e[i]);
            err = net_loss_grad(nw, dims[3 * i], dims[3 * i + 1], dims[3 * i + 2], st);
            if (err == cudaSuccess) err = net_adam(nw, ++step, static_cast<float>(lr), st);
        }
        nw.rho = own_rho;
        nw.e = own_e;
        double ls = 0.0;
        if (err == cudaSuccess) err = cudaMemcpyAsync(&ls, &nw.sc->loss_sum, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        loss_hist[ep] = ls / npairs;
    }
    nw.rho = own_rho;
    nw.e = own_e;
    NET_CUDA(err);
    NET_CUDA(cudaMemcpyAsync(w, nw.w, kNetWeights * sizeof(float), cudaMemcpyDeviceToHost, st));
    NET_CUDA(cudaStreamSynchronize(st));
    net_free(nw);
    return SMG_OK;
}

extern "C" int smg_net_set_tensor_cores(int on) {
    if (on != 0 && on != 1) return nfail(SMG_ERR_ARG, "on must be 0 or 1");
    net_tensor_cores() = (on == 1);
    return SMG_OK;
}

extern "C" int smg_net_tc_status(int *err) {
    if (!err) return nfail(SMG_ERR_ARG, "null pointer");
    cudaError_t e = conv16_tc_status(err);
    if (e != cudaSuccess) return nfail(SMG_ERR_CUDA, std::string("smg_net_tc_status: ") + cudaGetErrorString(e));
    return SMG_OK;
}
