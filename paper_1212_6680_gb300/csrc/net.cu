// net.cu -- kernels of the learned post-correction (see net.h): 3x3x3 convolutions on
// channel-last activations (forward, and the adjoint in the input for the backward pass, which
// is the same convolution with the taps mirrored and the channels transposed), per-block weight
// gradients reduced in FP64, the energy-norm loss, Adam, and the residual / judge / update
// kernels of the preconditioner.
//
// Convolution tiling: a CTA computes a 32 x 4 x 4 block of output points (256 threads, two
// points each: one x-row of 32 per warp, two (y, z) rows per thread) from a 34 x 6 x 6 halo
// tile of the input held in shared memory, with the layer's weights (as FP32, rounded to BF16
// first on the BF16 path) in shared memory too.  A multi-channel input tile is stored as
// 16-byte channel chunks, chunk-major ([chunk][z][y][x]), so the lanes of a warp, which read
// consecutive x, touch consecutive 16-byte words.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "net.h"
#include "plane_relax.cuh"

namespace smg {
namespace {

constexpr int TX = 32, TY = 4, TZ = 4;
constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2, HP = HX * HY * HZ;  // 1224 halo points
constexpr int TP = TX * TY * TZ;                                          // 512 tile points
constexpr int kRegion = HP * 16 + 64;  // bytes per channel chunk (the 64 B pad staggers banks)
constexpr int kConvThreads = 256;
constexpr int kWgThreads = 448;        // 432 = 27 taps x 16 used
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 608;        // 4 x 152 SMs
enum : int { EPI_RELU = 1, EPI_MASK = 2, EPI_SCALE = 4 };

// ---- 16-byte chunks of channels ---------------------------------------------------------------
template <class T> struct Chunk;
template <> struct Chunk<float> {
    static constexpr int E = 4;
    static __device__ __forceinline__ void unpack(const uint4 &u, float *f) {
        f[0] = __uint_as_float(u.x);
        f[1] = __uint_as_float(u.y);
        f[2] = __uint_as_float(u.z);
        f[3] = __uint_as_float(u.w);
    }
    static __device__ __forceinline__ uint4 pack(const float *f) {
        return make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]), __float_as_uint(f[3]));
    }
    static __device__ __forceinline__ float elem(const unsigned char *p, int i) {
        return reinterpret_cast<const float *>(p)[i];
    }
};
template <> struct Chunk<__nv_bfloat16> {
    static constexpr int E = 8;
    // a BF16 value is the upper half of the FP32 with the same bits: widening is a shift
    static __device__ __forceinline__ void unpack(const uint4 &u, float *f) {
        const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            f[2 * k] = __uint_as_float(w[k] << 16);
            f[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    static __device__ __forceinline__ uint4 pack(const float *f) {
        unsigned w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __nv_bfloat162 b = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
            w[k] = *reinterpret_cast<unsigned *>(&b);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
    static __device__ __forceinline__ float elem(const unsigned char *p, int i) {
        const unsigned short b = reinterpret_cast<const unsigned short *>(p)[i];
        return __uint_as_float(static_cast<unsigned>(b) << 16);
    }
};

struct ConvArgs {
    int nx, ny, nz;
    const void *in;       // CIN == 1: float [n]; else TI [n][16]
    void *out;            // COUT == 1: float [n]; else TO [n][16]
    const float *w;       // the layer's master weights [cout][cin][27]
    const void *mask;     // EPI_MASK: TM [n][16]; an output channel is kept where mask > 0
    const double *scale;  // EPI_SCALE: the output is multiplied by *scale
    int wround;           // round the weights to BF16 when staging them
};

template <int CIN, int COUT, class T>
constexpr size_t conv_smem_bytes() {  // T: the type of a multi-channel input
    return static_cast<size_t>((27 * CIN * COUT * 4 + 15) / 16 * 16) +
           (CIN == 1 ? static_cast<size_t>(HP) * 4 : static_cast<size_t>(CIN / Chunk<T>::E) * kRegion);
}

__device__ __forceinline__ void tile_origin(int b, int nx, int ny, int &x0, int &y0, int &z0) {
    const int ntx = (nx + TX - 1) / TX, nty = (ny + TY - 1) / TY;
    x0 = (b % ntx) * TX;
    b /= ntx;
    y0 = (b % nty) * TY;
    z0 = (b / nty) * TZ;
}

// Stage the input halo tile of a tile with origin (x0, y0, z0); zeros outside the grid.
template <int CIN, class T>
__device__ __forceinline__ void stage_input(unsigned char *xs, const void *in, int nx, int ny, int nz, int x0, int y0,
                                            int z0) {
    if constexpr (CIN == 1) {
        float *xf = reinterpret_cast<float *>(xs);
        const float *src = static_cast<const float *>(in);
        for (int i = threadIdx.x; i < HP; i += blockDim.x) {
            const int hx = i % HX, hy = (i / HX) % HY, hz = i / (HX * HY);
            const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
            float v = 0.0f;
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
                v = src[(static_cast<long long>(gz) * ny + gy) * nx + gx];
            xf[i] = v;
        }
    } else {
        constexpr int NG = CIN / Chunk<T>::E;
        const unsigned char *src = static_cast<const unsigned char *>(in);
        for (int i = threadIdx.x; i < NG * HP; i += blockDim.x) {
            const int g = i % NG, pt = i / NG;
            const int hx = pt % HX, hy = (pt / HX) % HY, hz = pt / (HX * HY);
            const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz) {
                const long long p = (static_cast<long long>(gz) * ny + gy) * nx + gx;
                v = *reinterpret_cast<const uint4 *>(src + (p * CIN + g * Chunk<T>::E) * sizeof(T));
            }
            *reinterpret_cast<uint4 *>(xs + g * kRegion + pt * 16) = v;
        }
    }
}

// ---- convolution ----------------------------------------------------------------------------------
// out[p][o] = sum_t sum_i W'[t][i][o] in[p + off_t][i], with W'[t][i][o] = W[o][i][t] (forward)
// or W[i][o][26 - t] (ADJ: the adjoint of the layer whose weights W are, with CIN / COUT its
// output / input channel counts).  TI, TO, TM: element types of a multi-channel input, output
// and mask (BF16 activations, FP32 gradients on the BF16 training path).
template <int CIN, int COUT, class TI, class TO, class TM, int EPI, bool ADJ>
__global__ void __launch_bounds__(kConvThreads, 2) conv_kernel(const ConvArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    float *ws = reinterpret_cast<float *>(sm);
    unsigned char *xs = sm + (27 * CIN * COUT * 4 + 15) / 16 * 16;
    int x0, y0, z0;
    tile_origin(blockIdx.x, a.nx, a.ny, x0, y0, z0);
    for (int i = threadIdx.x; i < 27 * CIN * COUT; i += blockDim.x) {
        const int o = i % COUT, ci = (i / COUT) % CIN, t = i / (COUT * CIN);
        float v = ADJ ? a.w[(ci * COUT + o) * 27 + 26 - t] : a.w[(o * CIN + ci) * 27 + t];
        if (a.wround) v = __bfloat162float(__float2bfloat16_rn(v));
        ws[i] = v;
    }
    stage_input<CIN, TI>(xs, a.in, a.nx, a.ny, a.nz, x0, y0, z0);
    __syncthreads();

    const int lx = threadIdx.x & 31, r0 = threadIdx.x >> 5;
    float acc[2][COUT];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[k][o] = 0.0f;
    int base[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int row = r0 + 8 * k, ly = row % TY, lz = row / TY;
        base[k] = (lz * HY + ly) * HX + lx;  // halo index of tap (-1, -1, -1)
    }
#pragma unroll 1
    for (int t = 0; t < 27; ++t) {
        const int off = ((t / 9) * HY + (t / 3) % 3) * HX + t % 3;
        if constexpr (CIN == 1) {
            const float *xf = reinterpret_cast<const float *>(xs);
            const float v0 = xf[base[0] + off], v1 = xf[base[1] + off];
            const float *wt = ws + t * COUT;
            if constexpr (COUT % 4 == 0) {
#pragma unroll
                for (int o4 = 0; o4 < COUT / 4; ++o4) {
                    const float4 w4 = reinterpret_cast<const float4 *>(wt)[o4];
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        acc[0][4 * o4 + q] = fmaf(wv[q], v0, acc[0][4 * o4 + q]);
                        acc[1][4 * o4 + q] = fmaf(wv[q], v1, acc[1][4 * o4 + q]);
                    }
                }
            } else {
#pragma unroll
                for (int o = 0; o < COUT; ++o) {
                    acc[0][o] = fmaf(wt[o], v0, acc[0][o]);
                    acc[1][o] = fmaf(wt[o], v1, acc[1][o]);
                }
            }
        } else {
            constexpr int E = Chunk<TI>::E, NG = CIN / E;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                float in0[E], in1[E];
                Chunk<TI>::unpack(*reinterpret_cast<const uint4 *>(xs + g * kRegion + (base[0] + off) * 16), in0);
                Chunk<TI>::unpack(*reinterpret_cast<const uint4 *>(xs + g * kRegion + (base[1] + off) * 16), in1);
#pragma unroll
                for (int c = 0; c < E; ++c) {
                    const float *wt = ws + (t * CIN + g * E + c) * COUT;
                    if constexpr (COUT % 4 == 0) {
#pragma unroll
                        for (int o4 = 0; o4 < COUT / 4; ++o4) {
                            const float4 w4 = reinterpret_cast<const float4 *>(wt)[o4];
                            acc[0][4 * o4 + 0] = fmaf(w4.x, in0[c], acc[0][4 * o4 + 0]);
                            acc[0][4 * o4 + 1] = fmaf(w4.y, in0[c], acc[0][4 * o4 + 1]);
                            acc[0][4 * o4 + 2] = fmaf(w4.z, in0[c], acc[0][4 * o4 + 2]);
                            acc[0][4 * o4 + 3] = fmaf(w4.w, in0[c], acc[0][4 * o4 + 3]);
                            acc[1][4 * o4 + 0] = fmaf(w4.x, in1[c], acc[1][4 * o4 + 0]);
                            acc[1][4 * o4 + 1] = fmaf(w4.y, in1[c], acc[1][4 * o4 + 1]);
                            acc[1][4 * o4 + 2] = fmaf(w4.z, in1[c], acc[1][4 * o4 + 2]);
                            acc[1][4 * o4 + 3] = fmaf(w4.w, in1[c], acc[1][4 * o4 + 3]);
                        }
                    } else {
                        // one output channel: the chunk's E weights are consecutive (ci fastest)
                        float wv;
                        if constexpr (COUT == 1 && E % 4 == 0) {
                            const float4 w4 = reinterpret_cast<const float4 *>(ws + (t * CIN + g * E))[c / 4];
                            wv = (c % 4 == 0) ? w4.x : (c % 4 == 1) ? w4.y : (c % 4 == 2) ? w4.z : w4.w;
                        } else {
                            wv = wt[0];
                        }
#pragma unroll
                        for (int o = 0; o < COUT; ++o) {
                            acc[0][o] = fmaf(COUT == 1 ? wv : wt[o], in0[c], acc[0][o]);
                            acc[1][o] = fmaf(COUT == 1 ? wv : wt[o], in1[c], acc[1][o]);
                        }
                    }
                }
            }
        }
    }

    const float sc = (EPI & EPI_SCALE) ? static_cast<float>(*a.scale) : 1.0f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int row = r0 + 8 * k, ly = row % TY, lz = row / TY;
        const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
        if (gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
        const long long p = (static_cast<long long>(gz) * a.ny + gy) * a.nx + gx;
        float v[COUT];
#pragma unroll
        for (int o = 0; o < COUT; ++o) {
            v[o] = acc[k][o] * sc;
            if (EPI & EPI_RELU) v[o] = fmaxf(v[o], 0.0f);
        }
        if constexpr (COUT == 1) {
            static_cast<float *>(a.out)[p] = v[0];
        } else {
            if (EPI & EPI_MASK) {
                constexpr int EM = Chunk<TM>::E;
                const uint4 *mk = reinterpret_cast<const uint4 *>(static_cast<const TM *>(a.mask) + p * COUT);
#pragma unroll
                for (int g = 0; g < COUT / EM; ++g) {
                    float m[EM];
                    Chunk<TM>::unpack(mk[g], m);
#pragma unroll
                    for (int c = 0; c < EM; ++c)
                        if (!(m[c] > 0.0f)) v[g * EM + c] = 0.0f;
                }
            }
            constexpr int E = Chunk<TO>::E;
            uint4 *dst = reinterpret_cast<uint4 *>(static_cast<TO *>(a.out) + p * COUT);
#pragma unroll
            for (int g = 0; g < COUT / E; ++g) dst[g] = Chunk<TO>::pack(v + g * E);
        }
    }
}

// ---- forward layers 1 and 3 (register-blocked in z) ------------------------------------------------
// A CTA of 256 threads owns a 32 x 4 x 4 block; thread (x, y, h) computes the 2 points
// (x, y, z0+2h .. z0+2h+1), so for every (dx, dy) the 4 input values around them are loaded once
// and serve the 3 dz taps of both points.  Weights are FP32 in shared memory, read as float4
// broadcasts.
constexpr int kL3Threads = 256;

// Layer 1: a1[p][o] = ReLU(scale * sum_t w1[o][0][t] rho[p + off_t]),  TO = BF16 or FP32.
// 256 threads, each two z-points of the 32 x 4 x 4 block.
template <class TO>
__global__ void __launch_bounds__(kL3Threads) layer1_kernel(int nx, int ny, int nz, const float *__restrict__ rho,
                                                          TO *__restrict__ out, const float *__restrict__ w,
                                                          const double *__restrict__ scale, int wround) {
    __shared__ __align__(16) float ws[27 * 16];  // [t][o]
    __shared__ float xs[HZ][HY][HX];
    int x0, y0, z0;
    tile_origin(blockIdx.x, nx, ny, x0, y0, z0);
    for (int i = threadIdx.x; i < 27 * 16; i += blockDim.x) {
        const int o = i & 15, t = i >> 4;
        float v = w[o * 27 + t];
        if (wround) v = __bfloat162float(__float2bfloat16_rn(v));
        ws[i] = v;
    }
    stage_input<1, float>(reinterpret_cast<unsigned char *>(&xs[0][0][0]), rho, nx, ny, nz, x0, y0, z0);
    __syncthreads();
    const int lx = threadIdx.x & 31, ly = (threadIdx.x >> 5) & 3, zh = threadIdx.x >> 7;
    float acc[2][16];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int o = 0; o < 16; ++o) acc[k][o] = 0.0f;
#pragma unroll 1
    for (int dxy = 0; dxy < 9; ++dxy) {
        const int dy = dxy / 3, dx = dxy % 3;
        float col[4];
#pragma unroll
        for (int zz = 0; zz < 4; ++zz) col[zz] = xs[2 * zh + zz][ly + dy][lx + dx];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
            const float4 *w4 = reinterpret_cast<const float4 *>(ws + ((dz * 3 + dy) * 3 + dx) * 16);
#pragma unroll
            for (int o4 = 0; o4 < 4; ++o4) {
                const float4 wv = w4[o4];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float v = col[k + dz];
                    acc[k][4 * o4 + 0] = fmaf(wv.x, v, acc[k][4 * o4 + 0]);
                    acc[k][4 * o4 + 1] = fmaf(wv.y, v, acc[k][4 * o4 + 1]);
                    acc[k][4 * o4 + 2] = fmaf(wv.z, v, acc[k][4 * o4 + 2]);
                    acc[k][4 * o4 + 3] = fmaf(wv.w, v, acc[k][4 * o4 + 3]);
                }
            }
        }
    }
    const float sc = static_cast<float>(*scale);
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= nx || gy >= ny) return;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int gz = z0 + 2 * zh + k;
        if (gz >= nz) break;
        float v[16];
#pragma unroll
        for (int o = 0; o < 16; ++o) v[o] = fmaxf(acc[k][o] * sc, 0.0f);
        const long long p = (static_cast<long long>(gz) * ny + gy) * nx + gx;
        uint4 *dst = reinterpret_cast<uint4 *>(out + p * 16);
        constexpr int E = Chunk<TO>::E;
#pragma unroll
        for (int g = 0; g < 16 / E; ++g) dst[g] = Chunk<TO>::pack(v + g * E);
    }
}

// Layer 3: delta[p] = scale * sum_t sum_c w3[0][c][t] a2[p + off_t][c].  256 threads, each two
// z-points of the 32 x 4 x 4 block; the input halo is copied as raw 16-byte channel chunks
// (chunk-major, as stage_input) and widened to FP32 at use.
template <class TI>
__global__ void __launch_bounds__(kL3Threads) layer3_kernel(int nx, int ny, int nz, const TI *__restrict__ a2,
                                                          float *__restrict__ out, const float *__restrict__ w,
                                                          const double *__restrict__ scale, int wround) {
    extern __shared__ __align__(16) unsigned char sm3[];
    float *ws = reinterpret_cast<float *>(sm3);       // [t][c]
    unsigned char *xs = sm3 + 27 * 16 * 4;              // [chunk][HP] x 16 B
    int x0, y0, z0;
    tile_origin(blockIdx.x, nx, ny, x0, y0, z0);
    for (int i = threadIdx.x; i < 27 * 16; i += blockDim.x) {
        const int c = i & 15, t = i >> 4;
        float v = w[c * 27 + t];
        if (wround) v = __bfloat162float(__float2bfloat16_rn(v));
        ws[i] = v;
    }
    stage_input<16, TI>(xs, a2, nx, ny, nz, x0, y0, z0);
    __syncthreads();
    constexpr int E = Chunk<TI>::E, NG = 16 / E;
    const int lx = threadIdx.x & 31, ly = (threadIdx.x >> 5) & 3, zh = threadIdx.x >> 7;  // points z 2zh, 2zh+1
    float acc[2] = {0.0f, 0.0f};
#pragma unroll 1
    for (int dxy = 0; dxy < 9; ++dxy) {
        const int dy = dxy / 3, dx = dxy % 3;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
            float col[4][E];
#pragma unroll
            for (int zz = 0; zz < 4; ++zz)
                Chunk<TI>::unpack(*reinterpret_cast<const uint4 *>(
                                      xs + g * kRegion + (((2 * zh + zz) * HY + ly + dy) * HX + lx + dx) * 16),
                                  col[zz]);
#pragma unroll
            for (int dz = 0; dz < 3; ++dz) {
                const float *wt = ws + ((dz * 3 + dy) * 3 + dx) * 16 + g * E;
#pragma unroll
                for (int q = 0; q < E / 4; ++q) {
                    const float4 wv = reinterpret_cast<const float4 *>(wt)[q];
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const float *v = col[k + dz] + 4 * q;
                        acc[k] = fmaf(wv.x, v[0], fmaf(wv.y, v[1], fmaf(wv.z, v[2], fmaf(wv.w, v[3], acc[k]))));
                    }
                }
            }
        }
    }
    const float sc = static_cast<float>(*scale);
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= nx || gy >= ny) return;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int gz = z0 + 2 * zh + k;
        if (gz >= nz) break;
        out[(static_cast<long long>(gz) * ny + gy) * nx + gx] = acc[k] * sc;
    }
}

// ---- weight gradient --------------------------------------------------------------------------------
// part[block][entry] = sum over the block's points p of gout[p][co] in[p + off_t][ci], entry
// (co * CIN + ci) * 27 + t (the master layout).  Thread j < 432 owns tap t = j / 16 and
// q = j % 16: with 16 in and 16 out channels q = ci and the thread sums all 16 co; with one input
// channel q = co; with one output channel q = ci.
struct WgradArgs {
    int nx, ny, nz;
    const void *in;    // CIN == 1: float [n]; else T [n][16]
    const void *gout;  // COUT == 1: float [n]; else TG [n][16]
    float *part;       // [gridDim.x][27 * CIN * COUT]
};

template <int CIN, int COUT, class T>
constexpr size_t wgrad_smem_bytes() {
    return (CIN == 1 ? static_cast<size_t>(HP) * 4 : static_cast<size_t>(CIN / Chunk<T>::E) * kRegion) +
           static_cast<size_t>(TP) * COUT * 4;
}

template <int CIN, int COUT, class T, class TG>
__global__ void __launch_bounds__(kWgThreads, 1) wgrad_kernel(const WgradArgs a) {
    extern __shared__ __align__(16) unsigned char sm[];
    constexpr int NO = (CIN == 16 && COUT == 16) ? 16 : 1;
    unsigned char *xs = sm;
    float *gs = reinterpret_cast<float *>(sm + (CIN == 1 ? HP * 4 : (CIN / Chunk<T>::E) * kRegion));
    const int j = threadIdx.x;
    const bool own = j < 432;
    const int t = j / 16, q = j % 16;
    const int off = own ? ((t / 9) * HY + (t / 3) % 3) * HX + t % 3 : 0;
    float acc[NO];
#pragma unroll
    for (int o = 0; o < NO; ++o) acc[o] = 0.0f;
    const int ntiles = ((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY) * ((a.nz + TZ - 1) / TZ);
    for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
        int x0, y0, z0;
        tile_origin(b, a.nx, a.ny, x0, y0, z0);
        stage_input<CIN, T>(xs, a.in, a.nx, a.ny, a.nz, x0, y0, z0);
        for (int i = threadIdx.x; i < TP * COUT; i += blockDim.x) {
            const int o = i % COUT, p = i / COUT;
            const int lx = p & 31, row = p >> 5, ly = row % TY, lz = row / TY;
            const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
            float v = 0.0f;
            if (gx < a.nx && gy < a.ny && gz < a.nz) {
                const long long gp = (static_cast<long long>(gz) * a.ny + gy) * a.nx + gx;
                if constexpr (COUT == 1) v = static_cast<const float *>(a.gout)[gp];
                else v = Chunk<TG>::elem(static_cast<const unsigned char *>(a.gout) + gp * COUT * sizeof(TG), o);
            }
            gs[i] = v;
        }
        __syncthreads();
        if (own) {
#pragma unroll 2
            for (int p = 0; p < TP; ++p) {
                const int lx = p & 31, row = p >> 5, ly = row % TY, lz = row / TY;
                const int hp = (lz * HY + ly) * HX + lx + off;
                float xin;
                if constexpr (CIN == 1) {
                    xin = reinterpret_cast<const float *>(xs)[hp];
                } else {
                    constexpr int E = Chunk<T>::E;
                    xin = Chunk<T>::elem(xs + (q / E) * kRegion + hp * 16, q % E);
                }
                if constexpr (NO == 16) {
                    const float4 *g4 = reinterpret_cast<const float4 *>(gs + p * 16);
#pragma unroll
                    for (int o4 = 0; o4 < 4; ++o4) {
                        const float4 g = g4[o4];
                        acc[4 * o4 + 0] = fmaf(g.x, xin, acc[4 * o4 + 0]);
                        acc[4 * o4 + 1] = fmaf(g.y, xin, acc[4 * o4 + 1]);
                        acc[4 * o4 + 2] = fmaf(g.z, xin, acc[4 * o4 + 2]);
                        acc[4 * o4 + 3] = fmaf(g.w, xin, acc[4 * o4 + 3]);
                    }
                } else if constexpr (CIN == 1) {
                    acc[0] = fmaf(gs[p * COUT + q], xin, acc[0]);
                } else {
                    acc[0] = fmaf(gs[p], xin, acc[0]);
                }
            }
        }
        __syncthreads();
    }
    if (!own) return;
    float *dst = a.part + static_cast<size_t>(blockIdx.x) * (27 * CIN * COUT);
    if constexpr (NO == 16) {
#pragma unroll
        for (int o = 0; o < 16; ++o) dst[(o * CIN + q) * 27 + t] = acc[o];
    } else if constexpr (CIN == 1) {
        dst[q * 27 + t] = acc[0];
    } else {
        dst[q * 27 + t] = acc[0];
    }
}

__global__ void wreduce_kernel(const float *part, int nblocks, int nentries, const double *scale, float *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nentries) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[static_cast<size_t>(b) * nentries + e];
    if (scale) s *= *scale;
    out[e] = static_cast<float>(s);
}

// ---- reductions and stencil kernels -------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kRedThreads / 32; ++k) s += sh[k];
    __syncthreads();
    return s;
}

// A v at point i = (x, y, z) of an nx x ny x nz grid (7-point, Dirichlet), v widened to double.
template <class V>
__device__ __forceinline__ double stencil_at(const V *v, int i, int x, int y, int z, int nx, int ny, int nz) {
    const int np = nx * ny;
    double nb = 0.0;
    if (x > 0) nb += ldv<double>(v + i - 1);
    if (x < nx - 1) nb += ldv<double>(v + i + 1);
    if (y > 0) nb += ldv<double>(v + i - nx);
    if (y < ny - 1) nb += ldv<double>(v + i + nx);
    if (z > 0) nb += ldv<double>(v + i - np);
    if (z < nz - 1) nb += ldv<double>(v + i + np);
    return 6.0 * ldv<double>(v + i) - nb;
}

__device__ __forceinline__ void decode(int i, int nx, int ny, int &x, int &y, int &z) {
    const int np = nx * ny;
    z = i / np;
    const int r = i - z * np;
    y = r / nx;
    x = r - y * nx;
}

// FP32 value of a storage element (FP64 narrowed on the integer pipe).
template <class S> __device__ __forceinline__ float ldf(const S *p);
template <> __device__ __forceinline__ float ldf<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <> __device__ __forceinline__ float ldf<double>(const double *p) { return narrow_f64(*p); }

// A v at point i in FP32 (7-point, Dirichlet).
template <class V>
__device__ __forceinline__ float stencil_f32(const V *v, int i, int x, int y, int z, int nx, int ny, int nz) {
    const int np = nx * ny;
    float nb = 0.0f;
    if (x > 0) nb += ldf(v + i - 1);
    if (x < nx - 1) nb += ldf(v + i + 1);
    if (y > 0) nb += ldf(v + i - nx);
    if (y < ny - 1) nb += ldf(v + i + nx);
    if (z > 0) nb += ldf(v + i - np);
    if (z < nz - 1) nb += ldf(v + i + np);
    return fmaf(6.0f, ldf(v + i), -nb);
}

// rho = r - A s in FP32 (the network's input and the judge's reference need no more: rho is
// stored as FP32 and fed to BF16 activations), part = sum rho^2 (FP32 per thread, FP64 across).
template <class S>
__global__ void __launch_bounds__(kRedThreads) rho_kernel(int nx, int ny, int nz, const double *r, const S *s,
                                                          float *rho, double *part) {
    const int n = nx * ny * nz;
    float acc = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int x, y, z;
        decode(i, nx, ny, x, y, z);
        const float v = narrow_f64(r[i]) - stencil_f32(s, i, x, y, z, nx, ny, nz);
        rho[i] = v;
        acc = fmaf(v, v, acc);
    }
    const double tot = block_sum(static_cast<double>(acc));
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kRedThreads) sumsq_kernel(int n, const float *v, double *part) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double d = v[i];
        acc = fma(d, d, acc);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void fin_rho_kernel(const double *part, int np, long long n, NetScal *sc) {
    double s = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) s += part[k];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        sc->rr = s;
        sc->rms = sqrt(s / static_cast<double>(n));
        sc->inv_rms = sc->rms > 0.0 ? 1.0 / sc->rms : 0.0;
    }
}

// the judge: part = sum (rho - A delta)^2, in FP32 per thread
__global__ void __launch_bounds__(kRedThreads) judge_kernel(int nx, int ny, int nz, const float *rho,
                                                            const float *delta, double *part) {
    const int n = nx * ny * nz;
    float acc = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int x, y, z;
        decode(i, nx, ny, x, y, z);
        const float v = rho[i] - stencil_f32(delta, i, x, y, z, nx, ny, nz);
        acc = fmaf(v, v, acc);
    }
    const double tot = block_sum(static_cast<double>(acc));
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void fin_judge_kernel(const double *part, int np, NetScal *sc) {
    double s = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) s += part[k];
    s = block_sum(s);
    if (threadIdx.x == 0) {
        sc->after = s;
        sc->accepted = (s < sc->rr) ? 1 : 0;
        sc->calls += 1;
        sc->accepts += sc->accepted;
    }
}

template <class S>
__global__ void apply_kernel(int n, const float *delta, S *s, const NetScal *sc) {
    if (!sc->accepted) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if constexpr (std::is_same<S, double>::value) s[i] += widen_f32(delta[i]);
        else stv<S, float>(s + i, ldv<float>(s + i) + delta[i]);
    }
}

// training loss: d = e - delta; ad = A d; part[2b] = sum d A d, part[2b+1] = sum e A e
__global__ void __launch_bounds__(kRedThreads) loss_kernel(int nx, int ny, int nz, const float *e,
                                                           const float *delta, float *ad, double *part) {
    const int n = nx * ny * nz, np = nx * ny;
    double a0 = 0.0, a1 = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int x, y, z;
        decode(i, nx, ny, x, y, z);
        auto d_at = [&](int k) { return static_cast<double>(e[k]) - static_cast<double>(delta[k]); };
        double nbd = 0.0, nbe = 0.0;
        if (x > 0) nbd += d_at(i - 1), nbe += e[i - 1];
        if (x < nx - 1) nbd += d_at(i + 1), nbe += e[i + 1];
        if (y > 0) nbd += d_at(i - nx), nbe += e[i - nx];
        if (y < ny - 1) nbd += d_at(i + nx), nbe += e[i + nx];
        if (z > 0) nbd += d_at(i - np), nbe += e[i - np];
        if (z < nz - 1) nbd += d_at(i + np), nbe += e[i + np];
        const double di = d_at(i), ei = e[i];
        const double Ad = 6.0 * di - nbd, Ae = 6.0 * ei - nbe;
        ad[i] = static_cast<float>(Ad);
        a0 = fma(di, Ad, a0);
        a1 = fma(ei, Ae, a1);
    }
    a0 = block_sum(a0);
    a1 = block_sum(a1);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a0;
        part[2 * blockIdx.x + 1] = a1;
    }
}

__global__ void fin_loss_kernel(const double *part, int np, NetScal *sc) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) {
        s0 += part[2 * k];
        s1 += part[2 * k + 1];
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x == 0) {
        sc->num = s0;
        sc->den = s1;
        sc->loss = s1 > 0.0 ? s0 / s1 : 0.0;
        sc->gscale = s1 > 0.0 ? -2.0 * sc->rms / s1 : 0.0;
        sc->loss_sum += sc->loss;
    }
}

__global__ void adam_kernel(float *w, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

template <class S>
__global__ void capture_kernel(int nx, int ny, int nz, const double *r, const S *s, const double *x,
                               const double *xstar, float *rho, float *e) {
    const int n = nx * ny * nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int xx, y, z;
        decode(i, nx, ny, xx, y, z);
        const double si = ldv<double>(s + i);
        rho[i] = narrow_f64(r[i] - stencil_at(s, i, xx, y, z, nx, ny, nz));
        e[i] = narrow_f64(xstar[i] - x[i] - si);
    }
}

__global__ void to_f32_kernel(long long n, const double *src, float *dst) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        dst[i] = narrow_f64(src[i]);
}
__global__ void to_f64_kernel(long long n, const float *src, double *dst) {
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        dst[i] = widen_f32(src[i]);
}

// ---- launch helpers ---------------------------------------------------------------------------------
int num_tiles(int nx, int ny, int nz) {
    return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY) * ((nz + TZ - 1) / TZ);
}

template <int CIN, int COUT, class TI, class TO, class TM, int EPI, bool ADJ>
cudaError_t conv(const ConvArgs &a, cudaStream_t st) {
    constexpr size_t smem = conv_smem_bytes<CIN, COUT, TI>();
    cudaError_t e =
        raise_smem_attr(reinterpret_cast<const void *>(&conv_kernel<CIN, COUT, TI, TO, TM, EPI, ADJ>), smem);
    if (e != cudaSuccess) return e;
    conv_kernel<CIN, COUT, TI, TO, TM, EPI, ADJ><<<num_tiles(a.nx, a.ny, a.nz), kConvThreads, smem, st>>>(a);
    return cudaGetLastError();
}

template <int CIN, int COUT, class T, class TG>
cudaError_t wgrad(const WgradArgs &a, int blocks, cudaStream_t st) {
    constexpr size_t smem = wgrad_smem_bytes<CIN, COUT, T>();
    cudaError_t e = raise_smem_attr(reinterpret_cast<const void *>(&wgrad_kernel<CIN, COUT, T, TG>), smem);
    if (e != cudaSuccess) return e;
    wgrad_kernel<CIN, COUT, T, TG><<<blocks, kWgThreads, smem, st>>>(a);
    return cudaGetLastError();
}

int red_blocks(long long n) {
    return static_cast<int>(std::max<long long>(1, std::min<long long>(kRedBlocks, (n + kRedThreads - 1) / kRedThreads)));
}

template <class T>
cudaError_t forward_t(NetWork &nw, int nx, int ny, int nz, cudaStream_t st) {
    const int wr = std::is_same<T, __nv_bfloat16>::value ? 1 : 0;
    cudaError_t e;
    const int tiles = num_tiles(nx, ny, nz);
    layer1_kernel<T><<<tiles, kL3Threads, 0, st>>>(nx, ny, nz, nw.rho, static_cast<T *>(nw.a1), nw.w + kNetW1,
                                                   &nw.sc->inv_rms, wr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ConvArgs a;
    if (std::is_same<T, __nv_bfloat16>::value && net_tensor_cores()) {
        if ((e = conv16_tc_prep(nw.w + kNetW2, nw.w2b, st)) != cudaSuccess) return e;
        if ((e = conv16_tc(nx, ny, nz, nw.a1, nw.a2, nw.w2b, st)) != cudaSuccess) return e;
        nw.launches += 1;
    } else {
        a = ConvArgs{nx, ny, nz, nw.a1, nw.a2, nw.w + kNetW2, nullptr, nullptr, wr};
        if ((e = conv<16, 16, T, T, T, EPI_RELU, false>(a, st)) != cudaSuccess) return e;
    }
    {
        constexpr size_t smem3 = 27 * 16 * 4 + static_cast<size_t>(16 / Chunk<T>::E) * kRegion;
        if ((e = raise_smem_attr(reinterpret_cast<const void *>(&layer3_kernel<T>), smem3)) != cudaSuccess) return e;
        layer3_kernel<T><<<tiles, kL3Threads, smem3, st>>>(nx, ny, nz, static_cast<const T *>(nw.a2), nw.delta,
                                                           nw.w + kNetW3, &nw.sc->rms, wr);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    nw.launches += 3;
    return cudaSuccess;
}

template <class T>
cudaError_t backward_t(NetWork &nw, int nx, int ny, int nz, cudaStream_t st) {
    const int wr = std::is_same<T, __nv_bfloat16>::value ? 1 : 0;
    const int blocks = std::min(nw.wpart_blocks, num_tiles(nx, ny, nz));
    cudaError_t e;
    // layer 3: gradient of the weights from a2 and gy = gscale * A d; g2 = mask(a2) adj3(gy)
    WgradArgs wa{nx, ny, nz, nw.a2, nw.ad, nw.wpart};
    if ((e = wgrad<16, 1, T, float>(wa, blocks, st)) != cudaSuccess) return e;
    wreduce_kernel<<<(16 * 27 + 255) / 256, 256, 0, st>>>(nw.wpart, blocks, 16 * 27, &nw.sc->gscale,
                                                          nw.grad + kNetW3);
    ConvArgs a{nx, ny, nz, nw.ad, nw.g2, nw.w + kNetW3, nw.a2, &nw.sc->gscale, wr};
    if ((e = conv<1, 16, float, float, T, EPI_MASK | EPI_SCALE, true>(a, st)) != cudaSuccess) return e;
    // layer 2
    wa = WgradArgs{nx, ny, nz, nw.a1, nw.g2, nw.wpart};
    if ((e = wgrad<16, 16, T, float>(wa, blocks, st)) != cudaSuccess) return e;
    wreduce_kernel<<<(16 * 16 * 27 + 255) / 256, 256, 0, st>>>(nw.wpart, blocks, 16 * 16 * 27, nullptr,
                                                               nw.grad + kNetW2);
    a = ConvArgs{nx, ny, nz, nw.g2, nw.g1, nw.w + kNetW2, nw.a1, nullptr, wr};
    if ((e = conv<16, 16, float, float, T, EPI_MASK, true>(a, st)) != cudaSuccess) return e;
    // layer 1: its input is rho / rms
    wa = WgradArgs{nx, ny, nz, nw.rho, nw.g1, nw.wpart};
    if ((e = wgrad<1, 16, T, float>(wa, blocks, st)) != cudaSuccess) return e;
    wreduce_kernel<<<(16 * 27 + 255) / 256, 256, 0, st>>>(nw.wpart, blocks, 16 * 27, &nw.sc->inv_rms,
                                                          nw.grad + kNetW1);
    nw.launches += 8;
    return cudaGetLastError();
}

}  // namespace

bool &net_tensor_cores() {
    static bool on = true;
    return on;
}

cudaError_t net_alloc(NetWork &nw, long long n, int act, bool training) {
    if (nw.n >= n && nw.act == act && (nw.training || !training)) return cudaSuccess;
    const bool keep_w = nw.w != nullptr;
    float *w_old = nw.w, *m_old = nw.m, *v_old = nw.v;
    nw.w = nw.m = nw.v = nullptr;
    net_free(nw);
    nw.n = n;
    nw.act = act;
    nw.training = training;
    const size_t ab = static_cast<size_t>(n) * kNetC * (act == 0 ? 2 : 4);
    cudaError_t e = cudaMalloc(&nw.a1, ab);
    if (e == cudaSuccess) e = cudaMalloc(&nw.a2, ab);
    if (e == cudaSuccess) e = cudaMalloc(&nw.rho, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&nw.delta, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&nw.part, 2 * kRedBlocks * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&nw.sc, sizeof(NetScal));
    if (e == cudaSuccess) e = cudaMalloc(&nw.w2b, kConv16TcWeightBytes);
    if (e == cudaSuccess) e = cudaMemset(nw.sc, 0, sizeof(NetScal));
    if (keep_w) {
        nw.w = w_old;
        nw.m = m_old;
        nw.v = v_old;
    } else if (e == cudaSuccess) {
        e = cudaMalloc(&nw.w, kNetWeights * sizeof(float));
    }
    if (training && e == cudaSuccess) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        nw.wpart_blocks = std::max(1, nsm);
        // the masked gradients stay FP32 on both paths
        const size_t gb = static_cast<size_t>(n) * kNetC * 4;
        e = cudaMalloc(&nw.g1, gb);
        if (e == cudaSuccess) e = cudaMalloc(&nw.g2, gb);
        if (e == cudaSuccess) e = cudaMalloc(&nw.e, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&nw.ad, n * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&nw.grad, kNetWeights * sizeof(float));
        if (e == cudaSuccess && !nw.m) {
            e = cudaMalloc(&nw.m, kNetWeights * sizeof(float));
            if (e == cudaSuccess) e = cudaMemset(nw.m, 0, kNetWeights * sizeof(float));
        }
        if (e == cudaSuccess && !nw.v) {
            e = cudaMalloc(&nw.v, kNetWeights * sizeof(float));
            if (e == cudaSuccess) e = cudaMemset(nw.v, 0, kNetWeights * sizeof(float));
        }
        if (e == cudaSuccess)
            e = cudaMalloc(&nw.wpart, static_cast<size_t>(nw.wpart_blocks) * 16 * 16 * 27 * sizeof(float));
    }
    if (e != cudaSuccess) net_free(nw);
    return e;
}

void net_free(NetWork &nw) {
    void *ps[] = {nw.a1, nw.a2, nw.g1, nw.g2, nw.rho, nw.delta, nw.e, nw.ad, nw.part, nw.sc, nw.w, nw.grad,
                  nw.m, nw.v, nw.wpart, nw.w2b};
    for (void *p : ps) cudaFree(p);
    const long long launches = nw.launches;
    nw = NetWork();
    nw.launches = launches;
}

cudaError_t net_forward(NetWork &nw, int nx, int ny, int nz, cudaStream_t st) {
    const long long n = static_cast<long long>(nx) * ny * nz;
    const int rb = red_blocks(n);
    sumsq_kernel<<<rb, kRedThreads, 0, st>>>(static_cast<int>(n), nw.rho, nw.part);
    fin_rho_kernel<<<1, kRedThreads, 0, st>>>(nw.part, rb, n, nw.sc);
    nw.launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return nw.act == 0 ? forward_t<__nv_bfloat16>(nw, nx, ny, nz, st) : forward_t<float>(nw, nx, ny, nz, st);
}

cudaError_t net_loss_grad(NetWork &nw, int nx, int ny, int nz, cudaStream_t st) {
    cudaError_t e = net_forward(nw, nx, ny, nz, st);
    if (e != cudaSuccess) return e;
    const long long n = static_cast<long long>(nx) * ny * nz;
    const int rb = red_blocks(n);
    loss_kernel<<<rb, kRedThreads, 0, st>>>(nx, ny, nz, nw.e, nw.delta, nw.ad, nw.part);
    fin_loss_kernel<<<1, kRedThreads, 0, st>>>(nw.part, rb, nw.sc);
    nw.launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return nw.act == 0 ? backward_t<__nv_bfloat16>(nw, nx, ny, nz, st) : backward_t<float>(nw, nx, ny, nz, st);
}

cudaError_t net_adam(NetWork &nw, int step, float lr, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = static_cast<float>(1.0 - std::pow(0.9, step));
    const float c2 = static_cast<float>(1.0 - std::pow(0.999, step));
    adam_kernel<<<(kNetWeights + 255) / 256, 256, 0, st>>>(nw.w, nw.grad, nw.m, nw.v, kNetWeights, lr, b1, b2, eps,
                                                           c1, c2);
    nw.launches += 1;
    return cudaGetLastError();
}

cudaError_t net_learned_correct(NetWork &nw, Prec storage, int nx, int ny, int nz, const double *r, void *s,
                                cudaStream_t st) {
    const long long n = static_cast<long long>(nx) * ny * nz;
    const int rb = red_blocks(n);
    switch (storage) {
    case Prec::F64: rho_kernel<double><<<rb, kRedThreads, 0, st>>>(nx, ny, nz, r, static_cast<const double *>(s), nw.rho, nw.part); break;
    case Prec::F32: rho_kernel<float><<<rb, kRedThreads, 0, st>>>(nx, ny, nz, r, static_cast<const float *>(s), nw.rho, nw.part); break;
    case Prec::BF16: rho_kernel<__nv_bfloat16><<<rb, kRedThreads, 0, st>>>(nx, ny, nz, r, static_cast<const __nv_bfloat16 *>(s), nw.rho, nw.part); break;
    }
    fin_rho_kernel<<<1, kRedThreads, 0, st>>>(nw.part, rb, n, nw.sc);
    nw.launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = nw.act == 0 ? forward_t<__nv_bfloat16>(nw, nx, ny, nz, st) : forward_t<float>(nw, nx, ny, nz, st);
    if (e != cudaSuccess) return e;
    judge_kernel<<<rb, kRedThreads, 0, st>>>(nx, ny, nz, nw.rho, nw.delta, nw.part);
    fin_judge_kernel<<<1, kRedThreads, 0, st>>>(nw.part, rb, nw.sc);
    const int ab = red_blocks(n);
    switch (storage) {
    case Prec::F64: apply_kernel<double><<<ab, kRedThreads, 0, st>>>(static_cast<int>(n), nw.delta, static_cast<double *>(s), nw.sc); break;
    case Prec::F32: apply_kernel<float><<<ab, kRedThreads, 0, st>>>(static_cast<int>(n), nw.delta, static_cast<float *>(s), nw.sc); break;
    case Prec::BF16: apply_kernel<__nv_bfloat16><<<ab, kRedThreads, 0, st>>>(static_cast<int>(n), nw.delta, static_cast<__nv_bfloat16 *>(s), nw.sc); break;
    }
    nw.launches += 3;
    return cudaGetLastError();
}

cudaError_t net_capture(Prec storage, int nx, int ny, int nz, const double *r, const void *s, const double *x,
                        const double *xstar, float *rho_out, float *e_out, cudaStream_t st) {
    const long long n = static_cast<long long>(nx) * ny * nz;
    const int blocks = red_blocks(n);
    switch (storage) {
    case Prec::F64: capture_kernel<double><<<blocks, kRedThreads, 0, st>>>(nx, ny, nz, r, static_cast<const double *>(s), x, xstar, rho_out, e_out); break;
    case Prec::F32: capture_kernel<float><<<blocks, kRedThreads, 0, st>>>(nx, ny, nz, r, static_cast<const float *>(s), x, xstar, rho_out, e_out); break;
    case Prec::BF16: capture_kernel<__nv_bfloat16><<<blocks, kRedThreads, 0, st>>>(nx, ny, nz, r, static_cast<const __nv_bfloat16 *>(s), x, xstar, rho_out, e_out); break;
    }
    return cudaGetLastError();
}

cudaError_t net_to_f32(long long n, const double *src, float *dst, cudaStream_t st) {
    to_f32_kernel<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}
cudaError_t net_to_f64(long long n, const float *src, double *dst, cudaStream_t st) {
    to_f64_kernel<<<red_blocks(n), kRedThreads, 0, st>>>(n, src, dst);
    return cudaGetLastError();
}

}  // namespace smg
