// conv_tc.cu -- the 16 -> 16 channel 3x3x3 convolution of the learned post-correction on the
// 5th-generation tensor cores (tcgen05): out = ReLU(conv(a1)) with BF16 activations and weights
// and FP32 accumulation in tensor memory.
//
// Implicit GEMM by shifted windows.  A CTA owns a 32 x 6 x 6 block of output points and stages
// the 34 x 8 x 8 halo block of the input in shared memory as two regions (channels 0-7 and
// 8-15), each a run of 16-byte rows in the halo's linear (z, y, x) order -- exactly the box of a
// 4D tiled TMA load (channels, x, y, z) with box (8, 34, 8, 8), whose out-of-range elements
// (the zero padding of the convolution) the copy engine fills with zeros.  For 128 consecutive
// linear positions q0 .. q0+127 and tap t with linear offset d_t, the A operand (128 points x 16
// input channels, K-major, no swizzle) is the same layout starting at row q0 + d_t: rows 16 B
// apart, 8-row core matrices 128 B apart (SBO), the second channel chunk one region further
// (LBO).  So every tap is one tcgen05.mma (M = 128, N = 16, K = 16) whose A descriptor differs
// only in its start address, accumulating into the same 16 TMEM columns.  Rows whose position is
// a halo point give unused results.  B (16 output x 16 input channels per tap, K-major) holds
// the 27 taps' weights.  One elected thread issues all MMAs of the CTA (13 row blocks x 27 taps),
// commits them to an mbarrier, and four warps per row block read the accumulators back
// (tcgen05.ld 32x32b: warp w reads TMEM lanes 32(w%4) ..) for the ReLU + BF16 epilogue.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "net.h"

namespace smg {
namespace {

constexpr int CTX = 32, CTY = 6, CTZ = 6;
constexpr int CHX = CTX + 2, CHY = CTY + 2, CHZ = CTZ + 2, CHP = CHX * CHY * CHZ;  // 2176 halo points
constexpr int QLO = (CHY + 1) * CHX + 1;                 // first interior position
constexpr int QHI = (CTZ * CHY + CTY) * CHX + CTX;       // last interior position
constexpr int DMAX = CHY * CHX + CHX + 1;                // largest |tap offset|
constexpr int NMT = (QHI - QLO + 1 + 127) / 128;         // 128-row blocks per CTA (13)
constexpr int ROWS = CHP + 128;                          // rows per channel region, with padding
constexpr int RS = ROWS * 16;                            // region stride in bytes (LBO), 128-B multiple
constexpr int A_BYTES = 2 * RS;
constexpr int B_BYTES = 27 * 512;                        // per tap: [chunk][16 out][8 in] BF16
constexpr int TC_COLS = 256;                             // TMEM columns allocated per CTA
constexpr int TC_THREADS = 256;
constexpr size_t TC_SMEM = A_BYTES + B_BYTES + 32;
constexpr uint32_t TMA_BYTES = 2u * CHP * 16u;           // two boxes of 8 channels x 34 x 8 x 8
constexpr long long kWaitLimit = 1ll << 26;              // mbarrier polls before giving up

// Every A row an MMA can read lies inside the staged regions; every accumulator fits.
static_assert(QLO - DMAX >= 0, "tap window below the staged rows");
static_assert(QLO + (NMT - 1) * 128 + 127 + DMAX < ROWS, "tap window beyond the staged rows");
static_assert(NMT * 16 <= TC_COLS, "accumulators exceed the allocated TMEM columns");
static_assert(RS % 16 == 0 && RS / 16 < (1 << 14), "LBO must be a 14-bit multiple of 16 B");
static_assert(2 * TC_SMEM <= 227 * 1024, "two CTAs per SM must fit");
static_assert(RS % 128 == 0 && A_BYTES % 128 == 0, "TMA destinations must be 128-byte aligned");

// tcgen05 instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading-dimension byte offset
// >> 4 (bits 16-29), stride-dimension byte offset >> 4 (bits 32-45), version 1 (bits 46-47), no
// swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

struct TcArgs {
    int nx, ny, nz;
    __nv_bfloat16 *out;        // [n][16]
    const uint4 *wb;           // the B operand of all taps, prepared by conv16_tc_prep (B_BYTES)
};

// B[t][chunk][n][8] = w[n][chunk*8 + e][t] as BF16 (the layer's FP32 weights rounded once).
__global__ void conv16_tc_prep_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * 256; i += gridDim.x * blockDim.x) {
        const int e = i & 7, n = (i >> 3) & 15, c = (i >> 7) & 1, t = i >> 8;
        wb[i] = __float2bfloat16_rn(w[(n * 16 + c * 8 + e) * 27 + t]);
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        __nanosleep(32);
    }
    return false;
}

// Set to 1 by a CTA whose wait for its accumulators gave up (read and cleared by conv16_tc_status).
__device__ int g_conv_tc_err = 0;

__global__ void __launch_bounds__(TC_THREADS, 2)
    conv16_tc_kernel(const __grid_constant__ CUtensorMap tmap, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *As = sm;
    unsigned char *Bs = sm + A_BYTES;
    uint64_t *mbar_ld = reinterpret_cast<uint64_t *>(Bs + B_BYTES);
    uint64_t *mbar_mma = mbar_ld + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar_ld + 2);
    int *s_fail = reinterpret_cast<int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    const int ntx = (a.nx + CTX - 1) / CTX, nty = (a.ny + CTY - 1) / CTY;
    int b = blockIdx.x;
    const int x0 = (b % ntx) * CTX;
    b /= ntx;
    const int y0 = (b % nty) * CTY;
    const int z0 = (b / nty) * CTZ;

    // a TMA destination must be 128-byte aligned in the shared window
    const bool aligned = (smem_u32(As) & 127u) == 0;
    if (threadIdx.x == 0) {
        *s_fail = aligned ? 0 : 1;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && aligned) {
        // input halo block: two boxes (channels 0-7, 8-15) of 34 x 8 x 8 points, zeros outside the grid
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar_ld)),
                     "r"(TMA_BYTES)
                     : "memory");
#pragma unroll
        for (int c = 0; c < 2; ++c)
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                "%4, %5}], [%6];" ::"r"(smem_u32(As + c * RS)),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(c * 8), "r"(x0 - 1), "r"(y0 - 1), "r"(z0 - 1),
                "r"(smem_u32(mbar_ld))
                : "memory");
    }
    // weights: the prepared B operand, 16 bytes per thread and step
    for (int i = threadIdx.x; i < B_BYTES / 16; i += TC_THREADS) reinterpret_cast<uint4 *>(Bs)[i] = a.wb[i];
    for (int i = threadIdx.x; i < 2 * 128; i += TC_THREADS)  // padding rows (read only by unused rows)
        *reinterpret_cast<uint4 *>(As + (i >> 7) * RS + (CHP + (i & 127)) * 16) = make_uint4(0u, 0u, 0u, 0u);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // make the generic-proxy shared-memory writes visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (threadIdx.x == 0 && aligned && !mbar_wait(smem_u32(mbar_ld), 0, kWaitLimit)) *s_fail = 1;
    if (threadIdx.x == 0 && *s_fail) {
        // nothing to compute: release the epilogue warps
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar_mma)) : "memory");
    } else if (threadIdx.x == 0) {
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
        for (int j = 0; j < NMT; ++j) {
            const int q0 = QLO + 128 * j;
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int d = ((t / 9) - 1) * CHY * CHX + (((t / 3) % 3) - 1) * CHX + (t % 3) - 1;
                const uint64_t ad = smem_desc(a0 + static_cast<uint32_t>(q0 + d) * 16u, RS, 128);
                const uint64_t bd = smem_desc(b0 + static_cast<uint32_t>(t) * 512u, 256, 128);
                const uint32_t acc = t > 0 ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + j * 16),
                    "l"(ad), "l"(bd), "r"(IDESC), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(mbar_mma))
                     : "memory");
    }

    // wait for the accumulators (bounded)
    bool done = mbar_wait(smem_u32(mbar_mma), 0, kWaitLimit);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (done && *s_fail) done = false;
    if (!done) {
        if (lane == 0) atomicExch(&g_conv_tc_err, 1);
    } else {
        const int quarter = warp & 3;
        for (int j = warp >> 2; j < NMT; j += 2) {
            uint32_t r[16];
            const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * quarter) << 16) + static_cast<uint32_t>(j * 16);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int q = QLO + 128 * j + 32 * quarter + lane;
            const int hx = q % CHX, hy = (q / CHX) % CHY, hz = q / (CHX * CHY);
            if (hx < 1 || hx > CTX || hy < 1 || hy > CTY || hz < 1 || hz > CTZ) continue;
            const int gx = x0 + hx - 1, gy = y0 + hy - 1, gz = z0 + hz - 1;
            if (gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
            unsigned w[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float lo = fmaxf(__uint_as_float(r[2 * k]), 0.0f);
                const float hi = fmaxf(__uint_as_float(r[2 * k + 1]), 0.0f);
                __nv_bfloat162 bb = __floats2bfloat162_rn(lo, hi);
                w[k] = *reinterpret_cast<unsigned *>(&bb);
            }
            const long long p = (static_cast<long long>(gz) * a.ny + gy) * a.nx + gx;
            uint4 *dst = reinterpret_cast<uint4 *>(a.out + p * 16);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
    }
    if (!done && threadIdx.x == 0) {
        // copies or MMAs may still be in flight: wait again (bounded) before the memory goes away
        if (aligned) mbar_wait(smem_u32(mbar_ld), 0, kWaitLimit);
        mbar_wait(smem_u32(mbar_mma), 0, kWaitLimit);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
}

}  // namespace

namespace {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace

cudaError_t conv16_tc_prep(const float *w, void *wb, cudaStream_t st) {
    conv16_tc_prep_kernel<<<(27 * 256 + 255) / 256, 256, 0, st>>>(w, static_cast<__nv_bfloat16 *>(wb));
    return cudaGetLastError();
}

cudaError_t conv16_tc(int nx, int ny, int nz, const void *in, void *out, const void *wb, cudaStream_t st) {
    cudaError_t e = raise_smem_attr(reinterpret_cast<const void *>(&conv16_tc_kernel), TC_SMEM);
    if (e != cudaSuccess) return e;
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return cudaErrorNotSupported;
    // the activations as a 4D tensor (channels, x, y, z) of BF16, channels innermost
    CUtensorMap map;
    const cuuint64_t dims[4] = {16, static_cast<cuuint64_t>(nx), static_cast<cuuint64_t>(ny),
                                static_cast<cuuint64_t>(nz)};
    const cuuint64_t strides[3] = {32, 32ull * nx, 32ull * nx * ny};  // bytes, dimensions 1..3
    const cuuint32_t box[4] = {8, CHX, CHY, CHZ};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(in), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int tiles = ((nx + CTX - 1) / CTX) * ((ny + CTY - 1) / CTY) * ((nz + CTZ - 1) / CTZ);
    TcArgs a{nx, ny, nz, static_cast<__nv_bfloat16 *>(out), static_cast<const uint4 *>(wb)};
    conv16_tc_kernel<<<tiles, TC_THREADS, TC_SMEM, st>>>(map, a);
    return cudaGetLastError();
}

cudaError_t conv16_tc_status(int *err) {
    cudaError_t e = cudaMemcpyFromSymbol(err, g_conv_tc_err, sizeof(int));
    if (e != cudaSuccess) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(g_conv_tc_err, &zero, sizeof(int));
}

}  // namespace smg
