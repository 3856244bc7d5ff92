// gram_tc.cu -- FP64-accurate Gram products G = U^T V of tall-skinny blocks on the tcgen05 tensor
// cores (LOBPCG's Rayleigh-Ritz and orthogonalisation products, section "Preconditioning of
// LOBPCG with SMG" of arXiv:1212.6680: the block method's dense inner products).
//
// The tensor cores multiply BF16 and accumulate in FP32; FP64 accuracy comes from splitting every
// entry into integer digits that BF16 holds exactly (an Ozaki-type splitting):
//   * each column j gets a power of two 2^E_j > max_i |x_ij| (a pre-pass over the column);
//   * x = sign * M * 2^(E - 49), M = round(|x| 2^(49 - E)) < 2^49, is cut into seven 7-bit digits
//     a_s = (M >> (42 - 7 s)) & 127, so x = sum_s a_s 2^(E - 7 (s + 1)) up to 2^(E - 50);
//   * u^T v = 2^(E_u + E_v) sum_{s,t} 2^(-7 (s + t + 2)) (a_s^T b_t): the digit products
//     a_s^T b_t over 64 rows are integers below 2^22, which the FP32 accumulator holds exactly.
// Digit pairs of equal weight d = s + t share an accumulator.  Pairs with d <= 7 are kept (the
// dropped ones are below 2^-63 of |u|^T|v| each); a CPU emulation of exactly this scheme gives
// ~4e-16 relative to ||u|| ||v|| where keeping only d <= 6 leaves ~1e-13.
//
// One MMA (M = 128, N = NP >= k1, K = 16) multiplies a "stacked" A operand -- rows 0..63 digit 2p
// of V's columns, rows 64..127 digit 2p+1 -- with digit s of U: accumulator lanes 0..63 receive
// the pair (s, 2p) (weight d = s + 2p) and lanes 64..127 the pair (s, 2p+1) (weight d + 1), both
// in the TMEM columns of region c = s + 2p.  Per 16-row K-step that is 19 MMAs (p = 0..3,
// s <= min(6, 7 - 2p)) into 8 regions of NP columns.
//
// Exactness and draining: per 64-row stage every region of weight <= 4 is an exact integer below
// 2^22; the CTA moves it out of TMEM after each stage (tcgen05.ld, FP32 -> integer by the 1.5 2^23
// rounding constant) and folds the five regions into one 64-bit integer per entry
// (sum_c R_c 2^(7 (4 - c)), exact over up to 512 stages).  Regions of weight >= 5 contribute
// below 2^-35 of the result: they stay in TMEM in FP32 over the CTA's whole row range (their FP32
// rounding is far below FP64's) and are read once at the end.  Each CTA writes its FP64 partial;
// a second kernel sums the partials.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "../../include/smg.h"
#include "gram_tc.h"
#include "smg_internal.h"

namespace smg {
namespace {

constexpr int GT_THREADS = 512;
constexpr int GT_ROWS = 64;                    // rows per stage (drain period)
constexpr int GT_KCH = GT_ROWS / 8;            // 8-element K chunks per stage
constexpr int GT_MAX_STAGES = 512;             // per CTA: keeps the 64-bit folds exact
constexpr int GT_VBYTES = 4 * GT_KCH * 128 * 16;  // four stacked M-tiles (64 KB)
constexpr int GT_REGIONS = 8;
constexpr int GT_EXACT = 5;                    // regions drained every stage (weights 0..4)
constexpr long long kGtWaitLimit = 1ll << 26;  // mbarrier polls before giving up

__device__ int g_gram_tc_err = 0;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (no swizzle, K-major): start >> 4, leading (K-direction core
// matrix) byte offset >> 4 at bits 16-29, stride (8-row group) byte offset >> 4 at bits 32-45,
// version 1 at bit 46.
__device__ __forceinline__ uint64_t gt_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;
    return d;
}

__device__ __forceinline__ bool gt_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kGtWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        __nanosleep(20);
    }
    return false;
}

// The seven digits of x relative to 2^E (E from the column's largest magnitude), as BF16 bit
// patterns (exact: integers below 128), sign applied.  Integer operations only.
__device__ __forceinline__ void gt_digits(double x, int E, uint32_t (&d)[7]) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t sign = static_cast<uint32_t>(b >> 48) & 0x8000u;
    const int ex = static_cast<int>((b >> 52) & 0x7ffu);
    unsigned long long M = 0;
    if (ex != 0) {
        const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
        // |x| 2^(49 - E) = m 2^(ex - 1075 + 49 - E) = m >> sh, sh >= 4; rounded to nearest
        const int sh = 1026 + E - ex;
        if (sh < 60) {
            M = (m + (1ull << (sh - 1))) >> sh;
            if (M >= (1ull << 49)) M = (1ull << 49) - 1;
        }
    }
#pragma unroll
    for (int s = 0; s < 7; ++s) {
        const uint32_t v = static_cast<uint32_t>(M >> (42 - 7 * s)) & 127u;
        // v as a float via 2^23 + v - 2^23; its upper 16 bits are the BF16 pattern (v < 256)
        const float f = __uint_as_float(0x4B000000u | v) - 8388608.0f;
        d[s] = (__float_as_uint(f) >> 16) | (v ? sign : 0u);
    }
}

// Pre-pass: the largest |x| of every column of U (bit patterns of non-negative doubles order
// like unsigned integers).
__global__ void gram_colmax_kernel(long long n, int k, const double *__restrict__ U, long long ld,
                                   unsigned long long *__restrict__ cmax) {
    const int j = blockIdx.y;
    const double *col = U + static_cast<long long>(j) * ld;
    unsigned long long m = 0;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(col[i])) & 0x7fffffffffffffffull;
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_down_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m != 0) atomicMax(cmax + j, m);
}

// E = floor(log2 max|x|) + 1, so every |x| < 2^E (0 for an all-zero column).
__device__ __forceinline__ int gt_exp(unsigned long long mx) {
    if (mx == 0) return 0;
    return static_cast<int>((mx >> 52) & 0x7ffu) - 1023 + 1;
}

template <int NP>
__global__ void __launch_bounds__(GT_THREADS, 1)
    gram_tc_kernel(long long n, int k1, const double *__restrict__ U, long long ldu, int k2,
                   const double *__restrict__ V, long long ldv, const unsigned long long *__restrict__ cmax_u,
                   const unsigned long long *__restrict__ cmax_v, int stages_per_cta, double *__restrict__ part) {
    constexpr int UBYTES = 7 * GT_KCH * NP * 16;  // seven digit matrices of U (N side)
    constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((static_cast<uint32_t>(NP) >> 3) << 17) |
                               ((128u >> 4) << 24);
    constexpr int CPW = NP / 4;  // accumulator columns each of the four warps of a lane quarter drains
    static_assert(GT_REGIONS * NP <= 512, "regions exceed the tensor memory");
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *Vs = sm;                 // [p 4][kchunk 8][row 128][8 bf16]
    unsigned char *Us = sm + GT_VBYTES;     // [s 7][kchunk 8][row NP][8 bf16]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(Us + UBYTES);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *s_fail = reinterpret_cast<int *>(tslot + 1);
    int *s_eu = s_fail + 1;                 // [64]
    int *s_ev = s_eu + 64;                  // [64]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const long long nst = (n + GT_ROWS - 1) / GT_ROWS;
    const long long st0 = static_cast<long long>(blockIdx.x) * stages_per_cta;
    const long long st1 = min(nst, st0 + stages_per_cta);

    for (int i = tid; i < (GT_VBYTES + UBYTES) / 16; i += GT_THREADS)
        reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);  // padding rows stay zero
    if (tid < 64) {
        s_eu[tid] = tid < k1 ? gt_exp(cmax_u[tid]) : 0;
        s_ev[tid] = tid < k2 ? gt_exp(cmax_v[tid]) : 0;
    }
    if (tid == 0) {
        *s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // this thread's share of the accumulators: lane quarter q (TMEM lanes 32q..), columns
    // [cb CPW, (cb + 1) CPW) of every region
    const int q = warp & 3, cb = warp >> 2;
    long long acc[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) acc[c] = 0;
    bool ok = true;
    uint32_t phase = 0;
    for (long long st = st0; st < st1; ++st) {
        const long long r0 = st * GT_ROWS;
        // ---- digits of this stage's 64 rows into shared memory ----
        // an item is (column j, row pair rp): 8 columns x 4 row pairs per warp access, so a warp's
        // 4-byte stores fill 128 contiguous bytes of a K chunk
        const int ncol = k1 + k2, ncg = (ncol + 7) / 8;
        for (int it = tid; it < ncg * 256; it += GT_THREADS) {
            const int jj = (it & 7) + 8 * ((it >> 5) % ncg);
            const int rp = ((it >> 3) & 3) + 4 * ((it >> 5) / ncg);
            if (jj >= ncol || rp >= GT_ROWS / 2) continue;
            const bool isu = jj < k1;
            const int j = isu ? jj : jj - k1;
            const double *col = isu ? U + static_cast<long long>(j) * ldu : V + static_cast<long long>(j) * ldv;
            const long long i0 = r0 + 2 * rp;
            const double x0 = i0 < n ? col[i0] : 0.0, x1 = i0 + 1 < n ? col[i0 + 1] : 0.0;
            uint32_t d0[7], d1[7];
            const int E = isu ? s_eu[j] : s_ev[j];
            gt_digits(x0, E, d0);
            gt_digits(x1, E, d1);
            const int kc = (2 * rp) >> 3, ko = (2 * rp) & 7;
#pragma unroll
            for (int s = 0; s < 7; ++s) {
                const uint32_t w = d0[s] | (d1[s] << 16);
                if (isu) {
                    *reinterpret_cast<uint32_t *>(Us + ((s * GT_KCH + kc) * NP + j) * 16 + ko * 2) = w;
                } else {
                    const int p = s >> 1, row = (s & 1) * 64 + j;
                    *reinterpret_cast<uint32_t *>(Vs + ((p * GT_KCH + kc) * 128 + row) * 16 + ko * 2) = w;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // ---- the stage's MMAs, issued by one thread ----
        if (tid == 0) {
            uint32_t touched = 0;  // regions written since they were last reset
            const uint32_t vb = smem_u32(Vs), ub = smem_u32(Us);
            for (int p = 0; p < 4; ++p) {
                const int smax = min(6, 7 - 2 * p);
                for (int s = 0; s <= smax; ++s) {
                    const int c = s + 2 * p;
                    // exact regions restart every stage; the others accumulate over the CTA
                    const bool fresh = c < GT_EXACT ? !((touched >> c) & 1u) : (st == st0 && !((touched >> c) & 1u));
#pragma unroll
                    for (int kk = 0; kk < GT_KCH / 2; ++kk) {
                        const uint64_t ad = gt_desc(vb + static_cast<uint32_t>((p * GT_KCH + 2 * kk) * 128 * 16), 128 * 16, 128);
                        const uint64_t bd = gt_desc(ub + static_cast<uint32_t>((s * GT_KCH + 2 * kk) * NP * 16), NP * 16, 128);
                        const uint32_t accf = (fresh && kk == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + c * NP),
                            "l"(ad), "l"(bd), "r"(IDESC), "r"(accf));
                    }
                    touched |= 1u << c;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mbar))
                         : "memory");
        }
        // ---- wait (one thread, bounded), then fold the exact regions into the 64-bit accumulators ----
        if (tid == 0 && !gt_wait(smem_u32(mbar), phase)) *s_fail = 1;
        phase ^= 1u;
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (*s_fail) {
            ok = false;
            break;
        }
#pragma unroll
        for (int c = 0; c < GT_EXACT; ++c) {
            uint32_t r[CPW];
            const uint32_t ta = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(c * NP + cb * CPW);
            if constexpr (CPW == 4) {
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(ta));
            } else if constexpr (CPW == 8) {
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(ta));
            } else if constexpr (CPW == 12) {
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7])
                             : "r"(ta));
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]) : "r"(ta + 8));
            } else {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(ta));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int x = 0; x < CPW; ++x) {
                // an integer-valued float below 2^22 in magnitude: adding 1.5 2^23 puts it in the
                // low mantissa bits
                const int v = static_cast<int>(__float_as_uint(__uint_as_float(r[x]) + 12582912.0f)) - 0x4B400000;
                acc[x] += static_cast<long long>(v) << (7 * (GT_EXACT - 1 - c));
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // the digits and the exact regions are reused by the next stage
    }
    if (!ok && lane == 0) atomicExch(&g_gram_tc_err, 1);
    // ---- this CTA's partial: exact part + the FP32 regions of weight >= 5 ----
    // lane quarter q: V column jv = 32 (q & 1) + lane, digit-pair weight offset h = q >> 1
    const int jv = 32 * (q & 1) + lane, h = q >> 1;
    double val[CPW];
#pragma unroll
    for (int x = 0; x < CPW; ++x) val[x] = ldexp(static_cast<double>(acc[x]), -7 * (GT_EXACT - 1) - 14 - 7 * h);
    if (ok && st0 < st1) {
#pragma unroll
        for (int c = GT_EXACT; c < GT_REGIONS; ++c) {
            const uint32_t ta = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(c * NP + cb * CPW);
#pragma unroll
            for (int x = 0; x < CPW; ++x) {
                uint32_t r;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(ta + x));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                val[x] += ldexp(static_cast<double>(__uint_as_float(r)), -7 * (c + 2 + h));
            }
        }
    }
    if (jv < k2) {
#pragma unroll
        for (int x = 0; x < CPW; ++x) {
            const int ju = cb * CPW + x;
            if (ju >= k1) continue;
            // part[cta][h][ju][jv]
            part[((static_cast<long long>(blockIdx.x) * 2 + h) * 64 + ju) * 64 + jv] =
                ldexp(val[x], s_eu[ju] + s_ev[jv]);
        }
    }
    if (!ok && tid == 0) gt_wait(smem_u32(mbar), phase ^ 1u);  // MMAs may still be in flight (bounded)
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// G (k1 x k2, row-major) = sum over CTAs and the two lane halves of the partials; one warp per
// entry (launched with 32 threads).
__global__ void gram_tc_reduce_kernel(int nparts, int k1, int k2, const double *__restrict__ part,
                                      double *__restrict__ G) {
    const int e = blockIdx.x;  // entry
    const int ju = e / k2, jv = e - ju * k2;
    double s = 0.0, c = 0.0;   // TwoSum-compensated sum
    for (int t = threadIdx.x; t < 2 * nparts; t += blockDim.x) {
        const double v = part[(static_cast<long long>(t) * 64 + ju) * 64 + jv];
        const double y = s + v, bp = y - s;
        c += (s - (y - bp)) + (v - bp);
        s = y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double vs = __shfl_down_sync(0xffffffffu, s, o), vc = __shfl_down_sync(0xffffffffu, c, o);
        const double y = s + vs, bp = y - s;
        c += ((s - (y - bp)) + (vs - bp)) + vc;
        s = y;
    }
    if (threadIdx.x == 0) G[e] = s + c;
}

}  // namespace

size_t gram_tc_workspace_bytes(long long n) {
    // gram_tc gives every CTA at least 32 stages (or all of them)
    const long long nst = (n + GT_ROWS - 1) / GT_ROWS;
    const long long maxctas = std::max<long long>(1, (nst + 31) / 32);
    return sizeof(unsigned long long) * 128 + sizeof(double) * static_cast<size_t>(maxctas) * 2 * 64 * 64;
}

cudaError_t gram_tc(long long n, int k1, const double *U, long long ldu, int k2, const double *V, long long ldv,
                    double *G, void *work, int num_sms, cudaStream_t st) {
    if (k1 < 1 || k2 < 1 || k1 > 64 || k2 > 64 || n < 1) return cudaErrorInvalidValue;
    unsigned long long *cmax = static_cast<unsigned long long *>(work);
    double *part = reinterpret_cast<double *>(cmax + 128);
    cudaError_t e = cudaMemsetAsync(cmax, 0, sizeof(unsigned long long) * 128, st);
    if (e != cudaSuccess) return e;
    {
        const int bx = static_cast<int>(std::min<long long>((n + 255) / 256, std::max(1, 4 * num_sms / std::max(1, k1))));
        gram_colmax_kernel<<<dim3(std::max(1, bx), k1), 256, 0, st>>>(n, k1, U, ldu, cmax);
        if (V != U || ldv != ldu || k2 != k1) {
            const int by = static_cast<int>(std::min<long long>((n + 255) / 256, std::max(1, 4 * num_sms / std::max(1, k2))));
            gram_colmax_kernel<<<dim3(std::max(1, by), k2), 256, 0, st>>>(n, k2, V, ldv, cmax + 64);
        } else {
            e = cudaMemcpyAsync(cmax + 64, cmax, sizeof(unsigned long long) * 64, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
    }
    const long long nst = (n + GT_ROWS - 1) / GT_ROWS;
    // one CTA per SM while that keeps at least 32 stages per CTA, at most GT_MAX_STAGES per CTA
    long long per = std::max<long long>(32, (nst + num_sms - 1) / num_sms);
    per = std::min<long long>(per, GT_MAX_STAGES);
    const int ctas = static_cast<int>((nst + per - 1) / per);
    const int NP = ((k1 + 15) / 16) * 16;
    const size_t smem = GT_VBYTES + 7 * GT_KCH * NP * 16 + 64 + 2 * 64 * sizeof(int);
    switch (NP) {
    case 16:
        e = cudaFuncSetAttribute(gram_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<16><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), part);
        break;
    case 32:
        e = cudaFuncSetAttribute(gram_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<32><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), part);
        break;
    case 48:
        e = cudaFuncSetAttribute(gram_tc_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<48><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), part);
        break;
    default:
        e = cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<64><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), part);
        break;
    }
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gram_tc_reduce_kernel<<<k1 * k2, 32, 0, st>>>(ctas, k1, k2, part, G);  // one warp per entry
    return cudaGetLastError();
}

cudaError_t gram_tc_status(int *err) {
    cudaError_t e = cudaMemcpyFromSymbol(err, g_gram_tc_err, sizeof(int));
    if (e != cudaSuccess) return e;
    const int zero = 0;
    return cudaMemcpyToSymbol(g_gram_tc_err, &zero, sizeof(int));
}

}  // namespace smg

// ---- C ABI ------------------------------------------------------------------------------------
extern "C" int smg_gram(long long n, int k1, const double *U, int k2, const double *V, double *G, void *stream) {
    if (n < 1 || k1 < 1 || k2 < 1 || k1 > 64 || k2 > 64) {
        smg::set_last_error("smg_gram: n >= 1 and 1 <= k1, k2 <= 64 required");
        return SMG_ERR_ARG;
    }
    if (U == nullptr || V == nullptr || G == nullptr) {
        smg::set_last_error("smg_gram: null pointer");
        return SMG_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    void *work = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&work, smg::gram_tc_workspace_bytes(n));
    if (e == cudaSuccess) e = smg::gram_tc(n, k1, U, n, k2, V, n, G, work, nsm, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    int err = 0;
    if (e == cudaSuccess) e = smg::gram_tc_status(&err);
    cudaFree(work);
    if (e != cudaSuccess) {
        smg::set_last_error(std::string("smg_gram: ") + cudaGetErrorString(e));
        return SMG_ERR_CUDA;
    }
    if (err != 0) {
        smg::set_last_error("smg_gram: a tensor-core wait timed out");
        return SMG_ERR_TIMEOUT;
    }
    return SMG_OK;
}
