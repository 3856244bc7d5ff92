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

// Phase-timing hook for latency studies: compiled out unless SMG_GRAM_TRACE names a device
// function `void f(int phase)`.
#ifdef SMG_GRAM_TRACE
#define GT_TRACE(k) SMG_GRAM_TRACE(k)
#else
#define GT_TRACE(k) ((void)0)
#endif

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

// The fixed-point magnitude M = round(|x| 2^(49 - E)) < 2^49 of x relative to 2^E (E from the
// column's largest magnitude) as two 32-bit words (hi has 17 bits), and x's sign bit.  Integer
// operations only.
__device__ __forceinline__ void gt_fixed(double x, int E, uint32_t &hi, uint32_t &lo, uint32_t &sgn) {
    const uint32_t bh = static_cast<uint32_t>(__double2hiint(x)), bl = static_cast<uint32_t>(__double2loint(x));
    sgn = bh & 0x80000000u;
    const int ex = static_cast<int>((bh >> 20) & 0x7ffu);
    hi = 0u;
    lo = 0u;
    // |x| 2^(49 - E) = m 2^-sh with the 53-bit significand m and sh = 1026 + E - ex >= 4
    const int sh = 1026 + E - ex;
    if (ex != 0 && sh < 54) {
        uint32_t mh = (bh & 0xfffffu) | 0x100000u, ml = bl;
        if (sh <= 32) {  // round to nearest: add 2^(sh-1), then shift
            const uint32_t t = ml + (1u << (sh - 1));
            mh += (t < ml) ? 1u : 0u;
            ml = t;
        } else {
            mh += 1u << (sh - 33);
        }
        if (sh < 32) {
            lo = __funnelshift_r(ml, mh, sh);
            hi = mh >> sh;
        } else {
            lo = mh >> (sh - 32);
        }
        if (hi >= (1u << 17)) {  // rounded up to 2^49: keep the largest 49-bit value
            hi = (1u << 17) - 1u;
            lo = 0xffffffffu;
        }
    }
}

// Digit s (7 bits, s = 0 most significant) of M = hi:lo.
template <int S>
__device__ __forceinline__ uint32_t gt_digit(uint32_t hi, uint32_t lo) {
    if constexpr (S == 0) return hi >> 10;
    else if constexpr (S == 1) return (hi >> 3) & 127u;
    else if constexpr (S == 2) return __funnelshift_r(lo, hi, 28) & 127u;
    else return (lo >> (42 - 7 * S)) & 127u;
}

// The seven digits of two entries (rows r, r+1 of one column) as BF16 pairs: word s holds digit
// s of the first entry in its low half and of the second in its high half.  A digit v < 128 is
// made a BF16 value by writing it into the significand of 128 (bits 0x4300 | v = 128 + v
// exactly) and subtracting 128 in BF16 arithmetic (exact), then the entry's sign is applied.
template <int S>
__device__ __forceinline__ uint32_t gt_pair(uint32_t h0, uint32_t l0, uint32_t h1, uint32_t l1, uint32_t sg) {
    const uint32_t w = 0x43004300u | gt_digit<S>(h0, l0) | (gt_digit<S>(h1, l1) << 16);
    const __nv_bfloat162 v = __hsub2(*reinterpret_cast<const __nv_bfloat162 *>(&w),
                                     __halves2bfloat162(__ushort_as_bfloat16(0x4300u), __ushort_as_bfloat16(0x4300u)));
    return *reinterpret_cast<const uint32_t *>(&v) ^ sg;
}

// Pre-pass: the largest |x| of every column of U (bit patterns of non-negative doubles order
// like unsigned integers).
__global__ void gram_colmax_kernel(long long n, int k, const double *__restrict__ U, long long ld,
                                   unsigned long long *__restrict__ cmax) {
    const int j = blockIdx.y;
    const double *col = U + static_cast<long long>(j) * ld;
    unsigned long long m = 0;
    // four independent loads in flight per thread
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        unsigned long long b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            b[u] = static_cast<unsigned long long>(__double_as_longlong(col[i + u * stride])) & 0x7fffffffffffffffull;
#pragma unroll
        for (int u = 0; u < 4; ++u) m = b[u] > m ? b[u] : m;
    }
    for (; i < n; i += stride) {
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

// Drain: fold the exact regions (weights 0..4) of this thread's accumulator share into acc.
template <int CPW>
__device__ __forceinline__ void gt_drain(uint32_t tmem, int q, int cb, int NP, long long (&acc)[CPW]) {
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
            // an integer-valued float below 2^22 in magnitude: adding 1.5 2^23 puts it in the low
            // mantissa bits
            const int v = static_cast<int>(__float_as_uint(__uint_as_float(r[x]) + 12582912.0f)) - 0x4B400000;
            acc[x] += static_cast<long long>(v) << (7 * (GT_EXACT - 1 - c));
        }
    }
}

// The digit-split Gram of the CTA's row range.  Items (column j, row pair): 8 columns x 4 row
// pairs per warp access, so a warp's 4-byte digit stores fill 128 contiguous bytes of a K chunk.
// A thread owns at most (NP + 64) / 16 items ((k1 <= NP plus k2 <= 64 columns) / 8 x 256 items /
// 512 threads); their rows
// are loaded into registers two stages ahead (two register sets, the stage loop unrolled by two so
// that each set is named statically), so a stage's loads have the whole previous stage to arrive.
// With two digit buffers (when they fit in shared memory) the digits of stage st are written while
// the MMAs of stage st-1 read the other buffer.
constexpr int GT_PREFETCH = 4;  // stages ahead the rows are prefetched into L2

template <int NP>
__global__ void __launch_bounds__(GT_THREADS, 1)
    gram_tc_kernel(long long n, int k1, const double *__restrict__ U, long long ldu, int k2,
                   const double *__restrict__ V, long long ldv, const unsigned long long *__restrict__ cmax_u,
                   const unsigned long long *__restrict__ cmax_v, int stages_per_cta, int sym,
                   double *__restrict__ part) {
    constexpr int UBYTES = 7 * GT_KCH * NP * 16;  // seven digit matrices of U (N side)
    constexpr int BUFB = GT_VBYTES + UBYTES;       // one digit buffer
    constexpr int NBUF = (2 * BUFB + 1024 <= 227 * 1024) ? 2 : 1;
    constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((static_cast<uint32_t>(NP) >> 3) << 17) |
                               ((128u >> 4) << 24);
    constexpr int CPW = NP / 4;  // accumulator columns each of the four warps of a lane quarter drains
    static_assert(GT_REGIONS * NP <= 512, "regions exceed the tensor memory");
    extern __shared__ __align__(1024) unsigned char sm[];
    // buffer b: V digits [p 4][kchunk 8][row 128][8 bf16], then U digits [s 7][kchunk 8][row NP][8 bf16]
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + NBUF * BUFB);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *s_fail = reinterpret_cast<int *>(tslot + 1);
    int *s_eu = s_fail + 1;                 // [64]
    int *s_ev = s_eu + 64;                  // [64]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const long long nst = (n + GT_ROWS - 1) / GT_ROWS;
    const long long st0 = static_cast<long long>(blockIdx.x) * stages_per_cta;
    const long long st1 = min(nst, st0 + stages_per_cta);

    for (int i = tid; i < NBUF * BUFB / 16; i += GT_THREADS)
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

    // this thread's items: column jj (U's columns, then V's) and row pair rp; packed jj | rp << 8
    // a symmetric product (V = U) slices U's columns once and stores them on both sides
    constexpr int GI = (NP + 64) / 16;  // items per thread
    const int ncol = sym ? k1 : k1 + k2, ncg = (ncol + 7) / 8;
    int pk[GI];
    const double *cp[GI];
#pragma unroll
    for (int q2 = 0; q2 < GI; ++q2) {
        const int it = tid + q2 * GT_THREADS;
        const int jj = (it & 7) + 8 * ((it >> 5) % ncg);
        const int rp = ((it >> 3) & 3) + 4 * ((it >> 5) / ncg);
        const bool valid = it < ncg * 256 && jj < ncol && rp < GT_ROWS / 2;
        pk[q2] = valid ? (jj | (rp << 8)) : -1;
        const int j = jj < k1 ? jj : jj - k1;
        cp[q2] = valid ? (jj < k1 ? U + static_cast<long long>(j) * ldu : V + static_cast<long long>(j) * ldv) + 2 * rp
                       : nullptr;
    }
    double xa0[GI], xb0[GI], xa1[GI], xb1[GI];
    auto load_stage = [&](long long st, double (&xa)[GI], double (&xb)[GI]) {
        const long long r0 = st * GT_ROWS;
#pragma unroll
        for (int q2 = 0; q2 < GI; ++q2) {
            xa[q2] = 0.0;
            xb[q2] = 0.0;
            if (pk[q2] >= 0 && st < st1) {
                // two scalar loads: a column of an odd-length block is only 8-byte aligned
                const long long i0 = r0 + 2 * (pk[q2] >> 8);
                if (i0 < n) xa[q2] = cp[q2][r0];
                if (i0 + 1 < n) xb[q2] = cp[q2][r0 + 1];
            }
        }
    };
    auto prefetch_stage = [&](long long st) {
        if (st >= st1) return;
        const long long r0 = st * GT_ROWS;
#pragma unroll
        for (int q2 = 0; q2 < GI; ++q2) {
            // one prefetch per 32-byte sector: the even lanes of a row-pair group
            if (pk[q2] >= 0 && ((pk[q2] >> 8) & 1) == 0 && r0 + 2 * (pk[q2] >> 8) < n)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(cp[q2] + r0));
        }
    };
    auto slice_stage = [&](int b, const double (&xa)[GI], const double (&xb)[GI]) {
        unsigned char *Vs = sm + b * BUFB, *Us = Vs + GT_VBYTES;
#pragma unroll
        for (int q2 = 0; q2 < GI; ++q2) {
            if (pk[q2] < 0) continue;
            const int jj = pk[q2] & 0xff, rp = pk[q2] >> 8;
            const bool isu = jj < k1;
            const int j = isu ? jj : jj - k1;
            const int E = isu ? s_eu[j] : s_ev[j];
            uint32_t h0, l0, s0, h1, l1, s1;
            gt_fixed(xa[q2], E, h0, l0, s0);
            gt_fixed(xb[q2], E, h1, l1, s1);
            const uint32_t sg = (s0 >> 16) | s1;
            uint32_t w[7];
            w[0] = gt_pair<0>(h0, l0, h1, l1, sg);
            w[1] = gt_pair<1>(h0, l0, h1, l1, sg);
            w[2] = gt_pair<2>(h0, l0, h1, l1, sg);
            w[3] = gt_pair<3>(h0, l0, h1, l1, sg);
            w[4] = gt_pair<4>(h0, l0, h1, l1, sg);
            w[5] = gt_pair<5>(h0, l0, h1, l1, sg);
            w[6] = gt_pair<6>(h0, l0, h1, l1, sg);
            const int kc = (2 * rp) >> 3, ko = (2 * rp) & 7;
            if (isu) {
                unsigned char *base = Us + (kc * NP + j) * 16 + ko * 2;
#pragma unroll
                for (int s = 0; s < 7; ++s) *reinterpret_cast<uint32_t *>(base + s * GT_KCH * NP * 16) = w[s];
            }
            if (!isu || sym) {
                unsigned char *base = Vs + (kc * 128 + j) * 16 + ko * 2;
#pragma unroll
                for (int s = 0; s < 7; ++s)
                    *reinterpret_cast<uint32_t *>(base + ((s >> 1) * GT_KCH * 128 + (s & 1) * 64) * 16) = w[s];
            }
        }
    };
    auto issue_mmas = [&](int b, bool first) {
        // 19 MMAs per 16-row K-step; exact regions restart every stage, the others accumulate
        // over the CTA's range (reset only in its first stage)
        const uint32_t vb = smem_u32(sm + b * BUFB), ub = vb + GT_VBYTES;
        uint32_t touched = 0;
        for (int p = 0; p < 4; ++p) {
            const int smax = min(6, 7 - 2 * p);
            const uint64_t a0 = gt_desc(vb + static_cast<uint32_t>(p * GT_KCH * 128 * 16), 128 * 16, 128);
            for (int s = 0; s <= smax; ++s) {
                const int c = s + 2 * p;
                const bool fresh = !((touched >> c) & 1u) && (c < GT_EXACT || first);
                const uint64_t b0 = gt_desc(ub + static_cast<uint32_t>(s * GT_KCH * NP * 16), NP * 16, 128);
#pragma unroll
                for (int kk = 0; kk < GT_KCH / 2; ++kk) {
                    // K-step kk: K chunks 2kk, 2kk+1 (start address + 2kk chunk strides, >> 4)
                    const uint64_t ad = a0 + static_cast<uint64_t>(kk * 2 * 128);
                    const uint64_t bd = b0 + static_cast<uint64_t>(kk * 2 * NP);
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
    };

    // this thread's share of the accumulators: lane quarter q (TMEM lanes 32q..), columns
    // [cb CPW, (cb + 1) CPW) of every region
    const int q = warp & 3, cb = warp >> 2;
    long long acc[CPW];
#pragma unroll
    for (int c = 0; c < CPW; ++c) acc[c] = 0;
    bool ok = true;
    uint32_t phase = 0;
    // wait (one thread, bounded) for the last committed MMAs, then drain them
    auto wait_drain = [&]() -> bool {
        if (tid == 0 && !gt_wait(smem_u32(mbar), phase)) *s_fail = 1;
        phase ^= 1u;
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (*s_fail) return false;
        GT_TRACE(2);
        gt_drain<CPW>(tmem, q, cb, NP, acc);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();  // the exact regions and a digit buffer are reused next
        GT_TRACE(3);
        return true;
    };
    // one stage: slice its rows (loaded two stages ago), hand the digits to the tensor cores,
    // load the rows of stage st + 2 into the registers just consumed
    auto stage = [&](long long st, double (&xa)[GI], double (&xb)[GI]) -> bool {
        GT_TRACE(0);
        const int b = NBUF == 2 ? static_cast<int>((st - st0) & 1) : 0;
        slice_stage(b, xa, xb);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        GT_TRACE(1);
        // two buffers: the previous stage's MMAs (reading the other buffer) ran during the slicing
        if (NBUF == 2 && st > st0 && !wait_drain()) return false;
        if (tid == 0) issue_mmas(b, st == st0);
        load_stage(st + 2, xa, xb);  // in flight during the next stage
        prefetch_stage(st + GT_PREFETCH);  // into L2, so that the register loads find it there
        if (NBUF == 1 && !wait_drain()) return false;
        return true;
    };
    for (int d = 2; d < GT_PREFETCH; ++d) prefetch_stage(st0 + d);
    if (st0 < st1) {
        load_stage(st0, xa0, xb0);
        load_stage(st0 + 1, xa1, xb1);
    }
    for (long long st = st0; st < st1 && ok; st += 2) {
        if (!stage(st, xa0, xb0)) {
            ok = false;
            break;
        }
        if (st + 1 < st1 && !stage(st + 1, xa1, xb1)) ok = false;
    }
    if (ok && NBUF == 2 && st0 < st1 && !wait_drain()) ok = false;
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
                    double *G, void *work, int num_sms, cudaStream_t st, bool reuse_u_cmax) {
    if (k1 < 1 || k2 < 1 || k1 > 64 || k2 > 64 || n < 1) return cudaErrorInvalidValue;
    unsigned long long *cmax = static_cast<unsigned long long *>(work);
    double *part = reinterpret_cast<double *>(cmax + 128);
    cudaError_t e = cudaMemsetAsync(cmax + (reuse_u_cmax ? 64 : 0), 0, sizeof(unsigned long long) * (reuse_u_cmax ? 64 : 128),
                                    st);
    if (e != cudaSuccess) return e;
    {
        // about 16 CTAs per SM over all columns
        const int bx = static_cast<int>(std::min<long long>((n + 255) / 256, std::max(1, 16 * num_sms / std::max(1, k1))));
        if (!reuse_u_cmax) gram_colmax_kernel<<<dim3(std::max(1, bx), k1), 256, 0, st>>>(n, k1, U, ldu, cmax);
        if (V != U || ldv != ldu || k2 != k1) {
            const int by = static_cast<int>(std::min<long long>((n + 255) / 256, std::max(1, 16 * num_sms / std::max(1, k2))));
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
    const int sym = (V == U && ldv == ldu && k2 == k1) ? 1 : 0;
    const size_t bufb = GT_VBYTES + 7 * GT_KCH * NP * 16;
    const size_t smem = ((2 * bufb + 1024 <= 227 * 1024) ? 2 : 1) * bufb + 64 + 2 * 64 * sizeof(int);
    switch (NP) {
    case 16:
        e = cudaFuncSetAttribute(gram_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<16><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), sym, part);
        break;
    case 32:
        e = cudaFuncSetAttribute(gram_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<32><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), sym, part);
        break;
    case 48:
        e = cudaFuncSetAttribute(gram_tc_kernel<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<48><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), sym, part);
        break;
    default:
        e = cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e == cudaSuccess)
            gram_tc_kernel<64><<<ctas, GT_THREADS, smem, st>>>(n, k1, U, ldu, k2, V, ldv, cmax, cmax + 64, static_cast<int>(per), sym, part);
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
