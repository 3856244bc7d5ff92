// lobpcg.cu -- block LOBPCG with SMG preconditioning.
//
// Locally optimal block preconditioned conjugate gradient (Knyazev's LOBPCG, which the paper
// runs through BLOPEX, section "Preconditioning of LOBPCG with SMG" of arXiv:1212.6680) for
// the m smallest eigenpairs of A:
//   R = A X - X Lambda;  W = T R (one batched V-cycle over the active columns);
//   Rayleigh-Ritz on span[X, W, P]:  (S^T A S) C = (S^T S) C Theta, S = [X W P];
//   X = S C_m, P = [W P] C_{WP,m}.
// Columns whose residual meets the tolerance are soft-locked (kept in X, dropped from W, P).
// W is orthogonalised against X and W, P are orthonormalised (Cholesky QR) before the
// Rayleigh-Ritz step, so S^T S stays well conditioned.
// Device: block kernels (Gram products with split-K partial sums, tall-skinny block updates)
// with FP64-accurate products carried out on the FP32 pipes ("double-float" arithmetic, see
// below).  Host: the k x k (k <= 3m) FP64 generalized eigenproblem by Cholesky reduction and
// cyclic Jacobi.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/smg.h"
#include "gram_tc.h"
#include "lobpcg.h"
#include "plane_relax.cuh"  // widen_f32 / narrow_f64 (integer-pipe conversions)

namespace smg {

namespace {

constexpr int kGT = 16;          // Gram output tile (kGT x kGT per CTA of kGT * kGT threads)
constexpr int kGRows = 64;       // rows staged per step
constexpr int kGChunk = 8192;    // rows per CTA (split-K; fewer for small products)
constexpr int kNormChunks = 256; // row chunks per column of the residual norms
constexpr int kMulCols = 16;     // output columns per block_mul thread

// ---- double-float arithmetic -------------------------------------------------------------------
// On this part an FP64 FMA costs as much SM time as ~64 FP32 ones, and the LOBPCG block kernels
// are nothing but FP64 multiply-adds.  They run instead on pairs of floats (hi, lo) with
// hi + lo = the FP64 operand to ~2^-48: Dekker's exact product via FMA (p = a*b,
// e = fma(a, b, -p), a*b = p + e exactly) plus the two cross terms, accumulated with Knuth's
// TwoSum (s = a + b and the exact rounding error of that addition), about a dozen FP32 operations
// per multiply-add.  Each FP64 input is split once (df_split); the final value is hi + lo in
// FP64.

// x = hi + lo with integer operations only (no FP64 or conversion instruction): hi keeps the top
// 24 significant bits of x (truncated, so exactly a float), lo the next 24 of the remaining 29
// mantissa bits (truncated: |x - hi - lo| < 2^-47 |x| for |x| >= 2^-75; below that lo underflows
// and only hi remains, 2^-24).  |x| < 2^-126 flushes to zero.  Entries of the normalised block
// vectors of a 128^3 problem are ~1e-3, far inside the exact range.
__device__ __forceinline__ void df_split(double x, float &hi, float &lo) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned sign = static_cast<unsigned>(b >> 32) & 0x80000000u;
    const int E = static_cast<int>((b >> 52) & 0x7ffu) - 1023;  // unbiased exponent
    if (E < -126 || E > 127) {  // zero, tiny, or beyond the float range (not met by this solver)
        hi = lo = 0.0f;
        if (E > 127) hi = __uint_as_float(sign | 0x7f800000u);
        return;
    }
    const unsigned mhi = static_cast<unsigned>((b >> 29) & 0x7fffffu);           // mantissa bits 51..29
    hi = __uint_as_float(sign | (static_cast<unsigned>(E + 127) << 23) | mhi);
    const unsigned L = static_cast<unsigned>(b & 0x1fffffffu);                   // mantissa bits 28..0
    if (L == 0u) {
        lo = 0.0f;
        return;
    }
    const int k = 31 - __clz(L);                  // L = 1.f x 2^k, lo = L x 2^(E - 52)
    const int fe = k + E - 52 + 127;
    if (fe <= 0) {
        lo = 0.0f;
        return;
    }
    const unsigned mant = (k >= 23) ? ((L >> (k - 23)) & 0x7fffffu) : ((L << (23 - k)) & 0x7fffffu);
    lo = __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | mant);
}

// (S, s) += a * b for a = ah + al, b = bh + bl.  The exact steps use the round-to-nearest
// intrinsics, which the compiler never contracts into FMAs (a fused S + ah*bh would break them).
__device__ __forceinline__ void df_mac(float &S, float &s, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    const float e = fmaf(ah, bh, -p);                  // ah*bh = p + e exactly
    const float t = fmaf(ah, bl, fmaf(al, bh, e));     // e + the cross terms (al*bl ~ 2^-48 dropped)
    const float u = __fadd_rn(S, p);                    // TwoSum(S, p)
    const float bb = __fsub_rn(u, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(u, bb)), __fsub_rn(p, bb));
    S = u;
    s = __fadd_rn(s, __fadd_rn(err, t));
}

__device__ __forceinline__ double df_value(float S, float s) { return widen_f32(S) + widen_f32(s); }

// Partial Gram: part[chunk][ti][tj] tile of U^T V over rows [chunk*rows, ...).  The tiles are
// small (no work on padding beyond the next multiple of 16) and, for a symmetric product
// (sym = 1, U^T V = V^T U), only the tiles on and above the diagonal are computed.  The 256
// threads form 4 row groups of 64; each thread accumulates a 2 x 2 block of the tile over every
// 4th staged row, reading its two U and two V operands (hi, lo) as one 16-byte shared-memory load
// each, so the kernel is bound by the FP32 pipe rather than by shared-memory loads.  The staged
// rows hold (hi, lo) pairs with the 16-byte column pairs XOR-swizzled by row (conflict-light
// stores, conflict-free loads).
__device__ __forceinline__ int gram_swz(int rr, int cc) { return ((((cc >> 1) ^ rr) & 7) << 1) | (cc & 1); }

__global__ void __launch_bounds__(256, 4) gram_partial_kernel(long long n, long long rows, int k1, int k2,
                                                           const double *__restrict__ U, const double *__restrict__ V,
                                                           double *__restrict__ part, int ntj, int sym) {
    __shared__ __align__(16) float2 su[kGRows][kGT], sv[kGRows][kGT];
    __shared__ double red[4][kGT * kGT];
    const int tile = blockIdx.y, ti = tile / ntj, tj = tile % ntj;
    if (sym && tj < ti) return;
    const int i0 = ti * kGT, j0 = tj * kGT;
    const long long r0 = static_cast<long long>(blockIdx.x) * rows;
    const long long r1 = min(n, r0 + rows);
    const int kg = threadIdx.x >> 6, t = threadIdx.x & 63, oi = t >> 3, oj = t & 7;  // outputs (2oi+a, 2oj+b)
    float S[4] = {0.0f, 0.0f, 0.0f, 0.0f}, sl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // this thread's staged elements: e = threadIdx.x + 256 q, row e % kGRows, column e / kGRows;
    // the next block's values are loaded into registers before the current block is computed
    constexpr int kPer = kGRows * kGT / (kGT * kGT);
    double nu[kPer], nv[kPer];
    auto fetch = [&](long long rb) {
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int e = threadIdx.x + q * kGT * kGT, rr = e % kGRows, cc = e / kGRows;
            const long long r = rb + rr;
            nu[q] = (r < r1 && i0 + cc < k1) ? U[static_cast<long long>(i0 + cc) * n + r] : 0.0;
            nv[q] = (r < r1 && j0 + cc < k2) ? V[static_cast<long long>(j0 + cc) * n + r] : 0.0;
        }
    };
    fetch(r0);
    for (long long rb = r0; rb < r1; rb += kGRows) {
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int e = threadIdx.x + q * kGT * kGT, rr = e % kGRows, cc = e / kGRows;
            float uh, ul, vh, vl;
            df_split(nu[q], uh, ul);
            df_split(nv[q], vh, vl);
            su[rr][gram_swz(rr, cc)] = make_float2(uh, ul);
            sv[rr][gram_swz(rr, cc)] = make_float2(vh, vl);
        }
        __syncthreads();
        if (rb + kGRows < r1) fetch(rb + kGRows);
#pragma unroll 4
        for (int q = 0; q < kGRows / 4; ++q) {
            const int rr = 4 * q + kg;
            const float4 a = *reinterpret_cast<const float4 *>(&su[rr][gram_swz(rr, 2 * oi)]);
            const float4 b = *reinterpret_cast<const float4 *>(&sv[rr][gram_swz(rr, 2 * oj)]);
            df_mac(S[0], sl[0], a.x, a.y, b.x, b.y);
            df_mac(S[1], sl[1], a.x, a.y, b.z, b.w);
            df_mac(S[2], sl[2], a.z, a.w, b.x, b.y);
            df_mac(S[3], sl[3], a.z, a.w, b.z, b.w);
        }
        __syncthreads();
    }
    const int o = (2 * oi) * kGT + 2 * oj;
    red[kg][o] = df_value(S[0], sl[0]);
    red[kg][o + 1] = df_value(S[1], sl[1]);
    red[kg][o + kGT] = df_value(S[2], sl[2]);
    red[kg][o + kGT + 1] = df_value(S[3], sl[3]);
    __syncthreads();
    const int idx = threadIdx.x;  // blockDim.x == kGT * kGT
    part[(static_cast<long long>(blockIdx.x) * gridDim.y + tile) * kGT * kGT + idx] =
        (red[0][idx] + red[1][idx]) + (red[2][idx] + red[3][idx]);
}

// Partial Gram of a narrow product (k1, k2 <= kSmallK): thread t of CTA `chunk` accumulates all
// k1 x k2 entries over rows chunk*rows + t, + 256, ... (coalesced loads of each column, no
// padding work), and the CTA adds its 256 partial sums in FP64; part[] takes the tiled kernel's
// layout (one 16 x 16 tile) so the same reduction follows.
constexpr int kSmallK = 4;
__global__ void __launch_bounds__(256) gram_small_kernel(long long n, long long rows, int k1, int k2,
                                                         const double *__restrict__ U, const double *__restrict__ V,
                                                         double *__restrict__ part) {
    __shared__ double red[8][kSmallK * kSmallK];
    const long long r0 = static_cast<long long>(blockIdx.x) * rows;
    const long long r1 = min(n, r0 + rows);
    float S[kSmallK][kSmallK], sl[kSmallK][kSmallK];
#pragma unroll
    for (int i = 0; i < kSmallK; ++i)
#pragma unroll
        for (int j = 0; j < kSmallK; ++j) S[i][j] = sl[i][j] = 0.0f;
    for (long long r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        float uh[kSmallK], ul[kSmallK], vh[kSmallK], vl[kSmallK];
#pragma unroll
        for (int i = 0; i < kSmallK; ++i) {
            df_split(i < k1 ? U[static_cast<long long>(i) * n + r] : 0.0, uh[i], ul[i]);
            df_split(i < k2 ? V[static_cast<long long>(i) * n + r] : 0.0, vh[i], vl[i]);
        }
#pragma unroll
        for (int i = 0; i < kSmallK; ++i)
#pragma unroll
            for (int j = 0; j < kSmallK; ++j)
                if (i < k1 && j < k2) df_mac(S[i][j], sl[i][j], uh[i], ul[i], vh[j], vl[j]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kSmallK; ++i)
#pragma unroll
        for (int j = 0; j < kSmallK; ++j) {
            double v = df_value(S[i][j], sl[i][j]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[w][i * kSmallK + j] = v;
        }
    __syncthreads();
    if (threadIdx.x < kSmallK * kSmallK) {
        const int i = threadIdx.x / kSmallK, j = threadIdx.x % kSmallK;
        double v = 0.0;
        for (int q = 0; q < 8; ++q) v += red[q][threadIdx.x];
        part[static_cast<long long>(blockIdx.x) * kGT * kGT + i * kGT + j] = v;
    }
}

// G[i][j] (k1 x k2 row-major) = sum over chunks of the partial tiles (compensated summation), one
// warp per entry: the lanes take every 32nd chunk, then the warp combines its 32 sums.  With
// sym, entries below the diagonal tiles come from the mirrored tile.
__device__ __forceinline__ void two_sum_add(double &s, double &c, double v) {
    const double t = s + v;
    const double bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}

__global__ void gram_reduce_kernel(int nchunks, int k1, int k2, int ntj, int ntiles, const double *__restrict__ part,
                                   double *__restrict__ G, int sym) {
    const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (idx >= k1 * k2) return;
    int i = idx / k2, j = idx % k2;
    if (sym && i / kGT > j / kGT) {
        const int t = i;
        i = j;
        j = t;
    }
    const int ti = i / kGT, tj = j / kGT, tile = ti * ntj + tj;
    const long long off = static_cast<long long>(tile) * kGT * kGT + (i - ti * kGT) * kGT + (j - tj * kGT);
    double s = 0.0, c = 0.0;
    for (int ch = lane; ch < nchunks; ch += 32) two_sum_add(s, c, part[static_cast<long long>(ch) * ntiles * kGT * kGT + off]);
    for (int o = 16; o > 0; o >>= 1) {
        const double so = __shfl_down_sync(0xffffffffu, s, o), co = __shfl_down_sync(0xffffffffu, c, o);
        two_sum_add(s, c, so);
        c += co;
    }
    if (lane == 0) G[idx] = s + c;
}

// Y = alpha * U C + beta * Y  (U: n x k, C: k x m2 row-major, Y: n x m2, column stride n), the
// products in double-float arithmetic.  A CTA covers NC output columns (NC a power of two, the
// smallest that holds the product's columns, at most kMulCols), so narrow products do no work on
// padding.  Y may overlap U when the product has a single column block (m2 <= NC, beta = 0):
// each thread reads all k entries of its row before it writes the row.  With `tri` set, C is
// upper triangular (the Cholesky QR transform) and the multiply-adds with its zeros below the
// diagonal are skipped (adding them would leave every sum unchanged).
template <int NC>
__global__ void block_mul_kernel(long long n, int k, int m2, const double *U, const double *__restrict__ C,
                                 double alpha, double beta, double *Y, int tri) {
    extern __shared__ __align__(16) float2 cs[];  // [k][NC] (hi, lo) pairs of C's column block
    const int j0 = blockIdx.y * NC;
    const int nc = min(NC, m2 - j0);
    for (int t = threadIdx.x; t < k * NC; t += blockDim.x) {
        const int i = t / NC, j = t % NC;
        float h, l;
        df_split((j < nc) ? C[i * m2 + j0 + j] : 0.0, h, l);
        cs[t] = make_float2(h, l);
    }
    __syncthreads();
    const long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float S[NC], sl[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) S[j] = sl[j] = 0.0f;
    double un = U[r];  // the next row's operand is loaded before the current row's multiply-adds
    const int kend = tri ? min(k, j0 + NC) : k;  // rows of C below the block's last column are zero
    for (int i = 0; i < kend; ++i) {
        float uh, ul;
        df_split(un, uh, ul);
        if (i + 1 < kend) un = U[static_cast<long long>(i + 1) * n + r];
        if constexpr (NC == 1) {
            if (tri && i > j0) continue;
            const float2 cc = cs[i];
            df_mac(S[0], sl[0], uh, ul, cc.x, cc.y);
        } else {
            const float4 *c4 = reinterpret_cast<const float4 *>(cs + i * NC);  // two (hi, lo) pairs per load
#pragma unroll
            for (int j = 0; j < NC; j += 2) {
                if (tri && i > j0 + j + 1) continue;  // C[i][j0 + j] = C[i][j0 + j + 1] = 0
                const float4 cc = c4[j / 2];
                df_mac(S[j], sl[j], uh, ul, cc.x, cc.y);
                df_mac(S[j + 1], sl[j + 1], uh, ul, cc.z, cc.w);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        if (j < nc) {
            const double acc = df_value(S[j], sl[j]);
            double *y = Y + static_cast<long long>(j0 + j) * n + r;
            *y = (beta == 0.0) ? alpha * acc : fma(alpha, acc, beta * *y);
        }
    }
}

// R = AX - X diag(lambda) for column blockIdx.y over one chunk of `rows` rows, and the chunk's sum of
// squares of that column of R in partial[column * gridDim.x + chunk]: the convergence test needs
// only the residual norms, not the whole Gram matrix R^T R.
constexpr int kNormThreads = 256;
__global__ void __launch_bounds__(kNormThreads) residual_norm_kernel(long long n, long long rows,
                                                                     const double *__restrict__ X,
                                                                     const double *__restrict__ AX,
                                                                     const double *__restrict__ lam,
                                                                     double *__restrict__ R,
                                                                     double *__restrict__ partial) {
    const int j = blockIdx.y;
    const long long r0 = static_cast<long long>(blockIdx.x) * rows, r1 = min(n, r0 + rows);
    const long long off = static_cast<long long>(j) * n;
    const double l = lam[j];
    double acc = 0.0;
    for (long long i = r0 + threadIdx.x; i < r1; i += kNormThreads) {
        const double v = fma(-l, X[off + i], AX[off + i]);
        R[off + i] = v;
        acc = fma(v, v, acc);
    }
    __shared__ double sh[kNormThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = (threadIdx.x < kNormThreads / 32) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partial[static_cast<long long>(j) * gridDim.x + blockIdx.x] = acc;
    }
}

// out[j] = the sum of column j's nch partials (one CTA per column, a fixed summation order)
__global__ void __launch_bounds__(kNormThreads) column_sum_kernel(int nch, const double *__restrict__ partial,
                                                                  double *__restrict__ out) {
    const int j = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nch; i += kNormThreads) acc += partial[static_cast<long long>(j) * nch + i];
    __shared__ double sh[kNormThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = (threadIdx.x < kNormThreads / 32) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) out[j] = acc;
    }
}

int cdiv(long long a, long long b) { return static_cast<int>((a + b - 1) / b); }

// ---- dense FP64 helpers ---------------------------------------------------------------------
// Forward substitution helpers for L (lower, row-major).
void lower_inverse_transpose(int k, const double *L, double *Z) {
    // Z = L^{-T} (upper triangular), column by column: L^T Z = I
    std::fill(Z, Z + static_cast<size_t>(k) * k, 0.0);
    for (int c = 0; c < k; ++c) {
        for (int i = k - 1; i >= 0; --i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int j = i + 1; j < k; ++j) v -= L[j * k + i] * Z[j * k + c];
            Z[i * k + c] = v / L[i * k + i];
        }
    }
}

}  // namespace

bool cholesky(int k, const double *A, double *L) {
    std::fill(L, L + static_cast<size_t>(k) * k, 0.0);
    for (int j = 0; j < k; ++j) {
        double d = A[j * k + j];
        for (int p = 0; p < j; ++p) d -= L[j * k + p] * L[j * k + p];
        if (!(d > 0.0) || !std::isfinite(d)) return false;
        const double ljj = std::sqrt(d);
        L[j * k + j] = ljj;
        for (int i = j + 1; i < k; ++i) {
            double v = A[i * k + j];
            for (int p = 0; p < j; ++p) v -= L[i * k + p] * L[j * k + p];
            L[i * k + j] = v / ljj;
        }
    }
    return true;
}

void jacobi_eigh(int k, const double *Ain, double *w, double *V) {
    std::vector<double> A(Ain, Ain + static_cast<size_t>(k) * k);
    std::fill(V, V + static_cast<size_t>(k) * k, 0.0);
    for (int i = 0; i < k; ++i) V[i * k + i] = 1.0;
    double norm = 0.0;
    for (double v : A) norm += v * v;
    norm = std::sqrt(norm);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) off += A[p * k + q] * A[p * k + q];
        if (std::sqrt(off) <= 1e-17 * norm || off == 0.0) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = A[p * k + q];
                if (apq == 0.0) continue;
                const double app = A[p * k + p], aqq = A[q * k + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {  // A <- A J
                    const double arp = A[r * k + p], arq = A[r * k + q];
                    A[r * k + p] = c * arp - s * arq;
                    A[r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {  // A <- J^T A
                    const double apr = A[p * k + r], aqr = A[q * k + r];
                    A[p * k + r] = c * apr - s * aqr;
                    A[q * k + r] = s * apr + c * aqr;
                }
                A[p * k + q] = A[q * k + p] = 0.0;
                for (int r = 0; r < k; ++r) {  // V <- V J
                    const double vrp = V[r * k + p], vrq = V[r * k + q];
                    V[r * k + p] = c * vrp - s * vrq;
                    V[r * k + q] = s * vrp + c * vrq;
                }
            }
    }
    std::vector<int> idx(k);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[a * k + a] < A[b * k + b]; });
    std::vector<double> Vs(static_cast<size_t>(k) * k);
    for (int c = 0; c < k; ++c) {
        w[c] = A[idx[c] * k + idx[c]];
        for (int r = 0; r < k; ++r) Vs[r * k + c] = V[r * k + idx[c]];
    }
    std::copy(Vs.begin(), Vs.end(), V);
}

// Symmetric eigen-decomposition by Householder reduction to tridiagonal form followed by the
// implicit symmetric QR algorithm with Wilkinson shifts (Golub & Van Loan, sections 8.3.1 and
// 8.3.3): O(k^3) with a small constant, where cyclic Jacobi needs several O(k^3) sweeps.
// A (k x k, row-major, symmetric) -> eigenvalues ascending in w, eigenvectors as columns of V.
// Returns false if the QR iteration did not converge (the caller then uses jacobi_eigh).
bool sym_eigh(int k, const double *Ain, double *w, double *V) {
    const int n = k;
    std::vector<double> A(Ain, Ain + static_cast<size_t>(n) * n), Q(static_cast<size_t>(n) * n, 0.0);
    std::vector<double> v(n), pv(n), wv(n), d(n), e(n, 0.0);
    for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
    // 1. A = Q T Q^T with T tridiagonal: a Householder reflection H = I - beta v v^T per column
    for (int j = 0; j + 2 < n; ++j) {
        const int m = n - j - 1, o = j + 1;  // x = A[o .. n-1][j]
        const double x0 = A[o * n + j];
        double sigma = 0.0;
        for (int i = 1; i < m; ++i) sigma += A[(o + i) * n + j] * A[(o + i) * n + j];
        if (sigma == 0.0) continue;  // already zero below the subdiagonal
        const double mu = std::sqrt(x0 * x0 + sigma);
        const double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
        const double beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) v[i] = A[(o + i) * n + j] / v0;
        // column j (and row j): H x = x - beta v (v . x)
        double vx = 0.0;
        for (int i = 0; i < m; ++i) vx += v[i] * A[(o + i) * n + j];
        const double sub = x0 - beta * vx;
        for (int i = 0; i < m; ++i) A[(o + i) * n + j] = A[j * n + o + i] = 0.0;
        A[o * n + j] = A[j * n + o] = sub;
        // trailing block: A22 <- H A22 H = A22 - v w^T - w v^T, p = beta A22 v, w = p - (beta/2)(p.v) v
        double pvv = 0.0;
        for (int r = 0; r < m; ++r) {
            double acc = 0.0;
            for (int c = 0; c < m; ++c) acc += A[(o + r) * n + o + c] * v[c];
            pv[r] = beta * acc;
            pvv += pv[r] * v[r];
        }
        for (int r = 0; r < m; ++r) wv[r] = pv[r] - 0.5 * beta * pvv * v[r];
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) A[(o + r) * n + o + c] -= v[r] * wv[c] + wv[r] * v[c];
        // Q <- Q H on columns o .. n-1
        for (int r = 0; r < n; ++r) {
            double acc = 0.0;
            for (int c = 0; c < m; ++c) acc += Q[r * n + o + c] * v[c];
            acc *= beta;
            for (int c = 0; c < m; ++c) Q[r * n + o + c] -= acc * v[c];
        }
    }
    for (int i = 0; i < n; ++i) d[i] = A[i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = A[(i + 1) * n + i];
    // 2. implicit symmetric QR steps (Wilkinson shift, bulge chasing with Givens rotations),
    //    rotations accumulated into Q, on the trailing unreduced block until T is diagonal
    const double eps = 2.220446049250313e-16;
    int steps = 0;
    for (;;) {
        for (int i = 0; i + 1 < n; ++i)
            if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
        int q = n - 1;
        while (q > 0 && e[q - 1] == 0.0) --q;
        if (q == 0) break;
        int p = q - 1;
        while (p > 0 && e[p - 1] != 0.0) --p;
        if (++steps > 60 * n) return false;
        const double a = d[q - 1], c2 = d[q], b = e[q - 1];
        const double delta = 0.5 * (a - c2);
        const double sgn = (delta >= 0.0) ? 1.0 : -1.0;
        const double shift = c2 - b * b / (delta + sgn * std::sqrt(delta * delta + b * b));
        double x = d[p] - shift, z = e[p];
        for (int kk = p; kk < q; ++kk) {
            const double r = std::sqrt(x * x + z * z);
            const double c = (r == 0.0) ? 1.0 : x / r, s = (r == 0.0) ? 0.0 : z / r;
            if (kk > p) e[kk - 1] = r;
            const double dk = d[kk], ek = e[kk], dk1 = d[kk + 1];
            d[kk] = c * c * dk + 2.0 * c * s * ek + s * s * dk1;
            d[kk + 1] = s * s * dk - 2.0 * c * s * ek + c * c * dk1;
            e[kk] = c * s * (dk1 - dk) + (c * c - s * s) * ek;
            if (kk + 1 < q) {
                z = s * e[kk + 1];
                e[kk + 1] *= c;
                x = e[kk];
            }
            for (int row = 0; row < n; ++row) {
                const double zk = Q[row * n + kk], zk1 = Q[row * n + kk + 1];
                Q[row * n + kk] = c * zk + s * zk1;
                Q[row * n + kk + 1] = -s * zk + c * zk1;
            }
        }
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int i, int j) { return d[i] < d[j]; });
    for (int c = 0; c < n; ++c) {
        w[c] = d[idx[c]];
        for (int r = 0; r < n; ++r) V[r * n + c] = Q[r * n + idx[c]];
    }
    return true;
}

namespace {

struct Ctx {
    const LobpcgOps &ops;
    LobpcgWork &w;
    cudaStream_t st;
    std::string &msg;
    long long n;
};

#define LCHK(call)                                                                 \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            c.msg = std::string("lobpcg: ") + #call + ": " + cudaGetErrorString(e_); \
            return SMG_ERR_CUDA;                                                   \
        }                                                                          \
    } while (0)

// G (k1 x k2, host row-major) = U^T V; sym: the product is symmetric (k1 = k2 and U^T V = V^T U,
// e.g. V = U or V = A U), so only its upper tiles are computed.  same_u: the previous call had the
// same U, unchanged since (the tensor-core path then reuses U's column maxima).
int gram(Ctx &c, int k1, const double *U, int k2, const double *V, std::vector<double> &G, bool sym = false,
         bool same_u = false) {
    const int nti = cdiv(k1, kGT), ntj = cdiv(k2, kGT);
    if (c.w.gram_tc_min > 0 && k1 >= c.w.gram_tc_min && k2 >= c.w.gram_tc_min && k1 <= 64 && k2 <= 64) {
        // FP64-accurate digit-split products on the tensor cores
        LCHK(gram_tc(c.n, k1, U, c.n, k2, V, c.n, c.w.gram, c.w.tc_work, c.w.num_sms, c.st, same_u));
        G.resize(static_cast<size_t>(k1) * k2);
        LCHK(cudaMemcpyAsync(c.w.h_buf, c.w.gram, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, c.st));
        LCHK(cudaStreamSynchronize(c.st));
        int err = 0;
        LCHK(gram_tc_status(&err));
        if (err != 0) {
            c.msg = "lobpcg: a tensor-core Gram product's wait timed out";
            return SMG_ERR_TIMEOUT;
        }
        std::memcpy(G.data(), c.w.h_buf, sizeof(double) * G.size());
        return SMG_OK;
    }
    if (k1 <= kSmallK && k2 <= kSmallK) {
        // narrow product: 4 CTAs per SM (as far as the partial buffer holds), rows a multiple of 256
        const long long want = std::max<long long>(1, std::min<long long>(4LL * c.w.num_sms, c.w.part_tiles));
        const long long rows = ((c.n + want - 1) / want + 255) / 256 * 256;
        const int nch = static_cast<int>(cdiv(c.n, rows));
        gram_small_kernel<<<nch, 256, 0, c.st>>>(c.n, rows, k1, k2, U, V, c.w.part);
        LCHK(cudaGetLastError());
        gram_reduce_kernel<<<cdiv(static_cast<long long>(k1) * k2 * 32, 256), 256, 0, c.st>>>(
            nch, k1, k2, 1, 1, c.w.part, c.w.gram, 0);
        LCHK(cudaGetLastError());
        G.resize(static_cast<size_t>(k1) * k2);
        LCHK(cudaMemcpyAsync(c.w.h_buf, c.w.gram, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, c.st));
        LCHK(cudaStreamSynchronize(c.st));
        std::memcpy(G.data(), c.w.h_buf, sizeof(double) * G.size());
        return SMG_OK;
    }
    // rows per CTA: kGChunk, halved (down to kGChunk / 8) while the product has fewer than 4 CTAs
    // per SM and the partial buffer has room (single-tile products would otherwise run one CTA
    // per SM, stalled on their global loads)
    const int s = (sym && k1 == k2) ? 1 : 0;
    const int active = s ? nti * (nti + 1) / 2 : nti * ntj;
    long long rows = kGChunk;
    while (rows > kGChunk / 8 && static_cast<long long>(cdiv(c.n, rows)) * active < 4LL * c.w.num_sms &&
           static_cast<long long>(cdiv(c.n, rows / 2)) * nti * ntj <= c.w.part_tiles)
        rows /= 2;
    const int nch = static_cast<int>(cdiv(c.n, rows));
    dim3 grid(nch, nti * ntj);
    gram_partial_kernel<<<grid, kGT * kGT, 0, c.st>>>(c.n, rows, k1, k2, U, V, c.w.part, ntj, s);
    LCHK(cudaGetLastError());
    gram_reduce_kernel<<<cdiv(static_cast<long long>(k1) * k2 * 32, 256), 256, 0, c.st>>>(
        nch, k1, k2, ntj, nti * ntj, c.w.part, c.w.gram, s);
    LCHK(cudaGetLastError());
    G.resize(static_cast<size_t>(k1) * k2);
    LCHK(cudaMemcpyAsync(c.w.h_buf, c.w.gram, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, c.st));
    LCHK(cudaStreamSynchronize(c.st));
    std::memcpy(G.data(), c.w.h_buf, sizeof(double) * G.size());
    return SMG_OK;
}

// Y = alpha U C + beta Y with C (k x m2, host row-major).  Y may overlap U (the product written
// in place) when m2 <= kMulCols and beta = 0 (block_mul_kernel).
int bmul(Ctx &c, int k, const double *U, int m2, const std::vector<double> &C, double alpha, double beta, double *Y,
         bool tri = false) {
    LCHK(cudaMemcpyAsync(c.w.coef, C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice, c.st));
    const int nc = (m2 <= 1) ? 1 : (m2 <= 2) ? 2 : (m2 <= 4) ? 4 : (m2 <= 8) ? 8 : kMulCols;
    dim3 grid(cdiv(c.n, 256), cdiv(m2, nc));
    const size_t smem = sizeof(float2) * k * nc;
    const int t = tri ? 1 : 0;
    switch (nc) {
    case 1: block_mul_kernel<1><<<grid, 256, smem, c.st>>>(c.n, k, m2, U, c.w.coef, alpha, beta, Y, t); break;
    case 2: block_mul_kernel<2><<<grid, 256, smem, c.st>>>(c.n, k, m2, U, c.w.coef, alpha, beta, Y, t); break;
    case 4: block_mul_kernel<4><<<grid, 256, smem, c.st>>>(c.n, k, m2, U, c.w.coef, alpha, beta, Y, t); break;
    case 8: block_mul_kernel<8><<<grid, 256, smem, c.st>>>(c.n, k, m2, U, c.w.coef, alpha, beta, Y, t); break;
    default: block_mul_kernel<kMulCols><<<grid, 256, smem, c.st>>>(c.n, k, m2, U, c.w.coef, alpha, beta, Y, t); break;
    }
    LCHK(cudaGetLastError());
    // the host vector C may be reused right after; the copy above is stream-ordered but reads
    // host memory asynchronously only for pinned memory, so pageable C is safe here
    return SMG_OK;
}

// Orthonormalize the q columns of Y in place (Cholesky QR), applying the same transform to AY
// when given.  Returns false when Y^T Y is numerically singular.
int ortho(Ctx &c, int q, double *Y, double *AY, double *tmp, bool &ok) {
    std::vector<double> G, L(static_cast<size_t>(q) * q), Z(static_cast<size_t>(q) * q);
    int rc = gram(c, q, Y, q, Y, G, true);
    if (rc) return rc;
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < i; ++j) G[i * q + j] = G[j * q + i] = 0.5 * (G[i * q + j] + G[j * q + i]);
    ok = cholesky(q, G.data(), L.data());
    if (!ok) return SMG_OK;
    lower_inverse_transpose(q, L.data(), Z.data());
    if (q <= kMulCols) {  // one column block: in place
        if ((rc = bmul(c, q, Y, q, Z, 1.0, 0.0, Y, true))) return rc;
        if (AY && (rc = bmul(c, q, AY, q, Z, 1.0, 0.0, AY, true))) return rc;
        return SMG_OK;
    }
    const size_t bytes = sizeof(double) * static_cast<size_t>(q) * c.n;
    if ((rc = bmul(c, q, Y, q, Z, 1.0, 0.0, tmp, true))) return rc;
    LCHK(cudaMemcpyAsync(Y, tmp, bytes, cudaMemcpyDeviceToDevice, c.st));
    if (AY) {
        if ((rc = bmul(c, q, AY, q, Z, 1.0, 0.0, tmp, true))) return rc;
        LCHK(cudaMemcpyAsync(AY, tmp, bytes, cudaMemcpyDeviceToDevice, c.st));
    }
    return SMG_OK;
}

// Generalized symmetric eigenproblem GA C = GB C Theta via GB = L L^T.
bool rayleigh_ritz(int k, std::vector<double> GA, const std::vector<double> &GB, std::vector<double> &theta,
                   std::vector<double> &C) {
    std::vector<double> L(static_cast<size_t>(k) * k), Z(static_cast<size_t>(k) * k), H(static_cast<size_t>(k) * k),
        T(static_cast<size_t>(k) * k), V(static_cast<size_t>(k) * k);
    std::vector<double> GBs(GB);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) {
            GA[i * k + j] = GA[j * k + i] = 0.5 * (GA[i * k + j] + GA[j * k + i]);
            GBs[i * k + j] = GBs[j * k + i] = 0.5 * (GBs[i * k + j] + GBs[j * k + i]);
        }
    if (!cholesky(k, GBs.data(), L.data())) return false;
    lower_inverse_transpose(k, L.data(), Z.data());  // Z = L^{-T}
    // H = Z^T GA Z
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double v = 0.0;
            for (int p = 0; p < k; ++p) v += GA[i * k + p] * Z[p * k + j];
            T[i * k + j] = v;
        }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double v = 0.0;
            for (int p = 0; p < k; ++p) v += Z[p * k + i] * T[p * k + j];
            H[i * k + j] = v;
        }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < i; ++j) H[i * k + j] = H[j * k + i] = 0.5 * (H[i * k + j] + H[j * k + i]);
    theta.resize(k);
    if (!sym_eigh(k, H.data(), theta.data(), V.data())) jacobi_eigh(k, H.data(), theta.data(), V.data());
    C.assign(static_cast<size_t>(k) * k, 0.0);
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            double v = 0.0;
            for (int p = 0; p < k; ++p) v += Z[i * k + p] * V[p * k + j];
            C[i * k + j] = v;
        }
    return true;
}

}  // namespace

void lobpcg_free(LobpcgWork &w) {
    cudaFree(w.S);
    cudaFree(w.AS);
    cudaFree(w.T1);
    cudaFree(w.T2);
    cudaFree(w.part);
    cudaFree(w.gram);
    cudaFree(w.coef);
    cudaFree(w.tc_work);
    if (w.h_buf) cudaFreeHost(w.h_buf);
    const int tc_min = w.gram_tc_min;
    w = LobpcgWork();
    w.gram_tc_min = tc_min;
}

int lobpcg_run(const LobpcgOps &ops, LobpcgWork &w, int m, double *Xuser, double *lambda, double tol, int maxit,
               int *iters, cudaStream_t st, std::string &msg) {
    const long long n = ops.n;
    Ctx c{ops, w, st, msg, n};
    if (w.n != n || w.m < m) {
        lobpcg_free(w);
        w.n = n;
        w.m = m;
        const size_t blk = sizeof(double) * static_cast<size_t>(n) * 3 * m;
        LCHK(cudaMalloc(&w.S, blk));
        LCHK(cudaMalloc(&w.AS, blk));
        LCHK(cudaMalloc(&w.T1, blk));
        if (m > kMulCols) LCHK(cudaMalloc(&w.T2, blk));  // P, AP outside S (see below)
        const int k = 3 * m, nt = cdiv(k, kGT);
        w.part_tiles = static_cast<long long>(cdiv(n, kGChunk)) * nt * nt;
        int dev = 0;
        LCHK(cudaGetDevice(&dev));
        LCHK(cudaDeviceGetAttribute(&w.num_sms, cudaDevAttrMultiProcessorCount, dev));
        LCHK(cudaMalloc(&w.part, sizeof(double) * static_cast<size_t>(w.part_tiles) * kGT * kGT));
        LCHK(cudaMalloc(&w.gram, sizeof(double) * k * k));
        LCHK(cudaMalloc(&w.coef, sizeof(double) * k * k));
        LCHK(cudaMallocHost(&w.h_buf, sizeof(double) * k * k));
        LCHK(cudaMalloc(&w.tc_work, gram_tc_workspace_bytes(n)));
    }
    const size_t col = sizeof(double) * static_cast<size_t>(n);
    double *X = w.S, *AX = w.AS;
    // P and AP for all m columns: with m <= kMulCols in S, AS themselves, columns [2m, 3m) (the
    // block products that form them are written in place, and W never reaches column 2m); else in
    // T2 (columns [0, m) and [m, 2m))
    const bool p_in_s = m <= kMulCols;
    double *Pf = p_in_s ? w.S + static_cast<size_t>(n) * 2 * m : w.T2;
    double *APf = p_in_s ? w.AS + static_cast<size_t>(n) * 2 * m : w.T2 + static_cast<size_t>(n) * m;
    int rc;
    LCHK(cudaMemcpyAsync(X, Xuser, col * m, cudaMemcpyDeviceToDevice, st));
    bool ok = false;
    if ((rc = ortho(c, m, X, nullptr, w.T1, ok))) return rc;
    if (!ok) {
        msg = "lobpcg: the initial block is rank deficient";
        return SMG_ERR_BREAKDOWN;
    }
    if ((rc = ops.apply_A(m, X, AX, st))) return rc;
    // Rayleigh-Ritz on X alone
    std::vector<double> GA, GB, theta, C;
    if ((rc = gram(c, m, X, m, AX, GA, true))) return rc;
    if ((rc = gram(c, m, X, m, X, GB, true))) return rc;
    if (!rayleigh_ritz(m, GA, GB, theta, C)) {
        msg = "lobpcg: Rayleigh-Ritz on the initial block failed";
        return SMG_ERR_BREAKDOWN;
    }
    if ((rc = bmul(c, m, X, m, C, 1.0, 0.0, w.T1))) return rc;
    LCHK(cudaMemcpyAsync(X, w.T1, col * m, cudaMemcpyDeviceToDevice, st));
    if ((rc = bmul(c, m, AX, m, C, 1.0, 0.0, w.T1))) return rc;
    LCHK(cudaMemcpyAsync(AX, w.T1, col * m, cudaMemcpyDeviceToDevice, st));
    std::vector<double> lam(theta.begin(), theta.begin() + m);
    bool haveP = false;
    int it = 0, status = SMG_ERR_NOCONV;
    double *d_lam = w.coef;  // reused for lambda right before the residual kernel
    for (it = 0;; ++it) {
        // residuals R = AX - X Lambda into T1[:, 0:m], with their squared norms (the diagonal of
        // R^T R, all the convergence test uses)
        double *R = w.T1;
        LCHK(cudaMemcpyAsync(d_lam, lam.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
        {
            const long long cap = w.part_tiles * kGT * kGT / m;  // partials the Gram buffer holds per column
            const int nch = static_cast<int>(std::max<long long>(1, std::min<long long>(
                std::min<long long>(kNormChunks, cdiv(n, kNormThreads)), cap)));
            const long long rows = (n + nch - 1) / nch;
            residual_norm_kernel<<<dim3(nch, m), kNormThreads, 0, st>>>(n, rows, X, AX, d_lam, R, w.part);
            LCHK(cudaGetLastError());
            column_sum_kernel<<<m, kNormThreads, 0, st>>>(nch, w.part, w.gram);
            LCHK(cudaGetLastError());
        }
        std::vector<double> rn2(m);
        LCHK(cudaMemcpyAsync(w.h_buf, w.gram, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
        LCHK(cudaStreamSynchronize(st));
        std::memcpy(rn2.data(), w.h_buf, sizeof(double) * m);
        std::vector<int> active;
        for (int j = 0; j < m; ++j) {
            const double rn = std::sqrt(std::max(0.0, rn2[j]));
            if (!std::isfinite(rn)) {
                msg = "lobpcg: NaN in a residual";
                return SMG_ERR_NAN;
            }
            if (rn > tol * std::fabs(lam[j])) active.push_back(j);
        }
        if (active.empty()) {
            status = SMG_OK;
            break;
        }
        if (it >= maxit) break;
        const int na = static_cast<int>(active.size());
        double *W = w.S + static_cast<size_t>(n) * m, *AW = w.AS + static_cast<size_t>(n) * m;
        // precondition the active residuals: W = T R_active (gathered first unless all are active)
        if (na == m) {
            if ((rc = ops.apply_T(na, R, W, st))) return rc;
        } else {
            for (int a = 0; a < na; ++a)
                LCHK(cudaMemcpyAsync(AW + static_cast<size_t>(n) * a, R + static_cast<size_t>(n) * active[a], col,
                                     cudaMemcpyDeviceToDevice, st));
            if ((rc = ops.apply_T(na, AW, W, st))) return rc;
        }
        // W -= X (X^T W)
        std::vector<double> XW;
        if ((rc = gram(c, m, X, na, W, XW))) return rc;
        if ((rc = bmul(c, m, X, na, XW, -1.0, 1.0, W))) return rc;
        if ((rc = ortho(c, na, W, nullptr, R, ok))) return rc;
        if (!ok) {
            msg = "lobpcg: the preconditioned residual block is rank deficient";
            return SMG_ERR_BREAKDOWN;
        }
        if ((rc = ops.apply_A(na, W, AW, st))) return rc;
        // P block: active columns of the last direction, orthonormalized
        int np = 0;
        double *Pa = w.S + static_cast<size_t>(n) * (m + na), *APa = w.AS + static_cast<size_t>(n) * (m + na);
        if (haveP) {
            // gather the active columns; in S the target column m + na + a never lies after its
            // source 2m + active[a] and never on a source still to be read, so column copies in
            // increasing a are safe, and with every column active nothing moves
            for (int a = 0; a < na; ++a) {
                const double *ps = Pf + static_cast<size_t>(n) * active[a], *aps = APf + static_cast<size_t>(n) * active[a];
                double *pd = Pa + static_cast<size_t>(n) * a, *apd = APa + static_cast<size_t>(n) * a;
                if (pd != ps) LCHK(cudaMemcpyAsync(pd, ps, col, cudaMemcpyDeviceToDevice, st));
                if (apd != aps) LCHK(cudaMemcpyAsync(apd, aps, col, cudaMemcpyDeviceToDevice, st));
            }
            if ((rc = ortho(c, na, Pa, APa, R, ok))) return rc;
            np = ok ? na : 0;
        }
        // Rayleigh-Ritz on S = [X W P]
        int k = m + na + np;
        if ((rc = gram(c, k, w.S, k, w.AS, GA, true))) return rc;
        if ((rc = gram(c, k, w.S, k, w.S, GB, true, true))) return rc;  // S's column maxima from GA
        if (!rayleigh_ritz(k, GA, GB, theta, C)) {
            if (np == 0) {
                msg = "lobpcg: Gram matrix of [X W] is not positive definite";
                return SMG_ERR_BREAKDOWN;
            }
            // drop P and retry
            np = 0;
            k = m + na;
            std::vector<double> GA2(static_cast<size_t>(k) * k), GB2(static_cast<size_t>(k) * k);
            const int kf = m + 2 * na;
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j) {
                    GA2[i * k + j] = GA[i * kf + j];
                    GB2[i * k + j] = GB[i * kf + j];
                }
            if (!rayleigh_ritz(k, GA2, GB2, theta, C)) {
                msg = "lobpcg: Gram matrix of [X W] is not positive definite";
                return SMG_ERR_BREAKDOWN;
            }
        }
        // C_m = C[:, 0:m]; X = S C_m, AX = AS C_m; P = S_WP C_WP,m, AP = AS_WP C_WP,m
        std::vector<double> Cm(static_cast<size_t>(k) * m), Cwp(static_cast<size_t>(k - m) * m);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < m; ++j) {
                Cm[i * m + j] = C[i * k + j];
                if (i >= m) Cwp[(i - m) * m + j] = C[i * k + j];
            }
        if (p_in_s) {
            // X, AX first, in place: they read every column of S, AS and write the first m; then
            // P, AP, in place into columns [2m, 3m): they read the W and P columns [m, k), which the
            // X update left alone (one column block each, so every thread reads its row first)
            if ((rc = bmul(c, k, w.S, m, Cm, 1.0, 0.0, X))) return rc;
            if ((rc = bmul(c, k, w.AS, m, Cm, 1.0, 0.0, AX))) return rc;
            if ((rc = bmul(c, k - m, W, m, Cwp, 1.0, 0.0, Pf))) return rc;
            if ((rc = bmul(c, k - m, AW, m, Cwp, 1.0, 0.0, APf))) return rc;
        } else {
            // P, AP into T2 first (they read the W and P columns of S, AS), then X, AX through T1
            if ((rc = bmul(c, k - m, W, m, Cwp, 1.0, 0.0, Pf))) return rc;
            if ((rc = bmul(c, k - m, AW, m, Cwp, 1.0, 0.0, APf))) return rc;
            double *Xn = w.T1;
            double *AXn = w.T1 + static_cast<size_t>(n) * m;
            if ((rc = bmul(c, k, w.S, m, Cm, 1.0, 0.0, Xn))) return rc;
            if ((rc = bmul(c, k, w.AS, m, Cm, 1.0, 0.0, AXn))) return rc;
            LCHK(cudaMemcpyAsync(X, Xn, col * m, cudaMemcpyDeviceToDevice, st));
            LCHK(cudaMemcpyAsync(AX, AXn, col * m, cudaMemcpyDeviceToDevice, st));
        }
        haveP = true;
        for (int j = 0; j < m; ++j) lam[j] = theta[j];
    }
    LCHK(cudaMemcpyAsync(Xuser, X, col * m, cudaMemcpyDeviceToDevice, st));
    LCHK(cudaStreamSynchronize(st));
    for (int j = 0; j < m; ++j) lambda[j] = lam[j];
    *iters = it;
    if (status == SMG_ERR_NOCONV) msg = "lobpcg: maximum number of iterations reached";
    return status;
}

}  // namespace smg
