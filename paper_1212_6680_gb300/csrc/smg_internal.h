// smg_internal.h -- internal types of libsmg (not part of the C ABI).
//
// Data layout in HBM
//   grid vectors      : [batch][z][y][x], x fastest; level l has nx*ny*nz_l points per vector.
//   zcoef (double)    : per plane p of the global plane list, 8 values
//                       {M(z,z-1), M(z,z), M(z,z+1), K(z,z-1), K(z,z), K(z,z+1), wm(z), wp(z)}
//                       of the level operator (A_l u)_z = sum_dz M L2D u_{z+dz} + K u_{z+dz}.
//   pcoef (double)    : per plane p, sum_ny lines x 8 values
//                       {S(y,y-1), S(y,y), S(y,y+1), T(y,y-1), T(y,y), T(y,y+1), wm(y), wp(y)}
//                       of the plane's 2D hierarchy (B_m u)_y = sum_dy S Lx u_{y+dy} + T u_{y+dy};
//                       2D level m starts at line line_base[m].
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

namespace smg {

constexpr int kMaxPlaneLevels = 16;
constexpr int kCoefPerLine = 8;
constexpr int kCoefPerPlane = 8;
constexpr int kMaxNx = 512;     // longest x-line one warp can hold (16 rows per lane); lines of
                                // 257-512 rows run on two warps by default (plane_wide.cu)
constexpr int kMaxNxWide = 2048; // x-lines split over up to 4 warps (plane_wide.cu)
constexpr int kMaxNy = 512;    // the plane's coefficient table (8 values per line of every 2D level) sits in shared memory
constexpr int kMaxNz = 4096;

// Host-side SMG hierarchy in FP64 (built once by smg_setup).
struct HostHierarchy {
    int nx = 0, ny = 0, nz = 0;
    int L = 0;                     // number of z-levels (the last has one plane)
    std::vector<int> nz_l;         // [L]
    std::vector<int> plane_base;   // [L] index of plane (l, 0) in the global plane list
    int nplanes_total = 0;
    std::vector<double> zcoef;     // [nplanes_total * 8]
    int P = 0;                     // number of 2D (y) levels (the last has one line)
    std::vector<int> ny_m;         // [P]
    std::vector<int> line_base;    // [P]
    int sum_ny = 0;
    std::vector<double> pcoef;     // [nplanes_total * sum_ny * 8]
};

// Levels of a semicoarsening hierarchy over n points (n, n/2, ... down to 1).
int hierarchy_levels(int n);
void build_hierarchy(int nx, int ny, int nz, HostHierarchy &H);

// Sets the message smg_last_error() returns on the calling thread.
void set_last_error(const std::string &msg);

// Programmatic dependent launch: a kernel launched through launch_pdl may begin while the previous
// kernel of the stream is still running.  Every kernel launched this way executes pdl_wait()
// (griddepcontrol.wait) before it reads or writes anything its predecessors touch, and may call
// pdl_trigger() so that its own successor can start its independent prologue early.  The
// process-wide switch (on by default) exists for measurement.
bool &pdl_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// The dynamic shared-memory limit of a kernel belongs to the kernel (per device), not to a
// handle: it is only ever raised, so that a handle with a smaller layout never lowers it under
// the launches of another handle that is still alive.
inline cudaError_t raise_smem_attr(const void *kernel, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> cur;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int &v = cur[std::make_pair(kernel, dev)];
    const int want = std::max(v, static_cast<int>(smem));
    if (want == v && v > 0) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, want);
    if (e == cudaSuccess) v = want;
    return e;
}

// Arguments of one plane-relaxation launch (one colour of one z-level, all batch entries).
struct PlaneRelaxArgs {
    int nx, ny, nz;          // level grid (ny is the same on every z-level)
    int colour;              // 0: red (even z), 1: black (odd z)
    int mode;                // 0: u = 0 everywhere, 1: own plane 0, 2: correction form
    int iters;               // plane-cycle steps (> 1 only on the coarsest level)
    const void *f;           // level right-hand side (storage type)
    void *u;                 // level iterate (storage type)
    long long vstride;       // elements between batch entries of f and u
    const double *zcoef;     // this level's plane coefficients (8 per plane)
    const double *pcoef;     // this level's plane tables (sum_ny * 8 per plane)
    const float *zcoef32;    // the same two tables rounded to FP32 (for FP32 compute)
    const float *pcoef32;
    void *gws;               // global workspace (compute type), one slot per CTA
    long long ws_per_plane;  // elements per CTA slot
    int P;                   // 2D levels
    int sum_ny;
    int ny_m[kMaxPlaneLevels];
    int line_base[kMaxPlaneLevels];
    int off_u[kMaxPlaneLevels];   // element offset of u_m (in shared memory or in the slot)
    int off_g[kMaxPlaneLevels];   // element offset of g_m
    unsigned smem_u_mask;         // bit m set: u_m lives in shared memory
    unsigned smem_g_mask;
    int R;                        // CTAs per plane (thread-block cluster size; 1 = no cluster)
    int MF;                       // 2D levels whose interior line factors are kept in shared memory
    int off_fs;                   // element offset of those factor sets in shared memory
    int vec;                      // 1: nx == 32 K and f, u, the workspace are 16-byte aligned
                                  // (wide lines: nx % 8 == 0 and the same alignment)
    int W;                        // x-line segments of 512 rows (1 unless nx > 512: plane_wide.cu)
    int lean;                     // 1: the shortened step order (the persistent multi-system
                                  // kernel, whose layout then keeps every factor set on chip; the
                                  // wide-line kernel)
    int solo_from;                // shortened-step cycle on a cluster: 2D levels >= solo_from belong
                                  // whole to CTA 0 (kMaxPlaneLevels: none)
    const void *wftab;            // wide lines: the precomputed line-solver data of this level's
                                  // planes in its compute type (wide_factor_table), or null
    const int *wfslot;            // with wftab: the table slot of each plane of the level (planes
                                  // with equal coefficient tables share one), or null: slot = plane
};

// Placement of the per-plane 2D-cycle arrays: shared memory where they fit, else global.
struct PlaneLayout {
    int K = 0;                    // rows of an x-line per lane (nx <= 32 K)
    size_t smem_bytes = 0;        // dynamic shared memory per CTA
    long long ws_per_plane = 0;   // global elements per CTA slot
    int off_u[kMaxPlaneLevels] = {0};
    int off_g[kMaxPlaneLevels] = {0};
    unsigned smem_u_mask = 0, smem_g_mask = 0;
    int MF = 0;                   // factor sets kept in shared memory (2D levels 0..MF-1)
    int off_fs = 0;
    int solo_from = kMaxPlaneLevels;  // cluster layouts: 2D levels >= solo_from held whole by CTA 0
};

// Elements of one shared-memory factor set of the x-line solver (fields x 32 lanes).
inline int trifac_set_elems(int K) { return (2 + (K > 1 ? 4 * K - 5 : 0) + 13) * 32; }
constexpr int kMaxFactorLevels = kMaxPlaneLevels;

// K > 0 sizes the factor sets for that x-line chunk instead of the one nx implies; all_sets keeps
// the factor sets of every 2D level in shared memory (the shortened-step kernel needs them);
// no_sets keeps none (the wide-line kernel factors its segments on the fly).
PlaneLayout plan_plane_layout(const HostHierarchy &H, size_t elem_bytes, size_t smem_budget, int K = 0,
                              bool all_sets = false, bool no_sets = false);
// Layout for a cluster of R CTAs per plane: each CTA holds the lines it owns (pairs (y/2) mod R)
// of the arrays kept on chip; an array that does not fit lives whole in the cluster's global
// slot.  The arrays of 2D levels >= solo_from are held whole (every line) by CTA 0 instead (the
// same space is reserved on every CTA).  smem_bytes = 0 when the coefficient table and factor
// sets alone exceed the budget.
PlaneLayout plan_plane_layout_cluster(const HostHierarchy &H, size_t elem_bytes, size_t smem_budget, int R,
                                      bool all_sets = false, int solo_from = kMaxPlaneLevels, bool no_sets = false);

// Kernel launchers (cycle.cu and its instantiation units).
enum class Prec { F64 = 0, F32 = 1, BF16 = 2 };
size_t storage_bytes(Prec p);

// Plane relaxation: S = storage type, compute in double (F64 / coarsest) or float.
cudaError_t launch_plane_relax(Prec storage, bool compute_f64, int K, int nplanes, int nb,
                               int threads, const PlaneRelaxArgs &a, size_t smem, cudaStream_t st);
// column: each thread walks several coarse planes and computes each fine residual once (else one
// coarse plane per thread); the results are bit-identical.
cudaError_t launch_restrict(Prec storage, int nx, int ny, int nzf, int nb, const void *f,
                            const void *u, void *fc, const double *zcoef, const float *zcoef32,
                            long long vstride_f, long long vstride_c, cudaStream_t st, bool column = true);
cudaError_t launch_prolong(Prec storage, int nx, int ny, int nzf, int nb, void *u, const void *uc,
                           const double *zcoef, const float *zcoef32, long long vstride_f,
                           long long vstride_c, cudaStream_t st);
// Compares the integer-pipe FP32 <-> FP64 conversions with the hardware ones on n values:
// mism[0] counts narrowing mismatches, mism[1] widening mismatches (device int[2]).
cudaError_t launch_check_conversions(long long n, const double *src, int *mism, cudaStream_t st);
cudaError_t launch_convert_to(Prec storage, long long n, const double *src, void *dst, cudaStream_t st);
cudaError_t launch_convert_from(Prec storage, long long n, const void *src, double *dst, cudaStream_t st);
cudaError_t launch_apply_A(int nx, int ny, int nz, int nb, const double *u, double *out, cudaStream_t st);
int set_plane_relax_smem(Prec storage, bool compute_f64, bool cluster, int K, size_t smem);
// The shortened-step plane cycle (plane_lean.cuh): nx <= 256 (K <= 8), every 2D level's factor
// sets in shared memory, and every line of a 2D level but its last sharing one line matrix
// (lean_uniform_level); FP32 or FP64 compute on one CTA or a cluster of a.R CTAs per plane.
bool lean_supported(int K);
cudaError_t launch_plane_lean(Prec storage, bool compute_f64, int K, int nplanes, int nb, int threads,
                              const PlaneRelaxArgs &a, size_t smem, cudaStream_t st);
int set_plane_lean_smem(Prec storage, bool compute_f64, bool cluster, int K, size_t smem);
bool lean_cluster_resident(Prec storage, bool compute_f64, int K, int R, int threads, size_t smem);
// True when, on every plane of z-level l and every 2D level, the lines before the last share the
// line matrix (S(y,y), T(y,y)) of line 0.
bool lean_uniform_level(const HostHierarchy &H, int l);
// Classes of the planes of z-level l with bit-identical coefficient tables (pcoef): slot[z] is
// the class of plane z (numbered in order of first appearance), rep[c] the first plane of class
// c; returns the number of classes.
int plane_classes(const HostHierarchy &H, int l, std::vector<int> &slot, std::vector<int> &rep);
// Plane relaxation with x-lines split over the warps of a team (plane_wide.cu): segments of
// 32 wk rows, wk = 16 (lines of 513-2048 rows) or 8 (257-512 rows), one warp each.
inline int wide_segments(int wk, int nx) { return wk > 0 ? (nx + 32 * wk - 1) / (32 * wk) : 1; }
// Line-solver data of wide-line planes, formed once instead of at every change of line matrix
// inside the plane cycle: for nplanes consecutive planes of one z-level (pcoef / pcoef32: their
// coefficient tables) and every 2D level m and line set (0: the first line's matrix, 1: the
// last line's), the segment factors, T_s^{-1} e_first, T_s^{-1} e_last and the reduced system's
// inverse rows of every segment, in the compute type (FP64 when f64, else FP32), computed by the
// same code as on the fly (bit-identical).  wide_factor_values(wk, P, W): values per plane.
// The table has nslots entries of that size; slot s holds the data of plane planes[s] (device
// array; null: plane s).
long long wide_factor_values(int wk, int P, int W);
cudaError_t launch_wide_factor_table(int wk, int nx, int W, int P, int sum_ny, const int *ny_m, const int *line_base,
                                     int nslots, const int *planes, const double *pcoef, const float *pcoef32,
                                     bool f64, void *tab, cudaStream_t st);
cudaError_t launch_plane_wide(int wk, Prec storage, bool compute_f64, int nplanes, int nb, int threads,
                              const PlaneRelaxArgs &a, size_t smem, cudaStream_t st);
int set_plane_wide_smem(int wk, Prec storage, bool compute_f64, bool cluster, size_t smem);
// Whether a cluster of R wide-line CTAs with `smem` bytes each fits on the GPU at once.
bool wide_cluster_resident(int wk, Prec storage, bool compute_f64, int R, int threads, size_t smem);
// True when a cluster of R CTAs of the plane kernel (FP64 or FP32 compute) can be resident.
bool cluster_resident(Prec storage, bool compute_f64, int K, int R, int threads, size_t smem);

}  // namespace smg
