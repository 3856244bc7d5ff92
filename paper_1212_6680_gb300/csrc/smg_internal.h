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

#include <cstdint>
#include <string>
#include <vector>

namespace smg {

constexpr int kMaxPlaneLevels = 16;
constexpr int kCoefPerLine = 8;
constexpr int kCoefPerPlane = 8;
constexpr int kMaxNx = 512;
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

void build_hierarchy(int nx, int ny, int nz, HostHierarchy &H);

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
};

// Placement of the per-plane 2D-cycle arrays: shared memory where they fit, else global.
struct PlaneLayout {
    int K = 0;                    // rows of an x-line per lane (nx <= 32 K)
    size_t smem_bytes = 0;        // dynamic shared memory per CTA
    long long ws_per_plane = 0;   // global elements per CTA slot
    int off_u[kMaxPlaneLevels] = {0};
    int off_g[kMaxPlaneLevels] = {0};
    unsigned smem_u_mask = 0, smem_g_mask = 0;
};

PlaneLayout plan_plane_layout(const HostHierarchy &H, size_t elem_bytes, size_t smem_budget);

// Kernel launchers (cycle.cu and its instantiation units).
enum class Prec { F64 = 0, F32 = 1, BF16 = 2 };
size_t storage_bytes(Prec p);

// Plane relaxation: S = storage type, compute in double (F64 / coarsest) or float.
cudaError_t launch_plane_relax(Prec storage, bool compute_f64, int K, int nplanes, int nb,
                               int threads, const PlaneRelaxArgs &a, size_t smem, cudaStream_t st);
cudaError_t launch_restrict(Prec storage, int nx, int ny, int nzf, int nb, const void *f,
                            const void *u, void *fc, const double *zcoef, long long vstride_f,
                            long long vstride_c, cudaStream_t st);
cudaError_t launch_prolong(Prec storage, int nx, int ny, int nzf, int nb, void *u, const void *uc,
                           const double *zcoef, long long vstride_f, long long vstride_c,
                           cudaStream_t st);
cudaError_t launch_convert_to(Prec storage, long long n, const double *src, void *dst, cudaStream_t st);
cudaError_t launch_convert_from(Prec storage, long long n, const void *src, double *dst, cudaStream_t st);
cudaError_t launch_apply_A(int nx, int ny, int nz, int nb, const double *u, double *out, cudaStream_t st);
int set_plane_relax_smem(Prec storage, bool compute_f64, int K, int threads, size_t smem);

}  // namespace smg
