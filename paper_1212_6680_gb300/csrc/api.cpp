// api.cpp -- the C ABI of libsmg (include/smg.h): handle lifetime, argument checks, the SMG
// V-cycle launch sequence and the Krylov driver of Algorithm 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/smg.h"
#include "krylov.h"
#include "lobpcg.h"
#include "net.h"
#include "smg_internal.h"

using namespace smg;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

// The grid limits every set-up shares: nullptr when (nx, ny, nz) is accepted, else the reason.
const char *grid_size_error(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1) return "grid sizes must be >= 1";
    if (nx > kMaxNxWide) return "nx must be <= 2048";
    if (ny > kMaxNy) return "ny must be <= 512";
    if (nz > kMaxNz) return "nz must be <= 4096";
    return nullptr;
}

#define SMG_CUDA(call)                                                                               \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(SMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
    } while (0)

// the most dynamic shared memory a plane CTA may use: 227 KB less 1 KB for the kernels' static
// shared memory (the per-level table of the plane cycle, reduction scratch)
constexpr size_t kSmemBudget = 227 * 1024 - 1024;
// the wide-line kernel keeps its exchange buffers and level table in static shared memory
constexpr size_t kWideSmemBudget = kSmemBudget - 2048;

// profiling classes: 0 plane relaxation on the finest level, 1 plane relaxation on the other
// levels (all but the coarsest), 2 the one-plane coarsest solve, 3 restriction + prolongation,
// 4 the Krylov kernels of one iteration, 5 the learned post-correction of one iteration
constexpr int kProfClasses = 6;

struct ProfClass {
    long long launches = 0;
    double ms = 0.0, bytes = 0.0;
};

struct PendingEvent {
    cudaEvent_t a, b;
    int cls;
    double bytes;
};

}  // namespace

void smg::set_last_error(const std::string &msg) { g_last_error = msg; }

struct smg_ctx {
    int nx = 0, ny = 0, nz = 0, npre = 1, npost = 1, coarse_iters = 1, threads = 512;
    Prec prec = Prec::F64;
    HostHierarchy H;
    double *d_zcoef = nullptr, *d_pcoef = nullptr;
    float *d_zcoef32 = nullptr, *d_pcoef32 = nullptr;  // the same tables rounded to FP32
    // level storage (current precision) for nb_alloc right-hand sides
    int nb_alloc = 0;
    Prec alloc_prec = Prec::F64;
    std::vector<void *> d_f, d_u;   // [L]; level 0 entries used only when the caller's buffers are not
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    PlaneLayout lay_c, lay_d;       // compute type = storage compute (float/double) and double (coarsest)
    PlaneLayout lay_cl[5];          // FP64-compute cluster layouts for R = 2, 4, 8, 16 (index log2 R)
    bool cl_ok[5] = {false, false, false, false, false};
    PlaneLayout lay_cl32[5];        // FP32-compute cluster layouts
    bool cl32_ok[5] = {false, false, false, false, false};
    int cluster_max = 16;           // largest cluster for FP64-compute plane relaxations (1 = none)
    int precond = 1;                // krylov_solve's preconditioner: 1 the SMG cycle, 0 none (T = I)
    int lean = 1;                   // 1: the shortened-step plane cycle where it applies
    int solo = 8;                   // shortened-step cluster layouts give the 2D levels of at most
                                    // `solo` lines to CTA 0 (0: none)
    int restrict_column = 1;        // 1: the restriction walks columns of coarse planes where it
                                    // pays (launch_restrict)
    int wide_min = 257;             // lines of at least this many rows run the wide-line kernel
    int wide_factors = 1;           // 1: wide-line planes read their line-solver data from tables
                                    // formed with the level vectors (d_wftab)
    unsigned char *d_wftab = nullptr;  // those tables (each level's in its compute type)
    std::vector<long long> wftab_off;  // [L] byte offset of level l's table in d_wftab, -1: none
    int *d_wfslot = nullptr;           // per level with a table: the slot of each plane (nz_l ints),
                                       // then the plane of each slot (one slot per plane class)
    std::vector<long long> wfslot_off; // [L] int offset of level l's slots in d_wfslot
    std::vector<char> lean_level;   // [L] the level's line matrices allow it (lean_uniform_level)
    PlaneLayout lay_lean64[5];      // FP64-compute shortened-step layouts: one CTA, clusters of 2..16
    bool lean64_ok[5] = {false, false, false, false, false};
    PlaneLayout lay_lean32[5];      // FP32-compute shortened-step layouts (every factor set on chip)
    PlaneLayout lay_wcl[2][5];      // wide-line cluster layouts: [FP64 compute][log2 R]
    bool wcl_ok[2][5] = {{false, false, false, false, false}, {false, false, false, false, false}};
    bool lean32_ok[5] = {false, false, false, false, false};
    int cluster_max32 = 0;          // largest cluster for FP32-compute plane relaxations; 0 = chosen
                                    // per size (see relax)
    int num_sms = 0;
    // Krylov vectors (one right-hand side)
    double *d_r = nullptr, *d_p = nullptr, *d_q = nullptr, *d_dr = nullptr;
    double *d_bh = nullptr, *d_xh = nullptr;  // device copies for host-pointer calls
    KrylovWork kw;
    KrylovScalars *h_sc = nullptr;  // pinned host mirror
    // profiling
    int profile = 0;                // 0 off, 1 level-0 launches, 2 every launch
    long long launches = 0;         // kernel launches issued by this handle
    ProfClass prof[kProfClasses];
    std::vector<PendingEvent> pending;
    std::vector<cudaEvent_t> event_pool;
    // relative recurrence residuals ||r_k|| / ||b|| of the last krylov_solve, k = 0 .. iters
    std::vector<double> hist;
    double *d_hist = nullptr;       // device copy written by the x/r update (hist_cap entries)
    int hist_cap = 0;
    // Device-side solve loop (SMG_OPT_GRAPH): one CUDA graph whose conditional while node repeats
    // V-cycle + Krylov tail until the recurrence residual meets tol, maxit is reached or a
    // breakdown is flagged; rebuilt when anything that changes an iteration's launches changes.
    int use_graph = 1;
    long long gen = 0;              // bumped by every such change
    struct SolveGraph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t exec = nullptr;
        long long gen = -1;
        const double *x = nullptr;  // the iterate the graph's kernels update
        bool ident = false;
        long long body_launches = 0;
    } sg;
    cudaStream_t gs = nullptr;      // capture and launch stream of the graph
    cudaEvent_t gev = nullptr;
    // LOBPCG state
    LobpcgWork lw;
    // learned post-correction (smg_set_learned) and training-pair capture (smg_collect_pairs)
    bool learned = false;
    NetWork nw;
    struct Capture {
        const double *xstar = nullptr;
        float *rho = nullptr, *e = nullptr;
        int max = 0, count = 0;
    } cap;

    long long N() const { return static_cast<long long>(nx) * ny * nz; }
    long long Nl(int l) const { return static_cast<long long>(nx) * ny * H.nz_l[l]; }
};

namespace {

void free_levels(smg_ctx *h) {
    h->gen += 1;
    cudaFree(h->d_wftab);
    h->d_wftab = nullptr;
    h->wftab_off.clear();
    cudaFree(h->d_wfslot);
    h->d_wfslot = nullptr;
    h->wfslot_off.clear();
    for (void *p : h->d_f) cudaFree(p);
    for (void *p : h->d_u) cudaFree(p);
    h->d_f.clear();
    h->d_u.clear();
    cudaFree(h->d_ws);
    h->d_ws = nullptr;
    h->ws_bytes = 0;
    h->nb_alloc = 0;
}

size_t compute_bytes(Prec p) { return p == Prec::F64 ? 8 : 4; }

int instantiated_K(int nx) {
    const int k = (nx + 31) / 32;
    if (k <= 4) return k;
    if (k <= 6) return 6;
    if (k <= 8) return 8;
    return 16;
}

int alloc_plane_workspace(smg_ctx *h, int nb);

// Rows per lane of the wide-line kernel's segments for this handle's lines, 0 when the lines go
// to the one-warp kernels: 16 beyond 512 rows (always), 8 from wide_min (257 by default) to 512.
int wide_rows(const smg_ctx *h) {
    if (h->nx > kMaxNx) return 16;
    return (h->nx > 256 && h->nx >= h->wide_min) ? 8 : 0;
}

// The shortened-step cycle on a cluster: the coarse 2D levels from the first one with at most
// max_lines lines are held whole by CTA 0, provided the layout still keeps on chip every array
// the spread layout `base` keeps; else the next coarser level is tried, and `base` is kept when
// none qualifies (or fewer than two levels would be solo: no barrier would become CTA 0's own).
PlaneLayout with_solo_levels(const HostHierarchy &H, size_t elem_bytes, int R, int max_lines, const PlaneLayout &base) {
    for (int s = 1; s + 2 <= H.P; ++s) {
        if (H.ny_m[s] > max_lines) continue;
        PlaneLayout ly = plan_plane_layout_cluster(H, elem_bytes, kSmemBudget, R, true, s);
        if (ly.smem_bytes == 0 || ly.smem_bytes > kSmemBudget || ly.MF != base.MF) continue;
        if ((ly.smem_u_mask & base.smem_u_mask) != base.smem_u_mask ||
            (ly.smem_g_mask & base.smem_g_mask) != base.smem_g_mask)
            continue;
        return ly;
    }
    return base;
}

// Allocate level vectors for nb right-hand sides in the current precision, and the plane
// workspace; configure the kernels' dynamic shared memory.
int ensure_levels(smg_ctx *h, int nb) {
    if (h->nb_alloc >= nb && h->alloc_prec == h->prec) return SMG_OK;
    free_levels(h);
    const HostHierarchy &H = h->H;
    const size_t sb = storage_bytes(h->prec);
    h->d_f.assign(H.L, nullptr);
    h->d_u.assign(H.L, nullptr);
    for (int l = 0; l < H.L; ++l) {
        const size_t bytes = static_cast<size_t>(h->Nl(l)) * nb * sb;
        SMG_CUDA(cudaMalloc(&h->d_f[l], bytes));
        SMG_CUDA(cudaMalloc(&h->d_u[l], bytes));
    }
    const bool f64c = (h->prec == Prec::F64);
    const int wk = wide_rows(h);
    const bool wide = wk > 0;
    if (wide) {
        // x-lines over several warps (plane_wide.cu): one CTA per plane, segment factors formed on
        // the fly, no cluster and no shortened-step layouts
        h->lay_c = plan_plane_layout(H, compute_bytes(h->prec), kWideSmemBudget, wk, false, true);
        h->lay_d = plan_plane_layout(H, 8, kWideSmemBudget, wk, false, true);
        if (set_plane_wide_smem(wk, h->prec, f64c, false, h->lay_c.smem_bytes) != 0 ||
            set_plane_wide_smem(wk, h->prec, true, false, h->lay_d.smem_bytes) != 0)
            return fail(SMG_ERR_CUDA, "cudaFuncSetAttribute (plane relaxation, wide lines) failed");
        // a plane spread over a cluster of R CTAs, each relaxing the lines it owns
        for (int c64 = 0; c64 < 2; ++c64) {
            for (int lr = 0; lr <= 4; ++lr) h->wcl_ok[c64][lr] = false;
            if (!c64 && f64c) continue;  // an FP64 cycle has no FP32-compute planes
            for (int lr = 1; lr <= 4; ++lr) {
                const int R = 1 << lr;
                PlaneLayout &ly = h->lay_wcl[c64][lr];
                ly = plan_plane_layout_cluster(H, c64 ? 8 : 4, kWideSmemBudget, R, false, kMaxPlaneLevels, true);
                if (ly.smem_bytes == 0 || ly.smem_bytes > kWideSmemBudget) continue;
                if (set_plane_wide_smem(wk, h->prec, c64 != 0, true, ly.smem_bytes) != 0) {
                    cudaGetLastError();
                    continue;
                }
                h->wcl_ok[c64][lr] = wide_cluster_resident(wk, h->prec, c64 != 0, R, h->threads, ly.smem_bytes);
            }
        }
        for (int lr = 0; lr <= 4; ++lr) h->cl_ok[lr] = h->cl32_ok[lr] = h->lean64_ok[lr] = h->lean32_ok[lr] = false;
        if (h->num_sms == 0) {
            int dev = 0;
            SMG_CUDA(cudaGetDevice(&dev));
            SMG_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
        }
        // line-solver tables, each level's in its compute type (FP64 on the coarsest level and in an
        // FP64 cycle, else FP32), one slot per class of planes with bit-identical coefficient
        // tables (the data depend on nothing else): the coarsest level always, the others while
        // all tables take at most 512 MB
        h->wftab_off.assign(H.L, -1);
        h->wfslot_off.assign(H.L, -1);
        if (h->wide_factors) {
            const int W = wide_segments(wk, h->nx);
            const long long per = wide_factor_values(wk, H.P, W);
            std::vector<std::vector<int>> slot(H.L), rep(H.L);
            for (int l = 0; l < H.L; ++l) plane_classes(H, l, slot[l], rep[l]);
            auto bytes_of = [&](int l) -> long long {
                const bool c64 = f64c || l == H.L - 1;
                return per * static_cast<long long>(rep[l].size()) * (c64 ? 8 : 4);
            };
            long long all = 0;
            for (int l = 0; l < H.L; ++l) all += bytes_of(l);
            const bool every = all <= (512ll << 20);
            long long off = 0;
            std::vector<int> ints;
            for (int l = every ? 0 : H.L - 1; l < H.L; ++l) {
                h->wftab_off[l] = off;
                off += (bytes_of(l) + 255) / 256 * 256;
                // slots of the planes, then the plane of each slot; every index checked here
                // bounds a device read (a table slot, a coefficient table)
                const int nc = static_cast<int>(rep[l].size());
                for (int z = 0; z < H.nz_l[l]; ++z)
                    if (slot[l][z] < 0 || slot[l][z] >= nc) return fail(SMG_ERR_HOST, "plane class out of range");
                for (int c = 0; c < nc; ++c)
                    if (rep[l][c] < 0 || rep[l][c] >= H.nz_l[l]) return fail(SMG_ERR_HOST, "plane class out of range");
                h->wfslot_off[l] = static_cast<long long>(ints.size());
                ints.insert(ints.end(), slot[l].begin(), slot[l].end());
                ints.insert(ints.end(), rep[l].begin(), rep[l].end());
            }
            SMG_CUDA(cudaMalloc(&h->d_wftab, static_cast<size_t>(off)));
            SMG_CUDA(cudaMalloc(&h->d_wfslot, sizeof(int) * ints.size()));
            SMG_CUDA(cudaMemcpy(h->d_wfslot, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice));
            for (int l = 0; l < H.L; ++l) {
                if (h->wftab_off[l] < 0) continue;
                const size_t pb = static_cast<size_t>(H.plane_base[l]) * H.sum_ny * kCoefPerLine;
                const int nc = static_cast<int>(rep[l].size());
                SMG_CUDA(launch_wide_factor_table(wk, h->nx, W, H.P, H.sum_ny, H.ny_m.data(), H.line_base.data(), nc,
                                                  h->d_wfslot + h->wfslot_off[l] + H.nz_l[l], h->d_pcoef + pb,
                                                  h->d_pcoef32 + pb, f64c || l == H.L - 1,
                                                  h->d_wftab + h->wftab_off[l], 0));
            }
            SMG_CUDA(cudaStreamSynchronize(0));
        }
        return alloc_plane_workspace(h, nb);
    }
    h->lay_c = plan_plane_layout(H, compute_bytes(h->prec), kSmemBudget);
    h->lay_d = plan_plane_layout(H, 8, kSmemBudget);
    const int K = instantiated_K(h->nx);
    if (set_plane_relax_smem(h->prec, f64c, false, K, h->lay_c.smem_bytes) != 0)
        return fail(SMG_ERR_CUDA, "cudaFuncSetAttribute (plane relaxation, level precision) failed");
    if (set_plane_relax_smem(h->prec, true, false, K, h->lay_d.smem_bytes) != 0)
        return fail(SMG_ERR_CUDA, "cudaFuncSetAttribute (plane relaxation, FP64 coarsest) failed");
    if (h->prec != Prec::F64 && lean_supported(K) &&
        set_plane_lean_smem(h->prec, false, false, K, h->lay_c.smem_bytes) != 0)
        return fail(SMG_ERR_CUDA, "cudaFuncSetAttribute (plane relaxation, shortened-step cycle) failed");
    if (h->num_sms == 0) {
        int dev = 0;
        SMG_CUDA(cudaGetDevice(&dev));
        SMG_CUDA(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // Cluster layouts (FP64 compute, and FP32 compute for the FP32/BF16 cycles): usable when
    // they fit in shared memory and the cluster can be resident; the kernels' shared-memory
    // limit is then set to the largest usable layout.
    for (int pass = 0; pass < 2; ++pass) {
        const bool cf64 = (pass == 0);
        if (!cf64 && h->prec == Prec::F64) break;
        PlaneLayout *lays = cf64 ? h->lay_cl : h->lay_cl32;
        bool *ok = cf64 ? h->cl_ok : h->cl32_ok;
        size_t cl_smem = 0;
        for (int lr = 1; lr <= 4; ++lr) {
            const int R = 1 << lr;
            ok[lr] = false;
            lays[lr] = plan_plane_layout_cluster(H, cf64 ? 8 : 4, kSmemBudget, R);
            if (lays[lr].smem_bytes == 0) continue;
            if (set_plane_relax_smem(h->prec, cf64, true, K, lays[lr].smem_bytes) != 0) {
                cudaGetLastError();
                continue;
            }
            ok[lr] = cluster_resident(h->prec, cf64, K, R, h->threads, lays[lr].smem_bytes);
            if (ok[lr]) cl_smem = std::max(cl_smem, lays[lr].smem_bytes);
        }
        if (cl_smem > 0 && set_plane_relax_smem(h->prec, cf64, true, K, cl_smem) != 0)
            return fail(SMG_ERR_CUDA, "cudaFuncSetAttribute (plane relaxation, cluster) failed");
    }
    // a shortened-step layout is usable when its shared memory can be granted and (cluster) its
    // CTAs fit on the GPU at once; a cluster layout takes its coarse levels solo where it can
    auto settle_lean = [&](bool c64, int lr, PlaneLayout &ly) -> bool {
        const int R = 1 << lr;
        auto usable = [&](const PlaneLayout &l) {
            if (set_plane_lean_smem(h->prec, c64, lr > 0, K, l.smem_bytes) != 0) {
                cudaGetLastError();
                return false;
            }
            return lr == 0 || lean_cluster_resident(h->prec, c64, K, R, h->threads, l.smem_bytes);
        };
        if (lr > 0 && h->solo) {
            const PlaneLayout sl = with_solo_levels(H, c64 ? 8 : 4, R, h->solo, ly);
            if (sl.solo_from < kMaxPlaneLevels && usable(sl)) {
                ly = sl;
                return true;
            }
        }
        return usable(ly);
    };
    // FP64-compute shortened-step layouts (every 2D level's factor sets on chip), one CTA or a
    // cluster per plane
    for (int lr = 0; lr <= 4; ++lr) {
        h->lean64_ok[lr] = false;
        if (!lean_supported(K)) break;
        const int R = 1 << lr;
        PlaneLayout &ly = h->lay_lean64[lr];
        ly = (lr == 0) ? plan_plane_layout(H, 8, kSmemBudget, 0, true) : plan_plane_layout_cluster(H, 8, kSmemBudget, R, true);
        if (ly.smem_bytes == 0 || ly.smem_bytes > kSmemBudget || ly.MF != H.P) continue;
        h->lean64_ok[lr] = settle_lean(true, lr, ly);
    }
    // the same for FP32 compute (FP32 and BF16 cycles): used where the general layout does not keep
    // every factor set on chip (one CTA) or the plane is spread over a cluster
    for (int lr = 0; lr <= 4; ++lr) {
        h->lean32_ok[lr] = false;
        if (!lean_supported(K) || h->prec == Prec::F64) break;
        const int R = 1 << lr;
        PlaneLayout &ly = h->lay_lean32[lr];
        ly = (lr == 0) ? plan_plane_layout(H, 4, kSmemBudget, 0, true) : plan_plane_layout_cluster(H, 4, kSmemBudget, R, true);
        if (ly.smem_bytes == 0 || ly.smem_bytes > kSmemBudget || ly.MF != H.P) continue;
        h->lean32_ok[lr] = settle_lean(false, lr, ly);
    }
    // a single-CTA lean layout can need more shared memory than the general one
    {
        size_t m32 = h->lay_c.smem_bytes;
        if (h->lean32_ok[0]) m32 = std::max(m32, h->lay_lean32[0].smem_bytes);
        if (h->prec != Prec::F64 && lean_supported(K) && set_plane_lean_smem(h->prec, false, false, K, m32) != 0)
            return fail(SMG_ERR_CUDA, "cudaFuncSetAttribute (plane relaxation, shortened-step cycle) failed");
    }
    return alloc_plane_workspace(h, nb);
}

// Global slots for the 2D-cycle arrays that are not on chip: one per CTA (at most one per plane
// of a colour of the finest level) or one per cluster, sized for the largest usable layout.
int alloc_plane_workspace(smg_ctx *h, int nb) {
    const HostHierarchy &H = h->H;
    size_t per = std::max(static_cast<size_t>(h->lay_c.ws_per_plane) * compute_bytes(h->prec),
                          static_cast<size_t>(h->lay_d.ws_per_plane) * 8);
    for (int lr = 1; lr <= 4; ++lr) {
        if (h->cl_ok[lr]) per = std::max(per, static_cast<size_t>(h->lay_cl[lr].ws_per_plane) * 8);
        if (h->cl32_ok[lr]) per = std::max(per, static_cast<size_t>(h->lay_cl32[lr].ws_per_plane) * 4);
    }
    for (int lr = 0; lr <= 4; ++lr) {
        if (h->lean64_ok[lr]) per = std::max(per, static_cast<size_t>(h->lay_lean64[lr].ws_per_plane) * 8);
        if (h->lean32_ok[lr]) per = std::max(per, static_cast<size_t>(h->lay_lean32[lr].ws_per_plane) * 4);
        if (h->wcl_ok[1][lr]) per = std::max(per, static_cast<size_t>(h->lay_wcl[1][lr].ws_per_plane) * 8);
        if (h->wcl_ok[0][lr]) per = std::max(per, static_cast<size_t>(h->lay_wcl[0][lr].ws_per_plane) * 4);
    }
    const long long slots = static_cast<long long>((H.nz + 1) / 2) * nb;
    h->ws_bytes = std::max<size_t>(per * slots, 256);
    SMG_CUDA(cudaMalloc(&h->d_ws, h->ws_bytes));
    h->nb_alloc = nb;
    h->alloc_prec = h->prec;
    return SMG_OK;
}

cudaEvent_t take_event(smg_ctx *h) {
    if (h->event_pool.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
}

// Event pair around a non-relaxation region (profile mode 2; the learned correction also in mode 1).
struct RegionTimer {
    smg_ctx *h;
    cudaStream_t st;
    int cls;
    double bytes;
    cudaEvent_t e0 = nullptr;
    RegionTimer(smg_ctx *h_, cudaStream_t st_, int cls_, double bytes_) : h(h_), st(st_), cls(cls_), bytes(bytes_) {
        // the learned correction (class 5) is also timed in profile mode 1, beside level 0
        if (h->profile == 2 || (h->profile == 1 && cls == 5)) {
            e0 = take_event(h);
            cudaEventRecord(e0, st);
        }
    }
    ~RegionTimer() {
        if (e0) {
            cudaEvent_t e1 = take_event(h);
            cudaEventRecord(e1, st);
            h->pending.push_back(PendingEvent{e0, e1, cls, bytes});
        }
    }
};

// One plane-relaxation launch: colour c of level l, all nb right-hand sides.
int relax(smg_ctx *h, int l, int colour, int mode, int iters, bool coarsest, const void *f, void *u, int nb,
          cudaStream_t st) {
    const HostHierarchy &H = h->H;
    const int nzl = H.nz_l[l];
    const int nplanes = colour == 0 ? (nzl + 1) / 2 : nzl / 2;
    if (nplanes == 0) return SMG_OK;
    const bool f64c = coarsest || h->prec == Prec::F64;
    // Each plane is spread over a cluster of R CTAs while the grid still fits on the SMs at once.
    // Defaults (measured on GB300 at 128^3 and 256^3): FP64 planes up to 16 CTAs for the one-plane
    // coarsest level and up to 8 elsewhere (beyond 8 the cluster barrier costs more than the
    // FP64 work it spreads); FP32 planes stay on one CTA while its 2D-cycle iterate u_0 fits in
    // shared memory (the cycle is then latency-bound and a cluster only adds barrier cost), and
    // use up to 4 CTAs when it does not (256-wide planes).  Planes with x-lines longer than 512
    // rows (plane_wide.cu) hold several lines per team of warps and are spread the same way, FP32
    // ones over up to 8 CTAs (the paper's 16n x n x n bricks: 1280 x 80 x 80 FPCG 116 -> 57 ms).
    int R = 1;
    const int wk = wide_rows(h);
    const int W = wide_segments(wk, h->nx);
    const bool *ok = (W > 1) ? h->wcl_ok[f64c ? 1 : 0] : (f64c ? h->cl_ok : h->cl32_ok);
    int rmax;
    if (f64c) rmax = coarsest ? h->cluster_max : std::min(h->cluster_max, 8);
    else if (h->cluster_max32 > 0) rmax = h->cluster_max32;
    else if (W > 1) rmax = 8;
    else rmax = (h->lay_c.smem_u_mask & 1u) ? 1 : 4;
    for (int cand = 2; cand <= rmax && cand <= 16; cand *= 2)
        if (ok[__builtin_ctz(cand)] && static_cast<long long>(nplanes) * nb * cand <= h->num_sms) R = cand;
    const PlaneLayout &lay =
        (R > 1) ? (W > 1 ? h->lay_wcl[f64c ? 1 : 0][__builtin_ctz(R)]
                         : (f64c ? h->lay_cl[__builtin_ctz(R)] : h->lay_cl32[__builtin_ctz(R)]))
                : ((f64c && h->prec != Prec::F64) ? h->lay_d : h->lay_c);
    PlaneRelaxArgs a;
    std::memset(&a, 0, sizeof(a));
    a.solo_from = kMaxPlaneLevels;
    a.lean = (W > 1 && h->lean) ? 1 : 0;  // wide lines: the shortened step order
    // the level's table was formed in its compute type: FP64 exactly when f64c (the coarsest level
    // or an FP64 cycle)
    if (W > 1 && h->d_wftab != nullptr && l < static_cast<int>(h->wftab_off.size()) && h->wftab_off[l] >= 0) {
        a.wftab = h->d_wftab + h->wftab_off[l];
        a.wfslot = h->d_wfslot + h->wfslot_off[l];
    }
    a.nx = h->nx;
    a.ny = h->ny;
    a.nz = nzl;
    a.colour = colour;
    a.mode = mode;
    a.iters = iters;
    a.f = f;
    a.u = u;
    a.vstride = h->Nl(l);
    a.zcoef = h->d_zcoef + static_cast<size_t>(H.plane_base[l]) * kCoefPerPlane;
    a.zcoef32 = h->d_zcoef32 + static_cast<size_t>(H.plane_base[l]) * kCoefPerPlane;
    a.pcoef32 = h->d_pcoef32 + static_cast<size_t>(H.plane_base[l]) * H.sum_ny * kCoefPerLine;
    a.pcoef = h->d_pcoef + static_cast<size_t>(H.plane_base[l]) * H.sum_ny * kCoefPerLine;
    a.gws = h->d_ws;
    a.ws_per_plane = lay.ws_per_plane;
    a.P = H.P;
    a.sum_ny = H.sum_ny;
    for (int m = 0; m < H.P; ++m) {
        a.ny_m[m] = H.ny_m[m];
        a.line_base[m] = H.line_base[m];
        a.off_u[m] = lay.off_u[m];
        a.off_g[m] = lay.off_g[m];
    }
    a.smem_u_mask = lay.smem_u_mask;
    a.smem_g_mask = lay.smem_g_mask;
    a.R = R;
    a.MF = lay.MF;
    a.off_fs = lay.off_fs;
    const int K = instantiated_K(h->nx);
    a.W = W;
    {
        auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
        const bool shape = (W > 1) ? (h->nx % 8 == 0) : (h->nx == 32 * K);
        a.vec = shape && al16(f) && al16(u) && al16(h->d_ws);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = (h->profile == 2) || (h->profile == 1 && l == 0);
    const int cls = coarsest ? 2 : (l == 0 ? 0 : 1);
    if (timed) {
        e0 = take_event(h);
        e1 = take_event(h);
        cudaEventRecord(e0, st);
    }
    // the shortened-step cycle: FP32 compute on one CTA per plane with the same layout; FP64
    // compute with its own layouts, the cluster chosen by the same rule as above
    bool use_lean = false;
    const PlaneLayout *llay = &lay;
    if (W == 1 && h->lean && lean_supported(K) && h->lean_level[l]) {
        if (!f64c) {
            if (iters == 1 && R == 1 && lay.MF == H.P) {
                use_lean = true;  // the general layout already keeps every factor set on chip
            } else if (iters == 1 && h->lean32_ok[__builtin_ctz(R)]) {
                use_lean = true;
                llay = &h->lay_lean32[__builtin_ctz(R)];
            }
        } else {
            int lrb = -1;
            for (int lr = 0; lr <= 4; ++lr) {
                const int cand = 1 << lr;
                if (cand > rmax && lr > 0) break;
                if (h->lean64_ok[lr] && (lr == 0 || static_cast<long long>(nplanes) * nb * cand <= h->num_sms)) lrb = lr;
            }
            if (lrb >= 0) {
                use_lean = true;
                llay = &h->lay_lean64[lrb];
                a.R = 1 << lrb;
            }
        }
    }
    if (use_lean && llay != &lay) {
        a.ws_per_plane = llay->ws_per_plane;
        for (int m = 0; m < H.P; ++m) {
            a.off_u[m] = llay->off_u[m];
            a.off_g[m] = llay->off_g[m];
        }
        a.smem_u_mask = llay->smem_u_mask;
        a.smem_g_mask = llay->smem_g_mask;
        a.MF = llay->MF;
        a.off_fs = llay->off_fs;
        a.solo_from = llay->solo_from;
    }
    cudaError_t err = (W > 1)  ? launch_plane_wide(wk, h->prec, f64c, nplanes, nb, h->threads, a, lay.smem_bytes, st)
                      : use_lean ? launch_plane_lean(h->prec, f64c, K, nplanes, nb, h->threads, a, llay->smem_bytes, st)
                                 : launch_plane_relax(h->prec, f64c, K, nplanes, nb, h->threads, a, lay.smem_bytes, st);
    if (err != cudaSuccess) return fail(SMG_ERR_CUDA, std::string("plane relaxation launch: ") + cudaGetErrorString(err));
    h->launches += 1;
    if (timed) {
        cudaEventRecord(e1, st);
        // algorithmic traffic: read f_z, write u_z (+ read u_z in correction form) for every
        // relaxed plane, and read each opposite-colour plane once when it can be nonzero
        const double np = static_cast<double>(h->nx) * h->ny;
        const int nother = nzl - nplanes;
        double planes = nplanes * (2.0 + (mode == 2 ? 1.0 : 0.0)) + (mode >= 1 ? nother : 0);
        planes *= iters;
        const double bytes = planes * np * nb * static_cast<double>(storage_bytes(h->prec));
        h->pending.push_back(PendingEvent{e0, e1, cls, bytes});
    }
    return SMG_OK;
}

// u0 = T f0 for nb right-hand sides; f0, u0 in storage precision, level-0 layout.
int run_cycle(smg_ctx *h, int nb, const void *f0, void *u0, cudaStream_t st) {
    const HostHierarchy &H = h->H;
    const int L = H.L;
    int rc;
    auto F = [&](int l) -> const void * { return l == 0 ? f0 : h->d_f[l]; };
    auto U = [&](int l) -> void * { return l == 0 ? u0 : h->d_u[l]; };
    for (int l = 0; l + 1 < L; ++l) {
        for (int s = 0; s < h->npre; ++s) {
            if ((rc = relax(h, l, 0, s == 0 ? 0 : 2, 1, false, F(l), U(l), nb, st)) != SMG_OK) return rc;
            if ((rc = relax(h, l, 1, s == 0 ? 1 : 2, 1, false, F(l), U(l), nb, st)) != SMG_OK) return rc;
        }
        RegionTimer rt(h, st, 3, 2.5 * h->Nl(l) * nb * storage_bytes(h->prec));
        cudaError_t e = launch_restrict(h->prec, h->nx, h->ny, H.nz_l[l], nb, F(l), U(l), h->d_f[l + 1],
                                        h->d_zcoef + static_cast<size_t>(H.plane_base[l]) * kCoefPerPlane,
                                        h->d_zcoef32 + static_cast<size_t>(H.plane_base[l]) * kCoefPerPlane,
                                        h->Nl(l), h->Nl(l + 1), st, h->restrict_column != 0);
        if (e != cudaSuccess) return fail(SMG_ERR_CUDA, std::string("restriction launch: ") + cudaGetErrorString(e));
        h->launches += 1;
    }
    if ((rc = relax(h, L - 1, 0, 0, h->coarse_iters, true, F(L - 1), U(L - 1), nb, st)) != SMG_OK) return rc;
    for (int l = L - 2; l >= 0; --l) {
        RegionTimer rt(h, st, 3, 2.5 * h->Nl(l) * nb * storage_bytes(h->prec));
        cudaError_t e = launch_prolong(h->prec, h->nx, h->ny, H.nz_l[l], nb, U(l), U(l + 1),
                                       h->d_zcoef + static_cast<size_t>(H.plane_base[l]) * kCoefPerPlane,
                                       h->d_zcoef32 + static_cast<size_t>(H.plane_base[l]) * kCoefPerPlane,
                                       h->Nl(l), h->Nl(l + 1), st);
        if (e != cudaSuccess) return fail(SMG_ERR_CUDA, std::string("prolongation launch: ") + cudaGetErrorString(e));
        h->launches += 1;
        for (int s = 0; s < h->npost; ++s) {
            if ((rc = relax(h, l, 1, 2, 1, false, F(l), U(l), nb, st)) != SMG_OK) return rc;
            if ((rc = relax(h, l, 0, 2, 1, false, F(l), U(l), nb, st)) != SMG_OK) return rc;
        }
    }
    return SMG_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_handle(smg_handle h) {
    if (h == nullptr) return fail(SMG_ERR_ARG, "null handle");
    return SMG_OK;
}

int ensure_krylov(smg_ctx *h) {
    if (h->d_r) return SMG_OK;
    const size_t b = static_cast<size_t>(h->N()) * sizeof(double);
    SMG_CUDA(cudaMalloc(&h->d_r, b));
    SMG_CUDA(cudaMalloc(&h->d_p, b));
    SMG_CUDA(cudaMalloc(&h->d_q, b));
    SMG_CUDA(cudaMalloc(&h->d_dr, b));
    SMG_CUDA(cudaMalloc(&h->kw.sc, sizeof(KrylovScalars)));
    SMG_CUDA(cudaMalloc(&h->kw.part, sizeof(double) * 2 * 2 * kMaxReduceBlocks));
    SMG_CUDA(cudaMalloc(&h->kw.counter, sizeof(unsigned)));
    SMG_CUDA(cudaMemset(h->kw.counter, 0, sizeof(unsigned)));
    SMG_CUDA(cudaMalloc(&h->kw.bar, 4 * sizeof(unsigned)));
    SMG_CUDA(cudaMemset(h->kw.bar, 0, 4 * sizeof(unsigned)));
    SMG_CUDA(cudaMemset(h->kw.sc, 0, sizeof(KrylovScalars)));
    SMG_CUDA(cudaMallocHost(&h->h_sc, sizeof(KrylovScalars)));
    return SMG_OK;
}

int read_scalars(smg_ctx *h, cudaStream_t st) {
    SMG_CUDA(cudaMemcpyAsync(h->h_sc, h->kw.sc, sizeof(KrylovScalars), cudaMemcpyDeviceToHost, st));
    SMG_CUDA(cudaStreamSynchronize(st));
    return SMG_OK;
}

void drop_solve_graph(smg_ctx *h) {
    if (h->sg.exec) cudaGraphExecDestroy(h->sg.exec);
    if (h->sg.g) cudaGraphDestroy(h->sg.g);
    h->sg = smg_ctx::SolveGraph();
}

// Build (or keep) the graph of the device-side solve loop: a conditional while node whose body is
// one iteration -- the V-cycle s = T r (unless T = I) and the four Krylov kernels -- captured from
// the same launch code as the host loop.  Returns false when the graph cannot be built (the host
// loop is used then).
bool ensure_solve_graph(smg_ctx *h, void *f0, void *u0, Prec kp, void *f0k, bool ident, double *x) {
    if (h->sg.exec && h->sg.gen == h->gen && h->sg.x == x && h->sg.ident == ident) return true;
    drop_solve_graph(h);
    if (h->gs == nullptr && cudaStreamCreateWithFlags(&h->gs, cudaStreamNonBlocking) != cudaSuccess) return false;
    if (h->gev == nullptr && cudaEventCreateWithFlags(&h->gev, cudaEventDisableTiming) != cudaSuccess) return false;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return false;
    cudaGraphConditionalHandle cond;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t node;
    bool ok = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
    }
    const long long l0 = h->launches;
    if (ok) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        ok = cudaStreamBeginCaptureToGraph(h->gs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            bool launched = ident || run_cycle(h, 1, f0, u0, h->gs) == SMG_OK;
            launched = launched && kry_iteration_tail(kp, h->nx, h->ny, h->nz, u0, x, h->d_r, h->d_p, h->d_q, h->d_dr,
                                                      f0k, h->kw, h->gs, cond, 1) == cudaSuccess;
            h->launches += 4;
            cudaGraph_t out = nullptr;
            ok = (cudaStreamEndCapture(h->gs, &out) == cudaSuccess) && launched;
        }
    }
    h->sg.body_launches = h->launches - l0;
    h->launches = l0;
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaGraphDestroy(g);
        h->use_graph = 0;  // this handle falls back to the host loop for good
        return false;
    }
    h->sg.g = g;
    h->sg.exec = exec;
    h->sg.gen = h->gen;
    h->sg.x = x;
    h->sg.ident = ident;
    return true;
}

int krylov_device(smg_ctx *h, int variant, const double *b, double *x, double tol, int maxit, int *iters,
                  double *relres, cudaStream_t st) {
    int rc;
    if ((rc = ensure_levels(h, 1)) != SMG_OK) return rc;
    if ((rc = ensure_krylov(h)) != SMG_OK) return rc;
    if (h->hist_cap < maxit + 2) {
        cudaFree(h->d_hist);
        h->d_hist = nullptr;
        h->hist_cap = 0;
        SMG_CUDA(cudaMalloc(&h->d_hist, sizeof(double) * (maxit + 2)));
        h->hist_cap = maxit + 2;
    }
    const bool f64 = (h->prec == Prec::F64);
    const bool ident = (h->precond == 0);                           // T = I: s is r itself
    void *f0 = f64 ? static_cast<void *>(h->d_r) : h->d_f[0];     // cycle input  = (S) r
    void *u0 = ident ? static_cast<void *>(h->d_r) : h->d_u[0];   // s = T r
    const Prec kp = ident ? Prec::F64 : h->prec;                    // storage type of s
    void *f0k = (f64 || ident) ? nullptr : f0;                      // what the Krylov kernels write
    const double tol2 = tol * tol;
    // the device-side loop: not with the learned correction, training-pair capture or per-launch
    // profiling (their host-side steps and events sit between the kernels of an iteration)
    const bool graph = h->use_graph && !h->learned && h->cap.count >= h->cap.max && h->profile == 0 &&
                       ensure_solve_graph(h, f0, u0, kp, f0k, ident, x);
    cudaStream_t ls = st;  // the stream the solve runs on
    if (graph) {
        SMG_CUDA(cudaEventRecord(h->gev, st));
        SMG_CUDA(cudaStreamWaitEvent(h->gs, h->gev, 0));
        ls = h->gs;
    }
    KrylovScalars init;
    std::memset(&init, 0, sizeof(init));
    init.variant = variant;
    init.maxit = maxit;
    init.tol2 = tol2;
    init.hist = h->d_hist;
    SMG_CUDA(cudaMemcpyAsync(h->kw.sc, &init, sizeof(init), cudaMemcpyHostToDevice, ls));
    // reduction counter and grid-barrier words start clean (a wait that gave up leaves them set)
    SMG_CUDA(cudaMemsetAsync(h->kw.counter, 0, sizeof(unsigned), ls));
    SMG_CUDA(cudaMemsetAsync(h->kw.bar, 0, 4 * sizeof(unsigned), ls));
    SMG_CUDA(kry_init_residual(kp, h->nx, h->ny, h->nz, b, x, h->d_r, f0k, h->kw, ls));
    h->launches += 1;
    int k = 0, status = SMG_ERR_NOCONV;
    double tt = -1.0;
    if ((rc = read_scalars(h, ls)) != SMG_OK) return rc;
    h->hist.assign(1, std::sqrt(h->h_sc->rr / (h->h_sc->bb > 0.0 ? h->h_sc->bb : 1.0)));
    for (;;) {
        const KrylovScalars &s = *h->h_sc;
        if (s.status != 0) {
            status = s.status;
            break;
        }
        const double bb = s.bb > 0.0 ? s.bb : 1.0;
        if (s.rr <= tol2 * bb) {
            SMG_CUDA(kry_true_residual(h->nx, h->ny, h->nz, b, x, h->kw, ls));
            h->launches += 1;
            if ((rc = read_scalars(h, ls)) != SMG_OK) return rc;
            tt = h->h_sc->tt;
            if (tt <= tol2 * bb) {
                status = SMG_OK;
                break;
            }
            // continue from the true residual, with beta = 0 on the next step
            SMG_CUDA(kry_init_residual(kp, h->nx, h->ny, h->nz, b, x, h->d_r, f0k, h->kw, ls));
            h->launches += 1;
            tt = -1.0;
        }
        if (k >= maxit) {
            status = SMG_ERR_NOCONV;
            break;
        }
        if (graph) {
            // iterations until the recurrence residual meets tol, maxit or a breakdown
            SMG_CUDA(cudaGraphLaunch(h->sg.exec, ls));
            if ((rc = read_scalars(h, ls)) != SMG_OK) return rc;
            h->launches += h->sg.body_launches * (h->h_sc->it - k);
            k = h->h_sc->it;
            continue;
        }
        if (!ident && (rc = run_cycle(h, 1, f0, u0, ls)) != SMG_OK) return rc;
        if (!ident && h->cap.count < h->cap.max) {
            // training pair of this iteration: rho = r - A s, e = x* - x - s
            const size_t off = static_cast<size_t>(h->cap.count) * h->N();
            SMG_CUDA(net_capture(h->prec, h->nx, h->ny, h->nz, h->d_r, u0, x, h->cap.xstar, h->cap.rho + off,
                                 h->cap.e + off, ls));
            h->cap.count += 1;
            h->launches += 1;
        }
        if (!ident && h->learned) {
            // flops of the three convolutions (2 x 27 x (16 + 256 + 16) per point)
            RegionTimer rt(h, ls, 5, 2.0 * 27 * (16 + 256 + 16) * static_cast<double>(h->N()));
            const long long l0 = h->nw.launches;
            SMG_CUDA(net_learned_correct(h->nw, h->prec, h->nx, h->ny, h->nz, h->d_r, u0, ls));
            h->launches += h->nw.launches - l0;
        }
        {
            RegionTimer rt(h, ls, 4, 0.0);
            SMG_CUDA(kry_iteration_tail(kp, h->nx, h->ny, h->nz, u0, x, h->d_r, h->d_p, h->d_q, h->d_dr, f0k, h->kw, ls));
        }
        h->launches += 4;
        k += 1;
        if ((rc = read_scalars(h, ls)) != SMG_OK) return rc;
    }
    if (tt < 0.0) {
        SMG_CUDA(kry_true_residual(h->nx, h->ny, h->nz, b, x, h->kw, ls));
        h->launches += 1;
        if ((rc = read_scalars(h, ls)) != SMG_OK) return rc;
        tt = h->h_sc->tt;
    }
    // the recurrence residuals of iterations 1 .. k, written on the device
    h->hist.resize(static_cast<size_t>(k) + 1);
    if (k > 0) {
        SMG_CUDA(cudaMemcpyAsync(h->hist.data() + 1, h->d_hist + 1, sizeof(double) * k, cudaMemcpyDeviceToHost, ls));
        SMG_CUDA(cudaStreamSynchronize(ls));
    }
    if (graph) {
        SMG_CUDA(cudaEventRecord(h->gev, ls));
        SMG_CUDA(cudaStreamWaitEvent(st, h->gev, 0));
    }
    const double bb = h->h_sc->bb > 0.0 ? h->h_sc->bb : 1.0;
    *iters = k;
    *relres = std::sqrt(tt / bb);
    if (status == SMG_ERR_NOCONV) return fail(SMG_ERR_NOCONV, "maximum number of iterations reached");
    if (status == SMG_ERR_BREAKDOWN) return fail(status, "breakdown: (p, Ap) <= 0 or (s_{k-1}, r_{k-1}) = 0");
    if (status == SMG_ERR_NAN) return fail(status, "NaN or Inf in a residual norm or inner product");
    if (status == SMG_ERR_TIMEOUT) return fail(status, "a grid-barrier wait of the Krylov kernel gave up");
    return status;
}

}  // namespace

// ================================================================================================
// C ABI
// ================================================================================================
extern "C" {

const char *smg_last_error(void) { return g_last_error.c_str(); }

int smg_setup(int nx, int ny, int nz, int npre, int npost, smg_handle *out) {
    if (out == nullptr) return fail(SMG_ERR_ARG, "out is null");
    *out = nullptr;
    if (const char *e = grid_size_error(nx, ny, nz)) return fail(SMG_ERR_ARG, e);
    if (npre < 1) return fail(SMG_ERR_ARG, "npre must be >= 1");
    if (npost < 0) return fail(SMG_ERR_ARG, "npost must be >= 0");
    smg_ctx *h = new smg_ctx();
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->npre = npre;
    h->npost = npost;
    build_hierarchy(nx, ny, nz, h->H);
    h->lean_level.assign(h->H.L, 0);
    for (int l = 0; l < h->H.L; ++l) h->lean_level[l] = lean_uniform_level(h->H, l) ? 1 : 0;
    const size_t zb = h->H.zcoef.size() * sizeof(double), pb = h->H.pcoef.size() * sizeof(double);
    cudaError_t e = cudaMalloc(&h->d_zcoef, zb);
    if (e == cudaSuccess) e = cudaMalloc(&h->d_pcoef, pb);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_zcoef, h->H.zcoef.data(), zb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->d_pcoef, h->H.pcoef.data(), pb, cudaMemcpyHostToDevice);
    {
        std::vector<float> z32(h->H.zcoef.begin(), h->H.zcoef.end()), p32(h->H.pcoef.begin(), h->H.pcoef.end());
        if (e == cudaSuccess) e = cudaMalloc(&h->d_zcoef32, z32.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&h->d_pcoef32, p32.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMemcpy(h->d_zcoef32, z32.data(), z32.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_pcoef32, p32.data(), p32.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        smg_destroy(h);
        return fail(SMG_ERR_CUDA, std::string("smg_setup: ") + cudaGetErrorString(e));
    }
    int rc = ensure_levels(h, 1);
    if (rc != SMG_OK) {
        smg_destroy(h);
        return rc;
    }
    *out = h;
    return SMG_OK;
}

int smg_set_precision(smg_handle h, int prec) {
    if (int rc = check_handle(h)) return rc;
    if (prec != SMG_FP64 && prec != SMG_FP32 && prec != SMG_BF16) return fail(SMG_ERR_ARG, "unknown precision");
    h->prec = static_cast<Prec>(prec);
    h->gen += 1;
    return SMG_OK;
}

int smg_set_option(smg_handle h, int option, int value) {
    if (int rc = check_handle(h)) return rc;
    h->gen += 1;
    switch (option) {
    case SMG_OPT_GRAPH:
        if (value != 0 && value != 1) return fail(SMG_ERR_ARG, "graph must be 0 or 1");
        h->use_graph = value;
        return SMG_OK;
    case SMG_OPT_FUSED_TAIL:
        if (value != 0 && value != 1) return fail(SMG_ERR_ARG, "fused_tail must be 0 or 1");
        h->kw.fused = value != 0;
        return SMG_OK;
    case SMG_OPT_COARSE_ITERS:
        if (value < 1 || value > 64) return fail(SMG_ERR_ARG, "coarse_iters must be in [1, 64]");
        h->coarse_iters = value;
        return SMG_OK;
    case SMG_OPT_THREADS:
        if (value != 256 && value != 512) return fail(SMG_ERR_ARG, "threads must be 256 or 512");
        if (value != h->threads) free_levels(h);  // the layouts and residency checks depend on it
        h->threads = value;
        return SMG_OK;
    case SMG_OPT_WIDE_MIN_ROWS:
        if (value != 257 && value != 513) return fail(SMG_ERR_ARG, "wide_min_rows must be 257 or 513");
        if (value != h->wide_min) free_levels(h);
        h->wide_min = value;
        return SMG_OK;
    case SMG_OPT_WIDE_FACTORS:
        if (value != 0 && value != 1) return fail(SMG_ERR_ARG, "wide_factors must be 0 or 1");
        if (value != h->wide_factors) free_levels(h);
        h->wide_factors = value;
        return SMG_OK;
    case SMG_OPT_RESTRICT_COLUMN:
        if (value != 0 && value != 1) return fail(SMG_ERR_ARG, "restrict_column must be 0 or 1");
        h->restrict_column = value;
        return SMG_OK;
    case SMG_OPT_SOLO:
        if (value < 0 || value > kMaxNy) return fail(SMG_ERR_ARG, "solo must be in [0, 512]");
        if (value != h->solo) free_levels(h);
        h->solo = value;
        return SMG_OK;
    case SMG_OPT_CLUSTER_MAX:
        if (value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
            return fail(SMG_ERR_ARG, "cluster_max must be 1, 2, 4, 8 or 16");
        h->cluster_max = value;
        return SMG_OK;
    case SMG_OPT_PRECOND:
        if (value != 0 && value != 1) return fail(SMG_ERR_ARG, "precond must be 0 (none) or 1 (SMG)");
        h->precond = value;
        return SMG_OK;
    case SMG_OPT_CLUSTER_MAX32:
        if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
            return fail(SMG_ERR_ARG, "cluster_max32 must be 0 (automatic), 1, 2, 4, 8 or 16");
        h->cluster_max32 = value;
        return SMG_OK;
    case SMG_OPT_GRAM_TC:
        if (value < 0 || value > 64) return fail(SMG_ERR_ARG, "gram_tc must be in [0, 64]");
        h->lw.gram_tc_min = value;
        return SMG_OK;
    case SMG_OPT_LEAN:
        if (value != 0 && value != 1) return fail(SMG_ERR_ARG, "lean must be 0 or 1");
        h->lean = value;
        return SMG_OK;
    case SMG_OPT_PROFILE:
        if (value < 0 || value > 2) return fail(SMG_ERR_ARG, "profile must be 0, 1 or 2");
        h->profile = value;
        return SMG_OK;
    }
    return fail(SMG_ERR_ARG, "unknown option");
}

int smg_apply_batched(smg_handle h, int nb, const double *R, double *S, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (nb < 1 || nb > 64) return fail(SMG_ERR_ARG, "nb must be in [1, 64]");
    if (R == nullptr || S == nullptr) return fail(SMG_ERR_ARG, "null vector");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc;
    if ((rc = ensure_levels(h, nb)) != SMG_OK) return rc;
    const long long n = h->N() * nb;
    if (h->prec == Prec::F64) {
        if ((rc = run_cycle(h, nb, R, S, st)) != SMG_OK) return rc;
    } else {
        SMG_CUDA(launch_convert_to(h->prec, n, R, h->d_f[0], st));
        if ((rc = run_cycle(h, nb, h->d_f[0], h->d_u[0], st)) != SMG_OK) return rc;
        SMG_CUDA(launch_convert_from(h->prec, n, h->d_u[0], S, st));
        h->launches += 2;
    }
    if (h->learned) {
        const long long l0 = h->nw.launches;
        for (int b = 0; b < nb; ++b)
            SMG_CUDA(net_learned_correct(h->nw, Prec::F64, h->nx, h->ny, h->nz, R + b * h->N(), S + b * h->N(), st));
        h->launches += h->nw.launches - l0;
    }
    return SMG_OK;
}

int smg_apply(smg_handle h, const double *r, double *s, void *stream) {
    return smg_apply_batched(h, 1, r, s, stream);
}

int smg_apply_A(smg_handle h, const double *u, double *out, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (u == nullptr || out == nullptr) return fail(SMG_ERR_ARG, "null vector");
    SMG_CUDA(launch_apply_A(h->nx, h->ny, h->nz, 1, u, out, static_cast<cudaStream_t>(stream)));
    return SMG_OK;
}

int krylov_solve(smg_handle h, int variant, const double *b, double *x, double tol, int maxit, int *iters,
                 double *relres, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    if (variant != SMG_PCG && variant != SMG_FPCG && variant != SMG_PSD) return fail(SMG_ERR_ARG, "unknown variant");
    if (b == nullptr || x == nullptr || iters == nullptr || relres == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(SMG_ERR_ARG, "tol must be > 0");
    if (maxit < 0) return fail(SMG_ERR_ARG, "maxit must be >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool bdev = is_device_ptr(b), xdev = is_device_ptr(x);
    if (bdev && xdev) return krylov_device(h, variant, b, x, tol, maxit, iters, relres, st);
    // host buffers: copy in, solve, copy out
    const size_t bytes = static_cast<size_t>(h->N()) * sizeof(double);
    if (h->d_bh == nullptr) {
        SMG_CUDA(cudaMalloc(&h->d_bh, bytes));
        SMG_CUDA(cudaMalloc(&h->d_xh, bytes));
    }
    const double *bd = b;
    double *xd = x;
    if (!bdev) {
        SMG_CUDA(cudaMemcpyAsync(h->d_bh, b, bytes, cudaMemcpyHostToDevice, st));
        bd = h->d_bh;
    }
    if (!xdev) {
        SMG_CUDA(cudaMemcpyAsync(h->d_xh, x, bytes, cudaMemcpyHostToDevice, st));
        xd = h->d_xh;
    }
    int rc = krylov_device(h, variant, bd, xd, tol, maxit, iters, relres, st);
    if (rc != SMG_OK && rc != SMG_ERR_NOCONV) return rc;
    if (!xdev) {
        SMG_CUDA(cudaMemcpyAsync(x, h->d_xh, bytes, cudaMemcpyDeviceToHost, st));
        SMG_CUDA(cudaStreamSynchronize(st));
    }
    return rc;
}

int lobpcg_solve(smg_handle h, int m, double *X, double *lambda, double tol, int maxit, int *iters, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (iters) *iters = 0;
    if (X == nullptr || lambda == nullptr || iters == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    if (m < 1 || m > 64 || 3LL * m > h->N()) return fail(SMG_ERR_ARG, "m must satisfy 1 <= m <= 64 and 3m <= N");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(SMG_ERR_ARG, "tol must be > 0");
    if (maxit < 0) return fail(SMG_ERR_ARG, "maxit must be >= 0");
    int rc;
    if ((rc = ensure_levels(h, m)) != SMG_OK) return rc;
    LobpcgOps ops;
    ops.n = h->N();
    ops.apply_A = [h](int nb, const double *u, double *out, cudaStream_t st) -> int {
        cudaError_t e = launch_apply_A(h->nx, h->ny, h->nz, nb, u, out, st);
        return e == cudaSuccess ? SMG_OK : fail(SMG_ERR_CUDA, std::string("apply_A: ") + cudaGetErrorString(e));
    };
    ops.apply_T = [h](int nb, const double *r, double *s, cudaStream_t st) -> int {
        return smg_apply_batched(h, nb, r, s, st);
    };
    std::string msg;
    rc = lobpcg_run(ops, h->lw, m, X, lambda, tol, maxit, iters, static_cast<cudaStream_t>(stream), msg);
    if (rc != SMG_OK) return fail(rc, msg);
    return SMG_OK;
}

int smg_profile_read(smg_handle h, int which, long long *launches, double *ms, double *bytes) {
    if (int rc = check_handle(h)) return rc;
    if (which < 0 || which >= kProfClasses || !launches || !ms || !bytes) return fail(SMG_ERR_ARG, "bad arguments");
    SMG_CUDA(cudaDeviceSynchronize());
    for (auto &p : h->pending) {
        float t = 0.0f;
        cudaEventElapsedTime(&t, p.a, p.b);
        h->prof[p.cls].launches += 1;
        h->prof[p.cls].ms += t;
        h->prof[p.cls].bytes += p.bytes;
        h->event_pool.push_back(p.a);
        h->event_pool.push_back(p.b);
    }
    h->pending.clear();
    *launches = h->prof[which].launches;
    *ms = h->prof[which].ms;
    *bytes = h->prof[which].bytes;
    h->prof[which] = ProfClass();
    return SMG_OK;
}

int smg_check_conversions(long long n, const double *src, int *mismatches, void *stream) {
    if (n < 0 || (n > 0 && (src == nullptr || mismatches == nullptr))) return fail(SMG_ERR_ARG, "bad arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    SMG_CUDA(cudaMemsetAsync(mismatches, 0, 2 * sizeof(int), st));
    SMG_CUDA(launch_check_conversions(n, src, mismatches, st));
    return SMG_OK;
}

int smg_set_learned(smg_handle h, const void *weights_bf16, int enable) {
    if (int rc = check_handle(h)) return rc;
    if (enable != 0 && enable != 1) return fail(SMG_ERR_ARG, "enable must be 0 or 1");
    h->gen += 1;
    if (!enable) {
        h->learned = false;
        return SMG_OK;
    }
    if (weights_bf16 == nullptr) return fail(SMG_ERR_ARG, "null weights");
    // BF16 bit patterns widen exactly to FP32 (the upper half of the FP32 word)
    const unsigned short *wb = static_cast<const unsigned short *>(weights_bf16);
    std::vector<float> w(kNetWeights);
    for (int i = 0; i < kNetWeights; ++i) {
        const uint32_t bits = static_cast<uint32_t>(wb[i]) << 16;
        std::memcpy(&w[i], &bits, sizeof(float));
        if (!std::isfinite(w[i])) return fail(SMG_ERR_ARG, "weights must be finite");
    }
    SMG_CUDA(net_alloc(h->nw, h->N(), 0, false));
    SMG_CUDA(cudaMemcpy(h->nw.w, w.data(), kNetWeights * sizeof(float), cudaMemcpyHostToDevice));
    SMG_CUDA(cudaMemset(h->nw.sc, 0, sizeof(NetScal)));
    h->learned = true;
    return SMG_OK;
}

int smg_learned_stats(smg_handle h, long long *calls, long long *accepted) {
    if (int rc = check_handle(h)) return rc;
    if (calls == nullptr || accepted == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    *calls = *accepted = 0;
    if (h->nw.sc == nullptr) return SMG_OK;
    NetScal sc;
    SMG_CUDA(cudaMemcpy(&sc, h->nw.sc, sizeof(sc), cudaMemcpyDeviceToHost));
    *calls = sc.calls;
    *accepted = sc.accepts;
    return SMG_OK;
}

int smg_collect_pairs(smg_handle h, const double *b, const double *xstar, double tol, int maxit, float *rho_out,
                      float *e_out, int max_pairs, int *npairs, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (npairs) *npairs = 0;
    if (!b || !xstar || !rho_out || !e_out || !npairs) return fail(SMG_ERR_ARG, "null pointer");
    if (max_pairs < 1 || maxit < 0 || !(tol > 0.0)) return fail(SMG_ERR_ARG, "max_pairs >= 1, maxit >= 0, tol > 0");
    if (!is_device_ptr(b) || !is_device_ptr(xstar) || !is_device_ptr(rho_out) || !is_device_ptr(e_out))
        return fail(SMG_ERR_ARG, "b, xstar, rho_out, e_out must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double *x = nullptr;
    SMG_CUDA(cudaMalloc(&x, static_cast<size_t>(h->N()) * sizeof(double)));
    cudaMemsetAsync(x, 0, static_cast<size_t>(h->N()) * sizeof(double), st);
    h->cap.xstar = xstar;
    h->cap.rho = rho_out;
    h->cap.e = e_out;
    h->cap.max = max_pairs;
    h->cap.count = 0;
    int iters = 0;
    double relres = 0.0;
    const int rc = krylov_device(h, SMG_FPCG, b, x, tol, maxit, &iters, &relres, st);
    *npairs = h->cap.count;
    h->cap = smg_ctx::Capture();
    cudaStreamSynchronize(st);
    cudaFree(x);
    return (rc == SMG_ERR_NOCONV) ? SMG_OK : rc;
}

int smg_krylov_history(smg_handle h, double *hist, int max, int *count) {
    if (int rc = check_handle(h)) return rc;
    if (count == nullptr || max < 0 || (max > 0 && hist == nullptr)) return fail(SMG_ERR_ARG, "bad arguments");
    *count = static_cast<int>(h->hist.size());
    for (int k = 0; k < max && k < *count; ++k) hist[k] = h->hist[k];
    return SMG_OK;
}

int smg_launch_count(smg_handle h, long long *count) {
    if (int rc = check_handle(h)) return rc;
    if (count == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    *count = h->launches;
    return SMG_OK;
}

int smg_setup_coefs(int nx, int ny, int nz, int l, int z, int m, double *zc, double *lines, int *nz_l, int *ny_m) {
    using namespace smg;
    if (const char *e = grid_size_error(nx, ny, nz)) return fail(SMG_ERR_ARG, e);
    if (zc == nullptr || lines == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    if (l < 0 || l >= hierarchy_levels(nz) || m < 0 || m >= hierarchy_levels(ny))
        return fail(SMG_ERR_ARG, "level or 2D level out of range");
    HostHierarchy H;
    try {
        build_hierarchy(nx, ny, nz, H);
    } catch (const std::exception &ex) {
        return fail(SMG_ERR_HOST, std::string("building the hierarchy failed: ") + ex.what());
    }
    if (z < 0 || z >= H.nz_l[l]) return fail(SMG_ERR_ARG, "plane out of range");
    const size_t plane = static_cast<size_t>(H.plane_base[l] + z);
    for (int k = 0; k < kCoefPerPlane; ++k) zc[k] = H.zcoef[plane * kCoefPerPlane + k];
    const double *pc = &H.pcoef[plane * H.sum_ny * kCoefPerLine];
    for (int y = 0; y < H.ny_m[m]; ++y)
        for (int k = 0; k < kCoefPerLine; ++k)
            lines[static_cast<size_t>(y) * kCoefPerLine + k] = pc[static_cast<size_t>(H.line_base[m] + y) * kCoefPerLine + k];
    if (nz_l) *nz_l = H.nz_l[l];
    if (ny_m) *ny_m = H.ny_m[m];
    return SMG_OK;
}

int smg_plane_classes(int nx, int ny, int nz, int l, int *cls) {
    using namespace smg;
    if (const char *e = grid_size_error(nx, ny, nz)) return fail(SMG_ERR_ARG, e);
    if (cls == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    if (l < 0 || l >= hierarchy_levels(nz)) return fail(SMG_ERR_ARG, "level out of range");
    HostHierarchy H;
    std::vector<int> slot, rep;
    try {
        build_hierarchy(nx, ny, nz, H);
        plane_classes(H, l, slot, rep);
    } catch (const std::exception &ex) {
        return fail(SMG_ERR_HOST, std::string("building the hierarchy failed: ") + ex.what());
    }
    for (int z = 0; z < H.nz_l[l]; ++z) cls[z] = slot[z];
    return static_cast<int>(rep.size());
}

int smg_plane_layout(int nx, int ny, int elem_bytes, int R, long long *out) {
    using namespace smg;
    if (out == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    if (nx < 1 || ny < 1 || nx > kMaxNx || ny > kMaxNy) return fail(SMG_ERR_ARG, "nx, ny must be in 1..512");
    if (elem_bytes != 4 && elem_bytes != 8) return fail(SMG_ERR_ARG, "elem_bytes must be 4 or 8");
    if (R != 1 && R != 2 && R != 4 && R != 8 && R != 16) return fail(SMG_ERR_ARG, "R must be 1, 2, 4, 8 or 16");
    HostHierarchy H;
    build_hierarchy(nx, ny, 1, H);
    const PlaneLayout P = (R == 1) ? plan_plane_layout(H, static_cast<size_t>(elem_bytes), kSmemBudget)
                                   : plan_plane_layout_cluster(H, static_cast<size_t>(elem_bytes), kSmemBudget, R);
    for (int i = 0; i < 64; ++i) out[i] = 0;
    out[0] = H.P;
    out[1] = P.K;
    out[2] = P.MF;
    out[3] = static_cast<long long>(P.smem_bytes);
    out[4] = P.ws_per_plane;
    out[5] = P.off_fs;
    out[6] = P.smem_u_mask;
    out[7] = P.smem_g_mask;
    out[8] = H.sum_ny;
    out[9] = kCoefPerLine;
    out[10] = trifac_set_elems(P.K);
    for (int m = 0; m < H.P && m < 16; ++m) {
        out[16 + m] = P.off_u[m];
        out[32 + m] = P.off_g[m];
        out[48 + m] = H.ny_m[m];
    }
    return SMG_OK;
}

int smg_plane_layout_kind(int nx, int ny, int elem_bytes, int R, int kind, int solo, long long *out) {
    using namespace smg;
    if (out == nullptr) return fail(SMG_ERR_ARG, "null pointer");
    if (kind < 0 || kind > 2) return fail(SMG_ERR_ARG, "kind must be 0, 1 or 2");
    const int nx_lo = (kind == 2) ? 257 : 1;
    const int nx_hi = (kind == 2) ? kMaxNxWide : (kind == 1 ? 256 : kMaxNx);
    if (nx < nx_lo || nx > nx_hi || ny < 1 || ny > kMaxNy)
        return fail(SMG_ERR_ARG, "nx outside the kind's range or ny outside 1..512");
    if (elem_bytes != 4 && elem_bytes != 8) return fail(SMG_ERR_ARG, "elem_bytes must be 4 or 8");
    if (R != 1 && R != 2 && R != 4 && R != 8 && R != 16) return fail(SMG_ERR_ARG, "R must be 1, 2, 4, 8 or 16");
    if (solo < 0 || solo > kMaxNy) return fail(SMG_ERR_ARG, "solo must be in [0, 512]");
    HostHierarchy H;
    build_hierarchy(nx, ny, 1, H);
    const size_t eb = static_cast<size_t>(elem_bytes);
    PlaneLayout P;
    if (kind == 0) {
        P = (R == 1) ? plan_plane_layout(H, eb, kSmemBudget) : plan_plane_layout_cluster(H, eb, kSmemBudget, R);
    } else if (kind == 1) {
        P = (R == 1) ? plan_plane_layout(H, eb, kSmemBudget, 0, true) : plan_plane_layout_cluster(H, eb, kSmemBudget, R, true);
        if (R > 1 && solo > 0 && P.smem_bytes > 0) P = with_solo_levels(H, eb, R, solo, P);
    } else {
        const int wk = nx > kMaxNx ? 16 : 8;
        P = (R == 1) ? plan_plane_layout(H, eb, kWideSmemBudget, wk, false, true)
                     : plan_plane_layout_cluster(H, eb, kWideSmemBudget, R, false, kMaxPlaneLevels, true);
        P.K = wk;
    }
    for (int i = 0; i < 64; ++i) out[i] = 0;
    out[0] = H.P;
    out[1] = P.K;
    out[2] = P.MF;
    out[3] = static_cast<long long>(P.smem_bytes);
    out[4] = P.ws_per_plane;
    out[5] = P.off_fs;
    out[6] = P.smem_u_mask;
    out[7] = P.smem_g_mask;
    out[8] = H.sum_ny;
    out[9] = kCoefPerLine;
    out[10] = trifac_set_elems(P.K);
    out[11] = std::min(P.solo_from, H.P);
    for (int m = 0; m < H.P && m < 16; ++m) {
        out[16 + m] = P.off_u[m];
        out[32 + m] = P.off_g[m];
        out[48 + m] = H.ny_m[m];
    }
    return SMG_OK;
}

int smg_destroy(smg_handle h) {
    if (h == nullptr) return SMG_OK;
    free_levels(h);
    cudaFree(h->d_zcoef);
    cudaFree(h->d_pcoef);
    cudaFree(h->d_zcoef32);
    cudaFree(h->d_pcoef32);
    cudaFree(h->d_r);
    cudaFree(h->d_p);
    cudaFree(h->d_q);
    cudaFree(h->d_dr);
    cudaFree(h->d_bh);
    cudaFree(h->d_xh);
    cudaFree(h->kw.sc);
    cudaFree(h->kw.part);
    cudaFree(h->kw.counter);
    cudaFree(h->kw.bar);
    if (h->h_sc) cudaFreeHost(h->h_sc);
    for (auto &p : h->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    lobpcg_free(h->lw);
    net_free(h->nw);
    drop_solve_graph(h);
    if (h->gs) cudaStreamDestroy(h->gs);
    if (h->gev) cudaEventDestroy(h->gev);
    cudaFree(h->d_hist);
    delete h;
    return SMG_OK;
}

}  // extern "C"
