// pond_internal.cuh -- shared definitions of the PonD CUDA library (sm_103a).
//
// Lattices: D2Q16, the tensor product of the four roots of He4
// (c^2 = 3 -+ sqrt 6), weights (3 -+ sqrt 6)/12, T_L = 1 (App. A generalised
// to a fourth-order Hermite set), and the paper's own D2Q9 (App. A: c = -1,
// 0, 1, W = 1/6, 2/3, 1/6, T_L = 1/3).  n1 speeds per dimension,
// populations q = n1 k + l, Q = n1^2.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cmath>

#include <string>
#include <vector>

#include "../../include/pond.h"

namespace pond {

// NVTX range over a host-side phase (a step, an adjoint phase, a halo
// copy): header-only NVTX v3, a no-op unless a profiler is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Keep the caller's current device across a call.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else if (prev == dev) prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// Lattice constants, computed on the host from their closed forms and passed
// to kernels by value (they land in the constant bank).
//
// The 1D gauge transform is G[k][a] = L_k(xi_a) where L_k is the Lagrange
// basis polynomial on the speeds c_j (M^-1 M of Eq. transform for a tensor
// lattice) and xi_a = (sqrt(theta_s) c_a + u_s - u') / sqrt(theta').
// Written around the identity, xi_a = c_a + delta_a, it is
//   L_k(c_a + delta) = [k == a] + d1[k][a] delta + d2[k][a] delta^2 + d3[k] delta^3
// with d1 = L_k'(c_a), d2 = L_k''(c_a)/2, d3 = L_k'''/6 (exact: L_k has
// degree n1 - 1, so d3 = 0 for D2Q9).  Arrays are sized for n1 = 4; D2Q9
// uses their leading 3 entries.
//
// pe0, pe2, pt0, pt2, inv_TL: dual basis of {1, c_x, c_y, |c|^2} under the
// weights W, onto which the mixed form's conservative collision projects
// the relaxed non-equilibrium part.  With the W-Gram matrix
// [[1, 2 T_L], [2 T_L, 2 K4 + 2 T_L^2]] of {1, |c|^2} (K4 = sum_a w_a c_a^4)
// and <c_x, c_x> = T_L, the duals are W (pe0 + pe2 |c|^2), W c_x / T_L,
// W c_y / T_L and W (pt0 + pt2 |c|^2).
struct Lattice {
    double c[4];
    double w[4];
    double d1[4][4];
    double d2[4][4];
    double d3[4];
    double T_L;
    double c_max;
    double pe0, pe2, pt0, pt2, inv_TL;
    int32_t n1;
    int32_t q;
};

struct LatticeF {
    float c[4];
    float w[4];
    float d1[4][4];
    float d2[4][4];
    float d3[4];
    float pe0, pe2, pt0, pt2, inv_TL;
};

// kind: POND_D2Q16 or POND_D2Q9
Lattice make_lattice(int kind = POND_D2Q16);
LatticeF to_float(const Lattice& L);
// constant-bank slot of a lattice in every translation unit
constexpr int lattice_slot(int n1) { return n1 == 4 ? 0 : 1; }

struct StepParams {
    double beta;
    double dt;
    double eps_abs;
    double eps_rel;
    double T_L;
    int32_t max_iter;
    int32_t fixed_iter;
    int32_t thermal;
    int32_t seed_mode;
};

// Device-side counters (one per context, zeroed per pond_step call).
struct DevStats {
    unsigned long long passes;
    unsigned long long nonconverged;
    unsigned long long nonphysical;
    unsigned long long halo_fallback;
    unsigned long long index_faults;  // debug builds: accesses skipped by a failed index check
    unsigned int max_passes;
    unsigned int pad;
    // persistent (batched) launches of the staged kernel: summed CTA busy
    // time, and resident CTAs x launch span, in globaltimer nanoseconds
    unsigned long long busy_ns;
    unsigned long long slot_ns;
    // per-launch scratch of those launches, folded into busy_ns / slot_ns
    // and zeroed by the launch's last CTA
    unsigned long long l_begin_inv;  // max of ~(CTA start time) = ~(earliest start)
    unsigned long long l_end;        // latest CTA exit
    unsigned long long l_busy;       // summed CTA busy time
    unsigned int l_done;             // CTAs exited
    unsigned int pad2;
};

// Per-grid descriptor of a batched context (node offset into packed arrays).
struct GridDesc {
    int32_t nx;
    int32_t ny;
    int64_t offset;
    // interior rectangle the step updates (the whole grid unless
    // pond_set_interior narrowed it; staged kernel only)
    int32_t ix0, iy0, iw, ih;
};

// Device state of one context: packed over all grids, plane stride = N.
template <typename Real>
struct StateBuf {
    Real* f;        // [Q][N]
    double* ux;     // [N]
    double* uy;     // [N]
    double* st;     // [N]  sqrt(theta) = sqrt(T / T_L)
};

// ---------------------------------------------------------------- kernels
// Launchers (defined in the .cu files); all return the launch status.

// Per-translation-unit constant-bank copies of the lattices (call once per
// device before launching): both D2Q16 and D2Q9, slot lattice_slot(n1).
cudaError_t upload_lattice_fp64();
cudaError_t upload_lattice_mixed();
cudaError_t upload_lattice_adjoint();
cudaError_t upload_lattice_adjoint_mixed();

// FP64 step of a single grid, lattice L.n1, nodes_per_warp 1, 2, (D2Q9) 3, or 32
// (one node per thread).
constexpr int FP64_NODE_PER_THREAD = 32;  // nodes_per_warp value of the node-per-thread kernel
// default mappings, measured fastest on both lattices at 2048^2 (D2Q16:
// 1.31e7 node-updates/s against 1.23e7 with two nodes per warp; D2Q9: 3.63e7
// against 2.66e7 with three)
constexpr int FP64_NODES_PER_WARP = FP64_NODE_PER_THREAD;
constexpr int FP64_NODES_PER_WARP_Q9 = FP64_NODE_PER_THREAD;
constexpr int fp64_default_npw(int n1) {
    return n1 == 3 ? FP64_NODES_PER_WARP_Q9 : FP64_NODES_PER_WARP;
}
// accepted nodes_per_warp values: 0 (default), 1, 2, 3 (D2Q9 only), 32
constexpr bool fp64_npw_valid(int npw, int lattice) {
    return npw == 0 || npw == 1 || npw == 2 || npw == FP64_NODE_PER_THREAD ||
           (npw == 3 && lattice == POND_D2Q9);
}
cudaError_t launch_step_fp64(const StateBuf<double>& in, const StateBuf<double>& out,
                             int32_t* iters, DevStats* stats, int nx, int ny,
                             const Lattice& L, const StepParams& P, int nodes_per_warp,
                             cudaStream_t s);

// Window (halo tile) size, in nodes, that the mixed tiled kernel stages:
// chosen by the host from a bound on the displacement spread.
struct TileWindow {
    int tx, ty;       // tile of target nodes
    int ww, wh;       // maximum staged window (tile + halo)
    int pair;         // 1: each thread owns two vertically adjacent nodes
    int n1;           // speeds per dimension of the lattice (4 or 3)
    int staged;       // 1: the reference-gauge staged kernel
    int real_bytes;   // 8 (FP64 form) or 4 (mixed form)
};

// Mixed-precision step over one or many grids (one CTA per tile; batched
// contexts use a persistent work list).
cudaError_t launch_step_mixed(const StateBuf<float>& in, const StateBuf<float>& out,
                              int32_t* iters, DevStats* stats, const GridDesc* grids_dev,
                              const int64_t* tile_prefix_dev, int n_grids,
                              int64_t n_tiles, int64_t plane, unsigned int* work_counter,
                              const TileWindow& win, int persistent_ctas,
                              const Lattice& L, const StepParams& P, cudaStream_t s);

// The reference-gauge staged kernel (pond_staged.cuh), FP64 and mixed
// forms, over one or many grids (tiles 32 x ty; ty 4 or 8 in FP64, 4, 8 or
// 16 in the mixed form), its per-device set-up (returns resident CTAs per SM
// for a dynamic shared-memory size) and that size for a window.
cudaError_t launch_step_staged_fp64(const StateBuf<double>& in, const StateBuf<double>& out,
                                    int32_t* iters, DevStats* stats, const GridDesc* grids_dev,
                                    const int64_t* tile_prefix_dev, int n_grids, int64_t n_tiles,
                                    int64_t plane, unsigned int* work_counter,
                                    const TileWindow& win, int persistent_ctas, const Lattice& L,
                                    const StepParams& P, cudaStream_t s);
cudaError_t launch_step_staged_mixed(const StateBuf<float>& in, const StateBuf<float>& out,
                                     int32_t* iters, DevStats* stats, const GridDesc* grids_dev,
                                     const int64_t* tile_prefix_dev, int n_grids, int64_t n_tiles,
                                     int64_t plane, unsigned int* work_counter,
                                     const TileWindow& win, int persistent_ctas, const Lattice& L,
                                     const StepParams& P, cudaStream_t s);
cudaError_t staged_prepare_fp64(int ty, int n1, size_t smem, int* ctas_per_sm);
cudaError_t staged_prepare_mixed(int ty, int n1, size_t smem, int* ctas_per_sm);
// Extra window extent, in nodes, that one step's departures need for a
// particle-speed spread `span`: ceil(span * dt + pad), bounded by 65536 so
// that an absurd spread (a finite but huge temperature or velocity, whose
// FP32 bounds may even be infinite or NaN) still gives a valid int.  The
// shared-memory caps then trim the window, and the stencils beyond it take
// the global-memory paths, which wrap any displacement.
inline int window_extent(double span, double dt, double pad) {
    const double e = std::fmax(span * dt + pad, 0.0);  // a NaN spread gives 0
    return (int)std::ceil(std::fmin(e, 65536.0));
}
// (as staged_smem_bytes: the FP64 form also holds the y-map table)
inline size_t staged_window_bytes(const TileWindow& w) {
    const size_t per_node = w.real_bytes == 8 ? 2 : 1;
    return (size_t)w.n1 * w.ww * w.wh * 4 * w.real_bytes +
           per_node * w.n1 * w.n1 * w.tx * w.ty * w.real_bytes;
}
constexpr int STAGED_TY_FP64[2] = {4, 8};
// default FP64 tile rows without autotuning: 32 x 8 on D2Q16 (measured 0-4 %
// faster than 32 x 4 from 256^2 to 2048^2), 32 x 4 on D2Q9 (the autotuner's
// choice at 2048^2)
constexpr int staged_ty_fp64_default(int n1) { return n1 == 4 ? 8 : 4; }
constexpr int STAGED_TY_MIXED[3] = {4, 8, 16};

// Tile shape of the mixed kernel, its shared-memory need for a window, and
// the per-device attribute set-up (returns resident CTAs per SM).
constexpr int MIXED_TX = 32, MIXED_TY = 8;  // default tile: 32 x 8 nodes
// tile shapes the autotuner tries: rows of 32-wide tiles, negative = the
// paired kernel (two stacked nodes per thread)
constexpr int MIXED_TY_CHOICES[4] = {4, 8, 16, -16};
size_t mixed_smem_bytes(const TileWindow& w);
cudaError_t mixed_prepare(int ty, bool pair, int n1, size_t smem_bytes, int* ctas_per_sm);

// Equilibrium initialisation f = rho W (Eq. equilibrium) and T -> sqrt(theta).
template <typename Real>
cudaError_t launch_init_state(const double* rho, const double* ux, const double* uy,
                              const double* T, const double* f_given, StateBuf<Real> st,
                              int64_t N, int64_t plane, const Lattice& L, cudaStream_t s);

// rho = sum f, T = st^2 T_L, and f (as FP64) read-out.
template <typename Real>
cudaError_t launch_read_state(StateBuf<Real> st, int64_t N, int64_t plane, double* rho,
                              double* ux, double* uy, double* T, double* f,
                              const Lattice& L, cudaStream_t s);

// Rectangle [x0, x0 + w) x [y0, y0 + h) of one grid's state to or from a
// device buffer of FP64 planes [Q + 3][h][w]: f (in its stored precision,
// widened exactly), u_x, u_y, sqrt(theta) (the stored gauge, bit for bit).
template <typename Real>
cudaError_t launch_pack_rect(StateBuf<Real> st, int nx, int x0, int y0, int w, int h, int q,
                             int64_t plane, double* buf, cudaStream_t s);
template <typename Real>
cudaError_t launch_unpack_rect(StateBuf<Real> st, int nx, int x0, int y0, int w, int h, int q,
                               int64_t plane, const double* buf, cudaStream_t s);

// Bounds of the particle velocities over the nodes, {min (u_x - c_max st),
// max (u_x + c_max st), min (u_y - c_max st), max (u_y + c_max st)} as
// floats in out5[0..3], and in out5[4] (read as an unsigned int) the number
// of nodes with st <= 0 or a non-finite gauge.
cudaError_t launch_disp_bounds(const double* ux, const double* uy, const double* st,
                               int64_t N, double c_max, float* out5, cudaStream_t s);

// Adjoint (pond_adjoint.cu, pond_adjoint_mixed.cu).
struct AdjointScratch;
struct AdjMixedScratch;
cudaError_t launch_minmax3(const double* ux, const double* uy, const double* st, long long N,
                           double* out6, cudaStream_t s);
// (u_x, u_y, T) -> (u_x, u_y, sqrt(T / T_L)) into the adjoint's forward gauge
cudaError_t launch_gauge_from_T(const double* ux, const double* uy, const double* T,
                                double* ux_o, double* uy_o, double* st_o, long long N,
                                double T_L, cudaStream_t s);

}  // namespace pond

struct pond_ctx {
    pond_config cfg;
    pond::Lattice L;
    pond::StepParams P;
    int32_t n_grids = 0;
    std::vector<pond::GridDesc> grids_host;
    std::vector<float> spans;  // per grid: {min vx, max vx, min vy, max vy}
    int64_t N = 0;  // total nodes
    int64_t N_active = 0;  // nodes a step updates (the interiors)
    int cur = 0;    // index of the current state buffer
    void* f[2] = {nullptr, nullptr};
    double* ux[2] = {nullptr, nullptr};
    double* uy[2] = {nullptr, nullptr};
    double* st[2] = {nullptr, nullptr};
    int32_t* iters = nullptr;
    pond::DevStats* stats = nullptr;
    pond::DevStats* stats_host = nullptr;  // pinned
    pond::GridDesc* grids_dev = nullptr;
    int64_t* tile_prefix_dev = nullptr;
    unsigned int* work_counter = nullptr;
    float* bounds_dev = nullptr;
    int64_t n_tiles = 0;
    int tile_ty = pond::MIXED_TY;  // rows of the mixed kernel's tile
    bool tile_pair = false;        // paired kernel (two stacked nodes per thread)
    bool tuned = false;
    pond::TileWindow win{};
    int persistent_ctas = 0;
    std::vector<char> grid_set;
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    void* staging = nullptr;       // device staging for host-side I/O
    size_t staging_bytes = 0;
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};  // two-step graphs per parity
    pond::AdjointScratch* adj = nullptr;
    pond::AdjMixedScratch* adjm = nullptr;
};

// the context runs the reference-gauge staged kernel
inline bool ctx_staged(const pond_ctx* ctx) { return ctx->cfg.kernel != POND_KERNEL_DIRECT; }

// One step of the context's configured kernel from `in` to `out` (used by
// pond_step and by the adjoints' forward recomputation, so both run the
// same arithmetic).
cudaError_t launch_ctx_step_fp64(pond_ctx* ctx, const pond::StateBuf<double>& in,
                                 const pond::StateBuf<double>& out, int32_t* iters,
                                 pond::DevStats* stats);
cudaError_t launch_ctx_step_mixed(pond_ctx* ctx, const pond::StateBuf<float>& in,
                                  const pond::StateBuf<float>& out, int32_t* iters,
                                  pond::DevStats* stats);

// nodes per warp of the context's FP64 step kernel
inline int fp64_npw(const pond_ctx* ctx) {
    return ctx->cfg.nodes_per_warp ? ctx->cfg.nodes_per_warp : pond::fp64_default_npw(ctx->L.n1);
}

void destroy_adjoint(pond_ctx* ctx);
void destroy_adjoint_mixed(pond_ctx* ctx);
// out_gauge: {u_x, u_y, T} of the step's output, or NULLs to recompute it
cudaError_t adjoint_step_mixed(pond_ctx* ctx, const double* const out_gauge[3],
                               const double* fbar, const double* gbar, double* fbar_out,
                               double* gbar_out, double* beta_bar_dev, double* minmax_dev);
