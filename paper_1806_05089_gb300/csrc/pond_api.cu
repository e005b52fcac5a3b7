// pond_api.cu -- C ABI of the PonD library (see include/pond.h).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <iterator>
#include <vector>

#include "pond_internal.cuh"

using namespace pond;

namespace {

const char* kVersion = "pond-gb300 0.2 (D2Q16 and D2Q9, sm_103a)";

pond_status fail(pond_ctx* c, pond_status s, const char* msg) {
    if (c) c->err = msg;
    return s;
}

pond_status cuda_fail(pond_ctx* c, cudaError_t e, const char* where) {
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    // a failed allocation (like any non-sticky error) is also left as the
    // runtime's last error, where the next launch check would find it and
    // report it again; clear it so the caller can carry on
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? POND_ERR_OOM : POND_ERR_CUDA;
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

bool mixed(const pond_ctx* c) { return c->cfg.precision == POND_FP32_MIXED; }

// contexts whose step runs a tile kernel (windows, tile shapes, autotune)
bool tiled(const pond_ctx* c) { return mixed(c) || ctx_staged(c); }

size_t real_size(const pond_ctx* c) { return mixed(c) ? sizeof(float) : sizeof(double); }

template <typename Real>
StateBuf<Real> buf(pond_ctx* c, int which, int64_t offset) {
    StateBuf<Real> b;
    b.f = static_cast<Real*>(c->f[which]) + offset;
    b.ux = c->ux[which] + offset;
    b.uy = c->uy[which] + offset;
    b.st = c->st[which] + offset;
    return b;
}

template <typename Real>
StateBuf<Real> buf_of(pond_ctx* c, int which, int64_t offset) {
    return buf<Real>(c, which, offset);
}

// Staging buffer for host-side input/output (20 FP64 fields of one grid).
pond_status ensure_staging(pond_ctx* ctx, int64_t nodes) {
    const size_t need = (size_t)20 * (size_t)nodes * sizeof(double);
    if (ctx->staging_bytes >= need) return POND_OK;
    if (ctx->staging) {
        CK(cudaStreamSynchronize(ctx->stream), "staging sync");
        CK(cudaFree(ctx->staging), "staging free");
        ctx->staging = nullptr;
        ctx->staging_bytes = 0;
    }
    CK(cudaMalloc(&ctx->staging, need), "staging alloc");
    ctx->staging_bytes = need;
    return POND_OK;
}

// Tile count and per-grid prefix of the mixed kernel for a tile of
// MIXED_TX x ty nodes (uploaded to the device).
pond_status set_tile_rows(pond_ctx* ctx, int code) {
    // code: rows of the 32-wide tile; negative selects the paired kernel
    const int ty = code < 0 ? -code : code;
    if (code < 0 && ctx->L.n1 != 4) return fail(ctx, POND_ERR_ARG, "paired tile shape: D2Q16 only");
    ctx->tile_pair = code < 0;
    std::vector<int64_t> prefix(ctx->n_grids + 1, 0);
    int64_t tiles = 0;
    for (int g = 0; g < ctx->n_grids; ++g) {
        prefix[g] = tiles;
        const GridDesc& G = ctx->grids_host[g];
        tiles += (int64_t)((G.iw + MIXED_TX - 1) / MIXED_TX) * ((G.ih + ty - 1) / ty);
    }
    prefix[ctx->n_grids] = tiles;
    CK(cudaMemcpyAsync(ctx->tile_prefix_dev, prefix.data(), sizeof(int64_t) * (ctx->n_grids + 1),
                       cudaMemcpyHostToDevice, ctx->stream),
       "tile prefix upload");
    CK(cudaStreamSynchronize(ctx->stream), "tile prefix sync");
    ctx->n_tiles = tiles;
    ctx->tile_ty = ty;
    return POND_OK;
}

// Window of the mixed kernel from the per-grid velocity spans.
pond_status update_window(pond_ctx* ctx) {
    if (!tiled(ctx)) return POND_OK;
    float sx = 0.f, sy = 0.f;
    for (int g = 0; g < ctx->n_grids; ++g) {
        if (!ctx->grid_set[g]) continue;
        const float* sp = &ctx->spans[4 * g];
        sx = std::fmax(sx, sp[1] - sp[0]);
        sy = std::fmax(sy, sp[3] - sp[2]);
    }
    const double dt = ctx->cfg.dt, margin = 1.0;
    TileWindow w;
    w.tx = MIXED_TX;
    w.ty = ctx->tile_ty;
    w.pair = ctx->tile_pair ? 1 : 0;
    w.n1 = ctx->L.n1;
    w.staged = ctx_staged(ctx) ? 1 : 0;
    w.real_bytes = mixed(ctx) ? 4 : 8;
    w.ww = w.tx + window_extent(sx, dt, 2 * margin) + 5;
    w.wh = w.ty + window_extent(sy, dt, 2 * margin) + 5;
    // cap the staged window at the shared memory a CTA can have; stencils
    // beyond it take the global-memory path
    auto bytes = [](const TileWindow& v) {
        return v.staged ? staged_window_bytes(v) : mixed_smem_bytes(v);
    };
    const size_t cap = 220 * 1024;
    while (bytes(w) > cap) {
        if (w.ww - w.tx >= w.wh - w.ty) --w.ww; else --w.wh;
    }
    const size_t smem = bytes(w);
    int per_sm = 0;
    if (!w.staged)
        CK(mixed_prepare(w.ty, w.pair != 0, w.n1, smem, &per_sm), "mixed kernel set-up");
    else if (mixed(ctx))
        CK(staged_prepare_mixed(w.ty, w.n1, smem, &per_sm), "staged kernel set-up");
    else
        CK(staged_prepare_fp64(w.ty, w.n1, smem, &per_sm), "staged kernel set-up");
    if (per_sm < 1) return fail(ctx, POND_ERR_CUDA, "tile kernel does not fit on an SM");
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "SM count");
    ctx->win = w;
    ctx->persistent_ctas = per_sm * sms;
    return POND_OK;
}

pond_status check_grid(pond_ctx* ctx, int32_t grid) {
    if (!ctx) return POND_ERR_ARG;
    if (grid < 0 || grid >= ctx->n_grids) return fail(ctx, POND_ERR_ARG, "grid index out of range");
    return POND_OK;
}

}  // namespace

cudaError_t launch_ctx_step_fp64(pond_ctx* ctx, const StateBuf<double>& in,
                                 const StateBuf<double>& out, int32_t* iters, DevStats* stats) {
    if (ctx_staged(ctx))
        return launch_step_staged_fp64(in, out, iters, stats, ctx->grids_dev, ctx->tile_prefix_dev,
                                       ctx->n_grids, ctx->n_tiles, ctx->N,
                                       ctx->n_grids > 1 ? ctx->work_counter : nullptr, ctx->win,
                                       ctx->persistent_ctas, ctx->L, ctx->P, ctx->stream);
    const GridDesc& G = ctx->grids_host[0];
    return launch_step_fp64(in, out, iters, stats, G.nx, G.ny, ctx->L, ctx->P, fp64_npw(ctx),
                            ctx->stream);
}

cudaError_t launch_ctx_step_mixed(pond_ctx* ctx, const StateBuf<float>& in,
                                  const StateBuf<float>& out, int32_t* iters, DevStats* stats) {
    unsigned int* counter = ctx->n_grids > 1 ? ctx->work_counter : nullptr;
    if (ctx_staged(ctx))
        return launch_step_staged_mixed(in, out, iters, stats, ctx->grids_dev, ctx->tile_prefix_dev,
                                        ctx->n_grids, ctx->n_tiles, ctx->N, counter, ctx->win,
                                        ctx->persistent_ctas, ctx->L, ctx->P, ctx->stream);
    return launch_step_mixed(in, out, iters, stats, ctx->grids_dev, ctx->tile_prefix_dev,
                             ctx->n_grids, ctx->n_tiles, ctx->N, counter, ctx->win,
                             ctx->persistent_ctas, ctx->L, ctx->P, ctx->stream);
}

// one step from buffer `in` into buffer `out` with the context's kernel
static pond_status launch_step_into(pond_ctx* ctx, int in, int out) {
    if (mixed(ctx))
        CK(launch_ctx_step_mixed(ctx, buf<float>(ctx, in, 0), buf<float>(ctx, out, 0), ctx->iters,
                                 ctx->stats),
           "mixed step launch");
    else
        CK(launch_ctx_step_fp64(ctx, buf<double>(ctx, in, 0), buf<double>(ctx, out, 0), ctx->iters,
                                ctx->stats),
           "fp64 step launch");
    return POND_OK;
}

static pond_status launch_one_step(pond_ctx* ctx) {
    const int in = ctx->cur, out = 1 - ctx->cur;
    pond_status s = launch_step_into(ctx, in, out);
    if (s != POND_OK) return s;
    ctx->cur = out;
    return POND_OK;
}

// Two steps captured as one CUDA graph per buffer parity (the state buffers
// alternate, so two steps return to the same layout).
static void drop_graphs(pond_ctx* ctx) {
    for (int i = 0; i < 2; ++i) {
        if (ctx->graph_exec[i]) cudaGraphExecDestroy(ctx->graph_exec[i]);
        ctx->graph_exec[i] = nullptr;
    }
}

static pond_status ensure_graph(pond_ctx* ctx) {
    if (ctx->graph_exec[ctx->cur]) return POND_OK;
    cudaStream_t cap = nullptr;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "graph stream");
    cudaStream_t user = ctx->stream;
    ctx->stream = cap;
    const int cur0 = ctx->cur;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    pond_status s = POND_OK;
    if (e == cudaSuccess) {
        s = launch_one_step(ctx);
        if (s == POND_OK) s = launch_one_step(ctx);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
    }
    ctx->stream = user;
    ctx->cur = cur0;
    cudaStreamDestroy(cap);
    if (s != POND_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    CK(e, "graph capture");
    e = cudaGraphInstantiate(&ctx->graph_exec[cur0], graph, 0);
    cudaGraphDestroy(graph);
    CK(e, "graph instantiate");
    return POND_OK;
}

static pond_status read_out(pond_ctx* ctx, int32_t grid, void* rho, void* ux, void* uy, void* T,
                            void* f, int32_t on_device) {
    pond_status s = check_grid(ctx, grid);
    if (s != POND_OK) return s;
    if (!ctx->grid_set[grid]) return fail(ctx, POND_ERR_STATE, "grid state never set");
    DeviceGuard dg(ctx->device);
    const GridDesc& G = ctx->grids_host[grid];
    const int64_t n = (int64_t)G.nx * G.ny;
    double *d_rho, *d_ux, *d_uy, *d_T, *d_f;
    if (on_device) {
        d_rho = static_cast<double*>(rho);
        d_ux = static_cast<double*>(ux);
        d_uy = static_cast<double*>(uy);
        d_T = static_cast<double*>(T);
        d_f = static_cast<double*>(f);
    } else {
        s = ensure_staging(ctx, n);
        if (s != POND_OK) return s;
        double* sb = static_cast<double*>(ctx->staging);
        d_rho = rho ? sb : nullptr;
        d_ux = ux ? sb + n : nullptr;
        d_uy = uy ? sb + 2 * n : nullptr;
        d_T = T ? sb + 3 * n : nullptr;
        d_f = f ? sb + 4 * n : nullptr;
    }
    if (mixed(ctx)) {
        CK(launch_read_state<float>(buf<float>(ctx, ctx->cur, G.offset), n, ctx->N, d_rho, d_ux,
                                    d_uy, d_T, d_f, ctx->L, ctx->stream),
           "read state");
    } else {
        CK(launch_read_state<double>(buf<double>(ctx, ctx->cur, G.offset), n, ctx->N, d_rho, d_ux,
                                     d_uy, d_T, d_f, ctx->L, ctx->stream),
           "read state");
    }
    if (!on_device) {
        const size_t fb = sizeof(double) * n;
        if (rho) CK(cudaMemcpyAsync(rho, d_rho, fb, cudaMemcpyDeviceToHost, ctx->stream), "D2H rho");
        if (ux) CK(cudaMemcpyAsync(ux, d_ux, fb, cudaMemcpyDeviceToHost, ctx->stream), "D2H ux");
        if (uy) CK(cudaMemcpyAsync(uy, d_uy, fb, cudaMemcpyDeviceToHost, ctx->stream), "D2H uy");
        if (T) CK(cudaMemcpyAsync(T, d_T, fb, cudaMemcpyDeviceToHost, ctx->stream), "D2H T");
        if (f) CK(cudaMemcpyAsync(f, d_f, ctx->L.q * fb, cudaMemcpyDeviceToHost, ctx->stream), "D2H f");
        CK(cudaStreamSynchronize(ctx->stream), "read sync");
    }
    return POND_OK;
}

extern "C" {

const char* pond_version(void) { return kVersion; }

void pond_config_default(pond_config* cfg, int32_t precision) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->precision = precision;
    cfg->thermal = 1;
    cfg->nu = 0.01;
    cfg->T_ref = 1.0;
    cfg->dt = 1.0;
    if (precision == POND_FP32_MIXED) {
        cfg->eps_abs = 1e-6;
        cfg->eps_rel = 1e-6;
    } else {
        cfg->eps_abs = 1e-12;
        cfg->eps_rel = 1e-10;
    }
    cfg->max_iter = 20;
    cfg->fixed_iter = 0;
    cfg->ckpt_every = 20;
    cfg->strict = 0;
    cfg->seed_mode = 0;
    cfg->use_graph = 0;
    cfg->autotune = 0;
    cfg->tile_rows = 0;
    cfg->lattice = POND_D2Q16;
}

pond_status pond_create(const pond_config* cfg, int32_t n_grids, const int32_t* nx,
                        const int32_t* ny, void* cuda_stream, pond_ctx** out) {
    if (!out) return POND_ERR_ARG;
    *out = nullptr;
    if (!cfg || !nx || !ny || n_grids < 1) return POND_ERR_ARG;
    if (cfg->precision != POND_FP64 && cfg->precision != POND_FP32_MIXED) return POND_ERR_ARG;
    if (!(cfg->nu > 0.0) || !(cfg->T_ref > 0.0) || !(cfg->dt > 0.0) || cfg->max_iter < 1 ||
        cfg->fixed_iter < 0 || cfg->seed_mode < 0 || cfg->seed_mode > 2)
        return POND_ERR_ARG;
    if (cfg->tile_rows != 0 && cfg->tile_rows != 4 && cfg->tile_rows != 8 && cfg->tile_rows != 16 &&
        cfg->tile_rows != -16)
        return POND_ERR_ARG;
    if (cfg->kernel < POND_KERNEL_DEFAULT || cfg->kernel > POND_KERNEL_DIRECT) return POND_ERR_ARG;
    if (cfg->lattice != POND_D2Q16 && cfg->lattice != POND_D2Q9) return POND_ERR_ARG;
    if (!pond::fp64_npw_valid(cfg->nodes_per_warp, cfg->lattice)) return POND_ERR_ARG;
    if (cfg->lattice == POND_D2Q9 && cfg->tile_rows < 0) return POND_ERR_ARG;  // paired: D2Q16
    for (int g = 0; g < n_grids; ++g)
        if (nx[g] < 1 || ny[g] < 1) return POND_ERR_ARG;

    // the default kernel is the staged one, except where the config asks for
    // a shape or mapping only the direct kernels have (the paired tile, an
    // FP64 nodes-per-warp mapping)
    int kernel = cfg->kernel;
    if (kernel == POND_KERNEL_DEFAULT)
        kernel = (cfg->tile_rows == -16 ||
                  (cfg->precision == POND_FP64 && cfg->nodes_per_warp != 0))
                     ? POND_KERNEL_DIRECT
                     : POND_KERNEL_STAGED;
    if (kernel == POND_KERNEL_STAGED &&
        (cfg->tile_rows < 0 || (cfg->precision == POND_FP64 && cfg->tile_rows == 16)))
        return POND_ERR_ARG;
    if (kernel == POND_KERNEL_DIRECT && cfg->precision == POND_FP64 && cfg->tile_rows != 0)
        return POND_ERR_ARG;  // the direct FP64 kernels have no tiles
    if (kernel == POND_KERNEL_DIRECT && cfg->precision == POND_FP64 && n_grids != 1)
        return POND_ERR_ARG;  // ... and step one grid

    pond_ctx* ctx = new (std::nothrow) pond_ctx();
    if (!ctx) return POND_ERR_OOM;
    ctx->cfg = *cfg;
    ctx->cfg.kernel = kernel;
    ctx->L = make_lattice(cfg->lattice);
    ctx->P.beta = 1.0 / (2.0 * cfg->nu / (cfg->T_ref * cfg->dt) + 1.0);
    ctx->P.dt = cfg->dt;
    ctx->P.eps_abs = cfg->eps_abs;
    ctx->P.eps_rel = cfg->eps_rel;
    ctx->P.T_L = ctx->L.T_L;
    ctx->P.max_iter = cfg->max_iter;
    ctx->P.fixed_iter = cfg->fixed_iter;
    ctx->P.thermal = cfg->thermal;
    ctx->P.seed_mode = cfg->seed_mode;
    ctx->n_grids = n_grids;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&ctx->device);
    ctx->grid_set.assign(n_grids, 0);
    ctx->spans.assign(4 * (size_t)n_grids, 0.f);
    int64_t off = 0, tiles = 0;
    std::vector<int64_t> prefix(n_grids + 1, 0);
    for (int g = 0; g < n_grids; ++g) {
        GridDesc d;
        d.nx = nx[g];
        d.ny = ny[g];
        d.offset = off;
        d.ix0 = 0;
        d.iy0 = 0;
        d.iw = nx[g];
        d.ih = ny[g];
        ctx->grids_host.push_back(d);
        off += (int64_t)nx[g] * ny[g];
        prefix[g] = tiles;
        tiles += (int64_t)((nx[g] + MIXED_TX - 1) / MIXED_TX) * ((ny[g] + MIXED_TY - 1) / MIXED_TY);
    }
    prefix[n_grids] = tiles;
    ctx->N = off;
    ctx->N_active = off;
    ctx->n_tiles = tiles;

    pond_status st = POND_OK;
    auto alloc = [&](void** p, size_t bytes, const char* what) -> bool {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e != cudaSuccess) {
            st = cuda_fail(ctx, e, what);
            return false;
        }
        return true;
    };
    const size_t rs = real_size(ctx);
    bool ok = true;
    for (int b = 0; b < 2 && ok; ++b) {
        ok = ok && alloc(&ctx->f[b], rs * ctx->L.q * (size_t)ctx->N, "alloc f");
        ok = ok && alloc((void**)&ctx->ux[b], sizeof(double) * ctx->N, "alloc ux");
        ok = ok && alloc((void**)&ctx->uy[b], sizeof(double) * ctx->N, "alloc uy");
        ok = ok && alloc((void**)&ctx->st[b], sizeof(double) * ctx->N, "alloc st");
    }
    ok = ok && alloc((void**)&ctx->iters, sizeof(int32_t) * ctx->N, "alloc iters");
    ok = ok && alloc((void**)&ctx->stats, sizeof(DevStats), "alloc stats");
    ok = ok && alloc((void**)&ctx->grids_dev, sizeof(GridDesc) * n_grids, "alloc grids");
    ok = ok && alloc((void**)&ctx->tile_prefix_dev, sizeof(int64_t) * (n_grids + 1), "alloc prefix");
    ok = ok && alloc((void**)&ctx->work_counter, sizeof(unsigned int), "alloc counter");
    ok = ok && alloc((void**)&ctx->bounds_dev, 8 * sizeof(float), "alloc bounds");
    if (ok) {
        cudaError_t e = cudaMallocHost((void**)&ctx->stats_host, sizeof(DevStats));
        if (e != cudaSuccess) {
            st = cuda_fail(ctx, e, "alloc pinned stats");
            ok = false;
        }
    }
    if (ok) {
        cudaError_t e = cudaMemcpy(ctx->grids_dev, ctx->grids_host.data(),
                                   sizeof(GridDesc) * n_grids, cudaMemcpyHostToDevice);

        if (e == cudaSuccess) e = cudaMemset(ctx->iters, 0, sizeof(int32_t) * ctx->N);
        if (e == cudaSuccess) e = upload_lattice_fp64();
        if (e == cudaSuccess) e = upload_lattice_mixed();
        if (e == cudaSuccess) e = upload_lattice_adjoint();
        if (e == cudaSuccess) e = upload_lattice_adjoint_mixed();
        if (e != cudaSuccess) {
            st = cuda_fail(ctx, e, "context set-up");
            ok = false;
        }
    }
    if (!ok) {
        pond_destroy(ctx);
        return st == POND_OK ? POND_ERR_CUDA : st;
    }
    if (tiled(ctx)) {
        const int ty0 = mixed(ctx) ? MIXED_TY : staged_ty_fp64_default(ctx->L.n1);
        st = set_tile_rows(ctx, cfg->tile_rows ? cfg->tile_rows : ty0);
        if (cfg->tile_rows) ctx->tuned = true;  // a forced shape is not retuned
        if (st != POND_OK) {
            pond_destroy(ctx);
            return st;
        }
        // provisional window until set_state measures the displacements
        for (int g = 0; g < n_grids; ++g) {
            ctx->spans[4 * g + 0] = -6.f;
            ctx->spans[4 * g + 1] = 6.f;
            ctx->spans[4 * g + 2] = -6.f;
            ctx->spans[4 * g + 3] = 6.f;
        }
        std::vector<char> saved = ctx->grid_set;
        ctx->grid_set.assign(n_grids, 1);
        st = update_window(ctx);
        ctx->grid_set = saved;
        if (st != POND_OK) {
            pond_destroy(ctx);
            return st;
        }
    }
    *out = ctx;
    return POND_OK;
}

pond_status pond_set_stream(pond_ctx* ctx, void* cuda_stream) {
    if (!ctx) return POND_ERR_ARG;
    const cudaStream_t next = static_cast<cudaStream_t>(cuda_stream);
    if (next == ctx->stream) return POND_OK;
    DeviceGuard dg(ctx->device);
    // work already queued on the old stream finishes before anything is
    // queued on the new one; the step graphs are captured again on next use
    CK(cudaStreamSynchronize(ctx->stream), "set_stream sync");
    drop_graphs(ctx);
    ctx->stream = next;
    return POND_OK;
}

pond_status pond_set_state(pond_ctx* ctx, int32_t grid, const void* rho, const void* ux,
                           const void* uy, const void* T, const void* f, int32_t on_device) {
    pond_status s = check_grid(ctx, grid);
    if (s != POND_OK) return s;
    if (!ux || !uy || !T || (!f && !rho))
        return fail(ctx, POND_ERR_ARG, "set_state: ux, uy, T and one of rho / f are required");
    DeviceGuard dg(ctx->device);
    NvtxRange nv("pond_set_state");
    const GridDesc& G = ctx->grids_host[grid];
    const int64_t n = (int64_t)G.nx * G.ny;
    const double *d_rho, *d_ux, *d_uy, *d_T, *d_f;
    if (on_device) {
        d_rho = static_cast<const double*>(rho);
        d_ux = static_cast<const double*>(ux);
        d_uy = static_cast<const double*>(uy);
        d_T = static_cast<const double*>(T);
        d_f = static_cast<const double*>(f);
    } else {
        s = ensure_staging(ctx, n);
        if (s != POND_OK) return s;
        double* sb = static_cast<double*>(ctx->staging);
        double* p_rho = sb;
        double* p_ux = sb + n;
        double* p_uy = sb + 2 * n;
        double* p_T = sb + 3 * n;
        double* p_f = sb + 4 * n;
        const size_t fb = sizeof(double) * n;
        if (rho) CK(cudaMemcpyAsync(p_rho, rho, fb, cudaMemcpyHostToDevice, ctx->stream), "H2D rho");
        CK(cudaMemcpyAsync(p_ux, ux, fb, cudaMemcpyHostToDevice, ctx->stream), "H2D ux");
        CK(cudaMemcpyAsync(p_uy, uy, fb, cudaMemcpyHostToDevice, ctx->stream), "H2D uy");
        CK(cudaMemcpyAsync(p_T, T, fb, cudaMemcpyHostToDevice, ctx->stream), "H2D T");
        if (f) CK(cudaMemcpyAsync(p_f, f, ctx->L.q * fb, cudaMemcpyHostToDevice, ctx->stream), "H2D f");
        d_rho = rho ? p_rho : nullptr;
        d_ux = p_ux;
        d_uy = p_uy;
        d_T = p_T;
        d_f = f ? p_f : nullptr;
    }
    if (mixed(ctx)) {
        CK(launch_init_state<float>(d_rho, d_ux, d_uy, d_T, d_f, buf<float>(ctx, ctx->cur, G.offset),
                                    n, ctx->N, ctx->L, ctx->stream),
           "init state");
    } else {
        CK(launch_init_state<double>(d_rho, d_ux, d_uy, d_T, d_f,
                                     buf<double>(ctx, ctx->cur, G.offset), n, ctx->N, ctx->L,
                                     ctx->stream),
           "init state");
    }
    // velocity spans of this grid, for the tile kernels' windows, and the
    // count of nodes with T <= 0 or a non-finite gauge (the gauge is checked
    // on the device, in the same pass, for host and device input alike)
    CK(launch_disp_bounds(ctx->ux[ctx->cur] + G.offset, ctx->uy[ctx->cur] + G.offset,
                          ctx->st[ctx->cur] + G.offset, n, ctx->L.c_max, ctx->bounds_dev,
                          ctx->stream),
       "bounds");
    float b5[5];
    CK(cudaMemcpyAsync(b5, ctx->bounds_dev, sizeof b5, cudaMemcpyDeviceToHost, ctx->stream), "D2H bounds");
    CK(cudaStreamSynchronize(ctx->stream), "set_state sync");
    unsigned int bad = 0;
    std::memcpy(&bad, &b5[4], sizeof bad);
    if (bad != 0 || !(std::isfinite(b5[0]) && std::isfinite(b5[1]) && std::isfinite(b5[2]) &&
                      std::isfinite(b5[3]))) {
        // the grid's buffers now hold the refused state: no step runs on it
        // until a valid pond_set_state
        ctx->grid_set[grid] = 0;
        return fail(ctx, POND_ERR_NONPHYSICAL, "set_state: T <= 0 or non-finite gauge");
    }
    for (int i = 0; i < 4; ++i) ctx->spans[4 * grid + i] = b5[i];
    ctx->grid_set[grid] = 1;
    const TileWindow before = ctx->win;
    s = update_window(ctx);
    if (before.ww != ctx->win.ww || before.wh != ctx->win.wh) drop_graphs(ctx);
    return s;
}

// ---------------------------------------------------------------- autotuner
// Times each tile shape of the mixed kernel on the current state (the step
// is recomputed into the spare buffer; the state does not advance) and keeps
// the fastest.  Choices are cached per process, and in the JSON file named by
// POND_AUTOTUNE_CACHE when set, under a signature of the grid set.
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;
bool g_tune_file_loaded = false;

std::string tune_key(const pond_ctx* ctx) {
    int64_t maxside = 0, minside = 1 << 30;
    for (const GridDesc& G : ctx->grids_host) {
        maxside = std::max<int64_t>(maxside, std::max(G.nx, G.ny));
        minside = std::min<int64_t>(minside, std::min(G.nx, G.ny));
    }
    float sx = 0.f, sy = 0.f;
    for (int g = 0; g < ctx->n_grids; ++g) {
        sx = std::fmax(sx, ctx->spans[4 * g + 1] - ctx->spans[4 * g]);
        sy = std::fmax(sy, ctx->spans[4 * g + 3] - ctx->spans[4 * g + 2]);
    }
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s|%s|q%d|grids=%d|nodes=%lld|side=%lld-%lld|span=%d-%d",
                  mixed(ctx) ? "mixed" : "fp64", ctx_staged(ctx) ? "staged" : "direct",
                  ctx->L.q, ctx->n_grids, (long long)ctx->N, (long long)minside,
                  (long long)maxside, window_extent(sx, 1.0, 0.0), window_extent(sy, 1.0, 0.0));
    return buf;
}

void tune_file_load() {
    const char* path = std::getenv("POND_AUTOTUNE_CACHE");
    if (!path || g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    FILE* fp = std::fopen(path, "r");
    if (!fp) return;
    // flat JSON object of "key": rows pairs
    std::string text;
    char chunk[4096];
    size_t n;
    while ((n = std::fread(chunk, 1, sizeof chunk, fp)) > 0) text.append(chunk, n);
    std::fclose(fp);
    size_t pos = 0;
    while ((pos = text.find('"', pos)) != std::string::npos) {
        const size_t end = text.find('"', pos + 1);
        if (end == std::string::npos) break;
        const std::string key = text.substr(pos + 1, end - pos - 1);
        const size_t colon = text.find(':', end);
        if (colon == std::string::npos) break;
        const int rows = std::atoi(text.c_str() + colon + 1);
        if (rows == 4 || rows == 8 || rows == 16 || rows == -16) g_tune_cache[key] = rows;
        pos = text.find_first_of(",}", colon);
        if (pos == std::string::npos) break;
    }
}

void tune_file_store() {
    const char* path = std::getenv("POND_AUTOTUNE_CACHE");
    if (!path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* fp = std::fopen(tmp.c_str(), "w");
    if (!fp) return;
    std::fprintf(fp, "{");
    bool first = true;
    for (const auto& kv : g_tune_cache) {
        std::fprintf(fp, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
        first = false;
    }
    std::fprintf(fp, "\n}\n");
    std::fclose(fp);
    std::rename(tmp.c_str(), path);
}
}  // namespace

static pond_status autotune(pond_ctx* ctx) {
    NvtxRange nv("pond_autotune");
    const std::string key = tune_key(ctx);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_file_load();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            pond_status s = set_tile_rows(ctx, it->second);
            if (s == POND_OK) s = update_window(ctx);
            ctx->tuned = true;
            return s;
        }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "autotune event");
    CK(cudaEventCreate(&e1), "autotune event");
    float best_ms = 1e30f;
    int best = ctx->tile_pair ? -ctx->tile_ty : ctx->tile_ty;
    pond_status s = POND_OK;
    std::vector<int> choices;
    if (!ctx_staged(ctx)) {
        for (int ty : MIXED_TY_CHOICES)
            if (ty > 0 || ctx->L.n1 == 4) choices.push_back(ty);  // paired: D2Q16 only
    } else if (mixed(ctx)) {
        choices.assign(std::begin(STAGED_TY_MIXED), std::end(STAGED_TY_MIXED));
    } else {
        choices.assign(std::begin(STAGED_TY_FP64), std::end(STAGED_TY_FP64));
    }
    for (int ty : choices) {
        s = set_tile_rows(ctx, ty);
        if (s == POND_OK) s = update_window(ctx);
        if (s != POND_OK) break;
        s = launch_step_into(ctx, ctx->cur, 1 - ctx->cur);  // warm-up
        if (s != POND_OK) break;
        cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < 3 && s == POND_OK; ++r) s = launch_step_into(ctx, ctx->cur, 1 - ctx->cur);
        cudaEventRecord(e1, ctx->stream);
        if (s != POND_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            s = fail(ctx, POND_ERR_CUDA, "autotune timing");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = ty;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != POND_OK) return s;
    s = set_tile_rows(ctx, best);
    if (s == POND_OK) s = update_window(ctx);
    if (s != POND_OK) return s;
    ctx->tuned = true;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    tune_file_store();
    return POND_OK;
}

pond_status pond_step(pond_ctx* ctx, int32_t nsteps, pond_stats* stats) {
    if (!ctx) return POND_ERR_ARG;
    NvtxRange nv("pond_step");
    if (nsteps < 0) return fail(ctx, POND_ERR_ARG, "nsteps < 0");
    for (int g = 0; g < ctx->n_grids; ++g)
        if (!ctx->grid_set[g]) return fail(ctx, POND_ERR_STATE, "pond_step before pond_set_state");
    DeviceGuard dg(ctx->device);
    if (ctx->cfg.autotune && tiled(ctx) && !ctx->tuned && nsteps > 0) {
        pond_status s = autotune(ctx);
        if (s != POND_OK) return s;
        drop_graphs(ctx);
    }
    if (stats) CK(cudaMemsetAsync(ctx->stats, 0, sizeof(DevStats), ctx->stream), "stats reset");
    int32_t left = nsteps;
    if (ctx->cfg.use_graph && left >= 2) {
        pond_status s = ensure_graph(ctx);
        if (s != POND_OK) return s;
        while (left >= 2) {
            CK(cudaGraphLaunch(ctx->graph_exec[ctx->cur], ctx->stream), "graph launch");
            left -= 2;
        }
    }
    while (left-- > 0) {
        pond_status s = launch_one_step(ctx);
        if (s != POND_OK) return s;
    }
    if (stats) {
        CK(cudaMemcpyAsync(ctx->stats_host, ctx->stats, sizeof(DevStats), cudaMemcpyDeviceToHost,
                           ctx->stream),
           "D2H stats");
        CK(cudaStreamSynchronize(ctx->stream), "step sync");
        const DevStats& d = *ctx->stats_host;
        stats->node_updates = (int64_t)nsteps * ctx->N_active;
        stats->passes = (int64_t)d.passes;
        stats->max_passes = (int32_t)d.max_passes;
        stats->tile_rows = tiled(ctx) ? (ctx->tile_pair ? -ctx->tile_ty : ctx->tile_ty) : 0;
        stats->nonconverged = (int64_t)d.nonconverged;
        stats->nonphysical = (int64_t)d.nonphysical;
        stats->halo_fallback = (int64_t)d.halo_fallback;
        stats->index_faults = (int64_t)d.index_faults;
        stats->busy_ns = (int64_t)d.busy_ns;
        stats->slot_ns = (int64_t)d.slot_ns;
        if (d.nonphysical) return fail(ctx, POND_ERR_NONPHYSICAL, "rho <= 0, T <= 0 or NaN met");
        if (ctx->cfg.strict && d.nonconverged)
            return fail(ctx, POND_ERR_NOT_CONVERGED, "a node hit max_iter without converging");
    }
    return POND_OK;
}

pond_status pond_moments(pond_ctx* ctx, int32_t grid, void* rho, void* ux, void* uy, void* T,
                         int32_t on_device) {
    return read_out(ctx, grid, rho, ux, uy, T, nullptr, on_device);
}

pond_status pond_get_state(pond_ctx* ctx, int32_t grid, void* f, void* ux, void* uy, void* T,
                           int32_t on_device) {
    return read_out(ctx, grid, nullptr, ux, uy, T, f, on_device);
}

pond_status pond_iterations(pond_ctx* ctx, int32_t grid, void* iters, int32_t on_device) {
    pond_status s = check_grid(ctx, grid);
    if (s != POND_OK) return s;
    if (!iters) return fail(ctx, POND_ERR_ARG, "iters is NULL");
    DeviceGuard dg(ctx->device);
    const GridDesc& G = ctx->grids_host[grid];
    const size_t bytes = sizeof(int32_t) * (size_t)G.nx * G.ny;
    CK(cudaMemcpyAsync(iters, ctx->iters + G.offset, bytes,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
       "copy iters");
    if (!on_device) CK(cudaStreamSynchronize(ctx->stream), "iters sync");
    return POND_OK;
}

pond_status pond_set_interior(pond_ctx* ctx, int32_t grid, int32_t x0, int32_t y0, int32_t w,
                              int32_t h) {
    pond_status s = check_grid(ctx, grid);
    if (s != POND_OK) return s;
    if (!ctx_staged(ctx)) return fail(ctx, POND_ERR_ARG, "set_interior: staged kernel only");
    GridDesc& G = ctx->grids_host[grid];
    if (x0 < 0 || y0 < 0 || w < 1 || h < 1 || (int64_t)x0 + w > G.nx || (int64_t)y0 + h > G.ny)
        return fail(ctx, POND_ERR_ARG, "set_interior: rectangle outside the grid");
    DeviceGuard dg(ctx->device);
    G.ix0 = x0;
    G.iy0 = y0;
    G.iw = w;
    G.ih = h;
    CK(cudaMemcpyAsync(ctx->grids_dev + grid, &G, sizeof(GridDesc), cudaMemcpyHostToDevice,
                       ctx->stream),
       "interior upload");
    CK(cudaStreamSynchronize(ctx->stream), "interior sync");
    s = set_tile_rows(ctx, ctx->tile_pair ? -ctx->tile_ty : ctx->tile_ty);
    if (s != POND_OK) return s;
    ctx->N_active = 0;
    for (const GridDesc& d : ctx->grids_host) ctx->N_active += (int64_t)d.iw * d.ih;
    drop_graphs(ctx);
    return POND_OK;
}

static pond_status rect_io(pond_ctx* ctx, int32_t grid, int32_t x0, int32_t y0, int32_t w,
                           int32_t h, double* buf, bool pack) {
    pond_status s = check_grid(ctx, grid);
    if (s != POND_OK) return s;
    if (!buf) return fail(ctx, POND_ERR_ARG, "rect: NULL buffer");
    const GridDesc& G = ctx->grids_host[grid];
    if (x0 < 0 || y0 < 0 || w < 0 || h < 0 || (int64_t)x0 + w > G.nx || (int64_t)y0 + h > G.ny)
        return fail(ctx, POND_ERR_ARG, "rect: rectangle outside the grid");
    DeviceGuard dg(ctx->device);
    NvtxRange nv(pack ? "pond_pack_rect" : "pond_unpack_rect");
    const int q = ctx->L.q;
    if (mixed(ctx)) {
        StateBuf<float> b = buf_of<float>(ctx, ctx->cur, G.offset);
        CK(pack ? launch_pack_rect<float>(b, G.nx, x0, y0, w, h, q, ctx->N, buf, ctx->stream)
                : launch_unpack_rect<float>(b, G.nx, x0, y0, w, h, q, ctx->N, buf, ctx->stream),
           "rect copy");
    } else {
        StateBuf<double> b = buf_of<double>(ctx, ctx->cur, G.offset);
        CK(pack ? launch_pack_rect<double>(b, G.nx, x0, y0, w, h, q, ctx->N, buf, ctx->stream)
                : launch_unpack_rect<double>(b, G.nx, x0, y0, w, h, q, ctx->N, buf, ctx->stream),
           "rect copy");
    }
    return POND_OK;
}

pond_status pond_pack_rect(pond_ctx* ctx, int32_t grid, int32_t x0, int32_t y0, int32_t w,
                           int32_t h, void* buf) {
    return rect_io(ctx, grid, x0, y0, w, h, static_cast<double*>(buf), true);
}

pond_status pond_unpack_rect(pond_ctx* ctx, int32_t grid, int32_t x0, int32_t y0, int32_t w,
                             int32_t h, const void* buf) {
    return rect_io(ctx, grid, x0, y0, w, h, const_cast<double*>(static_cast<const double*>(buf)),
                   false);
}

pond_status pond_max_displacement(pond_ctx* ctx, int32_t grid, double* out) {
    pond_status s = check_grid(ctx, grid);
    if (s != POND_OK) return s;
    if (!out) return fail(ctx, POND_ERR_ARG, "max_displacement: NULL output");
    if (!ctx->grid_set[grid]) return fail(ctx, POND_ERR_STATE, "grid state never set");
    DeviceGuard dg(ctx->device);
    const GridDesc& G = ctx->grids_host[grid];
    const int64_t n = (int64_t)G.nx * G.ny;
    CK(launch_disp_bounds(ctx->ux[ctx->cur] + G.offset, ctx->uy[ctx->cur] + G.offset,
                          ctx->st[ctx->cur] + G.offset, n, ctx->L.c_max, ctx->bounds_dev,
                          ctx->stream),
       "bounds");
    float b4[4];
    CK(cudaMemcpyAsync(b4, ctx->bounds_dev, sizeof b4, cudaMemcpyDeviceToHost, ctx->stream),
       "D2H bounds");
    CK(cudaStreamSynchronize(ctx->stream), "bounds sync");
    double m = 0.0;
    for (int i = 0; i < 4; ++i) m = std::fmax(m, std::fabs((double)b4[i]));
    *out = m * ctx->cfg.dt;
    return POND_OK;
}

void pond_destroy(pond_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard dg(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    destroy_adjoint(ctx);
    destroy_adjoint_mixed(ctx);
    drop_graphs(ctx);
    for (int b = 0; b < 2; ++b) {
        cudaFree(ctx->f[b]);
        cudaFree(ctx->ux[b]);
        cudaFree(ctx->uy[b]);
        cudaFree(ctx->st[b]);
    }
    cudaFree(ctx->iters);
    cudaFree(ctx->stats);
    cudaFree(ctx->grids_dev);
    cudaFree(ctx->tile_prefix_dev);
    cudaFree(ctx->work_counter);
    cudaFree(ctx->bounds_dev);
    cudaFree(ctx->staging);
    if (ctx->stats_host) cudaFreeHost(ctx->stats_host);
    delete ctx;
}

const char* pond_last_error(const pond_ctx* ctx) {
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

}  // extern "C"
