// runtime.cu -- host runtime behind the C ABI of include/hjb.h: problem
// objects, workspaces, TMA descriptors, the CUDA-graph convergence loop and
// the entry points hjb_create ... hjb_point_values.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <dlfcn.h>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hjb.h"
#include "hjb_internal.cuh"

using hjbk::Ctl;
using hjbk::SlotDesc;
using hjbk::SlotState;


namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CK(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(e_ == cudaErrorMemoryAllocation ? HJB_ERR_OOM : HJB_ERR_CUDA,       \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                          \
    } while (0)

#define TRY(expr)                \
    do {                         \
        int rc_ = (expr);        \
        if (rc_ != HJB_OK) return rc_; \
    } while (0)

// ----- TMA descriptor encoder from the driver (no link-time libcuda) --------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A caller-owned node field, read in place on the device or mirrored from
// host memory at every call.
struct Field {
    const void *user = nullptr;
    size_t bytes = 0;
    bool host = false;
    void *mirror = nullptr;

    void set(const void *p, size_t b) {
        user = p;
        bytes = b;
        host = p && !is_device_ptr(p);
    }
    const void *dev() const { return host ? mirror : user; }
    int refresh(cudaStream_t st) {
        if (!user || !host) return HJB_OK;
        if (!mirror) CK(cudaMalloc(&mirror, bytes));
        CK(cudaMemcpyAsync(mirror, user, bytes, cudaMemcpyHostToDevice, st));
        return HJB_OK;
    }
    void release() {
        if (mirror) cudaFree(mirror);
        mirror = nullptr;
    }
};

// Growable device allocation.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int ensure(size_t b) {
        if (b <= bytes && p) return HJB_OK;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        CK(cudaMalloc(&p, b));
        bytes = b;
        return HJB_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

// An output array: written in place when it is device memory, otherwise
// produced in a device staging buffer and copied back at the end.
struct OutArr {
    void *user = nullptr;
    size_t bytes = 0;
    bool host = false;
    DevBuf *stage = nullptr;
    int init(void *u, size_t b, DevBuf *s) {
        user = u;
        bytes = b;
        host = u && !is_device_ptr(u);
        stage = s;
        if (host) TRY(stage->ensure(b));
        return HJB_OK;
    }
    void *dev() const { return host ? stage->p : user; }
    int finish(cudaStream_t st) {
        if (user && host) CK(cudaMemcpyAsync(user, stage->p, bytes, cudaMemcpyDeviceToHost, st));
        return HJB_OK;
    }
};

// One launch of the convergence loop over a set of slots.
struct RunCtx {
    std::vector<SlotDesc> slots;
    DevBuf d_slots, d_state, d_ctl, vbuf, h_state_pinned, qlist, qflag;
    int qtiles = 0;  // tiles of all slots (queue capacity)
    int max_tiles = 0;
    SlotState *h_state = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    hjbh::SweepKey key{-1, -1, -1, -1, -1, -1, -1, -1, -1};
    int last_loop = 0;  // the last run used the cooperative loop kernel
    const uint32_t *diff = nullptr;  // decomposed solve: membership differences (twins)
    int local_iters = 1;             // applications of T per tile and sweep (2D)
    int near_start = 0;              // first queue: only tiles near a target (see queue_init)
    int li_in_graph = -1;
    int dyn_queue = 0;               // tile-queue sharing of this run (SweepArgs::dyn_queue)
    int dq_in_graph = -1;
    int spb = 0;
    const void *graph_slots = nullptr;
    const void *graph_q = nullptr;
    const void *graph_f = nullptr;
    int graph_nslots = -1;
    hjbk::ControlTable ctrl_in_graph;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        d_slots.release();
        d_state.release();
        d_ctl.release();
        vbuf.release();
        qlist.release();
        qflag.release();
        if (h_state) cudaFreeHost(h_state);
        h_state = nullptr;
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        ev0 = ev1 = nullptr;
    }
};

}  // namespace

struct hjb_problem {
    hjb_grid grid;
    int kind;
    double dubins_v;
    Field speed, current, log_speed, cost, labels, scale;
    double l_const, h, lambda, value_out;
    int weights = HJB_WEIGHTS_EXP;
    int interp = HJB_INTERP_Q1;
    int na, cdim;
    float ax[hjbk::MAX_CTRL], ay[hjbk::MAX_CTRL];
    int nb = 0;  // second player's set B (games), 0: none
    float bx[hjbk::MAX_CTRL], by[hjbk::MAX_CTRL];
    int ntargets;
    long long N;
    double dx[3];
    DevBuf speed_exp, trig;
    // coarse problem of the reconstruction
    DevBuf c_speed, c_current, c_cost, c_labels, c_trig, c_mask, c_vstage, c_grad, c_scale;
    DevBuf tile_bits, fine_mask_dev, scratch_u64;
    DevBuf tile_clear, c_tile_clear;  // per tile: no target node (fine grid, coarse grid)
    // re-splitting of the target components: labels (current, trial), the
    // trial's fine and coarse masks, counters and histograms
    DevBuf split_lab, split_fine, split_cl, split_small;
    // the last hjb_subdomains without re-splitting: its coarse auxiliary
    // solutions stay in `ra` for the coarse-to-fine warm start
    int ra_m = 0, ra_stride[3] = {1, 1, 1}, ra_wform = -1;
    DevBuf out_stage, out_stage2, out_stage3, in_stage;
    RunCtx full, ra, dec;
    RunCtx *batch = nullptr;
    // adjoint workspaces
    DevBuf adj_policy, adj_g, adj_L, adj_ctl, adj_v, adj_ref, adj_cell, adj_frac;
    cudaGraph_t adj_graph = nullptr;
    cudaGraphExec_t adj_exec = nullptr;
    cudaGraph_t ref_graph = nullptr;  // the refinement loop of hjb_backward
    cudaGraphExec_t ref_exec = nullptr;
    hjbh::AdjArgs ref_args_in_graph;
    int adj_apps_in_graph = 0, ref_apps_in_graph = 0;  // kernels of the cached loops
    hjbh::AdjArgs adj_args_in_graph;
    std::vector<const hjb_problem *> batch_key;
};

namespace {

// Step weights of the operator, beta I[V] + gamma l (hjb_discount.weights).
double beta_w(int weights, double lambda, double h) {
    return weights == HJB_WEIGHTS_IMPLICIT ? 1.0 / (1.0 + lambda * h) : std::exp(-lambda * h);
}
double gamma_w(int weights, double lambda, double h) {
    return weights == HJB_WEIGHTS_IMPLICIT ? h / (1.0 + lambda * h)
                                           : -std::expm1(-lambda * h) / lambda;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// Geometry of one slot's iteration buffers.

struct SlotGeo {
    int nx, ny, nz, pitch, zdup, nzl;
    long long zstride;
};

SlotGeo geo_of(int ndim, const int n[3], int periodic_z) {
    SlotGeo g;
    g.nx = n[0];
    g.ny = n[1];
    g.nz = ndim > 2 ? n[2] : 1;
    g.pitch = round_up(g.nx, 32);
    g.zdup = (ndim > 2 && periodic_z) ? 1 : 0;
    g.nzl = g.nz + 2 * g.zdup;
    g.zstride = static_cast<long long>(g.pitch) * g.ny;
    return g;
}

int encode_maps(SlotDesc &S, int ndim, int halo, int rows, int layers = hjbk::TZ) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(HJB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    for (int b = 0; b < 2; ++b) {
        CUresult r;
        if (ndim == 2) {
            cuuint64_t dims[2] = {static_cast<cuuint64_t>(S.nx), static_cast<cuuint64_t>(S.ny)};
            cuuint64_t strides[1] = {static_cast<cuuint64_t>(S.pitch) * 4};
            cuuint32_t box[2] = {static_cast<cuuint32_t>(hjbk::TW),
                                 static_cast<cuuint32_t>(rows + 2 * halo)};
            cuuint32_t es[2] = {1, 1};
            r = enc(&S.tmap[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, S.V[b], dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        } else {
            cuuint64_t dims[3] = {static_cast<cuuint64_t>(S.nx), static_cast<cuuint64_t>(S.ny),
                                  static_cast<cuuint64_t>(S.nz + 2 * S.zdup)};
            cuuint64_t strides[2] = {static_cast<cuuint64_t>(S.pitch) * 4,
                                     static_cast<cuuint64_t>(S.zstride) * 4};
            cuuint32_t box[3] = {static_cast<cuuint32_t>(hjbk::TW),
                                 static_cast<cuuint32_t>(hjbk::TY + 2 * halo),
                                 static_cast<cuuint32_t>(layers + 2)};
            cuuint32_t es[3] = {1, 1, 1};
            r = enc(&S.tmap[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, S.V[b], dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        }
        if (r != CUDA_SUCCESS) return fail(HJB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return HJB_OK;
}

// Per-call problem preparation: refresh host mirrors, exp(theta), and the
// largest foot displacement in cells (which selects the halo).
struct Prep {
    const float *speed = nullptr;
    const float *scale = nullptr;  // per-axis factors [N][2]
    const float *current = nullptr;
    const float *cost = nullptr;
    const uint8_t *labels = nullptr;
    double max_off_xy = 0.0;  // cells
    double max_off_z = 0.0;
    int launches = 0;         // kernels launched by prepare()
};

int prepare(hjb_problem *P, cudaStream_t st, Prep &out) {
    TRY(P->speed.refresh(st));
    TRY(P->current.refresh(st));
    TRY(P->log_speed.refresh(st));
    TRY(P->cost.refresh(st));
    TRY(P->labels.refresh(st));
    TRY(P->scale.refresh(st));
    out.scale = static_cast<const float *>(P->scale.dev());
    out.labels = static_cast<const uint8_t *>(P->labels.dev());
    out.cost = static_cast<const float *>(P->cost.dev());
    out.current = static_cast<const float *>(P->current.dev());
    if (P->log_speed.user) {
        TRY(P->speed_exp.ensure(P->N * sizeof(float)));
        hjbh::launch_exp(static_cast<const float *>(P->log_speed.dev()), P->speed_exp.as<float>(),
                         P->N, st);
        out.launches += 1;
        out.speed = P->speed_exp.as<float>();
    } else {
        out.speed = static_cast<const float *>(P->speed.dev());
    }
    if (P->kind == HJB_DYN_SPEED_CURRENT) {
        // largest control components, over the pairs a - b in a game
        double amax_x = 0, amax_y = 0;
        for (int k = 0; k < (P->nb ? P->nb : 1); ++k)
            for (int j = 0; j < P->na; ++j) {
                amax_x = std::fmax(amax_x, std::fabs(P->ax[j] - (P->nb ? P->bx[k] : 0.0f)));
                amax_y = std::fmax(amax_y, std::fabs(P->ay[j] - (P->nb ? P->by[k] : 0.0f)));
            }
        double sxmax = 1.0, symax = 1.0, cx = 0.0, cy = 0.0;
        if (out.speed || out.scale || out.current) {
            TRY(P->scratch_u64.ensure(64));
            unsigned *d = P->scratch_u64.as<unsigned>();
            CK(cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), st));
            if (out.speed) {
                hjbh::launch_absmax(out.speed, P->N, 1, 0, d, st);
                out.launches += 1;
            }
            if (out.scale) {
                hjbh::launch_absmax(out.scale, P->N, 2, 0, d, st);
                hjbh::launch_absmax(out.scale, P->N, 2, 1, d + 3, st);
                out.launches += 2;
            }
            if (out.current) {
                hjbh::launch_absmax(out.current, P->N, 2, 0, d + 1, st);
                hjbh::launch_absmax(out.current, P->N, 2, 1, d + 2, st);
                out.launches += 2;
            }
            unsigned h[4];
            CK(cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            float f[4];
            std::memcpy(f, h, sizeof f);
            if (out.speed) sxmax = symax = f[0];
            if (out.scale) {
                sxmax = f[0];
                symax = f[3];
            }
            cx = f[1];
            cy = f[2];
        }
        const double ox = (sxmax * amax_x + cx) * P->h / P->dx[0];
        const double oy = (symax * amax_y + cy) * P->h / P->dx[1];
        out.max_off_xy = std::fmax(ox, oy);
    } else {
        out.max_off_xy = std::fabs(P->dubins_v) * P->h / std::fmin(P->dx[0], P->dx[1]);
        double umax = 0;
        for (int j = 0; j < P->na; ++j) umax = std::fmax(umax, std::fabs(P->ax[j]));
        out.max_off_z = umax * P->h / P->dx[2];
    }
    return HJB_OK;
}

int halo_for(const hjb_problem *P, double max_off, double max_off_z, int *halo) {
    if (!std::isfinite(max_off) || !std::isfinite(max_off_z))
        return fail(HJB_ERR_INVALID_ARG, "a speed, log-speed or current field is not finite");
    // the cells reached by a foot displaced by up to M cells lie within
    // floor(M) + 1 nodes of the node
    const int need = static_cast<int>(std::floor(max_off)) + 1;
    if (P->kind == HJB_DYN_DUBINS) {
        if (need > 2 || max_off_z >= 1.0)
            return fail(HJB_ERR_UNSUPPORTED,
                        "Dubins feet move %.3f cells in (x,y) and %.3f in theta per step; the "
                        "3D sweep supports < 2 and < 1",
                        max_off, max_off_z);
        *halo = 2;
        return HJB_OK;
    }
    if (need <= 2)
        *halo = 2;
    else if (need <= 4)
        *halo = 4;
    else
        return fail(HJB_ERR_UNSUPPORTED,
                    "feet move up to %.3f cells per step; the sweep supports fewer than 4 (reduce h)",
                    max_off);
    return HJB_OK;
}

// Fill the fields of a slot that depend on the problem statement.
void fill_slot(SlotDesc &S, const hjb_problem *P, const SlotGeo &g, const Prep &pr, bool wform,
               double h, const double dx[3], int halo, double tol, int max_iters, int rows, int layers = hjbk::TZ) {
    const double beta = beta_w(P->weights, P->lambda, h);
    const double gamma = gamma_w(P->weights, P->lambda, h);
    const double c = P->l_const / P->lambda;
    S.nx = g.nx;
    S.ny = g.ny;
    S.nz = g.nz;
    S.pitch = g.pitch;
    S.zdup = g.zdup;
    S.zstride = g.zstride;
    S.tiles_x = (g.nx + hjbk::TX - 1) / hjbk::TX;
    S.tiles_y = (g.ny + rows - 1) / rows;
    S.tiles_z = P->grid.ndim > 2 ? (g.nz + layers - 1) / layers : 1;
    S.trows = rows;
    S.tlayers = P->grid.ndim > 2 ? layers : 1;
    S.ntiles = S.tiles_x * S.tiles_y * S.tiles_z;
    S.tile_bits = nullptr;
    S.tile_full = nullptr;
    S.tile_clear = nullptr;
    S.qbase = 0;
    S.halo = halo;
    S.hx = static_cast<float>(h / dx[0]);
    S.hy = static_cast<float>(h / dx[1]);
    S.hz = P->grid.ndim > 2 ? static_cast<float>(h / dx[2]) : 0.0f;
    S.beta = static_cast<float>(beta);
    S.gamma = static_cast<float>(gamma);
    S.gl = static_cast<float>(gamma * P->l_const);
    S.speed = pr.speed;
    S.scale2 = reinterpret_cast<const float2 *>(pr.scale);
    S.current = pr.current;
    S.cost = wform ? nullptr : pr.cost;
    S.labels = pr.labels;
    S.mask = nullptr;
    S.mask_bit = 0;
    S.only_target = 0;
    S.trig = nullptr;
    if (wform) {
        S.vout = static_cast<float>(c - P->value_out);
        S.vtarget = static_cast<float>(c);
    } else {
        S.vout = static_cast<float>(P->value_out);
        S.vtarget = 0.0f;
    }
    S.tol = static_cast<float>(tol);
    S.max_iters = max_iters;
}

int resolve_form(const hjb_problem *P, int use_w, bool *wform) {
    const bool const_cost = P->cost.user == nullptr;
    if (use_w < 0)
        *wform = const_cost;
    else if (use_w > 0) {
        if (!const_cost)
            return fail(HJB_ERR_INVALID_ARG, "use_w_form = 1 requires a constant cost (l == NULL)");
        *wform = true;
    } else
        *wform = false;
    return HJB_OK;
}

// Convergence loop driver: 0 = a CUDA-graph WHILE loop of one-sweep
// launches (default), 1 = one cooperative launch running every sweep with
// grid barriers.  HJB_LOOP=graph|coop selects it.
int loop_mode() {
    const char *e = std::getenv("HJB_LOOP");
    if (e && std::strcmp(e, "coop") == 0) return 1;
    return 0;
}

double default_tol(const hjb_problem *P, double h) {
    return 0.5e-4 * (1.0 - beta_w(P->weights, P->lambda, h));
}

// Dubins per-layer foot offsets (v h cos(th)/dx, v h sin(th)/dy) in FP64.
int dubins_trig(const hjb_problem *P, DevBuf &buf, int nz, double h, const double dx[3], double th0,
                double dth, cudaStream_t st) {
    std::vector<float2> t(nz);
    for (int k = 0; k < nz; ++k) {
        const double th = th0 + k * dth;
        t[k].x = static_cast<float>(P->dubins_v * h * std::cos(th) / dx[0]);
        t[k].y = static_cast<float>(P->dubins_v * h * std::sin(th) / dx[1]);
    }
    TRY(buf.ensure(nz * sizeof(float2)));
    CK(cudaMemcpyAsync(buf.p, t.data(), nz * sizeof(float2), cudaMemcpyHostToDevice, st));
    // the host vector dies at return: wait for the copy
    CK(cudaStreamSynchronize(st));
    return HJB_OK;
}

// The control vectors of the kernels.  In a game the entry k * na + j is
// the pair a_j - b_k, and the kernel takes the max over the nb blocks of the
// min within a block (the min over a for each b).
hjbk::ControlTable control_table(const hjb_problem *P) {
    hjbk::ControlTable c;
    std::memset(&c, 0, sizeof c);
    const int nb = P->nb ? P->nb : 1;
    c.count = P->na * nb;
    c.nb = nb;
    for (int k = 0; k < nb; ++k)
        for (int j = 0; j < P->na; ++j) {
            const float x = P->ax[j] - (P->nb ? P->bx[k] : 0.0f);
            const float y = P->ay[j] - (P->nb ? P->by[k] : 0.0f);
            c.ax[k * P->na + j] = x;
            c.ay[k * P->na + j] = y;
            c.a2[k * P->na + j] = make_float2(x, y);
        }
    return c;
}

// Kernel family for a problem: compile-time control counts (32, 64) only
// without a second player; a game runs the generic kernel with one control
// group (all pairs of a node in one thread) and 8-row tiles.
int key_na(const hjb_problem *P) {
    if (P->interp == HJB_INTERP_P1) return -1;  // generic count, P1 interpolation
    return P->nb ? 0 : P->na;
}
// Problems that run one control group in 8-row tiles (no tile-shape tuning).
bool fixed_shape(const hjb_problem *P) {
    return P->kind == HJB_DYN_DUBINS || P->nb || P->interp == HJB_INTERP_P1;
}

// Allocate iteration buffers for the slots (laid out back to back, each
// 256-byte aligned) and encode their TMA maps.
int alloc_slot_buffers(RunCtx &R, int ndim, int halo, int rows, int layers = hjbk::TZ) {
    // tile queues: one flag byte per tile per parity, lists of packed items
    int qt = 0, mt = 0;
    for (SlotDesc &S : R.slots) {
        S.qbase = qt;
        qt += S.ntiles;
        mt = S.ntiles > mt ? S.ntiles : mt;
    }
    if (qt >= (1 << 30)) return fail(HJB_ERR_INVALID_ARG, "too many tiles in one launch");
    R.qtiles = qt;
    R.max_tiles = mt;
    const size_t fb = (static_cast<size_t>(qt) + 3) / 4 * 4;
    TRY(R.qlist.ensure(2 * static_cast<size_t>(qt) * sizeof(int)));
    TRY(R.qflag.ensure(2 * fb));
    size_t total = 0;
    std::vector<size_t> off(R.slots.size());
    for (size_t i = 0; i < R.slots.size(); ++i) {
        const SlotDesc &S = R.slots[i];
        const size_t fl = static_cast<size_t>(S.nz + 2 * S.zdup) * S.zstride;
        off[i] = total;
        total += 2 * ((fl + 63) / 64 * 64);
    }
    TRY(R.vbuf.ensure(total * sizeof(float)));
    for (size_t i = 0; i < R.slots.size(); ++i) {
        SlotDesc &S = R.slots[i];
        const size_t fl = static_cast<size_t>(S.nz + 2 * S.zdup) * S.zstride;
        const size_t fl64 = (fl + 63) / 64 * 64;
        S.V[0] = R.vbuf.as<float>() + off[i];
        S.V[1] = R.vbuf.as<float>() + off[i] + fl64;
        TRY(encode_maps(S, ndim, halo, rows, layers));
    }
    return HJB_OK;
}

// Applications of T per tile and sweep pinned by the caller:
// opts->local_iters when positive, else HJB_LOCAL_ITERS, else 0 (not pinned:
// the autotuner's choice).  Clamped to 1..16.
int pinned_local_iters(const hjb_solve_opts *o) {
    static const int env = [] {
        const char *e = std::getenv("HJB_LOCAL_ITERS");
        return e ? std::atoi(e) : 0;
    }();
    const int v = (o && o->local_iters > 0) ? o->local_iters : (env > 0 ? env : 0);
    if (v <= 0) return 0;
    return v > 16 ? 16 : v;
}

// Applications of T per tile and sweep without a tuned choice: the pinned
// value, else 6, or 4 for a game, whose applications evaluate every (a, b)
// pair of controls, so that a longer stay on a tile costs more than the
// sweeps it saves (measured).
int local_iters(const hjb_solve_opts *o, const hjb_problem *P) {
    const int v = pinned_local_iters(o);
    if (v) return v;
    return (P && P->nb > 1) ? 4 : 6;
}

// How the CTAs of a sweep share its tile queue: by default the entries past
// each CTA's first one are handed out by a counter (items cost 1 to
// local_iters applications, so CTAs that drew cheap ones take more);
// HJB_QUEUE=static strides by the grid size instead.  Read at each solve.
int queue_mode() {
    const char *e = std::getenv("HJB_QUEUE");
    return (e && std::strcmp(e, "static") == 0) ? 0 : 1;
}

void set_queue_args(const RunCtx &R, hjbk::SweepArgs &a) {
    a.local_iters = R.local_iters;
    a.dyn_queue = R.dyn_queue;
    const size_t fb = (static_cast<size_t>(R.qtiles) + 3) / 4 * 4;
    a.qlist[0] = R.qlist.as<int>();
    a.qlist[1] = R.qlist.as<int>() + R.qtiles;
    a.qflag[0] = R.qflag.as<uint8_t>();
    a.qflag[1] = R.qflag.as<uint8_t>() + fb;
}

// Build (or reuse) the graph: a WHILE conditional node whose body runs
// `spb` sweeps; the last CTA of each sweep sets the loop condition.
int ensure_graph(RunCtx &R, const hjbh::SweepKey &key, int spb, const hjbk::ControlTable &ctrl,
                 float stall_tol) {
    const int n = static_cast<int>(R.slots.size());
    if (R.exec && R.key.dubins == key.dubins && R.key.wform == key.wform && R.key.na == key.na &&
        R.key.halo == key.halo && R.key.ty == key.ty && R.key.groups == key.groups &&
        R.key.lanes == key.lanes && R.key.layers == key.layers &&
        R.key.loop == key.loop && R.li_in_graph == R.local_iters &&
        R.dq_in_graph == R.dyn_queue &&
        R.spb == spb && R.graph_slots == R.d_slots.p &&
        R.graph_q == R.qlist.p && R.graph_f == R.qflag.p &&
        R.graph_nslots == n && std::memcmp(&R.ctrl_in_graph, &ctrl, sizeof ctrl) == 0)
        return HJB_OK;
    if (R.exec) cudaGraphExecDestroy(R.exec);
    if (R.graph) cudaGraphDestroy(R.graph);
    R.exec = nullptr;
    R.graph = nullptr;
    const void *fn = hjbh::sweep_kernel(key, nullptr);
    if (!fn) return fail(HJB_ERR_UNSUPPORTED, "no sweep kernel for this configuration");
    const int grid = hjbh::sweep_grid(key);
    CK(cudaGraphCreate(&R.graph, 0));
    cudaGraphConditionalHandle handle;
    CK(cudaGraphConditionalHandleCreate(&handle, R.graph, 1, cudaGraphCondAssignDefault));
    // (the params struct holds a union with non-trivial members: zeroed raw storage)
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, R.graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    hjbk::SweepArgs args;
    std::memset(&args, 0, sizeof args);
    args.slots = R.d_slots.as<SlotDesc>();
    args.state = R.d_state.as<SlotState>();
    args.ctl = R.d_ctl.as<Ctl>();
    set_queue_args(R, args);
    args.nslots = n;
    args.use_handle = 1;
    args.handle = handle;
    args.stall_tol = stall_tol;
    args.ctrl = ctrl;
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < spb; ++k) {
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof kp);
        kp.func = const_cast<void *>(fn);
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(hjbk::THREADS);
        kp.sharedMemBytes = 0;
        void *argv[1] = {&args};
        kp.kernelParams = argv;
        cudaGraphNode_t node;
        CK(cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
        prev = node;
    }
    CK(cudaGraphInstantiate(&R.exec, R.graph, 0));
    R.key = key;
    R.spb = spb;
    R.li_in_graph = R.local_iters;
    R.dq_in_graph = R.dyn_queue;
    R.graph_slots = R.d_slots.p;
    R.graph_q = R.qlist.p;
    R.graph_f = R.qflag.p;
    R.graph_nslots = n;
    R.ctrl_in_graph = ctrl;
    return HJB_OK;
}

int sweeps_per_body(const hjb_solve_opts *o) {
    if (o && o->sweeps_per_check > 0) return o->sweeps_per_check > 64 ? 64 : o->sweeps_per_check;
    return 8;
}

// Upload the slot table and allocate the state/control blocks.
int upload_slots(RunCtx &R, cudaStream_t st) {
    const size_t n = R.slots.size();
    TRY(R.d_slots.ensure(n * sizeof(SlotDesc)));
    TRY(R.d_state.ensure(n * sizeof(SlotState)));
    TRY(R.d_ctl.ensure(sizeof(Ctl)));
    if (!R.ev0) {
        CK(cudaEventCreate(&R.ev0));
        CK(cudaEventCreate(&R.ev1));
    }
    CK(cudaMemcpyAsync(R.d_slots.p, R.slots.data(), n * sizeof(SlotDesc), cudaMemcpyHostToDevice,
                       st));
    return HJB_OK;
}

// Run the convergence loop (graph), after init values and loop init.
int run_loop(RunCtx &R, const hjbh::SweepKey &key, int spb, const hjbk::ControlTable &ctrl,
             cudaStream_t st, int local = 1) {
    const int n = static_cast<int>(R.slots.size());
    R.local_iters = local;
    R.dyn_queue = queue_mode();
    hjbh::launch_loop_init(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), R.d_ctl.as<Ctl>(),
                           n, st, R.diff);
    {
        hjbk::SweepArgs qa;
        set_queue_args(R, qa);
        hjbh::launch_queue_init(R.d_slots.as<SlotDesc>(), n, R.max_tiles, R.d_ctl.as<Ctl>(),
                                qa.qlist[0], qa.qflag[0], qa.qflag[1], st, R.near_start);
        R.near_start = 0;
    }
    CK(cudaGetLastError());
    const float stall_tol = 8.0f * 1.1920929e-7f;
    R.last_loop = key.loop;
    if (key.loop) {
        // the whole loop in one cooperative launch (all CTAs co-resident)
        const void *fn = hjbh::sweep_kernel(key, nullptr);
        if (!fn) return fail(HJB_ERR_UNSUPPORTED, "no sweep kernel for this configuration");
        const int grid = hjbh::sweep_grid(key);
        hjbk::SweepArgs args;
        std::memset(&args, 0, sizeof args);
        args.slots = R.d_slots.as<SlotDesc>();
        args.state = R.d_state.as<SlotState>();
        args.ctl = R.d_ctl.as<Ctl>();
        set_queue_args(R, args);
        args.nslots = n;
        args.use_handle = 0;
        args.stall_tol = stall_tol;
        args.ctrl = ctrl;
        void *argv[1] = {&args};
        CK(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(hjbk::THREADS), argv, 0, st));
        return HJB_OK;
    }
    const char *ng = std::getenv("HJB_NO_GRAPH");
    if (ng && ng[0] == '1') {
        // host-driven loop (debugging aid): spb sweeps, then read nactive
        const void *fn = hjbh::sweep_kernel(key, nullptr);
        if (!fn) return fail(HJB_ERR_UNSUPPORTED, "no sweep kernel for this configuration");
        const int grid = hjbh::sweep_grid(key);
        hjbk::SweepArgs args;
        std::memset(&args, 0, sizeof args);
        args.slots = R.d_slots.as<SlotDesc>();
        args.state = R.d_state.as<SlotState>();
        args.ctl = R.d_ctl.as<Ctl>();
        set_queue_args(R, args);
        args.nslots = n;
        args.use_handle = 0;
        args.stall_tol = stall_tol;
        args.ctrl = ctrl;
        for (;;) {
            for (int k = 0; k < spb; ++k) {
                void *argv[1] = {&args};
                CK(cudaLaunchKernel(fn, dim3(grid), dim3(hjbk::THREADS), argv, 0, st));
            }
            int nact = 0, err = 0;
            CK(cudaMemcpyAsync(&nact, &R.d_ctl.as<Ctl>()->nactive, sizeof(int),
                               cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&err, &R.d_ctl.as<Ctl>()->error, sizeof(int), cudaMemcpyDeviceToHost,
                               st));
            CK(cudaStreamSynchronize(st));
            if (nact == 0 || err) break;
        }
        return HJB_OK;
    }
    TRY(ensure_graph(R, key, spb, ctrl, stall_tol));
    CK(cudaGraphLaunch(R.exec, st));
    return HJB_OK;
}

// Read back the slot states, the error flag and the number of sweep
// launches (synchronises the stream).
int read_state(RunCtx &R, cudaStream_t st, int *err, long long *launches = nullptr) {
    const size_t n = R.slots.size();
    if (!R.h_state || R.h_state_pinned.bytes < n * sizeof(SlotState)) {
        if (R.h_state) cudaFreeHost(R.h_state);
        R.h_state = nullptr;
        CK(cudaMallocHost(reinterpret_cast<void **>(&R.h_state), (n + 1) * sizeof(SlotState)));
        R.h_state_pinned.bytes = n * sizeof(SlotState);
    }
    CK(cudaMemcpyAsync(R.h_state, R.d_state.p, n * sizeof(SlotState), cudaMemcpyDeviceToHost, st));
    int *herr = reinterpret_cast<int *>(R.h_state + n);
    CK(cudaMemcpyAsync(herr, &R.d_ctl.as<Ctl>()->error, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    *err = herr[0];
    if (launches) *launches = R.last_loop ? 1 : static_cast<unsigned>(herr[1]);
    return HJB_OK;
}

void fill_stats(hjb_stats *s, const SlotState &st) {
    if (!s) return;
    std::memset(s, 0, sizeof *s);
    s->iterations = st.iters;
    s->converged = st.converged;
    s->node_updates = static_cast<long long>(st.updates);
    s->final_residual = st.final_res;
    s->tile_visits = static_cast<long long>(st.visits);
}

hjbh::GridDims dims_of(const hjb_problem *P) {
    hjbh::GridDims g;
    g.ndim = P->grid.ndim;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = d < g.ndim ? P->grid.n[d] : 1;
        g.periodic[d] = d < g.ndim ? P->grid.periodic[d] : 0;
    }
    return g;
}

int check_opts(const hjb_solve_opts *o) {
    if (o && o->max_iters < 0) return fail(HJB_ERR_INVALID_ARG, "max_iters < 0");
    if (o && o->n_subdomains > HJB_MAX_TARGETS)
        return fail(HJB_ERR_INVALID_ARG, "n_subdomains must be at most %d", HJB_MAX_TARGETS);
    if (o && o->subdomain_targets != HJB_SUBDOMAIN_TARGETS_ALL &&
        o->subdomain_targets != HJB_SUBDOMAIN_TARGETS_OWN)
        return fail(HJB_ERR_INVALID_ARG, "unknown subdomain_targets %d", o->subdomain_targets);
    return HJB_OK;
}

// ---------------------------------------------------------------------------
// Autotuner.  A choice is a point of the search space of the sweep:
//  - rows: 2D tile rows (tiles of 32 x 8, 32 x 4 or 32 x 2 nodes with 1, 2
//    or 4 control groups per node); fixed at 8 for the fixed-shape kernels
//    (Dubins, games, P1);
//  - li: applications of T per staged tile and sweep (small tiles follow a
//    narrow active front with less wasted work and finish an item sooner;
//    more applications per staging cross more of a tile per sweep but keep
//    a CTA longer on one item).
// The first call for a problem class runs the whole call once per candidate
// on the caller's data and keeps the fastest.  Choices live in a table keyed
// by the device and the problem class; the table is filled from the file
// HJB_TUNE_CACHE names (read and written) and from the tuning file shipped
// beside the library (read only; the choices measured for this library on
// its target GPU), and can be read and written through hjb_tune_get /
// hjb_tune_set / hjb_tune_load / hjb_tune_save.  HJB_TUNE=off never times:
// a call takes the table's choice or the fixed default, so repeated runs are
// bit-reproducible; HJB_TUNE=force times even when the table has a choice.
// HJB_TILE_ROWS=8|4|2 and HJB_LOCAL_ITERS (or hjb_solve_opts.local_iters)
// pin their axis.

struct Choice {
    int rows = 8;
    int lanes = 1;
    int li = 6;
    double ms = 0.0;
    int layers = hjbk::TZ;  // 3D: heading layers per tile (4 or 2)
};

std::mutex g_tune_mu;
std::map<std::string, Choice> g_tuned;
bool g_tune_files_read = false;

int forced_rows() {
    const char *e = std::getenv("HJB_TILE_ROWS");
    if (!e) return 0;
    const int r = std::atoi(e);
    return (r == 8 || r == 4 || r == 2) ? r : 0;
}

int forced_lanes() {
    const char *e = std::getenv("HJB_TILE_LANES");
    if (!e) return 0;
    const int l = std::atoi(e);
    return (l == 1 || l == 2) ? l : 0;
}

// The lane split (two lanes per node taking a_j and -a_j, 32 x 4 tiles)
// needs a control set whose second half is exactly the negated first half,
// one of the specialised control counts, Q1 and no second player.
bool lane_split_ok(const hjb_problem *P) {
    if (!P || P->nb || P->interp != HJB_INTERP_Q1 || P->kind != HJB_DYN_SPEED_CURRENT) return false;
    if (P->na != 32 && P->na != 64) return false;
    const int h = P->na / 2;
    for (int j = 0; j < h; ++j)
        if (P->ax[j + h] != -P->ax[j] || P->ay[j + h] != -P->ay[j]) return false;
    return true;
}

int tune_mode() {  // 0 off, 1 on (default), 2 force
    const char *e = std::getenv("HJB_TUNE");
    if (!e) return 1;
    if (std::strcmp(e, "off") == 0) return 0;
    if (std::strcmp(e, "force") == 0) return 2;
    return 1;
}

// Parse one cache line: {"key": "...", "rows": R, "local_iters": L, "ms": M}.
bool parse_tune_line(const std::string &line, std::string *key, Choice *c) {
    const size_t k0 = line.find("\"key\"");
    if (k0 == std::string::npos) return false;
    const size_t q0 = line.find('"', line.find(':', k0) + 1);
    const size_t q1 = q0 == std::string::npos ? q0 : line.find('"', q0 + 1);
    if (q1 == std::string::npos) return false;
    *key = line.substr(q0 + 1, q1 - q0 - 1);
    auto num = [&](const char *name, double *v) {
        const size_t a = line.find(name, q1);
        if (a == std::string::npos) return false;
        const size_t b = line.find(':', a);
        if (b == std::string::npos) return false;
        char *end = nullptr;
        *v = std::strtod(line.c_str() + b + 1, &end);
        return end != line.c_str() + b + 1;
    };
    double r = 0, l = 0, ms = 0, ln = 1, ly = hjbk::TZ;
    if (!num("\"rows\"", &r) || !num("\"local_iters\"", &l)) return false;
    num("\"ms\"", &ms);
    num("\"lanes\"", &ln);
    num("\"layers\"", &ly);
    if (!(ly == 4 || ly == 2)) return false;
    if (!(r == 8 || r == 4 || r == 2 || r == 1) || l < 1 || l > 16 ||
        !(ln == 1 || (ln == 2 && r == 4)))
        return false;
    c->rows = static_cast<int>(r);
    c->lanes = static_cast<int>(ln);
    c->layers = static_cast<int>(ly);
    c->li = static_cast<int>(l);
    c->ms = ms;
    return true;
}

// Merge the entries of a cache file into the table (caller holds the lock).
// Returns the number of entries read, or -1 if the file cannot be opened.
int load_tune_file(const char *path, bool overwrite) {
    FILE *f = std::fopen(path, "r");
    if (!f) return -1;
    int n = 0;
    char buf[1024];
    while (std::fgets(buf, sizeof buf, f)) {
        std::string key;
        Choice c;
        if (!parse_tune_line(buf, &key, &c)) continue;
        if (overwrite || !g_tuned.count(key)) g_tuned[key] = c;
        ++n;
    }
    std::fclose(f);
    return n;
}

int save_tune_file(const char *path) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "w");
    if (!f) return -1;
    std::fprintf(f, "[\n");
    size_t i = 0;
    for (const auto &kv : g_tuned) {
        std::fprintf(f,
                     "{\"key\": \"%s\", \"rows\": %d, \"lanes\": %d, \"layers\": %d, "
                     "\"local_iters\": %d, \"ms\": %.4f}%s\n",
                     kv.first.c_str(), kv.second.rows, kv.second.lanes, kv.second.layers,
                     kv.second.li, kv.second.ms, ++i < g_tuned.size() ? "," : "");
    }
    std::fprintf(f, "]\n");
    std::fclose(f);
    return std::rename(tmp.c_str(), path) == 0 ? 0 : -1;
}

// The tuning file shipped beside the library: <package>/tune_cache.json, one
// directory above the build directory that holds libhjb.so.
std::string shipped_tune_file() {
    Dl_info info;
    if (!dladdr(reinterpret_cast<void *>(&hjb_version), &info) || !info.dli_fname) return "";
    std::string so = info.dli_fname;
    const size_t a = so.rfind('/');
    if (a == std::string::npos) return "";
    const size_t b = so.rfind('/', a - 1);
    if (b == std::string::npos) return "";
    return so.substr(0, b) + "/tune_cache.json";
}

void read_tune_files() {  // caller holds the lock
    if (g_tune_files_read) return;
    g_tune_files_read = true;
    const std::string shipped = shipped_tune_file();
    if (!shipped.empty()) load_tune_file(shipped.c_str(), false);
    if (const char *e = std::getenv("HJB_TUNE_CACHE")) load_tune_file(e, true);
}

// Key of a problem class on the current device.
std::string tune_key(const char *op, const std::vector<long long> &cls) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    char name[256] = "unknown";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) std::snprintf(name, sizeof name, "%s", prop.name);
    for (char *c = name; *c; ++c)
        if (*c == '"' || *c == '\\' || *c == '|') *c = '_';
    std::string k = std::string(name) + "/" + std::to_string(sms) + "|" + op;
    for (long long v : cls) k += "|" + std::to_string(v);
    return k;
}

// Default choice when nothing is tuned: 32 x 8 tiles (the fixed shape of the
// 3D and generic kernels), the measured default applications per tile.
Choice default_choice(const hjb_problem *P) {
    Choice c;
    c.rows = hjbk::TY;
    c.li = local_iters(nullptr, P);
    return c;
}

// Run `run(choice, &ms)` with the table's choice for `key` when it is one of
// the candidates, otherwise (tuning on) time every candidate, keep the
// fastest and leave its outputs in place.  The first candidate is the
// default when tuning is off and the table has no choice.
template <typename Run>
int tuned_candidates(const std::string &key, const std::vector<Choice> &cand, Run run) {
    if (cand.empty()) return fail(HJB_ERR_UNSUPPORTED, "no candidate configuration");
    const int mode = tune_mode();
    Choice c = cand.front();
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        read_tune_files();
        auto it = g_tuned.find(key);
        if (it != g_tuned.end())
            for (const Choice &x : cand)
                if (x.rows == it->second.rows && x.lanes == it->second.lanes &&
                    x.li == it->second.li && x.layers == it->second.layers) {
                    c = it->second;
                    have = true;
                }
    }
    if (cand.size() == 1 || mode == 0 || (have && mode == 1)) return run(c, nullptr);
    std::vector<Choice> tried = cand;
    double best_ms = 1e300;
    size_t best = 0;
    int last_rc = HJB_OK;
    const bool verbose = std::getenv("HJB_TUNE_VERBOSE") != nullptr;
    for (size_t i = 0; i < tried.size(); ++i) {
        double ms = 0;
        const int rc = run(tried[i], &ms);
        if (rc != HJB_OK && rc != HJB_ERR_NOT_CONVERGED) return rc;
        last_rc = rc;
        tried[i].ms = ms;
        if (verbose)
            std::fprintf(stderr, "hjb tune %s: rows %d lanes %d layers %d li %d: %.4f ms\n",
                         key.c_str(), tried[i].rows, tried[i].lanes, tried[i].layers, tried[i].li, ms);
        if (ms < best_ms) {
            best_ms = ms;
            best = i;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = tried[best];
        if (const char *e = std::getenv("HJB_TUNE_CACHE")) save_tune_file(e);
    }
    return best + 1 == tried.size() ? last_rc : run(tried[best], nullptr);
}

// Run `run(choice, &ms)` with the tuned choice for `key`, tuning it first
// when needed.  fixed_rows: the kernel family has one tile shape; li_fixed:
// the caller (opts or HJB_LOCAL_ITERS) pinned the applications per tile.
template <typename Run>
int tuned_call(const std::string &key_class, const hjb_problem *P, bool fixed_rows, int li_pinned,
               Run run) {
    const int mode = tune_mode();
    // a caller that pins the applications per tile tunes (and finds) the
    // tile shape for that value only, under a key of its own
    const std::string key = li_pinned ? key_class + "|li" + std::to_string(li_pinned) : key_class;
    const int frows = fixed_rows ? hjbk::TY : forced_rows();
    const int flanes = fixed_rows ? 1 : forced_lanes();
    Choice c = default_choice(P);
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        read_tune_files();
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            c = it->second;
            have = true;
        }
    }
    if (frows) c.rows = frows;
    if (flanes) c.lanes = flanes;
    if (li_pinned) c.li = li_pinned;
    if (c.lanes == 2 && (c.rows != 4 || !lane_split_ok(P))) c.lanes = 1;
    const bool all_pinned = frows && flanes && li_pinned && !(P && P->kind == HJB_DYN_DUBINS);
    if (mode == 0 || all_pinned || (have && mode == 1)) return run(c, nullptr);
    std::vector<Choice> cand;
    const bool game = P && P->nb > 1;
    const int li_c[3] = {game ? 2 : 4, game ? 4 : 6, game ? 6 : 8};
    if (P && P->kind == HJB_DYN_DUBINS) {
        // 3D: tiles of 4 or 2 heading layers x applications per tile
        for (int ly : {4, 2})
            for (int l : li_c) {
                if (li_pinned && l != li_pinned) continue;
                cand.push_back(Choice{hjbk::TY, 1, l, 0.0, ly});
            }
        if (li_pinned && cand.empty())
            for (int ly : {4, 2}) cand.push_back(Choice{hjbk::TY, 1, li_pinned, 0.0, ly});
    }
    // tile shapes (rows, lanes) x applications per tile
    const int shapes[4][2] = {{8, 1}, {4, 1}, {4, 2}, {2, 1}};
    for (const auto &sh : shapes) {
        if (P && P->kind == HJB_DYN_DUBINS) break;
        if (frows && sh[0] != frows) continue;
        if (flanes && sh[1] != flanes) continue;
        if (sh[1] == 2 && !lane_split_ok(P)) continue;
        for (int l : li_c) {
            if (li_pinned && l != li_pinned) continue;
            Choice x;
            x.rows = sh[0];
            x.lanes = sh[1];
            x.li = l;
            cand.push_back(x);
        }
        if (li_pinned && (cand.empty() || cand.back().rows != sh[0] || cand.back().lanes != sh[1])) {
            Choice x;
            x.rows = sh[0];
            x.lanes = sh[1];
            x.li = li_pinned;
            cand.push_back(x);
        }
    }
    if (cand.empty()) return run(c, nullptr);
    double best_ms = 1e300;
    size_t best = 0;
    int last_rc = HJB_OK;
    const bool verbose = std::getenv("HJB_TUNE_VERBOSE") != nullptr;
    for (size_t i = 0; i < cand.size(); ++i) {
        double ms = 0;
        const int rc = run(cand[i], &ms);
        if (rc != HJB_OK && rc != HJB_ERR_NOT_CONVERGED) return rc;
        last_rc = rc;
        cand[i].ms = ms;
        if (verbose)
            std::fprintf(stderr, "hjb tune %s: rows %d lanes %d layers %d li %d: %.4f ms\n",
                         key.c_str(), cand[i].rows, cand[i].lanes, cand[i].layers, cand[i].li, ms);
        if (ms < best_ms) {
            best_ms = ms;
            best = i;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = cand[best];
        if (const char *e = std::getenv("HJB_TUNE_CACHE")) save_tune_file(e);
    }
    // the outputs of the last candidate are in place when it won
    return best + 1 == cand.size() ? last_rc : run(cand[best], nullptr);
}

}  // namespace

// ===========================================================================
// C ABI

extern "C" {

const char *hjb_last_error(void) { return g_err.c_str(); }

const char *hjb_version(void) { return "hjb-gb300 0.1 (sm_103a)"; }

int hjb_tune_get(const char *key, hjb_tune_choice *out) {
    g_err.clear();
    if (!key || !out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    read_tune_files();
    auto it = g_tuned.find(key);
    if (it == g_tuned.end()) return fail(HJB_ERR_INVALID_ARG, "no tuned choice for this key");
    out->tile_rows = it->second.rows;
    out->lanes = it->second.lanes;
    out->layers = it->second.layers;
    out->local_iters = it->second.li;
    out->ms = it->second.ms;
    return HJB_OK;
}

int hjb_tune_set(const char *key, const hjb_tune_choice *c) {
    g_err.clear();
    if (!key || !c) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!(c->tile_rows == 8 || c->tile_rows == 4 || c->tile_rows == 2 || c->tile_rows == 1) ||
        c->local_iters < 1 || c->local_iters > 16 ||
        !(c->lanes == 1 || (c->lanes == 2 && c->tile_rows == 4)) ||
        !(c->layers == 4 || c->layers == 2))
        return fail(HJB_ERR_INVALID_ARG,
                    "tile_rows must be 8, 4, 2 (or 1: the reconstruction's on-chip solve), lanes "
                    "1 (or 2 with 4 rows), layers 4 or 2 and local_iters 1..16");
    if (std::strchr(key, '"') || std::strchr(key, '\\') || std::strchr(key, '\n'))
        return fail(HJB_ERR_INVALID_ARG, "a key may not hold quotes, backslashes or newlines");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    read_tune_files();
    Choice x;
    x.rows = c->tile_rows;
    x.lanes = c->lanes;
    x.layers = c->layers;
    x.li = c->local_iters;
    x.ms = c->ms;
    g_tuned[key] = x;
    return HJB_OK;
}

int hjb_tune_load(const char *path, int *entries) {
    g_err.clear();
    if (!path) return fail(HJB_ERR_INVALID_ARG, "NULL path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    read_tune_files();
    const int n = load_tune_file(path, true);
    if (n < 0) return fail(HJB_ERR_INVALID_ARG, "cannot open %s", path);
    if (entries) *entries = n;
    return HJB_OK;
}

int hjb_tune_save(const char *path) {
    g_err.clear();
    if (!path) return fail(HJB_ERR_INVALID_ARG, "NULL path");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    read_tune_files();
    if (save_tune_file(path) != 0) return fail(HJB_ERR_INVALID_ARG, "cannot write %s", path);
    return HJB_OK;
}

int hjb_tune_clear(void) {
    g_err.clear();
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    g_tune_files_read = true;  // an explicit clear also drops the files' entries
    return HJB_OK;
}

int hjb_create(const hjb_grid *grid, const hjb_dynamics *dyn, const hjb_cost *cost,
               const hjb_discount *disc, const hjb_controls *controls, const hjb_target *target,
               hjb_problem **out) {
    g_err.clear();
    if (!grid || !dyn || !cost || !disc || !controls || !target || !out)
        return fail(HJB_ERR_INVALID_ARG, "NULL descriptor");
    *out = nullptr;
    if (grid->ndim != 2 && grid->ndim != 3) return fail(HJB_ERR_INVALID_ARG, "ndim must be 2 or 3");
    long long N = 1;
    for (int d = 0; d < grid->ndim; ++d) {
        const int n = grid->n[d];
        if (n < 2) return fail(HJB_ERR_INVALID_ARG, "n[%d] = %d < 2", d, n);
        if (!(grid->hi[d] > grid->lo[d])) return fail(HJB_ERR_INVALID_ARG, "hi[%d] <= lo[%d]", d, d);
        N *= n;
    }
    if (grid->n[0] > 65536 || grid->n[1] > 65536 || (grid->ndim > 2 && grid->n[2] > 65536))
        return fail(HJB_ERR_INVALID_ARG, "grid too large");
    if (N > (1LL << 31)) return fail(HJB_ERR_INVALID_ARG, "more than 2^31 nodes");
    {
        // tiles at the smallest shape the sweep may run (32 x 2 in 2D, 32 x 8 x 2 in 3D):
        // a work-queue entry holds a tile index in 22 bits
        const long long tx = (grid->n[0] + hjbk::TX - 1) / hjbk::TX;
        const long long tiles = grid->ndim == 2
                                    ? tx * ((grid->n[1] + 1) / 2)
                                    : tx * ((grid->n[1] + hjbk::TY - 1) / hjbk::TY) *
                                          ((grid->n[2] + 1) / 2);
        if (tiles > HJB_MAX_TILES)
            return fail(HJB_ERR_UNSUPPORTED, "the grid has %lld tiles, more than the %d a problem "
                        "may hold", tiles, HJB_MAX_TILES);
    }
    if (dyn->kind == HJB_DYN_SPEED_CURRENT) {
        if (grid->ndim != 2) return fail(HJB_ERR_UNSUPPORTED, "speed/current dynamics are 2D");
        if (grid->periodic[0] || grid->periodic[1])
            return fail(HJB_ERR_UNSUPPORTED, "periodic dimensions are supported for theta (Dubins) only");
        if (controls->dim != 2) return fail(HJB_ERR_INVALID_ARG, "controls must be 2D vectors");
        if ((dyn->speed ? 1 : 0) + (dyn->log_speed ? 1 : 0) + (dyn->scale ? 1 : 0) > 1)
            return fail(HJB_ERR_INVALID_ARG, "give one of speed, log_speed and scale");
    } else if (dyn->kind == HJB_DYN_DUBINS) {
        if (grid->ndim != 3 || !grid->periodic[2] || grid->periodic[0] || grid->periodic[1])
            return fail(HJB_ERR_INVALID_ARG, "Dubins needs a 3D grid, periodic in dimension 2 only");
        if (controls->dim != 1) return fail(HJB_ERR_INVALID_ARG, "Dubins controls are scalars");
        if (dyn->speed || dyn->current || dyn->log_speed || dyn->scale)
            return fail(HJB_ERR_UNSUPPORTED, "Dubins takes no node fields");
        if (controls->count_b)
            return fail(HJB_ERR_UNSUPPORTED, "games are supported for 2D speed/current dynamics");
    } else {
        return fail(HJB_ERR_INVALID_ARG, "unknown dynamics kind %d", dyn->kind);
    }
    if (controls->count < 1 || controls->count > HJB_MAX_CONTROLS || !controls->a)
        return fail(HJB_ERR_INVALID_ARG, "control count must be in [1, %d]", HJB_MAX_CONTROLS);
    for (int j = 0; j < controls->count * controls->dim; ++j)
        if (!std::isfinite(controls->a[j]) || std::fabs(controls->a[j]) > 1e6f)
            return fail(HJB_ERR_INVALID_ARG, "control component %d is not a finite value", j);
    if (controls->count_b < 0 || (controls->count_b > 0 && !controls->b) ||
        controls->count * (controls->count_b > 0 ? controls->count_b : 1) > HJB_MAX_CONTROLS)
        return fail(HJB_ERR_INVALID_ARG,
                    "the second player's set needs count_b >= 0 vectors and count * count_b <= %d",
                    HJB_MAX_CONTROLS);
    for (int j = 0; j < controls->count_b * controls->dim; ++j)
        if (!std::isfinite(controls->b[j]) || std::fabs(controls->b[j]) > 1e6f)
            return fail(HJB_ERR_INVALID_ARG, "component %d of the second player's set is not finite", j);
    if (!std::isfinite(dyn->dubins_v) || !std::isfinite(disc->h) || !std::isfinite(disc->lambda) ||
        !std::isfinite(target->value_out) || !std::isfinite(cost->l_const))
        return fail(HJB_ERR_INVALID_ARG, "non-finite scalar parameter");
    if (!(disc->h > 0) || !(disc->lambda > 0))
        return fail(HJB_ERR_INVALID_ARG, "h and lambda must be positive");
    if (disc->weights != HJB_WEIGHTS_EXP && disc->weights != HJB_WEIGHTS_IMPLICIT)
        return fail(HJB_ERR_INVALID_ARG, "unknown step weights %d", disc->weights);
    if (disc->interp != HJB_INTERP_Q1 && disc->interp != HJB_INTERP_P1)
        return fail(HJB_ERR_INVALID_ARG, "unknown interpolation %d", disc->interp);
    if (disc->interp == HJB_INTERP_P1 && dyn->kind != HJB_DYN_SPEED_CURRENT)
        return fail(HJB_ERR_UNSUPPORTED, "P1 interpolation is implemented for 2D problems");
    if (!target->labels) return fail(HJB_ERR_INVALID_ARG, "target labels are required");
    if (target->n_targets < 1 || target->n_targets > HJB_MAX_TARGETS)
        return fail(HJB_ERR_INVALID_ARG, "n_targets must be in [1, %d]", HJB_MAX_TARGETS);
    if (!cost->l && !(cost->l_const > 0))
        return fail(HJB_ERR_INVALID_ARG, "constant running cost must be positive");
    hjb_problem *P = new hjb_problem();
    P->grid = *grid;
    for (int d = grid->ndim; d < 3; ++d) {
        P->grid.n[d] = 1;
        P->grid.periodic[d] = 0;
        P->grid.lo[d] = 0;
        P->grid.hi[d] = 1;
    }
    P->kind = dyn->kind;
    P->dubins_v = dyn->dubins_v;
    P->N = N;
    P->speed.set(dyn->speed, N * sizeof(float));
    P->current.set(dyn->current, 2 * N * sizeof(float));
    P->log_speed.set(dyn->log_speed, N * sizeof(float));
    P->scale.set(dyn->scale, 2 * N * sizeof(float));
    P->cost.set(cost->l, N * sizeof(float));
    P->labels.set(target->labels, N);
    P->l_const = cost->l ? 1.0 : cost->l_const;
    P->h = disc->h;
    P->lambda = disc->lambda;
    P->weights = disc->weights;
    P->interp = disc->interp;
    P->value_out = target->value_out;
    P->ntargets = target->n_targets;
    P->na = controls->count;
    P->cdim = controls->dim;
    for (int j = 0; j < P->na; ++j) {
        P->ax[j] = controls->a[j * controls->dim];
        P->ay[j] = controls->dim > 1 ? controls->a[j * controls->dim + 1] : 0.0f;
    }
    P->nb = controls->count_b;
    for (int k = 0; k < P->nb; ++k) {
        P->bx[k] = controls->b[k * controls->dim];
        P->by[k] = controls->dim > 1 ? controls->b[k * controls->dim + 1] : 0.0f;
    }
    for (int d = 0; d < 3; ++d)
        P->dx[d] = P->grid.periodic[d] ? (P->grid.hi[d] - P->grid.lo[d]) / P->grid.n[d]
                                       : (P->grid.hi[d] - P->grid.lo[d]) / (P->grid.n[d] - 1);
    *out = P;
    return HJB_OK;
}

int hjb_destroy(hjb_problem *P) {
    if (!P) return HJB_OK;
    P->full.release();
    P->ra.release();
    P->dec.release();
    if (P->batch) {
        P->batch->release();
        delete P->batch;
    }
    if (P->adj_exec) cudaGraphExecDestroy(P->adj_exec);
    if (P->adj_graph) cudaGraphDestroy(P->adj_graph);
    if (P->ref_exec) cudaGraphExecDestroy(P->ref_exec);
    if (P->ref_graph) cudaGraphDestroy(P->ref_graph);
    P->adj_policy.release();
    P->adj_g.release();
    P->adj_L.release();
    P->adj_ctl.release();
    P->adj_ref.release();
    P->adj_cell.release();
    P->adj_frac.release();
    P->adj_v.release();
    DevBuf *bufs[] = {&P->speed_exp, &P->trig,     &P->c_speed,      &P->c_current,
                      &P->c_cost,    &P->c_labels, &P->c_trig,       &P->c_mask,
                      &P->c_vstage,  &P->c_grad,   &P->tile_bits, &P->c_scale,
                      &P->fine_mask_dev, &P->scratch_u64, &P->out_stage, &P->out_stage2,
                      &P->split_lab, &P->split_fine, &P->split_cl, &P->split_small,
                      &P->tile_clear, &P->c_tile_clear,
                      &P->out_stage3, &P->in_stage};
    for (DevBuf *b : bufs) b->release();
    P->speed.release();
    P->current.release();
    P->log_speed.release();
    P->cost.release();
    P->labels.release();
    P->scale.release();
    delete P;
    return HJB_OK;
}

}  // extern "C"

namespace {

int solve_full(hjb_problem *P, const hjb_solve_opts *opts, const Choice &ch, float *v_out,
               hjb_stats *stats, cudaStream_t st) {
    const int rows = ch.rows, li = ch.li;
    bool wform;
    TRY(resolve_form(P, opts ? opts->use_w_form : -1, &wform));
    Prep pr;
    TRY(prepare(P, st, pr));
    int halo;
    TRY(halo_for(P, pr.max_off_xy, pr.max_off_z, &halo));
    const double tol = (opts && opts->tol > 0) ? opts->tol : default_tol(P, P->h);
    const int max_iters = (opts && opts->max_iters > 0) ? opts->max_iters : 100000;
    RunCtx &R = P->full;
    const SlotGeo g = geo_of(P->grid.ndim, P->grid.n, P->grid.periodic[2]);
    R.slots.assign(1, SlotDesc());
    std::memset(R.slots.data(), 0, sizeof(SlotDesc));
    fill_slot(R.slots[0], P, g, pr, wform, P->h, P->dx, halo, tol, max_iters, rows, ch.layers);
    TRY(P->tile_clear.ensure(R.slots[0].ntiles));
    hjbh::launch_tile_clear(dims_of(P), R.slots[0].tiles_x, R.slots[0].tiles_y, R.slots[0].tiles_z,
                            rows, ch.layers, pr.labels, P->tile_clear.as<uint8_t>(), st);
    R.slots[0].tile_clear = P->tile_clear.as<uint8_t>();
    if (P->kind == HJB_DYN_DUBINS) {
        TRY(dubins_trig(P, P->trig, g.nz, P->h, P->dx, P->grid.lo[2], P->dx[2], st));
        R.slots[0].trig = P->trig.as<float2>();
    }
    TRY(alloc_slot_buffers(R, P->grid.ndim, halo, rows, ch.layers));
    TRY(upload_slots(R, st));
    OutArr out;
    TRY(out.init(v_out, P->N * sizeof(float), &P->out_stage));
    const float *vinit = nullptr;
    if (opts && opts->v_init) {
        if (is_device_ptr(opts->v_init)) {
            vinit = opts->v_init;
        } else {
            TRY(P->in_stage.ensure(P->N * sizeof(float)));
            CK(cudaMemcpyAsync(P->in_stage.p, opts->v_init, P->N * sizeof(float),
                               cudaMemcpyHostToDevice, st));
            vinit = P->in_stage.as<float>();
        }
    }
    const float c_over = static_cast<float>(P->l_const / P->lambda);
    CK(cudaEventRecord(R.ev0, st));
    hjbh::launch_init_values(R.d_slots.as<SlotDesc>(), 1, static_cast<int>(P->N), wform, c_over,
                             vinit, st);
    const hjbh::SweepKey key{P->kind == HJB_DYN_DUBINS ? 1 : 0, wform ? 1 : 0, key_na(P), halo, rows,
                             8 / rows / ch.lanes, loop_mode(), ch.lanes,
                             P->grid.ndim > 2 ? ch.layers : 1};
    const hjbk::ControlTable ctrl = control_table(P);
    // from W = 0 with a zero outside value only tiles near a target change in
    // the first sweep (T(0) = 0 elsewhere): queue just those
    R.near_start = wform && !vinit && R.slots[0].vout == 0.0f;
    TRY(run_loop(R, key, sweeps_per_body(opts), ctrl, st, li));
    hjbh::launch_extract(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), 0,
                         static_cast<float *>(out.dev()), wform, c_over, st);
    CK(cudaEventRecord(R.ev1, st));
    TRY(out.finish(st));
    int err = 0;
    long long sweeps = 0;
    TRY(read_state(R, st, &err, &sweeps));
    CK(cudaGetLastError());
    float ms = 0;
    cudaEventElapsedTime(&ms, R.ev0, R.ev1);
    if (stats) {
        fill_stats(stats, R.h_state[0]);
        stats->ms = ms;
        stats->launches = pr.launches + 5 + sweeps;
        stats->tile_rows = P->grid.ndim == 2 ? rows : 0;
        stats->tile_lanes = ch.lanes;
        stats->tile_layers = P->grid.ndim > 2 ? ch.layers : 0;
        stats->local_iters = R.local_iters;
    }
    if (err) return fail(HJB_ERR_TIMEOUT, "a bounded device wait gave up (TMA transfer lost)");
    if (!R.h_state[0].converged)
        return fail(HJB_ERR_NOT_CONVERGED, "not converged after %d iterations (residual %g)",
                    R.h_state[0].iters, R.h_state[0].final_res);
    return HJB_OK;
}

}  // namespace

extern "C" {

int hjb_solve(hjb_problem *P, const hjb_solve_opts *opts, float *v_out, hjb_stats *stats,
              void *stream) {
    g_err.clear();
    if (!P || !v_out) return fail(HJB_ERR_INVALID_ARG, "NULL problem or output");
    TRY(check_opts(opts));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::string key = tune_key("full", {P->kind, P->grid.n[0], P->grid.n[1], P->grid.n[2],
                                              P->na, P->nb, P->interp, P->cost.user ? 1 : 0});
    return tuned_call(key, P, fixed_shape(P), pinned_local_iters(opts), [&](Choice c, double *ms) {
        hjb_stats tmp;
        hjb_stats *sp = stats ? stats : &tmp;
        const int rc = solve_full(P, opts, c, v_out, sp, st);
        if (ms) *ms = sp->ms;
        return rc;
    });
}

}  // extern "C"

namespace {

// RA (Sec. 3, steps 1-3) and the projection (ISA step 2) for a division of
// the target into m components given by comp_labels (device [N], 0 free,
// k = component k; NULL: the problem's labels).  delta_in >= 0 is the
// threshold; < 0 derives it from ra (eq. rep).  fine_dev [N] and cl_dev
// [N_K] receive the fine and coarse sub-domain bits (device), vaux_dev
// [m][N_K] (optional) the auxiliary solutions; stats as for hjb_subdomains.
int ra_division(hjb_problem *P, const hjb_ra_opts *ra, const uint8_t *comp_labels, int m,
                double delta_in, uint32_t *fine_dev, uint32_t *cl_dev, float *vaux_dev,
                hjb_stats *stats, cudaStream_t st) {
    const int nd = P->grid.ndim;
    hjbh::GridDims fine = dims_of(P), coarse = fine;
    int stride[3] = {1, 1, 1};
    for (int d = 0; d < nd; ++d) {
        const int r = ra->coarse_stride[d];
        if (r < 1) return fail(HJB_ERR_INVALID_ARG, "coarse_stride[%d] < 1", d);
        stride[d] = r;
        if (fine.periodic[d]) {
            if (fine.n[d] % r) return fail(HJB_ERR_INVALID_ARG, "stride %d does not divide n[%d]", r, d);
            coarse.n[d] = fine.n[d] / r;
        } else {
            if ((fine.n[d] - 1) % r)
                return fail(HJB_ERR_INVALID_ARG, "stride %d does not divide n[%d]-1", r, d);
            coarse.n[d] = (fine.n[d] - 1) / r + 1;
        }
        if (coarse.n[d] < 2) return fail(HJB_ERR_INVALID_ARG, "coarse grid has < 2 nodes in dim %d", d);
    }
    const long long NK = static_cast<long long>(coarse.n[0]) * coarse.n[1] * coarse.n[2];
    const double hK = ra->h_coarse > 0 ? ra->h_coarse : P->h * stride[0];
    double dxK[3];
    for (int d = 0; d < 3; ++d) dxK[d] = P->dx[d] * stride[d];
    bool wform;
    TRY(resolve_form(P, -1, &wform));
    Prep pr;
    TRY(prepare(P, st, pr));
    // coarse fields
    TRY(P->c_labels.ensure(NK));
    if (pr.speed) TRY(P->c_speed.ensure(NK * sizeof(float)));
    if (pr.current) TRY(P->c_current.ensure(2 * NK * sizeof(float)));
    if (pr.cost) TRY(P->c_cost.ensure(NK * sizeof(float)));
    if (pr.scale) TRY(P->c_scale.ensure(2 * NK * sizeof(float)));
    hjbh::launch_gather_coarse(fine, coarse, stride, pr.speed, pr.current, pr.cost,
                               comp_labels ? comp_labels : pr.labels,
                               pr.scale, P->c_speed.as<float>(), P->c_current.as<float>(),
                               P->c_cost.as<float>(), P->c_labels.as<uint8_t>(),
                               P->c_scale.as<float>(), st);
    Prep cp = pr;
    cp.speed = pr.speed ? P->c_speed.as<float>() : nullptr;
    cp.scale = pr.scale ? P->c_scale.as<float>() : nullptr;
    cp.current = pr.current ? P->c_current.as<float>() : nullptr;
    cp.cost = pr.cost ? P->c_cost.as<float>() : nullptr;
    cp.labels = P->c_labels.as<uint8_t>();
    // the displacement in cells scales with h_K / dx_K
    const double scale = (hK / dxK[0]) / (P->h / P->dx[0]);
    int halo;
    TRY(halo_for(P, pr.max_off_xy * scale, pr.max_off_z * (hK / dxK[2 < nd ? 2 : 0]) /
                                               (P->h / P->dx[2 < nd ? 2 : 0]),
                 &halo));
    const double tol = ra->tol > 0 ? ra->tol : default_tol(P, hK);
    const int max_iters = ra->max_iters > 0 ? ra->max_iters : 100000;
    RunCtx &R = P->ra;
    const SlotGeo g = geo_of(nd, coarse.n, coarse.periodic[2]);
    R.slots.assign(m, SlotDesc());
    std::memset(R.slots.data(), 0, m * sizeof(SlotDesc));
    if (P->kind == HJB_DYN_DUBINS)
        TRY(dubins_trig(P, P->c_trig, g.nz, hK, dxK, P->grid.lo[2], dxK[2], st));
    const float c_over = static_cast<float>(P->l_const / P->lambda);
    // RA step 1 on a 2D coarse grid that fits on chip may run as one
    // thread-block cluster per auxiliary problem, solving it to convergence in
    // shared memory (tuned choice rows = 1), otherwise as the tile-queue sweep
    // of every auxiliary problem in one launch.  HJB_RA=tiles|chip pins the
    // path.
    const char *ra_env = std::getenv("HJB_RA");
    const bool chip_fits = nd == 2 && hjbh::coarse_fits(coarse.n[0], coarse.n[1], halo, nullptr,
                                                        nullptr, nullptr);
    bool on_chip = false;
    auto coarse_solve = [&](Choice c, double *ms) -> int {
        on_chip = c.rows == 1;
        const int rows = on_chip ? 2 : c.rows;
        R.slots.assign(m, SlotDesc());
        std::memset(R.slots.data(), 0, m * sizeof(SlotDesc));
        if (!on_chip) {
            const int ctx = (g.nx + hjbk::TX - 1) / hjbk::TX, cty = (g.ny + rows - 1) / rows;
            const int ctz = nd > 2 ? (g.nz + hjbk::TZ - 1) / hjbk::TZ : 1;
            TRY(P->c_tile_clear.ensure(static_cast<size_t>(ctx) * cty * ctz));
            hjbh::launch_tile_clear(coarse, ctx, cty, ctz, rows, hjbk::TZ, P->c_labels.as<uint8_t>(),
                                    P->c_tile_clear.as<uint8_t>(), st);
        }
        for (int k = 0; k < m; ++k) {
            fill_slot(R.slots[k], P, g, cp, wform, hK, dxK, halo, tol, max_iters, rows);
            if (!on_chip) R.slots[k].tile_clear = P->c_tile_clear.as<uint8_t>();
            R.slots[k].only_target = k + 1;  // RA step 1: dG := X_k
            if (P->kind == HJB_DYN_DUBINS) R.slots[k].trig = P->c_trig.as<float2>();
        }
        TRY(alloc_slot_buffers(R, nd, halo, rows));
        TRY(upload_slots(R, st));
        CK(cudaEventRecord(R.ev0, st));
        if (on_chip) {
            hjbh::launch_loop_init(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(),
                                   R.d_ctl.as<Ctl>(), m, st);
            const int crc = hjbh::launch_coarse_solve(
                R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), m, coarse.n[0], coarse.n[1],
                halo, P->interp, wform ? 1 : 0, control_table(P), 8.0f * 1.1920929e-7f, st);
            if (crc)
                return fail(HJB_ERR_CUDA, "launch of the on-chip coarse solve failed: %s",
                            cudaGetErrorString(cudaGetLastError()));
            R.last_loop = 1;
            R.local_iters = 1;
        } else {
            hjbh::launch_init_values(R.d_slots.as<SlotDesc>(), m, static_cast<int>(NK), wform,
                                     c_over, nullptr, st);
            const int lanes = c.lanes == 2 && rows == 4 && lane_split_ok(P) ? 2 : 1;
            const hjbh::SweepKey key{P->kind == HJB_DYN_DUBINS ? 1 : 0, wform ? 1 : 0, key_na(P),
                                     halo, rows, 8 / rows / lanes, loop_mode(), lanes,
                                     nd > 2 ? hjbk::TZ : 1};
            R.near_start = wform && R.slots[0].vout == 0.0f;  // see solve_full
            TRY(run_loop(R, key, 8, control_table(P), st, c.li));
        }
        if (ms) {
            CK(cudaEventRecord(R.ev1, st));
            CK(cudaEventSynchronize(R.ev1));
            float t = 0;
            cudaEventElapsedTime(&t, R.ev0, R.ev1);
            *ms = t;
        }
        return HJB_OK;
    };
    {
        const std::string key = tune_key("ra", {P->kind, coarse.n[0], coarse.n[1], coarse.n[2], P->na,
                                                P->nb, P->interp, P->cost.user ? 1 : 0, m, halo});
        std::vector<Choice> cand;
        const int li_c[3] = {2, 4, 6};
        if (fixed_shape(P)) {
            for (int l : li_c) cand.push_back(Choice{hjbk::TY, 1, l, 0.0, hjbk::TZ});
        } else {
            const bool chip = chip_fits && !(ra_env && std::strcmp(ra_env, "tiles") == 0);
            const bool tiles = !(chip_fits && ra_env && std::strcmp(ra_env, "chip") == 0);
            if (tiles) {
                cand.push_back(Choice{2, 1, 6, 0.0, hjbk::TZ});
                for (int r : {4, 2})
                    for (int l : li_c)
                        if (!(r == 2 && l == 6)) cand.push_back(Choice{r, 1, l, 0.0, hjbk::TZ});
                if (lane_split_ok(P))
                    for (int l : li_c) cand.push_back(Choice{4, 2, l, 0.0, hjbk::TZ});
            }
            if (chip) cand.push_back(Choice{1, 1, 1, 0.0, hjbk::TZ});
        }
        TRY(tuned_candidates(key, cand, coarse_solve));
    }
    // threshold of eq. (rep)
    double delta = delta_in;
    double lipschitz = 0.0;
    TRY(P->scratch_u64.ensure(64));
    unsigned long long *d_u64 = P->scratch_u64.as<unsigned long long>();
    CK(cudaMemsetAsync(d_u64, 0, 64, st));
    if (delta < 0) {
        double M = ra->M;
        if (M < 0) {
            const float dxf[3] = {static_cast<float>(dxK[0]), static_cast<float>(dxK[1]),
                                  static_cast<float>(dxK[2])};
            unsigned *gm = reinterpret_cast<unsigned *>(d_u64 + 4);
            hjbh::launch_grad_max(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), m,
                                  wform ? 1 : 0, coarse, dxf, gm, st);
            unsigned hb = 0;
            CK(cudaMemcpyAsync(&hb, gm, sizeof hb, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            float f;
            std::memcpy(&f, &hb, sizeof f);
            M = f;
        }
        const double C = ra->C > 0 ? ra->C : 0.0;
        const double q = ra->q > 0 ? ra->q : 1.0;
        delta = 2.0 * (C * std::pow(dxK[0], q) + M * dxK[0]);
        lipschitz = M;
    }
    hjbh::launch_label(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), m, coarse,
                       P->c_labels.as<uint8_t>(), static_cast<float>(delta), wform ? 1 : 0, cl_dev,
                       nullptr, d_u64, st);
    hjbh::launch_project(fine, coarse, stride, cl_dev, fine_dev, st);
    hjbh::launch_popcount(fine_dev, P->N, d_u64 + 1, st);
    if (vaux_dev)
        for (int k = 0; k < m; ++k)
            hjbh::launch_extract(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), k,
                                 vaux_dev + static_cast<size_t>(k) * NK, wform, c_over, st);
    CK(cudaEventRecord(R.ev1, st));
    unsigned long long hc[2];
    CK(cudaMemcpyAsync(hc, d_u64, sizeof hc, cudaMemcpyDeviceToHost, st));
    int err = 0;
    long long sweeps = 0;
    TRY(read_state(R, st, &err, &sweeps));
    CK(cudaGetLastError());
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        int conv = 1;
        for (int k = 0; k < m; ++k) {
            const SlotState &s = R.h_state[k];
            stats->iterations = s.iters > stats->iterations ? s.iters : stats->iterations;
            stats->node_updates += static_cast<long long>(s.updates);
            stats->tile_visits += static_cast<long long>(s.visits);
            stats->final_residual = std::fmax(stats->final_residual, s.final_res);
            conv &= s.converged ? 1 : 0;
        }
        stats->converged = conv;
        stats->ties = static_cast<long long>(hc[0]);
        stats->labelled = static_cast<long long>(hc[1]);
        stats->delta = delta;
        stats->lipschitz = lipschitz;
        stats->local_iters = R.local_iters;
        stats->launches = pr.launches + (on_chip ? 7 : 9) + sweeps +
                          (delta_in < 0 && ra->M < 0 ? 1 : 0) + (vaux_dev ? m : 0);
        stats->subdomains = m;
        float ms = 0;
        cudaEventElapsedTime(&ms, R.ev0, R.ev1);
        stats->ms = ms;
    }
    if (err) return fail(HJB_ERR_TIMEOUT, "a bounded device wait gave up (TMA transfer lost)");
    for (int k = 0; k < m; ++k)
        if (!R.h_state[k].converged)
            return fail(HJB_ERR_NOT_CONVERGED, "auxiliary problem %d did not converge", k + 1);
    return HJB_OK;
}


}  // namespace

extern "C" {

int hjb_subdomains(hjb_problem *P, const hjb_ra_opts *ra, uint32_t *fine_mask_out,
                   uint32_t *coarse_labels_out, float *v_aux_out, hjb_stats *stats,
                   void *stream) {
    g_err.clear();
    if (!P || !ra || !fine_mask_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (ra->max_splits < 0 || ra->max_splits > HJB_MAX_TARGETS ||
        !(ra->split_gain >= 0.0 && ra->split_gain < 1.0))
        return fail(HJB_ERR_INVALID_ARG, "max_splits must be in [0, %d] and split_gain in [0, 1)",
                    HJB_MAX_TARGETS);
    if (ra->max_splits > 0 && v_aux_out)
        return fail(HJB_ERR_INVALID_ARG, "v_aux_out must be NULL when components are re-split");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nd = P->grid.ndim;
    long long NK = 1;
    for (int d = 0; d < nd; ++d) {
        const int r = ra->coarse_stride[d], n = P->grid.n[d];
        if (r < 1) return fail(HJB_ERR_INVALID_ARG, "coarse_stride[%d] < 1", d);
        if (P->grid.periodic[d] ? n % r : (n - 1) % r)
            return fail(HJB_ERR_INVALID_ARG, "stride %d does not divide n[%d]%s", r, d,
                        P->grid.periodic[d] ? "" : "-1");
        const int nk = P->grid.periodic[d] ? n / r : (n - 1) / r + 1;
        if (nk < 2) return fail(HJB_ERR_INVALID_ARG, "coarse grid has < 2 nodes in dim %d", d);
        NK *= nk;
    }
    OutArr fm, cl, va;
    TRY(fm.init(fine_mask_out, P->N * sizeof(uint32_t), &P->out_stage2));
    TRY(cl.init(coarse_labels_out, NK * sizeof(uint32_t), &P->c_mask));
    uint32_t *cl_dev = static_cast<uint32_t *>(cl.dev());
    if (!cl_dev) {
        TRY(P->c_mask.ensure(NK * sizeof(uint32_t)));
        cl_dev = P->c_mask.as<uint32_t>();
    }
    if (v_aux_out)
        TRY(va.init(v_aux_out, static_cast<size_t>(P->ntargets) * NK * sizeof(float), &P->c_vstage));
    uint32_t *fine_dev = static_cast<uint32_t *>(fm.dev());
    TRY(P->split_small.ensure(64 * sizeof(unsigned long long) + 8 * sizeof(int) +
                              65536 * sizeof(unsigned)));
    unsigned long long *d_cnt = P->split_small.as<unsigned long long>();
    hjb_stats s0;
    std::memset(&s0, 0, sizeof s0);
    const int rc0 = ra_division(P, ra, nullptr, P->ntargets, ra->delta, fine_dev, cl_dev,
                                v_aux_out ? static_cast<float *>(va.dev()) : nullptr, &s0, st);
    if (rc0 != HJB_OK && rc0 != HJB_ERR_NOT_CONVERGED) return rc0;
    int m = P->ntargets;
    long long launches = s0.launches;
    // recursive re-splitting of the target components (Conclusions): split the
    // component whose sub-domain is largest in two along the x or y axis of
    // larger index extent at the median index; keep the split when both parts'
    // sub-domains are smaller than (1 - split_gain) times the split one's
    std::vector<unsigned long long> sizes(HJB_MAX_TARGETS, 0ull), tsizes(HJB_MAX_TARGETS, 0ull);
    const hjbh::GridDims fd = dims_of(P);
    if (ra->max_splits > 0) {
        const double gain = ra->split_gain > 0 ? ra->split_gain : 0.05;
        TRY(P->split_lab.ensure(2 * P->N));
        TRY(P->split_fine.ensure(P->N * sizeof(uint32_t)));
        TRY(P->split_cl.ensure(NK * sizeof(uint32_t)));
        uint8_t *comp = P->split_lab.as<uint8_t>(), *trial = comp + P->N;
        int *d_ext = reinterpret_cast<int *>(d_cnt + 64);
        unsigned *d_nodes = reinterpret_cast<unsigned *>(d_ext + 4);
        unsigned *d_hist = reinterpret_cast<unsigned *>(d_ext + 8);
        Prep pr;
        TRY(prepare(P, st, pr));
        CK(cudaMemcpyAsync(comp, pr.labels, P->N, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemsetAsync(d_cnt, 0, 32 * sizeof(unsigned long long), st));
        hjbh::launch_bitcount(fine_dev, P->N, m, d_cnt, st);
        CK(cudaMemcpyAsync(sizes.data(), d_cnt, 32 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        launches += pr.launches + 1;
        for (int step = 0; step < ra->max_splits && m < HJB_MAX_TARGETS; ++step) {
            int k = 0;
            for (int j = 1; j < m; ++j)
                if (sizes[j] > sizes[k]) k = j;
            // extents of component k + 1, then the histogram along the axis
            const int init_ext[4] = {1 << 30, -1, 1 << 30, -1};
            CK(cudaMemcpyAsync(d_ext, init_ext, sizeof init_ext, cudaMemcpyHostToDevice, st));
            CK(cudaMemsetAsync(d_nodes, 0, sizeof(unsigned), st));
            hjbh::launch_comp_extent(fd, comp, k + 1, d_ext, d_nodes, st);
            int ext[4];
            unsigned cnt = 0;
            CK(cudaMemcpyAsync(ext, d_ext, sizeof ext, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(&cnt, d_nodes, sizeof cnt, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (cnt < 2) break;
            const int axis = (ext[1] - ext[0]) >= (ext[3] - ext[2]) ? 0 : 1;
            const int n = fd.n[axis];
            if (n > 65536) break;
            CK(cudaMemsetAsync(d_hist, 0, n * sizeof(unsigned), st));
            hjbh::launch_comp_hist(fd, comp, k + 1, axis, d_hist, st);
            std::vector<unsigned> hist(n);
            CK(cudaMemcpyAsync(hist.data(), d_hist, n * sizeof(unsigned), cudaMemcpyDeviceToHost,
                               st));
            CK(cudaStreamSynchronize(st));
            const unsigned long long half = (cnt + 1ull) / 2;
            unsigned long long cum = 0;
            int s_split = -1;
            for (int j = 0; j < n; ++j) {
                cum += hist[j];
                if (cum >= half) {
                    s_split = j;
                    break;
                }
            }
            if (cum == cnt) {  // everything at or below: the next lower occupied index
                int t = s_split - 1;
                while (t >= 0 && hist[t] == 0) --t;
                s_split = t;
            }
            launches += 2;
            if (s_split < 0) break;
            CK(cudaMemcpyAsync(trial, comp, P->N, cudaMemcpyDeviceToDevice, st));
            hjbh::launch_comp_split(fd, trial, k + 1, axis, s_split, m + 1, st);
            hjb_stats ts;
            std::memset(&ts, 0, sizeof ts);
            const int trc = ra_division(P, ra, trial, m + 1, s0.delta, P->split_fine.as<uint32_t>(),
                                        P->split_cl.as<uint32_t>(), nullptr, &ts, st);
            if (trc != HJB_OK) return trc;
            CK(cudaMemsetAsync(d_cnt, 0, 32 * sizeof(unsigned long long), st));
            hjbh::launch_bitcount(P->split_fine.as<uint32_t>(), P->N, m + 1, d_cnt, st);
            CK(cudaMemcpyAsync(tsizes.data(), d_cnt, 32 * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            launches += ts.launches + 2;
            const double lim = (1.0 - gain) * static_cast<double>(sizes[k]);
            if (static_cast<double>(tsizes[k]) > lim || static_cast<double>(tsizes[m]) > lim) break;
            // keep the split
            CK(cudaMemcpyAsync(comp, trial, P->N, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(fine_dev, P->split_fine.p, P->N * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(cl_dev, P->split_cl.p, NK * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, st));
            sizes = tsizes;
            s0.iterations = ts.iterations;
            s0.node_updates += ts.node_updates;
            s0.labelled = ts.labelled;
            s0.ties = ts.ties;
            ++m;
        }
        if (ra->split_labels) {
            const bool host = !is_device_ptr(ra->split_labels);
            CK(cudaMemcpyAsync(ra->split_labels, comp, P->N,
                               host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st));
        }
    } else {
        CK(cudaMemsetAsync(d_cnt, 0, 32 * sizeof(unsigned long long), st));
        hjbh::launch_bitcount(fine_dev, P->N, m, d_cnt, st);
        CK(cudaMemcpyAsync(sizes.data(), d_cnt, 32 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, st));
        launches += 1;
    }
    TRY(cl.finish(st));
    TRY(fm.finish(st));
    if (v_aux_out) TRY(va.finish(st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (stats) {
        *stats = s0;
        stats->subdomains = m;
        stats->launches = launches;
        unsigned long long big = 0;
        for (int k = 0; k < m; ++k) big = sizes[k] > big ? sizes[k] : big;
        stats->largest = static_cast<long long>(big);
    }
    // the auxiliary solutions in P->ra belong to the original division only
    // when no split was kept (the splits re-run RA on other divisions)
    P->ra_m = (m == P->ntargets && ra->max_splits == 0) ? m : 0;
    for (int d = 0; d < 3; ++d) P->ra_stride[d] = d < nd ? ra->coarse_stride[d] : 1;
    {
        bool wf;
        P->ra_wform = resolve_form(P, -1, &wf) == HJB_OK ? (wf ? 1 : 0) : -1;
    }
    return rc0;
}
}  // extern "C"

namespace {

int solve_dec(hjb_problem *P, const uint32_t *fine_mask, const hjb_solve_opts *opts,
              const Choice &ch, float *v_out, hjb_stats *per_subdomain, hjb_stats *total,
              cudaStream_t st) {
    const int rows = ch.rows, li = ch.li;
    bool wform;
    TRY(resolve_form(P, opts ? opts->use_w_form : -1, &wform));
    Prep pr;
    TRY(prepare(P, st, pr));
    int halo;
    TRY(halo_for(P, pr.max_off_xy, pr.max_off_z, &halo));
    const double tol = (opts && opts->tol > 0) ? opts->tol : default_tol(P, P->h);
    const int max_iters = (opts && opts->max_iters > 0) ? opts->max_iters : 100000;
    const int m = (opts && opts->n_subdomains > 0) ? opts->n_subdomains : P->ntargets;
    const int nd = P->grid.ndim;
    const hjbh::GridDims fine = dims_of(P);
    // warm start (the same array for every sub-domain, inside its nodes)
    const float *vinit = nullptr;
    if (opts && opts->v_init) {
        if (is_device_ptr(opts->v_init)) {
            vinit = opts->v_init;
        } else {
            TRY(P->in_stage.ensure(P->N * sizeof(float)));
            CK(cudaMemcpyAsync(P->in_stage.p, opts->v_init, P->N * sizeof(float),
                               cudaMemcpyHostToDevice, st));
            vinit = P->in_stage.as<float>();
        }
    }
    const uint32_t *mask = fine_mask;
    if (!is_device_ptr(fine_mask)) {
        TRY(P->fine_mask_dev.ensure(P->N * sizeof(uint32_t)));
        CK(cudaMemcpyAsync(P->fine_mask_dev.p, fine_mask, P->N * sizeof(uint32_t),
                           cudaMemcpyHostToDevice, st));
        mask = P->fine_mask_dev.as<uint32_t>();
    }
    RunCtx &R = P->dec;
    const SlotGeo g = geo_of(nd, P->grid.n, P->grid.periodic[2]);
    R.slots.assign(m, SlotDesc());
    std::memset(R.slots.data(), 0, m * sizeof(SlotDesc));
    if (P->kind == HJB_DYN_DUBINS)
        TRY(dubins_trig(P, P->trig, g.nz, P->h, P->dx, P->grid.lo[2], P->dx[2], st));
    const int tiles_x = (g.nx + hjbk::TX - 1) / hjbk::TX;
    const int tiles_y = (g.ny + rows - 1) / rows;
    const int tiles_z = nd > 2 ? (g.nz + ch.layers - 1) / ch.layers : 1;
    const int nt = tiles_x * tiles_y * tiles_z;
    // per-tile OR and AND of the sub-domain bits, then 32 words of pairwise
    // membership differences
    TRY(P->tile_bits.ensure((2 * nt + 32) * sizeof(uint32_t)));
    TRY(P->tile_clear.ensure(nt));
    hjbh::launch_tile_clear(fine, tiles_x, tiles_y, tiles_z, rows, ch.layers, pr.labels,
                            P->tile_clear.as<uint8_t>(), st);
    uint32_t *tile_full = P->tile_bits.as<uint32_t>() + nt;
    uint32_t *diff = P->tile_bits.as<uint32_t>() + 2 * nt;
    const bool own = opts && opts->subdomain_targets == HJB_SUBDOMAIN_TARGETS_OWN;
    for (int k = 0; k < m; ++k) {
        fill_slot(R.slots[k], P, g, pr, wform, P->h, P->dx, halo, tol, max_iters, rows, ch.layers);
        R.slots[k].tile_clear = P->tile_clear.as<uint8_t>();
        R.slots[k].mask = mask;
        R.slots[k].mask_bit = k;
        R.slots[k].only_target = own ? k + 1 : 0;
        R.slots[k].tile_bits = P->tile_bits.as<uint32_t>();
        R.slots[k].tile_full = tile_full;
        if (P->kind == HJB_DYN_DUBINS) R.slots[k].trig = P->trig.as<float2>();
    }
    TRY(alloc_slot_buffers(R, nd, halo, rows, ch.layers));
    TRY(upload_slots(R, st));
    OutArr out;
    TRY(out.init(v_out, P->N * sizeof(float), &P->out_stage));
    const float c_over = static_cast<float>(P->l_const / P->lambda);
    CK(cudaEventRecord(R.ev0, st));
    CK(cudaMemsetAsync(diff, 0, 32 * sizeof(uint32_t), st));
    hjbh::launch_tile_bits(fine, tiles_x, tiles_y, tiles_z, rows, ch.layers, mask,
                           P->tile_bits.as<uint32_t>(), st, diff, m, tile_full);
    if (opts && opts->warm_start) {
        // coarse-to-fine warm start from the reconstruction's auxiliary solutions
        hjbh::launch_init_from_coarse(R.d_slots.as<SlotDesc>(), P->ra.d_slots.as<SlotDesc>(),
                                      P->ra.d_state.as<SlotState>(), m, static_cast<int>(P->N),
                                      P->ra_stride[0], P->ra_stride[1], st);
    } else {
        hjbh::launch_init_values(R.d_slots.as<SlotDesc>(), m, static_cast<int>(P->N), wform, c_over,
                                 vinit, st);
    }
    const hjbh::SweepKey key{P->kind == HJB_DYN_DUBINS ? 1 : 0, wform ? 1 : 0, key_na(P), halo, rows,
                             8 / rows / ch.lanes, loop_mode(), ch.lanes, nd > 2 ? ch.layers : 1};
    // sub-domains with equal node sets are solved once (V_k depends on the
    // node set alone when its targets are the target nodes inside it; not so
    // with one target component per sub-domain)
    R.diff = own ? nullptr : diff;
    R.near_start = wform && !vinit && !(opts && opts->warm_start) &&
                   R.slots[0].vout == 0.0f;  // see solve_full
    const int lrc = run_loop(R, key, sweeps_per_body(opts), control_table(P), st, li);
    R.diff = nullptr;
    TRY(lrc);
    hjbh::launch_assemble(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), m, fine, mask,
                          wform ? 1 : 0, c_over, static_cast<float>(P->value_out),
                          static_cast<float *>(out.dev()), st, R.d_ctl.as<Ctl>());
    CK(cudaEventRecord(R.ev1, st));
    TRY(out.finish(st));
    int err = 0;
    long long sweeps = 0;
    TRY(read_state(R, st, &err, &sweeps));
    CK(cudaGetLastError());
    float ms = 0;
    cudaEventElapsedTime(&ms, R.ev0, R.ev1);
    int conv = 1;
    hjb_stats tot;
    std::memset(&tot, 0, sizeof tot);
    for (int k = 0; k < m; ++k) {
        SlotState s = R.h_state[k];
        if (s.twin >= 0 && s.twin < k) {
            // solved as its twin: same iterate, no node-updates of its own
            const SlotState &t = R.h_state[s.twin];
            s.iters = t.iters;
            s.converged = t.converged;
            s.final_res = t.final_res;
            s.updates = 0ull;
            s.visits = 0u;
        }
        if (per_subdomain) {
            fill_stats(&per_subdomain[k], s);
            per_subdomain[k].ms = ms;
            per_subdomain[k].tile_rows = P->grid.ndim == 2 ? rows : 0;
            per_subdomain[k].tile_lanes = ch.lanes;
            per_subdomain[k].tile_layers = P->grid.ndim > 2 ? ch.layers : 0;
            per_subdomain[k].local_iters = R.local_iters;
        }
        tot.iterations = s.iters > tot.iterations ? s.iters : tot.iterations;
        tot.node_updates += static_cast<long long>(s.updates);
        tot.tile_visits += static_cast<long long>(s.visits);
        tot.final_residual = std::fmax(tot.final_residual, s.final_res);
        conv &= s.converged ? 1 : 0;
    }
    tot.converged = conv;
    tot.ms = ms;
    tot.launches = pr.launches + 6 + sweeps;
    tot.tile_rows = P->grid.ndim == 2 ? rows : 0;
    tot.tile_lanes = ch.lanes;
    tot.tile_layers = P->grid.ndim > 2 ? ch.layers : 0;
    tot.local_iters = R.local_iters;
    if (total) *total = tot;
    if (err) return fail(HJB_ERR_TIMEOUT, "a bounded device wait gave up (TMA transfer lost)");
    if (!conv) return fail(HJB_ERR_NOT_CONVERGED, "a sub-domain did not converge");
    return HJB_OK;
}

}  // namespace

extern "C" {

int hjb_solve_decomposed(hjb_problem *P, const uint32_t *fine_mask, const hjb_solve_opts *opts,
                         float *v_out, hjb_stats *per_subdomain, hjb_stats *total, void *stream) {
    g_err.clear();
    if (!P || !fine_mask || !v_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    TRY(check_opts(opts));
    if (opts && opts->warm_start) {
        bool wf;
        TRY(resolve_form(P, opts->use_w_form, &wf));
        if (P->grid.ndim != 2 || P->ra_m != P->ntargets || (opts->n_subdomains > 0 &&
            opts->n_subdomains != P->ntargets) || opts->v_init || P->ra_wform != (wf ? 1 : 0))
            return fail(HJB_ERR_INVALID_ARG,
                        "warm_start needs a 2D problem whose last hjb_subdomains call kept its "
                        "division (no splits), the same iterated form, and no v_init");
    }
    if (opts && opts->n_subdomains > P->ntargets &&
        opts->subdomain_targets == HJB_SUBDOMAIN_TARGETS_OWN)
        return fail(HJB_ERR_UNSUPPORTED,
                    "sub-domains of re-split components take every target node inside them "
                    "(HJB_SUBDOMAIN_TARGETS_ALL)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const std::string key = tune_key("decomposed",
                                     {P->kind, P->grid.n[0], P->grid.n[1], P->grid.n[2], P->na, P->nb,
                                      P->interp, P->cost.user ? 1 : 0,
                                      (opts && opts->n_subdomains > 0) ? opts->n_subdomains
                                                                       : P->ntargets,
                                      opts ? opts->subdomain_targets : 0,
                                      opts && opts->v_init ? 1 : 0,
                                      opts ? opts->warm_start : 0});
    return tuned_call(key, P, fixed_shape(P), pinned_local_iters(opts), [&](Choice c, double *ms) {
        hjb_stats tmp;
        hjb_stats *tp = total ? total : &tmp;
        const int rc = solve_dec(P, fine_mask, opts, c, v_out, per_subdomain, tp, st);
        if (ms) *ms = tp->ms;
        return rc;
    });
}

}  // extern "C"

namespace {

int solve_batch_impl(hjb_problem *const *problems, int count, const hjb_solve_opts *opts,
                     const Choice &ch, float *const *v_out, hjb_stats *per_problem,
                     cudaStream_t st) {
    const int rows = ch.rows, li = ch.li;
    hjb_problem *P0 = problems[0];
    if (!P0) return fail(HJB_ERR_INVALID_ARG, "NULL problem");
    bool wform;
    TRY(resolve_form(P0, opts ? opts->use_w_form : -1, &wform));
    std::vector<Prep> preps(count);
    int halo = 2;
    for (int i = 0; i < count; ++i) {
        hjb_problem *P = problems[i];
        if (!P || !v_out[i]) return fail(HJB_ERR_INVALID_ARG, "NULL problem or output %d", i);
        if (P->kind != P0->kind || P->na != P0->na || P->grid.ndim != P0->grid.ndim ||
            (P->cost.user == nullptr) != (P0->cost.user == nullptr) ||
            std::memcmp(P->ax, P0->ax, P->na * sizeof(float)) ||
            std::memcmp(P->ay, P0->ay, P->na * sizeof(float)) || P->l_const != P0->l_const ||
            P->nb != P0->nb || P->interp != P0->interp ||
            std::memcmp(P->bx, P0->bx, P->nb * sizeof(float)) ||
            std::memcmp(P->by, P0->by, P->nb * sizeof(float)) ||
            P->lambda != P0->lambda)
            return fail(HJB_ERR_INVALID_ARG,
                        "problem %d differs from problem 0 in dynamics kind, controls, cost form "
                        "or discount rate",
                        i);
        TRY(prepare(P, st, preps[i]));
        int hh;
        TRY(halo_for(P, preps[i].max_off_xy, preps[i].max_off_z, &hh));
        halo = hh > halo ? hh : halo;
    }
    if (!P0->batch) P0->batch = new RunCtx();
    RunCtx &R = *P0->batch;
    R.slots.assign(count, SlotDesc());
    std::memset(R.slots.data(), 0, count * sizeof(SlotDesc));
    long long maxN = 0;
    for (int i = 0; i < count; ++i) {
        hjb_problem *P = problems[i];
        const SlotGeo g = geo_of(P->grid.ndim, P->grid.n, P->grid.periodic[2]);
        const double tol = (opts && opts->tol > 0) ? opts->tol : default_tol(P, P->h);
        const int max_iters = (opts && opts->max_iters > 0) ? opts->max_iters : 100000;
        fill_slot(R.slots[i], P, g, preps[i], wform, P->h, P->dx, halo, tol, max_iters, rows,
                  ch.layers);
        if (P->kind == HJB_DYN_DUBINS) {
            TRY(dubins_trig(P, P->trig, g.nz, P->h, P->dx, P->grid.lo[2], P->dx[2], st));
            R.slots[i].trig = P->trig.as<float2>();
        }
        maxN = P->N > maxN ? P->N : maxN;
    }
    TRY(alloc_slot_buffers(R, P0->grid.ndim, halo, rows, ch.layers));
    TRY(upload_slots(R, st));
    const float c_over = static_cast<float>(P0->l_const / P0->lambda);
    std::vector<OutArr> outs(count);
    CK(cudaEventRecord(R.ev0, st));
    hjbh::launch_init_values(R.d_slots.as<SlotDesc>(), count, static_cast<int>(maxN), wform, c_over,
                             nullptr, st);
    const hjbh::SweepKey key{P0->kind == HJB_DYN_DUBINS ? 1 : 0, wform ? 1 : 0, key_na(P0), halo, rows,
                             8 / rows / ch.lanes, loop_mode(), ch.lanes,
                             P0->grid.ndim > 2 ? ch.layers : 1};
    TRY(run_loop(R, key, sweeps_per_body(opts), control_table(P0), st, li));
    for (int i = 0; i < count; ++i) {
        TRY(outs[i].init(v_out[i], problems[i]->N * sizeof(float), &problems[i]->out_stage));
        hjbh::launch_extract(R.d_slots.as<SlotDesc>(), R.d_state.as<SlotState>(), i,
                             static_cast<float *>(outs[i].dev()), wform, c_over, st);
    }
    CK(cudaEventRecord(R.ev1, st));
    for (int i = 0; i < count; ++i) TRY(outs[i].finish(st));
    int err = 0;
    long long sweeps = 0;
    TRY(read_state(R, st, &err, &sweeps));
    long long nl = 3 + sweeps + count;
    for (int i = 0; i < count; ++i) nl += preps[i].launches;
    CK(cudaGetLastError());
    float ms = 0;
    cudaEventElapsedTime(&ms, R.ev0, R.ev1);
    int conv = 1;
    for (int i = 0; i < count; ++i) {
        if (per_problem) {
            fill_stats(&per_problem[i], R.h_state[i]);
            per_problem[i].ms = ms;
            per_problem[i].launches = nl;
            per_problem[i].tile_rows = P0->grid.ndim == 2 ? rows : 0;
            per_problem[i].tile_lanes = ch.lanes;
            per_problem[i].tile_layers = P0->grid.ndim > 2 ? ch.layers : 0;
            per_problem[i].local_iters = R.local_iters;
        }
        conv &= R.h_state[i].converged ? 1 : 0;
    }
    if (err) return fail(HJB_ERR_TIMEOUT, "a bounded device wait gave up (TMA transfer lost)");
    if (!conv) return fail(HJB_ERR_NOT_CONVERGED, "a problem of the batch did not converge");
    return HJB_OK;
}

}  // namespace

extern "C" {

int hjb_solve_batch(hjb_problem *const *problems, int count, const hjb_solve_opts *opts,
                    float *const *v_out, hjb_stats *per_problem, void *stream) {
    g_err.clear();
    if (!problems || count < 1 || !v_out) return fail(HJB_ERR_INVALID_ARG, "empty batch");
    if (count > HJB_MAX_BATCH)
        return fail(HJB_ERR_INVALID_ARG, "at most %d problems per batch", HJB_MAX_BATCH);
    TRY(check_opts(opts));
    if (!problems[0]) return fail(HJB_ERR_INVALID_ARG, "NULL problem");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    long long nodes = 0;
    for (int i = 0; i < count; ++i) nodes += problems[i] ? problems[i]->N : 0;
    const hjb_problem *P0 = problems[0];
    const std::string key = tune_key("batch", {P0->kind, count, nodes, P0->na, P0->nb, P0->interp,
                                               P0->cost.user ? 1 : 0});
    std::vector<hjb_stats> tmp(count);
    return tuned_call(key, P0, fixed_shape(P0), pinned_local_iters(opts), [&](Choice c, double *ms) {
        hjb_stats *pp = per_problem ? per_problem : tmp.data();
        const int rc = solve_batch_impl(problems, count, opts, c, v_out, pp, st);
        if (ms) *ms = pp[0].ms;
        return rc;
    });
}

// The graph of an adjoint loop (WHILE conditional node): `reps` rounds of the
// kernels fns[0..nf) per body, each on `grid` CTAs with `smem` bytes of
// dynamic shared memory and `args` (whose handle is set here); the kernels'
// last CTA sets the condition.
int build_adj_loop(cudaGraph_t &graph, cudaGraphExec_t &exec, const void *const *fns, int nf,
                   int reps, hjbh::AdjArgs &args, int grid, size_t smem) {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    CK(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    CK(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    CK(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    args.handle = handle;
    args.use_handle = 1;
    cudaGraphNode_t prev = nullptr;
    for (int rep = 0; rep < reps; ++rep)
        for (int k = 0; k < nf; ++k) {
            cudaKernelNodeParams kp;
            std::memset(&kp, 0, sizeof kp);
            kp.func = const_cast<void *>(fns[k]);
            kp.gridDim = dim3(grid);
            kp.blockDim = dim3(hjbk::THREADS);
            kp.sharedMemBytes = static_cast<unsigned>(smem);
            void *argv[1] = {&args};
            kp.kernelParams = argv;
            cudaGraphNode_t node;
            CK(cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
            prev = node;
        }
    CK(cudaGraphInstantiate(&exec, graph, 0));
    return HJB_OK;
}

// An instantiated loop graph can be reused when its kernels' arguments
// (other than the condition handle) are the same.
bool same_adj_args(cudaGraphExec_t exec, const hjbh::AdjArgs &a, const hjbh::AdjArgs &b) {
    return exec && !std::memcmp(&a.ap, &b.ap, sizeof a.ap) &&
           !std::memcmp(&a.ctrl, &b.ctrl, sizeof a.ctrl) && a.policy == b.policy && a.g == b.g &&
           a.L[0] == b.L[0] && a.L[1] == b.L[1] && a.ctl == b.ctl && a.cell == b.cell &&
           a.frac == b.frac;
}

int hjb_backward(hjb_problem *P, const float *v, const float *grad_v, int wrt,
                 const hjb_solve_opts *opts, float *grad_out, hjb_stats *stats, void *stream) {
    g_err.clear();
    if (!P || !v || !grad_v || !grad_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (wrt != 0 && wrt != 1) return fail(HJB_ERR_INVALID_ARG, "wrt must be 0 (log-speed) or 1 (cost)");
    if (P->kind != HJB_DYN_SPEED_CURRENT)
        return fail(HJB_ERR_UNSUPPORTED, "the adjoint is implemented for 2D speed/current dynamics");
    if (P->nb || P->scale.user || P->interp != HJB_INTERP_Q1)
        return fail(HJB_ERR_UNSUPPORTED,
                    "the adjoint handles Q1 interpolation without games or per-axis scale fields");
    TRY(check_opts(opts));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Prep pr;
    TRY(prepare(P, st, pr));
    const long long N = P->N;
    // inputs into problem-owned buffers (the graph's arguments stay fixed)
    TRY(P->adj_v.ensure(N * sizeof(float)));
    TRY(P->adj_g.ensure(N * sizeof(float)));
    CK(cudaMemcpyAsync(P->adj_v.p, v, N * sizeof(float), cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(P->adj_g.p, grad_v, N * sizeof(float), cudaMemcpyDefault, st));
    TRY(P->adj_policy.ensure(N));
    TRY(P->adj_cell.ensure(N * sizeof(int)));
    TRY(P->adj_frac.ensure(N * sizeof(float2)));
    TRY(P->adj_L.ensure(2 * N * sizeof(float)));
    TRY(P->adj_ctl.ensure(sizeof(hjbh::AdjCtl)));
    TRY(P->scratch_u64.ensure(64));
    unsigned *d_ties = P->scratch_u64.as<unsigned>();
    CK(cudaMemsetAsync(d_ties, 0, sizeof(unsigned), st));
    hjbh::AdjProblem ap;
    ap.nx = P->grid.n[0];
    ap.ny = P->grid.n[1];
    ap.hx = static_cast<float>(P->h / P->dx[0]);
    ap.hy = static_cast<float>(P->h / P->dx[1]);
    ap.hd = P->h;
    ap.dxd = P->dx[0];
    ap.dyd = P->dx[1];
    ap.dx = static_cast<float>(P->dx[0]);
    ap.dy = static_cast<float>(P->dx[1]);
    ap.betad = beta_w(P->weights, P->lambda, P->h);
    ap.gammad = gamma_w(P->weights, P->lambda, P->h);
    ap.lconst = P->l_const;
    ap.cost = pr.cost;
    ap.beta = static_cast<float>(ap.betad);
    ap.gamma = static_cast<float>(ap.gammad);
    ap.h = static_cast<float>(P->h);
    ap.vout = static_cast<float>(P->value_out);
    ap.speed = pr.speed;
    ap.current = pr.current;
    ap.labels = pr.labels;
    const hjbk::ControlTable ctrl = control_table(P);
    // no absolute default: the iteration runs to the FP32 floor of lambda
    const double tol = (opts && opts->tol > 0) ? opts->tol : 0.0;
    const int max_iters = (opts && opts->max_iters > 0) ? opts->max_iters : 100000;
    float *L0 = P->adj_L.as<float>(), *L1 = L0 + N;
    hjbh::AdjCtl *ctl = P->adj_ctl.as<hjbh::AdjCtl>();
    RunCtx &R = P->full;
    if (!R.ev0) {
        CK(cudaEventCreate(&R.ev0));
        CK(cudaEventCreate(&R.ev1));
    }
    OutArr out;
    TRY(out.init(grad_out, N * sizeof(float), &P->out_stage));
    CK(cudaEventRecord(R.ev0, st));
    // controls within this relative margin of the best FP32 value are decided
    // in FP64 (the FP32 error of a control value is a few ulp)
    constexpr float POLICY_MARGIN = 1e-5f;
    hjbh::launch_policy(ap, ctrl, P->adj_v.as<float>(), nullptr, POLICY_MARGIN,
                        P->adj_policy.as<int8_t>(), d_ties, st);
    hjbh::launch_feet(ap, ctrl, P->adj_policy.as<int8_t>(), P->adj_cell.as<int>(),
                      P->adj_frac.as<float2>(), st);
    long long ref_launches = 0;
    int ref_iters = 0;
    // the tiles of the refinement and of the transposed iteration hold every
    // corner of a policy foot in their halo: the largest foot offset, rounded
    // up, plus the second corner
    const int tiles_hr = std::max(2, static_cast<int>(std::ceil(pr.max_off_xy)) + 1);
    if (tiles_hr > 7)
        return fail(HJB_ERR_UNSUPPORTED, "the adjoint takes feet of at most 6 cells (h |f| / dx)");
    const int tiles_grid = hjbh::refine_tiles_grid(ap.nx, ap.ny);
    // applications per staged tile and sweep of both loops (HJB_ADJ_APPS: 8,
    // 16 or 32; default 16)
    const char *ea = std::getenv("HJB_ADJ_APPS");
    const int ea_v = ea ? std::atoi(ea) : 16;
    const int apps = (ea_v == 8 || ea_v == 32) ? ea_v : 16;
    {
        // iterative refinement of the values the policy is decided on (see
        // refine_residual_kernel): HJB_ADJ_REFINE rounds, default 1, 0 = none
        const char *e = std::getenv("HJB_ADJ_REFINE");
        const int rounds = e ? std::max(0, std::min(4, std::atoi(e))) : 1;
        if (rounds > 0) TRY(P->adj_ref.ensure(3 * N * sizeof(float)));
        for (int round = 0; round < rounds; ++round) {
            float *r = P->adj_ref.as<float>(), *D0 = r + N, *D1 = D0 + N;
            hjbh::launch_refine_residual(ap, ctrl, P->adj_v.as<float>(), P->adj_policy.as<int8_t>(),
                                         r, st);
            hjbh::launch_adj_init(r, D0, D1, N, ctl, 0.0f, 5000, st);
            hjbh::AdjArgs ra;
            std::memset(&ra, 0, sizeof ra);
            ra.ap = ap;
            ra.ctrl = ctrl;
            ra.policy = P->adj_policy.as<int8_t>();
            ra.g = r;
            ra.L[0] = D0;
            ra.L[1] = D1;
            ra.ctl = ctl;
            ra.cell = P->adj_cell.as<int>();
            ra.frac = P->adj_frac.as<float2>();
            // tiles' halo: every corner of a policy foot (at most ceil of the
            // largest foot offset, plus the second corner)
            ra.hr = tiles_hr;
            const int rgrid = tiles_grid;
            const size_t rsmem = hjbh::refine_tiles_smem(ra.hr);
            hjbh::AdjCtl hr;
            const char *ng = std::getenv("HJB_NO_GRAPH");
            if (ng && ng[0] == '1') {
                // host-driven loop (profiling aid): 8 sweeps between reads of
                // the stopping flag
                void *argv[1] = {&ra};
                for (;;) {
                    for (int k = 0; k < 8; ++k)
                        CK(cudaLaunchKernel(hjbh::refine_tiles_kernel(apps), dim3(rgrid),
                                            dim3(hjbk::THREADS), argv, rsmem, st));
                    CK(cudaMemcpyAsync(&hr, ctl, sizeof hr, cudaMemcpyDeviceToHost, st));
                    CK(cudaStreamSynchronize(st));
                    if (hr.converged) break;
                }
            } else {
                // graph loop: 2 sweeps per body, the last CTA of each sets the
                // condition
                if (!same_adj_args(P->ref_exec, P->ref_args_in_graph, ra) ||
                    P->ref_args_in_graph.hr != ra.hr || P->ref_apps_in_graph != apps) {
                    const void *fns[1] = {hjbh::refine_tiles_kernel(apps)};
                    TRY(build_adj_loop(P->ref_graph, P->ref_exec, fns, 1, 2, ra, rgrid, rsmem));
                    P->ref_args_in_graph = ra;
                    P->ref_apps_in_graph = apps;
                }
                CK(cudaGraphLaunch(P->ref_exec, st));
                CK(cudaMemcpyAsync(&hr, ctl, sizeof hr, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
            }
            ref_launches += (hr.iters + 1) / 2 * 2;
            if (hr.error)
                return fail(HJB_ERR_CUDA, "a policy foot lies beyond the refinement tiles' halo");
            if (hr.converged != 2)
                return fail(HJB_ERR_NOT_CONVERGED,
                            "refinement of the policy values not converged after %d sweeps",
                            hr.iters);
            ref_iters += hr.iters;
            CK(cudaMemsetAsync(d_ties, 0, sizeof(unsigned), st));
            hjbh::launch_policy(ap, ctrl, P->adj_v.as<float>(), hr.parity ? D1 : D0,
                                POLICY_MARGIN + 2.0f * hr.lam_max, P->adj_policy.as<int8_t>(),
                                d_ties, st);
            hjbh::launch_feet(ap, ctrl, P->adj_policy.as<int8_t>(), P->adj_cell.as<int>(),
                              P->adj_frac.as<float2>(), st);
            ref_launches += 4;
        }
    }
    hjbh::launch_adj_init(P->adj_g.as<float>(), L0, L1, N, ctl, static_cast<float>(tol), max_iters,
                          st);
    // graph: WHILE { sweep } x 2
    hjbh::AdjArgs args;
    std::memset(&args, 0, sizeof args);
    args.ap = ap;
    args.ctrl = ctrl;
    args.policy = P->adj_policy.as<int8_t>();
    args.g = P->adj_g.as<float>();
    args.L[0] = L0;
    args.L[1] = L1;
    args.ctl = ctl;
    args.use_handle = 1;
    args.cell = P->adj_cell.as<int>();
    args.frac = P->adj_frac.as<float2>();
    args.hr = tiles_hr;
    const size_t asmem = hjbh::adj_tiles_smem(tiles_hr);
    const char *ng = std::getenv("HJB_NO_GRAPH");
    if (ng && ng[0] == '1') {
        // host-driven loop (profiling aid): the same kernel, 8 sweeps between
        // reads of the convergence flag
        args.use_handle = 0;
        void *argv[1] = {&args};
        for (;;) {
            for (int rep = 0; rep < 8; ++rep)
                CK(cudaLaunchKernel(hjbh::adj_tiles_kernel(apps), dim3(tiles_grid),
                                    dim3(hjbk::THREADS), argv, asmem, st));
            int conv = 0;
            CK(cudaMemcpyAsync(&conv, &ctl->converged, sizeof conv, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            if (conv) break;
        }
    } else if (!same_adj_args(P->adj_exec, P->adj_args_in_graph, args) ||
               P->adj_args_in_graph.hr != args.hr || P->adj_apps_in_graph != apps) {
        const void *fns[1] = {hjbh::adj_tiles_kernel(apps)};
        TRY(build_adj_loop(P->adj_graph, P->adj_exec, fns, 1, 2, args, tiles_grid, asmem));
        P->adj_args_in_graph = args;
        P->adj_apps_in_graph = apps;
    }
    if (args.use_handle) CK(cudaGraphLaunch(P->adj_exec, st));
    hjbh::AdjCtl hc;
    CK(cudaMemcpyAsync(&hc, ctl, sizeof hc, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const float *lam = hc.parity ? L1 : L0;
    hjbh::launch_adj_grad(ap, ctrl, P->adj_v.as<float>(), P->adj_policy.as<int8_t>(), lam, wrt,
                          static_cast<float *>(out.dev()), st);
    CK(cudaEventRecord(R.ev1, st));
    TRY(out.finish(st));
    unsigned ties = 0;
    CK(cudaMemcpyAsync(&ties, d_ties, sizeof ties, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->iterations = hc.iters;
        stats->converged = (hc.converged == 1 || hc.converged == 2) ? hc.converged : 0;
        stats->final_residual = hc.final_res;
        stats->node_updates = static_cast<long long>(hc.iters) * N * apps;
        stats->ties = ties;
        stats->launches = pr.launches + 4 + 2LL * ((hc.iters + 1) / 2) + ref_launches;
        stats->local_iters = ref_iters;  // iterations of the policy-value refinement
        float ms = 0;
        cudaEventElapsedTime(&ms, R.ev0, R.ev1);
        stats->ms = ms;
    }
    if (hc.converged != 1 && hc.converged != 2)
        return fail(HJB_ERR_NOT_CONVERGED, "adjoint not converged after %d iterations (residual %g)",
                    hc.iters, hc.final_res);
    return HJB_OK;
}

int hjb_point_values(hjb_problem *P, const float *v, const float *points, int npts, float *values,
                     float *grad_v, void *stream) {
    g_err.clear();
    if (!P || !v || !points || npts < 0) return fail(HJB_ERR_INVALID_ARG, "bad argument");
    if (P->grid.ndim != 2) return fail(HJB_ERR_UNSUPPORTED, "point values are implemented in 2D");
    if (npts == 0) return HJB_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long N = P->N;
    const float *vd = v;
    if (!is_device_ptr(v)) {
        TRY(P->in_stage.ensure(N * sizeof(float)));
        CK(cudaMemcpyAsync(P->in_stage.p, v, N * sizeof(float), cudaMemcpyHostToDevice, st));
        vd = P->in_stage.as<float>();
    }
    const float *pd = points;
    DevBuf pts_stage;
    if (!is_device_ptr(points)) {
        TRY(pts_stage.ensure(static_cast<size_t>(npts) * 2 * sizeof(float)));
        CK(cudaMemcpyAsync(pts_stage.p, points, static_cast<size_t>(npts) * 2 * sizeof(float),
                           cudaMemcpyHostToDevice, st));
        pd = pts_stage.as<float>();
    }
    OutArr ov, og;
    TRY(ov.init(values, static_cast<size_t>(npts) * sizeof(float), &P->out_stage2));
    TRY(og.init(grad_v, N * sizeof(float), &P->out_stage3));
    if (grad_v) CK(cudaMemsetAsync(og.dev(), 0, N * sizeof(float), st));
    hjbh::launch_points(P->grid.n[0], P->grid.n[1], P->grid.lo[0], P->grid.lo[1], P->dx[0],
                        P->dx[1], vd, pd, npts, values ? static_cast<float *>(ov.dev()) : nullptr,
                        grad_v ? static_cast<float *>(og.dev()) : nullptr, st);
    TRY(ov.finish(st));
    TRY(og.finish(st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    pts_stage.release();
    return HJB_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free full-domain solve (hjb_solve_static).
//
// For callers that cannot allocate device memory while they run --
// real-time loops that forbid cudaMalloc/cudaFree after start-up (both may
// synchronise the device), plug-ins whose host application owns every
// allocation -- this entry point keeps all of its working memory in one
// file-scope device array.  The array is a fixed 4 MiB on every GPU that
// loads the library, for as long as the process lives; it bounds the grid to
// STATIC_MAX_NODES nodes.  Each call re-initialises everything it reads, so
// no state carries over, but all calls share the array: calls that can
// overlap on the GPU (different streams, different host threads) race.

namespace {

constexpr size_t STATIC_SCRATCH_BYTES = size_t(4) << 20;
constexpr long long STATIC_MAX_NODES = 256LL * 1024;
constexpr int STATIC_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

std::mutex g_static_mu;
void *g_static_addr[STATIC_MAX_DEVICES];

// Device address of the scratch array for the current device.  The host
// name of a __device__ array is only a stand-in, so its address is looked up
// once per device, with that device current.
int static_scratch(unsigned char **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= STATIC_MAX_DEVICES)
        return fail(HJB_ERR_UNSUPPORTED, "device ordinal %d beyond %d", dev, STATIC_MAX_DEVICES);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(HJB_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                        cudaGetErrorString(e));
        g_static_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_static_addr[dev]);
    return HJB_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" int hjb_solve_static(const hjb_grid *grid, const hjb_dynamics *dyn, const hjb_cost *cost,
                                const hjb_discount *disc, const hjb_controls *controls,
                                const hjb_target *target, const hjb_solve_opts *opts, float *v_out,
                                hjb_stats *stats, void *stream) {
    g_err.clear();
    if (!grid || !dyn || !cost || !disc || !controls || !target || !v_out)
        return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (grid->ndim != 2 || dyn->kind != HJB_DYN_SPEED_CURRENT || grid->periodic[0] ||
        grid->periodic[1])
        return fail(HJB_ERR_UNSUPPORTED, "the static solve handles 2D speed/current problems");
    if (grid->n[0] < 2 || grid->n[1] < 2 || !(grid->hi[0] > grid->lo[0]) ||
        !(grid->hi[1] > grid->lo[1]))
        return fail(HJB_ERR_INVALID_ARG, "bad grid");
    const long long N = static_cast<long long>(grid->n[0]) * grid->n[1];
    if (N > STATIC_MAX_NODES)
        return fail(HJB_ERR_INVALID_ARG,
                    "grid of %lld nodes exceeds the static solve's maximum of %lld nodes", N,
                    STATIC_MAX_NODES);
    if (controls->count < 1 || controls->count > HJB_MAX_CONTROLS || controls->dim != 2 ||
        !controls->a)
        return fail(HJB_ERR_INVALID_ARG, "controls must be 1..%d 2D vectors", HJB_MAX_CONTROLS);
    for (int j = 0; j < 2 * controls->count; ++j)
        if (!std::isfinite(controls->a[j])) return fail(HJB_ERR_INVALID_ARG, "non-finite control");
    if (!(disc->h > 0) || !(disc->lambda > 0) || !std::isfinite(disc->h) ||
        !std::isfinite(disc->lambda))
        return fail(HJB_ERR_INVALID_ARG, "h and lambda must be positive");
    if (disc->weights != HJB_WEIGHTS_EXP && disc->weights != HJB_WEIGHTS_IMPLICIT)
        return fail(HJB_ERR_INVALID_ARG, "unknown step weights %d", disc->weights);
    if (disc->interp != HJB_INTERP_Q1)
        return fail(HJB_ERR_UNSUPPORTED, "the static solve uses Q1 interpolation");
    if (!target->labels || target->n_targets < 1 || target->n_targets > HJB_MAX_TARGETS)
        return fail(HJB_ERR_INVALID_ARG, "bad target description");
    if (!cost->l && !(cost->l_const > 0))
        return fail(HJB_ERR_INVALID_ARG, "constant running cost must be positive");
    if (dyn->speed && dyn->log_speed) return fail(HJB_ERR_INVALID_ARG, "give speed or log_speed");
    if (dyn->scale || controls->count_b)
        return fail(HJB_ERR_UNSUPPORTED, "the static solve takes no scale field and no second player");
    if (opts && opts->max_iters < 0) return fail(HJB_ERR_INVALID_ARG, "max_iters < 0");
    // every array must already be device memory: staging host data would allocate
    const void *ptrs[6] = {dyn->speed, dyn->current, dyn->log_speed, cost->l, target->labels, v_out};
    for (const void *q : ptrs)
        if (q && !is_device_ptr(q))
            return fail(HJB_ERR_INVALID_ARG, "the static solve takes device arrays only");
    if (opts && opts->v_init && !is_device_ptr(opts->v_init))
        return fail(HJB_ERR_INVALID_ARG, "the static solve takes device arrays only");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *base = nullptr;
    TRY(static_scratch(&base));

    // layout of the scratch array
    const int rows = hjbk::TY;
    const int nx = grid->n[0], ny = grid->n[1];
    const int pitch = (nx + 31) / 32 * 32;
    const int tiles = ((nx + hjbk::TX - 1) / hjbk::TX) * ((ny + rows - 1) / rows);
    size_t off = 0;
    const size_t o_ctl = off;
    off = align256(off + sizeof(Ctl));
    const size_t o_state = off;
    off = align256(off + sizeof(SlotState));
    const size_t o_slot = off;
    off = align256(off + sizeof(SlotDesc));
    const size_t o_red = off;
    off = align256(off + 64);
    const size_t o_qlist = off;
    off = align256(off + 2 * static_cast<size_t>(tiles) * sizeof(int));
    const size_t o_qflag = off;
    const size_t fb = (static_cast<size_t>(tiles) + 3) / 4 * 4;
    off = align256(off + 2 * fb);
    const size_t o_sexp = off;
    if (dyn->log_speed) off = align256(off + N * sizeof(float));
    const size_t vbytes = align256(static_cast<size_t>(pitch) * ny * sizeof(float));
    const size_t o_v0 = off;
    off += vbytes;
    const size_t o_v1 = off;
    off += vbytes;
    if (off > STATIC_SCRATCH_BYTES)
        return fail(HJB_ERR_INVALID_ARG, "grid %d x %d needs %zu bytes of the %zu-byte static scratch",
                    nx, ny, off, STATIC_SCRATCH_BYTES);
    Ctl *d_ctl = reinterpret_cast<Ctl *>(base + o_ctl);
    SlotState *d_state = reinterpret_cast<SlotState *>(base + o_state);
    SlotDesc *d_slot = reinterpret_cast<SlotDesc *>(base + o_slot);
    unsigned *d_red = reinterpret_cast<unsigned *>(base + o_red);

    // speed (exp of the log-speed field when given) and the largest foot
    // displacement, which selects the interpolation halo
    const float *speed = dyn->speed;
    if (dyn->log_speed) {
        float *sexp = reinterpret_cast<float *>(base + o_sexp);
        hjbh::launch_exp(dyn->log_speed, sexp, N, st);
        speed = sexp;
    }
    double dx[3] = {(grid->hi[0] - grid->lo[0]) / (nx - 1), (grid->hi[1] - grid->lo[1]) / (ny - 1),
                    1.0};
    double amax_x = 0, amax_y = 0;
    for (int j = 0; j < controls->count; ++j) {
        amax_x = std::fmax(amax_x, std::fabs(controls->a[2 * j]));
        amax_y = std::fmax(amax_y, std::fabs(controls->a[2 * j + 1]));
    }
    unsigned hm[3] = {0u, 0u, 0u};
    CK(cudaMemsetAsync(d_red, 0, 3 * sizeof(unsigned), st));
    if (speed) hjbh::launch_absmax(speed, N, 1, 0, d_red, st);
    if (dyn->current) {
        hjbh::launch_absmax(dyn->current, N, 2, 0, d_red + 1, st);
        hjbh::launch_absmax(dyn->current, N, 2, 1, d_red + 2, st);
    }
    CK(cudaMemcpyAsync(hm, d_red, sizeof hm, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    float fm[3];
    std::memcpy(fm, hm, sizeof fm);
    const double smax = speed ? fm[0] : 1.0;
    const double moff = std::fmax((smax * amax_x + fm[1]) * disc->h / dx[0],
                                  (smax * amax_y + fm[2]) * disc->h / dx[1]);
    if (!std::isfinite(moff)) return fail(HJB_ERR_INVALID_ARG, "a field is not finite");
    const int need = static_cast<int>(std::floor(moff)) + 1;
    if (need > 4) return fail(HJB_ERR_UNSUPPORTED, "feet move %.3f cells per step (< 4 supported)", moff);
    const int halo = need <= 2 ? 2 : 4;

    // the slot: the whole grid, W form when the running cost is constant
    const bool wform = cost->l == nullptr;
    const double lconst = cost->l ? 1.0 : cost->l_const;
    const double beta = beta_w(disc->weights, disc->lambda, disc->h);
    const double gamma = gamma_w(disc->weights, disc->lambda, disc->h);
    const double c = lconst / disc->lambda;
    SlotDesc S;
    std::memset(&S, 0, sizeof S);
    S.V[0] = reinterpret_cast<float *>(base + o_v0);
    S.V[1] = reinterpret_cast<float *>(base + o_v1);
    S.speed = speed;
    S.current = dyn->current;
    S.cost = wform ? nullptr : cost->l;
    S.labels = target->labels;
    S.nx = nx;
    S.ny = ny;
    S.nz = 1;
    S.pitch = pitch;
    S.zstride = static_cast<long long>(pitch) * ny;
    S.tiles_x = (nx + hjbk::TX - 1) / hjbk::TX;
    S.tiles_y = (ny + rows - 1) / rows;
    S.tiles_z = 1;
    S.ntiles = tiles;
    S.halo = halo;
    S.hx = static_cast<float>(disc->h / dx[0]);
    S.hy = static_cast<float>(disc->h / dx[1]);
    S.beta = static_cast<float>(beta);
    S.gamma = static_cast<float>(gamma);
    S.gl = static_cast<float>(gamma * lconst);
    S.vout = static_cast<float>(wform ? c - target->value_out : target->value_out);
    S.vtarget = static_cast<float>(wform ? c : 0.0);
    S.tol = static_cast<float>((opts && opts->tol > 0) ? opts->tol : 0.5e-4 * (1.0 - beta));
    S.max_iters = (opts && opts->max_iters > 0) ? opts->max_iters : 100000;
    TRY(encode_maps(S, 2, halo, rows));
    CK(cudaMemcpyAsync(d_slot, &S, sizeof S, cudaMemcpyHostToDevice, st));
    hjbk::ControlTable ctrl;
    std::memset(&ctrl, 0, sizeof ctrl);
    ctrl.count = controls->count;
    for (int j = 0; j < controls->count; ++j) {
        ctrl.ax[j] = controls->a[2 * j];
        ctrl.ay[j] = controls->a[2 * j + 1];
        ctrl.a2[j] = make_float2(ctrl.ax[j], ctrl.ay[j]);
    }
    const float c_over = static_cast<float>(c);
    hjbh::launch_init_values(d_slot, 1, static_cast<int>(N), wform ? 1 : 0, c_over,
                             opts ? opts->v_init : nullptr, st);
    hjbh::launch_loop_init(d_slot, d_state, d_ctl, 1, st);
    hjbk::SweepArgs args;
    std::memset(&args, 0, sizeof args);
    args.slots = d_slot;
    args.state = d_state;
    args.ctl = d_ctl;
    args.qlist[0] = reinterpret_cast<int *>(base + o_qlist);
    args.qlist[1] = args.qlist[0] + tiles;
    args.qflag[0] = base + o_qflag;
    args.qflag[1] = base + o_qflag + fb;
    args.nslots = 1;
    args.use_handle = 0;
    args.stall_tol = 8.0f * 1.1920929e-7f;
    args.local_iters = local_iters(opts, nullptr);
    args.dyn_queue = queue_mode();
    args.ctrl = ctrl;
    hjbh::launch_queue_init(d_slot, 1, tiles, d_ctl, args.qlist[0], args.qflag[0], args.qflag[1], st);
    const hjbh::SweepKey key{0, wform ? 1 : 0, controls->count, halo, rows, 1, 1, 1, 1};
    const void *fn = hjbh::sweep_kernel(key, nullptr);
    if (!fn) return fail(HJB_ERR_UNSUPPORTED, "no sweep kernel for this configuration");
    const int gridsz = hjbh::sweep_grid(key);
    void *argv[1] = {&args};
    CK(cudaLaunchCooperativeKernel(fn, dim3(gridsz), dim3(hjbk::THREADS), argv, 0, st));
    hjbh::launch_extract(d_slot, d_state, 0, v_out, wform ? 1 : 0, c_over, st);
    SlotState hs;
    int herr[2] = {0, 0};
    CK(cudaMemcpyAsync(&hs, d_state, sizeof hs, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(herr, &d_ctl->error, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    if (stats) {
        fill_stats(stats, hs);
        stats->launches = (dyn->log_speed ? 1 : 0) + (speed ? 1 : 0) + (dyn->current ? 2 : 0) + 5;
        stats->tile_rows = rows;
        stats->tile_lanes = 1;
        stats->local_iters = args.local_iters;
    }
    if (herr[0]) return fail(HJB_ERR_TIMEOUT, "a bounded device wait gave up");
    if (!hs.converged)
        return fail(HJB_ERR_NOT_CONVERGED, "not converged after %d iterations (residual %g)", hs.iters,
                    hs.final_res);
    return HJB_OK;
}
