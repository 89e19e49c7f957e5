// adjoint.cu -- gradient of a loss on the converged value function with
// respect to a node field (log-speed theta or running cost l).
//
// The paper (Festa, arXiv:1405.3521) stops at the forward solve; with the
// optimal policy pi frozen, the converged fixed point of Sec. 3 is the linear
// system V = beta P_pi V + b, so for a loss L(V):
//     (I - beta P_pi)^T lambda = dL/dV,
//     dL/dtheta_i = lambda_i beta h s_i grad I[V](y_i) . a_pi(i)   (s = e^theta)
//     dL/dl_i     = lambda_i gamma.
// pi is recomputed from V (no per-control data is stored), the transposed
// iteration lambda <- g + beta P_pi^T lambda scatters the Q1 weights of each
// node's foot with atomics, and its L-infinity residual is reduced in the
// same pass that re-arms the next target buffer; the last CTA of that pass
// takes the stopping decision and drives the CUDA-graph loop.
#include <math.h>

#include "hjb_internal.cuh"

using namespace hjbk;
using hjbh::AdjArgs;
using hjbh::AdjCtl;
using hjbh::AdjProblem;
using hjbh::REFINE_ROWS;

namespace {

// Foot of node (gx, gy) under control (ax, ay): the same arithmetic as the
// boundary path of the sweep (cell offsets in FP32, 1e-6-cell tolerance,
// clamping onto the face), returning the cell and the fractions.
struct Foot {
    bool inside;
    int cx, cy;
    float tx, ty;
};

__device__ __forceinline__ Foot foot_of(const AdjProblem &ap, int gx, int gy, float sx, float sy,
                                        float ox0, float oy0, float ax, float ay) {
    Foot f;
    float ox = fmaf(sx, ax, ox0), oy = fmaf(sy, ay, oy0);
    const float lox = -static_cast<float>(gx), hix = static_cast<float>(ap.nx - 1 - gx);
    const float loy = -static_cast<float>(gy), hiy = static_cast<float>(ap.ny - 1 - gy);
    f.inside = !((ox < lox - 1e-6f) | (ox > hix + 1e-6f) | (oy < loy - 1e-6f) | (oy > hiy + 1e-6f));
    ox = fminf(fmaxf(ox, lox), hix);
    oy = fminf(fmaxf(oy, loy), hiy);
    const float kx = floorf(ox), ky = floorf(oy);
    int cx = gx + static_cast<int>(kx), cy = gy + static_cast<int>(ky);
    float tx = ox - kx, ty = oy - ky;
    if (cx > ap.nx - 2) {
        cx = ap.nx - 2;
        tx = 1.0f;
    }
    if (cy > ap.ny - 2) {
        cy = ap.ny - 2;
        ty = 1.0f;
    }
    f.cx = cx;
    f.cy = cy;
    f.tx = tx;
    f.ty = ty;
    return f;
}

struct NodeDyn {
    float sx, sy, ox0, oy0, s;
};

__device__ __forceinline__ NodeDyn node_dyn(const AdjProblem &ap, long long i) {
    NodeDyn d;
    d.s = ap.speed ? ap.speed[i] : 1.0f;
    float cx = 0.0f, cy = 0.0f;
    if (ap.current) {
        const float2 c = reinterpret_cast<const float2 *>(ap.current)[i];
        cx = c.x;
        cy = c.y;
    }
    d.sx = d.s * ap.hx;
    d.sy = d.s * ap.hy;
    d.ox0 = cx * ap.hx;
    d.oy0 = cy * ap.hy;
    return d;
}

#define GRID_STRIDE(i, n)                                                                  \
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < (n); \
         i += static_cast<long long>(gridDim.x) * blockDim.x)

__device__ __forceinline__ double value_f64(const float *V, const float *dV, long long c) {
    return dV ? static_cast<double>(V[c]) + static_cast<double>(dV[c]) : static_cast<double>(V[c]);
}

// The control value I[V + dV](foot) of one control in FP64: the foot
// x + h (s a + c) in grid coordinates, outside the box beyond the 1e-6-cell
// tolerance, clamped onto it otherwise, and the bilinear interpolation of
// the values with the corner weights products of (1 - t) and t.  dV: the
// refinement correction, or null.  Returns false for a foot outside the box.
__device__ __forceinline__ bool control_value_f64(const AdjProblem &ap, const float *V,
                                                  const float *dV, int gx, int gy, double s,
                                                  double cx, double cy, float ax, float ay,
                                                  double &q) {
    const double ox = ap.hd * (s * static_cast<double>(ax) + cx) / ap.dxd;
    const double oy = ap.hd * (s * static_cast<double>(ay) + cy) / ap.dyd;
    if (ox < -static_cast<double>(gx) - 1e-6 || ox > static_cast<double>(ap.nx - 1 - gx) + 1e-6 ||
        oy < -static_cast<double>(gy) - 1e-6 || oy > static_cast<double>(ap.ny - 1 - gy) + 1e-6)
        return false;
    const double px = fmin(fmax(gx + ox, 0.0), static_cast<double>(ap.nx - 1));
    const double py = fmin(fmax(gy + oy, 0.0), static_cast<double>(ap.ny - 1));
    int ix = static_cast<int>(floor(px)), iy = static_cast<int>(floor(py));
    if (ix > ap.nx - 2) ix = ap.nx - 2;
    if (iy > ap.ny - 2) iy = ap.ny - 2;
    const double tx = px - ix, ty = py - iy;
    const double ex = 1.0 - tx, ey = 1.0 - ty;
    const long long c = static_cast<long long>(iy) * ap.nx + ix;
    double acc = (ex * ey) * value_f64(V, dV, c);
    acc += (tx * ey) * value_f64(V, dV, c + 1);
    acc += (ex * ty) * value_f64(V, dV, c + ap.nx);
    acc += (tx * ty) * value_f64(V, dV, c + ap.nx + 1);
    q = acc;
    return true;
}

// FP32 value of one control for the prefilter of the policy decision: the
// bilinear interpolation of V at the clamped foot, v_out outside the box;
// where the foot lies within 1e-4 cells of the box tolerance (so that the
// FP64 test may decide the other way) the smaller of the two.
__device__ __forceinline__ float control_value_f32(const AdjProblem &ap, const float *V, int gx,
                                                   int gy, float sx, float sy, float ox0,
                                                   float oy0, float ax, float ay) {
    const float ox = fmaf(sx, ax, ox0), oy = fmaf(sy, ay, oy0);
    const float lox = -static_cast<float>(gx), hix = static_cast<float>(ap.nx - 1 - gx);
    const float loy = -static_cast<float>(gy), hiy = static_cast<float>(ap.ny - 1 - gy);
    const bool out = (ox < lox - 1e-6f) | (ox > hix + 1e-6f) | (oy < loy - 1e-6f) |
                     (oy > hiy + 1e-6f);
    const bool amb = fabsf(ox - lox) < 1e-4f || fabsf(ox - hix) < 1e-4f ||
                     fabsf(oy - loy) < 1e-4f || fabsf(oy - hiy) < 1e-4f;
    if (out && !amb) return ap.vout;
    const Foot f = foot_of(ap, gx, gy, sx, sy, ox0, oy0, ax, ay);
    const long long c = static_cast<long long>(f.cy) * ap.nx + f.cx;
    const float lo = fmaf(f.tx, V[c + 1], fmaf(-f.tx, V[c], V[c]));
    const float hi = fmaf(f.tx, V[c + ap.nx + 1], fmaf(-f.tx, V[c + ap.nx], V[c + ap.nx]));
    const float q = fmaf(f.ty, hi, fmaf(-f.ty, lo, lo));
    return amb ? fminf(q, ap.vout) : q;
}

// Optimal policy pi_i = argmin_j I[V](foot_j), lowest index on ties.  The
// decision is taken in FP64 (the precision of the FP64 reference), on the
// values V + dV (dV: the refinement correction, or null): in FP32 the
// control values of neighbouring directions, which often differ by less
// than their rounding at this step size, would pick another control at many
// nodes and route adjoint mass differently.  An FP32 pass over every control
// finds the best FP32 value; only controls within `margin` of it (above the
// FP32 error of a control value plus twice max|dV|) are evaluated in FP64.
__global__ void policy_kernel(AdjProblem ap, const __grid_constant__ ControlTable C, const float *V,
                              const float *dV, float margin, int8_t *policy, unsigned *ties) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    unsigned nt = 0;
    GRID_STRIDE(i, N) {
        if (ap.labels[i] != 0) {
            policy[i] = -1;
            continue;
        }
        const int gx = static_cast<int>(i % ap.nx), gy = static_cast<int>(i / ap.nx);
        const NodeDyn nd = node_dyn(ap, i);
        float best32 = INFINITY;
        for (int j = 0; j < C.count; ++j)
            best32 = fminf(best32, control_value_f32(ap, V, gx, gy, nd.sx, nd.sy, nd.ox0, nd.oy0,
                                                     C.ax[j], C.ay[j]));
        const float cut = best32 + margin * fmaxf(1.0f, fabsf(best32));
        const double s = ap.speed ? static_cast<double>(ap.speed[i]) : 1.0;
        double cx = 0.0, cy = 0.0;
        if (ap.current) {
            const float2 c = reinterpret_cast<const float2 *>(ap.current)[i];
            cx = c.x;
            cy = c.y;
        }
        double best = INFINITY, second = INFINITY;
        int arg = 0;
        bool arg_inside = false;
        for (int j = 0; j < C.count; ++j) {
            if (control_value_f32(ap, V, gx, gy, nd.sx, nd.sy, nd.ox0, nd.oy0, C.ax[j],
                                  C.ay[j]) > cut)
                continue;
            double q = ap.vout;
            const bool inside =
                control_value_f64(ap, V, dV, gx, gy, s, cx, cy, C.ax[j], C.ay[j], q);
            if (q < best) {
                second = best;
                best = q;
                arg = j;
                arg_inside = inside;
            } else if (q < second) {
                second = q;
            }
        }
        if (second - best <= 1e-6) ++nt;
        policy[i] = arg_inside ? static_cast<int8_t>(arg) : static_cast<int8_t>(-2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nt += __shfl_xor_sync(0xffffffffu, nt, o);
    if ((threadIdx.x & 31) == 0 && nt) atomicAdd(ties, nt);
}

// The foot of each node's policy control (FP32, the arithmetic of the
// sweep's boundary path): corner cell index and fractions; -1 for targets,
// -2 for a foot outside the box.
__global__ void feet_kernel(AdjProblem ap, const __grid_constant__ ControlTable C,
                            const int8_t *policy, int *cell, float2 *frac) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    GRID_STRIDE(i, N) {
        const int p = policy[i];
        if (p < 0) {
            cell[i] = p == -1 ? -1 : -2;
            frac[i] = make_float2(0.0f, 0.0f);
            continue;
        }
        const int gx = static_cast<int>(i % ap.nx), gy = static_cast<int>(i / ap.nx);
        const NodeDyn d = node_dyn(ap, i);
        const Foot f = foot_of(ap, gx, gy, d.sx, d.sy, d.ox0, d.oy0, C.ax[p], C.ay[p]);
        cell[i] = f.cy * ap.nx + f.cx;
        frac[i] = make_float2(f.tx, f.ty);
    }
}

// Iterative refinement (mixed precision) of the values the policy is
// decided on.  The FP32 fixed point V differs from the FP64 one by the
// rounding carried along the characteristics (about 1e-6 at 1025^2), enough
// to pick the runner-up control where two directions are closer than that.
// With the policy pi frozen, V solves the linear system
// V = beta P_pi V + gamma l; its residual r is taken in FP64 and the
// correction dV = r + beta P_pi dV, a small quantity, is iterated in FP32
// (its own rounding is then ~1e-7 of ~1e-6) by refine_tiles.  The policy is decided again on
// V + dV, the exact FP64 values of pi up to that rounding.
__global__ void refine_residual_kernel(AdjProblem ap, const __grid_constant__ ControlTable C,
                                       const float *V, const int8_t *policy, float *r) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    GRID_STRIDE(i, N) {
        const int p = policy[i];
        if (p == -1) {
            r[i] = 0.0f;  // target (value fixed)
            continue;
        }
        double q = ap.vout;  // p == -2: the best foot leaves the box
        if (p >= 0) {
            const int gx = static_cast<int>(i % ap.nx), gy = static_cast<int>(i / ap.nx);
            const double s = ap.speed ? static_cast<double>(ap.speed[i]) : 1.0;
            double cx = 0.0, cy = 0.0;
            if (ap.current) {
                const float2 c = reinterpret_cast<const float2 *>(ap.current)[i];
                cx = c.x;
                cy = c.y;
            }
            control_value_f64(ap, V, nullptr, gx, gy, s, cx, cy, C.ax[p], C.ay[p], q);
        }
        const double l = ap.cost ? static_cast<double>(ap.cost[i]) : ap.lconst;
        r[i] = static_cast<float>(ap.betad * q + ap.gammad * l - static_cast<double>(V[i]));
    }
}

// Block Gauss-Seidel sweep of the refinement iteration dV = r + beta P_pi dV
// with the policy frozen: each CTA stages a tile of 32 x REFINE_ROWS nodes of
// dV_src with an hr-cell halo in shared memory, applies the iteration
// APPS times there (the halo held at the previous sweep's values; two
// buffers, so every application reads only the previous one: the result does
// not depend on the order of the CTAs), and writes the tile to dV_dst.  The
// same fixed point as the Jacobi iteration, reached in a fraction of the
// launches because a correction travels APPS steps within a tile per
// sweep.  The last CTA takes the stopping decision: the sweep's change
// within 4 ulp of max|dV| (the FP32 floor of the iteration), or 64 sweeps
// without a new minimum once below 64 ulp, or the sweep cap; a foot beyond
// the staged halo (which the halo derived from the fields rules out) stops
// the loop with the error flag set.
template <int APPS>
__global__ void refine_tiles(const __grid_constant__ AdjArgs A) {
    static_assert(TX * REFINE_ROWS == THREADS, "one thread per node of a refinement tile");
    extern __shared__ float s_buf[];
    AdjCtl *ctl = A.ctl;
    if (ctl->converged) return;
    const AdjProblem &ap = A.ap;
    const int hr = A.hr;
    const int W = TX + 2 * hr, HH = REFINE_ROWS + 2 * hr, SZ = W * HH;
    const int nx = ap.nx, ny = ap.ny;
    const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + REFINE_ROWS - 1) / REFINE_ROWS;
    const int par = ctl->parity;
    const float *src = A.L[par];
    float *dst = A.L[par ^ 1];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    float rmax = 0.0f, amax = 0.0f;
    bool bad = false;
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        const int x0 = tx * TX - hr, y0 = ty * REFINE_ROWS - hr;
        __syncthreads();  // the previous tile is done with the buffers
        for (int k = threadIdx.x; k < SZ; k += THREADS) {
            const int sy = k / W, sx = k - sy * W;
            const int gx = x0 + sx, gy = y0 + sy;
            const float v = (gx >= 0 && gx < nx && gy >= 0 && gy < ny)
                                ? __ldcg(src + static_cast<long long>(gy) * nx + gx)
                                : 0.0f;
            s_buf[k] = v;
            s_buf[SZ + k] = v;
        }
        const int gx = tx * TX + lx, gy = ty * REFINE_ROWS + ly;
        const bool in = gx < nx && gy < ny;
        const long long i = static_cast<long long>(gy) * nx + gx;
        int c = -1;
        float r = 0.0f;
        float2 f = make_float2(0.0f, 0.0f);
        int lc = 0;
        if (in) {
            c = A.cell[i];
            if (c != -1) r = A.g[i];
            if (c >= 0) {
                f = A.frac[i];
                const int cy = c / nx, cx = c - cy * nx;
                const int sx = cx - x0, sy = cy - y0;
                if (sx < 0 || sx + 1 >= W || sy < 0 || sy + 1 >= HH) {
                    bad = true;  // a foot beyond the halo: never with hr from the fields
                    c = -2;
                } else {
                    lc = sy * W + sx;
                }
            }
        }
        const int me = (ly + hr) * W + lx + hr;
        __syncthreads();
        const float dold = in ? s_buf[me] : 0.0f;
        float d = dold;
#pragma unroll 1
        for (int a = 0; a < APPS; ++a) {
            const float *cur = s_buf + (a & 1) * SZ;
            float *nxt = s_buf + ((a + 1) & 1) * SZ;
            if (in) {
                d = 0.0f;
                if (c != -1) {
                    d = r;
                    if (c >= 0) {
                        const float lo = fmaf(f.x, cur[lc + 1], fmaf(-f.x, cur[lc], cur[lc]));
                        const float hi = fmaf(f.x, cur[lc + W + 1],
                                              fmaf(-f.x, cur[lc + W], cur[lc + W]));
                        d = fmaf(ap.beta, fmaf(f.y, hi, fmaf(-f.y, lo, lo)), d);
                    }
                }
                nxt[me] = d;
            }
            __syncthreads();
        }
        if (in) {
            dst[i] = d;
            rmax = fmaxf(rmax, fabsf(d - dold));
            amax = fmaxf(amax, fabsf(d));
        }
    }
    if (bad) atomicExch(&ctl->error, 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    __shared__ float s_r[THREADS / 32], s_a[THREADS / 32];
    __shared__ int s_last;
    if (lx == 0) {
        s_r[ly] = rmax;
        s_a[ly] = amax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = s_r[0], ma = s_a[0];
        for (int w = 1; w < THREADS / 32; ++w) {
            m = fmaxf(m, s_r[w]);
            ma = fmaxf(ma, s_a[w]);
        }
        atomicMax(&ctl->res_bits, __float_as_uint(m));
        atomicMax(&ctl->lam_bits, __float_as_uint(ma));
        __threadfence();
        s_last = (atomicAdd(&ctl->done_ctas, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const float res = __uint_as_float(ctl->res_bits);
        const float am = __uint_as_float(ctl->lam_bits);
        ctl->res_bits = 0u;
        ctl->lam_bits = 0u;
        ctl->iters += 1;
        ctl->final_res = res;
        ctl->lam_max = am;
        ctl->parity = par ^ 1;
        ctl->done_ctas = 0u;
        constexpr float EPS = 1.1920929e-7f;
        if (res < ctl->best_res) {
            ctl->best_res = res;
            ctl->stall = 0;
        } else {
            ctl->stall += 1;
        }
        if (ctl->error)
            ctl->converged = 3;
        else if (res <= 4.0f * EPS * am || (ctl->stall >= 64 && ctl->best_res <= 64.0f * EPS * am))
            ctl->converged = 2;
        else if (ctl->iters >= ctl->max_iters)
            ctl->converged = 3;
        __threadfence();
        if (A.use_handle) cudaGraphSetConditional(A.handle, ctl->converged ? 0u : 1u);
    }
}

// Block Gauss-Seidel sweep of the transposed iteration lambda = g +
// beta P_pi^T lambda (dL/dV = g).  Each CTA owns a tile of 32 x REFINE_ROWS
// nodes.  The mass that the tile's hr-cell halo (the nodes whose policy feet
// can reach the tile) sends into it, beta times the Q1 weight times lambda,
// is constant during the sweep (the halo is held at the previous sweep's
// values): it is added to g once, in shared memory.  Then APPS times
// every tile node's lambda becomes that base plus the mass the tile's own
// nodes send it (shared-memory atomics), and the tile's lambda is written at
// the end.  Mass that leaves the tile is gathered by the neighbouring
// tile, whose halo holds this one.  As with the scattered global atomics
// this replaces, the order of the additions is not fixed, so lambda is
// reproducible to its FP32 rounding.  The last CTA takes the stopping
// decision: the sweep's change within 32 ulp of max|lambda|, or 64 sweeps
// without a new minimum once below 1024 ulp, or an optional absolute tol,
// or the sweep cap.
template <int APPS>
__global__ void adj_tiles(const __grid_constant__ AdjArgs A) {
    static_assert(TX * REFINE_ROWS == THREADS, "one thread per node of a tile");
    __shared__ float s_base[THREADS];  // g plus the halo's mass, per tile node
    __shared__ float s_acc[2][THREADS];
    AdjCtl *ctl = A.ctl;
    if (ctl->converged) return;
    const AdjProblem &ap = A.ap;
    const int hr = A.hr;
    const int W = TX + 2 * hr, HH = REFINE_ROWS + 2 * hr, SZ = W * HH;
    const int nx = ap.nx, ny = ap.ny;
    const int tiles_x = (nx + TX - 1) / TX, tiles_y = (ny + REFINE_ROWS - 1) / REFINE_ROWS;
    const int par = ctl->parity;
    const float *src = A.L[par];
    float *dst = A.L[par ^ 1];
    const int lx = threadIdx.x & 31, ly = threadIdx.x >> 5;
    float rmax = 0.0f, amax = 0.0f;
    for (int t = blockIdx.x; t < tiles_x * tiles_y; t += gridDim.x) {
        const int tx = t % tiles_x, ty = t / tiles_x;
        const int x0 = tx * TX - hr, y0 = ty * REFINE_ROWS - hr;
        const int tx0 = tx * TX, ty0 = ty * REFINE_ROWS;
        const int gx = tx0 + lx, gy = ty0 + ly;
        const bool in = gx < nx && gy < ny;
        const long long i = static_cast<long long>(gy) * nx + gx;
        __syncthreads();  // the previous tile is done with the shared arrays
        s_base[threadIdx.x] = in ? A.g[i] : 0.0f;
        __syncthreads();
        // the halo's mass is constant during the sweep: scatter it into the
        // base once (nodes of the tile itself are skipped here)
        for (int k = threadIdx.x; k < SZ; k += THREADS) {
            const int sy = k / W, sx = k - sy * W;
            const int hx = x0 + sx, hy = y0 + sy;
            const bool own = sx >= hr && sx < hr + TX && sy >= hr && sy < hr + REFINE_ROWS;
            if (own || hx < 0 || hx >= nx || hy < 0 || hy >= ny) continue;
            const long long j = static_cast<long long>(hy) * nx + hx;
            const int c = A.cell[j];
            if (c < 0) continue;
            const float bl = ap.beta * __ldcg(src + j);
            if (bl == 0.0f) continue;
            const float2 f = A.frac[j];
            const int cy = c / nx, cx = c - cy * nx;
            const float w[4] = {(1.0f - f.x) * (1.0f - f.y), f.x * (1.0f - f.y),
                                (1.0f - f.x) * f.y, f.x * f.y};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int ex = cx + (e & 1) - tx0, ey = cy + (e >> 1) - ty0;
                if (ex >= 0 && ex < TX && ey >= 0 && ey < REFINE_ROWS)
                    atomicAdd(&s_base[ey * TX + ex], bl * w[e]);
            }
        }
        // this thread's node of the tile: its lambda and the tile-local
        // corners (-1 outside the tile) and weights of its policy foot
        float lam = 0.0f;
        int cn[4] = {-1, -1, -1, -1};
        float wt[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (in) {
            lam = __ldcg(src + i);
            const int c = A.cell[i];
            if (c >= 0) {
                const float2 f = A.frac[i];
                const int cy = c / nx, cx = c - cy * nx;
                const float w[4] = {(1.0f - f.x) * (1.0f - f.y), f.x * (1.0f - f.y),
                                    (1.0f - f.x) * f.y, f.x * f.y};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int ex = cx + (e & 1) - tx0, ey = cy + (e >> 1) - ty0;
                    if (ex >= 0 && ex < TX && ey >= 0 && ey < REFINE_ROWS) {
                        cn[e] = ey * TX + ex;
                        wt[e] = ap.beta * w[e];
                    }
                }
            }
        }
        const float lold = lam;
        __syncthreads();  // the base is complete
        const float base = s_base[threadIdx.x];
#pragma unroll 1
        for (int a = 0; a < APPS; ++a) {
            // two accumulators: this application's is reset while the other
            // may still be read, so two barriers per application suffice
            float *acc = s_acc[a & 1];
            acc[threadIdx.x] = base;
            __syncthreads();
            if (lam != 0.0f) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (cn[e] >= 0) atomicAdd(&acc[cn[e]], lam * wt[e]);
            }
            __syncthreads();
            lam = acc[threadIdx.x];
        }
        if (in) {
            dst[i] = lam;
            rmax = fmaxf(rmax, fabsf(lam - lold));
            amax = fmaxf(amax, fabsf(lam));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    __shared__ float s_r[THREADS / 32], s_a[THREADS / 32];
    __shared__ int s_last;
    if (lx == 0) {
        s_r[ly] = rmax;
        s_a[ly] = amax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = s_r[0], ma = s_a[0];
        for (int w = 1; w < THREADS / 32; ++w) {
            m = fmaxf(m, s_r[w]);
            ma = fmaxf(ma, s_a[w]);
        }
        atomicMax(&ctl->res_bits, __float_as_uint(m));
        atomicMax(&ctl->lam_bits, __float_as_uint(ma));
        __threadfence();
        s_last = (atomicAdd(&ctl->done_ctas, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const float res = __uint_as_float(ctl->res_bits);
        const float lam_max = __uint_as_float(ctl->lam_bits);
        ctl->res_bits = 0u;
        ctl->lam_bits = 0u;
        ctl->iters += 1;
        ctl->final_res = res;
        ctl->lam_max = lam_max;
        ctl->parity = par ^ 1;
        ctl->done_ctas = 0u;
        constexpr float EPS = 1.1920929e-7f;
        if (res < ctl->best_res) {
            ctl->best_res = res;
            ctl->stall = 0;
        } else {
            ctl->stall += 1;
        }
        if (res <= ctl->tol)
            ctl->converged = 1;
        else if (res <= 32.0f * EPS * lam_max ||
                 (ctl->stall >= 64 && ctl->best_res <= 1024.0f * EPS * lam_max))
            ctl->converged = 2;
        else if (ctl->iters >= ctl->max_iters)
            ctl->converged = 3;
        __threadfence();
        if (A.use_handle) cudaGraphSetConditional(A.handle, ctl->converged ? 0u : 1u);
    }
}

__global__ void adj_init_kernel(const float *g, float *L0, float *L1, long long n, AdjCtl *ctl,
                                float tol, int max_iters) {
    GRID_STRIDE(i, n) {
        L0[i] = g[i];
        L1[i] = g[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->done_ctas = 0u;
        ctl->res_bits = 0u;
        ctl->iters = 0;
        ctl->parity = 0;
        ctl->converged = 0;
        ctl->final_res = 0.0f;
        ctl->tol = tol;
        ctl->max_iters = max_iters;
        ctl->error = 0;
        ctl->lam_bits = 0u;
        ctl->lam_max = 0.0f;
        ctl->best_res = INFINITY;
        ctl->stall = 0;
    }
}

__global__ void adj_grad_kernel(AdjProblem ap, const __grid_constant__ ControlTable C, const float *V,
                                const int8_t *policy, const float *lam, int wrt, float *out) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    GRID_STRIDE(i, N) {
        const int p = policy[i];
        float g = 0.0f;
        if (wrt == 1) {
            if (p != -1) g = lam[i] * ap.gamma;  // every free node
        } else if (p >= 0) {
            const int gx = static_cast<int>(i % ap.nx), gy = static_cast<int>(i / ap.nx);
            const NodeDyn d = node_dyn(ap, i);
            const Foot f = foot_of(ap, gx, gy, d.sx, d.sy, d.ox0, d.oy0, C.ax[p], C.ay[p]);
            const long long c = static_cast<long long>(f.cy) * ap.nx + f.cx;
            const float v00 = V[c], v10 = V[c + 1], v01 = V[c + ap.nx], v11 = V[c + ap.nx + 1];
            const float dgx = (1.0f - f.ty) * (v10 - v00) + f.ty * (v11 - v01);
            const float dgy = (1.0f - f.tx) * (v01 - v00) + f.tx * (v11 - v10);
            const float dot = dgx / ap.dx * C.ax[p] + dgy / ap.dy * C.ay[p];
            g = lam[i] * ap.beta * ap.h * d.s * dot;
        }
        out[i] = g;
    }
}

__global__ void points_kernel(int nx, int ny, float lo0, float lo1, float idx0, float idx1,
                              const float *V, const float *pts, int P, float *vals, float *grad) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    float gx = (pts[2 * k] - lo0) * idx0;
    float gy = (pts[2 * k + 1] - lo1) * idx1;
    gx = fminf(fmaxf(gx, 0.0f), static_cast<float>(nx - 1));
    gy = fminf(fmaxf(gy, 0.0f), static_cast<float>(ny - 1));
    int cx = static_cast<int>(floorf(gx)), cy = static_cast<int>(floorf(gy));
    cx = cx > nx - 2 ? nx - 2 : cx;
    cy = cy > ny - 2 ? ny - 2 : cy;
    const float tx = gx - cx, ty = gy - cy;
    const long long c = static_cast<long long>(cy) * nx + cx;
    const float w00 = (1.0f - tx) * (1.0f - ty), w10 = tx * (1.0f - ty), w01 = (1.0f - tx) * ty,
                w11 = tx * ty;
    if (vals) vals[k] = w00 * V[c] + w10 * V[c + 1] + w01 * V[c + nx] + w11 * V[c + nx + 1];
    if (grad) {
        const float s = 1.0f / static_cast<float>(P);
        atomicAdd(grad + c, w00 * s);
        atomicAdd(grad + c + 1, w10 * s);
        atomicAdd(grad + c + nx, w01 * s);
        atomicAdd(grad + c + nx + 1, w11 * s);
    }
}

int blocks_for(long long n) {
    long long b = (n + THREADS - 1) / THREADS;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return static_cast<int>(b);
}

}  // namespace

namespace hjbh {

void launch_policy(const AdjProblem &ap, const ControlTable &C, const float *V, const float *dV,
                   float margin, int8_t *policy, unsigned *ties_out, cudaStream_t st) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    policy_kernel<<<blocks_for(N), THREADS, 0, st>>>(ap, C, V, dV, margin, policy, ties_out);
}

void launch_feet(const AdjProblem &ap, const ControlTable &C, const int8_t *policy, int *cell,
                 float2 *frac, cudaStream_t st) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    feet_kernel<<<blocks_for(N), THREADS, 0, st>>>(ap, C, policy, cell, frac);
}

void launch_refine_residual(const AdjProblem &ap, const ControlTable &C, const float *V,
                            const int8_t *policy, float *r, cudaStream_t st) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    refine_residual_kernel<<<blocks_for(N), THREADS, 0, st>>>(ap, C, V, policy, r);
}

const void *refine_tiles_kernel(int apps) {
    if (apps == 32) return reinterpret_cast<const void *>(&refine_tiles<32>);
    if (apps == 8) return reinterpret_cast<const void *>(&refine_tiles<8>);
    return reinterpret_cast<const void *>(&refine_tiles<16>);
}

size_t refine_tiles_smem(int hr) {
    return 2 * sizeof(float) * static_cast<size_t>(TX + 2 * hr) * (REFINE_ROWS + 2 * hr);
}

int refine_tiles_grid(int nx, int ny) {
    return ((nx + TX - 1) / TX) * ((ny + REFINE_ROWS - 1) / REFINE_ROWS);
}

const void *adj_tiles_kernel(int apps) {
    if (apps == 32) return reinterpret_cast<const void *>(&adj_tiles<32>);
    if (apps == 8) return reinterpret_cast<const void *>(&adj_tiles<8>);
    return reinterpret_cast<const void *>(&adj_tiles<16>);
}

size_t adj_tiles_smem(int) { return 0; }

void launch_adj_init(const float *g, float *L0, float *L1, long long n, AdjCtl *ctl, float tol,
                     int max_iters, cudaStream_t st) {
    adj_init_kernel<<<blocks_for(n), THREADS, 0, st>>>(g, L0, L1, n, ctl, tol, max_iters);
}

void launch_adj_grad(const AdjProblem &ap, const ControlTable &C, const float *V,
                     const int8_t *policy, const float *lam, int wrt, float *out, cudaStream_t st) {
    const long long N = static_cast<long long>(ap.nx) * ap.ny;
    adj_grad_kernel<<<blocks_for(N), THREADS, 0, st>>>(ap, C, V, policy, lam, wrt, out);
}

void launch_points(int nx, int ny, double lo0, double lo1, double dx0, double dx1, const float *V,
                   const float *pts, int P, float *vals, float *grad, cudaStream_t st) {
    points_kernel<<<(P + THREADS - 1) / THREADS, THREADS, 0, st>>>(
        nx, ny, static_cast<float>(lo0), static_cast<float>(lo1), static_cast<float>(1.0 / dx0),
        static_cast<float>(1.0 / dx1), V, pts, P, vals, grad);
}

}  // namespace hjbh
