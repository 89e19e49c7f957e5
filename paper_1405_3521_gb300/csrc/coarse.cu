// coarse.cu -- RA step 1 of Festa (arXiv:1405.3521), Sec. 3: the m auxiliary
// problems V_k = T_k(V_k) on the coarse grid K, each with target component k
// only, solved to convergence entirely in on-chip memory.
//
// A coarse auxiliary problem is small (65 x 65 nodes, 17 KB, at the 1025^2
// workloads with stride 16) but needs about a hundred applications of T, so
// the tile-queue sweep spends much of its time on per-sweep fixed costs.
// Here each auxiliary problem gets one thread-block cluster of CL CTAs: CTA r
// of the cluster owns a band of rows of V_k, one node per thread, and keeps
// the band plus its interpolation halo rows in shared memory.  An
// application of T reads the band through a pair layout (V[c], V[c+1]) built
// from the current values, writes the new values into the other of two raw
// buffers (Jacobi) and pushes the rows that neighbouring bands read as halo
// into the neighbours' raw buffers (distributed shared memory); each CTA's
// L-inf change goes into a slot of its own shared memory, and one cluster
// barrier publishes both.  Every CTA then reads the same CL residual slots
// and takes the same stopping decision, so the CTAs of a cluster leave the
// loop together.  The iteration is the plain value iteration V^{n+1} =
// T(V^n) of Sec. 3 with the stopping rule of the tile sweep (||V^{n+1} -
// V^n|| <= tol, the iteration cap, or stagnation at rounding level).  The
// result is written to the slot's iteration buffer 0, where the labelling
// kernels read it.
//
// The evaluation of a control at a node is the one of the tile sweep: the
// foot by packed FP32x2 arithmetic, its cell and fractions with the 2^23
// magic constant, the four corner values as two 64-bit shared loads of the
// pair layout and the monotone two-product lerps; feet are tested against
// the box only at nodes near it.
#include <cooperative_groups.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "hjb_internal.cuh"

namespace cg = cooperative_groups;
using namespace hjbk;

namespace {

constexpr int CL = 8;        // CTAs per cluster (one cluster per auxiliary problem)
constexpr int CT = 1024;     // threads per CTA: one band node per thread
constexpr int CPW = 128;     // float2 per pair row (1 KB rows: the row address is a shift by 10)
constexpr int CXP = 4;       // columns of padding left of the grid in the pair layout
constexpr float FACE = 1e-6f;  // reading R2: feet within 1e-6 cells of a face are on it
constexpr float MAGIC = 8388607.5f;
constexpr float TWO23 = 8388608.0f;
constexpr int TWO23_BITS = 0x4B000000;

struct CoarseArgs {
    const SlotDesc *slots;
    SlotState *state;
    int m;
    int halo;       // interpolation halo in rows (a foot moves fewer than halo cells)
    int band_max;   // rows of the largest band
    int nbands;     // bands in use (<= CL); CTAs of rank >= nbands hold no rows
    float stall_tol;
    ControlTable ctrl;
};

// Rows [y0, y1) of band r of nb bands over ny rows.
__device__ __forceinline__ int band_start(int r, int nb, int ny) {
    return static_cast<int>((static_cast<long long>(r) * ny) / nb);
}

template <bool WFORM>
__device__ __forceinline__ float pick(float best, float q) {
    return WFORM ? fmaxf(best, q) : fminf(best, q);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Q1 interpolation of the pair layout at local coordinates P2 = (px, py)
// (px >= 0, py >= 0, so that the magic constant gives a cell index k >= 0
// with p - k in [0, 1]).  K is the shared address of the pair array minus
// the magic-constant bias: pair (ky, kx) sits at (bits(my) << 10) + (bits(mx)
// << 3) + K.
__device__ __forceinline__ float q1c(float2 P2, uint32_t K) {
    const float2 M2 = __fadd2_rn(P2, make_float2(MAGIC, MAGIC));
    const float2 Kn = __ffma2_rn(M2, make_float2(-1.0f, -1.0f), make_float2(TWO23, TWO23));
    const float2 F2 = __fadd2_rn(P2, Kn);  // (fx, fy) = p - k
    const uint32_t addr = (__float_as_uint(M2.y) << 10) + (__float_as_uint(M2.x) << 3) + K;
    float lo0, lo1, hi0, hi1;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(lo0), "=f"(lo1) : "r"(addr));
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+1024];" : "=f"(hi0), "=f"(hi1) : "r"(addr));
    // (1-f) a as fma(-f, a, a): a (1-f) rounded once
    const float2 lo = make_float2(lo0, lo1);
    const float2 ab = __ffma2_rn(make_float2(F2.y, F2.y), make_float2(hi0, hi1),
                                 __ffma2_rn(make_float2(-F2.y, -F2.y), lo, lo));
    return fmaf(F2.x, ab.y, fmaf(-F2.x, ab.x, ab.x));
}

// P1 variant: the triangle of the cell's split along its (0,0)-(1,1) diagonal.
__device__ __forceinline__ float p1c(float2 P2, uint32_t K) {
    const float2 M2 = __fadd2_rn(P2, make_float2(MAGIC, MAGIC));
    const float2 Kn = __ffma2_rn(M2, make_float2(-1.0f, -1.0f), make_float2(TWO23, TWO23));
    const float2 F2 = __fadd2_rn(P2, Kn);
    const uint32_t addr = (__float_as_uint(M2.y) << 10) + (__float_as_uint(M2.x) << 3) + K;
    float lo0, lo1, hi0, hi1;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(lo0), "=f"(lo1) : "r"(addr));
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+1024];" : "=f"(hi0), "=f"(hi1) : "r"(addr));
    const bool lower = F2.x >= F2.y;
    const float t1 = lower ? F2.x : F2.y, t2 = lower ? F2.y : F2.x;
    const float mid = lower ? lo1 : hi0;
    return fmaf(t2, hi1, fmaf(t1 - t2, mid, fmaf(-t1, lo0, lo0)));
}

template <bool P1>
__device__ __forceinline__ float interp(float2 P2, uint32_t K) {
    return P1 ? p1c(P2, K) : q1c(P2, K);
}

// One control at a node near the box: a foot whose offset leaves the closed
// box by more than FACE cells takes vout; feet within FACE are clamped onto
// the face.  b = (x lo, x hi, y lo, y hi) offset bounds; BASE2: the node's
// local coordinates.
template <bool WFORM, bool P1>
__device__ __forceinline__ float edge_value(uint32_t K, float2 O2, float4 b, float2 BASE2, float vout,
                                            float best) {
    const bool out = (O2.x < b.x - FACE) | (O2.x > b.y + FACE) | (O2.y < b.z - FACE) |
                     (O2.y > b.w + FACE);
    O2.x = fminf(fmaxf(O2.x, b.x), b.y);
    O2.y = fminf(fmaxf(O2.y, b.z), b.w);
    const float q = interp<P1>(__fadd2_rn(O2, BASE2), K);
    return pick<WFORM>(best, out ? vout : q);
}

// T's extremum over the controls at a free node (games: the max over b of
// the min over a, in the W form the min of the max).  NA > 0: that many
// controls with compile-time indices (constant-bank operands).
template <int NA, bool WFORM, bool P1>
__device__ __forceinline__ float node_value(const ControlTable &C, uint32_t K, float2 S2, float2 O02,
                                            float2 BASE2, bool edge, float4 b, float vout) {
    float best = WFORM ? -INFINITY : INFINITY;
    if constexpr (NA > 0) {
        if (!edge) {
            const float2 B2 = __fadd2_rn(BASE2, O02);
#pragma unroll
            for (int j = 0; j < NA; ++j)
                best = pick<WFORM>(best, interp<P1>(__ffma2_rn(S2, C.a2[j], B2), K));
        } else {
#pragma unroll 8
            for (int j = 0; j < NA; ++j)
                best = edge_value<WFORM, P1>(K, __ffma2_rn(S2, C.a2[j], O02), b, BASE2, vout, best);
        }
        return best;
    } else {
        const int na = C.count, nbk = C.nb > 1 ? C.nb : 1, nA = na / nbk;
        float outer = WFORM ? INFINITY : -INFINITY;
        for (int kb = 0; kb < na; kb += nA) {
            float inner = WFORM ? -INFINITY : INFINITY;
#pragma unroll 4
            for (int j = kb; j < kb + nA; ++j)
                inner = edge_value<WFORM, P1>(K, __ffma2_rn(S2, C.a2[j], O02), b, BASE2, vout, inner);
            outer = nbk > 1 ? (WFORM ? fminf(outer, inner) : fmaxf(outer, inner)) : inner;
        }
        return outer;
    }
}

template <int NA, bool WFORM, bool P1>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(CT, 1)
    coarse_solve_kernel(const __grid_constant__ CoarseArgs a) {
    extern __shared__ __align__(16) float smem[];
    __shared__ float s_res[2];   // this CTA's change over an application, by parity
    __shared__ float s_red[CT / 32];
    __shared__ float s_r;
    __shared__ int s_free[CT / 32];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = static_cast<int>(cluster.block_rank());
    const int k = blockIdx.x / CL;
    const SlotDesc &S = a.slots[k];
    const int nx = S.nx, ny = S.ny, H = a.halo, nb = a.nbands;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int y0 = rank < nb ? band_start(rank, nb, ny) : 0;
    const int y1 = rank < nb ? band_start(rank + 1, nb, ny) : 0;
    const int row0 = y0 - H;                    // grid row of buffer row 0
    const int brows = a.band_max + 2 * H;       // rows per buffer
    const int bsz = brows * nx;                 // floats per raw buffer
    float2 *pairs = reinterpret_cast<float2 *>(smem);  // [brows][CPW]
    float *raw = smem + 2 * brows * CPW;               // [2][brows][nx]
    const int nodes = (y1 - y0) * nx;
    const uint32_t K = smem_u32(pairs) - (static_cast<uint32_t>(TWO23_BITS) << 10) -
                       (static_cast<uint32_t>(TWO23_BITS) << 3);

    // starting iterate on the band and its halo rows: targets vtarget, free
    // nodes vout (in the W form: the value of never arriving); the pair
    // layout's padding holds zeros (read only with weight 0)
    for (int i = tid; i < brows * CPW; i += CT) pairs[i] = make_float2(0.0f, 0.0f);
    // rows of the buffers beyond the grid (halo of the first and last band)
    // stay zero: the interpolation reads them only with weight 0
    for (int i = tid; i < 2 * bsz; i += CT) raw[i] = 0.0f;
    __syncthreads();
    const int ylo = max(y0 - H, 0), yhi = min(y1 + H, ny);
    for (int i = tid; i < (yhi - ylo) * nx; i += CT) {
        const int gy = ylo + i / nx, gx = i - (i / nx) * nx;
        const int lab = S.labels[static_cast<long long>(gy) * nx + gx];
        const bool tgt = lab != 0 && (S.only_target == 0 || lab == S.only_target);
        const float v = tgt ? S.vtarget : S.vout;
        raw[(gy - row0) * nx + gx] = v;
        raw[bsz + (gy - row0) * nx + gx] = v;
    }
    // this thread's node: class, fields and local coordinates, fixed over
    // the iterations
    const bool has = tid < nodes;
    const int gy = has ? y0 + tid / nx : y0, gx = has ? tid - (tid / nx) * nx : 0;
    const long long gi = static_cast<long long>(gy) * nx + gx;
    bool isfree = false, edge = false;
    float2 S2 = make_float2(0.0f, 0.0f), O02 = S2;
    float add = S.gl;
    float4 bnd = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (has) {
        const int lab = S.labels[gi];
        isfree = !(lab != 0 && (S.only_target == 0 || lab == S.only_target));
        float sx = 1.0f, sy = 1.0f;
        if (S.scale2) {
            const float2 d = S.scale2[gi];
            sx = d.x;
            sy = d.y;
        } else if (S.speed) {
            sx = sy = S.speed[gi];
        }
        float cx = 0.0f, cy = 0.0f;
        if (S.current) {
            const float2 c = reinterpret_cast<const float2 *>(S.current)[gi];
            cx = c.x;
            cy = c.y;
        }
        S2 = make_float2(sx * S.hx, sy * S.hy);
        O02 = make_float2(cx * S.hx, cy * S.hy);
        if (!WFORM && S.cost) add = S.gamma * S.cost[gi];
        // a foot moves fewer than H cells: nodes H or more cells inside the
        // box never leave it (games and generic counts always test)
        edge = NA <= 0 || gx < H || gx > nx - 1 - H || gy < H || gy > ny - 1 - H;
        bnd = make_float4(-static_cast<float>(gx), static_cast<float>(nx - 1 - gx),
                          -static_cast<float>(gy), static_cast<float>(ny - 1 - gy));
    }
    const float2 BASE2 = make_float2(static_cast<float>(gx + CXP), static_cast<float>(gy - row0));
    const int lrow = gy - row0;
    int nfree = isfree ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) nfree += __shfl_xor_sync(0xffffffffu, nfree, o);
    if (lane == 0) s_free[warp] = nfree;
    if (tid < 2) s_res[tid] = 0.0f;
    // the neighbours' buffers are initialised before anyone pushes into them
    cluster.sync();

    const float beta = S.beta;
    float best_res = INFINITY;
    int stall = 0, iters = 0, converged = 0;
    int cur = 0;
    float vcur = has ? raw[lrow * nx + gx] : 0.0f;
    for (;;) {
        const float *B = raw + cur * bsz;
        float *D = raw + (cur ^ 1) * bsz;
        // pair layout of the current values (band and halo rows); the
        // previous application's reads of it ended at its cluster barrier
        for (int i = tid; i < brows * (nx + 1); i += CT) {
            const int r = i / (nx + 1), c = i - r * (nx + 1) - 1;  // c in [-1, nx - 1]
            const float lo = c >= 0 ? B[r * nx + c] : 0.0f;
            const float hi = c + 1 < nx ? B[r * nx + c + 1] : 0.0f;
            pairs[r * CPW + c + CXP] = make_float2(lo, hi);
        }
        __syncthreads();
        float v = vcur;
        if (isfree) {
            const float best =
                node_value<NA, WFORM, P1>(a.ctrl, K, S2, O02, BASE2, edge, bnd, S.vout);
            v = WFORM ? beta * best : fmaf(beta, best, add);
        }
        float rmax = isfree ? fabsf(v - vcur) : 0.0f;
        if (has) {
            D[lrow * nx + gx] = v;
            // rows that other bands read as halo: push into their buffers
            if (gy < y0 + H && rank > 0) {
                float *nbuf = cluster.map_shared_rank(D, rank - 1);
                nbuf[(gy - (band_start(rank - 1, nb, ny) - H)) * nx + gx] = v;
            }
            if (gy >= y1 - H && rank + 1 < nb) {
                float *nbuf = cluster.map_shared_rank(D, rank + 1);
                nbuf[(gy - (band_start(rank + 1, nb, ny) - H)) * nx + gx] = v;
            }
        }
        vcur = v;
        for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        if (lane == 0) s_red[warp] = rmax;
        __syncthreads();
        if (warp == 0) {
            float r = lane < CT / 32 ? s_red[lane] : 0.0f;
            for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
            if (lane == 0) s_res[iters & 1] = r;
        }
        // the application's values, halo pushes and residual slots are visible
        cluster.sync();
        if (warp == 0) {
            float r = 0.0f;
            if (lane < CL) r = *cluster.map_shared_rank(&s_res[iters & 1], lane);
            for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
            if (lane == 0) s_r = r;
        }
        __syncthreads();
        const float r = s_r;
        ++iters;
        cur ^= 1;
        // the stopping rule of the tile sweep, taken identically by every CTA
        if (r <= S.tol) {
            converged = 1;
            break;
        }
        if (iters >= S.max_iters) break;
        if (r < best_res) {
            best_res = r;
            stall = 0;
        } else if (++stall >= 64 && r <= a.stall_tol) {
            converged = 2;
            break;
        }
    }
    // the latest iterate of the band to the slot's buffer 0
    if (has) S.V[0][static_cast<long long>(gy) * S.pitch + gx] = vcur;
    if (tid == 0) {
        int f = 0;
        for (int w = 0; w < CT / 32; ++w) f += s_free[w];
        SlotState &st = a.state[k];
        atomicAdd(&st.updates, static_cast<unsigned long long>(f) * iters);
        if (rank == 0) {
            st.iters = iters;
            st.converged = converged;
            st.done = 1;
            st.final_parity = 0;
            st.final_res = s_r;
            st.best_res = best_res;
            st.visits = 0u;
        }
    }
    // no CTA leaves while a neighbour may still read its residual slot
    cluster.sync();
}

}  // namespace

namespace hjbh {

int coarse_fits(int nx, int ny, int halo, size_t *smem_bytes, int *nbands, int *band_max) {
    // bands of at least `halo` rows, so that a band's halo rows come from its
    // two neighbours only; one band node per thread; the padded row of the
    // pair layout holds the grid's width
    int nb = ny / halo;
    if (nb > CL) nb = CL;
    if (nb < 1) return 0;
    const int bmax = (ny + nb - 1) / nb;
    if (static_cast<long long>(bmax) * nx > CT || nx + 2 * CXP > CPW) return 0;
    const size_t bytes = (bmax + 2ull * halo) * (CPW * sizeof(float2) + 2ull * nx * sizeof(float));
    if (bytes > 200u * 1024u) return 0;
    if (smem_bytes) *smem_bytes = bytes;
    if (nbands) *nbands = nb;
    if (band_max) *band_max = bmax;
    return 1;
}

int launch_coarse_solve(const SlotDesc *slots, SlotState *state, int m, int nx, int ny, int halo,
                        int interp, int wform, const ControlTable &ctrl, float stall_tol,
                        cudaStream_t st) {
    size_t smem = 0;
    int nb = 0, bmax = 0;
    if (!coarse_fits(nx, ny, halo, &smem, &nb, &bmax)) return -1;
    CoarseArgs a;
    a.slots = slots;
    a.state = state;
    a.m = m;
    a.halo = halo;
    a.band_max = bmax;
    a.nbands = nb;
    a.stall_tol = stall_tol;
    a.ctrl = ctrl;
    const bool game = ctrl.nb > 1;
    const void *fn = nullptr;
#define HJB_COARSE(NA_)                                                                          \
    fn = interp ? (wform ? reinterpret_cast<const void *>(&coarse_solve_kernel<NA_, true, true>)  \
                         : reinterpret_cast<const void *>(&coarse_solve_kernel<NA_, false, true>)) \
                : (wform ? reinterpret_cast<const void *>(&coarse_solve_kernel<NA_, true, false>)  \
                         : reinterpret_cast<const void *>(&coarse_solve_kernel<NA_, false, false>))
    if (!game && ctrl.count == 64) {
        HJB_COARSE(64);
    } else if (!game && ctrl.count == 32) {
        HJB_COARSE(32);
    } else {
        HJB_COARSE(0);
    }
#undef HJB_COARSE
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return -2;
    if (std::getenv("HJB_TUNE_VERBOSE")) {
        // how many of the m clusters the GPU holds at once
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(m * CL);
        cfg.blockDim = dim3(CT);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = CL;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int clusters = -1;
        cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg);
        std::fprintf(stderr, "hjb coarse solve: %d clusters of %d CTAs, %d resident at once, %zu B "
                     "shared memory per CTA\n", m, CL, clusters, smem);
    }
    void *argv[1] = {&a};
    if (cudaLaunchKernel(fn, dim3(m * CL), dim3(CT), argv, smem, st) != cudaSuccess) return -2;
    return 0;
}

}  // namespace hjbh
