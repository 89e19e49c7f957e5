// coarse.cu -- RA step 1 of Festa (arXiv:1405.3521), Sec. 3: the m auxiliary
// problems V_k = T_k(V_k) on the coarse grid K, each with target component k
// only, solved to convergence entirely in on-chip memory.
//
// A coarse auxiliary problem is small (65 x 65 nodes, 17 KB, at the 1025^2
// workloads with stride 16) but needs about a hundred applications of T, so
// the tile-queue sweep spends most of its time on per-sweep fixed costs.
// Here each auxiliary problem gets one thread-block cluster of CL CTAs: CTA r
// of the cluster owns a band of rows of V_k and keeps the band plus its
// interpolation halo rows in shared memory (two buffers, Jacobi); after each
// application the rows that neighbouring bands read are pushed into the
// neighbours' shared memory (distributed shared memory), each CTA's L-inf
// change goes into a slot of its own shared memory, and one cluster barrier
// publishes both.  Every CTA then reads the same CL residual slots and takes
// the same stopping decision, so the clusters leave the loop together.  The
// iteration is the plain value iteration V^{n+1} = T(V^n) of Sec. 3 (Jacobi)
// with the stopping rule of the tile sweep (||V^{n+1} - V^n|| <= tol, the
// iteration cap, or stagnation at rounding level).  The result is written
// to the slot's iteration buffer 0, where the labelling kernels read it.
#include <cooperative_groups.h>
#include <math.h>

#include "hjb_internal.cuh"

namespace cg = cooperative_groups;
using namespace hjbk;

namespace {

constexpr int CL = 8;           // CTAs per cluster (one cluster per auxiliary problem)
constexpr int CT = 1024;        // threads per CTA
constexpr float FACE = 1e-6f;   // reading R2: feet within 1e-6 cells of a face are on it

struct CoarseArgs {
    const SlotDesc *slots;
    SlotState *state;
    int m;
    int halo;       // interpolation halo in rows (a foot moves fewer than halo cells)
    int band_max;   // rows of the largest band
    int nbands;     // bands in use (<= CL); CTAs of rank >= nbands hold no rows
    int interp;     // 0 Q1, 1 P1
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

// Interpolation of the band buffer at grid coordinates (px, py), already
// clamped into the box.  Row gy of the grid is buffer row gy - row0.
__device__ __forceinline__ float interp_at(const float *B, int nx, int ny, int row0, float px,
                                           float py, int p1) {
    int ix = static_cast<int>(floorf(px)), iy = static_cast<int>(floorf(py));
    ix = ix < 0 ? 0 : (ix > nx - 2 ? nx - 2 : ix);
    iy = iy < 0 ? 0 : (iy > ny - 2 ? ny - 2 : iy);
    const float fx = px - static_cast<float>(ix), fy = py - static_cast<float>(iy);
    const float *r0 = B + (iy - row0) * nx + ix;
    const float v00 = r0[0], v10 = r0[1], v01 = r0[nx], v11 = r0[nx + 1];
    if (p1) {
        // the triangle of the cell's split along its (0,0)-(1,1) diagonal
        const bool lower = fx >= fy;
        const float t1 = lower ? fx : fy, t2 = lower ? fy : fx;
        const float mid = lower ? v10 : v01;
        return fmaf(t2, v11, fmaf(t1 - t2, mid, (1.0f - t1) * v00));
    }
    // monotone two-product lerps (1 - f) a + f b
    const float a = fmaf(fx, v10, (1.0f - fx) * v00);
    const float b = fmaf(fx, v11, (1.0f - fx) * v01);
    return fmaf(fy, b, (1.0f - fy) * a);
}

// Value of one control (or control pair of a game) at a free node.
template <bool WFORM>
__device__ __forceinline__ float control_value(const SlotDesc &S, const float *B, int row0, int gx,
                                               int gy, float sx, float sy, float ox0, float oy0,
                                               float ax, float ay, int p1) {
    float ox = fmaf(sx, ax, ox0), oy = fmaf(sy, ay, oy0);  // foot offset in cells
    const float lox = -static_cast<float>(gx), hix = static_cast<float>(S.nx - 1 - gx);
    const float loy = -static_cast<float>(gy), hiy = static_cast<float>(S.ny - 1 - gy);
    if (ox < lox - FACE || ox > hix + FACE || oy < loy - FACE || oy > hiy + FACE) return S.vout;
    ox = fminf(fmaxf(ox, lox), hix);
    oy = fminf(fmaxf(oy, loy), hiy);
    return interp_at(B, S.nx, S.ny, row0, static_cast<float>(gx) + ox, static_cast<float>(gy) + oy,
                     p1);
}

template <bool WFORM>
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
    const int bsz = brows * nx;                 // floats per buffer
    const int nodes = (y1 - y0) * nx;
    const float c_tgt = S.vtarget;

    // starting iterate on the band and its halo rows: targets vtarget, free
    // nodes vout (in the W form: the value of never arriving)
    const int ylo = max(y0 - H, 0), yhi = min(y1 + H, ny);
    for (int i = tid; i < (yhi - ylo) * nx; i += CT) {
        const int gy = ylo + i / nx, gx = i - (i / nx) * nx;
        const int lab = S.labels[static_cast<long long>(gy) * nx + gx];
        const bool tgt = lab != 0 && (S.only_target == 0 || lab == S.only_target);
        const float v = tgt ? c_tgt : S.vout;
        smem[(gy - row0) * nx + gx] = v;
        smem[bsz + (gy - row0) * nx + gx] = v;
    }
    int nfree = 0;
    for (int i = tid; i < nodes; i += CT) {
        const int gy = y0 + i / nx, gx = i - (i / nx) * nx;
        const int lab = S.labels[static_cast<long long>(gy) * nx + gx];
        nfree += !(lab != 0 && (S.only_target == 0 || lab == S.only_target));
    }
    for (int o = 16; o > 0; o >>= 1) nfree += __shfl_xor_sync(0xffffffffu, nfree, o);
    if (lane == 0) s_free[warp] = nfree;
    if (tid < 2) s_res[tid] = 0.0f;
    // the neighbours' buffers are initialised before anyone pushes into them
    cluster.sync();

    const float beta = S.beta;
    const int na = a.ctrl.count, nbk = a.ctrl.nb > 1 ? a.ctrl.nb : 1, nA = na / nbk;
    const int p1 = a.interp;
    float best_res = INFINITY;
    int stall = 0, iters = 0, converged = 0;
    int cur = 0;
    for (;;) {
        const float *B = smem + cur * bsz;
        float *D = smem + (cur ^ 1) * bsz;
        float rmax = 0.0f;
        for (int i = tid; i < nodes; i += CT) {
            const int gy = y0 + i / nx, gx = i - (i / nx) * nx;
            const long long gi = static_cast<long long>(gy) * nx + gx;
            const int lab = S.labels[gi];
            const bool tgt = lab != 0 && (S.only_target == 0 || lab == S.only_target);
            float v = c_tgt;
            if (!tgt) {
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
                sx *= S.hx;
                sy *= S.hy;
                const float ox0 = cx * S.hx, oy0 = cy * S.hy;
                // games: the max over b of the min over a (W form: min of max)
                float outer = WFORM ? INFINITY : -INFINITY;
                for (int kb = 0; kb < na; kb += nA) {
                    float inner = WFORM ? -INFINITY : INFINITY;
#pragma unroll 4
                    for (int j = kb; j < kb + nA; ++j)
                        inner = pick<WFORM>(inner, control_value<WFORM>(S, B, row0, gx, gy, sx, sy,
                                                                         ox0, oy0, a.ctrl.ax[j],
                                                                         a.ctrl.ay[j], p1));
                    outer = nbk > 1 ? (WFORM ? fminf(outer, inner) : fmaxf(outer, inner)) : inner;
                }
                v = WFORM ? beta * outer
                          : fmaf(beta, outer, S.cost ? S.gamma * S.cost[gi] : S.gl);
                rmax = fmaxf(rmax, fabsf(v - B[(gy - row0) * nx + gx]));
            }
            D[(gy - row0) * nx + gx] = v;
            // rows that other bands read as halo: push into their buffers
            if (gy < y0 + H && rank > 0) {
                float *nbuf = cluster.map_shared_rank(D, rank - 1);
                const int nrow0 = band_start(rank - 1, nb, ny) - H;
                nbuf[(gy - nrow0) * nx + gx] = v;
            }
            if (gy >= y1 - H && rank + 1 < nb) {
                float *nbuf = cluster.map_shared_rank(D, rank + 1);
                const int nrow0 = band_start(rank + 1, nb, ny) - H;
                nbuf[(gy - nrow0) * nx + gx] = v;
            }
        }
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
    const float *B = smem + cur * bsz;
    for (int i = tid; i < nodes; i += CT) {
        const int gy = y0 + i / nx, gx = i - (i / nx) * nx;
        S.V[0][static_cast<long long>(gy) * S.pitch + gx] = B[(gy - row0) * nx + gx];
    }
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
    // two neighbours only
    int nb = ny / halo;
    if (nb > CL) nb = CL;
    if (nb < 1) return 0;
    const int bmax = (ny + nb - 1) / nb;
    const size_t bytes = 2ull * (bmax + 2 * halo) * nx * sizeof(float);
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
    a.interp = interp;
    a.stall_tol = stall_tol;
    a.ctrl = ctrl;
    const void *fn = wform ? reinterpret_cast<const void *>(&coarse_solve_kernel<true>)
                           : reinterpret_cast<const void *>(&coarse_solve_kernel<false>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return -2;
    void *argv[1] = {&a};
    if (cudaLaunchKernel(fn, dim3(m * CL), dim3(CT), argv, smem, st) != cudaSuccess) return -2;
    return 0;
}

}  // namespace hjbh
