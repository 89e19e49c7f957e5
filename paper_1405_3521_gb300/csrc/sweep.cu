// sweep.cu -- the value-iteration sweep: applications of the
// semi-Lagrangian operator T of Festa (arXiv:1405.3521), Sec. 3, eq. (Tdef),
//
//   [T(V)]_i = beta * min_a I[V](x_i + h f(x_i, a)) + gamma * l_i   (free node)
//
// to every free node of every active problem ("slot") of a launch, with the
// L-infinity change over the sweep (the residual of the stopping remark of
// Sec. 3) fused into the same kernel, and the convergence decision taken by
// the last CTA to finish (which also drives the CUDA-graph WHILE loop around
// the sweep).  A sweep applies T up to args.local_iters times to each staged
// tile: the first application reads the previous sweep's values (with one,
// the sweep is exactly one Jacobi application), each further one the
// tile's own latest values with the halo held -- the same fixed point, and
// still a beta-contraction per sweep.
//
// Design for sm_103a:
//  * persistent grid (SMs x resident CTAs) over a device work queue of
//    (slot, tile) items: a tile is queued for the next sweep only when a tile
//    of its 3x3 (3x3x3) neighbourhood changed bitwise in this sweep, since
//    otherwise its inputs, and hence its outputs, are those of the previous
//    sweep -- skipping it changes no iterate, while quiescent regions
//    (ahead of the front, and behind it once converged) cost nothing; tiles
//    of converged slots drop out of the queue;
//  * each tile of V plus its interpolation halo is staged in shared memory by
//    a TMA tensor load (cp.async.bulk.tensor) completing on an mbarrier, with
//    the next item's tile prefetched while the current one is computed;
//  * per node, the foot of every control is located with packed FP32x2 adds
//    against a 2^23 magic constant (cell index and fraction without
//    float-to-int conversions), the four corner values come from two 64-bit
//    shared loads of a (V[c], V[c+1]) pair layout addressed with shifts, and
//    the interpolation uses a monotone two-product lerp, so that in the
//    W = l/lambda - V form the FP32 iteration is itself monotone and ends at
//    an exact FP32 fixed point;
//  * feet are tested against the box only in tiles that touch the boundary.
#include <math.h>

#include "hjb_internal.cuh"

using namespace hjbk;

// Resident CTAs per SM the 2D sweep is compiled for (register budget).  At
// 4 (64 registers, no spills) the threads of a staged tile carry enough
// independent control evaluations to hide the shared-load and FMA latencies
// with 32 warps per SM; measured on the 1025^2 workloads against 8 (32
// registers): full solves 8 % and decomposed steps 3 % faster, the
// pursuit-evasion game 3 % slower.
#ifndef HJB_SWEEP2D_MINB
#define HJB_SWEEP2D_MINB 4
#endif
// Resident CTAs per SM the 3D sweep is compiled for (register budget), for
// tiles of 4 and of 2 heading layers.
#ifndef HJB_SWEEP3D_MINB
#define HJB_SWEEP3D_MINB 4
#endif
#ifndef HJB_SWEEP3D_MINB2
#define HJB_SWEEP3D_MINB2 6
#endif

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `phase` of an mbarrier, giving up after WAIT_NS.
__device__ bool mbar_wait_bounded(uint64_t *bar, unsigned phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > WAIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Node classes of Sec. 3 for one slot: ghost (outside a restricted
// sub-domain), target (the slot's part of dG) or free (G).
enum { CLS_FREE = 0, CLS_TARGET = 1, CLS_GHOST = 2 };
// inside: the node's tile lies wholly inside the slot's sub-domain (no mask
// read needed).
__device__ __forceinline__ int node_class(const SlotDesc &S, long long gi, bool inside = false) {
    if (!inside && S.mask != nullptr && !((S.mask[gi] >> S.mask_bit) & 1u)) return CLS_GHOST;
    const int lab = S.labels[gi];
    if (lab != 0 && (S.only_target == 0 || lab == S.only_target)) return CLS_TARGET;
    return CLS_FREE;
}

// Magic constant 2^23 - 1/2: for p in [1/2, 2^22), p + M rounds to
// 2^23 + rn(p - 1/2), so the float's low mantissa bits hold the cell index
// k in {floor(p) - 1, floor(p)} with p - k in [0, 1].
constexpr float MAGIC = 8388607.5f;
constexpr float TWO23 = 8388608.0f;
constexpr int TWO23_BITS = 0x4B000000;

// Bilinear interpolation of the pair layout at the tile-local foot
// P2 = (px, py) (py carries a +1 row shift so that it is >= 1/2).  The
// foot arithmetic runs on packed FP32x2 instructions; K is the shared
// address of the pair array minus the magic-constant bias, so that the byte
// address of pair (ky, kx) is (bits(my) << 9) + (bits(mx) << 3) + K.  The
// lerps use the two-product form (1-f) a + f b, which is monotone in a and b
// under FP32 rounding.  Its first product is taken as fma(-f, a, a), the
// exact a (1-f) rounded once, so no separate 1-f is computed; that is the
// rounded product of a and 1-f whenever 1-f is exact, as it is for the
// fraction of any coordinate >= 1/2 (a multiple of 2^-24 in [0, 1)).
__device__ __forceinline__ float q1_pairs(float2 P2, uint32_t K) {
    const float2 M2 = __fadd2_rn(P2, make_float2(MAGIC, MAGIC));
    const float2 Kn = __ffma2_rn(M2, make_float2(-1.0f, -1.0f), make_float2(TWO23, TWO23));
    const float2 F2 = __fadd2_rn(P2, Kn);  // (fx, fy) = p - k
    const uint32_t addr = (__float_as_uint(M2.y) << 9) + (__float_as_uint(M2.x) << 3) + K;
    float lo0, lo1, hi0, hi1;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(lo0), "=f"(lo1) : "r"(addr));
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+512];" : "=f"(hi0), "=f"(hi1) : "r"(addr));
    // lo = (v00, v10), hi = (v01, v11): the two lerps in y as one packed
    // pair (the same roundings as two scalar ones), then the lerp in x
    const float2 lo = make_float2(lo0, lo1);
    const float2 ab = __ffma2_rn(make_float2(F2.y, F2.y), make_float2(hi0, hi1),
                                 __ffma2_rn(make_float2(-F2.y, -F2.y), lo, lo));
    return fmaf(F2.x, ab.y, fmaf(-F2.x, ab.x, ab.x));
}

// P1 variant (the linear interpolant on the Kuhn triangles of each
// cell, split along the (0,0)-(1,1) diagonal): the same loads, the
// barycentric weights (1 - t1, t1 - t2, t2) with t1 = max(fx, fy), t2 =
// min(fx, fy) on the corners (0,0), (1,0) or (0,1), (1,1).  Non-negative
// weights in fused multiply-adds keep the value monotone in the data.
__device__ __forceinline__ float p1_pairs(float2 P2, uint32_t K) {
    const float2 M2 = __fadd2_rn(P2, make_float2(MAGIC, MAGIC));
    const float2 Kn = __ffma2_rn(M2, make_float2(-1.0f, -1.0f), make_float2(TWO23, TWO23));
    const float2 F2 = __fadd2_rn(P2, Kn);
    const uint32_t addr = (__float_as_uint(M2.y) << 9) + (__float_as_uint(M2.x) << 3) + K;
    float lo0, lo1, hi0, hi1;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(lo0), "=f"(lo1) : "r"(addr));
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+512];" : "=f"(hi0), "=f"(hi1) : "r"(addr));
    const bool lower = F2.x >= F2.y;  // the triangle (0,0), (1,0), (1,1)
    const float t1 = lower ? F2.x : F2.y, t2 = lower ? F2.y : F2.x;
    const float mid = lower ? lo1 : hi0;
    return fmaf(t2, hi1, fmaf(t1 - t2, mid, fmaf(-t1, lo0, lo0)));
}

// Interpolation of a kernel family: NA < 0 selects P1, otherwise Q1.
template <int NA>
__device__ __forceinline__ float interp_pairs(float2 P2, uint32_t K) {
    if constexpr (NA < 0)
        return p1_pairs(P2, K);
    else
        return q1_pairs(P2, K);
}

template <bool WFORM>
__device__ __forceinline__ float pick(float best, float q) {
    return WFORM ? fmaxf(best, q) : fminf(best, q);
}

// Controls [J0, J0 + NJ) at one node of a tile that does not touch the box
// boundary (no foot can leave the box).  S2 = (s hx, s hy), B2 = the node's
// tile-local position plus the current's displacement.  Compile-time control
// indices let the control components be constant-bank operands.
template <int J0, int NJ, bool WFORM>
__device__ __forceinline__ float range_interior(const ControlTable &C, uint32_t K, float2 S2,
                                                float2 B2, float best) {
#pragma unroll
    for (int j = 0; j < NJ; ++j)
        best = pick<WFORM>(best, q1_pairs(__ffma2_rn(S2, C.a2[J0 + j], B2), K));
    return best;
}

// Node bounds in cell offsets: a foot with offset o is outside the closed
// box when o < lo - 1e-6 or o > hi + 1e-6 (reading R2: 1e-6 grid cells of
// tolerance, in-tolerance feet clamped onto the face).
struct EdgeBounds {
    float lox, hix, loy, hiy;
};

template <bool WFORM, int NA = 0>
__device__ __forceinline__ float one_control_edge(uint32_t K, float2 O2, const EdgeBounds &eb,
                                                  float2 BASE2, float vout, float best) {
    const bool out = (O2.x < eb.lox - 1e-6f) | (O2.x > eb.hix + 1e-6f) | (O2.y < eb.loy - 1e-6f) |
                     (O2.y > eb.hiy + 1e-6f);
    O2.x = fminf(fmaxf(O2.x, eb.lox), eb.hix);
    O2.y = fminf(fmaxf(O2.y, eb.loy), eb.hiy);
    const float q = interp_pairs<NA>(__fadd2_rn(O2, BASE2), K);
    return pick<WFORM>(best, out ? vout : q);
}

template <int J0, int NJ, bool WFORM>
__device__ __forceinline__ float range_edge(const ControlTable &C, uint32_t K, float2 S2,
                                            float2 O02, const EdgeBounds &eb, float2 BASE2,
                                            float vout, float best) {
#pragma unroll
    for (int j = 0; j < NJ; ++j)
        best = one_control_edge<WFORM>(K, __ffma2_rn(S2, C.a2[J0 + j], O02), eb, BASE2, vout, best);
    return best;
}

// The controls of group g (of G groups splitting the control set): for a
// compile-time count NA the group's contiguous block, selected by a
// warp-uniform switch so that indices stay compile-time; otherwise every
// G-th control from g.
template <int NA, int G, bool WFORM>
__device__ __forceinline__ float controls_interior(int g, const ControlTable &C, uint32_t K,
                                                   float2 S2, float2 B2, float best) {
    if constexpr (NA > 0) {
        constexpr int NJ = NA / G;
        if (g == 0) return range_interior<0, NJ, WFORM>(C, K, S2, B2, best);
        if constexpr (G > 1)
            if (g == 1) return range_interior<NJ, NJ, WFORM>(C, K, S2, B2, best);
        if constexpr (G > 2) {
            if (g == 2) return range_interior<2 * NJ, NJ, WFORM>(C, K, S2, B2, best);
            return range_interior<3 * NJ, NJ, WFORM>(C, K, S2, B2, best);
        }
        return best;
    } else {
        const int na = C.count;
        if (C.nb > 1) {
            // game (one control group): the max over b of the min over a, in
            // the W form the min over b of the max over a
            const int nA = na / C.nb;
            float outer = WFORM ? INFINITY : -INFINITY;
            for (int k = 0; k < na; k += nA) {
                float inner = WFORM ? -INFINITY : INFINITY;
#pragma unroll 4
                for (int j = k; j < k + nA; ++j)
                    inner = pick<WFORM>(inner, interp_pairs<NA>(__ffma2_rn(S2, C.a2[j], B2), K));
                outer = WFORM ? fminf(outer, inner) : fmaxf(outer, inner);
            }
            return pick<WFORM>(best, outer);
        }
#pragma unroll 4
        for (int j = g; j < na; j += G)
            best = pick<WFORM>(best, interp_pairs<NA>(__ffma2_rn(S2, C.a2[j], B2), K));
        return best;
    }
}

template <int NA, int G, bool WFORM>
__device__ __forceinline__ float controls_edge(int g, const ControlTable &C, uint32_t K, float2 S2,
                                               float2 O02, const EdgeBounds &eb, float2 BASE2,
                                               float vout, float best) {
    if constexpr (NA > 0) {
        constexpr int NJ = NA / G;
        if (g == 0) return range_edge<0, NJ, WFORM>(C, K, S2, O02, eb, BASE2, vout, best);
        if constexpr (G > 1)
            if (g == 1) return range_edge<NJ, NJ, WFORM>(C, K, S2, O02, eb, BASE2, vout, best);
        if constexpr (G > 2) {
            if (g == 2) return range_edge<2 * NJ, NJ, WFORM>(C, K, S2, O02, eb, BASE2, vout, best);
            return range_edge<3 * NJ, NJ, WFORM>(C, K, S2, O02, eb, BASE2, vout, best);
        }
        return best;
    } else {
        const int na = C.count;
        if (C.nb > 1) {
            const int nA = na / C.nb;
            float outer = WFORM ? INFINITY : -INFINITY;
            for (int k = 0; k < na; k += nA) {
                float inner = WFORM ? -INFINITY : INFINITY;
#pragma unroll 4
                for (int j = k; j < k + nA; ++j)
                    inner = one_control_edge<WFORM, NA>(K, __ffma2_rn(S2, C.a2[j], O02), eb,
                                                        BASE2, vout, inner);
                outer = WFORM ? fminf(outer, inner) : fmaxf(outer, inner);
            }
            return pick<WFORM>(best, outer);
        }
#pragma unroll 4
        for (int j = g; j < na; j += G)
            best = one_control_edge<WFORM, NA>(K, __ffma2_rn(S2, C.a2[j], O02), eb, BASE2, vout,
                                               best);
        return best;
    }
}

// Block-wide exclusive scan of an int (256 threads); returns the total.
__device__ __forceinline__ int block_scan(int a, int &ea, int *sa) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ia = a;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int xa = __shfl_up_sync(0xffffffffu, ia, o);
        if (lane >= o) ia += xa;
    }
    if (lane == 31) sa[warp] = ia;
    __syncthreads();
    if (warp == 0) {
        int va = lane < THREADS / 32 ? sa[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int xa = __shfl_up_sync(0xffffffffu, va, o);
            if (lane >= o) va += xa;
        }
        if (lane < THREADS / 32) sa[lane] = va;
    }
    __syncthreads();
    ea = (warp ? sa[warp - 1] : 0) + ia - a;
    const int total = sa[THREADS / 32 - 1];
    __syncthreads();
    return total;
}

// Convergence step, run by the last CTA of a sweep: read and reset each
// active slot's residual, apply the stopping rule (residual <= tol, the
// iteration cap, or stagnation at rounding level), compact the active slot
// list, empty the tile queue this sweep consumed, and set the graph loop
// condition.
__device__ void finish_sweep(const SweepArgs &args) {
    Ctl *ctl = args.ctl;
    __shared__ int s_sa[THREADS / 32];
    // L2 reads: in the cooperative loop these were written by other CTAs
    const int n = __ldcg(&ctl->nactive);
    const int p = static_cast<int>(__ldcg(&ctl->sweep) & 1u);
    const int dst_parity = p ^ 1;
    const int err = __ldcg(&ctl->error);
    constexpr int PER = MAX_SLOTS / THREADS;
    int sid[PER], keep[PER];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = threadIdx.x * PER + k;
        keep[k] = 0;
        sid[k] = -1;
        if (i >= n) continue;
        const int s = __ldcg(&ctl->act_slot[i]);
        sid[k] = s;
        SlotState &st = args.state[s];
        const SlotDesc &S = args.slots[s];
        const float r = __uint_as_float(__ldcg(&st.res_bits));
        const int iters = __ldcg(&st.iters) + 1;
        st.res_bits = 0u;
        st.iters = iters;
        st.final_res = r;
        st.final_parity = dst_parity;
        int kp = 1;
        if (r <= S.tol) {
            st.converged = 1;
            kp = 0;
        } else if (iters >= S.max_iters || err) {
            kp = 0;
        } else {
            if (r < __ldcg(&st.best_res)) {
                st.best_res = r;
                st.stall = 0;
            } else {
                const int stall = __ldcg(&st.stall) + 1;
                st.stall = stall;
                if (stall >= 64 && r <= args.stall_tol) {
                    st.converged = 2;
                    kp = 0;
                }
            }
        }
        if (!kp) st.done = 1;
        keep[k] = kp;
        cnt += kp;
    }
    // every thread has read its entries of the active list before the scan's
    // barriers, so the list can be compacted in place afterwards
    int ec;
    const int tc = block_scan(cnt, ec, s_sa);
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (keep[k]) ctl->act_slot[ec++] = sid[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->nactive = tc;
        ctl->qcount[p] = 0;  // every entry of this sweep's queue was consumed
        ctl->qhead[p] = 0;
        if (n > 0) ctl->sweep = __ldcg(&ctl->sweep) + 1u;
        ctl->launches = __ldcg(&ctl->launches) + 1u;
        ctl->done_ctas = 0u;
        __threadfence();
        if (args.use_handle) cudaGraphSetConditional(args.handle, (tc > 0 && !err) ? 1u : 0u);
    }
}

// Count this CTA as finished; the last one runs finish_sweep.  Only the
// `working` CTAs (those that had an item, or CTA 0 when the queue is empty)
// take part, so a short queue costs few arrivals.
__device__ __forceinline__ void cta_done(const SweepArgs &args, bool failed, int working) {
    __shared__ int s_last;
    if (static_cast<int>(blockIdx.x) >= working) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (failed) atomicExch(&args.ctl->error, 1);
        __threadfence();
        const unsigned t = atomicAdd(&args.ctl->done_ctas, 1u);
        s_last = (t == static_cast<unsigned>(working) - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        finish_sweep(args);
    }
}

// Queue entry of a CTA's next item, taken by thread 0 and published in
// `next` (the other threads read it after the loop body's barriers; the
// value they get back here is unused).  Static: entry v + grid.  Dynamic:
// entries past the first grid-size ones are handed out in order by one
// counter, so a CTA whose items were cheap takes more of them.
__device__ __forceinline__ int next_entry(const SweepArgs &args, int &next, int v, int p,
                                          int nitems) {
    int vn = nitems;
    if (threadIdx.x == 0) {
        vn = args.dyn_queue ? static_cast<int>(gridDim.x) + atomicAdd(&args.ctl->qhead[p], 1)
                            : v + static_cast<int>(gridDim.x);
        next = vn;
    }
    return vn;
}

// Tile queue of the next sweep: called by warp 0 of a CTA whose tile changed
// (bitwise) in this sweep; lane t considers neighbour t of the tile
// neighbourhood (radius RX, RY, RZ in tiles: the halo of a tile reaches that
// far), skips tiles outside the grid or holding no node of the slot, claims
// the neighbour's flag, and the claimed neighbours are appended with one
// atomic per warp.  A tile none of whose neighbours changed would reproduce
// its previous values exactly, so it is not queued.
template <int RX, int RY, int RZ>
__device__ __forceinline__ void enqueue_neighbours(const SweepArgs &args, const SlotDesc &S,
                                                   int slot, int tx, int ty, int tz, int p) {
    constexpr int WX = 2 * RX + 1, WY = 2 * RY + 1, WZ = 2 * RZ + 1;
    static_assert(WX * WY * WZ <= 32, "neighbourhood larger than a warp");
    const int lane = threadIdx.x & 31;
    int nb = -1;
    if (lane < WX * WY * WZ) {
        const int dx = lane % WX - RX, dy = (lane / WX) % WY - RY, dz = lane / (WX * WY) - RZ;
        const int x = tx + dx, y = ty + dy;
        int z = tz + dz;
        if (RZ > 0) z = ((z % S.tiles_z) + S.tiles_z) % S.tiles_z;  // periodic heading
        if (x >= 0 && x < S.tiles_x && y >= 0 && y < S.tiles_y) {
            const int t = (z * S.tiles_y + y) * S.tiles_x + x;
            const bool member = S.tile_bits == nullptr || ((S.tile_bits[t] >> S.mask_bit) & 1u);
            if (member) {
                // byte flags: claim with an atomic OR on the containing word
                uint8_t *f = args.qflag[p ^ 1] + S.qbase + t;
                unsigned *w = reinterpret_cast<unsigned *>(reinterpret_cast<size_t>(f) & ~size_t(3));
                const unsigned bit = 1u << ((reinterpret_cast<size_t>(f) & 3u) * 8u);
                if ((atomicOr(w, bit) & bit) == 0u) nb = t;
            }
        }
    }
    const unsigned need = __ballot_sync(0xffffffffu, nb >= 0);
    if (need) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&args.ctl->qcount[p ^ 1], __popc(need));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (nb >= 0) args.qlist[p ^ 1][base + __popc(need & ((1u << lane) - 1u))] = (slot << 22) | nb;
    }
}

// Clear this sweep's queued flag of a tile (byte flag inside a word).
__device__ __forceinline__ void unflag(const SweepArgs &args, const SlotDesc &S, int tile, int p) {
    uint8_t *f = args.qflag[p] + S.qbase + tile;
    unsigned *w = reinterpret_cast<unsigned *>(reinterpret_cast<size_t>(f) & ~size_t(3));
    const unsigned sh = static_cast<unsigned>(reinterpret_cast<size_t>(f) & 3u) * 8u;
    atomicAnd(w, ~(0xffu << sh));
}

// Grid-wide barrier of the cooperative loop, fused with the convergence
// step: the last CTA to arrive runs finish_sweep and then releases the
// others by bumping the generation.  Waiters give up after WAIT_NS and
// raise the error flag, so a lost CTA cannot hang the loop.  Returns false
// when the loop must stop (all slots done, or an error).
__device__ bool grid_barrier_finish(const SweepArgs &args, bool failed) {
    __shared__ int s_last;
    __shared__ int s_go;
    Ctl *ctl = args.ctl;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (failed) atomicExch(&ctl->error, 1);
        const unsigned gen = *reinterpret_cast<volatile unsigned *>(&ctl->gen);
        __threadfence();
        const unsigned t = atomicAdd(&ctl->done_ctas, 1u);
        s_last = (t == gridDim.x - 1) ? 1 : 0;
        if (!s_last) {
            const unsigned long long t0 = global_ns();
            unsigned ns = 32;
            while (*reinterpret_cast<volatile unsigned *>(&ctl->gen) == gen) {
                if (*reinterpret_cast<volatile int *>(&ctl->error)) break;
                if (global_ns() - t0 > WAIT_NS) {
                    atomicExch(&ctl->error, 1);
                    break;
                }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
            }
            __threadfence();
        }
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        finish_sweep(args);  // resets done_ctas
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&ctl->gen, 1u);
        }
    }
    if (threadIdx.x == 0) {
        const int nact = *reinterpret_cast<volatile int *>(&ctl->nactive);
        const int err = *reinterpret_cast<volatile int *>(&ctl->error);
        s_go = (nact > 0 && !err) ? 1 : 0;
    }
    __syncthreads();
    return s_go != 0;
}

// --------------------------------------------------------------------------
// 2D sweep: f = s(x) a + c(x).  Tile 32 x TYT nodes, halo H (cells) in x
// and y; the 256 threads split the controls of a node in one of two ways:
//  * LANES = 1: G warp groups -- warp w handles row w / G of the tile for the
//    controls of group w % G, and the groups' partial extrema are combined
//    through shared memory;
//  * LANES = 2 (TYT = 4, G = 1; control sets with a_{j + A/2} = -a_j): the
//    lanes n and n + 16 of a warp handle node n of a 16-node half row, the
//    low half-warp with the controls a_j and the high one with -a_j
//    (j < A/2), through the same instruction stream with the node's speed
//    factors negated, and one shuffle combines them.  Each half-warp reads
//    16 neighbouring pairs per control, so its 64-bit shared loads stay free
//    of bank conflicts.
// The tile's values are read through a pair layout that is double-buffered
// across the applications of T to the staged tile: application li reads
// buffer li & 1 and writes its new values into the other, so one barrier
// per application (which also takes the early-exit vote) suffices.

template <int H, int TYT, int G>
struct Smem2d {
    static constexpr int ROWS = TYT + 2 * H;
    static constexpr int TILE = ROWS * TW;
    // each staging buffer starts on a 128-byte boundary (TMA destination rule)
    static constexpr int TILE_STRIDE = (TILE + 31) / 32 * 32;
    float tile[2][TILE_STRIDE];
    float2 pair[2][ROWS * PW];
    uint64_t bar[2];
    int item[2][3];
    int next;  // queue entry of the CTA's next item
    float red[THREADS / 32];
    int cnt[THREADS / 32];
    float part[G > 1 ? G : 1][G > 1 ? TYT : 1][32];
};

// One sweep over this launch's tile queue by one CTA.  `uses` counts the
// TMA phases consumed per staging buffer and persists across sweeps.
template <int NA, bool WFORM, int H, int TYT, int G, int LANES>
__device__ __forceinline__ bool pass2d(const SweepArgs &args, Smem2d<H, TYT, G> &sm,
                                       unsigned uses[2]) {
    using SM = Smem2d<H, TYT, G>;
    constexpr int ROWS = SM::ROWS;
    constexpr int TILE = SM::TILE;
    constexpr int RY = (H + TYT - 1) / TYT;  // tile neighbourhood reached by the halo
    constexpr uint32_t PAIR_BYTES = ROWS * PW * 8;
    static_assert(LANES == 1 || (LANES == 2 && G == 1 && TYT == 4 && NA > 0),
                  "the lane split pairs a_j with -a_j in 32 x 4 tiles");
    const Ctl *ctl = args.ctl;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int grp = LANES == 2 ? (lane >> 4) : warp % G;
    const int ly = LANES == 2 ? (warp >> 1) : warp / G;
    const int lx = LANES == 2 ? ((warp & 1) << 4) + (lane & 15) : lane;
    const int p = static_cast<int>(*reinterpret_cast<const volatile unsigned *>(&ctl->sweep) & 1u);
    const int src = p, dst = p ^ 1;
    const int nitems = *reinterpret_cast<const volatile int *>(&ctl->qcount[p]);
    const int *qlist = args.qlist[p];
    // pair (ky, kx) of buffer c sits at byte c * PAIR_BYTES + (ky - 1) * 512 +
    // kx * 8 of sm.pair, with kx = bits(mx) - 2^23 bits and ky = bits(my) -
    // 2^23 bits (see q1_pairs)
    const uint32_t K0 = smem_u32(sm.pair[0]) - (static_cast<uint32_t>(TWO23_BITS) << 9) -
                        (static_cast<uint32_t>(TWO23_BITS) << 3) - 512u;

    // thread 0: stage item v into buffer b (no copy for a finished slot)
    auto issue = [&](int v, int b) {
        const int e = __ldcg(qlist + v);  // written by other CTAs in the previous sweep
        const int slot = e >> 22, tile = e & 0x3FFFFF;
        const SlotDesc *S = args.slots + slot;
        const int live = __ldcg(&args.state[slot].done) ? 0 : 1;
        sm.item[b][0] = slot;
        sm.item[b][1] = tile;
        sm.item[b][2] = live;
        if (live) {
            const int tx = tile % S->tiles_x, ty = tile / S->tiles_x;
            mbar_expect_tx(&sm.bar[b], TILE * 4);
            tma_load_2d(sm.tile[b], &S->tmap[src], tx * TX - XPAD, ty * TYT - H, &sm.bar[b]);
        }
    };

    int v = blockIdx.x;
    // buffer of the first item: continue the alternation of earlier sweeps
    int b0 = static_cast<int>((uses[0] + uses[1]) & 1u);
    if (tid == 0 && v < nitems) issue(v, b0);
    __syncthreads();
    bool failed = false;
    for (int it = 0; v < nitems; ++it, v = sm.next) {
        const int b = (b0 + it) & 1;
        const int slot = sm.item[b][0], tile = sm.item[b][1], live = sm.item[b][2];
        __syncthreads();  // everyone has read sm.item[b] and sm.next; buffer b ^ 1 is free
        if (tid == 0) {
            const int vn = next_entry(args, sm.next, v, p, nitems);
            if (vn < nitems) issue(vn, b ^ 1);
        }
        const SlotDesc &S = args.slots[slot];
        if (!live) {
            if (tid == 0) unflag(args, S, tile, p);
            __syncthreads();  // sm.item[b ^ 1] and sm.next written above
            continue;
        }
        const bool ok = mbar_wait_bounded(&sm.bar[b], uses[b] & 1u);
        uses[b] += 1u;
        if (!__syncthreads_and(ok)) {
            failed = true;
            // let the prefetch of the next item (if any) land before leaving
            if (tid == 0 && sm.next < nitems && sm.item[b ^ 1][2])
                mbar_wait_bounded(&sm.bar[b ^ 1], uses[b ^ 1] & 1u);
            break;
        }
        // both pair buffers: (raw[r][c], raw[r][c+1]) for the TW-1 columns a
        // foot can use (the halo is the same in both and never rewritten)
        const float *T = sm.tile[b];
        for (int i = tid; i < ROWS * (TW - 1); i += THREADS) {
            const int r = i / (TW - 1), c = i - r * (TW - 1);
            const float2 q = make_float2(T[r * TW + c], T[r * TW + c + 1]);
            sm.pair[0][r * PW + c] = q;
            sm.pair[1][r * PW + c] = q;
        }
        const int nx = S.nx, ny = S.ny;
        const int tx = tile % S.tiles_x, ty = tile / S.tiles_x;
        const int gx = tx * TX + lx, gy = ty * TYT + ly;
        const float vold = T[(ly + H) * TW + lx + XPAD];
        const long long gi = static_cast<long long>(gy) * nx + gx;
        const bool inb = (gx < nx) && (gy < ny);
        // the node's fields are read before its class is known, so that their
        // loads and the label (and mask) loads are in flight together
        float sx = 1.0f, sy = 1.0f, cx = 0.0f, cy = 0.0f, lc = 0.0f;
        if (inb) {
            if (S.scale2) {
                const float2 d = S.scale2[gi];
                sx = d.x;
                sy = d.y;
            } else if (S.speed) {
                sx = sy = S.speed[gi];
            }
            if (S.current) {
                const float2 c = reinterpret_cast<const float2 *>(S.current)[gi];
                cx = c.x;
                cy = c.y;
            }
            if (!WFORM && S.cost) lc = S.cost[gi];
        }
        const bool inside = S.tile_full != nullptr && ((S.tile_full[tile] >> S.mask_bit) & 1u);
        // a tile without target nodes, in no sub-domain or wholly inside one,
        // holds free nodes only: no label or mask reads
        const bool clear = S.tile_clear != nullptr && S.tile_clear[tile] &&
                           (S.mask == nullptr || inside);
        const bool isfree = inb && (clear || node_class(S, gi, inside) == CLS_FREE);
        const bool mine = isfree && grp == 0;  // group 0 owns the node's result
        float2 S2 = make_float2(0.0f, 0.0f), O02 = S2;
        float add = S.gl;
        if (isfree) {
            const float sg = (LANES == 2 && grp) ? -1.0f : 1.0f;  // the high half takes -a_j
            S2 = make_float2(sg * sx * S.hx, sg * sy * S.hy);
            O02 = make_float2(cx * S.hx, cy * S.hy);
            if (!WFORM && S.cost) add = S.gamma * lc;
        }
        const float2 BASE2 = make_float2(static_cast<float>(lx + XPAD),
                                         static_cast<float>(ly + H + 1));
        const bool interior = (tx * TX >= H) && (tx * TX + TX - 1 + H <= nx - 1) &&
                              (ty * TYT >= H) && (ty * TYT + TYT - 1 + H <= ny - 1);
        // this node's two entries in the pair layout: (v, right) and (left, v)
        const int pr = (ly + H) * PW + lx + XPAD;
        __syncthreads();
        // args.local_iters applications of T to the tile's nodes, the halo
        // held at the previous sweep's values: each application reads the
        // tile's latest values (a block Gauss-Seidel step; same fixed point)
        float vnew = vold;
        int li = 0;  // applications done
        for (;;) {
            const uint32_t K = K0 + static_cast<uint32_t>(li & 1) * PAIR_BYTES;
            float best = WFORM ? -INFINITY : INFINITY;
            if (isfree) {
                if (interior) {
                    best = controls_interior<NA, LANES == 2 ? 2 : G, WFORM>(
                        LANES == 2 ? 0 : grp, args.ctrl, K, S2, __fadd2_rn(BASE2, O02), best);
                } else {
                    EdgeBounds eb;
                    eb.lox = -static_cast<float>(gx);
                    eb.hix = static_cast<float>(nx - 1 - gx);
                    eb.loy = -static_cast<float>(gy);
                    eb.hiy = static_cast<float>(ny - 1 - gy);
                    best = controls_edge<NA, LANES == 2 ? 2 : G, WFORM>(
                        LANES == 2 ? 0 : grp, args.ctrl, K, S2, O02, eb, BASE2, S.vout, best);
                }
            }
            if constexpr (LANES == 2) {
                best = pick<WFORM>(best, __shfl_xor_sync(0xffffffffu, best, 16));
            } else if constexpr (G > 1) {
                sm.part[grp][ly][lx] = best;
                __syncthreads();
                if (grp == 0) {
#pragma unroll
                    for (int q = 1; q < G; ++q) best = pick<WFORM>(best, sm.part[q][ly][lx]);
                }
            }
            const float vprev = vnew;
            if (mine) vnew = WFORM ? S.beta * best : fmaf(S.beta, best, add);
            if (++li >= args.local_iters) break;
            if (mine) {
                float2 *P = sm.pair[li & 1];
                P[pr].x = vnew;
                P[pr - 1].y = vnew;
            }
            // the new values are visible; stop early once the tile is stable
            if (!__syncthreads_or(mine && vnew != vprev)) break;
        }
        if (mine) S.V[dst][static_cast<long long>(gy) * S.pitch + gx] = vnew;
        const float r = warp_max(mine ? fabsf(vnew - vold) : 0.0f);
        const unsigned fm = __ballot_sync(0xffffffffu, mine);
        const unsigned cm = __ballot_sync(0xffffffffu, mine && (vnew != vold));
        if (lane == 0) {
            sm.red[warp] = r;
            sm.cnt[warp] = __popc(fm) | (cm ? 0x10000 : 0);
        }
        __syncthreads();
        if (tid < 32) {
            float m = 0.0f;
            int tot = 0, chg = 0;
#pragma unroll
            for (int w = 0; w < THREADS / 32; ++w) {
                m = fmaxf(m, sm.red[w]);
                tot += sm.cnt[w] & 0xffff;
                chg |= sm.cnt[w] >> 16;
            }
            if (tid == 0) {
                if (m > 0.0f) atomicMax(&args.state[slot].res_bits, __float_as_uint(m));
                atomicAdd(&args.state[slot].updates, static_cast<unsigned long long>(tot) * li);
                atomicAdd(&args.state[slot].visits, 1u);
                unflag(args, S, tile, p);
            }
            if (chg) enqueue_neighbours<1, RY, 0>(args, S, slot, tx, ty, 0, p);
        }
    }
    return failed;
}

template <int H, int TYT, int G>
__device__ __forceinline__ void init_bars(Smem2d<H, TYT, G> &sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// One sweep per launch (the body of the CUDA-graph WHILE loop).
template <int NA, bool WFORM, int H, int TYT, int G, int LANES>
__global__ void __launch_bounds__(THREADS, HJB_SWEEP2D_MINB) sweep2d_kernel(const __grid_constant__ SweepArgs args) {
    static_assert(TYT * G * LANES * 32 == THREADS, "tile rows x control groups must fill the CTA");
    __shared__ alignas(128) Smem2d<H, TYT, G> sm;
    const int p = static_cast<int>(args.ctl->sweep & 1u);
    const int nitems = args.ctl->qcount[p];
    const int working = nitems < 1 ? 1 : (nitems < static_cast<int>(gridDim.x) ? nitems : gridDim.x);
    if (static_cast<int>(blockIdx.x) >= working) return;
    init_bars(sm);
    unsigned uses[2] = {0u, 0u};
    const bool failed = pass2d<NA, WFORM, H, TYT, G, LANES>(args, sm, uses);
    cta_done(args, failed, working);
}

// The whole convergence loop in one cooperative launch: sweeps separated by
// a grid barrier that also takes the convergence decision.
template <int NA, bool WFORM, int H, int TYT, int G, int LANES>
__global__ void __launch_bounds__(THREADS, HJB_SWEEP2D_MINB) loop2d_kernel(const __grid_constant__ SweepArgs args) {
    static_assert(TYT * G * LANES * 32 == THREADS, "tile rows x control groups must fill the CTA");
    __shared__ alignas(128) Smem2d<H, TYT, G> sm;
    init_bars(sm);
    unsigned uses[2] = {0u, 0u};
    for (;;) {
        const bool failed = pass2d<NA, WFORM, H, TYT, G, LANES>(args, sm, uses);
        if (!grid_barrier_finish(args, failed)) break;
    }
}

// --------------------------------------------------------------------------
// 3D Dubins sweep: f = (v cos th, v sin th, u), th = dimension 2 (periodic).
// Tile 32 x 8 x TZ, halo 2 in x, y and 1 in th.  The (x, y) part of the foot
// does not depend on the control, so the bilinear values at the three
// heading layers a foot can reach are computed once per node and each
// control only interpolates in th.

template <int TZ3>
struct Smem3d {
    static constexpr int H = 2, HZ = 1;
    static constexpr int ROWS = TY + 2 * H;
    static constexpr int LAYER = ROWS * TW;
    static constexpr int TILE = (TZ3 + 2 * HZ) * LAYER;
    static constexpr int TILE_STRIDE = (TILE + 31) / 32 * 32;  // 128-byte aligned buffers
    float tile[2][TILE_STRIDE];
    uint64_t bar[2];
    int item[2][3];
    int next;  // queue entry of the CTA's next item
    float red[THREADS / 32];
    int cnt[THREADS / 32];
    float2 trig[TZ3];  // heading offsets of the item's layers
};

template <bool WFORM, int TZ3>
__device__ __forceinline__ bool pass3d(const SweepArgs &args, Smem3d<TZ3> &sm, unsigned uses[2]) {
    using SM = Smem3d<TZ3>;
    constexpr int H = SM::H, HZ = SM::HZ;
    constexpr int LAYER = SM::LAYER;
    constexpr int TILE = SM::TILE;
    const Ctl *ctl = args.ctl;
    const int tid = threadIdx.x;
    const int lx = tid & 31, ly = tid >> 5;
    const int p = static_cast<int>(*reinterpret_cast<const volatile unsigned *>(&ctl->sweep) & 1u);
    const int src = p, dst = p ^ 1;
    const int nitems = *reinterpret_cast<const volatile int *>(&ctl->qcount[p]);
    const int *qlist = args.qlist[p];

    auto issue = [&](int v, int b) {
        const int e = __ldcg(qlist + v);  // written by other CTAs in the previous sweep
        const int slot = e >> 22, tile = e & 0x3FFFFF;
        const SlotDesc *S = args.slots + slot;
        const int live = __ldcg(&args.state[slot].done) ? 0 : 1;
        sm.item[b][0] = slot;
        sm.item[b][1] = tile;
        sm.item[b][2] = live;
        if (live) {
            const int txy = S->tiles_x * S->tiles_y;
            const int tz = tile / txy, rem = tile - tz * txy;
            const int ty = rem / S->tiles_x, tx = rem - ty * S->tiles_x;
            mbar_expect_tx(&sm.bar[b], TILE * 4);
            tma_load_3d(sm.tile[b], &S->tmap[src], tx * TX - XPAD, ty * TY - H,
                        tz * TZ3 - HZ + S->zdup, &sm.bar[b]);
        }
    };

    int v = blockIdx.x;
    int b0 = static_cast<int>((uses[0] + uses[1]) & 1u);
    if (tid == 0 && v < nitems) issue(v, b0);
    __syncthreads();
    bool failed = false;
    for (int it = 0; v < nitems; ++it, v = sm.next) {
        const int b = (b0 + it) & 1;
        const int slot = sm.item[b][0], tile = sm.item[b][1], live = sm.item[b][2];
        __syncthreads();  // everyone has read sm.item[b] and sm.next; buffer b ^ 1 is free
        if (tid == 0) {
            const int vn = next_entry(args, sm.next, v, p, nitems);
            if (vn < nitems) issue(vn, b ^ 1);
        }
        const SlotDesc &S = args.slots[slot];
        if (!live) {
            if (tid == 0) unflag(args, S, tile, p);
            __syncthreads();  // sm.item[b ^ 1] and sm.next written above
            continue;
        }
        // the item's heading offsets, read once into shared memory (visible
        // after the barrier below)
        if (tid < TZ3) {
            const int gz = (tile / (S.tiles_x * S.tiles_y)) * TZ3 + tid;
            sm.trig[tid] = gz < S.nz ? S.trig[gz] : make_float2(0.0f, 0.0f);
        }
        const bool ok = mbar_wait_bounded(&sm.bar[b], uses[b] & 1u);
        uses[b] += 1u;
        if (!__syncthreads_and(ok)) {
            failed = true;
            if (tid == 0 && sm.next < nitems && sm.item[b ^ 1][2])
                mbar_wait_bounded(&sm.bar[b ^ 1], uses[b ^ 1] & 1u);
            break;
        }
        const int nx = S.nx, ny = S.ny, nz = S.nz;
        const int txy = S.tiles_x * S.tiles_y;
        const int tz = tile / txy, rem = tile - tz * txy;
        const int ty = rem / S.tiles_x, tx = rem - ty * S.tiles_x;
        const int gx = tx * TX + lx, gy = ty * TY + ly;
        float *T = sm.tile[b];
        const bool interior = (tx * TX >= H) && (tx * TX + TX - 1 + H <= nx - 1) &&
                              (ty * TY >= H) && (ty * TY + TY - 1 + H <= ny - 1);
        // the thread's column of TZ3 nodes: starting values and free flags
        float vold[TZ3], vnew[TZ3];
        unsigned freebits = 0u;
        const bool inside = S.tile_full != nullptr && ((S.tile_full[tile] >> S.mask_bit) & 1u);
        // a tile without target nodes, in no sub-domain or wholly inside one,
        // holds free nodes only: no label or mask reads
        const bool clear = S.tile_clear != nullptr && S.tile_clear[tile] &&
                           (S.mask == nullptr || inside);
#pragma unroll
        for (int lz = 0; lz < TZ3; ++lz) {
            const int gz = tz * TZ3 + lz;
            vold[lz] = T[(lz + HZ) * LAYER + (ly + H) * TW + lx + XPAD];
            vnew[lz] = vold[lz];
            const long long gi = (static_cast<long long>(gz) * ny + gy) * nx + gx;
            if ((gx < nx) && (gy < ny) && (gz < nz) &&
                (clear || node_class(S, gi, inside) == CLS_FREE))
                freebits |= 1u << lz;
        }
        // args.local_iters applications of T to the tile's nodes with the
        // halo held (the first reads the previous sweep's values)
        int li = 0;
        for (;;) {
            bool moved = false;
#pragma unroll
            for (int lz = 0; lz < TZ3; ++lz) {
                if (!((freebits >> lz) & 1u)) continue;
                const int gz = tz * TZ3 + lz;
                const long long gi = (static_cast<long long>(gz) * ny + gy) * nx + gx;
                    const float2 tr = sm.trig[lz];
                float ox = tr.x, oy = tr.y;
                bool out = false;
            if (!interior) {
                const float lox = -static_cast<float>(gx), hix = static_cast<float>(nx - 1 - gx);
                const float loy = -static_cast<float>(gy), hiy = static_cast<float>(ny - 1 - gy);
                out = (ox < lox - 1e-6f) | (ox > hix + 1e-6f) | (oy < loy - 1e-6f) |
                      (oy > hiy + 1e-6f);
                ox = fminf(fmaxf(ox, lox), hix);
                oy = fminf(fmaxf(oy, loy), hiy);
            }
            float best;
            if (out) {
                best = S.vout;
            } else {
                // bilinear (x, y) values at layers lz-1, lz, lz+1 of the tile
                const float px = static_cast<float>(lx + XPAD) + ox;
                const float py = static_cast<float>(ly + H + 1) + oy;
                const float mx = px + MAGIC, my = py + MAGIC;
                const float fx = px - (mx - TWO23), fy = py - (my - TWO23);
                const int idx = (__float_as_int(my) - (TWO23_BITS + 1)) * TW +
                                (__float_as_int(mx) - TWO23_BITS);
                float B[3];
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const float *P = T + (lz + HZ - 1 + t) * LAYER + idx;
                    const float a = fmaf(fx, P[1], fmaf(-fx, P[0], P[0]));
                    const float c = fmaf(fx, P[TW + 1], fmaf(-fx, P[TW], P[TW]));
                    B[t] = fmaf(fy, c, fmaf(-fy, a, a));
                }
                // heading: local coordinate of the node is lz + HZ + 1 (+1 shift)
                const float bz = static_cast<float>(lz + HZ + 1);
                const int kz0 = lz + HZ + 1;
                best = WFORM ? -INFINITY : INFINITY;
                const int na = args.ctrl.count;
                // heading interpolation of control j between the bilinear values
                auto heading = [&](int j) {
                    const float pz = fmaf(S.hz, args.ctrl.ax[j], bz);
                    const float mz = pz + MAGIC;
                    const float fz = pz - (mz - TWO23);
                    const int d = (__float_as_int(mz) - TWO23_BITS) - kz0;  // -1 or 0
                    const float lo = d < 0 ? B[0] : B[1];
                    const float hi = d < 0 ? B[1] : B[2];
                    return fmaf(fz, hi, fmaf(-fz, lo, lo));
                };
                if (na == 3) {
                    // the three turn rates of the car: straight-line code
                    best = pick<WFORM>(pick<WFORM>(heading(0), heading(1)), heading(2));
                } else {
#pragma unroll 4
                    for (int j = 0; j < na; ++j) best = pick<WFORM>(best, heading(j));
                }
            }
            const float v = WFORM ? S.beta * best
                                  : fmaf(S.beta, best, S.cost ? S.gamma * S.cost[gi] : S.gl);
            moved |= (v != vnew[lz]);
            vnew[lz] = v;
            }
            if (++li >= args.local_iters) break;
            // all reads of the tile done; stop early once the tile is stable
            if (!__syncthreads_or(moved)) break;
#pragma unroll
            for (int lz = 0; lz < TZ3; ++lz)
                if ((freebits >> lz) & 1u) T[(lz + HZ) * LAYER + (ly + H) * TW + lx + XPAD] = vnew[lz];
            if (freebits) fence_proxy_async_smem();  // the buffer takes a later TMA copy
            __syncthreads();
        }
        float rmax = 0.0f;
        bool chg = false;
        float *D = S.V[dst];
        const long long row = static_cast<long long>(gy) * S.pitch + gx;
#pragma unroll
        for (int lz = 0; lz < TZ3; ++lz) {
            if (!((freebits >> lz) & 1u)) continue;
            const int gz = tz * TZ3 + lz;
            D[static_cast<long long>(gz + S.zdup) * S.zstride + row] = vnew[lz];
            if (gz < S.zdup) D[static_cast<long long>(gz + nz + S.zdup) * S.zstride + row] = vnew[lz];
            if (gz >= nz - S.zdup)
                D[static_cast<long long>(gz - nz + S.zdup) * S.zstride + row] = vnew[lz];
            rmax = fmaxf(rmax, fabsf(vnew[lz] - vold[lz]));
            chg |= (vnew[lz] != vold[lz]);
        }
        const float r = warp_max(rmax);
        int c = __popc(freebits) * li;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        const unsigned cm = __ballot_sync(0xffffffffu, chg);
        if (lx == 0) {
            sm.red[ly] = r;
            sm.cnt[ly] = c | (cm ? 0x10000 : 0);
        }
        __syncthreads();
        if (tid < 32) {
            float m = 0.0f;
            int tot = 0, any = 0;
#pragma unroll
            for (int w = 0; w < THREADS / 32; ++w) {
                m = fmaxf(m, sm.red[w]);
                tot += sm.cnt[w] & 0xffff;
                any |= sm.cnt[w] >> 16;
            }
            if (tid == 0) {
                if (m > 0.0f) atomicMax(&args.state[slot].res_bits, __float_as_uint(m));
                atomicAdd(&args.state[slot].updates, static_cast<unsigned long long>(tot));
                atomicAdd(&args.state[slot].visits, 1u);
                unflag(args, S, tile, p);
            }
            if (any) enqueue_neighbours<1, 1, 1>(args, S, slot, tx, ty, tz, p);
        }
    }
    return failed;
}

template <int TZ3>
__device__ __forceinline__ void init_bars3(Smem3d<TZ3> &sm) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

template <bool WFORM, int TZ3>
__global__ void __launch_bounds__(THREADS, TZ3 == 2 ? HJB_SWEEP3D_MINB2 : HJB_SWEEP3D_MINB)
    sweep3d_kernel(const __grid_constant__ SweepArgs args) {
    __shared__ alignas(128) Smem3d<TZ3> sm;
    const int p = static_cast<int>(args.ctl->sweep & 1u);
    const int nitems = args.ctl->qcount[p];
    const int working = nitems < 1 ? 1 : (nitems < static_cast<int>(gridDim.x) ? nitems : gridDim.x);
    if (static_cast<int>(blockIdx.x) >= working) return;
    init_bars3(sm);
    unsigned uses[2] = {0u, 0u};
    const bool failed = pass3d<WFORM, TZ3>(args, sm, uses);
    cta_done(args, failed, working);
}

template <bool WFORM, int TZ3>
__global__ void __launch_bounds__(THREADS, TZ3 == 2 ? HJB_SWEEP3D_MINB2 : HJB_SWEEP3D_MINB)
    loop3d_kernel(const __grid_constant__ SweepArgs args) {
    __shared__ alignas(128) Smem3d<TZ3> sm;
    init_bars3(sm);
    unsigned uses[2] = {0u, 0u};
    for (;;) {
        const bool failed = pass3d<WFORM, TZ3>(args, sm, uses);
        if (!grid_barrier_finish(args, failed)) break;
    }
}

// --------------------------------------------------------------------------
// Helpers around the loop.

__global__ void loop_init_kernel(SlotState *state, Ctl *ctl, int nslots, const uint32_t *diff) {
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        SlotState &st = state[i];
        st.res_bits = 0u;
        st.iters = 0;
        st.done = 0;
        st.converged = 0;
        st.final_parity = 0;
        st.stall = 0;
        st.best_res = INFINITY;
        st.final_res = 0.0f;
        st.updates = 0ull;
        st.visits = 0u;
        // a sub-domain with the node set of a lower one has the same V
        int twin = -1;
        if (diff && i < 32)
            for (int j = 0; j < i; ++j)
                if (!((diff[j] >> i) & 1u)) {
                    twin = j;
                    break;
                }
        st.twin = twin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int na = 0;
        unsigned tm = 0u;
        for (int i = 0; i < nslots; ++i) {
            if (state[i].twin >= 0)
                tm |= 1u << i;
            else
                ctl->act_slot[na++] = i;
        }
        ctl->twin_mask = tm;
        ctl->nactive = na;
        ctl->sweep = 0u;
        ctl->done_ctas = 0u;
        ctl->error = 0;
        ctl->launches = 0u;
        ctl->gen = 0u;
        ctl->qcount[0] = 0;
        ctl->qcount[1] = 0;
        ctl->qhead[0] = 0;
        ctl->qhead[1] = 0;
    }
}

// Whether a tile's neighbourhood (the tiles its halo reaches: one tile in x
// and z, ceil(halo / rows) in y) holds a target node.
__device__ __forceinline__ bool near_target(const SlotDesc &S, int t) {
    const int txy = S.tiles_x * S.tiles_y;
    const int tz = t / txy, rem = t - tz * txy;
    const int ty = rem / S.tiles_x, tx = rem - ty * S.tiles_x;
    const int ry = (S.halo + S.trows - 1) / S.trows;
    const int rz = S.tiles_z > 1 ? 1 : 0;
    for (int dz = -rz; dz <= rz; ++dz) {
        const int z = ((tz + dz) % S.tiles_z + S.tiles_z) % S.tiles_z;  // periodic heading
        for (int dy = -ry; dy <= ry; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = tx + dx, y = ty + dy;
                if (x < 0 || x >= S.tiles_x || y < 0 || y >= S.tiles_y) continue;
                if (!S.tile_clear[(z * S.tiles_y + y) * S.tiles_x + x]) return true;
            }
    }
    return false;
}

// First queue: every member tile of every slot (with near_only, only those
// near a target), both flag arrays written (blockIdx.y = slot, threads over
// the slot's tiles).
__global__ void queue_init_kernel(const SlotDesc *slots, Ctl *ctl, int *qlist0, uint8_t *qflag0,
                                  uint8_t *qflag1, int near_only) {
    const int slot = blockIdx.y;
    const SlotDesc &S = slots[slot];
    const int lane = threadIdx.x & 31;
    const bool twin = slot < 32 && ((ctl->twin_mask >> slot) & 1u);
    for (int t0 = blockIdx.x * blockDim.x; t0 < S.ntiles; t0 += gridDim.x * blockDim.x) {
        const int t = t0 + threadIdx.x;
        bool member = false;
        if (t < S.ntiles) {
            member = !twin && (S.tile_bits == nullptr || ((S.tile_bits[t] >> S.mask_bit) & 1u));
            if (member && near_only && S.tile_clear != nullptr) member = near_target(S, t);
            qflag0[S.qbase + t] = member ? 1 : 0;
            qflag1[S.qbase + t] = 0;
        }
        const unsigned m = __ballot_sync(0xffffffffu, member);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&ctl->qcount[0], __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (member) qlist0[base + __popc(m & ((1u << lane) - 1u))] = (slot << 22) | t;
    }
}

// Starting iterate of every slot, written to both buffers (and the
// duplicated heading layers): targets take vtarget, ghosts and free nodes
// vout, or the warm start converted to the iterated variable.
__global__ void init_values_kernel(const SlotDesc *slots, int wform, float c_over,
                                   const float *v_init) {
    const SlotDesc &S = slots[blockIdx.y];
    const long long N = static_cast<long long>(S.nx) * S.ny * S.nz;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int cls = node_class(S, i);
        float v;
        if (cls == CLS_TARGET)
            v = S.vtarget;
        else if (cls == CLS_GHOST || v_init == nullptr)
            v = S.vout;
        else
            v = wform ? c_over - v_init[i] : v_init[i];
        const long long gx = i % S.nx;
        const long long r = i / S.nx;
        const long long gy = r % S.ny;
        const long long gz = r / S.ny;
        const long long row = gy * S.pitch + gx;
        for (int b = 0; b < 2; ++b) {
            float *D = S.V[b];
            D[(gz + S.zdup) * S.zstride + row] = v;
            if (gz < S.zdup) D[(gz + S.nz + S.zdup) * S.zstride + row] = v;
            if (gz >= S.nz - S.zdup) D[(gz - S.nz + S.zdup) * S.zstride + row] = v;
        }
    }
}

// Coarse-to-fine warm start of the decomposed solve (2D): the starting
// iterate of sub-domain k is the Q1 interpolation, at its free nodes, of the
// coarse auxiliary solution k of the reconstruction (slot k of `coarse`,
// iterated in the same variable), on a coarse grid whose nodes are every
// (r0, r1)-th fine node; targets take vtarget and ghosts vout, as in
// init_values_kernel.
__global__ void init_from_coarse_kernel(const SlotDesc *slots, const SlotDesc *coarse,
                                        const SlotState *cstate, int r0, int r1) {
    const SlotDesc &S = slots[blockIdx.y];
    const SlotDesc &K = coarse[blockIdx.y];
    const float *Vk = K.V[cstate[blockIdx.y].final_parity];
    const long long N = static_cast<long long>(S.nx) * S.ny;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int cls = node_class(S, i);
        const int gx = static_cast<int>(i % S.nx), gy = static_cast<int>(i / S.nx);
        float v;
        if (cls == CLS_TARGET) {
            v = S.vtarget;
        } else if (cls == CLS_GHOST) {
            v = S.vout;
        } else {
            int cx = gx / r0, cy = gy / r1;
            cx = cx > K.nx - 2 ? K.nx - 2 : cx;
            cy = cy > K.ny - 2 ? K.ny - 2 : cy;
            const float fx = static_cast<float>(gx - cx * r0) / static_cast<float>(r0);
            const float fy = static_cast<float>(gy - cy * r1) / static_cast<float>(r1);
            const float *q = Vk + static_cast<long long>(cy) * K.pitch + cx;
            const float a = fmaf(fx, q[1], (1.0f - fx) * q[0]);
            const float b = fmaf(fx, q[K.pitch + 1], (1.0f - fx) * q[K.pitch]);
            v = fmaf(fy, b, (1.0f - fy) * a);
        }
        const long long row = static_cast<long long>(gy) * S.pitch + gx;
        S.V[0][row] = v;
        S.V[1][row] = v;
    }
}

// Copy the latest iterate of one slot to a dense [N] array, converting
// W back to V = c_over - W in the W form.
__global__ void extract_kernel(const SlotDesc *slots, const SlotState *state, int slot, float *out,
                               int wform, float c_over) {
    const SlotDesc &S = slots[slot];
    const float *Vb = S.V[state[slot].final_parity];
    const long long N = static_cast<long long>(S.nx) * S.ny * S.nz;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long gx = i % S.nx;
        const long long r = i / S.nx;
        const long long gy = r % S.ny;
        const long long gz = r / S.ny;
        const float w = Vb[(gz + S.zdup) * S.zstride + gy * S.pitch + gx];
        out[i] = wform ? c_over - w : w;
    }
}

}  // namespace

namespace hjbh {

const void *sweep_kernel(const SweepKey &k, size_t *smem) {
    if (smem) *smem = 0;
    if (k.dubins) {
        if (k.halo != 2 || k.ty != TY || k.groups != 1 || k.lanes != 1) return nullptr;
        if (k.layers == 4) {
            if (k.loop)
                return k.wform ? reinterpret_cast<const void *>(&loop3d_kernel<true, 4>)
                               : reinterpret_cast<const void *>(&loop3d_kernel<false, 4>);
            return k.wform ? reinterpret_cast<const void *>(&sweep3d_kernel<true, 4>)
                           : reinterpret_cast<const void *>(&sweep3d_kernel<false, 4>);
        }
        if (k.layers == 2) {
            if (k.loop)
                return k.wform ? reinterpret_cast<const void *>(&loop3d_kernel<true, 2>)
                               : reinterpret_cast<const void *>(&loop3d_kernel<false, 2>);
            return k.wform ? reinterpret_cast<const void *>(&sweep3d_kernel<true, 2>)
                           : reinterpret_cast<const void *>(&sweep3d_kernel<false, 2>);
        }
        return nullptr;
    }
#define HJB_PICK(NA_, H_, TY_, G_, L_)                                                          \
    if (k.halo == H_ && k.ty == TY_ && k.groups == G_ && k.lanes == L_) {                        \
        if (k.loop)                                                                              \
            return k.wform ? reinterpret_cast<const void *>(                                     \
                                 &loop2d_kernel<NA_, true, H_, TY_, G_, L_>)                     \
                           : reinterpret_cast<const void *>(                                     \
                                 &loop2d_kernel<NA_, false, H_, TY_, G_, L_>);                   \
        return k.wform ? reinterpret_cast<const void *>(&sweep2d_kernel<NA_, true, H_, TY_, G_, L_>) \
                       : reinterpret_cast<const void *>(                                         \
                             &sweep2d_kernel<NA_, false, H_, TY_, G_, L_>);                       \
    }
#define HJB_PICK_SHAPES(NA_, H_) \
    HJB_PICK(NA_, H_, 8, 1, 1)   \
    HJB_PICK(NA_, H_, 4, 2, 1)   \
    HJB_PICK(NA_, H_, 2, 4, 1)
    switch (k.na) {
        case 64:
            HJB_PICK_SHAPES(64, 2)
            HJB_PICK_SHAPES(64, 4)
            HJB_PICK(64, 2, 4, 1, 2)
            HJB_PICK(64, 4, 4, 1, 2)
            break;
        case 32:
            HJB_PICK_SHAPES(32, 2)
            HJB_PICK_SHAPES(32, 4)
            HJB_PICK(32, 2, 4, 1, 2)
            HJB_PICK(32, 4, 4, 1, 2)
            break;
        case -1:  // generic count, P1 interpolation: one control group, 8-row tiles
            HJB_PICK(-1, 2, 8, 1, 1)
            HJB_PICK(-1, 4, 8, 1, 1)
            break;
        default:
            HJB_PICK_SHAPES(0, 2)
            HJB_PICK_SHAPES(0, 4)
            break;
    }
#undef HJB_PICK_SHAPES
#undef HJB_PICK
    return nullptr;
}

int sweep_grid(const SweepKey &k) {
    const void *f = sweep_kernel(k, nullptr);
    if (!f) return 0;
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, THREADS, 0);
    if (per < 1) per = 1;
    return sms * per;
}

void launch_loop_init(const SlotDesc * /*slots*/, SlotState *state, Ctl *ctl, int nslots,
                      cudaStream_t st, const uint32_t *diff) {
    loop_init_kernel<<<1, THREADS, 0, st>>>(state, ctl, nslots, diff);
}

void launch_queue_init(const SlotDesc *slots, int nslots, int max_tiles, Ctl *ctl, int *qlist0,
                       uint8_t *qflag0, uint8_t *qflag1, cudaStream_t st, int near_only) {
    int bx = (max_tiles + THREADS - 1) / THREADS;
    if (bx > 1024) bx = 1024;
    if (bx < 1) bx = 1;
    queue_init_kernel<<<dim3(bx, nslots), THREADS, 0, st>>>(slots, ctl, qlist0, qflag0, qflag1,
                                                            near_only);
}

void launch_init_values(const SlotDesc *slots, int nslots, int max_nodes, int wform, float c_over,
                        const float *v_init, cudaStream_t st) {
    int bx = (max_nodes + THREADS - 1) / THREADS;
    if (bx > 4096) bx = 4096;
    if (bx < 1) bx = 1;
    dim3 grid(bx, nslots);
    init_values_kernel<<<grid, THREADS, 0, st>>>(slots, wform, c_over, v_init);
}

void launch_init_from_coarse(const SlotDesc *slots, const SlotDesc *coarse,
                             const SlotState *cstate, int nslots, int max_nodes, int r0, int r1,
                             cudaStream_t st) {
    int bx = (max_nodes + THREADS - 1) / THREADS;
    if (bx > 4096) bx = 4096;
    if (bx < 1) bx = 1;
    init_from_coarse_kernel<<<dim3(bx, nslots), THREADS, 0, st>>>(slots, coarse, cstate, r0, r1);
}

void launch_extract(const SlotDesc *slots, const SlotState *state, int slot, float *out, int wform,
                    float c_over, cudaStream_t st) {
    extract_kernel<<<1184, THREADS, 0, st>>>(slots, state, slot, out, wform, c_over);
}

}  // namespace hjbh
