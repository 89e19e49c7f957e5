// subdomain.cu -- kernels of the reconstruction of independent sub-domains
// (RA, Sec. 3 of Festa, arXiv:1405.3521) and of the decomposed solve (ISA,
// Sec. 4): coarse-grid gather, labelling (RA steps 2-3), projection through
// the concave hull (ISA step 2), per-sub-domain tile work lists, assembly
// (ISA step 4), and small reductions used by the runtime.
#include <math.h>

#include "hjb_internal.cuh"

using namespace hjbk;

namespace {

__device__ __forceinline__ void unflat(const hjbh::GridDims &g, long long i, int idx[3]) {
    idx[0] = static_cast<int>(i % g.n[0]);
    const long long r = i / g.n[0];
    idx[1] = static_cast<int>(r % g.n[1]);
    idx[2] = g.ndim > 2 ? static_cast<int>(r / g.n[1]) : 0;
}

__device__ __forceinline__ long long flat(const hjbh::GridDims &g, int x, int y, int z) {
    return (static_cast<long long>(z) * g.n[1] + y) * g.n[0] + x;
}

__device__ __forceinline__ long long count(const hjbh::GridDims &g) {
    return static_cast<long long>(g.n[0]) * g.n[1] * (g.ndim > 2 ? g.n[2] : 1);
}

#define GRID_STRIDE(i, n)                                                                  \
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < (n); \
         i += static_cast<long long>(gridDim.x) * blockDim.x)

__global__ void gather_coarse_kernel(hjbh::GridDims fine, hjbh::GridDims coarse, int r0, int r1,
                                     int r2, const float *speed, const float *current,
                                     const float *cost, const uint8_t *labels, const float *scale,
                                     float *c_speed, float *c_current, float *c_cost,
                                     uint8_t *c_labels, float *c_scale) {
    const long long NK = count(coarse);
    GRID_STRIDE(k, NK) {
        int c[3];
        unflat(coarse, k, c);
        const long long i = flat(fine, c[0] * r0, c[1] * r1, c[2] * r2);
        if (c_speed) c_speed[k] = speed[i];
        if (c_current) {
            c_current[2 * k] = current[2 * i];
            c_current[2 * k + 1] = current[2 * i + 1];
        }
        if (c_cost) c_cost[k] = cost[i];
        if (c_scale) {
            c_scale[2 * k] = scale[2 * i];
            c_scale[2 * k + 1] = scale[2 * i + 1];
        }
        c_labels[k] = labels[i];
    }
}

// Value of slot k's latest iterate at node (x, y, z).
__device__ __forceinline__ float slot_value(const SlotDesc &S, const SlotState &st, int x, int y,
                                            int z) {
    const float *V = S.V[st.final_parity];
    return V[static_cast<long long>(z + S.zdup) * S.zstride + static_cast<long long>(y) * S.pitch + x];
}

// RA step 2 (V = min_k V_k) and step 3 (threshold of eq. rep) at every
// coarse node.  In the W form W = c - V, so min over V is max over W and the
// differences |V_k - V| = |W_k - W| are computed on W directly.
__global__ void label_kernel(const SlotDesc *slots, const SlotState *state, int m,
                             hjbh::GridDims coarse, const uint8_t *labels, float delta, int wform,
                             uint32_t *labels_out, float *vmin_out, unsigned long long *ties_out) {
    const long long NK = count(coarse);
    unsigned long long ties = 0;
    GRID_STRIDE(j, NK) {
        int c[3];
        unflat(coarse, j, c);
        float vk[HJB_MAX_TARGETS_DEV];
        float best = wform ? -INFINITY : INFINITY;
        for (int k = 0; k < m; ++k) {
            vk[k] = slot_value(slots[k], state[k], c[0], c[1], c[2]);
            best = wform ? fmaxf(best, vk[k]) : fminf(best, vk[k]);
        }
        const int lab = labels[j];
        uint32_t bits = 0u;
        for (int k = 0; k < m; ++k) {
            const float diff = fabsf(vk[k] - best);
            if (lab == k + 1 || diff <= delta) bits |= 1u << k;
            if (fabsf(diff - delta) <= 1e-6f) ++ties;
        }
        labels_out[j] = bits;
        if (vmin_out) vmin_out[j] = best;
    }
    if (ties) atomicAdd(ties_out, ties);
}

__device__ __forceinline__ float vmin_at(const SlotDesc *slots, const SlotState *state, int m,
                                         int wform, int x, int y, int z) {
    float best = wform ? -INFINITY : INFINITY;
    for (int k = 0; k < m; ++k) {
        const float v = slot_value(slots[k], state[k], x, y, z);
        best = wform ? fmaxf(best, v) : fminf(best, v);
    }
    return best;
}

// Largest discrete gradient norm of V = min_k V_k (centred differences,
// one-sided at non-periodic edges), an estimate of the Lipschitz constant M
// of Prop. 3.1.
__global__ void grad_max_kernel(const SlotDesc *slots, const SlotState *state, int m, int wform,
                                hjbh::GridDims g, float dx0, float dx1, float dx2, unsigned *out) {
    const long long NK = count(g);
    const float dx[3] = {dx0, dx1, dx2};
    float mx = 0.0f;
    GRID_STRIDE(j, NK) {
        int c[3];
        unflat(g, j, c);
        float s2 = 0.0f;
        for (int d = 0; d < g.ndim; ++d) {
            int a[3] = {c[0], c[1], c[2]}, b[3] = {c[0], c[1], c[2]};
            const int n = g.n[d];
            float span = 2.0f * dx[d];
            if (g.periodic[d]) {
                a[d] = (c[d] + n - 1) % n;
                b[d] = (c[d] + 1) % n;
            } else if (c[d] == 0) {
                b[d] = 1;
                span = dx[d];
            } else if (c[d] == n - 1) {
                a[d] = n - 2;
                span = dx[d];
            } else {
                a[d] = c[d] - 1;
                b[d] = c[d] + 1;
            }
            const float va = vmin_at(slots, state, m, wform, a[0], a[1], a[2]);
            const float vb = vmin_at(slots, state, m, wform, b[0], b[1], b[2]);
            const float gd = (vb - va) / span;
            s2 += gd * gd;
        }
        mx = fmaxf(mx, sqrtf(s2));
    }
    atomicMax(out, __float_as_uint(mx));
}

// ISA step 2 (projection remark of Sec. 4): x_j belongs to the projected
// sub-domain k iff it lies in Con, the union of the simplices of the coarse
// triangulation whose vertices all carry label k.  The coarse cells are split
// into Kuhn simplices; the fine node lies in the closed simplex selected by
// the ordering of its local coordinates t_d = loc_d / r_d, and belongs to
// Con iff every vertex with a non-zero barycentric weight is labelled.
// Everything is integer: coordinates are compared by cross-multiplication.
__global__ void project_kernel(hjbh::GridDims fine, hjbh::GridDims coarse, int r0, int r1, int r2,
                               const uint32_t *cl, uint32_t *out) {
    const long long N = count(fine);
    const int r[3] = {r0, r1, r2};
    GRID_STRIDE(i, N) {
        int idx[3];
        unflat(fine, i, idx);
        int cell[3] = {0, 0, 0}, loc[3] = {0, 0, 0};
        for (int d = 0; d < fine.ndim; ++d) {
            int c = idx[d] / r[d];
            if (!coarse.periodic[d] && c > coarse.n[d] - 2) c = coarse.n[d] - 2;
            cell[d] = c;
            loc[d] = idx[d] - c * r[d];
        }
        // sort dimensions by decreasing t_d (stable: lower dimension first on ties)
        int ord[3] = {0, 1, 2};
        for (int a = 1; a < fine.ndim; ++a) {
            for (int b = a; b > 0; --b) {
                const int p = ord[b - 1], q = ord[b];
                // t_q > t_p  <=>  loc_q r_p > loc_p r_q
                if (static_cast<long long>(loc[q]) * r[p] > static_cast<long long>(loc[p]) * r[q]) {
                    ord[b - 1] = q;
                    ord[b] = p;
                } else {
                    break;
                }
            }
        }
        uint32_t acc = 0xffffffffu;
        int v[3] = {cell[0], cell[1], cell[2]};
        for (int k = 0; k <= fine.ndim; ++k) {
            if (k > 0) v[ord[k - 1]] += 1;
            // weight of vertex k: t_{ord[k-1]} - t_{ord[k]} (t_{ord[-1]} = 1, t_{ord[D]} = 0)
            long long nh, dh, nl, dl;
            if (k == 0) {
                nh = 1;
                dh = 1;
            } else {
                nh = loc[ord[k - 1]];
                dh = r[ord[k - 1]];
            }
            if (k == fine.ndim) {
                nl = 0;
                dl = 1;
            } else {
                nl = loc[ord[k]];
                dl = r[ord[k]];
            }
            if (nh * dl > nl * dh) {
                int w[3] = {v[0], v[1], v[2]};
                for (int d = 0; d < fine.ndim; ++d)
                    if (coarse.periodic[d]) w[d] %= coarse.n[d];
                acc &= cl[flat(coarse, w[0], w[1], fine.ndim > 2 ? w[2] : 0)];
            }
        }
        out[i] = acc;
    }
}

// OR of the sub-domain bits over the nodes of each tile (one block per tile;
// tiles are 32 x ty (x TZ in 3D) nodes).
__global__ void tile_bits_kernel(hjbh::GridDims g, int tiles_x, int tiles_y, int ty_rows,
                                 int tz_layers, const uint32_t *mask, uint32_t *tile_bits,
                                 uint32_t *diff, int m, uint32_t *tile_full) {
    const int t = blockIdx.x;
    const int txy = tiles_x * tiles_y;
    const int tz = t / txy, rem = t - tz * txy;
    const int ty = rem / tiles_x, tx = rem - ty * tiles_x;
    const int x = tx * TX + (threadIdx.x & 31);
    const uint32_t mbits = m >= 32 ? 0xffffffffu : ((1u << m) - 1u);
    uint32_t bits = 0u, all = 0xffffffffu;
    // dk[k]: sub-domains whose membership differs from k's at a node seen here
    uint32_t dk[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) dk[k] = 0u;
    const int zn = g.ndim > 2 ? tz_layers : 1;
    for (int r = threadIdx.x >> 5; r < ty_rows * zn; r += THREADS / 32) {
        const int y = ty * ty_rows + r % ty_rows;
        const int z = g.ndim > 2 ? tz * tz_layers + r / ty_rows : 0;
        if (x < g.n[0] && y < g.n[1] && (g.ndim < 3 || z < g.n[2])) {
            const uint32_t v = mask[flat(g, x, y, z)];
            bits |= v;
            all &= v;
            if (diff) {
                const uint32_t b = v & mbits;
#pragma unroll
                for (int k = 0; k < 32; ++k) dk[k] |= ((b >> k) & 1u) ? (~b & mbits) : b;
            }
        }
    }
    bits = __reduce_or_sync(0xffffffffu, bits);
    all = __reduce_and_sync(0xffffffffu, all);
    __shared__ uint32_t s[THREADS / 32], s_all[THREADS / 32];
    __shared__ uint32_t s_d[THREADS / 32][32];
    if ((threadIdx.x & 31) == 0) {
        s[threadIdx.x >> 5] = bits;
        s_all[threadIdx.x >> 5] = all;
    }
    if (diff) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const uint32_t w = __reduce_or_sync(0xffffffffu, dk[k]);
            if ((threadIdx.x & 31) == 0) s_d[threadIdx.x >> 5][k] = w;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t b = 0u, a = 0xffffffffu;
        for (int w = 0; w < THREADS / 32; ++w) {
            b |= s[w];
            a &= s_all[w];
        }
        tile_bits[t] = b;
        if (tile_full) tile_full[t] = a;  // every node of the tile in these sub-domains
    }
    if (diff && threadIdx.x < 32) {
        uint32_t w = 0u;
        for (int q = 0; q < THREADS / 32; ++q) w |= s_d[q][threadIdx.x];
        // most words saturate early: skip the atomic when it adds nothing
        if (w & ~__ldcg(&diff[threadIdx.x])) atomicOr(&diff[threadIdx.x], w);
    }
}

// 1 for tiles without target nodes (one block per tile).
__global__ void tile_clear_kernel(hjbh::GridDims g, int tiles_x, int tiles_y, int ty_rows,
                                  int tz_layers, const uint8_t *labels, uint8_t *clear) {
    const int t = blockIdx.x;
    const int txy = tiles_x * tiles_y;
    const int tz = t / txy, rem = t - tz * txy;
    const int ty = rem / tiles_x, tx = rem - ty * tiles_x;
    const int x = tx * TX + (threadIdx.x & 31);
    const int zn = g.ndim > 2 ? tz_layers : 1;
    int any = 0;
    for (int r = threadIdx.x >> 5; r < ty_rows * zn; r += THREADS / 32) {
        const int y = ty * ty_rows + r % ty_rows;
        const int z = g.ndim > 2 ? tz * tz_layers + r / ty_rows : 0;
        if (x < g.n[0] && y < g.n[1] && (g.ndim < 3 || z < g.n[2]))
            any |= labels[flat(g, x, y, z)] != 0;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) clear[t] = any ? 0 : 1;
}

// ISA step 4: Vbar(j) = min{ V_k(j) : bit k of mask[j] } (max of W in the
// W form), value_out on nodes that belong to no sub-domain.
__global__ void assemble_kernel(const SlotDesc *slots, const SlotState *state, int m,
                                hjbh::GridDims g, const uint32_t *mask, int wform, float c_over,
                                float vout_v, float *out, const Ctl *ctl) {
    const long long N = count(g);
    const uint32_t skip = ctl ? ctl->twin_mask : 0u;
    GRID_STRIDE(i, N) {
        int c[3];
        unflat(g, i, c);
        uint32_t bits = mask[i] & ~skip;
        if (m < 32) bits &= (1u << m) - 1u;
        float best = wform ? -INFINITY : INFINITY;
        while (bits) {
            const int k = __ffs(bits) - 1;
            bits &= bits - 1u;
            const float v = slot_value(slots[k], state[k], c[0], c[1], c[2]);
            best = wform ? fmaxf(best, v) : fminf(best, v);
        }
        float res;
        if (isinf(best))
            res = vout_v;
        else
            res = wform ? c_over - best : best;
        out[i] = res;
    }
}

// Largest |x| over a strided field; a non-finite entry yields +inf so that
// the caller rejects the field.  One atomic per CTA (per-warp atomics on one
// address serialised the reduction).
__global__ void absmax_kernel(const float *x, long long n, int stride, int offset, unsigned *out) {
    __shared__ float s_m[THREADS / 32];
    float m = 0.0f;
    GRID_STRIDE(i, n) {
        float a = fabsf(x[i * stride + offset]);
        if (!(a <= 3.402823466e38f)) a = INFINITY;
        m = fmaxf(m, a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 1; w < THREADS / 32; ++w) m = fmaxf(m, s_m[w]);
        atomicMax(out, __float_as_uint(m));
    }
}

__global__ void exp_kernel(const float *th, float *s, long long n) {
    GRID_STRIDE(i, n) s[i] = expf(th[i]);
}

__global__ void popcount_kernel(const uint32_t *mask, long long n, unsigned long long *out) {
    __shared__ unsigned long long s_c[THREADS / 32];
    unsigned long long c = 0;
    GRID_STRIDE(i, n) c += __popc(mask[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_c[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 1; w < THREADS / 32; ++w) c += s_c[w];
        if (c) atomicAdd(out, c);
    }
}

// Nodes of each of the m sub-domains of a mask (out[k] += |bit k|).
__global__ void bitcount_kernel(const uint32_t *mask, long long n, int m, unsigned long long *out) {
    __shared__ unsigned s_cnt[32];
    if (threadIdx.x < 32) s_cnt[threadIdx.x] = 0u;
    __syncthreads();
    unsigned c[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) c[k] = 0u;
    GRID_STRIDE(i, n) {
        const uint32_t v = mask[i];
#pragma unroll
        for (int k = 0; k < 32; ++k) c[k] += (v >> k) & 1u;
    }
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const unsigned w = __reduce_add_sync(0xffffffffu, c[k]);
        if ((threadIdx.x & 31) == 0 && w && k < m) atomicAdd(&s_cnt[k], w);
    }
    __syncthreads();
    if (threadIdx.x < m && s_cnt[threadIdx.x])
        atomicAdd(&out[threadIdx.x], static_cast<unsigned long long>(s_cnt[threadIdx.x]));
}

// Index extents (x min, x max, y min, y max) and node count of target
// component `comp` (label value) of a label array.
__global__ void comp_extent_kernel(hjbh::GridDims g, const uint8_t *labels, int comp, int *ext,
                                   unsigned *nodes) {
    const long long N = count(g);
    int lox = 1 << 30, hix = -1, loy = 1 << 30, hiy = -1;
    unsigned c = 0;
    GRID_STRIDE(i, N) {
        if (labels[i] != comp) continue;
        int idx[3];
        unflat(g, i, idx);
        lox = min(lox, idx[0]);
        hix = max(hix, idx[0]);
        loy = min(loy, idx[1]);
        hiy = max(hiy, idx[1]);
        ++c;
    }
    if (c) {
        atomicMin(&ext[0], lox);
        atomicMax(&ext[1], hix);
        atomicMin(&ext[2], loy);
        atomicMax(&ext[3], hiy);
        atomicAdd(nodes, c);
    }
}

// Histogram of the component's nodes along one grid axis.
__global__ void comp_hist_kernel(hjbh::GridDims g, const uint8_t *labels, int comp, int axis,
                                 unsigned *hist) {
    const long long N = count(g);
    GRID_STRIDE(i, N) {
        if (labels[i] != comp) continue;
        int idx[3];
        unflat(g, i, idx);
        atomicAdd(&hist[idx[axis]], 1u);
    }
}

// Relabel the component's nodes with index > s on the axis as new_comp.
__global__ void comp_split_kernel(hjbh::GridDims g, uint8_t *labels, int comp, int axis, int s,
                                  int new_comp) {
    const long long N = count(g);
    GRID_STRIDE(i, N) {
        if (labels[i] != comp) continue;
        int idx[3];
        unflat(g, i, idx);
        if (idx[axis] > s) labels[i] = static_cast<uint8_t>(new_comp);
    }
}

int blocks_for(long long n) {
    long long b = (n + THREADS - 1) / THREADS;
    if (b > 4096) b = 4096;
    if (b < 1) b = 1;
    return static_cast<int>(b);
}

// Reductions to one counter: a grid of at most 4 CTAs per SM of a GB300
// (608), each thread striding over the field.
int reduction_blocks(long long n) {
    const int b = blocks_for(n);
    return b < 608 ? b : 608;
}

}  // namespace

namespace hjbh {

void launch_gather_coarse(const GridDims &fine, const GridDims &coarse, const int stride[3],
                          const float *speed, const float *current, const float *cost,
                          const uint8_t *labels, const float *scale, float *c_speed,
                          float *c_current, float *c_cost, uint8_t *c_labels, float *c_scale,
                          cudaStream_t st) {
    long long NK = static_cast<long long>(coarse.n[0]) * coarse.n[1] * (coarse.ndim > 2 ? coarse.n[2] : 1);
    gather_coarse_kernel<<<blocks_for(NK), THREADS, 0, st>>>(
        fine, coarse, stride[0], stride[1], coarse.ndim > 2 ? stride[2] : 1, speed, current, cost,
        labels, scale, speed ? c_speed : nullptr, current ? c_current : nullptr,
        cost ? c_cost : nullptr, c_labels, scale ? c_scale : nullptr);
}

void launch_label(const SlotDesc *slots, const SlotState *state, int m, const GridDims &coarse,
                  const uint8_t *labels, float delta, int wform, uint32_t *labels_out,
                  float *vmin_out, unsigned long long *ties_out, cudaStream_t st) {
    long long NK = static_cast<long long>(coarse.n[0]) * coarse.n[1] * (coarse.ndim > 2 ? coarse.n[2] : 1);
    label_kernel<<<blocks_for(NK), THREADS, 0, st>>>(slots, state, m, coarse, labels, delta, wform,
                                                    labels_out, vmin_out, ties_out);
}

void launch_grad_max(const SlotDesc *slots, const SlotState *state, int m, int wform,
                     const GridDims &coarse, const float dx[3], unsigned *out, cudaStream_t st) {
    long long NK = static_cast<long long>(coarse.n[0]) * coarse.n[1] * (coarse.ndim > 2 ? coarse.n[2] : 1);
    grad_max_kernel<<<blocks_for(NK), THREADS, 0, st>>>(slots, state, m, wform,
                                                       coarse, dx[0], dx[1], dx[2], out);
}

void launch_project(const GridDims &fine, const GridDims &coarse, const int stride[3],
                    const uint32_t *coarse_labels, uint32_t *fine_mask, cudaStream_t st) {
    long long N = static_cast<long long>(fine.n[0]) * fine.n[1] * (fine.ndim > 2 ? fine.n[2] : 1);
    project_kernel<<<blocks_for(N), THREADS, 0, st>>>(fine, coarse, stride[0], stride[1],
                                                     fine.ndim > 2 ? stride[2] : 1, coarse_labels,
                                                     fine_mask);
}

void launch_tile_bits(const GridDims &fine, int tiles_x, int tiles_y, int tiles_z, int ty, int tz,
                      const uint32_t *mask, uint32_t *tile_bits, cudaStream_t st, uint32_t *diff,
                      int m, uint32_t *tile_full) {
    const int nt = tiles_x * tiles_y * tiles_z;
    tile_bits_kernel<<<nt, THREADS, 0, st>>>(fine, tiles_x, tiles_y, ty, tz, mask, tile_bits, diff,
                                             m, tile_full);
}

void launch_tile_clear(const GridDims &g, int tiles_x, int tiles_y, int tiles_z, int ty, int tz,
                       const uint8_t *labels, uint8_t *clear, cudaStream_t st) {
    tile_clear_kernel<<<tiles_x * tiles_y * tiles_z, THREADS, 0, st>>>(g, tiles_x, tiles_y, ty, tz,
                                                                      labels, clear);
}

void launch_assemble(const SlotDesc *slots, const SlotState *state, int m, const GridDims &fine,
                     const uint32_t *mask, int wform, float c_over, float vout_v, float *out,
                     cudaStream_t st, const Ctl *ctl) {
    long long N = static_cast<long long>(fine.n[0]) * fine.n[1] * (fine.ndim > 2 ? fine.n[2] : 1);
    assemble_kernel<<<blocks_for(N), THREADS, 0, st>>>(slots, state, m, fine, mask, wform, c_over,
                                                      vout_v, out, ctl);
}

void launch_absmax(const float *x, long long n, int stride, int offset, unsigned *out,
                   cudaStream_t st) {
    absmax_kernel<<<reduction_blocks(n), THREADS, 0, st>>>(x, n, stride, offset, out);
}

void launch_exp(const float *theta, float *s, long long n, cudaStream_t st) {
    exp_kernel<<<blocks_for(n), THREADS, 0, st>>>(theta, s, n);
}

void launch_bitcount(const uint32_t *mask, long long n, int m, unsigned long long *out,
                     cudaStream_t st) {
    bitcount_kernel<<<blocks_for(n), THREADS, 0, st>>>(mask, n, m, out);
}

void launch_comp_extent(const GridDims &g, const uint8_t *labels, int comp, int *ext,
                        unsigned *count_out, cudaStream_t st) {
    const long long N = static_cast<long long>(g.n[0]) * g.n[1] * (g.ndim > 2 ? g.n[2] : 1);
    comp_extent_kernel<<<blocks_for(N), THREADS, 0, st>>>(g, labels, comp, ext, count_out);
}

void launch_comp_hist(const GridDims &g, const uint8_t *labels, int comp, int axis, unsigned *hist,
                      cudaStream_t st) {
    const long long N = static_cast<long long>(g.n[0]) * g.n[1] * (g.ndim > 2 ? g.n[2] : 1);
    comp_hist_kernel<<<blocks_for(N), THREADS, 0, st>>>(g, labels, comp, axis, hist);
}

void launch_comp_split(const GridDims &g, uint8_t *labels, int comp, int axis, int s, int new_comp,
                       cudaStream_t st) {
    const long long N = static_cast<long long>(g.n[0]) * g.n[1] * (g.ndim > 2 ? g.n[2] : 1);
    comp_split_kernel<<<blocks_for(N), THREADS, 0, st>>>(g, labels, comp, axis, s, new_comp);
}

void launch_popcount(const uint32_t *mask, long long n, unsigned long long *out, cudaStream_t st) {
    popcount_kernel<<<reduction_blocks(n), THREADS, 0, st>>>(mask, n, out);
}

}  // namespace hjbh
