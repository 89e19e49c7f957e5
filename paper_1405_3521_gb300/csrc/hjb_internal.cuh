// hjb_internal.cuh -- device-side data structures shared by the kernels and
// the host runtime of the GB300 HJB library.  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hjbk {

// 2D tile: 32 x 8 nodes, one node per thread (256 threads).
constexpr int TX = 32;
constexpr int TY = 8;
// 3D tile: 32 x 8 x TZ nodes, each thread walks TZ layers (the default; the
// sweep also has tiles of 2 layers).
constexpr int TZ = 4;
// x halo padding in shared memory: TMA boxes must start at x coordinates
// whose byte offset is a multiple of 16, so the x halo is widened to 4 floats.
constexpr int XPAD = 4;
constexpr int TW = TX + 2 * XPAD;  // shared-memory row width (floats)
constexpr int THREADS = 256;
constexpr int MAX_SLOTS = 1024;
constexpr int MAX_CTRL = 128;
#define HJB_MAX_TARGETS_DEV 32
// Bounded waits: a TMA transaction that has not completed after this many
// nanoseconds is treated as lost; the kernel records an error and returns.
constexpr unsigned long long WAIT_NS = 2000000000ull;

// Discrete control set, passed by value in the kernel parameters so that a
// fully unrolled loop reads the components as constant-bank operands.
struct ControlTable {
    float2 a2[MAX_CTRL];  // (ax, ay) pairs for the packed FP32x2 path
    float ax[MAX_CTRL];
    float ay[MAX_CTRL];
    int count;
    int nb;  // games: count = na * nb pairs a_j - b_k at k * na + j; else 1
};
// Shared-memory pair layout of the 2D sweep: row r, column c holds
// (V[r][c], V[r][c+1]) as a float2; rows are PW float2 (512 bytes) apart.
constexpr int PW = 64;

// One independent fixed-point problem ("slot") of a launch: the full grid,
// an auxiliary problem of the reconstruction, a sub-domain of the decomposed
// solve, or one problem of a batch.
struct alignas(128) SlotDesc {
    CUtensorMap tmap[2];        // TMA maps of the two iteration buffers
    float *V[2];                // pitched iteration buffers [nzl][ny][pitch]
    const float *speed;         // node field s (or null: s = 1)
    const float2 *scale2;       // node field of per-axis factors (or null; replaces speed)
    const float *current;       // node field c [N][2] (or null)
    const float *cost;          // node field l (or null: constant)
    const uint8_t *labels;      // target labels [N]
    const uint32_t *mask;       // sub-domain bitmask [N] (or null)
    const uint32_t *tile_bits;  // per-tile OR of the sub-domain bits (masked slots), or null
    const uint32_t *tile_full;  // per-tile AND of the sub-domain bits (tiles inside a sub-domain)
    const uint8_t *tile_clear;  // per tile: 1 = no target node in it (or null)
    const float2 *trig;         // Dubins: per heading layer (v h cos/dx, v h sin/dy)
    long long zstride;          // floats between layers of V
    int nx, ny, nz, pitch;
    int tiles_x, tiles_y, tiles_z, ntiles;  // ntiles = tiles_x * tiles_y * tiles_z
    int qbase;                  // offset of this slot's tiles in the queue flag arrays
    int mask_bit, only_target;  // restricted problem / auxiliary problem selectors
    int zdup;                   // duplicated heading layers on each side (periodic z)
    int halo;                   // interpolation halo in x, y (cells)
    float hx, hy, hz;           // h / spacing per dimension
    float beta;                 // exp(-lambda h)
    float gl;                   // gamma * l_const (V form)
    float gamma;                // (1 - beta)/lambda (V form with a cost field)
    float vout;                 // ghost / outside value in the iterated variable
    float vtarget;              // target value in the iterated variable
    float tol;
    int max_iters;
    int trows;                  // tile rows (2D 8, 4 or 2; 3D 8)
    int tlayers;                // tile heading layers (3D), 1 in 2D
};
static_assert(sizeof(SlotDesc) % 128 == 0, "slot descriptors are 128-byte aligned");

// Convergence state of a slot.
struct SlotState {
    unsigned res_bits;           // atomicMax target: residual of the running sweep
    int iters;
    int done;
    int converged;               // 1 tol reached, 2 stagnated at rounding level
    int final_parity;            // buffer holding the latest iterate
    int stall;
    float best_res;
    float final_res;
    unsigned long long updates;  // free-node evaluations of T
    int twin;                    // lower slot with the same node set (not solved), else -1
    unsigned visits;             // staged tile items processed (sum over sweeps)
};

// Launch-wide control block.
// The words every CTA hits each sweep (arrival counter, barrier generation,
// queue counters) sit on separate 128-byte lines so that the atomics of one
// do not contend with the polling of another.
struct Ctl {
    alignas(128) unsigned done_ctas;
    alignas(128) unsigned gen;  // generation of the cooperative loop's grid barrier
    alignas(128) int qcount[2];  // entries of the two tile queues (parity = sweep parity)
    // queue entries handed out past each CTA's first one (dynamic scheduling)
    alignas(128) int qhead[2];
    alignas(128) unsigned sweep;  // number of sweeps so far (parity of the source buffer)
    int nactive;
    int error;           // non-zero: a bounded wait gave up
    unsigned launches;   // sweep kernels run (including empty ones at the loop's end)
    unsigned twin_mask;  // slots (< 32) that duplicate a lower slot's node set
    int act_slot[MAX_SLOTS];
};

// Work queue of a sweep: the tiles whose 3x3 (3x3x3) tile neighbourhood
// changed in the previous sweep.  Entries pack (slot << 22) | tile.
struct SweepArgs {
    const SlotDesc *slots;
    SlotState *state;
    Ctl *ctl;
    int *qlist[2];
    uint8_t *qflag[2];
    int nslots;
    int use_handle;
    cudaGraphConditionalHandle handle;
    float stall_tol;
    int local_iters;  // applications of T per tile and sweep (2D; >= 1)
    // 1: a CTA takes its items after the first from a shared counter, so
    // CTAs that drew cheap tiles take more; 0: CTA b takes entries b,
    // b + grid, b + 2 grid, ...  The iterates do not depend on the order.
    int dyn_queue;
    ControlTable ctrl;
};

}  // namespace hjbk

// Host-side entry points of the kernels (defined in the .cu files).
namespace hjbh {

// Kernel selection key for the sweep.
struct SweepKey {
    int dubins;  // 0: 2D speed/current, 1: 3D Dubins
    int wform;   // iterate on W (max form) instead of V (min form)
    int na;      // number of controls
    int halo;    // 2 or 4 (2D), 2 (3D)
    int ty;      // tile rows: 8, 4 or 2 (2D); 8 (3D)
    int groups;  // warp groups splitting the controls of a node: 256 / (32 ty lanes)
    int loop;    // 1: the cooperative whole-loop kernel, 0: one sweep per launch
    int lanes;   // 2D: 1, or 2 lanes per node taking a_j and -a_j (32 x 4 tiles)
    int layers;  // 3D: heading layers per tile (4 or 2); 1 in 2D
};

// Returns the kernel function for a key (nullptr if unsupported) and the
// dynamic shared memory it needs.
const void *sweep_kernel(const SweepKey &k, size_t *smem);
// Occupancy-derived persistent grid size for the kernel.
int sweep_grid(const SweepKey &k);

// Kernels used around the loop (see their definitions for the contracts).
// diff (optional, decomposed solve): bit j of diff[k] is set iff the node
// sets of sub-domains k and j differ somewhere.  A slot whose node set equals
// that of a lower slot is marked as its twin and left out of the loop.
void launch_loop_init(const hjbk::SlotDesc *slots, hjbk::SlotState *state, hjbk::Ctl *ctl,
                      int nslots, cudaStream_t st, const uint32_t *diff = nullptr);
// Queue of the first sweep: every tile of every slot that holds a node of it
// (for masked slots: tile_bits carries the slot's bit); both flag arrays set.
// near_only: queue only tiles whose neighbourhood (the tiles a halo
// reaches) holds a target node -- exact when the start is a fixed point of T
// away from targets (the W form from W = 0 with a zero outside value).
void launch_queue_init(const hjbk::SlotDesc *slots, int nslots, int max_tiles, hjbk::Ctl *ctl,
                       int *qlist0, uint8_t *qflag0, uint8_t *qflag1, cudaStream_t st,
                       int near_only = 0);
void launch_init_values(const hjbk::SlotDesc *slots, int nslots, int max_nodes, int wform,
                        float c_over, const float *v_init, cudaStream_t st);
// Coarse-to-fine warm start (2D): slot k starts from the Q1 interpolation of
// coarse slot k (every (r0, r1)-th fine node is a coarse node).
void launch_init_from_coarse(const hjbk::SlotDesc *slots, const hjbk::SlotDesc *coarse,
                             const hjbk::SlotState *cstate, int nslots, int max_nodes, int r0,
                             int r1, cudaStream_t st);
void launch_extract(const hjbk::SlotDesc *slots, const hjbk::SlotState *state, int slot,
                    float *out, int wform, float c_over, cudaStream_t st);

// RA step 1 on chip (coarse.cu): whether an nx x ny coarse grid with the
// given interpolation halo fits the cluster kernel's shared memory (and its
// layout), and the launch solving the m auxiliary problems of slots[0..m)
// to convergence, one thread-block cluster per problem; the result goes to
// each slot's buffer 0 and its state (iters, converged, updates).  Returns 0
// on success.
int coarse_fits(int nx, int ny, int halo, size_t *smem_bytes, int *nbands, int *band_max);
int launch_coarse_solve(const hjbk::SlotDesc *slots, hjbk::SlotState *state, int m, int nx, int ny,
                        int halo, int interp, int wform, const hjbk::ControlTable &ctrl,
                        float stall_tol, cudaStream_t st);

// Grid geometry shared by the reconstruction kernels.
struct GridDims {
    int ndim;
    int n[3];
    int periodic[3];
};

// Fine -> coarse gather of node fields at the coarse stride (any pointer may
// be null).
void launch_gather_coarse(const GridDims &fine, const GridDims &coarse, const int stride[3],
                          const float *speed, const float *current, const float *cost,
                          const uint8_t *labels, const float *scale, float *c_speed,
                          float *c_current, float *c_cost, uint8_t *c_labels, float *c_scale,
                          cudaStream_t st);
// RA steps 2-3: labels of the coarse nodes from the m auxiliary solutions
// held by slots[0..m) (min property + threshold of eq. rep).  ties_out is an
// unsigned long long counter (accumulated); vmin_out optional.
void launch_label(const hjbk::SlotDesc *slots, const hjbk::SlotState *state, int m,
                  const GridDims &coarse, const uint8_t *labels, float delta, int wform,
                  uint32_t *labels_out, float *vmin_out, unsigned long long *ties_out,
                  cudaStream_t st);
// Largest centred-difference gradient norm of min_k V_k over the coarse grid
// (physical units, dx per dimension); result as float bits in *out (atomicMax).
void launch_grad_max(const hjbk::SlotDesc *slots, const hjbk::SlotState *state, int m,
                     int wform, const GridDims &coarse, const float dx[3], unsigned *out,
                     cudaStream_t st);
// ISA step 2: fine bitmask from coarse labels through the Kuhn simplices.
void launch_project(const GridDims &fine, const GridDims &coarse, const int stride[3],
                    const uint32_t *coarse_labels, uint32_t *fine_mask, cudaStream_t st);
// Per tile: 1 when none of its nodes is a target node (labels != 0); tiles
// of 32 x ty (x tz) nodes.
void launch_tile_clear(const GridDims &g, int tiles_x, int tiles_y, int tiles_z, int ty, int tz,
                       const uint8_t *labels, uint8_t *clear, cudaStream_t st);
// Per-tile OR (and, optionally, AND: tile_full) of the sub-domain bits of
// the decomposed solve.  diff
// (optional, [32], zeroed by the caller): bit j of diff[k] is OR-ed in where
// the node sets of sub-domains k and j differ (m sub-domains, m <= 32).
void launch_tile_bits(const GridDims &fine, int tiles_x, int tiles_y, int tiles_z, int ty, int tz,
                      const uint32_t *mask, uint32_t *tile_bits, cudaStream_t st,
                      uint32_t *diff = nullptr, int m = 0, uint32_t *tile_full = nullptr);
// ISA step 4: Vbar = min over the sub-domains containing each node.  Slots
// in ctl->twin_mask (ctl optional) are skipped: their twin holds the same V.
void launch_assemble(const hjbk::SlotDesc *slots, const hjbk::SlotState *state, int m,
                     const GridDims &fine, const uint32_t *mask, int wform, float c_over,
                     float vout_v, float *out, cudaStream_t st, const hjbk::Ctl *ctl = nullptr);
// Largest |value| of a node field (float bits, atomicMax) -- used for the
// interpolation halo.
void launch_absmax(const float *x, long long n, int stride, int offset, unsigned *out,
                   cudaStream_t st);
// s = exp(theta) elementwise.
void launch_exp(const float *theta, float *s, long long n, cudaStream_t st);
// Nodes of each of the m sub-domains (out[k] += |bit k|; out zeroed by the caller).
void launch_bitcount(const uint32_t *mask, long long n, int m, unsigned long long *out,
                     cudaStream_t st);
// Re-splitting of a target component (label value comp): index extents
// ext = {x min, x max, y min, y max} (initialised by the caller to
// {INT_MAX, -1, INT_MAX, -1}) and node count, the histogram of its nodes
// along a grid axis, and the relabelling of its nodes with index > s on
// that axis as new_comp.
void launch_comp_extent(const GridDims &g, const uint8_t *labels, int comp, int *ext,
                        unsigned *count_out, cudaStream_t st);
void launch_comp_hist(const GridDims &g, const uint8_t *labels, int comp, int axis, unsigned *hist,
                      cudaStream_t st);
void launch_comp_split(const GridDims &g, uint8_t *labels, int comp, int axis, int s, int new_comp,
                       cudaStream_t st);
// Count of bits per sub-domain (sum over k of |Sigma_k|) into *out.// Count of bits per sub-domain (sum over k of |Sigma_k|) into *out.
void launch_popcount(const uint32_t *mask, long long n, unsigned long long *out, cudaStream_t st);

// ----- adjoint (adjoint.cu) -------------------------------------------------

// Geometry and coefficients of a 2D speed/current problem for the adjoint.
struct AdjProblem {
    int nx, ny;
    float hx, hy;        // h / dx, h / dy
    double hd, dxd, dyd; // h, dx, dy in FP64 (the policy decision)
    double betad, gammad, lconst;  // step weights and constant cost in FP64
    const float *cost;   // running cost field l (or null: lconst)
    float dx, dy;
    float beta, gamma, h;
    float vout;          // value of feet outside the box (V form)
    const float *speed;  // s (or null)
    const float *current;
    const uint8_t *labels;
};

struct AdjCtl {
    unsigned done_ctas;
    unsigned res_bits;
    int iters;
    int parity;
    int converged;
    float final_res;
    float tol;
    int max_iters;
    int error;
    unsigned lam_bits;
    float lam_max;
    float best_res;
    int stall;
    int pad_[3];
};

// pi_i = argmin_j I[V](foot_j) (lowest index on ties), -1 on targets, -2
// when the minimising foot is outside the box (a zero row of P_pi).
void launch_policy(const AdjProblem &ap, const hjbk::ControlTable &C, const float *V,
                   const float *dV, float margin, int8_t *policy, unsigned *ties_out,
                   cudaStream_t st);
// The foot of every node's policy control in FP32 (cell index and fractions,
// see AdjArgs::cell), once per policy decision.
void launch_feet(const AdjProblem &ap, const hjbk::ControlTable &C, const int8_t *policy, int *cell,
                 float2 *frac, cudaStream_t st);
// Iterative refinement of the values the policy is decided on: r = the FP64
// residual (beta I[V](foot_pi) + gamma l) - V of the policy-frozen equation,
// then block Gauss-Seidel sweeps of dV <- r + beta P_pi dV (FP32) over staged
// tiles, one per launch of the refinement kernel (AdjArgs: g = r, L = the
// two dV buffers, hr the tiles' halo; shared memory refine_tiles_smem(hr)
// bytes, one CTA per tile: refine_tiles_grid).
void launch_refine_residual(const AdjProblem &ap, const hjbk::ControlTable &C, const float *V,
                            const int8_t *policy, float *r, cudaStream_t st);
const void *refine_tiles_kernel(int apps);
size_t refine_tiles_smem(int hr);
int refine_tiles_grid(int nx, int ny);
// One block Gauss-Seidel sweep of the transposed iteration over staged
// tiles (the refinement's tiles and grid; shared memory adj_tiles_smem(hr)
// bytes).
const void *adj_tiles_kernel(int apps);
size_t adj_tiles_smem(int hr);
struct AdjArgs {
    AdjProblem ap;
    hjbk::ControlTable ctrl;
    const int8_t *policy;
    const float *g;
    float *L[2];
    AdjCtl *ctl;
    int use_handle;
    cudaGraphConditionalHandle handle;
    // the foot of each node's policy control (launch_feet): corner cell
    // index (-1 target, -2 foot outside the box) and fractions (tx, ty)
    const int *cell;
    const float2 *frac;
    int hr;  // refinement tiles: halo in cells around each 32 x REFINE_ROWS tile
};
// Tiles of the adjoint's block Gauss-Seidel sweeps: 32 x REFINE_ROWS nodes;
// the applications per staged tile and sweep are a template parameter of
// the kernels (8, 16 or 32).
constexpr int REFINE_ROWS = 8;
void launch_adj_init(const float *g, float *L0, float *L1, long long n, AdjCtl *ctl, float tol,
                     int max_iters, cudaStream_t st);
// dL/dtheta (wrt = 0) or dL/dl (wrt = 1) from lambda.
void launch_adj_grad(const AdjProblem &ap, const hjbk::ControlTable &C, const float *V,
                     const int8_t *policy, const float *lam, int wrt, float *out, cudaStream_t st);
// Values of Q1 interpolation at points and (optionally) the gradient of
// their mean with respect to V (grad must be zeroed by the caller).
void launch_points(int nx, int ny, double lo0, double lo1, double dx0, double dx1,
                   const float *V, const float *pts, int P, float *vals, float *grad,
                   cudaStream_t st);

}  // namespace hjbh
