/*
 * hjb_oracle.c -- plain, slow, FP64 CPU oracle for semi-Lagrangian value
 * iteration and the independent sub-domain method of Festa,
 * "Reconstruction of independent sub-domains for a class of Hamilton Jacobi
 * equations and its application to parallel computing" (arXiv:1405.3521).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; it is written from the
 * paper's definitions, in the paper's order, with no blocking or fusion.
 *
 * Every function names the passage it follows.  Where the paper is
 * garbled or silent the reading used is stated beside the code:
 *   R1  operator form  [T(V)]_i = beta * min_a I[V](x_i + h f(x_i,a)) + gamma * l_i,
 *       beta = exp(-lambda h), gamma = (1 - beta)/lambda  (Sec. 3, eq. Tdef,
 *       with the sign convention of the dynamics y' = f of Sec. 2).
 *   R2  ghost value: a foot strictly outside the closed box (beyond 1e-6
 *       grid cells) takes the value v_out (the Kruzhkov image of the paper's
 *       +infinity on ghost nodes); feet within that tolerance are clamped
 *       onto the face.  Ghost NODES of a restricted problem carry v_out.
 *   R3  ISA step 3: the sub-problem on sub-domain k keeps every target node
 *       inside it as a target; nodes outside it are ghosts.
 *   R4  projection: Kuhn (Freudenthal) triangulation of each coarse cell; a
 *       fine node belongs to sub-domain k iff every vertex carrying a
 *       non-zero barycentric weight is labelled k.
 *   R10 ties in the control minimum go to the lowest control index.
 *   P1 (Sec. 3: linear interpolation in n dimensions; 2D, interp = 1): the
 *       linear interpolant on the triangle of the Kuhn split of the cell that
 *       holds the point; Q1 (multilinear) otherwise.  The adjoint functions
 *       assume Q1.
 *   Games (Sec. 2, max over b of min over a; Example ex4): with a second control set B
 *       the operator is beta * max_b min_a I[V](x_i + h f(x_i, a, b)) +
 *       gamma * l_i, f = D(x)(a - b) + c(x); D(x) = diag(scale) per node, or
 *       s(x) I, or I.
 *
 * Parity unpinned: none of the functions below is unpinned; the pins live in
 * tests/test_oracle_pins.py (brute force, BFS graph case, closed forms,
 * invariants, the restricted-solve property).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OHJB_FACE_TOL 1e-6 /* R2: grid-cell tolerance for "on the face" */

/* Problem statement of Sec. 2 discretised as in Sec. 3.  Arrays are node
 * fields in row-major order with x fastest; controls are [ncontrols][cdim]. */
typedef struct {
    int ndim;            /* 2 or 3 */
    int n[3];            /* nodes per dimension */
    double lo[3], hi[3]; /* box; a periodic dimension has period hi-lo */
    int periodic[3];
    int dyn;             /* 0: f = s(x) a + c(x);  1: Dubins f = (v cos th, v sin th, u) */
    const double *speed;   /* [N] or NULL (s = 1) */
    const double *current; /* [N][2] or NULL (c = 0) */
    double dubins_v;
    const double *cost;    /* [N] or NULL (l = cost_const) */
    double cost_const;
    double h;              /* fictitious time step */
    double lambda;         /* discount rate */
    int ncontrols, cdim;
    const double *controls;
    const int32_t *target; /* [N] 0 free, k >= 1 target component k */
    int ntargets;
    double v_out;          /* value of ghost nodes / feet outside the box */
    const double *scale;   /* [N][2] per-axis factors D(x) of f, or NULL (dyn 0) */
    int nb;                /* size of the second player's set B (0: none) */
    const double *controls_b; /* [nb][cdim] */
    int weights;           /* 0: beta = exp(-lambda h); 1: beta = 1/(1 + lambda h) */
    int interp;            /* 0: Q1 multilinear; 1: P1 on the Kuhn triangles (2D) */
} ohjb_problem;

static long long node_count(const ohjb_problem *p) {
    long long N = 1;
    for (int d = 0; d < p->ndim; ++d) N *= p->n[d];
    return N;
}

/* Grid spacing: n nodes on [lo,hi], or n nodes on a period (periodic). */
static double spacing(const ohjb_problem *p, int d) {
    return p->periodic[d] ? (p->hi[d] - p->lo[d]) / p->n[d]
                          : (p->hi[d] - p->lo[d]) / (p->n[d] - 1);
}

static void unflatten(const ohjb_problem *p, long long i, int idx[3]) {
    idx[0] = (int)(i % p->n[0]);
    long long r = i / p->n[0];
    idx[1] = (int)(r % p->n[1]);
    idx[2] = p->ndim > 2 ? (int)(r / p->n[1]) : 0;
}

static long long flatten(const ohjb_problem *p, const int idx[3]) {
    long long i = idx[0] + (long long)p->n[0] * idx[1];
    if (p->ndim > 2) i += (long long)p->n[0] * p->n[1] * idx[2];
    return i;
}

/* Q1 (multilinear) interpolation I[V] at grid coordinate g (Sec. 3, the
 * interpolation the scheme applies at the feet).  Non-periodic
 * coordinates must already lie in [0, n-1]; the cell is floor(g) clamped to
 * [0, n-2].  Periodic coordinates wrap modulo n.  If grad != NULL the
 * gradient with respect to the grid coordinates is written there. */
static double q1_at(const ohjb_problem *p, const double *V, const double *g,
                    double *grad) {
    int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
    double t[3] = {0, 0, 0};
    for (int d = 0; d < p->ndim; ++d) {
        int n = p->n[d];
        if (p->periodic[d]) {
            double gg = fmod(g[d], (double)n);
            if (gg < 0) gg += n;
            int c = (int)floor(gg);
            if (c >= n) c = n - 1;
            t[d] = gg - c;
            c0[d] = c;
            c1[d] = (c + 1) % n;
        } else {
            int c = (int)floor(g[d]);
            if (c < 0) c = 0;
            if (c > n - 2) c = n - 2;
            t[d] = g[d] - c;
            c0[d] = c;
            c1[d] = c + 1;
        }
    }
    if (p->interp == 1 && p->ndim == 2) {
        /* P1: the linear interpolant on the triangle of the Kuhn split of
         * the cell (diagonal from corner (0,0) to (1,1)) holding the point */
        double v00 = V[flatten(p, (int[3]){c0[0], c0[1], 0})];
        double v10 = V[flatten(p, (int[3]){c1[0], c0[1], 0})];
        double v01 = V[flatten(p, (int[3]){c0[0], c1[1], 0})];
        double v11 = V[flatten(p, (int[3]){c1[0], c1[1], 0})];
        double val;
        if (t[0] >= t[1]) {
            val = (1.0 - t[0]) * v00 + (t[0] - t[1]) * v10 + t[1] * v11;
            if (grad) {
                grad[0] = v10 - v00;
                grad[1] = v11 - v10;
            }
        } else {
            val = (1.0 - t[1]) * v00 + (t[1] - t[0]) * v01 + t[0] * v11;
            if (grad) {
                grad[0] = v11 - v01;
                grad[1] = v01 - v00;
            }
        }
        return val;
    }
    double acc = 0.0;
    double gacc[3] = {0, 0, 0};
    int corners = 1 << p->ndim;
    for (int m = 0; m < corners; ++m) {
        int idx[3] = {0, 0, 0};
        double w = 1.0;
        double dw[3] = {1, 1, 1};
        for (int d = 0; d < p->ndim; ++d) {
            int up = (m >> d) & 1;
            idx[d] = up ? c1[d] : c0[d];
            double wd = up ? t[d] : 1.0 - t[d];
            double dd = up ? 1.0 : -1.0;
            for (int e = 0; e < p->ndim; ++e) dw[e] *= (e == d) ? dd : wd;
            w *= wd;
        }
        double v = V[flatten(p, idx)];
        acc += w * v;
        for (int e = 0; e < p->ndim; ++e) gacc[e] += dw[e] * v;
    }
    if (grad)
        for (int e = 0; e < p->ndim; ++e) grad[e] = gacc[e];
    return acc;
}

/* Interpolate at a physical point y (clamped into the box). */
double ohjb_interp(const ohjb_problem *p, const double *V, const double *y) {
    double g[3] = {0, 0, 0};
    for (int d = 0; d < p->ndim; ++d) {
        g[d] = (y[d] - p->lo[d]) / spacing(p, d);
        if (!p->periodic[d]) {
            if (g[d] < 0) g[d] = 0;
            if (g[d] > p->n[d] - 1) g[d] = p->n[d] - 1;
        }
    }
    return q1_at(p, V, g, NULL);
}

/* Dynamics f(x_i, a_j) of Sec. 2 for the two families; with a second
 * player (k >= 0) the control enters as a_j - b_k (Example ex4). */
static void dynamics(const ohjb_problem *p, long long i, const int idx[3], int j, int k,
                     double f[3]) {
    const double *a = p->controls + (long long)j * p->cdim;
    if (p->dyn == 0) {
        double ux = a[0], uy = a[1];
        if (k >= 0) {
            const double *b = p->controls_b + (long long)k * p->cdim;
            ux -= b[0];
            uy -= b[1];
        }
        double sx = 1.0, sy = 1.0;
        if (p->scale) {
            sx = p->scale[2 * i];
            sy = p->scale[2 * i + 1];
        } else if (p->speed) {
            sx = sy = p->speed[i];
        }
        double cx = p->current ? p->current[2 * i] : 0.0;
        double cy = p->current ? p->current[2 * i + 1] : 0.0;
        f[0] = sx * ux + cx;
        f[1] = sy * uy + cy;
        f[2] = 0.0;
    } else {
        double th = p->lo[2] + idx[2] * spacing(p, 2);
        f[0] = p->dubins_v * cos(th);
        f[1] = p->dubins_v * sin(th);
        f[2] = a[0];
    }
}

/* Foot of the characteristic y = x_i + h f(x_i, a_j[, b_k]) in grid
 * coordinates.  Returns 0 when the foot is strictly outside the closed box
 * (reading R2). */
static int foot_game(const ohjb_problem *p, long long i, const int idx[3], int j, int k,
                     double g[3], double off[3]) {
    double f[3];
    dynamics(p, i, idx, j, k, f);
    int inside = 1;
    for (int d = 0; d < p->ndim; ++d) {
        double o = p->h * f[d] / spacing(p, d);
        off[d] = o;
        g[d] = idx[d] + o;
        if (!p->periodic[d]) {
            if (o < -(double)idx[d] - OHJB_FACE_TOL ||
                o > (double)(p->n[d] - 1 - idx[d]) + OHJB_FACE_TOL)
                inside = 0;
            if (g[d] < 0) g[d] = 0;
            if (g[d] > p->n[d] - 1) g[d] = p->n[d] - 1;
        }
    }
    return inside;
}

static int foot(const ohjb_problem *p, long long i, const int idx[3], int j, double g[3],
                double off[3]) {
    return foot_game(p, i, idx, j, -1, g, off);
}

/* Node classes of Sec. 3: ghost (Phi), boundary/target (dG), interior (G).
 * mask/bit select a restricted problem (ISA step 3, reading R3);
 * only_target = k keeps only target component k (RA step 1: dG := X_k). */
enum { NODE_FREE = 0, NODE_TARGET = 1, NODE_GHOST = 2 };
static int node_class(const ohjb_problem *p, long long i, const uint32_t *mask,
                      int bit, int only_target) {
    if (mask && !((mask[i] >> bit) & 1u)) return NODE_GHOST;
    int32_t lab = p->target[i];
    if (lab != 0 && (only_target == 0 || lab == only_target)) return NODE_TARGET;
    return NODE_FREE;
}

/* Step weights (R1): beta = e^{-lambda h}, gamma = (1 - beta) / lambda; or
 * the weights printed in the scheme of Sec. 3, beta = 1/(1 + lambda h) and
 * gamma = h/(1 + lambda h). */
static double beta_of(const ohjb_problem *p) {
    if (p->weights == 1) return 1.0 / (1.0 + p->lambda * p->h);
    return exp(-p->lambda * p->h);
}
static double gamma_of(const ohjb_problem *p) {
    if (p->weights == 1) return p->h / (1.0 + p->lambda * p->h);
    return (1.0 - exp(-p->lambda * p->h)) / p->lambda;
}

/* One application of the operator T of Sec. 3, eq. (Tdef), under readings
 * R1-R3, at one node.  Writes the minimising control index (R10). */
static double apply_node(const ohjb_problem *p, const double *V, long long i,
                         const uint32_t *mask, int bit, int only_target,
                         int32_t *arg) {
    int cls = node_class(p, i, mask, bit, only_target);
    if (arg) *arg = -1;
    if (cls == NODE_GHOST) return p->v_out;
    if (cls == NODE_TARGET) return 0.0; /* g = 0 on the target */
    int idx[3];
    unflatten(p, i, idx);
    double best = INFINITY;
    int32_t barg = -1;
    if (p->nb > 0) {
        /* max over the second player's b of the min over a (Example ex4);
         * arg: the minimising a under the maximising b */
        best = -INFINITY;
        for (int k = 0; k < p->nb; ++k) {
            double inner = INFINITY;
            int32_t ja = -1;
            for (int j = 0; j < p->ncontrols; ++j) {
                double g[3], off[3];
                double q = foot_game(p, i, idx, j, k, g, off) ? q1_at(p, V, g, NULL) : p->v_out;
                if (q < inner) {
                    inner = q;
                    ja = j;
                }
            }
            if (inner > best) {
                best = inner;
                barg = ja;
            }
        }
        if (arg) *arg = barg;
        double l = p->cost ? p->cost[i] : p->cost_const;
        return beta_of(p) * best + gamma_of(p) * l;
    }
    for (int j = 0; j < p->ncontrols; ++j) {
        double g[3], off[3];
        double q = foot(p, i, idx, j, g, off) ? q1_at(p, V, g, NULL) : p->v_out;
        if (q < best) {
            best = q;
            barg = j;
        }
    }
    if (arg) *arg = barg;
    double l = p->cost ? p->cost[i] : p->cost_const;
    return beta_of(p) * best + gamma_of(p) * l;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* One Jacobi application Vn = T(V) over all nodes; returns ||Vn - V||_inf
 * (the quantity of the stopping Remark of Sec. 3). */
double ohjb_apply(const ohjb_problem *p, const double *V, double *Vn,
                  int32_t *policy, const uint32_t *mask, int bit,
                  int only_target, int nthreads) {
    long long N = node_count(p);
    double r = 0.0;
    set_threads(nthreads);
#pragma omp parallel for schedule(static) reduction(max : r)
    for (long long i = 0; i < N; ++i) {
        int32_t a;
        double v = apply_node(p, V, i, mask, bit, only_target, &a);
        Vn[i] = v;
        if (policy) policy[i] = a;
        double dv = fabs(v - V[i]);
        if (dv > r) r = dv;
    }
    return r;
}

/* Starting point of the iteration: v_out on free and ghost nodes, 0 on the
 * target -- a supersolution, so the iteration decreases monotonically. */
void ohjb_initial(const ohjb_problem *p, double *V, const uint32_t *mask, int bit,
                  int only_target) {
    long long N = node_count(p);
    for (long long i = 0; i < N; ++i)
        V[i] = node_class(p, i, mask, bit, only_target) == NODE_TARGET ? 0.0
                                                                        : p->v_out;
}

/* Value iteration V^{n+1} = T(V^n) (Sec. 3) until ||V^{n+1}-V^n||_inf <= tol.
 * V holds the start on entry (see ohjb_initial) and the result on exit.
 * Returns the number of applications of T. */
int ohjb_solve(const ohjb_problem *p, double tol, int max_iters, double *V,
               const uint32_t *mask, int bit, int only_target, int nthreads,
               double *final_res) {
    long long N = node_count(p);
    double *W = (double *)malloc(sizeof(double) * N);
    if (!W) return -1;
    double r = INFINITY;
    int it = 0;
    while (it < max_iters) {
        r = ohjb_apply(p, V, W, NULL, mask, bit, only_target, nthreads);
        ++it;
        memcpy(V, W, sizeof(double) * N);
        if (r <= tol) break;
    }
    free(W);
    if (final_res) *final_res = r;
    return it;
}

/* Gauss-Seidel variant with alternating orderings: the same operator and the
 * same unique fixed point (T is a contraction), used only to reach tight
 * tolerances quickly on large reference grids.  Stops when one strict Jacobi
 * application changes V by at most tol. */
int ohjb_solve_gs(const ohjb_problem *p, double tol, int max_sweeps, double *V,
                  const uint32_t *mask, int bit, int only_target,
                  double *final_res) {
    long long N = node_count(p);
    double *W = (double *)malloc(sizeof(double) * N);
    if (!W) return -1;
    int sweeps = 0;
    double r = INFINITY;
    int nord = 1 << p->ndim;
    while (sweeps < max_sweeps) {
        int ord = sweeps % nord;
        double ch = 0.0;
        int nz = p->ndim > 2 ? p->n[2] : 1;
        for (int zz = 0; zz < nz; ++zz)
            for (int yy = 0; yy < p->n[1]; ++yy)
                for (int xx = 0; xx < p->n[0]; ++xx) {
                    int idx[3];
                    idx[0] = (ord & 1) ? p->n[0] - 1 - xx : xx;
                    idx[1] = (ord & 2) ? p->n[1] - 1 - yy : yy;
                    idx[2] = (ord & 4) ? nz - 1 - zz : zz;
                    long long i = flatten(p, idx);
                    double v = apply_node(p, V, i, mask, bit, only_target, NULL);
                    double dv = fabs(v - V[i]);
                    if (dv > ch) ch = dv;
                    V[i] = v;
                }
        ++sweeps;
        if (ch <= tol) {
            r = ohjb_apply(p, V, W, NULL, mask, bit, only_target, 1);
            if (r <= tol) break;
        }
    }
    free(W);
    if (final_res) *final_res = r;
    return sweeps;
}

/* ---------------------------------------------------------------------- */
/* RA: reconstruction algorithm (Sec. 3, algorithm "RA", steps 1-3).       */

/* Coarse grid K: every stride-th fine node (the superimposed grids of the
 * projection remark in Sec. 4).  Builds the coarse problem in *q, with
 * freshly allocated field arrays owned by the caller (ohjb_free_coarse). */
static int make_coarse(const ohjb_problem *p, const int stride[3], double h_coarse,
                       ohjb_problem *q) {
    *q = *p;
    for (int d = 0; d < p->ndim; ++d) {
        int r = stride[d];
        if (r < 1) return -1;
        if (p->periodic[d]) {
            if (p->n[d] % r) return -1;
            q->n[d] = p->n[d] / r;
        } else {
            if ((p->n[d] - 1) % r) return -1;
            q->n[d] = (p->n[d] - 1) / r + 1;
        }
    }
    q->h = h_coarse;
    long long NK = node_count(q);
    double *sp = p->speed ? (double *)malloc(sizeof(double) * NK) : NULL;
    double *cu = p->current ? (double *)malloc(sizeof(double) * 2 * NK) : NULL;
    double *co = p->cost ? (double *)malloc(sizeof(double) * NK) : NULL;
    double *sc = p->scale ? (double *)malloc(sizeof(double) * 2 * NK) : NULL;
    int32_t *ta = (int32_t *)malloc(sizeof(int32_t) * NK);
    for (long long k = 0; k < NK; ++k) {
        int ik[3], ifn[3] = {0, 0, 0};
        unflatten(q, k, ik);
        for (int d = 0; d < p->ndim; ++d) ifn[d] = ik[d] * stride[d];
        long long i = flatten(p, ifn);
        if (sp) sp[k] = p->speed[i];
        if (cu) {
            cu[2 * k] = p->current[2 * i];
            cu[2 * k + 1] = p->current[2 * i + 1];
        }
        if (co) co[k] = p->cost[i];
        if (sc) {
            sc[2 * k] = p->scale[2 * i];
            sc[2 * k + 1] = p->scale[2 * i + 1];
        }
        ta[k] = p->target[i];
    }
    q->speed = sp;
    q->current = cu;
    q->cost = co;
    q->scale = sc;
    q->target = ta;
    return 0;
}

static void free_coarse(ohjb_problem *q) {
    free((void *)q->speed);
    free((void *)q->current);
    free((void *)q->cost);
    free((void *)q->scale);
    free((void *)q->target);
}

/* Coarse grid sizes for a stride (for the Python side to size buffers). */
int ohjb_coarse_shape(const ohjb_problem *p, const int stride[3], int nK[3]) {
    ohjb_problem q;
    if (make_coarse(p, stride, p->h, &q)) return -1;
    for (int d = 0; d < 3; ++d) nK[d] = d < p->ndim ? q.n[d] : 1;
    free_coarse(&q);
    return 0;
}

/* RA steps 2-3 on given auxiliary solutions Vaux[m][NK]:
 * V = min_k V_k;  bit (k-1) of labels[j] set iff j in X_k or
 * |V_k(j) - V(j)| <= delta (eq. rep of Prop. 3.1).  Counts the (j,k) pairs
 * whose deciding quantity lies within tie_eps of the threshold (R10). */
long long ohjb_label(long long NK, int m, const double *Vaux, const int32_t *target,
                     double delta, double tie_eps, double *Vmin, uint32_t *labels) {
    long long ties = 0;
    for (long long j = 0; j < NK; ++j) {
        double v = INFINITY;
        for (int k = 0; k < m; ++k)
            if (Vaux[(long long)k * NK + j] < v) v = Vaux[(long long)k * NK + j];
        if (Vmin) Vmin[j] = v;
        uint32_t bits = 0;
        for (int k = 0; k < m; ++k) {
            double diff = fabs(Vaux[(long long)k * NK + j] - v);
            if (target[j] == k + 1 || diff <= delta) bits |= 1u << k;
            if (fabs(diff - delta) <= tie_eps) ++ties;
        }
        labels[j] = bits;
    }
    return ties;
}

/* Threshold of RA step 3 (eq. rep of Prop. 3.1): delta = 2 (C dx^q + M dx)
 * on the coarse grid K of the given stride, dx = dx_K the spacing of its
 * first dimension.  M is the Lipschitz constant of the value function
 * (hypothesis lip); M < 0 selects the estimate of reading R5, the largest
 * norm over the nodes of K of the discrete gradient of V = min_k V_k:
 * per dimension the centred difference (V(j + e_d) - V(j - e_d)) / (2 dx_d),
 * one-sided (V(j + e_d) - V(j)) / dx_d or (V(j) - V(j - e_d)) / dx_d on the
 * first and last node of a non-periodic dimension, wrapping on a periodic
 * one.  Vaux is [m][NK] as returned by RA step 1; M_out (optional) receives
 * the M used.  Returns delta, or -1 when the stride does not fit the grid. */
double ohjb_delta(const ohjb_problem *p, const int stride[3], const double *Vaux, double C,
                  double q, double M, double *M_out) {
    ohjb_problem K;
    if (make_coarse(p, stride, p->h, &K)) return -1.0;
    long long NK = node_count(&K);
    int m = p->ntargets;
    if (M < 0.0) {
        double *V = (double *)malloc(sizeof(double) * NK);
        for (long long j = 0; j < NK; ++j) {
            V[j] = INFINITY;
            for (int k = 0; k < m; ++k)
                if (Vaux[(long long)k * NK + j] < V[j]) V[j] = Vaux[(long long)k * NK + j];
        }
        M = 0.0;
        for (long long j = 0; j < NK; ++j) {
            int idx[3];
            unflatten(&K, j, idx);
            double norm2 = 0.0;
            for (int d = 0; d < K.ndim; ++d) {
                int lo[3] = {idx[0], idx[1], idx[2]}, hi[3] = {idx[0], idx[1], idx[2]};
                double span = 2.0 * spacing(&K, d);
                if (K.periodic[d]) {
                    lo[d] = (idx[d] + K.n[d] - 1) % K.n[d];
                    hi[d] = (idx[d] + 1) % K.n[d];
                } else if (idx[d] == 0) {
                    hi[d] = 1;
                    span = spacing(&K, d);
                } else if (idx[d] == K.n[d] - 1) {
                    lo[d] = K.n[d] - 2;
                    span = spacing(&K, d);
                } else {
                    lo[d] = idx[d] - 1;
                    hi[d] = idx[d] + 1;
                }
                double g = (V[flatten(&K, hi)] - V[flatten(&K, lo)]) / span;
                norm2 += g * g;
            }
            if (sqrt(norm2) > M) M = sqrt(norm2);
        }
        free(V);
    }
    if (M_out) *M_out = M;
    double dx = spacing(&K, 0);
    double delta = 2.0 * ((C > 0.0 ? C * pow(dx, q) : 0.0) + M * dx);
    free_coarse(&K);
    return delta;
}

/* RA (all three steps) on the coarse grid of the given stride.
 * Step 1 solves the m auxiliary problems V_k = T_k(V_k) whose target is
 * component k only (dG := X_k); Vaux receives them as [m][NK].  labels
 * receives the coarse bitmasks.  Returns the number of ties (R10), or -1. */
long long ohjb_ra(const ohjb_problem *p, const int stride[3], double h_coarse,
                  double delta, double tol, int max_iters, double *Vaux,
                  uint32_t *labels, int nthreads) {
    ohjb_problem q;
    if (make_coarse(p, stride, h_coarse, &q)) return -1;
    long long NK = node_count(&q);
    int m = p->ntargets;
    for (int k = 1; k <= m; ++k) {
        double *Vk = Vaux + (long long)(k - 1) * NK;
        ohjb_initial(&q, Vk, NULL, 0, k);
        ohjb_solve(&q, tol, max_iters, Vk, NULL, 0, k, nthreads, NULL);
    }
    long long ties = ohjb_label(NK, m, Vaux, q.target, delta, 1e-6, NULL, labels);
    free_coarse(&q);
    return ties;
}

/* ---------------------------------------------------------------------- */
/* ISA step 2: projection of coarse labels onto the fine grid through the  */
/* concave hull Con (Sec. 4, second observation after the algorithm),      */
/* reading R4 (Kuhn triangulation, integer local coordinates).            */

void ohjb_project(const ohjb_problem *p, const int stride[3], const uint32_t *coarse,
                  uint32_t *fine) {
    int nK[3] = {1, 1, 1};
    for (int d = 0; d < p->ndim; ++d)
        nK[d] = p->periodic[d] ? p->n[d] / stride[d] : (p->n[d] - 1) / stride[d] + 1;
    long long N = node_count(p);
    for (long long i = 0; i < N; ++i) {
        int idx[3];
        unflatten(p, i, idx);
        int cell[3] = {0, 0, 0}, loc[3] = {0, 0, 0};
        for (int d = 0; d < p->ndim; ++d) {
            int c = idx[d] / stride[d];
            if (!p->periodic[d] && c > nK[d] - 2) c = nK[d] - 2;
            cell[d] = c;
            loc[d] = idx[d] - c * stride[d]; /* 0..stride */
        }
        /* Kuhn simplex: order the dimensions by decreasing local coordinate
         * t_d = loc_d / stride_d (compared exactly by cross-multiplication).
         * The vertices are v_0 = cell origin, v_k = v_{k-1} + e_{sigma(k)}.
         * Barycentric weights: 1 - t_s1, t_s1 - t_s2, ..., t_sD. */
        int ord[3] = {0, 1, 2};
        for (int a = 0; a < p->ndim; ++a)
            for (int b = a + 1; b < p->ndim; ++b) {
                long long ta = (long long)loc[ord[a]] * stride[ord[b]];
                long long tb = (long long)loc[ord[b]] * stride[ord[a]];
                if (tb > ta) {
                    int t = ord[a];
                    ord[a] = ord[b];
                    ord[b] = t;
                }
            }
        uint32_t acc = 0xffffffffu;
        int vtx[3] = {cell[0], cell[1], cell[2]};
        for (int k = 0; k <= p->ndim; ++k) {
            /* weight of vertex k is non-zero iff t_{s_k} > t_{s_{k+1}}
             * (with t_{s_0} := 1 and t_{s_{D+1}} := 0) */
            long long num_hi, den_hi, num_lo, den_lo;
            if (k == 0) {
                num_hi = 1;
                den_hi = 1;
            } else {
                num_hi = loc[ord[k - 1]];
                den_hi = stride[ord[k - 1]];
            }
            if (k == p->ndim) {
                num_lo = 0;
                den_lo = 1;
            } else {
                num_lo = loc[ord[k]];
                den_lo = stride[ord[k]];
            }
            int nonzero = num_hi * den_lo > num_lo * den_hi;
            if (k > 0) vtx[ord[k - 1]] += 1;
            if (nonzero) {
                int w[3] = {0, 0, 0};
                for (int d = 0; d < p->ndim; ++d)
                    w[d] = p->periodic[d] ? vtx[d] % nK[d] : vtx[d];
                long long ci = w[0] + (long long)nK[0] * w[1];
                if (p->ndim > 2) ci += (long long)nK[0] * nK[1] * w[2];
                acc &= coarse[ci];
            }
        }
        fine[i] = acc;
    }
}

/* ISA steps 3-4 (Sec. 4): restricted solves on every sub-domain given by
 * fine_mask, then Vbar(j) = min{ V_k(j) : j in Sigma_k }.  The targets of
 * sub-problem k are every target node inside it (own_targets = 0: the
 * operator of Sec. 4 step 3 as written, reading R3), or only component k
 * (own_targets = 1: the target choice of RA step 1, dG := X_k, in Sec. 3).
 * Vk (optional) receives [m][N].  Returns the number of uncovered nodes
 * (nodes in no sub-domain; they receive v_out). */
long long ohjb_isa(const ohjb_problem *p, const uint32_t *fine_mask, double tol,
                   int max_iters, int use_gs, double *Vk, double *Vbar,
                   int *iters, int nthreads, int own_targets) {
    long long N = node_count(p);
    int m = p->ntargets;
    double *tmp = (double *)malloc(sizeof(double) * N);
    for (long long i = 0; i < N; ++i) Vbar[i] = INFINITY;
    for (int k = 0; k < m; ++k) {
        const int only = own_targets ? k + 1 : 0;
        ohjb_initial(p, tmp, fine_mask, k, only);
        int it;
        if (use_gs)
            it = ohjb_solve_gs(p, tol, max_iters, tmp, fine_mask, k, only, NULL);
        else
            it = ohjb_solve(p, tol, max_iters, tmp, fine_mask, k, only, nthreads, NULL);
        if (iters) iters[k] = it;
        if (Vk) memcpy(Vk + (long long)k * N, tmp, sizeof(double) * N);
        for (long long i = 0; i < N; ++i)
            if (((fine_mask[i] >> k) & 1u) && tmp[i] < Vbar[i]) Vbar[i] = tmp[i];
    }
    long long unc = 0;
    for (long long i = 0; i < N; ++i)
        if (Vbar[i] == INFINITY) {
            Vbar[i] = p->v_out;
            ++unc;
        }
    free(tmp);
    return unc;
}

/* ---------------------------------------------------------------------- */
/* Recursive re-splitting of the target components (Conclusions: the       */
/* unbalanced sub-domains of Example ex3 can be balanced by refining the   */
/* division of Gamma recursively, in a few steps).  Reading R22: each step */
/* splits the component whose projected sub-domain is largest (the lowest  */
/* index on ties) in two, along the x or y grid axis with the larger index */
/* extent of its fine target nodes (x on ties): the nodes whose index on   */
/* that axis is at most s keep the component, the others form a new one,  */
/* with s the smallest index holding at least half of the nodes (the next  */
/* lower occupied index when that would leave the second part empty).  RA  */
/* and the projection are re-run on the new division with the same        */
/* threshold (V = min_k V_k, and hence the estimated M, does not change    */
/* with the division); the step is kept only when the sub-domains of both  */
/* parts are smaller than (1 - min_gain) times the split one's, and the    */
/* refinement stops at the first step that is not (the largest sub-domain  */
/* no longer shrinks by splitting its component), after max_splits steps,  */
/* at 32 components, or when the chosen component cannot be split (a       */
/* single index on the axis).                                              */

/* RA steps 1-3 and the projection for the division `comp` into m
 * components; returns the largest sub-domain (nodes), sizes[k] its nodes. */
static long long ra_division(const ohjb_problem *p, const int32_t *comp, int m, const int stride[3],
                             double h_coarse, double delta, double tol, int max_iters,
                             int nthreads, uint32_t *fine, long long *sizes) {
    ohjb_problem q = *p;
    q.target = comp;
    q.ntargets = m;
    int nK[3];
    if (ohjb_coarse_shape(&q, stride, nK)) return -1;
    long long NK = (long long)nK[0] * nK[1] * (p->ndim > 2 ? nK[2] : 1);
    double *Vaux = (double *)malloc(sizeof(double) * m * NK);
    uint32_t *cl = (uint32_t *)malloc(sizeof(uint32_t) * NK);
    ohjb_ra(&q, stride, h_coarse, delta, tol, max_iters, Vaux, cl, nthreads);
    ohjb_project(&q, stride, cl, fine);
    long long N = node_count(p), largest = 0;
    for (int k = 0; k < m; ++k) {
        sizes[k] = 0;
        for (long long i = 0; i < N; ++i) sizes[k] += (fine[i] >> k) & 1u;
        if (sizes[k] > largest) largest = sizes[k];
    }
    free(Vaux);
    free(cl);
    return largest;
}

/* Split component k (1-based id k + 1) into k and m + 1; returns 0 when it
 * cannot be split. */
static int split_component(const ohjb_problem *p, int32_t *comp, int k, int m) {
    long long N = node_count(p);
    int lo[2] = {p->n[0], p->n[1]}, hi[2] = {-1, -1};
    long long cnt = 0;
    for (long long i = 0; i < N; ++i) {
        if (comp[i] != k + 1) continue;
        int idx[3];
        unflatten(p, i, idx);
        for (int d = 0; d < 2; ++d) {
            if (idx[d] < lo[d]) lo[d] = idx[d];
            if (idx[d] > hi[d]) hi[d] = idx[d];
        }
        ++cnt;
    }
    if (cnt < 2) return 0;
    int axis = (hi[0] - lo[0]) >= (hi[1] - lo[1]) ? 0 : 1;
    int n = p->n[axis];
    long long *hist = (long long *)calloc(n, sizeof(long long));
    for (long long i = 0; i < N; ++i) {
        if (comp[i] != k + 1) continue;
        int idx[3];
        unflatten(p, i, idx);
        hist[idx[axis]] += 1;
    }
    long long half = (cnt + 1) / 2, cum = 0;
    int s = -1;
    for (int j = 0; j < n; ++j) {
        cum += hist[j];
        if (cum >= half) {
            s = j;
            break;
        }
    }
    if (cum == cnt) { /* everything at or below s: use the next lower occupied index */
        int t = s - 1;
        while (t >= 0 && hist[t] == 0) --t;
        s = t;
    }
    free(hist);
    if (s < 0) return 0;
    for (long long i = 0; i < N; ++i) {
        if (comp[i] != k + 1) continue;
        int idx[3];
        unflatten(p, i, idx);
        if (idx[axis] > s) comp[i] = m + 1;
    }
    return 1;
}

/* Recursive re-splitting; comp_out [N] receives the final division, fine
 * [N] its projected sub-domains, *m_out its number of components; returns
 * the largest sub-domain (nodes), or -1 on a bad stride. */
long long ohjb_ra_split(const ohjb_problem *p, const int stride[3], double h_coarse,
                        double delta, double tol, int max_iters, int max_splits, double min_gain,
                        int nthreads, int32_t *comp_out, uint32_t *fine, int *m_out) {
    long long N = node_count(p);
    int m = p->ntargets;
    long long sizes[32];
    memcpy(comp_out, p->target, sizeof(int32_t) * N);
    long long largest = ra_division(p, comp_out, m, stride, h_coarse, delta, tol, max_iters,
                                    nthreads, fine, sizes);
    if (largest < 0) return -1;
    int32_t *trial = (int32_t *)malloc(sizeof(int32_t) * N);
    uint32_t *tfine = (uint32_t *)malloc(sizeof(uint32_t) * N);
    long long tsizes[32];
    for (int step = 0; step < max_splits && m < 32; ++step) {
        int k = 0;
        for (int j = 1; j < m; ++j)
            if (sizes[j] > sizes[k]) k = j;
        memcpy(trial, comp_out, sizeof(int32_t) * N);
        if (!split_component(p, trial, k, m)) break;
        long long tl = ra_division(p, trial, m + 1, stride, h_coarse, delta, tol, max_iters,
                                   nthreads, tfine, tsizes);
        double lim = (1.0 - min_gain) * (double)sizes[k];
        if ((double)tsizes[k] > lim || (double)tsizes[m] > lim) break;
        memcpy(comp_out, trial, sizeof(int32_t) * N);
        memcpy(fine, tfine, sizeof(uint32_t) * N);
        memcpy(sizes, tsizes, sizeof tsizes);
        largest = tl;
        ++m;
    }
    free(trial);
    free(tfine);
    *m_out = m;
    return largest;
}

/* ---------------------------------------------------------------------- */
/* Adjoint of the converged fixed point with the optimal policy frozen.    */
/* (The paper has no adjoint; this is the plain linear algebra of          */
/* V = beta P_pi V + b: the transposed system (I - beta P_pi)^T lam = g.)  */

/* Q1 weights of the foot of node i under control j: up to 2^ndim corner
 * indices and weights; returns 0 when the foot is outside (row of zeros). */
static int row_weights(const ohjb_problem *p, long long i, int j, long long *cidx,
                       double *cw, double *gradw_dir, const double *V) {
    int idx[3];
    unflatten(p, i, idx);
    double g[3], off[3];
    if (!foot(p, i, idx, j, g, off)) return 0;
    int c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
    double t[3] = {0, 0, 0};
    for (int d = 0; d < p->ndim; ++d) {
        int n = p->n[d];
        if (p->periodic[d]) {
            double gg = fmod(g[d], (double)n);
            if (gg < 0) gg += n;
            int c = (int)floor(gg);
            if (c >= n) c = n - 1;
            t[d] = gg - c;
            c0[d] = c;
            c1[d] = (c + 1) % n;
        } else {
            int c = (int)floor(g[d]);
            if (c < 0) c = 0;
            if (c > n - 2) c = n - 2;
            t[d] = g[d] - c;
            c0[d] = c;
            c1[d] = c + 1;
        }
    }
    int corners = 1 << p->ndim;
    for (int m = 0; m < corners; ++m) {
        int id[3] = {0, 0, 0};
        double w = 1.0;
        for (int d = 0; d < p->ndim; ++d) {
            int up = (m >> d) & 1;
            id[d] = up ? c1[d] : c0[d];
            w *= up ? t[d] : 1.0 - t[d];
        }
        cidx[m] = flatten(p, id);
        cw[m] = w;
    }
    if (gradw_dir) { /* grid-coordinate gradient of I[V] at the foot */
        double gr[3];
        q1_at(p, V, g, gr);
        for (int d = 0; d < p->ndim; ++d) gradw_dir[d] = gr[d];
    }
    return corners;
}

/* Optimal policy pi_i = argmin_j Q_j (lowest index on ties, R10); -1 on
 * targets.  Returns ||T(V) - V||_inf. */
double ohjb_policy(const ohjb_problem *p, const double *V, int32_t *policy,
                   int nthreads) {
    long long N = node_count(p);
    double *W = (double *)malloc(sizeof(double) * N);
    double r = ohjb_apply(p, V, W, policy, NULL, 0, 0, nthreads);
    free(W);
    return r;
}

/* lam = g + beta P_pi^T lam, Jacobi iteration until ||dlam||_inf <= tol.
 * Rows of target nodes and rows whose foot is outside the box are zero. */
int ohjb_adjoint(const ohjb_problem *p, const int32_t *policy, const double *g,
                 double tol, int max_iters, double *lam, double *final_res) {
    long long N = node_count(p);
    double beta = beta_of(p);
    double *nx = (double *)malloc(sizeof(double) * N);
    memcpy(lam, g, sizeof(double) * N);
    int it = 0;
    double r = INFINITY;
    while (it < max_iters) {
        memcpy(nx, g, sizeof(double) * N);
        for (long long i = 0; i < N; ++i) {
            if (policy[i] < 0 || p->target[i] != 0) continue;
            long long ci[8];
            double cw[8];
            int nc = row_weights(p, i, policy[i], ci, cw, NULL, NULL);
            for (int m = 0; m < nc; ++m) nx[ci[m]] += beta * cw[m] * lam[i];
        }
        r = 0.0;
        for (long long i = 0; i < N; ++i) {
            double d = fabs(nx[i] - lam[i]);
            if (d > r) r = d;
        }
        memcpy(lam, nx, sizeof(double) * N);
        ++it;
        if (r <= tol) break;
    }
    free(nx);
    if (final_res) *final_res = r;
    return it;
}

/* dL/dtheta_i for s = exp(theta), f = s a + c:
 *   lam_i * beta * h * s_i * (grad_y I[V](y_i) . a_pi(i)),
 * and dL/dl_i = lam_i * gamma.  Zero on targets and for outside feet (theta)
 * and on targets (cost). */
void ohjb_grad(const ohjb_problem *p, const double *V, const int32_t *policy,
               const double *lam, double *grad_theta, double *grad_cost) {
    long long N = node_count(p);
    double beta = beta_of(p), gam = gamma_of(p);
    for (long long i = 0; i < N; ++i) {
        if (grad_theta) grad_theta[i] = 0.0;
        if (grad_cost) grad_cost[i] = 0.0;
        if (policy[i] < 0 || p->target[i] != 0) continue;
        if (grad_cost) grad_cost[i] = lam[i] * gam;
        if (!grad_theta || p->dyn != 0) continue;
        long long ci[8];
        double cw[8], gr[3];
        int nc = row_weights(p, i, policy[i], ci, cw, gr, V);
        if (!nc) continue;
        const double *a = p->controls + (long long)policy[i] * p->cdim;
        double s = p->speed ? p->speed[i] : 1.0;
        double dot = 0.0;
        for (int d = 0; d < 2; ++d) dot += gr[d] / spacing(p, d) * a[d];
        grad_theta[i] = lam[i] * beta * p->h * s * dot;
    }
}

/* Loss L = (1/P) sum_p I[V](pts_p): values at the points, and the gradient
 * g = dL/dV (the Q1 weights divided by P, accumulated per node). */
void ohjb_points(const ohjb_problem *p, const double *V, const double *pts, int P,
                 double *vals, double *g) {
    long long N = node_count(p);
    if (g)
        for (long long i = 0; i < N; ++i) g[i] = 0.0;
    for (int k = 0; k < P; ++k) {
        const double *y = pts + (long long)k * p->ndim;
        if (vals) vals[k] = ohjb_interp(p, V, y);
        if (!g) continue;
        double gg[3];
        int c0[3] = {0, 0, 0};
        double t[3] = {0, 0, 0};
        for (int d = 0; d < p->ndim; ++d) {
            gg[d] = (y[d] - p->lo[d]) / spacing(p, d);
            if (gg[d] < 0) gg[d] = 0;
            if (gg[d] > p->n[d] - 1) gg[d] = p->n[d] - 1;
            int c = (int)floor(gg[d]);
            if (c > p->n[d] - 2) c = p->n[d] - 2;
            c0[d] = c;
            t[d] = gg[d] - c;
        }
        for (int m = 0; m < (1 << p->ndim); ++m) {
            int id[3] = {0, 0, 0};
            double w = 1.0;
            for (int d = 0; d < p->ndim; ++d) {
                int up = (m >> d) & 1;
                id[d] = c0[d] + up;
                w *= up ? t[d] : 1.0 - t[d];
            }
            g[flatten(p, id)] += w / P;
        }
    }
}

/* Nodes whose adjoint or gradient is not unique (R10): the policy at a node
 * is not determined when its two smallest control values I[V](foot) differ by
 * at most eps, and the gradient of the Q1 interpolant is one-sided when the
 * foot of the chosen control lies within face_eps cells of a cell face.
 * lambda flows from a node to the corners of its foot (the transposed system
 * (I - beta P_pi)^T lam = g), so with closure != 0 every node reached from
 * such a seed along that map is marked too.  out[i] = 1 marks a node; returns
 * their number.  second (optional) receives the runner-up control of every
 * free node (-1 elsewhere). */
long long ohjb_tie_influence(const ohjb_problem *p, const double *V, const int32_t *policy,
                             double eps, double face_eps, int closure, uint8_t *out,
                             int32_t *second_arg) {
    long long N = node_count(p);
    long long *queue = (long long *)malloc(sizeof(long long) * N);
    long long head = 0, tail = 0;
    for (long long i = 0; i < N; ++i) {
        out[i] = 0;
        if (second_arg) second_arg[i] = -1;
        if (policy[i] < 0 || p->target[i] != 0) continue;
        int idx[3];
        unflatten(p, i, idx);
        double best = INFINITY, second = INFINITY;
        int jb = -1, js = -1;
        for (int j = 0; j < p->ncontrols; ++j) {
            double g[3], off[3];
            double q = foot(p, i, idx, j, g, off) ? q1_at(p, V, g, NULL) : p->v_out;
            if (q < best) {
                second = best;
                js = jb;
                best = q;
                jb = j;
            } else if (q < second) {
                second = q;
                js = j;
            }
        }
        if (second_arg) second_arg[i] = js;
        int seed = (second - best) <= eps;
        double g[3], off[3];
        if (!seed && foot(p, i, idx, policy[i], g, off))
            for (int d = 0; d < p->ndim; ++d) {
                double t = g[d] - floor(g[d]);
                if (t <= face_eps || t >= 1.0 - face_eps) seed = 1;
            }
        if (seed) {
            out[i] = 1;
            queue[tail++] = i;
        }
    }
    while (closure && head < tail) {
        long long i = queue[head++];
        if (policy[i] < 0 || p->target[i] != 0) continue;
        long long ci[8];
        double cw[8];
        int nc = row_weights(p, i, policy[i], ci, cw, NULL, NULL);
        for (int m = 0; m < nc; ++m)
            if (cw[m] > 0.0 && !out[ci[m]]) {
                out[ci[m]] = 1;
                queue[tail++] = ci[m];
            }
    }
    free(queue);
    return tail;
}

/* Number of OpenMP threads the library would use (1 without OpenMP). */
int ohjb_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
