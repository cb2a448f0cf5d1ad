/*
 * msg_oracle.c -- plain, slow, scalar FP64 reference of the MSG-MIMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: only the test suite, the smoke check and the CPU baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; neither includes the other.
 *
 * What it computes (Robbe, Nuyens, Vandewalle, "Enhanced Multi-Index Monte
 * Carlo by means of Multiple Semi-Coarsened Multigrid for Anisotropic
 * Diffusion Problems", arXiv:1907.12334):
 *   - the model problem -div(a grad u) = h on [0,1]^2, u = 0 on the boundary,
 *     with a = exp(Z) (Sec. 1, Eq. (1.1));
 *   - Z = Phi diag(sqrt(lambda)) xi, a truncated Karhunen-Loeve sum (an input
 *     law added on top of the paper, which samples by circulant embedding);
 *   - the semi-coarsened grid hierarchy G^(p,q) (Sec. 2, Eq. (2.1)) with a
 *     direct finite-difference discretisation on every grid;
 *   - red-black Gauss-Seidel smoothing, full-weighting restriction combined
 *     over two parents (Eq. (2.3)), linear prolongation combined over two
 *     children with matrix-dependent weights (Eqs. (2.4)-(2.5)), the MSG
 *     mu-cycle (Algorithm 1) and the FMSG F-cycle with cubic interpolation and
 *     an adaptive number of cycles (Algorithm 2);
 *   - the quantities of interest of Sec. 4 (the integral of u, Q1, Q2, Q3);
 *   - the multi-index differences (Sec. 3, Eq. (3.2)) and the per-sample sum
 *     Y of the unbiased estimator (Eq. (3.6));
 *   - the counter-based generator for xi: Philox4x64-10 (Salmon, Moraes,
 *     Dror, Shaw, SC'11) and the Box-Muller transform.
 *
 * Readings of the paper that this file fixes (where the paper is silent or
 * ambiguous) are marked READING in the comments.
 *
 * Grid arrays include the boundary: grid (p,q) has nx = 2^p, ny = 2^q cells,
 * nodes (i,j), 0<=i<=nx, 0<=j<=ny, stored at j*(nx+1)+i (x fastest).
 * Unknowns are the interior nodes; boundary entries of u stay 0.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846264338327950288
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 and Box-Muller                                              */
/* ------------------------------------------------------------------------ */

/* One Philox4x64-10 block: four 64-bit outputs for counter ctr and key key.
 * Multipliers and Weyl increments are the published Philox4x64 constants. */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        __uint128_t p0 = (__uint128_t)0xD2E7470EE14C6C93ULL * x0;
        __uint128_t p1 = (__uint128_t)0xCA5A826395121157ULL * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        uint64_t n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Standard normals xi[0..M) of sample number s for a given seed.
 * Block j (terms 4j..4j+3) uses counter (j, s, 0, 0) and key (seed, 0).
 * A 64-bit word w becomes the uniform U = (w >> 11) * 2^-53 in [0,1); the
 * pairs (U0,U1), (U2,U3) go through Box-Muller:
 *   R = sqrt(-2 ln(1 - Ua)),  z_a = R cos(2 pi Ub),  z_b = R sin(2 pi Ub). */
void orc_normals(uint64_t seed, uint64_t s, int32_t M, double* xi)
{
    const double two_pi = 6.283185307179586476925286766559;
    const double inv53 = 1.0 / 9007199254740992.0; /* 2^-53 */
    for (int32_t j = 0; 4 * j < M; ++j) {
        uint64_t ctr[4] = {(uint64_t)j, s, 0, 0}, key[2] = {seed, 0}, w[4];
        orc_philox4x64_10(ctr, key, w);
        double z[4];
        for (int h = 0; h < 2; ++h) {
            double ua = (double)(w[2 * h] >> 11) * inv53;
            double ub = (double)(w[2 * h + 1] >> 11) * inv53;
            double rad = sqrt(-2.0 * log(1.0 - ua));
            z[2 * h] = rad * cos(two_pi * ub);
            z[2 * h + 1] = rad * sin(two_pi * ub);
        }
        for (int k = 0; k < 4 && 4 * j + k < M; ++k) xi[4 * j + k] = z[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Truncated KL field                                                       */
/* ------------------------------------------------------------------------ */

/* Z[x] = sum_m Phi[x][m] * sqrt_lambda[m] * xi[m], summed in m order.
 * Phi is row-major [npts][M]. */
void orc_kl_field(const double* Phi, const double* sqrt_lambda, const double* xi,
                  int64_t npts, int32_t M, double* Z)
{
    for (int64_t x = 0; x < npts; ++x) {
        double acc = 0.0;
        for (int32_t m = 0; m < M; ++m) acc += Phi[x * M + m] * sqrt_lambda[m] * xi[m];
        Z[x] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Grid hierarchy                                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    int p, q, nx, ny;
    double dx, dy;
    double* u;  /* (nx+1)(ny+1) nodes, current approximation v */
    double* b;  /* right-hand side */
    double* r;  /* residual */
    double* ax; /* a at x-face (i+1/2, j): ax[j*nx + i], 0<=i<nx, 0<=j<=ny */
    double* ay; /* a at y-face (i, j+1/2): ay[j*(nx+1) + i], 0<=i<=nx, 0<=j<ny */
    double* sol; /* saved FMSG solution on this grid (Algorithm 2 output) */
} ogrid;

typedef struct {
    int P, Q;   /* finest grid of the sample (storage extent) */
    int Pa, Qa; /* finest grid of the hierarchy Algorithm 1 currently works on */
    int mu, nu1, nu2, max_cycles;
    double eps, omega;
    ogrid* g; /* indexed [p*(Q+1)+q], 1<=p<=P, 1<=q<=Q */
    int* cycles; /* per relative diagonal s: max cycles over its grids */
    int* grid_cycles; /* [P][Q]: cycles used on grid (p,q) */
    double* grid_relres; /* [P][Q]: final ||r||/||b|| on grid (p,q) */
    double* relres; /* per relative diagonal s: max ||r||/||b|| after the last cycle */
    int status;
} ohier;

static ogrid* G(ohier* H, int p, int q) { return &H->g[p * (H->Q + 1) + q]; }

static int nodes(const ogrid* g) { return (g->nx + 1) * (g->ny + 1); }

void orc_hier_free(ohier* H)
{
    if (!H) return;
    if (H->g) {
        for (int p = 1; p <= H->P; ++p)
            for (int q = 1; q <= H->Q; ++q) {
                ogrid* g = G(H, p, q);
                free(g->u); free(g->b); free(g->r); free(g->ax); free(g->ay); free(g->sol);
            }
        free(H->g);
    }
    free(H->cycles);
    free(H->relres);
    free(H->grid_cycles);
    free(H->grid_relres);
    free(H);
}

ohier* orc_hier_new(int P, int Q)
{
    if (P < 1 || Q < 1 || P > 14 || Q > 14) return NULL;
    ohier* H = (ohier*)calloc(1, sizeof(ohier));
    if (!H) return NULL;
    H->P = P; H->Q = Q; H->Pa = P; H->Qa = Q;
    H->mu = 2; H->nu1 = 2; H->nu2 = 2; H->max_cycles = 50;
    H->eps = 1e-12; H->omega = 1.0;
    H->g = (ogrid*)calloc((size_t)(P + 1) * (Q + 1), sizeof(ogrid));
    H->cycles = (int*)calloc((size_t)(P + Q), sizeof(int));
    H->relres = (double*)calloc((size_t)(P + Q), sizeof(double));
    H->grid_cycles = (int*)calloc((size_t)P * Q, sizeof(int));
    H->grid_relres = (double*)calloc((size_t)P * Q, sizeof(double));
    if (!H->g || !H->cycles || !H->relres || !H->grid_cycles || !H->grid_relres) { orc_hier_free(H); return NULL; }
    for (int p = 1; p <= P; ++p)
        for (int q = 1; q <= Q; ++q) {
            ogrid* g = G(H, p, q);
            g->p = p; g->q = q; g->nx = 1 << p; g->ny = 1 << q;
            g->dx = 1.0 / g->nx; g->dy = 1.0 / g->ny;
            int n = nodes(g);
            g->u = (double*)calloc(n, sizeof(double));
            g->b = (double*)calloc(n, sizeof(double));
            g->r = (double*)calloc(n, sizeof(double));
            g->sol = (double*)calloc(n, sizeof(double));
            g->ax = (double*)calloc((size_t)g->nx * (g->ny + 1), sizeof(double));
            g->ay = (double*)calloc((size_t)(g->nx + 1) * g->ny, sizeof(double));
            if (!g->u || !g->b || !g->r || !g->sol || !g->ax || !g->ay) { orc_hier_free(H); return NULL; }
        }
    return H;
}

void orc_hier_set_params(ohier* H, int mu, int nu1, int nu2, int max_cycles, double eps, double omega)
{
    H->mu = mu; H->nu1 = nu1; H->nu2 = nu2; H->max_cycles = max_cycles;
    H->eps = eps; H->omega = omega;
}

/* Size (in doubles) of the field grid F = nodes of G^(P+1,Q+1). */
int64_t orc_field_points(int P, int Q)
{
    return (int64_t)((1 << (P + 1)) + 1) * ((1 << (Q + 1)) + 1);
}

/* Coefficients on every grid from the field Z given on F (row-major, x fastest).
 * READING (the paper does not say where, or how, a is evaluated on a grid).
 * The field lives on F, the nodes of G^(P+1,Q+1); the finest grid G^(P,Q)
 * takes a = exp(Z) at its face midpoints, i.e. at F-node (2i+1, 2j) for the
 * x-face (i+1/2, j) and (2i, 2j+1) for the y-face (i, j+1/2).  A coarser grid
 * (p,q) covers sx = 2^(P-p) finest x-faces with each of its x-faces and
 * sy = 2^(Q-q) finest y-faces with each y-face:
 *   mode 0 (default): the series (harmonic) mean of those finest-face values
 *     along the flux direction, a = sx / sum_k exp(-Z_k) (exp(Z) when sx = 1);
 *   mode 1: injection, a = exp(Z) at the coarse face midpoint, F-node
 *     ((2i+1) sx, 2j sy) and (2i sx, (2j+1) sy).
 * Both give every grid of a sample one realisation of a.  Injection makes the
 * coarse operators of fields much rougher than the coarse mesh poor copies of
 * the fine ones: on the 0.02-correlation-length field 3 of 32 samples at
 * 256 x 256 do not converge and the one-column grids need 45-60 cycles on
 * average; the series mean is the 1-D homogenised coefficient of the covered
 * segment and brings that to 1 of 32 and 7-10 cycles. */
void orc_hier_set_field_mode(ohier* H, const double* Z, int mode)
{
    int NFx = (1 << (H->P + 1)) + 1;
    for (int p = 1; p <= H->P; ++p)
        for (int q = 1; q <= H->Q; ++q) {
            ogrid* g = G(H, p, q);
            int sx = 1 << (H->P - p), sy = 1 << (H->Q - q);
            for (int j = 0; j <= g->ny; ++j)
                for (int i = 0; i < g->nx; ++i) {
                    int64_t row = (int64_t)(2 * j * sy) * NFx;
                    double a;
                    if (mode == 1 || sx == 1) {
                        a = exp(Z[row + (2 * i + 1) * sx]);
                    } else {
                        double s = 0.0;
                        for (int k = 0; k < sx; ++k) s += exp(-Z[row + 2 * (i * sx + k) + 1]);
                        a = sx / s;
                    }
                    g->ax[j * g->nx + i] = a;
                }
            for (int j = 0; j < g->ny; ++j)
                for (int i = 0; i <= g->nx; ++i) {
                    double a;
                    if (mode == 1 || sy == 1) {
                        a = exp(Z[(int64_t)((2 * j + 1) * sy) * NFx + 2 * i * sx]);
                    } else {
                        double s = 0.0;
                        for (int k = 0; k < sy; ++k) s += exp(-Z[(int64_t)(2 * (j * sy + k) + 1) * NFx + 2 * i * sx]);
                        a = sy / s;
                    }
                    g->ay[j * (g->nx + 1) + i] = a;
                }
        }
}

void orc_hier_set_field(ohier* H, const double* Z) { orc_hier_set_field_mode(H, Z, 0); }

/* Set the right-hand side on the finest grid from nodal values h (same node
 * layout as grid (P,Q)); h == NULL means h = 1 (the paper's source term). */
void orc_hier_set_rhs(ohier* H, const double* h)
{
    ogrid* g = G(H, H->P, H->Q);
    for (int j = 0; j < g->ny + 1; ++j)
        for (int i = 0; i < g->nx + 1; ++i) {
            int c = j * (g->nx + 1) + i;
            int interior = i > 0 && i < g->nx && j > 0 && j < g->ny;
            g->b[c] = interior ? (h ? h[c] : 1.0) : 0.0;
        }
}

/* ------------------------------------------------------------------------ */
/* Discrete operator and smoother                                           */
/* ------------------------------------------------------------------------ */

/* Standard conservative five-point difference (READING: the paper only says
 * "finite differences" obtained by direct discretisation on every grid):
 * (A v)_ij = -[a_e (v_{i+1,j} - v_ij) - a_w (v_ij - v_{i-1,j})] / dx^2
 *            -[a_n (v_{i,j+1} - v_ij) - a_s (v_ij - v_{i,j-1})] / dy^2 */
static double apply_at(const ogrid* g, const double* v, int i, int j)
{
    int W = g->nx + 1, c = j * W + i;
    double aw = g->ax[j * g->nx + i - 1], ae = g->ax[j * g->nx + i];
    double as = g->ay[(j - 1) * W + i], an = g->ay[j * W + i];
    double idx2 = 1.0 / (g->dx * g->dx), idy2 = 1.0 / (g->dy * g->dy);
    return -(ae * (v[c + 1] - v[c]) - aw * (v[c] - v[c - 1])) * idx2
           - (an * (v[c + W] - v[c]) - as * (v[c] - v[c - W])) * idy2;
}

/* Diagonal entry of A at an interior node. */
static double diag_at(const ogrid* g, int i, int j)
{
    int W = g->nx + 1;
    double aw = g->ax[j * g->nx + i - 1], ae = g->ax[j * g->nx + i];
    double as = g->ay[(j - 1) * W + i], an = g->ay[j * W + i];
    return (aw + ae) / (g->dx * g->dx) + (as + an) / (g->dy * g->dy);
}

/* out = A v on the interior (boundary of out set to 0). */
static void apply_A(const ogrid* g, const double* v, double* out)
{
    memset(out, 0, sizeof(double) * nodes(g));
    for (int j = 1; j < g->ny; ++j)
        for (int i = 1; i < g->nx; ++i) out[j * (g->nx + 1) + i] = apply_at(g, v, i, j);
}

/* One red-black Gauss-Seidel sweep (Sec. 2, numerical setup): red nodes
 * (i+j even) first, then black.  READING: the paper does not fix the colour
 * order; red first. */
static void smooth_rbgs(ogrid* g)
{
    int W = g->nx + 1;
    for (int colour = 0; colour < 2; ++colour)
        for (int j = 1; j < g->ny; ++j)
            for (int i = 1; i < g->nx; ++i) {
                if (((i + j) & 1) != colour) continue;
                int c = j * W + i;
                double d = diag_at(g, i, j);
                /* v_ij <- v_ij + (b - A v)_ij / A_ii : exact point solve */
                g->u[c] += (g->b[c] - apply_at(g, g->u, i, j)) / d;
            }
}

static void residual(ogrid* g)
{
    apply_A(g, g->u, g->r);
    int n = nodes(g);
    for (int c = 0; c < n; ++c) g->r[c] = g->b[c] - g->r[c];
    /* boundary: b and A v are both 0 there */
}

/* Discrete L2 norm ||v||_h = sqrt(dx dy sum_interior v^2). */
static double norm_h(const ogrid* g, const double* v)
{
    double s = 0.0;
    for (int j = 1; j < g->ny; ++j)
        for (int i = 1; i < g->nx; ++i) {
            double t = v[j * (g->nx + 1) + i];
            s += t * t;
        }
    return sqrt(g->dx * g->dy * s);
}

/* ------------------------------------------------------------------------ */
/* Transfer operators (Sec. 2)                                              */
/* ------------------------------------------------------------------------ */

/* Full weighting along x from fine (p+1,q) to coarse (p,q): stencil 1/4[1 2 1]. */
static double Rx_at(const ogrid* fine, const double* f, int ic, int j)
{
    int W = fine->nx + 1, c = j * W + 2 * ic;
    return 0.25 * (f[c - 1] + 2.0 * f[c] + f[c + 1]);
}

/* Full weighting along y from fine (p,q+1) to coarse (p,q). */
static double Ry_at(const ogrid* fine, const double* f, int i, int jc)
{
    int W = fine->nx + 1, c = 2 * jc * W + i;
    return 0.25 * (f[c - W] + 2.0 * f[c] + f[c + W]);
}

/* Restriction to (p,q) combined over its parents, Eq. (2.3):
 * only R_x from (p+1,q) when q = Q, only R_y from (p,q+1) when p = P,
 * otherwise the average of both.  src selects the residual (0) or the
 * right-hand side (1) of the parents (Algorithm 2 restricts the latter). */
static void restrict_to(ohier* H, int p, int q, int src)
{
    ogrid* g = G(H, p, q);
    int hasx = p < H->Pa, hasy = q < H->Qa;
    ogrid* fx = hasx ? G(H, p + 1, q) : NULL;
    ogrid* fy = hasy ? G(H, p, q + 1) : NULL;
    memset(g->b, 0, sizeof(double) * nodes(g));
    for (int j = 1; j < g->ny; ++j)
        for (int i = 1; i < g->nx; ++i) {
            double v;
            if (hasx && !hasy) v = Rx_at(fx, src ? fx->b : fx->r, i, j);
            else if (hasy && !hasx) v = Ry_at(fy, src ? fy->b : fy->r, i, j);
            else v = 0.5 * Rx_at(fx, src ? fx->b : fx->r, i, j) + 0.5 * Ry_at(fy, src ? fy->b : fy->r, i, j);
            g->b[j * (g->nx + 1) + i] = v;
        }
}

/* Linear interpolation along x from coarse (p-1,q) to fine node (i,j) of (p,q):
 * even i copies the coarse node, odd i averages its two coarse neighbours;
 * boundary values are 0. */
static double Px_lin(const ogrid* coarse, const double* v, int i, int j)
{
    int W = coarse->nx + 1;
    if ((i & 1) == 0) return v[j * W + i / 2];
    return 0.5 * (v[j * W + i / 2] + v[j * W + i / 2 + 1]);
}

static double Py_lin(const ogrid* coarse, const double* v, int i, int j)
{
    int W = coarse->nx + 1;
    if ((j & 1) == 0) return v[(j / 2) * W + i];
    return 0.5 * (v[(j / 2) * W + i] + v[(j / 2 + 1) * W + i]);
}

/* Cubic interpolation along one axis (Sec. 2, FMSG): fine odd node between
 * coarse c_k and c_{k+1} gets (-c_{k-1} + 9 c_k + 9 c_{k+1} - c_{k+2}) / 16.
 * READING of the boundary stencil 1/16[10 16 9 0 -1]: it is the interior
 * stencil with the ghost value outside the Dirichlet boundary taken as the
 * odd reflection c_{-1} = -c_1 (so the first fine odd node gets
 * (10 c_1 - c_2)/16); the same holds at the right end. */
static double cubic_line(const double* c, int stride, int m, int k)
{
    /* c: coarse line with nodes 0..m (boundary 0 at both ends), fine odd node 2k+1 */
    double cm1 = (k - 1 >= 0) ? c[(k - 1) * stride] : -c[1 * stride];
    double c0 = c[k * stride];
    double c1 = c[(k + 1) * stride];
    double c2 = (k + 2 <= m) ? c[(k + 2) * stride] : -c[(m - 1) * stride];
    return (-cm1 + 9.0 * c0 + 9.0 * c1 - c2) / 16.0;
}

static double Px_cub(const ogrid* coarse, const double* v, int i, int j)
{
    int W = coarse->nx + 1;
    if ((i & 1) == 0) return v[j * W + i / 2];
    return cubic_line(v + j * W, 1, coarse->nx, i / 2);
}

static double Py_cub(const ogrid* coarse, const double* v, int i, int j)
{
    int W = coarse->nx + 1;
    if ((j & 1) == 0) return v[(j / 2) * W + i];
    return cubic_line(v + i, W, coarse->ny, j / 2);
}

/* Matrix-dependent weights, Eq. (2.5): lambda_x = (A f)_ij, lambda_y = (A g)_ij
 * with f_ij = cos(i pi), g_ij = cos(j pi) on all nodes 0..2^p, 0..2^q.
 * READING: f and g keep their values on the boundary nodes when the stencil
 * reaches them (the paper defines them there). */
static void kappa_at(const ogrid* g, int i, int j, double* kx, double* ky)
{
    int W = g->nx + 1;
    double aw = g->ax[j * g->nx + i - 1], ae = g->ax[j * g->nx + i];
    double as = g->ay[(j - 1) * W + i], an = g->ay[j * W + i];
    double idx2 = 1.0 / (g->dx * g->dx), idy2 = 1.0 / (g->dy * g->dy);
    double f_c = cos(i * ORC_PI), f_w = cos((i - 1) * ORC_PI), f_e = cos((i + 1) * ORC_PI);
    double f_s = f_c, f_n = f_c; /* f does not vary with j */
    double g_c = cos(j * ORC_PI), g_s = cos((j - 1) * ORC_PI), g_n = cos((j + 1) * ORC_PI);
    double g_w = g_c, g_e = g_c;
    double lx = -(ae * (f_e - f_c) - aw * (f_c - f_w)) * idx2 - (an * (f_n - f_c) - as * (f_c - f_s)) * idy2;
    double ly = -(ae * (g_e - g_c) - aw * (g_c - g_w)) * idx2 - (an * (g_n - g_c) - as * (g_c - g_s)) * idy2;
    *kx = lx * lx / (lx * lx + ly * ly);
    *ky = ly * ly / (lx * lx + ly * ly);
}

/* Interpolation to (p,q) combined over its children, Eq. (2.4):
 * only P_x from (p-1,q) when q = 1, only P_y from (p,q-1) when p = 1,
 * otherwise kappa_x P_x + kappa_y P_y.  mode 0: linear, added to u with
 * damping omega (coarse-grid correction of Algorithm 1); mode 1: cubic,
 * replacing u (initial guess of Algorithm 2), taken from the children's
 * saved solutions. */
static void interpolate_to(ohier* H, int p, int q, int mode)
{
    ogrid* g = G(H, p, q);
    int hasx = p > 1, hasy = q > 1;
    ogrid* cx = hasx ? G(H, p - 1, q) : NULL;
    ogrid* cy = hasy ? G(H, p, q - 1) : NULL;
    for (int j = 1; j < g->ny; ++j)
        for (int i = 1; i < g->nx; ++i) {
            double vx = 0.0, vy = 0.0, wx = 0.0, wy = 0.0;
            if (hasx) vx = mode ? Px_cub(cx, cx->sol, i, j) : Px_lin(cx, cx->u, i, j);
            if (hasy) vy = mode ? Py_cub(cy, cy->sol, i, j) : Py_lin(cy, cy->u, i, j);
            if (hasx && hasy) kappa_at(g, i, j, &wx, &wy);
            else if (hasx) wx = 1.0;
            else wy = 1.0;
            double corr = wx * vx + wy * vy;
            int c = j * (g->nx + 1) + i;
            if (mode) g->u[c] = corr;
            else g->u[c] += H->omega * corr;
        }
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 and Algorithm 2                                               */
/* ------------------------------------------------------------------------ */

/* READING: the paper indexes the recursion by L with L = 0 the one-unknown
 * grid, while G^(0,0) of Eq. (2.1) has no interior node.  The recursion level
 * used here is the relative diagonal s = (p-1) + (q-1), so s = 0 is G^(1,1). */
/* Grids of the hierarchy on relative diagonal s, in increasing p. */
static int diag_grids(const ohier* H, int s, int* ps, int* qs)
{
    int n = 0;
    for (int p = 1; p <= H->Pa; ++p) {
        int q = s + 2 - p;
        if (q >= 1 && q <= H->Qa) { ps[n] = p; qs[n] = q; ++n; }
    }
    return n;
}

#define FOR_DIAG(H, s, p, q)                                                        \
    for (int _n = 0, _ps[32], _qs[32], _cnt = diag_grids((H), (s), _ps, _qs); _n < _cnt; ++_n) \
        for (int p = _ps[_n], q = _qs[_n], _once = 1; _once; _once = 0)

static void coarsest_solve(ohier* H)
{
    ogrid* g = G(H, 1, 1);
    int c = 1 * (g->nx + 1) + 1;
    g->u[c] = g->b[c] / diag_at(g, 1, 1);
}

void orc_mu_cycle(ohier* H, int s)
{
    if (s == 0) { coarsest_solve(H); return; }
    FOR_DIAG(H, s, p, q) { for (int k = 0; k < H->nu1; ++k) smooth_rbgs(G(H, p, q)); }
    FOR_DIAG(H, s, p, q) { residual(G(H, p, q)); }
    FOR_DIAG(H, s - 1, p, q) {
        restrict_to(H, p, q, 0);
        memset(G(H, p, q)->u, 0, sizeof(double) * nodes(G(H, p, q)));
    }
    for (int k = 0; k < H->mu; ++k) orc_mu_cycle(H, s - 1);
    FOR_DIAG(H, s, p, q) {
        interpolate_to(H, p, q, 0);
        for (int k = 0; k < H->nu2; ++k) smooth_rbgs(G(H, p, q));
    }
}

/* ||b - A v||_h / ||b||_h on one grid */
static double grid_relres(ogrid* g)
{
    residual(g);
    double nb = norm_h(g, g->b);
    return norm_h(g, g->r) / (nb > 0.0 ? nb : 1.0);
}

/* MSG-F-CYCLE(s), Algorithm 2, with the adaptive nu_0 of Sec. 2.
 *
 * READING: the paper repeats MSG-mu-CYCLE(s) on diagonal s until every grid
 * there has ||r||/||b|| <= eps.  Run as one mu-cycle shared by all grids of
 * the diagonal, the coarse grid between two fine grids receives the average
 * of two residuals of independent problems (Eq. (2.3)) and the error mode
 * alternating in sign from grid to grid is never corrected: measured rates
 * are 0.4-0.75 with a = 1 and above 0.95 on the anisotropic lognormal field,
 * so the criterion is out of reach.  Here each grid (p,q) of diagonal s is
 * iterated by Algorithm 1 with (p,q) as the finest grid of its own hierarchy
 * {(p',q'): p' <= p, q' <= q} (so the two-parent average only ever combines
 * residuals of one error), until its own ||r||/||b|| <= eps (at least one
 * cycle, at most max_cycles).  READING: the paper only says the cycle count is
 * increased until the criterion holds; a grid whose relative residual after
 * a cycle exceeds both 1 (the zero guess) and the relative residual of its
 * initial guess has diverged and stops there, flagged as not converged,
 * instead of running on to max_cycles.  (On strongly anisotropic grids the
 * interpolated initial guess can start well above 1 and a converging grid may
 * still be above 1 after its first cycle.)  The solution of each grid is saved
 * when its stage ends, before cycles on finer diagonals reuse its u and b as
 * scratch. */
static void f_cycle(ohier* H, int s)
{
    if (s == 0) {
        memset(G(H, 1, 1)->u, 0, sizeof(double) * nodes(G(H, 1, 1)));
    } else {
        FOR_DIAG(H, s - 1, p, q) { restrict_to(H, p, q, 1); }
        f_cycle(H, s - 1);
        FOR_DIAG(H, s, p, q) { interpolate_to(H, p, q, 1); }
    }
    int worst_n = 0;
    double worst_rr = 0.0;
    FOR_DIAG(H, s, p, q) {
        ogrid* g = G(H, p, q);
        H->Pa = p; H->Qa = q; /* the hierarchy below (p,q) */
        int n = 0;
        double rr = 0.0;
        const double rr0 = grid_relres(g); /* the initial guess */
        do {
            orc_mu_cycle(H, s);
            ++n;
            rr = grid_relres(g);
        } while (!(rr <= H->eps) && n < H->max_cycles && rr == rr && (rr <= 1.0 || rr <= rr0));
        H->Pa = H->P; H->Qa = H->Q;
        H->grid_cycles[(p - 1) * H->Q + (q - 1)] = n;
        H->grid_relres[(p - 1) * H->Q + (q - 1)] = rr;
        if (!(rr == rr)) H->status |= 2;          /* non-finite residual */
        else if (!(rr <= H->eps)) H->status |= 1; /* not converged within max_cycles */
        if (n > worst_n) worst_n = n;
        if (!(rr <= worst_rr)) worst_rr = rr;
        memcpy(g->sol, g->u, sizeof(double) * nodes(g));
    }
    H->cycles[s] = worst_n;
    H->relres[s] = worst_rr;
}

/* Full FMSG solve with b = h on the finest grid. Returns the status bits. */
int orc_fmsg(ohier* H)
{
    H->status = 0;
    f_cycle(H, H->P + H->Q - 2);
    return H->status;
}

/* ------------------------------------------------------------------------ */
/* Quantities of interest (Sec. 4)                                          */
/* ------------------------------------------------------------------------ */

#define QOI_INTEGRAL 0
#define QOI_POINT 1
#define QOI_SUBDOMAIN 2
#define QOI_FLUX 3

/* QoI of a nodal field v on grid g.
 *  0: integral of u over D, trapezoid rule (u = 0 on the boundary);
 *  1: Q1 = u(1/2, 1/2);
 *  2: Q2 = mean of u over [1/4,1/2]^2, 2-D trapezoid rule (needs p,q >= 2);
 *  3: Q3 = -int_0^1 a(1,y) du/dx(1,y) dy, trapezoid rule in y, one-sided
 *     first-order difference du/dx(1,y_j) = (0 - v_{nx-1,j})/dx; a(1,y_j) is
 *     exp(Z) at the F-node (2^(P+1), 2 j 2^(Q-q)). */
static double qoi_of(const ohier* H, const ogrid* g, const double* v, int qoi, const double* Z)
{
    int W = g->nx + 1;
    if (qoi == QOI_INTEGRAL) {
        double s = 0.0;
        for (int j = 1; j < g->ny; ++j)
            for (int i = 1; i < g->nx; ++i) s += v[j * W + i];
        return g->dx * g->dy * s;
    }
    if (qoi == QOI_POINT) return v[(g->ny / 2) * W + g->nx / 2];
    if (qoi == QOI_SUBDOMAIN) {
        if (g->p < 2 || g->q < 2) return NAN;
        int i0 = g->nx / 4, i1 = g->nx / 2, j0 = g->ny / 4, j1 = g->ny / 2;
        double s = 0.0;
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                double w = ((i == i0 || i == i1) ? 0.5 : 1.0) * ((j == j0 || j == j1) ? 0.5 : 1.0);
                s += w * v[j * W + i];
            }
        return s * g->dx * g->dy / (0.25 * 0.25);
    }
    if (qoi == QOI_FLUX) {
        int NFx = (1 << (H->P + 1)) + 1, sy = 1 << (H->Q - g->q);
        double s = 0.0;
        for (int j = 1; j < g->ny; ++j) {
            double a = exp(Z[(int64_t)(2 * j * sy) * NFx + (NFx - 1)]);
            s += a * v[j * W + g->nx - 1] / g->dx;
        }
        return g->dy * s;
    }
    return NAN;
}

/* ------------------------------------------------------------------------ */
/* Whole-sample entry points                                                */
/* ------------------------------------------------------------------------ */

/* Solve one sample by FMSG and return the QoI of every grid.
 * Z: field on F ((2^(P+1)+1) x (2^(Q+1)+1), x fastest).
 * Qout: [P][Q], Qout[(p-1)*Q + (q-1)] = QoI on grid (p,q).
 * cycles_out (optional, [P][Q]): cycles used on each grid.
 * relres_out (optional, [P][Q]): final ||r||/||b|| on each grid.
 * Returns status bits (1 = not converged, 2 = non-finite), or -1 on bad input. */
int orc_solve_sample(int P, int Q, const double* Z, int mu, int nu1, int nu2, int max_cycles,
                     double eps, double omega, int qoi, int coef_mode, double* Qout, int* cycles_out,
                     double* relres_out)
{
    ohier* H = orc_hier_new(P, Q);
    if (!H) return -1;
    orc_hier_set_params(H, mu, nu1, nu2, max_cycles, eps, omega);
    orc_hier_set_field_mode(H, Z, coef_mode);
    orc_hier_set_rhs(H, NULL);
    int st = orc_fmsg(H);
    for (int p = 1; p <= P; ++p)
        for (int q = 1; q <= Q; ++q) {
            ogrid* g = G(H, p, q);
            Qout[(p - 1) * Q + (q - 1)] = qoi_of(H, g, g->sol, qoi, Z);
        }
    for (int k = 0; k < P * Q; ++k) {
        if (cycles_out) cycles_out[k] = H->grid_cycles[k];
        if (relres_out) relres_out[k] = H->grid_relres[k];
    }
    orc_hier_free(H);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Multi-index differences and the per-sample estimator term (Sec. 3)       */
/* ------------------------------------------------------------------------ */

/* For a sample whose finest index is L = (L1, L2) and whose grid QoIs are
 * Qgrid[(p-1)*Qn + (q-1)] for 1<=p<=Pn, 1<=q<=Qn, the multi-index QoI is
 * Q_l = Qgrid at (p0 + l1, q0 + l2) (Sec. 3).  For 0 <= tau <= L:
 *   dQ_tau = D_2 D_1 Q_tau with D_i Q_l = Q_l - Q_{l - e_i} if l_i > 0, else Q_l
 * (Eq. (3.2)); dQ is written row-major [L1+1][L2+1].
 * If ptau != NULL (row-major [ld1][ld2] tail probabilities p_tau), Y = sum_tau
 * dQ_tau / p_tau (Eq. (3.6)) is returned through *Y. */
int orc_mimc_differences(int L1, int L2, int p0, int q0, int Pn, int Qn, const double* Qgrid,
                         const double* ptau, int ld1, int ld2, double* dQ, double* Y)
{
    if (p0 + L1 > Pn || q0 + L2 > Qn || p0 < 1 || q0 < 1) return -1;
    double y = 0.0;
    for (int t1 = 0; t1 <= L1; ++t1)
        for (int t2 = 0; t2 <= L2; ++t2) {
            /* apply D_1 then D_2 literally, as in the worked example of Sec. 3 */
            double d1_at_t2 = Qgrid[(p0 + t1 - 1) * Qn + (q0 + t2 - 1)];
            if (t1 > 0) d1_at_t2 -= Qgrid[(p0 + t1 - 2) * Qn + (q0 + t2 - 1)];
            double d = d1_at_t2;
            if (t2 > 0) {
                double d1_at_t2m1 = Qgrid[(p0 + t1 - 1) * Qn + (q0 + t2 - 2)];
                if (t1 > 0) d1_at_t2m1 -= Qgrid[(p0 + t1 - 2) * Qn + (q0 + t2 - 2)];
                d = d1_at_t2 - d1_at_t2m1;
            }
            dQ[t1 * (L2 + 1) + t2] = d;
            if (ptau) y += d / ptau[t1 * ld2 + t2];
        }
    if (ptau && Y) *Y = y;
    (void)ld1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Access for the pin tests: building blocks on a hierarchy handle          */
/* ------------------------------------------------------------------------ */

static ogrid* grid_checked(ohier* H, int p, int q)
{
    if (!H || p < 1 || q < 1 || p > H->P || q > H->Q) return NULL;
    return G(H, p, q);
}

/* which: 0 = u, 1 = b, 2 = r, 3 = sol; copies (nx+1)(ny+1) doubles */
int orc_grid_get(ohier* H, int p, int q, int which, double* out)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    double* src = which == 0 ? g->u : which == 1 ? g->b : which == 2 ? g->r : g->sol;
    memcpy(out, src, sizeof(double) * nodes(g));
    return 0;
}

int orc_grid_set(ohier* H, int p, int q, int which, const double* in)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    double* dst = which == 0 ? g->u : which == 1 ? g->b : which == 2 ? g->r : g->sol;
    memcpy(dst, in, sizeof(double) * nodes(g));
    return 0;
}

/* out = A v on grid (p,q) */
int orc_grid_apply(ohier* H, int p, int q, const double* v, double* out)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    apply_A(g, v, out);
    return 0;
}

int orc_grid_smooth(ohier* H, int p, int q, int sweeps)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    for (int k = 0; k < sweeps; ++k) smooth_rbgs(g);
    return 0;
}

int orc_grid_residual(ohier* H, int p, int q)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    residual(g);
    return 0;
}

/* src 0: restrict the parents' residuals; 1: their right-hand sides */
int orc_grid_restrict(ohier* H, int p, int q, int src)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g || (p == H->P && q == H->Q)) return -1;
    restrict_to(H, p, q, src);
    return 0;
}

/* mode 0: u += omega * linear combined correction from children's u;
 * mode 1: u = cubic combined interpolation of children's sol */
int orc_grid_interpolate(ohier* H, int p, int q, int mode)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g || (p == 1 && q == 1)) return -1;
    interpolate_to(H, p, q, mode);
    return 0;
}

/* kappa_x, kappa_y at every interior node of (p,q): arrays of (nx+1)(ny+1) */
int orc_grid_kappa(ohier* H, int p, int q, double* kx, double* ky)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    memset(kx, 0, sizeof(double) * nodes(g));
    memset(ky, 0, sizeof(double) * nodes(g));
    for (int j = 1; j < g->ny; ++j)
        for (int i = 1; i < g->nx; ++i) kappa_at(g, i, j, &kx[j * (g->nx + 1) + i], &ky[j * (g->nx + 1) + i]);
    return 0;
}

double orc_grid_qoi(ohier* H, int p, int q, int which, int qoi, const double* Z)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return NAN;
    const double* v = which == 0 ? g->u : which == 1 ? g->b : which == 2 ? g->r : g->sol;
    return qoi_of(H, g, v, qoi, Z);
}

/* per-grid cycles and final relative residuals, [P][Q] */
int orc_hier_cycles(ohier* H, int* cycles, double* relres)
{
    for (int k = 0; k < H->P * H->Q; ++k) {
        cycles[k] = H->grid_cycles[k];
        relres[k] = H->grid_relres[k];
    }
    return H->status;
}

/* face coefficients of grid (p,q): ax [(ny+1)][nx], ay [ny][(nx+1)] (unscaled a) */
int orc_grid_coef(ohier* H, int p, int q, double* ax, double* ay)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    memcpy(ax, g->ax, sizeof(double) * g->nx * (g->ny + 1));
    memcpy(ay, g->ay, sizeof(double) * (g->nx + 1) * g->ny);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Convergence study (Sec. 2, numerical experiments: residual norms over     */
/* W-cycles from a zero initial guess, MSG against multigrid with standard   */
/* coarsening).                                                              */
/* ------------------------------------------------------------------------ */

/* READING: the paper does not give the transfer operators of its "classic MG".
 * The textbook ones for vertex-centred grids are used: full weighting, the
 * tensor product of 1/4 [1 2 1] in x and y, from (p,q) to (p-1,q-1), and
 * bilinear interpolation back; the coarse operators are the direct
 * discretisations on the diagonal grids (P-k, Q-k) of the MSG hierarchy (the
 * same coefficients), with the same red-black smoother and damping.  Coarsening
 * stops at the first grid with a single interior line (p = 1 or q = 1), solved
 * exactly. */
static double Rfw_at(const ogrid* f, const double* r, int ic, int jc)
{
    int W = f->nx + 1, c = 2 * jc * W + 2 * ic;
    double edge = r[c - 1] + r[c + 1] + r[c - W] + r[c + W];
    double corner = r[c - W - 1] + r[c - W + 1] + r[c + W - 1] + r[c + W + 1];
    return (4.0 * r[c] + 2.0 * edge + corner) / 16.0;
}

/* bilinear interpolation from (p-1,q-1) to fine node (i,j) of (p,q) */
static double Pbl_at(const ogrid* co, const double* v, int i, int j)
{
    int W = co->nx + 1, i0 = i / 2, j0 = j / 2;
    if (!(i & 1) && !(j & 1)) return v[j0 * W + i0];
    if ((i & 1) && !(j & 1)) return 0.5 * (v[j0 * W + i0] + v[j0 * W + i0 + 1]);
    if (!(i & 1) && (j & 1)) return 0.5 * (v[j0 * W + i0] + v[(j0 + 1) * W + i0]);
    return 0.25 * (v[j0 * W + i0] + v[j0 * W + i0 + 1] + v[(j0 + 1) * W + i0] + v[(j0 + 1) * W + i0 + 1]);
}

/* exact solve of A u = b on a grid with one interior line (Thomas algorithm) */
static void line_solve(ogrid* g)
{
    const int row = g->ny == 2; /* one interior row (else one interior column) */
    const int n = row ? g->nx - 1 : g->ny - 1, W = g->nx + 1;
    double* cp = (double*)calloc((size_t)n + 1, sizeof(double));
    double* dp = (double*)calloc((size_t)n + 1, sizeof(double));
    for (int k = 0; k < n; ++k) {
        int i = row ? k + 1 : 1, j = row ? 1 : k + 1, c = j * W + i;
        double lo, up; /* couplings to the previous and next unknown of the line */
        if (row) { lo = -g->ax[j * g->nx + i - 1] / (g->dx * g->dx); up = -g->ax[j * g->nx + i] / (g->dx * g->dx); }
        else { lo = -g->ay[(j - 1) * W + i] / (g->dy * g->dy); up = -g->ay[j * W + i] / (g->dy * g->dy); }
        double d = diag_at(g, i, j) - (k > 0 ? lo * cp[k - 1] : 0.0);
        cp[k] = up / d;
        dp[k] = (g->b[c] - (k > 0 ? lo * dp[k - 1] : 0.0)) / d;
    }
    for (int k = n - 1; k >= 0; --k) {
        int i = row ? k + 1 : 1, j = row ? 1 : k + 1;
        double next = k + 1 < n ? g->u[row ? j * W + i + 1 : (j + 1) * W + i] : 0.0;
        g->u[j * W + i] = dp[k] - cp[k] * next;
    }
    free(cp);
    free(dp);
}

static void std_cycle(ohier* H, int p, int q)
{
    ogrid* g = G(H, p, q);
    if (p == 1 || q == 1) { line_solve(g); return; }
    for (int k = 0; k < H->nu1; ++k) smooth_rbgs(g);
    residual(g);
    ogrid* co = G(H, p - 1, q - 1);
    memset(co->b, 0, sizeof(double) * nodes(co));
    memset(co->u, 0, sizeof(double) * nodes(co));
    for (int jc = 1; jc < co->ny; ++jc)
        for (int ic = 1; ic < co->nx; ++ic) co->b[jc * (co->nx + 1) + ic] = Rfw_at(g, g->r, ic, jc);
    for (int k = 0; k < H->mu; ++k) std_cycle(H, p - 1, q - 1);
    for (int j = 1; j < g->ny; ++j)
        for (int i = 1; i < g->nx; ++i) g->u[j * (g->nx + 1) + i] += H->omega * Pbl_at(co, co->u, i, j);
    for (int k = 0; k < H->nu2; ++k) smooth_rbgs(g);
}

/* hist[k] = ||b - A u_k||_h / ||b||_h on the finest grid after k cycles from
 * u_0 = 0 with b = 1 (hist[0] = 1); method 0: MSG (Algorithm 1 over the whole
 * hierarchy), 1: standard coarsening. */
int orc_cycle_history(ohier* H, int method, int ncycles, double* hist)
{
    ogrid* g = G(H, H->P, H->Q);
    H->Pa = H->P;
    H->Qa = H->Q;
    orc_hier_set_rhs(H, NULL);
    memset(g->u, 0, sizeof(double) * nodes(g));
    hist[0] = grid_relres(g);
    for (int k = 1; k <= ncycles; ++k) {
        if (method == 0) orc_mu_cycle(H, H->P + H->Q - 2);
        else std_cycle(H, H->P, H->Q);
        hist[k] = grid_relres(g);
    }
    return 0;
}

/* Building blocks for the pins: which 0: out = full weighting of `in` (grid
 * (p,q)) on (p-1,q-1); 1: out = bilinear interpolation of `in` (grid
 * (p-1,q-1)) on (p,q); 2: exact line solve on (p,q) with b = in, out = u. */
int orc_std_block(ohier* H, int p, int q, int which, const double* in, double* out)
{
    ogrid* g = grid_checked(H, p, q);
    if (!g) return -1;
    if (which == 2) {
        if (p != 1 && q != 1) return -1;
        memcpy(g->b, in, sizeof(double) * nodes(g));
        memset(g->u, 0, sizeof(double) * nodes(g));
        line_solve(g);
        memcpy(out, g->u, sizeof(double) * nodes(g));
        return 0;
    }
    if (p < 2 || q < 2) return -1;
    ogrid* co = G(H, p - 1, q - 1);
    if (which == 0) {
        memset(out, 0, sizeof(double) * nodes(co));
        for (int jc = 1; jc < co->ny; ++jc)
            for (int ic = 1; ic < co->nx; ++ic) out[jc * (co->nx + 1) + ic] = Rfw_at(g, in, ic, jc);
    } else {
        memset(out, 0, sizeof(double) * nodes(g));
        for (int j = 1; j < g->ny; ++j)
            for (int i = 1; i < g->nx; ++i) out[j * (g->nx + 1) + i] = Pbl_at(co, in, i, j);
    }
    return 0;
}
