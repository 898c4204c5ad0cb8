/*
 * lbib_oracle.c -- plain FP64 CPU oracle of the LB-IB-MLS adhesion step.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline of the bench).
 * It follows the paper's method in its own order and notation, one plain loop
 * per operation, no blocking or fusion.  Every function names the passage it
 * implements.  Readings of passages the paper leaves open (MLS weight, the
 * direct-forcing factor, bond anchor geometry, ...) are stated where used.
 *
 * Per time step n (weak coupling, Sec. "Fluid-structure interaction"):
 *   1. collide every node with the Guo source of f_ib^n + g      (Eq. 1, 2, 4-6)
 *   2. stream by pulling, with the wall conditions               (Eq. 1 LHS)
 *   3. hydrodynamic loads at X^n from the new populations        (Eq. 7-8)
 *   4. bond kinetics and spring forces at X^n                    (Eq. 9-11)
 *   5. wall force                                                (Eq. 12)
 *   6. rigid-body update to X^{n+1}                              (Eq. 13-16)
 *   7. IB direct forcing at X^{n+1}, MLS interpolation/spreading (Sec. "LB-IB")
 * The stored state is the post-collision population f* of the last step.
 *
 * The node loops (streaming, collision, moments) may run in parallel over
 * nodes (an OpenMP parallel for, when built with -fopenmp): every node is
 * computed by the same statements from the same inputs, so the results do
 * not depend on the thread count.
 */
#include "lbib_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- D2Q9 (Eq. 3) ------------------------------------------------------- */
static const int32_t EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int32_t EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int32_t OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

void or_lattice(int32_t *ex, int32_t *ey, double *w, int32_t *opp) {
    for (int i = 0; i < 9; ++i) {
        ex[i] = EX[i];
        ey[i] = EY[i];
        w[i] = W[i];
        opp[i] = OPP[i];
    }
}

/* Eq. 2 with c_s^2 = 1/3: 1/c_s^2 = 3, 1/(2 c_s^4) = 4.5, 1/(2 c_s^2) = 1.5. */
void or_equilibrium(double rho, double ux, double uy, double *feq) {
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        feq[i] = W[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Eq. 4: F_i = (1 - 1/(2 tau)) w_i [ (e_i - u)/c_s^2 + (e_i.u) e_i / c_s^4 ] . F */
void or_guo_source(double tau, double ux, double uy, double Fx, double Fy, double *S) {
    double pref = 1.0 - 0.5 / tau;
    for (int i = 0; i < 9; ++i) {
        double eu = EX[i] * ux + EY[i] * uy;
        double cx = 3.0 * (EX[i] - ux) + 9.0 * eu * EX[i];
        double cy = 3.0 * (EY[i] - uy) + 9.0 * eu * EY[i];
        S[i] = pref * W[i] * (cx * Fx + cy * Fy);
    }
}

/* Eq. 1 right-hand side with the forcing term, moments by Eq. 5-6. */
void or_collide_node(const double *f, double tau, double Fx, double Fy, double *fpost) {
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += f[i] * EX[i];
        jy += f[i] * EY[i];
    }
    double ux = (jx + 0.5 * Fx) / rho;
    double uy = (jy + 0.5 * Fy) / rho;
    double feq[9], S[9];
    or_equilibrium(rho, ux, uy, feq);
    or_guo_source(tau, ux, uy, Fx, Fy, S);
    for (int i = 0; i < 9; ++i) fpost[i] = f[i] - (f[i] - feq[i]) / tau + S[i];
}

/* ---- simulation state --------------------------------------------------- */
typedef struct or_particle {
    int nv, fixed;
    double *vx, *vy;
    uint8_t *ligand, *bond;
    double *anchor_x;
    int8_t *anchor_wall;            /* 0 bottom, 1 top */
    double xc, yc, theta, u, v, omega;
    double xc1, yc1, theta1, u1, v1, omega1; /* values one step earlier */
    double sigma, area, mass, inertia, r_eq;
    double Fh[2], Mh, Fb[2], Mb, Fw[2];
    int n_ligands, n_probing, n_bonded;
    /* near-tie diagnostics of the last bond step (they change no result):
     * the smallest |U - P| over the draws compared with a probability, and
     * the smallest |gap - y_cr| over the ligands' probing tests */
    double margin_p, margin_gap;
    double gap[2];                  /* smallest element gaps to the wall lines */
} or_particle;

struct or_sim {
    or_config c;
    double *fpost, *fpre;    /* [9][ny][nx] */
    double *fibx, *fiby;     /* IB force density of the current step */
    int np, cap;
    or_particle *p;
    int64_t step;
    int primed;
};

static size_t NN(const or_sim *s) { return (size_t)s->c.nx * (size_t)s->c.ny; }
static int imod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

or_sim *or_create(const or_config *cfg) {
    if (!cfg || cfg->nx < 8 || cfg->ny < 4 || !(cfg->tau > 0.5)) return NULL;
    if ((cfg->wall_bottom == OR_WALL_PERIODIC) != (cfg->wall_top == OR_WALL_PERIODIC))
        return NULL;
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    s->c = *cfg;
    size_t n = NN(s);
    s->fpost = (double *)malloc(9 * n * sizeof(double));
    s->fpre = (double *)malloc(9 * n * sizeof(double));
    s->fibx = (double *)calloc(n, sizeof(double));
    s->fiby = (double *)calloc(n, sizeof(double));
    /* default initial state: f* = f^eq(rho = 1, u = 0) */
    for (int i = 0; i < 9; ++i)
        for (size_t k = 0; k < n; ++k) s->fpost[i * n + k] = W[i];
    return s;
}

void or_destroy(or_sim *s) {
    if (!s) return;
    for (int k = 0; k < s->np; ++k) {
        or_particle *p = &s->p[k];
        free(p->vx); free(p->vy); free(p->ligand); free(p->bond);
        free(p->anchor_x); free(p->anchor_wall);
    }
    free(s->p);
    free(s->fpost); free(s->fpre); free(s->fibx); free(s->fiby);
    free(s);
}

int or_set_populations(or_sim *s, const double *f_post) {
    if (!s || s->step != 0) return -1;
    memcpy(s->fpost, f_post, 9 * NN(s) * sizeof(double));
    s->primed = 0;
    return 0;
}

int or_get_populations(const or_sim *s, double *f_post) {
    memcpy(f_post, s->fpost, 9 * NN(s) * sizeof(double));
    return 0;
}

int64_t or_step_count(const or_sim *s) { return s->step; }

/* ---- particle geometry (Sec. "Pressure and viscous stresses") ----------- */
/* Element l joins vertex l to vertex l+1; its centroid is the midpoint, its
 * length S_l, and for a counter-clockwise polygon the outward normal is the
 * edge direction turned clockwise. */
void or_elements(int nv, const double *vx, const double *vy, double xc, double yc,
                 double theta, double *mx, double *my, double *nxo, double *nyo,
                 double *S) {
    double c = cos(theta), s = sin(theta);
    for (int l = 0; l < nv; ++l) {
        int m = (l + 1) % nv;
        double ax = xc + c * vx[l] - s * vy[l];
        double ay = yc + s * vx[l] + c * vy[l];
        double bx = xc + c * vx[m] - s * vy[m];
        double by = yc + s * vx[m] + c * vy[m];
        double dx = bx - ax, dy = by - ay;
        double len = sqrt(dx * dx + dy * dy);
        mx[l] = 0.5 * (ax + bx);
        my[l] = 0.5 * (ay + by);
        S[l] = len;
        nxo[l] = dy / len;
        nyo[l] = -dx / len;
    }
}

int or_add_particle(or_sim *s, const or_particle_in *in) {
    if (!s || !in || in->n_vertices < 3 || s->step != 0) return -1;
    if (s->np == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 4;
        s->p = (or_particle *)realloc(s->p, (size_t)s->cap * sizeof(or_particle));
    }
    or_particle *p = &s->p[s->np];
    memset(p, 0, sizeof(*p));
    int nv = in->n_vertices;
    p->nv = nv;
    p->fixed = in->fixed;
    p->vx = (double *)malloc(nv * sizeof(double));
    p->vy = (double *)malloc(nv * sizeof(double));
    memcpy(p->vx, in->vx, nv * sizeof(double));
    memcpy(p->vy, in->vy, nv * sizeof(double));
    p->ligand = (uint8_t *)calloc(nv, 1);
    p->bond = (uint8_t *)calloc(nv, 1);
    p->anchor_x = (double *)calloc(nv, sizeof(double));
    p->anchor_wall = (int8_t *)calloc(nv, 1);
    /* ligands spread evenly along the perimeter with density rho_l: element l
     * carries one when floor((l+1) rho_l) exceeds floor(l rho_l). */
    for (int l = 0; l < nv; ++l) {
        double a = floor((double)(l + 1) * in->ligand_density);
        double b = floor((double)l * in->ligand_density);
        p->ligand[l] = a > b;
        p->n_ligands += p->ligand[l];
    }
    /* area and polar moment of the polygon about its centroid (the origin of
     * the body frame); mass = rho_p * area, r = sqrt(area / pi) in Eq. 12 */
    double A = 0.0, J = 0.0;
    for (int l = 0; l < nv; ++l) {
        int m = (l + 1) % nv;
        double x0 = p->vx[l], y0 = p->vy[l], x1 = p->vx[m], y1 = p->vy[m];
        double cr = x0 * y1 - x1 * y0;
        A += 0.5 * cr;
        J += cr * (x0 * x0 + x0 * x1 + x1 * x1 + y0 * y0 + y0 * y1 + y1 * y1) / 12.0;
    }
    p->area = A;
    p->mass = in->rho_p * A;
    p->inertia = in->rho_p * J;
    p->r_eq = sqrt(A / M_PI);
    p->sigma = in->sigma;
    p->margin_p = p->margin_gap = INFINITY;
    p->gap[0] = p->gap[1] = INFINITY;
    p->xc = p->xc1 = in->xc;
    p->yc = p->yc1 = in->yc;
    p->theta = p->theta1 = in->theta;
    s->primed = 0;
    return s->np++;
}

/* ---- streaming with wall conditions (Eq. 1 LHS; walls Sec. "LB-IB") ------ */
/* Half-way bounce-back with a moving wall: a population arriving from behind
 * the wall is the node's own opposite post-collision value plus
 * 6 w_i rho_w (e_i . u_w), rho_w = 1.  Zou-He known-velocity walls (the
 * paper's wall treatment) rebuild the three unknown populations of the wall
 * row from the known ones and the wall velocity (u_w, 0). */
static void zou_he_bottom(double *f, double uw) {
    double rho = f[0] + f[1] + f[3] + 2.0 * (f[4] + f[7] + f[8]);
    f[2] = f[4];
    f[5] = f[7] - 0.5 * (f[1] - f[3]) + 0.5 * rho * uw;
    f[6] = f[8] + 0.5 * (f[1] - f[3]) - 0.5 * rho * uw;
}
static void zou_he_top(double *f, double uw) {
    double rho = f[0] + f[1] + f[3] + 2.0 * (f[2] + f[5] + f[6]);
    f[4] = f[2];
    f[7] = f[5] + 0.5 * (f[1] - f[3]) - 0.5 * rho * uw;
    f[8] = f[6] - 0.5 * (f[1] - f[3]) + 0.5 * rho * uw;
}

static void stream(or_sim *s) {
    const or_config *c = &s->c;
    int nx = c->nx, ny = c->ny;
    size_t n = NN(s);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double f[9];
            for (int i = 0; i < 9; ++i) {
                int xs = imod(x - EX[i], nx);
                int ys = y - EY[i];
                if (ys < 0 || ys >= ny) {
                    int wall = ys < 0 ? c->wall_bottom : c->wall_top;
                    double uw = ys < 0 ? c->u_bottom : c->u_top;
                    if (wall == OR_WALL_PERIODIC) {
                        ys = imod(ys, ny);
                        f[i] = s->fpost[i * n + (size_t)ys * nx + xs];
                    } else if (wall == OR_WALL_BOUNCE_BACK) {
                        f[i] = s->fpost[OPP[i] * n + (size_t)y * nx + x] +
                               6.0 * W[i] * (EX[i] * uw);
                    } else {
                        f[i] = 0.0; /* rebuilt by Zou-He below */
                    }
                } else {
                    f[i] = s->fpost[i * n + (size_t)ys * nx + xs];
                }
            }
            if (y == 0 && c->wall_bottom == OR_WALL_ZOU_HE) zou_he_bottom(f, c->u_bottom);
            if (y == ny - 1 && c->wall_top == OR_WALL_ZOU_HE) zou_he_top(f, c->u_top);
            for (int i = 0; i < 9; ++i) s->fpre[i * n + (size_t)y * nx + x] = f[i];
        }
}

static void collide(or_sim *s) {
    size_t n = NN(s);
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < n; ++k) {
        double f[9], fp[9];
        for (int i = 0; i < 9; ++i) f[i] = s->fpre[i * n + k];
        or_collide_node(f, s->c.tau, s->fibx[k] + s->c.gx, s->fiby[k] + s->c.gy, fp);
        for (int i = 0; i < 9; ++i) s->fpost[i * n + k] = fp[i];
    }
}

/* ---- moving least squares (Sec. "LB-IB", refs [13], [39]) ---------------- */
/* Reading: linear basis p = (1, x - X, y - Y); tensor-product cubic B-spline
 * weight with radius 2 per axis; support = the 4 x 4 nodes floor(X)-1 ..
 * floor(X)+2 in each direction (periodic in x, and in y for periodic walls),
 * limited in y to the lattice rows 0..ny-1 (Zou-He wall nodes are nodes of
 * the fluid domain and stay in the support, so a marker between the wall
 * row and row 1 is interpolated, not extrapolated).  A support with fewer
 * than two rows or two columns of non-zero weight cannot carry a linear fit
 * and yields no nodes. */
double or_weight(double r) {
    double a = fabs(r);
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) {
        double b = 2.0 - a;
        return b * b * b / 6.0;
    }
    return 0.0;
}

static void row_limits(const or_config *c, int *lo, int *hi) {
    *lo = 0;
    *hi = c->ny - 1;
}

/* Wall lines: y = 0 and ny - 1 for Zou-He (wall nodes), -1/2 and ny - 1/2 for
 * half-way bounce-back. */
static double wall_line(const or_config *c, int top) {
    int kind = top ? c->wall_top : c->wall_bottom;
    double y = top ? (double)(c->ny - 1) : 0.0;
    if (kind == OR_WALL_BOUNCE_BACK) y += top ? 0.5 : -0.5;
    return y;
}

/* Gaussian elimination with partial pivoting on a 3x3 system. */
static int solve3(const double A[3][3], const double *b, double *x) {
    double M[3][4];
    for (int r = 0; r < 3; ++r) {
        for (int q = 0; q < 3; ++q) M[r][q] = A[r][q];
        M[r][3] = b[r];
    }
    for (int k = 0; k < 3; ++k) {
        int piv = k;
        for (int r = k + 1; r < 3; ++r)
            if (fabs(M[r][k]) > fabs(M[piv][k])) piv = r;
        if (M[piv][k] == 0.0) return -1;
        if (piv != k)
            for (int q = 0; q < 4; ++q) {
                double t = M[k][q];
                M[k][q] = M[piv][q];
                M[piv][q] = t;
            }
        for (int r = k + 1; r < 3; ++r) {
            double m = M[r][k] / M[k][k];
            for (int q = k; q < 4; ++q) M[r][q] -= m * M[k][q];
        }
    }
    for (int k = 2; k >= 0; --k) {
        double acc = M[k][3];
        for (int q = k + 1; q < 3; ++q) acc -= M[k][q] * x[q];
        x[k] = acc / M[k][k];
    }
    return 0;
}

/* Support nodes, weights and basis offsets of a point; returns the count. */
static int mls_support(const or_config *c, double X, double Y, int32_t *ix, int32_t *iy,
                       double *wk, double *dxk, double *dyk) {
    int lo, hi;
    row_limits(c, &lo, &hi);
    int periodic_y = c->wall_bottom == OR_WALL_PERIODIC;
    /* a point beyond a wall line (a probe or marker of a particle pressed
     * against the wall) is outside the fluid: no fit (reading of the paper,
     * which places probes 1.2 dx along the normal without saying what happens
     * at a wall) */
    if (!periodic_y && (Y < wall_line(c, 0) || Y > wall_line(c, 1))) return 0;
    int x0 = (int)floor(X) - 1, y0 = (int)floor(Y) - 1;
    int nrow = 0, ncol = 0, n = 0;
    for (int a = 0; a < 4; ++a)
        if (fabs((double)(x0 + a) - X) < 2.0) ++ncol;
    for (int b = 0; b < 4; ++b) {
        int yy = y0 + b;
        if (!periodic_y && (yy < lo || yy > hi)) continue;
        if (fabs((double)yy - Y) < 2.0) ++nrow;
    }
    if (nrow < 2 || ncol < 2) return 0;
    for (int b = 0; b < 4; ++b) {
        int yy = y0 + b;
        if (!periodic_y && (yy < lo || yy > hi)) continue;
        for (int a = 0; a < 4; ++a) {
            int xx = x0 + a;
            double dx = (double)xx - X, dy = (double)yy - Y;
            ix[n] = imod(xx, c->nx);
            iy[n] = periodic_y ? imod(yy, c->ny) : yy;
            dxk[n] = dx;
            dyk[n] = dy;
            wk[n] = or_weight(dx) * or_weight(dy);
            ++n;
        }
    }
    return n;
}

static void mls_matrix(int n, const double *wk, const double *dxk, const double *dyk,
                       double A[3][3]) {
    memset(A, 0, 9 * sizeof(double));
    for (int k = 0; k < n; ++k) {
        double p[3] = {1.0, dxk[k], dyk[k]};
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) A[r][q] += wk[k] * p[r] * p[q];
    }
}

/* phi_k(X) = p(X)^T A^{-1} w_k p(x_k); with p(X) = (1, 0, 0) this is w_k
 * times the first component of A^{-1} p_k. */
int or_mls_shape(const or_config *c, double X, double Y, int32_t *ix, int32_t *iy,
                 double *phi) {
    double wk[16], dxk[16], dyk[16], A[3][3];
    int n = mls_support(c, X, Y, ix, iy, wk, dxk, dyk);
    if (n == 0) return 0;
    mls_matrix(n, wk, dxk, dyk, A);
    for (int k = 0; k < n; ++k) {
        double p[3] = {1.0, dxk[k], dyk[k]}, z[3];
        if (solve3(A, p, z) != 0) return 0;
        phi[k] = wk[k] * z[0];
    }
    return n;
}

/* Local weighted least-squares fit a = A^{-1} sum_k w_k p_k u_k; a_0 is the
 * value at (X, Y), (a_1, a_2) the diffuse gradient. */
int or_mls_fit(const or_config *c, const double *field, double X, double Y,
               double *value, double *ddx, double *ddy) {
    int32_t ix[16], iy[16];
    double wk[16], dxk[16], dyk[16], A[3][3], b[3] = {0, 0, 0}, a[3];
    int n = mls_support(c, X, Y, ix, iy, wk, dxk, dyk);
    *value = *ddx = *ddy = 0.0;
    if (n == 0) return 0;
    mls_matrix(n, wk, dxk, dyk, A);
    for (int k = 0; k < n; ++k) {
        double u = field[(size_t)iy[k] * c->nx + ix[k]];
        b[0] += wk[k] * u;
        b[1] += wk[k] * dxk[k] * u;
        b[2] += wk[k] * dyk[k] * u;
    }
    if (solve3(A, b, a) != 0) return 0;
    *value = a[0];
    *ddx = a[1];
    *ddy = a[2];
    return n;
}

void or_interp(const or_config *c, const double *field, int n, const double *X,
               const double *Y, double *out) {
    for (int l = 0; l < n; ++l) {
        int32_t ix[16], iy[16];
        double phi[16];
        int m = or_mls_shape(c, X[l], Y[l], ix, iy, phi);
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc += phi[k] * field[(size_t)iy[k] * c->nx + ix[k]];
        out[l] = acc;
    }
}

/* f_ib(x_k) += phi_k(X_l) F_l eps_l, the transpose of the interpolation. */
void or_spread(const or_config *c, int n, const double *X, const double *Y,
               const double *Fx, const double *Fy, const double *eps, double *fx,
               double *fy) {
    for (int l = 0; l < n; ++l) {
        int32_t ix[16], iy[16];
        double phi[16];
        int m = or_mls_shape(c, X[l], Y[l], ix, iy, phi);
        for (int k = 0; k < m; ++k) {
            size_t q = (size_t)iy[k] * c->nx + ix[k];
            fx[q] += phi[k] * Fx[l] * eps[l];
            fy[q] += phi[k] * Fy[l] * eps[l];
        }
    }
}

/* Solved spreading scales (Vanella & Balaras, ref. [39], cited with the MLS
 * transfer in Sec. "The combined LB-IB method").  Reading: eps is chosen so
 * that the MLS interpolation at the markers of the field spread from a
 * uniform marker force returns that force, i.e. sum_m A_lm eps_m = 1 with
 * A_lm = sum_k phi_k(X_l) phi_k(X_m) over the lattice nodes k.  The dense
 * system is solved by Gaussian elimination with partial pivoting; a marker
 * without a fit (no support) is left out (eps = 0, identity row). */
int or_vb_eps(const or_config *c, int n, const double *X, const double *Y, double *eps) {
    int32_t *ix = (int32_t *)malloc((size_t)n * 16 * 2 * sizeof(int32_t));
    int32_t *iy = ix + (size_t)n * 16;
    double *phi = (double *)malloc((size_t)n * 16 * sizeof(double));
    int *cnt = (int *)malloc((size_t)n * sizeof(int));
    double *M = (double *)calloc((size_t)n * (n + 1), sizeof(double));
    for (int l = 0; l < n; ++l)
        cnt[l] = or_mls_shape(c, X[l], Y[l], ix + 16 * l, iy + 16 * l, phi + 16 * l);
    /* augmented matrix [A | 1] */
    for (int l = 0; l < n; ++l) {
        double *row = M + (size_t)l * (n + 1);
        if (cnt[l] == 0) {
            row[l] = 1.0;
            continue;
        }
        for (int m = 0; m < n; ++m) {
            double a = 0.0;
            for (int i = 0; i < cnt[l]; ++i)
                for (int j = 0; j < cnt[m]; ++j)
                    if (ix[16 * l + i] == ix[16 * m + j] && iy[16 * l + i] == iy[16 * m + j])
                        a += phi[16 * l + i] * phi[16 * m + j];
            row[m] = a;
        }
        row[n] = 1.0;
    }
    int ok = 0;
    for (int k = 0; k < n && ok == 0; ++k) {
        int piv = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(M[(size_t)r * (n + 1) + k]) > fabs(M[(size_t)piv * (n + 1) + k])) piv = r;
        if (M[(size_t)piv * (n + 1) + k] == 0.0) {
            ok = -1;
            break;
        }
        if (piv != k)
            for (int q = 0; q <= n; ++q) {
                double t = M[(size_t)k * (n + 1) + q];
                M[(size_t)k * (n + 1) + q] = M[(size_t)piv * (n + 1) + q];
                M[(size_t)piv * (n + 1) + q] = t;
            }
        for (int r = k + 1; r < n; ++r) {
            double f = M[(size_t)r * (n + 1) + k] / M[(size_t)k * (n + 1) + k];
            if (f == 0.0) continue;
            for (int q = k; q <= n; ++q) M[(size_t)r * (n + 1) + q] -= f * M[(size_t)k * (n + 1) + q];
        }
    }
    if (ok == 0)
        for (int k = n - 1; k >= 0; --k) {
            double acc = M[(size_t)k * (n + 1) + n];
            for (int q = k + 1; q < n; ++q) acc -= M[(size_t)k * (n + 1) + q] * eps[q];
            eps[k] = acc / M[(size_t)k * (n + 1) + k];
        }
    for (int l = 0; l < n; ++l)
        if (cnt[l] == 0) eps[l] = 0.0;
    free(M);
    free(cnt);
    free(phi);
    free(ix);
    return ok;
}

/* ---- hydrodynamic loads (Eq. 7-8) --------------------------------------- */
/* Probe Q_l = X_l + 1.2 n_l; p and the velocity gradient come from the MLS
 * fit there and are taken as the centroid's.  Reading: pressure relative to
 * the reference state, p = c_s^2 (rho - 1); viscous stress
 * nu (grad u + grad u^T) with rho_ref = 1; the load on the body is
 * sum_l (-p n_l + tau_l . n_l) S_l and the moment sum_l r_l x (t_l S_l). */
void or_loads(const or_config *c, const double *rho, const double *ux, const double *uy,
              int nv, const double *vx, const double *vy, double xc, double yc,
              double theta, double *out) {
    double *mx = (double *)malloc(5 * nv * sizeof(double));
    double *my = mx + nv, *nxo = my + nv, *nyo = nxo + nv, *S = nyo + nv;
    or_elements(nv, vx, vy, xc, yc, theta, mx, my, nxo, nyo, S);
    double nu = (c->tau - 0.5) / 3.0;
    double Fx = 0.0, Fy = 0.0, M = 0.0;
    for (int l = 0; l < nv; ++l) {
        double qx = mx[l] + 1.2 * nxo[l], qy = my[l] + 1.2 * nyo[l];
        double r, drx, dry, a, dudx, dudy, b, dvdx, dvdy;
        /* a probe whose support cannot carry a linear fit (inside a wall)
         * contributes no traction */
        if (or_mls_fit(c, rho, qx, qy, &r, &drx, &dry) == 0) continue;
        or_mls_fit(c, ux, qx, qy, &a, &dudx, &dudy);
        or_mls_fit(c, uy, qx, qy, &b, &dvdx, &dvdy);
        double p = (r - 1.0) / 3.0;
        double txx = nu * 2.0 * dudx, tyy = nu * 2.0 * dvdy, txy = nu * (dudy + dvdx);
        double tx = -p * nxo[l] + txx * nxo[l] + txy * nyo[l];
        double ty = -p * nyo[l] + txy * nxo[l] + tyy * nyo[l];
        Fx += tx * S[l];
        Fy += ty * S[l];
        M += ((mx[l] - xc) * ty - (my[l] - yc) * tx) * S[l];
    }
    out[0] = Fx;
    out[1] = Fy;
    out[2] = M;
    free(mx);
}

/* ---- Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------- */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* One uniform per (sim, step, particle, element): key = (seed, sim_id),
 * counter = (step, particle << 32 | element, 0, 0); U = top 53 bits of the
 * first output word times 2^-53, in [0, 1). */
double or_uniform(uint64_t seed, uint64_t sim_id, int64_t step, int32_t pid, int32_t l) {
    uint64_t key[2] = {seed, sim_id};
    uint64_t ctr[4] = {(uint64_t)step, ((uint64_t)(uint32_t)pid << 32) | (uint32_t)l, 0, 0};
    uint64_t out[4];
    or_philox4x64(ctr, key, out);
    return (double)(out[0] >> 11) * (1.0 / 9007199254740992.0);
}

/* ---- bond kinetics (Eq. 9-11) ------------------------------------------- */
/* Eq. 10 with dt = 1. */
double or_prob_forward(double k_f, double Nl) { return 1.0 - exp(-k_f * Nl); }

/* Eq. 11 with dt = 1. */
double or_prob_reverse(double k_r0, double sigma, double sigma_star, double y,
                       double y_eq, double kBT) {
    double d = y - y_eq;
    double kr = k_r0 * exp((sigma - sigma_star) * d * d / (2.0 * kBT));
    return 1.0 - exp(-kr);
}

static void wall_lines(const or_config *c, double *yb, double *yt) {
    *yb = c->wall_bottom == OR_WALL_BOUNCE_BACK ? -0.5 : 0.0;
    *yt = c->wall_top == OR_WALL_BOUNCE_BACK ? (double)c->ny - 0.5 : (double)(c->ny - 1);
}

/* Reading of Eq. 9-11: a ligand probes a receptor wall when its element
 * centroid is closer to that wall than y_cr; N_l = probing ligands / nl.  A
 * free probing ligand binds when U < P_f (forward rate scaled by the wall's
 * receptor density) and anchors at (x_l, y_wall); a bound ligand breaks when
 * U < P_r with y_l = |anchor - X_l|.  One uniform per ligand and step.  The
 * spring of every bond present after the update pulls X_l along the unit
 * vector towards the anchor with magnitude sigma (y_l - y_eq). */
static void bonds(or_sim *s, int pid, const double *mx, const double *my) {
    const or_config *c = &s->c;
    or_particle *p = &s->p[pid];
    double yb, yt;
    wall_lines(c, &yb, &yt);
    int has_b = c->wall_bottom != OR_WALL_PERIODIC && c->receptor_bottom > 0.0;
    int has_t = c->wall_top != OR_WALL_PERIODIC && c->receptor_top > 0.0;
    double y_eq = c->y_eq_ratio * c->y_cr;
    double sigma_star = c->sigma_star_ratio * p->sigma;
    double mp = INFINITY, mg = INFINITY;
    int nprobe = 0;
    for (int l = 0; l < p->nv; ++l) {
        if (!p->ligand[l]) continue;
        int pb = has_b && (my[l] - yb) < c->y_cr;
        int pt = has_t && (yt - my[l]) < c->y_cr;
        nprobe += (pb || pt);
        if (has_b) mg = fmin(mg, fabs((my[l] - yb) - c->y_cr));
        if (has_t) mg = fmin(mg, fabs((yt - my[l]) - c->y_cr));
    }
    double Nl = (double)nprobe / (double)p->nv;
    for (int l = 0; l < p->nv; ++l) {
        if (!p->ligand[l]) continue;
        double U = or_uniform(c->seed, c->sim_id, s->step, pid, l);
        if (p->bond[l]) {
            double wy = p->anchor_wall[l] ? yt : yb;
            double dx = p->anchor_x[l] - mx[l], dy = wy - my[l];
            double y = sqrt(dx * dx + dy * dy);
            double Pr = or_prob_reverse(c->k_r0, p->sigma, sigma_star, y, y_eq, c->kBT);
            mp = fmin(mp, fabs(U - Pr));
            if (U < Pr) p->bond[l] = 0;
        } else {
            int pb = has_b && (my[l] - yb) < c->y_cr;
            int pt = has_t && (yt - my[l]) < c->y_cr;
            if (pb || pt) {
                double dens = pb ? c->receptor_bottom : c->receptor_top;
                double Pf = or_prob_forward(c->k_f * dens, Nl);
                mp = fmin(mp, fabs(U - Pf));
                if (U < Pf) {
                    p->bond[l] = 1;
                    p->anchor_x[l] = mx[l];
                    p->anchor_wall[l] = pb ? 0 : 1;
                }
            }
        }
    }
    double Fx = 0.0, Fy = 0.0, M = 0.0;
    int nb = 0;
    for (int l = 0; l < p->nv; ++l) {
        if (!p->bond[l]) continue;
        double wy = p->anchor_wall[l] ? yt : yb;
        double dx = p->anchor_x[l] - mx[l], dy = wy - my[l];
        double y = sqrt(dx * dx + dy * dy);
        double fx = 0.0, fy = 0.0;
        if (y > 0.0) {
            double mag = p->sigma * (y - y_eq);
            fx = mag * dx / y;
            fy = mag * dy / y;
        }
        Fx += fx;
        Fy += fy;
        M += (mx[l] - p->xc) * fy - (my[l] - p->yc) * fx;
        ++nb;
    }
    p->Fb[0] = Fx;
    p->Fb[1] = Fy;
    p->Mb = M;
    p->n_probing = nprobe;
    p->n_bonded = nb;
    p->margin_p = mp;
    p->margin_gap = mg;
}

/* Eq. 12: F_w = H_k / (8 sqrt 2) sqrt(r / eps^5) along the wall normal into
 * the fluid, applied at the centroid.  Reading: eps is the smallest
 * centroid-to-wall gap of the elements, clamped below by eps_min. */
static void wall_force(or_sim *s, int pid, const double *my) {
    const or_config *c = &s->c;
    or_particle *p = &s->p[pid];
    p->Fw[0] = p->Fw[1] = 0.0;
    p->gap[0] = p->gap[1] = INFINITY;
    if (c->wall_bottom == OR_WALL_PERIODIC) return;
    double yb, yt;
    wall_lines(c, &yb, &yt);
    double eb = 1e300, et = 1e300;
    for (int l = 0; l < p->nv; ++l) {
        if (my[l] - yb < eb) eb = my[l] - yb;
        if (yt - my[l] < et) et = yt - my[l];
    }
    p->gap[0] = eb;
    p->gap[1] = et;
    if (c->hamaker == 0.0) return;
    if (eb < c->eps_min) eb = c->eps_min;
    if (et < c->eps_min) et = c->eps_min;
    double k = c->hamaker / (8.0 * sqrt(2.0));
    p->Fw[1] = k * sqrt(p->r_eq / pow(eb, 5.0)) - k * sqrt(p->r_eq / pow(et, 5.0));
}

/* Eq. 15-16: u^n = 2/3 (2 u^{n-1} - u^{n-2}/2 + du/dt dt), dt = 1. */
double or_bdf2_velocity(double u1, double u2, double acc) {
    return 2.0 / 3.0 * (2.0 * u1 - 0.5 * u2 + acc);
}
/* Reading: the pose follows the same second-order backward form,
 * x^n = (4 x^{n-1} - x^{n-2} + 2 dt u^n) / 3. */
double or_bdf2_position(double x1, double x2, double u_new) {
    return (4.0 * x1 - x2 + 2.0 * u_new) / 3.0;
}

static void rigid_update(or_particle *p) {
    if (p->fixed) return;
    double Fx = p->Fh[0] + p->Fb[0] + p->Fw[0];
    double Fy = p->Fh[1] + p->Fb[1] + p->Fw[1];
    double M = p->Mh + p->Mb;
    double un = or_bdf2_velocity(p->u, p->u1, Fx / p->mass);       /* Eq. 13, 15 */
    double vn = or_bdf2_velocity(p->v, p->v1, Fy / p->mass);
    double wn = or_bdf2_velocity(p->omega, p->omega1, M / p->inertia); /* Eq. 14, 16 */
    double xn = or_bdf2_position(p->xc, p->xc1, un);
    double yn = or_bdf2_position(p->yc, p->yc1, vn);
    double tn = or_bdf2_position(p->theta, p->theta1, wn);
    p->u1 = p->u; p->v1 = p->v; p->omega1 = p->omega;
    p->u = un; p->v = vn; p->omega = wn;
    p->xc1 = p->xc; p->yc1 = p->yc; p->theta1 = p->theta;
    p->xc = xn; p->yc = yn; p->theta = tn;
}

/* Nodal rho and velocity of f_pre; with_force adds g/2 (the IB uses
 * u* = (sum f e + g/2) / rho, the velocity before its own force). */
static void moments(const or_sim *s, double *rho, double *ux, double *uy, double addx,
                    double addy) {
    size_t n = NN(s);
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < n; ++k) {
        double r = 0.0, jx = 0.0, jy = 0.0;
        for (int i = 0; i < 9; ++i) {
            double f = s->fpre[i * n + k];
            r += f;
            jx += f * EX[i];
            jy += f * EY[i];
        }
        rho[k] = r;
        ux[k] = (jx + addx) / r;
        uy[k] = (jy + addy) / r;
    }
}

/* IB direct forcing (Favier et al. [38] with MLS [13], [39]).  Reading: the
 * desired marker velocity is the rigid motion U_c + omega x (X_l - X_c); the
 * force density that makes the Guo half-step velocity u* + F/(2 rho) match it
 * is F_l = 2 rho_l (U^d_l - u*_l) / dt; spread with eps_l = S_l dx, or with
 * the solved scales of or_vb_eps when ib_spread = 1.
 * Multi-direct forcing (ib_iterations = M > 1): the velocity a marker sees
 * after its own particle's force is spread, u^m_l = u*_l + I_l[f^(m-1)] /
 * (2 rho_l) (I_l: the MLS interpolation at X_l, rho_l the marker's
 * interpolated density), is corrected again, F^m_l = F^(m-1)_l +
 * 2 rho_l (U^d_l - u^m_l) = F^(m-1)_l + F^0_l - I_l[f^(m-1)], for
 * m = 1 .. M-1, and F^(M-1) is spread.  Each particle iterates against its
 * own spread force only. */
static void ib_force(or_sim *s) {
    size_t n = NN(s);
    memset(s->fibx, 0, n * sizeof(double));
    memset(s->fiby, 0, n * sizeof(double));
    if (s->np == 0) return;
    double *rho = (double *)malloc(3 * n * sizeof(double));
    double *ux = rho + n, *uy = ux + n;
    moments(s, rho, ux, uy, 0.5 * s->c.gx, 0.5 * s->c.gy);
    for (int k = 0; k < s->np; ++k) {
        or_particle *p = &s->p[k];
        int nv = p->nv;
        double *buf = (double *)malloc(11 * nv * sizeof(double));
        double *mx = buf, *my = mx + nv, *nxo = my + nv, *nyo = nxo + nv, *S = nyo + nv;
        double *rl = S + nv, *ul = rl + nv, *vl = ul + nv, *Fx = vl + nv, *Fy = Fx + nv;
        or_elements(nv, p->vx, p->vy, p->xc, p->yc, p->theta, mx, my, nxo, nyo, S);
        if (s->c.ib_spread == 1) {
            /* the spreading scales replace the element lengths (S is not
             * used for anything else here) */
            double *eps = (double *)malloc(nv * sizeof(double));
            if (or_vb_eps(&s->c, nv, mx, my, eps) == 0) memcpy(S, eps, nv * sizeof(double));
            free(eps);
        }
        or_interp(&s->c, rho, nv, mx, my, rl);
        or_interp(&s->c, ux, nv, mx, my, ul);
        or_interp(&s->c, uy, nv, mx, my, vl);
        for (int l = 0; l < nv; ++l) {
            double udx = p->u - p->omega * (my[l] - p->yc);
            double udy = p->v + p->omega * (mx[l] - p->xc);
            Fx[l] = 2.0 * rl[l] * (udx - ul[l]);
            Fy[l] = 2.0 * rl[l] * (udy - vl[l]);
        }
        if (s->c.ib_iterations > 1) {
            /* F^0 kept in rl / ul (no longer needed), the particle's own
             * spread field in tx / ty */
            double *tx = (double *)malloc(2 * n * sizeof(double)), *ty = tx + n;
            double *Ix = (double *)malloc(2 * nv * sizeof(double)), *Iy = Ix + nv;
            for (int l = 0; l < nv; ++l) {
                rl[l] = Fx[l];
                ul[l] = Fy[l];
            }
            for (int m = 1; m < s->c.ib_iterations; ++m) {
                memset(tx, 0, 2 * n * sizeof(double));
                or_spread(&s->c, nv, mx, my, Fx, Fy, S, tx, ty);
                or_interp(&s->c, tx, nv, mx, my, Ix);
                or_interp(&s->c, ty, nv, mx, my, Iy);
                for (int l = 0; l < nv; ++l) {
                    Fx[l] = Fx[l] + rl[l] - Ix[l];
                    Fy[l] = Fy[l] + ul[l] - Iy[l];
                }
            }
            free(Ix);
            free(tx);
        }
        or_spread(&s->c, nv, mx, my, Fx, Fy, S, s->fibx, s->fiby);
        free(buf);
    }
    free(rho);
}

static void prime(or_sim *s) {
    if (s->primed) return;
    stream(s);
    ib_force(s);
    s->primed = 1;
}

static void particles_after_stream(or_sim *s) {
    if (s->np == 0) return;
    size_t n = NN(s);
    double *rho = (double *)malloc(3 * n * sizeof(double));
    double *ux = rho + n, *uy = ux + n;
    moments(s, rho, ux, uy, 0.0, 0.0);
    for (int k = 0; k < s->np; ++k) {
        or_particle *p = &s->p[k];
        int nv = p->nv;
        double out[3];
        or_loads(&s->c, rho, ux, uy, nv, p->vx, p->vy, p->xc, p->yc, p->theta, out);
        p->Fh[0] = out[0];
        p->Fh[1] = out[1];
        p->Mh = out[2];
        double *buf = (double *)malloc(5 * nv * sizeof(double));
        double *mx = buf, *my = mx + nv, *nxo = my + nv, *nyo = nxo + nv, *S = nyo + nv;
        or_elements(nv, p->vx, p->vy, p->xc, p->yc, p->theta, mx, my, nxo, nyo, S);
        bonds(s, k, mx, my);
        wall_force(s, k, my);
        free(buf);
        rigid_update(p);
    }
    free(rho);
}

int or_step(or_sim *s, int64_t nsteps) {
    if (!s || nsteps < 0) return -1;
    prime(s);
    for (int64_t t = 0; t < nsteps; ++t) {
        collide(s);
        stream(s);
        particles_after_stream(s);
        ib_force(s);
        s->step += 1;
    }
    return 0;
}

int or_fields(or_sim *s, double *rho, double *ux, double *uy) {
    prime(s);
    size_t n = NN(s);
    moments(s, rho, ux, uy, 0.0, 0.0);
#pragma omp parallel for schedule(static)
    for (size_t k = 0; k < n; ++k) {
        double jx = ux[k] * rho[k], jy = uy[k] * rho[k];
        ux[k] = (jx + 0.5 * (s->c.gx + s->fibx[k])) / rho[k];
        uy[k] = (jy + 0.5 * (s->c.gy + s->fiby[k])) / rho[k];
    }
    return 0;
}

int or_ib_force(or_sim *s, double *fx, double *fy) {
    prime(s);
    memcpy(fx, s->fibx, NN(s) * sizeof(double));
    memcpy(fy, s->fiby, NN(s) * sizeof(double));
    return 0;
}

int or_particle_get(const or_sim *s, int pid, or_particle_state *o) {
    if (!s || pid < 0 || pid >= s->np) return -1;
    const or_particle *p = &s->p[pid];
    o->xc = p->xc; o->yc = p->yc; o->theta = p->theta;
    o->u = p->u; o->v = p->v; o->omega = p->omega;
    o->Fh[0] = p->Fh[0]; o->Fh[1] = p->Fh[1]; o->Mh = p->Mh;
    o->Fb[0] = p->Fb[0]; o->Fb[1] = p->Fb[1]; o->Mb = p->Mb;
    o->Fw[0] = p->Fw[0]; o->Fw[1] = p->Fw[1];
    o->area = p->area; o->mass = p->mass; o->inertia = p->inertia; o->r_eq = p->r_eq;
    o->nl = p->nv; o->n_ligands = p->n_ligands;
    o->n_probing = p->n_probing; o->n_bonded = p->n_bonded;
    o->margin_p = p->margin_p; o->margin_gap = p->margin_gap;
    o->gap_bottom = p->gap[0]; o->gap_top = p->gap[1];
    return 0;
}

int or_bonds_get(const or_sim *s, int pid, uint8_t *bond, double *anchor_x,
                 int8_t *anchor_wall) {
    if (!s || pid < 0 || pid >= s->np) return -1;
    const or_particle *p = &s->p[pid];
    if (bond) memcpy(bond, p->bond, p->nv);
    if (anchor_x) memcpy(anchor_x, p->anchor_x, p->nv * sizeof(double));
    if (anchor_wall) memcpy(anchor_wall, p->anchor_wall, p->nv);
    return 0;
}

/* Overwrites a particle's bond state (bond flag, anchor x and anchor wall of
 * every element), e.g. to place a known bond before a step. */
int or_bonds_set(or_sim *s, int pid, const uint8_t *bond, const double *anchor_x,
                 const int8_t *anchor_wall) {
    if (!s || pid < 0 || pid >= s->np || !bond || !anchor_x || !anchor_wall) return -1;
    or_particle *p = &s->p[pid];
    for (int l = 0; l < p->nv; ++l) {
        p->bond[l] = bond[l] ? 1 : 0;
        p->anchor_x[l] = anchor_x[l];
        p->anchor_wall[l] = anchor_wall[l] ? 1 : 0;
    }
    return 0;
}
