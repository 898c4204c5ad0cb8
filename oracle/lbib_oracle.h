/*
 * lbib_oracle.h -- plain FP64 CPU oracle of the LB-IB-MLS adhesion time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; it is written from the
 * paper (Coclite et al., "Predicting different adhesive regimens of
 * circulating particles at blood capillary walls", arXiv:1808.01448) with
 * plain loops, in double precision, built with -ffp-contract=off.
 *
 * Notation follows the paper: f_i populations (Eq. 1), f_i^eq (Eq. 2), e_i
 * (Eq. 3), the Guo source F_i (Eq. 4), moments (Eq. 5-6), loads (Eq. 7-8),
 * bond spring (Eq. 9), forward / reverse probabilities (Eq. 10-11), the wall
 * force (Eq. 12) and the rigid-body update (Eq. 13-16).  Lattice units:
 * dx = dt = 1, c_s^2 = 1/3.
 */
#ifndef LBIB_ORACLE_H
#define LBIB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_WALL_ZOU_HE = 0, OR_WALL_BOUNCE_BACK = 1, OR_WALL_PERIODIC = 2 };

typedef struct or_config {
    int32_t nx, ny;
    int32_t wall_bottom, wall_top;  /* OR_WALL_*; periodic must be set on both */
    double tau;                      /* BGK relaxation time, nu = (tau - 1/2)/3 */
    double u_bottom, u_top;          /* tangential (x) wall velocities */
    double gx, gy;                   /* uniform body-force density */
    double k_f, k_r0, kBT;           /* Eq. 10-11 rates (per step) and k_B T */
    double sigma_star_ratio;         /* sigma* = ratio * sigma (Eq. 11) */
    double y_cr;                     /* critical bond length (lattice units) */
    double y_eq_ratio;               /* y_cr,eq = ratio * y_cr (Eq. 9) */
    double hamaker, eps_min;         /* Eq. 12 constant, lower clamp of the gap */
    double receptor_bottom, receptor_top; /* receptor density on each wall */
    uint64_t seed, sim_id;           /* Philox key */
    int32_t ib_iterations;           /* direct-forcing passes per step (<= 1: one) */
    int32_t ib_spread;               /* spreading scale eps_l: 0 element length S_l,
                                        1 solved (Vanella & Balaras, ref. [39]) */
} or_config;

typedef struct or_particle_in {
    int32_t n_vertices;              /* polygon in the body frame, CCW */
    int32_t fixed;                   /* 1: pose held fixed (loads still computed) */
    const double *vx, *vy;           /* vertex coordinates relative to the centroid */
    double xc, yc, theta;            /* initial pose */
    double rho_p;                    /* particle density (mass = rho_p * area) */
    double ligand_density;           /* fraction of elements carrying a ligand */
    double sigma;                    /* spring constant (Eq. 9) */
} or_particle_in;

typedef struct or_particle_state {
    double xc, yc, theta, u, v, omega;
    double Fh[2], Mh;                /* hydrodynamic load (Eq. 7-8) and moment */
    double Fb[2], Mb;                /* bond force and moment (Eq. 9) */
    double Fw[2];                    /* wall force (Eq. 12) */
    double area, mass, inertia, r_eq;
    int32_t nl, n_ligands, n_probing, n_bonded;
    /* near-tie diagnostics of the last bond step (no effect on results):
     * smallest |U - P| over the draws compared with P_f or P_r, and smallest
     * |gap - y_cr| over the ligands' probing tests (inf when there was none) */
    double margin_p, margin_gap;
    /* smallest element-centroid gap to the bottom / top wall line at the
     * pose of the last bond step (inf before the first step or with
     * periodic walls) */
    double gap_bottom, gap_top;
} or_particle_state;

typedef struct or_sim or_sim;

/* --- whole simulation ---------------------------------------------------- */
or_sim *or_create(const or_config *cfg);
void or_destroy(or_sim *s);
int or_add_particle(or_sim *s, const or_particle_in *p);   /* -> id or -1 */
/* post-collision populations f*_i, layout [9][ny][nx]; only before step 1 */
int or_set_populations(or_sim *s, const double *f_post);
int or_get_populations(const or_sim *s, double *f_post);
int or_step(or_sim *s, int64_t nsteps);
int64_t or_step_count(const or_sim *s);
/* rho and the physical velocity u = (sum f e + (g + f_ib)/2) / rho at the
 * current step, each [ny][nx] */
int or_fields(or_sim *s, double *rho, double *ux, double *uy);
/* current IB force density [ny][nx] for each component */
int or_ib_force(or_sim *s, double *fx, double *fy);
int or_particle_get(const or_sim *s, int pid, or_particle_state *out);
/* bond flag, anchor x and anchor wall (0 bottom, 1 top) of every element;
 * any pointer may be NULL */
int or_bonds_get(const or_sim *s, int pid, uint8_t *bond, double *anchor_x,
                 int8_t *anchor_wall);
int or_bonds_set(or_sim *s, int pid, const uint8_t *bond, const double *anchor_x,
                 const int8_t *anchor_wall);

/* --- building blocks (used by the sim, exported for the pins) ------------ */
void or_lattice(int32_t *ex, int32_t *ey, double *w, int32_t *opp);
void or_equilibrium(double rho, double ux, double uy, double *feq);
void or_guo_source(double tau, double ux, double uy, double Fx, double Fy, double *S);
void or_collide_node(const double *f, double tau, double Fx, double Fy, double *fpost);
double or_weight(double r);
/* MLS shape functions at (X, Y): writes up to 16 support nodes and phi;
 * returns the node count (0 when the support cannot fit a linear basis). */
int or_mls_shape(const or_config *c, double X, double Y, int32_t *ix, int32_t *iy,
                 double *phi);
/* MLS fit of a nodal field [ny][nx] at (X, Y): value and diffuse gradient. */
int or_mls_fit(const or_config *c, const double *field, double X, double Y,
               double *value, double *ddx, double *ddy);
/* Spread marker forces F_l eps_l into fx, fy ([ny][nx], accumulated). */
void or_spread(const or_config *c, int n, const double *X, const double *Y,
               const double *Fx, const double *Fy, const double *eps, double *fx,
               double *fy);
/* Spreading scales eps_l of n markers solved so that interpolating the
 * spread of a uniform marker force gives it back at every marker
 * (Vanella & Balaras, ref. [39]): sum_m A_lm eps_m = 1 with
 * A_lm = sum_k phi_k(X_l) phi_k(X_m).  Markers without a fit get eps = 0.
 * Returns 0, or -1 if the system is singular. */
int or_vb_eps(const or_config *c, int n, const double *X, const double *Y, double *eps);
/* Interpolate a nodal field at n points. */
void or_interp(const or_config *c, const double *field, int n, const double *X,
               const double *Y, double *out);
/* Hydrodynamic load (Eq. 7-8) from nodal moments rho, ux, uy for a polygon
 * (body-frame vertices) at pose (xc, yc, theta): out = {Fx, Fy, M}. */
void or_loads(const or_config *c, const double *rho, const double *ux, const double *uy,
              int nv, const double *vx, const double *vy, double xc, double yc,
              double theta, double *out);
/* Element centroids, outward normals and lengths of a polygon at a pose. */
void or_elements(int nv, const double *vx, const double *vy, double xc, double yc,
                 double theta, double *mx, double *my, double *nxo, double *nyo,
                 double *S);
void or_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out);
double or_uniform(uint64_t seed, uint64_t sim_id, int64_t step, int32_t pid, int32_t l);
double or_prob_forward(double k_f, double Nl);
double or_prob_reverse(double k_r0, double sigma, double sigma_star, double y,
                       double y_eq, double kBT);
/* One step of Eq. 15 (velocity) given the two previous values and the
 * acceleration; and the matching position update. */
double or_bdf2_velocity(double u1, double u2, double acc);
double or_bdf2_position(double x1, double x2, double u_new);

#ifdef __cplusplus
}
#endif
#endif
