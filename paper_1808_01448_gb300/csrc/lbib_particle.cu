// lbib_particle.cu -- per-particle kernel: loads, bonds, wall force, rigid
// update and IB direct forcing.  One CTA per particle; runs after the lattice
// kernel of step n and reads the populations it wrote.
//
//  1. markers X_l, n_l at the pose of step n (FP64)
//  2. loads (Eq. 7-8): probe Q_l = X_l + 1.2 n_l, MLS fit of rho and grad u
//     from the new populations; traction summed in FP64
//  3. bonds (Eq. 9-11): probing count N_l, one Philox4x64-10 uniform per
//     ligand and step, formation / rupture, spring forces summed in FP64
//  4. wall force (Eq. 12) from the smallest element gap
//  5. rigid update (Eq. 13-16 and the matching pose update), FP64
//  6. IB forcing at the new pose: MLS interpolation of u* and rho at each
//     marker, F_l = 2 rho_l (U^d_l - u*_l), spreading f_ib += phi_k F_l S_l into
//     an on-chip tile in a fixed colour order (markers of one colour have
//     disjoint supports), then the tile is written out for the next lattice
//     kernel.  In init mode only step 6 runs, at the current pose.
//
// MLS (refs [13], [39]): linear basis, tensor-product cubic B-spline weight of
// radius 2, 4 x 4 support.  The weight factorises, so the 3 x 3 moment matrix
// does too: along an axis whose four support rows are all fluid the 1D
// moments are exactly (1, 0, 1/3) (partition of unity and the B-spline's
// first and second moments); only an axis clipped by a wall needs its
// moments summed, which is done in FP64.  In the centred basis the matrix is
// diagonal, giving phi_k = w_k / W (1 - (dy_k - mu_y) mu_y / v_y) and the fit
// gradient sum w_k d'_k u_k / (W v).
#include "lbib_internal.cuh"

namespace lbib {

namespace {

constexpr int P_THREADS = 512;
constexpr int P_WARPS = P_THREADS / 32;

template <typename R>
__device__ __forceinline__ R bspline(R r) {
    r = fabs(r);
    if (r < (R)1) return (R)(2.0 / 3.0) - r * r + (R)0.5 * r * r * r;
    if (r < (R)2) {
        const R b = (R)2 - r;
        return b * b * b * (R)(1.0 / 6.0);
    }
    return (R)0;
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): multipliers and Weyl
// key increments from the paper's 4x64 parameter set.
__device__ __forceinline__ unsigned long long philox_first(unsigned long long c0,
                                                           unsigned long long c1,
                                                           unsigned long long c2,
                                                           unsigned long long c3,
                                                           unsigned long long k0,
                                                           unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return c0;
}

// Uniform in [0, 1) for (sim, step, particle, element): key (seed, sim_id),
// counter (step, particle << 32 | element, 0, 0), top 53 bits of word 0.
__device__ __forceinline__ double bond_uniform(const SimDev &s, long long step, int pid, int l) {
    const unsigned long long w = philox_first(
        (unsigned long long)step, ((unsigned long long)(unsigned)pid << 32) | (unsigned)l, 0ULL,
        0ULL, s.seed, s.sim_id);
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

// Support of a point (X, Y): base node, fractional offsets, and the y-axis
// moments (W0, mu, v) -- analytic (1, 0, 1/3) unless a wall clips a row.
template <typename R>
struct Support {
    int ix0, iy0;      // node of (a, b) = (0, 0), unwrapped
    R fx, fy;          // X - floor(X), Y - floor(Y)
    R invW, mu, mu_v;  // 1 / W0_y, mu_y, mu_y / v_y
    R inv_v;           // 1 / v_y
    unsigned rows;     // bit b set: row b is a fluid row
    bool ok;
};

// Support rows: every lattice row (wall nodes included) unless periodic.
__device__ __forceinline__ void row_limits(const SimDev &s, int &lo, int &hi) {
    lo = 0;
    hi = s.ny - 1;
}

template <typename R>
__device__ __forceinline__ Support<R> make_support(const SimDev &s, double X, double Y) {
    Support<R> sp;
    const double flx = floor(X), fly = floor(Y);
    sp.ix0 = (int)flx - 1;
    sp.iy0 = (int)fly - 1;
    sp.fx = (R)(X - flx);
    sp.fy = (R)(Y - fly);
    const bool periodic = s.wall_b == LBIB_WALL_PERIODIC;
    int lo, hi;
    row_limits(s, lo, hi);
    unsigned rows = 0;
    int nz = 0;
    for (int b = 0; b < 4; ++b) {
        const int yy = sp.iy0 + b;
        const bool valid = periodic || (yy >= lo && yy <= hi);
        if (valid) {
            rows |= 1u << b;
            if (fabs((double)yy - Y) < 2.0) ++nz;
        }
    }
    sp.rows = rows;
    sp.ok = nz >= 2;
    if (rows == 0xFu) {
        sp.invW = (R)1;
        sp.mu = (R)0;
        sp.mu_v = (R)0;
        sp.inv_v = (R)3;
    } else {
        // FP64 moments of the clipped axis and their closed-form solve
        double W0 = 0.0, W1 = 0.0, W2 = 0.0;
        for (int b = 0; b < 4; ++b) {
            if (!(rows & (1u << b))) continue;
            const double dy = (double)(sp.iy0 + b) - Y;
            const double w = bspline(dy);
            W0 += w;
            W1 += w * dy;
            W2 += w * dy * dy;
        }
        if (sp.ok && W0 > 0.0) {
            const double mu = W1 / W0;
            const double v = W2 / W0 - mu * mu;
            sp.invW = (R)(1.0 / W0);
            sp.mu = (R)mu;
            sp.mu_v = (R)(mu / v);
            sp.inv_v = (R)(1.0 / v);
        } else {
            sp.ok = false;
            sp.invW = sp.mu = sp.mu_v = sp.inv_v = (R)0;
        }
    }
    return sp;
}

// Half-warp (16 lanes) sum; both halves of the warp must call it.
template <typename T>
__device__ __forceinline__ T hw_sum(T v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sums of N doubles (all threads call; result in every thread).
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < N; ++j) red[warp * N + j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < N; ++j) {
        double acc = 0.0;
        for (int w = 0; w < P_WARPS; ++w) acc += red[w * N + j];
        v[j] = acc;
    }
    __syncthreads();
}

__device__ __forceinline__ double block_min(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double m = red[0];
    for (int w = 1; w < P_WARPS; ++w) m = fmin(m, red[w]);
    __syncthreads();
    return m;
}

__device__ __forceinline__ void wall_lines(const SimDev &s, double &yb, double &yt) {
    yb = s.wall_b == LBIB_WALL_BOUNCE_BACK ? -0.5 : 0.0;
    yt = s.wall_t == LBIB_WALL_BOUNCE_BACK ? (double)s.ny - 0.5 : (double)(s.ny - 1);
}

struct SmemLayout {
    double *mx, *my, *nxw, *nyw;  // world markers [nl]
    int *sp_i;                     // [nl][2] support base
    void *sp_r;                    // [nl][7] R: fx, fy, invW, mu, mu_v, Fx, Fy
    double *red;                   // reduction scratch
    void *tile;                    // [2][T][T] R
};

template <typename R>
__device__ SmemLayout carve(unsigned char *base, int nl, int T) {
    SmemLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *p = base + off;
        off += (bytes + 15) & ~size_t(15);
        return p;
    };
    L.mx = (double *)take(sizeof(double) * nl);
    L.my = (double *)take(sizeof(double) * nl);
    L.nxw = (double *)take(sizeof(double) * nl);
    L.nyw = (double *)take(sizeof(double) * nl);
    L.sp_i = (int *)take(sizeof(int) * 2 * nl);
    L.sp_r = take(sizeof(R) * 7 * nl);
    L.red = (double *)take(sizeof(double) * 8 * P_WARPS);
    L.tile = take(sizeof(R) * 2 * T * T);
    return L;
}

template <typename R>
size_t smem_bytes_for(int nl, int T) {
    auto up = [](size_t b) { return (b + 15) & ~size_t(15); };
    return 4 * up(sizeof(double) * nl) + up(sizeof(int) * 2 * nl) + up(sizeof(R) * 7 * nl) +
           up(sizeof(double) * 8 * P_WARPS) + up(sizeof(R) * 2 * T * T);
}

__device__ __forceinline__ void place_markers(const ParticleDev *P, double xc, double yc,
                                              double th, SmemLayout &L) {
    double sn, cs;
    sincos(th, &sn, &cs);
    for (int l = threadIdx.x; l < P->nl; l += P_THREADS) {
        const double bx = P->mbx[l], by = P->mby[l];
        L.mx[l] = xc + (cs * bx - sn * by);
        L.my[l] = yc + (sn * bx + cs * by);
        const double nbx = P->nbx[l], nby = P->nby[l];
        L.nxw[l] = cs * nbx - sn * nby;
        L.nyw[l] = sn * nbx + cs * nby;
    }
}

template <typename S, typename R>
__global__ void __launch_bounds__(P_THREADS) particle_kernel(BatchDev b, int flip, int init) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ParticleDev *P = b.parts[blockIdx.x];
    const SimDev &s = b.sims[b.part_sim[blockIdx.x]];
    const int nl = P->nl, T = P->T;
    SmemLayout L = carve<R>(smem_raw, nl, T);
    R *spr = (R *)L.sp_r;
    R *tile = (R *)L.tile;
    const S *__restrict__ pop = (const S *)s.pop[*s.cur ^ flip];
    const int lane = threadIdx.x & 31, hl = lane & 15;
    const int half = threadIdx.x >> 4;  // half-warp index
    const int nhalf = P_THREADS / 16;
    const int a = hl & 3, bb = hl >> 2;
    const int nx = s.nx, ny = s.ny;
    const bool periodic = s.wall_b == LBIB_WALL_PERIODIC;

    double xc = P->xc, yc = P->yc, th = P->th;
    double u = P->u, v = P->v, om = P->om;

    if (!init) {
        place_markers(P, xc, yc, th, L);
        __syncthreads();
        // ---- 2. hydrodynamic loads (Eq. 7-8) ------------------------------
        const R nu = (R)((s.tau - 0.5) / 3.0);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int base = 0; base < nl; base += nhalf) {
            const int l = base + half;
            const bool act = l < nl;
            double qx = 0.0, qy = 0.0;
            if (act) {
                qx = L.mx[l] + 1.2 * L.nxw[l];
                qy = L.my[l] + 1.2 * L.nyw[l];
            }
            Support<R> sp = make_support<R>(s, act ? qx : 0.0, act ? qy : 1.5);
            R s_rho = 0, s_ux = 0, s_uy = 0, s_vx = 0, s_vy = 0;
            if (act && sp.ok && (sp.rows & (1u << bb))) {
                const R dx = (R)(a - 1) - sp.fx, dy = (R)(bb - 1) - sp.fy;
                const R wx = bspline(dx), wy = bspline(dy);
                if (wx * wy != (R)0) {
                    int xx = (sp.ix0 + a) % nx;
                    if (xx < 0) xx += nx;
                    int yy = sp.iy0 + bb;
                    if (periodic) {
                        yy %= ny;
                        if (yy < 0) yy += ny;
                    }
                    R d[9];
                    pull_node<S, R>(s, pop, xx, yy, d);
                    R drho, jx, jy;
                    node_moments(d, drho, jx, jy);
                    const R irho = (R)1 / ((R)1 + drho);
                    const R ux = jx * irho, uy = jy * irho;
                    const R w = wx * wy * sp.invW;
                    const R phi = w * ((R)1 - (dy - sp.mu) * sp.mu_v);
                    const R dyc = dy - sp.mu;
                    s_rho = phi * drho;
                    s_ux = w * dx * ux;
                    s_uy = w * dyc * ux;
                    s_vx = w * dx * uy;
                    s_vy = w * dyc * uy;
                }
            }
            s_rho = hw_sum(s_rho);
            s_ux = hw_sum(s_ux);
            s_uy = hw_sum(s_uy);
            s_vx = hw_sum(s_vx);
            s_vy = hw_sum(s_vy);
            if (act && hl == 0 && sp.ok) {
                const R dudx = (R)3 * s_ux, dudy = s_uy * sp.inv_v;
                const R dvdx = (R)3 * s_vx, dvdy = s_vy * sp.inv_v;
                const R p = s_rho * (R)(1.0 / 3.0);
                const R nxl = (R)L.nxw[l], nyl = (R)L.nyw[l];
                const R txy = nu * (dudy + dvdx);
                const R tx = -p * nxl + nu * (R)2 * dudx * nxl + txy * nyl;
                const R ty = -p * nyl + txy * nxl + nu * (R)2 * dvdy * nyl;
                const double Sl = P->S[l];
                const double fx = (double)tx * Sl, fy = (double)ty * Sl;
                acc[0] += fx;
                acc[1] += fy;
                acc[2] += (L.mx[l] - xc) * fy - (L.my[l] - yc) * fx;
            }
        }
        block_sum<3>(acc, L.red);

        // ---- 3. bonds (Eq. 9-11) ------------------------------------------
        double yb, yt;
        wall_lines(s, yb, yt);
        const bool has_b = s.wall_b != LBIB_WALL_PERIODIC && s.rec_b > 0.0;
        const bool has_t = s.wall_t != LBIB_WALL_PERIODIC && s.rec_t > 0.0;
        double cnt[1] = {0.0};
        for (int l = threadIdx.x; l < nl; l += P_THREADS) {
            if (!P->ligand[l]) continue;
            const bool pb = has_b && (L.my[l] - yb) < s.y_cr;
            const bool pt = has_t && (yt - L.my[l]) < s.y_cr;
            cnt[0] += (pb || pt) ? 1.0 : 0.0;
        }
        block_sum<1>(cnt, L.red);
        const int nprobe = (int)cnt[0];
        const double Nl = (double)nprobe / (double)nl;
        const double Pf_b = 1.0 - exp(-(s.k_f * s.rec_b) * Nl);
        const double Pf_t = 1.0 - exp(-(s.k_f * s.rec_t) * Nl);
        const double y_eq = s.y_eq_ratio * s.y_cr;
        const double sigma = P->sigma, sstar = s.sigma_star_ratio * P->sigma;
        const long long step = *s.step - 1;   // index of the step being completed
        double fb[4] = {0.0, 0.0, 0.0, 0.0};
        double gmin_b = 1e300, gmin_t = 1e300;
        const int pid = (int)blockIdx.x - s.p0;   // particle index within its simulation
        for (int l = threadIdx.x; l < nl; l += P_THREADS) {
            gmin_b = fmin(gmin_b, L.my[l] - yb);
            gmin_t = fmin(gmin_t, yt - L.my[l]);
            if (!P->ligand[l]) continue;
            const double U = bond_uniform(s, step, pid, l);
            uint8_t bnd = P->bond[l];
            if (bnd) {
                const double wy = P->anchor_wall[l] ? yt : yb;
                const double dx = P->anchor_x[l] - L.mx[l], dy = wy - L.my[l];
                const double y = sqrt(dx * dx + dy * dy);
                const double dd = y - y_eq;
                const double kr = s.k_r0 * exp((sigma - sstar) * dd * dd / (2.0 * s.kBT));
                const double Pr = 1.0 - exp(-kr);
                if (U < Pr) bnd = 0;
            } else {
                const bool pb = has_b && (L.my[l] - yb) < s.y_cr;
                const bool pt = has_t && (yt - L.my[l]) < s.y_cr;
                if (pb || pt) {
                    const double Pf = pb ? Pf_b : Pf_t;
                    if (U < Pf) {
                        bnd = 1;
                        P->anchor_x[l] = L.mx[l];
                        P->anchor_wall[l] = pb ? 0 : 1;
                    }
                }
            }
            P->bond[l] = bnd;
            if (bnd) {
                const double wy = P->anchor_wall[l] ? yt : yb;
                const double dx = P->anchor_x[l] - L.mx[l], dy = wy - L.my[l];
                const double y = sqrt(dx * dx + dy * dy);
                if (y > 0.0) {
                    const double mag = sigma * (y - y_eq);
                    const double fx = mag * dx / y, fy = mag * dy / y;
                    fb[0] += fx;
                    fb[1] += fy;
                    fb[2] += (L.mx[l] - xc) * fy - (L.my[l] - yc) * fx;
                }
                fb[3] += 1.0;
            }
        }
        block_sum<4>(fb, L.red);
        gmin_b = block_min(gmin_b, L.red);
        gmin_t = block_min(gmin_t, L.red);

        // ---- 4-5. wall force (Eq. 12) and rigid update (Eq. 13-16) ---------
        double Fw = 0.0;
        if (s.wall_b != LBIB_WALL_PERIODIC && s.hamaker != 0.0) {
            const double eb = fmax(gmin_b, s.eps_min), et = fmax(gmin_t, s.eps_min);
            const double k = s.hamaker / (8.0 * sqrt(2.0));
            Fw = k * sqrt(P->r_eq / pow(eb, 5.0)) - k * sqrt(P->r_eq / pow(et, 5.0));
        }
        if (!P->fixed) {
            const double Fx = acc[0] + fb[0];
            const double Fy = acc[1] + fb[1] + Fw;
            const double M = acc[2] + fb[2];
            const double un = 2.0 / 3.0 * (2.0 * u - 0.5 * P->u1 + Fx / P->mass);
            const double vn = 2.0 / 3.0 * (2.0 * v - 0.5 * P->v1 + Fy / P->mass);
            const double wn = 2.0 / 3.0 * (2.0 * om - 0.5 * P->om1 + M / P->inertia);
            const double xn = (4.0 * xc - P->xc1 + 2.0 * un) / 3.0;
            const double yn = (4.0 * yc - P->yc1 + 2.0 * vn) / 3.0;
            const double tn = (4.0 * th - P->th1 + 2.0 * wn) / 3.0;
            __syncthreads();
            if (threadIdx.x == 0) {
                P->u1 = u; P->v1 = v; P->om1 = om;
                P->xc1 = xc; P->yc1 = yc; P->th1 = th;
                P->u = un; P->v = vn; P->om = wn;
                P->xc = xn; P->yc = yn; P->th = tn;
            }
            u = un; v = vn; om = wn;
            xc = xn; yc = yn; th = tn;
        }
        if (threadIdx.x == 0) {
            P->Fh[0] = acc[0]; P->Fh[1] = acc[1]; P->Mh = acc[2];
            P->Fb[0] = fb[0]; P->Fb[1] = fb[1]; P->Mb = fb[2];
            P->Fw[0] = 0.0; P->Fw[1] = Fw;
            P->n_probing = nprobe;
            P->n_bonded = (int)fb[3];
        }
        __syncthreads();
    }

    // ---- 6. IB direct forcing at the (new) pose ---------------------------
    place_markers(P, xc, yc, th, L);
    for (int i = threadIdx.x; i < 2 * T * T; i += P_THREADS) tile[i] = (R)0;
    __syncthreads();
    const R ghx = (R)(0.5 * s.gx), ghy = (R)(0.5 * s.gy);
    for (int base = 0; base < nl; base += nhalf) {
        const int l = base + half;
        const bool act = l < nl;
        Support<R> sp = make_support<R>(s, act ? L.mx[l] : 0.0, act ? L.my[l] : 1.5);
        R s_rho = 0, s_u = 0, s_v = 0;
        if (act && sp.ok && (sp.rows & (1u << bb))) {
            const R dx = (R)(a - 1) - sp.fx, dy = (R)(bb - 1) - sp.fy;
            const R wx = bspline(dx), wy = bspline(dy);
            if (wx * wy != (R)0) {
                int xx = (sp.ix0 + a) % nx;
                if (xx < 0) xx += nx;
                int yy = sp.iy0 + bb;
                if (periodic) {
                    yy %= ny;
                    if (yy < 0) yy += ny;
                }
                R d[9];
                pull_node<S, R>(s, pop, xx, yy, d);
                R drho, jx, jy;
                node_moments(d, drho, jx, jy);
                const R irho = (R)1 / ((R)1 + drho);
                const R phi = wx * wy * sp.invW * ((R)1 - (dy - sp.mu) * sp.mu_v);
                s_rho = phi * drho;
                s_u = phi * ((jx + ghx) * irho);
                s_v = phi * ((jy + ghy) * irho);
            }
        }
        s_rho = hw_sum(s_rho);
        s_u = hw_sum(s_u);
        s_v = hw_sum(s_v);
        if (act && hl == 0) {
            R Fx = 0, Fy = 0;
            if (sp.ok) {
                const R rl = (R)1 + s_rho;
                const R udx = (R)(u - om * (L.my[l] - yc));
                const R udy = (R)(v + om * (L.mx[l] - xc));
                const R eps = (R)P->S[l];
                Fx = (R)2 * rl * (udx - s_u) * eps;
                Fy = (R)2 * rl * (udy - s_v) * eps;
            }
            L.sp_i[2 * l] = sp.ix0;
            L.sp_i[2 * l + 1] = sp.iy0;
            R *q = spr + 7 * l;
            q[0] = sp.fx;
            q[1] = sp.fy;
            q[2] = sp.ok ? sp.invW : (R)0;
            q[3] = sp.mu;
            q[4] = sp.mu_v;
            q[5] = Fx;
            q[6] = Fy;
        }
    }
    __syncthreads();
    // tile origin: unwrapped node floor(X_c) - T/2 (and likewise in y)
    const int ox = (int)floor(xc) - T / 2;
    const int oy = (int)floor(yc) - T / 2;
    int lo, hi;
    row_limits(s, lo, hi);
    for (int c = 0; c < P->ncolors; ++c) {
        const int m0 = P->color_off[c], m1 = P->color_off[c + 1];
        const int ntask = (m1 - m0) * 16;
        for (int t = threadIdx.x; t < ntask; t += P_THREADS) {
            const int m = P->color_order[m0 + (t >> 4)];
            const int j = t & 15, ta = j & 3, tb = j >> 2;
            const R *q = spr + 7 * m;
            if (q[2] == (R)0) continue;
            const int iy = L.sp_i[2 * m + 1] + tb;
            if (!periodic && (iy < lo || iy > hi)) continue;
            const R dx = (R)(ta - 1) - q[0], dy = (R)(tb - 1) - q[1];
            const R phi = bspline(dx) * bspline(dy) * q[2] * ((R)1 - (dy - q[3]) * q[4]);
            const int tx = L.sp_i[2 * m] + ta - ox, ty = iy - oy;
            if ((unsigned)tx < (unsigned)T && (unsigned)ty < (unsigned)T) {
                tile[ty * T + tx] += phi * q[5];
                tile[T * T + ty * T + tx] += phi * q[6];
            }
        }
        __syncthreads();
    }
    R *gt = (R *)P->tile;
    for (int i = threadIdx.x; i < 2 * T * T; i += P_THREADS) gt[i] = tile[i];
    if (threadIdx.x == 0) {
        int oxw = ox % nx;
        if (oxw < 0) oxw += nx;
        int oyw = oy;
        if (periodic) {
            oyw %= ny;
            if (oyw < 0) oyw += ny;
        }
        P->tile_ox = oxw;
        P->tile_oy = oyw;
    }
}

template <typename F>
cudaError_t by_kind(int kind, F &&f) {
    switch (kind) {
        case ST_F32: return f(float{}, float{});
        case ST_F64: return f(double{}, double{});
        case ST_F16: return f(__half{}, float{});
        case ST_BF16: return f(__nv_bfloat16{}, float{});
    }
    return cudaErrorInvalidValue;
}

}  // namespace

int particle_smem_bytes(int kind, int T, int nl) {
    return (int)(kind == ST_F64 ? smem_bytes_for<double>(nl, T) : smem_bytes_for<float>(nl, T));
}

cudaError_t particle_kernel_setup(int kind, int smem) {
    return by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        return cudaFuncSetAttribute(particle_kernel<S, R>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    });
}

cudaError_t launch_particles(int kind, const BatchDev &b, int flip, int init, int smem,
                             cudaStream_t st) {
    if (b.nparts == 0) return cudaSuccess;
    return by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        particle_kernel<S, R><<<b.nparts, P_THREADS, smem, st>>>(b, flip, init);
        return cudaGetLastError();
    });
}

}  // namespace lbib
