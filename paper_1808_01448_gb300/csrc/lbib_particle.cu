// lbib_particle.cu -- per-particle kernel: loads, bonds, wall force, rigid
// update and IB direct forcing.  One CTA per particle; runs after the lattice
// kernel of step n and reads the populations it wrote.
//
//  1. markers X_l, n_l at the pose of step n (FP64)
//  2. loads (Eq. 7-8): probe Q_l = X_l + 1.2 n_l, MLS fit of rho and grad u
//     from the new populations; tractions summed in FP64
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
// does too: along an axis whose four support rows are all lattice rows the 1D
// moments are exactly (1, 0, 1/3) (partition of unity and the B-spline's
// first and second moments); only an axis clipped by a wall needs its
// moments summed, which is done in FP64.  In the centred basis the matrix is
// diagonal, giving phi_k = w_k / W (1 - (dy_k - mu_y) mu_y / v_y) and the fit
// gradient sum w_k d'_k u_k / (W v).
//
// GB300 has little FP64 throughput, so per-particle scalars (sincos, P_f,
// Eq. 12, the update) run on one thread, per-point setup on one thread per
// point (kept in shared memory), and the FP64 sums on one warp per quantity
// over per-element contributions kept in shared memory.  Each point's 4 x 4
// support is summed by the point's own thread from the staged moments.
#include "lbib_internal.cuh"

namespace lbib {

namespace {

// Threads of a particle CTA: one marker per thread, so at least the
// particle's element count; P_THREADS (>= LBIB_MAX_MARKERS) always fits, the
// 256-thread form holds a quarter of an SM's registers while it runs.
constexpr int P_THREADS = 512;

// Cubic B-spline of radius 2, branch-free (the nodes of a support straddle
// the two pieces).
template <typename R>
__device__ __forceinline__ R bspline(R r) {
    const R a = fabs(r);
    const R inner = (R)(2.0 / 3.0) - a * a + (R)0.5 * a * a * a;
    const R b = fmax((R)2 - a, (R)0);
    const R outer = b * b * b * (R)(1.0 / 6.0);
    return a < (R)1 ? inner : outer;
}

// 1 / rho for a density near 1: FP32 hardware approximation refined by one
// Newton-Raphson step r (2 - x r) (within an ulp or two); exact division on
// the FP64 path.
template <typename R>
__device__ __forceinline__ R recip_rho(R x) {
    if constexpr (sizeof(R) == 4) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r * fmaf(-x, r, 2.f);
    } else {
        return (R)1 / x;
    }
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

// Per-particle scalars, set by thread 0 (or one lane per degree of freedom).
template <typename R>
struct Pose {
    double xc, yc, th, u, v, om;
    double F[6];        // Fh x, y, M; Fb x, y, M (FP64 sums)
    double Fw;
    double gapb, gapt;  // smallest element gaps to the wall lines (FP64)
    double csd, snd;    // FP64 cos, sin of the angle (bond geometry)
    int ixc, iyc;       // floor of the centroid (base node of relative coordinates)
    R fxc, fyc;         // centroid minus its floor
    R cs, sn;           // cos, sin of the angle
    R gap0_b, gap0_t;   // centroid distance to the bottom / top wall line
    R uR, vR, omR;      // velocities in the compute precision
    int nprobe, nbonded;
};

// The pose in the compute precision, one degree of freedom at a time (so that
// the three lanes of the rigid update can each finish their own): 0 the
// centroid's x (floor node, offset, u), 1 its y (floor node, offset, wall
// distances, v), 2 the angle (cos and sin, omega).
template <typename R>
__device__ __forceinline__ void set_pose_dof(Pose<R> &ps, int k, double yb, double yt) {
    if (k == 0) {
        const double fx = floor(ps.xc);
        ps.ixc = (int)fx;
        ps.fxc = (R)(ps.xc - fx);
        ps.uR = (R)ps.u;
    } else if (k == 1) {
        const double fy = floor(ps.yc);
        ps.iyc = (int)fy;
        ps.fyc = (R)(ps.yc - fy);
        ps.gap0_b = (R)(ps.yc - yb);
        ps.gap0_t = (R)(yt - ps.yc);
        ps.vR = (R)ps.v;
    } else {
        R sn, cs;
        if constexpr (sizeof(R) == 4) {
            // angle reduced to [-pi, pi] in FP64, then the FP32 sine and cosine
            const double t = ps.th - 6.283185307179586 * rint(ps.th * 0.15915494309189535);
            sincosf((float)t, &sn, &cs);
        } else {
            sincos(ps.th, &sn, &cs);
        }
        ps.cs = cs;
        ps.sn = sn;
        ps.omR = (R)ps.om;
    }
}

template <typename R>
__device__ __noinline__ void set_pose(Pose<R> &ps, double yb, double yt) {
    for (int k = 0; k < 3; ++k) set_pose_dof(ps, k, yb, yt);
}

// MLS support parameters of the points (probes or markers), one slot per
// element, in shared memory.  Points are relative to the centroid's floor
// node, so FP32 keeps them to ~1e-5 lattice units.
template <typename R>
struct Points {
    int *ix0, *iy0;     // node of support corner (a, b) = (0, 0), unwrapped
    int *rows;          // bits 0-3: lattice rows of the support; bit 4: fit possible
    R *fx, *fy;         // X - floor(X), Y - floor(Y)
    R *invW, *mu, *mu_v, *inv_v;   // y-axis moments: 1 / W0, mu, mu / v, 1 / v
};

// Moments of a wall-clipped y axis, summed and solved in FP64: 1 / W0, mu,
// mu / v and 1 / v (returned by value, so that the caller's point stays in
// registers).
template <typename R>
struct AxisMoments {
    R invW, mu, mu_v, inv_v;
};

template <typename R>
__device__ __noinline__ AxisMoments<R> clipped_axis(R fy, unsigned rows) {
    double W0 = 0.0, W1 = 0.0, W2 = 0.0;
    for (int b = 0; b < 4; ++b) {
        if (!(rows & (1u << b))) continue;
        // offset and weight in the compute precision (the point itself is
        // known to it); moments and solve in FP64
        const R dyr = (R)(b - 1) - fy;
        const double dy = (double)dyr;
        const double w = (double)bspline(dyr);
        W0 += w;
        W1 += w * dy;
        W2 += w * dy * dy;
    }
    // reciprocal: FP32 seed, two Newton-Raphson steps r <- r (2 - a r) in
    // FP64 (relative error ~1e-7 squares to below FP64 rounding)
    auto rcp = [](double a) {
        double r = (double)__frcp_rn((float)a);
        r = r * (2.0 - a * r);
        return r * (2.0 - a * r);
    };
    // with D = W0 W2 - W1^2 = W0^2 v and r = 1 / (W0 D), one reciprocal gives
    // 1 / W0 = D r, mu = W1 / W0, 1 / v = W0^2 / D = W0^3 r and
    // mu / v = W1 W0 / D = W1 W0^2 r
    const double D = W0 * W2 - W1 * W1;
    const double r = rcp(W0 * D);
    const double iW = D * r;
    const double W0r = W0 * W0 * r;
    return AxisMoments<R>{(R)iW, (R)(W1 * iW), (R)(W1 * W0r), (R)(W0 * W0r)};
}

template <typename R>
__device__ __forceinline__ void setup_point(const SimDev &s, int bx, int by, R X, R Y,
                                            const Points<R> &pt, int l) {
    const R flx = floor(X), fly = floor(Y);
    const int ix0 = bx + (int)flx - 1, iy0 = by + (int)fly - 1;
    const R fx = X - flx, fy = Y - fly;
    const bool periodic = s.wall_b == LBIB_WALL_PERIODIC;
    unsigned rows = 0;
    int nz = 0;
    // a point beyond a wall line (y = 0 / ny - 1 for Zou-He, -1/2 / ny - 1/2
    // for bounce-back) is outside the fluid and has no fit
    const int iy = iy0 + 1;
    const bool below = s.wall_b == LBIB_WALL_BOUNCE_BACK ? (iy < -1 || (iy == -1 && fy < (R)0.5))
                                                         : iy < 0;
    const bool above = s.wall_t == LBIB_WALL_BOUNCE_BACK
                           ? (iy > s.ny - 1 || (iy == s.ny - 1 && fy > (R)0.5))
                           : (iy > s.ny - 1 || (iy == s.ny - 1 && fy > (R)0));
    if (!periodic && (below || above)) {
        pt.ix0[l] = ix0;
        pt.iy0[l] = iy0;
        pt.rows[l] = 0;
        pt.fx[l] = fx;
        pt.fy[l] = fy;
        return;
    }
    for (int b = 0; b < 4; ++b) {
        const int yy = iy0 + b;
        if (periodic || (yy >= 0 && yy <= s.ny - 1)) {
            rows |= 1u << b;
            if (fabs((R)(b - 1) - fy) < (R)2) ++nz;
        }
    }
    R invW = (R)1, mu = (R)0, mu_v = (R)0, inv_v = (R)3;
    if (nz >= 2 && rows != 0xFu) {
        const AxisMoments<R> m = clipped_axis<R>(fy, rows);
        invW = m.invW;
        mu = m.mu;
        mu_v = m.mu_v;
        inv_v = m.inv_v;
    }
    pt.ix0[l] = ix0;
    pt.iy0[l] = iy0;
    pt.rows[l] = (int)rows | (nz >= 2 ? 16 : 0);
    pt.fx[l] = fx;
    pt.fy[l] = fy;
    pt.invW[l] = invW;
    pt.mu[l] = mu;
    pt.mu_v[l] = mu_v;
    pt.inv_v[l] = inv_v;
}

// Order-preserving map of a (non-NaN) double to a 64-bit integer and back:
// the bits of a non-negative double order as integers; a negative one has
// its magnitude bits flipped.  min over keys = the FP64 minimum, exactly.
__device__ __forceinline__ long long gap_key(double g) {
    const long long b = __double_as_longlong(g);
    return b >= 0 ? b : b ^ 0x7fffffffffffffffLL;
}
__device__ __forceinline__ double key_gap(long long k) {
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffLL);
}

// FP64 sum of n values of an array by one warp.
template <typename R>
__device__ __forceinline__ double warp_sum_array(const R *a, int n) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int l = lane; l < n; l += 32) acc += (double)a[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// Node moments pulled from the populations (outside the staged region).
// flip: the pass's buffer flip; with in-place streaming the state parity is
// read here (*cur ^ flip), so the caller keeps no register for it.
template <typename R>
struct Moments {
    R drho, jx, jy;
};

template <typename S, typename R>
__device__ __noinline__ Moments<R> pull_moments(const SimDev &s, const S *pop, int x, int y,
                                                int flip) {
    R d[9];
    pull_node<S, R>(s, pop, x, y, d, s.aa ? *s.cur ^ flip : 0);
    Moments<R> m;
    node_moments(d, m.drho, m.jx, m.jy);
    return m;
}

// Walks the 4 x 4 support of point l (after setup_point) in a fixed order,
// calling f(w, dx, dyc, phi, drho, jx, jy) for every node of non-zero weight:
// w = the normalised weight w_k / W, dx and dyc = the node's offsets in the
// centred basis, phi = the MLS shape function, and the node's moments
// (staged region, else pulled).  One thread per point: the staged region is
// in shared memory, so the sixteen nodes are a short loop, not a reduction.
template <typename S, typename R, typename F>
__device__ __forceinline__ void support_sum(const SimDev &s, const S *pop, int flip,
                                            const Points<R> &pt,
                                            int l, const R *mr, const R *mjx, const R *mjy,
                                            const int4 *span, const int *pre, int cap, int Tm,
                                            int rx0, int ry0, F &&f) {
    const int rows = pt.rows[l];
    if (!(rows & 16)) return;
    const R fx = pt.fx[l], fy = pt.fy[l], invW = pt.invW[l], mu = pt.mu[l], mu_v = pt.mu_v[l];
    const int ix0 = pt.ix0[l], iy0 = pt.iy0[l];
    R wx[4], dxa[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        dxa[a] = (R)(a - 1) - fx;
        wx[a] = bspline(dxa[a]);
    }
    // rows as a loop: the pass runs each instruction about once, so compact
    // code (fewer instruction fetches) beats unrolled code here
#pragma unroll 1
    for (int b = 0; b < 4; ++b) {
        if (!(rows & (1 << b))) continue;
        const R dy = (R)(b - 1) - fy;
        const R wy = bspline(dy) * invW;
        if (wy == (R)0) continue;
        const R dyc = dy - mu;
        const R py = wy * ((R)1 - dyc * mu_v);
        const int v = iy0 + b - ry0;
        // the row's staged spans (none outside the region)
        const bool inr = (unsigned)v < (unsigned)Tm;
        const int4 q = inr ? span[v] : make_int4(0, -1, 0, -1);
        const int p0 = inr ? pre[v] : 0, n0 = max(q.y - q.x + 1, 0);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const R w = wx[a] * wy;
            if (w == (R)0) continue;
            const int u = ix0 + a - rx0;
            R drho, jx, jy;
            // staging index of (u, v) in the row's spans (-1: not staged)
            const int i = (u >= q.x && u <= q.y) ? p0 + (u - q.x)
                          : (u >= q.z && u <= q.w) ? p0 + n0 + (u - q.z) : -1;
            if (i >= 0 && i < cap) {
                drho = mr[i];
                jx = mjx[i];
                jy = mjy[i];
            } else {
                int xx = (ix0 + a) % s.nx;
                if (xx < 0) xx += s.nx;
                int yy = iy0 + b;
                if (s.wall_b == LBIB_WALL_PERIODIC) {
                    yy %= s.ny;
                    if (yy < 0) yy += s.ny;
                }
                const Moments<R> m = pull_moments<S, R>(s, pop, xx, yy, flip);
                drho = m.drho;
                jx = m.jx;
                jy = m.jy;
            }
            f(w, dxa[a], dyc, wx[a] * py, drho, jx, jy);
        }
    }
}

// Edge of the staged moment region: the force tile plus two nodes a side,
// so the supports of the probes and of the markers after the update (moves
// below one node per step) fall inside it.
__host__ __device__ __forceinline__ int region_edge(int T) { return T + 4; }

template <typename R> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };

// The spreading contributions (16 pairs per marker) reuse the staged
// moments' space when they fit in it.
// Staged nodes a particle keeps in shared memory: its band's span nodes in
// staging order (row by row, each row's spans in turn), at most this many;
// nodes past it are pulled from global memory with the same arithmetic.  A
// band is about ten nodes wide along the outline, so 16 per element plus 8
// per region row covers it; a dense Tm x Tm box never needs more.
__host__ __device__ __forceinline__ int stage_cap(int nl, int Tm) {
    const long long c = 16ll * nl + 8ll * Tm, box = (long long)Tm * Tm;
    return (int)(c < box ? c : box);
}

template <typename R>
__host__ __device__ __forceinline__ bool spread_in_moments(int nl, int cap) {
    const size_t m = ((sizeof(R) * (size_t)cap + 15) & ~size_t(15)) * 3;
    return 32 * sizeof(R) * (size_t)nl <= m;
}

// Solved spreading scales: the band of A (half bandwidth up to VB_PMAX,
// VB_W entries per marker), the p + 1 interior solutions, the scales, and
// the p x p Schur complement with its right-hand side.
constexpr int VB_PMAX = LBIB_VB_MAX_BAND;
constexpr int VB_W = VB_PMAX + 1;

template <typename R>
size_t vb_bytes(int nl) {
    auto up = [](size_t b) { return (b + 15) & ~size_t(15); };
    return 2 * up(sizeof(R) * VB_W * (size_t)nl) + up(sizeof(R) * nl) +
           up(sizeof(R) * VB_PMAX * VB_W);
}

template <typename R>
size_t smem_bytes_for(int nl, int T, bool vb) {
    auto up = [](size_t b) { return (b + 15) & ~size_t(15); };
    const size_t Tm = (size_t)region_edge(T);
    const size_t cap = (size_t)stage_cap(nl, (int)Tm);
    // the staged moments (and, where they do not fit there, the spreading
    // contributions) are laid out last, then the spreading-scale system
    const size_t moments = 3 * up(sizeof(R) * cap);
    const size_t spread = spread_in_moments<R>(nl, (int)cap) ? 0 : up(32 * sizeof(R) * (size_t)nl);
    return up(sizeof(Pose<R>)) + 21 * up(sizeof(R) * nl) + 3 * up(sizeof(int) * nl) + up(nl) +
           up(sizeof(int) * nl) + up(sizeof(int) * (nl + 1)) + up(sizeof(R) * 2 * T * T) +
           up(sizeof(double) * 3 * (P_THREADS / 32)) + up(sizeof(int4) * Tm) + up(sizeof(int) * (Tm + 1)) + moments + spread +
           (vb ? vb_bytes<R>(nl) : 0);
}

// MLS shape functions of point l (after setup_point) as separable factors:
// phi_(a,b) = wx[a] py[b] on the support node (ix0 + a, iy0 + b) (zero
// without a fit or for a row outside the lattice).
template <typename R>
__device__ __forceinline__ void point_phi(const Points<R> &pt, int l, R wx[4], R py[4]) {
    const int rows = pt.rows[l];
    const R fx = pt.fx[l], fy = pt.fy[l], invW = pt.invW[l], mu = pt.mu[l];
    const R mu_v = pt.mu_v[l];
#pragma unroll
    for (int a = 0; a < 4; ++a) wx[a] = (rows & 16) ? bspline((R)(a - 1) - fx) : (R)0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        py[b] = (R)0;
        if ((rows & 16) && (rows & (1 << b))) {
            const R dy = (R)(b - 1) - fy;
            const R wy = bspline(dy) * invW;
            const R dyc = dy - mu;
            py[b] = wy * ((R)1 - dyc * mu_v);
        }
    }
}

// Row l of the spreading-scale system (Vanella & Balaras, ref. [39]):
// A[l][d] = A_(l, l + d mod n) = sum_k phi_k(X_l) phi_k(X_(l+d)) for
// d = 0 .. p over the nodes the two supports share; a marker without a fit
// has the identity row (its scale is not used).
template <typename R>
__device__ void vb_row(const Points<R> &pt, int l, int n, int p, R *A) {
    R wl[4], pl[4];
    point_phi(pt, l, wl, pl);
    const bool fl = (pt.rows[l] & 16) != 0;
    R *row = A + (size_t)l * VB_W;
    R diag = (R)0;
    if (fl) {
        R sx = 0, sy = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            sx += wl[a] * wl[a];
            sy += pl[a] * pl[a];
        }
        diag = sx * sy;
    }
    row[0] = fl ? diag : (R)1;
#pragma unroll 1
    for (int d = 1; d < VB_W; ++d) {
        R acc = (R)0;
        const int m = l + d < n ? l + d : l + d - n;
        if (d <= p && fl && (pt.rows[m] & 16)) {
            const int dx = pt.ix0[m] - pt.ix0[l], dy = pt.iy0[m] - pt.iy0[l];
            if (dx > -4 && dx < 4 && dy > -4 && dy < 4) {
                R wm[4], pm[4];
                point_phi(pt, m, wm, pm);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int bb = b - dy;
                    if (bb < 0 || bb > 3) continue;
                    R sxm = 0;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int aa = a - dx;
                        if (aa >= 0 && aa <= 3) sxm += wl[a] * wm[aa];
                    }
                    acc += pl[b] * pm[bb] * sxm;
                }
            }
        }
        row[d] = acc;
    }
}

// Entry (i, j) of the original A from the band (rows of the border and the
// band entries that reach into it are never overwritten by the
// factorisation, which is all the solve reads here).
template <typename R>
__device__ __forceinline__ R vb_at(const R *A, int n, int p, int i, int j) {
    int d = j - i;
    if (d < 0) d += n;
    if (d <= p) return A[(size_t)i * VB_W + d];
    d = n - d;
    return d <= p ? A[(size_t)j * VB_W + d] : (R)0;
}

// A eps = 1 for the cyclic band A (half bandwidth p <= VB_PMAX, n >= 2 p + 2)
// by one warp, bordered: the interior B (the first m = n - p markers,
// banded without wrap) is factored B = L D L^T by lane 0, right-looking, with
// the active window W[a][b] = B_(k+a, k+b) (b >= a) in registers (entries
// past the band are zero and stay zero: a band factor has no fill outside
// the band); L is written over the interior band and 1 / D over its
// diagonal, the border rows and the band entries that reach into the border
// are left as they were.  Lanes 0 .. p then solve B Y_t = C_t (the coupling
// columns of the p border markers) and B z = 1; lanes build the p x p Schur
// complement S = E - C^T Y and 1 - C^T z; lane 0 solves S x = 1 - C^T z; the
// lanes form the interior scales z - Y x.  In the compute precision.
template <typename R>
__device__ __forceinline__ R vb_recip(R x) {
    if constexpr (sizeof(R) == 4) return __frcp_rn(x); else return (R)1 / x;
}

template <typename R>
__device__ __noinline__ void vb_solve(R *A, R *Y, R *eps, R *S, int n, int p) {
    const int lane = threadIdx.x & 31;
    const int m = n - p;
    if (lane == 0) {
        R W[VB_W][VB_W];
#pragma unroll
        for (int a = 0; a < VB_W; ++a)
#pragma unroll
            for (int b = a; b < VB_W; ++b)
                W[a][b] = (b < m) ? A[(size_t)a * VB_W + (b - a)] : (R)0;
#pragma unroll 1
        for (int k = 0; k < m; ++k) {
            const R r = vb_recip(W[0][0]);
            R la[VB_W], w0[VB_W];        // row k as it was before the update
#pragma unroll
            for (int b = 1; b < VB_W; ++b) {
                w0[b] = W[0][b];
                la[b] = w0[b] * r;
            }
            R *ak = A + (size_t)k * VB_W;
            ak[0] = r;
#pragma unroll
            for (int b = 1; b < VB_W; ++b)
                if (b <= p && k + b < m) ak[b] = la[b];
            // trailing update, shifted to the window of step k + 1
#pragma unroll
            for (int a = 0; a < VB_PMAX; ++a)
#pragma unroll
                for (int b = a; b < VB_PMAX; ++b)
                    W[a][b] = W[a + 1][b + 1] - la[a + 1] * w0[b + 1];
            // the window's new last column: column k + 1 + VB_PMAX of B as given
            const int col = k + 1 + VB_PMAX;
#pragma unroll
            for (int a = 0; a < VB_W; ++a)
                W[a][VB_PMAX] = (col < m && k + 1 + a < m)
                                    ? A[(size_t)(k + 1 + a) * VB_W + (VB_PMAX - a)] : (R)0;
        }
    }
    __syncwarp();
    if (lane <= p) {
        R *y = Y + (size_t)lane * n;
        // forward L y = rhs (rhs: coupling column `lane`, or ones), two
        // partial sums per row
        R win[VB_PMAX];
#pragma unroll
        for (int a = 0; a < VB_PMAX; ++a) win[a] = (R)0;
#pragma unroll 1
        for (int i = 0; i < m; ++i) {
            R v = lane == p ? (R)1
                            : ((i <= lane || i >= m + lane - p) ? vb_at(A, n, p, i, m + lane) : (R)0);
            R v2 = (R)0;
#pragma unroll
            for (int a = 1; a <= VB_PMAX; ++a) {
                const R l = i - a >= 0 ? A[(size_t)(i - a) * VB_W + a] : (R)0;
                if (a & 1) v -= l * win[a - 1]; else v2 -= l * win[a - 1];
            }
            v += v2;
#pragma unroll
            for (int a = VB_PMAX - 1; a > 0; --a) win[a] = win[a - 1];
            win[0] = v;
            y[i] = v;
        }
        // D z = y, L^T x = z
#pragma unroll
        for (int a = 0; a < VB_PMAX; ++a) win[a] = (R)0;
#pragma unroll 1
        for (int i = m - 1; i >= 0; --i) {
            const R *ai = A + (size_t)i * VB_W;
            R v = y[i] * ai[0], v2 = (R)0;
#pragma unroll
            for (int a = 1; a <= VB_PMAX; ++a) {
                const R l = i + a < m ? ai[a] : (R)0;
                if (a & 1) v -= l * win[a - 1]; else v2 -= l * win[a - 1];
            }
            v += v2;
#pragma unroll
            for (int a = VB_PMAX - 1; a > 0; --a) win[a] = win[a - 1];
            win[0] = v;
            y[i] = v;
        }
    }
    __syncwarp();
    // Schur complement S[q][r] (q, r < p) and its right-hand side S[q][p]:
    // the coupling C_(i,q) = A_(i, m+q) is non-zero only for i <= q (through
    // the wrap) and i >= m + q - p
    for (int e = lane; e < p * (p + 1); e += 32) {
        const int q = e / (p + 1), r = e - q * (p + 1);
        R acc = r < p ? vb_at(A, n, p, m + q, m + r) : (R)1;
        const R *yr = Y + (size_t)r * n;
        for (int i = 0; i <= q; ++i) acc -= vb_at(A, n, p, i, m + q) * yr[i];
        for (int i = max(m + q - p, q + 1); i < m; ++i) acc -= vb_at(A, n, p, i, m + q) * yr[i];
        S[q * VB_W + r] = acc;
    }
    __syncwarp();
    if (lane == 0) {
        // Gaussian elimination on the small symmetric positive-definite S
#pragma unroll 1
        for (int k = 0; k < p; ++k) {
            const R r = (R)1 / S[k * VB_W + k];
            for (int i = k + 1; i < p; ++i) {
                const R f = S[i * VB_W + k] * r;
                for (int j = k; j <= p; ++j) S[i * VB_W + j] -= f * S[k * VB_W + j];
            }
        }
        for (int k = p - 1; k >= 0; --k) {
            R v = S[k * VB_W + p];
            for (int j = k + 1; j < p; ++j) v -= S[k * VB_W + j] * eps[m + j];
            eps[m + k] = v / S[k * VB_W + k];
        }
    }
    __syncwarp();
    for (int i = lane; i < m; i += 32) {
        R v = Y[(size_t)p * n + i];
        for (int q = 0; q < p; ++q) v -= Y[(size_t)q * n + i] * eps[m + q];
        eps[i] = v;
    }
    __syncwarp();
}

// Reverse probability of Eq. 11 (dt = 1), in FP64 on every storage path:
// k_r = k_r0 exp((sigma - sigma*) d^2 / (2 k_B T)), P_r = 1 - exp(-k_r), with
// d = y_l - y_eq.
__device__ __noinline__ double prob_reverse(double k_r0, double dsig, double kBT2, double dd) {
    const double kr = k_r0 * exp(dsig * dd * dd / kBT2);
    return 1.0 - exp(-kr);
}

// The 256-thread form is capped at 64 registers (a quarter of an SM's), so
// that three bulk-pass CTAs fit beside it.
template <typename S, typename R, int PT>
__global__ void __launch_bounds__(PT, PT == 256 ? 4 : 1) particle_kernel(BatchDev b, int flip,
                                                                         int mode) {
    // mode bit 0: init (IB forcing only, at the current pose); bit 1: a step
    // without the near-box lattice pass
    const int init = mode & 1;
    const bool plain = (mode & 2) != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // descriptors copied to shared memory once: later reads do not wait on
    // global memory, nor get reloaded after the kernel's own global stores
    __shared__ __align__(16) unsigned char s_sim_raw[sizeof(SimDev)];
    __shared__ __align__(16) unsigned char s_par_raw[sizeof(ParticleDev)];
    ParticleDev *P = b.parts[blockIdx.x];
    // this thread's element record, loaded beside the descriptor (used only
    // if the descriptor says it is valid)
    R ev[ECACHE];
    const PartRec prec = b.prec ? b.prec[blockIdx.x] : PartRec{nullptr, 0, 0};
    if (prec.erec && (int)threadIdx.x < prec.nl) {
        const R *e = (const R *)prec.erec + (size_t)threadIdx.x * ECACHE;
#pragma unroll
        for (int k = 0; k < ECACHE; ++k) ev[k] = e[k];
    }
    {
        const int *src_s = (const int *)&b.sims[b.part_sim[blockIdx.x]];
        const int *src_p = (const int *)P;
        for (int i = threadIdx.x; i < (int)(sizeof(SimDev) / 4); i += PT)
            ((int *)s_sim_raw)[i] = src_s[i];
        for (int i = threadIdx.x; i < (int)(sizeof(ParticleDev) / 4); i += PT)
            ((int *)s_par_raw)[i] = src_p[i];
    }
    __syncthreads();
    const SimDev &s = *(const SimDev *)s_sim_raw;
    const ParticleDev &Pc = *(const ParticleDev *)s_par_raw;
    const int nl = Pc.nl, T = Pc.T, Tm = region_edge(T);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void *p = smem_raw + off;
        off += (bytes + 15) & ~size_t(15);
        return p;
    };
    Pose<R> &ps = *(Pose<R> *)take(sizeof(Pose<R>));
    R *gbx = (R *)take(sizeof(R) * nl);     // body-frame centroids, normals, lengths
    R *gby = (R *)take(sizeof(R) * nl);
    R *gnx = (R *)take(sizeof(R) * nl);
    R *gny = (R *)take(sizeof(R) * nl);
    R *sS = (R *)take(sizeof(R) * nl);
    R *rx = (R *)take(sizeof(R) * nl);      // marker offset from the centroid
    R *ry = (R *)take(sizeof(R) * nl);
    R *nxw = (R *)take(sizeof(R) * nl);     // outward normal
    R *nyw = (R *)take(sizeof(R) * nl);
    // per-element loads (0-2) and bond forces (3-5): quantity k at cq + k cstride
    const int cstride = (int)(((sizeof(R) * nl + 15) & ~size_t(15)) / sizeof(R));
    R *cq = (R *)take(6 * sizeof(R) * cstride);
    Points<R> pt;
    pt.ix0 = (int *)take(sizeof(int) * nl);
    pt.iy0 = (int *)take(sizeof(int) * nl);
    pt.rows = (int *)take(sizeof(int) * nl);
    pt.fx = (R *)take(sizeof(R) * nl);
    pt.fy = (R *)take(sizeof(R) * nl);
    pt.invW = (R *)take(sizeof(R) * nl);
    pt.mu = (R *)take(sizeof(R) * nl);
    pt.mu_v = (R *)take(sizeof(R) * nl);
    pt.inv_v = (R *)take(sizeof(R) * nl);
    uint8_t *lig8 = (uint8_t *)take(nl);
    int *corder = (int *)take(sizeof(int) * nl);
    int *coff = (int *)take(sizeof(int) * (nl + 1));
    double *lpart = (double *)take(sizeof(double) * 3 * (PT / 32));   // per-warp gap minima (keys)
    int4 *span = (int4 *)take(sizeof(int4) * Tm);       // staged spans per region row
    int *pre = (int *)take(sizeof(int) * (Tm + 1));     // staged nodes before each row
    R *tile = (R *)take(sizeof(R) * 2 * T * T);
    // staged moments of the band's span nodes in staging order, at most cap of
    // them, last (the spreading contributions follow them when they do not
    // fit in their space)
    const int cap = stage_cap(nl, Tm);
    R *mr = (R *)take(sizeof(R) * (size_t)cap);
    R *mjx = (R *)take(sizeof(R) * (size_t)cap);
    R *mjy = (R *)take(sizeof(R) * (size_t)cap);
    R *spread_own = spread_in_moments<R>(nl, cap) ? nullptr : (R *)take(32 * sizeof(R) * (size_t)nl);
    // solved spreading scales (ib_spread): band of A, interior solutions,
    // scales, Schur complement
    // (the 256-thread form is never launched for a particle that solves its
    // scales; leaving the code out of it keeps its register budget)
    const bool vb = PT >= 512 && s.ib_spread != 0 && Pc.vb_p > 0;
    R *vbA = nullptr, *vbY = nullptr, *vbE = nullptr, *vbS = nullptr;
    if (vb) {
        vbA = (R *)take(sizeof(R) * VB_W * (size_t)nl);
        vbY = (R *)take(sizeof(R) * VB_W * (size_t)nl);
        vbE = (R *)take(sizeof(R) * (size_t)nl);
        vbS = (R *)take(sizeof(R) * VB_PMAX * VB_W);
    }

    const S *__restrict__ pop = (const S *)s.pop[*s.cur ^ flip];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const double yb = s.wall_b == LBIB_WALL_BOUNCE_BACK ? -0.5 : 0.0;
    const double yt = s.wall_t == LBIB_WALL_BOUNCE_BACK ? (double)s.ny - 0.5 : (double)(s.ny - 1);

    if (tid == 0) {
        ps.xc = Pc.xc; ps.yc = Pc.yc; ps.th = Pc.th;
        ps.u = Pc.u; ps.v = Pc.v; ps.om = Pc.om;
        if (Pc.pose_ok) {
            // left by the last pass: the same values set_pose gives
            ps.ixc = Pc.pose_ixc;
            ps.iyc = Pc.pose_iyc;
            ps.fxc = (R)Pc.pose_r[0]; ps.fyc = (R)Pc.pose_r[1];
            ps.cs = (R)Pc.pose_r[2]; ps.sn = (R)Pc.pose_r[3];
            ps.gap0_b = (R)Pc.pose_r[4]; ps.gap0_t = (R)Pc.pose_r[5];
            ps.uR = (R)Pc.pose_r[6]; ps.vR = (R)Pc.pose_r[7]; ps.omR = (R)Pc.pose_r[8];
        } else {
            set_pose(ps, yb, yt);
        }
    }
    // FP64 cosine and sine of the angle for the bond geometry (beside the
    // compute-precision pose of thread 0)
    if (tid == 32 && !init) sincos(Pc.th, &ps.snd, &ps.csd);
    // element of this thread's bond: the upper half of the block takes the
    // bonds when both halves fit the elements, so that they run beside the
    // staging work of the lower half; its body-frame centroid in FP64
    const int kb = 2 * nl <= PT ? tid - PT / 2 : tid;
    const bool kb_ok = !init && (unsigned)kb < (unsigned)nl;
    double bmx = 0.0, bmy = 0.0;
    if (kb_ok) {
        bmx = Pc.mbx[kb];
        bmy = Pc.mby[kb];
    }
    // element data: from the record the last pass left (marker positions at
    // this pose included), else from the geometry arrays
    const bool cached = Pc.pose_ok && Pc.ecache && prec.erec == Pc.ecache;
    R *erec = (R *)Pc.ecache;
    if (tid < nl) {
        if (cached) {
            const R *v = ev;
            gbx[tid] = v[0]; gby[tid] = v[1]; gnx[tid] = v[2]; gny[tid] = v[3];
            sS[tid] = v[4];
            rx[tid] = v[5]; ry[tid] = v[6]; nxw[tid] = v[7]; nyw[tid] = v[8];
            lig8[tid] = (uint8_t)v[9];
            corder[tid] = (int)v[10];
            if (tid < Pc.ncolors) coff[tid] = (int)v[11];
        } else {
            gbx[tid] = (R)Pc.mbx[tid];
            gby[tid] = (R)Pc.mby[tid];
            gnx[tid] = (R)Pc.nbx[tid];
            gny[tid] = (R)Pc.nby[tid];
            sS[tid] = (R)Pc.S[tid];
            lig8[tid] = Pc.ligand[tid];
            corder[tid] = Pc.color_order[tid];
            if (tid < Pc.ncolors) coff[tid] = Pc.color_off[tid];
        }
    }
    if (tid == 0) coff[Pc.ncolors] = nl;     // the last colour ends at nl
    __syncthreads();

    // markers (offsets from the centroid) at the current pose
    auto place = [&]() {
        if (tid < nl) {
            const R cs = ps.cs, sn = ps.sn;
            const R bx = gbx[tid], by = gby[tid];
            rx[tid] = cs * bx - sn * by;
            ry[tid] = sn * bx + cs * by;
            const R nbx = gnx[tid], nby = gny[tid];
            nxw[tid] = cs * nbx - sn * nby;
            nyw[tid] = sn * nbx + cs * nby;
        }
    };
    if (!cached) place();
    const int rx0 = ps.ixc - Tm / 2, ry0 = ps.iyc - Tm / 2;
    for (int v = tid; v < Tm; v += PT) span[v] = make_int4(Tm, -1, Tm, -1);
    // ---- 3. bonds (Eq. 9-11), one element per thread: they need only the
    // pose, so they run with the staging, before the wait on the lattice pass.
    // On every storage path the bond geometry is FP64: the element centroid
    // X_l at the pose of step n, its gaps to the wall lines (probing test and
    // Eq. 12), the bond length and P_r, and the anchor of a new bond, so that
    // the decisions follow the pose to FP64 rounding.
    const bool has_b = s.wall_b != LBIB_WALL_PERIODIC && s.rec_b > 0.0;
    const bool has_t = s.wall_t != LBIB_WALL_PERIODIC && s.rec_t > 0.0;
    bool lig = false, pb = false, ptop = false;
    double Xl = 0.0, Yl = 0.0, gbd = 1e300, gtd = 1e300;
    if (kb_ok) {
        lig = lig8[kb] != 0;
        Xl = ps.xc + (ps.csd * bmx - ps.snd * bmy);
        Yl = ps.yc + (ps.snd * bmx + ps.csd * bmy);
        gbd = Yl - yb;
        gtd = yt - Yl;
        pb = lig && has_b && gbd < s.y_cr;
        ptop = lig && has_t && gtd < s.y_cr;
    }
    const int nprobe = __syncthreads_count(pb || ptop);

    // ---- stage the moments of the nodes the supports can touch ------------
    // The supports of a marker's probe and of the marker itself after a move
    // below one node lie in the bounding box of the probe's 4 x 4 support and
    // a 6 x 6 box around the marker's own.  Per region row, the boxes of the
    // markers whose outward normal points left (the outline runs down there)
    // make one span and the others a second; along a convex outline each of
    // these chains is monotone in y, so a span is an interval of the row (any
    // support node outside the staged nodes is pulled directly, with the same
    // arithmetic).  The nodes of the spans are counted per row and pulled.
    if (tid < nl) {
        const R X = ps.fxc + rx[tid], Y = ps.fyc + ry[tid];
        int bx0 = (int)floor(X) - 2, by0 = (int)floor(Y) - 2;
        int bx1 = bx0 + 5, by1 = by0 + 5;
        if (!init) {
            // the probe's MLS support needs only the pose: set up here, beside
            // the bond kinetics of the upper half of the block
            setup_point<R>(s, ps.ixc, ps.iyc, X + (R)1.2 * nxw[tid], Y + (R)1.2 * nyw[tid], pt, tid);
            const int px0 = (int)floor(X + (R)1.2 * nxw[tid]) - 1;
            const int py0 = (int)floor(Y + (R)1.2 * nyw[tid]) - 1;
            bx0 = min(bx0, px0);
            by0 = min(by0, py0);
            bx1 = max(bx1, px0 + 3);
            by1 = max(by1, py0 + 3);
        }
        const int h = Tm / 2;       // region coordinate of the centroid's floor node
        const int ulo = max(bx0 + h, 0), uhi = min(bx1 + h, Tm - 1);
        int *sp = (int *)span + (nxw[tid] < (R)0 ? 0 : 2);
        if (ulo <= uhi) {
#pragma unroll 1
            for (int v = max(by0 + h, 0); v <= min(by1 + h, Tm - 1); ++v) {
                const int yy = ry0 + v;
                if (s.wall_b != LBIB_WALL_PERIODIC && (yy < 0 || yy >= s.ny)) continue;
                atomicMin(sp + 4 * v, ulo);
                atomicMax(sp + 4 * v + 1, uhi);
            }
        }
    }
    bool bonded = false;
    if (kb_ok) {
        const int l = kb;
        double fx = 0.0, fy = 0.0;
        if (lig) {
            // one draw per (step, element); the step is this particle's count
            const double U = bond_uniform(s, Pc.step, (int)blockIdx.x - s.p0, l);
            uint8_t bnd = P->bond[l];
            double ax = P->anchor_x[l];
            int8_t aw = P->anchor_wall[l];
            const double y_eq = s.y_eq_ratio * s.y_cr;
            // bond vector anchor - X_l (the anchor lies on a wall line) and
            // length: of a bond that stays, as its reverse draw saw it; of a
            // new one, straight to its wall line (the anchor is at x = X_l)
            double dx = 0.0, dy = 0.0, y = 0.0;
            if (bnd) {
                dx = ax - Xl;
                dy = (aw ? yt : yb) - Yl;
                y = sqrt(dx * dx + dy * dy);
                const double Pr = prob_reverse(s.k_r0, Pc.sigma - s.sigma_star_ratio * Pc.sigma,
                                               2.0 * s.kBT, y - y_eq);
                if (U < Pr) bnd = 0;
            } else if (pb || ptop) {
                if (U < Pc.pf_tab[pb ? nprobe : nl + 1 + nprobe]) {
                    bnd = 1;
                    ax = Xl;
                    aw = pb ? 0 : 1;
                    P->anchor_x[l] = ax;
                    P->anchor_wall[l] = aw;
                    dx = ax - Xl;
                    dy = (aw ? yt : yb) - Yl;
                    y = sqrt(dx * dx + dy * dy);
                }
            }
            P->bond[l] = bnd;
            if (bnd) {
                bonded = true;
                if (y > 0.0) {
                    const double q = Pc.sigma * (y - y_eq) / y;     // one FP64 division
                    fx = q * dx;
                    fy = q * dy;
                }
            }
        }
        cq[3 * cstride + l] = (R)fx;
        cq[4 * cstride + l] = (R)fy;
        cq[5 * cstride + l] = (R)((Xl - ps.xc) * fy - (Yl - ps.yc) * fx);
    }
    if (!init) {
        // smallest element gaps to each wall line (Eq. 12): exact minima of
        // the FP64 gaps as order-preserving 64-bit integer keys (integer
        // instructions: an FP64 minimum costs ~64 cycles of its
        // sub-partition per warp), per warp by shuffles, the warps' minima in
        // the per-warp space
        long long mb = gap_key(gbd), mt = gap_key(gtd);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mb = min(mb, __shfl_xor_sync(0xffffffffu, mb, o));
            mt = min(mt, __shfl_xor_sync(0xffffffffu, mt, o));
        }
        if (lane == 0) {
            ((long long *)lpart)[2 * warp] = mb;
            ((long long *)lpart)[2 * warp + 1] = mt;
        }
    }
    const int nbonded = __syncthreads_count(bonded);
    // merge overlapping spans, count the nodes of each row, prefix sum (one warp)
    if (warp == 0) {
        int carry = 0;
        for (int base = 0; base < Tm; base += 32) {
            const int v = base + lane;
            int cnt = 0;
            if (v < Tm) {
                int4 q = span[v];
                if (q.y >= q.x && q.w >= q.z && q.z <= q.y + 1 && q.x <= q.w + 1)
                    q = make_int4(min(q.x, q.z), max(q.y, q.w), Tm, -1);
                span[v] = q;
                cnt = max(q.y - q.x + 1, 0) + max(q.w - q.z + 1, 0);
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (v < Tm) pre[v] = carry + incl - cnt;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) pre[Tm] = carry;
    } else if (!init && warp == 1) {
        if (lane == 0) {
            long long kb_ = gap_key(1e300), kt_ = gap_key(1e300);
            for (int w = 0; w < PT / 32; ++w) {
                kb_ = min(kb_, ((const long long *)lpart)[2 * w]);
                kt_ = min(kt_, ((const long long *)lpart)[2 * w + 1]);
            }
            ps.nprobe = nprobe;
            ps.nbonded = nbonded;
            ps.gapb = key_gap(kb_);
            ps.gapt = key_gap(kt_);
        }
    }
    __syncthreads();
    // populations of this step come from the lattice pass just before: wait
    // for it here (everything above reads only particle and geometry data)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int nlist = min(pre[Tm], cap);
    // the last warp, meanwhile: the FP64 sums of the bond loads and the wall
    // force (only the rigid update below needs them)
    constexpr int SW = PT / 32 - 1;
    if (warp == SW) {
        if (!init) {
#pragma unroll 1
            for (int q = 3; q < 6; ++q) {
                const double v = warp_sum_array<R>(cq + q * cstride, nl);
                if (lane == 0) ps.F[q] = v;
            }
            if (lane == 0) {
                // ---- 4. wall force (Eq. 12), FP64 ---------------------
                // F_w = H_k / (8 sqrt 2) sqrt(r / eps^5) off each wall, eps
                // the smallest element gap clamped below by eps_min
                double Fw = 0.0;
                if (s.wall_b != LBIB_WALL_PERIODIC && s.hamaker != 0.0) {
                    const double eb = fmax(ps.gapb, s.eps_min), et = fmax(ps.gapt, s.eps_min);
                    const double k = s.hamaker / (8.0 * 1.4142135623730951);
                    Fw = k * sqrt(Pc.r_eq / (eb * eb * eb * eb * eb)) -
                         k * sqrt(Pc.r_eq / (et * et * et * et * et));
                }
                ps.Fw = Fw;
            }
        }
    } else
#pragma unroll 2
    for (int k = tid; k < nlist; k += PT - 32) {
        // staged node k: row v is the last with pre[v] <= k, then its spans
        int lo = 0, hi = Tm;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pre[mid] <= k) lo = mid; else hi = mid;
        }
        const int v = lo;
        const int4 q = span[v];
        const int n0 = max(q.y - q.x + 1, 0), o = k - pre[v];
        const int u = o < n0 ? q.x + o : q.z + (o - n0);
        const int i = k;
        int xx = (rx0 + u) % s.nx;
        if (xx < 0) xx += s.nx;
        int yy = ry0 + v;
        if (s.wall_b == LBIB_WALL_PERIODIC) {
            yy %= s.ny;
            if (yy < 0) yy += s.ny;
        }
        if (!s.aa && (s.wall_b == LBIB_WALL_PERIODIC || (yy >= 1 && yy <= s.ny - 2))) {
            // interior node: nine plain pulls from rows yy - 1, yy, yy + 1
            const int nx = s.nx, N = nx * s.ny;
            const float inv = s.inv_scale;
            const int xm = xx == 0 ? nx - 1 : xx - 1, xp = xx == nx - 1 ? 0 : xx + 1;
            const int ym = yy == 0 ? s.ny - 1 : yy - 1, yp = yy == s.ny - 1 ? 0 : yy + 1;
            const int r0 = yy * nx, rm = ym * nx, rp = yp * nx;
            R d[9];
            auto ldp = [&](int i) { return Store<S>::ld(pop, pop_load_index(s, i), inv); };
            d[0] = ldp(r0 + xx);
            d[1] = ldp(N + r0 + xm);
            d[3] = ldp(3 * N + r0 + xp);
            d[2] = ldp(2 * N + rm + xx);
            d[5] = ldp(5 * N + rm + xm);
            d[6] = ldp(6 * N + rm + xp);
            d[4] = ldp(4 * N + rp + xx);
            d[7] = ldp(7 * N + rp + xp);
            d[8] = ldp(8 * N + rp + xm);
            node_moments(d, mr[i], mjx[i], mjy[i]);
        } else {
            const Moments<R> m = pull_moments<S, R>(s, pop, xx, yy, flip);
            mr[i] = m.drho;
            mjx[i] = m.jx;
            mjy[i] = m.jy;
        }
    }
    __syncthreads();

    if (!init) {
        // ---- 2. hydrodynamic loads (Eq. 7-8), one thread per probe --------
        const R nu = pick<R>(s.f_nu, s.d_nu);
        R tx = 0, ty = 0, tq = 0;
        if (tid < nl) {
            const int l = tid;
            // (its support was set up with the staging)
            R s_rho = 0, s_ux = 0, s_uy = 0, s_vx = 0, s_vy = 0;
            support_sum<S, R>(s, pop, flip, pt, l, mr, mjx, mjy, span, pre, cap, Tm, rx0, ry0,
                              [&](R w, R dx, R dyc, R phi, R drho, R jx, R jy) {
                                  const R irho = recip_rho((R)1 + drho);
                                  const R ux = jx * irho, uy = jy * irho;
                                  s_rho += phi * drho;
                                  s_ux += w * dx * ux;
                                  s_uy += w * dyc * ux;
                                  s_vx += w * dx * uy;
                                  s_vy += w * dyc * uy;
                              });
            if (pt.rows[l] & 16) {
                const R iv = pt.inv_v[l];
                const R dudx = (R)3 * s_ux, dudy = s_uy * iv;
                const R dvdx = (R)3 * s_vx, dvdy = s_vy * iv;
                const R p = s_rho * (R)(1.0 / 3.0);
                const R nxl = nxw[l], nyl = nyw[l];
                const R txy = nu * (dudy + dvdx);
                tx = (-p * nxl + nu * (R)2 * dudx * nxl + txy * nyl) * sS[l];
                ty = (-p * nyl + txy * nxl + nu * (R)2 * dvdy * nyl) * sS[l];
            }
            tq = rx[l] * ty - ry[l] * tx;
            cq[l] = tx;
            cq[cstride + l] = ty;
            cq[2 * cstride + l] = tq;
        }
        __syncthreads();
        // ---- 5. rigid update (Eq. 13-16), one degree of freedom per warp ---
        // Warp k sums load k over the probes in FP64 (the bond loads and the
        // wall force were summed during the staging), then its lane 0 updates
        // degree of freedom k: the three chains of FP64 arithmetic run side by
        // side, and only three warps issue FP64 instructions (each occupies
        // its sub-partition's FP64 pipe for ~64 cycles whatever its lanes).
        if (warp < 3) {
            const int k = warp;
            const double h = warp_sum_array<R>(cq + k * cstride, nl);
            if (lane == 0) {
                ps.F[k] = h;
                if (k == 2) P->Mh = h; else P->Fh[k] = h;
                if (!Pc.fixed) {
                    const double F = k == 0 ? h + ps.F[3] : (k == 1 ? h + ps.F[4] + ps.Fw : h + ps.F[5]);
                    const double im = k == 2 ? Pc.inv_inertia : Pc.inv_mass;
                    const double u0 = k == 0 ? ps.u : (k == 1 ? ps.v : ps.om);
                    const double u1 = k == 0 ? Pc.u1 : (k == 1 ? Pc.v1 : Pc.om1);
                    const double x0 = k == 0 ? ps.xc : (k == 1 ? ps.yc : ps.th);
                    const double x1 = k == 0 ? Pc.xc1 : (k == 1 ? Pc.yc1 : Pc.th1);
                    const double un = 2.0 / 3.0 * (2.0 * u0 - 0.5 * u1 + F * im);
                    const double xn = (4.0 * x0 - x1 + 2.0 * un) * (1.0 / 3.0);
                    double *Pu = k == 0 ? &P->u : (k == 1 ? &P->v : &P->om);
                    double *Pu1 = k == 0 ? &P->u1 : (k == 1 ? &P->v1 : &P->om1);
                    double *Px = k == 0 ? &P->xc : (k == 1 ? &P->yc : &P->th);
                    double *Px1 = k == 0 ? &P->xc1 : (k == 1 ? &P->yc1 : &P->th1);
                    *Pu1 = u0; *Pu = un; *Px1 = x0; *Px = xn;
                    if (k == 0) { ps.u = un; ps.xc = xn; }
                    if (k == 1) { ps.v = un; ps.yc = xn; }
                    if (k == 2) { ps.om = un; ps.th = xn; }
                    set_pose_dof(ps, k, yb, yt);     // this degree of freedom of the new pose
                }
            }
        }
        if (tid == 96) {
            P->Fb[0] = ps.F[3]; P->Fb[1] = ps.F[4]; P->Mb = ps.F[5];
            P->Fw[0] = 0.0; P->Fw[1] = ps.Fw;
            P->gap[0] = ps.gapb; P->gap[1] = ps.gapt;
            P->n_probing = ps.nprobe;
            P->n_bonded = ps.nbonded;
        }
        __syncthreads();
        place();
    }

    // ---- 6. IB direct forcing at the (new) pose ---------------------------
    const R ghx = (R)0.5 * pick<R>(s.f_gx, s.gx), ghy = (R)0.5 * pick<R>(s.f_gy, s.gy);
    R Fx = 0, Fy = 0;
    if (tid < nl)
        setup_point<R>(s, ps.ixc, ps.iyc, ps.fxc + rx[tid], ps.fyc + ry[tid], pt, tid);
    // solved spreading scales: every marker's row of A once all supports are
    // set up, then one warp solves A eps = 1 -- the last warp, beside the
    // interpolation below, when it holds no marker
    const int vb_warp = nl + 32 <= PT ? PT / 32 - 1 : 0;
    const bool vb_beside = nl + 32 <= PT;
    if (vb) {
        __syncthreads();
        if (tid < nl) vb_row<R>(pt, tid, nl, Pc.vb_p, vbA);
        __syncthreads();
        if (vb_beside && warp == vb_warp) vb_solve<R>(vbA, vbY, vbE, vbS, nl, Pc.vb_p);
    }
    if (tid < nl) {
        const int l = tid;
        R s_rho = 0, s_u = 0, s_v = 0;
        support_sum<S, R>(s, pop, flip, pt, l, mr, mjx, mjy, span, pre, cap, Tm, rx0, ry0,
                          [&](R, R, R, R phi, R drho, R jx, R jy) {
                              const R irho = recip_rho((R)1 + drho);
                              s_rho += phi * drho;
                              s_u += phi * ((jx + ghx) * irho);
                              s_v += phi * ((jy + ghy) * irho);
                          });
        if (pt.rows[l] & 16) {
            const R rl = (R)1 + s_rho;
            const R udx = ps.uR - ps.omR * ry[l];
            const R udy = ps.vR + ps.omR * rx[l];
            Fx = (R)2 * rl * (udx - s_u);
            Fy = (R)2 * rl * (udy - s_v);
        }
    }
    if (vb) {
        if (!vb_beside && warp == vb_warp) vb_solve<R>(vbA, vbY, vbE, vbS, nl, Pc.vb_p);
        __syncthreads();
    }
    // the spreading scale eps_l: the element length, or the solved scale
    const R el = tid < nl ? (vb ? vbE[tid] : sS[tid]) : (R)0;
    Fx *= el;
    Fy *= el;
    // the near-box pass of the next step may be scheduled from here on (it
    // waits for this pass to end before it reads the tiles)
    asm volatile("griddepcontrol.launch_dependents;");
    using R2 = typename Pair<R>::type;
    R2 *ctb = spread_in_moments<R>(nl, cap) ? (R2 *)mr : (R2 *)spread_own;
    const int ox = ps.ixc - T / 2;
    const int oy = ps.iyc - T / 2;
    auto marker_phi = [&](int l, R wx[4], R py[4]) { point_phi(pt, l, wx, py); };
    // one spreading pass of the markers' forces (Fx, Fy) into a zeroed tile
    auto spread_pass = [&]() {
        // a zero tile for the spreading (T is even: whole 16-byte words)
        for (int i = tid; i < (int)(2 * sizeof(R) * T * T / 16); i += PT)
            ((uint4 *)tile)[i] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        // each marker's sixteen contributions phi_k F_l eps_l, in the staged
        // moments' space once every support has been read (or a buffer of
        // their own when they do not fit there)
        if (tid < nl) {
            R wx[4], py[4];
            marker_phi(tid, wx, py);
#pragma unroll 1
            for (int b = 0; b < 4; ++b) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const R phi = wx[a] * py[b];
                    R2 c;
                    c.x = phi * Fx;
                    c.y = phi * Fy;
                    ctb[tid * 16 + b * 4 + a] = c;
                }
            }
        }
        __syncthreads();
        // colour-ordered spreading into the tile; origin floor(X_c) - T/2.
        // Markers of one colour have disjoint supports, so each tile node
        // takes its contributions in colour order (identical alone or in a
        // batch).
#pragma unroll 1
        for (int cl = 0; cl < Pc.ncolors; ++cl) {
            const int m0 = coff[cl], m1 = coff[cl + 1];
            for (int t = tid; t < (m1 - m0) * 16; t += PT) {
                const int m = corder[m0 + (t >> 4)];
                const int j = t & 15;
                const R2 c = ctb[m * 16 + j];
                if (c.x == (R)0 && c.y == (R)0) continue;
                const int tx = pt.ix0[m] + (j & 3) - ox, ty = pt.iy0[m] + (j >> 2) - oy;
                if ((unsigned)tx < (unsigned)T && (unsigned)ty < (unsigned)T) {
                    tile[ty * T + tx] += c.x;
                    tile[T * T + ty * T + tx] += c.y;
                }
            }
            __syncthreads();
        }
    };
    spread_pass();
    // multi-direct forcing: the slip each marker sees once this particle's
    // force is spread, corrected M - 1 more times, F <- F + F0 - eps_l I_l[f]
    // (F carries eps_l = S_l; I_l[f] = sum_k phi_k f_k over the tile)
    const R F0x = Fx, F0y = Fy;
#pragma unroll 1
    for (int it = 1; it < s.ib_iters; ++it) {
        if (tid < nl && (pt.rows[tid] & 16)) {
            R wx[4], py[4];
            marker_phi(tid, wx, py);
            R ix = 0, iy = 0;
#pragma unroll 1
            for (int b = 0; b < 4; ++b) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int tx = pt.ix0[tid] + a - ox, ty = pt.iy0[tid] + b - oy;
                    if ((unsigned)tx < (unsigned)T && (unsigned)ty < (unsigned)T) {
                        const R phi = wx[a] * py[b];
                        ix += phi * tile[ty * T + tx];
                        iy += phi * tile[T * T + ty * T + tx];
                    }
                }
            }
            Fx += F0x - el * ix;
            Fy += F0y - el * iy;
        }
        __syncthreads();    // every read of the tile before it is zeroed
        spread_pass();
    }
    R *gt = (R *)Pc.tile;
    for (int i = tid; i < (int)(2 * sizeof(R) * T * T / 16); i += PT)
        ((uint4 *)gt)[i] = ((const uint4 *)tile)[i];
    if (tid == 0) {
        int oxw = ox % s.nx;
        if (oxw < 0) oxw += s.nx;
        int oyw = oy;
        if (s.wall_b == LBIB_WALL_PERIODIC) {
            oyw %= s.ny;
            if (oyw < 0) oyw += s.ny;
        }
        P->tile_ox = oxw;
        P->tile_oy = oyw;
        // near box of the lattice step after next: its core centred on the
        // new pose, the box's x origin rounded down to a multiple of four
        const int half = near_core(Pc.T) / 2;
        int bx = (ps.ixc - half) % s.nx;
        if (bx < 0) bx += s.nx;
        bx &= ~3;
        int by = ps.iyc - half;
        if (s.wall_b == LBIB_WALL_PERIODIC) {
            by %= s.ny;
            if (by < 0) by += s.ny;
        }
        P->pend_ox = bx;
        P->pend_oy = by;
        if (init || plain) {
            // before the first step (or when no near pass publishes boxes)
            // both lattice steps use the box around the latest pose
            P->box_ox[0] = P->box_ox[1] = bx;
            P->box_oy[0] = P->box_oy[1] = by;
        }
        if (!init) P->step = Pc.step + 1;
        // the pose of the next pass (unchanged for a fixed particle)
        P->pose_ixc = ps.ixc;
        P->pose_iyc = ps.iyc;
        P->pose_r[0] = (double)ps.fxc; P->pose_r[1] = (double)ps.fyc;
        P->pose_r[2] = (double)ps.cs; P->pose_r[3] = (double)ps.sn;
        P->pose_r[4] = (double)ps.gap0_b; P->pose_r[5] = (double)ps.gap0_t;
        P->pose_r[6] = (double)ps.uR; P->pose_r[7] = (double)ps.vR; P->pose_r[8] = (double)ps.omR;
        P->pose_ok = 1;
    }
    // the element record for the next pass (markers placed at the latest pose)
    if (erec && tid < nl) {
        R *e = erec + (size_t)tid * ECACHE;
        R v[ECACHE];
        v[0] = gbx[tid]; v[1] = gby[tid]; v[2] = gnx[tid]; v[3] = gny[tid]; v[4] = sS[tid];
        v[5] = rx[tid]; v[6] = ry[tid]; v[7] = nxw[tid]; v[8] = nyw[tid];
        v[9] = (R)lig8[tid];
        v[10] = (R)corder[tid];
        v[11] = tid < Pc.ncolors ? (R)coff[tid] : (R)0;
#pragma unroll
        for (int k = 0; k < ECACHE; ++k) e[k] = v[k];
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

int particle_smem_bytes(int kind, int T, int nl, bool vb) {
    return (int)(kind == ST_F64 ? smem_bytes_for<double>(nl, T, vb)
                                : smem_bytes_for<float>(nl, T, vb));
}

// Largest dynamic shared memory the particle kernel can use: the device's
// opt-in per-block limit minus the kernel's static shared memory.
int particle_smem_limit(int kind) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaFuncAttributes fa{};
    cudaError_t e = by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        return cudaFuncGetAttributes(&fa, particle_kernel<S, R, P_THREADS>);
    });
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return optin - (int)fa.sharedSizeBytes;
}

cudaError_t particle_kernel_setup(int kind, int smem) {
    return by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        cudaError_t e = cudaFuncSetAttribute(particle_kernel<S, R, P_THREADS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if constexpr (sizeof(S) <= 4) {
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(particle_kernel<S, R, 256>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        }
        return e;
    });
}

cudaError_t launch_particles(int kind, const BatchDev &b, int flip, int mode, int smem,
                             cudaStream_t st, bool pdl) {
    if (b.nparts == 0) return cudaSuccess;
    return by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        // the 256-thread form when every particle fits (FP32 / 16-bit storage)
        const bool narrow = sizeof(S) <= 4 && b.pthreads == 256;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(b.nparts);
        cfg.blockDim = dim3(narrow ? 256 : P_THREADS);
        cfg.dynamicSmemBytes = (size_t)smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pdl ? 1 : 0;
        if constexpr (sizeof(S) <= 4) {
            if (narrow) return cudaLaunchKernelEx(&cfg, particle_kernel<S, R, 256>, b, flip, mode);
        }
        return cudaLaunchKernelEx(&cfg, particle_kernel<S, R, P_THREADS>, b, flip, mode);
    });
}

}  // namespace lbib
