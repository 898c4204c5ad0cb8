// lbib_lattice.cu -- fused stream-collide kernel over a batch of lattices,
// plus the small export/import kernels used by the read/write calls.
//
// One thread per node.  A node pulls its nine pre-collision populations from
// the post-collision buffer (Eq. 1 LHS, walls in pull_node), takes the
// moments of Eq. 5-6 with the half-force of the uniform body force g plus the
// IB force density f_ib of any particle tile covering it, relaxes to the
// equilibrium of Eq. 2 and adds the Guo source of Eq. 4, and writes its nine
// post-collision deviations to the other buffer.  Algorithmic traffic: 9
// reads + 9 writes of the storage type per node (72 B in FP32).
#include "lbib_internal.cuh"

namespace lbib {

namespace {

template <typename R>
__device__ __forceinline__ R recip(R x) {
    if constexpr (sizeof(R) == 4) return __frcp_rn(x); else return (R)1 / x;
}

// BGK collision with the Guo source (Eq. 1, 2, 4-6) of one node, in
// deviation form: d holds the pre-collision deviations on entry and the
// post-collision ones on return.  SC: d holds the deviations times the
// storage scale (16-bit storage, as loaded and stored without conversion):
// the three moments are scaled down, and omega and the Guo prefactor, which
// enter only the terms added to d, are scaled up once per thread, instead
// of nine multiplications on load and nine on store.  The scale is a power
// of two (unless the caller set another), so every rounding is the same as
// in the unscaled form.
// FAST (16-bit storage, whose rounding dominates its error): the compact
// pairwise form below.  Otherwise (FP32 / FP64 storage) the form that keeps
// the rounding of slow transients unbiased:
//  - the first-order (momentum) terms take weights W1 (axes) and W5
//    (diagonals) with 2 W1 + 4 W5 = 1 exactly in the compute precision, so
//    the equilibrium momentum is rho u to rounding; with 3 w_i rounded
//    separately it is (1 + 3e-8) rho u, the same excess at every node and
//    step, which in a flow driven by a body force of ~1e-7 per step grows
//    into a velocity error of ~5e-5 after 2000 steps;
//  - the Guo source is added as a term of its own, not rounded inside the
//    ~10^4 times larger equilibrium term, where it loses ~1e-4 of itself.
// Every product and sum of the collision is an explicit correctly rounded
// operation (no contraction left to the compiler), so a node's result is the
// same bits in every lattice path -- the four-node vector form, the per-node
// forms, the near-box pass, A/B or in-place streaming -- whatever the code
// around it.
template <typename R> __device__ __forceinline__ R op_mul(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fmul_rn(a, b); else return __dmul_rn(a, b);
}
template <typename R> __device__ __forceinline__ R op_add(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fadd_rn(a, b); else return __dadd_rn(a, b);
}
template <typename R> __device__ __forceinline__ R op_sub(R a, R b) {
    if constexpr (sizeof(R) == 4) return __fsub_rn(a, b); else return __dsub_rn(a, b);
}
template <typename R> __device__ __forceinline__ R op_fma(R a, R b, R c) {
    if constexpr (sizeof(R) == 4) return __fmaf_rn(a, b, c); else return __fma_rn(a, b, c);
}

// Two FP32 nodes side by side (float2): the sm_100 family's paired FFMA2 /
// FADD2 / FMUL2, per component the correctly rounded FP32 operation of the
// scalar form (a - b as fma(b, -1, a), rounded once as the subtraction), so
// each node of a pair gets the bits it gets alone, with half the
// instructions.
__device__ __forceinline__ float2 op_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 op_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 op_sub(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 op_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Scalar type of a lane and broadcast of a scalar.
template <typename V> struct Lane;
template <> struct Lane<float> {
    using S = float;
    static __device__ __forceinline__ float bc(float x) { return x; }
    static __device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
    static __device__ __forceinline__ bool bad(float drho, float ux, float uy) {
        return !(fabsf(drho) < 1.f) | !(fabsf(ux) + fabsf(uy) < 10.f);
    }
};
template <> struct Lane<double> {
    using S = double;
    static __device__ __forceinline__ double bc(double x) { return x; }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ bool bad(double drho, double ux, double uy) {
        return !(fabs(drho) < 1.0) | !(fabs(ux) + fabs(uy) < 10.0);
    }
};
template <> struct Lane<float2> {
    using S = float;
    static __device__ __forceinline__ float2 bc(float x) { return make_float2(x, x); }
    static __device__ __forceinline__ float2 rcp(float2 x) {
        return make_float2(__frcp_rn(x.x), __frcp_rn(x.y));
    }
    static __device__ __forceinline__ bool bad(float2 drho, float2 ux, float2 uy) {
        return Lane<float>::bad(drho.x, ux.x, uy.x) | Lane<float>::bad(drho.y, ux.y, uy.y);
    }
};

// The collision of one node (V = R) or of two FP32 nodes (V = float2);
// forced: F != 0 (the same for both nodes of a pair).
template <typename V, bool SC, bool FAST>
__device__ __forceinline__ void collide_core(const SimDev &s, V d[9], V Fx, V Fy, bool forced,
                                             bool &bad) {
    using R = typename Lane<V>::S;
    auto C = [](R x) { return Lane<V>::bc(x); };
    // moments (Eq. 5-6) in the order of node_moments
    V drho = op_add(op_add(op_add(d[0], d[1]), op_add(d[2], d[3])),
                    op_add(op_add(d[4], d[5]), op_add(d[6], d[7])));
    drho = op_add(drho, d[8]);
    V jx = op_add(op_add(op_sub(d[1], d[3]), op_sub(d[5], d[6])), op_sub(d[8], d[7]));
    V jy = op_sub(op_add(op_sub(d[2], d[4]), op_add(d[5], d[6])), op_add(d[7], d[8]));
    if constexpr (SC) {
        const V inv = C((R)s.inv_scale);
        drho = op_mul(drho, inv);
        jx = op_mul(jx, inv);
        jy = op_mul(jy, inv);
    }
    const V rho = op_add(C((R)1), drho);
    const V irho = Lane<V>::rcp(rho);
    const R om = pick<R>(s.f_om, s.d_om);
    const R pref0 = pick<R>(s.f_pref, s.d_pref);
    const R oms_s = SC ? op_mul(om, (R)s.scale) : om, pref_s = SC ? op_mul(pref0, (R)s.scale) : pref0;
    const V oms = C(oms_s), pref = C(pref_s), c = C(op_sub((R)1, om));
    // f^eq_i - w_i = w_i [A + 3 rho e.u + 4.5 rho (e.u)^2], A = (rho - 1) - 1.5 rho u.u
    // Guo: S_i = (1 - 1/2tau) w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F
    // Post-collision d_i (1 - om) + om (f^eq_i - w_i) + S_i, evaluated per pair
    // of opposite directions (e -> -e flips e.u and e.F): a part even in e,
    //   w [om A - 3 pref u.F] + 4.5 w (e.u) (om rho (e.u) + 2 pref (e.F)),
    // and an odd part 3 w (om rho (e.u) + pref (e.F)).
    // A node without force (F = 0 exactly: the bulk of a channel driven by
    // its walls alone) takes the same expressions with the force terms left
    // out, which are zero; the choice depends on F alone, so every path
    // takes the same one for a node.
    V ux, uy;
    if (forced) {
        ux = op_mul(op_fma(C((R)0.5), Fx, jx), irho);
        uy = op_mul(op_fma(C((R)0.5), Fy, jy), irho);
    } else {
        ux = op_mul(jx, irho);
        uy = op_mul(jy, irho);
    }
    const V A = op_fma(op_mul(C((R)-1.5), rho), op_fma(ux, ux, op_mul(uy, uy)), drho);
    if (forced) {
        const V uF = op_fma(ux, Fx, op_mul(uy, Fy));
        if constexpr (FAST) {
            const V orho = op_mul(oms, rho), p2 = C(op_mul((R)2, pref_s));
            const V base = op_fma(oms, A, op_mul(C(op_mul((R)-3, pref_s)), uF));
            d[0] = op_fma(c, d[0], op_mul(C((R)(4.0 / 9.0)), base));
            auto pair = [&](int i, int j, R w, V eu, V eF) {
                const V inner = op_fma(orho, eu, op_mul(p2, eF));
                const V even = op_mul(C(w), op_fma(op_mul(C((R)4.5), eu), inner, base));
                const V odd = op_mul(C(op_mul((R)3, w)), op_fma(orho, eu, op_mul(pref, eF)));
                d[i] = op_add(op_fma(c, d[i], even), odd);
                d[j] = op_sub(op_fma(c, d[j], even), odd);
            };
            pair(1, 3, (R)(1.0 / 9.0), ux, Fx);
            pair(2, 4, (R)(1.0 / 9.0), uy, Fy);
            pair(5, 7, (R)(1.0 / 36.0), op_add(ux, uy), op_add(Fx, Fy));
            pair(6, 8, (R)(1.0 / 36.0), op_sub(uy, ux), op_sub(Fy, Fx));
        } else {
            const R W1s = (R)(1.0 / 3.0), W5s = op_mul(op_sub((R)1, op_mul((R)2, W1s)), (R)0.25);
            const V r45 = op_mul(C((R)4.5), rho), m3uF = op_mul(C((R)-3), uF);
            const R w0 = (R)(4.0 / 9.0);
            d[0] = op_fma(c, d[0], op_fma(oms, op_mul(C(w0), A), op_mul(pref, op_mul(C(w0), m3uF))));
            // pair (i, j = opposite of i): even part w (om A' + pref S_even),
            // odd part W (om rho (e.u) + pref (e.F))
            auto pair = [&](int i, int j, R w, R W, V eu, V eF) {
                const V ee = op_mul(oms, op_mul(C(w), op_fma(op_mul(r45, eu), eu, A)));
                const V oo = op_mul(oms, op_mul(C(W), op_mul(rho, eu)));
                const V se = op_mul(pref, op_mul(C(w), op_fma(op_mul(C((R)9), eu), eF, m3uF)));
                const V so = op_mul(pref, op_mul(C(W), eF));
                d[i] = op_add(op_fma(c, d[i], op_add(ee, oo)), op_add(se, so));
                d[j] = op_add(op_fma(c, d[j], op_sub(ee, oo)), op_sub(se, so));
            };
            pair(1, 3, (R)(1.0 / 9.0), W1s, ux, Fx);
            pair(2, 4, (R)(1.0 / 9.0), W1s, uy, Fy);
            pair(5, 7, (R)(1.0 / 36.0), W5s, op_add(ux, uy), op_add(Fx, Fy));
            pair(6, 8, (R)(1.0 / 36.0), W5s, op_sub(uy, ux), op_sub(Fy, Fx));
        }
    } else {
        if constexpr (FAST) {
            const V orho = op_mul(oms, rho);
            const V base = op_mul(oms, A);
            d[0] = op_fma(c, d[0], op_mul(C((R)(4.0 / 9.0)), base));
            auto pair = [&](int i, int j, R w, V eu) {
                const V inner = op_mul(orho, eu);
                const V even = op_mul(C(w), op_fma(op_mul(C((R)4.5), eu), inner, base));
                const V odd = op_mul(C(op_mul((R)3, w)), inner);
                d[i] = op_add(op_fma(c, d[i], even), odd);
                d[j] = op_sub(op_fma(c, d[j], even), odd);
            };
            pair(1, 3, (R)(1.0 / 9.0), ux);
            pair(2, 4, (R)(1.0 / 9.0), uy);
            pair(5, 7, (R)(1.0 / 36.0), op_add(ux, uy));
            pair(6, 8, (R)(1.0 / 36.0), op_sub(uy, ux));
        } else {
            const R W1s = (R)(1.0 / 3.0), W5s = op_mul(op_sub((R)1, op_mul((R)2, W1s)), (R)0.25);
            const V r45 = op_mul(C((R)4.5), rho);
            const R w0 = (R)(4.0 / 9.0);
            d[0] = op_fma(c, d[0], op_mul(oms, op_mul(C(w0), A)));
            auto pair = [&](int i, int j, R w, R W, V eu) {
                const V ee = op_mul(oms, op_mul(C(w), op_fma(op_mul(r45, eu), eu, A)));
                const V oo = op_mul(oms, op_mul(C(W), op_mul(rho, eu)));
                d[i] = op_fma(c, d[i], op_add(ee, oo));
                d[j] = op_fma(c, d[j], op_sub(ee, oo));
            };
            pair(1, 3, (R)(1.0 / 9.0), W1s, ux);
            pair(2, 4, (R)(1.0 / 9.0), W1s, uy);
            pair(5, 7, (R)(1.0 / 36.0), W5s, op_add(ux, uy));
            pair(6, 8, (R)(1.0 / 36.0), W5s, op_sub(uy, ux));
        }
    }
    // non-finite state or a density outside (0, 2): the run has broken down
    // (the caller raises the error bit once for all its nodes)
    bad |= Lane<V>::bad(drho, ux, uy);
}

template <typename R, bool SC = false, bool FAST = false>
__device__ __forceinline__ void collide_node(const SimDev &s, R d[9], R Fx, R Fy, bool &bad) {
    collide_core<R, SC, FAST>(s, d, Fx, Fy, Fx != (R)0 || Fy != (R)0, bad);
}

// Two FP32 nodes at once (paired arithmetic, the same bits as two
// collide_node calls); nodes of which only one has a force go one by one.
template <bool SC, bool FAST>
__device__ __forceinline__ void collide_pair(const SimDev &s, float da[9], float db[9], float Fxa,
                                             float Fya, float Fxb, float Fyb, bool &bad) {
    const bool fa = Fxa != 0.f || Fya != 0.f, fb = Fxb != 0.f || Fyb != 0.f;
    if (fa != fb) {
        collide_core<float, SC, FAST>(s, da, Fxa, Fya, fa, bad);
        collide_core<float, SC, FAST>(s, db, Fxb, Fyb, fb, bad);
        return;
    }
    float2 d2[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d2[i] = make_float2(da[i], db[i]);
    collide_core<float2, SC, FAST>(s, d2, make_float2(Fxa, Fxb), make_float2(Fya, Fyb), fa, bad);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        da[i] = d2[i].x;
        db[i] = d2[i].y;
    }
}

// Four nodes under one force (F, the same for all four: no particle tile);
// the same bits as four collide_node calls.  From 16-bit storage (SC) the
// FP32 arithmetic runs in two pairs of paired instructions, which halves the
// collision's issue count there (where issue, not DRAM, limits the pass);
// from FP32 storage the pairs cost more in register pressure than they save,
// and from FP64 there is no paired form.  The debug build collides node by
// node, so comparing its bits with the release build's checks the pairs.
#ifdef LBIB_DEBUG
constexpr bool kPairedCollision = false;
#else
constexpr bool kPairedCollision = true;
#endif

template <typename R, bool SC, bool FAST>
__device__ __forceinline__ void collide_group4(const SimDev &s, R (*d)[9], R Fx, R Fy, bool &bad) {
    const bool forced = Fx != (R)0 || Fy != (R)0;
    if constexpr (sizeof(R) == 4 && SC && kPairedCollision) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 d2[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) d2[i] = make_float2(d[2 * h][i], d[2 * h + 1][i]);
            collide_core<float2, SC, FAST>(s, d2, make_float2(Fx, Fx), make_float2(Fy, Fy), forced, bad);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                d[2 * h][i] = d2[i].x;
                d[2 * h + 1][i] = d2[i].y;
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) collide_core<R, SC, FAST>(s, d[j], Fx, Fy, forced, bad);
    }
}

template <typename R, bool SC = false, bool FAST = false>
__device__ __forceinline__ void collide_node(const SimDev &s, R d[9], R Fx, R Fy) {
    bool bad = false;
    collide_node<R, SC, FAST>(s, d, Fx, Fy, bad);
    if (bad) atomicOr(s.err, ERR_UNSTABLE);
}

// SC: d is scaled (see collide_node); the dither hash takes the unscaled
// first deviation either way.
// AA streaming (s.aa): the slots of post_index for the step from state par.
template <typename S, typename R, bool STREAM = false, bool SC = false>
__device__ __forceinline__ void store_node(const SimDev &s, S *__restrict__ dst, int N, int k,
                                           const R d[9], int par = 0) {
    const float sc = SC ? 1.f : s.scale;
    if (!pop_index_ok(s, k) || !pop_index_ok(s, 8 * N + k)) return;
    if (s.aa) {
        const int y = div_nx(s, k), x = k - y * s.nx;
        const unsigned h = (sizeof(S) == 2 && s.sround)
                               ? dither_word(k, SC ? (float)d[0] * s.inv_scale : (float)d[0]) : 0u;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int j = post_index(s, i, k, x, y, par);
            if (sizeof(S) == 2 && s.sround)
                Store<S>::template st_r<STREAM>(dst, j, d[i], sc, dither_plane(h, i));
            else if constexpr (STREAM)
                Store<S>::st_cs(dst, j, d[i], sc);
            else
                Store<S>::st(dst, j, d[i], sc);
        }
        return;
    }
    if (sizeof(S) == 2 && s.sround) {
        const unsigned h = dither_word(k, SC ? (float)d[0] * s.inv_scale : (float)d[0]);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            Store<S>::template st_r<STREAM>(dst, i * N + k, d[i], sc, dither_plane(h, i));
        return;
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if constexpr (STREAM) Store<S>::st_cs(dst, i * N + k, d[i], sc);
        else Store<S>::st(dst, i * N + k, d[i], sc);
    }
}

// Pre-collision deviations of the four nodes (x0 .. x0 + 3, y) of a row away
// from the walls (or of a lattice periodic in y): one vector load per
// population plane, plus one scalar load for the node the x shift brings in
// from the next group (x periodic).  Same values as pull_node per node.
// AA (in-place streaming, see post_index) from parity 0 pulls population i
// from plane opp(i) of the same neighbour: OPP = true.
template <typename S, typename R, bool STREAM, bool OPP = false>
__device__ __forceinline__ void pull_group(const SimDev &s, const S *__restrict__ src, int x0,
                                           int y, R (*d)[9], float inv) {
    constexpr int OPq[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const int nx = s.nx, ny = s.ny, N = nx * ny;
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    const int r0 = y * nx, rm = ym * nx, rp = yp * nx;
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;       // left of the group
    const int xr = x0 + 4 == nx ? 0 : x0 + 4;        // right of the group
    auto ld1 = [&](int i) -> R {
        i = pop_load_index(s, i);
        if constexpr (STREAM) return Store<S>::ld_cs(src, i, inv); else return Store<S>::ld(src, i, inv);
    };
    R v[4];
    // (plane, row of the source, x shift of the pull: +1 pulls from x - 1)
    auto plane = [&](int i, int row, int sh) {
        const int q = OPP ? OPq[i] : i;
        Vec4<S, STREAM>::ld(src + pop_load_index(s, q * N + row + x0, 4), inv, v);
        if (sh == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) d[j][i] = v[j];
        } else if (sh > 0) {
            d[0][i] = ld1(q * N + row + xl);
#pragma unroll
            for (int j = 1; j < 4; ++j) d[j][i] = v[j - 1];
        } else {
#pragma unroll
            for (int j = 0; j < 3; ++j) d[j][i] = v[j + 1];
            d[3][i] = ld1(q * N + row + xr);
        }
    };
    plane(0, r0, 0);
    plane(1, r0, 1);
    plane(2, rm, 0);
    plane(3, r0, -1);
    plane(4, rp, 0);
    plane(5, rm, 1);
    plane(6, rm, -1);
    plane(7, rp, -1);
    plane(8, rp, 1);
}

// Near box of a batch particle for the step that reads buffer parity slot,
// from the batch's flat copy (both slots in one load, so the load does not
// wait for the parity).
struct BoxView {
    int ox, oy, NBx, NBy;
};
__device__ __forceinline__ BoxView near_box(const NearBox *nb, int slot) {
    const int4 o = *reinterpret_cast<const int4 *>(nb);
    const int2 e = *reinterpret_cast<const int2 *>(&nb->NBx);
    return BoxView{slot ? o.z : o.x, slot ? o.w : o.y, e.x, e.y};
}

// Node (x, y) inside a near box of the simulation's particles (the batch's
// near boxes nb[0 .. np); box slot = the parity of the buffer this step reads).
__device__ __forceinline__ bool in_near_box(const SimDev &s, const NearBox *nb, int np, int slot,
                                            int x, int y) {
    for (int k = 0; k < np; ++k) {
        const BoxView q = near_box(nb + k, slot);
        int dx = x - q.ox;
        if (dx < 0) dx += s.nx;
        int dy = y - q.oy;
        if (dy < 0 && s.wall_b == LBIB_WALL_PERIODIC) dy += s.ny;
        if (dx < q.NBx && (unsigned)dy < (unsigned)q.NBy) return true;
    }
    return false;
}

// Bit j set: node (x0 + j, y) lies outside every near box (x0 + 3 < nx).
__device__ __forceinline__ unsigned outside_near_boxes4(const SimDev &s, const NearBox *nb, int np,
                                                        int slot, int x0, int y) {
    unsigned keep = 0xFu;
    for (int k = 0; k < np; ++k) {
        const BoxView q = near_box(nb + k, slot);
        int dy = y - q.oy;
        if (dy < 0 && s.wall_b == LBIB_WALL_PERIODIC) dy += s.ny;
        if ((unsigned)dy >= (unsigned)q.NBy) continue;
        int dx = x0 - q.ox;
        if (dx < 0) dx += s.nx;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int e = dx + j;
            if (e >= s.nx) e -= s.nx;
            if (e < q.NBx) keep &= ~(1u << j);
        }
    }
    return keep;
}

// Calls f(tile) for each batch lattice tile holding a node of the near box
// [ox, ox + NBx) x [oy, oy + NBy) (x wrapped; rows wrapped for a periodic y,
// clipped to the lattice between walls), possibly more than once; lanes
// lane, lane + nlanes, ... of the caller share the calls.  Rows of at most a
// tile: every tile holding a node of the box's rows (a superset); wider rows:
// per row, the tiles of the box's span of it.
template <class F>
__device__ __forceinline__ void for_box_tiles(const SimDev &s, int ox, int oy, int NBx, int NBy,
                                              int lane, int nlanes, F &&f) {
    auto rows = [&](int r0, int r1) {
        const int a = s.tile0 + (int)(((long long)r0 * s.nx) / LB_TILE_NODES);
        const int e = s.tile0 + (int)(((long long)(r1 + 1) * s.nx - 1) / LB_TILE_NODES);
        for (int t = a + lane; t <= e; t += nlanes) f(t);
    };
    const bool periodic = s.wall_b == LBIB_WALL_PERIODIC;
    const int last = oy + NBy - 1;
    if (s.nx <= LB_TILE_NODES) {
        if (periodic) {
            if (last < s.ny) {
                rows(oy, last);
            } else {
                rows(oy, s.ny - 1);
                rows(0, min(last - s.ny, s.ny - 1));
            }
        } else {
            const int r0 = max(oy, 0), r1 = min(last, s.ny - 1);
            if (r0 <= r1) rows(r0, r1);
        }
        return;
    }
    const int w = min(NBx, s.nx);
    ox %= s.nx;
    if (ox < 0) ox += s.nx;
    auto span = [&](long long a, long long e) {   // lattice nodes a .. e
        for (int t = (int)(a / LB_TILE_NODES); t <= (int)(e / LB_TILE_NODES); ++t) f(s.tile0 + t);
    };
    const int nr = periodic ? min(NBy, s.ny) : NBy;
    for (int r = lane; r < nr; r += nlanes) {
        int y = oy + r;
        if (periodic) {
            y %= s.ny;
            if (y < 0) y += s.ny;
        } else if (y < 0 || y >= s.ny) {
            continue;
        }
        const long long row = (long long)y * s.nx;
        if (ox + w <= s.nx) {
            span(row + ox, row + ox + w - 1);
        } else {
            span(row + ox, row + s.nx - 1);
            span(row, row + ox + w - 1 - s.nx);
        }
    }
}

// One launch advances every simulation of a batch by one step.  A CTA of
// THREADS threads owns LB_TILE_NODES consecutive nodes (row-major) of one
// simulation.  With rows in whole aligned groups of four, each thread takes
// GROUPS groups of four consecutive nodes of one row (groups 4 * THREADS
// nodes apart), with vector loads and stores; the loads of all its groups
// are issued before any arithmetic.  Rows next to a wall take the per-node
// pull.  Otherwise a thread takes 4 * GROUPS nodes, THREADS apart (every
// scalar access of a warp still contiguous, the x - 1 / x + 1 pulls off by
// one element).  MINB caps registers through the launch bounds.  The
// variants share the tile, so a batch can switch between them.
// BULK: skip the nodes of the particles' near boxes (they carry no IB force
// and are updated by lattice_near_kernel, after the particle pass).
// flip bit 1 (DRY): a timing run that leaves the step counter alone; it
// writes only the buffer the next step overwrites.
template <typename S, typename R, bool BULK, int THREADS, int GROUPS, int MINB, bool AA = false>
__global__ void __launch_bounds__(THREADS, MINB) lattice_kernel(BatchDev b, int flip) {
    static_assert(THREADS * 4 * GROUPS == LB_TILE_NODES, "tile size");
    constexpr int NPT = 4 * GROUPS;
    const bool dry = (flip & 2) != 0;
    flip &= 1;
    const int tile = blockIdx.x;
    // the next step's bulk pass, a programmatic dependent of this one, may
    // start its CTAs once every CTA of this grid has started
    asm volatile("griddepcontrol.launch_dependents;");
    const TileDev t = b.tiles[tile];
    const SimDev &s = b.sims[t.sim];
    const int nx = s.nx;
    const int N = nx * s.ny;
    const int cur = b.par[t.sim] ^ flip;
    // the above is fixed for the batched call; when launched as a
    // programmatic dependent of the step before, wait for its grids here,
    // before reading what they wrote (populations, box counts and boxes,
    // the step counter)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const unsigned tboxes = BULK && t.np ? b.tile_boxes[tile] : 0u;
    if (!dry && t.k0 == 0 && threadIdx.x == 0) *s.step += 1;
    // a near box reaches this tile in this step's slot
    const bool boxes = ((tboxes >> (16 * cur)) & 0xFFFFu) != 0;
    const S *__restrict__ src = (const S *)s.pop[cur];
    S *__restrict__ dst = (S *)s.pop[cur ^ 1];
    const R gx = pick<R>(s.f_gx, s.gx), gy = pick<R>(s.f_gy, s.gy);
    R d[NPT][9];
    if (s.vec4) {
        // 16-bit storage: groups collide in the scaled form (collide_node)
        constexpr bool SC = sizeof(S) == 2;
        const int kt = t.k0 + 4 * (int)threadIdx.x;
        int kg[GROUPS], yg[GROUPS], xg[GROUPS];
        unsigned keep[GROUPS];
#pragma unroll
        for (int g = 0; g < GROUPS; ++g) {
            kg[g] = kt + g * 4 * THREADS;
            yg[g] = div_nx(s, kg[g]);
            xg[g] = kg[g] - yg[g] * nx;
            keep[g] = kg[g] < N ? 0xFu : 0u;
            if (BULK && boxes && keep[g]) keep[g] = outside_near_boxes4(s, b.nbox + t.p0, t.np, cur, xg[g], yg[g]);
#ifdef LBIB_DEBUG
            // the debug build checks the tile counts: a node of a near box in
            // a tile counted free of them is a bookkeeping error
            if (BULK && !boxes && t.np && keep[g] &&
                outside_near_boxes4(s, b.nbox + t.p0, t.np, cur, xg[g], yg[g]) != 0xFu)
                atomicOr(s.err, ERR_BOUNDS);
#endif
        }
#pragma unroll
        for (int g = 0; g < GROUPS; ++g) {
            if (!keep[g]) continue;
            const int y = yg[g];
            if (s.wall_b != LBIB_WALL_PERIODIC && (y == 0 || y == s.ny - 1)) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    pull_node<S, R, BULK>(s, src, xg[g] + j, y, d[4 * g + j], AA ? cur : 0);
                    if constexpr (SC) {
#pragma unroll
                        for (int i = 0; i < 9; ++i) d[4 * g + j][i] *= s.scale;
                    }
                }
            } else if (!AA || !s.aa) {
                pull_group<S, R, BULK>(s, src, xg[g], y, &d[4 * g], SC ? 1.f : s.inv_scale);
            } else if (cur) {
                // in place, parity 1: the node's own slots, plane i
                R v[4];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    Vec4<S, BULK>::ld(src + pop_load_index(s, i * N + kg[g], 4), SC ? 1.f : s.inv_scale, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) d[4 * g + j][i] = v[j];
                }
            } else {
                // in place, parity 0: the neighbours' opposite planes
                pull_group<S, R, BULK, true>(s, src, xg[g], y, &d[4 * g], SC ? 1.f : s.inv_scale);
            }
        }
        bool bad = false;
#pragma unroll
        for (int g = 0; g < GROUPS; ++g) {
            if (!keep[g]) continue;
            const int k = kg[g];
            if (BULK && gx == (R)0 && gy == (R)0) {
                // no body force and no particle tile: the force-free form
                collide_group4<R, SC, sizeof(S) == 2>(s, &d[4 * g], (R)0, (R)0, bad);
            } else if (BULK) {
                collide_group4<R, SC, sizeof(S) == 2>(s, &d[4 * g], gx, gy, bad);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    R Fx = gx, Fy = gy;
                    if (!BULK && s.np) tile_force<R>(s, b.parts, xg[g] + j, yg[g], Fx, Fy);
                    collide_node<R, SC, sizeof(S) == 2>(s, d[4 * g + j], Fx, Fy, bad);
                }
            }
            if constexpr (AA) {
                const float sc = SC ? 1.f : s.scale;
                const bool sr = sizeof(S) == 2 && s.sround;
                const int y = yg[g];
                const bool wallrow = s.wall_b != LBIB_WALL_PERIODIC && (y == 0 || y == s.ny - 1);
                unsigned h[4] = {0u, 0u, 0u, 0u};
                if (keep[g] == 0xFu && sr) {
    #pragma unroll
                    for (int j = 0; j < 4; ++j)
                        h[j] = dither_word(k + j, SC ? (float)d[4 * g + j][0] * s.inv_scale
                                                     : (float)d[4 * g + j][0]);
                }
                if (AA && keep[g] == 0xFu && s.aa && !wallrow && cur == 0) {
                    // in place, parity 0, away from the walls: population i to
                    // x + e_i, whole groups for the planes without an x
                    // component, one node at a time for the others (x periodic)
                    constexpr int EXq[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
                    constexpr int EYq[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    #pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        int yy = y + EYq[i];
                        if (yy < 0) yy += s.ny;
                        if (yy >= s.ny) yy -= s.ny;
                        const int row = i * N + yy * nx;
                        const R o[4] = {d[4 * g][i], d[4 * g + 1][i], d[4 * g + 2][i], d[4 * g + 3][i]};
                        unsigned r[4];
    #pragma unroll
                        for (int j = 0; j < 4; ++j) r[j] = dither_plane(h[j], i);
                        if (EXq[i] == 0) {
                            if (!pop_index_ok(s, row + xg[g], 4)) continue;
                            if (sr) Vec4<S, BULK>::st_r(dst + row + xg[g], o, sc, r);
                            else Vec4<S, BULK>::st(dst + row + xg[g], o, sc);
                        } else {
    #pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                int xx = xg[g] + j + EXq[i];
                                if (xx < 0) xx += nx;
                                if (xx >= nx) xx -= nx;
                                if (!pop_index_ok(s, row + xx)) continue;
                                if (sr) Store<S>::template st_r<BULK>(dst, row + xx, o[j], sc, r[j]);
                                else if constexpr (BULK) Store<S>::st_cs(dst, row + xx, o[j], sc);
                                else Store<S>::st(dst, row + xx, o[j], sc);
                            }
                        }
                    }
                } else if (keep[g] == 0xFu && (!AA || !s.aa || !wallrow)) {
                    // A/B, or in place from parity 1 (population i to plane
                    // opp(i) of the node itself)
                    constexpr int OPq[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    #pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int q = (AA && s.aa) ? OPq[i] : i;
                        const R o[4] = {d[4 * g][i], d[4 * g + 1][i], d[4 * g + 2][i], d[4 * g + 3][i]};
                        if (!pop_index_ok(s, q * N + k, 4)) continue;
                        if (sr) {
                            const unsigned r[4] = {dither_plane(h[0], i), dither_plane(h[1], i),
                                                   dither_plane(h[2], i), dither_plane(h[3], i)};
                            Vec4<S, BULK>::st_r(dst + q * N + k, o, sc, r);
                        } else {
                            Vec4<S, BULK>::st(dst + q * N + k, o, sc);
                        }
                    }
                } else {
    #pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (keep[g] & (1u << j))
                            store_node<S, R, BULK, SC>(s, dst, N, k + j, d[4 * g + j], cur);
                }
            } else {
                const float sc = SC ? 1.f : s.scale;
                if (keep[g] == 0xFu && sizeof(S) == 2 && s.sround) {
                    unsigned h[4];
    #pragma unroll
                    for (int j = 0; j < 4; ++j)
                        h[j] = dither_word(k + j, SC ? (float)d[4 * g + j][0] * s.inv_scale
                                                     : (float)d[4 * g + j][0]);
    #pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const R o[4] = {d[4 * g][i], d[4 * g + 1][i], d[4 * g + 2][i], d[4 * g + 3][i]};
                        const unsigned r[4] = {dither_plane(h[0], i), dither_plane(h[1], i),
                                               dither_plane(h[2], i), dither_plane(h[3], i)};
                        if (pop_index_ok(s, i * N + k, 4)) Vec4<S, BULK>::st_r(dst + i * N + k, o, sc, r);
                    }
                } else if (keep[g] == 0xFu) {
    #pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const R o[4] = {d[4 * g][i], d[4 * g + 1][i], d[4 * g + 2][i], d[4 * g + 3][i]};
                        if (pop_index_ok(s, i * N + k, 4)) Vec4<S, BULK>::st(dst + i * N + k, o, sc);
                    }
                } else {
    #pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (keep[g] & (1u << j))
                            store_node<S, R, BULK, SC>(s, dst, N, k + j, d[4 * g + j]);
                }
            }
        }
        if (bad) atomicOr(s.err, ERR_UNSTABLE);
        return;
    }
    const int k0 = t.k0 + (int)threadIdx.x;
    bool skip[NPT];
    // node coordinates: one division per thread, then step by THREADS
    int xs[NPT], ys[NPT];
    {
        int y = k0 / nx, x = k0 - y * nx;
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            xs[j] = x;
            ys[j] = y;
            x += THREADS;
            while (x >= nx) {
                x -= nx;
                ++y;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        skip[j] = k0 + j * THREADS >= N;
        if (BULK && !skip[j] && boxes) skip[j] = in_near_box(s, b.nbox + t.p0, t.np, cur, xs[j], ys[j]);
#ifdef LBIB_DEBUG
        if (BULK && !skip[j] && !boxes && t.np && in_near_box(s, b.nbox + t.p0, t.np, cur, xs[j], ys[j]))
            atomicOr(s.err, ERR_BOUNDS);
#endif
    }
#pragma unroll
    for (int j = 0; j < NPT; ++j)
        if (!skip[j]) pull_node<S, R, BULK>(s, src, xs[j], ys[j], d[j], cur);
    bool bad = false;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        if (!skip[j]) {
            R Fx = gx, Fy = gy;
            if (!BULK && s.np) tile_force<R>(s, b.parts, xs[j], ys[j], Fx, Fy);
            collide_node<R, false, sizeof(S) == 2>(s, d[j], Fx, Fy, bad);
            store_node<S, R, BULK>(s, dst, N, k0 + j * THREADS, d[j], cur);
        }
    }
    if (bad) atomicOr(s.err, ERR_UNSTABLE);
}

// The nodes of the near boxes (one box per particle; NBx x NBy nodes, rows
// outside the lattice skipped), with the IB force of every force tile of the
// simulation.  Runs after the particle pass that wrote the tiles.  The first
// CTA of each particle also publishes the box the last particle pass left for
// the next step but one.
template <typename S, typename R>
__global__ void __launch_bounds__(LB_THREADS) lattice_near_kernel(BatchDev b, int flip) {
    const int tile = blockIdx.x;
    const int pi = __ldg(b.near_part + tile);
    ParticleDev *P = b.parts[pi];
    const int si = b.part_sim[pi];
    const SimDev &s = b.sims[si];
    // the batch's copy of the parity word changes only between batched calls
    const int cur = b.par[si] ^ flip;
    // when launched as a programmatic dependent of the particle pass before
    // it, wait for that pass here: it wrote the force tiles and the next box
    // (everything read above is fixed for the call)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // then let the particle pass that follows start its prologue (which
    // reads what the particle pass before wrote); it waits for this grid to
    // complete before reading the populations
    asm volatile("griddepcontrol.launch_dependents;");
    const int NBx = P->NBx, NBy = P->NBy, ox = P->box_ox[cur], oy = P->box_oy[cur];
    const int t0 = __ldg(b.near_tile0 + pi);
    if (tile == t0 && threadIdx.x < 32) {
        // warp 0 of the particle's first CTA: move the box's count from the
        // tiles of the box it replaces in slot cur ^ 1 to those of the new one
        // (no bulk pass reads that slot before this grid ends), then publish
        const int px = P->pend_ox, py = P->pend_oy;
        NearBox &q = b.nbox[pi];
        const int old_ox = (cur ^ 1) ? q.ox1 : q.ox0, old_oy = (cur ^ 1) ? q.oy1 : q.oy0;
        const unsigned one = 1u << (16 * (cur ^ 1));
        for_box_tiles(s, old_ox, old_oy, NBx, NBy, (int)threadIdx.x, 32,
                      [&](int t) { atomicSub(b.tile_boxes + t, one); });
        for_box_tiles(s, px, py, NBx, NBy, (int)threadIdx.x, 32,
                      [&](int t) { atomicAdd(b.tile_boxes + t, one); });
        __syncwarp();
        if (threadIdx.x == 0) {
            P->box_ox[cur ^ 1] = px;
            P->box_oy[cur ^ 1] = py;
            // and into the batch's copy read by the bulk pass
            if (cur ^ 1) { q.ox1 = px; q.oy1 = py; } else { q.ox0 = px; q.oy0 = py; }
        }
    }
    const int nx = s.nx, ny = s.ny, N = nx * ny;
    const S *__restrict__ src = (const S *)s.pop[cur];
    S *__restrict__ dst = (S *)s.pop[cur ^ 1];
    const R gx = pick<R>(s.f_gx, s.gx), gy = pick<R>(s.f_gy, s.gy);
    const int k0 = (tile - t0) * NEAR_TILE_NODES + (int)threadIdx.x;
    int xs[NEAR_NPT], ys[NEAR_NPT];
    bool skip[NEAR_NPT];
#pragma unroll
    for (int j = 0; j < NEAR_NPT; ++j) {
        const int k = k0 + j * LB_THREADS;
        const int by = k / NBx, bx = k - by * NBx;
        int x = ox + bx;
        if (x >= nx) x -= nx;
        int y = oy + by;
        if (s.wall_b == LBIB_WALL_PERIODIC) {
            if (y < 0) y += ny;
            if (y >= ny) y -= ny;
        }
        xs[j] = x;
        ys[j] = y;
        skip[j] = k >= NBx * NBy || y < 0 || y >= ny;
    }
    R d[NEAR_NPT][9];
#pragma unroll
    for (int j = 0; j < NEAR_NPT; ++j)
        if (!skip[j]) pull_node<S, R>(s, src, xs[j], ys[j], d[j], cur);
    bool bad = false;
#pragma unroll
    for (int j = 0; j < NEAR_NPT; ++j) {
        if (!skip[j]) {
            R Fx = gx, Fy = gy;
            tile_force<R>(s, b.parts, xs[j], ys[j], Fx, Fy);
            collide_node<R, false, sizeof(S) == 2>(s, d[j], Fx, Fy, bad);
            store_node<S, R>(s, dst, N, ys[j] * nx + xs[j], d[j], cur);
        }
    }
    if (bad) atomicOr(s.err, ERR_UNSTABLE);
}

// ---- bulk pass with copy-engine staging (variants 4 and 5) -----------------
// Same 1024-node tiles and arithmetic as lattice_kernel (BULK, vector path).
// Thread 0 has the copy engine bring, for each of the nine population planes,
// the node range the tile pulls from -- the tile's range shifted by the
// plane's row offset, with a 16-byte margin on each side -- into shared memory
// with one bulk copy each, all completing on one mbarrier; the threads then
// take their groups of four nodes from shared memory.  Groups in the wall rows
// or at either end of a row (where x wraps) pull from global memory as in the
// other variants.  Only for storage of 4 or 2 bytes on lattices whose rows
// are whole 16-byte words and whose walls are not periodic (tma_ok).  The
// wait on the mbarrier is bounded: past the limit the simulation's error word
// gets ERR_TIMEOUT and the CTA leaves its tile unwritten.

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// Waits for the phase of the given parity of the mbarrier to complete, at
// most `limit` polls; true if it completed.
__device__ __forceinline__ bool mbar_wait(const uint64_t *bar, unsigned parity, int limit) {
    for (int it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait0(const uint64_t *bar, int limit) {
    return mbar_wait(bar, 0u, limit);
}

// Four consecutive staged values (p 16-byte aligned) and one staged value, in
// the compute type.
template <typename S> struct Staged4;
template <> struct Staged4<float> {
    static __device__ __forceinline__ void ld4(const float *p, float, float o[4]) {
        const float4 v = *(const float4 *)p;
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ float ld1(const float *p, float) { return *p; }
};
template <> struct Staged4<__half> {
    static __device__ __forceinline__ void ld4(const __half *p, float inv, float o[4]) {
        const uint2 u = *(const uint2 *)p;
        __half2 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        o[0] = fa.x * inv; o[1] = fa.y * inv; o[2] = fb.x * inv; o[3] = fb.y * inv;
    }
    static __device__ __forceinline__ float ld1(const __half *p, float inv) {
        return __half2float(*p) * inv;
    }
};
template <> struct Staged4<__nv_bfloat16> {
    static __device__ __forceinline__ void ld4(const __nv_bfloat16 *p, float inv, float o[4]) {
        const uint2 u = *(const uint2 *)p;
        __nv_bfloat162 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        o[0] = fa.x * inv; o[1] = fa.y * inv; o[2] = fb.x * inv; o[3] = fb.y * inv;
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16 *p, float inv) {
        return __bfloat162float(*p) * inv;
    }
};

template <typename S>
__host__ __device__ constexpr int tma_margin() { return 16 / (int)sizeof(S); }
template <typename S>
__host__ __device__ constexpr int tma_width() { return LB_TILE_NODES + 2 * tma_margin<S>(); }
template <typename S>
__host__ __device__ constexpr size_t tma_stage_bytes() {
    return 9 * (size_t)tma_width<S>() * sizeof(S);
}
template <typename S, int TILES>
__host__ __device__ constexpr size_t tma_smem_bytes() {
    return TILES * (tma_stage_bytes<S>() + 16);
}

// Thread 0: the bulk copies of one tile's nine source ranges into a stage,
// completing on its mbarrier (phase 0).
template <typename S>
__device__ __forceinline__ void tma_issue(const BatchDev &b, int flip, int tile, S *stg,
                                          uint64_t *bar) {
    constexpr int H = tma_margin<S>(), W = tma_width<S>();
    constexpr int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    const TileDev t = b.tiles[tile];
    const SimDev &s = b.sims[t.sim];
    const int nx = s.nx, N = nx * s.ny;
    const S *src = (const S *)s.pop[b.par[t.sim] ^ flip];
    const int k0 = t.k0;
    // plane i of node k comes from node k - EY[i] nx - EX[i]: stage nodes
    // [k0 - EY[i] nx - H, + W), clipped to the lattice (the clipped part is
    // only ever needed by wall-row groups, which pull from global memory)
    int lo[9], bytes[9];
    unsigned total = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int g0 = k0 - EY[i] * nx - H;
        const int a = max(g0, 0), e = min(g0 + W, N);
        lo[i] = a;
        bytes[i] = e > a ? (e - a) * (int)sizeof(S) : 0;
        total += (unsigned)bytes[i];
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(total) : "memory");
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        if (!bytes[i]) continue;
        const int g0 = k0 - EY[i] * nx - H;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(smem_addr(stg + i * W + (lo[i] - g0))), "l"(src + (size_t)i * N + lo[i]),
              "r"(bytes[i]), "r"(smem_addr(bar))
            : "memory");
    }
}

// One tile from its stage (every thread: one group of four nodes).  Returns
// false if the stage's copies did not complete within the bounded wait.
template <typename S, typename R>
__device__ __forceinline__ bool tma_tile(const BatchDev &b, int flip, bool dry, int tile,
                                         const S *stg, const uint64_t *bar,
                                         unsigned parity = 0) {
    constexpr int H = tma_margin<S>(), W = tma_width<S>();
    constexpr int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const TileDev t = b.tiles[tile];
    const unsigned tboxes = t.np ? b.tile_boxes[tile] : 0u;
    const SimDev &s = b.sims[t.sim];
    const int nx = s.nx, ny = s.ny, N = nx * ny;
    if (!dry && t.k0 == 0 && threadIdx.x == 0) *s.step += 1;
    const int cur = b.par[t.sim] ^ flip;
    const bool boxes = ((tboxes >> (16 * cur)) & 0xFFFFu) != 0;
    const S *__restrict__ src = (const S *)s.pop[cur];
    S *__restrict__ dst = (S *)s.pop[cur ^ 1];
    const int k0 = t.k0;
    // this thread's group of four nodes (decided while the copies run)
    const int kt = k0 + 4 * (int)threadIdx.x;
    const int y = div_nx(s, kt), x0 = kt - y * nx;
    unsigned keep = kt < N ? 0xFu : 0u;
    if (boxes && keep) keep = outside_near_boxes4(s, b.nbox + t.p0, t.np, cur, x0, y);
#ifdef LBIB_DEBUG
    if (!boxes && t.np && keep && outside_near_boxes4(s, b.nbox + t.p0, t.np, cur, x0, y) != 0xFu)
        atomicOr(s.err, ERR_BOUNDS);
#endif
    const bool wall = y == 0 || y == ny - 1;
    const bool global_pull = wall || x0 == 0 || x0 + 4 == nx;
    // 16-bit storage: the group collides in the scaled form (collide_node)
    constexpr bool SC = sizeof(S) == 2;
    R d[4][9];
    if (keep && global_pull) {
        if (wall) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                pull_node<S, R, true>(s, src, x0 + j, y, d[j]);
                if constexpr (SC) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) d[j][i] *= s.scale;
                }
            }
        } else {
            pull_group<S, R, true>(s, src, x0, y, d, SC ? 1.f : s.inv_scale);
        }
    }
    // the warp gives up as a whole (its lanes may see the limit at different
    // polls), and reports it
    if (!__all_sync(0xffffffffu, mbar_wait(bar, parity, b.wait_polls))) {
        if ((threadIdx.x & 31) == 0) atomicOr(s.err, ERR_TIMEOUT);
        return false;
    }
    if (!keep) return true;
    if (!global_pull) {
        const float inv = SC ? 1.f : s.inv_scale;
        const int j0 = kt - k0 + H;                 // staged index of node kt (no x shift)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const S *p = stg + i * W + j0;          // nodes kt .. kt + 3 of plane i's source row
            R v[4];
            Staged4<S>::ld4(p, inv, v);
            if (EX[i] == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) d[j][i] = v[j];
            } else if (EX[i] > 0) {                 // pulls from x - 1
                d[0][i] = Staged4<S>::ld1(p - 1, inv);
#pragma unroll
                for (int j = 1; j < 4; ++j) d[j][i] = v[j - 1];
            } else {                                // pulls from x + 1
#pragma unroll
                for (int j = 0; j < 3; ++j) d[j][i] = v[j + 1];
                d[3][i] = Staged4<S>::ld1(p + 4, inv);
            }
        }
    }
    const R gx = pick<R>(s.f_gx, s.gx), gy = pick<R>(s.f_gy, s.gy);
    bool bad = false;
    if (gx == (R)0 && gy == (R)0) collide_group4<R, SC, sizeof(S) == 2>(s, d, (R)0, (R)0, bad);
    else collide_group4<R, SC, sizeof(S) == 2>(s, d, gx, gy, bad);
    if (bad) atomicOr(s.err, ERR_UNSTABLE);
    const float sc = SC ? 1.f : s.scale;
    if (keep == 0xFu && sizeof(S) == 2 && s.sround) {
        unsigned h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            h[j] = dither_word(kt + j, SC ? (float)d[j][0] * s.inv_scale : (float)d[j][0]);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const R o[4] = {d[0][i], d[1][i], d[2][i], d[3][i]};
            const unsigned r[4] = {dither_plane(h[0], i), dither_plane(h[1], i),
                                   dither_plane(h[2], i), dither_plane(h[3], i)};
            if (pop_index_ok(s, i * N + kt, 4)) Vec4<S, true>::st_r(dst + (size_t)i * N + kt, o, sc, r);
        }
    } else if (keep == 0xFu) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const R o[4] = {d[0][i], d[1][i], d[2][i], d[3][i]};
            if (pop_index_ok(s, i * N + kt, 4)) Vec4<S, true>::st(dst + (size_t)i * N + kt, o, sc);
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (keep & (1u << j)) store_node<S, R, true, SC>(s, dst, N, kt + j, d[j]);
    }
    return true;
}

// TILES consecutive tiles per CTA, each in its own stage: the copies of all
// of them are issued at once, so the later tiles' data arrive while the first
// is computed.
template <typename S, typename R, int MINB, int TILES>
__global__ void __launch_bounds__(256, MINB) lattice_tma_kernel(BatchDev b, int flip) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // (as a programmatic dependent: wait for the step before)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const bool dry = (flip & 2) != 0;
    flip &= 1;
    auto stage = [&](int t) { return (S *)(smem_raw + t * (tma_stage_bytes<S>() + 16)); };
    auto barrier = [&](int t) {
        return (uint64_t *)(smem_raw + t * (tma_stage_bytes<S>() + 16) + tma_stage_bytes<S>());
    };
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < TILES; ++t)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(barrier(t))) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int first = blockIdx.x * TILES;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int t = 0; t < TILES; ++t)
            if (first + t < b.total_tiles) tma_issue<S>(b, flip, first + t, stage(t), barrier(t));
    }
#pragma unroll
    for (int t = 0; t < TILES; ++t) {
        if (first + t >= b.total_tiles) break;
        if (!tma_tile<S, R>(b, flip, dry, first + t, stage(t), barrier(t))) {
            // copies that did not complete in time: one more bounded wait on
            // each stage still in flight (they write this CTA's shared
            // memory), always of the full length, then leave the remaining
            // tiles
            for (int u = t; u < TILES && first + u < b.total_tiles; ++u) mbar_wait0(barrier(u), 1 << 16);
            return;
        }
    }
}

// Copy-engine pipeline: TILES consecutive tiles per CTA through a ring of
// STAGES shared-memory stages.  Warp 8 is the producer: its lane 0 issues
// the bulk copies of tile j into stage j % STAGES (completing on full[s])
// once the eight consumer warps have released the stage's previous tile
// (empty[s], one arrival per warp); the consumer warps compute tile j from
// its stage (tma_tile) and release it.  The copies of the next STAGES - 1
// tiles are in flight while a tile is computed, so the load latency is off
// the consumers' path.  Every wait is bounded: a consumer warp that gives up
// reports ERR_TIMEOUT and leaves; the producer, when a release does not come,
// waits (bounded, full length) for the copies it has in flight and leaves;
// at the end it waits for its last copies, so no copy outlives the CTA.
template <typename S>
__host__ __device__ constexpr int pipe_stages() { return sizeof(S) == 2 ? 4 : 2; }
constexpr int PIPE_TILES = 8;
constexpr int PIPE_THREADS = 288;
template <typename S>
__host__ __device__ constexpr size_t pipe_smem_bytes() {
    return pipe_stages<S>() * tma_stage_bytes<S>() + 2 * pipe_stages<S>() * sizeof(uint64_t);
}

template <typename S, typename R>
__global__ void __launch_bounds__(PIPE_THREADS, 2) lattice_pipe_kernel(BatchDev b, int flip) {
    constexpr int STAGES = pipe_stages<S>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // (as a programmatic dependent: wait for the step before)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const bool dry = (flip & 2) != 0;
    flip &= 1;
    auto stage = [&](int t) { return (S *)(smem_raw + t * tma_stage_bytes<S>()); };
    uint64_t *bars = (uint64_t *)(smem_raw + STAGES * tma_stage_bytes<S>());
    auto full = [&](int t) { return bars + t; };
    auto empty = [&](int t) { return bars + STAGES + t; };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int t = 0; t < STAGES; ++t) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(full(t))) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_addr(empty(t))) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int first = blockIdx.x * PIPE_TILES;
    const int n = min(PIPE_TILES, b.total_tiles - first);
    if (warp == 8) {
        if (lane != 0) return;
        for (int j = 0; j < n; ++j) {
            const int st = j % STAGES;
            if (j >= STAGES && !mbar_wait(empty(st), (unsigned)((j / STAGES) - 1) & 1u, b.wait_polls)) {
                for (int u = j - STAGES; u < j; ++u)
                    mbar_wait(full(u % STAGES), (unsigned)(u / STAGES) & 1u, 1 << 16);
                return;
            }
            // the consumers' reads of the stage come before the copy's writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_issue<S>(b, flip, first + j, stage(st), full(st));
        }
        for (int u = max(0, n - STAGES); u < n; ++u)
            mbar_wait(full(u % STAGES), (unsigned)(u / STAGES) & 1u, 1 << 16);
        return;
    }
    for (int j = 0; j < n; ++j) {
        const int st = j % STAGES;
        if (!tma_tile<S, R>(b, flip, dry, first + j, stage(st), full(st), (unsigned)(j / STAGES) & 1u))
            return;
        __syncwarp();
        if (lane == 0)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(empty(st))) : "memory");
    }
}

template <typename S, typename R>
__global__ void fields_kernel(SimDev s, ParticleDev *const *parts, double *rho_o, double *ux_o,
                              double *uy_o) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.nx * s.ny) return;
    const int y = k / s.nx, x = k - y * s.nx;
    const S *src = (const S *)s.pop[*s.cur];
    R d[9];
    pull_node<S, R>(s, src, x, y, d, *s.cur);
    R drho, jx, jy;
    node_moments(d, drho, jx, jy);
    R Fx = (R)s.gx, Fy = (R)s.gy;
    if (s.np) tile_force<R>(s, parts, x, y, Fx, Fy);
    const double rho = 1.0 + (double)drho;
    if (rho_o) rho_o[k] = rho;
    if (ux_o) ux_o[k] = ((double)jx + 0.5 * (double)Fx) / rho;
    if (uy_o) uy_o[k] = ((double)jy + 0.5 * (double)Fy) / rho;
}

// Post-collision populations of the last step ([9][ny][nx], full f): with
// AA streaming they sit where the step from the other parity stored them.
template <typename S>
__global__ void export_pops_kernel(SimDev s, double *out) {
    const size_t N = (size_t)s.nx * s.ny;
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 9 * N) return;
    const int i = (int)(k / N), n = (int)(k - (size_t)i * N);
    const int y = n / s.nx, x = n - y * s.nx;
    const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const S *src = (const S *)s.pop[*s.cur];
    out[k] = w + (double)Store<S>::ld(src, post_index(s, i, n, x, y, *s.cur ^ 1), s.inv_scale);
}

template <typename S, typename R>
__global__ void import_pops_kernel(SimDev s, const double *in) {
    const size_t N = (size_t)s.nx * s.ny;
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 9 * N) return;
    const int i = (int)(k / N), n = (int)(k - (size_t)i * N);
    const int y = n / s.nx, x = n - y * s.nx;
    const double w = i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    S *dst = (S *)s.pop[*s.cur];
    Store<S>::st(dst, post_index(s, i, n, x, y, *s.cur ^ 1), (R)(in[k] - w), s.scale);
}

template <typename R>
__global__ void ib_export_kernel(SimDev s, ParticleDev *const *parts, double *fx, double *fy) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.nx * s.ny) return;
    const int y = k / s.nx, x = k - y * s.nx;
    R a = 0, c = 0;
    tile_force<R>(s, parts, x, y, a, c);
    fx[k] = (double)a;
    fy[k] = (double)c;
}

__global__ void flip_kernel(int *const *curs, int *par, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        *curs[i] ^= 1;
        par[i] ^= 1;
    }
}

// The batch's copies of its members' parity words and near boxes.
__global__ void batch_refresh_kernel(BatchDev b, int *const *curs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b.total_tiles) b.tile_boxes[i] = 0u;
    if (i < b.nsims) b.par[i] = *curs[i];
    if (i < b.nparts) {
        const ParticleDev *P = b.parts[i];
        NearBox q;
        q.ox0 = P->box_ox[0];
        q.oy0 = P->box_oy[0];
        q.ox1 = P->box_ox[1];
        q.oy1 = P->box_oy[1];
        q.NBx = P->NBx;
        q.NBy = P->NBy;
        q.pad[0] = q.pad[1] = 0;
        b.nbox[i] = q;
    }
}

// The per-tile near-box counts of both slots (one warp per particle), after
// batch_refresh_kernel.
__global__ void tile_boxes_kernel(BatchDev b) {
    const int p = blockIdx.x;
    const SimDev &s = b.sims[b.part_sim[p]];
    const NearBox q = b.nbox[p];
    const int lane = (int)threadIdx.x;
    for_box_tiles(s, q.ox0, q.oy0, q.NBx, q.NBy, lane, 32,
                  [&](int t) { atomicAdd(b.tile_boxes + t, 1u); });
    for_box_tiles(s, q.ox1, q.oy1, q.NBx, q.NBy, lane, 32,
                  [&](int t) { atomicAdd(b.tile_boxes + t, 1u << 16); });
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

// Bulk-pass variants (threads, groups of four nodes per thread, minimum
// resident CTAs per SM); FP64 storage and the plain pass use variant 0.
// A lattice-pass kernel launch; pdl: as a programmatic dependent of the
// previous kernel on st.
cudaError_t launch_pass(void (*k)(BatchDev, int), unsigned grid, unsigned block, size_t smem,
                        cudaStream_t st, bool pdl, const BatchDev &b, int flip) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, b, flip);
}

template <typename S, typename R, bool BULK>
cudaError_t launch_variant(int variant, const BatchDev &b, int flip, cudaStream_t st,
                           bool pdl = false) {
    constexpr bool TUNED = BULK && sizeof(S) <= 4;
    if (b.any_aa) {
        // a member streams in place: the form with the in-place vector path
        // (its extra code costs the other forms registers, so it is apart)
        return launch_pass(lattice_kernel<S, R, BULK, 256, 1, sizeof(S) == 8 ? 1 : 4, true>,
                           b.total_tiles, 256, 0, st, pdl, b, flip);
    }
    if (!TUNED) variant = 0;
    if (variant >= 4 && !b.tma_ok) variant = 1;     // lattices unsuited to staging
    switch (variant) {
        case 4:
            if constexpr (TUNED) {
                return launch_pass(lattice_tma_kernel<S, R, 4, 1>, b.total_tiles, 256,
                                   tma_smem_bytes<S, 1>(), st, pdl, b, flip);
            }
            [[fallthrough]];
        case 5:
            if constexpr (TUNED) {
                return launch_pass(lattice_pipe_kernel<S, R>,
                                   (b.total_tiles + PIPE_TILES - 1) / PIPE_TILES, PIPE_THREADS,
                                   pipe_smem_bytes<S>(), st, pdl, b, flip);
            }
            [[fallthrough]];
        case 1:
            if constexpr (TUNED) {
                return launch_pass(lattice_kernel<S, R, BULK, 256, 1, 4>, b.total_tiles, 256, 0, st,
                                   pdl, b, flip);
            }
            [[fallthrough]];
        case 2:
            if constexpr (TUNED) {
                return launch_pass(lattice_kernel<S, R, BULK, 256, 1, 5>, b.total_tiles, 256, 0, st,
                                   pdl, b, flip);
            }
            [[fallthrough]];
        case 3:
            if constexpr (TUNED) {
                return launch_pass(lattice_kernel<S, R, BULK, 256, 1, 6>, b.total_tiles, 256, 0, st,
                                   pdl, b, flip);
            }
            [[fallthrough]];
        default:
            return launch_pass(lattice_kernel<S, R, BULK, 256, 1, 1>, b.total_tiles, 256, 0, st, pdl,
                               b, flip);
    }
    return cudaGetLastError();
}

cudaError_t lattice_kernel_setup(int kind) {
    return by_kind(kind, [&](auto sv, auto rv) -> cudaError_t {
        using S = decltype(sv);
        using R = decltype(rv);
        if constexpr (sizeof(S) <= 4)
            return cudaFuncSetAttribute(lattice_pipe_kernel<S, R>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)pipe_smem_bytes<S>());
        return cudaSuccess;
    });
}

cudaError_t launch_lattice(int kind, const BatchDev &b, int flip, int mode, cudaStream_t st,
                           bool pdl) {
    return by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        if (mode == 0) return launch_variant<S, R, false>(b.lat_variant, b, flip, st);
        if (mode == 1) return launch_variant<S, R, true>(b.lat_variant, b, flip, st, pdl);
        if (b.total_near_tiles == 0) return cudaSuccess;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(b.total_near_tiles);
        cfg.blockDim = dim3(LB_THREADS);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = pdl ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, lattice_near_kernel<S, R>, b, flip);
    });
}

cudaError_t launch_fields(int kind, const SimDev &s, ParticleDev *const *parts, double *rho,
                          double *ux, double *uy, cudaStream_t st) {
    const int n = s.nx * s.ny;
    return by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        fields_kernel<S, R><<<(n + 255) / 256, 256, 0, st>>>(s, parts, rho, ux, uy);
        return cudaGetLastError();
    });
}

cudaError_t launch_populations(int kind, const SimDev &s, double *out, cudaStream_t st) {
    const size_t n = 9 * (size_t)s.nx * s.ny;
    return by_kind(kind, [&](auto sv, auto) {
        using S = decltype(sv);
        export_pops_kernel<S><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, out);
        return cudaGetLastError();
    });
}

cudaError_t launch_set_populations(int kind, const SimDev &s, const double *in, cudaStream_t st) {
    const size_t n = 9 * (size_t)s.nx * s.ny;
    return by_kind(kind, [&](auto sv, auto rv) {
        using S = decltype(sv);
        using R = decltype(rv);
        import_pops_kernel<S, R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, in);
        return cudaGetLastError();
    });
}

cudaError_t launch_ib_export(int kind, const SimDev &s, ParticleDev *const *parts, double *fx,
                             double *fy, cudaStream_t st) {
    const int n = s.nx * s.ny;
    return by_kind(kind, [&](auto, auto rv) {
        using R = decltype(rv);
        ib_export_kernel<R><<<(n + 255) / 256, 256, 0, st>>>(s, parts, fx, fy);
        return cudaGetLastError();
    });
}

cudaError_t launch_flip(int *const *curs, int *par, int n, cudaStream_t st) {
    flip_kernel<<<(n + 127) / 128, 128, 0, st>>>(curs, par, n);
    return cudaGetLastError();
}

cudaError_t launch_batch_refresh(const BatchDev &b, int *const *curs, cudaStream_t st) {
    const int n = max(b.total_tiles, max(b.nsims, b.nparts));
    if (n == 0) return cudaSuccess;
    batch_refresh_kernel<<<(n + 127) / 128, 128, 0, st>>>(b, curs);
    if (b.nparts > 0) tile_boxes_kernel<<<b.nparts, 32, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace lbib
