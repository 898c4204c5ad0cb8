// lbib_internal.cuh -- device data structures and the lattice helpers shared
// by the lattice and particle kernels of the sm_103a library.
//
// Populations are stored as deviations d_i = f_i - w_i in structure-of-arrays
// planes [9][ny][nx] (one buffer per parity, A/B pull scheme).  The stored
// state is post-collision f*; a node's pre-collision populations of the next
// step are gathered by pulling from its neighbours (Eq. 1 left-hand side) with
// the wall conditions applied on the fly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbib.h"

namespace lbib {

enum StorageKind { ST_F32 = 0, ST_F64 = 1, ST_F16 = 2, ST_BF16 = 3 };

// Lattice kernel work tile: 256 threads x 4 nodes.  Where rows are whole
// multiples of four nodes (and the buffers suitably aligned) a thread takes
// four consecutive nodes of one row with vector loads and stores; otherwise
// four nodes 256 apart in the row-major order.
constexpr int LB_THREADS = 256;
constexpr int LB_NPT = 4;
constexpr int LB_TILE_NODES = LB_THREADS * LB_NPT;
// Near-box pass: one node per thread (short dependent-load chains, more CTAs).
constexpr int NEAR_NPT = 1;
constexpr int NEAR_TILE_NODES = LB_THREADS * NEAR_NPT;

// Error bits of the per-simulation device error word.
enum { ERR_UNSTABLE = 1, ERR_TIMEOUT = 2, ERR_BOUNDS = 4 };

// Per-simulation descriptor as seen by the kernels of one batch.
struct SimDev {
    int nx, ny, wall_b, wall_t;
    int p0, np;          // particle range in the batch's particle table
    int tile0, ntiles;   // lattice work tiles of this simulation
    int vec4;            // rows in whole groups of four aligned nodes
    int sround;          // 16-bit storage: stochastic rounding of the stores
    int ib_iters;        // direct-forcing passes per step (>= 1)
    int ib_spread;       // spreading scale: 0 element lengths, 1 solved (A eps = 1)
    int aa;              // in-place (AA) streaming: pop[0] == pop[1], *cur the state parity
    int pad_aa;
    // k / nx = umulhi(k, nx_m) >> nx_s for 0 <= k < 2^31 (div_nx below)
    unsigned nx_m;
    int nx_s;
    double tau, u_b, u_t, gx, gy;
    double k_f, k_r0, kBT, sigma_star_ratio, y_cr, y_eq_ratio;
    double hamaker, eps_min, rec_b, rec_t;
    unsigned long long seed, sim_id;
    float scale, inv_scale;   // storage scale of f - w (1 except F16)
    // collision and wall constants precomputed in both compute precisions
    // (the FP32 path does no double arithmetic per node)
    float f_om, f_pref, f_gx, f_gy, f_ub, f_ut, f_ub6, f_ut6;
    double d_om, d_pref, d_ub6, d_ut6;
    float f_nu;
    double d_nu;        // kinematic viscosity (tau - 1/2) / 3
    void *pop[2];             // A/B population buffers
    int *cur;                 // device: which buffer holds the latest f*
    long long *step;          // device: completed steps
    int *err;                 // device: error bits
};

// Bounds checks of the debug build (-DLBIB_DEBUG): an element index i of a
// population buffer ([9][ny][nx]) with `span` consecutive elements must lie
// in [0, 9 nx ny - span].  Out of range, the simulation's error word gets
// ERR_BOUNDS (reported as LBIB_E_BOUNDS), loads read element 0 instead and
// stores are dropped.  The debug build also checks the bulk pass's per-tile
// near-box counts (BatchDev::tile_boxes): a node of a near box in a tile
// counted free of them raises ERR_BOUNDS too.  Release builds compile the
// checks away.
__device__ __forceinline__ bool pop_index_ok(const SimDev &s, int i, int span = 1) {
#ifdef LBIB_DEBUG
    const int total = 9 * s.nx * s.ny;
    if (i < 0 || i > total - span) {
        if (s.err) atomicOr(s.err, ERR_BOUNDS);
        return false;
    }
#endif
    return true;
}
__device__ __forceinline__ int pop_load_index(const SimDev &s, int i, int span = 1) {
    return pop_index_ok(s, i, span) ? i : 0;
}

// Row of node index k: with t = ceil(log2 nx), m = ceil(2^(31+t) / nx) < 2^32
// and k = q nx + r, k m / 2^(31+t) = q + r / nx + k e / (nx 2^(31+t)) with
// e = m nx - 2^(31+t) < nx, and the last two terms stay below 1 for k < 2^31,
// so the shifted high product is exactly q.
__device__ __forceinline__ int div_nx(const SimDev &s, int k) {
    return (int)(__umulhi((unsigned)k, s.nx_m) >> s.nx_s);
}

// Rigid particle, resident in device memory (FP64 state and loads).
struct ParticleDev {
    double xc, yc, th, u, v, om;        // pose and velocities at step n
    double xc1, yc1, th1, u1, v1, om1;  // one step earlier
    double mass, inertia, r_eq, sigma;
    double inv_mass, inv_inertia;
    double Fh[2], Mh, Fb[2], Mb, Fw[2];
    double gap[2];                      // smallest element gap to the bottom / top wall line
    int nl, n_ligands, n_probing, n_bonded;
    int fixed, T, ncolors, tile_ox;     // T: force-tile edge; tile origin x in [0, nx)
    int tile_oy, NBx, vb_p, NBy;        // NBx, NBy: edges of the near box; vb_p: half
                                        // bandwidth of the spreading-scale system
    long long step;                     // completed steps of this particle (bond draws)
    // Near box of the lattice step that reads buffer parity p: nodes
    // [box_ox[p], +NBx) x [box_oy[p], +NBy), x wrapped to [0, nx).  The particle
    // kernel of step k leaves the box for step k + 2 in pend_ox / pend_oy; the
    // near lattice kernel of step k + 1 publishes it into the slot of step k + 2.
    int box_ox[2], box_oy[2];
    int pend_ox, pend_oy;
    // body-frame element centroids, outward normals and lengths
    const double *mbx, *mby, *nbx, *nby, *S;
    const uint8_t *ligand;
    const int *color_order;  // markers grouped by colour
    const int *color_off;    // [ncolors + 1]
    uint8_t *bond;
    double *anchor_x;
    int8_t *anchor_wall;
    void *tile;              // IB force density, [2][T][T] of the compute type
    double *pf_tab;          // P_f by probing count, bottom [nl+1] then top [nl+1]
    // Pose in the compute precision left by the last particle pass for the
    // next one (pose_ok = 1), so that a pass starts without the FP64 pose
    // arithmetic: the centroid's floor node, then its offset from it, cos and
    // sin of the angle, the centroid's distances to the bottom and top wall
    // lines, and the velocities u, v, omega.
    int pose_ok, pose_ixc, pose_iyc, pose_pad;
    double pose_r[9];
    // Per-element record of the compute type, [nl][ECACHE] (or null), rewritten
    // by every pass for the next one (valid with pose_ok): body-frame centroid
    // x, y, normal x, y, length, the marker offset x, y and normal x, y at the
    // pose above, ligand flag, colour order entry, colour offset (entries
    // 0 .. ncolors - 1).  Rewriting keeps it in L2 between passes.
    void *ecache;
};
constexpr int ECACHE = 12;

// Per batch particle: its element record (ParticleDev::ecache) and element
// count, so that a particle pass can load the record in the same round as the
// descriptor.
struct PartRec {
    void *erec;
    int nl, pad;
};

// Per lattice work tile: its simulation, its first node, and the range of the
// batch's particles (and near boxes) of that simulation.
struct TileDev {
    int sim, k0, p0, np;
};

// A particle's near boxes (ParticleDev::box_ox / box_oy, both parities) and
// edge, copied into one flat per-batch table so that the bulk pass finds
// them in one load round, independent of the parity.
struct NearBox {
    int ox0, oy0, ox1, oy1;
    int NBx, NBy, pad[2];
};

// The bulk pass reads its tile, the simulation's descriptor, its parity and
// its near boxes in two rounds of loads (tile; descriptor, parity and boxes),
// not through a chain of dependent loads: the batch keeps its own copies of
// the members' parity words (par) and near boxes (nbox).  They are refreshed
// from the members before every batched call, the parity flip updates both
// copies, and the near-box pass publishes each new box into both.  Most tiles
// meet no near box: per tile and box slot, tile_boxes counts the near boxes
// that reach into the tile (through their whole rows where a row is at most
// a tile, through their spans of each row on wider lattices), and a tile
// whose count is zero skips the near-box test altogether.  The counts are
// rebuilt with the copies and kept by the near-box pass, which moves a box's
// counts from its old tiles to its new ones when it publishes it.
struct BatchDev {
    SimDev *sims;
    ParticleDev **parts;
    const PartRec *prec;     // [nparts] or null
    int *part_sim;
    const TileDev *tiles;    // lattice work tile -> its simulation, first node, particles
    int *par;                // [nsims] copy of each member's parity word (*SimDev::cur)
    NearBox *nbox;           // [nparts] copy of each particle's near boxes
    unsigned *tile_boxes;    // [total_tiles] near boxes reaching the tile: slot 0 in
                             // the low 16 bits, slot 1 in the high 16 bits
    int *near_part;      // near-box work tile -> batch particle index
    int *near_tile0;     // first near-box tile of each batch particle
    int total_near_tiles;
    int nsims, nparts, total_tiles;
    int lat_variant;     // bulk-pass kernel variant (0 .. LBIB_LATTICE_VARIANTS - 1)
    int tma_ok;          // every lattice suits the copy-engine variants (4, 5)
    int pthreads;        // particle CTA width: 256 (every particle fits) or 512
    int wait_polls;      // polls of a bounded device wait before it gives up
    int any_aa;          // a member streams in place
};

// Stochastic rounding of 16-bit stores.  A node's dither word is a hash of
// its index and of the bits of its first post-collision deviation (so it is
// deterministic and independent of the batch), spread over the nine planes
// by one affine map each.  The conversion is the stochastic-rounding cvt of
// the sm_100 family, on pairs: for each 16-bit half of its random operand it
// adds the low 13 (FP16: the mantissa bits that FP32 -> FP16 drops) or 16
// (BF16) bits below the kept mantissa and truncates, which rounds up with
// probability equal to the dropped fraction, for either sign.  Value v of a
// node takes the upper 16 bits of its plane word; a pair of nodes packs
// theirs with one byte permute, and a single value takes the same bits in
// both halves, so every path gives a node the same bits.
__device__ __forceinline__ unsigned mix32(unsigned x) {   // "lowbias32" (C. Wellons)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ unsigned dither_word(int k, float d0) {
    return mix32((unsigned)k * 0x9e3779b9u ^ __float_as_uint(d0));
}
__device__ __forceinline__ unsigned dither_plane(unsigned h, int i) {
    // an affine bijection per plane (odd multiplier): one multiply-add
    return h * (0x9e3779b1u + 0x3c6ef372u * (unsigned)i) + 0x7f4a7c15u * (unsigned)(i + 1);
}
// the random operand of a pair: lo's upper 16 bits below hi's
__device__ __forceinline__ unsigned dither_pair(unsigned r_lo, unsigned r_hi) {
    return __byte_perm(r_lo, r_hi, 0x7632);
}
__device__ __forceinline__ unsigned cvt_rs_f16x2(float hi, float lo, unsigned rbits) {
    unsigned d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}
__device__ __forceinline__ unsigned cvt_rs_bf16x2(float hi, float lo, unsigned rbits) {
    unsigned d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}
__device__ __forceinline__ __half half_sr(float x, unsigned r) {
    return __ushort_as_half((unsigned short)cvt_rs_f16x2(x, x, dither_pair(r, r)));
}
__device__ __forceinline__ __nv_bfloat16 bf16_sr(float x, unsigned r) {
    return __ushort_as_bfloat16((unsigned short)cvt_rs_bf16x2(x, x, dither_pair(r, r)));
}

// Storage traits: load a deviation into the compute type, store one back.
template <typename S> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p, int i, float) { return __ldg(p + i); }
    static __device__ __forceinline__ void st(float *p, int i, float v, float) { p[i] = v; }
    // evict-first forms for the bulk pass, so that its stream does not push
    // the particle data and code out of L2
    static __device__ __forceinline__ float ld_cs(const float *p, int i, float) { return __ldcs(p + i); }
    static __device__ __forceinline__ void st_cs(float *p, int i, float v, float) { __stcs(p + i, v); }
    template <bool STREAM>
    static __device__ __forceinline__ void st_r(float *p, int i, float v, float sc, unsigned) {
        if constexpr (STREAM) st_cs(p, i, v, sc); else st(p, i, v, sc);
    }
};
template <> struct Store<double> {
    static __device__ __forceinline__ double ld(const double *p, int i, float) { return __ldg(p + i); }
    static __device__ __forceinline__ void st(double *p, int i, double v, float) { p[i] = v; }
    static __device__ __forceinline__ double ld_cs(const double *p, int i, float) { return __ldcs(p + i); }
    static __device__ __forceinline__ void st_cs(double *p, int i, double v, float) { __stcs(p + i, v); }
    template <bool STREAM>
    static __device__ __forceinline__ void st_r(double *p, int i, double v, float sc, unsigned) {
        if constexpr (STREAM) st_cs(p, i, v, sc); else st(p, i, v, sc);
    }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p, int i, float inv) {
        return __half2float(p[i]) * inv;
    }
    static __device__ __forceinline__ void st(__half *p, int i, float v, float scale) {
        p[i] = __float2half_rn(v * scale);
    }
    static __device__ __forceinline__ float ld_cs(const __half *p, int i, float inv) {
        return __half2float(__ldcs(p + i)) * inv;
    }
    static __device__ __forceinline__ void st_cs(__half *p, int i, float v, float scale) {
        __stcs(p + i, __float2half_rn(v * scale));
    }
    template <bool STREAM>
    static __device__ __forceinline__ void st_r(__half *p, int i, float v, float scale, unsigned r) {
        const __half h = half_sr(v * scale, r);
        if constexpr (STREAM) __stcs(p + i, h); else p[i] = h;
    }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, int i, float inv) {
        return __bfloat162float(p[i]) * inv;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, int i, float v, float scale) {
        p[i] = __float2bfloat16_rn(v * scale);
    }
    static __device__ __forceinline__ float ld_cs(const __nv_bfloat16 *p, int i, float inv) {
        return __bfloat162float(__ldcs(p + i)) * inv;
    }
    static __device__ __forceinline__ void st_cs(__nv_bfloat16 *p, int i, float v, float scale) {
        __stcs(p + i, __float2bfloat16_rn(v * scale));
    }
    template <bool STREAM>
    static __device__ __forceinline__ void st_r(__nv_bfloat16 *p, int i, float v, float scale,
                                                unsigned r) {
        const __nv_bfloat16 h = bf16_sr(v * scale, r);
        if constexpr (STREAM) __stcs(p + i, h); else p[i] = h;
    }
};

// Four consecutive deviations (16-byte aligned for FP32, 8 for FP16/BF16,
// 32 for FP64) into / out of the compute type.  STREAM: evict-first.
template <bool STREAM, typename T>
__device__ __forceinline__ T ldv(const T *p) {
    if constexpr (STREAM) return __ldcs(p); else return __ldg(p);
}
template <bool STREAM, typename T>
__device__ __forceinline__ void stv(T *p, T v) {
    if constexpr (STREAM) __stcs(p, v); else *p = v;
}
template <typename S, bool STREAM> struct Vec4;
template <bool STREAM> struct Vec4<float, STREAM> {
    static __device__ __forceinline__ void ld(const float *p, float, float o[4]) {
        const float4 v = ldv<STREAM>((const float4 *)p);
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    static __device__ __forceinline__ void st(float *p, const float o[4], float) {
        stv<STREAM>((float4 *)p, make_float4(o[0], o[1], o[2], o[3]));
    }
    static __device__ __forceinline__ void st_r(float *p, const float o[4], float sc,
                                                const unsigned *) {
        st(p, o, sc);
    }
};
template <bool STREAM> struct Vec4<double, STREAM> {
    static __device__ __forceinline__ void ld(const double *p, float, double o[4]) {
        const double2 a = ldv<STREAM>((const double2 *)p), b = ldv<STREAM>((const double2 *)p + 1);
        o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
    }
    static __device__ __forceinline__ void st(double *p, const double o[4], float) {
        stv<STREAM>((double2 *)p, make_double2(o[0], o[1]));
        stv<STREAM>((double2 *)p + 1, make_double2(o[2], o[3]));
    }
    static __device__ __forceinline__ void st_r(double *p, const double o[4], float sc,
                                                const unsigned *) {
        st(p, o, sc);
    }
};
template <bool STREAM> struct Vec4<__half, STREAM> {
    static __device__ __forceinline__ void ld(const __half *p, float inv, float o[4]) {
        const uint2 u = ldv<STREAM>((const uint2 *)p);
        __half2 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        o[0] = fa.x * inv; o[1] = fa.y * inv; o[2] = fb.x * inv; o[3] = fb.y * inv;
    }
    static __device__ __forceinline__ void st(__half *p, const float o[4], float sc) {
        const __half2 a = __floats2half2_rn(o[0] * sc, o[1] * sc);
        const __half2 b = __floats2half2_rn(o[2] * sc, o[3] * sc);
        uint2 u;
        memcpy(&u.x, &a, 4);
        memcpy(&u.y, &b, 4);
        stv<STREAM>((uint2 *)p, u);
    }
    static __device__ __forceinline__ void st_r(__half *p, const float o[4], float sc,
                                                const unsigned *r) {
        uint2 u;
        u.x = cvt_rs_f16x2(o[1] * sc, o[0] * sc, dither_pair(r[0], r[1]));
        u.y = cvt_rs_f16x2(o[3] * sc, o[2] * sc, dither_pair(r[2], r[3]));
        stv<STREAM>((uint2 *)p, u);
    }
};
template <bool STREAM> struct Vec4<__nv_bfloat16, STREAM> {
    static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, float inv, float o[4]) {
        const uint2 u = ldv<STREAM>((const uint2 *)p);
        __nv_bfloat162 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        o[0] = fa.x * inv; o[1] = fa.y * inv; o[2] = fb.x * inv; o[3] = fb.y * inv;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, const float o[4], float sc) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(o[0] * sc, o[1] * sc);
        const __nv_bfloat162 b = __floats2bfloat162_rn(o[2] * sc, o[3] * sc);
        uint2 u;
        memcpy(&u.x, &a, 4);
        memcpy(&u.y, &b, 4);
        stv<STREAM>((uint2 *)p, u);
    }
    static __device__ __forceinline__ void st_r(__nv_bfloat16 *p, const float o[4], float sc,
                                                const unsigned *r) {
        uint2 u;
        u.x = cvt_rs_bf16x2(o[1] * sc, o[0] * sc, dither_pair(r[0], r[1]));
        u.y = cvt_rs_bf16x2(o[3] * sc, o[2] * sc, dither_pair(r[2], r[3]));
        stv<STREAM>((uint2 *)p, u);
    }
};

// Precomputed constant in the compute precision R.
template <typename R>
__device__ __forceinline__ R pick(float f, double d) {
    if constexpr (sizeof(R) == 4) return f; else return d;
}

// In-place (AA) streaming keeps one buffer F, its state alternating in
// parity (the device word `cur`):
//  - parity 0, after a swap step: F[opp(i)][x] = g_i(x), the post-collision
//    population i of node x kept at the node in the opposite slot;
//  - parity 1, after a push step: F[i][x + e_i] = g_i(x), already streamed.
// A step from parity 1 reads f_i(x) = F[i][x] and stores g_i(x) in
// F[opp(i)][x]; a step from parity 0 reads f_i(x) = F[opp(i)][x - e_i] and
// stores g_i(x) in F[i][x + e_i].  Each node reads and writes the same nine
// slots, so the update is race-free in place.  A population leaving through
// a non-periodic wall is kept, as it is, in F[opp(i)][x] (both parities);
// the moving-wall term of bounce-back is added where it is read, as in the
// A/B pull, so the two schemes give the same bits.  The step of A/B stepping
// from the buffer `cur` is the step of AA stepping from parity `cur`.
//
// Pre-collision deviations of node (x, y) for the coming step, pulled from
// the post-collision buffer `src` (Eq. 1 LHS): population i comes from
// (x - e_i) (AA: from state parity `par` of the single buffer, as above).
// x is periodic; rows beyond the walls follow the wall kind:
//  - periodic: wrap in y;
//  - half-way bounce-back: the node's own opposite population plus the
//    moving-wall term 6 w_i (e_i . u_w) (rho_w = 1);
//  - Zou-He: the three unknowns are rebuilt from the known ones and the wall
//    velocity (u_w, 0), in deviation form (all weights cancel, rho = 1 + ...).
// Directions (Eq. 3): 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1)
// 7 (-1,-1) 8 (1,-1).

template <typename S, typename R, bool STREAM = false>
__device__ __forceinline__ void pull_node(const SimDev &s, const S *__restrict__ src, int x,
                                          int y, R d[9], int par = 0) {
    auto ld = [&](int i, float inv) -> R {
        i = pop_load_index(s, i);
        if constexpr (STREAM) return Store<S>::ld_cs(src, i, inv); else return Store<S>::ld(src, i, inv);
    };
    const int nx = s.nx, ny = s.ny;
    const int N = nx * ny;                 // 9 N < 2^31 is checked at creation
    const float inv = s.inv_scale;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x == nx - 1) ? 0 : x + 1;
    int ym = y - 1, yp = y + 1;
    bool bot = ym < 0, top = yp >= ny;
    if (s.wall_b == LBIB_WALL_PERIODIC) {
        if (bot) ym = ny - 1;
        if (top) yp = 0;
        bot = top = false;
    }
    const int r0 = y * nx, own = r0 + x;
    const bool aa = s.aa != 0;
    // population i (opposite o) pulled from neighbour node nb: A/B plane i
    // at nb; AA parity 0 plane o at nb; AA parity 1 plane i at the node
    auto pin = [&](int i, int o, int nb) -> R {
        return ld(!aa ? i * N + nb : (par ? i * N + own : o * N + nb), inv);
    };
    // population i from beyond a bounce-back wall: the node's own population
    // o after its last collision (A/B plane o; AA plane i)
    auto pwall = [&](int i, int o) -> R { return ld((aa ? i : o) * N + own, inv); };
    d[0] = ld(own, inv);
    d[1] = pin(1, 3, r0 + xm);
    d[3] = pin(3, 1, r0 + xp);
    if (!bot) {
        const int rm = ym * nx;
        d[2] = pin(2, 4, rm + x);
        d[5] = pin(5, 7, rm + xm);
        d[6] = pin(6, 8, rm + xp);
    } else if (s.wall_b == LBIB_WALL_BOUNCE_BACK) {
        const R uw6 = pick<R>(s.f_ub6, s.d_ub6);
        d[2] = pwall(2, 4);
        d[5] = pwall(5, 7) + uw6;
        d[6] = pwall(6, 8) - uw6;
    }
    if (!top) {
        const int rp = yp * nx;
        d[4] = pin(4, 2, rp + x);
        d[7] = pin(7, 5, rp + xp);
        d[8] = pin(8, 6, rp + xm);
    } else if (s.wall_t == LBIB_WALL_BOUNCE_BACK) {
        const R uw6 = pick<R>(s.f_ut6, s.d_ut6);
        d[4] = pwall(4, 2);
        d[7] = pwall(7, 5) - uw6;
        d[8] = pwall(8, 6) + uw6;
    }
    if (bot && s.wall_b == LBIB_WALL_ZOU_HE) {
        const R uw = pick<R>(s.f_ub, s.u_b);
        const R rho = (R)1 + d[0] + d[1] + d[3] + (R)2 * (d[4] + d[7] + d[8]);
        const R h = (R)0.5 * (d[1] - d[3]);
        d[2] = d[4];
        d[5] = d[7] - h + (R)0.5 * rho * uw;
        d[6] = d[8] + h - (R)0.5 * rho * uw;
    }
    if (top && s.wall_t == LBIB_WALL_ZOU_HE) {
        const R uw = pick<R>(s.f_ut, s.u_t);
        const R rho = (R)1 + d[0] + d[1] + d[3] + (R)2 * (d[2] + d[5] + d[6]);
        const R h = (R)0.5 * (d[1] - d[3]);
        d[4] = d[2];
        d[7] = d[5] + h - (R)0.5 * rho * uw;
        d[8] = d[6] - h + (R)0.5 * rho * uw;
    }
}

// Buffer index of post-collision population i of node k (at (x, y)) as the
// step from state `par` stores it: A/B plane i at k; AA (see above) parity 1
// plane opp(i) at k, parity 0 plane i at x + e_i, or plane opp(i) at k when
// x + e_i lies beyond a non-periodic wall.
__device__ __forceinline__ int post_index(const SimDev &s, int i, int k, int x, int y, int par) {
    constexpr int EXo[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int EYo[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    constexpr int OPo[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const int N = s.nx * s.ny;
    if (!s.aa) return i * N + k;
    if (par) return OPo[i] * N + k;
    int xx = x + EXo[i], yy = y + EYo[i];
    if (xx < 0) xx += s.nx;
    if (xx >= s.nx) xx -= s.nx;
    if (yy < 0 || yy >= s.ny) {
        if (s.wall_b != LBIB_WALL_PERIODIC) return OPo[i] * N + k;
        yy = yy < 0 ? yy + s.ny : yy - s.ny;
    }
    return i * N + yy * s.nx + xx;
}

// Density deviation and momentum of a set of deviations (sum_i w_i e_i = 0).
template <typename R>
__device__ __forceinline__ void node_moments(const R d[9], R &drho, R &jx, R &jy) {
    drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
}

// Core of the near box: the force tile plus four nodes a side.  It contains
// the force tile and the staged region (plus its pull halo) of the next
// particle pass for any motion below one node per step.
__host__ __device__ __forceinline__ int near_core(int T) { return T + 8; }
// Edges of the near box: in x the core widened by three nodes and rounded up
// to a multiple of four, so that the box can start on a multiple of four
// (the bulk pass's groups of four nodes then lie wholly inside a box or
// wholly outside it) and still contain the core; in y the core.
__host__ __device__ __forceinline__ int near_edge_x(int T) { return (near_core(T) + 6) & ~3; }
__host__ __device__ __forceinline__ int near_edge_y(int T) { return near_core(T); }

// Force-tile lookup: IB force density at (x, y) summed over the simulation's
// particles whose tile covers the node.
template <typename R>
__device__ __forceinline__ void tile_force(const SimDev &s, ParticleDev *const *parts, int x,
                                           int y, R &fx, R &fy) {
    for (int k = 0; k < s.np; ++k) {
        const ParticleDev *p = parts[s.p0 + k];
        const int T = p->T;
        int dx = x - p->tile_ox;
        if (dx < 0) dx += s.nx;
        int dy = y - p->tile_oy;
        if (dy < 0 && s.wall_b == LBIB_WALL_PERIODIC) dy += s.ny;
        if (dx < T && (unsigned)dy < (unsigned)T) {
            const R *t = (const R *)p->tile;
            fx += t[dy * T + dx];
            fy += t[T * T + dy * T + dx];
        }
    }
}

// Launchers (defined in the .cu files), one instantiation per storage kind.
// mode: 0 every node; 1 bulk (nodes outside the near boxes); 2 near boxes only.
// flip bit 1 marks a timing run of modes 0 / 1 (step counters untouched).
// pdl: launched as a programmatic dependent of the kernel before it on st
// (mode 1: the bulk pass of the step before; mode 2: the particle pass)
cudaError_t launch_lattice(int kind, const BatchDev &b, int flip, int mode, cudaStream_t st,
                           bool pdl = false);
// mode: 0 overlapped step, 1 init (IB forcing at the current pose), 2 step
// without the near-box pass.  pdl: launched as a programmatic dependent of
// the previous kernel on st
cudaError_t launch_particles(int kind, const BatchDev &b, int flip, int mode, int smem,
                             cudaStream_t st, bool pdl = false);
// Allows the lattice-pass variants their dynamic shared memory (once per
// storage kind and device, before the first launch).
cudaError_t lattice_kernel_setup(int kind);
cudaError_t launch_fields(int kind, const SimDev &s, ParticleDev *const *parts, double *rho,
                          double *ux, double *uy, cudaStream_t st);
cudaError_t launch_populations(int kind, const SimDev &s, double *out, cudaStream_t st);
cudaError_t launch_set_populations(int kind, const SimDev &s, const double *in, cudaStream_t st);
// Flip each member's parity word and the batch's copy of it.
cudaError_t launch_flip(int *const *curs, int *par, int n, cudaStream_t st);
// Copy the members' parity words and near boxes into the batch (par, nbox).
cudaError_t launch_batch_refresh(const BatchDev &b, int *const *curs, cudaStream_t st);
cudaError_t launch_ib_export(int kind, const SimDev &s, ParticleDev *const *parts, double *fx,
                             double *fy, cudaStream_t st);
// vb: the particle's simulation solves its spreading scales (ib_spread = 1)
int particle_smem_bytes(int kind, int T, int nl, bool vb);
cudaError_t particle_kernel_setup(int kind, int smem);
int particle_smem_limit(int kind);

}  // namespace lbib
