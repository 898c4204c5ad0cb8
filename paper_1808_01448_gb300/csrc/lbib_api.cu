// lbib_api.cu -- host implementation of the C ABI declared in include/lbib.h.
//
// Owns device memory (through the caller's allocator hook or cudaMalloc),
// builds particle geometry, marker colouring and force tiles, and drives the
// two kernels of a time step (lattice, then particles) for a batch of
// simulations, replaying CUDA graphs of GRAPH_STEPS steps.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbib_internal.cuh"

using namespace lbib;

namespace {

constexpr int GRAPH_STEPS = 32;   // steps per captured graph (even: parity-neutral)
constexpr int SHORT_STEPS = 4;    // steps per graph of the remainder of a call (even)
constexpr int SMEM_LIMIT = 227 * 1024;

thread_local std::string g_err;

lbib_status fail(lbib_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

lbib_status cuda_fail(cudaError_t e, const char *what) {
    return fail(LBIB_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                        \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);             \
    } while (0)

// NVTX range around a C-ABI call (visible in profilers' timelines).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// Polls of a bounded device wait (the copy-engine staging of the lattice
// pass) before it gives up and reports LBIB_E_TIMEOUT: LBIB_WAIT_POLLS from
// the environment when a batch is created (0 .. 2^24), else 65536.
int wait_polls_setting() {
    const char *e = getenv("LBIB_WAIT_POLLS");
    if (!e || !*e) return 1 << 16;
    char *end = nullptr;
    const long v = strtol(e, &end, 10);
    if (end == e || v < 0) return 1 << 16;
    return (int)std::min<long>(v, 1 << 24);
}

// L2 clearing before a timed step: writing a buffer larger than L2 evicts
// every line the step could reuse; reading it back then replaces the dirty
// lines of the write with clean ones.
__global__ void __launch_bounds__(512) l2_fill_kernel(uint4 *buf, size_t n, unsigned v) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride)
        buf[i] = make_uint4(v, v + 1, v + 2, v + 3);
}

__global__ void __launch_bounds__(512) l2_read_kernel(uint4 *buf, size_t n, unsigned v) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    unsigned acc = 0;
    for (size_t i = i0; i < n; i += stride) {
        const uint4 q = buf[i];
        acc |= (q.x ^ v) | (q.y ^ (v + 1)) | (q.z ^ (v + 2)) | (q.w ^ (v + 3));
    }
    if (acc && i0 < n) buf[i0].x = acc;     // never taken; keeps the loads
}

cudaError_t launch_l2_flush(void *buf, size_t bytes, bool clean, unsigned tag, cudaStream_t st) {
    const size_t n = bytes / sizeof(uint4);
    const int grid = (int)std::min<size_t>((n + 511) / 512, 4096);
    const unsigned v = 0x5a5a0000u ^ (tag << 2);
    l2_fill_kernel<<<grid, 512, 0, st>>>((uint4 *)buf, n, v);
    if (clean) l2_read_kernel<<<grid, 512, 0, st>>>((uint4 *)buf, n, v);
    return cudaGetLastError();
}

// Batched readback: block k < nparts copies particle record k, the last
// block the members' error words.
__global__ void __launch_bounds__(128) gather_states_kernel(ParticleDev *const *parts, int nparts,
                                                            const SimDev *sims, int nsims,
                                                            ParticleDev *out, int *err_out) {
    if ((int)blockIdx.x < nparts) {
        const unsigned *src = (const unsigned *)parts[blockIdx.x];
        unsigned *dst = (unsigned *)(out + blockIdx.x);
        for (int i = threadIdx.x; i < (int)(sizeof(ParticleDev) / 4); i += blockDim.x) dst[i] = src[i];
    } else {
        for (int i = threadIdx.x; i < nsims; i += blockDim.x) err_out[i] = *sims[i].err;
    }
}

size_t compute_size(int kind) { return kind == ST_F64 ? 8 : 4; }
size_t storage_size(int kind) {
    switch (kind) {
        case ST_F32: return 4;
        case ST_F64: return 8;
        default: return 2;
    }
}

struct HostParticle {
    std::vector<double> vx, vy;
    int fixed = 0;
    double xc = 0, yc = 0, th = 0, rho_p = 1, lig = 0, sigma = 0;
    int nl = 0, n_ligands = 0, T = 0, ncolors = 0;
    int vb_p = 0;                    // half bandwidth of the spreading-scale system
    double area = 0, mass = 0, inertia = 0, r_eq = 0, rmax = 0;
    std::vector<double> mbx, mby, nbx, nby, S;
    std::vector<uint8_t> ligand;
    std::vector<int> color_order, color_off;
    ParticleDev *d_part = nullptr;   // device struct
    void *d_ecache = nullptr;        // its element record (inside d_block)
    double *d_pftab = nullptr;       // its P_f table (inside d_block)
    void *d_block = nullptr;         // geometry, bonds, tile
    size_t d_bytes = 0;              // size of d_block
};

}  // namespace

struct lbib_sim {
    lbib_config cfg{};
    int kind = ST_F32;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    size_t N = 0;
    void *pop[2] = {nullptr, nullptr};
    int cur = 0;                  // host mirror of *d_cur
    int64_t step = 0;             // host count of enqueued steps
    int *d_cur = nullptr;         // small device block: cur, err, step
    int *d_err = nullptr;
    long long *d_step = nullptr;
    void *d_small = nullptr;
    double *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    float scale = 1.f;
    bool primed = false;
    std::vector<HostParticle> parts;
    lbib_batch *self = nullptr;           // private batch of one (lbib_step)
    std::vector<lbib_batch *> batches;    // user batches that contain this simulation
};

struct lbib_batch {
    std::vector<lbib_sim *> sims;
    int kind = ST_F32;
    cudaStream_t stream = nullptr;
    void *d_block = nullptr;
    int **d_curs = nullptr;             // device table of the members' parity words
    BatchDev bd{};
    int smem = 0;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t graph_short = nullptr;   // SHORT_STEPS steps, for remainders
    // timing: one graph exec per sample slot, each with events around the
    // first step's kernels
    int nsamples = 0;
    std::vector<cudaGraphExec_t> tgraphs;
    std::vector<cudaEvent_t> ev;        // 6 per slot: lattice, particle, near (start, end)
    std::vector<int> replayed;          // slot replayed since the last read
    int next_slot = 0;
    lbib_config acfg{};                 // allocator hook used for d_block
    size_t d_bytes = 0;                 // size of d_block
    bool is_self = false;
    bool orphan = false;                // a member was destroyed: the batch is unusable
    // overlapped stepping: the bulk lattice pass runs on s2 while the particle
    // pass of the previous step runs on `stream`
    // (s1: near + particle passes, high priority; s2: bulk passes, low
    // priority, so freed SMs go to the particle pass first)
    bool overlap = false;
    // each step's bulk pass launched as a programmatic dependent of the one
    // before: for batches whose step the bulk pass bounds (see make_batch)
    bool bulk_pdl = false;
    cudaStream_t s1 = nullptr, s2 = nullptr;
    cudaEvent_t evb[2] = {nullptr, nullptr}, evn[2] = {nullptr, nullptr};
    cudaEvent_t evfork = nullptr, evjoin = nullptr, evjoin1 = nullptr;
    // flushed stepping: a graph of GRAPH_STEPS steps, each after an L2 flush
    // of fbuf, with FEV events per step
    cudaGraphExec_t fgraph = nullptr;
    void *fbuf = nullptr;
    size_t fbytes = 0;
    int fclean = -1;
    std::vector<cudaEvent_t> fev;
    // batched state readback: the members' particle records and error words
    // gathered on the device, then one copy into pinned host memory
    void *d_rb = nullptr, *h_rb = nullptr;
    cudaEvent_t ev_rb = nullptr;        // the staged copy has landed
    bool rb_pending = false;            // a started readback awaits collection
    int *d_errs = nullptr, *h_errs = nullptr;   // members' error words (synchronize)
};

namespace {

void *dalloc(const lbib_config &c, cudaStream_t st, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c.alloc) return c.alloc(bytes, (void *)st, c.alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dfree(const lbib_config &c, cudaStream_t st, void *p) {
    if (!p) return;
    if (c.free) c.free(p, (void *)st, c.alloc_ctx);
    else cudaFree(p);
}

// Device descriptor of a channel from its configuration, its two population
// buffers (f - w of the storage type), its device words (current buffer,
// completed steps, error bits; step and err may be null for a pass that
// writes neither), its storage scale and its particles' range [p0, p0 + np)
// in a batch table.
SimDev simdev_from(const lbib_config &c, void *pop0, void *pop1, int *cur, long long *step,
                   int *err, float scale, int p0, int np, int tile0) {
    SimDev d{};
    d.nx = c.nx; d.ny = c.ny; d.wall_b = c.wall_bottom; d.wall_t = c.wall_top;
    {
        int t = 0;
        while ((1 << t) < c.nx) ++t;
        const unsigned long long p2 = 1ull << (31 + t);
        d.nx_m = (unsigned)((p2 + (unsigned long long)c.nx - 1) / (unsigned long long)c.nx);
        d.nx_s = t - 1;
    }
    d.p0 = p0; d.np = np;
    d.tile0 = tile0;
    d.ntiles = (int)(((size_t)c.nx * c.ny + LB_TILE_NODES - 1) / LB_TILE_NODES);
    d.tau = c.tau; d.u_b = c.u_bottom; d.u_t = c.u_top; d.gx = c.gx; d.gy = c.gy;
    d.k_f = c.k_f; d.k_r0 = c.k_r0; d.kBT = c.kBT; d.sigma_star_ratio = c.sigma_star_ratio;
    d.y_cr = c.y_cr; d.y_eq_ratio = c.y_eq_ratio; d.hamaker = c.hamaker; d.eps_min = c.eps_min;
    d.rec_b = c.receptor_bottom; d.rec_t = c.receptor_top;
    d.seed = c.seed; d.sim_id = c.sim_id;
    d.scale = scale; d.inv_scale = 1.f / scale;
    const double om = 1.0 / c.tau;
    d.d_om = om; d.d_pref = 1.0 - 0.5 * om;
    d.d_ub6 = c.u_bottom / 6.0; d.d_ut6 = c.u_top / 6.0;
    d.f_om = (float)om; d.f_pref = (float)d.d_pref;
    d.f_gx = (float)c.gx; d.f_gy = (float)c.gy;
    d.f_ub = (float)c.u_bottom; d.f_ut = (float)c.u_top;
    d.f_ub6 = (float)d.d_ub6; d.f_ut6 = (float)d.d_ut6;
    d.d_nu = (c.tau - 0.5) / 3.0; d.f_nu = (float)d.d_nu;
    d.pop[0] = pop0; d.pop[1] = pop1;
    d.cur = cur; d.step = step; d.err = err;
    d.aa = c.stream_mode == 1;
    // vector path (A/B streaming): whole groups of four nodes per row,
    // buffers 32-byte aligned
    d.vec4 = c.nx % 4 == 0 && ((uintptr_t)pop0 % 32) == 0 && ((uintptr_t)pop1 % 32) == 0;
    d.sround = c.rounding == LBIB_ROUND_STOCHASTIC;
    d.ib_iters = c.ib_iterations > 1 ? c.ib_iterations : 1;
    d.ib_spread = c.ib_spread != 0;
    return d;
}

SimDev make_simdev(const lbib_sim *s, int p0, int tile0) {
    return simdev_from(s->cfg, s->pop[0], s->pop[1], s->d_cur, s->d_step, s->d_err, s->scale, p0,
                       (int)s->parts.size(), tile0);
}

// Half bandwidth of a particle's spreading-scale system: the largest offset
// along the outline (cyclic) between two element centroids closer than
// 4 sqrt 2 (only such markers' 4 x 4 supports can share a node, at any pose),
// or -1 when it exceeds LBIB_VB_MAX_BAND or the outline is too short for a
// band of that width (n < 2 p + 2).
int vb_band(const double *mx, const double *my, int n) {
    const double r2 = 32.0;      // (4 sqrt 2)^2
    int p = 0;
    for (int l = 0; l < n; ++l)
        for (int d = 1; d <= n / 2; ++d) {
            const int m = (l + d) % n;
            const double dx = mx[m] - mx[l], dy = my[m] - my[l];
            if (dx * dx + dy * dy < r2) p = std::max(p, d);
        }
    if (p > LBIB_VB_MAX_BAND || n < 2 * p + 2) return -1;
    return std::max(p, 1);
}

// Marker colouring for the spreading: two markers of one colour are at least
// 4 sqrt 2 apart, so their 4 x 4 supports are disjoint in some axis for every
// rotation of the body, and each colour is one pass of the spreading.  Markers
// follow the outline, so colouring consecutive blocks of K or K + 1 markers
// 0, 1, 2, ... (K + 1 colours, same-colour markers at least K apart along the
// outline) usually needs fewer colours than a greedy pass, which leaves stray
// colours where the outline closes; so does a cyclic greedy pass (each marker
// takes the next free colour after its predecessor's).  The colouring with
// the fewest colours is kept.  No heap use.
// Returns the number of colours.
int color_markers(const double *mx, const double *my, int n, int *color) {
    const double D2 = 32.0 * (1.0 + 1e-9);
    auto valid = [&](const int *c) {
        for (int l = 0; l < n; ++l)
            for (int q = l + 1; q < n; ++q)
                if (c[l] == c[q]) {
                    const double dx = mx[l] - mx[q], dy = my[l] - my[q];
                    if (dx * dx + dy * dy < D2) return false;
                }
        return true;
    };
    // greedy in index order
    int nc = 0;
    for (int l = 0; l < n; ++l) {
        char used[LBIB_MAX_MARKERS + 1] = {0};
        for (int q = 0; q < l; ++q) {
            const double dx = mx[l] - mx[q], dy = my[l] - my[q];
            if (dx * dx + dy * dy < D2) used[color[q]] = 1;
        }
        int c = 0;
        while (c < nc && used[c]) ++c;
        color[l] = c;
        if (c == nc) ++nc;
    }
    // blocks of consecutive markers
    int blk[LBIB_MAX_MARKERS];
    for (int K = 2; K + 1 < nc && K <= n; ++K) {
        const int q = n / K, r = n % K;     // r blocks of K + 1, q - r of K
        if (q < r) continue;
        int l = 0;
        for (int b = 0; b < q; ++b)
            for (int j = 0; j < K + (b < r ? 1 : 0); ++j) blk[l++] = j;
        if (!valid(blk)) continue;
        for (int i = 0; i < n; ++i) color[i] = blk[i];
        nc = K + (r > 0 ? 1 : 0);
        break;
    }
    // cyclic greedy with C colours: each marker takes the first colour after
    // its predecessor's, in cyclic order, that no marker already coloured
    // within reach has
    for (int C = 2; C < nc; ++C) {
        bool ok = true;
        int prev = C - 1;
        for (int l = 0; l < n && ok; ++l) blk[l] = -1;
        for (int l = 0; l < n && ok; ++l) {
            char bad[LBIB_MAX_MARKERS + 1] = {0};
            for (int q = 0; q < n; ++q) {
                if (blk[q] < 0) continue;
                const double dx = mx[l] - mx[q], dy = my[l] - my[q];
                if (dx * dx + dy * dy < D2) bad[blk[q]] = 1;
            }
            int c = -1;
            for (int k = 1; k <= C; ++k)
                if (!bad[(prev + k) % C]) {
                    c = (prev + k) % C;
                    break;
                }
            if (c < 0) ok = false;
            else blk[l] = prev = c;
        }
        if (!ok) continue;
        for (int i = 0; i < n; ++i) color[i] = blk[i];
        nc = C;
        break;
    }
    return nc;
}

// Polygon elements, mass properties, ligands and marker colouring.
void build_geometry(HostParticle &p) {
    const int n = (int)p.vx.size();
    p.nl = n;
    p.mbx.resize(n); p.mby.resize(n); p.nbx.resize(n); p.nby.resize(n); p.S.resize(n);
    p.ligand.assign(n, 0);
    double A = 0, J = 0, rmax = 0;
    for (int l = 0; l < n; ++l) {
        const int m = (l + 1) % n;
        const double ax = p.vx[l], ay = p.vy[l], bx = p.vx[m], by = p.vy[m];
        const double dx = bx - ax, dy = by - ay, len = sqrt(dx * dx + dy * dy);
        p.mbx[l] = 0.5 * (ax + bx);
        p.mby[l] = 0.5 * (ay + by);
        p.S[l] = len;
        p.nbx[l] = dy / len;
        p.nby[l] = -dx / len;
        const double cr = ax * by - bx * ay;
        A += 0.5 * cr;
        J += cr * (ax * ax + ax * bx + bx * bx + ay * ay + ay * by + by * by) / 12.0;
        rmax = std::max(rmax, sqrt(ax * ax + ay * ay));
    }
    p.area = A;
    p.mass = p.rho_p * A;
    p.inertia = p.rho_p * J;
    p.r_eq = sqrt(A / M_PI);
    p.rmax = rmax;
    p.T = 2 * (int)ceil(rmax) + 8;
    p.n_ligands = 0;
    for (int l = 0; l < n; ++l) {
        p.ligand[l] = floor((double)(l + 1) * p.lig) > floor((double)l * p.lig);
        p.n_ligands += p.ligand[l];
    }
    std::vector<int> color(n, -1);
    const int nc = color_markers(p.mbx.data(), p.mby.data(), n, color.data());
    p.ncolors = nc;
    p.color_off.assign(nc + 1, 0);
    for (int l = 0; l < n; ++l) p.color_off[color[l] + 1]++;
    for (int c = 0; c < nc; ++c) p.color_off[c + 1] += p.color_off[c];
    p.color_order.resize(n);
    std::vector<int> fill(p.color_off.begin(), p.color_off.end() - 1);
    for (int l = 0; l < n; ++l) p.color_order[fill[color[l]]++] = l;
}

void ellipse_outline(double ax, double by, int n, std::vector<double> &vx,
                     std::vector<double> &vy) {
    const int M = 20000;
    std::vector<double> s(M + 1, 0.0);
    for (int i = 1; i <= M; ++i) {
        const double t0 = 2 * M_PI * (i - 1) / M, t1 = 2 * M_PI * i / M;
        const double dx = ax * (cos(t1) - cos(t0)), dy = by * (sin(t1) - sin(t0));
        s[i] = s[i - 1] + sqrt(dx * dx + dy * dy);
    }
    vx.resize(n);
    vy.resize(n);
    int i = 0;
    for (int k = 0; k < n; ++k) {
        const double target = s[M] * k / n;
        while (i < M && s[i + 1] < target) ++i;
        const double f = (s[i + 1] > s[i]) ? (target - s[i]) / (s[i + 1] - s[i]) : 0.0;
        const double t = 2 * M_PI * (i + f) / M;
        vx[k] = ax * cos(t);
        vy[k] = by * sin(t);
    }
}

lbib_status err_status(lbib_sim *s, int err) {
    if (err & ERR_BOUNDS)
        return fail(LBIB_E_BOUNDS, "simulation %llu: a population index failed the debug build's "
                    "bounds check", (unsigned long long)s->cfg.sim_id);
    if (err & ERR_TIMEOUT)
        return fail(LBIB_E_TIMEOUT, "simulation %llu: a bounded device wait of the lattice pass ran out",
                    (unsigned long long)s->cfg.sim_id);
    if (err & ERR_UNSTABLE)
        return fail(LBIB_E_UNSTABLE,
                    "simulation %llu became unstable (a node's state non-finite, |rho - 1| >= 1 "
                    "or |ux| + |uy| >= 10)",
                    (unsigned long long)s->cfg.sim_id);
    return LBIB_OK;
}

lbib_status check_err_word(lbib_sim *s) {
    int err = 0;
    CK(cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    return err_status(s, err);
}

// The public particle state from a device record and the host-side constants.
void fill_state(lbib_particle_state &o, const ParticleDev &h, const HostParticle &p) {
    o.xc = h.xc; o.yc = h.yc; o.theta = h.th; o.u = h.u; o.v = h.v; o.omega = h.om;
    o.Fh[0] = h.Fh[0]; o.Fh[1] = h.Fh[1]; o.Mh = h.Mh;
    o.Fb[0] = h.Fb[0]; o.Fb[1] = h.Fb[1]; o.Mb = h.Mb;
    o.Fw[0] = h.Fw[0]; o.Fw[1] = h.Fw[1];
    o.area = p.area; o.mass = p.mass; o.inertia = p.inertia; o.r_eq = p.r_eq;
    o.nl = p.nl; o.n_ligands = p.n_ligands; o.n_probing = h.n_probing;
    o.n_bonded = h.n_bonded;
    o.p_adhesion = h.n_probing > 0 ? (double)h.n_bonded / h.n_probing : 0.0;
    o.gap_bottom = h.gap[0];
    o.gap_top = h.gap[1];
}

lbib_status upload_particle(lbib_sim *s, HostParticle &p) {
    const int n = p.nl;
    const size_t rsz = compute_size(s->kind);
    const size_t bytes = sizeof(ParticleDev) + 5 * n * 8 + n + 4 * n + 4 * (p.ncolors + 1) + n +
                         16 * (size_t)(n + 1) +
                         8 * n + n + 2 * rsz * p.T * p.T + ECACHE * rsz * (size_t)n + 16 * 16;
    unsigned char *blk = (unsigned char *)dalloc(s->cfg, s->stream, bytes);
    if (!blk) return fail(LBIB_E_OOM, "device allocation of %zu bytes for a particle failed", bytes);
    p.d_block = blk;
    p.d_bytes = bytes;
    size_t off = 0;
    auto take = [&](size_t b) {
        unsigned char *q = blk + off;
        off += (b + 15) & ~size_t(15);
        return q;
    };
    ParticleDev h{};
    unsigned char *pd = take(sizeof(ParticleDev));
    double *mbx = (double *)take(8 * n), *mby = (double *)take(8 * n);
    double *nbx = (double *)take(8 * n), *nby = (double *)take(8 * n), *S = (double *)take(8 * n);
    uint8_t *lig = take(n);
    int *co = (int *)take(4 * n), *coff = (int *)take(4 * (p.ncolors + 1));
    uint8_t *bond = take(n);
    double *ax = (double *)take(8 * n);
    int8_t *aw = (int8_t *)take(n);
    void *tile = take(2 * rsz * p.T * p.T);
    double *pft = (double *)take(16 * (size_t)(n + 1));
    void *ecache = take(ECACHE * rsz * (size_t)n);
    h.xc = h.xc1 = p.xc; h.yc = h.yc1 = p.yc; h.th = h.th1 = p.th;
    h.mass = p.mass; h.inertia = p.inertia; h.r_eq = p.r_eq; h.sigma = p.sigma;
    h.inv_mass = 1.0 / p.mass; h.inv_inertia = 1.0 / p.inertia;
    h.nl = n; h.n_ligands = p.n_ligands; h.fixed = p.fixed; h.T = p.T; h.ncolors = p.ncolors;
    h.tile_ox = 0; h.tile_oy = -(1 << 28);   // no tile until the first IB pass
    h.gap[0] = h.gap[1] = INFINITY;          // no bond step yet
    h.NBx = near_edge_x(p.T); h.NBy = near_edge_y(p.T); h.step = 0;
    h.vb_p = p.vb_p;
    h.mbx = mbx; h.mby = mby; h.nbx = nbx; h.nby = nby; h.S = S;
    h.ligand = lig; h.color_order = co; h.color_off = coff;
    h.bond = bond; h.anchor_x = ax; h.anchor_wall = aw; h.tile = tile; h.pf_tab = pft;
    h.ecache = ecache;      // filled by the first pass (pose_ok = 0 until then)
    p.d_ecache = ecache;
    p.d_pftab = pft;
    p.d_part = (ParticleDev *)pd;
    cudaStream_t st = s->stream;
    CK(cudaMemcpyAsync(pd, &h, sizeof h, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(mbx, p.mbx.data(), 8 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(mby, p.mby.data(), 8 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(nbx, p.nbx.data(), 8 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(nby, p.nby.data(), 8 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(S, p.S.data(), 8 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(lig, p.ligand.data(), n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(co, p.color_order.data(), 4 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(coff, p.color_off.data(), 4 * (p.ncolors + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(bond, 0, n, st));
    CK(cudaMemsetAsync(ax, 0, 8 * n, st));
    CK(cudaMemsetAsync(aw, 0, n, st));
    CK(cudaMemsetAsync(tile, 0, 2 * rsz * p.T * p.T, st));
    CK(cudaStreamSynchronize(st));   // host vectors may be released afterwards
    return LBIB_OK;
}

void unregister(lbib_batch *b) {
    if (b->is_self || b->orphan) return;
    for (lbib_sim *s : b->sims) {
        auto &v = s->batches;
        v.erase(std::remove(v.begin(), v.end(), b), v.end());
    }
}

void free_batch(lbib_batch *b) {
    if (!b) return;
    unregister(b);
    if (b->s2 && !b->orphan) cudaStreamSynchronize(b->s2);
    if (b->s1 && !b->orphan) cudaStreamSynchronize(b->s1);
    for (cudaEvent_t e : {b->evb[0], b->evb[1], b->evn[0], b->evn[1], b->evfork, b->evjoin,
                          b->evjoin1})
        if (e) cudaEventDestroy(e);
    if (b->s2) cudaStreamDestroy(b->s2);
    if (b->s1) cudaStreamDestroy(b->s1);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_short) cudaGraphExecDestroy(b->graph_short);
    for (auto g : b->tgraphs)
        if (g) cudaGraphExecDestroy(g);
    for (auto e : b->ev) cudaEventDestroy(e);
    if (b->fgraph) cudaGraphExecDestroy(b->fgraph);
    for (auto e : b->fev) cudaEventDestroy(e);
    if (b->d_rb) dfree(b->acfg, b->orphan ? nullptr : b->stream, b->d_rb);
    if (b->h_rb) cudaFreeHost(b->h_rb);
    if (b->ev_rb) cudaEventDestroy(b->ev_rb);
    if (b->d_errs) dfree(b->acfg, b->orphan ? nullptr : b->stream, b->d_errs);
    if (b->h_errs) cudaFreeHost(b->h_errs);
    if (b->d_block) dfree(b->acfg, b->orphan ? nullptr : b->stream, b->d_block);
    delete b;
}

// Setup calls are allowed until the first step, while no user batch holds
// the simulation; they drop the private batch and the initial IB forcing.
lbib_status reopen_setup(lbib_sim *s, const char *what) {
    if (s->step > 0) return fail(LBIB_E_STATE, "%s: only before the first step", what);
    if (!s->batches.empty()) return fail(LBIB_E_STATE, "%s: the simulation is in a batch", what);
    if (s->self) {
        cudaStreamSynchronize(s->stream);
        free_batch(s->self);
        s->self = nullptr;
    }
    s->primed = false;
    return LBIB_OK;
}

lbib_status make_batch(lbib_sim *const *sims, int n, lbib_batch **out) {
    if (!sims || n <= 0 || !out) return fail(LBIB_E_ARG, "batch needs at least one simulation");
    lbib_batch *b = new (std::nothrow) lbib_batch();
    if (!b) return fail(LBIB_E_OOM, "host allocation failed");
    b->kind = sims[0]->kind;
    b->stream = sims[0]->stream;
    b->acfg = sims[0]->cfg;
    int nparts = 0, tiles = 0, smem = 0, near_tiles = 0;
    bool boxes_fit = true;
    for (int i = 0; i < n; ++i) {
        lbib_sim *s = sims[i];
        if (!s) { delete b; return fail(LBIB_E_ARG, "null simulation in batch"); }
        if (s->kind != b->kind) { delete b; return fail(LBIB_E_ARG, "batch members must share storage"); }
        if (s->device != sims[0]->device) { delete b; return fail(LBIB_E_ARG, "batch members must share the device"); }
        for (int j = 0; j < i; ++j)
            if (sims[j] == s) { delete b; return fail(LBIB_E_ARG, "simulation listed twice in batch"); }
        b->sims.push_back(s);
        nparts += (int)s->parts.size();
        tiles += (int)((s->N + LB_TILE_NODES - 1) / LB_TILE_NODES);
        for (auto &p : s->parts) {
            smem = std::max(smem, particle_smem_bytes(b->kind, p.T, p.nl, s->cfg.ib_spread != 0));
            const int NBx = near_edge_x(p.T), NBy = near_edge_y(p.T);
            near_tiles += (NBx * NBy + NEAR_TILE_NODES - 1) / NEAR_TILE_NODES;
            if (NBx > s->cfg.nx || (s->cfg.wall_bottom == LBIB_WALL_PERIODIC && NBy > s->cfg.ny))
                boxes_fit = false;
        }
    }
    const size_t bytes = sizeof(SimDev) * n + sizeof(ParticleDev *) * (nparts + 1) +
                         sizeof(PartRec) * (nparts + 1) +
                         sizeof(int) * (nparts + 1) + sizeof(int *) * n +
                         sizeof(TileDev) * (size_t)tiles + sizeof(int) * (size_t)(near_tiles + nparts) +
                         sizeof(int) * n + sizeof(NearBox) * (nparts + 1) +
                         sizeof(unsigned) * (size_t)tiles + 640;
    unsigned char *blk = (unsigned char *)dalloc(sims[0]->cfg, b->stream, bytes);
    if (!blk) { delete b; return fail(LBIB_E_OOM, "device allocation for the batch failed"); }
    b->d_block = blk;
    b->d_bytes = bytes;
    size_t off = 0;
    auto take = [&](size_t sz) {
        unsigned char *q = blk + off;
        off += (sz + 15) & ~size_t(15);
        return q;
    };
    SimDev *dsims = (SimDev *)take(sizeof(SimDev) * n);
    ParticleDev **dparts = (ParticleDev **)take(sizeof(ParticleDev *) * (nparts + 1));
    PartRec *dprec = (PartRec *)take(sizeof(PartRec) * (nparts + 1));
    int *dpsim = (int *)take(sizeof(int) * (nparts + 1));
    int **dcurs = (int **)take(sizeof(int *) * n);
    TileDev *dtiles = (TileDev *)take(sizeof(TileDev) * (size_t)tiles);
    int *dnpart = (int *)take(sizeof(int) * (size_t)(near_tiles + 1));
    int *dntile0 = (int *)take(sizeof(int) * (size_t)(nparts + 1));
    int *dpar = (int *)take(sizeof(int) * n);
    NearBox *dnbox = (NearBox *)take(sizeof(NearBox) * (nparts + 1));
    unsigned *dtboxes = (unsigned *)take(sizeof(unsigned) * (size_t)tiles);
    std::vector<SimDev> hs;
    std::vector<ParticleDev *> hp;
    std::vector<PartRec> hpr;
    std::vector<int> hps;
    std::vector<int *> hc;
    int tile0 = 0;
    for (int i = 0; i < n; ++i) {
        lbib_sim *s = sims[i];
        hs.push_back(make_simdev(s, (int)hp.size(), tile0));
        tile0 += hs.back().ntiles;
        for (auto &p : s->parts) {
            hp.push_back(p.d_part);
            hpr.push_back(PartRec{p.d_ecache, p.nl, 0});
            hps.push_back(i);
        }
        hc.push_back(s->d_cur);
    }
    hp.push_back(nullptr);
    hpr.push_back(PartRec{nullptr, 0, 0});
    hps.push_back(0);
    std::vector<TileDev> hts((size_t)tiles);
    for (int i = 0; i < n; ++i)
        for (int t = 0; t < hs[i].ntiles; ++t)
            hts[(size_t)hs[i].tile0 + t] = TileDev{i, t * LB_TILE_NODES, hs[i].p0, hs[i].np};
    std::vector<int> hnp, hnt0;
    for (int i = 0; i < n; ++i)
        for (auto &p : sims[i]->parts) {
            const int NBx = near_edge_x(p.T), NBy = near_edge_y(p.T);
            hnt0.push_back((int)hnp.size());
            for (int t = 0; t < (NBx * NBy + NEAR_TILE_NODES - 1) / NEAR_TILE_NODES; ++t)
                hnp.push_back((int)hnt0.size() - 1);
        }
    hnp.push_back(0);
    hnt0.push_back(0);
    cudaStream_t st = b->stream;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(dsims, hs.data(), sizeof(SimDev) * n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dparts, hp.data(), sizeof(ParticleDev *) * hp.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dprec, hpr.data(), sizeof(PartRec) * hpr.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dpsim, hps.data(), sizeof(int) * hps.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dcurs, hc.data(), sizeof(int *) * n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dtiles, hts.data(), sizeof(TileDev) * hts.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dnpart, hnp.data(), sizeof(int) * hnp.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(dntile0, hnt0.data(), sizeof(int) * hnt0.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaStreamSynchronize(st))) {
        free_batch(b);
        return cuda_fail(e, "batch upload");
    }
    const int smem_limit = nparts > 0 ? particle_smem_limit(b->kind) : 0;
    if (nparts > 0 && smem > smem_limit) {
        free_batch(b);
        return fail(LBIB_E_ARG, "particle kernel needs %d bytes of shared memory (limit %d)", smem,
                    smem_limit);
    }
    if (nparts > 0) {
        // allow the largest tile any batch may use (the attribute is per kernel)
        if ((e = particle_kernel_setup(b->kind, smem_limit)) != cudaSuccess) {
            free_batch(b);
            return cuda_fail(e, "particle kernel setup");
        }
    }
    b->smem = smem;
    b->bd.sims = dsims;
    b->bd.parts = dparts;
    b->bd.prec = dprec;
    b->bd.part_sim = dpsim;
    b->bd.tiles = dtiles;
    b->bd.par = dpar;
    b->bd.nbox = dnbox;
    b->bd.tile_boxes = dtboxes;
    b->bd.nsims = n;
    b->bd.nparts = nparts;
    b->bd.total_tiles = tile0;
    b->bd.near_part = dnpart;
    b->bd.near_tile0 = dntile0;
    b->bd.total_near_tiles = near_tiles;
    // variant 1 (256 threads, 64-register cap) is the fastest untuned choice
    // on every measured workload; FP64 storage runs variant 0 regardless
    b->bd.lat_variant = 1;
    // particle CTA width: 256 threads when every particle fits and there are
    // enough particles that the SMs their CTAs hold matter to the bulk pass
    // (the narrow CTA holds a quarter of an SM's registers, a little longer)
    {
        int max_nl = 0;
        for (int i = 0; i < n; ++i)
            for (auto &p : sims[i]->parts) max_nl = std::max(max_nl, p.nl);
        // (the solved spreading scales keep their factorisation window in
        // registers: 512-thread CTAs, which have twice the registers)
        bool vb = false;
        for (int i = 0; i < n; ++i) vb |= sims[i]->cfg.ib_spread != 0;
        b->bd.pthreads = (b->kind != ST_F64 && max_nl <= 256 && nparts >= 32 && !vb) ? 256 : 512;
    }
    // copy-engine staging (variants 4, 5): rows of whole 16-byte words,
    // walls that are not periodic, 4- or 2-byte storage
    int tma_ok = b->kind != ST_F64;
    for (int i = 0; i < n; ++i) {
        const int per16 = 16 / (int)storage_size(b->kind);
        if (!hs[i].vec4 || hs[i].nx % per16 != 0 || hs[i].wall_b == LBIB_WALL_PERIODIC || hs[i].aa)
            tma_ok = 0;
    }
    b->bd.tma_ok = tma_ok;
    b->bd.any_aa = 0;
    for (int i = 0; i < n; ++i) b->bd.any_aa |= hs[i].aa;
    b->bd.wait_polls = wait_polls_setting();
    if (tma_ok && (e = lattice_kernel_setup(b->kind)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "lattice kernel setup");
    }
    b->d_curs = dcurs;
    b->overlap = nparts > 0 && boxes_fit;
    // The next bulk pass's CTAs start during this one's tail and wait there
    // for it: a gain where the bulk pass bounds the step (many particles, or
    // much lattice per particle: C3 88.8 -> 87.6 us, C4 49.2 -> 48.5 us per
    // step), a loss where the particle pass's chain does (six 1024 x 256
    // channels with one particle each: 28.8 -> 29.6 us), since the waiting
    // CTAs hold SMs that chain could use.
    {
        long long nodes = 0;
        for (lbib_sim *s : b->sims) nodes += s->N;
        b->bulk_pdl = b->overlap && (nparts >= 32 || nodes >= 400000LL * nparts);
    }
    if (b->overlap) {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if ((e = cudaStreamCreateWithPriority(&b->s1, cudaStreamNonBlocking, greatest)) ||
            (e = cudaStreamCreateWithPriority(&b->s2, cudaStreamNonBlocking, least)) ||
            (e = cudaEventCreateWithFlags(&b->evjoin1, cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&b->evb[0], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&b->evb[1], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&b->evn[0], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&b->evn[1], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&b->evfork, cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&b->evjoin, cudaEventDisableTiming))) {
            free_batch(b);
            return cuda_fail(e, "batch streams");
        }
    }
    *out = b;
    return LBIB_OK;
}

// Waits for all work on a simulation's state: its own stream and the streams
// of the user batches that hold it (a batch steps its members on the first
// member's stream, which joins the batch's other streams at the end of every
// call).
lbib_status sync_sim(lbib_sim *s) {
    CK(cudaStreamSynchronize(s->stream));
    for (lbib_batch *b : s->batches)
        if (!b->orphan && b->stream != s->stream) CK(cudaStreamSynchronize(b->stream));
    return LBIB_OK;
}

lbib_status ensure_self(lbib_sim *s) {
    if (s->self) return LBIB_OK;
    lbib_sim *one[1] = {s};
    lbib_status r = make_batch(one, 1, &s->self);
    if (r == LBIB_OK) s->self->is_self = true;
    return r;
}

// Eq. 10 for every possible probing count n of a particle, for each wall:
// P_f = 1 - exp(-(k_f rho_r) n / nl), dt = 1.  Evaluated on the host once the
// receptors are final, so the device looks it up instead of computing exp.
lbib_status upload_pf_tables(lbib_sim *s) {
    for (auto &p : s->parts) {
        const int n = p.nl;
        std::vector<double> tab(2 * (size_t)(n + 1));
        for (int k = 0; k <= n; ++k) {
            const double Nl = (double)k / (double)n;
            tab[k] = 1.0 - exp(-(s->cfg.k_f * s->cfg.receptor_bottom) * Nl);
            tab[n + 1 + k] = 1.0 - exp(-(s->cfg.k_f * s->cfg.receptor_top) * Nl);
        }
        CK(cudaMemcpy(p.d_pftab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice));
    }
    return LBIB_OK;
}

// IB forcing of step 0 at the initial pose (the particle kernel in init mode).
lbib_status prime(lbib_sim *s, cudaStream_t st) {
    if (s->primed) return LBIB_OK;
    lbib_status r = ensure_self(s);
    if (r != LBIB_OK) return r;
    CK(cudaStreamSynchronize(st));
    r = upload_pf_tables(s);
    if (r != LBIB_OK) return r;
    if (!s->parts.empty()) {
        cudaError_t e = launch_particles(s->kind, s->self->bd, 0, 1, s->self->smem, st);
        if (e != cudaSuccess) return cuda_fail(e, "particle kernel (init)");
    }
    s->primed = true;
    return LBIB_OK;
}

// IB forcing recomputed at the particles' current poses from the current
// populations (the init-mode particle pass), after their state was changed
// from the host: what the end of a step leaves for the next one.
lbib_status reprime(lbib_sim *s) {
    s->primed = false;
    return prime(s, s->stream);
}

// Prime the members of a batch.  A fresh user batch (no member primed yet)
// takes one initial IB launch over all its particles instead of one launch
// and one private batch per simulation; otherwise each member is primed on
// its own.
lbib_status prime_members_once(lbib_batch *b) {
    bool none = true, all = true;
    for (lbib_sim *s : b->sims) {
        if (s->primed) none = false;
        else all = false;
    }
    if (all) return LBIB_OK;
    if (!none || b->is_self) {
        for (lbib_sim *s : b->sims) {
            lbib_status r = prime(s, b->stream);
            if (r != LBIB_OK) return r;
        }
        return LBIB_OK;
    }
    // the particles' uploads run on their simulations' streams
    CK(cudaStreamSynchronize(b->stream));
    for (lbib_sim *s : b->sims)
        if (s->stream != b->stream) CK(cudaStreamSynchronize(s->stream));
    for (lbib_sim *s : b->sims) {
        lbib_status r = upload_pf_tables(s);
        if (r != LBIB_OK) return r;
    }
    if (b->bd.nparts > 0) {
        cudaError_t e = launch_particles(b->kind, b->bd, 0, 1, b->smem, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "particle kernel (init)");
    }
    for (lbib_sim *s : b->sims) s->primed = true;
    return LBIB_OK;
}

// Before every batched call: prime the members, then copy their parity words
// and near boxes into the batch (what the members did on their own since the
// last call, restores included, is picked up here).
lbib_status prime_members(lbib_batch *b) {
    lbib_status r = prime_members_once(b);
    if (r != LBIB_OK) return r;
    cudaError_t e = launch_batch_refresh(b->bd, b->d_curs, b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch refresh");
    return LBIB_OK;
}

// Enqueue nsteps steps.  ev (or null) receives event records around the
// lattice / bulk pass [0, 1] of the middle step ks = nsteps / 2 (a step in
// the steady state of the two-stream schedule) and around the particle
// [2, 3] and near-box [4, 5] passes of the step after it (a record between
// two passes of the high-priority chain stops the later one from launching
// early, which would otherwise slow the sampled bulk pass).  capturing: the
// enqueue is being captured into a graph (the records become event-record
// nodes).
cudaError_t enqueue_steps(lbib_batch *b, int nsteps, cudaEvent_t *ev, bool capturing = true) {
    cudaError_t e = cudaSuccess;
    const unsigned fl = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    const int ks = nsteps / 2, kp = ks + 1 < nsteps ? ks + 1 : ks;
    auto mark = [&](int i, cudaStream_t st) {
        return (ev) ? cudaEventRecordWithFlags(ev[i], st, fl) : cudaSuccess;
    };
    if (!b->overlap) {
        for (int k = 0; k < nsteps; ++k) {
            const int f = k & 1;
            if (k == ks && (e = mark(0, b->stream))) return e;
            if ((e = launch_lattice(b->kind, b->bd, f, 0, b->stream))) return e;
            if (k == ks && (e = mark(1, b->stream))) return e;
            if (k == kp && (e = mark(2, b->stream))) return e;
            if ((e = launch_particles(b->kind, b->bd, f ^ 1, 2, b->smem, b->stream))) return e;
            if (k == kp && (e = mark(3, b->stream))) return e;
            if (ev && k == kp && ((e = mark(4, b->stream)) || (e = mark(5, b->stream)))) return e;
        }
        return e;
    }
    // Overlapped form.  Step k: bulk(k) on s2 after near(k-1); near(k) on the
    // main stream after bulk(k-1); then particle(k), which needs only near(k)
    // (its staged nodes lie in the near boxes).  bulk(k+1) therefore runs while
    // particle(k) runs.  The fork / join make the call ordered with all other
    // work on the main stream.
    if ((e = cudaEventRecord(b->evfork, b->stream)) ||
        (e = cudaStreamWaitEvent(b->s1, b->evfork, 0)) ||
        (e = cudaStreamWaitEvent(b->s2, b->evfork, 0)))
        return e;
    for (int k = 0; k < nsteps; ++k) {
        const int f = k & 1;
        if (k > 0 && (e = cudaStreamWaitEvent(b->s2, b->evn[(k - 1) & 1], 0))) return e;
        if (k == ks && (e = mark(0, b->s2))) return e;
        // programmatic dependent of the bulk pass of the step before (its
        // prologue overlaps that pass's tail; bulk-bound batches), unless an
        // event record sits between them
        if ((e = launch_lattice(b->kind, b->bd, f, 1, b->s2,
                                b->bulk_pdl && k > 0 && !(ev && (k == ks || k == ks + 1)))))
            return e;
        if (k == ks && (e = mark(1, b->s2))) return e;
        if ((e = cudaEventRecord(b->evb[k & 1], b->s2))) return e;
        if (k > 0 && (e = cudaStreamWaitEvent(b->s1, b->evb[(k - 1) & 1], 0))) return e;
        if (k == kp && (e = mark(4, b->s1))) return e;
        // programmatic dependent of the particle pass of the step before
        // (its CTAs are resident when that pass ends), unless an event record
        // sits between them
        if ((e = launch_lattice(b->kind, b->bd, f, 2, b->s1,
                                k > 0 && !(ev && (k == kp || k == kp + 1)))))
            return e;
        if (k == kp && (e = mark(5, b->s1))) return e;
        if ((e = cudaEventRecord(b->evn[k & 1], b->s1))) return e;
        if (k == kp && (e = mark(2, b->s1))) return e;
        // programmatic dependent of the near pass (its prologue overlaps it),
        // unless an event record sits between them
        if ((e = launch_particles(b->kind, b->bd, f ^ 1, 0, b->smem, b->s1, !(ev && k == kp)))) return e;
        if (k == kp && (e = mark(3, b->s1))) return e;
    }
    if ((e = cudaEventRecord(b->evjoin, b->s2)) || (e = cudaEventRecord(b->evjoin1, b->s1)) ||
        (e = cudaStreamWaitEvent(b->stream, b->evjoin, 0)) ||
        (e = cudaStreamWaitEvent(b->stream, b->evjoin1, 0)))
        return e;
    return e;
}

// Events per step of flushed stepping: flush start, step start, bulk-pass
// start and end, step end, near-pass start, particle-pass end.
constexpr int FEV = 7;

// Enqueue nsteps steps (inside a capture only), each after an L2 flush and
// bracketed by event records ev[FEV * k + ...]; ends with a parity flip when
// nsteps is odd.  The kernels are those of enqueue_steps; the L2 flush is a
// join point between steps.
cudaError_t enqueue_flushed_steps(lbib_batch *b, int nsteps, cudaEvent_t *ev) {
    const unsigned fl = cudaEventRecordExternal;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < nsteps; ++k) {
        const int f = k & 1;
        cudaEvent_t *E = ev + FEV * k;
        if ((e = cudaEventRecordWithFlags(E[0], b->stream, fl)) ||
            (e = launch_l2_flush(b->fbuf, b->fbytes, b->fclean, (unsigned)k, b->stream)) ||
            (e = cudaEventRecordWithFlags(E[1], b->stream, fl)))
            return e;
        if (!b->overlap) {
            if ((e = cudaEventRecordWithFlags(E[2], b->stream, fl)) ||
                (e = launch_lattice(b->kind, b->bd, f, 0, b->stream)) ||
                (e = cudaEventRecordWithFlags(E[3], b->stream, fl)) ||
                (e = cudaEventRecordWithFlags(E[5], b->stream, fl)) ||
                (e = launch_particles(b->kind, b->bd, f ^ 1, 2, b->smem, b->stream)) ||
                (e = cudaEventRecordWithFlags(E[6], b->stream, fl)))
                return e;
        } else {
            // near pass first; the particle pass follows it as a programmatic
            // dependent and the bulk pass is released when it ends, so that
            // the particle pass's CTAs are resident before the bulk pass
            // fills the SMs (as in the overlapped graph, where both wait on
            // the near pass)
            if ((e = cudaEventRecord(b->evfork, b->stream)) ||
                (e = cudaStreamWaitEvent(b->s1, b->evfork, 0)) ||
                (e = cudaStreamWaitEvent(b->s2, b->evfork, 0)) ||
                (e = cudaEventRecordWithFlags(E[5], b->s1, fl)) ||
                (e = launch_lattice(b->kind, b->bd, f, 2, b->s1)) ||
                (e = cudaEventRecord(b->evn[0], b->s1)) ||
                (e = launch_particles(b->kind, b->bd, f ^ 1, 0, b->smem, b->s1, true)) ||
                (e = cudaEventRecordWithFlags(E[6], b->s1, fl)) ||
                (e = cudaEventRecord(b->evjoin1, b->s1)) ||
                (e = cudaStreamWaitEvent(b->s2, b->evn[0], 0)) ||
                (e = cudaEventRecordWithFlags(E[2], b->s2, fl)) ||
                (e = launch_lattice(b->kind, b->bd, f, 1, b->s2)) ||
                (e = cudaEventRecordWithFlags(E[3], b->s2, fl)) ||
                (e = cudaEventRecord(b->evjoin, b->s2)) ||
                (e = cudaStreamWaitEvent(b->stream, b->evjoin, 0)) ||
                (e = cudaStreamWaitEvent(b->stream, b->evjoin1, 0)))
                return e;
        }
        if ((e = cudaEventRecordWithFlags(E[4], b->stream, fl))) return e;
    }
    if (nsteps & 1) e = launch_flip(b->d_curs, b->bd.par, (int)b->sims.size(), b->stream);
    return e;
}

// Graphs are captured with the batch's streams idle: a 4-step graph captured
// while a graph launched just before was still running replayed with results
// that differed from run to run (measured: 15-30 of 30 repeats of a batch and
// its solo runs; none with the wait, none over 20 repeats each at 8 and 16
// steps, none before the 4-step graphs existed).  Captures happen once per
// graph kind and launch configuration, so the wait costs nothing in steady
// state.
template <class Enqueue>
lbib_status capture_with(lbib_batch *b, Enqueue &&enqueue, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue();
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "graph capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    // per-node priorities keep the particle pass ahead of the bulk pass
    e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    return LBIB_OK;
}

lbib_status capture(lbib_batch *b, cudaEvent_t *ev, cudaGraphExec_t *out) {
    return capture_with(b, [&] { return enqueue_steps(b, GRAPH_STEPS, ev); }, out);
}

lbib_status batch_step_impl(lbib_batch *b, int64_t n) {
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    if (n < 0) return fail(LBIB_E_ARG, "nsteps must be >= 0");
    if (n == 0) return LBIB_OK;
    {
        lbib_status r = prime_members(b);
        if (r != LBIB_OK) return r;
    }
    const int64_t full = n / GRAPH_STEPS;
    const int rem = (int)(n % GRAPH_STEPS);
    if (full > 0 && !b->graph) {
        lbib_status r = capture(b, nullptr, &b->graph);
        if (r != LBIB_OK) return r;
    }
    for (int64_t i = 0; i < full; ++i) {
        cudaGraphExec_t g = b->graph;
        if (b->nsamples > 0) {
            // sampled replays carry event records around their first step
            const int slot = b->next_slot;
            b->next_slot = (slot + 1) % b->nsamples;
            g = b->tgraphs[slot];
            b->replayed[slot] = 1;
        }
        CK(cudaGraphLaunch(g, b->stream));
    }
    // the remainder: graphs of SHORT_STEPS steps (captured on first use and
    // kept), then the last few steps launched directly
    const int nshort = rem / SHORT_STEPS, tail = rem % SHORT_STEPS;
    if (nshort > 0 && !b->graph_short) {
        lbib_status r = capture_with(b, [&] { return enqueue_steps(b, SHORT_STEPS, nullptr); },
                                     &b->graph_short);
        if (r != LBIB_OK) return r;
    }
    for (int i = 0; i < nshort; ++i) CK(cudaGraphLaunch(b->graph_short, b->stream));
    if (tail > 0) {
        // with timing on, the middle direct step is sampled too (the next
        // slot's events)
        cudaEvent_t *ev = nullptr;
        if (b->nsamples > 0) {
            const int slot = b->next_slot;
            b->next_slot = (slot + 1) % b->nsamples;
            ev = &b->ev[6 * slot];
            b->replayed[slot] = 1;
        }
        cudaError_t e = enqueue_steps(b, tail, ev, false);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        if (tail & 1) {
            e = launch_flip(b->d_curs, b->bd.par, (int)b->sims.size(), b->stream);
            if (e != cudaSuccess) return cuda_fail(e, "parity flip");
        }
    }
    for (lbib_sim *s : b->sims) {
        s->step += n;
        s->cur ^= (int)(n & 1);
    }
    return LBIB_OK;
}

lbib_status ensure_scratch(lbib_sim *s, size_t bytes) {
    if (s->scratch_bytes >= bytes) return LBIB_OK;
    dfree(s->cfg, s->stream, s->d_scratch);
    s->d_scratch = (double *)dalloc(s->cfg, s->stream, bytes);
    s->scratch_bytes = s->d_scratch ? bytes : 0;
    if (!s->d_scratch) return fail(LBIB_E_OOM, "device scratch of %zu bytes", bytes);
    return LBIB_OK;
}

}  // namespace

extern "C" {

const char *lbib_last_error(void) { return g_err.c_str(); }

const char *lbib_version(void) {
#ifdef LBIB_DEBUG
    return "lbib 0.2 sm_103a (D2Q9 LB-IB-MLS, Philox4x64-10) debug: bounds-checked";
#else
    return "lbib 0.2 sm_103a (D2Q9 LB-IB-MLS, Philox4x64-10)";
#endif
}

lbib_status lbib_create(const lbib_config *cfg, lbib_sim **out) {
    if (!cfg || !out) return fail(LBIB_E_ARG, "null argument");
    *out = nullptr;
    const lbib_config &c = *cfg;
    if (c.nx < 8 || c.ny < 4 || (int64_t)c.nx * c.ny >= (1ll << 31) / 9)
        return fail(LBIB_E_ARG, "lattice %d x %d outside 8 x 4 .. 2^31/9 nodes", c.nx, c.ny);
    if (c.ib_iterations < 0 || c.ib_iterations > 16)
        return fail(LBIB_E_ARG, "ib_iterations %d outside 0 .. 16", c.ib_iterations);
    if (!(c.tau > 0.5) || !isfinite(c.tau)) return fail(LBIB_E_ARG, "tau must be > 1/2");
    for (int w : {c.wall_bottom, c.wall_top})
        if (w < 0 || w > 2) return fail(LBIB_E_ARG, "unknown wall kind %d", w);
    if ((c.wall_bottom == LBIB_WALL_PERIODIC) != (c.wall_top == LBIB_WALL_PERIODIC))
        return fail(LBIB_E_ARG, "periodic walls must be set on both sides");
    if (c.storage < 0 || c.storage > 3) return fail(LBIB_E_ARG, "unknown storage %d", c.storage);
    if (c.rounding != LBIB_ROUND_NEAREST && c.rounding != LBIB_ROUND_STOCHASTIC)
        return fail(LBIB_E_ARG, "unknown rounding %d", c.rounding);
    if (c.ib_spread != 0 && c.ib_spread != 1)
        return fail(LBIB_E_ARG, "ib_spread must be 0 or 1");
    if (c.stream_mode != 0 && c.stream_mode != 1)
        return fail(LBIB_E_ARG, "stream_mode must be 0 (A/B) or 1 (in place)");
    if (!(c.kBT > 0) || c.k_f < 0 || c.k_r0 < 0 || c.y_cr < 0 || c.eps_min <= 0 ||
        c.receptor_bottom < 0 || c.receptor_top < 0)
        return fail(LBIB_E_ARG, "bond / wall-force parameters out of range");
    lbib_sim *s = new (std::nothrow) lbib_sim();
    if (!s) return fail(LBIB_E_OOM, "host allocation failed");
    s->cfg = c;
    s->kind = c.storage;
    s->N = (size_t)c.nx * c.ny;
    cudaGetDevice(&s->device);
    if (c.cuda_stream) {
        s->stream = (cudaStream_t)c.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return cuda_fail(cudaGetLastError(), "cudaStreamCreate");
        }
        s->own_stream = true;
    }
    if (s->kind == ST_F16) {
        double sc = c.f16_scale;
        if (sc <= 0) {
            // keep |f - w| of a flow with speeds up to u_ref well inside the
            // normal range: scale ~ 2^floor(log2(64 / u_ref))
            const double uref = std::max({fabs(c.u_top), fabs(c.u_bottom),
                                          1e3 * std::max(fabs(c.gx), fabs(c.gy)), 1e-6});
            sc = exp2(floor(log2(64.0 / uref)));
            sc = std::min(sc, 1.0 * (1 << 24));
        }
        s->scale = (float)sc;
    }
    const size_t pb = 9 * s->N * storage_size(s->kind);
    s->pop[0] = dalloc(c, s->stream, pb);
    // in-place streaming: one buffer for both parities
    s->pop[1] = c.stream_mode == 1 ? s->pop[0] : dalloc(c, s->stream, pb);
    s->d_small = dalloc(c, s->stream, 64);
    if (!s->pop[0] || !s->pop[1] || !s->d_small) {
        lbib_destroy(s);
        return fail(LBIB_E_OOM, "device allocation of 2 x %zu bytes failed", pb);
    }
    s->d_step = (long long *)s->d_small;
    s->d_cur = (int *)((char *)s->d_small + 8);
    s->d_err = (int *)((char *)s->d_small + 12);
    cudaError_t e;
    if ((e = cudaMemsetAsync(s->d_small, 0, 64, s->stream)) ||
        (e = cudaMemsetAsync(s->pop[0], 0, pb, s->stream)) ||
        (e = cudaMemsetAsync(s->pop[1], 0, pb, s->stream)) ||
        (e = cudaStreamSynchronize(s->stream))) {
        lbib_destroy(s);
        return cuda_fail(e, "initialisation");
    }
    *out = s;
    return LBIB_OK;
}

lbib_status lbib_destroy(lbib_sim *s) {
    if (!s) return LBIB_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    // batches holding this simulation become orphans: they keep their own
    // memory (freed by lbib_batch_destroy) and refuse to step
    std::vector<lbib_batch *> held = s->batches;
    for (lbib_batch *b : held) {
        cudaStreamSynchronize(b->stream);
        unregister(b);
        b->orphan = true;
    }
    free_batch(s->self);
    for (auto &p : s->parts) dfree(s->cfg, s->stream, p.d_block);
    dfree(s->cfg, s->stream, s->pop[0]);
    if (s->pop[1] != s->pop[0]) dfree(s->cfg, s->stream, s->pop[1]);
    dfree(s->cfg, s->stream, s->d_small);
    dfree(s->cfg, s->stream, s->d_scratch);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return LBIB_OK;
}

lbib_status lbib_add_particle(lbib_sim *s, const lbib_particle *in, int32_t *pid) {
    if (!s || !in) return fail(LBIB_E_ARG, "null argument");
    {
        lbib_status r0 = reopen_setup(s, "lbib_add_particle");
        if (r0 != LBIB_OK) return r0;
    }
    if ((int)s->parts.size() >= LBIB_MAX_PARTICLES_PER_SIM)
        return fail(LBIB_E_ARG, "at most %d particles per simulation", LBIB_MAX_PARTICLES_PER_SIM);
    HostParticle p;
    if (in->vx && in->vy) {
        if (in->n_vertices < 3 || in->n_vertices > LBIB_MAX_MARKERS)
            return fail(LBIB_E_ARG, "n_vertices %d outside 3..%d", in->n_vertices, LBIB_MAX_MARKERS);
        p.vx.assign(in->vx, in->vx + in->n_vertices);
        p.vy.assign(in->vy, in->vy + in->n_vertices);
    } else {
        if (!(in->a > 0) || (in->shape == 1 && !(in->b > 0)) || in->shape < 0 || in->shape > 1)
            return fail(LBIB_E_ARG, "shape needs positive semi-axes");
        const double a = in->a, b = in->shape == 1 ? in->b : in->a;
        const double h = ((a - b) / (a + b)) * ((a - b) / (a + b));
        const double per = M_PI * (a + b) * (1 + 3 * h / (10 + sqrt(4 - 3 * h)));
        const int n = in->n_vertices > 0 ? in->n_vertices : std::max(8, (int)lround(per));
        if (n < 3 || n > LBIB_MAX_MARKERS) return fail(LBIB_E_ARG, "marker count %d", n);
        ellipse_outline(a, b, n, p.vx, p.vy);
    }
    for (size_t i = 0; i < p.vx.size(); ++i)
        if (!isfinite(p.vx[i]) || !isfinite(p.vy[i])) return fail(LBIB_E_ARG, "non-finite vertex");
    if (!(in->rho_p > 0) || in->ligand_density < 0 || in->ligand_density > 1 || in->sigma < 0 ||
        !isfinite(in->xc) || !isfinite(in->yc) || !isfinite(in->theta))
        return fail(LBIB_E_ARG, "particle parameters out of range");
    p.fixed = in->fixed != 0;
    p.xc = in->xc; p.yc = in->yc; p.th = in->theta;
    p.rho_p = in->rho_p; p.lig = in->ligand_density; p.sigma = in->sigma;
    build_geometry(p);
    if (!(p.area > 0)) return fail(LBIB_E_ARG, "outline must be counter-clockwise with positive area");
    if (p.rmax > LBIB_MAX_PARTICLE_RADIUS)
        return fail(LBIB_E_ARG, "particle radius %.2f above %.1f", p.rmax, LBIB_MAX_PARTICLE_RADIUS);
    if (p.T >= s->cfg.nx) return fail(LBIB_E_ARG, "force tile %d not narrower than the lattice", p.T);
    if (s->cfg.wall_bottom == LBIB_WALL_PERIODIC && p.T >= s->cfg.ny)
        return fail(LBIB_E_ARG, "force tile %d not lower than the periodic lattice", p.T);
    for (size_t l = 0; l < p.S.size(); ++l)
        if (!(p.S[l] > 0)) return fail(LBIB_E_ARG, "degenerate element %zu", l);
    const bool vb = s->cfg.ib_spread != 0;
    if (vb) {
        p.vb_p = vb_band(p.mbx.data(), p.mby.data(), p.nl);
        if (p.vb_p < 0)
            return fail(LBIB_E_ARG, "markers closer than 4 sqrt 2 lie more than %d elements apart "
                        "along the outline: too thin for the solved spreading scales",
                        LBIB_VB_MAX_BAND);
    }
    if (particle_smem_bytes(s->kind, p.T, p.nl, vb) > SMEM_LIMIT)
        return fail(LBIB_E_ARG, "particle needs more on-chip memory than one SM has");
    {
        const int lim = particle_smem_limit(s->kind);
        if (lim > 0 && particle_smem_bytes(s->kind, p.T, p.nl, vb) > lim)
            return fail(LBIB_E_ARG, "particle needs %d bytes of shared memory (limit %d)",
                        particle_smem_bytes(s->kind, p.T, p.nl, vb), lim);
    }
    lbib_status r = upload_particle(s, p);
    if (r != LBIB_OK) return r;
    s->parts.push_back(std::move(p));
    if (pid) *pid = (int32_t)s->parts.size() - 1;
    return LBIB_OK;
}

lbib_status lbib_set_receptors(lbib_sim *s, int32_t wall, double density) {
    if (!s) return fail(LBIB_E_ARG, "null simulation");
    if (wall < 0 || wall > 1 || !(density >= 0) || !isfinite(density))
        return fail(LBIB_E_ARG, "wall must be 0 or 1 and density >= 0");
    {
        lbib_status r0 = reopen_setup(s, "lbib_set_receptors");
        if (r0 != LBIB_OK) return r0;
    }
    (wall == 0 ? s->cfg.receptor_bottom : s->cfg.receptor_top) = density;
    return LBIB_OK;
}

lbib_status lbib_set_populations(lbib_sim *s, const double *f) {
    if (!s || !f) return fail(LBIB_E_ARG, "null argument");
    lbib_status r = reopen_setup(s, "lbib_set_populations");
    if (r != LBIB_OK) return r;
    // Page-locked host memory the device can address (cudaHostAlloc, a
    // registered range) is read by the import kernel in place; any other
    // source is copied into a device scratch first.  Either way the call
    // returns after the import, so the caller may reuse f at once.
    const double *src = nullptr;
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, f) == cudaSuccess) {
        if (pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr)
            src = (const double *)pa.devicePointer;
    } else {
        (void)cudaGetLastError();   // an unknown pointer: not an error of this call
    }
    if (!src) {
        r = ensure_scratch(s, 9 * s->N * sizeof(double));
        if (r != LBIB_OK) return r;
        CK(cudaMemcpyAsync(s->d_scratch, f, 9 * s->N * sizeof(double), cudaMemcpyHostToDevice,
                           s->stream));
        src = s->d_scratch;
    }
    SimDev d = make_simdev(s, 0, 0);
    CK(launch_set_populations(s->kind, d, src, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBIB_OK;
}

lbib_status lbib_step(lbib_sim *s, int64_t n) {
    NvtxRange nv("lbib_step");
    if (!s) return fail(LBIB_E_ARG, "null simulation");
    lbib_status r = ensure_self(s);
    if (r != LBIB_OK) return r;
    return batch_step_impl(s->self, n);
}

lbib_status lbib_batch_create(lbib_sim *const *sims, int32_t n, lbib_batch **out) {
    lbib_status r = make_batch(sims, n, out);
    if (r != LBIB_OK) return r;
    for (lbib_sim *s : (*out)->sims) s->batches.push_back(*out);
    return LBIB_OK;
}

lbib_status lbib_batch_step(lbib_batch *b, int64_t n) {
    NvtxRange nv("lbib_batch_step");
    if (!b) return fail(LBIB_E_ARG, "null batch");
    return batch_step_impl(b, n);
}

lbib_status lbib_batch_destroy(lbib_batch *b) {
    if (b && !b->orphan) cudaStreamSynchronize(b->stream);
    free_batch(b);
    return LBIB_OK;
}

lbib_status lbib_batch_set_timing(lbib_batch *b, int32_t nsamples) {
    if (!b || nsamples < 0 || nsamples > 64) return fail(LBIB_E_ARG, "nsamples must be 0..64");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    CK(cudaStreamSynchronize(b->stream));
    for (auto g : b->tgraphs)
        if (g) cudaGraphExecDestroy(g);
    for (auto e : b->ev) cudaEventDestroy(e);
    b->tgraphs.assign(nsamples, nullptr);
    b->ev.assign(6 * nsamples, nullptr);
    b->replayed.assign(nsamples, 0);
    b->next_slot = 0;
    b->nsamples = nsamples;
    for (auto &e : b->ev) CK(cudaEventCreate(&e));
    // capture every sampled graph now, so that timed stepping does no capture
    for (int s = 0; s < nsamples; ++s) {
        lbib_status r = capture(b, &b->ev[6 * s], &b->tgraphs[s]);
        if (r != LBIB_OK) return r;
    }
    return LBIB_OK;
}

lbib_status lbib_batch_kernel_times(lbib_batch *b, double *mean_ms, int64_t *count) {
    if (!b || !mean_ms || !count) return fail(LBIB_E_ARG, "null argument");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    CK(cudaStreamSynchronize(b->stream));
    double sum[3] = {0, 0, 0};
    int64_t cnt[3] = {0, 0, 0};
    for (int s = 0; s < b->nsamples; ++s) {
        if (!b->replayed[s]) continue;
        for (int k = 0; k < 3; ++k) {
            if (k == 2 && !b->overlap) continue;
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, b->ev[6 * s + 2 * k], b->ev[6 * s + 2 * k + 1]));
            sum[k] += ms;
            cnt[k]++;
        }
        b->replayed[s] = 0;
    }
    for (int k = 0; k < 3; ++k) {
        mean_ms[k] = cnt[k] ? sum[k] / cnt[k] : 0.0;
        count[k] = cnt[k];
    }
    return LBIB_OK;
}

lbib_status lbib_batch_step_flushed(lbib_batch *b, int64_t n, void *flush, size_t flush_bytes,
                                    int32_t clean, double *ms) {
    if (!b) return fail(LBIB_E_ARG, "null batch");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    if (n < 0) return fail(LBIB_E_ARG, "nsteps must be >= 0");
    if (!flush || ((uintptr_t)flush & 15) || (flush_bytes & 15))
        return fail(LBIB_E_ARG, "flush buffer must be 16-byte aligned, a multiple of 16 bytes");
    if (clean != 0 && clean != 1) return fail(LBIB_E_ARG, "clean must be 0 or 1");
    int dev = 0, l2 = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    if (flush_bytes < (size_t)l2)
        return fail(LBIB_E_ARG, "flush buffer of %zu bytes is smaller than L2 (%d bytes)",
                    flush_bytes, l2);
    double acc[4] = {0, 0, 0, 0};
    if (ms) ms[0] = ms[1] = ms[2] = ms[3] = 0;
    if (n == 0) return LBIB_OK;
    {
        lbib_status r = prime_members(b);
        if (r != LBIB_OK) return r;
    }
    if (b->fev.empty()) {
        b->fev.assign(FEV * GRAPH_STEPS, nullptr);
        for (auto &e : b->fev) CK(cudaEventCreate(&e));
    }
    if (b->fgraph && (b->fbuf != flush || b->fbytes != flush_bytes || b->fclean != clean)) {
        CK(cudaStreamSynchronize(b->stream));
        cudaGraphExecDestroy(b->fgraph);
        b->fgraph = nullptr;
    }
    b->fbuf = flush;
    b->fbytes = flush_bytes;
    b->fclean = clean;
    for (int64_t done = 0; done < n;) {
        const int m = (int)std::min<int64_t>(n - done, GRAPH_STEPS);
        cudaGraphExec_t g = b->fgraph, tmp = nullptr;
        auto enq = [&] { return enqueue_flushed_steps(b, m, b->fev.data()); };
        lbib_status r = LBIB_OK;
        if (m < GRAPH_STEPS) r = capture_with(b, enq, &tmp), g = tmp;
        else if (!g) r = capture_with(b, enq, &b->fgraph), g = b->fgraph;
        if (r != LBIB_OK) return r;
        cudaError_t e = cudaGraphLaunch(g, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (tmp) cudaGraphExecDestroy(tmp);
        if (e != cudaSuccess) return cuda_fail(e, "flushed steps");
        for (lbib_sim *s : b->sims) {
            s->step += m;
            s->cur ^= m & 1;
        }
        for (int k = 0; k < m; ++k) {
            const cudaEvent_t *E = &b->fev[FEV * k];
            float t[4] = {0, 0, 0, 0};
            CK(cudaEventElapsedTime(&t[0], E[1], E[4]));
            CK(cudaEventElapsedTime(&t[1], E[2], E[3]));
            CK(cudaEventElapsedTime(&t[2], E[0], E[1]));
            CK(cudaEventElapsedTime(&t[3], E[5], E[6]));
            for (int j = 0; j < 4; ++j) acc[j] += t[j];
        }
        done += m;
    }
    if (ms)
        for (int j = 0; j < 4; ++j) ms[j] = acc[j];
    return LBIB_OK;
}

// Enqueue the gather of every member's particle record and error word and
// their copy into the pinned staging buffer, then record ev_rb.
static lbib_status readback_start(lbib_batch *b) {
    const int np = b->bd.nparts, ns = b->bd.nsims;
    const size_t pbytes = sizeof(ParticleDev) * (size_t)np, bytes = pbytes + sizeof(int) * ns;
    if (!b->d_rb) {
        b->d_rb = dalloc(b->acfg, b->stream, bytes);
        if (!b->d_rb) return fail(LBIB_E_OOM, "device allocation of %zu bytes failed", bytes);
        if (cudaHostAlloc(&b->h_rb, bytes, cudaHostAllocDefault) != cudaSuccess) {
            b->h_rb = nullptr;
            return fail(LBIB_E_OOM, "pinned host allocation of %zu bytes failed", bytes);
        }
        CK(cudaEventCreateWithFlags(&b->ev_rb, cudaEventDisableTiming));
    }
    {
        lbib_status r = prime_members(b);
        if (r != LBIB_OK) return r;
    }
    int *derr = (int *)((char *)b->d_rb + pbytes);
    gather_states_kernel<<<np + 1, 128, 0, b->stream>>>(b->bd.parts, np, b->bd.sims, ns,
                                                        (ParticleDev *)b->d_rb, derr);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(b->h_rb, b->d_rb, bytes, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaEventRecord(b->ev_rb, b->stream));
    b->rb_pending = true;
    return LBIB_OK;
}

lbib_status lbib_batch_synchronize(lbib_batch *b) {
    if (!b) return fail(LBIB_E_ARG, "null batch");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    const int ns = b->bd.nsims;
    if (!b->d_errs) {
        b->d_errs = (int *)dalloc(b->acfg, b->stream, sizeof(int) * ns);
        if (!b->d_errs) return fail(LBIB_E_OOM, "device allocation of %zu bytes failed", sizeof(int) * ns);
        if (cudaHostAlloc((void **)&b->h_errs, sizeof(int) * ns, cudaHostAllocDefault) != cudaSuccess) {
            b->h_errs = nullptr;
            return fail(LBIB_E_OOM, "pinned host allocation failed");
        }
    }
    // the error words of every member in one copy, after all enqueued work
    gather_states_kernel<<<1, 128, 0, b->stream>>>(b->bd.parts, 0, b->bd.sims, ns, nullptr,
                                                   b->d_errs);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(b->h_errs, b->d_errs, sizeof(int) * ns, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < ns; ++i) {
        lbib_status r = err_status(b->sims[i], b->h_errs[i]);
        if (r != LBIB_OK) return r;
    }
    return LBIB_OK;
}

lbib_status lbib_batch_read_particles_async(lbib_batch *b) {
    if (!b) return fail(LBIB_E_ARG, "null batch");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    if (b->rb_pending) return fail(LBIB_E_STATE, "a started readback has not been collected");
    return readback_start(b);
}

lbib_status lbib_batch_read_particles(lbib_batch *b, lbib_particle_state *out, int32_t cap,
                                     int32_t *count, size_t *d2h_bytes) {
    if (!b) return fail(LBIB_E_ARG, "null batch");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    if (cap < 0 || (cap > 0 && !out)) return fail(LBIB_E_ARG, "cap must be >= 0, out non-null");
    const int np = b->bd.nparts, ns = b->bd.nsims;
    if (count) *count = np;
    const size_t pbytes = sizeof(ParticleDev) * (size_t)np;
    if (d2h_bytes) *d2h_bytes = pbytes + sizeof(int) * ns;
    if (!b->rb_pending) {
        lbib_status r = readback_start(b);
        if (r != LBIB_OK) return r;
    }
    b->rb_pending = false;
    CK(cudaEventSynchronize(b->ev_rb));
    const ParticleDev *hp = (const ParticleDev *)b->h_rb;
    const int *herr = (const int *)((const char *)b->h_rb + pbytes);
    int k = 0;
    for (int i = 0; i < ns; ++i) {
        lbib_sim *s = b->sims[i];
        lbib_status r = err_status(s, herr[i]);
        if (r != LBIB_OK) return r;
        for (const HostParticle &p : s->parts) {
            if (k < cap) fill_state(out[k], hp[k], p);
            ++k;
        }
    }
    return LBIB_OK;
}

lbib_status lbib_batch_set_particle_threads(lbib_batch *b, int32_t threads) {
    if (!b) return fail(LBIB_E_ARG, "null batch");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    if (threads != 256 && threads != 512) return fail(LBIB_E_ARG, "threads must be 256 or 512");
    if (threads == 256) {
        if (b->kind == ST_F64) return fail(LBIB_E_ARG, "FP64 storage runs 512-thread particle CTAs");
        for (lbib_sim *s : b->sims) {
            if (s->cfg.ib_spread)
                return fail(LBIB_E_ARG, "solved spreading scales run 512-thread particle CTAs");
            for (auto &p : s->parts)
                if (p.nl > 256) return fail(LBIB_E_ARG, "a particle has %d elements (> 256)", p.nl);
        }
    }
    if (b->bd.pthreads == threads) return LBIB_OK;
    CK(cudaStreamSynchronize(b->stream));
    b->bd.pthreads = threads;
    // captured graphs hold the launch configuration
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->graph_short) cudaGraphExecDestroy(b->graph_short);
    b->graph_short = nullptr;
    if (b->fgraph) cudaGraphExecDestroy(b->fgraph);
    b->fgraph = nullptr;
    if (b->nsamples > 0) return lbib_batch_set_timing(b, b->nsamples);
    return LBIB_OK;
}

// Captured graphs hold the kernel variant; a change of variant drops them.
static lbib_status use_variant(lbib_batch *b, int variant) {
    if (b->bd.lat_variant == variant) return LBIB_OK;
    CK(cudaStreamSynchronize(b->stream));
    b->bd.lat_variant = variant;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->graph_short) cudaGraphExecDestroy(b->graph_short);
    b->graph_short = nullptr;
    if (b->fgraph) cudaGraphExecDestroy(b->fgraph);
    b->fgraph = nullptr;
    if (b->nsamples > 0) return lbib_batch_set_timing(b, b->nsamples);
    return LBIB_OK;
}

lbib_status lbib_batch_set_variant(lbib_batch *b, int32_t variant) {
    if (!b) return fail(LBIB_E_ARG, "null batch");
    if (variant < 0 || variant >= LBIB_LATTICE_VARIANTS)
        return fail(LBIB_E_ARG, "lattice variant %d outside 0..%d", variant,
                    LBIB_LATTICE_VARIANTS - 1);
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    return use_variant(b, variant);
}

lbib_status lbib_batch_autotune(lbib_batch *b, int32_t reps, int32_t *variant, double *ms) {
    if (!b || reps < 1 || reps > 1000) return fail(LBIB_E_ARG, "reps must be 1..1000");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    {
        lbib_status r = prime_members(b);
        if (r != LBIB_OK) return r;
    }
    const int mode = b->overlap ? 1 : 0;
    // in-place streaming has one buffer: a timing run would overwrite the
    // state, so there is nothing to time (the per-node form runs anyway)
    for (lbib_sim *s : b->sims)
        if (s->cfg.stream_mode == 1) {
            if (variant) *variant = b->bd.lat_variant;
            if (ms)
                for (int v = 0; v < LBIB_LATTICE_VARIANTS; ++v) ms[v] = 0.0;
            return LBIB_OK;
        }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    double best = 0.0;
    int pick = 0;
    const int saved = b->bd.lat_variant;
    for (int v = 0; v < LBIB_LATTICE_VARIANTS && e == cudaSuccess; ++v) {
        b->bd.lat_variant = v;
        // one untimed run, then reps timed dry runs of the lattice pass
        if ((e = launch_lattice(b->kind, b->bd, 2, mode, b->stream))) break;
        if ((e = cudaEventRecord(e0, b->stream))) break;
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = launch_lattice(b->kind, b->bd, 2, mode, b->stream);   // reads the current buffer only
        if (e || (e = cudaEventRecord(e1, b->stream)) || (e = cudaEventSynchronize(e1))) break;
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, e0, e1))) break;
        const double mean = t / reps;
        if (ms) ms[v] = mean;
        if (v == 0 || mean < best) {
            best = mean;
            pick = v;
        }
    }
    b->bd.lat_variant = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "lattice pass timing");
    if (variant) *variant = pick;
    return use_variant(b, pick);
}

lbib_status lbib_batch_pass_nodes(lbib_batch *b, int64_t *nodes) {
    if (!b || !nodes) return fail(LBIB_E_ARG, "null argument");
    if (b->orphan) return fail(LBIB_E_STATE, "a member of this batch was destroyed");
    CK(cudaStreamSynchronize(b->stream));
    int64_t bulk = 0, near = 0, total = 0;
    for (lbib_sim *s : b->sims) {
        const int nx = s->cfg.nx, ny = s->cfg.ny;
        const bool periodic = s->cfg.wall_bottom == LBIB_WALL_PERIODIC;
        total += (int64_t)nx * ny;
        if (!b->overlap) {
            bulk += (int64_t)nx * ny;
            continue;
        }
        int cur = 0;
        CK(cudaMemcpy(&cur, s->d_cur, sizeof(int), cudaMemcpyDeviceToHost));
        std::vector<uint8_t> in_box((size_t)nx * ny, 0);
        for (const HostParticle &hp : s->parts) {
            ParticleDev P;
            CK(cudaMemcpy(&P, hp.d_part, sizeof(P), cudaMemcpyDeviceToHost));
            for (int by = 0; by < P.NBy; ++by) {
                int y = P.box_oy[cur] + by;
                if (periodic) y = ((y % ny) + ny) % ny;
                if (y < 0 || y >= ny) continue;
                near += P.NBx;   // one row of the box, as the near pass does it
                for (int bx = 0; bx < P.NBx; ++bx) {
                    const int x = ((P.box_ox[cur] + bx) % nx + nx) % nx;
                    in_box[(size_t)y * nx + x] = 1;
                }
            }
        }
        for (uint8_t v : in_box) bulk += !v;
    }
    nodes[0] = bulk;
    nodes[1] = near;
    nodes[2] = total;
    return LBIB_OK;
}

lbib_status lbib_synchronize(lbib_sim *s) {
    if (!s) return fail(LBIB_E_ARG, "null simulation");
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    return check_err_word(s);
}

lbib_status lbib_read_state(lbib_sim *s, lbib_state *st, lbib_particle_state *parts,
                            int32_t n_parts, double *rho, double *ux, double *uy, size_t n_nodes) {
    NvtxRange nv("lbib_read_state");
    if (!s) return fail(LBIB_E_ARG, "null simulation");
    if ((rho || ux || uy) && n_nodes != s->N)
        return fail(LBIB_E_ARG, "field buffers hold %zu nodes, lattice has %zu", n_nodes, s->N);
    lbib_status r = LBIB_OK;
    if (rho || ux || uy) {
        r = prime(s, s->stream);   // the fields include the IB force of this step
        if (r == LBIB_OK) r = ensure_self(s);
        if (r != LBIB_OK) return r;
    }
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    r = check_err_word(s);
    if (r != LBIB_OK) return r;
    if (st) {
        st->step = s->step;
        st->n_particles = (int32_t)s->parts.size();
        st->storage = s->kind;
        st->nx = s->cfg.nx;
        st->ny = s->cfg.ny;
    }
    if (parts) {
        const int m = std::min<int>(n_parts, (int)s->parts.size());
        for (int k = 0; k < m; ++k) {
            ParticleDev h;
            CK(cudaMemcpy(&h, s->parts[k].d_part, sizeof h, cudaMemcpyDeviceToHost));
            fill_state(parts[k], h, s->parts[k]);
        }
    }
    if (rho || ux || uy) {
        r = ensure_scratch(s, 3 * s->N * sizeof(double));
        if (r != LBIB_OK) return r;
        SimDev d = make_simdev(s, 0, 0);
        double *dr = s->d_scratch, *du = dr + s->N, *dv = du + s->N;
        CK(launch_fields(s->kind, d, s->self->bd.parts, dr, du, dv, s->stream));
        if (rho) CK(cudaMemcpyAsync(rho, dr, s->N * 8, cudaMemcpyDeviceToHost, s->stream));
        if (ux) CK(cudaMemcpyAsync(ux, du, s->N * 8, cudaMemcpyDeviceToHost, s->stream));
        if (uy) CK(cudaMemcpyAsync(uy, dv, s->N * 8, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    }
    return LBIB_OK;
}

lbib_status lbib_read_populations(lbib_sim *s, double *f) {
    if (!s || !f) return fail(LBIB_E_ARG, "null argument");
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    lbib_status r = ensure_scratch(s, 9 * s->N * sizeof(double));
    if (r != LBIB_OK) return r;
    SimDev d = make_simdev(s, 0, 0);
    CK(launch_populations(s->kind, d, s->d_scratch, s->stream));
    CK(cudaMemcpyAsync(f, s->d_scratch, 9 * s->N * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return check_err_word(s);
}

lbib_status lbib_read_bonds(lbib_sim *s, int32_t pid, uint8_t *bond, double *ax, int32_t n) {
    if (!s) return fail(LBIB_E_ARG, "null simulation");
    if (pid < 0 || pid >= (int)s->parts.size()) return fail(LBIB_E_ARG, "no particle %d", pid);
    if (n != s->parts[pid].nl) return fail(LBIB_E_ARG, "particle %d has %d elements", pid, s->parts[pid].nl);
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    ParticleDev h;
    CK(cudaMemcpy(&h, s->parts[pid].d_part, sizeof h, cudaMemcpyDeviceToHost));
    if (bond) CK(cudaMemcpy(bond, h.bond, n, cudaMemcpyDeviceToHost));
    if (ax) CK(cudaMemcpy(ax, h.anchor_x, 8 * (size_t)n, cudaMemcpyDeviceToHost));
    return LBIB_OK;
}

lbib_status lbib_read_ib_force(lbib_sim *s, double *fx, double *fy) {
    if (!s || !fx || !fy) return fail(LBIB_E_ARG, "null argument");
    lbib_status r = sync_sim(s);
    if (r != LBIB_OK) return r;
    r = prime(s, s->stream);
    if (r == LBIB_OK) r = ensure_self(s);
    if (r != LBIB_OK) return r;
    r = ensure_scratch(s, 2 * s->N * sizeof(double));
    if (r != LBIB_OK) return r;
    SimDev d = make_simdev(s, 0, 0);
    CK(launch_ib_export(s->kind, d, s->self->bd.parts, s->d_scratch, s->d_scratch + s->N, s->stream));
    CK(cudaMemcpyAsync(fx, s->d_scratch, s->N * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(fy, s->d_scratch + s->N, s->N * 8, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return LBIB_OK;
}

lbib_status lbib_get_particle_record(lbib_sim *s, int32_t pid, lbib_particle_record *out) {
    if (!s || !out) return fail(LBIB_E_ARG, "null argument");
    if (pid < 0 || pid >= (int)s->parts.size()) return fail(LBIB_E_ARG, "no particle %d", pid);
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    ParticleDev h;
    CK(cudaMemcpy(&h, s->parts[pid].d_part, sizeof h, cudaMemcpyDeviceToHost));
    out->xc = h.xc; out->yc = h.yc; out->theta = h.th;
    out->u = h.u; out->v = h.v; out->omega = h.om;
    out->xc1 = h.xc1; out->yc1 = h.yc1; out->theta1 = h.th1;
    out->u1 = h.u1; out->v1 = h.v1; out->omega1 = h.om1;
    out->step = h.step;
    return check_err_word(s);
}

lbib_status lbib_set_particle_record(lbib_sim *s, int32_t pid, const lbib_particle_record *in) {
    NvtxRange nv("lbib_set_particle_record");
    if (!s || !in) return fail(LBIB_E_ARG, "null argument");
    if (pid < 0 || pid >= (int)s->parts.size()) return fail(LBIB_E_ARG, "no particle %d", pid);
    const double v[12] = {in->xc, in->yc, in->theta, in->u, in->v, in->omega,
                          in->xc1, in->yc1, in->theta1, in->u1, in->v1, in->omega1};
    for (double x : v)
        if (!isfinite(x)) return fail(LBIB_E_ARG, "non-finite particle record");
    if (in->step < 0) return fail(LBIB_E_ARG, "negative particle step count");
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    ParticleDev h;
    CK(cudaMemcpy(&h, s->parts[pid].d_part, sizeof h, cudaMemcpyDeviceToHost));
    h.xc = in->xc; h.yc = in->yc; h.th = in->theta;
    h.u = in->u; h.v = in->v; h.om = in->omega;
    h.xc1 = in->xc1; h.yc1 = in->yc1; h.th1 = in->theta1;
    h.u1 = in->u1; h.v1 = in->v1; h.om1 = in->omega1;
    h.step = in->step;
    h.pose_ok = 0;          // the next pass derives its pose from these values
    CK(cudaMemcpy(s->parts[pid].d_part, &h, sizeof h, cudaMemcpyHostToDevice));
    return reprime(s);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoints: the whole state a later step depends on, as one host blob.
// Layout: CkptHeader, the current post-collision populations in the storage
// format ([9][ny][nx] of f - w, times the F16 scale), then per particle a
// CkptParticle and its bond flags [nl], anchor x [nl] and anchor walls [nl],
// each section padded to 8 bytes.  The IB force of the coming step is not
// stored: loading recomputes it at the restored pose from the restored
// populations, as the end of the saved step did.
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
    char magic[8];
    uint32_t version, header_bytes;
    int32_t nx, ny, storage, n_particles;
    int64_t step;
    double scale;
    uint64_t pop_bytes;
    int32_t stream_mode, parity;     // in-place streaming: the state parity
};

struct CkptParticle {
    int32_t nl, n_probing, n_bonded, pad;
    double xc, yc, th, u, v, om, xc1, yc1, th1, u1, v1, om1;
    int64_t step;
    double Fh[2], Mh, Fb[2], Mb, Fw[2];
};

const char CKPT_MAGIC[8] = {'L', 'B', 'I', 'B', 'C', 'K', 'P', 'T'};
constexpr uint32_t CKPT_VERSION = 2;

size_t pad8(size_t b) { return (b + 7) & ~size_t(7); }

size_t ckpt_bytes(const lbib_sim *s) {
    size_t b = sizeof(CkptHeader) + pad8(9 * s->N * storage_size(s->kind));
    for (const HostParticle &p : s->parts)
        b += sizeof(CkptParticle) + pad8(p.nl) + 8 * (size_t)p.nl + pad8(p.nl);
    return b;
}

}  // namespace

extern "C" {

lbib_status lbib_checkpoint_size(lbib_sim *s, size_t *bytes) {
    if (!s || !bytes) return fail(LBIB_E_ARG, "null argument");
    *bytes = ckpt_bytes(s);
    return LBIB_OK;
}

lbib_status lbib_checkpoint_save(lbib_sim *s, void *host, size_t bytes) {
    NvtxRange nv("lbib_checkpoint_save");
    if (!s || !host) return fail(LBIB_E_ARG, "null argument");
    if (bytes < ckpt_bytes(s))
        return fail(LBIB_E_ARG, "checkpoint needs %zu bytes, buffer holds %zu", ckpt_bytes(s), bytes);
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    lbib_status r = check_err_word(s);
    if (r != LBIB_OK) return r;
    unsigned char *o = (unsigned char *)host;
    CkptHeader hd{};
    memcpy(hd.magic, CKPT_MAGIC, 8);
    hd.version = CKPT_VERSION;
    hd.header_bytes = sizeof(CkptHeader);
    hd.nx = s->cfg.nx; hd.ny = s->cfg.ny; hd.storage = s->kind;
    hd.n_particles = (int32_t)s->parts.size();
    hd.step = s->step;
    hd.scale = s->scale;
    hd.pop_bytes = 9 * s->N * storage_size(s->kind);
    hd.stream_mode = s->cfg.stream_mode;
    hd.parity = s->cur;
    memcpy(o, &hd, sizeof hd);
    o += sizeof hd;
    CK(cudaMemcpy(o, s->pop[s->cur], hd.pop_bytes, cudaMemcpyDeviceToHost));
    o += pad8(hd.pop_bytes);
    for (const HostParticle &p : s->parts) {
        ParticleDev h;
        CK(cudaMemcpy(&h, p.d_part, sizeof h, cudaMemcpyDeviceToHost));
        CkptParticle c{};
        c.nl = p.nl; c.n_probing = h.n_probing; c.n_bonded = h.n_bonded;
        c.xc = h.xc; c.yc = h.yc; c.th = h.th; c.u = h.u; c.v = h.v; c.om = h.om;
        c.xc1 = h.xc1; c.yc1 = h.yc1; c.th1 = h.th1; c.u1 = h.u1; c.v1 = h.v1; c.om1 = h.om1;
        c.step = h.step;
        c.Fh[0] = h.Fh[0]; c.Fh[1] = h.Fh[1]; c.Mh = h.Mh;
        c.Fb[0] = h.Fb[0]; c.Fb[1] = h.Fb[1]; c.Mb = h.Mb;
        c.Fw[0] = h.Fw[0]; c.Fw[1] = h.Fw[1];
        memcpy(o, &c, sizeof c);
        o += sizeof c;
        CK(cudaMemcpy(o, h.bond, p.nl, cudaMemcpyDeviceToHost));
        o += pad8(p.nl);
        CK(cudaMemcpy(o, h.anchor_x, 8 * (size_t)p.nl, cudaMemcpyDeviceToHost));
        o += 8 * (size_t)p.nl;
        CK(cudaMemcpy(o, h.anchor_wall, p.nl, cudaMemcpyDeviceToHost));
        o += pad8(p.nl);
    }
    return LBIB_OK;
}

lbib_status lbib_checkpoint_load(lbib_sim *s, const void *host, size_t bytes) {
    NvtxRange nv("lbib_checkpoint_load");
    if (!s || !host) return fail(LBIB_E_ARG, "null argument");
    if (bytes < sizeof(CkptHeader)) return fail(LBIB_E_ARG, "checkpoint too short");
    const unsigned char *o = (const unsigned char *)host;
    CkptHeader hd;
    memcpy(&hd, o, sizeof hd);
    if (memcmp(hd.magic, CKPT_MAGIC, 8) != 0 || hd.version != CKPT_VERSION ||
        hd.header_bytes != sizeof(CkptHeader))
        return fail(LBIB_E_ARG, "not an lbib checkpoint of version %u", CKPT_VERSION);
    if (hd.nx != s->cfg.nx || hd.ny != s->cfg.ny || hd.storage != s->kind ||
        hd.n_particles != (int32_t)s->parts.size() || hd.scale != (double)s->scale ||
        hd.pop_bytes != 9 * s->N * storage_size(s->kind) || hd.step < 0 ||
        hd.stream_mode != s->cfg.stream_mode || hd.parity < 0 || hd.parity > 1)
        return fail(LBIB_E_ARG, "checkpoint of a %d x %d lattice (storage %d, %d particles) does "
                    "not match this simulation", hd.nx, hd.ny, hd.storage, hd.n_particles);
    if (bytes < ckpt_bytes(s)) return fail(LBIB_E_ARG, "checkpoint truncated");
    {
        // every particle's element count before anything is written
        const unsigned char *q = o + sizeof hd + pad8(hd.pop_bytes);
        for (const HostParticle &p : s->parts) {
            CkptParticle c;
            memcpy(&c, q, sizeof c);
            if (c.nl != p.nl) return fail(LBIB_E_ARG, "checkpoint particle with %d elements, "
                                          "simulation's has %d", c.nl, p.nl);
            q += sizeof c + pad8(p.nl) + 8 * (size_t)p.nl + pad8(p.nl);
        }
    }
    {
        lbib_status r_ = sync_sim(s);
        if (r_ != LBIB_OK) return r_;
    }
    o += sizeof hd;
    if (s->cfg.stream_mode == 1) {
        // in place: the layout of the buffer depends on the state parity
        s->cur = hd.parity;
        CK(cudaMemcpy(s->d_cur, &hd.parity, sizeof(int), cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(s->pop[s->cur], o, hd.pop_bytes, cudaMemcpyHostToDevice));
    o += pad8(hd.pop_bytes);
    for (HostParticle &p : s->parts) {
        CkptParticle c;
        memcpy(&c, o, sizeof c);
        o += sizeof c;
        ParticleDev h;
        CK(cudaMemcpy(&h, p.d_part, sizeof h, cudaMemcpyDeviceToHost));
        h.xc = c.xc; h.yc = c.yc; h.th = c.th; h.u = c.u; h.v = c.v; h.om = c.om;
        h.xc1 = c.xc1; h.yc1 = c.yc1; h.th1 = c.th1; h.u1 = c.u1; h.v1 = c.v1; h.om1 = c.om1;
        h.step = c.step;
        h.Fh[0] = c.Fh[0]; h.Fh[1] = c.Fh[1]; h.Mh = c.Mh;
        h.Fb[0] = c.Fb[0]; h.Fb[1] = c.Fb[1]; h.Mb = c.Mb;
        h.Fw[0] = c.Fw[0]; h.Fw[1] = c.Fw[1];
        h.n_probing = c.n_probing; h.n_bonded = c.n_bonded;
        h.pose_ok = 0;
        CK(cudaMemcpy(p.d_part, &h, sizeof h, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h.bond, o, p.nl, cudaMemcpyHostToDevice));
        o += pad8(p.nl);
        CK(cudaMemcpy(h.anchor_x, o, 8 * (size_t)p.nl, cudaMemcpyHostToDevice));
        o += 8 * (size_t)p.nl;
        CK(cudaMemcpy(h.anchor_wall, o, p.nl, cudaMemcpyHostToDevice));
        o += pad8(p.nl);
    }
    const long long st = hd.step;
    const int zero = 0;
    CK(cudaMemcpy(s->d_step, &st, sizeof st, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->d_err, &zero, sizeof zero, cudaMemcpyHostToDevice));
    s->step = hd.step;
    return reprime(s);
}

lbib_status lbib_device_bytes(lbib_sim *s, size_t *bytes) {
    if (!s || !bytes) return fail(LBIB_E_ARG, "null argument");
    size_t b = (s->pop[1] == s->pop[0] ? 1 : 2) * 9 * s->N * storage_size(s->kind) + 64 +
               s->scratch_bytes;
    for (const HostParticle &p : s->parts) b += p.d_bytes;
    if (s->self) b += s->self->d_bytes;
    *bytes = b;
    return LBIB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free IB forcing.
//
// Some callers cannot allocate device memory: plugins and solvers embedded in
// a host application that owns every device allocation through its own arena
// (and forbids cudaMalloc / cudaFree behind its back), and real-time loops
// that must not touch an allocator, which may synchronise the device or fail
// under memory pressure, once they run.  lbib_ib_force_noalloc serves them:
// the caller passes its own device input and output buffers, and the only
// extra device memory the call touches is one file-scope static array of
// NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds until
// the process exits.  The call allocates no device or host heap memory, and
// copies nothing from the host: the descriptors and the particle's tables
// travel as the parameters of a set-up kernel that writes them into the
// array.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 256 * 1024;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch on each device, looked up once per
// device (with that device current) by the first call made on it.  In host
// code the array's name is only a host-side stand-in for the symbol.
std::once_flag g_noalloc_once[NOALLOC_MAX_DEVICES];
unsigned char *g_noalloc_addr[NOALLOC_MAX_DEVICES];
cudaError_t g_noalloc_lookup[NOALLOC_MAX_DEVICES];

lbib_status noalloc_scratch(int dev, unsigned char **out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(LBIB_E_UNSUPPORTED, "device %d beyond the %d the scratch table covers", dev,
                    NOALLOC_MAX_DEVICES);
    std::call_once(g_noalloc_once[dev], [dev] {
        void *p = nullptr;
        g_noalloc_lookup[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (g_noalloc_lookup[dev] == cudaSuccess) g_noalloc_addr[dev] = (unsigned char *)p;
    });
    if (g_noalloc_lookup[dev] != cudaSuccess || !g_noalloc_addr[dev])
        return cuda_fail(g_noalloc_lookup[dev], "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = g_noalloc_addr[dev];
    return LBIB_OK;
}

// Everything the IB pass reads besides the populations, passed by value to
// the set-up kernel (about 26 KB of kernel parameters): the channel and
// particle descriptors with their device pointers into the scratch, the
// batch tables of one particle, and the element geometry (body-frame
// centroids x, y, outward normals x, y, lengths), ligand flags and marker
// colouring of an explicit polygon.
struct NoAllocSetup {
    SimDev sim;
    ParticleDev par;
    SimDev *d_sim;
    ParticleDev *d_par;
    ParticleDev **d_parts;      // [2]: the particle, then a null end marker
    int *d_psim;                // [2]
    int *d_cur;
    double *d_geo;              // [5][nl]
    uint8_t *d_lig;
    int *d_corder, *d_coff;
    uint8_t *d_bond;
    double *d_ax;
    int8_t *d_aw;
    double *d_pft;              // [2][nl + 1]
    int nl, ncolors;
    double geo[5 * LBIB_MAX_MARKERS];
    uint8_t lig[LBIB_MAX_MARKERS];
    int corder[LBIB_MAX_MARKERS], coff[LBIB_MAX_MARKERS + 1];
};
static_assert(sizeof(NoAllocSetup) <= 32764, "set-up parameters exceed the kernel parameter limit");

// One CTA writes the descriptors and tables into the scratch and clears the
// state the IB pass does not read (bonds, anchors, P_f table), so nothing of
// an earlier call remains.
__global__ void __launch_bounds__(256) noalloc_setup_kernel(const __grid_constant__ NoAllocSetup a) {
    const int t = threadIdx.x, n = a.nl;
    if (t == 0) {
        *a.d_sim = a.sim;
        *a.d_par = a.par;
        a.d_parts[0] = a.d_par;
        a.d_parts[1] = nullptr;
        a.d_psim[0] = a.d_psim[1] = 0;
        *a.d_cur = 0;
    }
    for (int i = t; i < 5 * n; i += blockDim.x) a.d_geo[i] = a.geo[(i / n) * LBIB_MAX_MARKERS + i % n];
    for (int i = t; i < n; i += blockDim.x) {
        a.d_lig[i] = a.lig[i];
        a.d_corder[i] = a.corder[i];
        a.d_bond[i] = 0;
        a.d_ax[i] = 0.0;
        a.d_aw[i] = 0;
    }
    for (int i = t; i <= a.ncolors; i += blockDim.x) a.d_coff[i] = a.coff[i];
    for (int i = t; i < 2 * (n + 1); i += blockDim.x) a.d_pft[i] = 0.0;
}

// Element geometry, ligands and marker colouring of an explicit polygon (the
// construction of build_geometry, into the fixed-size tables of a).
void noalloc_geometry(const lbib_particle &in, NoAllocSetup &a, double &area, double &J,
                      double &rmax, int &n_ligands) {
    const int n = in.n_vertices;
    constexpr int M = LBIB_MAX_MARKERS;
    double *mbx = a.geo, *mby = a.geo + M, *nbx = a.geo + 2 * M, *nby = a.geo + 3 * M;
    double *S = a.geo + 4 * M;
    area = J = rmax = 0.0;
    for (int l = 0; l < n; ++l) {
        const int m = (l + 1) % n;
        const double ax = in.vx[l], ay = in.vy[l], bx = in.vx[m], by = in.vy[m];
        const double dx = bx - ax, dy = by - ay, len = sqrt(dx * dx + dy * dy);
        mbx[l] = 0.5 * (ax + bx);
        mby[l] = 0.5 * (ay + by);
        S[l] = len;
        nbx[l] = len > 0 ? dy / len : 0.0;
        nby[l] = len > 0 ? -dx / len : 0.0;
        const double cr = ax * by - bx * ay;
        area += 0.5 * cr;
        J += cr * (ax * ax + ax * bx + bx * bx + ay * ay + ay * by + by * by) / 12.0;
        rmax = std::max(rmax, sqrt(ax * ax + ay * ay));
    }
    n_ligands = 0;
    for (int l = 0; l < n; ++l) {
        a.lig[l] = floor((double)(l + 1) * in.ligand_density) > floor((double)l * in.ligand_density);
        n_ligands += a.lig[l];
    }
    int color[M];
    const int nc = color_markers(mbx, mby, n, color);
    a.ncolors = nc;
    for (int c = 0; c <= nc; ++c) a.coff[c] = 0;
    for (int l = 0; l < n; ++l) a.coff[color[l] + 1]++;
    for (int c = 0; c < nc; ++c) a.coff[c + 1] += a.coff[c];
    int fill[M + 1];
    for (int c = 0; c < nc; ++c) fill[c] = a.coff[c];
    for (int l = 0; l < n; ++l) a.corder[fill[color[l]]++] = l;
}

}  // namespace

extern "C" lbib_status lbib_ib_force_noalloc(const lbib_config *cfg, const float *f_dev,
                                             const lbib_particle *in, double u, double v,
                                             double omega, double *fx_dev, double *fy_dev) {
    NvtxRange nv("lbib_ib_force_noalloc");
    if (!cfg || !f_dev || !in || !fx_dev || !fy_dev) return fail(LBIB_E_ARG, "null argument");
    const lbib_config &c = *cfg;
    if (c.nx < 8 || c.ny < 4 || (int64_t)c.nx * c.ny >= (1ll << 31) / 9)
        return fail(LBIB_E_ARG, "lattice %d x %d outside 8 x 4 .. 2^31/9 nodes", c.nx, c.ny);
    if (c.ib_iterations < 0 || c.ib_iterations > 16)
        return fail(LBIB_E_ARG, "ib_iterations %d outside 0 .. 16", c.ib_iterations);
    if (c.ib_spread != 0 && c.ib_spread != 1) return fail(LBIB_E_ARG, "ib_spread must be 0 or 1");
    if (!(c.tau > 0.5) || c.wall_bottom < 0 || c.wall_bottom > 2 || c.wall_top < 0 || c.wall_top > 2 ||
        (c.wall_bottom == LBIB_WALL_PERIODIC) != (c.wall_top == LBIB_WALL_PERIODIC))
        return fail(LBIB_E_ARG, "invalid channel configuration");
    if (c.storage != LBIB_STORE_F32)
        return fail(LBIB_E_ARG, "lbib_ib_force_noalloc takes FP32 deviations f - w (storage F32)");
    if (!in->vx || !in->vy || in->n_vertices < 3 || in->n_vertices > LBIB_MAX_MARKERS)
        return fail(LBIB_E_ARG, "an explicit outline of 3..%d vertices is required", LBIB_MAX_MARKERS);
    for (int i = 0; i < in->n_vertices; ++i)
        if (!isfinite(in->vx[i]) || !isfinite(in->vy[i])) return fail(LBIB_E_ARG, "non-finite vertex");
    if (!isfinite(in->xc) || !isfinite(in->yc) || !isfinite(in->theta) || !isfinite(u) ||
        !isfinite(v) || !isfinite(omega) || !(in->rho_p > 0))
        return fail(LBIB_E_ARG, "particle parameters out of range");
    NoAllocSetup a{};                       // ~26 KB on the caller's stack
    double area = 0, J = 0, rmax = 0;
    int n_ligands = 0;
    noalloc_geometry(*in, a, area, J, rmax, n_ligands);
    if (!(area > 0)) return fail(LBIB_E_ARG, "outline must be counter-clockwise with positive area");
    const int nl = in->n_vertices, T = 2 * (int)ceil(rmax) + 8;
    if (T >= c.nx || (c.wall_bottom == LBIB_WALL_PERIODIC && T >= c.ny))
        return fail(LBIB_E_ARG, "force tile %d does not fit the lattice", T);
    // scratch layout: SimDev | ParticleDev | parts[2], part_sim[2] | cur | geometry | tile
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t o_sim = 0, o_par = o_sim + up(sizeof(SimDev)), o_tab = o_par + up(sizeof(ParticleDev));
    const size_t o_cur = o_tab + up(2 * sizeof(void *) + 2 * sizeof(int));
    const size_t o_geo = o_cur + up(sizeof(int));
    const size_t geo_bytes = up(5 * 8 * (size_t)nl) + up(nl) + up(4 * (size_t)nl) +
                             up(4 * (size_t)(a.ncolors + 1)) + up(nl) + up(8 * (size_t)nl) + up(nl) +
                             up(16 * (size_t)(nl + 1));
    const size_t o_tile = o_geo + geo_bytes;
    const size_t need = o_tile + 2 * sizeof(float) * (size_t)T * T;
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(LBIB_E_ARG, "particle needs %zu bytes of scratch; the static scratch holds %zu",
                    need, NOALLOC_SCRATCH_BYTES);
    const bool vb = c.ib_spread != 0;
    int vbp = 0;
    if (vb) {
        vbp = vb_band(a.geo, a.geo + LBIB_MAX_MARKERS, nl);
        if (vbp < 0) return fail(LBIB_E_ARG, "particle too thin for the solved spreading scales");
    }
    const int smem = particle_smem_bytes(ST_F32, T, nl, vb);
    const int lim = particle_smem_limit(ST_F32);
    if (lim <= 0 || smem > lim)
        return fail(LBIB_E_ARG, "particle needs %d bytes of shared memory (limit %d)", smem, lim);
    int dev = 0;
    CK(cudaGetDevice(&dev));
    unsigned char *base = nullptr;
    lbib_status r = noalloc_scratch(dev, &base);
    if (r != LBIB_OK) return r;
    cudaStream_t st = (cudaStream_t)c.cuda_stream;

    // device addresses inside the scratch
    a.d_sim = (SimDev *)(base + o_sim);
    a.d_par = (ParticleDev *)(base + o_par);
    a.d_parts = (ParticleDev **)(base + o_tab);
    a.d_psim = (int *)(base + o_tab + 2 * sizeof(void *));
    a.d_cur = (int *)(base + o_cur);
    unsigned char *gp = base + o_geo;
    size_t go = 0;
    auto take = [&](size_t b) {
        unsigned char *q = gp + go;
        go += up(b);
        return q;
    };
    a.d_geo = (double *)take(5 * 8 * (size_t)nl);
    a.d_lig = take(nl);
    a.d_corder = (int *)take(4 * (size_t)nl);
    a.d_coff = (int *)take(4 * (size_t)(a.ncolors + 1));
    a.d_bond = take(nl);
    a.d_ax = (double *)take(8 * (size_t)nl);
    a.d_aw = (int8_t *)take(nl);
    a.d_pft = (double *)take(16 * (size_t)(nl + 1));
    void *tile = base + o_tile;
    a.nl = nl;

    // descriptors: the channel over the caller's populations (one buffer,
    // current index 0), the particle at the given pose and velocity
    a.sim = simdev_from(c, (void *)f_dev, (void *)f_dev, a.d_cur, nullptr, nullptr, 1.f, 0, 1, 0);
    ParticleDev &hp = a.par;
    hp.xc = hp.xc1 = in->xc; hp.yc = hp.yc1 = in->yc; hp.th = hp.th1 = in->theta;
    hp.u = u; hp.v = v; hp.om = omega;
    hp.mass = in->rho_p * area; hp.inertia = in->rho_p * J;
    hp.inv_mass = 1.0 / hp.mass; hp.inv_inertia = 1.0 / hp.inertia;
    hp.r_eq = sqrt(area / M_PI); hp.sigma = in->sigma;
    hp.nl = nl; hp.n_ligands = n_ligands; hp.fixed = 1; hp.T = T; hp.ncolors = a.ncolors;
    hp.NBx = near_edge_x(T);
    hp.NBy = near_edge_y(T);
    hp.vb_p = vbp;
    hp.mbx = a.d_geo; hp.mby = a.d_geo + nl; hp.nbx = a.d_geo + 2 * nl; hp.nby = a.d_geo + 3 * nl;
    hp.S = a.d_geo + 4 * nl;
    hp.ligand = a.d_lig; hp.color_order = a.d_corder; hp.color_off = a.d_coff;
    hp.bond = a.d_bond; hp.anchor_x = a.d_ax; hp.anchor_wall = a.d_aw; hp.tile = tile;
    hp.pf_tab = a.d_pft;

    BatchDev bd{};
    bd.sims = a.d_sim;
    bd.parts = a.d_parts;
    bd.part_sim = a.d_psim;
    bd.nsims = 1;
    bd.nparts = 1;
    bd.wait_polls = 1 << 16;
    CK(particle_kernel_setup(ST_F32, lim));
    noalloc_setup_kernel<<<1, 256, 0, st>>>(a);
    CK(cudaGetLastError());
    // the IB pass at the given pose writes the whole force tile, then the
    // tile is laid out on the lattice (every node of fx, fy is written)
    CK(launch_particles(ST_F32, bd, 0, 1, smem, st));
    CK(launch_ib_export(ST_F32, a.sim, a.d_parts, fx_dev, fy_dev, st));
    return LBIB_OK;
}
