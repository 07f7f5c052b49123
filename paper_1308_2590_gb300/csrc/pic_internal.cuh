// Internal definitions of libpic: the handle, device buffers, small vector
// type, device helpers shared by the kernels, and host launch entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "pic.h"

namespace pic {

constexpr int NMOM = 13;          // rho, S (9, row-major), dj (3)

// Checks build (compiled with PIC_CHECKS): the kernels test their invariants
// (cell indices in range, offsets in [0, 1), destinations inside their bin,
// the shared-memory canary after the push's accumulator) and record a broken
// one in the sticky flags (FLAG_CHECK) instead of touching memory out of
// range.  In the normal build every check compiles away.
#ifdef PIC_CHECKS
constexpr bool kChecks = true;
#else
constexpr bool kChecks = false;
#endif
constexpr int32_t FLAG_CHECK = 32;
constexpr uint32_t CANARY = 0xC0DEC0DEu;
constexpr uint32_t KEY_DEAD = 0xFFFFFFFFu;

// Four-component vector (x, y, z, spare) stored 4*sizeof(T)-aligned so that
// a node's field is one vector load.
template <typename T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;
};

void set_error(const char *fmt, ...);

// --------------------------------------------------------------------------- handle

// Particles of one species live in tile bins made of 32-slot segments: bin t
// occupies slots [bstart[t], bstart[t+1]) of the "bins" buffer (multiples of
// SEG), uses its first useg[t] segments, and segment j holds segn[j] valid
// particles at its front.  The species' particle order is: tiles ascending,
// inside a tile its segments in order, inside a segment its valid prefix.
// Three buffer sets rotate roles: bins, mirror (the leavers of the current
// step, kept in the segment they left, at its front, count segml[j]) and spare
// (output of the per-step regroup or of a full rebuild; staging of a load).
constexpr int SEG = 32;

// FP64 form: quantities each deposit computes and the next push needs again.
// The push of step n+1 gathers the node B the moments of step n were made with,
// at the same position and with the same u, so its 1/gamma, b = q dt B /
// (2 m gamma) and 1/(1 + |b|^2) are exactly the deposit's.  They are kept per
// particle (planes of NCARRY values beside the state) instead of recomputed:
// on this GPU's FP64 pipe a B gather, a reciprocal square root and a
// reciprocal cost far more than reading and writing 40 bytes.
constexpr int NCARRY = 5;   // 1/gamma, bx, by, bz, 1/(1 + |b|^2)

struct SpeciesBuf {
    double q = 0, m = 1;
    int64_t cap = 0;   // slots per buffer set (multiple of SEG)
    int64_t n = 0;     // host copy of the live count (exact after a sync)
    bool n_exact = true;   // n is the live count (no step since it was read or set)
    int bins = 0, mir = 1, spare = 2;
    int32_t *cell[3] = {nullptr, nullptr, nullptr};
    void *ox[3] = {nullptr, nullptr, nullptr}, *oy[3] = {nullptr, nullptr, nullptr};
    void *ux[3] = {nullptr, nullptr, nullptr}, *uy[3] = {nullptr, nullptr, nullptr};
    void *uz[3] = {nullptr, nullptr, nullptr}, *w[3] = {nullptr, nullptr, nullptr};
    double *carry[3] = {nullptr, nullptr, nullptr};   // FP64 form: [NCARRY][cap] carried quantities per set
    uint32_t *mkey = nullptr;   // [cap] destination tile of each mirror entry
    int32_t *segn[2] = {nullptr, nullptr};  // [cap/SEG] valid particles per bin segment
    int32_t *useg[2] = {nullptr, nullptr};  // [ntiles] segments in use per bin
    int scur = 0;               // segn[scur], useg[scur] describe the bins; the regroup writes the other pair
    int32_t *segml = nullptr;   // [cap/SEG] leavers per mirror segment (this step)
    int32_t *bstart = nullptr;  // [ntiles + 1] slot offsets of the bins
    int32_t *tcount = nullptr;  // [ntiles + 1] scratch: particles per tile
    int32_t *cstart = nullptr;  // [ntiles + 1] scratch: compact starts
    int32_t *cend = nullptr;    // [ntiles + 1] scratch: run ends of a rebuild
};

struct Timing {
    bool enabled = false;
    double ms[4] = {0, 0, 0, 0};
    int64_t launches[5] = {0, 0, 0, 0, 0};
};

}  // namespace pic

struct pic_t {
    pic_config cfg;
    cudaStream_t st = nullptr;
    bool fp32 = false;
    size_t rs = 8;                      // sizeof(real)
    bool periodic_x = true;
    int nx = 0, ny = 0, nxn = 0;
    int64_t nnode = 0, ncell = 0;
    int G = 0, nxp = 0, nyp = 0;        // ghost width and padded node-array dims
    int64_t npad = 0;
    int tnx = 16, tny = 16, ntx = 0, nty = 0, ntiles = 0;

    // fields, all V4<real>
    void *E[2] = {nullptr, nullptr};    // nodes [nnode]; E[ecur] = E^n
    int ecur = 0;
    void *H[2] = {nullptr, nullptr};    // cells [ncell]; H[hcur] current, H[1-hcur] previous
    int hcur = 0;
    void *Ehalf = nullptr;              // padded nodes: E^{n+1/2} seen by the push
    void *B[2] = {nullptr, nullptr};    // padded nodes: B[bcur] = node B the moments were made with
    int bcur = 0;
    void *M = nullptr;                  // raw moment sums, planar [13][nnode] real

    // CN solver work (FP64 V4 vectors of nnode) and reduction scratch
    void *cn = nullptr;
    double *cn_red = nullptr;           // per-block partials
    int cn_red_cap = 0;
    double *cn_out = nullptr;           // [iterations, residual]

    // particles
    int nsp = 0;
    pic::SpeciesBuf sp[PIC_MAX_SPECIES];
    int64_t *d_removed = nullptr;       // [nsp] cumulative wall removals
    int32_t *d_flags = nullptr;         // sticky: bit 0 far mover seen, bit 2 capacity, bit 3 TMA wait timeout
    int32_t *d_step_flags = nullptr;    // [2], one per step parity: bit 0 far mover, bit 1 bin overflow -> full rebuild
    int32_t *h_step_flags = nullptr;    // pinned: [4 p] d_step_flags[p], [4 p + 1] d_flags after a step of parity p,
                                        // [2] d_flags after a load
    const int32_t *guard = nullptr;     // steps: the previous step's flags; its particle kernels do nothing if set
    void *h_diag = nullptr;             // pinned host copy of the diagnostics record
    cudaEvent_t ev_flags[2] = {nullptr, nullptr};   // per step parity: that step's flags are on the host
    bool flags_pending = false;         // a step's regroup flags are in flight (its regroup already committed)
    int pending_p = 0;                  // that step's parity
    int halo = 1;                       // deposit halo of a tile, in cells
    void *Mlo = nullptr;                // FP32 form: compensation of the moment sums
    bool det = false;                   // deterministic deposit: exact fixed-point sums in Mfix
    unsigned long long *Mfix = nullptr; // [13][nnode] two's-complement fixed-point moment sums
    double *Mc = nullptr;               // FP64 L2-reduction push (linear shape): cell sums [13][ncell][4]
    double wabs[PIC_MAX_SPECIES] = {0, 0, 0, 0, 0, 0, 0, 0};  // sum of |w| loaded per species
    void *tmaps = nullptr;              // host storage of the TMA descriptors
    int32_t *chunk_prefix = nullptr;    // [nsp*ntiles + 1] work items of the push, exclusive scan
    int2 *items = nullptr;              // work item k of the push -> (species-tile index, run within it)
    int64_t items_cap = 0;
    int32_t *ticket = nullptr;          // work-queue counter of the persistent push
    int32_t *nbr = nullptr;             // [ntiles][9] neighbour count, then the neighbour tiles ascending
    uint8_t *occ = nullptr;             // [ntiles] tiles holding particles when the last push started
    uint8_t *touched = nullptr;         // [ntiles] node tiles whose moments the last push may have written
    int32_t *touch_list = nullptr;      // [ntiles] the touched tiles, in no particular order
    int32_t *rg_list = nullptr;         // [ntiles] tiles the regroup must visit (an occupied tile or neighbour)
    int32_t *list_n = nullptr;          // [2 + PIC_MAX_SPECIES] entries of touch_list, rg_list; regroup queues
    int regroup_blocks = 0;             // blocks per species of the list-driven regroup
    bool touch_all = true;              // moments may be non-zero anywhere (after init or a deposit at rest)
    bool moments_cleared = false;       // the last literal field solve zeroed the moments it read
    unsigned long long *d_bad = nullptr;  // per species: first invalid particle index of a load
    uint32_t *scan_sums = nullptr;      // per-block totals of the multi-block scans
    bool moments_stale = false;         // particles or B changed since the last deposit at rest
    cudaEvent_t ev_batch = nullptr;     // a batched step: this run's prologue is queued
    cudaStream_t st2 = nullptr;         // loads: regroups of converted species, beside the next conversion
    cudaEvent_t ev_load = nullptr;      // loads: st2's work joined back to st
    cudaEvent_t ev_conv[PIC_MAX_SPECIES] = {};   // loads: a species' conversion is done (st -> st2)
    cudaStream_t st3 = nullptr;         // loads: the species' sorts, beside the previous species' deposit at rest
    cudaEvent_t ev_sorted[PIC_MAX_SPECIES] = {};   // loads: a species is sorted into its bins (st3 -> st2)
    cudaEvent_t ev_sorts = nullptr;     // loads: every sort is done (st3 -> st2)
    cudaEvent_t ev_push = nullptr;      // steps: the push (and its moments) is done (st -> st2)
    cudaEvent_t ev_field = nullptr;     // steps: the field solve is done (st2 -> st)
    cudaEvent_t ev_cellm = nullptr;     // steps: the push's cell sums are in the node moments (st2 -> st)
    int push_blocks = 0;                // persistent grid size of the push

    // sort scratch
    uint32_t *keys[2] = {nullptr, nullptr};   // sort scratch, 2*cap entries
    uint32_t *vals[2] = {nullptr, nullptr};
    uint32_t *hist = nullptr;
    int64_t sort_cap = 0, hist_cap = 0;

    // staging for load / readback (device FP64)
    double *stage = nullptr;
    int64_t stage_cap = 0;

    // prefetched loads (pic_prefetch_species): two slots of device copies, loaded in the order filled
    struct Prefetch {
        double *buf = nullptr;          // per species the six arrays, one after another
        int64_t cap = 0;                // doubles
        int nsp = 0;
        int64_t n[PIC_MAX_SPECIES] = {};
        cudaEvent_t copied = nullptr;   // the copy is complete (pf_st -> st)
        cudaEvent_t freed = nullptr;    // the load that read it is complete (st -> pf_st)
    } pf[2];
    int pf_head = 0, pf_count = 0;      // oldest filled slot, filled slots
    cudaStream_t pf_st = nullptr;       // the prefetch copies

    // field ionisation: staging of the ionised particles (checkpoint form) and of multi-source appends
    int32_t *ion_cell = nullptr;
    double *ion_val = nullptr;          // [6][ion_cap]
    int64_t ion_cap = 0;
    int32_t *ion_dcell = nullptr;
    double *ion_dval = nullptr;         // [6][ion_dcap]
    int64_t ion_dcap = 0;

    // diagnostics scratch
    double *d_diag = nullptr;           // partial sums
    int diag_cap = 0;

    int64_t step = 0;
    int64_t rebuilds = 0;               // full regroups run by the step fallback
    int shape = 1;                      // particle shape order: 1 (area weighting) or 2 (quadratic spline)
    int push_blocks_s2 = 0;             // grid of the order-2 push
    int cn_iters_last = 0;
    double cn_res_last = 0.0;
    pic::Timing timing;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace pic {

// --------------------------------------------------------------------------- kernels' argument blocks

template <typename R>
struct GridArgs {
    int nx, ny, nxn, G, nxp;
    int periodic_x;
    R dx, dy, dt;
    R inv_dx, inv_dy;
    R hx, hy;       // 1/(2 dx), 1/(2 dy): the centred differences of the curls
    R khx, khy;     // dt/(2 dx), dt/(2 dy)
    int64_t nnode;
};

template <typename R>
GridArgs<R> grid_args(const pic_t *h) {
    GridArgs<R> g;
    g.nx = h->nx; g.ny = h->ny; g.nxn = h->nxn; g.G = h->G; g.nxp = h->nxp;
    g.periodic_x = h->periodic_x ? 1 : 0;
    g.dx = (R)h->cfg.dx; g.dy = (R)h->cfg.dy; g.dt = (R)h->cfg.dt;
    g.inv_dx = (R)(1.0 / h->cfg.dx); g.inv_dy = (R)(1.0 / h->cfg.dy);
    g.hx = (R)(0.5 / h->cfg.dx); g.hy = (R)(0.5 / h->cfg.dy);
    g.khx = (R)(0.5 * h->cfg.dt / h->cfg.dx); g.khy = (R)(0.5 * h->cfg.dt / h->cfg.dy);
    g.nnode = h->nnode;
    return g;
}

template <typename R>
__host__ __device__ inline int64_t pidx(const GridArgs<R> &g, int i, int j) {
    return (int64_t)(j + g.G) * g.nxp + (i + g.G);
}

// --------------------------------------------------------------------------- device helpers

// 1/sqrt(x) and 1/x: in FP32 the hardware approximations (2 ulp, far below the
// FP32 form's tolerances); in FP64 the library's correctly rounded forms.
__device__ inline float rsqrt_r(float x) { return rsqrtf(x); }
__device__ inline double rsqrt_r(double x) { return rsqrt(x); }
__device__ inline float rcp_r(float x) { return __fdividef(1.0f, x); }
__device__ inline double rcp_r(double x) { return __drcp_rn(x); }

// x >= 1 for a non-negative x.  FP64: an integer compare of the bits (ordered
// like the values for non-negative doubles), which keeps the comparison off
// the narrow FP64 pipe.
__device__ inline bool ge_one(double x) { return __double_as_longlong(x) >= 0x3FF0000000000000ll; }
__device__ inline bool ge_one(float x) { return x >= 1.0f; }

__device__ inline double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ inline float fma_r(float a, float b, float c) { return fmaf(a, b, c); }

// (R(b) v)_x = v_x + (v.b) b_x + v_y b_z - v_z b_y (and cyclically) before the
// division by 1 + |b|^2: three FMAs per component.
template <typename R>
__device__ inline R rot_row(R v0, R v1, R v2, R vb, R b0, R b1, R b2) {
    return fma_r(v1, b2, fma_r(-v2, b1, fma_r(vb, b0, v0)));
}

// The implicit push's velocity update and move (Eq. 2) from w = u + k E: the
// rows r of (1 + |b|^2) R(b) w, then u' = 2 ubar - u = r (2 inv) - u and the
// move in cells s = f + dt/dx ubar/gamma = f + r (inv/gamma) dt/dx (one
// product fewer than forming ubar first).
template <typename R>
__device__ inline void push_move(R bx, R by, R bz, R inv, R ig, R wx, R wy, R wz, R ux, R uy, R uz, R fx, R fy,
                                 R sdx, R sdy, R &nux, R &nuy, R &nuz, R &sx, R &sy) {
    const R vb = wx * bx + wy * by + wz * bz;
    const R rx = rot_row(wx, wy, wz, vb, bx, by, bz), ry = rot_row(wy, wz, wx, vb, by, bz, bx);
    const R rz = rot_row(wz, wx, wy, vb, bz, bx, by);
    const R i2 = R(2) * inv, ti = inv * ig;
    nux = fma_r(rx, i2, -ux);
    nuy = fma_r(ry, i2, -uy);
    nuz = fma_r(rz, i2, -uz);
    sx = fma_r(rx, ti * sdx, fx);
    sy = fma_r(ry, ti * sdy, fy);
}

// The 13 moments one particle contributes (Eq. 3): rho = w q,
// S = w q^2 dt^2 / (4 m gamma) R(b), dj = w q R(b) u / gamma, with
// gamma = sqrt(1 + |u|^2) and b = q dt B / (2 m gamma).
// kq = q dt / (2 m) and hq = q dt^2 / (4 m) are per-species constants (the S
// factor w q^2 dt^2 / (4 m gamma (1+|b|^2)) is the dj factor times hq).  Also
// returns 1/gamma, b and 1/(1 + |b|^2) (the FP64 form carries them to the next
// push).
template <typename R>
__device__ inline void particle_moments_c(R q, R kq, R hq, R w, R ux, R uy, R uz, R Bx, R By, R Bz, R *val, R &ig,
                                          R &bx, R &by, R &bz, R &inv) {
    ig = rsqrt_r(R(1) + ux * ux + uy * uy + uz * uz);
    R k = kq * ig;
    bx = k * Bx, by = k * By, bz = k * Bz;
    inv = rcp_r(R(1) + bx * bx + by * by + bz * bz);
    const R gi = ig * inv;
    val[0] = w * q;
    const R cj = val[0] * gi, cs = cj * hq;
    // cs times the rows of (I + [.x b] + b b^T) ((R v)_x = v_x + v_y bz - v_z by + (v.b) bx, ...):
    // with c = cs b each entry is one FMA, e.g. cs (bz + bx by) = cz + cx by
    const R cx = cs * bx, cy = cs * by, cz = cs * bz;
    val[1] = fma_r(cx, bx, cs);
    val[2] = fma_r(cx, by, cz);
    val[3] = fma_r(cx, bz, -cy);
    val[4] = fma_r(cy, bx, -cz);
    val[5] = fma_r(cy, by, cs);
    val[6] = fma_r(cy, bz, cx);
    val[7] = fma_r(cz, bx, cy);
    val[8] = fma_r(cz, by, -cx);
    val[9] = fma_r(cz, bz, cs);
    R vb = ux * bx + uy * by + uz * bz;
    val[10] = cj * rot_row(ux, uy, uz, vb, bx, by, bz);
    val[11] = cj * rot_row(uy, uz, ux, vb, by, bz, bx);
    val[12] = cj * rot_row(uz, ux, uy, vb, bz, bx, by);
}

// The same moments as class factors times unscaled parts (FP64 deposits, which
// fold the factors into the corner weights: 4 products per class instead of
// 13 scalings): rho = fr, S = fS part[1..9], dj = fj part[10..12] (part[0] is
// not set).  Same 1/gamma, b, 1/(1+|b|^2) as particle_moments_c.
template <typename R>
__device__ inline void particle_moment_parts(R q, R kq, R cq2, R w, R ux, R uy, R uz, R Bx, R By, R Bz, R *part,
                                             R &fr, R &fS, R &fj, R &ig, R &bx, R &by, R &bz, R &inv) {
    ig = rsqrt_r(R(1) + ux * ux + uy * uy + uz * uz);
    R k = kq * ig;
    bx = k * Bx, by = k * By, bz = k * Bz;
    inv = rcp_r(R(1) + bx * bx + by * by + bz * bz);
    const R gi = ig * inv;
    fr = w * q;
    fS = (w * cq2) * gi;
    fj = fr * gi;
    part[1] = R(1) + bx * bx;
    part[2] = bz + bx * by;
    part[3] = -by + bx * bz;
    part[4] = -bz + by * bx;
    part[5] = R(1) + by * by;
    part[6] = bx + by * bz;
    part[7] = by + bz * bx;
    part[8] = -bx + bz * by;
    part[9] = R(1) + bz * bz;
    R vb = ux * bx + uy * by + uz * bz;
    part[10] = rot_row(ux, uy, uz, vb, bx, by, bz);
    part[11] = rot_row(uy, uz, ux, vb, by, bz, bx);
    part[12] = rot_row(uz, ux, uy, vb, bz, bx, by);
}

// Deterministic deposit.  Every corner contribution of a particle is rounded
// once to an integer multiple of 2^-e[class] and the integers are summed with
// 64-bit integer additions, which are exact and associative: the sums do not
// depend on the order in which warps, blocks or atomics add them.  The classes
// are rho (moment 0), S (1..9) and dj (10..12).  |rho| and every |dj| component
// of one particle are at most |w q| (|R(b) u| <= |u| < gamma), every |S|
// entry at most |w| q^2 dt^2 / (4 m) (R(b) entries are at most 1 in size, and
// 1/gamma <= 1), and the bilinear weights of one particle on one node are at
// most 1, so a node sum stays below the class bound B = sum over all loaded
// particles; e = 62 - ceil(log2 B) keeps |sum| 2^e <= 2^62.
struct FixScale {
    int e[3];     // exponents of the classes rho, S, dj
    float s[3];   // 2^e (FP32 form)
    double inv[3];  // 2^-e
};

__host__ __device__ constexpr int mom_class(int k) { return k == 0 ? 0 : (k < 10 ? 1 : 2); }

// x 2^e rounded to the nearest integer (ties away from zero), from the bits of
// x with integer operations only.
__device__ inline long long fix_of(double x, const FixScale &f, int cls) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    const long long m = (b & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;
    const int sh = ex - 1075 + f.e[cls];   // |x| 2^e = m 2^sh
    long long r;
    if (ex == 0 || sh <= -64) r = 0;
    else if (sh >= 0) r = m << sh;          // sh <= 9 while |x| 2^e < 2^62
    else r = (m + (1ll << (-sh - 1))) >> (-sh);
    return b < 0 ? -r : r;
}
__device__ inline long long fix_of(float x, const FixScale &f, int cls) { return __float2ll_rn(x * f.s[cls]); }

// Butterfly reduce-scatter of 26 values over the warp: returns, in every
// lane, the warp sum of one of the 26 (index rs26_index(lane), -1 for the six
// lanes that end up with padding).  26 -> 13 -> 7 -> 4 -> 2 -> 1 values per lane.
template <typename R>
__device__ inline R reduce_scatter26(const R (&v)[26], int lane) {
    R a[14];
    bool b = (lane & 16) != 0;
#pragma unroll
    for (int j = 0; j < 13; ++j) {
        R lo = v[j], hi = v[j + 13];
        R s = b ? lo : hi, k = b ? hi : lo;
        a[j] = k + __shfl_xor_sync(0xffffffffu, s, 16);
    }
    a[13] = R(0);
    R c[8];
    b = (lane & 8) != 0;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        R lo = a[j], hi = a[j + 7];
        R s = b ? lo : hi, k = b ? hi : lo;
        c[j] = k + __shfl_xor_sync(0xffffffffu, s, 8);
    }
    c[7] = R(0);
    R d[4];
    b = (lane & 4) != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        R lo = c[j], hi = c[j + 4];
        R s = b ? lo : hi, k = b ? hi : lo;
        d[j] = k + __shfl_xor_sync(0xffffffffu, s, 4);
    }
    R e[2];
    b = (lane & 2) != 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        R lo = d[j], hi = d[j + 2];
        R s = b ? lo : hi, k = b ? hi : lo;
        e[j] = k + __shfl_xor_sync(0xffffffffu, s, 2);
    }
    b = (lane & 1) != 0;
    R s = b ? e[0] : e[1], k = b ? e[1] : e[0];
    return k + __shfl_xor_sync(0xffffffffu, s, 1);
}

__device__ inline int rs26_index(int lane) {
    int j2 = (lane & 1) + 2 * ((lane >> 1) & 1) + 4 * ((lane >> 2) & 1);
    if (j2 >= 7) return -1;
    int j1 = j2 + 7 * ((lane >> 3) & 1);
    if (j1 >= 13) return -1;
    return j1 + 13 * ((lane >> 4) & 1);
}

// c = cy * nx + cx split with a multiply-high (magic = ceil(2^32 / nx), c < 2^31).
__device__ inline void cell_split(int32_t c, int nx, uint32_t magic, int &cx, int &cy) {
    int q = (int)__umulhi((uint32_t)c, magic);
    int r = c - q * nx;
    if (r < 0) {
        q -= 1;
        r += nx;
    }
    cx = r;
    cy = q;
}

// a mod n for a in (-n, 2n)
__device__ inline int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Cell form of the bilinear weighting (Section 3.3, area weighting), used by
// every FP64 gather: per component F(fx, fy) = a + fx b + fy c + fx fy d with
// a = F00, b = F10 - F00, c = F01 - F00, d = (F11 - F10) - c -- three FMAs
// per component instead of the four corner weights and four products.  The
// FP64 push makes (a, b, c, d) once per cell of its tile; the coefficients
// and their evaluation come from these two functions alone, so that a
// particle's field is the same bits in the push and at rest.
template <typename R>
struct CellC {
    V4<R> k[3];   // per component: (a, b, c, d)
};

template <typename R>
__device__ inline V4<R> cell_coef1(R f00, R f10, R f01, R f11) {
    V4<R> v;
    v.x = f00;
    v.y = f10 - f00;
    v.z = f01 - f00;
    v.w = (f11 - f10) - v.z;
    return v;
}

template <typename R>
__device__ inline void cell_coef(const V4<R> &f00, const V4<R> &f10, const V4<R> &f01, const V4<R> &f11,
                                 CellC<R> &o) {
    o.k[0] = cell_coef1(f00.x, f10.x, f01.x, f11.x);
    o.k[1] = cell_coef1(f00.y, f10.y, f01.y, f11.y);
    o.k[2] = cell_coef1(f00.z, f10.z, f01.z, f11.z);
}

template <typename R>
__device__ inline R cell_eval(const V4<R> &k, R fx, R fy, R fxy) {
    return fma(fxy, k.w, fma(fy, k.z, fma(fx, k.y, k.x)));
}

// Bilinear gather of a padded V4 node field at cell (cx, cy), offsets (fx, fy)
// (FP64: the cell form above).
template <typename R>
__device__ inline void gather4(const V4<R> *__restrict__ F, const GridArgs<R> &g, int cx, int cy, R fx, R fy,
                               R &ox, R &oy, R &oz) {
    int64_t p00 = pidx(g, cx, cy);
    V4<R> a = F[p00], b = F[p00 + 1], c = F[p00 + g.nxp], d = F[p00 + g.nxp + 1];
    if constexpr (sizeof(R) == 8) {
        CellC<R> k;
        cell_coef(a, b, c, d, k);
        const R fxy = fx * fy;
        ox = cell_eval(k.k[0], fx, fy, fxy);
        oy = cell_eval(k.k[1], fx, fy, fxy);
        oz = cell_eval(k.k[2], fx, fy, fxy);
        return;
    }
    R w00 = (R(1) - fx) * (R(1) - fy), w10 = fx * (R(1) - fy), w01 = (R(1) - fx) * fy, w11 = fx * fy;
    ox = w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x;
    oy = w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y;
    oz = w00 * a.z + w10 * b.z + w01 * c.z + w11 * d.z;
}

// Unpadded node index of the corner (cx + di, cy + dj) with wrap.
template <typename R>
__device__ inline int64_t node_of(const GridArgs<R> &g, int cx, int cy, int di, int dj) {
    int i = cx + di, j = cy + dj;
    if (g.periodic_x && i >= g.nx) i -= g.nx;
    if (j >= g.ny) j -= g.ny;
    return (int64_t)j * g.nxn + i;
}

// FP64 deposit of one particle (in the push and at rest alike, so that a
// deposit at rest repeats the push's bitwise): per corner, the weight times
// each class factor, times the parts; every lane adds its own products in L2.
// The lanes of one cell would all add to one address in each instruction, so
// lane l starts at corner l mod 4 and, for the FP64 adds, at moment 3 ((l / 4)
// mod 4): 16 addresses per instruction, two lanes on each (the fixed-point
// adds keep the moment order: their class scale would become a run-time index).
template <bool kFix>
__device__ inline void deposit_fp64(double *M, unsigned long long *Mfix, const FixScale &fs, const GridArgs<double> &g,
                                    int cx, int cy, double fx, double fy, const double *part, double fr, double fS,
                                    double fj, int lane) {
    const double mx = 1.0 - fx, my = 1.0 - fy;
    const int rr = kFix ? 0 : (lane >> 2) & 3;
#pragma unroll
    for (int c0 = 0; c0 < 4; ++c0) {
        const int cc = (c0 + lane) & 3, ox = cc & 1, oy = cc >> 1;
        const double wc = (ox ? fx : mx) * (oy ? fy : my);   // the bilinear weight of corner (ox, oy)
        const int64_t node = node_of(g, cx, cy, ox, oy);
        const double wr = wc * fr, ws = wc * fS, wj = wc * fj;
#pragma unroll
        for (int kk = 0; kk < NMOM; ++kk) {
            if (kFix) {
                const double p = kk == 0 ? wr : (kk < 10 ? ws : wj) * part[kk];
                atomicAdd(&Mfix[(int64_t)kk * g.nnode + node], (unsigned long long)fix_of(p, fs, mom_class(kk)));
            } else {
                // moment (kk + 3 rr) mod 13: its factor and part selected (rho: factor wr, part 1)
                const int k1 = (kk + 3) % NMOM, k2 = (kk + 6) % NMOM, k3 = (kk + 9) % NMOM;
                const int km = rr == 0 ? kk : rr == 1 ? k1 : rr == 2 ? k2 : k3;
                auto fac = [&](int k) { return k == 0 ? wr : (k < 10 ? ws : wj); };
                auto prt = [&](int k) { return k == 0 ? 1.0 : part[k]; };
                const double f = rr == 0 ? fac(kk) : rr == 1 ? fac(k1) : rr == 2 ? fac(k2) : fac(k3);
                const double q = rr == 0 ? prt(kk) : rr == 1 ? prt(k1) : rr == 2 ? prt(k2) : prt(k3);
                atomicAdd(&M[(int64_t)km * g.nnode + node], f * q);
            }
        }
    }
}

// FP64 deposit of the push in cell form.  With P_k the particle's 13 moment
// values (particle_moments_c) and (fx, fy) its offsets in cell c, its
// corner contributions (1-fx)(1-fy) P, fx(1-fy) P, (1-fx) fy P and fx fy P
// (the area weighting of Section 3.3) are sums of A = P, X = fx P, Y = fy P and
// Z = fx fy P: corner (0,0) A - X - Y + Z, (1,0) X - Z, (0,1) Y - Z, (1,1) Z.
// The push adds A, X, Y, Z of every moment into its cell's sums (three
// products per moment instead of four, and no corner weights);
// k_cell_moments then adds every cell's corner values into the node moments.
// The four sums of a (moment, cell) are adjacent (one 32-byte sector); lane l
// starts at moment (l / 4) mod 2 and at sum l mod 4, so that the lanes of one
// cell spread each instruction's reductions over 8 addresses in 2 sectors
// (measured on the 1024 x 512 foil's push: 1, 2, 4, 8 moment offsets
// 2.225, 2.183, 2.191, 2.196 ms; 8 offsets with the sums in separate planes, 32
// sectors per instruction, 5.79 ms).
__device__ inline void deposit_fp64_cell(double *Mc, int64_t ncell, int64_t cell, double fx, double fy,
                                         const double *val, int lane) {
    const double fxy = fx * fy;
    double P[NMOM];
#pragma unroll
    for (int k = 0; k < NMOM; ++k) P[k] = val[k];
    // P rotated by rr: Q[k] = P[(k + rr) mod 13]
    const int rr = (lane >> 2) & 1;
    {
        double Q[NMOM];
#pragma unroll
        for (int k = 0; k < NMOM; ++k) Q[k] = rr ? P[(k + 1) % NMOM] : P[k];
#pragma unroll
        for (int k = 0; k < NMOM; ++k) P[k] = Q[k];
    }
#pragma unroll
    for (int kk = 0; kk < NMOM; ++kk) {
        const int km = kk + rr >= NMOM ? kk + rr - NMOM : kk + rr;
        const double a = P[kk], x = a * fx, y = a * fy, z = a * fxy;
        double *base = Mc + ((int64_t)km * ncell + cell) * 4;
#pragma unroll
        for (int c0 = 0; c0 < 4; ++c0) {
            const int kind = (c0 + lane) & 3;
            const double v = kind == 0 ? a : kind == 1 ? x : kind == 2 ? y : z;
            atomicAdd(base + kind, v);
        }
    }
}

// ---------------------------------------------------------------- shape orders 2-4
//
// The centred B-spline of degree N (2, 3, 4) over the (N + 1) x (N + 1) nodes
// nearest the particle (the higher-order weightings Section 3.3's last
// paragraph mentions beside the paper's linear one, up to fourth order).  Per
// axis, from the cell c and offset f: the first node is c - (N - 1)/2 for odd
// N, c - N/2 (one more when f >= 1/2, centring on the nearest node) for even
// N; node k weighs B_N of its distance (first + k - c) - f.  Along y and a
// periodic x the node indices wrap; along a walled x a node beyond a wall is
// folded onto the wall node (its weight stays in the box).
template <typename R, int N>
struct SplineN {
    int ix[N + 1], iy[N + 1];   // unpadded node column and row indices
    R wx[N + 1], wy[N + 1];
};

// B_N(x) from its piecewise polynomial form.
template <typename R, int N>
__device__ inline R bspline_w(R x) {
    const R a = x < R(0) ? -x : x;
    if (N == 2) {
        if (a <= R(0.5)) return R(0.75) - a * a;
        const R b = R(1.5) - a;
        return a <= R(1.5) ? R(0.5) * b * b : R(0);
    }
    if (N == 3) {
        if (a <= R(1)) return R(2.0 / 3.0) - a * a + R(0.5) * a * a * a;
        const R b = R(2) - a;
        return a <= R(2) ? b * b * b * R(1.0 / 6.0) : R(0);
    }
    if (a <= R(0.5)) return R(115.0 / 192.0) - R(0.625) * a * a + R(0.25) * a * a * a * a;
    if (a <= R(1.5)) return (R(55) + R(20) * a - R(120) * a * a + R(80) * a * a * a - R(16) * a * a * a * a) * R(1.0 / 96.0);
    const R b = R(5) - R(2) * a;
    return a <= R(2.5) ? b * b * b * b * R(1.0 / 384.0) : R(0);
}

template <typename R, int N>
__device__ inline void spline_axis(int c, R f, int n, bool periodic, int (&idx)[N + 1], R (&w)[N + 1]) {
    const int first = (N % 2) ? c - (N - 1) / 2 : c - N / 2 + (f >= R(0.5) ? 1 : 0);
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        w[k] = bspline_w<R, N>(R(first + k - c) - f);
        int i = first + k;
        if (periodic) {
            i %= n;
            if (i < 0) i += n;
        } else {
            i = i < 0 ? 0 : (i > n ? n : i);
        }
        idx[k] = i;
    }
}

template <typename R, int N>
__device__ inline SplineN<R, N> spline_n(const GridArgs<R> &g, int cx, int cy, R fx, R fy) {
    SplineN<R, N> s;
    spline_axis<R, N>(cx, fx, g.nx, g.periodic_x != 0, s.ix, s.wx);
    spline_axis<R, N>(cy, fy, g.ny, true, s.iy, s.wy);
    return s;
}

// Value of a padded V4 node field at the particle (rows first, then columns).
template <typename R, int N>
__device__ inline void gather_s(const V4<R> *__restrict__ F, const GridArgs<R> &g, const SplineN<R, N> &s, R &ox,
                                R &oy, R &oz) {
    ox = oy = oz = R(0);
#pragma unroll
    for (int b = 0; b <= N; ++b) {
        const V4<R> *row = F + (int64_t)(s.iy[b] + g.G) * g.nxp + g.G;
        R sx = R(0), sy = R(0), sz = R(0);
#pragma unroll
        for (int a = 0; a <= N; ++a) {
            const V4<R> v = row[s.ix[a]];
            sx += s.wx[a] * v.x;
            sy += s.wx[a] * v.y;
            sz += s.wx[a] * v.z;
        }
        ox += s.wy[b] * sx;
        oy += s.wy[b] * sy;
        oz += s.wy[b] * sz;
    }
}

// Element j of a short register array, by compare and select (no local memory).
template <int M, typename T>
__device__ inline T pick(const T (&v)[M], int j) {
    T r = v[0];
#pragma unroll
    for (int q = 1; q < M; ++q) r = (j == q) ? v[q] : r;
    return r;
}

// Deposit of one particle with a spline shape (in the push and at rest
// alike): node by node, every lane adds its own products in L2, the lanes of
// a warp starting at different nodes (lane mod (N + 1)^2).  kParts: the values
// are FP64 parts with the class factors fr, fS, fj (as deposit_fp64 takes
// them); otherwise the 13 moment values.  kFix: exact fixed-point sums.
template <typename R, bool kFix, bool kParts, int N>
__device__ inline void deposit_s(R *M, unsigned long long *Mfix, const FixScale &fs, const GridArgs<R> &g,
                                 const SplineN<R, N> &s, const R *val, R fr, R fS, R fj, int lane) {
    constexpr int NN = (N + 1) * (N + 1);
#pragma unroll 1
    for (int k0 = 0; k0 < NN; ++k0) {
        int k = k0 + lane % NN;
        k = k >= NN ? k - NN : k;
        const int a = k % (N + 1), b = k / (N + 1);
        const R wc = pick<N + 1>(s.wx, a) * pick<N + 1>(s.wy, b);
        const int64_t node = (int64_t)pick<N + 1>(s.iy, b) * g.nxn + pick<N + 1>(s.ix, a);
        const R wr = wc * fr, ws = wc * fS, wj = wc * fj;
#pragma unroll
        for (int kk = 0; kk < NMOM; ++kk) {
            const R p = kParts ? (kk == 0 ? wr : (kk < 10 ? ws : wj) * val[kk]) : wc * val[kk];
            if (kFix) atomicAdd(&Mfix[(int64_t)kk * g.nnode + node], (unsigned long long)fix_of(p, fs, mom_class(kk)));
            else atomicAdd(&M[(int64_t)kk * g.nnode + node], p);
        }
    }
}

// --------------------------------------------------------------------------- host entry points

int check_launch(const char *what);
void timing_begin(pic_t *h);
void timing_end(pic_t *h, int cls, int nlaunch);
inline void count_launch(pic_t *h, int n = 1) { h->timing.launches[4] += n; }

// fields (pic_field.cu)
int field_literal(pic_t *h);
int field_cn(pic_t *h);
int node_average(pic_t *h, int hsrc, int bdst);
int fill_ghosts(pic_t *h, void *padded);
int upload_fields(pic_t *h, const double *E3, const double *H3);
int download_fields(pic_t *h, double *E3, double *H3);

// particles (pic_particles.cu): conversion, deposit at rest, state export
int deposit_only(pic_t *h, int s);
int clear_moments(pic_t *h);
int clear_step_moments(pic_t *h);       // what a step's deposit adds into (the touched node tiles only)
int fix_to_moments(pic_t *h);           // deterministic deposit: Mfix -> M (+ Mlo)
int fix_scale(const pic_t *h, FixScale *out);
int load_convert(pic_t *h, int s, int buf, int64_t n, const double *const src[6], unsigned long long *bad,
                 bool over_link, const int32_t *csrc = nullptr);
// over_link: the arrays are page-locked host memory read in place; csrc: checkpoint form (src[0], src[1]
// are in-cell offsets, csrc the cell indices)   // *bad = first invalid index
int particles_to_stage(pic_t *h, int s, int64_t *n_out, bool raw = false);   // raw: in-cell offsets for x, y
int count_species(pic_t *h, int s, int64_t *n_out);

// batched particle step of several runs (pic_tile.cu launches, pic_api.cu drives)
struct BatchScratch {
    cudaStream_t st = nullptr;
    int cap = 0;                        // runs
    void *args_dev = nullptr;           // cap argument blocks
    void *args_host[2] = {nullptr, nullptr};     // pinned staging of the argument blocks (two, alternating)
    int32_t *idx = nullptr;             // device: run_items[cap + 1], run_tiles[cap + 1], ticket
    int32_t *idx_host[2] = {nullptr, nullptr};   // pinned staging of run_tiles
    cudaEvent_t ev_stage[2] = {nullptr, nullptr}, ev_push = nullptr, ev_done = nullptr;
    int slot = 0;                       // staging slot of the current step
};
size_t batch_args_bytes();              // one argument block (the larger of the two forms)
int batch_push(BatchScratch &b, pic_t **hs, int n);
int batch_regroup(BatchScratch &b, pic_t **hs, int n);
int push_work_list(pic_t *h);           // k_chunk_counts + scan on the run's stream

// tiled step (pic_tile.cu)
int tile_setup(pic_t *h);
int particle_tiles(pic_t *h, bool prepared = false);
int push_prep(pic_t *h, bool next);
int cell_moments(pic_t *h, bool all = false);   // FP64 cell sums -> node moments (touched tiles; all: every tile)
int reset_lists(pic_t *h);       // the tile lists and regroup queues, emptied before a push
int regroup_tiles(pic_t *h);     // per-tile stable cell sort of stayers + arrivals into the spare set
int scan_tiles(pic_t *h, const int32_t *in, int32_t *out);
int tile_counts(pic_t *h, int s);   // tcount[t] = particles of tile t (device)
int touch_map(pic_t *h);            // touched[] of the push just queued (occupancy dilated, far movers: all)

// sort and rebuild (pic_sort.cu)
enum RebuildSource { REBUILD_FROM_STEP = 0, REBUILD_FROM_LOAD = 1 };
int rebuild_species(pic_t *h, int s, int source, int64_t n_second);
int ensure_sort_capacity(pic_t *h, int64_t n);
int init_empty_bins(pic_t *h, int s);
int64_t slots_needed(const pic_t *h, int64_t n);
int64_t sort_hist_entries(int64_t cap);   // radix histogram entries for cap keys
int scan_i32_inplace(pic_t *h, int32_t *a, int64_t n);   // exclusive, multi-block
int scan_sums_entries();

// field ionisation (pic_ionize.cu): one chain's pass over its ion species -- decisions, staging of the
// ionised particles at offset of the staging planes (stride scap), compaction of the species
struct IonChain {
    int species;            // the ion species
    double c2ip, expo, K;   // |C|^2 Ip, 2 n* - 1, 2 (2 Ip)^(3/2) (atomic units)
    double fmax;            // field of the rate formula's maximum (atomic units)
    double field_au, dt_au; // the run's field unit and time step in atomic units
};
int collide(pic_t *h, const pic_collisions *p, unsigned long long *d_pairs);
int ion_chain(pic_t *h, const IonChain &c, uint64_t seed, int32_t *scell, double *sval, int64_t scap, int64_t offset,
              int64_t *n_out);

// diagnostics (pic_diag.cu)
int diagnostics(pic_t *h, pic_diag *out);
int moments_to_stage(pic_t *h);     // stage[13][nnode] = M (+ Mlo) / node area, FP64

}  // namespace pic
