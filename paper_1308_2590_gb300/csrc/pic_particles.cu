// Particle state outside the step: conversion of loaded global positions into
// (cell, offsets), deposit of the moments at rest (after a load or a field
// overwrite, Eq. 3), and export of the particles in the library's order.
// Particles are stored per species, structure-of-arrays, in tile bins
// (pic_internal.cuh).
#include <math.h>

#include "pic_internal.cuh"

namespace pic {

int scan_tiles(pic_t *h, const int32_t *in, int32_t *out);

template <typename R>
struct DepArgs {
    GridArgs<R> g;
    const int32_t *cell;
    const R *ox, *oy, *ux, *uy, *uz, *w;
    const int32_t *bstart, *useg, *segn;
    const V4<R> *B;
    R *M;
    unsigned long long *Mfix;
    FixScale fs;
    R q, m;
    R kq, cq2, hq;    // q dt / (2 m), q^2 dt^2 / (4 m), q dt^2 / (4 m): per species, from the host (as for the push)
    int32_t *flags;   // checks build: FLAG_CHECK on a broken invariant
    double *cr;       // FP64 form: the carried quantities of the bins ([NCARRY][ccap]), else nullptr
    int64_t ccap;
    double *Mc;       // FP64 L2-reduction form: the cell sums the push deposits into (else nullptr)
    int tnx, tny, ntx;  // tiles (FP64: the block's tile of B in cell form, in shared memory)
};

// Moments (Eq. 3) of particles at rest with the current node B, DEP_SPLIT
// blocks per tile bin, a warp per segment (block y of a tile takes every
// DEP_SPLIT-th group of its warps' segments: a plasma that fills a few of the
// tiles still puts enough warps on the FP64 pipe and the L2 reductions; 1 ->
// 4 blocks per tile measured 2.43 -> 2.08 ms FP64, 0.45 -> 0.40 ms FP32 for
// 6.55M particles of a laser foil).  FP32: lanes whose particles share a cell (at
// least 6 of them; bins are in cell order, so most segments hold one or two
// cells) first sum their 52 corner products with the butterfly reduce-scatter
// and add 26 values per corner pair; the other lanes add their own products.
// FP64: every lane adds its own products (the butterfly's FP64 adds would cost
// more of the scarce FP64 pipe than the L2 reductions they save), as the push
// does (deposit_fp64).  Global atomics (floating point, or exact fixed point
// when kFix).
template <typename R>
constexpr int min_group_at_rest() { return sizeof(R) == 4 ? 6 : 33; }
constexpr int DEP_SPLIT = 4;

template <typename R, bool kFix>
__device__ inline void add_moment(const DepArgs<R> &a, int k, int64_t node, R v) {
    if (kFix)
        atomicAdd(&a.Mfix[(int64_t)k * a.g.nnode + node], (unsigned long long)fix_of(v, a.fs, mom_class(k)));
    else
        atomicAdd(&a.M[(int64_t)k * a.g.nnode + node], v);
}

template <typename R, bool kFix>
__global__ void k_deposit_bins(DepArgs<R> a) {
    extern __shared__ __align__(16) unsigned char dsm[];
    constexpr bool kTab = sizeof(R) == 8;   // FP64: B of the tile's cells in cell form, as the push gathers it
    const int t = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t b0 = a.bstart[t];
    const int u = a.useg[t];
    const GridArgs<R> &g = a.g;
    if (u == 0) return;
    CellC<R> *tab = (CellC<R> *)dsm;
    const int X0 = (t % a.ntx) * a.tnx, Y0 = (t / a.ntx) * a.tny;
    const int tw = min(a.tnx, g.nx - X0), th = min(a.tny, g.ny - Y0);
    if constexpr (kTab) {
        for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
            const int ly = i / tw, lx = i - ly * tw;
            const int64_t p00 = pidx(g, X0 + lx, Y0 + ly);
            cell_coef(a.B[p00], a.B[p00 + 1], a.B[p00 + g.nxp], a.B[p00 + g.nxp + 1], tab[i]);
        }
        __syncthreads();
    }
    for (int j = blockIdx.y * nw + wid; j < u; j += nw * gridDim.y) {
        const int n = a.segn[b0 / SEG + j];
        bool valid = lane < n;
        const int64_t p = b0 + (int64_t)j * SEG + lane;
        if (kChecks && valid) {
            const int32_t cc = a.cell[p];
            const R ofx = a.ox[p], ofy = a.oy[p];
            if (cc < 0 || cc >= g.nx * g.ny || !(ofx >= R(0) && ofx < R(1)) || !(ofy >= R(0) && ofy < R(1))) {
                atomicOr(a.flags, FLAG_CHECK);
                valid = false;
            }
        }
        int32_t c = -1;
        R fx = R(0), fy = R(0);
        R val[NMOM];   // FP32: the moment values; FP64: their parts, with the class factors fr, fS, fj
        for (int k = 0; k < NMOM; ++k) val[k] = R(0);
        R fr = R(0), fS = R(0), fj = R(0);
        if (valid) {
            c = a.cell[p];
            const int cx = c % g.nx, cy = c / g.nx;
            fx = a.ox[p];
            fy = a.oy[p];
            R Bx, By, Bz;
            const int lx = cx - X0, ly = cy - Y0;
            if (kTab && lx >= 0 && lx < tw && ly >= 0 && ly < th) {   // the same bits as gather4
                const CellC<R> &cb = tab[ly * tw + lx];
                const R fxy = fx * fy;
                Bx = cell_eval(cb.k[0], fx, fy, fxy);
                By = cell_eval(cb.k[1], fx, fy, fxy);
                Bz = cell_eval(cb.k[2], fx, fy, fxy);
            } else {
                gather4(a.B, g, cx, cy, fx, fy, Bx, By, Bz);
            }
            R ig, bx, by, bz, inv;
            if (sizeof(R) == 8 && (kFix || !a.Mc))   // FP64 corner form: class factors and parts
                particle_moment_parts(a.q, a.kq, a.cq2, a.w[p], a.ux[p], a.uy[p], a.uz[p], Bx, By, Bz, val, fr, fS, fj,
                                      ig, bx, by, bz, inv);
            else   // the 13 moment values (the FP64 cell form as the push makes them)
                particle_moments_c(a.q, a.kq, a.hq, a.w[p], a.ux[p], a.uy[p], a.uz[p], Bx, By, Bz, val, ig, bx, by,
                                   bz, inv);
            if (sizeof(R) == 8 && a.cr) {   // what the next push needs of this B (carried, FP64 form)
                a.cr[p] = (double)ig;
                a.cr[a.ccap + p] = (double)bx;
                a.cr[2 * a.ccap + p] = (double)by;
                a.cr[3 * a.ccap + p] = (double)bz;
                a.cr[4 * a.ccap + p] = (double)inv;
            }
        }
        const R W[4] = {(R(1) - fx) * (R(1) - fy), fx * (R(1) - fy), (R(1) - fx) * fy, fx * fy};
        unsigned rem = __ballot_sync(0xffffffffu, valid);
        while (rem) {
            const int cand = __shfl_sync(0xffffffffu, c, __ffs(rem) - 1);
            const unsigned grp = __ballot_sync(0xffffffffu, valid && c == cand) & rem;
            if (__popc(grp) < min_group_at_rest<R>()) break;
            const bool mem = (grp >> lane) & 1u;
            const int ccx = cand % g.nx, ccy = cand / g.nx;
            const int idx = rs26_index(lane);
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                R v[26];
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
                    for (int k = 0; k < NMOM; ++k) v[c2 * NMOM + k] = mem ? W[2 * pass + c2] * val[k] : R(0);
                const R r = reduce_scatter26(v, lane);
                if (idx >= 0 && r != R(0)) {
                    const int corner = 2 * pass + idx / NMOM, k = idx % NMOM;
                    add_moment<R, kFix>(a, k, node_of(g, ccx, ccy, corner & 1, corner >> 1), r);
                }
            }
            rem &= ~grp;
        }
        if ((rem >> lane) & 1u) {
            const int cx = c % g.nx, cy = c / g.nx;
            if constexpr (sizeof(R) == 8) {
                // the push's own FP64 deposit (cell sums, or node moments for the exact form)
                if (!kFix && a.Mc)
                    deposit_fp64_cell(a.Mc, (int64_t)g.nx * g.ny, c, (double)fx, (double)fy, (const double *)val, lane);
                else
                    deposit_fp64<kFix>((double *)a.M, a.Mfix, a.fs, g, cx, cy, (double)fx, (double)fy,
                                       (const double *)val, (double)fr, (double)fS, (double)fj, lane);
            } else {
                const int64_t nd[4] = {node_of(g, cx, cy, 0, 0), node_of(g, cx, cy, 1, 0), node_of(g, cx, cy, 0, 1),
                                       node_of(g, cx, cy, 1, 1)};
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int q = 0; q < NMOM; ++q) add_moment<R, kFix>(a, q, nd[k], W[k] * val[q]);
            }
        }
    }
}

// Moments at rest with a spline shape of degree N: the same gather
// (gather_s), moments and per-lane deposit (deposit_s) as the spline-shape
// push, so that a deposit at rest repeats the push's products bitwise; a warp
// per segment, DEP_SPLIT blocks per tile bin.
template <typename R, bool kFix, int N>
__global__ void k_deposit_s(DepArgs<R> a) {
    constexpr bool kParts = sizeof(R) == 8;
    const int t = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t b0 = a.bstart[t];
    const int u = a.useg[t];
    const GridArgs<R> &g = a.g;
    for (int j = blockIdx.y * nw + wid; j < u; j += nw * gridDim.y) {
        const int n = a.segn[b0 / SEG + j];
        const int64_t p = b0 + (int64_t)j * SEG + lane;
        if (lane >= n) continue;
        const int32_t c = a.cell[p];
        const R fx = a.ox[p], fy = a.oy[p];
        if (kChecks && (c < 0 || c >= g.nx * g.ny || !(fx >= R(0) && fx < R(1)) || !(fy >= R(0) && fy < R(1)))) {
            atomicOr(a.flags, FLAG_CHECK);
            continue;
        }
        const SplineN<R, N> sp = spline_n<R, N>(g, c % g.nx, c / g.nx, fx, fy);
        R Bx, By, Bz;
        gather_s(a.B, g, sp, Bx, By, Bz);
        R val[NMOM];
        R fr = R(1), fS = R(1), fj = R(1), ig, bx, by, bz, inv;
        if constexpr (kParts)
            particle_moment_parts(a.q, a.kq, a.cq2, a.w[p], a.ux[p], a.uy[p], a.uz[p], Bx, By, Bz, val, fr, fS, fj, ig,
                                  bx, by, bz, inv);
        else
            particle_moments_c(a.q, a.kq, a.hq, a.w[p], a.ux[p], a.uy[p], a.uz[p], Bx, By, Bz, val, ig, bx, by, bz,
                               inv);
        if (sizeof(R) == 8 && a.cr) {   // what the next push needs of this B (carried, FP64 form)
            a.cr[p] = (double)ig;
            a.cr[a.ccap + p] = (double)bx;
            a.cr[2 * a.ccap + p] = (double)by;
            a.cr[3 * a.ccap + p] = (double)bz;
            a.cr[4 * a.ccap + p] = (double)inv;
        }
        deposit_s<R, kFix, kParts, N>(a.M, a.Mfix, a.fs, g, sp, val, fr, fS, fj, lane);
    }
}

// Fixed-point sums -> floating-point moments: FP64 M, or the FP32 pair (M, Mlo)
// with M + Mlo the sum to about 2^-48 relative.
template <typename R>
__global__ void k_fix_to_moments(const unsigned long long *__restrict__ fix, R *__restrict__ M, R *__restrict__ Mlo,
                                 int64_t nnode, FixScale fs) {
    const int64_t n = (int64_t)NMOM * nnode;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = (double)(long long)fix[i] * fs.inv[mom_class((int)(i / nnode))];
        const R hi = (R)d;
        M[i] = hi;
        if (sizeof(R) == 4) Mlo[i] = (R)(d - (double)hi);
    }
}

// Global positions -> (cell, offset): s = x/dx, cell = floor(s), offset = s - cell
// (a coordinate rounding onto the far edge folds back or stays in the last cell;
// an FP32 offset that rounds to 1 moves to the next cell with offset 0).
// Positions outside [0, Lx) x [0, Ly) or non-finite momenta / weights are
// rejected: the smallest such index goes to *bad (the load is then dropped).
struct LoadSrc {
    const double *a[6];   // x, y, ux, uy, uz, w: device memory or device-accessible host memory
};

constexpr int LOAD_BS = 256;
constexpr int LOAD_SM_PERMILLE = 500;   // conversion blocks per 1000 SMs (measured: 76 x 256 on GB300
                                        // reads the link at full rate beside a regroup at nearly full speed)

template <typename R>
__global__ void __launch_bounds__(LOAD_BS) k_load_convert(GridArgs<double> g, double Lx, double Ly, LoadSrc src, int64_t n,
                               int32_t *cell, R *ox, R *oy, R *ux, R *uy, R *uz, R *w,
                               unsigned long long *bad) {
    // grid-stride.  Arrays read over the CPU-GPU link: one small block on
    // half of the SMs keeps enough reads in flight for the link, while the
    // regroup of the species converted before runs beside it at nearly full
    // speed (a conversion grid over every SM slowed that regroup about
    // threefold).  Arrays in device memory: a full grid.
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double x = src.a[0][t], y = src.a[1][t];
        const double vx = src.a[2][t], vy = src.a[3][t], vz = src.a[4][t], vw = src.a[5][t];
        if (!(x >= 0.0 && x < Lx && y >= 0.0 && y < Ly) || !isfinite(vx) || !isfinite(vy) || !isfinite(vz) ||
            !isfinite(vw)) {
            atomicMin(bad, (unsigned long long)t);
            // an in-range placeholder, so that a regroup queued before the check stays in bounds
            cell[t] = 0;
            ox[t] = oy[t] = ux[t] = uy[t] = uz[t] = w[t] = R(0);
            continue;
        }
        double sxx = x / g.dx, syy = y / g.dy;
        double flx = floor(sxx), fly = floor(syy);
        int cx = (int)flx, cy = (int)fly;
        double fx = sxx - flx, fy = syy - fly;
        // x < Lx whose x/dx rounds to nx (walls): the last cell, at the largest offset below 1 of the
        // form's precision, so that every stored offset lies in [0, 1)
        if (cx >= g.nx) { if (g.periodic_x) cx -= g.nx; else { cx = g.nx - 1; fx = 0x1.fffffffffffffp-1; } }
        if (cx < 0) { if (g.periodic_x) cx += g.nx; else { cx = 0; fx = 0.0; } }
        if (cy >= g.ny) cy -= g.ny;
        if (cy < 0) cy += g.ny;
        R rfx = (R)fx, rfy = (R)fy;
        if (sizeof(R) == 4) {
            if (rfx >= R(1)) {
                if (g.periodic_x || cx + 1 < g.nx) { rfx = R(0); cx = (cx + 1 == g.nx) ? 0 : cx + 1; }
                else rfx = (R)0.99999994;
            }
            if (rfy >= R(1)) { rfy = R(0); cy = (cy + 1 == g.ny) ? 0 : cy + 1; }
        }
        cell[t] = cy * g.nx + cx;
        ox[t] = rfx;
        oy[t] = rfy;
        ux[t] = (R)vx;
        uy[t] = (R)vy;
        uz[t] = (R)vz;
        w[t] = (R)vw;
    }
}

// Checkpoint form (cell index, in-cell offsets, u, w) -> the species' spare
// buffer set, checked like a load: cell in range, offsets in [0, 1), all
// finite.  FP32 form: the offsets, u and w are rounded to FP32 (exact for
// values saved by an FP32 handle); an offset that rounds to 1 moves to the
// next cell with offset 0, as in a load.
template <typename R>
__global__ void __launch_bounds__(LOAD_BS) k_restore_convert(GridArgs<double> g, LoadSrc src, const int32_t *csrc,
                                                             int64_t n, int32_t *cell, R *ox, R *oy, R *ux, R *uy,
                                                             R *uz, R *w, unsigned long long *bad) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = csrc[t];
        const double fx = src.a[0][t], fy = src.a[1][t];
        const double vx = src.a[2][t], vy = src.a[3][t], vz = src.a[4][t], vw = src.a[5][t];
        if (c < 0 || (int64_t)c >= (int64_t)g.nx * g.ny || !(fx >= 0.0 && fx < 1.0) || !(fy >= 0.0 && fy < 1.0) ||
            !isfinite(vx) || !isfinite(vy) || !isfinite(vz) || !isfinite(vw)) {
            atomicMin(bad, (unsigned long long)t);
            cell[t] = 0;   // in-range placeholder (a regroup may run before the check is read)
            ox[t] = oy[t] = ux[t] = uy[t] = uz[t] = w[t] = R(0);
            continue;
        }
        int cx = c % g.nx, cy = c / g.nx;
        R rfx = (R)fx, rfy = (R)fy;
        if (sizeof(R) == 4) {
            if (rfx >= R(1)) {
                if (g.periodic_x || cx + 1 < g.nx) { rfx = R(0); cx = (cx + 1 == g.nx) ? 0 : cx + 1; }
                else rfx = (R)0.99999994;
            }
            if (rfy >= R(1)) { rfy = R(0); cy = (cy + 1 == g.ny) ? 0 : cy + 1; }
        }
        cell[t] = cy * g.nx + cx;
        ox[t] = rfx;
        oy[t] = rfy;
        ux[t] = (R)vx;
        uy[t] = (R)vy;
        uz[t] = (R)vz;
        w[t] = (R)vw;
    }
}

// Bins -> compact FP64 staging [x | y | ux | uy | uz | w | cell(int32)], in the
// particle order (tiles, then segments, then the valid prefix of each).
template <typename R>
__global__ void k_bins_to_stage(GridArgs<double> g, const int32_t *bstart, const int32_t *useg, const int32_t *segn,
                                const int32_t *cstart, int64_t n, const int32_t *cell, const R *ox, const R *oy,
                                const R *ux, const R *uy, const R *uz, const R *w, double *st, bool raw) {
    __shared__ int wcnt[32];
    __shared__ int run;
    const int t = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t b0 = bstart[t], sb = b0 / SEG;
    const int u = useg[t];
    if (threadIdx.x == 0) run = 0;
    __syncthreads();
    for (int j0 = 0; j0 < u; j0 += nw) {
        const int j = j0 + wid;
        const int nseg = (j < u) ? segn[sb + j] : 0;
        if (lane == 0) wcnt[wid] = nseg;
        __syncthreads();
        int before = 0, tot = 0;
        for (int q = 0; q < nw; ++q) {
            if (q < wid) before += wcnt[q];
            tot += wcnt[q];
        }
        if (lane < nseg) {
            const int64_t p = b0 + (int64_t)j * SEG + lane;
            const int64_t o = (int64_t)cstart[t] + run + before + lane;
            const int32_t c = cell[p];
            const int cx = c % g.nx, cy = c / g.nx;
            st[o] = raw ? (double)ox[p] : ((double)cx + (double)ox[p]) * g.dx;
            st[n + o] = raw ? (double)oy[p] : ((double)cy + (double)oy[p]) * g.dy;
            st[2 * n + o] = (double)ux[p];
            st[3 * n + o] = (double)uy[p];
            st[4 * n + o] = (double)uz[p];
            st[5 * n + o] = (double)w[p];
            ((int32_t *)(st + 6 * n))[o] = c;
        }
        __syncthreads();
        if (threadIdx.x == 0) run += tot;
        __syncthreads();
    }
}

// --------------------------------------------------------------------------- host side

template <typename R>
static int deposit_only_t(pic_t *h, int s) {
    SpeciesBuf &S = h->sp[s];
    if (S.cap == 0) return 0;
    DepArgs<R> a;
    a.g = grid_args<R>(h);
    int b = S.bins;
    a.cell = S.cell[b];
    a.ox = (const R *)S.ox[b]; a.oy = (const R *)S.oy[b];
    a.ux = (const R *)S.ux[b]; a.uy = (const R *)S.uy[b]; a.uz = (const R *)S.uz[b]; a.w = (const R *)S.w[b];
    a.bstart = S.bstart;
    a.useg = S.useg[S.scur];
    a.segn = S.segn[S.scur];
    a.B = (const V4<R> *)h->B[h->bcur];
    a.M = (R *)h->M;
    a.Mfix = h->Mfix;
    if (h->det)
        if (int rc = fix_scale(h, &a.fs)) return rc;
    a.q = (R)S.q;
    a.m = (R)S.m;
    a.kq = (R)(S.q * h->cfg.dt / (2.0 * S.m));
    a.cq2 = (R)(S.q * S.q * h->cfg.dt * h->cfg.dt / (4.0 * S.m));
    a.hq = (R)(S.q * h->cfg.dt * h->cfg.dt / (4.0 * S.m));
    a.flags = h->d_flags;
    a.cr = S.carry[b];
    a.ccap = S.cap;
    a.Mc = h->Mc;   // node moments after cell_moments(h, true)
    a.tnx = h->tnx;
    a.tny = h->tny;
    a.ntx = h->ntx;
    const size_t tab = h->fp32 ? 0 : (size_t)h->tnx * h->tny * sizeof(CellC<double>);
    const dim3 grid((unsigned)h->ntiles, DEP_SPLIT);
    if (h->shape >= 2) {
        switch (h->shape * 2 + (h->det ? 1 : 0)) {
            case 4: k_deposit_s<R, false, 2><<<grid, 256, 0, h->st>>>(a); break;
            case 5: k_deposit_s<R, true, 2><<<grid, 256, 0, h->st>>>(a); break;
            case 6: k_deposit_s<R, false, 3><<<grid, 256, 0, h->st>>>(a); break;
            case 7: k_deposit_s<R, true, 3><<<grid, 256, 0, h->st>>>(a); break;
            case 8: k_deposit_s<R, false, 4><<<grid, 256, 0, h->st>>>(a); break;
            default: k_deposit_s<R, true, 4><<<grid, 256, 0, h->st>>>(a); break;
        }
    } else {
        if (tab > 48 * 1024) {
            cudaFuncSetAttribute(k_deposit_bins<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab);
            cudaFuncSetAttribute(k_deposit_bins<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab);
        }
        if (h->det) k_deposit_bins<R, true><<<grid, 256, tab, h->st>>>(a);
        else k_deposit_bins<R, false><<<grid, 256, tab, h->st>>>(a);
    }
    count_launch(h);
    return check_launch("k_deposit_bins");
}

int deposit_only(pic_t *h, int s) {
    h->touch_all = true;   // the touched-tile map describes a push, not a deposit at rest
    return h->fp32 ? deposit_only_t<float>(h, s) : deposit_only_t<double>(h, s);
}

// Zero the 13 moment planes (and the FP32 compensation) on the nodes of the
// touched tiles only: a fixed grid takes the tiles of the touched list in
// turn.  Node column i belongs to tile min(i / tnx, ntx - 1), so a wall's last
// column joins the last tile.
template <typename R>
__global__ void __launch_bounds__(128) k_clear_touched(const int32_t *__restrict__ list, const int32_t *__restrict__ list_n,
                                                       int tnx, int tny, int ntx, int nx, int ny, int nxn, int64_t nnode,
                                                       R *__restrict__ M, R *__restrict__ Mlo) {
    const int n = list_n[0];
    for (int li = blockIdx.x; li < n; li += gridDim.x) {
        const int T = list[li];
        const int tx = T % ntx, ty = T / ntx;
        const int i0 = tx * tnx, j0 = ty * tny;
        const int i1 = (tx == ntx - 1) ? nxn : min(i0 + tnx, nx);
        const int j1 = min(j0 + tny, ny);
        const int w = i1 - i0, nn = w * (j1 - j0);
        for (int k = threadIdx.x; k < nn * NMOM; k += blockDim.x) {
            const int m = k / nn, r = k - m * nn;
            const int jj = r / w, ii = r - jj * w;
            const int64_t o = (int64_t)m * nnode + (int64_t)(j0 + jj) * nxn + i0 + ii;
            M[o] = R(0);
            if (Mlo) Mlo[o] = R(0);
        }
    }
}

int clear_moments(pic_t *h) {
    size_t b = (size_t)NMOM * h->nnode * h->rs;
    if (cudaMemsetAsync(h->M, 0, b, h->st) != cudaSuccess) return check_launch("clear M");
    if (h->Mlo && cudaMemsetAsync(h->Mlo, 0, b, h->st) != cudaSuccess) return check_launch("clear Mlo");
    if (h->Mfix && cudaMemsetAsync(h->Mfix, 0, (size_t)NMOM * h->nnode * 8, h->st) != cudaSuccess)
        return check_launch("clear Mfix");
    return 0;
}

// A step's deposit adds into Mfix (deterministic) or into M and Mlo; the
// conversion after a deterministic deposit overwrites M and Mlo whole.  M is
// zero everywhere before each push: the previous push wrote only inside its
// touched tiles, and those are cleared here (everything after a deposit at
// rest, which keeps no touched-tile map).
int clear_step_moments(pic_t *h) {
    if (!h->det) {
        if (h->moments_cleared) {   // zeroed by the literal field solve that read them
            h->moments_cleared = false;
            return 0;
        }
        if (h->touch_all) return clear_moments(h);
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        unsigned grid = (unsigned)(nsm > 0 ? 8 * nsm : 1024);
        if (grid > (unsigned)h->ntiles) grid = (unsigned)h->ntiles;
        if (h->fp32)
            k_clear_touched<float><<<grid, 128, 0, h->st>>>(h->touch_list, h->list_n, h->tnx, h->tny, h->ntx, h->nx,
                                                            h->ny, h->nxn, h->nnode, (float *)h->M, (float *)h->Mlo);
        else
            k_clear_touched<double><<<grid, 128, 0, h->st>>>(h->touch_list, h->list_n, h->tnx, h->tny, h->ntx, h->nx,
                                                             h->ny, h->nxn, h->nnode, (double *)h->M, nullptr);
        count_launch(h);
        return check_launch("k_clear_touched");
    }
    if (cudaMemsetAsync(h->Mfix, 0, (size_t)NMOM * h->nnode * 8, h->st) != cudaSuccess)
        return check_launch("clear Mfix");
    return 0;
}

// Class bounds from the weights loaded so far (see FixScale).
int fix_scale(const pic_t *h, FixScale *out) {
    double B[3] = {0, 0, 0};
    const double dt = h->cfg.dt;
    for (int s = 0; s < h->nsp; ++s) {
        const double q = h->sp[s].q, m = h->sp[s].m;
        B[0] += fabs(q) * h->wabs[s];
        B[1] += q * q * dt * dt / (4.0 * m) * h->wabs[s];
    }
    B[2] = B[0];
    for (int c = 0; c < 3; ++c) {
        int e = 0;
        if (B[c] > 0) {
            int x = 0;
            frexp(B[c], &x);   // B <= 2^x
            e = 62 - x;
        }
        if (e < -120) {
            set_error("deterministic deposit: moment bound %g is too large for 64-bit fixed point", B[c]);
            return PIC_ERR_ARG;
        }
        if (e > 120) e = 120;
        out->e[c] = e;
        out->s[c] = ldexpf(1.0f, e);
        out->inv[c] = ldexp(1.0, -e);
    }
    return 0;
}

template <typename R>
static int fix_to_moments_t(pic_t *h) {
    FixScale fs;
    if (int rc = fix_scale(h, &fs)) return rc;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t n = (int64_t)NMOM * h->nnode;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8 * (int64_t)nsm) blocks = 8 * (int64_t)nsm;
    k_fix_to_moments<R><<<(unsigned)blocks, 256, 0, h->st>>>(h->Mfix, (R *)h->M, (R *)h->Mlo, h->nnode, fs);
    count_launch(h);
    return check_launch("k_fix_to_moments");
}

int fix_to_moments(pic_t *h) { return h->fp32 ? fix_to_moments_t<float>(h) : fix_to_moments_t<double>(h); }

template <typename R>
static int load_convert_t(pic_t *h, int s, int buf, int64_t n, const double *const src[6], unsigned long long *bad,
                          bool over_link, const int32_t *csrc) {
    SpeciesBuf &S = h->sp[s];
    const double Lx = h->nx * h->cfg.dx, Ly = h->ny * h->cfg.dy;
    LoadSrc ls;
    for (int k = 0; k < 6; ++k) ls.a[k] = src[k];
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // arrays read over the CPU-GPU link: half of the SMs; arrays in device memory: eight blocks per SM
    const int64_t cap = over_link ? LOAD_SM_PERMILLE * (int64_t)nsm / 1000 : 8 * (int64_t)nsm;
    int64_t blocks = (n + LOAD_BS - 1) / LOAD_BS;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (csrc)
        k_restore_convert<R><<<(unsigned)blocks, LOAD_BS, 0, h->st>>>(
            grid_args<double>(h), ls, csrc, n, S.cell[buf], (R *)S.ox[buf], (R *)S.oy[buf], (R *)S.ux[buf],
            (R *)S.uy[buf], (R *)S.uz[buf], (R *)S.w[buf], bad);
    else
        k_load_convert<R><<<(unsigned)blocks, LOAD_BS, 0, h->st>>>(
            grid_args<double>(h), Lx, Ly, ls, n, S.cell[buf], (R *)S.ox[buf], (R *)S.oy[buf], (R *)S.ux[buf],
            (R *)S.uy[buf], (R *)S.uz[buf], (R *)S.w[buf], bad);
    count_launch(h);
    return check_launch("k_load_convert");
}

int load_convert(pic_t *h, int s, int buf, int64_t n, const double *const src[6], unsigned long long *bad,
                 bool over_link, const int32_t *csrc) {
    if (n == 0) return 0;
    return h->fp32 ? load_convert_t<float>(h, s, buf, n, src, bad, over_link, csrc)
                   : load_convert_t<double>(h, s, buf, n, src, bad, over_link, csrc);
}

int count_species(pic_t *h, int s, int64_t *n_out) {
    SpeciesBuf &S = h->sp[s];
    if (S.cap == 0) {
        *n_out = 0;
        return 0;
    }
    if (int rc = tile_counts(h, s)) return rc;
    if (int rc = scan_tiles(h, S.tcount, S.cstart)) return rc;
    int32_t tot = 0;
    cudaError_t e = cudaMemcpyAsync(&tot, S.cstart + h->ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        set_error("count readback: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    *n_out = tot;
    S.n = tot;
    S.n_exact = true;
    return 0;
}

int ensure_stage_doubles(pic_t *h, int64_t ndoubles);

template <typename R>
static int to_stage_t(pic_t *h, int s, int64_t n, bool raw) {
    SpeciesBuf &S = h->sp[s];
    int b = S.bins;
    k_bins_to_stage<R><<<h->ntiles, 256, 0, h->st>>>(grid_args<double>(h), S.bstart, S.useg[S.scur], S.segn[S.scur],
                                                     S.cstart, n, S.cell[b],
                                                     (const R *)S.ox[b], (const R *)S.oy[b], (const R *)S.ux[b],
                                                     (const R *)S.uy[b], (const R *)S.uz[b], (const R *)S.w[b],
                                                     h->stage, raw);
    count_launch(h);
    return check_launch("k_bins_to_stage");
}

// Compact copy of species s into the staging buffer; *n_out = live count.
// raw: the stored in-cell offsets instead of global positions.
int particles_to_stage(pic_t *h, int s, int64_t *n_out, bool raw) {
    int64_t n = 0;
    if (int rc = count_species(h, s, &n)) return rc;  // also leaves the compact starts in cstart
    *n_out = n;
    if (n == 0) return 0;
    if (int rc = ensure_stage_doubles(h, 7 * n)) return rc;
    return h->fp32 ? to_stage_t<float>(h, s, n, raw) : to_stage_t<double>(h, s, n, raw);
}

}  // namespace pic
