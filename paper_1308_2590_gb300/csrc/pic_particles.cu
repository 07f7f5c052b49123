// Particle loop of the PIC cycle (Section 3.3): gather E^{n+1/2} and B at each
// particle with linear weights inside its cell, implicit push (Eq. 2 with E
// factored out, one push per step), move, and deposit of rho, S, dj (Eq. 3)
// at the new position.  Particles are stored structure-of-arrays per species
// as an int32 linear cell index (j*nx + i) plus in-cell offsets in [0, 1).
#include <math.h>

#include "pic_internal.cuh"

namespace pic {

template <typename R>
struct PArgs {
    GridArgs<R> g;
    int32_t *cell;
    R *ox, *oy, *ux, *uy, *uz;
    const R *w;
    const V4<R> *Ehalf, *Bold, *Bnew;
    R *M;
    uint32_t *keys;
    const int64_t *d_count;
    unsigned long long *d_dead, *d_removed;
    int32_t *flags;
    int64_t n_bound;
    R q, m, kq, sdx, sdy;
    int tnx, tny, ntx, nty;
    uint32_t dead_key;
};

template <typename R>
__device__ inline void deposit_global(const PArgs<R> &a, int cx, int cy, R fx, R fy, R w, R ux, R uy, R uz) {
    const GridArgs<R> &g = a.g;
    R Bx, By, Bz;
    gather4(a.Bnew, g, cx, cy, fx, fy, Bx, By, Bz);
    R val[NMOM];
    particle_moments(a.q, a.m, g.dt, w, ux, uy, uz, Bx, By, Bz, val);
    R W[4] = {(R(1) - fx) * (R(1) - fy), fx * (R(1) - fy), (R(1) - fx) * fy, fx * fy};
    int64_t nd[4] = {node_of(g, cx, cy, 0, 0), node_of(g, cx, cy, 1, 0), node_of(g, cx, cy, 0, 1), node_of(g, cx, cy, 1, 1)};
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < NMOM; ++k) atomicAdd(&a.M[(int64_t)k * g.nnode + nd[c]], W[c] * val[k]);
}

// One thread per particle: gather at r^n, push, move, deposit at r^{n+1}.
// Writes the particle's sort key 2*tile' + (tile' != tile), or dead_key.
template <typename R>
__global__ void k_particle_naive(PArgs<R> a) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_bound) return;
    int64_t n = *a.d_count;
    if (p >= n) {
        a.keys[p] = a.dead_key;
        return;
    }
    const GridArgs<R> &g = a.g;
    int32_t c = a.cell[p];
    int cx = c % g.nx, cy = c / g.nx;
    R fx = a.ox[p], fy = a.oy[p];
    R Ex, Ey, Ez, Bx, By, Bz;
    gather4(a.Ehalf, g, cx, cy, fx, fy, Ex, Ey, Ez);
    gather4(a.Bold, g, cx, cy, fx, fy, Bx, By, Bz);
    R ux = a.ux[p], uy = a.uy[p], uz = a.uz[p];
    R ig = R(1) / sqrt(R(1) + ux * ux + uy * uy + uz * uz);
    R k = a.kq;
    R bx = k * Bx * ig, by = k * By * ig, bz = k * Bz * ig;
    R wx = ux + k * Ex, wy = uy + k * Ey, wz = uz + k * Ez;
    R ubx, uby, ubz;
    rotate(bx, by, bz, wx, wy, wz, ubx, uby, ubz);
    R nux = R(2) * ubx - ux, nuy = R(2) * uby - uy, nuz = R(2) * ubz - uz;
    R sx = fx + a.sdx * ubx * ig, sy = fy + a.sdy * uby * ig;
    R flx = floor(sx), fly = floor(sy);
    R nfx = sx - flx, nfy = sy - fly;
    int ncx = cx + (int)flx, ncy = cy + (int)fly;
    if (nfx >= R(1)) { nfx = R(0); ncx += 1; }
    if (nfy >= R(1)) { nfy = R(0); ncy += 1; }
    if (ncy < 0 || ncy >= g.ny) ncy = ((ncy % g.ny) + g.ny) % g.ny;
    bool dead = false;
    if (g.periodic_x) {
        if (ncx < 0 || ncx >= g.nx) ncx = ((ncx % g.nx) + g.nx) % g.nx;
    } else if (ncx < 0 || ncx >= g.nx) {
        dead = true;
    }
    a.ux[p] = nux;
    a.uy[p] = nuy;
    a.uz[p] = nuz;
    if (dead) {
        a.cell[p] = -1;
        a.keys[p] = a.dead_key;
        atomicAdd(a.d_dead, 1ull);
        atomicAdd(a.d_removed, 1ull);
        return;
    }
    a.cell[p] = ncy * g.nx + ncx;
    a.ox[p] = nfx;
    a.oy[p] = nfy;
    int tx0 = cx / a.tnx, ty0 = cy / a.tny, tx1 = ncx / a.tnx, ty1 = ncy / a.tny;
    uint32_t t0 = (uint32_t)(ty0 * a.ntx + tx0), t1 = (uint32_t)(ty1 * a.ntx + tx1);
    a.keys[p] = 2u * t1 + (t1 != t0 ? 1u : 0u);
    int dtx = abs(tx1 - tx0), dty = abs(ty1 - ty0);
    if ((dtx > 1 && dtx < a.ntx - 1) || (dty > 1 && dty < a.nty - 1)) atomicOr(a.flags, 1);
    deposit_global(a, ncx, ncy, nfx, nfy, a.w[p], nux, nuy, nuz);
}

// Deposit at the current positions with the current node B (after a load or
// a field overwrite).
template <typename R>
__global__ void k_deposit_only(PArgs<R> a) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t n = *a.d_count;
    if (p >= n) return;
    int32_t c = a.cell[p];
    int cx = c % a.g.nx, cy = c / a.g.nx;
    deposit_global(a, cx, cy, a.ox[p], a.oy[p], a.w[p], a.ux[p], a.uy[p], a.uz[p]);
}

// Global positions -> (cell, offset): s = x/dx, cell = floor(s), offset = s - cell
// (a coordinate rounding onto the far edge folds back or stays in the last cell).
template <typename R>
__global__ void k_load_convert(GridArgs<double> g, const double *__restrict__ st, int64_t n, int64_t off,
                               int32_t *cell, R *ox, R *oy, R *ux, R *uy, R *uz, R *w) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double x = st[t], y = st[n + t];
    double sxx = x / g.dx, syy = y / g.dy;
    double flx = floor(sxx), fly = floor(syy);
    int cx = (int)flx, cy = (int)fly;
    double fx = sxx - flx, fy = syy - fly;
    if (cx >= g.nx) { if (g.periodic_x) cx -= g.nx; else { cx = g.nx - 1; fx = 1.0; } }
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
    int64_t d = off + t;
    cell[d] = cy * g.nx + cx;
    ox[d] = rfx;
    oy[d] = rfy;
    ux[d] = (R)st[2 * n + t];
    uy[d] = (R)st[3 * n + t];
    uz[d] = (R)st[4 * n + t];
    w[d] = (R)st[5 * n + t];
}

template <typename R>
__global__ void k_to_stage(GridArgs<double> g, int64_t n, const int32_t *cell, const R *ox, const R *oy, const R *ux,
                           const R *uy, const R *uz, const R *w, double *st) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int32_t c = cell[t];
    int cx = c % g.nx, cy = c / g.nx;
    st[t] = ((double)cx + (double)ox[t]) * g.dx;
    st[n + t] = ((double)cy + (double)oy[t]) * g.dy;
    st[2 * n + t] = (double)ux[t];
    st[3 * n + t] = (double)uy[t];
    st[4 * n + t] = (double)uz[t];
    st[5 * n + t] = (double)w[t];
    ((int32_t *)(st + 6 * n))[t] = c;
}

__global__ void k_tile_keys(const int32_t *cell, int64_t n, int64_t n_bound, int nx, int tnx, int tny, int ntx,
                            uint32_t dead_key, uint32_t *keys) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_bound) return;
    if (t >= n) { keys[t] = dead_key; return; }
    int32_t c = cell[t];
    int cx = c % nx, cy = c / nx;
    keys[t] = 2u * (uint32_t)((cy / tny) * ntx + cx / tnx);
}

// --------------------------------------------------------------------------- host side

template <typename R>
static PArgs<R> make_args(pic_t *h, int s) {
    SpeciesBuf &S = h->sp[s];
    PArgs<R> a;
    a.g = grid_args<R>(h);
    int c = S.cur;
    a.cell = S.cell[c];
    a.ox = (R *)S.ox[c]; a.oy = (R *)S.oy[c];
    a.ux = (R *)S.ux[c]; a.uy = (R *)S.uy[c]; a.uz = (R *)S.uz[c];
    a.w = (const R *)S.w[c];
    a.Ehalf = (const V4<R> *)h->Ehalf;
    a.Bold = (const V4<R> *)h->B[h->bcur];
    a.Bnew = (const V4<R> *)h->B[1 - h->bcur];
    a.M = (R *)h->M;
    a.keys = h->keys[0];
    a.d_count = h->d_count + s;
    a.d_dead = (unsigned long long *)(h->d_dead + s);
    a.d_removed = (unsigned long long *)(h->d_removed + s);
    a.flags = h->d_flags;
    a.n_bound = S.n;
    a.q = (R)S.q; a.m = (R)S.m;
    a.kq = (R)(S.q * h->cfg.dt / (2.0 * S.m));
    a.sdx = (R)(h->cfg.dt / h->cfg.dx);
    a.sdy = (R)(h->cfg.dt / h->cfg.dy);
    a.tnx = h->tnx; a.tny = h->tny; a.ntx = h->ntx; a.nty = h->nty;
    a.dead_key = (uint32_t)(2 * h->ntiles + 2);
    return a;
}

template <typename R>
static int particle_step_t(pic_t *h, int s) {
    PArgs<R> a = make_args<R>(h, s);
    if (a.n_bound == 0) return 0;
    k_particle_naive<R><<<(unsigned)((a.n_bound + 255) / 256), 256, 0, h->st>>>(a);
    count_launch(h);
    return check_launch("k_particle_naive");
}

int particle_step(pic_t *h, int s) { return h->fp32 ? particle_step_t<float>(h, s) : particle_step_t<double>(h, s); }

template <typename R>
static int deposit_only_t(pic_t *h, int s) {
    PArgs<R> a = make_args<R>(h, s);
    a.Bnew = (const V4<R> *)h->B[h->bcur];  // moments of the current state use the current B
    if (a.n_bound == 0) return 0;
    k_deposit_only<R><<<(unsigned)((a.n_bound + 255) / 256), 256, 0, h->st>>>(a);
    count_launch(h);
    return check_launch("k_deposit_only");
}

int deposit_only(pic_t *h, int s) { return h->fp32 ? deposit_only_t<float>(h, s) : deposit_only_t<double>(h, s); }

int clear_moments(pic_t *h) {
    if (cudaMemsetAsync(h->M, 0, (size_t)NMOM * h->nnode * h->rs, h->st) != cudaSuccess) return check_launch("clear M");
    return 0;
}

template <typename R>
static int load_convert_t(pic_t *h, int s, int64_t off, int64_t n) {
    SpeciesBuf &S = h->sp[s];
    int c = S.cur;
    k_load_convert<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(grid_args<double>(h), h->stage, n, off, S.cell[c],
                                                                      (R *)S.ox[c], (R *)S.oy[c], (R *)S.ux[c],
                                                                      (R *)S.uy[c], (R *)S.uz[c], (R *)S.w[c]);
    count_launch(h);
    return check_launch("k_load_convert");
}

int load_convert(pic_t *h, int s, int64_t off, int64_t n) {
    return h->fp32 ? load_convert_t<float>(h, s, off, n) : load_convert_t<double>(h, s, off, n);
}

template <typename R>
static int to_stage_t(pic_t *h, int s, int64_t n) {
    SpeciesBuf &S = h->sp[s];
    int c = S.cur;
    k_to_stage<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(grid_args<double>(h), n, S.cell[c], (const R *)S.ox[c],
                                                                  (const R *)S.oy[c], (const R *)S.ux[c],
                                                                  (const R *)S.uy[c], (const R *)S.uz[c],
                                                                  (const R *)S.w[c], h->stage);
    count_launch(h);
    return check_launch("k_to_stage");
}

int particles_to_stage(pic_t *h, int s, int64_t n) {
    if (n == 0) return 0;
    return h->fp32 ? to_stage_t<float>(h, s, n) : to_stage_t<double>(h, s, n);
}

int tile_keys(pic_t *h, int s, int64_t n) {
    SpeciesBuf &S = h->sp[s];
    if (S.n == 0) return 0;
    k_tile_keys<<<(unsigned)((S.n + 255) / 256), 256, 0, h->st>>>(S.cell[S.cur], n, S.n, h->nx, h->tnx, h->tny, h->ntx,
                                                                  (uint32_t)(2 * h->ntiles + 2), h->keys[0]);
    count_launch(h);
    return check_launch("k_tile_keys");
}

}  // namespace pic
