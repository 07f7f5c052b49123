// Tiled particle step (Section 3.3 "forces, pusher, current"), one CTA per
// tile of cells:
//   * E^{n+1/2}, the push B and the deposit B of the tile (the deposit one with
//     a halo of H cells) are copied into shared memory by TMA;
//   * every particle of the tile is gathered, pushed and moved (Eq. 2 with E
//     factored out), then its 13 moments (Eq. 3) are added into a shared-memory
//     accumulator covering the tile plus halo: warps whose lanes share a cell
//     reduce their 52 corner products with a butterfly reduce-scatter first,
//     the rest add per lane; the accumulator is flushed to the global moments
//     once per tile (FP32: with a TwoSum compensation term);
//   * particles that stay are compacted in place in the tile's bin (stable);
//     leavers go, in order, to the tile's bin of a mirror array;
// then k_append gives every tile the leavers of its eight neighbour tiles
// that moved into it, in ascending source-tile order.  The result is the
// library's particle order (stayers first, then arrivals, each in previous
// order).  A bin overflow or a move farther than one tile sets a flag; the
// host then regroups that species with the full stable sort before the next
// push (pic_sort.cu).
#include <cuda.h>

#include "pic_internal.cuh"

namespace pic {

// --------------------------------------------------------------------------- TMA / mbarrier

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ inline void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ inline void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ inline void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// --------------------------------------------------------------------------- arguments

template <typename R>
struct SpPtr {
    int32_t *cell, *mcell;
    R *ox, *oy, *ux, *uy, *uz, *w;
    R *mox, *moy, *mux, *muy, *muz, *mw;
    uint32_t *mkey;
    const int32_t *bstart;
    int32_t *bcount, *nstay, *nleave;
    unsigned long long *removed;
    R q, m, kq;
};

template <typename R>
struct TileArgs {
    GridArgs<R> g;
    int tnx, tny, ntx, nty, ntiles, H;
    int EW, EH, RW, RH;             // node extents of the push tile and of the deposit region
    int offBo, offBn, offAcc, offBar, offScr;  // shared-memory carve (bytes)
    uint32_t tma_bytes;
    int nsp;
    SpPtr<R> sp[PIC_MAX_SPECIES];
    R sdx, sdy;
    R *M, *Mlo;
    const V4<R> *Bnew;              // padded global deposit B (escapes)
    int32_t *step_flags, *flags;
};

constexpr int TILE_BS = 256;
constexpr int TILE_WARPS = TILE_BS / 32;
constexpr unsigned FULL = 0xffffffffu;
constexpr int MIN_GROUP = 6;        // lanes sharing a cell before the butterfly pays off

__device__ inline int imod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Is tile (bx, by) one of the 3x3 tiles around (ax, ay)?
__device__ inline bool tile_near(int ax, int ay, int bx, int by, int ntx, int nty, bool periodic_x) {
    int dx = bx - ax, dy = imod(by - ay, nty);
    bool oky = (dy == 0 || dy == 1 || dy == nty - 1);
    bool okx;
    if (periodic_x) {
        int d = imod(dx, ntx);
        okx = (d == 0 || d == 1 || d == ntx - 1);
    } else {
        okx = (dx >= -1 && dx <= 1);
    }
    return okx && oky;
}

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
        a[j] = k + __shfl_xor_sync(FULL, s, 16);
    }
    a[13] = R(0);
    R c[8];
    b = (lane & 8) != 0;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
        R lo = a[j], hi = a[j + 7];
        R s = b ? lo : hi, k = b ? hi : lo;
        c[j] = k + __shfl_xor_sync(FULL, s, 8);
    }
    c[7] = R(0);
    R d[4];
    b = (lane & 4) != 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        R lo = c[j], hi = c[j + 4];
        R s = b ? lo : hi, k = b ? hi : lo;
        d[j] = k + __shfl_xor_sync(FULL, s, 4);
    }
    R e[2];
    b = (lane & 2) != 0;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        R lo = d[j], hi = d[j + 2];
        R s = b ? lo : hi, k = b ? hi : lo;
        e[j] = k + __shfl_xor_sync(FULL, s, 2);
    }
    b = (lane & 1) != 0;
    R s = b ? e[0] : e[1], k = b ? e[1] : e[0];
    return k + __shfl_xor_sync(FULL, s, 1);
}

__device__ inline int rs26_index(int lane) {
    int j2 = (lane & 1) + 2 * ((lane >> 1) & 1) + 4 * ((lane >> 2) & 1);
    if (j2 >= 7) return -1;
    int j1 = j2 + 7 * ((lane >> 3) & 1);
    if (j1 >= 13) return -1;
    return j1 + 13 * ((lane >> 4) & 1);
}

// Add the 13 moments of each lane's particle, weighted onto the four corners
// of its region cell, to the shared accumulator acc[k * RN + node].  key is the
// region node index of the cell's lower-left corner, or -1 (nothing to add).
// Called by all 32 lanes of the warp.
template <typename R>
__device__ inline void warp_deposit(R *acc, int RN, int RW, int key, const R *val, R fx, R fy) {
    const int lane = threadIdx.x & 31;
    const R W[4] = {(R(1) - fx) * (R(1) - fy), fx * (R(1) - fy), (R(1) - fx) * fy, fx * fy};
    unsigned active = __ballot_sync(FULL, key >= 0);
    while (active) {
        int leader = __ffs(active) - 1;
        int kl = __shfl_sync(FULL, key, leader);
        unsigned members = __ballot_sync(FULL, key == kl);
        if (__popc(members) >= MIN_GROUP) {
            bool mem = (key == kl);
            int idx = rs26_index(lane);
#pragma unroll
            for (int pass = 0; pass < 2; ++pass) {
                R v[26];
#pragma unroll
                for (int c2 = 0; c2 < 2; ++c2)
#pragma unroll
                    for (int k = 0; k < NMOM; ++k) v[c2 * NMOM + k] = mem ? W[2 * pass + c2] * val[k] : R(0);
                R r = reduce_scatter26(v, lane);
                if (idx >= 0 && r != R(0)) {
                    int corner = 2 * pass + idx / NMOM, k = idx % NMOM;
                    atomicAdd(&acc[k * RN + kl + (corner & 1) + (corner >> 1) * RW], r);
                }
            }
            active &= ~members;
        } else {
            if (active & (1u << lane)) {
                const int nd[4] = {key, key + 1, key + RW, key + RW + 1};
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int k = 0; k < NMOM; ++k) atomicAdd(&acc[k * RN + nd[c]], W[c] * val[k]);
            }
            active = 0;
        }
    }
}

// Block-wide exclusive prefix of two flags; returns the per-thread prefixes and
// the block totals.  Uses scr[0 .. 2*TILE_WARPS).
__device__ inline void block_prefix2(bool f0, bool f1, int *scr, int &p0, int &p1, int &t0, int &t1) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned b0 = __ballot_sync(FULL, f0), b1 = __ballot_sync(FULL, f1);
    if (lane == 0) {
        scr[wid] = __popc(b0);
        scr[TILE_WARPS + wid] = __popc(b1);
    }
    __syncthreads();
    p0 = p1 = t0 = t1 = 0;
#pragma unroll
    for (int w = 0; w < TILE_WARPS; ++w) {
        int a = scr[w], b = scr[TILE_WARPS + w];
        if (w < wid) {
            p0 += a;
            p1 += b;
        }
        t0 += a;
        t1 += b;
    }
    unsigned lt = (1u << lane) - 1u;
    p0 += __popc(b0 & lt);
    p1 += __popc(b1 & lt);
}

template <typename R>
__device__ inline void sm_gather(const V4<R> *F, int W, int lx, int ly, R fx, R fy, R &ox, R &oy, R &oz) {
    const V4<R> a = F[ly * W + lx], b = F[ly * W + lx + 1], c = F[(ly + 1) * W + lx], d = F[(ly + 1) * W + lx + 1];
    R w00 = (R(1) - fx) * (R(1) - fy), w10 = fx * (R(1) - fy), w01 = (R(1) - fx) * fy, w11 = fx * fy;
    ox = w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x;
    oy = w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y;
    oz = w00 * a.z + w10 * b.z + w01 * c.z + w11 * d.z;
}

template <typename R>
__global__ void __launch_bounds__(TILE_BS) k_particle_tile(const TileArgs<R> a, const __grid_constant__ CUtensorMap tmE,
                                                           const __grid_constant__ CUtensorMap tmBo,
                                                           const __grid_constant__ CUtensorMap tmBn) {
    extern __shared__ __align__(128) unsigned char smem[];
    const GridArgs<R> &g = a.g;
    const int t = blockIdx.x;
    const int tid = threadIdx.x;
    int total = 0;
    for (int s = 0; s < a.nsp; ++s) total += a.sp[s].bcount[t];
    if (total == 0) {
        if (tid < a.nsp) {
            a.sp[tid].nstay[t] = 0;
            a.sp[tid].nleave[t] = 0;
        }
        return;
    }
    const int tx = t % a.ntx, ty = t / a.ntx;
    const int X0 = tx * a.tnx, Y0 = ty * a.tny;
    V4<R> *sE = (V4<R> *)smem;
    V4<R> *sBo = (V4<R> *)(smem + a.offBo);
    V4<R> *sBn = (V4<R> *)(smem + a.offBn);
    R *acc = (R *)(smem + a.offAcc);
    uint64_t *bar = (uint64_t *)(smem + a.offBar);
    int *scr = (int *)(smem + a.offScr);
    const int RN = a.RW * a.RH;
    const int H = a.H;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, a.tma_bytes);
        tma_load_3d(sE, &tmE, 0, X0 + g.G, Y0 + g.G, bar);
        tma_load_3d(sBo, &tmBo, 0, X0 + g.G, Y0 + g.G, bar);
        tma_load_3d(sBn, &tmBn, 0, X0 + g.G - H, Y0 + g.G - H, bar);
    }
    for (int i = tid; i < NMOM * RN; i += TILE_BS) acc[i] = R(0);
    // one thread waits for the copies (bounded), the barrier publishes them
    if (tid == 0) {
        bool ok = false;
        for (int it = 0; it < (1 << 22) && !ok; ++it) ok = mbar_try_wait(bar, 0);
        if (!ok) {
            // record the timeout and give the copies one more bounded wait so
            // that none lands after this block has left
            atomicOr(a.flags, 8);
            for (int it = 0; it < (1 << 22) && !ok; ++it) ok = mbar_try_wait(bar, 0);
        }
        scr[0] = ok ? 1 : 0;
    }
    __syncthreads();
    if (scr[0] == 0) return;
    __syncthreads();

    const int RWc = a.RW - 1, RHc = a.RH - 1;  // region cells per row / column
    for (int s = 0; s < a.nsp; ++s) {
        const SpPtr<R> &P = a.sp[s];
        const int cnt = P.bcount[t];
        const int64_t b0 = P.bstart[t];
        int nst = 0, nlv = 0;
        for (int off = 0; off < cnt; off += TILE_BS) {
            const int i = off + tid;
            bool valid = i < cnt;
            const int64_t slot = b0 + i;
            int32_t c = 0;
            R fx = R(0), fy = R(0), ux = R(0), uy = R(0), uz = R(0), w = R(0);
            if (valid) {
                c = P.cell[slot];
                fx = P.ox[slot];
                fy = P.oy[slot];
                ux = P.ux[slot];
                uy = P.uy[slot];
                uz = P.uz[slot];
                w = P.w[slot];
            }
            const int cx = c % g.nx, cy = c / g.nx;
            int lx = cx - X0, ly = cy - Y0;
            if (valid && (lx < 0 || lx >= a.tnx || ly < 0 || ly >= a.tny)) {
                atomicOr(a.flags, 16);  // particle outside its bin's tile: skip it
                valid = false;
            }
            if (!valid) lx = ly = 0;
            // gather at r^n (Section 3.3: forces)
            R Ex, Ey, Ez, Bx, By, Bz;
            sm_gather(sE, a.EW, lx, ly, fx, fy, Ex, Ey, Ez);
            sm_gather(sBo, a.EW, lx, ly, fx, fy, Bx, By, Bz);
            // implicit push (Eq. 2, E factored out)
            const R ig = R(1) / sqrt(R(1) + ux * ux + uy * uy + uz * uz);
            const R k = P.kq;
            const R bx = k * Bx * ig, by = k * By * ig, bz = k * Bz * ig;
            R ubx, uby, ubz;
            rotate(bx, by, bz, ux + k * Ex, uy + k * Ey, uz + k * Ez, ubx, uby, ubz);
            const R nux = R(2) * ubx - ux, nuy = R(2) * uby - uy, nuz = R(2) * ubz - uz;
            // move in cell units
            const R sx = fx + a.sdx * ubx * ig, sy = fy + a.sdy * uby * ig;
            const R flx = floor(sx), fly = floor(sy);
            R nfx = sx - flx, nfy = sy - fly;
            int shx = (int)flx, shy = (int)fly;
            if (nfx >= R(1)) { nfx = R(0); shx += 1; }
            if (nfy >= R(1)) { nfy = R(0); shy += 1; }
            const int ncxu = cx + shx, ncyu = cy + shy;
            const int ncy = imod(ncyu, g.ny);
            int ncx = ncxu;
            bool dead = false;
            if (g.periodic_x) ncx = imod(ncxu, g.nx);
            else if (ncxu < 0 || ncxu >= g.nx) dead = true;
            const bool alive = valid && !dead;
            const int ttx = alive ? ncx / a.tnx : tx, tty = alive ? ncy / a.tny : ty;
            const int tn = tty * a.ntx + ttx;
            const bool stay = alive && tn == t;
            const bool leave = alive && tn != t;
            if (leave && !tile_near(tx, ty, ttx, tty, a.ntx, a.nty, g.periodic_x)) {
                atomicOr(a.step_flags, 1);
                atomicOr(a.flags, 1);
            }
            // deposit at r^{n+1} with the new B (Eq. 3)
            const int rx = lx + shx + H, ry = ly + shy + H;
            const bool inreg = alive && rx >= 0 && rx < RWc && ry >= 0 && ry < RHc;
            R nBx = R(0), nBy = R(0), nBz = R(0);
            if (inreg) sm_gather(sBn, a.RW, rx, ry, nfx, nfy, nBx, nBy, nBz);
            else if (alive) gather4(a.Bnew, g, ncx, ncy, nfx, nfy, nBx, nBy, nBz);
            R val[NMOM];
            particle_moments(P.q, P.m, g.dt, w, nux, nuy, nuz, nBx, nBy, nBz, val);
            warp_deposit(acc, RN, a.RW, inreg ? ry * a.RW + rx : -1, val, nfx, nfy);
            if (alive && !inreg) {
                const R Wg[4] = {(R(1) - nfx) * (R(1) - nfy), nfx * (R(1) - nfy), (R(1) - nfx) * nfy, nfx * nfy};
                const int64_t nd[4] = {node_of(g, ncx, ncy, 0, 0), node_of(g, ncx, ncy, 1, 0), node_of(g, ncx, ncy, 0, 1),
                                       node_of(g, ncx, ncy, 1, 1)};
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
#pragma unroll
                    for (int kk = 0; kk < NMOM; ++kk) atomicAdd(&a.M[(int64_t)kk * g.nnode + nd[cc]], Wg[cc] * val[kk]);
            }
            // stable compaction (all loads of this chunk are done after the barrier inside)
            int ps, pl, ts, tl;
            block_prefix2(stay, leave, scr, ps, pl, ts, tl);
            const int32_t ncell = ncy * g.nx + ncx;
            if (stay) {
                const int64_t d = b0 + nst + ps;
                P.cell[d] = ncell;
                P.ox[d] = nfx;
                P.oy[d] = nfy;
                P.ux[d] = nux;
                P.uy[d] = nuy;
                P.uz[d] = nuz;
                P.w[d] = w;
            } else if (leave) {
                const int64_t d = b0 + nlv + pl;
                P.mcell[d] = ncell;
                P.mox[d] = nfx;
                P.moy[d] = nfy;
                P.mux[d] = nux;
                P.muy[d] = nuy;
                P.muz[d] = nuz;
                P.mw[d] = w;
                P.mkey[d] = (uint32_t)tn;
            } else if (valid && dead) {
                atomicAdd(P.removed, 1ull);
            }
            nst += ts;
            nlv += tl;
            __syncthreads();
        }
        if (tid == 0) {
            P.nstay[t] = nst;
            P.nleave[t] = nlv;
        }
    }
    __syncthreads();
    // flush the tile + halo accumulator
    for (int idx = tid; idx < NMOM * RN; idx += TILE_BS) {
        const R v = acc[idx];
        if (v == R(0)) continue;
        const int k = idx / RN, r = idx - k * RN;
        const int ryn = r / a.RW, rxn = r - ryn * a.RW;
        int gx = X0 - H + rxn;
        const int gy = imod(Y0 - H + ryn, g.ny);
        if (g.periodic_x) gx = imod(gx, g.nx);
        else if (gx < 0 || gx >= g.nxn) continue;
        const int64_t gi = (int64_t)k * g.nnode + (int64_t)gy * g.nxn + gx;
        if (a.Mlo) {
            const R old = atomicAdd(&a.M[gi], v);
            const R sum = old + v;
            const R bb = sum - old;
            const R err = (old - (sum - bb)) + (v - bb);
            if (err != R(0)) atomicAdd(&a.Mlo[gi], err);
        } else {
            atomicAdd(&a.M[gi], v);
        }
    }
}

// Each tile takes, from the mirror bins of its (up to eight) neighbour tiles in
// ascending tile order, the leavers that moved into it and appends them after
// its stayers.
template <typename R>
__global__ void __launch_bounds__(TILE_BS) k_append(const TileArgs<R> a) {
    __shared__ int nb[8];
    __shared__ int nnb;
    __shared__ int scr[2 * TILE_WARPS];
    const int t = blockIdx.x, s = blockIdx.y;
    const int tid = threadIdx.x;
    const SpPtr<R> &P = a.sp[s];
    const bool px = a.g.periodic_x != 0;
    if (tid == 0) {
        const int tx = t % a.ntx, ty = t / a.ntx;
        int n = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                int x = tx + dx;
                if (px) x = imod(x, a.ntx);
                else if (x < 0 || x >= a.ntx) continue;
                int y = imod(ty + dy, a.nty);
                int id = y * a.ntx + x;
                if (id == t) continue;
                bool dup = false;
                for (int q = 0; q < n; ++q) dup |= (nb[q] == id);
                if (!dup) nb[n++] = id;
            }
        for (int i = 1; i < n; ++i)  // ascending
            for (int j = i; j > 0 && nb[j - 1] > nb[j]; --j) {
                int tmp = nb[j];
                nb[j] = nb[j - 1];
                nb[j - 1] = tmp;
            }
        nnb = n;
    }
    __syncthreads();
    const int64_t base = P.bstart[t];
    const int capt = P.bstart[t + 1] - P.bstart[t];
    int pos = P.nstay[t];
    bool over = false;
    for (int q = 0; q < nnb; ++q) {
        const int src = nb[q];
        const int64_t sb = P.bstart[src];
        const int nl = P.nleave[src];
        for (int off = 0; off < nl; off += TILE_BS) {
            const int i = off + tid;
            const bool mine = (i < nl) && P.mkey[sb + i] == (uint32_t)t;
            int pm, pdummy, tm, tdummy;
            block_prefix2(mine, false, scr, pm, pdummy, tm, tdummy);
            if (mine) {
                const int dst = pos + pm;
                if (dst < capt) {
                    const int64_t d = base + dst, si = sb + i;
                    P.cell[d] = P.mcell[si];
                    P.ox[d] = P.mox[si];
                    P.oy[d] = P.moy[si];
                    P.ux[d] = P.mux[si];
                    P.uy[d] = P.muy[si];
                    P.uz[d] = P.muz[si];
                    P.w[d] = P.mw[si];
                }
            }
            pos += tm;
            over |= (pos > capt);
            __syncthreads();
        }
    }
    if (tid == 0) {
        if (over) atomicOr(a.step_flags, 2);
        P.bcount[t] = over ? P.nstay[t] : pos;
    }
}

// --------------------------------------------------------------------------- host side

struct TMaps {
    CUtensorMap m[3];   // E^{n+1/2}, B[0], B[1]
    int boxE[2], boxB[2];
};

// cuTensorMapEncodeTiled is taken from the driver at run time, so that the
// library loads (for its CPU checks) on machines without a CUDA driver.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

static int make_map(CUtensorMap *m, void *base, bool fp32, int nxp, int nyp, int bw, int bh) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return PIC_ERR_CUDA;
    }
    cuuint64_t dims[3] = {4, (cuuint64_t)nxp, (cuuint64_t)nyp};
    size_t es = fp32 ? 4 : 8;
    cuuint64_t strides[2] = {4 * es, 4 * es * (cuuint64_t)nxp};
    cuuint32_t box[3] = {4, (cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                                        base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with CUresult %d", (int)r);
        return PIC_ERR_CUDA;
    }
    return 0;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Carve {
    int offBo, offBn, offAcc, offBar, offScr, bytes;
    uint32_t tma_bytes;
};

static Carve carve(const pic_t *h) {
    size_t v4 = 4 * h->rs;
    int EW = h->tnx + 1, EH = h->tny + 1, RW = h->tnx + 2 * h->halo + 1, RH = h->tny + 2 * h->halo + 1;
    Carve c;
    size_t o = align_up(EW * EH * v4, 128);
    c.offBo = (int)o;
    o += align_up(EW * EH * v4, 128);
    c.offBn = (int)o;
    o += align_up(RW * RH * v4, 128);
    c.offAcc = (int)o;
    o += align_up((size_t)NMOM * RW * RH * h->rs, 16);
    c.offBar = (int)o;
    o += 16;
    c.offScr = (int)o;
    o += 2 * TILE_WARPS * sizeof(int);
    c.bytes = (int)align_up(o, 128);
    c.tma_bytes = (uint32_t)((2 * EW * EH + RW * RH) * v4);
    return c;
}

int tile_setup(pic_t *h) {
    int RW = h->tnx + 2 * h->halo + 1, RH = h->tny + 2 * h->halo + 1;
    if (RW > 256 || RH > 256) {
        set_error("tile %dx%d with halo %d exceeds the 256-node TMA box", h->tnx, h->tny, h->halo);
        return PIC_ERR_ARG;
    }
    Carve c = carve(h);
    if (c.bytes > 220 * 1024) {
        set_error("tile %dx%d needs %d bytes of shared memory", h->tnx, h->tny, c.bytes);
        return PIC_ERR_ARG;
    }
    TMaps *tm = new TMaps();
    int rc = make_map(&tm->m[0], h->Ehalf, h->fp32, h->nxp, h->nyp, h->tnx + 1, h->tny + 1);
    if (!rc) rc = make_map(&tm->m[1], h->B[0], h->fp32, h->nxp, h->nyp, h->tnx + 1, h->tny + 1);
    if (!rc) rc = make_map(&tm->m[2], h->B[1], h->fp32, h->nxp, h->nyp, h->tnx + 1, h->tny + 1);
    // deposit-B maps (bigger box) for B[0], B[1]
    CUtensorMap *dep = new CUtensorMap[2];
    if (!rc) rc = make_map(&dep[0], h->B[0], h->fp32, h->nxp, h->nyp, RW, RH);
    if (!rc) rc = make_map(&dep[1], h->B[1], h->fp32, h->nxp, h->nyp, RW, RH);
    if (rc) {
        delete tm;
        delete[] dep;
        return rc;
    }
    struct Both {
        TMaps *a;
        CUtensorMap *b;
    };
    Both *both = new Both{tm, dep};
    h->tmaps = both;
    cudaError_t e;
    if (h->fp32)
        e = cudaFuncSetAttribute(k_particle_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, c.bytes);
    else
        e = cudaFuncSetAttribute(k_particle_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, c.bytes);
    if (e != cudaSuccess) {
        set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return 0;
}

void tile_free(pic_t *h) {
    struct Both {
        TMaps *a;
        CUtensorMap *b;
    };
    Both *both = (Both *)h->tmaps;
    if (both) {
        delete both->a;
        delete[] both->b;
        delete both;
    }
    h->tmaps = nullptr;
}

template <typename R>
static TileArgs<R> tile_args(pic_t *h) {
    TileArgs<R> a;
    a.g = grid_args<R>(h);
    a.tnx = h->tnx; a.tny = h->tny; a.ntx = h->ntx; a.nty = h->nty; a.ntiles = h->ntiles; a.H = h->halo;
    a.EW = h->tnx + 1; a.EH = h->tny + 1;
    a.RW = h->tnx + 2 * h->halo + 1; a.RH = h->tny + 2 * h->halo + 1;
    Carve c = carve(h);
    a.offBo = c.offBo; a.offBn = c.offBn; a.offAcc = c.offAcc; a.offBar = c.offBar; a.offScr = c.offScr;
    a.tma_bytes = c.tma_bytes;
    a.nsp = h->nsp;
    for (int s = 0; s < h->nsp; ++s) {
        SpeciesBuf &S = h->sp[s];
        SpPtr<R> &p = a.sp[s];
        int b = S.bins, m = S.mir;
        p.cell = S.cell[b]; p.ox = (R *)S.ox[b]; p.oy = (R *)S.oy[b];
        p.ux = (R *)S.ux[b]; p.uy = (R *)S.uy[b]; p.uz = (R *)S.uz[b]; p.w = (R *)S.w[b];
        p.mcell = S.cell[m]; p.mox = (R *)S.ox[m]; p.moy = (R *)S.oy[m];
        p.mux = (R *)S.ux[m]; p.muy = (R *)S.uy[m]; p.muz = (R *)S.uz[m]; p.mw = (R *)S.w[m];
        p.mkey = S.mkey;
        p.bstart = S.bstart; p.bcount = S.bcount; p.nstay = S.nstay; p.nleave = S.nleave;
        p.removed = (unsigned long long *)(h->d_removed + s);
        p.q = (R)S.q; p.m = (R)S.m; p.kq = (R)(S.q * h->cfg.dt / (2.0 * S.m));
    }
    a.sdx = (R)(h->cfg.dt / h->cfg.dx);
    a.sdy = (R)(h->cfg.dt / h->cfg.dy);
    a.M = (R *)h->M;
    a.Mlo = (R *)h->Mlo;
    a.Bnew = (const V4<R> *)h->B[1 - h->bcur];
    a.step_flags = h->d_step_flags;
    a.flags = h->d_flags;
    return a;
}

template <typename R>
static int particle_tiles_t(pic_t *h) {
    struct Both {
        TMaps *a;
        CUtensorMap *b;
    };
    Both *both = (Both *)h->tmaps;
    TileArgs<R> a = tile_args<R>(h);
    Carve c = carve(h);
    const CUtensorMap &mE = both->a->m[0];
    const CUtensorMap &mBo = both->a->m[1 + h->bcur];
    const CUtensorMap &mBn = both->b[1 - h->bcur];
    k_particle_tile<R><<<h->ntiles, TILE_BS, c.bytes, h->st>>>(a, mE, mBo, mBn);
    count_launch(h);
    return check_launch("k_particle_tile");
}

int particle_tiles(pic_t *h) { return h->fp32 ? particle_tiles_t<float>(h) : particle_tiles_t<double>(h); }

template <typename R>
static int append_t(pic_t *h) {
    TileArgs<R> a = tile_args<R>(h);
    k_append<R><<<dim3(h->ntiles, h->nsp), TILE_BS, 0, h->st>>>(a);
    count_launch(h);
    return check_launch("k_append");
}

int append_arrivals(pic_t *h) { return h->fp32 ? append_t<float>(h) : append_t<double>(h); }

}  // namespace pic
