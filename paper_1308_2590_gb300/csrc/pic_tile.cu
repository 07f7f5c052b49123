// Tiled particle step (Section 3.3 "forces, pusher, current").
//
// k_push: a persistent grid takes work items (species, tile, run of
// segments) from a queue.  For each item the tile's E^{n+1/2}, push B and
// deposit B (with a halo of H cells) are copied into shared memory by TMA;
// each warp then takes whole 32-slot segments of the tile's bin: gather,
// implicit push (Eq. 2 with E factored out), move, and the 13 moments of Eq. 3.
// The FP64 form first turns both tiles into per-cell coefficients of the
// bilinear weighting (cell_coef), so that a gather is three FMAs per component.
// FP32 deposit: every lane keeps, in registers, the 52 corner products of its
// particles in the warp's current cell K; a segment's lanes in K add there,
// and a further cell with at least MIN_GROUP of the segment's lanes becomes K
// after K is flushed (butterfly reduce-scatter over the warp into the shared
// accumulator over tile + halo), up to three cells per segment.  The few lanes
// left over add their own products to the global moments by L2 reductions.
// The accumulator goes to the global moments once per item (with a TwoSum
// compensation term).  FP64 deposit: per-lane
// reductions in L2.  The warp compacts the segment's stayers in place with one
// ballot and writes its leavers, in order, to the same segment of a mirror
// array.  No block-wide barrier sits inside the particle loop.
//
// k_regroup: every tile sorts its stayers and the leavers of its (up to
// eight) neighbour tiles that moved into it, stably by cell, into the spare
// buffer set.  This is the library's particle order: tiles ascending, cells
// row-major inside a tile, inside a cell the stayers in their order and then
// the arrivals in their previous order.  Since the bins are in cell order at
// every push, a warp's segments mostly lie in one or two cells.  A bin
// without room, or a move farther than one tile, sets a flag; the host then
// regroups the species with the full stable sort (pic_sort.cu) before the
// next push.
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <vector>

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

// Poll an mbarrier phase until it completes, for at most WAIT_LIMIT_NS of the
// global timer and at most 2^22 polls (one poll suspends for a few
// microseconds), whichever ends first; false if the wait ran out.
constexpr uint64_t WAIT_LIMIT_NS = 1000000000ull;
__device__ inline uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ inline bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return false;
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
    int32_t *useg, *segn, *segml;   // current counts (push reads/writes, the regroup reads)
    int32_t *useg2, *segn2;         // next counts (the regroup writes)
    int32_t *ocell;                 // spare set: the regroup's output
    R *oox, *ooy, *oux, *ouy, *ouz, *ow;
    unsigned long long *removed;
    R q, m, kq, cq2, hq;
    double *cr, *mcr, *ocr;         // FP64 form: carried quantities of bins, mirror, spare ([NCARRY][ccap])
    int64_t ccap;
};

template <typename R>
struct TileArgs {
    GridArgs<R> g;
    int tnx, tny, ntx, nty, ntiles, H;
    int EW, EH, RW, RH;             // node extents of the push tile and of the deposit region
    int offBo, offBn, offAcc, offBar, offScr;  // shared-memory carve (bytes); the fields start at SMEM_HEADER
    int offCanary;                  // checks build: four canary words after the accumulator
    int offQ;                       // FP32: the warps' straggler queues (QCAP entries of QWORDS words each)
    int offEc, offBc;               // FP64: cell coefficients of the E tile and of the deposit region
    uint32_t tma_bytes;
    int nsp;
    SpPtr<R> sp[PIC_MAX_SPECIES];
    R sdx, sdy;
    uint32_t magic_nx;              // ceil(2^32 / nx)
    R *M, *Mlo;
    double *Mc;                     // FP64 L2-reduction push: cell sums (deposit_fp64_cell)
    unsigned long long *Mfix;       // deterministic deposit: fixed-point sums
    FixScale fs;
    const V4<R> *Bnew;              // padded global deposit B (escapes; the batched push's deposit tile)
    const V4<R> *Eh, *Bo;           // padded E^{n+1/2} and push B (the batched push loads its tiles from them)
    int32_t *step_flags, *flags;
    const int32_t *guard;           // the previous step's flags (set: this step's kernels do nothing for the run)
    const int32_t *chunk_prefix;    // [nsp*ntiles + 1]
    const int2 *items;              // item -> (species-tile index, run within it); single-run launches
    const int32_t *nbr;             // [ntiles][9]: neighbour count, then the neighbour tiles ascending
    int32_t *ticket;
    int ch;                         // segments per work item
    const int32_t *rg_list;         // tiles the regroup visits (single-run launches)
    int32_t *list_n;                // [1]: entries of rg_list; [2 + s]: the regroup's queue counter of species s
};

// Segments per work item.  FP32: a whole tile of the bench workload (the
// item's shared accumulator flush is paid once per item).  FP64: shorter
// items (the deposit goes to L2, an item costs its field copies and
// coefficient tables), so that the queue's last items leave fewer blocks idle
// (32, 48, 64, 128 segments: 1.857, 1.845, 1.857, 1.922 ms per push on the
// 1024 x 512 foil).  Spline shapes: FP64 and degree 2 FP32 as short items.
constexpr int CH_SEGS_FP32 = 256;
constexpr int CH_SEGS_FP64 = 48;
constexpr int CH_SEGS_SPLINE = 32;
inline int item_segs(const pic_t *h) {
    if (h->fp32 && h->shape != 2) return CH_SEGS_FP32;
    return h->shape == 1 ? CH_SEGS_FP64 : CH_SEGS_SPLINE;
}

// Shared memory of the push: a fixed header (mbarrier, then the block's
// scratch words) at the same place for every run of a batch, then the
// tile's fields and the moment accumulator.
constexpr int SMEM_HEADER = 128;

constexpr int TILE_BS = 256;
constexpr int TILE_WARPS = TILE_BS / 32;
constexpr unsigned FULL = 0xffffffffu;
constexpr int MIN_GROUP = 2;        // lanes sharing a cell for a further register pass

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

template <typename R>
__device__ inline void sm_gather(const V4<R> *F, int W, int lx, int ly, R fx, R fy, R &ox, R &oy, R &oz) {
    const V4<R> a = F[ly * W + lx], b = F[ly * W + lx + 1], c = F[(ly + 1) * W + lx], d = F[(ly + 1) * W + lx + 1];
    R w00 = (R(1) - fx) * (R(1) - fy), w10 = fx * (R(1) - fy), w01 = (R(1) - fx) * fy, w11 = fx * fy;
    ox = w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x;
    oy = w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y;
    oz = w00 * a.z + w10 * b.z + w01 * c.z + w11 * d.z;
}


// FP32 deposit: every lane accumulates, in registers, the 52 corner products
// of its particles that fall in the warp's current cell K; the register sums
// are combined over the warp (butterfly reduce-scatter) into the shared
// accumulator when K changes.
__device__ inline void flush_acc_regs(float (&A)[52], int K, float *acc, int RN, int RW, int lane) {
    const int idx = rs26_index(lane);
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        float v[26];
#pragma unroll
        for (int q = 0; q < 26; ++q) v[q] = A[26 * pass + q];
        float r = reduce_scatter26(v, lane);
        if (idx >= 0 && r != 0.f) {
            const int corner = 2 * pass + idx / NMOM, k = idx % NMOM;
            atomicAdd(&acc[k * RN + K + (corner & 1) + (corner >> 1) * RW], r);
        }
    }
#pragma unroll
    for (int q = 0; q < 52; ++q) A[q] = 0.f;
}

// Deterministic deposit: the same two flushes into a fixed-point accumulator.
// The register sums of a warp are formed in a fixed order (the particle order
// of its segments), so each converted partial is reproducible; the integer
// additions then make the totals independent of the order of the atomics.
__device__ inline void flush_acc_regs_fix(float (&A)[52], int K, unsigned long long *acc, int RN, int RW, int lane,
                                          const FixScale &fs) {
    const int idx = rs26_index(lane);
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        float v[26];
#pragma unroll
        for (int q = 0; q < 26; ++q) v[q] = A[26 * pass + q];
        float r = reduce_scatter26(v, lane);
        if (idx >= 0 && r != 0.f) {
            const int corner = 2 * pass + idx / NMOM, k = idx % NMOM;
            atomicAdd(&acc[k * RN + K + (corner & 1) + (corner >> 1) * RW],
                      (unsigned long long)fix_of(r, fs, mom_class(k)));
        }
    }
#pragma unroll
    for (int q = 0; q < 52; ++q) A[q] = 0.f;
}

// FP32 stragglers (lanes whose new cell is not one of the segment's register
// cells, or lies outside the tile's deposit region) are queued per warp in
// shared memory and added to the global moments QCAP at a time, one per lane,
// instead of one by one with the rest of the warp idle.  Entry word f of slot
// i is at f * QCAP + i: cell x, cell y (int bits), offsets x, y, the 13
// moment values.  Each contribution is the same product as without the queue.
constexpr int QCAP = 32;
constexpr int QWORDS = 4 + NMOM;

template <typename R, bool kFix>
__device__ inline void drain_q(const float *qb, int qn, int lane, const TileArgs<R> &a, const GridArgs<R> &g) {
    __syncwarp();   // the entries written by the other lanes
    if (lane < qn) {
        const int ncx = __float_as_int(qb[lane]), ncy = __float_as_int(qb[QCAP + lane]);
        const R nfx = (R)qb[2 * QCAP + lane], nfy = (R)qb[3 * QCAP + lane];
        R val[NMOM];
#pragma unroll
        for (int q = 0; q < NMOM; ++q) val[q] = (R)qb[(4 + q) * QCAP + lane];
        const R Wg[4] = {(R(1) - nfx) * (R(1) - nfy), nfx * (R(1) - nfy), (R(1) - nfx) * nfy, nfx * nfy};
        const int64_t nd[4] = {node_of(g, ncx, ncy, 0, 0), node_of(g, ncx, ncy, 1, 0), node_of(g, ncx, ncy, 0, 1),
                               node_of(g, ncx, ncy, 1, 1)};
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
#pragma unroll
            for (int kk = 0; kk < NMOM; ++kk) {
                if (kFix)
                    atomicAdd(&a.Mfix[(int64_t)kk * g.nnode + nd[cc]],
                              (unsigned long long)fix_of(Wg[cc] * val[kk], a.fs, mom_class(kk)));
                else
                    atomicAdd(&a.M[(int64_t)kk * g.nnode + nd[cc]], Wg[cc] * val[kk]);
            }
    }
    __syncwarp();   // read before the queue is refilled
}

// A particle's state (and, in the FP64 form, its carried quantities).
template <typename R>
struct PState {
    int32_t c;
    R fx, fy, ux, uy, uz, w;
    R ig, bx, by, bz, inv;   // FP64 form: 1/gamma, b, 1/(1 + |b|^2) of the last deposit
};

template <typename R>
constexpr bool kCarry = sizeof(R) == 8;

template <typename R>
__device__ inline void load_carry(const double *cr, int64_t ccap, int64_t slot, PState<R> &s) {
    s.ig = (R)cr[slot];
    s.bx = (R)cr[ccap + slot];
    s.by = (R)cr[2 * ccap + slot];
    s.bz = (R)cr[3 * ccap + slot];
    s.inv = (R)cr[4 * ccap + slot];
}

template <typename R>
__device__ inline void store_carry(double *cr, int64_t ccap, int64_t slot, R ig, R bx, R by, R bz, R inv) {
    cr[slot] = (double)ig;
    cr[ccap + slot] = (double)bx;
    cr[2 * ccap + slot] = (double)by;
    cr[3 * ccap + slot] = (double)bz;
    cr[4 * ccap + slot] = (double)inv;
}

template <typename R>
__device__ inline void load_state(const SpPtr<R> &P, int64_t slot, bool valid, PState<R> &s) {
    if (valid) {
        s.c = P.cell[slot];
        s.fx = P.ox[slot];
        s.fy = P.oy[slot];
        s.ux = P.ux[slot];
        s.uy = P.uy[slot];
        s.uz = P.uz[slot];
        s.w = P.w[slot];
        if constexpr (kCarry<R>) load_carry(P.cr, P.ccap, slot, s);
    } else {
        s.c = 0;
        s.fx = s.fy = s.ux = s.uy = s.uz = s.w = R(0);
        s.ig = s.bx = s.by = s.bz = s.inv = R(0);
    }
}

// Resident blocks per SM the push is compiled for (128 registers a thread):
// the FP32 form's register accumulator needs them, and the FP64 form at 3
// blocks spills and runs slower.
template <typename R>
constexpr int push_min_blocks() { return 2; }

// kBatch: the launch serves several independent runs.  Their argument
// blocks are in device memory (runs[r]), run_items[r] is the exclusive prefix
// of their work-item counts (run_items[nrun] the total), the queue counter is
// a0.ticket, and each item's fields are loaded into shared memory with plain
// loads (the runs' TMA descriptors stay on the host side).
template <typename R, bool kFix, bool kBatch>
__global__ void __launch_bounds__(TILE_BS, push_min_blocks<R>())
    k_push(const __grid_constant__ TileArgs<R> a0, const TileArgs<R> *__restrict__ runs,
           const int32_t *__restrict__ run_items, int nrun, const __grid_constant__ CUtensorMap tmE,
           const __grid_constant__ CUtensorMap tmBo, const __grid_constant__ CUtensorMap tmBn) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr bool kShared = sizeof(R) == 4;  // FP32: shared accumulator; FP64: L2 reductions
    constexpr bool kCellG = sizeof(R) == 8;   // FP64: gathers from per-cell coefficient tables
    constexpr bool kCellDep = sizeof(R) == 8 && !kFix && !kBatch;   // FP64 L2 reductions into cell sums
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint64_t *bar = (uint64_t *)smem;
    int *scr = (int *)(smem + 16);
    V4<R> *sE = (V4<R> *)(smem + SMEM_HEADER);
    // work items: chunk_prefix over (species, tile), species-major, of one run or, batched, of every run
    if (!kBatch && a0.guard && (*a0.guard & 3)) return;   // the previous regroup failed: the host redoes the step
    const int nitems = kBatch ? run_items[nrun] : a0.chunk_prefix[a0.nsp * a0.ntiles];
    const unsigned lt = (1u << lane) - 1u;
    if (!kBatch && tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        if (kChecks)
            for (int k = 0; k < 4; ++k) ((volatile uint32_t *)(smem + a0.offCanary))[k] = CANARY + k;
    }
    __syncthreads();
    for (int iter = 0;; ++iter) {
        if (!kBatch && tid == 0) {
            const int item = atomicAdd(a0.ticket, 1);
            scr[0] = item;
            if (item < nitems) {
                const int2 it = a0.items[item];   // one load instead of a search over the prefix
                scr[1] = it.x;
                scr[2] = it.y;
            }
            scr[4] = 0;
        }
        if (kBatch && tid == 0) {
            int item = atomicAdd(a0.ticket, 1);
            scr[0] = item;
            if (item < nitems) {
                int r = 0;
                const TileArgs<R> *ar = &a0;
                if (kBatch) {
                    int lo = 0, hi = nrun;   // largest r with run_items[r] <= item
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (run_items[mid] <= item) lo = mid;
                        else hi = mid;
                    }
                    r = lo;
                    item -= run_items[r];
                    ar = runs + r;
                }
                int lo = 0, hi = ar->nsp * ar->ntiles;   // largest idx with chunk_prefix[idx] <= item
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if (ar->chunk_prefix[mid] <= item) lo = mid;
                    else hi = mid;
                }
                scr[1] = lo;
                scr[2] = item - ar->chunk_prefix[lo];
                scr[4] = r;
            }
        }
        __syncthreads();
        if (scr[0] >= nitems) break;
        const TileArgs<R> &a = kBatch ? runs[scr[4]] : a0;
        const GridArgs<R> &g = a.g;
        V4<R> *sBo = (V4<R> *)(smem + a.offBo);
        V4<R> *sBn = (V4<R> *)(smem + a.offBn);
        R *acc = (R *)(smem + a.offAcc);
        unsigned long long *accf = (unsigned long long *)(smem + a.offAcc);
        float *qb = (float *)(smem + a.offQ) + wid * (QCAP * QWORDS);   // this warp's straggler queue (FP32)
        int qn = 0;                                                     // its entries (warp-uniform)
        const int RN = a.RW * a.RH;
        const int H = a.H;
        const int RWc = a.RW - 1, RHc = a.RH - 1;  // region cells per row / column
        const int st = scr[1];
        const int s = st / a.ntiles, t = st - s * a.ntiles;
        const int seg0 = scr[2] * a.ch;
        const SpPtr<R> &P = a.sp[s];
        const int seg1 = min(seg0 + a.ch, P.useg[t]);
        const int tx = t % a.ntx, ty = t / a.ntx;
        const int X0 = tx * a.tnx, Y0 = ty * a.tny;
        const int tw = min(a.tnx, g.nx - X0), th = min(a.tny, g.ny - Y0);   // actual extent (ragged last tiles)
        if (!kBatch && tid == 0) {
            mbar_arrive_expect_tx(bar, a.tma_bytes);
            tma_load_3d(sE, &tmE, 0, X0 + g.G, Y0 + g.G, bar);
            if (!kCarry<R>) tma_load_3d(sBo, &tmBo, 0, X0 + g.G, Y0 + g.G, bar);   // FP64: b is carried
            tma_load_3d(sBn, &tmBn, 0, X0 + g.G - H, Y0 + g.G - H, bar);
        }
        if (kBatch) {
            // the padded arrays hold every node a tile box addresses (ghost ring >= tile + halo + 1)
            const int EN = a.EW * a.EH;
            for (int i = tid; i < EN; i += TILE_BS) {
                const int ly = i / a.EW, lx = i - ly * a.EW;
                const int64_t gi = (int64_t)(Y0 + ly + g.G) * g.nxp + (X0 + lx + g.G);
                sE[i] = a.Eh[gi];
                if (!kCarry<R>) sBo[i] = a.Bo[gi];
            }
            for (int i = tid; i < RN; i += TILE_BS) {
                const int ly = i / a.RW, lx = i - ly * a.RW;
                sBn[i] = a.Bnew[(int64_t)(Y0 - H + ly + g.G) * g.nxp + (X0 - H + lx + g.G)];
            }
        }
        if (kShared) {
            if (kFix)
                for (int i = tid; i < NMOM * RN; i += TILE_BS) accf[i] = 0ull;
            else
                for (int i = tid; i < NMOM * RN; i += TILE_BS) acc[i] = R(0);
        }
        if (!kBatch && tid == 0) {
            // one thread waits (bounded), the barrier publishes the copies
            bool ok = mbar_wait_bounded(bar, iter & 1);
            if (!ok) {
                atomicOr(a.flags, 8);
                ok = mbar_wait_bounded(bar, iter & 1);   // the copies in flight land before the block leaves
            }
            scr[3] = ok ? 1 : 0;
        }
        __syncthreads();
        if (!kBatch && scr[3] == 0) return;
        // FP64: the cell coefficients of both tiles (the gathers then take three FMAs per component)
        CellC<R> *sEc = (CellC<R> *)(smem + a.offEc);
        CellC<R> *sBc = (CellC<R> *)(smem + a.offBc);
        if constexpr (kCellG) {
            const int ecn = a.tnx * a.tny, bcn = RWc * RHc;
            for (int i = tid; i < ecn + bcn; i += TILE_BS) {
                if (i < ecn) {
                    const int yy = i / a.tnx, xx = i - yy * a.tnx, o = yy * a.EW + xx;
                    cell_coef(sE[o], sE[o + 1], sE[o + a.EW], sE[o + a.EW + 1], sEc[i]);
                } else {
                    const int j = i - ecn, yy = j / RWc, xx = j - yy * RWc, o = yy * a.RW + xx;
                    cell_coef(sBn[o], sBn[o + 1], sBn[o + a.RW], sBn[o + a.RW + 1], sBc[j]);
                }
            }
            __syncthreads();
        }
        const int64_t bbase = P.bstart[t];
        const int64_t sbase = bbase / SEG;
        // contiguous segments per warp, so that same-cell runs stay in one warp
        const int per = (seg1 - seg0 + TILE_WARPS - 1) / TILE_WARPS;
        const int my0 = seg0 + wid * per, my1 = min(my0 + per, seg1);
        float A[52];
#pragma unroll
        for (int q = 0; q < 52; ++q) A[q] = 0.f;
        int K = -1;
        PState<R> nx;
        int n_next = 0;
        if (my0 < my1) {
            n_next = P.segn[sbase + my0];
            load_state(P, bbase + (int64_t)my0 * SEG + lane, lane < n_next, nx);
        }
        for (int sg = my0; sg < my1; ++sg) {
            const PState<R> cu = nx;
            const int n = n_next;
            const int64_t slot0 = bbase + (int64_t)sg * SEG;
            if (sg + 1 < my1) {   // prefetch the next segment while this one is processed
                n_next = P.segn[sbase + sg + 1];
                load_state(P, slot0 + SEG + lane, lane < n_next, nx);
            }
            bool valid = lane < n;
            if (kChecks && valid &&
                (cu.c < 0 || cu.c >= g.nx * g.ny || !(cu.fx >= R(0) && cu.fx < R(1)) || !(cu.fy >= R(0) && cu.fy < R(1)))) {
                atomicOr(a.flags, FLAG_CHECK);
                valid = false;
            }
            int cx, cy;
            cell_split(cu.c, g.nx, a.magic_nx, cx, cy);
            int lx = cx - X0, ly = cy - Y0;
            if (valid && (lx < 0 || lx >= tw || ly < 0 || ly >= th)) {
                atomicOr(a.flags, 16);  // particle outside its bin's tile: skip it
                valid = false;
            }
            if (!valid) lx = ly = 0;
            const R fx = cu.fx, fy = cu.fy, ux = cu.ux, uy = cu.uy, uz = cu.uz, w = cu.w;
            // gather at r^n (Section 3.3: forces)
            R Ex, Ey, Ez;
            if constexpr (kCellG) {
                const CellC<R> &ce = sEc[ly * a.tnx + lx];
                const R fxy = fx * fy;
                Ex = cell_eval(ce.k[0], fx, fy, fxy);
                Ey = cell_eval(ce.k[1], fx, fy, fxy);
                Ez = cell_eval(ce.k[2], fx, fy, fxy);
            } else {
                sm_gather(sE, a.EW, lx, ly, fx, fy, Ex, Ey, Ez);
            }
            // implicit push (Eq. 2, E factored out)
            const R k = P.kq;
            R ig, bx, by, bz, binv;
            if constexpr (kCarry<R>) {
                // the B the moments were made with, at this position and u: the last deposit's b (carried)
                ig = cu.ig;
                bx = cu.bx;
                by = cu.by;
                bz = cu.bz;
                binv = cu.inv;
            } else {
                R Bx, By, Bz;
                sm_gather(sBo, a.EW, lx, ly, fx, fy, Bx, By, Bz);
                ig = rsqrt_r(R(1) + ux * ux + uy * uy + uz * uz);
                bx = k * Bx * ig;
                by = k * By * ig;
                bz = k * Bz * ig;
                binv = rcp_r(R(1) + bx * bx + by * by + bz * bz);
            }
            // u^{n+1} and the move in cell units
            R nux, nuy, nuz, sx, sy;
            push_move(bx, by, bz, binv, ig, ux + k * Ex, uy + k * Ey, uz + k * Ez, ux, uy, uz, fx, fy, a.sdx, a.sdy, nux,
                      nuy, nuz, sx, sy);
            const R flx = floor(sx), fly = floor(sy);
            R nfx = sx - flx, nfy = sy - fly;
            int shx = (int)flx, shy = (int)fly;
            if (ge_one(nfx)) { nfx = R(0); shx += 1; }   // nfx, nfy >= 0
            if (ge_one(nfy)) { nfy = R(0); shy += 1; }
            const int ncxu = cx + shx, ncyu = cy + shy;
            const int ncy = (shy > -g.ny && shy < g.ny) ? wrap1(ncyu, g.ny) : imod(ncyu, g.ny);
            int ncx = ncxu;
            bool dead = false;
            if (g.periodic_x) ncx = (shx > -g.nx && shx < g.nx) ? wrap1(ncxu, g.nx) : imod(ncxu, g.nx);
            else if (ncxu < 0 || ncxu >= g.nx) dead = true;
            const bool alive = valid && !dead;
            if (kChecks && alive &&
                !(nfx >= R(0) && nfx < R(1) && nfy >= R(0) && nfy < R(1) && ncx >= 0 && ncx < g.nx && ncy >= 0 && ncy < g.ny))
                atomicOr(a.flags, FLAG_CHECK);
            const int lnx = lx + shx, lny = ly + shy;   // new cell relative to the tile origin
            const bool intile = lnx >= 0 && lnx < tw && lny >= 0 && lny < th;
            const int ttx = (alive && !intile) ? ncx / a.tnx : tx, tty = (alive && !intile) ? ncy / a.tny : ty;
            const int tn = tty * a.ntx + ttx;
            const bool stay = alive && tn == t;
            const bool leave = alive && tn != t;
            if (leave && !tile_near(tx, ty, ttx, tty, a.ntx, a.nty, g.periodic_x)) {
                atomicOr(a.step_flags, 1);
                atomicOr(a.flags, 1);
            }
            // deposit at r^{n+1} with the new B (Eq. 3)
            const int rx = lnx + H, ry = lny + H;
            const bool inreg = alive && rx >= 0 && rx < RWc && ry >= 0 && ry < RHc;
            R nBx = R(0), nBy = R(0), nBz = R(0);
            R val[NMOM];   // FP32: the 13 moment values; FP64: their parts (the class factors go to the weights)
            R cig, cbx, cby, cbz, cinv;   // carried to the next push (FP64 form)
            R fr, fS, fj;                 // FP64: the class factors of the moments
            if (inreg) {
                if constexpr (kCellG) {
                    const CellC<R> &cb = sBc[ry * RWc + rx];
                    const R fxy = nfx * nfy;
                    nBx = cell_eval(cb.k[0], nfx, nfy, fxy);
                    nBy = cell_eval(cb.k[1], nfx, nfy, fxy);
                    nBz = cell_eval(cb.k[2], nfx, nfy, fxy);
                } else {
                    sm_gather(sBn, a.RW, rx, ry, nfx, nfy, nBx, nBy, nBz);
                }
            } else if (alive) gather4(a.Bnew, g, ncx, ncy, nfx, nfy, nBx, nBy, nBz);
            if constexpr (kShared || kCellDep)   // the 13 moment values
                particle_moments_c(P.q, P.kq, P.hq, w, nux, nuy, nuz, nBx, nBy, nBz, val, cig, cbx, cby, cbz, cinv);
            else   // class factors and parts (the corner-form FP64 deposit)
                particle_moment_parts(P.q, P.kq, P.cq2, w, nux, nuy, nuz, nBx, nBy, nBz, val, fr, fS, fj, cig, cbx, cby,
                                      cbz, cinv);
            unsigned strag = 0u;   // FP32: lanes left to the global path
            if (kShared) {
                const int key = inreg ? ry * a.RW + rx : -1;
                const float fxm = (float)nfx, fym = (float)nfy;
                // register passes: the lanes in the warp's cell K, then, while
                // the first remaining lane's cell holds at least MIN_GROUP of
                // the remaining lanes, that cell (after a flush of K)
                unsigned rem = __ballot_sync(FULL, key >= 0);
                const unsigned same = __match_any_sync(FULL, key);   // the lanes of my cell
                for (int pass = 0; pass < 3 && rem; ++pass) {
                    const unsigned inK = __ballot_sync(FULL, key == K) & rem;
                    if (inK) {
                        const bool mine = (inK >> lane) & 1u;
                        const float W0 = mine ? (1.f - fxm) * (1.f - fym) : 0.f, W1 = mine ? fxm * (1.f - fym) : 0.f;
                        const float W2 = mine ? (1.f - fxm) * fym : 0.f, W3 = mine ? fxm * fym : 0.f;
#pragma unroll
                        for (int q = 0; q < NMOM; ++q) {
                            const float vq = (float)val[q];
                            A[q] += W0 * vq;
                            A[NMOM + q] += W1 * vq;
                            A[2 * NMOM + q] += W2 * vq;
                            A[3 * NMOM + q] += W3 * vq;
                        }
                        rem &= ~inK;
                        if (!rem) break;
                    }
                    // the next cell: the first remaining lane's whose cell holds at least
                    // MIN_GROUP remaining lanes (a lone lane that moved ahead of a group
                    // does not send the group to the global path)
                    const unsigned grp = __ballot_sync(FULL, ((rem >> lane) & 1u) && __popc(same & rem) >= MIN_GROUP);
                    if (!grp) break;
                    const int cand = __shfl_sync(FULL, key, __ffs(grp) - 1);
                    if (K >= 0) {
                        if (kFix) flush_acc_regs_fix(A, K, accf, RN, a.RW, lane, a.fs);
                        else flush_acc_regs(A, K, (float *)acc, RN, a.RW, lane);
                    }
                    K = cand;
                }
                // the rest (a few lanes in further cells) add their own products in L2
                strag = rem;
            }
            if constexpr (kShared) {
                // stragglers and lanes outside the deposit region: into the warp's queue
                const bool gl = alive && (!inreg || ((strag >> lane) & 1u));
                const unsigned gm = __ballot_sync(FULL, gl);
                if (gm) {
                    const int np = __popc(gm);
                    if (qn + np > QCAP) {
                        drain_q<R, kFix>(qb, qn, lane, a, g);
                        qn = 0;
                    }
                    if (gl) {
                        const int slot = qn + __popc(gm & lt);
                        qb[slot] = __int_as_float(ncx);
                        qb[QCAP + slot] = __int_as_float(ncy);
                        qb[2 * QCAP + slot] = (float)nfx;
                        qb[3 * QCAP + slot] = (float)nfy;
#pragma unroll
                        for (int q = 0; q < NMOM; ++q) qb[(4 + q) * QCAP + slot] = (float)val[q];
                    }
                    qn += np;
                }
            } else if (alive) {
                // FP64: every lane adds its own products in L2 (the single-run push: cell sums)
                if constexpr (kCellDep)
                    deposit_fp64_cell(a.Mc, (int64_t)g.nx * g.ny, (int64_t)ncy * g.nx + ncx, nfx, nfy, val, lane);
                else
                    deposit_fp64<kFix>(a.M, a.Mfix, a.fs, g, ncx, ncy, nfx, nfy, val, fr, fS, fj, lane);
            }
            // warp compaction of the segment (every lane has loaded before any store)
            const unsigned ms = __ballot_sync(FULL, stay), ml = __ballot_sync(FULL, leave);
            const int32_t ncell = ncy * g.nx + ncx;
            if (stay) {
                const int64_t d = slot0 + __popc(ms & lt);
                P.cell[d] = ncell;
                P.ox[d] = nfx;
                P.oy[d] = nfy;
                P.ux[d] = nux;
                P.uy[d] = nuy;
                P.uz[d] = nuz;
                P.w[d] = w;
                if constexpr (kCarry<R>) store_carry(P.cr, P.ccap, d, cig, cbx, cby, cbz, cinv);
            } else if (leave) {
                const int64_t d = slot0 + __popc(ml & lt);
                P.mcell[d] = ncell;
                P.mox[d] = nfx;
                P.moy[d] = nfy;
                P.mux[d] = nux;
                P.muy[d] = nuy;
                P.muz[d] = nuz;
                P.mw[d] = w;
                P.mkey[d] = (uint32_t)tn;
                if constexpr (kCarry<R>) store_carry(P.mcr, P.ccap, d, cig, cbx, cby, cbz, cinv);
            } else if (valid && dead) {
                atomicAdd(P.removed, 1ull);
            }
            if (lane == 0) {
                P.segn[sbase + sg] = __popc(ms);
                P.segml[sbase + sg] = __popc(ml);
            }
        }
        if constexpr (kShared) {
            if (qn > 0) drain_q<R, kFix>(qb, qn, lane, a, g);   // the item's last stragglers
        }
        if (kShared) {
            if (K >= 0) {
                if (kFix) flush_acc_regs_fix(A, K, accf, RN, a.RW, lane, a.fs);
                else flush_acc_regs(A, K, (float *)acc, RN, a.RW, lane);
            }
        }
        __syncthreads();
        if (kShared) {
            // flush the tile + halo accumulator: one node per thread, its 13
            // moments issued back to back (FP32: TwoSum compensation of each add)
            for (int r = tid; r < RN; r += TILE_BS) {
                const int ryn = r / a.RW, rxn = r - ryn * a.RW;
                int gx = X0 - H + rxn;
                const int gy = imod(Y0 - H + ryn, g.ny);
                if (g.periodic_x) gx = imod(gx, g.nx);
                else if (gx < 0 || gx >= g.nxn) continue;
                const int64_t gn = (int64_t)gy * g.nxn + gx;
                if constexpr (kFix) {
#pragma unroll
                    for (int kq = 0; kq < NMOM; ++kq) {
                        const unsigned long long vf = accf[kq * RN + r];
                        if (vf != 0ull) atomicAdd(&a.Mfix[(int64_t)kq * g.nnode + gn], vf);
                    }
                } else {
                    R v[NMOM], old[NMOM];
#pragma unroll
                    for (int kq = 0; kq < NMOM; ++kq) {
                        v[kq] = acc[kq * RN + r];
                        old[kq] = (v[kq] != R(0)) ? atomicAdd(&a.M[(int64_t)kq * g.nnode + gn], v[kq]) : R(0);
                    }
#pragma unroll
                    for (int kq = 0; kq < NMOM; ++kq) {
                        const R sum = old[kq] + v[kq];
                        const R bb = sum - old[kq];
                        const R err = (old[kq] - (sum - bb)) + (v[kq] - bb);
                        if (err != R(0)) atomicAdd(&a.Mlo[(int64_t)kq * g.nnode + gn], err);
                    }
                }
            }
            __syncthreads();
        }
        if (kChecks && !kBatch && tid == 0)
            for (int k = 0; k < 4; ++k)
                if (((volatile uint32_t *)(smem + a0.offCanary))[k] != CANARY + k) atomicOr(a.flags, FLAG_CHECK);
    }
}

// Push with a spline shape of degree N = 2, 3, 4 (Section 3.3, last
// paragraph).  The same work items, state layout, implicit push (Eq. 2, E
// factored out), moments (Eq. 3) and in-place compaction as k_push; the
// (N + 1) x (N + 1) node gathers read the padded fields in global memory (the
// nodes around a particle reach beyond a tile's box), and every lane adds its
// (N + 1)^2 x 13 products in L2 (deposit_s; the FP32 form without the
// compensation term of the tile flush).  One warp per segment run, no shared
// memory.
template <typename R>
constexpr int push_s_min_blocks() { return sizeof(R) == 8 ? 2 : 0; }   // FP64: at most 128 registers; FP32: the default

template <typename R, bool kFix, int N>
__global__ void __launch_bounds__(TILE_BS, push_s_min_blocks<R>()) k_push_s(const __grid_constant__ TileArgs<R> a) {
    constexpr bool kParts = sizeof(R) == 8;
    if (a.guard && (*a.guard & 3)) return;   // the previous regroup failed: the host redoes the step
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __shared__ int scr[3];
    const GridArgs<R> &g = a.g;
    const int nitems = a.chunk_prefix[a.nsp * a.ntiles];
    const unsigned lt = (1u << lane) - 1u;
    for (;;) {
        if (tid == 0) {
            const int item = atomicAdd(a.ticket, 1);
            scr[0] = item;
            if (item < nitems) {
                const int2 it = a.items[item];
                scr[1] = it.x;
                scr[2] = it.y;
            }
        }
        __syncthreads();
        if (scr[0] >= nitems) break;
        const int st = scr[1];
        const int s = st / a.ntiles, t = st - s * a.ntiles;
        const int seg0 = scr[2] * a.ch;
        __syncthreads();   // scr is rewritten by the next item
        const SpPtr<R> &P = a.sp[s];
        const int seg1 = min(seg0 + a.ch, P.useg[t]);
        const int tx = t % a.ntx, ty = t / a.ntx;
        const int X0 = tx * a.tnx, Y0 = ty * a.tny;
        const int tw = min(a.tnx, g.nx - X0), th = min(a.tny, g.ny - Y0);
        const int64_t bbase = P.bstart[t];
        const int64_t sbase = bbase / SEG;
        const int per = (seg1 - seg0 + TILE_WARPS - 1) / TILE_WARPS;
        const int my0 = seg0 + wid * per, my1 = min(my0 + per, seg1);
        PState<R> nx;
        int n_next = 0;
        if (my0 < my1) {
            n_next = P.segn[sbase + my0];
            load_state(P, bbase + (int64_t)my0 * SEG + lane, lane < n_next, nx);
        }
        for (int sg = my0; sg < my1; ++sg) {
            const PState<R> cu = nx;
            const int n = n_next;
            const int64_t slot0 = bbase + (int64_t)sg * SEG;
            if (sg + 1 < my1) {
                n_next = P.segn[sbase + sg + 1];
                load_state(P, slot0 + SEG + lane, lane < n_next, nx);
            }
            bool valid = lane < n;
            if (kChecks && valid &&
                (cu.c < 0 || cu.c >= g.nx * g.ny || !(cu.fx >= R(0) && cu.fx < R(1)) || !(cu.fy >= R(0) && cu.fy < R(1)))) {
                atomicOr(a.flags, FLAG_CHECK);
                valid = false;
            }
            int cx, cy;
            cell_split(cu.c, g.nx, a.magic_nx, cx, cy);
            int lx = cx - X0, ly = cy - Y0;
            if (valid && (lx < 0 || lx >= tw || ly < 0 || ly >= th)) {
                atomicOr(a.flags, 16);
                valid = false;
            }
            if (!valid) {
                lx = ly = 0;
                cx = X0;
                cy = Y0;
            }
            const R fx = valid ? cu.fx : R(0), fy = valid ? cu.fy : R(0);
            const R ux = cu.ux, uy = cu.uy, uz = cu.uz, w = cu.w;
            // gather at r^n
            const SplineN<R, N> so = spline_n<R, N>(g, cx, cy, fx, fy);
            R Ex, Ey, Ez;
            gather_s(a.Eh, g, so, Ex, Ey, Ez);
            const R k = P.kq;
            R ig, bx, by, bz, binv;
            if constexpr (kCarry<R>) {
                ig = cu.ig;
                bx = cu.bx;
                by = cu.by;
                bz = cu.bz;
                binv = cu.inv;
            } else {
                R Bx, By, Bz;
                gather_s(a.Bo, g, so, Bx, By, Bz);
                ig = rsqrt_r(R(1) + ux * ux + uy * uy + uz * uz);
                bx = k * Bx * ig;
                by = k * By * ig;
                bz = k * Bz * ig;
                binv = rcp_r(R(1) + bx * bx + by * by + bz * bz);
            }
            R nux, nuy, nuz, sx, sy;
            push_move(bx, by, bz, binv, ig, ux + k * Ex, uy + k * Ey, uz + k * Ez, ux, uy, uz, fx, fy, a.sdx, a.sdy, nux,
                      nuy, nuz, sx, sy);
            const R flx = floor(sx), fly = floor(sy);
            R nfx = sx - flx, nfy = sy - fly;
            int shx = (int)flx, shy = (int)fly;
            if (ge_one(nfx)) { nfx = R(0); shx += 1; }   // nfx, nfy >= 0
            if (ge_one(nfy)) { nfy = R(0); shy += 1; }
            const int ncxu = cx + shx, ncyu = cy + shy;
            const int ncy = (shy > -g.ny && shy < g.ny) ? wrap1(ncyu, g.ny) : imod(ncyu, g.ny);
            int ncx = ncxu;
            bool dead = false;
            if (g.periodic_x) ncx = (shx > -g.nx && shx < g.nx) ? wrap1(ncxu, g.nx) : imod(ncxu, g.nx);
            else if (ncxu < 0 || ncxu >= g.nx) dead = true;
            const bool alive = valid && !dead;
            if (kChecks && alive &&
                !(nfx >= R(0) && nfx < R(1) && nfy >= R(0) && nfy < R(1) && ncx >= 0 && ncx < g.nx && ncy >= 0 && ncy < g.ny))
                atomicOr(a.flags, FLAG_CHECK);
            const int lnx = lx + shx, lny = ly + shy;
            const bool intile = lnx >= 0 && lnx < tw && lny >= 0 && lny < th;
            const int ttx = (alive && !intile) ? ncx / a.tnx : tx, tty = (alive && !intile) ? ncy / a.tny : ty;
            const int tn = tty * a.ntx + ttx;
            const bool stay = alive && tn == t;
            const bool leave = alive && tn != t;
            if (leave && !tile_near(tx, ty, ttx, tty, a.ntx, a.nty, g.periodic_x)) {
                atomicOr(a.step_flags, 1);
                atomicOr(a.flags, 1);
            }
            // deposit at r^{n+1} with the new B (Eq. 3)
            R val[NMOM];
            R cig = R(0), cbx = R(0), cby = R(0), cbz = R(0), cinv = R(0);
            R fr = R(1), fS = R(1), fj = R(1);
            if (alive) {
                const SplineN<R, N> sn = spline_n<R, N>(g, ncx, ncy, nfx, nfy);
                R nBx, nBy, nBz;
                gather_s(a.Bnew, g, sn, nBx, nBy, nBz);
                if constexpr (kParts)
                    particle_moment_parts(P.q, P.kq, P.cq2, w, nux, nuy, nuz, nBx, nBy, nBz, val, fr, fS, fj, cig,
                                          cbx, cby, cbz, cinv);
                else
                    particle_moments_c(P.q, P.kq, P.hq, w, nux, nuy, nuz, nBx, nBy, nBz, val, cig, cbx, cby, cbz,
                                       cinv);
                deposit_s<R, kFix, kParts, N>(a.M, a.Mfix, a.fs, g, sn, val, fr, fS, fj, lane);
            }
            // warp compaction of the segment (every lane has loaded before any store)
            const unsigned ms = __ballot_sync(FULL, stay), ml = __ballot_sync(FULL, leave);
            const int32_t ncell = ncy * g.nx + ncx;
            if (stay) {
                const int64_t d = slot0 + __popc(ms & lt);
                P.cell[d] = ncell;
                P.ox[d] = nfx;
                P.oy[d] = nfy;
                P.ux[d] = nux;
                P.uy[d] = nuy;
                P.uz[d] = nuz;
                P.w[d] = w;
                if constexpr (kCarry<R>) store_carry(P.cr, P.ccap, d, cig, cbx, cby, cbz, cinv);
            } else if (leave) {
                const int64_t d = slot0 + __popc(ml & lt);
                P.mcell[d] = ncell;
                P.mox[d] = nfx;
                P.moy[d] = nfy;
                P.mux[d] = nux;
                P.muy[d] = nuy;
                P.muz[d] = nuz;
                P.mw[d] = w;
                P.mkey[d] = (uint32_t)tn;
                if constexpr (kCarry<R>) store_carry(P.mcr, P.ccap, d, cig, cbx, cby, cbz, cinv);
            } else if (valid && dead) {
                atomicAdd(P.removed, 1ull);
            }
            if (lane == 0) {
                P.segn[sbase + sg] = __popc(ms);
                P.segml[sbase + sg] = __popc(ml);
            }
        }
    }
}

// Work items of the push: ch-segment runs of every (species, tile), in
// species-major, tile order; the counts are scanned afterwards (the entry
// after the last holds the total).  Also resets the work queue (the tile
// lists are reset separately, just before the push: reset_lists).
struct UsegPtrs {
    const int32_t *p[PIC_MAX_SPECIES];
};

__global__ void k_chunk_counts(UsegPtrs u, int nsp, int ntiles, int ch, int32_t *__restrict__ out,
                               int32_t *__restrict__ ticket, uint8_t *__restrict__ occ) {
    const int n = nsp * ntiles;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int s = i / ntiles, t = i - s * ntiles;
        out[i] = (u.p[s][t] + ch - 1) / ch;
        if (s == 0) {   // occupancy of the tile by any species at the start of the push
            int any = 0;
            for (int q = 0; q < nsp; ++q) any |= u.p[q][t];
            occ[t] = any != 0;
        }
    } else if (i == n) {
        out[n] = 0;
        *ticket = 0;
    }
}

// Node tiles a push may have deposited into.  A particle of occupied tile a
// ends in tile a-1, a or a+1 on each axis (a farther move sets bit 0 of the
// step flags), and its corner nodes lie in its new cell's tile or the next one
// (node column i is in tile min(i / tnx, ntx - 1)); the FP32 flush region is
// the tile plus a halo of fewer than a tile's cells.  So node tile T is touched
// if a tile of T-2 .. T+1 on both axes (wrapping where the box is periodic) was
// occupied (spline shapes reach further: touch_map), and every tile is touched
// after a far move.  The same pass lists
// the tiles the regroup must visit -- those with an occupied tile among T-1 ..
// T+1 on both axes (stayers or arrivals; after a far move the regroup's output
// is replaced by the full sort) -- and empties the next bins of the others.
struct UsegOut {
    int32_t *p[PIC_MAX_SPECIES];
};

__global__ void k_touch_map(const uint8_t *__restrict__ occ, const int32_t *__restrict__ step_flags,
                            const int32_t *__restrict__ guard, int ntx, int nty,
                            int periodic_x, uint8_t *__restrict__ touched, int32_t *__restrict__ touch_list,
                            int32_t *__restrict__ rg_list, int32_t *__restrict__ list_n, UsegOut useg2, int nsp,
                            int dlx, int dly, int dhx, int dhy) {
    const int T = blockIdx.x * blockDim.x + threadIdx.x;
    if (T >= ntx * nty) return;
    if (guard && (*guard & 3)) return;
    const bool far = (*step_flags & 1) != 0;
    const int tx = T % ntx, ty = T / ntx;
    bool touch = far, near = false;
    for (int dy = -dly; dy <= dhy; ++dy) {
        int y = ty + dy;
        y = y < 0 ? y + nty : (y >= nty ? y - nty : y);
        if (y < 0 || y >= nty) continue;   // fewer than 3 tile rows: a wrap may still leave the range
        for (int dx = -dlx; dx <= dhx; ++dx) {
            int x = tx + dx;
            if (periodic_x) x = x < 0 ? x + ntx : (x >= ntx ? x - ntx : x);
            if (x < 0 || x >= ntx) continue;
            if (occ[y * ntx + x]) {
                touch = true;
                if (dx >= -1 && dy >= -1) near = true;
            }
        }
    }
    touched[T] = touch ? 1 : 0;
    if (touch) touch_list[atomicAdd(&list_n[0], 1)] = T;
    if (near) rg_list[atomicAdd(&list_n[1], 1)] = T;
    else
        for (int s = 0; s < nsp; ++s) useg2.p[s][T] = 0;
}

int touch_map(pic_t *h) {
    UsegOut u2;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) u2.p[s] = (s < h->nsp) ? h->sp[s].useg[1 - h->sp[s].scur] : nullptr;
    // occupied tiles T - dl .. T + dh can deposit into node tile T: the nodes of a particle in cell c
    // are c + lo .. c + hi (order 1: 0 .. 1; 2: -1 .. 2; 3: -1 .. 2; 4: -2 .. 3), in node tiles
    // b - ceil(-lo / tile) .. b + ceil(hi / tile) of the new cell's tile b, itself within one tile
    // of the occupied one
    const int lo = -(h->shape / 2), hi = (h->shape + 2) / 2;
    const int dlx = 1 + (hi + h->tnx - 1) / h->tnx, dly = 1 + (hi + h->tny - 1) / h->tny;
    const int dhx = 1 + (-lo + h->tnx - 1) / h->tnx, dhy = 1 + (-lo + h->tny - 1) / h->tny;
    k_touch_map<<<(h->ntiles + 255) / 256, 256, 0, h->st>>>(h->occ, h->d_step_flags + (h->step & 1), h->guard,
                                                            h->ntx, h->nty,
                                                            h->periodic_x ? 1 : 0, h->touched, h->touch_list,
                                                            h->rg_list, h->list_n, u2, h->nsp, dlx, dly, dhx, dhy);
    count_launch(h);
    return check_launch("k_touch_map");
}

// The push's item table from the scanned item counts: item c of species-tile
// index i (c0 = prefix[i] <= c < prefix[i + 1]) -> (i, c - c0).
__global__ void k_item_table(const int32_t *__restrict__ prefix, int n, int2 *__restrict__ items) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c0 = prefix[i], c1 = prefix[i + 1];
    for (int c = c0; c < c1; ++c) items[c] = make_int2(i, c - c0);
}

// Exclusive block scan of one int per thread; *total = block sum.
__device__ inline int block_excl_scan_int(int v, int *wsum, int *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int x = (lane < TILE_WARPS) ? wsum[lane] : 0;
        int xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += y;
        }
        wsum[lane] = xi - x;
        if (lane == 31) wsum[32] = xi;
    }
    __syncthreads();
    const int ex = wsum[wid] + incl - v;
    *total = wsum[32];
    __syncthreads();
    return ex;
}

// Per-tile regroup after the push, one block per (tile, species).  The
// sequence is the tile's stayers (its bin segments in order, the valid prefix
// of each) followed by its arrivals (the leavers of the neighbour tiles bound
// for this tile: neighbours in ascending tile order, their mirror segments in
// order).  A stable counting sort of that sequence by cell inside the tile
// (row-major) writes the tile densely into the spare buffer set, and the
// tile's new counts to segn2 / useg2.  Ranges of the sort: the warps' stayer
// segment ranges, then the arrivals (sorted by the last warp).  If the bin
// cannot hold the result, or the arrivals overflow their list, the step flag
// asks for the full regroup, which rebuilds from the bins and the mirror.
constexpr int REGROUP_RANGES = TILE_WARPS + 1;
constexpr int ARR_MAX = 8192;

__host__ __device__ inline int regroup_smem_bytes(int tile_cells) {
    return (REGROUP_RANGES * tile_cells + ARR_MAX) * (int)sizeof(int);
}

template <typename R>
__device__ inline void load_particle(const SpPtr<R> &P, bool from_mirror, int64_t si, PState<R> &v) {
    if (from_mirror) {
        v.c = P.mcell[si]; v.fx = P.mox[si]; v.fy = P.moy[si];
        v.ux = P.mux[si]; v.uy = P.muy[si]; v.uz = P.muz[si]; v.w = P.mw[si];
    } else {
        v.c = P.cell[si]; v.fx = P.ox[si]; v.fy = P.oy[si];
        v.ux = P.ux[si]; v.uy = P.uy[si]; v.uz = P.uz[si]; v.w = P.w[si];
    }
    if constexpr (kCarry<R>) load_carry(from_mirror ? P.mcr : P.cr, P.ccap, si, v);
}

template <typename R>
__device__ inline void store_particle(const SpPtr<R> &P, int64_t d, const PState<R> &v) {
    P.ocell[d] = v.c; P.oox[d] = v.fx; P.ooy[d] = v.fy;
    P.oux[d] = v.ux; P.ouy[d] = v.uy; P.ouz[d] = v.uz; P.ow[d] = v.w;
    if constexpr (kCarry<R>) store_carry(P.ocr, P.ccap, d, v.ig, v.bx, v.by, v.bz, v.inv);
}

// kBatch: blocks of several runs; run_tiles[r] is the exclusive prefix of the
// runs' tile counts (blockIdx.x indexes the concatenation), runs[r] their
// argument blocks.
template <typename R, bool kBatch>
__device__ __forceinline__ void regroup_one(const TileArgs<R> &a, int t, int s, int *rsm) {
    __shared__ int s_nb[8], s_cnt[TILE_WARPS], s_base[TILE_WARPS + 1];
    __shared__ int wsum[33];
    if (s >= a.nsp) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const SpPtr<R> &P = a.sp[s];
    const GridArgs<R> &g = a.g;
    const int tx = t % a.ntx, ty = t / a.ntx;
    const int X0 = tx * a.tnx, Y0 = ty * a.tny;
    const int tw = min(a.tnx, g.nx - X0), th = min(a.tny, g.ny - Y0);
    const int nc = tw * th;
    int *hist = rsm;                          // [REGROUP_RANGES][nc]
    int *arr = rsm + REGROUP_RANGES * nc;     // mirror slots of the arrivals, in sequence order
    const int64_t tb = P.bstart[t] / SEG, to = P.bstart[t];
    const int ut = P.useg[t];
    const unsigned lt = (1u << lane) - 1u;
    const int nnb = a.nbr[t * 9];
    auto local_of = [&](int32_t c) {
        int cx, cy;
        cell_split(c, g.nx, a.magic_nx, cx, cy);
        const int lx = cx - X0, ly = cy - Y0;
        return (lx >= 0 && lx < tw && ly >= 0 && ly < th) ? ly * tw + lx : -1;
    };
    // nothing stays and no neighbour holds particles: an empty bin
    int busy = (tid == 0 && ut > 0);
    if (tid < nnb) {
        s_nb[tid] = a.nbr[t * 9 + 1 + tid];
        busy |= P.useg[s_nb[tid]] > 0;
    }
    if (!__syncthreads_or(busy)) {
        if (tid == 0) P.useg2[t] = 0;
        return;
    }
    for (int i = tid; i < REGROUP_RANGES * nc; i += TILE_BS) hist[i] = 0;
    // 1. the arrivals: warp q scans neighbour q's mirror (neighbours ascending), counts, then lists
    auto scan_mirror = [&](bool write, int pos) {
        const int src = s_nb[wid];
        const int64_t sb = P.bstart[src] / SEG, so = P.bstart[src];
        const int us = P.useg[src];
        int tot = 0;
        for (int j0 = 0; j0 < us; j0 += SEG) {
            const int j = j0 + lane;
            const int ml = (j < us) ? P.segml[sb + j] : 0;
            int c = 0;
            for (int r = 0; r < ml; ++r) c += (P.mkey[so + (int64_t)j * SEG + r] == (uint32_t)t);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            if (write && c) {
                int k = pos + tot + incl - c;
                for (int r = 0; r < ml; ++r) {
                    const int64_t si = so + (int64_t)j * SEG + r;
                    if (P.mkey[si] != (uint32_t)t) continue;
                    if (k < ARR_MAX) arr[k] = (int)si;
                    ++k;
                }
            }
            tot += __shfl_sync(FULL, incl, 31);
        }
        return tot;
    };
    if (wid < TILE_WARPS) {
        const int c = (wid < nnb) ? scan_mirror(false, 0) : 0;
        if (lane == 0) s_cnt[wid] = c;
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int w = 0; w < TILE_WARPS; ++w) {
            s_base[w] = acc;
            acc += s_cnt[w];
        }
        s_base[TILE_WARPS] = acc;
    }
    __syncthreads();
    const int narr = s_base[TILE_WARPS];
    if (narr > ARR_MAX) {
        if (tid == 0) atomicOr(a.step_flags, 2);
        return;
    }
    if (wid < nnb && s_cnt[wid] > 0) scan_mirror(true, s_base[wid]);
    // 2. counts per (range, cell); a warp's next segment is loaded while it works on this one
    const int per = (ut + TILE_WARPS - 1) / TILE_WARPS;
    const int j0w = min(wid * per, ut), j1w = min(j0w + per, ut);
    {
        // four segments' counts and cells are loaded before any is used
        constexpr int D = 4;
        for (int j0 = j0w; j0 < j1w; j0 += D) {
            int n[D];
            int32_t c[D];
#pragma unroll
            for (int u = 0; u < D; ++u) {
                const int j = j0 + u;
                n[u] = (j < j1w) ? P.segn[tb + j] : 0;
                c[u] = (j < j1w) ? P.cell[to + (int64_t)j * SEG + lane] : 0;
            }
#pragma unroll
            for (int u = 0; u < D; ++u) {
                int loc = -1;
                if (lane < n[u]) {
                    loc = local_of(c[u]);
                    if (loc < 0) atomicOr(a.flags, 16);
                }
                const unsigned m = __match_any_sync(FULL, loc >= 0 ? loc : -1 - lane);
                if (loc >= 0 && lane == __ffs(m) - 1) atomicAdd(&hist[wid * nc + loc], __popc(m));
            }
        }
    }
    __syncthreads();   // the arrival list and the stayer counts are complete
    for (int i = tid; i < narr; i += TILE_BS) {
        const int loc = local_of(P.mcell[arr[i]]);
        if (loc >= 0) atomicAdd(&hist[TILE_WARPS * nc + loc], 1);
        else atomicOr(a.flags, 16);
    }
    __syncthreads();
    // 3. cell-major exclusive scan over (cell, range): hist becomes the write bases
    int carry = 0;
    for (int c0 = 0; c0 < nc; c0 += TILE_BS) {
        const int c = c0 + tid;
        int col = 0;
        if (c < nc)
            for (int r = 0; r < REGROUP_RANGES; ++r) col += hist[r * nc + c];
        int blk = 0;
        int run = carry + block_excl_scan_int(col, wsum, &blk);
        if (c < nc)
            for (int r = 0; r < REGROUP_RANGES; ++r) {
                const int hcount = hist[r * nc + c];
                hist[r * nc + c] = run;
                run += hcount;
            }
        carry += blk;
    }
    const int total = carry;
    const int need = (total + SEG - 1) / SEG;
    const int capsegs = (int)((P.bstart[t + 1] - P.bstart[t]) / SEG);
    if (need > capsegs) {
        if (tid == 0) atomicOr(a.step_flags, 2);
        return;
    }
    __syncthreads();
    // 4. stable ranks inside each range, then the copy into the spare set
    {
        // two segments ahead: the next two are in flight while one is ranked and stored
        int n_a = 0, n_b = 0;
        PState<R> v_a, v_b;
        if (j0w < j1w) {
            n_a = P.segn[tb + j0w];
            load_particle(P, false, to + (int64_t)j0w * SEG + lane, v_a);
        }
        if (j0w + 1 < j1w) {
            n_b = P.segn[tb + j0w + 1];
            load_particle(P, false, to + (int64_t)(j0w + 1) * SEG + lane, v_b);
        }
        for (int j = j0w; j < j1w; ++j) {
            const int n = n_a;
            const PState<R> v = v_a;
            n_a = n_b;
            v_a = v_b;
            if (j + 2 < j1w) {
                n_b = P.segn[tb + j + 2];
                load_particle(P, false, to + (int64_t)(j + 2) * SEG + lane, v_b);
            }
            const int loc = (lane < n) ? local_of(v.c) : -1;
            const unsigned m = __match_any_sync(FULL, loc >= 0 ? loc : -1 - lane);
            const int base = (loc >= 0) ? hist[wid * nc + loc] : 0;
            __syncwarp();
            if (loc >= 0) {
                if (lane == __ffs(m) - 1) hist[wid * nc + loc] = base + __popc(m);
                const int64_t dst = to + base + __popc(m & lt);
                if (kChecks && (dst < to || dst >= P.bstart[t + 1])) atomicOr(a.flags, FLAG_CHECK);
                else store_particle(P, dst, v);
            }
            __syncwarp();
        }
    }
    if (wid == TILE_WARPS - 1)
        for (int i0 = 0; i0 < narr; i0 += SEG) {
            const int i = i0 + lane;
            PState<R> v;
            int loc = -1;
            if (i < narr) {
                load_particle(P, true, arr[i], v);
                loc = local_of(v.c);
            }
            const unsigned m = __match_any_sync(FULL, loc >= 0 ? loc : -1 - lane);
            const int base = (loc >= 0) ? hist[TILE_WARPS * nc + loc] : 0;
            __syncwarp();
            if (loc >= 0) {
                if (lane == __ffs(m) - 1) hist[TILE_WARPS * nc + loc] = base + __popc(m);
                const int64_t dst = to + base + __popc(m & lt);
                if (kChecks && (dst < to || dst >= P.bstart[t + 1])) atomicOr(a.flags, FLAG_CHECK);
                else store_particle(P, dst, v);
            }
            __syncwarp();
        }
    // 5. dense counts of the new bin
    for (int j = tid; j < need; j += TILE_BS) P.segn2[tb + j] = min(SEG, total - j * SEG);
    if (tid == 0) P.useg2[t] = need;
}

// One block per (tile, species) in a batched launch (every tile of every run);
// a single run's launch visits only the tiles of its regroup list, a fixed
// grid striding over the list.
template <typename R, bool kBatch>
__global__ void __launch_bounds__(TILE_BS) k_regroup(const __grid_constant__ TileArgs<R> a0,
                                                     const TileArgs<R> *__restrict__ runs,
                                                     const int32_t *__restrict__ run_tiles, int nrun) {
    extern __shared__ int rsm[];
    const int s = blockIdx.y;
    if (kBatch) {
        int t = blockIdx.x;
        int lo = 0, hi = nrun;   // largest run with run_tiles[run] <= blockIdx.x
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (run_tiles[mid] <= t) lo = mid;
            else hi = mid;
        }
        t -= run_tiles[lo];
        const int32_t *guard = runs[lo].guard;
        if (guard && (*guard & 3)) return;   // the run's previous regroup failed: the host redoes its step
        regroup_one<R, kBatch>(runs[lo], t, s, rsm);
    } else {
        // tiles from the list in turn (a queue per species: bins differ widely in size)
        if (a0.guard && (*a0.guard & 3)) return;
        __shared__ int s_li;
        const int n = a0.list_n[1];
        for (;;) {
            if (threadIdx.x == 0) s_li = atomicAdd(&a0.list_n[2 + s], 1);
            __syncthreads();
            const int li = s_li;
            if (li >= n) break;
            regroup_one<R, kBatch>(a0, a0.rg_list[li], s, rsm);
            __syncthreads();   // the shared arrays (and s_li) are reused by the next tile
        }
    }
}

// Particles per tile (sum of its segment counts).
__global__ void k_tile_counts(const int32_t *__restrict__ bstart, const int32_t *__restrict__ useg,
                              const int32_t *__restrict__ segn, int32_t *__restrict__ tcount) {
    __shared__ int wsum[TILE_WARPS];
    const int t = blockIdx.x;
    const int64_t sb = bstart[t] / SEG;
    const int u = useg[t];
    int c = 0;
    for (int j = threadIdx.x; j < u; j += blockDim.x) c += segn[sb + j];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += wsum[w];
        tcount[t] = tot;
    }
}

// Self-test of the bounded wait (no counterpart in the paper): one thread
// arms an mbarrier for 16 bytes of transaction that no copy will deliver and
// waits on it with the push's bound (mbar_wait_bounded); the wait runs out
// and the thread sets the timeout flag instead of hanging.  No copy is in flight when
// the block leaves.
__global__ void k_wait_selftest(int32_t *flag) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 16);
    if (!mbar_wait_bounded(&bar, 0)) atomicOr(flag, 8);
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
    // looked up once (handles are created from several threads by the serving runtime)
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        return (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                    cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                   ? (EncodeTiledFn)p
                   : nullptr;
    }();
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
    int offBo, offBn, offAcc, offBar, offScr, offCanary, offQ, offEc, offBc, bytes;
    uint32_t tma_bytes;
};

static Carve carve(const pic_t *h) {
    size_t v4 = 4 * h->rs;
    int EW = h->tnx + 1, EH = h->tny + 1, RW = h->tnx + 2 * h->halo + 1, RH = h->tny + 2 * h->halo + 1;
    Carve c;
    c.offBar = 0;
    c.offScr = 16;
    size_t o = SMEM_HEADER + align_up(EW * EH * v4, 128);
    c.offBo = (int)o;
    if (h->fp32) o += align_up(EW * EH * v4, 128);   // the FP64 form carries b: no push B tile
    c.offBn = (int)o;
    o += align_up(RW * RH * v4, 128);
    c.offAcc = (int)o;
    // shared moment accumulator of the FP32 form (fixed point when deterministic)
    const size_t acc_es = h->fp32 ? (h->det ? 8 : 4) : 0;
    o += align_up((size_t)NMOM * RW * RH * acc_es, 16);
    c.offQ = (int)o;
    if (h->fp32) o += (size_t)TILE_WARPS * QCAP * QWORDS * sizeof(float);
    // FP64: the cell coefficients (three V4 per cell) of the E tile and of the deposit region
    c.offEc = (int)o;
    if (!h->fp32) o += align_up((size_t)h->tnx * h->tny * 3 * v4, 128);
    c.offBc = (int)o;
    if (!h->fp32) o += align_up((size_t)(RW - 1) * (RH - 1) * 3 * v4, 128);
    c.offCanary = (int)o;
    if (kChecks) o += 4 * sizeof(uint32_t);
    c.bytes = (int)align_up(o, 128);
    // E^{n+1/2} and deposit B tiles; the push B tile too in the FP32 form (the FP64 form carries b)
    c.tma_bytes = (uint32_t)(((h->fp32 ? 2 : 1) * EW * EH + RW * RH) * v4);
    return c;
}

template <typename R, bool kFix, bool kBatch = false>
static int push_occupancy(pic_t *h, int bytes, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_push<R, kFix, kBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_push<R, kFix, kBatch>, TILE_BS, bytes);
    if (e != cudaSuccess) {
        set_error("push kernel set-up: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    return 0;
}

// The distinct neighbour tiles of every tile (periodic in y, and in x when
// the box is), ascending: the sources of its arrivals.
static int neighbour_table(pic_t *h) {
    std::vector<int32_t> tab((size_t)h->ntiles * 9, 0);
    for (int t = 0; t < h->ntiles; ++t) {
        const int tx = t % h->ntx, ty = t / h->ntx;
        int n = 0, nb[8];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                int x = tx + dx;
                if (h->periodic_x) x = (x + h->ntx) % h->ntx;
                else if (x < 0 || x >= h->ntx) continue;
                const int y = (ty + dy + h->nty) % h->nty;
                const int id = y * h->ntx + x;
                bool dup = (id == t);
                for (int q = 0; q < n; ++q) dup |= (nb[q] == id);
                if (!dup) nb[n++] = id;
            }
        std::sort(nb, nb + n);
        tab[(size_t)t * 9] = n;
        for (int q = 0; q < n; ++q) tab[(size_t)t * 9 + 1 + q] = nb[q];
    }
    if (cudaMalloc(&h->nbr, tab.size() * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        set_error("neighbour table allocation failed");
        return PIC_ERR_OOM;
    }
    if (cudaMemcpy(h->nbr, tab.data(), tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        set_error("neighbour table upload failed");
        return PIC_ERR_CUDA;
    }
    return 0;
}

int tile_setup(pic_t *h) {
    int RW = h->tnx + 2 * h->halo + 1, RH = h->tny + 2 * h->halo + 1;
    if (RW > 256 || RH > 256) {
        set_error("tile %dx%d with halo %d exceeds the 256-node TMA box", h->tnx, h->tny, h->halo);
        return PIC_ERR_ARG;
    }
    if (int rc = neighbour_table(h)) return rc;
    Carve c = carve(h);
    if (c.bytes > 220 * 1024) {
        set_error("tile %dx%d needs %d bytes of shared memory", h->tnx, h->tny, c.bytes);
        return PIC_ERR_ARG;
    }
    TMaps *tm = new TMaps();
    int rc = make_map(&tm->m[0], h->Ehalf, h->fp32, h->nxp, h->nyp, h->tnx + 1, h->tny + 1);
    if (!rc) rc = make_map(&tm->m[1], h->B[0], h->fp32, h->nxp, h->nyp, h->tnx + 1, h->tny + 1);
    if (!rc) rc = make_map(&tm->m[2], h->B[1], h->fp32, h->nxp, h->nyp, h->tnx + 1, h->tny + 1);
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
    h->tmaps = new Both{tm, dep};
    int per_sm = 0;
    if (h->det)
        rc = h->fp32 ? push_occupancy<float, true>(h, c.bytes, &per_sm) : push_occupancy<double, true>(h, c.bytes, &per_sm);
    else
        rc = h->fp32 ? push_occupancy<float, false>(h, c.bytes, &per_sm)
                     : push_occupancy<double, false>(h, c.bytes, &per_sm);
    if (rc) return rc;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    h->push_blocks = (per_sm > 0 ? per_sm : 1) * nsm;
    {
        // the spline-shape push: no shared memory, as many blocks as are resident (its heaviest
        // instance, degree 4, sets the count for all)
        int s2 = 0;
        cudaError_t es = h->fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s2, k_push_s<float, true, 4>, TILE_BS, 0)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s2, k_push_s<double, true, 4>, TILE_BS, 0);
        if (es != cudaSuccess || s2 < 1) {
            cudaGetLastError();
            s2 = 1;
        }
        h->push_blocks_s2 = s2 * nsm;
    }
    const int rb = regroup_smem_bytes(h->tnx * h->tny);
    cudaError_t e = h->fp32
                        ? cudaFuncSetAttribute(k_regroup<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rb)
                        : cudaFuncSetAttribute(k_regroup<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rb);
    if (e != cudaSuccess) {
        set_error("regroup kernel set-up: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    // the list-driven regroup: as many blocks per species as fit on the GPU at once (at most one per tile)
    int rper = 0;
    e = h->fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper, k_regroup<float, false>, TILE_BS, rb)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rper, k_regroup<double, false>, TILE_BS, rb);
    if (e != cudaSuccess || rper < 1) rper = 1;
    int64_t rb_total = (int64_t)rper * nsm / (h->nsp > 0 ? h->nsp : 1);
    if (rb_total < 1) rb_total = 1;
    if (rb_total > h->ntiles) rb_total = h->ntiles;
    h->regroup_blocks = (int)rb_total;
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
    if (h->items) cudaFree(h->items);
    h->items = nullptr;
    h->items_cap = 0;
    if (h->nbr) cudaFree(h->nbr);
    h->nbr = nullptr;
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
    a.offCanary = c.offCanary;
    a.offQ = c.offQ;
    a.offEc = c.offEc;
    a.offBc = c.offBc;
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
        p.bstart = S.bstart;
        p.useg = S.useg[S.scur]; p.segn = S.segn[S.scur];
        p.useg2 = S.useg[1 - S.scur]; p.segn2 = S.segn[1 - S.scur];
        const int o = S.spare;
        p.ocell = S.cell[o]; p.oox = (R *)S.ox[o]; p.ooy = (R *)S.oy[o];
        p.oux = (R *)S.ux[o]; p.ouy = (R *)S.uy[o]; p.ouz = (R *)S.uz[o]; p.ow = (R *)S.w[o];
        p.segml = S.segml;
        p.removed = (unsigned long long *)(h->d_removed + s);
        p.cr = S.carry[b]; p.mcr = S.carry[m]; p.ocr = S.carry[o];
        p.ccap = S.cap;
        p.q = (R)S.q; p.m = (R)S.m; p.kq = (R)(S.q * h->cfg.dt / (2.0 * S.m));
        p.cq2 = (R)(S.q * S.q * h->cfg.dt * h->cfg.dt / (4.0 * S.m));
        p.hq = (R)(S.q * h->cfg.dt * h->cfg.dt / (4.0 * S.m));
    }
    a.magic_nx = (uint32_t)((0x100000000ull + (uint64_t)h->nx - 1) / (uint64_t)h->nx);
    a.sdx = (R)(h->cfg.dt / h->cfg.dx);
    a.sdy = (R)(h->cfg.dt / h->cfg.dy);
    a.M = (R *)h->M;
    a.Mlo = (R *)h->Mlo;
    a.Mc = h->Mc;
    a.Mfix = h->Mfix;
    a.fs = FixScale{};
    a.Bnew = (const V4<R> *)h->B[1 - h->bcur];
    a.Eh = (const V4<R> *)h->Ehalf;
    a.Bo = (const V4<R> *)h->B[h->bcur];
    a.step_flags = h->d_step_flags + (h->step & 1);
    a.guard = h->guard;
    a.flags = h->d_flags;
    a.chunk_prefix = h->chunk_prefix;
    a.items = h->items;
    a.nbr = h->nbr;
    a.ticket = h->ticket;
    a.ch = item_segs(h);
    a.rg_list = h->rg_list;
    a.list_n = h->list_n;
    return a;
}

int push_work_list(pic_t *h) {
    UsegPtrs u;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s) u.p[s] = (s < h->nsp) ? h->sp[s].useg[h->sp[s].scur] : nullptr;
    const int nitems = h->nsp * h->ntiles;
    k_chunk_counts<<<(nitems + 256) / 256, 256, 0, h->st>>>(u, h->nsp, h->ntiles, item_segs(h), h->chunk_prefix,
                                                            h->ticket, h->occ);
    count_launch(h);
    return scan_i32_inplace(h, h->chunk_prefix, nitems + 1);
}

// The touch and regroup lists and the regroup queues, emptied for the next
// push (after whatever read the previous push's lists: the clear of its tiles).
int reset_lists(pic_t *h) {
    if (cudaMemsetAsync(h->list_n, 0, (2 + PIC_MAX_SPECIES) * sizeof(int32_t), h->st) != cudaSuccess)
        return check_launch("tile lists");
    return 0;
}

// ---------------------------------------------------------------------------- batched runs

size_t batch_args_bytes() {
    return sizeof(TileArgs<double>) > sizeof(TileArgs<float>) ? sizeof(TileArgs<double>) : sizeof(TileArgs<float>);
}

// Exclusive prefix of the runs' work-item totals (none for a run whose
// previous regroup failed: the host redoes its step); resets the batch queue.
template <typename R>
__global__ void k_batch_items(const TileArgs<R> *__restrict__ runs, int n, int32_t *__restrict__ items,
                              int32_t *__restrict__ ticket) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int acc = 0;
    for (int r = 0; r < n; ++r) {
        items[r] = acc;
        const TileArgs<R> &a = runs[r];
        if (!(a.guard && (*a.guard & 3))) acc += a.chunk_prefix[a.nsp * a.ntiles];
    }
    items[n] = acc;
    *ticket = 0;
}

template <typename R, bool kFix>
static int batch_push_t(BatchScratch &b, pic_t **hs, int n) {
    struct Both {
        TMaps *a;
        CUtensorMap *b;
    };
    // two staging slots alternate: a slot is rewritten only after its upload
    // of two steps ago has completed, so the host rarely waits here
    b.slot ^= 1;
    if (cudaEventSynchronize(b.ev_stage[b.slot]) != cudaSuccess) return check_launch("batch staging");
    TileArgs<R> *ha = (TileArgs<R> *)b.args_host[b.slot];
    int smem = 0;
    int32_t *tiles = b.idx_host[b.slot];
    tiles[0] = 0;
    for (int r = 0; r < n; ++r) {
        ha[r] = tile_args<R>(hs[r]);
        if (hs[r]->det)
            if (int rc = fix_scale(hs[r], &ha[r].fs)) return rc;
        const int bytes = carve(hs[r]).bytes;
        if (bytes > smem) smem = bytes;
        tiles[r + 1] = tiles[r] + hs[r]->ntiles;
    }
    int32_t *items = b.idx, *tiles_dev = b.idx + (b.cap + 1), *ticket = b.idx + 2 * (b.cap + 1);
    cudaMemcpyAsync(b.args_dev, ha, (size_t)n * sizeof(TileArgs<R>), cudaMemcpyHostToDevice, b.st);
    cudaMemcpyAsync(tiles_dev, tiles, (size_t)(n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, b.st);
    cudaEventRecord(b.ev_stage[b.slot], b.st);
    const TileArgs<R> *dargs = (const TileArgs<R> *)b.args_dev;
    k_batch_items<R><<<1, 32, 0, b.st>>>(dargs, n, items, ticket);
    int per_sm = 0;
    if (int rc = push_occupancy<R, kFix, true>(hs[0], smem, &per_sm)) return rc;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    TileArgs<R> a0 = ha[0];
    a0.ticket = ticket;
    Both *both = (Both *)hs[0]->tmaps;   // unused by the batched form; any valid descriptors
    k_push<R, kFix, true><<<(per_sm > 0 ? per_sm : 1) * nsm, TILE_BS, smem, b.st>>>(
        a0, dargs, items, n, both->a->m[0], both->a->m[1], both->b[0]);
    for (int r = 0; r < n; ++r) count_launch(hs[r]);
    return check_launch("k_push (batched)");
}

int batch_push(BatchScratch &b, pic_t **hs, int n) {
    pic_t *h = hs[0];
    if (h->fp32) return h->det ? batch_push_t<float, true>(b, hs, n) : batch_push_t<float, false>(b, hs, n);
    return h->det ? batch_push_t<double, true>(b, hs, n) : batch_push_t<double, false>(b, hs, n);
}

template <typename R>
static int batch_regroup_t(BatchScratch &b, pic_t **hs, int n) {
    int smem = 0, nsp = 0;
    for (int r = 0; r < n; ++r) {
        const int bytes = regroup_smem_bytes(hs[r]->tnx * hs[r]->tny);
        if (bytes > smem) smem = bytes;
        if (hs[r]->nsp > nsp) nsp = hs[r]->nsp;
    }
    if (cudaFuncSetAttribute(k_regroup<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return check_launch("regroup (batched) set-up");
    const TileArgs<R> *dargs = (const TileArgs<R> *)b.args_dev;
    const int32_t *tiles_dev = b.idx + (b.cap + 1);
    const int total = b.idx_host[b.slot][n];
    TileArgs<R> a0 = ((const TileArgs<R> *)b.args_host[b.slot])[0];
    k_regroup<R, true><<<dim3(total, nsp), TILE_BS, smem, b.st>>>(a0, dargs, tiles_dev, n);
    for (int r = 0; r < n; ++r) count_launch(hs[r]);
    return check_launch("k_regroup (batched)");
}

int batch_regroup(BatchScratch &b, pic_t **hs, int n) {
    return hs[0]->fp32 ? batch_regroup_t<float>(b, hs, n) : batch_regroup_t<double>(b, hs, n);
}

// Node moments from the cell sums of the FP64 deposit (deposit_fp64_cell):
// every cell of a listed tile (list == nullptr: of every tile) adds its corner
// values (0,0) A - X - Y + Z, (1,0) X - Z, (0,1) Y - Z, (1,1) Z of each moment
// into the node moments (zero before: the field solve or the deposit at rest
// has cleared them) and zeroes its sums.  A cell is read by one thread only;
// the corner nodes take L2 reductions.
__global__ void __launch_bounds__(256) k_cell_moments(const int32_t *__restrict__ list,
                                                      const int32_t *__restrict__ list_n, int tnx, int tny, int ntx,
                                                      int ntiles, GridArgs<double> g, double *__restrict__ Mc,
                                                      double *__restrict__ M, const int32_t *__restrict__ guard) {
    if (guard && (*guard & 3)) return;
    const int tc = tnx * tny;
    const int64_t ncell = (int64_t)g.nx * g.ny;
    const int64_t total = (int64_t)(list ? list_n[0] : ntiles) * tc;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int li = (int)(w / tc), c = (int)(w - (int64_t)li * tc);
        const int T = list ? list[li] : li, tx = T % ntx, ty = T / ntx;
        const int ly = c / tnx;
        const int cx = tx * tnx + (c - ly * tnx), cy = ty * tny + ly;
        if (cx >= g.nx || cy >= g.ny) continue;
        const int64_t cell = (int64_t)cy * g.nx + cx;
        const int64_t n00 = node_of(g, cx, cy, 0, 0), n10 = node_of(g, cx, cy, 1, 0);
        const int64_t n01 = node_of(g, cx, cy, 0, 1), n11 = node_of(g, cx, cy, 1, 1);
#pragma unroll
        for (int k = 0; k < NMOM; ++k) {
            V4<double> *q = (V4<double> *)(Mc + ((int64_t)k * ncell + cell) * 4);
            const V4<double> s = *q;
            const double A = s.x, X = s.y, Y = s.z, Z = s.w;
            if (A == 0.0 && X == 0.0 && Y == 0.0 && Z == 0.0) continue;
            *q = V4<double>{0.0, 0.0, 0.0, 0.0};
            double *m = M + (int64_t)k * g.nnode;
            atomicAdd(m + n00, (A - X) - (Y - Z));
            atomicAdd(m + n10, X - Z);
            atomicAdd(m + n01, Y - Z);
            atomicAdd(m + n11, Z);
        }
    }
}

int cell_moments(pic_t *h, bool all) {
    if (!h->Mc) return 0;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    k_cell_moments<<<(unsigned)(nsm > 0 ? 4 * nsm : 512), 256, 0, h->st>>>(
        all ? nullptr : h->touch_list, h->list_n, h->tnx, h->tny, h->ntx, h->ntiles, grid_args<double>(h), h->Mc,
        (double *)h->M, all ? nullptr : h->guard);
    count_launch(h);
    return check_launch("k_cell_moments");
}

// The push's work items in one block, for up to PREP_ONE_BLOCK (species, tile)
// entries: the same counts, occupancy bytes, exclusive prefix (total at the
// end) and item table as k_chunk_counts + scan + k_item_table, without the
// launches between them (they sit between the regroup and the next push).
// The segment counts are read once, coalesced, into shared memory.
constexpr int PREP_BS = 1024;
constexpr int PREP_ONE_BLOCK = 16 * 1024;
__global__ void __launch_bounds__(PREP_BS) k_prep_one_block(UsegPtrs u, int nsp, int ntiles, int ch,
                                                            int32_t *__restrict__ prefix, int32_t *__restrict__ ticket,
                                                            uint8_t *__restrict__ occ, int2 *__restrict__ items) {
    extern __shared__ int cnt[];   // [nsp * ntiles] segment counts, then chunk counts
    __shared__ int wsum[PREP_BS / 32];
    const int n = nsp * ntiles, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    {
        // every load in flight before the first store (n <= PREP_ONE_BLOCK)
        constexpr int PER = PREP_ONE_BLOCK / PREP_BS;
        int v[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * PREP_BS;
            const int ic = (i < n) ? i : 0;   // an in-range index even where the load is not taken
            const int s = ic / ntiles;
            v[k] = (i < n) ? u.p[s][ic - s * ntiles] : 0;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k)
            if (tid + k * PREP_BS < n) cnt[tid + k * PREP_BS] = v[k];
    }
    __syncthreads();
    for (int t = tid; t < ntiles; t += PREP_BS) {   // occupancy of the tile by any species at the start of the push
        int any = 0;
        for (int q = 0; q < nsp; ++q) any |= cnt[q * ntiles + t];
        occ[t] = any != 0;
    }
    __syncthreads();
    for (int i = tid; i < n; i += PREP_BS) cnt[i] = (cnt[i] + ch - 1) / ch;
    __syncthreads();
    const int per = (n + PREP_BS - 1) / PREP_BS;
    const int i0 = min(tid * per, n), i1 = min(i0 + per, n);
    int local = 0;
    for (int i = i0; i < i1; ++i) local += cnt[i];
    // exclusive block scan of the per-thread sums (entries are contiguous per thread)
    int incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int x = wsum[lane];
        int xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, xi, o);
            if (lane >= o) xi += y;
        }
        wsum[lane] = xi - x;
    }
    __syncthreads();
    int run = wsum[wid] + incl - local;
    for (int i = i0; i < i1; ++i) {
        const int c = cnt[i];
        prefix[i] = run;
        for (int k = 0; k < c; ++k) items[run + k] = make_int2(i, k);
        run += c;
    }
    if (tid == PREP_BS - 1) {
        prefix[n] = run;   // the last thread's running sum is the total
        *ticket = 0;
    }
}

// The push's work items: the chunk counts of every (species, tile), their scan
// and the item table, from the bins' layout in slot next ? scur ^ 1 : scur of
// each species (next: the slot the pending per-tile regroup writes, so that a
// step can prepare its push before the host has seen that regroup's flags).
int push_prep(pic_t *h, bool next) {
    UsegPtrs u;
    for (int s = 0; s < PIC_MAX_SPECIES; ++s)
        u.p[s] = (s < h->nsp) ? h->sp[s].useg[next ? h->sp[s].scur ^ 1 : h->sp[s].scur] : nullptr;
    const int nitems = h->nsp * h->ntiles;
    // item table: at most one item per used segment (grown before any launch that would use it)
    int64_t need = 1;
    for (int s = 0; s < h->nsp; ++s) need += h->sp[s].cap / SEG;
    if (need > h->items_cap) {
        cudaFree(h->items);
        h->items = nullptr;
        h->items_cap = 0;
        if (cudaMalloc(&h->items, (size_t)need * sizeof(int2)) != cudaSuccess) {
            cudaGetLastError();
            set_error("push item table allocation failed");
            return PIC_ERR_OOM;
        }
        h->items_cap = need;
    }
    if (nitems <= PREP_ONE_BLOCK) {
        const int sm = nitems * (int)sizeof(int);
        if (sm > 48 * 1024 && cudaFuncSetAttribute(k_prep_one_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   PREP_ONE_BLOCK * (int)sizeof(int)) != cudaSuccess)
            return check_launch("push work items set-up");
        k_prep_one_block<<<1, PREP_BS, sm, h->st>>>(u, h->nsp, h->ntiles, item_segs(h), h->chunk_prefix, h->ticket,
                                                    h->occ, h->items);
        count_launch(h);
        return check_launch("push work items");
    }
    k_chunk_counts<<<(nitems + 256) / 256, 256, 0, h->st>>>(u, h->nsp, h->ntiles, item_segs(h), h->chunk_prefix,
                                                            h->ticket, h->occ);
    count_launch(h);
    if (int rc = scan_i32_inplace(h, h->chunk_prefix, nitems + 1)) return rc;
    k_item_table<<<(nitems + 255) / 256, 256, 0, h->st>>>(h->chunk_prefix, nitems, h->items);
    count_launch(h);
    return check_launch("push work items");
}

template <typename R>
static int particle_tiles_t(pic_t *h, bool prepared) {
    struct Both {
        TMaps *a;
        CUtensorMap *b;
    };
    Both *both = (Both *)h->tmaps;
    if (!prepared)
        if (int rc = push_prep(h, false)) return rc;
    TileArgs<R> a = tile_args<R>(h);
    if (h->det)
        if (int rc = fix_scale(h, &a.fs)) return rc;
    Carve c = carve(h);
    const CUtensorMap &mE = both->a->m[0];
    const CUtensorMap &mBo = both->a->m[1 + h->bcur];
    const CUtensorMap &mBn = both->b[1 - h->bcur];
    if (h->shape >= 2) {
        const unsigned nb = (unsigned)h->push_blocks_s2;
        switch (h->shape * 2 + (h->det ? 1 : 0)) {
            case 4: k_push_s<R, false, 2><<<nb, TILE_BS, 0, h->st>>>(a); break;
            case 5: k_push_s<R, true, 2><<<nb, TILE_BS, 0, h->st>>>(a); break;
            case 6: k_push_s<R, false, 3><<<nb, TILE_BS, 0, h->st>>>(a); break;
            case 7: k_push_s<R, true, 3><<<nb, TILE_BS, 0, h->st>>>(a); break;
            case 8: k_push_s<R, false, 4><<<nb, TILE_BS, 0, h->st>>>(a); break;
            default: k_push_s<R, true, 4><<<nb, TILE_BS, 0, h->st>>>(a); break;
        }
        count_launch(h);
        return check_launch("k_push_s");
    }
    if (h->det) k_push<R, true, false><<<h->push_blocks, TILE_BS, c.bytes, h->st>>>(a, nullptr, nullptr, 0, mE, mBo, mBn);
    else k_push<R, false, false><<<h->push_blocks, TILE_BS, c.bytes, h->st>>>(a, nullptr, nullptr, 0, mE, mBo, mBn);
    count_launch(h);
    return check_launch("k_push");
}

int particle_tiles(pic_t *h, bool prepared) {
    return h->fp32 ? particle_tiles_t<float>(h, prepared) : particle_tiles_t<double>(h, prepared);
}

template <typename R>
static int regroup_t(pic_t *h) {
    TileArgs<R> a = tile_args<R>(h);
    k_regroup<R, false><<<dim3(h->regroup_blocks, h->nsp), TILE_BS, regroup_smem_bytes(h->tnx * h->tny), h->st>>>(a, nullptr,
                                                                                                       nullptr, 0);
    count_launch(h);
    return check_launch("k_regroup");
}

int regroup_tiles(pic_t *h) { return h->fp32 ? regroup_t<float>(h) : regroup_t<double>(h); }

int tile_counts(pic_t *h, int s) {
    SpeciesBuf &S = h->sp[s];
    k_tile_counts<<<h->ntiles, 256, 0, h->st>>>(S.bstart, S.useg[S.scur], S.segn[S.scur], S.tcount);
    count_launch(h);
    return check_launch("k_tile_counts");
}

}  // namespace pic

extern "C" PIC_API int pic_selftest_wait(void *cuda_stream, double *seconds) {
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int32_t *d_flag = nullptr, flag = 0;
    if (cudaMalloc(&d_flag, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_OOM;
    }
    cudaMemsetAsync(d_flag, 0, sizeof(int32_t), st);
    auto t0 = std::chrono::steady_clock::now();
    pic::k_wait_selftest<<<1, 32, 0, st>>>(d_flag);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    cudaFree(d_flag);
    if (e != cudaSuccess) return PIC_ERR_CUDA;
    return (flag & 8) ? PIC_ERR_TIMEOUT : PIC_OK;
}
