// Stable regrouping of a species by tile (the one-GPU counterpart of the
// paper's particle migration between strip processors, Section 3.3): a stable
// LSD radix sort of 32-bit keys with 8-bit digits, then one gather of every
// particle array through the resulting permutation.
//
// Keys: 2*tile + (particle arrived from another tile this step), so that each
// tile keeps first the particles that stayed, in their previous order, then
// the arrivals in their previous order; removed particles carry the largest
// key and end up past the live count.
#include "pic_internal.cuh"

namespace pic {

constexpr int RADIX = 256;
constexpr int SORT_BS = 256;
constexpr int SORT_ROUNDS = 16;
constexpr int SORT_IPB = SORT_BS * SORT_ROUNDS;   // items per block
constexpr int SCAN_BS = 1024;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_IPB = SCAN_BS * SCAN_IPT;

static int64_t sort_blocks(int64_t n) { return (n + SORT_IPB - 1) / SORT_IPB; }

__global__ void k_iota(uint32_t *v, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) v[t] = (uint32_t)t;
}

// Per-block digit histogram, stored digit-major: hist[d * nblocks + b].
__global__ void k_radix_hist(const uint32_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist,
                             int64_t nblocks) {
    __shared__ uint32_t h[RADIX];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * SORT_IPB;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        int64_t i = base + (int64_t)r * SORT_BS + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan, three phases: per-block scan + block totals, scan of the
// totals in one block, add back.
__global__ void k_scan_local(uint32_t *__restrict__ a, int64_t n, uint32_t *__restrict__ sums) {
    __shared__ uint32_t wsum[SCAN_BS / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_IPB + (int64_t)threadIdx.x * SCAN_IPT;
    uint32_t v[SCAN_IPT];
    uint32_t tot = 0;
    for (int k = 0; k < SCAN_IPT; ++k) {
        int64_t i = base + k;
        v[k] = (i < n) ? a[i] : 0u;
        tot += v[k];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t x = (lane < SCAN_BS / 32) ? wsum[lane] : 0u;
        uint32_t xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        if (lane < SCAN_BS / 32) wsum[lane] = xi - x;  // exclusive warp offsets
        if (lane == 31 && sums) sums[blockIdx.x] = xi;
    }
    __syncthreads();
    uint32_t run = wsum[wid] + incl - tot;
    for (int k = 0; k < SCAN_IPT; ++k) {
        int64_t i = base + k;
        if (i < n) a[i] = run;
        run += v[k];
    }
}

__global__ void k_scan_add(uint32_t *__restrict__ a, int64_t n, const uint32_t *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_IPB;
    uint32_t add = sums[blockIdx.x];
    for (int k = threadIdx.x; k < SCAN_IPB; k += SCAN_BS) {
        int64_t i = base + k;
        if (i < n) a[i] += add;
    }
}

// Stable scatter: items of a block are taken in order, 256 per round; within a
// round, rank = digit offset so far + earlier warps' count + earlier lanes' count.
__global__ void k_radix_scatter(const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, int64_t n,
                                int shift, const uint32_t *__restrict__ offs, int64_t nblocks,
                                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout) {
    __shared__ uint32_t run[RADIX];
    __shared__ uint32_t wcnt[SORT_BS / 32][RADIX];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * SORT_IPB;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        for (int w = 0; w < SORT_BS / 32; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        int64_t i = base + (int64_t)r * SORT_BS + threadIdx.x;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t val = valid ? vin[i] : 0u;
        int d = valid ? (int)((key >> shift) & (RADIX - 1)) : RADIX;
        unsigned mask = __match_any_sync(0xffffffffu, d);
        int rank = __popc(mask & lt);
        if (valid && (__ffs(mask) - 1) == lane) wcnt[wid][d] = (uint32_t)__popc(mask);
        __syncthreads();
        uint32_t acc = 0;
        for (int w = 0; w < SORT_BS / 32; ++w) {
            uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = acc;
            acc += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = run[d] + wcnt[wid][d] + (uint32_t)rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        run[threadIdx.x] += acc;
        __syncthreads();
    }
}

// --------------------------------------------------------------------------- full rebuild kernels

constexpr uint32_t DEAD = 0xFFFFFFFFu;

// Keys of the particle order: tile * cpt + (ly * tile_nx + lx), the cell
// inside the tile in row-major order (cpt = tile_nx * tile_ny).
struct KeyGeom {
    int nx, tnx, tny, ntx;
    uint32_t cpt;
};

__device__ inline uint32_t order_key(const KeyGeom &k, int32_t c) {
    const int cx = c % k.nx, cy = c / k.nx;
    const int tx = cx / k.tnx, ty = cy / k.tny;
    return (uint32_t)(ty * k.ntx + tx) * k.cpt + (uint32_t)((cy - ty * k.tny) * k.tnx + (cx - tx * k.tnx));
}

// keys of the bins part (the valid entries of every bin's segments)
__global__ void k_keys_bins(const int32_t *__restrict__ bstart, const int32_t *__restrict__ useg,
                            const int32_t *__restrict__ segn, const int32_t *__restrict__ cell, KeyGeom kg,
                            uint32_t *__restrict__ keys) {
    const int t = blockIdx.x;
    const int64_t b0 = bstart[t];
    const int u = useg[t];
    for (int64_t i = threadIdx.x; i < (int64_t)u * SEG; i += blockDim.x) {
        const int64_t j = i / SEG;
        if ((int)(i - j * SEG) < segn[b0 / SEG + j]) keys[b0 + i] = order_key(kg, cell[b0 + i]);
    }
}

// keys of the mirror part (the leavers of every bin's segments, at their new cells)
__global__ void k_keys_mirror(const int32_t *__restrict__ bstart, const int32_t *__restrict__ useg,
                              const int32_t *__restrict__ segml, const int32_t *__restrict__ mcell, KeyGeom kg,
                              int64_t cap, uint32_t *__restrict__ keys) {
    const int t = blockIdx.x;
    const int64_t b0 = bstart[t];
    const int u = useg[t];
    for (int64_t i = threadIdx.x; i < (int64_t)u * SEG; i += blockDim.x) {
        const int64_t j = i / SEG;
        if ((int)(i - j * SEG) < segml[b0 / SEG + j]) keys[cap + b0 + i] = order_key(kg, mcell[b0 + i]);
    }
}

// keys of freshly loaded particles (compact, in load order), from key index off
__global__ void k_keys_stage(const int32_t *__restrict__ cell, int64_t n, KeyGeom kg, int64_t off,
                             uint32_t *__restrict__ keys) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    keys[off + p] = order_key(kg, cell[p]);
}

// start / end of each tile's run in the sorted keys (tile = key / div)
__global__ void k_run_bounds(const uint32_t *__restrict__ keys, int64_t n, uint32_t div, int32_t *__restrict__ cstart,
                             int32_t *__restrict__ cend) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t k = keys[p];
    if (k == DEAD) return;
    uint32_t t = k / div;
    if (p == 0 || keys[p - 1] / div != t) cstart[t] = (int32_t)p;
    if (p + 1 == n || keys[p + 1] == DEAD || keys[p + 1] / div != t) cend[t] = (int32_t)(p + 1);
}

// New bins from the run lengths: capacity count + count/4 + 32 per tile while
// the buffer allows it, else exactly count; bstart is the exclusive scan.  If
// even the exact counts do not fit (cannot happen when the live count only
// shrinks), every bin is emptied and the capacity flag is raised.
__device__ inline long long block_excl_scan(long long c, long long *wsum, long long &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long x = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
        long long xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        wsum[lane] = xi - x;
        if (lane == 31) wsum[32] = xi;
    }
    __syncthreads();
    long long ex = wsum[wid] + incl - c;
    total = wsum[32];
    __syncthreads();
    return ex;
}

__global__ void k_layout(const int32_t *__restrict__ cstart, const int32_t *__restrict__ cend, int ntiles,
                         int64_t cap, int32_t *__restrict__ bstart, int32_t *__restrict__ tcount,
                         int32_t *__restrict__ useg, int32_t *__restrict__ flags) {
    __shared__ long long wsum[33];
    long long tot_slack = 0, tot_tight = 0;
    auto rnd = [](long long v) { return (v + SEG - 1) / SEG * SEG; };
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int t = base + threadIdx.x;
        long long cnt = (t < ntiles) ? (long long)(cend[t] - cstart[t]) : 0;
        long long ts, tt;
        block_excl_scan((t < ntiles) ? rnd(cnt + cnt / 4 + 2 * SEG) : 0, wsum, ts);
        block_excl_scan((t < ntiles) ? rnd(cnt) : 0, wsum, tt);
        tot_slack += ts;
        tot_tight += tt;
    }
    const int mode = (tot_slack <= cap) ? 0 : (tot_tight <= cap ? 1 : 2);
    long long carry = 0;
    for (int base = 0; base < ntiles; base += blockDim.x) {
        int t = base + threadIdx.x;
        long long cnt = (t < ntiles && mode != 2) ? (long long)(cend[t] - cstart[t]) : 0;
        long long c = (t < ntiles) ? (mode == 0 ? rnd(cnt + cnt / 4 + 2 * SEG) : rnd(cnt)) : 0;
        if (mode == 2) c = 0;
        long long tot;
        long long ex = block_excl_scan(c, wsum, tot);
        if (t < ntiles) {
            bstart[t] = (int32_t)(carry + ex);
            tcount[t] = (int32_t)cnt;
            useg[t] = (int32_t)((cnt + SEG - 1) / SEG);
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        bstart[ntiles] = (int32_t)carry;
        if (mode == 2) atomicOr(flags, 4);
    }
}

// Segment counts of a dense bin: full segments, then the remainder.
__global__ void k_layout_segs(const int32_t *__restrict__ bstart, const int32_t *__restrict__ tcount,
                              int32_t *__restrict__ segn) {
    const int t = blockIdx.x;
    const int64_t sb = bstart[t] / SEG;
    const int cnt = tcount[t];
    const int u = (cnt + SEG - 1) / SEG;
    for (int j = threadIdx.x; j < u; j += blockDim.x) segn[sb + j] = min(SEG, cnt - j * SEG);
}

template <typename R>
struct Buf7 {
    int32_t *cell;
    R *a[6];
    double *cr;      // FP64 form: the carried quantities ([NCARRY][ccap]), else nullptr
    int64_t ccap;
};

template <typename R>
__global__ void k_rebuild_gather(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n,
                                 uint32_t div, int64_t cap, const int32_t *__restrict__ cstart,
                                 const int32_t *__restrict__ bstart, const int32_t *__restrict__ flags, Buf7<R> s0,
                                 Buf7<R> s1, Buf7<R> d) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    uint32_t k = keys[p];
    if (k == DEAD || (*flags & 4)) return;
    uint32_t t = k / div;
    uint32_t v = vals[p];
    const Buf7<R> &src = (v < cap) ? s0 : s1;
    int64_t si = (v < cap) ? (int64_t)v : (int64_t)v - cap;
    int64_t di = (int64_t)bstart[t] + (p - cstart[t]);
    d.cell[di] = src.cell[si];
#pragma unroll
    for (int q = 0; q < 6; ++q) d.a[q][di] = src.a[q][si];
    if (d.cr)   // (a load's new particles carry nothing yet: their deposit at rest fills the planes)
#pragma unroll
        for (int q = 0; q < NCARRY; ++q) d.cr[q * d.ccap + di] = src.cr[q * src.ccap + si];
}

// --------------------------------------------------------------------------- host side

static int scan(pic_t *h, uint32_t *a, int64_t n) {
    int64_t nb = (n + SCAN_IPB - 1) / SCAN_IPB;
    uint32_t *sums = h->hist + h->hist_cap - 2 * SCAN_IPB;  // tail of the scratch
    if (nb > SCAN_IPB) {
        set_error("radix sort: too many items (%lld)", (long long)n);
        return PIC_ERR_CAPACITY;
    }
    k_scan_local<<<(unsigned)nb, SCAN_BS, 0, h->st>>>(a, n, sums);
    count_launch(h);
    if (nb > 1) {
        k_scan_local<<<1, SCAN_BS, 0, h->st>>>(sums, nb, nullptr);
        count_launch(h);
        k_scan_add<<<(unsigned)nb, SCAN_BS, 0, h->st>>>(a, n, sums);
        count_launch(h);
    }
    return check_launch("scan");
}

int64_t sort_hist_entries(int64_t cap) { return RADIX * sort_blocks(cap) + 2 * SCAN_IPB; }

int ensure_sort_capacity(pic_t *h, int64_t n) {
    if (n <= h->sort_cap) return 0;
    int64_t cap = n + n / 8 + 4096;
    cudaStreamSynchronize(h->st);
    for (int k = 0; k < 2; ++k) {
        cudaFree(h->keys[k]);
        cudaFree(h->vals[k]);
        h->keys[k] = h->vals[k] = nullptr;
    }
    cudaFree(h->hist);
    h->hist = nullptr;
    int64_t hist_entries = RADIX * sort_blocks(cap) + 2 * SCAN_IPB;
    for (int k = 0; k < 2; ++k) {
        if (cudaMalloc(&h->keys[k], cap * sizeof(uint32_t)) != cudaSuccess ||
            cudaMalloc(&h->vals[k], cap * sizeof(uint32_t)) != cudaSuccess) {
            set_error("sort scratch allocation of %lld items failed", (long long)cap);
            cudaGetLastError();
            return PIC_ERR_OOM;
        }
    }
    if (cudaMalloc(&h->hist, hist_entries * sizeof(uint32_t)) != cudaSuccess) {
        set_error("sort histogram allocation failed");
        cudaGetLastError();
        return PIC_ERR_OOM;
    }
    h->sort_cap = cap;
    h->hist_cap = hist_entries;
    return 0;
}

// Stable radix sort of keys[0][0..n) (values = index); returns the index of
// the key/value buffers that hold the result.
static int radix_sort(pic_t *h, int64_t n, int bits, int *cur_out) {
    int passes = (bits + 7) / 8;
    int64_t nb = sort_blocks(n);
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(h->vals[0], n);
    count_launch(h);
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        k_radix_hist<<<(unsigned)nb, SORT_BS, 0, h->st>>>(h->keys[cur], n, shift, h->hist, nb);
        count_launch(h);
        if (int rc = check_launch("k_radix_hist")) return rc;
        if (int rc = scan(h, h->hist, RADIX * nb)) return rc;
        k_radix_scatter<<<(unsigned)nb, SORT_BS, 0, h->st>>>(h->keys[cur], h->vals[cur], n, shift, h->hist, nb,
                                                             h->keys[1 - cur], h->vals[1 - cur]);
        count_launch(h);
        if (int rc = check_launch("k_radix_scatter")) return rc;
        cur = 1 - cur;
    }
    *cur_out = cur;
    return 0;
}

template <typename R>
static Buf7<R> buf7(SpeciesBuf &S, int b) {
    Buf7<R> x;
    x.cell = S.cell[b];
    x.a[0] = (R *)S.ox[b]; x.a[1] = (R *)S.oy[b]; x.a[2] = (R *)S.ux[b];
    x.a[3] = (R *)S.uy[b]; x.a[4] = (R *)S.uz[b]; x.a[5] = (R *)S.w[b];
    x.cr = S.carry[b];
    x.ccap = S.cap;
    return x;
}

int64_t slots_needed(const pic_t *h, int64_t n) {
    int64_t v = n + n / 2 + (3 * SEG) * (int64_t)h->ntiles + 1024;
    return (v + SEG - 1) / SEG * SEG;
}

// Exclusive scan of n int32 values in place, many blocks (the per-block
// totals go to the handle's own scratch, so it needs no sort scratch).
int scan_i32_inplace(pic_t *h, int32_t *a, int64_t n) {
    int64_t nb = (n + SCAN_IPB - 1) / SCAN_IPB;
    if (nb > SCAN_IPB) {
        set_error("scan of %lld items exceeds the scratch", (long long)n);
        return PIC_ERR_CAPACITY;
    }
    uint32_t *u = (uint32_t *)a;
    k_scan_local<<<(unsigned)nb, SCAN_BS, 0, h->st>>>(u, n, h->scan_sums);
    count_launch(h);
    if (nb > 1) {
        k_scan_local<<<1, SCAN_BS, 0, h->st>>>(h->scan_sums, nb, nullptr);
        k_scan_add<<<(unsigned)nb, SCAN_BS, 0, h->st>>>(u, n, h->scan_sums);
        count_launch(h, 2);
    }
    return check_launch("scan");
}

int scan_sums_entries() { return SCAN_IPB; }

__global__ void k_copy_pad(const int32_t *__restrict__ in, int n, int32_t *__restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t <= n) out[t] = (t < n) ? in[t] : 0;
}

// out[0..ntiles] = exclusive scan of in[0..ntiles) with the total at out[ntiles].
int scan_tiles(pic_t *h, const int32_t *in, int32_t *out) {
    k_copy_pad<<<(h->ntiles + 256) / 256, 256, 0, h->st>>>(in, h->ntiles, out);
    count_launch(h);
    return scan_i32_inplace(h, out, h->ntiles + 1);
}

int init_empty_bins(pic_t *h, int s) {
    SpeciesBuf &S = h->sp[s];
    size_t b = (size_t)(h->ntiles + 1) * sizeof(int32_t);
    cudaMemsetAsync(S.bstart, 0, b, h->st);
    cudaMemsetAsync(S.useg[0], 0, b, h->st);
    cudaMemsetAsync(S.useg[1], 0, b, h->st);
    cudaMemsetAsync(S.tcount, 0, b, h->st);
    S.scur = 0;
    return check_launch("init_empty_bins");
}

// Full stable regroup of species s into fresh bins.  The items are the bins'
// valid entries followed by a second buffer: the mirror's leavers (after a
// step) or n_second freshly loaded particles in the spare buffer (after a
// load).  Key (tile, cell inside the tile), stable sort, new bins with slack,
// one gather.  Since every bin entry precedes every second-buffer entry, the
// particles of one cell keep the bins' order and then the second buffer's.
int rebuild_species(pic_t *h, int s, int source, int64_t n_second) {
    SpeciesBuf &S = h->sp[s];
    const int64_t cap = S.cap;
    if (cap == 0) return 0;
    // a load into an empty species sorts only the new particles
    const bool fresh = (source == REBUILD_FROM_LOAD && S.n == 0);
    const int64_t n = fresh ? n_second : 2 * cap;
    if (n == 0) return 0;
    if (int rc = ensure_sort_capacity(h, n)) return rc;
    cudaMemsetAsync(h->keys[0], 0xFF, n * sizeof(uint32_t), h->st);
    int32_t *useg = S.useg[S.scur], *segn = S.segn[S.scur];
    KeyGeom kg{h->nx, h->tnx, h->tny, h->ntx, (uint32_t)(h->tnx * h->tny)};
    const uint32_t div = kg.cpt;
    const int64_t maxkey = (int64_t)h->ntiles * kg.cpt;
    int second, out;
    if (!fresh) {
        k_keys_bins<<<h->ntiles, 256, 0, h->st>>>(S.bstart, useg, segn, S.cell[S.bins], kg, h->keys[0]);
        count_launch(h);
    }
    if (source == REBUILD_FROM_STEP) {
        k_keys_mirror<<<h->ntiles, 256, 0, h->st>>>(S.bstart, useg, S.segml, S.cell[S.mir], kg, cap, h->keys[0]);
        count_launch(h);
        second = S.mir;
        out = S.spare;
    } else {
        if (n_second > 0) {
            k_keys_stage<<<(unsigned)((n_second + 255) / 256), 256, 0, h->st>>>(S.cell[S.spare], n_second, kg,
                                                                              fresh ? 0 : cap, h->keys[0]);
            count_launch(h);
        }
        second = S.spare;
        out = S.mir;
    }
    if (int rc = check_launch("rebuild keys")) return rc;
    if (maxkey >= 0xFFFFFFFell) {
        set_error("regroup keys exceed 32 bits (%lld)", (long long)maxkey);
        return PIC_ERR_ARG;
    }
    int bits = 1;
    while (((1ll << bits) - 1) <= maxkey) ++bits;
    int cur = 0;
    if (int rc = radix_sort(h, n, bits, &cur)) return rc;
    size_t tb = (size_t)(h->ntiles + 1) * sizeof(int32_t);
    cudaMemsetAsync(S.cstart, 0, tb, h->st);
    cudaMemsetAsync(S.cend, 0, tb, h->st);
    k_run_bounds<<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(h->keys[cur], n, div, S.cstart, S.cend);
    count_launch(h);
    k_layout<<<1, 1024, 0, h->st>>>(S.cstart, S.cend, h->ntiles, cap, S.bstart, S.tcount, useg, h->d_flags);
    count_launch(h);
    k_layout_segs<<<h->ntiles, 256, 0, h->st>>>(S.bstart, S.tcount, segn);
    count_launch(h);
    if (int rc = check_launch("rebuild layout")) return rc;
    unsigned nbk = (unsigned)((n + 255) / 256);
    // item v < cap comes from the first buffer (the bins, or the new particles when fresh), else the second
    const int first = fresh ? second : S.bins;
    if (h->fp32)
        k_rebuild_gather<float><<<nbk, 256, 0, h->st>>>(h->keys[cur], h->vals[cur], n, div, cap, S.cstart, S.bstart,
                                                        h->d_flags, buf7<float>(S, first), buf7<float>(S, second),
                                                        buf7<float>(S, out));
    else
        k_rebuild_gather<double><<<nbk, 256, 0, h->st>>>(h->keys[cur], h->vals[cur], n, div, cap, S.cstart, S.bstart,
                                                         h->d_flags, buf7<double>(S, first),
                                                         buf7<double>(S, second), buf7<double>(S, out));
    count_launch(h);
    if (int rc = check_launch("k_rebuild_gather")) return rc;
    int old = S.bins;
    S.bins = out;
    if (source == REBUILD_FROM_LOAD) S.mir = old;
    else S.spare = old;
    return 0;
}

}  // namespace pic

// --------------------------------------------------------------------------- allocation-free key sort
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (for example a framework's caching allocator that has
// reserved the device), and latency-critical serving loops in which a
// cudaMalloc/cudaFree would synchronise the whole device.  For them,
// pic_sort_keys_noalloc runs the same stable radix sort as the particle
// regroup, with every scratch buffer carved out of one fixed file-scope device
// array instead of allocated memory.  The array is part of the library image:
// every GPU that loads the library holds it until the process exits.

#include <mutex>

namespace pic {

constexpr int64_t NOALLOC_MAX_KEYS = PIC_NOALLOC_MAX_KEYS;
constexpr int64_t NOALLOC_BLOCKS = (NOALLOC_MAX_KEYS + SORT_IPB - 1) / SORT_IPB;
constexpr int64_t NOALLOC_HIST = RADIX * NOALLOC_BLOCKS;
// two key buffers, two value buffers, the digit histogram, the scan's block sums
constexpr int64_t NOALLOC_WORDS = 4 * NOALLOC_MAX_KEYS + NOALLOC_HIST + SCAN_IPB;
static_assert((NOALLOC_HIST + SCAN_IPB - 1) / SCAN_IPB <= SCAN_IPB, "scan of the histogram needs one level of sums");

static __device__ __align__(256) uint32_t g_noalloc_scratch[NOALLOC_WORDS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static uint32_t *g_noalloc_dev[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  In host code the
// name g_noalloc_scratch is only a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.
static int noalloc_scratch(uint32_t **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("pic_sort_keys_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
        return PIC_ERR_CUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("pic_sort_keys_noalloc: device ordinal %d not supported", dev);
        return PIC_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_error("pic_sort_keys_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return PIC_ERR_CUDA;
        }
        g_noalloc_dev[dev] = (uint32_t *)p;
    }
    *out = g_noalloc_dev[dev];
    return PIC_OK;
}

static int scan_noalloc(uint32_t *a, int64_t n, uint32_t *sums, cudaStream_t st) {
    int64_t nb = (n + SCAN_IPB - 1) / SCAN_IPB;
    k_scan_local<<<(unsigned)nb, SCAN_BS, 0, st>>>(a, n, sums);
    if (nb > 1) {
        k_scan_local<<<1, SCAN_BS, 0, st>>>(sums, nb, nullptr);
        k_scan_add<<<(unsigned)nb, SCAN_BS, 0, st>>>(a, n, sums);
    }
    return check_launch("pic_sort_keys_noalloc scan");
}

}  // namespace pic

extern "C" PIC_API int pic_sort_keys_noalloc(const uint32_t *keys, int64_t n, uint32_t max_key, uint32_t *perm,
                                             void *cuda_stream) {
    using namespace pic;
    if (n < 0 || (n > 0 && (keys == nullptr || perm == nullptr))) {
        set_error("pic_sort_keys_noalloc: negative count or NULL pointer");
        return PIC_ERR_ARG;
    }
    if (n > NOALLOC_MAX_KEYS) {
        set_error("pic_sort_keys_noalloc: %lld keys exceed the fixed scratch limit of %lld", (long long)n,
                  (long long)NOALLOC_MAX_KEYS);
        return PIC_ERR_CAPACITY;
    }
    if (n == 0) return PIC_OK;
    uint32_t *s = nullptr;
    if (int rc = noalloc_scratch(&s)) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t *kbuf[2] = {s, s + NOALLOC_MAX_KEYS};
    uint32_t *vbuf[2] = {s + 2 * NOALLOC_MAX_KEYS, s + 3 * NOALLOC_MAX_KEYS};
    uint32_t *hist = s + 4 * NOALLOC_MAX_KEYS;
    uint32_t *sums = hist + NOALLOC_HIST;
    int bits = 1;
    while ((1ull << bits) <= (unsigned long long)max_key) ++bits;
    int passes = (bits + 7) / 8;
    int64_t nb = (n + SORT_IPB - 1) / SORT_IPB;
    // every pass overwrites the histogram and the buffers it reads, so nothing
    // in the scratch has to start at zero
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(vbuf[0], n);
    if (int rc = check_launch("pic_sort_keys_noalloc iota")) return rc;
    const uint32_t *kin = keys;
    const uint32_t *vin = vbuf[0];
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        uint32_t *kout = kbuf[p & 1];
        uint32_t *vout = (p == passes - 1) ? perm : vbuf[(p + 1) & 1];
        k_radix_hist<<<(unsigned)nb, SORT_BS, 0, st>>>(kin, n, shift, hist, nb);
        if (int rc = check_launch("pic_sort_keys_noalloc hist")) return rc;
        if (int rc = scan_noalloc(hist, RADIX * nb, sums, st)) return rc;
        k_radix_scatter<<<(unsigned)nb, SORT_BS, 0, st>>>(kin, vin, n, shift, hist, nb, kout, vout);
        if (int rc = check_launch("pic_sort_keys_noalloc scatter")) return rc;
        kin = kout;
        vin = vout;
    }
    return PIC_OK;
}
