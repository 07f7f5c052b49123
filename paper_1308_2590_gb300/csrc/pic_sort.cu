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

template <typename R>
__global__ void k_gather_particles(const uint32_t *__restrict__ perm, int64_t n, const int32_t *__restrict__ c0,
                                   const R *__restrict__ a0, const R *__restrict__ a1, const R *__restrict__ a2,
                                   const R *__restrict__ a3, const R *__restrict__ a4, const R *__restrict__ a5,
                                   int32_t *__restrict__ c1, R *__restrict__ b0, R *__restrict__ b1, R *__restrict__ b2,
                                   R *__restrict__ b3, R *__restrict__ b4, R *__restrict__ b5) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t s = perm[t];
    c1[t] = c0[s];
    b0[t] = a0[s];
    b1[t] = a1[s];
    b2[t] = a2[s];
    b3[t] = a3[s];
    b4[t] = a4[s];
    b5[t] = a5[s];
}

__global__ void k_count_update(int64_t *count, int64_t *dead, int nsp) {
    int s = threadIdx.x;
    if (s < nsp) {
        count[s] -= dead[s];
        dead[s] = 0;
    }
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

int ensure_sort_capacity(pic_t *h, int64_t n) {
    if (n <= h->sort_cap) return 0;
    int64_t cap = n + n / 4 + 4096;
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

template <typename R>
static int gather_t(pic_t *h, int s, int64_t n, const uint32_t *perm) {
    SpeciesBuf &S = h->sp[s];
    int a = S.cur, b = 1 - S.cur;
    k_gather_particles<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(
        perm, n, S.cell[a], (const R *)S.ox[a], (const R *)S.oy[a], (const R *)S.ux[a], (const R *)S.uy[a],
        (const R *)S.uz[a], (const R *)S.w[a], S.cell[b], (R *)S.ox[b], (R *)S.oy[b], (R *)S.ux[b], (R *)S.uy[b],
        (R *)S.uz[b], (R *)S.w[b]);
    count_launch(h);
    S.cur = b;
    return check_launch("k_gather_particles");
}

// Sort keys[0][0..n) stably (values = original index), then regroup the species.
int sort_species(pic_t *h, int s, int64_t n, int max_key) {
    if (n == 0) return 0;
    if (int rc = ensure_sort_capacity(h, n)) return rc;
    int bits = 1;
    while ((1ll << bits) <= (int64_t)max_key) ++bits;
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
    int rc = h->fp32 ? gather_t<float>(h, s, n, h->vals[cur]) : gather_t<double>(h, s, n, h->vals[cur]);
    return rc;
}

int update_counts(pic_t *h) {
    k_count_update<<<1, 32, 0, h->st>>>(h->d_count, h->d_dead, h->nsp);
    count_launch(h);
    return check_launch("k_count_update");
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
