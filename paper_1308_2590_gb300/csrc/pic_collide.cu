// Binary Coulomb collisions (the paper names collisions, with ionisation, as
// what drives its growing particle counts, Sections 4 and 5; it states no
// model).  Reading: the binary collision model of Takizuka and Abe (J. Comput.
// Phys. 25, 205, 1977) applied to u = p/(m c) as the velocity, with the weight
// rule of Nanbu and Yonemura (1998).  A pass runs, for each (species a,
// species b) of its list in turn, over the cells: the particles of a cell are
// consecutive in a species' order (tile, then cell), so a cell is a run of
// indices.  Like particles pair as (0,1), (2,3), ... (odd N >= 3: the first
// three as (0,1), (1,2), (2,0) at half the variance); unlike ones pair the
// driving species' particle i (the species with more particles in the cell, a
// on a tie) with particle i mod N_other of the other.  Pairs of a cell run in
// that order in one thread, each seeing the previous pairs' updates.  Per pair
// (1, 2): g = u1 - u2, mu = m1 m2 / (m1 + m2), n_L = the cell density of the
// species (like) or the lower of the two (sum of w over dx dy), variance
// s2 = q1^2 q2^2 n_L lnL kappa dt / (2 mu^2 |g|^3) (kappa = r_e omega / c),
// delta = sqrt(s2) sqrt(-2 ln(1 - v0)) cos(2 pi v1), phi = 2 pi v2 and the
// rotation of g by the angle 2 atan(delta) about a random axis; u1 moves by
// m2/(m1+m2) dg when v3 < w2 / max(w1, w2), u2 by -m1/(m1+m2) dg when v3 <
// w1 / max(w1, w2).  v0..v3: Philox-4x64-10 at counter (index of the pair's
// first particle in its species' order, 16 + list position, step, 1), key
// (seed, 0).  Momentum and the kinetic energy sum m |u|^2 / 2 are conserved by
// every pair of equal weights.  The pass changes only u; the moments are
// redeposited at rest before they are next used.
#include <math.h>

#include "pic_internal.cuh"
#include "pic_philox.cuh"

namespace pic {

// For every particle of a species, in the species' order: its slot and cell.
// prefix[seg] is the index of the segment's first particle.
__global__ void k_col_index(int64_t nslot, const int32_t *__restrict__ prefix, const int32_t *__restrict__ cell,
                            int32_t *__restrict__ slot_by_index, int32_t *__restrict__ cell_by_index) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslot) return;
    const int64_t seg = slot / SEG;
    const int lane = (int)(slot - seg * SEG);
    const int32_t first = prefix[seg], count = prefix[seg + 1] - first;
    if (lane >= count) return;
    slot_by_index[first + lane] = (int32_t)slot;
    cell_by_index[first + lane] = cell[slot];
}

// 1 where a run of equal cells starts (entry n: 0), to be scanned into run ids.
__global__ void k_col_run_flags(int32_t n, const int32_t *__restrict__ cell_by_index, int32_t *__restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || cell_by_index[i] != cell_by_index[i - 1]) ? 1 : 0;
    else if (i == n) flag[n] = 0;
}

// Run r starts at run_start[r]; run_start[nruns] = n.
__global__ void k_col_run_starts(int32_t n, const int32_t *__restrict__ run_id, const int32_t *__restrict__ cell_by_index,
                                 int32_t *__restrict__ run_start) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (i == 0 || cell_by_index[i] != cell_by_index[i - 1]) run_start[run_id[i]] = (int32_t)i;
    if (i == n - 1) run_start[run_id[n]] = n;
}

// The other species' run of every grid cell (first index, count; count 0 elsewhere).
__global__ void k_col_table(int32_t nruns, const int32_t *__restrict__ run_start, const int32_t *__restrict__ cell_by_index,
                            int32_t *__restrict__ first, int32_t *__restrict__ count) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns) return;
    const int32_t s = run_start[r], c = cell_by_index[s];
    first[c] = s;
    count[c] = run_start[r + 1] - s;
}

template <typename R>
struct ColSpecies {
    const int32_t *slot, *cellix;   // by index in the species' order
    R *ux, *uy, *uz;
    const R *w;
    double q, m;
    int32_t n;
};

template <typename R>
struct ColArgs {
    ColSpecies<R> A, B;
    const int32_t *run_start;       // runs of species a
    int32_t nruns;
    const int32_t *bfirst, *bcount;   // species b's run of each cell (a != b)
    int like;
    double dt, lnL, kappa, inv_area;
    int spec;
    int64_t step;
    uint64_t seed;
    unsigned long long *pairs;
};

// One pair, in FP64 (u1 is driven, its index keys the draws).
__device__ inline void col_scatter(double (&u1)[3], double (&u2)[3], double m1, double m2, double q1, double q2,
                                   double w1, double w2, double nL, double dt, double lnL, double kappa, bool half,
                                   const double (&v)[4]) {
    const double g[3] = {u1[0] - u2[0], u1[1] - u2[1], u1[2] - u2[2]};
    const double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (gm == 0.0 || nL <= 0.0) return;
    const double mu = m1 * m2 / (m1 + m2);
    double s2 = q1 * q1 * q2 * q2 * nL * lnL * kappa * dt / (2.0 * mu * mu * (gm * gm * gm));
    if (half) s2 *= 0.5;
    const double delta = sqrt(s2) * sqrt(-2.0 * log(1.0 - v[0])) * cos(2.0 * M_PI * v[1]);
    const double phi = 2.0 * M_PI * v[2];
    const double sT = 2.0 * delta / (1.0 + delta * delta);
    const double cT1 = 2.0 * delta * delta / (1.0 + delta * delta);
    const double gp = sqrt(g[0] * g[0] + g[1] * g[1]);
    const double cp = cos(phi), sp = sin(phi);
    double dg[3];
    if (gp > 0.0) {
        dg[0] = g[0] / gp * g[2] * sT * cp - g[1] / gp * gm * sT * sp - g[0] * cT1;
        dg[1] = g[1] / gp * g[2] * sT * cp + g[0] / gp * gm * sT * sp - g[1] * cT1;
        dg[2] = -gp * sT * cp - g[2] * cT1;
    } else {
        dg[0] = gm * sT * cp;
        dg[1] = gm * sT * sp;
        dg[2] = -gm * cT1;
    }
    const double wmax = w1 > w2 ? w1 : w2;
    const double f1 = m2 / (m1 + m2), f2 = m1 / (m1 + m2);
    if (v[3] < w2 / wmax)
        for (int c = 0; c < 3; ++c) u1[c] = u1[c] + f1 * dg[c];
    if (v[3] < w1 / wmax)
        for (int c = 0; c < 3; ++c) u2[c] = u2[c] - f2 * dg[c];
}

__device__ inline void col_draws(int64_t index, int spec, int64_t step, uint64_t seed, double (&v)[4]) {
    uint64_t x[4] = {(uint64_t)index, (uint64_t)(16 + spec), (uint64_t)step, 1ull};
    philox4x64_10(x, seed, 0ull);
    for (int k = 0; k < 4; ++k) v[k] = philox_uniform(x[k]);
}

template <typename R>
__device__ inline void col_load(const ColSpecies<R> &S, int32_t i, double (&u)[3]) {
    const int32_t s = S.slot[i];
    u[0] = (double)S.ux[s];
    u[1] = (double)S.uy[s];
    u[2] = (double)S.uz[s];
}

template <typename R>
__device__ inline void col_store(const ColSpecies<R> &S, int32_t i, const double (&u)[3]) {
    const int32_t s = S.slot[i];
    S.ux[s] = (R)u[0];
    S.uy[s] = (R)u[1];
    S.uz[s] = (R)u[2];
}

template <typename R>
__device__ inline void col_pair(const ColArgs<R> &a, const ColSpecies<R> &S1, int32_t i, const ColSpecies<R> &S2,
                                int32_t j, double nL, bool half) {
    double u1[3], u2[3], v[4];
    col_load(S1, i, u1);
    col_load(S2, j, u2);
    col_draws(i, a.spec, a.step, a.seed, v);
    col_scatter(u1, u2, S1.m, S2.m, S1.q, S2.q, (double)S1.w[S1.slot[i]], (double)S2.w[S2.slot[j]], nL, a.dt, a.lnL,
                a.kappa, half, v);
    col_store(S1, i, u1);
    col_store(S2, j, u2);
}

// One thread per cell (run of species a).
template <typename R>
__global__ void k_collide(ColArgs<R> a) {
    const int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.nruns) return;
    const int32_t s = a.run_start[r], e = a.run_start[r + 1], na = e - s;
    double wa = 0.0;
    for (int32_t i = s; i < e; ++i) wa += (double)a.A.w[a.A.slot[i]];
    unsigned long long np = 0;
    if (a.like) {
        if (na >= 2) {
            const double nL = wa * a.inv_area;
            int32_t first = s;
            if (na % 2) {
                col_pair(a, a.A, s, a.A, s + 1, nL, true);
                col_pair(a, a.A, s + 1, a.A, s + 2, nL, true);
                col_pair(a, a.A, s + 2, a.A, s, nL, true);
                first = s + 3;
                np += 3;
            }
            for (int32_t i = first; i < e; i += 2) {
                col_pair(a, a.A, i, a.A, i + 1, nL, false);
                ++np;
            }
        }
    } else {
        const int32_t c = a.A.cellix[s];
        const int32_t sb = a.bfirst[c], nb = a.bcount[c];
        if (nb > 0) {
            double wb = 0.0;
            for (int32_t j = sb; j < sb + nb; ++j) wb += (double)a.B.w[a.B.slot[j]];
            const double nL = (wa < wb ? wa : wb) * a.inv_area;
            if (na >= nb) {
                for (int32_t t = 0; t < na; ++t) col_pair(a, a.A, s + t, a.B, sb + t % nb, nL, false);
                np += na;
            } else {
                for (int32_t t = 0; t < nb; ++t) col_pair(a, a.B, sb + t, a.A, s + t % na, nL, false);
                np += nb;
            }
        }
    }
    if (np) atomicAdd(a.pairs, np);
}

__global__ void k_col_seg_counts(const int32_t *__restrict__ bstart, const int32_t *__restrict__ useg,
                                 const int32_t *__restrict__ segn, int32_t *__restrict__ cnt) {
    const int t = blockIdx.x;
    const int64_t s0 = bstart[t] / SEG, s1 = bstart[t + 1] / SEG;
    const int u = useg[t];
    for (int64_t j = s0 + threadIdx.x; j < s1; j += blockDim.x) cnt[j] = (j - s0 < u) ? segn[j] : 0;
}

// Index maps and cell runs of one species in stream-ordered scratch.
struct ColMaps {
    int32_t *prefix = nullptr, *slot = nullptr, *cellix = nullptr, *runid = nullptr, *run_start = nullptr;
    int32_t n = 0, nruns = 0;
};

static void col_free(pic_t *h, ColMaps &m) {
    void *bufs[] = {m.prefix, m.slot, m.cellix, m.runid, m.run_start};
    for (void *p : bufs)
        if (p) cudaFreeAsync(p, h->st);
    m = ColMaps{};
}

static int col_read_i32(pic_t *h, const int32_t *src, int32_t *out, const char *what) {
    if (cudaMemcpyAsync(out, src, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
        return check_launch(what);
    return 0;
}

static int col_maps(pic_t *h, int s, ColMaps &m) {
    SpeciesBuf &S = h->sp[s];
    if (S.cap == 0) return 0;
    const int64_t nseg = S.cap / SEG;
    if (cudaMallocAsync((void **)&m.prefix, (nseg + 1) * sizeof(int32_t), h->st) != cudaSuccess) {
        cudaGetLastError();
        set_error("pic_collide: scratch allocation failed");
        return PIC_ERR_OOM;
    }
    cudaMemsetAsync(m.prefix, 0, (nseg + 1) * sizeof(int32_t), h->st);
    k_col_seg_counts<<<h->ntiles, 256, 0, h->st>>>(S.bstart, S.useg[S.scur], S.segn[S.scur], m.prefix);
    count_launch(h);
    if (int rc = check_launch("k_col_seg_counts")) return rc;
    if (int rc = scan_i32_inplace(h, m.prefix, nseg + 1)) return rc;
    if (int rc = col_read_i32(h, m.prefix + nseg, &m.n, "collision count")) return rc;
    if (m.n == 0) return 0;
    const size_t nb = (size_t)m.n * sizeof(int32_t), nb1 = ((size_t)m.n + 1) * sizeof(int32_t);
    if (cudaMallocAsync((void **)&m.slot, nb, h->st) != cudaSuccess ||
        cudaMallocAsync((void **)&m.cellix, nb, h->st) != cudaSuccess ||
        cudaMallocAsync((void **)&m.runid, nb1, h->st) != cudaSuccess ||
        cudaMallocAsync((void **)&m.run_start, nb1, h->st) != cudaSuccess) {
        cudaGetLastError();
        set_error("pic_collide: scratch allocation failed");
        return PIC_ERR_OOM;
    }
    k_col_index<<<(unsigned)((S.cap + 255) / 256), 256, 0, h->st>>>(S.cap, m.prefix, S.cell[S.bins], m.slot, m.cellix);
    k_col_run_flags<<<(unsigned)((m.n + 256) / 256), 256, 0, h->st>>>(m.n, m.cellix, m.runid);
    count_launch(h, 2);
    if (int rc = check_launch("collision index maps")) return rc;
    if (int rc = scan_i32_inplace(h, m.runid, (int64_t)m.n + 1)) return rc;
    if (int rc = col_read_i32(h, m.runid + m.n, &m.nruns, "collision runs")) return rc;
    k_col_run_starts<<<(unsigned)((m.n + 255) / 256), 256, 0, h->st>>>(m.n, m.runid, m.cellix, m.run_start);
    count_launch(h);
    return check_launch("k_col_run_starts");
}

template <typename R>
static ColSpecies<R> col_species(pic_t *h, int s, const ColMaps &m) {
    SpeciesBuf &S = h->sp[s];
    ColSpecies<R> c;
    const int b = S.bins;
    c.slot = m.slot;
    c.cellix = m.cellix;
    c.ux = (R *)S.ux[b];
    c.uy = (R *)S.uy[b];
    c.uz = (R *)S.uz[b];
    c.w = (const R *)S.w[b];
    c.q = S.q;
    c.m = S.m;
    c.n = m.n;
    return c;
}

template <typename R>
static int collide_t(pic_t *h, const pic_collisions *p, unsigned long long *d_pairs) {
    for (int k = 0; k < p->n_pairs; ++k) {
        const int sa = p->a[k], sb = p->b[k];
        ColMaps ma, mb;
        int rc = col_maps(h, sa, ma);
        if (!rc && sb != sa) rc = col_maps(h, sb, mb);
        int32_t *first = nullptr, *count = nullptr;
        const int64_t ncell = (int64_t)h->nx * h->ny;
        if (!rc && sb != sa && ma.n > 0 && mb.n > 0) {
            if (cudaMallocAsync((void **)&first, ncell * sizeof(int32_t), h->st) != cudaSuccess ||
                cudaMallocAsync((void **)&count, ncell * sizeof(int32_t), h->st) != cudaSuccess) {
                cudaGetLastError();
                set_error("pic_collide: scratch allocation failed");
                rc = PIC_ERR_OOM;
            } else {
                cudaMemsetAsync(count, 0, ncell * sizeof(int32_t), h->st);
                k_col_table<<<(unsigned)((mb.nruns + 255) / 256), 256, 0, h->st>>>(mb.nruns, mb.run_start, mb.cellix,
                                                                                   first, count);
                count_launch(h);
                rc = check_launch("k_col_table");
            }
        }
        if (!rc && ma.n > 0 && (sb == sa || mb.n > 0)) {
            ColArgs<R> a;
            a.A = col_species<R>(h, sa, ma);
            a.B = (sb == sa) ? a.A : col_species<R>(h, sb, mb);
            a.run_start = ma.run_start;
            a.nruns = ma.nruns;
            a.bfirst = first;
            a.bcount = count;
            a.like = (sb == sa) ? 1 : 0;
            a.dt = h->cfg.dt;
            a.lnL = p->ln_lambda;
            a.kappa = p->kappa;
            a.inv_area = 1.0 / (h->cfg.dx * h->cfg.dy);
            a.spec = k;
            a.step = h->step;
            a.seed = p->seed;
            a.pairs = d_pairs;
            k_collide<R><<<(unsigned)((ma.nruns + 127) / 128), 128, 0, h->st>>>(a);
            count_launch(h);
            rc = check_launch("k_collide");
        }
        if (first) cudaFreeAsync(first, h->st);
        if (count) cudaFreeAsync(count, h->st);
        col_free(h, ma);
        col_free(h, mb);
        if (rc) return rc;
    }
    return 0;
}

int collide(pic_t *h, const pic_collisions *p, unsigned long long *d_pairs) {
    return h->fp32 ? collide_t<float>(h, p, d_pairs) : collide_t<double>(h, p, d_pairs);
}

}  // namespace pic
