// Optical field ionisation (the paper's targets ionise as the laser arrives,
// Section 4 and Fig. 3; the paper states no rate).  Reading: the static
// tunnelling rate of Ammosov, Delone and Krainov for s-states, held at its
// maximum above the field of that maximum,
//   w = |C|^2 Ip (K / F')^(2 n* - 1) exp(-K / (3 F')),  K = 2 (2 Ip)^(3/2),
//   n* = Z / sqrt(2 Ip), |C|^2 = 2^(2 n*) / (n* Gamma(2 n*)), F' = min(F, F_m),
// in atomic units; the probability of a transition in a step is
// P = 1 - exp(-w dt), at most one per particle and pass.  The uniform number
// of a particle is the first output of Philox-4x64-10 (Salmon, Moraes, Dror
// and Shaw, SC 2011) at counter (its index in the species' order, species,
// step, 0) and key (seed, 0), taken as (out >> 11) 2^-53.
//
// A pass, per chain (ion species -> next charge state + electron): every
// particle's index from a scan of the segment counts, the decision, a scan of
// the decisions (the staging order is the species' order), the ionised
// particles written in the checkpoint form (cell, offsets, u, w) to a staging
// buffer, and the species' segments compacted in place.  The host then appends
// the staged particles to the target and electron species with one load
// (pic_api.cu), which re-orders them as any load does and redeposits.
#include <math.h>

#include "pic_internal.cuh"
#include "pic_philox.cuh"

namespace pic {

// Counts of the species' segments, in slot order (0 for the unused segments of
// a bin); one block per tile.
__global__ void k_ion_seg_counts(const int32_t *__restrict__ bstart, const int32_t *__restrict__ useg,
                                 const int32_t *__restrict__ segn, int32_t *__restrict__ cnt) {
    const int t = blockIdx.x;
    const int64_t s0 = bstart[t] / SEG, s1 = bstart[t + 1] / SEG;
    const int u = useg[t];
    for (int64_t j = s0 + threadIdx.x; j < s1; j += blockDim.x) cnt[j] = (j - s0 < u) ? segn[j] : 0;
}

// One thread per slot: the decision of the particle in that slot.  prefix[seg]
// is the index of the segment's first particle in the species' order.
template <typename R>
__global__ void k_ion_mark(GridArgs<R> g, int64_t nslot, const int32_t *__restrict__ prefix,
                           const int32_t *__restrict__ cell, const R *__restrict__ ox, const R *__restrict__ oy,
                           const V4<R> *__restrict__ E, IonChain c, int64_t step, uint64_t seed,
                           int32_t *__restrict__ flag_by_index, int32_t *__restrict__ slot_by_index,
                           int32_t *__restrict__ removed) {
    const int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= nslot) return;
    const int64_t seg = slot / SEG;
    const int lane = (int)(slot - seg * SEG);
    const int32_t first = prefix[seg], count = prefix[seg + 1] - first;
    if (lane >= count) {
        removed[slot] = 0;
        return;
    }
    const int32_t idx = first + lane;
    const int32_t cc = cell[slot];
    const int cx = cc % g.nx, cy = cc / g.nx;
    const double fx = (double)ox[slot], fy = (double)oy[slot];
    const double w00 = (1.0 - fx) * (1.0 - fy), w10 = fx * (1.0 - fy), w01 = (1.0 - fx) * fy, w11 = fx * fy;
    const V4<R> a = E[node_of(g, cx, cy, 0, 0)], b = E[node_of(g, cx, cy, 1, 0)];
    const V4<R> d = E[node_of(g, cx, cy, 0, 1)], e = E[node_of(g, cx, cy, 1, 1)];
    const double Ex = w00 * (double)a.x + w10 * (double)b.x + w01 * (double)d.x + w11 * (double)e.x;
    const double Ey = w00 * (double)a.y + w10 * (double)b.y + w01 * (double)d.y + w11 * (double)e.y;
    const double Ez = w00 * (double)a.z + w10 * (double)b.z + w01 * (double)d.z + w11 * (double)e.z;
    const double F = sqrt(Ex * Ex + Ey * Ey + Ez * Ez) * c.field_au;
    double prob = 0.0;
    if (F > 0.0) {
        const double Fp = F < c.fmax ? F : c.fmax;
        const double w = c.c2ip * pow(c.K / Fp, c.expo) * exp(-c.K / (3.0 * Fp));
        prob = -expm1(-w * c.dt_au);
    }
    uint64_t x[4] = {(uint64_t)idx, (uint64_t)c.species, (uint64_t)step, 0ull};
    philox4x64_10(x, seed, 0ull);
    const double u = (double)(x[0] >> 11) * 0x1.0p-53;
    const int32_t f = (u < prob) ? 1 : 0;
    flag_by_index[idx] = f;
    slot_by_index[idx] = (int32_t)slot;
    removed[slot] = f;
}

// The ionised particles, in the species' order, to the staging buffer in the
// checkpoint form: cells, then offsets x and y, u (3) and w as FP64 planes.
template <typename R>
__global__ void k_ion_stage(int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ slot_by_index,
                            const int32_t *__restrict__ removed, const int32_t *__restrict__ cell,
                            const R *__restrict__ ox, const R *__restrict__ oy, const R *__restrict__ ux,
                            const R *__restrict__ uy, const R *__restrict__ uz, const R *__restrict__ w,
                            int32_t *__restrict__ scell, double *__restrict__ sval, int64_t cap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t slot = slot_by_index[i];
    if (!removed[slot]) return;
    const int64_t p = pos[i];
    scell[p] = cell[slot];
    sval[p] = (double)ox[slot];
    sval[cap + p] = (double)oy[slot];
    sval[2 * cap + p] = (double)ux[slot];
    sval[3 * cap + p] = (double)uy[slot];
    sval[4 * cap + p] = (double)uz[slot];
    sval[5 * cap + p] = (double)w[slot];
}

// The species' segments without the ionised particles: each warp compacts one
// segment in place (every lane reads before any lane writes), keeping order.
template <typename R>
__global__ void k_ion_compact(const int32_t *__restrict__ bstart, const int32_t *__restrict__ useg,
                              int32_t *__restrict__ segn, const int32_t *__restrict__ removed, int32_t *cell, R *ox,
                              R *oy, R *ux, R *uy, R *uz, R *w) {
    const int t = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t b0 = bstart[t];
    const int u = useg[t];
    for (int j = wid; j < u; j += nw) {
        const int64_t sg = b0 / SEG + j, slot = b0 + (int64_t)j * SEG + lane;
        const int n = segn[sg];
        const bool keep = lane < n && !removed[slot];
        int32_t c = 0;
        R a = R(0), b = R(0), d = R(0), e = R(0), f = R(0), h = R(0);
        if (keep) {
            c = cell[slot];
            a = ox[slot]; b = oy[slot]; d = ux[slot]; e = uy[slot]; f = uz[slot]; h = w[slot];
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        __syncwarp();
        if (keep) {
            const int64_t dst = b0 + (int64_t)j * SEG + __popc(m & ((1u << lane) - 1u));
            cell[dst] = c;
            ox[dst] = a; oy[dst] = b; ux[dst] = d; uy[dst] = e; uz[dst] = f; w[dst] = h;
        }
        if (lane == 0) segn[sg] = __popc(m);
    }
}

static int ion_chain_t_launch_check(const char *what) { return check_launch(what); }

template <typename R>
static int ion_chain_t(pic_t *h, const IonChain &c, uint64_t seed, int32_t *scell, double *sval, int64_t scap,
                       int64_t offset, int64_t *n_out) {
    SpeciesBuf &S = h->sp[c.species];
    *n_out = 0;
    if (S.cap == 0) return 0;
    const int64_t nseg = S.cap / SEG;
    int32_t *prefix = (int32_t *)h->keys[1];     // nseg + 1 entries (sort scratch: 2 cap entries)
    int32_t *flag = (int32_t *)h->keys[0];       // per index, then its exclusive scan
    int32_t *slot_by_index = (int32_t *)h->vals[0];
    int32_t *removed = (int32_t *)h->vals[1];    // per slot
    cudaMemsetAsync(prefix, 0, (nseg + 1) * sizeof(int32_t), h->st);
    k_ion_seg_counts<<<h->ntiles, 256, 0, h->st>>>(S.bstart, S.useg[S.scur], S.segn[S.scur], prefix);
    count_launch(h);
    if (int rc = ion_chain_t_launch_check("k_ion_seg_counts")) return rc;
    if (int rc = scan_i32_inplace(h, prefix, nseg + 1)) return rc;
    int32_t n = 0;
    if (cudaMemcpyAsync(&n, prefix + nseg, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
        return ion_chain_t_launch_check("ionisation count");
    if (n == 0) return 0;
    GridArgs<R> g = grid_args<R>(h);
    const int b = S.bins;
    k_ion_mark<R><<<(unsigned)((S.cap + 255) / 256), 256, 0, h->st>>>(
        g, S.cap, prefix, S.cell[b], (const R *)S.ox[b], (const R *)S.oy[b], (const V4<R> *)h->E[h->ecur], c, h->step,
        seed, flag, slot_by_index, removed);
    count_launch(h);
    if (int rc = ion_chain_t_launch_check("k_ion_mark")) return rc;
    cudaMemsetAsync(flag + n, 0, sizeof(int32_t), h->st);
    if (int rc = scan_i32_inplace(h, flag, (int64_t)n + 1)) return rc;
    int32_t k = 0;
    if (cudaMemcpyAsync(&k, flag + n, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st) != cudaSuccess ||
        cudaStreamSynchronize(h->st) != cudaSuccess)
        return ion_chain_t_launch_check("ionisation decisions");
    if (k == 0) return 0;
    if (offset + k > scap) {
        set_error("pic_ionize: staging capacity exceeded");
        return PIC_ERR_STATE;
    }
    k_ion_stage<R><<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(
        n, flag, slot_by_index, removed, S.cell[b], (const R *)S.ox[b], (const R *)S.oy[b], (const R *)S.ux[b],
        (const R *)S.uy[b], (const R *)S.uz[b], (const R *)S.w[b], scell + offset, sval + offset, scap);
    count_launch(h);
    if (int rc = ion_chain_t_launch_check("k_ion_stage")) return rc;
    k_ion_compact<R><<<h->ntiles, 256, 0, h->st>>>(S.bstart, S.useg[S.scur], S.segn[S.scur], removed, S.cell[b],
                                                   (R *)S.ox[b], (R *)S.oy[b], (R *)S.ux[b], (R *)S.uy[b],
                                                   (R *)S.uz[b], (R *)S.w[b]);
    count_launch(h);
    if (int rc = ion_chain_t_launch_check("k_ion_compact")) return rc;
    *n_out = k;
    return 0;
}

int ion_chain(pic_t *h, const IonChain &c, uint64_t seed, int32_t *scell, double *sval, int64_t scap, int64_t offset,
              int64_t *n_out) {
    return h->fp32 ? ion_chain_t<float>(h, c, seed, scell, sval, scap, offset, n_out)
                   : ion_chain_t<double>(h, c, seed, scell, sval, scap, offset, n_out);
}

}  // namespace pic
